"""The error bound of the tensor-core fluence (k_fluence_tc), derived and
replayed on the CPU.  The kernel splits every value of A and t as
x = hi + lo with hi = tf32(x) and lo = tf32(x - hi) (cvt.rna: round to 10
fraction bits, ties away from zero), lets the tensor core add the four
products hi*hi + hi*lo + lo*hi + lo*lo of 32 candidate rows into an FP32
accumulator that starts from zero (128 products per stage, in an order the
hardware chooses), and adds the stage sums with Kahan compensation.  For
non-negative terms the relative error of mu is then at most

    split:  |a t - (a_hi + a_lo)(t_hi + t_lo)| <= (2 * 2^-22 + 2^-44) a t
    stage:  128 FP32 additions of non-negative terms, any order: 128 u
    stages: Kahan-compensated sum and the final subtraction: 3 u

with u = 2^-24, about 8.3e-6, below the 1e-5 the parity tests use.  The stage
term assumes the tensor core rounds each of its FP32 additions to nearest;
its internal accumulation is not specified, and one that truncated would
double that term (the GPU tests measure 2.4e-7 on the ward's shape and stay
within 1e-5 element by element on inputs spanning six decades).  These tests
check the pieces the bound rests on (the split's residual, exact TF32
products) and replay the kernel's arithmetic with the stage sums accumulated
in two orders (ascending and descending terms) on adversarial columns."""
import numpy as np
import pytest

U = 2.0 ** -24
ROWS = 32                      # candidate rows per stage
PRODUCTS = 4 * ROWS            # products one stage accumulator takes
BOUND = (2 * 2.0 ** -22 + 2.0 ** -44) + PRODUCTS * U + 3 * U
MU_TOL = 1e-5


def tf32_rna(x):
    """Round binary32 values to 10 fraction bits, ties away from zero (the
    cvt.rna.tf32.f32 rounding): add half a unit of the kept bits to the
    magnitude and drop the 13 low bits (a carry into the exponent is the
    correct rounding up)."""
    b = np.asarray(x, np.float32).view(np.uint32)
    sign = b & np.uint32(0x80000000)
    mag = b & np.uint32(0x7FFFFFFF)
    r = ((mag + np.uint32(0x1000)) & np.uint32(0xFFFFE000)) | sign
    return r.view(np.float32)


def split(x):
    x = np.asarray(x, np.float32)
    hi = tf32_rna(x)
    lo = tf32_rna((x - hi).astype(np.float32))
    return hi, lo


def test_rounding_is_to_nearest_ties_away():
    one = np.float32(1.0)
    ulp = np.float32(2.0 ** -10)           # TF32 unit at 1
    cases = np.array([one + ulp / 2, one + ulp / 4, one + 3 * ulp / 4, -(one + ulp / 2), np.float32(3.0)],
                     np.float32)
    want = np.array([one + ulp, one, one + ulp, -(one + ulp), np.float32(3.0)], np.float32)
    assert np.array_equal(tf32_rna(cases), want)
    r = tf32_rna(np.random.default_rng(0).uniform(-1e3, 1e3, 10000).astype(np.float32))
    assert np.all((r.view(np.uint32) & np.uint32(0x1FFF)) == 0)          # 10 fraction bits left


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_split_residual_and_exact_products(seed):
    rng = np.random.default_rng(seed)
    x = np.exp(rng.uniform(np.log(1e-6), np.log(1e4), 200000)).astype(np.float32)
    hi, lo = split(x)
    x64, hi64, lo64 = (v.astype(np.float64) for v in (x, hi, lo))
    assert np.all(np.abs(x64 - hi64 - lo64) <= 2.0 ** -22 * x64)         # the split's residual
    assert np.all(x - hi == (x64 - hi64))                                  # x - hi exact in FP32
    y = np.exp(rng.uniform(np.log(1e-3), np.log(60.0), x.size)).astype(np.float32)
    yh, yl = split(y)
    for p, q in ((hi, yh), (hi, yl), (lo, yh), (lo, yl)):
        prod32 = (p * q).astype(np.float32)
        assert np.array_equal(prod32.astype(np.float64), p.astype(np.float64) * q.astype(np.float64))


def kernel_arithmetic(a, t, descending=False):
    """mu = sum_i t[i] a[i] as k_fluence_tc computes it, one column: per stage
    of 32 rows the 128 products (exact in FP32) added in FP32 in the given
    order, then the stage sums Kahan-compensated, the result acc - comp."""
    ah, al = split(a)
    th, tl = split(t)
    acc, comp = np.float32(0), np.float32(0)
    for s0 in range(0, a.size, ROWS):
        sl = slice(s0, s0 + ROWS)
        terms = np.concatenate([ah[sl] * th[sl], ah[sl] * tl[sl], al[sl] * th[sl], al[sl] * tl[sl]])
        terms = np.sort(terms.astype(np.float32))
        if descending:
            terms = terms[::-1]
        st = np.float32(0)
        for v in terms:
            st = np.float32(st + v)
        y = np.float32(st - comp)
        tt = np.float32(acc + y)
        comp = np.float32(np.float32(tt - acc) - y)
        acc = tt
    return np.float32(acc - comp)


def test_bound_is_below_the_parity_tolerance():
    assert BOUND < MU_TOL
    assert BOUND == pytest.approx(8.3e-6, rel=0.01)


@pytest.mark.parametrize("kind", ["uniform", "decades", "one_dominant", "long"])
def test_replay_within_the_bound(kind):
    rng = np.random.default_rng({"uniform": 5, "decades": 6, "one_dominant": 7, "long": 8}[kind])
    n = 10000 if kind == "long" else 2000
    if kind == "uniform":
        a = rng.uniform(0, 10, n)
    elif kind == "decades":
        a = np.exp(rng.uniform(np.log(1e-4), np.log(1e2), n))
    elif kind == "one_dominant":
        a = rng.uniform(0, 1e-3, n)
        a[n // 2] = 1e3
    else:
        a = rng.uniform(0, 1, n)
    a = a.astype(np.float32)
    a[rng.uniform(size=n) < 0.3] = 0
    t = rng.uniform(0, 60, n).astype(np.float32)
    exact = float(np.dot(a.astype(np.float64), t.astype(np.float64)))
    for desc in (False, True):
        got = float(kernel_arithmetic(a, t, desc))
        assert abs(got - exact) <= BOUND * exact, (kind, desc, abs(got - exact) / exact)
