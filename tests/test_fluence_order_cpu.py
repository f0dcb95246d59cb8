"""The summation order of the fluence kernel (k_fluence), replayed in FP32 on
the CPU, stays within the error bound the parity tolerance is derived from:
each thread sums blocks of 32 candidate rows with fused multiply-adds, adds
the block sums with Kahan compensation, and the four row groups of a block
are added in a fixed order with compensation again, so for non-negative terms
the relative error is at most about (32 + 2 + 2) units of 2^-24, whatever the
number of candidates (the plain running sum would grow with it)."""
import math

import numpy as np
import pytest

U = 2.0 ** -24
GROUPS, CHUNK, BLOCK = 4, 128, 32


def _fma32(a, b, c):
    """fl32(a * b + c) rounded once, as a fused multiply-add does.

    The product of two binary32 numbers is exact in binary64; the binary64 sum
    s = fl64(p + c) carries an error e (p + c = s + e exactly, TwoSum).  Since
    |e| is below half a binary64 unit of s, rounding s to binary32 gives the
    correctly rounded p + c except when s lies exactly halfway between two
    binary32 numbers: then the sign of e decides (rounding s alone would
    round twice)."""
    p = a.astype(np.float64) * b.astype(np.float64)
    c64 = c.astype(np.float64)
    s = p + c64
    z = s - p
    e = (p - (s - z)) + (c64 - z)
    r = s.astype(np.float32)
    r64 = r.astype(np.float64)
    up = np.nextafter(r, np.float32(np.inf))
    dn = np.nextafter(r, np.float32(-np.inf))
    # s halfway between r and a neighbour (nearest-even chose r): the exact
    # value lies on e's side of the midpoint, so it rounds to the neighbour
    # when e points away from r
    tie_up = (s > r64) & (s - r64 == up.astype(np.float64) - s) & (e > 0)
    tie_dn = (s < r64) & (r64 - s == s - dn.astype(np.float64)) & (e < 0)
    return np.where(tie_up, up, np.where(tie_dn, dn, r))


def _kahan(s, c, x):
    y = (x - c).astype(np.float32)
    t = (s + y).astype(np.float32)
    c = ((t - s).astype(np.float32) - y).astype(np.float32)
    return t, c


def kernel_order(A, t):
    """mu[j] = sum_i t[i] A[i, j] in the kernel's order, FP32 throughout."""
    nc, ncol = A.shape
    per = ((-(-nc // GROUPS)) + BLOCK - 1) // BLOCK * BLOCK
    z = np.zeros(ncol, np.float32)
    groups = []
    for g in range(GROUPS):
        r0, r1 = min(nc, g * per), min(nc, g * per + per)
        part, acc, comp = z.copy(), z.copy(), z.copy()
        for c0 in range(r0, r1, CHUNK):
            c1 = min(r1, c0 + CHUNK)
            for i in range(c0, c1):
                part = _fma32(np.full(ncol, t[i], np.float32), A[i], part)
                q = i - c0 + 1
                if q % BLOCK == 0 or i == c1 - 1:
                    acc, comp = _kahan(acc, comp, part)
                    part = z.copy()
        groups.append((acc - comp).astype(np.float32))
    s, c = z.copy(), z.copy()
    for x in groups:
        s, c = _kahan(s, c, x)
    return s


def _exact(A, t):
    return np.array([math.fsum(float(t[i]) * float(A[i, j]) for i in range(A.shape[0]))
                     for j in range(A.shape[1])])


@pytest.mark.parametrize("nc", [1, 31, 33, 500, 2000, 10000])
@pytest.mark.parametrize("kind", ["uniform", "decreasing", "one_large"])
def test_kernel_order_meets_its_bound(nc, kind):
    rng = np.random.default_rng(nc)
    ncol = 16
    if kind == "uniform":
        A = rng.uniform(0, 10, (nc, ncol))
    elif kind == "decreasing":
        A = np.exp(-np.linspace(0, 25, nc))[:, None] * rng.uniform(0.5, 1.5, (nc, ncol))
    else:
        A = rng.uniform(0, 1e-3, (nc, ncol))
        A[nc // 2] = 1e3
    A = A.astype(np.float32)
    t = rng.uniform(0, 60, nc).astype(np.float32)
    got = kernel_order(A, t).astype(np.float64)
    want = _exact(A, t)
    rel = np.abs(got - want) / np.maximum(want, 1e-300)
    assert rel.max() <= 40 * U, rel.max()


def test_plain_running_sum_would_not():
    """The bound is a property of the blocking: one running FP32 sum over
    10,000 equal-sized terms drifts well past it."""
    nc = 10000
    A = np.full((nc, 1), 0.1, np.float32)
    t = np.full(nc, 1.1, np.float32)
    s = np.float32(0)
    for i in range(nc):
        s = np.float32(s + np.float32(t[i] * A[i, 0]))
    want = _exact(A, t)[0]
    assert abs(float(s) - want) / want > 40 * U
    assert abs(float(kernel_order(A, t)[0]) - want) / want <= 40 * U


def test_fma_emulation_rounds_once():
    """A case where rounding a*b + c first to binary64 and then to binary32
    lands on the wrong neighbour: a*b = 2^-4 - 2^-40 exactly, c = 2^20 + 2^-3;
    the binary64 sum is the binary32 midpoint 2^20 + 2^-3 + 2^-4, the exact
    value lies just below it, so a fused multiply-add gives 2^20 + 2^-3."""
    a = np.array([(1 + 2.0 ** -18) * 0.25], np.float32)
    b = np.array([(1 - 2.0 ** -18) * 0.25], np.float32)
    c = np.array([2.0 ** 20 + 2.0 ** -3], np.float32)
    assert float(a[0]) * float(b[0]) == 2.0 ** -4 - 2.0 ** -40
    twice = (a.astype(np.float64) * b + c.astype(np.float64)).astype(np.float32)
    assert twice[0] == np.float32(2.0 ** 20 + 2.0 ** -2)
    assert _fma32(a, b, c)[0] == c[0]
    assert _fma32(-a, b, -c)[0] == -c[0]
