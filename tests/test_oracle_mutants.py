"""Each plausible mistake planted in a copy of the C oracle must be caught by
at least one pin: evidence that the pins constrain every term of Eq. (7), the
visibility rule, the source layout and the grazing flags, and likewise the
area-mean closed form (solid angles, area normalisation, vertex checks,
fallback), the visibility-cube estimator (pixel solid angles and powers,
nearest hit, front faces, pixel centres) and the CPU hierarchy (child boxes,
box padding, slab clipping, leaf loops), whose results must then differ from
the brute force.  Runs on the CPU."""
import inspect
import os
import subprocess

import pytest

import oracle
from tests import _pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "uvc_oracle.c")

MUTANTS = {
    "no_cosine": ("power * nv_ / (four_pi * d * d * d)", "power / (four_pi * d * d)"),
    "inverse_square_of_d_only": ("(four_pi * d * d * d)", "(four_pi * d * d)"),
    "two_pi": ("const double four_pi = 4.0 * M_PI;", "const double four_pi = 2.0 * M_PI;"),
    "ignore_source_weights": ("(double)weights[m] * power", "power"),
    "facing_sign_flipped": ("if (nv_ > 0.0 && d > 0.0) {", "if (nv_ < 0.0 && d > 0.0) {"),
    "no_exclusion": ("if (t == ex0 || t == ex1) continue;\n                            if (segment_meets_triangle",
                     "if (segment_meets_triangle"),
    "ray_not_segment": ("return tau > 0.0 && tau < 1.0;", "return tau > 0.0;"),
    "closed_segment": ("return tau > 0.0 && tau < 1.0;", "return tau >= 0.0 && tau <= 1.0;"),
    "source_in_fp64": ("float ox = cand[3 * i] + offsets[3 * m];",
                       "double ox = (double)cand[3 * i] + (double)offsets[3 * m] + 1e-9;"),
    "barycentric_bound": ("if (w < 0.0 || u + w > 1.0) return 0;", "if (w < 0.0 || u + w > 1.5) return 0;"),
    "edge_flag_lost": ("        bits |= 1;", "        bits |= 0;"),
    "facing_flag_lost": ("flags |= 4;", "flags |= 0;"),
    "endpoint_flag_lost": ("        bits |= 2;", "        bits |= 0;"),
}


def _mutant_lib(old, new, tmp_path, unique=False):
    """A copy of the C oracle with `old` replaced by `new` (first occurrence),
    compiled and loaded."""
    src = open(SRC).read()
    if unique:
        assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    else:
        assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    mutated = tmp_path / "mut.c"
    mutated.write_text(src.replace(old, new, 1))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                           str(mutated), "-o", str(so), "-lm"])
    return oracle.load_library(str(so))


def _calls(fn):
    """The argument tuples a pin runs with: () for a plain test, each value of
    a one-name parametrize mark; pins taking fixtures are left out."""
    params = inspect.signature(fn).parameters
    if not params:
        return [()]
    marks = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
    if len(marks) == 1 and len(params) == 1 and marks[0].args[0] == next(iter(params)):
        return [(v,) for v in marks[0].args[1]]
    return []


def _caught_by(pins_module):
    caught = []
    for name in sorted(n for n in dir(pins_module) if n.startswith("test_")):
        fn = getattr(pins_module, name)
        for args in _calls(fn):
            try:
                fn(*args)
            except AssertionError:
                caught.append(name)
                break
    return caught


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    lib = _mutant_lib(*MUTANTS[name], tmp_path)

    def irr(*a, **kw):
        return oracle.irradiance(*a, lib=lib, **kw)

    caught = []
    for pin in _pins.ALL_PINS:
        try:
            pin(irr)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"mutant {name} passed every pin"


# Mistakes in the area-mean oracle (uvco_area_mean), each of which one of the
# area-mean pins (tests/test_oracle_area_mean.py) must catch.
AREA_MUTANTS = {
    "solid_angle_halved": ("return 2.0 * atan2(num, den);", "return atan2(num, den);"),
    "solid_angle_den_sign": ("+ vdot(R2, R3) * r1;", "- vdot(R2, R3) * r1;"),
    "area_not_divided": ("E += pw * om / (four_pi * (double)area[j]);", "E += pw * om / four_pi;"),
    "second_triangle_dropped": ("for (int t = 0; t < ntri; ++t) om += solid_angle",
                                "for (int t = 0; t < 1; ++t) om += solid_angle"),
    "vertex_checks_skipped": ("if (all && !seg_visible(T, nt, B, stack, ex0, ex1, o, chk[q])) all = 0;", ";"),
    "closed_form_unweighted": ("double pw = (double)weights[m] * power;", "double pw = power;"),
    "fallback_without_cosine": ("E += pw * nv_ / (four_pi * d * d * d);", "E += pw / (four_pi * d * d);"),
}


@pytest.mark.parametrize("name", sorted(AREA_MUTANTS))
def test_area_mean_mutant_is_caught(name, tmp_path, monkeypatch):
    from tests import test_oracle_area_mean as pins
    monkeypatch.setattr(oracle, "_lib", _mutant_lib(*AREA_MUTANTS[name], tmp_path, unique=True))
    assert _caught_by(pins), f"mutant {name} passed every area-mean pin"


# Mistakes in the visibility-cube oracle (uvco_raster), each of which one of
# the raster pins (tests/test_oracle_raster.py) must catch.
RASTER_MUTANTS = {
    "pixel_power_without_4pi": ("double pw = (double)weights[m] * power / (4.0 * M_PI);",
                                "double pw = (double)weights[m] * power;"),
    "pixel_solid_angle_sign": ("pixel_G(u1, v1) - pixel_G(u0, v1) - pixel_G(u1, v0) + pixel_G(u0, v0)",
                               "pixel_G(u1, v1) - pixel_G(u0, v1) + pixel_G(u1, v0) + pixel_G(u0, v0)"),
    "farthest_hit_wins": ("if (inside && tt < tbest)", "if (inside && (best < 0 || tt > tbest))"),
    "back_faces_receive": ("if (dn < 0.0) {", "if (dn != 0.0) {"),
    "ray_through_pixel_corner": ("float uf = (float)(2 * px + 1) / (float)R - 1.0f;",
                                 "float uf = (float)(2 * px) / (float)R - 1.0f;"),
    "barycentric_bound": ("int inside = uu >= 0.0 && ww >= 0.0 && uu + ww <= 1.0;",
                          "int inside = uu >= 0.0 && ww >= 0.0 && uu + ww <= 1.5;"),
    "edge_on_receivers_skipped": ("    if (det == 0.0) {\n        d3 q = vadd(o, vmul(dir, tmax));",
                                  "    if (det == 0.0) {\n        return 0;\n        d3 q = vadd(o, vmul(dir, tmax));"),
}


@pytest.mark.parametrize("name", sorted(RASTER_MUTANTS))
def test_raster_mutant_is_caught(name, tmp_path, monkeypatch):
    from tests import test_oracle_raster as pins
    monkeypatch.setattr(oracle, "_lib", _mutant_lib(*RASTER_MUTANTS[name], tmp_path, unique=True))
    assert _caught_by(pins), f"mutant {name} passed every raster pin"


# Mistakes in the oracle's CPU hierarchy (bvh_build, the box tests, the
# hierarchical visibility and grazing searches), each of which must make its
# results differ from the brute force somewhere in tests/test_oracle_bvh.py.
BVH_MUTANTS = {
    "right_box_misses_its_last_triangle": ("box_of(T, B->order, R->first, R->count, R->lo, R->hi);",
                                           "box_of(T, B->order, R->first, R->count - 1, R->lo, R->hi);"),
    "boxes_shrunk_for_visibility": ("const double pad = 1e-9 * B->diag + 1e-300;",
                                    "const double pad = -1e-3 * B->diag;"),
    "grazing_boxes_without_the_band": ("const double pad = eps + 1e-9 * B->diag + 1e-300;",
                                       "const double pad = -1e-3 * B->diag;"),
    "slab_exit_from_the_entry": ("if (tb < t1) t1 = tb;", "if (tb < t1) t1 = ta;"),
    "visibility_leaf_skips_its_last": (
        "for (int64_t q = nd->first; q < nd->first + nd->count; ++q) {\n"
        "                const int64_t t = B->order[q];\n"
        "                if (t == ex0 || t == ex1) continue;\n"
        "                if (segment_meets_triangle",
        "for (int64_t q = nd->first; q < nd->first + nd->count - 1; ++q) {\n"
        "                const int64_t t = B->order[q];\n"
        "                if (t == ex0 || t == ex1) continue;\n"
        "                if (segment_meets_triangle"),
}


@pytest.mark.parametrize("name", sorted(BVH_MUTANTS))
def test_bvh_mutant_is_caught(name, tmp_path, monkeypatch):
    from tests import test_oracle_bvh as pins
    monkeypatch.setattr(oracle, "_lib", _mutant_lib(*BVH_MUTANTS[name], tmp_path, unique=True))
    assert _caught_by(pins), f"mutant {name} passed every hierarchy pin"
