"""Pins against the numbers the paper prints (fixtures in tests/golden/,
each with its citation); CPU only.

* The synthetic inputs of the paper-shaped sweep (synth.py) carry the
  printed level table (Sec. 3.2.1), 1D model (Sec. 3.1.2) and moment tensor
  (Eq. 7) unchanged.
* The time-step rule of Eq. 5 (ews_cfl_dt in libews) admits every time step
  the paper ran, and so does the exact stability bound of the scheme that
  the solver enforces (reading R10, closed form written out here).
* The printed tables agree with each other in two ways that fix readings:
  every grid spacing is the domain size of Sec. 3.2 divided by the cell
  count, truncated to the printed digits; every "max f" is Eq. 6 (as
  ews_max_freq computes it, with the model's smallest S speed) divided by
  sqrt(2), truncated likewise (reading R11).
* Every S speed of the model table is its P speed / 1.74 rounded to the
  printed digits (a transcription check of the model table).
"""
import math
import os

import numpy as np
import pytest

from paper_2112_15071_gb300 import ews, synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rows(name):
    out = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append(line.split())
    return out


def levels():
    r = rows("paper_levels.txt")
    size = tuple(float(v) for v in r[0][1:4])
    assert r[0][0] == "size"
    lv = []
    for t in r[1:]:
        lv.append({"level": int(t[0]), "n": tuple(int(v) for v in t[1:4]), "steps": int(t[4]),
                   "dp_km": tuple(float(v) for v in t[5:8]), "dt": float(t[8]),
                   "fmax": float(t[9]), "fmax_digits": len(t[9].split(".")[1])})
    return size, lv


def medium():
    return np.array([[float(v) for v in t] for t in rows("paper_medium.txt")])


def trunc(x, digits):
    return math.floor(x * 10 ** digits + 1e-9) / 10 ** digits


def test_synthetic_inputs_carry_the_printed_tables():
    _, lv = levels()
    assert len(lv) == 11 == len(synth.PAPER_LEVELS) == len(synth.PAPER_LEVEL_SPACING)
    for L in lv:
        assert synth.PAPER_LEVELS[L["level"]] == L["n"] + (L["steps"],)
        assert synth.PAPER_LEVEL_SPACING[L["level"]] == L["dp_km"] + (L["dt"],)
    assert np.array_equal(synth.PAPER_LAYERS, medium())
    M = np.array([[float(v) for v in t] for t in rows("paper_moment_tensor.txt")])
    assert np.array_equal(synth.PAPER_MOMENT_TENSOR, M)
    assert np.array_equal(M, M.T)


@pytest.mark.parametrize("level", [0, 4, 10])
def test_paper_level_problem_uses_the_printed_level(level):
    _, lv = levels()
    L = lv[level]
    p = synth.paper_level(level, nt=4)
    assert (p.nx, p.ny, p.nz) == L["n"]
    assert p.spacing == pytest.approx(tuple(1e3 * d for d in L["dp_km"]), rel=1e-15)
    assert p.dt == L["dt"]
    M = synth.PAPER_MOMENT_TENSOR
    assert list(p.src_comp) == [M[0, 0], M[1, 1], M[2, 2], M[0, 1], M[0, 2], M[1, 2]]


def test_every_printed_time_step_is_stable():
    """Eq. 5 with the model's largest P speed, and the exact von Neumann
    bound of the 4th-order staggered leapfrog scheme, dt vp (7/3)
    sqrt(sum 1/h^2) <= 2 (the largest symbol of Eq. 4 is (9/8 + 1/24) 2/h)."""
    _, lv = levels()
    vp_max = medium()[:, 1].max() * 1e3
    for L in lv:
        h = tuple(1e3 * d for d in L["dp_km"])
        g = ews.ews_grid(*L["n"], *h)
        rule = ews.ews_cfl_dt(g, vp_max)
        assert rule == pytest.approx(0.495 * min(h) / vp_max, rel=1e-15)
        exact = 2.0 / (vp_max * (7.0 / 3.0) * math.sqrt(sum(1.0 / x ** 2 for x in h)))
        assert L["dt"] <= rule <= exact, (L["level"], L["dt"], rule, exact)


def test_spacings_are_domain_size_over_cells_truncated():
    size, lv = levels()
    for L in lv:
        for a in range(3):
            assert trunc(size[a] / L["n"][a], 2) == pytest.approx(L["dp_km"][a], abs=1e-12), \
                (L["level"], a)


def test_max_frequency_column_is_eq6_over_sqrt2():
    """Reading R11: the table's max f is not Eq. 6 itself but Eq. 6 / sqrt 2
    (truncated to the printed digits) at every level; ews_max_freq follows
    Eq. 6 as printed."""
    _, lv = levels()
    vs_min = medium()[:, 2].min() * 1e3
    for L in lv:
        h = tuple(1e3 * d for d in L["dp_km"])
        f6 = ews.ews_max_freq(ews.ews_grid(*L["n"], *h), vs_min)
        assert f6 == pytest.approx(vs_min / (5.0 * max(h)), rel=1e-15)
        assert trunc(f6 / math.sqrt(2.0), L["fmax_digits"]) == pytest.approx(L["fmax"], abs=1e-12)
        assert abs(f6 - L["fmax"]) > 0.25 * L["fmax"]        # Eq. 6 alone does not give it


def test_model_s_speeds_are_p_over_1_74():
    m = medium()
    for top, vp, vs, rho in m:
        assert round(vp / 1.74, 3) == pytest.approx(vs, abs=1e-12), top
    assert np.all(np.diff(m[:, 0]) > 0) and np.all(np.diff(m[:, 1]) > 0)
