"""The seeded synthetic inputs follow the recipes they stand for (CPU only):
grid, spacing, time step, boundary, source and receiver layout of each
workload, and the statistics of the layered + random model (layer speeds,
perturbation amplitude, correlation length of the Gaussian kernel, vp/vs,
Gardner density).  The generators hold none of the method's arithmetic;
these tests check that the workloads are what the measurements claim."""
import math

import numpy as np
import pytest

from paper_2112_15071_gb300 import synth

CFL = 0.495                                  # Eq. 5


def test_config1_recipe():
    p = synth.config1(nt=500)
    assert (p.nx, p.ny, p.nz, p.spacing) == (64, 64, 64, (10.0, 10.0, 10.0))
    assert p.dt == pytest.approx(0.5 * CFL * 10.0 / 3000.0, rel=1e-15)
    assert (p.boundary, p.width, p.src_kind) == ("sponge", 16, "moment")
    assert np.all(p.vp == 3000.0) and np.all(p.vs == 1730.0) and np.all(p.rho == 2500.0)
    assert list(p.src_pos) == [320.0, 320.0, 320.0]
    assert list(p.src_comp) == [1e15, 1e15, 1e15, 0.0, 0.0, 0.0]
    d = np.linalg.norm(p.rec_pos - p.src_pos, axis=1)
    assert len(d) == 8 and d.min() >= 199.9 and d.max() <= 213.0
    # moment-rate samples at t = (n + 1/2) dt, Ricker peak at t0 = 1.5 / f0
    t_peak = (np.argmax(p.wavelet) + 0.5) * p.dt
    assert abs(t_peak - 1.5 / 15.0) <= p.dt


def test_ricker_closed_form():
    dt, f0 = 1e-3, 10.0
    w = synth.ricker(400, dt, f0, shift=0.5)
    t = (np.arange(400) + 0.5) * dt - 1.5 / f0
    a = (math.pi * f0 * t) ** 2
    assert np.allclose(w, (1 - 2 * a) * np.exp(-a), rtol=0, atol=1e-7)
    assert abs(w[0]) < 2e-8                   # ~1e-8 of the peak: no step at the start


def test_layered_random_statistics():
    n, h, L = 96, 20.0, 200.0
    layers = (2000.0, 3000.0, 4000.0, 5000.0, 6000.0)
    vp, vs, rho = synth.layered_random(n, n, n, (h, h, h), seed=15071)
    k = np.arange(n)
    base = np.asarray(layers)[np.minimum(k * 5 // n, 4)][:, None, None]
    p = vp.astype(np.float64) / base - 1.0
    assert np.max(np.abs(p)) == pytest.approx(0.05, rel=1e-5)      # max |p| = 5 %
    assert np.allclose(vs, vp / np.float32(1.73), rtol=1e-6)
    assert np.allclose(rho, 310.0 * vp.astype(np.float64) ** 0.25, rtol=1e-6)
    # white noise convolved with exp(-r^2 / L^2) has autocorrelation
    # exp(-r^2 / (2 L^2)): 0.607 at lag L, 0.135 at lag 2 L (L = 10 cells)
    q = p - p.mean()
    var = np.mean(q * q)
    for lag, want in ((int(L / h), math.exp(-0.5)), (int(2 * L / h), math.exp(-2.0))):
        for axis in (0, 1, 2):
            c = np.mean(q * np.roll(q, lag, axis=axis)) / var
            assert abs(c - want) <= 0.1, (lag, axis, c)


def test_config2_recipe_layout():
    p = synth.config2(n=96, nt=10)
    assert p.spacing == (20.0, 20.0, 20.0) and (p.boundary, p.width) == ("cpml", 20)
    assert p.dt == pytest.approx(0.5 * CFL * 20.0 / 6300.0, rel=1e-15)
    assert p.src_kind == "moment" and p.f0 == 5.0
    assert np.allclose(p.src_comp, synth.double_couple(30, 60, 90))
    assert p.src_pos[2] == min(100, 96 - 3) * 20.0          # 2 km down, clamped to the grid
    assert p.rec_pos.shape == (256, 3) and np.all(p.rec_pos[:, 2] == 20 * 20.0)
    # receivers evenly over the interior in x and y
    xs = np.unique(p.rec_pos[:, 0])
    assert len(xs) == 16 and xs.min() > 20 * 20.0 and xs.max() < (96 - 20) * 20.0
    assert np.allclose(np.diff(xs), np.diff(xs)[0])


def test_full_size_config2_and_3_parameters():
    """Time steps of the full-size workloads (the recipes' closed form
    against the figures quoted for them), without generating their models."""
    assert 0.5 * CFL * 20.0 / 6300.0 == pytest.approx(7.857e-4, rel=1e-3)   # 256^3
    assert 0.5 * CFL * 50.0 / 6300.0 == pytest.approx(1.964e-3, rel=1e-3)   # 1024^2 x 512


def test_double_couple_is_traceless_with_scalar_moment():
    for sdr in ((30, 60, 90), (0, 90, 0), (45, 45, -90), (123, 17, 33)):
        m = synth.double_couple(*sdr, m0=2.0)
        M = np.array([[m[0], m[3], m[4]], [m[3], m[1], m[5]], [m[4], m[5], m[2]]])
        assert abs(np.trace(M)) <= 1e-12
        ev = np.sort(np.linalg.eigvalsh(M))
        assert np.allclose(ev, [-2.0, 0.0, 2.0], atol=1e-12)       # pure double couple


def test_config5_draws():
    shots = synth.config5_shots(2)
    for s in shots:
        assert s.nx == s.ny == s.nz and 96 <= s.nx <= 224 and s.nx % 8 == 0
        assert 800 <= s.nt <= 1600 and 5.0 <= s.f0 <= 15.0
        h = s.spacing[0]
        vs_min = 2000.0 * 0.95 / 1.73
        assert h == math.floor(vs_min / (12.5 * s.f0) * 2) / 2         # rounded down to 0.5 m
        assert (s.boundary, s.width) == ("sponge", 16)
        assert list(s.src_pos) == [(s.nx // 2) * h, (s.ny // 2) * h, (s.nz // 3) * h]
        assert s.rec_pos.shape == (64, 3)
    # the same seed gives the same draws
    again = synth.config5_shots(2)
    assert [(s.nx, s.nt, s.f0) for s in shots] == [(s.nx, s.nt, s.f0) for s in again]
