"""Invariances of the oracle's discrete scheme that any dropped or doubled
spacing, time-step or index term would break (CPU only).

* Scaling: with every spacing and the time step doubled (and, for the
  C-PML, the reference frequency halved), the scheme is the same scheme in
  units twice as large; every operation scales by a power of two, so each
  seismogram is exactly one quarter of the original (a moment or force
  deposited over 8x the volume with 2x the time step).  This holds bitwise.
* Translation: in a homogeneous medium without boundaries, shifting source
  and receivers by whole cells shifts the response (up to the far-field
  leakage of the stencil to the grid edges).
"""
import numpy as np
import pytest

from paper_2112_15071_gb300 import synth


def run(orc, p, scale, bnd, kind, nt):
    h = tuple(scale * x for x in p.spacing)
    s = orc.OracleSim(p.nx, p.ny, p.nz, h)
    s.set_medium_vel(p.vp, p.vs, p.rho)
    dt = scale * p.dt
    if bnd == "cpml":
        s.set_boundary("cpml", p.width, dt, p.f0 / scale)
    else:
        s.set_boundary(bnd, p.width)
    comp = synth.double_couple(20, 50, 70) if kind == "moment" else np.array([0.3e10, -1e10, 0.7e10])
    return s.forward(nt, dt, kind, scale * p.src_pos, comp, p.wavelet, scale * p.rec_pos)


@pytest.mark.parametrize("bnd", ["none", "sponge", "cpml"])
@pytest.mark.parametrize("kind", ["moment", "force"])
def test_doubling_all_units_quarters_every_seismogram(orc, bnd, kind):
    p = synth.small_problem(22, 19, 17, nt=60, h=10.0, boundary=bnd, width=4, kind=kind,
                            nrec=6, seed=11)
    p.spacing = (10.0, 12.5, 7.5)                 # unequal spacings
    a = run(orc, p, 1.0, bnd, kind, 60)
    b = run(orc, p, 2.0, bnd, kind, 60)
    assert np.max(np.abs(a)) > 0
    np.testing.assert_array_equal(b, a / 4.0)


def test_whole_cell_shift_shifts_the_response(orc):
    n, h = 44, 10.0
    vp, vs, rho = synth.homogeneous(n, n, n)
    dt = 0.5 * synth.PAPER_CFL * h / 3000.0
    nt = 40
    w = synth.ricker(nt, dt, 60.0, shift=0.5)
    src = np.array([19.3, 20.6, 18.8]) * h
    rec = src + np.array([[3.2, 0.4, -1.7], [-2.5, 2.9, 0.6], [0.0, -3.1, 2.2]]) * h
    out = []
    for shift in (np.zeros(3), np.array([2.0, 1.0, 3.0]) * h):
        s = orc.OracleSim(n, n, n, (h, h, h))
        s.set_medium_vel(vp, vs, rho)
        s.set_boundary("none")
        out.append(s.forward(nt, dt, "moment", src + shift, synth.double_couple(10, 80, 30), w,
                             rec + shift))
    a, b = out
    assert np.max(np.abs(a)) > 0
    assert np.max(np.abs(b - a)) <= 1e-10 * np.max(np.abs(a))
