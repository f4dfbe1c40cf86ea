"""Pins of the oracle's coarse medium grid (Sec. 2.2.1: medium textures
smaller than the wavefield textures, sampled by trilinear interpolation;
reading R17) against facts outside the oracle:

* with a medium grid equal to the wavefield grid it is reading R4 (the
  2- and 4-cell means), already pinned by the forward pins;
* linear interpolation reproduces a medium that is linear in position
  exactly, at every staggered point away from the clamped edges;
* an independent separable restatement with numpy.interp (per axis, in
  physical coordinates of the cell centres) gives the same values.
"""
import numpy as np
import pytest

from paper_2112_15071_gb300 import synth

H = 10.0


def medium_of(orc, n, coarse=None, fine=None):
    s = orc.OracleSim(*n, (H, H, H))
    if coarse is not None:
        s.set_medium_coarse(*coarse)
    else:
        s.set_medium_lame(*fine)
    return s.medium()         # bx by bz lam lp2m mxy mxz myz, each [nz][ny][nx]


def test_same_resolution_is_the_cell_means(orc):
    p = synth.small_problem(11, 9, 7, nt=1, width=1, nrec=1)
    lame = [a.astype(np.float64) for a in p.lame()]
    a = medium_of(orc, (11, 9, 7), coarse=lame)
    b = medium_of(orc, (11, 9, 7), fine=lame)
    assert np.max(np.abs(a - b) / np.abs(b)) <= 2e-16


@pytest.mark.parametrize("m", [(4, 5, 3), (7, 3, 6)])
def test_linear_medium_is_reproduced(orc, m):
    """Medium cells hold a linear function of their centre's position; the
    sampled value at each staggered point is that function at the point."""
    n = (16, 12, 14)
    mx, my, mz = m
    # centres of medium cells in fine-cell units: (c + 1/2) n / m - 1/2
    cen = [(np.arange(mm) + 0.5) * nn / mm - 0.5 for mm, nn in zip(m, n)]
    Z, Y, X = np.meshgrid(cen[2], cen[1], cen[0], indexing="ij")
    f = lambda x, y, z, c0: c0 + 3.0 * x - 2.0 * y + 1.5 * z
    lam = f(X, Y, Z, 1e10)
    mu = f(X, Y, Z, 2e10)
    rho = f(X, Y, Z, 3e3)
    med = medium_of(orc, n, coarse=(lam, mu, rho))
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    # points inside the hull of the medium cell centres on every axis
    def inside(x, a):
        return (x >= cen[a][0]) & (x <= cen[a][-1])
    pts = {0: (i + 0.5, j, k, 3e3), 1: (i, j + 0.5, k, 3e3), 2: (i, j, k + 0.5, 3e3),
           3: (i, j, k, 1e10), 5: (i + 0.5, j + 0.5, k, 2e10), 6: (i + 0.5, j, k + 0.5, 2e10),
           7: (i, j + 0.5, k + 0.5, 2e10)}
    for q, (x, y, z, c0) in pts.items():
        ok = inside(x, 0) & inside(y, 1) & inside(z, 2)
        assert ok.sum() > 10
        want = f(x, y, z, c0)
        got = 1.0 / med[q] if q < 3 else med[q]
        assert np.max(np.abs(got[ok] - want[ok]) / want[ok]) <= 1e-13, q


def test_separable_restatement(orc):
    """numpy.interp along each axis (physical positions of the medium cell
    centres, constant continuation past the end centres) == the oracle."""
    rng = np.random.default_rng(4)
    n = (13, 10, 9)
    m = (5, 4, 3)
    lam, mu, rho = (rng.uniform(1.0, 2.0, (m[2], m[1], m[0])) * s for s in (1e10, 1e10, 2e3))
    med = medium_of(orc, n, coarse=(lam, mu, rho))
    cen = [(np.arange(mm) + 0.5) * (nn * H / mm) for mm, nn in zip(m, n)]

    def sample(a, x, y, z):
        # x, y, z: positions in metres of one fine point; interpolate axis by axis
        t = np.array([[np.interp(x, cen[0], a[kk, jj, :]) for jj in range(m[1])]
                      for kk in range(m[2])])
        t = np.array([np.interp(y, cen[1], t[kk, :]) for kk in range(m[2])])
        return np.interp(z, cen[2], t)

    rng2 = np.random.default_rng(9)
    for _ in range(40):
        i, j, k = (int(rng2.integers(0, nn)) for nn in n)
        pos = lambda ox, oy, oz: ((i + 0.5 + ox) * H, (j + 0.5 + oy) * H, (k + 0.5 + oz) * H)
        checks = [(1.0 / med[0][k, j, i], sample(rho, *pos(0.5, 0, 0))),
                  (1.0 / med[2][k, j, i], sample(rho, *pos(0, 0, 0.5))),
                  (med[3][k, j, i], sample(lam, *pos(0, 0, 0))),
                  (med[4][k, j, i] - med[3][k, j, i], 2 * sample(mu, *pos(0, 0, 0))),
                  (med[5][k, j, i], sample(mu, *pos(0.5, 0.5, 0))),
                  (med[7][k, j, i], sample(mu, *pos(0, 0.5, 0.5)))]
        for got, want in checks:
            assert abs(got - want) <= 1e-13 * abs(want), (i, j, k, got, want)


def test_wavefield_grid_medium_is_linear_filtering(orc):
    """Reading R4 against the paper's own statement (Sec. 2.2.1: the medium
    is read with linear texture filtering at the staggered points, clamped
    at the edges): numpy.interp along each axis over the cell centres of the
    wavefield-grid medium, evaluated at the staggered points, gives the
    oracle's 2- and 4-cell means; rho is interpolated, then inverted."""
    rng = np.random.default_rng(8)
    n = (7, 6, 5)
    lam, mu, rho = (rng.uniform(1.0, 2.0, (n[2], n[1], n[0])) * s for s in (1e10, 1e10, 2e3))
    med = medium_of(orc, n, fine=(lam, mu, rho))
    cen = [np.arange(nn, dtype=np.float64) for nn in n]

    def sample(a, x, y, z):
        t = np.array([[np.interp(x, cen[0], a[kk, jj, :]) for jj in range(n[1])]
                      for kk in range(n[2])])
        t = np.array([np.interp(y, cen[1], t[kk, :]) for kk in range(n[2])])
        return np.interp(z, cen[2], t)

    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                checks = [(1.0 / med[0][k, j, i], sample(rho, i + 0.5, j, k)),
                          (1.0 / med[1][k, j, i], sample(rho, i, j + 0.5, k)),
                          (1.0 / med[2][k, j, i], sample(rho, i, j, k + 0.5)),
                          (med[3][k, j, i], sample(lam, i, j, k)),
                          (med[5][k, j, i], sample(mu, i + 0.5, j + 0.5, k)),
                          (med[6][k, j, i], sample(mu, i + 0.5, j, k + 0.5)),
                          (med[7][k, j, i], sample(mu, i, j + 0.5, k + 0.5))]
                for got, want in checks:
                    assert abs(got - want) <= 1e-13 * abs(want), (i, j, k, got, want)
