"""Pins of the FP64 oracle's adjoint gradient (CPU only).

The adjoint is the exact reverse of the discrete loop, so it must agree with
central finite differences of the (independently pinned) forward oracle to
the FD truncation level, for every boundary and source kind, in directional
and single-cell form; it must not depend on the checkpoint interval.
"""
import numpy as np
import pytest

from paper_2112_15071_gb300 import synth


def _setup(orc, boundary, kind, seed=3, dims=(14, 12, 13), nt=70):
    p = synth.small_problem(*dims, nt=nt, boundary=boundary, width=3, kind=kind, nrec=4,
                            seed=seed)
    lam, mu, rho = [a.astype(np.float64) for a in p.lame()]
    rng = np.random.default_rng(seed + 100)
    A = rng.standard_normal((3, p.rec_pos.shape[0], p.nt))

    def L(l, m, r):
        s = orc.OracleSim(p.nx, p.ny, p.nz, p.spacing)
        s.set_medium_lame(l, m, r)
        s.set_boundary(boundary, p.width, p.dt, p.f0)
        seis = s.forward(p.nt, p.dt, p.src_kind, p.src_pos, p.src_comp, p.wavelet, p.rec_pos)
        return float(np.sum(A * seis))

    return p, (lam, mu, rho), A, L


@pytest.mark.parametrize("boundary", ["none", "sponge"])
@pytest.mark.parametrize("kind", ["moment", "force"])
def test_gradient_matches_central_fd(orc, boundary, kind):
    p, m, A, L = _setup(orc, boundary, kind)
    g = orc.gradient(p, A, ckpt_every=16, medium=m)
    rng = np.random.default_rng(7)
    for idx in range(3):
        d = rng.standard_normal(m[0].shape)
        h = 1e-4 * np.abs(m[idx]).mean() / np.abs(d).mean()
        plus = [a + (h * d if i == idx else 0) for i, a in enumerate(m)]
        minus = [a - (h * d if i == idx else 0) for i, a in enumerate(m)]
        fd = (L(*plus) - L(*minus)) / (2 * h)
        an = float(np.sum(g[idx] * d))
        assert abs(fd - an) <= 1e-6 * abs(fd), (idx, fd, an)


def test_single_cell_fd(orc):
    p, m, A, L = _setup(orc, "sponge", "moment", seed=11)
    g = orc.gradient(p, A, ckpt_every=10, medium=m)
    for idx in range(3):
        gi = np.abs(g[idx])
        cells = np.argsort(gi.ravel())[-3:]              # where the gradient is largest
        for c in cells:
            cz, cy, cx = np.unravel_index(c, gi.shape)
            h = 1e-5 * m[idx][cz, cy, cx]
            plus = [a.copy() for a in m]
            minus = [a.copy() for a in m]
            plus[idx][cz, cy, cx] += h
            minus[idx][cz, cy, cx] -= h
            fd = (L(*plus) - L(*minus)) / (2 * h)
            assert abs(fd - g[idx][cz, cy, cx]) <= 1e-5 * abs(fd), (idx, c, fd)


def test_checkpoint_interval_does_not_matter(orc):
    p, m, A, _ = _setup(orc, "sponge", "force", seed=5)
    g1 = orc.gradient(p, A, ckpt_every=7, medium=m)
    g2 = orc.gradient(p, A, ckpt_every=0, medium=m)
    assert np.array_equal(g1, g2)


def test_misfit_gradient_of_l2_objective(orc):
    """J = 1/2 dt sum (s - d)^2 has dJ/ds = dt (s - d): FD on J."""
    p, m, _, _ = _setup(orc, "none", "moment", seed=21, nt=60)
    rng = np.random.default_rng(0)
    seis = orc.run_problem(p)
    obs = seis * (1 + 0.3 * rng.standard_normal(seis.shape))

    def J(l, mu, r):
        s = orc.OracleSim(p.nx, p.ny, p.nz, p.spacing)
        s.set_medium_lame(l, mu, r)
        s.set_boundary("none")
        x = s.forward(p.nt, p.dt, p.src_kind, p.src_pos, p.src_comp, p.wavelet, p.rec_pos)
        return 0.5 * p.dt * float(np.sum((x - obs) ** 2))

    g = orc.gradient(p, p.dt * (seis - obs), medium=m)
    d = rng.standard_normal(m[0].shape)
    h = 1e-4 * np.abs(m[2]).mean() / np.abs(d).mean()
    fd = (J(m[0], m[1], m[2] + h * d) - J(m[0], m[1], m[2] - h * d)) / (2 * h)
    assert abs(fd - float(np.sum(g[2] * d))) <= 1e-6 * abs(fd)


def test_cpml_adjoint_is_refused(orc):
    p = synth.small_problem(12, 12, 12, nt=10, boundary="cpml", width=3)
    with pytest.raises(ValueError):
        orc.gradient(p, np.zeros((3, p.rec_pos.shape[0], p.nt)))


@pytest.mark.parametrize("boundary", ["none", "sponge"])
@pytest.mark.parametrize("kind", ["moment", "force"])
def test_dot_product_with_the_tangent_model(orc, boundary, kind):
    """<J dm, A> = <dm, J^T A>: the oracle's adjoint gradient against its
    tangent-linear (forward-mode) model, to rounding, per parameter."""
    p, m, A, _ = _setup(orc, boundary, kind, seed=17)
    g = orc.gradient(p, A, ckpt_every=13, medium=m)
    rng = np.random.default_rng(23)
    for idx in range(3):
        dm = [np.zeros_like(m[0]) for _ in range(3)]
        dm[idx] = rng.standard_normal(m[0].shape) * np.abs(m[idx]).mean()
        ds = orc.tangent(p, dm, medium=m)
        lhs = float(np.sum(ds * A))
        rhs = float(np.sum(dm[idx] * g[idx]))
        assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs)), (idx, lhs, rhs)


def test_tangent_matches_finite_differences(orc):
    """The tangent model itself against central differences of the forward."""
    p, m, A, L = _setup(orc, "sponge", "force", seed=29)
    rng = np.random.default_rng(31)
    dm = [rng.standard_normal(m[0].shape) * np.abs(a).mean() for a in m]
    ds = orc.tangent(p, dm, medium=m)
    h = 1e-5
    def run(sign):
        s = orc.OracleSim(p.nx, p.ny, p.nz, p.spacing)
        s.set_medium_lame(*[a + sign * h * d for a, d in zip(m, dm)])
        s.set_boundary("sponge", p.width, p.dt, p.f0)
        return s.forward(p.nt, p.dt, p.src_kind, p.src_pos, p.src_comp, p.wavelet, p.rec_pos)
    fd = (run(1) - run(-1)) / (2 * h)
    assert np.linalg.norm(ds - fd) <= 1e-6 * np.linalg.norm(fd)
