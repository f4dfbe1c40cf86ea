"""Pins of the oracle's free surface (Sec. 2.5 vacuum formulation, reading
R16) against facts outside the oracle:

* an independent sparse-operator restatement (oracle/brute.py) whose 2-tap
  weights come from the moment conditions and whose switch is decided from
  the tap geometry;
* closed forms: on a cubic profile the 2nd-order difference errs by exactly
  h^2/4 times the profile's z^3 coefficient, the 4th-order one not at all,
  which fixes the planes the switch applies to;
* physics: the vertical velocity of a P wave at normal incidence doubles at a
  free surface, and surface waves travel at the Rayleigh speed, the root of
  the Rayleigh equation (Aki & Richards, Sec. 5.1);
* stability at the exact bound of the scheme with the surface in place.
"""
import numpy as np
import pytest
from scipy.optimize import brentq

from paper_2112_15071_gb300 import synth

H = 10.0
BOUND = 6.0 / (7.0 * np.sqrt(3.0))       # exact stability constant of Eq. 4 in 3D


def homogeneous_sim(orc, n, nz, ks, eps=1e-3, boundary="none", width=0, dt=0.0, f0=0.0):
    vp, vs, rho = synth.homogeneous(n, n, nz)
    s = orc.OracleSim(n, n, nz, (H, H, H))
    if ks is not None:
        s.set_free_surface(ks, eps)
    s.set_medium_vel(vp, vs, rho)
    s.set_boundary(boundary, width, dt, f0)
    return s


@pytest.mark.parametrize("boundary", ["none", "sponge", "cpml"])
@pytest.mark.parametrize("kind", ["moment", "force"])
def test_brute_force_with_surface(orc, boundary, kind):
    """Oracle == the sparse-operator restatement with a surface at ks = 3,
    50 steps, 8^3 and a ragged 9 x 7 x 10 grid."""
    from oracle import brute
    for (nx, ny, nz) in ((8, 8, 8), (9, 7, 10)):
        p = synth.small_problem(nx, ny, nz, nt=50, width=2, boundary=boundary, kind=kind,
                                nrec=3)
        p.free_surface = (3, 1e-2)
        so, sim = orc.run_problem(p, return_sim=True)
        b = brute.from_velocities(nx, ny, nz, p.spacing, p.vp, p.vs, p.rho,
                                  surface=p.free_surface)
        if boundary == "sponge":
            b.set_sponge(p.width)
        if boundary == "cpml":
            b.set_cpml(p.width, p.dt, p.f0)
        sb = b.forward(p.nt, p.dt, p.src_kind, p.src_pos, p.src_comp, p.wavelet, p.rec_pos)
        assert np.abs(sb).max() > 0
        assert np.linalg.norm(so - sb) <= 1e-13 * np.linalg.norm(sb)
        fo, fb = sim.get_state(), b.state()
        for q in range(9):
            assert np.max(np.abs(fo[q] - fb[q])) <= 1e-13 * max(np.abs(fb[q]).max(), 1e-300)


def test_second_order_planes_on_cubic(orc):
    """One pass from rest on a field cubic in z: the z-derivative is exact
    except on the switched planes, where it is 3 z0^2 + h^2 / 4.  The
    switched planes follow from the reading (outputs at integer z: ks-1, ks;
    at half-integer z: ks-2, ks-1, ks)."""
    n, nz, ks = 10, 24, 9
    dt = 1e-4
    z_int = np.arange(nz) * H                # sxx, vx, vy, sxy planes
    z_half = (np.arange(nz) + 0.5) * H       # vz, sxz, syz planes
    planes = np.arange(3, nz - 3)            # away from the zero exterior in z
    c = slice(3, n - 3)                      # interior columns

    def check(got, z_out, switched):
        want = 3.0 * z_out ** 2
        for k in planes:
            exp = want[k] + (H * H / 4.0 if k in switched else 0.0)
            g = got[k, c, c]
            assert np.max(np.abs(g - exp)) <= 1e-9 * exp, (k, g.ravel()[0], exp)

    # velocity pass: vz from szz (half-integer outputs), vx from sxz (integer)
    s = homogeneous_sim(orc, n, nz, ks)
    med = s.medium()                          # bx by bz lam lp2m mxy mxz myz
    st = np.zeros((9, nz, n, n))
    st[5] = (z_int ** 3)[:, None, None]       # szz on integer z
    st[7] = (z_half ** 3)[:, None, None]      # sxz on half-integer z
    s.set_state(st)
    s.step_velocity(dt)
    out = s.get_state()
    check(out[2] / (dt * med[2]), z_half, {ks - 2, ks - 1, ks})
    check(out[0] / (dt * med[0]), z_int, {ks - 1, ks})

    # stress pass: szz from vz (integer outputs), sxz from vx (half-integer)
    s = homogeneous_sim(orc, n, nz, ks)
    st = np.zeros((9, nz, n, n))
    st[2] = (z_half ** 3)[:, None, None]      # vz on half-integer z
    st[0] = (z_int ** 3)[:, None, None]       # vx on integer z
    s.set_state(st)
    s.step_stress(dt)
    out = s.get_state()
    check(out[5] / (dt * med[4]), z_int, {ks - 1, ks})
    check(out[7] / (dt * med[6]), z_half, {ks - 2, ks - 1, ks})


def test_vacuum_medium_and_surface_means(orc):
    """Above the surface the medium is eps times the column's surface cell;
    the xz / yz shear modulus on the surface plane is the harmonic mean."""
    n, nz, ks, eps = 6, 12, 5, 1e-3
    p = synth.small_problem(n, n, nz, nt=1, width=1, nrec=1)
    lam, mu, rho = synth.Problem.lame(p)
    s = orc.OracleSim(n, n, nz, (H, H, H))
    s.set_free_surface(ks, eps)
    s.set_medium_lame(lam, mu, rho)
    med = s.medium()
    lam64 = lam.astype(np.float64)
    mu64 = mu.astype(np.float64)
    rho64 = rho.astype(np.float64)
    lam_v, mu_v, rho_v = (a.copy() for a in (lam64, mu64, rho64))
    for a in (lam_v, mu_v, rho_v):
        a[:ks] = eps * a[ks]
    assert np.allclose(med[3], lam_v, rtol=1e-15, atol=0)
    assert np.allclose(med[4], lam_v + 2 * mu_v, rtol=1e-15, atol=0)
    k, j, i = ks - 1, 2, 3
    four = [mu_v[k, j, i], mu_v[k, j, i + 1], mu_v[k + 1, j, i], mu_v[k + 1, j, i + 1]]
    assert med[6][k, j, i] == pytest.approx(4.0 / sum(1.0 / m for m in four), rel=1e-14)
    four_y = [mu_v[k, j, i], mu_v[k, j + 1, i], mu_v[k + 1, j, i], mu_v[k + 1, j + 1, i]]
    assert med[7][k, j, i] == pytest.approx(4.0 / sum(1.0 / m for m in four_y), rel=1e-14)
    # one plane deeper: arithmetic
    four_a = [mu_v[ks, j, i], mu_v[ks, j, i + 1], mu_v[ks + 1, j, i], mu_v[ks + 1, j, i + 1]]
    assert med[6][ks, j, i] == pytest.approx(sum(four_a) / 4.0, rel=1e-14)
    # buoyancy of vz straddling the surface: 1 / mean of eps rho and rho
    assert med[2][ks - 1, j, i] == pytest.approx(
        1.0 / (0.5 * (rho_v[ks - 1, j, i] + rho_v[ks, j, i])), rel=1e-14)


def test_normal_incidence_doubling(orc):
    """An explosion 30 cells below the surface: the vertical velocity at the
    epicentre on the surface plane peaks at twice the whole-space value, at
    the same time, and the horizontal components stay ~0 there."""
    n, nz, ks, sk, f0, nt = 60, 70, 10, 40, 15.0, 420
    dt = 0.5 * synth.PAPER_CFL * H / 3000.0
    rec = np.array([[30 * H, 30 * H, (ks - 0.5) * H]])
    w = synth.ricker(nt, dt, f0, shift=0.5)
    pos = np.array([30 * H, 30 * H, sk * H])
    out = []
    for ksurf in (ks, None):
        s = homogeneous_sim(orc, n, nz, ksurf, boundary="sponge", width=10, dt=dt, f0=f0)
        out.append(s.forward(nt, dt, "moment", pos, synth.explosion(), w, rec))
    fs, ws = out
    ratio = np.abs(fs[2, 0]).max() / np.abs(ws[2, 0]).max()
    assert 1.9 <= ratio <= 2.1, ratio
    assert abs(int(np.argmax(np.abs(fs[2, 0]))) - int(np.argmax(np.abs(ws[2, 0])))) <= 2
    assert np.abs(fs[:2, 0]).max() <= 0.05 * np.abs(fs[2, 0]).max()


def rayleigh_speed(vp, vs):
    """Root c/vs of the Rayleigh equation (2 - x)^2 = 4 sqrt(1 - x vs^2/vp^2)
    sqrt(1 - x), x = (c / vs)^2."""
    g = (vs / vp) ** 2
    f = lambda x: (2.0 - x) ** 2 - 4.0 * np.sqrt(1.0 - g * x) * np.sqrt(1.0 - x)
    return np.sqrt(brentq(f, 0.5, 0.999))


@pytest.mark.slow
def test_rayleigh_wave_speed(orc):
    """A vertical force one cell below the surface; vertical surface motion
    at offsets 300 .. 900 m.  The lag of the cross-correlation between
    neighbouring receivers gives the Rayleigh speed within 3 % (not the S
    speed, 8 % faster)."""
    n, nz, ks, f0 = 140, 50, 10, 6.0
    dt = 0.5 * synth.PAPER_CFL * H / 3000.0
    nt = int(1.2 / dt)
    offs = np.array([30, 50, 70, 90])
    rec = np.array([[(30 + o) * H, 70 * H, (ks - 0.5) * H] for o in offs])
    s = homogeneous_sim(orc, n, nz, ks, boundary="sponge", width=10, dt=dt, f0=f0)
    w = synth.ricker(nt, dt, f0, shift=0.0)
    seis = s.forward(nt, dt, "force", np.array([30 * H, 70 * H, (ks + 1) * H]),
                     np.array([0.0, 0.0, 1e10]), w, rec)
    vz = seis[2]
    vp, vs = 3000.0, 1730.0
    cr = rayleigh_speed(vp, vs) * vs
    speeds = []
    for q in range(len(offs) - 1):
        cc = np.correlate(vz[q + 1], vz[q], mode="full")
        m = int(np.argmax(cc))
        y0, y1, y2 = cc[m - 1: m + 2]
        lag = m - (nt - 1) + 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
        speeds.append((offs[q + 1] - offs[q]) * H / (lag * dt))
    for c in speeds:
        assert abs(c / cr - 1.0) <= 0.03, (speeds, cr)
        assert abs(c / vs - 1.0) >= 0.05, (speeds, vs)


def test_stable_at_the_bound_with_surface(orc):
    """A random state below the surface at dt = 0.99 x the exact bound, 4000
    steps: the fields stay bounded (no growth between the two halves)."""
    n, ks = 16, 5
    s = homogeneous_sim(orc, n, n, ks)
    rng = np.random.default_rng(3)
    st = rng.standard_normal((9, n, n, n))
    st[:3] *= 1e-3
    st[3:] *= 1e6
    st[:, :ks] = 0.0
    s.set_state(st)
    dt = 0.99 * BOUND * H / 3000.0
    peaks = []
    for _ in range(8):
        for _ in range(500):
            s.step_velocity(dt)
            s.step_stress(dt)
        peaks.append(np.abs(s.get_state()[:3]).max())
    assert np.all(np.isfinite(peaks))
    assert max(peaks[4:]) <= 4.0 * max(peaks[:4]), peaks


def _surface_setup(orc, boundary, kind, seed=3, dims=(14, 12, 16), nt=70, ks=5, eps=1e-2):
    """Adjoint set-up with a surface: source below it, receivers on it and
    below it; L = <A, seis> for a fixed random A."""
    p = synth.small_problem(*dims, nt=nt, boundary=boundary, width=3, kind=kind, nrec=4,
                            seed=seed)
    h = p.spacing[2]
    p.free_surface = (ks, eps)
    p.src_pos = p.src_pos.copy()
    p.src_pos[2] = (ks + 3.4) * h
    p.rec_pos = p.rec_pos.copy()
    p.rec_pos[::2, 2] = (ks - 0.5) * h
    p.rec_pos[1::2, 2] = (ks + 1.3) * h
    lam, mu, rho = [a.astype(np.float64) for a in p.lame()]
    rng = np.random.default_rng(seed + 100)
    A = rng.standard_normal((3, p.rec_pos.shape[0], p.nt))

    def L(l, m, r):
        s = orc.OracleSim(p.nx, p.ny, p.nz, p.spacing)
        s.set_free_surface(*p.free_surface)
        s.set_medium_lame(l, m, r)
        s.set_boundary(boundary, p.width, p.dt, p.f0)
        seis = s.forward(p.nt, p.dt, p.src_kind, p.src_pos, p.src_comp, p.wavelet, p.rec_pos)
        return float(np.sum(A * seis))

    return p, (lam, mu, rho), A, L


@pytest.mark.parametrize("boundary", ["none", "sponge"])
@pytest.mark.parametrize("kind", ["moment", "force"])
def test_surface_dot_product(orc, boundary, kind):
    """<J dm, A> = <dm, J^T A> with the surface: the adjoint's transposed
    differences (column by column from the switched weights), harmonic-mean
    chain rule and vacuum folding against the tangent model, to rounding."""
    p, m, A, _ = _surface_setup(orc, boundary, kind, seed=17)
    g = orc.gradient(p, A, ckpt_every=13, medium=m)
    rng = np.random.default_rng(23)
    for idx in range(3):
        dm = [np.zeros_like(m[0]) for _ in range(3)]
        dm[idx] = rng.standard_normal(m[0].shape) * np.abs(m[idx]).mean()
        ds = orc.tangent(p, dm, medium=m)
        lhs = float(np.sum(ds * A))
        rhs = float(np.sum(dm[idx] * g[idx]))
        assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs)), (idx, lhs, rhs)


@pytest.mark.parametrize("kind", ["moment", "force"])
def test_surface_gradient_matches_central_fd(orc, kind):
    """The adjoint gradient with the surface against central differences of
    the forward oracle (directional, each parameter); the model values above
    the surface are unused, so their gradient is zero."""
    p, m, A, L = _surface_setup(orc, "sponge", kind, seed=9)
    g = orc.gradient(p, A, ckpt_every=16, medium=m)
    ks = p.free_surface[0]
    for idx in range(3):
        assert np.all(g[idx][:ks] == 0.0)
    rng = np.random.default_rng(7)
    for idx in range(3):
        d = rng.standard_normal(m[0].shape)
        h = 1e-4 * np.abs(m[idx]).mean() / np.abs(d).mean()
        plus = [a + (h * d if i == idx else 0) for i, a in enumerate(m)]
        minus = [a - (h * d if i == idx else 0) for i, a in enumerate(m)]
        fd = (L(*plus) - L(*minus)) / (2 * h)
        an = float(np.sum(g[idx] * d))
        assert abs(fd - an) <= 1e-6 * abs(fd), (idx, fd, an)


def test_surface_tangent_matches_finite_differences(orc):
    p, m, A, L = _surface_setup(orc, "sponge", "moment", seed=29)
    rng = np.random.default_rng(31)
    dm = [rng.standard_normal(m[0].shape) * np.abs(a).mean() for a in m]
    ds = orc.tangent(p, dm, medium=m)
    h = 1e-5

    def run(sign):
        s = orc.OracleSim(p.nx, p.ny, p.nz, p.spacing)
        s.set_free_surface(*p.free_surface)
        s.set_medium_lame(*[a + sign * h * d for a, d in zip(m, dm)])
        s.set_boundary("sponge", p.width, p.dt, p.f0)
        return s.forward(p.nt, p.dt, p.src_kind, p.src_pos, p.src_comp, p.wavelet, p.rec_pos)
    fd = (run(1) - run(-1)) / (2 * h)
    assert np.linalg.norm(ds - fd) <= 1e-6 * np.linalg.norm(fd)
