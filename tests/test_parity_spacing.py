"""GPU parity against the FP64 oracle on grids whose spacing differs per axis.

Eq. 4 divides each derivative by its own axis spacing, and the paper's
level-of-detail table (Sec. 3.2.1) runs grids with dx != dy != dz.  With
equal spacings the x, y and z coefficients of the CUDA passes coincide, so
a swapped or mis-indexed per-axis coefficient (the Eq. 4 weights / h, the
C-PML damping d0 of each axis, the trilinear tap weights of sources and
receivers, the per-axis stability bound) would pass every cubic-grid test.
Here every such path runs with three different spacings against the
oracle, whose per-axis arithmetic is pinned independently (Eq. 4 quartics
and the unit-scaling invariance with unequal spacings).  Bars as for the
cubic grids: forward 1e-5 relative L2, gradient 1e-4 against the FP64
adjoint.
"""
import numpy as np
import pytest

from paper_2112_15071_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
TOL_ADJ = 1e-4
SPACINGS = [(10.0, 14.0, 7.0), (13.0, 6.5, 9.0)]


@pytest.fixture(scope="module")
def ews():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_15071_gb300 import ews as E
    E.load()
    return E


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def check_state(got, want, tol=TOL):
    for q in range(9):
        if np.linalg.norm(want[q]) == 0:
            assert np.all(got[q] == 0), q
            continue
        assert rel(got[q], want[q]) <= tol, (q, rel(got[q], want[q]))


@pytest.mark.parametrize("spacing,dims", [(SPACINGS[0], (70, 45, 37)),
                                          (SPACINGS[1], (33, 65, 40))])
@pytest.mark.parametrize("boundary", ["none", "sponge", "cpml"])
@pytest.mark.parametrize("kind", ["moment", "force"])
def test_forward_unequal_spacing(ews, orc, spacing, dims, boundary, kind):
    p = synth.small_problem(*dims, nt=150, boundary=boundary, kind=kind, width=6,
                            seed=sum(dims) + 7, spacing=spacing)
    assert len(set(p.spacing)) == 3
    want, osim = orc.run_problem(p, return_sim=True)
    sim = ews.simulation_for(p)
    got = sim.run(p.nt, p.dt)
    assert np.abs(want).max() > 0
    assert rel(got, want) <= TOL, rel(got, want)
    check_state(sim.get_state(), osim.get_state())


def test_axes_are_distinguished(ews, orc):
    """The same problem with its spacings permuted gives a different
    response, so the comparison above can see a swapped axis."""
    p = synth.small_problem(40, 36, 30, nt=100, boundary="sponge", kind="moment", width=5,
                            seed=5, spacing=(10.0, 14.0, 7.0))
    q = synth.small_problem(40, 36, 30, nt=100, boundary="sponge", kind="moment", width=5,
                            seed=5, spacing=(10.0, 14.0, 7.0))
    q.spacing = (14.0, 10.0, 7.0)
    q.src_pos = q.src_pos * np.array([1.4, 1 / 1.4, 1.0])
    q.rec_pos = q.rec_pos * np.array([1.4, 1 / 1.4, 1.0])
    a = ews.simulation_for(p).run(p.nt, p.dt)
    b = ews.simulation_for(q).run(q.nt, q.dt)
    assert rel(a, b) > 1e-2
    assert rel(b, orc.run_problem(q)) <= TOL


@pytest.mark.parametrize("boundary", ["sponge", "cpml"])
@pytest.mark.parametrize("kind", ["moment", "force"])
def test_free_surface_unequal_spacing(ews, orc, boundary, kind):
    """The surface's 2nd-order z-difference takes 1/dz, not 1/dx."""
    sp = SPACINGS[0]
    ks = 8
    p = synth.small_problem(48, 40, 36, nt=100, boundary=boundary, kind=kind, width=5,
                            nrec=6, seed=17, spacing=sp)
    p.free_surface = (ks, 1e-3)
    p.src_pos = p.src_pos.copy()
    p.src_pos[2] = max(p.src_pos[2], (ks + 4.3) * sp[2])
    p.rec_pos = p.rec_pos.copy()
    p.rec_pos[::2, 2] = (ks - 0.5) * sp[2]
    p.rec_pos[1::2, 2] = np.maximum(p.rec_pos[1::2, 2], (ks + 1.2) * sp[2])
    want, osim = orc.run_problem(p, return_sim=True)
    sim = ews.simulation_for(p)
    got = sim.run(p.nt, p.dt)
    assert rel(got, want) <= TOL, rel(got, want)
    check_state(sim.get_state(), osim.get_state())


def test_coarse_medium_unequal_spacing(ews, orc):
    p = synth.small_problem(70, 45, 37, nt=90, boundary="cpml", kind="force", width=6,
                            seed=23, spacing=SPACINGS[0], layered=False)
    # layer speeds of the coarse recipe within the problem's CFL speed
    synth.with_coarse_medium(p, (9, 7, 5), seed=23, layer_vp=(2400.0, 2700.0, 2950.0))
    want = orc.run_problem(p)
    got = ews.simulation_for(p).run(p.nt, p.dt)
    assert rel(got, want) <= TOL, rel(got, want)


@pytest.mark.parametrize("boundary", ["none", "sponge"])
@pytest.mark.parametrize("kind", ["moment", "force"])
def test_adjoint_unequal_spacing(ews, orc, boundary, kind):
    p = synth.small_problem(40, 36, 28, nt=120, boundary=boundary, kind=kind, width=5,
                            nrec=6, seed=31, spacing=SPACINGS[1])
    lame = p.lame()
    A = np.random.default_rng(6).standard_normal((3, p.rec_pos.shape[0], p.nt)).astype(np.float32)
    want = orc.gradient(p, A.astype(np.float64), ckpt_every=25,
                        medium=[a.astype(np.float64) for a in lame])
    sim = ews.simulation_for(p)
    sim.set_model_lame(*lame)
    for budget in (-1, 0):              # history resident / recomputed per segment
        sim.set_history_budget(budget)
        got = sim.adjoint(p.nt, p.dt, A, ckpt_every=25)
        for q in range(3):
            assert np.abs(want[q]).max() > 0
            assert rel(got[q], want[q]) <= TOL_ADJ, (budget, q, rel(got[q], want[q]))


def test_adjoint_free_surface_unequal_spacing(ews, orc):
    sp = SPACINGS[0]
    ks = 8
    p = synth.small_problem(40, 36, 30, nt=120, boundary="sponge", kind="moment", width=5,
                            nrec=6, seed=37, spacing=sp)
    p.free_surface = (ks, 1e-3)
    p.src_pos = p.src_pos.copy()
    p.src_pos[2] = max(p.src_pos[2], (ks + 4.3) * sp[2])
    p.rec_pos = p.rec_pos.copy()
    p.rec_pos[::2, 2] = (ks - 0.5) * sp[2]
    p.rec_pos[1::2, 2] = np.maximum(p.rec_pos[1::2, 2], (ks + 1.2) * sp[2])
    lame = p.lame()
    A = np.random.default_rng(7).standard_normal((3, p.rec_pos.shape[0], p.nt)).astype(np.float32)
    want = orc.gradient(p, A.astype(np.float64), ckpt_every=30,
                        medium=[a.astype(np.float64) for a in lame])
    sim = ews.simulation_for(p)
    sim.set_model_lame(*lame)
    got = sim.adjoint(p.nt, p.dt, A, ckpt_every=30)
    for q in range(3):
        assert rel(got[q], want[q]) <= TOL_ADJ, (q, rel(got[q], want[q]))


def test_batched_forward_unequal_spacing(ews, orc):
    """Shots of different per-axis spacings in one persistent launch."""
    import torch
    probs = [synth.small_problem(40, 36, 28, nt=70, boundary="sponge", kind="moment", width=5,
                                 nrec=6, seed=41, spacing=SPACINGS[0]),
             synth.small_problem(33, 65, 40, nt=50, boundary="sponge", kind="force", width=5,
                                 nrec=6, seed=42, spacing=SPACINGS[1])]
    shots = [{"sim": ews.simulation_for(p), "nt": p.nt, "dt": p.dt,
              "seis": torch.zeros((3, p.rec_pos.shape[0], p.nt), device="cuda")} for p in probs]
    ews.ews_batch(shots)
    torch.cuda.synchronize()
    for p, d in zip(probs, shots):
        assert rel(d["seis"].cpu().numpy(), orc.run_problem(p)) <= TOL


@pytest.mark.parametrize("level", [0, 2])
def test_paper_level_printed_spacing(ews, orc, level):
    """Levels 0 and 2 of the paper's level-of-detail table (Sec. 3.2.1: grid,
    per-axis spacing and time step as printed; Sec. 3.1.2 1D model; Eq. 7
    tensor), 100 steps.  The printed Ricker frequency would put the pulse
    far past 100 steps, so the wavelet is a Ricker peaking at step 40, and
    the receivers sit a few cells around the source."""
    nt = 100
    p = synth.paper_level(level, nt=nt)
    assert len(set(p.spacing)) == 3
    t0 = 40 * p.dt
    p.wavelet = synth.ricker(nt, p.dt, 1.5 / t0, t0=t0, shift=0.5)
    sp = np.array(p.spacing)
    off = np.array([[3.3, 0.4, 0.0], [-2.6, 1.7, 2.2], [0.5, -3.1, -2.4], [1.2, 2.8, 3.6]])
    p.rec_pos = p.src_pos + off * sp
    want, osim = orc.run_problem(p, return_sim=True)
    sim = ews.simulation_for(p)
    got = sim.run(nt, p.dt)
    assert np.abs(want).max() > 0
    assert rel(got, want) <= TOL, rel(got, want)
    check_state(sim.get_state(), osim.get_state())


def test_stability_bound_per_axis(ews):
    """The run is refused just above dt vp_max (7/3) sqrt(1/dx^2 + 1/dy^2 +
    1/dz^2) = 2 and accepted just below it: the per-axis form of the exact
    bound, not a bound from one spacing."""
    sp = SPACINGS[0]
    p = synth.small_problem(40, 36, 28, nt=20, boundary="sponge", kind="moment", width=5,
                            seed=3, spacing=sp)
    sim = ews.simulation_for(p)
    vmax = float(p.vp.astype(np.float64).max())
    limit = 2.0 / ((7.0 / 3.0) * vmax * np.sqrt(sum(1.0 / h ** 2 for h in sp)))
    assert limit > 6.0 / (7.0 * np.sqrt(3.0)) * min(sp) / vmax * 1.05   # not the cubic form
    with pytest.raises(ews.EwsError) as e:
        sim.run(10, limit * 1.001)
    assert e.value.status == ews.EWS_ECFL
    sim.run(10, limit * 0.999)


def test_one_step_full_size_unequal_spacing(ews, orc):
    """256^3 with C-PML 20 and spacings (20, 25, 15) m: one step from a
    seeded random state, every element of every field against the oracle
    (the benchmark's launch shape with per-axis C-PML profiles)."""
    p = synth.config2(nt=4)
    p.spacing = (20.0, 25.0, 15.0)
    p.src_pos = p.src_pos * np.array([1.0, 1.25, 0.75])
    p.rec_pos = p.rec_pos * np.array([1.0, 1.25, 0.75])
    p.dt = 0.9 * synth.PAPER_CFL * 15.0 / float(p.vp.max())
    st = synth.random_state(p.nx, p.ny, p.nz, seed=13)
    st[3:] *= 1e6
    sim = ews.simulation_for(p)
    sim.set_state(st)
    seis = np.zeros((3, sim.nrec, 1), np.float32)
    sim.advance(0, 1, p.dt, seis, 1)
    got = sim.get_state()
    o = orc.OracleSim(p.nx, p.ny, p.nz, p.spacing)
    o.set_medium_vel(p.vp, p.vs, p.rho)
    o.set_boundary("cpml", p.width, p.dt, p.f0)
    o.set_state(st)
    o.step_velocity(p.dt)
    want_seis = o.sample(p.rec_pos)
    o.step_stress(p.dt, "moment", p.src_pos, p.src_comp, p.wavelet[0])
    want = o.get_state()
    for q in range(9):
        err = np.abs(got[q] - want[q]).max() / np.abs(want[q]).max()
        assert err <= TOL, (q, err)
    assert rel(seis[:, :, 0], want_seis) <= TOL
