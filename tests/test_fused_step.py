"""The fused time step (tile shape "fused"): the velocity pass (Eq. 1) and the
stress pass (Eq. 2/3) of a step in one launch, which reads one set of
wavefields and writes a second one, recomputing the new velocity of a 2-cell
ring around each tile.  The arithmetic per cell is that of the two passes, so
seismograms and wavefields equal the 32 x 8 passes to the rounding of
separately compiled code (FP32, 1e-6) and match the FP64 oracle -- on ragged
grids with partial tiles and z-chunks, with a sponge or no absorbing edge,
moment and force sources (the force added inside the step, also where its
taps straddle tiles and z-chunks), even and odd step counts (an odd count
ends with the state copied back), runs in chunks and snapshots.  Where it
does not apply (C-PML, 16-bit storage, free surface) the run falls back to
the 32 x 8 passes."""
import numpy as np
import pytest

from paper_2112_15071_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_SHAPE = 1e-6      # against the two-pass step (same arithmetic, FP32 rounding)
TOL_ORACLE = 1e-5     # against the FP64 oracle (the two-pass tolerance)


@pytest.fixture(scope="module")
def ews():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_15071_gb300 import ews as E
    E.load()
    yield E
    E.ews_tile_tuning_clear()


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run(ews, p, shape, **kw):
    sim = ews.simulation_for(p, **kw)
    sim.set_tile_shape(shape)
    seis = sim.run(p.nt, p.dt)
    assert sim.tile_shape == shape
    return seis, sim.get_state(), sim


@pytest.mark.parametrize("boundary", ["none", "sponge"])
@pytest.mark.parametrize("kind", ["moment", "force"])
@pytest.mark.parametrize("nt", [60, 61])
def test_fused_equals_the_two_passes(ews, boundary, kind, nt):
    p = synth.small_problem(70, 45, 37, nt=nt, boundary=boundary, kind=kind, width=6, seed=201)
    ref_seis, ref_state, _ = run(ews, p, "32x8")
    assert np.abs(ref_seis).max() > 0
    seis, state, sim = run(ews, p, "fused")
    assert rel(seis, ref_seis) <= TOL_SHAPE, rel(seis, ref_seis)
    for q in range(9):
        assert rel(state[q], ref_state[q]) <= TOL_SHAPE, q
    # one launch per step, no separate passes
    _, launches = sim.profile()
    assert launches[ews.EWS_KERNEL_VELOCITY] == 0 and launches[ews.EWS_KERNEL_STRESS] == 0


@pytest.mark.parametrize("kind", ["moment", "force"])
def test_fused_matches_the_oracle(ews, orc, kind):
    p = synth.small_problem(33, 65, 40, nt=120, boundary="sponge", kind=kind, width=6,
                            seed=202, spacing=(10.0, 14.0, 7.0))
    want, osim = orc.run_problem(p, return_sim=True)
    got, state, _ = run(ews, p, "fused")
    assert rel(got, want) <= TOL_ORACLE, rel(got, want)
    ost = osim.get_state()
    for q in range(9):
        assert rel(state[q], ost[q]) <= TOL_ORACLE, q


@pytest.mark.parametrize("kind", ["moment", "force"])
def test_one_fused_step_from_a_random_state(ews, orc, kind):
    """Every element of every field after one step from a seeded random state
    (all differences active everywhere, including the grid's edges and the
    tiles' rings) against the oracle."""
    p = synth.small_problem(70, 45, 37, nt=4, boundary="sponge", kind=kind, width=6, seed=203)
    st = synth.random_state(p.nx, p.ny, p.nz, seed=13)
    st[3:] *= 1e6
    sim = ews.simulation_for(p)
    sim.set_tile_shape("fused")
    sim.set_state(st)
    seis = np.zeros((3, sim.nrec, 1), np.float32)
    sim.advance(0, 1, p.dt, seis, 1)
    got = sim.get_state()
    o = orc.OracleSim(p.nx, p.ny, p.nz, p.spacing)
    o.set_medium_vel(p.vp, p.vs, p.rho)
    o.set_boundary("sponge", p.width, p.dt, p.f0)
    o.set_state(st)
    if kind == "force":
        o.step_velocity(p.dt, "force", p.src_pos, p.src_comp, p.wavelet[0])
        want_seis = o.sample(p.rec_pos)
        o.step_stress(p.dt)
    else:
        o.step_velocity(p.dt)
        want_seis = o.sample(p.rec_pos)
        o.step_stress(p.dt, "moment", p.src_pos, p.src_comp, p.wavelet[0])
    want = o.get_state()
    for q in range(9):
        err = np.abs(got[q] - want[q]).max() / np.abs(want[q]).max()
        assert err <= TOL_ORACLE, (q, err)
    assert rel(seis[:, :, 0], want_seis) <= TOL_ORACLE


@pytest.mark.parametrize("corner", [(31.6, 7.6, 18.6), (32.4, 8.4, 19.4), (1.3, 42.6, 34.6)])
def test_force_taps_across_tiles_and_z_chunks(ews, orc, corner):
    """A point force whose trilinear taps straddle a tile corner (x = 32,
    y = 8) and the z-chunk edge (37 planes in two chunks of 19), or sit at
    the grid's edge: every CTA whose ring holds a tap adds it, the owner
    alone writes it."""
    p = synth.small_problem(70, 45, 37, nt=50, boundary="none", kind="force", width=6, seed=204)
    p.src_pos = np.array(corner) * np.array(p.spacing)
    p.rec_pos = np.array([[31.5, 7.5, 18.5], [32.5, 8.5, 19.5], [10.0, 30.0, 5.0]]) * np.array(p.spacing)
    ref_seis, ref_state, _ = run(ews, p, "32x8")
    seis, state, _ = run(ews, p, "fused")
    assert rel(seis, ref_seis) <= TOL_SHAPE
    for q in range(9):
        assert rel(state[q], ref_state[q]) <= TOL_SHAPE, q
    want, osim = orc.run_problem(p, return_sim=True)
    assert rel(seis, want) <= TOL_ORACLE
    ost = osim.get_state()
    for q in range(9):
        assert rel(state[q], ost[q]) <= TOL_ORACLE, q


def test_odd_chunks_snapshots_and_replay(ews):
    p = synth.small_problem(40, 36, 28, nt=45, boundary="sponge", kind="force", width=5, seed=205)
    a, sa, sim = run(ews, p, "fused")
    # the captured loop replayed gives the same result
    assert np.array_equal(sim.run(p.nt, p.dt), a)
    # chunks of odd and even length continue from the state of the last one
    sim2 = ews.simulation_for(p)
    sim2.set_tile_shape("fused")
    b = np.zeros_like(a)
    for n0, k in ((0, 7), (7, 6), (13, 13), (26, 19)):
        sim2.advance(n0, k, p.dt, b, p.nt)
    assert np.array_equal(a, b)
    assert np.array_equal(sim2.get_state(), sa)
    # snapshots every 5 steps (odd chunks) equal those of the two passes
    mask = (1 << 0) | (1 << 4) | (1 << 8)
    snaps = {}
    for shape in ("32x8", "fused"):
        s = ews.simulation_for(p, snapshot_every=5, snapshot_mask=mask)
        s.set_tile_shape(shape)
        out = np.zeros((9, 3, p.nz, p.ny, p.nx), np.float32)
        s.run(p.nt, p.dt, snapshots=out)
        snaps[shape] = out
    assert np.abs(snaps["32x8"]).max() > 0
    for k in range(9):
        for m in range(3):
            assert rel(snaps["fused"][k, m], snaps["32x8"][k, m]) <= TOL_SHAPE, (k, m)


def test_fused_falls_back_where_it_does_not_apply(ews):
    cases = []
    cases.append((synth.small_problem(40, 36, 30, nt=20, boundary="cpml", width=5, seed=206), {}))
    cases.append((synth.small_problem(40, 36, 30, nt=20, boundary="sponge", width=5, seed=207),
                  {"storage": "bf16"}))
    q = synth.small_problem(40, 36, 30, nt=20, boundary="sponge", width=5, seed=208)
    q.free_surface = (6, 1e-3)
    cases.append((q, {}))
    for p, kw in cases:
        sim = ews.simulation_for(p, **kw)
        sim.set_tile_shape("fused")
        got = sim.run(p.nt, p.dt)
        assert sim.tile_shape == "32x8"
        ref = ews.simulation_for(p, **kw)
        ref.set_tile_shape("32x8")
        assert np.array_equal(got, ref.run(p.nt, p.dt))


def test_tuner_keeps_the_second_set_only_when_it_picks_fused(ews):
    p = synth.small_problem(64, 48, 40, nt=30, boundary="sponge", kind="moment", width=6,
                            seed=209)
    field = 4 * ((p.nx + 31) // 32 * 32) * p.ny * p.nz
    base = ews.ews_memory_in_use()
    s8 = ews.simulation_for(p)
    s8.set_tile_shape("32x8")
    want = s8.run(p.nt, p.dt)
    d8 = ews.ews_memory_in_use() - base
    s8.close()
    assert ews.ews_memory_in_use() == base
    ews.ews_tile_tuning_clear()
    sim = ews.simulation_for(p)                           # automatic shape
    got = sim.run(p.nt, p.dt)
    d = ews.ews_memory_in_use() - base
    tuned = ews.ews_tile_tuned(ews.ews_grid(p.nx, p.ny, p.nz, *p.spacing), "sponge", "f32")
    assert tuned in (ews.EWS_TILE_32X8, ews.EWS_TILE_32X4, ews.EWS_TILE_32X16, ews.EWS_TILE_FUSED)
    assert d == d8 + (9 * field if tuned == ews.EWS_TILE_FUSED else 0)
    assert rel(got, want) <= TOL_SHAPE
    sim.close()
    assert ews.ews_memory_in_use() == base
    # an imported entry makes the next simulation take the fused step
    ews.ews_tile_tuning_import([{"nx": p.nx, "ny": p.ny, "nz": p.nz, "boundary": "sponge",
                                 "storage": "f32", "shape": "fused"}])
    sim = ews.simulation_for(p)
    assert rel(sim.run(p.nt, p.dt), want) <= TOL_SHAPE
    assert sim.tile_shape == "fused"
