"""The library's device-memory accounting and its optional cap
(ews_set_memory_limit): a call whose allocations would exceed the cap
returns EWS_ENOMEM without asking CUDA, releases what it had set up, and
leaves the other simulations and the CUDA context usable -- the same path a
full device takes, exercised here without a failing device allocation."""
import numpy as np
import pytest

from paper_2112_15071_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ews():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_15071_gb300 import ews as E
    E.load()
    yield E
    E.ews_set_memory_limit(-1)


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_accounting_follows_create_and_destroy(ews):
    base = ews.ews_memory_in_use()
    p = synth.small_problem(40, 36, 28, nt=20, boundary="cpml", width=5, seed=3)
    sim = ews.simulation_for(p)
    sim.run(p.nt, p.dt)
    held = ews.ews_memory_in_use()
    pitch = (p.nx + 31) // 32 * 32
    # at least the 9 wavefields, 3 medium arrays and 18 C-PML arrays
    assert held - base >= (9 + 3 + 18) * 4 * pitch * p.ny * p.nz
    sim.close()
    assert ews.ews_memory_in_use() == base


def test_capped_create_and_gradient_return_enomem(ews):
    p = synth.small_problem(40, 36, 28, nt=60, boundary="sponge", width=5, seed=4)
    sim = ews.simulation_for(p)
    want = sim.run(p.nt, p.dt)
    obs = (want * 1.1).astype(np.float32)
    held = ews.ews_memory_in_use()
    try:
        ews.ews_set_memory_limit(held + (1 << 20))
        assert ews.ews_memory_limit() == held + (1 << 20)
        with pytest.raises(ews.EwsError) as e:          # ~100 MB of wavefields and medium
            ews.Simulation(128, 128, 128, (10.0, 10.0, 10.0), boundary="sponge", width=8)
        assert e.value.status == ews.EWS_ENOMEM
        assert "memory limit" in str(e.value)
        assert ews.ews_memory_in_use() == held       # the partial set-up was released
        # the existing simulation still runs, with the same result
        assert np.array_equal(sim.run(p.nt, p.dt), want)
        # the gradient's adjoint state and checkpoints do not fit under the cap
        with pytest.raises(ews.EwsError) as e:
            sim.gradient(p.nt, p.dt, obs, ckpt_every=20)
        assert e.value.status == ews.EWS_ENOMEM
        assert np.array_equal(sim.run(p.nt, p.dt), want)
    finally:
        ews.ews_set_memory_limit(-1)
    # without the cap the same simulation computes the gradient a fresh one does
    m1, g1 = sim.gradient(p.nt, p.dt, obs, ckpt_every=20)
    fresh = ews.simulation_for(p)
    m2, g2 = fresh.gradient(p.nt, p.dt, obs, ckpt_every=20)
    assert m1 == pytest.approx(m2, rel=1e-6)
    for q in range(3):
        assert rel(g1[q], g2[q]) <= 1e-6


def test_history_budget_stays_under_the_cap(ews):
    """With the automatic history budget, a cap that leaves room for the
    checkpoints but not for the whole velocity history makes the gradient
    recompute segments instead of failing, and the result is unchanged."""
    p = synth.small_problem(40, 36, 28, nt=120, boundary="sponge", width=5, seed=6)
    obs = (ews.simulation_for(p).run(p.nt, p.dt) * 0.9).astype(np.float32)
    ref = ews.simulation_for(p)
    m0, g0 = ref.gradient(p.nt, p.dt, obs, ckpt_every=20)   # history resident
    sim = ews.simulation_for(p)
    sim.run(p.nt, p.dt)
    pitch = (p.nx + 31) // 32 * 32
    field = 4 * pitch * p.ny * p.nz
    # adjoint state (17 FP32 + 8 FP64 fields), 6 checkpoints of 9 fields,
    # 40 history slots of 3 fields (the full history needs 121), staging
    room = (17 + 16 + 6 * 9 + 40 * 3 + 3) * field + (1 << 20)
    try:
        ews.ews_set_memory_limit(ews.ews_memory_in_use() + room)
        m1, g1 = sim.gradient(p.nt, p.dt, obs, ckpt_every=20)
        assert ews.ews_memory_in_use() <= ews.ews_memory_limit()
    finally:
        ews.ews_set_memory_limit(-1)
    assert m1 == pytest.approx(m0, rel=1e-6)
    for q in range(3):
        assert rel(g1[q], g0[q]) <= 1e-5


def test_capped_batch_returns_enomem(ews):
    import torch
    probs = [synth.small_problem(40, 36, 28, nt=40, boundary="sponge", width=5, seed=7 + i)
             for i in range(2)]
    shots = []
    for p in probs:
        d = {"sim": ews.simulation_for(p), "nt": p.nt, "dt": p.dt,
             "seis": torch.zeros((3, p.rec_pos.shape[0], p.nt), device="cuda"),
             "observed": torch.zeros((3, p.rec_pos.shape[0], p.nt), device="cuda")}
        for k in ("g_lam", "g_mu", "g_rho"):
            d[k] = torch.zeros((p.nz, p.ny, p.nx), device="cuda")
        shots.append(d)
    try:
        ews.ews_set_memory_limit(ews.ews_memory_in_use())
        with pytest.raises(ews.EwsError) as e:
            ews.ews_batch(shots, ckpt_every=20)
        assert e.value.status == ews.EWS_ENOMEM
    finally:
        ews.ews_set_memory_limit(-1)
    ews.ews_batch(shots, ckpt_every=20)
    torch.cuda.synchronize()
    for p, d in zip(probs, shots):
        want = ews.simulation_for(p).run(p.nt, p.dt)
        assert rel(d["seis"].cpu().numpy(), want) <= 1e-6


def test_gradient_batch_runs_in_waves_under_the_limit(ews):
    """Three gradient shots whose gradient state fits the limit two at a time
    but not three at once: ews_batch splits them into waves (the forward shot
    rides with the first) and gives the results of the one-by-one path, which
    itself releases earlier shots' gradient state when it needs the room."""
    import torch
    probs = [synth.small_problem(40, 36, 28, nt=60, boundary="sponge", width=5, seed=20 + i,
                                 kind=("moment", "force")[i % 2]) for i in range(4)]
    rng = np.random.default_rng(3)

    def shots():
        out = []
        for i, p in enumerate(probs):
            sim = ews.simulation_for(p)
            sim.set_history_budget(0)                  # one segment of history per shot
            d = {"sim": sim, "nt": p.nt, "dt": p.dt,
                 "seis": torch.zeros((3, p.rec_pos.shape[0], p.nt), device="cuda")}
            if i < 3:
                obs = rng.standard_normal((3, p.rec_pos.shape[0], p.nt)).astype(np.float32) * 1e-9
                d["observed"] = torch.from_numpy(obs).cuda()
                for k in ("g_lam", "g_mu", "g_rho"):
                    d[k] = torch.zeros((p.nz, p.ny, p.nx), device="cuda")
            out.append(d)
        return out

    rng = np.random.default_rng(3)
    a = shots()
    rng = np.random.default_rng(3)
    b = shots()
    torch.cuda.synchronize()
    pitch = (probs[0].nx + 31) // 32 * 32
    field = 4 * pitch * probs[0].ny * probs[0].nz
    # per gradient shot: 17 FP32 + 8 FP64 adjoint fields, 2 checkpoints of 9
    # fields, 21 history slots of 3 fields, seismogram buffers: ~120 fields
    per_shot = (17 + 16 + 18 + 63 + 4) * field
    try:
        ews.ews_set_memory_limit(ews.ews_memory_in_use() + 2.5 * per_shot)
        ma = ews.ews_batch(a, ckpt_every=20)
        torch.cuda.synchronize()
        for d in a:                                    # the last wave's state
            d["sim"].release_workspace()
        mb = ews.ews_batch(b, ckpt_every=20, mode=ews.EWS_BATCH_SEQUENTIAL)
        torch.cuda.synchronize()
    finally:
        ews.ews_set_memory_limit(-1)
    for i in range(4):
        assert rel(a[i]["seis"].cpu().numpy(), b[i]["seis"].cpu().numpy()) <= 1e-6, i
        if i < 3:
            assert ma[i] == pytest.approx(mb[i], rel=1e-6)
            for k in ("g_lam", "g_mu", "g_rho"):
                assert rel(a[i][k].cpu().numpy(), b[i][k].cpu().numpy()) <= 1e-5, (i, k)
