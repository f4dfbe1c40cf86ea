"""Batched shots in one persistent launch (ews_batch).

The executor runs the same stencil, source, receiver and adjoint work items
as ews_run / ews_gradient, scheduled by per-shot dependency counters; so
each shot's seismograms and gradients must agree with the one-by-one path
(the forward up to FP32 rounding order of separately compiled copies of the
same arithmetic; the gradient to accumulation order), for uneven shot sizes
and step counts, any number of resident CTAs and any z-chunk.  A dependency
that can never be met ends in EWS_ETIMEOUT after the bounded wait, and the
context stays usable.
"""
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
    return E


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def shots_for(ews, probs, grad=False, obs=None):
    import torch
    out = []
    for i, p in enumerate(probs):
        sim = ews.simulation_for(p)
        d = {"sim": sim, "nt": p.nt, "dt": p.dt,
             "seis": torch.zeros((3, p.rec_pos.shape[0], p.nt), device="cuda")}
        if grad:
            d["observed"] = torch.from_numpy(obs[i]).cuda()
            for k in ("g_lam", "g_mu", "g_rho"):
                d[k] = torch.zeros((p.nz, p.ny, p.nx), device="cuda")
        out.append(d)
    return out


def problems(kinds=("moment", "force", "moment"), nts=(70, 45, 90)):
    dims = [(40, 36, 28), (70, 45, 37), (33, 65, 40)]
    return [synth.small_problem(*dims[i], nt=nts[i], boundary="sponge", width=5, kind=kinds[i],
                                nrec=6, seed=30 + i) for i in range(len(kinds))]


@pytest.mark.parametrize("zchunk,ctas", [(0, 0), (8, 1), (13, 2), (64, 0)])   # 64: whole columns
def test_forward_batch_matches_run(ews, zchunk, ctas):
    import torch
    probs = problems()
    shots = shots_for(ews, probs)
    ews.ews_batch(shots, zchunk=zchunk, ctas_per_sm=ctas)
    torch.cuda.synchronize()
    for p, d in zip(probs, shots):
        want = ews.simulation_for(p).run(p.nt, p.dt)
        got = d["seis"].cpu().numpy()
        assert rel(got, want) <= 1e-6, rel(got, want)
        # the batched run leaves the shot's final state in its simulation
        ref = ews.simulation_for(p)
        ref.run(p.nt, p.dt)
        assert rel(d["sim"].get_state(), ref.get_state()) <= 1e-6


def test_gradient_batch_matches_one_by_one(ews, orc):
    import torch
    probs = problems(kinds=("moment", "force"), nts=(60, 75))
    rng = np.random.default_rng(2)
    obs = [(orc.run_problem(p) * (1 + 0.2 * rng.standard_normal((3, p.rec_pos.shape[0], p.nt))))
           .astype(np.float32) for p in probs]
    a = shots_for(ews, probs, grad=True, obs=obs)
    b = shots_for(ews, probs, grad=True, obs=obs)
    a[1]["sim"].set_history_budget(0)         # one shot recomputes its segments
    ma = ews.ews_batch(a, ckpt_every=20)
    mb = ews.ews_batch(b, mode=ews.EWS_BATCH_SEQUENTIAL, ckpt_every=20)
    torch.cuda.synchronize()
    for i in range(len(probs)):
        assert ma[i] == pytest.approx(mb[i], rel=1e-6)
        assert rel(a[i]["seis"].cpu().numpy(), b[i]["seis"].cpu().numpy()) <= 1e-6
        for k in ("g_lam", "g_mu", "g_rho"):
            assert rel(a[i][k].cpu().numpy(), b[i][k].cpu().numpy()) <= 1e-5, (i, k)
    # and against the FP64 adjoint of the oracle for the first shot
    p = probs[0]
    seis = orc.run_problem(p)
    want = orc.gradient(p, p.dt * (seis - obs[0].astype(np.float64)), ckpt_every=20)
    for q, k in enumerate(("g_lam", "g_mu", "g_rho")):
        assert rel(a[0][k].cpu().numpy(), want[q]) <= 1e-4


def test_mixed_forward_and_gradient_shots(ews, orc):
    import torch
    probs = problems(kinds=("moment", "force"), nts=(50, 40))
    obs = [orc.run_problem(probs[0]).astype(np.float32) * 1.1]
    shots = shots_for(ews, probs[:1], grad=True, obs=obs) + shots_for(ews, probs[1:])
    ews.ews_batch(shots, ckpt_every=16)
    torch.cuda.synchronize()
    want = ews.simulation_for(probs[1]).run(probs[1].nt, probs[1].dt)
    assert rel(shots[1]["seis"].cpu().numpy(), want) <= 1e-6
    sim = ews.simulation_for(probs[0])
    mis, g = sim.gradient(probs[0].nt, probs[0].dt, obs[0], ckpt_every=16)
    for q, k in enumerate(("g_lam", "g_mu", "g_rho")):
        assert rel(shots[0][k].cpu().numpy(), g[q]) <= 1e-5


def test_validation(ews):
    p = problems()[0]
    a = ews.simulation_for(p)
    c = synth.small_problem(40, 36, 28, nt=20, boundary="cpml", width=5)
    with pytest.raises(ews.EwsError) as e:
        ews.ews_batch([{"sim": a, "nt": p.nt, "dt": p.dt}, {"sim": a, "nt": p.nt, "dt": p.dt}])
    assert e.value.status == ews.EWS_EINVAL
    import torch
    cobs = torch.zeros((3, c.rec_pos.shape[0], c.nt), device="cuda")
    cg = {k: torch.zeros((c.nz, c.ny, c.nx), device="cuda") for k in ("g_lam", "g_mu", "g_rho")}
    with pytest.raises(ews.EwsError) as e:           # no C-PML adjoint
        ews.ews_batch([dict({"sim": ews.simulation_for(c), "nt": c.nt, "dt": c.dt,
                             "observed": cobs}, **cg)])
    assert e.value.status == ews.EWS_EINVAL
    with pytest.raises(ews.EwsError) as e:
        ews.ews_batch([{"sim": a, "nt": p.nt, "dt": p.dt * 10}])
    assert e.value.status == ews.EWS_ECFL


def test_unsatisfiable_dependency_times_out(ews):
    """The last item waits for an item that never exists: the bounded wait
    gives up, every CTA leaves, the call returns EWS_ETIMEOUT, and the next
    batch on the same context runs normally."""
    import torch
    probs = problems(nts=(10, 10, 10))
    shots = shots_for(ews, probs)
    with pytest.raises(ews.EwsError) as e:
        ews.ews_batch(shots, zchunk=16, dep_wait_ms=200, test_unsatisfiable=True)
    assert e.value.status == ews.EWS_ETIMEOUT
    shots = shots_for(ews, probs)
    ews.ews_batch(shots, zchunk=16)
    torch.cuda.synchronize()
    want = ews.simulation_for(probs[0]).run(probs[0].nt, probs[0].dt)
    assert rel(shots[0]["seis"].cpu().numpy(), want) <= 1e-6


def test_batched_gradient_with_bf16_checkpoints(ews):
    """BF16 checkpoints in the batched executor (every segment recomputed)
    give the one-by-one BF16-checkpoint gradient: a power-of-two scale does
    not change BF16 rounding, so the unscaled batched form and the scaled
    single-shot form store the same values."""
    import torch
    probs = problems(nts=(60, 45, 70))
    rng = np.random.default_rng(9)
    obs = [rng.standard_normal((3, p.rec_pos.shape[0], p.nt)).astype(np.float32) * 1e-3
           for p in probs]
    runs = []
    for mode in (ews.EWS_BATCH_PERSISTENT, ews.EWS_BATCH_SEQUENTIAL):
        shots = shots_for(ews, probs, grad=True, obs=obs)
        for d in shots:
            d["sim"].set_checkpoint_storage("bf16")
            d["sim"].set_history_budget(0)
        ews.ews_batch(shots, ckpt_every=15, mode=mode)
        torch.cuda.synchronize()
        runs.append(shots)
    f32 = shots_for(ews, probs, grad=True, obs=obs)
    for d in f32:
        d["sim"].set_history_budget(0)
    ews.ews_batch(f32, ckpt_every=15)
    torch.cuda.synchronize()
    a, b = runs
    for i in range(len(probs)):
        for k in ("g_lam", "g_mu", "g_rho"):
            assert rel(a[i][k].cpu().numpy(), b[i][k].cpu().numpy()) <= 1e-5, (i, k)
            e = rel(a[i][k].cpu().numpy(), f32[i][k].cpu().numpy())
            assert 0 < e <= 3e-2, (i, k, e)


@pytest.mark.parametrize("zchunk", [0, 11])
def test_cpml_forward_batch_matches_run(ews, zchunk):
    """C-PML shots in the executor (memory-variable buffer per item, memory
    variables zeroed by the first stage) match the one-by-one path."""
    import torch
    dims = [(40, 36, 28), (70, 45, 37), (33, 65, 40)]
    probs = [synth.small_problem(*dims[i], nt=(60, 45, 70)[i], boundary="cpml", width=6,
                                 kind=("moment", "force", "moment")[i], nrec=6, seed=40 + i)
             for i in range(3)]
    shots = shots_for(ews, probs)
    ews.ews_batch(shots, zchunk=zchunk)
    torch.cuda.synchronize()
    for p, d in zip(probs, shots):
        want = ews.simulation_for(p).run(p.nt, p.dt)
        assert rel(d["seis"].cpu().numpy(), want) <= 1e-6, rel(d["seis"].cpu().numpy(), want)
    # a second batch on the same simulations starts from rest again
    shots2 = [dict(d, seis=torch.zeros_like(d["seis"])) for d in shots]
    ews.ews_batch(shots2, zchunk=zchunk)
    torch.cuda.synchronize()
    for d, e in zip(shots, shots2):
        assert rel(e["seis"].cpu().numpy(), d["seis"].cpu().numpy()) <= 1e-7


def test_imported_tuning_is_used_without_retuning(ews, tmp_path):
    """A table written by save_batch_tuning and read back by
    load_batch_tuning serves ews_batch with zchunk = 0: no grid is tuned
    again (the table is unchanged afterwards) and the results still match
    the one-by-one path."""
    import torch
    probs = problems()[:2]
    forced = [{"nx": p.nx, "ny": p.ny, "nz": p.nz, "boundary": "sponge", "free_surface": False,
               "zchunk": 12} for p in probs]
    path = str(tmp_path / "tuning.json")
    ews.ews_batch_tuning_clear()
    ews.ews_batch_tuning_import(forced)
    assert ews.save_batch_tuning(path) == 2
    ews.ews_batch_tuning_clear()
    try:
        assert ews.load_batch_tuning(path) == 2
        shots = shots_for(ews, probs)
        ews.ews_batch(shots)
        torch.cuda.synchronize()
        key = lambda e: (e["nx"], e["ny"], e["nz"])
        assert sorted(ews.ews_batch_tuning_export(), key=key) == sorted(forced, key=key)
        for p, d in zip(probs, shots):
            want = ews.simulation_for(p).run(p.nt, p.dt)
            assert rel(d["seis"].cpu().numpy(), want) <= 1e-6
    finally:
        ews.ews_batch_tuning_clear()
