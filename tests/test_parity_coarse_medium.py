"""GPU parity of the coarse medium grid (Sec. 2.2.1: medium textures
smaller than the wavefield textures, read with trilinear interpolation;
reading R17) against the FP64 oracle.

The passes' coarse-medium form samples lambda, mu and rho at every
staggered point from the medium grid instead of loading medium tiles of the
wavefield grid.  Bar: FP32 seismograms and wavefields within 1e-5 relative
L2 of the oracle, as for the plain forward.
"""
import numpy as np
import pytest

from paper_2112_15071_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


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


def coarse_problem(dims, m, boundary, kind, nt=90, seed=81):
    p = synth.small_problem(*dims, nt=nt, boundary=boundary, width=5, kind=kind, nrec=6,
                            seed=seed, layered=False)
    # layer speeds of the coarse recipe within the problem's CFL speed
    return synth.with_coarse_medium(p, m, seed=seed, layer_vp=(2400.0, 2700.0, 2950.0))


@pytest.mark.parametrize("boundary", ["none", "sponge", "cpml"])
@pytest.mark.parametrize("kind", ["moment", "force"])
@pytest.mark.parametrize("dims,m", [((70, 45, 37), (9, 7, 5)), ((33, 65, 40), (33, 13, 16)),
                                    ((40, 36, 28), (1, 5, 1))])
def test_coarse_forward_matches_oracle(ews, orc, boundary, kind, dims, m):
    p = coarse_problem(dims, m, boundary, kind)
    want, osim = orc.run_problem(p, return_sim=True)
    sim = ews.simulation_for(p)
    got = sim.run(p.nt, p.dt)
    assert np.abs(want).max() > 0
    assert rel(got, want) <= TOL, rel(got, want)
    st, ost = sim.get_state(), osim.get_state()
    for q in range(9):
        if np.linalg.norm(ost[q]) > 0:
            assert rel(st[q], ost[q]) <= TOL, (q, rel(st[q], ost[q]))


def test_same_resolution_equals_fine_path(ews):
    """A medium grid equal to the wavefield grid gives the fine path's
    result (the interpolation at half offsets is the cell means)."""
    p = synth.small_problem(48, 40, 36, nt=80, boundary="sponge", width=5, seed=90)
    lam, mu, rho = p.lame()
    fine = ews.simulation_for(p).run(p.nt, p.dt)
    sim = ews.simulation_for(p)
    sim.set_model_coarse(lam, mu, rho)
    got = sim.run(p.nt, p.dt)
    assert rel(got, fine) <= 1e-6, rel(got, fine)


@pytest.mark.parametrize("storage,cap", [("bf16", 3e-2), ("f16", 5e-3)])
def test_coarse_16bit_storage(ews, orc, storage, cap):
    p = coarse_problem((48, 40, 40), (12, 10, 10), "sponge", "moment", nt=150)
    want = orc.run_problem(p)
    got = ews.simulation_for(p, storage=storage).run(p.nt, p.dt)
    e = rel(got, want)
    print(f"\ncoarse medium, {storage} storage: rel L2 {e:.2e}")
    assert e <= cap, e


def test_coarse_validation(ews):
    import torch
    p = coarse_problem((40, 36, 30), (8, 8, 6), "sponge", "moment", nt=10)
    sim = ews.simulation_for(p)
    lam, mu, rho = p.coarse_medium
    bad = rho.copy()
    bad[1, 2, 3] = -1.0
    with pytest.raises(ews.EwsError) as e:
        sim.set_model_coarse(lam, mu, bad)
    assert e.value.status == ews.EWS_EINVAL
    with pytest.raises(ews.EwsError) as e:
        sim.run(p.nt, p.dt)                       # the failed upload leaves no model
    assert e.value.status == ews.EWS_ESTATE
    sim.set_model_coarse(lam, mu, rho)
    sim.run(p.nt, p.dt)
    with pytest.raises(ews.EwsError) as e:
        sim.set_free_surface(8, 1e-3)
    assert e.value.status == ews.EWS_EINVAL
    obs = torch.zeros((3, p.rec_pos.shape[0], p.nt), device="cuda")
    g = [torch.zeros((p.nz, p.ny, p.nx), device="cuda") for _ in range(3)]
    with pytest.raises(ews.EwsError) as e:
        ews.ews_gradient(sim.handle, p.nt, p.dt, obs, *g)
    assert e.value.status == ews.EWS_EINVAL
    with pytest.raises(ews.EwsError) as e:
        ews.ews_batch([{"sim": sim, "nt": p.nt, "dt": p.dt}])
    assert e.value.status == ews.EWS_EINVAL
    # back to the wavefield-grid medium
    sim.set_model_vel(p.vp, p.vs, p.rho)
    sim.run(p.nt, p.dt)


def test_coarse_grid_releases_the_cell_medium(ews):
    """With a coarse grid the wavefield grid's medium arrays (3 floats per
    cell) are released, and allocated again for a wavefield-grid medium."""
    import torch
    p = synth.config2(n=192, nt=4)
    sim = ews.simulation_for(p)
    sim.run(p.nt, p.dt)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    synth.with_coarse_medium(p, (48, 48, 48))
    sim.set_model_coarse(*p.coarse_medium)
    sim.run(p.nt, p.dt)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    cells = p.nx * p.ny * p.nz
    assert free1 - free0 >= 0.9 * 3 * 4 * cells, (free1 - free0) / (12 * cells)
    sim.set_model_vel(p.vp, p.vs, p.rho)
    sim.run(p.nt, p.dt)
