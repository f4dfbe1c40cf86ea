"""Parity at the large forward size (1024 x 1024 x 512, sponge 20), in the
launch configuration the benchmark times, on sampled outputs.

The FP64 oracle cannot hold this grid, but one time step is local: the new
wavefields of a cell depend only on the old state within 4 cells and on the
medium within 3.  So for sampled interior cells (away from the sponge) the
oracle runs the same step on the 9^3 block around the cell, and its centre
must equal the GPU step of the full grid.  Inputs (model and state) come
from torch's seeded generator, not from the CUDA path.
"""
import numpy as np
import pytest

from paper_2112_15071_gb300 import synth

pytestmark = pytest.mark.gpu

R = 4                     # block half-width: v needs sigma within 2, sigma needs v within 2


@pytest.fixture(scope="module")
def big():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_15071_gb300 import ews
    ews.load()
    dev = torch.device("cuda")
    p = synth.config3(nt=4, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(71)
    st = torch.randn((9, p.nz, p.ny, p.nx), generator=gen, device=dev)
    st[:3] *= 1e-3
    st[3:] *= 1e6
    rng = np.random.default_rng(5)
    lo = p.width + R
    cells = np.stack([rng.integers(lo, n - lo, 48) for n in (p.nz, p.ny, p.nx)], axis=1)
    yield ews, p, st, cells
    del st
    torch.cuda.empty_cache()


def oracle_centres(orc, p, st, cells):
    """The oracle's one-step result at the centre of each block."""
    out = np.zeros((len(cells), 9))
    for n, (k, j, i) in enumerate(cells):
        sl = (slice(k - R, k + R + 1), slice(j - R, j + R + 1), slice(i - R, i + R + 1))
        vp, vs, rho = (a[sl].double().cpu().numpy() for a in (p.vp, p.vs, p.rho))
        o = orc.OracleSim(2 * R + 1, 2 * R + 1, 2 * R + 1, p.spacing)
        o.set_medium_vel(vp, vs, rho)
        o.set_boundary("none")
        o.set_state(st[(slice(None),) + sl].double().cpu().numpy())
        o.step_velocity(p.dt)
        o.step_stress(p.dt)
        out[n] = o.get_state()[:, R, R, R]
    return out


def gpu_step(ews, p, st, storage, shape=None):
    """One step of the scheme (no source, no receivers) on the full grid."""
    import torch
    sim = ews.Simulation(p.nx, p.ny, p.nz, p.spacing, boundary=p.boundary, width=p.width,
                         storage=storage)
    if shape:
        sim.set_tile_shape(shape)
    sim.set_model_vel(p.vp, p.vs, p.rho)
    sim.set_state(st)
    sim.advance(0, 1, p.dt, None, 1)
    got = torch.empty_like(st)
    ews.ews_get_state(sim.handle, got)
    torch.cuda.synchronize()
    sim.close()
    return got


def test_fp32_step_at_full_size(big, orc):
    ews, p, st, cells = big
    got = gpu_step(ews, p, st, "f32")
    want = oracle_centres(orc, p, st, cells)
    scale = st.abs().amax(dim=(1, 2, 3)).double().cpu().numpy()
    g = got[:, cells[:, 0], cells[:, 1], cells[:, 2]].double().cpu().numpy().T
    err = np.abs(g - want) / scale
    assert err.max() <= 1e-5, err.max(axis=0)


def test_fused_step_at_full_size(big, orc):
    """The fused step (both passes in one launch, one z-chunk per tile at
    this size, the state copied back after the odd step): the sampled cells
    against the oracle, and every element against the two-pass step."""
    ews, p, st, cells = big
    got = gpu_step(ews, p, st, "f32", shape="fused")
    want = oracle_centres(orc, p, st, cells)
    scale = st.abs().amax(dim=(1, 2, 3)).double().cpu().numpy()
    g = got[:, cells[:, 0], cells[:, 1], cells[:, 2]].double().cpu().numpy().T
    err = np.abs(g - want) / scale
    assert err.max() <= 1e-5, err.max(axis=0)
    ref = gpu_step(ews, p, st, "f32", shape="32x8")
    d = ((got - ref).abs().amax(dim=(1, 2, 3)) / ref.abs().amax(dim=(1, 2, 3))).cpu().numpy()
    del got, ref
    assert d.max() <= 1e-6, d


def test_bf16_step_at_full_size(big, orc):
    """BF16 storage, state representable in BF16: the velocity pass equals the
    FP32 step rounded to BF16 (1 ulp), the stress pass agrees to a few ulps."""
    ews, p, st, cells = big
    import torch
    sb = st.to(torch.bfloat16).float()
    got = gpu_step(ews, p, sb, "bf16")
    want = oracle_centres(orc, p, sb, cells)
    g = got[:, cells[:, 0], cells[:, 1], cells[:, 2]].double().cpu().numpy().T
    rel = np.abs(g - want) / np.maximum(np.abs(want), 1e-30)
    assert np.all(rel[:, :3] <= 2.0 ** -8 * 1.01), rel[:, :3].max()
    scale = sb.abs().amax(dim=(1, 2, 3)).double().cpu().numpy()
    assert (np.abs(g - want) / scale)[:, 3:].max() <= 2.0 ** -8 * 4


def test_free_surface_step_at_bench_size(orc):
    """The free-surface forms of the passes at the size and boundary the
    benchmark times them (256^3, C-PML 20, surface at ks = 20 below the top
    slab): one step from a seeded random state; at sampled cells two to four
    planes below the surface (outside every C-PML slab, but fed by the
    switched planes), the oracle's step on the 9^3 block around each cell,
    with the surface at the same place in the block, matches the GPU."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_15071_gb300 import ews
    ews.load()
    dev = torch.device("cuda")
    p = synth.config2(n=256, nt=4)
    ks, eps = p.width, 1e-3
    gen = torch.Generator(device=dev)
    gen.manual_seed(73)
    st = torch.randn((9, p.nz, p.ny, p.nx), generator=gen, device=dev)
    st[:3] *= 1e-3
    st[3:] *= 1e6
    st[:, :ks] = 0.0                      # nothing above the surface
    sim = ews.Simulation(p.nx, p.ny, p.nz, p.spacing, boundary="cpml", width=p.width, f0=p.f0)
    sim.set_free_surface(ks, eps)
    sim.set_model_vel(p.vp, p.vs, p.rho)
    sim.set_state(st)
    sim.advance(0, 1, p.dt, None, 1)
    got = torch.empty_like(st)
    ews.ews_get_state(sim.handle, got)
    torch.cuda.synchronize()
    sim.close()
    rng = np.random.default_rng(6)
    lo, hi = p.width + R, p.nx - p.width - R
    cells = np.stack([rng.integers(ks + 2, ks + 5, 24), rng.integers(lo, hi, 24),
                      rng.integers(lo, hi, 24)], axis=1)
    want = np.zeros((len(cells), 9))
    for n, (k, j, i) in enumerate(cells):
        sl = (slice(k - R, k + R + 1), slice(j - R, j + R + 1), slice(i - R, i + R + 1))
        vp, vs, rho = (a[sl].astype(np.float64) for a in (p.vp, p.vs, p.rho))
        o = orc.OracleSim(2 * R + 1, 2 * R + 1, 2 * R + 1, p.spacing)
        o.set_free_surface(ks - (k - R), eps)
        o.set_medium_vel(vp, vs, rho)
        o.set_boundary("none")
        o.set_state(st[(slice(None),) + sl].double().cpu().numpy())
        o.step_velocity(p.dt)
        o.step_stress(p.dt)
        want[n] = o.get_state()[:, R, R, R]
    scale = st.abs().amax(dim=(1, 2, 3)).double().cpu().numpy()
    g = got[:, cells[:, 0], cells[:, 1], cells[:, 2]].double().cpu().numpy().T
    err = np.abs(g - want) / scale
    assert err.max() <= 1e-5, err.max(axis=0)
