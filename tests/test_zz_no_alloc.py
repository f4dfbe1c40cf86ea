"""The forward run that allocates nothing (ews_forward_noalloc).

Callers whose device memory is owned by someone else -- a framework's
caching allocator, a fixed pool in a long-running service -- or that cannot
take the device-wide synchronisation of cudaFree, cannot let the library
call cudaMalloc.  For them ews_forward_noalloc keeps all working state in one
static device array.  These tests run it twice in a row through the C ABI, on
two different problems, and check each result against the regular
ews_create / ews_run path within the parity tolerance used everywhere else
(relative L2 1e-5); check that a call leaves the device's free memory
unchanged; and run it at its size limits against the FP64 oracle.  They live
in a file of its own that pytest collects last.
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


def regular_run(E, p):
    import torch
    sim = E.simulation_for(p)
    seis = torch.zeros((3, sim.nrec, p.nt), device="cuda")
    sim.run(p.nt, p.dt, seis)
    torch.cuda.synchronize()
    out = seis.cpu().numpy()
    sim.close()
    return out


def noalloc_inputs(E, p):
    """Device copies of the caller-owned inputs and a NaN-filled output."""
    import torch
    dev = torch.device("cuda")
    lam, mu, rho = (torch.from_numpy(a).to(dev) for a in p.lame())
    wav = torch.from_numpy(p.wavelet).to(dev)
    seis = torch.full((3, p.rec_pos.shape[0], p.nt), float("nan"), device=dev)
    grid = E.ews_grid(p.nx, p.ny, p.nz, *p.spacing)
    opt = E.ews_options(E.BOUNDARY[p.boundary], p.width, 0, 0, 0, 0.0, 0.0, p.f0)
    torch.cuda.synchronize()
    return grid, opt, lam, mu, rho, wav, seis


def noalloc_call(E, p, inputs):
    grid, opt, lam, mu, rho, wav, seis = inputs
    E.ews_forward_noalloc(grid, opt, lam, mu, rho, E.SOURCE[p.src_kind], p.src_pos, p.src_comp,
                          wav, p.rec_pos, p.nt, p.dt, seis)


def noalloc_run(E, p):
    import torch
    inputs = noalloc_inputs(E, p)
    noalloc_call(E, p, inputs)
    torch.cuda.synchronize()
    return inputs[-1].cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(a.astype(np.float64) - b) / np.linalg.norm(b))


def test_two_calls_in_a_row_match_the_regular_path(ews):
    first = synth.small_problem(40, 36, 28, nt=90, boundary="sponge", width=6, kind="moment",
                                seed=5)
    second = synth.small_problem(33, 45, 30, nt=70, boundary="none", width=6, kind="force",
                                 seed=9)
    want1 = regular_run(ews, first)
    want2 = regular_run(ews, second)
    got1 = noalloc_run(ews, first)
    got2 = noalloc_run(ews, second)
    assert np.all(np.isfinite(got1)) and np.all(np.isfinite(got2))
    assert np.abs(want1).max() > 0 and np.abs(want2).max() > 0
    assert rel_l2(got1, want1) <= TOL, rel_l2(got1, want1)
    # the shared array held the first run's wavefields; the second call must
    # not see them
    assert rel_l2(got2, want2) <= TOL, rel_l2(got2, want2)
    # and running the first problem again gives its answer again
    assert rel_l2(noalloc_run(ews, first), want1) <= TOL


def test_no_device_memory_is_allocated(ews):
    """The property the entry point exists for: with the caller's buffers in
    place and after a first call (which looks up the static array and loads
    the kernels), a further call leaves the device's free memory unchanged
    and the library's allocation count at zero growth."""
    import torch
    p = synth.small_problem(40, 36, 28, nt=60, boundary="sponge", width=6, kind="force", seed=12)
    inputs = noalloc_inputs(ews, p)
    noalloc_call(ews, p, inputs)
    torch.cuda.synchronize()
    first = inputs[-1].cpu().numpy()
    free0, _ = torch.cuda.mem_get_info()
    held0 = ews.ews_memory_in_use()
    noalloc_call(ews, p, inputs)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert ews.ews_memory_in_use() == held0
    assert np.array_equal(inputs[-1].cpu().numpy(), first)


def test_at_the_size_limits_against_the_oracle(ews, orc):
    """64^3 is exactly EWS_NOALLOC_MAX_CELLS padded cells (x pitch 64), with
    EWS_NOALLOC_MAX_RECEIVERS receivers: seismograms within the parity bar of
    the FP64 oracle."""
    assert 64 * 64 * 64 == 1 << 18
    p = synth.small_problem(64, 64, 64, nt=80, boundary="sponge", width=8, kind="moment",
                            seed=21, nrec=64)
    want = orc.run_problem(p)
    got = noalloc_run(ews, p)
    assert np.abs(want).max() > 0
    assert rel_l2(got, want) <= TOL, rel_l2(got, want)


def test_limits_are_enforced(ews):
    big = synth.small_problem(96, 64, 48, nt=4, boundary="sponge", width=6)   # 96*64*48 > 2^18
    with pytest.raises(ews.EwsError) as e:
        noalloc_run(ews, big)
    assert e.value.status == ews.EWS_EINVAL
    assert "no-allocation limit" in str(e.value)
    over = synth.small_problem(65, 64, 64, nt=4, boundary="sponge", width=6)   # pitch 96
    with pytest.raises(ews.EwsError) as e:
        noalloc_run(ews, over)
    assert e.value.status == ews.EWS_EINVAL
    many = synth.small_problem(40, 36, 28, nt=4, boundary="sponge", width=6, nrec=65)
    with pytest.raises(ews.EwsError) as e:
        noalloc_run(ews, many)
    assert e.value.status == ews.EWS_EINVAL
    assert "limit" in str(e.value)
    cp = synth.small_problem(40, 36, 28, nt=4, boundary="cpml", width=6)
    with pytest.raises(ews.EwsError) as e:
        noalloc_run(ews, cp)
    assert e.value.status == ews.EWS_EINVAL
