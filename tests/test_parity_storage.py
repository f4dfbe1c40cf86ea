"""Reduced-precision wavefield storage (BF16 / FP16 with per-field scales).

The paper keeps every field in float textures (Sec. 3), so storage in 16
bits is an addition whose error is measured, not bounded.  These tests pin
what is exact about it and measure the rest against the FP64 oracle:

* state I/O rounds exactly like torch's round-to-nearest-even casts, with the
  per-field power-of-two scale applied exactly;
* one velocity pass from a state representable in the storage type equals
  the FP32 pass rounded to that type (to 1 unit in the last place), so the
  16-bit tile layouts, halo offsets and scale algebra are right; the stress
  pass of the same step agrees with FP32 to the storage precision;
* whole-run seismogram error against the oracle (FP32 storage stays within
  the 1e-5 parity bound; BF16 / FP16 errors are printed and kept under a
  loose cap that catches a broken path);
* FP16 overflow is reported as EWS_ERANGE, never silently stored.
"""
import numpy as np
import pytest

from paper_2112_15071_gb300 import synth

pytestmark = pytest.mark.gpu

TDTYPE = {"bf16": "bfloat16", "f16": "float16"}
MANT = {"bf16": 8, "f16": 11}          # significand bits incl. the implicit one


@pytest.fixture(scope="module")
def ews():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_15071_gb300 import ews as E
    E.load()
    return E


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def round_to(x, storage, scale):
    """x stored with `scale` in `storage` and read back (torch RNE casts)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, np.float32))
    s = torch.from_numpy(np.asarray(scale, np.float32)).reshape(-1, *([1] * (t.dim() - 1)))
    return ((t * s).to(getattr(torch, TDTYPE[storage])).float() / s).numpy()


def ulp(x, storage, scale):
    """One unit in the last place of each stored value, in field units."""
    s = np.asarray(scale, np.float64).reshape(-1, *([1] * (np.ndim(x) - 1)))
    y = np.abs(np.asarray(x, np.float64) * s)
    e = np.floor(np.log2(np.maximum(y, 1e-30)))
    emin = -126 if storage == "bf16" else -14
    e = np.maximum(e, emin)
    return np.ldexp(1.0, (e - (MANT[storage] - 1)).astype(int)) / s


def bare_sim(ews, p, storage, scales=None):
    """Simulation with the problem's medium and receivers but no source."""
    sim = ews.Simulation(p.nx, p.ny, p.nz, p.spacing, boundary=p.boundary, width=p.width,
                         f0=p.f0, storage=storage)
    sim.set_model_vel(p.vp, p.vs, p.rho)
    sim.set_receivers(p.rec_pos)
    if scales is not None:
        sim.set_field_scales(scales)
    return sim


F16_SCALES = np.array([2.0 ** 10] * 3 + [2.0 ** -14] * 6, np.float32)


def state_for(p, storage, seed=5):
    """Random state with velocity ~1e-3 m/s and stress ~1e5 Pa (physical
    magnitudes of the small cases), representable at the test scales."""
    x = synth.random_state(p.nx, p.ny, p.nz, seed=seed)
    x[:3] *= 1e-3
    x[3:] *= 1e5
    sc = F16_SCALES if storage == "f16" else np.ones(9, np.float32)
    return round_to(x, storage, sc), sc


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_state_io_rounds_like_torch(ews, storage):
    p = synth.small_problem(37, 45, 33, nt=10, boundary="sponge", width=5)
    x = synth.random_state(p.nx, p.ny, p.nz, seed=3)
    x[:3] *= 1e-3
    x[3:] *= 1e5
    sc = F16_SCALES if storage == "f16" else np.ones(9, np.float32)
    sim = bare_sim(ews, p, storage, sc)
    sim.set_state(x)
    got = sim.get_state()
    assert np.array_equal(got, round_to(x, storage, sc))
    assert np.array_equal(sim.field_scales(), sc)


@pytest.mark.parametrize("boundary", ["none", "sponge", "cpml"])
@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_one_step_equals_rounded_fp32(ews, storage, boundary):
    p = synth.small_problem(70, 45, 37, nt=10, boundary=boundary, width=6, seed=11)
    x, sc = state_for(p, storage)
    ref = bare_sim(ews, p, "f32")
    ref.set_state(x)
    ref.advance(0, 1, p.dt, None, 1)
    y32 = ref.get_state()
    sim = bare_sim(ews, p, storage, sc)
    sim.set_state(x)
    sim.advance(0, 1, p.dt, None, 1)
    y = sim.get_state()
    # velocity pass: inputs identical, so the result is the FP32 one rounded
    v_want = round_to(y32[:3], storage, sc[:3])
    err = np.abs(y[:3].astype(np.float64) - v_want)
    assert np.all(err <= ulp(y32[:3], storage, sc[:3]) * 1.0001), float(err.max())
    # stress pass: its velocity input already carries one rounding
    for q in range(3, 9):
        assert rel(y[q], y32[q]) <= 2.0 ** -MANT[storage] * 4, (q, rel(y[q], y32[q]))


def _seis_errors(ews, orc, p, storages):
    want = orc.run_problem(p)
    out = {}
    for st in storages:
        sim = ews.simulation_for(p, storage=st)
        out[st] = rel(sim.run(p.nt, p.dt), want)
    return out


@pytest.mark.parametrize("case", ["cpml_moment", "sponge_force"])
def test_seismogram_error_against_oracle(ews, orc, case):
    boundary, kind = case.split("_")
    p = synth.small_problem(64, 56, 48, nt=300, boundary=boundary, width=8, kind=kind,
                            nrec=8, seed=21)
    e = _seis_errors(ews, orc, p, ["f32", "bf16", "f16"])
    print(f"\n{case}: seismogram rel L2 vs FP64 oracle: " +
          ", ".join(f"{k} {v:.2e}" for k, v in e.items()))
    assert e["f32"] <= 1e-5
    # measured on GB300: bf16 1.1e-2 / 6.6e-3, f16 1.4e-3 / 9.6e-4 (caps ~3x that)
    assert e["f16"] <= 5e-3
    assert e["bf16"] <= 3e-2


def test_f16_default_scales_are_powers_of_two_per_group(ews):
    p = synth.small_problem(40, 36, 28, nt=40, boundary="sponge", width=5, kind="moment")
    sim = ews.simulation_for(p, storage="f16")
    sim.run(p.nt, p.dt)
    sc = sim.field_scales().astype(np.float64)
    m, e = np.frexp(sc)
    assert np.all(m == 0.5)
    assert len(set(sc[:3])) == 1 and len(set(sc[3:])) == 1
    assert sc[0] > sc[3]            # velocities are far smaller than stresses in SI units
    simb = ews.simulation_for(p, storage="bf16")
    simb.run(p.nt, p.dt)
    assert np.array_equal(simb.field_scales(), np.ones(9, np.float32))


def test_f16_overflow_is_reported(ews):
    p = synth.small_problem(40, 36, 28, nt=40, boundary="sponge", width=5, kind="moment")
    sim = ews.simulation_for(p, storage="f16")
    sim.set_field_scales(np.full(9, 2.0 ** 60, np.float32))
    with pytest.raises(ews.EwsError) as e:
        sim.run(p.nt, p.dt)
    assert e.value.status == ews.EWS_ERANGE
    x = synth.random_state(p.nx, p.ny, p.nz) * 1e6
    with pytest.raises(ews.EwsError) as e:
        sim.set_state(x)
    assert e.value.status == ews.EWS_ERANGE


def test_scale_and_mode_validation(ews):
    p = synth.small_problem(40, 36, 28, nt=20, boundary="sponge", width=5)
    sim = ews.simulation_for(p, storage="bf16")
    for bad in (np.full(9, 3.0), np.zeros(9), np.full(9, np.inf)):
        with pytest.raises(ews.EwsError) as e:
            sim.set_field_scales(bad.astype(np.float32))
        assert e.value.status == ews.EWS_EINVAL
    f32 = ews.simulation_for(p)
    with pytest.raises(ews.EwsError):
        f32.set_field_scales(np.full(9, 2.0, np.float32))
    f32.set_field_scales(np.ones(9, np.float32))
    with pytest.raises(ews.EwsError) as e:
        sim.adjoint(p.nt, p.dt, np.zeros((3, p.rec_pos.shape[0], p.nt), np.float32))
    assert e.value.status == ews.EWS_EINVAL


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_snapshots_match_state(ews, storage):
    p = synth.small_problem(40, 36, 28, nt=30, boundary="cpml", width=5, kind="force")
    sim = ews.simulation_for(p, storage=storage, snapshot_every=30, snapshot_mask=0b111000111)
    snaps = np.zeros((6, p.nz, p.ny, p.nx), np.float32)
    sim.run(p.nt, p.dt, snapshots=snaps)
    st = sim.get_state()
    assert np.array_equal(snaps, st[[0, 1, 2, 6, 7, 8]])
    assert np.abs(st).max() > 0


def test_device_state_io_16bit(ews):
    import torch
    p = synth.small_problem(40, 36, 28, nt=20, boundary="sponge", width=5)
    x, sc = state_for(p, "bf16")
    sim = bare_sim(ews, p, "bf16")
    sim.set_state(torch.from_numpy(x).cuda())
    out = torch.zeros((9, p.nz, p.ny, p.nx), device="cuda")
    ews.ews_get_state(sim.handle, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), x)
