"""Thin ctypes binding of libews (include/ews.h).

Every function here has the name of the C entry point it marshals to and
does argument marshalling only: all numerical work runs in the CUDA kernels
of libews.  There is no CPU fallback: if libews.so is missing or no CUDA
device is usable, the calls raise.

Arrays may be numpy arrays (host) or torch CUDA tensors (device, passed by
pointer with on_device = 1).  Shapes follow include/ews.h: 3D arrays are
[nz][ny][nx] float32, seismograms [3][nrec][nt], state [9][nz][ny][nx].
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

EWS_OK, EWS_EINVAL, EWS_ECFL, EWS_ENOMEM, EWS_ECUDA, EWS_ENONFINITE, EWS_ETIMEOUT, \
    EWS_ESTATE, EWS_ERANGE = range(9)
STATUS_NAMES = ("EWS_OK", "EWS_EINVAL", "EWS_ECFL", "EWS_ENOMEM", "EWS_ECUDA",
                "EWS_ENONFINITE", "EWS_ETIMEOUT", "EWS_ESTATE", "EWS_ERANGE")
EWS_BOUNDARY_NONE, EWS_BOUNDARY_SPONGE, EWS_BOUNDARY_CPML = 0, 1, 2
EWS_STORAGE_F32, EWS_STORAGE_BF16, EWS_STORAGE_F16 = 0, 1, 2
STORAGE = {"f32": 0, "bf16": 1, "f16": 2}
EWS_SOURCE_MOMENT, EWS_SOURCE_FORCE = 0, 1
EWS_KERNEL_VELOCITY, EWS_KERNEL_STRESS, EWS_KERNEL_INJECT, EWS_KERNEL_RECORD = 0, 1, 2, 3
EWS_KERNEL_POINTS, EWS_KERNEL_STEP = 4, 5
EWS_NKERNEL = 8
KERNEL_NAMES = ("velocity", "stress", "inject", "record", "points", "step")
BOUNDARY = {"none": 0, "sponge": 1, "cpml": 2}
SOURCE = {"moment": 0, "force": 1}
FIELDS = ("vx", "vy", "vz", "sxx", "syy", "szz", "sxy", "sxz", "syz")


class EwsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


class ews_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double)]


class ews_options(C.Structure):
    _fields_ = [("boundary", C.c_int), ("width", C.c_int), ("storage", C.c_int),
                ("snapshot_every", C.c_int), ("snapshot_mask", C.c_uint),
                ("sponge_alpha", C.c_double), ("pml_R", C.c_double), ("pml_f0", C.c_double)]


class ews_batch_shot(C.Structure):
    _fields_ = [("sim", C.c_void_p), ("nt", C.c_int), ("dt", C.c_double),
                ("seis", C.c_void_p), ("observed", C.c_void_p), ("g_lam", C.c_void_p),
                ("g_mu", C.c_void_p), ("g_rho", C.c_void_p), ("misfit", C.c_double)]


class ews_batch_options(C.Structure):
    _fields_ = [("mode", C.c_int), ("ckpt_every", C.c_int), ("zchunk", C.c_int),
                ("ctas_per_sm", C.c_int), ("dep_wait_ms", C.c_int),
                ("test_unsatisfiable", C.c_int)]


class ews_tuned_zchunk(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("boundary", C.c_int),
                ("free_surface", C.c_int), ("zchunk", C.c_int)]


class ews_tuned_tile(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("boundary", C.c_int),
                ("storage", C.c_int), ("shape", C.c_int)]


EWS_BATCH_PERSISTENT, EWS_BATCH_SEQUENTIAL = 0, 1
EWS_TILE_AUTO, EWS_TILE_32X8, EWS_TILE_32X4, EWS_TILE_32X16, EWS_TILE_FUSED = 0, 1, 2, 3, 4
TILE = {"auto": EWS_TILE_AUTO, "32x8": EWS_TILE_32X8, "32x4": EWS_TILE_32X4,
        "32x16": EWS_TILE_32X16, "fused": EWS_TILE_FUSED}

_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) of every entry point declared in include/ews.h
_P, _I, _D, _U = C.c_void_p, C.c_int, C.c_double, C.c_uint
SIGNATURES = [
    ("ews_create", _I, [C.POINTER(ews_grid), C.POINTER(ews_options), C.POINTER(_P)]),
    ("ews_destroy", None, [_P]),
    ("ews_set_stream", _I, [_P, _P]),
    ("ews_set_model_lame", _I, [_P, _P, _P, _P, _I]),
    ("ews_set_model_vel", _I, [_P, _P, _P, _P, _I]),
    ("ews_set_source", _I, [_P, _I, _P, _P, _P, _I]),
    ("ews_set_receivers", _I, [_P, _I, _P]),
    ("ews_set_free_surface", _I, [_P, _I, _D]),
    ("ews_set_model_coarse", _I, [_P, _I, _I, _I, _P, _P, _P, _I, _I]),
    ("ews_run", _I, [_P, _I, _D, _P, _I, _P]),
    ("ews_advance", _I, [_P, _I, _I, _D, _P, _I, _I]),
    ("ews_reset", _I, [_P]),
    ("ews_get_state", _I, [_P, _P, _I]),
    ("ews_set_state", _I, [_P, _P, _I]),
    ("ews_set_field_scales", _I, [_P, _P]),
    ("ews_set_history_budget", _I, [_P, _D]),
    ("ews_set_checkpoint_storage", _I, [_P, _I]),
    ("ews_release_workspace", _I, [_P]),
    ("ews_get_field_scales", _I, [_P, _P]),
    ("ews_adjoint", _I, [_P, _I, _D, _P, _I, _P, _P, _P, _I, _I]),
    ("ews_gradient", _I, [_P, _I, _D, _P, _I, _P, _P, _P, _P, _I, _I]),
    ("ews_set_profiling", _I, [_P, _I]),
    ("ews_get_profile", _I, [_P, _P, _P, _I]),
    ("ews_forward_noalloc", _I, [C.POINTER(ews_grid), C.POINTER(ews_options), _P, _P, _P, _I,
                             _P, _P, _P, _I, _P, _I, _D, _P, _P]),
    ("ews_batch", _I, [_I, C.POINTER(ews_batch_shot), C.POINTER(ews_batch_options), _P]),
    ("ews_batch_tuned_zchunk", _I, [C.POINTER(ews_grid), _I, _I]),
    ("ews_batch_tuning_export", _I, [C.POINTER(ews_tuned_zchunk), _I]),
    ("ews_batch_tuning_import", _I, [C.POINTER(ews_tuned_zchunk), _I]),
    ("ews_batch_tuning_clear", None, []),
    ("ews_fwi_iteration", _I, [_I, C.POINTER(ews_batch_shot), _P, _P, _P, _D, _I, _P, _P, _P,
                               _P]),
    ("ews_set_tile_shape", _I, [_P, _I]),
    ("ews_get_tile_shape", _I, [_P]),
    ("ews_tile_tuned", _I, [C.POINTER(ews_grid), _I, _I]),
    ("ews_tile_tuning_export", _I, [C.POINTER(ews_tuned_tile), _I]),
    ("ews_tile_tuning_import", _I, [C.POINTER(ews_tuned_tile), _I]),
    ("ews_tile_tuning_clear", None, []),
    ("ews_set_memory_limit", _I, [_D]),
    ("ews_memory_limit", _D, []),
    ("ews_memory_in_use", _D, []),
    ("ews_cfl_dt", _D, [C.POINTER(ews_grid), _D]),
    ("ews_max_freq", _D, [C.POINTER(ews_grid), _D]),
    ("ews_last_error", C.c_char_p, []),
    ("ews_version", _I, []),
]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libews.so (building it in-tree if needed).  Raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                if not build_if_missing:
                    raise OSError(f"libews.so not built ({_build.LIB})")
                _build.build()
            lib = C.CDLL(_build.LIB)
            for name, res, args in SIGNATURES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int):
    if status != EWS_OK:
        msg = load().ews_last_error()
        raise EwsError(status, msg.decode() if msg else "")


def _ptr(a, dtype=np.float32):
    """(pointer, on_device) of a numpy array or torch tensor."""
    if a is None:
        return None, 0
    if hasattr(a, "data_ptr"):                      # torch tensor
        import torch
        assert a.is_contiguous(), "tensor must be contiguous"
        want = {np.float32: torch.float32, np.float64: torch.float64}[dtype]
        assert a.dtype == want, f"tensor dtype must be {want}"
        return C.c_void_p(a.data_ptr()), int(a.is_cuda)
    arr = np.asarray(a)
    assert arr.dtype == dtype and arr.flags.c_contiguous, \
        f"array must be C-contiguous {np.dtype(dtype).name}"
    return arr.ctypes.data_as(C.c_void_p), 0


# --- entry points (same names as include/ews.h) ----------------------------

def ews_version() -> int:
    return load().ews_version()


def ews_last_error() -> str:
    m = load().ews_last_error()
    return m.decode() if m else ""


def ews_set_memory_limit(nbytes: float):
    _check(load().ews_set_memory_limit(float(nbytes)))


def ews_memory_limit() -> float:
    return load().ews_memory_limit()


def ews_memory_in_use() -> float:
    return load().ews_memory_in_use()


def ews_cfl_dt(grid: ews_grid, vmax: float) -> float:
    return load().ews_cfl_dt(C.byref(grid), float(vmax))


def ews_max_freq(grid: ews_grid, vmin: float) -> float:
    return load().ews_max_freq(C.byref(grid), float(vmin))


def ews_create(grid: ews_grid, opt: ews_options | None):
    h = C.c_void_p()
    _check(load().ews_create(C.byref(grid), C.byref(opt) if opt is not None else None,
                             C.byref(h)))
    return h


def ews_destroy(sim):
    if sim:
        load().ews_destroy(sim)


def ews_set_stream(sim, stream_handle: int):
    _check(load().ews_set_stream(sim, C.c_void_p(stream_handle)))


def ews_set_model_lame(sim, lam, mu, rho):
    (pl, d0), (pm, d1), (pr, d2) = _ptr(lam), _ptr(mu), _ptr(rho)
    assert d0 == d1 == d2, "model arrays must share residency"
    _check(load().ews_set_model_lame(sim, pl, pm, pr, d0))


def ews_set_model_vel(sim, vp, vs, rho):
    (pa, d0), (pb, d1), (pr, d2) = _ptr(vp), _ptr(vs), _ptr(rho)
    assert d0 == d1 == d2, "model arrays must share residency"
    _check(load().ews_set_model_vel(sim, pa, pb, pr, d0))


def ews_set_source(sim, kind: int, pos, comp, wavelet):
    p = np.ascontiguousarray(pos, np.float64).reshape(3)
    c = np.zeros(6)
    cc = np.asarray(comp, np.float64).ravel()
    c[:cc.size] = cc
    w = np.ascontiguousarray(wavelet, np.float32).ravel()
    _check(load().ews_set_source(sim, int(kind), p.ctypes.data_as(C.c_void_p),
                                 c.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p),
                                 int(w.size)))


def ews_set_receivers(sim, pos):
    r = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
    _check(load().ews_set_receivers(sim, int(r.shape[0]),
                                    r.ctypes.data_as(C.c_void_p) if r.size else None))


def ews_set_model_coarse(sim, a, b, rho, from_velocities: bool = False):
    """Medium on its own grid; a, b, rho are [mz][my][mx] float32."""
    shape = tuple(a.shape)
    assert tuple(b.shape) == shape and tuple(rho.shape) == shape
    (pa, d0), (pb, d1), (pr, d2) = _ptr(a), _ptr(b), _ptr(rho)
    assert d0 == d1 == d2, "model arrays must share residency"
    mz, my, mx = shape
    _check(load().ews_set_model_coarse(sim, int(mx), int(my), int(mz), pa, pb, pr,
                                       int(bool(from_velocities)), d0))


def ews_set_free_surface(sim, ks: int, eps: float = 1e-3):
    _check(load().ews_set_free_surface(sim, int(ks), float(eps)))


def ews_run(sim, nt: int, dt: float, seis, snapshots=None):
    ps, dev = _ptr(seis)
    pn, devn = _ptr(snapshots)
    if snapshots is not None:
        assert devn == dev, "seis and snapshots must share residency"
    _check(load().ews_run(sim, int(nt), float(dt), ps, dev, pn))


def ews_advance(sim, n0: int, nsteps: int, dt: float, seis, ld: int):
    ps, dev = _ptr(seis)
    _check(load().ews_advance(sim, int(n0), int(nsteps), float(dt), ps, int(ld), dev))


def ews_reset(sim):
    _check(load().ews_reset(sim))


def ews_get_state(sim, out):
    p, dev = _ptr(out)
    _check(load().ews_get_state(sim, p, dev))


def ews_set_state(sim, state):
    p, dev = _ptr(state)
    _check(load().ews_set_state(sim, p, dev))


def ews_set_field_scales(sim, scale):
    """scale: 9 powers of two (state order), or None for the defaults."""
    if scale is None:
        _check(load().ews_set_field_scales(sim, None))
        return
    a = np.ascontiguousarray(scale, np.float32).reshape(9)
    _check(load().ews_set_field_scales(sim, a.ctypes.data_as(C.c_void_p)))


def ews_get_field_scales(sim):
    a = np.zeros(9, np.float32)
    _check(load().ews_get_field_scales(sim, a.ctypes.data_as(C.c_void_p)))
    return a


def ews_set_history_budget(sim, nbytes: float):
    _check(load().ews_set_history_budget(sim, float(nbytes)))


def ews_set_checkpoint_storage(sim, storage):
    storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    _check(load().ews_set_checkpoint_storage(sim, storage))


def ews_release_workspace(sim):
    _check(load().ews_release_workspace(sim))


def ews_adjoint(sim, nt: int, dt: float, seis_adj, g_lam, g_mu, g_rho, ckpt_every: int = 0):
    pa, da = _ptr(seis_adj)
    (pl, d0), (pm, d1), (pr, d2) = _ptr(g_lam), _ptr(g_mu), _ptr(g_rho)
    assert d0 == d1 == d2, "gradient outputs must share residency"
    _check(load().ews_adjoint(sim, int(nt), float(dt), pa, da, pl, pm, pr, d0, int(ckpt_every)))


def ews_gradient(sim, nt: int, dt: float, observed, g_lam, g_mu, g_rho, ckpt_every: int = 0):
    """Returns the L2 misfit; gradients are written into g_lam, g_mu, g_rho."""
    po, do = _ptr(observed)
    (pl, d0), (pm, d1), (pr, d2) = _ptr(g_lam), _ptr(g_mu), _ptr(g_rho)
    assert d0 == d1 == d2, "gradient outputs must share residency"
    mis = C.c_double(0.0)
    _check(load().ews_gradient(sim, int(nt), float(dt), po, do, C.byref(mis), pl, pm, pr, d0,
                               int(ckpt_every)))
    return mis.value


def ews_batch(shots, mode: int = EWS_BATCH_PERSISTENT, ckpt_every: int = 0, zchunk: int = 0,
              ctas_per_sm: int = 0, dep_wait_ms: int = 0, test_unsatisfiable: bool = False,
              stream_handle: int = 0):
    """Run shots in one batched launch.  Each shot is a dict with keys
    sim (Simulation), nt, dt and optional seis (CUDA tensor [3][nrec][nt]),
    observed, g_lam, g_mu, g_rho (CUDA tensors).  Returns the misfits."""
    arr = (ews_batch_shot * len(shots))()
    for i, d in enumerate(shots):
        b = arr[i]
        b.sim = d["sim"].handle.value if hasattr(d["sim"], "handle") else d["sim"]
        b.nt = int(d["nt"])
        b.dt = float(d["dt"])
        for key in ("seis", "observed", "g_lam", "g_mu", "g_rho"):
            t = d.get(key)
            if t is not None:
                p, dev = _ptr(t)
                assert dev == 1, f"{key} must be a CUDA tensor"
                setattr(b, key, p.value)
    opt = ews_batch_options(int(mode), int(ckpt_every), int(zchunk), int(ctas_per_sm),
                            int(dep_wait_ms), int(bool(test_unsatisfiable)))
    _check(load().ews_batch(len(shots), arr, C.byref(opt), C.c_void_p(stream_handle)))
    return [arr[i].misfit for i in range(len(shots))]


def ews_fwi_iteration(shots, lam, mu, rho, max_rel_step: float = 0.02, ckpt_every: int = 0,
                      stream_handle: int = 0):
    """One multi-shot inversion iteration.  shots: dicts with sim, nt, dt and
    observed (CUDA tensor); lam, mu, rho: CUDA tensors [nz][ny][nx] updated
    in place.  Returns (misfit before, misfit after, accepted step)."""
    arr = (ews_batch_shot * len(shots))()
    for i, d in enumerate(shots):
        arr[i].sim = d["sim"].handle.value if hasattr(d["sim"], "handle") else d["sim"]
        arr[i].nt = int(d["nt"])
        arr[i].dt = float(d["dt"])
        p, dev = _ptr(d["observed"])
        assert dev == 1, "observed must be a CUDA tensor"
        arr[i].observed = p.value
    ptrs = []
    for t in (lam, mu, rho):
        p, dev = _ptr(t)
        assert dev == 1, "the model must be CUDA tensors"
        ptrs.append(p)
    j0, j1, a = C.c_double(), C.c_double(), C.c_double()
    _check(load().ews_fwi_iteration(len(shots), arr, ptrs[0], ptrs[1], ptrs[2],
                                    float(max_rel_step), int(ckpt_every), C.byref(j0),
                                    C.byref(j1), C.byref(a), C.c_void_p(stream_handle)))
    return j0.value, j1.value, a.value


def ews_batch_tuned_zchunk(grid: ews_grid, boundary: int, free_surface: bool) -> int:
    return load().ews_batch_tuned_zchunk(C.byref(grid), int(boundary), int(bool(free_surface)))


_BOUNDARY_NAMES = {v: k for k, v in BOUNDARY.items()}
TUNING_FORMAT = "ews-batch-tuning/1"


def ews_batch_tuning_export() -> list:
    """The autotuner table as a list of dicts (nx, ny, nz, boundary name,
    free_surface, zchunk)."""
    lib = load()
    n = lib.ews_batch_tuning_export(None, 0)
    arr = (ews_tuned_zchunk * max(n, 1))()
    n = min(n, lib.ews_batch_tuning_export(arr, n))
    return [{"nx": e.nx, "ny": e.ny, "nz": e.nz, "boundary": _BOUNDARY_NAMES.get(e.boundary, e.boundary),
             "free_surface": bool(e.free_surface), "zchunk": e.zchunk} for e in arr[:n]]


def ews_batch_tuning_import(entries) -> None:
    """Add entries (dicts as ews_batch_tuning_export returns) to the table."""
    entries = list(entries)
    arr = (ews_tuned_zchunk * max(len(entries), 1))()
    for k, e in enumerate(entries):
        b = e["boundary"]
        arr[k] = ews_tuned_zchunk(int(e["nx"]), int(e["ny"]), int(e["nz"]),
                                  BOUNDARY[b] if isinstance(b, str) else int(b),
                                  int(bool(e["free_surface"])), int(e["zchunk"]))
    _check(load().ews_batch_tuning_import(arr, len(entries)))


def ews_batch_tuning_clear() -> None:
    load().ews_batch_tuning_clear()


_TILE_NAMES = {v: k for k, v in TILE.items()}
_STORAGE_NAMES = {v: k for k, v in STORAGE.items()}


def ews_set_tile_shape(sim, shape):
    _check(load().ews_set_tile_shape(sim, TILE[shape] if isinstance(shape, str) else int(shape)))


def ews_get_tile_shape(sim) -> int:
    return load().ews_get_tile_shape(sim)


def ews_tile_tuned(grid: ews_grid, boundary, storage) -> int:
    b = BOUNDARY[boundary] if isinstance(boundary, str) else int(boundary)
    st = STORAGE[storage] if isinstance(storage, str) else int(storage)
    return load().ews_tile_tuned(C.byref(grid), b, st)


def ews_tile_tuning_export() -> list:
    """The tile-shape table as a list of dicts (nx, ny, nz, boundary name,
    storage name, shape name)."""
    lib = load()
    n = lib.ews_tile_tuning_export(None, 0)
    arr = (ews_tuned_tile * max(n, 1))()
    n = min(n, lib.ews_tile_tuning_export(arr, n))
    return [{"nx": e.nx, "ny": e.ny, "nz": e.nz,
             "boundary": _BOUNDARY_NAMES.get(e.boundary, e.boundary),
             "storage": _STORAGE_NAMES.get(e.storage, e.storage),
             "shape": _TILE_NAMES.get(e.shape, e.shape)} for e in arr[:n]]


def ews_tile_tuning_import(entries) -> None:
    """Add entries (dicts as ews_tile_tuning_export returns) to the table."""
    entries = list(entries)
    arr = (ews_tuned_tile * max(len(entries), 1))()
    for k, e in enumerate(entries):
        b, st, sh = e["boundary"], e["storage"], e["shape"]
        arr[k] = ews_tuned_tile(int(e["nx"]), int(e["ny"]), int(e["nz"]),
                                BOUNDARY[b] if isinstance(b, str) else int(b),
                                STORAGE[st] if isinstance(st, str) else int(st),
                                TILE[sh] if isinstance(sh, str) else int(sh))
    _check(load().ews_tile_tuning_import(arr, len(entries)))


def ews_tile_tuning_clear() -> None:
    load().ews_tile_tuning_clear()


def _device_name():
    try:
        import torch
        return torch.cuda.get_device_name() if torch.cuda.is_available() else None
    except Exception:
        return None


def save_batch_tuning(path: str, device: str | None = None) -> int:
    """Write the autotuner tables (batch z-chunks, and the tile shapes of the
    forward passes under "tiles") to a JSON file, tagged with the GPU they
    were timed on (default: the current CUDA device).  Returns the z-chunk
    entry count."""
    import json
    entries = ews_batch_tuning_export()
    tiles = ews_tile_tuning_export()
    doc = {"format": TUNING_FORMAT, "device": device if device is not None else _device_name(),
           "entries": entries, "tiles": tiles}
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
    return len(entries)


def load_batch_tuning(path: str, device: str | None = None) -> int:
    """Import a table written by save_batch_tuning.  Entries timed on another
    GPU are not imported (returns 0); device defaults to the current CUDA
    device.  Returns the number of entries imported."""
    import json
    with open(path) as f:
        doc = json.load(f)
    if doc.get("format") != TUNING_FORMAT:
        raise ValueError(f"{path}: not an autotuner table ({doc.get('format')!r})")
    here = device if device is not None else _device_name()
    if doc.get("device") is not None and here is not None and doc["device"] != here:
        return 0
    ews_batch_tuning_import(doc["entries"])
    ews_tile_tuning_import(doc.get("tiles", []))
    return len(doc["entries"])


def ews_set_profiling(sim, on: bool):
    _check(load().ews_set_profiling(sim, int(bool(on))))


def ews_get_profile(sim, reset: bool = False):
    """(ms[EWS_NKERNEL], launches[EWS_NKERNEL]) accumulated per kernel class."""
    ms = np.zeros(EWS_NKERNEL, np.float64)
    n = np.zeros(EWS_NKERNEL, np.int64)
    _check(load().ews_get_profile(sim, ms.ctypes.data_as(C.c_void_p),
                                  n.ctypes.data_as(C.c_void_p), int(bool(reset))))
    return ms, n


def ews_forward_noalloc(grid: ews_grid, opt: ews_options | None, lam, mu, rho, kind: int, pos,
                        comp, wavelet, rec_pos, nt: int, dt: float, seis, stream_handle: int = 0):
    """Forward run without any device allocation (see include/ews.h).
    lam, mu, rho, wavelet and seis must be CUDA tensors (device pointers)."""
    ptrs = []
    for a in (lam, mu, rho, wavelet, seis):
        p, dev = _ptr(a)
        assert dev == 1, "ews_forward_noalloc takes device buffers"
        ptrs.append(p)
    p = np.ascontiguousarray(pos, np.float64).reshape(3)
    c = np.zeros(6)
    cc = np.asarray(comp, np.float64).ravel()
    c[:cc.size] = cc
    r = np.ascontiguousarray(rec_pos, np.float64).reshape(-1, 3)
    _check(load().ews_forward_noalloc(
        C.byref(grid), C.byref(opt) if opt is not None else None, ptrs[0], ptrs[1], ptrs[2],
        int(kind), p.ctypes.data_as(C.c_void_p), c.ctypes.data_as(C.c_void_p), ptrs[3],
        int(r.shape[0]), r.ctypes.data_as(C.c_void_p) if r.size else None, int(nt), float(dt),
        ptrs[4], C.c_void_p(stream_handle)))


# --- convenience object ------------------------------------------------------

class Simulation:
    """Owns one ews_sim handle.  Mirrors the C calls one to one."""

    def __init__(self, nx, ny, nz, spacing, boundary="sponge", width=16, f0=0.0,
                 snapshot_every=0, snapshot_mask=0, sponge_alpha=0.0, pml_R=0.0,
                 storage=EWS_STORAGE_F32):
        self.grid = ews_grid(int(nx), int(ny), int(nz), *map(float, spacing))
        storage = STORAGE[storage] if isinstance(storage, str) else storage
        self.opt = ews_options(BOUNDARY[boundary] if isinstance(boundary, str) else boundary,
                               int(width), int(storage), int(snapshot_every),
                               int(snapshot_mask), float(sponge_alpha), float(pml_R),
                               float(f0))
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self._h = ews_create(self.grid, self.opt)
        self.nrec = 0

    def close(self):
        if getattr(self, "_h", None):
            ews_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream_handle: int):
        ews_set_stream(self._h, stream_handle)

    def set_model_vel(self, vp, vs, rho):
        ews_set_model_vel(self._h, vp, vs, rho)

    def set_model_lame(self, lam, mu, rho):
        ews_set_model_lame(self._h, lam, mu, rho)

    def set_source(self, kind, pos, comp, wavelet):
        ews_set_source(self._h, SOURCE[kind] if isinstance(kind, str) else kind, pos, comp,
                       wavelet)

    def set_checkpoint_storage(self, storage):
        """Element type of the adjoint's checkpoints: "f32", "bf16" or "f16"."""
        ews_set_checkpoint_storage(self._h, storage)

    def set_model_coarse(self, a, b, rho, from_velocities=False):
        """Medium on its own (coarser) grid, sampled trilinearly (Sec. 2.2.1)."""
        ews_set_model_coarse(self._h, a, b, rho, from_velocities)

    def set_free_surface(self, ks, eps=1e-3):
        """Vacuum free surface above plane ks (set the model afterwards)."""
        ews_set_free_surface(self._h, ks, eps)

    def set_receivers(self, pos):
        ews_set_receivers(self._h, pos)
        self.nrec = int(np.asarray(pos).reshape(-1, 3).shape[0])

    def run(self, nt, dt, seis=None, snapshots=None):
        if seis is None:
            seis = np.zeros((3, self.nrec, nt), np.float32)
        ews_run(self._h, nt, dt, seis if self.nrec else None, snapshots)
        return seis

    def advance(self, n0, nsteps, dt, seis, ld):
        ews_advance(self._h, n0, nsteps, dt, seis, ld)

    def reset(self):
        ews_reset(self._h)

    def adjoint(self, nt, dt, seis_adj, ckpt_every=0, out=None):
        """dL/d(lambda, mu, rho), [3][nz][ny][nx], for dL/dseis = seis_adj."""
        if out is None:
            out = np.zeros((3, self.nz, self.ny, self.nx), np.float32)
        ews_adjoint(self._h, nt, dt, seis_adj, out[0], out[1], out[2], ckpt_every)
        return out

    def gradient(self, nt, dt, observed, ckpt_every=0, out=None):
        """(misfit, dJ/d(lambda, mu, rho)) for the L2 misfit against observed."""
        if out is None:
            out = np.zeros((3, self.nz, self.ny, self.nx), np.float32)
        mis = ews_gradient(self._h, nt, dt, observed, out[0], out[1], out[2], ckpt_every)
        return mis, out

    def set_tile_shape(self, shape):
        ews_set_tile_shape(self._h, shape)

    @property
    def tile_shape(self) -> str:
        return _TILE_NAMES.get(ews_get_tile_shape(self._h), "?")

    def set_profiling(self, on=True):
        ews_set_profiling(self._h, on)

    def profile(self, reset=False):
        return ews_get_profile(self._h, reset)

    def get_state(self, out=None):
        if out is None:
            out = np.zeros((9, self.nz, self.ny, self.nx), np.float32)
        ews_get_state(self._h, out)
        return out

    def set_state(self, state):
        ews_set_state(self._h, state)

    def release_workspace(self):
        ews_release_workspace(self._h)

    def set_history_budget(self, nbytes):
        ews_set_history_budget(self._h, nbytes)

    def set_field_scales(self, scale):
        ews_set_field_scales(self._h, scale)

    def field_scales(self):
        return ews_get_field_scales(self._h)


def simulation_for(prob, **kw) -> Simulation:
    """Simulation set up from a ``synth.Problem`` (model, source, receivers)."""
    sim = Simulation(prob.nx, prob.ny, prob.nz, prob.spacing, boundary=prob.boundary,
                     width=prob.width, f0=prob.f0, **kw)
    if prob.free_surface is not None:
        sim.set_free_surface(*prob.free_surface)
    if prob.coarse_medium is not None:
        sim.set_model_coarse(*[np.ascontiguousarray(a, np.float32) for a in prob.coarse_medium])
    else:
        sim.set_model_vel(prob.vp, prob.vs, prob.rho)
    sim.set_source(prob.src_kind, prob.src_pos, prob.src_comp, prob.wavelet)
    sim.set_receivers(prob.rec_pos)
    return sim
