"""C-ABI library: builds, loads without a GPU and exports every entry point
declared in include/ews.h; host-side validation paths (CPU only)."""
import os
import re

import numpy as np
import pytest

from paper_2112_15071_gb300 import ews

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "ews.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ews_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("ews_create", "ews_destroy", "ews_set_model_lame", "ews_set_model_vel",
              "ews_set_source", "ews_set_receivers", "ews_run", "ews_cfl_dt",
              "ews_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    lib = ews.load()
    for s in declared_symbols():
        assert hasattr(lib, s), s
    bound = {name for name, _, _ in ews.SIGNATURES}
    assert set(declared_symbols()) <= bound


def test_binding_names_match_the_abi():
    for s in declared_symbols():
        assert callable(getattr(ews, s)), s


def test_version_and_time_step_rules():
    assert ews.ews_version() >= 100
    g = ews.ews_grid(64, 64, 32, 10.0, 20.0, 5.0)
    # Eq. 5: 0.495 dx_min / v_max ; Eq. 6: v_min / (5 dx_max)
    assert ews.ews_cfl_dt(g, 3000.0) == pytest.approx(0.495 * 5.0 / 3000.0, rel=1e-15)
    assert ews.ews_max_freq(g, 1730.0) == pytest.approx(1730.0 / (5 * 20.0), rel=1e-15)
    assert ews.ews_cfl_dt(g, 0.0) == 0.0


@pytest.mark.parametrize("dims", [(3, 8, 8), (8, 0, 8), (8, 8, -1)])
def test_create_rejects_bad_grids_before_touching_the_device(dims):
    g = ews.ews_grid(*dims, 10.0, 10.0, 10.0)
    with pytest.raises(ews.EwsError) as e:
        ews.ews_create(g, None)
    assert e.value.status == ews.EWS_EINVAL


def test_create_rejects_bad_options():
    g = ews.ews_grid(16, 16, 16, 10.0, 10.0, 10.0)
    for opt in (ews.ews_options(2, 9, 0, 0, 0, 0.0, 0.0, 0.0),      # 2W > n
                ews.ews_options(7, 2, 0, 0, 0, 0.0, 0.0, 0.0),      # unknown boundary
                ews.ews_options(1, 0, 0, 0, 0, 0.0, 0.0, 0.0),      # width 0
                ews.ews_options(1, 2, 0, 0, 1 << 12, 0.0, 0.0, 0.0)):  # bad mask
        with pytest.raises(ews.EwsError) as e:
            ews.ews_create(g, opt)
        assert e.value.status == ews.EWS_EINVAL
    bad = ews.ews_grid(16, 16, 16, 10.0, -1.0, 10.0)
    with pytest.raises(ews.EwsError):
        ews.ews_create(bad, None)


def test_null_handles_are_rejected():
    with pytest.raises(ews.EwsError) as e:
        ews.ews_run(None, 10, 1e-3, None)
    assert e.value.status == ews.EWS_EINVAL
    ews.ews_destroy(None)
    assert "null" in ews.ews_last_error()


def test_cpu_box_has_no_fallback():
    """Without a usable device, creating a simulation fails loudly."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    g = ews.ews_grid(40, 40, 40, 10.0, 10.0, 10.0)
    with pytest.raises(ews.EwsError) as e:
        ews.ews_create(g, None)
    assert e.value.status == ews.EWS_ECUDA


def test_oracle_and_product_share_no_code():
    """The CUDA package and the oracle never import or include each other."""
    pkg = os.path.join(ROOT, "paper_2112_15071_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, re.M), f
                assert "ews_oracle" not in txt and "liborc" not in txt, f
    orc = os.path.join(ROOT, "oracle")
    for f in os.listdir(orc):
        if f.endswith((".py", ".c", ".h")):
            txt = open(os.path.join(orc, f)).read()
            assert not re.search(r"^\s*(from|import)\s+paper_2112_15071_gb300", txt, re.M), f
            assert not re.search(r"#\s*include\s*[<\"].*(ews|csrc)", txt), f


def test_every_entry_point_is_documented():
    """Each declaration in include/ews.h follows a comment (its contract),
    or directly follows a sibling declaration that shares it."""
    lines = open(os.path.join(ROOT, "include", "ews.h")).read().split("\n")
    decl = re.compile(r"^(ews_status|int|double|void|const char\*)\s+\**\s*(ews_[a-z_0-9]+)\s*\(")
    seen = 0
    for n, line in enumerate(lines):
        m = decl.match(line)
        if not m:
            continue
        seen += 1
        k = n - 1
        while k >= 0 and not lines[k].strip():
            k -= 1
        prev = lines[k].strip()
        assert prev.endswith("*/") or prev.endswith(");"), m.group(2)
    assert seen == len(declared_symbols())


@pytest.mark.parametrize("case,msg", [
    ("big_side", "above the no-allocation limit"),
    ("big_cells", "padded cells"),
    ("cpml", "C-PML needs memory variables"),
    ("bf16", "only F32 storage"),
    ("nt0", "nt must be positive"),
    ("many_receivers", "no-allocation limit is 64"),
    ("source_out", "source outside"),
    ("receiver_out", "receiver 1 outside"),
    ("bad_dt", "dt must be positive"),
])
def test_noalloc_validates_on_the_host(case, msg):
    """ews_forward_noalloc checks every argument before any device work, so
    its limits and errors hold on a machine without a GPU.  The device
    pointers are placeholders: nothing reads them before the checks."""
    import ctypes as C
    lib = ews.load()
    n = {"big_side": (1100, 8, 8), "big_cells": (512, 512, 8)}.get(case, (40, 36, 28))
    g = ews.ews_grid(*n, 10.0, 10.0, 10.0)
    opt = ews.ews_options(ews.EWS_BOUNDARY_SPONGE, 4, 0, 0, 0, 0.0, 0.0, 0.0)
    if case == "cpml":
        opt.boundary = ews.EWS_BOUNDARY_CPML
    if case == "bf16":
        opt.storage = ews.EWS_STORAGE_BF16
    fake = C.c_void_p(0x1000)
    pos = np.array([200.0, 180.0, 140.0])
    if case == "source_out":
        pos = np.array([1.0, 180.0, 140.0])
    nrec = 70 if case == "many_receivers" else 2
    rec = np.tile(np.array([150.0, 150.0, 100.0]), (nrec, 1))
    if case == "receiver_out":
        rec[1, 2] = 1e6
    comp = np.zeros(6)
    nt = 0 if case == "nt0" else 10
    dt = -1.0 if case == "bad_dt" else 1e-3
    st = lib.ews_forward_noalloc(C.byref(g), C.byref(opt), fake, fake, fake, ews.EWS_SOURCE_MOMENT,
                                 pos.ctypes.data_as(C.c_void_p), comp.ctypes.data_as(C.c_void_p),
                                 fake, nrec, rec.ctypes.data_as(C.c_void_p), nt, dt, fake, None)
    assert st == ews.EWS_EINVAL
    assert msg in ews.ews_last_error()


def test_batch_validates_on_the_host():
    """ews_batch rejects empty batches, unknown modes, negative options and
    missing simulations before any device work."""
    import ctypes as C
    lib = ews.load()
    shots = (ews.ews_batch_shot * 1)()
    shots[0].nt = 10
    shots[0].dt = 1e-3
    assert lib.ews_batch(0, shots, None, None) == ews.EWS_EINVAL
    assert "no shots" in ews.ews_last_error()
    o = ews.ews_batch_options(5, 0, 0, 0, 0, 0)
    assert lib.ews_batch(1, shots, C.byref(o), None) == ews.EWS_EINVAL
    assert "unknown batch mode" in ews.ews_last_error()
    o = ews.ews_batch_options(0, 0, -8, 0, 0, 0)
    assert lib.ews_batch(1, shots, C.byref(o), None) == ews.EWS_EINVAL
    assert "negative" in ews.ews_last_error()
    assert lib.ews_batch(1, shots, None, None) == ews.EWS_EINVAL
    assert "null simulation" in ews.ews_last_error()


def test_memory_limit_calls_are_host_only():
    """ews_set_memory_limit / ews_memory_limit / ews_memory_in_use touch host
    state only: without a device nothing is held, a limit can be set and
    read back, a negative value removes it and NaN is refused."""
    assert ews.ews_memory_in_use() == 0.0
    try:
        ews.ews_set_memory_limit(123456789.0)
        assert ews.ews_memory_limit() == 123456789.0
        ews.ews_set_memory_limit(-5.0)
        assert ews.ews_memory_limit() < 0
        with pytest.raises(ews.EwsError) as e:
            ews.ews_set_memory_limit(float("nan"))
        assert e.value.status == ews.EWS_EINVAL
    finally:
        ews.ews_set_memory_limit(-1.0)
