"""The benchmark's roofline bookkeeping (CPU only): algorithmic bytes per
launch counted by brute force over the fields each pass touches and over
the C-PML slab cells, against bench.algorithmic_bytes; and the committed
traffic lines parse."""
import os
import re
import types

import numpy as np

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def brute_bytes(nx, ny, nz, W, es):
    n = nx * ny * nz
    # fields read / written per cell and pass (Eq. 1 reads the 6 stresses and
    # rho and updates the 3 velocities; Eq. 2/3 read the 3 velocities, lambda
    # and mu and update the 6 stresses)
    vel = (6 + 3 + 3) * es * n + 4 * n
    st = (3 + 6 + 6) * es * n + 8 * n
    # C-PML: every cell inside the slab of direction d carries 3 memory
    # variables per pass, read and written in FP32
    dirs = 0
    if W:
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        for a, m in ((i, nx), (j, ny), (k, nz)):
            dirs += int(np.count_nonzero((a < W) | (a >= m - W)))
    return vel + 24 * dirs, st + 24 * dirs, dirs


def test_algorithmic_bytes_match_brute_force():
    for (nx, ny, nz, bnd, W) in ((40, 36, 28, "cpml", 5), (33, 65, 40, "sponge", 6),
                                 (64, 64, 64, "cpml", 20)):
        for es in (4, 2):
            p = types.SimpleNamespace(nx=nx, ny=ny, nz=nz, boundary=bnd, width=W)
            a = bench.algorithmic_bytes(p, es)
            v, s, d = brute_bytes(nx, ny, nz, W if bnd == "cpml" else 0, es)
            assert (a["velocity"], a["stress"], a["slab_cell_dirs"]) == (v, s, d)
            assert a["step_min"] == (18 * es + 12) * nx * ny * nz + 48 * d


def test_bench_workload_figures():
    """The per-launch figures quoted for the 256^3 C-PML workload."""
    p = types.SimpleNamespace(nx=256, ny=256, nz=256, boundary="cpml", width=20)
    a = bench.algorithmic_bytes(p, 4)
    assert a["stress"] == 1329594368 and a["velocity"] == 1061158912


def test_committed_traffic_lines_parse():
    pat = re.compile(r"bench-traffic:\s*kernel=(\S+)\s+workload=(\S+)\s+sha=([0-9a-f]{16})\s+"
                     r"bytes_per_launch=([0-9]+)")
    found = 0
    for f in os.listdir(os.path.join(ROOT, "profiles")):
        for m in pat.finditer(open(os.path.join(ROOT, "profiles", f)).read()):
            found += 1
            assert int(m.group(4)) > 0
    assert found >= 2


def test_a_failing_section_keeps_the_headline_line(capsys):
    def boom(x):
        raise RuntimeError(f"no memory for {x}")
    assert bench.section(lambda a, b: a + b, 2, 3) == 5
    r = bench.section(boom, "the sweep")
    assert r == {"error": "RuntimeError: no memory for the sweep"}
    assert "RuntimeError" in capsys.readouterr().err
