"""Mutation study of the oracle's pins (test infrastructure, CPU only).

Plants one plausible mistake at a time -- a wrong Eq. 4 weight, tap or
spacing, a sign, a transposed medium index, a dropped volume or buoyancy
factor, a wrong staggering offset, sponge index, C-PML sign, surface mean
or switch extent, coarse-grid convention -- in a COPY of ews_oracle.c
under _build/mutants/<name>/ (git-ignored), and runs the CPU pin tests that rest
on the paper and the mathematics (closed forms, brute force, invariants,
printed values; the adjoint-vs-forward consistency tests are left out)
against that copy.  Every mistake must fail at least one pin.  The oracle
itself is never modified.

    python tests/oracle_mutation_study.py [name ...]
"""
import os
import shutil
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "_build", "mutants")
SRC = open(os.path.join(ROOT, "oracle", "ews_oracle.c")).read()
TESTS = ["test_oracle_pins.py", "test_oracle_invariances.py", "test_oracle_free_surface.py",
         "test_oracle_coarse_medium.py", "test_golden_paper.py"]

M = [
    ("eq4_outer_weight", "#define ORC_C2 (-1.0 / 24.0)", "#define ORC_C2 (-1.0 / 12.0)"),
    ("dplus_wrong_axis_h", "return (ORC_C1 * (fp1 - f0) + ORC_C2 * (fp2 - fm1)) / s->h[a];",
     "return (ORC_C1 * (fp1 - f0) + ORC_C2 * (fp2 - fm1)) / s->h[0];"),
    ("dminus_wrong_tap", "return (ORC_C1 * (f0 - fm1) + ORC_C2 * (fp1 - fm2)) / s->h[a];",
     "return (ORC_C1 * (f0 - fm1) + ORC_C2 * (fp1 - fm1)) / s->h[a];"),
    ("shear_sign", "f[SXY][c] += dt * s->mxy[c] * (vxy + vyx);", "f[SXY][c] += dt * s->mxy[c] * (vxy - vyx);"),
    ("lambda_l2m_swap", "f[SXX][c] += dt * (l2m * exx + l * (eyy + ezz));",
     "f[SXX][c] += dt * (l * exx + l2m * (eyy + ezz));"),
    ("rho_mean_transposed", "s->bx[c] = 1.0 / (0.5 * (rho[c] + rho[IDX(s, ip, j, k)]));",
     "s->bx[c] = 1.0 / (0.5 * (rho[c] + rho[IDX(s, i, jp, k)]));"),
    ("mu_mean_transposed", "s->mxz[c] = 0.25 * (mu[c] + mu[IDX(s, ip, j, k)] + mu[IDX(s, i, j, kp)]",
     "s->mxz[c] = 0.25 * (mu[c] + mu[IDX(s, i, jp, k)] + mu[IDX(s, i, j, kp)]"),
    ("moment_no_volume", "if (idx[m] >= 0) s->f[q][idx[m]] -= w[m] * dt * M[c] * amp / vol;",
     "if (idx[m] >= 0) s->f[q][idx[m]] -= w[m] * dt * M[c] * amp;"),
    ("force_no_buoyancy", "s->f[q][idx[m]] += w[m] * dt * b[q][idx[m]] * F[q] * amp / vol;",
     "s->f[q][idx[m]] += w[m] * dt * F[q] * amp / vol;"),
    ("pml_sign", "psi[c] = s->pb[a][ia] * psi[c] + s->pa[a][ia] * d;",
     "psi[c] = s->pb[a][ia] * psi[c] - s->pa[a][ia] * d;"),
    ("sponge_index", "double gg = s->g[0][i] * s->g[1][j] * s->g[2][k];",
     "double gg = s->g[0][i] * s->g[1][i] * s->g[2][k];"),
    ("stagger_sign", "double u = pos[a] / s->h[a] - OFF[q][a];", "double u = pos[a] / s->h[a] + OFF[q][a];"),
    ("vz_dzy_wrong_difference", "double dzy = pml_term(s, 7, 1, j, c, d_minus(s, f[SYZ], 1, i, j, k));",
     "double dzy = pml_term(s, 7, 1, j, c, d_plus(s, f[SYZ], 1, i, j, k));"),
    ("surface_arith_mean", "s->mxz[c] = 4.0 / (1.0 / mu[c] + 1.0 / mu[IDX(s, ip, j, k)]",
     "s->mxz[c] = 4.0 / (4.0 / mu[c] + 0.0 / mu[IDX(s, ip, j, k)]"),
    ("surface_switch_extent", "return z0 - 1.5 < zs && zs < z0 + 1.5;", "return z0 - 0.5 < zs && zs < z0 + 0.5;"),
    ("coarse_centre_convention", "double c = (x[d] + 0.5) * (double)m[d] / (double)n[d] - 0.5;",
     "double c = x[d] * (double)m[d] / (double)n[d];"),
]


def conftest(mdir):
    return f'''import os, sys
import pytest
sys.path.insert(0, {ROOT!r})
sys.path.insert(0, {mdir!r})

def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: gpu")
    config.addinivalue_line("markers", "slow: slow")

@pytest.fixture(scope="session")
def orc():
    from oracle import oracle
    assert oracle.__file__.startswith({mdir!r}), oracle.__file__
    oracle.build()
    return oracle
'''


def main():
    only = sys.argv[1:]
    base = OUT
    survived = 0
    for name, old, new in M:
        if only and name not in only:
            continue
        assert SRC.count(old) == 1, name
        mdir = os.path.join(base, name)
        if os.path.exists(mdir):
            shutil.rmtree(mdir)
        os.makedirs(os.path.join(mdir, "oracle"))
        os.makedirs(os.path.join(mdir, "t"))
        for f in ("__init__.py", "oracle.py", "brute.py", "stokes.py"):
            shutil.copy(os.path.join(ROOT, "oracle", f), os.path.join(mdir, "oracle", f))
        open(os.path.join(mdir, "oracle", "ews_oracle.c"), "w").write(SRC.replace(old, new))
        for t in TESTS:
            shutil.copy(os.path.join(ROOT, "tests", t), os.path.join(mdir, "t", t))
        shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(mdir, "t", "golden"))
        open(os.path.join(mdir, "t", "conftest.py"), "w").write(conftest(mdir))
        t0 = time.time()
        r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-rfE", "-m", "not gpu",
                            "-p", "no:cacheprovider", "--rootdir", mdir, "-c", os.devnull,
                            os.path.join(mdir, "t")], capture_output=True, text=True, timeout=1800,
                           cwd=mdir)
        fails = [l.split()[1].split("::") for l in r.stdout.splitlines() if l.startswith("FAILED")]
        errors = [l for l in r.stdout.splitlines() if l.startswith("ERROR")]
        status = "caught" if fails else ("BROKEN" if errors or r.returncode != 0 else "SURVIVED")
        by = {}
        for f in fails:
            key = f[0].replace("t/", "") + "::" + f[1].split("[")[0]
            by[key] = by.get(key, 0) + 1
        survived += not fails
        print(f"{name:28s} {status:9s} {time.time() - t0:6.1f}s  " +
              "; ".join(f"{k} x{v}" for k, v in sorted(by.items())), flush=True)
    return 1 if survived else 0


if __name__ == "__main__":
    sys.exit(main())
