"""ctypes front end of the FP64 CPU oracle (``ews_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product path.  It
imports nothing from the CUDA package; both sides are fed the same seeded
arrays and compared afterwards.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ews_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liborc.so")

BND = {"none": 0, "sponge": 1, "cpml": 2}
KIND = {"moment": 0, "force": 1}
FIELDS = ("vx", "vy", "vz", "sxx", "syy", "szz", "sxy", "sxz", "syz")

SPONGE_ALPHA = 0.3
PML_R = 1e-3

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP, no FP contraction)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            P, D, I, L_ = C.c_void_p, C.c_double, C.c_int, C.c_long
            L.orc_create.restype = P
            L.orc_create.argtypes = [L_, L_, L_, D, D, D]
            L.orc_destroy.argtypes = [P]
            L.orc_set_medium.argtypes = [P, P, P, P]
            L.orc_set_free_surface.argtypes = [P, L_, D]
            L.orc_set_medium_coarse.argtypes = [P, L_, L_, L_, P, P, P]
            L.orc_vpmax.restype = D
            L.orc_vpmax.argtypes = [P]
            L.orc_set_boundary.argtypes = [P, I, I, D, D, D, D]
            L.orc_step_velocity.restype = I
            L.orc_step_velocity.argtypes = [P, D, I, P, P, D]
            L.orc_step_stress.restype = I
            L.orc_step_stress.argtypes = [P, D, I, P, P, D]
            L.orc_sample.restype = I
            L.orc_sample.argtypes = [P, I, P, P]
            L.orc_forward.restype = I
            L.orc_forward.argtypes = [P, I, D, I, P, P, P, I, P, P, I, C.c_uint, P]
            L.orc_get_state.argtypes = [P, P]
            L.orc_set_state.argtypes = [P, P]
            L.orc_get_psi.restype = I
            L.orc_get_psi.argtypes = [P, P]
            L.orc_get_medium.argtypes = [P, P]
            L.orc_energy.restype = D
            L.orc_energy.argtypes = [P, P]
            L.orc_gradient.restype = I
            L.orc_gradient.argtypes = [P, I, D, I, P, P, P, I, P, P, I, P, P, P]
            L.orc_tangent.restype = I
            L.orc_tangent.argtypes = [P, I, D, I, P, P, P, I, P, P, P, P, P]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.c_void_p)


def lame_from_velocities(vp, vs, rho):
    """lambda = rho (vp^2 - 2 vs^2), mu = rho vs^2, in FP64."""
    vp = np.asarray(vp, np.float64)
    vs = np.asarray(vs, np.float64)
    rho = np.asarray(rho, np.float64)
    mu = rho * vs * vs
    return rho * vp * vp - 2.0 * mu, mu, rho


class OracleSim:
    """One oracle simulation: grid, medium, boundary and wavefield state."""

    def __init__(self, nx, ny, nz, spacing):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.spacing = tuple(float(h) for h in spacing)
        self.n = self.nx * self.ny * self.nz
        self._L = lib()
        self._h = self._L.orc_create(self.nx, self.ny, self.nz, *self.spacing)
        self.boundary = "none"

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.orc_destroy(h)
            self._h = None

    # --- medium -------------------------------------------------------
    def set_free_surface(self, ks: int, eps: float = 1e-3):
        """Vacuum free surface above plane ks (reading R16); ks < 0 removes
        it.  Takes effect at the next set_medium_*."""
        self._L.orc_set_free_surface(self._h, int(ks), float(eps))

    def set_medium_lame(self, lam, mu, rho):
        arrs = [np.ascontiguousarray(a, np.float64).reshape(-1) for a in (lam, mu, rho)]
        for a in arrs:
            assert a.size == self.n
        self._L.orc_set_medium(self._h, *[_p(a) for a in arrs])

    def set_medium_vel(self, vp, vs, rho):
        self.set_medium_lame(*lame_from_velocities(vp, vs, rho))

    def set_medium_coarse(self, lam, mu, rho):
        """Medium on its own grid of [mz][my][mx] cells over the same box
        (reading R17: trilinear sampling at the staggered positions)."""
        arrs = [np.ascontiguousarray(a, np.float64) for a in (lam, mu, rho)]
        mz, my, mx = arrs[0].shape
        for a in arrs:
            assert a.shape == (mz, my, mx)
        self._L.orc_set_medium_coarse(self._h, mx, my, mz, *[_p(a) for a in arrs])

    @property
    def vpmax(self) -> float:
        return self._L.orc_vpmax(self._h)

    def medium(self) -> np.ndarray:
        out = np.zeros((8, self.n))
        self._L.orc_get_medium(self._h, _p(out))
        return out.reshape(8, self.nz, self.ny, self.nx)

    def set_boundary(self, kind: str, width: int = 0, dt: float = 0.0,
                     f0: float = 0.0, alpha: float = SPONGE_ALPHA, R: float = PML_R):
        self.boundary = kind
        self._L.orc_set_boundary(self._h, BND[kind], int(width), float(alpha),
                                 float(R), float(f0), float(dt))

    # --- state ----------------------------------------------------------
    def get_state(self) -> np.ndarray:
        out = np.zeros((9, self.n))
        self._L.orc_get_state(self._h, _p(out))
        return out.reshape(9, self.nz, self.ny, self.nx)

    def set_state(self, state):
        a = np.ascontiguousarray(state, np.float64).reshape(9, self.n)
        self._L.orc_set_state(self._h, _p(a))

    def get_psi(self) -> np.ndarray:
        out = np.zeros((18, self.n))
        if self._L.orc_get_psi(self._h, _p(out)) != 0:
            raise RuntimeError("no C-PML memory variables")
        return out.reshape(18, self.nz, self.ny, self.nx)

    # --- stepping -------------------------------------------------------
    def step_velocity(self, dt, src_kind=None, pos=None, comp=None, amp=0.0):
        k, p, c = self._src(src_kind, pos, comp)
        if self._L.orc_step_velocity(self._h, float(dt), k, _p(p), _p(c), float(amp)) != 0:
            raise ValueError("source outside the grid")

    def step_stress(self, dt, src_kind=None, pos=None, comp=None, amp=0.0):
        k, p, c = self._src(src_kind, pos, comp)
        if self._L.orc_step_stress(self._h, float(dt), k, _p(p), _p(c), float(amp)) != 0:
            raise ValueError("source outside the grid")

    @staticmethod
    def _src(kind, pos, comp):
        k = -1 if kind is None else KIND[kind]
        p = np.zeros(3) if pos is None else np.ascontiguousarray(pos, np.float64)
        c = np.zeros(6)
        if comp is not None:
            cc = np.asarray(comp, np.float64).ravel()
            c[:cc.size] = cc
        return k, p, c

    def sample(self, rec_pos) -> np.ndarray:
        r = np.ascontiguousarray(rec_pos, np.float64).reshape(-1, 3)
        out = np.zeros((3, r.shape[0]))
        if self._L.orc_sample(self._h, r.shape[0], _p(r), _p(out)) != 0:
            raise ValueError("receiver outside the grid")
        return out

    def energy(self, vprev) -> float:
        a = np.ascontiguousarray(vprev, np.float64).reshape(3, self.n)
        return self._L.orc_energy(self._h, _p(a))

    def forward(self, nt, dt, src_kind, pos, comp, wavelet, rec_pos,
                snap_every=0, snap_mask=0):
        """Full time loop from the current state; returns seis [3][nrec][nt]
        (and snapshots [nsnap][nmask][nz][ny][nx] when requested)."""
        k, p, c = self._src(src_kind, pos, comp)
        w = np.ascontiguousarray(wavelet, np.float64)
        assert w.size >= nt
        r = np.ascontiguousarray(rec_pos, np.float64).reshape(-1, 3)
        nrec = r.shape[0]
        seis = np.zeros((3, nrec, nt))
        nmask = bin(snap_mask).count("1")
        nsnap = nt // snap_every if snap_every > 0 else 0
        snap = np.zeros((max(nsnap, 1), max(nmask, 1), self.n)) if nsnap and nmask else None
        rc = self._L.orc_forward(self._h, int(nt), float(dt), k, _p(p), _p(c), _p(w),
                                 nrec, _p(r) if nrec else None, _p(seis),
                                 int(snap_every), C.c_uint(snap_mask),
                                 _p(snap) if snap is not None else None)
        if rc != 0:
            raise ValueError("source or receiver outside the grid")
        if snap is not None:
            return seis, snap.reshape(nsnap, nmask, self.nz, self.ny, self.nx)
        return seis


def gradient(prob, sadj, ckpt_every=0, nt=None, medium=None):
    """dL/d(lambda, mu, rho) per cell for dL/dseis = sadj ([3][nrec][nt]),
    FP64.  `medium` optionally overrides (lambda, mu, rho)."""
    nt = prob.nt if nt is None else nt
    s = OracleSim(prob.nx, prob.ny, prob.nz, prob.spacing)
    if prob.free_surface is not None:
        s.set_free_surface(*prob.free_surface)
    if medium is None:
        s.set_medium_vel(prob.vp, prob.vs, prob.rho)
    else:
        s.set_medium_lame(*medium)
    s.set_boundary(prob.boundary, prob.width, prob.dt, prob.f0)
    k, p, c = s._src(prob.src_kind, prob.src_pos, prob.src_comp)
    w = np.ascontiguousarray(prob.wavelet, np.float64)
    r = np.ascontiguousarray(prob.rec_pos, np.float64).reshape(-1, 3)
    a = np.ascontiguousarray(sadj, np.float64)
    assert a.shape == (3, r.shape[0], nt)
    g = np.zeros((3, s.n))
    rc = s._L.orc_gradient(s._h, int(nt), float(prob.dt), k, _p(p), _p(c), _p(w), r.shape[0],
                           _p(r), _p(a), int(ckpt_every), _p(g[0]), _p(g[1]), _p(g[2]))
    if rc != 0:
        raise ValueError(f"oracle gradient failed ({rc})")
    return g.reshape(3, s.nz, s.ny, s.nx)


def tangent(prob, dmodel, nt=None, medium=None):
    """Seismogram perturbation [3][nrec][nt] of the model perturbation
    dmodel = (dlambda, dmu, drho) (forward-mode derivative of the loop),
    FP64.  `medium` optionally overrides (lambda, mu, rho)."""
    nt = prob.nt if nt is None else nt
    s = OracleSim(prob.nx, prob.ny, prob.nz, prob.spacing)
    if prob.free_surface is not None:
        s.set_free_surface(*prob.free_surface)
    if medium is None:
        s.set_medium_vel(prob.vp, prob.vs, prob.rho)
    else:
        s.set_medium_lame(*medium)
    s.set_boundary(prob.boundary, prob.width, prob.dt, prob.f0)
    k, p, c = s._src(prob.src_kind, prob.src_pos, prob.src_comp)
    w = np.ascontiguousarray(prob.wavelet, np.float64)
    r = np.ascontiguousarray(prob.rec_pos, np.float64).reshape(-1, 3)
    d = [np.ascontiguousarray(a, np.float64).reshape(-1) for a in dmodel]
    out = np.zeros((3, r.shape[0], nt))
    rc = s._L.orc_tangent(s._h, int(nt), float(prob.dt), k, _p(p), _p(c), _p(w), r.shape[0],
                          _p(r), _p(d[0]), _p(d[1]), _p(d[2]), _p(out))
    if rc != 0:
        raise ValueError(f"oracle tangent failed ({rc})")
    return out


def run_problem(prob, nt=None, state=None, boundary=None, snap_every=0, snap_mask=0,
                return_sim=False):
    """Run a ``synth.Problem`` through the oracle; returns seis [3][nrec][nt]."""
    nt = prob.nt if nt is None else nt
    s = OracleSim(prob.nx, prob.ny, prob.nz, prob.spacing)
    if prob.free_surface is not None:
        s.set_free_surface(*prob.free_surface)
    if prob.coarse_medium is not None:
        s.set_medium_coarse(*prob.coarse_medium)
    else:
        s.set_medium_vel(prob.vp, prob.vs, prob.rho)
    s.set_boundary(boundary or prob.boundary, prob.width, prob.dt, prob.f0)
    if state is not None:
        s.set_state(state)
    out = s.forward(nt, prob.dt, prob.src_kind, prob.src_pos, prob.src_comp,
                    prob.wavelet, prob.rec_pos, snap_every, snap_mask)
    return (out, s) if return_sim else out
