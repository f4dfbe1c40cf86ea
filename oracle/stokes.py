"""Closed-form homogeneous whole-space response (Stokes solution).

TEST INFRASTRUCTURE ONLY.  Used to pin the FP64 oracle to the physics of
Eq. 1 and Eq. 2 (Sec. 2.1) independently of any discretisation.

Formulas: Aki & Richards, Quantitative Seismology, eq. 4.23 (point force)
and eq. 4.29 (moment tensor), displacement for a source at the origin:

  force X(t) along axis j:
    u_i = (3 g_i g_j - d_ij) / (4 pi rho r^3) * I(t)
          + g_i g_j / (4 pi rho a^2 r) X(t - r/a)
          - (g_i g_j - d_ij) / (4 pi rho b^2 r) X(t - r/b)
  moment M_pq m(t):
    u_n = (15 g_n g_p g_q - 3 g_n d_pq - 3 g_p d_nq - 3 g_q d_np) / (4 pi rho r^4) I(t)
          + (6 g_n g_p g_q - g_n d_pq - g_p d_nq - g_q d_np) / (4 pi rho a^2 r^2) m(t - r/a)
          - (6 g_n g_p g_q - g_n d_pq - g_p d_nq - 2 g_q d_np) / (4 pi rho b^2 r^2) m(t - r/b)
          + g_n g_p g_q / (4 pi rho a^3 r) m'(t - r/a)
          - (g_n g_p g_q - d_np g_q) / (4 pi rho b^3 r) m'(t - r/b)
  with I(t) = int_{r/a}^{r/b} tau s(t - tau) d tau for the source function s.

The solver injects a *moment rate* r(t) (sigma -= dt M r / V) and a *force*
r(t) (v += dt b F r / V), and records particle *velocity*.  Velocity is the
time derivative of displacement, so:
  moment source -> velocity = displacement formula with m(t) := r(t);
  force source  -> velocity = displacement formula with X(t) := r'(t).
"""
from __future__ import annotations

import math

import numpy as np


def ricker(t, f0, t0):
    a = (math.pi * f0 * (np.asarray(t, np.float64) - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def ricker_dot(t, f0, t0):
    tt = np.asarray(t, np.float64) - t0
    c = (math.pi * f0) ** 2
    a = c * tt * tt
    return 2.0 * c * tt * (2.0 * a - 3.0) * np.exp(-a)


def _near_integral(s, t, r, a, b, nq=400):
    """I(t) = int_{r/a}^{r/b} tau s(t - tau) dtau by Gauss-Legendre."""
    x, w = np.polynomial.legendre.leggauss(nq)
    lo, hi = r / a, r / b
    tau = 0.5 * (hi - lo) * x + 0.5 * (hi + lo)
    ww = 0.5 * (hi - lo) * w
    return (s(t[:, None] - tau[None, :]) * tau[None, :]) @ ww


def force_velocity(t, xrel, F, rho, alpha, beta, f0, t0):
    """Velocity [3][len(t)] at offset xrel (m) from a point force F (N) with
    force time function r(t) (Ricker f0, t0)."""
    t = np.asarray(t, np.float64)
    r = float(np.linalg.norm(xrel))
    g = np.asarray(xrel, np.float64) / r
    X = lambda tt: ricker_dot(tt, f0, t0)          # noqa: E731
    I = _near_integral(X, t, r, alpha, beta)
    Xa, Xb = X(t - r / alpha), X(t - r / beta)
    out = np.zeros((3, t.size))
    c = 1.0 / (4.0 * math.pi * rho)
    for i in range(3):
        for j in range(3):
            if F[j] == 0.0:
                continue
            d = 1.0 if i == j else 0.0
            out[i] += F[j] * c * ((3 * g[i] * g[j] - d) / r ** 3 * I
                                  + g[i] * g[j] / (alpha ** 2 * r) * Xa
                                  - (g[i] * g[j] - d) / (beta ** 2 * r) * Xb)
    return out


def moment_velocity(t, xrel, M6, rho, alpha, beta, f0, t0):
    """Velocity [3][len(t)] at offset xrel (m) from a moment tensor
    (Mxx, Myy, Mzz, Mxy, Mxz, Myz) with moment-rate function r(t)."""
    t = np.asarray(t, np.float64)
    mxx, myy, mzz, mxy, mxz, myz = M6
    M = np.array([[mxx, mxy, mxz], [mxy, myy, myz], [mxz, myz, mzz]], np.float64)
    r = float(np.linalg.norm(xrel))
    g = np.asarray(xrel, np.float64) / r
    m = lambda tt: ricker(tt, f0, t0)              # noqa: E731
    md = lambda tt: ricker_dot(tt, f0, t0)         # noqa: E731
    I = _near_integral(m, t, r, alpha, beta)
    ma, mb = m(t - r / alpha), m(t - r / beta)
    mda, mdb = md(t - r / alpha), md(t - r / beta)
    d = np.eye(3)
    c = 1.0 / (4.0 * math.pi * rho)
    out = np.zeros((3, t.size))
    for n in range(3):
        for p in range(3):
            for q in range(3):
                if M[p, q] == 0.0:
                    continue
                ggg = g[n] * g[p] * g[q]
                near = 15 * ggg - 3 * g[n] * d[p, q] - 3 * g[p] * d[n, q] - 3 * g[q] * d[n, p]
                ip = 6 * ggg - g[n] * d[p, q] - g[p] * d[n, q] - g[q] * d[n, p]
                is_ = 6 * ggg - g[n] * d[p, q] - g[p] * d[n, q] - 2 * g[q] * d[n, p]
                fs = ggg - d[n, p] * g[q]
                out[n] += M[p, q] * c * (near / r ** 4 * I
                                         + ip / (alpha ** 2 * r ** 2) * ma
                                         - is_ / (beta ** 2 * r ** 2) * mb
                                         + ggg / (alpha ** 3 * r) * mda
                                         - fs / (beta ** 3 * r) * mdb)
    return out
