"""Brute-force restatement of the scheme as assembled sparse operators.

TEST INFRASTRUCTURE ONLY.  This is a second, structurally different statement
of the same discrete method as ``ews_oracle.c`` (which works pointwise with
stencils): here every operator is an explicit sparse matrix, assembled from
1-D building blocks, and the time loop is matrix-vector products.  It exists
to pin the C oracle on tiny grids (8^3 and similar).

Nothing is typed twice from the C code:
  * the staggered derivative weights are *derived* by solving the moment
    (Taylor) conditions for a 4-point stencil on the half-integer offsets
    -3/2, -1/2, +1/2, +3/2 (Sec. 2.1.2, Eq. 4);
  * interpolation weights for sources and receivers come from ``np.interp``
    applied to unit vectors (Sec. 2.4), and the medium averages are sparse
    averaging matrices (Sec. 2.2.1);
  * the 3-D operators are Kronecker products for the C-ordered [z][y][x]
    layout.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def staggered_weights(offsets=(-1.5, -0.5, 0.5, 1.5)) -> np.ndarray:
    """Weights w of f'(0) ~ sum_m w_m f(o_m) / h on the given offsets, exact
    for polynomials of the highest degree they allow (solve the moment
    conditions).  Four offsets give Eq. 4; two give the 2nd-order difference
    the free surface of Sec. 2.5 switches to."""
    o = np.asarray(offsets, np.float64)
    A = np.vstack([o ** p for p in range(o.size)])
    rhs = np.zeros(o.size)
    rhs[1] = 1.0
    return np.linalg.solve(A, rhs)


def d1(n: int, h: float, shifted_output: bool, surface: float | None = None) -> sp.csr_matrix:
    """1-D staggered derivative, n x n, zero outside the grid.

    shifted_output=True : input on integer points, output at i + 1/2.
    shifted_output=False: input on half points (element m at m + 1/2),
                          output at integer point i.
    surface: position (in cells) of a free-surface plane; an output whose
    four taps lie on both sides of it uses the two inner taps only.
    """
    wide = (-1.5, -0.5, 0.5, 1.5)
    rows, cols, vals = [], [], []
    for i in range(n):
        out_pos = i + 0.5 if shifted_output else float(i)
        offs = wide
        if surface is not None and out_pos + wide[0] < surface < out_pos + wide[-1]:
            offs = (-0.5, 0.5)
        w = staggered_weights(offs)
        for m, off in enumerate(offs):
            in_pos = out_pos + off
            col = int(round(in_pos)) if shifted_output else int(round(in_pos - 0.5))
            if 0 <= col < n:
                rows.append(i)
                cols.append(col)
                vals.append(w[m] / h)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def avg1(n: int) -> sp.csr_matrix:
    """Mean of element i and i+1 (index clamped at the top edge)."""
    rows, cols, vals = [], [], []
    for i in range(n):
        for c in (i, min(i + 1, n - 1)):
            rows.append(i)
            cols.append(c)
            vals.append(0.5)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def interp1(n: int, u: float) -> np.ndarray:
    """Linear-interpolation weights of fractional index u on 0..n-1."""
    eye = np.eye(n)
    return np.array([np.interp(u, np.arange(n), eye[m]) for m in range(n)])


class Brute:
    FIELD_OFF = {
        "vx": (0.5, 0, 0), "vy": (0, 0.5, 0), "vz": (0, 0, 0.5),
        "sxx": (0, 0, 0), "syy": (0, 0, 0), "szz": (0, 0, 0),
        "sxy": (0.5, 0.5, 0), "sxz": (0.5, 0, 0.5), "syz": (0, 0.5, 0.5),
    }
    NAMES = ("vx", "vy", "vz", "sxx", "syy", "szz", "sxy", "sxz", "syz")

    def __init__(self, nx, ny, nz, spacing, lam, mu, rho, surface=None):
        """surface: optional (ks, eps), a free surface by the vacuum
        formulation of Sec. 2.5: the cells above plane ks get eps times the
        medium of the cell below the surface in their column, the xz / yz
        shear points on the plane z = ks - 1/2 take the harmonic mean of
        their 4 cells, and the z-derivatives whose stencil straddles that
        plane drop to 2nd order."""
        self.nx, self.ny, self.nz = nx, ny, nz
        self.h = spacing
        self.N = nx * ny * nz
        Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)

        def kron3(az, ay, ax):
            return sp.kron(az, sp.kron(ay, ax)).tocsr()

        hx, hy, hz = spacing
        # P: forward-shifted derivative (integer -> half); M: half -> integer
        self.Px = kron3(Iz, Iy, d1(nx, hx, True))
        self.Mx = kron3(Iz, Iy, d1(nx, hx, False))
        self.Py = kron3(Iz, d1(ny, hy, True), Ix)
        self.My = kron3(Iz, d1(ny, hy, False), Ix)
        zs = None if surface is None else surface[0] - 0.5
        self.Pz = kron3(d1(nz, hz, True, zs), Iy, Ix)
        self.Mz = kron3(d1(nz, hz, False, zs), Iy, Ix)

        arrs = []
        for a in (lam, mu, rho):
            a = np.array(a, np.float64).reshape(nz, ny, nx)
            if surface is not None:
                ks, eps = surface
                a[:ks] = eps * a[ks]
            arrs.append(a.ravel())
        lam, mu, rho = arrs
        self._rho = rho
        Ax = kron3(Iz, Iy, avg1(nx))
        Ay = kron3(Iz, avg1(ny), Ix)
        Az = kron3(avg1(nz), Iy, Ix)
        self.b = {"vx": 1.0 / (Ax @ rho), "vy": 1.0 / (Ay @ rho), "vz": 1.0 / (Az @ rho)}
        self.lam = lam
        self.mu = mu
        self.mu_s = {"sxy": Ax @ (Ay @ mu), "sxz": Ax @ (Az @ mu), "syz": Ay @ (Az @ mu)}
        if surface is not None and surface[0] >= 1:
            # harmonic means on the surface plane: 4 / (sum of 1/mu) is the
            # reciprocal of the arithmetic mean of 1/mu
            on = (np.arange(self.N) // (nx * ny)) == surface[0] - 1
            inv = 1.0 / mu
            for key, A in (("sxz", Ax @ Az), ("syz", Ay @ Az)):
                self.mu_s[key] = np.where(on, 1.0 / (A @ inv), self.mu_s[key])
        self.gain = np.ones(self.N)
        self.pml = None
        self.f = {k: np.zeros(self.N) for k in self.NAMES}

    # --- boundaries -------------------------------------------------------
    def _axis_index(self):
        k, j, i = np.meshgrid(np.arange(self.nz), np.arange(self.ny), np.arange(self.nx),
                              indexing="ij")
        return i.ravel(), j.ravel(), k.ravel()

    def set_sponge(self, width: int, alpha: float = 0.3):
        idx = self._axis_index()
        g = np.ones(self.N)
        for a, n in enumerate((self.nx, self.ny, self.nz)):
            d = np.minimum(idx[a], n - 1 - idx[a])
            ga = np.where(d < width, np.exp(-(alpha * (width - d) / width) ** 2), 1.0)
            g *= ga
        self.gain = g

    def set_cpml(self, width: int, dt: float, f0: float, R: float = 1e-3):
        vpmax = float(np.max(np.sqrt((self.lam + 2 * self.mu) / np.asarray(
            self._rho_cells(), np.float64))))
        idx = self._axis_index()
        coef = []
        for a, n in enumerate((self.nx, self.ny, self.nz)):
            i = idx[a]
            inside = (i < width) | (i >= n - width)
            q = np.where(i < width, (width - i) / width, (i - (n - 1 - width)) / width)
            q = np.where(inside, q, 0.0)
            L = width * self.h[a]
            dd = -3.0 * vpmax * np.log(R) / (2.0 * L) * q * q
            al = np.pi * f0 * (1.0 - q)
            b = np.exp(-(dd + al) * dt)
            with np.errstate(invalid="ignore", divide="ignore"):
                aa = np.where(dd + al > 0, dd * (b - 1.0) / (dd + al), 0.0)
            coef.append((inside, aa, b))
        self.pml = {"coef": coef, "psi": {}}

    def _rho_cells(self):
        return self._rho

    def set_rho_cells(self, rho):
        self._rho = np.asarray(rho, np.float64).ravel()

    def _d(self, key, axis, val):
        """Apply the C-PML memory variable of one derivative term."""
        if self.pml is None:
            return val
        inside, a, b = self.pml["coef"][axis]
        psi = self.pml["psi"].setdefault(key, np.zeros(self.N))
        psi[:] = np.where(inside, b * psi + a * val, 0.0)
        return val + psi

    # --- sources and receivers (Sec. 2.4; transposed for injection) --------
    def point_weights(self, name, pos):
        ox, oy, oz = self.FIELD_OFF[name]
        wx = interp1(self.nx, pos[0] / self.h[0] - ox)
        wy = interp1(self.ny, pos[1] / self.h[1] - oy)
        wz = interp1(self.nz, pos[2] / self.h[2] - oz)
        return np.einsum("k,j,i->kji", wz, wy, wx).ravel()

    # --- one time step ----------------------------------------------------
    def step(self, dt, kind=None, pos=None, comp=None, amp=0.0):
        f = self.f
        vol = self.h[0] * self.h[1] * self.h[2]
        rx = (self._d("vx_x", 0, self.Px @ f["sxx"]) + self._d("vx_y", 1, self.My @ f["sxy"])
              + self._d("vx_z", 2, self.Mz @ f["sxz"]))
        ry = (self._d("vy_x", 0, self.Mx @ f["sxy"]) + self._d("vy_y", 1, self.Py @ f["syy"])
              + self._d("vy_z", 2, self.Mz @ f["syz"]))
        rz = (self._d("vz_x", 0, self.Mx @ f["sxz"]) + self._d("vz_y", 1, self.My @ f["syz"])
              + self._d("vz_z", 2, self.Pz @ f["szz"]))
        for name, r in (("vx", rx), ("vy", ry), ("vz", rz)):
            f[name] = f[name] + dt * self.b[name] * r
        if kind == "force":
            for c, name in enumerate(("vx", "vy", "vz")):
                f[name] = f[name] + (self.point_weights(name, pos) * dt * self.b[name]
                                     * comp[c] * amp / vol)
        for name in ("vx", "vy", "vz"):
            f[name] = f[name] * self.gain

        exx = self._d("exx", 0, self.Mx @ f["vx"])
        eyy = self._d("eyy", 1, self.My @ f["vy"])
        ezz = self._d("ezz", 2, self.Mz @ f["vz"])
        gxy = self._d("sxy_y", 1, self.Py @ f["vx"]) + self._d("sxy_x", 0, self.Px @ f["vy"])
        gxz = self._d("sxz_z", 2, self.Pz @ f["vx"]) + self._d("sxz_x", 0, self.Px @ f["vz"])
        gyz = self._d("syz_z", 2, self.Pz @ f["vy"]) + self._d("syz_y", 1, self.Py @ f["vz"])
        lam, mu = self.lam, self.mu
        tr = exx + eyy + ezz
        f["sxx"] = f["sxx"] + dt * (lam * tr + 2 * mu * exx)
        f["syy"] = f["syy"] + dt * (lam * tr + 2 * mu * eyy)
        f["szz"] = f["szz"] + dt * (lam * tr + 2 * mu * ezz)
        f["sxy"] = f["sxy"] + dt * self.mu_s["sxy"] * gxy
        f["sxz"] = f["sxz"] + dt * self.mu_s["sxz"] * gxz
        f["syz"] = f["syz"] + dt * self.mu_s["syz"] * gyz
        if kind == "moment":
            for c, name in enumerate(("sxx", "syy", "szz", "sxy", "sxz", "syz")):
                f[name] = f[name] - self.point_weights(name, pos) * dt * comp[c] * amp / vol
        for name in ("sxx", "syy", "szz", "sxy", "sxz", "syz"):
            f[name] = f[name] * self.gain

    def sample_matrix(self, rec_pos):
        return {name: np.stack([self.point_weights(name, r) for r in rec_pos])
                for name in ("vx", "vy", "vz")}

    def forward(self, nt, dt, kind, pos, comp, wavelet, rec_pos):
        S = self.sample_matrix(rec_pos)
        seis = np.zeros((3, len(rec_pos), nt))
        for n in range(nt):
            self.step(dt, kind, pos, comp, wavelet[n])
            # The stress half-step leaves the velocities alone, so v after
            # the whole step is v^{n+1/2}, the value the receivers record.
            for c, name in enumerate(("vx", "vy", "vz")):
                seis[c, :, n] = S[name] @ self.f[name]
        return seis

    def state(self):
        return np.stack([self.f[k].reshape(self.nz, self.ny, self.nx) for k in self.NAMES])

    def set_state(self, st):
        for q, k in enumerate(self.NAMES):
            self.f[k] = np.asarray(st[q], np.float64).ravel().copy()


def from_velocities(nx, ny, nz, spacing, vp, vs, rho, surface=None) -> Brute:
    vp = np.asarray(vp, np.float64)
    vs = np.asarray(vs, np.float64)
    rho = np.asarray(rho, np.float64)
    mu = rho * vs ** 2
    lam = rho * vp ** 2 - 2 * mu
    return Brute(nx, ny, nz, spacing, lam, mu, rho, surface)
