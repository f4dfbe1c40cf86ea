// ews_adjoint.cu -- adjoint (reverse-mode) kernels of the staggered scheme.
//
// Two formulations of the same exact discrete adjoint.
//
// (1) Transformed variables (used whenever mu > 0 everywhere).  With the
// true adjoint a of v and s of sigma, the variables alpha = B G a and
// tau = G C s obey  alpha <- G (alpha - dt B Dsig(tau)),
// tau <- G (tau - dt C Dv(alpha)):  the forward step with dt -> -dt, so the
// reverse sweep runs the TMA stencil passes of ews_stencil.cu on a second
// set of fields.  The receiver residual enters alpha like a point force
// (k_adj_inject).  The gradient needs G s = C^-1 tau and G a = alpha / B;
// the pointwise inverses are applied once, in k_grad_finalize_t, to time
// sums accumulated by the reverse velocity pass:
//   acc0 = sum dt tr(E) tr(tau),  acc1 = sum dt E_ii tau_ii,
//   acc2..4 = sum dt gamma tau at the xy, xz, yz points,
//   acc5..7 = sum (v^{n+1/2} / G - v^{n-1/2}) alpha at the v points,
// with E = Dv(v^{n+1/2}) the forward strain rates.  Then
//   dJ/dlambda = acc0 / (3 lambda + 2 mu),
//   dJ/dmu     = (acc1 - lambda acc0 / (3 lambda + 2 mu)) / mu + shear sums / mu_mean,
//   dJ/drho    = -1/2 sum over the v points of the cell of acc5..7.
// C^-1 does not exist where mu = 0, so media with a fluid cell use (2).
//
// (2) Direct variables (naive kernels below).  The forward step n is  V: v' = G (v + dt B Dsig(sigma) + f_n),  R: s_n = S v',
// T: sigma' = G (sigma + dt C Dv(v') - m_n),  with Dv = -Dsig^T (zero
// exterior, Eq. 4 operators).  Going back through T, R, V with adjoint
// states P (velocity-like, 3 fields) and Q (stress-like, 6 fields) kept so
// that the true velocity adjoint is G P:
//   k_adj_stress  (reverse of T):  w = G Q;  P <- G P - dt Dsig(C w);
//                                  acc_C += dt Dv(v^{n+1/2}) (x) w
//   k_adj_record  (reverse of R):  P <- P + S^T sadj_n
//   k_adj_velocity (reverse of V): u = G P;  Q <- G Q - dt Dv(B u);
//                                  acc_B += (v^{n+1/2} / G - v^{n-1/2}) u / B
// (the last line is dt Dsig(sigma^n) u + (f_n / B) u with Dsig(sigma^n) taken
// from the velocity history; the force terms cancel).  Each kernel reads
// neighbours only of the field it does not write, so updates are in place.
// Accumulators: FP32 within a checkpoint segment, flushed into FP64 across
// segments; k_grad_finalize applies the chain rule of the staggered means
// (mu: 4-cell shear means, rho: 2-cell means inverted).
#include "ews_internal.cuh"
#include "ews_ops.cuh"

namespace ews {

namespace {

__device__ __forceinline__ long long cidx(const DevGrid& g, int i, int j, int k) {
    return (long long)k * g.plane + (long long)j * g.pitch + i;
}
__device__ __forceinline__ bool inside(const DevGrid& g, int i, int j, int k) {
    return (unsigned)i < (unsigned)g.nx && (unsigned)j < (unsigned)g.ny && (unsigned)k < (unsigned)g.nz;
}
__device__ __forceinline__ float med(const float* __restrict__ m, const DevGrid& g, int i, int j,
                                     int k) {
    return __ldg(m + cidx(g, min(i, g.nx - 1), min(j, g.ny - 1), min(k, g.nz - 1)));
}
template <int BND>
__device__ __forceinline__ float gain(const DevBoundary& B, int i, int j, int k) {
    if (BND != BND_SPONGE) return 1.0f;
    return __ldg(B.g[0] + i) * __ldg(B.g[1] + j) * __ldg(B.g[2] + k);
}
__device__ __forceinline__ float d4(float c1, float c2, float m32, float m12, float p12, float p32) {
    return c1 * (p12 - m12) + c2 * (p32 - m32);
}

// tau = C (G Q) at a normal-stress point (components xx, yy, zz) or a shear
// point (xy, xz, yz); zero outside the grid (zero exterior).
template <int BND>
__device__ __forceinline__ float tau_n(const AdjFields& A, const DevMedium& M, const DevBoundary& B,
                                       const DevGrid& g, int c, int i, int j, int k) {
    if (!inside(g, i, j, k)) return 0.0f;
    const long long o = cidx(g, i, j, k);
    const float lam = __ldg(M.lam + o), mu = __ldg(M.mu + o);
    const float q0 = A.q[0][o], q1 = A.q[1][o], q2 = A.q[2][o];
    const float qc = c == 0 ? q0 : (c == 1 ? q1 : q2);
    return gain<BND>(B, i, j, k) * (2.0f * mu * qc + lam * (q0 + q1 + q2));
}
template <int BND>
__device__ __forceinline__ float tau_s(const AdjFields& A, const DevMedium& M, const DevBoundary& B,
                                       const DevGrid& g, int c, int i, int j, int k) {
    if (!inside(g, i, j, k)) return 0.0f;
    const long long o = cidx(g, i, j, k);
    const float m0 = med(M.mu, g, i, j, k);
    float mb;
    if (c == 0) mb = 0.25f * (m0 + med(M.mu, g, i + 1, j, k) + med(M.mu, g, i, j + 1, k) + med(M.mu, g, i + 1, j + 1, k));
    else if (c == 1) mb = 0.25f * (m0 + med(M.mu, g, i + 1, j, k) + med(M.mu, g, i, j, k + 1) + med(M.mu, g, i + 1, j, k + 1));
    else mb = 0.25f * (m0 + med(M.mu, g, i, j + 1, k) + med(M.mu, g, i, j, k + 1) + med(M.mu, g, i, j + 1, k + 1));
    return gain<BND>(B, i, j, k) * mb * A.q[3 + c][o];
}

// q = B (G P) at a v point of component c; zero outside the grid.
template <int BND>
__device__ __forceinline__ float qv(const AdjFields& A, const DevMedium& M, const DevBoundary& B,
                                    const DevGrid& g, int c, int i, int j, int k) {
    if (!inside(g, i, j, k)) return 0.0f;
    const float r0 = med(M.rho, g, i, j, k);
    const float r1 = med(M.rho, g, i + (c == 0), j + (c == 1), k + (c == 2));
    return gain<BND>(B, i, j, k) * 2.0f / (r0 + r1) * A.p[c][cidx(g, i, j, k)];
}

__device__ __forceinline__ float hv(const float* __restrict__ f, const DevGrid& g, int i, int j, int k) {
    return inside(g, i, j, k) ? __ldg(f + cidx(g, i, j, k)) : 0.0f;
}

template <int BND>
__global__ void __launch_bounds__(256) k_adj_stress(DevGrid g, AdjFields A, DevMedium M,
                                                    DevBoundary B, const float* __restrict__ vh0,
                                                    const float* __restrict__ vh1,
                                                    const float* __restrict__ vh2, float dt) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const long long o = cidx(g, i, j, k);
    // Dsig(tau) at the three v points of this cell
    const float dvx = d4(g.c1x, g.c2x, tau_n<BND>(A, M, B, g, 0, i - 1, j, k), tau_n<BND>(A, M, B, g, 0, i, j, k),
                         tau_n<BND>(A, M, B, g, 0, i + 1, j, k), tau_n<BND>(A, M, B, g, 0, i + 2, j, k)) +
                      d4(g.c1y, g.c2y, tau_s<BND>(A, M, B, g, 0, i, j - 2, k), tau_s<BND>(A, M, B, g, 0, i, j - 1, k),
                         tau_s<BND>(A, M, B, g, 0, i, j, k), tau_s<BND>(A, M, B, g, 0, i, j + 1, k)) +
                      d4(g.c1z, g.c2z, tau_s<BND>(A, M, B, g, 1, i, j, k - 2), tau_s<BND>(A, M, B, g, 1, i, j, k - 1),
                         tau_s<BND>(A, M, B, g, 1, i, j, k), tau_s<BND>(A, M, B, g, 1, i, j, k + 1));
    const float dvy = d4(g.c1x, g.c2x, tau_s<BND>(A, M, B, g, 0, i - 2, j, k), tau_s<BND>(A, M, B, g, 0, i - 1, j, k),
                         tau_s<BND>(A, M, B, g, 0, i, j, k), tau_s<BND>(A, M, B, g, 0, i + 1, j, k)) +
                      d4(g.c1y, g.c2y, tau_n<BND>(A, M, B, g, 1, i, j - 1, k), tau_n<BND>(A, M, B, g, 1, i, j, k),
                         tau_n<BND>(A, M, B, g, 1, i, j + 1, k), tau_n<BND>(A, M, B, g, 1, i, j + 2, k)) +
                      d4(g.c1z, g.c2z, tau_s<BND>(A, M, B, g, 2, i, j, k - 2), tau_s<BND>(A, M, B, g, 2, i, j, k - 1),
                         tau_s<BND>(A, M, B, g, 2, i, j, k), tau_s<BND>(A, M, B, g, 2, i, j, k + 1));
    const float dvz = d4(g.c1x, g.c2x, tau_s<BND>(A, M, B, g, 1, i - 2, j, k), tau_s<BND>(A, M, B, g, 1, i - 1, j, k),
                         tau_s<BND>(A, M, B, g, 1, i, j, k), tau_s<BND>(A, M, B, g, 1, i + 1, j, k)) +
                      d4(g.c1y, g.c2y, tau_s<BND>(A, M, B, g, 2, i, j - 2, k), tau_s<BND>(A, M, B, g, 2, i, j - 1, k),
                         tau_s<BND>(A, M, B, g, 2, i, j, k), tau_s<BND>(A, M, B, g, 2, i, j + 1, k)) +
                      d4(g.c1z, g.c2z, tau_n<BND>(A, M, B, g, 2, i, j, k - 1), tau_n<BND>(A, M, B, g, 2, i, j, k),
                         tau_n<BND>(A, M, B, g, 2, i, j, k + 1), tau_n<BND>(A, M, B, g, 2, i, j, k + 2));
    const float G = gain<BND>(B, i, j, k);
    // strain rates of v^{n+1/2} at this cell's stress points (Eq. 2 terms)
    const float exx = d4(g.c1x, g.c2x, hv(vh0, g, i - 2, j, k), hv(vh0, g, i - 1, j, k), hv(vh0, g, i, j, k), hv(vh0, g, i + 1, j, k));
    const float eyy = d4(g.c1y, g.c2y, hv(vh1, g, i, j - 2, k), hv(vh1, g, i, j - 1, k), hv(vh1, g, i, j, k), hv(vh1, g, i, j + 1, k));
    const float ezz = d4(g.c1z, g.c2z, hv(vh2, g, i, j, k - 2), hv(vh2, g, i, j, k - 1), hv(vh2, g, i, j, k), hv(vh2, g, i, j, k + 1));
    const float gxy = d4(g.c1y, g.c2y, hv(vh0, g, i, j - 1, k), hv(vh0, g, i, j, k), hv(vh0, g, i, j + 1, k), hv(vh0, g, i, j + 2, k)) +
                      d4(g.c1x, g.c2x, hv(vh1, g, i - 1, j, k), hv(vh1, g, i, j, k), hv(vh1, g, i + 1, j, k), hv(vh1, g, i + 2, j, k));
    const float gxz = d4(g.c1z, g.c2z, hv(vh0, g, i, j, k - 1), hv(vh0, g, i, j, k), hv(vh0, g, i, j, k + 1), hv(vh0, g, i, j, k + 2)) +
                      d4(g.c1x, g.c2x, hv(vh2, g, i - 1, j, k), hv(vh2, g, i, j, k), hv(vh2, g, i + 1, j, k), hv(vh2, g, i + 2, j, k));
    const float gyz = d4(g.c1z, g.c2z, hv(vh1, g, i, j, k - 1), hv(vh1, g, i, j, k), hv(vh1, g, i, j, k + 1), hv(vh1, g, i, j, k + 2)) +
                      d4(g.c1y, g.c2y, hv(vh2, g, i, j - 1, k), hv(vh2, g, i, j, k), hv(vh2, g, i, j + 1, k), hv(vh2, g, i, j + 2, k));
    const float w0 = G * A.q[0][o], w1 = G * A.q[1][o], w2 = G * A.q[2][o];
    A.acc[0][o] += dt * (exx + eyy + ezz) * (w0 + w1 + w2);
    A.acc[1][o] += dt * 2.0f * (exx * w0 + eyy * w1 + ezz * w2);
    A.acc[2][o] += dt * gxy * G * A.q[3][o];
    A.acc[3][o] += dt * gxz * G * A.q[4][o];
    A.acc[4][o] += dt * gyz * G * A.q[5][o];
    A.p[0][o] = G * A.p[0][o] - dt * dvx;
    A.p[1][o] = G * A.p[1][o] - dt * dvy;
    A.p[2][o] = G * A.p[2][o] - dt * dvz;
}

template <int BND>
__global__ void __launch_bounds__(256) k_adj_velocity(DevGrid g, AdjFields A, DevMedium M,
                                                      DevBoundary B, const float* __restrict__ vn,
                                                      const float* __restrict__ vp, size_t fstride,
                                                      float dt) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const long long o = cidx(g, i, j, k);
    // strain rates of q = B G P at this cell's stress points
    const float exx = d4(g.c1x, g.c2x, qv<BND>(A, M, B, g, 0, i - 2, j, k), qv<BND>(A, M, B, g, 0, i - 1, j, k),
                         qv<BND>(A, M, B, g, 0, i, j, k), qv<BND>(A, M, B, g, 0, i + 1, j, k));
    const float eyy = d4(g.c1y, g.c2y, qv<BND>(A, M, B, g, 1, i, j - 2, k), qv<BND>(A, M, B, g, 1, i, j - 1, k),
                         qv<BND>(A, M, B, g, 1, i, j, k), qv<BND>(A, M, B, g, 1, i, j + 1, k));
    const float ezz = d4(g.c1z, g.c2z, qv<BND>(A, M, B, g, 2, i, j, k - 2), qv<BND>(A, M, B, g, 2, i, j, k - 1),
                         qv<BND>(A, M, B, g, 2, i, j, k), qv<BND>(A, M, B, g, 2, i, j, k + 1));
    const float gxy = d4(g.c1y, g.c2y, qv<BND>(A, M, B, g, 0, i, j - 1, k), qv<BND>(A, M, B, g, 0, i, j, k),
                         qv<BND>(A, M, B, g, 0, i, j + 1, k), qv<BND>(A, M, B, g, 0, i, j + 2, k)) +
                      d4(g.c1x, g.c2x, qv<BND>(A, M, B, g, 1, i - 1, j, k), qv<BND>(A, M, B, g, 1, i, j, k),
                         qv<BND>(A, M, B, g, 1, i + 1, j, k), qv<BND>(A, M, B, g, 1, i + 2, j, k));
    const float gxz = d4(g.c1z, g.c2z, qv<BND>(A, M, B, g, 0, i, j, k - 1), qv<BND>(A, M, B, g, 0, i, j, k),
                         qv<BND>(A, M, B, g, 0, i, j, k + 1), qv<BND>(A, M, B, g, 0, i, j, k + 2)) +
                      d4(g.c1x, g.c2x, qv<BND>(A, M, B, g, 2, i - 1, j, k), qv<BND>(A, M, B, g, 2, i, j, k),
                         qv<BND>(A, M, B, g, 2, i + 1, j, k), qv<BND>(A, M, B, g, 2, i + 2, j, k));
    const float gyz = d4(g.c1z, g.c2z, qv<BND>(A, M, B, g, 1, i, j, k - 1), qv<BND>(A, M, B, g, 1, i, j, k),
                         qv<BND>(A, M, B, g, 1, i, j, k + 1), qv<BND>(A, M, B, g, 1, i, j, k + 2)) +
                      d4(g.c1y, g.c2y, qv<BND>(A, M, B, g, 2, i, j - 1, k), qv<BND>(A, M, B, g, 2, i, j, k),
                         qv<BND>(A, M, B, g, 2, i, j + 1, k), qv<BND>(A, M, B, g, 2, i, j + 2, k));
    const float G = gain<BND>(B, i, j, k);
    A.q[0][o] = G * A.q[0][o] - dt * exx;
    A.q[1][o] = G * A.q[1][o] - dt * eyy;
    A.q[2][o] = G * A.q[2][o] - dt * ezz;
    A.q[3][o] = G * A.q[3][o] - dt * gxy;
    A.q[4][o] = G * A.q[4][o] - dt * gxz;
    A.q[5][o] = G * A.q[5][o] - dt * gyz;
    // buoyancy gradient: (v^{n+1/2} / G - v^{n-1/2}) (G P) / b at the v points
    const float r0 = med(M.rho, g, i, j, k);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float r1 = med(M.rho, g, i + (c == 0), j + (c == 1), k + (c == 2));
        const float binv = 0.5f * (r0 + r1);
        const float dv = __ldg(vn + c * fstride + o) / G - __ldg(vp + c * fstride + o);
        A.acc[5 + c][o] += dv * G * A.p[c][o] * binv;
    }
}

// Receiver residual injection (transpose of k_record).
__global__ void k_adj_record(DevGrid g, AdjFields A, const Tap* __restrict__ taps, int nrec,
                             const float* __restrict__ sadj, int ld, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * nrec) return;
    const float a = __ldg(sadj + (long long)t * ld + n);
    const Tap* tp = taps + 8 * t;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const Tap q = tp[m];
        atomicAdd(A.p[q.q] + cidx(g, q.i, q.j, q.k), q.w * a);
    }
}

// acc64 += acc32; acc32 = 0 (8 accumulators).
__global__ void k_acc_flush(DevGrid g, AdjFields A) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    ops::flush_cell(A, cidx(g, i, j, k));
}

// Chain rule of the staggered means; output dense [nz][ny][nx].
__global__ void k_grad_finalize(DevGrid g, AdjFields A, DevMedium M, float* __restrict__ glam,
                                float* __restrict__ gmu, float* __restrict__ grho) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const long long o = cidx(g, i, j, k);
    double mu = A.acc64[1][o];
    double rho = 0.0;
    // shear means: point (a, b) of a plane uses cells a, min(a+1), b, min(b+1)
    for (int da = -1; da <= 0; ++da)
        for (int db = -1; db <= 0; ++db) {
            // xy: (i+da, j+db, k)
            int a = i + da, b = j + db;
            if (a >= 0 && b >= 0) {
                const int ap = min(a + 1, g.nx - 1), bp = min(b + 1, g.ny - 1);
                const int mult = (a == i && b == j) + (ap == i && b == j) + (a == i && bp == j) + (ap == i && bp == j);
                if (mult) mu += 0.25 * mult * A.acc64[2][cidx(g, a, b, k)];
            }
            // xz: (i+da, j, k+db)
            a = i + da; b = k + db;
            if (a >= 0 && b >= 0) {
                const int ap = min(a + 1, g.nx - 1), bp = min(b + 1, g.nz - 1);
                const int mult = (a == i && b == k) + (ap == i && b == k) + (a == i && bp == k) + (ap == i && bp == k);
                if (mult) mu += 0.25 * mult * A.acc64[3][cidx(g, a, j, b)];
            }
            // yz: (i, j+da, k+db)
            a = j + da; b = k + db;
            if (a >= 0 && b >= 0) {
                const int ap = min(a + 1, g.ny - 1), bp = min(b + 1, g.nz - 1);
                const int mult = (a == j && b == k) + (ap == j && b == k) + (a == j && bp == k) + (ap == j && bp == k);
                if (mult) mu += 0.25 * mult * A.acc64[4][cidx(g, i, a, b)];
            }
        }
    // buoyancy b = 2 / (rho(a) + rho(min(a+1))) along each axis
    for (int c = 0; c < 3; ++c)
        for (int d = -1; d <= 0; ++d) {
            const int ii = i + (c == 0 ? d : 0), jj = j + (c == 1 ? d : 0), kk = k + (c == 2 ? d : 0);
            if (ii < 0 || jj < 0 || kk < 0) continue;
            const int a = c == 0 ? ii : (c == 1 ? jj : kk);
            const int n = c == 0 ? g.nx : (c == 1 ? g.ny : g.nz);
            const int self = c == 0 ? i : (c == 1 ? j : k);
            const int ap = min(a + 1, n - 1);
            const int mult = (a == self) + (ap == self);
            if (!mult) continue;
            const double r0 = med(M.rho, g, ii, jj, kk);
            const double r1 = med(M.rho, g, ii + (c == 0), jj + (c == 1), kk + (c == 2));
            const double b = 2.0 / (r0 + r1);
            rho += -0.5 * b * b * mult * A.acc64[5 + c][cidx(g, ii, jj, kk)];
        }
    const long long od = ((long long)k * g.ny + j) * g.nx + i;
    glam[od] = (float)A.acc64[0][o];
    gmu[od] = (float)mu;
    grho[od] = (float)rho;
}

// Transformed formulation: residual injection alpha += G B S^T sadj_n (one
// thread per component and receiver, 8 taps each).
__global__ void k_adj_inject(DevGrid g, AdjFields A, DevMedium M, DevBoundary B,
                             const Tap* __restrict__ taps, int nrec,
                             const float* __restrict__ sadj, int ld, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * nrec) return;
    ops::adj_inject_one(g, A, M, B, taps, sadj, ld, n, t);
}

// Transformed formulation: buoyancy term of step n0 (first step of a
// segment), acc5..7 += (v^{n0+1/2} / G - v^{n0-1/2}) alpha.
__global__ void k_rho_term(DevGrid g, AdjFields A, DevBoundary B, const float* __restrict__ vn,
                           const float* __restrict__ vp, long long fstride) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    ops::rho_term_cell(A, B, vn, vp, fstride, cidx(g, i, j, k), i, j, k);
}

// Transformed formulation: pointwise inverses and the chain rule of the
// staggered means; output dense [nz][ny][nx].
__global__ void k_grad_finalize_t(DevGrid g, AdjFields A, DevMedium M, float* __restrict__ glam,
                                  float* __restrict__ gmu, float* __restrict__ grho) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    ops::finalize_t_cell(g, A, M, glam, gmu, grho, i, j, k);
}

// L2 misfit: sadj = dt (s - d), misfit += dt / 2 (s - d)^2.
__global__ void k_residual(const float* __restrict__ s, const float* __restrict__ d,
                           float* __restrict__ sadj, long long n, float dt, double* misfit) {
    double acc = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const float r = s[t] - d[t];
        sadj[t] = dt * r;
        acc += 0.5 * (double)dt * (double)r * (double)r;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(misfit, acc);
}

dim3 plane_grid(const DevGrid& g) { return dim3((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz); }

}  // namespace

namespace {

// 16-bit checkpoints (storage BF16 / FP16): per field q the state is stored
// as s_q times its value, s_q = 2^(14 - e) with max |f_q| = m 2^e (m in
// [0.5, 1)), so the largest stored magnitude is below 2^14 (FP16 holds up
// to 65504); s_q = 1 for an all-zero field.  The maxima are gathered on the
// device (float bits of non-negative values order like unsigned ints).
__global__ void k_state_absmax(const float* __restrict__ f, long long fs, unsigned* amax) {
    const int q = blockIdx.y;
    float m = 0.0f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < fs;
         i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(f[q * fs + i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(amax + q, __float_as_uint(m));
}

__device__ __forceinline__ float ckpt_scale_of(unsigned amax_bits) {
    const float m = __uint_as_float(amax_bits);
    if (!(m > 0.0f) || !isfinite(m)) return 1.0f;
    int e;
    frexpf(m, &e);
    return ldexpf(1.0f, 14 - e);
}

template <typename H>
__global__ void k_ckpt_store(const float* __restrict__ f, long long fs, const unsigned* amax,
                             float* scales, H* dst) {
    const int q = blockIdx.y;
    const float s = ckpt_scale_of(amax[q]);
    if (blockIdx.x == 0 && threadIdx.x == 0) scales[q] = s;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < fs;
         i += (long long)gridDim.x * blockDim.x)
        dst[q * fs + i] = ops::Io<H>::put(f[q * fs + i] * s);
}

template <typename H>
__global__ void k_ckpt_load(const H* __restrict__ src, long long fs, const float* scales, float* f) {
    const int q = blockIdx.y;
    const float inv = 1.0f / scales[q];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < fs;
         i += (long long)gridDim.x * blockDim.x)
        f[q * fs + i] = ops::Io<H>::get(src + q * fs + i) * inv;
}

}  // namespace

cudaError_t launch_ckpt_store(const float* fields, long long fs, int storage, unsigned* amax,
                              float* scales, void* dst, cudaStream_t st) {
    const dim3 grid(1024, NFIELD);
    cudaError_t e = cudaMemsetAsync(amax, 0, NFIELD * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    k_state_absmax<<<grid, 256, 0, st>>>(fields, fs, amax);
    if (storage == EWS_STORAGE_BF16)
        k_ckpt_store<__nv_bfloat16><<<grid, 256, 0, st>>>(fields, fs, amax, scales,
                                                          static_cast<__nv_bfloat16*>(dst));
    else
        k_ckpt_store<__half><<<grid, 256, 0, st>>>(fields, fs, amax, scales, static_cast<__half*>(dst));
    return cudaGetLastError();
}

cudaError_t launch_ckpt_load(const void* src, long long fs, int storage, const float* scales,
                             float* fields, cudaStream_t st) {
    const dim3 grid(1024, NFIELD);
    if (storage == EWS_STORAGE_BF16)
        k_ckpt_load<__nv_bfloat16><<<grid, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(src), fs,
                                                         scales, fields);
    else
        k_ckpt_load<__half><<<grid, 256, 0, st>>>(static_cast<const __half*>(src), fs, scales, fields);
    return cudaGetLastError();
}

cudaError_t launch_residual(const float* seis, const float* obs, float* sadj, long long n,
                            float dt, double* misfit, cudaStream_t st) {
    const int blocks = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    k_residual<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(seis, obs, sadj, n, dt, misfit);
    return cudaGetLastError();
}

cudaError_t launch_adj_stress(const DevGrid& g, const AdjFields& A, const DevMedium& M,
                              const DevBoundary& B, const float* vh, size_t fstride, float dt,
                              cudaStream_t st) {
    const float *v0 = vh, *v1 = vh + fstride, *v2 = vh + 2 * fstride;
    if (B.kind == BND_SPONGE)
        k_adj_stress<BND_SPONGE><<<plane_grid(g), dim3(32, 8), 0, st>>>(g, A, M, B, v0, v1, v2, dt);
    else
        k_adj_stress<BND_NONE><<<plane_grid(g), dim3(32, 8), 0, st>>>(g, A, M, B, v0, v1, v2, dt);
    return cudaGetLastError();
}

cudaError_t launch_adj_velocity(const DevGrid& g, const AdjFields& A, const DevMedium& M,
                                const DevBoundary& B, const float* vn, const float* vp,
                                size_t fstride, float dt, cudaStream_t st) {
    if (B.kind == BND_SPONGE)
        k_adj_velocity<BND_SPONGE><<<plane_grid(g), dim3(32, 8), 0, st>>>(g, A, M, B, vn, vp, fstride, dt);
    else
        k_adj_velocity<BND_NONE><<<plane_grid(g), dim3(32, 8), 0, st>>>(g, A, M, B, vn, vp, fstride, dt);
    return cudaGetLastError();
}

cudaError_t launch_adj_record(const DevGrid& g, const AdjFields& A, const Tap* taps, int nrec,
                              const float* sadj, int ld, int n, cudaStream_t st) {
    if (nrec <= 0) return cudaSuccess;
    k_adj_record<<<(3 * nrec + 127) / 128, 128, 0, st>>>(g, A, taps, nrec, sadj, ld, n);
    return cudaGetLastError();
}

cudaError_t launch_acc_flush(const DevGrid& g, const AdjFields& A, cudaStream_t st) {
    k_acc_flush<<<plane_grid(g), dim3(32, 8), 0, st>>>(g, A);
    return cudaGetLastError();
}

cudaError_t launch_grad_finalize(const DevGrid& g, const AdjFields& A, const DevMedium& M,
                                 float* glam, float* gmu, float* grho, cudaStream_t st) {
    k_grad_finalize<<<plane_grid(g), dim3(32, 8), 0, st>>>(g, A, M, glam, gmu, grho);
    return cudaGetLastError();
}

cudaError_t launch_adj_inject(const DevGrid& g, const AdjFields& A, const DevMedium& M,
                              const DevBoundary& B, const Tap* taps, int nrec, const float* sadj,
                              int ld, int n, cudaStream_t st) {
    if (nrec <= 0) return cudaSuccess;
    const dim3 grid((3 * nrec + 127) / 128);
    k_adj_inject<<<grid, 128, 0, st>>>(g, A, M, B, taps, nrec, sadj, ld, n);
    return cudaGetLastError();
}

cudaError_t launch_rho_term(const DevGrid& g, const AdjFields& A, const DevBoundary& B,
                            const float* vn, const float* vp, long long fstride, cudaStream_t st) {
    k_rho_term<<<plane_grid(g), dim3(32, 8), 0, st>>>(g, A, B, vn, vp, fstride);
    return cudaGetLastError();
}

cudaError_t launch_grad_finalize_t(const DevGrid& g, const AdjFields& A, const DevMedium& M,
                                   float* glam, float* gmu, float* grho, cudaStream_t st) {
    k_grad_finalize_t<<<plane_grid(g), dim3(32, 8), 0, st>>>(g, A, M, glam, gmu, grho);
    return cudaGetLastError();
}

}  // namespace ews
