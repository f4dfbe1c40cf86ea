// ews_ops.cuh -- per-element device operations shared by the stand-alone
// kernels (ews_forward.cu, ews_adjoint.cu) and the batched executor
// (ews_stencil.cu): source taps, receiver samples, residual injection and
// the gradient accumulator steps.  Each function does the work of one
// thread; the callers own the launch shape.
//
// Loads of data that the batched executor rewrites within one launch
// (wavefields, history, accumulators) are plain loads, never the
// non-coherent read-only path; the medium and the boundary profiles are
// read-only for a whole launch and use __ldg.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "ews_internal.cuh"

namespace ews {
namespace ops {

__device__ __forceinline__ long long cidx(const DevGrid& g, int i, int j, int k) {
    return (long long)k * g.plane + (long long)j * g.pitch + i;
}

// Medium value with indices past the top edge clamped (Sec. 2.2.1 reading).
__device__ __forceinline__ float med(const float* __restrict__ m, const DevGrid& g, int i, int j,
                                     int k) {
    return __ldg(m + cidx(g, min(i, g.nx - 1), min(j, g.ny - 1), min(k, g.nz - 1)));
}

// Sponge gain of cell (i, j, k) (1 without a sponge).
__device__ __forceinline__ float gain(const DevBoundary& B, int i, int j, int k) {
    if (B.kind != BND_SPONGE) return 1.0f;
    return __ldg(B.g[0] + i) * __ldg(B.g[1] + j) * __ldg(B.g[2] + k);
}

// Buoyancy at the v point of component c of cell (i, j, k): 2 / (rho + rho').
__device__ __forceinline__ float buoy(const DevMedium& M, const DevGrid& g, int c, int i, int j,
                                      int k) {
    return 2.0f / (med(M.rho, g, i, j, k) + med(M.rho, g, i + (c == 0), j + (c == 1), k + (c == 2)));
}

template <typename T> struct Io;
template <> struct Io<float> {
    __device__ static float get(const float* p) { return *p; }
    __device__ static float put(float x) { return x; }
};
template <> struct Io<__nv_bfloat16> {
    __device__ static float get(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    __device__ static __nv_bfloat16 put(float x) { return __float2bfloat16_rn(x); }
};
template <> struct Io<__half> {
    __device__ static float get(const __half* p) { return __half2float(*p); }
    __device__ static __half put(float x) { return __float2half_rn(x); }
};

// Source tap t at step n (Sec. 2.4 reading): the tap weight holds -dt M / V
// (moment) or dt F / V (force, times the buoyancy here); the sponge gain is
// applied to the injected amount.  Several taps may hit one element.
template <typename T>
__device__ __forceinline__ void inject_tap(const DevGrid& g, const DevFields& F, const DevMedium& M,
                                           const DevBoundary& B, const DevSource& S,
                                           const float* __restrict__ wavelet, int n, int t,
                                           int* err) {
    const Tap tp = S.tap[t];
    float amp = tp.w * __ldg(wavelet + n);
    if (S.kind == 1) {
        if (g.cm[2]) {           // coarse medium: 1 / rho sampled at the v point
            const int c = tp.q - VX;
            amp *= 1.0f / coarse_at(g, 2, tp.i + (c == 0 ? 0.5f : 0.0f), tp.j + (c == 1 ? 0.5f : 0.0f),
                                    tp.k + (c == 2 ? 0.5f : 0.0f));
        } else {
            amp *= buoy(M, g, tp.q - VX, tp.i, tp.j, tp.k);
        }
    }
    amp *= gain(B, tp.i, tp.j, tp.k);
    T* f = reinterpret_cast<T*>(F.f[tp.q]) + cidx(g, tp.i, tp.j, tp.k);
    if constexpr (sizeof(T) == 4) {
        atomicAdd(f, amp);
    } else {
        const float now = Io<T>::get(f) + amp;    // estimate for the range check
        atomicAdd(f, Io<T>::put(amp));
        if (std::is_same<T, __half>::value && fabsf(now) > 65504.0f) atomicOr(err, 4);
    }
}

// Receiver sample t (component t / nrec): 8 trilinear taps (Sec. 2.4).
template <typename T>
__device__ __forceinline__ float record_one(const DevGrid& g, const DevFields& F,
                                            const Tap* __restrict__ taps, int t) {
    const Tap* tp = taps + 8 * t;
    float acc = 0.0f;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const Tap q = tp[m];
        acc += q.w * Io<T>::get(reinterpret_cast<const T*>(F.f[q.q]) + cidx(g, q.i, q.j, q.k));
    }
    return acc;
}

// Reverse sweep in transformed variables: one tap of a residual sample a
// injected into alpha (alpha += G B S^T sadj_n).
__device__ __forceinline__ void adj_inject_tap(const DevGrid& g, const AdjFields& A,
                                               const DevMedium& M, const DevBoundary& B,
                                               const Tap& q, float a) {
    atomicAdd(A.p[q.q] + cidx(g, q.i, q.j, q.k),
              gain(B, q.i, q.j, q.k) * buoy(M, g, q.q - VX, q.i, q.j, q.k) * q.w * a);
}

// All 8 taps of residual sample t.
__device__ __forceinline__ void adj_inject_one(const DevGrid& g, const AdjFields& A,
                                               const DevMedium& M, const DevBoundary& B,
                                               const Tap* __restrict__ taps,
                                               const float* sadj, int ld, int n, int t) {
    const float a = sadj[(long long)t * ld + n];
    const Tap* tp = taps + 8 * t;
#pragma unroll
    for (int m = 0; m < 8; ++m) adj_inject_tap(g, A, M, B, tp[m], a);
}

// Buoyancy term of a segment's first reverse step at element o of cell
// (i, j, k): acc5..7 += (v^{n+1/2} / G - v^{n-1/2}) alpha.
__device__ __forceinline__ void rho_term_cell(const AdjFields& A, const DevBoundary& B,
                                              const float* vn, const float* vp, long long fs,
                                              long long o, int i, int j, int k) {
    const float iG = 1.0f / gain(B, i, j, k);
#pragma unroll
    for (int c = 0; c < 3; ++c)
        A.acc[5 + c][o] += (vn[c * fs + o] * iG - vp[c * fs + o]) * A.p[c][o];
}

// acc64 += acc32; acc32 = 0 at element o.
__device__ __forceinline__ void flush_cell(const AdjFields& A, long long o) {
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        A.acc64[a][o] += (double)A.acc[a][o];
        A.acc[a][o] = 0.0f;
    }
}

// Derivative of a 4-cell shear mean with respect to one of its cells, which
// occurs mult times among the 4 (top edge clamped): mult / 4 for the
// arithmetic mean; mult mean^2 / (4 mu_cell^2) for the harmonic mean of the
// xz / yz points on a free-surface plane (reading of Sec. 2.5).
__device__ __forceinline__ float shear_d(float mean, float mu_cell, int mult, bool harmonic) {
    if (!harmonic) return 0.25f * mult;
    const float r = mean / mu_cell;
    return 0.25f * mult * r * r;
}

// 4-cell shear mean of mu, harmonic on a free-surface plane.
__device__ __forceinline__ float shear_mean(float a, float b, float c, float d, bool harmonic) {
    return harmonic ? 4.0f / (1.0f / a + 1.0f / b + 1.0f / c + 1.0f / d) : 0.25f * (a + b + c + d);
}

struct Grad3 {
    double lam, mu, rho;
};

// Gradients with respect to the medium of cell (i, j, k) as the passes use
// it, from the transformed-variable accumulators:
// dJ/dlambda = acc0 / (3 lambda + 2 mu);
// dJ/dmu = (acc1 - lambda acc0 / (3 lambda + 2 mu)) / mu + the shear sums
//          over the 4-cell means (each point / its mean times the mean's
//          derivative, top edge clamped);
// dJ/drho = -1/2 sum over the 2-cell v points of the cell of acc5..7.
// The time sums arrive in FP64; the difference acc1 - lambda acc0 / kappa
// (which can cancel) and the sums over points stay in FP64, while the
// medium factors (reciprocals, means) are FP32: each carries a relative
// error of ~1e-7, far below the gradient's FP32 accumulation error, and
// FP64 division is a long instruction sequence at GB300's low FP64 rate.
__device__ __forceinline__ Grad3 grad_t_cell(const DevGrid& g, const AdjFields& A,
                                             const DevMedium& M, int i, int j, int k) {
    const long long o = cidx(g, i, j, k);
    const float lamf = __ldg(M.lam + o), mu0f = __ldg(M.mu + o);
    const double rkap = (double)(1.0f / (3.0f * lamf + 2.0f * mu0f));
    const double a0 = A.acc64[0][o];
    double mu = (A.acc64[1][o] - (double)lamf * a0 * rkap) * (double)(1.0f / mu0f);
    double rho = 0.0;
    for (int da = -1; da <= 0; ++da)
        for (int db = -1; db <= 0; ++db) {
            int a = i + da, b = j + db;
            if (a >= 0 && b >= 0) {           // xy point (a, b, k)
                const int ap = min(a + 1, g.nx - 1), bp = min(b + 1, g.ny - 1);
                const int mult = (a == i && b == j) + (ap == i && b == j) + (a == i && bp == j) + (ap == i && bp == j);
                if (mult) {
                    const float mb = 0.25f * (med(M.mu, g, a, b, k) + med(M.mu, g, ap, b, k) +
                                              med(M.mu, g, a, bp, k) + med(M.mu, g, ap, bp, k));
                    mu += A.acc64[2][cidx(g, a, b, k)] * (double)(0.25f * mult / mb);
                }
            }
            a = i + da; b = k + db;
            if (a >= 0 && b >= 0) {           // xz point (a, j, b)
                const int ap = min(a + 1, g.nx - 1), bp = min(b + 1, g.nz - 1);
                const int mult = (a == i && b == k) + (ap == i && b == k) + (a == i && bp == k) + (ap == i && bp == k);
                if (mult) {
                    const bool h = b == g.fs - 1;
                    const float mb = shear_mean(med(M.mu, g, a, j, b), med(M.mu, g, ap, j, b),
                                                med(M.mu, g, a, j, bp), med(M.mu, g, ap, j, bp), h);
                    mu += A.acc64[3][cidx(g, a, j, b)] * (double)(shear_d(mb, mu0f, mult, h) / mb);
                }
            }
            a = j + da; b = k + db;
            if (a >= 0 && b >= 0) {           // yz point (i, a, b)
                const int ap = min(a + 1, g.ny - 1), bp = min(b + 1, g.nz - 1);
                const int mult = (a == j && b == k) + (ap == j && b == k) + (a == j && bp == k) + (ap == j && bp == k);
                if (mult) {
                    const bool h = b == g.fs - 1;
                    const float mb = shear_mean(med(M.mu, g, i, a, b), med(M.mu, g, i, ap, b),
                                                med(M.mu, g, i, a, bp), med(M.mu, g, i, ap, bp), h);
                    mu += A.acc64[4][cidx(g, i, a, b)] * (double)(shear_d(mb, mu0f, mult, h) / mb);
                }
            }
        }
    for (int c = 0; c < 3; ++c)
        for (int d = -1; d <= 0; ++d) {
            const int ii = i + (c == 0 ? d : 0), jj = j + (c == 1 ? d : 0), kk = k + (c == 2 ? d : 0);
            if (ii < 0 || jj < 0 || kk < 0) continue;
            const int a = c == 0 ? ii : (c == 1 ? jj : kk);
            const int n = c == 0 ? g.nx : (c == 1 ? g.ny : g.nz);
            const int self = c == 0 ? i : (c == 1 ? j : k);
            const int mult = (a == self) + (min(a + 1, n - 1) == self);
            if (mult) rho += (-0.5 * mult) * A.acc64[5 + c][cidx(g, ii, jj, kk)];
        }
    return Grad3{a0 * rkap, mu, rho};
}

// Gradients of the input model at cell (i, j, k), dense [nz][ny][nx]
// output.  With a free surface the cells above it hold eps times the
// surface cell of their column (reading of Sec. 2.5): their own input
// values are unused (gradient 0) and the surface cell collects eps times
// their gradients.
__device__ __forceinline__ void finalize_t_cell(const DevGrid& g, const AdjFields& A,
                                                const DevMedium& M, float* glam, float* gmu,
                                                float* grho, int i, int j, int k) {
    const long long od = ((long long)k * g.ny + j) * g.nx + i;
    Grad3 r{0.0, 0.0, 0.0};
    if (k >= g.fs) {
        r = grad_t_cell(g, A, M, i, j, k);
        if (k == g.fs)
            for (int kk = 0; kk < k; ++kk) {
                const Grad3 v = grad_t_cell(g, A, M, i, j, kk);
                r.lam += g.fs_eps * v.lam;
                r.mu += g.fs_eps * v.mu;
                r.rho += g.fs_eps * v.rho;
            }
    }
    glam[od] = (float)r.lam;
    gmu[od] = (float)r.mu;
    grho[od] = (float)r.rho;
}

}  // namespace ops
}  // namespace ews
