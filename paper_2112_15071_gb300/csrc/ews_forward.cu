// ews_forward.cu -- small kernels around the stencil passes (sm_103a):
// point-source injection, receiver sampling (Sec. 2.4) and the medium
// set-up (vp/vs -> Lame, validity flags, vp_max).  The velocity and stress
// passes themselves are in ews_stencil.cu.
#include "ews_internal.cuh"

namespace ews {

namespace {

__device__ __forceinline__ float med(const float* __restrict__ m, const DevGrid& g,
                                     int i, int j, int k) {
    i = min(i, g.nx - 1);
    j = min(j, g.ny - 1);
    k = min(k, g.nz - 1);
    return __ldg(m + (long long)k * g.plane + (long long)j * g.pitch + i);
}

// Point-source injection (one thread per tap).  Runs after the pass it
// belongs to; the sponge gain is applied to the injected amount, which
// equals injecting before the gain.
__global__ void k_inject(DevGrid g, DevFields F, DevMedium M, DevBoundary B, DevSource S,
                         const float* __restrict__ wavelet, int n) {
    const int t = threadIdx.x;
    if (t >= S.ntap) return;
    const Tap tp = S.tap[t];
    const long long c = (long long)tp.k * g.plane + (long long)tp.j * g.pitch + tp.i;
    float amp = tp.w * __ldg(wavelet + n);
    if (S.kind == 1) {
        const float r0 = med(M.rho, g, tp.i, tp.j, tp.k);
        const float r1 = med(M.rho, g, tp.i + (tp.q == VX), tp.j + (tp.q == VY),
                             tp.k + (tp.q == VZ));
        amp *= 2.0f / (r0 + r1);
    }
    if (B.kind == BND_SPONGE)
        amp *= __ldg(B.g[0] + tp.i) * __ldg(B.g[1] + tp.j) * __ldg(B.g[2] + tp.k);
    // several taps may hit the same element (e.g. a source on a grid point)
    atomicAdd(F.f[tp.q] + c, amp);
}

// Receiver sampling: one thread per (component, receiver), 8 taps each.
__global__ void k_record(DevGrid g, DevFields F, const Tap* __restrict__ taps, int nrec,
                         float* __restrict__ seis, int ld, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * nrec) return;
    const Tap* tp = taps + 8 * t;
    float acc = 0.0f;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const Tap q = tp[m];
        acc += q.w * F.f[q.q][(long long)q.k * g.plane + (long long)q.j * g.pitch + q.i];
    }
    seis[(long long)t * ld + n] = acc;
}

// In-place medium set-up on pitched arrays: optional (vp, vs) -> (lambda,
// mu), validity flags and vp_max (as float bits; all values are >= 0).
// flags_vpmax[0]: bit0 non-finite, bit1 rho <= 0, bit2 mu < 0, bit3
// lambda + 2 mu <= 0;  flags_vpmax[1]: vp_max bits.
__global__ void k_medium_setup(DevGrid g, float* a, float* b, float* rho, int from_vel,
                               unsigned* flags_vpmax) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    unsigned flag = 0;
    float vp = 0.0f;
    if (i < g.nx && j < g.ny) {
        const long long c = (long long)k * g.plane + (long long)j * g.pitch + i;
        const float r = rho[c];
        float lam = a[c], mu = b[c];
        if (from_vel) {
            const float p = a[c], s = b[c];
            mu = r * s * s;
            lam = r * p * p - 2.0f * mu;
            a[c] = lam;
            b[c] = mu;
        }
        if (!isfinite(r) || !isfinite(lam) || !isfinite(mu)) flag |= 1u;
        if (!(r > 0.0f)) flag |= 2u;
        if (mu < 0.0f) flag |= 4u;
        if (!(lam + 2.0f * mu > 0.0f)) flag |= 8u;
        if (flag == 0) vp = sqrtf((lam + 2.0f * mu) / r);
    }
    // warp-level reduce, then one atomic per warp
    for (int o = 16; o > 0; o >>= 1) {
        flag |= __shfl_xor_sync(0xffffffffu, flag, o);
        vp = fmaxf(vp, __shfl_xor_sync(0xffffffffu, vp, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (flag) atomicOr(flags_vpmax, flag);
        atomicMax(flags_vpmax + 1, __float_as_uint(vp));
    }
}

}  // namespace

static dim3 plane_grid(const DevGrid& g) {
    return dim3((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
}

cudaError_t launch_inject(const DevGrid& g, const DevFields& F, const DevMedium& M,
                          const DevBoundary& B, const DevSource& S, const float* wavelet,
                          int n, cudaStream_t st) {
    if (S.kind < 0 || S.ntap == 0) return cudaSuccess;
    k_inject<<<1, kMaxSrcTaps, 0, st>>>(g, F, M, B, S, wavelet, n);
    return cudaGetLastError();
}

cudaError_t launch_record(const DevGrid& g, const DevFields& F, const Tap* taps, int nrec,
                          float* seis, int ld, int n, cudaStream_t st) {
    if (nrec <= 0) return cudaSuccess;
    const int nt = 3 * nrec;
    k_record<<<(nt + 127) / 128, 128, 0, st>>>(g, F, taps, nrec, seis, ld, n);
    return cudaGetLastError();
}

cudaError_t launch_medium_setup(const DevGrid& g, float* a, float* b, float* rho,
                                int from_velocities, unsigned* flags_vpmax, cudaStream_t st) {
    k_medium_setup<<<plane_grid(g), dim3(32, 8), 0, st>>>(g, a, b, rho, from_velocities,
                                                          flags_vpmax);
    return cudaGetLastError();
}

}  // namespace ews
