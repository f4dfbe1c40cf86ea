// ews_forward.cu -- small kernels around the stencil passes (sm_103a):
// point-source injection, receiver sampling (Sec. 2.4), the medium set-up
// (vp/vs -> Lame, validity flags, bounds) and the conversion of 16-bit
// stored fields to and from float32.  The velocity and stress passes
// themselves are in ews_stencil.cu.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "ews_internal.cuh"
#include "ews_ops.cuh"

namespace ews {

namespace {

using ops::Io;
using ops::med;

// Point-source injection (one thread per tap).  Runs after the pass it
// belongs to.
template <typename T>
__global__ void k_inject(DevGrid g, DevFields F, DevMedium M, DevBoundary B, DevSource S,
                         const float* __restrict__ wavelet, int n, int* err) {
    const int t = threadIdx.x;
    if (t >= S.ntap) return;
    ops::inject_tap<T>(g, F, M, B, S, wavelet, n, t, err);
}

// Receiver sampling: one thread per (component, receiver), 8 taps each.
// A non-finite sample means the wavefield has blown up or was given a
// NaN / Inf: flag bit 16 of *err (a watchdog that costs no extra traffic).
template <typename T>
__global__ void k_record(DevGrid g, DevFields F, const Tap* __restrict__ taps, int nrec,
                         float* __restrict__ seis, int ld, int n, float i0, float i1, float i2,
                         int* err) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * nrec) return;
    float acc = ops::record_one<T>(g, F, taps, t);
    if constexpr (sizeof(T) == 2) acc *= (t < nrec ? i0 : t < 2 * nrec ? i1 : i2);
    if (!isfinite(acc)) atomicOr(err, 16);
    seis[(long long)t * ld + n] = acc;
}

// The point terms that follow the stress pass, in one launch: block 0
// injects the moment-rate source (one thread per tap; S.kind < 0: none),
// blocks 1.. sample the receivers from v^{n+1/2}, which the stress pass
// leaves unchanged (as k_record).
template <typename T>
__global__ void k_post_stress(DevGrid g, DevFields F, DevMedium M, DevBoundary B, DevSource S,
                              const float* __restrict__ wavelet, const Tap* __restrict__ taps,
                              int nrec, float* __restrict__ seis, int ld, int n, float i0, float i1,
                              float i2, int* err) {
    if (blockIdx.x == 0) {
        if (S.kind >= 0 && (int)threadIdx.x < S.ntap)
            ops::inject_tap<T>(g, F, M, B, S, wavelet, n, threadIdx.x, err);
        return;
    }
    const int t = (blockIdx.x - 1) * blockDim.x + threadIdx.x;
    if (t >= 3 * nrec) return;
    float acc = ops::record_one<T>(g, F, taps, t);
    if constexpr (sizeof(T) == 2) acc *= (t < nrec ? i0 : t < 2 * nrec ? i1 : i2);
    if (!isfinite(acc)) atomicOr(err, 16);
    seis[(long long)t * ld + n] = acc;
}

// Stored field -> dense float32 (out = stored * inv_s) and back.
template <typename T>
__global__ void k_field_out(DevGrid g, const T* __restrict__ f, float inv_s, float* __restrict__ d) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    d[((long long)k * g.ny + j) * g.nx + i] =
        Io<T>::get(f + (long long)k * g.plane + (long long)j * g.pitch + i) * inv_s;
}
template <typename T>
__global__ void k_field_in(DevGrid g, const float* __restrict__ d, float s, T* __restrict__ f,
                           int* err) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const float x = d[((long long)k * g.ny + j) * g.nx + i] * s;
    if (std::is_same<T, __half>::value && fabsf(x) > 65504.0f) atomicOr(err, 4);
    f[(long long)k * g.plane + (long long)j * g.pitch + i] = Io<T>::put(x);
}

// In-place medium set-up on pitched arrays: optional (vp, vs) -> (lambda,
// mu), validity flags and bounds (as float bits of non-negative values, so
// unsigned atomics order them).  flags[0]: bit0 non-finite, bit1 rho <= 0,
// bit2 mu < 0, bit3 lambda + 2 mu <= 0;  flags[1]: max vp; flags[2]: min
// rho; flags[3]: min sqrt(rho mu) over mu > 0; flags[4]: max sqrt(rho (lambda + 2 mu)).
// flags[0] bit4 (16) marks a cell with mu == 0, which is valid.
__global__ void k_medium_setup(DevGrid g, float* a, float* b, float* rho, int from_vel,
                               unsigned* flags) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    unsigned flag = 0;
    float vp = 0.0f, zp = 0.0f;
    float rmin = 3.0e38f, zsmin = 3.0e38f;
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
        if (flag == 0) {
            vp = sqrtf((lam + 2.0f * mu) / r);
            zp = sqrtf(r * (lam + 2.0f * mu));
            if (k >= g.fs) {                   // the medium below a free surface
                rmin = r;
                if (mu > 0.0f) zsmin = sqrtf(r * mu);
            }
            if (mu == 0.0f) flag |= 16u;       // a fluid cell (not an error)
        }
    }
    // warp-level reduce, then across the 8 warps of the block, then one
    // atomic per block and quantity
    for (int o = 16; o > 0; o >>= 1) {
        flag |= __shfl_xor_sync(0xffffffffu, flag, o);
        vp = fmaxf(vp, __shfl_xor_sync(0xffffffffu, vp, o));
        zp = fmaxf(zp, __shfl_xor_sync(0xffffffffu, zp, o));
        rmin = fminf(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
        zsmin = fminf(zsmin, __shfl_xor_sync(0xffffffffu, zsmin, o));
    }
    __shared__ float red[8][5];
    const int w = threadIdx.y;                 // blockDim = (32, 8): one warp per row
    if (threadIdx.x == 0) {
        red[w][0] = __uint_as_float(flag);
        red[w][1] = vp;
        red[w][2] = rmin;
        red[w][3] = zsmin;
        red[w][4] = zp;
    }
    __syncthreads();
    if (w == 0 && threadIdx.x == 0) {
        for (int q = 1; q < 8; ++q) {
            flag |= __float_as_uint(red[q][0]);
            vp = fmaxf(vp, red[q][1]);
            rmin = fminf(rmin, red[q][2]);
            zsmin = fminf(zsmin, red[q][3]);
            zp = fmaxf(zp, red[q][4]);
        }
        if (flag) atomicOr(flags, flag);
        atomicMax(flags + 1, __float_as_uint(vp));
        atomicMin(flags + 2, __float_as_uint(rmin));
        atomicMin(flags + 3, __float_as_uint(zsmin));
        atomicMax(flags + 4, __float_as_uint(zp));
    }
}

// Vacuum formulation of the free surface (Sec. 2.5 reading): every cell
// above plane ks takes eps times the Lame parameters and density of the
// first cell below the surface in its column.  Velocity input (vp, vs, rho):
// the speeds are kept and rho is scaled, which gives the same Lame values.
__global__ void k_vacuum(DevGrid g, float* a, float* b, float* rho, int from_vel, float eps) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny || k >= g.fs) return;
    const long long c = (long long)k * g.plane + (long long)j * g.pitch + i;
    const long long src = (long long)g.fs * g.plane + (long long)j * g.pitch + i;
    rho[c] = eps * rho[src];
    a[c] = from_vel ? a[src] : eps * a[src];
    b[c] = from_vel ? b[src] : eps * b[src];
}

}  // namespace

static dim3 plane_grid(const DevGrid& g) {
    return dim3((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
}

cudaError_t launch_inject(const DevGrid& g, const DevFields& F, const DevMedium& M,
                          const DevBoundary& B, const DevSource& S, const float* wavelet,
                          int n, int storage, int* err, cudaStream_t st) {
    if (S.kind < 0 || S.ntap == 0) return cudaSuccess;
    switch (storage) {
        case EWS_STORAGE_BF16:
            k_inject<__nv_bfloat16><<<1, kMaxSrcTaps, 0, st>>>(g, F, M, B, S, wavelet, n, err);
            break;
        case EWS_STORAGE_F16:
            k_inject<__half><<<1, kMaxSrcTaps, 0, st>>>(g, F, M, B, S, wavelet, n, err);
            break;
        default:
            k_inject<float><<<1, kMaxSrcTaps, 0, st>>>(g, F, M, B, S, wavelet, n, err);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_record(const DevGrid& g, const DevFields& F, const Tap* taps, int nrec,
                          float* seis, int ld, int n, int storage, const float inv[3], int* err,
                          cudaStream_t st) {
    if (nrec <= 0) return cudaSuccess;
    const int nt = 3 * nrec;
    const dim3 grid((nt + 127) / 128);
    switch (storage) {
        case EWS_STORAGE_BF16:
            k_record<__nv_bfloat16><<<grid, 128, 0, st>>>(g, F, taps, nrec, seis, ld, n, inv[0], inv[1], inv[2], err);
            break;
        case EWS_STORAGE_F16:
            k_record<__half><<<grid, 128, 0, st>>>(g, F, taps, nrec, seis, ld, n, inv[0], inv[1], inv[2], err);
            break;
        default:
            k_record<float><<<grid, 128, 0, st>>>(g, F, taps, nrec, seis, ld, n, 1.f, 1.f, 1.f, err);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_post_stress(const DevGrid& g, const DevFields& F, const DevMedium& M,
                               const DevBoundary& B, const DevSource& S, const float* wavelet,
                               const Tap* taps, int nrec, float* seis, int ld, int n, int storage,
                               const float inv[3], int* err, cudaStream_t st) {
    static_assert(kMaxSrcTaps <= 128, "source taps of one block");
    const dim3 grid(1 + (3 * nrec + 127) / 128);
    switch (storage) {
        case EWS_STORAGE_BF16:
            k_post_stress<__nv_bfloat16><<<grid, 128, 0, st>>>(g, F, M, B, S, wavelet, taps, nrec, seis, ld, n, inv[0], inv[1], inv[2], err);
            break;
        case EWS_STORAGE_F16:
            k_post_stress<__half><<<grid, 128, 0, st>>>(g, F, M, B, S, wavelet, taps, nrec, seis, ld, n, inv[0], inv[1], inv[2], err);
            break;
        default:
            k_post_stress<float><<<grid, 128, 0, st>>>(g, F, M, B, S, wavelet, taps, nrec, seis, ld, n, 1.f, 1.f, 1.f, err);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_vacuum(const DevGrid& g, float* a, float* b, float* rho, int from_velocities,
                          float eps, cudaStream_t st) {
    if (g.fs <= 0 || g.fs >= g.nz) return cudaSuccess;
    const dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.fs);
    k_vacuum<<<grid, dim3(32, 8), 0, st>>>(g, a, b, rho, from_velocities, eps);
    return cudaGetLastError();
}

cudaError_t launch_medium_setup(const DevGrid& g, float* a, float* b, float* rho,
                                int from_velocities, unsigned* flags, cudaStream_t st) {
    k_medium_setup<<<plane_grid(g), dim3(32, 8), 0, st>>>(g, a, b, rho, from_velocities, flags);
    return cudaGetLastError();
}

cudaError_t launch_field_out(const DevGrid& g, const void* field, int storage, float inv_s,
                             float* dense, cudaStream_t st) {
    switch (storage) {
        case EWS_STORAGE_BF16:
            k_field_out<<<plane_grid(g), dim3(32, 8), 0, st>>>(
                g, static_cast<const __nv_bfloat16*>(field), inv_s, dense);
            break;
        case EWS_STORAGE_F16:
            k_field_out<<<plane_grid(g), dim3(32, 8), 0, st>>>(
                g, static_cast<const __half*>(field), inv_s, dense);
            break;
        default:
            k_field_out<<<plane_grid(g), dim3(32, 8), 0, st>>>(
                g, static_cast<const float*>(field), inv_s, dense);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_field_in(const DevGrid& g, const float* dense, int storage, float s,
                            void* field, int* err, cudaStream_t st) {
    switch (storage) {
        case EWS_STORAGE_BF16:
            k_field_in<<<plane_grid(g), dim3(32, 8), 0, st>>>(
                g, dense, s, static_cast<__nv_bfloat16*>(field), err);
            break;
        case EWS_STORAGE_F16:
            k_field_in<<<plane_grid(g), dim3(32, 8), 0, st>>>(
                g, dense, s, static_cast<__half*>(field), err);
            break;
        default:
            k_field_in<<<plane_grid(g), dim3(32, 8), 0, st>>>(
                g, dense, s, static_cast<float*>(field), err);
            break;
    }
    return cudaGetLastError();
}

}  // namespace ews
