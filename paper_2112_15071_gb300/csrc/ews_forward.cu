// ews_forward.cu -- forward-pass kernels of libews (sm_103a).
//
// Velocity pass (Eq. 1) and stress pass (Eq. 2/3) of the staggered scheme,
// each with the 4th-order operator of Eq. 4, the medium means of
// Sec. 2.2.1 formed in registers, zero exterior (Sec. 2.2.2), and the
// absorbing edge (Sec. 2.5: sponge, or C-PML memory variables) fused in.
// Source injection and receiver sampling (Sec. 2.4) are tiny kernels that
// follow the pass they belong to.
#include "ews_internal.cuh"

namespace ews {

namespace {

__device__ __forceinline__ float fetch(const float* __restrict__ f, const DevGrid& g,
                                       int i, int j, int k) {
    bool in = (unsigned)i < (unsigned)g.nx && (unsigned)j < (unsigned)g.ny &&
              (unsigned)k < (unsigned)g.nz;
    return in ? __ldg(f + (long long)k * g.plane + (long long)j * g.pitch + i) : 0.0f;
}

__device__ __forceinline__ float med(const float* __restrict__ m, const DevGrid& g,
                                     int i, int j, int k) {
    i = min(i, g.nx - 1);
    j = min(j, g.ny - 1);
    k = min(k, g.nz - 1);
    return __ldg(m + (long long)k * g.plane + (long long)j * g.pitch + i);
}

// Eq. 4 with the samples at -3/2, -1/2, +1/2, +3/2 around the output point.
__device__ __forceinline__ float d4(float c1, float c2, float fm32, float fm12, float fp12,
                                    float fp32) {
    return c1 * (fp12 - fm12) + c2 * (fp32 - fm32);
}

// Slab helpers: index along the axis inside the 2W-wide slab storage.
__device__ __forceinline__ bool in_slab(int i, int n, int W) { return i < W || i >= n - W; }
__device__ __forceinline__ int slab_idx(int i, int n, int W) { return i < W ? i : i - (n - 2 * W); }

__device__ __forceinline__ float pml(float* __restrict__ psi, long long pc, float a, float b,
                                     float d) {
    float p = b * psi[pc] + a * d;
    psi[pc] = p;
    return d + p;
}

template <int BND>
__global__ void __launch_bounds__(256) k_velocity(DevGrid g, DevFields F, DevMedium M,
                                                  DevBoundary B, float dt) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const float* sxx = F.f[SXX];
    const float* syy = F.f[SYY];
    const float* szz = F.f[SZZ];
    const float* sxy = F.f[SXY];
    const float* sxz = F.f[SXZ];
    const float* syz = F.f[SYZ];
    // vx at (i+1/2, j, k)
    float dxx = d4(g.c1x, g.c2x, fetch(sxx, g, i - 1, j, k), fetch(sxx, g, i, j, k),
                   fetch(sxx, g, i + 1, j, k), fetch(sxx, g, i + 2, j, k));
    float dxy = d4(g.c1y, g.c2y, fetch(sxy, g, i, j - 2, k), fetch(sxy, g, i, j - 1, k),
                   fetch(sxy, g, i, j, k), fetch(sxy, g, i, j + 1, k));
    float dxz = d4(g.c1z, g.c2z, fetch(sxz, g, i, j, k - 2), fetch(sxz, g, i, j, k - 1),
                   fetch(sxz, g, i, j, k), fetch(sxz, g, i, j, k + 1));
    // vy at (i, j+1/2, k)
    float dyx = d4(g.c1x, g.c2x, fetch(sxy, g, i - 2, j, k), fetch(sxy, g, i - 1, j, k),
                   fetch(sxy, g, i, j, k), fetch(sxy, g, i + 1, j, k));
    float dyy = d4(g.c1y, g.c2y, fetch(syy, g, i, j - 1, k), fetch(syy, g, i, j, k),
                   fetch(syy, g, i, j + 1, k), fetch(syy, g, i, j + 2, k));
    float dyz = d4(g.c1z, g.c2z, fetch(syz, g, i, j, k - 2), fetch(syz, g, i, j, k - 1),
                   fetch(syz, g, i, j, k), fetch(syz, g, i, j, k + 1));
    // vz at (i, j, k+1/2)
    float dzx = d4(g.c1x, g.c2x, fetch(sxz, g, i - 2, j, k), fetch(sxz, g, i - 1, j, k),
                   fetch(sxz, g, i, j, k), fetch(sxz, g, i + 1, j, k));
    float dzy = d4(g.c1y, g.c2y, fetch(syz, g, i, j - 2, k), fetch(syz, g, i, j - 1, k),
                   fetch(syz, g, i, j, k), fetch(syz, g, i, j + 1, k));
    float dzz = d4(g.c1z, g.c2z, fetch(szz, g, i, j, k - 1), fetch(szz, g, i, j, k),
                   fetch(szz, g, i, j, k + 1), fetch(szz, g, i, j, k + 2));
    if (BND == BND_CPML) {
        const int W = B.W;
        if (in_slab(i, g.nx, W)) {
            long long pc = ((long long)k * g.ny + j) * (2 * W) + slab_idx(i, g.nx, W);
            float a = __ldg(B.pa[0] + i), b = __ldg(B.pb[0] + i);
            dxx = pml(B.psx[0], pc, a, b, dxx);
            dyx = pml(B.psx[1], pc, a, b, dyx);
            dzx = pml(B.psx[2], pc, a, b, dzx);
        }
        if (in_slab(j, g.ny, W)) {
            long long pc = ((long long)k * (2 * W) + slab_idx(j, g.ny, W)) * g.pitch + i;
            float a = __ldg(B.pa[1] + j), b = __ldg(B.pb[1] + j);
            dxy = pml(B.psy[0], pc, a, b, dxy);
            dyy = pml(B.psy[1], pc, a, b, dyy);
            dzy = pml(B.psy[2], pc, a, b, dzy);
        }
        if (in_slab(k, g.nz, W)) {
            long long pc = ((long long)slab_idx(k, g.nz, W) * g.ny + j) * g.pitch + i;
            float a = __ldg(B.pa[2] + k), b = __ldg(B.pb[2] + k);
            dxz = pml(B.psz[0], pc, a, b, dxz);
            dyz = pml(B.psz[1], pc, a, b, dyz);
            dzz = pml(B.psz[2], pc, a, b, dzz);
        }
    }
    // buoyancy at the v points: 1 / mean of the two adjacent densities
    const float r0 = med(M.rho, g, i, j, k);
    const float bx = 2.0f / (r0 + med(M.rho, g, i + 1, j, k));
    const float by = 2.0f / (r0 + med(M.rho, g, i, j + 1, k));
    const float bz = 2.0f / (r0 + med(M.rho, g, i, j, k + 1));
    const long long c = (long long)k * g.plane + (long long)j * g.pitch + i;
    float vx = F.f[VX][c] + dt * bx * (dxx + dxy + dxz);
    float vy = F.f[VY][c] + dt * by * (dyx + dyy + dyz);
    float vz = F.f[VZ][c] + dt * bz * (dzx + dzy + dzz);
    if (BND == BND_SPONGE) {
        const float G = __ldg(B.g[0] + i) * __ldg(B.g[1] + j) * __ldg(B.g[2] + k);
        vx *= G;
        vy *= G;
        vz *= G;
    }
    F.f[VX][c] = vx;
    F.f[VY][c] = vy;
    F.f[VZ][c] = vz;
}

template <int BND>
__global__ void __launch_bounds__(256) k_stress(DevGrid g, DevFields F, DevMedium M,
                                                DevBoundary B, float dt) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const float* vx = F.f[VX];
    const float* vy = F.f[VY];
    const float* vz = F.f[VZ];
    // normal strain rates at (i, j, k)
    float exx = d4(g.c1x, g.c2x, fetch(vx, g, i - 2, j, k), fetch(vx, g, i - 1, j, k),
                   fetch(vx, g, i, j, k), fetch(vx, g, i + 1, j, k));
    float eyy = d4(g.c1y, g.c2y, fetch(vy, g, i, j - 2, k), fetch(vy, g, i, j - 1, k),
                   fetch(vy, g, i, j, k), fetch(vy, g, i, j + 1, k));
    float ezz = d4(g.c1z, g.c2z, fetch(vz, g, i, j, k - 2), fetch(vz, g, i, j, k - 1),
                   fetch(vz, g, i, j, k), fetch(vz, g, i, j, k + 1));
    // shear terms at the shear points
    float vxy = d4(g.c1y, g.c2y, fetch(vx, g, i, j - 1, k), fetch(vx, g, i, j, k),
                   fetch(vx, g, i, j + 1, k), fetch(vx, g, i, j + 2, k));
    float vyx = d4(g.c1x, g.c2x, fetch(vy, g, i - 1, j, k), fetch(vy, g, i, j, k),
                   fetch(vy, g, i + 1, j, k), fetch(vy, g, i + 2, j, k));
    float vxz = d4(g.c1z, g.c2z, fetch(vx, g, i, j, k - 1), fetch(vx, g, i, j, k),
                   fetch(vx, g, i, j, k + 1), fetch(vx, g, i, j, k + 2));
    float vzx = d4(g.c1x, g.c2x, fetch(vz, g, i - 1, j, k), fetch(vz, g, i, j, k),
                   fetch(vz, g, i + 1, j, k), fetch(vz, g, i + 2, j, k));
    float vyz = d4(g.c1z, g.c2z, fetch(vy, g, i, j, k - 1), fetch(vy, g, i, j, k),
                   fetch(vy, g, i, j, k + 1), fetch(vy, g, i, j, k + 2));
    float vzy = d4(g.c1y, g.c2y, fetch(vz, g, i, j - 1, k), fetch(vz, g, i, j, k),
                   fetch(vz, g, i, j + 1, k), fetch(vz, g, i, j + 2, k));
    if (BND == BND_CPML) {
        const int W = B.W;
        if (in_slab(i, g.nx, W)) {
            long long pc = ((long long)k * g.ny + j) * (2 * W) + slab_idx(i, g.nx, W);
            float a = __ldg(B.pa[0] + i), b = __ldg(B.pb[0] + i);
            exx = pml(B.psx[3], pc, a, b, exx);
            vyx = pml(B.psx[4], pc, a, b, vyx);
            vzx = pml(B.psx[5], pc, a, b, vzx);
        }
        if (in_slab(j, g.ny, W)) {
            long long pc = ((long long)k * (2 * W) + slab_idx(j, g.ny, W)) * g.pitch + i;
            float a = __ldg(B.pa[1] + j), b = __ldg(B.pb[1] + j);
            eyy = pml(B.psy[3], pc, a, b, eyy);
            vxy = pml(B.psy[4], pc, a, b, vxy);
            vzy = pml(B.psy[5], pc, a, b, vzy);
        }
        if (in_slab(k, g.nz, W)) {
            long long pc = ((long long)slab_idx(k, g.nz, W) * g.ny + j) * g.pitch + i;
            float a = __ldg(B.pa[2] + k), b = __ldg(B.pb[2] + k);
            ezz = pml(B.psz[3], pc, a, b, ezz);
            vxz = pml(B.psz[4], pc, a, b, vxz);
            vyz = pml(B.psz[5], pc, a, b, vyz);
        }
    }
    const long long c = (long long)k * g.plane + (long long)j * g.pitch + i;
    const float lam = __ldg(M.lam + c);
    const float mu0 = __ldg(M.mu + c);
    const float l2m = lam + 2.0f * mu0;
    const float mxp = med(M.mu, g, i + 1, j, k);
    const float myp = med(M.mu, g, i, j + 1, k);
    const float mzp = med(M.mu, g, i, j, k + 1);
    const float mxy = 0.25f * (mu0 + mxp + myp + med(M.mu, g, i + 1, j + 1, k));
    const float mxz = 0.25f * (mu0 + mxp + mzp + med(M.mu, g, i + 1, j, k + 1));
    const float myz = 0.25f * (mu0 + myp + mzp + med(M.mu, g, i, j + 1, k + 1));
    float s0 = F.f[SXX][c] + dt * (l2m * exx + lam * (eyy + ezz));
    float s1 = F.f[SYY][c] + dt * (l2m * eyy + lam * (exx + ezz));
    float s2 = F.f[SZZ][c] + dt * (l2m * ezz + lam * (exx + eyy));
    float s3 = F.f[SXY][c] + dt * mxy * (vxy + vyx);
    float s4 = F.f[SXZ][c] + dt * mxz * (vxz + vzx);
    float s5 = F.f[SYZ][c] + dt * myz * (vyz + vzy);
    if (BND == BND_SPONGE) {
        const float G = __ldg(B.g[0] + i) * __ldg(B.g[1] + j) * __ldg(B.g[2] + k);
        s0 *= G; s1 *= G; s2 *= G; s3 *= G; s4 *= G; s5 *= G;
    }
    F.f[SXX][c] = s0;
    F.f[SYY][c] = s1;
    F.f[SZZ][c] = s2;
    F.f[SXY][c] = s3;
    F.f[SXZ][c] = s4;
    F.f[SYZ][c] = s5;
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

cudaError_t launch_velocity(const DevGrid& g, const DevFields& F, const DevMedium& M,
                            const DevBoundary& B, float dt, cudaStream_t st) {
    dim3 blk(32, 8), grd = plane_grid(g);
    switch (B.kind) {
        case BND_SPONGE: k_velocity<BND_SPONGE><<<grd, blk, 0, st>>>(g, F, M, B, dt); break;
        case BND_CPML: k_velocity<BND_CPML><<<grd, blk, 0, st>>>(g, F, M, B, dt); break;
        default: k_velocity<BND_NONE><<<grd, blk, 0, st>>>(g, F, M, B, dt); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_stress(const DevGrid& g, const DevFields& F, const DevMedium& M,
                          const DevBoundary& B, float dt, cudaStream_t st) {
    dim3 blk(32, 8), grd = plane_grid(g);
    switch (B.kind) {
        case BND_SPONGE: k_stress<BND_SPONGE><<<grd, blk, 0, st>>>(g, F, M, B, dt); break;
        case BND_CPML: k_stress<BND_CPML><<<grd, blk, 0, st>>>(g, F, M, B, dt); break;
        default: k_stress<BND_NONE><<<grd, blk, 0, st>>>(g, F, M, B, dt); break;
    }
    return cudaGetLastError();
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
