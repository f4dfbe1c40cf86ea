// ews_stencil.cu -- velocity and stress passes of the staggered scheme on
// sm_103a: TMA plane tiles into an mbarrier ring, register queues along z.
//
// Each CTA owns a 32 x TY (x, y) column of cells (each thread ROWS vertically
// adjacent cells of it) and marches through z.  For every z-plane p one
// thread issues TMA tile loads of all fields the pass reads into one slot of
// a 4-slot shared-memory ring:
//   * "halo" boxes of 40 x (TY + 4) cells (x from x0-4, y from y0-2) for
//     fields whose x or y derivative is taken, so every Eq. 4 tap (+-3/2
//     around a staggered point) of the tile sits in shared memory;
//   * "core" boxes of 32 x TY cells for fields read only at the cell itself.
// TMA writes zeros outside the grid, which is exactly the zero exterior of
// the wavefields (Sec. 2.2.2 reading), so there are no edge branches.
// z-derivatives come from per-thread register queues of 4 planes.  Output
// plane k is computed when plane k+2 lands; plane k's slot is then refilled
// with plane k+4.  The z-loop is unrolled by the ring depth, so slot
// indices, queue rotations and shared-memory offsets are all compile-time
// constants.
//
// Each CTA takes one (tile, z-chunk); all tiles share the chunk boundaries
// and chunk c of every tile is resident in the same wave, so neighbouring
// tiles march through z together and halo re-reads are served by L2.  Every
// mbarrier wait is bounded: on timeout the CTA records the failure in *err,
// waits (bounded too) for its copies in flight and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <new>

#include "ews_internal.cuh"
#ifndef EWS_L2PROMO
#define EWS_L2PROMO CU_TENSOR_MAP_L2_PROMOTION_L2_256B
#endif

namespace ews {

namespace {

#ifndef EWS_TILE_Y
#define EWS_TILE_Y 8
#endif
#ifndef EWS_ROWS
#define EWS_ROWS 1
#endif
#ifndef EWS_WAVES
#define EWS_WAVES 4
#endif
constexpr int TX = 32, TY = EWS_TILE_Y;
constexpr int HX = TX + 8, HY = TY + 4;          // halo box
constexpr int HALO = HX * HY;                     // floats per halo tile
constexpr int CORE = TX * TY;                     // floats per core tile
constexpr int NSLOT = 4;                          // ring depth (planes) = unroll
constexpr int MAXH = 6, MAXC = 7;
constexpr int ROWS = EWS_ROWS;                    // cells per thread (adjacent y rows)
constexpr int RY = TY / ROWS;                     // thread rows
constexpr int NTH = TX * RY;                      // threads per CTA
// one slot holds every tile of one plane: velocity 6 halo + 4 core,
// stress 4 halo + 7 core
constexpr int SLOT_MAIN = (6 * HALO + 4 * CORE) > (4 * HALO + 7 * CORE)
                              ? (6 * HALO + 4 * CORE) : (4 * HALO + 7 * CORE);
static_assert((SLOT_MAIN * 4) % 128 == 0 && (HALO * 4) % 128 == 0 && (CORE * 4) % 128 == 0,
              "TMA destinations must stay 128-byte aligned");
static_assert(TY % ROWS == 0, "rows per thread must divide the tile height");
template <int BND>
__host__ __device__ constexpr int slot_floats() { return SLOT_MAIN; }
// C-PML memory variables of the output plane live in one extra buffer of 9
// core tiles (3 terms for each damped direction), refilled for the next
// output plane as soon as the current one has been consumed.
constexpr int PSI_FLOATS = 9 * CORE;
template <int BND>
constexpr size_t smem_bytes() {
    return (NSLOT * SLOT_MAIN + (BND == BND_CPML ? PSI_FLOATS : 0)) * sizeof(float) +
           8 * (NSLOT + 1);
}
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait

// --- PTX wrappers -------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on the phase `parity` of an mbarrier.
__device__ __noinline__ bool mbar_wait_slow(uint64_t* bar, uint32_t parity) {
    const unsigned long long t0 = now_ns();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (now_ns() - t0 > kWaitNs) return false;
        __nanosleep(64);
    }
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    return mbar_try(bar, parity) || mbar_wait_slow(bar, parity);
}

__device__ __forceinline__ void tma_load_3d(float* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

struct Maps {
    CUtensorMap halo[MAXH];
    CUtensorMap core[MAXC];
    CUtensorMap psi[9];      // C-PML terms of this pass: [3 * direction + term]
};

struct PassParams {
    DevGrid g;
    DevFields F;
    DevBoundary B;
    float dt;
    int ntx, nty;
    int zchunk;           // planes per z-chunk
    int* err;
};

// Issue the TMA loads of z-plane `z` of tile (x0, y0) into `slot`.
template <int NH, int NC>
__device__ __forceinline__ void issue_plane(const Maps& m, float* slot, uint64_t* bar, int x0,
                                            int y0, int z) {
    mbar_expect_tx(bar, (NH * HALO + NC * CORE) * (uint32_t)sizeof(float));
#pragma unroll
    for (int h = 0; h < NH; ++h) tma_load_3d(slot + h * HALO, &m.halo[h], bar, x0 - 4, y0 - 2, z);
#pragma unroll
    for (int c = 0; c < NC; ++c)
        tma_load_3d(slot + NH * HALO + c * CORE, &m.core[c], bar, x0, y0, z);
}

// Issue the TMA loads of the C-PML memory variables of plane `z` for the
// damped directions in `dirs` (bit d = direction d) into `buf`.
__device__ __forceinline__ void issue_psi(const Maps& m, float* buf, uint64_t* bar, int x0, int y0,
                                          int z, unsigned dirs) {
    mbar_expect_tx(bar, __popc(dirs) * 3 * CORE * (uint32_t)sizeof(float));
#pragma unroll
    for (int d = 0; d < 3; ++d)
        if ((dirs >> d) & 1u)
#pragma unroll
            for (int q = 0; q < 3; ++q)
                tma_load_3d(buf + (3 * d + q) * CORE, &m.psi[3 * d + q], bar, x0, y0, z);
}

__device__ __forceinline__ bool in_slab(int i, int n, int W) { return i < W || i >= n - W; }
__device__ __forceinline__ int slab_idx(int i, int n, int W) { return i < W ? i : i - (n - 2 * W); }

__device__ __forceinline__ void ring_init(uint64_t* bars, int tid) {
    if (tid == 0) {
        for (int s = 0; s <= NSLOT; ++s) mbar_init(&bars[s], 1);   // ring + psi buffer
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
}

// Bounded-failure exit: record, wait for the loads still in flight
// (planes m .. issued - 1 of the chunk), leave.
__device__ __noinline__ void fail_exit(int* err, int bit, uint64_t* bars, int m, int issued,
                                       bool psi_pending, uint32_t psi_parity) {
    atomicOr(err, bit);
    if (psi_pending && !mbar_wait(&bars[NSLOT], psi_parity)) return;
    for (int q = m; q < issued; ++q)
        if (!mbar_wait(&bars[q & (NSLOT - 1)], (uint32_t)((q >> 2) & 1))) return;
}

// Per-thread geometry shared by both passes.
template <int BND>
struct Geo {
    int x0, y0, z0, P4, i, j0, hc, cc, cx, W;
    unsigned tdirs;                                   // tile inside the x / y slabs
    bool own[ROWS], sy[ROWS], sx;
    int cy[ROWS];
    float gx, gy[ROWS];
    float pax, pbx, pay[ROWS], pby[ROWS];            // C-PML a, b of the x and y slabs
    long long obase;                                  // j0 * pitch + i

    __device__ __forceinline__ Geo(const PassParams& P) {
        const DevGrid& g = P.g;
        const int tx = threadIdx.x, ty = threadIdx.y;
        const int ntile = P.ntx * P.nty;
        const int t = (int)(blockIdx.x % ntile);
        z0 = (int)(blockIdx.x / ntile) * P.zchunk;
        const int z1 = min(g.nz, z0 + P.zchunk);
        P4 = z1 - z0 + 4;                             // planes z0-2 .. z1+1
        x0 = (t % P.ntx) * TX;
        y0 = (t / P.ntx) * TY;
        i = x0 + tx;
        j0 = y0 + ROWS * ty;
        hc = (ROWS * ty + 2) * HX + tx + 4;           // row 0 cell in a halo tile
        cc = ROWS * ty * TX + tx;                     // row 0 cell in a core tile
        cx = (i + 1 < g.nx) ? 1 : 0;                  // medium clamp at the top edges
        W = P.B.W;
        tdirs = 0;
        if (BND == BND_CPML) {
            if (x0 < W || x0 + TX > g.nx - W) tdirs |= 1u;
            if (y0 < W || y0 + TY > g.ny - W) tdirs |= 2u;
        }
        sx = BND == BND_CPML && in_slab(i, g.nx, W);
        gx = (BND == BND_SPONGE && i < g.nx) ? __ldg(P.B.g[0] + i) : 1.0f;
        pax = sx ? __ldg(P.B.pa[0] + i) : 0.f;
        pbx = sx ? __ldg(P.B.pb[0] + i) : 0.f;
        obase = (long long)j0 * g.pitch + i;
#pragma unroll
        for (int rr = 0; rr < ROWS; ++rr) {
            const int j = j0 + rr;
            own[rr] = i < g.nx && j < g.ny;
            cy[rr] = (j + 1 < g.ny) ? HX : 0;
            sy[rr] = BND == BND_CPML && in_slab(j, g.ny, W);
            gy[rr] = (BND == BND_SPONGE && own[rr]) ? __ldg(P.B.g[1] + j) : 1.0f;
            pay[rr] = sy[rr] ? __ldg(P.B.pa[1] + j) : 0.f;
            pby[rr] = sy[rr] ? __ldg(P.B.pb[1] + j) : 0.f;
        }
    }
    // damped directions whose memory variables plane z needs
    __device__ __forceinline__ unsigned dirs(int z, int nz) const {
        return tdirs | ((z >= 0 && z < nz && (z < W || z >= nz - W)) ? 4u : 0u);
    }
};

// psi = b psi + a d; d += psi for the three terms of one damped direction.
__device__ __forceinline__ void pml_upd(float& p0, float& p1, float& p2, float a, float b,
                                        float& d0, float& d1, float& d2) {
    p0 = b * p0 + a * d0; d0 += p0;
    p1 = b * p1 + a * d1; d1 += p1;
    p2 = b * p2 + a * d2; d2 += p2;
}

// ------------------------------------------------------------------------------
// Velocity pass (Eq. 1 + Eq. 4): halo tiles sxx syy sxy sxz syz rho, core
// tiles szz vx vy vz.
// ------------------------------------------------------------------------------
enum { VH_SXX, VH_SYY, VH_SXY, VH_SXZ, VH_SYZ, VH_RHO };
enum { VC_SZZ, VC_VX, VC_VY, VC_VZ };

template <int BND>
struct VelQ {
    float zz[ROWS][4], xz[ROWS][4], yz[ROWS][4];   // sigma_zz k-1..k+2, sigma_xz/yz k-2..k+1
};

// One arrival of the z-loop, ring position PH = m mod 4.  Returns false if
// the CTA must stop (a wait gave up).
template <int BND, int PH>
__device__ __forceinline__ bool vel_step(const Maps& maps, const PassParams& P, const Geo<BND>& G,
                                         VelQ<BND>& Q, float* sm, uint64_t* bars, int m,
                                         uint32_t& psi_n) {
    const DevGrid& g = P.g;
    constexpr int SF = slot_floats<BND>();
    constexpr int S0 = PH, S1 = (PH + 3) & 3, S2 = (PH + 2) & 3;   // planes p, p-1, p-2
    const int k = G.z0 - 4 + m;                                    // output plane
    const bool out = m >= 4;
    // per-plane boundary coefficients of the output plane, fetched before the wait
    const bool sz = BND == BND_CPML && out && in_slab(k, g.nz, G.W);
    const float paz = sz ? __ldg(P.B.pa[2] + k) : 0.f, pbz = sz ? __ldg(P.B.pb[2] + k) : 0.f;
    const float G3 = (BND == BND_SPONGE && out) ? G.gx * __ldg(P.B.g[2] + k) : 1.0f;
    const unsigned kd = (BND == BND_CPML && out) ? G.dirs(k, g.nz) : 0u;   // damped dirs of k
    bool ok = mbar_wait(&bars[S0], (uint32_t)((m >> 2) & 1));
    if (BND == BND_CPML && kd) ok = mbar_wait(&bars[NSLOT], psi_n & 1u) && ok;
    const float* sl0 = sm + S0 * SF;
    const float* sl1 = sm + S1 * SF;
    // push own-column values: sigma_zz of plane p, sigma_xz / sigma_yz of p - 1
#pragma unroll
    for (int rr = 0; rr < ROWS; ++rr) {
        Q.zz[rr][PH] = sl0[6 * HALO + VC_SZZ * CORE + G.cc + rr * TX];
        if (m > 0) {
            Q.xz[rr][PH] = sl1[VH_SXZ * HALO + G.hc + rr * HX];
            Q.yz[rr][PH] = sl1[VH_SYZ * HALO + G.hc + rr * HX];
        }
    }
    if (out && ok) {
        constexpr int A = (PH + 1) & 3, B = (PH + 2) & 3, C = (PH + 3) & 3, D = PH;  // oldest..newest
        const float* sk = sm + S2 * SF + G.hc;           // plane k, own cell
        const float* hxx = sk + VH_SXX * HALO;
        const float* hyy = sk + VH_SYY * HALO;
        const float* hxy = sk + VH_SXY * HALO;
        const float* hxz = sk + VH_SXZ * HALO;
        const float* hyz = sk + VH_SYZ * HALO;
        const float* hr = sk + VH_RHO * HALO;
        const float* hr1 = sl1 + VH_RHO * HALO + G.hc;            // plane k + 1
        const float* vc = sm + S2 * SF + 6 * HALO + G.cc;
        const bool ktop = k + 1 < g.nz;
        const long long o = (long long)k * g.plane + G.obase;
#pragma unroll
        for (int rr = 0; rr < ROWS; ++rr) {
            if (!G.own[rr]) continue;
            const int R = rr * HX;
            const float* qxz = Q.xz[rr];
            const float* qyz = Q.yz[rr];
            const float* qzz = Q.zz[rr];
            // vx at (i+1/2, j, k)
            float dxx = g.c1x * (hxx[R + 1] - hxx[R]) + g.c2x * (hxx[R + 2] - hxx[R - 1]);
            float dxy = g.c1y * (hxy[R] - hxy[R - HX]) + g.c2y * (hxy[R + HX] - hxy[R - 2 * HX]);
            float dxz = g.c1z * (qxz[C] - qxz[B]) + g.c2z * (qxz[D] - qxz[A]);
            // vy at (i, j+1/2, k)
            float dyx = g.c1x * (hxy[R] - hxy[R - 1]) + g.c2x * (hxy[R + 1] - hxy[R - 2]);
            float dyy = g.c1y * (hyy[R + HX] - hyy[R]) + g.c2y * (hyy[R + 2 * HX] - hyy[R - HX]);
            float dyz = g.c1z * (qyz[C] - qyz[B]) + g.c2z * (qyz[D] - qyz[A]);
            // vz at (i, j, k+1/2)
            float dzx = g.c1x * (hxz[R] - hxz[R - 1]) + g.c2x * (hxz[R + 1] - hxz[R - 2]);
            float dzy = g.c1y * (hyz[R] - hyz[R - HX]) + g.c2y * (hyz[R + HX] - hyz[R - 2 * HX]);
            float dzz = g.c1z * (qzz[C] - qzz[B]) + g.c2z * (qzz[D] - qzz[A]);
            if (BND == BND_CPML) {
                // memory variables of plane k from the slot, updated, stored
                const float* ps = sm + NSLOT * SLOT_MAIN + G.cc + rr * TX;
                const long long oo = o + rr * g.pitch;
                if (G.sx) {
                    float p0 = ps[0 * CORE], p1 = ps[1 * CORE], p2 = ps[2 * CORE];
                    pml_upd(p0, p1, p2, G.pax, G.pbx, dxx, dyx, dzx);
                    P.B.psi[0][oo] = p0; P.B.psi[1][oo] = p1; P.B.psi[2][oo] = p2;
                }
                if (G.sy[rr]) {
                    float p0 = ps[3 * CORE], p1 = ps[4 * CORE], p2 = ps[5 * CORE];
                    pml_upd(p0, p1, p2, G.pay[rr], G.pby[rr],
                            dxy, dyy, dzy);
                    P.B.psi[6][oo] = p0; P.B.psi[7][oo] = p1; P.B.psi[8][oo] = p2;
                }
                if (sz) {
                    float p0 = ps[6 * CORE], p1 = ps[7 * CORE], p2 = ps[8 * CORE];
                    pml_upd(p0, p1, p2, paz, pbz, dxz, dyz, dzz);
                    P.B.psi[12][oo] = p0; P.B.psi[13][oo] = p1; P.B.psi[14][oo] = p2;
                }
            }
            // buoyancy at the v points: 1 / mean of the two adjacent densities
            const float r0 = hr[R];
            const float bx = __fdividef(2.0f, r0 + hr[R + G.cx]);
            const float by = __fdividef(2.0f, r0 + hr[R + G.cy[rr]]);
            const float bz = __fdividef(2.0f, r0 + (ktop ? hr1[R] : r0));
            float vx = vc[VC_VX * CORE + rr * TX] + P.dt * bx * (dxx + dxy + dxz);
            float vy = vc[VC_VY * CORE + rr * TX] + P.dt * by * (dyx + dyy + dyz);
            float vz = vc[VC_VZ * CORE + rr * TX] + P.dt * bz * (dzx + dzy + dzz);
            if (BND == BND_SPONGE) {
                const float Gs = G3 * G.gy[rr];
                vx *= Gs; vy *= Gs; vz *= Gs;
            }
            const long long oo = o + rr * g.pitch;
            P.F.f[VX][oo] = vx;
            P.F.f[VY][oo] = vy;
            P.F.f[VZ][oo] = vz;
        }
    }
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0 && threadIdx.y == 0)
            fail_exit(P.err, 1, bars, m, min(G.P4, max(NSLOT, m + 2)), kd != 0u, psi_n & 1u);
        return false;
    }
    if (BND == BND_CPML) {
        if (kd) ++psi_n;
        // the psi buffer is free: fetch the memory variables of the next output plane
        const int kn = k + 1;
        if (m >= 3 && kn < G.z0 + G.P4 - 4 && threadIdx.x == 0 && threadIdx.y == 0) {
            const unsigned dn = G.dirs(kn, g.nz);
            if (dn) issue_psi(maps, sm + NSLOT * SLOT_MAIN, &bars[NSLOT], G.x0, G.y0, kn, dn);
        }
    }
    // plane k's slot (S2) is free: refill it with plane z0 - 2 + (m + 2)
    if (m >= 2 && m + 2 < G.P4 && threadIdx.x == 0 && threadIdx.y == 0)
        issue_plane<6, 4>(maps, sm + S2 * SF, &bars[S2], G.x0, G.y0, G.z0 + m);
    return true;
}

// CTAs per SM that the shared-memory footprint allows; the register budget of
// the kernels is sized for exactly that many.
template <int BND>
constexpr int min_blocks() {
    return (227 * 1024) / (int)(smem_bytes<BND>() + 1024) < 1   ? 1
           : (227 * 1024) / (int)(smem_bytes<BND>() + 1024) > 4 ? 4
                                                                : (227 * 1024) / (int)(smem_bytes<BND>() + 1024);
}

template <int BND>
__global__ void __launch_bounds__(NTH, min_blocks<BND>()) k_velocity(const __grid_constant__ Maps maps,
                                                                  const PassParams P) {
    extern __shared__ __align__(128) float sm[];
    constexpr int SF = slot_floats<BND>();
    uint64_t* bars = reinterpret_cast<uint64_t*>(
        sm + NSLOT * SF + (BND == BND_CPML ? PSI_FLOATS : 0));
    ring_init(bars, threadIdx.y * TX + threadIdx.x);
    const Geo<BND> G(P);
    if (threadIdx.x == 0 && threadIdx.y == 0)
        for (int s = 0; s < NSLOT && s < G.P4; ++s)
            issue_plane<6, 4>(maps, sm + s * SF, &bars[s], G.x0, G.y0, G.z0 - 2 + s);
    VelQ<BND> Q;
#pragma unroll
    for (int rr = 0; rr < ROWS; ++rr)
#pragma unroll
        for (int q = 0; q < 4; ++q) { Q.zz[rr][q] = 0.f; Q.xz[rr][q] = 0.f; Q.yz[rr][q] = 0.f; }
    uint32_t psi_n = 0;                            // psi-buffer fills consumed
    for (int m = 0; m < G.P4; m += 4) {
        if (!vel_step<BND, 0>(maps, P, G, Q, sm, bars, m, psi_n)) return;
        if (m + 1 < G.P4 && !vel_step<BND, 1>(maps, P, G, Q, sm, bars, m + 1, psi_n)) return;
        if (m + 2 < G.P4 && !vel_step<BND, 2>(maps, P, G, Q, sm, bars, m + 2, psi_n)) return;
        if (m + 3 < G.P4 && !vel_step<BND, 3>(maps, P, G, Q, sm, bars, m + 3, psi_n)) return;
    }
}

// ------------------------------------------------------------------------------
// Stress pass (Eq. 2/3 + Eq. 4): halo tiles vx vy vz mu, core tiles lambda
// and the six stresses.
// ------------------------------------------------------------------------------
enum { SH_VX, SH_VY, SH_VZ, SH_MU };
enum { SC_LAM, SC_SXX, SC_SYY, SC_SZZ, SC_SXY, SC_SXZ, SC_SYZ };

template <int BND>
struct StrQ {
    float vx[ROWS][4], vy[ROWS][4], vz[ROWS][4];   // vx/vy k-1..k+2, vz k-2..k+1
};

template <int BND, int PH>
__device__ __forceinline__ bool str_step(const Maps& maps, const PassParams& P, const Geo<BND>& G,
                                         StrQ<BND>& Q, float* sm, uint64_t* bars, int m,
                                         uint32_t& psi_n) {
    const DevGrid& g = P.g;
    constexpr int SF = slot_floats<BND>();
    constexpr int S0 = PH, S1 = (PH + 3) & 3, S2 = (PH + 2) & 3;   // planes p, p-1, p-2
    const int k = G.z0 - 4 + m;
    const bool out = m >= 4;
    // per-plane boundary coefficients of the output plane, fetched before the wait
    const bool sz = BND == BND_CPML && out && in_slab(k, g.nz, G.W);
    const float paz = sz ? __ldg(P.B.pa[2] + k) : 0.f, pbz = sz ? __ldg(P.B.pb[2] + k) : 0.f;
    const float G3 = (BND == BND_SPONGE && out) ? G.gx * __ldg(P.B.g[2] + k) : 1.0f;
    const unsigned kd = (BND == BND_CPML && out) ? G.dirs(k, g.nz) : 0u;   // damped dirs of k
    bool ok = mbar_wait(&bars[S0], (uint32_t)((m >> 2) & 1));
    if (BND == BND_CPML && kd) ok = mbar_wait(&bars[NSLOT], psi_n & 1u) && ok;
    const float* sl0 = sm + S0 * SF;
    const float* sl1 = sm + S1 * SF;
    // push own-column values: vx, vy of plane p, vz of plane p - 1
#pragma unroll
    for (int rr = 0; rr < ROWS; ++rr) {
        Q.vx[rr][PH] = sl0[SH_VX * HALO + G.hc + rr * HX];
        Q.vy[rr][PH] = sl0[SH_VY * HALO + G.hc + rr * HX];
        if (m > 0) Q.vz[rr][PH] = sl1[SH_VZ * HALO + G.hc + rr * HX];
    }
    if (out && ok) {
        constexpr int A = (PH + 1) & 3, B = (PH + 2) & 3, C = (PH + 3) & 3, D = PH;
        const float* sk = sm + S2 * SF + G.hc;           // plane k, own cell
        const float* hvx = sk + SH_VX * HALO;
        const float* hvy = sk + SH_VY * HALO;
        const float* hvz = sk + SH_VZ * HALO;
        const float* hmu = sk + SH_MU * HALO;
        const float* hmu1 = (k + 1 < g.nz ? sl1 + G.hc : sk) + SH_MU * HALO;   // plane k + 1
        const float* cr = sm + S2 * SF + 4 * HALO + G.cc;
        const long long o = (long long)k * g.plane + G.obase;
#pragma unroll
        for (int rr = 0; rr < ROWS; ++rr) {
            if (!G.own[rr]) continue;
            const int R = rr * HX;
            const float* qvx = Q.vx[rr];
            const float* qvy = Q.vy[rr];
            const float* qvz = Q.vz[rr];
            // normal strain rates at (i, j, k)
            float exx = g.c1x * (hvx[R] - hvx[R - 1]) + g.c2x * (hvx[R + 1] - hvx[R - 2]);
            float eyy = g.c1y * (hvy[R] - hvy[R - HX]) + g.c2y * (hvy[R + HX] - hvy[R - 2 * HX]);
            float ezz = g.c1z * (qvz[C] - qvz[B]) + g.c2z * (qvz[D] - qvz[A]);
            // shear terms at the shear points
            float vxy = g.c1y * (hvx[R + HX] - hvx[R]) + g.c2y * (hvx[R + 2 * HX] - hvx[R - HX]);
            float vyx = g.c1x * (hvy[R + 1] - hvy[R]) + g.c2x * (hvy[R + 2] - hvy[R - 1]);
            float vxz = g.c1z * (qvx[C] - qvx[B]) + g.c2z * (qvx[D] - qvx[A]);
            float vzx = g.c1x * (hvz[R + 1] - hvz[R]) + g.c2x * (hvz[R + 2] - hvz[R - 1]);
            float vyz = g.c1z * (qvy[C] - qvy[B]) + g.c2z * (qvy[D] - qvy[A]);
            float vzy = g.c1y * (hvz[R + HX] - hvz[R]) + g.c2y * (hvz[R + 2 * HX] - hvz[R - HX]);
            if (BND == BND_CPML) {
                const float* ps = sm + NSLOT * SLOT_MAIN + G.cc + rr * TX;
                const long long oo = o + rr * g.pitch;
                if (G.sx) {
                    float p0 = ps[0 * CORE], p1 = ps[1 * CORE], p2 = ps[2 * CORE];
                    pml_upd(p0, p1, p2, G.pax, G.pbx, exx, vyx, vzx);
                    P.B.psi[3][oo] = p0; P.B.psi[4][oo] = p1; P.B.psi[5][oo] = p2;
                }
                if (G.sy[rr]) {
                    float p0 = ps[3 * CORE], p1 = ps[4 * CORE], p2 = ps[5 * CORE];
                    pml_upd(p0, p1, p2, G.pay[rr], G.pby[rr],
                            eyy, vxy, vzy);
                    P.B.psi[9][oo] = p0; P.B.psi[10][oo] = p1; P.B.psi[11][oo] = p2;
                }
                if (sz) {
                    float p0 = ps[6 * CORE], p1 = ps[7 * CORE], p2 = ps[8 * CORE];
                    pml_upd(p0, p1, p2, paz, pbz, ezz, vxz, vyz);
                    P.B.psi[15][oo] = p0; P.B.psi[16][oo] = p1; P.B.psi[17][oo] = p2;
                }
            }
            // medium: lambda, mu at the cell; mu means at the shear points
            const int cyr = G.cy[rr];
            const float lam = cr[SC_LAM * CORE + rr * TX];
            const float mu0 = hmu[R], mxp = hmu[R + G.cx], myp = hmu[R + cyr];
            const float mzp = hmu1[R];
            const float mxy = 0.25f * (mu0 + mxp + myp + hmu[R + G.cx + cyr]);
            const float mxz = 0.25f * (mu0 + mxp + mzp + hmu1[R + G.cx]);
            const float myz = 0.25f * (mu0 + myp + mzp + hmu1[R + cyr]);
            const float l2m = lam + 2.0f * mu0;
            float s0 = cr[SC_SXX * CORE + rr * TX] + P.dt * (l2m * exx + lam * (eyy + ezz));
            float s1 = cr[SC_SYY * CORE + rr * TX] + P.dt * (l2m * eyy + lam * (exx + ezz));
            float s2 = cr[SC_SZZ * CORE + rr * TX] + P.dt * (l2m * ezz + lam * (exx + eyy));
            float s3 = cr[SC_SXY * CORE + rr * TX] + P.dt * mxy * (vxy + vyx);
            float s4 = cr[SC_SXZ * CORE + rr * TX] + P.dt * mxz * (vxz + vzx);
            float s5 = cr[SC_SYZ * CORE + rr * TX] + P.dt * myz * (vyz + vzy);
            if (BND == BND_SPONGE) {
                const float Gs = G3 * G.gy[rr];
                s0 *= Gs; s1 *= Gs; s2 *= Gs; s3 *= Gs; s4 *= Gs; s5 *= Gs;
            }
            const long long oo = o + rr * g.pitch;
            P.F.f[SXX][oo] = s0;
            P.F.f[SYY][oo] = s1;
            P.F.f[SZZ][oo] = s2;
            P.F.f[SXY][oo] = s3;
            P.F.f[SXZ][oo] = s4;
            P.F.f[SYZ][oo] = s5;
        }
    }
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0 && threadIdx.y == 0)
            fail_exit(P.err, 2, bars, m, min(G.P4, max(NSLOT, m + 2)), kd != 0u, psi_n & 1u);
        return false;
    }
    if (BND == BND_CPML) {
        if (kd) ++psi_n;
        // the psi buffer is free: fetch the memory variables of the next output plane
        const int kn = k + 1;
        if (m >= 3 && kn < G.z0 + G.P4 - 4 && threadIdx.x == 0 && threadIdx.y == 0) {
            const unsigned dn = G.dirs(kn, g.nz);
            if (dn) issue_psi(maps, sm + NSLOT * SLOT_MAIN, &bars[NSLOT], G.x0, G.y0, kn, dn);
        }
    }
    if (m >= 2 && m + 2 < G.P4 && threadIdx.x == 0 && threadIdx.y == 0)
        issue_plane<4, 7>(maps, sm + S2 * SF, &bars[S2], G.x0, G.y0, G.z0 + m);
    return true;
}

template <int BND>
__global__ void __launch_bounds__(NTH, min_blocks<BND>()) k_stress(const __grid_constant__ Maps maps,
                                                                const PassParams P) {
    extern __shared__ __align__(128) float sm[];
    constexpr int SF = slot_floats<BND>();
    uint64_t* bars = reinterpret_cast<uint64_t*>(
        sm + NSLOT * SF + (BND == BND_CPML ? PSI_FLOATS : 0));
    ring_init(bars, threadIdx.y * TX + threadIdx.x);
    const Geo<BND> G(P);
    if (threadIdx.x == 0 && threadIdx.y == 0)
        for (int s = 0; s < NSLOT && s < G.P4; ++s)
            issue_plane<4, 7>(maps, sm + s * SF, &bars[s], G.x0, G.y0, G.z0 - 2 + s);
    StrQ<BND> Q;
#pragma unroll
    for (int rr = 0; rr < ROWS; ++rr)
#pragma unroll
        for (int q = 0; q < 4; ++q) { Q.vx[rr][q] = 0.f; Q.vy[rr][q] = 0.f; Q.vz[rr][q] = 0.f; }
    uint32_t psi_n = 0;                            // psi-buffer fills consumed
    for (int m = 0; m < G.P4; m += 4) {
        if (!str_step<BND, 0>(maps, P, G, Q, sm, bars, m, psi_n)) return;
        if (m + 1 < G.P4 && !str_step<BND, 1>(maps, P, G, Q, sm, bars, m + 1, psi_n)) return;
        if (m + 2 < G.P4 && !str_step<BND, 2>(maps, P, G, Q, sm, bars, m + 2, psi_n)) return;
        if (m + 3 < G.P4 && !str_step<BND, 3>(maps, P, G, Q, sm, bars, m + 3, psi_n)) return;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool encode(CUtensorMap* map, const DevGrid& g, const float* base, bool halo) {
    auto fn = encoder();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    cuuint64_t strides[2] = {(cuuint64_t)g.pitch * sizeof(float),
                             (cuuint64_t)g.plane * sizeof(float)};
    cuuint32_t box[3] = {(cuuint32_t)(halo ? HX : TX), (cuuint32_t)(halo ? HY : TY), 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims,
                    strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    EWS_L2PROMO, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <typename K>
cudaError_t prepare(K kern, size_t smem, int* blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, NTH, smem);
}

template <int BND>
cudaError_t occupancy(int* occ) {
    int a = 0, b = 0;
    cudaError_t e = prepare(k_velocity<BND>, smem_bytes<BND>(), &a);
    if (e == cudaSuccess) e = prepare(k_stress<BND>, smem_bytes<BND>(), &b);
    *occ = a < b ? a : b;
    return e;
}

}  // namespace

struct StencilPlan {
    Maps vmaps, smaps;
    int kind = 0;
    int grid = 0;
    int ntx = 0, nty = 0;
    int zchunk = 0;
};

cudaError_t stencil_plan_create(const DevGrid& g, const DevFields& F, const DevMedium& M,
                                const DevBoundary& B, StencilPlan** out) {
    StencilPlan* p = new StencilPlan();
    p->kind = B.kind;
    bool ok = true;
    // velocity: halo sxx syy sxy sxz syz rho; core szz vx vy vz
    const float* vh[6] = {F.f[SXX], F.f[SYY], F.f[SXY], F.f[SXZ], F.f[SYZ], M.rho};
    const float* vc[4] = {F.f[SZZ], F.f[VX], F.f[VY], F.f[VZ]};
    for (int h = 0; h < 6; ++h) ok &= encode(&p->vmaps.halo[h], g, vh[h], true);
    for (int c = 0; c < 4; ++c) ok &= encode(&p->vmaps.core[c], g, vc[c], false);
    // stress: halo vx vy vz mu; core lambda sxx syy szz sxy sxz syz
    const float* sh[4] = {F.f[VX], F.f[VY], F.f[VZ], M.mu};
    const float* sc[7] = {M.lam, F.f[SXX], F.f[SYY], F.f[SZZ], F.f[SXY], F.f[SXZ], F.f[SYZ]};
    for (int h = 0; h < 4; ++h) ok &= encode(&p->smaps.halo[h], g, sh[h], true);
    for (int c = 0; c < 7; ++c) ok &= encode(&p->smaps.core[c], g, sc[c], false);
    // C-PML memory variables: psi[6 d + t]; velocity pass t = 0..2, stress 3..5
    if (B.kind == BND_CPML)
        for (int d = 0; d < 3; ++d)
            for (int q = 0; q < 3; ++q) {
                ok &= encode(&p->vmaps.psi[3 * d + q], g, B.psi[6 * d + q], false);
                ok &= encode(&p->smaps.psi[3 * d + q], g, B.psi[6 * d + 3 + q], false);
            }
    if (!ok) {
        delete p;
        return cudaErrorInvalidValue;
    }
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        switch (B.kind) {
            case BND_SPONGE: e = occupancy<BND_SPONGE>(&occ); break;
            case BND_CPML: e = occupancy<BND_CPML>(&occ); break;
            default: e = occupancy<BND_NONE>(&occ); break;
        }
    }
    if (e != cudaSuccess || occ < 1) {
        delete p;
        return e != cudaSuccess ? e : cudaErrorInvalidConfiguration;
    }
    // Launch geometry: every tile column is cut into the same z-chunks and
    // chunk c of all tiles is resident at once, so neighbouring tiles march
    // through z together and the halo planes one CTA loads are still in L2
    // when its neighbours load them.  Use as many chunks as the resident
    // slots allow (at least 8 planes each); past one wave, whole columns.
    p->ntx = (g.nx + TX - 1) / TX;
    p->nty = (g.ny + TY - 1) / TY;
    const long long ntile = (long long)p->ntx * p->nty;
    const long long slots = (long long)sms * occ;
    long long nchunk = (slots * EWS_WAVES) / ntile;
    if (nchunk > g.nz / 8) nchunk = g.nz / 8;
    if (nchunk < 1) nchunk = 1;
    p->zchunk = (int)((g.nz + nchunk - 1) / nchunk);
    nchunk = (g.nz + p->zchunk - 1) / p->zchunk;
    p->grid = (int)(ntile * nchunk);
    *out = p;
    return cudaSuccess;
}

void stencil_plan_destroy(StencilPlan* p) { delete p; }

size_t stencil_plan_bytes() { return sizeof(StencilPlan); }

// Same plan as stencil_plan_create, built in caller-provided storage of at
// least stencil_plan_bytes() bytes (aligned to 64), without any allocation.
cudaError_t stencil_plan_fill(void* storage, const DevGrid& g, const DevFields& F,
                              const DevMedium& M, const DevBoundary& B, StencilPlan** out) {
    StencilPlan* p = ::new (storage) StencilPlan();
    p->kind = B.kind;
    bool ok = true;
    const float* vh[6] = {F.f[SXX], F.f[SYY], F.f[SXY], F.f[SXZ], F.f[SYZ], M.rho};
    const float* vc[4] = {F.f[SZZ], F.f[VX], F.f[VY], F.f[VZ]};
    for (int h = 0; h < 6; ++h) ok &= encode(&p->vmaps.halo[h], g, vh[h], true);
    for (int c = 0; c < 4; ++c) ok &= encode(&p->vmaps.core[c], g, vc[c], false);
    const float* sh[4] = {F.f[VX], F.f[VY], F.f[VZ], M.mu};
    const float* sc[7] = {M.lam, F.f[SXX], F.f[SYY], F.f[SZZ], F.f[SXY], F.f[SXZ], F.f[SYZ]};
    for (int h = 0; h < 4; ++h) ok &= encode(&p->smaps.halo[h], g, sh[h], true);
    for (int c = 0; c < 7; ++c) ok &= encode(&p->smaps.core[c], g, sc[c], false);
    if (B.kind == BND_CPML)
        for (int d = 0; d < 3; ++d)
            for (int q = 0; q < 3; ++q) {
                ok &= encode(&p->vmaps.psi[3 * d + q], g, B.psi[6 * d + q], false);
                ok &= encode(&p->smaps.psi[3 * d + q], g, B.psi[6 * d + 3 + q], false);
            }
    if (!ok) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        switch (B.kind) {
            case BND_SPONGE: e = occupancy<BND_SPONGE>(&occ); break;
            case BND_CPML: e = occupancy<BND_CPML>(&occ); break;
            default: e = occupancy<BND_NONE>(&occ); break;
        }
    }
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    p->ntx = (g.nx + TX - 1) / TX;
    p->nty = (g.ny + TY - 1) / TY;
    const long long ntile = (long long)p->ntx * p->nty;
    const long long slots = (long long)sms * occ;
    long long nchunk = (slots * EWS_WAVES) / ntile;
    if (nchunk > g.nz / 8) nchunk = g.nz / 8;
    if (nchunk < 1) nchunk = 1;
    p->zchunk = (int)((g.nz + nchunk - 1) / nchunk);
    nchunk = (g.nz + p->zchunk - 1) / p->zchunk;
    p->grid = (int)(ntile * nchunk);
    *out = p;
    return cudaSuccess;
}

cudaError_t launch_velocity(const StencilPlan* sp, const DevGrid& g, const DevFields& F,
                            const DevBoundary& B, float dt, int* err, cudaStream_t st) {
    PassParams P{g, F, B, dt, sp->ntx, sp->nty, sp->zchunk, err};
    dim3 blk(TX, RY);
    switch (B.kind) {
        case BND_SPONGE:
            k_velocity<BND_SPONGE><<<sp->grid, blk, smem_bytes<BND_SPONGE>(), st>>>(sp->vmaps, P);
            break;
        case BND_CPML:
            k_velocity<BND_CPML><<<sp->grid, blk, smem_bytes<BND_CPML>(), st>>>(sp->vmaps, P);
            break;
        default:
            k_velocity<BND_NONE><<<sp->grid, blk, smem_bytes<BND_NONE>(), st>>>(sp->vmaps, P);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_stress(const StencilPlan* sp, const DevGrid& g, const DevFields& F,
                          const DevBoundary& B, float dt, int* err, cudaStream_t st) {
    PassParams P{g, F, B, dt, sp->ntx, sp->nty, sp->zchunk, err};
    dim3 blk(TX, RY);
    switch (B.kind) {
        case BND_SPONGE:
            k_stress<BND_SPONGE><<<sp->grid, blk, smem_bytes<BND_SPONGE>(), st>>>(sp->smaps, P);
            break;
        case BND_CPML:
            k_stress<BND_CPML><<<sp->grid, blk, smem_bytes<BND_CPML>(), st>>>(sp->smaps, P);
            break;
        default:
            k_stress<BND_NONE><<<sp->grid, blk, smem_bytes<BND_NONE>(), st>>>(sp->smaps, P);
            break;
    }
    return cudaGetLastError();
}

}  // namespace ews
