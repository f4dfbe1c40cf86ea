// ews_stencil.cu -- velocity and stress passes of the staggered scheme on
// sm_103a: TMA plane tiles into an mbarrier ring, register queues along z.
//
// Each CTA owns a 32 x TY (x, y) column of cells (each thread ROWS vertically
// adjacent cells of it) and marches through z.  For every z-plane p one
// thread issues TMA tile loads of all fields the pass reads into one slot of
// a 4-slot shared-memory ring:
//   * halo boxes for fields whose x or y derivative is taken, each only as
//     wide as its derivatives need, so every Eq. 4 tap (+-3/2 around a
//     staggered point) of the tile sits in shared memory: 40 x TY cells (x
//     from x0-4) for x-derivatives only, 32 x (TY + 4) (y from y0-2) for
//     y-derivatives only, 40 x (TY + 4) for both;
//   * medium boxes of 40 x (TY + 1) cells (x from x0-4, y from y0): the cell
//     and its +x / +y neighbours for the staggered means;
//   * "core" boxes of 32 x TY cells for fields read only at the cell itself.
// The 9 wavefields are stored as FP32, BF16 or FP16 (the medium always as
// FP32); arithmetic is FP32.  A 16-bit field f holds s_f times its value, a
// power-of-two scale per field: derivatives are taken on stored values and
// multiplied by 1/s_f, updates by dt s_f of the output field.  16-bit halo
// boxes are 48 cells wide (x from x0-8) so that every copy starts on a
// 16-byte boundary.
// With C-PML, the memory variables of the output plane come through a
// separate two-entry buffer, filled two planes ahead (so their load latency
// overlaps two planes of work, like the field ring's).
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
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <new>
#include <type_traits>

#include "ews_internal.cuh"
#include "ews_ops.cuh"
#ifndef EWS_L2PROMO
#define EWS_L2PROMO CU_TENSOR_MAP_L2_PROMOTION_L2_256B
#endif

// This file is compiled once per tile shape.  The default build (32 x 8
// tiles) has every pass form, the batched executor and the entry points of
// ews_internal.cuh; a build with EWS_SHAPE_NS defined (ews_stencil_t4.cu,
// ews_stencil_t16.cu) holds only the plain forward passes (no free
// surface, no coarse medium grid, no history capture) with its own tile
// shape, inside namespace ews::EWS_SHAPE_NS.
#ifdef EWS_SHAPE_NS
#define EWS_FULL 0
#else
#define EWS_FULL 1
#endif

namespace ews {
#ifdef EWS_SHAPE_NS
namespace EWS_SHAPE_NS {
#endif

namespace {

#ifndef EWS_TILE_Y
#define EWS_TILE_Y 8
#endif
#ifndef EWS_ROWS
#define EWS_ROWS 1
#endif
constexpr int TX = 32, TY = EWS_TILE_Y;
constexpr int HY = TY + 4;                        // halo rows: y0-2 .. y0+TY+1
constexpr int HXF = TX + 8;                       // FP32 halo box: x0-4 .. x0+TX+3
constexpr int CORE = TX * TY;                     // elements per core tile
constexpr int NSLOT = 4;                          // ring depth (planes) = unroll
constexpr int MAXH = 6, MAXC = 1;
constexpr int ROWS = EWS_ROWS;                    // cells per thread (adjacent y rows)
constexpr int RY = TY / ROWS;                     // thread rows
constexpr int NTH = TX * RY;                      // threads per CTA
static_assert(TY % ROWS == 0, "rows per thread must divide the tile height");
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait

// Storage of the 9 wavefields: FP32, BF16 or FP16 (arithmetic is FP32).  A
// TMA tile must start on a 16-byte boundary, so a halo box of 16-bit fields
// starts 8 cells left of the tile (4 for FP32).
template <typename T> struct St;
template <> struct St<float> {
    static constexpr int HO = 4;
    static constexpr CUtensorMapDataType dtype = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    __device__ static float ld(const float* p) { return *p; }
    __device__ static float put(float x) { return x; }
};
template <> struct St<__nv_bfloat16> {
    static constexpr int HO = 8;
    static constexpr CUtensorMapDataType dtype = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    __device__ static float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    __device__ static __nv_bfloat16 put(float x) { return __float2bfloat16_rn(x); }
};
template <> struct St<__half> {
    static constexpr int HO = 8;
    static constexpr CUtensorMapDataType dtype = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    __device__ static float ld(const __half* p) { return __half2float(*p); }
    __device__ static __half put(float x) { return __float2half_rn(x); }
};

constexpr int r128(int b) { return (b + 127) / 128 * 128; }

// Slot layout of one plane, in bytes, following the copies that fill it
// (fields in their physical slot order, fslot):
//   velocity pass: sxx, sxz (x halos, one copy), syy, syz (y halos, one
//   copy), sxy (x and y halo), the rho medium box, and szz vx vy vz (core
//   tiles, one copy);
//   stress pass: vx vy vz (x and y halos, one copy), the lambda and mu medium
//   boxes (one copy), and the six stress core tiles in slot order (one copy).
// *_TX are the bytes the TMA copies of one plane deliver (the mbarrier's
// transaction count).  A copy's tiles lie back to back; each copy starts on
// a 128-byte boundary.
template <typename T>
struct Lay {
    static constexpr int ES = (int)sizeof(T);
    static constexpr int HX = TX + 2 * St<T>::HO;             // field x-halo box width
    static constexpr int XB = HX * TY * ES;                    // x-halo tile bytes
    static constexpr int YB = TX * HY * ES;                    // y-halo tile bytes
    static constexpr int HB = HX * HY * ES;                    // x- and y-halo tile bytes
    static constexpr int CB = CORE * ES;                       // core tile bytes
    static constexpr int MB = HXF * (TY + 1) * 4;              // FP32 medium box bytes
    static constexpr int FCB = CORE * 4;                       // FP32 core tile bytes
    static constexpr int HBF = HXF * HY * 4;                   // FP32 x- and y-halo tile bytes
    // velocity pass
    static constexpr int V_SXX = 0;
    static constexpr int V_SXZ = V_SXX + XB;
    static constexpr int V_SYY = r128(V_SXZ + XB);
    static constexpr int V_SYZ = V_SYY + YB;
    static constexpr int V_SXY = r128(V_SYZ + YB);
    static constexpr int V_RHO = r128(V_SXY + HB);
    static constexpr int V_CORE = r128(V_RHO + MB);
    static constexpr int V_BYTES = V_CORE + 4 * CB;
    static constexpr int V_TX = 2 * XB + 2 * YB + HB + MB + 4 * CB;
    // stress pass
    static constexpr int S_MU = r128(3 * HB);
    static constexpr int S_LAM = r128(S_MU + MB);
    static constexpr int S_CORE = S_LAM + FCB;
    static constexpr int S_BYTES = S_CORE + 6 * CB;
    static constexpr int S_TX = 3 * HB + MB + FCB + 6 * CB;
    static constexpr int VSLOT = r128(V_BYTES), SSLOT = r128(S_BYTES);
    static_assert(CB % 16 == 0 && XB % 16 == 0 && YB % 16 == 0 && HB % 16 == 0,
                  "tiles of one copy keep 16-byte alignment");
};

// Kernel modes of the velocity pass: plain forward; forward that also
// copies v^{n+1/2} into a history slot (checkpoint recomputation); reverse
// (adjoint) pass that also accumulates the gradient products, for which each
// slot carries the three velocity-history halo tiles of the same plane.
enum { M_FWD = 0, M_CAP = 1, M_GRAD = 2 };
// Velocity-pass slot (the reverse mode adds the three FP32 history tiles).
template <typename T, int MODE>
__host__ __device__ constexpr int vslot_bytes() {
    return MODE == M_GRAD ? r128(Lay<T>::V_BYTES + 3 * Lay<T>::HBF) : Lay<T>::VSLOT;
}

// C-PML memory variables: a two-entry buffer of 9 FP32 core tiles each (3
// terms for each damped direction).  Output plane k uses entry (k - z0) & 1,
// which is refilled with plane k + 2 as soon as plane k has been consumed.
constexpr int PSI_BYTES = 9 * CORE * 4;
constexpr int NPSI = 2;
// The reverse velocity pass reads, at its output cells only, the 8 FP32
// gradient accumulators and v^{m+3/2} (3 components): a two-entry buffer of
// 11 FP32 core tiles, used like the psi buffer (entry (k - z0) & 1, refilled
// with plane k + 2 after plane k).  C-PML has no reverse pass, so the two
// buffers never coexist and share the place below the ring.
constexpr int AUX_TILES = 11;
constexpr int AUX_BYTES = AUX_TILES * CORE * 4;
// Dynamic shared memory of a pass kernel: [psi buffer (C-PML) or accumulator
// buffer (reverse velocity pass)] [ring of NSLOT plane slots] [barriers].
__device__ __forceinline__ float* psi_base(unsigned char* ring) {
    return reinterpret_cast<float*>(ring - NPSI * PSI_BYTES);
}
__device__ __forceinline__ float* aux_base(unsigned char* ring) {
    return reinterpret_cast<float*>(ring - NPSI * AUX_BYTES);
}
template <int BND, bool GRAD>
constexpr size_t pre_bytes() {
    return BND == BND_CPML ? (size_t)NPSI * PSI_BYTES : GRAD ? (size_t)NPSI * AUX_BYTES : 0;
}
constexpr int NBAR = NSLOT + NPSI;                // ring barriers, then psi-buffer barriers
template <int BND, typename T, int MODE = M_FWD>
constexpr size_t smem_v() {
    return pre_bytes<BND, MODE == M_GRAD>() + (size_t)NSLOT * vslot_bytes<T, MODE>() + 8 * NBAR;
}
template <int BND, typename T>
constexpr size_t smem_s() {
    return pre_bytes<BND, false>() + (size_t)NSLOT * Lay<T>::SSLOT + 8 * NBAR;
}
// CTAs per SM that a shared-memory footprint allows (at most 4, and at most
// 3 for FP32 storage, whose passes need more than 64 registers); the register
// budget of the kernels is sized for exactly that many.
template <typename T>
constexpr int blocks_for(size_t smem) {
    return (227 * 1024) / (int)(smem + 1024) < 1 ? 1
           : (227 * 1024) / (int)(smem + 1024) > (sizeof(T) == 4 ? 3 : 4)
               ? (sizeof(T) == 4 ? 3 : 4)
               : (227 * 1024) / (int)(smem + 1024);
}

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

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z, int w) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z),
        "r"(w)
        : "memory");
}

// Tensor maps of one pass, in slot order: halo[] then core[] as listed in
// the slot layout above, then the C-PML terms [3 * direction + term].
static_assert(MAXH == kMapsHalo && MAXC == kMapsCore, "tensor-map counts of Maps");

// Issue the TMA loads of z-plane `z` of tile (x0, y0) into `slot`.
// CM: the medium is sampled from a coarse grid, so its tiles are not loaded.
template <typename T, int MODE, bool CM = false>
__device__ __forceinline__ void issue_vel(const Maps& m, unsigned char* slot, uint64_t* bar,
                                          int x0, int y0, int z, int hslot) {
    using L = Lay<T>;
    constexpr int HO = St<T>::HO;
    mbar_expect_tx(bar, (uint32_t)(L::V_TX + (MODE == M_GRAD ? 3 * L::HBF : 0) - (CM ? L::MB : 0)));
    tma_load_4d(slot + L::V_SXX, &m.halo[0], bar, x0 - HO, y0, z, fslot(SXX));      // sxx sxz
    tma_load_4d(slot + L::V_SYY, &m.halo[1], bar, x0, y0 - 2, z, fslot(SYY));       // syy syz
    tma_load_3d(slot + L::V_SXY, &m.halo[2], bar, x0 - HO, y0 - 2, z);                  // sxy
    if constexpr (!CM) tma_load_3d(slot + L::V_RHO, &m.halo[5], bar, x0 - 4, y0, z);
    tma_load_4d(slot + L::V_CORE, &m.core[0], bar, x0, y0, z, fslot(SZZ));          // szz vx vy vz
    if constexpr (MODE == M_GRAD)      // vx vy vz of history slot hslot, one copy
        tma_load_4d(slot + L::V_BYTES, &m.hist, bar, x0 - 4, y0 - 2, z, 3 * hslot);
}
template <typename T, bool CM = false>
__device__ __forceinline__ void issue_str(const Maps& m, unsigned char* slot, uint64_t* bar,
                                          int x0, int y0, int z) {
    using L = Lay<T>;
    mbar_expect_tx(bar, (uint32_t)(L::S_TX - (CM ? L::MB + L::FCB : 0)));
    tma_load_4d(slot, &m.halo[0], bar, x0 - St<T>::HO, y0 - 2, z, fslot(VX));   // vx vy vz
    if constexpr (!CM) {
        tma_load_3d(slot + L::S_MU, &m.halo[3], bar, x0 - 4, y0, z);                 // mu
        tma_load_3d(slot + L::S_LAM, &m.halo[4], bar, x0, y0, z);                    // lambda
    }
    tma_load_4d(slot + L::S_CORE, &m.core[0], bar, x0, y0, z, 0);                     // 6 stresses
}

// Issue the TMA loads of the C-PML memory variables of plane `z` for the
// damped directions in `dirs` (bit d = direction d) into `buf`: one copy of
// the 3 terms of each direction (arrays 6 d + t0 .. 6 d + t0 + 2; t0 = 0 for
// the velocity pass, 3 for the stress pass).
__device__ __forceinline__ void issue_psi(const Maps& m, float* buf, uint64_t* bar, int x0, int y0,
                                          int z, unsigned dirs, int t0) {
    mbar_expect_tx(bar, __popc(dirs) * 3 * CORE * (uint32_t)sizeof(float));
#pragma unroll
    for (int d = 0; d < 3; ++d)
        if ((dirs >> d) & 1u) tma_load_4d(buf + 3 * d * CORE, &m.psi, bar, x0, y0, z, 6 * d + t0);
}

__device__ __forceinline__ bool in_slab(int i, int n, int W) { return i < W || i >= n - W; }

__device__ __forceinline__ void ring_init(uint64_t* bars, int tid) {
    if (tid == 0) {
        for (int s = 0; s < NBAR; ++s) mbar_init(&bars[s], 1);     // ring + psi buffers
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
}

// Bounded-failure exit: record, wait for the loads still in flight
// (planes m .. issued - 1 of the chunk, and the psi-buffer entries whose bit
// is set in psi_pend, each on the phase given by its bit of psi_par), leave.
__device__ __noinline__ void fail_exit(int* err, int bit, uint64_t* bars, int m, int issued,
                                       unsigned psi_pend, unsigned psi_par) {
    atomicOr(err, bit);
    for (int b = 0; b < NPSI; ++b)
        if (((psi_pend >> b) & 1u) && !mbar_wait(&bars[NSLOT + b], (psi_par >> b) & 1u)) return;
    for (int q = m; q < issued; ++q)
        if (!mbar_wait(&bars[q & (NSLOT - 1)], (uint32_t)((q >> 2) & 1))) return;
}

// Per-thread geometry shared by both passes.
template <int BND, typename T>
struct Geo {
    int x0, y0, z0, P4, i, j0, hc, hf16, cc, cx, W;
    unsigned tdirs;                                   // tile inside the x / y slabs
    bool own[ROWS], sy[ROWS], sx;
    int cy[ROWS];                                     // medium y+1 offset (clamped) in FP32 tiles
    float gx, gy[ROWS];
    float pax, pbx, pay[ROWS], pby[ROWS];            // C-PML a, b of the x and y slabs
    long long obase;                                  // j0 * pitch + i

    // item = (z-chunk) * ntile + tile: the CTA index of a pass launch, or a
    // work item of the batched executor
    __device__ __forceinline__ Geo(const PassParams& P, int item) {
        const DevGrid& g = P.g;
        const int tx = threadIdx.x, ty = threadIdx.y;
        const int ntile = P.ntx * P.nty;
        const int t = item % ntile;
        z0 = (item / ntile) * P.zchunk;
        const int z1 = min(g.nz, z0 + P.zchunk);
        P4 = z1 - z0 + 4;                             // planes z0-2 .. z1+1
        x0 = (t % P.ntx) * TX;
        y0 = (t / P.ntx) * TY;
        i = x0 + tx;
        j0 = y0 + ROWS * ty;
        hc = (ROWS * ty + 2) * Lay<T>::HX + tx + St<T>::HO;   // row 0 cell, x- and y-halo tile
        hf16 = ROWS * ty * HXF + tx + 4;                      // row 0 cell, FP32 medium box
        cc = ROWS * ty * TX + tx;                             // row 0 cell, core tile
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
            cy[rr] = (j + 1 < g.ny) ? HXF : 0;
            sy[rr] = BND == BND_CPML && in_slab(j, g.ny, W);
            gy[rr] = (BND == BND_SPONGE && own[rr]) ? __ldg(P.B.g[1] + j) : 1.0f;
            pay[rr] = sy[rr] ? __ldg(P.B.pa[1] + j) : 0.f;
            pby[rr] = sy[rr] ? __ldg(P.B.pb[1] + j) : 0.f;
        }
    }
    // row 0 cell in an x-halo tile (no halo rows) and in a y-halo tile (the
    // core tile's row stride, two halo rows above)
    __device__ __forceinline__ int hcx() const { return hc - 2 * Lay<T>::HX; }
    __device__ __forceinline__ int hcy() const { return cc + 2 * TX; }
    // row 0 cell in an FP32 medium box (x from x0-4, no halo rows above);
    // with FP32 fields it is the x-halo tile's offset
    __device__ __forceinline__ int hf() const { return sizeof(T) == 4 ? hcx() : hf16; }
    // damped directions whose memory variables plane z needs
    __device__ __forceinline__ unsigned dirs(int z, int nz) const {
        return tdirs | ((z >= 0 && z < nz && (z < W || z >= nz - W)) ? 4u : 0u);
    }
};

// C-PML psi buffer, entry b = (k - z0) & 1 for output plane k.  The first
// two output planes are fetched up front; after plane k has been consumed by
// every thread its entry is refilled with plane k + 2 (one thread issues the
// copies).  psi_pend (bit b): a fill of entry b is in flight (tracked by the
// issuing thread, for the failure exit); psi_par (bit b): the phase the next
// wait on entry b expects (toggled by every thread at each consumed fill).
template <int BND, typename T>
__device__ __forceinline__ void psi_prologue(const Maps& maps, const Geo<BND, T>& G, float* psib,
                                             uint64_t* bars, int nz, int t0, unsigned& psi_pend) {
    const int z1 = G.z0 + G.P4 - 4;
    if (threadIdx.x == 0 && threadIdx.y == 0)
        for (int b = 0; b < NPSI; ++b) {
            const int kq = G.z0 + b;
            const unsigned dn = kq < z1 ? G.dirs(kq, nz) : 0u;
            if (dn) {
                issue_psi(maps, psib + b * 9 * CORE, &bars[NSLOT + b], G.x0, G.y0, kq, dn, t0);
                psi_pend |= 1u << b;
            }
        }
}
template <int BND, typename T>
__device__ __forceinline__ void psi_refill(const Maps& maps, const Geo<BND, T>& G, float* psib,
                                           uint64_t* bars, int b, int k, unsigned kd, int nz, int t0,
                                           unsigned& psi_pend, unsigned& psi_par) {
    if (kd) {
        psi_pend &= ~(1u << b);
        psi_par ^= 1u << b;
    }
    const int kn = k + 2;
    if (k >= G.z0 && kn < G.z0 + G.P4 - 4 && threadIdx.x == 0 && threadIdx.y == 0) {
        const unsigned dn = G.dirs(kn, nz);
        if (dn) {
            issue_psi(maps, psib + b * 9 * CORE, &bars[NSLOT + b], G.x0, G.y0, kn, dn, t0);
            psi_pend |= 1u << b;
        }
    }
}

// Accumulator buffer of the reverse velocity pass (entry b for output plane
// k): the 8 accumulators of plane k and, when the buoyancy term is due,
// v^{m+3/2} (history slot hslot + 1) there.  Same bookkeeping as the psi
// buffer (every output plane has a fill).
template <int BND, typename T>
__device__ __forceinline__ void aux_issue(const Maps& maps, const Geo<BND, T>& G, float* auxb,
                                          uint64_t* bars, int b, int kq, const VelExtra& X,
                                          unsigned& pend) {
    float* buf = auxb + b * AUX_TILES * CORE;
    const bool vn = X.vnext != nullptr;
    mbar_expect_tx(&bars[NSLOT + b], (uint32_t)((vn ? AUX_TILES : 8) * CORE * 4));
    tma_load_4d(buf, &maps.acc, &bars[NSLOT + b], G.x0, G.y0, kq, 0);
    if (vn) tma_load_4d(buf + 8 * CORE, &maps.hcore, &bars[NSLOT + b], G.x0, G.y0, kq, 3 * (X.hslot + 1));
    pend |= 1u << b;
}
template <int BND, typename T>
__device__ __forceinline__ void aux_prologue(const Maps& maps, const Geo<BND, T>& G, float* auxb,
                                             uint64_t* bars, const VelExtra& X, unsigned& pend) {
    if (threadIdx.x == 0 && threadIdx.y == 0)
        for (int b = 0; b < NPSI; ++b)
            if (G.z0 + b < G.z0 + G.P4 - 4) aux_issue(maps, G, auxb, bars, b, G.z0 + b, X, pend);
}
template <int BND, typename T>
__device__ __forceinline__ void aux_refill(const Maps& maps, const Geo<BND, T>& G, float* auxb,
                                           uint64_t* bars, int b, int k, const VelExtra& X,
                                           unsigned& pend, unsigned& par) {
    if (k < G.z0) return;
    pend &= ~(1u << b);
    par ^= 1u << b;
    if (k + 2 < G.z0 + G.P4 - 4 && threadIdx.x == 0 && threadIdx.y == 0)
        aux_issue(maps, G, auxb, bars, b, k + 2, X, pend);
}

// psi = b psi + a d; d += psi for the three terms of one damped direction.
__device__ __forceinline__ void pml_upd(float& p0, float& p1, float& p2, float a, float b,
                                        float& d0, float& d1, float& d2) {
    p0 = b * p0 + a * d0; d0 += p0;
    p1 = b * p1 + a * d1; d1 += p1;
    p2 = b * p2 + a * d2; d2 += p2;
}

// Field tile element as FP32.
template <typename T>
__device__ __forceinline__ float F(const T* p, int o) { return St<T>::ld(p + o); }
template <typename T> constexpr bool kScaled = sizeof(T) == 2;            // 16-bit storage
template <typename T> constexpr bool kHalf = std::is_same<T, __half>::value;
// a stored value beyond the FP16 range (it would round to infinity)
__device__ __forceinline__ bool over(float x) { return fabsf(x) > 65504.0f; }

// ------------------------------------------------------------------------------
// Velocity pass (Eq. 1 + Eq. 4).
// ------------------------------------------------------------------------------
// the four core tiles of a velocity-pass slot (physical slots 5..8)
enum { VC_SZZ, VC_VX, VC_VY, VC_VZ };
static_assert(fslot(SZZ) == 5 && fslot(VX) == 6 && fslot(VY) == 7 &&
                  fslot(VZ) == 8 && fslot(SXZ) == fslot(SXX) + 1 &&
                  fslot(SYZ) == fslot(SYY) + 1,
              "the copies of the velocity pass follow the physical field order");

// Coarse medium grid: bilinear samples of the medium grid (at the thread's
// x-y positions) on the two medium planes around the current output plane,
// for the quantities sampled at integer z (zi) and at half-integer z (zh);
// refreshed when the output plane crosses a medium plane, so each plane
// costs one z-interpolation per quantity.
template <int NQ>
struct CoarseZ {
    float lo[ROWS][NQ], hi[ROWS][NQ];
    int lvl;
};
// Bilinear sample of medium array q on medium plane lvl.
__device__ __forceinline__ float coarse_bilin(const DevGrid& g, int q, Ax x, Ax y, int lvl) {
    const int ox = g.mx > 1 ? 1 : 0, oy = g.my > 1 ? g.mx : 0;
    const float* p = g.cm[q] + ((long long)lvl * g.my + y.i0) * g.mx + x.i0;
    return lerp1(lerp1(__ldg(p), __ldg(p + ox), x.f), lerp1(__ldg(p + oy), __ldg(p + oy + ox), x.f),
                 y.f);
}

struct VelQ {
    float zz[ROWS][4], xz[ROWS][4], yz[ROWS][4];   // sigma_zz k-1..k+2, sigma_xz/yz k-2..k+1
    float hx[ROWS][4], hy[ROWS][4], hz[ROWS][4];   // M_GRAD history: vx/vy k-1..k+2, vz k-2..k+1
    CoarseZ<2> ci;    // rho at (i+1/2, j), (i, j+1/2), integer z
    CoarseZ<1> ch;    // rho at (i, j), half-integer z
};

// One arrival of the z-loop, ring position PH = m mod 4.  Returns false if
// the CTA must stop (a wait gave up).
// RS: slot stride of the ring (0: the pass's own slot size).
template <int BND, typename T, int MODE, int PH, int FS, int RS>
__device__ __forceinline__ bool vel_step(const Maps& maps, const PassParams& P,
                                         const Geo<BND, T>& G, VelQ& Q, unsigned char* sm,
                                         uint64_t* bars, int m, unsigned& psi_pend,
                                         unsigned& psi_par, bool& ovf) {
    float* psib = psi_base(sm);
    using L = Lay<T>;
    constexpr int HX = L::HX;
    constexpr int SB = RS ? RS : vslot_bytes<T, MODE>();
    constexpr int PB = PH & 1;                                     // psi entry of plane k
    const DevGrid& g = P.g;
    constexpr int S0 = PH, S1 = (PH + 3) & 3, S2 = (PH + 2) & 3;   // planes p, p-1, p-2
    const int k = G.z0 - 4 + m;                                    // output plane
    const bool out = m >= 4;
    // per-plane boundary coefficients of the output plane, fetched before the wait
    const bool sz = BND == BND_CPML && out && in_slab(k, g.nz, G.W);
    const float paz = sz ? __ldg(P.B.pa[2] + k) : 0.f, pbz = sz ? __ldg(P.B.pb[2] + k) : 0.f;
    const float G3 = (BND == BND_SPONGE && out) ? G.gx * __ldg(P.B.g[2] + k) : 1.0f;
    const unsigned kd = (BND == BND_CPML && out) ? G.dirs(k, g.nz) : 0u;   // damped dirs of k
    bool ok = mbar_wait(&bars[S0], (uint32_t)((m >> 2) & 1));
    if (BND == BND_CPML && kd) ok = mbar_wait(&bars[NSLOT + PB], (psi_par >> PB) & 1u) && ok;
    // M_GRAD: gradient accumulators and v^{m+3/2} of the output cells, from
    // the accumulator buffer (fetched two planes ahead)
    float ga[ROWS][8], gv[ROWS][3];
    if constexpr (MODE == M_GRAD) {
        if (out) ok = mbar_wait(&bars[NSLOT + PB], (psi_par >> PB) & 1u) && ok;
        const float* ax = aux_base(sm) + PB * AUX_TILES * CORE + G.cc;
#pragma unroll
        for (int rr = 0; rr < ROWS; ++rr) {
#pragma unroll
            for (int q = 0; q < 8; ++q) ga[rr][q] = ax[q * CORE + rr * TX];
#pragma unroll
            for (int c = 0; c < 3; ++c) gv[rr][c] = P.X.vnext ? ax[(8 + c) * CORE + rr * TX] : 0.f;
        }
    }
    const unsigned char* sl0 = sm + S0 * SB;
    const unsigned char* sl1 = sm + S1 * SB;
    const unsigned char* sl2 = sm + S2 * SB;
    // push own-column values: sigma_zz of plane p, sigma_xz / sigma_yz of p - 1
#pragma unroll
    for (int rr = 0; rr < ROWS; ++rr) {
        Q.zz[rr][PH] = F((const T*)(sl0 + L::V_CORE + VC_SZZ * L::CB), G.cc + rr * TX);
        if (m > 0) {
            Q.xz[rr][PH] = F((const T*)(sl1 + L::V_SXZ), G.hcx() + rr * HX);
            Q.yz[rr][PH] = F((const T*)(sl1 + L::V_SYZ), G.hcy() + rr * TX);
        }
        if constexpr (MODE == M_GRAD) {   // history: vx, vy of plane p; vz of plane p - 1
            Q.hx[rr][PH] = F((const T*)(sl0 + L::V_BYTES + 0 * L::HBF), G.hc + rr * HX);
            Q.hy[rr][PH] = F((const T*)(sl0 + L::V_BYTES + 1 * L::HBF), G.hc + rr * HX);
            if (m > 0) Q.hz[rr][PH] = F((const T*)(sl1 + L::V_BYTES + 2 * L::HBF), G.hc + rr * HX);
        }
    }
    if (out && ok) {
        constexpr int A = (PH + 1) & 3, B = (PH + 2) & 3, C = (PH + 3) & 3, D = PH;  // oldest..newest
        const T* hxx = (const T*)(sl2 + L::V_SXX) + G.hcx();     // plane k, own cell (x halo)
        const T* hyy = (const T*)(sl2 + L::V_SYY) + G.hcy();     // (y halo)
        const T* hxy = (const T*)(sl2 + L::V_SXY) + G.hc;      // (x and y halo)
        const T* hxz = (const T*)(sl2 + L::V_SXZ) + G.hcx();
        const T* hyz = (const T*)(sl2 + L::V_SYZ) + G.hcy();
        const float* hr = (const float*)(sl2 + L::V_RHO) + G.hf();
        const float* hr1 = (const float*)(sl1 + L::V_RHO) + G.hf();   // plane k + 1
        const T* vc = (const T*)(sl2 + L::V_CORE) + G.cc;
        const bool ktop = k + 1 < g.nz;
        constexpr int ZF = FS & 3;                         // z-difference form
        const ZW zw = zweights<ZF == ZS_NONE ? ZS_NONE : ZS_FWD>(g, k);   // surface forms only
        const ZT zt = ZF == ZS_ADJ ? ztransposed(g, k) : ZT{};
        const long long o = (long long)k * g.plane + G.obase;
#pragma unroll
        for (int rr = 0; rr < ROWS; ++rr) {
            if (!G.own[rr]) continue;
            const int R = rr * HX, RY = rr * TX, RF = rr * HXF;
            const float* qxz = Q.xz[rr];
            const float* qyz = Q.yz[rr];
            const float* qzz = Q.zz[rr];
            // vx at (i+1/2, j, k)
            float dxx = g.c1x * (F(hxx, R + 1) - F(hxx, R)) + g.c2x * (F(hxx, R + 2) - F(hxx, R - 1));
            float dxy = g.c1y * (F(hxy, R) - F(hxy, R - HX)) + g.c2y * (F(hxy, R + HX) - F(hxy, R - 2 * HX));
            float dxz = zdiff<ZF, false>(g, zw, zt, qxz[A], qxz[B], qxz[C], qxz[D]);
            // vy at (i, j+1/2, k)
            float dyx = g.c1x * (F(hxy, R) - F(hxy, R - 1)) + g.c2x * (F(hxy, R + 1) - F(hxy, R - 2));
            float dyy = g.c1y * (F(hyy, RY + TX) - F(hyy, RY)) + g.c2y * (F(hyy, RY + 2 * TX) - F(hyy, RY - TX));
            float dyz = zdiff<ZF, false>(g, zw, zt, qyz[A], qyz[B], qyz[C], qyz[D]);
            // vz at (i, j, k+1/2)
            float dzx = g.c1x * (F(hxz, R) - F(hxz, R - 1)) + g.c2x * (F(hxz, R + 1) - F(hxz, R - 2));
            float dzy = g.c1y * (F(hyz, RY) - F(hyz, RY - TX)) + g.c2y * (F(hyz, RY + TX) - F(hyz, RY - 2 * TX));
            float dzz = zdiff<ZF, true>(g, zw, zt, qzz[A], qzz[B], qzz[C], qzz[D]);
            if constexpr (kScaled<T>) {     // stored -> physical units
                dxx *= P.inv[SXX]; dxy *= P.inv[SXY]; dxz *= P.inv[SXZ];
                dyx *= P.inv[SXY]; dyy *= P.inv[SYY]; dyz *= P.inv[SYZ];
                dzx *= P.inv[SXZ]; dzy *= P.inv[SYZ]; dzz *= P.inv[SZZ];
            }
            if (BND == BND_CPML) {
                // memory variables of plane k from the psi buffer, updated, stored
                const float* ps = psib + PB * 9 * CORE + G.cc + rr * TX;
                const long long oo = o + rr * g.pitch;
                if (G.sx) {
                    float p0 = ps[0 * CORE], p1 = ps[1 * CORE], p2 = ps[2 * CORE];
                    pml_upd(p0, p1, p2, G.pax, G.pbx, dxx, dyx, dzx);
                    P.B.psi[0][oo] = p0; P.B.psi[1][oo] = p1; P.B.psi[2][oo] = p2;
                }
                if (G.sy[rr]) {
                    float p0 = ps[3 * CORE], p1 = ps[4 * CORE], p2 = ps[5 * CORE];
                    pml_upd(p0, p1, p2, G.pay[rr], G.pby[rr], dxy, dyy, dzy);
                    P.B.psi[6][oo] = p0; P.B.psi[7][oo] = p1; P.B.psi[8][oo] = p2;
                }
                if (sz) {
                    float p0 = ps[6 * CORE], p1 = ps[7 * CORE], p2 = ps[8 * CORE];
                    pml_upd(p0, p1, p2, paz, pbz, dxz, dyz, dzz);
                    P.B.psi[12][oo] = p0; P.B.psi[13][oo] = p1; P.B.psi[14][oo] = p2;
                }
            }
            // buoyancy at the v points: 1 / mean of the two adjacent densities
            if constexpr (MODE == M_GRAD) {
                // Gradient products of this reverse step m (stress points of
                // the cell; the medium enters at the end): strain rates E of
                // the forward v^{m+1/2} (Eq. 2/3 operators) against u, the
                // adjoint stress variable before this pass.
                const T* vhx = (const T*)(sl2 + L::V_BYTES + 0 * L::HBF) + G.hc;
                const T* vhy = (const T*)(sl2 + L::V_BYTES + 1 * L::HBF) + G.hc;
                const T* vhz = (const T*)(sl2 + L::V_BYTES + 2 * L::HBF) + G.hc;
                const float* qhx = Q.hx[rr];
                const float* qhy = Q.hy[rr];
                const float* qhz = Q.hz[rr];
                const float exx = g.c1x * (F(vhx, R) - F(vhx, R - 1)) + g.c2x * (F(vhx, R + 1) - F(vhx, R - 2));
                const float eyy = g.c1y * (F(vhy, R) - F(vhy, R - HX)) + g.c2y * (F(vhy, R + HX) - F(vhy, R - 2 * HX));
                constexpr int FW = ZF == ZS_NONE ? ZS_NONE : ZS_FWD;   // forward strain rates
                const float ezz = zdiff<FW, false>(g, zw, zt, qhz[A], qhz[B], qhz[C], qhz[D]);
                const float gxy = g.c1y * (F(vhx, R + HX) - F(vhx, R)) + g.c2y * (F(vhx, R + 2 * HX) - F(vhx, R - HX)) +
                                  g.c1x * (F(vhy, R + 1) - F(vhy, R)) + g.c2x * (F(vhy, R + 2) - F(vhy, R - 1));
                const float gxz = zdiff<FW, true>(g, zw, zt, qhx[A], qhx[B], qhx[C], qhx[D]) +
                                  g.c1x * (F(vhz, R + 1) - F(vhz, R)) + g.c2x * (F(vhz, R + 2) - F(vhz, R - 1));
                const float gyz = zdiff<FW, true>(g, zw, zt, qhy[A], qhy[B], qhy[C], qhy[D]) +
                                  g.c1y * (F(vhz, R + HX) - F(vhz, R)) + g.c2y * (F(vhz, R + 2 * HX) - F(vhz, R - HX));
                const float uxx = F(hxx, R), uyy = F(hyy, RY), uzz = F(vc, VC_SZZ * CORE + rr * TX);
                const float gdt = P.X.gdt;
                const long long oo = o + rr * g.pitch;
                P.X.acc[0][oo] = ga[rr][0] + gdt * (exx + eyy + ezz) * (uxx + uyy + uzz);
                P.X.acc[1][oo] = ga[rr][1] + gdt * (exx * uxx + eyy * uyy + ezz * uzz);
                P.X.acc[2][oo] = ga[rr][2] + gdt * gxy * F(hxy, R);
                P.X.acc[3][oo] = ga[rr][3] + gdt * gxz * F(hxz, R);
                P.X.acc[4][oo] = ga[rr][4] + gdt * gyz * F(hyz, RY);
                if (P.X.vnext) {
                    // buoyancy term of step m + 1: (v^{m+3/2} / G - v^{m+1/2}) times
                    // the adjoint velocity variable before this pass
                    const float Gs = (BND == BND_SPONGE) ? G3 * G.gy[rr] : 1.0f;
                    const float iG = 1.0f / Gs;
                    P.X.acc[5][oo] = ga[rr][5] + (gv[rr][0] * iG - F(vhx, R)) * F(vc, VC_VX * CORE + rr * TX);
                    P.X.acc[6][oo] = ga[rr][6] + (gv[rr][1] * iG - F(vhy, R)) * F(vc, VC_VY * CORE + rr * TX);
                    P.X.acc[7][oo] = ga[rr][7] + (gv[rr][2] * iG - F(vhz, R)) * F(vc, VC_VZ * CORE + rr * TX);
                }
            }
            float bx, by, bz;
            if constexpr ((FS & VAR_COARSE) != 0) {
                // coarse medium: 1 / rho sampled at each v point
                const Ax zk = axis_at((float)k, g.rz, g.mz), zh = axis_at(k + 0.5f, g.rz, g.mz);
                const int up = g.mz > 1 ? 1 : 0;
                if (zk.i0 != Q.ci.lvl || zh.i0 != Q.ch.lvl) {   // uniform across the CTA
                    const float fi = (float)G.i, fj = (float)(G.j0 + rr);
                    const Ax xi = axis_at(fi, g.rx, g.mx), xh = axis_at(fi + 0.5f, g.rx, g.mx);
                    const Ax yj = axis_at(fj, g.ry, g.my), yh = axis_at(fj + 0.5f, g.ry, g.my);
                    Q.ci.lo[rr][0] = coarse_bilin(g, 2, xh, yj, zk.i0);
                    Q.ci.hi[rr][0] = coarse_bilin(g, 2, xh, yj, zk.i0 + up);
                    Q.ci.lo[rr][1] = coarse_bilin(g, 2, xi, yh, zk.i0);
                    Q.ci.hi[rr][1] = coarse_bilin(g, 2, xi, yh, zk.i0 + up);
                    Q.ch.lo[rr][0] = coarse_bilin(g, 2, xi, yj, zh.i0);
                    Q.ch.hi[rr][0] = coarse_bilin(g, 2, xi, yj, zh.i0 + up);
                    if (rr == ROWS - 1) {
                        Q.ci.lvl = zk.i0;
                        Q.ch.lvl = zh.i0;
                    }
                }
                bx = __fdividef(1.0f, lerp1(Q.ci.lo[rr][0], Q.ci.hi[rr][0], zk.f));
                by = __fdividef(1.0f, lerp1(Q.ci.lo[rr][1], Q.ci.hi[rr][1], zk.f));
                bz = __fdividef(1.0f, lerp1(Q.ch.lo[rr][0], Q.ch.hi[rr][0], zh.f));
            } else {
                const float r0 = hr[RF];
                bx = __fdividef(2.0f, r0 + hr[RF + G.cx]);
                by = __fdividef(2.0f, r0 + hr[RF + G.cy[rr]]);
                bz = __fdividef(2.0f, r0 + (ktop ? hr1[RF] : r0));
            }
            float vx = F(vc, VC_VX * CORE + rr * TX) + P.dto[VX] * bx * (dxx + dxy + dxz);
            float vy = F(vc, VC_VY * CORE + rr * TX) + P.dto[VY] * by * (dyx + dyy + dyz);
            float vz = F(vc, VC_VZ * CORE + rr * TX) + P.dto[VZ] * bz * (dzx + dzy + dzz);
            if (BND == BND_SPONGE) {
                const float Gs = G3 * G.gy[rr];
                vx *= Gs; vy *= Gs; vz *= Gs;
            }
            if constexpr (kHalf<T>) ovf |= over(vx) | over(vy) | over(vz);
            const long long oo = o + rr * g.pitch;
            ((T*)P.F.f[VX])[oo] = St<T>::put(vx);
            ((T*)P.F.f[VY])[oo] = St<T>::put(vy);
            ((T*)P.F.f[VZ])[oo] = St<T>::put(vz);
            if constexpr (MODE == M_CAP) {   // v^{n+1/2} into its history slot
                P.X.vcap[oo] = vx;
                P.X.vcap[P.X.fstride + oo] = vy;
                P.X.vcap[2 * P.X.fstride + oo] = vz;
            }
        }
    }
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0 && threadIdx.y == 0)
            fail_exit(P.err, 1, bars, m, min(G.P4, max(NSLOT, m + 2)), psi_pend, psi_par);
        return false;
    }
    if (BND == BND_CPML) psi_refill(maps, G, psib, bars, PB, k, kd, g.nz, 0, psi_pend, psi_par);
    if constexpr (MODE == M_GRAD) aux_refill(maps, G, aux_base(sm), bars, PB, k, P.X, psi_pend, psi_par);
    // plane k's slot (S2) is free: refill it with plane z0 - 2 + (m + 2)
    if (m >= 2 && m + 2 < G.P4 && threadIdx.x == 0 && threadIdx.y == 0)
        issue_vel<T, MODE, (FS & VAR_COARSE) != 0>(maps, sm + S2 * SB, &bars[S2], G.x0, G.y0, G.z0 + m, P.X.hslot);
    return true;
}

// One (tile, z-chunk) of the velocity pass; the ring barriers must be freshly
// initialised.  Returns false if a wait gave up (the error is recorded).
template <int BND, typename T, int MODE, int FS = ZS_NONE, int RS = 0>
__device__ __forceinline__ bool vel_tile(const Maps& maps, const PassParams& P, int item,
                                         unsigned char* sm, uint64_t* bars) {
    constexpr int SB = RS ? RS : vslot_bytes<T, MODE>();
    const Geo<BND, T> G(P, item);
    if (threadIdx.x == 0 && threadIdx.y == 0)
        for (int s = 0; s < NSLOT && s < G.P4; ++s)
            issue_vel<T, MODE, (FS & VAR_COARSE) != 0>(maps, sm + s * SB, &bars[s], G.x0, G.y0, G.z0 - 2 + s, P.X.hslot);
    unsigned psi_pend = 0, psi_par = 0;            // psi-buffer entries in flight / phases
    if (BND == BND_CPML) psi_prologue(maps, G, psi_base(sm), bars, P.g.nz, 0, psi_pend);
    if constexpr (MODE == M_GRAD) aux_prologue(maps, G, aux_base(sm), bars, P.X, psi_pend);
    VelQ Q;
#pragma unroll
    for (int rr = 0; rr < ROWS; ++rr)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            Q.zz[rr][q] = 0.f; Q.xz[rr][q] = 0.f; Q.yz[rr][q] = 0.f;
            Q.hx[rr][q] = 0.f; Q.hy[rr][q] = 0.f; Q.hz[rr][q] = 0.f;
    Q.ci.lvl = -1;
    Q.ch.lvl = -1;
        }
    bool ovf = false;                              // an FP16 value out of range
    for (int m = 0; m < G.P4; m += 4) {
        if (!vel_step<BND, T, MODE, 0, FS, RS>(maps, P, G, Q, sm, bars, m, psi_pend, psi_par, ovf)) return false;
        if (m + 1 < G.P4 && !vel_step<BND, T, MODE, 1, FS, RS>(maps, P, G, Q, sm, bars, m + 1, psi_pend, psi_par, ovf)) return false;
        if (m + 2 < G.P4 && !vel_step<BND, T, MODE, 2, FS, RS>(maps, P, G, Q, sm, bars, m + 2, psi_pend, psi_par, ovf)) return false;
        if (m + 3 < G.P4 && !vel_step<BND, T, MODE, 3, FS, RS>(maps, P, G, Q, sm, bars, m + 3, psi_pend, psi_par, ovf)) return false;
    }
    if constexpr (kHalf<T>)
        if (__syncthreads_or(ovf) && threadIdx.x == 0 && threadIdx.y == 0) atomicOr(P.err, 4);
    return true;
}

// CTAs per SM of a pass form.  The coarse-medium forms keep their medium
// samples in registers (at most 3 CTAs per SM, 85 registers a thread); the
// reverse form with its fused gradient products needs about 100 (2 per SM).
// The plain FP32 velocity pass without C-PML fits 64 registers without
// spilling and runs 4 CTAs per SM where its shared memory allows (at 256^3
// with a sponge: 143 instead of 154 us).
template <int BND, typename T, int MODE, int FS>
constexpr int var_blocks() {
    return MODE == M_GRAD ? 2
           : (FS & VAR_COARSE) && blocks_for<T>(smem_v<BND, T, MODE>()) > 3
               ? 3
           : (BND != BND_CPML && sizeof(T) == 4 && FS == ZS_NONE &&
              (227 * 1024) / (int)(smem_v<BND, T, MODE>() + 1024) >= 4)
               ? 4
               : blocks_for<T>(smem_v<BND, T, MODE>());
}
template <int BND, typename T, int FS>
constexpr int str_blocks() {
    return (FS & VAR_COARSE) && blocks_for<T>(smem_s<BND, T>()) > 3 ? 3
                                                                     : blocks_for<T>(smem_s<BND, T>());
}

template <int BND, typename T, int MODE, int FS = ZS_NONE>
__global__ void __launch_bounds__(NTH, (var_blocks<BND, T, MODE, FS>())) k_velocity(
    const __grid_constant__ Maps maps, const PassParams P) {
    extern __shared__ __align__(128) unsigned char sm[];
    constexpr int SB = vslot_bytes<T, MODE>();
    unsigned char* ring = sm + pre_bytes<BND, MODE == M_GRAD>();
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + NSLOT * SB);
    ring_init(bars, threadIdx.y * TX + threadIdx.x);
    vel_tile<BND, T, MODE, FS>(maps, P, (int)blockIdx.x, ring, bars);
}

// ------------------------------------------------------------------------------
// Stress pass (Eq. 2/3 + Eq. 4).
// ------------------------------------------------------------------------------
enum { SH_VX, SH_VY, SH_VZ };
// the six stress core tiles of a stress-pass slot, in physical slot order
enum {
    SC_SXX = fslot(SXX), SC_SYY = fslot(SYY), SC_SZZ = fslot(SZZ),
    SC_SXY = fslot(SXY), SC_SXZ = fslot(SXZ), SC_SYZ = fslot(SYZ)
};

struct StrQ {
    float vx[ROWS][4], vy[ROWS][4], vz[ROWS][4];   // vx/vy k-1..k+2, vz k-2..k+1
    CoarseZ<3> ci;    // lambda, mu at (i, j); mu at (i+1/2, j+1/2); integer z
    CoarseZ<2> ch;    // mu at (i+1/2, j), (i, j+1/2); half-integer z
};

template <int BND, typename T, int PH, int FS, int RS>
__device__ __forceinline__ bool str_step(const Maps& maps, const PassParams& P,
                                         const Geo<BND, T>& G, StrQ& Q, unsigned char* sm,
                                         uint64_t* bars, int m, unsigned& psi_pend,
                                         unsigned& psi_par, bool& ovf) {
    float* psib = psi_base(sm);
    using L = Lay<T>;
    constexpr int HX = L::HX;
    constexpr int SB = RS ? RS : L::SSLOT;
    constexpr int HS = L::HB;                                      // halo tile stride
    constexpr int PB = PH & 1;                                     // psi entry of plane k
    const DevGrid& g = P.g;
    constexpr int S0 = PH, S1 = (PH + 3) & 3, S2 = (PH + 2) & 3;   // planes p, p-1, p-2
    const int k = G.z0 - 4 + m;
    const bool out = m >= 4;
    const bool sz = BND == BND_CPML && out && in_slab(k, g.nz, G.W);
    const float paz = sz ? __ldg(P.B.pa[2] + k) : 0.f, pbz = sz ? __ldg(P.B.pb[2] + k) : 0.f;
    const float G3 = (BND == BND_SPONGE && out) ? G.gx * __ldg(P.B.g[2] + k) : 1.0f;
    const unsigned kd = (BND == BND_CPML && out) ? G.dirs(k, g.nz) : 0u;
    bool ok = mbar_wait(&bars[S0], (uint32_t)((m >> 2) & 1));
    if (BND == BND_CPML && kd) ok = mbar_wait(&bars[NSLOT + PB], (psi_par >> PB) & 1u) && ok;
    const unsigned char* sl0 = sm + S0 * SB;
    const unsigned char* sl1 = sm + S1 * SB;
    const unsigned char* sl2 = sm + S2 * SB;
    // push own-column values: vx, vy of plane p, vz of plane p - 1
#pragma unroll
    for (int rr = 0; rr < ROWS; ++rr) {
        Q.vx[rr][PH] = F((const T*)(sl0 + SH_VX * HS), G.hc + rr * HX);
        Q.vy[rr][PH] = F((const T*)(sl0 + SH_VY * HS), G.hc + rr * HX);
        if (m > 0) Q.vz[rr][PH] = F((const T*)(sl1 + SH_VZ * HS), G.hc + rr * HX);
    }
    if (out && ok) {
        constexpr int A = (PH + 1) & 3, B = (PH + 2) & 3, C = (PH + 3) & 3, D = PH;
        const T* hvx = (const T*)(sl2 + SH_VX * HS) + G.hc;       // plane k, own cell
        const T* hvy = (const T*)(sl2 + SH_VY * HS) + G.hc;
        const T* hvz = (const T*)(sl2 + SH_VZ * HS) + G.hc;
        const float* hmu = (const float*)(sl2 + L::S_MU) + G.hf();
        const float* hmu1 = (const float*)((k + 1 < g.nz ? sl1 : sl2) + L::S_MU) + G.hf();   // k + 1
        const float* lc = (const float*)(sl2 + L::S_LAM) + G.cc;
        const T* cr = (const T*)(sl2 + L::S_CORE) + G.cc;
        const long long o = (long long)k * g.plane + G.obase;
        constexpr int ZF = FS & 3;                         // z-difference form
        const ZW zw = zweights<ZF == ZS_NONE ? ZS_NONE : ZS_FWD>(g, k);   // surface forms only
        const ZT zt = ZF == ZS_ADJ ? ztransposed(g, k) : ZT{};
#pragma unroll
        for (int rr = 0; rr < ROWS; ++rr) {
            if (!G.own[rr]) continue;
            const int R = rr * HX, RF = rr * HXF;
            const float* qvx = Q.vx[rr];
            const float* qvy = Q.vy[rr];
            const float* qvz = Q.vz[rr];
            // normal strain rates at (i, j, k)
            float exx = g.c1x * (F(hvx, R) - F(hvx, R - 1)) + g.c2x * (F(hvx, R + 1) - F(hvx, R - 2));
            float eyy = g.c1y * (F(hvy, R) - F(hvy, R - HX)) + g.c2y * (F(hvy, R + HX) - F(hvy, R - 2 * HX));
            float ezz = zdiff<ZF, false>(g, zw, zt, qvz[A], qvz[B], qvz[C], qvz[D]);
            // shear terms at the shear points
            float vxy = g.c1y * (F(hvx, R + HX) - F(hvx, R)) + g.c2y * (F(hvx, R + 2 * HX) - F(hvx, R - HX));
            float vyx = g.c1x * (F(hvy, R + 1) - F(hvy, R)) + g.c2x * (F(hvy, R + 2) - F(hvy, R - 1));
            float vxz = zdiff<ZF, true>(g, zw, zt, qvx[A], qvx[B], qvx[C], qvx[D]);
            float vzx = g.c1x * (F(hvz, R + 1) - F(hvz, R)) + g.c2x * (F(hvz, R + 2) - F(hvz, R - 1));
            float vyz = zdiff<ZF, true>(g, zw, zt, qvy[A], qvy[B], qvy[C], qvy[D]);
            float vzy = g.c1y * (F(hvz, R + HX) - F(hvz, R)) + g.c2y * (F(hvz, R + 2 * HX) - F(hvz, R - HX));
            if constexpr (kScaled<T>) {     // stored -> physical units
                exx *= P.inv[VX]; vxy *= P.inv[VX]; vxz *= P.inv[VX];
                eyy *= P.inv[VY]; vyx *= P.inv[VY]; vyz *= P.inv[VY];
                ezz *= P.inv[VZ]; vzx *= P.inv[VZ]; vzy *= P.inv[VZ];
            }
            if (BND == BND_CPML) {
                const float* ps = psib + PB * 9 * CORE + G.cc + rr * TX;
                const long long oo = o + rr * g.pitch;
                if (G.sx) {
                    float p0 = ps[0 * CORE], p1 = ps[1 * CORE], p2 = ps[2 * CORE];
                    pml_upd(p0, p1, p2, G.pax, G.pbx, exx, vyx, vzx);
                    P.B.psi[3][oo] = p0; P.B.psi[4][oo] = p1; P.B.psi[5][oo] = p2;
                }
                if (G.sy[rr]) {
                    float p0 = ps[3 * CORE], p1 = ps[4 * CORE], p2 = ps[5 * CORE];
                    pml_upd(p0, p1, p2, G.pay[rr], G.pby[rr], eyy, vxy, vzy);
                    P.B.psi[9][oo] = p0; P.B.psi[10][oo] = p1; P.B.psi[11][oo] = p2;
                }
                if (sz) {
                    float p0 = ps[6 * CORE], p1 = ps[7 * CORE], p2 = ps[8 * CORE];
                    pml_upd(p0, p1, p2, paz, pbz, ezz, vxz, vyz);
                    P.B.psi[15][oo] = p0; P.B.psi[16][oo] = p1; P.B.psi[17][oo] = p2;
                }
            }
            // medium: lambda, mu at the cell; mu means at the shear points
            float lam, mu0, mxy, mxz, myz;
            if constexpr ((FS & VAR_COARSE) != 0) {
                // coarse medium: lambda, mu at the cell, mu at each shear point
                const Ax zk = axis_at((float)k, g.rz, g.mz), zh = axis_at(k + 0.5f, g.rz, g.mz);
                const int up = g.mz > 1 ? 1 : 0;
                if (zk.i0 != Q.ci.lvl || zh.i0 != Q.ch.lvl) {   // uniform across the CTA
                    const float fi = (float)G.i, fj = (float)(G.j0 + rr);
                    const Ax xi = axis_at(fi, g.rx, g.mx), xh = axis_at(fi + 0.5f, g.rx, g.mx);
                    const Ax yj = axis_at(fj, g.ry, g.my), yh = axis_at(fj + 0.5f, g.ry, g.my);
                    Q.ci.lo[rr][0] = coarse_bilin(g, 0, xi, yj, zk.i0);
                    Q.ci.hi[rr][0] = coarse_bilin(g, 0, xi, yj, zk.i0 + up);
                    Q.ci.lo[rr][1] = coarse_bilin(g, 1, xi, yj, zk.i0);
                    Q.ci.hi[rr][1] = coarse_bilin(g, 1, xi, yj, zk.i0 + up);
                    Q.ci.lo[rr][2] = coarse_bilin(g, 1, xh, yh, zk.i0);
                    Q.ci.hi[rr][2] = coarse_bilin(g, 1, xh, yh, zk.i0 + up);
                    Q.ch.lo[rr][0] = coarse_bilin(g, 1, xh, yj, zh.i0);
                    Q.ch.hi[rr][0] = coarse_bilin(g, 1, xh, yj, zh.i0 + up);
                    Q.ch.lo[rr][1] = coarse_bilin(g, 1, xi, yh, zh.i0);
                    Q.ch.hi[rr][1] = coarse_bilin(g, 1, xi, yh, zh.i0 + up);
                    if (rr == ROWS - 1) {
                        Q.ci.lvl = zk.i0;
                        Q.ch.lvl = zh.i0;
                    }
                }
                lam = lerp1(Q.ci.lo[rr][0], Q.ci.hi[rr][0], zk.f);
                mu0 = lerp1(Q.ci.lo[rr][1], Q.ci.hi[rr][1], zk.f);
                mxy = lerp1(Q.ci.lo[rr][2], Q.ci.hi[rr][2], zk.f);
                mxz = lerp1(Q.ch.lo[rr][0], Q.ch.hi[rr][0], zh.f);
                myz = lerp1(Q.ch.lo[rr][1], Q.ch.hi[rr][1], zh.f);
            } else {
                const int cyr = G.cy[rr];
                lam = lc[rr * TX];
                mu0 = hmu[RF];
                const float mxp = hmu[RF + G.cx], myp = hmu[RF + cyr];
                const float mzp = hmu1[RF];
                mxy = 0.25f * (mu0 + mxp + myp + hmu[RF + G.cx + cyr]);
                mxz = 0.25f * (mu0 + mxp + mzp + hmu1[RF + G.cx]);
                myz = 0.25f * (mu0 + myp + mzp + hmu1[RF + cyr]);
                if constexpr (ZF != ZS_NONE) {
                    // xz / yz shear points on the free-surface plane z = ks - 1/2:
                    // harmonic mean of the 4 cells (vacuum-formulation reading)
                    if (k == g.fs - 1) {
                        mxz = 4.0f / (1.0f / mu0 + 1.0f / mxp + 1.0f / mzp + 1.0f / hmu1[RF + G.cx]);
                        myz = 4.0f / (1.0f / mu0 + 1.0f / myp + 1.0f / mzp + 1.0f / hmu1[RF + cyr]);
                    }
                }
            }
            const float l2m = lam + 2.0f * mu0;
            float s0 = F(cr, SC_SXX * CORE + rr * TX) + P.dto[SXX] * (l2m * exx + lam * (eyy + ezz));
            float s1 = F(cr, SC_SYY * CORE + rr * TX) + P.dto[SYY] * (l2m * eyy + lam * (exx + ezz));
            float s2 = F(cr, SC_SZZ * CORE + rr * TX) + P.dto[SZZ] * (l2m * ezz + lam * (exx + eyy));
            float s3 = F(cr, SC_SXY * CORE + rr * TX) + P.dto[SXY] * mxy * (vxy + vyx);
            float s4 = F(cr, SC_SXZ * CORE + rr * TX) + P.dto[SXZ] * mxz * (vxz + vzx);
            float s5 = F(cr, SC_SYZ * CORE + rr * TX) + P.dto[SYZ] * myz * (vyz + vzy);
            if (BND == BND_SPONGE) {
                const float Gs = G3 * G.gy[rr];
                s0 *= Gs; s1 *= Gs; s2 *= Gs; s3 *= Gs; s4 *= Gs; s5 *= Gs;
            }
            if constexpr (kHalf<T>)
                ovf |= over(s0) | over(s1) | over(s2) | over(s3) | over(s4) | over(s5);
            const long long oo = o + rr * g.pitch;
            ((T*)P.F.f[SXX])[oo] = St<T>::put(s0);
            ((T*)P.F.f[SYY])[oo] = St<T>::put(s1);
            ((T*)P.F.f[SZZ])[oo] = St<T>::put(s2);
            ((T*)P.F.f[SXY])[oo] = St<T>::put(s3);
            ((T*)P.F.f[SXZ])[oo] = St<T>::put(s4);
            ((T*)P.F.f[SYZ])[oo] = St<T>::put(s5);
        }
    }
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0 && threadIdx.y == 0)
            fail_exit(P.err, 2, bars, m, min(G.P4, max(NSLOT, m + 2)), psi_pend, psi_par);
        return false;
    }
    if (BND == BND_CPML) psi_refill(maps, G, psib, bars, PB, k, kd, g.nz, 3, psi_pend, psi_par);
    if (m >= 2 && m + 2 < G.P4 && threadIdx.x == 0 && threadIdx.y == 0)
        issue_str<T, (FS & VAR_COARSE) != 0>(maps, sm + S2 * SB, &bars[S2], G.x0, G.y0, G.z0 + m);
    return true;
}

template <int BND, typename T, int FS = ZS_NONE, int RS = 0>
__device__ __forceinline__ bool str_tile(const Maps& maps, const PassParams& P, int item,
                                         unsigned char* sm, uint64_t* bars) {
    const Geo<BND, T> G(P, item);
    if (threadIdx.x == 0 && threadIdx.y == 0)
        for (int s = 0; s < NSLOT && s < G.P4; ++s)
            issue_str<T, (FS & VAR_COARSE) != 0>(maps, sm + s * (RS ? RS : Lay<T>::SSLOT), &bars[s], G.x0, G.y0, G.z0 - 2 + s);
    unsigned psi_pend = 0, psi_par = 0;            // psi-buffer entries in flight / phases
    if (BND == BND_CPML) psi_prologue(maps, G, psi_base(sm), bars, P.g.nz, 3, psi_pend);
    StrQ Q;
#pragma unroll
    for (int rr = 0; rr < ROWS; ++rr)
#pragma unroll
        for (int q = 0; q < 4; ++q) { Q.vx[rr][q] = 0.f; Q.vy[rr][q] = 0.f; Q.vz[rr][q] = 0.f; }
    Q.ci.lvl = -1;
    Q.ch.lvl = -1;
    bool ovf = false;                              // an FP16 value out of range
    for (int m = 0; m < G.P4; m += 4) {
        if (!str_step<BND, T, 0, FS, RS>(maps, P, G, Q, sm, bars, m, psi_pend, psi_par, ovf)) return false;
        if (m + 1 < G.P4 && !str_step<BND, T, 1, FS, RS>(maps, P, G, Q, sm, bars, m + 1, psi_pend, psi_par, ovf)) return false;
        if (m + 2 < G.P4 && !str_step<BND, T, 2, FS, RS>(maps, P, G, Q, sm, bars, m + 2, psi_pend, psi_par, ovf)) return false;
        if (m + 3 < G.P4 && !str_step<BND, T, 3, FS, RS>(maps, P, G, Q, sm, bars, m + 3, psi_pend, psi_par, ovf)) return false;
    }
    if constexpr (kHalf<T>)
        if (__syncthreads_or(ovf) && threadIdx.x == 0 && threadIdx.y == 0) atomicOr(P.err, 4);
    return true;
}

template <int BND, typename T, int FS = ZS_NONE>
__global__ void __launch_bounds__(NTH, (str_blocks<BND, T, FS>())) k_stress(const __grid_constant__ Maps maps,
                                                                            const PassParams P) {
    extern __shared__ __align__(128) unsigned char sm[];
    unsigned char* ring = sm + pre_bytes<BND, false>();
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + NSLOT * Lay<T>::SSLOT);
    ring_init(bars, threadIdx.y * TX + threadIdx.x);
    str_tile<BND, T, FS>(maps, P, (int)blockIdx.x, ring, bars);
}

#if EWS_FULL
// ------------------------------------------------------------------------------
// Batched executor: one persistent launch over the work items of many shots
// (see BatchShot / BatchEntry).  Each CTA claims an item, waits (bounded) for
// the shot's earlier stages, runs it, and counts it done.
// ------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed_u(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Re-arm the ring for the next item: every copy of the previous item has
// been waited for, so the barriers can be invalidated and initialised again.
__device__ __forceinline__ void ring_rearm(uint64_t* bars, int tid) {
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < NBAR; ++s)
            asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bars[s])) : "memory");
        for (int s = 0; s < NBAR; ++s) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
}

// The executor's tensor maps live in global memory, written by the host
// before the launch: acquire them for the tensor-map proxy before the
// issuing thread's first copy through them.
__device__ __forceinline__ void acquire_maps(const Maps* m) {
    const CUtensorMap* t = reinterpret_cast<const CUtensorMap*>(m);
    for (int k = 0; k < (int)(sizeof(Maps) / sizeof(CUtensorMap)); ++k)
        asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(t + k)
                     : "memory");
}

// Stage the pass parameters of an item in shared memory.
__device__ __forceinline__ void stage_params(PassParams* dst, const PassParams& src, int tid) {
    static_assert(sizeof(PassParams) % 4 == 0, "PassParams is copied as words");
    const int* a = reinterpret_cast<const int*>(&src);
    int* b = reinterpret_cast<int*>(dst);
    for (int w = tid; w < (int)(sizeof(PassParams) / 4); w += NTH) b[w] = a[w];
}

// Cell box of a pass item (the same decomposition as Geo).
struct ItemBox {
    int x0, y0, z0, z1;
    __device__ __forceinline__ ItemBox(const PassParams& P, int item) {
        const int ntile = P.ntx * P.nty;
        const int t = item % ntile;
        z0 = (item / ntile) * P.zchunk;
        z1 = min(P.g.nz, z0 + P.zchunk);
        x0 = (t % P.ntx) * TX;
        y0 = (t / P.ntx) * TY;
    }
    __device__ __forceinline__ bool has(int i, int j, int k) const {
        return i >= x0 && i < x0 + TX && j >= y0 && j < y0 + TY && k >= z0 && k < z1;
    }
};

// Ring slot of the batched executor: large enough for every pass it runs.
template <bool GRAD>
constexpr int batch_slot() {
    constexpr int v = GRAD ? vslot_bytes<float, M_GRAD>() : vslot_bytes<float, M_FWD>();
    return v > Lay<float>::SSLOT ? v : Lay<float>::SSLOT;
}

template <int BND, bool GRAD, bool FS = false>
__global__ void __launch_bounds__(NTH, GRAD ? 2 : 3)
    k_batch(const BatchShot* __restrict__ shots, const BatchEntry* __restrict__ entries,
            int nentries, unsigned* cur, unsigned* taken, unsigned long long* done, int* err,
            unsigned long long wait_ns) {
    extern __shared__ __align__(128) unsigned char sm[];
    // one ring for every item kind: slots as large as the largest pass's
    constexpr int SB = batch_slot<GRAD>();
    unsigned char* ring = sm + pre_bytes<BND, GRAD>();
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + NSLOT * SB);
    __shared__ PassParams sP;
    __shared__ int s_e, s_it, s_stop, s_key;
    __shared__ unsigned long long s_fenced[4];   // map sets acquired, bit per shot < 64
    __shared__ double s_red[NTH / 32];
    const int tid = threadIdx.y * TX + threadIdx.x;
    ring_init(bars, tid);
    if (tid == 0) {
        s_key = -1;
        for (int q = 0; q < 4; ++q) s_fenced[q] = 0;
    }
    while (true) {
        if (tid == 0) {
            int e = -1, it = 0, stop = 0;
            while (true) {               // claim the next item in entry order
                if (ld_relaxed(err)) break;
                const unsigned c = ld_relaxed_u(cur);
                if (c >= (unsigned)nentries) break;
                const unsigned t = atomicAdd(&taken[c], 1u);
                if (t < (unsigned)entries[c].nitems) {
                    e = (int)c;
                    it = (int)t;
                    break;
                }
                atomicCAS(cur, c, c + 1);
            }
            if (e >= 0) {                // wait for the shot's earlier stages (acquire)
                const int shot = entries[e].shot;
                const unsigned long long need = (unsigned long long)entries[e].need;
                const unsigned long long t0 = now_ns();
                while (ld_acquire(&done[shot]) < need) {
                    if (ld_relaxed(err)) { stop = 1; break; }
                    if (now_ns() - t0 > wait_ns) { atomicOr(err, 8); stop = 1; break; }
                    __nanosleep(64);
                }
                // the awaited generic stores are visible to this thread's TMA copies
                asm volatile("fence.proxy.async.global;" ::: "memory");
            }
            s_e = e;
            s_it = it;
            s_stop = stop;
        }
        __syncthreads();
        if (s_e < 0 || s_stop) break;
        const int it = s_it;
        const BatchEntry E = entries[s_e];
        const BatchShot& B = shots[E.shot];
        const DevGrid& g = B.pf.g;
        const long long fs = B.fs;
        bool ok = true;
        switch (E.kind) {
            case BK_VEL:
            case BK_VEL_CAP:
            case BK_VEL_GRAD:
            case BK_STR:
            case BK_STR_ADJ: {
                const bool adj = E.kind == BK_VEL_GRAD || E.kind == BK_STR_ADJ;
                const int key = 2 * E.shot + (adj ? 1 : 0);
                if (s_key != key) {          // stage this shot's pass parameters once
                    stage_params(&sP, adj ? B.pa : B.pf, tid);
                    __syncthreads();
                    if (tid == 0) s_key = key;
                }
                const int set = E.kind == BK_VEL || E.kind == BK_VEL_CAP ? 0
                                : E.kind == BK_STR                     ? 1
                                : E.kind == BK_STR_ADJ                 ? 2
                                                                       : 3;
                if (tid == 0) {
                    if (E.kind == BK_VEL_CAP) {
                        sP.X.vcap = B.vhist + (long long)E.slot * 3 * fs;
                        sP.X.fstride = fs;
                    } else if (E.kind == BK_VEL_GRAD) {
                        sP.X.hslot = E.slot;
                        sP.X.vnext = E.flag ? B.vhist + (long long)(E.slot + 1) * 3 * fs : nullptr;
                    }
                    const Maps* mp = set == 0 ? &B.vf : set == 1 ? &B.sf : set == 2 ? &B.sa : &B.va;
                    if (E.shot >= 64 || !((s_fenced[set] >> E.shot) & 1ull)) {
                        acquire_maps(mp);
                        if (E.shot < 64) s_fenced[set] |= 1ull << E.shot;
                    }
                }
                ring_rearm(bars, tid);
                constexpr int ZF = FS ? ZS_FWD : ZS_NONE, ZA = FS ? ZS_ADJ : ZS_NONE;
                if (E.kind == BK_VEL)
                    ok = vel_tile<BND, float, M_FWD, ZF, SB>(B.vf, sP, it, ring, bars);
                else if (E.kind == BK_VEL_CAP)
                    ok = vel_tile<BND, float, M_CAP, ZF, SB>(B.vf, sP, it, ring, bars);
                else if (E.kind == BK_STR)
                    ok = str_tile<BND, float, ZF, SB>(B.sf, sP, it, ring, bars);
                else if (E.kind == BK_STR_ADJ)
                    ok = str_tile<BND, float, ZA, SB>(B.sa, sP, it, ring, bars);
                else if constexpr (GRAD)
                    ok = vel_tile<BND, float, M_GRAD, ZA, SB>(B.va, sP, it, ring, bars);
                if (!ok) break;
                // Point terms of this step inside the item's cells, after its
                // stores (the next pass starts only when every item is done):
                // the force after the velocity pass (also into the captured
                // history), the moment after the stress pass, the residual
                // after the reverse velocity pass; and, at the stress pass,
                // the receivers whose first tap lies in the item (v^{n+1/2}
                // is final once the stress pass may start).
                __syncthreads();
                const ItemBox box(sP, it);
                if ((E.kind == BK_VEL || E.kind == BK_VEL_CAP) && B.S.kind == 1 && tid < B.S.ntap) {
                    const Tap& q = B.S.tap[tid];
                    if (box.has(q.i, q.j, q.k)) {
                        ops::inject_tap<float>(g, B.pf.F, B.M, B.pf.B, B.S, B.wavelet, E.n, tid, err);
                        if (E.kind == BK_VEL_CAP) {
                            DevFields H = B.pf.F;
                            for (int c = 0; c < 3; ++c)
                                H.f[c] = B.vhist + ((long long)E.slot * 3 + c) * fs;
                            ops::inject_tap<float>(g, H, B.M, B.pf.B, B.S, B.wavelet, E.n, tid, err);
                        }
                    }
                }
                if (E.kind == BK_STR && B.S.kind == 0 && tid < B.S.ntap) {
                    const Tap& q = B.S.tap[tid];
                    if (box.has(q.i, q.j, q.k))
                        ops::inject_tap<float>(g, B.pf.F, B.M, B.pf.B, B.S, B.wavelet, E.n, tid, err);
                }
                if (E.kind == BK_STR && E.flag && B.seis)
                    for (int t = tid; t < 3 * B.nrec; t += NTH) {
                        const Tap& q = B.rtaps[8 * t];
                        if (box.has(q.i, q.j, q.k))
                        {
                            const float v = ops::record_one<float>(g, B.pf.F, B.rtaps, t);
                            if (!isfinite(v)) atomicOr(err, 16);
                            B.seis[(long long)t * B.nt + E.n] = v;
                        }
                    }
                if (E.kind == BK_VEL_GRAD && B.nrec > 0)
                    for (int t = tid; t < 3 * B.nrec; t += NTH) {
                        const float a = B.sadj[(long long)t * B.nt + E.n];
                        for (int m = 0; m < 8; ++m) {
                            const Tap& q = B.rtaps[8 * t + m];
                            if (box.has(q.i, q.j, q.k)) ops::adj_inject_tap(g, B.A, B.M, B.pf.B, q, a);
                        }
                    }
                break;
            }
            case BK_RESID: {
                double acc = 0.0;
                const long long n = 3LL * B.nrec * B.nt;
                for (long long t = tid; t < n; t += NTH) {
                    const float r = B.seis[t] - B.obs[t];
                    B.sadj[t] = B.dt * r;
                    acc += 0.5 * (double)B.dt * (double)r * (double)r;
                }
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if ((tid & 31) == 0) s_red[tid >> 5] = acc;
                __syncthreads();
                if (tid == 0) {
                    double sum = 0.0;
                    for (int w = 0; w < NTH / 32; ++w) sum += s_red[w];
                    *B.misfit = sum;
                }
                break;
            }
            default: {                       // elementwise stages over a cell range
                const long long o0 = (long long)it * kBatchElem;
                const long long o1 = o0 + kBatchElem < fs ? o0 + kBatchElem : fs;
                const DevFields& F = B.pf.F;
                for (long long o = o0 + tid; o < o1; o += NTH) {
                    switch (E.kind) {
                        case BK_SAVE:          // BF16 keeps FP32's range: no scale needed
                            for (int q = 0; q < NFIELD; ++q) {
                                const long long c = ((long long)E.slot * NFIELD + q) * fs + o;
                                if (B.ck16)
                                    reinterpret_cast<__nv_bfloat16*>(B.ckpt)[c] = __float2bfloat16_rn(F.f[q][o]);
                                else
                                    B.ckpt[c] = F.f[q][o];
                            }
                            break;
                        case BK_LOAD:
                            for (int q = 0; q < NFIELD; ++q) {
                                const long long c = ((long long)E.slot * NFIELD + q) * fs + o;
                                F.f[q][o] = B.ck16 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(B.ckpt)[c])
                                                   : B.ckpt[c];
                            }
                            break;
                        case BK_HIST0:
                            for (int q = 0; q < 3; ++q) B.vhist[q * fs + o] = F.f[q][o];
                            break;
                        case BK_ZERO_F:
                            for (int q = 0; q < NFIELD; ++q) F.f[q][o] = 0.0f;
                            if constexpr (BND == BND_CPML)   // C-PML memory variables from rest
                                for (int t = 0; t < 18; ++t) B.pf.B.psi[t][o] = 0.0f;
                            break;
                        case BK_ZERO_A:
                            for (int q = 0; q < 3; ++q) B.A.p[q][o] = 0.0f;
                            for (int q = 0; q < 6; ++q) B.A.q[q][o] = 0.0f;
                            for (int q = 0; q < 8; ++q) {
                                B.A.acc[q][o] = 0.0f;
                                B.A.acc64[q][o] = 0.0;
                            }
                            break;
                        case BK_FLUSH:
                            ops::flush_cell(B.A, o);
                            break;
                        case BK_RHO:
                        case BK_FINAL: {
                            const int k = (int)(o / g.plane);
                            const long long r = o - (long long)k * g.plane;
                            const int j = (int)(r / g.pitch), i = (int)(r - (long long)j * g.pitch);
                            if (i >= g.nx || k >= g.nz) break;
                            if (E.kind == BK_RHO)
                                ops::rho_term_cell(B.A, B.pf.B, B.vhist + 3 * fs, B.vhist, fs, o, i, j, k);
                            else
                                ops::finalize_t_cell(g, B.A, B.M, B.gl, B.gm, B.gr, i, j, k);
                            break;
                        }
                        default:
                            break;
                    }
                }
                break;
            }
        }
        __syncthreads();
        if (!ok) break;                      // a pipeline wait gave up (recorded)
        if (tid == 0) {                      // release: this item's stores, then the count
            __threadfence();
            atomicAdd(&done[E.shot], 1ull);
        }
    }
}
#endif  // EWS_FULL

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

// Tensor map of nt pitched [nz][ny][pitch] arrays lying tstride bytes apart,
// as a 4D tensor [array][nz][ny][pitch], with a box of bw x bh x 1 x bt.
bool encode4(CUtensorMap* map, const DevGrid& g, const void* base, CUtensorMapDataType dt,
             int esize, long long tstride, int nt, int bw, int bh, int bt) {
    auto fn = encoder();
    if (!fn) return false;
    cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)nt};
    cuuint64_t strides[3] = {(cuuint64_t)g.pitch * esize, (cuuint64_t)g.plane * esize,
                             (cuuint64_t)tstride};
    cuuint32_t box[4] = {(cuuint32_t)bw, (cuuint32_t)bh, 1, (cuuint32_t)bt};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(map, dt, 4, const_cast<void*>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, EWS_L2PROMO,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Tensor map of one pitched [nz][ny][pitch] array with a box of bw x bh x 1.
bool encode(CUtensorMap* map, const DevGrid& g, const void* base, CUtensorMapDataType dt,
            int esize, int bw, int bh) {
    auto fn = encoder();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    cuuint64_t strides[2] = {(cuuint64_t)g.pitch * esize, (cuuint64_t)g.plane * esize};
    cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(map, dt, 3, const_cast<void*>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, EWS_L2PROMO,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <typename K>
cudaError_t prepare(K kern, size_t smem, int* blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, NTH, smem);
}

template <int BND, typename T>
cudaError_t occupancy(int* occ) {
    int a = 0, b = 0, c = 0;
    cudaError_t e = prepare(k_velocity<BND, T, M_FWD>, smem_v<BND, T>(), &a);
    if (e == cudaSuccess) e = prepare(k_stress<BND, T>, smem_s<BND, T>(), &b);
#if EWS_FULL
    // free-surface variants: same slots, occupancy taken from the plain ones
    if (e == cudaSuccess) e = prepare(k_velocity<BND, T, M_FWD, ZS_FWD>, smem_v<BND, T>(), &c);
    if (e == cudaSuccess) e = prepare(k_stress<BND, T, ZS_FWD>, smem_s<BND, T>(), &c);
    // coarse-medium variants (the medium tiles' slot space stays unused)
    if (e == cudaSuccess) e = prepare(k_velocity<BND, T, M_FWD, VAR_COARSE>, smem_v<BND, T>(), &c);
    if (e == cudaSuccess) e = prepare(k_stress<BND, T, VAR_COARSE>, smem_s<BND, T>(), &c);
    if constexpr (std::is_same<T, float>::value) {     // history and reverse modes
        if (e == cudaSuccess) e = prepare(k_velocity<BND, T, M_CAP>, smem_v<BND, T, M_CAP>(), &c);
        if (e == cudaSuccess) e = prepare(k_velocity<BND, T, M_CAP, ZS_FWD>, smem_v<BND, T, M_CAP>(), &c);
        if constexpr (BND != BND_CPML) {
            if (e == cudaSuccess)
                e = prepare(k_velocity<BND, T, M_GRAD>, smem_v<BND, T, M_GRAD>(), &c);
            if (e == cudaSuccess)
                e = prepare(k_velocity<BND, T, M_GRAD, ZS_ADJ>, smem_v<BND, T, M_GRAD>(), &c);
            if (e == cudaSuccess) e = prepare(k_stress<BND, T, ZS_ADJ>, smem_s<BND, T>(), &c);
        }
    }
#endif
    (void)c;
    *occ = a < b ? a : b;
    return e;
}

// CTAs per SM of the reverse velocity pass (0 where it does not exist).
template <typename T>
cudaError_t occupancy_grad(int kind, int* occ) {
    *occ = 0;
#if EWS_FULL
    if constexpr (std::is_same<T, float>::value) {
        if (kind == BND_SPONGE)
            return prepare(k_velocity<BND_SPONGE, T, M_GRAD>, smem_v<BND_SPONGE, T, M_GRAD>(), occ);
        if (kind == BND_NONE)
            return prepare(k_velocity<BND_NONE, T, M_GRAD>, smem_v<BND_NONE, T, M_GRAD>(), occ);
    }
#else
    (void)kind;
#endif
    return cudaSuccess;
}

template <typename T>
cudaError_t occupancy_for(int kind, int* occ) {
    switch (kind) {
        case BND_SPONGE: return occupancy<BND_SPONGE, T>(occ);
        case BND_CPML: return occupancy<BND_CPML, T>(occ);
        default: return occupancy<BND_NONE, T>(occ);
    }
}

// Tensor maps of both passes for storage type T (slot order of Lay<T>).
template <typename T>
bool encode_maps(Maps* vm, Maps* smp, const DevGrid& g, const DevFields& F, const DevMedium& M,
                 const DevBoundary& B) {
    constexpr CUtensorMapDataType dt = St<T>::dtype;
    constexpr int es = (int)sizeof(T), HX = Lay<T>::HX;
    const CUtensorMapDataType f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    bool ok = true;
    // The 9 fields lie in one allocation, field q in physical slot
    // fslot(q), slots fsb bytes apart: runs of neighbouring slots are
    // one 4D tensor [slot][nz][ny][pitch].
    static_assert(fslot(SXX) == 0 && fslot(SXZ) == 1, "sxx, sxz in slots 0, 1");
    const char* f0 = (const char*)F.f[SXX];                                    // slot 0
    const long long fsb = (const char*)F.f[SXZ] - (const char*)F.f[SXX];
    for (int q = 0; q < NFIELD; ++q)
        if ((const char*)F.f[q] - f0 != fslot(q) * fsb) return false;
    // velocity: sxx sxz (x halos), syy syz (y halos), sxy (x and y halo),
    // rho medium box, szz vx vy vz (cores)
    ok &= encode4(&vm->halo[0], g, f0, dt, es, fsb, NFIELD, HX, TY, 2);
    ok &= encode4(&vm->halo[1], g, f0, dt, es, fsb, NFIELD, TX, HY, 2);
    ok &= encode(&vm->halo[2], g, F.f[SXY], dt, es, HX, HY);
    ok &= encode4(&vm->core[0], g, f0, dt, es, fsb, NFIELD, TX, TY, 4);
    // stress: vx vy vz (x and y halos); lambda, mu (medium boxes); the six
    // stresses (cores)
    ok &= encode4(&smp->halo[0], g, f0, dt, es, fsb, NFIELD, HX, HY, 3);
    ok &= encode4(&smp->core[0], g, f0, dt, es, fsb, NFIELD, TX, TY, 6);
    // medium (without the wavefield-grid medium, i.e. with a coarse medium
    // grid, these maps are unused): rho and mu boxes, the lambda core
    if (M.lam) {
        ok &= encode(&vm->halo[5], g, M.rho, f32, 4, HXF, TY + 1);
        ok &= encode(&smp->halo[3], g, M.mu, f32, 4, HXF, TY + 1);
        ok &= encode(&smp->halo[4], g, M.lam, f32, 4, TX, TY);
    }
    // C-PML memory variables (FP32, 18 arrays psi[6 d + t], velocity pass t =
    // 0..2, stress 3..5): one copy per damped direction
    if (B.kind == BND_CPML) {
        const long long psb = (const char*)B.psi[1] - (const char*)B.psi[0];
        for (int t = 1; t < 18; ++t)
            if ((const char*)B.psi[t] - (const char*)B.psi[0] != t * psb) return false;
        ok &= encode4(&vm->psi, g, B.psi[0], f32, 4, psb, 18, TX, TY, 3);
        smp->psi = vm->psi;
    }
    return ok;
}

}  // namespace

struct StencilPlan {
    Maps vmaps, smaps;
    bool has_hist = false;
    int kind = 0;
    int storage = EWS_STORAGE_F32;
    int grid = 0;
    int ntx = 0, nty = 0;
    int zchunk = 0;
    // the reverse velocity pass with the gradient products (fewer CTAs per
    // SM) has its own z-chunks
    int grid_grad = 0, zchunk_grad = 0;
};

namespace {

// Planes per z-chunk of a pass over ntile tile columns with `slots` CTAs
// resident at once: the chunk count n (chunks of at least min_planes
// planes) that minimises the modelled pass time, the waves of (tile, chunk)
// CTAs times the planes each CTA marches through, ceil(ntile n / slots) x
// (nz / n + halo) with `halo` the planes a chunk loads beyond its own on
// each side; ties go to more chunks.  Measured against the earlier rule of
// about four waves (GB300, Gcell/s): 192^3 sponge 48.4 vs 44.5, 192^3 C-PML
// 35.4 vs 33.8, 128^3 sponge 50.5 vs 39.4, 1024 x 1024 x 512 BF16 (32 x 16
// tiles) 78.9 vs 75.9, 256^3 C-PML unchanged (7 chunks either way).  Chunks
// of at least 4 planes: small grids, whose few columns leave most SMs idle,
// get more CTAs (64 x 64 x 32 sponge: 11.3 Gcell/s with 4-plane chunks, 9.1
// with at least 8 planes; 64^3 19.9 vs 17.5).
int chunk_planes(long long ntile, long long slots, int nz, int min_planes, int halo) {
    long long best_n = 1, best_cost = -1;
    for (long long n = 1; n <= std::max(1, nz / min_planes); ++n) {
        const long long zc = (nz + n - 1) / n;
        const long long nn = (nz + zc - 1) / zc;               // chunks of zc planes
        const long long cost = ((ntile * nn + slots - 1) / slots) * (zc + halo);
        if (best_cost < 0 || cost <= best_cost) {
            best_cost = cost;
            best_n = n;
        }
    }
    return (int)((nz + best_n - 1) / best_n);
}

cudaError_t plan_build(StencilPlan* p, const DevGrid& g, const DevFields& F, const DevMedium& M,
                       const DevBoundary& B, int storage) {
    p->kind = B.kind;
    p->storage = storage;
    bool ok;
    switch (storage) {
        case EWS_STORAGE_BF16: ok = encode_maps<__nv_bfloat16>(&p->vmaps, &p->smaps, g, F, M, B); break;
        case EWS_STORAGE_F16: ok = encode_maps<__half>(&p->vmaps, &p->smaps, g, F, M, B); break;
        case EWS_STORAGE_F32: ok = encode_maps<float>(&p->vmaps, &p->smaps, g, F, M, B); break;
        default: return cudaErrorInvalidValue;
    }
    if (!ok) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        switch (storage) {
            case EWS_STORAGE_BF16: e = occupancy_for<__nv_bfloat16>(B.kind, &occ); break;
            case EWS_STORAGE_F16: e = occupancy_for<__half>(B.kind, &occ); break;
            default: e = occupancy_for<float>(B.kind, &occ); break;
        }
    }
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    // Launch geometry: every tile column is cut into the same z-chunks and
    // chunk c of all tiles is resident at once, so neighbouring tiles march
    // through z together and the halo planes one CTA loads are still in L2
    // when its neighbours load them.
    p->ntx = (g.nx + TX - 1) / TX;
    p->nty = (g.ny + TY - 1) / TY;
    const long long ntile = (long long)p->ntx * p->nty;
    p->zchunk = chunk_planes(ntile, (long long)sms * occ, g.nz, 4, 2);
    p->grid = (int)(ntile * ((g.nz + p->zchunk - 1) / p->zchunk));
    int occ_grad = 0;
    if (storage == EWS_STORAGE_F32 && (e = occupancy_grad<float>(B.kind, &occ_grad)) != cudaSuccess)
        return e;
    p->zchunk_grad = occ_grad > 0 ? chunk_planes(ntile, (long long)sms * occ_grad, g.nz, 4, 2)
                                  : p->zchunk;
    p->grid_grad = (int)(ntile * ((g.nz + p->zchunk_grad - 1) / p->zchunk_grad));
    return cudaSuccess;
}

PassParams pass_params(const StencilPlan* sp, const DevGrid& g, const DevFields& F,
                       const DevBoundary& B, const float dto[9], const float inv[9], int* err) {
    PassParams P{};
    P.g = g;
    P.F = F;
    P.B = B;
    for (int q = 0; q < NFIELD; ++q) {
        P.dto[q] = dto[q];
        P.inv[q] = inv[q];
    }
    P.ntx = sp->ntx;
    P.nty = sp->nty;
    P.zchunk = sp->zchunk;
    P.err = err;
    return P;
}

template <typename T, int MODE, int FS>
void launch_v_fs(const StencilPlan* sp, const PassParams& P, cudaStream_t st) {
    dim3 blk(TX, RY);
    switch (sp->kind) {
        case BND_SPONGE:
            k_velocity<BND_SPONGE, T, MODE, FS><<<sp->grid, blk, smem_v<BND_SPONGE, T, MODE>(), st>>>(sp->vmaps, P);
            break;
        case BND_CPML:
            if constexpr (MODE != M_GRAD)
                k_velocity<BND_CPML, T, MODE, FS><<<sp->grid, blk, smem_v<BND_CPML, T, MODE>(), st>>>(sp->vmaps, P);
            break;
        default:
            k_velocity<BND_NONE, T, MODE, FS><<<sp->grid, blk, smem_v<BND_NONE, T, MODE>(), st>>>(sp->vmaps, P);
            break;
    }
}

// With a free surface the reverse (M_GRAD) pass takes the transposed
// z-weights, the others the forward ones.
template <typename T, int MODE = M_FWD>
void launch_v(const StencilPlan* sp, const PassParams& P, cudaStream_t st) {
#if EWS_FULL
    if constexpr (MODE == M_FWD)
        if (P.g.cm[0]) return launch_v_fs<T, MODE, VAR_COARSE>(sp, P, st);
    if (P.g.fs != kNoSurface) {
        if constexpr (MODE == M_GRAD)
            return launch_v_fs<T, MODE, ZS_ADJ>(sp, P, st);
        else
            return launch_v_fs<T, MODE, ZS_FWD>(sp, P, st);
    }
#endif
    launch_v_fs<T, MODE, ZS_NONE>(sp, P, st);
}

template <typename T, int FS>
void launch_s_fs(const StencilPlan* sp, const PassParams& P, cudaStream_t st) {
    dim3 blk(TX, RY);
    switch (sp->kind) {
        case BND_SPONGE:
            k_stress<BND_SPONGE, T, FS><<<sp->grid, blk, smem_s<BND_SPONGE, T>(), st>>>(sp->smaps, P);
            break;
        case BND_CPML:
            k_stress<BND_CPML, T, FS><<<sp->grid, blk, smem_s<BND_CPML, T>(), st>>>(sp->smaps, P);
            break;
        default:
            k_stress<BND_NONE, T, FS><<<sp->grid, blk, smem_s<BND_NONE, T>(), st>>>(sp->smaps, P);
            break;
    }
}

// reverse: the stress pass of the reverse sweep (transposed z-weights with
// a free surface; FP32 storage only).
template <typename T>
void launch_s(const StencilPlan* sp, const PassParams& P, cudaStream_t st, bool reverse) {
#if EWS_FULL
    if (P.g.cm[0]) return launch_s_fs<T, VAR_COARSE>(sp, P, st);
    if (P.g.fs != kNoSurface) {
        if constexpr (std::is_same<T, float>::value)
            if (reverse) return launch_s_fs<T, ZS_ADJ>(sp, P, st);
        return launch_s_fs<T, ZS_FWD>(sp, P, st);
    }
#else
    (void)reverse;
#endif
    launch_s_fs<T, ZS_NONE>(sp, P, st);
}

}  // namespace

cudaError_t stencil_plan_create(const DevGrid& g, const DevFields& F, const DevMedium& M,
                                const DevBoundary& B, int storage, StencilPlan** out) {
    StencilPlan* p = new StencilPlan();
    cudaError_t e = plan_build(p, g, F, M, B, storage);
    if (e != cudaSuccess) {
        delete p;
        return e;
    }
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
    cudaError_t e = plan_build(p, g, F, M, B, EWS_STORAGE_F32);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

int stencil_plan_storage(const StencilPlan* p) { return p->storage; }

cudaError_t launch_velocity(const StencilPlan* sp, const DevGrid& g, const DevFields& F,
                            const DevBoundary& B, const float dto[9], const float inv[9],
                            int* err, cudaStream_t st) {
    const PassParams P = pass_params(sp, g, F, B, dto, inv, err);
    switch (sp->storage) {
        case EWS_STORAGE_BF16: launch_v<__nv_bfloat16>(sp, P, st); break;
        case EWS_STORAGE_F16: launch_v<__half>(sp, P, st); break;
        default: launch_v<float>(sp, P, st); break;
    }
    return cudaGetLastError();
}

#if EWS_FULL
cudaError_t launch_velocity_cap(const StencilPlan* sp, const DevGrid& g, const DevFields& F,
                                const DevBoundary& B, const float dto[9], const VelExtra& X,
                                int* err, cudaStream_t st) {
    if (sp->storage != EWS_STORAGE_F32) return cudaErrorInvalidValue;
    const float one[NFIELD] = {1, 1, 1, 1, 1, 1, 1, 1, 1};
    PassParams P = pass_params(sp, g, F, B, dto, one, err);
    P.X = X;
    launch_v<float, M_CAP>(sp, P, st);
    return cudaGetLastError();
}

cudaError_t launch_velocity_grad(const StencilPlan* sp, const DevGrid& g, const DevFields& F,
                                 const DevBoundary& B, const float dto[9], const VelExtra& X,
                                 int* err, cudaStream_t st) {
    if (sp->storage != EWS_STORAGE_F32 || sp->kind == BND_CPML || !sp->has_hist)
        return cudaErrorInvalidValue;
    const float one[NFIELD] = {1, 1, 1, 1, 1, 1, 1, 1, 1};
    StencilPlan q = *sp;                 // the reverse pass's own z-chunks
    q.zchunk = sp->zchunk_grad;
    q.grid = sp->grid_grad;
    PassParams P = pass_params(&q, g, F, B, dto, one, err);
    P.X = X;
    launch_v<float, M_GRAD>(&q, P, st);
    return cudaGetLastError();
}

cudaError_t stencil_plan_set_history(StencilPlan* p, const DevGrid& g, const float* hist,
                                     long long fstride, int nslot, const float* acc) {
    const CUtensorMapDataType f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const long long fsb = fstride * 4;
    // history: the 3 components of a slot, x and y halos (strain rates) or
    // core tiles (v^{m+3/2} of the buoyancy term); accumulators: all 8
    p->has_hist = encode4(&p->vmaps.hist, g, hist, f32, 4, fsb, 3 * nslot, HXF, HY, 3) &&
                  encode4(&p->vmaps.hcore, g, hist, f32, 4, fsb, 3 * nslot, TX, TY, 3) &&
                  encode4(&p->vmaps.acc, g, acc, f32, 4, fsb, 8, TX, TY, 8);
    return p->has_hist ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BND, bool GRAD>
constexpr size_t batch_smem() {
    return pre_bytes<BND, GRAD>() + (size_t)NSLOT * batch_slot<GRAD>() + 8 * NBAR;
}

template <int BND, bool GRAD, bool FS>
cudaError_t batch_prepare(int* per_sm) {
    return prepare(k_batch<BND, GRAD, FS>, batch_smem<BND, GRAD>(), per_sm);
}

// C-PML shots have no reverse executor (no C-PML adjoint).
template <int BND>
cudaError_t batch_occupancy_b(int exec, int* per_sm) {
    switch (exec) {
        case BX_LEAN: return batch_prepare<BND, false, false>(per_sm);
        case BX_LEAN_FS: return batch_prepare<BND, false, true>(per_sm);
        default: break;
    }
    if constexpr (BND != BND_CPML) {
        if (exec == BX_GRAD) return batch_prepare<BND, true, false>(per_sm);
        if (exec == BX_GRAD_FS) return batch_prepare<BND, true, true>(per_sm);
    }
    return cudaErrorInvalidValue;
}

cudaError_t batch_occupancy(int bnd, int exec, int* per_sm) {
    if (bnd == BND_SPONGE) return batch_occupancy_b<BND_SPONGE>(exec, per_sm);
    if (bnd == BND_NONE) return batch_occupancy_b<BND_NONE>(exec, per_sm);
    if (bnd == BND_CPML) return batch_occupancy_b<BND_CPML>(exec, per_sm);
    return cudaErrorInvalidValue;
}

template <int BND, bool GRAD, bool FS>
void batch_go(int grid, const BatchShot* shots, const BatchEntry* entries, int nentries,
              unsigned* cur, unsigned* taken, unsigned long long* done, int* err,
              unsigned long long wait_ns, cudaStream_t st) {
    k_batch<BND, GRAD, FS><<<grid, dim3(TX, RY), batch_smem<BND, GRAD>(), st>>>(
        shots, entries, nentries, cur, taken, done, err, wait_ns);
}

template <int BND>
cudaError_t launch_batch_b(int exec, int grid, const BatchShot* shots, const BatchEntry* entries,
                           int nentries, unsigned* cur, unsigned* taken,
                           unsigned long long* done, int* err, unsigned long long wait_ns,
                           cudaStream_t st) {
    switch (exec) {
        case BX_LEAN: batch_go<BND, false, false>(grid, shots, entries, nentries, cur, taken, done, err, wait_ns, st); break;
        case BX_LEAN_FS: batch_go<BND, false, true>(grid, shots, entries, nentries, cur, taken, done, err, wait_ns, st); break;
        case BX_GRAD:
        case BX_GRAD_FS:
            if constexpr (BND != BND_CPML) {
                if (exec == BX_GRAD)
                    batch_go<BND, true, false>(grid, shots, entries, nentries, cur, taken, done, err, wait_ns, st);
                else
                    batch_go<BND, true, true>(grid, shots, entries, nentries, cur, taken, done, err, wait_ns, st);
                break;
            }
            return cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_batch(int bnd, int exec, int grid, const BatchShot* shots,
                         const BatchEntry* entries, int nentries, unsigned* cur,
                         unsigned* taken, unsigned long long* done, int* err,
                         unsigned long long wait_ns, cudaStream_t st) {
    if (bnd == BND_SPONGE)
        return launch_batch_b<BND_SPONGE>(exec, grid, shots, entries, nentries, cur, taken, done, err, wait_ns, st);
    if (bnd == BND_NONE)
        return launch_batch_b<BND_NONE>(exec, grid, shots, entries, nentries, cur, taken, done, err, wait_ns, st);
    if (bnd == BND_CPML)
        return launch_batch_b<BND_CPML>(exec, grid, shots, entries, nentries, cur, taken, done, err, wait_ns, st);
    return cudaErrorInvalidValue;
}

void stencil_plan_export(const StencilPlan* p, Maps* vmaps, Maps* smaps, int* ntx, int* nty,
                         int* zchunk, int* items) {
    *vmaps = p->vmaps;
    *smaps = p->smaps;
    *ntx = p->ntx;
    *nty = p->nty;
    *zchunk = p->zchunk;
    *items = p->grid;
}
#endif  // EWS_FULL

cudaError_t launch_stress(const StencilPlan* sp, const DevGrid& g, const DevFields& F,
                          const DevBoundary& B, const float dto[9], const float inv[9],
                          int* err, cudaStream_t st, bool reverse) {
    const PassParams P = pass_params(sp, g, F, B, dto, inv, err);
    switch (sp->storage) {
        case EWS_STORAGE_BF16: launch_s<__nv_bfloat16>(sp, P, st, false); break;
        case EWS_STORAGE_F16: launch_s<__half>(sp, P, st, false); break;
        default: launch_s<float>(sp, P, st, reverse); break;
    }
    return cudaGetLastError();
}

#ifdef EWS_SHAPE_NS
}  // namespace EWS_SHAPE_NS
#endif
}  // namespace ews
