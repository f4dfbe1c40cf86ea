// ews_internal.cuh -- device data structures and kernel launchers of libews.
//
// Layout in HBM (one simulation):
//   * 9 wavefields in one allocation, each [nz][ny][pitch] of the storage
//     type (float32, or bf16 / fp16 holding s_q times the value for a
//     per-field power-of-two scale s_q) with pitch = nx rounded up to 32
//     elements (rows of 64 or 128 bytes, 16-byte aligned for TMA).  Padding
//     columns stay zero and are never written.  Field q starts at element
//     q * fstride of the allocation (fstride a multiple of 64 elements).
//     DevFields carries the field base addresses as float*; kernels for
//     16-bit storage cast them to the storage type.
//   * lambda, mu, rho per cell in a second allocation, same layout.  The
//     staggered-point means of Sec. 2.2.1 are formed in registers by the
//     stencil kernels; nothing else about the medium is stored.
//   * C-PML memory variables: 18 arrays with the field layout (6 per damped
//       direction); only slab cells are used, so stencil tiles can bring
//       them in with the same TMA boxes as the fields.
//   * seismograms [3][nrec][nt] float32; wavelet [nt] float32.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ews.h"

namespace ews {

enum { VX, VY, VZ, SXX, SYY, SZZ, SXY, SXZ, SYZ, NFIELD };

// Physical slot fslot(q) of field q (state order above) in a 9-field allocation
// (wavefields, adjoint fields, the no-allocation scratch): slots 0..8 hold
// sxx sxz syy syz sxy szz vx vy vz.  Each pass's fields then sit next to
// each other in the shapes it fetches them in (sxx/sxz with x halos, syy/syz
// with y halos, szz vx vy vz as core tiles; vx vy vz with x and y halos, the
// six stresses as core tiles), so one 4D TMA copy brings several tiles.
// Checkpoints copy the whole allocation, and the velocity history copies
// slots 6..8 (vx vy vz) as one block.
__host__ __device__ constexpr int fslot(int q) {
    return q == VX ? 6 : q == VY ? 7 : q == VZ ? 8 : q == SXX ? 0 : q == SYY ? 2 : q == SZZ ? 5
         : q == SXY ? 4 : q == SXZ ? 1 : 3;
}
enum { BND_NONE = 0, BND_SPONGE = 1, BND_CPML = 2 };

struct DevGrid {
    int nx, ny, nz;
    int pitch;            // elements per row
    long long plane;      // elements per z-plane = pitch * ny
    // Eq. 4 weights divided by the axis spacing (reading: the 1/h factor)
    float c1x, c2x, c1y, c2y, c1z, c2z;
    // free surface (Sec. 2.5, vacuum formulation): plane index ks of the
    // first cell below the surface (kNoSurface without one) and the weight
    // 1/dz of the 2nd-order z-difference used next to it
    int fs;
    float c1z2;
    float fs_eps;         // vacuum fraction above the surface
    // coarse medium grid (Sec. 2.2.1: medium textures smaller than the
    // wavefield textures, sampled by trilinear interpolation): lambda, mu,
    // rho as dense [mz][my][mx] arrays (null: the medium has the wavefield
    // grid's cells), and m / n per axis
    const float* cm[3];
    int mx, my, mz;
    float rx, ry, rz;
};
constexpr int kNoSurface = -(1 << 28);

// Trilinear sampling of a coarse medium array (reading of Sec. 2.2.1): a
// wavefield-grid position x (cells) maps to the medium coordinate
// c = (x + 1/2) m / n - 1/2, clamped to [0, m - 1]; i0 is the lower of the
// two medium cells used and f the weight of the upper one.
struct Ax {
    int i0;
    float f;
};
__device__ __forceinline__ Ax axis_at(float x, float r, int m) {
    float c = fmaf(x + 0.5f, r, -0.5f);
    c = fminf(fmaxf(c, 0.0f), (float)(m - 1));
    const int i0 = min((int)c, max(m - 2, 0));
    return Ax{i0, c - (float)i0};
}
__device__ __forceinline__ float lerp1(float a, float b, float t) { return fmaf(t, b - a, a); }
// q: 0 lambda, 1 mu, 2 rho.  Axes of extent 1 read the same cell twice.
__device__ __forceinline__ float coarse_tri(const DevGrid& g, int q, Ax x, Ax y, Ax z) {
    const int ox = g.mx > 1 ? 1 : 0, oy = g.my > 1 ? g.mx : 0;
    const long long oz = g.mz > 1 ? (long long)g.mx * g.my : 0;
    const float* p = g.cm[q] + ((long long)z.i0 * g.my + y.i0) * g.mx + x.i0;
    const float c00 = lerp1(__ldg(p), __ldg(p + ox), x.f);
    const float c10 = lerp1(__ldg(p + oy), __ldg(p + oy + ox), x.f);
    const float c01 = lerp1(__ldg(p + oz), __ldg(p + oz + ox), x.f);
    const float c11 = lerp1(__ldg(p + oz + oy), __ldg(p + oz + oy + ox), x.f);
    return lerp1(lerp1(c00, c10, y.f), lerp1(c01, c11, y.f), z.f);
}
// Coarse-medium value q at wavefield-grid position (x, y, z) in cells.
__device__ __forceinline__ float coarse_at(const DevGrid& g, int q, float x, float y, float z) {
    return coarse_tri(g, q, axis_at(x, g.rx, g.mx), axis_at(y, g.ry, g.my),
                      axis_at(z, g.rz, g.mz));
}

// Forms of the passes' z-differences: no free surface; the forward form
// with a surface; the transposed form of the reverse sweep with a surface.
// A pass variant is one of these, or VAR_COARSE (no surface, the medium
// sampled from a coarse grid instead of read as tiles).
enum { ZS_NONE = 0, ZS_FWD = 1, ZS_ADJ = 2, VAR_COARSE = 4 };

// z-difference forms at output plane k (free-surface reading): a
// z-derivative whose Eq. 4 stencil would take samples on both sides of the
// surface plane z = (ks - 1/2) dz uses the 2nd-order difference: outputs at
// integer z (planes ks-1, ks: i2) and at half-integer z (planes ks-2 .. ks:
// h2).  Without a surface (FS = ZS_NONE) both are false.
struct ZW {
    bool i2, h2;
    __host__ __device__ float c1i(const DevGrid& g) const { return i2 ? g.c1z2 : g.c1z; }
    __host__ __device__ float c2i(const DevGrid& g) const { return i2 ? 0.0f : g.c2z; }
    __host__ __device__ float c1h(const DevGrid& g) const { return h2 ? g.c1z2 : g.c1z; }
    __host__ __device__ float c2h(const DevGrid& g) const { return h2 ? 0.0f : g.c2z; }
};
template <int FS>
__host__ __device__ __forceinline__ ZW zweights(const DevGrid& g, int k) {
    if constexpr (FS != ZS_NONE)
        return ZW{(unsigned)(k - g.fs + 1) < 2u, (unsigned)(k - g.fs + 2) < 3u};
    else
        return ZW{false, false};
}

// Transposed z-weights at output plane k, per tap (A..D = the four samples
// from the lowest plane up), for the reverse sweep with a surface.  The
// transpose of the forward difference that maps half-z samples to integer-z
// outputs is the map from integer-z samples to half-z outputs whose row k
// holds, at each sample, the weight that sample's own output row gives to
// plane k: an integer-z output at k (samples on half planes k-2 .. k+1)
// takes the half-output weights of those planes, and a half-z output at k
// (samples on integer planes k-1 .. k+2) the integer-output weights.
struct ZT {
    float iA, iB, iC, iD, hA, hB, hC, hD;
};
__host__ __device__ __forceinline__ ZT ztransposed(const DevGrid& g, int k) {
    const ZW m2 = zweights<ZS_FWD>(g, k - 2), m1 = zweights<ZS_FWD>(g, k - 1);
    const ZW z0 = zweights<ZS_FWD>(g, k), p1 = zweights<ZS_FWD>(g, k + 1);
    const ZW p2 = zweights<ZS_FWD>(g, k + 2);
    return ZT{-m2.c2h(g), -m1.c1h(g), z0.c1h(g), p1.c2h(g),
              -m1.c2i(g), -z0.c1i(g), p1.c1i(g), p2.c2i(g)};
}

// One z-difference from the four samples a..d (lowest plane first) of an
// integer-z (HALF false) or half-integer-z (HALF true) output.
template <int FS, bool HALF>
__device__ __forceinline__ float zdiff(const DevGrid& g, const ZW& zw, const ZT& zt, float a,
                                       float b, float c, float d) {
    if constexpr (FS == ZS_ADJ) {
        return HALF ? zt.hA * a + zt.hB * b + zt.hC * c + zt.hD * d
                    : zt.iA * a + zt.iB * b + zt.iC * c + zt.iD * d;
    } else if constexpr (FS == ZS_FWD) {
        // Eq. 4, or its inner pair alone on the switched planes
        return (HALF ? zw.h2 : zw.i2) ? g.c1z2 * (c - b) : g.c1z * (c - b) + g.c2z * (d - a);
    } else {
        return g.c1z * (c - b) + g.c2z * (d - a);
    }
}

struct DevFields {
    float* f[NFIELD];
};

struct DevMedium {
    const float* lam;
    const float* mu;
    const float* rho;
};

struct DevBoundary {
    int kind;             // BND_*
    int W;                // slab width in cells
    const float* g[3];    // sponge profile per axis, length n_axis
    const float* pa[3];   // C-PML a(i) per axis
    const float* pb[3];   // C-PML b(i) per axis
    // C-PML memory variables, full-size and pitched like the fields:
    // psi[6 * d + t], d = damped direction (x, y, z), t = 0..2 velocity-pass
    // terms, 3..5 stress-pass terms.  Only cells inside the slab of
    // direction d are ever read or written.
    float* psi[18];
};

// One injection or sampling tap: field q, element (i, j, k), weight w.
struct Tap {
    int q, i, j, k;
    float w;
};

static constexpr int kMaxSrcTaps = 48;   // 6 components x 8 neighbours

struct DevSource {
    int kind;             // 0 moment, 1 force, -1 none
    int ntap;
    Tap tap[kMaxSrcTaps]; // w already holds -dt M_c w_tri / V or dt F_c w_tri / V
};

// Adjoint state (ews_adjoint.cu): p velocity-like, q stress-like, FP32
// per-segment accumulators and FP64 totals (meaning per formulation in
// ews_adjoint.cu; both keep lambda / normal-mu terms in acc[0..1], shear
// terms at the xy/xz/yz points in acc[2..4], buoyancy terms at the vx/vy/vz
// points in acc[5..7]).
struct AdjFields {
    float* p[3];
    float* q[6];
    float* acc[8];
    double* acc64[8];
};

cudaError_t launch_adj_stress(const DevGrid& g, const AdjFields& A, const DevMedium& M,
                              const DevBoundary& B, const float* vh, size_t fstride, float dt,
                              cudaStream_t st);
cudaError_t launch_adj_velocity(const DevGrid& g, const AdjFields& A, const DevMedium& M,
                                const DevBoundary& B, const float* vn, const float* vp,
                                size_t fstride, float dt, cudaStream_t st);
cudaError_t launch_adj_record(const DevGrid& g, const AdjFields& A, const Tap* taps, int nrec,
                              const float* sadj, int ld, int n, cudaStream_t st);
cudaError_t launch_acc_flush(const DevGrid& g, const AdjFields& A, cudaStream_t st);
cudaError_t launch_grad_finalize(const DevGrid& g, const AdjFields& A, const DevMedium& M,
                                 float* glam, float* gmu, float* grho, cudaStream_t st);
cudaError_t launch_residual(const float* seis, const float* obs, float* sadj, long long n,
                            float dt, double* misfit, cudaStream_t st);
// 16-bit checkpoint of the 9 fields (each fs floats) into dst (storage
// BF16 / FP16, 9 * fs elements), with per-field power-of-two scales written
// to scales[9] (amax: 9 unsigned of scratch); and its restore.
cudaError_t launch_ckpt_store(const float* fields, long long fs, int storage, unsigned* amax,
                              float* scales, void* dst, cudaStream_t st);
cudaError_t launch_ckpt_load(const void* src, long long fs, int storage, const float* scales,
                             float* fields, cudaStream_t st);
// Transformed formulation (p = alpha, q = tau; see ews_adjoint.cu).
cudaError_t launch_adj_inject(const DevGrid& g, const AdjFields& A, const DevMedium& M,
                              const DevBoundary& B, const Tap* taps, int nrec, const float* sadj,
                              int ld, int n, cudaStream_t st);
cudaError_t launch_rho_term(const DevGrid& g, const AdjFields& A, const DevBoundary& B,
                            const float* vn, const float* vp, long long fstride, cudaStream_t st);
cudaError_t launch_grad_finalize_t(const DevGrid& g, const AdjFields& A, const DevMedium& M,
                                   float* glam, float* gmu, float* grho, cudaStream_t st);

// Thread-local error message for ews_last_error() (ews_capi.cu).
ews_status report(ews_status s, const char* fmt, ...);

// Device allocations of the library (ews_mem.cu): counted against the
// optional process-wide limit of ews_set_memory_limit.  dev_malloc returns
// cudaErrorMemoryAllocation, without calling CUDA, for a request above the
// limit; dev_headroom is the room left under it (INFINITY without a limit).
cudaError_t dev_malloc(void** p, size_t bytes);
void dev_free(void* p);
double dev_headroom();

// Stencil passes (ews_stencil.cu): TMA tensor maps and launch geometry are
// built once per simulation (the field and medium addresses never change).
// Extra operands of the velocity pass when it captures the velocity history
// (checkpoint recomputation) or runs as the reverse (adjoint) pass with the
// gradient products fused in.
struct VelExtra {
    float* vcap;          // capture: destination of v^{n+1/2} (3 fields, fstride apart)
    const float* vnext;   // reverse: v^{m+3/2} (3 fields) for the buoyancy term, or null
    float* acc[8];        // reverse: FP32 gradient accumulators (AdjFields order)
    long long fstride;    // elements between the fields of a history slot
    float gdt;            // reverse: dt of the forward step
    int hslot;            // reverse: history slot holding v^{m+1/2}
};

struct StencilPlan;

// Tensor maps of one pass (ews_stencil.cu), in the order of its shared-memory
// slot layout: halo tiles, core tiles (fields that lie next to each other in
// the field allocation go through one 4D map over [field][nz][ny][pitch], so
// one copy brings several tiles), the C-PML memory variables (one 4D map over
// the 18 arrays: one copy brings the 3 terms of a damped direction), and the
// velocity-history map of the reverse pass.
static constexpr int kMapsHalo = 6, kMapsCore = 1;
struct Maps {
    CUtensorMap halo[kMapsHalo];
    CUtensorMap core[kMapsCore];
    CUtensorMap psi;      // C-PML memory variables [term][nz][ny][pitch] (4D)
    CUtensorMap hist;     // velocity history [slot * 3 + component][nz][ny][pitch] (4D),
                          // x and y halo boxes of the 3 components of a slot
    CUtensorMap hcore;    // the same history, core boxes of the 3 components
    CUtensorMap acc;      // the 8 FP32 gradient accumulators [q][nz][ny][pitch] (4D)
};

// Parameters of one pass launch (or one batched work item).
struct PassParams {
    DevGrid g;
    DevFields F;
    DevBoundary B;
    float dto[9];         // per output field: dt x its storage scale
    float inv[9];         // per input field: 1 / its storage scale (16-bit storage)
    int ntx, nty;
    int zchunk;           // planes per z-chunk
    int* err;
    VelExtra X;           // history / gradient operands of the capture and reverse modes
};

// ---- batched executor (ews_stencil.cu kernel, ews_batch.cu programs) ----
//
// One persistent launch runs the programs of many independent shots.  A
// program is a sequence of stages; a stage is a set of work items (tiles x
// z-chunks of a pass, chunks of cells of an elementwise step, or a single
// item).  Stages of all shots are merged into one list of entries ordered by
// the fraction of its program a stage completes, so shots progress together.
// CTAs claim items entry by entry (an entry's items are handed out only
// after every item of the previous entries was), and an item of stage r of
// shot s starts once every item of stages < r of s has finished (per-shot
// done counter, bounded wait).  Claims follow the entry order, so every
// awaited item was claimed earlier by a running CTA: no deadlock, whatever
// the number of resident CTAs.
// Point terms ride on the pass items that own their cells: the force of
// step n on the velocity-pass items (also into the history when capturing),
// the moment on the stress-pass items, the residual on the reverse
// velocity-pass items, and the receivers (when flag) on the stress-pass
// items holding their first tap.
enum BatchKind {
    BK_VEL = 0,       // forward velocity pass of step n
    BK_VEL_CAP,       // forward velocity pass of step n writing history slot `slot`
    BK_VEL_GRAD,      // reverse velocity pass of step n, history slot `slot`; flag: buoyancy term
    BK_STR,           // forward stress pass of step n; flag: record the receivers
    BK_STR_ADJ,       // reverse stress pass
    BK_SAVE,          // fields -> checkpoint `slot`
    BK_LOAD,          // checkpoint `slot` -> fields
    BK_HIST0,         // v -> history slot 0
    BK_ZERO_F,        // fields (and C-PML-free state) := 0
    BK_ZERO_A,        // adjoint fields and accumulators := 0
    BK_RESID,         // residual dt (s - d) and misfit
    BK_FLUSH,         // FP64 accumulators += FP32 ones; FP32 := 0
    BK_RHO,           // buoyancy term of a segment's first reverse step
    BK_FINAL,         // gradients from the accumulators
    BK_NKIND
};

struct BatchEntry {
    int shot, kind, n, slot;
    long long need;       // items of the shot's earlier stages
    int nitems;
    int flag;             // see BatchKind
};

struct alignas(64) BatchShot {
    Maps vf, sf;          // forward field maps
    Maps va, sa;          // adjoint field maps (va.hist: velocity history)
    PassParams pf;        // forward passes (dto = dt)
    PassParams pa;        // reverse passes (dto = -dt; X.acc, X.fstride, X.gdt set)
    DevMedium M;
    DevSource S;          // tap weights hold dt and 1 / V
    const float* wavelet;
    const Tap* rtaps;
    int nrec, nt;         // receivers; steps (seismogram leading dimension)
    float* seis;          // [3][nrec][nt] or null
    AdjFields A;
    float* vhist;         // history slots of 3 fields
    float* ckpt;          // checkpoints of 9 fields
    long long fs;         // elements per field (padded)
    const float* obs;     // observed seismograms (gradient shots)
    float* sadj;          // residual dt (s - d)
    double* misfit;
    float *gl, *gm, *gr;  // dense gradients
    int items_pass;       // tiles x z-chunks of one pass
    int items_elem;       // cell chunks of one elementwise stage
    float dt;
    int ck16;             // checkpoints stored as BF16 (1) or FP32 (0)
};
static constexpr int kBatchElem = 8192;   // cells per elementwise work item

// Executor forms: the lean one (forward stages, 3 CTAs per SM), the one with
// the reverse passes (larger slots, 2 per SM), and both again with the
// free-surface z-differences (grids with a surface; shots without one run
// unchanged in them).
enum { BX_LEAN = 0, BX_GRAD = 1, BX_LEAN_FS = 2, BX_GRAD_FS = 3 };

// Launch the executor `exec` over `nentries` entries (device tables; the
// counters cur/taken/done start at zero).  grid: CTAs to launch.  err bits:
// 1 / 2 stencil waits, 8 a dependency wait gave up.
cudaError_t launch_batch(int bnd, int exec, int grid, const BatchShot* shots,
                         const BatchEntry* entries, int nentries, unsigned* cur,
                         unsigned* taken, unsigned long long* done, int* err,
                         unsigned long long wait_ns, cudaStream_t st);
// CTAs per SM the executor achieves (sets its shared-memory attribute).
cudaError_t batch_occupancy(int bnd, int exec, int* per_sm);
// The plan's tensor maps and pass parameters, for a BatchShot.
void stencil_plan_export(const StencilPlan* p, Maps* vmaps, Maps* smaps, int* ntx, int* nty,
                         int* zchunk, int* items);

// The passes take, per field q, dto[q] = dt s_q (used for the fields they
// write) and inv[q] = 1 / s_q (used for the 16-bit fields they read); with
// FP32 storage s_q = 1.  *err collects bit 1 / 2 (a velocity / stress pipeline
// wait gave up), bit 4 (a value beyond the FP16 range was stored) and bit
// 16 (a receiver recorded a NaN or Inf).
struct StencilPlan;
cudaError_t stencil_plan_create(const DevGrid& g, const DevFields& F, const DevMedium& M,
                                const DevBoundary& B, int storage, StencilPlan** out);
void stencil_plan_destroy(StencilPlan* p);
size_t stencil_plan_bytes();
cudaError_t stencil_plan_fill(void* storage, const DevGrid& g, const DevFields& F,
                              const DevMedium& M, const DevBoundary& B, StencilPlan** out);
int stencil_plan_storage(const StencilPlan* p);
cudaError_t launch_velocity(const StencilPlan* sp, const DevGrid& g, const DevFields& F,
                            const DevBoundary& B, const float dto[9], const float inv[9],
                            int* err, cudaStream_t st);
cudaError_t launch_stress(const StencilPlan* sp, const DevGrid& g, const DevFields& F,
                          const DevBoundary& B, const float dto[9], const float inv[9],
                          int* err, cudaStream_t st, bool reverse = false);
// FP32 storage only.  Velocity pass that also writes v^{n+1/2} to X.vcap:
cudaError_t launch_velocity_cap(const StencilPlan* sp, const DevGrid& g, const DevFields& F,
                                const DevBoundary& B, const float dto[9], const VelExtra& X,
                                int* err, cudaStream_t st);
// Reverse velocity pass on the adjoint fields F (dto = -dt) with the gradient
// products of reverse step m accumulated into X.acc (history tiles from the
// map set by stencil_plan_set_history; boundary none or sponge):
cudaError_t launch_velocity_grad(const StencilPlan* sp, const DevGrid& g, const DevFields& F,
                                 const DevBoundary& B, const float dto[9], const VelExtra& X,
                                 int* err, cudaStream_t st);
// The plain forward passes built again with other tile shapes
// (ews_stencil_t4.cu: 32 x 4 cells; ews_stencil_t16.cu: 32 x 16 cells, two
// rows per thread), each in its own namespace.  Every cell runs the same
// arithmetic in the same order as in the 32 x 8 passes (separately
// compiled, so results agree to FP32 rounding).  No free surface, coarse medium grid or history capture: the
// callers use these only for plain forward steps.
#define EWS_SHAPE_DECLS(NS)                                                                  \
    namespace NS {                                                                           \
    struct StencilPlan;                                                                      \
    cudaError_t stencil_plan_create(const DevGrid& g, const DevFields& F, const DevMedium& M, \
                                    const DevBoundary& B, int storage, StencilPlan** out);   \
    void stencil_plan_destroy(StencilPlan* p);                                               \
    cudaError_t launch_velocity(const StencilPlan* sp, const DevGrid& g, const DevFields& F, \
                                const DevBoundary& B, const float dto[9], const float inv[9], \
                                int* err, cudaStream_t st);                                  \
    cudaError_t launch_stress(const StencilPlan* sp, const DevGrid& g, const DevFields& F,   \
                              const DevBoundary& B, const float dto[9], const float inv[9],  \
                              int* err, cudaStream_t st, bool reverse = false);              \
    }
EWS_SHAPE_DECLS(t32x4)
EWS_SHAPE_DECLS(t32x16)

// One launch per time step (ews_fused.cu): the velocity and stress passes of
// step n fused, reading sigma^n, v^{n-1/2} from one set of wavefields and
// writing v^{n+1/2}, sigma^{n+1} to a second set (dir 0: A -> B, dir 1:
// B -> A), with a point force of step n (S.kind 1) added inside.  FP32
// storage with unit scales, sponge or no absorbing boundary, no free surface
// or coarse medium grid.
namespace fused {
struct FusedPlan;
bool fused_supported(const DevGrid& g, const DevBoundary& B, int storage);
cudaError_t fused_plan_create(const DevGrid& g, const DevFields& A, const DevFields& Bf,
                              const DevMedium& M, const DevBoundary& B, FusedPlan** out);
void fused_plan_destroy(FusedPlan* p);
cudaError_t launch_fused(const FusedPlan* p, int dir, const DevGrid& g, const DevMedium& M,
                         const DevBoundary& B, float dt, const DevSource& S, const float* wavelet,
                         int n, int* err, cudaStream_t st);
}  // namespace fused

// History buffer of the reverse pass: nslot slots of 3 fields, slot s field c
// at hist + (3 s + c) * fstride, pitched like the wavefields; and its 8 FP32
// gradient accumulators, accumulator q at acc + q * fstride.
cudaError_t stencil_plan_set_history(StencilPlan* p, const DevGrid& g, const float* hist,
                                     long long fstride, int nslot, const float* acc);

// Sources, receivers, medium set-up and storage conversion (ews_forward.cu).
// All run on `st`; `storage` is the EWS_STORAGE_* type of the wavefields.
// Source tap weights already include the field scale; receivers multiply
// each sample by inv[component].
cudaError_t launch_inject(const DevGrid& g, const DevFields& F, const DevMedium& M,
                          const DevBoundary& B, const DevSource& S, const float* wavelet,
                          int n, int storage, int* err, cudaStream_t st);
cudaError_t launch_record(const DevGrid& g, const DevFields& F, const Tap* taps, int nrec,
                          float* seis, int ld, int n, int storage, const float inv[3], int* err,
                          cudaStream_t st);
// Moment-source injection (S.kind MOMENT, else none) and receiver sampling
// of step n in one launch, after the stress pass.
cudaError_t launch_post_stress(const DevGrid& g, const DevFields& F, const DevMedium& M,
                               const DevBoundary& B, const DevSource& S, const float* wavelet,
                               const Tap* taps, int nrec, float* seis, int ld, int n, int storage,
                               const float inv[3], int* err, cudaStream_t st);
// flags[0]: validity bits (bit4: some mu == 0); flags[1..4]: float bits of max vp, min rho,
// min sqrt(rho mu) over cells with mu > 0 (else FLT_MAX), max sqrt(rho (lambda + 2 mu));
// the two minima only over cells below a free surface.
// launch_vacuum: the cells above the free surface g.fs take eps times the medium
// of the cell below the surface (raw input arrays, before launch_medium_setup).
cudaError_t launch_vacuum(const DevGrid& g, float* a, float* b, float* rho, int from_velocities,
                          float eps, cudaStream_t st);
cudaError_t launch_medium_setup(const DevGrid& g, float* a, float* b, float* rho,
                                int from_velocities, unsigned* flags, cudaStream_t st);
// One field between its stored form (pitched, `storage` type, scaled by s)
// and a dense [nz][ny][nx] float32 array: out = stored / s, stored = s in.
cudaError_t launch_field_out(const DevGrid& g, const void* field, int storage, float inv_s,
                             float* dense, cudaStream_t st);
cudaError_t launch_field_in(const DevGrid& g, const float* dense, int storage, float s,
                            void* field, int* err, cudaStream_t st);

}  // namespace ews
