// ews_noalloc.cu -- ews_forward_noalloc: a whole forward run whose working
// memory is one file-scope device array instead of cudaMalloc'ed buffers.
//
// Who needs it: callers that must not allocate device memory while they
// run -- a process whose device memory is owned by another allocator (a
// framework's caching allocator, a pre-sized pool in a long-running
// service) that must not be fragmented or grown behind its back, and code
// that cannot afford the implicit device-wide synchronisation cudaFree
// brings.  They pass the medium, wavelet and seismogram buffers they already
// own; everything else (9 wavefields, pitched medium copies, boundary
// profiles, receiver taps, flags) lives in g_scratch below.
//
// g_scratch is a static __device__ array: every GPU that loads libews holds
// it (about 12 MiB) until the process exits.  Host code cannot pass the
// array's name to a kernel (on the host it is only a stand-in symbol), so the
// first call on each device looks up its device address with
// cudaGetSymbolAddress while that device is current and caches it (one
// atomic slot per device, so host threads making their first calls at the
// same time are safe).  Make that first call before capturing any stream on
// the device.  All calls share the one array and it keeps the previous
// call's contents: this entry point clears what must start at zero, and
// calls that overlap on the GPU (other streams, other host threads) race on
// it.  Host-side staging is small (a few KB of stack; the stencil plan's
// tensor maps in thread-local storage), so the call also suits service
// threads with small stacks.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>

#include "ews_internal.cuh"

namespace ews {
namespace {

constexpr long long kMaxCells = EWS_NOALLOC_MAX_CELLS;    // padded cells per field
constexpr int kMaxRec = EWS_NOALLOC_MAX_RECEIVERS;
constexpr int kMaxDim = EWS_NOALLOC_MAX_DIM;
constexpr int kTapWords = (int)(sizeof(Tap) / sizeof(float));
static_assert(sizeof(Tap) % sizeof(float) == 0, "taps are packed in float words");

// Layout of the scratch array, in floats.
constexpr size_t kOffFields = 0;                                   // 9 wavefields
constexpr size_t kOffMedium = 9 * (size_t)kMaxCells;               // lambda, mu, rho
constexpr size_t kOffProf = 12 * (size_t)kMaxCells;                // sponge g[3][kMaxDim]
constexpr size_t kOffTaps = kOffProf + 9 * (size_t)kMaxDim;        // receiver taps
constexpr size_t kOffFlags = kOffTaps + 24 * (size_t)kMaxRec * kTapWords;
constexpr size_t kScratchFloats = kOffFlags + 64;                  // flags, vp_max, err

static __device__ __align__(256) float g_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::atomic<float*> g_scratch_dev[kMaxDevices];   // device address of g_scratch, per device

ews_status scratch_address(float** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return report(EWS_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return report(EWS_ECUDA, "device index %d unsupported", dev);
    float* a = g_scratch_dev[dev].load(std::memory_order_acquire);
    if (!a) {
        // Two threads may both look it up; they store the same address.
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return report(EWS_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        a = static_cast<float*>(p);
        g_scratch_dev[dev].store(a, std::memory_order_release);
    }
    *out = a;
    return EWS_OK;
}

// Trilinear taps of point p on the grid of field q (Sec. 2.1.1 offsets).
void point_taps(const ews_grid& gr, int q, const double p[3], double scale, Tap out[8]) {
    static const double off[NFIELD][3] = {{0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5},
                                          {0, 0, 0},   {0, 0, 0},   {0, 0, 0},
                                          {0.5, 0.5, 0}, {0.5, 0, 0.5}, {0, 0.5, 0.5}};
    const double h[3] = {gr.dx, gr.dy, gr.dz};
    int i0[3];
    double fr[3];
    for (int a = 0; a < 3; ++a) {
        const double u = p[a] / h[a] - off[q][a];
        const double fl = std::floor(u);
        i0[a] = (int)fl;
        fr[a] = u - fl;
    }
    int m = 0;
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di, ++m) {
                out[m].q = q;
                out[m].i = i0[0] + di;
                out[m].j = i0[1] + dj;
                out[m].k = i0[2] + dk;
                out[m].w = (float)(scale * (di ? fr[0] : 1 - fr[0]) * (dj ? fr[1] : 1 - fr[1]) *
                                   (dk ? fr[2] : 1 - fr[2]));
            }
}

bool position_ok(const ews_grid& gr, const double p[3]) {
    const int n[3] = {gr.nx, gr.ny, gr.nz};
    const double h[3] = {gr.dx, gr.dy, gr.dz};
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(p[a]) || p[a] < h[a] * (1.0 - 1e-12) ||
            p[a] > (n[a] - 2) * h[a] * (1.0 + 1e-12))
            return false;
    return true;
}

// On failure after device work was queued, wait for the work already on
// the stream (its kernels may still be writing the shared array) before
// returning, so the next call, on any stream, does not race with it.
#define NA_CK(call)                                                                    \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            (void)cudaStreamSynchronize(stream);                                       \
            return report(EWS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));        \
        }                                                                              \
    } while (0)

}  // namespace
}  // namespace ews

using namespace ews;

extern "C" ews_status ews_forward_noalloc(const ews_grid* grid, const ews_options* opt,
                                          const float* lam, const float* mu, const float* rho,
                                          int src_kind, const double pos[3],
                                          const double comp[6], const float* wavelet, int nrec,
                                          const double* rec_pos, int nt, double dt, float* seis,
                                          void* cuda_stream) {
    // ---- host-side checks (no device work yet) ----
    if (!grid || !lam || !mu || !rho || !wavelet || !pos || !comp)
        return report(EWS_EINVAL, "null argument");
    const ews_grid gr = *grid;
    if (gr.nx < 4 || gr.ny < 4 || gr.nz < 4 || !(gr.dx > 0) || !(gr.dy > 0) || !(gr.dz > 0))
        return report(EWS_EINVAL, "bad grid");
    if (gr.nx > kMaxDim || gr.ny > kMaxDim || gr.nz > kMaxDim)
        return report(EWS_EINVAL, "grid side above the no-allocation limit of %d cells", kMaxDim);
    const int pitch = (gr.nx + 31) / 32 * 32;
    const long long padded = (long long)pitch * gr.ny * gr.nz;
    if (padded > kMaxCells)
        return report(EWS_EINVAL,
                      "grid needs %lld padded cells per field (x rounded up to 32); the "
                      "no-allocation limit is %lld",
                      padded, (long long)kMaxCells);
    const int bnd = opt ? opt->boundary : EWS_BOUNDARY_SPONGE;
    const int W = opt ? opt->width : 16;
    if (bnd == EWS_BOUNDARY_CPML)
        return report(EWS_EINVAL, "C-PML needs memory variables; use ews_create/ews_run");
    if (bnd != EWS_BOUNDARY_NONE && bnd != EWS_BOUNDARY_SPONGE)
        return report(EWS_EINVAL, "unknown boundary kind");
    if (bnd == EWS_BOUNDARY_SPONGE && (W < 1 || 2 * W > gr.nx || 2 * W > gr.ny || 2 * W > gr.nz))
        return report(EWS_EINVAL, "bad sponge width");
    if (opt && opt->storage != EWS_STORAGE_F32) return report(EWS_EINVAL, "only F32 storage");
    if (nt <= 0) return report(EWS_EINVAL, "nt must be positive");
    if (nrec < 0 || nrec > kMaxRec)
        return report(EWS_EINVAL, "%d receivers; the no-allocation limit is %d", nrec, kMaxRec);
    if (nrec > 0 && (!rec_pos || !seis)) return report(EWS_EINVAL, "receivers need positions and seis");
    if (src_kind != EWS_SOURCE_MOMENT && src_kind != EWS_SOURCE_FORCE)
        return report(EWS_EINVAL, "unknown source kind");
    if (!position_ok(gr, pos)) return report(EWS_EINVAL, "source outside the valid range");
    for (int r = 0; r < nrec; ++r)
        if (!position_ok(gr, rec_pos + 3 * r))
            return report(EWS_EINVAL, "receiver %d outside the valid range", r);
    if (!(dt > 0) || !std::isfinite(dt)) return report(EWS_EINVAL, "dt must be positive");
    for (int c = 0; c < (src_kind == EWS_SOURCE_MOMENT ? 6 : 3); ++c)
        if (!std::isfinite(comp[c])) return report(EWS_ENONFINITE, "source component not finite");

    float* base = nullptr;
    ews_status st = scratch_address(&base);
    if (st != EWS_OK) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    DevGrid g{};
    g.nx = gr.nx;
    g.ny = gr.ny;
    g.nz = gr.nz;
    g.pitch = pitch;
    g.plane = (long long)pitch * gr.ny;
    g.c1x = (float)(9.0 / 8.0 / gr.dx);
    g.c2x = (float)(-1.0 / 24.0 / gr.dx);
    g.c1y = (float)(9.0 / 8.0 / gr.dy);
    g.c2y = (float)(-1.0 / 24.0 / gr.dy);
    g.c1z = (float)(9.0 / 8.0 / gr.dz);
    g.c2z = (float)(-1.0 / 24.0 / gr.dz);
    g.fs = kNoSurface;
    g.c1z2 = (float)(1.0 / gr.dz);
    g.fs_eps = 0.0f;
    DevFields F;
    for (int q = 0; q < NFIELD; ++q) F.f[q] = base + kOffFields + fslot(q) * (size_t)kMaxCells;
    float* mlam = base + kOffMedium;
    float* mmu = mlam + kMaxCells;
    float* mrho = mmu + kMaxCells;
    DevMedium M{mlam, mmu, mrho};
    Tap* rtaps = reinterpret_cast<Tap*>(base + kOffTaps);
    unsigned* flags = reinterpret_cast<unsigned*>(base + kOffFlags);
    int* err = reinterpret_cast<int*>(base + kOffFlags + 8);

    // ---- medium: dense caller arrays -> pitched scratch, validate, vp_max ----
    const float* src[3] = {lam, mu, rho};
    float* dst[3] = {mlam, mmu, mrho};
    for (int a = 0; a < 3; ++a)
        NA_CK(cudaMemcpy2DAsync(dst[a], pitch * sizeof(float), src[a], gr.nx * sizeof(float),
                                gr.nx * sizeof(float), (size_t)gr.ny * gr.nz,
                                cudaMemcpyDeviceToDevice, stream));
    NA_CK(cudaMemsetAsync(flags, 0, 5 * sizeof(unsigned), stream));   // bounds 2..4 unused here
    NA_CK(launch_medium_setup(g, mlam, mmu, mrho, 0, flags, stream));
    unsigned hf[2] = {0, 0};
    NA_CK(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, stream));
    NA_CK(cudaStreamSynchronize(stream));
    if (hf[0] & 1u) return report(EWS_ENONFINITE, "model contains NaN or Inf");
    if (hf[0] & 14u) return report(EWS_EINVAL, "model has rho <= 0, mu < 0 or lambda + 2 mu <= 0");
    float vpmax;
    static_assert(sizeof(vpmax) == sizeof(hf[1]), "vp_max travels as float bits");
    std::memcpy(&vpmax, &hf[1], sizeof(vpmax));
    const double kk = std::sqrt(1.0 / (gr.dx * gr.dx) + 1.0 / (gr.dy * gr.dy) + 1.0 / (gr.dz * gr.dz));
    if (dt > 2.0 / ((7.0 / 3.0) * vpmax * kk) * (1.0 + 1e-12))
        return report(EWS_ECFL, "dt exceeds the stability bound");

    // ---- sponge profiles and receiver taps, computed here, copied in ----
    // One axis (and a chunk of receivers) at a time through small host
    // buffers: an asynchronous copy from pageable memory has staged its
    // source when it returns, so the buffer can be refilled at once.  The
    // C-PML rows (pa, pb) are unused by these passes and are zeroed.
    float prof[kMaxDim];
    const int n3[3] = {gr.nx, gr.ny, gr.nz};
    const double alpha = (opt && opt->sponge_alpha > 0) ? opt->sponge_alpha : 0.3;
    for (int a = 0; a < 3; ++a) {
        for (int i = 0; i < n3[a]; ++i) {
            float gval = 1.0f;
            const int d = i < n3[a] - 1 - i ? i : n3[a] - 1 - i;
            if (bnd == EWS_BOUNDARY_SPONGE && d < W) {
                const double x = alpha * (W - d) / W;
                gval = (float)std::exp(-x * x);
            }
            prof[i] = gval;
        }
        NA_CK(cudaMemcpyAsync(base + kOffProf + a * kMaxDim, prof, n3[a] * sizeof(float),
                              cudaMemcpyHostToDevice, stream));
    }
    NA_CK(cudaMemsetAsync(base + kOffProf + 3 * kMaxDim, 0, 6 * kMaxDim * sizeof(float), stream));
    constexpr int kRecChunk = 16;
    Tap taps[8 * kRecChunk];
    for (int c = 0; c < 3; ++c)
        for (int r0 = 0; r0 < nrec; r0 += kRecChunk) {
            const int nr = nrec - r0 < kRecChunk ? nrec - r0 : kRecChunk;
            for (int r = 0; r < nr; ++r)
                point_taps(gr, VX + c, rec_pos + 3 * (r0 + r), 1.0, &taps[8 * r]);
            NA_CK(cudaMemcpyAsync(rtaps + 8 * (c * nrec + r0), taps, sizeof(Tap) * 8 * nr,
                                  cudaMemcpyHostToDevice, stream));
        }
    DevBoundary B{};
    B.kind = bnd == EWS_BOUNDARY_SPONGE ? BND_SPONGE : BND_NONE;
    B.W = W;
    for (int a = 0; a < 3; ++a) {
        B.g[a] = base + kOffProf + a * kMaxDim;
        B.pa[a] = base + kOffProf + (3 + a) * kMaxDim;
        B.pb[a] = base + kOffProf + (6 + a) * kMaxDim;
    }
    DevSource S{};
    S.kind = src_kind;
    S.ntap = 0;
    const double vol = gr.dx * gr.dy * gr.dz;
    const int nc = src_kind == EWS_SOURCE_MOMENT ? 6 : 3;
    for (int c = 0; c < nc; ++c) {
        if (comp[c] == 0.0) continue;
        if (src_kind == EWS_SOURCE_MOMENT)
            point_taps(gr, SXX + c, pos, -dt * comp[c] / vol, &S.tap[S.ntap]);
        else
            point_taps(gr, VX + c, pos, dt * comp[c] / vol, &S.tap[S.ntap]);
        S.ntap += 8;
    }

    // ---- state starts at zero; the plan is built in thread-local storage ----
    NA_CK(cudaMemsetAsync(base + kOffFields, 0, 9 * (size_t)kMaxCells * sizeof(float), stream));
    NA_CK(cudaMemsetAsync(err, 0, sizeof(int), stream));
    // The plan (tensor maps, launch geometry) only has to live until the
    // launches below have taken their parameters: thread-local host storage.
    alignas(64) static thread_local unsigned char plan_buf[16384];
    if (stencil_plan_bytes() > sizeof(plan_buf)) {
        (void)cudaStreamSynchronize(stream);
        return report(EWS_ECUDA, "plan storage too small");
    }
    StencilPlan* plan = nullptr;
    NA_CK(stencil_plan_fill(plan_buf, g, F, M, B, &plan));

    // ---- Sec. 2.3 loop ----
    float dto[NFIELD], inv[NFIELD];
    for (int q = 0; q < NFIELD; ++q) {
        dto[q] = (float)dt;
        inv[q] = 1.0f;
    }
    const int f32 = EWS_STORAGE_F32;
    for (int n = 0; n < nt; ++n) {
        NA_CK(launch_velocity(plan, g, F, B, dto, inv, err, stream));
        if (src_kind == EWS_SOURCE_FORCE) NA_CK(launch_inject(g, F, M, B, S, wavelet, n, f32, err, stream));
        if (nrec > 0) NA_CK(launch_record(g, F, rtaps, nrec, seis, nt, n, f32, inv, err, stream));
        NA_CK(launch_stress(plan, g, F, B, dto, inv, err, stream));
        if (src_kind == EWS_SOURCE_MOMENT) NA_CK(launch_inject(g, F, M, B, S, wavelet, n, f32, err, stream));
    }
    int herr = 0;
    NA_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    NA_CK(cudaStreamSynchronize(stream));
    if (herr & 3) return report(EWS_ETIMEOUT, "a pipeline wait in the stencil kernels gave up");
    if (herr) return report(EWS_ENONFINITE, "a receiver recorded NaN or Inf");
    return EWS_OK;
}
