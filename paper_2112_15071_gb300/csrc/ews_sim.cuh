// ews_sim.cuh -- the simulation object behind the opaque ews_sim handle,
// shared by the C ABI (ews_capi.cu) and the batched executor's host side
// (ews_batch.cu).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/ews.h"
#include "ews_internal.cuh"

namespace ews {

// Host-side description of the point source (taps are rebuilt per dt).
struct SourceSpec {
    int kind = -1;
    double pos[3] = {0, 0, 0};
    double comp[6] = {0, 0, 0, 0, 0, 0};
};

// One captured time loop: a CUDA graph of steps n0 .. n0 + nsteps - 1 with
// everything its kernel parameters depend on as the key.
struct GraphEntry {
    unsigned long long gen;
    int n0, nsteps, ld;
    double dt;
    const float* dseis;
    const float* vcap;
    cudaGraphExec_t exec;
    long long launches[EWS_NKERNEL];
};

}  // namespace ews

using namespace ews;   // internal header: the object's members use ews types

struct ews_sim {
    using SourceSpec = ews::SourceSpec;
    using GraphEntry = ews::GraphEntry;
    ews_grid grid{};
    ews_options opt{};
    DevGrid g{};
    size_t fstride = 0;           // elements between fields (and medium arrays)
    int es = 4;                   // bytes per stored wavefield element
    float* fields = nullptr;      // 9 * fstride elements of the storage type
    float* medium = nullptr;      // 3 * fstride floats: lambda, mu, rho
    float* cmed = nullptr;        // coarse medium grid: lambda, mu, rho, dense [mz][my][mx]
    bool model_set = false;
    float vpmax = 0.0f;
    float rho_min = 0.0f, zs_min = 0.0f, zp_max = 0.0f;   // medium bounds
    double fs_eps = 0.0;          // vacuum fraction above the free surface (g.fs)
    bool has_fluid = false;       // some cell has mu == 0
    // per-field storage scales (16-bit storage holds scale[q] x value)
    float scale[NFIELD] = {1, 1, 1, 1, 1, 1, 1, 1, 1};
    bool scale_user = false;      // set by ews_set_field_scales
    bool fresh = true;            // wavefields are all zero
    float* stage = nullptr;       // dense float32 staging for 16-bit state I/O
    size_t stage_cap = 0;
    // boundary
    float* prof = nullptr;        // g[3][n], pa[3][n], pb[3][n] packed
    float* psi = nullptr;         // C-PML memory variables
    size_t psi_floats = 0;
    DevBoundary B{};
    double pml_dt = -1.0;
    // source
    SourceSpec src;
    double wsum = 0;              // sum of |wavelet|
    DevSource S{};
    float* wavelet = nullptr;
    int wavelet_nt = 0;
    // receivers
    int nrec = 0;
    Tap* rtaps = nullptr;         // [3 * nrec][8]
    float* seis_buf = nullptr;    // internal [3][nrec][cap] when caller is on host
    size_t seis_cap = 0;
    unsigned* flags = nullptr;    // device scratch for medium checks
    int* err = nullptr;           // device flag: bounded waits that gave up
    StencilPlan* plan = nullptr;
    // tile shape of the forward passes of plain steps (EWS_TILE_*): asked for,
    // and in use; plans of the other shapes, created on first use
    int tile_req = EWS_TILE_AUTO;
    int tile_used = EWS_TILE_32X8;
    void* tplan[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    // second set of wavefields of the fused step (9 * fstride floats, laid
    // out like `fields`), held with its plan
    float* fields2 = nullptr;
    cudaStream_t stream = nullptr;
    // launch accounting and optional per-launch event timing
    long long launches[EWS_NKERNEL] = {};
    double kernel_ms[EWS_NKERNEL] = {};
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;     // reused across calls
    std::vector<int> ev_class;            // class of the launch ending at event m
    size_t ev_used = 0;
    // adjoint buffers (allocated on first use)
    float* adj = nullptr;                 // P (3), Q (6), FP32 accumulators (8)
    double* acc64 = nullptr;              // FP64 accumulators (8)
    float* ckpt = nullptr;                // checkpoints, nck x 9 fields (FP32 or 16-bit)
    size_t ckpt_cap = 0;                  // fields' worth of floats
    int ckpt_storage = EWS_STORAGE_F32;   // element type of the checkpoints held now
    int ckpt_pref = EWS_STORAGE_F32;      // type ews_adjoint / ews_gradient use
    float* ckpt_scale = nullptr;          // 16-bit checkpoints: [nck][9] field scales
    unsigned* ckpt_amax = nullptr;        // [9] absolute maxima of the state being saved
    int ckpt_scale_cap = 0;
    float* vhist = nullptr;               // velocity history, (K + 1) x 3 fields
    size_t vhist_cap = 0;
    float* aux = nullptr;                 // seismogram-sized adjoint source + observed
    size_t aux_cap = 0;
    float* gout = nullptr;                // gradient staging for host outputs
    double* dmisfit = nullptr;
    double hist_budget = -1;              // bytes of resident velocity history (< 0: auto)
    // captured time loops (used when per-launch profiling is off)
    std::vector<GraphEntry> graphs;
    unsigned long long gen = 1;           // bumped when a kernel parameter source changes
    cudaStream_t cap_stream = nullptr;    // private stream the loops are captured on
    StencilPlan* adj_plan = nullptr;      // stencil plan of the adjoint fields
    const float* adj_hist = nullptr;      // history buffer the plan's map points at
    int adj_hist_slots = 0;

    void* field(int q) const { return (char*)fields + (size_t)fslot(q) * fstride * es; }
    DevFields F() const {
        DevFields f;
        for (int q = 0; q < NFIELD; ++q) f.f[q] = (float*)field(q);
        return f;
    }
    DevFields F2() const {
        DevFields f;
        for (int q = 0; q < NFIELD; ++q) f.f[q] = fields2 + (size_t)fslot(q) * fstride;
        return f;
    }
    bool wide() const { return opt.storage == EWS_STORAGE_F32; }
    DevMedium M() const {          // null while a coarse medium grid replaces it
        DevMedium m;
        m.lam = medium;
        m.mu = medium ? medium + fstride : nullptr;
        m.rho = medium ? medium + 2 * fstride : nullptr;
        return m;
    }
    long long ncell() const { return (long long)grid.nx * grid.ny * grid.nz; }
};


namespace ews {

// Helpers of ews_capi.cu used by the batched executor.  They record an
// error message (ews_last_error) and return its status on failure.
ews_status sim_ready(ews_sim* s, int n_end, double dt);        // model, dt, boundary profiles
DevSource sim_source(const ews_sim* s, double dt);             // source taps for this dt
// Adjoint buffers for nt steps with `nckpt` checkpoints and `hslots`
// history slots (allocated once, grown when needed).
ews_status sim_adjoint_buffers(ews_sim* s, int nt, int nckpt, int hslots, bool with_obs,
                               int ckpt_storage = EWS_STORAGE_F32);
// Stencil plan of the adjoint fields with its history map on s->vhist.
ews_status sim_adjoint_plan(ews_sim* s);
// History budget in bytes: the set value, or (automatic) `share` of the
// device memory free now plus what the history buffer already holds.
double sim_history_budget(const ews_sim* s, double share);

}  // namespace ews
