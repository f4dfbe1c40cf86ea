// ews_capi.cu -- C ABI of libews: simulation object, validation, device
// memory, and the time loop of Sec. 2.3 (velocity pass, receivers, stress
// pass each step).  Declarations and the contract of every call are in
// include/ews.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/ews.h"
#include "ews_internal.cuh"
#include "ews_sim.cuh"

using namespace ews;

namespace {

thread_local char g_err[512] = "";

// A failed device allocation leaves its (non-sticky) error for
// cudaGetLastError; take it so that a later call's error check does not
// report it as its own (a refusal by the library's memory limit leaves
// none, and an unrelated pending error is left alone).  With a limit set,
// the message says so.
void enomem_tail(ews_status s) {
    if (s != EWS_ENOMEM) return;
    if (cudaPeekAtLastError() == cudaErrorMemoryAllocation) (void)cudaGetLastError();
    const double lim = ews_memory_limit();
    if (lim >= 0) {
        const size_t n = strlen(g_err);
        snprintf(g_err + n, sizeof(g_err) - n, " [libews memory limit %.0f bytes, %.0f in use]",
                 lim, ews_memory_in_use());
    }
}

ews_status fail(ews_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    enomem_tail(s);
    return s;
}

#define CK(call)                                                                     \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return fail(e_ == cudaErrorMemoryAllocation ? EWS_ENOMEM : EWS_ECUDA,    \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,   \
                        __LINE__);                                                   \
    } while (0)

// Eq. 4 weights.
constexpr double kC1 = 9.0 / 8.0;
constexpr double kC2 = -1.0 / 24.0;

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// ---- tile shapes of the forward passes ----
// Plain forward steps (no free surface, no coarse medium grid, no history
// capture) may run the passes of another tile shape; the others use 32 x 8.
bool tile_eligible(const ews_sim* s) { return s->g.fs == kNoSurface && !s->g.cm[0]; }

// The fused step serves FP32 storage at unit scales, sponge or no boundary.
bool fused_eligible(const ews_sim* s) {
    if (!tile_eligible(s) || !fused::fused_supported(s->g, s->B, s->opt.storage)) return false;
    for (int q = 0; q < NFIELD; ++q)
        if (s->scale[q] != 1.0f) return false;
    return true;
}

// Shape of the forward passes of a plain (vcap null) or capturing step.
int fwd_shape(const ews_sim* s, bool capture) {
    if (capture || !tile_eligible(s)) return EWS_TILE_32X8;
    if (s->tile_used == EWS_TILE_FUSED && !fused_eligible(s)) return EWS_TILE_32X8;
    return s->tile_used;
}

void drop_fused(ews_sim* s) {
    fused::fused_plan_destroy(static_cast<fused::FusedPlan*>(s->tplan[EWS_TILE_FUSED]));
    s->tplan[EWS_TILE_FUSED] = nullptr;
    dev_free(s->fields2);
    s->fields2 = nullptr;
}

void drop_tile_plans(ews_sim* s) {
    t32x4::stencil_plan_destroy(static_cast<t32x4::StencilPlan*>(s->tplan[EWS_TILE_32X4]));
    t32x16::stencil_plan_destroy(static_cast<t32x16::StencilPlan*>(s->tplan[EWS_TILE_32X16]));
    s->tplan[EWS_TILE_32X4] = s->tplan[EWS_TILE_32X16] = nullptr;
    drop_fused(s);
}

ews_status tile_plan(ews_sim* s, int shape) {
    if (shape == EWS_TILE_32X8 || s->tplan[shape]) return EWS_OK;
    if (shape == EWS_TILE_FUSED) {
        const size_t bytes = (size_t)NFIELD * s->fstride * sizeof(float);
        cudaError_t e = dev_malloc((void**)&s->fields2, bytes);
        if (e != cudaSuccess) {
            s->fields2 = nullptr;
            return fail(EWS_ENOMEM, "second wavefield set of the fused step (%zu bytes): %s", bytes,
                        cudaGetErrorString(e));
        }
        fused::FusedPlan* p = nullptr;
        e = cudaMemsetAsync(s->fields2, 0, bytes, s->stream);
        if (e == cudaSuccess) e = fused::fused_plan_create(s->g, s->F(), s->F2(), s->M(), s->B, &p);
        if (e != cudaSuccess) {
            dev_free(s->fields2);
            s->fields2 = nullptr;
            return fail(EWS_ECUDA, "fused step plan: %s", cudaGetErrorString(e));
        }
        s->tplan[shape] = p;
        return EWS_OK;
    }
    if (shape == EWS_TILE_32X4) {
        t32x4::StencilPlan* p = nullptr;
        CK(t32x4::stencil_plan_create(s->g, s->F(), s->M(), s->B, s->opt.storage, &p));
        s->tplan[shape] = p;
    } else {
        t32x16::StencilPlan* p = nullptr;
        CK(t32x16::stencil_plan_create(s->g, s->F(), s->M(), s->B, s->opt.storage, &p));
        s->tplan[shape] = p;
    }
    return EWS_OK;
}


}  // namespace

namespace ews {
// Record an error message for ews_last_error() from other translation units.
ews_status report(ews_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    enomem_tail(s);                                    // as in fail()
    return s;
}
}  // namespace ews

namespace {

ews_status check_pos(const ews_sim* s, const double p[3], const char* what) {
    const int n[3] = {s->grid.nx, s->grid.ny, s->grid.nz};
    const double h[3] = {s->grid.dx, s->grid.dy, s->grid.dz};
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(p[a]) || p[a] < h[a] * (1.0 - 1e-12) ||
            p[a] > (n[a] - 2) * h[a] * (1.0 + 1e-12))
            return fail(EWS_EINVAL, "%s position %g on axis %d outside [%g, %g]", what, p[a],
                        a, h[a], (n[a] - 2) * h[a]);
    }
    return EWS_OK;
}

// Trilinear taps of point p on the grid of field q (offsets of Sec. 2.1.1).
void taps_for(const ews_sim* s, int q, const double p[3], double scale, Tap out[8]) {
    static const double off[NFIELD][3] = {{0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5},
                                          {0, 0, 0},   {0, 0, 0},   {0, 0, 0},
                                          {0.5, 0.5, 0}, {0.5, 0, 0.5}, {0, 0.5, 0.5}};
    const double h[3] = {s->grid.dx, s->grid.dy, s->grid.dz};
    const int n[3] = {s->grid.nx, s->grid.ny, s->grid.nz};
    int i0[3];
    double fr[3];
    for (int a = 0; a < 3; ++a) {
        double u = p[a] / h[a] - off[q][a];
        double fl = std::floor(u);
        i0[a] = (int)fl;
        fr[a] = u - fl;
        if (i0[a] >= n[a] - 1) {  // exactly on the last point: weight 1 there
            i0[a] = n[a] - 2;
            fr[a] = 1.0;
        }
    }
    int m = 0;
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di, ++m) {
                double w = (di ? fr[0] : 1 - fr[0]) * (dj ? fr[1] : 1 - fr[1]) *
                           (dk ? fr[2] : 1 - fr[2]);
                out[m].q = q;
                out[m].i = i0[0] + di;
                out[m].j = i0[1] + dj;
                out[m].k = i0[2] + dk;
                out[m].w = (float)(w * scale);
            }
}

// Sponge profiles and C-PML coefficients for the current dt.
ews_status upload_boundary(ews_sim* s, double dt) {
    const int n[3] = {s->grid.nx, s->grid.ny, s->grid.nz};
    const double h[3] = {s->grid.dx, s->grid.dy, s->grid.dz};
    const int W = s->opt.width;
    const int nmax = std::max(n[0], std::max(n[1], n[2]));
    std::vector<float> host(9 * (size_t)nmax, 0.0f);
    const double alpha = s->opt.sponge_alpha > 0 ? s->opt.sponge_alpha : 0.3;
    const double R = s->opt.pml_R > 0 ? s->opt.pml_R : 1e-3;
    for (int a = 0; a < 3; ++a) {
        float* g = &host[(0 * 3 + a) * (size_t)nmax];
        float* pa = &host[(1 * 3 + a) * (size_t)nmax];
        float* pb = &host[(2 * 3 + a) * (size_t)nmax];
        for (int i = 0; i < n[a]; ++i) {
            g[i] = 1.0f;
            int d = std::min(i, n[a] - 1 - i);
            if (s->opt.boundary == EWS_BOUNDARY_SPONGE && d < W) {
                double x = alpha * (W - d) / W;
                g[i] = (float)std::exp(-x * x);
            }
            if (s->opt.boundary == EWS_BOUNDARY_CPML && (i < W || i >= n[a] - W)) {
                double q = i < W ? double(W - i) / W : double(i - (n[a] - 1 - W)) / W;
                double d0 = -3.0 * s->vpmax * std::log(R) / (2.0 * W * h[a]);
                double dd = d0 * q * q;
                double al = M_PI * s->opt.pml_f0 * (1.0 - q);
                double b = std::exp(-(dd + al) * dt);
                pb[i] = (float)b;
                pa[i] = (float)((dd + al) > 0 ? dd * (b - 1.0) / (dd + al) : 0.0);
            }
        }
    }
    CK(cudaMemcpyAsync(s->prof, host.data(), host.size() * sizeof(float),
                       cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    for (int a = 0; a < 3; ++a) {
        s->B.g[a] = s->prof + (0 * 3 + a) * (size_t)nmax;
        s->B.pa[a] = s->prof + (1 * 3 + a) * (size_t)nmax;
        s->B.pb[a] = s->prof + (2 * 3 + a) * (size_t)nmax;
    }
    s->pml_dt = dt;
    return EWS_OK;
}

ews_status copy_field_in(ews_sim* s, float* dst, const float* src, int on_device) {
    const ews_grid& gr = s->grid;
    CK(cudaMemcpy2DAsync(dst, s->g.pitch * sizeof(float), src, gr.nx * sizeof(float),
                         gr.nx * sizeof(float), (size_t)gr.ny * gr.nz,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                         s->stream));
    return EWS_OK;
}

ews_status copy_field_out(ews_sim* s, float* dst, const float* src, int on_device) {
    const ews_grid& gr = s->grid;
    CK(cudaMemcpy2DAsync(dst, gr.nx * sizeof(float), src, s->g.pitch * sizeof(float),
                         gr.nx * sizeof(float), (size_t)gr.ny * gr.nz,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                         s->stream));
    return EWS_OK;
}

template <typename T>
ews_status ensure_buf(T** buf, size_t* cap, size_t need, const char* what);

// Wavefield q to / from a dense float32 [nz][ny][nx] array (host or device),
// converting 16-bit storage with the field's scale.
ews_status field_out(ews_sim* s, int q, float* dst, int on_device) {
    if (s->wide()) return copy_field_out(s, dst, (const float*)s->field(q), on_device);
    float* d = dst;
    if (!on_device) {
        ews_status st = ensure_buf(&s->stage, &s->stage_cap, (size_t)s->ncell(), "staging");
        if (st != EWS_OK) return st;
        d = s->stage;
    }
    CK(launch_field_out(s->g, s->field(q), s->opt.storage, 1.0f / s->scale[q], d, s->stream));
    if (!on_device)
        CK(cudaMemcpyAsync(dst, d, (size_t)s->ncell() * sizeof(float), cudaMemcpyDeviceToHost,
                           s->stream));
    if (!on_device) CK(cudaStreamSynchronize(s->stream));   // the staging buffer is reused
    return EWS_OK;
}

ews_status field_in(ews_sim* s, int q, const float* src, int on_device) {
    if (s->wide()) return copy_field_in(s, (float*)s->field(q), src, on_device);
    const float* d = src;
    if (!on_device) {
        ews_status st = ensure_buf(&s->stage, &s->stage_cap, (size_t)s->ncell(), "staging");
        if (st != EWS_OK) return st;
        CK(cudaMemcpyAsync(s->stage, src, (size_t)s->ncell() * sizeof(float),
                           cudaMemcpyHostToDevice, s->stream));
        d = s->stage;
    }
    CK(launch_field_in(s->g, d, s->opt.storage, s->scale[q], s->field(q), s->err, s->stream));
    if (!on_device) CK(cudaStreamSynchronize(s->stream));
    return EWS_OK;
}

ews_status set_model(ews_sim* s, const float* a, const float* b, const float* rho,
                     int on_device, int from_vel) {
    if (!s) return fail(EWS_EINVAL, "null simulation");
    if (!a || !b || !rho) return fail(EWS_EINVAL, "null model array");
    if (s->g.cm[0]) {                          // back from a coarse medium grid
        for (int q = 0; q < 3; ++q) s->g.cm[q] = nullptr;
        s->gen++;
    }
    if (!s->medium) {                          // released while a coarse grid was in use
        s->model_set = false;
        CK(dev_malloc((void**)&s->medium, 3 * s->fstride * sizeof(float)));
        CK(cudaMemsetAsync(s->medium, 0, 3 * s->fstride * sizeof(float), s->stream));
        StencilPlan* np = nullptr;
        CK(stencil_plan_create(s->g, s->F(), s->M(), s->B, s->opt.storage, &np));
        stencil_plan_destroy(s->plan);
        s->plan = np;
        drop_tile_plans(s);
        s->gen++;
    }
    DevMedium M = s->M();
    ews_status st;
    if ((st = copy_field_in(s, (float*)M.lam, a, on_device)) != EWS_OK) return st;
    if ((st = copy_field_in(s, (float*)M.mu, b, on_device)) != EWS_OK) return st;
    if ((st = copy_field_in(s, (float*)M.rho, rho, on_device)) != EWS_OK) return st;
    CK(launch_vacuum(s->g, (float*)M.lam, (float*)M.mu, (float*)M.rho, from_vel,
                     (float)s->fs_eps, s->stream));
    CK(cudaMemsetAsync(s->flags, 0, 5 * sizeof(unsigned), s->stream));
    CK(cudaMemsetAsync(s->flags + 2, 0x7F, 2 * sizeof(unsigned), s->stream));   // min slots: 3.4e38
    CK(launch_medium_setup(s->g, (float*)M.lam, (float*)M.mu, (float*)M.rho, from_vel,
                           s->flags, s->stream));
    unsigned hf[5];
    CK(cudaMemcpyAsync(hf, s->flags, sizeof(hf), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->model_set = false;
    if (hf[0] & 1u) return fail(EWS_ENONFINITE, "model contains NaN or Inf");
    if (hf[0] & 2u) return fail(EWS_EINVAL, "model has rho <= 0");
    if (hf[0] & 4u) return fail(EWS_EINVAL, "model has mu < 0 (vs^2 < 0)");
    if (hf[0] & 8u) return fail(EWS_EINVAL, "model has lambda + 2 mu <= 0");
    float bnd[4];
    std::memcpy(bnd, &hf[1], sizeof(bnd));
    s->vpmax = bnd[0];
    s->rho_min = bnd[1];
    s->zs_min = bnd[2];
    s->zp_max = bnd[3];
    s->has_fluid = (hf[0] & 16u) != 0;
    s->model_set = true;
    s->pml_dt = -1.0;
    return EWS_OK;
}

ews_status check_dt(const ews_sim* s, double dt) {
    if (!(dt > 0) || !std::isfinite(dt)) return fail(EWS_EINVAL, "dt must be positive");
    const ews_grid& g = s->grid;
    double k = std::sqrt(1.0 / (g.dx * g.dx) + 1.0 / (g.dy * g.dy) + 1.0 / (g.dz * g.dz));
    double lim = 2.0 / ((7.0 / 3.0) * s->vpmax * k);
    if (dt > lim * (1.0 + 1e-12))
        return fail(EWS_ECFL, "dt = %g exceeds the stability bound %g (vp_max = %g)", dt, lim,
                    (double)s->vpmax);
    return EWS_OK;
}

ews_status ensure_ready(ews_sim* s, int n_end, double dt) {
    if (!s) return fail(EWS_EINVAL, "null simulation");
    if (!s->model_set) return fail(EWS_ESTATE, "ews_set_model_* has not succeeded");
    ews_status st = check_dt(s, dt);
    if (st != EWS_OK) return st;
    if (s->S.kind >= 0 && n_end > s->wavelet_nt)
        return fail(EWS_EINVAL, "steps up to %d exceed the wavelet length %d", n_end,
                    s->wavelet_nt);
    if (s->pml_dt != dt && (st = upload_boundary(s, dt)) != EWS_OK) return st;
    return EWS_OK;
}

// Account one launch of class cls (or open a bracket when cls < 0); with
// profiling on, record an event after it on the simulation's stream.
ews_status mark(ews_sim* s, int cls) {
    if (cls >= 0) s->launches[cls] += 1;
    if (!s->profiling) return EWS_OK;
    if (s->ev_used == s->ev_pool.size()) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        s->ev_pool.push_back(e);
        s->ev_class.push_back(-1);
    }
    s->ev_class[s->ev_used] = cls;
    CK(cudaEventRecord(s->ev_pool[s->ev_used], s->stream));
    ++s->ev_used;
    return EWS_OK;
}

// Power of two at or below x (x > 0, finite).
float pow2_floor(double x) {
    int e;
    std::frexp(x, &e);
    return (float)std::ldexp(1.0, e - 1);
}

// Default per-field scales of FP16 storage (Sec. 2.4 source terms): the
// amplitude the source can put into one cell, summed over the whole
// wavelet, bounds the field it drives; the other field group follows
// through the impedance relation |sigma| = Z |v| of a plane wave (smallest
// impedance for v, largest for sigma).  Each scale maps its bound to 2^13,
// 8x below the FP16 maximum; kernels flag any stored value beyond it.
void auto_scales(ews_sim* s, double dt) {
    if (s->opt.storage != EWS_STORAGE_F16 || s->scale_user) return;
    const double vol = s->grid.dx * s->grid.dy * s->grid.dz;
    const double zs = (s->zs_min > 0 && s->zs_min < 1e38f) ? s->zs_min : s->zp_max;
    double vb = 0, sb = 0;
    if (s->src.kind >= 0 && s->wsum > 0) {
        double cmax = 0;
        for (int c = 0; c < 6; ++c) cmax = std::max(cmax, std::fabs(s->src.comp[c]));
        const double inj = cmax * dt * s->wsum / vol;
        if (s->src.kind == EWS_SOURCE_MOMENT) {
            sb = inj;
            vb = zs > 0 ? sb / zs : 0;
        } else {
            vb = s->rho_min > 0 ? inj / s->rho_min : 0;
            sb = vb * s->zp_max;
        }
    }
    for (int q = 0; q < NFIELD; ++q) {
        const double bound = q < 3 ? vb : sb;
        double sc = (bound > 0 && std::isfinite(bound)) ? 8192.0 / bound : 1.0;
        sc = std::min(std::max(sc, 0x1p-100), 0x1p100);
        const float v = pow2_floor(sc);
        if (v != s->scale[q]) s->gen++;
        s->scale[q] = v;
    }
}

// Source taps for this dt: dt, the cell volume and the field scale folded
// into the trilinear weights (Sec. 2.4 reading).
DevSource source_taps(const ews_sim* s, const SourceSpec& src, double dt) {
    DevSource S{};
    S.kind = -1;
    if (src.kind >= 0 && s->wavelet) {
        const double vol = s->grid.dx * s->grid.dy * s->grid.dz;
        S.kind = src.kind;
        S.ntap = 0;
        if (src.kind == EWS_SOURCE_MOMENT) {
            for (int c = 0; c < 6; ++c) {
                if (src.comp[c] == 0.0) continue;
                taps_for(s, SXX + c, src.pos, -dt * src.comp[c] / vol * s->scale[SXX + c],
                         &S.tap[S.ntap]);
                S.ntap += 8;
            }
        } else {
            for (int c = 0; c < 3; ++c) {
                if (src.comp[c] == 0.0) continue;
                taps_for(s, VX + c, src.pos, dt * src.comp[c] / vol * s->scale[VX + c],
                         &S.tap[S.ntap]);
                S.ntap += 8;
            }
        }
    }
    return S;
}

cudaError_t vel_launch(ews_sim* s, int shape, const DevFields& F, const float dto[9],
                       const float inv[9]) {
    switch (shape) {
        case EWS_TILE_32X4:
            return t32x4::launch_velocity(static_cast<t32x4::StencilPlan*>(s->tplan[shape]), s->g, F,
                                          s->B, dto, inv, s->err, s->stream);
        case EWS_TILE_32X16:
            return t32x16::launch_velocity(static_cast<t32x16::StencilPlan*>(s->tplan[shape]), s->g,
                                           F, s->B, dto, inv, s->err, s->stream);
        default:
            return launch_velocity(s->plan, s->g, F, s->B, dto, inv, s->err, s->stream);
    }
}

cudaError_t str_launch(ews_sim* s, int shape, const DevFields& F, const float dto[9],
                       const float inv[9]) {
    switch (shape) {
        case EWS_TILE_32X4:
            return t32x4::launch_stress(static_cast<t32x4::StencilPlan*>(s->tplan[shape]), s->g, F,
                                        s->B, dto, inv, s->err, s->stream);
        case EWS_TILE_32X16:
            return t32x16::launch_stress(static_cast<t32x16::StencilPlan*>(s->tplan[shape]), s->g,
                                         F, s->B, dto, inv, s->err, s->stream);
        default:
            return launch_stress(s->plan, s->g, F, s->B, dto, inv, s->err, s->stream);
    }
}

// Steps n0 .. n0 + nsteps - 1 with the fused step: step n0 + m reads the
// wavefield set it wrote in step n0 + m - 1 (the simulation's own set at
// m = 0) and writes the other; receivers and a moment source run on the set
// just written, as after the two passes.  An odd step count ends with the
// state copied back into the simulation's own set.
ews_status steps_fused(ews_sim* s, const SourceSpec& src, int n0, int nsteps, double dt,
                       float* dseis, int ld) {
    const fused::FusedPlan* fp = static_cast<const fused::FusedPlan*>(s->tplan[EWS_TILE_FUSED]);
    DevMedium M = s->M();
    const DevSource S = source_taps(s, src, dt);
    const DevFields set[2] = {s->F(), s->F2()};
    const float inv[NFIELD] = {1, 1, 1, 1, 1, 1, 1, 1, 1};
    const int stor = s->opt.storage;
    s->fresh = false;
    ews_status st;
    if ((st = mark(s, -1)) != EWS_OK) return st;
    for (int n = n0; n < n0 + nsteps; ++n) {
        const int dir = (n - n0) & 1;
        const DevFields& out = set[dir ^ 1];
        CK(fused::launch_fused(fp, dir, s->g, M, s->B, (float)dt, S, s->wavelet, n, s->err,
                               s->stream));
        if ((st = mark(s, EWS_KERNEL_STEP)) != EWS_OK) return st;
        const bool rec = s->nrec > 0 && dseis;
        if (S.kind == EWS_SOURCE_MOMENT && rec) {
            CK(launch_post_stress(s->g, out, M, s->B, S, s->wavelet, s->rtaps, s->nrec, dseis, ld, n,
                                  stor, inv, s->err, s->stream));
            if ((st = mark(s, EWS_KERNEL_POINTS)) != EWS_OK) return st;
        } else {
            if (rec) {
                CK(launch_record(s->g, out, s->rtaps, s->nrec, dseis, ld, n, stor, inv, s->err,
                                 s->stream));
                if ((st = mark(s, EWS_KERNEL_RECORD)) != EWS_OK) return st;
            }
            if (S.kind == EWS_SOURCE_MOMENT) {
                CK(launch_inject(s->g, out, M, s->B, S, s->wavelet, n, stor, s->err, s->stream));
                if ((st = mark(s, EWS_KERNEL_INJECT)) != EWS_OK) return st;
            }
        }
    }
    if (nsteps & 1)
        CK(cudaMemcpyAsync(s->fields, s->fields2, (size_t)NFIELD * s->fstride * sizeof(float),
                           cudaMemcpyDeviceToDevice, s->stream));
    return EWS_OK;
}

ews_status steps_direct(ews_sim* s, const SourceSpec& src, int n0, int nsteps, double dt,
                        float* dseis, int ld, float* vcap) {
    const int shape = fwd_shape(s, vcap != nullptr);
    ews_status st0 = tile_plan(s, shape);
    if (st0 != EWS_OK) return st0;
    if (shape == EWS_TILE_FUSED) return steps_fused(s, src, n0, nsteps, dt, dseis, ld);
    DevFields F = s->F();
    DevMedium M = s->M();
    const DevSource S = source_taps(s, src, dt);
    // dt x scale of each output field, 1 / scale of each input field
    float dto[NFIELD], inv[NFIELD];
    for (int q = 0; q < NFIELD; ++q) {
        dto[q] = (float)(dt * s->scale[q]);
        inv[q] = 1.0f / s->scale[q];
    }
    const int stor = s->opt.storage;
    s->fresh = false;
    ews_status st;
    if ((st = mark(s, -1)) != EWS_OK) return st;
    for (int n = n0; n < n0 + nsteps; ++n) {
        if (vcap) {   // v^{n+1/2} also into the history slot of step n
            VelExtra X{};
            X.vcap = vcap + (size_t)(n - n0 + 1) * 3 * s->fstride;
            X.fstride = (long long)s->fstride;
            CK(launch_velocity_cap(s->plan, s->g, F, s->B, dto, X, s->err, s->stream));
        } else {
            CK(vel_launch(s, shape, F, dto, inv));
        }
        if ((st = mark(s, EWS_KERNEL_VELOCITY)) != EWS_OK) return st;
        if (S.kind == EWS_SOURCE_FORCE) {
            CK(launch_inject(s->g, F, M, s->B, S, s->wavelet, n, stor, s->err, s->stream));
            if ((st = mark(s, EWS_KERNEL_INJECT)) != EWS_OK) return st;
            if (vcap) {   // the captured v^{n+1/2} includes the force term too
                DevFields H = F;
                for (int c = 0; c < 3; ++c)
                    H.f[c] = vcap + (size_t)(n - n0 + 1) * 3 * s->fstride + c * s->fstride;
                CK(launch_inject(s->g, H, M, s->B, S, s->wavelet, n, stor, s->err, s->stream));
            }
        }
        // receivers sample v^{n+1/2}: before the stress pass, or after it
        // together with the moment source (the stress pass leaves v alone)
        const bool rec = s->nrec > 0 && dseis;
        const bool fuse = rec && S.kind == EWS_SOURCE_MOMENT;
        if (rec && !fuse) {
            CK(launch_record(s->g, F, s->rtaps, s->nrec, dseis, ld, n, stor, inv, s->err, s->stream));
            if ((st = mark(s, EWS_KERNEL_RECORD)) != EWS_OK) return st;
        }
        CK(str_launch(s, shape, F, dto, inv));
        if ((st = mark(s, EWS_KERNEL_STRESS)) != EWS_OK) return st;
        if (fuse) {
            CK(launch_post_stress(s->g, F, M, s->B, S, s->wavelet, s->rtaps, s->nrec, dseis, ld, n,
                                  stor, inv, s->err, s->stream));
            if ((st = mark(s, EWS_KERNEL_POINTS)) != EWS_OK) return st;
        } else if (S.kind == EWS_SOURCE_MOMENT) {
            CK(launch_inject(s->g, F, M, s->B, S, s->wavelet, n, stor, s->err, s->stream));
            if ((st = mark(s, EWS_KERNEL_INJECT)) != EWS_OK) return st;
        }
    }
    return EWS_OK;
}

// The time loop of steps_direct, captured once into a CUDA graph per
// (state generation, step range, dt, output buffers) and replayed: one
// graph launch per call instead of 4-5 kernel launches per step.  With
// per-launch profiling on, the launches go out directly (events between
// them).
ews_status steps(ews_sim* s, const SourceSpec& src, int n0, int nsteps, double dt,
                 float* dseis, int ld, float* vcap = nullptr) {
    if (s->profiling || nsteps <= 0) return steps_direct(s, src, n0, nsteps, dt, dseis, ld, vcap);
    GraphEntry* hit = nullptr;
    for (GraphEntry& ge : s->graphs)
        if (ge.gen == s->gen && ge.n0 == n0 && ge.nsteps == nsteps && ge.ld == ld && ge.dt == dt &&
            ge.dseis == dseis && ge.vcap == vcap)
            hit = &ge;
    if (!hit) {
        if (!s->cap_stream) CK(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
        // the tile shape's plan exists before the capture starts
        ews_status sp = tile_plan(s, fwd_shape(s, vcap != nullptr));
        if (sp != EWS_OK) return sp;
        long long before[EWS_NKERNEL];
        std::memcpy(before, s->launches, sizeof(before));
        cudaStream_t user = s->stream;
        s->stream = s->cap_stream;
        CK(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
        const ews_status st = steps_direct(s, src, n0, nsteps, dt, dseis, ld, vcap);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s->cap_stream, &graph);
        s->stream = user;
        GraphEntry ge{};
        for (int k = 0; k < EWS_NKERNEL; ++k) ge.launches[k] = s->launches[k] - before[k];
        std::memcpy(s->launches, before, sizeof(before));
        if (st != EWS_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            if (st != EWS_OK) return st;
            return fail(EWS_ECUDA, "time-loop capture: %s", cudaGetErrorString(e));
        }
        const cudaError_t ei = cudaGraphInstantiate(&ge.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) return fail(EWS_ECUDA, "graph instantiate: %s", cudaGetErrorString(ei));
        ge.gen = s->gen;
        ge.n0 = n0;
        ge.nsteps = nsteps;
        ge.ld = ld;
        ge.dt = dt;
        ge.dseis = dseis;
        ge.vcap = vcap;
        if (s->graphs.size() >= 16) {          // keep the 16 most recent loops
            cudaGraphExecDestroy(s->graphs.front().exec);
            s->graphs.erase(s->graphs.begin());
        }
        s->graphs.push_back(ge);
        hit = &s->graphs.back();
    }
    CK(cudaGraphLaunch(hit->exec, s->stream));
    for (int k = 0; k < EWS_NKERNEL; ++k) s->launches[k] += hit->launches[k];
    s->fresh = false;
    return EWS_OK;
}

// ---- tile-shape tuner ----
// Per process: (nx, ny, nz, boundary, storage) -> EWS_TILE_* shape.
std::mutex g_tile_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_tile;

std::tuple<int, int, int, int, int> tile_key(const ews_sim* s) {
    return std::make_tuple(s->grid.nx, s->grid.ny, s->grid.nz, s->opt.boundary, s->opt.storage);
}

void set_tile_used(ews_sim* s, int shape) {
    if (shape != s->tile_used) {
        s->tile_used = shape;
        s->gen++;                               // recapture the time loops
    }
}

// Before a run from rest: the requested shape, else the table's entry for
// this grid, else the fastest of a few timed steps with each shape (taken
// from rest and thrown away: the caller resets the wavefields afterwards).
// With per-launch profiling on, an untuned grid keeps 32 x 8 (the trial
// launches would land in the profile).
ews_status choose_tile(ews_sim* s, int nt, double dt) {
    if (!tile_eligible(s)) {
        set_tile_used(s, EWS_TILE_32X8);
        return EWS_OK;
    }
    if (s->tile_req != EWS_TILE_AUTO) {
        set_tile_used(s, s->tile_req == EWS_TILE_FUSED && !fused_eligible(s) ? EWS_TILE_32X8
                                                                              : s->tile_req);
        return EWS_OK;
    }
    const auto key = tile_key(s);
    {
        std::lock_guard<std::mutex> lk(g_tile_mu);
        auto it = g_tile.find(key);
        if (it != g_tile.end()) {
            set_tile_used(s, it->second == EWS_TILE_FUSED && !fused_eligible(s) ? EWS_TILE_32X8
                                                                                : it->second);
            return EWS_OK;
        }
    }
    if (s->profiling) {
        set_tile_used(s, EWS_TILE_32X8);
        return EWS_OK;
    }
    const int T = std::min(nt, 6);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(EWS_ECUDA, "tile tuner: %s", cudaGetErrorString(ce));
    }
    int best = EWS_TILE_32X8;
    float best_ms = 1e30f;
    ews_status st = EWS_OK;
    std::vector<int> cand = {EWS_TILE_32X8, EWS_TILE_32X4, EWS_TILE_32X16};
    // the fused step, if it applies and its second wavefield set takes at
    // most a quarter of the device memory still free
    if (fused_eligible(s)) {
        size_t fr = 0, tot = 0;
        const double set = (double)NFIELD * s->fstride * sizeof(float);
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess &&
            set <= 0.25 * std::min((double)fr, dev_headroom()) &&
            tile_plan(s, EWS_TILE_FUSED) == EWS_OK)
            cand.push_back(EWS_TILE_FUSED);
    }
    for (int shape : cand) {
        s->tile_used = shape;
        float ms = 1e30f;
        for (int rep = 0; rep < 3 && st == EWS_OK; ++rep) {   // the first is a warm-up
            ce = cudaEventRecord(e0, s->stream);
            if (ce == cudaSuccess && (st = steps_direct(s, s->src, 0, T, dt, nullptr, T, nullptr)) != EWS_OK)
                break;
            if (ce == cudaSuccess) ce = cudaEventRecord(e1, s->stream);
            if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
            float t = 0.0f;
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
            if (ce != cudaSuccess) break;
            if (rep > 0) ms = std::min(ms, t);
        }
        if (st != EWS_OK || ce != cudaSuccess) break;
        // another shape replaces 32 x 8 (timed first) only if it is 2 %
        // faster, so shapes within timing noise of each other do not
        // change from run to run
        if (shape == EWS_TILE_32X8 ? ms < best_ms : ms < 0.98f * best_ms) {
            best_ms = ms;
            best = shape;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s->tile_used = EWS_TILE_32X8;
    if (best != EWS_TILE_FUSED || st != EWS_OK || ce != cudaSuccess) {
        // the second wavefield set is only kept for the shape that uses it
        const cudaError_t se = cudaStreamSynchronize(s->stream);
        if (se == cudaSuccess) drop_fused(s);
    }
    if (st != EWS_OK) return st;
    if (ce != cudaSuccess) return fail(EWS_ECUDA, "tile tuner: %s", cudaGetErrorString(ce));
    // the trial steps leave no trace: the error flag (an FP16 trial from
    // unscaled fields may overflow) is cleared; the wavefields are reset by
    // the caller
    CK(cudaMemsetAsync(s->err, 0, sizeof(int), s->stream));
    {
        std::lock_guard<std::mutex> lk(g_tile_mu);
        g_tile[key] = best;
    }
    set_tile_used(s, best);
    return EWS_OK;
}

// Collect the durations of the launches bracketed since the last collect
// (the stream must have been synchronised).
ews_status collect_profile(ews_sim* s) {
    for (size_t m = 1; m < s->ev_used; ++m) {
        if (s->ev_class[m] < 0) continue;
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, s->ev_pool[m - 1], s->ev_pool[m]));
        s->kernel_ms[s->ev_class[m]] += ms;
    }
    s->ev_used = 0;
    return EWS_OK;
}

// Grow a device buffer to at least `need` elements of T.
template <typename T>
ews_status ensure_buf(T** buf, size_t* cap, size_t need, const char* what) {
    if (*buf && *cap >= need) return EWS_OK;
    dev_free(*buf);
    *buf = nullptr;
    *cap = 0;
    cudaError_t e = dev_malloc((void**)buf, need * sizeof(T));
    if (e != cudaSuccess) return fail(EWS_ENOMEM, "%s (%zu bytes): %s", what, need * sizeof(T),
                                      cudaGetErrorString(e));
    *cap = need;
    return EWS_OK;
}

// Reverse sweep for dL/dseis = sadj (device, [3][nrec][nt]); or, when obs is
// given, first the L2 misfit residual of a recorded forward run.
// Checkpoint c of the current state (FP32 copy, or 16-bit with per-field
// scales), and its restore.
ews_status ckpt_save(ews_sim* s, int c) {
    const size_t fs = s->fstride;
    if (s->ckpt_storage == EWS_STORAGE_F32) {
        CK(cudaMemcpyAsync(s->ckpt + (size_t)c * 9 * fs, s->fields, 9 * fs * sizeof(float),
                           cudaMemcpyDeviceToDevice, s->stream));
        return EWS_OK;
    }
    uint16_t* base = reinterpret_cast<uint16_t*>(s->ckpt) + (size_t)c * 9 * fs;
    CK(launch_ckpt_store(s->fields, (long long)fs, s->ckpt_storage, s->ckpt_amax,
                         s->ckpt_scale + 9 * c, base, s->stream));
    return EWS_OK;
}

ews_status ckpt_load(ews_sim* s, int c) {
    const size_t fs = s->fstride;
    if (s->ckpt_storage == EWS_STORAGE_F32) {
        CK(cudaMemcpyAsync(s->fields, s->ckpt + (size_t)c * 9 * fs, 9 * fs * sizeof(float),
                           cudaMemcpyDeviceToDevice, s->stream));
        return EWS_OK;
    }
    const uint16_t* base = reinterpret_cast<const uint16_t*>(s->ckpt) + (size_t)c * 9 * fs;
    CK(launch_ckpt_load(base, (long long)fs, s->ckpt_storage, s->ckpt_scale + 9 * c, s->fields,
                        s->stream));
    return EWS_OK;
}

ews_status adjoint_core(ews_sim* s, int nt, double dt, int ckpt_every, const float* sadj_dev,
                        const float* obs_dev, double* misfit, float* g_lam, float* g_mu,
                        float* g_rho, int g_on_device) {
    ews_status st = ensure_ready(s, nt, dt);
    if (st != EWS_OK) return st;
    if (s->opt.boundary == EWS_BOUNDARY_CPML)
        return fail(EWS_EINVAL, "the adjoint supports the none and sponge boundaries");
    if (!s->wide()) return fail(EWS_EINVAL, "the adjoint needs F32 wavefield storage");
    if (s->g.fs != kNoSurface && s->has_fluid)
        return fail(EWS_EINVAL, "gradients with a free surface need mu > 0 below it");
    if (s->g.cm[0])
        return fail(EWS_EINVAL, "gradients with a coarse medium grid are not built");
    const int K = ckpt_every > 0 ? (ckpt_every < nt ? ckpt_every : nt) : (nt < 50 ? nt : 50);
    const int nck = (nt + K - 1) / K;
    const size_t fs = s->fstride;
    const bool transformed = !s->has_fluid;
    // Resident history: the trailing segments [n_res, nt) whose velocity
    // history fits the budget (at least the last segment) are captured by
    // the first forward pass; earlier segments are recomputed into the same
    // buffer from their checkpoints.
    const double slot_bytes = 3.0 * fs * sizeof(float);
    const long long budget_slots = (long long)(sim_history_budget(s, 0.5) / slot_bytes);
    int c_res = nck - 1;                       // first resident segment
    if (transformed)
        while (c_res > 0 && (long long)(nt - (c_res - 1) * K) + 1 <= budget_slots) --c_res;
    const int n_res = c_res * K;
    const int hslots = std::max(K, nt - n_res) + 1;
    // checkpoints only for the segments that will be recomputed
    if ((st = sim_adjoint_buffers(s, nt, transformed ? c_res : nck, transformed ? hslots : K + 1,
                                  obs_dev != nullptr, s->ckpt_pref)) != EWS_OK)
        return st;
    const size_t nseis = (size_t)3 * s->nrec * nt;
    AdjFields A;
    for (int c = 0; c < 3; ++c) A.p[c] = s->adj + fslot(VX + c) * fs;
    for (int c = 0; c < 6; ++c) A.q[c] = s->adj + fslot(SXX + c) * fs;
    for (int c = 0; c < 8; ++c) { A.acc[c] = s->adj + (9 + c) * fs; A.acc64[c] = s->acc64 + c * fs; }
    // forward with checkpoints (and seismograms when a misfit is asked for);
    // the resident segments also write their velocity history
    if ((st = ews_reset(s)) != EWS_OK) return st;
    float* dseis = obs_dev ? s->aux : nullptr;
    for (int c = 0; c < nck; ++c) {
        const int n0 = c * K, n1 = n0 + K < nt ? n0 + K : nt;
        if ((!transformed || c < c_res) &&   // resident segments are never restored
            (st = ckpt_save(s, c)) != EWS_OK)
            return st;
        if (transformed && c >= c_res) {
            if (c == c_res)
                CK(cudaMemcpyAsync(s->vhist, s->field(VX), 3 * fs * sizeof(float),
                                   cudaMemcpyDeviceToDevice, s->stream));
            // steps() puts v^{n+1/2} at slot n - n0 + 1 of the buffer it is given
            float* base = s->vhist + (size_t)(n0 - n_res) * 3 * fs;
            if ((st = steps(s, s->src, n0, n1 - n0, dt, dseis, nt, base)) != EWS_OK) return st;
        } else if ((st = steps(s, s->src, n0, n1 - n0, dt, dseis, nt)) != EWS_OK) {
            return st;
        }
    }
    const float* sadj = sadj_dev;
    if (obs_dev) {
        float* sa = s->aux + nseis;
        CK(cudaMemsetAsync(s->dmisfit, 0, sizeof(double), s->stream));
        CK(launch_residual(s->aux, obs_dev, sa, (long long)nseis, (float)dt, s->dmisfit, s->stream));
        sadj = sa;
    }
    CK(cudaMemsetAsync(s->adj, 0, 17 * fs * sizeof(float), s->stream));
    CK(cudaMemsetAsync(s->acc64, 0, 8 * fs * sizeof(double), s->stream));
    const float fdt = (float)dt;
    if (transformed) {
        // Reverse sweep in (alpha, tau): the forward passes with -dt on the
        // adjoint fields, gradient products fused into the velocity pass.
        DevFields AF;
        for (int q = 0; q < NFIELD; ++q) AF.f[q] = s->adj + fslot(q) * fs;
        if ((st = sim_adjoint_plan(s)) != EWS_OK) return st;
        float mdt[NFIELD], one[NFIELD];
        for (int q = 0; q < NFIELD; ++q) {
            mdt[q] = -fdt;
            one[q] = 1.0f;
        }
        // segment ranges in reverse: the resident range first, then the
        // recomputed segments
        for (int c = c_res; c >= 0; --c) {
            const int n0 = c * K, n1 = c == c_res ? nt : n0 + K;
            if (c < c_res) {
                if ((st = ckpt_load(s, c)) != EWS_OK) return st;
                CK(cudaMemcpyAsync(s->vhist, s->field(VX), 3 * fs * sizeof(float),
                                   cudaMemcpyDeviceToDevice, s->stream));
                if ((st = steps(s, s->src, n0, n1 - n0, dt, nullptr, nt, s->vhist)) != EWS_OK)
                    return st;
            }
            for (int m = n1 - 1; m >= n0; --m) {
                VelExtra X{};
                for (int q = 0; q < 8; ++q) X.acc[q] = A.acc[q];
                X.fstride = (long long)fs;
                X.gdt = fdt;
                X.hslot = m - n0 + 1;
                X.vnext = m + 1 < n1 ? s->vhist + (size_t)(m - n0 + 2) * 3 * fs : nullptr;
                CK(launch_velocity_grad(s->adj_plan, s->g, AF, s->B, mdt, X, s->err, s->stream));
                if (s->nrec > 0 && sadj)
                    CK(launch_adj_inject(s->g, A, s->M(), s->B, s->rtaps, s->nrec, sadj, nt, m,
                                         s->stream));
                CK(launch_stress(s->adj_plan, s->g, AF, s->B, mdt, one, s->err, s->stream, true));
                if ((m - n0) % K == 0 && m > n0) CK(launch_acc_flush(s->g, A, s->stream));
            }
            CK(launch_rho_term(s->g, A, s->B, s->vhist + 3 * fs, s->vhist, (long long)fs, s->stream));
            CK(launch_acc_flush(s->g, A, s->stream));
        }
    }
    for (int c = transformed ? -1 : nck - 1; c >= 0; --c) {
        const int n0 = c * K, n1 = n0 + K < nt ? n0 + K : nt;
        if ((st = ckpt_load(s, c)) != EWS_OK) return st;
        CK(cudaMemcpyAsync(s->vhist, s->field(VX), 3 * fs * sizeof(float), cudaMemcpyDeviceToDevice,
                           s->stream));
        if ((st = steps(s, s->src, n0, n1 - n0, dt, nullptr, nt, s->vhist)) != EWS_OK) return st;
        for (int n = n1 - 1; n >= n0; --n) {
            const float* vn = s->vhist + (size_t)(n - n0 + 1) * 3 * fs;
            const float* vp = s->vhist + (size_t)(n - n0) * 3 * fs;
            CK(launch_adj_stress(s->g, A, s->M(), s->B, vn, fs, fdt, s->stream));
            if (s->nrec > 0 && sadj)
                CK(launch_adj_record(s->g, A, s->rtaps, s->nrec, sadj, nt, n, s->stream));
            CK(launch_adj_velocity(s->g, A, s->M(), s->B, vn, vp, fs, fdt, s->stream));
        }
        CK(launch_acc_flush(s->g, A, s->stream));
    }
    const size_t ncell = (size_t)s->ncell();
    float *gl = g_lam, *gm = g_mu, *gr = g_rho;
    if (!g_on_device) {
        size_t cap = s->gout ? 3 * ncell : 0;
        if ((st = ensure_buf(&s->gout, &cap, 3 * ncell, "gradient staging")) != EWS_OK) return st;
        gl = s->gout;
        gm = s->gout + ncell;
        gr = s->gout + 2 * ncell;
    }
    if (transformed)
        CK(launch_grad_finalize_t(s->g, A, s->M(), gl, gm, gr, s->stream));
    else
        CK(launch_grad_finalize(s->g, A, s->M(), gl, gm, gr, s->stream));
    if (!g_on_device) {
        CK(cudaMemcpyAsync(g_lam, gl, ncell * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaMemcpyAsync(g_mu, gm, ncell * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaMemcpyAsync(g_rho, gr, ncell * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
    }
    if (misfit && obs_dev)
        CK(cudaMemcpyAsync(misfit, s->dmisfit, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaGetLastError());
    if (herr) {
        CK(cudaMemsetAsync(s->err, 0, sizeof(int), s->stream));
        if (herr & 3) return fail(EWS_ETIMEOUT, "a pipeline wait in the stencil kernels gave up");
        return fail(EWS_ENONFINITE, "a receiver recorded NaN or Inf during the gradient's forward run");
    }
    if (s->profiling && (st = collect_profile(s)) != EWS_OK) return st;
    return EWS_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

namespace ews {

ews_status sim_ready(ews_sim* s, int n_end, double dt) { return ensure_ready(s, n_end, dt); }

DevSource sim_source(const ews_sim* s, double dt) { return source_taps(s, s->src, dt); }

ews_status sim_adjoint_buffers(ews_sim* s, int nt, int nckpt, int hslots, bool with_obs,
                               int ckpt_storage) {
    const size_t fs = s->fstride;
    const int nck = nckpt > 0 ? nckpt : 1;
    s->ckpt_storage = ckpt_storage;
    if (ckpt_storage != EWS_STORAGE_F32 && nck > s->ckpt_scale_cap) {
        dev_free(s->ckpt_scale);
        s->ckpt_scale = nullptr;
        s->ckpt_scale_cap = 0;
        cudaError_t e = dev_malloc((void**)&s->ckpt_scale, (size_t)nck * 9 * sizeof(float));
        if (e != cudaSuccess) return fail(EWS_ENOMEM, "checkpoint scales: %s", cudaGetErrorString(e));
        s->ckpt_scale_cap = nck;
        if (!s->ckpt_amax) {
            e = dev_malloc((void**)&s->ckpt_amax, 9 * sizeof(unsigned));
            if (e != cudaSuccess) return fail(EWS_ENOMEM, "checkpoint maxima: %s", cudaGetErrorString(e));
        }
    }
    if (!s->adj) {
        // all three or none: a later call tests s->adj alone
        const char* what = "adjoint state";
        cudaError_t e = dev_malloc((void**)&s->adj, 17 * fs * sizeof(float));
        if (e == cudaSuccess) {
            what = "adjoint accumulators";
            e = dev_malloc((void**)&s->acc64, 8 * fs * sizeof(double));
        }
        if (e == cudaSuccess) {
            what = "misfit";
            e = dev_malloc((void**)&s->dmisfit, sizeof(double));
        }
        if (e != cudaSuccess) {
            dev_free(s->adj);
            dev_free(s->acc64);
            dev_free(s->dmisfit);
            s->adj = nullptr;
            s->acc64 = nullptr;
            s->dmisfit = nullptr;
            return fail(EWS_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
        }
    }
    ews_status st;
    const size_t ck_floats = ckpt_storage == EWS_STORAGE_F32 ? (size_t)nck * 9 * fs
                                                              : ((size_t)nck * 9 * fs + 1) / 2;
    if ((st = ensure_buf(&s->ckpt, &s->ckpt_cap, ck_floats, "checkpoints")) != EWS_OK) return st;
    if ((st = ensure_buf(&s->vhist, &s->vhist_cap, (size_t)hslots * 3 * fs, "velocity history")) != EWS_OK)
        return st;
    const size_t nseis = (size_t)3 * s->nrec * nt;
    if (with_obs && (st = ensure_buf(&s->aux, &s->aux_cap, 2 * (nseis ? nseis : 1), "adjoint source")) != EWS_OK)
        return st;
    return EWS_OK;
}

double sim_history_budget(const ews_sim* s, double share) {
    if (s->hist_budget >= 0) return s->hist_budget;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return 0.0;
    const double held = (double)s->vhist_cap * sizeof(float);
    const double room = dev_headroom();          // under the library's memory limit
    const double avail = (double)free_b < room ? (double)free_b : room;
    return share * (avail + held);
}

ews_status sim_adjoint_plan(ews_sim* s) {
    const size_t fs = s->fstride;
    DevFields AF;
    for (int q = 0; q < NFIELD; ++q) AF.f[q] = s->adj + fslot(q) * fs;
    if (!s->adj_plan) {
        cudaError_t e = stencil_plan_create(s->g, AF, s->M(), s->B, EWS_STORAGE_F32, &s->adj_plan);
        if (e != cudaSuccess) return fail(EWS_ECUDA, "adjoint stencil plan: %s", cudaGetErrorString(e));
    }
    const int cap_slots = (int)(s->vhist_cap / (3 * fs));
    if (s->adj_hist != s->vhist || s->adj_hist_slots != cap_slots) {
        CK(stencil_plan_set_history(s->adj_plan, s->g, s->vhist, (long long)fs, cap_slots,
                                    s->adj + 9 * fs));
        s->adj_hist = s->vhist;
        s->adj_hist_slots = cap_slots;
    }
    return EWS_OK;
}

}  // namespace ews

extern "C" {

int ews_version(void) { return 100; }

ews_status ews_set_tile_shape(ews_sim* s, int shape) {
    if (!s) return fail(EWS_EINVAL, "null simulation");
    if (shape < EWS_TILE_AUTO || shape > EWS_TILE_FUSED)
        return fail(EWS_EINVAL, "unknown tile shape %d", shape);
    s->tile_req = shape;
    if (shape != EWS_TILE_AUTO) set_tile_used(s, tile_eligible(s) ? shape : EWS_TILE_32X8);
    return EWS_OK;
}

int ews_get_tile_shape(ews_sim* s) { return s ? s->tile_used : 0; }

int ews_tile_tuned(const ews_grid* grid, int boundary, int storage) {
    if (!grid) return 0;
    std::lock_guard<std::mutex> lk(g_tile_mu);
    auto it = g_tile.find(std::make_tuple(grid->nx, grid->ny, grid->nz, boundary, storage));
    return it == g_tile.end() ? 0 : it->second;
}

int ews_tile_tuning_export(ews_tuned_tile* out, int cap) {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    int n = 0;
    for (const auto& kv : g_tile) {
        if (out && n < cap) {
            ews_tuned_tile& e = out[n];
            e.nx = std::get<0>(kv.first);
            e.ny = std::get<1>(kv.first);
            e.nz = std::get<2>(kv.first);
            e.boundary = std::get<3>(kv.first);
            e.storage = std::get<4>(kv.first);
            e.shape = kv.second;
        }
        ++n;
    }
    return n;
}

ews_status ews_tile_tuning_import(const ews_tuned_tile* in, int n) {
    if (n < 0 || (n > 0 && !in)) return fail(EWS_EINVAL, "ews_tile_tuning_import: no entries");
    for (int k = 0; k < n; ++k) {
        const ews_tuned_tile& e = in[k];
        if (e.nx < 4 || e.ny < 4 || e.nz < 4 || e.boundary < EWS_BOUNDARY_NONE ||
            e.boundary > EWS_BOUNDARY_CPML || e.storage < EWS_STORAGE_F32 ||
            e.storage > EWS_STORAGE_F16 || e.shape < EWS_TILE_32X8 || e.shape > EWS_TILE_FUSED ||
            (e.shape == EWS_TILE_FUSED &&
             (e.boundary == EWS_BOUNDARY_CPML || e.storage != EWS_STORAGE_F32)))
            return fail(EWS_EINVAL,
                        "ews_tile_tuning_import: entry %d (%d x %d x %d, boundary %d, storage %d, "
                        "shape %d) is invalid; nothing imported",
                        k, e.nx, e.ny, e.nz, e.boundary, e.storage, e.shape);
    }
    std::lock_guard<std::mutex> lk(g_tile_mu);
    for (int k = 0; k < n; ++k) {
        const ews_tuned_tile& e = in[k];
        g_tile[std::make_tuple(e.nx, e.ny, e.nz, e.boundary, e.storage)] = e.shape;
    }
    return EWS_OK;
}

void ews_tile_tuning_clear(void) {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    g_tile.clear();
}

const char* ews_last_error(void) { return g_err; }

double ews_cfl_dt(const ews_grid* g, double vmax) {
    if (!g || !(vmax > 0)) return 0.0;
    return 0.495 * std::min(g->dx, std::min(g->dy, g->dz)) / vmax;
}

double ews_max_freq(const ews_grid* g, double vmin) {
    if (!g || !(vmin > 0)) return 0.0;
    return vmin / (5.0 * std::max(g->dx, std::max(g->dy, g->dz)));
}

ews_status ews_create(const ews_grid* grid, const ews_options* opt, ews_sim** out) {
    g_err[0] = 0;
    if (!grid || !out) return fail(EWS_EINVAL, "null argument");
    *out = nullptr;
    if (grid->nx < 4 || grid->ny < 4 || grid->nz < 4)
        return fail(EWS_EINVAL, "grid must have at least 4 cells per axis");
    if (!(grid->dx > 0) || !(grid->dy > 0) || !(grid->dz > 0))
        return fail(EWS_EINVAL, "grid spacing must be positive");
    if ((long long)grid->nx * grid->ny * grid->nz > (1LL << 34))
        return fail(EWS_EINVAL, "grid too large");
    ews_options o{};
    if (opt) {
        o = *opt;
    } else {
        o.boundary = EWS_BOUNDARY_SPONGE;
        o.width = 16;
    }
    if (o.boundary < 0 || o.boundary > 2) return fail(EWS_EINVAL, "unknown boundary kind");
    if (o.boundary != EWS_BOUNDARY_NONE) {
        if (o.width < 1) return fail(EWS_EINVAL, "boundary width must be >= 1");
        if (2 * o.width > grid->nx || 2 * o.width > grid->ny || 2 * o.width > grid->nz)
            return fail(EWS_EINVAL, "2 * width exceeds the grid");
    }
    if (o.storage != EWS_STORAGE_F32 && o.storage != EWS_STORAGE_BF16 &&
        o.storage != EWS_STORAGE_F16)
        return fail(EWS_EINVAL, "unknown storage type %d", o.storage);
    if (o.snapshot_every < 0) return fail(EWS_EINVAL, "snapshot_every < 0");
    if (o.snapshot_mask >> NFIELD) return fail(EWS_EINVAL, "snapshot_mask has unknown bits");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(EWS_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));

    ews_sim* s = new (std::nothrow) ews_sim();
    if (!s) return fail(EWS_ENOMEM, "host allocation failed");
    s->grid = *grid;
    s->opt = o;
    s->S.kind = -1;
    DevGrid& g = s->g;
    g.nx = grid->nx;
    g.ny = grid->ny;
    g.nz = grid->nz;
    g.pitch = round_up(grid->nx, 32);
    g.plane = (long long)g.pitch * g.ny;
    g.c1x = (float)(kC1 / grid->dx);
    g.c2x = (float)(kC2 / grid->dx);
    g.c1y = (float)(kC1 / grid->dy);
    g.c2y = (float)(kC2 / grid->dy);
    g.c1z = (float)(kC1 / grid->dz);
    g.c2z = (float)(kC2 / grid->dz);
    g.fs = kNoSurface;
    g.c1z2 = (float)(1.0 / grid->dz);
    g.fs_eps = 0.0f;
    s->fstride = (size_t)((g.plane * g.nz + 63) / 64 * 64);
    s->es = o.storage == EWS_STORAGE_F32 ? 4 : 2;
    s->B.kind = o.boundary;
    s->B.W = o.width;

    auto cleanup = [&](ews_status st) {
        ews_destroy(s);
        return st;
    };
    e = dev_malloc((void**)&s->fields, NFIELD * s->fstride * s->es);
    if (e != cudaSuccess) return cleanup(fail(EWS_ENOMEM, "wavefields: %s", cudaGetErrorString(e)));
    e = dev_malloc((void**)&s->medium, 3 * s->fstride * sizeof(float));
    if (e != cudaSuccess) return cleanup(fail(EWS_ENOMEM, "medium: %s", cudaGetErrorString(e)));
    const int nmax = std::max(g.nx, std::max(g.ny, g.nz));
    e = dev_malloc((void**)&s->prof, 9 * (size_t)nmax * sizeof(float));
    if (e != cudaSuccess) return cleanup(fail(EWS_ENOMEM, "profiles: %s", cudaGetErrorString(e)));
    e = dev_malloc((void**)&s->flags, 5 * sizeof(unsigned));
    if (e != cudaSuccess) return cleanup(fail(EWS_ENOMEM, "flags: %s", cudaGetErrorString(e)));
    e = dev_malloc((void**)&s->err, sizeof(int));
    if (e != cudaSuccess) return cleanup(fail(EWS_ENOMEM, "err: %s", cudaGetErrorString(e)));
    if (o.boundary == EWS_BOUNDARY_CPML) {
        s->psi_floats = 18 * s->fstride;
        e = dev_malloc((void**)&s->psi, s->psi_floats * sizeof(float));
        if (e != cudaSuccess)
            return cleanup(fail(EWS_ENOMEM, "C-PML memory: %s", cudaGetErrorString(e)));
        for (int t = 0; t < 18; ++t) s->B.psi[t] = s->psi + t * s->fstride;
    }
    e = cudaMemset(s->fields, 0, NFIELD * s->fstride * s->es);
    if (e == cudaSuccess) e = cudaMemset(s->medium, 0, 3 * s->fstride * sizeof(float));
    if (e == cudaSuccess && s->psi) e = cudaMemset(s->psi, 0, s->psi_floats * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(s->err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cleanup(fail(EWS_ECUDA, "memset: %s", cudaGetErrorString(e)));
    e = stencil_plan_create(s->g, s->F(), s->M(), s->B, o.storage, &s->plan);
    if (e != cudaSuccess)
        return cleanup(fail(EWS_ECUDA, "stencil plan (TMA descriptors): %s", cudaGetErrorString(e)));
    *out = s;
    return EWS_OK;
}

void ews_destroy(ews_sim* s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    else cudaDeviceSynchronize();
    dev_free(s->fields);
    dev_free(s->medium);
    dev_free(s->cmed);
    dev_free(s->prof);
    dev_free(s->flags);
    dev_free(s->err);
    stencil_plan_destroy(s->plan);
    stencil_plan_destroy(s->adj_plan);
    drop_tile_plans(s);
    dev_free(s->psi);
    dev_free(s->wavelet);
    dev_free(s->rtaps);
    dev_free(s->seis_buf);
    dev_free(s->adj);
    dev_free(s->acc64);
    dev_free(s->ckpt);
    dev_free(s->ckpt_scale);
    dev_free(s->ckpt_amax);
    dev_free(s->vhist);
    dev_free(s->aux);
    dev_free(s->gout);
    dev_free(s->dmisfit);
    dev_free(s->stage);
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    for (GraphEntry& ge : s->graphs) cudaGraphExecDestroy(ge.exec);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    delete s;
}

ews_status ews_set_stream(ews_sim* s, void* stream) {
    if (!s) return fail(EWS_EINVAL, "null simulation");
    s->stream = (cudaStream_t)stream;
    return EWS_OK;
}

ews_status ews_set_model_lame(ews_sim* s, const float* lam, const float* mu, const float* rho,
                              int on_device) {
    return set_model(s, lam, mu, rho, on_device, 0);
}

ews_status ews_set_model_vel(ews_sim* s, const float* vp, const float* vs, const float* rho,
                             int on_device) {
    return set_model(s, vp, vs, rho, on_device, 1);
}

ews_status ews_set_model_coarse(ews_sim* s, int mx, int my, int mz, const float* a,
                                const float* b, const float* rho, int from_velocities,
                                int on_device) {
    if (!s) return fail(EWS_EINVAL, "null simulation");
    if (!a || !b || !rho) return fail(EWS_EINVAL, "null model array");
    if (mx < 1 || my < 1 || mz < 1) return fail(EWS_EINVAL, "medium grid %d x %d x %d", mx, my, mz);
    if (s->g.fs != kNoSurface)
        return fail(EWS_EINVAL, "a coarse medium grid with a free surface is not built");
    const size_t m = (size_t)mx * my * mz;
    s->model_set = false;
    for (int q = 0; q < 3; ++q) s->g.cm[q] = nullptr;
    dev_free(s->cmed);
    s->cmed = nullptr;
    CK(dev_malloc((void**)&s->cmed, 3 * m * sizeof(float)));
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(s->cmed, a, m * sizeof(float), kind, s->stream));
    CK(cudaMemcpyAsync(s->cmed + m, b, m * sizeof(float), kind, s->stream));
    CK(cudaMemcpyAsync(s->cmed + 2 * m, rho, m * sizeof(float), kind, s->stream));
    // validation, velocity -> Lame conversion and the medium bounds on the
    // medium grid's own cells (the interpolated values lie between them)
    DevGrid gc{};
    gc.nx = mx;
    gc.ny = my;
    gc.nz = mz;
    gc.pitch = mx;
    gc.plane = (long long)mx * my;
    gc.fs = kNoSurface;
    CK(cudaMemsetAsync(s->flags, 0, 5 * sizeof(unsigned), s->stream));
    CK(cudaMemsetAsync(s->flags + 2, 0x7F, 2 * sizeof(unsigned), s->stream));
    CK(launch_medium_setup(gc, s->cmed, s->cmed + m, s->cmed + 2 * m, from_velocities, s->flags,
                           s->stream));
    unsigned hf[5];
    CK(cudaMemcpyAsync(hf, s->flags, sizeof(hf), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (hf[0] & 1u) return fail(EWS_ENONFINITE, "model contains NaN or Inf");
    if (hf[0] & 2u) return fail(EWS_EINVAL, "model has rho <= 0");
    if (hf[0] & 4u) return fail(EWS_EINVAL, "model has mu < 0 (vs^2 < 0)");
    if (hf[0] & 8u) return fail(EWS_EINVAL, "model has lambda + 2 mu <= 0");
    float bnd[4];
    std::memcpy(bnd, &hf[1], sizeof(bnd));
    s->vpmax = bnd[0];
    s->rho_min = bnd[1];
    s->zs_min = bnd[2];
    s->zp_max = bnd[3];
    s->has_fluid = (hf[0] & 16u) != 0;
    for (int q = 0; q < 3; ++q) s->g.cm[q] = s->cmed + q * m;
    s->g.mx = mx;
    s->g.my = my;
    s->g.mz = mz;
    s->g.rx = (float)((double)mx / s->g.nx);
    s->g.ry = (float)((double)my / s->g.ny);
    s->g.rz = (float)((double)mz / s->g.nz);
    s->model_set = true;
    s->pml_dt = -1.0;
    s->gen++;
    // The medium arrays of the wavefield grid are not read with a coarse
    // grid: release them (3 floats per cell; allocated again by a later
    // ews_set_model_lame / _vel).  Plans and graphs that point at them go.
    if (s->medium) {
        CK(cudaStreamSynchronize(s->stream));
        for (GraphEntry& ge : s->graphs) cudaGraphExecDestroy(ge.exec);
        s->graphs.clear();
        stencil_plan_destroy(s->adj_plan);
        s->adj_plan = nullptr;
        s->adj_hist = nullptr;
        s->adj_hist_slots = 0;
        drop_tile_plans(s);
        dev_free(s->medium);
        s->medium = nullptr;
    }
    return EWS_OK;
}

ews_status ews_set_source(ews_sim* s, int kind, const double pos[3], const double comp[6],
                          const float* wavelet, int nt) {
    if (!s) return fail(EWS_EINVAL, "null simulation");
    if (kind != EWS_SOURCE_MOMENT && kind != EWS_SOURCE_FORCE)
        return fail(EWS_EINVAL, "unknown source kind %d", kind);
    if (!pos || !comp || !wavelet || nt <= 0) return fail(EWS_EINVAL, "bad source arguments");
    ews_status st = check_pos(s, pos, "source");
    if (st != EWS_OK) return st;
    const int nc = kind == EWS_SOURCE_MOMENT ? 6 : 3;
    for (int c = 0; c < nc; ++c)
        if (!std::isfinite(comp[c])) return fail(EWS_ENONFINITE, "source component not finite");
    for (int n = 0; n < nt; ++n)
        if (!std::isfinite(wavelet[n])) return fail(EWS_ENONFINITE, "wavelet not finite");
    if (nt > s->wavelet_nt) {
        dev_free(s->wavelet);
        s->wavelet = nullptr;
        s->wavelet_nt = 0;
        CK(dev_malloc((void**)&s->wavelet, nt * sizeof(float)));
    }
    CK(cudaMemcpyAsync(s->wavelet, wavelet, nt * sizeof(float), cudaMemcpyHostToDevice,
                       s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->wavelet_nt = nt;
    s->gen++;
    s->wsum = 0;
    for (int n = 0; n < nt; ++n) s->wsum += std::fabs((double)wavelet[n]);
    SourceSpec& sp = s->src;
    sp.kind = kind;
    for (int a = 0; a < 3; ++a) sp.pos[a] = pos[a];
    for (int c = 0; c < 6; ++c) sp.comp[c] = c < nc ? comp[c] : 0.0;
    s->S.kind = kind;
    return EWS_OK;
}

ews_status ews_set_checkpoint_storage(ews_sim* s, int storage) {
    if (!s) return fail(EWS_EINVAL, "null simulation");
    if (storage != EWS_STORAGE_F32 && storage != EWS_STORAGE_BF16 && storage != EWS_STORAGE_F16)
        return fail(EWS_EINVAL, "unknown checkpoint storage %d", storage);
    s->ckpt_pref = storage;
    return EWS_OK;
}

ews_status ews_set_free_surface(ews_sim* s, int ks, double eps) {
    if (!s) return fail(EWS_EINVAL, "null simulation");
    if (ks >= 0 && s->g.cm[0])
        return fail(EWS_EINVAL, "a free surface with a coarse medium grid is not built");
    if (ks >= s->g.nz) return fail(EWS_EINVAL, "surface plane %d outside the grid (nz = %d)", ks, s->g.nz);
    if (ks >= 0 && !(eps > 0.0 && eps <= 1.0))
        return fail(EWS_EINVAL, "vacuum fraction %g outside (0, 1]", eps);
    s->g.fs = ks < 0 ? kNoSurface : ks;
    s->fs_eps = ks < 0 ? 0.0 : eps;
    s->g.fs_eps = (float)s->fs_eps;
    s->model_set = false;          // the medium above the surface must be set again
    s->gen++;
    return EWS_OK;
}

ews_status ews_set_receivers(ews_sim* s, int nrec, const double* pos) {
    if (!s) return fail(EWS_EINVAL, "null simulation");
    if (nrec < 0 || (nrec > 0 && !pos)) return fail(EWS_EINVAL, "bad receiver arguments");
    for (int r = 0; r < nrec; ++r) {
        ews_status st = check_pos(s, pos + 3 * r, "receiver");
        if (st != EWS_OK) return st;
    }
    std::vector<Tap> taps((size_t)24 * nrec);
    for (int c = 0; c < 3; ++c)
        for (int r = 0; r < nrec; ++r) taps_for(s, VX + c, pos + 3 * r, 1.0, &taps[(size_t)8 * (c * nrec + r)]);
    dev_free(s->rtaps);
    s->rtaps = nullptr;
    s->nrec = 0;
    if (nrec > 0) {
        CK(dev_malloc((void**)&s->rtaps, taps.size() * sizeof(Tap)));
        CK(cudaMemcpyAsync(s->rtaps, taps.data(), taps.size() * sizeof(Tap),
                           cudaMemcpyHostToDevice, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    }
    s->nrec = nrec;
    s->gen++;
    return EWS_OK;
}

ews_status ews_reset(ews_sim* s) {
    if (!s) return fail(EWS_EINVAL, "null simulation");
    CK(cudaMemsetAsync(s->fields, 0, NFIELD * s->fstride * s->es, s->stream));
    if (s->psi) CK(cudaMemsetAsync(s->psi, 0, s->psi_floats * sizeof(float), s->stream));
    s->fresh = true;
    return EWS_OK;
}

ews_status ews_advance(ews_sim* s, int n0, int nsteps, double dt, float* seis, int ld,
                       int seis_on_device) {
    if (!s) return fail(EWS_EINVAL, "null simulation");
    if (n0 < 0 || nsteps < 0) return fail(EWS_EINVAL, "negative step range");
    if (s->nrec > 0 && seis && ld < n0 + nsteps) return fail(EWS_EINVAL, "ld too small");
    ews_status st = ensure_ready(s, n0 + nsteps, dt);
    if (st != EWS_OK) return st;
    if (s->fresh) auto_scales(s, dt);
    float* dseis = nullptr;
    if (s->nrec > 0 && seis) {
        if (seis_on_device) {
            dseis = seis;
        } else {
            size_t need = (size_t)3 * s->nrec * ld;
            if (need > s->seis_cap) {
                dev_free(s->seis_buf);
                s->seis_buf = nullptr;
                s->seis_cap = 0;
                CK(dev_malloc((void**)&s->seis_buf, need * sizeof(float)));
                s->seis_cap = need;
            }
            dseis = s->seis_buf;
        }
    }
    if ((st = steps(s, s->src, n0, nsteps, dt, dseis, ld)) != EWS_OK) return st;
    if (dseis && !seis_on_device) {
        // copy back only the columns written by this call
        CK(cudaMemcpy2DAsync(seis + n0, ld * sizeof(float), dseis + n0, ld * sizeof(float),
                             nsteps * sizeof(float), 3 * (size_t)s->nrec,
                             cudaMemcpyDeviceToHost, s->stream));
    }
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaGetLastError());
    if (herr) {
        CK(cudaMemsetAsync(s->err, 0, sizeof(int), s->stream));
        if (herr & 3)
            return fail(EWS_ETIMEOUT, "a pipeline wait in the stencil kernels gave up (flags %d)",
                        herr);
        if (herr & 4)   // an FP16 overflow is the cause of any Inf the receivers saw
            return fail(EWS_ERANGE, "a wavefield value exceeded the FP16 range: lower the "
                                    "field scales (ews_set_field_scales)");
        return fail(EWS_ENONFINITE, "a receiver recorded NaN or Inf in steps %d..%d: the "
                                    "wavefield is not finite", n0, n0 + nsteps - 1);
    }
    if (s->profiling && (st = collect_profile(s)) != EWS_OK) return st;
    return EWS_OK;
}

ews_status ews_run(ews_sim* s, int nt, double dt, float* seis, int seis_on_device,
                   float* snapshots) {
    if (!s) return fail(EWS_EINVAL, "null simulation");
    if (nt <= 0) return fail(EWS_EINVAL, "nt must be positive");
    if (s->nrec > 0 && !seis) return fail(EWS_EINVAL, "seis is NULL but receivers are set");
    ews_status st = ensure_ready(s, nt, dt);
    if (st != EWS_OK) return st;
    if ((st = choose_tile(s, nt, dt)) != EWS_OK) return st;
    if ((st = ews_reset(s)) != EWS_OK) return st;
    const int every = s->opt.snapshot_every;
    const unsigned mask = s->opt.snapshot_mask;
    if (!snapshots || every <= 0 || mask == 0)
        return ews_advance(s, 0, nt, dt, seis, nt, seis_on_device);
    // snapshot loop: advance in chunks of `every` steps
    const size_t ncell = (size_t)s->ncell();
    size_t slot = 0;
    for (int n0 = 0; n0 + every <= nt; n0 += every) {
        if ((st = ews_advance(s, n0, every, dt, seis, nt, seis_on_device)) != EWS_OK) return st;
        for (int q = 0; q < NFIELD; ++q)
            if (mask & (1u << q)) {
                st = field_out(s, q, snapshots + slot * ncell, seis_on_device);
                if (st != EWS_OK) return st;
                ++slot;
            }
    }
    int done = (nt / every) * every;
    if (done < nt && (st = ews_advance(s, done, nt - done, dt, seis, nt, seis_on_device)) != EWS_OK)
        return st;
    CK(cudaStreamSynchronize(s->stream));
    return EWS_OK;
}

ews_status ews_set_profiling(ews_sim* s, int on) {
    if (!s) return fail(EWS_EINVAL, "null simulation");
    s->profiling = on != 0;
    s->ev_used = 0;
    return EWS_OK;
}

ews_status ews_get_profile(ews_sim* s, double* ms, long long* launches, int reset) {
    if (!s) return fail(EWS_EINVAL, "null simulation");
    for (int k = 0; k < EWS_NKERNEL; ++k) {
        if (ms) ms[k] = s->kernel_ms[k];
        if (launches) launches[k] = s->launches[k];
        if (reset) {
            s->kernel_ms[k] = 0.0;
            s->launches[k] = 0;
        }
    }
    return EWS_OK;
}

ews_status ews_get_state(ews_sim* s, float* out, int on_device) {
    if (!s || !out) return fail(EWS_EINVAL, "null argument");
    const size_t ncell = (size_t)s->ncell();
    for (int q = 0; q < NFIELD; ++q) {
        ews_status st = field_out(s, q, out + q * ncell, on_device);
        if (st != EWS_OK) return st;
    }
    CK(cudaStreamSynchronize(s->stream));
    return EWS_OK;
}

ews_status ews_set_state(ews_sim* s, const float* in, int on_device) {
    if (!s || !in) return fail(EWS_EINVAL, "null argument");
    const size_t ncell = (size_t)s->ncell();
    for (int q = 0; q < NFIELD; ++q) {
        ews_status st = field_in(s, q, in + q * ncell, on_device);
        if (st != EWS_OK) return st;
    }
    if (s->psi) CK(cudaMemsetAsync(s->psi, 0, s->psi_floats * sizeof(float), s->stream));
    s->fresh = false;
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (herr) {
        CK(cudaMemsetAsync(s->err, 0, sizeof(int), s->stream));
        CK(cudaStreamSynchronize(s->stream));
        return fail(EWS_ERANGE, "a state value exceeds the FP16 range at the field scales");
    }
    return EWS_OK;
}

ews_status ews_release_workspace(ews_sim* s) {
    if (!s) return fail(EWS_EINVAL, "null simulation");
    if (s->stream) CK(cudaStreamSynchronize(s->stream));
    else CK(cudaDeviceSynchronize());
    for (GraphEntry& ge : s->graphs) cudaGraphExecDestroy(ge.exec);
    s->graphs.clear();
    stencil_plan_destroy(s->adj_plan);
    s->adj_plan = nullptr;
    s->adj_hist = nullptr;
    s->adj_hist_slots = 0;
    float** fbufs[] = {&s->adj, &s->ckpt, &s->vhist, &s->aux, &s->gout, &s->stage, &s->seis_buf};
    for (float** b : fbufs) {
        dev_free(*b);
        *b = nullptr;
    }
    dev_free(s->acc64);
    s->acc64 = nullptr;
    dev_free(s->dmisfit);
    s->dmisfit = nullptr;
    s->ckpt_cap = s->vhist_cap = s->aux_cap = s->stage_cap = s->seis_cap = 0;
    return EWS_OK;
}

ews_status ews_set_history_budget(ews_sim* s, double bytes) {
    if (!s) return fail(EWS_EINVAL, "null simulation");
    if (std::isnan(bytes) || !std::isfinite(bytes)) return fail(EWS_EINVAL, "budget must be finite");
    s->hist_budget = bytes < 0 ? -1.0 : bytes;
    return EWS_OK;
}

ews_status ews_set_field_scales(ews_sim* s, const float* scale) {
    if (!s) return fail(EWS_EINVAL, "null simulation");
    if (!scale) {                      // back to the defaults
        for (int q = 0; q < NFIELD; ++q) s->scale[q] = 1.0f;
        s->scale_user = false;
        s->gen++;
        return ews_reset(s);
    }
    for (int q = 0; q < NFIELD; ++q) {
        const float v = scale[q];
        int e;
        if (!(v > 0) || !std::isfinite(v) || std::frexp(v, &e) != 0.5f)
            return fail(EWS_EINVAL, "field scale %d (%g) is not a positive power of two", q,
                        (double)v);
    }
    if (s->wide()) {
        for (int q = 0; q < NFIELD; ++q)
            if (scale[q] != 1.0f) return fail(EWS_EINVAL, "F32 storage takes no field scales");
    }
    for (int q = 0; q < NFIELD; ++q) s->scale[q] = scale[q];
    s->scale_user = true;
    s->gen++;
    return ews_reset(s);
}

ews_status ews_get_field_scales(ews_sim* s, float* scale) {
    if (!s || !scale) return fail(EWS_EINVAL, "null argument");
    for (int q = 0; q < NFIELD; ++q) scale[q] = s->scale[q];
    return EWS_OK;
}

ews_status ews_adjoint(ews_sim* s, int nt, double dt, const float* seis_adj, int adj_on_device,
                       float* g_lam, float* g_mu, float* g_rho, int g_on_device,
                       int ckpt_every) {
    if (!s) return fail(EWS_EINVAL, "null simulation");
    if (nt <= 0 || !g_lam || !g_mu || !g_rho) return fail(EWS_EINVAL, "bad arguments");
    if (s->nrec > 0 && !seis_adj) return fail(EWS_EINVAL, "seis_adj is NULL");
    const float* dadj = seis_adj;
    if (s->nrec > 0 && !adj_on_device) {
        const size_t nseis = (size_t)3 * s->nrec * nt;
        ews_status st = ensure_buf(&s->aux, &s->aux_cap, 2 * nseis, "adjoint source");
        if (st != EWS_OK) return st;
        CK(cudaMemcpyAsync(s->aux + nseis, seis_adj, nseis * sizeof(float), cudaMemcpyHostToDevice,
                           s->stream));
        dadj = s->aux + nseis;
    }
    return adjoint_core(s, nt, dt, ckpt_every, dadj, nullptr, nullptr, g_lam, g_mu, g_rho,
                        g_on_device);
}

ews_status ews_gradient(ews_sim* s, int nt, double dt, const float* observed, int obs_on_device,
                        double* misfit, float* g_lam, float* g_mu, float* g_rho,
                        int g_on_device, int ckpt_every) {
    if (!s) return fail(EWS_EINVAL, "null simulation");
    if (nt <= 0 || !g_lam || !g_mu || !g_rho || !observed)
        return fail(EWS_EINVAL, "bad arguments");
    const size_t nseis = (size_t)3 * s->nrec * nt;
    ews_status st = ensure_buf(&s->aux, &s->aux_cap, 3 * (nseis ? nseis : 1), "adjoint source");
    if (st != EWS_OK) return st;
    const float* dobs = observed;
    if (!obs_on_device) {
        CK(cudaMemcpyAsync(s->aux + 2 * nseis, observed, nseis * sizeof(float),
                           cudaMemcpyHostToDevice, s->stream));
        dobs = s->aux + 2 * nseis;
    }
    return adjoint_core(s, nt, dt, ckpt_every, nullptr, dobs, misfit, g_lam, g_mu, g_rho,
                        g_on_device);
}

}  // extern "C"
