// ews_internal.cuh -- device data structures and kernel launchers of libews.
//
// Layout in HBM (one simulation):
//   * 9 wavefields in one allocation, each [nz][ny][pitch] float32 with
//     pitch = nx rounded up to 32 floats (128-byte rows, 16-byte aligned for
//     vector and TMA access).  Padding columns stay zero and are never
//     written.  Field q starts at base + q * fstride (fstride a multiple of
//     64 floats).
//   * lambda, mu, rho per cell in a second allocation, same layout.  The
//     staggered-point means of Sec. 2.2.1 are formed in registers by the
//     stencil kernels; nothing else about the medium is stored.
//   * C-PML memory variables: 18 arrays with the field layout (6 per damped
//       direction); only slab cells are used, so stencil tiles can bring
//       them in with the same TMA boxes as the fields.
//   * seismograms [3][nrec][nt] float32; wavelet [nt] float32.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ews.h"

namespace ews {

enum { VX, VY, VZ, SXX, SYY, SZZ, SXY, SXZ, SYZ, NFIELD };
enum { BND_NONE = 0, BND_SPONGE = 1, BND_CPML = 2 };

struct DevGrid {
    int nx, ny, nz;
    int pitch;            // floats per row
    long long plane;      // floats per z-plane = pitch * ny
    // Eq. 4 weights divided by the axis spacing (reading: the 1/h factor)
    float c1x, c2x, c1y, c2y, c1z, c2z;
};

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

// Adjoint state (ews_adjoint.cu): P velocity-like (true adjoint = G P),
// Q stress-like, FP32 per-segment accumulators and FP64 totals:
// acc[0] lambda, [1] mu at normal points, [2..4] mu at xy/xz/yz shear points,
// [5..7] buoyancy at vx/vy/vz points.
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

// Thread-local error message for ews_last_error() (ews_capi.cu).
ews_status report(ews_status s, const char* fmt, ...);

// Stencil passes (ews_stencil.cu): TMA tensor maps and launch geometry are
// built once per simulation (the field and medium addresses never change).
struct StencilPlan;
cudaError_t stencil_plan_create(const DevGrid& g, const DevFields& F, const DevMedium& M,
                                const DevBoundary& B, StencilPlan** out);
void stencil_plan_destroy(StencilPlan* p);
size_t stencil_plan_bytes();
cudaError_t stencil_plan_fill(void* storage, const DevGrid& g, const DevFields& F,
                              const DevMedium& M, const DevBoundary& B, StencilPlan** out);
cudaError_t launch_velocity(const StencilPlan* sp, const DevGrid& g, const DevFields& F,
                            const DevBoundary& B, float dt, int* err, cudaStream_t st);
cudaError_t launch_stress(const StencilPlan* sp, const DevGrid& g, const DevFields& F,
                          const DevBoundary& B, float dt, int* err, cudaStream_t st);

// Sources, receivers and medium set-up (ews_forward.cu).  All run on `st`.
cudaError_t launch_inject(const DevGrid& g, const DevFields& F, const DevMedium& M,
                          const DevBoundary& B, const DevSource& S, const float* wavelet,
                          int n, cudaStream_t st);
cudaError_t launch_record(const DevGrid& g, const DevFields& F, const Tap* taps, int nrec,
                          float* seis, int ld, int n, cudaStream_t st);
cudaError_t launch_medium_setup(const DevGrid& g, float* a, float* b, float* rho,
                                int from_velocities, unsigned* flags_vpmax,
                                cudaStream_t st);

}  // namespace ews
