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
//   * C-PML memory variables only inside the damping slabs (6 per axis):
//       x slabs [nz][ny][2W], y slabs [nz][2W][pitch], z slabs [2W][ny][pitch].
//   * seismograms [3][nrec][nt] float32; wavelet [nt] float32.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

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
    // memory variables, index 0..2 velocity terms, 3..5 stress terms
    float* psx[6];
    float* psy[6];
    float* psz[6];
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

// Launchers (ews_forward.cu).  All run on `st`.
cudaError_t launch_velocity(const DevGrid& g, const DevFields& F, const DevMedium& M,
                            const DevBoundary& B, float dt, cudaStream_t st);
cudaError_t launch_stress(const DevGrid& g, const DevFields& F, const DevMedium& M,
                          const DevBoundary& B, float dt, cudaStream_t st);
cudaError_t launch_inject(const DevGrid& g, const DevFields& F, const DevMedium& M,
                          const DevBoundary& B, const DevSource& S, const float* wavelet,
                          int n, cudaStream_t st);
cudaError_t launch_record(const DevGrid& g, const DevFields& F, const Tap* taps, int nrec,
                          float* seis, int ld, int n, cudaStream_t st);
cudaError_t launch_medium_setup(const DevGrid& g, float* a, float* b, float* rho,
                                int from_velocities, unsigned* flags_vpmax,
                                cudaStream_t st);

}  // namespace ews
