/*
 * ews.h -- C ABI of libews, a single-GPU (GB300, sm_103a) solver for the 3D
 * elastic velocity-stress staggered-grid finite-difference scheme of
 * "Elastic 3D Wavefield Simulation on budget GPUs using the GLSL shading
 * language" (arXiv 2112.15071).
 *
 * Problem statement (paper Sec. 2.1-2.5):
 *   Eq. 1   rho dv/dt = div sigma + f
 *   Eq. 2   dsigma/dt = C : (grad v + grad v^T) / 2, isotropic C(lambda, mu)
 *   Eq. 4   4th-order staggered first derivative (weights 9/8, -1/24, / h)
 *   Eq. 5   dt_max = 0.495 dx_min / v_max
 *   Sec. 2.1.1  staggered positions (Graves 1996), Sec. 2.2.1 medium by
 *   interpolation at staggered points, Sec. 2.2.2 out-of-range fetches,
 *   Sec. 2.4 receivers by trilinear interpolation, Sec. 2.5 absorbing edges.
 *
 * Conventions shared by every call:
 *   - Every 3D array is C-ordered [nz][ny][nx] (x fastest), float32, dense
 *     (no padding), SI units.  Element [k][j][i] of a staggered field holds
 *     the value at its Sec. 2.1.1 position relative to cell (i, j, k):
 *       sxx, syy, szz at (i, j, k);      vx at (i+1/2, j, k);
 *       sxy at (i+1/2, j+1/2, k);        vy at (i, j+1/2, k);
 *       sxz at (i+1/2, j, k+1/2);        vz at (i, j, k+1/2);
 *       syz at (i, j+1/2, k+1/2).
 *   - Positions are metres from the normal-stress point of cell (0, 0, 0),
 *     z positive downwards.  A source or receiver position p must satisfy
 *     d <= p <= (n - 2) d on every axis (all trilinear neighbours of every
 *     staggered component lie inside the grid).
 *   - Wavefield values outside the grid are zero; medium values are clamped
 *     to the edge (reading of Sec. 2.2.2 / 2.2.1).
 *   - Wavefield state order is (vx, vy, vz, sxx, syy, szz, sxy, sxz, syz);
 *     field bit q of a mask selects field q.
 *   - Ownership: the caller owns every buffer it passes.  set_* calls copy
 *     their inputs (to the device) before returning, so the caller may free
 *     them afterwards.  Output buffers are written in place.  A pointer
 *     flagged *_on_device must be a device pointer of the current CUDA
 *     device (e.g. a torch CUDA tensor); otherwise it is host memory.
 *   - Errors: nothing is thrown across the ABI.  Every call returns an
 *     ews_status; ews_last_error() gives a message (thread-local).  On error
 *     outputs may be partially written and must be discarded.
 *   - Streams: all device work of a simulation runs on its stream (default:
 *     the legacy default stream; see ews_set_stream).  Calls that return data
 *     to host memory synchronise that stream before returning.
 *   - There is no CPU fallback: without a usable CUDA device ews_create
 *     returns EWS_ECUDA.
 */
#ifndef EWS_H
#define EWS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EWS_OK = 0,
    EWS_EINVAL = 1,      /* bad argument (sizes, positions, model values)   */
    EWS_ECFL = 2,        /* dt above the scheme's exact stability bound     */
    EWS_ENOMEM = 3,      /* device allocation failed                        */
    EWS_ECUDA = 4,       /* CUDA runtime or driver error                    */
    EWS_ENONFINITE = 5,  /* NaN/Inf in a model or in the wavefield          */
    EWS_ETIMEOUT = 6,    /* a bounded device wait gave up                   */
    EWS_ESTATE = 7,      /* call out of order (e.g. run before set_model)   */
    EWS_ERANGE = 8       /* a scaled FP16 wavefield value left FP16's range */
} ews_status;

enum { EWS_BOUNDARY_NONE = 0, EWS_BOUNDARY_SPONGE = 1, EWS_BOUNDARY_CPML = 2 };
enum { EWS_STORAGE_F32 = 0, EWS_STORAGE_BF16 = 1, EWS_STORAGE_F16 = 2 };
enum { EWS_SOURCE_MOMENT = 0, EWS_SOURCE_FORCE = 1 };

typedef struct {
    int nx, ny, nz;          /* cells per axis, each >= 4                    */
    double dx, dy, dz;       /* spacing (m), > 0; may differ per axis        */
} ews_grid;

typedef struct {
    /* Absorbing edges (Sec. 2.5).  SPONGE: every field is multiplied after
     * its update by G(i) G(j) G(k), G(d) = exp(-(alpha (W - d) / W)^2) for a
     * cell d < W cells from a face.  CPML: convolutional PML (kappa = 1,
     * quadratic profile, d0 = -3 vp_max ln(R) / (2 W h), alpha_pml = pi f0
     * (1 - q)).  NONE: zero exterior only. */
    int boundary;
    int width;               /* W in cells; 2 W <= n on every axis           */
    /* Storage type of the 9 resident wavefields; arithmetic is FP32 and the
     * medium is always FP32.  BF16 / F16 hold s_q times field q for a
     * per-field power-of-two scale s_q (ews_set_field_scales).  Defaults:
     * s_q = 1 for BF16 (it has FP32's exponent range); for F16, scales
     * derived at each run start from the source amplitude summed over the
     * wavelet and the medium's impedance bounds, mapping that bound to 2^13.
     * Reduced storage is an addition to the method (the paper keeps float
     * textures, Sec. 3); its error is measured, not bounded.  The adjoint
     * (ews_adjoint / ews_gradient) needs F32. */
    int storage;
    int snapshot_every;      /* 0: no snapshots                               */
    unsigned snapshot_mask;  /* fields copied at each snapshot               */
    double sponge_alpha;     /* <= 0 selects 0.3                              */
    double pml_R;            /* <= 0 selects 1e-3                             */
    double pml_f0;           /* Hz, C-PML frequency shift; 0 disables alpha  */
} ews_options;

typedef struct ews_sim ews_sim;

/* Create a simulation on the current CUDA device.  Allocates the 9
 * wavefields (of the storage type) and 3 FP32 medium arrays (and C-PML
 * memory variables, FP32).
 * opt may be NULL (sponge, W = 16).  *out receives the handle. */
ews_status ews_create(const ews_grid* grid, const ews_options* opt, ews_sim** out);

/* Release every device allocation of the simulation.  NULL is ignored. */
void ews_destroy(ews_sim* sim);

/* Run all later device work of sim on this cudaStream_t (NULL = default). */
ews_status ews_set_stream(ews_sim* sim, void* cuda_stream);

/* Medium from Lame parameters and density, each [nz][ny][nx] (Sec. 2.1:
 * lambda, mu, rho define the isotropic medium).  Requires rho > 0, mu >= 0,
 * lambda + 2 mu > 0, all finite; else EWS_EINVAL / EWS_ENONFINITE. */
ews_status ews_set_model_lame(ews_sim* sim, const float* lam, const float* mu,
                              const float* rho, int on_device);

/* Medium from vp, vs, rho (Sec. 3.1.2 table form): lambda = rho (vp^2 -
 * 2 vs^2), mu = rho vs^2, converted on the device. */
ews_status ews_set_model_vel(ews_sim* sim, const float* vp, const float* vs,
                             const float* rho, int on_device);

/* Medium on its own, usually coarser, grid of mx x my x mz cells covering
 * the same box (Sec. 2.2.1: medium textures smaller than the wavefield
 * textures, read with trilinear interpolation).  a, b, rho are dense
 * [mz][my][mx] float32 (host, or device with on_device = 1): lambda, mu if
 * from_velocities = 0, else vp, vs (converted on the device).  The passes
 * sample it at every staggered point instead of reading medium arrays of
 * the wavefield grid: a wavefield-grid position x (cells, per axis) maps to
 * the medium coordinate c = (x + 1/2) m / n - 1/2, clamped to [0, m - 1],
 * and the value is the linear interpolation of the two medium cells around
 * c on each axis (1 / rho at the v points, lambda and mu at the cells, mu
 * at the shear points).  With m = n this equals ews_set_model_lame / _vel.
 * Same validity rules (EWS_EINVAL / EWS_ENONFINITE); vp_max for the
 * stability check is taken over the medium cells.  A later
 * ews_set_model_lame / _vel returns to the wavefield-grid medium.  Not
 * combined with a free surface, gradients or batched shots (EWS_EINVAL). */
ews_status ews_set_model_coarse(ews_sim* sim, int mx, int my, int mz, const float* a,
                                const float* b, const float* rho, int from_velocities,
                                int on_device);

/* Free surface by the vacuum formulation (Sec. 2.5, surface boundary):
 * the cells above plane ks (k < ks) take eps times lambda, mu and rho of the
 * cell (i, j, ks) below the surface in their column (the values the model
 * arrays hold there are ignored); the shear modulus at the xz and yz shear
 * points on the surface plane z = (ks - 1/2) dz is the harmonic mean of
 * their 4 cells (arithmetic means elsewhere); and every z-derivative whose
 * Eq. 4 stencil would take samples on both sides of that plane uses the
 * 2nd-order difference (f(+1/2) - f(-1/2)) / dz instead: outputs at
 * integer z on planes ks-1 and ks, at half-integer z on planes ks-2 .. ks.  ks < 0 removes the surface; 0 <= ks < nz; eps in
 * (0, 1] (1e-3 is a usual value).  The damping of the top face still
 * applies, so the surface is normally placed at or below it (ks >= width).
 * The medium must be set (again) after this call: until then runs return
 * EWS_ESTATE.  Forward runs, gradients (ews_adjoint / ews_gradient: the
 * reverse sweep takes the transposed z-differences and the chain rule of the
 * harmonic means; model values above the surface get a zero gradient) and
 * batched forward and gradient shots support the surface; a fluid cell (mu
 * = 0) below the surface makes the gradient return EWS_EINVAL. */
ews_status ews_set_free_surface(ews_sim* sim, int ks, double eps);

/* Point source.  kind MOMENT: comp = (Mxx, Myy, Mzz, Mxy, Mxz, Myz) in N m
 * (Sec. 3.1.1, Eq. 7 gives such a tensor); each step n the stress pass does
 * sigma_ij -= dt M_ij wavelet[n] / (dx dy dz), spread over the 8 trilinear
 * neighbours on the sigma_ij grid.  wavelet[n] is the moment-rate function
 * at t = (n + 1/2) dt.  kind FORCE: comp = (Fx, Fy, Fz) in N; the velocity
 * pass does v_i += dt b_i F_i wavelet[n] / (dx dy dz) (b = 1 / rho at the v_i
 * point), wavelet[n] at t = n dt.  wavelet has nt float32 samples (host). */
ews_status ews_set_source(ews_sim* sim, int kind, const double pos[3],
                          const double comp[6], const float* wavelet, int nt);

/* Receivers: pos is [nrec][3] metres (host).  Each step records vx, vy, vz
 * of v^{n+1/2}, each trilinearly interpolated on its own staggered grid
 * (Sec. 2.4).  nrec may be 0. */
ews_status ews_set_receivers(ews_sim* sim, int nrec, const double* pos);

/* Reset the wavefields and C-PML memory to zero, then run nt steps of
 * Sec. 2.3's loop: velocity pass (+ force) -> absorbing edge -> record
 * receivers -> stress pass (- moment) -> absorbing edge.
 *   seis      [3][nrec][nt] float32 output (component-major), may be NULL
 *             when nrec == 0; host or device per seis_on_device.
 *   snapshots [nt / snapshot_every][popcount(mask)][nz][ny][nx] float32,
 *             taken after the stress pass of every snapshot_every-th step;
 *             NULL to skip; same residency as seis.
 * dt must satisfy the exact bound dt vp_max (7/3) sqrt(1/dx^2 + 1/dy^2 +
 * 1/dz^2) <= 2 (equal spacings: dt <= 6 / (7 sqrt 3) h / vp_max, Eq. 5's
 * 0.495 rounded), else EWS_ECFL.  nt must not exceed the wavelet length. */
ews_status ews_run(ews_sim* sim, int nt, double dt, float* seis, int seis_on_device,
                   float* snapshots);

/* Continue from the current state: steps n0 .. n0 + nsteps - 1 (wavelet
 * samples n0 ..), recording into columns n0 .. of seis, which is
 * [3][nrec][ld] with ld >= n0 + nsteps.  No reset. */
ews_status ews_advance(ews_sim* sim, int n0, int nsteps, double dt, float* seis,
                       int ld, int seis_on_device);

/* Adjoint gradient (not in the paper, which only runs the forward model;
 * this is the exact reverse of the discrete loop of ews_run).  For a scalar
 * L of the seismograms with dL/dseis = seis_adj ([3][nrec][nt], host or
 * device per adj_on_device), writes dL/dlambda, dL/dmu, dL/drho per cell
 * ([nz][ny][nx] float32 each, host or device per g_on_device).  Runs the
 * forward loop from rest storing the 9 wavefields every ckpt_every steps
 * (0: 50), then steps the adjoint back segment by segment, recomputing each
 * segment's velocity history v^{n+1/2} from its checkpoint.  The trailing
 * segments whose history fits in the history budget (see
 * ews_set_history_budget; by default half the free device memory; at
 * least one segment) keep the history written by the first forward pass
 * and are not recomputed.  Accumulation is FP32
 * within ckpt_every steps and FP64 across them.  Boundaries NONE and SPONGE
 * (C-PML: EWS_EINVAL); F32 storage only.  Extra device memory: checkpoints
 * (nt / ckpt_every) x 9 fields, history max(ckpt_every + 1, budgeted
 * slots) x 3 fields, 17 FP32 + 8 FP64 fields. */
ews_status ews_adjoint(ews_sim* sim, int nt, double dt, const float* seis_adj,
                       int adj_on_device, float* g_lam, float* g_mu, float* g_rho,
                       int g_on_device, int ckpt_every);

/* Element type of the wavefield checkpoints of ews_adjoint / ews_gradient:
 * EWS_STORAGE_F32 (default), EWS_STORAGE_BF16 or EWS_STORAGE_F16 (half the
 * memory).  A 16-bit checkpoint holds s_q times field q, s_q = 2^(14 - e)
 * per field and checkpoint with max |f_q| = m 2^e, m in [0.5, 1) (s_q = 1
 * for a zero field), so FP16 cannot overflow; segments recomputed from a
 * 16-bit checkpoint start from the rounded state, so the gradient differs
 * from the FP32-checkpoint one by about the storage precision.  Resident
 * history (ews_set_history_budget) needs no checkpoints.  Batched shots
 * (ews_batch) take BF16 checkpoints as asked for (without scale: BF16 has
 * FP32's exponent range, and a power-of-two scale does not change its
 * rounding) and keep FP16 ones in FP32.  Not in the paper. */
ews_status ews_set_checkpoint_storage(ews_sim* sim, int storage);

/* Device memory the adjoint may use for resident velocity history, in
 * bytes.  Each resident time step costs 3 fields (12 bytes per cell); with a
 * budget covering all nt steps the gradient needs no recomputation.  0: one
 * segment (every earlier segment recomputed from its checkpoint).  < 0
 * (the default): automatic, half of the device memory free at the call
 * (for ews_batch, that half shared among the gradient shots).  Not in the
 * paper. */
ews_status ews_set_history_budget(ews_sim* sim, double bytes);

/* Gradient of the L2 misfit J = dt/2 sum_(c,r,n) (seis - observed)^2 with
 * respect to lambda, mu, rho (one forward with checkpoints, then the
 * reverse sweep of ews_adjoint with dL/dseis = dt (seis - observed)).
 * observed is [3][nrec][nt] (host or device per obs_on_device); *misfit
 * (may be NULL) receives J. */
ews_status ews_gradient(ews_sim* sim, int nt, double dt, const float* observed,
                        int obs_on_device, double* misfit, float* g_lam, float* g_mu,
                        float* g_rho, int g_on_device, int ckpt_every);

/* Free the working memory the simulation keeps between calls: adjoint
 * state and accumulators, checkpoints, velocity history, seismogram and
 * state staging, the adjoint stencil plan and captured time-loop graphs
 * (the wavefields, medium, source and receivers stay).  Later calls
 * allocate again as needed.  Synchronises the simulation's stream. */
ews_status ews_release_workspace(ews_sim* sim);

/* Zero the wavefields and C-PML memory variables. */
ews_status ews_reset(ews_sim* sim);

/* Copy the 9 wavefields out of / into the simulation, [9][nz][ny][nx]
 * float32 in physical units (16-bit storage is converted with the field
 * scales; set_state returns EWS_ERANGE if a scaled value exceeds FP16). */
ews_status ews_get_state(ews_sim* sim, float* out, int on_device);
ews_status ews_set_state(ews_sim* sim, const float* in, int on_device);

/* Per-field storage scales s[9] (state order) for BF16 / F16 storage: each
 * a positive power of two, so scaling itself never rounds.  Field q is
 * stored as s[q] times its value; stencil derivatives are formed on stored
 * values and multiplied by 1 / s[input field], updates by dt s[output
 * field].  scale = NULL restores the defaults (see ews_options.storage).
 * With F32 storage only all-ones is accepted.  Zeroes the wavefields (as
 * ews_reset) so no field is ever read at another scale than it was
 * written with.  This has no counterpart in the paper. */
ews_status ews_set_field_scales(ews_sim* sim, const float* scale);
/* The scales in use (after a run: the ones that run used). */
ews_status ews_get_field_scales(ews_sim* sim, float* scale);

/* ---- Tile shape of the forward passes (not in the paper) ----
 * The velocity and stress passes march tiles of cells through z; the tile
 * shape that runs fastest depends on the grid, the boundary and the storage
 * type (on a GB300 at 256^3: 32 x 8 with C-PML, 32 x 4 for FP32 with a
 * sponge, 32 x 16 for BF16 with a sponge).  Every shape runs the same
 * arithmetic per cell in the same order (separately compiled, so results
 * agree to FP32 rounding).  EWS_TILE_FUSED runs both passes of a step in one
 * launch (32 x 8 tiles, the velocity of a 2-cell ring around each tile
 * recomputed by its neighbours), reading one set of wavefields and writing a
 * second one that the library allocates (9 more wavefields of device
 * memory, released when the tuner picks another shape); it serves FP32
 * storage at unit field scales with a sponge or no absorbing boundary, and
 * other runs fall back to 32 x 8.  It moves 84 bytes per cell instead of
 * 120 but recomputes the ring, so on a GB300 it is bound by instruction
 * issue and runs slower than the two passes (0.78x at 256^3, 0.89x at
 * 1024 x 1024 x 512); the tuner times it where the second set takes at
 * most a quarter of the free device memory.  With EWS_TILE_AUTO (the default),
 * ews_run picks the shape for its grid size, boundary and storage type from
 * a per-process table, filling a missing entry by timing a few steps with
 * each shape before the run (the wavefields are reset afterwards); plain
 * forward steps use it (runs with a free surface or a coarse medium grid,
 * the adjoint's forward part and batched shots keep 32 x 8). */
enum {
    EWS_TILE_AUTO = 0,
    EWS_TILE_32X8 = 1,
    EWS_TILE_32X4 = 2,
    EWS_TILE_32X16 = 3,
    EWS_TILE_FUSED = 4
};

/* Use this shape for later runs (EWS_TILE_AUTO: the tuned one). */
ews_status ews_set_tile_shape(ews_sim* sim, int shape);
/* The shape the forward passes of the last run used (EWS_TILE_32X8 ..
 * EWS_TILE_FUSED). */
int ews_get_tile_shape(ews_sim* sim);

/* Tile-shape table, one entry per grid size, boundary and storage type;
 * can be exported and imported so that a tuning outlives the process (the
 * Python binding stores it with the z-chunk table).  Host memory only. */
typedef struct {
    int nx, ny, nz;           /* wavefield grid                                      */
    int boundary;             /* EWS_BOUNDARY_*                                      */
    int storage;              /* EWS_STORAGE_*                                       */
    int shape;                /* EWS_TILE_32X8 .. EWS_TILE_FUSED                     */
} ews_tuned_tile;

/* Shape of the table entry for a grid (0 if not tuned yet). */
int ews_tile_tuned(const ews_grid* grid, int boundary, int storage);
/* Copy up to cap entries into out; returns the number of entries. */
int ews_tile_tuning_export(ews_tuned_tile* out, int cap);
/* Add entries (replacing entries with the same key); any invalid entry gives
 * EWS_EINVAL and nothing is imported. */
ews_status ews_tile_tuning_import(const ews_tuned_tile* in, int n);
/* Empty the table. */
void ews_tile_tuning_clear(void);

/* Kernel classes for launch counting and timing. */
enum {
    EWS_KERNEL_VELOCITY = 0,   /* velocity pass, Eq. 1 (+ absorbing edge)      */
    EWS_KERNEL_STRESS = 1,     /* stress pass, Eq. 2 (+ absorbing edge)        */
    EWS_KERNEL_INJECT = 2,     /* point-source injection                       */
    EWS_KERNEL_RECORD = 3,     /* receiver sampling, Sec. 2.4                  */
    EWS_KERNEL_POINTS = 4,     /* moment injection + receivers in one launch   */
    EWS_KERNEL_STEP = 5,       /* velocity + stress passes in one launch       */
    EWS_NKERNEL = 8
};

/* When on, every kernel launch of the simulation is bracketed by CUDA
 * events on its stream and its duration accumulated per class.  Launch
 * counts are accumulated whether or not timing is on. */
ews_status ews_set_profiling(ews_sim* sim, int on);

/* Accumulated milliseconds and launch counts per kernel class since the
 * last reset (arrays of EWS_NKERNEL entries; either may be NULL).  If reset
 * is nonzero the accumulators are zeroed after reading. */
ews_status ews_get_profile(ews_sim* sim, double* ms, long long* launches, int reset);

/* Limits of ews_forward_noalloc. */
#define EWS_NOALLOC_MAX_CELLS (1 << 18)   /* nx rounded up to 32, times ny, times nz */
#define EWS_NOALLOC_MAX_DIM 1024          /* cells per axis                          */
#define EWS_NOALLOC_MAX_RECEIVERS 64

/* Forward run that allocates no memory (the paper has no counterpart: this
 * is a service for callers).  Some callers cannot let a library call
 * cudaMalloc: their device memory belongs to another allocator (a
 * framework's caching allocator, a fixed pool in a long-running service)
 * that must not be grown or fragmented behind its back, or they cannot take
 * the device-wide synchronisation that cudaFree implies.  This call runs the
 * same loop as ews_create + ews_set_* + ews_run, with the same kernels, but
 * keeps every wavefield, the pitched medium copies, the sponge profiles and
 * the receiver taps in one static device array of about 12 MiB that every
 * GPU loading the library holds until the process exits.
 *   lam, mu, rho  device pointers, dense [nz][ny][nx] float32 (caller-owned)
 *   wavelet       device pointer, >= nt float32 samples (as ews_set_source)
 *   rec_pos       host [nrec][3] metres, nrec <= EWS_NOALLOC_MAX_RECEIVERS
 *   seis          device [3][nrec][nt] float32 output (caller-owned)
 *   opt           NULL (sponge, W = 16) or boundary NONE / SPONGE; C-PML is
 *                 rejected (its memory variables would not fit); snapshot
 *                 fields are ignored.
 * Sizes beyond EWS_NOALLOC_MAX_CELLS / _DIM / _RECEIVERS give EWS_EINVAL
 * with a message naming the limit.  The first call on each device looks up
 * the device address of the static array (cudaGetSymbolAddress, with that
 * device current); make it before capturing any stream on that device.
 * Every call shares the one array and starts by clearing the wavefields, so
 * results do not depend on earlier calls, but calls that overlap on the GPU
 * (other streams or host threads) race on it.  The call synchronises
 * `cuda_stream` (NULL = default stream) before returning, on success and on
 * every error found after its first device operation, so no work of a
 * failed call is left writing the shared array.  Host threads may make
 * their first calls concurrently; the host-side staging is a few KB of
 * stack plus thread-local storage. */
ews_status ews_forward_noalloc(const ews_grid* grid, const ews_options* opt,
                               const float* lam, const float* mu, const float* rho,
                               int src_kind, const double pos[3], const double comp[6],
                               const float* wavelet, int nrec, const double* rec_pos,
                               int nt, double dt, float* seis, void* cuda_stream);

/* ---- Batched shots (not in the paper, which runs one model at a time) ----
 * Many independent shots, each a configured simulation (model, source and
 * receivers set; F32 storage; the same boundary for all shots; C-PML for
 * forward shots only), run forward - and, when observed data are given,
 * through the L2 misfit gradient of ews_gradient - in persistent kernel
 * launches replayed as one CUDA graph: one launch for the forward shots
 * and the forward part of the gradient shots, then per segment of the
 * reverse sweep a recomputation launch and a reverse launch.  A launch
 * takes work items (a 32 x 8 x zchunk tile of a pass, a chunk of cells, or
 * a source/receiver step) of all shots from a device queue; an item waits
 * (bounded, EWS_ETIMEOUT) until its shot's earlier stages are done, so
 * shots of uneven size and step count share the GPU without a grid-wide
 * barrier.  Results equal those of ews_run / ews_gradient on each
 * simulation alone (bitwise for the forward, to accumulation order for the
 * gradient). */
typedef struct {
    ews_sim* sim;             /* configured simulation, used exclusively by this call */
    int nt;                   /* steps (<= the wavelet length)                        */
    double dt;                /* time step (checked like ews_run)                     */
    float* seis;              /* device [3][nrec][nt] output, or NULL                 */
    const float* observed;    /* device [3][nrec][nt]: also compute the gradient      */
    float* g_lam;             /* device dense [nz][ny][nx] outputs when observed set  */
    float* g_mu;
    float* g_rho;
    double misfit;            /* out: J = dt/2 sum (seis - observed)^2                */
} ews_batch_shot;

enum { EWS_BATCH_PERSISTENT = 0, EWS_BATCH_SEQUENTIAL = 1 };

typedef struct {
    int mode;                 /* EWS_BATCH_PERSISTENT, or EWS_BATCH_SEQUENTIAL: each
                               * shot through ews_run / ews_gradient in turn (the
                               * one-by-one reference)                                 */
    int ckpt_every;           /* gradient checkpoint interval (0: 50)                 */
    int zchunk;               /* planes per tile in z; 0: picked per grid size by the
                               * autotuner (timed trial launches; see the table below) */
    int ctas_per_sm;          /* resident CTAs per SM to launch (0: as many as fit)   */
    int dep_wait_ms;          /* give-up time of one dependency wait (0: 4000 ms)     */
    int test_unsatisfiable;   /* testing only: the last item waits for an item that
                               * never exists, so the launch must end in EWS_ETIMEOUT */
} ews_batch_options;

/* Run nshots shots; opt may be NULL (persistent, autotuned).  All device
 * work runs on cuda_stream (NULL: default stream), which is synchronised
 * before return.  Errors: EWS_EINVAL (mixed boundaries, C-PML gradient
 * shots, 16-bit storage, coarse medium grids, fluid cells for gradients,
 * missing outputs), EWS_ECFL, EWS_ENOMEM, EWS_ETIMEOUT (a dependency or
 * pipeline wait gave up), EWS_ECUDA. */
ews_status ews_batch(int nshots, ews_batch_shot* shots, const ews_batch_options* opt,
                     void* cuda_stream);

/* One iteration of multi-shot full-waveform inversion on one model (not
 * in the paper, which only runs the forward model; its case study is many
 * stations for one earthquake).  All shots share one grid; each shot's
 * simulation has its source and receivers set and `observed` data
 * (device [3][nrec][nt]); their g_* and seis fields are ignored.  lam, mu,
 * rho: device dense [nz][ny][nx], the current model, replaced by the
 * updated one.  The iteration: L2 misfit and gradients of all shots in one
 * batched launch (ews_batch), their sum g, the direction d = -s_p g_p with
 * s_p = max|m_p| / max|g_p| per parameter, misfits of batched forward runs
 * at steps max_rel_step and max_rel_step / 2 and at the minimum of the
 * parabola through those and J(0) (within [0.1, 2] max_rel_step), and the
 * model of the smallest misfit, if smaller than J(0) (else the model is
 * kept and *step = 0).  Trial models keep rho and mu at least half, and the
 * bulk modulus at least half, of their current values.  Outputs: *misfit0
 * = J at the current model, *misfit1 = J at the returned model, *step = the
 * accepted step.  Every simulation ends holding the returned model. */
ews_status ews_fwi_iteration(int nshots, ews_batch_shot* shots, float* lam, float* mu,
                             float* rho, double max_rel_step, int ckpt_every, double* misfit0,
                             double* misfit1, double* step, void* cuda_stream);

/* Autotuner table.  ews_batch with zchunk = 0 picks the planes per tile in
 * z for each grid from timed trial launches of the forward executor (the
 * choice serves forward and gradient shots of that grid) and keeps it for
 * the life of the process, one entry per grid size, boundary kind and
 * surface form (shots with a free surface run other kernel forms).  A
 * batch of several shots then also times the first forward steps with
 * longer z-chunks (64 and 128 planes, whole tile columns) against the
 * table's values and keeps the fastest for all its launches, cached per
 * batch composition (not part of the table; cleared with it).  The table can be exported and imported, so
 * that a tuning persists across processes (the Python binding stores it
 * as JSON); entries are specific to the GPU they were timed on.  All four
 * calls touch host memory only. */
typedef struct {
    int nx, ny, nz;           /* wavefield grid                                      */
    int boundary;             /* EWS_BOUNDARY_*                                      */
    int free_surface;         /* 1: entry of shots with a free surface, else 0       */
    int zchunk;               /* planes per tile in z, 1 .. nz                       */
} ews_tuned_zchunk;

/* zchunk of the table entry for a grid (0 if not tuned yet). */
int ews_batch_tuned_zchunk(const ews_grid* grid, int boundary, int free_surface);

/* Copy up to cap entries into out (ordered by nx, ny, nz, boundary,
 * surface form); returns the number of entries in the table (out may be
 * NULL to count them). */
int ews_batch_tuning_export(ews_tuned_zchunk* out, int cap);

/* Add n entries to the table, replacing entries with the same key.  All
 * entries are checked first (sizes >= 1, a known boundary, free_surface 0
 * or 1, 1 <= zchunk <= nz); any invalid one gives EWS_EINVAL and nothing is
 * imported. */
ews_status ews_batch_tuning_import(const ews_tuned_zchunk* in, int n);

/* Empty the table (the next ews_batch with zchunk = 0 tunes again). */
void ews_batch_tuning_clear(void);

/* ---- Device memory held by the library (not in the paper) ----
 * Every device allocation libews makes (simulations, adjoint state,
 * checkpoints, velocity history, batch and inversion buffers) is counted.
 * ews_set_memory_limit caps the total, process-wide and over all devices:
 * an allocation that would take the count above `bytes` fails before CUDA
 * is asked, exactly as when the device is full -- the call returns
 * EWS_ENOMEM, releases what it had set up and leaves the simulation (and the
 * CUDA context) usable, and ews_last_error names the limit.  The automatic
 * history budget of the adjoint stays within the room the limit leaves.
 * bytes < 0 removes the limit (the default); a limit below the current use
 * only refuses later allocations.  NaN gives EWS_EINVAL.  Host-only calls.
 * (ews_forward_noalloc allocates nothing and is not counted.) */
ews_status ews_set_memory_limit(double bytes);
/* The limit in force (< 0: none). */
double ews_memory_limit(void);
/* Bytes of device memory the library holds now. */
double ews_memory_in_use(void);

/* Time-step rule of Sec. 2.1.3, Eq. 5: 0.495 min(dx, dy, dz) / vmax. */
double ews_cfl_dt(const ews_grid* grid, double vmax);

/* Source-frequency rule of Sec. 2.1.3, Eq. 6: vmin / (5 max(dx, dy, dz)). */
double ews_max_freq(const ews_grid* grid, double vmin);

/* Message of the last error on this thread ("" if none). */
const char* ews_last_error(void);

/* ABI version (major * 100 + minor). */
int ews_version(void);

#ifdef __cplusplus
}
#endif
#endif /* EWS_H */
