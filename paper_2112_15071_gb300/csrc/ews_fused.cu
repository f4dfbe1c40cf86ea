// ews_fused.cu -- one launch per time step: the velocity pass (Eq. 1) and the
// stress pass (Eq. 2/3) of Sec. 2.3 fused, for FP32 wavefields with a sponge
// or no absorbing boundary.
//
// The two-pass step moves 120 bytes per cell (velocity: 10 reads, 3 writes;
// stress: 11 reads, 6 writes).  This step reads sigma^n, v^{n-1/2} and the
// medium once and writes v^{n+1/2} and sigma^{n+1} once: 84 bytes.  To need
// no exchange between CTAs it reads from one set of wavefields (A) and
// writes to a second set (B), so nothing a neighbour still reads is ever
// overwritten, and each CTA computes the new velocity on its 32 x 8 tile
// plus the 2-cell ring its stress differences reach (36 x 12 cells, the ring
// computed redundantly by the neighbours too) and on 2 planes above and below
// its z-chunk.  The ring's velocity stays in shared memory; the CTA writes
// only its own cells and planes.
//
// Pipeline per CTA (tile x0, y0; z-chunk z0 .. z1): plane p of sigma^n,
// v^{n-1/2} and rho arrives in a 4-slot TMA ring (boxes over the 36 x 12
// velocity region and its halo).  Thread (tx, ty) owns tile cell (x0 + tx,
// y0 + ty); threads below 176 also own one cell of the ring.  At arrival p
// each thread computes the new velocity of plane kv = p - 2 at its cells
// (z-derivatives from per-thread register queues) into a 4-plane shared
// ring; after one barrier, the stress of plane ks = kv - 2 at its tile cell
// (x / y differences of the new velocity from the shared ring, z-differences
// and sigma^n of the cell from register queues, lambda and mu from a
// 3-entry TMA buffer).  One barrier per plane: the 4-plane ring keeps a
// plane until every thread has passed the next barrier after its last
// reader, and the TMA refills of a slot or an entry go out after the barrier
// that follows its last use.  Every mbarrier wait is bounded.  A point force
// (Sec. 2.4 source term of Eq. 1) is added to the new velocity of its tap
// cells before the stress uses them; a moment source and the receivers run
// after the step, on B, as in the two-pass loop.  The arithmetic per cell is
// that of the two passes.
#define EWS_TILE_Y 8
#define EWS_ROWS 1
#define EWS_SHAPE_NS fused
#include "ews_stencil.cu"

namespace ews {
namespace fused {
namespace {

constexpr int EX = TX + 4, EY = TY + 4;          // velocity region: x0-2 .. x0+33, y0-2 .. y0+9
constexpr int NE = EX * EY;                      // 432 cells
constexpr int NRING = NE - CORE;                 // 176 ring cells
constexpr int BW = TX + 8;                       // box width (x from x0-4: 16-byte aligned)
// slot: sxx sxz (x halos, rows y0-2..y0+9), syy syz (y halos, rows y0-4..y0+11),
// sxy (both), szz vx vy vz (the region), rho (the region + 1 row / column)
constexpr int XB = BW * EY * 4, YB = BW * (EY + 4) * 4, ZB = BW * EY * 4, RB = BW * (EY + 1) * 4;
constexpr int O_XP = 0, O_YP = O_XP + 2 * XB, O_XY = O_YP + 2 * YB, O_ZV = O_XY + YB;
constexpr int O_RHO = O_ZV + 4 * ZB, FSLOT = r128(O_RHO + RB);
constexpr int F_TX = 2 * XB + 3 * YB + 4 * ZB + RB;
static_assert(O_YP % 128 == 0 && O_XY % 128 == 0 && O_ZV % 128 == 0 && O_RHO % 128 == 0,
              "TMA destinations 128-byte aligned");
// stress-side entries: lambda (core tile) and mu (box x0-4.., y0..y0+8)
constexpr int LB = CORE * 4, MUB = BW * (TY + 1) * 4, SENT = r128(LB + MUB), NSENT = 3;
constexpr int NVN = 4;                           // planes of the new-velocity ring
constexpr int VNEW = 3 * NE * 4;                 // new velocity of one plane over the region
constexpr int F_SMEM = NSLOT * FSLOT + NSENT * SENT + NVN * VNEW + 8 * (NSLOT + NSENT);
static_assert(2 * (F_SMEM + 1024) <= 227 * 1024, "two CTAs per SM");

struct FusedMaps {
    CUtensorMap xp, yp, xy, zv, rho, lam, mu;
};

struct FusedParams {
    DevGrid g;
    DevFields fin, fout;        // sigma^n, v^{n-1/2} from fin; v^{n+1/2}, sigma^{n+1} to fout
    DevMedium M;
    DevBoundary B;
    float dt;
    int ntx, nty, zchunk;
    int* err;
    DevSource S;                // force taps (kind 1) of this step; else ntap 0
    const float* wavelet;
    int n;
    int sk0, sk1;               // planes of the force taps
};

__device__ __forceinline__ void issue_v(const FusedMaps& m, unsigned char* slot, uint64_t* bar,
                                        int x0, int y0, int z) {
    mbar_expect_tx(bar, (uint32_t)F_TX);
    tma_load_4d(slot + O_XP, &m.xp, bar, x0 - 4, y0 - 2, z, fslot(SXX));      // sxx sxz
    tma_load_4d(slot + O_YP, &m.yp, bar, x0 - 4, y0 - 4, z, fslot(SYY));      // syy syz
    tma_load_3d(slot + O_XY, &m.xy, bar, x0 - 4, y0 - 4, z);                  // sxy
    tma_load_4d(slot + O_ZV, &m.zv, bar, x0 - 4, y0 - 2, z, fslot(SZZ));      // szz vx vy vz
    tma_load_3d(slot + O_RHO, &m.rho, bar, x0 - 4, y0 - 2, z);
}
__device__ __forceinline__ void issue_s(const FusedMaps& m, unsigned char* ent, uint64_t* bar,
                                        int x0, int y0, int z) {
    mbar_expect_tx(bar, (uint32_t)(LB + MUB));
    tma_load_3d(ent, &m.lam, bar, x0, y0, z);
    tma_load_3d(ent + LB, &m.mu, bar, x0 - 4, y0, z);
}

// Per-thread queues.  Cell 0 is the thread's tile cell, cell 1 its ring cell.
struct FQ {
    float zz[2][4], xz[2][4], yz[2][4];          // sigma z-queues of the two cells
    float vx[4], vy[4], vz[4];                   // new-velocity z-queues of the tile cell
    float sg[2][6];                              // sigma^n of the tile cell, planes by parity
    float vzp;                                   // new vz of the tile cell, previous plane
    bool bad;                                    // a stress-side wait gave up
};

template <int BND>
struct FGeo {
    int x0, y0, z0, z1, ke;                      // medium planes z0 .. ke - 1 for the stress
    int e[2];                                    // region index of the cells
    int ox[2], oy[2];                            // offsets in the x-row / y-row boxes
    int cxr[2], cyr[2];                          // rho +x / +y offsets (clamped at the top edges)
    bool in[2];                                  // the cell lies inside the grid (x, y)
    bool ring;                                   // the thread has a ring cell
    float gx[2], gy[2];                          // sponge gains G(i), G(j)
    int ci[2], cj[2];                            // grid i, j of the cells
    int mcx, mcy;                                // mu +x / +y offsets of the tile cell (clamped)
    __device__ __forceinline__ FGeo(const FusedParams& P, int item) {
        const DevGrid& g = P.g;
        const int ntile = P.ntx * P.nty;
        const int t = item % ntile;
        z0 = (item / ntile) * P.zchunk;
        z1 = min(g.nz, z0 + P.zchunk);
        ke = min(z1 + 1, g.nz);
        x0 = (t % P.ntx) * TX;
        y0 = (t / P.ntx) * TY;
        const int tid = threadIdx.y * TX + threadIdx.x;
        ring = tid < NRING;
        // ring cells: rows 0, 1, TY+2, TY+3 of the region, then columns 0, 1,
        // TX+2, TX+3 of rows 2 .. TY+1
        int rx, ry;
        if (tid < 4 * EX) {
            const int q = tid / EX;
            rx = tid % EX;
            ry = q < 2 ? q : q + TY;
        } else {
            const int s = min(tid, NRING - 1) - 4 * EX;
            ry = 2 + s / 4;
            rx = (s & 3) < 2 ? (s & 3) : (s & 3) + TX;
        }
        const int exs[2] = {(int)threadIdx.x + 2, rx}, eys[2] = {(int)threadIdx.y + 2, ry};
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int ex = exs[c], ey = eys[c];
            e[c] = ey * EX + ex;
            ci[c] = x0 - 2 + ex;
            cj[c] = y0 - 2 + ey;
            in[c] = (c == 0 || ring) && ci[c] >= 0 && ci[c] < g.nx && cj[c] >= 0 && cj[c] < g.ny;
            ox[c] = ey * BW + ex + 2;
            oy[c] = (ey + 2) * BW + ex + 2;
            cxr[c] = (ci[c] + 1 < g.nx) ? 1 : 0;
            cyr[c] = (cj[c] + 1 < g.ny) ? BW : 0;
            gx[c] = (BND == BND_SPONGE && in[c]) ? __ldg(P.B.g[0] + ci[c]) : 1.0f;
            gy[c] = (BND == BND_SPONGE && in[c]) ? __ldg(P.B.g[1] + cj[c]) : 1.0f;
        }
        mcx = (ci[0] + 1 < g.nx) ? 1 : 0;
        mcy = (cj[0] + 1 < g.ny) ? BW : 0;
    }
};

// Plane k of the stress-side medium buffer: entry k mod 3, filled for the
// ((k - z0) / 3)-th time.
__device__ __forceinline__ int sent_of(int k) { return ((k % NSENT) + NSENT) % NSENT; }

// Bounded-failure exit of thread 0 at the barrier of arrival m (m = number
// of arrivals after the last one): record, then wait (bounded) for the
// copies still in flight -- ring arrivals m .. issued - 1, and the last
// filling of each medium-buffer entry -- so the CTA leaves no copy into its
// shared memory behind.
__device__ __noinline__ void fused_fail(int* err, uint64_t* bars, int m, int z0, int z1, int ke) {
    atomicOr(err, 1);
    const int P8 = z1 - z0 + 8;
    const int issued = min(P8, max(NSLOT, m + 2));
    for (int q = m; q < issued; ++q)
        if (!mbar_wait(&bars[q & (NSLOT - 1)], (uint32_t)((q >> 2) & 1))) return;
    // medium planes issued: z0 .. last (after the barrier of arrival m',
    // plane z0 - 9 + m' is refilled with plane z0 - 6 + m')
    const int last = min(ke - 1, max(z0 + NSENT - 1, z0 + m - 7));
    for (int k = max(z0, last - NSENT + 1); k <= last; ++k)
        if (!mbar_wait(&bars[NSLOT + sent_of(k)], (uint32_t)(((k - z0) / NSENT) & 1))) return;
}

// New velocity (Eq. 1) of region cell c at plane kv, from the slot of plane
// kv (sl2), rho of plane kv + 1 (sl1) and the sigma z-queues.
template <int BND, int PH, int c>
__device__ __forceinline__ void vel_cell(const FusedParams& P, const FGeo<BND>& G, const FQ& Q,
                                         const float* sl1, const float* sl2, bool ktop, float gz,
                                         float& vx, float& vy, float& vz, float* sn) {
    const DevGrid& g = P.g;
    constexpr int A = (PH + 1) & 3, B = (PH + 2) & 3, C = (PH + 3) & 3, D = PH;  // oldest..newest
    const float* hxx = sl2 + O_XP / 4 + G.ox[c];
    const float* hxz = hxx + XB / 4;
    const float* hyy = sl2 + O_YP / 4 + G.oy[c];
    const float* hyz = hyy + YB / 4;
    const float* hxy = sl2 + O_XY / 4 + G.oy[c];
    const float* vc = sl2 + O_ZV / 4 + G.ox[c];
    const float* hr = sl2 + O_RHO / 4 + G.ox[c];
    const float* hr1 = sl1 + O_RHO / 4 + G.ox[c];                  // plane kv + 1
    const float* qxz = Q.xz[c];
    const float* qyz = Q.yz[c];
    const float* qzz = Q.zz[c];
    // vx at (i+1/2, j, k)
    const float dxx = g.c1x * (hxx[1] - hxx[0]) + g.c2x * (hxx[2] - hxx[-1]);
    const float dxy = g.c1y * (hxy[0] - hxy[-BW]) + g.c2y * (hxy[BW] - hxy[-2 * BW]);
    const float dxz = g.c1z * (qxz[C] - qxz[B]) + g.c2z * (qxz[D] - qxz[A]);
    // vy at (i, j+1/2, k)
    const float dyx = g.c1x * (hxy[0] - hxy[-1]) + g.c2x * (hxy[1] - hxy[-2]);
    const float dyy = g.c1y * (hyy[BW] - hyy[0]) + g.c2y * (hyy[2 * BW] - hyy[-BW]);
    const float dyz = g.c1z * (qyz[C] - qyz[B]) + g.c2z * (qyz[D] - qyz[A]);
    // vz at (i, j, k+1/2)
    const float dzx = g.c1x * (hxz[0] - hxz[-1]) + g.c2x * (hxz[1] - hxz[-2]);
    const float dzy = g.c1y * (hyz[0] - hyz[-BW]) + g.c2y * (hyz[BW] - hyz[-2 * BW]);
    const float dzz = g.c1z * (qzz[C] - qzz[B]) + g.c2z * (qzz[D] - qzz[A]);
    if (c == 0) {               // sigma^n of the tile cell, for its stress two planes later
        sn[0] = hxx[0];         // sxx
        sn[1] = hyy[0];         // syy
        sn[2] = qzz[B];         // szz (plane kv)
        sn[3] = hxy[0];         // sxy
        sn[4] = hxz[0];         // sxz
        sn[5] = hyz[0];         // syz
    }
    // buoyancy at the v points: 1 / mean of the two adjacent densities
    const float r0 = hr[0];
    const float bx = __fdividef(2.0f, r0 + hr[G.cxr[c]]);
    const float by = __fdividef(2.0f, r0 + hr[G.cyr[c]]);
    const float bz = __fdividef(2.0f, r0 + (ktop ? hr1[0] : r0));
    vx = vc[1 * (ZB / 4)] + P.dt * bx * (dxx + dxy + dxz);
    vy = vc[2 * (ZB / 4)] + P.dt * by * (dyx + dyy + dyz);
    vz = vc[3 * (ZB / 4)] + P.dt * bz * (dzx + dzy + dzz);
    if (BND == BND_SPONGE) {
        const float Gs = G.gx[c] * gz * G.gy[c];
        vx *= Gs; vy *= Gs; vz *= Gs;
    }
}

// One arrival of the fused pipeline, ring position PH = m mod 4: plane
// p = z0 - 4 + m lands; new velocity of plane kv = p - 2; stress of plane
// ks = kv - 2.  Returns false if the CTA must stop (a wait gave up).
template <int BND, int PH>
__device__ __forceinline__ bool fused_step(const FusedMaps& maps, const FusedParams& P,
                                           const FGeo<BND>& G, FQ& Q, unsigned char* sm,
                                           uint64_t* bars, int m) {
    const DevGrid& g = P.g;
    constexpr int S0 = PH, S1 = (PH + 3) & 3, S2 = (PH + 2) & 3;     // planes p, p-1, p-2
    constexpr int A = (PH + 1) & 3, B = (PH + 2) & 3, C = (PH + 3) & 3, D = PH;
    constexpr int SQ = PH & 1;                                       // sigma^n queue entry
    const int P8 = G.z1 - G.z0 + 8;
    const int p = G.z0 - 4 + m, kv = p - 2, ks = kv - 2;
    const bool dov = m >= 4, dos = m >= 8 && ks < G.z1;
    unsigned char* sent = sm + NSLOT * FSLOT;
    float* vnew = reinterpret_cast<float*>(sent + NSENT * SENT);
    uint64_t* sbars = bars + NSLOT;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const float gz = (BND == BND_SPONGE && dov && kv >= 0 && kv < g.nz) ? __ldg(P.B.g[2] + kv) : 1.0f;
    const float gzs = (BND == BND_SPONGE && dos) ? __ldg(P.B.g[2] + ks) : 1.0f;
    const bool ok = mbar_wait(&bars[S0], (uint32_t)((m >> 2) & 1));
    const float* sl0 = reinterpret_cast<const float*>(sm + S0 * FSLOT);
    const float* sl1 = reinterpret_cast<const float*>(sm + S1 * FSLOT);
    const float* sl2 = reinterpret_cast<const float*>(sm + S2 * FSLOT);
    // sigma_zz of plane p, sigma_xz / sigma_yz of plane p - 1
    Q.zz[0][PH] = sl0[O_ZV / 4 + G.ox[0]];
    if (m > 0) {
        Q.xz[0][PH] = sl1[O_XP / 4 + XB / 4 + G.ox[0]];
        Q.yz[0][PH] = sl1[O_YP / 4 + YB / 4 + G.oy[0]];
    }
    if (G.ring) {
        Q.zz[1][PH] = sl0[O_ZV / 4 + G.ox[1]];
        if (m > 0) {
            Q.xz[1][PH] = sl1[O_XP / 4 + XB / 4 + G.ox[1]];
            Q.yz[1][PH] = sl1[O_YP / 4 + YB / 4 + G.oy[1]];
        }
    }
    // ---- new velocity of plane kv at the thread's cells ----
    float* vn = vnew + (kv & (NVN - 1)) * 3 * NE;
    float vx0 = 0.f, vy0 = 0.f, vz0 = 0.f;
    float sn[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (dov && ok) {
        const bool kin = kv >= 0 && kv < g.nz;
        const bool ktop = kv + 1 < g.nz;
        if (kin && G.in[0]) {
            vel_cell<BND, PH, 0>(P, G, Q, sl1, sl2, ktop, gz, vx0, vy0, vz0, sn);
            if (kv >= G.z0 && kv < G.z1) {       // own plane: to the output set
                const long long o = (long long)kv * g.plane + (long long)G.cj[0] * g.pitch + G.ci[0];
                P.fout.f[VX][o] = vx0;
                P.fout.f[VY][o] = vy0;
                P.fout.f[VZ][o] = vz0;
            }
        }
        vn[G.e[0]] = vx0;
        vn[NE + G.e[0]] = vy0;
        vn[2 * NE + G.e[0]] = vz0;
        if (G.ring) {
            float vx1 = 0.f, vy1 = 0.f, vz1 = 0.f;
            if (kin && G.in[1]) vel_cell<BND, PH, 1>(P, G, Q, sl1, sl2, ktop, gz, vx1, vy1, vz1, sn);
            vn[G.e[1]] = vx1;
            vn[NE + G.e[1]] = vy1;
            vn[2 * NE + G.e[1]] = vz1;
        }
    }
    if (__syncthreads_or(!ok || Q.bad)) {
        if (tid == 0) fused_fail(P.err, bars, m, G.z0, G.z1, G.ke);
        return false;
    }
    if (tid == 0) {
        // the slot of plane p - 2 is free: refill it with plane p + 2
        if (m >= 2 && m + 2 < P8) issue_v(maps, sm + S2 * FSLOT, &bars[S2], G.x0, G.y0, p + 2);
        // the medium entry of plane ks - 1 (stress of the previous arrival) is
        // free: refill it with plane ks + 2
        const int kd = ks - 1;
        if (m >= 9 && kd < G.z1 && kd + NSENT < G.ke)
            issue_s(maps, sent + sent_of(kd) * SENT, &sbars[sent_of(kd)], G.x0, G.y0, kd + NSENT);
    }
    // point force of step n (Sec. 2.4 source term of Eq. 1) on its tap cells
    // inside the region, before the stress reads them
    if (dov && kv >= P.sk0 && kv <= P.sk1) {               // uniform across the CTA
        if (tid < P.S.ntap) {
            const Tap tp = P.S.tap[tid];
            const int ex = tp.i - (G.x0 - 2), ey = tp.j - (G.y0 - 2);
            if (tp.k == kv && ex >= 0 && ex < EX && ey >= 0 && ey < EY) {
                float amp = tp.w * __ldg(P.wavelet + P.n);
                amp *= ops::buoy(P.M, g, tp.q - VX, tp.i, tp.j, tp.k);
                amp *= ops::gain(P.B, tp.i, tp.j, tp.k);
                atomicAdd(vn + (tp.q - VX) * NE + ey * EX + ex, amp);
                if (kv >= G.z0 && kv < G.z1 && ex >= 2 && ex < 2 + TX && ey >= 2 && ey < 2 + TY)
                    atomicAdd((tp.q == VX ? P.fout.f[VX] : tp.q == VY ? P.fout.f[VY] : P.fout.f[VZ]) +
                                  ops::cidx(g, tp.i, tp.j, tp.k), amp);
            }
        }
        __syncthreads();
        vx0 = vn[G.e[0]];
        vy0 = vn[NE + G.e[0]];
        vz0 = vn[2 * NE + G.e[0]];
    }
    // new-velocity queues of the tile cell: vx, vy of plane kv, vz of kv - 1
    if (dov) {
        Q.vx[PH] = vx0;
        Q.vy[PH] = vy0;
        Q.vz[PH] = Q.vzp;
        Q.vzp = vz0;
    }
    // ---- stress of plane ks at the tile cell (Eq. 2/3) ----
    if (dos) {
        const int sb = sent_of(ks), sb1 = sent_of(ks + 1);
        bool okS = mbar_wait(&sbars[sb], (uint32_t)(((ks - G.z0) / NSENT) & 1));
        if (ks + 1 < G.ke)
            okS = mbar_wait(&sbars[sb1], (uint32_t)(((ks + 1 - G.z0) / NSENT) & 1)) && okS;
        Q.bad |= !okS;
        if (okS && G.in[0]) {
            const float* hvx = vnew + (ks & (NVN - 1)) * 3 * NE + G.e[0];   // plane ks
            const float* hvy = hvx + NE;
            const float* hvz = hvx + 2 * NE;
            // normal strain rates at (i, j, k)
            const float exx = g.c1x * (hvx[0] - hvx[-1]) + g.c2x * (hvx[1] - hvx[-2]);
            const float eyy = g.c1y * (hvy[0] - hvy[-EX]) + g.c2y * (hvy[EX] - hvy[-2 * EX]);
            const float ezz = g.c1z * (Q.vz[C] - Q.vz[B]) + g.c2z * (Q.vz[D] - Q.vz[A]);
            // shear terms at the shear points
            const float vxy = g.c1y * (hvx[EX] - hvx[0]) + g.c2y * (hvx[2 * EX] - hvx[-EX]);
            const float vyx = g.c1x * (hvy[1] - hvy[0]) + g.c2x * (hvy[2] - hvy[-1]);
            const float vxz = g.c1z * (Q.vx[C] - Q.vx[B]) + g.c2z * (Q.vx[D] - Q.vx[A]);
            const float vzx = g.c1x * (hvz[1] - hvz[0]) + g.c2x * (hvz[2] - hvz[-1]);
            const float vyz = g.c1z * (Q.vy[C] - Q.vy[B]) + g.c2z * (Q.vy[D] - Q.vy[A]);
            const float vzy = g.c1y * (hvz[EX] - hvz[0]) + g.c2y * (hvz[2 * EX] - hvz[-EX]);
            // medium: lambda, mu at the cell; mu means at the shear points
            const unsigned char* e0 = sent + sb * SENT;
            const unsigned char* e1 = sent + (ks + 1 < g.nz ? sb1 : sb) * SENT;   // plane ks + 1
            const int tc = threadIdx.y * TX + threadIdx.x;
            const float lam = reinterpret_cast<const float*>(e0)[tc];
            const int mo = threadIdx.y * BW + threadIdx.x + 4;
            const float* hmu = reinterpret_cast<const float*>(e0 + LB) + mo;
            const float* hmu1 = reinterpret_cast<const float*>(e1 + LB) + mo;
            const float mu0 = hmu[0], mxp = hmu[G.mcx], myp = hmu[G.mcy], mzp = hmu1[0];
            const float mxy = 0.25f * (mu0 + mxp + myp + hmu[G.mcx + G.mcy]);
            const float mxz = 0.25f * (mu0 + mxp + mzp + hmu1[G.mcx]);
            const float myz = 0.25f * (mu0 + myp + mzp + hmu1[G.mcy]);
            const float l2m = lam + 2.0f * mu0;
            const float* sg = Q.sg[SQ];
            float s0 = sg[0] + P.dt * (l2m * exx + lam * (eyy + ezz));
            float s1 = sg[1] + P.dt * (l2m * eyy + lam * (exx + ezz));
            float s2 = sg[2] + P.dt * (l2m * ezz + lam * (exx + eyy));
            float s3 = sg[3] + P.dt * mxy * (vxy + vyx);
            float s4 = sg[4] + P.dt * mxz * (vxz + vzx);
            float s5 = sg[5] + P.dt * myz * (vyz + vzy);
            if (BND == BND_SPONGE) {
                const float Gs = G.gx[0] * gzs * G.gy[0];
                s0 *= Gs; s1 *= Gs; s2 *= Gs; s3 *= Gs; s4 *= Gs; s5 *= Gs;
            }
            const long long o = (long long)ks * g.plane + (long long)G.cj[0] * g.pitch + G.ci[0];
            P.fout.f[SXX][o] = s0;
            P.fout.f[SYY][o] = s1;
            P.fout.f[SZZ][o] = s2;
            P.fout.f[SXY][o] = s3;
            P.fout.f[SXZ][o] = s4;
            P.fout.f[SYZ][o] = s5;
        }
    }
    // sigma^n of plane kv waits in the entry of plane ks for two arrivals
#pragma unroll
    for (int q = 0; q < 6; ++q) Q.sg[SQ][q] = sn[q];
    return true;
}

template <int BND>
__global__ void __launch_bounds__(NTH, 2) k_fused(const __grid_constant__ FusedMaps maps,
                                                  const FusedParams P) {
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + NSLOT * FSLOT + NSENT * SENT + NVN * VNEW);
    const int tid = threadIdx.y * TX + threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < NSLOT + NSENT; ++s) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    const FGeo<BND> G(P, (int)blockIdx.x);
    const int P8 = G.z1 - G.z0 + 8;               // arrivals: planes z0-4 .. z1+3
    if (tid == 0) {
        for (int s = 0; s < NSLOT && s < P8; ++s)
            issue_v(maps, sm + s * FSLOT, &bars[s], G.x0, G.y0, G.z0 - 4 + s);
        unsigned char* sent = sm + NSLOT * FSLOT;
        for (int k = G.z0; k < G.z0 + NSENT && k < G.ke; ++k)
            issue_s(maps, sent + sent_of(k) * SENT, &bars[NSLOT + sent_of(k)], G.x0, G.y0, k);
    }
    FQ Q;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        Q.zz[0][q] = Q.zz[1][q] = Q.xz[0][q] = Q.xz[1][q] = Q.yz[0][q] = Q.yz[1][q] = 0.f;
        Q.vx[q] = Q.vy[q] = Q.vz[q] = 0.f;
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) Q.sg[0][q] = Q.sg[1][q] = 0.f;
    Q.vzp = 0.f;
    Q.bad = false;
    for (int m = 0; m < P8; m += 4) {
        if (!fused_step<BND, 0>(maps, P, G, Q, sm, bars, m)) return;
        if (m + 1 < P8 && !fused_step<BND, 1>(maps, P, G, Q, sm, bars, m + 1)) return;
        if (m + 2 < P8 && !fused_step<BND, 2>(maps, P, G, Q, sm, bars, m + 2)) return;
        if (m + 3 < P8 && !fused_step<BND, 3>(maps, P, G, Q, sm, bars, m + 3)) return;
    }
    // a medium wait of the last stress planes that gave up
    if (__syncthreads_or(Q.bad) && tid == 0) fused_fail(P.err, bars, P8, G.z0, G.z1, G.ke);
}

bool encode_fused(FusedMaps* fm, const DevGrid& g, const DevFields& F, const DevMedium& M) {
    const CUtensorMapDataType f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const char* f0 = (const char*)F.f[SXX];                                    // slot 0
    const long long fsb = (const char*)F.f[SXZ] - (const char*)F.f[SXX];
    for (int q = 0; q < NFIELD; ++q)
        if ((const char*)F.f[q] - f0 != fslot(q) * fsb) return false;
    bool ok = true;
    ok &= encode4(&fm->xp, g, f0, f32, 4, fsb, NFIELD, BW, EY, 2);
    ok &= encode4(&fm->yp, g, f0, f32, 4, fsb, NFIELD, BW, EY + 4, 2);
    ok &= encode(&fm->xy, g, F.f[SXY], f32, 4, BW, EY + 4);
    ok &= encode4(&fm->zv, g, f0, f32, 4, fsb, NFIELD, BW, EY, 4);
    ok &= encode(&fm->rho, g, M.rho, f32, 4, BW, EY + 1);
    ok &= encode(&fm->lam, g, M.lam, f32, 4, TX, TY);
    ok &= encode(&fm->mu, g, M.mu, f32, 4, BW, TY + 1);
    return ok;
}

}  // namespace

struct FusedPlan {
    FusedMaps dir[2];             // reading A (dir 0) or B (dir 1)
    DevFields f[2];
    int kind = 0;
    int ntx = 0, nty = 0, zchunk = 0, grid = 0;
};

bool fused_supported(const DevGrid& g, const DevBoundary& B, int storage) {
    return storage == EWS_STORAGE_F32 && (B.kind == BND_SPONGE || B.kind == BND_NONE) &&
           g.fs == kNoSurface && !g.cm[0];
}

cudaError_t fused_plan_create(const DevGrid& g, const DevFields& A, const DevFields& Bf,
                              const DevMedium& M, const DevBoundary& B, FusedPlan** out) {
    FusedPlan* p = new FusedPlan();
    p->kind = B.kind;
    p->f[0] = A;
    p->f[1] = Bf;
    if (!encode_fused(&p->dir[0], g, A, M) || !encode_fused(&p->dir[1], g, Bf, M)) {
        delete p;
        return cudaErrorInvalidValue;
    }
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto kern = B.kind == BND_SPONGE ? k_fused<BND_SPONGE> : k_fused<BND_NONE>;
    if (e == cudaSuccess) e = prepare(kern, F_SMEM, &occ);
    if (e == cudaSuccess && occ < 1) e = cudaErrorInvalidConfiguration;
    if (e != cudaSuccess) {
        delete p;
        return e;
    }
    p->ntx = (g.nx + TX - 1) / TX;
    p->nty = (g.ny + TY - 1) / TY;
    const long long ntile = (long long)p->ntx * p->nty;
    // a chunk loads 4 planes beyond its own on each side
    p->zchunk = chunk_planes(ntile, (long long)sms * occ, g.nz, 16, 4);
    p->grid = (int)(ntile * ((g.nz + p->zchunk - 1) / p->zchunk));
    *out = p;
    return cudaSuccess;
}

void fused_plan_destroy(FusedPlan* p) { delete p; }

cudaError_t launch_fused(const FusedPlan* p, int dir, const DevGrid& g, const DevMedium& M,
                         const DevBoundary& B, float dt, const DevSource& S, const float* wavelet,
                         int n, int* err, cudaStream_t st) {
    FusedParams P{};
    P.g = g;
    P.fin = p->f[dir];
    P.fout = p->f[dir ^ 1];
    P.M = M;
    P.B = B;
    P.dt = dt;
    P.ntx = p->ntx;
    P.nty = p->nty;
    P.zchunk = p->zchunk;
    P.err = err;
    P.S.kind = -1;
    P.S.ntap = 0;
    P.sk0 = 1 << 30;
    P.sk1 = -(1 << 30);
    if (S.kind == 1 && S.ntap > 0) {
        P.S = S;
        P.wavelet = wavelet;
        P.n = n;
        for (int t = 0; t < S.ntap; ++t) {
            P.sk0 = S.tap[t].k < P.sk0 ? S.tap[t].k : P.sk0;
            P.sk1 = S.tap[t].k > P.sk1 ? S.tap[t].k : P.sk1;
        }
    }
    const dim3 blk(TX, RY);
    if (p->kind == BND_SPONGE)
        k_fused<BND_SPONGE><<<p->grid, blk, F_SMEM, st>>>(p->dir[dir], P);
    else
        k_fused<BND_NONE><<<p->grid, blk, F_SMEM, st>>>(p->dir[dir], P);
    return cudaGetLastError();
}

}  // namespace fused
}  // namespace ews
