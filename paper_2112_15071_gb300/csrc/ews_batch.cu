// ews_batch.cu -- host side of the batched executor (ews_batch in
// include/ews.h): per-shot programs of stages, their merge into one entry
// list, the z-chunk autotuner (per-size table, its export / import, and the
// batch-level choice of longer chunks), and the one-by-one reference mode.
// The executor kernel itself is k_batch in ews_stencil.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "ews_sim.cuh"

namespace ews {
namespace {

#define BCK(call)                                                                      \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return report(e_ == cudaErrorMemoryAllocation ? EWS_ENOMEM : EWS_ECUDA,    \
                          "%s: %s", #call, cudaGetErrorString(e_));                    \
    } while (0)

struct Stage {
    int kind, n, slot, flag, nitems;
};

long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }

// One forward time step n: velocity pass (capturing v^{n+1/2} into history
// slot `slot` when >= 0) and stress pass; the source and receiver terms ride
// on their items.
void push_step(std::vector<Stage>& P, const BatchShot& B, int n, int slot, bool record) {
    P.push_back({slot >= 0 ? BK_VEL_CAP : BK_VEL, n, slot, 0, B.items_pass});
    P.push_back({BK_STR, n, 0, record ? 1 : 0, B.items_pass});
}

// The stages of ews_run on one shot.
void forward_program(std::vector<Stage>& P, const BatchShot& B, int nt) {
    P.push_back({BK_ZERO_F, 0, 0, 0, B.items_elem});
    for (int n = 0; n < nt; ++n) push_step(P, B, n, -1, true);
}

// The stages of ews_gradient on one shot (transformed reverse sweep), in
// two parts.  Forward part: forward with checkpoints (the resident range
// [c_res K, nt) writes its history) and the residual.  Reverse part: per
// segment in reverse, restore and recompute (not for the resident range),
// reverse steps, buoyancy term and flushes; finally the gradients.  The
// forward part runs in the lean executor (3 CTAs per SM), the reverse part
// in the one with the reverse velocity pass (larger slots, 2 per SM).
void gradient_forward_program(std::vector<Stage>& P, const BatchShot& B, int nt, int K, int c_res) {
    const int nck = (nt + K - 1) / K;
    const int n_res = c_res * K;
    P.push_back({BK_ZERO_F, 0, 0, 0, B.items_elem});
    for (int c = 0; c < nck; ++c) {
        const int n0 = c * K, n1 = std::min(n0 + K, nt);
        if (c < c_res) P.push_back({BK_SAVE, 0, c, 0, B.items_elem});
        if (c == c_res) P.push_back({BK_HIST0, 0, 0, 0, B.items_elem});
        for (int n = n0; n < n1; ++n) push_step(P, B, n, c >= c_res ? n - n_res + 1 : -1, true);
    }
    P.push_back({BK_RESID, 0, 0, 0, 1});
}

// The reverse part as segments, last first: per segment a recompute phase
// (restore the checkpoint and rerun the segment with history capture; empty
// for the resident range) and a reverse phase (reverse steps, buoyancy
// term, flushes).  The first reverse phase also zeroes the adjoint state,
// the last one finalises the gradients.  Recompute phases run in the lean
// executor (3 CTAs per SM), reverse phases in the one with the reverse
// velocity pass (2 per SM).
struct Phases {
    std::vector<std::vector<Stage>> rec, rev;
};
void gradient_reverse_phases(Phases& F, const BatchShot& B, int nt, int K, int c_res) {
    for (int c = c_res; c >= 0; --c) {
        std::vector<Stage> R, P;
        const int n0 = c * K, n1 = c == c_res ? nt : n0 + K;
        if (c < c_res) {
            R.push_back({BK_LOAD, 0, c, 0, B.items_elem});
            R.push_back({BK_HIST0, 0, 0, 0, B.items_elem});
            for (int n = n0; n < n1; ++n) push_step(R, B, n, n - n0 + 1, false);
        }
        if (c == c_res) P.push_back({BK_ZERO_A, 0, 0, 0, B.items_elem});
        for (int m = n1 - 1; m >= n0; --m) {
            P.push_back({BK_VEL_GRAD, m, m - n0 + 1, m + 1 < n1 ? 1 : 0, B.items_pass});
            P.push_back({BK_STR_ADJ, m, 0, 0, B.items_pass});
            if ((m - n0) % K == 0 && m > n0) P.push_back({BK_FLUSH, 0, 0, 0, B.items_elem});
        }
        P.push_back({BK_RHO, 0, 0, 0, B.items_elem});
        P.push_back({BK_FLUSH, 0, 0, 0, B.items_elem});
        if (c == 0) P.push_back({BK_FINAL, 0, 0, 0, B.items_elem});
        F.rec.push_back(std::move(R));
        F.rev.push_back(std::move(P));
    }
}

// First resident segment of the history budget (as in the adjoint of
// ews_capi.cu): the trailing segments whose history fits, at least one.
int resident_from(const ews_sim* s, int nt, int K, int nshots) {
    const int nck = (nt + K - 1) / K;
    const double budget = sim_history_budget(s, 0.5 / nshots);   // automatic: a share per shot
    const long long slots = (long long)(budget / (3.0 * s->fstride * sizeof(float)));
    int c_res = nck - 1;
    while (c_res > 0 && (long long)(nt - (c_res - 1) * K) + 1 <= slots) --c_res;
    return c_res;
}

// Everything the executor needs about one shot.
ews_status fill_shot(BatchShot& B, ews_sim* s, const ews_batch_shot& in, int zchunk, int* err,
                     bool grad) {
    std::memset(&B, 0, sizeof(B));
    const size_t fs = s->fstride;
    int ntx, nty, zc, items;
    stencil_plan_export(s->plan, &B.vf, &B.sf, &ntx, &nty, &zc, &items);
    const int nz = s->g.nz;
    zc = std::min(std::max(zchunk, 1), nz);
    B.items_pass = ntx * nty * (int)ceil_div(nz, zc);
    B.items_elem = (int)ceil_div((long long)fs, kBatchElem);
    PassParams& P = B.pf;
    P.g = s->g;
    P.F = s->F();
    P.B = s->B;
    for (int q = 0; q < NFIELD; ++q) {
        P.dto[q] = (float)in.dt;
        P.inv[q] = 1.0f;
    }
    P.ntx = ntx;
    P.nty = nty;
    P.zchunk = zc;
    P.err = err;
    B.M = s->M();
    B.S = sim_source(s, in.dt);
    B.wavelet = s->wavelet;
    B.rtaps = s->rtaps;
    B.nrec = s->nrec;
    B.nt = in.nt;
    B.seis = in.seis;
    B.fs = (long long)fs;
    B.dt = (float)in.dt;
    if (!grad) return EWS_OK;
    int a, b, c, d;
    stencil_plan_export(s->adj_plan, &B.va, &B.sa, &a, &b, &c, &d);
    PassParams& Q = B.pa;
    Q = P;
    for (int q = 0; q < NFIELD; ++q) {
        Q.F.f[q] = s->adj + fslot(q) * fs;
        Q.dto[q] = -(float)in.dt;
    }
    for (int q = 0; q < 3; ++q) B.A.p[q] = s->adj + fslot(VX + q) * fs;
    for (int q = 0; q < 6; ++q) B.A.q[q] = s->adj + fslot(SXX + q) * fs;
    for (int q = 0; q < 8; ++q) {
        B.A.acc[q] = s->adj + (9 + q) * fs;
        B.A.acc64[q] = s->acc64 + q * fs;
        Q.X.acc[q] = B.A.acc[q];
    }
    Q.X.fstride = (long long)fs;
    Q.X.gdt = (float)in.dt;
    B.vhist = s->vhist;
    B.ckpt = s->ckpt;
    B.ck16 = s->ckpt_storage == EWS_STORAGE_BF16 ? 1 : 0;
    B.obs = in.observed;
    const size_t nseis = (size_t)3 * s->nrec * in.nt;
    if (!B.seis) B.seis = s->aux;                 // forward seismograms for the residual
    B.sadj = s->aux + nseis;
    B.misfit = s->dmisfit;
    B.gl = in.g_lam;
    B.gm = in.g_mu;
    B.gr = in.g_rho;
    return EWS_OK;
}

struct Entry {
    double key;
    BatchEntry e;
};

// Run the programs of `shots` in one persistent launch.
ews_status run_persistent(std::vector<BatchShot>& shots, std::vector<std::vector<Stage>>& progs,
                          int bnd, int exec, int ctas_per_sm, int* d_err, cudaStream_t st,
                          float* ms_out, unsigned long long wait_ns = 0, bool stall = false) {
    const int ns = (int)shots.size();
    std::vector<Entry> all;
    size_t total = 0;
    for (const auto& p : progs) total += p.size();
    all.reserve(total);
    for (int s = 0; s < ns; ++s) {
        long long need = 0;
        const double R = (double)progs[s].size();
        for (size_t r = 0; r < progs[s].size(); ++r) {
            const Stage& g = progs[s][r];
            BatchEntry e{};
            e.shot = s;
            e.kind = g.kind;
            e.n = g.n;
            e.slot = g.slot;
            e.flag = g.flag;
            e.need = need;
            e.nitems = g.nitems;
            all.push_back({(r + 0.5) / R, e});
            need += g.nitems;
        }
    }
    // every shot advances through its program at the same relative pace
    std::stable_sort(all.begin(), all.end(), [](const Entry& a, const Entry& b) {
        return a.key < b.key || (a.key == b.key && a.e.shot < b.e.shot);
    });
    std::vector<BatchEntry> ent(all.size());
    for (size_t i = 0; i < all.size(); ++i) ent[i] = all[i].e;
    if (stall && !ent.empty()) ent.back().need += 1;   // waits for an item that never exists
    const int nent = (int)ent.size();

    int dev = 0, sms = 0, per_sm = 0;
    BCK(cudaGetDevice(&dev));
    BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    BCK(batch_occupancy(bnd, exec, &per_sm));
    if (per_sm < 1) return report(EWS_ECUDA, "batched executor does not fit on an SM");
    if (ctas_per_sm > 0) per_sm = std::min(per_sm, ctas_per_sm);

    BatchShot* d_shots = nullptr;
    BatchEntry* d_ent = nullptr;
    unsigned* d_cnt = nullptr;       // cur, taken[nent]
    unsigned long long* d_done = nullptr;
    auto cleanup = [&]() {
        dev_free(d_shots);
        dev_free(d_ent);
        dev_free(d_cnt);
        dev_free(d_done);
    };
    cudaError_t e = dev_malloc((void**)&d_shots, sizeof(BatchShot) * ns);
    if (e == cudaSuccess) e = dev_malloc((void**)&d_ent, sizeof(BatchEntry) * nent);
    if (e == cudaSuccess) e = dev_malloc((void**)&d_cnt, sizeof(unsigned) * (nent + 1));
    if (e == cudaSuccess) e = dev_malloc((void**)&d_done, sizeof(unsigned long long) * ns);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_shots, shots.data(), sizeof(BatchShot) * ns, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_ent, ent.data(), sizeof(BatchEntry) * nent, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, sizeof(unsigned) * (nent + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_done, 0, sizeof(unsigned long long) * ns, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess && ms_out) e = cudaEventCreate(&t0);
    if (e == cudaSuccess && ms_out) e = cudaEventCreate(&t1);
    if (e == cudaSuccess && ms_out) e = cudaEventRecord(t0, st);
    if (e == cudaSuccess)
        e = launch_batch(bnd, exec, sms * per_sm, d_shots, d_ent, nent, d_cnt, d_cnt + 1, d_done,
                         d_err, wait_ns ? wait_ns : 4000000000ull, st);
    if (e == cudaSuccess && ms_out) e = cudaEventRecord(t1, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && ms_out) e = cudaEventElapsedTime(ms_out, t0, t1);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost);
    cleanup();
    if (e != cudaSuccess)
        return report(e == cudaErrorMemoryAllocation ? EWS_ENOMEM : EWS_ECUDA, "batched launch: %s",
                      cudaGetErrorString(e));
    if (herr & 11)
        return report(EWS_ETIMEOUT, "batched executor: a %s wait gave up (flags %d)",
                      (herr & 8) ? "dependency" : "pipeline", herr);
    if (herr & 16) return report(EWS_ENONFINITE, "batched executor: a receiver recorded NaN or Inf");
    return EWS_OK;
}

// ---- a sequence of persistent launches under one CUDA graph ----

// Device tables of one persistent launch (entries and counters).
struct Prepared {
    BatchEntry* ent = nullptr;
    unsigned* cnt = nullptr;
    unsigned long long* done = nullptr;
    int nent = 0, exec = 0, grid = 0;
};

void release(std::vector<Prepared>& v) {
    for (Prepared& p : v) {
        dev_free(p.ent);
        dev_free(p.cnt);
        dev_free(p.done);
    }
    v.clear();
}

// Merge the programs into one entry list (as run_persistent) and upload it.
ews_status prepare_launch(const std::vector<std::vector<Stage>>& progs, int exec, int bnd,
                          int ctas_per_sm, bool stall, cudaStream_t st, Prepared* out) {
    const int ns = (int)progs.size();
    std::vector<Entry> all;
    for (int sh = 0; sh < ns; ++sh) {
        long long need = 0;
        const double R = (double)progs[sh].size();
        for (size_t r = 0; r < progs[sh].size(); ++r) {
            const Stage& g = progs[sh][r];
            BatchEntry e{};
            e.shot = sh;
            e.kind = g.kind;
            e.n = g.n;
            e.slot = g.slot;
            e.flag = g.flag;
            e.need = need;
            e.nitems = g.nitems;
            all.push_back({(r + 0.5) / R, e});
            need += g.nitems;
        }
    }
    std::stable_sort(all.begin(), all.end(), [](const Entry& a, const Entry& b) {
        return a.key < b.key || (a.key == b.key && a.e.shot < b.e.shot);
    });
    std::vector<BatchEntry> ent(all.size());
    for (size_t i = 0; i < all.size(); ++i) ent[i] = all[i].e;
    if (stall && !ent.empty()) ent.back().need += 1;   // waits for an item that never exists
    int dev = 0, sms = 0, per_sm = 0;
    BCK(cudaGetDevice(&dev));
    BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    BCK(batch_occupancy(bnd, exec, &per_sm));
    if (per_sm < 1) return report(EWS_ECUDA, "batched executor does not fit on an SM");
    if (ctas_per_sm > 0) per_sm = std::min(per_sm, ctas_per_sm);
    Prepared p;
    p.nent = (int)ent.size();
    p.exec = exec;
    p.grid = sms * per_sm;
    cudaError_t e = dev_malloc((void**)&p.ent, sizeof(BatchEntry) * std::max(p.nent, 1));
    if (e == cudaSuccess) e = dev_malloc((void**)&p.cnt, sizeof(unsigned) * (p.nent + 1));
    if (e == cudaSuccess) e = dev_malloc((void**)&p.done, sizeof(unsigned long long) * ns);
    if (e == cudaSuccess && p.nent)
        e = cudaMemcpyAsync(p.ent, ent.data(), sizeof(BatchEntry) * p.nent, cudaMemcpyHostToDevice, st);
    *out = p;
    if (e != cudaSuccess)
        return report(e == cudaErrorMemoryAllocation ? EWS_ENOMEM : EWS_ECUDA, "batched tables: %s",
                      cudaGetErrorString(e));
    return EWS_OK;
}

// Counter resets and the launch of a prepared table, on `st` (capturable).
cudaError_t enqueue(const Prepared& p, int bnd, int nshots, const BatchShot* d_shots, int* d_err,
                    unsigned long long wait_ns, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(p.cnt, 0, sizeof(unsigned) * (p.nent + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.done, 0, sizeof(unsigned long long) * nshots, st);
    if (e == cudaSuccess)
        e = launch_batch(bnd, p.exec, p.grid, d_shots, p.ent, p.nent, p.cnt, p.cnt + 1, p.done, d_err,
                         wait_ns, st);
    return e;
}

// ---- autotuner: planes per tile in z, per grid size ----
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_tuned;

ews_status tune_zchunk(ews_sim* s, const ews_batch_shot& in, int bnd, int exec, int ctas,
                       int* d_err, cudaStream_t st, int* out) {
    const auto key = std::make_tuple(s->g.nx, s->g.ny, s->g.nz, bnd, exec);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            *out = it->second;
            return EWS_OK;
        }
    }
    const int nz = s->g.nz;
    std::vector<int> cand;
    for (int z : {8, 12, 16, 24, 32, 48, 64, 96, 128})
        if (z <= nz) cand.push_back(z);
    if (cand.empty() || cand.back() != nz) cand.push_back(nz);
    const int T = std::min(in.nt, 6);                 // trial: a few forward steps
    int best = cand.front();
    float best_ms = 1e30f;
    for (int z : cand) {
        std::vector<BatchShot> shots(1);
        ews_batch_shot probe = in;
        probe.seis = nullptr;
        probe.nt = T;
        ews_status r = fill_shot(shots[0], s, probe, z, d_err, false);
        if (r != EWS_OK) return r;
        std::vector<std::vector<Stage>> progs(1);
        for (int n = 0; n < T; ++n) push_step(progs[0], shots[0], n, -1, false);
        float ms = 0, ms2 = 0;
        if ((r = run_persistent(shots, progs, bnd, exec, ctas, d_err, st, &ms)) != EWS_OK) return r;
        if ((r = run_persistent(shots, progs, bnd, exec, ctas, d_err, st, &ms2)) != EWS_OK) return r;
        ms = std::min(ms, ms2);
        if (ms < best_ms) {
            best_ms = ms;
            best = z;
        }
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = best;
    *out = best;
    return EWS_OK;
}

// ---- batch level: the per-size table or longer z-chunks ----
// The table comes from trials of one shot alone, where short z-chunks buy
// parallelism.  A batch of many forward shots has that parallelism already,
// and longer chunks (fewer halo planes, items and dependency waits) can be
// faster: the 48-shot forward batch of cubes 96..224 ran at 41.5 Gcell/s
// with the table, 42.4 with 64-plane chunks, 43.2 with 128-plane chunks.
// So such a batch times its first steps with each candidate (the table;
// 64 and 128 planes; whole tile columns) and keeps the fastest; the choice
// is cached per batch composition.  Gradient batches take the choice of
// their forward steps for every launch (48 gradient shots: 24.4 s with the
// table, 23.2 s with the choice).
constexpr int kBatchChunks[] = {0, 64, 128, 1 << 30};            // 0: the table
std::map<std::vector<std::tuple<int, int, int, int, int>>, int> g_choice;   // under g_tune_mu

int chunk_for(int choice, int table_zc, int nz) {
    return choice == 0 ? table_zc : std::min(kBatchChunks[choice], nz);
}

ews_status choose_batch_chunks(const ews_batch_shot* shots, int nshots, const std::vector<int>& zc,
                               int bnd, int exec, int ctas, int* d_err, cudaStream_t st,
                               int* choice) {
    std::vector<std::tuple<int, int, int, int, int>> key;
    for (int i = 0; i < nshots; ++i) {
        const ews_sim* s = shots[i].sim;
        key.emplace_back(s->g.nx, s->g.ny, s->g.nz, bnd, exec);
    }
    std::sort(key.begin(), key.end());
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_choice.find(key);
        if (it != g_choice.end()) {
            *choice = it->second;
            return EWS_OK;
        }
    }
    int T = 6;                                        // trial: the first few forward steps
    for (int i = 0; i < nshots; ++i) T = std::min(T, shots[i].nt);
    const int ncand = (int)(sizeof(kBatchChunks) / sizeof(kBatchChunks[0]));
    std::vector<std::vector<int>> tried;
    int best = 0;
    float best_ms = 1e30f;
    for (int c = 0; c < ncand; ++c) {
        std::vector<int> z(nshots);
        for (int i = 0; i < nshots; ++i) z[i] = chunk_for(c, zc[i], shots[i].sim->g.nz);
        if (std::find(tried.begin(), tried.end(), z) != tried.end()) continue;   // same launch
        tried.push_back(z);
        std::vector<BatchShot> bs(nshots);
        std::vector<std::vector<Stage>> progs(nshots);
        for (int i = 0; i < nshots; ++i) {
            ews_batch_shot probe = shots[i];
            probe.seis = nullptr;
            probe.nt = T;
            ews_status r = fill_shot(bs[i], probe.sim, probe, z[i], d_err, false);
            if (r != EWS_OK) return r;
            for (int n = 0; n < T; ++n) push_step(progs[i], bs[i], n, -1, false);
        }
        float ms = 0, ms2 = 0;
        ews_status r;
        if ((r = run_persistent(bs, progs, bnd, exec, ctas, d_err, st, &ms)) != EWS_OK) return r;
        if ((r = run_persistent(bs, progs, bnd, exec, ctas, d_err, st, &ms2)) != EWS_OK) return r;
        ms = std::min(ms, ms2);
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    *choice = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_choice[key] = best;
    return EWS_OK;
}

// The persistent executor over all the given shots in one captured graph.
ews_status batch_persistent(int nshots, ews_batch_shot* shots, const ews_batch_options& o, int bnd,
                            bool grad, bool any_fs, cudaStream_t st) {
    const int K0 = o.ckpt_every > 0 ? o.ckpt_every : 50;
    int* d_err = shots[0].sim->err;            // any of the shots' error flags
    std::vector<BatchShot> bs(nshots);
    std::vector<std::vector<Stage>> progs(nshots);
    std::vector<Phases> phases(nshots);
    std::vector<int> zcs(nshots, 0), cres(nshots, 0);
    for (int i = 0; i < nshots; ++i) {
        ews_batch_shot& b = shots[i];
        ews_sim* s = b.sim;
        const int K = std::min(K0, b.nt);
        int c_res = 0;
        if (b.observed) {
            c_res = resident_from(s, b.nt, K, nshots);
            const int hslots = std::max(K, b.nt - c_res * K) + 1;
            // BF16 checkpoints as asked for (FP16 ones are kept in FP32 here:
            // their scales would need a reduction over the state first)
            const int ck = s->ckpt_pref == EWS_STORAGE_BF16 ? EWS_STORAGE_BF16 : EWS_STORAGE_F32;
            ews_status r = sim_adjoint_buffers(s, b.nt, c_res, hslots, true, ck);
            if (r == EWS_OK) r = sim_adjoint_plan(s);
            if (r != EWS_OK) return r;
        }
        zcs[i] = o.zchunk;
        cres[i] = c_res;
        if (zcs[i] == 0) {
            ews_status r = tune_zchunk(s, b, bnd, s->g.fs != kNoSurface ? BX_LEAN_FS : BX_LEAN,
                                       o.ctas_per_sm, d_err, st, &zcs[i]);
            if (r != EWS_OK) return r;
        }
    }
    const int lean = any_fs ? BX_LEAN_FS : BX_LEAN, rev = any_fs ? BX_GRAD_FS : BX_GRAD;
    int choice = 0;                            // the per-size table
    if (o.zchunk == 0 && nshots > 1) {
        ews_status r = choose_batch_chunks(shots, nshots, zcs, bnd, lean, o.ctas_per_sm, d_err, st,
                                           &choice);
        if (r != EWS_OK) return r;
    }
    for (int i = 0; i < nshots; ++i) {
        ews_batch_shot& b = shots[i];
        ews_sim* s = b.sim;
        const int K = std::min(K0, b.nt);
        ews_status r = fill_shot(bs[i], s, b, chunk_for(choice, zcs[i], s->g.nz), d_err,
                                 b.observed != nullptr);
        if (r != EWS_OK) return r;
        if (b.observed) {
            gradient_forward_program(progs[i], bs[i], b.nt, K, cres[i]);
            gradient_reverse_phases(phases[i], bs[i], b.nt, K, cres[i]);
        } else {
            forward_program(progs[i], bs[i], b.nt);
        }
    }
    const unsigned long long wait =
        o.dep_wait_ms ? (unsigned long long)o.dep_wait_ms * 1000000ull : 4000000000ull;
    // The launches: the forward part of every shot, then the reverse parts
    // segment phase by segment phase (a recomputation launch and a reverse
    // launch per phase; shots with fewer segments join for the last phases,
    // so all finish in the last one).  They are prepared up front and run as
    // one captured CUDA graph, with one synchronisation at the end.
    std::vector<Prepared> launches;
    BatchShot* d_shots = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cs = nullptr;
    auto cleanup = [&]() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
        release(launches);
        dev_free(d_shots);
    };
    ews_status r = EWS_OK;
    auto add = [&](const std::vector<std::vector<Stage>>& pr, int exec, bool stall) {
        Prepared p;
        if (r == EWS_OK) r = prepare_launch(pr, exec, bnd, o.ctas_per_sm, stall, st, &p);
        launches.push_back(p);
    };
    add(progs, lean, o.test_unsatisfiable != 0);
    size_t nph = 0;
    for (const auto& f : phases) nph = std::max(nph, f.rev.size());
    for (size_t ph = 0; ph < nph && grad; ++ph) {
        std::vector<std::vector<Stage>> rec(nshots), rv(nshots);
        bool any_rec = false;
        for (int i = 0; i < nshots; ++i) {
            const size_t n = phases[i].rev.size(), off = nph - n;
            if (ph < off) continue;
            rec[i] = phases[i].rec[ph - off];
            rv[i] = phases[i].rev[ph - off];
            any_rec |= !rec[i].empty();
        }
        if (any_rec) add(rec, lean, false);
        add(rv, rev, false);
    }
    if (r != EWS_OK) {
        cleanup();
        return r;
    }
    cudaError_t e = dev_malloc((void**)&d_shots, sizeof(BatchShot) * nshots);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_shots, bs.data(), sizeof(BatchShot) * nshots, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);        // tables in place
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = cudaSuccess;
        for (const Prepared& p : launches)
            if (le == cudaSuccess) le = enqueue(p, bnd, nshots, d_shots, d_err, wait, cs);
        e = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(gexec, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost);
    cleanup();
    if (e != cudaSuccess)
        return report(e == cudaErrorMemoryAllocation ? EWS_ENOMEM : EWS_ECUDA, "batched launches: %s",
                      cudaGetErrorString(e));
    if (herr & 11)
        return report(EWS_ETIMEOUT, "batched executor: a %s wait gave up (flags %d)",
                      (herr & 8) ? "dependency" : "pipeline", herr);
    if (herr & 16) return report(EWS_ENONFINITE, "batched executor: a receiver recorded NaN or Inf");
    for (int i = 0; i < nshots; ++i) {
        ews_sim* s = shots[i].sim;
        s->fresh = false;
        if (shots[i].observed)
            BCK(cudaMemcpy(&shots[i].misfit, s->dmisfit, sizeof(double), cudaMemcpyDeviceToHost));
    }
    return EWS_OK;
}

// Gradient shots in waves.  The gradient state of a shot (adjoint fields,
// accumulators, checkpoints and a segment of velocity history: about 1.2 to
// 1.6 KB per cell) is set up for every shot of a launch at once; when that
// does not fit the device (or the library's memory limit), the shots are
// split in two halves run one after the other (the forward shots go with the
// first), recursively, and each finished wave releases its shots' gradient
// state (ews_release_workspace) for the next.
ews_status batch_waves(ews_batch_shot* shots, const std::vector<int>& idx,
                       const ews_batch_options& o, int bnd, bool any_fs, cudaStream_t st) {
    std::vector<ews_batch_shot> sub(idx.size());
    std::vector<int> grads;
    bool grad = false;
    for (size_t k = 0; k < idx.size(); ++k) {
        sub[k] = shots[idx[k]];
        if (sub[k].observed) {
            grad = true;
            grads.push_back((int)k);
        }
    }
    ews_status r = batch_persistent((int)sub.size(), sub.data(), o, bnd, grad, any_fs, st);
    if (r == EWS_OK) {
        for (size_t k = 0; k < idx.size(); ++k) shots[idx[k]].misfit = sub[k].misfit;
        return EWS_OK;
    }
    if (r != EWS_ENOMEM || grads.size() < 2) return r;
    // too much gradient state at once: release what was set up, split, retry
    for (int k : grads) {
        const ews_status rr = ews_release_workspace(sub[k].sim);
        if (rr != EWS_OK) return rr;
    }
    std::vector<int> first, second;
    const size_t half = grads.size() / 2;
    size_t g = 0;
    for (size_t k = 0; k < idx.size(); ++k) {
        if (sub[k].observed) {
            (g++ < half ? first : second).push_back(idx[k]);
        } else {
            first.push_back(idx[k]);                 // forward shots go with the first wave
        }
    }
    if ((r = batch_waves(shots, first, o, bnd, any_fs, st)) != EWS_OK) return r;
    for (int i : first)
        if (shots[i].observed && (r = ews_release_workspace(shots[i].sim)) != EWS_OK) return r;
    return batch_waves(shots, second, o, bnd, any_fs, st);
}

}  // namespace
}  // namespace ews

extern "C" {

int ews_batch_tuned_zchunk(const ews_grid* grid, int boundary, int free_surface) {
    if (!grid) return 0;
    std::lock_guard<std::mutex> lk(ews::g_tune_mu);
    auto it = ews::g_tuned.find(std::make_tuple(grid->nx, grid->ny, grid->nz, boundary,
                                                free_surface ? (int)ews::BX_LEAN_FS
                                                             : (int)ews::BX_LEAN));
    return it == ews::g_tuned.end() ? 0 : it->second;
}

// The autotuner times trial launches of the forward executor only (its
// result serves forward and gradient shots alike), so the table has one
// entry per grid, boundary and surface form.
int ews_batch_tuning_export(ews_tuned_zchunk* out, int cap) {
    std::lock_guard<std::mutex> lk(ews::g_tune_mu);
    int n = 0;
    for (const auto& kv : ews::g_tuned) {
        if (out && n < cap) {
            ews_tuned_zchunk& e = out[n];
            e.nx = std::get<0>(kv.first);
            e.ny = std::get<1>(kv.first);
            e.nz = std::get<2>(kv.first);
            e.boundary = std::get<3>(kv.first);
            e.free_surface = std::get<4>(kv.first) == ews::BX_LEAN_FS ? 1 : 0;
            e.zchunk = kv.second;
        }
        ++n;
    }
    return n;
}

ews_status ews_batch_tuning_import(const ews_tuned_zchunk* in, int n) {
    if (n < 0 || (n > 0 && !in)) return ews::report(EWS_EINVAL, "ews_batch_tuning_import: no entries");
    for (int k = 0; k < n; ++k) {
        const ews_tuned_zchunk& e = in[k];
        if (e.nx < 1 || e.ny < 1 || e.nz < 1 || e.boundary < EWS_BOUNDARY_NONE ||
            e.boundary > EWS_BOUNDARY_CPML || (e.free_surface != 0 && e.free_surface != 1) ||
            e.zchunk < 1 || e.zchunk > e.nz)
            return ews::report(EWS_EINVAL,
                               "ews_batch_tuning_import: entry %d (%d x %d x %d, boundary %d, "
                               "surface %d, zchunk %d) is invalid; nothing imported",
                               k, e.nx, e.ny, e.nz, e.boundary, e.free_surface, e.zchunk);
    }
    std::lock_guard<std::mutex> lk(ews::g_tune_mu);
    ews::g_choice.clear();                      // batch-level choices were made against the old entries
    for (int k = 0; k < n; ++k) {
        const ews_tuned_zchunk& e = in[k];
        ews::g_tuned[std::make_tuple(e.nx, e.ny, e.nz, e.boundary,
                                     e.free_surface ? (int)ews::BX_LEAN_FS : (int)ews::BX_LEAN)] =
            e.zchunk;
    }
    return EWS_OK;
}

void ews_batch_tuning_clear(void) {
    std::lock_guard<std::mutex> lk(ews::g_tune_mu);
    ews::g_tuned.clear();
    ews::g_choice.clear();
}

ews_status ews_batch(int nshots, ews_batch_shot* shots, const ews_batch_options* opt,
                     void* cuda_stream) {
    using namespace ews;
    if (nshots <= 0 || !shots) return report(EWS_EINVAL, "no shots");
    ews_batch_options o{};
    if (opt) o = *opt;
    if (o.mode != EWS_BATCH_PERSISTENT && o.mode != EWS_BATCH_SEQUENTIAL)
        return report(EWS_EINVAL, "unknown batch mode %d", o.mode);
    if (o.ckpt_every < 0 || o.zchunk < 0 || o.ctas_per_sm < 0 || o.dep_wait_ms < 0)
        return report(EWS_EINVAL, "negative batch option");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int bnd = shots[0].sim ? shots[0].sim->opt.boundary : -1;
    bool grad = false, any_fs = false;
    for (int i = 0; i < nshots; ++i) {
        const ews_batch_shot& b = shots[i];
        ews_sim* s = b.sim;
        if (!s) return report(EWS_EINVAL, "shot %d: null simulation", i);
        for (int j = 0; j < i; ++j)
            if (shots[j].sim == s) return report(EWS_EINVAL, "shot %d: simulation used twice", i);
        if (s->opt.boundary != bnd) return report(EWS_EINVAL, "shot %d: boundary differs", i);
        if (bnd == EWS_BOUNDARY_CPML && b.observed)
            return report(EWS_EINVAL, "shot %d: gradients take the none or sponge boundary", i);
        if (s->opt.storage != EWS_STORAGE_F32) return report(EWS_EINVAL, "shot %d: F32 storage only", i);
        if (b.nt <= 0) return report(EWS_EINVAL, "shot %d: nt must be positive", i);
        if (b.observed) {
            grad = true;
            if (!b.g_lam || !b.g_mu || !b.g_rho)
                return report(EWS_EINVAL, "shot %d: gradient outputs missing", i);
        }
        ews_status r = sim_ready(s, b.nt, b.dt);
        if (r != EWS_OK) return r;
        if (b.observed && s->has_fluid)
            return report(EWS_EINVAL, "shot %d: fluid cells (mu = 0) are not batched", i);
        if (s->g.fs != kNoSurface) any_fs = true;
        if (s->g.cm[0]) return report(EWS_EINVAL, "shot %d: coarse medium grids are not batched", i);
    }
    const int K0 = o.ckpt_every > 0 ? o.ckpt_every : 50;

    if (o.mode == EWS_BATCH_SEQUENTIAL) {      // one shot after the other
        for (int i = 0; i < nshots; ++i) {
            ews_batch_shot& b = shots[i];
            ews_sim* s = b.sim;
            ews_status r = ews_set_stream(s, st);
            if (r != EWS_OK) return r;
            if (b.observed) {
                r = ews_gradient(s, b.nt, b.dt, b.observed, 1, &b.misfit, b.g_lam, b.g_mu,
                                 b.g_rho, 1, K0);
                if (r == EWS_ENOMEM && i > 0) {
                    // the earlier shots' gradient state stays set up until
                    // released: release it and try this shot again
                    for (int j = 0; j < i && r == EWS_ENOMEM; ++j)
                        if (shots[j].observed && ews_release_workspace(shots[j].sim) != EWS_OK)
                            return EWS_ECUDA;
                    r = ews_gradient(s, b.nt, b.dt, b.observed, 1, &b.misfit, b.g_lam, b.g_mu,
                                     b.g_rho, 1, K0);
                }
                if (r == EWS_OK && b.seis && s->nrec > 0)
                    BCK(cudaMemcpyAsync(b.seis, s->aux, (size_t)3 * s->nrec * b.nt * sizeof(float),
                                        cudaMemcpyDeviceToDevice, st));
            } else {
                r = ews_run(s, b.nt, b.dt, b.seis, 1, nullptr);
            }
            if (r != EWS_OK) return r;
        }
        BCK(cudaStreamSynchronize(st));
        return EWS_OK;
    }

    if (!grad) return batch_persistent(nshots, shots, o, bnd, false, any_fs, st);
    std::vector<int> all(nshots);
    for (int i = 0; i < nshots; ++i) all[i] = i;
    return batch_waves(shots, all, o, bnd, any_fs, st);
}

}  // extern "C"
