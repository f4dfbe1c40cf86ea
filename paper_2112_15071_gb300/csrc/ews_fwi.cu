// ews_fwi.cu -- one iteration of multi-shot full-waveform inversion on one
// model (the many-stations, one-earthquake setting of the paper's case study
// turned into an inversion step; the paper itself only runs the forward
// model): batched L2-misfit gradients of all shots (ews_batch), their sum,
// a steepest-descent direction scaled per parameter, and a step length from
// a parabola through the misfits at 0, a/2 and a.  Elementwise work runs in
// the kernels below.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ews_sim.cuh"

namespace ews {
namespace {

#define FCK(call)                                                                      \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return report(e_ == cudaErrorMemoryAllocation ? EWS_ENOMEM : EWS_ECUDA,    \
                          "%s: %s", #call, cudaGetErrorString(e_));                    \
    } while (0)

constexpr int kThreads = 256;

int blocks_for(long long n) { return (int)std::min<long long>((n + kThreads - 1) / kThreads, 4096); }

// out[c] = sum over shots of g[s][c] (g: device array of nshots pointers).
__global__ void k_sum_shots(const float* const* __restrict__ g, int nshots, long long n,
                            float* __restrict__ out) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int s = 0; s < nshots; ++s) acc += g[s][c];
        out[c] = (float)acc;
    }
}

// *out = max |a| (float bits of a non-negative value, unsigned atomics).
__global__ void k_absmax(const float* __restrict__ a, long long n, unsigned* out) {
    float m = 0.0f;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(a[c]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// Trial model m + alpha d with d = -scale g per parameter, kept physical:
// rho and mu at least half their current values, the bulk modulus
// lambda + 2/3 mu at least half its current value.
__global__ void k_trial_model(const float* __restrict__ lam, const float* __restrict__ mu,
                              const float* __restrict__ rho, const float* __restrict__ gl,
                              const float* __restrict__ gm, const float* __restrict__ gr,
                              float sl, float sm, float sr, float alpha, long long n,
                              float* __restrict__ tl, float* __restrict__ tm,
                              float* __restrict__ tr) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const float r = fmaxf(rho[c] - alpha * sr * gr[c], 0.5f * rho[c]);
        const float m = fmaxf(mu[c] - alpha * sm * gm[c], 0.5f * mu[c]);
        const float k0 = lam[c] + (2.0f / 3.0f) * mu[c];
        const float k = fmaxf(lam[c] - alpha * sl * gl[c] + (2.0f / 3.0f) * m, 0.5f * k0);
        tr[c] = r;
        tm[c] = m;
        tl[c] = k - (2.0f / 3.0f) * m;
    }
}

// *out += dt / 2 sum (s - d)^2.
__global__ void k_misfit(const float* __restrict__ s, const float* __restrict__ d, long long n,
                         float dt, double* out) {
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const double r = (double)s[c] - (double)d[c];
        acc += r * r;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, 0.5 * (double)dt * acc);
}

}  // namespace
}  // namespace ews

extern "C" ews_status ews_fwi_iteration(int nshots, ews_batch_shot* shots, float* lam, float* mu,
                                        float* rho, double max_rel_step, int ckpt_every,
                                        double* misfit0, double* misfit1, double* step,
                                        void* cuda_stream) {
    using namespace ews;
    if (nshots <= 0 || !shots || !lam || !mu || !rho) return report(EWS_EINVAL, "bad arguments");
    if (!(max_rel_step > 0) || !(max_rel_step < 1)) return report(EWS_EINVAL, "max_rel_step in (0, 1)");
    const ews_grid g0 = shots[0].sim ? shots[0].sim->grid : ews_grid{};
    for (int i = 0; i < nshots; ++i) {
        const ews_sim* s = shots[i].sim;
        if (!s) return report(EWS_EINVAL, "shot %d: null simulation", i);
        if (s->grid.nx != g0.nx || s->grid.ny != g0.ny || s->grid.nz != g0.nz ||
            s->grid.dx != g0.dx || s->grid.dy != g0.dy || s->grid.dz != g0.dz)
            return report(EWS_EINVAL, "shot %d: all shots must share one grid", i);
        if (!shots[i].observed) return report(EWS_EINVAL, "shot %d: observed data missing", i);
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const long long n = (long long)g0.nx * g0.ny * g0.nz;
    // workspace: per-shot gradients, the summed gradient, trial model, per-shot seismograms
    std::vector<float*> gs(3 * nshots, nullptr), seis(nshots, nullptr);
    float *gt = nullptr, *trial = nullptr;
    const float** d_gl = nullptr;
    unsigned* d_max = nullptr;
    double* d_mis = nullptr;
    auto cleanup = [&]() {
        for (float* p : gs) dev_free(p);
        for (float* p : seis) dev_free(p);
        dev_free(gt);
        dev_free(trial);
        dev_free(d_gl);
        dev_free(d_max);
        dev_free(d_mis);
    };
    ews_status result = EWS_OK;
    auto run = [&]() -> ews_status {
        for (auto& p : gs) FCK(dev_malloc((void**)&p, n * sizeof(float)));
        for (int i = 0; i < nshots; ++i) {
            const ews_sim* s = shots[i].sim;
            FCK(dev_malloc((void**)&seis[i], sizeof(float) * 3 * std::max(1, s->nrec) * shots[i].nt));
        }
        FCK(dev_malloc((void**)&gt, 3 * n * sizeof(float)));
        FCK(dev_malloc((void**)&trial, 3 * n * sizeof(float)));
        FCK(dev_malloc((void**)&d_gl, 3 * nshots * sizeof(float*)));
        FCK(dev_malloc((void**)&d_max, 6 * sizeof(unsigned)));
        FCK(dev_malloc((void**)&d_mis, sizeof(double)));
        // misfit and gradient of every shot at the current model, one launch
        std::vector<ews_batch_shot> b(shots, shots + nshots);
        for (int i = 0; i < nshots; ++i) {
            ews_status r = ews_set_model_lame(b[i].sim, lam, mu, rho, 1);
            if (r != EWS_OK) return r;
            b[i].seis = seis[i];
            b[i].g_lam = gs[3 * i];
            b[i].g_mu = gs[3 * i + 1];
            b[i].g_rho = gs[3 * i + 2];
        }
        ews_batch_options o{};
        o.ckpt_every = ckpt_every;
        ews_status r = ews_batch(nshots, b.data(), &o, st);
        if (r != EWS_OK) return r;
        double J0 = 0;
        for (int i = 0; i < nshots; ++i) J0 += b[i].misfit;
        // summed gradient per parameter
        std::vector<const float*> hp(3 * nshots);
        for (int q = 0; q < 3; ++q)
            for (int i = 0; i < nshots; ++i) hp[q * nshots + i] = gs[3 * i + q];
        FCK(cudaMemcpyAsync(d_gl, hp.data(), hp.size() * sizeof(float*), cudaMemcpyHostToDevice, st));
        for (int q = 0; q < 3; ++q)
            k_sum_shots<<<blocks_for(n), kThreads, 0, st>>>(d_gl + q * nshots, nshots, n, gt + q * n);
        FCK(cudaGetLastError());
        // per-parameter scale: a unit step changes each parameter by at most
        // its largest magnitude
        FCK(cudaMemsetAsync(d_max, 0, 6 * sizeof(unsigned), st));
        const float* model[3] = {lam, mu, rho};
        for (int q = 0; q < 3; ++q) {
            k_absmax<<<blocks_for(n), kThreads, 0, st>>>(gt + q * n, n, d_max + q);
            k_absmax<<<blocks_for(n), kThreads, 0, st>>>(model[q], n, d_max + 3 + q);
        }
        FCK(cudaGetLastError());
        unsigned hm[6];
        FCK(cudaMemcpyAsync(hm, d_max, sizeof(hm), cudaMemcpyDeviceToHost, st));
        FCK(cudaStreamSynchronize(st));
        float sc[3];
        for (int q = 0; q < 3; ++q) {
            float gmax, mmax;
            std::memcpy(&gmax, &hm[q], 4);
            std::memcpy(&mmax, &hm[3 + q], 4);
            sc[q] = gmax > 0 ? mmax / gmax : 0.0f;
        }
        // misfit of all shots at a trial step (batched forward runs)
        auto misfit_at = [&](double alpha, double* J) -> ews_status {
            k_trial_model<<<blocks_for(n), kThreads, 0, st>>>(lam, mu, rho, gt, gt + n, gt + 2 * n,
                                                             sc[0], sc[1], sc[2], (float)alpha, n,
                                                             trial, trial + n, trial + 2 * n);
            FCK(cudaGetLastError());
            std::vector<ews_batch_shot> f(nshots);
            for (int i = 0; i < nshots; ++i) {
                ews_status rr = ews_set_model_lame(shots[i].sim, trial, trial + n, trial + 2 * n, 1);
                if (rr != EWS_OK) return rr;
                f[i] = ews_batch_shot{};
                f[i].sim = shots[i].sim;
                f[i].nt = shots[i].nt;
                f[i].dt = shots[i].dt;
                f[i].seis = seis[i];
            }
            ews_status rr = ews_batch(nshots, f.data(), nullptr, st);
            if (rr != EWS_OK) return rr;
            FCK(cudaMemsetAsync(d_mis, 0, sizeof(double), st));
            for (int i = 0; i < nshots; ++i) {
                const long long ns = 3LL * shots[i].sim->nrec * shots[i].nt;
                if (ns > 0)
                    k_misfit<<<blocks_for(ns), kThreads, 0, st>>>(seis[i], shots[i].observed, ns,
                                                                 (float)shots[i].dt, d_mis);
            }
            FCK(cudaGetLastError());
            FCK(cudaMemcpyAsync(J, d_mis, sizeof(double), cudaMemcpyDeviceToHost, st));
            FCK(cudaStreamSynchronize(st));
            return EWS_OK;
        };
        const double a1 = max_rel_step, a2 = 0.5 * max_rel_step;
        double J1 = 0, J2 = 0;
        if ((r = misfit_at(a1, &J1)) != EWS_OK) return r;
        if ((r = misfit_at(a2, &J2)) != EWS_OK) return r;
        // parabola through (0, J0), (a2, J2), (a1, J1); its minimum if convex
        const double c2 = 2.0 * (J1 - 2.0 * J2 + J0) / (a1 * a1);
        const double c1 = (4.0 * J2 - J1 - 3.0 * J0) / a1;
        double a = J1 < J2 ? a1 : a2;
        if (c2 > 0) a = std::min(std::max(-c1 / (2.0 * c2), 0.1 * a1), 2.0 * a1);
        double Ja = 0;
        if ((r = misfit_at(a, &Ja)) != EWS_OK) return r;
        const double best = std::min(std::min(J1, J2), Ja);
        if (best >= J0) {            // no decrease: keep the model
            a = 0;
            Ja = J0;
            for (int i = 0; i < nshots; ++i)
                if ((r = ews_set_model_lame(shots[i].sim, lam, mu, rho, 1)) != EWS_OK) return r;
        } else {
            if (best < Ja) {         // a trial point beat the parabola's minimum
                a = best == J1 ? a1 : a2;
                Ja = best;
                if ((r = misfit_at(a, &Ja)) != EWS_OK) return r;
            }
            // the simulations already hold the accepted model; copy it out
            FCK(cudaMemcpyAsync(lam, trial, n * sizeof(float), cudaMemcpyDeviceToDevice, st));
            FCK(cudaMemcpyAsync(mu, trial + n, n * sizeof(float), cudaMemcpyDeviceToDevice, st));
            FCK(cudaMemcpyAsync(rho, trial + 2 * n, n * sizeof(float), cudaMemcpyDeviceToDevice, st));
            FCK(cudaStreamSynchronize(st));
        }
        if (misfit0) *misfit0 = J0;
        if (misfit1) *misfit1 = Ja;
        if (step) *step = a;
        return EWS_OK;
    };
    result = run();
    cleanup();
    return result;
}
