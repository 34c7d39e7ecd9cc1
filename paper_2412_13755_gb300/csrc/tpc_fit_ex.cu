// NEXT-3: Kalman-filter variants of the fit -- material in the pad-row
// planes (multiple-scattering process noise, mean energy loss), the outward
// refit, and a Rauch-Tung-Striebel smoother giving the state at every
// cluster.  One thread per track, in FP64: the variants refine found tracks
// (they are not on the pattern-recognition path), and the smoother's gain
// inverts predicted covariances that are nearly singular without process
// noise, which FP32 cannot carry.
#include <algorithm>

#include "tpc_fit_ex.cuh"

namespace tpc {

namespace {

__global__ void __launch_bounds__(128) k_fit_ex(
    const int32_t* __restrict__ trk_off, const int32_t* __restrict__ trk_hits, int32_t n_tracks,
    const int32_t* __restrict__ n_tracks_dev, HitSrc H, const Geo* __restrict__ geo, ExPrm P,
    float* params, float* cov, float* chi2o, int32_t* ndfo, double* smoothed,
    const int32_t* __restrict__ st) {
    const bool rejected = input_rejected(st);
    int T = n_tracks;
    if (n_tracks_dev) T = min(T, *n_tracks_dev);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        const int b = trk_off[t], n = trk_off[t + 1] - b;
        KFD s;
        double chi2 = 0.0;
        double* filt = smoothed ? smoothed + (size_t)20 * b : nullptr;
        bool ok = !rejected && fit_ex(trk_hits + b, n, H, geo, P, s, chi2, filt);
        if (ok && filt) ok = smooth_back(trk_hits + b, n, H, geo, P, filt);
        float* po = params + (int64_t)t * 5;
        float* co = cov + (int64_t)t * 15;
        for (int i = 0; i < 5; ++i) po[i] = ok ? (float)(s.p[i] + (i < 3 ? s.lo[i] : 0.0)) : 0.f;
        for (int i = 0; i < 15; ++i) co[i] = ok ? (float)s.C[i] : 0.f;
        chi2o[t] = ok ? (float)chi2 : 0.f;
        ndfo[t] = ok ? 2 * n - 5 : -1;
        if (!ok && filt)
            for (int i = 0; i < 20 * n; ++i) filt[i] = 0.0;
    }
}

}  // namespace

cudaError_t run_fit_ex(tpc_ctx* c, const int32_t* trk_off, const int32_t* trk_hits, int32_t n_tracks,
                       const int32_t* n_tracks_dev, const tpc_fit_options* o, float* params, float* cov,
                       float* chi2, int32_t* ndf, double* smoothed, cudaStream_t s) {
    if (n_tracks <= 0) return cudaSuccess;
    const tpc_params& p = c->prm;
    ExPrm P;
    P.sy2 = p.sigma_y2;
    P.sz2 = p.sigma_z2;
    P.kb = KAPPA * (double)p.bz;
    P.snp_max = p.snp_max;
    P.bz = p.bz;
    P.seed_snp = p.seed_snp_max;
    P.seed_qpt = p.seed_qpt_max;
    for (int i = 0; i < 5; ++i) P.prior[i] = p.prior[i];
    P.x0 = o ? o->mat_x_x0 : 0.0;
    P.eloss = o ? o->mat_eloss : 0.0;
    P.mass = o ? o->mass : 0.13957;
    P.outward = o && o->direction == 1;
    const HitSrc H{c->y, c->z, c->row, c->evt_sector_off, c->n_events * NSEC};
    // single-warp blocks: the FP64 pipe of every SM takes part even when
    // the tracks fill fewer than 128 x SMs lanes
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n_tracks + 31) / 32, (int64_t)c->n_sm * 128));
    c->mark(10, s);
    tpc::LaunchCount{}, k_fit_ex<<<(unsigned)blocks, 32, 0, s>>>(
        trk_off, trk_hits, n_tracks, n_tracks_dev, H, c->ws.at<Geo>(c->ws.L.geo), P, params, cov, chi2, ndf,
        smoothed, c->ws.at<int32_t>(c->ws.L.status));
    c->mark(11, s);
    return cudaGetLastError();
}

}  // namespace tpc
