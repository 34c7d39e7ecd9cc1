// S5: Kalman fit of caller hit lists (one thread per track, state and
// covariance in registers: compensated FP32 state, float-float covariance,
// Neumaier-compensated chi2).
#include <algorithm>

#include "tpc_fit.cuh"

namespace tpc {

namespace {

__global__ void __launch_bounds__(128) k_fit(
    const int32_t* __restrict__ trk_off, const int32_t* __restrict__ trk_hits, int32_t n_tracks,
    const int32_t* __restrict__ n_tracks_dev, const float* __restrict__ y,
    const float* __restrict__ z, const uint16_t* __restrict__ row,
    const int64_t* __restrict__ evt_off, int G, const Geo* __restrict__ geo, FitPrm P,
    float* params, float* cov, float* chi2o, int32_t* ndfo, const int32_t* __restrict__ st) {
    // clusters that failed validation are not read: every track reports a
    // failed fit
    const bool rejected = input_rejected(st);
    int T = n_tracks;
    if (n_tracks_dev) T = min(T, *n_tracks_dev);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        const int b = trk_off[t], n = trk_off[t + 1] - b;
        KF s;
        NSum chi2;
        ff Cf[15];
        const bool ok = !rejected && fit_track(trk_hits + b, n, y, z, row, evt_off, G, geo, P, s, Cf, chi2);
        float* po = params + (int64_t)t * 5;
        float* co = cov + (int64_t)t * 15;
        if (ok) {
#pragma unroll
            for (int i = 0; i < 3; ++i) s.p[i] += s.lo[i];
#pragma unroll
            for (int i = 0; i < 5; ++i) po[i] = s.p[i];
#pragma unroll
            for (int i = 0; i < 15; ++i) co[i] = Cf[i].hi + Cf[i].lo;
            chi2o[t] = chi2.value();
            ndfo[t] = 2 * n - 5;
        } else {
#pragma unroll
            for (int i = 0; i < 5; ++i) po[i] = 0.f;
#pragma unroll
            for (int i = 0; i < 15; ++i) co[i] = 0.f;
            chi2o[t] = 0.f;
            ndfo[t] = -1;
        }
    }
}

// The FP32-covariance variant (fit_track_f32); FP64 redos are counted in
// the status block.
__global__ void __launch_bounds__(128) k_fit32(
    const int32_t* __restrict__ trk_off, const int32_t* __restrict__ trk_hits, int32_t n_tracks,
    const int32_t* __restrict__ n_tracks_dev, const float* __restrict__ y,
    const float* __restrict__ z, const uint16_t* __restrict__ row,
    const int64_t* __restrict__ evt_off, int G, const Geo* __restrict__ geo, FitPrm P,
    float fp64_ratio, float fp64_det, float* params, float* cov, float* chi2o, int32_t* ndfo,
    int32_t* st) {
    const bool rejected = input_rejected(st);
    int T = n_tracks;
    if (n_tracks_dev) T = min(T, *n_tracks_dev);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        const int b = trk_off[t], n = trk_off[t + 1] - b;
        KF s;
        NSum chi2;
        const bool ok = !rejected && fit_track_f32(trk_hits + b, n, y, z, row, evt_off, G, geo, P, fp64_ratio,
                                                   fp64_det, &st[ST_FP64], s, chi2);
        float* po = params + (int64_t)t * 5;
        float* co = cov + (int64_t)t * 15;
        if (ok) {
#pragma unroll
            for (int i = 0; i < 5; ++i) po[i] = s.p[i] + (i < 3 ? s.lo[i] : 0.f);
#pragma unroll
            for (int i = 0; i < 15; ++i) co[i] = s.C[i];
            chi2o[t] = chi2.value();
            ndfo[t] = 2 * n - 5;
        } else {
#pragma unroll
            for (int i = 0; i < 5; ++i) po[i] = 0.f;
#pragma unroll
            for (int i = 0; i < 15; ++i) co[i] = 0.f;
            chi2o[t] = 0.f;
            ndfo[t] = -1;
        }
    }
}

}  // namespace

cudaError_t run_fit(tpc_ctx* c, const int32_t* trk_off, const int32_t* trk_hits, int32_t n_tracks,
                    const int32_t* n_tracks_dev, float* params, float* cov, float* chi2,
                    int32_t* ndf, cudaStream_t s) {
    if (n_tracks <= 0) return cudaSuccess;
    const tpc_params& p = c->prm;
    FitPrm fp;
    fp.sy2 = p.sigma_y2;
    fp.sz2 = p.sigma_z2;
    fp.kb = (float)(KAPPA * (double)p.bz);
    fp.snp_max = p.snp_max;
    fp.bz = p.bz;
    fp.seed_snp = p.seed_snp_max;
    fp.seed_qpt = p.seed_qpt_max;
    for (int i = 0; i < 5; ++i) fp.prior[i] = p.prior[i];
    // one warp per block: the tracks the device count leaves are few
    // compared with the capacity the grid is sized for, and single-warp
    // blocks spread the working warps over every SM instead of packing them
    // four to an SM on the first ones
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n_tracks + 31) / 32, (int64_t)c->n_sm * 128));
    c->mark(10, s);
    tpc::LaunchCount{}, k_fit<<<(unsigned)blocks, 32, 0, s>>>(trk_off, trk_hits, n_tracks, n_tracks_dev, c->y, c->z,
                                           c->row, c->evt_sector_off, c->n_events * NSEC,
                                           c->ws.at<Geo>(c->ws.L.geo), fp, params, cov, chi2, ndf,
                                           c->ws.at<int32_t>(c->ws.L.status));
    c->mark(11, s);
    return cudaGetLastError();
}

cudaError_t run_fit32(tpc_ctx* c, const int32_t* trk_off, const int32_t* trk_hits, int32_t n_tracks,
                      const int32_t* n_tracks_dev, float* params, float* cov, float* chi2,
                      int32_t* ndf, cudaStream_t s) {
    if (n_tracks <= 0) return cudaSuccess;
    const tpc_params& p = c->prm;
    FitPrm fp;
    fp.sy2 = p.sigma_y2;
    fp.sz2 = p.sigma_z2;
    fp.kb = (float)(KAPPA * (double)p.bz);
    fp.snp_max = p.snp_max;
    fp.bz = p.bz;
    fp.seed_snp = p.seed_snp_max;
    fp.seed_qpt = p.seed_qpt_max;
    for (int i = 0; i < 5; ++i) fp.prior[i] = p.prior[i];
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n_tracks + 31) / 32, (int64_t)c->n_sm * 128));
    c->mark(10, s);
    tpc::LaunchCount{}, k_fit32<<<(unsigned)blocks, 32, 0, s>>>(
        trk_off, trk_hits, n_tracks, n_tracks_dev, c->y, c->z, c->row, c->evt_sector_off, c->n_events * NSEC,
        c->ws.at<Geo>(c->ws.L.geo), fp, p.fp64_ratio, p.fp64_det, params, cov, chi2, ndf,
        c->ws.at<int32_t>(c->ws.L.status));
    c->mark(11, s);
    return cudaGetLastError();
}

}  // namespace tpc
