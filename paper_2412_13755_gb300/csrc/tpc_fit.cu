// S5: Kalman fit of caller hit lists (one thread per track, state and
// covariance in registers, FP32 with FP64 redo of cancelling updates,
// Neumaier-compensated chi2).
#include <algorithm>

#include "tpc_dev.cuh"

namespace tpc {

namespace {

struct FitPrm {
    float sy2, sz2, kb, snp_max, fp64_ratio, fp64_det, fp64_weak_qpt;
    double bz, seed_snp, seed_qpt;
    float prior[5];
};

__global__ void __launch_bounds__(128) k_fit(
    const int32_t* __restrict__ trk_off, const int32_t* __restrict__ trk_hits, int32_t n_tracks,
    const int32_t* __restrict__ n_tracks_dev, const float* __restrict__ y,
    const float* __restrict__ z, const uint16_t* __restrict__ row,
    const int64_t* __restrict__ evt_off, int G, const Geo* __restrict__ geo, FitPrm P,
    float* params, float* cov, float* chi2o, int32_t* ndfo, int32_t* st, int32_t* refit) {
    int T = n_tracks;
    if (n_tracks_dev) T = min(T, *n_tracks_dev);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        const int b = trk_off[t], n = trk_off[t + 1] - b;
        const int32_t* h = trk_hits + b;
        bool ok = n >= 3;
        KF s;
        NSum chi2;
        if (ok) {
            int rows[3], secs[3];
            float ys[3], zs[3];
            const int pick[3] = {0, n / 2, n - 1};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int c = h[pick[k]];
                rows[k] = row[c];
                secs[k] = group_of(evt_off, G, c) % NSEC;
                ys[k] = y[c];
                zs[k] = z[c];
            }
            kf_seed(s, rows, secs, ys, zs, true, geo, P.bz, P.seed_snp, P.seed_qpt, P.prior);
            int g = -1;
            int64_t gb = 0, ge = 0;
            for (int j = 0; j < n && ok; ++j) {
                const int c = h[j];
                if (c < gb || c >= ge) {  // group lookup, cached while hits stay in one group
                    g = group_of(evt_off, G, c);
                    gb = evt_off[g];
                    ge = evt_off[g + 1];
                }
                MoveJ mj;
                ok = kf_move<float>(s, geo->row_xd[row[c]], g % NSEC, geo, P.kb, P.snp_max, &mj);
                if (ok) chi2.add(kf_update(s, y[c], z[c], P.sy2, P.sz2, P.fp64_ratio, P.fp64_det,
                                           &st[ST_FP64], &mj));
            }
        }
        // A track whose curvature stays weakly determined (final q/pT variance
        // above fp64_weak_qpt x its prior) is an ill-conditioned fit: its
        // sub-micron sagittas are at the FP32 rounding level of the state
        // increments.  Such tracks are queued and refit in FP64 by k_fit_d.
        if (ok && s.C[14] > P.fp64_weak_qpt * P.prior[4]) refit[atomicAdd(&st[ST_NREFIT], 1)] = t;
        float* po = params + (int64_t)t * 5;
        float* co = cov + (int64_t)t * 15;
        if (ok) {
#pragma unroll
            for (int i = 0; i < 3; ++i) s.p[i] += s.lo[i];
#pragma unroll
            for (int i = 0; i < 5; ++i) po[i] = s.p[i];
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

// FP64 refit (seed, transport, update) of the queued weak-curvature tracks.
__global__ void __launch_bounds__(128) k_fit_d(
    const int32_t* __restrict__ trk_off, const int32_t* __restrict__ trk_hits,
    const float* __restrict__ y, const float* __restrict__ z, const uint16_t* __restrict__ row,
    const int64_t* __restrict__ evt_off, int G, const Geo* __restrict__ geo, FitPrm P,
    float* params, float* cov, float* chi2o, int32_t* ndfo, int32_t* st,
    const int32_t* __restrict__ refit) {
    const int nq = st[ST_NREFIT];
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        const int t = refit[q];
        const int b = trk_off[t], n = trk_off[t + 1] - b;
        const int32_t* h = trk_hits + b;
        KFD sd;
        {
            KF s0;
            int rows[3], secs[3];
            float ys[3], zs[3];
            const int pick[3] = {0, n / 2, n - 1};
            for (int k = 0; k < 3; ++k) {
                const int c = h[pick[k]];
                rows[k] = row[c];
                secs[k] = group_of(evt_off, G, c) % NSEC;
                ys[k] = y[c];
                zs[k] = z[c];
            }
            kf_seed(s0, rows, secs, ys, zs, true, geo, P.bz, P.seed_snp, P.seed_qpt, P.prior);
            sd.x = s0.x;
            sd.frame = s0.frame;
            for (int i = 0; i < 5; ++i) sd.p[i] = s0.p[i];
            sd.lo[0] = sd.lo[1] = sd.lo[2] = 0.0;
            for (int i = 0; i < 15; ++i) sd.C[i] = s0.C[i];
        }
        bool okd = true;
        double chi2 = 0.0;
        for (int j = 0; j < n && okd; ++j) {
            const int c = h[j];
            const int g = group_of(evt_off, G, c);
            okd = kf_move<double>(sd, geo->row_xd[row[c]], g % NSEC, geo, KAPPA * P.bz, (double)P.snp_max);
            if (okd) chi2 += kf_update_d(sd, y[c], z[c], P.sy2, P.sz2);
        }
        if (!okd) continue;  // keep the FP32 result
        atomicAdd(&st[ST_FP64], n);
        float* po = params + (int64_t)t * 5;
        float* co = cov + (int64_t)t * 15;
        for (int i = 0; i < 5; ++i) po[i] = (float)(sd.p[i] + (i < 3 ? sd.lo[i] : 0.0));
        for (int i = 0; i < 15; ++i) co[i] = (float)sd.C[i];
        chi2o[t] = (float)chi2;
        ndfo[t] = 2 * n - 5;
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
    fp.fp64_ratio = p.fp64_ratio;
    fp.fp64_det = p.fp64_det;
    fp.fp64_weak_qpt = p.fp64_weak_qpt;
    fp.bz = p.bz;
    fp.seed_snp = p.seed_snp_max;
    fp.seed_qpt = p.seed_qpt_max;
    for (int i = 0; i < 5; ++i) fp.prior[i] = p.prior[i];
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n_tracks + 127) / 128, 152 * 32));
    c->mark(10, s);
    int32_t* st = c->ws.at<int32_t>(c->ws.L.status);
    int32_t* refit = c->ws.at<int32_t>(c->ws.L.refit);
    cudaError_t e = fill_i32(st + ST_NREFIT, 1, 0, s);
    if (e != cudaSuccess) return e;
    tpc::LaunchCount{}, k_fit<<<(unsigned)blocks, 128, 0, s>>>(trk_off, trk_hits, n_tracks, n_tracks_dev, c->y, c->z,
                                           c->row, c->evt_sector_off, c->n_events * NSEC,
                                           c->ws.at<Geo>(c->ws.L.geo), fp, params, cov, chi2, ndf,
                                           st, refit);
    tpc::LaunchCount{}, k_fit_d<<<152 * 2, 128, 0, s>>>(trk_off, trk_hits, c->y, c->z, c->row,
                                                        c->evt_sector_off, c->n_events * NSEC,
                                                        c->ws.at<Geo>(c->ws.L.geo), fp, params, cov,
                                                        chi2, ndf, st, refit);
    c->mark(11, s);
    return cudaGetLastError();
}

}  // namespace tpc
