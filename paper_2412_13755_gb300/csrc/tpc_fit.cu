// S5: Kalman fit of caller hit lists (one thread per track, state and
// covariance in registers: compensated FP32 state, float-float covariance,
// Neumaier-compensated chi2).
#include <algorithm>

#include "tpc_dev.cuh"

namespace tpc {

namespace {

struct FitPrm {
    float sy2, sz2, kb, snp_max;
    double bz, seed_snp, seed_qpt;
    float prior[5];
};

__global__ void __launch_bounds__(128) k_fit(
    const int32_t* __restrict__ trk_off, const int32_t* __restrict__ trk_hits, int32_t n_tracks,
    const int32_t* __restrict__ n_tracks_dev, const float* __restrict__ y,
    const float* __restrict__ z, const uint16_t* __restrict__ row,
    const int64_t* __restrict__ evt_off, int G, const Geo* __restrict__ geo, FitPrm P,
    float* params, float* cov, float* chi2o, int32_t* ndfo) {
    int T = n_tracks;
    if (n_tracks_dev) T = min(T, *n_tracks_dev);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        const int b = trk_off[t], n = trk_off[t + 1] - b;
        const int32_t* h = trk_hits + b;
        bool ok = n >= 3;
        KF s;
        NSum chi2;
        ff Cf[15];
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
#pragma unroll
            for (int i = 0; i < 15; ++i) Cf[i] = ff_from(s.C[i]);
            int g = -1;
            int64_t gb = 0, ge = 0;
            // the next hit's index and data are read a step ahead, so that
            // their loads overlap the current step's arithmetic
            int cn = h[0];
            int rn = row[cn];
            float yn = y[cn], zn = z[cn];
            for (int j = 0; j < n && ok; ++j) {
                const int c = cn, rc = rn;
                const float yc = yn, zc = zn;
                if (j + 1 < n) cn = h[j + 1];
                if (c < gb || c >= ge) {  // group lookup, cached while hits stay in one group
                    g = group_of(evt_off, G, c);
                    gb = evt_off[g];
                    ge = evt_off[g + 1];
                }
                MoveJ mj;
                ok = kf_move<float, true, false>(s, geo->row_xd[rc], g % NSEC, geo, P.kb, P.snp_max, &mj);
                if (j + 1 < n) {
                    rn = row[cn];
                    yn = y[cn];
                    zn = z[cn];
                }
                if (ok) {
                    if (mj.j00 == 1.f && mj.j22 == 1.f && mj.j10 == 0.f && mj.j20 == 0.f)
                        cov_jct_ff_frame(Cf, mj.j02, mj.j04, mj.j12, mj.j13, mj.j14, mj.j24);
                    else
                        cov_jct_ff(Cf, mj.j00, mj.j02, mj.j04, mj.j10, mj.j12, mj.j13, mj.j14, mj.j20, mj.j22,
                                   mj.j24);
                    chi2.add(kf_update_ff(s, Cf, yc, zc, P.sy2, P.sz2));
                }
            }
        }
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
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n_tracks + 127) / 128, 152 * 32));
    c->mark(10, s);
    tpc::LaunchCount{}, k_fit<<<(unsigned)blocks, 128, 0, s>>>(trk_off, trk_hits, n_tracks, n_tracks_dev, c->y, c->z,
                                           c->row, c->evt_sector_off, c->n_events * NSEC,
                                           c->ws.at<Geo>(c->ws.L.geo), fp, params, cov, chi2, ndf);
    c->mark(11, s);
    return cudaGetLastError();
}

}  // namespace tpc
