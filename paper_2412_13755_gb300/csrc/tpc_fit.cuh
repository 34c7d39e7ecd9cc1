// S5: the Kalman fit of one track (outermost cluster first), shared by the
// fit kernel and, so that it can be checked against the FP64 oracle without
// a GPU, by host programs.  Compensated FP32 state, float-float covariance,
// Neumaier-compensated chi2.
#pragma once

#include "tpc_dev.cuh"

namespace tpc {

struct FitPrm {
    float sy2, sz2, kb, snp_max;
    double bz, seed_snp, seed_qpt;
    float prior[5];
};

// Fits the n clusters h[0..n) (input indices) from the seed of the first,
// middle and last; returns false when n < 3 or a transport fails.  s, Cf
// and chi2 hold the state at the last cluster.
TPC_HD bool fit_track(const int32_t* h, int n, const float* __restrict__ y,
                      const float* __restrict__ z, const uint16_t* __restrict__ row,
                      const int64_t* __restrict__ evt_off, int G, const Geo* __restrict__ geo,
                      FitPrm P, KF& s, ff Cf[15], NSum& chi2) {
    bool ok = n >= 3;
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
        // the next hit's index and data are read a step ahead, so that their
        // loads overlap the current step's arithmetic
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
    return ok;
}

// The same fit with the covariance in FP32 and an update redone in FP64
// when it cancels (a posterior variance below fp64_ratio x its prior, or det
// S <= fp64_det S00 S11; kf_update counts each redo in *n_fp64): the
// precision pattern of the tracklet lanes, where float-float is not carried.
// s.C holds the covariance at the last cluster.
TPC_HD bool fit_track_f32(const int32_t* h, int n, const float* __restrict__ y,
                          const float* __restrict__ z, const uint16_t* __restrict__ row,
                          const int64_t* __restrict__ evt_off, int G, const Geo* __restrict__ geo,
                          FitPrm P, float fp64_ratio, float fp64_det, int* n_fp64, KF& s, NSum& chi2) {
    bool ok = n >= 3;
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
        // the next hit's index and data are read a step ahead
        int cn = h[0];
        int rn = row[cn];
        float yn = y[cn], zn = z[cn];
        for (int j = 0; j < n && ok; ++j) {
            const int c = cn, rc = rn;
            const float yc = yn, zc = zn;
            if (j + 1 < n) cn = h[j + 1];
            if (c < gb || c >= ge) {
                g = group_of(evt_off, G, c);
                gb = evt_off[g];
                ge = evt_off[g + 1];
            }
            MoveJ mj;
            mj.valid = false;
            ok = kf_move<float>(s, geo->row_xd[rc], g % NSEC, geo, P.kb, P.snp_max, &mj);
            if (j + 1 < n) {
                rn = row[cn];
                yn = y[cn];
                zn = z[cn];
            }
            if (ok) chi2.add(kf_update(s, yc, zc, P.sy2, P.sz2, fp64_ratio, fp64_det, n_fp64, &mj));
        }
    }
    return ok;
}

}  // namespace tpc
