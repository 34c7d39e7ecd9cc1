// The FP32-covariance fit (tpc_fit.cuh: fit_track_f32, the per-track
// function of tpc_fit_tracks_fp32 and the precision pattern of the tracklet
// lanes: kf_move<float> with the covariance in FP32, kf_update with its FP64
// redo of cancelling updates) run over whole tracks on the host: reads a
// batch and track lists from argv[1], writes every track's fit to argv[2],
// for comparison with the FP64 oracle.  Host code only; no kernel is
// launched.
//   input:  n, G, T (int64); y[n], z[n] (float); row[n] (uint16);
//           evt_off[G+1] (int64); trk_off[T+1], trk_hits[...] (int32);
//           sy2, sz2, snp_max, bz, seed_snp, seed_qpt, prior[5],
//           fp64_ratio, fp64_det (float, the library's parameters);
//   output: per track params[5], cov[15], chi2 (float), ndf (int32), then
//           the number of FP64 redos (int32).
#include <cstdio>
#include <vector>

#include "tpc_fit.cuh"  // FitPrm and the Kalman pieces

using namespace tpc;

template <class T>
static bool rd(FILE* f, T* p, size_t n) { return fread(p, sizeof(T), n, f) == n; }

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    int64_t nGT[3];
    if (!rd(f, nGT, 3) || nGT[0] < 0 || nGT[1] < 1 || nGT[2] < 0) return 3;
    const int64_t n = nGT[0], G = nGT[1], T = nGT[2];
    std::vector<float> y(n), z(n);
    std::vector<uint16_t> row(n);
    std::vector<int64_t> off(G + 1);
    std::vector<int32_t> toff(T + 1);
    if (!rd(f, y.data(), n) || !rd(f, z.data(), n) || !rd(f, row.data(), n) || !rd(f, off.data(), G + 1) ||
        !rd(f, toff.data(), T + 1))
        return 3;
    std::vector<int32_t> hits(toff[T]);
    float prm[13];
    if (!rd(f, hits.data(), hits.size()) || !rd(f, prm, 13)) return 3;
    fclose(f);
    for (int64_t i = 0; i < n; ++i)
        if (row[i] >= NROW) return 4;
    for (int32_t h : hits)
        if (h < 0 || h >= n) return 4;
    FitPrm P;
    P.sy2 = prm[0];
    P.sz2 = prm[1];
    P.snp_max = prm[2];
    P.kb = (float)(KAPPA * (double)prm[3]);
    P.bz = prm[3];
    P.seed_snp = prm[4];
    P.seed_qpt = prm[5];
    for (int i = 0; i < 5; ++i) P.prior[i] = prm[6 + i];
    const Geo geo = make_geo();
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    int n_fp64 = 0;
    for (int64_t t = 0; t < T; ++t) {
        const int b = toff[t], m = toff[t + 1] - b;
        const int32_t* h = hits.data() + b;
        KF s;
        NSum chi2;
        const bool ok = fit_track_f32(h, m, y.data(), z.data(), row.data(), off.data(), (int)G, &geo, P,
                                      prm[11], prm[12], &n_fp64, s, chi2);
        float out[21] = {};
        int32_t ndf = -1;
        if (ok) {
            for (int i = 0; i < 5; ++i) out[i] = s.p[i] + (i < 3 ? s.lo[i] : 0.f);
            for (int i = 0; i < 15; ++i) out[5 + i] = s.C[i];
            out[20] = chi2.value();
            ndf = 2 * m - 5;
        }
        fwrite(out, 4, 21, o);
        fwrite(&ndf, 4, 1, o);
    }
    fwrite(&n_fp64, 4, 1, o);
    fclose(o);
    printf("ok\n");
    return 0;
}
