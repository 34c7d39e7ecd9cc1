// The Kalman-filter variants' per-track functions (tpc_fit_ex.cuh: fit_ex
// with material, inward or outward, and the smoother smooth_back) run on the
// host over whole tracks, for comparison with the FP64 oracle.  Host code
// only; no kernel is launched.
//   input:  n, G, T (int64); y[n], z[n] (float); row[n] (uint16);
//           evt_off[G+1] (int64); trk_off[T+1], trk_hits[...] (int32);
//           sy2, sz2, snp_max, bz, seed_snp, seed_qpt, prior[5], x0, eloss,
//           mass (float); direction, smooth (int32)
//   output: per track params[5], cov[15], chi2, ndf (double), then, when
//           smooth, 20 doubles per hit of the lists.
#include <cstdio>
#include <vector>

#include "tpc_fit_ex.cuh"

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
    float prm[14];
    int32_t mode[2];
    if (!rd(f, hits.data(), hits.size()) || !rd(f, prm, 14) || !rd(f, mode, 2)) return 3;
    fclose(f);
    for (int64_t i = 0; i < n; ++i)
        if (row[i] >= NROW) return 4;
    for (int32_t h : hits)
        if (h < 0 || h >= n) return 4;
    ExPrm P;
    P.sy2 = prm[0];
    P.sz2 = prm[1];
    P.snp_max = prm[2];
    P.kb = KAPPA * (double)prm[3];
    P.bz = prm[3];
    P.seed_snp = prm[4];
    P.seed_qpt = prm[5];
    for (int i = 0; i < 5; ++i) P.prior[i] = prm[6 + i];
    P.x0 = prm[11];
    P.eloss = prm[12];
    P.mass = prm[13];
    P.outward = mode[0] == 1;
    const bool smooth = mode[1] != 0 && !P.outward;
    const Geo geo = make_geo();
    const HitSrc H{y.data(), z.data(), row.data(), off.data(), (int)G};
    std::vector<double> sm(smooth ? (size_t)20 * hits.size() : 0, 0.0);
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    for (int64_t t = 0; t < T; ++t) {
        const int b = toff[t], m = toff[t + 1] - b;
        KFD s;
        double chi2 = 0.0;
        double* filt = smooth ? sm.data() + (size_t)20 * b : nullptr;
        bool ok = fit_ex(hits.data() + b, m, H, &geo, P, s, chi2, filt);
        if (ok && filt) ok = smooth_back(hits.data() + b, m, H, &geo, P, filt);
        double out[22];
        for (int i = 0; i < 5; ++i) out[i] = ok ? s.p[i] + (i < 3 ? s.lo[i] : 0.0) : 0.0;
        for (int i = 0; i < 15; ++i) out[5 + i] = ok ? s.C[i] : 0.0;
        out[20] = ok ? chi2 : 0.0;
        out[21] = ok ? 2 * m - 5 : -1;
        if (!ok && filt)
            for (int i = 0; i < 20 * m; ++i) filt[i] = 0.0;
        fwrite(out, sizeof(double), 22, o);
    }
    if (smooth) fwrite(sm.data(), sizeof(double), sm.size(), o);
    fclose(o);
    return 0;
}
