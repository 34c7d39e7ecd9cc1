// The A/C-side association's per-pair functions (tpc_sides.cuh: the
// junction test and the six-parameter fit with t0) and the five-parameter
// end fits they start from (tpc_fit_ex.cuh), run on the host over given
// (inner, outer) pairs of tracks, for comparison with the FP64 oracle.
// Host code only; no kernel is launched.
//   input:  n, G, T, P (int64); y[n], z[n] (float); row[n] (uint16);
//           evt_off[G+1] (int64); trk_off[T+1], trk_hits[...] (int32);
//           pairs[2 P] (int32: inner, outer); sy2, sz2, snp_max, bz,
//           seed_snp, seed_qpt, prior[5] (float); t0_prior, v_drift (double)
//   output: per pair ok, c4, zmem, t0s, params6[6], cov6[21], chi2, dchi2
//           (double)
#include <cstdio>
#include <vector>

#include "tpc_sides.cuh"

using namespace tpc;

template <class T>
static bool rd(FILE* f, T* p, size_t n) { return fread(p, sizeof(T), n, f) == n; }

static bool ends_of(const int32_t* h, int m, const HitSrc& H, const Geo* geo, ExPrm P, SideEnd& e) {
    KFD s;
    double c2;
    P.outward = false;
    if (!fit_ex(h, m, H, geo, P, s, c2, nullptr)) return false;
    for (int k = 0; k < 5; ++k) e.p_in[k] = s.p[k] + (k < 3 ? s.lo[k] : 0.0);
    for (int k = 0; k < 15; ++k) e.C_in[k] = s.C[k];
    e.x_in = s.x;
    e.s_in = s.frame;
    e.chi2_in = c2;
    P.outward = true;
    if (!fit_ex(h, m, H, geo, P, s, c2, nullptr)) return false;
    for (int k = 0; k < 5; ++k) e.p_out[k] = s.p[k] + (k < 3 ? s.lo[k] : 0.0);
    for (int k = 0; k < 15; ++k) e.C_out[k] = s.C[k];
    e.x_out = s.x;
    e.s_out = s.frame;
    return true;
}

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    int64_t hdr[4];
    if (!rd(f, hdr, 4) || hdr[0] < 0 || hdr[1] < 1 || hdr[2] < 0 || hdr[3] < 0) return 3;
    const int64_t n = hdr[0], G = hdr[1], T = hdr[2], NP = hdr[3];
    std::vector<float> y(n), z(n);
    std::vector<uint16_t> row(n);
    std::vector<int64_t> off(G + 1);
    std::vector<int32_t> toff(T + 1);
    if (!rd(f, y.data(), n) || !rd(f, z.data(), n) || !rd(f, row.data(), n) || !rd(f, off.data(), G + 1) ||
        !rd(f, toff.data(), T + 1))
        return 3;
    std::vector<int32_t> hits(toff[T]), pairs(2 * NP);
    float prm[11];
    double sd[2];
    if (!rd(f, hits.data(), hits.size()) || !rd(f, pairs.data(), pairs.size()) || !rd(f, prm, 11) || !rd(f, sd, 2))
        return 3;
    fclose(f);
    for (int64_t i = 0; i < n; ++i)
        if (row[i] >= NROW) return 4;
    for (int32_t h : hits)
        if (h < 0 || h >= n) return 4;
    for (int32_t t : pairs)
        if (t < 0 || t >= T) return 4;
    ExPrm P;
    P.sy2 = prm[0];
    P.sz2 = prm[1];
    P.snp_max = prm[2];
    P.kb = KAPPA * (double)prm[3];
    P.bz = prm[3];
    P.seed_snp = prm[4];
    P.seed_qpt = prm[5];
    for (int i = 0; i < 5; ++i) P.prior[i] = prm[6 + i];
    P.x0 = 0.0;
    P.eloss = 0.0;
    P.mass = 0.13957;
    P.outward = false;
    SidesPrm S{10, 8, 30.0, 3.0, 10.0, 40.0, sd[0], sd[1]};
    const Geo geo = make_geo();
    const HitSrc H{y.data(), z.data(), row.data(), off.data(), (int)G};
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    for (int64_t k = 0; k < NP; ++k) {
        const int i = pairs[2 * k], j = pairs[2 * k + 1];
        double out[34] = {};
        SideEnd a, b;
        const int bi = toff[i], ni = toff[i + 1] - bi, bo = toff[j], no = toff[j + 1] - bo;
        double c4 = 0, zmem = 0, t0s = 0, q[6], C[21], chi2 = 0;
        bool ok = ends_of(hits.data() + bi, ni, H, &geo, P, a) && ends_of(hits.data() + bo, no, H, &geo, P, b);
        ok = ok && junction(a, side_sgn(sector_of(H, hits[bi])), b, &geo, P, S, c4, zmem, t0s);
        ok = ok && fit_t0(hits.data() + bo, no, hits.data() + bi, ni, t0s, H, &geo, P, S, q, C, chi2);
        out[0] = ok ? 1.0 : 0.0;
        if (ok) {
            out[1] = c4;
            out[2] = zmem;
            out[3] = t0s;
            for (int u = 0; u < 6; ++u) out[4 + u] = q[u];
            for (int u = 0; u < 21; ++u) out[10 + u] = C[u];
            out[31] = chi2;
            out[32] = chi2 - a.chi2_in - b.chi2_in;
        }
        fwrite(out, sizeof(double), 34, o);
    }
    fclose(o);
    return 0;
}
