// The adjoint kernel's per-track function (tpc_adjoint.cuh, adjoint_track:
// forward fit with checkpoints and the hand-written reverse sweep) run on
// the host for every track, summing as the kernel does, for comparison with
// the FP64 oracle's dual-number gradients.  Host code only; no kernel is
// launched.
//   input:  n, G, T (int64); y[n], z[n] (float); row[n] (uint16);
//           evt_off[G+1] (int64); trk_off[T+1], trk_hits[...] (int32);
//           align[216] (double); with_field (int32), grid n_band, n_y, n_z
//           (int32), u_lo, u_inv, z_inv (float), field[3 n_vox] (double);
//           sy2, sz2, snp_max, bz, seed_snp, seed_qpt, fp64_ratio,
//           fp64_det, prior[5] (float, the library's parameters);
//   output: chi2 (double), grad_align[216], grad_field[3 n_vox] (double),
//           status, detail (int32).
#include <cstdio>
#include <vector>

#include "tpc_adjoint.cuh"

using namespace tpc;

template <class T>
static bool rd(FILE* f, T* p, size_t n) { return fread(p, sizeof(T), n, f) == n; }

struct HostAcc {
    double c2 = 0.0;
    std::vector<double> al = std::vector<double>(216, 0.0);
    std::vector<double> fl;
    bool field_on = false;
    int st = 0, det = 0;
    void chi2(double v) { c2 += v; }
    void align(int i, double v) { al[i] += v; }
    void field(int64_t i, double v) { fl[i] += v; }
    bool want_field() const { return field_on; }
    void status(int code, int detail) {
        if (!st) {
            st = code;
            det = detail;
        }
    }
};

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
    double align[216];
    int32_t gi[4];
    float gf[3];
    if (!rd(f, hits.data(), hits.size()) || !rd(f, align, 216) || !rd(f, gi, 4) || !rd(f, gf, 3)) return 3;
    const FieldGridD fg{gi[1], gi[2], gi[3], gf[0], gf[1], gf[2]};
    const int64_t nv = (int64_t)NSEC * fg.n_band * fg.n_y * fg.n_z;
    std::vector<double> field(3 * nv);
    float prm[13];
    if (!rd(f, field.data(), field.size()) || !rd(f, prm, 13)) return 3;
    fclose(f);
    for (int64_t i = 0; i < n; ++i)
        if (row[i] >= NROW) return 4;
    for (int32_t h : hits)
        if (h < 0 || h >= n) return 4;
    tpc_params p;
    p.sigma_y2 = prm[0];
    p.sigma_z2 = prm[1];
    p.snp_max = prm[2];
    p.bz = prm[3];
    p.seed_snp_max = prm[4];
    p.seed_qpt_max = prm[5];
    p.fp64_ratio = prm[6];
    p.fp64_det = prm[7];
    for (int i = 0; i < 5; ++i) p.prior[i] = prm[8 + i];
    const AdjPrm P = adj_prm(p, true);
    const Geo geo = make_geo();
    std::vector<float> tab(NSEC * ROT_TAB);
    for (int s = 0; s < NSEC; ++s) adj_table_sector(align + 6 * s, tab.data() + s * ROT_TAB);
    HostAcc acc;
    acc.field_on = gi[0] != 0;
    acc.fl.assign(3 * nv, 0.0);
    std::vector<float> seg(CK * PRE_W);
    for (int64_t t = 0; t < T; ++t) {
        const int b = toff[t], m = toff[t + 1] - b;
        AdjHits hv = adj_hits_direct(hits.data() + b, y.data(), z.data(), row.data(), off.data(), (int)G);
        if (gi[0])
            adjoint_track<true>(hv, m, tab.data(), &geo, P, field.data(), fg, seg.data(), 1, acc);
        else
            adjoint_track<false>(hv, m, tab.data(), &geo, P, nullptr, fg, seg.data(), 1, acc);
    }
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    fwrite(&acc.c2, 8, 1, o);
    fwrite(acc.al.data(), 8, 216, o);
    fwrite(acc.fl.data(), 8, acc.fl.size(), o);
    const int32_t sd[2] = {acc.st, acc.det};
    fwrite(sd, 4, 2, o);
    fclose(o);
    printf("ok\n");
    return 0;
}
