// The device transport (tpc_dev.cuh, kf_move<float>) run on the host: reads
// cases from argv[1] and writes the moved states and Jacobians to argv[2],
// for comparison with the oracle's FP64 transport.  Host code only; no
// kernel is launched.
//   input:  n (int64), then per case x1, p[5], x2 (double), s1, s2 (int32),
//           kb, snp_max (float);
//   output: per case ok (int32), p_out[5] (double, value plus compensation),
//           jac[25] (double, row-major d p_out / d p).
#include <cstdio>
#include <vector>

#include "tpc_dev.cuh"

using namespace tpc;

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    int64_t n;
    if (fread(&n, sizeof n, 1, f) != 1 || n < 0) return 3;
    const Geo geo = make_geo();
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    for (int64_t i = 0; i < n; ++i) {
        double x1, p[5], x2;
        int32_t s12[2];
        float kp[2];
        if (fread(&x1, 8, 1, f) != 1 || fread(p, 8, 5, f) != 5 || fread(&x2, 8, 1, f) != 1 ||
            fread(s12, 4, 2, f) != 2 || fread(kp, 4, 2, f) != 2)
            return 3;
        KF s;
        s.x = x1;
        s.frame = s12[0];
        for (int k = 0; k < 5; ++k) s.p[k] = (float)p[k];
        for (int k = 0; k < 3; ++k) s.lo[k] = 0.f;
        for (int k = 0; k < 15; ++k) s.C[k] = 0.f;
        MoveJ mj;
        mj.valid = false;
        const int32_t ok = kf_move<float>(s, x2, s12[1], &geo, kp[0], kp[1], &mj) ? 1 : 0;
        double out[30] = {};
        if (ok) {
            for (int k = 0; k < 5; ++k) out[k] = (double)s.p[k] + (k < 3 ? (double)s.lo[k] : 0.0);
            double* J = out + 5;
            J[0] = mj.j00; J[2] = mj.j02; J[4] = mj.j04;
            J[5] = mj.j10; J[6] = 1.0; J[7] = mj.j12; J[8] = mj.j13; J[9] = mj.j14;
            J[10] = mj.j20; J[12] = mj.j22; J[14] = mj.j24;
            J[18] = 1.0; J[24] = 1.0;
        }
        fwrite(&ok, 4, 1, o);
        fwrite(out, 8, 30, o);
    }
    fclose(f);
    fclose(o);
    printf("ok\n");
    return 0;
}
