// NEXT-4: the drift-time offset t0 as a sixth state parameter, and the
// association of the A- and C-side segments of membrane-crossing tracks.
// A collision at drift-time offset t0 (us) is seen at z' = z - v t0 on side
// A (sectors 0..17) and at z' = z + v t0 on side C, the convention of the
// continuous-readout time frame (Sec. 1, Sec. 4).  The state (y, z, sin
// phi, tan lambda, q/pT, t0) carries the true z; the helix transport leaves
// t0 unchanged; a cluster of side sgn (+1 A, -1 C) measures
// (y, z - sgn v t0).  The per-track and per-pair pieces below are shared by
// the kernels in tpc_sides.cu and, so that they can be checked against the
// FP64 oracle without a GPU, by host programs.  FP64 throughout: the
// association refines found tracks and runs on a few per cent of them.
#pragma once

#include "tpc_fit_ex.cuh"

namespace tpc {

struct SidesPrm {
    int n_min, gap_max;
    double chi2_junction, z_membrane, z_pre, chi2_joint, t0_prior, v_drift;
};

// Packed symmetric 6x6, upper triangle row by row:
// 00 01 02 03 04 05 11 12 13 14 15 22 23 24 25 33 34 35 44 45 55
TPC_HD constexpr int s6(int i, int j) {
    return (i <= j ? i : j) * 6 - (i <= j ? i : j) * ((i <= j ? i : j) - 1) / 2 + (i <= j ? j : i) -
           (i <= j ? i : j);
}
static_assert(s6(0, 5) == 5 && s6(1, 1) == 6 && s6(2, 2) == 11 && s6(3, 3) == 15 && s6(4, 4) == 18 &&
                  s6(5, 5) == 20 && s6(5, 3) == 17,
              "packed 6x6 index");

TPC_HD int side_sgn(int sector) { return sector < NPHI ? 1 : -1; }

// The two ends of one found track, as the association sees them.
struct SideEnd {
    double p_in[5], C_in[15], x_in, chi2_in;  // inward fit: state at the innermost cluster
    double p_out[5], C_out[15], x_out;        // outward fit: state at the outermost cluster
    int32_t s_in, s_out;                      // sectors of those clusters
    int32_t ok;                               // bit 0: inward fit done; bit 1: outward fit done
};

// Kalman update of the six-parameter state with one cluster, a = -sgn v:
// H = [[1 0 0 0 0 0], [0 1 0 0 0 a]], S = H C H^T + R, K = C H^T S^-1,
// q += K r, C -= K H C.  Returns the predicted-residual chi2 r^T S^-1 r.
TPC_HD double kf6_update(double q[6], double C[21], double my, double mz, double a, double sy2, double sz2) {
    double h0[6], h1[6];  // rows of H C
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        h0[i] = C[s6(0, i)];
        h1[i] = C[s6(1, i)] + a * C[s6(5, i)];
    }
    const double r0 = my - q[0], r1 = mz - (q[1] + a * q[5]);
    const double S00 = h0[0] + sy2, S01 = h0[1] + a * h0[5], S11 = h1[1] + a * h1[5] + sz2;
    const double det = S00 * S11 - S01 * S01;
    const double i00 = S11 / det, i01 = -S01 / det, i11 = S00 / det;
    double k0[6], k1[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        k0[i] = h0[i] * i00 + h1[i] * i01;
        k1[i] = h0[i] * i01 + h1[i] * i11;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) q[i] += k0[i] * r0 + k1[i] * r1;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i; j < 6; ++j) C[s6(i, j)] -= k0[i] * h0[j] + k1[i] * h1[j];
    return r0 * r0 * i00 + 2.0 * r0 * r1 * i01 + r1 * r1 * i11;
}

// C <- G C G^T with G = diag(J, 1): the five helix rows follow the
// transport's Jacobian J (row-major 5x5), t0 is carried unchanged.
TPC_HD void cov6_move(double C[21], const double J[25]) {
    double M[6][6], T[6][6];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 6; ++j) M[i][j] = C[s6(i, j)];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            double a = 0.0;
#pragma unroll
            for (int l = 0; l < 5; ++l) a += J[i * 5 + l] * M[l][j];
            T[i][j] = a;
        }
#pragma unroll
    for (int j = 0; j < 6; ++j) T[5][j] = M[5][j];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i; j < 6; ++j) {
            double a;
            if (j < 5) {
                a = 0.0;
#pragma unroll
                for (int l = 0; l < 5; ++l) a += T[i][l] * J[j * 5 + l];
            } else {
                a = T[i][5];
            }
            C[s6(i, j)] = a;
        }
}

// r^T M^-1 r for a 4x4 SPD M (row-major) by Cholesky; false when M is not
// positive definite.
TPC_HD bool chi2_spd4(const double r[4], const double M[16], double& out) {
    double L[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) L[i][j] = 0.0;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j <= i; ++j) {
            double v = M[i * 4 + j];
            for (int l = 0; l < j; ++l) v -= L[i][l] * L[j][l];
            if (i == j) {
                if (!(v > 0.0)) return false;
                L[i][i] = sqrt(v);
            } else {
                L[i][j] = v / L[j][j];
            }
        }
    double w[4];
    out = 0.0;
    for (int i = 0; i < 4; ++i) {
        double v = r[i];
        for (int l = 0; l < i; ++l) v -= L[i][l] * w[l];
        w[i] = v / L[i][i];
        out += w[i] * w[i];
    }
    return true;
}

// The junction test of inner track i against outer track o: i's outward
// state moved to o's innermost plane; c4 = the chi2 of (y, sin phi, tan
// lambda, q/pT) against o's inward state with the sum of both covariances;
// zmem = the mean of the two apparent z there (the true z at the
// junction); t0s = (z'_o - z'_i) / (2 sgn_i v).  False when the move fails
// or the covariance is not positive definite.
TPC_HD bool junction(const SideEnd& a, int sgn_i, const SideEnd& b, const Geo* __restrict__ geo, const ExPrm& P,
                     const SidesPrm& S, double& c4, double& zmem, double& t0s) {
    KFD s;
    s.x = a.x_out;
    s.frame = a.s_out;
#pragma unroll
    for (int k = 0; k < 5; ++k) s.p[k] = a.p_out[k];
    s.lo[0] = s.lo[1] = s.lo[2] = 0.0;
#pragma unroll
    for (int k = 0; k < 15; ++k) s.C[k] = a.C_out[k];
    if (!kf_move<double>(s, b.x_in, b.s_in, geo, P.kb, P.snp_max)) return false;
    const int ix[4] = {0, 2, 3, 4};
    double r[4], M[16];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        r[u] = b.p_in[ix[u]] - (s.p[ix[u]] + (ix[u] < 3 ? s.lo[ix[u]] : 0.0));
#pragma unroll
        for (int w = 0; w < 4; ++w) M[u * 4 + w] = s.C[sx(ix[u], ix[w])] + b.C_in[sx(ix[u], ix[w])];
    }
    if (!chi2_spd4(r, M, c4)) return false;
    const double zi = s.p[1] + s.lo[1];
    zmem = 0.5 * (zi + b.p_in[1]);
    t0s = (b.p_in[1] - zi) / (2.0 * sgn_i * S.v_drift);
    return true;
}

// The joint fit of the outer segment's clusters ho[0..no) (outermost first)
// followed by the inner segment's hi[0..ni), with t0.  Seed: the
// three-cluster seed of the outer segment alone (first, middle and last of
// ho, one side, so its z is that side's apparent z'), made the true z with
// t0 = t0_seed; prior covariance diagonal, the helix prior of the
// five-parameter fit and t0_prior^2.  q, C: state and covariance at the
// innermost cluster.
TPC_HD bool fit_t0(const int32_t* ho, int no, const int32_t* hi, int ni, double t0_seed, const HitSrc& H,
                   const Geo* __restrict__ geo, const ExPrm& P, const SidesPrm& S, double q[6], double C[21],
                   double& chi2) {
    if (no < 3 || ni < 1) return false;
    KFD s;
    {
        int rows[3], secs[3];
        float ys[3], zs[3];
        const int pick[3] = {0, no / 2, no - 1};
        for (int k = 0; k < 3; ++k) {
            const int c = ho[pick[k]];
            rows[k] = H.row[c];
            secs[k] = sector_of(H, c);
            ys[k] = H.y[c];
            zs[k] = H.z[c];
        }
        kf_seed(s, rows, secs, ys, zs, true, geo, P.bz, P.seed_snp, P.seed_qpt, P.prior);
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) q[i] = s.p[i] + (i < 3 ? s.lo[i] : 0.0);
    q[1] += side_sgn(sector_of(H, ho[0])) * S.v_drift * t0_seed;
    q[5] = t0_seed;
#pragma unroll
    for (int i = 0; i < 21; ++i) C[i] = 0.0;
#pragma unroll
    for (int i = 0; i < 5; ++i) C[s6(i, i)] = (double)P.prior[i];
    C[s6(5, 5)] = S.t0_prior * S.t0_prior;
    chi2 = 0.0;
    for (int j = 0; j < no + ni; ++j) {
        const int c = j < no ? ho[j] : hi[j - no];
        const int sec = sector_of(H, c);
#pragma unroll
        for (int i = 0; i < 5; ++i) s.p[i] = q[i];
        s.lo[0] = s.lo[1] = s.lo[2] = 0.0;
        double J[25];
        if (!kf_move<double, true, false>(s, geo->row_xd[H.row[c]], sec, geo, P.kb, P.snp_max, nullptr, nullptr,
                                          J))
            return false;
#pragma unroll
        for (int i = 0; i < 5; ++i) q[i] = s.p[i] + (i < 3 ? s.lo[i] : 0.0);
        cov6_move(C, J);
        chi2 += kf6_update(q, C, (double)H.y[c], (double)H.z[c], -side_sgn(sec) * S.v_drift, P.sy2, P.sz2);
    }
    return true;
}

}  // namespace tpc
