// NEXT-3: the per-track pieces of the Kalman-filter variants (material in
// the pad-row planes, outward refit, Rauch-Tung-Striebel smoother), shared
// by the kernel in tpc_fit_ex.cu and, so that they can be checked against
// the FP64 oracle without a GPU, by host programs.  FP64 throughout.
#pragma once

#include "tpc_fit.cuh"

namespace tpc {

struct ExPrm {
    double sy2, sz2, kb, snp_max, bz, seed_snp, seed_qpt;
    double x0, eloss, mass;
    float prior[5];
    bool outward;
};

// The material of one plane.  Along the motion (undo = false) the plane
// acts after the crossing: the energy drops by eloss times the path factor
// 1/(cos phi cos lambda), mapping q/pT to w' = w p / p'; against the motion
// (undo = true) the energy is restored.  Either way the deflection of the
// plane adds its covariance, two projected angles of the Highland width
// theta0 (x/X0 = x0 times the path factor, at the momentum arriving at the
// plane): Q_ss = theta0^2 cos^2 phi (1 + t^2), Q_tt = theta0^2 (1 + t^2)^2,
// Q_tw = theta0^2 (1 + t^2) w t, Q_ww = theta0^2 w^2 t^2.  jw (optional)
// receives d w'/d t and d w'/d w.
TPC_HD void mat_step(KFD& s, const ExPrm& P, bool undo, double jw[2]) {
    const double sn = s.p[2] + s.lo[2], t = s.p[3], w = s.p[4];
    const double c2 = 1.0 - sn * sn;
    const double tt = 1.0 + t * t;
    const double path = sqrt(tt / c2);
    const double pm = sqrt(tt) / fabs(w);
    const double m2 = P.mass * P.mass;
    const double e = sqrt(pm * pm + m2);
    double p_arr = pm, e_arr = e;
    if (jw) {
        jw[0] = 0.0;
        jw[1] = 1.0;
    }
    if (P.eloss > 0.0) {
        const double de = path * P.eloss;
        const double e2 = undo ? e + de : e - de;
        const double p2 = sqrt(e2 * e2 - m2);
        const double r = e2 * pm * pm / (p2 * p2 * e);
        const double w2 = w * pm / p2;
        const double dw_dw = w2 / w * r, dw_dt = w2 * t / tt * (1.0 - r);
        // C' = J C J^T with J the identity except row 4 = (0, 0, 0, dw_dt, dw_dw)
        double row4[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) row4[i] = dw_dt * s.C[sx(3, i)] + dw_dw * s.C[sx(4, i)];
        const double c44 = dw_dt * row4[3] + dw_dw * row4[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) s.C[sx(4, i)] = row4[i];
        s.C[sx(4, 4)] = c44;
        s.p[4] = w2;
        if (undo) {
            p_arr = p2;
            e_arr = e2;
        }
        if (jw) {
            jw[0] = dw_dt;
            jw[1] = dw_dw;
        }
    }
    if (P.x0 > 0.0) {
        const double xx0 = path * P.x0;
        const double th0 = 0.0136 / ((p_arr / e_arr) * p_arr) * sqrt(xx0) * (1.0 + 0.038 * log(xx0));
        const double q = th0 * th0, wn = s.p[4];
        s.C[sx(2, 2)] += q * c2 * tt;
        s.C[sx(3, 3)] += q * tt * tt;
        s.C[sx(3, 4)] += q * tt * wn * t;
        s.C[sx(4, 4)] += q * wn * wn * t * t;
    }
}

TPC_HD void mat_mul5(const double* A, const double* B, double* out) {  // out = A B
    double tmp[25];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            double a = 0.0;
#pragma unroll
            for (int l = 0; l < 5; ++l) a += A[i * 5 + l] * B[l * 5 + k];
            tmp[i * 5 + k] = a;
        }
#pragma unroll
    for (int i = 0; i < 25; ++i) out[i] = tmp[i];
}

// Inverse of a packed SPD 5x5 by Cholesky (full, row-major); false when
// not positive definite.
TPC_HD bool spd_inv5(const double* M, double* inv) {
    double L[5][5];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) L[i][j] = 0.0;
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j <= i; ++j) {
            double v = M[sx(i, j)];
            for (int l = 0; l < j; ++l) v -= L[i][l] * L[j][l];
            if (i == j) {
                if (!(v > 0.0)) return false;
                L[i][i] = sqrt(v);
            } else {
                L[i][j] = v / L[j][j];
            }
        }
    for (int c = 0; c < 5; ++c) {
        double v[5], x[5];
        for (int i = 0; i < 5; ++i) {
            double a = i == c ? 1.0 : 0.0;
            for (int l = 0; l < i; ++l) a -= L[i][l] * v[l];
            v[i] = a / L[i][i];
        }
        for (int i = 4; i >= 0; --i) {
            double a = v[i];
            for (int l = i + 1; l < 5; ++l) a -= L[l][i] * x[l];
            x[i] = a / L[i][i];
        }
        for (int i = 0; i < 5; ++i) inv[i * 5 + c] = x[i];
    }
    return true;
}

struct HitSrc {
    const float* y;
    const float* z;
    const uint16_t* row;
    const int64_t* evt_off;
    int G;
};

TPC_HD int sector_of(const HitSrc& H, int c) { return group_of(H.evt_off, H.G, c) % NSEC; }

// One move of the filter's direction from the plane of hit a to the plane
// of hit b (planes in between of one sector crossed one by one, each with
// its material): along the motion the plane left acts first; against it
// the plane reached is undone last.  F (optional) accumulates the move's
// Jacobian (left-multiplied).
TPC_HD bool filter_move(KFD& s, const HitSrc& H, int a, int b, bool along, const ExPrm& P,
                        const Geo* __restrict__ geo, bool mat, double* F) {
    double J[25], jw[2];
    auto chain_w = [&]() {
        if (F && P.eloss > 0.0) {
            double Jm[25];
#pragma unroll
            for (int i = 0; i < 25; ++i) Jm[i] = i % 6 == 0 ? 1.0 : 0.0;
            Jm[4 * 5 + 3] = jw[0];
            Jm[4 * 5 + 4] = jw[1];
            mat_mul5(Jm, F, F);
        }
    };
    const int sa = sector_of(H, a), sb = sector_of(H, b);
    if (mat && along) {
        mat_step(s, P, false, F ? jw : nullptr);
        chain_w();
    }
    if (mat && sa == sb) {
        const int r0 = H.row[a], r1 = H.row[b], stp = r1 > r0 ? 1 : -1;
        for (int r = r0 + stp; r != r1; r += stp) {
            if (!kf_move<double>(s, geo->row_xd[r], sb, geo, P.kb, P.snp_max, nullptr, nullptr, F ? J : nullptr))
                return false;
            if (F) mat_mul5(J, F, F);
            mat_step(s, P, !along, F ? jw : nullptr);
            chain_w();
        }
    }
    if (!kf_move<double>(s, geo->row_xd[H.row[b]], sb, geo, P.kb, P.snp_max, nullptr, nullptr, F ? J : nullptr))
        return false;
    if (F) mat_mul5(J, F, F);
    if (mat && !along) {
        mat_step(s, P, true, F ? jw : nullptr);
        chain_w();
    }
    return true;
}

// The fit of one track in FP64, inward (list order, state at the innermost
// cluster) or outward (reversed, state at the outermost); with `filt`, the
// filtered state and covariance after each update are written to
// filt[20 j ...] (list position j).
TPC_HD bool fit_ex(const int32_t* h, int n, const HitSrc& H, const Geo* __restrict__ geo, const ExPrm& P,
                   KFD& s, double& chi2, double* filt) {
    if (n < 3) return false;
    const bool mat = P.x0 > 0.0 || P.eloss > 0.0;
    auto hit = [&](int j) { return P.outward ? h[n - 1 - j] : h[j]; };
    int rows[3], secs[3];
    float ys[3], zs[3];
    const int pick[3] = {0, n / 2, n - 1};
    for (int k = 0; k < 3; ++k) {
        const int c = hit(pick[k]);
        rows[k] = H.row[c];
        secs[k] = sector_of(H, c);
        ys[k] = H.y[c];
        zs[k] = H.z[c];
    }
    kf_seed(s, rows, secs, ys, zs, !P.outward, geo, P.bz, P.seed_snp, P.seed_qpt, P.prior);
    chi2 = 0.0;
    for (int j = 0; j < n; ++j) {
        const int c = hit(j);
        if (j == 0) {
            if (!kf_move<double>(s, geo->row_xd[H.row[c]], sector_of(H, c), geo, P.kb, P.snp_max)) return false;
        } else if (!filter_move(s, H, hit(j - 1), c, P.outward, P, geo, mat, nullptr)) {
            return false;
        }
        chi2 += kf_update_d(s, (double)H.y[c], (double)H.z[c], P.sy2, P.sz2);
        if (filt) {
            double* o = filt + (size_t)20 * j;
            for (int i = 0; i < 3; ++i) o[i] = s.p[i] + s.lo[i];
            o[3] = s.p[3];
            o[4] = s.p[4];
            for (int i = 0; i < 15; ++i) o[5 + i] = s.C[i];
        }
    }
    return true;
}

// Rauch-Tung-Striebel, back from the innermost hit over the stored filtered
// states of an inward fit (overwritten by the smoothed ones): gain
// A = C_f F^T C_p^-1 with F the Jacobian of the prediction from hit j to
// j + 1 and C_p its covariance; covariance C_f + A (C_s - C_p) A^T; state
// x_b + (I - A F) (x_f - x_b), x_b the smoothed state of hit j + 1 moved back
// to hit j along the motion (the textbook x_f + A (x_s - f(x_f)) for a
// linear move, exact for a move without material).
TPC_HD bool smooth_back(const int32_t* h, int n, const HitSrc& H, const Geo* __restrict__ geo,
                        const ExPrm& P, double* st) {
    const bool mat = P.x0 > 0.0 || P.eloss > 0.0;
    for (int j = n - 2; j >= 0; --j) {
        const double* f = st + (size_t)20 * j;
        double* sn = st + (size_t)20 * (j + 1);
        // prediction from the filtered state at j to the plane of j + 1
        KFD q;
        q.x = geo->row_xd[H.row[h[j]]];
        q.frame = sector_of(H, h[j]);
        for (int i = 0; i < 5; ++i) q.p[i] = f[i];
        q.lo[0] = q.lo[1] = q.lo[2] = 0.0;
        for (int i = 0; i < 15; ++i) q.C[i] = f[5 + i];
        double F[25];
        for (int i = 0; i < 25; ++i) F[i] = i % 6 == 0 ? 1.0 : 0.0;
        if (!filter_move(q, H, h[j], h[j + 1], false, P, geo, mat, F)) return false;
        double Pinv[25];
        if (!spd_inv5(q.C, Pinv)) return false;
        double CfFt[25], A[25], AF[25];
        for (int i = 0; i < 5; ++i)
            for (int k = 0; k < 5; ++k) {
                double a = 0.0;
                for (int l = 0; l < 5; ++l) a += f[5 + sx(i, l)] * F[k * 5 + l];
                CfFt[i * 5 + k] = a;
            }
        mat_mul5(CfFt, Pinv, A);
        mat_mul5(A, F, AF);
        // the smoothed state of j + 1 moved back to j along the motion
        KFD b;
        b.x = geo->row_xd[H.row[h[j + 1]]];
        b.frame = sector_of(H, h[j + 1]);
        for (int i = 0; i < 5; ++i) b.p[i] = sn[i];
        b.lo[0] = b.lo[1] = b.lo[2] = 0.0;
        for (int i = 0; i < 15; ++i) b.C[i] = 0.0;
        if (!filter_move(b, H, h[j + 1], h[j], true, P, geo, mat, nullptr)) return false;
        double xb[5], xn[5], D[25], AD[25], Cn[15];
        for (int i = 0; i < 5; ++i) xb[i] = b.p[i] + (i < 3 ? b.lo[i] : 0.0);
        for (int i = 0; i < 5; ++i) {
            double a = xb[i];
            for (int l = 0; l < 5; ++l) a += ((i == l ? 1.0 : 0.0) - AF[i * 5 + l]) * (f[l] - xb[l]);
            xn[i] = a;
        }
        for (int i = 0; i < 5; ++i)
            for (int k = 0; k < 5; ++k) D[i * 5 + k] = sn[5 + sx(i, k)] - q.C[sx(i, k)];
        mat_mul5(A, D, AD);
        for (int i = 0; i < 5; ++i)
            for (int k = i; k < 5; ++k) {
                double a = f[5 + sx(i, k)];
                for (int l = 0; l < 5; ++l) a += AD[i * 5 + l] * A[k * 5 + l];
                Cn[sx(i, k)] = a;
            }
        double* o = st + (size_t)20 * j;
        for (int i = 0; i < 5; ++i) o[i] = xn[i];
        for (int i = 0; i < 15; ++i) o[5 + i] = Cn[i];
    }
    return true;
}

}  // namespace tpc
