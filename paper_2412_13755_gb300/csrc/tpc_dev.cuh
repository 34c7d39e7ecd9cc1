// Device building blocks: status word, geometry lookups, and the FP32
// Kalman-filter pieces (helix transport with frame rotation, 2-d update with
// FP64 fallback, three-point seed).  Used by the find, fit and adjoint
// kernels.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "tpc_ff.cuh"
#include "tpc_internal.h"

namespace tpc {

constexpr double KAPPA = 2.99792458e-3;  // cm^-1 T^-1 (GeV/c)

__device__ __forceinline__ void set_status(int32_t* st, int code, int detail) {
    if (atomicCAS(&st[ST_STATUS], 0, code) == 0) atomicExch(&st[ST_DETAIL], detail);
}

// The loaded batch failed validation (rows, offsets, finite coordinates).
// Every kernel that reads clusters or their offsets returns early on such
// a batch, so that nothing is indexed from invalid input.  The flag is its
// own slot: the status word keeps the first error of a context, which may
// predate the load.
__device__ __forceinline__ bool input_rejected(const int32_t* st) {
    return *reinterpret_cast<const volatile int32_t*>(&st[ST_INPUT_BAD]) != 0;
}
__device__ __forceinline__ void reject_input(int32_t* st, int detail) {
    set_status(st, TPC_ERR_INPUT, detail);
    atomicExch(&st[ST_INPUT_BAD], 1);
}

// largest g with off[g] <= i (off non-decreasing, off[0] = 0)
TPC_HD int group_of(const int64_t* __restrict__ off, int G, int64_t i) {
    int lo = 0, hi = G;  // answer in [lo, hi)
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
#if defined(__CUDA_ARCH__)
        const int64_t o = __ldg(off + mid);
#else
        const int64_t o = off[mid];
#endif
        if (o <= i) lo = mid; else hi = mid;
    }
    return lo;
}

TPC_HD float t_sqrt(float v) { return sqrtf(v); }
TPC_HD double t_sqrt(double v) { return sqrt(v); }
TPC_HD float t_asin(float v) { return asinf(v); }
TPC_HD double t_asin(double v) { return asin(v); }
TPC_HD float t_abs(float v) { return fabsf(v); }
TPC_HD double t_abs(double v) { return fabs(v); }

template <class R>
struct KFT {
    double x;     // plane position in the current frame (cm)
    int frame;    // sector of the current frame
    R p[5];       // y, z, sin phi, tan lambda, q/pT
    R lo[3];      // compensation terms of y, z, sin phi (p[i] + lo[i] is the value)
    R C[15];      // packed covariance
};

// hi + lo += d, exactly up to the final rounding of lo (TwoSum); the pair
// is renormalised so that |lo| stays below half an ulp of hi.
template <class R>
TPC_HD void add_comp(R& hi, R& lo, R d) {
    const R s = hi + d;
    const R bp = s - hi;
    const R err = (hi - (s - bp)) + (d - bp);
    const R t = lo + err;
    hi = s + t;
    lo = t - (hi - s);
}
using KF = KFT<float>;
using KFD = KFT<double>;

// Covariance transform C <- J C J^T for the Jacobian structure of a
// transport (+ rotation):
//   J = [[j00, 0, j02, 0,   j04],
//        [j10, 1, j12, j13, j14],
//        [j20, 0, j22, 0,   j24],
//        [0,   0, 0,   1,   0  ],
//        [0,   0, 0,   0,   1  ]]
template <class R>
TPC_HD void cov_jct(R C[15], R j00, R j02, R j04, R j10, R j12, R j13, R j14, R j20, R j22,
                    R j24) {
    R c[5][5];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) c[i][j] = C[sx(i, j)];
    R A0[5], A1[5], A2[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        A0[j] = j00 * c[0][j] + j02 * c[2][j] + j04 * c[4][j];
        A1[j] = j10 * c[0][j] + c[1][j] + j12 * c[2][j] + j13 * c[3][j] + j14 * c[4][j];
        A2[j] = j20 * c[0][j] + j22 * c[2][j] + j24 * c[4][j];
    }
    C[sx(0, 0)] = A0[0] * j00 + A0[2] * j02 + A0[4] * j04;
    C[sx(0, 1)] = A0[0] * j10 + A0[1] + A0[2] * j12 + A0[3] * j13 + A0[4] * j14;
    C[sx(0, 2)] = A0[0] * j20 + A0[2] * j22 + A0[4] * j24;
    C[sx(0, 3)] = A0[3];
    C[sx(0, 4)] = A0[4];
    C[sx(1, 1)] = A1[0] * j10 + A1[1] + A1[2] * j12 + A1[3] * j13 + A1[4] * j14;
    C[sx(1, 2)] = A1[0] * j20 + A1[2] * j22 + A1[4] * j24;
    C[sx(1, 3)] = A1[3];
    C[sx(1, 4)] = A1[4];
    C[sx(2, 2)] = A2[0] * j20 + A2[2] * j22 + A2[4] * j24;
    C[sx(2, 3)] = A2[3];
    C[sx(2, 4)] = A2[4];
}

// What an FP64 redo of a cancelling update needs from the preceding move:
// the Jacobian entries and the covariance before the transport.
struct MoveJ {
    float j00, j02, j04, j10, j12, j13, j14, j20, j22, j24;
    float Cpre[15];
    bool valid;
};

// Move the state to plane x_to of sector `to`: rotate the frame on a sector
// change (x' = x cos da + y sin da, y' = -x sin da + y cos da,
// phi' = phi - da), then transport along the helix (uniform Bz, no
// material):
//   s2 = s1 - k dx, y2 = y1 + dx (s1+s2)/(c1+c2),
//   z2 = z1 + t arc sign(dx), arc = chord * asin(u)/u, u = |k| chord / 2.
// The covariance follows with the analytic Jacobian of the composition.
// Returns false (state untouched or partially moved) when |sin phi| would
// reach snp_max.  CanRotate = false is the move between row planes of one
// frame by the caller's step *dx_same_frame (required): no rotation code, no
// FP64 plane arithmetic, and s.x is left to the caller.  MoveCov = false
// leaves s.C alone (for a caller that transforms its own covariance with the
// Jacobian returned in mj).
// jfull (optional) receives the full Jacobian of the move, row-major 5x5.
template <class R, bool CanRotate = true, bool MoveCov = true>
TPC_HD bool kf_move(KFT<R>& s, double x_to, int to, const Geo* __restrict__ geo, R kb, R snp_max,
                    MoveJ* mj = nullptr, const R* dx_same_frame = nullptr, R* jfull = nullptr) {
    double xs = CanRotate ? s.x : 0.0;
    R ys = s.p[0], ss = s.p[2];
    R ys_lo = s.lo[0], ss_lo = s.lo[2];
    R ca = R(1), sa = R(0), dsn = R(1);
    const bool rot = CanRotate && to != s.frame;
    if (rot) {
        const int k = ((to % NPHI) - (s.frame % NPHI) + NPHI) % NPHI;
        const double cad = geo->da_cos[k], sad = geo->da_sin[k];
        if (t_abs(ss) >= snp_max) return false;
        const R c = t_sqrt(R(1) - ss * ss);
        const double y0 = (double)s.p[0] + (double)s.lo[0];
        const double xn = s.x * cad + y0 * sad;
        const double yn = y0 * cad - s.x * sad;
        ca = (R)cad;
        sa = (R)sad;
        const R sn = ss * ca - c * sa;
        if (t_abs(sn) >= snp_max) return false;
        dsn = ca + ss * sa / c;
        xs = xn;
        ys = (R)yn;
        ys_lo = (R)(yn - (double)ys);
        ss = sn;
        ss_lo = R(0);
    }
    // dx_same_frame: the caller's exact step between row planes of one frame
    const R dx = (!rot && dx_same_frame) ? *dx_same_frame : (R)(x_to - xs);
    const R t = s.p[3], w = s.p[4];
    const R k = w * kb;
    const R s1 = ss;
    const R s2 = s1 - k * dx;
    if (t_abs(s2) >= snp_max) return false;
    const R c1 = t_sqrt(R(1) - s1 * s1);
    const R c2 = t_sqrt(R(1) - s2 * s2);
    const R B = c1 + c2;
    const R tn = (s1 + s2) / B;
    const R sg = dx >= R(0) ? R(1) : R(-1);
    const R adx = t_abs(dx);
    const R h = t_sqrt(R(1) + tn * tn);
    const R L = adx * h;
    const R v = k * k * L * L * R(0.25);  // u^2
    const R e = R(1) / t_sqrt(R(1) - v);
    R g, m;  // asin(u)/u and (e - g)/v
    if (v < R(1e-2)) {
        g = R(1) + v * (R(1.0 / 6.0) + v * (R(3.0 / 40.0) + v * (R(5.0 / 112.0) + v * R(35.0 / 1152.0))));
        m = R(1.0 / 3.0) + v * (R(0.3) + v * (R(15.0 / 56.0) + v * R(35.0 / 144.0)));
    } else {
        const R u = t_sqrt(v);
        g = t_asin(u) / u;
        m = (e - g) / v;
    }
    const R arc = L * g;
    const R dtn_s1p = (R(1) + tn * s1 / c1) / B;
    const R dtn_s2p = (R(1) + tn * s2 / c2) / B;
    const R ds2_w = -kb * dx;
    const R dtn_s1 = dtn_s1p + dtn_s2p;
    const R dtn_w = dtn_s2p * ds2_w;
    const R dtn_dx = -dtn_s2p * k;
    const R dy_s1 = dx * dtn_s1;
    const R dy_w = dx * dtn_w;
    const R dy_dx = tn + dx * dtn_dx;
    const R dL_tn = adx * tn / h;
    const R darc_k = k * L * L * L * m * R(0.25);
    const R tsg = t * sg;
    const R dz_s1 = tsg * e * dL_tn * dtn_s1;
    const R dz_w = tsg * (e * dL_tn * dtn_w + darc_k * kb);
    const R dz_t = arc * sg;
    R j00 = R(1), j10 = R(0), j20 = R(0), j02 = dy_s1, j12 = dz_s1, j22 = R(1);
    if (rot) {
        const R dz_dx = tsg * e * (h * sg + dL_tn * dtn_dx);
        j00 = ca - dy_dx * sa;
        j10 = -dz_dx * sa;
        j20 = k * sa;
        j02 = dy_s1 * dsn;
        j12 = dz_s1 * dsn;
        j22 = dsn;
    }
    if (mj) {
        mj->j00 = (float)j00; mj->j02 = (float)j02; mj->j04 = (float)dy_w; mj->j10 = (float)j10;
        mj->j12 = (float)j12; mj->j13 = (float)dz_t; mj->j14 = (float)dz_w; mj->j20 = (float)j20;
        mj->j22 = (float)j22; mj->j24 = (float)ds2_w;
#pragma unroll
        for (int i = 0; i < 15; ++i) mj->Cpre[i] = (float)s.C[i];
        mj->valid = true;
    }
    if (jfull) {
        const R J[25] = {j00, R(0), j02, R(0), dy_w,  j10, R(1), j12, dz_t, dz_w,  j20, R(0), j22, R(0), ds2_w,
                         R(0), R(0), R(0), R(1), R(0),  R(0), R(0), R(0), R(0), R(1)};
#pragma unroll
        for (int i = 0; i < 25; ++i) jfull[i] = J[i];
    }
    if (MoveCov) cov_jct<R>(s.C, j00, j02, dy_w, j10, j12, dz_t, dz_w, j20, j22, ds2_w);
    add_comp(ys, ys_lo, dx * tn);
    s.p[0] = ys;
    s.lo[0] = ys_lo;
    add_comp(s.p[1], s.lo[1], tsg * arc);
    add_comp(ss, ss_lo, -k * dx);
    s.p[2] = ss;
    s.lo[2] = ss_lo;
    if (CanRotate) {
        s.x = x_to;
        s.frame = to;
    }
    return true;
}

// The update with the covariance step in FP64: the transport J C J^T of
// the preceding move (when mj carries it) and the update itself, the state
// increment applied in FP64 to the compensated state.  Returns the
// predicted-residual chi2 term.
TPC_HD float kf_update_cov_d(KF& s, float my, float mz, float sy2, float sz2, const MoveJ* mj) {
    double Cd[15];
    if (mj && mj->valid) {
#pragma unroll
        for (int i = 0; i < 15; ++i) Cd[i] = mj->Cpre[i];
        cov_jct<double>(Cd, mj->j00, mj->j02, mj->j04, mj->j10, mj->j12, mj->j13, mj->j14, mj->j20,
                        mj->j22, mj->j24);
    } else {
#pragma unroll
        for (int i = 0; i < 15; ++i) Cd[i] = s.C[i];
    }
    const double dr0 = (double)my - ((double)s.p[0] + (double)s.lo[0]);
    const double dr1 = (double)mz - ((double)s.p[1] + (double)s.lo[1]);
    const double D00 = Cd[0] + (double)sy2, D01 = Cd[1], D11 = Cd[5] + (double)sz2;
    const double ddet = D00 * D11 - D01 * D01;
    const double e00 = D11 / ddet, e01 = -D01 / ddet, e11 = D00 / ddet;
    double c0[5], c1[5], k0[5], k1[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        c0[i] = Cd[sx(0, i)];
        c1[i] = Cd[sx(1, i)];
        k0[i] = c0[i] * e00 + c1[i] * e01;
        k1[i] = c0[i] * e01 + c1[i] * e11;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double v = (double)s.p[i] + (double)s.lo[i] + k0[i] * dr0 + k1[i] * dr1;
        s.p[i] = (float)v;
        s.lo[i] = (float)(v - (double)s.p[i]);
    }
#pragma unroll
    for (int i = 3; i < 5; ++i) s.p[i] = (float)((double)s.p[i] + k0[i] * dr0 + k1[i] * dr1);
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = i; j < 5; ++j)
            s.C[sx(i, j)] = (float)(Cd[sx(i, j)] - (k0[i] * c0[j] + k1[i] * c1[j]));
    return (float)(dr0 * dr0 * e00 + 2.0 * dr0 * dr1 * e01 + dr1 * dr1 * e11);
}

// Update with a covariance carried in FP64 across the whole fit (Cd, the
// covariance of the FP32 state s): FP64 gain and covariance step, the state
// increment applied in FP64 to the compensated state.  Returns the
// predicted-residual chi2 term.
TPC_HD double kf_update_dcov(KF& s, double Cd[15], float my, float mz, double sy2, double sz2) {
    const double dr0 = (double)my - ((double)s.p[0] + (double)s.lo[0]);
    const double dr1 = (double)mz - ((double)s.p[1] + (double)s.lo[1]);
    const double D00 = Cd[0] + sy2, D01 = Cd[1], D11 = Cd[5] + sz2;
    const double idet = 1.0 / (D00 * D11 - D01 * D01);
    const double e00 = D11 * idet, e01 = -D01 * idet, e11 = D00 * idet;
    double c0[5], c1[5], k0[5], k1[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        c0[i] = Cd[sx(0, i)];
        c1[i] = Cd[sx(1, i)];
        k0[i] = c0[i] * e00 + c1[i] * e01;
        k1[i] = c0[i] * e01 + c1[i] * e11;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double v = (double)s.p[i] + (double)s.lo[i] + k0[i] * dr0 + k1[i] * dr1;
        s.p[i] = (float)v;
        s.lo[i] = (float)(v - (double)s.p[i]);
    }
#pragma unroll
    for (int i = 3; i < 5; ++i) s.p[i] = (float)((double)s.p[i] + k0[i] * dr0 + k1[i] * dr1);
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = i; j < 5; ++j) Cd[sx(i, j)] -= k0[i] * c0[j] + k1[i] * c1[j];
    return dr0 * dr0 * e00 + 2.0 * dr0 * dr1 * e01 + dr1 * dr1 * e11;
}

// Covariance transform C <- J C J^T in float-float for the Jacobian of
// cov_jct (J exact in FP32).
TPC_HD void cov_jct_ff(ff C[15], float j00, float j02, float j04, float j10, float j12, float j13,
                       float j14, float j20, float j22, float j24) {
    ff c[5][5];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) c[i][j] = C[sx(i, j)];
    ff A0[5], A1[5], A2[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        A0[j] = ff_fma_f(ff_fma_f(ff_mul_f(c[0][j], j00), c[2][j], j02), c[4][j], j04);
        A1[j] = ff_fma_f(ff_fma_f(ff_fma_f(ff_fma_f(c[1][j], c[0][j], j10), c[2][j], j12), c[3][j], j13),
                         c[4][j], j14);
        A2[j] = ff_fma_f(ff_fma_f(ff_mul_f(c[0][j], j20), c[2][j], j22), c[4][j], j24);
    }
    C[sx(0, 0)] = ff_fma_f(ff_fma_f(ff_mul_f(A0[0], j00), A0[2], j02), A0[4], j04);
    C[sx(0, 1)] = ff_fma_f(ff_fma_f(ff_fma_f(ff_fma_f(A0[1], A0[0], j10), A0[2], j12), A0[3], j13), A0[4], j14);
    C[sx(0, 2)] = ff_fma_f(ff_fma_f(ff_mul_f(A0[0], j20), A0[2], j22), A0[4], j24);
    C[sx(0, 3)] = A0[3];
    C[sx(0, 4)] = A0[4];
    C[sx(1, 1)] = ff_fma_f(ff_fma_f(ff_fma_f(ff_fma_f(A1[1], A1[0], j10), A1[2], j12), A1[3], j13), A1[4], j14);
    C[sx(1, 2)] = ff_fma_f(ff_fma_f(ff_mul_f(A1[0], j20), A1[2], j22), A1[4], j24);
    C[sx(1, 3)] = A1[3];
    C[sx(1, 4)] = A1[4];
    C[sx(2, 2)] = ff_fma_f(ff_fma_f(ff_mul_f(A2[0], j20), A2[2], j22), A2[4], j24);
    C[sx(2, 3)] = A2[3];
    C[sx(2, 4)] = A2[4];
}

// The same transform for a move inside one frame, where J = I except for
// j02, j04, j12, j13, j14, j24 (j00 = j22 = 1, j10 = j20 = 0): the products
// with the unit and zero entries are skipped.
TPC_HD void cov_jct_ff_frame(ff C[15], float j02, float j04, float j12, float j13, float j14,
                             float j24) {
    ff c[5][5];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) c[i][j] = C[sx(i, j)];
    ff A0[5], A1[5], A2[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        A0[j] = ff_fma_f(ff_fma_f(c[0][j], c[2][j], j02), c[4][j], j04);
        A1[j] = ff_fma_f(ff_fma_f(ff_fma_f(c[1][j], c[2][j], j12), c[3][j], j13), c[4][j], j14);
        A2[j] = ff_fma_f(c[2][j], c[4][j], j24);
    }
    C[sx(0, 0)] = ff_fma_f(ff_fma_f(A0[0], A0[2], j02), A0[4], j04);
    C[sx(0, 1)] = ff_fma_f(ff_fma_f(ff_fma_f(A0[1], A0[2], j12), A0[3], j13), A0[4], j14);
    C[sx(0, 2)] = ff_fma_f(A0[2], A0[4], j24);
    C[sx(0, 3)] = A0[3];
    C[sx(0, 4)] = A0[4];
    C[sx(1, 1)] = ff_fma_f(ff_fma_f(ff_fma_f(A1[1], A1[2], j12), A1[3], j13), A1[4], j14);
    C[sx(1, 2)] = ff_fma_f(A1[2], A1[4], j24);
    C[sx(1, 3)] = A1[3];
    C[sx(1, 4)] = A1[4];
    C[sx(2, 2)] = ff_fma_f(A2[2], A2[4], j24);
    C[sx(2, 3)] = A2[3];
    C[sx(2, 4)] = A2[4];
}

// Kalman update with the covariance in float-float: S, its inverse, the
// gain and C - K H C in float-float; the state increment from the gain in
// FP32 on the compensated state.  Returns the predicted-residual chi2 term.
TPC_HD float kf_update_ff(KF& s, ff C[15], float my, float mz, float sy2, float sz2) {
    const float r0 = (my - s.p[0]) - s.lo[0], r1 = (mz - s.p[1]) - s.lo[1];
    const ff S00 = ff_add(C[0], ff_from(sy2)), S01 = C[1], S11 = ff_add(C[5], ff_from(sz2));
    const ff det = ff_add(ff_mul(S00, S11), ff_neg(ff_mul(S01, S01)));
    const ff idet = ff_rcp(det);
    const ff i00 = ff_mul(S11, idet), i01 = ff_neg(ff_mul(S01, idet)), i11 = ff_mul(S00, idet);
    ff C0[5], C1[5], K0[5], K1[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        C0[i] = C[sx(0, i)];
        C1[i] = C[sx(1, i)];
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        K0[i] = ff_dot2(C0[i], i00, C1[i], i01);
        K1[i] = ff_dot2(C0[i], i01, C1[i], i11);
    }
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = i; j < 5; ++j)
            C[sx(i, j)] = ff_add(C[sx(i, j)], ff_neg(ff_dot2(K0[i], C0[j], K1[i], C1[j])));
#pragma unroll
    for (int i = 0; i < 3; ++i) add_comp(s.p[i], s.lo[i], K0[i].hi * r0 + K1[i].hi * r1);
#pragma unroll
    for (int i = 3; i < 5; ++i) s.p[i] += K0[i].hi * r0 + K1[i].hi * r1;
    return r0 * r0 * i00.hi + 2.f * r0 * r1 * i01.hi + r1 * r1 * i11.hi;
}

// Kalman update with cluster (my, mz): S = C_yz + R, K = C H^T S^-1,
// p += K r, C -= K H C (upper triangle), returns the predicted-residual chi2
// term r^T S^-1 r.  When the update cancels (a posterior variance below
// fp64_ratio x its prior, or det S <= fp64_det S00 S11) the covariance step
// is redone in FP64 -- the transport J C J^T of the preceding move (when mj
// carries it) and the update -- and counted.
TPC_HD float kf_update(KF& s, float my, float mz, float sy2, float sz2, float fp64_ratio,
                       float fp64_det, int* n_fp64, const MoveJ* mj = nullptr) {
    const float r0 = (my - s.p[0]) - s.lo[0], r1 = (mz - s.p[1]) - s.lo[1];
    const float S00 = s.C[0] + sy2, S01 = s.C[1], S11 = s.C[5] + sz2;
    const float det = S00 * S11 - S01 * S01;
    const float i00 = S11 / det, i01 = -S01 / det, i11 = S00 / det;
    float C0[5], C1[5], K0[5], K1[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        C0[i] = s.C[sx(0, i)];
        C1[i] = s.C[sx(1, i)];
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        K0[i] = C0[i] * i00 + C1[i] * i01;
        K1[i] = C0[i] * i01 + C1[i] * i11;
    }
    float Cn[15];
    bool cancel = !(det > fp64_det * S00 * S11);
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = i; j < 5; ++j) Cn[sx(i, j)] = s.C[sx(i, j)] - (K0[i] * C0[j] + K1[i] * C1[j]);
#pragma unroll
    for (int i = 0; i < 5; ++i) cancel |= !(Cn[sx(i, i)] >= fp64_ratio * s.C[sx(i, i)]);
    if (!cancel) {
#pragma unroll
        for (int i = 0; i < 3; ++i) add_comp(s.p[i], s.lo[i], K0[i] * r0 + K1[i] * r1);
#pragma unroll
        for (int i = 3; i < 5; ++i) s.p[i] += K0[i] * r0 + K1[i] * r1;
#pragma unroll
        for (int i = 0; i < 15; ++i) s.C[i] = Cn[i];
        return r0 * r0 * i00 + 2.f * r0 * r1 * i01 + r1 * r1 * i11;
    }
    // FP64 redo of the covariance step
#if defined(__CUDA_ARCH__)
    if (n_fp64) atomicAdd(n_fp64, 1);
#else
    if (n_fp64) ++*n_fp64;
#endif
    return kf_update_cov_d(s, my, mz, sy2, sz2, mj);
}

// Plain FP64 update (used when a whole track is refit in FP64).
TPC_HD double kf_update_d(KFD& s, double my, double mz, double sy2, double sz2) {
    const double r0 = my - (s.p[0] + s.lo[0]), r1 = mz - (s.p[1] + s.lo[1]);
    const double S00 = s.C[0] + sy2, S01 = s.C[1], S11 = s.C[5] + sz2;
    const double idet = 1.0 / (S00 * S11 - S01 * S01);
    const double i00 = S11 * idet, i01 = -S01 * idet, i11 = S00 * idet;
    double C0[5], C1[5], K0[5], K1[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        C0[i] = s.C[sx(0, i)];
        C1[i] = s.C[sx(1, i)];
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        K0[i] = C0[i] * i00 + C1[i] * i01;
        K1[i] = C0[i] * i01 + C1[i] * i11;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) add_comp(s.p[i], s.lo[i], K0[i] * r0 + K1[i] * r1);
#pragma unroll
    for (int i = 3; i < 5; ++i) s.p[i] += K0[i] * r0 + K1[i] * r1;
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = i; j < 5; ++j) s.C[sx(i, j)] -= K0[i] * C0[j] + K1[i] * C1[j];
    return r0 * r0 * i00 + 2.0 * r0 * r1 * i01 + r1 * r1 * i11;
}

// Neumaier-compensated FP32 accumulation.
struct NSum {
    float s = 0.f, c = 0.f;
    TPC_HD void add(float v) {
        const float t = s + v;
        if (fabsf(s) >= fabsf(v)) c += (s - t) + v; else c += (v - t) + s;
        s = t;
    }
    TPC_HD float value() const { return s + c; }
};

// Three-point seed (FP64): circle through the innermost, middle and
// outermost clusters of the list (nominal planes, uncorrected coordinates)
// in the frame of the first cluster in fit order gives q/pT and sin phi at
// that cluster; tan lambda = dz / arc between the end clusters; (y, z) of the
// first cluster.  Clamped to |sin phi| <= snp_max_seed, |q/pT| <= qpt_max.
template <class R>
TPC_HD void kf_seed(KFT<R>& s, const int rows[3], const int secs[3], const float ys[3],
                    const float zs[3], bool first_is_outer, const Geo* __restrict__ geo, double bz,
                    double snp_max_seed, double qpt_max, const float prior[5]) {
    const int fr = secs[0];
    double px[3], py[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double x = geo->row_xd[rows[i]], y = (double)ys[i];
        if (secs[i] == fr) {
            px[i] = x;
            py[i] = y;
        } else {
            const int k = ((fr % NPHI) - (secs[i] % NPHI) + NPHI) % NPHI;  // rotation secs[i] -> fr
            const double cd = geo->da_cos[k], sd = geo->da_sin[k];
            px[i] = x * cd + y * sd;
            py[i] = -x * sd + y * cd;
        }
    }
    const int i0 = first_is_outer ? 2 : 0, i2 = first_is_outer ? 0 : 2;
    const double ax = px[1] - px[i0], ay = py[1] - py[i0];
    const double bx = px[i2] - px[1], by = py[i2] - py[1];
    const double cx = px[i2] - px[i0], cy = py[i2] - py[i0];
    const double la = sqrt(ax * ax + ay * ay), lb = sqrt(bx * bx + by * by);
    const double L = sqrt(cx * cx + cy * cy);
    const double cross = ax * by - ay * bx;
    double k = 0.0;
    if (la > 0 && lb > 0 && L > 0) k = -2.0 * cross / (la * lb * L);
    double hk = fmin(0.999, fmax(-0.999, k * L * 0.5));
    const double theta = atan2(cy, cx);
    const double half = asin(hk);
    const double phi = first_is_outer ? theta - half : theta + half;
    const double sn = fmin(snp_max_seed, fmax(-snp_max_seed, sin(phi)));
    const double au = fabs(hk);
    const double arc = (au < 1e-9 || k == 0.0) ? L : 2.0 * asin(au) / fabs(k);
    const double t = arc > 0 ? ((double)zs[i2] - (double)zs[i0]) / arc : 0.0;
    double w = bz != 0.0 ? k / (KAPPA * bz) : 0.0;
    w = fmin(qpt_max, fmax(-qpt_max, w));
    s.x = geo->row_xd[rows[0]];
    s.frame = fr;
    s.p[0] = ys[0];
    s.p[1] = zs[0];
    s.p[2] = (R)sn;
    s.p[3] = (R)t;
    s.p[4] = (R)w;
    s.lo[0] = s.lo[1] = s.lo[2] = R(0);
#pragma unroll
    for (int i = 0; i < 15; ++i) s.C[i] = R(0);
    s.C[sx(0, 0)] = prior[0];
    s.C[sx(1, 1)] = prior[1];
    s.C[sx(2, 2)] = prior[2];
    s.C[sx(3, 3)] = prior[3];
    s.C[sx(4, 4)] = prior[4];
}

// The same three-point seed in FP32 for clusters of one frame, with x of
// the planes in FP32: sin phi at the first cluster is expanded as
// sin(theta -/+ h) = sin theta cos h -/+ cos theta sin h, with
// sin theta = cy/L, cos theta = cx/L, sin h = hk, cos h = sqrt(1 - hk^2), so
// only the arc length needs an inverse sine.  The seed only sets the
// linearisation point and the prior centre of the fit.
__device__ __forceinline__ void kf_seed_f(KF& s, const int rows[3], int frame, const float ys[3],
                                          const float zs[3], bool first_is_outer,
                                          const Geo* __restrict__ geo, float kb_unit,
                                          float snp_max_seed, float qpt_max, const float prior[5]) {
    // points in increasing x (selects, not indices: the arrays stay in registers)
    const int r0 = first_is_outer ? rows[2] : rows[0], r2 = first_is_outer ? rows[0] : rows[2];
    const float y0 = first_is_outer ? ys[2] : ys[0], y2 = first_is_outer ? ys[0] : ys[2];
    const float z0 = first_is_outer ? zs[2] : zs[0], z2 = first_is_outer ? zs[0] : zs[2];
    const float x0 = geo->row_xf[r0], x1 = geo->row_xf[rows[1]], x2 = geo->row_xf[r2];
    const float ax = x1 - x0, ay = ys[1] - y0;
    const float bx = x2 - x1, by = y2 - ys[1];
    const float cx = x2 - x0, cy = y2 - y0;
    const float la = sqrtf(ax * ax + ay * ay), lb = sqrtf(bx * bx + by * by);
    const float L = sqrtf(cx * cx + cy * cy);
    const float cross = ax * by - ay * bx;
    float k = 0.f;
    if (la > 0.f && lb > 0.f && L > 0.f) k = -2.f * cross / (la * lb * L);
    const float hk = fminf(0.999f, fmaxf(-0.999f, k * L * 0.5f));
    float sn = 0.f;
    if (L > 0.f) {
        const float st = cy / L, ct = cx / L, ch = sqrtf(1.f - hk * hk);
        sn = first_is_outer ? st * ch - ct * hk : st * ch + ct * hk;
    }
    sn = fminf(snp_max_seed, fmaxf(-snp_max_seed, sn));
    const float au = fabsf(hk);
    const float arc = (au < 1e-9f || k == 0.f) ? L : 2.f * asinf(au) / fabsf(k);
    const float t = arc > 0.f ? (z2 - z0) / arc : 0.f;
    float w = kb_unit != 0.f ? k / kb_unit : 0.f;
    w = fminf(qpt_max, fmaxf(-qpt_max, w));
    s.x = geo->row_xd[rows[0]];
    s.frame = frame;
    s.p[0] = ys[0];
    s.p[1] = zs[0];
    s.p[2] = sn;
    s.p[3] = t;
    s.p[4] = w;
    s.lo[0] = s.lo[1] = s.lo[2] = 0.f;
#pragma unroll
    for (int i = 0; i < 15; ++i) s.C[i] = 0.f;
    s.C[sx(0, 0)] = prior[0];
    s.C[sx(1, 1)] = prior[1];
    s.C[sx(2, 2)] = prior[2];
    s.C[sx(3, 3)] = prior[3];
    s.C[sx(4, 4)] = prior[4];
}

}  // namespace tpc
