// S6 (alignment and distortion-map adjoints): the per-track forward fit
// and hand-written reverse sweep with their helpers, shared by the adjoint
// kernel and, so that the sweep can be checked against the FP64 oracle
// without a GPU, by host programs.  The kernel sums through atomics; a
// host program through plain sums (the Acc parameter).
#pragma once

#include "tpc_dev.cuh"

namespace tpc {

namespace {

constexpr int CK = 8;       // clusters per checkpoint segment
constexpr int PRE_W = 23;   // words of a recomputed state in the segment store: p[5], lo[3], C[15]
constexpr int ND = 6;       // tangent directions: y, s, t, w, x_from, x_to

struct D6 {
    float v;
    float d[ND];
};
TPC_HD D6 dc(float v) {
    D6 r;
    r.v = v;
#pragma unroll
    for (int i = 0; i < ND; ++i) r.d[i] = 0.f;
    return r;
}
TPC_HD D6 operator+(const D6& a, const D6& b) {
    D6 r; r.v = a.v + b.v;
#pragma unroll
    for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
}
TPC_HD D6 operator-(const D6& a, const D6& b) {
    D6 r; r.v = a.v - b.v;
#pragma unroll
    for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
}
TPC_HD D6 operator-(const D6& a) {
    D6 r; r.v = -a.v;
#pragma unroll
    for (int i = 0; i < ND; ++i) r.d[i] = -a.d[i];
    return r;
}
TPC_HD D6 operator*(const D6& a, const D6& b) {
    D6 r; r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
TPC_HD D6 operator/(const D6& a, const D6& b) {
    D6 r; r.v = a.v / b.v;
    const float ib = 1.f / b.v;
#pragma unroll
    for (int i = 0; i < ND; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}
TPC_HD D6 operator*(const D6& a, float b) {
    D6 r; r.v = a.v * b;
#pragma unroll
    for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b;
    return r;
}
TPC_HD D6 operator*(float b, const D6& a) { return a * b; }
TPC_HD D6 operator+(const D6& a, float b) { D6 r = a; r.v += b; return r; }
TPC_HD D6 operator+(float b, const D6& a) { D6 r = a; r.v += b; return r; }
TPC_HD D6 operator-(float b, const D6& a) { return dc(b) - a; }
TPC_HD D6 operator-(const D6& a, float b) { D6 r = a; r.v -= b; return r; }
TPC_HD D6 t_sqrt(const D6& a) {
    D6 r; r.v = sqrtf(a.v);
    const float f = 0.5f / r.v;
#pragma unroll
    for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * f;
    return r;
}
TPC_HD D6 t_asin(const D6& a) {
    D6 r; r.v = asinf(a.v);
    const float f = 1.f / sqrtf(1.f - a.v * a.v);
#pragma unroll
    for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * f;
    return r;
}
TPC_HD D6 operator/(float a, const D6& b) { return dc(a) / b; }
TPC_HD float val(const D6& a) { return a.v; }
template <class T> TPC_HD T dc1(float v);
template <> TPC_HD float dc1<float>(float v) { return v; }
template <> TPC_HD D6 dc1<D6>(float v) { return dc(v); }
TPC_HD float val(float a) { return a; }

// The transport of kf_move written over a generic scalar: rotation (when
// rot) then helix transport from x_from to x_to.  Outputs the moved y, the z
// increment, the moved sin phi and the ten non-trivial entries of the
// Jacobian d(p_out)/d(p_in).
template <class T>
struct MoveEval {
    T y2, dz, s2;
    T j00, j02, j04, j10, j12, j13, j14, j20, j22, j24;
};

template <class T>
TPC_HD bool move_eval(const T& y, const T& s, const T& t, const T& w,
                                          const T& xf, const T& xt, bool rot, float ca, float sa,
                                          float kb, float snp_max, MoveEval<T>& o) {
    T xs = xf, ys = y, ss = s;
    T dsn = dc1<T>(1.f);
    if (rot) {
        const T c = t_sqrt(1.f - s * s);
        xs = xf * ca + y * sa;
        ys = y * ca - xf * sa;
        ss = s * ca - c * sa;
        dsn = ca + s * sa / c;
    }
    const T dx = xt - xs;
    const T k = w * kb;
    const T s1 = ss;
    const T s2 = s1 - k * dx;
    if (fabsf(val(s1)) >= snp_max || fabsf(val(s2)) >= snp_max) return false;
    const T c1 = t_sqrt(1.f - s1 * s1);
    const T c2 = t_sqrt(1.f - s2 * s2);
    const T B = c1 + c2;
    const T tn = (s1 + s2) / B;
    const float sg = val(dx) >= 0.f ? 1.f : -1.f;
    const T adx = dx * sg;
    const T h = t_sqrt(1.f + tn * tn);
    const T L = adx * h;
    const T v = k * k * L * L * 0.25f;
    const T e = 1.f / t_sqrt(1.f - v);
    T g, m;
    if (val(v) < 1e-2f) {
        g = 1.f + v * (1.f / 6.f + v * (3.f / 40.f + v * (5.f / 112.f + v * (35.f / 1152.f))));
        m = 1.f / 3.f + v * (0.3f + v * (15.f / 56.f + v * (35.f / 144.f)));
    } else {
        const T u = t_sqrt(v);
        g = t_asin(u) / u;
        m = (e - g) / v;
    }
    const T arc = L * g;
    const T dtn_s1p = (1.f + tn * s1 / c1) / B;
    const T dtn_s2p = (1.f + tn * s2 / c2) / B;
    const T ds2_w = dx * (-kb);
    const T dtn_s1 = dtn_s1p + dtn_s2p;
    const T dtn_w = dtn_s2p * ds2_w;
    const T dtn_dx = -(dtn_s2p * k);
    const T dy_s1 = dx * dtn_s1;
    const T dy_w = dx * dtn_w;
    const T dy_dx = tn + dx * dtn_dx;
    const T dL_tn = adx * tn / h;
    const T darc_k = k * L * L * L * m * 0.25f;
    const T tsg = t * sg;
    const T dz_s1 = tsg * e * dL_tn * dtn_s1;
    const T dz_w = tsg * (e * dL_tn * dtn_w + darc_k * kb);
    o.j13 = arc * sg;
    o.j04 = dy_w;
    o.j14 = dz_w;
    o.j24 = ds2_w;
    if (rot) {
        const T dz_dx = tsg * e * (h * sg + dL_tn * dtn_dx);
        o.j00 = ca - dy_dx * sa;
        o.j10 = -(dz_dx * sa);
        o.j20 = k * sa;
        o.j02 = dy_s1 * dsn;
        o.j12 = dz_s1 * dsn;
        o.j22 = dsn;
    } else {
        o.j00 = dc1<T>(1.f);
        o.j10 = dc1<T>(0.f);
        o.j20 = dc1<T>(0.f);
        o.j02 = dy_s1;
        o.j12 = dz_s1;
        o.j22 = dc1<T>(1.f);
    }
    o.y2 = ys + dx * tn;
    o.dz = tsg * arc;
    o.s2 = s2;
    return true;
}

struct AdjPrm {
    float sy2, sz2, kb, snp_max, fp64_ratio, fp64_det;
    double bz, seed_snp, seed_qpt;
    float prior[5];
    int want_grad;
};

// the adjoint's parameters from the library's (host)
inline AdjPrm adj_prm(const tpc_params& p, bool want_grad) {
    AdjPrm ap;
    ap.sy2 = p.sigma_y2;
    ap.sz2 = p.sigma_z2;
    ap.kb = (float)(KAPPA * (double)p.bz);
    ap.snp_max = p.snp_max;
    ap.fp64_ratio = p.fp64_ratio;
    ap.fp64_det = p.fp64_det;
    ap.bz = p.bz;
    ap.seed_snp = p.seed_snp_max;
    ap.seed_qpt = p.seed_qpt_max;
    for (int i = 0; i < 5; ++i) ap.prior[i] = p.prior[i];
    ap.want_grad = want_grad;
    return ap;
}

struct Pre {        // state before the transport of one cluster
    double x;
    int frame;
    float p[5];
    float lo[3];
    float C[15];
};

TPC_HD void corrected_pos(const double* __restrict__ th, double xr, double y,
                                              double z, double& xo, double& yo, double& zo) {
    const double ca = cos(th[3]), sa = sin(th[3]), cb = cos(th[4]), sb = sin(th[4]);
    const double cg = cos(th[5]), sg = sin(th[5]);
    const double y1 = ca * y - sa * z, z1 = sa * y + ca * z;
    const double x2 = cb * xr + sb * z1, z2 = cb * z1 - sb * xr;
    xo = cg * x2 - sg * y1 + th[0];
    yo = sg * x2 + cg * y1 + th[1];
    zo = z2 + th[2];
}

// d(position)/d(a,b,g) contracted with the position adjoint (xb, yb, zb)
TPC_HD void rot_grad(const double* __restrict__ th, double xr, double y, double z,
                                         double xb, double yb, double zb, double out[3]) {
    const double ca = cos(th[3]), sa = sin(th[3]), cb = cos(th[4]), sb = sin(th[4]);
    const double cg = cos(th[5]), sg = sin(th[5]);
    const double y1 = ca * y - sa * z, z1 = sa * y + ca * z;
    const double x2 = cb * xr + sb * z1, z2 = cb * z1 - sb * xr;
    // d/da: y1' = -sa y - ca z, z1' = ca y - sa z
    const double y1a = -sa * y - ca * z, z1a = ca * y - sa * z;
    const double x2a = sb * z1a, z2a = cb * z1a;
    out[0] = xb * (cg * x2a - sg * y1a) + yb * (sg * x2a + cg * y1a) + zb * z2a;
    // d/db: x2' = -sb xr + cb z1, z2' = -sb z1 - cb xr
    const double x2b = -sb * xr + cb * z1, z2b = -sb * z1 - cb * xr;
    out[1] = xb * (cg * x2b) + yb * (sg * x2b) + zb * z2b;
    // d/dg
    out[2] = xb * (-sg * x2 - cg * y1) + yb * (cg * x2 - sg * y1);
}

// Per-sector tables of the alignment correction (k_adj_tables fills them
// from the 216 parameters)
// (once per call): R - I, dR/da, dR/db, dR/dg (3x3 each, acting on
// (x_row, y, z)) and the shift t.  The per-hit correction is then the small
// FP32 increment (R - I) p + t, and the angle gradient a 27-term FP32
// contraction, instead of six FP64 sines and cosines per hit.
constexpr int ROT_TAB = 39;  // floats per sector: R - I (9), dR (27), t (3)

// corrected position of (x_row, y, z) in sector table o: x as FP64 (a
// plane position), y and z as FP32
TPC_HD void corr_tab(const float* o, double xr, float y, float z, double& xc,
                                         float& yc, float& zc) {
    const float xf = (float)xr;
    const float dx = o[0] * xf + o[1] * y + o[2] * z + o[36];
    const float dy = o[3] * xf + o[4] * y + o[5] * z + o[37];
    const float dz = o[6] * xf + o[7] * y + o[8] * z + o[38];
    xc = xr + (double)dx;
    yc = y + dy;
    zc = z + dz;
}

// the angle gradient: (xb, yb, zb) . dR_k (x_row, y, z) for k = a, b, g
TPC_HD void rot_grad_tab(const float* o, float xr, float y, float z, float xb,
                                             float yb, float zb, float out[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float* d = o + 9 + 9 * k;
        out[k] = xb * (d[0] * xr + d[1] * y + d[2] * z) + yb * (d[3] * xr + d[4] * y + d[5] * z) +
                 zb * (d[6] * xr + d[7] * y + d[8] * z);
    }
}

// the displacement of the cluster's voxel added to its corrected position;
// returns the voxel
TPC_HD int add_field(const double* __restrict__ field, const FieldGridD& fg,
                                         const Geo* __restrict__ geo, int r, int sec, float y, float z,
                                         double& xc, float& yc, float& zc) {
    const int v = field_voxel(y, z, r, NROW, geo->row_xf[r], sec, fg);
    const double* f = field + 3 * (int64_t)v;
    xc += f[0];
    yc = yc + (float)f[1];
    zc = zc + (float)f[2];
    return v;
}

// One sector's table from its 6 parameters th (o[ROT_TAB]).
TPC_HD void adj_table_sector(const double* th, float* o) {
    const double e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    double th0[6] = {0.0, 0.0, 0.0, th[3], th[4], th[5]};
    for (int col = 0; col < 3; ++col) {
        double xo, yo, zo;
        corrected_pos(th0, e[col][0], e[col][1], e[col][2], xo, yo, zo);
        o[0 * 3 + col] = (float)(xo - e[col][0]);
        o[1 * 3 + col] = (float)(yo - e[col][1]);
        o[2 * 3 + col] = (float)(zo - e[col][2]);
        for (int r = 0; r < 3; ++r) {
            double g3[3];
            rot_grad(th0, e[col][0], e[col][1], e[col][2], e[r][0], e[r][1], e[r][2], g3);
            for (int k = 0; k < 3; ++k) o[9 + k * 9 + r * 3 + col] = (float)g3[k];  // dR_k[r][col]
        }
    }
    for (int i = 0; i < 3; ++i) o[36 + i] = (float)th[i];
}

// a run of one voxel's position adjoints into the field gradient
template <class Acc>
TPC_HD void flush_field(Acc& acc, int v, double f[3]) {
    if (v >= 0)
        for (int i = 0; i < 3; ++i) acc.field(3 * (int64_t)v + i, f[i]);
    f[0] = f[1] = f[2] = 0.0;
}

// One track's chi2 and, if P.want_grad, its gradient: the forward fit on
// corrected clusters (+ field[v] when FIELD) with a checkpoint every CK
// clusters, then the reverse sweep.  acc receives the chi2
// (acc.chi2), the per-sector shift and angle gradients (acc.align(i, v),
// i = 6 sector + k), the voxel gradients (acc.field(i, v) when
// acc.want_field()) and capacity errors (acc.status).  tab holds the
// per-sector rotation tables.
// Where one track's clusters are read: through its hit list (the group of
// each cluster found by binary search, cached while the hits stay in one
// group), or from a copy gathered in track order (position, row and sector
// at the track's offset into gyz, grow, gsec).
struct AdjHit {
    float y, z;
    int row, sec;
};
struct AdjHits {
    const int32_t* h;
    const float* y;
    const float* z;
    const uint16_t* row;
    const int64_t* evt_off;
    int G;
    const float2* gyz;  // gathered copy, or nullptr
    const uint8_t* grow;
    const uint8_t* gsec;
    int64_t gbase;
    int gcur;
    int64_t gb, ge;
    TPC_HD AdjHit at(int j) {
        AdjHit r;
        if (gyz) {
            const float2 v = gyz[gbase + j];
            r.y = v.x;
            r.z = v.y;
            r.row = grow[gbase + j];
            r.sec = gsec[gbase + j];
            return r;
        }
        const int c = h[j];
        if (c < gb || c >= ge) {
            gcur = group_of(evt_off, G, c);
            gb = evt_off[gcur];
            ge = evt_off[gcur + 1];
        }
        r.y = y[c];
        r.z = z[c];
        r.row = row[c];
        r.sec = gcur % NSEC;
        return r;
    }
};

TPC_HD AdjHits adj_hits_direct(const int32_t* h, const float* y, const float* z, const uint16_t* row,
                               const int64_t* evt_off, int G) {
    return AdjHits{h, y, z, row, evt_off, G, nullptr, nullptr, nullptr, 0, -1, 0, 0};
}

// seg: the store of one segment's recomputed states, CK x PRE_W words, word
// w of entry k at seg[(k PRE_W + w) seg_stride] (the kernel gives each
// thread a column of shared memory, stride = threads per block; a host
// program a plain array, stride 1).
template <bool FIELD, class Acc>
TPC_HD void adjoint_track(AdjHits& hits, int n, const float* tab, const Geo* __restrict__ geo, const AdjPrm& P,
                          const double* __restrict__ field, const FieldGridD& fg, float* seg, int seg_stride,
                          Acc& acc) {
    if (n < 3) return;
    // seed from the uncorrected clusters
    KF s;
    {
        int rows[3], secs[3];
        float ys[3], zs[3];
        const int pick[3] = {0, n / 2, n - 1};
        for (int k = 0; k < 3; ++k) {
            const AdjHit a = hits.at(pick[k]);
            rows[k] = a.row;
            secs[k] = a.sec;
            ys[k] = a.y;
            zs[k] = a.z;
        }
        kf_seed(s, rows, secs, ys, zs, true, geo, P.bz, P.seed_snp, P.seed_qpt, P.prior);
    }
    const int nck = (n + CK - 1) / CK;
    Pre ck[(NROW + 4 * CK) / CK];  // checkpoints (tracks longer than this are refused)
    if (nck > (int)(sizeof(ck) / sizeof(ck[0]))) {
        acc.status(TPC_ERR_CAPACITY, 5);
        return;
    }
    NSum chi2;
    bool ok = true;
    for (int j = 0; j < n && ok; ++j) {
        if (P.want_grad && j % CK == 0) {  // checkpoints only for the reverse sweep
            Pre& q = ck[j / CK];
            q.x = s.x; q.frame = s.frame;
            for (int i = 0; i < 5; ++i) q.p[i] = s.p[i];
            for (int i = 0; i < 3; ++i) q.lo[i] = s.lo[i];
            for (int i = 0; i < 15; ++i) q.C[i] = s.C[i];
        }
        const AdjHit hc = hits.at(j);
        const int sec = hc.sec;
        double xc;
        float yc, zc;
        corr_tab(tab + sec * ROT_TAB, geo->row_xd[hc.row], hc.y, hc.z, xc, yc, zc);
        if constexpr (FIELD) add_field(field, fg, geo, hc.row, sec, hc.y, hc.z, xc, yc, zc);
        MoveJ mj;
        ok = kf_move<float>(s, xc, sec, geo, P.kb, P.snp_max, &mj);
        if (ok) chi2.add(kf_update(s, yc, zc, P.sy2, P.sz2, P.fp64_ratio, P.fp64_det, nullptr, &mj));
    }
    if (!ok) return;
    acc.chi2((double)chi2.value());
    if (!P.want_grad) return;

    // reverse sweep
    float pb[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    float A[15];
    for (int i = 0; i < 15; ++i) A[i] = 0.f;
    // the alignment gradient of the run of consecutive clusters in one
    // sector, flushed when the sector changes
    int gsec = -1;
    double gacc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    float xbar_from_next = 0.f;  // x_from adjoint of the step after the current one
    int vcur = -1;               // voxel of the run of clusters being summed
    double facc[3] = {0.0, 0.0, 0.0};
    double segx[CK];
    int segf[CK];
    for (int k = nck - 1; k >= 0; --k) {
        const int j0 = k * CK, j1 = min(n, j0 + CK);
        // recompute the segment's pre-transport states
        KF r;
        r.x = ck[k].x; r.frame = ck[k].frame;
        for (int i = 0; i < 5; ++i) r.p[i] = ck[k].p[i];
        for (int i = 0; i < 3; ++i) r.lo[i] = ck[k].lo[i];
        for (int i = 0; i < 15; ++i) r.C[i] = ck[k].C[i];
        for (int j = j0; j < j1; ++j) {
            {
                float* o = seg + (size_t)(j - j0) * PRE_W * seg_stride;
                for (int i = 0; i < 5; ++i) o[i * seg_stride] = r.p[i];
                for (int i = 0; i < 3; ++i) o[(5 + i) * seg_stride] = r.lo[i];
                for (int i = 0; i < 15; ++i) o[(8 + i) * seg_stride] = r.C[i];
                segx[j - j0] = r.x;
                segf[j - j0] = r.frame;
            }
            const AdjHit hc = hits.at(j);
            const int sec = hc.sec;
            double xc;
            float yc, zc;
            corr_tab(tab + sec * ROT_TAB, geo->row_xd[hc.row], hc.y, hc.z, xc, yc, zc);
            if constexpr (FIELD) add_field(field, fg, geo, hc.row, sec, hc.y, hc.z, xc, yc, zc);
            MoveJ mj;
            kf_move<float>(r, xc, sec, geo, P.kb, P.snp_max, &mj);
            kf_update(r, yc, zc, P.sy2, P.sz2, P.fp64_ratio, P.fp64_det, nullptr, &mj);
        }
        for (int j = j1 - 1; j >= j0; --j) {
            Pre q;
            {
                const float* o = seg + (size_t)(j - j0) * PRE_W * seg_stride;
                for (int i = 0; i < 5; ++i) q.p[i] = o[i * seg_stride];
                for (int i = 0; i < 3; ++i) q.lo[i] = o[(5 + i) * seg_stride];
                for (int i = 0; i < 15; ++i) q.C[i] = o[(8 + i) * seg_stride];
                q.x = segx[j - j0];
                q.frame = segf[j - j0];
            }
            const AdjHit hc = hits.at(j);
            const int sec = hc.sec;
            const float* tb = tab + sec * ROT_TAB;
            const double xr = geo->row_xd[hc.row];
            double xc;
            float yc, zc;
            corr_tab(tb, xr, hc.y, hc.z, xc, yc, zc);
            int vox = -1;
            if constexpr (FIELD) vox = add_field(field, fg, geo, hc.row, sec, hc.y, hc.z, xc, yc, zc);
            // forward of this step again: transport, then update pieces
            KF m;
            m.x = q.x; m.frame = q.frame;
            for (int i = 0; i < 5; ++i) m.p[i] = q.p[i];
            for (int i = 0; i < 3; ++i) m.lo[i] = q.lo[i];
            for (int i = 0; i < 15; ++i) m.C[i] = q.C[i];
            kf_move<float>(m, xc, sec, geo, P.kb, P.snp_max);
            float Cm[5][5];
            for (int a = 0; a < 5; ++a)
                for (int bb = 0; bb < 5; ++bb) Cm[a][bb] = m.C[sx(a, bb)];
            const float r0 = (yc - m.p[0]) - m.lo[0];
            const float r1 = (zc - m.p[1]) - m.lo[1];
            const float S00 = Cm[0][0] + P.sy2, S01 = Cm[0][1], S11 = Cm[1][1] + P.sz2;
            const float det = S00 * S11 - S01 * S01;
            const float W00 = S11 / det, W01 = -S01 / det, W11 = S00 / det;
            float Bm[5][2], Km[5][2];
            for (int i = 0; i < 5; ++i) {
                Bm[i][0] = Cm[i][0];
                Bm[i][1] = Cm[i][1];
                Km[i][0] = Bm[i][0] * W00 + Bm[i][1] * W01;
                Km[i][1] = Bm[i][0] * W01 + Bm[i][1] * W11;
            }
            // ---- update backward
            float Af[5][5];
            for (int a = 0; a < 5; ++a)
                for (int bb = 0; bb < 5; ++bb) Af[a][bb] = A[sx(a, bb)];
            const float Wr0 = W00 * r0 + W01 * r1, Wr1 = W01 * r0 + W11 * r1;
            float rb0 = 2.f * Wr0, rb1 = 2.f * Wr1;
            for (int i = 0; i < 5; ++i) {
                rb0 += Km[i][0] * pb[i];
                rb1 += Km[i][1] * pb[i];
            }
            // AB = A B (5x2)
            float AB[5][2];
            for (int i = 0; i < 5; ++i) {
                AB[i][0] = 0.f;
                AB[i][1] = 0.f;
                for (int l = 0; l < 5; ++l) {
                    AB[i][0] += Af[i][l] * Bm[l][0];
                    AB[i][1] += Af[i][l] * Bm[l][1];
                }
            }
            // Wbar = r r^T + B^T Kbar - B^T A B, Kbar = pb r^T
            float Wb[2][2];
            const float rr[2] = {r0, r1};
            for (int a = 0; a < 2; ++a)
                for (int bb = 0; bb < 2; ++bb) {
                    float v = rr[a] * rr[bb];
                    for (int i = 0; i < 5; ++i) v += Bm[i][a] * pb[i] * rr[bb] - Bm[i][a] * AB[i][bb];
                    Wb[a][bb] = v;
                }
            // Bbar = Kbar W - 2 A B W
            float Bb[5][2];
            for (int i = 0; i < 5; ++i) {
                const float k0 = pb[i] * r0 - 2.f * AB[i][0];
                const float k1 = pb[i] * r1 - 2.f * AB[i][1];
                Bb[i][0] = k0 * W00 + k1 * W01;
                Bb[i][1] = k0 * W01 + k1 * W11;
            }
            // Sbar = -W Wbar W
            float T0[2][2], Sb[2][2];
            const float Wm[2][2] = {{W00, W01}, {W01, W11}};
            for (int a = 0; a < 2; ++a)
                for (int bb = 0; bb < 2; ++bb) T0[a][bb] = Wm[a][0] * Wb[0][bb] + Wm[a][1] * Wb[1][bb];
            for (int a = 0; a < 2; ++a)
                for (int bb = 0; bb < 2; ++bb) Sb[a][bb] = -(T0[a][0] * Wm[0][bb] + T0[a][1] * Wm[1][bb]);
            // position adjoints of the measurement
            const float ybar = rb0, zbar = rb1;
            // p- adjoint
            float pm[5];
            for (int i = 0; i < 5; ++i) pm[i] = pb[i];
            pm[0] -= rb0;
            pm[1] -= rb1;
            // A- = A + sym(E), E = Sbar in block, Bbar in columns 0,1
            float Am[5][5];
            for (int a = 0; a < 5; ++a)
                for (int bb = 0; bb < 5; ++bb) {
                    float e1 = 0.f, e2 = 0.f;
                    if (bb < 2) e1 += Bb[a][bb];
                    if (a < 2) e2 += Bb[bb][a];
                    if (a < 2 && bb < 2) {
                        e1 += Sb[a][bb];
                        e2 += Sb[bb][a];
                    }
                    Am[a][bb] = Af[a][bb] + 0.5f * (e1 + e2);
                }
            // ---- transport backward (forward-mode derivatives of G and J)
            const bool rot = sec != q.frame;
            float cad = 1.f, sad = 0.f;
            if (rot) {
                const int kk = ((sec % NPHI) - (q.frame % NPHI) + NPHI) % NPHI;
                cad = (float)geo->da_cos[kk];
                sad = (float)geo->da_sin[kk];
            }
            // seed the six tangent directions at the pre-transport point;
            // positions relative to x_from keep FP32 precision
            const float yv = q.p[0] + q.lo[0];
            const float sv = q.p[2] + q.lo[2];
            D6 Dy = dc(yv), Ds = dc(sv), Dt = dc(q.p[3]), Dw = dc(q.p[4]);
            D6 Dxf = dc(0.f), Dxt = dc((float)(xc - q.x));
            Dy.d[0] = 1.f; Ds.d[1] = 1.f; Dt.d[2] = 1.f; Dw.d[3] = 1.f; Dxf.d[4] = 1.f; Dxt.d[5] = 1.f;
            if (rot) {
                // the rotation mixes x into y: evaluate with the absolute x
                Dxf.v = (float)q.x;
                Dxt.v = (float)xc;
            }
            MoveEval<D6> me;
            move_eval<D6>(Dy, Ds, Dt, Dw, Dxf, Dxt, rot, cad, sad, P.kb, P.snp_max, me);
            float J[5][5] = {};
            J[0][0] = me.j00.v; J[0][2] = me.j02.v; J[0][4] = me.j04.v;
            J[1][0] = me.j10.v; J[1][1] = 1.f; J[1][2] = me.j12.v; J[1][3] = me.j13.v; J[1][4] = me.j14.v;
            J[2][0] = me.j20.v; J[2][2] = me.j22.v; J[2][4] = me.j24.v;
            J[3][3] = 1.f; J[4][4] = 1.f;
            // pre-transport covariance (full)
            float Cp[5][5];
            for (int a = 0; a < 5; ++a)
                for (int bb = 0; bb < 5; ++bb) Cp[a][bb] = q.C[sx(a, bb)];
            // Jbar = 2 A- J C
            float AJ[5][5], Jb[5][5];
            for (int a = 0; a < 5; ++a)
                for (int bb = 0; bb < 5; ++bb) {
                    float v = 0.f;
                    for (int l = 0; l < 5; ++l) v += Am[a][l] * J[l][bb];
                    AJ[a][bb] = v;
                }
            for (int a = 0; a < 5; ++a)
                for (int bb = 0; bb < 5; ++bb) {
                    float v = 0.f;
                    for (int l = 0; l < 5; ++l) v += AJ[a][l] * Cp[l][bb];
                    Jb[a][bb] = 2.f * v;
                }
            // A_pre = J^T A- J
            float An[15];
            for (int a = 0; a < 5; ++a)
                for (int bb = a; bb < 5; ++bb) {
                    float v = 0.f;
                    for (int l = 0; l < 5; ++l) v += J[l][a] * AJ[l][bb];
                    An[sx(a, bb)] = v;
                }
            // p_pre adjoint: J^T pm, plus sum Jbar_ab dJ_ab/dq
            float qb[ND];
            for (int d = 0; d < ND; ++d) {
                float v = pm[0] * me.y2.d[d] + pm[1] * me.dz.d[d] + pm[2] * me.s2.d[d];
                v += Jb[0][0] * me.j00.d[d] + Jb[0][2] * me.j02.d[d] + Jb[0][4] * me.j04.d[d];
                v += Jb[1][0] * me.j10.d[d] + Jb[1][2] * me.j12.d[d] + Jb[1][3] * me.j13.d[d] +
                     Jb[1][4] * me.j14.d[d];
                v += Jb[2][0] * me.j20.d[d] + Jb[2][2] * me.j22.d[d] + Jb[2][4] * me.j24.d[d];
                qb[d] = v;
            }
            // t and w pass through G unchanged: add their identity terms
            float pn[5];
            pn[0] = qb[0];
            pn[1] = pm[1];
            pn[2] = qb[1];
            pn[3] = qb[2] + pm[3];
            pn[4] = qb[3] + pm[4];
            const float xbar_to = qb[5];
            const float xbar_from = qb[4];
            for (int i = 0; i < 5; ++i) pb[i] = pn[i];
            for (int i = 0; i < 15; ++i) A[i] = An[i];
            // cluster j's corrected position adjoint: arrival (x_to, y, z)
            // plus the departure of step j+1 (x_from)
            const double xb = (double)xbar_to + (double)xbar_from_next;
            xbar_from_next = xbar_from;
            float gr[3];
            rot_grad_tab(tb, (float)xr, hc.y, hc.z, (float)xb, ybar, zbar, gr);
            if (sec != gsec) {
                if (gsec >= 0)
                    for (int i = 0; i < 6; ++i) acc.align(gsec * 6 + i, gacc[i]);
                gsec = sec;
                for (int i = 0; i < 6; ++i) gacc[i] = 0.0;
            }
            gacc[0] += xb;
            gacc[1] += ybar;
            gacc[2] += zbar;
            gacc[3] += gr[0];
            gacc[4] += gr[1];
            gacc[5] += gr[2];
            if constexpr (FIELD) {
                if (acc.want_field()) {
                    if (vox != vcur) {
                        flush_field(acc, vcur, facc);
                        vcur = vox;
                    }
                    facc[0] += xb;
                    facc[1] += ybar;
                    facc[2] += zbar;
                }
            }
        }
    }
    if constexpr (FIELD) {
        if (acc.want_field()) flush_field(acc, vcur, facc);
    }
    if (gsec >= 0)
        for (int i = 0; i < 6; ++i) acc.align(gsec * 6 + i, gacc[i]);
}

}  // namespace

}  // namespace tpc
