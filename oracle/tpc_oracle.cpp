// TPC tracking oracle (FP64 CPU restatement).  TEST INFRASTRUCTURE ONLY:
// loaded by the tests, the smoke check and the benchmark's CPU-baseline leg;
// the CUDA library never calls it and the two share no code.
//
// The paper (arXiv 2412.13755) says TPC tracking runs on the GPUs of the
// online farm and takes 99% of their compute (Sec. 4.2 and Sec. 5), but
// describes no algorithm.  Each step below states the reading it follows:
//   S1  binning per (event, sector, pad row), canonical id = input index;
//   S2  cellular-automaton neighbour choice between pad rows (triplet D^2);
//   S3  chaining of mutual links into segments;
//   S4  greedy merging of segments within a sector or across phi-adjacent
//       sectors by a 5-d chi2 on fitted states;
//   S5  Kalman fit of (y, z, sin phi, tan lambda, q/pT) with 5x5 covariance
//       in a uniform Bz, exact helix transport;
//   S6  d(sum chi2)/d(216 per-sector rigid-body corrections), exact
//       derivative of the fit as computed (forward-mode dual numbers).
// Floating point that decides an integer in S2 (window cuts, D^2 and its
// comparisons) is evaluated in FP32 with one rounding per operation, the
// precision the GPU kernel decides in; everything else is FP64 (an FP64
// diagnostic mode of S2 measures how many decisions that changes).
//
// Pins (tests/test_oracle_*.py) tie each part to something other than this
// file: the transport to the generator's global-frame crossings and to
// central differences; the fit to closed-form least squares in the linear
// case and to unit-width pulls; the seed to exact helix points; extension
// and merging to noise-free tracks and to the least-squares chi2 identity;
// the whole find to brute-force chain enumeration on tiny events; the
// gradients to central differences.  Parity unpinned beyond those cases
// and determinism: the tie-break orders of S2, S3b and S4, the greedy merge
// order and the tracklet ownership rule, which are heuristic rules with no
// closed form (pinned only by their stated definitions).
#include "tpc_oracle.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <limits>
#include <map>
#include <vector>
#include <type_traits>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int NSEC = 36;
constexpr int NPHI = 18;
constexpr int NROW = 152;
constexpr double KAPPA = 2.99792458e-3;  // cm^-1 T^-1 (GeV/c)
constexpr double PI = 3.14159265358979323846;
const double TAN_HALF = std::tan(10.0 * PI / 180.0);

int g_threads = 0;

// ---- geometry (pad-row planes, sector frames) ---------------------------
double row_x(int r) { return 85.0 + r * (162.0 / 151.0); }
float row_xf(int r) { return (float)row_x(r); }
double sector_alpha(int s) { return ((s % NPHI) + 0.5) * (20.0 * PI / 180.0); }
double delta_alpha(int from, int to) {
    double d = sector_alpha(to) - sector_alpha(from);
    while (d > PI) d -= 2 * PI;
    while (d <= -PI) d += 2 * PI;
    return d;
}

// ---- dual numbers for the exact derivative of the fit (S6) ---------------
template <int N>
struct Dual {
    double v;
    double d[N];
    Dual() : v(0) { for (int i = 0; i < N; ++i) d[i] = 0; }
    Dual(double x) : v(x) { for (int i = 0; i < N; ++i) d[i] = 0; }
};
template <int N> Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r; r.v = a.v + b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int N> Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r; r.v = a.v - b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <int N> Dual<N> operator-(const Dual<N>& a) {
    Dual<N> r; r.v = -a.v; for (int i = 0; i < N; ++i) r.d[i] = -a.d[i]; return r; }
template <int N> Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r; r.v = a.v * b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <int N> Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r; r.v = a.v / b.v;
    for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
    return r; }
template <int N> Dual<N> operator+(const Dual<N>& a, double b) { return a + Dual<N>(b); }
template <int N> Dual<N> operator+(double a, const Dual<N>& b) { return Dual<N>(a) + b; }
template <int N> Dual<N> operator-(const Dual<N>& a, double b) { return a - Dual<N>(b); }
template <int N> Dual<N> operator-(double a, const Dual<N>& b) { return Dual<N>(a) - b; }
template <int N> Dual<N> operator*(const Dual<N>& a, double b) {
    Dual<N> r; r.v = a.v * b; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b; return r; }
template <int N> Dual<N> operator*(double a, const Dual<N>& b) { return b * a; }
template <int N> Dual<N> operator/(const Dual<N>& a, double b) { return a * (1.0 / b); }
template <int N> Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }
template <int N> Dual<N>& operator+=(Dual<N>& a, const Dual<N>& b) { a = a + b; return a; }
template <int N> Dual<N>& operator-=(Dual<N>& a, const Dual<N>& b) { a = a - b; return a; }
template <int N> Dual<N> sqrt(const Dual<N>& a) {
    Dual<N> r; r.v = std::sqrt(a.v); double f = 0.5 / r.v;
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * f;
    return r; }
template <int N> Dual<N> asin(const Dual<N>& a) {
    Dual<N> r; r.v = std::asin(a.v); double f = 1.0 / std::sqrt(1.0 - a.v * a.v);
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * f;
    return r; }
template <int N> Dual<N> sin(const Dual<N>& a) {
    Dual<N> r; r.v = std::sin(a.v); double f = std::cos(a.v);
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * f;
    return r; }
template <int N> Dual<N> cos(const Dual<N>& a) {
    Dual<N> r; r.v = std::cos(a.v); double f = -std::sin(a.v);
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * f;
    return r; }
template <int N> double val(const Dual<N>& a) { return a.v; }
inline double val(double a) { return a; }
using std::asin;
using std::cos;
using std::sin;
using std::sqrt;

// ---- operation counting (the algorithmic work of a Kalman step) ---------
// A double that counts the arithmetic performed on it: +, -, *, / and each
// square root or arcsine count one operation, except an operation whose
// operand is an exact 0 (or 1 for *, /): those are structural zeros and
// ones of the Jacobians and cost an implementation that exploits the
// structure nothing.  Used single-threaded (the counter is per thread).
thread_local long long g_ops = 0;
struct Cnt {
    double v;
    Cnt() : v(0) {}
    Cnt(double x) : v(x) {}
};
inline bool triv_add(double a, double b) { return a == 0.0 || b == 0.0; }
inline bool triv_mul(double a, double b) { return a == 0.0 || b == 0.0 || a == 1.0 || b == 1.0; }
inline Cnt operator+(const Cnt& a, const Cnt& b) { if (!triv_add(a.v, b.v)) ++g_ops; return Cnt(a.v + b.v); }
inline Cnt operator-(const Cnt& a, const Cnt& b) { if (!triv_add(a.v, b.v)) ++g_ops; return Cnt(a.v - b.v); }
inline Cnt operator-(const Cnt& a) { return Cnt(-a.v); }
inline Cnt operator*(const Cnt& a, const Cnt& b) { if (!triv_mul(a.v, b.v)) ++g_ops; return Cnt(a.v * b.v); }
inline Cnt operator/(const Cnt& a, const Cnt& b) { if (b.v != 1.0 && a.v != 0.0) ++g_ops; return Cnt(a.v / b.v); }
inline Cnt operator+(const Cnt& a, double b) { return a + Cnt(b); }
inline Cnt operator+(double a, const Cnt& b) { return Cnt(a) + b; }
inline Cnt operator-(const Cnt& a, double b) { return a - Cnt(b); }
inline Cnt operator-(double a, const Cnt& b) { return Cnt(a) - b; }
inline Cnt operator*(const Cnt& a, double b) { return a * Cnt(b); }
inline Cnt operator*(double a, const Cnt& b) { return Cnt(a) * b; }
inline Cnt operator/(const Cnt& a, double b) { return a / Cnt(b); }
inline Cnt operator/(double a, const Cnt& b) { return Cnt(a) / b; }
inline Cnt& operator+=(Cnt& a, const Cnt& b) { a = a + b; return a; }
inline Cnt& operator-=(Cnt& a, const Cnt& b) { a = a - b; return a; }
inline Cnt sqrt(const Cnt& a) { ++g_ops; return Cnt(std::sqrt(a.v)); }
inline Cnt asin(const Cnt& a) { ++g_ops; return Cnt(std::asin(a.v)); }
inline Cnt sin(const Cnt& a) { ++g_ops; return Cnt(std::sin(a.v)); }
inline Cnt cos(const Cnt& a) { ++g_ops; return Cnt(std::cos(a.v)); }
inline double val(const Cnt& a) { return a.v; }

// ---- symmetric 5x5 storage ----------------------------------------------
// order 00 01 02 03 04 11 12 13 14 22 23 24 33 34 44
inline int sidx(int i, int j) {
    if (i > j) std::swap(i, j);
    static const int base[5] = {0, 5, 9, 12, 14};
    return base[i] + (j - i);
}

// ---- S5: helix transport between planes x1 -> x2 of one frame ------------
// Exact for a uniform Bz without material:
//   s2 = s1 - k dx,  k = KAPPA Bz w
//   y2 = y1 + dx (s1+s2)/(c1+c2)              (tan of the mean direction)
//   chord L = |dx| sqrt(1 + ((s1+s2)/(c1+c2))^2), arc = L asin(u)/u, u = |k|L/2
//   z2 = z1 + t * arc * sign(dx)
// F is the analytic Jacobian d(p2)/d(p1); dX2 = d(p2)/d(x2) = -d(p2)/d(x1).
template <class T>
bool transport(const T& x1, const T& x2, T p[5], T F[25], T dX2[5],
               const orc_params& prm) {
    const T dx = x2 - x1;
    const T s1 = p[2], t = p[3], w = p[4];
    const double kb = KAPPA * prm.bz;
    const T k = w * kb;
    const T s2 = s1 - k * dx;
    if (std::fabs(val(s1)) >= prm.snp_max || std::fabs(val(s2)) >= prm.snp_max) return false;
    const T c1 = sqrt(1.0 - s1 * s1);
    const T c2 = sqrt(1.0 - s2 * s2);
    const T A = s1 + s2, B = c1 + c2;
    const T tn = A / B;
    const double sg = val(dx) >= 0 ? 1.0 : -1.0;
    const T adx = dx * sg;
    const T h = sqrt(1.0 + tn * tn);
    const T L = adx * h;
    const T v = k * k * L * L * 0.25;  // u^2
    T g, m;                            // g = asin(u)/u, m = (1/sqrt(1-v) - g)/v
    const T e = 1.0 / sqrt(1.0 - v);
    if (val(v) < 1e-6) {
        g = 1.0 + v * (1.0 / 6.0) + v * v * (3.0 / 40.0) + v * v * v * (5.0 / 112.0);
        m = (1.0 / 3.0) + v * 0.3 + v * v * (15.0 / 56.0);
    } else {
        const T u = sqrt(v);
        g = asin(u) / u;
        m = (e - g) / v;
    }
    const T arc = L * g;
    // derivatives of tn
    const T dtn_s1p = (1.0 + tn * s1 / c1) / B;  // partial wrt s1 at fixed s2
    const T dtn_s2p = (1.0 + tn * s2 / c2) / B;  // partial wrt s2 at fixed s1
    const T ds2_w = dx * (-kb);
    const T dtn_s1 = dtn_s1p + dtn_s2p;
    const T dtn_w = dtn_s2p * ds2_w;
    const T dtn_dx = dtn_s2p * (-k);
    const T dy_s1 = dx * dtn_s1;
    const T dy_w = dx * dtn_w;
    const T dy_dx = tn + dx * dtn_dx;
    const T dL_tn = adx * tn / h;
    const T dL_s1 = dL_tn * dtn_s1;
    const T dL_w = dL_tn * dtn_w;
    const T dL_dx = h * sg + dL_tn * dtn_dx;
    const T darc_k = k * L * L * L * m * 0.25;  // d(arc)/dk at fixed L
    const T darc_s1 = e * dL_s1;
    const T darc_w = e * dL_w + darc_k * kb;
    const T darc_dx = e * dL_dx;
    const T tsg = t * sg;

    for (int i = 0; i < 25; ++i) F[i] = T(0.0);
    F[0 * 5 + 0] = T(1.0);
    F[0 * 5 + 2] = dy_s1;
    F[0 * 5 + 4] = dy_w;
    F[1 * 5 + 1] = T(1.0);
    F[1 * 5 + 2] = tsg * darc_s1;
    F[1 * 5 + 3] = arc * sg;
    F[1 * 5 + 4] = tsg * darc_w;
    F[2 * 5 + 2] = T(1.0);
    F[2 * 5 + 4] = ds2_w;
    F[3 * 5 + 3] = T(1.0);
    F[4 * 5 + 4] = T(1.0);
    dX2[0] = dy_dx;
    dX2[1] = tsg * darc_dx;
    dX2[2] = -k;
    dX2[3] = T(0.0);
    dX2[4] = T(0.0);

    p[0] = p[0] + dx * tn;
    p[1] = p[1] + tsg * arc;
    p[2] = s2;
    return true;
}

// Move the state from plane x of frame `frame` to plane x_to of frame `to`:
// on a sector change rotate the frame by da (x' = x cos + y sin,
// y' = -x sin + y cos, phi' = phi - da), then transport from x'(y) to x_to.
// J is the full Jacobian of the composition with respect to p.
template <class T>
bool move_state(T& x, T p[5], int& frame, const T& x_to, int to, T J[25],
                T dXto[5], const orc_params& prm) {
    T F[25];
    if (to != frame) {
        const double da = delta_alpha(frame, to);
        const double ca = std::cos(da), sa = std::sin(da);
        const T s = p[2];
        if (std::fabs(val(s)) >= prm.snp_max) return false;
        const T c = sqrt(1.0 - s * s);
        const T xn = x * ca + p[0] * sa;
        const T yn = p[0] * ca - x * sa;
        const T sn = s * ca - c * sa;
        if (std::fabs(val(sn)) >= prm.snp_max) return false;
        const T dsn_ds = ca + s * sa / c;
        T q[5] = {yn, p[1], sn, p[3], p[4]};
        if (!transport(xn, x_to, q, F, dXto, prm)) return false;
        // d p_to / d p = F * Jrot + dT/dx1 (x) d xn / d p,  dT/dx1 = -dXto
        for (int i = 0; i < 5; ++i) {
            for (int j = 0; j < 5; ++j) J[i * 5 + j] = F[i * 5 + j];
            J[i * 5 + 0] = F[i * 5 + 0] * ca - dXto[i] * sa;
            J[i * 5 + 2] = F[i * 5 + 2] * dsn_ds;
        }
        for (int i = 0; i < 5; ++i) p[i] = q[i];
    } else {
        if (!transport(x, x_to, p, F, dXto, prm)) return false;
        for (int i = 0; i < 25; ++i) J[i] = F[i];
    }
    x = x_to;
    frame = to;
    return true;
}

template <class T>
void cov_transform(T C[15], const T J[25]) {
    T full[25], tmp[25];
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) full[i * 5 + j] = C[sidx(i, j)];
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            T acc(0.0);
            for (int l = 0; l < 5; ++l) acc += J[i * 5 + l] * full[l * 5 + j];
            tmp[i * 5 + j] = acc;
        }
    for (int i = 0; i < 5; ++i)
        for (int j = i; j < 5; ++j) {
            T acc(0.0);
            for (int l = 0; l < 5; ++l) acc += tmp[i * 5 + l] * J[j * 5 + l];
            C[sidx(i, j)] = acc;
        }
}

// Kalman update with the 2-d measurement (my, mz) of (y, z):
// S = H C H^T + R, K = C H^T S^-1, p += K r, C -= K H C, chi2 += r^T S^-1 r
// (r = predicted residual).
template <class T>
void kf_update(T p[5], T C[15], const T& my, const T& mz, double sy2, double sz2,
               T& chi2, T res_out[2] = nullptr, T sinv_out[3] = nullptr) {
    const T r0 = my - p[0], r1 = mz - p[1];
    const T S00 = C[sidx(0, 0)] + sy2, S01 = C[sidx(0, 1)], S11 = C[sidx(1, 1)] + sz2;
    const T det = S00 * S11 - S01 * S01;
    const T i00 = S11 / det, i01 = -S01 / det, i11 = S00 / det;
    T K0[5], K1[5], C0[5], C1[5];
    for (int i = 0; i < 5; ++i) {
        C0[i] = C[sidx(0, i)];
        C1[i] = C[sidx(1, i)];
    }
    for (int i = 0; i < 5; ++i) {
        K0[i] = C0[i] * i00 + C1[i] * i01;
        K1[i] = C0[i] * i01 + C1[i] * i11;
    }
    for (int i = 0; i < 5; ++i) p[i] = p[i] + K0[i] * r0 + K1[i] * r1;
    for (int i = 0; i < 5; ++i)
        for (int j = i; j < 5; ++j) C[sidx(i, j)] = C[sidx(i, j)] - (K0[i] * C0[j] + K1[i] * C1[j]);
    chi2 = chi2 + r0 * r0 * i00 + 2.0 * r0 * r1 * i01 + r1 * r1 * i11;
    if (res_out) { res_out[0] = r0; res_out[1] = r1; }
    if (sinv_out) { sinv_out[0] = i00; sinv_out[1] = i01; sinv_out[2] = i11; }
}

// ---- fit seed ------------------------------------------------------------
// Circle through the innermost, middle and outermost clusters (nominal row
// planes, uncorrected coordinates) gives q/pT and sin phi; tan lambda is the
// z difference over the arc between the two end clusters; (y, z) are those
// of the first cluster in fit order.  The seed is a pattern-recognition
// product and does not depend on the alignment corrections.
struct Seed {
    double x, p[5];
    int frame;
};

void local_to_frame(int from, double x, double y, int to, double& xo, double& yo) {
    const double a = sector_alpha(from), b = sector_alpha(to);
    const double X = x * std::cos(a) - y * std::sin(a);
    const double Y = x * std::sin(a) + y * std::cos(a);
    xo = X * std::cos(b) + Y * std::sin(b);
    yo = -X * std::sin(b) + Y * std::cos(b);
}

// hits in fit order (first = start of the fit)
template <class F>
Seed make_seed(const F* y, const F* z, const uint16_t* row, const int32_t* sec,
               const int32_t* hits, int n, bool first_is_outer, const orc_params& prm) {
    Seed sd;
    const int h0 = hits[0], hm = hits[n / 2], hl = hits[n - 1];
    sd.frame = sec[h0];
    sd.x = row_x(row[h0]);
    double px[3], py[3], pz[3];
    const int hh[3] = {h0, hm, hl};
    for (int i = 0; i < 3; ++i) {
        local_to_frame(sec[hh[i]], row_x(row[hh[i]]), (double)y[hh[i]], sd.frame, px[i], py[i]);
        pz[i] = (double)z[hh[i]];
    }
    // motion order: innermost q0 -> middle q1 -> outermost q2
    const int i0 = first_is_outer ? 2 : 0, i2 = first_is_outer ? 0 : 2;
    const double ax = px[1] - px[i0], ay = py[1] - py[i0];
    const double bx = px[i2] - px[1], by = py[i2] - py[1];
    const double cx = px[i2] - px[i0], cy = py[i2] - py[i0];
    const double la = std::sqrt(ax * ax + ay * ay), lb = std::sqrt(bx * bx + by * by);
    const double L = std::sqrt(cx * cx + cy * cy);
    const double cross = ax * by - ay * bx;
    double k = 0.0;
    if (la > 0 && lb > 0 && L > 0) k = -2.0 * cross / (la * lb * L);
    double hk = k * L * 0.5;
    hk = std::max(-0.999, std::min(0.999, hk));
    const double theta = std::atan2(cy, cx);
    const double half = std::asin(hk);
    const double phi = first_is_outer ? theta - half : theta + half;
    double s = std::sin(phi);
    s = std::max(-prm.seed_snp_max, std::min(prm.seed_snp_max, s));
    const double au = std::fabs(hk);
    const double arc = (au < 1e-9 || k == 0.0) ? L : 2.0 * std::asin(au) / std::fabs(k);
    const double t = arc > 0 ? (pz[i2] - pz[i0]) / arc : 0.0;
    double w = (prm.bz != 0.0) ? k / (KAPPA * prm.bz) : 0.0;
    w = std::max(-prm.seed_qpt_max, std::min(prm.seed_qpt_max, w));
    sd.p[0] = (double)y[h0];
    sd.p[1] = (double)z[h0];
    sd.p[2] = s;
    sd.p[3] = t;
    sd.p[4] = w;
    return sd;
}

// corrected cluster position (sector-local): p' = R(a,b,g) (x_r, y, z) + D,
// R = Rz(g) Ry(b) Rx(a)
template <class T>
void corrected(const T th[6], double xr, double y, double z, T& xo, T& yo, T& zo) {
    const T ca = cos(th[3]), sa = sin(th[3]);
    const T cb = cos(th[4]), sb = sin(th[4]);
    const T cg = cos(th[5]), sg = sin(th[5]);
    // Rx
    const T x1 = T(xr);
    const T y1 = ca * y - sa * z;
    const T z1 = sa * y + ca * z;
    // Ry
    const T x2 = cb * x1 + sb * z1;
    const T z2 = cb * z1 - sb * x1;
    // Rz
    xo = cg * x2 - sg * y1 + th[0];
    yo = sg * x2 + cg * y1 + th[1];
    zo = z2 + th[2];
}

// No displacement field: the corrected position is the aligned one.
struct NoDisp {
    std::nullptr_t operator()(int) const { return nullptr; }
};

// ---- NEXT-3: material in the pad-row planes --------------------------------
// The material of one plane acts on a track right after it crosses the
// plane: a multiple-scattering deflection (two independent projected angles
// of width theta0, the Highland formula for x/X0 = mat_x_x0 times the path
// factor 1/(cos phi cos lambda)) and the mean energy loss mat_eloss times
// the same factor.  A fit that moves against the motion (inward) undoes the
// plane it arrives at: the energy is restored, then the deflection's
// covariance is added, so the state is the one arriving at the plane.  A
// fit along the motion applies the plane after its update.  With the angles
// dphi = theta1 / cos(lambda), dlambda = theta2:
//   Q_ss = theta0^2 cos^2(phi) (1 + t^2),  Q_tt = theta0^2 (1 + t^2)^2,
//   Q_tw = theta0^2 (1 + t^2) w t,          Q_ww = theta0^2 w^2 t^2,
// and the energy change maps w' = w p / p' (p^2 = (1 + t^2) / w^2), whose
// Jacobian row d w'/d(t, w) transforms the covariance first.
// The energy change of one plane: w' and its derivatives d w'/d w and
// d w'/d t (the loss itself taken as fixed), and the momentum and energy
// arriving at the plane (before the loss).
template <class T>
struct ElossMap {
    T w2, dw_dw, dw_dt, p_arr, e_arr;
};
template <class T>
ElossMap<T> eloss_map(const T p[5], const orc_params& prm, bool undo) {
    const T s = p[2], t = p[3], w = p[4];
    const T c2 = 1.0 - s * s;
    const T tt = 1.0 + t * t;
    const T path = sqrt(tt / c2);                      // 1 / (cos phi cos lambda)
    const T pm = sqrt(tt) / (val(w) >= 0 ? w : -w);    // momentum before this step
    const double m2 = prm.mass * prm.mass;
    const T e = sqrt(pm * pm + m2);
    ElossMap<T> m{w, T(1.0), T(0.0), pm, e};
    if (prm.mat_eloss > 0.0) {
        const T de = path * prm.mat_eloss;
        const T e2 = undo ? e + de : e - de;
        const T p2 = sqrt(e2 * e2 - m2);
        const T r = e2 * pm * pm / (p2 * p2 * e);
        m.w2 = w * pm / p2;
        m.dw_dw = m.w2 / w * r;
        m.dw_dt = m.w2 * t / tt * (1.0 - r);
        if (undo) {
            m.p_arr = p2;
            m.e_arr = e2;
        }
    }
    return m;
}

template <class T>
void material_step(T p[5], T C[15], const orc_params& prm, bool undo) {
    if (prm.mat_x_x0 <= 0.0 && prm.mat_eloss <= 0.0) return;
    const ElossMap<T> m = eloss_map(p, prm, undo);
    if (prm.mat_eloss > 0.0) {
        // C' = J C J^T, J = identity except row 4 = (0, 0, 0, dw_dt, dw_dw)
        T row4[5];
        for (int i = 0; i < 5; ++i) row4[i] = m.dw_dt * C[sidx(3, i)] + m.dw_dw * C[sidx(4, i)];
        const T c44 = m.dw_dt * row4[3] + m.dw_dw * row4[4];
        for (int i = 0; i < 4; ++i) C[sidx(4, i)] = row4[i];
        C[sidx(4, 4)] = c44;
        p[4] = m.w2;
    }
    if (prm.mat_x_x0 > 0.0) {
        const T s = p[2], t = p[3], wn = p[4];
        const T c2 = 1.0 - s * s;
        const T tt = 1.0 + t * t;
        const T xx0 = sqrt(tt / c2) * prm.mat_x_x0;
        const T beta = m.p_arr / m.e_arr;
        // Highland: 13.6 MeV / (beta c p) sqrt(x/X0) (1 + 0.038 ln(x/X0))
        const T lnx = T(std::log(val(xx0)));
        const T th0 = 0.0136 / (beta * m.p_arr) * sqrt(xx0) * (1.0 + 0.038 * lnx);
        const T q = th0 * th0;
        C[sidx(2, 2)] += q * c2 * tt;
        C[sidx(3, 3)] += q * tt * tt;
        C[sidx(3, 4)] += q * tt * wn * t;
        C[sidx(4, 4)] += q * wn * wn * t * t;
    }
}

// What a recording fit hands out per hit j: the state predicted at the hit's
// plane (after the transport and the material, before the update), the
// filtered state after the update, and the Jacobian of the prediction with
// respect to the previous filtered state (identity for j = 0).
struct NoRec {
    template <class T> void operator()(int, const T*, const T*, const T*, const T*, const T*) const {}
};

// One full fit.  th(i) returns the 6 correction parameters of cluster hit i's
// sector as T (or null alignment); disp(j) returns the displacement (x, y, z)
// added to the j-th cluster of the list after the alignment (or null).
// Returns false when a transport fails.
template <class T, class ThFn, class DispFn = NoDisp, class RecFn = NoRec>
bool kf_fit(const float* y, const float* z, const uint16_t* row, const int32_t* sec,
            const int32_t* hits, int n, bool first_is_outer, const orc_params& prm,
            ThFn th, T p[5], T C[15], T& chi2, T* xlast = nullptr, DispFn disp = DispFn(),
            RecFn rec = RecFn()) {
    constexpr bool REC = !std::is_same<RecFn, NoRec>::value;
    const Seed sd = make_seed(y, z, row, sec, hits, n, first_is_outer, prm);
    for (int i = 0; i < 5; ++i) p[i] = T(sd.p[i]);
    for (int i = 0; i < 15; ++i) C[i] = T(0.0);
    for (int i = 0; i < 5; ++i) C[sidx(i, i)] = T(prm.prior[i]);
    T x = T(sd.x);
    int frame = sd.frame;
    chi2 = T(0.0);
    T J[25], dX[5];
    const bool mat = prm.mat_x_x0 > 0.0 || prm.mat_eloss > 0.0;
    // composite Jacobian of one prediction (recording fits only)
    T F[25];
    auto f_reset = [&]() {
        for (int i = 0; i < 25; ++i) F[i] = T(i % 6 == 0 ? 1.0 : 0.0);
    };
    auto f_chain = [&](const T* Js) {  // F <- Js F
        T tmp[25];
        for (int i = 0; i < 5; ++i)
            for (int k = 0; k < 5; ++k) {
                T acc(0.0);
                for (int l = 0; l < 5; ++l) acc += Js[i * 5 + l] * F[l * 5 + k];
                tmp[i * 5 + k] = acc;
            }
        for (int i = 0; i < 25; ++i) F[i] = tmp[i];
    };
    // material with its state Jacobian for the record (material_step moves
    // the covariance itself; the recorded F needs the w row)
    auto mat_step = [&](bool undo) {
        if constexpr (REC) {
            if (prm.mat_eloss > 0.0) {
                const ElossMap<T> m = eloss_map(p, prm, undo);
                T Jm[25];
                for (int i = 0; i < 25; ++i) Jm[i] = T(i % 6 == 0 ? 1.0 : 0.0);
                Jm[4 * 5 + 3] = m.dw_dt;
                Jm[4 * 5 + 4] = m.dw_dw;
                f_chain(Jm);
            }
        }
        material_step(p, C, prm, undo);
    };
    for (int j = 0; j < n; ++j) {
        const int h = hits[j];
        T xc, yc, zc;
        const T* t6 = th(h);
        if (t6) {
            corrected<T>(t6, row_x(row[h]), (double)y[h], (double)z[h], xc, yc, zc);
        } else {
            xc = T(row_x(row[h]));
            yc = T((double)y[h]);
            zc = T((double)z[h]);
        }
        const T* d3 = disp(j);
        if (d3) {
            xc = xc + d3[0];
            yc = yc + d3[1];
            zc = zc + d3[2];
        }
        if constexpr (REC) f_reset();
        if (mat && j > 0) {
            const int hp = hits[j - 1];
            // along the motion: the previous plane acts after its update
            if (!first_is_outer) mat_step(false);
            // the planes crossed between the two hits (same sector)
            if (sec[hp] == sec[h]) {
                const int r0 = row[hp], r1 = row[h], step = r1 > r0 ? 1 : -1;
                for (int r = r0 + step; r != r1; r += step) {
                    if (!move_state(x, p, frame, T(row_x(r)), sec[h], J, dX, prm)) return false;
                    cov_transform(C, J);
                    if constexpr (REC) f_chain(J);
                    mat_step(first_is_outer);
                }
            }
        }
        if (!move_state(x, p, frame, xc, sec[h], J, dX, prm)) return false;
        cov_transform(C, J);
        if constexpr (REC) f_chain(J);
        // against the motion: undo the plane the track arrives at
        if (mat && j > 0 && first_is_outer) mat_step(true);
        T pp[5], Cp[15];
        if constexpr (REC) {
            for (int i = 0; i < 5; ++i) pp[i] = p[i];
            for (int i = 0; i < 15; ++i) Cp[i] = C[i];
        }
        kf_update(p, C, yc, zc, prm.sigma_y2, prm.sigma_z2, chi2);
        if constexpr (REC) rec(j, pp, Cp, F, p, C);
    }
    if (xlast) *xlast = x;
    return true;
}

// ---- S2 neighbour decision in FP32 ----------------------------------------
// Gap pairs in the order of increasing g_d + g_u, then increasing g_u.
struct Gap { int d, u; };
std::vector<Gap> gap_order(int max_gap) {
    std::vector<Gap> g;
    for (int sum = 2; sum <= 2 * max_gap; ++sum)
        for (int gu = 1; gu <= max_gap; ++gu) {
            const int gd = sum - gu;
            if (gd >= 1 && gd <= max_gap) g.push_back({gd, gu});
        }
    return g;
}

// D^2 of the triplet (d, c, u): straight-line interpolation of c from d and
// u, residuals normalised by the variance of (c - interpolation).
// Evaluated in FP32, one rounding per operation (compiled without
// contraction).
float triplet_d2(float xd, float yd, float zd, float xc, float yc, float zc,
                 float xu, float yu, float zu, float sy2, float sz2) {
    const float a = (xc - xd) / (xu - xd);
    const float yh = yd + a * (yu - yd);
    const float zh = zd + a * (zu - zd);
    const float ry = yc - yh;
    const float rz = zc - zh;
    const float b = 1.0f - a;
    const float f = (1.0f + a * a) + b * b;
    return (ry * ry) / (sy2 * f) + (rz * rz) / (sz2 * f);
}

bool in_window(float xa, float ya, float za, float xb, float yb, float zb, float wy, float wz) {
    const float dx = std::fabs(xb - xa);
    return std::fabs(yb - ya) <= wy * dx && std::fabs(zb - za) <= wz * dx;
}

// The same two tests in FP64 (the diagnostic mode that measures how many
// neighbour decisions FP32 rounding changes): row planes and window slopes
// in double, coordinates widened from their FP32 storage.
double triplet_d2_f64(double xd, double yd, double zd, double xc, double yc, double zc,
                      double xu, double yu, double zu, double sy2, double sz2) {
    const double a = (xc - xd) / (xu - xd);
    const double ry = yc - (yd + a * (yu - yd));
    const double rz = zc - (zd + a * (zu - zd));
    const double b = 1.0 - a;
    const double f = (1.0 + a * a) + b * b;
    return (ry * ry) / (sy2 * f) + (rz * rz) / (sz2 * f);
}

bool in_window_f64(double xa, double ya, double za, double xb, double yb, double zb, double wy, double wz) {
    const double dx = std::fabs(xb - xa);
    return std::fabs(yb - ya) <= wy * dx && std::fabs(zb - za) <= wz * dx;
}

struct Segment {
    int event, sector;
    std::vector<int32_t> hits;  // outermost first (input-order indices)
    int32_t canon;              // smallest input index
    bool ok_in = false, ok_out = false;
    double p_in[5], c_in[15];   // inward fit: state at the innermost cluster
    double p_out[5], c_out[15]; // outward fit: state at the outermost cluster
    int row_min, row_max;
};

// S1-S3 for one (event, sector) group.
void group_ca(const float* y, const float* z, const uint16_t* row, int64_t beg, int64_t end,
              int event, int sector, const orc_params& prm, std::vector<Segment>& segs,
              std::vector<std::vector<int32_t>>& rows, orc_diag* diag) {
    const int64_t n = end - beg;
    rows.assign(NROW, std::vector<int32_t>());
    if (n <= 0) return;
    // S1: rows, canonical order = input order
    for (int64_t i = beg; i < end; ++i) rows[row[i]].push_back((int32_t)i);
    std::vector<int32_t> cdn(n, -1), cup(n, -1), ldn(n, -1), lup(n, -1);
    std::vector<double> d2v(n, std::numeric_limits<double>::infinity());
    std::vector<double> d2n(n, std::numeric_limits<double>::infinity());
    const std::vector<Gap> gaps = gap_order(prm.max_gap);
    const bool f64 = prm.s2_fp64 != 0;
    // admissibility and D^2 of the triplet (d, c, u): FP32 with one rounding
    // per operation (the rule), or FP64 (diagnostic); an FP32 D^2 is exact
    // in double, so the comparisons below decide alike in both modes
    auto admissible = [&](int rc, int64_t c, int rb, int32_t b) {
        if (f64)
            return in_window_f64(row_x(rc), y[c], z[c], row_x(rb), y[b], z[b], prm.win_y, prm.win_z);
        return in_window(row_xf(rc), y[c], z[c], row_xf(rb), y[b], z[b], prm.win_y, prm.win_z);
    };
    auto triplet = [&](int rd, int32_t d, int rc, int64_t c, int ru, int32_t u) -> double {
        if (f64)
            return triplet_d2_f64(row_x(rd), y[d], z[d], row_x(rc), y[c], z[c], row_x(ru), y[u], z[u],
                                  (double)prm.sigma_y2, (double)prm.sigma_z2);
        return triplet_d2(row_xf(rd), y[d], z[d], row_xf(rc), y[c], z[c], row_xf(ru), y[u], z[u],
                          prm.sigma_y2, prm.sigma_z2);
    };
    // S2a: each cluster chooses its best (down, up) pair
    for (int64_t c = beg; c < end; ++c) {
        const int r = row[c];
        double best_seen = std::numeric_limits<double>::infinity();
        for (const Gap& gp : gaps) {
            const int rd = r - gp.d, ru = r + gp.u;
            if (rd < 0 || ru >= NROW) continue;
            bool found = false;
            double bd2 = 0, second = std::numeric_limits<double>::infinity();
            int32_t bd = -1, bu = -1;
            for (int32_t d : rows[rd]) {
                if (!admissible(r, c, rd, d)) continue;
                for (int32_t u : rows[ru]) {
                    if (!admissible(r, c, ru, u)) continue;
                    const double d2 = triplet(rd, d, r, c, ru, u);
                    if (d2 < best_seen) best_seen = d2;
                    if (!(d2 <= (double)prm.chi2_link)) {
                        if (found && d2 < second) second = d2;
                        continue;
                    }
                    const bool better = !found || d2 < bd2 || (d2 == bd2 && (u < bu || (u == bu && d < bd)));
                    if (better) {
                        if (found) second = std::min(second, bd2);
                        found = true;
                        bd2 = d2; bd = d; bu = u;
                    } else {
                        second = std::min(second, d2);
                    }
                }
            }
            if (found) {
                cdn[c - beg] = bd;
                cup[c - beg] = bu;
                d2v[c - beg] = bd2;
                d2n[c - beg] = second;
                break;
            }
        }
        if (cdn[c - beg] < 0) d2v[c - beg] = best_seen;
    }
    // S2b: endpoints without a triplet of their own accept the best claimant
    // (smallest D^2, then smallest canonical id)
    std::vector<int32_t> claim_up(n, -1), claim_dn(n, -1);
    auto better_claim = [&](int32_t a, int32_t b) {  // a better than b?
        if (b < 0) return true;
        const double da = d2v[a - beg], db = d2v[b - beg];
        return da < db || (da == db && a < b);
    };
    for (int64_t c = beg; c < end; ++c) {
        const int32_t u = cup[c - beg], d = cdn[c - beg];
        if (u >= 0 && cdn[u - beg] < 0 && better_claim((int32_t)c, claim_up[u - beg])) claim_up[u - beg] = (int32_t)c;
        if (d >= 0 && cup[d - beg] < 0 && better_claim((int32_t)c, claim_dn[d - beg])) claim_dn[d - beg] = (int32_t)c;
    }
    // S2c: links: mutual choices, or claims of endpoints
    for (int64_t c = beg; c < end; ++c) {
        const int32_t u = cup[c - beg], d = cdn[c - beg];
        if (u >= 0) {
            if (cdn[u - beg] == (int32_t)c || (cdn[u - beg] < 0 && claim_up[u - beg] == (int32_t)c)) {
                lup[c - beg] = u;
                ldn[u - beg] = (int32_t)c;
            }
        }
        if (d >= 0) {
            if (cup[d - beg] == (int32_t)c || (cup[d - beg] < 0 && claim_dn[d - beg] == (int32_t)c)) {
                ldn[c - beg] = d;
                lup[d - beg] = (int32_t)c;
            }
        }
    }
    if (diag) {
        for (int64_t c = beg; c < end; ++c) {
            if (diag->choice_dn) diag->choice_dn[c] = cdn[c - beg];
            if (diag->choice_up) diag->choice_up[c] = cup[c - beg];
            if (diag->d2) diag->d2[c] = (float)d2v[c - beg];
            if (diag->d2_next) diag->d2_next[c] = (float)d2n[c - beg];
            if (diag->link_dn) diag->link_dn[c] = ldn[c - beg];
            if (diag->link_up) diag->link_up[c] = lup[c - beg];
        }
    }
    // S3: chains from clusters with no down link and an up link
    for (int64_t c = beg; c < end; ++c) {
        if (ldn[c - beg] >= 0 || lup[c - beg] < 0) continue;
        std::vector<int32_t> chain;
        int32_t cur = (int32_t)c;
        while (cur >= 0) {
            chain.push_back(cur);
            cur = lup[cur - beg];
        }
        if ((int)chain.size() < prm.n_seg) continue;
        Segment s;
        s.event = event;
        s.sector = sector;
        s.hits.assign(chain.rbegin(), chain.rend());  // outermost first
        s.canon = *std::min_element(chain.begin(), chain.end());
        s.row_min = row[chain.front()];
        s.row_max = row[chain.back()];
        segs.push_back(std::move(s));
    }
}

// 5x5 SPD solve by Cholesky; returns false when not positive definite.
bool chi2_5(const double dp[5], const double M[15], double& out) {
    double Lm[5][5] = {};
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = M[sidx(i, j)];
            for (int l = 0; l < j; ++l) s -= Lm[i][l] * Lm[j][l];
            if (i == j) {
                if (!(s > 0)) return false;
                Lm[i][i] = std::sqrt(s);
            } else {
                Lm[i][j] = s / Lm[j][j];
            }
        }
    double v[5];
    for (int i = 0; i < 5; ++i) {
        double s = dp[i];
        for (int l = 0; l < i; ++l) s -= Lm[i][l] * v[l];
        v[i] = s / Lm[i][i];
    }
    out = 0;
    for (int i = 0; i < 5; ++i) out += v[i] * v[i];
    return true;
}

// Moves a filtered state (p, C at plane x of `sector`) to the plane of row r
// of the same sector: helix transport with the covariance J C J^T.  Returns
// false (state untouched) when the transport fails.
bool move_to_row(double& x, double p[5], double C[15], int sector, int r, const orc_params& prm) {
    double J[25], dX[5];
    int frame = sector;
    if (!move_state<double>(x, p, frame, row_x(r), sector, J, dX, prm)) return false;
    cov_transform(C, J);
    return true;
}

// S3b: Kalman-guided extension.  From the state at plane x (frame =
// sector), visit rows r_start, r_start+dir, ... ; in each row take the
// cluster of the group with the smallest predicted-residual chi2
// r^T (C_yz + R)^-1 r (ties: smaller canonical id) if it is <= chi2_ext and
// update with it; stop after ext_max_miss consecutive rows without one, at
// the last row, when the transport fails, or when the prediction leaves the
// sector's acceptance.
// A decision of the extension (a row's choice) and its relative margin, for
// tracing disagreements to near-ties: (cluster, margin).
using Decisions = std::vector<std::pair<int32_t, double>>;

inline double rel_gap(double u, double v) {
    const double m = std::max(std::fabs(u), std::fabs(v));
    return m > 0 ? std::fabs(u - v) / m : 0.0;
}

void extend_tracklet(const float* y, const float* z, const std::vector<std::vector<int32_t>>& rows,
                     int sector, double& x, double p[5], double C[15], int r_start, int dir,
                     const orc_params& prm, std::vector<int32_t>& added, Decisions* dec = nullptr,
                     double* stop_margin = nullptr) {
    int misses = 0;
    for (int r = r_start; r >= 0 && r < NROW; r += dir) {
        double J[25], dX[5];
        int frame = sector;
        if (stop_margin) {  // diagnostics: the transport's |sin phi| limit
            const double s2 = p[2] - KAPPA * prm.bz * p[4] * (row_x(r) - x);
            *stop_margin = std::min(*stop_margin, rel_gap(std::fabs(s2), prm.snp_max));
        }
        if (!move_state<double>(x, p, frame, row_x(r), sector, J, dX, prm)) break;
        // the state and its covariance move together, so that the state the
        // extension ends with is consistent at its plane
        cov_transform(C, J);
        // the track has left the sector when its prediction is outside the
        // row's acceptance |y| <= x tan(10 deg)
        if (stop_margin) *stop_margin = std::min(*stop_margin, rel_gap(std::fabs(p[0]), row_x(r) * TAN_HALF));
        if (std::fabs(p[0]) > row_x(r) * TAN_HALF) break;
        const double S00 = C[sidx(0, 0)] + prm.sigma_y2, S01 = C[sidx(0, 1)], S11 = C[sidx(1, 1)] + prm.sigma_z2;
        const double det = S00 * S11 - S01 * S01;
        int32_t best = -1;
        double bchi = 0;
        // diagnostics only: the two smallest chi2 of the row, cut or not
        int32_t d1 = -1, d2 = -1;
        double c1 = 0, c2 = 0;
        for (int32_t c : rows[r]) {
            const double r0 = (double)y[c] - p[0], r1 = (double)z[c] - p[1];
            const double chi = (r0 * r0 * S11 - 2.0 * r0 * r1 * S01 + r1 * r1 * S00) / det;
            if (dec) {
                if (d1 < 0 || chi < c1) {
                    d2 = d1; c2 = c1; d1 = c; c1 = chi;
                } else if (d2 < 0 || chi < c2) {
                    d2 = c; c2 = chi;
                }
            }
            if (!(chi <= prm.chi2_ext)) continue;
            if (best < 0 || chi < bchi || (chi == bchi && c < best)) {
                best = c;
                bchi = chi;
            }
        }
        if (dec && d1 >= 0) {
            double m = rel_gap(c1, prm.chi2_ext);
            if (d2 >= 0) m = std::min(m, rel_gap(c1, c2));
            dec->push_back({d1, m});
            if (d2 >= 0) dec->push_back({d2, m});
        }
        if (best >= 0) {
            double chi2 = 0;
            kf_update(p, C, (double)y[best], (double)z[best], prm.sigma_y2, prm.sigma_z2, chi2);
            added.push_back(best);
            misses = 0;
        } else if (++misses >= prm.ext_max_miss) {
            break;
        }
    }
}

struct MergePair {
    double chi2;
    int a, b;  // segment indices: a inner, b outer
};

// S3b for one segment (hits outermost first): inward fit and inward
// extension; the final inward-filtered state, moved to the outermost hit
// row, starts the outward extension.  Without process noise that state
// carries every hit (the move is exact), so it stands for an outward fit
// over all of them; the outward fit itself is used only when the inward fit
// or that move fails.  Returns the tracklet's hits, outermost first.
std::vector<int32_t> build_tracklet(const float* y, const float* z, const uint16_t* row,
                                    const int32_t* sec, const std::vector<std::vector<int32_t>>& rows,
                                    const Segment& sg, const orc_params& prm, Decisions* dec = nullptr) {
    auto no_align = [](int) -> const double* { return nullptr; };
    std::vector<int32_t> H = sg.hits;
    double p[5], C[15], chi2, x;
    bool have_out = false;
    // diagnostics: the smallest margin of the decisions that end the two
    // extensions (acceptance edge, transport limit), charged to every hit
    double stop = std::numeric_limits<double>::infinity();
    double* stop_p = dec ? &stop : nullptr;
    if (kf_fit<double>(y, z, row, sec, H.data(), (int)H.size(), true, prm, no_align, p, C, chi2, &x)) {
        std::vector<int32_t> add;
        extend_tracklet(y, z, rows, sg.sector, x, p, C, row[H.back()] - 1, -1, prm, add, dec, stop_p);
        H.insert(H.end(), add.begin(), add.end());
        have_out = move_to_row(x, p, C, sg.sector, row[H.front()], prm);
    }
    if (!have_out) {
        std::vector<int32_t> rev(H.rbegin(), H.rend());
        have_out = kf_fit<double>(y, z, row, sec, rev.data(), (int)rev.size(), false, prm, no_align, p, C,
                                  chi2, &x);
    }
    if (have_out) {
        std::vector<int32_t> add;
        extend_tracklet(y, z, rows, sg.sector, x, p, C, row[H.front()] + 1, +1, prm, add, dec, stop_p);
        std::vector<int32_t> H2(add.rbegin(), add.rend());
        H2.insert(H2.end(), H.begin(), H.end());
        H.swap(H2);
    }
    if (dec && stop < std::numeric_limits<double>::infinity())
        for (int32_t h : H) dec->push_back({h, stop});
    return H;
}

// S5 on a tracklet (hits outermost first): inward fit, state at the
// innermost hit; the state at the outermost hit is that state moved there
// (the outward fit only when the inward fit or the move fails).
void fit_segment(const float* y, const float* z, const uint16_t* row, const int32_t* sec, Segment& s,
                 const orc_params& prm) {
    auto no_align = [](int) -> const double* { return nullptr; };
    double chi2, x;
    s.ok_in = kf_fit<double>(y, z, row, sec, s.hits.data(), (int)s.hits.size(), true, prm, no_align, s.p_in,
                             s.c_in, chi2, &x);
    s.ok_out = false;
    if (s.ok_in) {
        for (int k = 0; k < 5; ++k) s.p_out[k] = s.p_in[k];
        for (int k = 0; k < 15; ++k) s.c_out[k] = s.c_in[k];
        s.ok_out = move_to_row(x, s.p_out, s.c_out, s.sector, row[s.hits.front()], prm);
    }
    if (!s.ok_out) {
        std::vector<int32_t> rev(s.hits.rbegin(), s.hits.rend());
        s.ok_out = kf_fit<double>(y, z, row, sec, rev.data(), (int)rev.size(), false, prm, no_align, s.p_out,
                                  s.c_out, chi2);
    }
}

// S4 compatibility of an inner segment A and an outer segment B: A's state
// at its outermost cluster, moved to B's innermost plane (rotating on a
// sector change), against B's state there:
//   chi2_5 = dp^T (C_A + C_B)^-1 dp,  dp = p_B - p_A.
bool merge_chi2_value(const Segment& A, const Segment& B, const orc_params& prm, double& chi2) {
    if (!A.ok_out || !B.ok_in) return false;
    double p[5], C[15], J[25], dX[5];
    std::memcpy(p, A.p_out, sizeof p);
    std::memcpy(C, A.c_out, sizeof C);
    double x = row_x(A.row_max);
    int frame = A.sector;
    if (!move_state<double>(x, p, frame, row_x(B.row_min), B.sector, J, dX, prm)) return false;
    cov_transform(C, J);
    double dp[5], M[15];
    for (int i = 0; i < 5; ++i) dp[i] = B.p_in[i] - p[i];
    for (int i = 0; i < 15; ++i) M[i] = C[i] + B.c_in[i];
    return chi2_5(dp, M, chi2);
}

// S4 candidate test: A's outward-fit state at its outermost cluster is moved
// to B's innermost plane and compared with B's inward-fit state there.
bool merge_chi2(const Segment& A, const Segment& B, const float* z, const orc_params& prm,
                double& chi2, bool* evaluated = nullptr) {
    if (evaluated) *evaluated = false;
    if (A.event != B.event) return false;
    if ((A.sector < NPHI) != (B.sector < NPHI)) return false;
    const int dphi = ((B.sector % NPHI) - (A.sector % NPHI) + NPHI) % NPHI;
    if (!(dphi == 0 || dphi == 1 || dphi == NPHI - 1)) return false;
    // rows: B starts at or above A's last row; across a sector boundary the
    // two row ranges may overlap by up to merge_max_overlap rows (a track
    // grazing the boundary crosses the row planes of both sectors)
    const int gap = B.row_min - A.row_max;
    const int min_gap = (dphi == 0) ? 0 : -prm.merge_max_overlap;
    if (gap < min_gap || gap > prm.merge_max_row_gap) return false;
    // z gate in FP32
    const float zb = z[B.hits.back()], za = z[A.hits.front()];
    const float dxr = std::fabs(row_xf(B.row_min) - row_xf(A.row_max));
    if (!(std::fabs(zb - za) <= prm.merge_z_slope * dxr + prm.merge_z_margin)) return false;
    if (!merge_chi2_value(A, B, prm, chi2)) return false;
    if (evaluated) *evaluated = true;
    return chi2 <= prm.chi2_merge;
}

}  // namespace

extern "C" {

void orc_default_params(orc_params* p) {
    p->win_y = 3.0f;
    p->win_z = 3.5f;
    p->chi2_link = 16.0f;
    p->sigma_y2 = 0.01f;
    p->sigma_z2 = 0.0225f;
    p->max_gap = 3;
    p->n_seg = 5;
    p->n_min = 10;
    p->merge_max_row_gap = 24;
    p->merge_max_overlap = 8;
    p->merge_z_slope = 3.5f;
    p->merge_z_margin = 2.0f;
    p->chi2_merge = 30.0;
    p->chi2_ext = 16.0;
    p->ext_max_miss = 3;
    p->bz = 0.5;
    p->prior[0] = 4.0;
    p->prior[1] = 4.0;
    p->prior[2] = 0.25;
    p->prior[3] = 0.25;
    p->prior[4] = 25.0;
    p->seed_snp_max = 0.99;
    p->seed_qpt_max = 5.0;
    p->snp_max = 0.999;
    p->s2_fp64 = 0;
    p->mat_x_x0 = 0.0;
    p->mat_eloss = 0.0;
    p->mass = 0.13957;
}

void orc_set_threads(int n) { g_threads = n; }
int orc_get_threads(void) {
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

int64_t orc_find_tracks(const float* y, const float* z, const uint16_t* row, int64_t n,
                        const int64_t* off, int32_t n_events, const orc_params* prm_,
                        int32_t* track_of_cluster, int32_t* trk_off, int32_t* trk_hits,
                        orc_diag* diag) {
    const orc_params& prm = *prm_;
    const int G = n_events * NSEC;
    if (off[0] != 0 || off[G] != n) return -1;
    for (int g = 0; g < G; ++g)
        if (off[g + 1] < off[g]) return -1;
    for (int64_t i = 0; i < n; ++i)
        if (row[i] >= NROW || !std::isfinite(y[i]) || !std::isfinite(z[i])) return -1;
    const int nt = orc_get_threads();
    // S1-S3 per group
    std::vector<std::vector<Segment>> per_group(G);
    std::vector<std::vector<std::vector<int32_t>>> grp_rows(G);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int g = 0; g < G; ++g)
        group_ca(y, z, row, off[g], off[g + 1], g / NSEC, g % NSEC, prm, per_group[g], grp_rows[g], diag);
    std::vector<Segment> seeds;
    for (int g = 0; g < G; ++g)
        for (auto& s : per_group[g]) seeds.push_back(std::move(s));
    std::sort(seeds.begin(), seeds.end(), [](const Segment& a, const Segment& b) { return a.canon < b.canon; });
    const int S0 = (int)seeds.size();
    // sector of every cluster
    std::vector<int32_t> sec(n);
    for (int g = 0; g < G; ++g)
        for (int64_t i = off[g]; i < off[g + 1]; ++i) sec[i] = g % NSEC;
    // S3b: each segment seeds a tracklet (build_tracklet)
    std::vector<std::vector<int32_t>> tl_hits(S0);
    const bool want_ext = diag && diag->ext_margin;
    std::vector<Decisions> tl_dec(want_ext ? S0 : 0);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int i = 0; i < S0; ++i) {
        const Segment& sg = seeds[i];
        tl_hits[i] = build_tracklet(y, z, row, sec.data(), grp_rows[sg.event * NSEC + sg.sector], sg, prm,
                                    want_ext ? &tl_dec[i] : nullptr);
    }
    if (want_ext) {
        for (int64_t i = 0; i < n; ++i) diag->ext_margin[i] = std::numeric_limits<double>::infinity();
        for (const Decisions& d : tl_dec)
            for (const auto& e : d) diag->ext_margin[e.first] = std::min(diag->ext_margin[e.first], e.second);
    }
    // S3c: every cluster belongs to the best tracklet containing it: more
    // clusters first, then the smaller canonical id of the seed segment.
    // A tracklet keeps the clusters it owns if they are >= n_seg.
    std::vector<int64_t> owner(n, std::numeric_limits<int64_t>::max());
    auto tl_key = [&](int i) { return ((int64_t)(NROW * 4 - (int)tl_hits[i].size()) << 32) | (int64_t)seeds[i].canon; };
    for (int i = 0; i < S0; ++i) {
        const int64_t k = tl_key(i);
        for (int32_t h : tl_hits[i]) owner[h] = std::min(owner[h], k);
    }
    std::vector<Segment> segs;
    for (int i = 0; i < S0; ++i) {
        const int64_t k = tl_key(i);
        Segment t;
        t.event = seeds[i].event;
        t.sector = seeds[i].sector;
        for (int32_t h : tl_hits[i])
            if (owner[h] == k) t.hits.push_back(h);
        if ((int)t.hits.size() < prm.n_seg) continue;
        t.canon = *std::min_element(t.hits.begin(), t.hits.end());
        t.row_min = row[t.hits.back()];
        t.row_max = row[t.hits.front()];
        segs.push_back(std::move(t));
    }
    std::sort(segs.begin(), segs.end(), [](const Segment& a, const Segment& b) { return a.canon < b.canon; });
    const int S = (int)segs.size();
    // S5 on tracklets: inward fit (state at the innermost hit); the state at
    // the outermost hit is that state moved there (the outward fit only when
    // the inward fit or the move fails)
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int i = 0; i < S; ++i) {
        fit_segment(y, z, row, sec.data(), segs[i], prm);
    }
    // S4 candidates
    std::vector<std::vector<MergePair>> cand_b(S);
    // pairs whose chi2 was evaluated and found above the cut (diagnostics)
    std::vector<std::vector<MergePair>> rej_b(diag ? S : 0);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int b = 0; b < S; ++b)
        for (int a = 0; a < S; ++a) {
            if (a == b) continue;
            double c2;
            bool evaluated;
            if (merge_chi2(segs[a], segs[b], z, prm, c2, &evaluated)) cand_b[b].push_back({c2, a, b});
            else if (diag && evaluated) rej_b[b].push_back({c2, a, b});
        }
    std::vector<MergePair> cand;
    for (auto& v : cand_b)
        for (auto& m : v) cand.push_back(m);
    // greedy: ascending chi2, ties by canonical ids of A then B
    std::sort(cand.begin(), cand.end(), [&](const MergePair& p, const MergePair& q) {
        if (p.chi2 != q.chi2) return p.chi2 < q.chi2;
        if (segs[p.a].canon != segs[q.a].canon) return segs[p.a].canon < segs[q.a].canon;
        return segs[p.b].canon < segs[q.b].canon;
    });
    std::vector<int> next(S, -1), prev(S, -1);
    for (const MergePair& m : cand) {
        if (next[m.a] < 0 && prev[m.b] < 0) {
            next[m.a] = m.b;
            prev[m.b] = m.a;
        }
    }
    // decision margins per segment (for tracing disagreements)
    std::vector<double> margin(S, std::numeric_limits<double>::infinity());
    {
        std::vector<std::vector<double>> side_a(S), side_b(S);
        for (const MergePair& m : cand) {
            side_a[m.a].push_back(m.chi2);
            side_b[m.b].push_back(m.chi2);
        }
        auto rel = [](double u, double v) { return std::fabs(u - v) / std::max(std::fabs(u), std::fabs(v)); };
        for (const MergePair& m : cand) {
            double mg = rel(m.chi2, prm.chi2_merge);
            for (double o : side_a[m.a]) if (o != m.chi2) mg = std::min(mg, rel(o, m.chi2));
            for (double o : side_b[m.b]) if (o != m.chi2) mg = std::min(mg, rel(o, m.chi2));
            margin[m.a] = std::min(margin[m.a], mg);
            margin[m.b] = std::min(margin[m.b], mg);
        }
        // a pair refused by the cut is a decision too
        for (const auto& v : rej_b)
            for (const MergePair& m : v) {
                const double mg = rel(m.chi2, prm.chi2_merge);
                margin[m.a] = std::min(margin[m.a], mg);
                margin[m.b] = std::min(margin[m.b], mg);
            }
    }
    // tracks: chains of merged segments, hits outermost first
    struct Track { int32_t canon; std::vector<int32_t> hits; };
    std::vector<Track> tracks;
    for (int s0 = 0; s0 < S; ++s0) {
        if (next[s0] >= 0) continue;  // start from the outermost segment
        Track t;
        t.canon = std::numeric_limits<int32_t>::max();
        for (int s = s0; s >= 0; s = prev[s]) {
            for (int32_t h : segs[s].hits) t.hits.push_back(h);
            t.canon = std::min(t.canon, segs[s].canon);
        }
        if ((int)t.hits.size() >= prm.n_min) tracks.push_back(std::move(t));
    }
    std::sort(tracks.begin(), tracks.end(), [](const Track& a, const Track& b) { return a.canon < b.canon; });
    for (int64_t i = 0; i < n; ++i) track_of_cluster[i] = -1;
    trk_off[0] = 0;
    for (size_t t = 0; t < tracks.size(); ++t) {
        int32_t o = trk_off[t];
        for (int32_t h : tracks[t].hits) {
            trk_hits[o++] = h;
            track_of_cluster[h] = (int32_t)t;
        }
        trk_off[t + 1] = o;
    }
    if (diag) {
        if (diag->seg_of)
            for (int64_t i = 0; i < n; ++i) diag->seg_of[i] = -1;
        if (diag->merge_margin)
            for (int64_t i = 0; i < n; ++i) diag->merge_margin[i] = std::numeric_limits<double>::infinity();
        for (int s = 0; s < S; ++s)
            for (int32_t h : segs[s].hits) {
                if (diag->seg_of) diag->seg_of[h] = s;
                if (diag->merge_margin) diag->merge_margin[h] = margin[s];
            }
    }
    return (int64_t)tracks.size();
}

static int fit_common(const float* y, const float* z, const uint16_t* row, const int32_t* sec,
                      const int32_t* trk_off, const int32_t* trk_hits, int32_t T,
                      const double* align, const orc_params* prm, int reverse, double* params,
                      double* cov, double* chi2o, int32_t* ndf) {
    const int nt = orc_get_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int t = 0; t < T; ++t) {
        const int n = trk_off[t + 1] - trk_off[t];
        std::vector<int32_t> hits(trk_hits + trk_off[t], trk_hits + trk_off[t + 1]);
        if (reverse) std::reverse(hits.begin(), hits.end());
        double p[5], C[15], chi2 = 0;
        bool ok = n >= 3;
        if (ok) {
            auto th = [&](int h) -> const double* { return align ? align + 6 * sec[h] : nullptr; };
            ok = kf_fit<double>(y, z, row, sec, hits.data(), n, !reverse, *prm, th, p, C, chi2);
        }
        if (ok) {
            for (int i = 0; i < 5; ++i) params[t * 5 + i] = p[i];
            for (int i = 0; i < 15; ++i) cov[t * 15 + i] = C[i];
            chi2o[t] = chi2;
            ndf[t] = 2 * n - 5;
        } else {
            for (int i = 0; i < 5; ++i) params[t * 5 + i] = 0;
            for (int i = 0; i < 15; ++i) cov[t * 15 + i] = 0;
            chi2o[t] = 0;
            ndf[t] = -1;
        }
    }
    return 0;
}

int orc_fit_tracks(const float* y, const float* z, const uint16_t* row, const int32_t* sec,
                   const int32_t* trk_off, const int32_t* trk_hits, int32_t T, const double* align,
                   const orc_params* prm, double* params, double* cov, double* chi2, int32_t* ndf) {
    return fit_common(y, z, row, sec, trk_off, trk_hits, T, align, prm, 0, params, cov, chi2, ndf);
}

int orc_fit_tracks_dir(const float* y, const float* z, const uint16_t* row, const int32_t* sec,
                       const int32_t* trk_off, const int32_t* trk_hits, int32_t T,
                       const double* align, const orc_params* prm, int reverse, double* params,
                       double* cov, double* chi2, int32_t* ndf) {
    return fit_common(y, z, row, sec, trk_off, trk_hits, T, align, prm, reverse, params, cov, chi2, ndf);
}

// Per track, the touched sectors (at most 24/6 = 4 per pass; more sectors
// are handled in further passes) carry dual parts for their 6 parameters.
constexpr int ND = 24;
using D24 = Dual<ND>;

int orc_fit_adjoint(const float* y, const float* z, const uint16_t* row, const int32_t* sec,
                    const int32_t* trk_off, const int32_t* trk_hits, int32_t T, const double* align,
                    const orc_params* prm, double* chi2_total, double* grad) {
    const int nt = orc_get_threads();
    std::vector<double> tchi2(T, 0.0);
    std::vector<std::vector<double>> tgrad(grad ? T : 0);
    static const double zero6[6] = {0, 0, 0, 0, 0, 0};
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int t = 0; t < T; ++t) {
        const int n = trk_off[t + 1] - trk_off[t];
        const int32_t* hits = trk_hits + trk_off[t];
        if (n < 3) continue;
        if (!grad) {
            double p[5], C[15], chi2;
            auto th = [&](int h) -> const double* { return align ? align + 6 * sec[h] : zero6; };
            if (kf_fit<double>(y, z, row, sec, hits, n, true, *prm, th, p, C, chi2)) tchi2[t] = chi2;
            continue;
        }
        std::vector<int> touched;
        for (int j = 0; j < n; ++j)
            if (std::find(touched.begin(), touched.end(), sec[hits[j]]) == touched.end())
                touched.push_back(sec[hits[j]]);
        std::vector<double> g(216, 0.0);
        bool ok = true;
        double chi2v = 0.0;
        for (size_t base = 0; base < touched.size() && ok; base += ND / 6) {
            std::vector<D24> th(36 * 6);
            for (int s = 0; s < 36; ++s)
                for (int q = 0; q < 6; ++q) th[s * 6 + q] = D24(align ? align[s * 6 + q] : 0.0);
            for (size_t k = base; k < touched.size() && k < base + ND / 6; ++k)
                for (int q = 0; q < 6; ++q) th[touched[k] * 6 + q].d[(k - base) * 6 + q] = 1.0;
            D24 p[5], C[15], chi2;
            auto thf = [&](int h) -> const D24* { return th.data() + 6 * sec[h]; };
            ok = kf_fit<D24>(y, z, row, sec, hits, n, true, *prm, thf, p, C, chi2);
            if (!ok) break;
            chi2v = chi2.v;
            for (size_t k = base; k < touched.size() && k < base + ND / 6; ++k)
                for (int q = 0; q < 6; ++q) g[touched[k] * 6 + q] = chi2.d[(k - base) * 6 + q];
        }
        if (ok) {
            tchi2[t] = chi2v;
            tgrad[t] = std::move(g);
        }
    }
    double tot = 0.0;
    for (int t = 0; t < T; ++t) tot += tchi2[t];
    *chi2_total = tot;
    if (grad) {
        for (int i = 0; i < 216; ++i) grad[i] = 0.0;
        for (int t = 0; t < T; ++t)
            if (!tgrad[t].empty())
                for (int i = 0; i < 216; ++i) grad[i] += tgrad[t][i];
    }
    return 0;
}

// ---- distortion map (Sec. 4.2: the TPC space-charge distortion evaluation)
// The paper names the task and gives no method.  Reading: a piecewise-
// constant displacement per voxel of the sector frames, added to the aligned
// cluster position; its gradient is the exact derivative of the summed fit
// chi2, the same quantity as the alignment gradient with the per-sector
// parameters replaced by per-voxel ones.
static bool grid_ok(const orc_field_grid* g) {
    return g && g->n_band >= 1 && g->n_band <= NROW && NROW % g->n_band == 0 && g->n_y >= 1 &&
           g->n_z >= 1 && (int64_t)NSEC * g->n_band * g->n_y * g->n_z < (int64_t)1 << 30;
}

// bin of an FP32 coordinate f (already scaled to bin units): clamped to
// [0, nbin - 1]; NaN goes to bin 0
static int clamp_bin(float f, int nbin) {
    if (!(f >= 1.0f)) return 0;
    if (f >= (float)nbin) return nbin - 1;
    return (int)f;
}

static int32_t voxel_of(float y, float z, int r, int s, const orc_field_grid& g) {
    const int band = r * g.n_band / NROW;
    const float u = y / row_xf(r);
    const int iy = clamp_bin((u - g.u_lo) * g.u_inv, g.n_y);
    const int iz = clamp_bin(std::fabs(z) * g.z_inv, g.n_z);
    return ((s * g.n_band + band) * g.n_y + iy) * g.n_z + iz;
}

int64_t orc_voxel_of(const float* y, const float* z, const uint16_t* row, const int32_t* sec,
                     int64_t n, const orc_field_grid* grid, int32_t* vox) {
    if (!grid_ok(grid)) return -1;
    for (int64_t i = 0; i < n; ++i) vox[i] = voxel_of(y[i], z[i], row[i], sec[i], *grid);
    return (int64_t)NSEC * grid->n_band * grid->n_y * grid->n_z;
}

// eight voxels (3 components each) carry dual parts per pass
constexpr int NVP = ND / 3;

int orc_field_adjoint(const float* y, const float* z, const uint16_t* row, const int32_t* sec,
                      const int32_t* trk_off, const int32_t* trk_hits, int32_t T,
                      const double* align, const orc_field_grid* grid, const double* field,
                      const orc_params* prm, double* chi2_total, double* grad_field) {
    if (!grid_ok(grid)) return -1;
    const int64_t NV = (int64_t)NSEC * grid->n_band * grid->n_y * grid->n_z;
    const int nt = orc_get_threads();
    std::vector<double> tchi2(T, 0.0);
    // per track: (voxel, d chi2 / d field[voxel][0..2]) of its touched voxels
    std::vector<std::vector<std::pair<int32_t, std::array<double, 3>>>> tgrad(grad_field ? T : 0);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int t = 0; t < T; ++t) {
        const int n = trk_off[t + 1] - trk_off[t];
        const int32_t* hits = trk_hits + trk_off[t];
        if (n < 3) continue;
        std::vector<int32_t> vox(n);
        for (int j = 0; j < n; ++j) vox[j] = voxel_of(y[hits[j]], z[hits[j]], row[hits[j]], sec[hits[j]], *grid);
        if (!grad_field) {
            double p[5], C[15], chi2;
            auto th = [&](int h) -> const double* { return align ? align + 6 * sec[h] : nullptr; };
            auto disp = [&](int j) -> const double* { return field + 3 * (int64_t)vox[j]; };
            if (kf_fit<double>(y, z, row, sec, hits, n, true, *prm, th, p, C, chi2, nullptr, disp))
                tchi2[t] = chi2;
            continue;
        }
        std::vector<int32_t> touched;
        for (int j = 0; j < n; ++j)
            if (std::find(touched.begin(), touched.end(), vox[j]) == touched.end()) touched.push_back(vox[j]);
        std::vector<std::pair<int32_t, std::array<double, 3>>> g;
        std::vector<D24> th(align ? 36 * 6 : 0);
        for (size_t i = 0; i < th.size(); ++i) th[i] = D24(align[i]);
        bool ok = true;
        double chi2v = 0.0;
        for (size_t base = 0; base < touched.size() && ok; base += NVP) {
            std::vector<D24> d(3 * (size_t)n);
            for (int j = 0; j < n; ++j) {
                for (int c = 0; c < 3; ++c) d[3 * j + c] = D24(field[3 * (int64_t)vox[j] + c]);
                for (size_t k = base; k < touched.size() && k < base + NVP; ++k)
                    if (touched[k] == vox[j])
                        for (int c = 0; c < 3; ++c) d[3 * j + c].d[(k - base) * 3 + c] = 1.0;
            }
            D24 p[5], C[15], chi2;
            auto thf = [&](int h) -> const D24* { return align ? th.data() + 6 * sec[h] : nullptr; };
            auto disp = [&](int j) -> const D24* { return d.data() + 3 * j; };
            ok = kf_fit<D24>(y, z, row, sec, hits, n, true, *prm, thf, p, C, chi2, nullptr, disp);
            if (!ok) break;
            chi2v = chi2.v;
            for (size_t k = base; k < touched.size() && k < base + NVP; ++k)
                g.push_back({touched[k], {chi2.d[(k - base) * 3 + 0], chi2.d[(k - base) * 3 + 1],
                                          chi2.d[(k - base) * 3 + 2]}});
        }
        if (ok) {
            tchi2[t] = chi2v;
            tgrad[t] = std::move(g);
        }
    }
    double tot = 0.0;
    for (int t = 0; t < T; ++t) tot += tchi2[t];
    *chi2_total = tot;
    if (grad_field) {
        for (int64_t i = 0; i < 3 * NV; ++i) grad_field[i] = 0.0;
        for (int t = 0; t < T; ++t)
            for (const auto& e : tgrad[t])
                for (int c = 0; c < 3; ++c) grad_field[3 * (int64_t)e.first + c] += e.second[c];
    }
    return 0;
}

// Per-voxel diagonal blocks of the field's Gauss-Newton matrix: the fit
// loop of kf_fit, in passes of eight voxels whose components carry the dual
// parts, accumulating 2 dr^T S^-1 dr of every predicted residual.
int orc_field_gn_blocks(const float* y, const float* z, const uint16_t* row, const int32_t* sec,
                        const int32_t* trk_off, const int32_t* trk_hits, int32_t T,
                        const double* align, const orc_field_grid* grid, const double* field,
                        const orc_params* prm, double* blocks) {
    if (!grid_ok(grid)) return -1;
    const int64_t NV = (int64_t)NSEC * grid->n_band * grid->n_y * grid->n_z;
    const int nt = orc_get_threads();
    std::vector<std::vector<std::pair<int32_t, std::array<double, 9>>>> tb(T);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int t = 0; t < T; ++t) {
        const int n = trk_off[t + 1] - trk_off[t];
        const int32_t* hits = trk_hits + trk_off[t];
        if (n < 3) continue;
        std::vector<int32_t> vox(n);
        for (int j = 0; j < n; ++j) vox[j] = voxel_of(y[hits[j]], z[hits[j]], row[hits[j]], sec[hits[j]], *grid);
        std::vector<int32_t> touched;
        for (int j = 0; j < n; ++j)
            if (std::find(touched.begin(), touched.end(), vox[j]) == touched.end()) touched.push_back(vox[j]);
        std::vector<D24> th(align ? 36 * 6 : 0);
        for (size_t i = 0; i < th.size(); ++i) th[i] = D24(align[i]);
        const Seed sd = make_seed(y, z, row, sec, hits, n, true, *prm);
        std::vector<std::pair<int32_t, std::array<double, 9>>> out;
        bool ok = true;
        for (size_t base = 0; base < touched.size() && ok; base += NVP) {
            const int kn = (int)std::min<size_t>(NVP, touched.size() - base);
            D24 p[5], C[15], chi2(0.0), J[25], dX[5];
            for (int i = 0; i < 5; ++i) p[i] = D24(sd.p[i]);
            for (int i = 0; i < 15; ++i) C[i] = D24(0.0);
            for (int i = 0; i < 5; ++i) C[sidx(i, i)] = D24(prm->prior[i]);
            D24 x(sd.x);
            int frame = sd.frame;
            std::vector<std::array<double, 9>> acc(kn);
            for (auto& a : acc) a.fill(0.0);
            for (int j = 0; j < n && ok; ++j) {
                const int h = hits[j];
                D24 xc, yc, zc;
                if (align) {
                    corrected<D24>(th.data() + 6 * sec[h], row_x(row[h]), (double)y[h], (double)z[h], xc, yc, zc);
                } else {
                    xc = D24(row_x(row[h]));
                    yc = D24((double)y[h]);
                    zc = D24((double)z[h]);
                }
                D24 d3[3];
                for (int c = 0; c < 3; ++c) d3[c] = D24(field[3 * (int64_t)vox[j] + c]);
                for (int k = 0; k < kn; ++k)
                    if (touched[base + k] == vox[j])
                        for (int c = 0; c < 3; ++c) d3[c].d[k * 3 + c] = 1.0;
                xc = xc + d3[0];
                yc = yc + d3[1];
                zc = zc + d3[2];
                ok = move_state(x, p, frame, xc, sec[h], J, dX, *prm);
                if (!ok) break;
                cov_transform(C, J);
                D24 res[2], si[3];
                kf_update(p, C, yc, zc, prm->sigma_y2, prm->sigma_z2, chi2, res, si);
                for (int k = 0; k < kn; ++k)
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) {
                            const int ia = k * 3 + a, ib = k * 3 + b;
                            acc[k][3 * a + b] +=
                                2.0 * (res[0].d[ia] * (si[0].v * res[0].d[ib] + si[1].v * res[1].d[ib]) +
                                       res[1].d[ia] * (si[1].v * res[0].d[ib] + si[2].v * res[1].d[ib]));
                        }
            }
            if (ok)
                for (int k = 0; k < kn; ++k) out.push_back({touched[base + k], acc[k]});
        }
        if (ok) tb[t] = std::move(out);
    }
    for (int64_t i = 0; i < 9 * NV; ++i) blocks[i] = 0.0;
    for (int t = 0; t < T; ++t)
        for (const auto& e : tb[t])
            for (int i = 0; i < 9; ++i) blocks[9 * (int64_t)e.first + i] += e.second[i];
    return 0;
}

// Gauss-Newton matrix: sum over tracks and clusters of 2 dr^T S^-1 dr, with
// dr the derivative of each predicted residual with respect to the
// parameters of the track's touched sectors.
int orc_gauss_newton(const float* y, const float* z, const uint16_t* row, const int32_t* sec,
                     const int32_t* trk_off, const int32_t* trk_hits, int32_t T, const double* align,
                     const orc_params* prm, double* gn) {
    const int nt = orc_get_threads();
    std::vector<std::vector<double>> part(nt, std::vector<double>(216 * 216, 0.0));
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int t = 0; t < T; ++t) {
#ifdef _OPENMP
        const int tid = omp_get_thread_num();
#else
        const int tid = 0;
#endif
        const int n = trk_off[t + 1] - trk_off[t];
        const int32_t* hits = trk_hits + trk_off[t];
        if (n < 3) continue;
        std::vector<int> touched;
        for (int j = 0; j < n; ++j)
            if (std::find(touched.begin(), touched.end(), sec[hits[j]]) == touched.end())
                touched.push_back(sec[hits[j]]);
        if ((int)touched.size() > ND / 6) continue;
        std::vector<D24> th(36 * 6);
        for (int s = 0; s < 36; ++s)
            for (int q = 0; q < 6; ++q) th[s * 6 + q] = D24(align ? align[s * 6 + q] : 0.0);
        for (size_t k = 0; k < touched.size(); ++k)
            for (int q = 0; q < 6; ++q) th[touched[k] * 6 + q].d[k * 6 + q] = 1.0;
        const Seed sd = make_seed(y, z, row, sec, hits, n, true, *prm);
        D24 p[5], C[15], chi2(0.0), J[25], dX[5];
        for (int i = 0; i < 5; ++i) p[i] = D24(sd.p[i]);
        for (int i = 0; i < 15; ++i) C[i] = D24(0.0);
        for (int i = 0; i < 5; ++i) C[sidx(i, i)] = D24(prm->prior[i]);
        D24 x(sd.x);
        int frame = sd.frame;
        bool ok = true;
        std::vector<double> local(24 * 24, 0.0);
        for (int j = 0; j < n && ok; ++j) {
            const int h = hits[j];
            D24 xc, yc, zc;
            corrected<D24>(th.data() + 6 * sec[h], row_x(row[h]), (double)y[h], (double)z[h], xc, yc, zc);
            ok = move_state(x, p, frame, xc, sec[h], J, dX, *prm);
            if (!ok) break;
            cov_transform(C, J);
            D24 res[2], si[3];
            kf_update(p, C, yc, zc, prm->sigma_y2, prm->sigma_z2, chi2, res, si);
            const int m = (int)touched.size() * 6;
            for (int a = 0; a < m; ++a)
                for (int b = 0; b < m; ++b)
                    local[a * 24 + b] += 2.0 * (res[0].d[a] * (si[0].v * res[0].d[b] + si[1].v * res[1].d[b]) +
                                                res[1].d[a] * (si[1].v * res[0].d[b] + si[2].v * res[1].d[b]));
        }
        if (!ok) continue;
        for (size_t ka = 0; ka < touched.size(); ++ka)
            for (size_t kb = 0; kb < touched.size(); ++kb)
                for (int qa = 0; qa < 6; ++qa)
                    for (int qb = 0; qb < 6; ++qb)
                        part[tid][(touched[ka] * 6 + qa) * 216 + touched[kb] * 6 + qb] +=
                            local[(ka * 6 + qa) * 24 + kb * 6 + qb];
    }
    for (int i = 0; i < 216 * 216; ++i) {
        double s = 0;
        for (int k = 0; k < nt; ++k) s += part[k][i];
        gn[i] = s;
    }
    return 0;
}

int orc_seed(const float* y, const float* z, const uint16_t* row, const int32_t* sector_of,
             const int32_t* hits, int32_t n, int first_is_outer, const orc_params* prm,
             double* x0, int32_t* frame, double* p) {
    if (n < 3) return 1;
    const Seed sd = make_seed(y, z, row, sector_of, hits, n, first_is_outer != 0, *prm);
    *x0 = sd.x;
    *frame = sd.frame;
    for (int i = 0; i < 5; ++i) p[i] = sd.p[i];
    return 0;
}

int orc_propagate(double x1, int s1, const double* p, double x2, int s2, const orc_params* prm,
                  double* p_out, double* jac, double* dx1, double* dx2) {
    double q[5], J[25], dX[5];
    for (int i = 0; i < 5; ++i) q[i] = p[i];
    double x = x1;
    int frame = s1;
    if (!move_state<double>(x, q, frame, x2, s2, J, dX, *prm)) return 1;
    for (int i = 0; i < 5; ++i) p_out[i] = q[i];
    for (int i = 0; i < 25; ++i) jac[i] = J[i];
    // derivative with respect to the start plane: by the same chain rule,
    // moving x1 shifts the transport start (and x' on a sector change).
    if (dx2)
        for (int i = 0; i < 5; ++i) dx2[i] = dX[i];
    if (dx1) {
        const double ca = s1 == s2 ? 1.0 : std::cos(delta_alpha(s1, s2));
        for (int i = 0; i < 5; ++i) dx1[i] = -dX[i] * ca;
        if (s1 != s2) {
            // y' = -x sin + y cos also moves with x1
            const double sa = std::sin(delta_alpha(s1, s2));
            // d p_out / d y' = F[:,0]; recover F[:,0] = (J[:,0] + dX sa)/ca
            for (int i = 0; i < 5; ++i) {
                const double f0 = (jac[i * 5 + 0] + dX[i] * sa) / ca;
                dx1[i] += -f0 * sa;
            }
        }
    }
    return 0;
}

int64_t orc_bruteforce_chains(const float* y, const float* z, const uint16_t* row, int64_t n,
                              int32_t sector, const orc_params* prm_, double chi2ndf_max,
                              int64_t cap_chains, int64_t cap_hits, int32_t* out_off,
                              int32_t* out_hits) {
    // Exhaustive depth-first enumeration of maximal admissible chains of one
    // group.  A chain (innermost first) has strictly rising rows; a step of
    // g rows (g <= max_gap) may skip rows only when none of the skipped rows
    // holds an admissible continuation; every consecutive pair lies inside
    // the windows and every interior triplet has D^2 <= chi2_link.  A chain
    // is maximal when it cannot be extended outwards and is not the outer
    // part of a longer admissible chain.  Kept: length >= n_min and FP64 fit
    // chi2/ndf <= chi2ndf_max.
    const orc_params& prm = *prm_;
    std::vector<int32_t> sec(n, sector);
    std::vector<std::vector<int32_t>> byrow(NROW);
    for (int64_t i = 0; i < n; ++i) byrow[row[i]].push_back((int32_t)i);
    auto step_ok = [&](const std::vector<int32_t>& path, int32_t u) {
        const int32_t c = path.back();
        const float xc = row_xf(row[c]), xu = row_xf(row[u]);
        if (!in_window(xc, y[c], z[c], xu, y[u], z[u], prm.win_y, prm.win_z)) return false;
        if (path.size() < 2) return true;
        const int32_t d = path[path.size() - 2];
        const float xd = row_xf(row[d]);
        const float d2 = triplet_d2(xd, y[d], z[d], xc, y[c], z[c], xu, y[u], z[u], prm.sigma_y2, prm.sigma_z2);
        return d2 <= prm.chi2_link;
    };
    std::vector<std::vector<int32_t>> leaves;
    std::vector<int32_t> path;
    std::function<void()> dfs = [&]() {
        const int r = row[path.back()];
        bool extended = false;
        for (int g = 1; g <= prm.max_gap && r + g < NROW; ++g) {
            bool any = false;
            for (int32_t u : byrow[r + g]) {
                if (!step_ok(path, u)) continue;
                any = true;
                path.push_back(u);
                dfs();
                path.pop_back();
            }
            if (any) { extended = true; break; }  // no skipping past a continuation
        }
        if (!extended) leaves.push_back(path);
    };
    for (int r = 0; r < NROW; ++r)
        for (int32_t c : byrow[r]) {
            path.assign(1, c);
            dfs();
        }
    // drop chains that are the outer part of a longer chain
    std::vector<std::vector<int32_t>> found;
    for (size_t i = 0; i < leaves.size(); ++i) {
        const auto& a = leaves[i];
        bool suffix = false;
        for (size_t j = 0; j < leaves.size() && !suffix; ++j) {
            const auto& b = leaves[j];
            if (b.size() <= a.size()) continue;
            suffix = std::equal(a.begin(), a.end(), b.end() - a.size());
        }
        if (suffix || (int)a.size() < prm.n_min) continue;
        std::vector<int32_t> hits(a.rbegin(), a.rend());  // outermost first
        double p[5], C[15], chi2;
        auto no_align = [](int) -> const double* { return nullptr; };
        if (!kf_fit<double>(y, z, row, sec.data(), hits.data(), (int)hits.size(), true, prm, no_align, p,
                            C, chi2))
            continue;
        if (chi2 / (2.0 * (double)hits.size() - 5.0) <= chi2ndf_max) found.push_back(a);
    }
    int64_t total = 0;
    for (auto& f : found) total += (int64_t)f.size();
    if ((int64_t)found.size() > cap_chains || total > cap_hits)
        return -std::max<int64_t>((int64_t)found.size(), total);
    out_off[0] = 0;
    int64_t o = 0;
    for (size_t i = 0; i < found.size(); ++i) {
        for (int32_t h : found[i]) out_hits[o++] = h;
        out_off[i + 1] = (int32_t)o;
    }
    return (int64_t)found.size();
}

int orc_seed_f64(const double* y, const double* z, const uint16_t* row, const int32_t* sector_of,
                 const int32_t* hits, int32_t n, int first_is_outer, const orc_params* prm, double* x0,
                 int32_t* frame, double* p) {
    if (n < 3) return 1;
    const Seed sd = make_seed(y, z, row, sector_of, hits, n, first_is_outer != 0, *prm);
    *x0 = sd.x;
    *frame = sd.frame;
    for (int i = 0; i < 5; ++i) p[i] = sd.p[i];
    return 0;
}

int64_t orc_tracklet(const float* y, const float* z, const uint16_t* row, int64_t beg, int64_t end,
                     int32_t sector, const int32_t* seg_hits, int32_t nseg, const orc_params* prm,
                     int32_t* out, int32_t cap) {
    if (beg < 0 || end < beg || nseg < 3 || sector < 0 || sector >= NSEC) return -1;
    std::vector<std::vector<int32_t>> rows(NROW);
    for (int64_t i = beg; i < end; ++i) {
        if (row[i] >= NROW) return -1;
        rows[row[i]].push_back((int32_t)i);
    }
    std::vector<int32_t> sec((size_t)end, sector);
    Segment sg;
    sg.event = 0;
    sg.sector = sector;
    sg.hits.assign(seg_hits, seg_hits + nseg);
    for (int32_t h : sg.hits)
        if (h < beg || h >= end) return -1;
    sg.canon = *std::min_element(sg.hits.begin(), sg.hits.end());
    sg.row_max = row[sg.hits.front()];
    sg.row_min = row[sg.hits.back()];
    const std::vector<int32_t> H = build_tracklet(y, z, row, sec.data(), rows, sg, *prm);
    if ((int64_t)H.size() > cap) return -(int64_t)H.size();
    for (size_t i = 0; i < H.size(); ++i) out[i] = H[i];
    return (int64_t)H.size();
}

int orc_merge_chi2(const float* y, const float* z, const uint16_t* row, const int32_t* hits_a, int32_t na,
                   int32_t sec_a, const int32_t* hits_b, int32_t nb, int32_t sec_b, const orc_params* prm,
                   double* chi2, int32_t* gates_pass) {
    if (na < 3 || nb < 3 || sec_a < 0 || sec_a >= NSEC || sec_b < 0 || sec_b >= NSEC) return 1;
    int32_t hmax = 0;
    for (int i = 0; i < na; ++i) hmax = std::max(hmax, hits_a[i]);
    for (int i = 0; i < nb; ++i) hmax = std::max(hmax, hits_b[i]);
    std::vector<int32_t> sec((size_t)hmax + 1, 0);
    Segment A, B;
    for (int k = 0; k < 2; ++k) {
        Segment& S = k == 0 ? A : B;
        const int32_t* h = k == 0 ? hits_a : hits_b;
        const int32_t m = k == 0 ? na : nb;
        S.event = 0;
        S.sector = k == 0 ? sec_a : sec_b;
        S.hits.assign(h, h + m);
        for (int32_t q : S.hits) sec[q] = S.sector;
        S.canon = *std::min_element(S.hits.begin(), S.hits.end());
        S.row_max = row[S.hits.front()];
        S.row_min = row[S.hits.back()];
    }
    fit_segment(y, z, row, sec.data(), A, *prm);
    fit_segment(y, z, row, sec.data(), B, *prm);
    if (!merge_chi2_value(A, B, *prm, *chi2)) return 2;
    double c2;
    *gates_pass = merge_chi2(A, B, z, *prm, c2) ? 1 : 0;
    return 0;
}

int orc_kf_ops(const float* y, const float* z, const uint16_t* row, const int32_t* sec,
               const int32_t* trk_off, const int32_t* trk_hits, int32_t T, const orc_params* prm,
               double* ops, int64_t* steps) {
    auto no_align = [](int) -> const Cnt* { return nullptr; };
    long long total = 0;
    int64_t n_steps = 0;
    for (int t = 0; t < T; ++t) {
        const int n = trk_off[t + 1] - trk_off[t];
        if (n < 3) continue;
        Cnt p[5], C[15], chi2;
        g_ops = 0;
        if (!kf_fit<Cnt>(y, z, row, sec, trk_hits + trk_off[t], n, true, *prm, no_align, p, C, chi2)) continue;
        total += g_ops;
        n_steps += n;
    }
    *ops = (double)total;
    *steps = n_steps;
    return 0;
}

// 5x5 SPD inverse by Cholesky (full matrix out, row-major); false when not
// positive definite.
static bool spd_inverse5(const double M[15], double inv[25]) {
    double L[5][5] = {};
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = M[sidx(i, j)];
            for (int l = 0; l < j; ++l) s -= L[i][l] * L[j][l];
            if (i == j) {
                if (!(s > 0)) return false;
                L[i][i] = std::sqrt(s);
            } else {
                L[i][j] = s / L[j][j];
            }
        }
    for (int c = 0; c < 5; ++c) {  // solve L L^T x = e_c
        double v[5], x[5];
        for (int i = 0; i < 5; ++i) {
            double s = i == c ? 1.0 : 0.0;
            for (int l = 0; l < i; ++l) s -= L[i][l] * v[l];
            v[i] = s / L[i][i];
        }
        for (int i = 4; i >= 0; --i) {
            double s = v[i];
            for (int l = i + 1; l < 5; ++l) s -= L[l][i] * x[l];
            x[i] = s / L[i][i];
        }
        for (int i = 0; i < 5; ++i) inv[i * 5 + c] = x[i];
    }
    return true;
}

int orc_smooth_tracks(const float* y, const float* z, const uint16_t* row, const int32_t* sec,
                      const int32_t* trk_off, const int32_t* trk_hits, int32_t T, const orc_params* prm,
                      double* out, double* chi2o, int32_t* ndf) {
    const int nt = orc_get_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int t = 0; t < T; ++t) {
        const int b = trk_off[t], n = trk_off[t + 1] - b;
        struct Step { double pp[5], Cp[15], F[25], pf[5], Cf[15]; };
        std::vector<Step> st((size_t)std::max(n, 0));
        auto rec = [&](int j, const double* pp, const double* Cp, const double* F, const double* pf,
                       const double* Cf) {
            Step& q = st[j];
            std::memcpy(q.pp, pp, sizeof q.pp);
            std::memcpy(q.Cp, Cp, sizeof q.Cp);
            std::memcpy(q.F, F, sizeof q.F);
            std::memcpy(q.pf, pf, sizeof q.pf);
            std::memcpy(q.Cf, Cf, sizeof q.Cf);
        };
        auto no_align = [](int) -> const double* { return nullptr; };
        double p[5], C[15], chi2 = 0;
        bool ok = n >= 3 && kf_fit<double>(y, z, row, sec, trk_hits + b, n, true, *prm, no_align, p, C, chi2,
                                           nullptr, NoDisp(), rec);
        // Rauch-Tung-Striebel: from the last filtered state back over the hits
        double xs[5], Cs[15];
        if (ok) {
            std::memcpy(xs, st[n - 1].pf, sizeof xs);
            std::memcpy(Cs, st[n - 1].Cf, sizeof Cs);
            double* o = out + (size_t)(b + n - 1) * 20;
            std::memcpy(o, xs, sizeof xs);
            std::memcpy(o + 5, Cs, sizeof Cs);
        }
        for (int j = n - 2; j >= 0 && ok; --j) {
            const Step &f = st[j], &nx = st[j + 1];
            double Pinv[25];
            if (!spd_inverse5(nx.Cp, Pinv)) {
                ok = false;
                break;
            }
            // A = Cf F^T Pinv
            double CfF[25], A[25];
            for (int i = 0; i < 5; ++i)
                for (int k = 0; k < 5; ++k) {
                    double acc = 0;
                    for (int l = 0; l < 5; ++l) acc += f.Cf[sidx(i, l)] * nx.F[k * 5 + l];
                    CfF[i * 5 + k] = acc;
                }
            for (int i = 0; i < 5; ++i)
                for (int k = 0; k < 5; ++k) {
                    double acc = 0;
                    for (int l = 0; l < 5; ++l) acc += CfF[i * 5 + l] * Pinv[l * 5 + k];
                    A[i * 5 + k] = acc;
                }
            // state: the smoothed state of hit j + 1 moved back to hit j
            // along the motion (xb = f^-1(xs)), then
            //   xn = xb + (I - A F) (pf - xb),
            // which is the textbook pf + A (xs - f(pf)) for a linear f and
            // exact for a deterministic segment (A F = I without material)
            double xb[5], xq = row_x(row[trk_hits[b + j + 1]]);
            std::memcpy(xb, xs, sizeof xb);
            {
                const int h1 = trk_hits[b + j + 1], h0 = trk_hits[b + j];
                int frame = sec[h1];
                double Cd[15] = {}, Jd[25], dX[5];
                const bool mat = prm->mat_x_x0 > 0.0 || prm->mat_eloss > 0.0;
                if (mat) material_step(xb, Cd, *prm, false);
                if (mat && sec[h0] == sec[h1]) {
                    const int r0 = row[h1], r1 = row[h0], stp = r1 > r0 ? 1 : -1;
                    for (int r = r0 + stp; r != r1 && ok; r += stp) {
                        ok = move_state<double>(xq, xb, frame, row_x(r), sec[h0], Jd, dX, *prm);
                        if (ok) material_step(xb, Cd, *prm, false);
                    }
                }
                if (ok) ok = move_state<double>(xq, xb, frame, row_x(row[h0]), sec[h0], Jd, dX, *prm);
                if (!ok) break;
            }
            double AF[25];
            for (int i = 0; i < 5; ++i)
                for (int k = 0; k < 5; ++k) {
                    double acc = 0;
                    for (int l = 0; l < 5; ++l) acc += A[i * 5 + l] * nx.F[l * 5 + k];
                    AF[i * 5 + k] = acc;
                }
            double D[25], xn[5], Cn[15];
            for (int i = 0; i < 5; ++i) {
                double acc = xb[i];
                for (int l = 0; l < 5; ++l) acc += ((i == l ? 1.0 : 0.0) - AF[i * 5 + l]) * (f.pf[l] - xb[l]);
                xn[i] = acc;
            }
            for (int i = 0; i < 5; ++i)
                for (int k = 0; k < 5; ++k) D[i * 5 + k] = Cs[sidx(i, k)] - nx.Cp[sidx(i, k)];
            double AD[25];
            for (int i = 0; i < 5; ++i)
                for (int k = 0; k < 5; ++k) {
                    double acc = 0;
                    for (int l = 0; l < 5; ++l) acc += A[i * 5 + l] * D[l * 5 + k];
                    AD[i * 5 + k] = acc;
                }
            for (int i = 0; i < 5; ++i)
                for (int k = i; k < 5; ++k) {
                    double acc = f.Cf[sidx(i, k)];
                    for (int l = 0; l < 5; ++l) acc += AD[i * 5 + l] * A[k * 5 + l];
                    Cn[sidx(i, k)] = acc;
                }
            std::memcpy(xs, xn, sizeof xs);
            std::memcpy(Cs, Cn, sizeof Cs);
            double* o = out + (size_t)(b + j) * 20;
            std::memcpy(o, xs, sizeof xs);
            std::memcpy(o + 5, Cs, sizeof Cs);
        }
        if (!ok)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < 20; ++i) out[(size_t)(b + j) * 20 + i] = 0.0;
        chi2o[t] = ok ? chi2 : 0.0;
        ndf[t] = ok ? 2 * n - 5 : -1;
    }
    return 0;
}

// ---- NEXT-2: clusterization of pad-time digits ------------------------------
// A digit (t, p) of a pad-row plane is a peak when its count is at least
// q_peak, above each of its four neighbours earlier in raster order and at
// least each of the four later ones (outside the array: 0), so that a
// plateau yields one peak.  Its cluster sums the 5 x 5 window around it
// (clipped to the array): Q, and the count-weighted pad and time offsets,
// all exact integers; the position follows in FP32, one rounding per
// operation: cp = p + Sp/Q, y = (cp - 79.5) PAD_W; ct = t + St/Q,
// |z| = (ct + 0.5) T_W (negative on the C side).  Clusters are written per
// plane (event, sector, row) in raster order of their peaks.
int64_t orc_find_clusters(const uint16_t* digits, int32_t n_events, int32_t n_time, int32_t q_peak,
                          float* y, float* z, uint16_t* row, uint16_t* charge, int64_t* evt_sector_off,
                          int64_t cap) {
    constexpr int NP = 160;
    const int64_t planes = (int64_t)n_events * NSEC * NROW;
    std::vector<std::vector<std::array<float, 3>>> found((size_t)planes);
    const int nt = orc_get_threads();
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
    for (int64_t pl = 0; pl < planes; ++pl) {
        const uint16_t* d = digits + (size_t)pl * n_time * NP;
        auto at = [&](int t, int p) -> int {
            return (t < 0 || t >= n_time || p < 0 || p >= NP) ? 0 : (int)d[(size_t)t * NP + p];
        };
        const bool side_c = (pl / NROW) % NSEC >= NPHI;
        for (int t = 0; t < n_time; ++t)
            for (int p = 0; p < NP; ++p) {
                const int q = at(t, p);
                if (q < q_peak) continue;
                if (!(q > at(t - 1, p - 1) && q > at(t - 1, p) && q > at(t - 1, p + 1) && q > at(t, p - 1) &&
                      q >= at(t, p + 1) && q >= at(t + 1, p - 1) && q >= at(t + 1, p) && q >= at(t + 1, p + 1)))
                    continue;
                int64_t Q = 0, Sp = 0, St = 0;
                for (int dt = -2; dt <= 2; ++dt)
                    for (int dp = -2; dp <= 2; ++dp) {
                        const int v = at(t + dt, p + dp);
                        Q += v;
                        Sp += (int64_t)v * dp;
                        St += (int64_t)v * dt;
                    }
                const float cp = (float)p + (float)Sp / (float)Q;
                const float yy = (cp - 79.5f) * 0.6f;
                const float ct = (float)t + (float)St / (float)Q;
                const float az = (ct + 0.5f) * 0.5f;
                found[(size_t)pl].push_back({yy, side_c ? -az : az, (float)std::min<int64_t>(Q, 65535)});
            }
    }
    int64_t total = 0;
    for (auto& f : found) total += (int64_t)f.size();
    if (total > cap) return -total;
    int64_t o = 0;
    for (int64_t g = 0; g < (int64_t)n_events * NSEC; ++g) {
        evt_sector_off[g] = o;
        for (int r = 0; r < NROW; ++r)
            for (const auto& c : found[(size_t)(g * NROW + r)]) {
                y[o] = c[0];
                z[o] = c[1];
                row[o] = (uint16_t)r;
                charge[o] = (uint16_t)c[2];
                ++o;
            }
    }
    evt_sector_off[(int64_t)n_events * NSEC] = o;
    return total;
}

}  // extern "C"

// ---- NEXT-4: the drift-time offset t0 as a sixth state parameter ----------
// A collision at drift-time offset t0 (us) is seen at z' = z - v t0 on side
// A (sectors 0..17) and at z' = z + v t0 on side C (the time-frame
// convention of the pile-up frame).  The state (y, z, sin phi, tan lambda,
// q/pT, t0) carries the true z; the helix transport leaves t0 unchanged; a
// cluster of side sgn (+1 A, -1 C) measures (y, z - sgn v t0).  Found tracks
// never span both sides (the merge joins one side only), so a track that
// crosses the central membrane is found as two: an inner segment and an
// outer one, on opposite sides of one phi sector, with adjacent row ranges.
namespace {

// symmetric 6x6 storage, upper triangle row by row:
// 00 01 02 03 04 05 11 12 13 14 15 22 23 24 25 33 34 35 44 45 55
inline int s6(int i, int j) {
    if (i > j) std::swap(i, j);
    static const int base[6] = {0, 6, 11, 15, 18, 20};
    return base[i] + (j - i);
}

inline int side_sign(int sector) { return sector < NPHI ? 1 : -1; }

// SPD solve r^T M^-1 r by Cholesky for a dense n x n M (row-major); false
// when M is not positive definite.
bool chi2_dense(const double* r, const double* M, int n, double& out) {
    double L[36] = {};
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = M[i * n + j];
            for (int l = 0; l < j; ++l) s -= L[i * 6 + l] * L[j * 6 + l];
            if (i == j) {
                if (!(s > 0)) return false;
                L[i * 6 + i] = std::sqrt(s);
            } else {
                L[i * 6 + j] = s / L[j * 6 + j];
            }
        }
    double v[6];
    out = 0;
    for (int i = 0; i < n; ++i) {
        double s = r[i];
        for (int l = 0; l < i; ++l) s -= L[i * 6 + l] * v[l];
        v[i] = s / L[i * 6 + i];
        out += v[i] * v[i];
    }
    return true;
}

// Kalman update of the six-parameter state with one cluster of side sgn:
// H = [[1 0 0 0 0 0], [0 1 0 0 0 a]], a = -sgn v;  S = H C H^T + R,
// K = C H^T S^-1, p += K r, C -= K H C, chi2 += r^T S^-1 r.
void kf6_update(double p[6], double C[21], double my, double mz, double a, double sy2, double sz2,
                double& chi2) {
    double HC0[6], HC1[6];  // rows of H C
    for (int i = 0; i < 6; ++i) {
        HC0[i] = C[s6(0, i)];
        HC1[i] = C[s6(1, i)] + a * C[s6(5, i)];
    }
    const double r0 = my - p[0], r1 = mz - (p[1] + a * p[5]);
    const double S00 = HC0[0] + sy2, S01 = HC0[1] + a * HC0[5];
    const double S11 = HC1[1] + a * HC1[5] + sz2;
    const double det = S00 * S11 - S01 * S01;
    const double i00 = S11 / det, i01 = -S01 / det, i11 = S00 / det;
    double K0[6], K1[6];  // K = (H C)^T S^-1
    for (int i = 0; i < 6; ++i) {
        K0[i] = HC0[i] * i00 + HC1[i] * i01;
        K1[i] = HC0[i] * i01 + HC1[i] * i11;
    }
    for (int i = 0; i < 6; ++i) p[i] += K0[i] * r0 + K1[i] * r1;
    for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j) C[s6(i, j)] -= K0[i] * HC0[j] + K1[i] * HC1[j];
    chi2 += r0 * r0 * i00 + 2.0 * r0 * r1 * i01 + r1 * r1 * i11;
}

// C6 <- J6 C6 J6^T with J6 = diag(J, 1): the t0 row and column follow the
// five helix parameters' Jacobian, Var(t0) is unchanged.
void cov6_transform(double C[21], const double J[25]) {
    double full[36], tmp[36];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) full[i * 6 + j] = C[s6(i, j)];
    auto J6 = [&](int i, int l) { return i < 5 ? (l < 5 ? J[i * 5 + l] : 0.0) : (l == 5 ? 1.0 : 0.0); };
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double acc = 0.0;
            for (int l = 0; l < 6; ++l) acc += J6(i, l) * full[l * 6 + j];
            tmp[i * 6 + j] = acc;
        }
    for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j) {
            double acc = 0.0;
            for (int l = 0; l < 6; ++l) acc += tmp[i * 6 + l] * J6(j, l);
            C[s6(i, j)] = acc;
        }
}

// The joint fit of a hit list whose first n_outer hits are the outer
// segment (outermost first) and the rest the inner one, continuing inward.
// Seed: the three-cluster seed of the outer segment alone (its first,
// middle and last clusters, one side, so its z is the apparent z' of that
// side), its z made the true z with t0_seed; prior covariance diagonal,
// the helix parameters' prior as in the five-parameter fit and t0_prior^2
// for t0.  State and covariance at the innermost cluster on return.
bool fit_t0(const float* y, const float* z, const uint16_t* row, const int32_t* sec, const int32_t* hits,
            int n, int n_outer, double t0_seed, const orc_params& prm, const orc_sides_params& sp, double p6[6],
            double C6[21], double& chi2) {
    if (n_outer < 3 || n <= n_outer) return false;
    const Seed sd = make_seed(y, z, row, sec, hits, n_outer, true, prm);
    double p[5];
    for (int i = 0; i < 5; ++i) p[i] = sd.p[i];
    double t0 = t0_seed;
    p[1] = sd.p[1] + side_sign(sec[hits[0]]) * sp.v_drift * t0_seed;
    for (int i = 0; i < 21; ++i) C6[i] = 0.0;
    for (int i = 0; i < 5; ++i) C6[s6(i, i)] = prm.prior[i];
    C6[s6(5, 5)] = sp.t0_prior * sp.t0_prior;
    double x = sd.x;
    int frame = sd.frame;
    chi2 = 0.0;
    for (int j = 0; j < n; ++j) {
        const int h = hits[j];
        double J[25], dX[5];
        if (!move_state<double>(x, p, frame, row_x(row[h]), sec[h], J, dX, prm)) return false;
        cov6_transform(C6, J);
        double q[6] = {p[0], p[1], p[2], p[3], p[4], t0};
        kf6_update(q, C6, (double)y[h], (double)z[h], -side_sign(sec[h]) * sp.v_drift, prm.sigma_y2,
                   prm.sigma_z2, chi2);
        for (int i = 0; i < 5; ++i) p[i] = q[i];
        t0 = q[5];
    }
    for (int i = 0; i < 5; ++i) p6[i] = p[i];
    p6[5] = t0;
    return true;
}

// One found track as seen by the association.
struct SideTrack {
    bool usable = false;  // one side, >= n_min clusters, inward fit done (the outer role)
    bool out_ok = false;  // outward fit done too (the inner role)
    int event = 0, sgn = 0;
    int r_in = 0, r_out = 0;   // rows of the innermost and outermost clusters
    int s_in = 0, s_out = 0;   // their sectors
    double x_in = 0, p_in[5] = {}, C_in[15] = {}, chi2_in = 0;  // inward fit: state at the innermost cluster
    double x_out = 0, p_out[5] = {}, C_out[15] = {};            // outward fit: state at the outermost cluster
};

struct SideCand {
    int i, o;        // inner and outer track
    double t0s;      // t0 from the two junction states
    double dchi2;    // chi2 increase of the joint fit
    double p6[6], C6[21], chi2;
};

inline double rel_m(double u, double v) {
    const double m = std::max(std::fabs(u), std::fabs(v));
    return m > 0 ? std::fabs(u - v) / m : 0.0;
}

}  // namespace

extern "C" {

void orc_default_sides_params(orc_sides_params* p) {
    p->n_min = 10;
    p->gap_max = 8;
    p->chi2_junction = 30.0;
    p->z_membrane = 3.0;
    p->z_pre = 10.0;
    p->chi2_joint = 40.0;
    p->t0_prior = 1.0;
    p->v_drift = 2.58;
}

int orc_fit_t0(const float* y, const float* z, const uint16_t* row, const int32_t* sector_of,
               const int32_t* hits, int32_t n, int32_t n_outer, double t0_seed, const orc_params* prm,
               const orc_sides_params* sp, double* params6, double* cov6, double* chi2) {
    return fit_t0(y, z, row, sector_of, hits, n, n_outer, t0_seed, *prm, *sp, params6, cov6, *chi2) ? 0 : 1;
}

// Association of the A- and C-side segments of membrane-crossing tracks.
//  1. Per found track: usable when all its clusters lie on one side and it
//     has >= n_min of them; the inward fit gives the state at its innermost
//     cluster and the segment's chi2, the outward fit the state at its
//     outermost cluster.  The outer role needs the inward fit, the inner
//     role both.
//  2. Candidates (i inner, o outer): one event, opposite sides, the same
//     or an adjacent phi sector at the junction (i's outermost cluster,
//     o's innermost: a low-pT track may cross a sector border there too),
//     1 <= row(o innermost) - row(i outermost) <= gap_max.
//  2b. Coarse gate: the mean of the apparent z of i's outermost and o's
//     innermost cluster lies within z_pre of the membrane (the true z near
//     the junction; segments of different collisions are v |t0_a - t0_b|
//     apart there).
//  3. Junction: i's outward state moved to o's innermost plane; the 4-d
//     chi2 of (y, sin phi, tan lambda, q/pT) against o's inward state with
//     the sum of both covariances must be <= chi2_junction; with z'_i and
//     z'_o the two apparent z there, the true z at the junction,
//     (z'_i + z'_o)/2, must lie within z_membrane of the membrane; t0 seed
//     (z'_o - z'_i)/(2 sgn_i v).
//  4. The joint fit (o's clusters, then i's) with t0: dchi2 = chi2_joint -
//     chi2_i - chi2_o must be <= chi2_joint cut.
//  5. Every track keeps its best candidate by (dchi2 rounded to FP32,
//     partner index); a pair is accepted when each is the other's best.
// Outputs per track (T entries; both members of a pair get the pair's
// joint fit): partner (-1: none), t0, params6 [6], cov6 [21], chi2, ndf,
// dchi2.  margin (optional, T entries): the smallest relative margin of the
// decisions that involved the track (gates and the best-vs-next order),
// infinity when none.  Returns the number of pairs, -1 on invalid input.
int64_t orc_match_sides(const float* y, const float* z, const uint16_t* row, int64_t n, const int64_t* off,
                        int32_t n_events, const int32_t* trk_off, const int32_t* trk_hits, int32_t T,
                        const orc_params* prm_, const orc_sides_params* sp_, int32_t* partner, double* t0o,
                        double* params6, double* cov6, double* chi2o, int32_t* ndfo, double* dchi2o,
                        double* margin) {
    const orc_params& prm = *prm_;
    const orc_sides_params& sp = *sp_;
    const int G = n_events * NSEC;
    if (off[0] != 0 || off[G] != n || T < 0) return -1;
    for (int g = 0; g < G; ++g)
        if (off[g + 1] < off[g]) return -1;
    std::vector<int32_t> sec(n), evt(n);
    for (int g = 0; g < G; ++g)
        for (int64_t c = off[g]; c < off[g + 1]; ++c) {
            sec[c] = g % NSEC;
            evt[c] = g / NSEC;
        }
    for (int t = 0; t < T; ++t) {
        partner[t] = -1;
        t0o[t] = 0.0;
        for (int i = 0; i < 6; ++i) params6[t * 6 + i] = 0.0;
        for (int i = 0; i < 21; ++i) cov6[t * 21 + i] = 0.0;
        chi2o[t] = 0.0;
        ndfo[t] = -1;
        dchi2o[t] = 0.0;
        if (margin) margin[t] = std::numeric_limits<double>::infinity();
    }
    // 1. per-track classification and the two fits
    std::vector<SideTrack> st(T);
    const int nt = orc_get_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int t = 0; t < T; ++t) {
        const int b = trk_off[t], m = trk_off[t + 1] - b;
        SideTrack& s = st[t];
        if (m < std::max(3, sp.n_min)) continue;
        const int32_t* h = trk_hits + b;
        s.sgn = side_sign(sec[h[0]]);
        s.event = evt[h[0]];
        bool one = true;
        for (int j = 0; j < m; ++j) one = one && side_sign(sec[h[j]]) == s.sgn && evt[h[j]] == s.event;
        if (!one) continue;
        s.r_out = row[h[0]];
        s.s_out = sec[h[0]];
        s.r_in = row[h[m - 1]];
        s.s_in = sec[h[m - 1]];
        auto th = [](int) -> const double* { return nullptr; };
        double xl = 0;
        if (!kf_fit<double>(y, z, row, sec.data(), h, m, true, prm, th, s.p_in, s.C_in, s.chi2_in, &xl)) continue;
        s.x_in = xl;
        s.usable = true;
        std::vector<int32_t> rev(h, h + m);
        std::reverse(rev.begin(), rev.end());
        double c2o;
        if (!kf_fit<double>(y, z, row, sec.data(), rev.data(), m, false, prm, th, s.p_out, s.C_out, c2o, &xl)) continue;
        s.x_out = xl;
        s.out_ok = true;
    }
    // 2-3. candidates, bucketed by (event, side, phi sector, row) of the
    // outer segment's innermost cluster
    std::map<int64_t, std::vector<int>> by_inner_end;
    for (int t = 0; t < T; ++t)
        if (st[t].usable) {
            const int64_t key = ((int64_t)(st[t].event * 2 + (st[t].sgn > 0 ? 0 : 1)) * NPHI + st[t].s_in % NPHI) * NROW + st[t].r_in;
            by_inner_end[key].push_back(t);
        }
    std::vector<std::vector<SideCand>> cand_i(T);
    // (partner, margin) of every evaluated candidate, listed at the inner track
    std::vector<std::vector<std::pair<int, double>>> gm_i(T);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int i = 0; i < T; ++i) {
        const SideTrack& a = st[i];
        if (!a.usable || !a.out_ok) continue;
        for (int dp = -1; dp <= 1; ++dp)
        for (int gap = 1; gap <= sp.gap_max; ++gap) {
            const int r = a.r_out + gap;
            if (r >= NROW) break;
            const int ph = (a.s_out % NPHI + dp + NPHI) % NPHI;
            const int64_t key = ((int64_t)(a.event * 2 + (a.sgn > 0 ? 1 : 0)) * NPHI + ph) * NROW + r;
            auto it = by_inner_end.find(key);
            if (it == by_inner_end.end()) continue;
            for (int o : it->second) {
                const SideTrack& b = st[o];
                // coarse gate on the two end clusters' apparent z (their sum
                // is exact in FP64): segments of different collisions lie
                // v |t0_a - t0_b| apart there
                const double zc = 0.5 * ((double)z[trk_hits[trk_off[i]]] + (double)z[trk_hits[trk_off[o + 1] - 1]]);
                if (std::fabs(zc) > sp.z_pre) continue;
                // the inner segment's outward state moved to o's innermost plane
                double x = a.x_out, p[5], C[15], J[25], dX[5];
                for (int k = 0; k < 5; ++k) p[k] = a.p_out[k];
                for (int k = 0; k < 15; ++k) C[k] = a.C_out[k];
                int frame = a.s_out;
                if (!move_state<double>(x, p, frame, b.x_in, b.s_in, J, dX, prm)) continue;
                cov_transform(C, J);
                static const int ix[4] = {0, 2, 3, 4};
                double rv[4], M[16];
                for (int u = 0; u < 4; ++u) {
                    rv[u] = b.p_in[ix[u]] - p[ix[u]];
                    for (int w = 0; w < 4; ++w) M[u * 4 + w] = C[sidx(ix[u], ix[w])] + b.C_in[sidx(ix[u], ix[w])];
                }
                double c4;
                if (!chi2_dense(rv, M, 4, c4)) continue;
                const double zmem = 0.5 * (p[1] + b.p_in[1]);
                double m_i = std::min(rel_m(c4, sp.chi2_junction), rel_m(std::fabs(zmem), sp.z_membrane));
                if (c4 > sp.chi2_junction || std::fabs(zmem) > sp.z_membrane) {
                    gm_i[i].push_back({o, m_i});
                    continue;
                }
                SideCand cd;
                cd.i = i;
                cd.o = o;
                cd.t0s = (b.p_in[1] - p[1]) / (2.0 * a.sgn * sp.v_drift);
                // 4. the joint fit
                const int bi = trk_off[i], ni = trk_off[i + 1] - bi;
                const int bo = trk_off[o], no = trk_off[o + 1] - bo;
                std::vector<int32_t> jh(trk_hits + bo, trk_hits + bo + no);
                jh.insert(jh.end(), trk_hits + bi, trk_hits + bi + ni);
                if (!fit_t0(y, z, row, sec.data(), jh.data(), ni + no, no, cd.t0s, prm, sp, cd.p6, cd.C6, cd.chi2)) {
                    gm_i[i].push_back({o, m_i});
                    continue;
                }
                cd.dchi2 = cd.chi2 - a.chi2_in - b.chi2_in;
                m_i = std::min(m_i, rel_m(cd.dchi2, sp.chi2_joint));
                gm_i[i].push_back({o, m_i});
                if (cd.dchi2 > sp.chi2_joint) continue;
                cand_i[i].push_back(cd);
            }
        }
    }
    std::vector<SideCand> cand;
    for (auto& v : cand_i)
        for (auto& c : v) cand.push_back(c);
    // margins of the gate decisions reach both members
    std::vector<double> mrg2(T, std::numeric_limits<double>::infinity());
    for (int i = 0; i < T; ++i)
        for (const auto& om : gm_i[i]) {
            mrg2[i] = std::min(mrg2[i], om.second);
            mrg2[om.first] = std::min(mrg2[om.first], om.second);
        }
    // 5. mutual best by (dchi2 as FP32, partner index)
    using Key = std::pair<float, int>;
    const Key none{std::numeric_limits<float>::infinity(), std::numeric_limits<int>::max()};
    std::vector<Key> best(T, none), second(T, none);
    auto offer = [&](int t, Key k) {
        if (k < best[t]) {
            second[t] = best[t];
            best[t] = k;
        } else if (k < second[t]) {
            second[t] = k;
        }
    };
    for (const auto& c : cand) {
        offer(c.i, {(float)c.dchi2, c.o});
        offer(c.o, {(float)c.dchi2, c.i});
    }
    for (int t = 0; t < T; ++t)
        if (best[t].second != none.second && second[t].second != none.second)
            mrg2[t] = std::min(mrg2[t], rel_m(best[t].first, second[t].first));
    int64_t pairs = 0;
    for (const auto& c : cand) {
        if (best[c.i].second != c.o || best[c.o].second != c.i) continue;
        ++pairs;
        for (int t : {c.i, c.o}) {
            partner[t] = t == c.i ? c.o : c.i;
            t0o[t] = c.p6[5];
            for (int k = 0; k < 6; ++k) params6[t * 6 + k] = c.p6[k];
            for (int k = 0; k < 21; ++k) cov6[t * 21 + k] = c.C6[k];
            chi2o[t] = c.chi2;
            ndfo[t] = 2 * (trk_off[c.i + 1] - trk_off[c.i] + trk_off[c.o + 1] - trk_off[c.o]) - 6;
            dchi2o[t] = c.dchi2;
        }
    }
    if (margin)
        for (int t = 0; t < T; ++t) margin[t] = mrg2[t];
    return pairs;
}

}  // extern "C"
