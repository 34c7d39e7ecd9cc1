// Host checks of the float-float arithmetic of the fit and the merge
// (tpc_ff.cuh).  Each operation is compared with the same operation in long
// double (at least 64 significant bits, so its own error is far below the
// bounds tested) on seeded random operands:
//   - TwoSum is exact: s + e equals a + b, and s = fl(a + b);
//   - every result is normalised: fl(hi + lo) = hi;
//   - add, fma_f and dot2 err by at most c u^2 times the sum of the absolute
//     values of their terms, mul, mul_f, rcp and sqrt by c u^2 relative,
//     u = 2^-24 the FP32 unit roundoff, c a small constant from counting the
//     roundings of each operation (stated at each check);
//   - the Cholesky chi2 d^T M^-1 d errs by at most 64 kappa u^2 relative,
//     kappa the condition number of M after the symmetric diagonal scaling
//     that makes its diagonal one (Cholesky is invariant under that scaling),
//     and it reports failure on a matrix with a negative eigenvalue; the
//     long-double Cholesky used as reference is itself checked against the
//     closed form of the random matrix's eigen-decomposition.
// Build without floating-point contraction.  Prints the worst observed error
// of each operation in units of u^2, then "ok" or the failures.
#include <cmath>
#include <cstdio>
#include <cstdint>

#include "tpc_ff.cuh"

using namespace tpc;
typedef long double ld;

static const ld U = 1.0L / 16777216.0L;  // 2^-24
static const ld U2 = U * U;

static uint64_t rng_state = 0x243f6a8885a308d3ull;
static uint64_t next_u64() {  // xorshift64*
    rng_state ^= rng_state >> 12;
    rng_state ^= rng_state << 25;
    rng_state ^= rng_state >> 27;
    return rng_state * 0x2545f4914f6cdd1dull;
}
static ld unit() { return (ld)(next_u64() >> 11) * (1.0L / 9007199254740992.0L); }  // [0, 1)
// a random value with 53 random significant bits, random sign, |x| in
// [2^e_lo, 2^e_hi)
static ld rand_val(int e_lo, int e_hi) {
    const int e = e_lo + (int)(next_u64() % (uint64_t)(e_hi - e_lo));
    const ld m = 1.0L + unit();
    return (next_u64() & 1 ? -1.0L : 1.0L) * std::ldexp(m, e);
}
static ff to_ff(ld x) {
    const float hi = (float)x;
    return ff{hi, (float)(x - (ld)hi)};
}
static ld val(ff x) { return (ld)x.hi + (ld)x.lo; }
static ff rand_ff(int e_lo, int e_hi) { return to_ff(rand_val(e_lo, e_hi)); }

static int failures = 0;
#define CHECK(cond, ...)                          \
    do {                                          \
        if (!(cond) && failures++ < 20) {         \
            std::printf("FAIL %s:", #cond);       \
            std::printf(" " __VA_ARGS__);         \
            std::printf("\n");                    \
        }                                         \
    } while (0)

static bool normalised(ff x) { return bits::add(x.hi, x.lo) == x.hi; }

struct Worst {
    const char* name;
    ld bound;  // in units of u^2
    ld worst = 0;
    void see(ld err_in_u2) {
        if (err_in_u2 > worst) worst = err_in_u2;
    }
    void report() {
        std::printf("%-10s worst %.3Lf u^2 (bound %.0Lf)\n", name, worst, bound);
        CHECK(worst <= bound, "%s: %.3Lf u^2 above the bound %.0Lf", name, worst, bound);
    }
};

static void check_two_sum() {
    // operands within 2^12 of each other in magnitude, so that a + b is
    // exact in long double and in double alike
    for (int t = 0; t < 200000; ++t) {
        const float a = (float)rand_val(-20, 20);
        const float b = (float)rand_val(-20, 20);
        const ff s = two_sum(a, b);
        CHECK(s.hi == bits::add(a, b), "two_sum hi %a + %a", a, b);
        CHECK((ld)s.hi + (ld)s.lo == (ld)a + (ld)b, "two_sum not exact %a + %a", a, b);
        const float big = std::fabs(a) >= std::fabs(b) ? a : b, small = std::fabs(a) >= std::fabs(b) ? b : a;
        const ff f = fast_two_sum(big, small);
        CHECK((ld)f.hi + (ld)f.lo == (ld)a + (ld)b, "fast_two_sum not exact %a + %a", a, b);
    }
}

static void check_ops() {
    // add: TwoSum of the high parts is exact; then the low parts' sum and
    // its addition to the error each round once, at most u (|x| + |y|) u;
    // the final FastTwoSum is exact: 2 u^2 plus the low parts' own share
    Worst w_add{"add", 3}, w_mul{"mul", 6}, w_mulf{"mul_f", 3}, w_fma{"fma_f", 6}, w_dot{"dot2", 8},
        w_rcp{"rcp", 8}, w_sqrt{"sqrt", 8};
    for (int t = 0; t < 400000; ++t) {
        const ff x = rand_ff(-30, 30), y = rand_ff(-30, 30);
        const ld X = val(x), Y = val(y);

        const ff s = ff_add(x, y);
        CHECK(normalised(s), "add not normalised");
        w_add.see(std::fabs(val(s) - (X + Y)) / ((std::fabs(X) + std::fabs(Y)) * U2));

        // mul: the TwoProduct of the high parts is exact; two fused
        // cross terms round once each (about u^2 |xy| each), the dropped
        // lo*lo term is at most u^2 |xy|
        const ff p = ff_mul(x, y);
        CHECK(normalised(p), "mul not normalised");
        w_mul.see(std::fabs(val(p) - X * Y) / (std::fabs(X * Y) * U2));

        const float f = (float)rand_val(-30, 30);
        const ff pf = ff_mul_f(x, f);
        CHECK(normalised(pf), "mul_f not normalised");
        w_mulf.see(std::fabs(val(pf) - X * (ld)f) / (std::fabs(X * (ld)f) * U2));

        // fma_f: the product's error term rounds once (2 u^2 |x f|), the
        // sums of the low parts twice (u^2 (|acc| + 2 |x f|) and
        // u^2 (|acc| + |x f|)): at most 5 u^2 of |acc| + |x f|
        const ff acc = rand_ff(-30, 30);
        const ff a = ff_fma_f(acc, x, f);
        CHECK(normalised(a), "fma_f not normalised");
        w_fma.see(std::fabs(val(a) - (val(acc) + X * (ld)f)) /
                  ((std::fabs(val(acc)) + std::fabs(X * (ld)f)) * U2));

        const ff x2 = rand_ff(-30, 30), y2 = rand_ff(-30, 30);
        const ff d = ff_dot2(x, y, x2, y2);
        CHECK(normalised(d), "dot2 not normalised");
        const ld D = X * Y + val(x2) * val(y2);
        w_dot.see(std::fabs(val(d) - D) / ((std::fabs(X * Y) + std::fabs(val(x2) * val(y2))) * U2));

        // rcp: one Newton step squares the FP32 reciprocal's error (u^2)
        // and the float-float steps add a few roundings of size u^2
        const ff r = ff_rcp(x);
        CHECK(normalised(r), "rcp not normalised");
        w_rcp.see(std::fabs(val(r) * X - 1.0L) / U2);

        // sqrt: Heron's step squares the FP32 root's error; the correction
        // is rounded once relative to itself (u times u)
        const ff ax = ff{std::fabs(x.hi), x.hi < 0 ? -x.lo : x.lo};
        const ff q = ff_sqrt(ax);
        CHECK(normalised(q), "sqrt not normalised");
        const ld Q = std::sqrt(val(ax));
        w_sqrt.see(std::fabs(val(q) - Q) / (Q * U2));
    }
    // cancellation: x + y with y close to -x stays within the same bound
    // relative to |x| + |y| (not relative to |x + y|)
    for (int t = 0; t < 100000; ++t) {
        const ld X = rand_val(-30, 30);
        const ld Y = -X * (1.0L + std::ldexp(rand_val(0, 1), -(int)(next_u64() % 40)));
        const ff x = to_ff(X), y = to_ff(Y);
        const ff s = ff_add(x, y);
        w_add.see(std::fabs(val(s) - (val(x) + val(y))) / ((std::fabs(val(x)) + std::fabs(val(y))) * U2));
    }
    w_add.report();
    w_mul.report();
    w_mulf.report();
    w_fma.report();
    w_dot.report();
    w_rcp.report();
    w_sqrt.report();
}

// d^T M^-1 d in long double by Cholesky (the same definition, at least 64 bits)
static bool chi2_ld(const ld M[5][5], const ld d[5], ld& out) {
    ld L[5][5] = {};
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j <= i; ++j) {
            ld acc = M[i][j];
            for (int l = 0; l < j; ++l) acc -= L[i][l] * L[j][l];
            if (i == j) {
                if (!(acc > 0)) return false;
                L[i][i] = std::sqrt(acc);
            } else {
                L[i][j] = acc / L[j][j];
            }
        }
    ld c2 = 0;
    ld v[5];
    for (int i = 0; i < 5; ++i) {
        ld acc = d[i];
        for (int l = 0; l < i; ++l) acc -= L[i][l] * v[l];
        v[i] = acc / L[i][i];
        c2 += v[i] * v[i];
    }
    out = c2;
    return true;
}

// a random orthogonal 5x5 as the product of five Householder reflections
static void rand_orth(ld Q[5][5]) {
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) Q[i][j] = i == j;
    for (int k = 0; k < 5; ++k) {
        ld v[5], n2 = 0;
        for (int i = 0; i < 5; ++i) {
            v[i] = 2 * unit() - 1;
            n2 += v[i] * v[i];
        }
        for (int i = 0; i < 5; ++i) {  // Q <- Q (I - 2 v v^T / |v|^2)
            ld qv = 0;
            for (int j = 0; j < 5; ++j) qv += Q[i][j] * v[j];
            for (int j = 0; j < 5; ++j) Q[i][j] -= 2 * qv * v[j] / n2;
        }
    }
}

static void check_chol() {
    ld worst = 0, worst_ref = 0;
    int n_indef = 0;
    for (int t = 0; t < 20000; ++t) {
        // S = Q diag(lambda) Q^T with eigenvalues spread over up to 10^6,
        // then M = D S D with a diagonal D over 10^-4 .. 10^2 (the mixed
        // units of a track covariance: cm, sin phi, tan lambda, q/pT)
        ld Q[5][5], lam[5], Dg[5], S[5][5], M[5][5];
        rand_orth(Q);
        const ld spread = std::pow(10.0L, 6 * unit());
        for (int i = 0; i < 5; ++i) lam[i] = std::pow(spread, unit());
        lam[0] = 1;
        lam[1] = spread;
        const bool indefinite = t % 10 == 9;
        if (indefinite) lam[2] = -lam[2];
        for (int i = 0; i < 5; ++i) Dg[i] = std::pow(10.0L, -4 + 6 * unit());
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) {
                ld s = 0;
                for (int k = 0; k < 5; ++k) s += Q[i][k] * lam[k] * Q[j][k];
                S[i][j] = s;
            }
        ff Mf[15], df[5];
        ld Mr[5][5], dr[5];
        for (int i = 0; i < 5; ++i)
            for (int j = i; j < 5; ++j) {
                Mf[sx(i, j)] = to_ff(Dg[i] * S[i][j] * Dg[j]);
                Mr[i][j] = Mr[j][i] = val(Mf[sx(i, j)]);  // the exact matrix the float-float code sees
            }
        for (int i = 0; i < 5; ++i) {
            df[i] = to_ff(Dg[i] * rand_val(-3, 3));
            dr[i] = val(df[i]);
        }
        ff c2;
        const bool ok = chol_chi2_ff(df, Mf, c2);
        ld ref;
        const bool ok_ref = chi2_ld(Mr, dr, ref);
        if (indefinite) {
            CHECK(!ok_ref, "reference Cholesky accepted an indefinite matrix");
            CHECK(!ok, "float-float Cholesky accepted an indefinite matrix");
            n_indef += !ok;
            continue;
        }
        CHECK(ok && ok_ref, "Cholesky failed on a positive definite matrix (spread %Lg)", spread);
        if (!(ok && ok_ref)) continue;
        // condition number of the unit-diagonal scaling of the rounded M:
        // the rounding changes the eigenvalues of S by far less than the
        // smallest one, so the construction's kappa is used
        ld s_min = lam[0], s_max = lam[0];
        for (int i = 0; i < 5; ++i) {
            s_min = std::fmin(s_min, lam[i]);
            s_max = std::fmax(s_max, lam[i]);
        }
        ld dmin = S[0][0], dmax = S[0][0];
        for (int i = 0; i < 5; ++i) {
            dmin = std::fmin(dmin, S[i][i]);
            dmax = std::fmax(dmax, S[i][i]);
        }
        // kappa of diag(S)^-1/2 S diag(S)^-1/2 is at most kappa(S) dmax / dmin
        const ld kappa = s_max / s_min * dmax / dmin;
        const ld e = std::fabs(val(c2) - ref) / (ref * kappa * U2);
        if (e > worst) worst = e;
        // the long-double reference against the closed form of the
        // construction, sum_k (Q^T D^-1 d)_k^2 / lambda_k, which differs only
        // by the rounding of M to float-float (about kappa u^2)
        ld closed = 0;
        for (int k = 0; k < 5; ++k) {
            ld w = 0;
            for (int i = 0; i < 5; ++i) w += Q[i][k] * dr[i] / Dg[i];
            closed += w * w / lam[k];
        }
        const ld e_ref = std::fabs(closed - ref) / (ref * kappa * U2);
        if (e_ref > worst_ref) worst_ref = e_ref;
    }
    std::printf("chol_chi2  worst %.3Lf kappa u^2 (bound 64); %d indefinite rejected\n", worst, n_indef);
    std::printf("reference  worst %.3Lf kappa u^2 from the closed form (bound 64)\n", worst_ref);
    CHECK(worst <= 64, "chol_chi2 error %.3Lf kappa u^2", worst);
    CHECK(worst_ref <= 64, "long-double reference off the closed form by %.3Lf kappa u^2", worst_ref);
}

int main() {
    check_two_sum();
    check_ops();
    check_chol();
    if (failures) {
        std::printf("%d failures\n", failures);
        return 1;
    }
    std::printf("ok\n");
    return 0;
}
