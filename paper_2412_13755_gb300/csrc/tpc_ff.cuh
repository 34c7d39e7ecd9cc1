// Float-float arithmetic (an FP32 pair hi + lo) and the packed 5x5
// symmetric index, for the device kernels and, so that their error bounds
// can be tested without a GPU, for the host.
#pragma once

#include "tpc_bits.cuh"

namespace tpc {

// Packed symmetric 5x5: 00 01 02 03 04 11 12 13 14 22 23 24 33 34 44.
// Closed form (row a of the upper triangle starts at 5a - a(a-1)/2), not
// recursive, so that constant indices fold at compile time and the packed
// arrays stay in registers.
TPC_HD constexpr int sx(int i, int j) {
    return (i <= j ? i : j) * 5 - (i <= j ? i : j) * ((i <= j ? i : j) - 1) / 2 + (i <= j ? j : i) -
           (i <= j ? i : j);
}
static_assert(sx(0, 0) == 0 && sx(0, 4) == 4 && sx(1, 1) == 5 && sx(2, 1) == 6 && sx(2, 2) == 9 &&
                  sx(3, 3) == 12 && sx(4, 3) == 13 && sx(4, 4) == 14,
              "packed index");

// ---- float-float covariance --------------------------------------------
// A covariance entry as an unevaluated sum hi + lo of two FP32 numbers
// (about 48 significant bits), updated with error-free transformations:
// TwoSum (Knuth) for sums and TwoProduct through the fused multiply-add for
// products.  Every operation is an explicitly rounded intrinsic on the
// device (plain IEEE operations on the host, built without contraction), so
// the compiler cannot contract them into other fused operations.  The Kalman update C - K H C cancels by orders of magnitude once
// a track is well measured; FP32 storage loses the small directions there,
// while GB300's FP64 rate is a small fraction of its FP32 rate.
struct ff {
    float hi, lo;
};
TPC_HD ff ff_from(float a) { return ff{a, 0.f}; }
// a + b exactly as s + e (Knuth's TwoSum)
TPC_HD ff two_sum(float a, float b) {
    const float s = bits::add(a, b);
    const float v = bits::sub(s, a);
    return ff{s, bits::add(bits::sub(a, bits::sub(s, v)), bits::sub(b, v))};
}
// a + b = s + e for |a| >= |b| (Dekker's FastTwoSum)
TPC_HD ff fast_two_sum(float a, float b) {
    const float s = bits::add(a, b);
    return ff{s, bits::sub(b, bits::sub(s, a))};
}
// x + y (the lo parts added in FP32, then renormalised)
TPC_HD ff ff_add(ff x, ff y) {
    ff s = two_sum(x.hi, y.hi);
    s.lo = bits::add(s.lo, bits::add(x.lo, y.lo));
    return fast_two_sum(s.hi, s.lo);
}
TPC_HD ff ff_neg(ff x) { return ff{-x.hi, -x.lo}; }
// x * f for an FP32 f: TwoProduct of the hi part (exact through the FMA)
TPC_HD ff ff_mul_f(ff x, float f) {
    const float p = bits::mul(x.hi, f);
    const float e = bits::fma(x.lo, f, bits::fma(x.hi, f, -p));
    return fast_two_sum(p, e);
}
TPC_HD ff ff_mul(ff x, ff y) {
    const float p = bits::mul(x.hi, y.hi);
    float e = bits::fma(x.hi, y.hi, -p);
    e = bits::fma(x.hi, y.lo, e);
    e = bits::fma(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}
// 1 / x: an FP32 reciprocal refined by one Newton step r + r (1 - x r)
// carried in float-float
TPC_HD ff ff_rcp(ff x) {
    const float r = bits::rcp(x.hi);
    const ff xr = ff_mul_f(x, r);
    const ff one_minus = ff_add(ff_from(1.f), ff_neg(xr));
    return ff_add(ff_from(r), ff_mul_f(one_minus, r));
}
// acc + x * f: the product's error term joins the sum's low part, with one
// renormalisation at the end
TPC_HD ff ff_fma_f(ff acc, ff x, float f) {
    const float p = bits::mul(x.hi, f);
    const float e = bits::fma(x.lo, f, bits::fma(x.hi, f, -p));
    const ff s = two_sum(acc.hi, p);
    return fast_two_sum(s.hi, bits::add(s.lo, bits::add(acc.lo, e)));
}
// x1 y1 + x2 y2 in float-float: both products as (p, e) with p = fl(x.hi
// y.hi) and e the rest (TwoProduct through the FMA, plus the cross terms),
// the two p summed exactly and the errors added to the low part
TPC_HD ff ff_dot2(ff x1, ff y1, ff x2, ff y2) {
    const float p1 = bits::mul(x1.hi, y1.hi), p2 = bits::mul(x2.hi, y2.hi);
    const float e1 = bits::fma(x1.lo, y1.hi, bits::fma(x1.hi, y1.lo, bits::fma(x1.hi, y1.hi, -p1)));
    const float e2 = bits::fma(x2.lo, y2.hi, bits::fma(x2.hi, y2.lo, bits::fma(x2.hi, y2.hi, -p2)));
    const ff s = two_sum(p1, p2);
    return fast_two_sum(s.hi, bits::add(s.lo, bits::add(e1, e2)));
}

// sqrt(x) for x > 0: the FP32 root refined by one Newton (Heron) step
// s + (x - s^2) / (2 s), the residual x - s^2 formed exactly with TwoProduct
TPC_HD ff ff_sqrt(ff x) {
    const float s = bits::sqrt(x.hi);
    const float p = bits::mul(s, s);
    const float pe = bits::fma(s, s, -p);
    const ff r = ff_add(x, ff{-p, -pe});
    return fast_two_sum(s, bits::div(r.hi, bits::mul(2.f, s)));
}

// chi2 = d^T M^-1 d for a 5x5 symmetric positive definite M (packed upper
// triangle) by Cholesky factorisation and forward substitution, in
// float-float.  Returns false when a pivot is not positive.
TPC_HD bool chol_chi2_ff(const ff d[5], const ff M[15], ff& out) {
    ff Lm[5][5], inv[5];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            ff acc = M[sx(i, j)];
#pragma unroll
            for (int l = 0; l < j; ++l) acc = ff_add(acc, ff_neg(ff_mul(Lm[i][l], Lm[j][l])));
            if (i == j) {
                if (!(acc.hi > 0.f)) return false;
                Lm[i][i] = ff_sqrt(acc);
                inv[i] = ff_rcp(Lm[i][i]);
            } else {
                Lm[i][j] = ff_mul(acc, inv[j]);
            }
        }
    ff v[5], c2 = ff_from(0.f);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        ff acc = d[i];
#pragma unroll
        for (int l = 0; l < i; ++l) acc = ff_add(acc, ff_neg(ff_mul(Lm[i][l], v[l])));
        v[i] = ff_mul(acc, inv[i]);
        c2 = ff_add(c2, ff_mul(v[i], v[i]));
    }
    out = c2;
    return true;
}

}  // namespace tpc
