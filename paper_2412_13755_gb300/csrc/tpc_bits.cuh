// Helpers of the find kernels that are exact functions of their arguments:
// the row masks of the tracklet lanes, the neighbour window test and the
// triplet D^2 with its cut.  They compile for the device and, so that their
// index and rounding logic can be tested bit for bit without a GPU, for the
// host (the host arithmetic is IEEE binary32 with round to nearest; build
// such code without floating-point contraction).
#pragma once

#include <math.h>
#include <stdint.h>

#ifdef __CUDACC__
#define TPC_HD __host__ __device__ __forceinline__
#else
#define TPC_HD inline
#endif

namespace tpc {
namespace bits {

#if defined(__CUDA_ARCH__)
TPC_HD int clz32(uint32_t x) { return __clz(x); }
TPC_HD int ffs32(uint32_t x) { return __ffs(x); }
TPC_HD int popc32(uint32_t x) { return __popc(x); }
TPC_HD float add(float a, float b) { return __fadd_rn(a, b); }
TPC_HD float sub(float a, float b) { return __fsub_rn(a, b); }
TPC_HD float mul(float a, float b) { return __fmul_rn(a, b); }
TPC_HD float div(float a, float b) { return __fdiv_rn(a, b); }
TPC_HD float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
TPC_HD float rcp(float a) { return __frcp_rn(a); }
TPC_HD float sqrt(float a) { return __fsqrt_rn(a); }
#else
TPC_HD int clz32(uint32_t x) { return x ? __builtin_clz(x) : 32; }
TPC_HD int ffs32(uint32_t x) { return __builtin_ffs((int)x); }
TPC_HD int popc32(uint32_t x) { return __builtin_popcount(x); }
TPC_HD float add(float a, float b) { return a + b; }
TPC_HD float sub(float a, float b) { return a - b; }
TPC_HD float mul(float a, float b) { return a * b; }
TPC_HD float div(float a, float b) { return a / b; }
TPC_HD float fma(float a, float b, float c) { return fmaf(a, b, c); }
TPC_HD float rcp(float a) { return 1.0f / a; }
TPC_HD float sqrt(float a) { return sqrtf(a); }
#endif

}  // namespace bits

// ---- input validation (S0)

// One cluster is valid when its pad row exists (row < nrow) and both
// coordinates are finite.
TPC_HD bool cluster_valid(uint16_t row, float y, float z, int nrow) {
    return (int)row < nrow && isfinite(y) && isfinite(z);
}

// Check g (0 <= g <= G) of the group offsets off[0..G] over n clusters: 0
// when entry g is consistent, else -1 (off[0] != 0), -2 (off[G] != n) or -3
// (off[g + 1] < off[g]).  The offsets are a valid partition of [0, n) iff
// every g passes; then every group's range lies inside [0, n).
TPC_HD int offset_check(const int64_t* off, int G, int64_t n, int g) {
    const int64_t o = off[g];
    if (g == 0 && o != 0) return -1;
    if (g == G && o != n) return -2;
    if (g < G && off[g + 1] < o) return -3;
    return 0;
}

// ---- neighbour search (S2)

// window test, FP32, one rounding per operation
TPC_HD bool in_win(float xa, float ya, float za, float xb, float yb, float zb, float wy, float wz) {
    const float dx = fabsf(bits::sub(xb, xa));
    return fabsf(bits::sub(yb, ya)) <= bits::mul(wy, dx) && fabsf(bits::sub(zb, za)) <= bits::mul(wz, dx);
}

// Triplet D^2, FP32 with one rounding per operation: c is compared with
// the straight line from d to u at x_c, a = (x_c - x_d) / (x_u - x_d),
//   D^2 = ry^2 / (sy2 f) + rz^2 / (sz2 f),  f = 1 + a^2 + (1 - a)^2.
// The row-dependent part (a, f) is computed once per gap pair.  A pair with
// D^2 <= chi2 has ry^2 <= chi2 sy2 f and rz^2 <= chi2 sz2 f; tested with a
// relative margin of 1e-5 over the rounding, these bounds reject most pairs
// before the two divisions, and leave D^2 unchanged for the others.
struct TripletRows {
    float a, dy, dz, ty, tz;
};
TPC_HD TripletRows triplet_rows(float xd, float xc, float xu, float sy2, float sz2, float chi2) {
    TripletRows t;
    t.a = bits::div(bits::sub(xc, xd), bits::sub(xu, xd));
    const float b = bits::sub(1.0f, t.a);
    const float f = bits::add(bits::add(1.0f, bits::mul(t.a, t.a)), bits::mul(b, b));
    t.dy = bits::mul(sy2, f);
    t.dz = bits::mul(sz2, f);
    t.ty = bits::mul(bits::mul(chi2, t.dy), 1.00001f);
    t.tz = bits::mul(bits::mul(chi2, t.dz), 1.00001f);
    return t;
}
// D^2 of the triplet (d, c, u), or +inf where the bounds show D^2 > chi2
TPC_HD float triplet_d2_cut(const TripletRows& t, float yd, float zd, float yc, float zc, float yu, float zu) {
    const float ry = bits::sub(yc, bits::add(yd, bits::mul(t.a, bits::sub(yu, yd))));
    const float rz = bits::sub(zc, bits::add(zd, bits::mul(t.a, bits::sub(zu, zd))));
    const float ry2 = bits::mul(ry, ry), rz2 = bits::mul(rz, rz);
    if (ry2 > t.ty || rz2 > t.tz) return INFINITY;
    return bits::add(bits::div(ry2, t.dy), bits::div(rz2, t.dz));
}

// ---- row masks of the tracklet lanes (S3b)

// Rows holding a hit of a tracklet: bit r of the 160-bit mask m[0..4] (rows
// 0..151 used).  The word loops are unrolled, so that a mask in a kernel
// stays in registers.
constexpr int MASK_W = 5;
constexpr int MASK_NONE_ABOVE = 32 * MASK_W;  // mask_above's "no row"
// highest row below r with a hit, -1 if none
TPC_HD int mask_below(const uint32_t (&m)[MASK_W], int r) {
    int best = -1;
#pragma unroll
    for (int w = 0; w < MASK_W; ++w) {
        const int k = r - 32 * w;  // bits 0..k-1 of word w lie below r
        const uint32_t b = k <= 0 ? 0u : k >= 32 ? m[w] : m[w] & ((1u << k) - 1u);
        if (b) best = 32 * w + 31 - bits::clz32(b);
    }
    return best;
}
// lowest row above r with a hit, MASK_NONE_ABOVE if none
TPC_HD int mask_above(const uint32_t (&m)[MASK_W], int r) {
    int best = MASK_NONE_ABOVE;
#pragma unroll
    for (int w = MASK_W - 1; w >= 0; --w) {
        const int k = r + 1 - 32 * w;  // bits k..31 of word w lie above r
        const uint32_t b = k <= 0 ? m[w] : k >= 32 ? 0u : m[w] & ~((1u << k) - 1u);
        if (b) best = 32 * w + bits::ffs32(b) - 1;
    }
    return best;
}
// row of the j-th hit (from 0) counted from the top or from the bottom, -1
// if there are not that many
TPC_HD int mask_nth(const uint32_t (&m)[MASK_W], int j, bool from_top) {
    int row = -1, left = j;
#pragma unroll
    for (int i = 0; i < MASK_W; ++i) {
        const int w = from_top ? MASK_W - 1 - i : i;
        const uint32_t mw = from_top ? m[MASK_W - 1 - i] : m[i];  // static indices only
        const int c = bits::popc32(mw);
        if (row < 0) {
            if (left < c) {
                uint32_t b = mw;
                if (from_top) {
                    for (int t = 0; t < left; ++t) b &= ~(1u << (31 - bits::clz32(b)));
                    row = 32 * w + 31 - bits::clz32(b);
                } else {
                    for (int t = 0; t < left; ++t) b &= b - 1u;
                    row = 32 * w + bits::ffs32(b) - 1;
                }
            } else {
                left -= c;
            }
        }
    }
    return row;
}
TPC_HD void mask_set(uint32_t (&m)[MASK_W], int r) {
    const uint32_t bit = 1u << (r & 31);
    const int wr = r >> 5;
#pragma unroll
    for (int w = 0; w < MASK_W; ++w) m[w] |= wr == w ? bit : 0u;
}

// ---- distortion map voxels

// Voxel grid of a displacement field over the sector frames (the C ABI's
// tpc_field_grid).
struct FieldGridD {
    int n_band, n_y, n_z;
    float u_lo, u_inv, z_inv;
};

// bin of an FP32 coordinate already scaled to bin units, clamped to
// [0, nbin - 1] (NaN to 0)
TPC_HD int field_bin(float f, int nbin) {
    if (!(f >= 1.0f)) return 0;
    if (f >= (float)nbin) return nbin - 1;
    return (int)f;
}

// voxel of a cluster of sector sec on pad row r of n_rows (plane position
// rounded to FP32: xr) at local (y, z): the quotient y / xr, the difference
// and both products each rounded once
TPC_HD int field_voxel(float y, float z, int r, int n_rows, float xr, int sec, const FieldGridD& g) {
    const int band = r * g.n_band / n_rows;
    const float u = bits::div(y, xr);
    const int iy = field_bin(bits::mul(bits::sub(u, g.u_lo), g.u_inv), g.n_y);
    const int iz = field_bin(bits::mul(fabsf(z), g.z_inv), g.n_z);
    return ((sec * g.n_band + band) * g.n_y + iy) * g.n_z + iz;
}

}  // namespace tpc
