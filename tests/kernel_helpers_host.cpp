// Host checks of the find kernels' exact helpers (tpc_bits.cuh): the row
// masks against brute force, and the triplet D^2 cut against the uncut
// D^2 evaluated from its definition with the same FP32 operations.
// Build without floating-point contraction.  Prints "ok" or the failures.
#include <cstdio>
#include <cstdlib>

#include "tpc_bits.cuh"

using namespace tpc;

static uint64_t rng_state = 0x9e3779b97f4a7c15ull;
static uint64_t next_u64() {  // xorshift64*
    rng_state ^= rng_state >> 12;
    rng_state ^= rng_state << 25;
    rng_state ^= rng_state >> 27;
    return rng_state * 0x2545f4914f6cdd1dull;
}
static float uniform(float lo, float hi) { return lo + (hi - lo) * (float)((next_u64() >> 40) * (1.0 / 16777216.0)); }

static int failures = 0;
#define CHECK(cond, ...)                          \
    do {                                          \
        if (!(cond) && failures++ < 20) {         \
            std::printf("FAIL %s:", #cond);       \
            std::printf(" " __VA_ARGS__);         \
            std::printf("\n");                    \
        }                                         \
    } while (0)

static void check_masks() {
    const int rows = 152;
    for (int trial = 0; trial < 2000; ++trial) {
        bool set[160] = {};
        uint32_t m[MASK_W] = {0, 0, 0, 0, 0};
        const int density = (int)(next_u64() % 100);  // percent of rows with a hit
        for (int r = 0; r < rows; ++r)
            if ((int)(next_u64() % 100) < density) {
                set[r] = true;
                mask_set(m, r);
            }
        int n = 0;
        for (int r = 0; r < rows; ++r) n += set[r];
        int pc = 0;
        for (int w = 0; w < MASK_W; ++w) pc += bits::popc32(m[w]);
        CHECK(pc == n, "popcount %d vs %d", pc, n);
        for (int r = -1; r <= rows; ++r) {
            int below = -1, above = MASK_NONE_ABOVE;
            for (int q = r - 1; q >= 0; --q)
                if (set[q]) { below = q; break; }
            for (int q = r + 1; q < rows; ++q)
                if (set[q]) { above = q; break; }
            CHECK(mask_below(m, r) == below, "below(%d) = %d, want %d", r, mask_below(m, r), below);
            CHECK(mask_above(m, r) == above, "above(%d) = %d, want %d", r, mask_above(m, r), above);
        }
        int k = 0;
        for (int r = rows - 1; r >= 0; --r)
            if (set[r]) {
                CHECK(mask_nth(m, k, true) == r, "nth top %d = %d, want %d", k, mask_nth(m, k, true), r);
                ++k;
            }
        CHECK(mask_nth(m, n, true) == -1, "nth top past the end");
        k = 0;
        for (int r = 0; r < rows; ++r)
            if (set[r]) {
                CHECK(mask_nth(m, k, false) == r, "nth bottom %d = %d, want %d", k, mask_nth(m, k, false), r);
                ++k;
            }
        CHECK(mask_nth(m, n, false) == -1, "nth bottom past the end");
    }
}

// the triplet D^2 of its definition, FP32, one rounding per operation
static float d2_definition(float xd, float yd, float zd, float xc, float yc, float zc, float xu, float yu,
                           float zu, float sy2, float sz2) {
    const float a = (xc - xd) / (xu - xd);
    const float yh = yd + a * (yu - yd);
    const float zh = zd + a * (zu - zd);
    const float ry = yc - yh, rz = zc - zh;
    const float b = 1.0f - a;
    const float f = (1.0f + a * a) + b * b;
    return (ry * ry) / (sy2 * f) + (rz * rz) / (sz2 * f);
}

static void check_triplets() {
    const float sy2 = 0.01f, sz2 = 0.0225f, chi2 = 16.0f, pitch = (float)(162.0 / 151.0);
    long passed = 0, cut = 0;
    for (int trial = 0; trial < 400000; ++trial) {
        const int r = 3 + (int)(next_u64() % 146);
        const int gd = 1 + (int)(next_u64() % 3), gu = 1 + (int)(next_u64() % 3);
        const float xc = (float)(85.0 + r * (162.0 / 151.0));
        const float xd = (float)(85.0 + (r - gd) * (162.0 / 151.0));
        const float xu = (float)(85.0 + (r + gu) * (162.0 / 151.0));
        const float yc = uniform(-40.f, 40.f), zc = uniform(-250.f, 250.f);
        const float ty = uniform(-2.f, 2.f), tz = uniform(-3.f, 3.f);  // line slopes
        // scatter around the line: mostly near the cut, some far from it
        const float s = (next_u64() % 4 == 0) ? 5.f : 0.6f;
        const float yd = yc - ty * gd * pitch + uniform(-s, s), zd = zc - tz * gd * pitch + uniform(-s, s);
        const float yu = yc + ty * gu * pitch + uniform(-s, s), zu = zc + tz * gu * pitch + uniform(-s, s);
        const TripletRows t = triplet_rows(xd, xc, xu, sy2, sz2, chi2);
        const float got = triplet_d2_cut(t, yd, zd, yc, zc, yu, zu);
        const float want = d2_definition(xd, yd, zd, xc, yc, zc, xu, yu, zu, sy2, sz2);
        if (isinf(got)) {
            ++cut;
            CHECK(want > chi2, "a pair with D^2 %.9g <= %g was cut", want, chi2);
        } else {
            CHECK(got == want, "D^2 %.9g differs from the definition %.9g", got, want);
            passed += want <= chi2;
        }
    }
    std::printf("triplets: %ld within the cut, %ld rejected by the bounds\n", passed, cut);
    CHECK(passed > 1000 && cut > 1000, "both outcomes exercised");
}

// S0 validation: the per-entry offset checks all pass exactly when the
// offsets partition [0, n) (first 0, last n, non-decreasing), and a valid
// partition keeps every group's range inside [0, n); the cluster check
// rejects rows past the last and every non-finite coordinate.
static void check_validation() {
    for (int trial = 0; trial < 20000; ++trial) {
        const int G = 1 + (int)(next_u64() % 40);
        int64_t off[64];
        int64_t n = 0;
        off[0] = 0;
        for (int g = 0; g < G; ++g) off[g + 1] = off[g] + (int64_t)(next_u64() % 5);
        n = off[G];
        const int kind = (int)(next_u64() % 4);  // 0: valid; 1-3: one entry perturbed
        if (kind > 0) {
            const int g = (int)(next_u64() % (G + 1));
            off[g] += (int64_t)(next_u64() % 7) - 3;
        }
        if (next_u64() % 8 == 0) n += (int64_t)(next_u64() % 3) - 1;
        bool def = off[0] == 0 && off[G] == n;
        for (int g = 0; g < G; ++g) def = def && off[g + 1] >= off[g];
        bool pass = true;
        for (int g = 0; g <= G; ++g) pass = pass && offset_check(off, G, n, g) == 0;
        CHECK(pass == def, "offset check %d vs definition %d (G %d)", (int)pass, (int)def, G);
        if (pass)
            for (int g = 0; g < G; ++g) CHECK(off[g] >= 0 && off[g + 1] <= n, "group %d outside [0, n)", g);
    }
    const float inf = INFINITY, nan = NAN;
    CHECK(cluster_valid(0, 1.f, -2.f, 152), "row 0");
    CHECK(cluster_valid(151, 1e30f, -1e30f, 152), "row 151");
    CHECK(!cluster_valid(152, 1.f, 1.f, 152), "row 152");
    CHECK(!cluster_valid(65535, 1.f, 1.f, 152), "row 65535");
    CHECK(!cluster_valid(3, nan, 1.f, 152), "NaN y");
    CHECK(!cluster_valid(3, 1.f, nan, 152), "NaN z");
    CHECK(!cluster_valid(3, inf, 1.f, 152), "inf y");
    CHECK(!cluster_valid(3, 1.f, -inf, 152), "-inf z");
}

int main() {
    check_validation();
    check_masks();
    check_triplets();
    if (failures == 0) std::printf("ok\n");
    return failures == 0 ? 0 : 1;
}
