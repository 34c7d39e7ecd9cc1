// The distortion-map voxel of each cluster by the kernels' helper
// (tpc_bits.cuh, field_voxel), compiled for the host.  Reads from the file
// named by argv[1]: n (int64), the grid (3 int32, 3 float), the pad-row
// plane positions rounded to FP32 (152 floats), then y[n], z[n] (float),
// row[n] (uint16), sector[n] (int32); writes vox[n] (int32) to argv[2].
// Build without floating-point contraction.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "tpc_bits.cuh"

using namespace tpc;

template <class T>
static bool rd(FILE* f, T* p, size_t n) { return fread(p, sizeof(T), n, f) == n; }

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    int64_t n;
    int32_t gi[3];
    float gf[3], xr[152];
    if (!rd(f, &n, 1) || !rd(f, gi, 3) || !rd(f, gf, 3) || !rd(f, xr, 152) || n < 0) return 3;
    std::vector<float> y(n), z(n);
    std::vector<uint16_t> row(n);
    std::vector<int32_t> sec(n), vox(n);
    if (!rd(f, y.data(), n) || !rd(f, z.data(), n) || !rd(f, row.data(), n) || !rd(f, sec.data(), n))
        return 3;
    fclose(f);
    const FieldGridD g{gi[0], gi[1], gi[2], gf[0], gf[1], gf[2]};
    for (int64_t i = 0; i < n; ++i) {
        if (row[i] >= 152) return 4;
        vox[i] = field_voxel(y[i], z[i], row[i], 152, xr[row[i]], sec[i], g);
    }
    FILE* o = fopen(argv[2], "wb");
    if (!o || fwrite(vox.data(), sizeof(int32_t), n, o) != (size_t)n) return 5;
    fclose(o);
    printf("ok\n");
    return 0;
}
