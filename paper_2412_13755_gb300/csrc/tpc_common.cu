// Shared device utilities: geometry table, status word, input validation,
// and a three-phase exclusive scan of int32 arrays.
#include <cmath>

#include "tpc_dev.cuh"

namespace tpc {

namespace {

__global__ void k_init_geo(Geo* geo, Geo g) { *geo = g; }

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_validate(const float* __restrict__ y, const float* __restrict__ z,
                           const uint16_t* __restrict__ row, int64_t n,
                           const int64_t* __restrict__ off, int G, int32_t* st) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tid <= G) {
        const int bad = offset_check(off, G, n, (int)tid);
        if (bad) reject_input(st, bad);
    }
    for (int64_t i = tid; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!cluster_valid(row[i], y[i], z[i], NROW)) reject_input(st, (int)(i & 0x7fffffff));
    }
}

constexpr int SCAN_T = 512;           // threads per scan block
constexpr int SCAN_I = 8;             // items per thread
constexpr int SCAN_B = SCAN_T * SCAN_I;

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t* sh, int32_t& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        int32_t s = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sh[lane] = s;
    }
    __syncthreads();
    const int32_t before = (wid > 0 ? sh[wid - 1] : 0) + x - v;
    total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(const int32_t* __restrict__ in, int64_t L,
                                                        int32_t* __restrict__ tmp) {
    __shared__ int32_t sh[32];
    const int64_t base = blockIdx.x * (int64_t)SCAN_B;
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k) {
        const int64_t i = base + k * SCAN_T + threadIdx.x;
        if (i < L) s += in[i];
    }
    int32_t tot;
    block_exclusive_scan(s, sh, tot);
    if (threadIdx.x == 0) tmp[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_top(int32_t* tmp, int64_t nb, int32_t* out_total) {
    __shared__ int32_t sh[32];
    int32_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
        const int64_t i = b0 + threadIdx.x;
        const int32_t v = i < nb ? tmp[i] : 0;
        int32_t tot;
        const int32_t ex = block_exclusive_scan(v, sh, tot);
        if (i < nb) tmp[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *out_total = carry;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_down(const int32_t* __restrict__ in, int64_t L,
                                                      const int32_t* __restrict__ tmp,
                                                      int32_t* __restrict__ out) {
    __shared__ int32_t sh[32];
    const int64_t base = blockIdx.x * (int64_t)SCAN_B + (int64_t)threadIdx.x * SCAN_I;
    int32_t v[SCAN_I];
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k) {
        const int64_t i = base + k;
        v[k] = i < L ? in[i] : 0;
        s += v[k];
    }
    int32_t tot;
    int32_t run = block_exclusive_scan(s, sh, tot) + tmp[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k) {
        const int64_t i = base + k;
        if (i < L) out[i] = run;
        run += v[k];
    }
}

}  // namespace

cudaError_t scan_i32(const int32_t* in, int32_t* out, int64_t L, int32_t* tmp, cudaStream_t s) {
    const int64_t nb = (L + SCAN_B - 1) / SCAN_B;
    if (nb > 0) {
        // the reduce pass reads items strided by SCAN_T; the down pass reads
        // them contiguously per thread: both cover the block's SCAN_B items
        tpc::LaunchCount{}, k_scan_reduce<<<(unsigned)nb, SCAN_T, 0, s>>>(in, L, tmp);
        tpc::LaunchCount{}, k_scan_top<<<1, 1024, 0, s>>>(tmp, nb, out + L);
        tpc::LaunchCount{}, k_scan_down<<<(unsigned)nb, SCAN_T, 0, s>>>(in, L, tmp, out);
    } else {
        tpc::LaunchCount{}, k_fill_i32<<<1, 32, 0, s>>>(out, 1, 0);
    }
    return cudaGetLastError();
}

cudaError_t fill_i32(int32_t* p, int64_t n, int32_t v, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
    tpc::LaunchCount{}, k_fill_i32<<<(unsigned)blocks, 256, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

cudaError_t init_geo(const Workspace& ws, cudaStream_t s) {
    const Geo g = make_geo();
    tpc::LaunchCount{}, k_init_geo<<<1, 1, 0, s>>>(ws.at<Geo>(ws.L.geo), g);
    return cudaGetLastError();
}

cudaError_t reset_status(const Workspace& ws, cudaStream_t s) {
    return fill_i32(ws.at<int32_t>(ws.L.status), ST_N_SLOTS, 0, s);
}

cudaError_t validate_clusters(const tpc_ctx* c, cudaStream_t s) {
    const int G = c->n_events * NSEC;
    const int64_t work = std::max<int64_t>(c->n, G + 1);
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 152 * 8));
    const cudaError_t e = fill_i32(c->ws.at<int32_t>(c->ws.L.status) + ST_INPUT_BAD, 1, 0, s);
    if (e != cudaSuccess) return e;
    tpc::LaunchCount{}, k_validate<<<(unsigned)blocks, 256, 0, s>>>(c->y, c->z, c->row, c->n, c->evt_sector_off, G,
                                                c->ws.at<int32_t>(c->ws.L.status));
    return cudaGetLastError();
}

}  // namespace tpc
