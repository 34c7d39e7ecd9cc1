// NEXT-2: clusterization of pad-time digits (the paper's TPC clustering on
// the GPU, Sec. 4.2; its digit format is not given, this is the build's).
//
// Digits: u16 [planes][n_time][160], planes = events x 36 sectors x 152 pad
// rows, pads contiguous.  A tile is TT time bins of one plane plus two halo
// bins on each side: 36 consecutive time rows, one contiguous span of
// memory, moved into shared memory by one bulk asynchronous copy (TMA,
// cp.async.bulk with an mbarrier), three stages per block so that two
// tiles' copies run under the current tile's work.  Persistent blocks take
// tiles round robin.  In a tile every digit is tested for the raster peak
// rule; peaks are ranked in raster order by a block-wide ballot scan and
// their 5 x 5 integer sums and FP32 positions written to the tile's slots
// of the scratch.  A scan over the tiles' counts and one scatter pass then
// write the clusters in plane order, raster order within a plane: the same
// order and the same bits as the definition.
#include <algorithm>

#include "tpc_dev.cuh"

namespace tpc {

namespace {

constexpr int CNP = 160;               // pads per row plane
constexpr int CTT = 32;                // time bins per tile
constexpr int CHALO = 2;               // 5 x 5 window
constexpr int CTR = CTT + 2 * CHALO;   // time rows staged per tile
constexpr int CTHREADS = 128;
constexpr int CSTAGES = 3;             // tiles in shared memory per block (2 in flight ahead)
constexpr int CMAXP = 96;              // peak slots per tile
constexpr int CGROUPS = CNP / 8;       // 8-pad groups per time row
constexpr int CITEMS = CTT * CGROUPS;  // items (8 pads of one time row) per full tile
constexpr int CPER = CITEMS / CTHREADS;  // consecutive items per thread
static_assert(CITEMS % CTHREADS == 0, "whole items per thread");
constexpr unsigned CWAIT_LIMIT = 1u << 22;  // mbarrier polls before giving up

struct PeakRec {
    float y, z;
    uint32_t charge;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: false when the barrier did not complete within the limit
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    for (unsigned i = 0; i < CWAIT_LIMIT; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// one bulk copy global -> shared of `bytes` (a multiple of 16, both
// addresses 16-byte aligned), completing on `bar`
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

struct TileGeom {
    int plane;     // tiles number below 2^31 (checked at the call)
    int t0;        // first time bin of the tile
    int lo, hi;    // staged time rows [lo, hi) (clipped to [0, n_time))
};

__device__ __forceinline__ TileGeom tile_geom(int64_t tile, int n_tch, int n_time) {
    TileGeom g;
    const int t32 = (int)tile;
    g.plane = t32 / n_tch;
    g.t0 = (t32 - g.plane * n_tch) * CTT;
    g.lo = max(g.t0 - CHALO, 0);
    g.hi = min(g.t0 + CTT + CHALO, n_time);
    return g;
}

__global__ void __launch_bounds__(CTHREADS) k_clusterize(const uint16_t* __restrict__ digits, int n_time,
                                                         int64_t n_tiles, int n_tch, int q_peak,
                                                         PeakRec* __restrict__ recs, int32_t* __restrict__ cnt,
                                                         int32_t* st) {
    __shared__ __align__(128) uint16_t buf[CSTAGES][CTR * CNP];
    __shared__ __align__(8) uint64_t bar[CSTAGES];
    __shared__ int32_t wsum[CTHREADS / 32];
    __shared__ int32_t s_wc[CPER][CTHREADS / 32];
    __shared__ int32_t s_cand[CITEMS];
    __shared__ int16_t s_peak[CMAXP];
    __shared__ int32_t s_ncand;
    __shared__ int32_t s_count;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) {
        for (int k = 0; k < CSTAGES; ++k) mbar_init(&bar[k], 1);
        fence_async_shared();
    }
    __syncthreads();
    auto issue = [&](int64_t tile, int stage) {  // thread 0 only
        const TileGeom g = tile_geom(tile, n_tch, n_time);
        const unsigned bytes = (unsigned)(g.hi - g.lo) * CNP * 2u;
        const uint16_t* src = digits + ((size_t)g.plane * (size_t)n_time + (size_t)g.lo) * CNP;
        uint16_t* dst = buf[stage] + (g.lo - (g.t0 - CHALO)) * CNP;
        fence_async_shared();
        mbar_expect_tx(&bar[stage], bytes);
        bulk_load(dst, src, bytes, &bar[stage]);
    };
    int64_t tile = blockIdx.x;
    // prologue: the first CSTAGES tiles of this block in flight
    if (tid == 0)
        for (int k = 0; k < CSTAGES; ++k) {
            const int64_t tk = tile + (int64_t)k * gridDim.x;
            if (tk < n_tiles) issue(tk, k);
        }
    unsigned phase[CSTAGES];
    for (int k = 0; k < CSTAGES; ++k) phase[k] = 0u;
    for (int it = 0; tile < n_tiles; ++it, tile += gridDim.x) {
        const int stage = it % CSTAGES;
        if (!mbar_wait(&bar[stage], phase[stage])) {
            // give up: report, wait (bounded) for the copies in flight, leave
            if (tid == 0) set_status(st, TPC_ERR_TIMEOUT, 10);
            for (int k = 1; k < CSTAGES; ++k) {
                const int sk = (stage + k) % CSTAGES;
                if (tile + (int64_t)k * gridDim.x < n_tiles) mbar_wait(&bar[sk], phase[sk]);
            }
            return;
        }
        phase[stage] ^= 1u;
        const TileGeom g = tile_geom(tile, n_tch, n_time);
        uint16_t* b = buf[stage];
        // zero the halo rows outside the plane (first and last tiles only):
        // rows [0, lo - t0 + 2) and [hi - t0 + 2, CTR) of the stage
        {
            const int r_lo = g.lo - (g.t0 - CHALO), r_hi = g.hi - (g.t0 - CHALO);
            const int n_lo = r_lo * CNP, n_hi = (CTR - r_hi) * CNP;
            for (int i = tid; i < n_lo; i += CTHREADS) b[i] = 0;
            for (int i = tid; i < n_hi; i += CTHREADS) b[r_hi * CNP + i] = 0;
        }
        __syncthreads();
        auto at = [&](int r, int p) -> int {  // r: staged row, p: pad (0 outside)
            return (p < 0 || p >= CNP) ? 0 : (int)b[r * CNP + p];
        };
        const int t_end = min(CTT, n_time - g.t0);
        // items: 8 consecutive pads of one time row, raster order; thread
        // tid takes the CPER consecutive items from tid * CPER, so that a
        // scan of per-thread counts ranks the peaks in raster order
        const int n_items = t_end * CGROUPS;
        // phase 1: items (8 pads of one time row) with a digit at the
        // threshold, compacted in raster order; item k * CTHREADS + tid
        unsigned bal[CPER];
#pragma unroll
        for (int k = 0; k < CPER; ++k) {
            const int item = k * CTHREADS + tid;
            bool cand = false;
            if (item < n_items) {
                const int r = item / CGROUPS + CHALO, p0 = (item % CGROUPS) * 8;
                const uint4 v = *reinterpret_cast<const uint4*>(b + r * CNP + p0);
                const unsigned mx2 = __vmaxu2(__vmaxu2(v.x, v.y), __vmaxu2(v.z, v.w));
                cand = (int)max(mx2 & 0xffffu, mx2 >> 16) >= q_peak;
            }
            bal[k] = __ballot_sync(0xffffffffu, cand);
            if (lane == 0) s_wc[k][wid] = __popc(bal[k]);
        }
        __syncthreads();
        {
            int o = 0;
#pragma unroll
            for (int k = 0; k < CPER; ++k) {
                int ok_ = o;
#pragma unroll
                for (int w = 0; w < CTHREADS / 32; ++w) {
                    if (w < wid) ok_ += s_wc[k][w];
                    o += s_wc[k][w];
                }
                if (bal[k] & (1u << lane)) s_cand[ok_ + __popc(bal[k] & ((1u << lane) - 1u))] = k * CTHREADS + tid;
            }
            if (tid == 0) s_ncand = o;
        }
        __syncthreads();
        // phase 2: the peak test on the candidate items, one per thread;
        // peaks ranked in raster order by a scan of the per-item counts
        const int n_cand = s_ncand;
        int peaks_before = 0;
        for (int base = 0; base < n_cand; base += CTHREADS) {
            const int j = base + tid;
            unsigned mask = 0;
            int item = 0;
            if (j < n_cand) {
                item = s_cand[j];
                const int r = item / CGROUPS + CHALO, p0 = (item % CGROUPS) * 8;
                int w[3][10];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const uint16_t* rp = b + (r - 1 + d) * CNP;
                    const uint4 u = *reinterpret_cast<const uint4*>(rp + p0);
                    const unsigned u4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                    for (int e = 0; e < 8; ++e) w[d][e + 1] = (int)((u4[e >> 1] >> (16 * (e & 1))) & 0xffffu);
                    w[d][0] = p0 > 0 ? (int)rp[p0 - 1] : 0;
                    w[d][9] = p0 + 8 < CNP ? (int)rp[p0 + 8] : 0;
                }
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int q = w[1][e + 1];
                    const bool pk = (q >= q_peak) & (q > w[0][e]) & (q > w[0][e + 1]) & (q > w[0][e + 2]) &
                                    (q > w[1][e]) & (q >= w[1][e + 2]) & (q >= w[2][e]) & (q >= w[2][e + 1]) &
                                    (q >= w[2][e + 2]);
                    mask |= (unsigned)pk << e;
                }
            }
            const int c = __popc(mask);
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane == 31) wsum[wid] = incl;
            __syncthreads();
            int before = peaks_before + incl - c, total = 0;
#pragma unroll
            for (int w = 0; w < CTHREADS / 32; ++w) {
                if (w < wid) before += wsum[w];
                total += wsum[w];
            }
            while (mask) {
                const int e = __ffs(mask) - 1;
                mask &= mask - 1;
                if (before < CMAXP) s_peak[before] = (int16_t)(item * 8 + e);
                ++before;
            }
            peaks_before += total;
            __syncthreads();
        }
        if (peaks_before > CMAXP && tid == 0) set_status(st, TPC_ERR_CAPACITY, 11);
        const int n_pk = min(peaks_before, CMAXP);
        // phase 3: the 5 x 5 sums and positions of the peaks, one per thread
        const bool side_c = (g.plane / NROW) % NSEC >= NPHI;  // 32-bit
        for (int j = tid; j < n_pk; j += CTHREADS) {
            const int code = s_peak[j];
            const int item = code >> 3, e = code & 7;
            const int r = item / CGROUPS + CHALO, p = (item % CGROUPS) * 8 + e;
            int Q = 0, Sp = 0, St = 0;
#pragma unroll
            for (int dt = -2; dt <= 2; ++dt)
#pragma unroll
                for (int dp = -2; dp <= 2; ++dp) {
                    const int v = at(r + dt, p + dp);
                    Q += v;
                    Sp += v * dp;
                    St += v * dt;
                }
            const int t = g.t0 + r - CHALO;
            const float cp = __fadd_rn((float)p, __fdiv_rn((float)Sp, (float)Q));
            const float yy = __fmul_rn(__fsub_rn(cp, 79.5f), 0.6f);
            const float ct = __fadd_rn((float)t, __fdiv_rn((float)St, (float)Q));
            const float az = __fmul_rn(__fadd_rn(ct, 0.5f), 0.5f);
            recs[tile * CMAXP + j] = PeakRec{yy, side_c ? -az : az, (uint32_t)min(Q, 65535)};
        }
        const int total = n_pk;
        if (tid == 0) s_count = total;
        __syncthreads();
        if (tid == 0) {
            cnt[tile] = min(s_count, CMAXP);
            // every thread is done with this stage: its next tile may come
            const int64_t ahead = tile + (int64_t)CSTAGES * gridDim.x;
            if (ahead < n_tiles) issue(ahead, stage);
        }
    }
}

__global__ void k_cluster_write(const PeakRec* __restrict__ recs, const int32_t* __restrict__ cnt,
                                const int32_t* __restrict__ off, int64_t n_tiles, int n_tch, int64_t cap,
                                float* y, float* z, uint16_t* row, uint16_t* charge, int64_t* evt_sector_off,
                                int32_t G, int32_t* n_out, int32_t* st) {
    // one warp per tile
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w > n_tiles) return;
    if (w == n_tiles) {
        if (lane == 0) {
            const int64_t total = off[n_tiles];
            *n_out = (int32_t)(total < cap ? total : cap);
            if (total > cap) set_status(st, TPC_ERR_CAPACITY, 12);
        }
        return;
    }
    const int64_t plane = w / n_tch;
    if (w % ((int64_t)n_tch * NROW) == 0 && lane == 0) {
        const int64_t g = plane / NROW;
        const int64_t a = off[w], b = off[n_tiles];
        evt_sector_off[g] = a < cap ? a : cap;
        if (g == G - 1) evt_sector_off[G] = b < cap ? b : cap;
    }
    const int n = cnt[w];
    for (int k = lane; k < n; k += 32) {
        const int64_t o = (int64_t)off[w] + k;
        if (o >= cap) break;
        const PeakRec r = recs[w * CMAXP + k];
        y[o] = r.y;
        z[o] = r.z;
        row[o] = (uint16_t)(plane % NROW);
        charge[o] = (uint16_t)r.charge;
    }
}

__global__ void k_cluster_status(const int32_t* __restrict__ st, int32_t* out) {
    out[0] = st[0];
    out[1] = st[1];
}

struct ClusterLayout {
    int64_t n_tiles;
    size_t recs, cnt, off, scan, status, total;
};

ClusterLayout cluster_layout(int32_t n_events, int32_t n_time) {
    ClusterLayout L;
    const int n_tch = (n_time + CTT - 1) / CTT;
    L.n_tiles = (int64_t)n_events * NSEC * NROW * n_tch;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += (bytes + 255) & ~size_t(255);
        return at;
    };
    L.recs = take(sizeof(PeakRec) * (size_t)L.n_tiles * CMAXP);
    L.cnt = take(4 * (size_t)(L.n_tiles + 1));
    L.off = take(4 * (size_t)(L.n_tiles + 1));
    L.scan = take(4 * (size_t)(L.n_tiles / 4096 + 64));
    L.status = take(4 * 2);
    L.total = o;
    return L;
}

}  // namespace

}  // namespace tpc

using namespace tpc;

extern "C" size_t tpc_cluster_workspace_bytes(int32_t n_events, int32_t n_time) {
    if (n_events < 1 || n_time < 1 || n_time > 4096) return 0;
    const ClusterLayout L = cluster_layout(n_events, n_time);
    if (L.n_tiles * CMAXP >= ((int64_t)1 << 31)) return 0;
    return L.total;
}

extern "C" tpc_status tpc_find_clusters(const uint16_t* digits, int32_t n_events, int32_t n_time,
                                        int32_t q_peak, void* workspace, size_t workspace_bytes, float* y,
                                        float* z, uint16_t* row, uint16_t* charge, int64_t* evt_sector_off,
                                        int64_t cap, int32_t* n_clusters_dev, int32_t* status_dev,
                                        tpc_stream_t stream) {
    if (!digits || !workspace || !y || !z || !row || !charge || !evt_sector_off || !n_clusters_dev ||
        !status_dev || cap < 0 || q_peak < 1)
        return TPC_ERR_ARG;
    const size_t need = tpc_cluster_workspace_bytes(n_events, n_time);
    if (need == 0) return TPC_ERR_ARG;
    if (workspace_bytes < need) return TPC_ERR_CAPACITY;
    if (((uintptr_t)workspace & 255) != 0 || ((uintptr_t)digits & 15) != 0) return TPC_ERR_ARG;
    const ClusterLayout L = cluster_layout(n_events, n_time);
    char* ws = static_cast<char*>(workspace);
    auto* recs = reinterpret_cast<PeakRec*>(ws + L.recs);
    auto* cnt = reinterpret_cast<int32_t*>(ws + L.cnt);
    auto* off = reinterpret_cast<int32_t*>(ws + L.off);
    auto* scan = reinterpret_cast<int32_t*>(ws + L.scan);
    auto* st = reinterpret_cast<int32_t*>(ws + L.status);
    const cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 152;
    const int n_tch = (n_time + CTT - 1) / CTT;
    cudaError_t e = fill_i32(st, 2, 0, s);
    if (e == cudaSuccess) e = fill_i32(cnt, L.n_tiles + 1, 0, s);
    if (e != cudaSuccess) return TPC_ERR_CUDA;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(L.n_tiles, (int64_t)sms * 6));
    tpc::LaunchCount{}, k_clusterize<<<(unsigned)blocks, CTHREADS, 0, s>>>(digits, n_time, L.n_tiles, n_tch,
                                                                        q_peak, recs, cnt, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = scan_i32(cnt, off, L.n_tiles, scan, s);
    if (e == cudaSuccess) {
        const int64_t warps = L.n_tiles + 1;
        const int64_t wblocks = (warps * 32 + 255) / 256;
        tpc::LaunchCount{}, k_cluster_write<<<(unsigned)wblocks, 256, 0, s>>>(
            recs, cnt, off, L.n_tiles, n_tch, cap, y, z, row, charge, evt_sector_off, n_events * NSEC,
            n_clusters_dev, st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        tpc::LaunchCount{}, k_cluster_status<<<1, 1, 0, s>>>(st, status_dev);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? TPC_OK : TPC_ERR_CUDA;
}
