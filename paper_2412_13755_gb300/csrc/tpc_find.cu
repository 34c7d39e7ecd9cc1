// S1-S4 of the tracking path: (row, z cell, y cell) binning, cellular-automaton
// neighbour finding, chaining, Kalman-guided tracklet construction and
// selection, segment merging across sectors, and the canonical track output.
//
// Integer decisions that floating point takes in the neighbour step (window
// cuts, triplet D^2 and its comparisons) are evaluated in FP32 with explicit
// round-to-nearest intrinsics (no contraction), so they are bit-identical to
// an FP32 evaluation of the same formula on any IEEE machine.  Every tie is
// broken by the clusters' input indices (canonical ids), so the output does
// not depend on the order in which the GPU visits clusters.
#include <algorithm>
#include <type_traits>

#include <cooperative_groups.h>

#include "tpc_bits.cuh"
#include "tpc_dev.cuh"

namespace tpc {

namespace {

constexpr int TPB = 256;
constexpr uint64_t KEY_MAX = ~0ull;

inline unsigned grid_for(int64_t n, int per = TPB) {
    const int64_t b = (n + per - 1) / per;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152LL * 64));
}

__device__ __forceinline__ uint32_t f2o(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float o2f(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

struct Cells {  // per-group z-cell description
    const float* zmin;
    const float* inv;
    const int32_t* nz;
    const int32_t* kbase;
    const int32_t* off;  // cell offsets into the binned arrays
};

// Self-check: an index outside [0, bound) is reported in the status word
// (TPC_ERR_STATE, detail = site) and the caller skips the access.
__device__ __forceinline__ bool in_range(int64_t i, int64_t bound, int32_t* st, int site) {
    if (i >= 0 && i < bound) return true;
    set_status(st, TPC_ERR_STATE, site);
    return false;
}

// Kept tracklets are binned per group by the row bucket of their outer end
// (MRB rows per bucket) and, within it, by the z of their outer end.
struct TlBins {  // per-group (outer row bucket, z) bins of the kept tracklets' outer ends
    const float* zmin;
    const float* inv;
    const int32_t* nb;
    const int32_t* base;
};

__device__ __forceinline__ int tl_bin(const TlBins& t, int g, float z) {
    const int nb = t.nb[g];
    const float f = (z - t.zmin[g]) * t.inv[g];
    int k = f >= 0.f ? (int)f : 0;  // monotone in z
    return k < nb - 1 ? k : nb - 1;
}

__device__ __forceinline__ int zcell(const Cells& c, int g, float z) {
    const int nz = c.nz[g];
    const float f = (z - c.zmin[g]) * c.inv[g];
    int k = f >= 0.f ? (int)f : 0;  // monotone in z
    return k < nz - 1 ? k : nz - 1;
}

// y cell of row r: uniform in y / (x_r tan 10 deg) over the acceptance,
// clamped (monotone in y)
__device__ __forceinline__ int ycell(const Geo* __restrict__ geo, int r, float y) {
    const float f = y * geo->ycell_inv[r] + 0.5f * CELL_NY;
    const int k = f >= 0.f ? (int)f : 0;
    return k < CELL_NY - 1 ? k : CELL_NY - 1;
}

// The cells of row r (group g) covering z in [zlo, zhi] and y in [ylo, yhi]:
// one contiguous run of binned clusters per z cell,
// [off[base + iz * CELL_NY + iy0], off[base + iz * CELL_NY + iy1 + 1]) for
// iz0 <= iz <= iz1.
struct CellWin {
    int base, iz0, iz1, iy0, iy1;
};
__device__ __forceinline__ CellWin cell_win(const Cells& cells, const Geo* __restrict__ geo, int g, int r,
                                            float zlo, float zhi, float ylo, float yhi) {
    CellWin w;
    w.base = cells.kbase[g] + r * cells.nz[g] * CELL_NY;
    w.iz0 = zcell(cells, g, zlo);
    w.iz1 = zcell(cells, g, zhi);
    w.iy0 = ycell(geo, r, ylo);
    w.iy1 = ycell(geo, r, yhi);
    return w;
}
__device__ __forceinline__ void cell_run(const Cells& cells, const CellWin& w, int iz, int& b, int& e) {
    b = cells.off[w.base + iz * CELL_NY + w.iy0];
    e = cells.off[w.base + iz * CELL_NY + w.iy1 + 1];
}

// ---------------------------------------------------------------- S1 ------
__global__ void k_zrange(const float* __restrict__ z, int64_t n, const int64_t* __restrict__ off,
                         int G, uint32_t* zmin_u, uint32_t* zmax_u, int32_t* grp_of,
                        const int32_t* __restrict__ st) {
    if (input_rejected(st)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int g = group_of(off, G, i);
        grp_of[i] = g;
        const uint32_t o = f2o(z[i]);
        // lanes of one group combine before the atomics
        const unsigned act = __activemask();
        const unsigned same = __match_any_sync(act, g);
        const uint32_t mn = __reduce_min_sync(same, o);
        const uint32_t mx = __reduce_max_sync(same, o);
        if ((threadIdx.x & 31) == (__ffs(same) - 1)) {
            atomicMin(&zmin_u[g], mn);
            atomicMax(&zmax_u[g], mx);
        }
    }
}

// one block: z cells per group and their key bases
__global__ void __launch_bounds__(1024) k_cells(const int64_t* __restrict__ off, int G,
                                                const uint32_t* zmin_u, const uint32_t* zmax_u,
                                                float* zmin, float* inv, int32_t* nz,
                                                int32_t* kbase, int64_t Kcap, int32_t* st) {
    if (input_rejected(st)) return;
    __shared__ int32_t sh[32];
    __shared__ int64_t carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int g0 = 0; g0 < G; g0 += blockDim.x) {
        const int g = g0 + threadIdx.x;
        int32_t cnt = 0;
        if (g < G) {
            const int64_t ng = off[g + 1] - off[g];
            int64_t k = ng / (NROW * CELL_OCC * CELL_NY);
            k = k < 1 ? 1 : (k > NZ_MAX ? NZ_MAX : k);
            float lo = 0.f, hi = 0.f;
            if (ng > 0) {
                lo = o2f(zmin_u[g]);
                hi = o2f(zmax_u[g]);
            }
            const float w = hi - lo;
            // z cells of at least ZCELL_MIN cm: a dense group (a pile-up
            // frame) gets fuller cells rather than windows over many runs
            const int64_t kz = (int64_t)(w / ZCELL_MIN) + 1;
            k = k < kz ? k : kz;
            zmin[g] = lo;
            inv[g] = w > 0.f ? (float)k / w : 0.f;
            nz[g] = (int32_t)k;
            cnt = (int32_t)(NROW * CELL_NY * k);
        }
        // block exclusive scan of cnt
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        int32_t x = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sh[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int32_t s = sh[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            sh[lane] = s;
        }
        __syncthreads();
        const int64_t base = carry_s;
        const int32_t ex = (wid > 0 ? sh[wid - 1] : 0) + x - cnt;
        if (g < G) kbase[g] = (int32_t)(base + ex);
        const int32_t tot = sh[31];
        __syncthreads();
        if (threadIdx.x == 0) carry_s = base + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        kbase[G] = (int32_t)carry_s;
        if (carry_s > Kcap) set_status(st, TPC_ERR_CAPACITY, 1);
    }
}

// one block: tracklet z bins per group (<= 16 cm wide; at most
// 1 + n_g/64 bins so that the total is bounded by the cluster count)
__global__ void __launch_bounds__(1024) k_tl_bins(const int64_t* __restrict__ off, int G,
                                                  const uint32_t* zmin_u, const uint32_t* zmax_u,
                                                  float* zmin, float* inv, int32_t* nb,
                                                  int32_t* base,
                        const int32_t* __restrict__ st) {
    if (input_rejected(st)) return;
    __shared__ int32_t sh[32];
    __shared__ int64_t carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int g0 = 0; g0 < G; g0 += blockDim.x) {
        const int g = g0 + threadIdx.x;
        int32_t cnt = 0;
        if (g < G) {
            const int64_t ng = off[g + 1] - off[g];
            float lo = 0.f, hi = 0.f;
            if (ng > 0) {
                lo = o2f(zmin_u[g]);
                hi = o2f(zmax_u[g]);
            }
            const float w = hi - lo;
            int64_t k = (int64_t)ceilf(w / 16.f);
            const int64_t kmax = 1 + ng / 64;
            k = k < 1 ? 1 : (k > kmax ? kmax : k);
            zmin[g] = lo;
            inv[g] = w > 0.f ? (float)k / w : 0.f;
            nb[g] = (int32_t)k;
            cnt = (int32_t)(NMRB * k);
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        int32_t x = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sh[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int32_t v = sh[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            sh[lane] = v;
        }
        __syncthreads();
        const int64_t b0 = carry_s;
        const int32_t ex = (wid > 0 ? sh[wid - 1] : 0) + x - cnt;
        if (g < G) base[g] = (int32_t)(b0 + ex);
        const int32_t tot = sh[31];
        __syncthreads();
        if (threadIdx.x == 0) carry_s = b0 + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) base[G] = (int32_t)carry_s;
}

__global__ void k_hist(const float* __restrict__ y, const float* __restrict__ z,
                       const uint16_t* __restrict__ row, int64_t n,
                       const int32_t* __restrict__ grp_of, Cells cells, const Geo* __restrict__ geo,
                       int32_t* cnt, int32_t* key_in, int32_t* slot_in, int64_t Kcap,
                        const int32_t* __restrict__ st) {
    if (input_rejected(st)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int g = grp_of[i];
        const int r = row[i];
        const int key = cells.kbase[g] + (r * cells.nz[g] + zcell(cells, g, z[i])) * CELL_NY + ycell(geo, r, y[i]);
        int slot = 0;
        if (key >= 0 && key < Kcap) slot = atomicAdd(&cnt[key], 1);
        key_in[i] = key;
        slot_in[i] = slot;
    }
}

__global__ void k_scatter(const float* __restrict__ y, const float* __restrict__ z,
                          const uint16_t* __restrict__ row, int64_t n,
                          const int32_t* __restrict__ grp_of,
                          const int32_t* __restrict__ key_in, const int32_t* __restrict__ slot_in,
                          const int32_t* __restrict__ cell_off, int64_t Kcap, float2* yzb,
                          int32_t* orig, int32_t* grpb, uint8_t* rowb,
                        const int32_t* __restrict__ st) {
    if (input_rejected(st)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int key = key_in[i];
        if (key < 0 || key >= Kcap) continue;
        const int64_t pos = cell_off[key] + slot_in[i];
        yzb[pos] = make_float2(y[i], z[i]);
        orig[pos] = (int32_t)i;
        grpb[pos] = grp_of[i];
        rowb[pos] = (uint8_t)row[i];
    }
}

// ---------------------------------------------------------------- S2 ------
struct NbPrm {
    float win_y, win_z, chi2_link, sy2, sz2;
    int max_gap;
};

// The cells holding every candidate of row rr that can pass in_win for the
// cluster at (xc, yc, zc): the window half-widths win_y |dx|, win_z |dx|
// widened by a relative 1e-4 and 1e-3 cm against rounding.
__device__ __forceinline__ CellWin nb_win(const Cells& cells, const Geo* __restrict__ geo, int g, int rr,
                                          float xr, float xc, float yc, float zc, const NbPrm& P) {
    const float dx = fabsf(__fsub_rn(xr, xc));
    const float wz = __fmul_rn(P.win_z, dx) * 1.0001f + 1e-3f;
    const float wy = __fmul_rn(P.win_y, dx) * 1.0001f + 1e-3f;
    return cell_win(cells, geo, g, rr, zc - wz, zc + wz, yc - wy, yc + wy);
}

// Serial evaluation of one gap pair (gd, gu) for cluster c; the reference
// used by the warp kernel when a candidate list overflows.
__device__ void pair_scan_serial(int64_t c, int gd, int gu, const float2* __restrict__ yzb,
                                 const int32_t* __restrict__ orig,
                                 int g, int r, float xc, float yc, float zc, const Cells& cells,
                                 const Geo* __restrict__ geo, const NbPrm& P, int& bd, int& bu,
                                 float& bd2) {
    const int rd = r - gd, ru = r + gu;
    const float xd = geo->row_xf[rd], xu = geo->row_xf[ru];
    const CellWin wd = nb_win(cells, geo, g, rd, xd, xc, yc, zc, P);
    const CellWin wu = nb_win(cells, geo, g, ru, xu, xc, yc, zc, P);
    const TripletRows tr = triplet_rows(xd, xc, xu, P.sy2, P.sz2, P.chi2_link);
    int pd = -1, pu = -1, pod = 0, pou = 0;
    float pd2 = 0.f;
    for (int izd = wd.iz0; izd <= wd.iz1; ++izd) {
      int db, de;
      cell_run(cells, wd, izd, db, de);
      for (int d = db; d < de; ++d) {
        const float2 vd = yzb[d];
        const float ydd = vd.x, zdd = vd.y;
        if (!in_win(xc, yc, zc, xd, ydd, zdd, P.win_y, P.win_z)) continue;
        for (int izu = wu.iz0; izu <= wu.iz1; ++izu) {
          int ub, ue;
          cell_run(cells, wu, izu, ub, ue);
          for (int u = ub; u < ue; ++u) {
            const float2 vu = yzb[u];
            const float yuu = vu.x, zuu = vu.y;
            if (!in_win(xc, yc, zc, xu, yuu, zuu, P.win_y, P.win_z)) continue;
            const float d2 = triplet_d2_cut(tr, ydd, zdd, yc, zc, yuu, zuu);
            if (!(d2 <= P.chi2_link)) continue;
            bool better = pd < 0 || d2 < pd2;
            if (!better && d2 == pd2) {
                const int ou = orig[u], od = orig[d];
                better = ou < pou || (ou == pou && od < pod);
            }
            if (better) {
                pd = d; pu = u; pd2 = d2; pod = orig[d]; pou = orig[u];
            }
          }
        }
      }
    }
    bd = pd;
    bu = pu;
    bd2 = pd2;
}

constexpr int NB_LIST = 64;     // candidates kept per row and cluster
constexpr int NB_WARPS = 8;     // warps per block
struct NbLists {
    float y[6][NB_LIST];
    float z[6][NB_LIST];
    int idx[6][NB_LIST];
    int cnt[6];
};

// Neighbour search by sub-warps of NG lanes, one cluster per sub-warp
// (same rule and result as the serial search).  The admissible window
// candidates of each needed row offset (down rows r-1..r-3 -> lists 0..2, up
// rows r+1..r+3 -> lists 3..5) are compacted into the sub-warp's shared
// memory lists once; the lanes then evaluate the (down, up) pairs of each gap
// pair in order and reduce to the best pair (smallest D^2, then canonical id
// of u, then of d).  A cluster whose needed list exceeds NS_CAP entries is
// queued for the full-warp kernel below, which redoes it.
constexpr int NG2 = 8;         // lanes per cluster, later gap pairs
constexpr int NB_GAP_MAX = 3;  // largest gap of the neighbour search (tpc_params.max_gap <= 3)
constexpr int NS_CAP = 24;     // list capacity per row offset (<= 254)
// warps per block of the sub-warp kernel: NG, so that the lists of its
// 32 clusters per block take the same shared memory for every NG
template <int NG> __host__ __device__ constexpr int ns_warps() { return NG; }
struct NsLists {
    float y[6][NS_CAP];
    float z[6][NS_CAP];
    int idx[6][NS_CAP];
};
// The kernel takes the clusters of one or two queues, each from its own
// first gap sum (sum_lo, sum_lo_b) up to sum_hi: the clusters whose
// first-pass up list overflowed from (1, 1) on, and those the first pass
// left without a pair from sum 3 on.  The gap pairs keep their order, so the
// result is the one of a single serial search.  With next_queue set, a
// cluster still without a pair after sum_hi is queued there instead of being
// written.
template <int NG>
__global__ void __launch_bounds__(ns_warps<NG>() * 32) k_neighbours_sub(
    int64_t n, const int32_t* __restrict__ in_queue, int in_slot, int sum_lo, int sum_hi,
    const float2* __restrict__ yzb,
    const int32_t* __restrict__ orig, const int32_t* __restrict__ grpb,
    const uint8_t* __restrict__ rowb, Cells cells, const Geo* __restrict__ geo, NbPrm P,
    int32_t* choice_dn, int32_t* choice_up, float* d2out, int32_t* st, int32_t* ovf_queue,
    int32_t* next_queue, int next_slot, const int32_t* __restrict__ in_queue_b, int in_slot_b,
    int sum_lo_b) {
    if (input_rejected(st)) return;
    constexpr int GPW = 32 / NG;  // clusters per warp
    __shared__ NsLists sh_all[ns_warps<NG>() * GPW];
    const int lane = threadIdx.x & 31;
    const int gq = lane / NG, li = lane % NG;
    const unsigned gm = ((1u << NG) - 1u) << (gq * NG);
    const unsigned lt = (1u << li) - 1u;
    NsLists& sh = sh_all[(threadIdx.x >> 5) * GPW + gq];
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // items: the first queue, then (optionally) a second queue that starts
    // at gap sum sum_lo_b
    const int64_t nin_a = in_queue ? (int64_t)st[in_slot] : n;
    const int64_t nin = nin_a + (in_queue_b ? (int64_t)st[in_slot_b] : 0);
    const int sum_end = min(sum_hi, 2 * P.max_gap);
    for (int64_t c0 = wid * GPW; c0 < nin; c0 += nw * GPW) {
        if (c0 + gq >= nin) continue;  // the whole sub-warp leaves together
        const int64_t item = c0 + gq;
        const bool from_b = item >= nin_a;
        const int64_t c = from_b ? in_queue_b[item - nin_a] : in_queue ? in_queue[item] : item;
        const int s_lo = from_b ? sum_lo_b : sum_lo;
        const int g = grpb[c], r = rowb[c];
        const float2 vc = yzb[c];
        const float xc = geo->row_xf[r], yc = vc.x, zc = vc.y;
        // list k: bit k of `built`; its count (capped at NS_CAP + 1) in bits 8k..8k+7 of `cnts`
        unsigned built = 0;
        uint64_t cnts = 0;
        int bd = -1, bu = -1;
        float bd2 = 0.f;
        bool ovf = false;
        for (int sum = s_lo; sum <= sum_end && bd < 0 && !ovf; ++sum) {
            for (int gu = 1; gu <= P.max_gap && bd < 0 && !ovf; ++gu) {
                const int gd = sum - gu;
                if (gd < 1 || gd > P.max_gap) continue;
                const int rd = r - gd, ru = r + gu;
                if (rd < 0 || ru >= NROW) continue;
                const int kd = gd - 1, ku = 2 + gu;
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    const int k = side == 0 ? kd : ku;
                    if (built & (1u << k)) continue;
                    const int rr = side == 0 ? rd : ru;
                    const float xr = geo->row_xf[rr];
                    const CellWin w = nb_win(cells, geo, g, rr, xr, xc, yc, zc, P);
                    int cnt = 0;
                    for (int iz = w.iz0; iz <= w.iz1; ++iz) {
                        int b, e;
                        cell_run(cells, w, iz, b, e);
                        for (int base = b; base < e; base += NG) {
                            const int q = base + li;
                            float yq = 0.f, zq = 0.f;
                            bool pass = false;
                            if (q < e) {
                                const float2 vq = yzb[q];
                                yq = vq.x;
                                zq = vq.y;
                                pass = in_win(xc, yc, zc, xr, yq, zq, P.win_y, P.win_z);
                            }
                            const unsigned bal = (__ballot_sync(gm, pass) >> (gq * NG)) & ((1u << NG) - 1u);
                            const int pos = cnt + __popc(bal & lt);
                            if (pass && pos < NS_CAP) {
                                sh.idx[k][pos] = q;
                                sh.y[k][pos] = yq;
                                sh.z[k][pos] = zq;
                            }
                            cnt += __popc(bal);
                        }
                    }
                    built |= 1u << k;
                    cnts |= (uint64_t)min(cnt, NS_CAP + 1) << (8 * k);
                }
                __syncwarp(gm);
                const int nd = (int)((cnts >> (8 * kd)) & 255u), nu = (int)((cnts >> (8 * ku)) & 255u);
                if (nd == 0 || nu == 0) continue;
                if (nd > NS_CAP || nu > NS_CAP) {
                    ovf = true;
                    break;
                }
                const float xd = geo->row_xf[rd], xu = geo->row_xf[ru];
                const TripletRows tr = triplet_rows(xd, xc, xu, P.sy2, P.sz2, P.chi2_link);
                int pd = -1, pu = -1, pod = 0, pou = 0;
                float pd2 = 0.f;
                const int total = nd * nu;
                const float rnu = 1.f / (float)nu;
                for (int pp = li; pp < total; pp += NG) {
                    // pp / nu: pp < 2^16, so the rounded quotient is exact
                    const int i = (int)(((float)pp + 0.5f) * rnu), j = pp - i * nu;
                    const float d2 = triplet_d2_cut(tr, sh.y[kd][i], sh.z[kd][i], yc, zc, sh.y[ku][j], sh.z[ku][j]);
                    if (!(d2 <= P.chi2_link)) continue;
                    const int d = sh.idx[kd][i], u = sh.idx[ku][j];
                    bool better = pd < 0 || d2 < pd2;
                    if (!better && d2 == pd2) {
                        const int ou = orig[u], od = orig[d];
                        better = ou < pou || (ou == pou && od < pod);
                    }
                    if (better) {
                        pd = d; pu = u; pd2 = d2; pod = orig[d]; pou = orig[u];
                    }
                }
                // sub-warp argmin of (D^2, canonical u, canonical d)
#pragma unroll
                for (int o = NG / 2; o >= 1; o >>= 1) {
                    const int od_ = __shfl_xor_sync(gm, pd, o);
                    const int ou_ = __shfl_xor_sync(gm, pu, o);
                    const float o2 = __shfl_xor_sync(gm, pd2, o);
                    const int ood = __shfl_xor_sync(gm, pod, o);
                    const int oou = __shfl_xor_sync(gm, pou, o);
                    const bool take = od_ >= 0 && (pd < 0 || o2 < pd2 ||
                                                   (o2 == pd2 && (oou < pou || (oou == pou && ood < pod))));
                    if (take) {
                        pd = od_; pu = ou_; pd2 = o2; pod = ood; pou = oou;
                    }
                }
                if (pd >= 0) {
                    bd = pd;
                    bu = pu;
                    bd2 = pd2;
                }
                __syncwarp(gm);
            }
        }
        if (li == 0) {
            if (ovf) {
                ovf_queue[atomicAdd(&st[ST_NB_OVF], 1)] = (int32_t)c;
            } else if (bd < 0 && next_queue && sum_end < 2 * P.max_gap) {
                next_queue[atomicAdd(&st[next_slot], 1)] = (int32_t)c;  // later gap pairs
            } else {
                choice_dn[c] = bd;
                choice_up[c] = bu;
                d2out[c] = bd2;
            }
        }
        __syncwarp(gm);
    }
}

// First gap pair (1, 1), one lane per cluster.  The admissible up
// candidates (row r+1) go into a register list of NF entries; the down
// candidates (row r-1) stream from their cells, each paired with the list.
// A cluster without a pair here is queued for the later gap pairs
// (k_neighbours_sub, pass 2); one whose up list would overflow is queued for
// the sub-warp kernel from the first gap pair on (longer lists).
constexpr int NF = 6;
__global__ void __launch_bounds__(256, 4) k_neighbours_first(
    int64_t n, const float2* __restrict__ yzb,
    const int32_t* __restrict__ orig, const int32_t* __restrict__ grpb,
    const uint8_t* __restrict__ rowb, Cells cells, const Geo* __restrict__ geo, NbPrm P,
    int32_t* choice_dn, int32_t* choice_up, float* d2out, int32_t* st, int32_t* dense_queue,
    int32_t* next_queue, int next_slot) {
    if (input_rejected(st)) return;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int g = grpb[c], r = rowb[c];
        if (r < 1 || r + 1 >= NROW) {
            next_queue[atomicAdd(&st[next_slot], 1)] = (int32_t)c;
            continue;
        }
        const float2 vc = yzb[c];
        const float xc = geo->row_xf[r], yc = vc.x, zc = vc.y;
        const float xd = geo->row_xf[r - 1], xu = geo->row_xf[r + 1];
        // up list
        float uy[NF], uz[NF];
        int ui[NF];
        int nu = 0;
        const CellWin wu = nb_win(cells, geo, g, r + 1, xu, xc, yc, zc, P);
        for (int iz = wu.iz0; iz <= wu.iz1; ++iz) {
            int b, e;
            cell_run(cells, wu, iz, b, e);
            for (int q = b; q < e; ++q) {
                const float2 vq = yzb[q];
                const float yq = vq.x, zq = vq.y;
                if (!in_win(xc, yc, zc, xu, yq, zq, P.win_y, P.win_z)) continue;
#pragma unroll
                for (int k = 0; k < NF; ++k)
                    if (k == nu) {
                        uy[k] = yq;
                        uz[k] = zq;
                        ui[k] = q;
                    }
                ++nu;
            }
        }
        if (nu > NF) {
            dense_queue[atomicAdd(&st[ST_NB_Q3], 1)] = (int32_t)c;
            continue;
        }
        int bd = -1, bu = -1, pod = 0, pou = 0;
        float bd2 = 0.f;
        if (nu > 0) {
            const TripletRows tr = triplet_rows(xd, xc, xu, P.sy2, P.sz2, P.chi2_link);
            const CellWin wd = nb_win(cells, geo, g, r - 1, xd, xc, yc, zc, P);
            for (int iz = wd.iz0; iz <= wd.iz1; ++iz) {
                int b, e;
                cell_run(cells, wd, iz, b, e);
                for (int d = b; d < e; ++d) {
                    const float2 vd = yzb[d];
                    const float ydd = vd.x, zdd = vd.y;
                    if (!in_win(xc, yc, zc, xd, ydd, zdd, P.win_y, P.win_z)) continue;
#pragma unroll
                    for (int k = 0; k < NF; ++k) {
                        if (k >= nu) break;
                        const float d2 = triplet_d2_cut(tr, ydd, zdd, yc, zc, uy[k], uz[k]);
                        if (!(d2 <= P.chi2_link)) continue;
                        const int u = ui[k];
                        bool better = bd < 0 || d2 < bd2;
                        if (!better && d2 == bd2) {
                            const int ou = orig[u], od = orig[d];
                            better = ou < pou || (ou == pou && od < pod);
                        }
                        if (better) {
                            bd = d; bu = u; bd2 = d2; pod = orig[d]; pou = orig[u];
                        }
                    }
                }
            }
        }
        if (bd < 0 && 2 * P.max_gap > 2) {
            next_queue[atomicAdd(&st[next_slot], 1)] = (int32_t)c;
            continue;
        }
        choice_dn[c] = bd;
        choice_up[c] = bu;
        d2out[c] = bd2;
    }
}

// Warp-cooperative neighbour search for the queued clusters (same rule and
// result): one warp per cluster; the window candidates of each needed row
// offset are compacted into shared memory once, then the lanes evaluate the
// (down, up) pairs of a gap pair in parallel and reduce to the best pair
// (smallest D^2, then canonical id of u, then of d).
__global__ void __launch_bounds__(NB_WARPS * 32) k_neighbours_warp(
    const int32_t* __restrict__ queue, const int32_t* __restrict__ st,
    const float2* __restrict__ yzb,
    const int32_t* __restrict__ orig, const int32_t* __restrict__ grpb,
    const uint8_t* __restrict__ rowb, Cells cells, const Geo* __restrict__ geo, NbPrm P,
    int32_t* choice_dn, int32_t* choice_up, float* d2out) {
    if (input_rejected(st)) return;
    __shared__ NbLists sh_all[NB_WARPS];
    NbLists& sh = sh_all[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nq = st[ST_NB_OVF];
    for (int64_t qi = wid; qi < nq; qi += nw) {
        const int64_t c = queue[qi];
        const int g = grpb[c], r = rowb[c];
        const float2 vc = yzb[c];
        const float xc = geo->row_xf[r], yc = vc.x, zc = vc.y;
        unsigned built = 0;  // bit k: list k (k < 3: down rows r-1-k, k >= 3: up rows r+k-2)
        int bd = -1, bu = -1;
        float bd2 = 0.f;
        for (int sum = 2; sum <= 2 * P.max_gap && bd < 0; ++sum) {
            for (int gu = 1; gu <= P.max_gap && bd < 0; ++gu) {
                const int gd = sum - gu;
                if (gd < 1 || gd > P.max_gap) continue;
                const int rd = r - gd, ru = r + gu;
                if (rd < 0 || ru >= NROW) continue;
                const int kd = gd - 1, ku = 2 + gu;
                // build the two lists if needed
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    const int k = side == 0 ? kd : ku;
                    if (built & (1u << k)) continue;
                    const int rr = side == 0 ? rd : ru;
                    const float xr = geo->row_xf[rr];
                    const CellWin w = nb_win(cells, geo, g, rr, xr, xc, yc, zc, P);
                    int cnt = 0;
                    for (int iz = w.iz0; iz <= w.iz1; ++iz) {
                        int b, e;
                        cell_run(cells, w, iz, b, e);
                        for (int base = b; base < e; base += 32) {
                            const int q = base + lane;
                            float yq = 0.f, zq = 0.f;
                            bool pass = false;
                            if (q < e) {
                                const float2 vq = yzb[q];
                                yq = vq.x;
                                zq = vq.y;
                                pass = in_win(xc, yc, zc, xr, yq, zq, P.win_y, P.win_z);
                            }
                            const unsigned bal = __ballot_sync(0xffffffffu, pass);
                            const int pos = cnt + __popc(bal & lt);
                            if (pass && pos < NB_LIST) {
                                sh.idx[k][pos] = q;
                                sh.y[k][pos] = yq;
                                sh.z[k][pos] = zq;
                            }
                            cnt += __popc(bal);
                        }
                    }
                    if (lane == 0) sh.cnt[k] = cnt;
                    built |= 1u << k;
                }
                __syncwarp();
                const int nd = sh.cnt[kd], nu = sh.cnt[ku];
                if (nd == 0 || nu == 0) continue;
                if (nd > NB_LIST || nu > NB_LIST) {
                    // overflow: the serial scan of this gap pair
                    int sd = -1, su = -1;
                    float s2 = 0.f;
                    if (lane == 0)
                        pair_scan_serial(c, gd, gu, yzb, orig, g, r, xc, yc, zc, cells, geo, P, sd, su, s2);
                    bd = __shfl_sync(0xffffffffu, sd, 0);
                    bu = __shfl_sync(0xffffffffu, su, 0);
                    bd2 = __shfl_sync(0xffffffffu, s2, 0);
                    continue;
                }
                const float xd = geo->row_xf[rd], xu = geo->row_xf[ru];
                const TripletRows tr = triplet_rows(xd, xc, xu, P.sy2, P.sz2, P.chi2_link);
                int pd = -1, pu = -1, pod = 0, pou = 0;
                float pd2 = 0.f;
                const int total = nd * nu;
                for (int p = lane; p < total; p += 32) {
                    const int i = p / nu, j = p - i * nu;
                    const float d2 = triplet_d2_cut(tr, sh.y[kd][i], sh.z[kd][i], yc, zc, sh.y[ku][j], sh.z[ku][j]);
                    if (!(d2 <= P.chi2_link)) continue;
                    const int d = sh.idx[kd][i], u = sh.idx[ku][j];
                    bool better = pd < 0 || d2 < pd2;
                    if (!better && d2 == pd2) {
                        const int ou = orig[u], od = orig[d];
                        better = ou < pou || (ou == pou && od < pod);
                    }
                    if (better) {
                        pd = d; pu = u; pd2 = d2; pod = orig[d]; pou = orig[u];
                    }
                }
                // warp argmin of (D^2, canonical u, canonical d)
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) {
                    const int od_ = __shfl_xor_sync(0xffffffffu, pd, o);
                    const int ou_ = __shfl_xor_sync(0xffffffffu, pu, o);
                    const float o2 = __shfl_xor_sync(0xffffffffu, pd2, o);
                    const int ood = __shfl_xor_sync(0xffffffffu, pod, o);
                    const int oou = __shfl_xor_sync(0xffffffffu, pou, o);
                    bool take = od_ >= 0 && (pd < 0 || o2 < pd2 ||
                                             (o2 == pd2 && (oou < pou || (oou == pou && ood < pod))));
                    if (take) {
                        pd = od_; pu = ou_; pd2 = o2; pod = ood; pou = oou;
                    }
                }
                if (pd >= 0) {
                    bd = pd;
                    bu = pu;
                    bd2 = pd2;
                }
                __syncwarp();
            }
        }
        if (lane == 0) {
            choice_dn[c] = bd;
            choice_up[c] = bu;
            d2out[c] = bd2;
        }
        __syncwarp();
    }
}

__device__ __forceinline__ uint64_t claim_key(float d2, int32_t orig) {
    return ((uint64_t)__float_as_uint(d2) << 32) | (uint32_t)orig;
}

// endpoints without a triplet of their own accept their best claimant
__global__ void k_claims(int64_t n, const int32_t* __restrict__ cdn, const int32_t* __restrict__ cup,
                         const float* __restrict__ d2, const int32_t* __restrict__ orig,
                         unsigned long long* claim_up, unsigned long long* claim_dn,
                        const int32_t* __restrict__ st) {
    if (input_rejected(st)) return;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int u = cup[c], d = cdn[c];
        if (u < 0) continue;
        const unsigned long long key = claim_key(d2[c], orig[c]);
        if (cdn[u] < 0) atomicMin(&claim_up[u], key);
        if (cup[d] < 0) atomicMin(&claim_dn[d], key);
    }
}

// links: mutual choices, or the winning claim of an endpoint
__global__ void k_links(int64_t n, const int32_t* __restrict__ cdn, const int32_t* __restrict__ cup,
                        const float* __restrict__ d2, const int32_t* __restrict__ orig,
                        const unsigned long long* __restrict__ claim_up,
                        const unsigned long long* __restrict__ claim_dn, int32_t* link_dn,
                        int32_t* link_up,
                        const int32_t* __restrict__ st) {
    if (input_rejected(st)) return;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int u = cup[c], d = cdn[c];
        if (u < 0) continue;
        const unsigned long long key = claim_key(d2[c], orig[c]);
        const int cu = cdn[u];
        if (cu == (int)c || (cu < 0 && claim_up[u] == key)) {
            link_up[c] = u;
            link_dn[u] = (int32_t)c;
        }
        const int cd = cup[d];
        if (cd == (int)c || (cd < 0 && claim_dn[d] == key)) {
            link_dn[c] = d;
            link_up[d] = (int32_t)c;
        }
    }
}

// ---------------------------------------------------------------- S3 ------
// Chains of links from their lower ends; each one of at least n_seg
// clusters takes a segment slot, whose row table (the chain's cluster per
// row, -1 elsewhere) and row mask it writes for the tracklet lanes.
__global__ void k_chains(int64_t n, const int32_t* __restrict__ link_dn,
                         const int32_t* __restrict__ link_up, const int32_t* __restrict__ orig,
                         const int32_t* __restrict__ grpb, const uint8_t* __restrict__ rowb, int n_seg,
                         int64_t Scap, int32_t* seg_start, int32_t* seg_grp, int32_t* seg_canon,
                         int32_t* tl_rowhit, uint4* tl_mask, int32_t* st) {
    if (input_rejected(st)) return;
    // warp-uniform loop: a warp takes 32 consecutive clusters, and the
    // slots of its chains are consecutive (one atomic per warp), so the slot
    // order follows the binned order of the chain starts within a warp
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t c0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); c0 < n;
         c0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = c0 + lane;
        const bool start = c < n && link_dn[c] < 0 && link_up[c] >= 0;
        int len = 0, cur = (int)c;
        int32_t mn = 0x7fffffff;
        if (start) {
            while (cur >= 0 && len <= NROW) {
                mn = min(mn, orig[cur]);
                ++len;
                cur = link_up[cur];
            }
        }
        const bool qual = start && len >= n_seg;
        const unsigned bal = __ballot_sync(0xffffffffu, qual);
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(&st[ST_NSEG], __popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (!qual) continue;
        const int slot = base + __popc(bal & lt);
        if (slot >= Scap) {
            set_status(st, TPC_ERR_CAPACITY, 2);
            continue;
        }
        seg_start[slot] = (int32_t)c;
        seg_grp[slot] = grpb[c];
        seg_canon[slot] = mn;
        int32_t* hit = tl_rowhit + (int64_t)slot * NROW;
        int4* h4 = reinterpret_cast<int4*>(hit);  // NROW * 4 bytes per slot: 16-byte aligned
        for (int i = 0; i < NROW / 4; ++i) h4[i] = make_int4(-1, -1, -1, -1);
        uint32_t m0 = 0, m1 = 0, m2 = 0, m3 = 0, m4 = 0;
        cur = (int)c;
        for (int k = 0; k < len; ++k) {
            const int rr = rowb[cur];
            hit[rr] = cur;
            const uint32_t bit = 1u << (rr & 31);
            const int w = rr >> 5;
            m0 |= w == 0 ? bit : 0u;
            m1 |= w == 1 ? bit : 0u;
            m2 |= w == 2 ? bit : 0u;
            m3 |= w == 3 ? bit : 0u;
            m4 |= w == 4 ? bit : 0u;
            cur = link_up[cur];
        }
        tl_mask[2 * (int64_t)slot] = make_uint4(m0, m1, m2, m3);
        tl_mask[2 * (int64_t)slot + 1] = make_uint4(m4, 0u, 0u, 0u);
    }
}

// ---------------------------------------------------------------- S3b -----
struct TlPrm {
    float sy2, sz2, chi2_ext, kb, snp_max, fp64_ratio, fp64_det, pitch;
    int ext_max_miss, n_seg;
    double bz, seed_snp, seed_qpt;
    float prior[5];
};

// Three-point seed (FP32) of a tracklet's hits for one fit direction:
// first, middle (n/2-th in fit order) and last hit.
__device__ __forceinline__ void seed_mask(const int32_t* hit, const uint32_t (&m)[MASK_W], int rmin, int rmax,
                                          int n, bool inward, const float2* __restrict__ yzb, int sector,
                                          const Geo* __restrict__ geo, const TlPrm& P, KF& s) {
    int rows[3];
    rows[0] = inward ? rmax : rmin;
    rows[1] = mask_nth(m, n / 2, inward);
    rows[2] = inward ? rmin : rmax;
    int h[3];
    float ys[3], zs[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) h[i] = hit[rows[i]];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float2 v = __ldg(&yzb[h[i]]);
        ys[i] = v.x;
        zs[i] = v.y;
    }
    kf_seed_f(s, rows, sector, ys, zs, inward, geo, P.kb, (float)P.seed_snp, (float)P.seed_qpt, P.prior);
}

// Tracklet lanes.  Every lane owns one slot at a time and runs a small state
// machine, one Kalman step per loop iteration, so that the lanes of a warp
// execute the same transport / update code:
//   build:  inward fit of the chain -> inward extension -> the state moved
//           to the outermost hit row -> outward extension
//   refit:  inward fit of the kept hits (state at the innermost) -> the
//           state moved to the outermost hit row (state there)
// An outward fit of all hits stands in for the moved state only when the
// inward fit or the move fails; a failed fit skips its extension.
// Extension: in each row the cluster with the smallest predicted-residual
// chi2 (ties: smaller canonical id) if <= chi2_ext; stop after ext_max_miss
// empty rows, at the last row, on a transport failure, or when the
// prediction leaves the row's acceptance.  Finished lanes take the next slot
// from an atomic work queue.
// The slot's row table and row mask are prepared before the launch (by the
// chain kernel for the build, by the keep kernel for the refit); a lane
// keeps the mask in registers, so that the next hit row of a fit is known
// without a load and the hit's coordinates are fetched before the transport.
// PH_TO_OUTER is the move of the inward state to the outermost hit row, run
// as a step so that it shares the transport with the other lanes' steps.
enum { PH_FIT_IN = 0, PH_EXT_IN = 1, PH_FIT_OUT = 2, PH_EXT_OUT = 3, PH_TO_OUTER = 6 };
constexpr int EXT_ZB = 2;  // z cells of an extension window read in one batch
constexpr int EXT_CH = 4;  // candidate loads in flight per lane

__global__ void __launch_bounds__(128, 4) k_tracklet_lanes(
    int refit, const int32_t* __restrict__ items, int count_slot, const int32_t* __restrict__ seg_grp,
    const int32_t* __restrict__ seg_canon, const float2* __restrict__ yzb, const int32_t* __restrict__ orig,
    Cells cells, const Geo* __restrict__ geo, TlPrm P, int64_t Scap, int32_t* st, int32_t* tl_rowhit,
    const uint4* __restrict__ tl_mask, int32_t* tl_n, unsigned long long* tl_key, float* tl_state,
    int32_t* tl_ok, int4* gs_meta, int tile) {
    if (input_rejected(st)) return;
    const int nitems = min((int64_t)st[count_slot], Scap);
    int32_t* queue = &st[refit ? ST_Q_REFIT : ST_Q_BUILD];
    int s = -1, item = 0, phase = 0, r = 0, rmin = 0, rmax = 0, n = 0, misses = 0, g = 0, sector = 0, ok = 0;
    int xr = 0;  // row plane of the state (the state never leaves its sector)
    int steps = 0;
    // z cells of the slot's group
    float gz0 = 0.f, ginv = 0.f;
    int gnz = 1, gkb = 0;
    int t_next = 0, t_end = 0;  // slots of the current ticket
    int32_t* hit = nullptr;
    uint32_t m[MASK_W];
    KF kf;
    for (;;) {
        if (s < 0) {
            // take the next slot (a ticket covers `tile` consecutive items)
            if (t_next >= t_end) {
                t_next = atomicAdd(queue, tile);
                t_end = t_next + tile;
            }
            item = t_next++;
            if (item >= nitems) break;
            s = items ? items[item] : item;
            hit = tl_rowhit + (int64_t)s * NROW;
            g = seg_grp[s];
            sector = g % NSEC;
            ok = 0;
            gz0 = cells.zmin[g];
            ginv = cells.inv[g];
            gnz = cells.nz[g];
            gkb = cells.kbase[g];
            const uint4 ma = tl_mask[2 * (int64_t)s], mb = tl_mask[2 * (int64_t)s + 1];
            m[0] = ma.x;
            m[1] = ma.y;
            m[2] = ma.z;
            m[3] = ma.w;
            m[4] = mb.x;
            n = __popc(m[0]) + __popc(m[1]) + __popc(m[2]) + __popc(m[3]) + __popc(m[4]);
            rmin = mask_above(m, -1);
            rmax = mask_below(m, NROW);
            misses = 0;
            phase = PH_FIT_IN;
            seed_mask(hit, m, rmin, rmax, n, true, yzb, sector, geo, P, kf);
            xr = rmax;
            r = rmax + 1;
        }
        // ---- one step of the current phase
        const bool fit = phase == PH_FIT_IN || phase == PH_FIT_OUT;
        const bool to_outer_step = phase == PH_TO_OUTER;
        const int dir = (phase == PH_FIT_IN || phase == PH_EXT_IN) ? -1 : 1;
        int target = r + dir;
        if (fit) target = dir < 0 ? mask_below(m, r) : mask_above(m, r);
        if (to_outer_step) target = rmax;
        bool end_phase;
        if (fit) end_phase = target < rmin || target > rmax;
        else if (to_outer_step) end_phase = false;
        else end_phase = target < 0 || target >= NROW || misses >= P.ext_max_miss;
        // a fit step's hit, fetched before the transport
        int c = -1;
        float2 cv = make_float2(0.f, 0.f);
        if (fit && !end_phase) {
            c = hit[target];
            cv = __ldg(&yzb[c]);
        }
        bool moved = false;
        if (!end_phase) {
            // within one sector the planes are rows: the step is an exact
            // multiple of the row pitch (zero for the first hit after a seed)
            const float dxr = (float)(target - xr) * P.pitch;
            moved = kf_move<float, false>(kf, 0.0, sector, geo, P.kb, P.snp_max, nullptr, &dxr);
            ++steps;
            if (moved) xr = target;
            if (!moved) end_phase = true;
            else if (!fit && !to_outer_step && fabsf(kf.p[0] + kf.lo[0]) > geo->row_xf[target] * geo->tan_half)
                end_phase = true;
        }
        if (!end_phase && !to_outer_step) {
            if (!fit) {
                const float S00 = kf.C[0] + P.sy2, S01 = kf.C[1], S11 = kf.C[5] + P.sz2;
                const float det = S00 * S11 - S01 * S01;
                const float wz = sqrtf(P.chi2_ext * S11) * 1.001f + 1e-3f;
                const float wy = sqrtf(P.chi2_ext * S00) * 1.001f + 1e-3f;
                // cells of the window: z cells k0..k1, y cells y0..y1 of the row
                const int cb = gkb + target * gnz * CELL_NY;
                const float f0 = (kf.p[1] - wz - gz0) * ginv, f1 = (kf.p[1] + wz - gz0) * ginv;
                const int k0 = min(f0 >= 0.f ? (int)f0 : 0, gnz - 1);
                const int k1 = min(f1 >= 0.f ? (int)f1 : 0, gnz - 1);
                const float yp = kf.p[0] + kf.lo[0];
                const int y0 = ycell(geo, target, yp - wy - 1e-3f), y1 = ycell(geo, target, yp + wy + 1e-3f);
                float bchi = 0.f;
                const float idet = 1.f / det;
                // best candidate so far: smallest chi2, then smaller
                // canonical id (read only on an exact tie)
                auto consider = [&](int q, float2 vq) {
                    const float r1 = (vq.y - kf.p[1]) - kf.lo[1];
                    const float r0 = (vq.x - kf.p[0]) - kf.lo[0];
                    if (fabsf(r1) > wz || fabsf(r0) > wy) return;
                    const float chi = (r0 * r0 * S11 - 2.f * r0 * r1 * S01 + r1 * r1 * S00) * idet;
                    if (!(chi <= P.chi2_ext)) return;
                    if (c < 0 || chi < bchi || (chi == bchi && __ldg(&orig[q]) < __ldg(&orig[c]))) {
                        c = q;
                        cv = vq;
                        bchi = chi;
                    }
                };
                // The runs of the first EXT_ZB z cells: their offsets are
                // loaded in one batch and their candidates walked as one
                // list, EXT_CH loads in flight at a time.
                int qb[EXT_ZB], qe[EXT_ZB];
#pragma unroll
                for (int i = 0; i < EXT_ZB; ++i) {
                    const int at = cb + (k0 + i) * CELL_NY;
                    const bool in = k0 + i <= k1;
                    qb[i] = in ? __ldg(&cells.off[at + y0]) : 0;
                    qe[i] = in ? __ldg(&cells.off[at + y1 + 1]) : 0;
                }
                int pre[EXT_ZB + 1];
                pre[0] = 0;
#pragma unroll
                for (int i = 0; i < EXT_ZB; ++i) pre[i + 1] = pre[i] + (qe[i] - qb[i]);
                for (int t0 = 0; t0 < pre[EXT_ZB]; t0 += EXT_CH) {
                    int qq[EXT_CH];
                    float2 vv[EXT_CH];
#pragma unroll
                    for (int j = 0; j < EXT_CH; ++j) {
                        const int t = t0 + j;
                        int q = qb[EXT_ZB - 1] + (t - pre[EXT_ZB - 1]);
#pragma unroll
                        for (int i = EXT_ZB - 2; i >= 0; --i)
                            if (t < pre[i + 1]) q = qb[i] + (t - pre[i]);
                        qq[j] = q;
                        if (t < pre[EXT_ZB]) vv[j] = __ldg(&yzb[q]);
                    }
#pragma unroll
                    for (int j = 0; j < EXT_CH; ++j)
                        if (t0 + j < pre[EXT_ZB]) consider(qq[j], vv[j]);
                }
                for (int kz = k0 + EXT_ZB; kz <= k1; ++kz) {
                    const int b = __ldg(&cells.off[cb + kz * CELL_NY + y0]);
                    const int e = __ldg(&cells.off[cb + kz * CELL_NY + y1 + 1]);
#pragma unroll 4
                    for (int q = b; q < e; ++q) consider(q, __ldg(&yzb[q]));
                }
                if (c >= 0) {
                    hit[target] = c;
                    mask_set(m, target);
                    ++n;
                    if (dir < 0) rmin = target; else rmax = target;
                    misses = 0;
                } else {
                    ++misses;
                }
            }
            if (c >= 0) kf_update(kf, cv.x, cv.y, P.sy2, P.sz2, P.fp64_ratio, P.fp64_det, &st[ST_FP64], nullptr);
            r = target;
            continue;
        }
        // ---- phase transitions
        // After the inward pass the filtered state, moved to the outermost
        // hit row, carries every hit (exact transport, no process noise): it
        // is the outward state; an outward fit only replaces it when the
        // inward fit or that move failed.
        bool to_outer = false;
        if (to_outer_step) {
            // the moved state is the outward state; if the move failed, an
            // outward fit stands in
            if (moved) {
                ok |= 2;
                phase = PH_EXT_OUT + 1;
            } else {
                phase = PH_FIT_OUT;
            }
        } else if (phase == PH_FIT_IN) {
            if (moved || target < rmin || target > rmax) ok |= 1;  // fit completed
            if (refit && (ok & 1)) {
                float* out = tl_state + (int64_t)s * 40;
                for (int i = 0; i < 3; ++i) out[i] = kf.p[i] + kf.lo[i];
                for (int i = 3; i < 5; ++i) out[i] = kf.p[i];
                for (int i = 0; i < 15; ++i) out[5 + i] = kf.C[i];
            }
            if (!refit && (ok & 1)) {
                phase = PH_EXT_IN;
                r = rmin;
                misses = 0;
                continue;
            }
            to_outer = (ok & 1) != 0;
            phase = PH_FIT_OUT;
        } else if (phase == PH_EXT_IN) {
            to_outer = true;
            phase = PH_FIT_OUT;
        } else if (phase == PH_FIT_OUT) {
            if (moved || target < rmin || target > rmax) ok |= 2;
            phase = PH_EXT_OUT + 1;  // outward state ready (or the fit failed)
        } else {
            phase = PH_EXT_OUT + 2;  // finished
        }
        if (to_outer) {
            phase = PH_TO_OUTER;
            continue;
        }
        if (phase == PH_EXT_OUT + 1) {
            if (refit) {
                if (ok & 2) {
                    float* out = tl_state + (int64_t)s * 40;
                    for (int i = 0; i < 3; ++i) out[20 + i] = kf.p[i] + kf.lo[i];
                    for (int i = 3; i < 5; ++i) out[20 + i] = kf.p[i];
                    for (int i = 0; i < 15; ++i) out[25 + i] = kf.C[i];
                }
                tl_ok[s] = ok;
                // the fit flags of the merge's per-position record
                gs_meta[item].x = rmax | (rmin << 8) | (ok << 16);
                s = -1;
                continue;
            }
            if (ok & 2) {
                phase = PH_EXT_OUT;
                r = rmax;
                misses = 0;
                continue;
            }
        }
        if (phase == PH_FIT_OUT) {
            seed_mask(hit, m, rmin, rmax, n, false, yzb, sector, geo, P, kf);
            xr = rmin;
            r = rmin - 1;
            continue;
        }
        // finished building this tracklet
        tl_n[s] = n;
        tl_key[s] = ((unsigned long long)(NROW * 4 - n) << 32) | (uint32_t)seg_canon[s];
        s = -1;
    }
    if (!refit) atomicAdd(reinterpret_cast<unsigned long long*>(&st[ST_KFSTEPS]), (unsigned long long)steps);
}

// every cluster belongs to the best tracklet containing it
__global__ void k_owner(const int32_t* __restrict__ tl_rowhit, const unsigned long long* __restrict__ tl_key,
                        int64_t Scap, const int32_t* st, unsigned long long* owner) {
    if (input_rejected(st)) return;
    const int nseg = min((int64_t)st[ST_NSEG], Scap);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)nseg * NROW;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int h = tl_rowhit[i];
        if (h >= 0) atomicMin(&owner[h], tl_key[i / NROW]);
    }
}

// keep tracklets owning >= n_seg clusters (hits they do not own are
// cleared); the refits of the kept ones run in k_tracklet_lanes.  One warp
// per slot, the lanes over the rows: the row table, the owners and the
// canonical ids of the five 32-row rounds are each loaded in one batch, and
// a warp counts its kept slots in a register (one atomic per warp).
__global__ void k_keep(int32_t* tl_rowhit, const unsigned long long* __restrict__ tl_key,
                       const unsigned long long* __restrict__ owner, const int32_t* __restrict__ seg_grp,
                       const float2* __restrict__ yzb, const int32_t* __restrict__ orig, int n_seg,
                       int64_t Scap, int32_t* st, int32_t* tl_keep, int32_t* tl_canon,
                       int32_t* tl_rmin, int32_t* tl_rmax, float* tl_zin, float* tl_zout,
                       int32_t* tl_ok, int32_t* grp_tl_cnt, TlBins tb, int32_t* tl_binkey,
                       int64_t KT, uint4* tl_mask) {
    if (input_rejected(st)) return;
    const int nseg = min((int64_t)st[ST_NSEG], Scap);
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int kept = 0;  // slots kept by this warp (lane 0)
    for (int64_t s = w0; s < nseg; s += nw) {
        int32_t* hit = tl_rowhit + s * NROW;
        const unsigned long long key = tl_key[s];
        int h[MASK_W];
#pragma unroll
        for (int w = 0; w < MASK_W; ++w) {
            const int r = 32 * w + lane;
            h[w] = r < NROW ? hit[r] : -1;
        }
        bool own[MASK_W];
#pragma unroll
        for (int w = 0; w < MASK_W; ++w) own[w] = h[w] >= 0 && owner[h[w]] == key;
        int32_t canon = 0x7fffffff;
#pragma unroll
        for (int w = 0; w < MASK_W; ++w) {
            if (own[w]) canon = min(canon, orig[h[w]]);
            else if (h[w] >= 0) hit[32 * w + lane] = -1;
        }
        int n = 0, rmin = NROW, rmax = -1;
        uint32_t mw[MASK_W];
#pragma unroll
        for (int w = 0; w < MASK_W; ++w) {
            const int r0 = 32 * w;
            const unsigned m = __ballot_sync(0xffffffffu, own[w]);
            mw[w] = m;
            if (m) {
                n += __popc(m);
                rmin = min(rmin, r0 + __ffs(m) - 1);
                rmax = max(rmax, r0 + 31 - __clz(m));
            }
        }
        canon = __reduce_min_sync(0xffffffffu, canon);
        // the innermost and outermost kept hits, from the lanes holding them
        int hin_w = h[0], hout_w = h[0];
#pragma unroll
        for (int w = 1; w < MASK_W; ++w) {
            if ((rmin >> 5) == w) hin_w = h[w];
            if ((rmax >> 5) == w) hout_w = h[w];
        }
        const int h_in = __shfl_sync(0xffffffffu, hin_w, rmin & 31);
        const int h_out = __shfl_sync(0xffffffffu, hout_w, rmax & 31);
        if (lane != 0) continue;
        tl_ok[s] = 0;
        if (n < n_seg) {
            tl_keep[s] = 0;
            continue;
        }
        const int g = seg_grp[s];
        tl_keep[s] = 1;
        tl_mask[2 * s] = make_uint4(mw[0], mw[1], mw[2], mw[3]);
        tl_mask[2 * s + 1] = make_uint4(mw[4], 0u, 0u, 0u);
        tl_canon[s] = canon;
        tl_rmin[s] = rmin;
        tl_rmax[s] = rmax;
        const float zin = yzb[h_in].y, zout = yzb[h_out].y;
        tl_zin[s] = zin;
        tl_zout[s] = zout;
        const int bkey = tb.base[g] + (rmax / MRB) * tb.nb[g] + tl_bin(tb, g, zout);
        if (!in_range(bkey, KT, st, 301)) {
            tl_keep[s] = 0;
            continue;
        }
        tl_binkey[s] = bkey;
        ++kept;
        atomicAdd(&grp_tl_cnt[bkey], 1);
    }
    if (lane == 0 && kept > 0) atomicAdd(&st[ST_NTL], kept);
}

__global__ void k_tl_scatter(const int32_t* __restrict__ tl_keep, const int32_t* __restrict__ seg_grp,
                             const int32_t* __restrict__ grp_tl_off, int64_t Scap, const int32_t* st,
                             int32_t* grp_tl_cur, int32_t* tl_sorted,
                             const int32_t* __restrict__ tl_rmin, const int32_t* __restrict__ tl_rmax,
                             const float* __restrict__ tl_zin, const float* __restrict__ tl_zout,
                             int4* gs_meta,
                             const int32_t* __restrict__ tl_binkey, int32_t* st_w) {
    if (input_rejected(st)) return;
    const int nseg = min((int64_t)st[ST_NSEG], Scap);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x) {
        if (!tl_keep[s]) continue;
        const int key = tl_binkey[s];
        const int q = grp_tl_off[key] + atomicAdd(&grp_tl_cur[key], 1);
        if (!in_range(q, Scap, st_w, 302)) continue;
        tl_sorted[q] = s;
        // packed per-position merge data read coalesced by the candidate search
        // (the refit adds its fit flags in bits 16-17)
        gs_meta[q] = make_int4(tl_rmax[s] | (tl_rmin[s] << 8),
                               __float_as_int(tl_zout[s]), __float_as_int(tl_zin[s]), s);
    }
}

// ---------------------------------------------------------------- S4 ------
struct MgPrm {
    int merge_gap, merge_ov;
    float mz_slope, mz_margin;
    double chi2_merge;
    float kbf, snp_maxf, pitch;
    int64_t KT, S;
};

__device__ __forceinline__ bool ma_ok(const int4* __restrict__ gs_meta, int qa, int b) {
    return gs_meta[qa].w != b;
}

// For tracklet B (inner end), candidates A (outer end) in the same or a
// phi-adjacent sector of the same side and event: A's outward-fit state at
// its outermost row is moved to B's innermost plane and compared with B's
// inward-fit state there (chi2 of the 5-d difference, solved in FP64).  One
// warp per B; the lanes stride over the group-sorted candidates.
__global__ void __launch_bounds__(256, 4) k_merge_cand(
    const int32_t* __restrict__ seg_grp, const float* __restrict__ tl_state,
    const int32_t* __restrict__ grp_tl_off, const int4* __restrict__ gs_meta,
    const Geo* __restrict__ geo, MgPrm P, int32_t* st, int32_t* cand_n, int32_t* cand_a,
    float* cand_c2, TlBins tb, int32_t* match_act) {
    if (input_rejected(st)) return;
    // The cheap gates (row gap, z, and the 1-d chi2 of tan lambda and q/pT,
    // which the transport and the frame rotation leave unchanged) run over
    // every A in the bins; the A that pass are collected in the warp's list
    // and taken 32 at a time through the transport, the 1-d chi2 of y, z,
    // sin phi and the 5-d chi2, so that those run on full warps.
    __shared__ int sh_q[8][64];
    int* wq = sh_q[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int nkept = st[ST_NTL];
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const float lim = (float)P.chi2_merge * 1.01f;
    for (int qb = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; qb < nkept; qb += warps) {
        const int4 mb = gs_meta[qb];
        const int b = mb.w;
        if (lane == 0) cand_n[b] = 0;
        if (!((mb.x >> 16) & 1)) continue;
        const int rb = (mb.x >> 8) & 0xff;
        const float zb_in = __int_as_float(mb.z);
        const int gb = seg_grp[b];
        const int ev = gb / NSEC, sb = gb % NSEC, side = sb / NPHI, phb = sb % NPHI;
        const float* stb = tl_state + (int64_t)b * 40;
        const float tb3 = stb[3], tb4 = stb[4], vb3 = stb[5 + 12], vb4 = stb[5 + 14];
        int nc = 0;    // warp-uniform count of candidates
        int nbuf = 0;  // warp-uniform length of the list
        // the expensive test of the first k entries of the list (lane i: entry i)
        auto flush = [&](int k) {
            bool pass = false;
            float c2f = 0.f;
            int a = -1;
            if (lane < k) {
                const int qa = wq[lane];
                const int4 ma = gs_meta[qa];
                a = ma.w;
                if (!in_range(a, P.S, st, 205)) a = b;
                const int ra = ma.x & 0xff;
                const int sa = seg_grp[a] % NSEC;
                const float* sta = tl_state + (int64_t)a * 40;
                KF s;
                s.x = geo->row_xd[ra];
                s.frame = sa;
                for (int i = 0; i < 5; ++i) s.p[i] = sta[20 + i];
                s.lo[0] = s.lo[1] = s.lo[2] = 0.f;
                for (int i = 0; i < 15; ++i) s.C[i] = sta[25 + i];
                pass = kf_move<float>(s, geo->row_xd[rb], sb, geo, P.kbf, P.snp_maxf);
                // each component's 1-d chi2 is a lower bound of the 5-d
                // chi2: reject in FP32 (1% margin) before the solve
                if (pass) {
                    const int di[4] = {0, 1, 2, 3};
                    const int ci[4] = {0, 5, 9, 12};
#pragma unroll
                    for (int k2 = 0; k2 < 4; ++k2) {
                        const float d = stb[di[k2]] - (s.p[di[k2]] + (di[k2] < 3 ? s.lo[di[k2]] : 0.f));
                        const float v = s.C[ci[k2]] + stb[5 + ci[k2]];
                        pass = pass && d * d <= lim * v;
                    }
                }
                if (pass) {
                    // float-float: the differences and sums of the FP32
                    // states are exact, the solve carries ~48 bits
                    ff d[5], M[15];
#pragma unroll
                    for (int i = 0; i < 3; ++i)
                        d[i] = ff_add(ff_from(stb[i]), ff_neg(two_sum(s.p[i], s.lo[i])));
#pragma unroll
                    for (int i = 3; i < 5; ++i) d[i] = two_sum(stb[i], -s.p[i]);
#pragma unroll
                    for (int i = 0; i < 15; ++i) M[i] = two_sum(s.C[i], stb[5 + i]);
                    ff c2;
                    pass = chol_chi2_ff(d, M, c2);
                    // c2 <= chi2_merge on the float-float value
                    const double lim2 = P.chi2_merge;
                    pass = pass && ((double)c2.hi + (double)c2.lo) <= lim2;
                    c2f = c2.hi + c2.lo;
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, pass);
            if (pass) {
                const int kk = nc + __popc(bal & lt);
                if (kk < MAX_CAND) {
                    cand_a[(int64_t)b * MAX_CAND + kk] = a;
                    cand_c2[(int64_t)b * MAX_CAND + kk] = c2f;
                }
            }
            nc += __popc(bal);
        };
        for (int dp = -1; dp <= 1; ++dp) {
          const int sa = side * NPHI + (phb + dp + NPHI) % NPHI;
          const int ga = ev * NSEC + sa;
          const int min_gap = dp == 0 ? 0 : -P.merge_ov;
          // outer rows ra with rb - merge_gap <= ra <= rb - min_gap, by bucket
          const int ra_lo = max(rb - P.merge_gap, 0), ra_hi = min(rb - min_gap, NROW - 1);
          for (int j = ra_lo / MRB; ra_lo <= ra_hi && j <= ra_hi / MRB; ++j) {
            // the z gate |z_B - z_A| <= slope |dx| + margin, with |dx| at
            // most that of the bucket's farthest allowed row, bounds the bins
            const int r0 = max(j * MRB, ra_lo), r1 = min(j * MRB + MRB - 1, ra_hi);
            const float xb = geo->row_xf[rb];
            const float dxm = fmaxf(fabsf(xb - geo->row_xf[r0]), fabsf(xb - geo->row_xf[r1]));
            const float wmax = P.mz_slope * dxm * 1.001f + P.mz_margin + 1e-3f;
            const int kb = tb.base[ga] + j * tb.nb[ga];
            const int k0 = kb + tl_bin(tb, ga, zb_in - wmax);
            const int k1 = kb + tl_bin(tb, ga, zb_in + wmax);
            if (!in_range(k0, P.KT + 1, st, 201) || !in_range(k1 + 1, P.KT + 1, st, 202)) continue;
            int q0 = grp_tl_off[k0], q1 = grp_tl_off[k1 + 1];
            if (!in_range(q0, nkept + 1, st, 203) || !in_range(q1, nkept + 1, st, 204) || q1 < q0)
                q0 = q1 = 0;
            for (int qa0 = q0; qa0 < q1; qa0 += 32) {
                const int qa = qa0 + lane;
                bool pass = false;
                if (qa < q1 && qa != qb && ma_ok(gs_meta, qa, b)) {
                    const int4 ma = gs_meta[qa];
                    int a = ma.w;
                    if (!in_range(a, P.S, st, 205)) a = b;
                    const int ra = ma.x & 0xff;
                    const int gap = rb - ra;
                    pass = ((ma.x >> 17) & 1) && gap >= min_gap && gap <= P.merge_gap;
                    if (pass) {
                        const float dxr = fabsf(__fsub_rn(geo->row_xf[rb], geo->row_xf[ra]));
                        pass = fabsf(__fsub_rn(zb_in, __int_as_float(ma.y))) <=
                               __fadd_rn(__fmul_rn(P.mz_slope, dxr), P.mz_margin);
                    }
                    if (pass) {
                        // tan lambda and q/pT are unchanged by the transport
                        // and the frame rotation: their 1-d chi2 (lower
                        // bounds of the 5-d chi2) reject before the move
                        const float* sta = tl_state + (int64_t)a * 40;
                        const float dt = tb3 - sta[23], dw = tb4 - sta[24];
                        pass = dt * dt <= lim * (sta[25 + 12] + vb3) && dw * dw <= lim * (sta[25 + 14] + vb4);
                    }
                }
                const unsigned bal = __ballot_sync(0xffffffffu, pass);
                if (pass) wq[nbuf + __popc(bal & lt)] = qa;
                nbuf += __popc(bal);
                __syncwarp();
                if (nbuf >= 32) {
                    flush(32);
                    // keep the entries beyond the first 32
                    const int rest = nbuf - 32;
                    const int v = lane < rest ? wq[32 + lane] : 0;
                    __syncwarp();
                    if (lane < rest) wq[lane] = v;
                    nbuf = rest;
                    __syncwarp();
                }
            }
          }
        }
        if (nbuf > 0) flush(nbuf);
        __syncwarp();
        if (lane == 0) {
            cand_n[b] = min(nc, MAX_CAND);
            if (nc > MAX_CAND) set_status(st, TPC_ERR_CAPACITY, 3);
            if (nc) {
                atomicAdd(&st[ST_NCAND], min(nc, MAX_CAND));
                // the B ends with candidates, the first list of the matching
                match_act[atomicAdd(&st[ST_MATCH_LIVE], 1)] = b;
            }
        }
    }
}

// Greedy matching in ascending chi2 (ties: canonical ids), computed as
// rounds of locally dominant candidates: a candidate whose key is the best
// among the live candidates of its A (outer end) and of its B (inner end) is
// accepted; candidates touching an accepted end die.  One thread-block
// cluster of MATCH_CTAS blocks: a thread per live B end, the three phases of
// a round separated by cluster barriers, the round counters in the shared
// memory of block 0 (distributed shared memory).
constexpr int MATCH_CTAS = 8;
__global__ void __cluster_dims__(MATCH_CTAS, 1, 1) __launch_bounds__(1024) k_match(
    const int32_t* __restrict__ cand_n, const int32_t* __restrict__ cand_a,
    const float* __restrict__ cand_c2, const int32_t* __restrict__ tl_canon, int64_t Scap,
    int32_t* st, unsigned long long* best_a, unsigned long long* best_b, int32_t* nxt,
    int32_t* prv, int32_t* act) {
    if (input_rejected(st)) return;
    // An (a, b) pair whose key (chi2, canonical ids) is the smallest of every
    // live pair at a and of every live pair at b is matched; both ends are
    // then used.  The rounds run over a compacted list of the B ends that
    // still have a live candidate (first written by the candidate search);
    // best_a / best_b hold KEY_MAX between rounds.  Counters of round r:
    // list length cnt[r & 1], next list length cnt[(r & 1) ^ 1], live flag
    // live[r & 1]; each is cleared a round before it is written.
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    __shared__ int sh_cnt[2], sh_live[2];
    int* cnt = cl.map_shared_rank(sh_cnt, 0);
    int* live = cl.map_shared_rank(sh_live, 0);
    const int tid = (int)cl.block_rank() * blockDim.x + threadIdx.x;
    const int nthreads = MATCH_CTAS * blockDim.x;
    const bool lead = cl.block_rank() == 0 && threadIdx.x == 0;
    if (lead) {
        cnt[0] = (int)min((int64_t)st[ST_MATCH_LIVE], Scap);
        cnt[1] = 0;
        live[0] = live[1] = 0;
    }
    cl.sync();
    int32_t* cur = act;
    int32_t* nx = act + Scap;
    for (int round = 0; round < 4096; ++round) {
        const int ra = round & 1, rb = ra ^ 1;
        const int na = cnt[ra];
        if (na == 0) break;
        if (lead) {
            cnt[rb] = 0;
            live[rb] = 0;
        }
        bool any = false;
        for (int i = tid; i < na; i += nthreads) {
            const int b = cur[i];
            if (prv[b] >= 0) continue;
            for (int k = 0; k < cand_n[b]; ++k) {
                const int a = cand_a[(int64_t)b * MAX_CAND + k];
                if (nxt[a] >= 0) continue;
                const uint64_t c2 = __float_as_uint(cand_c2[(int64_t)b * MAX_CAND + k]);
                atomicMin(&best_a[a], (c2 << 32) | (uint32_t)tl_canon[b]);
                atomicMin(&best_b[b], (c2 << 32) | (uint32_t)tl_canon[a]);
                any = true;
            }
        }
        if (any) live[ra] = 1;
        cl.sync();
        if (!live[ra]) break;
        for (int i = tid; i < na; i += nthreads) {
            const int b = cur[i];
            if (prv[b] >= 0) continue;
            for (int k = 0; k < cand_n[b]; ++k) {
                const int a = cand_a[(int64_t)b * MAX_CAND + k];
                if (nxt[a] >= 0) continue;
                const uint64_t c2 = __float_as_uint(cand_c2[(int64_t)b * MAX_CAND + k]);
                if (best_a[a] == ((c2 << 32) | (uint32_t)tl_canon[b]) &&
                    best_b[b] == ((c2 << 32) | (uint32_t)tl_canon[a])) {
                    nxt[a] = b;
                    prv[b] = a;
                    atomicAdd(&st[ST_NMERGE], 1);
                }
            }
        }
        cl.sync();
        // reset the keys that were touched; keep the B ends still unmatched
        for (int i = tid; i < na; i += nthreads) {
            const int b = cur[i];
            best_b[b] = KEY_MAX;
            bool keep = false;
            for (int k = 0; k < cand_n[b]; ++k) {
                const int a = cand_a[(int64_t)b * MAX_CAND + k];
                best_a[a] = KEY_MAX;
                keep |= nxt[a] < 0;
            }
            if (keep && prv[b] < 0) nx[atomicAdd(&cnt[rb], 1)] = b;
        }
        cl.sync();
        int32_t* t = cur;
        cur = nx;
        nx = t;
    }
    // block 0 keeps its shared memory until every block has read it
    cl.sync();
}

// ---------------------------------------------------------------- output --
// Chains of merged tracklets (walk from the outermost, i.e. nxt < 0).
// One warp per track head (the outermost kept tracklet of a merge chain,
// nxt < 0): length and canonical id (smallest input index) of the chain.
__global__ void k_track_heads(const int32_t* __restrict__ tl_keep, const int32_t* __restrict__ nxt,
                              const int32_t* __restrict__ prv, const int32_t* __restrict__ tl_canon,
                              const int32_t* __restrict__ tl_rowhit, int n_min, int64_t Scap,
                              const int32_t* st, int32_t* trk_flag, int32_t* trk_len_at,
                              int32_t* trk_head_at) {
    if (input_rejected(st)) return;
    const int nseg = min((int64_t)st[ST_NSEG], Scap);
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = w0; s < nseg; s += nw) {
        if (!tl_keep[s] || nxt[s] >= 0) continue;
        int len = 0, guard = 0;
        int32_t canon = 0x7fffffff;
        for (int t = (int)s; t >= 0 && guard < 4096; t = prv[t], ++guard) {
            const int32_t* hit = tl_rowhit + (int64_t)t * NROW;
            for (int r0 = 0; r0 < NROW; r0 += 32)
                len += __popc(__ballot_sync(0xffffffffu, r0 + lane < NROW && hit[r0 + lane] >= 0));
            canon = min(canon, tl_canon[t]);
        }
        if (len < n_min || lane != 0) continue;
        trk_flag[canon] = 1;
        trk_len_at[canon] = len;
        trk_head_at[canon] = (int32_t)s;
    }
}

__global__ void k_track_len(int64_t n, const int32_t* __restrict__ trk_flag,
                            const int32_t* __restrict__ trk_rank, const int32_t* __restrict__ trk_len_at,
                            const int32_t* __restrict__ trk_head_at, int32_t track_cap,
                            int32_t* len_by_rank, int32_t* head_by_rank, int32_t* st,
                            int32_t* n_tracks_dev) {
    if (input_rejected(st)) {  // rejected input: no tracks
        if (blockIdx.x == 0 && threadIdx.x == 0) *n_tracks_dev = 0;
        return;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!trk_flag[i]) continue;
        const int r = trk_rank[i];
        if (r < track_cap) {
            len_by_rank[r] = trk_len_at[i];
            head_by_rank[r] = trk_head_at[i];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int T = trk_rank[n];
        st[ST_NTRACKS] = T;
        *n_tracks_dev = min(T, track_cap);
        if (T > track_cap) set_status(st, TPC_ERR_CAPACITY, 4);
    }
}

// One warp per output track: the hits of its chain of tracklets, outermost
// first, in the track's slice of the CSR, and the track index per cluster.
__global__ void k_track_write(const int32_t* __restrict__ st_r, int32_t track_cap,
                              const int32_t* __restrict__ head_by_rank, const int32_t* __restrict__ prv,
                              const int32_t* __restrict__ tl_rowhit, const int32_t* __restrict__ orig,
                              const int32_t* __restrict__ trk_off, int64_t n, int32_t* toc,
                              int32_t* trk_hits, int32_t* st_w) {
    if (input_rejected(st_r)) return;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int T = min(st_r[ST_NTRACKS], track_cap);
    for (int64_t r = w0; r < T; r += nw) {
        int o = trk_off[r], guard = 0;
        for (int t = head_by_rank[r]; t >= 0 && guard < 4096; t = prv[t], ++guard) {
            const int32_t* hit = tl_rowhit + (int64_t)t * NROW;
            // rows from the outermost down, 32 at a time
            for (int r0 = NROW - 1; r0 >= 0; r0 -= 32) {
                const int rr = r0 - lane;
                const int h = rr >= 0 ? hit[rr] : -1;
                const unsigned m = __ballot_sync(0xffffffffu, h >= 0);
                if (h >= 0) {
                    const int pos = o + __popc(m & ((1u << lane) - 1u));
                    if (pos < n) {
                        const int oi = orig[h];
                        trk_hits[pos] = oi;
                        toc[oi] = (int32_t)r;
                    } else {
                        set_status(st_w, TPC_ERR_STATE, 401);
                    }
                }
                o += __popc(m);
            }
        }
    }
}

__global__ void k_fill_u64(unsigned long long* p, int64_t n, unsigned long long v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_fill_u32(uint32_t* p, int64_t n, uint32_t v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// The per-call initialisations of a find in one launch: a table of (array,
// count, value, 4- or 8-byte element); each entry owns a run of blocks of
// MF_PER elements each.
constexpr int MF_T = 256, MF_PER = MF_T * 16, MF_MAX = 24;
struct FillDesc {
    void* p;
    int64_t n;
    unsigned long long v;
    int32_t w;     // element bytes: 4 or 8
    int32_t blk0;  // first block of the entry
};
struct FillSet {
    int32_t nd;
    FillDesc d[MF_MAX];
};
__global__ void __launch_bounds__(MF_T) k_multi_fill(FillSet f) {
    int k = 0;
    while (k + 1 < f.nd && (int)blockIdx.x >= f.d[k + 1].blk0) ++k;
    const FillDesc d = f.d[k];
    const int64_t b0 = (int64_t)((int)blockIdx.x - d.blk0) * MF_PER;
    const int64_t e = min(b0 + (int64_t)MF_PER, d.n);
    if (d.w == 8) {
        auto* q = static_cast<unsigned long long*>(d.p);
        for (int64_t i = b0 + threadIdx.x; i < e; i += MF_T) q[i] = d.v;
    } else {
        auto* q = static_cast<uint32_t*>(d.p);
        for (int64_t i = b0 + threadIdx.x; i < e; i += MF_T) q[i] = (uint32_t)d.v;
    }
}

}  // namespace

#define TPC_TRY(x)                                  \
    do {                                            \
        cudaError_t e_ = (x);                       \
        if (e_ != cudaSuccess) return e_;           \
    } while (0)

cudaError_t run_find(tpc_ctx* c, int32_t* toc, int32_t* trk_off, int32_t* trk_hits,
                     int32_t* n_tracks_dev, int32_t track_cap, cudaStream_t s) {
    const Workspace& W = c->ws;
    const Layout& L = W.L;
    const tpc_params& p = c->prm;
    const int64_t n = c->n;
    const int G = c->n_events * NSEC;
    int32_t* st = W.at<int32_t>(L.status);
    const Geo* geo = W.at<Geo>(L.geo);
    int32_t* scan_tmp = W.at<int32_t>(L.scan_a);

    c->mark(0, s);
    // Every per-call initialisation in one launch, ahead of the kernels: the
    // per-call counters (the status word and the FP64 count are cumulative)
    // and each buffer that a later stage fills before use (none of them is
    // written before its stage; the first up-claim table is not here: it
    // serves as a neighbour queue before the claims)
    {
        FillSet f{};
        int blk = 0;
        auto add = [&](void* ptr, int64_t cnt, unsigned long long v, int w) {
            if (cnt <= 0) return;
            f.d[f.nd] = FillDesc{ptr, cnt, v, w, blk};
            blk += (int)((cnt + MF_PER - 1) / MF_PER);
            ++f.nd;
        };
        add(st + ST_NSEG, ST_NTRACKS - ST_NSEG + 1, 0, 4);
        add(st + ST_MATCH_LIVE, ST_NB_Q2 + 1 - ST_MATCH_LIVE, 0, 4);
        add(W.at<uint32_t>(L.g_zmin_u), G, 0xffffffffu, 4);
        add(W.at<uint32_t>(L.g_zmax_u), G, 0u, 4);
        add(W.at<int32_t>(L.cell_cnt), L.K + 1, 0, 4);
        add(W.at<unsigned long long>(L.claim_dn), n, KEY_MAX, 8);
        add(W.at<int32_t>(L.link_dn), n, 0xffffffffu, 4);
        add(W.at<int32_t>(L.link_up), n, 0xffffffffu, 4);
        add(W.at<unsigned long long>(L.owner), n, KEY_MAX, 8);
        add(W.at<int32_t>(L.grp_tl_cnt), L.KT + 1, 0, 4);
        add(W.at<int32_t>(L.grp_tl_cur), L.KT, 0, 4);
        add(W.at<int32_t>(L.cand_n), L.S, 0, 4);
        add(W.at<int32_t>(L.nxt), L.S, 0xffffffffu, 4);
        add(W.at<int32_t>(L.prv), L.S, 0xffffffffu, 4);
        add(W.at<unsigned long long>(L.best_a), L.S, KEY_MAX, 8);
        add(W.at<unsigned long long>(L.best_b), L.S, KEY_MAX, 8);
        add(W.at<int32_t>(L.trk_flag), n, 0, 4);
        add(W.at<int32_t>(L.len_by_rank), track_cap, 0, 4);
        add(toc, n, 0xffffffffu, 4);
        tpc::LaunchCount{}, k_multi_fill<<<(unsigned)std::max(blk, 1), MF_T, 0, s>>>(f);
        TPC_TRY(cudaGetLastError());
    }
    // S1: z range per group, cells, histogram, scan, scatter
    int32_t* grp_of = W.at<int32_t>(L.d2);  // group of every input cluster (d2 is free in S1)
    tpc::LaunchCount{}, k_zrange<<<grid_for(n), TPB, 0, s>>>(c->z, n, c->evt_sector_off, G, W.at<uint32_t>(L.g_zmin_u),
                                         W.at<uint32_t>(L.g_zmax_u), grp_of, st);
    tpc::LaunchCount{}, k_cells<<<1, 1024, 0, s>>>(c->evt_sector_off, G, W.at<uint32_t>(L.g_zmin_u),
                               W.at<uint32_t>(L.g_zmax_u), W.at<float>(L.g_zmin), W.at<float>(L.g_inv),
                               W.at<int32_t>(L.g_nz), W.at<int32_t>(L.g_kbase), L.K, st);
    Cells cells{W.at<float>(L.g_zmin), W.at<float>(L.g_inv), W.at<int32_t>(L.g_nz),
                W.at<int32_t>(L.g_kbase), W.at<int32_t>(L.cell_off)};
    tpc::LaunchCount{}, k_hist<<<grid_for(n), TPB, 0, s>>>(c->y, c->z, c->row, n, grp_of, cells, geo,
                                       W.at<int32_t>(L.cell_cnt), W.at<int32_t>(L.key_in),
                                       W.at<int32_t>(L.slot_in), L.K, st);
    TPC_TRY(scan_i32(W.at<int32_t>(L.cell_cnt), W.at<int32_t>(L.cell_off), L.K, scan_tmp, s));
    float2* yzb = W.at<float2>(L.yzb);
    int32_t* orig = W.at<int32_t>(L.orig);
    int32_t* grpb = W.at<int32_t>(L.grpb);
    uint8_t* rowb = W.at<uint8_t>(L.rowb);
    tpc::LaunchCount{}, k_scatter<<<grid_for(n), TPB, 0, s>>>(c->y, c->z, c->row, n, grp_of,
                                          W.at<int32_t>(L.key_in), W.at<int32_t>(L.slot_in),
                                          W.at<int32_t>(L.cell_off), L.K, yzb, orig, grpb, rowb, st);
    TPC_TRY(cudaGetLastError());

    c->mark(1, s);
    // S2: neighbours, claims, links
    int32_t* cdn = W.at<int32_t>(L.choice_dn);
    int32_t* cup = W.at<int32_t>(L.choice_up);
    float* d2 = W.at<float>(L.d2);
    NbPrm nb{p.win_y, p.win_z, p.chi2_link, p.sigma_y2, p.sigma_z2, p.max_gap};
    int32_t* nb_queue = W.at<int32_t>(L.key_in);    // free after S1
    int32_t* nb_queue2 = W.at<int32_t>(L.slot_in);  // free after S1
    int32_t* nb_queue3 = reinterpret_cast<int32_t*>(W.at<unsigned long long>(L.claim_up));  // free until the claims
    // pass 1: gap pair (1, 1) for all; pass 2: the later gap pairs for the
    // rest, and every gap pair for the clusters whose pass-1 list overflowed
    tpc::LaunchCount{}, k_neighbours_first<<<grid_for(n), TPB, 0, s>>>(
        n, yzb, orig, grpb, rowb, cells, geo, nb, cdn, cup, d2, st, nb_queue3, nb_queue2, ST_NB_Q2);
    // one launch over both queues: the dense ones from (1, 1), then the rest
    // from gap sum 3
    // lanes per queued cluster: a tuning knob of this queued stage
    auto sub_pass = [&](auto ng) {
        constexpr int NG = decltype(ng)::value;
        tpc::LaunchCount{}, k_neighbours_sub<NG><<<grid_for(n / 4, 32 * 4), ns_warps<NG>() * 32, 0, s>>>(
            n, nb_queue3, ST_NB_Q3, 2, 2 * NB_GAP_MAX, yzb, orig, grpb, rowb, cells, geo, nb, cdn, cup, d2, st,
            nb_queue, nullptr, 0, nb_queue2, ST_NB_Q2, 3);
    };
    if (c->tune.nb_sub_lanes == 4) sub_pass(std::integral_constant<int, 4>{});
    else if (c->tune.nb_sub_lanes == 16) sub_pass(std::integral_constant<int, 16>{});
    else sub_pass(std::integral_constant<int, NG2>{});
    tpc::LaunchCount{}, k_neighbours_warp<<<152 * 8, NB_WARPS * 32, 0, s>>>(nb_queue, st, yzb, orig, grpb,
                                                                        rowb, cells, geo, nb, cdn, cup, d2);
    c->mark(2, s);
    auto* claim_up = W.at<unsigned long long>(L.claim_up);
    auto* claim_dn = W.at<unsigned long long>(L.claim_dn);
    tpc::LaunchCount{}, k_fill_u64<<<grid_for(n), TPB, 0, s>>>(claim_up, n, KEY_MAX);
    tpc::LaunchCount{}, k_claims<<<grid_for(n), TPB, 0, s>>>(n, cdn, cup, d2, orig, claim_up, claim_dn, st);
    int32_t* ldn = W.at<int32_t>(L.link_dn);
    int32_t* lup = W.at<int32_t>(L.link_up);
    tpc::LaunchCount{}, k_links<<<grid_for(n), TPB, 0, s>>>(n, cdn, cup, d2, orig, claim_up, claim_dn, ldn, lup, st);

    c->mark(3, s);
    // S3: chains
    int32_t* tl_rowhit = W.at<int32_t>(L.tl_rowhit);
    auto* tl_mask = W.at<uint4>(L.tl_mask);
    tpc::LaunchCount{}, k_chains<<<grid_for(n), TPB, 0, s>>>(n, ldn, lup, orig, grpb, rowb, p.n_seg, L.S,
                                         W.at<int32_t>(L.seg_start), W.at<int32_t>(L.seg_grp),
                                         W.at<int32_t>(L.seg_canon), tl_rowhit, tl_mask, st);
    c->mark(4, s);
    // S3b: tracklets
    TlPrm tp;
    tp.sy2 = p.sigma_y2;
    tp.sz2 = p.sigma_z2;
    tp.chi2_ext = p.chi2_ext;
    tp.kb = (float)(KAPPA * (double)p.bz);
    tp.snp_max = p.snp_max;
    tp.fp64_ratio = p.fp64_ratio;
    tp.fp64_det = p.fp64_det;
    tp.pitch = (float)(162.0 / 151.0);
    tp.ext_max_miss = p.ext_max_miss;
    tp.n_seg = p.n_seg;
    tp.bz = p.bz;
    tp.seed_snp = p.seed_snp_max;
    tp.seed_qpt = p.seed_qpt_max;
    for (int i = 0; i < 5; ++i) tp.prior[i] = p.prior[i];
    const unsigned sgrid = grid_for(L.S, 128);
    // persistent lanes: enough resident warps to fill the GPU
    const unsigned lgrid = (unsigned)c->n_sm * (unsigned)c->tune.lane_blocks_per_sm;
    const int tile = c->tune.lane_tile;
    auto* tl_key = W.at<unsigned long long>(L.tl_key);
    tpc::LaunchCount{}, k_tracklet_lanes<<<lgrid, 128, 0, s>>>(
        0, nullptr, ST_NSEG, W.at<int32_t>(L.seg_grp), W.at<int32_t>(L.seg_canon), yzb,
        orig, cells, geo, tp, L.S, st, tl_rowhit, tl_mask, W.at<int32_t>(L.tl_n), tl_key, nullptr, nullptr,
        nullptr, tile);
    c->mark(5, s);
    auto* owner = W.at<unsigned long long>(L.owner);
    tpc::LaunchCount{}, k_owner<<<grid_for(L.S * NROW), TPB, 0, s>>>(tl_rowhit, tl_key, L.S, st, owner);
    int32_t* grp_cnt = W.at<int32_t>(L.grp_tl_cnt);
    TlBins tb{W.at<float>(L.tb_zmin), W.at<float>(L.tb_inv), W.at<int32_t>(L.tb_nb), W.at<int32_t>(L.tb_base)};
    tpc::LaunchCount{}, k_tl_bins<<<1, 1024, 0, s>>>(c->evt_sector_off, G, W.at<uint32_t>(L.g_zmin_u),
                                                   W.at<uint32_t>(L.g_zmax_u), W.at<float>(L.tb_zmin),
                                                   W.at<float>(L.tb_inv), W.at<int32_t>(L.tb_nb),
                                                   W.at<int32_t>(L.tb_base), st);
    tpc::LaunchCount{}, k_keep<<<grid_for(L.S * 32, 128), 128, 0, s>>>(tl_rowhit, tl_key, owner, W.at<int32_t>(L.seg_grp), yzb,
                                 orig, p.n_seg, L.S, st, W.at<int32_t>(L.tl_keep),
                                 W.at<int32_t>(L.tl_canon), W.at<int32_t>(L.tl_rmin),
                                 W.at<int32_t>(L.tl_rmax), W.at<float>(L.tl_zin),
                                 W.at<float>(L.tl_zout), W.at<int32_t>(L.tl_ok), grp_cnt, tb,
                                 W.at<int32_t>(L.tl_binkey), L.KT, tl_mask);
    TPC_TRY(scan_i32(grp_cnt, W.at<int32_t>(L.grp_tl_off), L.KT, scan_tmp, s));
    tpc::LaunchCount{}, k_tl_scatter<<<sgrid, 128, 0, s>>>(W.at<int32_t>(L.tl_keep), W.at<int32_t>(L.seg_grp),
                                       W.at<int32_t>(L.grp_tl_off), L.S, st,
                                       W.at<int32_t>(L.grp_tl_cur), W.at<int32_t>(L.tl_sorted),
                                       W.at<int32_t>(L.tl_rmin), W.at<int32_t>(L.tl_rmax),
                                       W.at<float>(L.tl_zin), W.at<float>(L.tl_zout),
                                       W.at<int4>(L.gs_meta), W.at<int32_t>(L.tl_binkey), st);
    // refit of the kept tracklets, in their merge order
    tpc::LaunchCount{}, k_tracklet_lanes<<<lgrid, 128, 0, s>>>(
        1, W.at<int32_t>(L.tl_sorted), ST_NTL, W.at<int32_t>(L.seg_grp), W.at<int32_t>(L.seg_canon), yzb,
        orig, cells, geo, tp, L.S, st, tl_rowhit, tl_mask, W.at<int32_t>(L.tl_n), tl_key,
        W.at<float>(L.tl_state), W.at<int32_t>(L.tl_ok), W.at<int4>(L.gs_meta), tile);
    c->mark(6, s);
    // S4: merge candidates and greedy matching
    MgPrm mp{p.merge_max_row_gap, p.merge_max_overlap, p.merge_z_slope, p.merge_z_margin,
             (double)p.chi2_merge, (float)(KAPPA * (double)p.bz), p.snp_max, (float)(162.0 / 151.0),
             L.KT, L.S};
    // cand_n of slots that are not kept must read 0 for the matching
    tpc::LaunchCount{}, k_merge_cand<<<grid_for(L.S * 32, 256), 256, 0, s>>>(
        W.at<int32_t>(L.seg_grp), W.at<float>(L.tl_state), W.at<int32_t>(L.grp_tl_off),
        W.at<int4>(L.gs_meta), geo, mp, st, W.at<int32_t>(L.cand_n), W.at<int32_t>(L.cand_a),
        W.at<float>(L.cand_c2), tb, W.at<int32_t>(L.match_act));
    c->mark(7, s);
    int32_t* nxt = W.at<int32_t>(L.nxt);
    int32_t* prv = W.at<int32_t>(L.prv);
    auto* best_a = W.at<unsigned long long>(L.best_a);
    auto* best_b = W.at<unsigned long long>(L.best_b);
    tpc::LaunchCount{}, k_match<<<MATCH_CTAS, 1024, 0, s>>>(W.at<int32_t>(L.cand_n), W.at<int32_t>(L.cand_a), W.at<float>(L.cand_c2),
                               W.at<int32_t>(L.tl_canon), L.S, st, best_a, best_b, nxt, prv,
                               W.at<int32_t>(L.match_act));
    c->mark(8, s);
    // output: canonical order by smallest input index
    int32_t* flag = W.at<int32_t>(L.trk_flag);
    tpc::LaunchCount{}, k_track_heads<<<grid_for(L.S * 32, 128), 128, 0, s>>>(W.at<int32_t>(L.tl_keep), nxt, prv, W.at<int32_t>(L.tl_canon),
                                        tl_rowhit, p.n_min, L.S, st, flag, W.at<int32_t>(L.trk_len_at),
                                        W.at<int32_t>(L.trk_head_at));
    int32_t* rank = W.at<int32_t>(L.trk_rank);
    TPC_TRY(scan_i32(flag, rank, n, scan_tmp, s));
    int32_t* len_by_rank = W.at<int32_t>(L.len_by_rank);
    int32_t* head_by_rank = W.at<int32_t>(L.head_by_rank);
    tpc::LaunchCount{}, k_track_len<<<grid_for(n), TPB, 0, s>>>(n, flag, rank, W.at<int32_t>(L.trk_len_at),
                                            W.at<int32_t>(L.trk_head_at), track_cap, len_by_rank,
                                            head_by_rank, st, n_tracks_dev);
    TPC_TRY(scan_i32(len_by_rank, trk_off, track_cap, scan_tmp, s));
    tpc::LaunchCount{}, k_track_write<<<grid_for((int64_t)track_cap * 32), TPB, 0, s>>>(
        st, track_cap, head_by_rank, prv, tl_rowhit, orig, trk_off, n, toc, trk_hits, st);
    c->mark(9, s);
    return cudaGetLastError();
}

}  // namespace tpc
