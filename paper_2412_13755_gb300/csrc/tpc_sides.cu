// NEXT-4: association of the A- and C-side segments of membrane-crossing
// tracks with the drift-time offset t0 as a sixth fit parameter.
//
// Found tracks never span both sides (the merge joins one side), so a track
// that crosses the central membrane comes out as an inner and an outer
// segment on opposite sides of one phi sector (or of two adjacent ones),
// with adjacent row ranges.  Steps, one kernel each:
//   class   per track: usable when one side, one event, >= n_min clusters;
//           count it in the bucket (event, side, phi sector, row) of its
//           innermost cluster; initialise the outputs
//   scan    bucket offsets
//   scatter bucket lists
//   need    a track is fitted when it meets a structural candidate
//   fit     inward and outward FP64 fits (state at the innermost and at the
//           outermost cluster)
//   pairs   junction test of every structural candidate (4-d chi2, true z
//           at the junction), survivors appended to the candidate list
//   joint   the six-parameter fit of each candidate, its chi2 increase;
//           each track keeps its best candidate by a 64-bit atomicMin on
//           (chi2 increase as FP32, partner index)
//   pick    a candidate is a pair when each member is the other's best; the
//           joint fit is written to both members
// Decisions are taken in FP64 (the FP32 rounding of the chi2 increase only
// orders candidates), so the result does not depend on launch order.
#include <algorithm>
#include <cmath>

#include "tpc_internal.h"
#include "tpc_sides.cuh"

namespace tpc {

namespace {

constexpr int SIDES_T = 128;

struct SideCls {
    int32_t r_in, r_out;
    int32_t key_in;  // bucket of the innermost cluster, -1: not usable
    int32_t info;    // bit 1: side C of the outermost cluster's sector; bits 2..: event
    float z_in, z_out;  // apparent z of the innermost and outermost cluster
};

struct SideCand {
    int32_t i, o;  // inner and outer track
    double t0s;    // t0 from the junction states
    double dchi2;  // chi2 increase of the joint fit (infinity: rejected)
    double q[6], C[21], chi2;  // the joint fit
};

__host__ __device__ inline int bucket_key(int event, int sector, int r) {
    return ((event * 2 + (sector >= NPHI ? 1 : 0)) * NPHI + sector % NPHI) * NROW + r;
}

// (FP32 of the chi2 increase in an order-preserving bit pattern) << 32 | partner
__device__ __forceinline__ unsigned long long cand_key(double d, int partner) {
    const uint32_t b = __float_as_uint(__double2float_rn(d));
    const uint32_t o = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    return ((unsigned long long)o << 32) | (uint32_t)partner;
}

__device__ __forceinline__ int n_eff(int32_t n_tracks, const int32_t* n_tracks_dev) {
    int T = n_tracks;
    if (n_tracks_dev) T = min(T, *n_tracks_dev);
    return max(T, 0);
}

__global__ void __launch_bounds__(SIDES_T) k_sides_class(
    const int32_t* __restrict__ trk_off, const int32_t* __restrict__ trk_hits, int32_t n_tracks,
    const int32_t* __restrict__ n_tracks_dev, HitSrc H, SidesPrm S, SideCls* cls, int32_t* need, int32_t* role,
    unsigned long long* best, int32_t* bcnt, int32_t* partner, double* t0, double* params6, double* cov6,
    double* chi2, int32_t* ndf, double* dchi2, const int32_t* __restrict__ st) {
    const bool rejected = input_rejected(st);
    const int T = n_eff(n_tracks, n_tracks_dev);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tracks; t += gridDim.x * blockDim.x) {
        if (t >= T) {  // beyond the device count: only the flag the scan reads
            need[t] = 0;
            continue;
        }
        role[t] = 0;
        partner[t] = -1;
        t0[t] = 0.0;
        for (int k = 0; k < 6; ++k) params6[(int64_t)t * 6 + k] = 0.0;
        for (int k = 0; k < 21; ++k) cov6[(int64_t)t * 21 + k] = 0.0;
        chi2[t] = 0.0;
        ndf[t] = -1;
        dchi2[t] = 0.0;
        need[t] = 0;
        best[t] = ~0ull;
        SideCls c{0, 0, -1, 0, 0.f, 0.f};
        const int b = trk_off[t], m = trk_off[t + 1] - b;
        if (!rejected && m >= max(3, S.n_min)) {
            const int g0 = group_of(H.evt_off, H.G, trk_hits[b]);
            const int side0 = (g0 % NSEC) >= NPHI, ev = g0 / NSEC;
            bool one = true;
            int gl = g0;
            for (int j = 1; j < m && one; ++j) {
                gl = group_of(H.evt_off, H.G, trk_hits[b + j]);
                one = ((gl % NSEC) >= NPHI) == side0 && gl / NSEC == ev;
            }
            if (one) {
                c.r_out = H.row[trk_hits[b]];
                c.r_in = H.row[trk_hits[b + m - 1]];
                c.key_in = bucket_key(ev, gl % NSEC, c.r_in);
                c.info = (side0 << 1) | (ev << 2);
                c.z_out = H.z[trk_hits[b]];
                c.z_in = H.z[trk_hits[b + m - 1]];
                atomicAdd(&bcnt[c.key_in], 1);
            }
        }
        cls[t] = c;
    }
}

__global__ void __launch_bounds__(SIDES_T) k_sides_scatter(int32_t n_tracks, const int32_t* __restrict__ n_tracks_dev,
                                                          const SideCls* __restrict__ cls,
                                                          const int32_t* __restrict__ boff, int32_t* bfill,
                                                          int32_t* blist) {
    const int T = n_eff(n_tracks, n_tracks_dev);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        const int k = cls[t].key_in;
        if (k >= 0) blist[boff[k] + atomicAdd(&bfill[k], 1)] = t;
    }
}

// The buckets of the outer candidates of inner track t: same event, the
// other side, the same or an adjacent phi sector of its outermost cluster,
// rows r_out + 1 .. r_out + gap_max; f(o) for every track o listed there
// whose innermost cluster passes the coarse z gate with t's outermost (the
// mean apparent z within z_pre of the membrane; exact in FP64).
template <class F>
__device__ __forceinline__ void for_outer(const SideCls& a, int sec_out, const SidesPrm& S,
                                          const SideCls* __restrict__ cls, const int32_t* __restrict__ boff,
                                          const int32_t* __restrict__ blist, F f) {
    const int ev = a.info >> 2;
    const int other = (sec_out >= NPHI) ? 0 : NPHI;
    for (int dp = -1; dp <= 1; ++dp) {
        const int ph = (sec_out % NPHI + dp + NPHI) % NPHI;
        for (int gap = 1; gap <= S.gap_max; ++gap) {
            const int r = a.r_out + gap;
            if (r >= NROW) break;
            const int k = bucket_key(ev, other + ph, r);
            for (int q = boff[k]; q < boff[k + 1]; ++q) {
                const int o = blist[q];
                if (fabs(0.5 * ((double)a.z_out + (double)cls[o].z_in)) <= S.z_pre) f(o);
            }
        }
    }
}

__global__ void __launch_bounds__(SIDES_T) k_sides_need(const int32_t* __restrict__ trk_off,
                                                       const int32_t* __restrict__ trk_hits, int32_t n_tracks,
                                                       const int32_t* __restrict__ n_tracks_dev, HitSrc H, SidesPrm S,
                                                       const SideCls* __restrict__ cls,
                                                       const int32_t* __restrict__ boff,
                                                       const int32_t* __restrict__ blist, int32_t* need,
                                                       int32_t* role) {
    const int T = n_eff(n_tracks, n_tracks_dev);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        const SideCls a = cls[t];
        if (a.key_in < 0) continue;
        const int sec_out = sector_of(H, trk_hits[trk_off[t]]);
        bool any = false;
        for_outer(a, sec_out, S, cls, boff, blist, [&](int o) {
            if (o != t) {
                need[o] = 1;
                atomicOr(&role[o], 1);  // the outer role: the inward fit
                any = true;
            }
        });
        if (any) {
            need[t] = 1;
            atomicOr(&role[t], 3);  // the inner role: both fits
        }
    }
}

// The needed tracks as a dense list (need_off: exclusive scan of need), so
// that the FP64 fits and junction tests run on full warps.
__global__ void __launch_bounds__(SIDES_T) k_sides_compact(int32_t n_tracks, const int32_t* __restrict__ n_tracks_dev,
                                                          const int32_t* __restrict__ need,
                                                          const int32_t* __restrict__ need_off, int32_t* list,
                                                          SideEnd* ends) {
    const int T = n_eff(n_tracks, n_tracks_dev);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        ends[t].ok = 0;
        if (need[t]) list[need_off[t]] = t;
    }
}

// The fits each listed track's roles need: the inward fit (state at the
// innermost cluster, the segment's chi2) always, the outward fit (state at
// the outermost cluster) for the inner role.
__global__ void __launch_bounds__(SIDES_T) k_sides_fit(const int32_t* __restrict__ trk_off,
                                                      const int32_t* __restrict__ trk_hits, HitSrc H,
                                                      const Geo* __restrict__ geo, ExPrm P,
                                                      const int32_t* __restrict__ list,
                                                      const int32_t* __restrict__ n_list,
                                                      const int32_t* __restrict__ role, SideEnd* ends) {
    const int N = *n_list;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < N; u += gridDim.x * blockDim.x) {
        const int t = list[u];
        SideEnd& e = ends[t];
        const int b = trk_off[t], m = trk_off[t + 1] - b;
        KFD s;
        double c2;
        P.outward = false;
        if (!fit_ex(trk_hits + b, m, H, geo, P, s, c2, nullptr)) continue;
        for (int k = 0; k < 5; ++k) e.p_in[k] = s.p[k] + (k < 3 ? s.lo[k] : 0.0);
        for (int k = 0; k < 15; ++k) e.C_in[k] = s.C[k];
        e.x_in = s.x;
        e.s_in = s.frame;
        e.chi2_in = c2;
        int ok = 1;
        if (role[t] & 2) {
            P.outward = true;
            if (fit_ex(trk_hits + b, m, H, geo, P, s, c2, nullptr)) {
                for (int k = 0; k < 5; ++k) e.p_out[k] = s.p[k] + (k < 3 ? s.lo[k] : 0.0);
                for (int k = 0; k < 15; ++k) e.C_out[k] = s.C[k];
                e.x_out = s.x;
                e.s_out = s.frame;
                ok |= 2;
            }
        }
        e.ok = ok;
    }
}

__global__ void __launch_bounds__(SIDES_T) k_sides_pairs(const int32_t* __restrict__ trk_off,
                                                        const int32_t* __restrict__ trk_hits, HitSrc H,
                                                        const Geo* __restrict__ geo, ExPrm P, SidesPrm S,
                                                        const SideCls* __restrict__ cls,
                                                        const int32_t* __restrict__ boff,
                                                        const int32_t* __restrict__ blist,
                                                        const int32_t* __restrict__ list,
                                                        const int32_t* __restrict__ n_list,
                                                        const SideEnd* __restrict__ ends, SideCand* cand,
                                                        int32_t cap, int32_t* n_cand, int32_t* st) {
    const int N = *n_list;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < N; u += gridDim.x * blockDim.x) {
        const int t = list[u];
        const SideCls a = cls[t];
        if (a.key_in < 0 || ends[t].ok != 3) continue;
        const int sec_out = sector_of(H, trk_hits[trk_off[t]]);
        const int sgn_i = side_sgn(sec_out);
        for_outer(a, sec_out, S, cls, boff, blist, [&](int o) {
            if (o == t || !(ends[o].ok & 1)) return;
            double c4, zmem, t0s;
            if (!junction(ends[t], sgn_i, ends[o], geo, P, S, c4, zmem, t0s)) return;
            if (c4 > S.chi2_junction || fabs(zmem) > S.z_membrane) return;
            const int k = atomicAdd(n_cand, 1);
            if (k < cap) {
                cand[k].i = t;
                cand[k].o = o;
                cand[k].t0s = t0s;
            } else {
                set_status(st, TPC_ERR_CAPACITY, 301);
            }
        });
    }
}

__global__ void __launch_bounds__(SIDES_T) k_sides_joint(const int32_t* __restrict__ trk_off,
                                                        const int32_t* __restrict__ trk_hits, HitSrc H,
                                                        const Geo* __restrict__ geo, ExPrm P, SidesPrm S,
                                                        const SideEnd* __restrict__ ends, SideCand* cand,
                                                        int32_t cap, const int32_t* __restrict__ n_cand,
                                                        unsigned long long* best) {
    const int N = min(*n_cand, cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        SideCand& c = cand[k];
        const int bi = trk_off[c.i], ni = trk_off[c.i + 1] - bi;
        const int bo = trk_off[c.o], no = trk_off[c.o + 1] - bo;
        double d = INFINITY;
        if (fit_t0(trk_hits + bo, no, trk_hits + bi, ni, c.t0s, H, geo, P, S, c.q, c.C, c.chi2)) {
            d = c.chi2 - ends[c.i].chi2_in - ends[c.o].chi2_in;
            if (!(d <= S.chi2_joint)) d = INFINITY;
        }
        c.dchi2 = d;
        if (d != INFINITY) {
            atomicMin(&best[c.i], cand_key(d, c.o));
            atomicMin(&best[c.o], cand_key(d, c.i));
        }
    }
}

__global__ void __launch_bounds__(SIDES_T) k_sides_pick(const int32_t* __restrict__ trk_off,
                                                       const SideCand* __restrict__ cand, int32_t cap,
                                                       const int32_t* __restrict__ n_cand,
                                                       const unsigned long long* __restrict__ best,
                                                       int32_t* partner, double* t0, double* params6, double* cov6,
                                                       double* chi2o, int32_t* ndf, double* dchi2,
                                                       int32_t* n_pairs) {
    const int N = min(*n_cand, cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        const SideCand& c = cand[k];
        if (c.dchi2 == INFINITY) continue;
        if (best[c.i] != cand_key(c.dchi2, c.o) || best[c.o] != cand_key(c.dchi2, c.i)) continue;
        const int ni = trk_off[c.i + 1] - trk_off[c.i];
        const int no = trk_off[c.o + 1] - trk_off[c.o];
        const double* q = c.q;
        const double* C = c.C;
        const double chi2 = c.chi2;
        atomicAdd(n_pairs, 1);
        const int mem[2] = {c.i, c.o};
        for (int u = 0; u < 2; ++u) {
            const int t = mem[u];
            partner[t] = mem[1 - u];
            t0[t] = q[5];
            for (int j = 0; j < 6; ++j) params6[(int64_t)t * 6 + j] = q[j];
            for (int j = 0; j < 21; ++j) cov6[(int64_t)t * 21 + j] = C[j];
            chi2o[t] = chi2;
            ndf[t] = 2 * (ni + no) - 6;
            dchi2[t] = c.dchi2;
        }
    }
}

}  // namespace

SidesLayout sides_layout(int64_t max_tracks, int32_t n_events, int64_t cand_cap) {
    SidesLayout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += (bytes + 255) & ~(size_t)255;
        return at;
    };
    L.K = (int64_t)n_events * 2 * NPHI * NROW;
    L.ends = take(sizeof(SideEnd) * (size_t)max_tracks);
    L.cls = take(sizeof(SideCls) * (size_t)max_tracks);
    L.need = take(4 * (size_t)max_tracks);
    L.role = take(4 * (size_t)max_tracks);
    L.need_off = take(4 * (size_t)(max_tracks + 1));
    L.list = take(4 * (size_t)max_tracks);
    L.scan_t = take(4 * (size_t)(max_tracks / 4096 + 64));
    L.best = take(8 * (size_t)max_tracks);
    L.blist = take(4 * (size_t)max_tracks);
    L.bcnt = take(4 * (size_t)L.K);
    L.boff = take(4 * (size_t)(L.K + 1));
    L.bfill = take(4 * (size_t)L.K);
    L.scan = take(4 * (size_t)(L.K / 4096 + 64));
    L.cand = take(sizeof(SideCand) * (size_t)cand_cap);
    L.counters = take(4 * 4);
    L.total = o;
    return L;
}

cudaError_t run_match_sides(tpc_ctx* c, const int32_t* trk_off, const int32_t* trk_hits, int32_t n_tracks,
                            const int32_t* n_tracks_dev, const SidesPrm& S, char* ws, const SidesLayout& L,
                            int32_t cand_cap, int32_t* partner, double* t0, double* params6, double* cov6,
                            double* chi2, int32_t* ndf, double* dchi2, int32_t* n_pairs_dev, cudaStream_t s) {
    const tpc_params& p = c->prm;
    ExPrm P;
    P.sy2 = p.sigma_y2;
    P.sz2 = p.sigma_z2;
    P.kb = KAPPA * (double)p.bz;
    P.snp_max = p.snp_max;
    P.bz = p.bz;
    P.seed_snp = p.seed_snp_max;
    P.seed_qpt = p.seed_qpt_max;
    for (int i = 0; i < 5; ++i) P.prior[i] = p.prior[i];
    P.x0 = 0.0;
    P.eloss = 0.0;
    P.mass = 0.13957;
    P.outward = false;
    const HitSrc H{c->y, c->z, c->row, c->evt_sector_off, c->n_events * NSEC};
    const Geo* geo = c->ws.at<Geo>(c->ws.L.geo);
    int32_t* st = c->ws.at<int32_t>(c->ws.L.status);
    auto* ends = reinterpret_cast<SideEnd*>(ws + L.ends);
    auto* cls = reinterpret_cast<SideCls*>(ws + L.cls);
    auto* need = reinterpret_cast<int32_t*>(ws + L.need);
    auto* role = reinterpret_cast<int32_t*>(ws + L.role);
    auto* need_off = reinterpret_cast<int32_t*>(ws + L.need_off);
    auto* list = reinterpret_cast<int32_t*>(ws + L.list);
    auto* scan_t = reinterpret_cast<int32_t*>(ws + L.scan_t);
    auto* best = reinterpret_cast<unsigned long long*>(ws + L.best);
    auto* blist = reinterpret_cast<int32_t*>(ws + L.blist);
    auto* bcnt = reinterpret_cast<int32_t*>(ws + L.bcnt);
    auto* boff = reinterpret_cast<int32_t*>(ws + L.boff);
    auto* bfill = reinterpret_cast<int32_t*>(ws + L.bfill);
    auto* scan = reinterpret_cast<int32_t*>(ws + L.scan);
    auto* cand = reinterpret_cast<SideCand*>(ws + L.cand);
    auto* n_cand = reinterpret_cast<int32_t*>(ws + L.counters);
    const int64_t blocks =
        std::max<int64_t>(1, std::min<int64_t>((n_tracks + SIDES_T - 1) / SIDES_T, (int64_t)c->n_sm * 8));
    const int64_t cblocks =
        std::max<int64_t>(1, std::min<int64_t>((cand_cap + SIDES_T - 1) / SIDES_T, (int64_t)c->n_sm * 8));
    // the FP64 kernels over the dense lists: single-warp blocks, so that
    // the first entries spread over every SM's FP64 pipe
    const int64_t wblocks = std::max<int64_t>(1, std::min<int64_t>((n_tracks + 31) / 32, (int64_t)c->n_sm * 64));
    const int64_t wcblocks = std::max<int64_t>(1, std::min<int64_t>((cand_cap + 31) / 32, (int64_t)c->n_sm * 64));
    c->mark(14, s);
    cudaError_t e = fill_i32(bcnt, L.K, 0, s);
    if (e == cudaSuccess) e = fill_i32(bfill, L.K, 0, s);
    if (e == cudaSuccess) e = fill_i32(n_cand, 1, 0, s);
    if (e == cudaSuccess) e = fill_i32(n_pairs_dev, 1, 0, s);
    if (e != cudaSuccess) return e;
    if (n_tracks > 0) {
        tpc::LaunchCount{}, k_sides_class<<<(unsigned)blocks, SIDES_T, 0, s>>>(
            trk_off, trk_hits, n_tracks, n_tracks_dev, H, S, cls, need, role, best, bcnt, partner, t0, params6, cov6,
            chi2, ndf, dchi2, st);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = scan_i32(bcnt, boff, L.K, scan, s);
        if (e == cudaSuccess) {
            tpc::LaunchCount{}, k_sides_scatter<<<(unsigned)blocks, SIDES_T, 0, s>>>(n_tracks, n_tracks_dev, cls,
                                                                                 boff, bfill, blist);
            tpc::LaunchCount{}, k_sides_need<<<(unsigned)blocks, SIDES_T, 0, s>>>(
                trk_off, trk_hits, n_tracks, n_tracks_dev, H, S, cls, boff, blist, need, role);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = scan_i32(need, need_off, n_tracks, scan_t, s);
        if (e == cudaSuccess) {
            const int32_t* n_list = need_off + n_tracks;
            tpc::LaunchCount{}, k_sides_compact<<<(unsigned)blocks, SIDES_T, 0, s>>>(n_tracks, n_tracks_dev, need,
                                                                                 need_off, list, ends);
            tpc::LaunchCount{}, k_sides_fit<<<(unsigned)wblocks, 32, 0, s>>>(trk_off, trk_hits, H, geo, P, list,
                                                                          n_list, role, ends);
            tpc::LaunchCount{}, k_sides_pairs<<<(unsigned)wblocks, 32, 0, s>>>(
                trk_off, trk_hits, H, geo, P, S, cls, boff, blist, list, n_list, ends, cand, cand_cap, n_cand, st);
            tpc::LaunchCount{}, k_sides_joint<<<(unsigned)wcblocks, 32, 0, s>>>(
                trk_off, trk_hits, H, geo, P, S, ends, cand, cand_cap, n_cand, best);
            tpc::LaunchCount{}, k_sides_pick<<<(unsigned)cblocks, SIDES_T, 0, s>>>(
                trk_off, cand, cand_cap, n_cand, best, partner, t0, params6, cov6, chi2, ndf, dchi2, n_pairs_dev);
            e = cudaGetLastError();
        }
    }
    c->mark(15, s);
    return e;
}

}  // namespace tpc
