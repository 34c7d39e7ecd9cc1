// Internal declarations shared by the translation units of libtpctrack.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cmath>
#include <string>

#include "../../include/tpc_track.h"
#include "tpc_bits.cuh"

namespace tpc {

// kernels launched by this library in this process (host-side count)
extern std::atomic<long long> g_launches;
struct LaunchCount {
    LaunchCount() { g_launches.fetch_add(1, std::memory_order_relaxed); }
};

constexpr int NSEC = 36;
constexpr int NPHI = 18;
constexpr int NROW = 152;
constexpr int MAX_CAND = 16;     // merge candidates kept per tracklet
constexpr int CELL_OCC = 1;      // target clusters per (row, z-cell, y-cell)
constexpr int CELL_NY = 16;      // y cells per (row, z-cell), uniform in y / (x tan 10 deg)
constexpr int MRB = 8;           // outer-row bucket of the merge's tracklet bins (rows)
constexpr int NMRB = (NROW + MRB - 1) / MRB;
constexpr int NZ_MAX = 8192;     // z cells per row at most
constexpr float ZCELL_MIN = 8.f;  // shortest z cell (cm)

// Geometry table written into the workspace at set-up.
struct Geo {
    double row_xd[NROW];   // pad-row plane x (cm), FP64
    float row_xf[NROW];    // the same rounded to FP32 (neighbour decisions)
    float ycell_inv[NROW]; // CELL_NY / (2 x tan 10 deg): y-cell index scale per row
    float tan_half;        // tan(10 deg)
    float pad0;
    double tan_half_d;
    double alpha[NPHI];    // sector centre angles
    double da_cos[NPHI];   // cos / sin of the frame rotation from phi-index
    double da_sin[NPHI];   // i to phi-index (i + k) mod 18, k = 0..17
};

// The geometry table (host computation; copied to the workspace once).
inline Geo make_geo() {
    Geo g;
    const double pi = 3.14159265358979323846;
    for (int r = 0; r < NROW; ++r) {
        g.row_xd[r] = 85.0 + r * (162.0 / 151.0);
        g.row_xf[r] = (float)g.row_xd[r];
    }
    g.tan_half = (float)std::tan(10.0 * pi / 180.0);
    g.pad0 = 0.f;
    for (int r = 0; r < NROW; ++r)
        g.ycell_inv[r] = (float)(CELL_NY / (2.0 * g.row_xd[r] * std::tan(10.0 * pi / 180.0)));
    g.tan_half_d = std::tan(10.0 * pi / 180.0);
    for (int i = 0; i < NPHI; ++i) g.alpha[i] = (i + 0.5) * (20.0 * pi / 180.0);
    for (int k = 0; k < NPHI; ++k) {
        double d = g.alpha[k] - g.alpha[0];
        while (d > pi) d -= 2 * pi;
        while (d <= -pi) d += 2 * pi;
        g.da_cos[k] = std::cos(d);
        g.da_sin[k] = std::sin(d);
    }
    return g;
}

// Device status word and counters (int32 slots in the workspace).
enum StatusSlot {
    ST_STATUS = 0, ST_DETAIL, ST_NSEG, ST_NTL, ST_NCAND, ST_NMERGE, ST_NTRACKS, ST_FP64,
    ST_MATCH_LIVE, ST_Q_BUILD, ST_Q_REFIT, ST_NB_Q3, ST_KFSTEPS = 12 /* 64-bit: slots 12-13 */,
    ST_NB_OVF = 14, ST_NB_Q2 = 15,
    ST_INPUT_BAD = 16,  // nonzero when the last validated batch was rejected
    ST_ADJ_NEXT = 17,   // the adjoint's work cursor (next track to hand out)
    ST_N_SLOTS = 18
};

// Workspace layout: byte offsets of every buffer, computed from capacities.
struct Layout {
    int64_t N = 0;   // max clusters
    int32_t E = 0;   // max events
    int64_t G = 0;   // groups = E*36
    int64_t K = 0;   // cell capacity
    int64_t S = 0;   // segment / tracklet slots
    int64_t T = 0;   // output tracks capacity used internally
    int64_t KT = 0;  // tracklet (group, z-bin) keys
    int64_t scan_tmp = 0;
    size_t total = 0;
    // offsets
    size_t geo, status, g_zmin_u, g_zmax_u, g_nz, g_inv, g_zmin, g_kbase, key_in, slot_in,
        cell_cnt, cell_off, yzb, orig, grpb, rowb, choice_dn, choice_up, d2, claim_up,
        claim_dn, link_dn, link_up, owner, seg_start, seg_grp, seg_canon, tl_rowhit, tl_mask,
        tl_n, tl_key, tl_keep, tl_canon, tl_rmin, tl_rmax, tl_zin, tl_zout, tl_state, tl_ok,
        grp_tl_cnt, grp_tl_off, grp_tl_cur, tl_sorted, gs_meta, tl_binkey, tb_zmin, tb_inv, tb_nb, tb_base, cand_n, cand_a, cand_c2, best_a, best_b,
        nxt, prv, match_act, trk_flag, trk_rank, trk_len_at, trk_head_at, len_by_rank, head_by_rank, scan_a, scan_b,
        adj_grad, adj_chi2, adj_rot, adj_ckpt;
    int64_t adj_tracks = 0;  // tracks the adjoint scratch holds per launch chunk
};

Layout make_layout(int64_t max_clusters, int32_t max_events);

struct Workspace {
    char* base = nullptr;
    Layout L;
    template <class T> T* at(size_t off) const { return reinterpret_cast<T*>(base + off); }
};

}  // namespace tpc

struct tpc_ctx {
    tpc_params prm;
    tpc::Workspace ws;
    bool have_ws = false;
    // loaded batch
    const float* y = nullptr;
    const float* z = nullptr;
    const uint16_t* row = nullptr;
    const uint16_t* charge = nullptr;
    const int64_t* evt_sector_off = nullptr;
    int64_t n = 0;
    int32_t n_events = 0;
    bool have_clusters = false;
    std::string last_error;
    tpc_tune tune{8, 1, 8};
    int n_sm = 152;                     // SMs of the device (queried at set-up)
    cudaGraphExec_t graph = nullptr;    // S7 graph (tpc_graph_capture)
    long long graph_kernels = 0;        // kernels in that graph
    // stage timing: marks 0..9 around the find stages, 10/11 fit, 12/13 adjoint,
    // 14/15 the A/C-side association
    bool timing = false;
    bool capturing = false;  // inside tpc_graph_capture: marks become event nodes of the graph
    cudaEvent_t marks[16] = {};
    void mark(int i, cudaStream_t s) {
        if (timing) cudaEventRecordWithFlags(marks[i], s, capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
    }
};

namespace tpc {
// launchers (return cudaGetLastError of their launches)
cudaError_t init_geo(const Workspace& ws, cudaStream_t s);
cudaError_t reset_status(const Workspace& ws, cudaStream_t s);
cudaError_t validate_clusters(const tpc_ctx* c, cudaStream_t s);
cudaError_t run_find(tpc_ctx* c, int32_t* toc, int32_t* trk_off, int32_t* trk_hits,
                     int32_t* n_tracks_dev, int32_t track_cap, cudaStream_t s);
cudaError_t run_fit(tpc_ctx* c, const int32_t* trk_off, const int32_t* trk_hits, int32_t n_tracks,
                    const int32_t* n_tracks_dev, float* params, float* cov, float* chi2,
                    int32_t* ndf, cudaStream_t s);
cudaError_t run_fit32(tpc_ctx* c, const int32_t* trk_off, const int32_t* trk_hits, int32_t n_tracks,
                      const int32_t* n_tracks_dev, float* params, float* cov, float* chi2,
                      int32_t* ndf, cudaStream_t s);
cudaError_t run_fit_ex(tpc_ctx* c, const int32_t* trk_off, const int32_t* trk_hits, int32_t n_tracks,
                       const int32_t* n_tracks_dev, const tpc_fit_options* o, float* params, float* cov,
                       float* chi2, int32_t* ndf, double* smoothed, cudaStream_t s);
cudaError_t run_adjoint(tpc_ctx* c, const int32_t* trk_off, const int32_t* trk_hits,
                        int32_t n_tracks, const double* align, double* chi2_total, double* grad,
                        cudaStream_t s);
cudaError_t run_adjoint_field(tpc_ctx* c, const int32_t* trk_off, const int32_t* trk_hits,
                              int32_t n_tracks, const double* align, const FieldGridD& fg,
                              const double* field, double* chi2_total, double* grad_align,
                              double* grad_field, cudaStream_t s);
// NEXT-4: the A/C-side association (tpc_sides.cu); its scratch is the
// caller's (tpc_sides_workspace_bytes)
struct SidesPrm;
struct SidesLayout {
    int64_t K;  // buckets: events x 2 sides x 18 phi sectors x 152 rows
    size_t ends, cls, need, role, need_off, list, scan_t, best, blist, bcnt, boff, bfill, scan, cand, counters, total;
};
SidesLayout sides_layout(int64_t max_tracks, int32_t n_events, int64_t cand_cap);
cudaError_t run_match_sides(tpc_ctx* c, const int32_t* trk_off, const int32_t* trk_hits, int32_t n_tracks,
                            const int32_t* n_tracks_dev, const SidesPrm& S, char* ws, const SidesLayout& L,
                            int32_t cand_cap, int32_t* partner, double* t0, double* params6, double* cov6,
                            double* chi2, int32_t* ndf, double* dchi2, int32_t* n_pairs_dev, cudaStream_t s);
cudaError_t fill_i32(int32_t* p, int64_t n, int32_t v, cudaStream_t s);
// exclusive scan of in[0..L) into out[0..L] (out[L] = total); tmp from the workspace
cudaError_t scan_i32(const int32_t* in, int32_t* out, int64_t L, int32_t* tmp, cudaStream_t s);
}  // namespace tpc
