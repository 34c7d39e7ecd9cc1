// C ABI of libtpctrack: context, workspace layout, argument checks, and the
// entry points declared in include/tpc_track.h.  No C++ exception leaves
// these functions.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "tpc_internal.h"
#include "tpc_sides.cuh"

using namespace tpc;

namespace tpc {

std::atomic<long long> g_launches{0};

Layout make_layout(int64_t N, int32_t E) {
    Layout L;
    L.N = N;
    L.E = E;
    L.G = (int64_t)E * NSEC;
    L.K = (int64_t)NROW * CELL_NY * L.G + N / CELL_OCC + 16;
    L.S = N / 16 + 4096;
    L.T = N + 1;
    L.KT = NMRB * (L.G + N / 64) + 16;  // (group, outer row bucket, z bin) keys
    const int64_t scan_items =
        std::max<int64_t>(std::max<int64_t>(N + 1, L.K + 1), std::max<int64_t>(L.G + 1, L.KT + 1));
    L.scan_tmp = scan_items / 4096 + 64;
    L.adj_tracks = 0;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += (bytes + 255) & ~size_t(255);
        return at;
    };
    const size_t n4 = 4 * (size_t)N, n8 = 8 * (size_t)N, s4 = 4 * (size_t)L.S, s8 = 8 * (size_t)L.S;
    const size_t g4 = 4 * (size_t)(L.G + 1);
    L.geo = take(sizeof(Geo));
    L.status = take(4 * ST_N_SLOTS);
    L.g_zmin_u = take(g4);
    L.g_zmax_u = take(g4);
    L.g_nz = take(g4);
    L.g_inv = take(g4);
    L.g_zmin = take(g4);
    L.g_kbase = take(g4);
    L.key_in = take(n4);
    L.slot_in = take(n4);
    L.cell_cnt = take(4 * (size_t)(L.K + 1));
    L.cell_off = take(4 * (size_t)(L.K + 1));
    L.yzb = take(n8);
    L.orig = take(n4);
    L.grpb = take(n4);
    L.rowb = take((size_t)N);
    L.choice_dn = take(n4);
    L.choice_up = take(n4);
    L.d2 = take(n4);
    L.claim_up = take(n8);
    L.claim_dn = take(n8);
    L.link_dn = take(n4);
    L.link_up = take(n4);
    L.owner = take(n8);
    L.seg_start = take(s4);
    L.seg_grp = take(s4);
    L.seg_canon = take(s4);
    L.tl_rowhit = take(s4 * NROW);
    L.tl_mask = take(s8 * 4);
    L.tl_n = take(s4);
    L.tl_key = take(s8);
    L.tl_keep = take(s4);
    L.tl_canon = take(s4);
    L.tl_rmin = take(s4);
    L.tl_rmax = take(s4);
    L.tl_zin = take(s4);
    L.tl_zout = take(s4);
    L.tl_state = take(s4 * 40);
    L.tl_ok = take(s4);
    const size_t kt4 = 4 * (size_t)(L.KT + 1);
    L.grp_tl_cnt = take(kt4);
    L.grp_tl_off = take(kt4 + 4);
    L.grp_tl_cur = take(kt4);
    L.tl_binkey = take(s4);
    L.tb_zmin = take(g4);
    L.tb_inv = take(g4);
    L.tb_nb = take(g4);
    L.tb_base = take(g4 + 4);
    L.tl_sorted = take(s4);
    L.gs_meta = take(s4 * 4);
    L.cand_n = take(s4);
    L.cand_a = take(s4 * MAX_CAND);
    L.cand_c2 = take(s4 * MAX_CAND);
    L.best_a = take(s8);
    L.best_b = take(s8);
    L.nxt = take(s4);
    L.prv = take(s4);
    L.match_act = take(2 * s4);
    L.trk_flag = take(n4);
    L.trk_rank = take(n4 + 4);
    L.trk_len_at = take(n4);
    L.trk_head_at = take(n4);
    L.len_by_rank = take(4 * (size_t)L.T);
    L.head_by_rank = take(4 * (size_t)L.T);
    L.scan_a = take(4 * (size_t)L.scan_tmp);
    L.scan_b = take(4 * (size_t)L.scan_tmp);
    L.adj_grad = take(8 * 216 * 2);
    L.adj_chi2 = take(8 * 2);
    L.adj_rot = take(4 * NSEC * 39);
    L.adj_ckpt = take(0);
    L.total = o;
    return L;
}

// capacities whose 32-bit indexed tables (cell keys, tracklet-bin keys,
// cluster and track indices) fit
static bool layout_ok(int64_t max_clusters, int32_t max_events) {
    if (max_clusters < 0 || max_clusters > ((int64_t)1 << 30) || max_events < 1) return false;
    const Layout L = make_layout(max_clusters, max_events);
    const int64_t lim = ((int64_t)1 << 31) - 1;
    return L.K + 1 < lim && L.KT + 1 < lim && L.T < lim && L.G + 1 < lim;
}

}  // namespace tpc

static tpc_status fail(tpc_ctx* c, tpc_status st, const char* msg) {
    if (c) {
        try {
            c->last_error = msg;
        } catch (...) {
        }
    }
    return st;
}

static tpc_status cuda_fail(tpc_ctx* c, cudaError_t e, const char* where) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
    return fail(c, TPC_ERR_CUDA, buf);
}

extern "C" {

void tpc_default_params(tpc_params* p) {
    if (!p) return;
    p->win_y = 3.0f;
    p->win_z = 3.5f;
    p->chi2_link = 16.0f;
    p->sigma_y2 = 0.01f;
    p->sigma_z2 = 0.0225f;
    p->max_gap = 3;
    p->n_seg = 5;
    p->n_min = 10;
    p->merge_max_row_gap = 24;
    p->merge_max_overlap = 8;
    p->merge_z_slope = 3.5f;
    p->merge_z_margin = 2.0f;
    p->chi2_merge = 30.0f;
    p->chi2_ext = 16.0f;
    p->ext_max_miss = 3;
    p->bz = 0.5f;
    p->prior[0] = 4.0f;
    p->prior[1] = 4.0f;
    p->prior[2] = 0.25f;
    p->prior[3] = 0.25f;
    p->prior[4] = 25.0f;
    p->seed_snp_max = 0.99f;
    p->seed_qpt_max = 5.0f;
    p->snp_max = 0.999f;
    p->fp64_ratio = 1e-4f;
    p->fp64_det = 1e-6f;
    p->fp64_weak_qpt = 1e-3f;
}

tpc_status tpc_create(tpc_ctx** ctx, const tpc_params* params) {
    if (!ctx) return TPC_ERR_ARG;
    tpc_ctx* c = new (std::nothrow) tpc_ctx();
    if (!c) return TPC_ERR_ARG;
    if (params) c->prm = *params; else tpc_default_params(&c->prm);
    if (c->prm.max_gap < 1 || c->prm.max_gap > 3 || c->prm.n_seg < 3 || c->prm.n_min < 3 ||
        c->prm.ext_max_miss < 1) {
        delete c;
        return TPC_ERR_ARG;
    }
    *ctx = c;
    return TPC_OK;
}

void tpc_destroy(tpc_ctx* ctx) {
    if (!ctx) return;
    for (auto& e : ctx->marks)
        if (e) cudaEventDestroy(e);
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    delete ctx;
}

tpc_status tpc_stage_timing(tpc_ctx* c, int enable) {
    if (!c) return TPC_ERR_ARG;
    if (enable && !c->marks[0]) {
        for (auto& e : c->marks) {
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return cuda_fail(c, r, "tpc_stage_timing");
        }
    }
    c->timing = enable != 0;
    return TPC_OK;
}

tpc_status tpc_stage_times(tpc_ctx* c, float* ms) {
    if (!c || !ms) return TPC_ERR_ARG;
    if (!c->marks[0]) return fail(c, TPC_ERR_STATE, "stage timing was never enabled");
    // pairs of marks per stage; a pair never recorded reads as 0
    static const int pairs[TPC_N_STAGES][2] = {{0, 1}, {1, 2}, {2, 3},   {3, 4},   {4, 5}, {5, 6}, {6, 7},
                                               {7, 8}, {8, 9}, {10, 11}, {12, 13}, {0, 9}, {14, 15}};
    for (int i = 0; i < TPC_N_STAGES; ++i) {
        float v = 0.f;
        if (cudaEventSynchronize(c->marks[pairs[i][1]]) == cudaSuccess &&
            cudaEventElapsedTime(&v, c->marks[pairs[i][0]], c->marks[pairs[i][1]]) != cudaSuccess) {
            v = 0.f;
            cudaGetLastError();
        }
        ms[i] = v;
    }
    return TPC_OK;
}

size_t tpc_workspace_bytes(const tpc_ctx* ctx, int64_t max_clusters, int32_t max_events) {
    (void)ctx;
    if (!layout_ok(max_clusters, max_events)) return 0;
    return make_layout(max_clusters, max_events).total;
}

tpc_status tpc_set_workspace(tpc_ctx* c, void* dev_ptr, size_t bytes, int64_t max_clusters,
                             int32_t max_events) {
    if (!c || !dev_ptr || !layout_ok(max_clusters, max_events))
        return fail(c, TPC_ERR_ARG, "tpc_set_workspace: bad argument");
    if (((uintptr_t)dev_ptr & 255) != 0) return fail(c, TPC_ERR_ARG, "workspace not 256-byte aligned");
    Layout L = make_layout(max_clusters, max_events);
    if (bytes < L.total) return fail(c, TPC_ERR_CAPACITY, "workspace too small");
    c->ws.base = static_cast<char*>(dev_ptr);
    c->ws.L = L;
    c->have_ws = true;
    c->have_clusters = false;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
        c->n_sm = sms;
    cudaError_t e = init_geo(c->ws, nullptr);
    if (e == cudaSuccess) e = reset_status(c->ws, nullptr);
    if (e != cudaSuccess) return cuda_fail(c, e, "tpc_set_workspace");
    return TPC_OK;
}

tpc_status tpc_load_clusters(tpc_ctx* c, const float* y, const float* z, const uint16_t* row,
                             const uint16_t* charge, int64_t n, const int64_t* evt_sector_off,
                             int32_t n_events, tpc_stream_t stream) {
    if (!c) return TPC_ERR_ARG;
    if (!c->have_ws) return fail(c, TPC_ERR_STATE, "no workspace");
    if (n < 0 || n_events < 1 || !evt_sector_off || (n > 0 && (!y || !z || !row)))
        return fail(c, TPC_ERR_ARG, "tpc_load_clusters: bad argument");
    if (n > c->ws.L.N || n_events > c->ws.L.E)
        return fail(c, TPC_ERR_CAPACITY, "batch larger than the workspace");
    c->y = y;
    c->z = z;
    c->row = row;
    c->charge = charge;
    c->n = n;
    c->n_events = n_events;
    c->evt_sector_off = evt_sector_off;
    c->have_clusters = true;
    cudaError_t e = validate_clusters(c, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "tpc_load_clusters");
    return TPC_OK;
}

tpc_status tpc_find_tracks(tpc_ctx* c, int32_t* toc, int32_t* trk_off, int32_t* trk_hits,
                           int32_t* n_tracks_dev, int32_t track_cap, tpc_stream_t stream) {
    if (!c) return TPC_ERR_ARG;
    if (!c->have_ws || !c->have_clusters) return fail(c, TPC_ERR_STATE, "no workspace or clusters");
    if (!toc || !trk_off || !trk_hits || !n_tracks_dev || track_cap < 0 || track_cap > c->ws.L.T - 1)
        return fail(c, TPC_ERR_ARG, "tpc_find_tracks: bad argument");
    cudaError_t e = run_find(c, toc, trk_off, trk_hits, n_tracks_dev, track_cap, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "tpc_find_tracks");
    return TPC_OK;
}

tpc_status tpc_fit_tracks(tpc_ctx* c, const int32_t* trk_off, const int32_t* trk_hits,
                          int32_t n_tracks, const int32_t* n_tracks_dev, float* params, float* cov,
                          float* chi2, int32_t* ndf, tpc_stream_t stream) {
    if (!c) return TPC_ERR_ARG;
    if (!c->have_ws || !c->have_clusters) return fail(c, TPC_ERR_STATE, "no workspace or clusters");
    if (n_tracks < 0 || (n_tracks > 0 && (!trk_off || !trk_hits || !params || !cov || !chi2 || !ndf)))
        return fail(c, TPC_ERR_ARG, "tpc_fit_tracks: bad argument");
    if (n_tracks > c->ws.L.T - 1) return fail(c, TPC_ERR_CAPACITY, "tpc_fit_tracks: too many tracks");
    cudaError_t e = run_fit(c, trk_off, trk_hits, n_tracks, n_tracks_dev, params, cov, chi2, ndf,
                            (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "tpc_fit_tracks");
    return TPC_OK;
}

tpc_status tpc_fit_tracks_fp32(tpc_ctx* c, const int32_t* trk_off, const int32_t* trk_hits,
                               int32_t n_tracks, const int32_t* n_tracks_dev, float* params, float* cov,
                               float* chi2, int32_t* ndf, tpc_stream_t stream) {
    if (!c) return TPC_ERR_ARG;
    if (!c->have_ws || !c->have_clusters) return fail(c, TPC_ERR_STATE, "no workspace or clusters");
    if (n_tracks < 0 || (n_tracks > 0 && (!trk_off || !trk_hits || !params || !cov || !chi2 || !ndf)))
        return fail(c, TPC_ERR_ARG, "tpc_fit_tracks_fp32: bad argument");
    if (n_tracks > c->ws.L.T - 1) return fail(c, TPC_ERR_CAPACITY, "tpc_fit_tracks_fp32: too many tracks");
    cudaError_t e = run_fit32(c, trk_off, trk_hits, n_tracks, n_tracks_dev, params, cov, chi2, ndf,
                              (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "tpc_fit_tracks_fp32");
    return TPC_OK;
}

tpc_status tpc_fit_tracks_ex(tpc_ctx* c, const int32_t* trk_off, const int32_t* trk_hits, int32_t n_tracks,
                             const int32_t* n_tracks_dev, const tpc_fit_options* o, float* params, float* cov,
                             float* chi2, int32_t* ndf, double* smoothed, tpc_stream_t stream) {
    if (!c) return TPC_ERR_ARG;
    if (!c->have_ws || !c->have_clusters) return fail(c, TPC_ERR_STATE, "no workspace or clusters");
    if (n_tracks < 0 || (n_tracks > 0 && (!trk_off || !trk_hits || !params || !cov || !chi2 || !ndf)))
        return fail(c, TPC_ERR_ARG, "tpc_fit_tracks_ex: bad argument");
    if (o && (o->mat_x_x0 < 0.f || o->mat_eloss < 0.f || !(o->mass > 0.f) || o->direction < 0 ||
              o->direction > 1 || (o->direction == 1 && smoothed)))
        return fail(c, TPC_ERR_ARG, "tpc_fit_tracks_ex: bad options");
    if (n_tracks > c->ws.L.T - 1) return fail(c, TPC_ERR_CAPACITY, "tpc_fit_tracks_ex: too many tracks");
    cudaError_t e = run_fit_ex(c, trk_off, trk_hits, n_tracks, n_tracks_dev, o, params, cov, chi2, ndf,
                               smoothed, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "tpc_fit_tracks_ex");
    return TPC_OK;
}

tpc_status tpc_fit_adjoint(tpc_ctx* c, const int32_t* trk_off, const int32_t* trk_hits,
                           int32_t n_tracks, const double* align, double* chi2_total, double* grad,
                           tpc_stream_t stream) {
    if (!c) return TPC_ERR_ARG;
    if (!c->have_ws || !c->have_clusters) return fail(c, TPC_ERR_STATE, "no workspace or clusters");
    if (n_tracks < 0 || !align || !chi2_total || (n_tracks > 0 && (!trk_off || !trk_hits)))
        return fail(c, TPC_ERR_ARG, "tpc_fit_adjoint: bad argument");
    cudaError_t e = run_adjoint(c, trk_off, trk_hits, n_tracks, align, chi2_total, grad,
                                (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "tpc_fit_adjoint");
    return TPC_OK;
}

static bool sides_prm(const tpc_sides_options* o, SidesPrm& S) {
    S = SidesPrm{10, 8, 30.0, 3.0, 10.0, 40.0, 1.0, 2.58};
    if (!o) return true;
    if (o->n_min < 3 || o->n_min > NROW * 4 || o->gap_max < 1 || o->gap_max >= NROW ||
        !(o->chi2_junction > 0.0) || !(o->z_membrane > 0.0) || !(o->z_pre > 0.0) || !std::isfinite(o->z_pre) ||
        !(o->chi2_joint > 0.0) ||
        !(o->t0_prior > 0.0) || !(o->v_drift > 0.0) || !std::isfinite(o->chi2_junction) ||
        !std::isfinite(o->z_membrane) || !std::isfinite(o->chi2_joint) || !std::isfinite(o->t0_prior) ||
        !std::isfinite(o->v_drift))
        return false;
    S = SidesPrm{o->n_min,      o->gap_max,    o->chi2_junction, o->z_membrane,
                 o->z_pre,      o->chi2_joint, o->t0_prior,      o->v_drift};
    return true;
}

size_t tpc_sides_workspace_bytes(int32_t max_tracks, int32_t n_events, int32_t cand_cap) {
    if (max_tracks < 0 || n_events < 1 || n_events > (1 << 16) || cand_cap < 0) return 0;
    return sides_layout(max_tracks, n_events, cand_cap).total;
}

tpc_status tpc_match_sides(tpc_ctx* c, const int32_t* trk_off, const int32_t* trk_hits, int32_t n_tracks,
                           const int32_t* n_tracks_dev, const tpc_sides_options* o, void* workspace,
                           size_t workspace_bytes, int32_t cand_cap, int32_t* partner, double* t0,
                           double* params6, double* cov6, double* chi2, int32_t* ndf, double* dchi2,
                           int32_t* n_pairs_dev, tpc_stream_t stream) {
    if (!c) return TPC_ERR_ARG;
    if (!c->have_ws || !c->have_clusters) return fail(c, TPC_ERR_STATE, "no workspace or clusters");
    SidesPrm S;
    if (!sides_prm(o, S)) return fail(c, TPC_ERR_ARG, "tpc_match_sides: bad options");
    if (n_tracks < 0 || cand_cap < 0 || !workspace || !n_pairs_dev ||
        (n_tracks > 0 && (!trk_off || !trk_hits || !partner || !t0 || !params6 || !cov6 || !chi2 || !ndf ||
                          !dchi2)))
        return fail(c, TPC_ERR_ARG, "tpc_match_sides: bad argument");
    if (((uintptr_t)workspace & 255) != 0) return fail(c, TPC_ERR_ARG, "tpc_match_sides: workspace not 256-byte aligned");
    if (n_tracks > c->ws.L.T - 1) return fail(c, TPC_ERR_CAPACITY, "tpc_match_sides: too many tracks");
    const SidesLayout L = sides_layout(n_tracks, c->n_events, cand_cap);
    if (workspace_bytes < L.total) return fail(c, TPC_ERR_ARG, "tpc_match_sides: workspace too small");
    cudaError_t e = run_match_sides(c, trk_off, trk_hits, n_tracks, n_tracks_dev, S, static_cast<char*>(workspace),
                                    L, cand_cap, partner, t0, params6, cov6, chi2, ndf, dchi2, n_pairs_dev,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "tpc_match_sides");
    return TPC_OK;
}

int64_t tpc_field_voxels(const tpc_field_grid* g) {
    if (!g || g->n_band < 1 || g->n_band > NROW || NROW % g->n_band != 0 || g->n_y < 1 ||
        g->n_z < 1 || g->n_y >= (1 << 26) || g->n_z >= (1 << 26))
        return -1;
    const int64_t nv = (int64_t)NSEC * g->n_band * g->n_y * g->n_z;
    return nv < ((int64_t)1 << 26) ? nv : -1;
}

tpc_status tpc_fit_adjoint_field(tpc_ctx* c, const int32_t* trk_off, const int32_t* trk_hits,
                                 int32_t n_tracks, const double* align, const tpc_field_grid* grid,
                                 const double* field, double* chi2_total, double* grad_align,
                                 double* grad_field, tpc_stream_t stream) {
    if (!c) return TPC_ERR_ARG;
    if (!c->have_ws || !c->have_clusters) return fail(c, TPC_ERR_STATE, "no workspace or clusters");
    if (n_tracks < 0 || !align || !field || !chi2_total || (n_tracks > 0 && (!trk_off || !trk_hits)) ||
        tpc_field_voxels(grid) < 0)
        return fail(c, TPC_ERR_ARG, "tpc_fit_adjoint_field: bad argument");
    const FieldGridD fg{grid->n_band, grid->n_y, grid->n_z, grid->u_lo, grid->u_inv, grid->z_inv};
    cudaError_t e = run_adjoint_field(c, trk_off, trk_hits, n_tracks, align, fg, field, chi2_total,
                                      grad_align, grad_field, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "tpc_fit_adjoint_field");
    return TPC_OK;
}

tpc_status tpc_set_tune(tpc_ctx* c, const tpc_tune* t) {
    if (!c) return TPC_ERR_ARG;
    if (!t) {
        c->tune = tpc_tune{8, 1, 8};
        return TPC_OK;
    }
    if (t->lane_blocks_per_sm < 1 || t->lane_blocks_per_sm > 16 || t->lane_tile < 1 || t->lane_tile > 16 ||
        (t->nb_sub_lanes != 4 && t->nb_sub_lanes != 8 && t->nb_sub_lanes != 16))
        return fail(c, TPC_ERR_ARG, "tpc_set_tune: out of range");
    c->tune = *t;
    return TPC_OK;
}

tpc_status tpc_autotune(tpc_ctx* c, int32_t* toc, int32_t* trk_off, int32_t* trk_hits,
                        int32_t* n_tracks_dev, int32_t track_cap, tpc_tune* best, tpc_stream_t stream) {
    if (!c) return TPC_ERR_ARG;
    if (!c->have_ws || !c->have_clusters) return fail(c, TPC_ERR_STATE, "no workspace or clusters");
    if (!toc || !trk_off || !trk_hits || !n_tracks_dev || track_cap < 0 || track_cap > c->ws.L.T - 1)
        return fail(c, TPC_ERR_ARG, "tpc_autotune: bad argument");
    const cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "tpc_autotune");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(c, cudaGetLastError(), "tpc_autotune");
    }
    const bool timing = c->timing;
    c->timing = false;
    tpc_tune best_t = c->tune;
    float best_ms = 1e30f;
    cudaError_t err = cudaSuccess;
    // one find per configuration, after a warm-up find of the same one
    auto time_find = [&](const tpc_tune& t, float& ms) {
        c->tune = t;
        ms = 0.f;
        for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {
            err = cudaEventRecord(e0, s);
            if (err == cudaSuccess) err = run_find(c, toc, trk_off, trk_hits, n_tracks_dev, track_cap, s);
            if (err == cudaSuccess) err = cudaEventRecord(e1, s);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        }
        if (err == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best_t = t;
        }
    };
    // coordinate search: the second neighbour pass, then the tracklet lanes
    static const int subs[3] = {4, 8, 16};
    for (int i = 0; i < 3 && err == cudaSuccess; ++i) {
        tpc_tune t = best_t;
        t.nb_sub_lanes = subs[i];
        float ms;
        time_find(t, ms);
    }
    static const int bps[3] = {4, 8, 16};
    static const int tiles[2] = {1, 4};
    const tpc_tune base = best_t;
    for (int bi = 0; bi < 3 && err == cudaSuccess; ++bi)
        for (int ti = 0; ti < 2 && err == cudaSuccess; ++ti) {
            tpc_tune t = base;
            t.lane_blocks_per_sm = bps[bi];
            t.lane_tile = tiles[ti];
            float ms;
            time_find(t, ms);
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->timing = timing;
    c->tune = best_t;
    if (err != cudaSuccess) return cuda_fail(c, err, "tpc_autotune");
    if (best) *best = best_t;
    return TPC_OK;
}

// S7: load, validation, find and fit of one batch, enqueued on one stream.
static tpc_status enqueue_batch(tpc_ctx* c, const float* y, const float* z, const uint16_t* row,
                                const uint16_t* charge, int64_t n, const int64_t* evt_sector_off,
                                int32_t n_events, const tpc_batch_outputs* o, cudaStream_t s,
                                const char* what) {
    if (!c) return TPC_ERR_ARG;
    if (!c->have_ws) return fail(c, TPC_ERR_STATE, "no workspace");
    if (!o || n < 0 || n_events < 1 || !evt_sector_off || (n > 0 && (!y || !z || !row)) ||
        !o->track_of_cluster || !o->trk_off || !o->trk_hits || !o->n_tracks_dev || o->track_cap < 0 ||
        (o->params && (!o->cov || !o->chi2 || !o->ndf)))
        return fail(c, TPC_ERR_ARG, what);
    if (n > c->ws.L.N || n_events > c->ws.L.E || o->track_cap > c->ws.L.T - 1)
        return fail(c, TPC_ERR_CAPACITY, "batch larger than the workspace");
    c->y = y;
    c->z = z;
    c->row = row;
    c->charge = charge;
    c->n = n;
    c->n_events = n_events;
    c->evt_sector_off = evt_sector_off;
    c->have_clusters = true;
    cudaError_t e = validate_clusters(c, s);
    if (e == cudaSuccess)
        e = run_find(c, o->track_of_cluster, o->trk_off, o->trk_hits, o->n_tracks_dev, o->track_cap, s);
    if (e == cudaSuccess && o->params)
        e = run_fit(c, o->trk_off, o->trk_hits, o->track_cap, o->n_tracks_dev, o->params, o->cov, o->chi2,
                    o->ndf, s);
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    return TPC_OK;
}

tpc_status tpc_track_batch(tpc_ctx* c, const float* y, const float* z, const uint16_t* row,
                           const uint16_t* charge, int64_t n, const int64_t* evt_sector_off,
                           int32_t n_events, const tpc_batch_outputs* out, tpc_stream_t stream) {
    return enqueue_batch(c, y, z, row, charge, n, evt_sector_off, n_events, out, (cudaStream_t)stream,
                         "tpc_track_batch");
}

tpc_status tpc_graph_capture(tpc_ctx* c, const float* y, const float* z, const uint16_t* row,
                             const uint16_t* charge, int64_t n, const int64_t* evt_sector_off,
                             int32_t n_events, const tpc_batch_outputs* out) {
    if (!c) return TPC_ERR_ARG;
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(c, e, "tpc_graph_capture");
    // with stage timing on, the stage events are recorded into the graph as
    // event nodes, so that every replay carries its own stage times
    c->capturing = true;
    const long long l0 = g_launches.load(std::memory_order_relaxed);
    tpc_status st = TPC_OK;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = enqueue_batch(c, y, z, row, charge, n, evt_sector_off, n_events, out, cs, "tpc_graph_capture");
        // the capture always ends, also after a failed enqueue
        e = cudaStreamEndCapture(cs, &g);
    }
    c->capturing = false;
    const long long kernels = g_launches.load(std::memory_order_relaxed) - l0;
    cudaGraphExec_t x = nullptr;
    if (st == TPC_OK && e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (st != TPC_OK) return st;
    if (e != cudaSuccess) return cuda_fail(c, e, "tpc_graph_capture");
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = x;
    c->graph_kernels = kernels;
    return TPC_OK;
}

tpc_status tpc_graph_launch(tpc_ctx* c, tpc_stream_t stream) {
    if (!c) return TPC_ERR_ARG;
    if (!c->graph) return fail(c, TPC_ERR_STATE, "no graph captured");
    const cudaError_t e = cudaGraphLaunch(c->graph, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "tpc_graph_launch");
    g_launches.fetch_add(c->graph_kernels, std::memory_order_relaxed);
    return TPC_OK;
}

tpc_status tpc_get_stats(tpc_ctx* c, tpc_stats* out, tpc_stream_t stream) {
    if (!c) return TPC_ERR_ARG;
    if (!c->have_ws) return fail(c, TPC_ERR_STATE, "no workspace");
    int32_t h[ST_N_SLOTS];
    cudaError_t e = cudaMemcpyAsync(h, c->ws.at<int32_t>(c->ws.L.status), sizeof h,
                                    cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "tpc_get_stats");
    if (out) {
        out->n_clusters = c->n;
        out->n_segments = h[ST_NSEG];
        out->n_tracklets = h[ST_NTL];
        out->n_merge_cand = h[ST_NCAND];
        out->n_merges = h[ST_NMERGE];
        out->n_tracks = h[ST_NTRACKS];
        out->n_fp64_updates = h[ST_FP64];
        out->status = h[ST_STATUS];
        out->status_detail = h[ST_DETAIL];
        out->n_launches = g_launches.load(std::memory_order_relaxed);
        long long ks;
        memcpy(&ks, &h[ST_KFSTEPS], sizeof ks);
        out->n_kf_steps = ks;
        out->n_nb_second = h[ST_NB_Q2];
        out->n_nb_dense = h[ST_NB_Q3];
        out->n_nb_full = h[ST_NB_OVF];
        out->reserved = 0;
    }
    if (h[ST_STATUS] != 0) {
        char buf[160];
        snprintf(buf, sizeof buf, "device status %d (detail %d)", h[ST_STATUS], h[ST_DETAIL]);
        fail(c, (tpc_status)h[ST_STATUS], buf);
    }
    return (tpc_status)h[ST_STATUS];
}

tpc_status tpc_last_error(tpc_ctx* c, char* buf, size_t len) {
    if (!c) return TPC_ERR_ARG;
    tpc_status st = TPC_OK;
    if (c->have_ws) st = tpc_get_stats(c, nullptr, nullptr);
    if (buf && len) {
        snprintf(buf, len, "%s", c->last_error.c_str());
    }
    return st;
}

tpc_status tpc_reset_status(tpc_ctx* c, tpc_stream_t stream) {
    if (!c) return TPC_ERR_ARG;
    if (!c->have_ws) return fail(c, TPC_ERR_STATE, "no workspace");
    cudaError_t e = reset_status(c->ws, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "tpc_reset_status");
    c->last_error.clear();
    return TPC_OK;
}

}  // extern "C"
