/*
 * tpc_track.h -- C ABI of the GB300 TPC tracking library (libtpctrack.so).
 *
 * What it computes.  ALICE's online farm runs TPC track reconstruction on
 * its GPUs; it is the step that loads them fully during data taking and
 * takes 99% of their compute (arXiv 2412.13755, Sec. 4.2 and Sec. 5), and a
 * whole time frame is processed in one operation inside GPU memory (Sec. 4).
 * The paper names the step but does not describe it; this library implements
 * it as cellular-automaton neighbour finding between pad rows, chaining and
 * Kalman-guided extension into tracklets, merging across sector boundaries,
 * a Kalman fit of the 5-parameter helix (y, z, sin phi, tan lambda, q/pT)
 * with 5x5 covariance in a uniform Bz, and the exact gradient of the summed
 * fit chi2 with respect to per-sector alignment corrections.
 *
 * Geometry: 36 sectors (phi-index s mod 18, side A for s < 18), centre angle
 * (s mod 18 + 1/2) * 20 deg, local x = X cos a + Y sin a, y = -X sin a +
 * Y cos a; 152 pad rows at x = 85 + r * 162/151 cm, accepted |y| <= x tan 10.
 *
 * Conventions for every entry point:
 *  - Array arguments are DEVICE pointers owned by the caller unless the
 *    comment says "host".  The library never allocates device memory: its
 *    scratch lives in the caller's workspace (tpc_set_workspace).
 *  - Calls are asynchronous on the given stream and never synchronise the
 *    host (except tpc_last_error and tpc_get_stats, which read back).
 *    Output counts stay on the device.
 *  - Errors: a non-zero tpc_status for argument/launch errors.  Errors found
 *    by kernels (capacity exceeded, bad cluster) are written to a device
 *    status word; tpc_last_error reads it (synchronising the stream).
 *  - No C++ exception crosses this boundary.  A context must not be used
 *    from two host threads at once; calls on one context that overlap on the
 *    GPU (different streams) race on its workspace.
 *  - Cluster indices in inputs and outputs are input-order indices.
 */
#ifndef TPC_TRACK_H
#define TPC_TRACK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* tpc_stream_t; /* = cudaStream_t, NULL = legacy default */
typedef struct tpc_ctx tpc_ctx;

typedef enum {
    TPC_OK = 0,
    TPC_ERR_ARG = 1,       /* bad argument (null pointer, size, order)        */
    TPC_ERR_CUDA = 2,      /* a CUDA call failed; tpc_last_error has the text */
    TPC_ERR_CAPACITY = 3,  /* workspace or output capacity exceeded           */
    TPC_ERR_TIMEOUT = 4,   /* a bounded device wait gave up                   */
    TPC_ERR_STATE = 5,     /* call out of order (no workspace, no clusters)   */
    TPC_ERR_INPUT = 6      /* a cluster failed validation (row >= 152, NaN)   */
} tpc_status;

/* Reconstruction parameters (cuts, windows, fit prior).  The paper gives
 * none; tpc_default_params fills the values this library is tested with. */
typedef struct {
    float win_y, win_z;        /* neighbour window |dy| <= win_y |dx| ...    */
    float chi2_link;           /* triplet D^2 cut                            */
    float sigma_y2, sigma_z2;  /* cluster variances (cm^2)                   */
    int32_t max_gap;           /* pad rows searched above / below (1..3)     */
    int32_t n_seg;             /* minimum chain length that seeds a tracklet */
    int32_t n_min;             /* minimum clusters of an output track        */
    int32_t merge_max_row_gap; /* rows allowed between merged tracklets      */
    int32_t merge_max_overlap; /* row overlap allowed across a sector border */
    float merge_z_slope, merge_z_margin; /* |dz| <= slope |dx| + margin      */
    float chi2_merge;          /* 5-d merge chi2 cut                         */
    float chi2_ext;            /* 2-d predicted-residual cut of extensions   */
    int32_t ext_max_miss;      /* extension stops after this many empty rows */
    float bz;                  /* field (T)                                  */
    float prior[5];            /* diagonal prior covariance at the seed      */
    float seed_snp_max;        /* clamp of the seed |sin phi|                */
    float seed_qpt_max;        /* clamp of the seed |q/pT| (c/GeV)           */
    float snp_max;             /* transport fails when |sin phi| reaches it  */
    float fp64_ratio;          /* tracklet building and tpc_fit_tracks_fp32:
                                  redo an update in FP64 when a posterior
                                  variance drops below fp64_ratio x prior    */
    float fp64_det;            /* ... or det S <= fp64_det S00 S11           */
    float fp64_weak_qpt;       /* reserved (not read): tpc_fit_tracks keeps
                                  its covariance in float-float for every
                                  track                                      */
} tpc_params;

/* Counters a call leaves in the workspace (read back by tpc_get_stats). */
typedef struct {
    int64_t n_clusters;
    int32_t n_segments;       /* CA chains seeding tracklets                 */
    int32_t n_tracklets;      /* tracklets kept after cluster ownership      */
    int32_t n_merge_cand;     /* merge candidates passing the chi2 cut       */
    int32_t n_merges;         /* accepted merges                             */
    int32_t n_tracks;         /* output tracks                               */
    int32_t n_fp64_updates;   /* Kalman updates redone in FP64 (all calls)   */
    int32_t status;           /* device status word (tpc_status)            */
    int32_t status_detail;
    int64_t n_launches;       /* kernels this library has launched in this
                                 process (host-side count, all contexts)    */
    int64_t n_kf_steps;       /* Kalman steps of the tracklet build in the
                                 last tpc_find_tracks                       */
    /* neighbour search of the last tpc_find_tracks: clusters without a pair
     * at the first gap pair (1,1), searched from gap sum 3 on by the 8-lane
     * kernel; clusters whose first-pass up list overflowed, searched from
     * (1,1) on by the 8-lane kernel; clusters whose 8-lane list overflowed,
     * searched again by the full-warp kernel */
    int32_t n_nb_second;
    int32_t n_nb_dense;
    int32_t n_nb_full;
    int32_t reserved;
} tpc_stats;

/* Fills p with the library's default parameters. */
void tpc_default_params(tpc_params* p);

/* Creates a context (host object; no device memory).  params may be NULL
 * for the defaults.  Returns TPC_ERR_ARG if ctx is NULL. */
tpc_status tpc_create(tpc_ctx** ctx, const tpc_params* params);
void tpc_destroy(tpc_ctx* ctx);

/* Device bytes of scratch needed for batches of up to max_clusters clusters
 * in up to max_events events (and fits / gradients of up to max_clusters
 * hits).  Pure host computation.  Returns 0 for capacities the library does
 * not take: max_clusters < 0 or > 2^30, max_events < 1, or so many events
 * that the binning's 32-bit cell keys would overflow (87,552 keys per event
 * plus one per cluster must stay below 2^31 - 17: about 24,500 events of
 * small batches, 12,300 at 2^30 clusters). */
size_t tpc_workspace_bytes(const tpc_ctx* ctx, int64_t max_clusters, int32_t max_events);

/* Hands the library a caller-owned device buffer of `bytes` (256-byte
 * aligned) sized by tpc_workspace_bytes for the same capacities.  The buffer
 * must outlive every call that uses it.  TPC_ERR_CAPACITY if too small,
 * TPC_ERR_ARG for capacities tpc_workspace_bytes refuses. */
tpc_status tpc_set_workspace(tpc_ctx* ctx, void* dev_ptr, size_t bytes,
                             int64_t max_clusters, int32_t max_events);

/* S0 (the whole time frame resident in GPU memory, Sec. 4): registers the
 * cluster arrays of a batch.  y, z: local coordinates (cm, FP32); row: pad
 * row (u16, < 152); charge: u16 (may be NULL, unused by the reconstruction);
 * n clusters in input order, grouped by event*36 + sector with device
 * offsets evt_sector_off[n_events*36 + 1] (int64, non-decreasing, first 0,
 * last n).  The arrays are read by later calls, not copied: keep them alive
 * and unchanged until the last call that uses them.  Enqueues a validation
 * kernel: a row >= 152, a non-finite coordinate or offsets that are not
 * non-decreasing from 0 to n set TPC_ERR_INPUT in the status word (detail:
 * the cluster index, or -1 / -2 / -3 for the first offset, the last offset,
 * the order).  A rejected batch is never indexed: every later kernel that
 * reads clusters or offsets checks the rejection on the device and returns
 * at once, so tpc_find_tracks yields no tracks (n_tracks_dev 0, every
 * track_of_cluster -1, trk_off all 0, trk_hits untouched), tpc_fit_tracks
 * reports every track as a failed fit (ndf -1) and the adjoint calls add
 * nothing.  The rejection holds until the next load.  TPC_ERR_CAPACITY if n
 * or n_events exceed the workspace. */
tpc_status tpc_load_clusters(tpc_ctx* ctx, const float* y, const float* z,
                             const uint16_t* row, const uint16_t* charge, int64_t n,
                             const int64_t* evt_sector_off, int32_t n_events,
                             tpc_stream_t stream);

/* S1-S4: pattern recognition of the loaded batch.
 * Outputs (device, caller-owned):
 *   track_of_cluster[n]  track index of each input cluster, -1 = none;
 *   trk_off[track_cap+1] CSR offsets of the tracks' hits;
 *   trk_hits[n]          input-order cluster indices, each track outermost
 *                        pad row first;
 *   n_tracks_dev[1]      number of tracks.
 * Tracks are ordered by their smallest input cluster index.  If more than
 * track_cap tracks are found the status word gets TPC_ERR_CAPACITY and the
 * outputs are truncated. */
tpc_status tpc_find_tracks(tpc_ctx* ctx, int32_t* track_of_cluster, int32_t* trk_off,
                           int32_t* trk_hits, int32_t* n_tracks_dev, int32_t track_cap,
                           tpc_stream_t stream);

/* S5: Kalman fit of caller-supplied hit lists over the loaded clusters.
 * trk_off[n_tracks+1], trk_hits[...] as produced by tpc_find_tracks (input
 * indices, outermost first).  n_tracks_dev (device int32, may be NULL)
 * overrides n_tracks when it is smaller, so the output of tpc_find_tracks can
 * be fed without a host round trip; n_tracks is then the capacity.  Outputs
 * per track, state at the innermost cluster in that cluster's sector frame:
 *   params[T*5]  (y, z, sin phi, tan lambda, q/pT);
 *   cov[T*15]    upper triangle row-major (00 01 02 03 04 11 12 ... 44);
 *   chi2[T]      predicted-residual chi2 (compensated FP32 sum);
 *   ndf[T]       2 n - 5, or -1 when the transport failed (params zeroed).
 * The state is FP32 with compensated y, z, sin phi; the covariance is kept
 * in float-float (hi + lo FP32 pairs, error-free transformations) through
 * every transport and update, so that C - K H C keeps its small directions
 * without FP64 arithmetic. */
tpc_status tpc_fit_tracks(tpc_ctx* ctx, const int32_t* trk_off, const int32_t* trk_hits,
                          int32_t n_tracks, const int32_t* n_tracks_dev, float* params,
                          float* cov, float* chi2, int32_t* ndf, tpc_stream_t stream);

/* S5 with the precision pattern of the tracklet lanes instead of
 * float-float: the same inputs, outputs and fit as tpc_fit_tracks (Sec. 4.2
 * names the TPC track fit as part of the GPU reconstruction), with the
 * covariance in FP32 and an update redone in FP64 when it cancels (a
 * posterior variance below fp64_ratio x its prior, or det S <= fp64_det S00
 * S11); each redo is counted in tpc_stats.n_fp64_updates.  Faster than
 * tpc_fit_tracks, with parameters within about 1e-4 of an FP64 fit instead
 * of 1e-5. */
tpc_status tpc_fit_tracks_fp32(tpc_ctx* ctx, const int32_t* trk_off, const int32_t* trk_hits,
                               int32_t n_tracks, const int32_t* n_tracks_dev, float* params,
                               float* cov, float* chi2, int32_t* ndf, tpc_stream_t stream);

/* S6: alignment chi2 and gradient.  align[216] (device FP64) holds per-sector
 * corrections (dx, dy, dz, a, b, g): a cluster's corrected position in its
 * sector frame is R(a,b,g) (x_row, y, z) + (dx, dy, dz), R = Rz(g) Ry(b) Rx(a).
 * Each track is fitted on the corrected positions (seeded from the
 * uncorrected ones); chi2_total[1] (FP64) receives the sum of the track chi2
 * and, if grad is not NULL, grad[216] (FP64) receives its exact derivative
 * (hand-written reverse sweep, per-track recomputation from checkpoints,
 * FP64 cross-track reduction).  Tracks whose transport fails contribute 0. */
tpc_status tpc_fit_adjoint(tpc_ctx* ctx, const int32_t* trk_off, const int32_t* trk_hits,
                           int32_t n_tracks, const double* align, double* chi2_total,
                           double* grad, tpc_stream_t stream);

/* Distortion map: the online TPC space-charge distortion evaluation
 * (Sec. 4.2, "Processing and calibration"; the paper gives no method), read
 * as a piecewise-constant 3-d displacement per voxel of the sector frames,
 * added to the aligned cluster position and estimated from the summed track
 * chi2.  A cluster of sector s on pad row r at local (y, z) lies in voxel
 *   v = ((s n_band + band) n_y + iy) n_z + iz,   band = r n_band / 152,
 *   iy = clamp(floor((y / x_r - u_lo) u_inv), 0, n_y - 1),
 *   iz = clamp(floor(|z| z_inv), 0, n_z - 1),
 * with the quotient, the difference and both products each rounded to FP32
 * (x_r the pad-row plane position rounded to FP32; NaN goes to bin 0). */
typedef struct {
    int32_t n_band;  /* pad-row bands, a divisor of 152                  */
    int32_t n_y;     /* bins of y / x_r                                  */
    int32_t n_z;     /* bins of |z|                                      */
    float u_lo;      /* lower edge of the y / x_r bins                   */
    float u_inv;     /* inverse width of the y / x_r bins                */
    float z_inv;     /* inverse width of the |z| bins (cm^-1)            */
} tpc_field_grid;

/* Host: number of voxels, 36 n_band n_y n_z, or -1 for an invalid grid
 * (NULL, a non-positive count, n_band not dividing 152, 2^26 voxels or more). */
int64_t tpc_field_voxels(const tpc_field_grid* grid);

/* S6 with a displacement field: as tpc_fit_adjoint, with the corrected
 * position R (x_r, y, z) + (dx, dy, dz) + field[v] (align[216] device FP64,
 * all zeros for no rigid correction; field[3 v + c] device FP64, c = x, y, z
 * in the sector frame).  chi2_total[1] receives the summed chi2; if not NULL,
 * grad_align[216] receives its derivative with respect to align and
 * grad_field[3 n_vox] its derivative with respect to the field (exact
 * reverse sweep; voxels without clusters get 0).  Returns TPC_ERR_ARG for
 * an invalid grid or a NULL align, field or chi2_total. */
tpc_status tpc_fit_adjoint_field(tpc_ctx* ctx, const int32_t* trk_off, const int32_t* trk_hits,
                                 int32_t n_tracks, const double* align,
                                 const tpc_field_grid* grid, const double* field,
                                 double* chi2_total, double* grad_align, double* grad_field,
                                 tpc_stream_t stream);

/* Reads the device status word and counters of the last calls (synchronises
 * the stream) into *out (may be NULL) and returns the status.  buf (host, may
 * be NULL) receives a one-line description. */
tpc_status tpc_get_stats(tpc_ctx* ctx, tpc_stats* out, tpc_stream_t stream);
tpc_status tpc_last_error(tpc_ctx* ctx, char* buf, size_t len);

/* Launch configuration of the work-queue kernels (S7, the batched path;
 * the paper gives none).  Two stages consume device-side queues: the
 * tracklet lanes (persistent blocks taking segments by atomic ticket) and
 * the second neighbour pass (clusters queued by the first pass, one
 * sub-warp each). */
typedef struct {
    int32_t lane_blocks_per_sm; /* tracklet lanes: persistent blocks per SM, 1..16 */
    int32_t lane_tile;          /* tracklet lanes: segments per ticket, 1..16       */
    int32_t nb_sub_lanes;       /* second neighbour pass: lanes per queued cluster,
                                   4, 8 or 16                                        */
} tpc_tune;

/* Sets the configuration used by later calls (NULL restores the default
 * 8 blocks/SM, tile 1, 8 lanes per queued cluster). */
tpc_status tpc_set_tune(tpc_ctx* ctx, const tpc_tune* tune);

/* Autotuner: runs tpc_find_tracks on the loaded batch (outputs into the
 * given buffers, as tpc_find_tracks) per candidate configuration and times
 * each with CUDA events on the stream (a warm-up pass, then a timed pass).
 * Coordinate search: the second neighbour pass's lanes per queued cluster
 * in {4, 8, 16}, then the tracklet lanes' blocks/SM in {4, 8, 16} x tile
 * in {1, 4}.  Keeps the fastest for later calls and writes it to *best (may
 * be NULL).  Every configuration gives the same tracks.  Synchronises the
 * stream; not for use during graph capture. */
tpc_status tpc_autotune(tpc_ctx* ctx, int32_t* track_of_cluster, int32_t* trk_off,
                        int32_t* trk_hits, int32_t* n_tracks_dev, int32_t track_cap,
                        tpc_tune* best, tpc_stream_t stream);

/* Stage timing (no counterpart in the paper; a measurement aid).  When
 * enabled, the library records CUDA events on the launch stream around its
 * main kernels (inside a graph captured with timing on, as event nodes of
 * the graph); tpc_stage_times then synchronises and writes, for the last
 * call or replay of each kind, the milliseconds of the stages listed in
 * TPC_STAGE_NAMES (ms_out[TPC_N_STAGES]).  Disabled by default; enabling it
 * creates the events (host-side CUDA objects, no device memory). */
#define TPC_N_STAGES 13
#define TPC_STAGE_NAMES                                                         \
    "bin", "neighbours", "links", "chains", "tracklets", "select", "merge_cand", \
        "match", "output", "fit", "adjoint", "find_total", "sides"
tpc_status tpc_stage_timing(tpc_ctx* ctx, int enable);
tpc_status tpc_stage_times(tpc_ctx* ctx, float* ms_out);

/* Pattern recognition without allocation (the paper has no counterpart;
 * this is an interface for a kind of caller).  Some callers cannot allocate
 * device memory at all: a host program or plugin whose device memory is
 * owned entirely by another allocator and that may only pass the library its
 * input and output buffers; or an online path that must not pay the implicit
 * synchronisation of cudaMalloc.  For them this call runs the same S1-S4
 * kernels as tpc_find_tracks with its scratch in a fixed device array of
 * TPC_NOALLOC_SCRATCH_BYTES that is part of the library image: every GPU
 * that loads libtpctrack holds that array until the process exits, and the
 * call itself allocates nothing (no cudaMalloc/cudaFree, no context object).
 *
 * Limits: n <= TPC_NOALLOC_MAX_CLUSTERS, n_events <= TPC_NOALLOC_MAX_EVENTS,
 * track_cap <= TPC_NOALLOC_MAX_CLUSTERS; larger requests return
 * TPC_ERR_CAPACITY before anything is launched.  params may be NULL
 * (defaults).  Inputs and outputs are as for tpc_load_clusters and
 * tpc_find_tracks (device pointers, caller-owned); status_dev (device int32)
 * receives the device status word of this call (TPC_OK, or e.g.
 * TPC_ERR_INPUT / TPC_ERR_CAPACITY found by the kernels).  Input that fails
 * validation is not indexed: the call then returns no tracks, as
 * tpc_find_tracks does after a rejected load.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array and it keeps the
 * previous call's contents; the call re-initialises what it needs.  Calls
 * whose work overlaps on the GPU (several streams or host threads at once)
 * race on the array and corrupt each other's results: serialise them. */
#define TPC_NOALLOC_MAX_CLUSTERS 65536
#define TPC_NOALLOC_MAX_EVENTS 4
#define TPC_NOALLOC_SCRATCH_BYTES (20u << 20)
tpc_status tpc_find_tracks_noalloc(const tpc_params* params, const float* y, const float* z,
                                   const uint16_t* row, int64_t n, const int64_t* evt_sector_off,
                                   int32_t n_events, int32_t* track_of_cluster, int32_t* trk_off,
                                   int32_t* trk_hits, int32_t* n_tracks_dev, int32_t* status_dev,
                                   int32_t track_cap, tpc_stream_t stream);

/* S7: the whole tracking path over one batch in one call (paper Sec. 4: a
 * time frame is processed in one operation inside GPU memory): S0 load and
 * validation, S1-S4 find, and, when params is not NULL, the S5 fit of every
 * found track, all enqueued on `stream` without a host synchronisation.
 * Inputs as for tpc_load_clusters (the batch stays registered, as after
 * that call); find outputs as for tpc_find_tracks; fit outputs have
 * track_cap rows (params[5], cov[15], chi2, ndf per track), of which the
 * first *n_tracks_dev are written.  Events of any size mix in one batch:
 * every kernel runs over all events at once, and the two queued stages
 * take their work from device-side queues (see tpc_tune). */
typedef struct {
    int32_t* track_of_cluster; /* [n]                                      */
    int32_t* trk_off;          /* [track_cap + 1]                          */
    int32_t* trk_hits;         /* [n]                                      */
    int32_t* n_tracks_dev;     /* [1]                                      */
    int32_t track_cap;
    float* params;             /* [track_cap * 5] or NULL: no fit          */
    float* cov;                /* [track_cap * 15]                         */
    float* chi2;               /* [track_cap]                              */
    int32_t* ndf;              /* [track_cap]                              */
} tpc_batch_outputs;
tpc_status tpc_track_batch(tpc_ctx* ctx, const float* y, const float* z, const uint16_t* row,
                           const uint16_t* charge, int64_t n, const int64_t* evt_sector_off,
                           int32_t n_events, const tpc_batch_outputs* out, tpc_stream_t stream);

/* S7 as one CUDA graph held by the context: records tpc_track_batch with
 * these arguments (every kernel of load, find and fit) into a graph on a
 * stream of the library's own and instantiates it, replacing any graph the
 * context held; nothing runs.  tpc_graph_launch then runs the whole batch
 * as one graph launch on `stream`.  A replay reads the same input and
 * output buffers, so refill the inputs in place between replays (the
 * sizes n and n_events are fixed by the capture).  With stage timing
 * enabled at capture time the stage events are recorded into the graph as
 * event nodes: tpc_stage_times after a replay gives that replay's stages.
 * TPC_ERR_STATE from tpc_graph_launch if nothing was captured. */
tpc_status tpc_graph_capture(tpc_ctx* ctx, const float* y, const float* z, const uint16_t* row,
                             const uint16_t* charge, int64_t n, const int64_t* evt_sector_off,
                             int32_t n_events, const tpc_batch_outputs* out);
tpc_status tpc_graph_launch(tpc_ctx* ctx, tpc_stream_t stream);

/* NEXT-3, Kalman-filter variants of the S5 fit (the paper is silent; the
 * standard refinements of a track fit).  Material concentrated in the
 * pad-row planes: a track crossing a plane is deflected by multiple
 * scattering (two projected angles of the Highland width for mat_x_x0
 * radiation lengths times the path factor 1/(cos phi cos lambda), as
 * process noise in sin phi, tan lambda and q/pT) and loses mat_eloss GeV
 * times the same factor (a deterministic map of q/pT); the fit crosses every
 * plane between two clusters of one sector.  direction 0 fits inward (state
 * arriving at the innermost cluster), 1 outward, along the motion (the
 * outward refit: state arriving at the outermost cluster). */
typedef struct {
    float mat_x_x0;    /* radiation lengths of one plane at normal incidence (0: none) */
    float mat_eloss;   /* mean energy loss in one plane at normal incidence, GeV (0: none) */
    float mass;        /* particle mass, GeV (the pion's by default)                 */
    int32_t direction; /* 0 inward, 1 outward                                        */
} tpc_fit_options;

/* tpc_fit_tracks with the options above (NULL: no material, inward), in
 * FP64 per track; outputs as for tpc_fit_tracks.  smoothed (device, may be
 * NULL; inward fits only, else TPC_ERR_ARG) receives for every cluster of
 * every fitted track the Rauch-Tung-Striebel smoothed state (5) and
 * covariance (15, packed as cov) at that cluster's plane, as doubles at
 * smoothed[20 * (trk_off[t] + j) ...] for the j-th cluster of track t (list
 * order); a failed track's entries are zero. */
tpc_status tpc_fit_tracks_ex(tpc_ctx* ctx, const int32_t* trk_off, const int32_t* trk_hits,
                             int32_t n_tracks, const int32_t* n_tracks_dev,
                             const tpc_fit_options* options, float* params, float* cov,
                             float* chi2, int32_t* ndf, double* smoothed, tpc_stream_t stream);

/* NEXT-2: clusterization of pad-time digits (paper Sec. 4.2: TPC
 * clustering runs on the GPUs; the paper gives no digit format, this is the
 * build's).  digits (device, 16-byte aligned): u16 ADC counts
 * [n_events * 36 * 152][n_time][160], one dense array per pad-row plane
 * (planes ordered by event, sector, row), pads contiguous; pad p covers
 * local y in [(p - 80) 0.6, (p - 79) 0.6) cm, time bin t covers |z| in
 * [0.5 t, 0.5 (t + 1)) cm (z < 0 on the C side).  A digit is a peak when its
 * count is >= q_peak, greater than its four neighbours earlier in raster
 * order (time, then pad) and at least its four later ones (outside the
 * array: 0).  Its cluster sums the 5 x 5 window around it (clipped):
 * charge Q, and in FP32 with one rounding per operation
 * y = (p + Sp/Q - 79.5) 0.6, |z| = (t + St/Q + 0.5) 0.5, Sp and St the
 * count-weighted pad and time offsets (exact integers).  Outputs (device,
 * caller-owned, cap entries): y, z (f32), row, charge (u16, Q clamped to
 * 65535), written per plane in raster order of the peaks, so that the
 * result is the input of tpc_load_clusters with its group offsets
 * evt_sector_off[n_events * 36 + 1] (i64); n_clusters_dev[1] the count;
 * status_dev[2] (device int32) the status and detail of this call
 * (TPC_ERR_CAPACITY when more than cap clusters, or more than 96 peaks in
 * one 32-time-bin tile of a plane, were found: the excess is dropped;
 * TPC_ERR_TIMEOUT when a tile's copy did not arrive).  workspace: device,
 * 256-byte aligned, tpc_cluster_workspace_bytes(n_events, n_time) bytes
 * (0 for n_events < 1 or n_time outside 1..4096).  Asynchronous on stream;
 * TPC_ERR_ARG / TPC_ERR_CAPACITY for bad arguments or a small workspace,
 * before anything is launched. */
size_t tpc_cluster_workspace_bytes(int32_t n_events, int32_t n_time);
tpc_status tpc_find_clusters(const uint16_t* digits, int32_t n_events, int32_t n_time,
                             int32_t q_peak, void* workspace, size_t workspace_bytes, float* y,
                             float* z, uint16_t* row, uint16_t* charge, int64_t* evt_sector_off,
                             int64_t cap, int32_t* n_clusters_dev, int32_t* status_dev,
                             tpc_stream_t stream);

/* Clears the device status word and counters (asynchronous). */
tpc_status tpc_reset_status(tpc_ctx* ctx, tpc_stream_t stream);

/* NEXT-4: the drift-time offset t0 as a sixth state parameter, and the
 * association of the A- and C-side segments of membrane-crossing tracks.
 * The paper reconstructs continuous-readout time frames (Sec. 1, Sec. 4)
 * and gives no algorithm; this is the build's reading.  A collision at
 * drift-time offset t0 (us) is seen at z' = z - v t0 on side A (sectors
 * 0..17) and z' = z + v t0 on side C.  Found tracks never span both sides,
 * so a track that crosses the central membrane is found as an inner and an
 * outer segment, on opposite sides of one phi sector (or of two adjacent
 * ones), with adjacent row ranges.  A candidate pair (inner i, outer o)
 * passes when
 *   - 1 <= row(o's innermost cluster) - row(i's outermost) <= gap_max;
 *   - before any fit, the mean of the apparent z of those two clusters is
 *     within z_pre of the membrane (segments of different collisions lie
 *     v |t0_a - t0_b| apart there; the sum of the two FP32 values is exact
 *     in FP64);
 *   - i's outward-fit state, moved to o's innermost plane, agrees with o's
 *     inward-fit state in (y, sin phi, tan lambda, q/pT): 4-d chi2 with the
 *     sum of both covariances <= chi2_junction;
 *   - the true z at the junction, the mean of the two apparent z there, is
 *     within z_membrane of the membrane;
 *   - the six-parameter fit of o's clusters then i's (state y, z, sin phi,
 *     tan lambda, q/pT, t0 with z the true z; seeded from o's three-cluster
 *     seed with t0 = (z'_o - z'_i) / (2 sgn_i v) at the junction, prior
 *     sigma t0_prior) raises the chi2 by at most chi2_joint over the two
 *     five-parameter fits.
 * Each track keeps its best candidate by (chi2 increase rounded to FP32,
 * partner index); a pair is accepted when each member is the other's best.
 * All fits in FP64.  NULL options select the defaults below. */
typedef struct {
    int32_t n_min;        /* minimum clusters of a segment (default 10)       */
    int32_t gap_max;      /* default 8                                        */
    double chi2_junction; /* default 30                                       */
    double z_membrane;    /* cm, default 3                                    */
    double z_pre;         /* cm, default 10                                   */
    double chi2_joint;    /* default 40                                       */
    double t0_prior;      /* us, default 1                                    */
    double v_drift;       /* cm/us, default 2.58                              */
} tpc_sides_options;

/* Device bytes of the caller's scratch for tpc_match_sides: max_tracks
 * tracks, n_events events, cand_cap candidate pairs after the junction
 * test.  0 for invalid sizes. */
size_t tpc_sides_workspace_bytes(int32_t max_tracks, int32_t n_events, int32_t cand_cap);

/* Pairs the segments among the found tracks trk_off[n_tracks + 1],
 * trk_hits (outermost first, input-order cluster indices of the loaded
 * batch, as tpc_find_tracks writes them) and fits each pair with t0.
 * n_tracks_dev (device, may be NULL) caps the count on the device.
 * workspace: device, 256-byte aligned, tpc_sides_workspace_bytes(n_tracks,
 * loaded events, cand_cap) bytes.  Outputs (device, caller-owned; entries
 * [0, track count) are written, both members of a pair get the pair's
 * joint fit): partner[n] (the other member, -1 none), t0[n] (us),
 * params6[6 n] (y, z, sin phi, tan lambda, q/pT, t0 at the inner segment's
 * innermost cluster, z the true z), cov6[21 n] (upper triangle row by row),
 * chi2[n], ndf[n] (2 (clusters of both) - 6; -1 unpaired), dchi2[n] (the
 * chi2 increase); n_pairs_dev[1].  More candidates than cand_cap set
 * TPC_ERR_CAPACITY in the device status word (read by tpc_get_stats); the
 * pairs are then incomplete.  Asynchronous on stream.  Errors:
 * TPC_ERR_STATE (no workspace or clusters), TPC_ERR_ARG (null pointer,
 * bad options, misaligned or short scratch), TPC_ERR_CAPACITY (n_tracks
 * above the context's track capacity). */
tpc_status tpc_match_sides(tpc_ctx* ctx, const int32_t* trk_off, const int32_t* trk_hits, int32_t n_tracks,
                           const int32_t* n_tracks_dev, const tpc_sides_options* options, void* workspace,
                           size_t workspace_bytes, int32_t cand_cap, int32_t* partner, double* t0,
                           double* params6, double* cov6, double* chi2, int32_t* ndf, double* dchi2,
                           int32_t* n_pairs_dev, tpc_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif
