/*
 * TPC tracking oracle: a plain, slow, FP64 CPU restatement of the tracking
 * path (row binning, cellular-automaton neighbour finding, chaining, segment
 * merging, Kalman fit, alignment gradient).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA library and the CUDA library never calls it.
 *
 * The paper (ALICE O2 EPN farm, arXiv 2412.13755) states that TPC tracking
 * runs on the GPUs and takes 99% of their compute (Sec. 4.2, Sec. 5) but
 * gives no algorithm; every rule here is the build's stated reading, listed
 * beside each function.  Arrays are host pointers owned by the caller.
 */
#ifndef TPC_ORACLE_H
#define TPC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    float win_y;              /* |y_u - y_c| <= win_y |x_u - x_c|           */
    float win_z;              /* |z_u - z_c| <= win_z |x_u - x_c|           */
    float chi2_link;          /* triplet D^2 cut                            */
    float sigma_y2, sigma_z2; /* measurement variances (cm^2)               */
    int32_t max_gap;          /* rows searched on each side (1..max_gap)    */
    int32_t n_seg;            /* minimum chain length kept as a segment     */
    int32_t n_min;            /* minimum clusters of an output track        */
    int32_t merge_max_row_gap;/* row gap allowed between merged segments    */
    int32_t merge_max_overlap;/* row overlap allowed across a sector border */
    float merge_z_slope;      /* z gate: |dz| <= slope * dx + margin        */
    float merge_z_margin;
    double chi2_merge;        /* 5-d merge chi2 cut                         */
    double chi2_ext;          /* 2-d predicted-residual cut of extensions   */
    int32_t ext_max_miss;     /* extension stops after this many empty rows */
    double bz;                /* field (T)                                  */
    double prior[5];          /* diagonal prior covariance of the fit seed  */
    double seed_snp_max;      /* clamp of the seed |sin phi|                */
    double seed_qpt_max;      /* clamp of the seed |q/pT| (c/GeV)           */
    double snp_max;           /* transport fails when |sin phi| reaches it  */
    int32_t s2_fp64;          /* 1: window tests and triplet D^2 in FP64 (a
                                 diagnostic mode; 0, the default, decides in
                                 FP32 with one rounding per operation)      */
    double mat_x_x0;          /* material of one pad-row plane, radiation
                                 lengths at normal incidence (0: none)      */
    double mat_eloss;         /* mean energy loss in one plane at normal
                                 incidence (GeV; 0: none)                   */
    double mass;              /* particle mass for the material (GeV)       */
} orc_params;

/* Fills the default parameter set of the build's reading. */
void orc_default_params(orc_params* p);

/* Per-cluster diagnostics of the neighbour step (input-order indices). */
typedef struct {
    int32_t* choice_dn;   /* [n] chosen down partner of each cluster or -1 */
    int32_t* choice_up;   /* [n] chosen up partner or -1                    */
    float*   d2;          /* [n] D^2 of the chosen triplet                  */
    float*   d2_next;     /* [n] runner-up D^2 at the winning gap pair (inf)*/
    int32_t* link_dn;     /* [n] final down link or -1                      */
    int32_t* link_up;     /* [n] final up link or -1                        */
    int32_t* seg_of;      /* [n] segment id (canonical order) or -1         */
    double*  merge_margin;/* [n] relative margin of the merge decision that
                             placed this cluster's segment (inf: none)      */
    double*  ext_margin;  /* [n] smallest relative margin of the extension
                             decisions in which this cluster was the best
                             or second-best candidate of a row: best chi2
                             against the cut and against the runner-up
                             (inf: none)                                    */
} orc_diag;

/* S1-S4: whole pipeline.  Inputs in input order, grouped per event*36+sector
 * by evt_sector_off[n_events*36+1].  Outputs: track_of_cluster[n] (canonical
 * track index or -1), trk_off[cap+1], trk_hits[n] (input-order indices,
 * outermost first).  Returns the number of tracks, or -1 on bad input.
 * diag may be NULL. */
int64_t orc_find_tracks(const float* y, const float* z, const uint16_t* row,
                        int64_t n, const int64_t* evt_sector_off,
                        int32_t n_events, const orc_params* prm,
                        int32_t* track_of_cluster, int32_t* trk_off,
                        int32_t* trk_hits, orc_diag* diag);

/* S5: FP64 Kalman fit of caller hit lists (outermost first).  The state is
 * reported at the innermost cluster.  sector_of[n] gives each cluster's
 * sector.  align[216] (or NULL) holds per-sector corrections applied to the
 * cluster positions.  params[T*5], cov[T*15], chi2[T], ndf[T] (ndf = -1 when
 * the transport fails).  Returns 0. */
int orc_fit_tracks(const float* y, const float* z, const uint16_t* row,
                   const int32_t* sector_of, const int32_t* trk_off,
                   const int32_t* trk_hits, int32_t n_tracks,
                   const double* align, const orc_params* prm,
                   double* params, double* cov, double* chi2, int32_t* ndf);

/* Same fit, hits consumed in the order given (reverse = 1: innermost first,
 * state reported at the outermost cluster). */
int orc_fit_tracks_dir(const float* y, const float* z, const uint16_t* row,
                       const int32_t* sector_of, const int32_t* trk_off,
                       const int32_t* trk_hits, int32_t n_tracks,
                       const double* align, const orc_params* prm, int reverse,
                       double* params, double* cov, double* chi2, int32_t* ndf);

/* S6: total chi2 over tracks and (if grad != NULL) its exact derivative with
 * respect to the 216 alignment parameters, by forward-mode dual numbers
 * through the FP64 fit.  Failed fits contribute nothing. */
int orc_fit_adjoint(const float* y, const float* z, const uint16_t* row,
                    const int32_t* sector_of, const int32_t* trk_off,
                    const int32_t* trk_hits, int32_t n_tracks,
                    const double* align, const orc_params* prm,
                    double* chi2_total, double* grad);

/* Gauss-Newton matrix (216x216, row-major) of the total chi2 from the
 * residual derivatives, for the alignment descent and null-mode analysis. */
int orc_gauss_newton(const float* y, const float* z, const uint16_t* row,
                     const int32_t* sector_of, const int32_t* trk_off,
                     const int32_t* trk_hits, int32_t n_tracks,
                     const double* align, const orc_params* prm, double* gn);

/* The fit seed of a hit list given in fit order (first_is_outer = 1 for
 * the inward fit): plane x0 and frame of the first cluster, state p[5]. */
int orc_seed(const float* y, const float* z, const uint16_t* row, const int32_t* sector_of,
             const int32_t* hits, int32_t n, int first_is_outer, const orc_params* prm,
             double* x0, int32_t* frame, double* p);

/* The same seed for points given in FP64 (pins with exact helix points). */
int orc_seed_f64(const double* y, const double* z, const uint16_t* row, const int32_t* sector_of,
                 const int32_t* hits, int32_t n, int first_is_outer, const orc_params* prm,
                 double* x0, int32_t* frame, double* p);

/* S3b of one segment (seg_hits outermost first, all in the group [beg, end)
 * of sector `sector`): the tracklet the find builds from it, outermost
 * first, into out[cap].  Returns its length, -1 for a bad argument, or
 * -(length) when cap is too small. */
int64_t orc_tracklet(const float* y, const float* z, const uint16_t* row, int64_t beg,
                     int64_t end, int32_t sector, const int32_t* seg_hits, int32_t nseg,
                     const orc_params* prm, int32_t* out, int32_t cap);

/* S4 of two segments (hits outermost first): inner A in sector sec_a,
 * outer B in sec_b, each fitted as the find fits its tracklets.  Writes the
 * chi2_5 of A's state moved to B's innermost plane against B's state there,
 * and whether the merge's gates and cut accept the pair.  Returns 0, 1 for
 * a bad argument, 2 when a fit or the move fails. */
int orc_merge_chi2(const float* y, const float* z, const uint16_t* row, const int32_t* hits_a,
                   int32_t na, int32_t sec_a, const int32_t* hits_b, int32_t nb, int32_t sec_b,
                   const orc_params* prm, double* chi2, int32_t* gates_pass);

/* Work of the fit: the arithmetic operations (+ - * /, square roots and
 * arcsines; operations on exact zeros and multiplications by exact ones,
 * the Jacobians' structure, not counted) that the FP64 fit of the given
 * tracks performs, summed, and the number of Kalman steps (clusters)
 * taken.  Single-threaded.  Returns 0. */
int orc_kf_ops(const float* y, const float* z, const uint16_t* row, const int32_t* sec,
               const int32_t* trk_off, const int32_t* trk_hits, int32_t T,
               const orc_params* prm, double* ops, int64_t* steps);

/* NEXT-3: the fit with a Rauch-Tung-Striebel smoother.  The inward fit of
 * each track (material per the orc_params) records, per hit, its predicted
 * and filtered states and the prediction's Jacobian; the smoother then runs
 * back from the innermost hit.  out[(trk_off[t] + j) * 20 ...] receives the
 * smoothed state (5) and covariance (15) at the j-th hit of track t (list
 * order, outermost first; the state arriving at that hit's plane).  chi2 and
 * ndf as for orc_fit_tracks.  A failed track gets zeros and ndf -1. */
int orc_smooth_tracks(const float* y, const float* z, const uint16_t* row, const int32_t* sector_of,
                      const int32_t* trk_off, const int32_t* trk_hits, int32_t n_tracks,
                      const orc_params* prm, double* out, double* chi2, int32_t* ndf);

/* NEXT-2: clusters of pad-time digits (u16 [n_events*36*152][n_time][160],
 * planes ordered by event, sector, row): peaks by the raster rule, 5 x 5
 * count-weighted centroids (see the source), written per plane in raster
 * order of the peaks into y, z, row, charge (cap entries) with group
 * offsets evt_sector_off[n_events*36 + 1].  Returns the number of
 * clusters, or -(number) when cap is too small. */
int64_t orc_find_clusters(const uint16_t* digits, int32_t n_events, int32_t n_time, int32_t q_peak,
                          float* y, float* z, uint16_t* row, uint16_t* charge,
                          int64_t* evt_sector_off, int64_t cap);

/* One propagation: state p (y, z, sin phi, tan lambda, q/pT) at plane x1 of
 * sector s1 -> plane x2 of sector s2.  Writes p_out[5], jac[25] (row-major
 * d p_out / d p) and dx1[5], dx2[5].  Returns 0, or 1 when it fails. */
int orc_propagate(double x1, int s1, const double* p, double x2, int s2,
                  const orc_params* prm, double* p_out, double* jac,
                  double* dx1, double* dx2);

/* C10: all admissible chains of one (event, sector) group: strictly rising
 * rows, row steps <= max_gap, each interior triplet inside the windows with
 * D^2 <= chi2_link, length >= n_min, and FP64 fit chi2/ndf <= chi2ndf_max.
 * Writes chains innermost first into out_hits with offsets out_off.
 * Returns the number of chains, or -(needed) when a capacity is too small. */
int64_t orc_bruteforce_chains(const float* y, const float* z, const uint16_t* row,
                              int64_t n, int32_t sector, const orc_params* prm,
                              double chi2ndf_max, int64_t cap_chains,
                              int64_t cap_hits, int32_t* out_off,
                              int32_t* out_hits);

/* Distortion map: a displacement field over voxels of the sector frames,
 * the quantity the online TPC space-charge distortion evaluation estimates
 * (Sec. 4.2, "Processing and calibration"; the paper gives no method).  The
 * reading: a piecewise-constant 3-d displacement per voxel, added to the
 * (aligned) cluster position, estimated by minimising the summed track chi2.
 * A cluster of sector s on pad row r at local (y, z) lies in voxel
 *   v = ((s n_band + band) n_y + iy) n_z + iz,   band = r n_band / 152,
 *   iy = clamp(floor((y / x_r - u_lo) u_inv), 0, n_y - 1),
 *   iz = clamp(floor(|z| z_inv), 0, n_z - 1),
 * the quotient, the difference and both products each rounded to FP32
 * (x_r the pad-row plane position rounded to FP32), so that membership is
 * an exact function of the measured cluster. */
typedef struct {
    int32_t n_band, n_y, n_z;   /* row bands (divide 152 rows), y/x bins, |z| bins */
    float u_lo, u_inv;          /* y/x bins: lower edge and inverse width          */
    float z_inv;                /* |z| bins: inverse width (cm^-1)                 */
} orc_field_grid;

/* Voxel of each cluster (vox[n]); returns the number of voxels,
 * 36 n_band n_y n_z, or -1 for an invalid grid. */
int64_t orc_voxel_of(const float* y, const float* z, const uint16_t* row,
                     const int32_t* sector_of, int64_t n, const orc_field_grid* grid,
                     int32_t* vox);

/* Summed fit chi2 with the corrected positions R (x_r, y, z) + D + field[v]
 * (align[216] as in orc_fit_adjoint, may be NULL = none; field[3 v + c],
 * c = x, y, z in the sector frame) and, if grad_field is not NULL, its exact
 * derivative d chi2 / d field (forward-mode dual numbers, eight voxels of a
 * track per pass).  Returns 0, or -1 for an invalid grid. */
int orc_field_adjoint(const float* y, const float* z, const uint16_t* row,
                      const int32_t* sector_of, const int32_t* trk_off,
                      const int32_t* trk_hits, int32_t n_tracks, const double* align,
                      const orc_field_grid* grid, const double* field,
                      const orc_params* prm, double* chi2_total, double* grad_field);

/* Per-voxel 3x3 diagonal blocks of the Gauss-Newton matrix of the summed
 * chi2 with respect to the field: sum over tracks and clusters of
 * 2 dr^T S^-1 dr, dr the derivative of each predicted residual with respect
 * to the voxel's three components (through the whole fit, dual numbers).
 * blocks[9 v + 3 a + b]; voxels without clusters get 0.  Returns 0, or -1
 * for an invalid grid.  The preconditioner of a block-Jacobi descent. */
int orc_field_gn_blocks(const float* y, const float* z, const uint16_t* row,
                        const int32_t* sector_of, const int32_t* trk_off,
                        const int32_t* trk_hits, int32_t n_tracks, const double* align,
                        const orc_field_grid* grid, const double* field,
                        const orc_params* prm, double* blocks);

/* NEXT-4: the drift-time offset t0 as a sixth state parameter.  A
 * collision at offset t0 (us) is seen at z' = z - v t0 on side A (sectors
 * 0..17) and z' = z + v t0 on side C.  The association pairs the one-side
 * found tracks that are the inner and outer segments of one
 * membrane-crossing track (the build's reading; the paper gives no
 * algorithm: it reconstructs continuous-readout time frames, Sec. 1 and
 * Sec. 4). */
typedef struct {
    int32_t n_min;         /* minimum clusters of a segment                   */
    int32_t gap_max;       /* 1 <= row(outer's innermost) - row(inner's
                              outermost) <= gap_max                           */
    double chi2_junction;  /* 4-d (y, sin phi, tan lambda, q/pT) junction cut */
    double z_membrane;     /* |true z at the junction| cut (cm)               */
    double z_pre;          /* coarse gate before any fit: |z'(i's outermost
                              cluster) + z'(o's innermost)| / 2 <= z_pre (cm) */
    double chi2_joint;     /* cut on the joint fit's chi2 increase            */
    double t0_prior;       /* prior sigma of t0 in the joint fit (us)         */
    double v_drift;        /* drift velocity (cm/us)                          */
} orc_sides_params;

void orc_default_sides_params(orc_sides_params* p);

/* The six-parameter fit (y, z, sin phi, tan lambda, q/pT, t0; z the true
 * z) of hits[0..n): the first n_outer are the outer segment (outermost
 * first, one side), the rest continue inward on the other side.  Seeded
 * from the outer segment's three-cluster seed with t0 = t0_seed.  State at
 * the innermost cluster; cov6 packed as the upper triangle row by row (21).
 * Returns 0, 1 when the fit fails. */
int orc_fit_t0(const float* y, const float* z, const uint16_t* row, const int32_t* sector_of,
               const int32_t* hits, int32_t n, int32_t n_outer, double t0_seed,
               const orc_params* prm, const orc_sides_params* sp, double* params6,
               double* cov6, double* chi2);

/* Pairs the A- and C-side segments of membrane-crossing tracks among the
 * found tracks (trk_off[T + 1], trk_hits: outermost first) and fits each
 * pair with t0.  Outputs per track (both members of a pair get its joint
 * fit): partner[T] (-1 none), t0[T], params6[6 T], cov6[21 T], chi2[T],
 * ndf[T], dchi2[T] (the joint fit's chi2 increase); margin[T] (may be
 * NULL): smallest relative margin of the decisions that involved the track.
 * Returns the number of pairs, -1 on invalid input. */
int64_t orc_match_sides(const float* y, const float* z, const uint16_t* row, int64_t n,
                        const int64_t* off, int32_t n_events, const int32_t* trk_off,
                        const int32_t* trk_hits, int32_t T, const orc_params* prm,
                        const orc_sides_params* sp, int32_t* partner, double* t0,
                        double* params6, double* cov6, double* chi2, int32_t* ndf,
                        double* dchi2, double* margin);

/* Threads used by the OpenMP loops (0 = library default). */
void orc_set_threads(int n);
int orc_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
