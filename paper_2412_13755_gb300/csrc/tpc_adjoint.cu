// S6: alignment chi2 and its exact gradient with respect to the 216
// per-sector rigid-body corrections.
//
// Forward: the Kalman fit of each track on corrected cluster positions
// p' = R(a,b,g) (x_row, y, z) + (dx, dy, dz) (R = Rz(g) Ry(b) Rx(a)), seeded
// from the uncorrected clusters, with a state checkpoint every CK clusters.
// Backward (hand-written reverse sweep): per checkpoint segment, recompute
// the forward states, then walk the clusters in reverse through
//   update:    p+ = p- + K r, C+ = C- - B S^-1 B^T, chi2 += r^T S^-1 r
//   transport: p- = G(p; x_from, x_to), C- = J C J^T
// carrying the adjoints of p (5) and of the symmetric C (15).  The
// derivatives of the transport Jacobian J with respect to the state and the
// plane positions come from a forward-mode evaluation of the transport with
// six tangent directions.  Per-track partials (FP32) are reduced across
// tracks in FP64 (shared-memory block sums, then global atomics).
//
// Distortion map (the online space-charge distortion evaluation of Sec. 4.2,
// read as a piecewise-constant displacement per voxel of the sector frames):
// the same kernel, instantiated with a field, adds field[v] to each corrected
// cluster and scatters the cluster's position adjoint into the gradient of
// its voxel.  A track's consecutive clusters mostly share a voxel, so each
// lane sums a run in registers and flushes it with three FP64 atomics.
#include <algorithm>

#include "tpc_adjoint.cuh"

namespace tpc {

namespace {

// Per-sector tables of the alignment correction, from the 216 parameters
// (once per call): R - I, dR/da, dR/db, dR/dg (3x3 each, acting on
// (x_row, y, z)) and the shift t.  The per-hit correction is then the small
// FP32 increment (R - I) p + t, and the angle gradient a 27-term FP32
// contraction, instead of six FP64 sines and cosines per hit.
__global__ void k_adj_tables(const double* __restrict__ align, float* tab) {
    const int sec = threadIdx.x;
    if (sec >= NSEC) return;
    adj_table_sector(align + 6 * sec, tab + sec * ROT_TAB);
}

// The kernel's sums: block shared memory for the chi2 and the 216
// alignment slots, global atomics for the field, the status word.
struct AdjAccDevice {
    double* sg;
    double* schi2;
    double* grad_field;
    int32_t* st;
    __device__ __forceinline__ void chi2(double v) { atomicAdd(schi2, v); }
    __device__ __forceinline__ void align(int i, double v) { atomicAdd(&sg[i], v); }
    __device__ __forceinline__ void field(int64_t i, double v) { atomicAdd(&grad_field[i], v); }
    __device__ __forceinline__ bool want_field() const { return grad_field != nullptr; }
    __device__ __forceinline__ void status(int code, int detail) { set_status(st, code, detail); }
};

constexpr int ADJ_T = 128;
constexpr size_t ADJ_SEG_BYTES = sizeof(float) * CK * PRE_W * ADJ_T;

// The tracks' clusters copied in track order (position, row, sector at each
// entry of trk_hits), when they fit the copy's capacity: the three sweeps
// over a track then read consecutive entries instead of one scattered
// cluster per hit three times over.
__global__ void k_adj_gather(const int32_t* __restrict__ trk_off, const int32_t* __restrict__ trk_hits,
                             int32_t T, const float* __restrict__ y, const float* __restrict__ z,
                             const uint16_t* __restrict__ row, const int64_t* __restrict__ evt_off, int G,
                             int64_t cap, float2* gyz, uint8_t* grow, uint8_t* gsec,
                             const int32_t* __restrict__ st) {
    if (input_rejected(st)) return;
    const int64_t total = trk_off[T];
    if (total > cap) return;  // the sweeps read through the hit lists instead
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int c = trk_hits[k];
        gyz[k] = make_float2(y[c], z[c]);
        grow[k] = (uint8_t)row[c];
        gsec[k] = (uint8_t)(group_of(evt_off, G, c) % NSEC);
    }
}

template <bool FIELD>
__global__ void __launch_bounds__(ADJ_T) k_adjoint(
    const int32_t* __restrict__ trk_off, const int32_t* __restrict__ trk_hits, int32_t T,
    const float* __restrict__ yin, const float* __restrict__ zin, const uint16_t* __restrict__ row,
    const int64_t* __restrict__ evt_off, int G, const float* __restrict__ rot_tab,
    const Geo* __restrict__ geo, AdjPrm P, double* chi2_total, double* grad, int32_t* st,
    const double* __restrict__ field, FieldGridD fg, double* grad_field, const float2* __restrict__ gyz,
    const uint8_t* __restrict__ grow, const uint8_t* __restrict__ gsec, int64_t gcap) {
    if (input_rejected(st)) return;  // clusters that failed validation are not read
    __shared__ double sg[216];
    __shared__ double schi2;
    __shared__ float tab[NSEC * ROT_TAB];
    // the recomputed states of each thread's current segment, one column per
    // thread (CK x PRE_W words x ADJ_T threads): the reverse sweep's working
    // set stays on chip
    extern __shared__ float seg_sh[];
    for (int i = threadIdx.x; i < NSEC * ROT_TAB; i += blockDim.x) tab[i] = rot_tab[i];
    for (int i = threadIdx.x; i < 216; i += blockDim.x) sg[i] = 0.0;
    if (threadIdx.x == 0) schi2 = 0.0;
    __syncthreads();
    AdjAccDevice acc{sg, &schi2, grad_field, st};
    const bool gathered = T > 0 && gyz != nullptr && (int64_t)trk_off[T] <= gcap;
    // tracks handed out 32 at a time to whichever warp is free, so that the
    // blocks finish together (a fixed grid stride leaves a third of the
    // threads idle at the end when tracks per thread is not whole)
    const int lane = threadIdx.x & 31;
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&st[ST_ADJ_NEXT], 32);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= T) break;
        const int t = base + lane;
        if (t < T) {
            const int b = trk_off[t];
            AdjHits hits = adj_hits_direct(trk_hits + b, yin, zin, row, evt_off, G);
            if (gathered) {
                hits.gyz = gyz;
                hits.grow = grow;
                hits.gsec = gsec;
                hits.gbase = b;
            }
            adjoint_track<FIELD>(hits, trk_off[t + 1] - b, tab, geo, P, field, fg, seg_sh + threadIdx.x, ADJ_T,
                                 acc);
        }
    }
    __syncthreads();
    if (P.want_grad && (!FIELD || grad != nullptr))
        for (int i = threadIdx.x; i < 216; i += blockDim.x)
            if (sg[i] != 0.0) atomicAdd(&grad[i], sg[i]);
    if (threadIdx.x == 0) atomicAdd(chi2_total, schi2);
}

template <bool FIELD>
cudaError_t adjoint_smem_opt_in() {
    static cudaError_t e = cudaFuncSetAttribute(k_adjoint<FIELD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)ADJ_SEG_BYTES);
    return e;
}

// The gathered copy lives in the find's binned-cluster scratch (positions,
// rows, groups: N entries each), unused between find calls.
#define ADJ_GATHER_ARGS(c, ap)                                                                    \
    (ap).want_grad ? (c)->ws.at<float2>((c)->ws.L.yzb) : nullptr, (c)->ws.at<uint8_t>((c)->ws.L.rowb), \
        (c)->ws.at<uint8_t>((c)->ws.L.grpb), (int64_t)(c)->ws.L.N

cudaError_t adj_gather(tpc_ctx* c, const int32_t* trk_off, const int32_t* trk_hits, int32_t n_tracks,
                       cudaStream_t s) {
    const int64_t blocks = (int64_t)c->n_sm * 8;
    tpc::LaunchCount{}, k_adj_gather<<<(unsigned)blocks, 256, 0, s>>>(
        trk_off, trk_hits, n_tracks, c->y, c->z, c->row, c->evt_sector_off, c->n_events * NSEC,
        (int64_t)c->ws.L.N, c->ws.at<float2>(c->ws.L.yzb), c->ws.at<uint8_t>(c->ws.L.rowb),
        c->ws.at<uint8_t>(c->ws.L.grpb), c->ws.at<int32_t>(c->ws.L.status));
    return cudaGetLastError();
}

__global__ void k_zero_f64(double* p, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = 0.0;
}

}  // namespace


cudaError_t run_adjoint(tpc_ctx* c, const int32_t* trk_off, const int32_t* trk_hits,
                        int32_t n_tracks, const double* align, double* chi2_total, double* grad,
                        cudaStream_t s) {
    const AdjPrm ap = adj_prm(c->prm, grad != nullptr);
    c->mark(12, s);
    tpc::LaunchCount{}, k_zero_f64<<<1, 32, 0, s>>>(chi2_total, 1);
    if (grad) tpc::LaunchCount{}, k_zero_f64<<<1, 256, 0, s>>>(grad, 216);
    if (n_tracks > 0) {
        float* rot_tab = c->ws.at<float>(c->ws.L.adj_rot);
        tpc::LaunchCount{}, k_adj_tables<<<1, 64, 0, s>>>(align, rot_tab);
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n_tracks + 127) / 128, 152 * 4));
        cudaError_t e = adjoint_smem_opt_in<false>();
        if (e == cudaSuccess) e = fill_i32(c->ws.at<int32_t>(c->ws.L.status) + ST_ADJ_NEXT, 1, 0, s);
        // the reverse sweep alone needs the segment store and reads each
        // track three times; forward only keeps L1 and reads through the lists
        if (e == cudaSuccess && ap.want_grad) e = adj_gather(c, trk_off, trk_hits, n_tracks, s);
        if (e != cudaSuccess) return e;
        tpc::LaunchCount{}, k_adjoint<false><<<(unsigned)blocks, ADJ_T, ap.want_grad ? ADJ_SEG_BYTES : 0, s>>>(trk_off, trk_hits, n_tracks, c->y, c->z, c->row,
                                                   c->evt_sector_off, c->n_events * NSEC, rot_tab,
                                                   c->ws.at<Geo>(c->ws.L.geo), ap, chi2_total, grad,
                                                   c->ws.at<int32_t>(c->ws.L.status),
                                                   nullptr, FieldGridD{}, nullptr, ADJ_GATHER_ARGS(c, ap));
    }
    c->mark(13, s);
    return cudaGetLastError();
}

cudaError_t run_adjoint_field(tpc_ctx* c, const int32_t* trk_off, const int32_t* trk_hits,
                              int32_t n_tracks, const double* align, const FieldGridD& fg,
                              const double* field, double* chi2_total, double* grad_align,
                              double* grad_field, cudaStream_t s) {
    const AdjPrm ap = adj_prm(c->prm, grad_align != nullptr || grad_field != nullptr);
    const int64_t nv = (int64_t)NSEC * fg.n_band * fg.n_y * fg.n_z;
    c->mark(12, s);
    tpc::LaunchCount{}, k_zero_f64<<<1, 32, 0, s>>>(chi2_total, 1);
    if (grad_align) tpc::LaunchCount{}, k_zero_f64<<<1, 256, 0, s>>>(grad_align, 216);
    if (grad_field) {
        const cudaError_t e = cudaMemsetAsync(grad_field, 0, (size_t)(3 * nv) * sizeof(double), s);
        if (e != cudaSuccess) return e;
    }
    if (n_tracks > 0) {
        float* rot_tab = c->ws.at<float>(c->ws.L.adj_rot);
        tpc::LaunchCount{}, k_adj_tables<<<1, 64, 0, s>>>(align, rot_tab);
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n_tracks + 127) / 128, 152 * 4));
        cudaError_t e = adjoint_smem_opt_in<true>();
        if (e == cudaSuccess) e = fill_i32(c->ws.at<int32_t>(c->ws.L.status) + ST_ADJ_NEXT, 1, 0, s);
        // the reverse sweep alone needs the segment store and reads each
        // track three times; forward only keeps L1 and reads through the lists
        if (e == cudaSuccess && ap.want_grad) e = adj_gather(c, trk_off, trk_hits, n_tracks, s);
        if (e != cudaSuccess) return e;
        tpc::LaunchCount{}, k_adjoint<true><<<(unsigned)blocks, ADJ_T, ap.want_grad ? ADJ_SEG_BYTES : 0, s>>>(
            trk_off, trk_hits, n_tracks, c->y, c->z, c->row, c->evt_sector_off, c->n_events * NSEC,
            rot_tab, c->ws.at<Geo>(c->ws.L.geo), ap, chi2_total, grad_align,
            c->ws.at<int32_t>(c->ws.L.status), field, fg, grad_field, ADJ_GATHER_ARGS(c, ap));
    }
    c->mark(13, s);
    return cudaGetLastError();
}

}  // namespace tpc
