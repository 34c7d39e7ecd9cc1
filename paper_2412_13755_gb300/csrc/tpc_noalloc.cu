// tpc_find_tracks_noalloc: the pattern-recognition call for callers that
// cannot allocate device memory.  Its scratch is a file-scope device array
// of fixed size (TPC_NOALLOC_SCRATCH_BYTES) that every GPU which loads this
// library holds until the process exits; the call itself allocates nothing.
#include <mutex>

#include "tpc_internal.h"

using namespace tpc;

namespace {

constexpr size_t NOALLOC_BYTES = TPC_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Device address of the scratch array, looked up once per device.  The name
// g_noalloc_scratch in host code is only a host-side stand-in, never a
// device pointer.
constexpr int MAX_DEVICES = 128;
void* g_scratch_ptr[MAX_DEVICES] = {};
std::mutex g_scratch_mu;

__global__ void k_copy_status(const int32_t* __restrict__ st, int32_t* out) { *out = st[ST_STATUS]; }

}  // namespace

extern "C" tpc_status tpc_find_tracks_noalloc(const tpc_params* params, const float* y,
                                              const float* z, const uint16_t* row, int64_t n,
                                              const int64_t* evt_sector_off, int32_t n_events,
                                              int32_t* track_of_cluster, int32_t* trk_off,
                                              int32_t* trk_hits, int32_t* n_tracks_dev,
                                              int32_t* status_dev, int32_t track_cap,
                                              tpc_stream_t stream) {
    if (n < 0 || n_events < 1 || !evt_sector_off || !track_of_cluster || !trk_off || !trk_hits ||
        !n_tracks_dev || !status_dev || track_cap < 0 || (n > 0 && (!y || !z || !row)))
        return TPC_ERR_ARG;
    if (n > TPC_NOALLOC_MAX_CLUSTERS || n_events > TPC_NOALLOC_MAX_EVENTS ||
        track_cap > TPC_NOALLOC_MAX_CLUSTERS)
        return TPC_ERR_CAPACITY;
    tpc_ctx c;
    if (params) c.prm = *params; else tpc_default_params(&c.prm);
    if (c.prm.max_gap < 1 || c.prm.max_gap > 3 || c.prm.n_seg < 3 || c.prm.n_min < 3 ||
        c.prm.ext_max_miss < 1)
        return TPC_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return TPC_ERR_CUDA;
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TPC_ERR_CUDA;
            g_scratch_ptr[dev] = p;
        }
        base = g_scratch_ptr[dev];
    }
    const Layout L = make_layout(TPC_NOALLOC_MAX_CLUSTERS, TPC_NOALLOC_MAX_EVENTS);
    if (L.total > NOALLOC_BYTES) return TPC_ERR_CAPACITY;
    c.ws.base = static_cast<char*>(base);
    c.ws.L = L;
    c.have_ws = true;
    c.y = y;
    c.z = z;
    c.row = row;
    c.charge = nullptr;
    c.n = n;
    c.n_events = n_events;
    c.evt_sector_off = evt_sector_off;
    c.have_clusters = true;
    const cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's contents: the geometry table and
    // the status word are rewritten; every other buffer is initialised by
    // the find kernels themselves
    cudaError_t e = init_geo(c.ws, s);
    if (e == cudaSuccess) e = reset_status(c.ws, s);
    if (e == cudaSuccess) e = validate_clusters(&c, s);
    if (e == cudaSuccess) e = run_find(&c, track_of_cluster, trk_off, trk_hits, n_tracks_dev, track_cap, s);
    if (e == cudaSuccess) {
        tpc::LaunchCount{}, k_copy_status<<<1, 1, 0, s>>>(c.ws.at<int32_t>(L.status), status_dev);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? TPC_OK : TPC_ERR_CUDA;
}
