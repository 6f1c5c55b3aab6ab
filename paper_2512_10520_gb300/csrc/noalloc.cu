// noalloc.cu -- the compacting transport with its scratch list in a fixed
// device array, for callers that must not allocate device memory.
//
// Who needs this: a caller whose process hands all of the GPU's memory to one
// allocator (a framework pool that reserved the device up front, so a second
// cudaMalloc fails or fragments it), a caller on a latency-critical path where
// an allocation's implicit synchronisation or its occasional multi-millisecond
// cost is not acceptable, and a caller whose memory budget must be known at
// load time.  Such callers still pass their own muon arrays; the only memory
// this entry point needs beyond them is the compaction list, and that lives in
// g_noalloc_scratch below.
//
// The array is a file-scope __device__ object: every GPU on which a handle is
// created holds its MT_NOALLOC_MAX_MUONS-sized copy until the process exits,
// and all calls on a device share that one copy.  CUDA loads a library's
// device code and objects lazily, on first use, and loading takes device
// memory; so mt_create, which allocates anyway, looks up the array and loads
// the compacting kernels of its world (noalloc_prepare below), and this entry
// point itself never triggers a load.
#include <mutex>

#include "mt_internal.cuh"

namespace mt {
int64_t compact_workspace_bytes(int64_t n);
cudaError_t compact_preload(const WorldParams &w);
}

namespace {

constexpr size_t kNoAllocBytes =
    256 + 2 * 4 * 16 * (size_t)MT_NOALLOC_MAX_MUONS + 2 * (size_t)mt::kSortBins * sizeof(unsigned);

// The compaction list (two 64-byte entries per muon), its counters, and the
// histogram and offsets of its spatial order.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on `dev` (which is current).  In host
// code the symbol name is only a stand-in for the device object, so the
// address is asked for once per device and kept.
mt_status scratch_address(int dev, void **out)
{
    if (dev < 0 || dev >= kMaxDevices) {
        mt::set_error("mt_transport_noalloc: device %d outside [0, %d)", dev, kMaxDevices);
        return MT_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return mt::cuda_fail(e, "mt_transport_noalloc: cudaGetSymbolAddress");
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return MT_OK;
}

}  // namespace

namespace mt {
// Called by mt_create with the handle's device current: creates the scratch
// array on that device and loads the kernels mt_transport_noalloc launches for
// this world.  A failure here is left for mt_transport_noalloc to report.
void noalloc_prepare(const WorldParams &w, int dev)
{
    void *p = nullptr;
    if (scratch_address(dev, &p) == MT_OK) compact_preload(w);
    cudaGetLastError();
}
}  // namespace mt

extern "C" mt_status mt_transport_noalloc(mt_handle *h, const mt_muon_soa *s, int64_t n, float step_len,
                                          int32_t max_steps, uint64_t seed, void *stream)
{
    if (!h) {
        mt::set_error("null handle");
        return MT_ERR_INVALID_ARG;
    }
    if (n > MT_NOALLOC_MAX_MUONS) {
        mt::set_error("mt_transport_noalloc takes at most %d muons per call (got %lld); split the batch or use "
                      "mt_transport_cfg with a workspace",
                      MT_NOALLOC_MAX_MUONS, (long long)n);
        return MT_ERR_INVALID_ARG;
    }
    if ((int64_t)kNoAllocBytes < mt::compact_workspace_bytes(MT_NOALLOC_MAX_MUONS)) {
        mt::set_error("mt_transport_noalloc: static scratch smaller than the compaction list needs");
        return MT_ERR_INVALID_ARG;
    }
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return mt::cuda_fail(e, "mt_transport_noalloc: cudaGetDevice");
    if (prev != h->device) {
        e = cudaSetDevice(h->device);
        if (e != cudaSuccess) return mt::cuda_fail(e, "mt_transport_noalloc: cudaSetDevice");
    }
    void *ws = nullptr;
    mt_status st = scratch_address(h->device, &ws);
    if (st == MT_OK) {
        mt_launch_cfg cfg = {MT_LAUNCH_COMPACT, 0, 0, 0, ws, (int64_t)kNoAllocBytes};
        st = mt_transport_cfg(h, s, n, step_len, max_steps, seed, nullptr, 0, &cfg, stream);
    }
    if (prev != h->device) cudaSetDevice(prev);
    return st;
}
