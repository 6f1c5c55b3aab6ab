// transport.cu -- sm_103a kernels of the plain transport (Algorithm 1 of
// "Ultra-Fast Muon Transport via Histogram Sampling on GPUs"): a static grid with
// one thread per muon for its whole track, and a persistent grid whose lanes
// pick up the next muon of their block's range when the current one stops.
#include <cfloat>
#include <cstdio>

#include "step.cuh"

namespace mt {

// Static form: one thread per muon (grid-stride), the whole track in one go.
template <int GEOM, int FIELD>
__global__ void __launch_bounds__(kBlock) transport_kernel(const WorldParams w, const mt_muon_soa soa, int64_t n,
                                                           const RunParams rp)
{
    __shared__ SmemWorld sw;
    stage_world(sw, w, rp);
    __syncthreads();
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x) {
        State s;
        float q;
        int k;
        uint32_t id_lo, id_hi;
        if (!load_muon(w, soa, m, rp, s, q, k, id_lo, id_hi)) continue;
        int out = MT_MAX_STEPS;
#pragma unroll 1
        for (; k < rp.max_steps; ++k) {
            const int r = step<GEOM, FIELD>(w, sw, s, q, k, id_lo, id_hi, (uint32_t)rp.instance, rp);
            if (r != MT_ALIVE) {
                out = r;
                break;
            }
        }
        store_muon(w, soa, m, s, k, out);
    }
}

// Persistent form: a resident grid; block b owns the contiguous muon range
// [b n / B, (b+1) n / B) and its lanes take the next muon of that range from a
// shared counter as soon as their current muon stops, so warps stay full while
// track lengths differ (a few steps to max_steps).  The counter is claimed once
// per warp per refill (ballot + popc); every loop bound is finite (the range is
// finite and each muon runs at most max_steps steps).
template <int GEOM, int FIELD>
__global__ void __launch_bounds__(kBlock) transport_persistent(const WorldParams w, const mt_muon_soa soa, int64_t n,
                                                               const RunParams rp)
{
    __shared__ SmemWorld sw;
    __shared__ unsigned long long next;
    const int64_t begin = n * (int64_t)blockIdx.x / gridDim.x;
    const int64_t end = n * (int64_t)(blockIdx.x + 1) / gridDim.x;
    stage_world(sw, w, rp);
    if (threadIdx.x == 0) next = (unsigned long long)begin;
    __syncthreads();
    const unsigned lane = threadIdx.x & 31u;
    int64_t m = -1;   // -1: needs a muon; end: range exhausted
    State s;
    float q = 0.0f;
    int k = 0;
    uint32_t id_lo = 0, id_hi = 0;
#pragma unroll 1
    while (true) {
        const bool need = m < 0;
        const unsigned need_mask = __ballot_sync(0xFFFFFFFFu, need);
        if (need_mask) {
            const int leader = __ffs(need_mask) - 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(&next, (unsigned long long)__popc(need_mask));
            base = __shfl_sync(0xFFFFFFFFu, base, leader);
            if (need) {
                const int64_t cand = (int64_t)base + __popc(need_mask & ((1u << lane) - 1u));
                if (cand >= end)
                    m = end;
                else if (load_muon(w, soa, cand, rp, s, q, k, id_lo, id_hi))
                    m = cand;
            }
        }
        if (__all_sync(0xFFFFFFFFu, m == end)) break;
        if (m >= 0 && m < end) {
            int r = MT_ALIVE;
            if (k >= rp.max_steps)
                r = MT_MAX_STEPS;
            else
                r = step<GEOM, FIELD>(w, sw, s, q, k, id_lo, id_hi, (uint32_t)rp.instance, rp);
            if (r != MT_ALIVE) {
                store_muon(w, soa, m, s, k, r);
                m = -1;
            } else {
                ++k;
            }
        }
    }
}

__global__ void repack_field_kernel(const float *raw, float4 *pairs, int nx, int ny, int nz)
{
    const int64_t total = (int64_t)(nx - 1) * ny * nz;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % (nx - 1);
        const int64_t jk = e / (nx - 1);
        const int64_t j = jk % ny, k = jk / ny;
        const float *n0 = raw + 3 * ((k * ny + j) * nx + i);
        pairs[2 * e] = make_float4(n0[0], n0[1], n0[2], 0.0f);
        pairs[2 * e + 1] = make_float4(n0[3], n0[4], n0[5], 0.0f);
    }
}

cudaError_t launch_repack_field(const float *raw, float4 *pairs, int nx, int ny, int nz, cudaStream_t st)
{
    const int64_t total = (int64_t)(nx - 1) * ny * nz;
    const int64_t blocks = (total + 255) / 256;
    repack_field_kernel<<<(unsigned)(blocks < 65535 * 16 ? blocks : 65535 * 16), 256, 0, st>>>(raw, pairs, nx, ny, nz);
    return cudaGetLastError();
}

template <int GEOM, int FIELD>
static cudaError_t launch(const WorldParams &w, const mt_muon_soa &s, int64_t n, const RunParams &rp, cudaStream_t st,
                          const mt_launch_cfg &cfg)
{
    if (cfg.mode == MT_LAUNCH_STATIC || cfg.mode == MT_LAUNCH_AUTO) {   // AUTO here only for n >= 2^31
        const int64_t blocks = (n + kBlock - 1) / kBlock;
        const unsigned grid = (unsigned)(blocks < 0x7FFFFFFF ? blocks : 0x7FFFFFFF);
        transport_kernel<GEOM, FIELD><<<grid, kBlock, 0, st>>>(w, s, n, rp);
        return cudaGetLastError();
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, transport_persistent<GEOM, FIELD>, kBlock, 0);
    if (cfg.blocks_per_sm > 0 && cfg.blocks_per_sm < per_sm) per_sm = cfg.blocks_per_sm;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sms * per_sm;
    const int64_t max_useful = (n + kBlock - 1) / kBlock;   // no block with an empty range
    if (grid > max_useful) grid = max_useful;
    if (grid < 1) grid = 1;
    transport_persistent<GEOM, FIELD><<<(unsigned)grid, kBlock, 0, st>>>(w, s, n, rp);
    return cudaGetLastError();
}

}  // namespace mt

namespace mt {
int64_t compact_workspace_bytes(int64_t n);
cudaError_t launch_compact(const WorldParams &w, const mt_muon_soa &soa, int64_t n, const RunParams &rp,
                           cudaStream_t st, int S, int blocks_per_sm, int order, void *ws, int64_t ws_bytes,
                           bool &ws_too_small);
}  // namespace mt

using namespace mt;

extern "C" int64_t mt_transport_workspace_bytes(int64_t n) { return compact_workspace_bytes(n < 0 ? 0 : n); }

namespace mt {
// Default pass length of the compacting transport.  The muons in flight during
// a pass span about S d of z, so the field map's working set is the node
// layers of that slab; the longest S in {128, 96, 64, 48, 32, 24, 16} whose
// slab fits the L2 budget keeps the gathers L2 hits.  Without the spatial
// order the budget is three quarters of L2 (measured on shield1e8, 400 x 400
// x 1200 map, 16M muons, unordered: S = 16 4.78e10 muon-steps/s, S = 64
// 4.07e10).  With it the warps in flight hold neighbouring map columns, so at
// any moment they touch only part of the slab and the budget is 2.5 L2
// (shield1e8, ordered: S = 16 5.48e10, 32 5.67e10, 48 5.68e10, 64 5.78e10,
// 96 5.74e10, 128 5.66e10; S = 64 is a 290 MB slab).  On shield1e6 (200 x 200
// x 600) S = 128 fits either budget and is among the fastest: ordered, with
// two muon groups, 5.80e10 muon-steps/s at 128 and at 96, 5.74e10 at 64 and
// 5.76e10 at 160.  Without a map the pass length is 64.
int default_steps_per_pass(const WorldParams &w, float step_len, bool ordered)
{
    if (w.field_kind != MT_FIELD_MAP && w.field_kind != MT_FIELD_MAP_NEAREST) return 64;
    int dev = 0, l2 = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess || l2 <= 0) return 64;
    const double layer = w.field_kind == MT_FIELD_MAP ? 32.0 * (w.fdims[0] - 1) * (double)w.fdims[1]
                                                      : 16.0 * w.fdims[0] * (double)w.fdims[1];
    const double sz = (double)w.frs_h[2] + (double)w.frs_l[2];
    const double budget = (ordered ? 2.5 : 0.75) * l2;
    const int cand[7] = {128, 96, 64, 48, 32, 24, 16};
    // the map read at every RK4 stage takes at most 64 steps (measured on
    // shield1e6: 2.15e10 muon-steps/s against 2.00e10 at 128)
    const int longest = w.field_per_stage ? 64 : 128;
    for (int S : cand)
        if (S <= longest && layer * (S * (double)step_len / sz + 2.0) <= budget) return S;
    return 16;
}
}  // namespace mt

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

mt_status check_soa(const mt_muon_soa *s, int64_t n)
{
    if (!s) {
        set_error("null muon SoA");
        return MT_ERR_INVALID_ARG;
    }
    if (n < 0) {
        set_error("n = %lld < 0", (long long)n);
        return MT_ERR_INVALID_ARG;
    }
    if (n > 0 && (!s->x || !s->y || !s->z || !s->px || !s->py || !s->pz || !s->q || !s->steps || !s->status)) {
        set_error("null muon array with n > 0");
        return MT_ERR_INVALID_ARG;
    }
    if (s->id_offset < 0) {
        set_error("negative id_offset");
        return MT_ERR_INVALID_ARG;
    }
    return MT_OK;
}

}  // namespace

extern "C" mt_status mt_transport_cfg(mt_handle *h, const mt_muon_soa *s, int64_t n, float step_len,
                                      int32_t max_steps, uint64_t seed, const float *alpha, int32_t n_block,
                                      const mt_launch_cfg *cfg, void *stream)
{
    if (!h) {
        set_error("null handle");
        return MT_ERR_INVALID_ARG;
    }
    mt_status st = check_soa(s, n);
    if (st != MT_OK) return st;
    if (!(step_len > 0.0f) || !isfinite(step_len) || max_steps < 0) {
        set_error("step_len must be positive and finite, max_steps >= 0");
        return MT_ERR_INVALID_ARG;
    }
    if (alpha && (n_block < 0 || n_block > MT_MAX_BOXES)) {
        set_error("n_block %d outside [0, %d]", n_block, MT_MAX_BOXES);
        return MT_ERR_INVALID_ARG;
    }
    mt_launch_cfg lc = {MT_LAUNCH_AUTO, 0, 0, 0, nullptr, 0};
    if (cfg) lc = *cfg;
    if (lc.mode < MT_LAUNCH_AUTO || lc.mode > MT_LAUNCH_COMPACT || lc.blocks_per_sm < 0 || lc.steps_per_pass < 0 ||
        lc.order < MT_ORDER_AUTO || lc.order > MT_ORDER_NEVER) {
        set_error("bad launch configuration (mode %d, blocks_per_sm %d, steps_per_pass %d, order %d)", lc.mode,
                  lc.blocks_per_sm, lc.steps_per_pass, lc.order);
        return MT_ERR_INVALID_ARG;
    }
    if (lc.mode == MT_LAUNCH_COMPACT && n >= (int64_t)1 << 31) {
        set_error("compact mode takes n < 2^31 muons per call (got %lld)", (long long)n);
        return MT_ERR_INVALID_ARG;
    }
    if (n == 0) return MT_OK;
    RunParams rp;
    rp.d = step_len;
    rp.kd = (float)(0.299792458 * (double)step_len);
    rp.max_steps = max_steps;
    set_seed(rp, seed);
    rp.alpha = alpha;
    rp.n_block = alpha ? n_block : 0;
    rp.instance = s->instance;
    rp.id_offset = s->id_offset;
    DeviceGuard g(h->device);
    cudaStream_t cs = (cudaStream_t)stream;
    cudaError_t e;
    const WorldParams &w = h->w;
    if (lc.mode == MT_LAUNCH_COMPACT || (lc.mode == MT_LAUNCH_AUTO && n < ((int64_t)1 << 31))) {
        bool small = false;
        e = launch_compact(w, *s, n, rp, cs,
                           lc.steps_per_pass > 0 ? lc.steps_per_pass
                                              : default_steps_per_pass(w, step_len, call_ordered(w, n, lc.order)),
                           lc.blocks_per_sm, lc.order,
                           lc.workspace, lc.workspace_bytes, small);
        if (small) {
            set_error("workspace of %lld bytes at %p is too small or not 256-byte aligned (need %lld)",
                      (long long)lc.workspace_bytes, lc.workspace, (long long)compact_workspace_bytes(n));
            return MT_ERR_INVALID_ARG;
        }
        if (e != cudaSuccess) return cuda_fail(e, "compacting transport");
        return MT_OK;
    }
    if (w.geom_kind == MT_GEOM_BOXES) {
        if (w.field_kind == MT_FIELD_MAP && w.field_per_stage)
            e = launch<MT_GEOM_BOXES, kFieldMapStaged>(w, *s, n, rp, cs, lc);
        else if (w.field_kind == MT_FIELD_MAP)
            e = launch<MT_GEOM_BOXES, MT_FIELD_MAP>(w, *s, n, rp, cs, lc);
        else if (w.field_kind == MT_FIELD_MAP_NEAREST)
            e = launch<MT_GEOM_BOXES, MT_FIELD_MAP_NEAREST>(w, *s, n, rp, cs, lc);
        else if (w.field_kind == MT_FIELD_BOX)
            e = launch<MT_GEOM_BOXES, MT_FIELD_BOX>(w, *s, n, rp, cs, lc);
        else
            e = launch<MT_GEOM_BOXES, MT_FIELD_NONE>(w, *s, n, rp, cs, lc);
    } else if (w.geom_kind == MT_GEOM_POLYHEDRA) {
        if (w.field_kind == MT_FIELD_MAP && w.field_per_stage)
            e = launch<MT_GEOM_POLYHEDRA, kFieldMapStaged>(w, *s, n, rp, cs, lc);
        else if (w.field_kind == MT_FIELD_MAP)
            e = launch<MT_GEOM_POLYHEDRA, MT_FIELD_MAP>(w, *s, n, rp, cs, lc);
        else if (w.field_kind == MT_FIELD_MAP_NEAREST)
            e = launch<MT_GEOM_POLYHEDRA, MT_FIELD_MAP_NEAREST>(w, *s, n, rp, cs, lc);
        else if (w.field_kind == MT_FIELD_BOX)
            e = launch<MT_GEOM_POLYHEDRA, MT_FIELD_BOX>(w, *s, n, rp, cs, lc);
        else
            e = launch<MT_GEOM_POLYHEDRA, MT_FIELD_NONE>(w, *s, n, rp, cs, lc);
    } else {
        if (w.field_kind == MT_FIELD_MAP && w.field_per_stage)
            e = launch<MT_GEOM_VOXELS, kFieldMapStaged>(w, *s, n, rp, cs, lc);
        else if (w.field_kind == MT_FIELD_MAP)
            e = launch<MT_GEOM_VOXELS, MT_FIELD_MAP>(w, *s, n, rp, cs, lc);
        else if (w.field_kind == MT_FIELD_MAP_NEAREST)
            e = launch<MT_GEOM_VOXELS, MT_FIELD_MAP_NEAREST>(w, *s, n, rp, cs, lc);
        else
            e = launch<MT_GEOM_VOXELS, MT_FIELD_NONE>(w, *s, n, rp, cs, lc);
    }
    if (e != cudaSuccess) return cuda_fail(e, "transport launch");
    return MT_OK;
}

extern "C" int64_t mt_transport_launches(const mt_handle *h, int64_t n, float step_len, int32_t max_steps,
                                         const mt_launch_cfg *cfg)
{
    if (!h || n < 0 || !(step_len > 0.0f) || !isfinite(step_len) || max_steps < 0) return -1;
    mt_launch_cfg lc = {MT_LAUNCH_AUTO, 0, 0, 0, nullptr, 0};
    if (cfg) lc = *cfg;
    if (lc.mode < MT_LAUNCH_AUTO || lc.mode > MT_LAUNCH_COMPACT || lc.steps_per_pass < 0 ||
        lc.order < MT_ORDER_AUTO || lc.order > MT_ORDER_NEVER)
        return -1;
    if (n == 0) return 0;
    if (lc.mode == MT_LAUNCH_COMPACT || (lc.mode == MT_LAUNCH_AUTO && n < ((int64_t)1 << 31))) {
        DeviceGuard g(h->device);
        const int S = lc.steps_per_pass > 0 ? lc.steps_per_pass
                                           : default_steps_per_pass(h->w, step_len, call_ordered(h->w, n, lc.order));
        return compact_call_launches(h->w, n, max_steps, S, lc.order);
    }
    return 1;
}

extern "C" mt_status mt_transport_scaled(mt_handle *h, const mt_muon_soa *s, int64_t n, float step_len,
                                         int32_t max_steps, uint64_t seed, const float *alpha, int32_t n_block,
                                         void *stream)
{
    return mt_transport_cfg(h, s, n, step_len, max_steps, seed, alpha, n_block, nullptr, stream);
}

extern "C" mt_status mt_transport(mt_handle *h, const mt_muon_soa *s, int64_t n, float step_len, int32_t max_steps,
                                  uint64_t seed, void *stream)
{
    return mt_transport_cfg(h, s, n, step_len, max_steps, seed, nullptr, 0, nullptr, stream);
}
