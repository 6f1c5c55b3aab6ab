// compact.cu -- lockstep transport with periodic compaction of live muons.
//
// Every live muon advances S steps per pass; survivors are appended to the
// other half of a double-buffered live list, finished muons are written back
// to the caller's arrays.  All muons in flight during a pass are within S
// steps of each other, so they sit in the same few-metre slab of the field map
// (which stays in L2), and warps never carry lanes whose muon has stopped for
// more than S steps.
//
// Live-list entries (64 B per muon) are described in step.cuh.  Counters:
// six 64-bit words; pass p reads its live count from ctr[p % 3], appends to
// ctr[(p+1) % 3] and clears ctr[(p+2) % 3] for the pass after it; it takes its
// work from ctr[3 + p % 3] and clears ctr[3 + (p+1) % 3], last used two passes
// before.
#include <cstdio>

#include "compact.cuh"

namespace mt {

// Muon groups of one call.  A call of at least MT_GROUP_MIN_MUONS muons runs as
// two independent halves, each a compacting transport of its own (lists,
// counters, order) on a stream of its own, so that one half's passes fill the
// SMs that the other half's pass tail leaves idle: near the end of a pass the
// last chunks' warps run alone.  The halves wait on nothing of each other.
// Measured on shield1e6 (10^6 muons, spatial order on): one group 20.16 ms
// per call, two 19.00, three 19.22, four 19.51.
#ifndef MT_GROUP_MIN_MUONS
#define MT_GROUP_MIN_MUONS (1 << 19)
#endif

static int compact_groups(int64_t n, int64_t ng[2])
{
    if (n >= MT_GROUP_MIN_MUONS) {
        ng[0] = n / 2;
        ng[1] = n - n / 2;
        return 2;
    }
    ng[0] = n;
    ng[1] = 0;
    return 1;
}

// One group's workspace: counters (256 B), the two live lists, then the
// spatial order's histogram and offsets (kSortBins each); a multiple of 256.
static int64_t group_workspace_bytes(int64_t n)
{
    const int64_t cap = n > 0 ? n : 1;
    const int64_t b = 256 + 2 * 4 * cap * (int64_t)sizeof(float4) + 2 * (int64_t)kSortBins * (int64_t)sizeof(unsigned);
    return (b + 255) & ~(int64_t)255;
}

int64_t compact_workspace_bytes(int64_t n)
{
    int64_t ng[2];
    const int G = compact_groups(n, ng);
    int64_t b = 0;
    for (int g = 0; g < G; ++g) b += group_workspace_bytes(ng[g]);
    return b;
}

// The call's order mode for its groups: MT_ORDER_ALWAYS or MT_ORDER_NEVER,
// decided on the call's muon count (auto: 2^19 or more, maps only).
static int resolve_order(const WorldParams &w, int64_t n, int order_mode)
{
    if (w.sort_bins <= 0 || order_mode == MT_ORDER_NEVER) return MT_ORDER_NEVER;
    if (order_mode == MT_ORDER_ALWAYS || n >= MT_SORT_MIN_MUONS) return MT_ORDER_ALWAYS;
    return MT_ORDER_NEVER;
}

bool call_ordered(const WorldParams &w, int64_t n, int order_mode)
{
    return resolve_order(w, n, order_mode) == MT_ORDER_ALWAYS;
}

// Launch plan of one compacting call: its passes, and whether the live list is
// reordered (after compact_init and after the passes reorder_after names).
CompactPlan compact_plan(const WorldParams &w, int64_t n, int max_steps, int S, int order_mode)
{
    CompactPlan pl;
    // a muon that starts at step 0 needs ceil(max_steps / S) passes
    pl.passes = max_steps > 0 ? (max_steps + S - 1) / S : 1;
    pl.order = w.sort_bins > 0 && order_mode != MT_ORDER_NEVER &&
               (order_mode == MT_ORDER_ALWAYS || n >= MT_SORT_MIN_MUONS);
    pl.every = sort_every(S);
    return pl;
}

static bool reorder_after(const CompactPlan &pl, int p)
{
    return pl.order && p + 1 < pl.passes && (p + 1) % pl.every == 0;
}

static int64_t compact_launches(const CompactPlan &pl)
{
    int64_t c = 1 + pl.passes;
    if (pl.order) c += 2;
    for (int p = 0; p < pl.passes; ++p)
        if (reorder_after(pl, p)) c += 2;
    return c;
}

int64_t compact_call_launches(const WorldParams &w, int64_t n, int max_steps, int S, int order_mode)
{
    int64_t ng[2];
    const int G = compact_groups(n, ng);
    const int om = resolve_order(w, n, order_mode);
    int64_t c = 0;
    for (int g = 0; g < G; ++g)
        if (ng[g] > 0) c += compact_launches(compact_plan(w, ng[g], max_steps, S, om));
    return c;
}

template <int GEOM, int FIELD>
static cudaError_t run_passes(const WorldParams &w, const mt_muon_soa &soa, int64_t n, const RunParams &rp,
                              cudaStream_t st, int S, int blocks_per_sm, int order_mode, char *ws)
{
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(ws);
    LiveBuf buf[2] = {live_buf_at(ws + 256, n), live_buf_at(ws + 256 + 4 * n * (int64_t)sizeof(float4), n)};
    unsigned *hist = reinterpret_cast<unsigned *>(ws + 256 + 2 * 4 * n * (int64_t)sizeof(float4));
    unsigned *offs = hist + kSortBins;
    cudaError_t e = cudaMemsetAsync(ctr, 0, 6 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    // Spatial order (maps only): the list is reordered after compact_init and
    // after every sort_every(S)-th pass but the last.
    const CompactPlan plan = compact_plan(w, n, rp.max_steps, S, order_mode);
    const int passes = plan.passes;
    const bool order = plan.order;
    if (order) {
        e = cudaFuncSetAttribute(sort_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, kScanSmem);
        if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, (size_t)w.sort_bins * sizeof(unsigned), st);
        if (e != cudaSuccess) return e;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, compact_pass<GEOM, FIELD>, kBlock, 0);
    if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sms * per_sm;
    const int64_t need = (n + kBlock - 1) / kBlock;
    if (grid > need) grid = need;
    const int64_t init_grid = need < 65535 * 8 ? need : 65535 * 8;
    const int64_t scatter_grid = grid < (int64_t)sms * 8 ? (int64_t)sms * 8 : grid;
    // scan the counts of the list just written to buf[src] and scatter it to the other list
    auto reorder = [&](int src, const unsigned long long *cnt) {
        sort_scan<<<1, 1024, kScanSmem, st>>>(hist, offs, w.sort_bins);
        cudaError_t f = cudaGetLastError();
        if (f != cudaSuccess) return f;
        sort_scatter<<<(unsigned)scatter_grid, kBlock, 0, st>>>(w, buf[src], buf[src ^ 1], cnt, offs);
        return cudaGetLastError();
    };
    // the current list is buf[cur]; a pass appends to the other one, which
    // becomes current unless it is reordered back into buf[cur]
    int cur = 0;
    compact_init<<<(unsigned)init_grid, kBlock, 0, st>>>(w, soa, n, rp, buf[order ? 1 : 0], ctr, order ? hist : nullptr);
    e = cudaGetLastError();
    if (e == cudaSuccess && order) e = reorder(1, ctr);
    if (e != cudaSuccess) return e;
    for (int p = 0; p < passes; ++p) {
        const bool count = reorder_after(plan, p);
        compact_pass<GEOM, FIELD><<<(unsigned)grid, kBlock, 0, st>>>(w, soa, rp, buf[cur], buf[cur ^ 1], ctr + p % 3,
                                                                     ctr + (p + 1) % 3, ctr + (p + 2) % 3,
                                                                     ctr + 3 + p % 3, ctr + 3 + (p + 1) % 3, S,
                                                                     count ? hist : nullptr);
        e = cudaGetLastError();
        if (e == cudaSuccess && count) e = reorder(cur ^ 1, ctr + (p + 1) % 3);
        if (e != cudaSuccess) return e;
        if (!count) cur ^= 1;
    }
    return cudaSuccess;
}

// One group's passes, dispatched on the world's geometry and field kinds.
static cudaError_t dispatch_passes(const WorldParams &w, const mt_muon_soa &soa, int64_t n, const RunParams &rp,
                                   cudaStream_t st, int S, int blocks_per_sm, int order, char *buf)
{
    cudaError_t e;
    if (w.geom_kind == MT_GEOM_BOXES) {
        if (w.field_kind == MT_FIELD_MAP && w.field_per_stage)
            e = run_passes<MT_GEOM_BOXES, kFieldMapStaged>(w, soa, n, rp, st, S, blocks_per_sm, order, buf);
        else if (w.field_kind == MT_FIELD_MAP)
            e = run_passes<MT_GEOM_BOXES, MT_FIELD_MAP>(w, soa, n, rp, st, S, blocks_per_sm, order, buf);
        else if (w.field_kind == MT_FIELD_MAP_NEAREST)
            e = run_passes<MT_GEOM_BOXES, MT_FIELD_MAP_NEAREST>(w, soa, n, rp, st, S, blocks_per_sm, order, buf);
        else if (w.field_kind == MT_FIELD_BOX)
            e = run_passes<MT_GEOM_BOXES, MT_FIELD_BOX>(w, soa, n, rp, st, S, blocks_per_sm, order, buf);
        else
            e = run_passes<MT_GEOM_BOXES, MT_FIELD_NONE>(w, soa, n, rp, st, S, blocks_per_sm, order, buf);
    } else if (w.geom_kind == MT_GEOM_POLYHEDRA) {
        if (w.field_kind == MT_FIELD_MAP && w.field_per_stage)
            e = run_passes<MT_GEOM_POLYHEDRA, kFieldMapStaged>(w, soa, n, rp, st, S, blocks_per_sm, order, buf);
        else if (w.field_kind == MT_FIELD_MAP)
            e = run_passes<MT_GEOM_POLYHEDRA, MT_FIELD_MAP>(w, soa, n, rp, st, S, blocks_per_sm, order, buf);
        else if (w.field_kind == MT_FIELD_MAP_NEAREST)
            e = run_passes<MT_GEOM_POLYHEDRA, MT_FIELD_MAP_NEAREST>(w, soa, n, rp, st, S, blocks_per_sm, order, buf);
        else if (w.field_kind == MT_FIELD_BOX)
            e = run_passes<MT_GEOM_POLYHEDRA, MT_FIELD_BOX>(w, soa, n, rp, st, S, blocks_per_sm, order, buf);
        else
            e = run_passes<MT_GEOM_POLYHEDRA, MT_FIELD_NONE>(w, soa, n, rp, st, S, blocks_per_sm, order, buf);
    } else {
        if (w.field_kind == MT_FIELD_MAP && w.field_per_stage)
            e = run_passes<MT_GEOM_VOXELS, kFieldMapStaged>(w, soa, n, rp, st, S, blocks_per_sm, order, buf);
        else if (w.field_kind == MT_FIELD_MAP)
            e = run_passes<MT_GEOM_VOXELS, MT_FIELD_MAP>(w, soa, n, rp, st, S, blocks_per_sm, order, buf);
        else if (w.field_kind == MT_FIELD_MAP_NEAREST)
            e = run_passes<MT_GEOM_VOXELS, MT_FIELD_MAP_NEAREST>(w, soa, n, rp, st, S, blocks_per_sm, order, buf);
        else
            e = run_passes<MT_GEOM_VOXELS, MT_FIELD_NONE>(w, soa, n, rp, st, S, blocks_per_sm, order, buf);
    }
    return e;
}

// The muons [off, off + m) of soa as a SoA of their own (ids follow from rp).
static mt_muon_soa soa_part(const mt_muon_soa &s, int64_t off)
{
    mt_muon_soa p = s;
    p.x = s.x + off;
    p.y = s.y + off;
    p.z = s.z + off;
    p.px = s.px + off;
    p.py = s.py + off;
    p.pz = s.pz + off;
    p.q = s.q + off;
    p.steps = s.steps + off;
    p.status = s.status + off;
    return p;
}

// Host entry used by mt_transport_cfg (MT_LAUNCH_COMPACT).  ws may be null:
// then the scratch comes from the stream-ordered allocator and is returned on
// the same stream.  A call of two groups runs the second on a stream it
// creates, forked from st and joined back into it with events.
cudaError_t launch_compact(const WorldParams &w, const mt_muon_soa &soa, int64_t n, const RunParams &rp,
                           cudaStream_t st, int S, int blocks_per_sm, int order, void *ws, int64_t ws_bytes,
                           bool &ws_too_small)
{
    ws_too_small = false;
    const int64_t need = compact_workspace_bytes(n);
    char *buf = reinterpret_cast<char *>(ws);
    bool own = false;
    if (buf) {
        if (ws_bytes < need || (reinterpret_cast<uintptr_t>(buf) & 255u)) {
            ws_too_small = true;
            return cudaSuccess;
        }
    } else {
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&buf), (size_t)need, st);
        if (e != cudaSuccess) return e;
        own = true;
    }
    int64_t ng[2];
    const int G = compact_groups(n, ng);
    const int om = resolve_order(w, n, order);
    cudaError_t e = cudaSuccess;
    if (G == 1) {
        e = dispatch_passes(w, soa, n, rp, st, S, blocks_per_sm, om, buf);
    } else {
        cudaStream_t aux = nullptr;
        cudaEvent_t fork = nullptr, join = nullptr;
        e = cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, fork, 0);
        if (e == cudaSuccess) e = dispatch_passes(w, soa, ng[0], rp, st, S, blocks_per_sm, om, buf);
        if (e == cudaSuccess) {
            RunParams r1 = rp;
            r1.id_offset += ng[0];
            e = dispatch_passes(w, soa_part(soa, ng[0]), ng[1], r1, aux, S, blocks_per_sm, om,
                                buf + group_workspace_bytes(ng[0]));
        }
        // join whatever the second stream was given, also after an error, so
        // that nothing on it outlives the scratch freed on st
        if (aux && join) {
            cudaError_t f = cudaEventRecord(join, aux);
            if (f == cudaSuccess) f = cudaStreamWaitEvent(st, join, 0);
            if (f != cudaSuccess) {
                cudaStreamSynchronize(aux);
                if (e == cudaSuccess) e = f;
            }
        }
        // released once their work is done
        if (join) cudaEventDestroy(join);
        if (fork) cudaEventDestroy(fork);
        if (aux) cudaStreamDestroy(aux);
    }
    if (own) {
        cudaError_t f = cudaFreeAsync(buf, st);
        if (e == cudaSuccess) e = f;
    }
    return e;
}

// Load compact_init and the pass kernel of this world's geometry and field
// kind onto the current device.  Kernels are loaded lazily on their first
// launch, and loading takes device memory; mt_create calls this so that
// mt_transport_noalloc allocates nothing, also on its first call.
template <int GEOM, int FIELD>
static cudaError_t preload_passes()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, compact_init);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, compact_pass<GEOM, FIELD>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, sort_scan);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, sort_scatter);
    return e;
}

cudaError_t compact_preload(const WorldParams &w)
{
    const bool staged = w.field_kind == MT_FIELD_MAP && w.field_per_stage;
    if (w.geom_kind == MT_GEOM_BOXES) {
        if (staged) return preload_passes<MT_GEOM_BOXES, kFieldMapStaged>();
        if (w.field_kind == MT_FIELD_MAP) return preload_passes<MT_GEOM_BOXES, MT_FIELD_MAP>();
        if (w.field_kind == MT_FIELD_MAP_NEAREST) return preload_passes<MT_GEOM_BOXES, MT_FIELD_MAP_NEAREST>();
        if (w.field_kind == MT_FIELD_BOX) return preload_passes<MT_GEOM_BOXES, MT_FIELD_BOX>();
        return preload_passes<MT_GEOM_BOXES, MT_FIELD_NONE>();
    }
    if (w.geom_kind == MT_GEOM_POLYHEDRA) {
        if (staged) return preload_passes<MT_GEOM_POLYHEDRA, kFieldMapStaged>();
        if (w.field_kind == MT_FIELD_MAP) return preload_passes<MT_GEOM_POLYHEDRA, MT_FIELD_MAP>();
        if (w.field_kind == MT_FIELD_MAP_NEAREST) return preload_passes<MT_GEOM_POLYHEDRA, MT_FIELD_MAP_NEAREST>();
        if (w.field_kind == MT_FIELD_BOX) return preload_passes<MT_GEOM_POLYHEDRA, MT_FIELD_BOX>();
        return preload_passes<MT_GEOM_POLYHEDRA, MT_FIELD_NONE>();
    }
    if (staged) return preload_passes<MT_GEOM_VOXELS, kFieldMapStaged>();
    if (w.field_kind == MT_FIELD_MAP) return preload_passes<MT_GEOM_VOXELS, MT_FIELD_MAP>();
    if (w.field_kind == MT_FIELD_MAP_NEAREST) return preload_passes<MT_GEOM_VOXELS, MT_FIELD_MAP_NEAREST>();
    return preload_passes<MT_GEOM_VOXELS, MT_FIELD_NONE>();
}

}  // namespace mt
