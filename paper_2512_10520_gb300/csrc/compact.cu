// compact.cu -- lockstep transport with periodic compaction of live muons.
//
// Every live muon advances S steps per pass; survivors are appended to the
// other half of a double-buffered live list, finished muons are written back
// to the caller's arrays.  All muons in flight during a pass are within S
// steps of each other, so they sit in the same few-metre slab of the field map
// (which stays in L2), and warps never carry lanes whose muon has stopped for
// more than S steps.
//
// Live-list entry (64 B, four 16-byte words, structure of arrays):
//   w0 = (x, y, z, q)      w1 = (px, py, pz, k as bits)
//   w2 = (xl, yl, zl, idx) w3 = (pxl, pyl, pzl, 0)
// where (x..pz) + (xl..pzl) is the compensated state, k the next step, idx the
// muon's index in the caller's arrays.  Counters: three 64-bit words; pass p
// reads its live count from ctr[p % 3], appends to ctr[(p+1) % 3] and clears
// ctr[(p+2) % 3] for the pass after it.
#include <cstdio>

#include "step.cuh"

namespace mt {

struct LiveBuf {
    float4 *w0, *w1, *w2, *w3;
};

__host__ __device__ inline LiveBuf live_buf_at(void *base, int64_t cap)
{
    float4 *p = reinterpret_cast<float4 *>(base);
    return LiveBuf{p, p + cap, p + 2 * cap, p + 3 * cap};
}

// Warp-aggregated append: returns this lane's slot (valid when keep).
__device__ __forceinline__ int64_t warp_append(unsigned long long *ctr, bool keep)
{
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, keep);
    if (!mask) return -1;
    const unsigned lane = threadIdx.x & 31u;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if ((int)lane == leader) base = atomicAdd(ctr, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    return (int64_t)base + __popc(mask & ((1u << lane) - 1u));
}

__device__ __forceinline__ void put_live(const LiveBuf &b, int64_t i, const State &s, float q, int k, int64_t idx)
{
    b.w0[i] = make_float4(s.x, s.y, s.z, q);
    b.w1[i] = make_float4(s.px, s.py, s.pz, __int_as_float(k));
    b.w2[i] = make_float4(s.xl, s.yl, s.zl, __int_as_float((int)idx));
    b.w3[i] = make_float4(s.pxl, s.pyl, s.pzl, 0.0f);
}

__device__ __forceinline__ void get_live(const LiveBuf &b, int64_t i, State &s, float &q, int &k, int64_t &idx)
{
    const float4 a = b.w0[i], c = b.w1[i], e = b.w2[i], g = b.w3[i];
    s.x = a.x; s.y = a.y; s.z = a.z; q = a.w;
    s.px = c.x; s.py = c.y; s.pz = c.z; k = __float_as_int(c.w);
    s.xl = e.x; s.yl = e.y; s.zl = e.z; idx = __float_as_int(e.w);
    s.pxl = g.x; s.pyl = g.y; s.pzl = g.z;
}

__global__ void __launch_bounds__(kBlock) compact_init(const mt_muon_soa soa, int64_t n, const RunParams rp,
                                                       LiveBuf out, unsigned long long *ctr)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t m = base + threadIdx.x;
        State s;
        float q = 0.0f;
        int k = 0;
        uint32_t id_lo, id_hi;
        const bool live = m < n && load_muon(soa, m, rp, s, q, k, id_lo, id_hi);
        const int64_t slot = warp_append(&ctr[0], live);
        if (live) put_live(out, slot, s, q, k, m);
    }
}

template <int GEOM, int FIELD>
__global__ void __launch_bounds__(kBlock) compact_pass(const WorldParams w, const mt_muon_soa soa, const RunParams rp,
                                                       LiveBuf in, LiveBuf out, unsigned long long *ctr, int pass,
                                                       int S)
{
    __shared__ SmemWorld sw;
    const int64_t count = (int64_t)ctr[pass % 3];
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr[(pass + 2) % 3] = 0ull;
    if (count == 0) return;
    stage_world(sw, w, rp);
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < count; base += stride) {
        const int64_t i = base + threadIdx.x;
        bool keep = false;
        State s;
        float q = 0.0f;
        int k = 0;
        int64_t idx = 0;
        if (i < count) {
            get_live(in, i, s, q, k, idx);
            const uint64_t id = (uint64_t)(rp.id_offset + idx);
            const uint32_t id_lo = (uint32_t)id, id_hi = (uint32_t)(id >> 32);
            const int kend = min(k + S, rp.max_steps);
            int r = MT_ALIVE;
#pragma unroll 1
            for (; k < kend; ++k) {
                r = step<GEOM, FIELD>(w, sw, s, q, k, id_lo, id_hi, rp);
                if (r != MT_ALIVE) break;
            }
            if (r == MT_ALIVE && k >= rp.max_steps) r = MT_MAX_STEPS;
            if (r != MT_ALIVE)
                store_muon(soa, idx, s, k, r);
            else
                keep = true;
        }
        const int64_t slot = warp_append(&ctr[(pass + 1) % 3], keep);
        if (keep) put_live(out, slot, s, q, k, idx);
    }
}

int64_t compact_workspace_bytes(int64_t n)
{
    const int64_t cap = n > 0 ? n : 1;
    return 256 + 2 * 4 * cap * (int64_t)sizeof(float4);
}

template <int GEOM, int FIELD>
static cudaError_t run_passes(const WorldParams &w, const mt_muon_soa &soa, int64_t n, const RunParams &rp,
                              cudaStream_t st, int S, int blocks_per_sm, char *ws)
{
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(ws);
    LiveBuf buf[2] = {live_buf_at(ws + 256, n), live_buf_at(ws + 256 + 4 * n * (int64_t)sizeof(float4), n)};
    cudaError_t e = cudaMemsetAsync(ctr, 0, 3 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
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
    compact_init<<<(unsigned)init_grid, kBlock, 0, st>>>(soa, n, rp, buf[0], ctr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // a muon that starts at step 0 needs ceil(max_steps / S) passes
    const int passes = rp.max_steps > 0 ? (rp.max_steps + S - 1) / S : 1;
    for (int p = 0; p < passes; ++p) {
        compact_pass<GEOM, FIELD><<<(unsigned)grid, kBlock, 0, st>>>(w, soa, rp, buf[p & 1], buf[(p + 1) & 1], ctr,
                                                                     p, S);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Host entry used by mt_transport_cfg (MT_LAUNCH_COMPACT).  ws may be null:
// then the scratch comes from the stream-ordered allocator and is returned on
// the same stream.
cudaError_t launch_compact(const WorldParams &w, const mt_muon_soa &soa, int64_t n, const RunParams &rp,
                           cudaStream_t st, int S, int blocks_per_sm, void *ws, int64_t ws_bytes, bool &ws_too_small)
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
    cudaError_t e;
    if (w.geom_kind == MT_GEOM_BOXES) {
        if (w.field_kind == MT_FIELD_MAP)
            e = run_passes<MT_GEOM_BOXES, MT_FIELD_MAP>(w, soa, n, rp, st, S, blocks_per_sm, buf);
        else if (w.field_kind == MT_FIELD_BOX)
            e = run_passes<MT_GEOM_BOXES, MT_FIELD_BOX>(w, soa, n, rp, st, S, blocks_per_sm, buf);
        else
            e = run_passes<MT_GEOM_BOXES, MT_FIELD_NONE>(w, soa, n, rp, st, S, blocks_per_sm, buf);
    } else {
        if (w.field_kind == MT_FIELD_MAP)
            e = run_passes<MT_GEOM_VOXELS, MT_FIELD_MAP>(w, soa, n, rp, st, S, blocks_per_sm, buf);
        else
            e = run_passes<MT_GEOM_VOXELS, MT_FIELD_NONE>(w, soa, n, rp, st, S, blocks_per_sm, buf);
    }
    if (own) {
        cudaError_t f = cudaFreeAsync(buf, st);
        if (e == cudaSuccess) e = f;
    }
    return e;
}

}  // namespace mt
