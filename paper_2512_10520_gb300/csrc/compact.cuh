// compact.cuh -- kernels of the lockstep compacting transport, shared by the
// plain transport (compact.cu) and the checkpointing forward of the adjoint
// (adjoint.cu).
#pragma once

#include "step.cuh"

// Resident blocks per SM the compiler must allow for (register budget of the
// pass kernels): 5 blocks of 256 threads = 48 registers per thread (measured
// fastest on shield1e6: 40 registers spill and run 5 % slower).
#ifndef MT_PASS_MIN_BLOCKS
#define MT_PASS_MIN_BLOCKS 5
#endif
// The same for the polyhedron geometry, whose containment test needs more
// registers (measured on tapered1e6: 4 blocks = 64 registers, 33.2 ms; 5 blocks
// spill, 36.8 ms).
#ifndef MT_PASS_MIN_BLOCKS_POLY
#define MT_PASS_MIN_BLOCKS_POLY 4
#endif

namespace mt {
// Per-stage field reads (three more map lookups live in the RK4 step) take
// the polyhedron budget as well.
template <int GEOM, int FIELD>
constexpr int pass_min_blocks()
{
    return (GEOM == MT_GEOM_POLYHEDRA || FIELD == kFieldMapStaged) ? MT_PASS_MIN_BLOCKS_POLY : MT_PASS_MIN_BLOCKS;
}
}  // namespace mt

namespace mt {

// Spatial order of the live list.  The survivors of a pass are reordered by
// the cell of a coarse xy grid over the field map (2 x 2 map cells or more)
// that they stand in, so the 32 muons of a warp share their field-map corners
// and each trilinear gather touches a few lines instead of 32 scattered ones.
// It is a counting sort in three steps: as a pass appends a survivor it also
// takes the next rank of its key from a histogram; an exclusive scan of the
// histogram gives each key's first slot; a scatter moves every entry to its
// key's first slot plus its rank.  A muon's result does not depend on its
// place in the list, so the order changes the speed only.
//
// Measured (GB300, muon-steps/s; 64-step passes, the order after every pass /
// every second pass): shield1e6 1e6 muons +2.2 % / +2.8 %, tapered1e6 +9.2 % /
// +7.9 %, 262144 muons -1.2 % / +0.2 %, 65536 muons -14 % / -10 % (the scan and
// the scatter cost about 40 us per reorder whatever the size).  With two muon
// groups and 128-step passes, a reorder after every pass is the faster on
// shield1e6 (5.80 against 5.72e10; every third pass 5.67e10).  So the list
// is reordered about every MT_SORT_STEPS steps (after every pass of 64 steps
// or more, every second of 32, every fourth of 16), in calls of at least
// 2^19 muons.
#ifndef MT_SORT_STEPS
#define MT_SORT_STEPS 64
#endif
#ifndef MT_SORT_MIN_MUONS
#define MT_SORT_MIN_MUONS (1 << 19)
#endif

// Passes between reorders for passes of S steps.
__host__ __device__ constexpr int sort_every(int S) { return S >= MT_SORT_STEPS ? 1 : (MT_SORT_STEPS + S - 1) / S; }

__device__ __forceinline__ uint32_t sort_key(const WorldParams &w, float uh, float vh)
{
    const int i = min(max(__float2int_rd(uh), 0), w.fdims[0] - 2) >> w.sort_shift;
    const int j = min(max(__float2int_rd(vh), 0), w.fdims[1] - 2) >> w.sort_shift;
    return (uint32_t)(j * w.sort_nx + i);
}

// Rank of this lane's entry among the entries of its key (valid where keep):
// hist[key] is advanced by one atomic per distinct key of the warp.
__device__ __forceinline__ unsigned sort_rank(unsigned *hist, bool keep, uint32_t key)
{
    const unsigned m = __ballot_sync(0xFFFFFFFFu, keep);
    unsigned r = 0u;
    if (keep) {
        const unsigned lane = threadIdx.x & 31u;
        const unsigned peers = __match_any_sync(m, key);
        const int leader = __ffs(peers) - 1;
        if ((int)lane == leader) r = atomicAdd(hist + key, (unsigned)__popc(peers));
        r = __shfl_sync(peers, r, leader) + __popc(peers & ((1u << lane) - 1u));
    }
    return r;
}

// One block of 1024 threads, bins <= kSortBins: offs = exclusive prefix sum of
// hist[0 .. bins), and hist cleared for the next count (v: 1024 * kScanStride
// words of shared memory, wsum: 32).  The counts are staged
// in shared memory (one coalesced sweep), each thread scans kSortBins / 1024
// consecutive bins, and a block scan of the threads' totals joins them.
constexpr int kScanPer = kSortBins / 1024;
constexpr int kScanStride = kScanPer + 1;   // padded rows: no bank conflicts
constexpr int kScanSmem = 1024 * kScanStride * (int)sizeof(unsigned);   // dynamic shared memory of sort_scan
__device__ __forceinline__ void scan_counts(unsigned *hist, unsigned *offs, int bins, unsigned *v, unsigned *wsum)
{
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
#pragma unroll
    for (int r = 0; r < kScanPer; ++r) {
        const int b = r * 1024 + t;
        v[(b / kScanPer) * kScanStride + b % kScanPer] = b < bins ? hist[b] : 0u;
    }
    __syncthreads();
    unsigned tot = 0u;
#pragma unroll
    for (int r = 0; r < kScanPer; ++r) {
        const unsigned c = v[t * kScanStride + r];
        v[t * kScanStride + r] = tot;
        tot += c;
    }
    unsigned x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const unsigned s = wsum[lane];
        unsigned z = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xFFFFFFFFu, z, o);
            if (lane >= o) z += y;
        }
        wsum[lane] = z - s;
    }
    __syncthreads();
    const unsigned base = wsum[wid] + x - tot;
#pragma unroll
    for (int r = 0; r < kScanPer; ++r) v[t * kScanStride + r] += base;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kScanPer; ++r) {
        const int b = r * 1024 + t;
        if (b < bins) {
            offs[b] = v[(b / kScanPer) * kScanStride + b % kScanPer];
            hist[b] = 0u;
        }
    }
}

static __global__ void __launch_bounds__(1024) sort_scan(unsigned *hist, unsigned *offs, int bins)
{
    extern __shared__ unsigned v[];   // [1024][kScanStride]
    __shared__ unsigned wsum[32];
    scan_counts(hist, offs, bins, v, wsum);
}

// Move the *cnt entries of src to dst in key order: an entry goes to its key's
// first slot (offs, from sort_scan) plus its rank (the fourth word of w3).
// The ranks of a key are 0 .. count - 1 by construction, so every slot is below
// *cnt; the test on it only keeps a broken count from writing past the list.
static __global__ void __launch_bounds__(kBlock) sort_scatter(const WorldParams w, LiveBuf src, LiveBuf dst,
                                                              const unsigned long long *cnt, const unsigned *offs)
{
    const int64_t count = (int64_t)*cnt;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const float4 a = src.w0[i], b = src.w1[i], c = src.w2[i], d = src.w3[i];
        const int64_t pos = (int64_t)__ldg(offs + sort_key(w, a.x, a.y)) + __float_as_uint(d.w);
        if (pos < count) {
            dst.w0[pos] = a;
            dst.w1[pos] = b;
            dst.w2[pos] = c;
            dst.w3[pos] = d;
        }
    }
}

// Pack the live muons (status ALIVE or MAX_STEPS, finite state) of the
// caller's arrays into a live list, positions in the world's frame; non-finite
// states are marked MT_INVALID.
static __global__ void __launch_bounds__(kBlock) compact_init(const WorldParams w, const mt_muon_soa soa, int64_t n,
                                                              const RunParams rp, LiveBuf out, unsigned long long *ctr,
                                                              unsigned *hist)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t m = base + threadIdx.x;
        State s;
        float q = 0.0f;
        int k = 0;
        uint32_t id_lo, id_hi;
        const bool live = m < n && load_muon(w, soa, m, rp, s, q, k, id_lo, id_hi);
        const int64_t slot = warp_append(&ctr[0], live);
        const unsigned rank = hist ? sort_rank(hist, live, live ? sort_key(w, s.x, s.y) : 0u) : 0u;
        if (live) put_live(out, slot, s, q, k, m, rank);
    }
}

// One pass: live count from *cin, survivors appended at *cout; *czero (if not
// null) is cleared for the pass after this one.  Warps take the live list in
// chunks of 32 entries from the counter *work (zero at the start of the pass),
// so a warp whose muons stop early takes more chunks and the SMs finish the
// pass together; *wzero (if not null) is cleared for a later pass.  hist (if
// not null): each survivor takes its rank in the spatial order from it.
template <int GEOM, int FIELD>
__global__ void __launch_bounds__(kBlock, pass_min_blocks<GEOM, FIELD>()) compact_pass(const WorldParams w, const mt_muon_soa soa, const RunParams rp,
                                                       LiveBuf in, LiveBuf out, const unsigned long long *cin,
                                                       unsigned long long *cout, unsigned long long *czero,
                                                       unsigned long long *work, unsigned long long *wzero, int S,
                                                       unsigned *hist)
{
    __shared__ SmemWorld sw;
    const int64_t count = (int64_t)*cin;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (czero) *czero = 0ull;
        if (wzero) *wzero = 0ull;
    }
    if (count == 0) return;
    stage_world(sw, w, rp);
    __syncthreads();
    const unsigned lane = threadIdx.x & 31u;
    for (;;) {
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(work, 32ull);
        const int64_t base = (int64_t)__shfl_sync(0xFFFFFFFFu, b, 0);
        if (base >= count) break;
        const int64_t i = base + lane;
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
                r = step<GEOM, FIELD>(w, sw, s, q, k, id_lo, id_hi, (uint32_t)rp.instance, rp);
                if (r != MT_ALIVE) break;
            }
            if (r == MT_ALIVE && k >= rp.max_steps) r = MT_MAX_STEPS;
            if (r != MT_ALIVE)
                store_muon(w, soa, idx, s, k, r);
            else
                keep = true;
        }
        const int64_t slot = warp_append(cout, keep);
        const unsigned rank = hist ? sort_rank(hist, keep, keep ? sort_key(w, s.x, s.y) : 0u) : 0u;
        if (keep) put_live(out, slot, s, q, k, idx, rank);
    }
}

}  // namespace mt
