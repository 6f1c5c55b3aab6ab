// batched.cu -- many independent worlds (geometry + field map) sharing one
// histogram set, transported together: lockstep passes over every live muon of
// every instance, fed to a resident grid by a device work queue of
// (instance, chunk) items, with per-instance compaction between passes.
//
// Live list: the live muons of instance i occupy region [off_i, off_i + n_i) of
// each of the two live buffers (entries as in step.cuh).  Per pass p:
//   plan  : one block turns the live count of every instance into work items of
//           up to BLOCK muons, an exclusive scan cof (cof[n_inst] = items), and
//           clears the queue and the counters of the pass after next;
//   pass  : each block pops items from the queue; all of its lanes take the
//           same instance, whose world it stages in shared memory once per
//           instance change; each lane advances its muon S steps, finished
//           muons go back to the instance's arrays, survivors are appended to
//           the instance's region of the other buffer.
// All loops are bounded: the queue is finite and each muon runs at most
// max_steps steps.
#include <algorithm>
#include <cstring>
#include <vector>

#include "compact.cuh"

// Resident threads per SM the compiler must allow for in batch_pass (register
// budget).  Voxel worlds: 1280 threads = 48 registers, no spill (measured on
// worlds256, 256 instances with the spatial order: 594.6 ms against 623.9 ms
// at 1024 threads = 64 registers).  Box worlds take 1280 too although they
// spill 4-16 bytes there (shield1e8 as one instance of 10^8 muons: 2081 ms
// against 2129 ms at 1024).  The variants that spill at 64 registers
// (per-stage field reads; polyhedra) keep 768.
#ifndef MT_BATCH_THREADS_PER_SM_VOXELS
#define MT_BATCH_THREADS_PER_SM_VOXELS 1280
#endif
#ifndef MT_BATCH_THREADS_PER_SM
#define MT_BATCH_THREADS_PER_SM 1280
#endif
#ifndef MT_BATCH_THREADS_PER_SM_WIDE
#define MT_BATCH_THREADS_PER_SM_WIDE 768
#endif

namespace mt {
template <int GEOM, int FIELD>
constexpr int batch_threads_per_sm()
{
    return (GEOM == MT_GEOM_POLYHEDRA || FIELD == kFieldMapStaged) ? MT_BATCH_THREADS_PER_SM_WIDE
           : GEOM == MT_GEOM_VOXELS                                 ? MT_BATCH_THREADS_PER_SM_VOXELS
                                                                    : MT_BATCH_THREADS_PER_SM;
}
}  // namespace mt

struct mt_batch {
    int device = 0;
    int n_inst = 0;
    int geom_kind = -1, field_kind = -1, field_per_stage = -1;
    int hist_n_mat = 0;
    mt::WorldParams tables;                 // histogram part shared by every instance
    mt::DevOwner own_tables;
    std::vector<mt::WorldParams> inst;      // host copies, tables filled in
    std::vector<mt::DevOwner> inst_own;
    std::vector<char> is_set;
    mt::WorldParams *d_inst = nullptr;      // device copy of inst
    bool dirty = true;
    // launch shape chosen by mt_batch_autotune (0 = defaults)
    int tuned_block = 0, tuned_S = 0, tuned_staging = 0;
    // CUDA graph of the last launch sequence and the arguments it was made for
    cudaGraphExec_t graph = nullptr;
    std::vector<char> graph_key;
    // scratch the batch keeps for graph replays without a caller workspace
    // (a captured graph holds its addresses), grown as needed
    char *graph_ws = nullptr;
    int64_t graph_ws_bytes = 0;
};

namespace mt {

struct BatchWs {
    unsigned int *cnt;          // [3][n_inst] live counts (rotating)
    unsigned int *sub;          // [n_inst] live entries handed out in the current pass
    unsigned int *cof;          // [n_inst + 1] item offsets of the current pass
    unsigned int *queue;        // [1] next item
    unsigned long long *off;    // [n_inst + 1] region offsets
    mt_muon_soa *soa;           // [n_inst] caller arrays
    unsigned *hist, *offs;      // [n_inst][kSortBins] each: the spatial order's counts and first slots
    char *live0, *live1;        // two live buffers of N entries
    int64_t N;
    const WorldParams *inst;    // device table of this group's instances
};

// Instance groups of one batched call: with MT_BATCH_GROUP_MIN_MUONS muons or
// more the call runs as two independent batches of about equal muon counts on
// two streams, so one group's passes fill the SMs the other's pass tails
// leave idle, as the plain transport's two muon groups do.  The groups split
// at the instance boundary nearest to half the muons when that leaves them
// within N/16 of each other; otherwise the instance holding muon N/2 is cut
// there, its first `cut` muons in group 0 and the rest in group 1 (a muon's
// draws depend only on its instance word and id, so results are the same).
#ifndef MT_BATCH_GROUP_MIN_MUONS
#define MT_BATCH_GROUP_MIN_MUONS (1 << 19)
#endif

struct BatchSplit {
    int G = 1;
    int i0[2] = {0, 0}, i1[2] = {0, 0};   // instances [i0, i1) of each group
    int s = 0;                             // first instance of group 1
    int64_t cut = 0;                       // > 0: muons of instance s in group 0
};

static BatchSplit batch_groups(int n_inst, const int64_t *n)
{
    BatchSplit sp;
    sp.i1[0] = n_inst;
    int64_t N = 0;
    for (int i = 0; i < n_inst; ++i) N += n[i] > 0 ? n[i] : 0;
    if (n_inst < 1 || N < MT_BATCH_GROUP_MIN_MUONS) return sp;
    int64_t run = 0, best = -1;
    int split = n_inst;
    for (int s = 1; s < n_inst; ++s) {
        run += n[s - 1] > 0 ? n[s - 1] : 0;
        const int64_t d = run * 2 > N ? run * 2 - N : N - run * 2;
        if (best < 0 || d < best) {
            best = d;
            split = s;
        }
    }
    sp.G = 2;
    sp.i1[1] = n_inst;
    if (best >= 0 && best <= N / 16) {
        sp.s = split;
        sp.i1[0] = sp.i0[1] = split;
        return sp;
    }
    const int64_t h = N / 2;
    int64_t o = 0;
    int s = 0;
    for (; s < n_inst; ++s) {
        const int64_t ns = n[s] > 0 ? n[s] : 0;
        if (o + ns > h) break;
        o += ns;
    }
    // o <= h < o + n[s], and h > 0, so s > 0 when the cut is 0
    sp.s = s;
    sp.cut = h - o;
    sp.i0[1] = s;
    sp.i1[0] = sp.cut > 0 ? s + 1 : s;
    return sp;
}

// Muons of instance i (i0[g] <= i < i1[g]) in group g.
static int64_t group_count(const BatchSplit &sp, int g, int i, const int64_t *n)
{
    const int64_t ni = n[i] > 0 ? n[i] : 0;
    if (sp.G == 1 || sp.cut == 0 || i != sp.s) return ni;
    return g == 0 ? sp.cut : ni - sp.cut;
}

static int64_t round256(int64_t x) { return (x + 255) & ~(int64_t)255; }

static int64_t batch_ws_layout(int n_inst, int64_t N, BatchWs *ws, char *base)
{
    int64_t o = 0;
    const int64_t c_cnt = o;
    o = round256(o + 3 * (int64_t)n_inst * 4);
    const int64_t c_sub = o;
    o = round256(o + (int64_t)n_inst * 4);
    const int64_t c_cof = o;
    o = round256(o + ((int64_t)n_inst + 1) * 4);
    const int64_t c_q = o;
    o = round256(o + 4);
    const int64_t c_off = o;
    o = round256(o + ((int64_t)n_inst + 1) * 8);
    const int64_t c_soa = o;
    o = round256(o + (int64_t)n_inst * (int64_t)sizeof(mt_muon_soa));
    const int64_t c_hist = o;
    o = round256(o + 2 * (int64_t)n_inst * kSortBins * (int64_t)sizeof(unsigned));
    const int64_t cap = N > 0 ? N : 1;
    const int64_t c_l0 = o;
    o += 4 * cap * (int64_t)sizeof(float4);
    const int64_t c_l1 = o;
    o += 4 * cap * (int64_t)sizeof(float4);
    if (ws && base) {
        ws->cnt = reinterpret_cast<unsigned int *>(base + c_cnt);
        ws->sub = reinterpret_cast<unsigned int *>(base + c_sub);
        ws->cof = reinterpret_cast<unsigned int *>(base + c_cof);
        ws->queue = reinterpret_cast<unsigned int *>(base + c_q);
        ws->off = reinterpret_cast<unsigned long long *>(base + c_off);
        ws->soa = reinterpret_cast<mt_muon_soa *>(base + c_soa);
        ws->hist = reinterpret_cast<unsigned *>(base + c_hist);
        ws->offs = ws->hist + (int64_t)n_inst * kSortBins;
        ws->live0 = base + c_l0;
        ws->live1 = base + c_l1;
        ws->N = cap;
    }
    return o;
}

__device__ __forceinline__ int find_region(const unsigned long long *off, int n_inst, unsigned long long g)
{
    int lo = 0, hi = n_inst;   // off[lo] <= g < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= g)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Warp-aggregated append to a 32-bit counter shared by the whole warp.
__device__ __forceinline__ int64_t warp_append_u32(unsigned int *ctr, bool keep)
{
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, keep);
    if (!mask) return -1;
    const unsigned lane = threadIdx.x & 31u;
    const int leader = __ffs(mask) - 1;
    unsigned int base = 0;
    if ((int)lane == leader) base = atomicAdd(ctr, (unsigned)__popc(mask));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    return (int64_t)base + __popc(mask & ((1u << lane) - 1u));
}

// Pack the live muons of every instance into its region of live buffer 0
// (positions in the instance's frame).
// Key of the spatial order in the batch's histogram: instance i's bins start at
// i * kSortBins (an instance without a sort grid has the one key 0).
__device__ __forceinline__ uint32_t batch_key(const WorldParams &w, int i, const State &s)
{
    return (uint32_t)i * (uint32_t)kSortBins + (w.sort_bins > 0 ? sort_key(w, s.x, s.y) : 0u);
}

// hist (if not null): each muon takes its rank within its key (spatial order).
__global__ void __launch_bounds__(256) batch_init(const WorldParams *inst, const unsigned long long *off, int n_inst,
                                                  const mt_muon_soa *soa, RunParams rp, LiveBuf out,
                                                  unsigned int *cnt, unsigned *hist)
{
    const unsigned long long N = off[n_inst];
    const unsigned lane = threadIdx.x & 31u;
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < N;
         base += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long g = base + threadIdx.x;
        int i = -1;
        bool live = false;
        State s;
        float q = 0.0f;
        int k = 0;
        int64_t m = 0;
        if (g < N) {
            i = find_region(off, n_inst, g);
            m = (int64_t)(g - off[i]);
            RunParams r = rp;
            r.id_offset = soa[i].id_offset;
            r.instance = soa[i].instance;
            uint32_t a, b;
            live = load_muon(inst[i], soa[i], m, r, s, q, k, a, b);
        }
        // lanes of one warp may straddle two instances: aggregate per instance
        const unsigned act = __ballot_sync(0xFFFFFFFFu, live);
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, live ? i : -1) & act;
        int64_t slot = 0;
        if (live) {
            const int leader = __ffs(peers) - 1;
            unsigned int b0 = 0;
            if ((int)lane == leader) b0 = atomicAdd(&cnt[i], (unsigned)__popc(peers));
            b0 = __shfl_sync(peers, b0, leader);
            slot = (int64_t)off[i] + b0 + __popc(peers & ((1u << lane) - 1u));
        }
        const unsigned rank = hist ? sort_rank(hist, live, live ? batch_key(inst[i], i, s) : 0u) : 0u;
        if (live) put_live(out, slot, s, q, k, m, rank);
    }
}

// Spatial order, step 2: one block per instance turns its counts into first slots.
__global__ void __launch_bounds__(1024) batch_scan(const WorldParams *inst, unsigned *hist, unsigned *offs)
{
    extern __shared__ unsigned v[];   // [1024][kScanStride]
    __shared__ unsigned wsum[32];
    const int i = blockIdx.x;
    const int bins = inst[i].sort_bins > 0 ? inst[i].sort_bins : 1;
    scan_counts(hist + (int64_t)i * kSortBins, offs + (int64_t)i * kSortBins, bins, v, wsum);
}

// Spatial order, step 3: the live entries of every instance (cnt[i] of them at
// off[i] in src) move to off[i] + first slot of their key + rank in dst.  A
// key's ranks are 0 .. count - 1 by construction, so every slot lies in the
// instance's live range; the test only keeps a broken count from writing
// outside it.
__global__ void __launch_bounds__(256) batch_scatter(const WorldParams *inst, const unsigned long long *off, int n_inst,
                                                     const unsigned int *cnt, LiveBuf src, LiveBuf dst,
                                                     const unsigned *offs)
{
    const unsigned long long N = off[n_inst];
    for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < N;
         g += (unsigned long long)gridDim.x * blockDim.x) {
        const int i = find_region(off, n_inst, g);
        const unsigned long long e = g - off[i];
        const unsigned int c = cnt[i];
        if (e >= c) continue;
        const float4 a = src.w0[g], b = src.w1[g], cc = src.w2[g], d = src.w3[g];
        State s;
        s.x = a.x;
        s.y = a.y;
        const unsigned long long pos = (unsigned long long)__ldg(offs + batch_key(inst[i], i, s)) + __float_as_uint(d.w);
        if (pos < c) {
            const unsigned long long to = off[i] + pos;
            dst.w0[to] = a;
            dst.w1[to] = b;
            dst.w2[to] = cc;
            dst.w3[to] = d;
        }
    }
}

// Items of pass p: ceil(live_i / block) per instance, exclusive scan in cof;
// the hand-out counters of the instances are cleared.
__global__ void __launch_bounds__(1024) batch_plan(const unsigned int *cnt_in, unsigned int *cnt_zero, int n_inst,
                                                   int block, unsigned int *cof, unsigned int *queue,
                                                   unsigned int *sub)
{
    __shared__ unsigned int carry;
    if (threadIdx.x == 0) {
        carry = 0;
        *queue = 0;
    }
    __syncthreads();
    for (int base = 0; base < n_inst; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const unsigned int items = i < n_inst ? (cnt_in[i] + block - 1) / block : 0u;
        if (i < n_inst) {
            cnt_zero[i] = 0;
            sub[i] = 0;
        }
        // block-wide exclusive scan of items
        __shared__ unsigned int warp_sums[32];
        unsigned int v = items;
        const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int t = __shfl_up_sync(0xFFFFFFFFu, v, o);
            if ((int)lane >= o) v += t;
        }
        if (lane == 31) warp_sums[wid] = v;
        __syncthreads();
        if (wid == 0) {
            unsigned int ws = lane < (blockDim.x >> 5) ? warp_sums[lane] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned int t = __shfl_up_sync(0xFFFFFFFFu, ws, o);
                if ((int)lane >= o) ws += t;
            }
            warp_sums[lane] = ws;
        }
        __syncthreads();
        const unsigned int incl = v + (wid ? warp_sums[wid - 1] : 0u);
        if (i < n_inst) cof[i] = carry + incl - items;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) cof[n_inst] = carry;
}

// One pass over every instance.  A block pops an item from the queue, which
// names an instance (items of instances are contiguous), stages that world if
// it is not the one staged, and then its warps take chunks of 32 of the
// instance's live entries from sub[i] until none are left, so a warp whose
// muons stop early does not wait for the others.  Items whose instance has
// nothing left to hand out are dropped without staging.
// WS (world staging): MT_BATCH_STAGE_SHARED copies the instance's
// WorldParams into shared memory; MT_BATCH_STAGE_GLOBAL reads them in place
// from the instance table (through L1), which saves the copy and a barrier
// at every instance change.  The small tables (boxes, bin edges, slab index)
// go to shared memory either way.
template <int GEOM, int FIELD, int BLOCK, int WS>
__global__ void __launch_bounds__(BLOCK, batch_threads_per_sm<GEOM, FIELD>() / BLOCK) batch_pass(const WorldParams *__restrict__ inst, const mt_muon_soa *soa,
                                                   const unsigned long long *off, int n_inst, RunParams rp,
                                                   LiveBuf in, LiveBuf out, const unsigned int *cnt_in,
                                                   unsigned int *cnt_out, const unsigned int *cof,
                                                   unsigned int *queue, unsigned int *sub, int S, unsigned *hist)
{
    __shared__ SmemWorld sw;
    __shared__ WorldParams wi;
    __shared__ int s_item, s_inst;
    __shared__ mt_muon_soa s_soa;
    int cur = -1;
    const unsigned int total = cof[n_inst];
    const unsigned lane = threadIdx.x & 31u;
#pragma unroll 1
    while (true) {
        if (threadIdx.x == 0) {
            const unsigned int item = atomicAdd(queue, 1u);
            s_item = (int)item;
            s_inst = -1;
            if (item < total) {
                int lo = 0, hi = n_inst;   // cof[lo] <= item < cof[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (cof[mid] <= item)
                        lo = mid;
                    else
                        hi = mid;
                }
                // lo is the last instance with cof[lo] <= item, so instances without
                // items (cof[j] == cof[j + 1]) are never chosen
                s_inst = *reinterpret_cast<volatile unsigned int *>(&sub[lo]) < cnt_in[lo] ? lo : -1;
            }
        }
        __syncthreads();
        const unsigned int item = (unsigned int)s_item;
        const int i = s_inst;
        if (item >= total) break;
        if (i < 0) {
            __syncthreads();
            continue;
        }
        const WorldParams *wp;
        if constexpr (WS == MT_BATCH_STAGE_GLOBAL)
            wp = inst + i;
        else
            wp = &wi;
        if (i != cur) {
            if constexpr (WS != MT_BATCH_STAGE_GLOBAL) {
                const int words = (int)(sizeof(WorldParams) / 4);
                const int *src = reinterpret_cast<const int *>(&inst[i]);
                int *dst = reinterpret_cast<int *>(&wi);
                for (int t = threadIdx.x; t < words; t += BLOCK) dst[t] = src[t];
            }
            if (threadIdx.x == 0) s_soa = soa[i];
            __syncthreads();
            RunParams r0 = rp;
            stage_world(sw, *wp, r0);
            __syncthreads();
            cur = i;
        }
        const WorldParams &wr = *wp;
        const int64_t id0 = s_soa.id_offset;
        const uint32_t word = (uint32_t)s_soa.instance;
        const int64_t n_i = (int64_t)cnt_in[i];
#pragma unroll 1
        for (;;) {
            unsigned int c = 0;
            if (lane == 0) c = atomicAdd(&sub[i], 32u);
            c = __shfl_sync(0xFFFFFFFFu, c, 0);
            if ((int64_t)c >= n_i) break;
            const int64_t e = (int64_t)c + lane;
            bool keep = false;
            State s;
            float q = 0.0f;
            int k = 0;
            int64_t idx = 0;
            if (e < n_i) {
                get_live(in, (int64_t)off[i] + e, s, q, k, idx);
                const uint64_t id = (uint64_t)(id0 + idx);
                const uint32_t id_lo = (uint32_t)id, id_hi = (uint32_t)(id >> 32);
                const int kend = min(k + S, rp.max_steps);
                int st = MT_ALIVE;
#pragma unroll 1
                for (; k < kend; ++k) {
                    st = step<GEOM, FIELD, NoRecord, false>(wr, sw, s, q, k, id_lo, id_hi, word, rp);
                    if (st != MT_ALIVE) break;
                }
                if (st == MT_ALIVE && k >= rp.max_steps) st = MT_MAX_STEPS;
                if (st != MT_ALIVE)
                    store_muon(wr, s_soa, idx, s, k, st);
                else
                    keep = true;
            }
            const int64_t slot = warp_append_u32(&cnt_out[i], keep);
            const unsigned rank = hist ? sort_rank(hist, keep, keep ? batch_key(wr, i, s) : 0u) : 0u;
            if (keep) put_live(out, (int64_t)off[i] + slot, s, q, k, idx, rank);
        }
        __syncthreads();
    }
}

template <int GEOM, int FIELD, int BLOCK, int WS>
static cudaError_t run_batch(mt_batch *b, const BatchWs &ws, int n_inst, const RunParams &rp, int S, bool order,
                             cudaStream_t st)
{
    const LiveBuf L[2] = {live_buf_at(ws.live0, ws.N), live_buf_at(ws.live1, ws.N)};
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_pass<GEOM, FIELD, BLOCK, WS>, BLOCK, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sms * per_sm;
    const int64_t need = (ws.N + BLOCK - 1) / BLOCK;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    const int64_t ig = std::min<int64_t>(need < 1 ? 1 : need, 65535 * 8);
    const int64_t sg = std::min<int64_t>(need < 1 ? 1 : need, (int64_t)sms * 8);
    cudaError_t e = cudaSuccess;
    if (order) e = cudaMemsetAsync(ws.hist, 0, (size_t)n_inst * kSortBins * sizeof(unsigned), st);
    // the live entries of the list just written to L[src] go to the other list in key order
    auto reorder = [&](int src, const unsigned int *c) {
        batch_scan<<<n_inst, 1024, kScanSmem, st>>>(ws.inst, ws.hist, ws.offs);
        cudaError_t f = cudaGetLastError();
        if (f != cudaSuccess) return f;
        batch_scatter<<<(unsigned)sg, 256, 0, st>>>(ws.inst, ws.off, n_inst, c, L[src], L[src ^ 1], ws.offs);
        return cudaGetLastError();
    };
    // the current list is L[cur]; a pass appends to the other one, which becomes
    // current unless it is reordered back into L[cur]
    int cur = 0;
    if (e == cudaSuccess) {
        batch_init<<<(unsigned)ig, 256, 0, st>>>(ws.inst, ws.off, n_inst, ws.soa, rp, L[order ? 1 : 0], ws.cnt,
                                                 order ? ws.hist : nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && order) e = reorder(1, ws.cnt);
    const int passes = rp.max_steps > 0 ? (rp.max_steps + S - 1) / S : 1;
    for (int p = 0; p < passes && e == cudaSuccess; ++p) {
        unsigned int *c_in = ws.cnt + (p % 3) * n_inst;
        unsigned int *c_out = ws.cnt + ((p + 1) % 3) * n_inst;
        unsigned int *c_zero = ws.cnt + ((p + 2) % 3) * n_inst;
        const bool count = order && p + 1 < passes && (p + 1) % sort_every(S) == 0;
        batch_plan<<<1, 1024, 0, st>>>(c_in, c_zero, n_inst, BLOCK, ws.cof, ws.queue, ws.sub);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        batch_pass<GEOM, FIELD, BLOCK, WS><<<(unsigned)grid, BLOCK, 0, st>>>(
            ws.inst, ws.soa, ws.off, n_inst, rp, L[cur], L[cur ^ 1], c_in, c_out, ws.cof, ws.queue, ws.sub, S,
            count ? ws.hist : nullptr);
        e = cudaGetLastError();
        if (e == cudaSuccess && count) e = reorder(cur ^ 1, c_out);
        if (!count) cur ^= 1;
    }
    return e;
}

template <int BLOCK, int WS>
static cudaError_t dispatch_batch_ws(mt_batch *b, const BatchWs &ws, int n_inst, const RunParams &rp, int S,
                                     bool order, cudaStream_t st)
{
    const int f = b->field_kind;
    const bool staged = b->field_per_stage != 0;
#define MT_BATCH_FIELDS(G)                                                                                     \
    return f == MT_FIELD_MAP && staged ? run_batch<G, kFieldMapStaged, BLOCK, WS>(b, ws, n_inst, rp, S, order, st)      \
           : f == MT_FIELD_MAP         ? run_batch<G, MT_FIELD_MAP, BLOCK, WS>(b, ws, n_inst, rp, S, order, st)         \
           : f == MT_FIELD_MAP_NEAREST ? run_batch<G, MT_FIELD_MAP_NEAREST, BLOCK, WS>(b, ws, n_inst, rp, S, order, st) \
           : f == MT_FIELD_BOX         ? run_batch<G, MT_FIELD_BOX, BLOCK, WS>(b, ws, n_inst, rp, S, order, st)         \
                                       : run_batch<G, MT_FIELD_NONE, BLOCK, WS>(b, ws, n_inst, rp, S, order, st)
    if (b->geom_kind == MT_GEOM_BOXES) MT_BATCH_FIELDS(MT_GEOM_BOXES);
    if (b->geom_kind == MT_GEOM_POLYHEDRA) MT_BATCH_FIELDS(MT_GEOM_POLYHEDRA);
#undef MT_BATCH_FIELDS
    if (f == MT_FIELD_MAP && staged)
        return run_batch<MT_GEOM_VOXELS, kFieldMapStaged, BLOCK, WS>(b, ws, n_inst, rp, S, order, st);
    if (f == MT_FIELD_MAP) return run_batch<MT_GEOM_VOXELS, MT_FIELD_MAP, BLOCK, WS>(b, ws, n_inst, rp, S, order, st);
    if (f == MT_FIELD_MAP_NEAREST)
        return run_batch<MT_GEOM_VOXELS, MT_FIELD_MAP_NEAREST, BLOCK, WS>(b, ws, n_inst, rp, S, order, st);
    return run_batch<MT_GEOM_VOXELS, MT_FIELD_NONE, BLOCK, WS>(b, ws, n_inst, rp, S, order, st);
}

static cudaError_t dispatch_batch(mt_batch *b, const BatchWs &ws, int n_inst, const RunParams &rp, int block, int S,
                                  int staging, bool order, cudaStream_t st)
{
    if (staging == MT_BATCH_STAGE_GLOBAL)
        return block == 128 ? dispatch_batch_ws<128, MT_BATCH_STAGE_GLOBAL>(b, ws, n_inst, rp, S, order, st)
                            : dispatch_batch_ws<256, MT_BATCH_STAGE_GLOBAL>(b, ws, n_inst, rp, S, order, st);
    return block == 128 ? dispatch_batch_ws<128, MT_BATCH_STAGE_SHARED>(b, ws, n_inst, rp, S, order, st)
                        : dispatch_batch_ws<256, MT_BATCH_STAGE_SHARED>(b, ws, n_inst, rp, S, order, st);
}

}  // namespace mt

using namespace mt;

namespace {

struct DevGuardB {
    int prev = -1;
    explicit DevGuardB(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevGuardB()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

mt_status sync_instances(mt_batch *b)
{
    if (!b->dirty) return MT_OK;
    for (int i = 0; i < b->n_inst; ++i)
        if (!b->is_set[i]) {
            set_error("batch instance %d has no world (mt_batch_set_instance)", i);
            return MT_ERR_INVALID_ARG;
        }
    cudaError_t e = cudaSuccess;
    if (!b->d_inst) {
        e = cudaMalloc(&b->d_inst, sizeof(WorldParams) * (size_t)b->n_inst);
        if (e != cudaSuccess) return cuda_fail(e, "batch instance table");
    }
    e = cudaMemcpy(b->d_inst, b->inst.data(), sizeof(WorldParams) * (size_t)b->n_inst, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "batch instance table");
    b->dirty = false;
    return MT_OK;
}

}  // namespace

extern "C" {

mt_status mt_batch_create(const mt_hist_desc *hist, int32_t n_inst, mt_batch **out)
{
    if (!out) {
        set_error("null output pointer");
        return MT_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (n_inst < 1 || n_inst > (1 << 20)) {
        set_error("n_inst %d outside [1, 2^20]", n_inst);
        return MT_ERR_INVALID_ARG;
    }
    mt_status st = validate_hist(hist);
    if (st != MT_OK) return st;
    mt_batch *b = new mt_batch();
    memset(&b->tables, 0, sizeof(b->tables));
    cudaGetDevice(&b->device);
    st = build_hist(hist, b->tables, b->own_tables);
    if (st != MT_OK) {
        b->own_tables.release();
        delete b;
        return st;
    }
    b->n_inst = n_inst;
    b->hist_n_mat = hist->n_mat;
    b->inst.assign(n_inst, b->tables);
    b->inst_own.resize(n_inst);
    b->is_set.assign(n_inst, 0);
    *out = b;
    return MT_OK;
}

mt_status mt_batch_set_instance(mt_batch *b, int32_t i, const mt_geometry_desc *g, const mt_field_desc *f)
{
    if (!b || i < 0 || i >= b->n_inst) {
        set_error("null batch or instance %d out of range", i);
        return MT_ERR_INVALID_ARG;
    }
    mt_status st = validate_geometry(g, b->hist_n_mat);
    if (st == MT_OK) st = validate_field(f, g);
    if (st != MT_OK) return st;
    if ((b->geom_kind >= 0 && g->kind != b->geom_kind) || (b->field_kind >= 0 && f->kind != b->field_kind) ||
        (b->field_per_stage >= 0 && f->per_stage != b->field_per_stage)) {
        set_error("every instance of a batch needs the same geometry kind and field kind");
        return MT_ERR_INVALID_ARG;
    }
    DevGuardB guard(b->device);
    b->inst_own[i].release();
    WorldParams w = b->tables;
    st = build_geometry(g, f, w, b->inst_own[i]);
    if (st == MT_OK) st = build_field(f, w, b->inst_own[i]);
    if (st != MT_OK) {
        b->inst_own[i].release();
        b->is_set[i] = 0;
        return st;
    }
    b->inst[i] = w;
    b->is_set[i] = 1;
    b->geom_kind = g->kind;
    b->field_kind = f->kind;
    b->field_per_stage = f->per_stage;
    b->dirty = true;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return MT_OK;
}

void mt_batch_destroy(mt_batch *b)
{
    if (!b) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->graph_ws) cudaFree(b->graph_ws);
    for (auto &o : b->inst_own) o.release();
    b->own_tables.release();
    if (b->d_inst) cudaFree(b->d_inst);
    if (prev >= 0) cudaSetDevice(prev);
    delete b;
}

int64_t mt_batch_device_bytes(const mt_batch *b)
{
    if (!b) return 0;
    int64_t t = b->own_tables.bytes;
    for (const auto &o : b->inst_own) t += o.bytes;
    return t;
}

int64_t mt_batch_workspace_bytes(const mt_batch *b, const int64_t *n)
{
    if (!b || !n) return -1;
    const BatchSplit sp = batch_groups(b->n_inst, n);
    int64_t bytes = 0;
    for (int g = 0; g < sp.G; ++g) {
        int64_t N = 0;
        for (int i = sp.i0[g]; i < sp.i1[g]; ++i) N += group_count(sp, g, i, n);
        bytes += round256(batch_ws_layout(sp.i1[g] - sp.i0[g], N, nullptr, nullptr));
    }
    return bytes;
}

mt_status mt_transport_batched(mt_batch *b, const mt_muon_soa *soas, const int64_t *n, float step_len,
                               int32_t max_steps, uint64_t seed, const mt_batch_cfg *cfg, void *stream)
{
    if (!b || !soas || !n) {
        set_error("null batch, muon arrays or counts");
        return MT_ERR_INVALID_ARG;
    }
    if (!(step_len > 0.0f) || !isfinite(step_len) || max_steps < 0) {
        set_error("step_len must be positive and finite, max_steps >= 0");
        return MT_ERR_INVALID_ARG;
    }
    mt_batch_cfg c = {0, 0, 0, 0, MT_ORDER_AUTO, 0, nullptr, 0};
    if (cfg) c = *cfg;
    int block = c.block ? c.block : (b->tuned_block ? b->tuned_block : 256);
    int S = c.steps_per_pass ? c.steps_per_pass : b->tuned_S;
    const bool untuned = !S;
    if (untuned) S = 64;   // lowered below, once the call's order is known
    int staging = c.staging ? c.staging : (b->tuned_staging ? b->tuned_staging : MT_BATCH_STAGE_SHARED);
    if ((block != 128 && block != 256) || S < 1 ||
        (staging != MT_BATCH_STAGE_SHARED && staging != MT_BATCH_STAGE_GLOBAL) || c.order < MT_ORDER_AUTO ||
        c.order > MT_ORDER_NEVER) {
        set_error("batch launch: block must be 128 or 256, steps_per_pass >= 1, staging %d or %d and order %d..%d "
                  "(got %d, %d, %d, %d)",
                  MT_BATCH_STAGE_SHARED, MT_BATCH_STAGE_GLOBAL, MT_ORDER_AUTO, MT_ORDER_NEVER, block, S, staging,
                  c.order);
        return MT_ERR_INVALID_ARG;
    }
    std::vector<unsigned long long> off(b->n_inst + 1, 0);
    for (int i = 0; i < b->n_inst; ++i) {
        if (n[i] < 0 || n[i] >= ((int64_t)1 << 31)) {
            set_error("instance %d: n = %lld outside [0, 2^31)", i, (long long)n[i]);
            return MT_ERR_INVALID_ARG;
        }
        if (n[i] > 0 && (!soas[i].x || !soas[i].y || !soas[i].z || !soas[i].px || !soas[i].py || !soas[i].pz ||
                         !soas[i].q || !soas[i].steps || !soas[i].status || soas[i].id_offset < 0)) {
            set_error("instance %d: null muon array or negative id_offset", i);
            return MT_ERR_INVALID_ARG;
        }
        off[i + 1] = off[i] + (unsigned long long)n[i];
    }
    const int64_t N = (int64_t)off[b->n_inst];
    // instance groups (see batch_groups) and their workspaces, one after the other
    const BatchSplit sp = batch_groups(b->n_inst, n);
    const int G = sp.G;
    const int *gi0 = sp.i0, *gi1 = sp.i1;
    int64_t gN[2] = {0, 0}, gws[2] = {0, 0};
    for (int g = 0; g < G; ++g) {
        for (int i = gi0[g]; i < gi1[g]; ++i) gN[g] += group_count(sp, g, i, n);
        gws[g] = round256(batch_ws_layout(gi1[g] - gi0[g], gN[g], nullptr, nullptr));
    }
    const int64_t need = gws[0] + gws[1];
    // spatial order of the live lists (maps only; see compact.cuh)
    const bool order = (b->field_kind == MT_FIELD_MAP || b->field_kind == MT_FIELD_MAP_NEAREST) &&
                       c.order != MT_ORDER_NEVER && (c.order == MT_ORDER_ALWAYS || N >= MT_SORT_MIN_MUONS);
    if (untuned)   // the plain transport's choice for the instance with the largest map layers
        for (int i = 0; i < b->n_inst; ++i)
            if (b->is_set[i]) S = std::min(S, default_steps_per_pass(b->inst[i], step_len, order));
    if (c.workspace && (c.workspace_bytes < need || (reinterpret_cast<uintptr_t>(c.workspace) & 255u))) {
        set_error("batch workspace of %lld bytes too small or not 256-byte aligned (need %lld)",
                  (long long)c.workspace_bytes, (long long)need);
        return MT_ERR_INVALID_ARG;
    }
    DevGuardB guard(b->device);
    mt_status st = sync_instances(b);
    if (st != MT_OK) return st;
    if (N == 0) return MT_OK;
    cudaStream_t cs = (cudaStream_t)stream;
    char *base = reinterpret_cast<char *>(c.workspace);
    bool own = false;
    cudaError_t e = cudaSuccess;
    if (!base && c.use_graph) {
        if (b->graph_ws_bytes < need) {
            // the old scratch may still be in use by earlier work on any stream
            if (b->graph_ws) {
                e = cudaDeviceSynchronize();
                if (e == cudaSuccess) e = cudaFree(b->graph_ws);
                b->graph_ws = nullptr;
                b->graph_ws_bytes = 0;
                if (b->graph) {
                    cudaGraphExecDestroy(b->graph);
                    b->graph = nullptr;
                }
            }
            if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&b->graph_ws), (size_t)need);
            if (e != cudaSuccess) return cuda_fail(e, "batch graph workspace");
            b->graph_ws_bytes = need;
        }
        base = b->graph_ws;
    } else if (!base) {
        e = cudaMallocAsync(reinterpret_cast<void **>(&base), (size_t)need, cs);
        if (e != cudaSuccess) return cuda_fail(e, "batch workspace");
        own = true;
    }
    BatchWs ws[2]{};
    for (int g = 0; g < G; ++g) {
        batch_ws_layout(gi1[g] - gi0[g], gN[g], &ws[g], base + (g ? gws[0] : 0));
        ws[g].inst = b->d_inst + gi0[g];
    }
    RunParams rp;
    rp.d = step_len;
    rp.kd = (float)(0.299792458 * (double)step_len);
    rp.max_steps = max_steps;
    set_seed(rp, seed);
    rp.alpha = nullptr;
    rp.n_block = 0;
    rp.instance = 0;
    rp.id_offset = 0;
    // per-call inputs of each group: region offsets from its first instance,
    // its instances' arrays, cleared counters
    for (int g = 0; g < G && e == cudaSuccess; ++g) {
        const int ni = gi1[g] - gi0[g];
        std::vector<unsigned long long> og(ni + 1, 0);
        std::vector<mt_muon_soa> sg(soas + gi0[g], soas + gi1[g]);
        for (int i = 0; i < ni; ++i) og[i + 1] = og[i] + (unsigned long long)group_count(sp, g, gi0[g] + i, n);
        if (g == 1 && sp.cut > 0) {   // the second part of the cut instance: its muons from `cut` on
            mt_muon_soa &p = sg[0];
            const int64_t c0 = sp.cut;
            p.x += c0;
            p.y += c0;
            p.z += c0;
            p.px += c0;
            p.py += c0;
            p.pz += c0;
            p.q += c0;
            p.steps += c0;
            p.status += c0;
            p.id_offset += c0;
        }
        e = cudaMemcpyAsync(ws[g].off, og.data(), og.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ws[g].soa, sg.data(), sizeof(mt_muon_soa) * (size_t)ni, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaMemsetAsync(ws[g].cnt, 0, 3 * (size_t)ni * sizeof(unsigned int), cs);
    }
    if (e == cudaSuccess && order) e = cudaFuncSetAttribute(batch_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, kScanSmem);
    // both groups' launch sequences on s0: group 1 on the second stream `aux`,
    // forked from s0 and joined back into it (aux is created before and
    // destroyed after any graph capture of this sequence)
    cudaStream_t aux = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    if (e == cudaSuccess && G == 2) e = cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking);
    if (e == cudaSuccess && G == 2) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e == cudaSuccess && G == 2) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    auto launch_groups = [&](cudaStream_t s0) -> cudaError_t {
        if (G == 1) return dispatch_batch(b, ws[0], gi1[0] - gi0[0], rp, block, S, staging, order, s0);
        // fork before either group's work, so that the two run side by side
        cudaError_t f = cudaEventRecord(fork, s0);
        if (f == cudaSuccess) f = cudaStreamWaitEvent(aux, fork, 0);
        if (f == cudaSuccess) f = dispatch_batch(b, ws[0], gi1[0] - gi0[0], rp, block, S, staging, order, s0);
        if (f == cudaSuccess) f = dispatch_batch(b, ws[1], gi1[1] - gi0[1], rp, block, S, staging, order, aux);
        // joined also after an error, so nothing on aux outlives the scratch
        cudaError_t j = cudaEventRecord(join, aux);
        if (j == cudaSuccess) j = cudaStreamWaitEvent(s0, join, 0);
        if (j != cudaSuccess && f == cudaSuccess) f = j;
        return f;
    };
    if (e == cudaSuccess) {
        if (c.use_graph) {
            // capture the launch sequence once per (arguments) and replay it
            std::vector<char> key(sizeof(void *) + 7 * sizeof(int) + sizeof(float) + sizeof(uint64_t) + 16);
            char *kp = key.data();
            memcpy(kp, &base, sizeof(void *));
            kp += sizeof(void *);
            const int ints[7] = {block, S, max_steps, staging, order ? 1 : 0, G == 2 ? sp.s : -1, sp.cut > 0 ? 1 : 0};
            memcpy(kp, ints, sizeof(ints));
            kp += sizeof(ints);
            memcpy(kp, &step_len, sizeof(float));
            kp += sizeof(float);
            memcpy(kp, &seed, sizeof(uint64_t));
            kp += sizeof(uint64_t);
            memcpy(kp, &N, sizeof(int64_t));
            kp += sizeof(int64_t);
            memcpy(kp, &gN[0], sizeof(int64_t));
            if (!b->graph || b->graph_key != key) {
                if (b->graph) {
                    cudaGraphExecDestroy(b->graph);
                    b->graph = nullptr;
                }
                cudaStream_t cap = nullptr;
                e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
                cudaGraph_t gr = nullptr;
                if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    cudaError_t le = launch_groups(cap);
                    e = cudaStreamEndCapture(cap, &gr);
                    if (le != cudaSuccess) e = le;
                }
                if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, gr, 0);
                if (gr) cudaGraphDestroy(gr);
                if (cap) cudaStreamDestroy(cap);
                if (e == cudaSuccess) b->graph_key = key;
            }
            if (e == cudaSuccess) e = cudaGraphLaunch(b->graph, cs);
        } else {
            e = launch_groups(cs);
        }
    }
    // released once their work is done
    if (join) cudaEventDestroy(join);
    if (fork) cudaEventDestroy(fork);
    if (aux) cudaStreamDestroy(aux);
    if (own) {
        const cudaError_t f = cudaFreeAsync(base, cs);
        if (e == cudaSuccess) e = f;
    }
    if (e != cudaSuccess) return cuda_fail(e, "batched transport");
    return MT_OK;
}

mt_status mt_batch_autotune(mt_batch *b, const mt_muon_soa *soas, const int64_t *n, float step_len, int32_t max_steps,
                            uint64_t seed, int64_t sample_per_instance, mt_batch_cfg *best, void *stream)
{
    if (!b || !soas || !n || sample_per_instance < 1) {
        set_error("null batch, muon arrays or counts, or sample_per_instance < 1");
        return MT_ERR_INVALID_ARG;
    }
    DevGuardB guard(b->device);
    cudaStream_t cs = (cudaStream_t)stream;
    // scratch copies of the first min(n_i, sample) muons of every instance
    std::vector<int64_t> m(b->n_inst);
    int64_t M = 0;
    for (int i = 0; i < b->n_inst; ++i) {
        if (n[i] < 0) {
            set_error("instance %d: n < 0", i);
            return MT_ERR_INVALID_ARG;
        }
        m[i] = std::min<int64_t>(n[i], sample_per_instance);
        M += m[i];
    }
    if (M == 0) {
        if (best) *best = mt_batch_cfg{256, 64, 0, MT_BATCH_STAGE_SHARED, MT_ORDER_AUTO, 0, nullptr, 0};
        return MT_OK;
    }
    const size_t per = 4 * 6 + 1 + 4 + 1;   // bytes per muon over the nine arrays
    char *init = nullptr, *work = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&init), (size_t)M * per + 9 * 256, cs);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&work), (size_t)M * per + 9 * 256, cs);
    if (e != cudaSuccess) return cuda_fail(e, "autotune scratch");
    auto carve = [&](char *base, std::vector<mt_muon_soa> &out) {
        const size_t sizes[9] = {4, 4, 4, 4, 4, 4, 1, 4, 1};
        char *q = base;
        void *arr[9];
        for (int a = 0; a < 9; ++a) {
            arr[a] = q;
            q += ((size_t)M * sizes[a] + 255) & ~(size_t)255;
        }
        out.resize(b->n_inst);
        int64_t o = 0;
        for (int i = 0; i < b->n_inst; ++i) {
            mt_muon_soa s = soas[i];
            s.x = (float *)arr[0] + o;
            s.y = (float *)arr[1] + o;
            s.z = (float *)arr[2] + o;
            s.px = (float *)arr[3] + o;
            s.py = (float *)arr[4] + o;
            s.pz = (float *)arr[5] + o;
            s.q = (int8_t *)arr[6] + o;
            s.steps = (int32_t *)arr[7] + o;
            s.status = (uint8_t *)arr[8] + o;
            out[i] = s;
            o += m[i];
        }
    };
    std::vector<mt_muon_soa> si, sw;
    carve(init, si);
    carve(work, sw);
    for (int i = 0; i < b->n_inst && e == cudaSuccess; ++i) {
        if (!m[i]) continue;
        const size_t sz4 = (size_t)m[i] * 4, sz1 = (size_t)m[i];
        const void *src[9] = {soas[i].x, soas[i].y, soas[i].z, soas[i].px, soas[i].py, soas[i].pz, soas[i].q,
                              soas[i].steps, soas[i].status};
        void *dst[9] = {si[i].x, si[i].y, si[i].z, si[i].px, si[i].py, si[i].pz, si[i].q, si[i].steps, si[i].status};
        const size_t sz[9] = {sz4, sz4, sz4, sz4, sz4, sz4, sz1, sz4, sz1};
        for (int a = 0; a < 9 && e == cudaSuccess; ++a)
            e = cudaMemcpyAsync(dst[a], src[a], sz[a], cudaMemcpyDeviceToDevice, cs);
    }
    // the search: block size x steps per pass x world staging
    const int blocks[2] = {128, 256};
    const int Ss[5] = {32, 64, 128, 256, 512};
    const int stagings[2] = {MT_BATCH_STAGE_SHARED, MT_BATCH_STAGE_GLOBAL};
    float best_ms = 1e30f;
    mt_batch_cfg bc = {256, 64, 0, MT_BATCH_STAGE_SHARED, MT_ORDER_AUTO, 0, nullptr, 0};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    mt_status st = MT_OK;
    for (int gi = 0; gi < 2 && e == cudaSuccess && st == MT_OK; ++gi)
    for (int bi = 0; bi < 2 && e == cudaSuccess && st == MT_OK; ++bi)
        for (int si_ = 0; si_ < 5 && e == cudaSuccess && st == MT_OK; ++si_) {
            mt_batch_cfg c = {blocks[bi], Ss[si_], 0, stagings[gi], MT_ORDER_AUTO, 0, nullptr, 0};
            for (int rep = 0; rep < 2 && e == cudaSuccess && st == MT_OK; ++rep) {   // warm-up, then timed
                e = cudaMemcpyAsync(work, init, (size_t)M * per + 9 * 256, cudaMemcpyDeviceToDevice, cs);
                if (e != cudaSuccess) break;
                e = cudaEventRecord(e0, cs);
                if (e == cudaSuccess) st = mt_transport_batched(b, sw.data(), m.data(), step_len, max_steps, seed, &c, cs);
                if (e == cudaSuccess && st == MT_OK) e = cudaEventRecord(e1, cs);
                if (e == cudaSuccess && st == MT_OK) e = cudaEventSynchronize(e1);
            }
            float ms = 0.0f;
            if (e == cudaSuccess && st == MT_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
                best_ms = ms;
                bc = c;
            }
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(init, cs);
    cudaFreeAsync(work, cs);
    if (st != MT_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    b->tuned_block = bc.block;
    b->tuned_S = bc.steps_per_pass;
    b->tuned_staging = bc.staging;
    if (best) *best = bc;
    return MT_OK;
}

}  // extern "C"
