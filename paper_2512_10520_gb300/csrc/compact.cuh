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

// Pack the live muons (status ALIVE or MAX_STEPS, finite state) of the
// caller's arrays into a live list, positions in the world's frame; non-finite
// states are marked MT_INVALID.
static __global__ void __launch_bounds__(kBlock) compact_init(const WorldParams w, const mt_muon_soa soa, int64_t n,
                                                              const RunParams rp, LiveBuf out, unsigned long long *ctr)
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
        if (live) put_live(out, slot, s, q, k, m);
    }
}

// One pass: live count from *cin, survivors appended at *cout; *czero (if not
// null) is cleared for the pass after this one.  Warps take the live list in
// chunks of 32 entries from the counter *work (zero at the start of the pass),
// so a warp whose muons stop early takes more chunks and the SMs finish the
// pass together; *wzero (if not null) is cleared for a later pass.
template <int GEOM, int FIELD>
__global__ void __launch_bounds__(kBlock, pass_min_blocks<GEOM, FIELD>()) compact_pass(const WorldParams w, const mt_muon_soa soa, const RunParams rp,
                                                       LiveBuf in, LiveBuf out, const unsigned long long *cin,
                                                       unsigned long long *cout, unsigned long long *czero,
                                                       unsigned long long *work, unsigned long long *wzero, int S)
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
        if (keep) put_live(out, slot, s, q, k, idx);
    }
}

}  // namespace mt
