// mt_internal.cuh -- device data layout and handle of libmt (CUDA path only).
//
// HBM layout of one world (all built once by mt_create):
//   boxes   : DevBox[n_box]          float hi/lo pairs of every face, material, block, B
//   hist    : HistRec[n_mat*n_pbin]  per histogram: guide/pair offsets and jitter scales
//   guide   : u32[n_hist << gbits]   Chen-Asau guide table over the 32-bit draw space
//   pairs   : uint2[sum m_h]         (upper threshold, cell) of the selectable cells
//   e2      : float2[n_pbin+1]       squared log10 bin edges as (hi, lo) float pairs
//   fmap    : float4[nz][ny][nx-1][2] x-adjacent node pairs (Bx,By,Bz,0 | Bx,By,Bz,0)
//   vox     : u8[nz][ny][nx]         voxel materials
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/mt.h"

namespace mt {


struct DevBox {
    float lo_hi[3], lo_lo[3];
    float hi_hi[3], hi_lo[3];
    float B[3];
    int32_t material;
    int32_t block;
    int32_t pad;
};

// Guide entry: bit 31 clear -> the answer cell; set -> binary search over
// pairs[lo .. lo+span] with lo = bits 0..14 and span = bits 15..29.
struct HistRec {
    uint32_t guide_off;
    uint32_t pair_off;
    float fscale;     // f_max / nf
    float tscale;     // theta_max / ntheta
};

constexpr int kZSlabs = 256;   // z slabs of the box-candidate index

// Field template value of the kernels for MT_FIELD_MAP with per_stage set.
constexpr int kFieldMapStaged = 4;

// Most bins of the live list's spatial order (keys 0 .. kSortBins - 1; a
// multiple of 1024).
constexpr int kSortBins = 16384;

struct WorldParams {
    // geometry
    int32_t geom_kind;
    int32_t n_box;
    const uint32_t *zmask;         // [kZSlabs] candidate boxes per z slab (bit b = box b)
    float zslab_lo, zslab_inv;     // slab = floor((z - zslab_lo) * zslab_inv), clamped
    int32_t world_mat;
    int32_t n_mat;
    const DevBox *boxes;
    const uint8_t *vox;
    int32_t vdims[3];
    float vorigin[3];
    float vinv[3];
    float vorigin_lo[3];
    float vspacing[3];
    float vspacing_lo[3];
    const float4 *poly;            // solids: [n_box][6] float4 (see api.cu: build_geometry)
    const double *poly64;          // solids: [n_box][18] z0, z1, bottom[4][2], top[4][2]
    const float4 *pinner;          // solids: [n_box] inner rectangle (x0, x1, y0, y1)
    // world bounds in frame units: the muon leaves where x >= xmax or x <= xmin
    // (|x| >= x_max in metres), likewise y, or z >= zmax
    float xmax_hi, xmax_lo, ymax_hi, ymax_lo, zmax_hi, zmax_lo;
    float xmin_hi, xmin_lo, ymin_hi, ymin_lo;
    float pmin2;
    // Frame of the muon position: the state holds u = (r - o) / s per axis, in
    // cell units of the field map's node grid when there is a map (node i of an
    // axis at u = i), else metres (o = 0, s = 1).  Every geometric constant of
    // the world (faces, bounds, voxel and slab grids, solids) is stored in the
    // same units.  o, s and 1/s as hi + lo pairs.
    float fro_h[3], fro_l[3];
    float frs_h[3], frs_l[3];
    float fri_h[3], fri_l[3];
    // field
    int32_t field_kind;
    int32_t field_per_stage;       // MT_FIELD_MAP read at every RK4 stage (kernels: kFieldMapStaged)
    const float4 *fmap;            // trilinear: x-adjacent node pairs; nearest: nodes [nz][ny][nx]
    int32_t fdims[3];
    // nearest-node cells in frame units (origin -1/2, spacing 1)
    float forigin[3];
    float forigin_lo[3];
    float fspacing[3];
    float fspacing_lo[3];
    float finv[3];                 // trilinear map: 1 / node spacing in 1/m (field gradients)
    // xy grid of the live list's spatial order (maps only): the key of a muon is
    // (j >> sort_shift) * sort_nx + (i >> sort_shift) for its map cell (i, j),
    // sort_shift >= 1; sort_bins = 0 leaves the list unordered
    int32_t sort_shift, sort_nx, sort_bins;
    // histograms
    const HistRec *hist;
    const uint32_t *guide;
    const uint2 *pairs;
    const float2 *e2;
    int32_t n_pbin;
    int32_t nf;
    int32_t ntheta;
    int32_t gshift;
    int32_t axes;             // MT_AXES_LINEAR or MT_AXES_LOG
    const float4 *hist_log;   // log axes: per histogram {f_min, d hi, d lo, 0}, {t_min, d hi, d lo, 0}, d = log2 cell width
    int32_t sampler;          // MT_SAMPLER_ICDF or MT_SAMPLER_ALIAS
    const uint2 *alias;       // alias columns {Prob_j, alias cell (a << 16) | b}, at HistRec.guide_off
    int32_t alias_bits;       // log2(nf * ntheta)
    int32_t theta_bits;       // log2(ntheta)
    int32_t pbin_custom;      // 1: explicit bin edges (binary search over e2), 0: log10 bins
    float log2_plo;
    float pbin_scale;   // n_pbin / log2(p_hi / p_lo)
    float pbin_eps;     // bound on the error of the FP32 bin coordinate (times 4), at least 1e-4
};

struct RunParams {
    float d;
    float kd;            // kappa * d
    int32_t max_steps;
    uint32_t key0, key1;
    // Philox round keys: round r uses (key0 + r * 0x9E3779B9, key1 + r * 0xBB67AE85).
    // Held in the launch parameters, they enter the round's xor as constant
    // operands instead of being advanced in registers every step.
    uint32_t rk[2][10];
    const float *alpha;   // device [n_block][3] or null
    int32_t n_block;
    int32_t instance;
    int64_t id_offset;
};

// The seed's two key words and the round keys derived from them.
inline void set_seed(RunParams &rp, uint64_t seed)
{
    rp.key0 = (uint32_t)seed;
    rp.key1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rp.rk[0][r] = rp.key0 + (uint32_t)r * 0x9E3779B9u;
        rp.rk[1][r] = rp.key1 + (uint32_t)r * 0xBB67AE85u;
    }
}

}  // namespace mt

namespace mt {
// Device allocations owned by a handle or a batch.
struct DevOwner {
    std::vector<void *> bufs;
    int64_t bytes = 0;
    void release();
};
}  // namespace mt

struct mt_handle {
    int device;
    mt::WorldParams w;
    mt::DevOwner own;
};

namespace mt {
void set_error(const char *fmt, ...);
mt_status cuda_fail(cudaError_t e, const char *what);
mt_status validate_hist(const mt_hist_desc *h);
mt_status validate_geometry(const mt_geometry_desc *g, int n_mat);
mt_status validate_field(const mt_field_desc *f, const mt_geometry_desc *g);
mt_status build_hist(const mt_hist_desc *hd, WorldParams &w, DevOwner &own);
mt_status build_geometry(const mt_geometry_desc *g, const mt_field_desc *f, WorldParams &w, DevOwner &own);
mt_status build_field(const mt_field_desc *f, WorldParams &w, DevOwner &own);
void noalloc_prepare(const WorldParams &w, int dev);   // noalloc.cu
struct CompactPlan {   // compact.cu
    int passes;
    bool order;
    int every;   // passes between reorders
};
CompactPlan compact_plan(const WorldParams &w, int64_t n, int max_steps, int S, int order_mode);
int64_t compact_call_launches(const WorldParams &w, int64_t n, int max_steps, int S, int order_mode);
// whether a compacting call of n muons reorders its live list (compact.cu)
bool call_ordered(const WorldParams &w, int64_t n, int order_mode);
int default_steps_per_pass(const WorldParams &w, float step_len, bool ordered);   // transport.cu
}  // namespace mt
