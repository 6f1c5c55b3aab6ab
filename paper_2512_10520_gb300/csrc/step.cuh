// step.cuh -- one step of Algorithm 1 on a register-resident muon, shared by
// every transport kernel (plain, compacting, batched, adjoint recompute).
//
// Position and momentum are carried as unevaluated sums hi + lo of two floats
// (compensated accumulation), so 1500 steps of FP32 arithmetic stay within
// ~1e-9 relative of the exact track; every discrete decision (box faces, world
// bounds, momentum-bin edges, voxel faces) compares the full hi + lo value
// against bounds also stored as hi + lo pairs.  The position is held in the
// world's frame (WorldParams): cell units of the field map when there is one,
// so that the map's cell and in-cell fraction come straight from the state.  The only stochastic input is one
// Philox4x32-10 call per step in matter, keyed by the seed and counted by
// (step, muon id, instance), so a muon's track does not depend on which
// thread, block or launch runs it.
#pragma once

#include "mt_internal.cuh"

namespace mt {

constexpr int kBlock = 256;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies whose halves are xor-mixed with the other words and the
// round key; the key advances by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// The same generator with the ten round keys given (see RunParams::rk).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const uint32_t (&rk)[2][10])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ rk[0][r], lo1, hi0 ^ c.w ^ rk[1][r], lo0);
    }
    return c;
}

// U(w) = (w >> 8) * 2^-24, exact in FP32.
__device__ __forceinline__ float u01(uint32_t w) { return __uint2float_rz(w >> 8) * 5.9604644775390625e-8f; }

// hi + lo accumulation of a small increment (Fast2Sum of hi and d + lo).
__device__ __forceinline__ void acc(float &hi, float &lo, float d)
{
    const float y = d + lo;
    const float t = hi + y;
    lo = y - (t - hi);
    hi = t;
}

// (xh + xl) >= (bh + bl) for normalised pairs.
__device__ __forceinline__ bool ge2(float xh, float xl, float bh, float bl)
{
    return xh > bh || (xh == bh && xl >= bl);
}

struct State {
    float x, y, z, px, py, pz;
    float xl, yl, zl, pxl, pyl, pzl;
};

// Histogram records staged in shared memory when the set has at most this many
// (n_mat x n_pbin); larger sets read them from global memory.  A warp's lanes
// mostly hold different (material, bin) records, so a global load of them takes
// one L1 wavefront per lane where shared memory serves 8 lanes per wavefront.
constexpr int kHistSmem = 512;

// Shared-memory copy of the small per-world tables.
struct SmemWorld {
    HistRec hist[kHistSmem];
    float lo_hi[3][MT_MAX_BOXES], lo_lo[3][MT_MAX_BOXES];
    float hi_hi[3][MT_MAX_BOXES], hi_lo[3][MT_MAX_BOXES];
    float B[3][MT_MAX_BOXES];
    int32_t mat[MT_MAX_BOXES];
    int32_t block[MT_MAX_BOXES];
    float alpha[3][MT_MAX_BOXES];
    float2 e2[MT_MAX_PBINS + 1];
    uint32_t zmask[kZSlabs];
    float4 inner[MT_MAX_BOXES];   // solids: (x0, x1, y0, y1) of a rectangle inside every slice
};

__device__ __forceinline__ void stage_world(SmemWorld &sw, const WorldParams &w, const RunParams &rp)
{
    for (int t = threadIdx.x; t < w.n_box; t += blockDim.x) {
        const DevBox b = w.boxes[t];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            sw.lo_hi[a][t] = b.lo_hi[a];
            sw.lo_lo[a][t] = b.lo_lo[a];
            sw.hi_hi[a][t] = b.hi_hi[a];
            sw.hi_lo[a][t] = b.hi_lo[a];
            sw.B[a][t] = b.B[a];
        }
        sw.mat[t] = b.material;
        sw.block[t] = b.block;
    }
    for (int t = threadIdx.x; t < MT_MAX_BOXES; t += blockDim.x)
#pragma unroll
        for (int a = 0; a < 3; ++a) sw.alpha[a][t] = (rp.alpha && t < rp.n_block) ? rp.alpha[3 * t + a] : 1.0f;
    for (int t = threadIdx.x; t <= w.n_pbin; t += blockDim.x) sw.e2[t] = w.e2[t];
    if (w.n_mat * w.n_pbin <= kHistSmem)
        for (int t = threadIdx.x; t < w.n_mat * w.n_pbin; t += blockDim.x) sw.hist[t] = w.hist[t];
    for (int t = threadIdx.x; t < kZSlabs; t += blockDim.x) sw.zmask[t] = w.zmask ? w.zmask[t] : 0u;
    if (w.pinner)
        for (int t = threadIdx.x; t < w.n_box; t += blockDim.x) sw.inner[t] = w.pinner[t];
}

// lo <= r < hi for box (or bounding box) b, r and the faces as hi + lo pairs.
// Unless a hi word of r equals a face, the test on the hi words is the pair test
// (ge2 reduces to > and its negation to < without a tie); the lo words are read
// only on a tie.
__device__ __forceinline__ bool in_box(const SmemWorld &sw, int b, const State &s)
{
    const float z0 = sw.lo_hi[2][b], z1 = sw.hi_hi[2][b], x0 = sw.lo_hi[0][b], x1 = sw.hi_hi[0][b];
    const float y0 = sw.lo_hi[1][b], y1 = sw.hi_hi[1][b];
    const bool tie = s.z == z0 || s.z == z1 || s.x == x0 || s.x == x1 || s.y == y0 || s.y == y1;
    if (!tie) return s.z > z0 && s.z < z1 && s.x > x0 && s.x < x1 && s.y > y0 && s.y < y1;
    return ge2(s.z, s.zl, z0, sw.lo_lo[2][b]) && !ge2(s.z, s.zl, z1, sw.hi_lo[2][b]) &&
           ge2(s.x, s.xl, x0, sw.lo_lo[0][b]) && !ge2(s.x, s.xl, x1, sw.hi_lo[0][b]) &&
           ge2(s.y, s.yl, y0, sw.lo_lo[1][b]) && !ge2(s.y, s.yl, y1, sw.hi_lo[1][b]);
}

// GetMaterial for ordered boxes: first box with lo <= r < hi on all axes.  Only
// the boxes listed for the point's z slab are tested (the paper prunes its
// candidate volumes with a spatial grid the same way), in list order.
__device__ __forceinline__ int find_box(const WorldParams &w, const SmemWorld &sw, const State &s)
{
    const int slab = min(max(__float2int_rd((s.z - w.zslab_lo) * w.zslab_inv), 0), kZSlabs - 1);
    uint32_t cand = sw.zmask[slab];
    while (cand) {
        const int b = __ffs(cand) - 1;
        cand &= cand - 1u;
        if (in_box(sw, b, s)) return b;
    }
    return -1;
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// floor((x - origin) / spacing) of a point given as a hi + lo pair, for a
// grid whose origin and spacing are hi + lo pairs as well.  The offset
// x - origin is formed as a pair; when the cell coordinate lies within 1e-4
// of a face, the face position (index * spacing, also as a pair) settles which
// side of it the point is on.
__device__ __forceinline__ int grid_cell(float xh, float xl, float oh, float ol, float sh, float sl, float inv)
{
    float dh, de;
    two_sum(xh, -oh, dh, de);
    const float dl = de + (xl - ol);
    const float u = (dh + dl) * inv;
    int i = __float2int_rd(u);
    const float fr = u - (float)i;
    if (fr < 1e-4f || fr > 0.9999f) {
        const int ic = __float2int_rn(u);
        const float fic = (float)ic;
        const float fh = fic * sh;
        const float fl = fmaf(fic, sl, fmaf(fic, sh, -fh));
        i = ((dh - fh) + (dl - fl)) >= 0.0f ? ic : ic - 1;
    }
    return i;
}

// GetMaterial for a voxel grid: floor((r - origin) / spacing) inside the grid.
__device__ __forceinline__ int voxel_material(const WorldParams &w, const State &s)
{
    const float r[3] = {s.x, s.y, s.z};
    const float rl[3] = {s.xl, s.yl, s.zl};
    int idx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int i = grid_cell(r[a], rl[a], w.vorigin[a], w.vorigin_lo[a], w.vspacing[a], w.vspacing_lo[a], w.vinv[a]);
        if (i < 0 || i >= w.vdims[a]) return -1;
        idx[a] = i;
    }
    return __ldg(w.vox + ((int64_t)idx[2] * w.vdims[1] + idx[1]) * w.vdims[0] + idx[0]);
}

// Nearest-node field (the paper's lookup, Sec. Simulation item 3): the node
// whose Voronoi cell holds the point, found as the cell of a grid shifted by
// half a spacing (origin stored shifted); zero when that node is off the map.
__device__ __forceinline__ float3 field_map_nearest(const WorldParams &w, const State &s)
{
    const float r[3] = {s.x, s.y, s.z};
    const float rl[3] = {s.xl, s.yl, s.zl};
    int idx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int i = grid_cell(r[a], rl[a], w.forigin[a], w.forigin_lo[a], w.fspacing[a], w.fspacing_lo[a], w.finv[a]);
        if (i < 0 || i >= w.fdims[a]) return make_float3(0.0f, 0.0f, 0.0f);
        idx[a] = i;
    }
    const float4 b = __ldg(w.fmap + ((int64_t)idx[2] * w.fdims[1] + idx[1]) * w.fdims[0] + idx[0]);
    return make_float3(b.x, b.y, b.z);
}

// Containment in solid b of the polyhedron geometry (Sec. Simulation item 1,
// Eq. 2), in FP64 from the solid's original double-precision data: the
// definition's arithmetic, used when the FP32 filter below cannot decide.
// z0 <= z < z1 has been decided already.
// Inlined (measured on tapered1e6 at 64 registers: 33.2 ms against 36.0 ms for a
// call, whose register saves cost more than the rarely run code itself).
#ifndef MT_SOLID_FP64_INLINE
#define MT_SOLID_FP64_INLINE 1
#endif
#if MT_SOLID_FP64_INLINE
static __device__ __forceinline__ bool in_solid_fp64(
#else
static __device__ __noinline__ bool in_solid_fp64(
#endif
    const WorldParams &w, int b, const State &s)
{
    // one edge at a time, both ends recomputed from memory: few values live
    const double *d = w.poly64 + 18 * b;   // the solid in frame units
    const double x = (double)s.x + (double)s.xl, y = (double)s.y + (double)s.yl, z = (double)s.z + (double)s.zl;
    const double z0 = __ldg(d), z1 = __ldg(d + 1);
    const double t = (z - z0) / (z1 - z0);
#pragma unroll 1
    for (int i = 0; i < 4; ++i) {
        const int j = (i + 1) & 3;
        const double bix = __ldg(d + 2 + 2 * i), biy = __ldg(d + 3 + 2 * i);
        const double bjx = __ldg(d + 2 + 2 * j), bjy = __ldg(d + 3 + 2 * j);
        const double vix = bix + t * (__ldg(d + 10 + 2 * i) - bix), viy = biy + t * (__ldg(d + 11 + 2 * i) - biy);
        const double vjx = bjx + t * (__ldg(d + 10 + 2 * j) - bjx), vjy = bjy + t * (__ldg(d + 11 + 2 * j) - bjy);
        const double ex = vjx - vix, ey = vjy - viy;
        if (ex * (y - viy) - ey * (x - vix) < 0.0) return false;
    }
    return true;
}

// Eq. 2 with a certified FP32 filter, for a point already known to lie in the
// solid's z range.  Each S_i is formed in FP32 from the hi + lo position and
// the interpolated slice, both in frame units (a positive diagonal scaling of
// the plane keeps the sign of every S_i).  Its rounding error (from t, v_i, e_i, dx, dy and S)
// is at most 14 eps (|e_x| + |e_y| + 2M) (|dx| + |dy| + 2M), eps = 2^-24, M the
// solid's coordinate scale; the solid's constant bound is 100 eps times that
// product's maximum over the points that reach the test (its bounding box).
// S_i < -bound proves the point outside; when every S_i > bound it is inside;
// otherwise (the point within ~1e-4 m of a side face) the FP64 test decides,
// so the decision is the definition's at the GPU's position.
__device__ __forceinline__ bool in_solid_sides(const WorldParams &w, int b, const State &s)
{
    const float4 *P = w.poly + 6 * b;
    const float4 zz = __ldg(P);   // z0 hi, z0 lo, 1 / (z1 - z0), bound
    float dzh, dze;
    two_sum(s.z, -zz.x, dzh, dze);
    const float t = (dzh + (dze + (s.zl - zz.y))) * zz.z;
    const float4 b0 = __ldg(P + 1), b1 = __ldg(P + 2), d0 = __ldg(P + 3), d1 = __ldg(P + 4);
    const float vx[4] = {fmaf(t, d0.x, b0.x), fmaf(t, d0.z, b0.z), fmaf(t, d1.x, b1.x), fmaf(t, d1.z, b1.z)};
    const float vy[4] = {fmaf(t, d0.y, b0.y), fmaf(t, d0.w, b0.w), fmaf(t, d1.y, b1.y), fmaf(t, d1.w, b1.w)};
    const float bound = zz.w;
    bool undecided = false;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int j = (i + 1) & 3;
        const float ex = vx[j] - vx[i], ey = vy[j] - vy[i];
        const float dx = (s.x - vx[i]) + s.xl, dy = (s.y - vy[i]) + s.yl;
        const float S = fmaf(ex, dy, -(ey * dx));
        if (S < -bound) return false;
        undecided |= S <= bound;
    }
    return !undecided || in_solid_fp64(w, b, s);
}

// GetMaterial for solids.  The candidates come from the z-slab grid of
// candidate masks in shared memory (a one-dimensional spatial hash; the paper
// prunes its polyhedra with a spatial grid before the exact test), in list
// order.  A candidate is skipped unless the point lies in its bounding box
// (x and y grown by 1e-4 m, z exactly [z0, z1), tested on the hi + lo pairs);
// a point inside the solid's inner rectangle (1e-4 m clear of every slice's
// sides, so the FP32 comparison decides) is inside; otherwise Eq. 2 decides.
// The first containing solid wins.
__device__ __forceinline__ int find_solid(const WorldParams &w, const SmemWorld &sw, const State &s)
{
    const int slab = min(max(__float2int_rd((s.z - w.zslab_lo) * w.zslab_inv), 0), kZSlabs - 1);
    uint32_t cand = sw.zmask[slab];
    while (cand) {
        const int b = __ffs(cand) - 1;
        cand &= cand - 1u;
        if (!in_box(sw, b, s)) continue;
        const float4 in = sw.inner[b];
        if (s.x > in.x && s.x < in.y && s.y > in.z && s.y < in.w) return b;
        if (in_solid_sides(w, b, s)) return b;
    }
    return -1;
}

// |p|^2 of the hi + lo momentum to first order in lo.
__device__ __forceinline__ float p2_of(const State &s)
{
    const float P2 = fmaf(s.px, s.px, fmaf(s.py, s.py, s.pz * s.pz));
    return fmaf(2.0f * s.px, s.pxl, fmaf(2.0f * s.py, s.pyl, fmaf(2.0f * s.pz, s.pzl, P2)));
}

// (h + l)^2 as an unnormalised pair.
__device__ __forceinline__ void sq2(float h, float l, float &sh, float &sl)
{
    sh = h * h;
    sl = fmaf(2.0f * h, l, fmaf(h, h, -sh));
}


// GetMomentumBin on log10 bins (a fast FP32 estimate) or over explicit edges
// (binary search), confirmed against the squared edges held as hi + lo pairs
// whenever the estimate is near a bin face or |p|^2 lies within 4e-6 of an edge.
__device__ __forceinline__ int momentum_bin(const WorldParams &w, const SmemWorld &sw, const State &s, float P2)
{
    int i;
    if (w.pbin_custom) {
        // explicit edges: binary search of P^2 over the squared edges (hi words);
        // the exact hi + lo test below settles a P^2 within 4e-6 of an edge
        int lo = 0, hi = w.n_pbin;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (sw.e2[mid].x <= P2)
                lo = mid;
            else
                hi = mid;
        }
        i = lo;
    } else {
        // The estimate's bin coordinate u is within pbin_eps / 4 of the exact one
        // (the FP32 log2 and the roundings, bounded on the host), so a fraction of
        // u farther than pbin_eps from an integer settles the bin; otherwise the
        // squared edges decide below.
        const float u = fmaf(0.5f, __log2f(P2), -w.log2_plo) * w.pbin_scale;
        i = __float2int_rd(u);
        const float fr = u - (float)i;
        i = min(max(i, 0), w.n_pbin - 1);
        if (fr > w.pbin_eps && fr < 1.0f - w.pbin_eps) return i;
    }
    const float elo = sw.e2[i].x, ehi = sw.e2[i + 1].x;
    const bool near_lo = i > 0 && P2 < elo * 1.000004f;
    const bool near_hi = i < w.n_pbin - 1 && P2 > ehi * 0.999996f;
    if (near_lo || near_hi) {
        float ah, al, bh, bl, ch, cl;
        sq2(s.px, s.pxl, ah, al);
        sq2(s.py, s.pyl, bh, bl);
        sq2(s.pz, s.pzl, ch, cl);
        float sh, se;
        two_sum(ah, bh, sh, se);
        float th, te;
        two_sum(sh, ch, th, te);
        const float tl = se + te + al + bl + cl;
        if (near_lo) {
            const float2 e = sw.e2[i];
            if ((th - e.x) + (tl - e.y) < 0.0f) --i;
        } else {
            const float2 e = sw.e2[i + 1];
            if ((th - e.x) + (tl - e.y) >= 0.0f) ++i;
        }
    }
    return i;
}

// Inverse CDF through the guide table; returns the cell as (a << 16) | b.
__device__ __forceinline__ uint32_t sample_cell(const uint32_t *guide, const uint2 *pairs, int gshift, uint32_t w0)
{
    const uint32_t e = __ldg(guide + (w0 >> gshift));
    if (!(e & 0x80000000u)) return e;
    int lo = (int)(e & 0x7FFFu);
    int hi = lo + (int)((e >> 15) & 0x7FFFu);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&pairs[mid].x) <= w0)
            lo = mid + 1;
        else
            hi = mid;
    }
    return __ldg(&pairs[lo].y);
}

// Alias draw (Sec. Methodology, "The Alias Method"): one load of column
// j = w0 >> (32 - n); the column's own cell when (w0 << n) mod 2^32 < Prob_j,
// else its alias.  Returns the cell as (a << 16) | b.
__device__ __forceinline__ uint32_t sample_alias(const uint2 *col, int nbits, int tbits, uint32_t w0)
{
    const uint32_t j = w0 >> (32 - nbits);
    const uint2 e = __ldg(col + j);
    if ((w0 << nbits) < e.x) return ((j >> tbits) << 16) | (j & ((1u << tbits) - 1u));
    return e.y;
}

// sin(t) and 1 - cos(t).  For |t| <= 0.5 (every scattering angle of the
// stored histograms in practice) the Maclaurin series, truncated after the
// t^9 and t^10 terms (remainders below 2e-11 relative), evaluated in Horner
// form; beyond that sincosf.
__device__ __forceinline__ void sin_omc(float t, float &s, float &omc)
{
    const float t2 = t * t;
    if (t2 <= 0.25f) {
        s = t * fmaf(-t2 * (1.0f / 6.0f), fmaf(-t2 * (1.0f / 20.0f), fmaf(-t2 * (1.0f / 42.0f),
                     fmaf(-t2, 1.0f / 72.0f, 1.0f), 1.0f), 1.0f), 1.0f);
        omc = 0.5f * t2 * fmaf(-t2 * (1.0f / 12.0f), fmaf(-t2 * (1.0f / 30.0f), fmaf(-t2 * (1.0f / 56.0f),
                               fmaf(-t2, 1.0f / 90.0f, 1.0f), 1.0f), 1.0f), 1.0f);
    } else {
        float c;
        sincosf(t, &s, &c);
        omc = s * s / (1.0f + c);
    }
}

// Coefficients of the scattering update p <- (1 + c1) p + P c2 t^ (see
// scatter) from a sampled cell.  Linear axes (f = dp/p, theta):
// c1 = (1 - f) cos(theta) - 1 and c2 = (1 - f) sin(theta), so |p| becomes
// (1 - f) P at angle theta.  Log axes (f = -dPz/P, t = dPt/P, the paper's
// histogram variables): c1 = -f and c2 = t, Algorithm 1's dz = -P f and
// dt = P t added as they are.
__device__ __forceinline__ void coeffs_angle(float f, float theta, float &c1, float &c2)
{
    float st, omc;
    sin_omc(theta, st, omc);
    c1 = -fmaf(f, 1.0f - omc, omc);
    c2 = (1.0f - f) * st;
}

// Value at cell a + jitter u of a log-spaced axis with lower edge v0 and
// log2 cell width d: v0 2^((a + u) d).  a d is split off exactly (d held as
// hi + lo, the product as a pair) and its integer part applied by ldexpf, so
// exp2f sees only a fraction below ~2 and the value carries ~1e-7 relative
// error (a plain FP32 exponent of up to ~33 would carry ~2e-6).
// h = (v0, d hi, d lo, -).
__device__ __forceinline__ float log_axis_value(float4 h, int a, float u)
{
    const float fa = (float)a;
    const float p = fa * h.y;
    const float e = fmaf(fa, h.z, fmaf(fa, h.y, -p));
    const float n = floorf(p);
    const float r = fmaf(u, h.y, (p - n) + e);
    return ldexpf(h.x * exp2f(r), (int)n);
}

// Eq. 3: p <- p + Rot(dp) with dp = [dt cos phi, dt sin phi, dz] in the frame whose
// z axis is p^.  Written as p <- p + c1 p + P c2 t, with dz = P c1 and dt = P c2,
// where t = R x^ cos(phi) + R y^ sin(phi) is the rotated transverse unit vector
// (R: the Rodrigues rotation taking z^ to p^).  The whole increment is small,
// so it is accumulated into the hi + lo momentum.  Returns 1/|p| before the
// update.  g = 1/(1 + uz) scales only the transverse kick (|c2| <~ 1e-2 of |p|),
// so its 2-ulp fast reciprocal moves p by ~1e-9 relative at most.
__device__ __forceinline__ float scatter(State &s, float c1, float c2, float cphi, float sphi)
{
    const float P2 = p2_of(s);
    float rP = rsqrtf(P2);
    rP = rP * fmaf(-0.5f * P2 * rP, rP, 1.5f);
    const float P = P2 * rP;
    const float ux = s.px * rP, uy = s.py * rP, uz = s.pz * rP;
    const float kick = P * c2;
    const float s2 = fmaf(ux, ux, uy * uy);
    float tx, ty, tz;
    if (uz < 0.0f && s2 < 1e-24f) {                   // p^ = -z^: R = diag(1,-1,-1)
        tx = cphi;
        ty = -sphi;
        tz = 0.0f;
    } else {
        // 1/(1+uz); for uz < 0, (1 - uz)/s2 avoids the cancellation in 1 + uz
        const float g = __fdividef(uz >= 0.0f ? 1.0f : 1.0f - uz, uz >= 0.0f ? 1.0f + uz : s2);
        const float wv = fmaf(cphi, ux, sphi * uy);
        tx = fmaf(-(ux * wv), g, cphi);
        ty = fmaf(-(uy * wv), g, sphi);
        tz = -wv;
    }
    acc(s.px, s.pxl, fmaf(c1, s.px, kick * tx));
    acc(s.py, s.pyl, fmaf(c1, s.py, kick * ty));
    acc(s.pz, s.pzl, fmaf(c1, s.pz, kick * tz));
    return rP;
}

// a + t (b - a)
__device__ __forceinline__ float lerp(float t, float a, float b) { return fmaf(t, b - a, a); }

// Cell index and in-cell fraction of one axis of the node map, from the
// position in cell units (uh + ul): the cell is floor(uh) (the last cell at the
// far node) and the fraction (uh - i) + ul, whose subtraction is exact, so the
// fraction carries the position's full ~1e-14 relative precision however far
// the cell is from the origin.  False outside [0, n - 1].  (When uh is a whole
// number and ul < 0 the fraction is a hair below 0 in the upper cell: the
// trilinear value is continuous across the face, so this is the same value.)
__device__ __forceinline__ bool cell_axis(float uh, float ul, int n, int &i, float &t)
{
    if (!(uh >= 0.0f && uh <= (float)(n - 1))) return false;
    i = min(__float2int_rd(uh), n - 2);
    t = (uh - (float)i) + ul;
    return true;
}

// One x-adjacent node pair (two float4, 32 bytes, 32-byte aligned) of the
// read-only field map.  With MT_FIELD_V8 the pair is one 256-bit load, which
// takes one L1 wavefront per lane where two 128-bit loads take two (the
// scattered corner gathers keep the L1/TEX pipeline at ~85 % of its peak).
#ifndef MT_FIELD_V8
#define MT_FIELD_V8 1
#endif
__device__ __forceinline__ void load_pair(const float4 *p, float4 &a, float4 &b)
{
#if MT_FIELD_V8
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
#else
    a = __ldg(p);
    b = __ldg(p + 1);
#endif
}

// Trilinear value as the weighted sum of the eight corners (1: measured 1.5 %
// faster on shield1e6 than nested lerps, 0).
#ifndef MT_TRILINEAR_WEIGHTS
#define MT_TRILINEAR_WEIGHTS 1
#endif

// Trilinear field from the pair layout; zero outside the node box.
__device__ __forceinline__ float3 field_map(const WorldParams &w, const State &s)
{
    const int nx = w.fdims[0], ny = w.fdims[1], nz = w.fdims[2];
    int i, j, k;
    float tx, ty, tz;
    if (!cell_axis(s.x, s.xl, nx, i, tx) || !cell_axis(s.y, s.yl, ny, j, ty) || !cell_axis(s.z, s.zl, nz, k, tz))
        return make_float3(0.0f, 0.0f, 0.0f);
    const int64_t row = nx - 1;
    const float4 *p00 = w.fmap + 2 * (((int64_t)k * ny + j) * row + i);
    const float4 *p10 = p00 + 2 * row;                 // j + 1
    const float4 *p01 = p00 + 2 * row * ny;            // k + 1
    const float4 *p11 = p01 + 2 * row;                 // j + 1, k + 1
    float4 a0, a1, b0, b1, c0, c1, d0, d1;
    load_pair(p00, a0, a1);
    load_pair(p10, b0, b1);
    load_pair(p01, c0, c1);
    load_pair(p11, d0, d1);
#if MT_TRILINEAR_WEIGHTS
    const float ux = 1.0f - tx, uy = 1.0f - ty, uz = 1.0f - tz;
    const float w00 = uy * uz, w10 = ty * uz, w01 = uy * tz, w11 = ty * tz;
    const float wa0 = ux * w00, wa1 = tx * w00, wb0 = ux * w10, wb1 = tx * w10;
    const float wc0 = ux * w01, wc1 = tx * w01, wd0 = ux * w11, wd1 = tx * w11;
#define MT_TRI(c)                                                                                              \
    fmaf(wd1, d1.c, fmaf(wd0, d0.c, fmaf(wc1, c1.c, fmaf(wc0, c0.c, fmaf(wb1, b1.c, fmaf(wb0, b0.c,             \
                                                                                      fmaf(wa1, a1.c, wa0 * a0.c)))))))
    return make_float3(MT_TRI(x), MT_TRI(y), MT_TRI(z));
#undef MT_TRI
#endif
    const float ax = lerp(tx, a0.x, a1.x), ay = lerp(tx, a0.y, a1.y), az = lerp(tx, a0.z, a1.z);
    const float bx = lerp(tx, b0.x, b1.x), by = lerp(tx, b0.y, b1.y), bz = lerp(tx, b0.z, b1.z);
    const float cx = lerp(tx, c0.x, c1.x), cy = lerp(tx, c0.y, c1.y), cz = lerp(tx, c0.z, c1.z);
    const float dx = lerp(tx, d0.x, d1.x), dy = lerp(tx, d0.y, d1.y), dz = lerp(tx, d0.z, d1.z);
    const float ex = lerp(ty, ax, bx), ey = lerp(ty, ay, by), ez = lerp(ty, az, bz);
    const float gx = lerp(ty, cx, dx), gy = lerp(ty, cy, dy), gz = lerp(ty, cz, dz);
    return make_float3(lerp(tz, ex, gx), lerp(tz, ey, gy), lerp(tz, ez, gz));
}

// o = a x h
__device__ __forceinline__ void cross_h(float ax, float ay, float az, float hx, float hy, float hz, float &ox,
                                        float &oy, float &oz)
{
    ox = fmaf(ay, hz, -(az * hy));
    oy = fmaf(az, hx, -(ax * hz));
    oz = fmaf(ax, hy, -(ay * hx));
}

// RK4 over path length d with B fixed: dr/ds = p/P0, dp/ds = kappa q (p x B)/P0.
// kd = kappa d, rounded once on the host.  With h = kappa q d B / P0 the stage increments are k_i = p_i x h, and the
// position increment reduces to (d/P0) (p + (k1 + k2 + k3)/6).
//
// With B and P0 held, the momentum equation is linear, p' = L p with L v = v x h
// per unit step, and the four stages combine to the degree-4 Taylor polynomial of
// exp(L): dp = (L + L^2/2 + L^3/6 + L^4/24) p and dr = (d/P0)(p + L p/2 + L^2 p/6
// + L^3 p/24) (k1 = Lp, k2 = Lp + L^2p/2, k3 = Lp + L^2p/2 + L^3p/4, k4 = Lp + L^2p
// + L^3p/2 + L^4p/4).  In Horner form w = p + L(p/2 + L(p/6 + Lp/24)) gives
// dr = (d/P0) w and dp = L w: four cross products and no stage sums.  This is the
// same map as the stage form in exact arithmetic, with fewer roundings (against
// an FP64 stage-form transport: smaller position errors; and 2% less time per step).
// Position increment dr (metres) in frame units: dr (1/s) with 1/s held as a
// hi + lo pair, so the frame adds no systematic scale error to the track (a
// float 1/s alone would stretch every step by up to 3e-8).
__device__ __forceinline__ float to_units(float dr, float ih, float il) { return fmaf(dr, ih, dr * il); }

// rP0 = 1/P0 when the caller knows it (> 0), else it is computed from p.  w:
// the world, for its position frame.
__device__ __forceinline__ void rk4(State &s, float3 B, float q, float d, float kd, float rP0, const WorldParams &w)
{
    const float px = s.px, py = s.py, pz = s.pz;
    float rP = rP0;
    if (!(rP > 0.0f)) {
        const float P2 = p2_of(s);
        rP = rsqrtf(P2);
        rP = rP * fmaf(-0.5f * P2 * rP, rP, 1.5f);
    }
    const float c = (kd * q) * rP;
    const float hx = c * B.x, hy = c * B.y, hz = c * B.z;
    float ax, ay, az, bx, by, bz;
    cross_h(px, py, pz, hx, hy, hz, ax, ay, az);                                  // L p
    cross_h(fmaf(ax, 1.0f / 24.0f, px * (1.0f / 6.0f)), fmaf(ay, 1.0f / 24.0f, py * (1.0f / 6.0f)),
            fmaf(az, 1.0f / 24.0f, pz * (1.0f / 6.0f)), hx, hy, hz, bx, by, bz);   // L (p/6 + Lp/24)
    cross_h(fmaf(0.5f, px, bx), fmaf(0.5f, py, by), fmaf(0.5f, pz, bz), hx, hy, hz, ax, ay, az);
    const float wx = px + ax, wy = py + ay, wz = pz + az;                           // w
    cross_h(wx, wy, wz, hx, hy, hz, bx, by, bz);                                  // L w
    const float a = d * rP;
    acc(s.x, s.xl, to_units(a * wx, w.fri_h[0], w.fri_l[0]));
    acc(s.y, s.yl, to_units(a * wy, w.fri_h[1], w.fri_l[1]));
    acc(s.z, s.zl, to_units(a * wz, w.fri_h[2], w.fri_l[2]));
    acc(s.px, s.pxl, bx);
    acc(s.py, s.pyl, by);
    acc(s.pz, s.pzl, bz);
}

// RK4 with the field read at each stage's position (variant of the step, see
// mt_field_desc.per_stage): B1 is the scaled field at the step's start and sc
// the block scale applied to the later stages.  Stage positions r + (d/2) p/P0,
// r + (d/2) p2/P0 and r + d p3/P0 are formed as normalised hi + lo pairs (the
// map lookup takes its cell from the hi word).  The updates are those of rk4
// with h_i from each stage's field.
__device__ __forceinline__ void stage_at(State &t, const State &s, float ax, float ay, float az, float px, float py,
                                         float pz)
{
    two_sum(s.x, fmaf(ax, px, s.xl), t.x, t.xl);
    two_sum(s.y, fmaf(ay, py, s.yl), t.y, t.yl);
    two_sum(s.z, fmaf(az, pz, s.zl), t.z, t.zl);
}

__device__ __forceinline__ void rk4_staged(const WorldParams &w, State &s, float3 B1, float3 sc, float q, float d,
                                           float kd)
{
    const float px = s.px, py = s.py, pz = s.pz;
    const float P2 = p2_of(s);
    float rP = rsqrtf(P2);
    rP = rP * fmaf(-0.5f * P2 * rP, rP, 1.5f);
    const float c = (kd * q) * rP;
    const float a = d * rP;
    float k1x, k1y, k1z, k2x, k2y, k2z, k3x, k3y, k3z, k4x, k4y, k4z;
    cross_h(px, py, pz, c * B1.x, c * B1.y, c * B1.z, k1x, k1y, k1z);
    State t = s;
    const float ax = a * w.fri_h[0], ay = a * w.fri_h[1], az = a * w.fri_h[2];   // metres -> frame units
    stage_at(t, s, 0.5f * ax, 0.5f * ay, 0.5f * az, px, py, pz);
    float3 B = field_map(w, t);
    const float p2x = fmaf(0.5f, k1x, px), p2y = fmaf(0.5f, k1y, py), p2z = fmaf(0.5f, k1z, pz);
    cross_h(p2x, p2y, p2z, c * (sc.x * B.x), c * (sc.y * B.y), c * (sc.z * B.z), k2x, k2y, k2z);
    stage_at(t, s, 0.5f * ax, 0.5f * ay, 0.5f * az, p2x, p2y, p2z);
    B = field_map(w, t);
    const float p3x = fmaf(0.5f, k2x, px), p3y = fmaf(0.5f, k2y, py), p3z = fmaf(0.5f, k2z, pz);
    cross_h(p3x, p3y, p3z, c * (sc.x * B.x), c * (sc.y * B.y), c * (sc.z * B.z), k3x, k3y, k3z);
    stage_at(t, s, ax, ay, az, p3x, p3y, p3z);
    B = field_map(w, t);
    cross_h(px + k3x, py + k3y, pz + k3z, c * (sc.x * B.x), c * (sc.y * B.y), c * (sc.z * B.z), k4x, k4y, k4z);
    const float sixth = 1.0f / 6.0f;
    acc(s.x, s.xl, to_units(a * fmaf(sixth, k1x + k2x + k3x, px), w.fri_h[0], w.fri_l[0]));
    acc(s.y, s.yl, to_units(a * fmaf(sixth, k1y + k2y + k3y, py), w.fri_h[1], w.fri_l[1]));
    acc(s.z, s.zl, to_units(a * fmaf(sixth, k1z + k2z + k3z, pz), w.fri_h[2], w.fri_l[2]));
    acc(s.px, s.pxl, sixth * (k1x + 2.0f * (k2x + k3x) + k4x));
    acc(s.py, s.pyl, sixth * (k1y + 2.0f * (k2y + k3y) + k4y));
    acc(s.pz, s.pzl, sixth * (k1z + 2.0f * (k2z + k3z) + k4z));
}

// (xh + xl) <= (bh + bl) for normalised pairs.
__device__ __forceinline__ bool le2(float xh, float xl, float bh, float bl)
{
    return xh < bh || (xh == bh && xl <= bl);
}

// Termination test of Algorithm 1 at the start of a step.  |x| >= x_max in
// metres is x >= xmax or x <= xmin in frame units.
__device__ __forceinline__ int check_stop(const WorldParams &w, const State &s, float P2)
{
    if (P2 < w.pmin2) return MT_STOPPED;
    // strictly inside on the hi words: no pair test below can fire
    if (s.z < w.zmax_hi && s.x < w.xmax_hi && s.x > w.xmin_hi && s.y < w.ymax_hi && s.y > w.ymin_hi)
        return MT_ALIVE;
    if (ge2(s.z, s.zl, w.zmax_hi, w.zmax_lo)) return MT_EXIT_Z;
    if (ge2(s.x, s.xl, w.xmax_hi, w.xmax_lo) || le2(s.x, s.xl, w.xmin_hi, w.xmin_lo) ||
        ge2(s.y, s.yl, w.ymax_hi, w.ymax_lo) || le2(s.y, s.yl, w.ymin_hi, w.ymin_lo))
        return MT_EXIT_XY;
    return MT_ALIVE;
}

// Recorder hooks of step(): the plain kernels pass NoRecord (every hook
// compiles away); the adjoint's recompute passes a tape writer, so the tape
// comes from exactly the arithmetic of the forward pass.
struct NoRecord {
    __device__ __forceinline__ void begin(const State &, int, bool) {}
    __device__ __forceinline__ void draw(const State &, float, float, float) {}
    __device__ __forceinline__ void field(float3) {}
};

// One full step k of Algorithm 1 for the muon with id (id_hi, id_lo) of
// instance inst (the Philox counter's words).  Returns MT_ALIVE or the break
// status.  RK: Philox takes its round keys from rp.rk (measured faster in the
// compaction passes) or advances them from rp.key0/key1 (faster in the
// batched pass); both give the same words.
template <int GEOM, int FIELD, class Rec = NoRecord, bool RK = true>
__device__ __forceinline__ int step(const WorldParams &w, const SmemWorld &sw, State &s, float q, int k,
                                    uint32_t id_lo, uint32_t id_hi, uint32_t inst, const RunParams &rp,
                                    Rec &&rec = Rec())
{
    const float P2 = fmaf(s.px, s.px, fmaf(s.py, s.py, s.pz * s.pz));
    const int stop = check_stop(w, s, P2);
    if (stop != MT_ALIVE) return stop;
    int box = -1, mat;
    if (GEOM == MT_GEOM_BOXES) {
        box = find_box(w, sw, s);
        mat = box >= 0 ? sw.mat[box] : w.world_mat;
    } else if (GEOM == MT_GEOM_POLYHEDRA) {
        box = find_solid(w, sw, s);
        mat = box >= 0 ? sw.mat[box] : w.world_mat;
    } else {
        const int vm = voxel_material(w, s);
        mat = vm >= 0 ? vm : w.world_mat;
    }
    rec.begin(s, box, mat != 0);
    // 1/P0 for the RK4 step when scattering set it: on the linear axes the
    // update leaves |p| = (1 - f) P exactly (c1 and c2 are built so), so
    // 1/P0 = (1/P) / (1 - f) and |p| need not be formed again
    float rP0 = 0.0f;
    if (mat != 0) {
        const int ib = momentum_bin(w, sw, s, P2);
        const uint4 ctr = make_uint4((uint32_t)k, id_lo, id_hi, inst);
        const uint4 rnd = RK ? philox4x32_10(ctr, rp.rk) : philox4x32_10(ctr, rp.key0, rp.key1);
        // the guide (or alias) row of histogram h sits at h * its length, so its
        // load need not wait for the histogram record's
        const int h = (mat - 1) * w.n_pbin + ib;
        HistRec hr;
        if (w.n_mat * w.n_pbin <= kHistSmem) {
            hr = sw.hist[h];
        } else {
            const uint4 hraw = __ldg(reinterpret_cast<const uint4 *>(w.hist + h));
            hr = {hraw.x, hraw.y, __uint_as_float(hraw.z), __uint_as_float(hraw.w)};
        }
        const uint32_t ab =
            w.sampler == MT_SAMPLER_ALIAS
                ? sample_alias(w.alias + ((int64_t)h << w.alias_bits), w.alias_bits, w.theta_bits, rnd.x)
                : sample_cell(w.guide + ((int64_t)h << (32 - w.gshift)), w.pairs + hr.pair_off, w.gshift, rnd.x);
        const float f = ((float)(ab >> 16) + u01(rnd.y)) * hr.fscale;
        const float th = ((float)(ab & 0xFFFFu) + u01(rnd.z)) * hr.tscale;
        const float phs = fmaf(6.283185307179586f, u01(rnd.w), -3.14159265358979f);   // phi - pi
        float sp, cp;
        __sincosf(phs, &sp, &cp);
        float c1, c2;
        if (w.axes == MT_AXES_LOG) {
            // f and t log-spaced: cell + jitter in log f, log t (the cell's
            // linear values f, th above are not used)
            const float4 *hl = w.hist_log + 2 * ((mat - 1) * w.n_pbin + ib);
            const float4 hf = __ldg(hl), ht = __ldg(hl + 1);
            c1 = -log_axis_value(hf, (int)(ab >> 16), u01(rnd.y));
            c2 = log_axis_value(ht, (int)(ab & 0xFFFFu), u01(rnd.z));
        } else {
            coeffs_angle(f, th, c1, c2);
        }
        rec.draw(s, c1, c2, phs);   // s: the momentum before scattering
        const float rP = scatter(s, c1, c2, -cp, -sp);
        if (w.axes != MT_AXES_LOG) rP0 = __fdividef(rP, 1.0f - f);
    }
    float3 B = make_float3(0.0f, 0.0f, 0.0f);
    if (FIELD == MT_FIELD_BOX) {
        if (box >= 0) B = make_float3(sw.B[0][box], sw.B[1][box], sw.B[2][box]);
    } else if (FIELD == MT_FIELD_MAP || FIELD == kFieldMapStaged) {
        B = field_map(w, s);
    } else if (FIELD == MT_FIELD_MAP_NEAREST) {
        B = field_map_nearest(w, s);
    }
    rec.field(B);   // before the block scale
    float3 sc = make_float3(1.0f, 1.0f, 1.0f);
    if (GEOM != MT_GEOM_VOXELS && FIELD != MT_FIELD_NONE && box >= 0) {
        const int blk = sw.block[box];
        if (blk >= 0) {
            sc = make_float3(sw.alpha[0][blk], sw.alpha[1][blk], sw.alpha[2][blk]);
            B.x *= sc.x;
            B.y *= sc.y;
            B.z *= sc.z;
        }
    }
    if (FIELD == kFieldMapStaged)
        rk4_staged(w, s, B, sc, q, rp.d, rp.kd);
    else
        rk4(s, B, q, rp.d, rp.kd, rP0, w);
    return MT_ALIVE;
}

// Metres -> frame units: u = (x - o) / s as a hi + lo pair, from the exact
// difference x - oh (two_sum) and a double-float product with 1/s (~1e-14
// relative).  With o = 0 and s = 1 it returns (x, 0) exactly.
__device__ __forceinline__ void to_frame(float x, float oh, float ol, float ih, float il, float &uh, float &ul)
{
    float dh, de;
    two_sum(x, -oh, dh, de);
    const float dl = de - ol;
    const float p = dh * ih;
    const float e = fmaf(dh, il, fmaf(dl, ih, fmaf(dh, ih, -p)));
    uh = p + e;
    ul = e - (uh - p);
}

// Frame units -> metres: o + u s from the hi + lo pairs, rounded once at the
// end; with o = 0 and s = 1 it returns uh + ul, the plain sum of the pair.
__device__ __forceinline__ float from_frame(float uh, float ul, float oh, float ol, float sh, float sl)
{
    const float p = uh * sh;
    const float e = fmaf(uh, sl, fmaf(ul, sh, fmaf(uh, sh, -p)));
    float th, te;
    two_sum(oh, p, th, te);
    return th + ((te + e) + ol);
}

// Load muon m into registers (position converted to the world's frame).
// Returns false (and handles the muon) when there is nothing to transport: a
// terminal status is left as it is, a non-finite state is marked MT_INVALID.
__device__ __forceinline__ bool load_muon(const WorldParams &w, const mt_muon_soa &soa, int64_t m,
                                          const RunParams &rp, State &s, float &q, int &k, uint32_t &id_lo,
                                          uint32_t &id_hi)
{
    const uint8_t st0 = soa.status[m];
    if (st0 != MT_ALIVE && st0 != MT_MAX_STEPS) return false;
    const float x = soa.x[m], y = soa.y[m], z = soa.z[m];
    s.px = soa.px[m];
    s.py = soa.py[m];
    s.pz = soa.pz[m];
    s.pxl = s.pyl = s.pzl = 0.0f;
    if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(s.px) && isfinite(s.py) && isfinite(s.pz))) {
        soa.status[m] = MT_INVALID;
        return false;
    }
    to_frame(x, w.fro_h[0], w.fro_l[0], w.fri_h[0], w.fri_l[0], s.x, s.xl);
    to_frame(y, w.fro_h[1], w.fro_l[1], w.fri_h[1], w.fri_l[1], s.y, s.yl);
    to_frame(z, w.fro_h[2], w.fro_l[2], w.fri_h[2], w.fri_l[2], s.z, s.zl);
    q = (float)soa.q[m];
    k = soa.steps[m];
    const uint64_t id = (uint64_t)(rp.id_offset + m);
    id_lo = (uint32_t)id;
    id_hi = (uint32_t)(id >> 32);
    return true;
}

__device__ __forceinline__ void store_muon(const WorldParams &w, const mt_muon_soa &soa, int64_t m, const State &s,
                                           int k, int status)
{
    soa.x[m] = from_frame(s.x, s.xl, w.fro_h[0], w.fro_l[0], w.frs_h[0], w.frs_l[0]);
    soa.y[m] = from_frame(s.y, s.yl, w.fro_h[1], w.fro_l[1], w.frs_h[1], w.frs_l[1]);
    soa.z[m] = from_frame(s.z, s.zl, w.fro_h[2], w.fro_l[2], w.frs_h[2], w.frs_l[2]);
    soa.px[m] = s.px + s.pxl;
    soa.py[m] = s.py + s.pyl;
    soa.pz[m] = s.pz + s.pzl;
    soa.steps[m] = k;
    soa.status[m] = (uint8_t)status;
}

// Live-list entries of the compacting kernels (64 B per muon, four 16-byte
// words in structure-of-arrays order): w0 = (x, y, z, q), w1 = (px, py, pz, k),
// w2 = (xl, yl, zl, idx), w3 = (pxl, pyl, pzl, 0), the position in the world's
// frame.
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

// tag: the fourth word of w3 (the entry's rank within its key in the compacting
// transport's spatial order; 0 elsewhere).
__device__ __forceinline__ void put_live(const LiveBuf &b, int64_t i, const State &s, float q, int k, int64_t idx,
                                         unsigned tag = 0u)
{
    b.w0[i] = make_float4(s.x, s.y, s.z, q);
    b.w1[i] = make_float4(s.px, s.py, s.pz, __int_as_float(k));
    b.w2[i] = make_float4(s.xl, s.yl, s.zl, __int_as_float((int)idx));
    b.w3[i] = make_float4(s.pxl, s.pyl, s.pzl, __uint_as_float(tag));
}

__device__ __forceinline__ void get_live(const LiveBuf &b, int64_t i, State &s, float &q, int &k, int64_t &idx)
{
    const float4 a = b.w0[i], c = b.w1[i], e = b.w2[i], g = b.w3[i];
    s.x = a.x; s.y = a.y; s.z = a.z; q = a.w;
    s.px = c.x; s.py = c.y; s.pz = c.z; k = __float_as_int(c.w);
    s.xl = e.x; s.yl = e.y; s.zl = e.z; idx = __float_as_int(e.w);
    s.pxl = g.x; s.pyl = g.y; s.pzl = g.z;
}

}  // namespace mt
