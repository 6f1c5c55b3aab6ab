// adjoint.cu -- the differentiable form: pathwise gradients of a loss of the
// final muon states with respect to per-magnet field scales alpha[block][c].
//
// The paper's Discussion proposes making the histogram transport a
// differentiable layer.  Here every random choice of a step (material, box,
// momentum bin, cell, f, theta, phi) and every muon's step count are held
// fixed (common random numbers), and the derivative of the remaining smooth
// map -- scattering rotation (Eq. 3), trilinear field (with dB/dr) and the RK4
// step of Eq. 4 -- is propagated backwards by hand-written adjoints.
//
// Forward (mt_transport_ckpt): the compacting transport with a pass length of
// K = ckpt_every steps whose live lists are all kept: the list that enters
// pass p is the checkpoint of every muon alive at step p K.
// Backward (mt_adjoint_ckpt): passes in reverse order; for pass p, a recorded
// pass recomputes each live muon's (at most K) steps from the checkpoint with
// the forward's own step function, writing a tape of the pass, and a reverse
// pass walks the tape backwards, carrying (dL/dr, dL/dp) in a per-muon buffer
// from pass to pass and accumulating dL/dalpha.
// Full-tape form (mt_transport_tape / mt_adjoint_tape): the forward's passes
// record their tapes directly (every pass kept), so the backward only runs
// the reverse passes.
//
// Checkpoint buffer: [ counts | dL/dalpha | list 0 | list 1 | ... | list P ]:
// P + 1 live counts (uint64), the dL/dalpha accumulator (double
// [MT_MAX_BOXES][3]), then P + 1 live lists of four float4 arrays of n entries
// (step.cuh), each section 256-byte aligned, P = ceil(max_steps / K).  The
// tape buffer appends the tape region offsets, a flag and the tape region.
#include <cstdio>
#include <vector>

#include "compact.cuh"

namespace mt {

constexpr int kTapeMax = 64;

// Resident blocks per SM of the reverse pass: 4 blocks of 256 (64 registers, no
// spill since the step's divides became fast reciprocals; measured on diff1e6,
// K = 32: backward 52.8 ms against 53.8 ms at 3 blocks and 80 registers).
#ifndef MT_ADJ_MIN_BLOCKS
#define MT_ADJ_MIN_BLOCKS 4
#endif

__host__ __device__ inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

struct CkptLayout {
    int passes;
    int64_t alpha_off, sort_off, lists_off, list_bytes, total;
};

static CkptLayout ckpt_layout(int64_t n, int32_t max_steps, int32_t K)
{
    CkptLayout L;
    const int64_t cap = n > 0 ? n : 1;
    L.passes = max_steps > 0 ? (max_steps + K - 1) / K : 1;
    // live counts of every pass, then the passes' work counters; dL/dalpha; the
    // spatial order's counts and first slots; the live list of every pass
    L.alpha_off = round_up((int64_t)(L.passes + 1) * 16, 256);
    L.sort_off = round_up(L.alpha_off + 3 * MT_MAX_BOXES * 8, 256);
    L.lists_off = round_up(L.sort_off + 2 * (int64_t)kSortBins * (int64_t)sizeof(unsigned), 256);
    L.list_bytes = 4 * cap * (int64_t)sizeof(float4);
    L.total = L.lists_off + (L.passes + 1) * L.list_bytes;
    return L;
}

// Tape buffer of the full-tape form: a checkpoint buffer (above) followed by
// the region offsets of every pass (uint64 [P + 1]), an overflow flag and the
// tape region, sized for n muons alive through every pass.
struct TapeLayout {
    CkptLayout ck;
    int64_t off_off, flag_off, region_off, region_cap, total;
};

// Whether the tape holds the field at each step (16 more bytes per step) or
// the reverse sweep evaluates it again at the recorded r (measured on diff1e6:
// recording is faster, 38 against 54 ms for the backward).
#ifndef MT_TAPE_RECORD_B
#define MT_TAPE_RECORD_B 1
#endif

// bytes of one recorded step
__host__ __device__ constexpr int64_t tape_step_bytes(bool rb) { return rb ? 56 : 40; }

__host__ __device__ inline int64_t tape_pass_bytes(int64_t count, int K)
{
    return round_up(tape_step_bytes(MT_TAPE_RECORD_B) * K * round_up(count, 32), 256);
}

static TapeLayout tape_layout(int64_t n, int32_t max_steps, int32_t K)
{
    TapeLayout T;
    T.ck = ckpt_layout(n, max_steps, K);
    T.off_off = T.ck.total;
    T.flag_off = round_up(T.off_off + (int64_t)(T.ck.passes + 1) * 8, 256);
    T.region_off = T.flag_off + 256;
    T.region_cap = (int64_t)T.ck.passes * tape_pass_bytes(n > 0 ? n : 1, K);
    T.total = T.region_off + T.region_cap;
    return T;
}

// One recorded step takes 40 (or 56) bytes in three (four) planes, so that a
// warp's stores and loads are contiguous: plane a = (rx, ry, rz, meta), plane
// b = (px, py, pz, c1), plane c = (c2, phi - pi), plane d = (Bx, By, Bz, -)
// when the field is recorded, with r (in the world's frame units) and p at the
// step's start, (c1, c2) the
// coefficients of the scattering update (step.cuh: scatter), B there before
// the block scale, and meta bit 0 = scattered, bits 8..15 = box + 1.  Step j of
// entry t sits at base + step_bytes j T (T entries per plane, a multiple of
// 32).  Written and read once with streaming (evict-first) hints, so it passes
// through L2 without pushing out the field map.
template <bool RB>
struct TapeRef {
    char *base;
    int64_t T;
    int64_t tid;
    __device__ __forceinline__ char *row(int j) const { return base + tape_step_bytes(RB) * (int64_t)j * T; }
    __device__ __forceinline__ float4 *a(int j) const { return reinterpret_cast<float4 *>(row(j)) + tid; }
    __device__ __forceinline__ float4 *b(int j) const { return reinterpret_cast<float4 *>(row(j) + 16 * T) + tid; }
    __device__ __forceinline__ float2 *c(int j) const { return reinterpret_cast<float2 *>(row(j) + 32 * T) + tid; }
    __device__ __forceinline__ float4 *d(int j) const { return reinterpret_cast<float4 *>(row(j) + 40 * T) + tid; }
};

// Each plane is stored as soon as its values exist, so the recorder holds no
// values across the step: a at the step's start (and b there too when the step
// does not scatter), b and c at the draw, d at the field lookup.
template <bool RB>
struct TapeWriter {
    const TapeRef<RB> *tr;
    int j;
    bool on = true;
    __device__ __forceinline__ void begin(const State &s, int box, bool scattered)
    {
        if (!on) return;
        const int meta = ((box + 1) << 8) | (scattered ? 1 : 0);
        __stcs(tr->a(j), make_float4(s.x + s.xl, s.y + s.yl, s.z + s.zl, __int_as_float(meta)));
        if (!scattered) __stcs(tr->b(j), make_float4(s.px + s.pxl, s.py + s.pyl, s.pz + s.pzl, 0.0f));
    }
    __device__ __forceinline__ void draw(const State &s, float c1, float c2, float phs)
    {
        if (!on) return;
        __stcs(tr->b(j), make_float4(s.px + s.pxl, s.py + s.pyl, s.pz + s.pzl, c1));
        __stcs(tr->c(j), make_float2(c2, phs));
    }
    __device__ __forceinline__ void field(float3 B)
    {
        if (RB && on) __stcs(tr->d(j), make_float4(B.x, B.y, B.z, 0.0f));
    }
};

struct TapeEntry {
    float4 a, b, d;
    float2 c;
};

// The reverse pass asks L1 for the lines of a lane's next tape step
// (prefetch.global.L1) while it reverses the current one; the prefetch holds no
// register or shared memory (measured on diff1e6: backward 56.0 ms against
// 57.3 ms without; copying the next step into shared memory with cp.async
// instead took 66 ms).
#ifndef MT_ADJ_PREFETCH
#define MT_ADJ_PREFETCH 1
#endif

__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

template <bool RB>
__device__ __forceinline__ TapeEntry load_tape(const TapeRef<RB> &tr, int j)
{
    TapeEntry t;
    t.a = __ldcs(tr.a(j));
    t.b = __ldcs(tr.b(j));
    t.c = (__float_as_int(t.a.w) & 1) ? __ldcs(tr.c(j)) : make_float2(0.0f, 0.0f);
    t.d = RB ? __ldcs(tr.d(j)) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    return t;
}

__device__ __forceinline__ void cross3(const float a[3], const float b[3], float o[3])
{
    o[0] = fmaf(a[1], b[2], -(a[2] * b[1]));
    o[1] = fmaf(a[2], b[0], -(a[0] * b[2]));
    o[2] = fmaf(a[0], b[1], -(a[1] * b[0]));
}

__device__ __forceinline__ float dot3(const float a[3], const float b[3])
{
    return fmaf(a[0], b[0], fmaf(a[1], b[1], a[2] * b[2]));
}

// rb += J(r)^T Bb with J[c][a] = dB_c/dr_a of the unscaled trilinear map (zero
// outside the node box); r in the map's cell units, rb per metre.
__device__ __forceinline__ void field_map_jt(const WorldParams &w, const float r[3], const float Bb[3], float rb[3])
{
    const int nx = w.fdims[0], ny = w.fdims[1], nz = w.fdims[2];
    int i, j, k;
    float tx, ty, tz;
    if (!cell_axis(r[0], 0.0f, nx, i, tx) || !cell_axis(r[1], 0.0f, ny, j, ty) || !cell_axis(r[2], 0.0f, nz, k, tz))
        return;
    const int64_t row = nx - 1;
    const float4 *p00 = w.fmap + 2 * (((int64_t)k * ny + j) * row + i);
    const float4 *p10 = p00 + 2 * row;
    const float4 *p01 = p00 + 2 * row * ny;
    const float4 *p11 = p01 + 2 * row;
    // project the corners on Bb first: v_q = Bb . B(corner q)
    float v[8];
    const float4 *src[4] = {p00, p10, p01, p11};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float4 c, e;
        load_pair(src[q], c, e);
        v[2 * q] = fmaf(Bb[0], c.x, fmaf(Bb[1], c.y, Bb[2] * c.z));
        v[2 * q + 1] = fmaf(Bb[0], e.x, fmaf(Bb[1], e.y, Bb[2] * e.z));
    }
    // v: (i,j,k) (i+1,j,k) (i,j+1,k) (i+1,j+1,k) (i,j,k+1) (i+1,j,k+1) (i,j+1,k+1) (i+1,j+1,k+1)
    const float a = lerp(tx, v[0], v[1]), b = lerp(tx, v[2], v[3]);
    const float cc = lerp(tx, v[4], v[5]), d = lerp(tx, v[6], v[7]);
    rb[0] = fmaf(lerp(tz, lerp(ty, v[1] - v[0], v[3] - v[2]), lerp(ty, v[5] - v[4], v[7] - v[6])), w.finv[0], rb[0]);
    rb[1] = fmaf(lerp(tz, b - a, d - cc), w.finv[1], rb[1]);
    rb[2] = fmaf(lerp(ty, cc, d) - lerp(ty, a, b), w.finv[2], rb[2]);
}

// The forward's scattering update in plain FP32 on a recorded momentum.
__device__ __forceinline__ void scatter_fp32(const float p[3], float c1, float c2, float cphi, float sphi, float ps[3])
{
    const float P2 = dot3(p, p);
    float rP = rsqrtf(P2);
    rP = rP * fmaf(-0.5f * P2 * rP, rP, 1.5f);
    const float P = P2 * rP;
    const float ux = p[0] * rP, uy = p[1] * rP, uz = p[2] * rP;
    const float kick = P * c2;
    const float s2 = fmaf(ux, ux, uy * uy);
    float tx, ty, tz;
    if (uz < 0.0f && s2 < 1e-24f) {
        tx = cphi;
        ty = -sphi;
        tz = 0.0f;
    } else {
        const float g = __fdividef(uz >= 0.0f ? 1.0f : 1.0f - uz, uz >= 0.0f ? 1.0f + uz : s2);   // as scatter
        const float wv = fmaf(cphi, ux, sphi * uy);
        tx = fmaf(-(ux * wv), g, cphi);
        ty = fmaf(-(uy * wv), g, sphi);
        tz = -wv;
    }
    ps[0] = fmaf(c1, p[0], fmaf(kick, tx, p[0]));
    ps[1] = fmaf(c1, p[1], fmaf(kick, ty, p[1]));
    ps[2] = fmaf(c1, p[2], fmaf(kick, tz, p[2]));
}

// dL/dalpha of the current magnet block, flushed to shared memory when the
// muon changes block (rare: it stays in a block for hundreds of steps).
struct AlphaAcc {
    int blk = -1;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
    __device__ __forceinline__ void flush(float (*sacc)[MT_MAX_BOXES])
    {
        if (blk >= 0) {
            atomicAdd(&sacc[0][blk], a0);
            atomicAdd(&sacc[1][blk], a1);
            atomicAdd(&sacc[2][blk], a2);
        }
        a0 = a1 = a2 = 0.0f;
    }
    __device__ __forceinline__ void add(int b, float x, float y, float z, float (*sacc)[MT_MAX_BOXES])
    {
        if (b != blk) {
            flush(sacc);
            blk = b;
        }
        a0 += x;
        a1 += y;
        a2 += z;
    }
};

// Reverse of one forward step recorded in t: (rb, pb) enter as dL/d(r, p) after
// the step and leave as dL/d(r, p) before it.
//
// RK4 for dp/ds = p x w with w fixed (B held over the step) is, exactly, the
// degree-4 Taylor polynomial of the rotation: with h = kappa q d B / P0 and
// v1 = ps x h, v2 = v1 x h, v3 = v2 x h, v4 = v3 x h,
//   p' = ps + v1 + v2/2 + v3/6 + v4/24,  r' = r + (d/P0)(ps + v1/2 + v2/6 + v3/24)
// (the stage form k1..k4 of the forward expands to the same polynomials), so
// its adjoint is taken in that form, which keeps fewer values live.
template <int GEOM, int FIELD, bool RB>
__device__ __forceinline__ void reverse_step(const WorldParams &w, const SmemWorld &sw, const TapeEntry &t, float q,
                                             float d, float kd, float rb[3], float pb[3], AlphaAcc &acc,
                                             float (*sacc)[MT_MAX_BOXES])
{
    const int meta = __float_as_int(t.a.w);
    const int box = (meta >> 8) - 1;
    const bool scat = meta & 1;
    const float r0[3] = {t.a.x, t.a.y, t.a.z};
    const float p0[3] = {t.b.x, t.b.y, t.b.z};
    const float sm10 = t.b.w, kf0 = t.c.x;   // scattering coefficients c1, c2
    // -- field before the block scale, evaluated again at the recorded r
    float Bm[3] = {0.0f, 0.0f, 0.0f};
    if (RB) {
        Bm[0] = t.d.x;
        Bm[1] = t.d.y;
        Bm[2] = t.d.z;
    } else if (FIELD == MT_FIELD_BOX) {
        if (box >= 0) {
            Bm[0] = sw.B[0][box];
            Bm[1] = sw.B[1][box];
            Bm[2] = sw.B[2][box];
        }
    } else if (FIELD == MT_FIELD_MAP || FIELD == MT_FIELD_MAP_NEAREST) {
        State at;
        at.x = r0[0];
        at.y = r0[1];
        at.z = r0[2];
        at.xl = at.yl = at.zl = 0.0f;
        const float3 b = FIELD == MT_FIELD_MAP ? field_map(w, at) : field_map_nearest(w, at);
        Bm[0] = b.x;
        Bm[1] = b.y;
        Bm[2] = b.z;
    }
    float sphi = 0.0f, cphi = 0.0f;
    if (scat) {
        __sincosf(t.c.y, &sphi, &cphi);
        sphi = -sphi;
        cphi = -cphi;
    }
    // -- scattered momentum ps = p + sm1 p + P kf tv(u) (recomputed in FP32)
    float ps[3] = {p0[0], p0[1], p0[2]};
    if (scat) scatter_fp32(p0, sm10, kf0, cphi, sphi, ps);
    int blk = -1;
    float sc[3] = {1.0f, 1.0f, 1.0f};
    if (GEOM != MT_GEOM_VOXELS && FIELD != MT_FIELD_NONE && box >= 0) {
        blk = sw.block[box];
        if (blk >= 0) {
            sc[0] = sw.alpha[0][blk];
            sc[1] = sw.alpha[1][blk];
            sc[2] = sw.alpha[2][blk];
        }
    }
    const float B[3] = {sc[0] * Bm[0], sc[1] * Bm[1], sc[2] * Bm[2]};
    // -- RK4 (Taylor form)
    const float P02 = dot3(ps, ps);
    float rP0 = rsqrtf(P02);
    rP0 = rP0 * fmaf(-0.5f * P02 * rP0, rP0, 1.5f);
    const float cc = (kd * q) * rP0;
    const float a = d * rP0;
    const float h[3] = {cc * B[0], cc * B[1], cc * B[2]};
    float v1[3], v2[3], v3[3];
    cross3(ps, h, v1);
    cross3(v1, h, v2);
    cross3(v2, h, v3);
    float rsum[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
        rsum[c] = fmaf(1.0f / 24.0f, v3[c], fmaf(1.0f / 6.0f, v2[c], fmaf(0.5f, v1[c], ps[c])));
    const float abar = dot3(rb, rsum);
    float vb[3], hb[3] = {0.0f, 0.0f, 0.0f}, tmp[3];
    // v4 = v3 x h: v3b += h x v4b, hb += v4b x v3, with v4b = pb / 24
#pragma unroll
    for (int c = 0; c < 3; ++c) vb[c] = (1.0f / 24.0f) * pb[c];
    cross3(vb, v3, tmp);
#pragma unroll
    for (int c = 0; c < 3; ++c) hb[c] += tmp[c];
    cross3(h, vb, tmp);
    // v3b = pb/6 + a rb/24 + h x v4b;  v3 = v2 x h
#pragma unroll
    for (int c = 0; c < 3; ++c) vb[c] = fmaf(1.0f / 6.0f, pb[c], fmaf(a * (1.0f / 24.0f), rb[c], tmp[c]));
    cross3(vb, v2, tmp);
#pragma unroll
    for (int c = 0; c < 3; ++c) hb[c] += tmp[c];
    cross3(h, vb, tmp);
    // v2b = pb/2 + a rb/6 + h x v3b;  v2 = v1 x h
#pragma unroll
    for (int c = 0; c < 3; ++c) vb[c] = fmaf(0.5f, pb[c], fmaf(a * (1.0f / 6.0f), rb[c], tmp[c]));
    cross3(vb, v1, tmp);
#pragma unroll
    for (int c = 0; c < 3; ++c) hb[c] += tmp[c];
    cross3(h, vb, tmp);
    // v1b = pb + a rb/2 + h x v2b;  v1 = ps x h
#pragma unroll
    for (int c = 0; c < 3; ++c) vb[c] = fmaf(0.5f * a, rb[c], pb[c] + tmp[c]);
    cross3(vb, ps, tmp);
#pragma unroll
    for (int c = 0; c < 3; ++c) hb[c] += tmp[c];
    cross3(h, vb, tmp);
    float psb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) psb[c] = fmaf(a, rb[c], pb[c] + tmp[c]);
    // h = cc B with cc = kappa q d / P0, a = d / P0, P0 = |ps|
    const float ccb = dot3(hb, B);
    const float P0b = -fmaf(ccb, cc, abar * a) * rP0;
#pragma unroll
    for (int c = 0; c < 3; ++c) psb[c] = fmaf(P0b * rP0, ps[c], psb[c]);
    // -- field: B = sc (.) Bm(r)
    const float Bb[3] = {cc * hb[0], cc * hb[1], cc * hb[2]};
    if (blk >= 0) acc.add(blk, Bb[0] * Bm[0], Bb[1] * Bm[1], Bb[2] * Bm[2], sacc);
    if (FIELD == MT_FIELD_MAP) {
        const float Bmb[3] = {sc[0] * Bb[0], sc[1] * Bb[1], sc[2] * Bb[2]};
        field_map_jt(w, r0, Bmb, rb);
    }
    // -- scattering: ps = (1 + sm1) p + P kf tv(u), u = p / P, held draws (sm1, kf, phi)
    const float(&p)[3] = p0;
    const float sm1 = sm10, kf = kf0;
    if (!scat) {
        pb[0] = psb[0];
        pb[1] = psb[1];
        pb[2] = psb[2];
        return;
    }
    const float P2 = dot3(p, p);
    float rPs = rsqrtf(P2);
    rPs = rPs * fmaf(-0.5f * P2 * rPs, rPs, 1.5f);
    const float P = P2 * rPs;
    const float u[3] = {p[0] * rPs, p[1] * rPs, p[2] * rPs};
    const float s2 = fmaf(u[0], u[0], u[1] * u[1]);
    float tv[3], ub[3] = {0.0f, 0.0f, 0.0f};
    if (u[2] < 0.0f && s2 < 1e-24f) {
        tv[0] = cphi;
        tv[1] = -sphi;
        tv[2] = 0.0f;
    } else {
        const float g = __fdividef(u[2] >= 0.0f ? 1.0f : 1.0f - u[2], u[2] >= 0.0f ? 1.0f + u[2] : s2);
        const float wv = fmaf(cphi, u[0], sphi * u[1]);
        tv[0] = fmaf(-(u[0] * wv), g, cphi);
        tv[1] = fmaf(-(u[1] * wv), g, sphi);
        tv[2] = -wv;
        const float kick = P * kf;
        const float tb[3] = {kick * psb[0], kick * psb[1], kick * psb[2]};
        const float sx = fmaf(tb[0], u[0], tb[1] * u[1]);
        const float wb = fmaf(-sx, g, -tb[2]);
        const float gb = -sx * wv;
        ub[0] = fmaf(wb, cphi, -tb[0] * wv * g);
        ub[1] = fmaf(wb, sphi, -tb[1] * wv * g);
        ub[2] = -gb * g * g;
    }
    const float Pb = kf * dot3(tv, psb);
    const float uu = dot3(u, ub);
#pragma unroll
    for (int c = 0; c < 3; ++c) pb[c] = fmaf(1.0f + sm1, psb[c], fmaf(Pb, u[c], fmaf(-u[c], uu, ub[c]) * rPs));
}

// Recorded pass: every live muon of list `in` advances its (at most S) steps
// with the forward's own step function, recording each step into the pass
// tape at column = list entry (T = entries rounded up to 32); the number of
// steps each entry took goes into the spare word of its list entry.  The tape
// region's offset is read from tape_off[0] and its end written to tape_off[1];
// a region that would run past region_cap is not written and sets *flag.
// FWD: the full-tape forward (finished muons stored, survivors appended to
// `out`, as in compact_pass); otherwise the recomputation of one checkpointed
// pass in the backward (nothing but the tape and the step counts is written).
// Resident blocks per SM of the recorded pass: 4 (64 registers; measured on
// diff1e6 with the planes stored as soon as their values exist: checkpoint
// backward 55.4 ms against 55.7 ms at 5 blocks, which spill 8 bytes).
// 0: the plain pass's.
#ifndef MT_TAPE_MIN_BLOCKS
#define MT_TAPE_MIN_BLOCKS 4
#endif
template <int GEOM, int FIELD>
constexpr int tape_min_blocks()
{
    return MT_TAPE_MIN_BLOCKS > 0 ? MT_TAPE_MIN_BLOCKS : pass_min_blocks<GEOM, FIELD>();
}

// Philox round keys from the launch parameters in the recorded passes (see step)
#ifndef MT_TAPE_RK
#define MT_TAPE_RK 1
#endif

template <int GEOM, int FIELD, bool FWD>
__global__ void __launch_bounds__(kBlock, tape_min_blocks<GEOM, FIELD>())
    tape_pass(const WorldParams w, const mt_muon_soa soa, const RunParams rp, LiveBuf in, LiveBuf out,
              const unsigned long long *cin, unsigned long long *cout, int S, char *tape_base,
              unsigned long long *tape_off, int64_t region_cap, unsigned int *flag, unsigned long long *work,
              unsigned long long *wzero)
{
    __shared__ SmemWorld sw;
    const int64_t count = (int64_t)*cin;
    const unsigned long long off = tape_off[0];
    const int64_t bytes = tape_pass_bytes(count, S);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        tape_off[1] = off + (count ? bytes : 0);
        if (wzero) *wzero = 0ull;
    }
    if (count == 0) return;
    const bool room = (int64_t)off + bytes <= region_cap;
    if (!room && blockIdx.x == 0 && threadIdx.x == 0) *flag = 1u;
    stage_world(sw, w, rp);
    __syncthreads();
    TapeRef<MT_TAPE_RECORD_B> tr{tape_base + off, round_up(count, 32), 0};
    const unsigned lane = threadIdx.x & 31u;
    for (;;) {
        // 32-entry chunks from the pass's work counter (see compact_pass)
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
            tr.tid = i;
            const uint64_t id = (uint64_t)(rp.id_offset + idx);
            const uint32_t id_lo = (uint32_t)id, id_hi = (uint32_t)(id >> 32);
            const int kend = min(k + S, rp.max_steps);
            int r = MT_ALIVE, ns = 0;
#pragma unroll 1
            for (; k < kend; ++k) {
                TapeWriter<MT_TAPE_RECORD_B> wr{&tr, ns};
                wr.on = room;
                r = step<GEOM, FIELD, TapeWriter<MT_TAPE_RECORD_B> &, MT_TAPE_RK>(w, sw, s, q, k, id_lo, id_hi,
                                                                               (uint32_t)rp.instance, rp, wr);
                if (r != MT_ALIVE) break;
                ++ns;
            }
            reinterpret_cast<float *>(in.w3 + i)[3] = __int_as_float(ns);
            if (FWD) {
                if (r == MT_ALIVE && k >= rp.max_steps) r = MT_MAX_STEPS;
                if (r != MT_ALIVE)
                    store_muon(w, soa, idx, s, k, r);
                else
                    keep = true;
            }
        }
        if (FWD) {
            const int64_t slot = warp_append(cout, keep);
            if (keep) put_live(out, slot, s, q, k, idx);
        }
    }
}

// Reverse of one recorded pass: each entry of list `ck` walks its recorded
// steps backwards (tape of the pass at tape_base + tape_off[0], column = list
// entry), carrying (dL/dr, dL/dp) of muon idx in adj[6][n] and accumulating
// dL/dalpha.  Nothing is done when *flag is set (the tape was not written).
// cols (if not null): only the *sel_count entries cols[0 ..] of the list are
// reversed (the full tape's entries with a nonzero cotangent).
template <int GEOM, int FIELD>
__global__ void __launch_bounds__(kBlock, MT_ADJ_MIN_BLOCKS)
    adjoint_pass(const WorldParams w, const RunParams rp, LiveBuf ck, const unsigned long long *count_p, float *adj,
                 int64_t n, double *dalpha, const char *tape_base, const unsigned long long *tape_off,
                 const unsigned int *flag, unsigned long long *work, unsigned long long *wzero, const unsigned *cols,
                 const unsigned long long *sel_count)
{
    __shared__ SmemWorld sw;
    __shared__ float sacc[3][MT_MAX_BOXES];
    const int64_t count = (int64_t)*count_p;
    const int64_t todo = cols ? (int64_t)*sel_count : count;
    if (wzero && blockIdx.x == 0 && threadIdx.x == 0) *wzero = 0ull;
    if (todo == 0 || *flag) return;
    stage_world(sw, w, rp);
    for (int t = threadIdx.x; t < 3 * MT_MAX_BOXES; t += blockDim.x) (&sacc[0][0])[t] = 0.0f;
    __syncthreads();
    AlphaAcc acc;
    TapeRef<MT_TAPE_RECORD_B> tr{const_cast<char *>(tape_base) + *tape_off, round_up(count, 32), 0};
    const unsigned lane = threadIdx.x & 31u;
    for (;;) {
        // 32-entry chunks from the pass's work counter (see compact_pass)
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(work, 32ull);
        const int64_t base = (int64_t)__shfl_sync(0xFFFFFFFFu, b, 0);
        if (base >= todo) break;
        const int64_t li = base + lane;
        if (li >= todo) continue;
        const int64_t i = cols ? (int64_t)cols[li] : li;
        tr.tid = i;
        const float q = ck.w0[i].w;
        const int64_t idx = __float_as_int(ck.w2[i].w);
        const int ns = __float_as_int(ck.w3[i].w);
        float rb[3] = {adj[idx], adj[n + idx], adj[2 * n + idx]};
        float pb[3] = {adj[3 * n + idx], adj[4 * n + idx], adj[5 * n + idx]};
        // a zero adjoint stays zero through the pass and adds nothing to dL/dalpha
        if (rb[0] == 0.0f && rb[1] == 0.0f && rb[2] == 0.0f && pb[0] == 0.0f && pb[1] == 0.0f && pb[2] == 0.0f)
            continue;
#pragma unroll 1
        for (int j = ns - 1; j >= 0; --j) {
            const TapeEntry t = load_tape(tr, j);
#if MT_ADJ_PREFETCH
            if (j > 0) {
                prefetch_l1(tr.a(j - 1));
                prefetch_l1(tr.b(j - 1));
                prefetch_l1(tr.c(j - 1));
                if (MT_TAPE_RECORD_B) prefetch_l1(tr.d(j - 1));
            }
#endif
            reverse_step<GEOM, FIELD, MT_TAPE_RECORD_B>(w, sw, t, q, rp.d, rp.kd, rb, pb, acc, sacc);
        }
        adj[idx] = rb[0];
        adj[n + idx] = rb[1];
        adj[2 * n + idx] = rb[2];
        adj[3 * n + idx] = pb[0];
        adj[4 * n + idx] = pb[1];
        adj[5 * n + idx] = pb[2];
    }
    acc.flush(sacc);
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * MT_MAX_BOXES; t += blockDim.x) {
        const float v = sacc[t % 3][t / 3];
        if (v != 0.0f) atomicAdd(&dalpha[t], (double)v);
    }
}

// Acceptance loss of the differentiable form: mean over all n muons of
// s((h - |x_e|)/w) s((h - |y_e|)/w), (x_e, y_e) the straight-line extrapolation
// of the final state to z = zL; STOPPED / INVALID muons and pz <= 0 give 0.
__global__ void __launch_bounds__(kBlock) acceptance_loss_kernel(const mt_muon_soa s, int64_t n, float zL, float half,
                                                                 float width, double *loss, float *g)
{
    __shared__ double part[kBlock / 32];
    double local = 0.0;
    const float inv_n = 1.0f / (float)n;
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t st = s.status[m];
        const float pz = s.pz[m];
        float gx = 0.0f, gy = 0.0f, gz = 0.0f, gpx = 0.0f, gpy = 0.0f, gpz = 0.0f;
        if (st != MT_STOPPED && st != MT_INVALID && pz > 0.0f) {
            const float x = s.x[m], y = s.y[m], z = s.z[m], px = s.px[m], py = s.py[m];
            const float lz = zL - z;
            const float xe = fmaf(lz, px / pz, x), ye = fmaf(lz, py / pz, y);
            const float sa = 1.0f / (1.0f + expf(-(half - fabsf(xe)) / width));
            const float sb = 1.0f / (1.0f + expf(-(half - fabsf(ye)) / width));
            local += (double)(sa * sb);
            const float dxe = sa * (1.0f - sa) * sb * (xe >= 0.0f ? -1.0f : 1.0f) / width * inv_n;
            const float dye = sb * (1.0f - sb) * sa * (ye >= 0.0f ? -1.0f : 1.0f) / width * inv_n;
            gx = dxe;
            gy = dye;
            gz = -(dxe * px + dye * py) / pz;
            gpx = dxe * lz / pz;
            gpy = dye * lz / pz;
            gpz = -(dxe * px + dye * py) * lz / (pz * pz);
        }
        if (g) {
            g[m] = gx;
            g[n + m] = gy;
            g[2 * n + m] = gz;
            g[3 * n + m] = gpx;
            g[4 * n + m] = gpy;
            g[5 * n + m] = gpz;
        }
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xFFFFFFFFu, local, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += part[i];
        atomicAdd(loss, t / (double)n);
    }
}

static int resident_grid(const void *kernel, int64_t work)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sms * per_sm;
    const int64_t need = (work + kBlock - 1) / kBlock;
    if (grid > need) grid = need;
    return (int)(grid < 1 ? 1 : grid);
}

// Muon groups of the checkpointing form, as in the plain transport: from
// MT_CKPT_GROUP_MIN_MUONS muons, the muons [0, n/2) and [n/2, n) are two
// checkpointed transports of their own (each with its own layout in the
// checkpoint buffer, one after the other), run side by side on two streams in
// the forward and again in the backward, whose recorded and reverse passes
// leave most of the SMs' warp slots free.
#ifndef MT_CKPT_GROUP_MIN_MUONS
#define MT_CKPT_GROUP_MIN_MUONS (1 << 19)
#endif

struct CkptGroups {
    int G;
    int64_t n[2];      // muons of each group
    int64_t start[2];  // first muon of each group
    int64_t off[2];    // byte offset of each group's layout in the checkpoint buffer
};

static CkptGroups ckpt_groups(int64_t n, int32_t max_steps, int32_t K)
{
    CkptGroups g;
    g.G = n >= MT_CKPT_GROUP_MIN_MUONS ? 2 : 1;
    g.n[0] = g.G == 2 ? n / 2 : n;
    g.n[1] = n - g.n[0];
    g.start[0] = 0;
    g.start[1] = g.n[0];
    g.off[0] = 0;
    g.off[1] = round_up(ckpt_layout(g.n[0], max_steps, K).total, 256);
    return g;
}

int64_t ckpt_bytes(int64_t n, int32_t max_steps, int32_t K)
{
    const CkptGroups g = ckpt_groups(n, max_steps, K);
    int64_t b = 0;
    for (int i = 0; i < g.G; ++i) b += round_up(ckpt_layout(g.n[i], max_steps, K).total, 256);
    return b;
}

// The muons [off, ...) of s as a SoA of their own (their ids follow from rp).
static mt_muon_soa soa_from(const mt_muon_soa &s, int64_t off)
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

// A second stream forked from st; join() makes st wait for everything given
// to it, also after an error, and releases stream and events once their work
// is done.
struct Fork {
    cudaStream_t aux = nullptr;
    cudaEvent_t fork = nullptr, join_ev = nullptr;
    cudaError_t begin(cudaStream_t st)
    {
        cudaError_t e = cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join_ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, fork, 0);
        return e;
    }
    cudaError_t join(cudaStream_t st)
    {
        cudaError_t e = cudaSuccess;
        if (aux && join_ev) {
            e = cudaEventRecord(join_ev, aux);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, join_ev, 0);
            if (e != cudaSuccess) cudaStreamSynchronize(aux);
        }
        if (join_ev) cudaEventDestroy(join_ev);
        if (fork) cudaEventDestroy(fork);
        if (aux) cudaStreamDestroy(aux);
        aux = nullptr;
        fork = join_ev = nullptr;
        return e;
    }
};

template <int GEOM, int FIELD>
static cudaError_t ckpt_forward(const WorldParams &w, const mt_muon_soa &soa, int64_t n, const RunParams &rp,
                                cudaStream_t st, int K, char *ck)
{
    const CkptLayout L = ckpt_layout(n, rp.max_steps, K);
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(ck);
    unsigned *hist = reinterpret_cast<unsigned *>(ck + L.sort_off), *offs = hist + kSortBins;
    auto list = [&](int p) { return live_buf_at(ck + L.lists_off + p * L.list_bytes, n); };
    // Spatial order of the saved lists (field maps, as the plain transport takes
    // it): after compact_init and every sort_every(K)-th pass, survivors go to
    // the list two ahead, still unused, and are scattered in key order into the
    // next one.  The backward then reads every list in that order too.
    const bool order = w.sort_bins > 0 && n >= MT_SORT_MIN_MUONS && L.passes > 1;
    cudaError_t e = cudaMemsetAsync(ck, 0, (size_t)L.lists_off, st);
    if (e == cudaSuccess && order)
        e = cudaFuncSetAttribute(sort_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, kScanSmem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = resident_grid((const void *)compact_pass<GEOM, FIELD>, n);
    const int sgrid = grid < sms * 8 ? sms * 8 : grid;
    auto reorder = [&](const LiveBuf &src, const LiveBuf &dst, const unsigned long long *cnt) {
        sort_scan<<<1, 1024, kScanSmem, st>>>(hist, offs, w.sort_bins);
        cudaError_t f = cudaGetLastError();
        if (f != cudaSuccess) return f;
        sort_scatter<<<sgrid, kBlock, 0, st>>>(w, src, dst, cnt, offs);
        return cudaGetLastError();
    };
    const int64_t need = (n + kBlock - 1) / kBlock;
    compact_init<<<(unsigned)(need < 65535 * 8 ? need : 65535 * 8), kBlock, 0, st>>>(
        w, soa, n, rp, list(order ? 1 : 0), ctr, order ? hist : nullptr);
    e = cudaGetLastError();
    if (e == cudaSuccess && order) e = reorder(list(1), list(0), ctr);
    if (e != cudaSuccess) return e;
    for (int p = 0; p < L.passes; ++p) {
        const bool count = order && p + 2 <= L.passes && (p + 1) % sort_every(K) == 0;
        compact_pass<GEOM, FIELD><<<grid, kBlock, 0, st>>>(w, soa, rp, list(p), list(count ? p + 2 : p + 1), ctr + p,
                                                            ctr + p + 1, nullptr, ctr + L.passes + 1 + p, nullptr, K,
                                                            count ? hist : nullptr);
        e = cudaGetLastError();
        if (e == cudaSuccess && count) e = reorder(list(p + 2), list(p + 1), ctr + p + 1);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int GEOM, int FIELD>
static cudaError_t tape_forward(const WorldParams &w, const mt_muon_soa &soa, int64_t n, const RunParams &rp,
                                cudaStream_t st, int K, char *buf)
{
    const TapeLayout T = tape_layout(n, rp.max_steps, K);
    const CkptLayout &L = T.ck;
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(buf);
    unsigned long long *toff = reinterpret_cast<unsigned long long *>(buf + T.off_off);
    unsigned int *flag = reinterpret_cast<unsigned int *>(buf + T.flag_off);
    cudaError_t e = cudaMemsetAsync(buf, 0, (size_t)L.lists_off, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf + T.off_off, 0, (size_t)(T.region_off - T.off_off), st);
    if (e != cudaSuccess) return e;
    const int64_t need = (n + kBlock - 1) / kBlock;
    compact_init<<<(unsigned)(need < 65535 * 8 ? need : 65535 * 8), kBlock, 0, st>>>(
        w, soa, n, rp, live_buf_at(buf + L.lists_off, n), ctr, nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int grid = resident_grid((const void *)tape_pass<GEOM, FIELD, true>, n);
    for (int p = 0; p < L.passes; ++p) {
        tape_pass<GEOM, FIELD, true><<<grid, kBlock, 0, st>>>(
            w, soa, rp, live_buf_at(buf + L.lists_off + p * L.list_bytes, n),
            live_buf_at(buf + L.lists_off + (p + 1) * L.list_bytes, n), ctr + p, ctr + p + 1, K,
            buf + T.region_off, toff + p, T.region_cap, flag, ctr + L.passes + 1 + p, nullptr);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The entries of checkpointed list `in` (*cin of them) whose muon has a
// nonzero cotangent in gfin = dL/d(final state) [6][n] (all entries when gfin
// is null), appended to `out` at *cout.  The backward is linear in gfin, so a
// muon whose six components are all zero keeps a zero adjoint through every
// step and adds nothing to dL/dalpha: the backward leaves it out and its rows
// of dL/d(initial state) keep the zeros they start from.  Under the acceptance
// loss that is every stopped muon and every muon extrapolated 1.4 m or more
// outside the acceptance (the sigmoids underflow to zero), most of a shield's.
__global__ void __launch_bounds__(kBlock) select_live(LiveBuf in, const unsigned long long *cin, const float *gfin,
                                                      int64_t n, LiveBuf out, unsigned long long *cout)
{
    const int64_t count = (int64_t)*cin;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < count; base += stride) {
        const int64_t i = base + threadIdx.x;
        bool keep = false;
        float4 a, b, c, d;
        if (i < count) {
            c = in.w2[i];
            const int64_t m = (int64_t)__float_as_int(c.w);
            keep = !gfin || gfin[m] != 0.0f || gfin[n + m] != 0.0f || gfin[2 * n + m] != 0.0f ||
                   gfin[3 * n + m] != 0.0f || gfin[4 * n + m] != 0.0f || gfin[5 * n + m] != 0.0f;
            if (keep) {
                a = in.w0[i];
                b = in.w1[i];
                d = in.w3[i];
            }
        }
        const int64_t slot = warp_append(cout, keep);
        if (keep) {
            out.w0[slot] = a;
            out.w1[slot] = b;
            out.w2[slot] = c;
            out.w3[slot] = d;
        }
    }
}

// The positions in list `in` (*cin entries) of the muons with a nonzero
// cotangent in gfin (see select_live), appended to cols at *cout: the full
// tape's backward reverses those columns only.
__global__ void __launch_bounds__(kBlock) select_cols(LiveBuf in, const unsigned long long *cin, const float *gfin,
                                                      int64_t n, unsigned *cols, unsigned long long *cout)
{
    const int64_t count = (int64_t)*cin;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < count; base += stride) {
        const int64_t i = base + threadIdx.x;
        bool keep = false;
        if (i < count) {
            const int64_t m = (int64_t)__float_as_int(in.w2[i].w);
            keep = gfin[m] != 0.0f || gfin[n + m] != 0.0f || gfin[2 * n + m] != 0.0f || gfin[3 * n + m] != 0.0f ||
                   gfin[4 * n + m] != 0.0f || gfin[5 * n + m] != 0.0f;
        }
        const int64_t slot = warp_append(cout, keep);
        if (keep) cols[slot] = (unsigned)i;
    }
}

// Scratch of the recompute form's backward: two slots, each a 256-byte header
// (region offsets at bytes 0-15, the flag at 64, the recorded pass's and the
// reverse pass's work counters at 128 and 136, the selected entries' count at
// 192), the tape of one pass of up to n entries, and the pass's selected list
// (up to n entries).  Pass p uses slot p % 2.
static int64_t ckpt_tape_cap(int64_t n, int K) { return round_up(tape_pass_bytes(n > 0 ? n : 1, K), 256); }
static int64_t ckpt_slot_bytes(int64_t n, int K)
{
    return 256 + ckpt_tape_cap(n, K) + 4 * (n > 0 ? n : 1) * (int64_t)sizeof(float4);
}
static int64_t ckpt_scratch_bytes(int64_t n, int K) { return 2 * ckpt_slot_bytes(n, K); }

// Resident blocks per SM of the two kernels of the checkpoint backward (0: as
// many as fit).  The recorded pass of segment p - 1 runs on a second stream
// while the reverse pass of segment p runs on the caller's, so the one starts
// as the other's blocks retire.  Both want every warp slot they can get:
// measured on diff1e6 (K = 32), full grids 55.9 ms; 2 + 1 blocks per SM side
// by side 77.5 ms, 1 + 2 71.6 ms, 1 + 1 77.2 ms.
#ifndef MT_ADJ_REC_BLOCKS
#define MT_ADJ_REC_BLOCKS 0
#endif
#ifndef MT_ADJ_SWEEP_BLOCKS
#define MT_ADJ_SWEEP_BLOCKS 0
#endif

static int split_grid(const void *kernel, int per_sm_cap, int64_t work)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0);
    if (per_sm_cap > 0 && per_sm_cap < per_sm) per_sm = per_sm_cap;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sms * per_sm;
    const int64_t need = (work + kBlock - 1) / kBlock;
    if (grid > need) grid = need;
    return (int)(grid < 1 ? 1 : grid);
}

// The reverse sweep over the checkpointed passes, last pass first.  Segment
// p's recorded pass (slot p % 2) may start once the reverse pass of segment
// p + 2, the slot's previous user, is done; segment p's reverse pass waits for
// its recorded pass and (in stream order) for segment p + 1's reverse pass,
// whose adjoint state it continues.
template <int GEOM, int FIELD>
static cudaError_t ckpt_backward(const WorldParams &w, int64_t n, const RunParams &rp, cudaStream_t st, int K,
                                 char *ck, float *adj, char *scratch, const float *gfin, int64_t ld)
{
    const CkptLayout L = ckpt_layout(n, rp.max_steps, K);
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(ck);
    double *dalpha = reinterpret_cast<double *>(ck + L.alpha_off);
    const int64_t slot = ckpt_slot_bytes(n, K);
    const int64_t cap = ckpt_tape_cap(n, K);
    cudaError_t e = cudaMemsetAsync(dalpha, 0, 3 * MT_MAX_BOXES * sizeof(double), st);
    for (int s = 0; s < 2 && e == cudaSuccess; ++s) e = cudaMemsetAsync(scratch + s * slot, 0, 256, st);
    if (e != cudaSuccess) return e;
    const int rgrid = split_grid((const void *)tape_pass<GEOM, FIELD, false>, MT_ADJ_REC_BLOCKS, n);
    const int agrid = split_grid((const void *)adjoint_pass<GEOM, FIELD>, MT_ADJ_SWEEP_BLOCKS, n);
    const int sgrid = resident_grid((const void *)select_live, n);
    const int P = L.passes;
    cudaStream_t aux = nullptr;
    std::vector<cudaEvent_t> ev(2 * P + 1, nullptr);   // [0, P): recorded, [P, 2P): reversed, 2P: fork
    e = cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking);
    for (size_t i = 0; i < ev.size() && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2 * P], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev[2 * P], 0);
    auto hdr = [&](int p) { return scratch + (p & 1) * slot; };
    // segment p's entries with a nonzero cotangent, in its slot
    auto selected = [&](int p) { return live_buf_at(hdr(p) + 256 + cap, n); };
    auto record = [&](int p) {
        char *h = hdr(p);
        unsigned long long *wc = reinterpret_cast<unsigned long long *>(h + 128);
        unsigned long long *cnt = reinterpret_cast<unsigned long long *>(h + 192);
        const LiveBuf sel = selected(p);
        if (p + 2 < P && e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev[P + p + 2], 0);
        if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), aux);
        if (e != cudaSuccess) return;
        select_live<<<sgrid, kBlock, 0, aux>>>(live_buf_at(ck + L.lists_off + p * L.list_bytes, n), ctr + p, gfin, ld,
                                               sel, cnt);
        tape_pass<GEOM, FIELD, false><<<rgrid, kBlock, 0, aux>>>(
            w, mt_muon_soa{}, rp, sel, sel, cnt, nullptr, K, h + 256, reinterpret_cast<unsigned long long *>(h), cap,
            reinterpret_cast<unsigned int *>(h + 64), wc, wc + 1);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(ev[p], aux);
    };
    auto reverse = [&](int p) {
        char *h = hdr(p);
        unsigned long long *wc = reinterpret_cast<unsigned long long *>(h + 128);
        const unsigned long long *cnt = reinterpret_cast<const unsigned long long *>(h + 192);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev[p], 0);
        if (e != cudaSuccess) return;
        adjoint_pass<GEOM, FIELD><<<agrid, kBlock, 0, st>>>(w, rp, selected(p), cnt, adj, ld, dalpha, h + 256,
                                                           reinterpret_cast<const unsigned long long *>(h),
                                                           reinterpret_cast<const unsigned int *>(h + 64), wc + 1, wc,
                                                           nullptr, nullptr);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(ev[P + p], st);
    };
    // enqueue order: the recording one segment ahead of the reverse pass
    if (P > 0) record(P - 1);
    for (int p = P - 1; p >= 0 && e == cudaSuccess; --p) {
        if (p > 0) record(p - 1);
        reverse(p);
    }
    // the caller's stream has waited for every recorded pass (the last is
    // segment 0's); stream and events are released once their work is done
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (aux) cudaStreamDestroy(aux);
    return e;
}

// scratch: the selected columns of one pass (n u32) and the passes' counts of
// them (L.passes u64), see tape_backward_scratch_bytes.
static int64_t tape_backward_scratch_bytes(int64_t n, int32_t max_steps, int K)
{
    const CkptLayout L = ckpt_layout(n, max_steps, K);
    return round_up((n > 0 ? n : 1) * 4, 256) + round_up((int64_t)L.passes * 8, 256);
}

template <int GEOM, int FIELD>
static cudaError_t tape_backward(const WorldParams &w, int64_t n, const RunParams &rp, cudaStream_t st, int K,
                                 char *buf, float *adj, char *scratch, const float *gfin, int64_t ld)
{
    const TapeLayout T = tape_layout(n, rp.max_steps, K);
    const CkptLayout &L = T.ck;
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(buf);
    const unsigned long long *toff = reinterpret_cast<const unsigned long long *>(buf + T.off_off);
    const unsigned int *flag = reinterpret_cast<const unsigned int *>(buf + T.flag_off);
    double *dalpha = reinterpret_cast<double *>(buf + L.alpha_off);
    // the passes' work counters (used by the forward) are cleared for the sweep
    unsigned long long *wc = ctr + L.passes + 1;
    cudaError_t e = cudaMemsetAsync(dalpha, 0, 3 * MT_MAX_BOXES * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(wc, 0, (size_t)(L.passes + 1) * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    unsigned *cols = reinterpret_cast<unsigned *>(scratch);
    unsigned long long *sel = reinterpret_cast<unsigned long long *>(scratch + round_up((n > 0 ? n : 1) * 4, 256));
    if (e == cudaSuccess) e = cudaMemsetAsync(sel, 0, (size_t)L.passes * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const int grid = resident_grid((const void *)adjoint_pass<GEOM, FIELD>, n);
    const int sgrid = resident_grid((const void *)select_cols, n);
    for (int p = L.passes - 1; p >= 0; --p) {
        const LiveBuf lp = live_buf_at(buf + L.lists_off + p * L.list_bytes, n);
        select_cols<<<sgrid, kBlock, 0, st>>>(lp, ctr + p, gfin, ld, cols, sel + p);
        adjoint_pass<GEOM, FIELD><<<grid, kBlock, 0, st>>>(w, rp, lp, ctr + p, adj, ld, dalpha, buf + T.region_off,
                                                          toff + p, flag, wc + p, nullptr, cols, sel + p);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// dL/dalpha as float (the sum of two groups' accumulators when src1 is not
// null); NaN when the forward ran out of tape (flag set).
__global__ void alpha_out(const double *src, const double *src1, float *dst, int m, const unsigned int *flag,
                          const unsigned int *flag1)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool bad = (flag && *flag) || (flag1 && *flag1);
    if (t < m) dst[t] = bad ? __int_as_float(0x7FC00000) : (float)(src[t] + (src1 ? src1[t] : 0.0));
}

#define MT_DISPATCH_FIELDS(FN, G, ...)                                                  \
    (w.field_kind == MT_FIELD_MAP           ? FN<G, MT_FIELD_MAP>(__VA_ARGS__)           \
     : w.field_kind == MT_FIELD_MAP_NEAREST ? FN<G, MT_FIELD_MAP_NEAREST>(__VA_ARGS__)   \
     : w.field_kind == MT_FIELD_BOX         ? FN<G, MT_FIELD_BOX>(__VA_ARGS__)           \
                                            : FN<G, MT_FIELD_NONE>(__VA_ARGS__))
#define MT_DISPATCH(FN, ...)                                                           \
    (w.geom_kind == MT_GEOM_BOXES       ? MT_DISPATCH_FIELDS(FN, MT_GEOM_BOXES, __VA_ARGS__)     \
     : w.geom_kind == MT_GEOM_POLYHEDRA ? MT_DISPATCH_FIELDS(FN, MT_GEOM_POLYHEDRA, __VA_ARGS__) \
     : w.field_kind == MT_FIELD_MAP     ? FN<MT_GEOM_VOXELS, MT_FIELD_MAP>(__VA_ARGS__)          \
     : w.field_kind == MT_FIELD_MAP_NEAREST ? FN<MT_GEOM_VOXELS, MT_FIELD_MAP_NEAREST>(__VA_ARGS__) \
                                        : FN<MT_GEOM_VOXELS, MT_FIELD_NONE>(__VA_ARGS__))

}  // namespace mt

using namespace mt;

namespace {

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

mt_status fill_run(RunParams &rp, float step_len, int32_t max_steps, uint64_t seed, const float *alpha,
                   int32_t n_block, int64_t id_offset, int32_t instance)
{
    if (!(step_len > 0.0f) || !isfinite(step_len) || max_steps < 0) {
        set_error("step_len must be positive and finite, max_steps >= 0");
        return MT_ERR_INVALID_ARG;
    }
    if (alpha && (n_block < 0 || n_block > MT_MAX_BOXES)) {
        set_error("n_block %d outside [0, %d]", n_block, MT_MAX_BOXES);
        return MT_ERR_INVALID_ARG;
    }
    rp.d = step_len;
    rp.kd = (float)(0.299792458 * (double)step_len);
    rp.max_steps = max_steps;
    set_seed(rp, seed);
    rp.alpha = alpha;
    rp.n_block = alpha ? n_block : 0;
    rp.instance = instance;
    rp.id_offset = id_offset;
    return MT_OK;
}

mt_status check_ckpt(int64_t n, int32_t max_steps, int32_t K, const void *ck, int64_t bytes)
{
    if (K < 1 || K > kTapeMax) {
        set_error("ckpt_every %d outside [1, %d]", K, kTapeMax);
        return MT_ERR_INVALID_ARG;
    }
    if (n < 0 || n >= ((int64_t)1 << 31)) {
        set_error("n = %lld outside [0, 2^31)", (long long)n);
        return MT_ERR_INVALID_ARG;
    }
    if (!ck || (reinterpret_cast<uintptr_t>(ck) & 255u) || bytes < ckpt_bytes(n, max_steps, K)) {
        set_error("checkpoint buffer %p of %lld bytes: need %lld bytes, 256-byte aligned", ck, (long long)bytes,
                  (long long)ckpt_bytes(n, max_steps, K));
        return MT_ERR_INVALID_ARG;
    }
    return MT_OK;
}

}  // namespace

extern "C" int64_t mt_ckpt_bytes(int64_t n, int32_t max_steps, int32_t ckpt_every)
{
    if (ckpt_every < 1) return -1;
    return ckpt_bytes(n, max_steps, ckpt_every);
}

extern "C" mt_status mt_transport_ckpt(mt_handle *h, const mt_muon_soa *s, int64_t n, float step_len, int32_t max_steps,
                                       uint64_t seed, const float *alpha, int32_t n_block, int32_t ckpt_every,
                                       void *ckpt, int64_t ckpt_bytes_, void *stream)
{
    if (!h || !s) {
        set_error("null handle or muon SoA");
        return MT_ERR_INVALID_ARG;
    }
    if (n > 0 && (!s->x || !s->y || !s->z || !s->px || !s->py || !s->pz || !s->q || !s->steps || !s->status)) {
        set_error("null muon array with n > 0");
        return MT_ERR_INVALID_ARG;
    }
    if (h && h->w.field_per_stage) {
        set_error("the differentiable form holds the field over each step: per_stage is not supported");
        return MT_ERR_INVALID_ARG;
    }
    RunParams rp;
    mt_status stt = fill_run(rp, step_len, max_steps, seed, alpha, n_block, s->id_offset, s->instance);
    if (stt != MT_OK) return stt;
    stt = check_ckpt(n, max_steps, ckpt_every, ckpt, ckpt_bytes_);
    if (stt != MT_OK) return stt;
    if (n == 0) return MT_OK;
    DevGuard g(h->device);
    const WorldParams &w = h->w;
    cudaStream_t st = (cudaStream_t)stream;
    const CkptGroups G = ckpt_groups(n, max_steps, ckpt_every);
    cudaError_t e;
    if (G.G == 1) {
        e = MT_DISPATCH(ckpt_forward, w, *s, n, rp, st, ckpt_every, (char *)ckpt);
    } else {
        Fork f;
        e = f.begin(st);
        if (e == cudaSuccess) e = MT_DISPATCH(ckpt_forward, w, *s, G.n[0], rp, st, ckpt_every, (char *)ckpt);
        if (e == cudaSuccess) {
            RunParams r1 = rp;
            r1.id_offset += G.start[1];
            e = MT_DISPATCH(ckpt_forward, w, soa_from(*s, G.start[1]), G.n[1], r1, f.aux, ckpt_every,
                            (char *)ckpt + G.off[1]);
        }
        const cudaError_t j = f.join(st);
        if (e == cudaSuccess) e = j;
    }
    if (e != cudaSuccess) return cuda_fail(e, "checkpointing transport");
    return MT_OK;
}

extern "C" mt_status mt_adjoint_ckpt(mt_handle *h, int64_t n, float step_len, int32_t max_steps, uint64_t seed,
                                     const float *alpha, int32_t n_block, int32_t ckpt_every, void *ckpt,
                                     int64_t ckpt_bytes_, int64_t id_offset, int32_t instance, const float *dL_dfinal,
                                     float *dL_dinitial, float *dL_dalpha, void *stream)
{
    if (!h) {
        set_error("null handle");
        return MT_ERR_INVALID_ARG;
    }
    if (h && h->w.field_per_stage) {
        set_error("the differentiable form holds the field over each step: per_stage is not supported");
        return MT_ERR_INVALID_ARG;
    }
    RunParams rp;
    mt_status stt = fill_run(rp, step_len, max_steps, seed, alpha, n_block, id_offset, instance);
    if (stt != MT_OK) return stt;
    if (n != 0) {
        stt = check_ckpt(n, max_steps, ckpt_every, ckpt, ckpt_bytes_);
        if (stt != MT_OK) return stt;
    }
    if (id_offset < 0 || n < 0 || (n > 0 && !dL_dfinal) || (alpha && n_block > 0 && !dL_dalpha)) {
        set_error("negative id_offset or n, or null dL_dfinal / dL_dalpha");
        return MT_ERR_INVALID_ARG;
    }
    DevGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const WorldParams &w = h->w;
    if (n == 0) {
        if (alpha && n_block > 0) {
            const cudaError_t e = cudaMemsetAsync(dL_dalpha, 0, 3 * n_block * sizeof(float), st);
            if (e != cudaSuccess) return cuda_fail(e, "adjoint");
        }
        return MT_OK;
    }
    // scratch: the tape of the reverse sweep, and the adjoint state unless the
    // caller asked for dL/d(initial state) in place
    // each group its own tape slots; the adjoint state [6][n] is shared, group
    // 1's rows starting at its first muon
    const CkptGroups G = ckpt_groups(n, max_steps, ckpt_every);
    const int64_t tb0 = round_up(ckpt_scratch_bytes(G.n[0], ckpt_every), 256);
    const int64_t tbytes = tb0 + (G.G == 2 ? ckpt_scratch_bytes(G.n[1], ckpt_every) : 0);
    const int64_t abytes = dL_dinitial ? 0 : ((6 * n * (int64_t)sizeof(float) + 255) & ~(int64_t)255);
    const int64_t aoff = round_up(tbytes, 256);
    char *scratch = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&scratch), (size_t)(aoff + abytes), st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint scratch");
    float *adj = dL_dinitial ? dL_dinitial : reinterpret_cast<float *>(scratch + aoff);
    e = cudaMemcpyAsync(adj, dL_dfinal, 6 * n * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && G.G == 1) {
        e = MT_DISPATCH(ckpt_backward, w, n, rp, st, ckpt_every, (char *)ckpt, adj, scratch, dL_dfinal, n);
    } else if (e == cudaSuccess) {
        Fork f;
        e = f.begin(st);
        if (e == cudaSuccess)
            e = MT_DISPATCH(ckpt_backward, w, G.n[0], rp, st, ckpt_every, (char *)ckpt, adj, scratch, dL_dfinal, n);
        if (e == cudaSuccess) {
            RunParams r1 = rp;
            r1.id_offset += G.start[1];
            e = MT_DISPATCH(ckpt_backward, w, G.n[1], r1, f.aux, ckpt_every, (char *)ckpt + G.off[1],
                            adj + G.start[1], scratch + tb0, dL_dfinal + G.start[1], n);
        }
        const cudaError_t j = f.join(st);
        if (e == cudaSuccess) e = j;
    }
    if (e == cudaSuccess && alpha && n_block > 0) {
        const CkptLayout L0 = ckpt_layout(G.n[0], max_steps, ckpt_every);
        const double *a1 = nullptr;
        if (G.G == 2)
            a1 = reinterpret_cast<const double *>((char *)ckpt + G.off[1] +
                                                  ckpt_layout(G.n[1], max_steps, ckpt_every).alpha_off);
        alpha_out<<<1, 128, 0, st>>>(reinterpret_cast<const double *>((char *)ckpt + L0.alpha_off), a1, dL_dalpha,
                                     3 * n_block, nullptr, nullptr);
        e = cudaGetLastError();
    }
    const cudaError_t f = cudaFreeAsync(scratch, st);
    if (e == cudaSuccess) e = f;
    if (e != cudaSuccess) return cuda_fail(e, "adjoint");
    return MT_OK;
}

// The full-tape form's muon groups: those of the checkpoint form, each with its
// own tape layout in the buffer, one after the other.
static int64_t tape_group_off(const CkptGroups &g, int32_t max_steps, int K)
{
    return round_up(tape_layout(g.n[0], max_steps, K).total, 256);
}

static int64_t tape_bytes(int64_t n, int32_t max_steps, int K)
{
    const CkptGroups g = ckpt_groups(n, max_steps, K);
    int64_t b = 0;
    for (int i = 0; i < g.G; ++i) b += round_up(tape_layout(g.n[i], max_steps, K).total, 256);
    return b;
}

extern "C" int64_t mt_tape_bytes(int64_t n, int32_t max_steps, int32_t steps_per_pass)
{
    if (steps_per_pass < 1 || steps_per_pass > kTapeMax || n < 0 || max_steps < 0) return -1;
    return tape_bytes(n, max_steps, steps_per_pass);
}

namespace {

mt_status check_tape(int64_t n, int32_t max_steps, int32_t K, const void *buf, int64_t bytes)
{
    if (K < 1 || K > kTapeMax) {
        set_error("steps_per_pass %d outside [1, %d]", K, kTapeMax);
        return MT_ERR_INVALID_ARG;
    }
    if (n < 0 || n >= ((int64_t)1 << 31)) {
        set_error("n = %lld outside [0, 2^31)", (long long)n);
        return MT_ERR_INVALID_ARG;
    }
    const int64_t need = tape_bytes(n, max_steps, K);
    if (!buf || (reinterpret_cast<uintptr_t>(buf) & 255u) || bytes < need) {
        set_error("tape buffer %p of %lld bytes: need %lld bytes, 256-byte aligned", buf, (long long)bytes,
                  (long long)need);
        return MT_ERR_INVALID_ARG;
    }
    return MT_OK;
}

}  // namespace

extern "C" mt_status mt_transport_tape(mt_handle *h, const mt_muon_soa *s, int64_t n, float step_len, int32_t max_steps,
                                       uint64_t seed, const float *alpha, int32_t n_block, int32_t steps_per_pass,
                                       void *tape, int64_t tape_bytes_, void *stream)
{
    if (!h || !s) {
        set_error("null handle or muon SoA");
        return MT_ERR_INVALID_ARG;
    }
    if (n > 0 && (!s->x || !s->y || !s->z || !s->px || !s->py || !s->pz || !s->q || !s->steps || !s->status)) {
        set_error("null muon array with n > 0");
        return MT_ERR_INVALID_ARG;
    }
    if (h && h->w.field_per_stage) {
        set_error("the differentiable form holds the field over each step: per_stage is not supported");
        return MT_ERR_INVALID_ARG;
    }
    RunParams rp;
    mt_status stt = fill_run(rp, step_len, max_steps, seed, alpha, n_block, s->id_offset, s->instance);
    if (stt != MT_OK) return stt;
    stt = check_tape(n, max_steps, steps_per_pass, tape, tape_bytes_);
    if (stt != MT_OK) return stt;
    if (n == 0) return MT_OK;
    DevGuard g(h->device);
    const WorldParams &w = h->w;
    cudaStream_t st = (cudaStream_t)stream;
    const CkptGroups G = ckpt_groups(n, max_steps, steps_per_pass);
    cudaError_t e;
    if (G.G == 1) {
        e = MT_DISPATCH(tape_forward, w, *s, n, rp, st, steps_per_pass, (char *)tape);
    } else {
        Fork f;
        e = f.begin(st);
        if (e == cudaSuccess) e = MT_DISPATCH(tape_forward, w, *s, G.n[0], rp, st, steps_per_pass, (char *)tape);
        if (e == cudaSuccess) {
            RunParams r1 = rp;
            r1.id_offset += G.start[1];
            e = MT_DISPATCH(tape_forward, w, soa_from(*s, G.start[1]), G.n[1], r1, f.aux, steps_per_pass,
                            (char *)tape + tape_group_off(G, max_steps, steps_per_pass));
        }
        const cudaError_t j = f.join(st);
        if (e == cudaSuccess) e = j;
    }
    if (e != cudaSuccess) return cuda_fail(e, "taped transport");
    return MT_OK;
}

extern "C" mt_status mt_adjoint_tape(mt_handle *h, int64_t n, float step_len, int32_t max_steps, const float *alpha,
                                     int32_t n_block, int32_t steps_per_pass, void *tape, int64_t tape_bytes_,
                                     const float *dL_dfinal, float *dL_dinitial, float *dL_dalpha, void *stream)
{
    if (!h) {
        set_error("null handle");
        return MT_ERR_INVALID_ARG;
    }
    if (h && h->w.field_per_stage) {
        set_error("the differentiable form holds the field over each step: per_stage is not supported");
        return MT_ERR_INVALID_ARG;
    }
    RunParams rp;
    mt_status stt = fill_run(rp, step_len, max_steps, 0, alpha, n_block, 0, 0);
    if (stt != MT_OK) return stt;
    if (n != 0) {
        stt = check_tape(n, max_steps, steps_per_pass, tape, tape_bytes_);
        if (stt != MT_OK) return stt;
    }
    if (n < 0 || (n > 0 && !dL_dfinal) || (alpha && n_block > 0 && !dL_dalpha)) {
        set_error("negative n, or null dL_dfinal / dL_dalpha");
        return MT_ERR_INVALID_ARG;
    }
    DevGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const WorldParams &w = h->w;
    if (n == 0) {
        if (alpha && n_block > 0) {
            const cudaError_t e = cudaMemsetAsync(dL_dalpha, 0, 3 * n_block * sizeof(float), st);
            if (e != cudaSuccess) return cuda_fail(e, "adjoint");
        }
        return MT_OK;
    }
    // scratch: the selected columns, then the adjoint state unless the caller
    // takes dL/d(initial state)
    float *adj = dL_dinitial;
    const CkptGroups G = ckpt_groups(n, max_steps, steps_per_pass);
    const int64_t cb0 = round_up(tape_backward_scratch_bytes(G.n[0], max_steps, steps_per_pass), 256);
    const int64_t cbytes = cb0 + (G.G == 2 ? tape_backward_scratch_bytes(G.n[1], max_steps, steps_per_pass) : 0);
    const int64_t aoff = round_up(cbytes, 256);
    char *scratch = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&scratch),
                                    (size_t)(aoff + (adj ? 0 : 6 * n * (int64_t)sizeof(float))), st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint scratch");
    if (!adj) adj = reinterpret_cast<float *>(scratch + aoff);
    e = cudaMemcpyAsync(adj, dL_dfinal, 6 * n * sizeof(float), cudaMemcpyDeviceToDevice, st);
    char *tape1 = (char *)tape + (G.G == 2 ? tape_group_off(G, max_steps, steps_per_pass) : 0);
    if (e == cudaSuccess && G.G == 1) {
        e = MT_DISPATCH(tape_backward, w, n, rp, st, steps_per_pass, (char *)tape, adj, scratch, dL_dfinal, n);
    } else if (e == cudaSuccess) {
        Fork f;
        e = f.begin(st);
        if (e == cudaSuccess)
            e = MT_DISPATCH(tape_backward, w, G.n[0], rp, st, steps_per_pass, (char *)tape, adj, scratch, dL_dfinal, n);
        if (e == cudaSuccess)
            e = MT_DISPATCH(tape_backward, w, G.n[1], rp, f.aux, steps_per_pass, tape1, adj + G.start[1],
                            scratch + cb0, dL_dfinal + G.start[1], n);
        const cudaError_t j = f.join(st);
        if (e == cudaSuccess) e = j;
    }
    if (e == cudaSuccess && alpha && n_block > 0) {
        const TapeLayout T0 = tape_layout(G.n[0], max_steps, steps_per_pass);
        const double *a1 = nullptr;
        const unsigned int *f1 = nullptr;
        if (G.G == 2) {
            const TapeLayout T1 = tape_layout(G.n[1], max_steps, steps_per_pass);
            a1 = reinterpret_cast<const double *>(tape1 + T1.ck.alpha_off);
            f1 = reinterpret_cast<const unsigned int *>(tape1 + T1.flag_off);
        }
        alpha_out<<<1, 128, 0, st>>>(reinterpret_cast<const double *>((char *)tape + T0.ck.alpha_off), a1, dL_dalpha,
                                     3 * n_block, reinterpret_cast<const unsigned int *>((char *)tape + T0.flag_off),
                                     f1);
        e = cudaGetLastError();
    }
    if (scratch) {
        const cudaError_t f = cudaFreeAsync(scratch, st);
        if (e == cudaSuccess) e = f;
    }
    if (e != cudaSuccess) return cuda_fail(e, "adjoint (tape)");
    return MT_OK;
}

extern "C" mt_status mt_transport_adjoint(mt_handle *h, const mt_muon_soa *s0, int64_t n, float step_len,
                                          int32_t max_steps, uint64_t seed, const float *alpha, int32_t n_block,
                                          const float *dL_dfinal, float *dL_dalpha, int32_t ckpt_every, void *stream)
{
    if (!h || !s0) {
        set_error("null handle or muon SoA");
        return MT_ERR_INVALID_ARG;
    }
    if (h && h->w.field_per_stage) {
        set_error("the differentiable form holds the field over each step: per_stage is not supported");
        return MT_ERR_INVALID_ARG;
    }
    if (ckpt_every < 1 || ckpt_every > kTapeMax || n < 0 || n >= ((int64_t)1 << 31)) {
        set_error("ckpt_every %d outside [1, %d] or n out of range", ckpt_every, kTapeMax);
        return MT_ERR_INVALID_ARG;
    }
    if (n == 0) return mt_adjoint_ckpt(h, 0, step_len, max_steps, seed, alpha, n_block, ckpt_every, nullptr, 0,
                                       s0->id_offset, s0->instance, dL_dfinal, nullptr, dL_dalpha, stream);
    DevGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t cb = ckpt_bytes(n, max_steps, ckpt_every);
    const int64_t soa_bytes = 30 * n + 9 * 256;
    char *buf = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&buf), (size_t)(cb + soa_bytes), st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint scratch");
    // private copy of the initial state (the forward updates its SoA in place)
    mt_muon_soa c = *s0;
    char *q = buf + cb;
    auto take = [&](void *src, size_t bytes) {
        void *dst = q;
        q += (bytes + 255) & ~(size_t)255;
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
        return dst;
    };
    c.x = (float *)take(s0->x, 4 * n);
    c.y = (float *)take(s0->y, 4 * n);
    c.z = (float *)take(s0->z, 4 * n);
    c.px = (float *)take(s0->px, 4 * n);
    c.py = (float *)take(s0->py, 4 * n);
    c.pz = (float *)take(s0->pz, 4 * n);
    c.q = (int8_t *)take(s0->q, n);
    c.steps = (int32_t *)take(s0->steps, 4 * n);
    c.status = (uint8_t *)take(s0->status, n);
    mt_status stt = MT_OK;
    if (e == cudaSuccess)
        stt = mt_transport_ckpt(h, &c, n, step_len, max_steps, seed, alpha, n_block, ckpt_every, buf, cb, stream);
    if (e == cudaSuccess && stt == MT_OK)
        stt = mt_adjoint_ckpt(h, n, step_len, max_steps, seed, alpha, n_block, ckpt_every, buf, cb, s0->id_offset,
                              s0->instance, dL_dfinal, nullptr, dL_dalpha, stream);
    const cudaError_t f = cudaFreeAsync(buf, st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint state copy");
    if (stt != MT_OK) return stt;
    if (f != cudaSuccess) return cuda_fail(f, "adjoint scratch release");
    return MT_OK;
}

extern "C" mt_status mt_acceptance_loss(const mt_muon_soa *s, int64_t n, double z_plane, double half_width,
                                        double edge, double *loss, float *dL_dfinal, void *stream)
{
    if (!s || !loss || n < 0 || !(edge > 0.0) || !(half_width > 0.0)) {
        set_error("acceptance loss: null pointer, n < 0 or non-positive width");
        return MT_ERR_INVALID_ARG;
    }
    if (n > 0 && (!s->x || !s->y || !s->z || !s->px || !s->py || !s->pz || !s->status)) {
        set_error("null muon array with n > 0");
        return MT_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), st);
    if (e == cudaSuccess && n > 0) {
        const int64_t blocks = (n + kBlock - 1) / kBlock;
        acceptance_loss_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), kBlock, 0, st>>>(
            *s, n, (float)z_plane, (float)half_width, (float)edge, loss, dL_dfinal);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(e, "acceptance loss");
    return MT_OK;
}
