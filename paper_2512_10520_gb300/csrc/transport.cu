// transport.cu -- sm_103a kernels of the transport step loop (Algorithm 1 of
// "Ultra-Fast Muon Transport via Histogram Sampling on GPUs").
//
// One thread owns one muon for its whole track and keeps the state in
// registers.  Position and momentum are carried as unevaluated sums hi + lo of
// two floats (compensated accumulation), so 1500 steps of FP32 arithmetic stay
// within ~1e-9 relative of the exact track; every discrete decision (box
// faces, world bounds, momentum-bin edges) compares the full hi + lo value
// against bounds also stored as hi + lo pairs.  The only stochastic input is
// one Philox4x32-10 call per step in matter, keyed by (seed) and counted by
// (step, muon id, instance), so a muon's track does not depend on which thread,
// block or launch runs it.
#include <cfloat>
#include <cstdio>

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

// Shared-memory copy of the small per-world tables.
struct SmemWorld {
    float lo_hi[3][MT_MAX_BOXES], lo_lo[3][MT_MAX_BOXES];
    float hi_hi[3][MT_MAX_BOXES], hi_lo[3][MT_MAX_BOXES];
    float B[3][MT_MAX_BOXES];
    int32_t mat[MT_MAX_BOXES];
    int32_t block[MT_MAX_BOXES];
    float alpha[3][MT_MAX_BOXES];
    float2 e2[MT_MAX_PBINS + 1];
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
}

// GetMaterial for ordered boxes: first box with lo <= r < hi on all axes.
__device__ __forceinline__ int find_box(const SmemWorld &sw, int n_box, const State &s)
{
    for (int b = 0; b < n_box; ++b) {
        if (ge2(s.z, s.zl, sw.lo_hi[2][b], sw.lo_lo[2][b]) && !ge2(s.z, s.zl, sw.hi_hi[2][b], sw.hi_lo[2][b]) &&
            ge2(s.x, s.xl, sw.lo_hi[0][b], sw.lo_lo[0][b]) && !ge2(s.x, s.xl, sw.hi_hi[0][b], sw.hi_lo[0][b]) &&
            ge2(s.y, s.yl, sw.lo_hi[1][b], sw.lo_lo[1][b]) && !ge2(s.y, s.yl, sw.hi_hi[1][b], sw.hi_lo[1][b]))
            return b;
    }
    return -1;
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// GetMaterial for a voxel grid: floor((r - origin) / spacing) inside the grid.
// The offset r - origin is formed as a hi + lo pair; when the cell coordinate
// lies within 1e-4 of a face, the face position (index * spacing, also as a
// pair) settles which side of it the muon is on.
__device__ __forceinline__ int voxel_material(const WorldParams &w, const State &s)
{
    const float r[3] = {s.x, s.y, s.z};
    const float rl[3] = {s.xl, s.yl, s.zl};
    int idx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float dh, de;
        two_sum(r[a], -w.vorigin[a], dh, de);
        const float dl = de + (rl[a] - w.vorigin_lo[a]);
        const float u = (dh + dl) * w.vinv[a];
        int i = __float2int_rd(u);
        const float fr = u - (float)i;
        if (fr < 1e-4f || fr > 0.9999f) {
            const int ic = __float2int_rn(u);
            const float fic = (float)ic;
            const float fh = fic * w.vspacing[a];
            const float fl = fmaf(fic, w.vspacing[a], -fh) + fic * w.vspacing_lo[a];
            i = ((dh - fh) + (dl - fl)) >= 0.0f ? ic : ic - 1;
        }
        if (i < 0 || i >= w.vdims[a]) return -1;
        idx[a] = i;
    }
    return __ldg(w.vox + ((int64_t)idx[2] * w.vdims[1] + idx[1]) * w.vdims[0] + idx[0]);
}

// |p|^2 of the hi + lo momentum to first order in lo.
__device__ __forceinline__ float p2_of(const State &s)
{
    float P2 = s.px * s.px + s.py * s.py + s.pz * s.pz;
    return fmaf(2.0f * s.px, s.pxl, fmaf(2.0f * s.py, s.pyl, fmaf(2.0f * s.pz, s.pzl, P2)));
}

// (h + l)^2 as an unnormalised pair.
__device__ __forceinline__ void sq2(float h, float l, float &sh, float &sl)
{
    sh = h * h;
    sl = fmaf(h, h, -sh) + 2.0f * h * l;
}


// GetMomentumBin on log10 bins: a fast FP32 estimate, confirmed against the
// squared edges held as hi + lo pairs whenever |p|^2 lies within 4e-6 of one.
__device__ __forceinline__ int momentum_bin(const WorldParams &w, const SmemWorld &sw, const State &s, float P2)
{
    int i = __float2int_rd((0.5f * __log2f(P2) - w.log2_plo) * w.pbin_scale);
    i = min(max(i, 0), w.n_pbin - 1);
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

// Eq. 3: p <- p + Rot(dp) with dp = [dt cos phi, dt sin phi, dz] in the frame whose
// z axis is p^.  Written as p <- p + (s - 1) p + P (1-f) sin(theta) t, where
// s = (1-f) cos(theta) and t = R x^ cos(phi) + R y^ sin(phi) is the rotated
// transverse unit vector (R: the Rodrigues rotation taking z^ to p^).  The whole
// increment is small, so it is accumulated into the hi + lo momentum.
__device__ __forceinline__ void scatter(State &s, float f, float theta, float cphi, float sphi)
{
    const float P2 = p2_of(s);
    float rP = rsqrtf(P2);
    rP = rP * fmaf(-0.5f * P2 * rP, rP, 1.5f);
    const float P = P2 * rP;
    const float ux = s.px * rP, uy = s.py * rP, uz = s.pz * rP;
    float st, ct;
    sincosf(theta, &st, &ct);
    const float omc = st * st / (1.0f + ct);          // 1 - cos(theta)
    const float sm1 = -fmaf(f, ct, omc);              // (1-f) cos(theta) - 1
    const float kick = P * (1.0f - f) * st;
    const float s2 = fmaf(ux, ux, uy * uy);
    float tx, ty, tz;
    if (uz < 0.0f && s2 < 1e-24f) {                   // p^ = -z^: R = diag(1,-1,-1)
        tx = cphi;
        ty = -sphi;
        tz = 0.0f;
    } else {
        const float g = uz >= 0.0f ? 1.0f / (1.0f + uz) : (1.0f - uz) / s2;   // 1/(1+uz)
        const float wv = fmaf(cphi, ux, sphi * uy);
        tx = cphi - ux * wv * g;
        ty = sphi - uy * wv * g;
        tz = -wv;
    }
    acc(s.px, s.pxl, fmaf(sm1, s.px, kick * tx));
    acc(s.py, s.pyl, fmaf(sm1, s.py, kick * ty));
    acc(s.pz, s.pzl, fmaf(sm1, s.pz, kick * tz));
}

// a + t (b - a)
__device__ __forceinline__ float lerp(float t, float a, float b) { return fmaf(t, b - a, a); }

// Cell index and in-cell fraction of one axis of the node map.  The offset from
// the cell's lower node, (x - origin) - i * spacing, is formed from hi + lo
// pairs, so the fraction carries ~1e-7 relative error however far the cell is
// from the origin (the plain FP32 coordinate would lose ~2e-7 m, which matters
// where the field changes by tens of T/m at a magnet edge).
__device__ __forceinline__ bool map_axis(float xh, float xl, float oh, float ol, float sh, float sl, float inv, int n,
                                         int &i, float &t)
{
    float dh, de;
    two_sum(xh, -oh, dh, de);
    const float dl = de + (xl - ol);
    const float u = (dh + dl) * inv;
    if (!(u >= 0.0f && u <= (float)(n - 1))) return false;
    i = min((int)u, n - 2);
    const float fi = (float)i;
    const float ph = fi * sh;
    const float pl = fmaf(fi, sh, -ph) + fi * sl;
    t = ((dh - ph) + (dl - pl)) * inv;
    return true;
}

// Trilinear field from the pair layout; zero outside the node box.
__device__ __forceinline__ float3 field_map(const WorldParams &w, const State &s)
{
    const int nx = w.fdims[0], ny = w.fdims[1], nz = w.fdims[2];
    int i, j, k;
    float tx, ty, tz;
    if (!map_axis(s.x, s.xl, w.forigin[0], w.forigin_lo[0], w.fspacing[0], w.fspacing_lo[0], w.finv[0], nx, i, tx) ||
        !map_axis(s.y, s.yl, w.forigin[1], w.forigin_lo[1], w.fspacing[1], w.fspacing_lo[1], w.finv[1], ny, j, ty) ||
        !map_axis(s.z, s.zl, w.forigin[2], w.forigin_lo[2], w.fspacing[2], w.fspacing_lo[2], w.finv[2], nz, k, tz))
        return make_float3(0.0f, 0.0f, 0.0f);
    const int64_t row = nx - 1;
    const float4 *p00 = w.fmap + 2 * (((int64_t)k * ny + j) * row + i);
    const float4 *p10 = p00 + 2 * row;                 // j + 1
    const float4 *p01 = p00 + 2 * row * ny;            // k + 1
    const float4 *p11 = p01 + 2 * row;                 // j + 1, k + 1
    const float4 a0 = __ldg(p00), a1 = __ldg(p00 + 1);
    const float4 b0 = __ldg(p10), b1 = __ldg(p10 + 1);
    const float4 c0 = __ldg(p01), c1 = __ldg(p01 + 1);
    const float4 d0 = __ldg(p11), d1 = __ldg(p11 + 1);
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
    ox = ay * hz - az * hy;
    oy = az * hx - ax * hz;
    oz = ax * hy - ay * hx;
}

// RK4 over path length d with B fixed: dr/ds = p/P0, dp/ds = kappa q (p x B)/P0.
// kd = kappa d, rounded once on the host.  With h = kappa q d B / P0 the stage increments are k_i = p_i x h, and the
// position increment reduces to (d/P0) (p + (k1 + k2 + k3)/6).
__device__ __forceinline__ void rk4(State &s, float3 B, float q, float d, float kd)
{
    const float px = s.px, py = s.py, pz = s.pz;
    const float P2 = p2_of(s);
    float rP = rsqrtf(P2);
    rP = rP * fmaf(-0.5f * P2 * rP, rP, 1.5f);
    const float c = (kd * q) * rP;
    const float hx = c * B.x, hy = c * B.y, hz = c * B.z;
float k1x, k1y, k1z, k2x, k2y, k2z, k3x, k3y, k3z, k4x, k4y, k4z;
    cross_h(px, py, pz, hx, hy, hz, k1x, k1y, k1z);
    cross_h(fmaf(0.5f, k1x, px), fmaf(0.5f, k1y, py), fmaf(0.5f, k1z, pz), hx, hy, hz, k2x, k2y, k2z);
    cross_h(fmaf(0.5f, k2x, px), fmaf(0.5f, k2y, py), fmaf(0.5f, k2z, pz), hx, hy, hz, k3x, k3y, k3z);
    cross_h(px + k3x, py + k3y, pz + k3z, hx, hy, hz, k4x, k4y, k4z);
    const float sixth = 1.0f / 6.0f;
    const float a = d * rP;
    acc(s.x, s.xl, a * fmaf(sixth, k1x + k2x + k3x, px));
    acc(s.y, s.yl, a * fmaf(sixth, k1y + k2y + k3y, py));
    acc(s.z, s.zl, a * fmaf(sixth, k1z + k2z + k3z, pz));
    acc(s.px, s.pxl, sixth * (k1x + 2.0f * (k2x + k3x) + k4x));
    acc(s.py, s.pyl, sixth * (k1y + 2.0f * (k2y + k3y) + k4y));
    acc(s.pz, s.pzl, sixth * (k1z + 2.0f * (k2z + k3z) + k4z));
}

// Termination test of Algorithm 1 at the start of a step.
__device__ __forceinline__ int check_stop(const WorldParams &w, const State &s, float P2)
{
    if (P2 < w.pmin2) return MT_STOPPED;
    if (ge2(s.z, s.zl, w.zmax_hi, w.zmax_lo)) return MT_EXIT_Z;
    const float ax = fabsf(s.x), axl = s.x < 0.0f ? -s.xl : s.xl;
    const float ay = fabsf(s.y), ayl = s.y < 0.0f ? -s.yl : s.yl;
    if (ge2(ax, axl, w.xmax_hi, w.xmax_lo) || ge2(ay, ayl, w.ymax_hi, w.ymax_lo)) return MT_EXIT_XY;
    return MT_ALIVE;
}

// One full step k of Algorithm 1.  Returns MT_ALIVE or the break status.
template <int GEOM, int FIELD>
__device__ __forceinline__ int step(const WorldParams &w, const SmemWorld &sw, State &s, float q, int k,
                                    uint32_t id_lo, uint32_t id_hi, const RunParams &rp)
{
    const float P2 = s.px * s.px + s.py * s.py + s.pz * s.pz;
    const int stop = check_stop(w, s, P2);
    if (stop != MT_ALIVE) return stop;
    int box = -1, mat;
    if (GEOM == MT_GEOM_BOXES) {
        box = find_box(sw, w.n_box, s);
        mat = box >= 0 ? sw.mat[box] : w.world_mat;
    } else {
        const int vm = voxel_material(w, s);
        mat = vm >= 0 ? vm : w.world_mat;
    }
    if (mat != 0) {
        const int ib = momentum_bin(w, sw, s, P2);
        const uint4 rnd = philox4x32_10(make_uint4((uint32_t)k, id_lo, id_hi, (uint32_t)rp.instance), rp.key0, rp.key1);
        const uint4 hraw = __ldg(reinterpret_cast<const uint4 *>(w.hist + (mat - 1) * w.n_pbin + ib));
        const HistRec hr = {hraw.x, hraw.y, __uint_as_float(hraw.z), __uint_as_float(hraw.w)};
        const uint32_t ab = sample_cell(w.guide + hr.guide_off, w.pairs + hr.pair_off, w.gshift, rnd.x);
        const float f = ((float)(ab >> 16) + u01(rnd.y)) * hr.fscale;
        const float th = ((float)(ab & 0xFFFFu) + u01(rnd.z)) * hr.tscale;
        float sp, cp;
        __sincosf(fmaf(6.283185307179586f, u01(rnd.w), -3.14159265358979f), &sp, &cp);   // phi - pi
        scatter(s, f, th, -cp, -sp);
    }
    float3 B = make_float3(0.0f, 0.0f, 0.0f);
    if (FIELD == MT_FIELD_BOX) {
        if (box >= 0) B = make_float3(sw.B[0][box], sw.B[1][box], sw.B[2][box]);
    } else if (FIELD == MT_FIELD_MAP) {
        B = field_map(w, s);
    }
    if (GEOM == MT_GEOM_BOXES && FIELD != MT_FIELD_NONE && box >= 0) {
        const int blk = sw.block[box];
        if (blk >= 0) {
            B.x *= sw.alpha[0][blk];
            B.y *= sw.alpha[1][blk];
            B.z *= sw.alpha[2][blk];
        }
    }
    rk4(s, B, q, rp.d, rp.kd);
    return MT_ALIVE;
}

template <int GEOM, int FIELD>
__global__ void __launch_bounds__(kBlock) transport_kernel(const WorldParams w, const mt_muon_soa soa, int64_t n,
                                                           const RunParams rp)
{
    __shared__ SmemWorld sw;
    stage_world(sw, w, rp);
    __syncthreads();
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t st0 = soa.status[m];
        if (st0 != MT_ALIVE && st0 != MT_MAX_STEPS) continue;
        State s;
        s.x = soa.x[m];
        s.y = soa.y[m];
        s.z = soa.z[m];
        s.px = soa.px[m];
        s.py = soa.py[m];
        s.pz = soa.pz[m];
        s.xl = s.yl = s.zl = s.pxl = s.pyl = s.pzl = 0.0f;
        const float q = (float)soa.q[m];
        if (!(isfinite(s.x) && isfinite(s.y) && isfinite(s.z) && isfinite(s.px) && isfinite(s.py) && isfinite(s.pz))) {
            soa.status[m] = MT_INVALID;
            continue;
        }
        const uint64_t id = (uint64_t)(rp.id_offset + m);
        const uint32_t id_lo = (uint32_t)id, id_hi = (uint32_t)(id >> 32);
        int k = soa.steps[m];
        int out = MT_MAX_STEPS;
#pragma unroll 1
        for (; k < rp.max_steps; ++k) {
            const int r = step<GEOM, FIELD>(w, sw, s, q, k, id_lo, id_hi, rp);
            if (r != MT_ALIVE) {
                out = r;
                break;
            }
        }
        soa.x[m] = s.x + s.xl;
        soa.y[m] = s.y + s.yl;
        soa.z[m] = s.z + s.zl;
        soa.px[m] = s.px + s.pxl;
        soa.py[m] = s.py + s.pyl;
        soa.pz[m] = s.pz + s.pzl;
        soa.steps[m] = k;
        soa.status[m] = (uint8_t)out;
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
static cudaError_t launch(const WorldParams &w, const mt_muon_soa &s, int64_t n, const RunParams &rp, cudaStream_t st)
{
    const int64_t blocks = (n + kBlock - 1) / kBlock;
    const unsigned grid = (unsigned)(blocks < 0x7FFFFFFF ? blocks : 0x7FFFFFFF);
    transport_kernel<GEOM, FIELD><<<grid, kBlock, 0, st>>>(w, s, n, rp);
    return cudaGetLastError();
}

}  // namespace mt

using namespace mt;

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

extern "C" mt_status mt_transport_scaled(mt_handle *h, const mt_muon_soa *s, int64_t n, float step_len,
                                         int32_t max_steps, uint64_t seed, const float *alpha, int32_t n_block,
                                         void *stream)
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
    if (n == 0) return MT_OK;
    RunParams rp;
    rp.d = step_len;
    rp.kd = (float)(0.299792458 * (double)step_len);
    rp.max_steps = max_steps;
    rp.key0 = (uint32_t)seed;
    rp.key1 = (uint32_t)(seed >> 32);
    rp.alpha = alpha;
    rp.n_block = alpha ? n_block : 0;
    rp.instance = s->instance;
    rp.id_offset = s->id_offset;
    DeviceGuard g(h->device);
    cudaStream_t cs = (cudaStream_t)stream;
    cudaError_t e;
    const WorldParams &w = h->w;
    if (w.geom_kind == MT_GEOM_BOXES) {
        if (w.field_kind == MT_FIELD_MAP)
            e = launch<MT_GEOM_BOXES, MT_FIELD_MAP>(w, *s, n, rp, cs);
        else if (w.field_kind == MT_FIELD_BOX)
            e = launch<MT_GEOM_BOXES, MT_FIELD_BOX>(w, *s, n, rp, cs);
        else
            e = launch<MT_GEOM_BOXES, MT_FIELD_NONE>(w, *s, n, rp, cs);
    } else {
        if (w.field_kind == MT_FIELD_MAP)
            e = launch<MT_GEOM_VOXELS, MT_FIELD_MAP>(w, *s, n, rp, cs);
        else
            e = launch<MT_GEOM_VOXELS, MT_FIELD_NONE>(w, *s, n, rp, cs);
    }
    if (e != cudaSuccess) return cuda_fail(e, "transport launch");
    return MT_OK;
}

extern "C" mt_status mt_transport(mt_handle *h, const mt_muon_soa *s, int64_t n, float step_len, int32_t max_steps,
                                  uint64_t seed, void *stream)
{
    return mt_transport_scaled(h, s, n, step_len, max_steps, seed, nullptr, 0, stream);
}
