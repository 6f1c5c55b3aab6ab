// api.cu -- host side of libmt: descriptor validation, sampling-table
// construction and the device-resident world (mt_create / mt_destroy).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <vector>

#include "mt_internal.cuh"

namespace mt {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

mt_status cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MT_ERR_OOM : MT_ERR_CUDA;
}

// Defined in transport.cu: repack a [nz][ny][nx][3] map into x-adjacent node pairs.
cudaError_t launch_repack_field(const float *raw, float4 *pairs, int nx, int ny, int nz, cudaStream_t st);

static void split(double v, float &hi, float &lo)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

static bool finite3(const double v[3])
{
    return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]);
}

// Sampling tables of one histogram set (cells are encoded as (a << 16) | b with
// a the f bin and b the theta bin).  T_j = floor(2^32 S_j / S_total) with S_j
// the left-to-right FP64 prefix sum; the selectable cells (T_{c-1} < T_c) with
// their upper thresholds U_k form the pair list; the guide table over the
// 2^gbits equal slices of the draw space stores either the answer cell (when
// no threshold falls inside the slice) or the pair range to search.
static int log2_exact(int64_t v)
{
    int b = 0;
    while (((int64_t)1 << b) < v) ++b;
    return ((int64_t)1 << b) == v ? b : -1;
}

// Alias columns of one histogram from its thresholds T (T[ncell-1] = 2^32):
// the cells' integer masses T_c - T_{c-1} are dealt into ncell columns of
// capacity 2^(32-n) by Vose's construction (small/large stacks filled in cell
// order, popped from the top); column j keeps q_j of its own cell, Prob_j =
// q_j 2^n (saturated at 2^32 - 1 for a full column), and takes the rest from
// its alias.  Entries {Prob_j, alias cell encoded (a << 16) | b}.
static void alias_columns(const std::vector<uint64_t> &T, int ncell, int ntheta, uint2 *out)
{
    const int n = log2_exact(ncell);
    const uint64_t cap = 1ull << (32 - n);
    std::vector<uint64_t> q(ncell);
    std::vector<int> small, large;
    small.reserve(ncell);
    large.reserve(ncell);
    uint64_t prev = 0;
    for (int c = 0; c < ncell; ++c) {
        const uint64_t t = std::max(T[c], prev);
        q[c] = t - prev;
        prev = t;
        (q[c] < cap ? small : large).push_back(c);
    }
    auto enc = [ntheta](int c) { return ((uint32_t)(c / ntheta) << 16) | (uint32_t)(c % ntheta); };
    while (!small.empty() && !large.empty()) {
        const int sc = small.back();
        small.pop_back();
        const int lc = large.back();
        large.pop_back();
        out[sc] = make_uint2((uint32_t)(q[sc] << n), enc(lc));
        q[lc] -= cap - q[sc];
        (q[lc] < cap ? small : large).push_back(lc);
    }
    for (const int c : large) out[c] = make_uint2(0xFFFFFFFFu, enc(c));
    for (const int c : small) out[c] = make_uint2(0xFFFFFFFFu, enc(c));   // not reached with exact masses
}

static mt_status build_tables(const mt_hist_desc *h, int gbits, std::vector<HistRec> &rec,
                              std::vector<uint32_t> &guide, std::vector<uint2> &pairs, std::vector<uint2> &alias)
{
    const bool use_alias = h->sampler == MT_SAMPLER_ALIAS;
    const int ncell = h->nf * h->ntheta;
    const int64_t n_hist = (int64_t)h->n_mat * h->n_pbin;
    const int G = 1 << gbits;
    const int shift = 32 - gbits;
    std::vector<uint64_t> T(ncell);
    std::vector<uint64_t> U;
    std::vector<uint32_t> cells;
    rec.resize(n_hist);
    guide.resize(use_alias ? 0 : (size_t)n_hist * G);
    pairs.clear();
    alias.resize(use_alias ? (size_t)n_hist * ncell : 0);
    for (int64_t hi = 0; hi < n_hist; ++hi) {
        const double *w = h->weights + hi * ncell;
        double total = 0.0;
        for (int j = 0; j < ncell; ++j) {
            if (!(w[j] >= 0.0) || !std::isfinite(w[j])) {
                set_error("histogram %lld cell %d: weight %g is negative or not finite", (long long)hi, j, w[j]);
                return MT_ERR_TABLE;
            }
            total += w[j];
        }
        if (!(total > 0.0) || !std::isfinite(total)) {
            set_error("histogram %lld has no positive finite mass", (long long)hi);
            return MT_ERR_TABLE;
        }
        double S = 0.0;
        for (int j = 0; j < ncell - 1; ++j) {
            S += w[j];
            T[j] = (uint64_t)std::floor(S / total * 4294967296.0);
        }
        T[ncell - 1] = 1ull << 32;
        if (use_alias) {
            alias_columns(T, ncell, h->ntheta, alias.data() + (size_t)hi * ncell);
            rec[hi].guide_off = (uint32_t)(hi * ncell);
            rec[hi].pair_off = 0;
            rec[hi].fscale = (float)(h->f_max[hi] / h->nf);
            rec[hi].tscale = (float)(h->theta_max[hi] / h->ntheta);
            continue;
        }
        U.clear();
        cells.clear();
        uint64_t prev = 0;
        for (int c = 0; c < ncell; ++c) {
            if (T[c] > prev) {
                U.push_back(T[c]);
                cells.push_back(((uint32_t)(c / h->ntheta) << 16) | (uint32_t)(c % h->ntheta));
            }
            prev = T[c] > prev ? T[c] : prev;
        }
        const int m = (int)cells.size();
        rec[hi].pair_off = (uint32_t)pairs.size();
        rec[hi].guide_off = (uint32_t)(hi * G);
        const double fm = h->f_max[hi], tm = h->theta_max[hi];
        rec[hi].fscale = (float)(fm / h->nf);
        rec[hi].tscale = (float)(tm / h->ntheta);
        for (int k = 0; k < m; ++k)
            pairs.push_back(make_uint2((uint32_t)(U[k] > 0xFFFFFFFFull ? 0xFFFFFFFFull : U[k]), cells[k]));
        int lo = 0;
        for (int g = 0; g < G; ++g) {
            const uint64_t start = (uint64_t)g << shift;
            const uint64_t last = (((uint64_t)g + 1) << shift) - 1;
            while (lo < m - 1 && U[lo] < start) ++lo;
            int hi2 = lo;
            while (hi2 < m - 1 && U[hi2] <= last) ++hi2;
            uint32_t e;
            if (hi2 == lo)
                e = cells[lo];
            else
                e = 0x80000000u | (uint32_t)lo | ((uint32_t)(hi2 - lo) << 15);
            guide[(size_t)hi * G + g] = e;
        }
    }
    return MT_OK;
}

mt_status validate_hist(const mt_hist_desc *h)
{
    if (!h) {
        set_error("null histogram descriptor");
        return MT_ERR_INVALID_ARG;
    }
    if (h->n_mat < 1 || h->n_mat > MT_MAX_MATERIALS || h->n_pbin < 1 || h->n_pbin > MT_MAX_PBINS) {
        set_error("hist: n_mat %d / n_pbin %d out of range", h->n_mat, h->n_pbin);
        return MT_ERR_INVALID_ARG;
    }
    if (h->nf < 1 || h->ntheta < 1 || (int64_t)h->nf * h->ntheta < 2 || (int64_t)h->nf * h->ntheta > MT_MAX_CELLS) {
        set_error("hist: nf*ntheta = %lld outside [2, %d]", (long long)h->nf * h->ntheta, MT_MAX_CELLS);
        return MT_ERR_INVALID_ARG;
    }
    if (h->p_edges) {
        if (h->p_edges[0] != h->p_lo || h->p_edges[h->n_pbin] != h->p_hi) {
            set_error("hist: p_edges must start at p_lo and end at p_hi");
            return MT_ERR_INVALID_ARG;
        }
        for (int i = 0; i < h->n_pbin; ++i)
            if (!(h->p_edges[i + 1] > h->p_edges[i] * (1.0 + 1e-5))) {
                set_error("hist: p_edges must increase by at least 1e-5 relatively (edge %d)", i + 1);
                return MT_ERR_INVALID_ARG;
            }
    }
    if (h->axes != MT_AXES_LINEAR && h->axes != MT_AXES_LOG) {
        set_error("hist: unknown axes %d", h->axes);
        return MT_ERR_INVALID_ARG;
    }
    if (h->axes == MT_AXES_LOG) {
        if (!h->f_min || !h->theta_min) {
            set_error("hist: log axes need f_min and theta_min");
            return MT_ERR_INVALID_ARG;
        }
        for (int64_t i = 0; i < (int64_t)h->n_mat * h->n_pbin; ++i)
            if (!(h->f_min[i] > 0.0) || !(h->f_min[i] < h->f_max[i]) || !(h->theta_min[i] > 0.0) ||
                !(h->theta_min[i] < h->theta_max[i])) {
                set_error("hist: log axes need 0 < f_min < f_max and 0 < theta_min < theta_max (histogram %lld)",
                          (long long)i);
                return MT_ERR_INVALID_ARG;
            }
    }
    if (h->sampler != MT_SAMPLER_ICDF && h->sampler != MT_SAMPLER_ALIAS) {
        set_error("hist: unknown sampler %d", h->sampler);
        return MT_ERR_INVALID_ARG;
    }
    if (h->sampler == MT_SAMPLER_ALIAS && (log2_exact(h->nf) < 0 || log2_exact(h->ntheta) < 0)) {
        set_error("hist: the alias sampler needs nf and ntheta powers of two (got %d x %d)", h->nf, h->ntheta);
        return MT_ERR_INVALID_ARG;
    }
    if (!(h->p_lo > 0.0) || !(h->p_hi > h->p_lo) || !std::isfinite(h->p_hi)) {
        set_error("hist: need 0 < p_lo < p_hi");
        return MT_ERR_INVALID_ARG;
    }
    if (!h->weights || !h->f_max || !h->theta_max) {
        set_error("hist: null array");
        return MT_ERR_INVALID_ARG;
    }
    for (int64_t i = 0; i < (int64_t)h->n_mat * h->n_pbin; ++i)
        if (!(h->f_max[i] > 0.0) || !(h->theta_max[i] > 0.0) || !std::isfinite(h->f_max[i]) ||
            !std::isfinite(h->theta_max[i])) {
            set_error("hist: f_max/theta_max[%lld] must be positive and finite", (long long)i);
            return MT_ERR_INVALID_ARG;
        }
    return MT_OK;
}

mt_status validate_geometry(const mt_geometry_desc *g, int n_mat)
{
    if (!g) {
        set_error("null geometry descriptor");
        return MT_ERR_INVALID_ARG;
    }
    if (!(g->x_max > 0.0) || !(g->y_max > 0.0) || std::isnan(g->z_max) || !(g->p_min >= 0.0) ||
        !std::isfinite(g->p_min)) {
        set_error("geometry: bad world bounds or p_min");
        return MT_ERR_INVALID_ARG;
    }
    if (g->world_material < 0 || g->world_material > n_mat) {
        set_error("geometry: world material %d outside [0, %d]", g->world_material, n_mat);
        return MT_ERR_INVALID_ARG;
    }
    if (g->kind == MT_GEOM_BOXES) {
        if (g->n_boxes < 0 || g->n_boxes > MT_MAX_BOXES || (g->n_boxes > 0 && !g->boxes)) {
            set_error("geometry: n_boxes %d outside [0, %d] or null boxes", g->n_boxes, MT_MAX_BOXES);
            return MT_ERR_INVALID_ARG;
        }
        for (int b = 0; b < g->n_boxes; ++b) {
            const mt_box &bx = g->boxes[b];
            if (!finite3(bx.lo) || !finite3(bx.hi) || !finite3(bx.B) || bx.material < 0 ||
                bx.material > n_mat || bx.block_id < -1 || bx.block_id >= MT_MAX_BOXES) {
                set_error("geometry: box %d invalid (material %d, block %d)", b, bx.material, bx.block_id);
                return MT_ERR_INVALID_ARG;
            }
        }
    } else if (g->kind == MT_GEOM_VOXELS) {
        if (!g->voxels || g->vox_dims[0] < 1 || g->vox_dims[1] < 1 || g->vox_dims[2] < 1 ||
            !finite3(g->vox_origin) || !(g->vox_spacing[0] > 0) || !(g->vox_spacing[1] > 0) ||
            !(g->vox_spacing[2] > 0)) {
            set_error("geometry: bad voxel grid");
            return MT_ERR_INVALID_ARG;
        }
        const int64_t nv = (int64_t)g->vox_dims[0] * g->vox_dims[1] * g->vox_dims[2];
        for (int64_t i = 0; i < nv; ++i)
            if (g->voxels[i] > n_mat) {
                set_error("geometry: voxel %lld material %d > n_mat", (long long)i, g->voxels[i]);
                return MT_ERR_INVALID_ARG;
            }
    } else if (g->kind == MT_GEOM_POLYHEDRA) {
        if (g->n_polys < 0 || g->n_polys > MT_MAX_BOXES || (g->n_polys > 0 && !g->polys)) {
            set_error("geometry: n_polys %d outside [0, %d] or null polys", g->n_polys, MT_MAX_BOXES);
            return MT_ERR_INVALID_ARG;
        }
        for (int b = 0; b < g->n_polys; ++b) {
            const mt_polyhedron &P = g->polys[b];
            bool ok = std::isfinite(P.z0) && std::isfinite(P.z1) && P.z1 > P.z0 && finite3(P.B) &&
                      P.material >= 0 && P.material <= n_mat && P.block_id >= -1 && P.block_id < MT_MAX_BOXES;
            for (int end = 0; end < 2 && ok; ++end) {
                const double(*q)[2] = end ? P.top : P.bottom;
                for (int i = 0; i < 4 && ok; ++i) {
                    const int j = (i + 1) % 4, k = (i + 2) % 4;
                    ok = std::isfinite(q[i][0]) && std::isfinite(q[i][1]);
                    // strictly convex and counter-clockwise: every turn is to the left
                    const double c = (q[j][0] - q[i][0]) * (q[k][1] - q[j][1]) - (q[j][1] - q[i][1]) * (q[k][0] - q[j][0]);
                    ok = ok && c > 0.0;
                }
            }
            if (!ok) {
                set_error("geometry: solid %d invalid (z0 < z1, strictly convex counter-clockwise quadrilaterals, "
                          "material %d, block %d)", b, P.material, P.block_id);
                return MT_ERR_INVALID_ARG;
            }
        }
    } else {
        set_error("geometry: unknown kind %d", g->kind);
        return MT_ERR_INVALID_ARG;
    }
    return MT_OK;
}

mt_status validate_field(const mt_field_desc *f, const mt_geometry_desc *g)
{
    if (!f) {
        set_error("null field descriptor");
        return MT_ERR_INVALID_ARG;
    }
    if (f->per_stage != 0 && (f->per_stage != 1 || f->kind != MT_FIELD_MAP)) {
        set_error("field: per_stage must be 0, or 1 with MT_FIELD_MAP");
        return MT_ERR_INVALID_ARG;
    }
    if (f->kind == MT_FIELD_MAP || f->kind == MT_FIELD_MAP_NEAREST) {
        if (!f->B || f->dims[0] < 2 || f->dims[1] < 2 || f->dims[2] < 2 || !finite3(f->origin) ||
            !(f->spacing[0] > 0) || !(f->spacing[1] > 0) || !(f->spacing[2] > 0)) {
            set_error("field: bad map (dims >= 2, spacing > 0, B non-null)");
            return MT_ERR_INVALID_ARG;
        }
        const int64_t nv = 3ll * f->dims[0] * f->dims[1] * f->dims[2];
        for (int64_t i = 0; i < nv; ++i)
            if (!std::isfinite(f->B[i])) {
                set_error("field: non-finite value at %lld", (long long)i);
                return MT_ERR_INVALID_ARG;
            }
    } else if (f->kind == MT_FIELD_BOX) {
        if (g->kind == MT_GEOM_VOXELS) {
            set_error("field: per-box field needs box or polyhedron geometry");
            return MT_ERR_INVALID_ARG;
        }
    } else if (f->kind != MT_FIELD_NONE) {
        set_error("field: unknown kind %d", f->kind);
        return MT_ERR_INVALID_ARG;
    }
    return MT_OK;
}

template <class T>
static mt_status upload(DevOwner &own, const T *src, size_t count, const char *what, const T **dst)
{
    size_t nb = count * sizeof(T);
    if (nb == 0) nb = sizeof(T);
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, nb);
    if (e != cudaSuccess) return cuda_fail(e, what);
    own.bufs.push_back(p);
    own.bytes += (int64_t)nb;
    if (count) {
        e = cudaMemcpy(p, src, count * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, what);
    }
    *dst = (const T *)p;
    return MT_OK;
}

void DevOwner::release()
{
    for (void *p : bufs)
        if (p) cudaFree(p);
    bufs.clear();
    bytes = 0;
}

// Sampling tables and bin edges of a histogram set (validated) into w.
mt_status build_hist(const mt_hist_desc *hd, WorldParams &w, DevOwner &own)
{
    const int ncell = hd->nf * hd->ntheta;
    // At least four guide slots per cell, up to 32K: a slot that holds a cell
    // boundary sends its draws to the binary search, and a warp waits for its
    // longest search.  Measured on shield1e6 (8192 cells): one slot per cell
    // 5.33e10 muon-steps/s, two 5.39e10, four 5.42e10, eight 5.42e10 (the guide
    // rows of its 192 histograms grow from 6 to 24 MB at four).
    int gbits = 12;
    while ((1 << gbits) < 4 * ncell && gbits < 15) ++gbits;
    std::vector<HistRec> rec;
    std::vector<uint32_t> guide;
    std::vector<uint2> pairs;
    std::vector<uint2> alias;
    mt_status st = build_tables(hd, gbits, rec, guide, pairs, alias);
    if (st != MT_OK) return st;
    std::vector<float2> e2(hd->n_pbin + 1);
    w.pbin_custom = hd->p_edges ? 1 : 0;
    for (int k = 0; k <= hd->n_pbin; ++k) {
        const double E = hd->p_edges ? hd->p_edges[k] : hd->p_lo * std::pow(hd->p_hi / hd->p_lo, (double)k / hd->n_pbin);
        float a, b;
        split(E * E, a, b);
        e2[k] = make_float2(a, b);
    }
    if ((st = upload(own, rec.data(), rec.size(), "histogram records", &w.hist)) != MT_OK) return st;
    w.axes = hd->axes;
    if (hd->axes == MT_AXES_LOG) {
        const int64_t nh = (int64_t)hd->n_mat * hd->n_pbin;
        // per histogram two records (v0, log2 cell width as hi + lo, 0) for f and t
        std::vector<float4> hl(2 * nh);
        for (int64_t i = 0; i < nh; ++i) {
            float dh, dl;
            split(std::log2(hd->f_max[i] / hd->f_min[i]) / hd->nf, dh, dl);
            hl[2 * i] = make_float4((float)hd->f_min[i], dh, dl, 0.0f);
            split(std::log2(hd->theta_max[i] / hd->theta_min[i]) / hd->ntheta, dh, dl);
            hl[2 * i + 1] = make_float4((float)hd->theta_min[i], dh, dl, 0.0f);
        }
        if ((st = upload(own, hl.data(), hl.size(), "log axes", &w.hist_log)) != MT_OK) return st;
    }
    w.sampler = hd->sampler;
    if (hd->sampler == MT_SAMPLER_ALIAS) {
        if ((st = upload(own, alias.data(), alias.size(), "alias tables", &w.alias)) != MT_OK) return st;
        w.alias_bits = log2_exact((int64_t)hd->nf * hd->ntheta);
        w.theta_bits = log2_exact(hd->ntheta);
    } else {
        if ((st = upload(own, guide.data(), guide.size(), "guide tables", &w.guide)) != MT_OK) return st;
        if ((st = upload(own, pairs.data(), pairs.size(), "threshold pairs", &w.pairs)) != MT_OK) return st;
    }
    if ((st = upload(own, e2.data(), e2.size(), "bin edges", &w.e2)) != MT_OK) return st;
    w.n_mat = hd->n_mat;
    w.n_pbin = hd->n_pbin;
    w.nf = hd->nf;
    w.ntheta = hd->ntheta;
    w.gshift = 32 - gbits;
    w.log2_plo = (float)std::log2(hd->p_lo);
    w.pbin_scale = (float)(hd->n_pbin / std::log2(hd->p_hi / hd->p_lo));
    {
        // Error of the kernel's bin coordinate u = (0.5 log2(P^2) - log2 p_lo) * scale
        // near the bin faces (P in [p_lo / 2, 2 p_hi]): the log2 intrinsic (2^-22
        // absolute on [0.5, 2], else 2 ulp), the roundings of the fma and the
        // product, and those of log2 p_lo and scale as stored.
        auto ulp = [](double v) { return v > 0.0 ? std::ldexp(1.0, std::ilogb(v) - 23) : std::ldexp(1.0, -149); };
        const double lp = std::fabs(std::log2(hd->p_lo)), scale = w.pbin_scale;
        const double L = std::max(std::fabs(2.0 * std::log2(hd->p_lo) - 2.0), std::fabs(2.0 * std::log2(hd->p_hi) + 2.0));
        const double umax = hd->n_pbin + 2.0;
        const double err = 0.5 * std::max(std::ldexp(1.0, -22), 2.0 * ulp(L)) * scale + 0.5 * ulp(0.5 * L + lp) * scale +
                           0.5 * ulp(umax) + umax * std::ldexp(1.0, -24) + 0.5 * ulp(lp) * scale;
        const double eps = std::max(4.0 * err, 1e-4);
        w.pbin_eps = eps < 0.1 ? (float)eps : 1.0f;   // 1: every estimate goes to the edges
    }
    return MT_OK;
}

// Smallest value over t in [0, 1] of S_i(c, t) for edge i of solid P at the
// point c, with the slice interpolated linearly in t (Eq. 2's S_i is then a
// quadratic in t).
static double edge_min_over_z(const mt_polyhedron &P, int i, const double c[2])
{
    const int j = (i + 1) % 4;
    const double e0x = P.bottom[j][0] - P.bottom[i][0], e0y = P.bottom[j][1] - P.bottom[i][1];
    const double e1x = P.top[j][0] - P.top[i][0], e1y = P.top[j][1] - P.top[i][1];
    const double dex = e1x - e0x, dey = e1y - e0y;
    const double dvx = P.top[i][0] - P.bottom[i][0], dvy = P.top[i][1] - P.bottom[i][1];
    const double d0x = c[0] - P.bottom[i][0], d0y = c[1] - P.bottom[i][1];
    const double A = e0x * d0y - e0y * d0x;
    const double B = dex * d0y - e0x * dvy - dey * d0x + e0y * dvx;
    const double C = -dex * dvy + dey * dvx;
    double m = std::min(A, A + B + C);
    if (C > 0.0) {
        const double t = -B / (2.0 * C);
        if (t > 0.0 && t < 1.0) m = std::min(m, A + t * (B + t * C));
    }
    return m;
}

// An axis-aligned rectangle inside every slice of solid P, shrunk by `margin`
// on each side: the largest rectangle centred on the mean of the eight
// vertices, with the half-widths of the narrower end scaled by s, for which
// every edge's S_i stays positive at all four corners and every z (checked
// with edge_min_over_z; S_i is linear in the point, so the corners bound the
// rectangle).  Empty (lo > hi) when no s in [0, 1] passes.
static void inner_box(const mt_polyhedron &P, double margin, double out[4])
{
    double cx = 0.0, cy = 0.0, hx = 1e300, hy = 1e300;
    for (int end = 0; end < 2; ++end) {
        const double(*v)[2] = end ? P.top : P.bottom;
        double x0 = v[0][0], x1 = v[0][0], y0 = v[0][1], y1 = v[0][1];
        for (int i = 0; i < 4; ++i) {
            cx += v[i][0] / 8.0;
            cy += v[i][1] / 8.0;
            x0 = std::min(x0, v[i][0]);
            x1 = std::max(x1, v[i][0]);
            y0 = std::min(y0, v[i][1]);
            y1 = std::max(y1, v[i][1]);
        }
        hx = std::min(hx, 0.5 * (x1 - x0));
        hy = std::min(hy, 0.5 * (y1 - y0));
    }
    auto ok = [&](double s) {
        const double r[4] = {cx - s * hx - margin, cx + s * hx + margin, cy - s * hy - margin, cy + s * hy + margin};
        for (int i = 0; i < 4; ++i)
            for (int k = 0; k < 4; ++k) {
                const double c[2] = {r[k & 1], r[2 + (k >> 1)]};
                if (!(edge_min_over_z(P, i, c) > 0.0)) return false;
            }
        return true;
    };
    double lo = 0.0, hi = 1.0;
    if (!ok(0.0)) {
        out[0] = 1.0;
        out[1] = -1.0;
        out[2] = 1.0;
        out[3] = -1.0;
        return;
    }
    for (int it = 0; it < 40; ++it) {
        const double mid = 0.5 * (lo + hi);
        (ok(mid) ? lo : hi) = mid;
    }
    out[0] = cx - lo * hx;
    out[1] = cx + lo * hx;
    out[2] = cy - lo * hy;
    out[3] = cy + lo * hy;
}

// z-slab candidate index of boxes or solids with z ranges [zlo_b, zhi_b):
// slab s of kZSlabs over the union of the ranges holds every volume whose z
// range meets the slab or its two neighbours (the slab of a point is computed
// in FP32 and may be off by one near a slab face; the exact test decides).
static mt_status build_zslabs(const double *zlo_b, const double *zhi_b, int n, WorldParams &w, DevOwner &own)
{
    std::vector<uint32_t> zmask(kZSlabs, 0u);
    double zlo = 0.0, zhi = 1.0;
    if (n > 0) {
        zlo = zlo_b[0];
        zhi = zhi_b[0];
        for (int b = 1; b < n; ++b) {
            zlo = std::min(zlo, zlo_b[b]);
            zhi = std::max(zhi, zhi_b[b]);
        }
        if (!(zhi > zlo)) zhi = zlo + 1.0;
    }
    const double dz = (zhi - zlo) / kZSlabs;
    for (int b = 0; b < n; ++b) {
        if (!(zhi_b[b] > zlo_b[b])) continue;   // empty: never contains a point
        int s0 = (int)std::floor((zlo_b[b] - zlo) / dz) - 1;
        int s1 = (int)std::floor((zhi_b[b] - zlo) / dz) + 1;
        s0 = std::max(s0, 0);
        s1 = std::min(s1, kZSlabs - 1);
        for (int sl = s0; sl <= s1; ++sl) zmask[sl] |= 1u << b;
    }
    mt_status st = upload(own, zmask.data(), zmask.size(), "z-slab index", &w.zmask);
    if (st != MT_OK) return st;
    w.zslab_lo = (float)zlo;
    w.zslab_inv = (float)(1.0 / dz);
    return MT_OK;
}

// Position frame of a world (see WorldParams): the field map's node grid when
// there is a map, else metres.  Positions are converted to frame units in
// double and stored as hi + lo pairs.
struct Frame {
    double o[3], s[3];
    double u(int a, double v) const { return (v - o[a]) / s[a]; }   // metres -> units
    double len(int a, double v) const { return v / s[a]; }          // a length along axis a
};

static Frame frame_of(const mt_field_desc *f)
{
    Frame F;
    const bool map = f && (f->kind == MT_FIELD_MAP || f->kind == MT_FIELD_MAP_NEAREST);
    for (int a = 0; a < 3; ++a) {
        F.o[a] = map ? f->origin[a] : 0.0;
        F.s[a] = map ? f->spacing[a] : 1.0;
    }
    return F;
}

// Geometry and world bounds (validated) into w, in the frame that the field
// desc f sets (frame_of).
mt_status build_geometry(const mt_geometry_desc *g, const mt_field_desc *f, WorldParams &w, DevOwner &own)
{
    mt_status st;
    const Frame F = frame_of(f);
    for (int a = 0; a < 3; ++a) {
        split(F.o[a], w.fro_h[a], w.fro_l[a]);
        split(F.s[a], w.frs_h[a], w.frs_l[a]);
        split(1.0 / F.s[a], w.fri_h[a], w.fri_l[a]);
    }
    w.geom_kind = g->kind;
    w.world_mat = g->world_material;
    split(F.u(0, g->x_max), w.xmax_hi, w.xmax_lo);
    split(F.u(0, -g->x_max), w.xmin_hi, w.xmin_lo);
    split(F.u(1, g->y_max), w.ymax_hi, w.ymax_lo);
    split(F.u(1, -g->y_max), w.ymin_hi, w.ymin_lo);
    split(F.u(2, g->z_max), w.zmax_hi, w.zmax_lo);
    w.pmin2 = (float)(g->p_min * g->p_min);
    if (g->kind == MT_GEOM_BOXES) {
        std::vector<DevBox> boxes(g->n_boxes);
        for (int b = 0; b < g->n_boxes; ++b) {
            const mt_box &s = g->boxes[b];
            DevBox &d = boxes[b];
            for (int a = 0; a < 3; ++a) {
                split(F.u(a, s.lo[a]), d.lo_hi[a], d.lo_lo[a]);
                split(F.u(a, s.hi[a]), d.hi_hi[a], d.hi_lo[a]);
                d.B[a] = (float)s.B[a];
            }
            d.material = s.material;
            d.block = s.block_id;
            d.pad = 0;
        }
        w.n_box = g->n_boxes;
        if ((st = upload(own, boxes.data(), boxes.size(), "boxes", &w.boxes)) != MT_OK) return st;
        std::vector<double> zlo(g->n_boxes), zhi(g->n_boxes);
        for (int b = 0; b < g->n_boxes; ++b) {
            zlo[b] = F.u(2, g->boxes[b].lo[2]);
            zhi[b] = F.u(2, g->boxes[b].hi[2]);
        }
        if ((st = build_zslabs(zlo.data(), zhi.data(), g->n_boxes, w, own)) != MT_OK) return st;
    } else if (g->kind == MT_GEOM_POLYHEDRA) {
        // Per solid:
        //  - a DevBox record with the bounding box (x, y grown by 1e-4 m, z exactly
        //    [z0, z1)), material, block and field, staged into shared memory and
        //    indexed by the z-slab grid like boxes;
        //  - the inner rectangle (shared memory), a rectangle inside every slice,
        //    1e-4 m clear of the sides;
        //  - five float4 for the FP32 side test: {z0 hi, z0 lo, 1/(z1 - z0), bound},
        //    {bx0, by0, bx1, by1}, {bx2, by2, bx3, by3} (bottom vertices),
        //    {dx0, dy0, dx1, dy1}, {dx2, dy2, dx3, dy3} (top - bottom), and a spare;
        //  - the FP64 data z0, z1, bottom[4][2], top[4][2] for undecided tests.
        //  All of it is in frame units: the solid is mapped by the frame's
        //  diagonal scaling, which keeps it a convex solid with the same vertex
        //  order (so Eq. 2's signs), and its bounding-box margin and the inner
        //  rectangle's clearance are 1e-4 m along each axis.
        const int n = g->n_polys;
        const double margin_m = 1e-4;
        std::vector<DevBox> recs(n);
        std::vector<float4> pf((size_t)n * 6), pin(n);
        std::vector<double> pd((size_t)n * 18), zlo(n), zhi(n);
        for (int b = 0; b < n; ++b) {
            const mt_polyhedron &Pm = g->polys[b];
            mt_polyhedron P = Pm;
            P.z0 = F.u(2, Pm.z0);
            P.z1 = F.u(2, Pm.z1);
            for (int i = 0; i < 4; ++i)
                for (int c = 0; c < 2; ++c) {
                    P.bottom[i][c] = F.u(c, Pm.bottom[i][c]);
                    P.top[i][c] = F.u(c, Pm.top[i][c]);
                }
            const double mx = F.len(0, margin_m), my = F.len(1, margin_m);
            double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300, M1 = 0.0, M2 = 0.0, E = 0.0;
            for (int end = 0; end < 2; ++end) {
                const double(*v)[2] = end ? P.top : P.bottom;
                for (int i = 0; i < 4; ++i) {
                    const int j = (i + 1) % 4;
                    x0 = std::min(x0, v[i][0]);
                    x1 = std::max(x1, v[i][0]);
                    y0 = std::min(y0, v[i][1]);
                    y1 = std::max(y1, v[i][1]);
                    M1 = std::max(M1, std::max(std::fabs(v[i][0]), std::fabs(v[i][1])));
                    E = std::max(E, std::fabs(v[j][0] - v[i][0]) + std::fabs(v[j][1] - v[i][1]));
                }
            }
            for (int i = 0; i < 4; ++i)
                for (int c = 0; c < 2; ++c) M2 = std::max(M2, std::fabs(P.top[i][c] - P.bottom[i][c]));
            DevBox &d = recs[b];
            memset(&d, 0, sizeof(d));
            const double lo3[3] = {x0 - mx, y0 - my, P.z0}, hi3[3] = {x1 + mx, y1 + my, P.z1};
            for (int a = 0; a < 3; ++a) {
                split(lo3[a], d.lo_hi[a], d.lo_lo[a]);
                split(hi3[a], d.hi_hi[a], d.hi_lo[a]);
                d.B[a] = (float)P.B[a];
            }
            d.material = P.material;
            d.block = P.block_id;
            zlo[b] = P.z0;
            zhi[b] = P.z1;
            // error bound of the FP32 side test (step.cuh: in_solid_sides):
            // 100 eps (E + 2M)(D + 2M), E the largest |e_x| + |e_y| of an edge at
            // either end (edges move linearly in z), D the largest |dx| + |dy|
            // over the bounding box, M = M1 + M2
            const double M = M1 + M2;
            const double D = (x1 - x0) + (y1 - y0) + 2.0 * (mx + my);
            const double bound = 100.0 * std::ldexp(1.0, -24) * (E + 2.0 * M) * (D + 2.0 * M);
            float z0h, z0l;
            split(P.z0, z0h, z0l);
            float bv[8], dv[8];
            for (int i = 0; i < 4; ++i)
                for (int c = 0; c < 2; ++c) {
                    bv[2 * i + c] = (float)P.bottom[i][c];
                    dv[2 * i + c] = (float)(P.top[i][c] - P.bottom[i][c]);
                }
            float4 *q = &pf[(size_t)b * 6];
            q[0] = make_float4(z0h, z0l, (float)(1.0 / (P.z1 - P.z0)), (float)(bound * (1.0 + 1e-6)));
            q[1] = make_float4(bv[0], bv[1], bv[2], bv[3]);
            q[2] = make_float4(bv[4], bv[5], bv[6], bv[7]);
            q[3] = make_float4(dv[0], dv[1], dv[2], dv[3]);
            q[4] = make_float4(dv[4], dv[5], dv[6], dv[7]);
            q[5] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            // inner rectangle found in metres (its clearance is a length), then mapped
            double ib[4];
            inner_box(Pm, margin_m, ib);
            pin[b] = make_float4((float)F.u(0, ib[0]), (float)F.u(0, ib[1]), (float)F.u(1, ib[2]), (float)F.u(1, ib[3]));
            if (ib[0] <= ib[1]) {   // keep the float rectangle inside the exact one
                pin[b].x = std::nextafter(pin[b].x, INFINITY);
                pin[b].y = std::nextafter(pin[b].y, -INFINITY);
                pin[b].z = std::nextafter(pin[b].z, INFINITY);
                pin[b].w = std::nextafter(pin[b].w, -INFINITY);
            }
            // the FP64 fallback's data: the solid mapped to frame units in FP64
            // (Eq. 2's signs are those of the solid as given)
            double *r = &pd[(size_t)b * 18];
            r[0] = P.z0;
            r[1] = P.z1;
            for (int i = 0; i < 4; ++i)
                for (int c = 0; c < 2; ++c) {
                    r[2 + 2 * i + c] = P.bottom[i][c];
                    r[10 + 2 * i + c] = P.top[i][c];
                }
        }
        w.n_box = n;
        if ((st = upload(own, recs.data(), recs.size(), "solid records", &w.boxes)) != MT_OK) return st;
        if ((st = upload(own, pf.data(), pf.size(), "solids", &w.poly)) != MT_OK) return st;
        if ((st = upload(own, pin.data(), pin.size(), "solid inner rectangles", &w.pinner)) != MT_OK) return st;
        if ((st = upload(own, pd.data(), pd.size(), "solids (FP64)", &w.poly64)) != MT_OK) return st;
        if ((st = build_zslabs(zlo.data(), zhi.data(), n, w, own)) != MT_OK) return st;
    } else {
        const size_t nv = (size_t)g->vox_dims[0] * g->vox_dims[1] * g->vox_dims[2];
        if ((st = upload(own, g->voxels, nv, "voxels", &w.vox)) != MT_OK) return st;
        w.n_box = 0;
        for (int a = 0; a < 3; ++a) {
            w.vdims[a] = g->vox_dims[a];
            split(F.u(a, g->vox_origin[a]), w.vorigin[a], w.vorigin_lo[a]);
            split(F.len(a, g->vox_spacing[a]), w.vspacing[a], w.vspacing_lo[a]);
            w.vinv[a] = (float)(1.0 / F.len(a, g->vox_spacing[a]));
        }
    }
    return MT_OK;
}

// xy grid of the live list's spatial order: the map's xy cells merged 2 x 2
// (measured on shield1e6 and tapered1e6 faster than single cells, whose
// histogram is 4 times longer), or 4 x 4, ... until at most kSortBins remain.
#ifndef MT_SORT_SHIFT_MIN
#define MT_SORT_SHIFT_MIN 1
#endif
static void set_sort_grid(WorldParams &w)
{
    const int cx = w.fdims[0] - 1, cy = w.fdims[1] - 1;
    w.sort_shift = 0;
    w.sort_nx = 0;
    w.sort_bins = 0;
    if (cx < 1 || cy < 1) return;
    int sh = MT_SORT_SHIFT_MIN;
    while ((int64_t)(((cx - 1) >> sh) + 1) * (((cy - 1) >> sh) + 1) > kSortBins) ++sh;
    w.sort_shift = sh;
    w.sort_nx = ((cx - 1) >> sh) + 1;
    w.sort_bins = w.sort_nx * (((cy - 1) >> sh) + 1);
}

// Field (validated) into w; a map is uploaded and repacked into x-adjacent node pairs.
mt_status build_field(const mt_field_desc *f, WorldParams &w, DevOwner &own)
{
    w.field_kind = f->kind;
    w.field_per_stage = f->per_stage;
    if (f->kind == MT_FIELD_MAP_NEAREST) {
        // nodes as float4 (Bx, By, Bz, 0); cells of the nearest-node lookup are the
        // nodes' Voronoi cells, i.e. a grid whose origin is half a spacing below
        const int64_t nn = (int64_t)f->dims[0] * f->dims[1] * f->dims[2];
        std::vector<float4> nodes(nn);
        for (int64_t i = 0; i < nn; ++i) nodes[i] = make_float4(f->B[3 * i], f->B[3 * i + 1], f->B[3 * i + 2], 0.0f);
        mt_status st = upload(own, nodes.data(), nodes.size(), "field nodes", &w.fmap);
        if (st != MT_OK) return st;
        for (int a = 0; a < 3; ++a) {   // in frame units, node i at u = i
            w.fdims[a] = f->dims[a];
            w.forigin[a] = -0.5f;
            w.forigin_lo[a] = 0.0f;
            w.fspacing[a] = 1.0f;
            w.fspacing_lo[a] = 0.0f;
            w.finv[a] = 1.0f;
        }
        set_sort_grid(w);
        return MT_OK;
    }
    if (f->kind != MT_FIELD_MAP) return MT_OK;
    const int nx = f->dims[0], ny = f->dims[1], nz = f->dims[2];
    const size_t nraw = 3ull * nx * ny * nz;
    const size_t npair = 2ull * (size_t)(nx - 1) * ny * nz;
    void *raw = nullptr, *pairs = nullptr;
    cudaError_t e = cudaMalloc(&raw, nraw * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(e, "field staging");
    e = cudaMemcpy(raw, f->B, nraw * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&pairs, npair * sizeof(float4));
    if (e == cudaSuccess) {
        own.bufs.push_back(pairs);
        own.bytes += (int64_t)(npair * sizeof(float4));
        e = launch_repack_field((const float *)raw, (float4 *)pairs, nx, ny, nz, 0);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(raw);
    if (e != cudaSuccess) return cuda_fail(e, "field map upload");
    w.fmap = (const float4 *)pairs;
    for (int a = 0; a < 3; ++a) {   // the frame is this map's node grid
        w.fdims[a] = f->dims[a];
        w.forigin[a] = 0.0f;
        w.forigin_lo[a] = 0.0f;
        w.fspacing[a] = 1.0f;
        w.fspacing_lo[a] = 0.0f;
        w.finv[a] = (float)(1.0 / f->spacing[a]);
    }
    set_sort_grid(w);
    return MT_OK;
}

}  // namespace mt

using namespace mt;

extern "C" {

int32_t mt_abi_version(void) { return MT_ABI_VERSION; }

const char *mt_last_error(void) { return g_err; }

void mt_destroy(mt_handle *h)
{
    if (!h) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    h->own.release();
    if (prev >= 0) cudaSetDevice(prev);
    delete h;
}

int64_t mt_device_bytes(const mt_handle *h) { return h ? h->own.bytes : 0; }

mt_status mt_create(const mt_geometry_desc *g, const mt_field_desc *f, const mt_hist_desc *hd, mt_handle **out)
{
    g_err[0] = 0;
    if (!out) {
        set_error("null output pointer");
        return MT_ERR_INVALID_ARG;
    }
    *out = nullptr;
    mt_status st = validate_hist(hd);
    if (st == MT_OK) st = validate_geometry(g, hd->n_mat);
    if (st == MT_OK) st = validate_field(f, g);
    if (st != MT_OK) return st;
    // table construction first: it checks the weights before any device work
    mt_handle *h = new mt_handle();
    memset(&h->w, 0, sizeof(h->w));
    cudaGetDevice(&h->device);
    st = build_hist(hd, h->w, h->own);
    if (st == MT_OK) st = build_geometry(g, f, h->w, h->own);
    if (st == MT_OK) st = build_field(f, h->w, h->own);
    if (st != MT_OK) {
        mt_destroy(h);
        return st;
    }
    noalloc_prepare(h->w, h->device);
    *out = h;
    return MT_OK;
}

}  // extern "C"
