/*
 * oracle.c -- double-precision CPU oracle for histogram-sampling muon transport
 * (Cattelan, Qasim, Owen, Serra, "Ultra-Fast Muon Transport via Histogram
 * Sampling on GPUs", arXiv 2512.10520).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or constant generator with the CUDA path: it derives its own sampling
 * thresholds from the raw histogram weights and runs Algorithm 1 step by step
 * in FP64, one muon at a time, with no blocking, fusion or reordering.
 *
 * What it computes, per muon (Algorithm 1, Sec. "Simulation"):
 *   for k = steps_done .. max_steps-1:
 *     P = |p|; break with a status if P < p_min, z >= z_max, |x| >= x_max
 *       or |y| >= y_max                                   (termination test)
 *     M = GetMaterial(r): first containing box or solid,  (Sec. Simulation, item 1;
 *         or a voxel                                       solids by Eq. 2)
 *     if M is not vacuum:
 *       i = GetMomentumBin(P), log10 bins                 (Sec. Momentum binning)
 *       (w0..w3) = Philox4x32-10(key = seed, ctr = (k, id_lo, id_hi, instance))
 *       cell = #{ j < ncell-1 : T_j <= w0 }               (inverse CDF of H_{M,i})
 *         or the alias column of w0 (Sec. Methodology, "The Alias Method")
 *       f, theta = cell centre axes + uniform jitter      (Sec. Simulation, item 2)
 *       phi = 2 pi U                                      (isotropic azimuth)
 *       p <- p + Rot(dp), dp = [dt cos phi, dt sin phi, dz]   (Eq. 3, Rodrigues)
 *     B = GetField(r)                                     (Sec. Simulation, item 3)
 *     (r, p) <- RK4Step(r, p, B, d), dP/dt = q v x B      (Eq. 4)
 *     steps_done = k + 1
 *
 * Readings where the paper is silent or garbled:
 *  - sampler: inverse CDF over uint32 thresholds T_j = floor(2^32 S_j / S_tot)
 *    with S_j the left-to-right FP64 prefix sum of the cell weights (the paper
 *    uses Walker's alias method; inverse CDF gives a different but equally
 *    valid draw -> cell map and makes the cell choice exact in integers);
 *  - histogram axes are linear: f = dp/p in [0, f_max), theta in [0, theta_max);
 *    jitter is uniform inside the chosen cell on both axes (draws w1, w2);
 *  - dz, dt of Algorithm 1 are dz = P((1-f) cos theta - 1), dt = P(1-f) sin theta,
 *    so the update keeps |p_new| = (1-f) P and angle(p, p_new) = theta exactly;
 *  - Eq. 3 is read as p <- p + Rot(dp) with Rot(v) = v cos a + (k x v) sin a +
 *    k (k.v)(1 - cos a), k = z x p^ / |z x p^|, cos a = p^_z, sin a = |z x p^|;
 *    if |z x p^| < 1e-12, Rot = I for p^_z > 0 and diag(1,-1,-1) otherwise;
 *  - the field is looked up once per step at the step's start position and held
 *    fixed over the RK4 stages; trilinear on nodes, zero outside the node box;
 *  - RK4 integrates dr/ds = p/P0, dp/ds = kappa q (p x B)/P0 over s in [0, d],
 *    P0 = |p| after the scattering update, kappa = 0.299792458 GeV/(T m);
 *  - termination uses |x| and |y|, is tested at the start of a step, and a loss
 *    below the cut mid-step stops the muon at the next test;
 *  - momentum bins outside [p_lo, p_hi) are clamped to the edge bins;
 *  - U(w) = (w >> 8) 2^-24 (exact in FP32 and FP64).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_KAPPA 0.299792458           /* GeV / (T m) per unit charge */
#define OR_TWO_PI 6.283185307179586476925286766559

enum { OR_ALIVE = 0, OR_STOPPED = 1, OR_EXIT_Z = 2, OR_EXIT_XY = 3, OR_MAX_STEPS = 4, OR_INVALID = 5 };

typedef struct or_world {
    /* geometry */
    int32_t geom_kind;          /* 0: ordered axis-aligned boxes, 1: voxel grid, 2: ordered solids */
    int32_t n_box;              /* boxes, or solids (geom_kind 2) */
    const double *box_lo;       /* [n_box][3], half-open boxes lo <= r < hi */
    const double *box_hi;       /* [n_box][3] */
    const int32_t *box_mat;     /* [n_box] material id (0 = vacuum) */
    const int32_t *box_block;   /* [n_box] field-scale block id or -1 */
    const double *box_B;        /* [n_box][3] uniform field inside the box / solid (field_kind 1) */
    const double *poly_z;       /* solids: [n_box][2] z0 < z1 */
    const double *poly_xy;      /* solids: [n_box][2][4][2] bottom (z0) then top (z1) quadrilateral */
    int32_t world_mat;
    int32_t vox_dims[3];        /* nx, ny, nz */
    double vox_origin[3];
    double vox_spacing[3];
    const uint8_t *vox;         /* [nz][ny][nx] material ids */
    double x_max, y_max, z_max, p_min;
    /* field */
    int32_t field_kind;         /* 0: none, 1: per-box uniform, 2: trilinear node map, 3: nearest node */
    int32_t fdims[3];
    double forigin[3];
    double fspacing[3];
    const float *Bmap;          /* [nz][ny][nx][3] */
    int32_t field_per_stage;    /* 1: RK4 reads the map at each stage's position (map kinds only) */
    const double *alpha;        /* [n_block][3] field scales, or NULL */
    int32_t n_block;
    /* histograms */
    int32_t n_mat, n_pbin, nf, ntheta;
    double p_lo, p_hi;
    const double *p_edges;      /* [n_pbin + 1] momentum-bin edges, or NULL for log10 bins */
    const double *f_max;        /* [n_mat][n_pbin] */
    const double *theta_max;    /* [n_mat][n_pbin] */
    const uint64_t *T;          /* [n_mat][n_pbin][nf*ntheta-1] from or_build_thresholds */
    int32_t axes;               /* 0: linear (f = dp/p, theta); 1: log (f = -dPz/P, t = dPt/P) */
    const double *f_min;        /* log axes: [n_mat][n_pbin] lower edge of the f axis */
    const double *theta_min;    /* log axes: [n_mat][n_pbin] lower edge of the t axis */
    int32_t sampler;            /* 0: inverse CDF over T, 1: alias tables below */
    const uint32_t *alias_prob; /* [n_mat][n_pbin][nf*ntheta] from or_build_alias */
    const int32_t *alias_idx;   /* [n_mat][n_pbin][nf*ntheta] */
} or_world;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11.  Ten rounds of a multiply/xor S-box with a Weyl  */
/* key schedule.                                                             */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t m0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t m1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(m0 >> 32), lo0 = (uint32_t)m0;
        uint32_t hi1 = (uint32_t)(m1 >> 32), lo1 = (uint32_t)m1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        x0 = y0;
        x1 = lo1;
        x2 = y2;
        x3 = lo0;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

double or_uniform(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------------ */
/* Histogram -> normalised discrete CDF -> uint32 thresholds (Sec. Building  */
/* histograms: each histogram, once normalised, is a joint discrete PDF).    */
/* T_j = floor(2^32 * S_j / S_tot), j = 0..ncell-2; stored in 64 bits, since */
/* a trailing run of empty cells gives T_j = 2^32 (never <= any 32-bit draw). */
/* Returns 0, or -1 (negative / non-finite weight), -2 (empty histogram).    */
/* ------------------------------------------------------------------------ */
int or_build_thresholds(int64_t n_hist, int32_t ncell, const double *w, uint64_t *T)
{
    for (int64_t h = 0; h < n_hist; ++h) {
        const double *wh = w + h * (int64_t)ncell;
        double total = 0.0;
        for (int32_t j = 0; j < ncell; ++j) {
            if (!(wh[j] >= 0.0) || !isfinite(wh[j])) return -1;
            total += wh[j];
        }
        if (!(total > 0.0) || !isfinite(total)) return -2;
        double S = 0.0;
        for (int32_t j = 0; j < ncell - 1; ++j) {
            S += wh[j];
            double C = S / total;
            T[h * (int64_t)(ncell - 1) + j] = (uint64_t)floor(C * 4294967296.0);
        }
    }
    return 0;
}

/* Inverse CDF: the cell whose interval [T_{c-1}, T_c) holds the draw. */
int32_t or_sample_cell(const uint64_t *T, int32_t ncell, uint32_t w0)
{
    int32_t c = 0;
    for (int32_t j = 0; j < ncell - 1; ++j)
        if (T[j] <= (uint64_t)w0) ++c;
    return c;
}

/* ------------------------------------------------------------------------ */
/* Walker's alias method (Sec. Methodology, "The Alias Method"): the N cells */
/* become N equiprobable columns, each holding at most two outcomes, the    */
/* column's own cell (taken with probability Prob_j) and an alias cell.     */
/* Built here in integers from the masses m_c = T_c - T_{c-1} of the        */
/* thresholds above (T_{-1} = 0, T_{N-1} = 2^32), which sum to 2^32, so the  */
/* alias map draws from exactly the quantised distribution that the inverse */
/* CDF draws from; only the draw -> cell map differs.  N must be a power of  */
/* two, N = 2^n; a column then holds C = 2^(32-n) units of mass.            */
/* Construction (Vose's variant of Walker's): every cell starts with        */
/* q_c = m_c; the cells with q_c < C go on a "small" stack and the others on */
/* a "large" stack, each pushed in increasing cell order.  While both are   */
/* non-empty: pop s (small) and l (large); column s keeps q_s of its own    */
/* cell and takes the remaining C - q_s from l (Alias_s = l); q_l drops by  */
/* C - q_s and l is pushed on the small stack if q_l < C, else back on the  */
/* large one.  Columns still on the large stack hold C of their own cell.   */
/* In integers no cell is left on the small stack (the masses sum to N C).  */
/* Prob_j = q_j 2^n is column j's own share in units of 2^-32 of the        */
/* column, stored as min(Prob_j, 2^32 - 1).  A draw w0 picks column         */
/* j = w0 >> (32 - n) at position r = (w0 << n) mod 2^32; the cell is j when */
/* r < Prob_j, else Alias_j.  Returns 0, or -3 if N is not a power of two.  */
/* ------------------------------------------------------------------------ */
int or_build_alias(int64_t n_hist, int32_t ncell, const uint64_t *T, uint32_t *prob, int32_t *alias)
{
    if (ncell < 2 || (ncell & (ncell - 1)) != 0) return -3;
    int32_t n = 0;
    while ((1 << n) < ncell) ++n;
    const uint64_t C = 1ull << (32 - n);
    uint64_t *q = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)ncell);
    int32_t *small = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncell);
    int32_t *large = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncell);
    if (!q || !small || !large) {
        free(q);
        free(small);
        free(large);
        return -4;
    }
    for (int64_t h = 0; h < n_hist; ++h) {
        const uint64_t *Th = T + h * (int64_t)(ncell - 1);
        uint32_t *P = prob + h * (int64_t)ncell;
        int32_t *A = alias + h * (int64_t)ncell;
        int32_t ns = 0, nl = 0;
        uint64_t prev = 0;
        for (int32_t c = 0; c < ncell; ++c) {
            uint64_t t = c < ncell - 1 ? Th[c] : (1ull << 32);
            if (t < prev) t = prev;       /* thresholds never decrease; guard anyway */
            q[c] = t - prev;
            prev = t;
            if (q[c] < C)
                small[ns++] = c;
            else
                large[nl++] = c;
        }
        while (ns > 0 && nl > 0) {
            const int32_t sc = small[--ns];
            const int32_t lc = large[--nl];
            P[sc] = (uint32_t)(q[sc] << n);
            A[sc] = lc;
            q[lc] -= C - q[sc];
            if (q[lc] < C)
                small[ns++] = lc;
            else
                large[nl++] = lc;
        }
        while (nl > 0) {
            const int32_t lc = large[--nl];
            P[lc] = 0xFFFFFFFFu;
            A[lc] = lc;
        }
        while (ns > 0) {                  /* unreachable with exact integer masses */
            const int32_t sc = small[--ns];
            P[sc] = 0xFFFFFFFFu;
            A[sc] = sc;
        }
    }
    free(q);
    free(small);
    free(large);
    return 0;
}

/* Alias draw: column j = w0 >> (32 - n), position r = (w0 << n) mod 2^32. */
int32_t or_sample_alias(const uint32_t *prob, const int32_t *alias, int32_t ncell, uint32_t w0)
{
    int32_t n = 0;
    while ((1 << n) < ncell) ++n;
    const uint32_t j = w0 >> (32 - n);
    const uint32_t r = w0 << n;
    return r < prob[j] ? (int32_t)j : alias[j];
}

/* GetMomentumBin: base-10 logarithmic bins on [p_lo, p_hi], clamped. */
int32_t or_momentum_bin(double P, double p_lo, double p_hi, int32_t n_pbin)
{
    double u = (log10(P) - log10(p_lo)) * (double)n_pbin / log10(p_hi / p_lo);
    double i = floor(u);
    if (!(i >= 0.0)) return 0;          /* also catches NaN */
    if (i > (double)(n_pbin - 1)) return n_pbin - 1;
    return (int32_t)i;
}

/* GetMomentumBin over explicit edges (the bounded-variation bins of Appendix
 * A): the i with edges[i] <= P < edges[i+1], found by binary search, clamped
 * to the edge bins. */
int32_t or_momentum_bin_edges(double P, const double *edges, int32_t n_pbin)
{
    if (!(P >= edges[1])) return 0;    /* also catches NaN */
    if (P >= edges[n_pbin - 1]) return n_pbin - 1;
    int32_t lo = 1, hi = n_pbin - 1;   /* edges[lo] <= P < edges[hi] */
    while (hi - lo > 1) {
        int32_t mid = (lo + hi) / 2;
        if (edges[mid] <= P)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

/* GetMaterial: first box (list order) with lo <= r < hi, else the world;
 * or the voxel holding r, else the world.  *box receives the box index or -1. */
/* Containment in solid b (Sec. Simulation item 1, Eq. 2): the solid spans
 * z0 <= z < z1; its cross-section at height z is the quadrilateral with
 * vertices v_i = bottom_i + t (top_i - bottom_i), t = (z - z0) / (z1 - z0);
 * with e_i = v_{i+1} - v_i (indices mod 4), the point is inside when every
 * S_i = e_ix (y - v_iy) - e_iy (x - v_ix) has the same sign.  The vertices are
 * counter-clockwise seen from +z, so that sign is non-negative: a point on an
 * edge is inside. */
int or_in_solid(const or_world *w, int32_t b, const double r[3])
{
    const double z0 = w->poly_z[2 * b], z1 = w->poly_z[2 * b + 1];
    if (!(r[2] >= z0 && r[2] < z1)) return 0;
    const double t = (r[2] - z0) / (z1 - z0);
    const double *bot = w->poly_xy + 16 * (int64_t)b, *top = bot + 8;
    double vx[4], vy[4];
    for (int i = 0; i < 4; ++i) {
        vx[i] = bot[2 * i] + t * (top[2 * i] - bot[2 * i]);
        vy[i] = bot[2 * i + 1] + t * (top[2 * i + 1] - bot[2 * i + 1]);
    }
    for (int i = 0; i < 4; ++i) {
        const int j = (i + 1) % 4;
        const double ex = vx[j] - vx[i], ey = vy[j] - vy[i];
        const double S = ex * (r[1] - vy[i]) - ey * (r[0] - vx[i]);
        if (S < 0.0) return 0;
    }
    return 1;
}

int32_t or_material(const or_world *w, const double r[3], int32_t *box)
{
    *box = -1;
    if (w->geom_kind == 2) {
        for (int32_t b = 0; b < w->n_box; ++b)
            if (or_in_solid(w, b, r)) {
                *box = b;
                return w->box_mat[b];
            }
        return w->world_mat;
    }
    if (w->geom_kind == 0) {
        for (int32_t b = 0; b < w->n_box; ++b) {
            const double *lo = w->box_lo + 3 * b, *hi = w->box_hi + 3 * b;
            int inside = 1;
            for (int a = 0; a < 3; ++a)
                if (!(r[a] >= lo[a] && r[a] < hi[a])) inside = 0;
            if (inside) {
                *box = b;
                return w->box_mat[b];
            }
        }
        return w->world_mat;
    }
    int64_t idx[3];
    for (int a = 0; a < 3; ++a) {
        double u = floor((r[a] - w->vox_origin[a]) / w->vox_spacing[a]);
        if (!(u >= 0.0 && u < (double)w->vox_dims[a])) return w->world_mat;
        idx[a] = (int64_t)u;
    }
    return w->vox[(idx[2] * w->vox_dims[1] + idx[1]) * w->vox_dims[0] + idx[0]];
}

/* Trilinear interpolation of the node map; zero outside [origin, origin+(dims-1)*spacing]. */
static void or_field_map(const or_world *w, const double r[3], double B[3])
{
    int64_t i0[3];
    double t[3];
    B[0] = B[1] = B[2] = 0.0;
    for (int a = 0; a < 3; ++a) {
        double u = (r[a] - w->forigin[a]) / w->fspacing[a];
        if (!(u >= 0.0 && u <= (double)(w->fdims[a] - 1))) return;
        double fl = floor(u);
        if (fl > (double)(w->fdims[a] - 2)) fl = (double)(w->fdims[a] - 2);
        i0[a] = (int64_t)fl;
        t[a] = u - fl;
    }
    const int64_t nx = w->fdims[0], ny = w->fdims[1];
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                double wgt = (di ? t[0] : 1.0 - t[0]) * (dj ? t[1] : 1.0 - t[1]) *
                             (dk ? t[2] : 1.0 - t[2]);
                const float *node = w->Bmap + 3 * (((i0[2] + dk) * ny + (i0[1] + dj)) * nx + (i0[0] + di));
                for (int c = 0; c < 3; ++c) B[c] += wgt * (double)node[c];
            }
}

/* Nearest-node lookup of the map (the paper's grid retrieval, Sec. Simulation
 * item 3): node i of an axis owns [origin + (i - 1/2) s, origin + (i + 1/2) s),
 * i = floor((r - origin)/s + 1/2); zero when that node is outside the map. */
static void or_field_nearest(const or_world *w, const double r[3], double B[3])
{
    int64_t i[3];
    B[0] = B[1] = B[2] = 0.0;
    for (int a = 0; a < 3; ++a) {
        double u = floor((r[a] - w->forigin[a]) / w->fspacing[a] + 0.5);
        if (!(u >= 0.0 && u <= (double)(w->fdims[a] - 1))) return;
        i[a] = (int64_t)u;
    }
    const float *node = w->Bmap + 3 * ((i[2] * w->fdims[1] + i[1]) * w->fdims[0] + i[0]);
    for (int c = 0; c < 3; ++c) B[c] = (double)node[c];
}

/* GetField: none / per-box uniform / trilinear map / nearest node, then the per-block scale
 * alpha[block][c] when r lies in a box that carries a block id. */
void or_field(const or_world *w, const double r[3], int32_t box, double B[3])
{
    B[0] = B[1] = B[2] = 0.0;
    if (w->field_kind == 1) {
        if (box >= 0)
            for (int c = 0; c < 3; ++c) B[c] = w->box_B[3 * box + c];
    } else if (w->field_kind == 2) {
        or_field_map(w, r, B);
    } else if (w->field_kind == 3) {
        or_field_nearest(w, r, B);
    }
    if (w->alpha && box >= 0 && w->box_block) {
        int32_t blk = w->box_block[box];
        if (blk >= 0 && blk < w->n_block)
            for (int c = 0; c < 3; ++c) B[c] *= w->alpha[3 * blk + c];
    }
}

/* Eq. 3 (Rodrigues): p <- p + Rot(dp), dp = [dt cos phi, dt sin phi, dz] in
 * the frame whose z axis is the direction of travel, rotated into the global
 * frame; here dz = P cz and dt = P ct. */
void or_scatter_c(const double p[3], double cz, double ct, double phi, double out[3])
{
    double P = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    double ph[3] = {p[0] / P, p[1] / P, p[2] / P};
    double dt = P * ct;
    double dz = P * cz;
    double dp[3] = {dt * cos(phi), dt * sin(phi), dz};
    double rot[3];
    double s = sqrt(ph[0] * ph[0] + ph[1] * ph[1]);
    if (s < 1e-12) {
        if (ph[2] > 0.0) {
            rot[0] = dp[0]; rot[1] = dp[1]; rot[2] = dp[2];
        } else {
            rot[0] = dp[0]; rot[1] = -dp[1]; rot[2] = -dp[2];
        }
    } else {
        double k[3] = {-ph[1] / s, ph[0] / s, 0.0};
        double ca = ph[2], sa = s;
        double kxv[3] = {k[1] * dp[2] - k[2] * dp[1], k[2] * dp[0] - k[0] * dp[2], k[0] * dp[1] - k[1] * dp[0]};
        double kv = k[0] * dp[0] + k[1] * dp[1] + k[2] * dp[2];
        for (int c = 0; c < 3; ++c) rot[c] = dp[c] * ca + kxv[c] * sa + k[c] * kv * (1.0 - ca);
    }
    for (int c = 0; c < 3; ++c) out[c] = p[c] + rot[c];
}

/* dz / P and dt / P of Algorithm 1 from a draw: linear axes (f = dp/p, theta):
 * cz = (1-f) cos theta - 1, ct = (1-f) sin theta, so |p_new| = (1-f) P and
 * angle(p, p_new) = theta; log axes (f = -dPz/P, t = dPt/P, the histogram
 * variables of Sec. Building histograms): cz = -f, ct = t. */
void or_dp_coeffs(int32_t axes, double f, double theta_or_t, double *cz, double *ct)
{
    if (axes == 1) {
        *cz = -f;
        *ct = theta_or_t;
    } else {
        *cz = (1.0 - f) * cos(theta_or_t) - 1.0;
        *ct = (1.0 - f) * sin(theta_or_t);
    }
}

/* Linear-axes scattering from (f, theta). */
void or_scatter(const double p[3], double f, double theta, double phi, double out[3])
{
    double cz, ct;
    or_dp_coeffs(0, f, theta, &cz, &ct);
    or_scatter_c(p, cz, ct, phi, out);
}

/* Eq. 4 with E = 0, integrated by classical RK4 over the path length d with B
 * held fixed: dr/ds = p/P0, dp/ds = kappa q (p x B)/P0. */
static void or_deriv(const double p[3], const double B[3], double qk, double P0, double dr[3], double dp[3])
{
    for (int c = 0; c < 3; ++c) dr[c] = p[c] / P0;
    dp[0] = qk * (p[1] * B[2] - p[2] * B[1]) / P0;
    dp[1] = qk * (p[2] * B[0] - p[0] * B[2]) / P0;
    dp[2] = qk * (p[0] * B[1] - p[1] * B[0]) / P0;
}

void or_rk4(double r[3], double p[3], const double B[3], int32_t q, double d)
{
    double P0 = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    double qk = OR_KAPPA * (double)q;
    double k1r[3], k1p[3], k2r[3], k2p[3], k3r[3], k3p[3], k4r[3], k4p[3], tmp[3];
    or_deriv(p, B, qk, P0, k1r, k1p);
    for (int c = 0; c < 3; ++c) tmp[c] = p[c] + 0.5 * d * k1p[c];
    or_deriv(tmp, B, qk, P0, k2r, k2p);
    for (int c = 0; c < 3; ++c) tmp[c] = p[c] + 0.5 * d * k2p[c];
    or_deriv(tmp, B, qk, P0, k3r, k3p);
    for (int c = 0; c < 3; ++c) tmp[c] = p[c] + d * k3p[c];
    or_deriv(tmp, B, qk, P0, k4r, k4p);
    for (int c = 0; c < 3; ++c) {
        r[c] += d / 6.0 * (k1r[c] + 2.0 * k2r[c] + 2.0 * k3r[c] + k4r[c]);
        p[c] += d / 6.0 * (k1p[c] + 2.0 * k2p[c] + 2.0 * k3p[c] + k4p[c]);
    }
}

/* RK4 with the field read at each stage's position (a variant of the step:
 * Algorithm 1 reads the field once, at the start of the step): classical RK4
 * on y = (r, p) with F(r, p) = (p/P0, kappa q p x B(r)/P0), P0 = |p| at the
 * start of the step, B(r) the map at r times the scale of the block that
 * holds the step's start (box), the stages at r + d/2 k1r, r + d/2 k2r and
 * r + d k3r. */
void or_rk4_staged(const or_world *w, double r[3], double p[3], int32_t box, int32_t q, double d)
{
    double P0 = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    double qk = OR_KAPPA * (double)q;
    double k1r[3], k1p[3], k2r[3], k2p[3], k3r[3], k3p[3], k4r[3], k4p[3], tr[3], tp[3], B[3];
    or_field(w, r, box, B);
    or_deriv(p, B, qk, P0, k1r, k1p);
    for (int c = 0; c < 3; ++c) {
        tr[c] = r[c] + 0.5 * d * k1r[c];
        tp[c] = p[c] + 0.5 * d * k1p[c];
    }
    or_field(w, tr, box, B);
    or_deriv(tp, B, qk, P0, k2r, k2p);
    for (int c = 0; c < 3; ++c) {
        tr[c] = r[c] + 0.5 * d * k2r[c];
        tp[c] = p[c] + 0.5 * d * k2p[c];
    }
    or_field(w, tr, box, B);
    or_deriv(tp, B, qk, P0, k3r, k3p);
    for (int c = 0; c < 3; ++c) {
        tr[c] = r[c] + d * k3r[c];
        tp[c] = p[c] + d * k3p[c];
    }
    or_field(w, tr, box, B);
    or_deriv(tp, B, qk, P0, k4r, k4p);
    for (int c = 0; c < 3; ++c) {
        r[c] += d / 6.0 * (k1r[c] + 2.0 * k2r[c] + 2.0 * k3r[c] + k4r[c]);
        p[c] += d / 6.0 * (k1p[c] + 2.0 * k2p[c] + 2.0 * k3p[c] + k4p[c]);
    }
}

/* One step's random choices (recorded for the adjoint and for tests). */
typedef struct or_step_draw {
    int32_t mat, box, pbin, cell;
    double f, theta, phi;
} or_step_draw;

/* Material, bin and histogram draw for step k (Algorithm 1, inside "if M is
 * not vacuum").  Returns 1 if the muon is in matter and d holds the draw. */
static int or_draw_step(const or_world *w, const double r[3], const double p[3], int32_t k,
                        uint64_t id, int32_t inst, uint64_t seed, or_step_draw *d)
{
    d->mat = or_material(w, r, &d->box);
    d->pbin = -1;
    d->cell = -1;
    d->f = d->theta = d->phi = 0.0;
    if (d->mat == 0) return 0;
    double P = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    int32_t i = w->p_edges ? or_momentum_bin_edges(P, w->p_edges, w->n_pbin)
                           : or_momentum_bin(P, w->p_lo, w->p_hi, w->n_pbin);
    uint32_t ctr[4] = {(uint32_t)k, (uint32_t)id, (uint32_t)(id >> 32), (uint32_t)inst};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t u[4];
    or_philox4x32_10(ctr, key, u);
    const int32_t ncell = w->nf * w->ntheta;
    const int64_t hidx = (int64_t)(d->mat - 1) * w->n_pbin + i;
    int32_t c = w->sampler == 1 ? or_sample_alias(w->alias_prob + hidx * ncell, w->alias_idx + hidx * ncell, ncell, u[0])
                                : or_sample_cell(w->T + hidx * (ncell - 1), ncell, u[0]);
    int32_t a = c / w->ntheta, b = c % w->ntheta;
    d->pbin = i;
    d->cell = c;
    if (w->axes == 1) {
        /* log-spaced axes: jitter uniform in log f and log t inside the cell */
        const double lf0 = log(w->f_min[hidx]), lf1 = log(w->f_max[hidx]);
        const double lt0 = log(w->theta_min[hidx]), lt1 = log(w->theta_max[hidx]);
        d->f = exp(lf0 + ((double)a + or_uniform(u[1])) / (double)w->nf * (lf1 - lf0));
        d->theta = exp(lt0 + ((double)b + or_uniform(u[2])) / (double)w->ntheta * (lt1 - lt0));
    } else {
        d->f = ((double)a + or_uniform(u[1])) / (double)w->nf * w->f_max[hidx];
        d->theta = ((double)b + or_uniform(u[2])) / (double)w->ntheta * w->theta_max[hidx];
    }
    d->phi = OR_TWO_PI * or_uniform(u[3]);
    return 1;
}

/* The scattering update of a step's draw (Algorithm 1: dz, dt, then Eq. 3). */
static void or_scatter_draw(const or_world *w, const double p[3], const or_step_draw *d, double out[3])
{
    double cz, ct;
    or_dp_coeffs(w->axes, d->f, d->theta, &cz, &ct);
    or_scatter_c(p, cz, ct, d->phi, out);
}

/* Termination test at the start of a step; returns a status or OR_ALIVE. */
static int or_check(const or_world *w, const double r[3], const double p[3])
{
    double P = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    if (P < w->p_min) return OR_STOPPED;
    if (r[2] >= w->z_max) return OR_EXIT_Z;
    if (fabs(r[0]) >= w->x_max || fabs(r[1]) >= w->y_max) return OR_EXIT_XY;
    return OR_ALIVE;
}

/* Algorithm 1 for one muon.  Muons whose status is terminal (not ALIVE and
 * not MAX_STEPS) are left unchanged. */
void or_transport_one(const or_world *w, double r[3], double p[3], int32_t q, int32_t *steps,
                      uint8_t *status, uint64_t id, int32_t inst, double d, int32_t max_steps,
                      uint64_t seed)
{
    if (*status != OR_ALIVE && *status != OR_MAX_STEPS) return;
    for (int c = 0; c < 3; ++c)
        if (!isfinite(r[c]) || !isfinite(p[c])) {
            *status = OR_INVALID;
            return;
        }
    int st = OR_MAX_STEPS;
    for (int32_t k = *steps; k < max_steps; ++k) {
        int t = or_check(w, r, p);
        if (t != OR_ALIVE) {
            st = t;
            break;
        }
        or_step_draw dr;
        if (or_draw_step(w, r, p, k, id, inst, seed, &dr)) or_scatter_draw(w, p, &dr, p);
        if (w->field_per_stage) {
            or_rk4_staged(w, r, p, dr.box, q, d);   /* reads the field at each stage itself */
        } else {
            double B[3];
            or_field(w, r, dr.box, B);
            or_rk4(r, p, B, q, d);
        }
        *steps = k + 1;
    }
    *status = (uint8_t)st;
}

typedef struct or_job {
    const or_world *w;
    int64_t begin, end;
    double *x, *y, *z, *px, *py, *pz;
    const int8_t *q;
    int32_t *steps;
    uint8_t *status;
    int64_t id_offset;
    int32_t inst;
    double d;
    int32_t max_steps;
    uint64_t seed;
} or_job;

static void *or_worker(void *arg)
{
    or_job *j = (or_job *)arg;
    for (int64_t m = j->begin; m < j->end; ++m) {
        double r[3] = {j->x[m], j->y[m], j->z[m]};
        double p[3] = {j->px[m], j->py[m], j->pz[m]};
        or_transport_one(j->w, r, p, j->q[m], &j->steps[m], &j->status[m], (uint64_t)(j->id_offset + m),
                         j->inst, j->d, j->max_steps, j->seed);
        j->x[m] = r[0]; j->y[m] = r[1]; j->z[m] = r[2];
        j->px[m] = p[0]; j->py[m] = p[1]; j->pz[m] = p[2];
    }
    return NULL;
}

/* Transport n muons (FP64 SoA, in place) on n_threads POSIX threads.
 * Muon m has id id_offset + m.  Returns 0 or -1 on bad arguments. */
int or_transport(const or_world *w, int64_t n, double *x, double *y, double *z, double *px, double *py,
                 double *pz, const int8_t *q, int32_t *steps, uint8_t *status, int64_t id_offset,
                 int32_t inst, double d, int32_t max_steps, uint64_t seed, int32_t n_threads)
{
    if (!w || n < 0 || n_threads < 1) return -1;
    if (n == 0) return 0;
    if (n_threads > 256) n_threads = 256;
    if ((int64_t)n_threads > n) n_threads = (int32_t)n;
    pthread_t th[256];
    or_job jobs[256];
    for (int32_t t = 0; t < n_threads; ++t) {
        or_job j = {w, n * t / n_threads, n * (t + 1) / n_threads, x, y, z, px, py, pz, q, steps, status,
                    id_offset, inst, d, max_steps, seed};
        jobs[t] = j;
    }
    for (int32_t t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, or_worker, &jobs[t]);
    or_worker(&jobs[0]);
    for (int32_t t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
    return 0;
}

/* Record the draws of one muon's trajectory (tests of the sampler and rotation):
 * for each executed step s, mat/box/pbin/cell and f/theta/phi.  Returns the
 * number of steps executed. */
int32_t or_trace(const or_world *w, double r[3], double p[3], int32_t q, int32_t steps0, uint64_t id,
                 int32_t inst, double d, int32_t max_steps, uint64_t seed, int32_t *ibuf /* [max][4] */,
                 double *dbuf /* [max][9]: r before, p after scatter */, double *fbuf /* [max][3] */)
{
    int32_t s = 0;
    for (int32_t k = steps0; k < max_steps; ++k) {
        if (or_check(w, r, p) != OR_ALIVE) break;
        or_step_draw dr;
        for (int c = 0; c < 3; ++c) dbuf[9 * s + c] = r[c];
        if (or_draw_step(w, r, p, k, id, inst, seed, &dr)) or_scatter_draw(w, p, &dr, p);
        for (int c = 0; c < 3; ++c) dbuf[9 * s + 3 + c] = p[c];
        double B[3];
        or_field(w, r, dr.box, B);
        for (int c = 0; c < 3; ++c) dbuf[9 * s + 6 + c] = B[c];
        ibuf[4 * s + 0] = dr.mat; ibuf[4 * s + 1] = dr.box; ibuf[4 * s + 2] = dr.pbin; ibuf[4 * s + 3] = dr.cell;
        fbuf[3 * s + 0] = dr.f; fbuf[3 * s + 1] = dr.theta; fbuf[3 * s + 2] = dr.phi;
        if (w->field_per_stage)
            or_rk4_staged(w, r, p, dr.box, q, d);
        else
            or_rk4(r, p, B, q, d);
        ++s;
    }
    return s;
}

/* The draw of one step at a given state (sampler tests): ibuf = {mat, box,
 * pbin, cell}, dbuf = {f, theta, phi}.  Returns 1 in matter, 0 in vacuum. */
int32_t or_draw(const or_world *w, const double r[3], const double p[3], int32_t k, uint64_t id,
                int32_t inst, uint64_t seed, int32_t *ibuf, double *dbuf)
{
    or_step_draw dr;
    int in_matter = or_draw_step(w, r, p, k, id, inst, seed, &dr);
    ibuf[0] = dr.mat; ibuf[1] = dr.box; ibuf[2] = dr.pbin; ibuf[3] = dr.cell;
    dbuf[0] = dr.f; dbuf[1] = dr.theta; dbuf[2] = dr.phi;
    return in_matter;
}

/* ======================================================================== */
/* Differentiable form (the paper's Discussion suggests gradients of the     */
/* transport with respect to geometry and field parameters).  Parameters are */
/* per-block field scales alpha[block][c]; the draws of every step (material,*/
/* box, momentum bin, cell, f, theta, phi) and the number of steps are held  */
/* fixed (common random numbers), which gives the pathwise derivative.       */
/* ======================================================================== */

static double or_sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* Acceptance loss: mean over all n muons of s((h - |x_e|)/w) s((h - |y_e|)/w),
 * s the logistic function, (x_e, y_e) the straight-line extrapolation of the
 * final state to the plane z = zL.  Muons that stopped or are invalid, or have
 * pz <= 0, contribute 0 with zero gradient.  g (may be NULL) receives
 * dL/d(x, y, z, px, py, pz) as six arrays of n. */
double or_acceptance_loss(int64_t n, const double *x, const double *y, const double *z, const double *px,
                          const double *py, const double *pz, const uint8_t *status, double zL, double h,
                          double w, double *g)
{
    double L = 0.0;
    for (int64_t m = 0; m < n; ++m) {
        if (g)
            for (int c = 0; c < 6; ++c) g[c * n + m] = 0.0;
        if (status[m] == OR_STOPPED || status[m] == OR_INVALID || !(pz[m] > 0.0)) continue;
        double lz = zL - z[m];
        double xe = x[m] + lz * px[m] / pz[m];
        double ye = y[m] + lz * py[m] / pz[m];
        double a = (h - fabs(xe)) / w, b = (h - fabs(ye)) / w;
        double sa = or_sigmoid(a), sb = or_sigmoid(b);
        L += sa * sb;
        if (g) {
            double dxe = sa * (1.0 - sa) * sb * (xe >= 0.0 ? -1.0 : 1.0) / w / (double)n;
            double dye = sb * (1.0 - sb) * sa * (ye >= 0.0 ? -1.0 : 1.0) / w / (double)n;
            g[0 * n + m] = dxe;
            g[1 * n + m] = dye;
            g[2 * n + m] = -(dxe * px[m] + dye * py[m]) / pz[m];
            g[3 * n + m] = dxe * lz / pz[m];
            g[4 * n + m] = dye * lz / pz[m];
            g[5 * n + m] = -(dxe * px[m] + dye * py[m]) * lz / (pz[m] * pz[m]);
        }
    }
    return n > 0 ? L / (double)n : 0.0;
}

typedef struct or_tape {
    double r[3], p[3];
    int32_t scattered, box;
    double f, theta, phi;
} or_tape;

/* Unscaled field at r (map / per-box / none) and, for maps, its Jacobian
 * dBm_c/dr_a in J[c][a] (zero outside the node box). */
static void or_field_unscaled(const or_world *w, const double r[3], int32_t box, double Bm[3], double J[3][3])
{
    for (int c = 0; c < 3; ++c) {
        Bm[c] = 0.0;
        for (int a = 0; a < 3; ++a) J[c][a] = 0.0;
    }
    if (w->field_kind == 1) {
        if (box >= 0)
            for (int c = 0; c < 3; ++c) Bm[c] = w->box_B[3 * box + c];
        return;
    }
    if (w->field_kind == 3) {          /* piecewise constant: J = 0 */
        or_field_nearest(w, r, Bm);
        return;
    }
    if (w->field_kind != 2) return;
    int64_t i0[3];
    double t[3];
    for (int a = 0; a < 3; ++a) {
        double u = (r[a] - w->forigin[a]) / w->fspacing[a];
        if (!(u >= 0.0 && u <= (double)(w->fdims[a] - 1))) return;
        double fl = floor(u);
        if (fl > (double)(w->fdims[a] - 2)) fl = (double)(w->fdims[a] - 2);
        i0[a] = (int64_t)fl;
        t[a] = u - fl;
    }
    const int64_t nx = w->fdims[0], ny = w->fdims[1];
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                double fx = di ? t[0] : 1.0 - t[0], fy = dj ? t[1] : 1.0 - t[1], fz = dk ? t[2] : 1.0 - t[2];
                double gx = (di ? 1.0 : -1.0) * fy * fz / w->fspacing[0];
                double gy = (dj ? 1.0 : -1.0) * fx * fz / w->fspacing[1];
                double gz = (dk ? 1.0 : -1.0) * fx * fy / w->fspacing[2];
                const float *node = w->Bmap + 3 * (((i0[2] + dk) * ny + (i0[1] + dj)) * nx + (i0[0] + di));
                for (int c = 0; c < 3; ++c) {
                    Bm[c] += fx * fy * fz * (double)node[c];
                    J[c][0] += gx * (double)node[c];
                    J[c][1] += gy * (double)node[c];
                    J[c][2] += gz * (double)node[c];
                }
            }
}

static int32_t or_block_of(const or_world *w, int32_t box)
{
    if (!w->alpha || box < 0 || !w->box_block) return -1;
    int32_t blk = w->box_block[box];
    return (blk >= 0 && blk < w->n_block) ? blk : -1;
}

/* Reverse of or_scatter_c with (cz, ct, phi) fixed: pbar += (d out/d p)^T obar. */
static void or_scatter_vjp(const double p[3], double cz, double ct, double phi, const double obar[3], double pbar[3])
{
    double P = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    double ph[3] = {p[0] / P, p[1] / P, p[2] / P};
    double cp = cos(phi), sp = sin(phi);
    double dt = P * ct, dz = P * cz;
    double dp[3] = {dt * cp, dt * sp, dz};
    double s = sqrt(ph[0] * ph[0] + ph[1] * ph[1]);
    double dpbar[3] = {0, 0, 0}, phbar[3] = {0, 0, 0}, Pbar = 0.0;
    for (int c = 0; c < 3; ++c) pbar[c] += obar[c];            /* out = p + rot */
    if (s < 1e-12) {
        double sg = ph[2] > 0.0 ? 1.0 : -1.0;
        dpbar[0] = obar[0];
        dpbar[1] = sg * obar[1];
        dpbar[2] = sg * obar[2];
    } else {
        double k[3] = {-ph[1] / s, ph[0] / s, 0.0};
        double ca = ph[2], sa = s;
        double kxv[3] = {k[1] * dp[2] - k[2] * dp[1], k[2] * dp[0] - k[0] * dp[2], k[0] * dp[1] - k[1] * dp[0]};
        double kv = k[0] * dp[0] + k[1] * dp[1] + k[2] * dp[2];
        double kbar[3] = {0, 0, 0}, kxvbar[3], cabar = 0.0, sabar = 0.0, kvbar = 0.0, sbar = 0.0;
        double rk = obar[0] * k[0] + obar[1] * k[1] + obar[2] * k[2];
        for (int c = 0; c < 3; ++c) {
            dpbar[c] += obar[c] * ca;
            cabar += obar[c] * dp[c];
            kxvbar[c] = obar[c] * sa;
            sabar += obar[c] * kxv[c];
            kbar[c] += obar[c] * kv * (1.0 - ca);
        }
        kvbar = rk * (1.0 - ca);
        cabar -= rk * kv;
        for (int c = 0; c < 3; ++c) {                          /* kv = k . dp */
            kbar[c] += kvbar * dp[c];
            dpbar[c] += kvbar * k[c];
        }
        /* kxv = k x dp: kbar += dp x kxvbar, dpbar += kxvbar x k */
        kbar[0] += dp[1] * kxvbar[2] - dp[2] * kxvbar[1];
        kbar[1] += dp[2] * kxvbar[0] - dp[0] * kxvbar[2];
        kbar[2] += dp[0] * kxvbar[1] - dp[1] * kxvbar[0];
        dpbar[0] += kxvbar[1] * k[2] - kxvbar[2] * k[1];
        dpbar[1] += kxvbar[2] * k[0] - kxvbar[0] * k[2];
        dpbar[2] += kxvbar[0] * k[1] - kxvbar[1] * k[0];
        sbar += sabar;
        phbar[2] += cabar;
        /* k = (-ph1/s, ph0/s, 0) */
        phbar[1] += -kbar[0] / s;
        phbar[0] += kbar[1] / s;
        sbar += -(kbar[0] * k[0] + kbar[1] * k[1]) / s;
        phbar[0] += sbar * ph[0] / s;                          /* s = |ph_xy| */
        phbar[1] += sbar * ph[1] / s;
    }
    double dtbar = dpbar[0] * cp + dpbar[1] * sp, dzbar = dpbar[2];
    Pbar += dtbar * ct + dzbar * cz;
    double php = phbar[0] * p[0] + phbar[1] * p[1] + phbar[2] * p[2];
    for (int c = 0; c < 3; ++c) pbar[c] += phbar[c] / P;       /* ph = p / P */
    Pbar -= php / (P * P);
    for (int c = 0; c < 3; ++c) pbar[c] += Pbar * p[c] / P;    /* P = |p| */
}

/* Reverse of F(x) = (x/P0, qk (x x B)/P0) given its cotangent (ar, ap). */
static void or_deriv_vjp(const double x[3], const double B[3], double qk, double P0, const double ar[3],
                         const double ap[3], double xbar[3], double Bbar[3], double *P0bar)
{
    double xB[3] = {x[1] * B[2] - x[2] * B[1], x[2] * B[0] - x[0] * B[2], x[0] * B[1] - x[1] * B[0]};
    double Bxa[3] = {B[1] * ap[2] - B[2] * ap[1], B[2] * ap[0] - B[0] * ap[2], B[0] * ap[1] - B[1] * ap[0]};
    double axx[3] = {ap[1] * x[2] - ap[2] * x[1], ap[2] * x[0] - ap[0] * x[2], ap[0] * x[1] - ap[1] * x[0]};
    double dotr = 0.0, dotp = 0.0;
    for (int c = 0; c < 3; ++c) {
        xbar[c] += ar[c] / P0 + qk * Bxa[c] / P0;
        Bbar[c] += qk * axx[c] / P0;
        dotr += ar[c] * x[c];
        dotp += ap[c] * xB[c];
    }
    *P0bar -= (dotr + qk * dotp) / (P0 * P0);
}

/* Reverse of or_rk4: given (rbar, pbar) of the outputs, overwrite them with the
 * cotangents of the inputs (r, p) and accumulate Bbar. */
static void or_rk4_vjp(const double p[3], const double B[3], int32_t q, double d, double rbar[3], double pbar[3],
                       double Bbar[3])
{
    double P0 = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    double qk = OR_KAPPA * (double)q;
    double k1r[3], k1p[3], k2r[3], k2p[3], k3r[3], k3p[3], k4r[3], k4p[3];
    double t1[3], t2[3], t3[3];
    or_deriv(p, B, qk, P0, k1r, k1p);
    for (int c = 0; c < 3; ++c) t1[c] = p[c] + 0.5 * d * k1p[c];
    or_deriv(t1, B, qk, P0, k2r, k2p);
    for (int c = 0; c < 3; ++c) t2[c] = p[c] + 0.5 * d * k2p[c];
    or_deriv(t2, B, qk, P0, k3r, k3p);
    for (int c = 0; c < 3; ++c) t3[c] = p[c] + d * k3p[c];
    or_deriv(t3, B, qk, P0, k4r, k4p);
    double ro[3], po[3], a1r[3], a1p[3], a2r[3], a2p[3], a3r[3], a3p[3], a4r[3], a4p[3];
    for (int c = 0; c < 3; ++c) {
        ro[c] = rbar[c];
        po[c] = pbar[c];
        a1r[c] = d / 6.0 * ro[c];
        a2r[c] = d / 3.0 * ro[c];
        a3r[c] = d / 3.0 * ro[c];
        a4r[c] = d / 6.0 * ro[c];
        a1p[c] = d / 6.0 * po[c];
        a2p[c] = d / 3.0 * po[c];
        a3p[c] = d / 3.0 * po[c];
        a4p[c] = d / 6.0 * po[c];
    }
    double P0bar = 0.0, t3bar[3] = {0, 0, 0}, t2bar[3] = {0, 0, 0}, t1bar[3] = {0, 0, 0};
    double pb[3] = {po[0], po[1], po[2]};
    or_deriv_vjp(t3, B, qk, P0, a4r, a4p, t3bar, Bbar, &P0bar);
    for (int c = 0; c < 3; ++c) {
        pb[c] += t3bar[c];
        a3p[c] += d * t3bar[c];
    }
    or_deriv_vjp(t2, B, qk, P0, a3r, a3p, t2bar, Bbar, &P0bar);
    for (int c = 0; c < 3; ++c) {
        pb[c] += t2bar[c];
        a2p[c] += 0.5 * d * t2bar[c];
    }
    or_deriv_vjp(t1, B, qk, P0, a2r, a2p, t1bar, Bbar, &P0bar);
    for (int c = 0; c < 3; ++c) {
        pb[c] += t1bar[c];
        a1p[c] += 0.5 * d * t1bar[c];
    }
    or_deriv_vjp(p, B, qk, P0, a1r, a1p, pb, Bbar, &P0bar);
    for (int c = 0; c < 3; ++c) pb[c] += P0bar * p[c] / P0;
    for (int c = 0; c < 3; ++c) {
        pbar[c] = pb[c];
        /* rbar passes through unchanged (r enters additively) */
    }
}

/* Forward with a tape, then the reverse sweep, for one muon.  g6 holds
 * dL/d(final x,y,z,px,py,pz); dalpha[3*block + c] accumulates dL/dalpha. */
static void or_adjoint_one(const or_world *w, const double r0[3], const double p0[3], int32_t q, int32_t steps0,
                           uint8_t status0, uint64_t id, int32_t inst, double d, int32_t max_steps, uint64_t seed,
                           const double g6[6], double *dalpha, or_tape *tape)
{
    if (status0 != OR_ALIVE && status0 != OR_MAX_STEPS) return;
    double r[3] = {r0[0], r0[1], r0[2]}, p[3] = {p0[0], p0[1], p0[2]};
    for (int c = 0; c < 3; ++c)
        if (!isfinite(r[c]) || !isfinite(p[c])) return;
    int32_t ns = 0;
    for (int32_t k = steps0; k < max_steps; ++k) {
        if (or_check(w, r, p) != OR_ALIVE) break;
        or_tape *t = &tape[ns++];
        for (int c = 0; c < 3; ++c) {
            t->r[c] = r[c];
            t->p[c] = p[c];
        }
        or_step_draw dr;
        t->scattered = or_draw_step(w, r, p, k, id, inst, seed, &dr);
        t->box = dr.box;
        t->f = dr.f;
        t->theta = dr.theta;
        t->phi = dr.phi;
        if (t->scattered) or_scatter_draw(w, p, &dr, p);
        if (w->field_per_stage) {
            or_rk4_staged(w, r, p, dr.box, q, d);   /* reads the field at each stage itself */
        } else {
            double B[3];
            or_field(w, r, dr.box, B);
            or_rk4(r, p, B, q, d);
        }
    }
    double rbar[3] = {g6[0], g6[1], g6[2]}, pbar[3] = {g6[3], g6[4], g6[5]};
    for (int32_t s = ns - 1; s >= 0; --s) {
        const or_tape *t = &tape[s];
        double ps[3] = {t->p[0], t->p[1], t->p[2]};
        double cz = 0.0, ct = 0.0;
        if (t->scattered) {
            or_dp_coeffs(w->axes, t->f, t->theta, &cz, &ct);
            or_scatter_c(t->p, cz, ct, t->phi, ps);
        }
        double Bm[3], J[3][3], B[3];
        or_field_unscaled(w, t->r, t->box, Bm, J);
        int32_t blk = or_block_of(w, t->box);
        for (int c = 0; c < 3; ++c) B[c] = blk >= 0 ? w->alpha[3 * blk + c] * Bm[c] : Bm[c];
        double Bbar[3] = {0, 0, 0};
        or_rk4_vjp(ps, B, q, d, rbar, pbar, Bbar);     /* rbar unchanged, pbar -> cotangent of ps */
        for (int c = 0; c < 3; ++c) {
            double Bmbar = blk >= 0 ? w->alpha[3 * blk + c] * Bbar[c] : Bbar[c];
            if (blk >= 0) dalpha[3 * blk + c] += Bbar[c] * Bm[c];
            for (int a = 0; a < 3; ++a) rbar[a] += J[c][a] * Bmbar;
        }
        if (t->scattered) {
            double pb[3] = {0, 0, 0};
            or_scatter_vjp(t->p, cz, ct, t->phi, pbar, pb);
            for (int c = 0; c < 3; ++c) pbar[c] = pb[c];
        }
    }
}

typedef struct or_adj_job {
    const or_world *w;
    int64_t begin, end, n;
    const double *x, *y, *z, *px, *py, *pz;
    const int8_t *q;
    const int32_t *steps;
    const uint8_t *status;
    int64_t id_offset;
    int32_t inst;
    double d;
    int32_t max_steps;
    uint64_t seed;
    const double *g;
    double dalpha[3 * 64];
} or_adj_job;

static void *or_adj_worker(void *arg)
{
    or_adj_job *j = (or_adj_job *)arg;
    or_tape *tape = (or_tape *)malloc(sizeof(or_tape) * (size_t)(j->max_steps > 0 ? j->max_steps : 1));
    if (!tape) return NULL;
    for (int64_t m = j->begin; m < j->end; ++m) {
        double r[3] = {j->x[m], j->y[m], j->z[m]}, p[3] = {j->px[m], j->py[m], j->pz[m]};
        double g6[6];
        for (int c = 0; c < 6; ++c) g6[c] = j->g[c * j->n + m];
        or_adjoint_one(j->w, r, p, j->q[m], j->steps[m], j->status[m], (uint64_t)(j->id_offset + m), j->inst, j->d,
                       j->max_steps, j->seed, g6, j->dalpha, tape);
    }
    free(tape);
    return NULL;
}

/* dL/dalpha for n muons given their INITIAL state and dL/d(final state) g
 * ([6][n] SoA).  dalpha has n_block*3 entries (overwritten).  Returns 0, or -1
 * for bad arguments (alpha must be set, n_block <= 64). */
int or_adjoint(const or_world *w, int64_t n, const double *x, const double *y, const double *z, const double *px,
               const double *py, const double *pz, const int8_t *q, const int32_t *steps, const uint8_t *status,
               int64_t id_offset, int32_t inst, double d, int32_t max_steps, uint64_t seed, const double *g,
               double *dalpha, int32_t n_threads)
{
    if (!w || !w->alpha || w->n_block < 1 || w->n_block > 64 || n < 0 || n_threads < 1) return -1;
    if (w->field_per_stage) return -3;          /* the adjoint holds the field over the step */
    for (int i = 0; i < 3 * w->n_block; ++i) dalpha[i] = 0.0;
    if (n == 0) return 0;
    if (n_threads > 256) n_threads = 256;
    if ((int64_t)n_threads > n) n_threads = (int32_t)n;
    or_adj_job *jobs = (or_adj_job *)calloc((size_t)n_threads, sizeof(or_adj_job));
    pthread_t th[256];
    if (!jobs) return -1;
    for (int32_t t = 0; t < n_threads; ++t) {
        or_adj_job *j = &jobs[t];
        j->w = w;
        j->begin = n * t / n_threads;
        j->end = n * (t + 1) / n_threads;
        j->n = n;
        j->x = x; j->y = y; j->z = z; j->px = px; j->py = py; j->pz = pz;
        j->q = q; j->steps = steps; j->status = status;
        j->id_offset = id_offset; j->inst = inst; j->d = d; j->max_steps = max_steps; j->seed = seed; j->g = g;
    }
    for (int32_t t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, or_adj_worker, &jobs[t]);
    or_adj_worker(&jobs[0]);
    for (int32_t t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
    for (int32_t t = 0; t < n_threads; ++t)
        for (int i = 0; i < 3 * w->n_block; ++i) dalpha[i] += jobs[t].dalpha[i];
    free(jobs);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Forward-mode dual numbers: an independent check of the adjoint.  Every     */
/* quantity carries its derivatives with respect to the OR_NT field scales.  */
/* ------------------------------------------------------------------------ */
#define OR_NT 18
typedef struct { double v, d[OR_NT]; } or_dual;

static or_dual dc(double v) { or_dual r; r.v = v; for (int i = 0; i < OR_NT; ++i) r.d[i] = 0.0; return r; }
static or_dual dadd(or_dual a, or_dual b) { for (int i = 0; i < OR_NT; ++i) a.d[i] += b.d[i]; a.v += b.v; return a; }
static or_dual dsub(or_dual a, or_dual b) { for (int i = 0; i < OR_NT; ++i) a.d[i] -= b.d[i]; a.v -= b.v; return a; }
static or_dual dmul(or_dual a, or_dual b)
{
    or_dual r;
    r.v = a.v * b.v;
    for (int i = 0; i < OR_NT; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
static or_dual dscale(or_dual a, double s) { for (int i = 0; i < OR_NT; ++i) a.d[i] *= s; a.v *= s; return a; }
static or_dual ddiv(or_dual a, or_dual b)
{
    or_dual r;
    r.v = a.v / b.v;
    for (int i = 0; i < OR_NT; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;
    return r;
}
static or_dual dsqrt(or_dual a)
{
    or_dual r;
    r.v = sqrt(a.v);
    for (int i = 0; i < OR_NT; ++i) r.d[i] = a.d[i] / (2.0 * r.v);
    return r;
}
static or_dual dnorm3(const or_dual v[3]) { return dsqrt(dadd(dadd(dmul(v[0], v[0]), dmul(v[1], v[1])), dmul(v[2], v[2]))); }

static void dscatter(or_dual p[3], double cz, double ct, double phi)
{
    or_dual P = dnorm3(p);
    or_dual ph[3] = {ddiv(p[0], P), ddiv(p[1], P), ddiv(p[2], P)};
    or_dual dt = dscale(P, ct);
    or_dual dz = dscale(P, cz);
    or_dual dp[3] = {dscale(dt, cos(phi)), dscale(dt, sin(phi)), dz};
    or_dual rot[3];
    or_dual s = dsqrt(dadd(dmul(ph[0], ph[0]), dmul(ph[1], ph[1])));
    if (s.v < 1e-12) {
        double sg = ph[2].v > 0.0 ? 1.0 : -1.0;
        rot[0] = dp[0];
        rot[1] = dscale(dp[1], sg);
        rot[2] = dscale(dp[2], sg);
    } else {
        or_dual k[3] = {dscale(ddiv(ph[1], s), -1.0), ddiv(ph[0], s), dc(0.0)};
        or_dual ca = ph[2], sa = s, omc = dsub(dc(1.0), ph[2]);
        or_dual kxv[3] = {dsub(dmul(k[1], dp[2]), dmul(k[2], dp[1])), dsub(dmul(k[2], dp[0]), dmul(k[0], dp[2])),
                          dsub(dmul(k[0], dp[1]), dmul(k[1], dp[0]))};
        or_dual kv = dadd(dadd(dmul(k[0], dp[0]), dmul(k[1], dp[1])), dmul(k[2], dp[2]));
        for (int c = 0; c < 3; ++c) rot[c] = dadd(dadd(dmul(dp[c], ca), dmul(kxv[c], sa)), dmul(dmul(k[c], kv), omc));
    }
    for (int c = 0; c < 3; ++c) p[c] = dadd(p[c], rot[c]);
}

static void dderiv(const or_dual x[3], const or_dual B[3], double qk, or_dual P0, or_dual dr[3], or_dual dp[3])
{
    for (int c = 0; c < 3; ++c) dr[c] = ddiv(x[c], P0);
    or_dual xB[3] = {dsub(dmul(x[1], B[2]), dmul(x[2], B[1])), dsub(dmul(x[2], B[0]), dmul(x[0], B[2])),
                     dsub(dmul(x[0], B[1]), dmul(x[1], B[0]))};
    for (int c = 0; c < 3; ++c) dp[c] = ddiv(dscale(xB[c], qk), P0);
}

static void drk4(or_dual r[3], or_dual p[3], const or_dual B[3], int32_t q, double d)
{
    or_dual P0 = dnorm3(p);
    double qk = OR_KAPPA * (double)q;
    or_dual k1r[3], k1p[3], k2r[3], k2p[3], k3r[3], k3p[3], k4r[3], k4p[3], t[3];
    dderiv(p, B, qk, P0, k1r, k1p);
    for (int c = 0; c < 3; ++c) t[c] = dadd(p[c], dscale(k1p[c], 0.5 * d));
    dderiv(t, B, qk, P0, k2r, k2p);
    for (int c = 0; c < 3; ++c) t[c] = dadd(p[c], dscale(k2p[c], 0.5 * d));
    dderiv(t, B, qk, P0, k3r, k3p);
    for (int c = 0; c < 3; ++c) t[c] = dadd(p[c], dscale(k3p[c], d));
    dderiv(t, B, qk, P0, k4r, k4p);
    for (int c = 0; c < 3; ++c) {
        or_dual sr = dadd(dadd(k1r[c], dscale(k2r[c], 2.0)), dadd(dscale(k3r[c], 2.0), k4r[c]));
        or_dual sp = dadd(dadd(k1p[c], dscale(k2p[c], 2.0)), dadd(dscale(k3p[c], 2.0), k4p[c]));
        r[c] = dadd(r[c], dscale(sr, d / 6.0));
        p[c] = dadd(p[c], dscale(sp, d / 6.0));
    }
}

static void dfield(const or_world *w, const or_dual r[3], int32_t box, or_dual B[3])
{
    for (int c = 0; c < 3; ++c) B[c] = dc(0.0);
    if (w->field_kind == 1) {
        if (box >= 0)
            for (int c = 0; c < 3; ++c) B[c] = dc(w->box_B[3 * box + c]);
    } else if (w->field_kind == 2) {
        int64_t i0[3];
        or_dual t[3];
        int inside = 1;
        for (int a = 0; a < 3; ++a) {
            double u = (r[a].v - w->forigin[a]) / w->fspacing[a];
            if (!(u >= 0.0 && u <= (double)(w->fdims[a] - 1))) inside = 0;
            double fl = floor(u);
            if (fl > (double)(w->fdims[a] - 2)) fl = (double)(w->fdims[a] - 2);
            i0[a] = (int64_t)fl;
            t[a] = dsub(dscale(dsub(r[a], dc(w->forigin[a])), 1.0 / w->fspacing[a]), dc(fl));
        }
        if (inside) {
            const int64_t nx = w->fdims[0], ny = w->fdims[1];
            for (int dk = 0; dk < 2; ++dk)
                for (int dj = 0; dj < 2; ++dj)
                    for (int di = 0; di < 2; ++di) {
                        or_dual fx = di ? t[0] : dsub(dc(1.0), t[0]);
                        or_dual fy = dj ? t[1] : dsub(dc(1.0), t[1]);
                        or_dual fz = dk ? t[2] : dsub(dc(1.0), t[2]);
                        or_dual wgt = dmul(dmul(fx, fy), fz);
                        const float *node = w->Bmap + 3 * (((i0[2] + dk) * ny + (i0[1] + dj)) * nx + (i0[0] + di));
                        for (int c = 0; c < 3; ++c) B[c] = dadd(B[c], dscale(wgt, (double)node[c]));
                    }
        }
    } else if (w->field_kind == 3) {
        const double rv[3] = {r[0].v, r[1].v, r[2].v};
        double Bn[3];
        or_field_nearest(w, rv, Bn);
        for (int c = 0; c < 3; ++c) B[c] = dc(Bn[c]);
    }
    int32_t blk = or_block_of(w, box);
    if (blk >= 0)
        for (int c = 0; c < 3; ++c) {
            or_dual a = dc(w->alpha[3 * blk + c]);
            if (3 * blk + c < OR_NT) a.d[3 * blk + c] = 1.0;
            B[c] = dmul(a, B[c]);
        }
}

/* Final state of one muon and its derivatives with respect to the field scales
 * (tangent directions 3*block + c, at most OR_NT of them):
 * out6 = final (x,y,z,px,py,pz), tan[6][OR_NT].  Returns the number of steps. */
int32_t or_transport_tangent(const or_world *w, const double r0[3], const double p0[3], int32_t q, int32_t steps0,
                             uint64_t id, int32_t inst, double d, int32_t max_steps, uint64_t seed, double out6[6],
                             double *tan)
{
    or_dual r[3], p[3];
    for (int c = 0; c < 3; ++c) {
        r[c] = dc(r0[c]);
        p[c] = dc(p0[c]);
    }
    int32_t ns = 0;
    for (int32_t k = steps0; k < max_steps; ++k) {
        double rv[3] = {r[0].v, r[1].v, r[2].v}, pv[3] = {p[0].v, p[1].v, p[2].v};
        if (or_check(w, rv, pv) != OR_ALIVE) break;
        or_step_draw dr;
        if (or_draw_step(w, rv, pv, k, id, inst, seed, &dr)) {
            double cz, ct;
            or_dp_coeffs(w->axes, dr.f, dr.theta, &cz, &ct);
            dscatter(p, cz, ct, dr.phi);
        }
        or_dual B[3];
        dfield(w, r, dr.box, B);
        drk4(r, p, B, q, d);
        ++ns;
    }
    for (int c = 0; c < 3; ++c) {
        out6[c] = r[c].v;
        out6[3 + c] = p[c].v;
        for (int i = 0; i < OR_NT; ++i) {
            tan[c * OR_NT + i] = r[c].d[i];
            tan[(3 + c) * OR_NT + i] = p[c].d[i];
        }
    }
    return ns;
}

/* ------------------------------------------------------------------------ */
/* Offline phase (Sec. Building histograms, Appendix A) with a parametric    */
/* stand-in for the paper's Geant4 runs.  One sample of the step of a muon of */
/* momentum p [GeV] through x [cm] of a material (rho [g/cm^3], Z/A, I [MeV],  */
/* X0 [cm], b [cm^2/g]) draws from eight uniforms u[0..7]:                    */
/*   ionisation: a Moyal loss of the PDG thin-absorber width xi and most      */
/*     probable value dmp (density effect with the plasma energy), from a      */
/*     normal z = sqrt(-2 ln u1) cos(2 pi u2) as xi (-ln z^2) + dmp, floored   */
/*     at 0, f = dE / p;                                                       */
/*   radiative tail: with probability b rho x / <v>, v ~ v^-2 on [1e-3, 1)     */
/*     (inverse CDF of u4) is added to f when u3 is below that probability;   */
/*   scattering: theta = theta0 sqrt(-2 ln u7) (a Rayleigh space angle of the */
/*     Highland width theta0), or 2 theta0 / sqrt(u6) when u5 < 0.01 (single  */
/*     scatter tail).                                                          */
/* Uniforms are (w >> 8 + 1/2) 2^-24 of the words of Philox4x32-10 with key   */
/* = seed and counters (s, h, 0x0FF1, 0) and (s, h, 0x0FF1, 1) for sample s of */
/* stream h.                                                                   */
/* ------------------------------------------------------------------------ */
typedef struct or_material_c {
    double rho, za, I, X0, b;
} or_material_c;

#define OR_K_BETHE 0.307075
#define OR_ME 0.51099895
#define OR_MMU 105.6583755

static double or_u_open(uint32_t w) { return ((double)(w >> 8) + 0.5) * (1.0 / 16777216.0); }

double or_highland(double p_gev, double x_cm, double X0)
{
    double pm = p_gev * 1e3, E = sqrt(pm * pm + OR_MMU * OR_MMU), beta = pm / E, t = x_cm / X0;
    return 13.6 / (beta * pm) * sqrt(t) * (1.0 + 0.038 * log(t));
}

void or_physics_sample(const or_material_c *m, double p, double x_cm, const double u[8], double *f, double *theta)
{
    double pm = p * 1e3;
    double E = sqrt(pm * pm + OR_MMU * OR_MMU);
    double beta2 = (pm / E) * (pm / E);
    double bg = pm / OR_MMU;
    double xi = 0.5 * OR_K_BETHE * m->za * m->rho * x_cm / beta2;
    double hw = 28.816e-6 * sqrt(m->rho * m->za);
    double delta = 2.0 * log(bg) + 2.0 * log(hw / m->I) - 1.0;
    if (delta < 0.0) delta = 0.0;
    double dmp = xi * (log(2.0 * OR_ME * bg * bg / m->I) + log(xi / m->I) + 0.2 - beta2 - delta);
    double z = sqrt(-2.0 * log(u[1])) * cos(OR_TWO_PI * u[2]);
    double z2 = z * z;
    if (z2 < 1e-300) z2 = 1e-300;
    double dE = dmp + xi * (-log(z2));
    if (dE < 0.0) dE = 0.0;
    double ff = dE / pm;
    const double v0 = 1e-3;
    double mean_v = log(1.0 / v0) / (1.0 / v0 - 1.0);
    double p_rad = m->b * m->rho * x_cm / mean_v;
    if (p_rad > 1.0) p_rad = 1.0;
    if (u[3] < p_rad) ff += 1.0 / (1.0 / v0 - u[4] * (1.0 / v0 - 1.0));
    double th0 = or_highland(p, x_cm, m->X0);
    *theta = u[5] < 0.01 ? 2.0 * th0 / sqrt(u[6]) : th0 * sqrt(-2.0 * log(u[7]));
    *f = ff;
}

static void or_physics_uniforms(uint64_t seed, uint64_t s, uint32_t h, double u[8])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    for (int half = 0; half < 2; ++half) {
        uint32_t ctr[4] = {(uint32_t)s, h, 0x0FF1u, (uint32_t)half};
        or_philox4x32_10(ctr, key, w);
        for (int j = 0; j < 4; ++j) u[4 * half + j] = or_u_open(w[j]);
    }
}

/* Histograms H[m][i] (linear axes) from n_samples samples each: p ~ U(edge_i,
 * edge_{i+1}) from u0, stream h = m n_pbin + i; f binned on [0, f_max) and
 * theta on [0, theta_max[m][i]) with theta_max = 5 theta0(edge_i); samples
 * outside the axes are counted in the edge cells.  counts [n_mat][n_pbin][nf][ntheta]. */
int or_build_histograms(const or_material_c *mats, int32_t n_mat, int32_t n_pbin, const double *edges, int32_t nf,
                        int32_t ntheta, double f_max, double x_cm, int64_t n_samples, uint64_t seed, double *counts,
                        double *theta_max)
{
    for (int32_t m = 0; m < n_mat; ++m)
        for (int32_t i = 0; i < n_pbin; ++i) {
            const uint32_t h = (uint32_t)(m * n_pbin + i);
            const double tm = 5.0 * or_highland(edges[i], x_cm, mats[m].X0);
            theta_max[h] = tm;
            double *H = counts + (int64_t)h * nf * ntheta;
            for (int64_t k = 0; k < (int64_t)nf * ntheta; ++k) H[k] = 0.0;
            for (int64_t s = 0; s < n_samples; ++s) {
                double u[8], f, th;
                or_physics_uniforms(seed, (uint64_t)s, h, u);
                const double p = edges[i] + u[0] * (edges[i + 1] - edges[i]);
                or_physics_sample(&mats[m], p, x_cm, u, &f, &th);
                double a = floor(f / f_max * nf), b = floor(th / tm * ntheta);
                if (!(a >= 0.0)) a = 0.0;
                if (a > nf - 1) a = nf - 1;
                if (!(b >= 0.0)) b = 0.0;
                if (b > ntheta - 1) b = ntheta - 1;
                H[(int64_t)a * ntheta + (int64_t)b] += 1.0;
            }
        }
    return 0;
}

/* Pilot estimator of Appendix A: phi(p) = (1/K) sum_k log(-dPz_k/P) for K
 * samples at the probe momentum p (stream h = probe index), with
 * -dPz/P = 1 - (1 - f) cos theta = f + (1 - f) 2 sin^2(theta/2), f capped at 1. */
int or_pilot_phi(const or_material_c *m, const double *probes, int32_t n_probe, int64_t K, double x_cm, uint64_t seed,
                 double *phi)
{
    for (int32_t j = 0; j < n_probe; ++j) {
        double acc = 0.0;
        for (int64_t s = 0; s < K; ++s) {
            double u[8], f, th;
            or_physics_uniforms(seed, (uint64_t)s, (uint32_t)j, u);
            or_physics_sample(m, probes[j], x_cm, u, &f, &th);
            if (f > 1.0) f = 1.0;
            const double sh = sin(0.5 * th);
            acc += log(f + (1.0 - f) * 2.0 * sh * sh);
        }
        phi[j] = acc / (double)K;
    }
    return 0;
}

/* Bounded-variation bin edges (Appendix A) on a probe grid: from edge p_i the
 * next edge is the largest probe p_j with max_{i <= k <= j} |phi_k - phi_i| <=
 * eps (at least the next probe, the grid's resolution); the last edge is the
 * last probe.  Returns the number of edges written (<= max_edges), or -1 if
 * they do not fit. */
int32_t or_bv_edges(const double *probes, const double *phi, int32_t n_probe, double eps, double *edges,
                    int32_t max_edges)
{
    if (n_probe < 2 || max_edges < 2) return -1;
    int32_t n = 0, i = 0;
    edges[n++] = probes[0];
    while (i < n_probe - 1) {
        int32_t j = i + 1;
        while (j + 1 < n_probe && fabs(phi[j + 1] - phi[i]) <= eps) {
            int ok = 1;
            for (int32_t k = i + 1; k <= j + 1; ++k)
                if (fabs(phi[k] - phi[i]) > eps) ok = 0;
            if (!ok) break;
            ++j;
        }
        if (n >= max_edges) return -1;
        edges[n++] = probes[j];
        i = j;
    }
    return n;
}
