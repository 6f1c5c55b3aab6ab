/*
 * mt.h -- C ABI of the GB300 (sm_103a) muon transport library libmt.so.
 *
 * Implements the online phase of "Ultra-Fast Muon Transport via Histogram
 * Sampling on GPUs" (arXiv 2512.10520): the per-muon transport loop of
 * Algorithm 1 (Sec. "Simulation").  Each muon repeatedly
 *   (1) looks up its material in the geometry        (Sec. Simulation, item 1),
 *   (2) draws a fractional momentum loss f and a polar scattering angle theta
 *       from the precomputed histogram H_{M,i} of its material M and log10
 *       momentum bin i (Sec. Momentum binning), by inverse CDF over a
 *       Philox4x32-10 draw, plus uniform jitter and an isotropic azimuth, and
 *       rotates that kick into the global frame with Rodrigues' formula (Eq. 3),
 *   (3) advances one fixed step d through the magnetic field with an RK4
 *       Lorentz-force step (Eq. 4), the field looked up once per step,
 * until its momentum falls below p_min or it leaves the world box.
 *
 * Conventions shared by every entry point:
 *  - Units: metres, GeV/c, tesla.  kappa = 0.299792458 GeV/(T m) per unit charge.
 *  - Every function returns an mt_status; nothing throws, traps or aborts across
 *    the ABI.  On failure mt_last_error() returns a thread-local message.
 *  - Pointers named "host" are host memory; pointers in mt_muon_soa and those
 *    named "device" are device memory of the handle's GPU.
 *  - A handle is immutable after mt_create and may be used from several host
 *    threads and streams at once; results depend only on the inputs, the seed
 *    and the muon ids, never on launch configuration or chunking.
 */
#ifndef MT_H
#define MT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MT_ABI_VERSION 1

typedef enum mt_status {
    MT_OK = 0,
    MT_ERR_INVALID_ARG = 1,  /* a null pointer, a negative size, a bad descriptor field */
    MT_ERR_CUDA = 2,         /* a CUDA runtime call failed (message says which)       */
    MT_ERR_OOM = 3,          /* device allocation failed                              */
    MT_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up                    */
    MT_ERR_TABLE = 5,        /* histogram weights negative, non-finite or all zero    */
    MT_ERR_DEVICE = 6        /* a device-side check failed (index out of range)       */
} mt_status;

/* Per-muon status byte (Algorithm 1's break conditions). */
enum {
    MT_ALIVE = 0,      /* not terminated; transported by the next call            */
    MT_STOPPED = 1,    /* |p| < p_min at the start of a step                      */
    MT_EXIT_Z = 2,     /* z >= z_max at the start of a step                       */
    MT_EXIT_XY = 3,    /* |x| >= x_max or |y| >= y_max at the start of a step     */
    MT_MAX_STEPS = 4,  /* ran out of steps; resumable like MT_ALIVE               */
    MT_INVALID = 5     /* non-finite position or momentum on entry                */
};

enum { MT_GEOM_BOXES = 0, MT_GEOM_VOXELS = 1, MT_GEOM_POLYHEDRA = 2 };
enum { MT_FIELD_NONE = 0, MT_FIELD_BOX = 1, MT_FIELD_MAP = 2, MT_FIELD_MAP_NEAREST = 3 };

#define MT_MAX_BOXES 32
#define MT_MAX_MATERIALS 15
#define MT_MAX_PBINS 256
#define MT_MAX_CELLS 32768

/* Axis-aligned half-open box lo <= r < hi.  Boxes are tested in list order and
 * the first one containing r gives the material (Sec. Simulation, item 1).
 * block_id >= 0 marks a magnet block whose field is scaled by alpha[block_id]
 * in the differentiable form; B is the uniform field inside the box when the
 * field kind is MT_FIELD_BOX. */
typedef struct mt_box {
    double lo[3];
    double hi[3];
    int32_t material;   /* 0 = vacuum, 1..n_mat = histogrammed material */
    int32_t block_id;   /* -1 or a field-scale block index < MT_MAX_BOXES */
    double B[3];
} mt_box;

/* A solid of the convex-polyhedron geometry (Sec. Simulation item 1): it spans
 * z0 <= z < z1, and its cross-section at height z is the quadrilateral whose
 * vertices move linearly from bottom[i] (at z0) to top[i] (at z1), with
 * t = (z - z0) / (z1 - z0).  Both quadrilaterals are strictly convex and
 * counter-clockwise seen from +z.  A point is inside when, for every edge
 * e_i = v_{i+1} - v_i of its slice, S_i = e_ix (y - v_iy) - e_iy (x - v_ix) >= 0
 * (Eq. 2: all signs consistent; points on the side faces are inside).  Solids
 * are tested in list order and the first containing one gives the material;
 * material, block_id and B as for mt_box. */
typedef struct mt_polyhedron {
    double z0, z1;
    double bottom[4][2];
    double top[4][2];
    int32_t material;
    int32_t block_id;
    double B[3];
} mt_polyhedron;

/* Geometry and the break conditions of Algorithm 1 (inputs p_min, r_max). */
typedef struct mt_geometry_desc {
    int32_t kind;                 /* MT_GEOM_BOXES, MT_GEOM_VOXELS or MT_GEOM_POLYHEDRA  */
    int32_t n_boxes;              /* boxes: 0..MT_MAX_BOXES                              */
    const mt_box *boxes;          /* host, n_boxes entries                               */
    int32_t world_material;       /* material outside every box / voxel grid             */
    int32_t vox_dims[3];          /* voxels: nx, ny, nz (each >= 1)                      */
    double vox_origin[3];         /* voxels: corner of voxel (0,0,0)                     */
    double vox_spacing[3];        /* voxels: edge lengths (> 0)                          */
    const uint8_t *voxels;        /* host, [nz][ny][nx] material ids                     */
    double x_max, y_max, z_max;   /* stop when |x| >= x_max, |y| >= y_max or z >= z_max  */
    double p_min;                 /* stop when |p| < p_min                               */
    const mt_polyhedron *polys;   /* polyhedra: host, n_polys entries                    */
    int32_t n_polys;              /* polyhedra: 0..MT_MAX_BOXES                          */
    int32_t reserved;             /* 0                                                   */
} mt_geometry_desc;

/* Magnetic field.  MT_FIELD_MAP: node-based map, node (i,j,k) at
 * origin + (i,j,k)*spacing, trilinear interpolation, zero outside the node box
 * (the paper's regular-grid field, Sec. Simulation item 3).
 * MT_FIELD_MAP_NEAREST: the same map read at the nearest node, the paper's own
 * lookup: along each axis node i owns [origin + (i - 1/2) s, origin + (i + 1/2) s);
 * zero where that node is outside the map.  No dB/dr (piecewise constant).
 * MT_FIELD_BOX: the uniform field B of the box or solid holding the point. */
typedef struct mt_field_desc {
    int32_t kind;                 /* MT_FIELD_NONE / _BOX / _MAP / _MAP_NEAREST       */
    int32_t dims[3];              /* map: nx, ny, nz (each >= 2)                      */
    double origin[3];
    double spacing[3];            /* > 0                                             */
    const float *B;               /* host, [nz][ny][nx][3] float32 (Bx, By, Bz)       */
    int32_t per_stage;            /* MT_FIELD_MAP only: 1 = RK4 reads the map at each */
    int32_t reserved;             /*   stage's position (see below); 0 = once a step  */
} mt_field_desc;

/* per_stage = 1 is a variant of the step: Algorithm 1 reads the field once, at
 * the start of the step, and holds it over the RK4 stages (the default); with
 * per_stage the stages at r + d/2 k1, r + d/2 k2 and r + d k3 read the map
 * there (scaled by the block of the step's start), which makes the step fourth
 * order in a varying field.  The differentiable form does not take it
 * (MT_ERR_INVALID_ARG). */

/* Histogram set H_{M,i} (Sec. Building histograms): for materials M = 1..n_mat
 * and log10 momentum bins i = 0..n_pbin-1 on [p_lo, p_hi] (edges
 * p_lo (p_hi/p_lo)^(i/n_pbin); momenta outside use the edge bins), a joint
 * histogram of f = dp/p on [0, f_max) (nf bins) and theta on [0, theta_max)
 * (ntheta bins).  weights are non-negative counts or probabilities; each
 * histogram must have a positive, finite sum. */
typedef struct mt_hist_desc {
    int32_t n_mat;                /* 1..MT_MAX_MATERIALS                              */
    int32_t n_pbin;               /* 1..MT_MAX_PBINS                                  */
    double p_lo, p_hi;            /* 0 < p_lo < p_hi                                  */
    int32_t nf, ntheta;           /* nf * ntheta in [2, MT_MAX_CELLS]                 */
    const double *weights;        /* host, [n_mat][n_pbin][nf][ntheta]                */
    const double *f_max;          /* host, [n_mat][n_pbin], > 0                       */
    const double *theta_max;      /* host, [n_mat][n_pbin], > 0                       */
    int32_t sampler;              /* MT_SAMPLER_ICDF (0, default) or MT_SAMPLER_ALIAS */
    int32_t axes;                 /* MT_AXES_LINEAR (0, default) or MT_AXES_LOG       */
    const double *f_min;          /* log axes: host, [n_mat][n_pbin], 0 < f_min < f_max */
    const double *theta_min;      /* log axes: host, [n_mat][n_pbin], 0 < t_min < t_max */
    const double *p_edges;        /* host, n_pbin + 1 momentum-bin edges, or NULL for */
                                  /*   log10 bins (see below)                         */
} mt_hist_desc;

/* Momentum bins.  p_edges NULL: n_pbin log10 bins on [p_lo, p_hi].  Otherwise
 * explicit edges (e.g. the bounded-variation bins of Appendix A, mt_bv_edges):
 * strictly increasing, p_edges[0] = p_lo, p_edges[n_pbin] = p_hi, neighbours at
 * least 1e-5 apart relatively; the step finds the bin by binary search (the
 * run-time search Appendix A calls for).  Momenta outside use the edge bins. */

/* Histogram axes.  MT_AXES_LINEAR: f = dp/p on [0, f_max) and the polar angle
 * theta on [0, theta_max), linear bins; the step sets |p| to (1 - f) |p| at
 * angle theta.  MT_AXES_LOG: the paper's variables (Sec. Building histograms)
 * f = -dPz/|P| on [f_min, f_max) and t = dPt/|P| on [theta_min, theta_max),
 * log-spaced bins with the jitter uniform in log f and log t; the step adds
 * Algorithm 1's dp = [P t cos phi, P t sin phi, -P f] in the muon's frame. */
#define MT_AXES_LINEAR 0
#define MT_AXES_LOG 1

/* Samplers of a histogram cell from the draw w0 (Philox word 0).  Both use the
 * integer masses m_c = T_c - T_{c-1} of the thresholds T_c = floor(2^32 S_c /
 * S_total) (S_c the FP64 prefix sums of the weights, T_{ncell-1} = 2^32), so
 * both draw from exactly one quantised distribution:
 *  - MT_SAMPLER_ICDF: inverse CDF, cell = #{c < ncell-1 : T_c <= w0};
 *  - MT_SAMPLER_ALIAS: Walker's alias method (Sec. Methodology, "The Alias
 *    Method"), O(1): ncell = 2^n equiprobable columns, built by Vose's
 *    construction in integers (small/large stacks filled in cell order, popped
 *    from the top); column j = w0 >> (32-n) keeps its own cell when
 *    (w0 << n) mod 2^32 < Prob_j and takes Alias_j otherwise.  Needs nf and
 *    ntheta powers of two (MT_ERR_INVALID_ARG otherwise). */
#define MT_SAMPLER_ICDF 0
#define MT_SAMPLER_ALIAS 1

/* Muon state, structure of arrays in device memory, caller-owned, updated in
 * place (Algorithm 1's inputs r and p).  Muon m has the global id
 * id_offset + m; the Philox counter of step k is (k, id_lo, id_hi, instance). */
typedef struct mt_muon_soa {
    float *x, *y, *z;             /* position [m]                                     */
    float *px, *py, *pz;          /* momentum [GeV/c]                                 */
    int8_t *q;                    /* charge (+1 mu+, -1 mu-)                          */
    int32_t *steps;               /* steps already taken; step k runs from here       */
    uint8_t *status;              /* MT_ALIVE ... MT_INVALID                          */
    int64_t id_offset;
    int32_t instance;
    int32_t reserved;
} mt_muon_soa;

typedef struct mt_handle mt_handle;

/* Library ABI version (MT_ABI_VERSION of the build). */
int32_t mt_abi_version(void);

/* Thread-local description of the last failure in this thread ("" if none). */
const char *mt_last_error(void);

/* Build the device-resident static data of one world: geometry, field map and
 * sampling tables (the paper keeps all of its static inputs resident in GPU
 * global memory for the whole run, Sec. Simulation).  For each histogram the library normalises the weights into a
 * discrete CDF and quantises it to uint32 thresholds
 * T_j = floor(2^32 S_j / S_total) (S_j the left-to-right FP64 prefix sum), so the
 * cell of a 32-bit draw w is #{j < ncell-1 : T_j <= w}.
 * Runs on the current CUDA device, synchronously.  The caller keeps ownership
 * of every descriptor array and may free them when this returns.
 * Errors: MT_ERR_INVALID_ARG (bad descriptor), MT_ERR_TABLE (bad weights),
 * MT_ERR_OOM, MT_ERR_CUDA.  *out is NULL on failure. */
mt_status mt_create(const mt_geometry_desc *geometry, const mt_field_desc *field,
                    const mt_hist_desc *hist, mt_handle **out);

/* Release a handle and its device memory (NULL is a no-op).  The caller must
 * make sure no launch that uses it is still running. */
void mt_destroy(mt_handle *h);

/* Device bytes held by the handle (tables + field map). */
int64_t mt_device_bytes(const mt_handle *h);

/* Transport n muons in place (Algorithm 1), asynchronously on `stream`
 * (a cudaStream_t; NULL = legacy default stream).  Runs the MT_LAUNCH_AUTO
 * launch shape of mt_transport_cfg, whose scratch list comes from the
 * stream-ordered allocator (cudaMallocAsync / cudaFreeAsync on `stream`).  For each muon whose status
 * is MT_ALIVE or MT_MAX_STEPS it runs steps k = steps .. max_steps-1 and stops
 * at the first break condition; terminal statuses are left untouched.
 * step_len is d [m].  seed is the 64-bit Philox key.
 * Errors (returned before anything is enqueued): MT_ERR_INVALID_ARG for a null
 * handle/soa, null arrays with n > 0, n < 0, non-finite or non-positive
 * step_len, max_steps < 0; MT_ERR_OOM if the scratch allocation fails;
 * MT_ERR_CUDA if a launch fails. */
mt_status mt_transport(mt_handle *h, const mt_muon_soa *s, int64_t n, float step_len,
                       int32_t max_steps, uint64_t seed, void *stream);

/* As mt_transport, with the field inside magnet block b scaled component-wise
 * by alpha[3*b + c] (device, n_block x 3 floats, n_block <= MT_MAX_BOXES);
 * alpha = NULL is mt_transport.  This is the forward map of the
 * differentiable form (field-scale parameters of the paper's Discussion). */
mt_status mt_transport_scaled(mt_handle *h, const mt_muon_soa *s, int64_t n, float step_len,
                              int32_t max_steps, uint64_t seed, const float *alpha, int32_t n_block,
                              void *stream);

/* Launch shape of the transport kernels (performance only: results do not
 * depend on it).
 *  MT_LAUNCH_STATIC     one thread per muon over a grid covering all n muons;
 *  MT_LAUNCH_PERSISTENT a resident grid of (SM count x blocks_per_sm) blocks
 *                       whose lanes pick up the next muon of their block's range
 *                       as soon as the current one stops;
 *  MT_LAUNCH_COMPACT    lockstep passes: every live muon advances steps_per_pass
 *                       steps (warps take 32-muon chunks of the live list from
 *                       a per-pass counter), then the survivors are compacted into a scratch
 *                       list (two 64-byte entries per muon plus 256 bytes and
 *                       the spatial order's 128 KB, see
 *                       mt_transport_workspace_bytes) for the next pass; n must
 *                       be below 2^31.  With a field map the survivors can be
 *                       reordered by the coarse xy cell of the map they stand
 *                       in (a counting sort about every 64 steps), so a warp's
 *                       muons share their field-map corners; the order changes
 *                       no result.  A call of 2^19 muons or more runs as two
 *                       groups of half the muons, each with its own list, the
 *                       second on a stream the call creates (forked from and
 *                       joined back to `stream` with events, released when its
 *                       work is done), so one group's passes fill the SMs the
 *                       other's pass tails leave idle; the workspace holds both;
 *  MT_LAUNCH_AUTO       the fastest measured form: MT_LAUNCH_COMPACT with the
 *                       default pass length (the static grid for n >= 2^31). */
enum { MT_LAUNCH_AUTO = 0, MT_LAUNCH_STATIC = 1, MT_LAUNCH_PERSISTENT = 2, MT_LAUNCH_COMPACT = 3 };
enum { MT_ORDER_AUTO = 0, MT_ORDER_ALWAYS = 1, MT_ORDER_NEVER = 2 };
typedef struct mt_launch_cfg {
    int32_t mode;             /* MT_LAUNCH_*                                              */
    int32_t blocks_per_sm;    /* 0 = as many as fit (occupancy calculator)                */
    int32_t steps_per_pass;   /* MT_LAUNCH_COMPACT: steps between compactions, 0 = the    */
                              /*   longest of 128, 96, 64, 48, 32, 24, 16 whose slab of   */
                              /*   the field map fits in 3/4 of L2, or in 2.5 L2 when the */
                              /*   live list is ordered (64 without a map)                */
    int32_t order;            /* MT_LAUNCH_COMPACT, field maps: spatial order of the live */
                              /*   list: MT_ORDER_AUTO (at least 2^19 muons), _ALWAYS,    */
                              /*   _NEVER                                                 */
    void *workspace;          /* MT_LAUNCH_COMPACT: device scratch (256-byte aligned), or */
    int64_t workspace_bytes;  /*   NULL = taken from the stream-ordered allocator         */
} mt_launch_cfg;

/* Scratch bytes MT_LAUNCH_COMPACT needs for n muons. */
int64_t mt_transport_workspace_bytes(int64_t n);

/* Number of kernel launches one mt_transport_cfg call with these arguments
 * makes (the pass length and the spatial order as that call chooses them;
 * cfg may be NULL = auto); -1 for a null handle or invalid arguments.
 * Launches nothing. */
int64_t mt_transport_launches(const mt_handle *h, int64_t n, float step_len, int32_t max_steps,
                              const mt_launch_cfg *cfg);

/* mt_transport_scaled with an explicit launch shape (cfg may be NULL = auto).
 * Errors as mt_transport, plus MT_ERR_INVALID_ARG for an unknown mode or
 * order, a negative blocks_per_sm or steps_per_pass, a workspace that is too small or
 * not 256-byte aligned, or n >= 2^31 in compact mode; MT_ERR_OOM if the
 * stream-ordered allocation fails. */
mt_status mt_transport_cfg(mt_handle *h, const mt_muon_soa *s, int64_t n, float step_len, int32_t max_steps,
                           uint64_t seed, const float *alpha, int32_t n_block, const mt_launch_cfg *cfg,
                           void *stream);

/* ---------------------------------------------------------------------------
 * Batched form: many independent worlds (each its own geometry and field map,
 * all sharing one histogram set) transported in one sequence of launches.
 * The live muons of every instance advance in lockstep passes of
 * steps_per_pass steps; a device work queue hands items naming an instance to
 * a resident grid whose blocks stage that instance's world in shared memory,
 * and the block's warps take 32-muon chunks of the instance until none are
 * left; survivors are compacted per instance between passes.  From 2^19
 * muons in all, the call runs as two groups of about equal muon counts, each
 * its own launch sequence, the second on a stream the call creates (forked
 * from and joined back to `stream`).  The groups split at an instance
 * boundary when one leaves them within 1/16 of the muons of each other, else
 * inside the instance at the midpoint (a single instance included).  The paper
 * runs one geometry per launch; scanning many magnet configurations is the
 * design-optimisation use it motivates (Sec. Introduction).
 * ------------------------------------------------------------------------- */
typedef struct mt_batch mt_batch;

/* World staging of the batched pass (mt_batch_cfg.staging): each block copies
 * the current instance's world parameters into shared memory, or reads them
 * in place from the device table of instances (through L1). */
enum { MT_BATCH_STAGE_SHARED = 1, MT_BATCH_STAGE_GLOBAL = 2 };

typedef struct mt_batch_cfg {
    int32_t block;            /* threads per block: 128 or 256; 0 = tuned / 256      */
    int32_t steps_per_pass;   /* steps between compactions; 0 = tuned, else as the   */
                              /*   plain transport picks it for the largest map        */
    int32_t use_graph;        /* 1 = capture the launch sequence in a CUDA graph once */
                              /*     per (workspace, sizes, arguments) and replay it  */
    int32_t staging;          /* MT_BATCH_STAGE_*; 0 = tuned / shared                 */
    int32_t order;            /* field maps: spatial order of every instance's live   */
                              /*   list between passes, as mt_launch_cfg.order        */
                              /*   (MT_ORDER_AUTO: 2^19 muons or more in the batch)   */
    int32_t reserved;         /* 0                                                    */
    void *workspace;          /* device scratch (256-byte aligned) of at least        */
    int64_t workspace_bytes;  /*   mt_batch_workspace_bytes, or NULL: stream-ordered  */
                              /*   scratch per call, or with use_graph the batch's    */
                              /*   own, kept for replays (growing it synchronises the */
                              /*   device)                                            */
} mt_batch_cfg;

/* A batch of n_inst worlds sharing the histogram set `hist` (copied, as in
 * mt_create).  Every instance must then be given a world with
 * mt_batch_set_instance before the batch is transported.  Synchronous. */
mt_status mt_batch_create(const mt_hist_desc *hist, int32_t n_inst, mt_batch **out);

/* Geometry and field of instance i (copied to the device, synchronously; the
 * caller may free its arrays on return).  All instances need the same geometry
 * kind and field kind.  Errors: MT_ERR_INVALID_ARG for a bad descriptor, an
 * index out of range or a different kind, MT_ERR_OOM, MT_ERR_CUDA. */
mt_status mt_batch_set_instance(mt_batch *b, int32_t i, const mt_geometry_desc *geometry,
                                const mt_field_desc *field);

/* Release a batch and its device memory (NULL is a no-op). */
void mt_batch_destroy(mt_batch *b);

/* Device bytes held by the batch (tables, every instance's geometry and map). */
int64_t mt_batch_device_bytes(const mt_batch *b);

/* Scratch bytes mt_transport_batched needs for the counts n[0..n_inst-1]. */
int64_t mt_batch_workspace_bytes(const mt_batch *b, const int64_t *n);

/* Transport the muons of every instance in place (Algorithm 1 in each world).
 * soas, n: host arrays of n_inst entries; soas[i] describes instance i's muons
 * (device arrays, ids id_offset + m, Philox counter word 3 = soas[i].instance).
 * Results equal n_inst separate mt_transport calls.  Asynchronous on `stream`;
 * calls on one batch must not overlap (the batch holds the cached graph).
 * Errors: MT_ERR_INVALID_ARG (null arrays, unset instance, bad cfg or counts),
 * MT_ERR_OOM, MT_ERR_CUDA. */
mt_status mt_transport_batched(mt_batch *b, const mt_muon_soa *soas, const int64_t *n, float step_len,
                               int32_t max_steps, uint64_t seed, const mt_batch_cfg *cfg, void *stream);

/* Pick the block size (128, 256) and pass length (32, 64, 128) that transport
 * a sample (the first sample_per_instance muons of every instance, copied to
 * scratch; the caller's muons are not modified) fastest; the choice is kept
 * in the batch for calls whose cfg leaves them 0 and returned in *best (may be
 * NULL).  Synchronises `stream`. */
mt_status mt_batch_autotune(mt_batch *b, const mt_muon_soa *soas, const int64_t *n, float step_len,
                            int32_t max_steps, uint64_t seed, int64_t sample_per_instance, mt_batch_cfg *best,
                            void *stream);

/* ---------------------------------------------------------------------------
 * Differentiable form.  The paper's Discussion proposes turning the histogram
 * transport into a differentiable layer so that magnet fields can be optimised
 * by gradient descent.  Parameters: per-magnet field scales alpha (device,
 * n_block x 3 floats, B inside block b scaled component-wise by alpha[3b+c]).
 * Gradients are pathwise: every draw of every step (material, box, momentum
 * bin, cell, f, theta, phi) and every muon's step count are held fixed (common
 * random numbers); the scattering rotation (Eq. 3), the trilinear field (with
 * its gradient in r) and the RK4 step (Eq. 4) are differentiated by
 * hand-written adjoints.  Checkpoints every ckpt_every = K steps (1..64) bound
 * the memory: the backward recomputes each K-step segment from its checkpoint.
 * ------------------------------------------------------------------------- */

/* Bytes of checkpoint storage for n muons (n < 2^31). */
int64_t mt_ckpt_bytes(int64_t n, int32_t max_steps, int32_t ckpt_every);

/* Checkpointing forward: exactly mt_transport_scaled (same results), keeping
 * the state of every muon alive at steps 0, K, 2K, ... in `ckpt` (device,
 * 256-byte aligned, at least mt_ckpt_bytes bytes, caller-owned and reused by
 * mt_adjoint_ckpt).  From 2^19 muons the two halves of the muons are
 * checkpointed as two groups side by side, the second on a stream the call
 * creates (forked from and joined back to `stream`), each with its own part of
 * `ckpt`.  Errors as mt_transport_scaled, plus MT_ERR_INVALID_ARG for K
 * outside [1, 64], n >= 2^31 or a checkpoint buffer too small / unaligned. */
mt_status mt_transport_ckpt(mt_handle *h, const mt_muon_soa *s, int64_t n, float step_len, int32_t max_steps,
                            uint64_t seed, const float *alpha, int32_t n_block, int32_t ckpt_every, void *ckpt,
                            int64_t ckpt_bytes, void *stream);

/* Backward from the checkpoints of one mt_transport_ckpt call, which must be
 * given the same n, step_len, max_steps, seed, alpha (values), ckpt_every,
 * id_offset and instance.  dL_dfinal: device [6][n] floats, dL/d(x, y, z, px,
 * py, pz) of the final state (SoA rows).  dL_dalpha: device [n_block][3],
 * overwritten.  dL_dinitial (may be NULL): device [6][n], receives dL/d(initial
 * state) in the same layout.  The checkpoint buffer's header is used as the
 * gradient accumulator; its lists are only read.  Only the muons whose six
 * dL_dfinal components are not all zero are recomputed and reversed (the
 * backward is linear in dL_dfinal); the others' rows of dL_dinitial are 0.  The
 * two muon groups of mt_transport_ckpt run side by side as in the forward.
 * Scratch (per group two slots, each the tape of one K-step segment, 56 K n
 * bytes, and a list of 64 n bytes, plus 6n floats when dL_dinitial is NULL)
 * comes from the stream-ordered allocator.  Errors: MT_ERR_INVALID_ARG for
 * null or inconsistent arguments, MT_ERR_OOM, MT_ERR_CUDA. */
mt_status mt_adjoint_ckpt(mt_handle *h, int64_t n, float step_len, int32_t max_steps, uint64_t seed,
                          const float *alpha, int32_t n_block, int32_t ckpt_every, void *ckpt, int64_t ckpt_bytes,
                          int64_t id_offset, int32_t instance, const float *dL_dfinal, float *dL_dinitial,
                          float *dL_dalpha, void *stream);

/* dL/dalpha in one call from the INITIAL muon state s0 (left unchanged): a
 * checkpointing forward on a private copy, then mt_adjoint_ckpt.  All scratch
 * (checkpoints and the state copy) comes from the stream-ordered allocator. */
mt_status mt_transport_adjoint(mt_handle *h, const mt_muon_soa *s0, int64_t n, float step_len, int32_t max_steps,
                               uint64_t seed, const float *alpha, int32_t n_block, const float *dL_dfinal,
                               float *dL_dalpha, int32_t ckpt_every, void *stream);

/* Full-tape form (no recompute).  The checkpointing forward above keeps a
 * state every K steps and the backward recomputes each K-step segment; with
 * the GPU's high-bandwidth memory large enough to hold every recorded step
 * (56 bytes per muon-step, e.g. 60 GB for 1e6 muons x ~1080 steps), the
 * forward can instead record the whole trajectory once and the backward only
 * walks it backwards.  Same gradients as mt_adjoint_ckpt (the same recorded
 * quantities, the same reverse arithmetic).  steps_per_pass (1..64) sets the
 * compaction interval of the forward. */

/* Bytes of a tape buffer for n muons (n < 2^31): enough for every muon to run
 * all max_steps steps (the tape actually used is 56 bytes x muon-steps taken).
 * -1 for bad arguments. */
int64_t mt_tape_bytes(int64_t n, int32_t max_steps, int32_t steps_per_pass);

/* Forward that records the tape: exactly mt_transport_scaled (same results),
 * with every step written into `tape` (device, 256-byte aligned, at least
 * mt_tape_bytes bytes, caller-owned, read by mt_adjoint_tape).  Errors as
 * mt_transport_ckpt.  A region that would overrun the buffer (only possible
 * with a buffer smaller than mt_tape_bytes, which is rejected) is not written
 * and makes mt_adjoint_tape return NaN gradients. */
mt_status mt_transport_tape(mt_handle *h, const mt_muon_soa *s, int64_t n, float step_len, int32_t max_steps,
                            uint64_t seed, const float *alpha, int32_t n_block, int32_t steps_per_pass, void *tape,
                            int64_t tape_bytes, void *stream);

/* Backward from the tape of one mt_transport_tape call (same n, step_len,
 * max_steps, alpha values, steps_per_pass).  dL_dfinal, dL_dinitial and
 * dL_dalpha as in mt_adjoint_ckpt; only the muons whose dL_dfinal is not all
 * zero are reversed.  Scratch (their list positions in one pass, 4n bytes,
 * plus 6n floats when dL_dinitial is NULL) comes from the stream-ordered
 * allocator. */
mt_status mt_adjoint_tape(mt_handle *h, int64_t n, float step_len, int32_t max_steps, const float *alpha,
                          int32_t n_block, int32_t steps_per_pass, void *tape, int64_t tape_bytes,
                          const float *dL_dfinal, float *dL_dinitial, float *dL_dalpha, void *stream);

/* Acceptance loss of final states: L = (1/n) sum over muons of
 * s((h - |x_e|)/e) s((h - |y_e|)/e), s the logistic function and (x_e, y_e)
 * the straight-line extrapolation of (x, y) to the plane z = z_plane; muons
 * that stopped or are invalid, or have pz <= 0, contribute 0.  *loss (device
 * double) is overwritten; dL_dfinal (device [6][n] floats, may be NULL)
 * receives dL/d(x, y, z, px, py, pz).  Reads x..pz and status of s only. */
mt_status mt_acceptance_loss(const mt_muon_soa *s, int64_t n, double z_plane, double half_width, double edge,
                             double *loss, float *dL_dfinal, void *stream);

/* ---------------------------------------------------------------------------
 * Offline phase (Sec. Building histograms, Appendix A) on the GPU, with a
 * parametric physics sampler standing in for the paper's Geant4 runs.  A
 * sample of the step of a muon of momentum p through step_len of a material:
 * a Moyal ionisation loss (PDG thin-absorber width and most probable loss with
 * the density effect), a radiative loss v ~ v^-2 on [1e-3, 1) added with
 * probability b rho x / <v>, and a Rayleigh space angle of the Highland width
 * theta0 (or, 1 % of samples, a single-scatter tail 2 theta0 / sqrt(u)); its
 * eight uniforms come from Philox4x32-10 with key = seed and counters
 * (s, h, 0x0FF1, 0|1) for sample s of stream h.  FP64 arithmetic.
 * ------------------------------------------------------------------------- */
typedef struct mt_material {
    double rho;        /* density [g/cm^3]                         */
    double z_over_a;   /* Z/A                                      */
    double I_mev;      /* mean excitation energy [MeV]             */
    double X0_cm;      /* radiation length [cm]                    */
    double b_rad;      /* radiative loss coefficient [cm^2/g]      */
} mt_material;

/* Histograms H[m][i] of n_samples samples each (stream h = m n_pbin + i),
 * p uniform in [edges[i], edges[i+1]) (host, n_pbin + 1 increasing edges),
 * f = dp/p binned on [0, f_max) into nf bins and theta on [0, theta_max) into
 * ntheta bins, theta_max[h] = 5 theta0(edges[i]) (written to the host array
 * theta_max [n_mat][n_pbin]); samples off the axes go to the edge cells.
 * weights: device [n_mat][n_pbin][nf][ntheta] doubles (counts), overwritten.
 * Ready for mt_hist_desc (copy weights to the host).  Asynchronous on stream;
 * theta_max is written before return.  Errors: MT_ERR_INVALID_ARG,
 * MT_ERR_OOM, MT_ERR_CUDA. */
mt_status mt_build_histograms(const mt_material *mats, int32_t n_mat, int32_t n_pbin, const double *edges,
                              int32_t nf, int32_t ntheta, double f_max, double step_len, int64_t n_samples,
                              uint64_t seed, double *weights, double *theta_max, void *stream);

/* Pilot estimator of Appendix A: phi[j] = (1/K) sum over K samples at momentum
 * probes[j] (stream j) of log(-dPz/P), -dPz/P = f + (1 - f) 2 sin^2(theta/2)
 * with f capped at 1.  probes, phi: host arrays of n_probe (<= 65535).
 * Synchronises stream. */
mt_status mt_pilot_phi(const mt_material *mat, const double *probes, int32_t n_probe, int64_t K, double step_len,
                       uint64_t seed, double *phi, void *stream);

/* Bounded-variation bin edges of Appendix A on an increasing probe grid: from
 * edge p_i the next edge is the largest probe p_j with |phi_k - phi_i| <= eps
 * for every probe i < k <= j (at least the next probe, the grid's
 * resolution); the first and last edges are the first and last probes.
 * Writes the edges to edges (host, max_edges) and returns their number, or -1
 * (bad arguments, or more than max_edges; mt_last_error says which). */
int32_t mt_bv_edges(const double *probes, const double *phi, int32_t n_probe, double eps, double *edges,
                    int32_t max_edges);

/* Largest n that mt_transport_noalloc accepts. */
#define MT_NOALLOC_MAX_MUONS 65536

/* mt_transport for callers that must not allocate device memory: a process
 * whose framework has already reserved the GPU's memory in its own pool, a
 * latency-critical path that cannot afford an allocation's synchronisation, or
 * a deployment whose memory use must be fixed when the library is loaded.  (The
 * paper has no counterpart: it describes no allocation policy.)
 * It runs the compacting transport (MT_LAUNCH_COMPACT, default pass length) with
 * its scratch list in an 8 MiB array that the library reserves in device
 * memory, held until the process exits; it calls no cudaMalloc, cudaFree or
 * other allocating routine.  CUDA creates a library's device objects and loads
 * its kernels lazily, and that takes device memory, so mt_create (which
 * allocates anyway) creates the array on its device and loads the kernels this
 * call launches for its world: no call of this entry point triggers either.
 *  - n may be at most MT_NOALLOC_MAX_MUONS; larger n returns MT_ERR_INVALID_ARG
 *    before anything is enqueued.  Other arguments and errors as mt_transport.
 *  - All calls on one device share that array and leave their contents in it;
 *    each call clears the counters it needs.  Calls that can overlap on the GPU
 *    (different streams, or different host threads without ordering) race on the
 *    array: order them, e.g. on one stream.
 *  - The array's device address is looked up once per device (thread-safe),
 *    by mt_create; should that have failed, the first call here retries it,
 *    so make the first call before any stream capture. */
mt_status mt_transport_noalloc(mt_handle *h, const mt_muon_soa *s, int64_t n, float step_len, int32_t max_steps,
                               uint64_t seed, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MT_H */
