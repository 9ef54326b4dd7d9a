/*
 * gbt.h -- C ABI of libgbt, GB300-native Gaussian beam summation.
 *
 * The library computes, on one GPU, the two processes of Gaussian beam
 * tracing named in Sec. 3.1 of arXiv 2501.13382: ray tracing (RT) of a fan
 * of rays with specular reflections off planar facets, and Gaussian beam
 * summation (GBS), the sum of every beam's contribution (Eq. 1, with the
 * beam parameters of Eq. 2) at every observation point (Eq. 3).
 *
 * Conventions shared by every entry point
 *  - Pointers marked "device" must point to memory of the current CUDA device;
 *    pointers marked "host" to ordinary host memory.  The caller owns every
 *    buffer it passes; the library owns only its opaque handles and the
 *    device memory inside them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Every call is stream-ordered and returns without waiting for the GPU,
 *    except where a call says it synchronises.
 *  - Every call returns a gbt_status.  Invalid arguments are rejected before
 *    any work is queued (GBT_ERR_INVALID_ARG) and nothing is written.  A
 *    failed CUDA call returns GBT_ERR_CUDA.  Problems a kernel detects (an
 *    index out of range, a bounded wait that ran out) set a device status
 *    word that gbt_sync reports.  gbt_last_error() describes the most recent
 *    failure on the calling thread.  No C++ exception crosses this ABI.
 *  - Complex numbers are interleaved float pairs (re, im) ("complex64").
 *  - Time convention exp(-i omega t): a beam's phase grows as exp(+i k s).
 */
#ifndef GBT_H
#define GBT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GBT_VERSION 2
#define GBT_MAX_FREQ 16          /* frequencies per sum call */

typedef enum gbt_status {
    GBT_OK = 0,
    GBT_ERR_INVALID_ARG = 1,     /* rejected before any launch */
    GBT_ERR_OOM = 2,             /* device allocation failed */
    GBT_ERR_CUDA = 3,            /* a CUDA runtime call failed */
    GBT_ERR_TIMEOUT = 4,         /* a bounded device wait ran out (via gbt_sync) */
    GBT_ERR_DEVICE_STATUS = 5,   /* a kernel flagged an internal error (via gbt_sync) */
    GBT_ERR_UNSUPPORTED = 6      /* valid request the library does not handle */
} gbt_status;

enum { GBT_WINDOW_SEGMENT = 0,   /* a beam acts on 0 <= s_loc < L of its segment */
       GBT_WINDOW_LINE = 1 };    /* a beam acts on its whole unfolded ray, s >= 0 */
enum { GBT_PRECISION_F32 = 0,    /* FP32 arithmetic, float-float phase, compensated sums */
       GBT_PRECISION_F64 = 1 };  /* FP64 everywhere (comparison path; slow on GB300) */
enum { GBT_FAN_FIBONACCI = 0,    /* directions generated on the device */
       GBT_FAN_EXPLICIT = 1,     /* directions supplied by the caller */
       GBT_FAN_LATLONG = 2 };    /* grid of polar x azimuth take-off angles, on the device */

typedef struct gbt_scene_s gbt_scene_t;   /* opaque handles */
typedef struct gbt_trace_s gbt_trace_t;
typedef struct gbt_batch_s gbt_batch_t;

/* ------------------------------------------------------------ allocator --
 * Optional allocator for the library's own device memory (handles and
 * scratch).  Without one the library uses cudaMallocAsync / cudaFreeAsync on
 * the call's stream.  `alloc` returns NULL on failure (-> GBT_ERR_OOM).  The
 * setting is process-wide and applies to allocations made after the call.
 * Passing NULL restores the default. */
typedef struct gbt_allocator {
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*free)(void *ptr, void *stream, void *ctx);
    void *ctx;
} gbt_allocator;

gbt_status gbt_set_allocator(const gbt_allocator *allocator);

/* --------------------------------------------------------------- scene --
 * Reflecting geometry for the RT process (Sec. 3.1: rays interact with
 * triangular facets; Sec. 4.1: an infinite rigid plate).  The optional ground
 * is the plane z = ground_z with normal +z (primitive id 0); triangles are
 * primitives 1..n_tri in the order given.  Triangles that share a facet id are
 * one planar facet: a ray leaving a facet cannot hit it again.  A reflection
 * off primitive p multiplies the beam by gamma[material(p)] (supplied at sum
 * time).  Host arrays are copied; the caller may free them on return.
 * Synchronises `stream` once (upload).
 *
 * Nearest-hit search (`accel`; every choice finds the same hits, bit for bit):
 *   GBT_ACCEL_AUTO    the BVH below (the faster search on every scene measured,
 *                     from 768 triangles up);
 *   GBT_ACCEL_BVH     a bounding-volume hierarchy built on the host at creation
 *                     (binned surface-area heuristic over triangle centroids,
 *                     leaves of at most 4 triangles, each node holding its two
 *                     children's padded FP32 boxes), traversed near child first
 *                     with a per-ray stack;
 *   GBT_ACCEL_LINEAR  padded FP32 boxes of clusters of 8 triangles and of each
 *                     triangle tested in index order: the whole scene resident
 *                     in shared memory up to 1,024 triangles, staged through it
 *                     in chunks of 1,024 above. */
typedef struct gbt_scene_desc {
    double c;                     /* speed of sound, m/s (> 0) */
    int32_t ground_enabled;       /* 0 / 1 */
    int32_t ground_material;      /* material index of the ground */
    double ground_z;              /* ground height, m */
    int64_t n_tri;                /* >= 0 */
    const double *tri_xyz;        /* host, n_tri * 9: v0, v1, v2 (x, y, z each) */
    const int32_t *tri_material;  /* host, n_tri, each in [0, n_materials) */
    const int32_t *tri_face;      /* host, n_tri facet ids >= 0, or NULL (own facet each) */
    int32_t n_materials;          /* >= 1 */
    int32_t accel;                /* GBT_ACCEL_AUTO (0), GBT_ACCEL_BVH, GBT_ACCEL_LINEAR */
} gbt_scene_desc;

enum { GBT_ACCEL_AUTO = 0, GBT_ACCEL_BVH = 1, GBT_ACCEL_LINEAR = 2 };

gbt_status gbt_scene_create(const gbt_scene_desc *desc, void *stream, gbt_scene_t **out);
/* Waits for the device (every stream), then frees the scene; its traces must be
 * destroyed first.  NULL is a no-op. */
gbt_status gbt_scene_destroy(gbt_scene_t *scene);

/* --------------------------------------------------------------- trace --
 * RT process (Sec. 2, Sec. 3.1; Sec. 3.3 for the fan of take-off directions).
 * Traces rays [ray_begin, ray_begin + ray_count) of a fan of n_rays rays from
 * `pos` in a homogeneous medium: nearest hit with t > 1e-9 m (ties: lowest
 * primitive id), specular reflection d' = d - 2 (d.n) n, until the path
 * length reaches max_path (the last segment is cut there) or the first hit
 * after max_reflections reflections.  The Fibonacci fan is
 * z_i = 1 - (2i+1)/N, phi_i = i pi (3 - sqrt 5); every ray carries the
 * solid-angle weight 4 pi / N unless the sum supplies per-ray weights.
 * The latitude-longitude fan is the paper's grid of take-off angles (Sec. 3.3;
 * its input tables give the elevation range 0..180 and the azimuth range
 * 0..360 degrees): n_theta rows of n_phi = N / n_theta rays, ray
 * g = it * n_phi + ip at the centre of its cell,
 *   theta = theta_deg[0] + (it + 1/2) dtheta   (polar angle from +z),
 *   phi   = phi_deg[0]   + (ip + 1/2) dphi,
 *   d = (sin theta cos phi, sin theta sin phi, cos theta),
 * carrying its cell's solid angle dphi (cos theta_lo - cos theta_hi) as weight
 * (explicit fans carry 4 pi / N).
 * FP64 throughout, without fused multiply-add, in a fixed operation order.
 *
 * The result is a CSR list of straight segments in ray order (ray_off over
 * the traced rays); per segment: origin, unit direction, length L, arclength
 * s0 at its start, global ray index, depth in its ray, the material of the
 * reflection that starts it (-1 for the first) and the primitive that ends it
 * (-1 if none).  Asynchronous: the segment count stays on the device until
 * gbt_trace_info is called.  `scene` must outlive the trace. */
typedef struct gbt_source_desc {
    double pos[3];                /* source position, m */
    int64_t n_rays;               /* fan size N (>= 1) */
    int64_t ray_begin;            /* first ray traced (chunking), 0 normally */
    int64_t ray_count;            /* rays traced; 0 = n_rays - ray_begin */
    int32_t fan;                  /* GBT_FAN_FIBONACCI, GBT_FAN_EXPLICIT or GBT_FAN_LATLONG */
    int32_t max_reflections;      /* >= 0 */
    const double *dirs;           /* device, ray_count * 3 unit vectors (EXPLICIT only) */
    double max_path;              /* m (> 0) */
    /* GBT_FAN_LATLONG only: n_rays = n_theta * n_phi */
    int64_t n_theta;              /* polar rows (>= 1, divides n_rays) */
    double theta_deg[2];          /* polar range, 0 <= [0] < [1] <= 180 */
    double phi_deg[2];            /* azimuth range, [0] < [1] <= [0] + 360 */
} gbt_source_desc;

gbt_status gbt_trace(const gbt_scene_t *scene, const gbt_source_desc *src, void *stream,
                     gbt_trace_t **out);

typedef struct gbt_trace_info {
    int64_t n_fan;                /* fan size N */
    int64_t ray_begin, n_rays;    /* traced ray range */
    int64_t seg_capacity;         /* n_rays * (max_reflections + 1) */
    int64_t n_segments;           /* exact count (this call synchronises the trace's stream) */
    /* read-only device views, valid until gbt_trace_destroy */
    const int32_t *ray_off;       /* n_rays + 1 */
    const double *seg_o;          /* n_segments * 3 */
    const double *seg_t;          /* n_segments * 3 */
    const double *seg_L;          /* n_segments */
    const double *seg_s0;         /* n_segments */
    const int32_t *seg_ray;       /* n_segments, global ray index */
    const int32_t *seg_depth;     /* n_segments */
    const int32_t *seg_bmat;      /* n_segments */
    const int32_t *seg_hit;       /* n_segments */
} gbt_trace_info;

gbt_status gbt_trace_info_get(const gbt_trace_t *trace, gbt_trace_info *info);
/* Waits for the device (every stream), then frees the trace and its workspace.
 * NULL is a no-op. */
gbt_status gbt_trace_destroy(gbt_trace_t *trace);

/* Segment list of a trace computed elsewhere (a saved trace, another tracer), in
 * the layout gbt_trace_info exposes.  Device arrays; they are copied, so the
 * caller may free them when gbt_trace_import returns. */
typedef struct gbt_segments {
    int64_t n_segments;           /* >= 0 */
    const int32_t *ray_off;       /* n_rays + 1 offsets: ray_off[0] = 0, non-decreasing, at
                                     most max_reflections + 1 segments per ray,
                                     ray_off[n_rays] = n_segments */
    const double *seg_o;          /* n_segments * 3, segment origins, m */
    const double *seg_t;          /* n_segments * 3, unit directions */
    const double *seg_L;          /* n_segments, lengths, m */
    const double *seg_s0;         /* n_segments, unfolded arclength at the segment start, m */
    const int32_t *seg_bmat;      /* n_segments, material of the reflection that starts the
                                     segment (-1 for a ray's first); out-of-range materials
                                     are flagged by the sums' status word */
    const int32_t *seg_hit;       /* n_segments end primitives, or NULL (-1 each) */
} gbt_segments;

/* Trace handle over such a segment list, for the sums and the adjoint as if
 * gbt_trace had produced it: `src` as for gbt_trace (fan size and kind, which set
 * the default ray weights, traced ray range, max_reflections); segment j of ray
 * i gets ray index ray_begin + i and depth j - ray_off[i].  The offsets are
 * checked on the host (one synchronisation of `stream`); GBT_ERR_INVALID_ARG if
 * they do not describe such a list. */
gbt_status gbt_trace_import(const gbt_scene_t *scene, const gbt_source_desc *src,
                            const gbt_segments *segs, void *stream, gbt_trace_t **out);

/* ----------------------------------------------------------------- sum --
 * GBS process (Eq. 3): for every receiver x, frequency f and segment j with
 *   s_loc = (x - o_j).t_j,  s = s0_j + s_loc,  n^2 = |(x - o_j) x t_j|^2,
 *   E = s - i b_f,  k = 2 pi f / c,
 * the beam of Eq. 1 (P = I/c and Q(s) = Q0 + c P s from Eq. 2, isotropic,
 * Q0 = -i b_f I) contributes
 *   W_ray * Gamma_path_j * (k b_f / (8 pi^2)) * exp(i k s + i k n^2 / (2E)) / E
 * when k n^2 b_f / (2 (s^2 + b_f^2)) <= cutoff and the pair lies in the
 * window (SEGMENT: 0 <= s_loc < L_j; LINE: s >= 0).  Gamma_path_j is the
 * product of gamma over the reflections before segment j.  The constant
 * k b / (8 pi^2) makes a dense fan sum to the point source exp(ikr)/(4 pi r).
 *
 * F32 precision: FP32 arithmetic with float-float arclength and phase
 * reduction, FP32 MUFU exp/sin/cos, compensated per-receiver accumulation;
 * relative L2 error against an FP64 evaluation measured at 1e-7..4e-7 on the
 * synthetic open-plane and city workloads (tested to 1e-6 with 4 kHz phases
 * over 1 km paths).  Where a receiver group is compact for the call's highest
 * frequency (K max|x'| <= 90 turns), the receivers' projection on a segment is
 * formed in FP32 (a term's phase moves by at most about 1e-4 rad); a pair within
 * that projection's error bound of an end of its window is decided and evaluated
 * in float-float, so the window decisions are those of the exact arithmetic.  F64 precision: every step in FP64 (2.6e-8, the rounding of
 * the complex64 output), at FP64 speed.
 * With more than 8 frequencies the F32 path runs one pair launch per group of
 * at most 8 (frequencies sorted by value when every b_f is equal, otherwise in
 * the given order); each group costs a full pass over the pairs.
 * `out` (n_freq * n_recv complex64, frequency-major) is overwritten, or added
 * to when `accumulate` is 1.  Scratch comes from the trace's workspace, so
 * calls on one trace must not overlap on different streams.
 *
 * Propagation losses (optional).  The paper's input tables (Sec. 4.5, Tables
 * 2-3) give the air temperature, humidity and pressure and a flow-impedance
 * setting of the surfaces, with no formulas; the library takes standard ones:
 *  - absorption of air: every beam is scaled by exp(-a_f s) over its unfolded
 *    arclength s, with a_f = absorption[f] (Np/m, the pressure-amplitude decay
 *    rate; gbt_air_absorption gives the ISO 9613-1 value);
 *  - porous surfaces: a material m with flow_resistivity[m] = sigma > 0
 *    (kPa s m^-2) reflects with gamma_m times the plane-wave reflection factor
 *    R = (Z cos(theta) - 1) / (Z cos(theta) + 1) of a locally reacting surface
 *    at the reflection's angle of incidence theta, Z / (rho c) = 1 +
 *    9.08 (f / sigma)^-0.75 + i 11.9 (f / sigma)^-0.73 (Delany and Bazley,
 *    exp(-i omega t)); sigma <= 0 (the paper's negative setting) or a NULL array
 *    is a hard surface, whose reflection is gamma_m alone.
 * The losses change no cull decision (the cutoff tests the Gaussian alone).
 * Batches with losses run in the CONCURRENT form; the FUSED form rejects them
 * (GBT_ERR_UNSUPPORTED). */
typedef struct gbt_sum_args {
    const float *recv;            /* device, n_recv * 3 (x, y, z), m */
    int64_t n_recv;               /* >= 0 */
    const int32_t *recv_order;    /* device permutation of [0, n_recv) or NULL; receivers
                                     are processed in this order (see gbt_recv_order) */
    int32_t n_freq;               /* 1 .. GBT_MAX_FREQ */
    int32_t window;               /* GBT_WINDOW_SEGMENT / GBT_WINDOW_LINE */
    double freq_hz[GBT_MAX_FREQ]; /* > 0 */
    double beam_b[GBT_MAX_FREQ];  /* beam parameter b_f, m (> 0) */
    const float *gamma;           /* device, n_materials reflection coefficients */
    const float *ray_weight;      /* device, n_fan per-ray weights, or NULL (the fan's own:
                                     4 pi / N, or the lat-long cell solid angles) */
    float *out;                   /* device, n_freq * n_recv * 2 floats */
    double cutoff;                /* C (> 0); 16 drops less than 1.2e-7 of a beam */
    int32_t precision;            /* GBT_PRECISION_F32 / GBT_PRECISION_F64 */
    int32_t accumulate;           /* 0 overwrite, 1 add into out */
    int32_t seg_split;            /* segment ranges per receiver tile; 0 = automatic */
    int32_t tile_cull;            /* 1: skip, per warp of 64 receivers, segments whose beams
                                     provably reach none of them (same result, less work);
                                     0: test every pair */
    int64_t max_device_bytes;     /* gbt_solve only: device budget for one chunk; 0 = auto */
    double absorption[GBT_MAX_FREQ]; /* air's amplitude decay rate per frequency, Np/m
                                     (>= 0; all 0 = lossless air) */
    const float *flow_resistivity; /* device, n_materials effective flow resistivities,
                                     kPa s m^-2 (<= 0: hard), or NULL: every surface hard */
} gbt_sum_args;

gbt_status gbt_sum(const gbt_trace_t *trace, const gbt_sum_args *args, void *stream);

/* Spatially coherent processing order of receivers (Morton order of their
 * positions quantised to their bounding box), written to order_out (device,
 * n_recv int32).  The order changes results only by rounding: each warp of 64
 * receivers forms its exact geometry relative to its first receiver, so
 * compact warps (neighbouring receivers) are both faster (they see similar
 * beams, which keeps the warp's lanes busy) and the most accurate; a given
 * order always gives the same result. */
gbt_status gbt_recv_order(const float *recv, int64_t n_recv, int32_t *order_out, void *stream);

/* Same result as gbt_recv_order (the identical permutation), for callers that
 * cannot allocate device memory when they need it: hosts that own every
 * device allocation and forbid libraries from calling the CUDA allocator, or
 * latency-critical loops that must not allocate because an allocation may
 * block or fail.  The paper has no counterpart; this is a library service.
 * Allocates nothing: the sort's scratch is a fixed 8 MiB device array inside
 * the library, held by every GPU that loads it until the process exits.
 * n_recv must be <= 1,048,576 (GBT_ERR_INVALID_ARG otherwise, before any
 * work).  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process, which
 * assumes the device's primary context is not reset (after cudaDeviceReset the
 * address is stale: do not call this entry point again in that process); make
 * that first call before any stream capture.
 * All calls share the array and every call clears what it needs, but calls
 * that overlap on the GPU race on it: order them on one stream (or wait
 * between them).  recv and order_out are device pointers owned by the caller. */
gbt_status gbt_recv_order_noalloc(const float *recv, int64_t n_recv, int32_t *order_out,
                                  void *stream);

/* Amplitude decay rate of air (Np/m) for pure tones at freq_hz[0 .. n) in an
 * atmosphere at temperature_c (degrees C), relative humidity humidity_pct (%)
 * and pressure pressure_kpa (kPa): the attenuation coefficient of ISO 9613-1
 * (classical and rotational absorption plus the vibrational relaxation of
 * oxygen and nitrogen) divided by 20 log10(e) dB per neper.  The paper's cases
 * use 20 C, 70 % and 1 atm (Tables 2-3).  Host arrays; no GPU work.
 * GBT_ERR_INVALID_ARG for n < 0, NULL arrays, non-positive frequencies or
 * pressure, humidity outside [0, 100] or temperature outside [-50, 60] C. */
gbt_status gbt_air_absorption(int32_t n, const double *freq_hz, double temperature_c,
                              double humidity_pct, double pressure_kpa, double *np_per_m);

/* ------------------------------------------------------------ backward --
 * Adjoint of gbt_sum for a real loss L.  grad_out (device, n_freq * n_recv
 * complex64) holds g = dL/dRe p + i dL/dIm p.  Writes (overwrites)
 *   grad_gamma[m]      = dL/dgamma_m        (device, n_materials floats)
 *   grad_ray_weight[i] = dL/dW_i            (device, n_fan floats; NULL to skip)
 *   grad_b[f]          = dL/db_f            (device, n_freq doubles; NULL to skip)
 * using dL/dtheta = sum Re(conj(g) dp/dtheta).  The cull mask and window are
 * held fixed (the summand is differentiated where it is kept).  Contributions
 * are recomputed, never stored per (receiver, segment).  F32 only.  With
 * losses the contributions carry them; the losses depend on none of the
 * differentiated parameters. */
gbt_status gbt_sum_backward(const gbt_trace_t *trace, const gbt_sum_args *args,
                            const float *grad_out, float *grad_gamma, float *grad_ray_weight,
                            double *grad_b, void *stream);

/* --------------------------------------------------------------- solve --
 * RT + GBS for one source with the ray range split into chunks so that one
 * chunk's trace fits args->max_device_bytes (the paper's chunking when rays
 * exceed device memory, Sec. 4.5.1).  Chunks are summed in ray order and
 * accumulated into args->out; with more than one chunk, chunk i + 1 is traced
 * on a private stream while chunk i is summed on `stream` (two trace slots,
 * ordered by events; the call returns without waiting).  The result equals one
 * unchunked trace + sum up to rounding.  src->ray_begin / ray_count must be 0. */
gbt_status gbt_solve(const gbt_scene_t *scene, const gbt_source_desc *src,
                     const gbt_sum_args *args, void *stream);

/* --------------------------------------------------------------- batch --
 * Many GBS instances (sources x frequency sets, uneven segment counts) run as
 * one unit, captured in a CUDA graph on the first submit and replayed
 * afterwards.  Each instance is a trace plus sum arguments; the result of each
 * instance equals gbt_sum on it up to rounding.  Two execution forms:
 *   FUSED       one persistent launch fed by a device work queue of
 *               (instance, receiver tile, segment range) items, instances
 *               longest first (the load-imbalance remedy of Sec. 3.4 taken to
 *               the whole batch);
 *   CONCURRENT  each instance's single-sum kernels on one of a few branch
 *               streams forked from the submit stream and joined back, so one
 *               instance's draining tail overlaps the next instance's start.
 * AUTO takes the faster of the two measured at create when autotune is set,
 * else CONCURRENT.  All traces and buffers must stay alive and unchanged in
 * shape while the batch exists; their contents may change between submits. */
enum { GBT_BATCH_AUTO = 0, GBT_BATCH_FUSED = 1, GBT_BATCH_CONCURRENT = 2 };

typedef struct gbt_batch_desc {
    int32_t n_instances;              /* >= 1 */
    const gbt_trace_t *const *traces; /* host array of n_instances handles */
    const gbt_sum_args *args;         /* host array of n_instances argument sets; all F32,
                                         one window; an instance with more than 8
                                         frequencies runs as one instance per group of 8
                                         consecutive ones, each writing its rows of out */
    int32_t use_graph;                /* 1: capture on first submit, then replay */
    int32_t autotune;                 /* 1: time the candidate forms / work splittings at
                                         create (running the batch a few times), keep the best */
    int32_t form;                     /* GBT_BATCH_AUTO, _FUSED or _CONCURRENT */
} gbt_batch_desc;

/* Create synchronises `stream` once (it reads each trace's segment count to
 * order the instances longest first and to size their work) and allocates
 * the batch's device workspace; with autotune it also runs the batch a few
 * times.  Submit queues the whole batch on `stream` (graph replay after the
 * first submit when use_graph is set); outputs land in each instance's out.
 * GBT_ERR_INVALID_ARG for an unknown form. */
gbt_status gbt_batch_create(const gbt_batch_desc *desc, void *stream, gbt_batch_t **out);
gbt_status gbt_batch_submit(gbt_batch_t *batch, void *stream);
gbt_status gbt_batch_destroy(gbt_batch_t *batch);

/* ------------------------------------------------------------ synthesis --
 * Time signals from per-frequency fields: the superposition of the
 * time-harmonic fields of Eq. 1 under the exp(-i omega t) convention.  For
 * receiver r and t_n = t0 + n dt,
 *   h[n, r] = Re sum_f A_f p[f, r] exp(-i 2 pi freq_f t_n),
 * with complex amplitudes A_f (A_f = S(freq_f) df synthesises a source
 * spectrum S).  p: device, n_freq * n_recv complex64, frequency-major (the
 * layout of gbt_sum's out); freq_hz: host, n_freq values; amp: host, n_freq
 * complex amplitudes as (re, im) doubles; out: device, n_t * n_recv float32,
 * time-major, overwritten, or added to when accumulate is 1 (more than
 * GBT_MAX_FREQ frequencies: several accumulating calls).  The phasors
 * A_f exp(-i 2 pi freq_f t_n) are formed on the device (the phase in turns
 * reduced to [0, 1) in FP64, then FP32 sine and cosine of the reduced turn),
 * the sums in FP32.  n_freq 1 .. GBT_MAX_FREQ, n_t 1 .. 2^20, n_recv >= 0.
 * Asynchronous: one kernel launch, no scratch, nothing waits for the GPU (the
 * host arrays are read before the call returns). */
gbt_status gbt_synthesize(const float *p, int32_t n_freq, int64_t n_recv, const double *freq_hz,
                          const double *amp, double t0, double dt, int64_t n_t, float *out,
                          int32_t accumulate, void *stream);

/* Bound on the device memory of the tile pre-cull's segment lists: at most `entries`
 * list entries (4 bytes each, plus 2 bytes of warp-tile words) per sum, for the sums
 * planned after this call; 0 restores the default (an eighth of all (tile, segment)
 * pairs, at least 16M entries).  Tiles are laid out lightest first; a tile whose list
 * does not fit tests every segment instead, which gives the same field up to FP32
 * rounding of the regrouped partial sums (the kept terms do not depend on it).
 * Process-wide, no GPU work; GBT_ERR_INVALID_ARG for entries < 0. */
gbt_status gbt_list_capacity_set(int64_t entries);

/* ---------------------------------------------------------- measurement --
 * Kernel timing: while enabled, each launch of the GBS pair kernel (forward
 * or backward) is bracketed by CUDA events recorded on its launch stream.
 * gbt_timing_read waits for the recorded events and returns the number of
 * launches and their summed device time since the last reset. */
gbt_status gbt_timing_enable(int32_t enable);
gbt_status gbt_timing_read(int64_t *launches, double *total_ms, int32_t reset);

/* Kernel launch count: every kernel the library puts on a stream (tracer,
 * scan, compaction, prepass, tile order, pair kernel, merge, receiver order,
 * adjoint kernels) adds one, counted on the host at launch time in all threads;
 * reset != 0 zeroes the count after reading it.  A graph replay of a batch
 * counts the kernels of the captured graph once per submit.  No GPU work. */
gbt_status gbt_launches_read(int64_t *launches, int32_t reset);

/* Work statistics of one gbt_sum call (same arguments): number of
 * (receiver, segment) pairs, pairs kept by the frequency-union prefilter, and
 * (receiver, segment, frequency) triples whose beam contributes (window and
 * cutoff met).  Runs a counting variant of the F32 kernel; synchronises.
 * With more than 8 frequencies, pairs_prefiltered and pairs_tested add up the
 * counts of each group of at most 8 frequencies (see gbt_sum). */
typedef struct gbt_sum_stats {
    int64_t n_segments;
    int64_t pairs;
    int64_t pairs_prefiltered;
    int64_t triples_kept;
    int64_t pairs_tested;         /* pairs that reached the per-pair test (all, unless tile_cull) */
} gbt_sum_stats;

gbt_status gbt_sum_stats_get(const gbt_trace_t *trace, const gbt_sum_args *args,
                             gbt_sum_stats *stats, void *stream);

/* ---------------------------------------------------------------- misc -- */

/* Waits for `stream`, then reads and clears the device status word: returns
 * GBT_ERR_TIMEOUT or GBT_ERR_DEVICE_STATUS if a kernel flagged a problem.  The
 * status word is one per device, shared by every stream: it reports flags raised
 * by any of the library's kernels on the current device that finished before the
 * read, including those of the library's private streams (a chunked solve's trace
 * stream, a batch's branch streams), and clearing it clears them for every caller.
 * To cover work still running on other streams, synchronise those streams (or the
 * device) first. */
gbt_status gbt_sync(void *stream);

/* Self test of the failure path for device waits (no counterpart in the paper):
 * launches one thread that waits on a shared-memory barrier phase that nothing
 * completes, with the same bounded try-wait loop the pair kernel uses, for at
 * most `spins` tries (1 .. 2^24).  The wait runs out, the kernel flags a
 * timeout and returns; the following gbt_sync returns GBT_ERR_TIMEOUT and
 * clears the flag, and the context stays usable. */
gbt_status gbt_selftest_timeout(int64_t spins, void *stream);

/* Description of the last failure on the calling thread ("" if none). */
const char *gbt_last_error(void);

int32_t gbt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GBT_H */
