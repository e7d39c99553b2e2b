/*
 * sand.h — C-ABI of libsand: the SAND query path on one GB300 (sm_103a).
 *
 * SAND (arxiv 2604.25936) answers a signed-distance query at a 3D point x by
 * reading the exit layer d(x) of x from a volumetric network-depth map (an
 * octree, Sec. 3.2, Eq. 7) and evaluating a tailed MLP only up to that layer
 * (Sec. 3.4): y_d = t_1 + ... + t_d with t_i the tail of hidden layer i
 * (Eq. 2; multiplicative tails for i >= 2 follow Eq. 3).  Exit layer 0 marks
 * a far leaf whose stored SDF value at the leaf centre is returned without
 * running the network (Eq. 7).
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are device pointers on the model's device; h_* are
 *     host pointers.  The caller owns every buffer it passes; the library
 *     owns the model (weights, depth map) and its optional default workspace.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Queries are stream-ordered and asynchronous: they return once
 *     the work is enqueued.  Loaders and sand_free synchronise the device.
 *   - Every call returns a sand_status; on failure sand_last_error() gives a
 *     message (thread-local, valid until the next call on the same thread).
 *   - Points are float32 xyz triples, array-of-structures [n][3], at least
 *     4-byte aligned (16-byte alignment enables vector loads).  The domain is
 *     [-1,1]^3; points outside are answered by the nearest boundary leaf.  A
 *     point with a NaN coordinate gets exit layer 0xFF, SDF NaN, gradient NaN,
 *     and sets SAND_FLAG_NAN_INPUT in the workspace flags (sand_query_stats).
 *   - n == 0 is a valid no-op.
 *   - A model is not safe to call from several host threads at once: its default
 *     workspace, the staging buffer and copy streams of host queries and its
 *     packed tensor-core weights are shared by every call on it.  Callers that
 *     share a model across threads serialise their calls, or submit through a
 *     server (sand_server_*), which takes requests from any thread.
 */
#ifndef SAND_H_
#define SAND_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sand_model_s *sand_model;

typedef enum {
    SAND_OK = 0,
    SAND_EINVAL = 1,        /* an argument is out of range or a pointer is NULL / misaligned */
    SAND_ENOMEM = 2,        /* a device or host allocation failed, or the workspace is too small */
    SAND_EFORMAT = 3,       /* a model / depth-map file or descriptor is malformed */
    SAND_ECUDA = 4,         /* a CUDA runtime call failed (message carries cudaGetErrorString) */
    SAND_ETIMEOUT = 5,      /* a bounded device-side wait gave up (see SAND_FLAG_TIMEOUT) */
    SAND_ENOMAP = 6,        /* a SAND query before a depth map was loaded */
    SAND_EUNSUPPORTED = 7   /* this model shape / precision / device is not supported */
} sand_status;

/* Arithmetic of the hidden-layer products W_i h_{i-1} (Eq. 2).  The first
 * layer, the sine argument and its range reduction, the tails and the
 * accumulation y_i = y_{i-1} + t_i are always float32.  In a SAND query without
 * gradients of a model on raw coordinates, points whose exit layer is 1 are
 * computed entirely in float32 on the CUDA cores whatever the mode, every such
 * point the same way; no point's result depends on the other points of a call.
 *   SAND_FP32       tcgen05 tensor cores, each float32 operand split into two
 *                   fp16 terms (weights pre-scaled by a power of two), three
 *                   products per layer, float32 accumulation: float32-class error.
 *   SAND_FP32_SIMT  plain float32 FMA on the CUDA cores (reference kernel).
 *   SAND_FP16 / SAND_BF16 / SAND_FP8  one tcgen05 product per layer with
 *                   fp16 / bf16 / e4m3 operands (per-layer weight scales) and
 *                   float32 accumulation. */
typedef enum {
    SAND_FP32 = 0,
    SAND_FP32_SIMT = 1,
    SAND_FP16 = 2,
    SAND_BF16 = 3,
    SAND_FP8 = 4
} sand_precision;

typedef enum { SAND_TAIL_LINEAR = 0, SAND_TAIL_MULT = 1 } sand_tail_kind;
typedef enum { SAND_ACT_SINE = 0, SAND_ACT_RELU = 1, SAND_ACT_FINER = 2 } sand_activation;
typedef enum { SAND_ENC_NONE = 0, SAND_ENC_FOURIER = 1 } sand_encoder;

/* Shape of a T-MLP (Eq. 2 / Eq. 3).
 *   n_layers  L, the number of hidden layers and of tails (1 .. 14)
 *   width     W, hidden units per layer (16 .. 512)
 *   in_dim    3 without an encoder, 2 * n_freq with Fourier features
 *   activation SAND_ACT_SINE: h = sin(omega0 * (W h + b)) (SIREN);
 *             SAND_ACT_RELU: h = max(0, W h + b);
 *             SAND_ACT_FINER: h = sin(omega0 * (|z| + 1) * z), z = W h + b, the
 *             variable-periodic sine of the FINER backbone (Sec. 2 cites it, the
 *             SAND-FINER rows of Table 1 use it; the formula is FINER's own)
 *   encoder   SAND_ENC_FOURIER: h_0 = [sin(2 pi B x), cos(2 pi B x)], B [n_freq][3]
 *   tail_kind SAND_TAIL_MULT: t_i = (a_i.h_i + c_i)(b_i.h_i + e_i) for i >= 2 (Eq. 3);
 *             tail 1 is always affine.                                          */
typedef struct {
    int32_t n_layers;
    int32_t width;
    int32_t in_dim;
    int32_t tail_kind;
    int32_t activation;
    int32_t encoder;
    int32_t n_freq;
    float omega0;
} sand_tmlp_desc;

/* Pointer octree over [-1,1]^3 (Sec. 3.2): node 0 is the root; child[i] = -1
 * marks a leaf, else the index of the first of its 8 consecutive children in
 * octant order ix | iy << 1 | iz << 2, where the upper half (coordinate >= the
 * cell midpoint) has bit 1.  depth[i] is a leaf's exit layer (0 .. n_layers;
 * 0 = far leaf), far[i] its stored SDF value at the centre (Eq. 7). */
typedef struct {
    int32_t max_level;   /* deepest leaf level, 0 .. 10 (root = level 0) */
    int32_t n_layers;    /* largest exit layer the map may hold */
    int32_t n_nodes;
} sand_depth_map_desc;

/* Per-query options; a NULL opts pointer means all defaults (zero-initialised). */
typedef struct {
    int32_t precision;      /* sand_precision (default SAND_FP32) */
    int32_t max_depth;      /* level of detail (Sec. 3.4): exit layer <- min(d, max_depth) for d > 0; 0 = off */
    int32_t full_depth;     /* 1: ignore the depth map and run every point to layer L (plain T-MLP) */
    int32_t all_tails;      /* with full_depth on a tensor-core precision: d_out is [n][L], the cumulative
                               outputs y_1 .. y_L of every point (every level of detail at once);
                               not with gradients */
    uint8_t *d_exit_layers; /* optional device [n]: exit layer used per point (0xFF = NaN point) */
    void *d_workspace;      /* optional device scratch of >= sand_workspace_bytes() bytes, 256-byte aligned;
                               NULL = the model's own workspace (grown on demand; one stream at a time) */
    size_t workspace_bytes;
    void *const *stage_events; /* optional: 3 caller-created cudaEvent_t handles, recorded on the stream
                               before the lookup, before the T-MLP kernel and after it (stage timing) */
    uint32_t wait_limit_us; /* limit of every bounded wait inside the tensor-core kernel, in microseconds
                               (0 = 2 s).  A wait that runs out makes the kernel stop issuing work, finish
                               what is in flight, free its tensor memory and return; the query's results
                               are then undefined and sand_read_stats reports SAND_ETIMEOUT.  Only the
                               plain, gradient and all-tails queries take it (dynamic exit and sphere
                               tracing: SAND_EINVAL) */
    int32_t reserved;
} sand_query_opts;

/* Load a model file: "TMLP", u32 version 1, 7 x i32 (n_layers, width, in_dim,
 * tail_kind, activation, encoder, n_freq), f32 omega0, u64 n_params, then the
 * float32 parameter block (layout of sand_load_tmlp_mem).  `device` is the CUDA
 * ordinal the model lives on.  On success *out owns device memory until sand_free. */
sand_status sand_load_tmlp(const char *path, int device, sand_model *out);

/* Load a model from host memory.  h_params holds n_params float32 values in
 * this order (row-major): B [n_freq][3] (Fourier encoder only), W1 [W][in_dim],
 * b1 [W], W_2..W_L [L-1][W][W] (row = output unit), b_2..b_L [L-1][W],
 * tail weights [L][2][W] (row 1 used only by multiplicative tails i >= 2),
 * tail biases [L][2].  The library copies what it needs. */
sand_status sand_load_tmlp_mem(const sand_tmlp_desc *desc, const float *h_params, size_t n_params,
                               int device, sand_model *out);

/* Load the depth map from a file: "SDMO", u32 version 1, i32 max_level,
 * i32 n_layers, i32 n_nodes, 6 x f32 bounding box (must be -1,-1,-1,1,1,1),
 * int32 child[n], uint8 depth[n] padded to 4 bytes, float32 far[n].
 * Replaces any previous map. */
sand_status sand_load_depth_map(sand_model m, const char *path);

/* Load the depth map from host arrays (see sand_depth_map_desc).  The octree is
 * re-encoded losslessly on the device at its finest level: up to level 7 as a
 * dense exit-layer grid (2 MiB at level 7) plus a dense far-value grid when the
 * map has far leaves; deeper maps (levels 8 .. 10) as a table over the cells of
 * level max_level - 3 whose entries either hold a leaf's exit layer and far
 * value or point to a brick of 8^3 finest cells (exit layers, and far values
 * only for bricks holding far leaves).  SAND_EUNSUPPORTED above level 10. */
sand_status sand_load_depth_map_mem(sand_model m, const sand_depth_map_desc *desc, const int32_t *h_child,
                                    const uint8_t *h_depth, const float *h_far);

/* Device bytes of workspace a query of n points needs (with_grad: for sand_query_sdf_grad). */
size_t sand_workspace_bytes(sand_model m, int64_t n, int with_grad);

/* SAND inference (Sec. 3.4): d_out[i] = y_{d(x_i)}(x_i), or the stored far value
 * when d(x_i) = 0.  d_points: device float32 [n][3]; d_out: device float32 [n]. */
sand_status sand_query_sdf(sand_model m, const float *d_points, int64_t n, float *d_out,
                           const sand_query_opts *opts, void *stream);

/* As sand_query_sdf, plus the input gradient d_grad[i] = dy/dx at x_i (surface
 * normal direction for sphere tracing); zero for exit layer 0, NaN for points
 * outside the domain.  d_out may be NULL in full-depth mode only (a SAND query
 * writes the stored far values there: SAND_EINVAL).  d_grad: device float32
 * [n][3].  Every precision takes gradients: the tensor-core modes carry three
 * tangent rows per point through the same MMAs as the value row (forward mode),
 * SAND_FP32_SIMT runs the CUDA-core kernel; SAND_FP8 tangents are e4m3-rounded
 * like the activations. */
sand_status sand_query_sdf_grad(sand_model m, const float *d_points, int64_t n, float *d_out, float *d_grad,
                                const sand_query_opts *opts, void *stream);

/* End-to-end query from HOST memory: copies h_points to the device, runs the
 * query, copies the SDF back to h_out.  From 2^20 points on the work goes in up
 * to four chunks as a pipeline.  The points are cut into blocks of 2^18; of every
 * ten blocks chunk 0 takes one, chunks 1 and 2 four each and chunk 3 one (small
 * first and last chunks, each chunk sampling the whole input).  A chunk is copied
 * up on a copy stream of the model's own, its query runs on `stream` once it has
 * arrived, and its values are copied down on a second copy stream once it is
 * done, so the copies of one chunk overlap the queries of the others.  Each chunk is a query of its own points, which leaves every point's
 * result unchanged (results do not depend on the batch); sand_read_stats then
 * describes the last chunk.  The copies wait for the work queued on `stream`
 * before the call.  Pinned host memory gives full copy bandwidth (and lets the
 * copies run asynchronously).  Synchronous: returns after h_out is written, and
 * on every error path only after the three streams have drained. */
sand_status sand_query_sdf_host(sand_model m, const float *h_points, int64_t n, float *h_out,
                                const sand_query_opts *opts, void *stream);

/* No counterpart in the paper.  sand_query_sdf for callers that must not
 * allocate device memory during a query: for example a host framework whose
 * own memory pool owns the GPU's budget, or a latency-critical serving loop
 * that cannot afford cudaMalloc's implicit device synchronisation.  Same
 * arguments and results as sand_query_sdf, but opts->d_workspace must be NULL:
 * the scratch comes from one static device array inside libsand sized for
 * SAND_NOALLOC_MAX_POINTS points (about 17 MiB), which each GPU using it keeps
 * until the process exits.  n above SAND_NOALLOC_MAX_POINTS returns
 * SAND_EINVAL.  Nothing is allocated: the precision's device weights must
 * already exist, else SAND_EUNSUPPORTED.  SAND_FP32_SIMT's always do; a model
 * keeps the packed weights of one tensor-core precision at a time, those of
 * its most recent tensor-core query (or of sand_server_create), so query once
 * with the precision through sand_query_sdf first.  A precision the model
 * cannot take at all is SAND_EUNSUPPORTED with a message that says so.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress), so make it
 * before any stream capture.  Calls share the array: calls that may overlap on
 * the GPU (unordered streams) race and corrupt each other's results. */
#define SAND_NOALLOC_MAX_POINTS (1 << 20)
sand_status sand_query_sdf_noalloc(sand_model m, const float *d_points, int64_t n, float *d_out,
                                   const sand_query_opts *opts, void *stream);

/* Octree-free dynamic exit (the ablation of Table 6): no depth map; every point runs
 * layer by layer and stops at the first layer i whose tail |t_i| < r (the residual it
 * adds, Eq. 2), returning y_i, or at layer L.  Rows stop individually; a 128-row tile of
 * the tensor-core kernel stops issuing MMAs once all its rows have stopped (the points
 * are not sorted, so stopped rows ride along until then).  d_out [n]; d_exit_layers
 * [n] optional (the layer each point stopped at).  opts: only the precision (a
 * tensor-core one) is taken; the model's own workspace is used. */
sand_status sand_query_sdf_dynamic(sand_model m, const float *d_points, int64_t n, float r, float *d_out,
                                   uint8_t *d_exit_layers, const sand_query_opts *opts, void *stream);

/* ---------------------------------------------------------------- sphere tracing
 * Rendering use of the SAND SDF (Sec. 3.4 queries at ray samples; the paper
 * gives no tracing algorithm, this is classic sphere tracing).  Ray r has origin
 * o (d_origin[0..2] shared by every ray, or d_origin[3r..3r+2] when
 * per_ray_origin) and direction d_dirs[3r..3r+2] (float32, not normalised by the
 * library; unit length makes t a distance).  It starts at t = the parameter where
 * it enters [-1, 1]^3 (0 when o is inside) and repeats, at most max_steps times:
 * y = SAND query of p = fma(t, d, o) (float32 per component); |y| < hit_eps gives
 * SAND_RAY_HIT (t kept); otherwise t <- t + y, and leaving the ray's interval in
 * the domain gives SAND_RAY_MISS.  A NaN y gives SAND_RAY_NAN, the step limit
 * SAND_RAY_STEPS.  Rays that never enter the domain are SAND_RAY_MISS with 0 steps.
 * Outputs (device, caller-owned, each nullable): d_t [n] final t, d_state [n],
 * d_steps [n] queries made for the ray, d_grad [n][3] the input gradient of
 * y at the hit points (the surface normal direction, not normalised; 0 for rays
 * that did not hit), from a gradient query in qopts' precision (on the tensor
 * cores for SAND_FP32, SAND_FP16, SAND_BF16 and SAND_FP8; on the CUDA cores for
 * SAND_FP32_SIMT).
 * qopts: precision and max_depth apply to every step; its other fields must be
 * zero (the tracer owns its workspace: a grow-only device buffer of
 * sand_trace_state_bytes(n_rays) kept by the model, so trace calls on one model
 * must be stream-ordered).  The march is stream-ordered and needs no host round
 * trip; with poll_every = k > 0 the host reads the active-ray count every k
 * steps (a stream synchronisation) and stops early when it is 0. */
typedef enum { SAND_RAY_MISS = 0, SAND_RAY_HIT = 1, SAND_RAY_STEPS = 2, SAND_RAY_NAN = 3 } sand_ray_state;
typedef struct {
    int max_steps;     /* 1 .. 255 */
    float hit_eps;     /* > 0 */
    int poll_every;    /* 0 = launch all max_steps steps without reading back */
    int reserved;
} sand_trace_opts;
size_t sand_trace_state_bytes(int64_t n_rays);
sand_status sand_sphere_trace(sand_model m, const float *d_origin, int per_ray_origin, const float *d_dirs,
                              int64_t n_rays, const sand_trace_opts *topts, const sand_query_opts *qopts, float *d_t,
                              uint8_t *d_state, uint8_t *d_steps, float *d_grad, void *stream);

/* ---------------------------------------------------------------- depth-map construction
 * The volumetric network-depth map from the network itself (Sec. 3.2): for every leaf
 * of the octree (desc, h_child as in sand_load_depth_map_mem) with h_near[node] != 0
 * (the leaves whose cells meet the shape), Eq. 6 stores the maximum over k^3 sample
 * points x of Eq. 5,
 *   d(x) = min{ i : |y_L(x) - y_i(x)| < r  and  sign y_i(x) = sign y_L(x) },
 * (sign(0) taken as +1; i = L always qualifies), y_i the cumulative outputs of Eq. 2
 * evaluated on the tensor cores in opts->precision.  The samples are the cell-centred
 * k x k x k lattice of the leaf, x = lo + (s + 1/2) side / k per axis (k a power of two,
 * so every sample is exact in float32).  Far leaves get depth 0 (they answer with their
 * stored value, Eq. 7), or with far_sign the sign-only case of Eq. 5, max-pooled.
 * h_depth_out [n_nodes]: the leaves' depths, 0 for inner nodes.  Synchronous (the
 * result is on the host on return); host arrays are the caller's.  The paper's
 * r = 1.5e-4 assumes shapes normalised to the unit cube. */
typedef struct {
    int samples_per_axis;  /* k: 1, 2, 4, 8 or 16 */
    float r;               /* > 0 */
    int far_sign;          /* 0: far leaves keep depth 0; 1: sign-only case of Eq. 5 */
    int precision;         /* a tensor-core sand_precision (SAND_FP32: float32 accuracy) */
} sand_map_build_opts;
sand_status sand_build_depth_map(sand_model m, const sand_depth_map_desc *desc, const int32_t *h_child,
                                 const uint8_t *h_near, const sand_map_build_opts *opts, uint8_t *h_depth_out,
                                 void *stream);

/* Flags and counters a query leaves in its workspace (read after the query's
 * stream has been synchronised by this call). */
#define SAND_FLAG_NAN_INPUT 1u
#define SAND_FLAG_TIMEOUT 2u
typedef struct {
    uint32_t flags;          /* SAND_FLAG_* raised by the last query on this workspace */
    uint32_t n_network;      /* points evaluated by the network (exit layer >= 1) */
    uint32_t count[16];      /* points per exit layer 0 .. 14; count[15] = NaN points */
} sand_query_stats;
sand_status sand_read_stats(sand_model m, const void *d_workspace, sand_query_stats *out, void *stream);

/* ---------------------------------------------------------------- serving
 * Continuous batching over resident models (the paper has no serving layer;
 * this serves the query of Sec. 3.4 to many concurrent clients).  Requests carry
 * host buffers (pinned memory lets the copies overlap); a scheduler thread keeps
 * up to n_streams batches in flight, packing each model's queued requests in
 * arrival order into one query while the batch fits max_batch_points and the free
 * part of a device arena of mem_budget bytes reserved at creation (a request
 * needs 16 + sand_workspace_bytes bytes per point); requests that arrive while
 * batches run join the next batch as a stream and memory free up.  Every result
 * is identical to running the request alone through sand_query_sdf.  The models
 * must stay alive and must not be queried concurrently by the caller while the
 * server runs. */
typedef struct sand_server_s *sand_server;
typedef struct {
    int32_t n_streams;          /* batches in flight (default 3, at most 16) */
    int32_t precision;          /* sand_precision of every query */
    size_t mem_budget;          /* device arena for in-flight batches (default 1 GiB) */
    int64_t max_batch_points;   /* upper bound of points per batch (default 2^22; a larger request runs alone) */
    const int32_t *model_precision; /* optional [n_models]: per-model sand_precision overriding `precision`;
                                   one handle listed twice may not take two tensor-core precisions
                                   (a model packs one at a time): SAND_EINVAL */
} sand_server_opts;
typedef struct {
    int64_t requests, batches, points;   /* completed so far */
    double p50_ms, p99_ms, max_ms;       /* submit-to-result latency of completed requests */
    double queries_per_s;                /* points completed / (last completion - first submit) */
    size_t arena_bytes;
    double span_ms;                      /* last completion - first submit */
    double batch_ms_sum;                 /* sum over completed batches of their time on the device, from
                                            an event before their first copy to one after their last:
                                            above span_ms when batches were in flight at once (copies
                                            of one beside the query of another; the tensor-core kernel
                                            takes every SM, so two queries' kernels queue) */
} sand_server_report;
/* Start a server over n_models loaded models (all on one device).  Packs their
 * weights for opts->precision and reserves the arena; nothing is allocated later. */
sand_status sand_server_create(const sand_model *models, int n_models, const sand_server_opts *opts, sand_server *out);
/* Queue a request: SDF of h_points[n][3] under model `model` into h_out[n].  Both
 * buffers must stay valid until sand_server_wait returns for *ticket. */
sand_status sand_server_submit(sand_server s, int model, const float *h_points, int64_t n, float *h_out,
                               uint64_t *ticket);
/* Block until the request completed (SAND_ETIMEOUT after timeout_s seconds;
 * SAND_EINVAL for a negative or NaN timeout_s, values above 1e7 s are clamped);
 * *latency_ms (nullable) receives its submit-to-result time. */
sand_status sand_server_wait(sand_server s, uint64_t ticket, double timeout_s, double *latency_ms);
/* Latency percentiles and throughput of the requests completed so far. */
sand_status sand_server_stats(sand_server s, sand_server_report *out);
/* Finish queued work, stop the threads, release streams and the arena. */
sand_status sand_server_destroy(sand_server s);

/* ---- issue-rate probes (the roofline denominators of the epilogue pipes) ----
 * Launch n_blocks x 256 threads on `device` and `stream`; each thread runs 8
 * independent chains of `iters` steps and writes one float to d_sink (device,
 * n_blocks x 256 floats, 4-byte aligned; the values carry no meaning).
 *   SAND_PROBE_FFMA: one float32 fused multiply-add per step and chain, so
 *     2 x 8 x iters x 256 x n_blocks FLOP per launch;
 *   SAND_PROBE_SIN: one hardware sine of a radian argument (the form the sine
 *     activations of Eq. 2 take) and one multiply per step and chain, so
 *     8 x iters x 256 x n_blocks sines per launch.
 * Asynchronous: time it with events on `stream`.  SAND_EINVAL for an unknown
 * kind, n_blocks outside 1..2^20, iters <= 0 or a bad d_sink. */
typedef enum { SAND_PROBE_FFMA = 0, SAND_PROBE_SIN = 1 } sand_probe_kind;
sand_status sand_probe_rate(int kind, int device, int n_blocks, int iters, float *d_sink, void *stream);

/* ---------------------------------------------------------------- training
 * T-MLP training steps (Sec. 3.3): the loss is Eq. 4 with the L1 SDF loss of Eq. 8,
 *     L = sum_{i=1..L} (1/n) sum_x | y_i(x) - y_gt(x) |,
 * summed over every tail, so every hidden layer is supervised; the optimiser is Adam (Sec. 4.1:
 * learning rate 1e-4).  |r|' is taken as sign(r) with sign(0) = 0.  A trainer owns a float32
 * master copy of the model's parameters (in the parameter-block order of sand_load_tmlp_mem),
 * Adam's two moments, and device buffers for batches of up to max_points points; the model it
 * was made from is not changed until sand_trainer_commit.
 * The hidden-layer products of the forward pass, of the backward pass (dL/dh_{l-1} = W_l^T
 * delta_l) and of the weight gradients (dL/dW_l = sum_x delta_l h_{l-1}^T) run on the tcgen05
 * tensor cores with float32-class accuracy (each operand split into two fp16 terms, three
 * products, float32 accumulation), everything else in float32 on the CUDA cores.  Supported:
 * raw-coordinate models (no Fourier encoder) of width 64, 128 or 256, every activation and
 * tail kind; else SAND_EUNSUPPORTED.  Calls on one trainer must be stream-ordered. */
typedef struct sand_trainer_s *sand_trainer;
typedef struct {
    int64_t max_points;  /* largest batch (default 2^17) */
    float lr;            /* Adam step size (default 1e-4) */
    float beta1, beta2;  /* Adam decay rates (defaults 0.9, 0.999) */
    float eps;           /* Adam epsilon (default 1e-8) */
    int32_t reserved;
} sand_train_opts;
sand_status sand_trainer_create(sand_model m, const sand_train_opts *opts, sand_trainer *out);
/* One step on a batch: d_points device float32 [n][3], d_targets device float32 [n] (y_gt), 1 <= n
 * <= max_points.  Computes the loss and the gradient of every parameter; with update != 0 then
 * applies one Adam step.  d_loss (device float32 [1], nullable) receives L; d_grad (device float32
 * [n_params], nullable) receives dL/dparams in the parameter-block order (a Fourier matrix would
 * get 0).  Stream-ordered and asynchronous. */
sand_status sand_train_step(sand_trainer t, const float *d_points, const float *d_targets, int64_t n, float *d_loss,
                            float *d_grad, int update, void *stream);
/* The trainer's current parameters (host float32 [n_params], parameter-block order); synchronous. */
sand_status sand_trainer_params(sand_trainer t, float *h_params, size_t n_params);
/* Copy the trainer's parameters into its model (its packed weights are rebuilt on the next query);
 * synchronous. */
sand_status sand_trainer_commit(sand_trainer t);
/* SAND_ETIMEOUT if a bounded device-side wait of a training kernel gave up since the trainer was
 * made (synchronises the stream), else SAND_OK. */
sand_status sand_trainer_status(sand_trainer t, void *stream);
sand_status sand_trainer_destroy(sand_trainer t);

/* Describe a loaded model. */
sand_status sand_model_desc(sand_model m, sand_tmlp_desc *out);

/* Release the model's device memory. */
sand_status sand_free(sand_model m);

/* Message for the last failing call on this thread ("" if none). */
const char *sand_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SAND_H_ */
