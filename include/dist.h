/*
 * dist.h -- C ABI of libdist: differentiable sphere tracing of a DeepSDF-style
 * latent-conditioned MLP signed distance function on one NVIDIA B300 (sm_103a).
 *
 * Method: DIST (Liu et al., CVPR 2020, arXiv 1911.13225).  The problem
 * statement (Sec. 3.4 and Eq. 3 of Sec. 4.2.1): given a decoder f_theta(p, z),
 * a latent code z, a camera (intrinsics K, extrinsics) and an image size,
 * render depth, surface normal and soft silhouette by sphere tracing every
 * pixel's ray with at most `max_steps` queries and convergence threshold
 * `eps`, then back-propagate image-plane losses to z.
 *
 * Conventions for every entry point:
 *  - All functions return a dist_status and never abort, trap or print.
 *    On failure dist_last_error() returns a message for the calling thread.
 *  - "device" pointers are CUDA global-memory pointers on the current device;
 *    "host" pointers are ordinary CPU memory.  The caller owns every buffer it
 *    passes; the library owns decoders, workspaces and servers it creates.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Trace/loss/backward calls are stream-ordered: they enqueue
 *    work and return without synchronising and without allocating memory.
 *  - Pixels of several cameras are concatenated in camera order, each camera's
 *    pixels row-major (index = offset + y * W + x).  Cameras use OpenCV axes:
 *    x right, y down, z forward (the depth formula of Sec. 3.3).
 *  - Background pixels have depth +inf (Sec. 3.2, "Initialization").
 *  - One device per process: the library sizes its grids and sets its
 *    kernels' shared-memory limits for the device that is current at its
 *    first launch, and every later call must run with that device current.
 */
#ifndef DIST_H
#define DIST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DIST_OK = 0,
  DIST_E_INVALID = 1,     /* bad argument: NULL pointer, size out of range,
                             camera inside the bounding sphere, ...       */
  DIST_E_NOMEM = 2,       /* allocation failed, workspace too small, or a
                             serving request refused by the memory budget  */
  DIST_E_CUDA = 3,        /* a CUDA runtime call failed                   */
  DIST_E_TIMEOUT = 4,     /* a bounded wait ran out                       */
  DIST_E_BUSY = 5,        /* serving: result not ready / no free slot     */
  DIST_E_UNSUPPORTED = 6  /* e.g. BF16 tensor-core path asked for a decoder
                             shape it does not cover                      */
} dist_status;

/* Precision of the marching decoder queries.  BF16 and FP16 run the GEMM
 * layers on the tensor cores (16-bit operands, FP32 accumulation) and hand a
 * ray to FP32-class queries once |f| < eps_bf16; FP32 runs every query in
 * FP32 on the CUDA cores (the plain FP32 trace); FP32_TC runs every query on
 * the tensor cores with each operand carried as a sum of two FP16 numbers
 * (22 significant bits, FP32 accumulation), the DeepSDF shape only. */
typedef enum {
  DIST_PREC_FP32 = 0,
  DIST_PREC_BF16 = 1,
  DIST_PREC_FP16 = 2,
  DIST_PREC_FP32_TC = 3
} dist_precision;

/* Kernel of the FP32-class queries after a BF16/FP16 hand-over. */
typedef enum { DIST_REFINE_TC = 0, DIST_REFINE_SIMT = 1 } dist_refine_engine;

/* Step rule of the FP32-class queries after a BF16/FP16 hand-over: MARCH
 * keeps the paper's aggressive step (alpha_refine); SECANT takes one unit
 * step (Eq. 1's final step) and then secant steps through the last two
 * FP32-class samples (a step with a slope above -1e-3 or longer than 8 |f|
 * falls back to the aggressive step).  Either converges on |f| < eps. */
typedef enum { DIST_REFINE_MARCH = 0, DIST_REFINE_SECANT = 1 } dist_refine_rule;
typedef enum { DIST_GRAD_EXACT = 0, DIST_GRAD_PAPER = 1 } dist_grad_mode;

/* Ray outcome codes written to dist_trace_out.status. */
enum { DIST_RAY_INIT_MISS = 0, DIST_RAY_HIT = 1, DIST_RAY_LEFT = 2, DIST_RAY_MAX_STEPS = 3 };

/* ---------------------------------------------------------------- decoder */

/* Shape of the DeepSDF decoder (Sec. B.1: 9 FC layers, hidden 512, latent
 * 256, DeepSDF's skip concatenation).  Layer 0 reads [z (latent_dim), x, y, z];
 * layer `skip` reads [h, z, x, y, z] where h is the output of layer skip-1
 * (width - latent_dim - 3 values); hidden layers use ReLU; layer n_hidden is
 * the head (width -> 1) followed by tanh.  skip = -1: no skip layer.
 * The texture network of Sec. B.1 (colour for texture re-rendering) has the
 * same layers with a longer code at layer 0 and three outputs (reading: layer
 * 0 reads [code (latent_dim0), x, y, z], e.g. [shape code, texture code]; the
 * skip layer reads the code's last latent_dim entries, the texture code;
 * the head is width -> out_dim, each output followed by tanh).  Such a
 * decoder is used by dist_render_color only. */
typedef struct {
  int latent_dim;
  int width;       /* 128, 256, 384 or 512 */
  int n_hidden;    /* 2..16 */
  int skip;        /* -1 or 1..n_hidden-1 */
  int latent_dim0; /* layer-0 code length, latent_dim..1024; 0 = latent_dim */
  int out_dim;     /* 1 (SDF) or 3 (colour); 0 = 1 */
} dist_decoder_desc;

typedef struct dist_decoder dist_decoder;

/* Upload a decoder.  W[l] (host, float32, row-major [out_l][in_l]) and b[l]
 * (host, float32, [out_l]) for l = 0..n_hidden.  The library copies and
 * repacks the weights (FP32 copies in both orientations, and BF16 tensor-core
 * tiles when the shape is the DeepSDF one: width 512, 8 hidden, skip 4);
 * the host arrays may be freed on return.  Synchronous; allocates.
 * Errors: DIST_E_INVALID (bad desc / NULL), DIST_E_NOMEM, DIST_E_CUDA. */
dist_status dist_decoder_create(const dist_decoder_desc* desc,
                                const float* const* W, const float* const* b,
                                dist_decoder** out);
dist_status dist_decoder_destroy(dist_decoder* dec);
/* 1 if the BF16 tensor-core MLP covers this decoder, else 0. */
int dist_decoder_has_bf16(const dist_decoder* dec);
/* Not from the paper: every device-side wait of the tensor-core kernels is
 * bounded (1 s by default).  A launch that gives up sets bits in a device
 * error word of the decoder (1: weight loader, 2: MMA issuer, 4: epilogue or
 * step update of a forward kernel, 8/16/32: the adjoint's roles; 64: an
 * FP32-class activation beyond the FP16 range), drains its copies and MMAs,
 * frees its tensor memory and returns early (its outputs, and those of the
 * launches that depend on them, are then invalid).  This call synchronises
 * the device, returns the word in *code (0 = nothing since the last call)
 * and clears it.  Returns DIST_E_TIMEOUT if a wait ran out (bits 1..32),
 * else DIST_OK. */
dist_status dist_decoder_device_error(const dist_decoder* dec, int32_t* code);
/* Not from the paper: failure-detection settings of the tensor-core forward
 * kernel (the march, dist_sdf_eval, colour).  wait_ns: the limit of each of
 * its device-side waits, 1e4..1e10 ns (default 1e9).  withhold_copies = 1 is
 * for tests of the failure path: the kernel's weight loader issues no copies,
 * so the MMA issuer's first wait for a weight stage runs out after wait_ns;
 * the kernel then takes its abort path (error bits 2 and 4, see
 * dist_decoder_device_error) without faulting, and the decoder works
 * normally again once withhold_copies is 0.  Host-side state; set it only
 * while no call of this decoder is running. */
dist_status dist_decoder_set_wait_limit(dist_decoder* dec, uint64_t wait_ns, int withhold_copies);

/* ----------------------------------------------------------------- camera */

typedef struct {
  float fx, fy, cx, cy;  /* pinhole intrinsics K (pixels) */
  float R[9];            /* camera-to-world rotation, row-major; its columns
                            are the camera x, y, z axes in world frame    */
  float c[3];            /* camera centre in world frame                  */
  int H, W;              /* image size                                     */
  int shape;             /* index of this camera's latent code            */
} dist_camera;

/* ------------------------------------------------------------- parameters */

typedef struct {
  int max_steps;       /* queries per ray (Sec. B.4 uses 100; Tab. 1 50)   */
  float eps;           /* convergence threshold on |f| (Sec. 3.2: 5e-5)    */
  float alpha;         /* aggressive marching factor (Sec. 3.2: 1.5)       */
  int k_min;           /* samples with the smallest |f| kept per ray for the
                          paper's gradient (Sec. B.4: K = 1 or 3); 1..3    */
  float normal_delta;  /* 0: analytic normals; > 0: central differences
                          with this step (Sec. 3.3)                         */
  int grad_mode;       /* dist_grad_mode for the depth term                */
  int precision;       /* dist_precision of the marching queries           */
  float eps_bf16;      /* BF16/FP16 path: |f| below which a ray switches
                          to FP32 queries at the same point                 */
  float radius;        /* bounding sphere radius (Sec. 3.2: unit sphere)   */
  int refine_steps;    /* BF16/FP16 path: 0 = FP32 queries continue until
                          |f| < eps; n > 0 = after n FP32 queries a ray with
                          |f| < 4 eps_bf16 is also accepted as a hit (unit
                          final step, Eq. 1), its silhouette then reported
                          as |f| - 4 eps_bf16.  Ignored for FP32.          */
  float alpha_refine;  /* BF16/FP16 path: step factor of the FP32 queries
                          after the hand-over; 0 = alpha (the paper's
                          aggressive step), 1 = unit steps.  Ignored for
                          FP32.                                             */
  int refine_engine;   /* BF16/FP16 path: dist_refine_engine of the queries
                          after the hand-over (TC: the FP32_TC kernel,
                          SIMT: FP32 CUDA-core kernel)                      */
  int refine_rule;     /* BF16/FP16 path: dist_refine_rule of the queries
                          after the hand-over                               */
  int coarse_levels;   /* coarse-to-fine tracing (Sec. 3.2): 0 = off; n > 0
                          = start on an image 2^n times coarser per side
                          (the paper: 2) and split every ray into its four
                          children after every `coarse_every` march
                          iterations.  Every camera's H and W must be
                          multiples of 2^n; 0..4.  With a BF16/FP16 march
                          it needs refine_steps 0 and refine_engine TC.
                          What a child inherits is not stated in the
                          paper: it has its own direction and bounding-
                          sphere interval, and takes over its parent's ray
                          distance (raised to its own entry; past its own
                          exit it has left the sphere), step count, k
                          smallest-|f| samples (|f| raised to eps) and
                          outcome if the parent left the sphere or ran out
                          of queries; a child of a parent that missed the
                          sphere starts at its own entry.                   */
  int coarse_every;    /* march iterations per coarse level (the paper: 3) */
  int latency_mode;    /* tensor-core march with FP32-class TC queries
                          (refine_engine TC): 1 (default) = a step whose
                          lists fit in as many tiles (128 16-bit rays or
                          64 FP32-class rays each) as four-SM clusters fit
                          on the GPU at once (at most 37) spreads each tile over
                          four SMs, a quarter of every layer's columns per
                          SM; 0 = one tile per SM throughout.  Both
                          give the same f for every query.                   */
  float eps_mid;       /* BF16 march only: 0 (default) = a ray whose BF16
                          |f| < eps_bf16 goes straight to FP32-class
                          queries; in (0, eps_bf16) = it goes to FP16
                          queries first (same tensor rate, 3 more mantissa
                          bits) and from there to FP32-class queries once
                          its FP16 |f| < eps_mid (or its FP16 samples change
                          sign with |f| < 16 eps_mid), so fewer queries pay
                          the FP32-class cost.  Needs refine_engine TC,
                          refine_steps 0, refine_rule MARCH, coarse_levels
                          0; ignored for other precisions.                   */
} dist_trace_params;

/* Fill `p` with the paper's defaults: max_steps 50, eps 5e-5, alpha 1.5,
 * k_min 1, normal_delta 0, exact gradients, FP32, eps_bf16 1e-3, radius 1,
 * refine_steps 0, alpha_refine 0, refine_engine TC, refine_rule MARCH,
 * coarse_levels 0 (off), coarse_every 3, latency_mode 1, eps_mid 0. */
void dist_trace_params_default(dist_trace_params* p);

/* -------------------------------------------------------------- workspace */

typedef struct dist_workspace dist_workspace;

/* Library-owned device scratch for up to `max_rays` pixels per call: ray
 * state (32 B/ray), active-ray lists and per-step counters.  Allocates
 * (synchronous).  One workspace must not be used by two calls that overlap
 * on the device. */
dist_status dist_workspace_create(int64_t max_rays, int max_steps,
                                  dist_workspace** out);
dist_status dist_workspace_destroy(dist_workspace* ws);

/* ----------------------------------------------------------------- tracing */

/* Per-pixel results, caller-owned DEVICE buffers of n_pixels (= sum H*W)
 * entries unless stated.  Pointers marked "optional" may be NULL. */
typedef struct {
  float* depth;      /* z_c = d / sqrt(x~^2+y~^2+1) (Sec. 3.3); +inf = bg  */
  float* sil;        /* soft silhouette: min_n |f(p_n)| - eps, or
                        dist(origin, ray) - radius for rays missing the
                        bounding sphere (Sec. A.3); < 0 <=> hit             */
  uint8_t* mask;     /* 1 = converged hit                                   */
  int32_t* steps;    /* queries made for the ray                            */
  int32_t* status;   /* DIST_RAY_* outcome (optional)                       */
  float* d_hit;      /* ray distance after the unit final step (Eq. 1);
                        +inf when not a hit                                 */
  float* d_min;      /* [n_pixels][k_min] ray distances of the k samples
                        with the smallest |f| (ascending |f|), NaN if fewer */
  float* f_min;      /* [n_pixels][k_min] signed f at those samples         */
  float* normal;     /* [n_pixels][3] (optional): filled by dist_trace_fwd
                        when non-NULL, else by dist_render_normals          */
  unsigned long long* queries;  /* optional, device [2]: += MLP queries made
                        while marching, [0] 16-bit (BF16 or FP16), [1] FP32
                        or FP32-class                                       */
  float* grad_len;   /* (optional) written with `normal` when normal_delta >
                        0: |g| of the central difference g_a = (f(p + delta
                        e_a) - f(p - delta e_a)) / (2 delta) at the hit, 0
                        elsewhere (Sec. 3.3; normal = g / |g|).  With it,
                        dist_trace_bwd forms the normal loss's coefficients
                        from `normal` and `grad_len` instead of evaluating
                        the six probes again; both must then come from a
                        forward with the same params                        */
} dist_trace_out;

/* Forward render: unit-sphere initialisation (Sec. 3.2), then up to
 * max_steps iterations of {compact the unfinished rays, query the MLP,
 * converge/step} (Alg. 1 with aggressive marching and dynamic synchronized
 * inference, Sec. 3.2 and B.2), then depth / silhouette / mask (Sec. 3.3).
 * z: device float [n_shapes][latent_dim].  cams: HOST array of n_cams.
 * Errors: DIST_E_INVALID (NULL/sizes, n_pixels > workspace, camera inside
 * the bounding sphere, shape index out of range, k_min outside 1..3),
 * DIST_E_UNSUPPORTED (BF16 asked, decoder not covered), DIST_E_CUDA. */
dist_status dist_trace_fwd(const dist_decoder* dec, const float* z, int n_shapes,
                           const dist_camera* cams, int n_cams,
                           const dist_trace_params* params,
                           const dist_trace_out* out, dist_workspace* ws,
                           void* stream);

/* Surface normals at the hits of a previous dist_trace_fwd (same arguments;
 * reads out->mask and out->d_hit): the normalised analytic gradient of f
 * (normal_delta = 0) or the paper's central differences (Sec. 3.3).
 * normal: device float [n_pixels][3]; zero for non-hit pixels.  When normal
 * is out->normal, out->grad_len (if set) is written too. */
dist_status dist_render_normals(const dist_decoder* dec, const float* z, int n_shapes,
                                const dist_camera* cams, int n_cams,
                                const dist_trace_params* params,
                                const dist_trace_out* fwd, float* normal,
                                dist_workspace* ws, void* stream);

/* Evaluate the decoder f(p, z_shape) (Sec. 3.4: f_theta(p, z)) at n points:
 * pts: device float [n][3]; shape: device int32 [n] latent index per point;
 * f: device float [n]; grad: device float [n][3] = grad_p f, or NULL.
 * precision DIST_PREC_FP32 (SIMT kernels; grad allowed), DIST_PREC_BF16 or
 * DIST_PREC_FP16 (tensor-core kernels; grad must be NULL), DIST_PREC_FP32_TC
 * (tensor-core kernels with two-term FP16 operands; with grad, f and grad_p f
 * both come from the FP32-class adjoint kernel, whose f may differ from the
 * forward kernel's in the last bits).  n <= 10 * workspace max_rays.
 * Shape indices outside [0, n_shapes) are clamped into range.
 * Errors: DIST_E_INVALID, DIST_E_UNSUPPORTED, DIST_E_CUDA. */
dist_status dist_sdf_eval(const dist_decoder* dec, const float* z, int n_shapes,
                          const float* pts, const int32_t* shape, int64_t n, int precision,
                          float* f, float* grad, dist_workspace* ws, void* stream);

/* dist_sdf_eval without a workspace and without allocating (the paper has
 * no counterpart: this is a convenience of this library).  Meant for callers
 * that cannot call cudaMalloc: a plugin that must live inside a host
 * application's fixed GPU memory budget, a framework whose pool owns all
 * device memory, or a latency-critical thread that must not take the device
 * synchronisation an allocation can imply.  The scratch (folded latent
 * biases, packed points, gradient staging) is a built-in device array of
 * 2,359,552 bytes that every GPU which loads the library keeps until the
 * process exits.  Limits: 1 <= n <= 65536 points and 1 <= n_shapes <= 64;
 * larger sizes return DIST_E_INVALID.  Arguments, precisions (FP32 with or
 * without grad; BF16, FP16 and FP32_TC without) and results are those of
 * dist_sdf_eval, bit for bit (the same kernels; no workspace).  The first
 * call on a device, made with that device current, looks up the array's
 * device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  All calls share the one
 * array, so calls whose work overlaps on the GPU (different streams, or
 * threads without ordering) race and corrupt each other's results; a call
 * rewrites every scratch entry it reads, so nothing carries over between
 * ordered calls.  Allocates nothing and frees nothing. */
dist_status dist_sdf_eval_static(const dist_decoder* dec, const float* z, int n_shapes,
                                 const float* pts, const int32_t* shape, int64_t n,
                                 int precision, float* f, float* grad, void* stream);

/* ------------------------------------------------------------------- loss */

typedef struct {
  float w_depth;   /* L1 depth (Sec. 4.2.1, B.3)                         */
  float w_normal;  /* negative dot product of normals (Sec. B.3)         */
  float w_sil;     /* silhouette loss, Eq. 4 of Sec. A.3                  */
  float w_reg;     /* ||z||^2 regulariser (Sec. B.4)                      */
} dist_loss_weights;

/* Image-plane loss of a rendered batch and its per-pixel upstream gradients.
 * Depth and normal terms are means over M = (rendered hit) and (target depth
 * finite) (Sec. B.3: over the rendered foreground); the silhouette term is a
 * mean over all pixels; the regulariser is w_reg * sum ||z||^2.
 * Inputs (device): depth, mask, sil, normal (NULL if w_normal == 0), targets
 * tgt_depth [n] (+inf = background), tgt_normal [n][3] (NULL if unused),
 * tgt_sil [n] (1 = foreground; NULL if unused), z [n_shapes][latent_dim].
 * Outputs (device): loss (double, 1 value, overwritten), g_depth [n],
 * g_normal [n][3] (may be NULL if w_normal == 0), g_sil [n] (may be NULL if
 * w_sil == 0), dz [n_shapes][latent_dim] OVERWRITTEN with 2 w_reg z, so that
 * dist_trace_bwd can accumulate into it.  The workspace provides the small
 * reduction scratch. */
dist_status dist_loss(int64_t n_pixels, const float* depth, const uint8_t* mask,
                      const float* sil, const float* normal,
                      const float* tgt_depth, const float* tgt_normal,
                      const float* tgt_sil, const float* z, int n_shapes, int latent_dim,
                      const dist_loss_weights* w, double* loss,
                      float* g_depth, float* g_normal, float* g_sil, float* dz,
                      dist_workspace* ws, void* stream);

/* Multi-view photometric loss (Sec. 4.2: each colour image warped into the
 * other views by the rendered depth; Sec. B.3: visibility by the depth test
 * (z_j(P) - D_j)^2 < 1e-3).  For each ordered pair (i, j) in `pairs` (host,
 * [n_pairs][2]), every pixel of view i with a finite depth is lifted to its
 * world point, projected into view j and image j sampled there bilinearly
 * between pixel centres; a projection whose four neighbours are not all
 * inside view j and hit there, or that fails the depth test, is not visible.
 * loss = w * (sum over visible pixels of all pairs of the channel-summed L1
 * colour difference) / (number of them), 0 with none.  Inputs (device):
 * depth [n] (dist_trace_out.depth of the same cameras, +inf background),
 * images [n][channels] (1..4 channels, pixels in camera order, row-major).
 * Outputs (device): loss (double), g_depth [n] = dL/d depth OVERWRITTEN (the
 * visibility decisions and the other view's depth are held fixed), to pass
 * to dist_trace_bwd.  Uses the workspace's camera table and reduction
 * scratch; no decoder is involved. */
dist_status dist_photo_loss(const dist_camera* cams, int n_cams, const float* depth,
                            const float* images, int channels, const int32_t* pairs,
                            int n_pairs, float w, double* loss, float* g_depth,
                            dist_workspace* ws, void* stream);

/* --------------------------------------------------------------- backward */

/* dL/dz += sum over pixels of upstream gradients times the latent Jacobians
 * of the rendered depth, normal and silhouette (device dz [n_shapes][L],
 * ACCUMULATED).  Depth: grad_mode EXACT differentiates the converged root
 * implicitly, dd/dz = -(df/dz)/(grad_p f . v) at the hit (grazing rays,
 * |grad_p f . v| < 1e-3 |grad_p f|, contribute 0); PAPER keeps the first term
 * of Eq. 2 over the k_min smallest-|f| samples, alpha * sum_k df(p_k)/dz
 * (Sec. 3.4, B.2).  Silhouette: sign(f_min) df(p_min)/dz (Sec. A.3 with the
 * first-term rule).  Normal: needs normal_delta > 0; VJP of the central-
 * difference normal with the hit point held fixed.  The decoder is
 * re-evaluated at these points only (no per-step graph is stored): the depth
 * probes in the trace's precision (16-bit tensor-core adjoint after a BF16 or
 * FP16 march, FP32-class tensor-core adjoint after FP32_TC, FP32 CUDA cores
 * after FP32); the silhouette and central-difference probes at FP32-class
 * accuracy whatever the march's (the FP32-class tensor-core adjoint where the
 * trace's FP32-class queries run on the tensor cores, else FP32 CUDA cores).
 * Upstream gradients g_depth [n], g_normal [n][3], g_sil [n] are device
 * arrays or NULL.  Per-ray sums are reduced in FP64. */
dist_status dist_trace_bwd(const dist_decoder* dec, const float* z, int n_shapes,
                           const dist_camera* cams, int n_cams,
                           const dist_trace_params* params,
                           const dist_trace_out* fwd,
                           const float* g_depth, const float* g_normal,
                           const float* g_sil, float* dz,
                           dist_workspace* ws, void* stream);

/* One Adam step on the latent codes, the optimiser of the inverse problem
 * (Sec. 4.2: shape from depth by optimising z through the renderer; Sec.
 * B.4: Adam, lr 1e-2; the update is Adam as published, Kingma & Ba 2015):
 *   m = beta1 m + (1 - beta1) dz,  v = beta2 v + (1 - beta2) dz^2,
 *   z -= lr / (1 - beta1^t) * m / (sqrt(v / (1 - beta2^t)) + eps).
 * z, m, v: device float [n], updated in place (m and v start at 0); dz:
 * device float [n], the gradient (e.g. of dist_loss + dist_trace_bwd);
 * t: the step number, from 1.  Element-wise FP32, so (z, m, v, t) fully
 * determine the result (a checkpoint of them resumes bit for bit).
 * Errors: DIST_E_INVALID (NULL, n < 1, t < 1, lr <= 0, beta outside [0, 1),
 * eps <= 0), DIST_E_CUDA. */
dist_status dist_adam_step(float* z, const float* dz, float* m, float* v, int64_t n, int t,
                           float lr, float beta1, float beta2, float eps, void* stream);

/* Gradients of the loss with respect to each camera's extrinsics (Sec. 4.2:
 * the pose optimised through the renderer with the shape fixed, from depth
 * and silhouette).  A camera enters each ray through its centre c and the
 * direction v = R v_cam / |R v_cam|, v_cam the unit pixel direction in the
 * camera frame.  Depth: the exact implicit derivative of the converged root,
 * dd = -(grad_p f . (dc + d dv)) / (grad_p f . v) at the hit (grazing rays
 * contribute 0, as in dist_trace_bwd), times 1/sqrt(x~^2+y~^2+1).
 * Silhouette of a ray that entered the bounding sphere: the first-term rule,
 * sign(f_min) grad_p f(p_min) . (dc + d_min dv) with d_min held fixed; of a
 * ray that missed it: the exact derivative of the distance from the origin
 * to the ray.  R is differentiated as a free 3 x 3 matrix (v renormalised).
 * Output dcam (device, [n_cams][12], OVERWRITTEN): dL/dc (3 floats) then
 * dL/dR row-major (9 floats) per camera; per-camera sums are reduced in
 * FP64.  grad_p f comes from the decoder adjoint in the trace's precision.
 * g_depth [n], g_sil [n] are device arrays or NULL.  Uses the workspace's
 * probe buffers and reduction scratch. */
dist_status dist_trace_bwd_camera(const dist_decoder* dec, const float* z, int n_shapes,
                                  const dist_camera* cams, int n_cams,
                                  const dist_trace_params* params,
                                  const dist_trace_out* fwd, const float* g_depth,
                                  const float* g_sil, float* dcam, dist_workspace* ws,
                                  void* stream);

/* Texture re-rendering (Sec. B.1): the colour of every hit pixel of a trace
 * from a colour decoder (out_dim 3, see dist_decoder_desc) at the hit point
 * p = c + d_hit v, rgb = tanh(head) per channel; background pixels get 0.
 * codes (device, [n_shapes][latent_dim0]): the colour decoder's code per
 * shape (the paper: [shape code, texture code]); each camera's `shape` picks
 * it.  fwd and ws must come from the dist_trace_fwd of the same cameras (the
 * workspace holds the rays).  precision: DIST_PREC_FP32 (CUDA cores) or
 * BF16 / FP16 (tensor cores; the head in FP32).  Output rgb (device,
 * [n][3]) OVERWRITTEN. */
dist_status dist_render_color(const dist_decoder* tex, const float* codes, int n_shapes,
                              const dist_camera* cams, int n_cams, const dist_trace_out* fwd,
                              int precision, float* rgb, dist_workspace* ws, void* stream);

/* ---------------------------------------------------------------- serving */

typedef struct dist_server dist_server;

typedef enum { DIST_REQ_RENDER = 0, DIST_REQ_RENDER_BACKWARD = 1 } dist_request_kind;

/* One request.  All pointers are HOST memory owned by the caller and must
 * stay valid until dist_serve_poll reports the request done. */
typedef struct {
  int kind;                  /* dist_request_kind                          */
  dist_camera cam;           /* cam.shape is ignored                       */
  const float* z;            /* [latent_dim] latent code                   */
  const float* tgt_depth;    /* [H*W], RENDER_BACKWARD only (L1 depth)     */
  float* depth;              /* [H*W] out                                  */
  float* sil;                /* [H*W] out (optional)                       */
  uint8_t* mask;             /* [H*W] out (optional)                       */
  float* dz;                 /* [latent_dim] out, RENDER_BACKWARD only     */
  double* loss;              /* out, RENDER_BACKWARD only                  */
} dist_request;

/* A continuous-batching render server on its own thread and stream: requests
 * are admitted while the ray pool (max_rays) and the device-memory budget
 * allow, their rays march together with those already in flight, and each
 * request completes as soon as its own rays finish.  Allocates. */
dist_status dist_serve_create(const dist_decoder* dec, const dist_trace_params* params,
                              int64_t max_rays, size_t mem_budget_bytes,
                              int max_requests, dist_server** out);
/* Non-blocking.  DIST_E_INVALID for a malformed request, DIST_E_NOMEM if the
 * request alone exceeds the pool or the budget, DIST_E_BUSY if the queue of
 * pending requests is full. */
dist_status dist_serve_submit(dist_server* s, const dist_request* req, uint64_t* ticket);
/* Non-blocking: *done = 1 once the request's outputs are in its host buffers
 * (the ticket is then retired), else 0. DIST_E_INVALID for an unknown
 * ticket; a failed request returns its error status. */
dist_status dist_serve_poll(dist_server* s, uint64_t ticket, int* done);
/* Stops the server thread (bounded wait) and frees its memory. */
dist_status dist_serve_destroy(dist_server* s);

/* ------------------------------------------------------------ measurement */

/* Not from the paper: instrumentation used to measure the kernels against
 * their roofline.  While enabled, every decoder-MLP launch of the march in
 * dist_trace_fwd (the dominant kernels) is bracketed by CUDA events recorded
 * on the stream it is launched on, and every kernel launch of the library is
 * counted, as is every decoder adjoint launch (normals and backward).
 * enable = 1 resets the counters and starts recording (host-side state, not
 * thread-safe); 0 stops.  dist_profile_read synchronises the recorded events
 * and returns, per kernel kind ([0] BF16 tensor-core MLP of the march,
 * [1] FP32 SIMT MLP of the march, [2] decoder adjoint), the summed kernel
 * time in ms and the number of timed launches, plus the count of all library
 * kernel launches.  Each array argument points to 3 host values; any pointer
 * may be NULL.  At most 65536 launches are timed per enable. */
dist_status dist_profile_enable(int enable);
dist_status dist_profile_read(double* mlp_ms, int64_t* mlp_launches, int64_t* all_launches);

/* ------------------------------------------------------------------- misc */

/* Message of the last error on the calling thread ("" if none). */
const char* dist_last_error(void);
/* Library version string. */
const char* dist_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DIST_H */
