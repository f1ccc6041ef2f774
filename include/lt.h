/* lt.h -- C ABI of liblt: constant-memory reverse-mode differentiable light tracing on
 * one NVIDIA GB300 (sm_103a).
 *
 * The problem (paper "Constant-Memory Differentiable Light Tracing", Sec. 3.2): given a
 * scene with parameters theta (diffuse albedo textures, emitted radiance Le, height-field
 * vertex heights), render the light-traced image I (Sec. 3.1, Eq. 1-2: every light path
 * x0..xk splats each unoccluded non-specular vertex's sensor connection L_i at film
 * position u_i through a reconstruction filter, Eq. 20), and given the image-space adjoint
 * dI = dLoss/dI compute dLoss/dtheta = d<dI, I>/dtheta without a tape that grows with path
 * depth.  Two constant-memory methods: ResLRB (Sec. 4.2) and LRB-3-pass (Sec. 4.3), each
 * detached (values only) or attached (vertices and splat positions move, Sec. 3.3, 4.4).
 * A naive reverse-mode baseline with a per-vertex tape is provided for comparison.
 *
 * Conventions
 *  - Every call is asynchronous on the CUDA stream passed as `stream` (a cudaStream_t;
 *    NULL = legacy default stream) unless stated otherwise.
 *  - "DEVICE" pointers are CUDA device memory owned by the caller; "HOST" pointers are
 *    read before the call returns.  The library never frees caller memory.
 *  - Errors: host-side validation returns immediately with a status and a message
 *    readable through lt_last_error() (thread-local).  Device-side checks (index bounds,
 *    bounded waits) set an error word in the scene; lt_sync_status() reads and clears it.
 *    No call aborts the process or traps the GPU; no C++ exception crosses the ABI.
 *  - Float images are row-major [H][W][3] (row 0 at the top of the film), FP32.
 *  - Random numbers: Philox4x32-10 keyed by the 64-bit seed, counter (path index, vertex
 *    depth, stream); every path is replayed from its index, nothing else is stored.
 */
#ifndef LT_H
#define LT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LT_OK = 0,
  LT_ERR_INVALID_ARG = 1,   /* a host-side argument check failed                    */
  LT_ERR_OOM = 2,           /* allocation failed or caller workspace too small      */
  LT_ERR_CUDA = 3,          /* a CUDA runtime call failed                           */
  LT_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up (reserved: no kernel
                               of the library waits on another thread or launch)    */
  LT_ERR_DEVICE_CHECK = 5,  /* a device-side bounds/consistency check fired         */
  LT_ERR_UNSUPPORTED = 6    /* valid request the library does not implement         */
} lt_status;

enum { LT_MAT_DIFFUSE = 0, LT_MAT_DIELECTRIC = 1, LT_MAT_EMITTER = 2 };
enum { LT_EST_PLAIN = 0, LT_EST_RESLRB = 1, LT_EST_NAIVE = 2, LT_EST_BUFFERED = 3 };
enum { LT_TARGET_LUMINANCE = 0, LT_TARGET_MLP = 1 };

typedef struct lt_scene lt_scene; /* opaque: device geometry, BVH, error word */

/* Scene description (all HOST pointers, copied by lt_scene_create).
 * Primitives: quads first (ids 0..n_quads-1), then triangles.  A quad is the
 * parallelogram o + s e1 + t e2, s,t in [0,1]; a triangle is (v0, v1, v2) with
 * vertex k at verts[tris[3i+k]] plus (0, heights[vert_h[.]], 0) when vert_h >= 0.
 * Geometric normal = cross(e1, e2) (cross(v1-v0, v2-v0)).  Diffuse surfaces are
 * two-sided Lambertian with albedo texture h x w x 3 at albedo[mat_tex_off...]
 * (bilinear, texel centres, clamp to edge, texture coordinates = (s, t) on quads and the
 * barycentrics (b1, b2) on triangles).  Dielectrics are smooth with index mat_ior.
 * The emitter is a one-sided Lambertian quad emitting along its normal; it absorbs
 * any ray that hits it.  Pinhole camera: image plane at distance 1, vertical field of
 * view fov_y_deg, width x height pixels. */
typedef struct {
  int n_quads;
  const float* quads;      /* [n_quads][9] o, e1, e2                               */
  int n_verts;
  const float* verts;      /* [n_verts][3] base positions                          */
  const int* vert_h;       /* [n_verts] height-parameter index or -1               */
  int n_tris;
  const int* tris;         /* [n_tris][3] vertex indices                           */
  const int* prim_mat;     /* [n_quads + n_tris] material index                    */
  int n_mats;
  const int* mat_type;     /* [n_mats] LT_MAT_*                                    */
  const float* mat_ior;    /* [n_mats]                                             */
  const int* mat_tex_off;  /* [n_mats] offset (floats) into the albedo array       */
  const int* mat_tex_w;    /* [n_mats]                                             */
  const int* mat_tex_h;    /* [n_mats]                                             */
  int emitter_quad;        /* quad index of the area emitter                       */
  float cam_pos[3], cam_look[3], cam_up[3];
  float fov_y_deg;
  int width, height;
  int n_albedo;            /* length of the albedo parameter array                 */
  int n_heights;           /* length of the heights parameter array                */
} lt_scene_desc;

/* Per-call parameters theta (DEVICE pointers, FP32, caller-owned, read only). */
typedef struct {
  const float* albedo;   /* [n_albedo]; > 0 wherever d_albedo is requested (below)  */
  const float* Le;       /* [3]; each component > 0 wherever d_Le is requested      */
} lt_params;

/* Largest n_paths and path_offset any call accepts (LT_ERR_INVALID_ARG beyond): every byte
 * count derived from a path count then fits in size_t with room to spare. */
#define LT_MAX_PATHS ((int64_t)1 << 40)

typedef struct {
  uint64_t seed;        /* Philox key                                               */
  int64_t path_offset;  /* first path index (Philox counter) traced by this call    */
  int64_t n_paths;      /* number of paths traced by this call (<= LT_MAX_PATHS)    */
  int64_t n_norm;       /* N of the estimator's 1/N; 0 means n_paths                */
  int max_depth;        /* traced intersections x1..xD per path, 1..64              */
  int attached;         /* 0 detached, 1 attached (geometry derivatives)            */
  int target;           /* reservoir target: LT_TARGET_LUMINANCE or LT_TARGET_MLP   */
  const void* mlp;      /* DEVICE lt_mlp weights when target == LT_TARGET_MLP       */
  int block_size;       /* threads per block, 0 = library default                   */
  int blocks_per_sm;    /* resident blocks per SM for the persistent grid, 0 = auto */
  const uint8_t* path_mask; /* DEVICE [n_paths] optional: 0 = skip path (testing)   */
  uint32_t* path_hash;  /* DEVICE [n_paths] optional out: decision hash per path    */
  float* path_dbg;      /* DEVICE [n_paths][4] optional out (see each call)         */
  uint64_t* census;     /* DEVICE [5] optional out, lt_backward_lrb3 and
                           lt_primal(LT_EST_PLAIN) only: adds the work done (rays
                           traced, BVH box tests, primitive tests, path vertices,
                           valid connections) using a counting kernel variant; for
                           measurement, not for timed runs                        */
  void* lrb3_state;     /* DEVICE optional, for lt_backward_lrb3 (and written by a
                           plain lt_primal, see lrb3_mask_ready): per-path state of
                           lt_lrb3_state_bytes(opts) bytes.  Given, passes 2 and 3 run
                           as two kernels and pass 2 stores each path's delta_total
                           and connection-validity mask there (the paper's three-pass
                           form; 48 B per path and 4.2 MB, flat in depth); NULL, one fused kernel
                           keeps them in registers.  Same result either way.      */
  size_t lrb3_state_bytes; /* size of lrb3_state                                    */
  int lrb3_mask_ready;  /* lt_primal(LT_EST_PLAIN) given lrb3_state also stores each
                           path's connection-validity mask there, the list of the
                           paths that have a valid connection, and each path's first
                           valid connection (film position, contribution).  Set 1 in
                           the opts of lt_backward_lrb3 when that primal ran with the
                           same seed, paths, depth, scene and parameters: pass 2 then
                           takes validity from the mask, traces no visibility rays,
                           stops each path after its last valid connection, forms
                           delta_total of a path with one valid connection from the
                           stored connection without replaying it, and passes 2 and 3
                           visit only the listed paths (the others have delta_total
                           zero; their stored colour words and path_dbg rows are left
                           as they are and not read).                           */
  int rr_depth;         /* Russian roulette: after each vertex of depth >= rr_depth a
                           path continues with probability rr_prob (Philox stream 2
                           of that depth) and its throughput is divided by rr_prob;
                           0 = off.  Every pass replays the same decisions; 1/rr_prob
                           is a constant factor of the path's function.            */
  float rr_prob;        /* survival probability in (0, 1] when rr_depth > 0          */
  int filter;           /* reconstruction filter of splat and adjoint read (Eq. 20-21):
                           0 tent of radius 1 pixel; 1 truncated Gaussian, standard
                           deviation 0.5 pixel, radius 1.5 pixel, shifted to reach 0
                           at the radius and normalised to unit integral           */
  int bvh_width;        /* BVH node width traversed: 2 (threaded binary BVH, stackless),
                           4 or 8 (wide BVH, ordered stack traversal); 0 = 4.  The
                           scene holds all three; results agree up to ties.        */
  int scatter;          /* how gradients and splats reach memory (Eq. 3 scatter, Eq. 20
                           splat); results agree up to the order of float additions:
                           0 default: albedo then height gradients accumulate per block
                             in shared memory when the arrays fit in 46 KB, and are added
                             to the caller's arrays once per block; an array that does
                             not fit is added with plain global atomics, and so are the
                             splats;
                           1 as 0, the per-block arrays up to the device's opt-in shared
                             memory per block (227 KB on GB300; fewer blocks may then be
                             resident per SM);
                           2 no per-block arrays, plain global atomics;
                           3 no per-block arrays, warp-aggregated global atomics (lanes of
                             a warp adding to the same element sum first) for the
                             gradients and for the plain primal's splats.           */
  int literal;          /* lt_backward_lrb3, attached: 0 exact transport of the splat-
                           position adjoint along specular chains (default); 1 the
                           paper's transport (Sec. 3.3, Eq. 4-7, Eq. 18-19, Sec. 5):
                           forward-accumulated 4x4 Jacobians of the two-point segment
                           parameterisation (v_{k-1}, v_k) of surface coordinates, the
                           position rows of each connection summed as A_pos in pass 2 and
                           projected back in pass 3 with the inverse of the accumulated
                           Jacobian, zero when it is singular by construction (a zero
                           block entered it) or |det| < det_eps times the product of
                           its row norms (Hadamard's bound).  After a diffuse vertex
                           the next vertex keeps its surface coordinates, so that
                           Jacobian is singular and chains starting there lose their
                           position transport (biased) unless jac_noise is set.  Runs
                           one fused kernel, one path per thread; the radiance terms are
                           those of the exact form                                */
  int jac_noise;        /* with literal: zero-mean noise eps [I 0], eps = +-1 (Philox
                           stream 4 at that depth, keyed by noise_seed), in the zero
                           block of the Jacobian at diffuse vertices: unbiased over the
                           noise                                                  */
  uint64_t noise_seed;  /* Philox key of that noise                                 */
  float det_eps;        /* with literal: relative determinant guard; 0 = 1e-6      */
} lt_render_opts;

/* Gradient outputs (DEVICE, FP32, caller-owned).  NULL skips a parameter group.
 * Overwritten unless accumulate != 0. */
typedef struct {
  float* d_albedo;   /* [n_albedo]: the adjoints apply the log-derivative identity (Eq. 3)
                        at each diffuse vertex, dividing its weight by the albedo there;
                        a texel of zero albedo seen by a path makes its entries
                        non-finite */
  float* d_Le;       /* [3]: a path's value is linear in Le (Eq. 2), so every backward
                        forms this gradient as the path's contribution divided by Le; a
                        zero component of Le makes that entry non-finite (the other
                        outputs stay valid) */
  float* d_heights;  /* [n_heights] */
  int accumulate;
} lt_grads;

/* Build the scene: copies the description to the device, builds a binned-SAH BVH over
 * all primitives (host, once) and uploads it.  Heights start at zero; call
 * lt_scene_refit to set them.  Returns LT_ERR_INVALID_ARG for inconsistent arrays. */
lt_status lt_scene_create(const lt_scene_desc* desc, void* stream, lt_scene** out);

/* Set the height-field parameters (DEVICE [n_heights]) and refit triangle geometry and
 * BVH bounds on the device (topology unchanged).  Must precede any render call that
 * should see the heights.  Attached derivatives are taken at these heights. */
lt_status lt_scene_refit(lt_scene* scene, const float* heights, void* stream);

/* Free the scene's device memory (cudaFree, which waits for work in flight on the
 * device) and the handle.  NULL is accepted and ignored.  The scene must not be in use
 * by a batch that is still alive; the handle is invalid afterwards. */
void lt_scene_destroy(lt_scene* scene);

/* Primal light tracing (Sec. 3.1; ResLRB primal Sec. 4.2 and its listing; naive AD
 * forward pass).  image: DEVICE [H][W][3], overwritten.
 *   estimator LT_EST_PLAIN : splat every valid connection (LRB-3-pass pass 1).
 *   estimator LT_EST_RESLRB: stream connections into a capacity-1 weighted reservoir
 *       (Eq. 8) and splat only the winner reweighted by Omega_k/omega_R (Eq. 9); writes
 *       one record per path into `aux` (DEVICE, n_paths * lt_record_size()).
 *   estimator LT_EST_NAIVE : splat every connection and write the per-vertex tape into
 *       `aux` (DEVICE workspace of aux_bytes >= lt_naive_workspace_bytes(opts), else
 *       LT_ERR_OOM).
 * path_dbg (optional): [n_paths][4] = (n valid connections, depth reached, 0, 0). */
lt_status lt_primal(lt_scene* scene, const lt_params* params, const lt_render_opts* opts, int estimator,
                    float* image, void* aux, size_t aux_bytes, void* stream);

/* LRB-3-pass backward (Sec. 4.3, Eq. 14-19): pass 2 accumulates
 * delta_total = sum_i Lbar_i * L_i (and in the attached case the positional adjoint),
 * pass 3 replays again, backpropagates each splat with Lbar_i (Eq. 15), subtracts
 * (Eq. 16) and backpropagates the scattering factors with delta_rem (Eq. 17).  Without
 * opts->lrb3_state both passes run fused per path and no per-path state reaches global
 * memory; with it, pass 2 and pass 3 are two kernels that hand delta_total and the
 * connection-validity mask over through that buffer (memory flat in depth either way).
 * LT_ERR_INVALID_ARG if lrb3_state_bytes < lt_lrb3_state_bytes(opts).
 * d_image: DEVICE [H][W][3] adjoint dI.  path_dbg (optional) [n_paths][4] =
 * (delta_total rgb, n valid connections). */
lt_status lt_backward_lrb3(lt_scene* scene, const lt_params* params, const lt_render_opts* opts,
                           const float* d_image, const lt_grads* grads, void* stream);

/* ResLRB backward (Sec. 4.2.1-4.2.2, Eq. 11-13): reads each path's record written by
 * lt_primal(LT_EST_RESLRB) with the same opts, replays the path up to the selected
 * vertex R and applies the log-derivative identity weighted by Lbar_R * S, plus the
 * splat-position channel in the attached case. */
lt_status lt_backward_reslrb(lt_scene* scene, const lt_params* params, const lt_render_opts* opts,
                             const float* d_image, const void* records, const lt_grads* grads, void* stream);

/* Naive reverse-mode baseline: reverse sweep over the tape written by
 * lt_primal(LT_EST_NAIVE) with the same opts (memory linear in max_depth). */
lt_status lt_backward_naive(lt_scene* scene, const lt_params* params, const lt_render_opts* opts,
                            const float* d_image, const void* workspace, size_t ws_bytes,
                            const lt_grads* grads, void* stream);

/* Film pipeline (Sec. 4.3.1 pass 1, "develop, evaluate loss, backpropagate"): L2 loss
 * loss = sum (I - T)^2 / n and d_image = 2 (I - T) / n over n floats.  DEVICE pointers;
 * loss: DEVICE [1] (overwritten). */
lt_status lt_film_l2(const float* image, const float* target, int64_t n, float* d_image, float* loss,
                     void* stream);

/* ---------------------------------------------------------------------------------
 * Learned reservoir target.  A 16 -> 64 -> 64 -> 1 ReLU network (BF16 weights, FP32
 * accumulation on tensor cores) predicts, from a sensor connection's features, the log of
 * the adjoint weight |Lbar_i * L_i|_1 / lum(L_i) the connection will see; ResLRB then uses
 * omega_i = lum(L_i) (exp(sigma * y_i) + 1e-3) (sigma = target scale) in place of the
 * luminance of Eq. 8.  Because Eq. 10 holds for any positive weights the estimator stays
 * unbiased; only its variance changes.  Parameter block: LT_MLP_PARAMS floats (DEVICE,
 * FP32): W1[16][64] b1[64] W2[64][64] b2[64] W3[64] b3 | feature mean[16] | feature
 * 1/std[16] | target scale | target mean | padding.  Pass it as opts->mlp with
 * opts->target = LT_TARGET_MLP to lt_primal(LT_EST_RESLRB).
 * Features (16): vertex position (3), arrival-side normal (3), arrival direction (3),
 * log throughput (3), (depth index + 1) / max_depth, film u / width, film v / height,
 * log of the connection weight. */
#define LT_MLP_PARAMS 5352
#define LT_MLP_WEIGHTS 5313

/* Training pairs from an LRB-3 pass-2 replay (Eq. 14): for every valid connection, its 16
 * features into feats [capacity][16] and its target log(|Lbar*L|_1 / lum(L) + floor) into
 * targets [capacity] (DEVICE), in no particular order (rows are claimed atomically).
 * *count (DEVICE int64, zeroed by this call) receives the number of connections found;
 * only the first `capacity` are written.  opts->path_mask skips paths. */
lt_status lt_mlp_collect(lt_scene* scene, const lt_params* params, const lt_render_opts* opts,
                         const float* d_image, float target_floor, float* feats, float* targets,
                         int64_t capacity, int64_t* count, void* stream);

/* Set the standardisation statistics of the parameter block from n training pairs. */
lt_status lt_mlp_init_stats(float* mlp, const float* feats, const float* targets, int64_t n, void* stream);

/* Gradient of the mean squared error of the standardized target over samples [0, n) of a
 * batch of size `batch` (added into grad [LT_MLP_WEIGHTS], DEVICE; the mean loss is added
 * into *loss, DEVICE).  Forward and backward GEMM tiles run on tensor cores. */
lt_status lt_mlp_grad(const float* mlp, const float* feats, const float* targets, int64_t n, int64_t batch,
                      float* grad, float* loss, void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8; `step` counts from 1) on the trainable
 * block, with moment buffers m, v [LT_MLP_WEIGHTS] (DEVICE). */
lt_status lt_mlp_adam(float* mlp, float* m, float* v, const float* grad, int step, float learning_rate,
                      void* stream);

/* Network outputs (standardized target units) for n feature rows (DEVICE). */
lt_status lt_mlp_forward(const float* mlp, const float* feats, int64_t n, float* out, void* stream);

/* ---------------------------------------------------------------------------------
 * Naive-AD gradient without any allocation (no counterpart in the paper).
 * Some callers cannot hand the library a workspace or let it allocate one: an application
 * that owns a fixed GPU memory budget and forbids allocations once it is running, or a
 * render loop for which cudaMalloc/cudaFree are off limits because they can synchronise
 * the whole device and stall every other stream.  For them this call runs the same two
 * kernels as lt_primal(LT_EST_NAIVE) followed by lt_backward_naive, but keeps the
 * per-vertex tape in one fixed scratch array of LT_NAIVE_STATIC_BYTES that is compiled
 * into the library: every GPU that loads liblt holds that memory until the process exits.
 * The caller still passes the fixed adjoint d_image (DEVICE [H][W][3]), the image to
 * overwrite (DEVICE [H][W][3]) and the gradient outputs.
 *  - Requests whose tape (lt_naive_workspace_bytes(opts)) exceeds LT_NAIVE_STATIC_BYTES are
 *    rejected with LT_ERR_INVALID_ARG; nothing is launched.
 *  - The scene's device must be the current device.  The first call on a device looks up
 *    the scratch array's device address for that device (once, cached afterwards); make
 *    that first call before any stream capture on that device begins.  The cached address
 *    belongs to the device's current context: after cudaDeviceReset (or any other teardown
 *    of the primary context) the library may be loaded at another address, so do not call
 *    this function again in that process after such a reset.
 *  - All calls on a device share the one array and it keeps whatever the last call left;
 *    each call writes every tape entry it later reads, so nothing needs clearing, but two
 *    calls whose work overlaps on the GPU (for example on two streams) race on the array
 *    and must be serialised by the caller. */
#define LT_NAIVE_STATIC_BYTES (32u << 20)
lt_status lt_naive_gradient_static(lt_scene* scene, const lt_params* params, const lt_render_opts* opts,
                                   const float* d_image, float* image, const lt_grads* grads, void* stream);

/* ---------------------------------------------------------------------------------
 * Batched passes (no counterpart in the paper, which renders one scene at a time):
 * many scenes with uneven path budgets, depths and geometry run their paths in ONE
 * persistent launch per pass and kernel variant.  Each item's path range is cut into
 * chunks of 32 * paths_per_thread paths; a warp takes the next chunk of its launch with
 * one atomic, so items of any size share the GPU without a launch per item.  Backward
 * passes run attached items on scenes with dielectrics (specular chains) in a second
 * persistent kernel, a parallel branch of the same graph, because that kernel variant
 * needs about twice the registers.  Each pass (its clears, height refits and kernels) is
 * captured once into a CUDA graph and replayed by lt_batch_run.  Per path the work is the same as the single-scene call
 * with the item's opts, so results match those calls up to floating-point summation
 * order (atomics).
 *
 * An item fixes every buffer the passes use (all DEVICE, caller-owned, alive and unmoved
 * until lt_batch_destroy; the scene too).  Buffer contents are read at each run, so
 * parameters, heights and d_image may change between runs. */
typedef struct {
  lt_scene* scene;
  lt_params params;
  const float* heights;    /* [n_heights] or NULL: primal passes refit the scene first;
                              two items with heights must not share a scene          */
  lt_render_opts opts;     /* seed, path_offset, n_paths, n_norm, max_depth, attached,
                              path_mask, path_hash, path_dbg, lrb3_state and
                              lrb3_mask_ready are used as by the single-scene calls
                              (each item its own state).  When every item has an
                              lrb3_state, LT_PASS_LRB3 runs pass 2 for all items, then
                              pass 3, as separate persistent launches, and
                              LT_PASS_PRIMAL stores the validity masks that
                              lrb3_mask_ready lets pass 2 reuse.  The launch shape
                              and BVH width come from the batch configuration       */
  float* image;            /* [H][W][3] primal passes: overwritten                   */
  void* records;           /* [n_paths][lt_record_size] ResLRB records, or NULL when the
                              ResLRB passes are not run                              */
  const float* d_image;    /* [H][W][3] adjoint read by the backward passes           */
  lt_grads grads;          /* overwritten by the backward passes unless accumulate    */
} lt_batch_item;

/* Passes.  PRIMAL = lt_primal(LT_EST_PLAIN) of every item; PRIMAL_RESLRB =
 * lt_primal(LT_EST_RESLRB) (luminance target) writing `records`; LRB3 =
 * lt_backward_lrb3; RESLRB = lt_backward_reslrb reading `records`. */
enum { LT_PASS_PRIMAL = 0, LT_PASS_PRIMAL_RESLRB = 1, LT_PASS_LRB3 = 2, LT_PASS_RESLRB = 3 };

/* Launch shape of the persistent kernels.  blocks_per_sm = 0: as many blocks as fit on an
 * SM at once (occupancy of the pass's kernel), so the grid is resident. */
typedef struct {
  int block_size;        /* 64, 128 or 256                                             */
  int paths_per_thread;  /* 1, 2, 4 or 8: chunk = 32 * paths_per_thread paths          */
  int blocks_per_sm;     /* 0 = occupancy, else 1..32                                  */
  int bvh_width;         /* 2, 4 or 8 (see lt_render_opts.bvh_width)                   */
} lt_batch_config;

typedef struct lt_batch lt_batch; /* opaque: item table on the device, captured graphs */

/* Copy the items (n >= 1) and build the device item table.  All scenes must be on the
 * current device.  Default configuration: block 128, 4 paths per thread, occupancy,
 * BVH width 4.
 * Synchronises `stream` once (table upload). */
lt_status lt_batch_create(const lt_batch_item* items, int n, void* stream, lt_batch** out);

/* Run one pass for every item on `stream`: launches the pass's CUDA graph (captured on
 * first use on a stream the batch owns, and again after lt_batch_set_config).  Passes of
 * one batch share state and must not overlap on the GPU (serialise them on one stream).
 * LT_ERR_INVALID_ARG: unknown pass, or a ResLRB pass with an item without records. */
lt_status lt_batch_run(lt_batch* batch, int pass, void* stream);

/* Set the launch shape of the batch's persistent kernels.  LT_ERR_INVALID_ARG for a NULL
 * batch or a cfg outside the ranges of lt_batch_config (the configuration is then left
 * unchanged).  The captured graphs are dropped and recaptured at the next run. */
lt_status lt_batch_set_config(lt_batch* batch, const lt_batch_config* cfg);
/* Copy the current configuration into *cfg (LT_ERR_INVALID_ARG if either is NULL). */
lt_status lt_batch_get_config(const lt_batch* batch, lt_batch_config* cfg);

/* Autotuner: time the pass (graph replay, CUDA events on `stream`, best of `reps` after
 * one warm-up) for every block_size in {64, 128, 256} x paths_per_thread in {1, 2, 4, 8}
 * x bvh_width in {2, 4, 8} at occupancy, keep the fastest as the batch configuration and
 * return it in *best (and its time per pass in *best_ms, either may be NULL).  Blocking: synchronises `stream`.
 * The pass runs many times; outputs hold one complete run of the pass afterwards (a
 * backward pass with accumulate set accumulates every run). */
lt_status lt_batch_tune(lt_batch* batch, int pass, int reps, void* stream, lt_batch_config* best, float* best_ms);

/* Free the item table, the captured graphs and the batch's own streams and events; the
 * items' scenes and buffers stay the caller's.  NULL is accepted and ignored.  No run of
 * the batch may be in flight. */
void lt_batch_destroy(lt_batch* batch);

/* ---------------------------------------------------------------------------------
 * Bidirectional estimator: the paper's light tracer combined with camera-side samples, the
 * "combined bidirectional formulation" its discussion names as a next step ("Toward more
 * complex integrators": path replay backpropagation on the camera side, LRB-3-pass on the
 * light side).  Two strategies estimate the same paths x0 (on the emitter), x1..xk
 * (diffuse) -> camera:
 *   light: a light path and its sensor connection at xk (opts->n_paths paths, Sec. 3.1);
 *   camera: a camera sample through a film position uniform over the film, traced to
 *       xk = y1, x(k-1) = y2, ... by cosine sampling, with next-event estimation from
 *       x1 = ym to a point x0 uniform on the emitter (n_cam samples, Philox stream 3:
 *       counter (c, 0) the film position, (c, m) at camera vertex m the cosine direction
 *       (u0, u1) and the emitter point (u2, u3)).
 * They are combined with the balance heuristic: with Lambertian surfaces, cosine sampling
 * and cosine emission a segment between two surfaces has the same area density in both
 * directions, so the density ratio of the camera strategy to the light strategy is
 * R = p_film(xk) / pf0 (the film's area density at xk over the light tracer's density of x1
 * from x0, cos0 cos1 / (pi r01^2)), and a sample of either strategy splats
 * N L / (N + M R) (L: the light tracer's splat value of the path, which carries 1/N;
 * N = opts->n_norm or n_paths, M = n_cam).  Each camera sample splats the sum of its
 * vertices' contributions at its film position.  Which strategy owns a path is thus a
 * weight, not a choice: every path reaches the image through both, in proportions N : M R.
 * Detached only (albedo, Le); scenes without dielectrics; no Russian roulette
 * (LT_ERR_UNSUPPORTED otherwise).  The camera side's adjoint is path replay
 * backpropagation: a camera sample contributes at one film position, so one adjoint read
 * serves all its vertices; a first walk sums the contributions, a replay weights each
 * vertex's albedo with the adjoint of the contributions from that vertex on.  The light
 * side's adjoint is LRB-3-pass (Eq. 14-17) with the weights (constant in the parameters).
 * Memory is constant in depth on both sides. */
typedef struct {
  int64_t n_cam;            /* camera samples M (0..LT_MAX_PATHS)                         */
  const uint8_t* cam_mask;  /* DEVICE [n_cam] optional: 0 = skip the sample (testing)     */
  uint32_t* cam_hash;       /* DEVICE [n_cam] optional out (lt_bidir_primal): decision hash
                               of each camera sample (primitives hit, next-event validity) */
} lt_bidir_opts;

/* Bidirectional image: image DEVICE [H][W][3], overwritten.  opts->path_hash (optional)
 * receives the light paths' decision hashes. */
lt_status lt_bidir_primal(lt_scene* scene, const lt_params* params, const lt_render_opts* opts,
                          const lt_bidir_opts* bidir, float* image, void* stream);

/* Gradient of <d_image, I_bidir> (albedo and Le; d_heights, if given, is zeroed unless
 * accumulate): LRB-3-pass on the light paths, path replay backpropagation on the camera
 * samples, both with the same opts and bidir as the primal. */
lt_status lt_bidir_backward(lt_scene* scene, const lt_params* params, const lt_render_opts* opts,
                            const lt_bidir_opts* bidir, const float* d_image, const lt_grads* grads, void* stream);

/* Buffered two-pass backward (the paper's lrb_2pass baseline, Sec. 4.1 and Sec. 6.2): the
 * primal lt_primal(LT_EST_BUFFERED) splats like LT_EST_PLAIN and also stores every traced
 * vertex's splat record (film position and contribution L_i, 20 B per vertex, memory
 * linear in max_depth) in `buffer`; this call computes delta_total = sum_i Lbar_i * L_i
 * from those records without tracing (Eq. 14) and then replays each path once to
 * backpropagate (Eq. 15-17), so two traversals in all instead of LRB-3's three.  Same
 * result as lt_backward_lrb3.  buffer: DEVICE, lt_lrb2_buffer_bytes(opts) bytes, written
 * by lt_primal(LT_EST_BUFFERED) with the same opts (LT_ERR_OOM if smaller).  path_dbg
 * (optional) [n_paths][4] = (delta_total rgb, n valid connections). */
lt_status lt_backward_lrb2(lt_scene* scene, const lt_params* params, const lt_render_opts* opts,
                           const float* d_image, void* buffer, size_t buffer_bytes, const lt_grads* grads,
                           void* stream);
size_t lt_lrb2_buffer_bytes(const lt_render_opts* opts);

/* Bytes of the optional LRB-3 per-path state (opts->lrb3_state): 16 B (delta_total rgb,
 * validity bits 0-31), 4 B (validity bits 32-63) and 4 B (the list of paths with a valid
 * connection) per path, then the list's length and the passes' counters (256 B), then
 * 20 B per path (film position and contribution of the path's first valid connection,
 * written by the plain primal: pass 2 takes delta_total of a path with exactly one valid
 * connection from it instead of replaying the path), then 4 B per path and a fixed 4.2 MB
 * (the order in which the plain primal takes the paths, sorted by the cell of each path's
 * first direction, and the counting sort's work area; the order changes no result); each
 * array 256-B aligned. */
size_t lt_lrb3_state_bytes(const lt_render_opts* opts);

/* Bytes of one ResLRB record (constant per path). */
size_t lt_record_size(const lt_render_opts* opts);
/* Bytes of the naive-AD tape for opts (n_paths * max_depth * record); 0 for invalid opts. */
size_t lt_naive_workspace_bytes(const lt_render_opts* opts);

/* Read and clear the scene's device error word (synchronises `stream`). */
lt_status lt_sync_status(lt_scene* scene, void* stream);

/* Thread-local message describing the last failed call on this thread. */
const char* lt_last_error(void);

/* Library build string (architecture, version). */
const char* lt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LT_H */
