/*
 * gs.h -- C ABI of libgs: the differentiable 16x16-tile Gaussian rasterizer
 * with the entropy term on blending weights and the periodic scale reset of
 * "Speeding Up the Learning of 3D Gaussians with Much Shorter Gaussian Lists"
 * (arXiv 2603.09277), built for NVIDIA GB300 (sm_103a).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers named in a struct or argument as "device" are CUDA device
 *    memory owned by the caller (the library never frees them).  "host"
 *    pointers are ordinary host memory read during the call.
 *  - Every call enqueues work on `stream` (a cudaStream_t; NULL is the legacy
 *    default stream) and returns without synchronising, except gs_bin_sort
 *    when `num_pairs_host` is non-NULL (it then waits for the pair count).
 *  - Return value: GS_OK (0) or a negative GS_ERR_* code.  Argument errors are
 *    detected on the host before anything is enqueued.  GS_ERR_CUDA keeps the
 *    cudaError_t text for gs_last_error_string().
 *  - Outputs are fully overwritten, gradients included (the calls zero them).
 *  - Views: V cameras of possibly different sizes.  Per-(view, Gaussian)
 *    arrays have V*N rows, row v*N + g.  Per-pixel arrays hold the views back
 *    to back, view v starting at pixel offset sum_{u<v} W_u H_u, row-major
 *    within a view.  Tiles are numbered globally: view v's tile (tx, ty) is
 *    tile_offset_v + ty * TX_v + tx with TX_v = ceil(W_v / 16),
 *    TY_v = ceil(H_v / 16), tile_offset_v = sum_{u<v} TX_u TY_u.
 *  - Pixel (x, y) is sampled at (x + 0.5, y + 0.5); the background is black.
 *  - A view is at most 65535 tiles wide and high (1,048,560 pixels at 16-pixel
 *    tiles); larger cameras are invalid arguments.
 *
 * Error behaviour on the device: no kernel traps or asserts.  Capacity
 * overflow of the pair buffers is reported through a device status word
 * (GS_ERR_CAPACITY) together with the required pair count.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* gs_stream; /* cudaStream_t */

enum gs_status {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = -1,
    GS_ERR_CUDA = -2,
    GS_ERR_CAPACITY = -3,
    GS_ERR_TIMEOUT = -4,
    GS_ERR_UNSUPPORTED = -5
};

/* Staging precision of the per-Gaussian render records (Gaussian attributes
 * only; exponent, transmittance and every accumulation stay FP32). */
enum gs_attr_dtype { GS_ATTR_F32 = 0, GS_ATTR_F16 = 1, GS_ATTR_BF16 = 2 };

#define GS_TILE 16 /* default tile side in pixels; 8 is the other supported side */
#define GS_MAX_VIEWS 64
#define GS_SH_COEFFS_MAX 16

/* Pinhole camera (Sec. 3: "for rendering from a given camera viewpoint").
 * world_to_cam: row-major 3x4 [R | t], camera x right, y down, z forward.
 * cam_pos: camera centre in world space (used for the SH view direction). */
typedef struct {
    int width, height;
    float fx, fy, cx, cy;
    float world_to_cam[12];
    float cam_pos[3];
} gs_camera;

/* Thresholds and projection constants.  The paper states none of them; the
 * defaults follow the 3DGS family it builds on:
 *   alpha_max 0.99 (alpha clamp), alpha_min 1/255 (entries below are
 *   skipped), t_min 1e-4 (the walk stops before blending an entry that would
 *   leave T < t_min), dilation 0.3 (added to the 2D covariance diagonal),
 *   near_z 0.2, fov_clamp 1.3 (x/z and y/z clamp of the EWA Jacobian in
 *   units of the half field of view). */
typedef struct {
    float alpha_max, alpha_min, t_min, dilation, near_z, fov_clamp;
    int sh_degree;  /* degree in use, 0..3 */
    int sh_stride;  /* SH coefficients stored per Gaussian, >= (sh_degree+1)^2, <= 16 */
    int attr_dtype; /* enum gs_attr_dtype */
    int tile_size;  /* tile side in pixels: 16 (3DGS; 0 also means 16) or 8 (LiteGS and the
                       paper's own runs, Sec. 5 "Effect of tile sizes"); every call of one
                       pipeline must use the same side */
    int sh_layout;  /* layout of the SH coefficients and of their gradient: 0 = [N][sh_stride][3]
                       (a Gaussian's coefficients together), 1 = [sh_stride][N][3] (each
                       coefficient of all Gaussians together: the loads of one coefficient are
                       contiguous, and a degree below sh_stride reads only its coefficients) */
} gs_params;

/* Projected per-(view, Gaussian) attributes, V*N rows, device memory. */
typedef struct {
    void* records;           /* required: gs_record_bytes(attr_dtype) per row, 16-B aligned */
    float* depth;            /* required [V*N]: FP32 camera-space depth of every row */
    int* rect;               /* [V*N][4]: tile rect x0, y0, x1, y1 (half-open); required
                                unless rect8 is set and every view is at most 255 tiles wide and
                                high, where NULL leaves it out (gs_bin_sort then reads rect8
                                alone; the projection saves 16 bytes of writes per row) */
    unsigned* tiles_touched; /* required [V*N]: (x1-x0)(y1-y0), 0 when culled */
    int* radius;             /* optional [V*N]: ceil(3 sqrt(lambda_max)) px */
    float* mean2d;           /* optional [V*N][2] */
    float* conic_opacity;    /* optional [V*N][4]: a, b, c, sigma; d = -1/2(a dx^2 + 2b dx dy + c dy^2) */
    float* rgb;              /* optional [V*N][3]: clamped SH colour */
    unsigned* rect8;         /* optional [V*N]: the rect of every visible row packed in 8-bit
                                fields, x0 | y0 << 8 | x1 << 16 | y1 << 24, written by
                                gs_preprocess when every view is at most 255 tiles per side
                                (rows it culls, and wider views, leave it untouched) and read by
                                gs_bin_sort under the same condition, where it replaces the
                                random 16-byte gather of `rect` in depth order by a 4-byte one;
                                when set for gs_bin_sort it must hold gs_preprocess's output for
                                the same cameras and tile side */
} gs_proj;

/* Optional launch controls of the render calls (NULL = defaults). */
typedef struct {
    const unsigned* tile_order;    /* device [total_tiles]: tile processing order, e.g. from
                                      gs_tile_queue (longest list first); NULL = natural order */
    unsigned* work_counter;        /* device [1]: work-claim counter for a persistent launch,
                                      reset by the call on the stream; required if ctas > 0 */
    int ctas;                      /* 0: one CTA per tile; > 0: persistent grid of that many
                                      CTAs claiming tiles from tile_order through work_counter */
    unsigned long long* stats;     /* device [2] (optional): += blended pairs, += evaluated pairs
                                      (forward only) */
    void* ev_begin;                /* optional cudaEvent_t recorded on the stream right before the
                                      blending kernel (for live per-kernel timing) */
    void* ev_end;                  /* optional cudaEvent_t recorded right after it */
    int pixels_per_thread;         /* 1, 2 or 4 pixels of a column per thread (0 = 2); 4 only
                                      with 16-pixel tiles */
    int batch;                     /* list entries staged in shared memory per batch: 256, or
                                      128 with F32 records and 16-pixel tiles (0 = 256) */
    void* zero_beside;             /* gs_render_fwd (optional): device memory that the blending
                                      kernel zeroes with streaming stores at the start of its
                                      CTAs (ragged ends off 16-byte boundaries by a memset on
                                      `stream`); meant for the grad2d buffer of the following
                                      gs_render_bwd, whose own zeroing would otherwise sit
                                      between the two blending kernels (the forward is bound by
                                      instruction issue and leaves the memory bandwidth mostly
                                      idle) */
    unsigned long long zero_bytes; /* bytes of zero_beside to zero (0: none) */
    int grad2d_zeroed;             /* gs_render_bwd: nonzero when grad2d is already zero (e.g.
                                      through the forward's zero_beside); the call then skips
                                      its own zeroing of grad2d */
} gs_launch;

/* ---------------------------------------------------------------------- */
/* Sizes and helpers                                                       */
/* ---------------------------------------------------------------------- */

/* Bytes of one render record for the given staging dtype (48 for F32, 32 for
 * F16/BF16); -1 for an unknown dtype. */
int gs_record_bytes(int attr_dtype);

/* Total number of tiles of side tile_size (16 or 8; 0 means 16) over the V
 * views (host cams), or -1. */
long long gs_total_tiles(const gs_camera* cams_host, int V, int tile_size);

/* Total pixels over the V views, or -1. */
long long gs_total_pixels(const gs_camera* cams_host, int V);

/* Workspace bytes that gs_bin_sort needs for n_rows = V*N projected rows, a
 * pair capacity and a tile count. */
size_t gs_bin_sort_workspace_size(long long n_rows, long long pair_capacity, long long total_tiles);

/* Workspace bytes that gs_loss_l1_entropy needs for `total_pixels` pixels. */
size_t gs_loss_workspace_size(long long total_pixels);

/* Workspace bytes that gs_tile_queue needs. */
size_t gs_tile_queue_workspace_size(long long total_tiles);

const char* gs_status_string(int status);
/* Text of the last CUDA error seen by this thread's calls ("" if none). */
const char* gs_last_error_string(void);
/* Library build string (architecture and version). */
const char* gs_version(void);
/* Number of kernels this process has launched through libgs so far (all
 * threads, all devices); for launch accounting. */
unsigned long long gs_kernel_launches(void);

/* Live per-kernel timing of the stages without a gs_launch argument: the
 * calling thread's next calls record ev_begin / ev_end (cudaEvent_t, or NULL
 * to stop) on their stream right before and after the stage's kernel.
 * Stages: GS_STAGE_EXPANSION (gs_bin_sort's expansion of the super-tile rows
 * into the per-tile lists), GS_STAGE_PROJECTION (gs_preprocess's kernel),
 * GS_STAGE_ADJOINT (gs_render_bwd's projection adjoint).  Returns
 * GS_ERR_INVALID_ARG for an unknown stage. */
enum gs_stage { GS_STAGE_EXPANSION = 1, GS_STAGE_PROJECTION = 2, GS_STAGE_ADJOINT = 3 };
int gs_stage_events(int stage, void* ev_begin, void* ev_end);

/* Status of the bounds-checked debug build (the library compiled with
 * -DGS_DEBUG_BOUNDS): *status = the id of the first index check that failed
 * since the last clear (0: none; 1xx blending, 2xx list construction, 3xx
 * projection adjoint), the failing access having been skipped; clear != 0
 * resets it.  Synchronous (reads device memory).  The normal build has no
 * checks: *status = 0 and GS_ERR_UNSUPPORTED. */
int gs_debug_bounds_status(unsigned* status, int clear);

/* ---------------------------------------------------------------------- */
/* Hot path                                                                */
/* ---------------------------------------------------------------------- */

/* Projection of every Gaussian into every view (Sec. 3, Background: the
 * 3D covariance Sigma = R S S^T R^T from the quaternion (w, x, y, z) and
 * s = exp(log_scale), EWA splatting to a 2D mean and covariance, the
 * inverse covariance, opacity sigmoid(logit), SH colour up to degree 3 plus
 * 0.5 clamped at 0), the 3-sigma radius and the tile rect.
 *   means [N][3], log_scales [N][3], quats [N][4] (need not be unit length),
 *   opacity_logits [N], sh [N][prm->sh_stride][3] (prm->sh_layout 0) or
 *   [prm->sh_stride][N][3] (layout 1): device, FP32.
 *   cams_host [V], prm host.  out: device buffers with V*N rows.
 * A Gaussian is culled (tiles_touched 0) when its FP32 depth (the FP32
 * rounding of the FP64 camera-space z) is <= near_z, its 2D covariance is
 * singular, a projected value is not finite, or its rect is empty.
 * GS_ERR_INVALID when out->rect is NULL and out->rect8 is NULL or a view is
 * more than 255 tiles wide or high. */
int gs_preprocess(const float* means, const float* log_scales, const float* quats,
                  const float* opacity_logits, const float* sh, int N,
                  const gs_camera* cams_host, int V, const gs_params* prm, const gs_proj* out,
                  gs_stream stream);

/* Per-tile Gaussian lists (Sec. 3: "the splatting process produces a
 * Gaussian list at each pixel"; sorted by depth for the blending of Sec. 3).
 * Result: sorted_vals[0..P) holds row indices v*N + g ordered by
 * (global tile, FP32 depth bits, g), i.e. the order of the 64-bit key
 * (tile << 32) | depth_bits with ties by Gaussian id; tile_ranges[2t],
 * tile_ranges[2t+1] = [start, end) of tile t in sorted_vals (0, 0 if empty).
 *   proj: output of gs_preprocess (depth, tiles_touched and the rects are
 *   read: rect8 when set and every view is at most 255 tiles wide and high,
 *   else rect, which must then be set).
 *   tile_size: the tile side gs_preprocess used (prm->tile_size).
 *   workspace: device, >= gs_bin_sort_workspace_size(V*N, pair_capacity,
 *   total_tiles) bytes, 256-B aligned.
 *   sorted_vals [pair_capacity], tile_ranges [2*total_tiles], num_pairs_dev [1],
 *   status_dev [1]: device outputs.  sorted_keys [pair_capacity] (optional):
 *   the 64-bit keys in sorted order.
 *   num_pairs_host (optional): if non-NULL the call synchronises `stream`,
 *   writes P there and returns GS_ERR_CAPACITY when P > pair_capacity
 *   (nothing beyond the count is then written).  If NULL (the form for CUDA
 *   graph capture) nothing is synchronised; on overflow the device writes
 *   *status_dev = GS_ERR_CAPACITY, keeps P in *num_pairs_dev, empties every
 *   range, and the caller regrows and reruns. */
int gs_bin_sort(const gs_proj* proj, int N, const gs_camera* cams_host, int V, int tile_size,
                void* workspace, size_t workspace_bytes, long long pair_capacity,
                unsigned* sorted_vals, unsigned long long* sorted_keys, unsigned* tile_ranges,
                long long* num_pairs_dev, long long* num_pairs_host, int* status_dev,
                gs_stream stream);

/* Front-to-back alpha blending per tile (16x16 or 8x8 pixels, Sec. 3) with the entropy of
 * the blending weights (Sec. 4.3).  Per pixel, over its tile's list:
 *   alpha = min(alpha_max, sigma exp(d)); entries with alpha < alpha_min are
 *   skipped; the walk stops before blending an entry with
 *   T (1 - alpha) < t_min; w = alpha T; C += w c; T *= 1 - alpha.
 *   H = -sum w ln w - T ln T over the blended entries and the background.
 * Outputs (device, per pixel): image [P][3], final_T [P], last_idx [P]
 * (1-based list position of the last blended entry, 0 if none), entropy [P]
 * (may be NULL).  opt: see gs_launch (NULL = one CTA per tile).  Launch
 * options without a kernel (pixels_per_thread other than 0/1/2/4, or 4 with
 * 8-pixel tiles; batch other than 0/128/256, or 128 with F16/BF16 records
 * or 8-pixel tiles; ctas < 0; ctas > 0 without work_counter) return
 * GS_ERR_INVALID_ARG, here and in gs_render_bwd. */
int gs_render_fwd(const gs_proj* proj, int N, const gs_camera* cams_host, int V,
                  const gs_params* prm, const unsigned* sorted_vals, const unsigned* tile_ranges,
                  float* image, float* final_T, unsigned* last_idx, float* entropy,
                  const gs_launch* opt, gs_stream stream);

/* Loss of Sec. 3 (L_base with lambda = 0, i.e. the L1 term) plus the
 * entropy term of Sec. 4.3, per view averaged over its M_v pixels, then
 * averaged over the V views:
 *   L = (1/V) sum_v [ (1/(3 M_v)) sum |C - C*| + gamma (1/M_v) sum_j H_j ].
 * Writes loss_dev [1] (double, device), dL_dimage [P][3] = sign(C - C*) /
 * (3 M_v V) with sign(0) = 0, and dL_dentropy [P] = gamma / (M_v V) (may be
 * NULL).  entropy may be NULL when gamma == 0.  workspace: device,
 * gs_loss_workspace_size(P) bytes. */
int gs_loss_l1_entropy(const float* image, const float* target, const float* entropy,
                       const gs_camera* cams_host, int V, float gamma, double* loss_dev,
                       float* dL_dimage, float* dL_dentropy, void* workspace,
                       size_t workspace_bytes, gs_stream stream);

/* Workspace bytes that gs_loss_base needs for the V views (host cams). */
size_t gs_loss_base_workspace_size(const gs_camera* cams_host, int V);

/* The full L_base of Sec. 3 Eq. base with its D-SSIM term, plus the entropy
 * term of Sec. 4.3, per view averaged, then over the V views:
 *   L = (1/V) sum_v [ (1 - lambda) L1_v + lambda (1 - SSIM_v) + gamma (1/M_v) sum_j H_j ].
 * The paper does not define D-SSIM; it is 1 - SSIM with the SSIM of 3DGS:
 * an 11x11 Gaussian window of sigma 1.5 (normalised), zero padding outside
 * the image, C1 = 0.01^2, C2 = 0.03^2, mean over the view's pixels and
 * channels.  lambda in [0, 1] (0 gives gs_loss_l1_entropy; 3DGS uses 0.2).
 * Writes loss_dev, dL_dimage (the L1 and D-SSIM gradients) and dL_dentropy
 * like gs_loss_l1_entropy.  workspace: device,
 * gs_loss_base_workspace_size(cams, V) bytes (about 60 B per pixel). */
int gs_loss_base(const float* image, const float* target, const float* entropy,
                 const gs_camera* cams_host, int V, float lambda, float gamma, double* loss_dev,
                 float* dL_dimage, float* dL_dentropy, void* workspace, size_t workspace_bytes,
                 gs_stream stream);

/* Reverse-order adjoint of gs_render_fwd and gs_preprocess (Sec. 4.4 and
 * Suppl. B-C).  Per pixel, from its last blended entry back to the first:
 * T_i = T_{i+1} / (1 - alpha_i), the colour part of dL/dalpha_i, and the
 * entropy part (-ln w_i - 1) T_i + R_{i+1} / (1 - alpha_i) carried by
 * Algorithm 1's running R; then alpha -> sigma, exponent -> conic, 2D mean
 * (Suppl. C), colour; then through the projection to the parameters.
 *   dL_dimage [P][3], dL_dentropy [P] (may be NULL: no entropy term),
 *   final_T, last_idx: from gs_render_fwd.  Parameters as in gs_preprocess.
 *   grad2d [V*N][12] device scratch/output (zeroed by the call): per row,
 *   summed over the pixels where the row is blended, the moments
 *   dd dx, dd dy, dd dx^2, dd dx dy, dd dy^2, dd (dd = dL/dalpha alpha where
 *   alpha is below its clamp, 0 where clamped; dx, dy = pixel centre minus
 *   the 2D mean), then dL/d(r, g, b) and 3 floats of scratch (the list of
 *   Gaussians some view sees, for the projection adjoint).  From these,
 *   dL/dsigma = dd-sum / sigma, dL/dconic = -(1/2) sum dd d d^T and
 *   dL/dmean2d = conic (dd dx-sum, dd dy-sum).
 *   g_* : device, shapes of the parameters (g_sh in prm->sh_layout), overwritten.
 * Part of the work (the zeroing of g_*, the list of Gaussians some view sees)
 * runs on a second stream of the library's own, forked from `stream` by an
 * event and joined back before the projection adjoint, so every result is
 * ordered on `stream` as usual and a stream capture records that work as a
 * parallel branch; the second stream is created by the first call on a
 * device made outside a stream capture (until then the call uses `stream`
 * alone).  Calls from several host threads are serialised while they
 * enqueue. */
int gs_render_bwd(const gs_proj* proj, int N, const gs_camera* cams_host, int V,
                  const gs_params* prm, const unsigned* sorted_vals, const unsigned* tile_ranges,
                  const float* final_T, const unsigned* last_idx, const float* dL_dimage,
                  const float* dL_dentropy, const float* means, const float* log_scales,
                  const float* quats, const float* opacity_logits, const float* sh,
                  float* grad2d, float* g_means, float* g_log_scales, float* g_quats,
                  float* g_opacity_logits, float* g_sh, const gs_launch* opt, gs_stream stream);

/* The 2D gradients of Suppl. C per (view, Gaussian) row, from the moment
 * rows gs_render_bwd leaves in grad2d (reading c10: the conic is stored as
 * (a, b, c) with d = -1/2 (a dx^2 + 2 b dx dy + c dy^2), so b's gradient
 * counts both off-diagonal entries of the symmetric matrix):
 *   out[row][0..1] = dL/d(mean2d x, y) = K (sum dd dx, sum dd dy)
 *   out[row][2..4] = dL/d(a, b, c) = (-sum dd dx^2 / 2, -sum dd dx dy, -sum dd dy^2 / 2)
 *   out[row][5]    = dL/dsigma (opacity after the sigmoid) = sum dd / sigma
 *   out[row][6..8] = dL/d(r, g, b) of the clamped colour
 * with dd = dL/dalpha alpha where alpha is below its clamp, (dx, dy) = pixel
 * centre minus 2D mean, K the conic taken from the render record (so in the
 * record's staging precision).  Rows of culled or unseen Gaussians get zeros.
 *   proj: the gs_preprocess output of the same call sequence (records and
 *   tiles_touched are read); grad2d [V*N][12] from gs_render_bwd, 16-B
 *   aligned; out [V*N][9] device, overwritten. */
int gs_grad2d_attributes(const gs_proj* proj, int N, int V, const gs_params* prm,
                         const float* grad2d, float* out, gs_stream stream);

/* Scale reset (Sec. 4.2): s <- zeta s for every Gaussian, i.e.
 * log_scales[i] += ln(zeta) in place, n = 3N floats.  0 < zeta < 1, else
 * GS_ERR_INVALID_ARG.  Optimiser state is not touched. */
int gs_scale_reset(float* log_scales, long long n, float zeta, gs_stream stream);

/* Tile work queue for the batched launch: the global tile ids ordered by
 * list length (end - start), longest first, ties by tile id.
 *   tile_ranges [2*total_tiles] device in; tile_order [total_tiles] device out;
 *   workspace: gs_tile_queue_workspace_size(total_tiles) bytes. */
int gs_tile_queue(const unsigned* tile_ranges, long long total_tiles, unsigned* tile_order,
                  void* workspace, size_t workspace_bytes, gs_stream stream);

/* ---------------------------------------------------------------------- */
/* Tile queue without allocation                                           */
/* ---------------------------------------------------------------------- */

/* Largest tile count gs_tile_queue_static accepts. */
#define GS_TILE_QUEUE_STATIC_MAX_TILES 65536

/* Same result as gs_tile_queue (tile ids ordered by list length, longest
 * first, ties by tile id), for callers that cannot allocate device memory:
 * code whose device memory comes from a fixed pool or arena owned by a host
 * application, code on a latency-critical thread where cudaMalloc /
 * cudaFree would synchronise the device, and code paths that must not
 * allocate at all.  The paper has no counterpart; this is a library
 * convenience.
 *
 * Instead of a caller-provided workspace it uses a scratch array in device
 * global memory that the library declares at file scope (about 1.35 MB,
 * enough for GS_TILE_QUEUE_STATIC_MAX_TILES tiles); every GPU that loads
 * the library holds that memory until the process exits.  The call itself
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine).
 *   tile_ranges [2*total_tiles] device in; tile_order [total_tiles] device out.
 *   total_tiles > GS_TILE_QUEUE_STATIC_MAX_TILES: GS_ERR_INVALID_ARG, with the
 *   limit in gs_last_error_string(), before anything is enqueued.
 * The first call on a device looks up the scratch array's device address on
 * the current device (cudaGetSymbolAddress) and caches it with the id of
 * the current CUDA context; a call in another context of that device (after
 * cudaDeviceReset, say) looks it up again.  Make the first call in a context
 * before any stream capture in it.
 * All calls share the one array and it keeps the last call's contents (no
 * part needs to start at zero: a call writes every word before reading it).
 * Calls whose work overlaps on the GPU (different streams without ordering,
 * or different host threads) race on the array: order them on one stream or
 * with events. */
int gs_tile_queue_static(const unsigned* tile_ranges, long long total_tiles, unsigned* tile_order,
                         gs_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* GS_H */
