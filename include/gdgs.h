/*
 * gdgs.h — C ABI of the GDGS view-synthesis path on one GPU (sm_103a).
 *
 * The path follows the render steps of the paper's Algorithm 1 (Sec. 2.2):
 *   1. project 3D Gaussians whose attribute is an image gradient (gx, gy per
 *      channel): Sigma = R S S^T R^T (Eq. 3dgs / Eq. gdgs) and
 *      Sigma2D = J W Sigma W^T J^T (Eq. sig2d, Sec. 2.2 "Projection");
 *   2. alpha-composite them front to back in view-depth order into per-channel
 *      gradient maps (Eq. color applied to the gradient attribute, Eq. gdgs2d),
 *      touching only the 16x16 tiles that some splat reaches (the field is
 *      sparse, Sec. 2.2);
 *   3. take the divergence (the Laplacian field, Sec. 1.5) and solve the Neumann
 *      Poisson problem Delta c = rho (Eq. p2d) with a linear-complexity multigrid
 *      solver (Sec. 2.1, Sec. 2.2 "Poisson Equation"), fixing the constant the
 *      Neumann problem leaves free ("with possible constant difference", Sec. 2.1)
 *      with a supplied per-channel mean.
 *
 * Conventions shared by every call
 *  - Pointers named "device" must point to GPU memory on the current device;
 *    "host" pointers to CPU memory. The library never allocates device memory:
 *    all scratch comes from one caller-owned workspace of gdgs_workspace_size()
 *    bytes (device, 256-byte aligned). The one exception is the fixed 32 MiB
 *    array that gdgs_poisson_reconstruct_static uses instead of a workspace,
 *    reserved on each GPU when the library is loaded. Host structs are read
 *    during the call only.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Every call only enqueues work on it and returns; results are ready
 *    when the stream is synchronised.
 *  - Return value: a status code below. Argument errors (null pointers, sizes out
 *    of range, misaligned buffers, workspace too small) are found on the host and
 *    returned at once, with nothing enqueued. Errors found on the GPU (capacity
 *    exceeded, non-finite input, no convergence) are written to a status word in
 *    the workspace and returned by gdgs_sync_status(). No call traps the device
 *    or throws across the ABI.
 *  - Calls that share a workspace must not overlap on the GPU (enqueue them on one
 *    stream, or synchronise between them).
 *  - Layouts are row-major, C-contiguous float32 unless stated.
 */
#ifndef GDGS_H
#define GDGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GDGS_API __attribute__((visibility("default")))
#else
#define GDGS_API
#endif

#define GDGS_ABI_VERSION 2
#define GDGS_TILE 16        /* raster tile edge in pixels */
#define GDGS_MAX_CHANNELS 4

/* Status codes. */
enum {
  GDGS_OK = 0,
  GDGS_ERR_INVALID_ARG = 1,  /* bad pointer, size, option or alignment (host) */
  GDGS_ERR_WORKSPACE = 2,    /* workspace null, misaligned or too small (host) */
  GDGS_ERR_CUDA = 3,         /* a CUDA launch or copy failed (host) */
  GDGS_ERR_NO_CONVERGE = 4,  /* multigrid hit max_cycles above rtol (device) */
  GDGS_ERR_NONFINITE = 5,    /* NaN/Inf in an input Gaussian or map (device) */
  GDGS_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up (device) */
  GDGS_ERR_CAPACITY = 7      /* more (tile, splat) pairs than the pair buffer holds (device) */
};

/* What each Gaussian carries (gdgs_gaussians.attribute). */
enum {
  GDGS_ATTR_GRADIENT = 0,  /* (gx, gy) per channel; the image is recovered from div g */
  GDGS_ATTR_LAPLACIAN = 1  /* one value per channel: the Laplacian field itself
                              (Eq. gdgs, the paper-literal form) */
};

/* Gaussians, structure of arrays, all device pointers (Sec. 1.2, Eq. 3dgs):
 *   mean    [n][3]  centre tau_k in world space
 *   scale   [n][3]  linear per-axis scale, S = diag(scale)
 *   quat    [n][4]  rotation (w, x, y, z); normalised by the library
 *   opacity [n]     alpha_k
 *   grad    [n][channels][K]  attribute per channel: K = 2 (gx, gy) for
 *                   GDGS_ATTR_GRADIENT, K = 1 (A_k of Eq. gdgs) for GDGS_ATTR_LAPLACIAN
 * Every array must be 4-byte aligned; n >= 0, 1 <= channels <= 4. */
typedef struct gdgs_gaussians {
  int64_t n;
  int32_t channels;
  int32_t attribute;  /* GDGS_ATTR_GRADIENT (0) or GDGS_ATTR_LAPLACIAN (1) */
  const float *mean;
  const float *scale;
  const float *quat;
  const float *opacity;
  const float *grad;
} gdgs_gaussians;

/* Pinhole camera (host struct, by value semantics). OpenCV axes: x right, y down,
 * z forward. world_to_cam is the row-major 3x4 matrix [W | t] whose 3x3 part is
 * the W of Eq. sig2d. Pixel (row i, column j) has its centre at x = j + 0.5,
 * y = i + 0.5. Gaussians with camera depth <= near_plane are culled.
 * Depth precision: the camera depth t_z = W[2] . mean + t[2] is evaluated in
 * float-float arithmetic (about 44 bits). The near cull compares it with
 * near_plane, and the front-to-back order ("sorted from the view direction",
 * Eq. color) follows it to 2^-31 relative: two Gaussians whose depths differ by
 * more than that are composited in exact depth order; closer ones may come in
 * either order; equal depths computed from equal terms keep ascending index. */
typedef struct gdgs_camera {
  float world_to_cam[12];
  float fx, fy, cx, cy;
  float near_plane;
  int32_t width, height;
} gdgs_camera;

/* Rasteriser options (the paper fixes none of them; defaults below).
 *   alpha_min  splats with alpha*G below this are skipped          (1/255)
 *   alpha_max  alpha*G is clamped to this                          (0.99)
 *   t_min      a pixel stops once its transmittance falls below    (1e-4)
 *   dilation   added to the diagonal of Sigma2D, in pixels^2       (0.3)
 *   exp_coef   G = exp(-exp_coef d^T Sigma2D^-1 d); the paper's kernel has
 *              no 1/2 (Eq. 3dgs), so the default is                (1.0)
 *   pairs_per_gaussian  capacity of the (tile, splat) pair buffer as a
 *              multiple of n; overflow sets GDGS_ERR_CAPACITY      (16) */
typedef struct gdgs_raster_opts {
  float alpha_min;
  float alpha_max;
  float t_min;
  float dilation;
  float exp_coef;
  int32_t pairs_per_gaussian;
} gdgs_raster_opts;

/* Multigrid options (Sec. 2.1 lists multigrid among the linear-complexity
 * solvers; the paper fixes no parameters).
 *   nu1, nu2        red-black Gauss-Seidel sweeps before / after the coarse
 *                   correction, each in 1..3                         (2, 1)
 *   max_cycles      upper bound on V-cycles, 1..64                   (30)
 *   rtol            stop when ||rho - L u||_2 <= rtol ||rho||_2       (1e-6)
 *   coarse_max_dim  coarsen until both grid sides are <= this; the
 *                   coarsest grid is solved directly in FP64, 2..16   (8)
 *   rho_threshold   t of the hard threshold T(x) = x if |x| >= t else 0
 *                   applied to the Laplacian field rho before the solve
 *                   (Eq. thresh); 0 keeps rho as it is                 (0)
 *   omega           over-relaxation of the red-black Gauss-Seidel smoother,
 *                   u <- u + omega (u_GS - u), in [0.5, 1.9]; it changes how
 *                   fast the cycles converge, not what they converge to (1.2)
 *   storage         number format of the multigrid corrections and coarse
 *                   right-hand sides in memory: GDGS_STORAGE_F32, _BF16 or
 *                   _F16 (arithmetic is FP32 throughout; the residual r_k,
 *                   the iterate (float-float) and the coarse solve (FP64)
 *                   keep their precision, so the cycles are an iterative
 *                   refinement that reaches rtol in every format)  (F32) */
typedef struct gdgs_solver_opts {
  int32_t nu1;
  int32_t nu2;
  int32_t max_cycles;
  float rtol;
  int32_t coarse_max_dim;
  float rho_threshold;
  float omega;
  int32_t storage;
} gdgs_solver_opts;

enum { GDGS_STORAGE_F32 = 0, GDGS_STORAGE_BF16 = 1, GDGS_STORAGE_F16 = 2 };

/* Filled by gdgs_sync_status() from the workspace after the stream has drained. */
typedef struct gdgs_solve_stats {
  int32_t status;          /* device status word (a GDGS_* code) */
  int32_t cycles;          /* V-cycles run by the last solve */
  double rel_residual;     /* ||rho - L u||_2 / ||rho||_2 of the returned solution */
  double rho_norm;         /* ||rho||_2 over all channels */
  double mean_set[GDGS_MAX_CHANNELS]; /* per-channel mean that was imposed */
  int64_t n_pairs;         /* (tile, splat) pairs emitted by the last raster */
  int32_t n_active_tiles;  /* tiles with at least one splat */
  int32_t n_visible;       /* Gaussians that survived the culls */
} gdgs_solve_stats;

/* Projection outputs (all device pointers, each may be NULL to skip it). */
typedef struct gdgs_projected {
  float *mean2d;    /* [n][2] projected centre in pixels (x, y) */
  float *cov2d;     /* [n][3] Sigma2D incl. dilation: xx, xy, yy */
  float *depth;     /* [n] camera-space z rounded to float (0 if culled) */
  int32_t *rect;    /* [n][4] touched tiles x0, y0, x1, y1 (half open; empty if culled) */
} gdgs_projected;

/* ABI version of the loaded library (GDGS_ABI_VERSION at build time). */
GDGS_API int gdgs_abi_version(void);

/* Fill an options struct with the defaults documented above. */
GDGS_API void gdgs_default_raster_opts(gdgs_raster_opts *opts);
GDGS_API void gdgs_default_solver_opts(gdgs_solver_opts *opts);

/* Human-readable name of a status code; never NULL, static storage. */
GDGS_API const char *gdgs_status_string(int status);

/* Bytes of device workspace needed by any call below for n Gaussians, `channels`
 * channels and a width x height image (n = 0 sizes a Poisson-only workspace).
 * NULL options mean the defaults. Returns 0 if an argument is out of range. */
GDGS_API size_t gdgs_workspace_size(int64_t n, int32_t channels, int32_t width, int32_t height,
                           const gdgs_raster_opts *ropts, const gdgs_solver_opts *sopts);

/* Step 1 (Eq. 3dgs, Eq. sig2d): project the Gaussians. Writes the internal splat
 * records into the workspace and, for each non-NULL field of `out`, a copy of
 * that quantity. */
GDGS_API int gdgs_project(const gdgs_gaussians *g, const gdgs_camera *cam,
                 const gdgs_raster_opts *ropts, const gdgs_projected *out,
                 void *ws, size_t ws_bytes, void *stream);

/* Steps 1-2 (Eq. gdgs2d): project, bin the splats into 16x16 tiles, sort each
 * tile's splats front to back, and composite the attribute into
 *   grad_maps  device [channels][K][height][width]: K = 2 (component 0 = gx,
 *              1 = gy) for gradient Gaussians, K = 1 (the field rho) for
 *              Laplacian Gaussians.
 * tile_mask  device [ceil(height/16)][ceil(width/16)] bytes, or NULL.
 *   With a mask, only tiles some splat reaches are written and the mask says
 *   which (1) — other tiles of grad_maps are left untouched and mean zero.
 *   Without a mask every pixel is written (zeros where no splat reaches).
 * grad_maps must be 16-byte aligned. */
GDGS_API int gdgs_render_gradients(const gdgs_gaussians *g, const gdgs_camera *cam,
                          const gdgs_raster_opts *ropts, float *grad_maps,
                          uint8_t *tile_mask, void *ws, size_t ws_bytes, void *stream);

/* Step 3 (Eq. p2d): rho = div(grad_maps) with zero flux through the image border,
 * then solve the Neumann problem L u = rho by multigrid V-cycles and return
 *   image  device [channels][height][width], mean(image[c]) = mean[c].
 * grad_maps  device [channels][2][height][width]; tile_mask as written by
 *            gdgs_render_gradients (tiles with mask 0 are read as zero), or NULL.
 * mean       host [channels].
 * image and grad_maps must be 16-byte aligned and must not overlap. */
GDGS_API int gdgs_poisson_reconstruct(const float *grad_maps, const uint8_t *tile_mask,
                             int32_t channels, int32_t height, int32_t width,
                             const float *mean, const gdgs_solver_opts *sopts,
                             float *image, void *ws, size_t ws_bytes, void *stream);

/* Step 3 for a Laplacian field given directly (Eq. p2d with rho = the composite
 * of Laplacian Gaussians, Eq. gdgs / Eq. gdgs2d): T(rho) per the solver options,
 * then the Neumann solve as in gdgs_poisson_reconstruct.
 * rho  device [channels][height][width]; tile_mask as written by
 *      gdgs_render_gradients (tiles with mask 0 are read as zero), or NULL. */
GDGS_API int gdgs_poisson_reconstruct_rho(const float *rho, const uint8_t *tile_mask,
                                          int32_t channels, int32_t height, int32_t width,
                                          const float *mean, const gdgs_solver_opts *sopts,
                                          float *image, void *ws, size_t ws_bytes, void *stream);

/* Steps 1-3 of Algorithm 1's render path in one call: project, rasterise the
 * sparse attribute maps (kept inside the workspace), the divergence (gradient
 * Gaussians) or the field itself (Laplacian Gaussians), and the Poisson solve into
 * image (device [channels][height][width], 16-byte aligned). */
GDGS_API int gdgs_render_view(const gdgs_gaussians *g, const gdgs_camera *cam, const float *mean,
                     const gdgs_raster_opts *ropts, const gdgs_solver_opts *sopts,
                     float *image, void *ws, size_t ws_bytes, void *stream);

/* gdgs_render_view with the camera read from device memory when the kernels run
 * (no paper counterpart: a serving variant). `cam` (host) gives the image size the
 * workspace is planned for; its pose and intrinsics are ignored. `cam_dev` (device,
 * one gdgs_camera, 4-byte aligned) supplies world_to_cam, fx, fy, cx, cy and
 * near_plane; its width and height must equal cam's. Because no camera value is
 * baked into the launches, a CUDA graph captured from one call (the multigrid
 * cycle loop is then recorded as a conditional WHILE node) replays correctly for
 * any camera written to cam_dev before the replay. cam_dev's values cannot be checked
 * on the host: a near_plane below 0 (or NaN) is read as 0. Errors as gdgs_render_view. */
GDGS_API int gdgs_render_view_devcam(const gdgs_gaussians *g, const gdgs_camera *cam,
                                     const gdgs_camera *cam_dev, const float *mean,
                                     const gdgs_raster_opts *ropts,
                                     const gdgs_solver_opts *sopts, float *image, void *ws,
                                     size_t ws_bytes, void *stream);

/* Gradients of a loss with respect to the Gaussians (device arrays, the layouts of
 * gdgs_gaussians; overwritten). */
typedef struct gdgs_gaussian_grads {
  float *d_mean;     /* [n][3] */
  float *d_scale;    /* [n][3] */
  float *d_quat;     /* [n][4] */
  float *d_opacity;  /* [n]    */
  float *d_attr;     /* [n][channels][2] (gradient) or [n][channels] (Laplacian) */
} gdgs_gaussian_grads;

/* Backward of gdgs_render_view (Algorithm 1's render steps differentiated; the
 * training loop itself is not part of this library): given d_image = d loss /
 * d image (device [channels][height][width]), write d loss / d (mean, scale,
 * quat, opacity, attribute) into `grads`.
 *   ws: the workspace of the gdgs_render_view call of the same (g, cam, ropts,
 *   sopts) whose image is being differentiated, not used by any call since (its
 *   projected splats, sorted pairs, tile lists and rho are read; its gradient-map
 *   region is reused).
 *   ws_adj: a second workspace of gdgs_workspace_size(0, channels, width,
 *   height, NULL, sopts) bytes for the adjoint solve (L is symmetric: the same
 *   zero-mean Neumann solve, applied to d_image); gdgs_sync_status(ws_adj, ...)
 *   reports its convergence.
 * The alpha tests, the T_min stop, culls, the depth order and the threshold's
 * decision are piecewise constant and contribute no derivative. Errors as
 * gdgs_render_view; GDGS_ERR_WORKSPACE if either workspace is too small. */
GDGS_API int gdgs_render_view_backward(const gdgs_gaussians *g, const gdgs_camera *cam,
                                       const gdgs_raster_opts *ropts,
                                       const gdgs_solver_opts *sopts, const float *d_image,
                                       const gdgs_gaussian_grads *grads, void *ws,
                                       size_t ws_bytes, void *ws_adj, size_t ws_adj_bytes,
                                       void *stream);

/* Wait for `stream`, then read the device status word and statistics of the last
 * call that used `ws`. `stats` (host) may be NULL. Returns the device status (or
 * GDGS_ERR_CUDA if the synchronisation itself failed). */
GDGS_API int gdgs_sync_status(const void *ws, gdgs_solve_stats *stats, void *stream);

/* Step 3 without a caller workspace (the paper has no counterpart: this is a
 * deployment variant). For callers that cannot allocate device memory where they
 * need the solve - inside a CUDA stream capture, in a plug-in whose host
 * application owns the device allocator, or in a loop that forbids allocation
 * after start-up - the scratch lives in a fixed 32 MiB __device__ array of the
 * library, held on every GPU that loads it until the process exits.
 *   Arguments as for gdgs_poisson_reconstruct; `stats` (host, nullable): when
 *   given, the call waits for `stream` and fills it (and returns the device
 *   status), otherwise it only enqueues. Waiting is not allowed while `stream`
 *   is being captured: there `stats` must be NULL (a non-NULL `stats` returns
 *   GDGS_ERR_INVALID_ARG with nothing enqueued), and the status of the replayed
 *   solve is read afterwards with gdgs_poisson_static_status().
 *   Sizes whose workspace (gdgs_workspace_size(0, ...)) exceeds 32 MiB are
 *   rejected with GDGS_ERR_WORKSPACE before anything is enqueued; about
 *   640 x 480 x 3 or 1024 x 1024 x 1 fit.
 *   No cudaMalloc, cudaFree or other allocating call is made for the scratch.
 *   The first call on a device looks the array's address up
 *   (cudaGetSymbolAddress) and should come before any stream capture on that
 *   device. Outside a capture, the first call for each image size and solver
 *   option set also builds and instantiates the CUDA graph of its cycle loop
 *   (driver objects, created once; GDGS_GRAPHS=0 in the environment runs the
 *   cycles as plain launches and creates none).
 *   All calls share the one array, which keeps the last call's contents (what
 *   must start at zero is cleared by each call); calls that overlap on the GPU
 *   race and must be ordered by the caller (one stream, or synchronisation). */
GDGS_API int gdgs_poisson_reconstruct_static(const float *grad_maps, const uint8_t *tile_mask,
                                             int32_t channels, int32_t height, int32_t width,
                                             const float *mean, const gdgs_solver_opts *sopts,
                                             float *image, gdgs_solve_stats *stats, void *stream);

/* Wait for `stream`, then read the device status word and statistics of the last
 * gdgs_poisson_reconstruct_static solve on the current device (for example one
 * replayed from a captured graph). `stats` (host) may be NULL. Returns the device
 * status, or GDGS_ERR_CUDA if the synchronisation failed. */
GDGS_API int gdgs_poisson_static_status(gdgs_solve_stats *stats, void *stream);

/* ---- diagnostics (host side; not needed on the render path) ---------------- */

/* Per-kernel timing record filled by gdgs_profile_end(). */
typedef struct gdgs_kernel_time {
  char name[48];     /* kernel name, e.g. "raster", "mg0_down" */
  int64_t launches;  /* launches recorded while profiling */
  double total_ms;   /* summed CUDA-event time between each launch's start and end events */
} gdgs_kernel_time;

/* Number of kernels this library has enqueued in this process, all streams. */
GDGS_API uint64_t gdgs_kernel_launch_count(void);

/* Start recording a CUDA event pair around every kernel launched by any later
 * call, on that call's stream. Adds host work per launch; not for stream capture. */
GDGS_API int gdgs_profile_begin(void);

/* Stop recording, wait for the recorded events and aggregate them by kernel
 * name into out[0 .. *n_entries) (at most max_entries; host memory). */
GDGS_API int gdgs_profile_end(gdgs_kernel_time *out, int32_t max_entries, int32_t *n_entries);

#ifdef __cplusplus
}
#endif

#endif /* GDGS_H */
