// C ABI of libgdgs (see include/gdgs.h): argument checks, workspace layout and
// the launch sequence of the render path (Algorithm 1's render steps, Sec. 2.2).
#include <math.h>
#include <string.h>

#include "gdgs_internal.cuh"

namespace gdgs {

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Carver {
  size_t cur = 0;
  size_t take(size_t bytes) {
    const size_t o = cur;
    cur = align_up(cur + bytes);
    return o;
  }
};

LevelGeom level_geom(int H0, int W0, int l) {
  LevelGeom g{};
  const long long s = 1ll << l;
  g.H = (int)((H0 + s - 1) / s);
  g.W = (int)((W0 + s - 1) / s);
  g.shift = l;
  g.H0 = H0;
  g.W0 = W0;
  g.lastx = (float)(W0 - (long long)(g.W - 1) * s) / (float)s;
  g.lasty = (float)(H0 - (long long)(g.H - 1) * s) / (float)s;
  g.ex = 2.f / (1.f + g.lastx);
  g.ey = 2.f / (1.f + g.lasty);
  g.plane = (long long)g.H * g.W;
  return g;
}

bool raster_opts_ok(const gdgs_raster_opts &o) {
  return isfinite(o.alpha_min) && isfinite(o.alpha_max) && isfinite(o.t_min) &&
         isfinite(o.dilation) && isfinite(o.exp_coef) && o.alpha_min > 0.f &&
         o.alpha_min < 1.f && o.alpha_max >= o.alpha_min && o.alpha_max < 1.f &&
         o.t_min >= 0.f && o.t_min < 1.f && o.dilation >= 0.f && o.exp_coef > 0.f &&
         o.pairs_per_gaussian >= 1 && o.pairs_per_gaussian <= 1024;
}

bool solver_opts_ok(const gdgs_solver_opts &o) {
  return o.nu1 >= 1 && o.nu1 <= 3 && o.nu2 >= 1 && o.nu2 <= 3 && o.max_cycles >= 1 &&
         o.max_cycles <= kMaxCycles && isfinite(o.rtol) && o.rtol >= 0.f &&
         o.coarse_max_dim >= 2 && o.coarse_max_dim <= 16 && isfinite(o.rho_threshold) &&
         o.rho_threshold >= 0.f && o.omega >= 0.5f && o.omega <= 1.9f && o.storage >= 0 &&
         o.storage <= 2;
}

}  // namespace

bool make_plan(int64_t n, int C, int W, int H, const gdgs_raster_opts &ro,
               const gdgs_solver_opts &so, Plan *p) {
  if (n < 0 || C < 1 || C > GDGS_MAX_CHANNELS || W < 1 || H < 1) return false;
  if ((int64_t)W * H > (1ll << 30)) return false;
  const int tx = (W + kTile - 1) / kTile, ty = (H + kTile - 1) / kTile;
  if (tx > 65535 || ty > 65535) return false;
  if (!raster_opts_ok(ro) || !solver_opts_ok(so)) return false;
  memset(p, 0, sizeof(*p));
  p->n = n;
  p->C = C;
  p->W = W;
  p->H = H;
  p->tiles_x = tx;
  p->tiles_y = ty;
  p->T = tx * ty;
  const int64_t cap = n * (int64_t)ro.pairs_per_gaussian;
  if (cap > 0x7fffffffll) return false;
  p->pair_cap = (unsigned)cap;
  const int64_t dblk = (n + kRadixBlockSmall - 1) / kRadixBlockSmall;  // depth sort
  const int64_t pblk = (cap + kRadixBlock - 1) / kRadixBlock;           // pair sort
  p->radix_blocks_max = (int)(dblk > pblk ? dblk : pblk);

  // multigrid levels: coarsen until both sides <= coarse_max_dim, at least 2 levels
  int levels = 1;
  while (true) {
    const LevelGeom g = level_geom(H, W, levels - 1);
    if (levels >= 2 && g.H <= so.coarse_max_dim && g.W <= so.coarse_max_dim) break;
    if (levels >= kMaxLevels) return false;
    ++levels;
  }
  p->levels = levels;
  for (int l = 0; l < levels; ++l) p->lv[l] = level_geom(H, W, l);
  p->nc = p->lv[levels - 1].H * p->lv[levels - 1].W;

  Carver cv;
  p->off_ctrl = cv.take(sizeof(Ctrl));
  // the cached coarse factor sits at a fixed offset with room for the largest
  // coarsest grid, so workspaces laid out for other sizes never overwrite it
  p->off_coarse = cv.take(kCoarseTagBytes + sizeof(double) * (size_t)kMaxCoarse * kMaxCoarse);
  p->off_sub = cv.take(sizeof(Ctrl) * (size_t)C);
  if (n > 0) {
    p->off_smean = cv.take(16 * (size_t)n);
    p->off_sconic = cv.take(16 * (size_t)n);
    p->off_rect = cv.take(8 * (size_t)n);
    for (int b = 0; b < 2; ++b) {
      p->off_dkey[b] = cv.take(4 * (size_t)n);
      p->off_dval[b] = cv.take(4 * (size_t)n);
      p->off_pkey[b] = cv.take(4 * (size_t)p->pair_cap);
      p->off_pval[b] = cv.take(4 * (size_t)p->pair_cap);
    }
    p->off_dlo = cv.take(4 * (size_t)n);
    p->off_hist = cv.take(4 * 256 * (size_t)(p->radix_blocks_max + 1));
    p->off_blocksum = cv.take(8 * (size_t)((n + kBinBlock - 1) / kBinBlock + 2));
    p->off_gtiles = cv.take(4 * (size_t)n);
    p->off_maps = cv.take(4 * (size_t)C * 2 * W * H);
    p->off_dsplat = cv.take(24 * (size_t)n);
  }
  p->off_range = cv.take(8 * (size_t)p->T);
  p->off_active = cv.take(4 * (size_t)p->T);
  p->off_mask = cv.take((size_t)p->T);
  const size_t plane0 = (size_t)W * H * C * sizeof(float);
  p->off_rho = cv.take(plane0);
  p->off_uhi = cv.take(plane0);
  p->off_ulo = cv.take(plane0);
  p->off_e0 = cv.take(plane0);
  p->off_r[0] = cv.take(plane0);
  p->off_r[1] = cv.take(plane0);
  for (int l = 1; l < levels; ++l) {
    const size_t b = sizeof(float) * (size_t)C * p->lv[l].plane;
    p->off_lu[l] = cv.take(b);
    p->off_lf[l] = cv.take(b);
    p->off_luo[l] = cv.take(b);
  }
  p->total = cv.cur;
  return true;
}

}  // namespace gdgs

using namespace gdgs;

namespace {

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

gdgs_raster_opts ropts_or_default(const gdgs_raster_opts *o) {
  gdgs_raster_opts r;
  if (o) return *o;
  gdgs_default_raster_opts(&r);
  return r;
}

gdgs_solver_opts sopts_or_default(const gdgs_solver_opts *o) {
  gdgs_solver_opts r;
  if (o) return *o;
  gdgs_default_solver_opts(&r);
  return r;
}

int attr_floats(const gdgs_gaussians *g) {
  return g->attribute == GDGS_ATTR_LAPLACIAN ? g->channels : 2 * g->channels;
}

int check_gaussians(const gdgs_gaussians *g) {
  if (!g || g->n < 0 || g->channels < 1 || g->channels > GDGS_MAX_CHANNELS) return GDGS_ERR_INVALID_ARG;
  if (g->attribute != GDGS_ATTR_GRADIENT && g->attribute != GDGS_ATTR_LAPLACIAN)
    return GDGS_ERR_INVALID_ARG;
  if (g->n > 0) {
    const void *ptrs[5] = {g->mean, g->scale, g->quat, g->opacity, g->grad};
    for (const void *q : ptrs)
      if (!q || !aligned(q, 4)) return GDGS_ERR_INVALID_ARG;
  }
  return GDGS_OK;
}

int check_camera(const gdgs_camera *c) {
  if (!c || c->width < 1 || c->height < 1) return GDGS_ERR_INVALID_ARG;
  for (int i = 0; i < 12; ++i)
    if (!isfinite(c->world_to_cam[i])) return GDGS_ERR_INVALID_ARG;
  if (!isfinite(c->fx) || !isfinite(c->fy) || !isfinite(c->cx) || !isfinite(c->cy) ||
      !isfinite(c->near_plane) || c->fx == 0.f || c->fy == 0.f || c->near_plane < 0.f)
    return GDGS_ERR_INVALID_ARG;
  return GDGS_OK;
}

int check_ws(void *ws, size_t ws_bytes, const Plan &p) {
  if (!ws || !aligned(ws, kAlign) || ws_bytes < p.total) return GDGS_ERR_WORKSPACE;
  return GDGS_OK;
}

ProjectArgs project_args(const gdgs_gaussians *g, const gdgs_camera *cam,
                         const gdgs_raster_opts &ro, const Plan &p, char *ws) {
  ProjectArgs a{};
  a.mean = g->mean;
  a.scale = g->scale;
  a.quat = g->quat;
  a.opacity = g->opacity;
  a.grad = g->grad;
  a.n = g->n;
  a.C = g->channels;
  a.Q = attr_floats(g);
  memcpy(a.w2c, cam->world_to_cam, sizeof(a.w2c));
  a.fx = cam->fx;
  a.fy = cam->fy;
  a.cx = cam->cx;
  a.cy = cam->cy;
  a.znear = cam->near_plane;
  a.W = cam->width;
  a.H = cam->height;
  a.tiles_x = p.tiles_x;
  a.tiles_y = p.tiles_y;
  a.alpha_min = ro.alpha_min;
  a.dilation = ro.dilation;
  a.exp_coef = ro.exp_coef;
  a.smean = (float4 *)(ws + p.off_smean);
  a.sconic = (float4 *)(ws + p.off_sconic);
  a.key = (uint32_t *)(ws + p.off_dkey[0]);  // sorted in place by the depth sort
  a.key_lo = (uint32_t *)(ws + p.off_dlo);
  a.rect = (uint2 *)(ws + p.off_rect);
  a.ctrl = (Ctrl *)(ws + p.off_ctrl);
  return a;
}

int to_status(cudaError_t e) { return e == cudaSuccess ? GDGS_OK : GDGS_ERR_CUDA; }

// Steps 1-2 into `maps` (and `mask` when use_mask).
cudaError_t raster_path(const gdgs_gaussians *g, const gdgs_camera *cam,
                        const gdgs_raster_opts &ro, const Plan &p, char *ws, float *maps,
                        uint8_t *mask, bool use_mask, cudaStream_t st,
                        const gdgs_camera *cam_dev = nullptr) {
  Ctrl *ctrl = (Ctrl *)(ws + p.off_ctrl);
  ProjectArgs pa = project_args(g, cam, ro, p, ws);
  pa.cam_dev = cam_dev;
  cudaError_t e = launch_project(pa, st);
  if (e != cudaSuccess) return e;
  uint32_t *hist = (uint32_t *)(ws + p.off_hist);
  uint2 *range = (uint2 *)(ws + p.off_range);
  uint32_t *active = (uint32_t *)(ws + p.off_active);
  uint8_t *mk = mask ? mask : (uint8_t *)(ws + p.off_mask);
  const uint32_t *pval_sorted = (const uint32_t *)(ws + p.off_pval[0]);
  if (g->n > 0) {
    // 1. depth order of the Gaussians (float-float depth: lo digit, then hi bits)
    uint32_t *dk0 = (uint32_t *)(ws + p.off_dkey[0]), *dv0 = (uint32_t *)(ws + p.off_dval[0]);
    uint32_t *dk1 = (uint32_t *)(ws + p.off_dkey[1]), *dv1 = (uint32_t *)(ws + p.off_dval[1]);
    const int dblocks = (int)((g->n + kRadixBlockSmall - 1) / kRadixBlockSmall);
    bool alt = false;
    e = radix_sort_pairs(dk0, dv0, dk1, dv1, true, (const uint32_t *)(ws + p.off_dlo), nullptr,
                         (unsigned)g->n, 32, hist, kRadixItemsSmall, dblocks, &alt, st);
    if (e != cudaSuccess) return e;
    const uint32_t *order = alt ? dv1 : dv0;
    // 2. emit (tile, Gaussian) pairs in depth order
    BinArgs b{};
    b.order = order;
    b.rect = (const uint2 *)(ws + p.off_rect);
    b.smean = (const float4 *)(ws + p.off_smean);
    b.sconic = (const float4 *)(ws + p.off_sconic);
    b.alpha_min = ro.alpha_min;
    b.n = g->n;
    b.tiles_x = p.tiles_x;
    b.T = p.T;
    b.pair_cap = p.pair_cap;
    b.blocksum = (unsigned long long *)(ws + p.off_blocksum);
    b.tiles = (uint32_t *)(ws + p.off_gtiles);
    b.pkey = (uint32_t *)(ws + p.off_pkey[0]);
    b.pval = (uint32_t *)(ws + p.off_pval[0]);
    b.ctrl = ctrl;
    e = launch_emit_pairs(b, st);
    if (e != cudaSuccess) return e;
    // 3. stable sort of the pairs by tile id
    int tbits = 0;
    while ((1 << tbits) < p.T) ++tbits;
    uint32_t *pk0 = (uint32_t *)(ws + p.off_pkey[0]), *pv0 = (uint32_t *)(ws + p.off_pval[0]);
    uint32_t *pk1 = (uint32_t *)(ws + p.off_pkey[1]), *pv1 = (uint32_t *)(ws + p.off_pval[1]);
    alt = false;
    const int pblocks = (int)(((int64_t)p.pair_cap + kRadixBlock - 1) / kRadixBlock);
    e = radix_sort_pairs(pk0, pv0, pk1, pv1, false, nullptr, &ctrl->n_pairs, p.pair_cap, tbits,
                         hist, kRadixItems, pblocks, &alt, st);
    if (e != cudaSuccess) return e;
    const uint32_t *pk_sorted = alt ? pk1 : pk0;
    pval_sorted = alt ? pv1 : pv0;
    // 4. tile ranges, mask and active list
    e = launch_tile_ranges(pk_sorted, ctrl, p.pair_cap, p.T, range, active, mk, st);
    if (e != cudaSuccess) return e;
  } else {
    e = cudaMemsetAsync(range, 0, 8 * (size_t)p.T, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(mk, 0, (size_t)p.T, st);
    if (e != cudaSuccess) return e;
  }
  // 5. composite
  RasterArgs r{};
  r.smean = (const float4 *)(ws + p.off_smean);
  r.sconic = (const float4 *)(ws + p.off_sconic);
  r.grad = g->grad;
  r.pval = pval_sorted;
  r.range = range;
  r.active = active;
  r.use_active = (use_mask && g->n > 0) ? 1 : 0;
  if (use_mask && g->n == 0) return cudaSuccess;  // nothing active, mask already zero
  r.Q = attr_floats(g);
  r.alpha_min = ro.alpha_min;
  r.alpha_max = ro.alpha_max;
  r.t_min = ro.t_min;
  r.W = p.W;
  r.H = p.H;
  r.tiles_x = p.tiles_x;
  r.T = p.T;
  r.maps = maps;
  r.ctrl = ctrl;
  return launch_raster(r, st);
}

}  // namespace

extern "C" {

int gdgs_abi_version(void) { return GDGS_ABI_VERSION; }

void gdgs_default_raster_opts(gdgs_raster_opts *o) {
  if (!o) return;
  o->alpha_min = 1.0f / 255.0f;
  o->alpha_max = 0.99f;
  o->t_min = 1e-4f;
  o->dilation = 0.3f;
  o->exp_coef = 1.0f;
  o->pairs_per_gaussian = 16;
}

void gdgs_default_solver_opts(gdgs_solver_opts *o) {
  if (!o) return;
  o->nu1 = 2;
  o->nu2 = 1;
  o->max_cycles = 30;
  o->rtol = 1e-6f;
  o->coarse_max_dim = 8;
  o->rho_threshold = 0.f;
  o->omega = 1.2f;
  o->storage = GDGS_STORAGE_F32;
}

const char *gdgs_status_string(int s) {
  switch (s) {
    case GDGS_OK: return "ok";
    case GDGS_ERR_INVALID_ARG: return "invalid argument";
    case GDGS_ERR_WORKSPACE: return "workspace null, misaligned or too small";
    case GDGS_ERR_CUDA: return "CUDA launch or copy failed";
    case GDGS_ERR_NO_CONVERGE: return "multigrid did not reach rtol within max_cycles";
    case GDGS_ERR_NONFINITE: return "non-finite input value";
    case GDGS_ERR_TIMEOUT: return "bounded device wait timed out";
    case GDGS_ERR_CAPACITY: return "pair buffer capacity exceeded";
    default: return "unknown status";
  }
}

size_t gdgs_workspace_size(int64_t n, int32_t channels, int32_t width, int32_t height,
                           const gdgs_raster_opts *ropts, const gdgs_solver_opts *sopts) {
  Plan p;
  if (!make_plan(n, channels, width, height, ropts_or_default(ropts), sopts_or_default(sopts), &p))
    return 0;
  return p.total;
}

int gdgs_project(const gdgs_gaussians *g, const gdgs_camera *cam, const gdgs_raster_opts *ropts,
                 const gdgs_projected *out, void *ws, size_t ws_bytes, void *stream) {
  int s;
  if ((s = check_gaussians(g)) || (s = check_camera(cam))) return s;
  const gdgs_raster_opts ro = ropts_or_default(ropts);
  const gdgs_solver_opts so = sopts_or_default(nullptr);
  Plan p;
  if (!make_plan(g->n, g->channels, cam->width, cam->height, ro, so, &p)) return GDGS_ERR_INVALID_ARG;
  if ((s = check_ws(ws, ws_bytes, p))) return s;
  cudaStream_t st = (cudaStream_t)stream;
  char *w = (char *)ws;
  cudaError_t e = cudaMemsetAsync(w + p.off_ctrl, 0, sizeof(Ctrl), st);
  if (e != cudaSuccess) return GDGS_ERR_CUDA;
  ProjectArgs a = project_args(g, cam, ro, p, w);
  if (out) {
    a.o_mean2d = out->mean2d;
    a.o_cov2d = out->cov2d;
    a.o_depth = out->depth;
    a.o_rect = out->rect;
  }
  return to_status(launch_project(a, st));
}

int gdgs_render_gradients(const gdgs_gaussians *g, const gdgs_camera *cam,
                          const gdgs_raster_opts *ropts, float *grad_maps, uint8_t *tile_mask,
                          void *ws, size_t ws_bytes, void *stream) {
  int s;
  if ((s = check_gaussians(g)) || (s = check_camera(cam))) return s;
  if (!grad_maps || !aligned(grad_maps, 16)) return GDGS_ERR_INVALID_ARG;
  const gdgs_raster_opts ro = ropts_or_default(ropts);
  const gdgs_solver_opts so = sopts_or_default(nullptr);
  Plan p;
  if (!make_plan(g->n, g->channels, cam->width, cam->height, ro, so, &p)) return GDGS_ERR_INVALID_ARG;
  if ((s = check_ws(ws, ws_bytes, p))) return s;
  cudaStream_t st = (cudaStream_t)stream;
  char *w = (char *)ws;
  if (cudaMemsetAsync(w + p.off_ctrl, 0, sizeof(Ctrl), st) != cudaSuccess) return GDGS_ERR_CUDA;
  return to_status(raster_path(g, cam, ro, p, w, grad_maps, tile_mask, tile_mask != nullptr, st));
}

static int poisson_common(const float *field, int input_is_rho, const uint8_t *tile_mask,
                          int32_t channels, int32_t height, int32_t width, const float *mean,
                          const gdgs_solver_opts *sopts, float *image, void *ws, size_t ws_bytes,
                          void *stream) {
  if (!field || !image || !mean || !aligned(field, 16) || !aligned(image, 16))
    return GDGS_ERR_INVALID_ARG;
  if (channels < 1 || channels > GDGS_MAX_CHANNELS) return GDGS_ERR_INVALID_ARG;
  const gdgs_raster_opts ro = ropts_or_default(nullptr);
  const gdgs_solver_opts so = sopts_or_default(sopts);
  Plan p;
  if (!make_plan(0, channels, width, height, ro, so, &p)) return GDGS_ERR_INVALID_ARG;
  for (int c = 0; c < channels; ++c)
    if (!isfinite(mean[c])) return GDGS_ERR_INVALID_ARG;
  const size_t plane = (size_t)width * height * channels;
  const size_t fbytes = plane * (input_is_rho ? 1 : 2) * sizeof(float);
  const char *ib = (const char *)image, *gb = (const char *)field;
  if (ib < gb + fbytes && gb < ib + plane * sizeof(float)) return GDGS_ERR_INVALID_ARG;
  int s;
  if ((s = check_ws(ws, ws_bytes, p))) return s;
  cudaStream_t st = (cudaStream_t)stream;
  char *w = (char *)ws;
  if (cudaMemsetAsync(w + p.off_ctrl, 0, sizeof(Ctrl), st) != cudaSuccess) return GDGS_ERR_CUDA;
  PoissonArgs a{};
  a.maps = field;
  a.input_is_rho = input_is_rho;
  a.threshold = so.rho_threshold;
  a.mask = tile_mask;
  a.C = channels;
  a.H = height;
  a.W = width;
  a.tiles_x = p.tiles_x;
  for (int c = 0; c < channels; ++c) a.mean[c] = mean[c];
  a.image = image;
  a.nu1 = so.nu1;
  a.nu2 = so.nu2;
  a.omega = so.omega;
  a.storage = so.storage;
  a.max_cycles = so.max_cycles;
  a.rtol = so.rtol;
  a.plan = &p;
  a.ws = w;
  a.ctrl = (Ctrl *)(w + p.off_ctrl);
  return to_status(run_poisson(a, st));
}

int gdgs_poisson_reconstruct(const float *grad_maps, const uint8_t *tile_mask, int32_t channels,
                             int32_t height, int32_t width, const float *mean,
                             const gdgs_solver_opts *sopts, float *image, void *ws,
                             size_t ws_bytes, void *stream) {
  return poisson_common(grad_maps, 0, tile_mask, channels, height, width, mean, sopts, image, ws,
                        ws_bytes, stream);
}

int gdgs_poisson_reconstruct_rho(const float *rho, const uint8_t *tile_mask, int32_t channels,
                                 int32_t height, int32_t width, const float *mean,
                                 const gdgs_solver_opts *sopts, float *image, void *ws,
                                 size_t ws_bytes, void *stream) {
  return poisson_common(rho, 1, tile_mask, channels, height, width, mean, sopts, image, ws,
                        ws_bytes, stream);
}

static int render_view_impl(const gdgs_gaussians *g, const gdgs_camera *cam,
                            const gdgs_camera *cam_dev, const float *mean,
                            const gdgs_raster_opts *ropts, const gdgs_solver_opts *sopts,
                            float *image, void *ws, size_t ws_bytes, void *stream) {
  int s;
  if ((s = check_gaussians(g)) || (s = check_camera(cam))) return s;
  if (!image || !mean || !aligned(image, 16)) return GDGS_ERR_INVALID_ARG;
  const gdgs_raster_opts ro = ropts_or_default(ropts);
  const gdgs_solver_opts so = sopts_or_default(sopts);
  Plan p;
  if (!make_plan(g->n, g->channels, cam->width, cam->height, ro, so, &p)) return GDGS_ERR_INVALID_ARG;
  for (int c = 0; c < g->channels; ++c)
    if (!isfinite(mean[c])) return GDGS_ERR_INVALID_ARG;
  if ((s = check_ws(ws, ws_bytes, p))) return s;
  cudaStream_t st = (cudaStream_t)stream;
  char *w = (char *)ws;
  if (cudaMemsetAsync(w + p.off_ctrl, 0, sizeof(Ctrl), st) != cudaSuccess) return GDGS_ERR_CUDA;
  uint8_t *mask = (uint8_t *)(w + p.off_mask);
  float *maps = (float *)(w + p.off_maps);
  cudaError_t e = raster_path(g, cam, ro, p, w, maps, mask, true, st, cam_dev);
  if (e != cudaSuccess) return GDGS_ERR_CUDA;
  PoissonArgs a{};
  a.maps = maps;
  a.input_is_rho = g->attribute == GDGS_ATTR_LAPLACIAN;
  a.threshold = so.rho_threshold;
  a.mask = mask;
  a.C = g->channels;
  a.H = cam->height;
  a.W = cam->width;
  a.tiles_x = p.tiles_x;
  for (int c = 0; c < g->channels; ++c) a.mean[c] = mean[c];
  a.image = image;
  a.nu1 = so.nu1;
  a.nu2 = so.nu2;
  a.omega = so.omega;
  a.storage = so.storage;
  a.max_cycles = so.max_cycles;
  a.rtol = so.rtol;
  a.plan = &p;
  a.ws = w;
  a.ctrl = (Ctrl *)(w + p.off_ctrl);
  return to_status(run_poisson(a, st));
}

int gdgs_render_view(const gdgs_gaussians *g, const gdgs_camera *cam, const float *mean,
                     const gdgs_raster_opts *ropts, const gdgs_solver_opts *sopts, float *image,
                     void *ws, size_t ws_bytes, void *stream) {
  return render_view_impl(g, cam, nullptr, mean, ropts, sopts, image, ws, ws_bytes, stream);
}

int gdgs_render_view_devcam(const gdgs_gaussians *g, const gdgs_camera *cam,
                            const gdgs_camera *cam_dev, const float *mean,
                            const gdgs_raster_opts *ropts, const gdgs_solver_opts *sopts,
                            float *image, void *ws, size_t ws_bytes, void *stream) {
  if (!cam_dev || !aligned(cam_dev, 4)) return GDGS_ERR_INVALID_ARG;
  return render_view_impl(g, cam, cam_dev, mean, ropts, sopts, image, ws, ws_bytes, stream);
}

int gdgs_render_view_backward(const gdgs_gaussians *g, const gdgs_camera *cam,
                              const gdgs_raster_opts *ropts, const gdgs_solver_opts *sopts,
                              const float *d_image, const gdgs_gaussian_grads *grads, void *ws,
                              size_t ws_bytes, void *ws_adj, size_t ws_adj_bytes, void *stream) {
  int s;
  if ((s = check_gaussians(g)) || (s = check_camera(cam))) return s;
  if (!d_image || !grads || !grads->d_mean || !grads->d_scale || !grads->d_quat ||
      !grads->d_opacity || !grads->d_attr)
    return GDGS_ERR_INVALID_ARG;
  const gdgs_raster_opts ro = ropts_or_default(ropts);
  const gdgs_solver_opts so = sopts_or_default(sopts);
  Plan p, pa;
  if (!make_plan(g->n, g->channels, cam->width, cam->height, ro, so, &p) ||
      !make_plan(0, g->channels, cam->width, cam->height, ro, so, &pa))
    return GDGS_ERR_INVALID_ARG;
  if ((s = check_ws(ws, ws_bytes, p)) || (s = check_ws(ws_adj, ws_adj_bytes, pa))) return s;
  cudaStream_t st = (cudaStream_t)stream;
  char *w = (char *)ws, *wa = (char *)ws_adj;
  const int C = g->channels, Q = attr_floats(g);
  const size_t n = (size_t)g->n, plane = (size_t)cam->width * cam->height;
  // gradients accumulate (atomics) or are written per Gaussian: clear first
  if (cudaMemsetAsync(grads->d_attr, 0, 4 * n * Q, st) != cudaSuccess ||
      (n && cudaMemsetAsync(w + p.off_dsplat, 0, 24 * n, st) != cudaSuccess) ||
      cudaMemsetAsync(wa + pa.off_ctrl, 0, sizeof(Ctrl), st) != cudaSuccess)
    return GDGS_ERR_CUDA;
  // 1. d rho = the zero-mean solve of d image (L symmetric), into the forward
  //    workspace's correction array (the multigrid scratch is not read below)
  float *rbar = (float *)(w + p.off_e0);
  PoissonArgs a{};
  a.maps = d_image;
  a.input_is_rho = 1;
  a.threshold = 0.f;
  a.mask = nullptr;
  a.C = C;
  a.H = cam->height;
  a.W = cam->width;
  a.tiles_x = pa.tiles_x;
  for (int c = 0; c < GDGS_MAX_CHANNELS; ++c) a.mean[c] = 0.f;
  a.image = rbar;
  a.nu1 = so.nu1;
  a.nu2 = so.nu2;
  a.omega = so.omega;
  a.storage = so.storage;
  a.max_cycles = so.max_cycles;
  a.rtol = so.rtol;
  a.plan = &pa;
  a.ws = wa;
  a.ctrl = (Ctrl *)(wa + pa.off_ctrl);
  cudaError_t e = run_poisson(a, st);
  if (e != cudaSuccess) return to_status(e);
  if (n == 0) return GDGS_OK;
  // 2. through the threshold and the divergence into d maps
  DivAdjArgs d{};
  d.rbar = rbar;
  d.rho_fwd = so.rho_threshold > 0.f ? (const float *)(w + p.off_rho) : nullptr;
  d.mask = (const uint8_t *)(w + p.off_mask);
  d.input_is_rho = g->attribute == GDGS_ATTR_LAPLACIAN;
  d.C = C;
  d.H = cam->height;
  d.W = cam->width;
  d.tiles_x = p.tiles_x;
  d.mbar = (float *)(w + p.off_maps);
  if ((e = launch_divergence_adjoint(d, st)) != cudaSuccess) return to_status(e);
  // 3. the composite, tile by tile, back to front
  int tbits = 0;
  while ((1 << tbits) < p.T) ++tbits;
  const bool alt = ((tbits + 7) / 8) % 2 == 1;  // the pair sort's passes swap buffers
  RasterBwdArgs r{};
  r.smean = (const float4 *)(w + p.off_smean);
  r.sconic = (const float4 *)(w + p.off_sconic);
  r.attr = g->grad;
  r.pval = (const uint32_t *)(w + p.off_pval[alt ? 1 : 0]);
  r.range = (const uint2 *)(w + p.off_range);
  r.active = (const uint32_t *)(w + p.off_active);
  r.Q = Q;
  r.W = cam->width;
  r.H = cam->height;
  r.tiles_x = p.tiles_x;
  r.T = p.T;
  r.alpha_min = ro.alpha_min;
  r.alpha_max = ro.alpha_max;
  r.t_min = ro.t_min;
  r.mbar = (const float *)(w + p.off_maps);
  r.dsplat = (float *)(w + p.off_dsplat);
  r.dattr = grads->d_attr;
  r.ctrl = (Ctrl *)(w + p.off_ctrl);
  if ((e = launch_raster_backward(r, st)) != cudaSuccess) return to_status(e);
  // 4. the projection
  ProjBwdArgs pb{};
  pb.mean = g->mean;
  pb.scale = g->scale;
  pb.quat = g->quat;
  pb.n = g->n;
  memcpy(pb.w2c, cam->world_to_cam, sizeof(pb.w2c));
  pb.fx = cam->fx;
  pb.fy = cam->fy;
  pb.dilation = ro.dilation;
  pb.exp_coef = ro.exp_coef;
  pb.dsplat = (const float *)(w + p.off_dsplat);
  pb.d_mean = grads->d_mean;
  pb.d_scale = grads->d_scale;
  pb.d_quat = grads->d_quat;
  pb.d_opacity = grads->d_opacity;
  (void)plane;
  return to_status(launch_project_backward(pb, st));
}

int gdgs_sync_status(const void *ws, gdgs_solve_stats *stats, void *stream) {
  if (!ws) return GDGS_ERR_WORKSPACE;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return GDGS_ERR_CUDA;
  Ctrl c;
  if (cudaMemcpy(&c, ws, sizeof(Ctrl), cudaMemcpyDeviceToHost) != cudaSuccess) return GDGS_ERR_CUDA;
  int status = c.status;
  double rel = 0.0;
  if (c.max_cycles > 0) {  // a solve ran
    const double r0 = c.rnorm2[0];
    rel = r0 > 0 ? sqrt(c.final_rnorm2 / r0) : 0.0;
    if (status == GDGS_OK && !(rel == rel)) status = GDGS_ERR_NONFINITE;
    if (status == GDGS_OK && !c.stopped && rel > c.rtol) status = GDGS_ERR_NO_CONVERGE;
  }
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->status = status;
    stats->cycles = c.cycles;
    stats->rel_residual = rel;
    stats->rho_norm = sqrt(c.rnorm2[0]);
    for (int i = 0; i < GDGS_MAX_CHANNELS; ++i) stats->mean_set[i] = c.mean_set[i];
    stats->n_pairs = (int64_t)c.n_pairs;
    stats->n_active_tiles = (int32_t)c.n_active;
    stats->n_visible = c.n_visible;
  }
  return status;
}

}  // extern "C"
