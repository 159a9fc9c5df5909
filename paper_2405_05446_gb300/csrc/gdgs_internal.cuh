// Internal declarations shared by the CUDA translation units of libgdgs.
// Not part of the ABI; include/gdgs.h is the public contract.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/gdgs.h"

namespace gdgs {

constexpr int kTile = GDGS_TILE;        // raster tile edge (pixels)
constexpr int kMaxCycles = 64;          // bound on V-cycles per solve
constexpr int kMaxLevels = 24;          // bound on multigrid levels
constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 8;          // keys per thread per radix block (pair sort)
constexpr int kRadixBlock = kRadixThreads * kRadixItems;
constexpr int kRadixItemsSmall = 2;     // depth sort (fewer keys): more, shorter blocks
constexpr int kRadixBlockSmall = kRadixThreads * kRadixItemsSmall;
constexpr int kBinBlock = 256;  // Gaussians per block of the pair count and emission
constexpr uint32_t kInvalidKey = 0xFFFFFFFFu;

// Device control block at offset 0 of every workspace. Zeroed at the start of
// each call (except the fields after `persist_begin`, of which there are none:
// the coarse-solver cache lives in its own region).
struct Ctrl {
  int status;          // first device error (atomicCAS from GDGS_OK)
  int stopped;         // multigrid: convergence observed
  int cycles;          // multigrid: V-cycles behind the returned iterate
  int n_visible;       // Gaussians that survived projection
  unsigned long long n_pairs;  // (tile, splat) pairs requested (uncapped)
  unsigned n_active;   // tiles with at least one pair
  unsigned pad0;
  int max_cycles;
  int channels;
  int iter;            // cycle index when the cycle loop runs as a graph
  int pad1;
  double rtol;
  double rnorm2[kMaxCycles + 1];             // ||rho - L u_k||^2, k = 0..
  double sum_u[kMaxCycles + 1][GDGS_MAX_CHANNELS];  // sum of u_k per channel
  double final_rnorm2;                       // residual of the returned iterate
  double mean_set[GDGS_MAX_CHANNELS];
  double rho_sum[GDGS_MAX_CHANNELS];         // sum and sum of squares of rho per channel
  double rho_sq[GDGS_MAX_CHANNELS];
  float rho_mean[GDGS_MAX_CHANNELS];         // the constant removed from rho (least squares)
  float escale[kMaxCycles + 1];              // cycle k solves for s_k e (a power of two)
  // channel split: every channel ran its own cycle loop (control block of its
  // own, off_sub); kf_c[c] is the cycle count of channel c's returned iterate
  int split;
  int kf_c[GDGS_MAX_CHANNELS];
};

// Diagnostics hooks around every kernel launch (diag.cu).
void diag_before(const char *name, cudaStream_t st);
void diag_after(cudaStream_t st);
bool diag_profiling();
void diag_set_capturing(bool on);  // launches on this thread are being captured into a graph
unsigned long long graph_kernel_count();  // kernels run by graph-launched cycle loops
// Programmatic dependent launch. Every kernel of the library begins with
// griddep_enter(), which waits until the kernel launched before it on the
// stream has completed and its writes are visible (griddepcontrol.wait).
// Kernels are launched with the programmatic-serialization attribute (below),
// so a dependent grid is launched as soon as every CTA of its predecessor has
// exited, overlapping the launch with the predecessor's completion, instead of
// after a full launch round trip. No kernel triggers its dependents early
// (griddepcontrol.launch_dependents): CTAs launched early would sit resident
// while they wait and take SM slots from kernels of other streams (measured:
// 583 against 721 mixed views/s when four streams serve views). The wait comes
// before any global access of every thread, so the order of all reads and
// writes is that of plain stream order, and a kernel completes only after its
// predecessor has.
__device__ __forceinline__ void griddep_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

bool pdl_enabled();  // GDGS_PDL=0 turns the attribute off (diag.cu)

// Launch with the programmatic-serialization attribute (when enabled). Errors
// are reported by the caller's cudaGetLastError, as for <<<>>> launches.
template <typename... K, typename... A>
inline void launch_k(void (*kern)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     A &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, static_cast<A &&>(args)...);
}

struct LaunchScope {
  cudaStream_t st;
  LaunchScope(const char *name, cudaStream_t s) : st(s) { diag_before(name, s); }
  ~LaunchScope() { diag_after(st); }
};

__device__ __forceinline__ void set_status(Ctrl *c, int code) {
  atomicCAS(&c->status, GDGS_OK, code);
}

// Geometry of one multigrid level. Level l has ceil(N0 / 2^l) cells per side;
// cell J covers fine pixels [J 2^l, min((J+1) 2^l, N0)), so only the last cell
// of a side may be narrower. Widths are normalised by 2^l (full cell = 1).
struct LevelGeom {
  int H, W;            // cells
  int shift;           // l
  int H0, W0;          // finest grid
  float lastx, lasty;  // normalised width of the last column / height of the last row
  float ex, ey;        // 2 / (1 + lastx), 2 / (1 + lasty): face factors next to them
  long long plane;     // floats per channel plane (H * W)
};

// ---------------------------------------------------------------- workspace plan
struct Plan {
  int64_t n;
  int C, W, H;
  int tiles_x, tiles_y, T;
  unsigned pair_cap;
  int radix_blocks_max;
  // offsets in bytes from the workspace base
  size_t off_ctrl;
  size_t off_smean, off_sconic, off_rect;              // projected splats [n]
  size_t off_dkey[2], off_dval[2];                     // depth sort [n]
  size_t off_dlo;                                      // depth sort secondary key [n]
  size_t off_hist;                                     // radix histograms
  size_t off_blocksum;                                 // scan partials
  size_t off_gtiles;                                   // tiles per depth-ordered Gaussian
  size_t off_pkey[2], off_pval[2];                     // pairs [pair_cap]
  size_t off_range, off_active, off_mask;              // per tile
  size_t off_maps;                                     // [C][2][H][W]
  size_t off_dsplat;                                   // backward: [n][6]
  size_t off_rho, off_uhi, off_ulo, off_e0, off_r[2];  // level 0 [C][H][W]
  size_t off_lu[kMaxLevels], off_lf[kMaxLevels];       // levels >= 1: down-pass u, f
  size_t off_luo[kMaxLevels];                          // levels >= 1: up-pass u (never in place)
  size_t off_coarse;                                   // tag + FP64 inverse
  size_t off_sub;                                      // per-channel control blocks [C]
  int levels;         // number of levels (finest = 0, coarsest = levels-1)
  int nc;             // unknowns on the coarsest level
  LevelGeom lv[kMaxLevels];
  size_t total;
};

bool make_plan(int64_t n, int C, int W, int H, const gdgs_raster_opts &ro,
               const gdgs_solver_opts &so, Plan *p);

constexpr size_t kCoarseTagBytes = 256;
struct CoarseTag {
  unsigned long long magic;
  int H0, W0, levels, Hc, Wc, nc;
  int version;
  int pad;
  unsigned long long hash;  // digest of the cached factor
};
constexpr int kMaxCoarse = 16 * 16;  // unknowns of the largest coarsest grid

// ---------------------------------------------------------------- launchers
// Each returns cudaSuccess or the launch error; all enqueue on `st`.
struct ProjectArgs {
  const float *mean, *scale, *quat, *opacity, *grad;
  int64_t n;
  int C;
  int Q;           // attribute floats per Gaussian
  float w2c[12];
  float fx, fy, cx, cy, znear;
  int W, H, tiles_x, tiles_y;
  const gdgs_camera *cam_dev;  // when set, w2c .. znear are read from it on the device
  float alpha_min, dilation, exp_coef;
  // outputs (workspace)
  float4 *smean;   // mx_hi, my_hi, mx_lo, my_lo
  float4 *sconic;  // conic * exp_coef * log2(e) (a, 2b, c), opacity
  uint32_t *key;   // float bits of the depth's hi part, kInvalidKey when culled
  uint32_t *key_lo;  // 8-bit digit of the depth's lo part in units of ulp(hi) / 256
  uint2 *rect;     // x0 | x1 << 16, y0 | y1 << 16 (tiles, half open)
  // optional outputs
  float *o_mean2d, *o_cov2d, *o_depth;
  int32_t *o_rect;
  Ctrl *ctrl;
};
cudaError_t launch_project(const ProjectArgs &a, cudaStream_t st);

// Stable LSD radix sort of 32-bit keys with 32-bit values over bits
// [0, nbits). n = min(*n_dev, cap) if n_dev else cap. vals_in == nullptr means
// the values are the element indices. lo_keys (nullable): a secondary key whose
// low 8 bits order elements with equal keys (one extra pass, run first).
// Blocks of kRadixThreads * items keys (items kRadixItems or kRadixItemsSmall),
// max_blocks of them at most; hist holds 256 * (max_blocks + 1) words. Returns
// in *out_is_alt whether the result sits in the alternate buffers.
cudaError_t radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt,
                             uint32_t *vals_alt, bool implicit_vals, const uint32_t *lo_keys,
                             const unsigned long long *n_dev, unsigned cap, int nbits,
                             uint32_t *hist, int items, int max_blocks, bool *out_is_alt,
                             cudaStream_t st);

struct BinArgs {
  const uint32_t *order;   // Gaussian indices in depth order [n]
  const uint2 *rect;
  const float4 *smean, *sconic;  // projected splats (ellipse test of each tile of the rect)
  float alpha_min;
  int64_t n;
  int tiles_x, T;
  unsigned pair_cap;
  unsigned long long *blocksum;  // [ceil(n / kBinBlock) + 1]
  uint32_t *tiles;         // [n] tiles each depth-ordered Gaussian reaches (count -> emit)
  uint32_t *pkey, *pval;   // emitted pairs
  Ctrl *ctrl;
};
cudaError_t launch_emit_pairs(const BinArgs &a, cudaStream_t st);

cudaError_t launch_tile_ranges(const uint32_t *sorted_keys, Ctrl *ctrl, unsigned pair_cap,
                               int T, uint2 *range, uint32_t *active, uint8_t *mask,
                               cudaStream_t st);

// A projected splat staged for the 16x16 tile whose origin is (x0, y0), as the
// forward and the backward rasteriser both evaluate it (the backward replays
// the forward's arithmetic exactly). The centre relative to the tile origin is
// split into a part h on a 2^-12 pixel grid and a remainder l (|l| <= 2^-13 px,
// carried from the projection's float-float centre): a pixel centre minus h is
// exact in FP32, and l enters through the linear and constant terms of the
// expanded exponent, so no offset is rounded at the tile's scale. With
// X = px - h, Y = py - h_y and the stored conic (A, B', C) (k log2 e folded in):
//   p2 = A dx^2 + B' dx dy + C dy^2, dx = X - l_x, dy = Y - l_y,
//      = X (A X + B' Y + a) + Y (C Y + b) + c0,
//   a = -(2 A l_x + B' l_y), b = -(B' l_x + 2 C l_y), c0 = A l_x^2 + B' l_x l_y + C l_y^2,
// and alpha = opacity 2^-p2 = 2^(L - (p2 - c0)) with L = log2(opacity) - c0.
struct StagedSplat {
  float4 geo;   // h_x, h_y, A, B'
  float4 geo2;  // C, L, a, b
  float lx, ly;
};

__device__ __forceinline__ float2 split_tile_offset(float hi, float lo, float origin) {
  // hi - origin exactly as s + e (TwoSum), then s = h + (s - h) with h on the grid
  const float s = __fadd_rn(hi, -origin), bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(-origin, bb));
  const float h = __fmul_rn(rintf(__fmul_rn(s, 4096.f)), 1.f / 4096.f);
  return make_float2(h, __fadd_rn(__fsub_rn(s, h), __fadd_rn(e, lo)));  // s - h is exact
}

// smean = (x_hi, y_hi, x_lo, y_lo), sconic = (A, B', C, opacity)
__device__ __forceinline__ StagedSplat stage_splat(float4 m, float4 k, float x0f, float y0f) {
  const float2 ox = split_tile_offset(m.x, m.z, x0f), oy = split_tile_offset(m.y, m.w, y0f);
  const float lx = ox.y, ly = oy.y;
  const float a = -fmaf(2.f * k.x, lx, k.y * ly), b = -fmaf(k.y, lx, 2.f * k.z * ly);
  const float c0 = fmaf(k.x * lx, lx, fmaf(k.y * lx, ly, k.z * ly * ly));
  StagedSplat st;
  st.geo = make_float4(ox.x, oy.x, k.x, k.y);
  st.geo2 = make_float4(k.z, log2f(k.w) - c0, a, b);
  st.lx = lx;
  st.ly = ly;
  return st;
}

// p2 - c0 at the pixel centre (fpx, fpy) relative to the tile origin.
__device__ __forceinline__ float staged_exponent(const float4 &ge, const float4 &ge2, float fpx,
                                                 float fpy, float &X, float &Y) {
  X = fpx - ge.x;
  Y = fpy - ge.y;
  return fmaf(X, fmaf(ge.z, X, fmaf(ge.w, Y, ge2.z)), Y * fmaf(ge2.x, Y, ge2.w));
}

// Rasterisers: a warp holds a 4 x 8 pixel block of a 16 x 16 tile (warp w: rows
// 4 (w >> 1) .. +3, columns 8 (w & 1) .. +7). Warps whose 4 x 8 pixel blocks the bounding box of the splat's ellipse p2 <=
// log2(opacity / alpha_min) + 1e-3 (the exponent cut of the composite) can
// reach, widened like the binning's cut (0.1 % + 0.01) so that no reachable
// pixel is dropped. The ellipse's half-extents are sqrt(lim 4A / D) vertically
// and sqrt(lim 4C / D) horizontally, D = 4AC - B'^2, around the tile-relative
// centre (h_x + l_x, h_y + l_y); pixel (c, r) has its centre at (c + 0.5, r + 0.5).
__device__ __forceinline__ uint8_t warp_block_mask(const StagedSplat &st, float4 k, float amin) {
  const float A = k.x, B = k.y, C = k.z;
  const float lim = (log2f(k.w / amin) + 1e-3f) * 1.001f + 0.01f;
  const float D = fmaf(4.f * A, C, -B * B);
  if (!(lim > 0.f) || !(D > 0.f)) return 0xffu;  // degenerate: keep for every warp
  const float hy = sqrtf(lim * 4.f * A / D) * 1.0001f + 1e-3f;
  const float hx = sqrtf(lim * 4.f * C / D) * 1.0001f + 1e-3f;
  const float cy = st.geo.y + st.ly, cx = st.geo.x + st.lx;
  const float r0 = ceilf(cy - hy - 0.5f), r1 = floorf(cy + hy - 0.5f);  // reachable pixel rows
  const float c0 = ceilf(cx - hx - 0.5f), c1 = floorf(cx + hx - 0.5f);  // and columns
  if (!(r1 >= 0.f) || !(r0 <= (float)(kTile - 1)) || !(c1 >= 0.f) || !(c0 <= (float)(kTile - 1)))
    return 0u;
  const int i0 = max(0, (int)r0) >> 2, i1 = min(kTile - 1, (int)r1) >> 2;  // row blocks 0..3
  const int j0 = max(0, (int)c0) >> 3, j1 = min(kTile - 1, (int)c1) >> 3;  // column blocks 0..1
  const unsigned rows = ((2u << i1) - 1u) & ~((1u << i0) - 1u);
  // row block i -> warps 2i (left block) and 2i + 1 (right block)
  const unsigned even = (rows & 1u) | ((rows & 2u) << 1) | ((rows & 4u) << 2) | ((rows & 8u) << 3);
  return (uint8_t)((j0 == 0 ? even : 0u) | (j1 == 1 ? even << 1 : 0u));
}

// The batch entries (of cnt) whose mask includes this warp, compacted in batch
// order into list; returns their number. Called by all 32 lanes of the warp.
__device__ __forceinline__ int warp_list(const uint8_t *wmask, int cnt, uint8_t *list, int warp,
                                         int lane) {
  int nl = 0;
  for (int k0 = 0; k0 < cnt; k0 += 32) {
    const int k = k0 + lane;
    const bool in = k < cnt && ((wmask[k] >> warp) & 1u);
    const unsigned b = __ballot_sync(0xffffffffu, in);
    if (in) list[nl + __popc(b & ((1u << lane) - 1u))] = (uint8_t)k;
    nl += __popc(b);
  }
  __syncwarp();
  return nl;
}

struct RasterArgs {
  const float4 *smean, *sconic;
  const float *grad;
  const uint32_t *pval;     // Gaussian index of each sorted pair
  const uint2 *range;       // [T]
  const uint32_t *active;   // [T] active tile ids (when use_active)
  int use_active;           // 1: only active tiles (count in ctrl->n_active)
  int Q, W, H, tiles_x, T;  // Q attribute floats per Gaussian = output planes
  int grad_pairs;           // set by launch_raster: Q even and grad 8-byte aligned
  float alpha_min, alpha_max, t_min;
  float *maps;              // [Q][H][W]
  Ctrl *ctrl;
};
cudaError_t launch_raster(const RasterArgs &a, cudaStream_t st);

struct PoissonArgs {
  const float *maps;        // [C][2][H][W], or [C][H][W] when input_is_rho
  int input_is_rho;         // the field rho itself instead of gradient maps
  float threshold;          // hard threshold on rho (0: none)
  const uint8_t *mask;      // [tiles_y][tiles_x] or null
  int C, H, W, tiles_x;
  float mean[GDGS_MAX_CHANNELS];
  float *image;             // [C][H][W]
  int nu1, nu2, max_cycles;
  float rtol;
  float omega;              // smoother over-relaxation
  int storage;              // GDGS_STORAGE_*: multigrid corrections and coarse right-hand sides
  const Plan *plan;
  char *ws;
  Ctrl *ctrl;
};
cudaError_t run_poisson(const PoissonArgs &a, cudaStream_t st);

// ---------------------------------------------------------------- backward
struct DivAdjArgs {
  const float *rbar;     // d loss / d rho [C][H][W]
  const float *rho_fwd;  // the forward's thresholded rho (null: no threshold)
  const uint8_t *mask;   // forward tile mask (null: none)
  int input_is_rho;      // Laplacian attribute: maps are rho itself
  int C, H, W, tiles_x;
  float *mbar;           // d loss / d maps [Q][H][W]
};
cudaError_t launch_divergence_adjoint(const DivAdjArgs &a, cudaStream_t st);

struct RasterBwdArgs {
  const float4 *smean, *sconic;
  const float *attr;        // per-Gaussian attribute [n][Q]
  const uint32_t *pval;     // the forward's sorted pairs
  const uint2 *range;
  const uint32_t *active;
  int Q, W, H, tiles_x, T;
  float alpha_min, alpha_max, t_min;
  const float *mbar;        // d loss / d maps [Q][H][W]
  float *dsplat;            // [n][6]: centre x, y; stored conic A, B, C; opacity (accumulated)
  float *dattr;             // [n][Q] (accumulated)
  Ctrl *ctrl;
};
cudaError_t launch_raster_backward(const RasterBwdArgs &a, cudaStream_t st);

struct ProjBwdArgs {
  const float *mean, *scale, *quat;
  int64_t n;
  float w2c[12];
  float fx, fy;
  float dilation, exp_coef;
  const float *dsplat;
  float *d_mean, *d_scale, *d_quat, *d_opacity;
};
cudaError_t launch_project_backward(const ProjBwdArgs &a, cudaStream_t st);

}  // namespace gdgs
