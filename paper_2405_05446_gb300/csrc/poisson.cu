// Poisson reconstruction of the image from its gradient maps (K6-K11).
//
// rho = div(g) (the Laplacian field is the divergence of the gradient field,
// Sec. 1.5 "Sparsity"), then the Neumann problem L u = rho of Eq. p2d is solved
// by multigrid, one of the linear-complexity solvers the paper lists (Sec. 2.1,
// Sec. 2.2 "Poisson Equation"), and the free constant ("possible constant
// difference", Sec. 2.1) is fixed by a supplied per-channel mean.
//
// Discretisation. L is the 5-point Neumann Laplacian on the pixel grid,
// L u(i,j) = sum over in-grid neighbours n of (u_n - u_ij). Coarse level l has
// ceil(N / 2^l) cells per side; cell J covers fine pixels [J 2^l, min((J+1) 2^l,
// N)), so only a side's last cell can be narrow. Each level is the finite-volume
// rediscretisation on its cells: face coefficient = face length / distance
// between the two cell centres, right-hand side = sum of the children's
// residuals. Transfers: restriction sums 2x2 children; prolongation is bilinear
// in the cell-centre coordinates (constant beyond the outermost centres). The
// coarsest grid (both sides <= coarse_max_dim) is solved directly in FP64 with a
// dense inverse of -L + 11^T / n (SPD; its solution of a compatible system is the
// zero-mean solution of L u = f), built once per grid shape by Gauss-Jordan on
// the device and cached in the workspace under a tag.
//
// Iteration. The finest iterate u is a float-float pair (hi + lo): an FP32
// image carries a representation error that alone gives a relative residual
// ~1e-5 on 1080p scenes, above the 1e-6 target. Cycle k solves L e = r_k with an
// FP32 V(nu1, nu2)-cycle from e = 0, then u += e with an error-free sum and
// r_{k+1} = r_k - L e (r_0 = rho), whose norm decides convergence on the device.
// The final iterate's residual rho - L u is recomputed in float-float arithmetic.
//
// Smoother and blocking. Red-black Gauss-Seidel. On the large levels a CTA
// owns a 32 x 128 output tile, loads it with a halo of 2 nu + 1 rows (rounded
// up to 4 in x) into shared memory and runs all sweeps there: every half-sweep
// shrinks the valid region by one cell, and the halo absorbs that. Shared
// memory keeps the even-x and odd-x cells of each row in separate planes, so
// the cells of one colour in a row are contiguous and a half-sweep updates them
// four at a time with 16-byte loads; work units away from the grid border take
// that path, the few at the border a scalar path with the exact boundary
// coefficients. Down kernels fuse the pre-sweeps with residual and restriction,
// up kernels the prolongation with the post-sweeps (and, on the finest level,
// the update of u, the new residual and its norm). An up pass writes its level
// to an array of its own: the CTAs of one launch read each other's tiles as
// halo, so an in-place update would race. Levels under kSmallLevel
// cells use 16 x 64 tiles. The levels from the first with at most kTailCells
// cells per channel down to the coarsest run in one kernel, one CTA per
// channel, entirely in shared memory; it also solves the coarsest grid with
// the cached FP64 inverse.
//
// With even widths and V(2, 1), the finest level's down pass and the up passes
// of levels 0-2 run as streaming warps instead of tiles (see the section on
// them below): a warp owns a 64-column strip and carries every stage of its
// pass down a segment of rows in registers, one row per step.
//
// Convergence is decided on the device, so the cycle loop runs as a CUDA graph
// with a WHILE node: no launch is spent after convergence.
#include <stdlib.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "gdgs_internal.cuh"

namespace gdgs {

namespace {

constexpr int kBX = 32, kBY = 8;     // 256 threads
constexpr int kMgThreads = kBX * kBY;
// Output tiles of the level kernels: large levels use 32 x 128 cells, levels
// with fewer cells per channel than kSmallLevel 16 x 64 (more CTAs, shorter
// serial work per CTA, which is what bounds the small grids).
constexpr long long kSmallLevel = 160000;

// ------------------------------------------------------------------ storage formats
//
// Multigrid corrections and coarse right-hand sides live in memory as FP32,
// BF16 or FP16 (GDGS_STORAGE_*); all arithmetic is FP32. The format is a kernel
// argument, so the branches below are uniform.

__device__ __forceinline__ const void *s_at(const void *p, size_t n, int s) {
  return reinterpret_cast<const char *>(p) + n * (s == GDGS_STORAGE_F32 ? 4 : 2);
}
__device__ __forceinline__ void *s_at(void *p, size_t n, int s) {
  return reinterpret_cast<char *>(p) + n * (s == GDGS_STORAGE_F32 ? 4 : 2);
}

__device__ __forceinline__ float s_ld(const void *p, size_t i, int s) {
  if (s == GDGS_STORAGE_BF16) return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16 *>(p) + i));
  if (s == GDGS_STORAGE_F16) return __half2float(__ldg(reinterpret_cast<const __half *>(p) + i));
  return __ldg(reinterpret_cast<const float *>(p) + i);
}

__device__ __forceinline__ void s_st(void *p, size_t i, float v, int s) {
  if (s == GDGS_STORAGE_BF16) reinterpret_cast<__nv_bfloat16 *>(p)[i] = __float2bfloat16_rn(v);
  else if (s == GDGS_STORAGE_F16) reinterpret_cast<__half *>(p)[i] = __float2half_rn(v);
  else reinterpret_cast<float *>(p)[i] = v;
}

// Four consecutive elements starting at i (i % 4 == 0, 16- or 8-byte aligned).
__device__ __forceinline__ float4 s_ld4(const void *p, size_t i, int s) {
  if (s == GDGS_STORAGE_F32) return __ldg(reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(p) + i));
  const uint2 r = __ldg(reinterpret_cast<const uint2 *>(reinterpret_cast<const unsigned short *>(p) + i));
  float2 a, b;
  if (s == GDGS_STORAGE_BF16) {
    a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&r.x));
    b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&r.y));
  } else {
    a = __half22float2(*reinterpret_cast<const __half2 *>(&r.x));
    b = __half22float2(*reinterpret_cast<const __half2 *>(&r.y));
  }
  return make_float4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ void s_st4(void *p, size_t i, float4 v, int s) {
  if (s == GDGS_STORAGE_F32) {
    *reinterpret_cast<float4 *>(reinterpret_cast<float *>(p) + i) = v;
    return;
  }
  uint2 r;
  if (s == GDGS_STORAGE_BF16) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    r.x = *reinterpret_cast<const unsigned *>(&a);
    r.y = *reinterpret_cast<const unsigned *>(&b);
  } else {
    const __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
    r.x = *reinterpret_cast<const unsigned *>(&a);
    r.y = *reinterpret_cast<const unsigned *>(&b);
  }
  *reinterpret_cast<uint2 *>(reinterpret_cast<unsigned short *>(p) + i) = r;
}

// ------------------------------------------------------------------ operator

__device__ __forceinline__ float wxf(const LevelGeom &g, int J) { return J == g.W - 1 ? g.lastx : 1.f; }
__device__ __forceinline__ float wyf(const LevelGeom &g, int I) { return I == g.H - 1 ? g.lasty : 1.f; }

struct Coef {
  float e, w, s, n;
};

// Face coefficients of cell (I, J): face length / centre distance; 0 on the border.
__device__ __forceinline__ Coef coef(const LevelGeom &g, int I, int J) {
  const float wx = wxf(g, J), wy = wyf(g, I);
  Coef c;
  c.e = (J + 1 < g.W) ? wy * (J + 1 == g.W - 1 ? g.ex : 1.f) : 0.f;
  c.w = (J > 0) ? wy * (J == g.W - 1 ? g.ex : 1.f) : 0.f;
  c.s = (I + 1 < g.H) ? wx * (I + 1 == g.H - 1 ? g.ey : 1.f) : 0.f;
  c.n = (I > 0) ? wx * (I == g.H - 1 ? g.ey : 1.f) : 0.f;
  return c;
}

// All four face coefficients are 1 (full cell, full neighbours).
__device__ __forceinline__ bool interior(const LevelGeom &g, int I, int J) {
  return I > 0 && J > 0 && I < g.H - 2 && J < g.W - 2;
}

// Differences to the centre keep the rounding relative to L u, not to u: a
// correction as large as the image itself still gets an accurate residual.
__device__ __forceinline__ float residual(const LevelGeom &g, int I, int J, float u, float uE,
                                          float uW, float uS, float uN, float f) {
  if (interior(g, I, J)) return f - (((uE - u) + (uW - u)) + ((uS - u) + (uN - u)));
  const Coef c = coef(g, I, J);
  return f - (c.e * (uE - u) + c.w * (uW - u) + c.s * (uS - u) + c.n * (uN - u));
}

// Error-free accumulation of e into the float-float pair (hi, lo).
__device__ __forceinline__ void ds_add(float &hi, float &lo, float e) {
  const float s = __fadd_rn(hi, e);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(e, bb));
  const float l = __fadd_rn(lo, err);
  const float h2 = __fadd_rn(s, l);
  lo = __fsub_rn(l, __fsub_rn(h2, s));
  hi = h2;
}

struct P1 {
  int i0, i1;
  float w1;
};

// 1D bilinear weights for child index i of level `shift` from level shift+1
// (nc cells), with n0 fine cells; centres are compared in doubled fine units.
__device__ __forceinline__ P1 prolong1d(int i, int shift, int n0, int nc) {
  const int cf = (i << shift) + min((i + 1) << shift, n0);
  const int I0 = i >> 1;
  const int C0 = (I0 << (shift + 1)) + min((I0 + 1) << (shift + 1), n0);
  P1 p{I0, I0, 0.f};
  if (cf != C0) {
    const int I1 = cf < C0 ? I0 - 1 : I0 + 1;
    if (I1 >= 0 && I1 < nc) {
      const int C1 = (I1 << (shift + 1)) + min((I1 + 1) << (shift + 1), n0);
      p.i1 = I1;
      p.w1 = (float)abs(cf - C0) / (float)abs(C1 - C0);
    }
  }
  return p;
}

__device__ __forceinline__ bool should_stop(Ctrl *ctrl, int k, int first) {
  if (*(volatile int *)&ctrl->stopped) return true;
  const double thr = ctrl->rtol * ctrl->rtol * ctrl->rnorm2[0];
  if (ctrl->rnorm2[k] <= thr) {
    if (first && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&
        threadIdx.y == 0) {
      ctrl->stopped = 1;
      ctrl->cycles = k;
    }
    return true;
  }
  return false;
}

// should_stop evaluated once per block (its FP64 products are slow here) and
// shared; the result is uniform over the block.
__device__ __forceinline__ bool block_should_stop(Ctrl *ctrl, int k, int first) {
  __shared__ int s_stop;
  if (threadIdx.x == 0 && threadIdx.y == 0) s_stop = should_stop(ctrl, k, first) ? 1 : 0;
  __syncthreads();
  return s_stop != 0;
}

// Two block-wide sums in one pass; valid in the first thread of the block.
__device__ void block_sum2(float &a, float &b) {
  __shared__ float2 part2[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthreads = blockDim.x * blockDim.y;
  const int lane = tid & 31, w = tid >> 5;
  __syncthreads();
  if (lane == 0) part2[w] = make_float2(a, b);
  __syncthreads();
  float sa = 0.f, sb = 0.f;
  if (tid == 0)
    for (int i = 0; i < (nthreads + 31) / 32; ++i) {
      sa += part2[i].x;
      sb += part2[i].y;
    }
  a = sa;
  b = sb;
}

// Block-wide sum; the result is valid in the first thread of the block.
__device__ float block_sum(float v) {
  __shared__ float part[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthreads = blockDim.x * blockDim.y;
  const int lane = tid & 31, w = tid >> 5;
  __syncthreads();
  if (lane == 0) part[w] = v;
  __syncthreads();
  float s = 0.f;
  if (tid == 0)
    for (int i = 0; i < (nthreads + 31) / 32; ++i) s += part[i];
  return s;
}

__device__ __forceinline__ int cycle_index(const Ctrl *ctrl, int k) { return k >= 0 ? k : ctrl->iter; }

// ------------------------------------------------------------------ tiles in shared memory
//
// A region of RY rows x RXP cells, origin (ry0, rx0) with rx0 even. Cell (y, x)
// of the region lives in plane x & 1 at plane + y * S + 4 + (x >> 1); each plane
// row has 4 pad slots on either side (zeroed), so the quad loops may read one
// cell past the region edge. A plane is padded to 16 mod 32 floats so that the
// two planes of a cell pair sit in different banks.

template <int NU, int TY_ = 32, int TX_ = 128>
struct Geo {
  static constexpr int TY = TY_, TX = TX_;
  static constexpr int HY = 2 * NU + 1;
  static constexpr int HX = (HY + 3) / 4 * 4;
  static constexpr int RY = TY + 2 * HY;
  static constexpr int RXP = TX + 2 * HX;
  static constexpr int NC = RXP / 2;
  static constexpr int NQ = NC / 4;
  static constexpr int S = NC + 8;
  static constexpr int PLANE = RY * S + ((16 - (RY * S) % 32) + 32) % 32;
  static constexpr int ARR = 2 * PLANE;
  static constexpr int CRY = RY / 2 + 4, CRX = RXP / 2 + 4;  // coarse box bound
  static_assert(RXP % 8 == 0 && S % 4 == 0 && PLANE % 4 == 0 && CRX % 4 == 0, "quad alignment");
  static_assert(HX % 4 == 0 && TX % 8 == 0 && (TY * TX / 4) % (kBX * kBY) == 0, "vector paths");
};

template <class G>
__device__ __forceinline__ float &at(float *A, int y, int x) {
  return A[(x & 1) * G::PLANE + y * G::S + 4 + (x >> 1)];
}

template <class G>
__device__ __forceinline__ void zero_pads(float *A) {
  const int tid = threadIdx.y * kBX + threadIdx.x;
  for (int i = tid; i < 2 * G::RY * 8; i += kMgThreads) {
    const int plane = i / (G::RY * 8), r = i % (G::RY * 8);
    const int y = r >> 3, j = r & 7;
    A[plane * G::PLANE + y * G::S + (j < 4 ? j : G::NC + j)] = 0.f;
  }
}

// Loads src (a level array) into the split layout; cells outside the grid read 0.
// All loads of a thread are issued before its stores, so they overlap.
template <class G>
__device__ __forceinline__ void load_split(float *A, const void *__restrict__ src, int sf,
                                           const LevelGeom &g, int ry0, int rx0, float off,
                                           float scale) {
  constexpr int NY = (G::RY + kBY - 1) / kBY, NX = (G::RXP + kBX - 1) / kBX;
  float v[NY][NX];
#pragma unroll
  for (int i = 0; i < NY; ++i) {
    const int y = threadIdx.y + kBY * i, gy = ry0 + y;
    const bool rin = y < G::RY && gy >= 0 && gy < g.H;
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      const int x = threadIdx.x + kBX * j, gx = rx0 + x;
      v[i][j] = (rin && x < G::RXP && gx >= 0 && gx < g.W)
                    ? (s_ld(src, (size_t)gy * g.W + gx, sf) - off) * scale
                    : 0.f;
    }
  }
#pragma unroll
  for (int i = 0; i < NY; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      const int y = threadIdx.y + kBY * i, x = threadIdx.x + kBX * j;
      if (y < G::RY && x < G::RXP) at<G>(A, y, x) = v[i][j];
    }
  zero_pads<G>(A);
}

// The same with 16-byte loads, for W % 4 == 0: rx0 is a multiple of 4 too, so
// every group of 4 cells is wholly inside or outside the grid. A group (x, x+1,
// x+2, x+3) goes to the even plane as (x, x+2) and to the odd one as (x+1, x+3).
template <class G>
__device__ __forceinline__ void load_split4(float *A, const void *__restrict__ src, int sf,
                                            const LevelGeom &g, int ry0, int rx0, float off,
                                            float scale) {
  constexpr int NG = G::RXP / 4, TOT = G::RY * NG;
  constexpr int PER = (TOT + kMgThreads - 1) / kMgThreads;
  const int tid = threadIdx.y * kBX + threadIdx.x;
  float4 v[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int idx = tid + i * kMgThreads;
    const int y = idx / NG, q = idx - y * NG;
    const int gy = ry0 + y, gx = rx0 + 4 * q;
    const bool in = idx < TOT && gy >= 0 && gy < g.H && gx >= 0 && gx < g.W;
    v[i] = in ? s_ld4(src, (size_t)gy * g.W + gx, sf) : make_float4(off, off, off, off);
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int idx = tid + i * kMgThreads;
    if (idx < TOT) {
      const int y = idx / NG, q = idx - y * NG;
      float *row = A + y * G::S + 4 + 2 * q;
      *reinterpret_cast<float2 *>(row) = make_float2((v[i].x - off) * scale, (v[i].z - off) * scale);
      *reinterpret_cast<float2 *>(row + G::PLANE) =
          make_float2((v[i].y - off) * scale, (v[i].w - off) * scale);
    }
  }
  zero_pads<G>(A);
}

// 16-byte paths need rows that start on 16 bytes: W % 4 == 0 (channel planes
// are then 16-byte multiples as well; level arrays are 256-byte aligned).
__device__ __forceinline__ bool vec4_ok(const LevelGeom &g) { return (g.W & 3) == 0; }

// (src - off) * scale for cells inside the grid, 0 outside.
template <class G>
__device__ __forceinline__ void load_tile(float *A, const void *__restrict__ src, int sf,
                                          const LevelGeom &g, int ry0, int rx0, float off,
                                          float scale) {
  if (vec4_ok(g)) load_split4<G>(A, src, sf, g, ry0, rx0, off, scale);
  else load_split<G>(A, src, sf, g, ry0, rx0, off, scale);
}

// Writes the output tile (region rows HY.., columns HX..) of U to dst.
template <class G>
__device__ __forceinline__ void store_tile(const float *U, void *dst, int sf, const LevelGeom &g,
                                           int ty0, int tx0) {
  const int tid = threadIdx.y * kBX + threadIdx.x;
  if (vec4_ok(g)) {
    constexpr int NG = G::TX / 4, TOT = G::TY * NG;
#pragma unroll
    for (int i = 0; i < TOT / kMgThreads; ++i) {
      const int idx = tid + i * kMgThreads;
      const int y = idx / NG, q = idx - y * NG;
      const int gy = ty0 + y, gx = tx0 + 4 * q;
      if (gy >= g.H || gx >= g.W) continue;
      const float *row = U + (y + G::HY) * G::S + 4 + ((4 * q + G::HX) >> 1);
      const float2 e = *reinterpret_cast<const float2 *>(row);
      const float2 o = *reinterpret_cast<const float2 *>(row + G::PLANE);
      s_st4(dst, (size_t)gy * g.W + gx, make_float4(e.x, o.x, e.y, o.y), sf);
    }
    return;
  }
  for (int y = threadIdx.y; y < G::TY; y += kBY)
    for (int x = threadIdx.x; x < G::TX; x += kBX) {
      const int gy = ty0 + y, gx = tx0 + x;
      if (gy < g.H && gx < g.W)
        s_st(dst, (size_t)gy * g.W + gx, at<G>(const_cast<float *>(U), y + G::HY, x + G::HX), sf);
    }
}

template <class G>
__device__ __forceinline__ void zero_split(float *A) {
  const int tid = threadIdx.y * kBX + threadIdx.x;
  float4 *a4 = reinterpret_cast<float4 *>(A);
  for (int i = tid; i < G::ARR / 4; i += kMgThreads) a4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Face factors of the region's rows and columns, so that a cell's coefficients
// are products: e = wy(I) cE(J), w = wy(I) cW(J), s = wx(J) cS(I), n = wx(J) cN(I)
// (all zero for cells outside the grid). Columns are stored per plane.
template <class G>
struct Factors {
  float wy[G::RY], cS[G::RY], cN[G::RY];
  float4 wx[2][G::NQ], cE[2][G::NQ], cW[2][G::NQ];
};

template <class G>
__device__ __forceinline__ void build_factors(Factors<G> *fa, const LevelGeom &g, int ry0, int rx0) {
  const int tid = threadIdx.y * kBX + threadIdx.x;
  for (int y = tid; y < G::RY; y += kMgThreads) {
    const int gy = ry0 + y;
    const bool in = gy >= 0 && gy < g.H;
    fa->wy[y] = in ? wyf(g, gy) : 0.f;
    fa->cS[y] = (in && gy + 1 < g.H) ? (gy + 1 == g.H - 1 ? g.ey : 1.f) : 0.f;
    fa->cN[y] = (in && gy > 0) ? (gy == g.H - 1 ? g.ey : 1.f) : 0.f;
  }
  float *wx = reinterpret_cast<float *>(fa->wx), *cE = reinterpret_cast<float *>(fa->cE),
        *cW = reinterpret_cast<float *>(fa->cW);
  for (int x = tid; x < G::RXP; x += kMgThreads) {
    const int gx = rx0 + x;
    const bool in = gx >= 0 && gx < g.W;
    const int o = (x & 1) * G::NC + (x >> 1);
    wx[o] = in ? wxf(g, gx) : 0.f;
    cE[o] = (in && gx + 1 < g.W) ? (gx + 1 == g.W - 1 ? g.ex : 1.f) : 0.f;
    cW[o] = (in && gx > 0) ? (gx == g.W - 1 ? g.ex : 1.f) : 0.f;
  }
}

// One red-black half-sweep (colour col: (gy + gx) & 1 == col) over rows 1..RY-2
// of the region. A work unit is one quad of same-colour cells of a row: away
// from the grid border all coefficients are 1; near it they come from the
// factor tables (cells outside the grid keep their value).
template <class G>
__device__ __forceinline__ void half_sweep(float *U, const float *F, const Factors<G> *fa,
                                           const LevelGeom &g, int ry0, int rx0, int col,
                                           float omega) {
  constexpr int NU_ = (G::RY - 2) * G::NQ;
  const int tid = threadIdx.y * kBX + threadIdx.x;
  const int lane = threadIdx.x;
#pragma unroll 1
  for (int it = 0; it < (NU_ + kMgThreads - 1) / kMgThreads; ++it) {
    const int idx = tid + kMgThreads * it;
    const bool act = idx < NU_;
    const int y = act ? 1 + idx / G::NQ : 1;
    const int q = act ? idx - (y - 1) * G::NQ : 0;
    const int m0 = q * 4;
    const int gy = ry0 + y;
    const bool updE = ((gy + rx0) & 1) == col;  // colour of the even-x cells of this row
    const int tp = updE ? 0 : G::PLANE, qp = updE ? G::PLANE : 0;
    float *Trow = U + tp + y * G::S + 4;
    const float *Qrow = U + qp + y * G::S + 4;
    const float4 qv = *reinterpret_cast<const float4 *>(Qrow + m0);
    // the one neighbour outside the quad comes from the adjacent lane's quad
    // (same row) or, at a row or warp edge, from shared memory
    float left = __shfl_up_sync(0xffffffffu, qv.w, 1);
    float right = __shfl_down_sync(0xffffffffu, qv.x, 1);
    if (updE && (lane == 0 || q == 0)) left = Qrow[m0 - 1];
    if (!updE && (lane == kBX - 1 || q == G::NQ - 1)) right = Qrow[m0 + 4];
    const float qx = updE ? left : right;
    const float4 up = *reinterpret_cast<const float4 *>(Trow - G::S + m0);
    const float4 dn = *reinterpret_cast<const float4 *>(Trow + G::S + m0);
    const float4 f = *reinterpret_cast<const float4 *>(F + tp + y * G::S + 4 + m0);
    // west / east neighbours of the four cells
    const float w0 = updE ? qx : qv.x, w1 = updE ? qv.x : qv.y, w2 = updE ? qv.y : qv.z,
                w3 = updE ? qv.z : qv.w;
    const float e0 = updE ? qv.x : qv.y, e1 = updE ? qv.y : qv.z, e2 = updE ? qv.z : qv.w,
                e3 = updE ? qv.w : qx;
    const int gx0 = rx0 + 2 * m0;
    float4 r;
    const bool fast = gy >= 1 && gy <= g.H - 3 && gx0 >= 1 && gx0 + 7 <= g.W - 3;
    if (__all_sync(0xffffffffu, fast || !act)) {  // warp-uniform: no predicated border path
      r.x = 0.25f * ((w0 + e0) + (up.x + dn.x) - f.x);
      r.y = 0.25f * ((w1 + e1) + (up.y + dn.y) - f.y);
      r.z = 0.25f * ((w2 + e2) + (up.z + dn.z) - f.z);
      r.w = 0.25f * ((w3 + e3) + (up.w + dn.w) - f.w);
      if (omega != 1.f) {  // u + omega (u_GS - u)
        const float4 old = *reinterpret_cast<const float4 *>(Trow + m0);
        r.x = fmaf(omega, r.x - old.x, old.x);
        r.y = fmaf(omega, r.y - old.y, old.y);
        r.z = fmaf(omega, r.z - old.z, old.z);
        r.w = fmaf(omega, r.w - old.w, old.w);
      }
    } else {
      const int pl = updE ? 0 : 1;
      const float wy = fa->wy[y], cS = fa->cS[y], cN = fa->cN[y];
      const float4 wx = fa->wx[pl][q], cE = fa->cE[pl][q], cW = fa->cW[pl][q];
      const float4 old = *reinterpret_cast<const float4 *>(Trow + m0);
#define GDGS_CELL(C, W_, E_)                                                                  \
  {                                                                                          \
    const float ae = wy * cE.C, aw = wy * cW.C, as = wx.C * cS, an = wx.C * cN;              \
    const float d = (ae + aw) + (as + an);                                                   \
    r.C = d > 0.f ? (ae * E_ + aw * W_ + as * dn.C + an * up.C - f.C) / d : old.C;           \
  }
      GDGS_CELL(x, w0, e0) GDGS_CELL(y, w1, e1) GDGS_CELL(z, w2, e2) GDGS_CELL(w, w3, e3)
#undef GDGS_CELL
      r.x = fmaf(omega, r.x - old.x, old.x);
      r.y = fmaf(omega, r.y - old.y, old.y);
      r.z = fmaf(omega, r.z - old.z, old.z);
      r.w = fmaf(omega, r.w - old.w, old.w);
    }
    if (act) *reinterpret_cast<float4 *>(Trow + m0) = r;
  }
}

// The first half-sweep of a down pass (colour col) on u = 0: the same values
// half_sweep computes from zero neighbours, omega (-f / d) with the same
// rounding (-f / 4 away from the border), from f alone; the other colour and the
// halo stay 0.
template <class G>
__device__ __forceinline__ void half_sweep_from_zero(float *U, const float *F,
                                                     const Factors<G> *fa, const LevelGeom &g,
                                                     int ry0, int rx0, int col, float omega) {
  constexpr int NU_ = (G::RY - 2) * G::NQ;
  const int tid = threadIdx.y * kBX + threadIdx.x;
  for (int idx = tid; idx < NU_; idx += kMgThreads) {
    const int y = 1 + idx / G::NQ;
    const int q = idx - (y - 1) * G::NQ;
    const int m0 = q * 4;
    const int gy = ry0 + y;
    const bool updE = ((gy + rx0) & 1) == col;
    const int tp = updE ? 0 : G::PLANE;
    const float4 f = *reinterpret_cast<const float4 *>(F + tp + y * G::S + 4 + m0);
    const int gx0 = rx0 + 2 * m0;
    float4 r;
    if (gy >= 1 && gy <= g.H - 3 && gx0 >= 1 && gx0 + 7 <= g.W - 3) {
      r = make_float4(0.25f * (0.f - f.x), 0.25f * (0.f - f.y), 0.25f * (0.f - f.z),
                      0.25f * (0.f - f.w));
      if (omega != 1.f)
        r = make_float4(__fmul_rn(omega, r.x), __fmul_rn(omega, r.y), __fmul_rn(omega, r.z),
                        __fmul_rn(omega, r.w));
    } else {
      const int pl = updE ? 0 : 1;
      const float wy = fa->wy[y], cS = fa->cS[y], cN = fa->cN[y];
      const float4 wx = fa->wx[pl][q], cE = fa->cE[pl][q], cW = fa->cW[pl][q];
#define GDGS_CELL0(C)                                                              \
  {                                                                               \
    const float ae = wy * cE.C, aw = wy * cW.C, as = wx.C * cS, an = wx.C * cN;   \
    const float d = (ae + aw) + (as + an);                                        \
    r.C = d > 0.f ? __fmul_rn(omega, (0.f - f.C) / d) : 0.f;                      \
  }
      GDGS_CELL0(x) GDGS_CELL0(y) GDGS_CELL0(z) GDGS_CELL0(w)
#undef GDGS_CELL0
    }
    *reinterpret_cast<float4 *>(U + tp + y * G::S + 4 + m0) = r;
  }
}

// Residual f - L u at region cell (y, x) (grid cell (gy, gx) in the grid).
template <class G>
__device__ __forceinline__ float tile_residual(float *U, float *F, const LevelGeom &g, int y, int x,
                                               int gy, int gx) {
  return residual(g, gy, gx, at<G>(U, y, x), at<G>(U, y, x + 1), at<G>(U, y, x - 1),
                  at<G>(U, y + 1, x), at<G>(U, y - 1, x), at<G>(F, y, x));
}

// Sum of the four children's residuals for each coarse cell under the output
// tile (ty0, tx0) -> fc. A work unit is a pair of coarse cells (fine columns
// J .. J+3 of rows I, I+1); away from the border (warp-uniform test) its eight
// residuals come from 8-byte loads of the split planes, elsewhere from the
// general cell formula.
template <class G>
__device__ __forceinline__ void restrict_tile(float *U, float *F, const LevelGeom &g,
                                              const LevelGeom &gc, int ty0, int tx0, void *fc,
                                              int sf, float fout) {
  const int ry0 = ty0 - G::HY, rx0 = tx0 - G::HX;
  const int tid = threadIdx.y * kBX + threadIdx.x;
  constexpr int CW2 = G::TX / 4, NP = (G::TY / 2) * CW2;
  static_assert(NP % 32 == 0, "whole warps per pass");
#pragma unroll
  for (int i = 0; i < (NP + kMgThreads - 1) / kMgThreads; ++i) {
    const int idx = tid + i * kMgThreads;
    if (idx >= NP) break;  // whole warps
    const int cy = idx / CW2, cq = idx - cy * CW2;
    const int CI = (ty0 >> 1) + cy, CJ = (tx0 >> 1) + 2 * cq;
    const int I = 2 * CI, J = 2 * CJ;
    const bool valid = CI < gc.H && CJ < gc.W;
    const bool fast = valid && I >= 1 && I + 1 <= g.H - 3 && J >= 1 && J + 3 <= g.W - 3;
    if (__all_sync(0xffffffffu, fast || !valid)) {
      if (!valid) continue;
      const int y = I - ry0, m = (J - rx0) >> 1;  // m even: 8-byte aligned pairs
      const float *E = U + y * G::S + 4 + m, *O = E + G::PLANE;
      const float *FE = F + y * G::S + 4 + m, *FO = FE + G::PLANE;
      float2 e[4], o[4];  // rows y-1 .. y+2, cells m, m+1 of each plane
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        e[r] = *reinterpret_cast<const float2 *>(E + (r - 1) * G::S);
        o[r] = *reinterpret_cast<const float2 *>(O + (r - 1) * G::S);
      }
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const int r = kk + 1;
        const float oL = O[kk * G::S - 1], eR = E[kk * G::S + 2];
        const float2 fe = *reinterpret_cast<const float2 *>(FE + kk * G::S);
        const float2 fo = *reinterpret_cast<const float2 *>(FO + kk * G::S);
        float u = e[r].x;
        s0 += fe.x - (((o[r].x - u) + (oL - u)) + ((e[r + 1].x - u) + (e[r - 1].x - u)));
        u = o[r].x;
        s0 += fo.x - (((e[r].y - u) + (e[r].x - u)) + ((o[r + 1].x - u) + (o[r - 1].x - u)));
        u = e[r].y;
        s1 += fe.y - (((o[r].y - u) + (o[r].x - u)) + ((e[r + 1].y - u) + (e[r - 1].y - u)));
        u = o[r].y;
        s1 += fo.y - (((eR - u) + (e[r].y - u)) + ((o[r + 1].y - u) + (o[r - 1].y - u)));
      }
      s_st(fc, (size_t)CI * gc.W + CJ, s0 * fout, sf);
      s_st(fc, (size_t)CI * gc.W + CJ + 1, s1 * fout, sf);
    } else if (valid) {
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const int cj = CJ + d;
        if (cj >= gc.W) break;
        float sum = 0.f;
#pragma unroll
        for (int di = 0; di < 2; ++di)
#pragma unroll
          for (int dj = 0; dj < 2; ++dj) {
            const int gy = I + di, gx = 2 * cj + dj;
            if (gy < g.H && gx < g.W) sum += tile_residual<G>(U, F, g, gy - ry0, gx - rx0, gy, gx);
          }
        s_st(fc, (size_t)CI * gc.W + cj, sum * fout, sf);
      }
    }
  }
}

// Coarse values around the region: rows cy0.., columns cx0.. of the coarse level.
template <class G>
__device__ __forceinline__ void load_coarse(float *EC, const void *__restrict__ uc, int sf,
                                            const LevelGeom &gc, int cy0, int cx0) {
  constexpr int NY = (G::CRY + kBY - 1) / kBY, NX = (G::CRX + kBX - 1) / kBX;
  float v[NY][NX];
#pragma unroll
  for (int i = 0; i < NY; ++i) {
    const int y = threadIdx.y + kBY * i, gy = cy0 + y;
    const bool rin = y < G::CRY && gy >= 0 && gy < gc.H;
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      const int x = threadIdx.x + kBX * j, gx = cx0 + x;
      v[i][j] = (rin && x < G::CRX && gx >= 0 && gx < gc.W) ? s_ld(uc, (size_t)gy * gc.W + gx, sf) : 0.f;
    }
  }
#pragma unroll
  for (int i = 0; i < NY; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      const int y = threadIdx.y + kBY * i, x = threadIdx.x + kBX * j;
      if (y < G::CRY && x < G::CRX) EC[y * G::CRX + x] = v[i][j];
    }
}

// U += P(EC) on the region. Work unit: the 8 cells (4 even-x, 4 odd-x) of a row
// that share coarse columns m0 .. m0 + 5 of the box; away from the border the
// weights are the regular 3/4, 1/4 pattern.
template <class G>
__device__ __forceinline__ void prolong_tile(float *U, const float *EC, const LevelGeom &g,
                                             const LevelGeom &gc, int ry0, int rx0, int cy0, int cx0) {
  const int tid = threadIdx.y * kBX + threadIdx.x;
  for (int idx = tid; idx < G::RY * G::NQ; idx += kMgThreads) {
    const int y = idx / G::NQ;
    const int m0 = (idx - y * G::NQ) * 4;
    const int gy = ry0 + y;
    if (gy < 0 || gy >= g.H) continue;
    const int gx0 = rx0 + 2 * m0;
    if (gy >= 2 && gy <= g.H - 4 && gx0 >= 2 && gx0 + 7 <= g.W - 4) {
      const int r0 = (gy >> 1) - cy0;
      const int r1 = (gy & 1) ? r0 + 1 : r0 - 1;
      const int c0 = (gx0 >> 1) - 1 - cx0;  // coarse column of cell gx0 minus one
      // c0 = m0 is a multiple of 4 and CRX too: 16- and 8-byte loads
      const float4 a4 = *reinterpret_cast<const float4 *>(EC + r0 * G::CRX + c0);
      const float2 a2 = *reinterpret_cast<const float2 *>(EC + r0 * G::CRX + c0 + 4);
      const float4 b4 = *reinterpret_cast<const float4 *>(EC + r1 * G::CRX + c0);
      const float2 b2 = *reinterpret_cast<const float2 *>(EC + r1 * G::CRX + c0 + 4);
      const float v[6] = {0.75f * a4.x + 0.25f * b4.x, 0.75f * a4.y + 0.25f * b4.y,
                          0.75f * a4.z + 0.25f * b4.z, 0.75f * a4.w + 0.25f * b4.w,
                          0.75f * a2.x + 0.25f * b2.x, 0.75f * a2.y + 0.25f * b2.y};
      float *Ee = U + y * G::S + 4 + m0;
      float *Eo = U + G::PLANE + y * G::S + 4 + m0;
      float4 e = *reinterpret_cast<float4 *>(Ee);
      float4 o = *reinterpret_cast<float4 *>(Eo);
      e.x += 0.75f * v[1] + 0.25f * v[0];
      e.y += 0.75f * v[2] + 0.25f * v[1];
      e.z += 0.75f * v[3] + 0.25f * v[2];
      e.w += 0.75f * v[4] + 0.25f * v[3];
      o.x += 0.75f * v[1] + 0.25f * v[2];
      o.y += 0.75f * v[2] + 0.25f * v[3];
      o.z += 0.75f * v[3] + 0.25f * v[4];
      o.w += 0.75f * v[4] + 0.25f * v[5];
      *reinterpret_cast<float4 *>(Ee) = e;
      *reinterpret_cast<float4 *>(Eo) = o;
    } else {
      const P1 py = prolong1d(gy, g.shift, g.H0, gc.H);
      const float *ra = EC + (py.i0 - cy0) * G::CRX;
      const float *rb = EC + (py.i1 - cy0) * G::CRX;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int x = 2 * m0 + (i & 3) * 2 + (i >> 2);
        const int gx = rx0 + x;
        if (gx < 0 || gx >= g.W) continue;
        const P1 px = prolong1d(gx, g.shift, g.W0, gc.W);
        const int j0 = px.i0 - cx0, j1 = px.i1 - cx0;
        const float a0 = ra[j0] + px.w1 * (ra[j1] - ra[j0]);
        const float a1 = rb[j0] + px.w1 * (rb[j1] - rb[j0]);
        at<G>(U, y, x) += a0 + py.w1 * (a1 - a0);
      }
    }
  }
}

// Finest level, W % 4 == 0: u_{k+1} = u_k + e in float-float, r_{k+1} = r_k - L e
// (r_k is F, e is U), the sums of u_{k+1} and of r_{k+1}^2; 16-byte global
// accesses, residuals from the split planes away from the border (warp-uniform).
template <class G>
__device__ __forceinline__ void finest_epilogue4(const float *U, const float *F, const LevelGeom &g,
                                                 int ty0, int tx0, int k, float *uh, float *ul,
                                                 float *rn, Ctrl *ctrl, int c, float inv_s) {
  constexpr int NG = G::TX / 4, TOT = G::TY * NG, PER = TOT / kMgThreads;
  const int tid = threadIdx.y * kBX + threadIdx.x;
  float4 vh[PER], vl[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int idx = tid + i * kMgThreads;
    const int y = idx / NG, q = idx - y * NG;
    const int gy = ty0 + y, gx = tx0 + 4 * q;
    const bool in = k > 0 && gy < g.H && gx < g.W;
    const size_t p = (size_t)gy * g.W + gx;
    vh[i] = in ? *reinterpret_cast<const float4 *>(uh + p) : make_float4(0.f, 0.f, 0.f, 0.f);
    vl[i] = in ? *reinterpret_cast<const float4 *>(ul + p) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  float su = 0.f, rn2 = 0.f;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int idx = tid + i * kMgThreads;
    const int y = idx / NG, q = idx - y * NG;
    const int gy = ty0 + y, gx = tx0 + 4 * q;
    const bool valid = gy < g.H && gx < g.W;
    const int yy = y + G::HY, xx = 4 * q + G::HX, m = xx >> 1;
    const float *E = U + yy * G::S + 4 + m, *O = E + G::PLANE;
    const float2 e = *reinterpret_cast<const float2 *>(E);
    const float2 o = *reinterpret_cast<const float2 *>(O);
    float r[4] = {0.f, 0.f, 0.f, 0.f};
    const bool fast = valid && gy >= 1 && gy <= g.H - 3 && gx >= 1 && gx + 3 <= g.W - 3;
    if (__all_sync(0xffffffffu, fast || !valid)) {
      if (valid) {
        const float oL = O[-1], eR = E[2];
        const float2 eN = *reinterpret_cast<const float2 *>(E - G::S);
        const float2 eS = *reinterpret_cast<const float2 *>(E + G::S);
        const float2 oN = *reinterpret_cast<const float2 *>(O - G::S);
        const float2 oS = *reinterpret_cast<const float2 *>(O + G::S);
        const float *FE = F + yy * G::S + 4 + m;
        const float2 fe = *reinterpret_cast<const float2 *>(FE);
        const float2 fo = *reinterpret_cast<const float2 *>(FE + G::PLANE);
        r[0] = fe.x - (((o.x - e.x) + (oL - e.x)) + ((eS.x - e.x) + (eN.x - e.x)));
        r[1] = fo.x - (((e.y - o.x) + (e.x - o.x)) + ((oS.x - o.x) + (oN.x - o.x)));
        r[2] = fe.y - (((o.y - e.y) + (o.x - e.y)) + ((eS.y - e.y) + (eN.y - e.y)));
        r[3] = fo.y - (((eR - o.y) + (e.y - o.y)) + ((oS.y - o.y) + (oN.y - o.y)));
      }
    } else if (valid) {
#pragma unroll
      for (int d = 0; d < 4; ++d)
        r[d] = tile_residual<G>(const_cast<float *>(U), const_cast<float *>(F), g, yy, xx + d, gy,
                                gx + d);
    }
    if (!valid) continue;
    const float ev[4] = {e.x * inv_s, o.x * inv_s, e.y * inv_s, o.y * inv_s};
#pragma unroll
    for (int d = 0; d < 4; ++d) r[d] *= inv_s;
    float hv[4] = {vh[i].x, vh[i].y, vh[i].z, vh[i].w}, lv[4] = {vl[i].x, vl[i].y, vl[i].z, vl[i].w};
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      ds_add(hv[d], lv[d], ev[d]);
      su += hv[d] + lv[d];
      rn2 = fmaf(r[d], r[d], rn2);
    }
    const size_t p = (size_t)gy * g.W + gx;
    *reinterpret_cast<float4 *>(uh + p) = make_float4(hv[0], hv[1], hv[2], hv[3]);
    *reinterpret_cast<float4 *>(ul + p) = make_float4(lv[0], lv[1], lv[2], lv[3]);
    *reinterpret_cast<float4 *>(rn + p) = make_float4(r[0], r[1], r[2], r[3]);
  }
  block_sum2(su, rn2);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    atomicAdd(&ctrl->sum_u[k + 1][c], (double)su);
    atomicAdd(&ctrl->rnorm2[k + 1], (double)rn2);
  }
}

// ------------------------------------------------------------------ level kernels

// Arrays of a level in the storage format sf (corrections, coarse right-hand
// sides) and in FP32 (the finest level's r_k and iterate). Cycle k solves for
// s_k e, s_k = ctrl->escale[k] a power of two that brings the RMS of r_k near 1;
// a level l >= 1 stores its right-hand side times 4^-l. Both scalings are exact,
// and they keep FP16 values in range.
struct LvArgs {
  LevelGeom g, gc;
  const void *f;     // right-hand side times 4^-l (level >= 1)
  void *u;           // correction of this level after the down pass
  void *uo;          // correction after the up pass (levels >= 1): a separate array, because
                     // an up CTA reads its halo from u while its neighbours write their tiles
  void *fc;          // coarse right-hand side times 4^-(l+1) (down)
  const void *uc;    // coarse correction (up)
  int sf;            // GDGS_STORAGE_* of f, u, uo, fc, uc
  float fin, fout;   // 4^l and 4^-(l+1)
  int level0;        // finest level: right-hand side r_k, u update
  const float *rho;  // r_0
  float *rb[2];      // r_{k+1} is written to rb[k & 1]
  float *uhi, *ulo;  // float-float iterate
  float omega;       // smoother over-relaxation
};

// Right-hand side of this level for channel c in cycle k: (src - off) * scale.
// r_0 = rho - mean(rho): a field whose sum is not zero (possible for the
// composite of Laplacian values) is solved in the least-squares sense.
struct Rhs {
  const void *src;
  int sf;
  float off, scale;
};

__device__ __forceinline__ Rhs rhs_of(const LvArgs &a, const Ctrl *ctrl, int k, int c) {
  Rhs r;
  if (!a.level0) {
    r.src = s_at(a.f, (size_t)c * a.g.plane, a.sf);
    r.sf = a.sf;
    r.off = 0.f;
    r.scale = a.fin;
    return r;
  }
  r.src = (k == 0 ? a.rho : a.rb[(k - 1) & 1]) + (size_t)c * a.g.plane;
  r.sf = GDGS_STORAGE_F32;
  r.off = k == 0 ? ctrl->rho_mean[c] : 0.f;
  r.scale = ctrl->escale[k];
  return r;
}

// Down: nu1 sweeps on L u = f from u = 0, write u, restrict f - L u.
template <int NU, int TY_, int TX_>
__global__ void __launch_bounds__(kMgThreads) mg_down_kernel(LvArgs a, Ctrl *ctrl, int k_in, int first) {
  griddep_enter();
  using G = Geo<NU, TY_, TX_>;
  extern __shared__ float4 sm4[];
  float *F = reinterpret_cast<float *>(sm4), *U = F + G::ARR;
  Factors<G> *fa = reinterpret_cast<Factors<G> *>(U + G::ARR);
  const int k = cycle_index(ctrl, k_in);
  if (a.level0 ? *(volatile int *)&ctrl->stopped != 0 : block_should_stop(ctrl, k, first)) return;
  const LevelGeom &g = a.g;
  const int c = blockIdx.z;
  const int ty0 = blockIdx.y * G::TY, tx0 = blockIdx.x * G::TX;
  const int ry0 = ty0 - G::HY, rx0 = tx0 - G::HX;
  const Rhs rh = rhs_of(a, ctrl, k, c);
  load_tile<G>(F, rh.src, rh.sf, g, ry0, rx0, rh.off, rh.scale);
  zero_split<G>(U);
  build_factors<G>(fa, g, ry0, rx0);
  __syncthreads();
  half_sweep_from_zero<G>(U, F, fa, g, ry0, rx0, 0, a.omega);
  __syncthreads();
#pragma unroll
  for (int s = 1; s < 2 * NU; ++s) {
    half_sweep<G>(U, F, fa, g, ry0, rx0, s & 1, a.omega);
    __syncthreads();
  }
  store_tile<G>(U, s_at(a.u, (size_t)c * g.plane, a.sf), a.sf, g, ty0, tx0);
  restrict_tile<G>(U, F, g, a.gc, ty0, tx0, s_at(a.fc, (size_t)c * a.gc.plane, a.sf), a.sf, a.fout);
}

// Up: u += P u_{l+1}, nu2 sweeps, write u. On the finest level instead:
// u_{k+1} = u_k + e (float-float), r_{k+1} = r_k - L e, ||r_{k+1}||^2, sum(u_{k+1}).
template <int NU, int TY_, int TX_>
__global__ void __launch_bounds__(kMgThreads, 4) mg_up_kernel(LvArgs a, Ctrl *ctrl, int k_in) {
  griddep_enter();
  using G = Geo<NU, TY_, TX_>;
  extern __shared__ float4 sm4[];
  float *F = reinterpret_cast<float *>(sm4), *U = F + G::ARR, *EC = U + G::ARR;
  Factors<G> *fa = reinterpret_cast<Factors<G> *>(EC + G::CRY * G::CRX + (4 - (G::CRY * G::CRX) % 4) % 4);
  const int k = cycle_index(ctrl, k_in);
  if (block_should_stop(ctrl, k, 0)) return;
  const LevelGeom &g = a.g;
  const int c = blockIdx.z;
  const int ty0 = blockIdx.y * G::TY, tx0 = blockIdx.x * G::TX;
  const int ry0 = ty0 - G::HY, rx0 = tx0 - G::HX;
  const int cy0 = (ry0 >> 1) - 1, cx0 = (rx0 >> 1) - 1;
  const Rhs rh = rhs_of(a, ctrl, k, c);
  load_tile<G>(F, rh.src, rh.sf, g, ry0, rx0, rh.off, rh.scale);
  load_tile<G>(U, s_at(a.u, (size_t)c * g.plane, a.sf), a.sf, g, ry0, rx0, 0.f, 1.f);
  load_coarse<G>(EC, s_at(a.uc, (size_t)c * a.gc.plane, a.sf), a.sf, a.gc, cy0, cx0);
  build_factors<G>(fa, g, ry0, rx0);
  __syncthreads();
  prolong_tile<G>(U, EC, g, a.gc, ry0, rx0, cy0, cx0);
  __syncthreads();
#pragma unroll
  for (int s = 0; s < 2 * NU; ++s) {
    half_sweep<G>(U, F, fa, g, ry0, rx0, s & 1, a.omega);
    __syncthreads();
  }
  if (!a.level0) {
    store_tile<G>(U, s_at(a.uo, (size_t)c * g.plane, a.sf), a.sf, g, ty0, tx0);
    return;
  }
  const size_t cb = (size_t)c * g.plane;
  float *uh = a.uhi + cb, *ul = a.ulo + cb, *rn = a.rb[k & 1] + cb;
  const float inv_s = 1.f / rh.scale;  // exact: a power of two
  if (vec4_ok(g)) {
    finest_epilogue4<G>(U, F, g, ty0, tx0, k, uh, ul, rn, ctrl, c, inv_s);
    return;
  }
  constexpr int NY = G::TY / kBY, NX = G::TX / kBX;
  float vh[NY][NX], vl[NY][NX];
#pragma unroll
  for (int i = 0; i < NY; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      const int gy = ty0 + threadIdx.y + kBY * i, gx = tx0 + threadIdx.x + kBX * j;
      const bool in = k > 0 && gy < g.H && gx < g.W;
      const size_t p = (size_t)gy * g.W + gx;
      vh[i][j] = in ? uh[p] : 0.f;
      vl[i][j] = in ? ul[p] : 0.f;
    }
  float su = 0.f, rn2 = 0.f;
#pragma unroll
  for (int i = 0; i < NY; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      const int y = threadIdx.y + kBY * i, x = threadIdx.x + kBX * j;
      const int gy = ty0 + y, gx = tx0 + x;
      if (gy >= g.H || gx >= g.W) continue;
      const size_t p = (size_t)gy * g.W + gx;
      const int yy = y + G::HY, xx = x + G::HX;
      float hi = vh[i][j], lo = vl[i][j];
      ds_add(hi, lo, at<G>(U, yy, xx) * inv_s);
      uh[p] = hi;
      ul[p] = lo;
      su += hi + lo;
      const float r = tile_residual<G>(U, F, g, yy, xx, gy, gx) * inv_s;
      rn[p] = r;
      rn2 = fmaf(r, r, rn2);
    }
  block_sum2(su, rn2);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    atomicAdd(&ctrl->sum_u[k + 1][c], (double)su);
    atomicAdd(&ctrl->rnorm2[k + 1], (double)rn2);
  }
}

template <class G>
struct DownShape {
  static constexpr size_t smem = 2 * G::ARR * sizeof(float) + sizeof(Factors<G>);
};
template <class G>
struct UpShape {
  static constexpr size_t smem =
      (2 * G::ARR + (G::CRY * G::CRX + 3) / 4 * 4) * sizeof(float) + sizeof(Factors<G>);
};

// ------------------------------------------------------------------ finest level: streaming warps
//
// The finest level has unit cells: every face coefficient is 1 inside the grid
// and 0 on its border. With W even and V(2, 1) its down and up passes run as
// register pipelines instead of tiles. A warp owns a strip of kStripW = 64
// columns (lane l holds the cell pair sx + 2l, sx + 2l + 1, one cell of each
// colour in every row) and streams down a segment of rows. Each step loads one
// row and moves every stage of the pass on by one row, every stage a row behind
// the one before it, so a stage finds the rows around its own in the state it
// needs: red-black ordering makes the wavefront give exactly the sweep-by-sweep
// result. Horizontal neighbours come by warp shuffle; there is no shared memory
// and no barrier. The outer lanes' shuffles and the rows above the first loaded
// one give wrong values, which move inward by one cell per stage, so a strip
// stores its middle 56 columns (strips overlap by 8) and a segment begins as
// many rows above its first output row as the pass has stages after the first.
// Steps whose rows, in strips whose columns, are all away from the grid border
// use the constant coefficients (the tiled kernels' fast formulas); the others
// take the tiled kernels' general cell formulas.

constexpr int kStripW = 64;          // columns per strip, two per lane
constexpr int kStripX = 4;           // halo columns on each side of a strip's output
constexpr int kStripOut = kStripW - 2 * kStripX;
constexpr int kStreamThreads = 128;  // four independent warps per CTA
constexpr int kStreamPre = 4;        // rows loaded ahead of their use, per stream (up pass)
constexpr int kStreamPreDown = 4;    // the same for the down pass's one input stream

struct StreamGrid {
  int nstrips, nseg, S;  // strips of kStripOut output columns, segments of S output rows (S % 8 == 0)
};

template <int SF>
__device__ __forceinline__ float2 s_ld2(const void *p, size_t i) {  // i even
  if (SF == GDGS_STORAGE_F32) return __ldg(reinterpret_cast<const float2 *>(reinterpret_cast<const float *>(p) + i));
  const unsigned r = __ldg(reinterpret_cast<const unsigned *>(reinterpret_cast<const unsigned short *>(p) + i));
  if (SF == GDGS_STORAGE_BF16) return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&r));
  return __half22float2(*reinterpret_cast<const __half2 *>(&r));
}

template <int SF>
__device__ __forceinline__ void s_st2(void *p, size_t i, float2 v) {  // i even
  if (SF == GDGS_STORAGE_F32) {
    *reinterpret_cast<float2 *>(reinterpret_cast<float *>(p) + i) = v;
  } else if (SF == GDGS_STORAGE_BF16) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(v.x, v.y);
    *reinterpret_cast<unsigned *>(reinterpret_cast<unsigned short *>(p) + i) = *reinterpret_cast<const unsigned *>(&b);
  } else {
    const __half2 b = __floats2half2_rn(v.x, v.y);
    *reinterpret_cast<unsigned *>(reinterpret_cast<unsigned short *>(p) + i) = *reinterpret_cast<const unsigned *>(&b);
  }
}

template <int I>
__device__ __forceinline__ float &cell(float2 &v) {
  if constexpr (I == 0) return v.x;
  else return v.y;
}

// West and east neighbours of cell I of a lane's pair in row v: one is the
// lane's other cell, the other that of the adjacent lane (the outer lanes get
// their own value back: wrong, and inside the strip's halo).
template <int I>
__device__ __forceinline__ void horiz(const float2 &v, float &w, float &e) {
  if constexpr (I == 0) {
    w = __shfl_up_sync(0xffffffffu, v.y, 1);
    e = v.y;
  } else {
    w = v.x;
    e = __shfl_down_sync(0xffffffffu, v.x, 1);
  }
}

// Cell formulas. Each is written with explicit roundings (no a * b + c for the
// compiler to fuse or not), so it is one sequence of operations wherever it is
// inlined, and which formula a cell gets depends on the cell's position alone,
// never on the step, strip or segment computing it. So a cell computed by two
// strips or segments gets the same bits in both, and the update of u and the
// residuals of the cells next to it use one value of e.
//
// A full cell (all four face coefficients 1) takes the tiled kernels' interior
// formula; the others the general form of the same operator, with the face
// coefficients of coef() and 1 / (their sum) as a correctly rounded reciprocal
// (0 outside the grid, where a cell stays 0). On the finest level the
// coefficients are 0 or 1; on a coarser one the cells next to a narrow last row
// or column have others.

// Rows and columns whose cells have all four face coefficients 1: neighbours on
// both sides, and none of them the narrow last cell. L0: the finest level, whose
// cells are all full-size (its geometry constants are then known when compiling).
template <bool L0>
__device__ __forceinline__ bool full_row(const LevelGeom &g, int y) {
  return y >= 1 && y <= g.H - 2 && (L0 || y <= g.H - 3 || g.lasty == 1.f);
}
template <bool L0>
__device__ __forceinline__ bool full_col(const LevelGeom &g, int x) {
  return x >= 1 && x <= g.W - 2 && (L0 || x <= g.W - 3 || g.lastx == 1.f);
}

// 1 / d (0 for d = 0). On the finest level d counts neighbours (0 .. 4) and is
// looked up; elsewhere it is a sum of face coefficients.
template <bool L0>
__device__ __forceinline__ float inv_sum(float d) {
  if constexpr (L0) return d > 3.5f ? 0.25f : d > 2.5f ? (1.f / 3.f) : d > 1.5f ? 0.5f : d > 0.5f ? 1.f : 0.f;
  else return d > 0.f ? __frcp_rn(d) : 0.f;
}

__device__ __forceinline__ float gs_fast(float old, float w, float e, float n, float s, float f,
                                         float omega) {
  const float v = __fmul_rn(0.25f, __fsub_rn(__fadd_rn(__fadd_rn(w, e), __fadd_rn(n, s)), f));
  return omega != 1.f ? fmaf(omega, __fsub_rn(v, old), old) : v;
}

__device__ __forceinline__ float gs_mask(float old, float w, float e, float n, float s, float f,
                                         float cw, float ce, float cn, float cs, float invd,
                                         float omega) {
  float a = __fmul_rn(ce, e);
  a = fmaf(cw, w, a);
  a = fmaf(cs, s, a);
  a = fmaf(cn, n, a);
  const float v = __fmul_rn(__fsub_rn(a, f), invd);
  return fmaf(omega, __fsub_rn(v, old), old);
}

__device__ __forceinline__ float res_fast(float u, float e, float w, float s, float n, float f) {
  return __fsub_rn(f, __fadd_rn(__fadd_rn(__fsub_rn(e, u), __fsub_rn(w, u)),
                                __fadd_rn(__fsub_rn(s, u), __fsub_rn(n, u))));
}

__device__ __forceinline__ float res_mask(float u, float e, float w, float s, float n, float f,
                                          float cw, float ce, float cn, float cs) {
  float a = __fmul_rn(ce, __fsub_rn(e, u));
  a = fmaf(cw, __fsub_rn(w, u), a);
  a = fmaf(cs, __fsub_rn(s, u), a);
  a = fmaf(cn, __fsub_rn(n, u), a);
  return __fsub_rn(f, a);
}

// First half-sweep from e = 0: omega (-f / d).
__device__ __forceinline__ float gs0_fast(float f, float omega) {
  const float v = __fmul_rn(0.25f, -f);
  return omega != 1.f ? __fmul_rn(omega, v) : v;
}
__device__ __forceinline__ float gs0_mask(float f, float invd, float omega) {
  const float v = __fmul_rn(-f, invd);
  return omega != 1.f ? __fmul_rn(omega, v) : v;
}

// Regular prolongation weights: 3/4 on the nearer value, 1/4 on the farther.
__device__ __forceinline__ float lerp_reg(float near_, float far_) {
  return fmaf(0.75f, near_, __fmul_rn(0.25f, far_));
}

// Row factors of a row for the general steps: coef() of cell (y, x) is
// e = wy ce(x), w = wy cw(x), s = wx(x) cs, n = wx(x) cn.
struct RowMask {
  float wy, cn, cs;  // cell height (0 outside the grid); north / south face parts
  bool full;
};

template <bool L0>
__device__ __forceinline__ RowMask row_mask(const LevelGeom &g, int y) {
  RowMask r;
  const bool in = y >= 0 && y < g.H;
  const float ly = L0 ? 1.f : g.lasty, ey = L0 ? 1.f : g.ey;
  r.wy = in ? (y == g.H - 1 ? ly : 1.f) : 0.f;
  r.cn = (in && y > 0) ? (y == g.H - 1 ? ey : 1.f) : 0.f;
  r.cs = (in && y + 1 < g.H) ? (y + 1 == g.H - 1 ? ey : 1.f) : 0.f;
  r.full = full_row<L0>(g, y);
  return r;
}

// Per-warp strip and segment, the lane's pair and its column masks. Step
// modes: 0 = rows and columns all full, 1 = rows full (column masks per lane),
// 2 = general (row masks per row as well).
template <bool L0>
struct StripLane {
  int x;           // column of the lane's even cell
  bool in;         // the pair lies inside the grid (W even: both cells or neither)
  bool out;        // the lane stores its pair: a middle lane, inside the grid
  int y0, y1;      // output rows [y0, y1): y0 a multiple of 8, y1 <= H rounded up to even
  int sx;          // first column of the strip
  float wx[2];     // cell width (0 outside the grid), per cell
  float cw[2], ce[2];  // west / east face parts, per cell (coef() in a full row)
  float invd[2];   // 1 / (sum of the face coefficients) of each cell in a full row
  bool fcol[2];    // the cell's column is full

  // Smoother update of cell I of a row (row masks m used in mode 2 only).
  template <int MODE, int I>
  __device__ __forceinline__ float sweep(const RowMask &m, float old, float w, float e, float n,
                                         float s, float f, float omega) const {
    const float fast = gs_fast(old, w, e, n, s, f, omega);
    if constexpr (MODE == 0) {
      return fast;
    } else if constexpr (MODE == 1) {
      return fcol[I] ? fast : gs_mask(old, w, e, n, s, f, cw[I], ce[I], wx[I], wx[I], invd[I], omega);
    } else {
      const float cwm = __fmul_rn(cw[I], m.wy), cem = __fmul_rn(ce[I], m.wy);
      const float cnm = __fmul_rn(m.cn, wx[I]), csm = __fmul_rn(m.cs, wx[I]);
      const float id = inv_sum<L0>(__fadd_rn(__fadd_rn(cwm, cem), __fadd_rn(cnm, csm)));
      return (m.full && fcol[I]) ? fast : gs_mask(old, w, e, n, s, f, cwm, cem, cnm, csm, id, omega);
    }
  }

  template <int MODE, int I>
  __device__ __forceinline__ float sweep0(const RowMask &m, float f, float omega) const {
    const float fast = gs0_fast(f, omega);
    if constexpr (MODE == 0) {
      return fast;
    } else if constexpr (MODE == 1) {
      return fcol[I] ? fast : gs0_mask(f, invd[I], omega);
    } else {
      const float cwm = __fmul_rn(cw[I], m.wy), cem = __fmul_rn(ce[I], m.wy);
      const float cnm = __fmul_rn(m.cn, wx[I]), csm = __fmul_rn(m.cs, wx[I]);
      const float id = inv_sum<L0>(__fadd_rn(__fadd_rn(cwm, cem), __fadd_rn(cnm, csm)));
      return (m.full && fcol[I]) ? fast : gs0_mask(f, id, omega);
    }
  }

  // Residual of cell I (0 outside the grid: all masks 0 and f = 0 there).
  template <int MODE, int I>
  __device__ __forceinline__ float res(const RowMask &m, float u, float e, float w, float s, float n,
                                       float f) const {
    const float fast = res_fast(u, e, w, s, n, f);
    if constexpr (MODE == 0) {
      return fast;
    } else if constexpr (MODE == 1) {
      return fcol[I] ? fast : res_mask(u, e, w, s, n, f, cw[I], ce[I], wx[I], wx[I]);
    } else {
      const float cwm = __fmul_rn(cw[I], m.wy), cem = __fmul_rn(ce[I], m.wy);
      const float cnm = __fmul_rn(m.cn, wx[I]), csm = __fmul_rn(m.cs, wx[I]);
      return (m.full && fcol[I]) ? fast : res_mask(u, e, w, s, n, f, cwm, cem, cnm, csm);
    }
  }
};

template <bool L0>
__device__ __forceinline__ bool strip_lane(const LevelGeom &g, const StreamGrid &sg, StripLane<L0> &sl) {
  const int lane = threadIdx.x & 31;
  const int wid = blockIdx.x * (kStreamThreads / 32) + (threadIdx.x >> 5);
  if (wid >= sg.nstrips * sg.nseg) return false;
  const int seg = wid / sg.nstrips, strip = wid - seg * sg.nstrips;
  sl.sx = strip * kStripOut - kStripX;
  sl.x = sl.sx + 2 * lane;
  sl.in = sl.x >= 0 && sl.x < g.W;
  sl.out = sl.in && lane >= kStripX / 2 && lane < 32 - kStripX / 2;
  sl.y0 = seg * sg.S;
  sl.y1 = min(sl.y0 + sg.S, (g.H + 1) & ~1);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int x = sl.x + i;
    const float lx = L0 ? 1.f : g.lastx, ex = L0 ? 1.f : g.ex;
    sl.wx[i] = sl.in ? (x == g.W - 1 ? lx : 1.f) : 0.f;
    sl.cw[i] = (sl.in && x > 0) ? (x == g.W - 1 ? ex : 1.f) : 0.f;
    sl.ce[i] = (sl.in && x + 1 < g.W) ? (x + 1 == g.W - 1 ? ex : 1.f) : 0.f;
    sl.invd[i] = inv_sum<L0>(__fadd_rn(__fadd_rn(sl.cw[i], sl.ce[i]), __fadd_rn(sl.wx[i], sl.wx[i])));
    sl.fcol[i] = full_col<L0>(g, x);
  }
  return true;
}

// Down pass (nu1 = 2): stage 0 is the first half-sweep from e = 0 on row t;
// stages 1-3 the next half-sweeps on rows t-1 .. t-3; row t-3 is then final and
// stored; the residual of row t-4 is summed into the coarse right-hand side.
// E[j] and F[j] hold row t - j of e and of the right-hand side. L0: the finest
// level (right-hand side r_k in FP32); otherwise the level's stored right-hand
// side (format SF, times 4^-l).
template <int SF, bool L0>
struct DownStream {
  LevelGeom g, gc;
  StripLane<L0> sl;
  const void *src;
  float off, scale, omega, fout;
  void *u, *fc;
  float2 E[6], F[5], Q[kStreamPreDown];
  float rpair;

  __device__ __forceinline__ float2 load(int row) const {
    if (!(sl.in && row >= 0 && row < g.H)) return make_float2(0.f, 0.f);
    const size_t i = (size_t)row * g.W + sl.x;
    if constexpr (L0) return __ldg(reinterpret_cast<const float2 *>(static_cast<const float *>(src) + i));
    else return s_ld2<SF>(src, i);
  }

  template <int MODE, int PAR>
  __device__ __forceinline__ void step(int t) {
    constexpr int I = PAR;  // every stage of this step updates cell PAR of its row
#pragma unroll
    for (int j = 5; j > 0; --j) E[j] = E[j - 1];
#pragma unroll
    for (int j = 4; j > 0; --j) F[j] = F[j - 1];
    const float2 q = Q[0];
#pragma unroll
    for (int j = 0; j + 1 < kStreamPreDown; ++j) Q[j] = Q[j + 1];
    Q[kStreamPreDown - 1] = load(t + kStreamPreDown);
    const bool rin = MODE == 0 || (sl.in && t >= 0 && t < g.H);
    F[0] = rin ? make_float2(__fmul_rn(__fsub_rn(q.x, off), scale), __fmul_rn(__fsub_rn(q.y, off), scale))
               : make_float2(0.f, 0.f);
    E[0] = make_float2(0.f, 0.f);
    RowMask m[5];
    if constexpr (MODE == 2) {
#pragma unroll
      for (int s = 0; s < 5; ++s) m[s] = row_mask<L0>(g, t - s);
    }
    // stage 0: colour 0 of row t from zero
    cell<I>(E[0]) = sl.template sweep0<MODE, I>(m[0], cell<I>(F[0]), omega);
    // stages 1-3: colours 1, 0, 1 of rows t-1, t-2, t-3
#pragma unroll
    for (int s = 1; s <= 3; ++s) {
      float w, e;
      horiz<I>(E[s], w, e);
      cell<I>(E[s]) = sl.template sweep<MODE, I>(m[s], cell<I>(E[s]), w, e, cell<I>(E[s + 1]),
                                        cell<I>(E[s - 1]), cell<I>(F[s]), omega);
    }
    {
      const int y = t - 3;
      if (sl.out && y >= sl.y0 && y < sl.y1 && y < g.H) s_st2<SF>(u, (size_t)y * g.W + sl.x, E[3]);
    }
    // residual of row t-4, summed over 2 x 2 children into the coarse right-hand side
    const int y = t - 4;
    const float2 uu = E[4], n = E[5], so = E[3], f = F[4];
    const float wl = __shfl_up_sync(0xffffffffu, uu.y, 1);
    const float er = __shfl_down_sync(0xffffffffu, uu.x, 1);
    const float r0 = sl.template res<MODE, 0>(m[4], uu.x, uu.y, wl, so.x, n.x, f.x);
    const float r1 = sl.template res<MODE, 1>(m[4], uu.y, er, uu.x, so.y, n.y, f.y);
    const float rs = __fadd_rn(r0, r1);
    if constexpr (PAR == 0) {
      rpair = rs;  // row t-4 even: the first row of a coarse row
    } else {
      const int ci = (y - 1) >> 1;
      if (sl.out && y - 1 >= sl.y0 && y - 1 < sl.y1 && ci < gc.H)
        s_st(fc, (size_t)ci * gc.W + (sl.x >> 1), __fmul_rn(__fadd_rn(rpair, rs), fout), SF);
    }
  }
};

// Prolongation of the coarse correction onto row t (e0: the lane's pair of it):
// the regular 3/4, 1/4 weights for cells in rows [2, H - 4] and columns
// [2, W - 4], the general bilinear weights (first vertical, then horizontal)
// elsewhere; decided per cell. c_lo, c_hi: the coarse rows around row t (t = 2I
// + 1: rows I, I + 1; t = 2I: rows I - 1, I), in the lane's coarse column.
template <int MODE, int PAR, bool L0>
__device__ __forceinline__ void prolong_row(const LevelGeom &g, const LevelGeom &gc, const StripLane<L0> &sl,
                                            const P1 &pxe, const P1 &pxo, const bool (&preg)[2],
                                            float c_lo, float c_hi, int t, float2 &e0) {
  const float av = PAR ? lerp_reg(c_lo, c_hi) : lerp_reg(c_hi, c_lo);
  const float al = __shfl_up_sync(0xffffffffu, av, 1);
  const float ar = __shfl_down_sync(0xffffffffu, av, 1);
  if constexpr (MODE == 0) {
    e0.x = __fadd_rn(e0.x, lerp_reg(av, al));
    e0.y = __fadd_rn(e0.y, lerp_reg(av, ar));
    return;
  }
  float bv;
  bool rreg, tin;
  if constexpr (MODE == 1) {  // regular rows: i1 is the farther coarse row, w1 = 1/4
    bv = PAR ? fmaf(0.25f, __fsub_rn(c_hi, c_lo), c_lo) : fmaf(0.25f, __fsub_rn(c_lo, c_hi), c_hi);
    rreg = tin = true;
  } else {
    tin = t >= 0 && t < g.H;
    rreg = t >= 2 && t <= g.H - 4;
    const P1 py = tin ? prolong1d(t, L0 ? 0 : g.shift, L0 ? g.H : g.H0, gc.H) : P1{0, 0, 0.f};
    const int lo_row = (t >> 1) - (PAR ? 0 : 1);
    const float c0 = py.i0 == lo_row ? c_lo : c_hi, c1 = py.i1 == lo_row ? c_lo : c_hi;
    bv = fmaf(py.w1, __fsub_rn(c1, c0), c0);
  }
  const float bl = __shfl_up_sync(0xffffffffu, bv, 1);
  const float br = __shfl_down_sync(0xffffffffu, bv, 1);
  if (tin && sl.in) {
    const float ae = pxe.i1 == pxe.i0 ? bv : bl;
    const float ao = pxo.i1 == pxo.i0 ? bv : br;
    e0.x = __fadd_rn(e0.x, (rreg && preg[0]) ? lerp_reg(av, al) : fmaf(pxe.w1, __fsub_rn(ae, bv), bv));
    e0.y = __fadd_rn(e0.y, (rreg && preg[1]) ? lerp_reg(av, ar) : fmaf(pxo.w1, __fsub_rn(ao, bv), bv));
  }
}

// Up pass on the finest level (nu2 = 1): row t gets the prolonged coarse
// correction, rows t-1 and t-2 the two half-sweeps (colours 0 and 1), and row
// t-3, then final, the update of the iterate: u += e / s_k in float-float,
// r_{k+1} = (f - L e) / s_k, and the sums of u_{k+1} and of r_{k+1}^2. E[j] and
// F[j] hold row t - j; c_lo and c_hi the coarse rows around row t (t = 2I + 1:
// rows I, I + 1; t = 2I: rows I - 1, I).
template <int SF>
struct UpStream {
  LevelGeom g, gc;
  static constexpr bool L0 = true;
  StripLane<true> sl;
  const float *src;
  const void *ue, *uc;
  float *uh, *ul, *rn;
  float off, scale, inv_s, omega;
  int k;
  P1 pxe, pxo;    // horizontal prolongation of the lane's two cells
  bool preg[2];   // the cell's column takes the regular weights
  float2 E[5], F[4], QF[kStreamPre], QE[kStreamPre], QH[kStreamPre], QL[kStreamPre];
  float QC[2], c_lo, c_hi;
  // The lane's FP32 sums of u_{k+1} and r_{k+1}^2 over its cells, in row order
  // (so their roundings depend on the segment height, as the tiled kernels'
  // depend on the tile shape; the iterate itself does not).
  float su, rn2;

  __device__ __forceinline__ float2 load_f(int row) const {
    return (sl.in && row >= 0 && row < g.H)
               ? __ldg(reinterpret_cast<const float2 *>(src + (size_t)row * g.W + sl.x))
               : make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ float2 load_e(int row) const {
    return (sl.in && row >= 0 && row < g.H) ? s_ld2<SF>(ue, (size_t)row * g.W + sl.x)
                                            : make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ float load_c(int ci) const {
    return (sl.in && ci >= 0 && ci < gc.H) ? s_ld(uc, (size_t)ci * gc.W + (sl.x >> 1), SF) : 0.f;
  }
  __device__ __forceinline__ bool stores(int row) const {
    return sl.out && row >= sl.y0 && row < sl.y1 && row < g.H;
  }
  // The iterate of an output row (zero before the first cycle). Each cell is
  // read and then written by the one lane that stores it.
  __device__ __forceinline__ void load_u(int row, float2 &h, float2 &l) const {
    const bool v = k > 0 && stores(row);
    const size_t p = v ? (size_t)row * g.W + sl.x : 0;
    h = v ? *reinterpret_cast<const float2 *>(uh + p) : make_float2(0.f, 0.f);
    l = v ? *reinterpret_cast<const float2 *>(ul + p) : make_float2(0.f, 0.f);
  }

  template <int MODE, int PAR>
  __device__ __forceinline__ void step(int t) {
#pragma unroll
    for (int j = 4; j > 0; --j) E[j] = E[j - 1];
#pragma unroll
    for (int j = 3; j > 0; --j) F[j] = F[j - 1];
    const float2 qf = QF[0];
    E[0] = QE[0];
#pragma unroll
    for (int j = 0; j + 1 < kStreamPre; ++j) {
      QF[j] = QF[j + 1];
      QE[j] = QE[j + 1];
    }
    QF[kStreamPre - 1] = load_f(t + kStreamPre);
    QE[kStreamPre - 1] = load_e(t + kStreamPre);
    const bool rin = MODE == 0 || (sl.in && t >= 0 && t < g.H);
    F[0] = rin ? make_float2(__fmul_rn(__fsub_rn(qf.x, off), scale), __fmul_rn(__fsub_rn(qf.y, off), scale))
               : make_float2(0.f, 0.f);
    if constexpr (PAR == 1) {
      c_lo = c_hi;
      c_hi = QC[0];
      QC[0] = QC[1];
      QC[1] = load_c(((t + 1) >> 1) + 2);
    }
    prolong_row<MODE, PAR, L0>(g, gc, sl, pxe, pxo, preg, c_lo, c_hi, t, E[0]);
    RowMask m[4];
    if constexpr (MODE == 2) {
#pragma unroll
      for (int s = 1; s < 4; ++s) m[s] = row_mask<L0>(g, t - s);
    }
    // half-sweeps: colour 0 on row t-1, colour 1 on row t-2 (cell 1 - PAR of each)
    constexpr int I = 1 - PAR;
#pragma unroll
    for (int s = 1; s <= 2; ++s) {
      float w, e;
      horiz<I>(E[s], w, e);
      cell<I>(E[s]) = sl.sweep<MODE, I>(m[s], cell<I>(E[s]), w, e, cell<I>(E[s + 1]),
                                        cell<I>(E[s - 1]), cell<I>(F[s]), omega);
    }
    // row t-3 is final
    const int y = t - 3;
    const float2 uu = E[3], n = E[4], so = E[2], f = F[3];
    const float wl = __shfl_up_sync(0xffffffffu, uu.y, 1);
    const float er = __shfl_down_sync(0xffffffffu, uu.x, 1);
    float r0 = sl.res<MODE, 0>(m[3], uu.x, uu.y, wl, so.x, n.x, f.x);
    float r1 = sl.res<MODE, 1>(m[3], uu.y, er, uu.x, so.y, n.y, f.y);
    float2 h = QH[0], l = QL[0];
#pragma unroll
    for (int j = 0; j + 1 < kStreamPre; ++j) {
      QH[j] = QH[j + 1];
      QL[j] = QL[j + 1];
    }
    load_u(y + kStreamPre, QH[kStreamPre - 1], QL[kStreamPre - 1]);
    // computed on every lane, stored (and summed) by the lanes that own row y:
    // no branch, so the steps of a loop body schedule as one block
    const bool st = stores(y);
    ds_add(h.x, l.x, __fmul_rn(uu.x, inv_s));
    ds_add(h.y, l.y, __fmul_rn(uu.y, inv_s));
    r0 = __fmul_rn(r0, inv_s);
    r1 = __fmul_rn(r1, inv_s);
    su += st ? __fadd_rn(__fadd_rn(h.x, l.x), __fadd_rn(h.y, l.y)) : 0.f;
    rn2 += st ? fmaf(r1, r1, __fmul_rn(r0, r0)) : 0.f;
    const size_t p = st ? (size_t)y * g.W + sl.x : 0;
    if (st) {
      *reinterpret_cast<float2 *>(uh + p) = h;
      *reinterpret_cast<float2 *>(ul + p) = l;
      *reinterpret_cast<float2 *>(rn + p) = make_float2(r0, r1);
    }
  }
};

// Up pass on a level l >= 1 (nu2 = 1): row t gets the prolonged coarse
// correction, rows t-1 and t-2 the two half-sweeps (colours 0 and 1); row t-2 is
// then final and stored (format SF) to the level's up-pass array. E[j] and F[j]
// hold row t - j; c_lo and c_hi as in UpStream.
template <int SF>
struct UpStreamC {
  LevelGeom g, gc;
  static constexpr bool L0 = false;
  StripLane<false> sl;
  const void *src, *ue, *uc;
  void *uo;
  float scale, omega;
  P1 pxe, pxo;
  bool preg[2];
  float2 E[4], F[3], QF[kStreamPre], QE[kStreamPre];
  float QC[2], c_lo, c_hi;

  __device__ __forceinline__ float2 load2(const void *p, int row) const {
    return (sl.in && row >= 0 && row < g.H) ? s_ld2<SF>(p, (size_t)row * g.W + sl.x)
                                            : make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ float load_c(int ci) const {
    return (sl.in && ci >= 0 && ci < gc.H) ? s_ld(uc, (size_t)ci * gc.W + (sl.x >> 1), SF) : 0.f;
  }

  template <int MODE, int PAR>
  __device__ __forceinline__ void step(int t) {
#pragma unroll
    for (int j = 3; j > 0; --j) E[j] = E[j - 1];
#pragma unroll
    for (int j = 2; j > 0; --j) F[j] = F[j - 1];
    const float2 qf = QF[0];
    E[0] = QE[0];
#pragma unroll
    for (int j = 0; j + 1 < kStreamPre; ++j) {
      QF[j] = QF[j + 1];
      QE[j] = QE[j + 1];
    }
    QF[kStreamPre - 1] = load2(src, t + kStreamPre);
    QE[kStreamPre - 1] = load2(ue, t + kStreamPre);
    F[0] = make_float2(__fmul_rn(qf.x, scale), __fmul_rn(qf.y, scale));
    if constexpr (PAR == 1) {
      c_lo = c_hi;
      c_hi = QC[0];
      QC[0] = QC[1];
      QC[1] = load_c(((t + 1) >> 1) + 2);
    }
    prolong_row<MODE, PAR, L0>(g, gc, sl, pxe, pxo, preg, c_lo, c_hi, t, E[0]);
    RowMask m[3];
    if constexpr (MODE == 2) {
#pragma unroll
      for (int s = 1; s < 3; ++s) m[s] = row_mask<L0>(g, t - s);
    }
    constexpr int I = 1 - PAR;
#pragma unroll
    for (int s = 1; s <= 2; ++s) {
      float w, e;
      horiz<I>(E[s], w, e);
      cell<I>(E[s]) = sl.sweep<MODE, I>(m[s], cell<I>(E[s]), w, e, cell<I>(E[s + 1]),
                                        cell<I>(E[s - 1]), cell<I>(F[s]), omega);
    }
    const int y = t - 2;
    if (sl.out && y >= sl.y0 && y < sl.y1 && y < g.H) s_st2<SF>(uo, (size_t)y * g.W + sl.x, E[2]);
  }
};

// Runs steps t in [tA, tE) (tE - tA even) of a stream whose first step has
// parity P0: steps in [lo, hi) (hi - lo a multiple of U, lo of parity P0), whose
// rows are all full, take mode MID (0 or 1), the others the general mode 2. U
// is the stream's prefetch depth: after U steps every ring slot holds the row
// loaded U steps earlier, so a loaded register is never copied before its use
// (a copy would wait for the load).
template <int P0, int MID, int U, class St>
__device__ __forceinline__ void run_stream(St &s, int tA, int lo, int hi, int tE) {
  constexpr int P1_ = 1 - P0;
  static_assert(U % 2 == 0, "steps come in pairs");
  int t = tA;
#pragma unroll 1
  for (; t < lo; t += 2) {
    s.template step<2, P0>(t);
    s.template step<2, P1_>(t + 1);
  }
#pragma unroll 1
  for (; t < hi; t += U) {
#pragma unroll
    for (int i = 0; i < U; i += 2) {
      s.template step<MID, P0>(t + i);
      s.template step<MID, P1_>(t + i + 1);
    }
  }
#pragma unroll 1
  for (; t < tE; t += 2) {
    s.template step<2, P0>(t);
    s.template step<2, P1_>(t + 1);
  }
}

// [lo, hi) for run_stream: the steps in [first, last), starting at a step
// congruent to rem modulo mod (a power of two; rem of the stream's parity) and
// trimmed to a multiple of U steps; empty (lo = hi = tE) if none.
__device__ __forceinline__ void full_range(int tA, int tE, int first, int last, int U, int rem,
                                           int mod, int &lo, int &hi) {
  lo = hi = tE;
  int l = max(tA, first);
  l += (rem - l) & (mod - 1);
  const int h = min(tE, last);
  if (h - l < U) return;
  lo = l;
  hi = l + (h - l) / U * U;
}

// Last row (exclusive) of the full rows: H - 1, or H - 2 when the last row is narrow.
template <bool L0>
__device__ __forceinline__ int full_row_end(const LevelGeom &g) { return (L0 || g.lasty == 1.f) ? g.H - 1 : g.H - 2; }
template <bool L0>
__device__ __forceinline__ int full_col_end(const LevelGeom &g) { return (L0 || g.lastx == 1.f) ? g.W - 1 : g.W - 2; }

template <int SF, bool L0>
__global__ void __launch_bounds__(kStreamThreads) mg_down_stream_kernel(LvArgs a, Ctrl *ctrl, int k_in,
                                                                       int first, StreamGrid sg) {
  griddep_enter();
  const int k = cycle_index(ctrl, k_in);
  if (L0 ? *(volatile int *)&ctrl->stopped != 0 : should_stop(ctrl, k, first)) return;
  DownStream<SF, L0> d;
  d.g = a.g;
  d.gc = a.gc;
  if (!strip_lane(a.g, sg, d.sl)) return;
  const int c = blockIdx.z;
  const Rhs rh = rhs_of(a, ctrl, k, c);
  d.src = rh.src;
  d.off = rh.off;
  d.scale = rh.scale;
  d.omega = a.omega;
  d.fout = a.fout;
  d.u = s_at(a.u, (size_t)c * a.g.plane, SF);
  d.fc = s_at(a.fc, (size_t)c * a.gc.plane, SF);
  d.rpair = 0.f;
  const int tA = d.sl.y0 - 4, tE = d.sl.y1 + 4;
#pragma unroll
  for (int j = 0; j < 6; ++j) d.E[j] = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < 5; ++j) d.F[j] = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < kStreamPreDown; ++j) d.Q[j] = d.load(tA + j);
  // full rows t - 4 .. t
  int lo, hi;
  full_range(tA, tE, 6, full_row_end<L0>(a.g), kStreamPreDown, 0, 2, lo, hi);
  if (d.sl.sx >= 1 && d.sl.sx + kStripW <= full_col_end<L0>(a.g)) run_stream<0, 0, kStreamPreDown>(d, tA, lo, hi, tE);
  else run_stream<0, 1, kStreamPreDown>(d, tA, lo, hi, tE);
}

template <int SF>
__global__ void __launch_bounds__(kStreamThreads) mg_upc_stream_kernel(LvArgs a, Ctrl *ctrl, int k_in,
                                                                      StreamGrid sg) {
  griddep_enter();
  const int k = cycle_index(ctrl, k_in);
  if (should_stop(ctrl, k, 0)) return;
  UpStreamC<SF> u;
  u.g = a.g;
  u.gc = a.gc;
  if (!strip_lane(a.g, sg, u.sl)) return;
  const int c = blockIdx.z;
  const Rhs rh = rhs_of(a, ctrl, k, c);
  u.src = rh.src;
  u.scale = rh.scale;
  u.omega = a.omega;
  u.ue = s_at(a.u, (size_t)c * a.g.plane, SF);
  u.uc = s_at(a.uc, (size_t)c * a.gc.plane, SF);
  u.uo = s_at(a.uo, (size_t)c * a.g.plane, SF);
  u.pxe = u.sl.in ? prolong1d(u.sl.x, a.g.shift, a.g.W0, a.gc.W) : P1{0, 0, 0.f};
  u.pxo = u.sl.in ? prolong1d(u.sl.x + 1, a.g.shift, a.g.W0, a.gc.W) : P1{0, 0, 0.f};
  u.preg[0] = u.sl.x >= 2 && u.sl.x <= a.g.W - 4;
  u.preg[1] = u.sl.x + 1 >= 2 && u.sl.x + 1 <= a.g.W - 4;
  const int tA = u.sl.y0 - 2, tE = u.sl.y1 + 2;  // even: the first step has parity 0
#pragma unroll
  for (int j = 0; j < 4; ++j) u.E[j] = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < 3; ++j) u.F[j] = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < kStreamPre; ++j) {
    u.QF[j] = u.load2(u.src, tA + j);
    u.QE[j] = u.load2(u.ue, tA + j);
  }
  // t = tA = 2I: coarse rows I - 1, I in use, I + 1 and I + 2 loaded ahead
  const int I0 = tA >> 1;
  u.c_lo = u.load_c(I0 - 1);
  u.c_hi = u.load_c(I0);
  u.QC[0] = u.load_c(I0 + 1);
  u.QC[1] = u.load_c(I0 + 2);
  // full rows: prolongation row t in [2, H - 4], sweep rows t - 2, t - 1 full
  int lo, hi;
  full_range(tA, tE, 4, a.g.H - 3, kStreamPre, 0, 2, lo, hi);
  if (u.sl.sx >= 2 && u.sl.sx + kStripW - 1 <= a.g.W - 4) run_stream<0, 0, kStreamPre>(u, tA, lo, hi, tE);
  else run_stream<0, 1, kStreamPre>(u, tA, lo, hi, tE);
}

template <int SF>
__global__ void __launch_bounds__(kStreamThreads) mg0_up_stream_kernel(LvArgs a, Ctrl *ctrl, int k_in,
                                                                      StreamGrid sg) {
  griddep_enter();
  const int k = cycle_index(ctrl, k_in);
  if (should_stop(ctrl, k, 0)) return;
  UpStream<SF> u;
  u.g = a.g;
  u.gc = a.gc;
  u.su = 0.f;
  u.rn2 = 0.f;
  const int c = blockIdx.z;
  if (strip_lane(a.g, sg, u.sl)) {
    const Rhs rh = rhs_of(a, ctrl, k, c);
    u.src = static_cast<const float *>(rh.src);
    u.off = rh.off;
    u.scale = rh.scale;
    u.inv_s = 1.f / rh.scale;  // exact: a power of two
    u.omega = a.omega;
    u.k = k;
    const size_t cb = (size_t)c * a.g.plane;
    u.ue = s_at(a.u, cb, SF);
    u.uc = s_at(a.uc, (size_t)c * a.gc.plane, SF);
    u.uh = a.uhi + cb;
    u.ul = a.ulo + cb;
    u.rn = a.rb[k & 1] + cb;
    u.pxe = u.sl.in ? prolong1d(u.sl.x, 0, a.g.W, a.gc.W) : P1{0, 0, 0.f};
    u.pxo = u.sl.in ? prolong1d(u.sl.x + 1, 0, a.g.W, a.gc.W) : P1{0, 0, 0.f};
    u.preg[0] = u.sl.x >= 2 && u.sl.x <= a.g.W - 4;
    u.preg[1] = u.sl.x + 1 >= 2 && u.sl.x + 1 <= a.g.W - 4;
    const int tA = u.sl.y0 - 3, tE = u.sl.y1 + 3;
#pragma unroll
    for (int j = 0; j < 5; ++j) u.E[j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 4; ++j) u.F[j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < kStreamPre; ++j) {
      u.QF[j] = u.load_f(tA + j);
      u.QE[j] = u.load_e(tA + j);
      u.load_u(tA - 3 + j, u.QH[j], u.QL[j]);
    }
    u.c_lo = 0.f;
    u.c_hi = u.load_c((tA - 1) >> 1);
    u.QC[0] = u.load_c((tA + 1) >> 1);
    u.QC[1] = u.load_c(((tA + 1) >> 1) + 1);
    // full rows: prolongation row t in [2, H - 4], sweep and residual rows
    // t - 3 .. t - 1 in [1, H - 2]
    int lo, hi;
    full_range(tA, tE, 5, a.g.H - 3, kStreamPre, 1, 2, lo, hi);
    if (u.sl.sx >= 2 && u.sl.sx + kStripW - 1 <= a.g.W - 4) run_stream<1, 0, kStreamPre>(u, tA, lo, hi, tE);
    else run_stream<1, 1, kStreamPre>(u, tA, lo, hi, tE);
  }
  double su = u.su, rn2 = u.rn2;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    su += __shfl_xor_sync(0xffffffffu, su, o);
    rn2 += __shfl_xor_sync(0xffffffffu, rn2, o);
  }
  __shared__ double s_part[2][kStreamThreads / 32];
  if ((threadIdx.x & 31) == 0) {
    s_part[0][threadIdx.x >> 5] = su;
    s_part[1][threadIdx.x >> 5] = rn2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
#pragma unroll
    for (int w = 0; w < kStreamThreads / 32; ++w) {
      a0 += s_part[0][w];
      a1 += s_part[1][w];
    }
    atomicAdd(&ctrl->sum_u[k + 1][c], a0);
    atomicAdd(&ctrl->rnorm2[k + 1], a1);
  }
}

// ------------------------------------------------------------------ tail: the small levels in one CTA
//
// Levels t..L (t the first level >= 1 with at most kTailCells cells per
// channel, L the coarsest) fit in one CTA's shared memory, so one CTA per
// channel runs their whole part of the V-cycle: pre-sweeps, residual and
// restriction from t down to L-1, the FP64 coarse solve on L, prolongation and
// post-sweeps back up to t. Phases are separated by __syncthreads only. The
// operator, transfers and sweep order are those of the tiled kernels (same
// coef, residual and prolong1d), on the natural row-major layout.

constexpr long long kTailCells = 4096;
constexpr int kTailThreads = 1024;

struct TailArgs {
  LevelGeom lv[kMaxLevels];  // lv[i] = level t + i; lv[n - 1] is the coarsest
  int off_u[kMaxLevels];     // shared-memory float offsets: u of level i (f follows)
  int off_t[kMaxLevels];     // and its row / column tables
  int off_minv;              // the staged coarse inverse (doubles), or -1: read from global
  int off_fd;                // -f of the coarsest level in FP64
  int n;                     // levels in the tail (>= 1)
  const void *f_top;         // right-hand side of level t times 4^-t [C][plane] (storage sf)
  void *u_top;               // correction of level t [C][plane] (output, storage sf)
  int sf;                    // GDGS_STORAGE_*
  float fin;                 // 4^t
  const double *Minv;        // [nc][nc] inverse of -L + 11^T / nc on the coarsest level
  int nu1, nu2;
  float omega;
};

__host__ __device__ __forceinline__ int tail_stride(const LevelGeom &g) {
  return (int)((g.plane + 3) & ~3ll);
}

// Shared-memory layout of the tail: u and f of every level, then per level the
// row tables (H entries each: wy, cS, cN, and the prolongation rows i0, i1, w
// from the next coarser level) and the column tables (W entries each: wx, cE,
// cW, i0, i1, w), then -f of the coarsest level and the partial sums of its
// product in FP64, then (for small coarsest grids) the FP64 inverse, stored
// transposed. A cell's face coefficients are products of one row and one
// column factor (e = wy cE, w = wy cW, s = wx cS, n = wx cN), so every sweep,
// residual and prolongation is branch-free. Offsets are computed on the host.
constexpr int kTailMinvStage = 64;  // stage the inverse when nc <= this

// Threads per row of the coarse solve's product (nc <= 1024 cells).
__host__ __device__ __forceinline__ int tail_parts(int nc) {
  const int p = kTailThreads / (nc > 0 ? nc : 1);
  return p < 1 ? 1 : (p > 8 ? 8 : p);
}

inline size_t tail_layout(const LevelGeom *lv, int n, TailArgs *a) {
  size_t o = 0;
  for (int i = 0; i < n; ++i) {
    if (a) a->off_u[i] = (int)o;
    o += 2 * (size_t)tail_stride(lv[i]);
  }
  for (int i = 0; i < n; ++i) {
    if (a) a->off_t[i] = (int)o;
    o += 6 * (size_t)(lv[i].H + lv[i].W);
  }
  const long long nc = lv[n - 1].plane;
  o = (o + 1) & ~(size_t)1;  // 8-byte alignment for the doubles
  if (a) a->off_fd = (int)o;
  o += 2 * (size_t)nc * (1 + tail_parts((int)nc));  // -f, then the partial sums
  if (nc <= kTailMinvStage) {
    if (a) a->off_minv = (int)o;
    o += 2 * (size_t)(nc * nc);
  } else if (a) {
    a->off_minv = -1;
  }
  return o;
}

struct TailLevel {
  int H, W;
  float *u, *f;
  const float *wy, *cS, *cN, *wx, *cE, *cW;
  const int *ri0, *ri1, *ci0, *ci1;
  const float *rw, *cw;
};

__device__ __forceinline__ TailLevel tail_level_at(float *S, const TailArgs &a, int i) {
  TailLevel t;
  t.H = a.lv[i].H;
  t.W = a.lv[i].W;
  t.u = S + a.off_u[i];
  t.f = t.u + tail_stride(a.lv[i]);
  float *R = S + a.off_t[i], *Cc = R + 6 * t.H;
  t.wy = R;
  t.cS = R + t.H;
  t.cN = R + 2 * t.H;
  t.ri0 = reinterpret_cast<const int *>(R + 3 * t.H);
  t.ri1 = reinterpret_cast<const int *>(R + 4 * t.H);
  t.rw = R + 5 * t.H;
  t.wx = Cc;
  t.cE = Cc + t.W;
  t.cW = Cc + 2 * t.W;
  t.ci0 = reinterpret_cast<const int *>(Cc + 3 * t.W);
  t.ci1 = reinterpret_cast<const int *>(Cc + 4 * t.W);
  t.cw = Cc + 5 * t.W;
  return t;
}

// Row and column tables of every tail level (the same factors as build_factors).
__device__ void tail_build_tables(float *S, const TailArgs &a) {
  for (int i = 0; i < a.n; ++i) {
    const LevelGeom &g = a.lv[i];
    const TailLevel t = tail_level_at(S, a, i);
    float *R = const_cast<float *>(t.wy), *Cc = const_cast<float *>(t.wx);
    const bool has_c = i + 1 < a.n;
    for (int k = threadIdx.x; k < t.H + t.W; k += kTailThreads) {
      const bool row = k < t.H;
      const int r = row ? k : k - t.H, n = row ? t.H : t.W;
      const float last = row ? g.ey : g.ex;
      float *T = row ? R : Cc;
      T[r] = row ? wyf(g, r) : wxf(g, r);
      T[n + r] = r + 1 < n ? (r + 1 == n - 1 ? last : 1.f) : 0.f;  // cS / cE
      T[2 * n + r] = r > 0 ? (r == n - 1 ? last : 1.f) : 0.f;      // cN / cW
      P1 p{r >> 1, r >> 1, 0.f};
      if (has_c) {
        const LevelGeom &gc = a.lv[i + 1];
        p = row ? prolong1d(r, g.shift, g.H0, gc.H) : prolong1d(r, g.shift, g.W0, gc.W);
      }
      reinterpret_cast<int *>(T)[3 * n + r] = p.i0;
      reinterpret_cast<int *>(T)[4 * n + r] = p.i1;
      T[5 * n + r] = p.w1;
    }
  }
}

// Gauss-Seidel value of cell (I, J) from its neighbours, with the row factors
// of row I (wy, cS, cN) and the column tables.
__device__ __forceinline__ float tail_gs(const TailLevel &t, const float *ur, const float *fr,
                                         int I, int J, float wy, float cS, float cN) {
  const int W = t.W;
  const float wx = t.wx[J];
  const float ae = wy * t.cE[J], aw = wy * t.cW[J], as = wx * cS, an = wx * cN;
  const float uE = J + 1 < W ? ur[J + 1] : 0.f;
  const float uW = J > 0 ? ur[J - 1] : 0.f;
  const float uS = I + 1 < t.H ? ur[J + W] : 0.f;
  const float uN = I > 0 ? ur[J - W] : 0.f;
  const float d = (ae + aw) + (as + an);
  return __fdividef((ae * uE + aw * uW) + (as * uS + an * uN) - fr[J], d);
}

// One red-black half-sweep over the cells with (I + J) & 1 == col; a warp per
// row, two cells of the row per lane and iteration (loads first). With
// from_zero (the first pre-sweep of a level) the other cells are set to 0
// instead of being read, so u needs no clearing pass.
__device__ __forceinline__ void tail_half_sweep(const TailLevel &t, int col, bool from_zero,
                                                float omega) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int H = t.H, W = t.W;
  for (int I = warp; I < H; I += kTailThreads / 32) {
    const float wy = t.wy[I], cS = t.cS[I], cN = t.cN[I];
    float *ur = t.u + I * W;
    const float *fr = t.f + I * W;
    if (from_zero) {
      for (int J = lane; J < W; J += 32) {
        float v = 0.f;
        if (((I + J) & 1) == col) {
          const float d = wy * (t.cE[J] + t.cW[J]) + t.wx[J] * (cS + cN);
          v = omega * __fdividef(-fr[J], d);
        }
        ur[J] = v;
      }
      continue;
    }
    for (int J0 = 2 * lane + ((I + col) & 1); J0 < W; J0 += 128) {
      const int J1 = J0 + 64;
      const bool two = J1 < W;
      const float g0 = tail_gs(t, ur, fr, I, J0, wy, cS, cN);
      const float g1 = two ? tail_gs(t, ur, fr, I, J1, wy, cS, cN) : 0.f;
      const float o0 = ur[J0], o1 = two ? ur[J1] : 0.f;
      ur[J0] = fmaf(omega, g0 - o0, o0);
      if (two) ur[J1] = fmaf(omega, g1 - o1, o1);
    }
  }
}

__device__ __forceinline__ float tail_residual(const TailLevel &t, int I, int J, float wy, float cS,
                                               float cN) {
  const int W = t.W, q = I * W + J;
  const float u = t.u[q], wx = t.wx[J];
  const float dE = J + 1 < W ? t.u[q + 1] - u : 0.f;
  const float dW = J > 0 ? t.u[q - 1] - u : 0.f;
  const float dS = I + 1 < t.H ? t.u[q + W] - u : 0.f;
  const float dN = I > 0 ? t.u[q - W] - u : 0.f;
  return t.f[q] - ((wy * t.cE[J] * dE + wy * t.cW[J] * dW) + (wx * cS * dS + wx * cN * dN));
}

// Stage the coarse inverse into shared memory (transposed) when it is small.
__device__ void tail_stage_inverse(float *S, const TailArgs &a) {
  const int tid = threadIdx.x;
  if (a.off_minv < 0) return;
  const int nc = (int)a.lv[a.n - 1].plane, n2 = nc * nc;
  double *M = reinterpret_cast<double *>(S + a.off_minv);
  for (int q0 = tid; q0 < n2; q0 += 4 * kTailThreads) {
    double v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int q = q0 + j * kTailThreads;
      v[j] = q < n2 ? __ldg(a.Minv + q) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int q = q0 + j * kTailThreads;
      if (q < n2) {
        const int row = q / nc;
        M[(q - row * nc) * nc + row] = v[j];
      }
    }
  }
}

// The tail's part of one V-cycle, in one CTA: from the right-hand side of its
// first level (already in shared memory, tables built) to the corrected u of
// that level. Phases are separated by __syncthreads.
__device__ void tail_vcycle(float *S, const TailArgs &a) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int kWarps = kTailThreads / 32;
  for (int i = 0; i + 1 < a.n; ++i) {  // down: sweeps from 0, restrict the residual
    const TailLevel t = tail_level_at(S, a, i), tc = tail_level_at(S, a, i + 1);
    for (int s = 0; s < 2 * a.nu1; ++s) {
      tail_half_sweep(t, s & 1, s == 0, a.omega);
      __syncthreads();
    }
    for (int CI = warp; CI < tc.H; CI += kWarps) {
      const int I = 2 * CI;
      const bool two = I + 1 < t.H;
      const float wy0 = t.wy[I], cS0 = t.cS[I], cN0 = t.cN[I];
      const float wy1 = two ? t.wy[I + 1] : 0.f, cS1 = two ? t.cS[I + 1] : 0.f,
                  cN1 = two ? t.cN[I + 1] : 0.f;
      for (int CJ = lane; CJ < tc.W; CJ += 32) {
        const int J = 2 * CJ;
        float sum = tail_residual(t, I, J, wy0, cS0, cN0);
        if (J + 1 < t.W) sum += tail_residual(t, I, J + 1, wy0, cS0, cN0);
        if (two) {
          sum += tail_residual(t, I + 1, J, wy1, cS1, cN1);
          if (J + 1 < t.W) sum += tail_residual(t, I + 1, J + 1, wy1, cS1, cN1);
        }
        tc.f[CI * tc.W + CJ] = sum;
      }
    }
    __syncthreads();
  }
  {  // coarsest: u = Minv (-f) in FP64. FP64 issues slowly, so the products are
     // spread over P threads per row, each a run of columns (read from the
     // transposed staged inverse: consecutive rows are consecutive words), and
     // one thread per row adds the P partial sums in order.
    const TailLevel t = tail_level_at(S, a, a.n - 1);
    const int nc = t.H * t.W, P = tail_parts(nc), len = (nc + P - 1) / P;
    const bool staged = a.off_minv >= 0;
    const double *M = staged ? reinterpret_cast<const double *>(S + a.off_minv) : a.Minv;
    const size_t rs = staged ? 1 : (size_t)nc, cs = staged ? (size_t)nc : 1;  // (row, j) at row rs + j cs
    double *fd = reinterpret_cast<double *>(S + a.off_fd), *part = fd + nc;
    for (int j = tid; j < nc; j += kTailThreads) fd[j] = -(double)t.f[j];
    __syncthreads();
    for (int w = tid; w < P * nc; w += kTailThreads) {
      const int p = w / nc, row = w - p * nc;
      const int j1 = min(nc, (p + 1) * len);
      const double *mr = M + (size_t)row * rs;
      double s0 = 0.0, s1 = 0.0;
      int j = p * len;
      for (; j + 1 < j1; j += 2) {
        s0 = fma(mr[j * cs], fd[j], s0);
        s1 = fma(mr[(j + 1) * cs], fd[j + 1], s1);
      }
      if (j < j1) s0 = fma(mr[j * cs], fd[j], s0);
      part[w] = s0 + s1;
    }
    __syncthreads();
    for (int row = tid; row < nc; row += kTailThreads) {
      double s = 0.0;
      for (int p = 0; p < P; ++p) s += part[p * nc + row];
      t.u[row] = (float)s;
    }
    __syncthreads();
  }
  for (int i = a.n - 2; i >= 0; --i) {  // up: prolongate the correction, post-sweeps
    const TailLevel t = tail_level_at(S, a, i), tc = tail_level_at(S, a, i + 1);
    for (int I = warp; I < t.H; I += kWarps) {
      const float *ra = tc.u + t.ri0[I] * tc.W, *rb = tc.u + t.ri1[I] * tc.W;
      const float wr = t.rw[I];
      float *ur = t.u + I * t.W;
      for (int J0 = lane; J0 < t.W; J0 += 128) {  // four columns per lane: loads first
        float add[4], cur[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int J = J0 + 32 * k;
          add[k] = cur[k] = 0.f;
          if (J < t.W) {
            const int j0 = t.ci0[J], j1 = t.ci1[J];
            const float wc = t.cw[J];
            const float a0 = ra[j0] + wc * (ra[j1] - ra[j0]);
            const float a1 = rb[j0] + wc * (rb[j1] - rb[j0]);
            add[k] = a0 + wr * (a1 - a0);
            cur[k] = ur[J];
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (J0 + 32 * k < t.W) ur[J0 + 32 * k] = cur[k] + add[k];
      }
    }
    __syncthreads();
    for (int s = 0; s < 2 * a.nu2; ++s) {
      tail_half_sweep(t, s & 1, false, a.omega);
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kTailThreads)
mg_tail_kernel(TailArgs a, Ctrl *ctrl, int k_in, int first) {
  griddep_enter();
  extern __shared__ float4 sm4[];
  float *S = reinterpret_cast<float *>(sm4);
  const int k = cycle_index(ctrl, k_in);
  if (block_should_stop(ctrl, k, first)) return;
  const int c = blockIdx.x;
  const int tid = threadIdx.x;
  {  // right-hand side of the top level and the coarse inverse: loads first
    const TailLevel t = tail_level_at(S, a, 0);
    const void *src = s_at(a.f_top, (size_t)c * a.lv[0].plane, a.sf);
    const int np = (int)a.lv[0].plane;
    for (int q0 = tid; q0 < np; q0 += 4 * kTailThreads) {
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int q = q0 + j * kTailThreads;
        v[j] = q < np ? s_ld(src, q, a.sf) * a.fin : 0.f;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int q = q0 + j * kTailThreads;
        if (q < np) t.f[q] = v[j];
      }
    }
    tail_stage_inverse(S, a);
    tail_build_tables(S, a);
    __syncthreads();
  }
  tail_vcycle(S, a);
  {
    const TailLevel t = tail_level_at(S, a, 0);
    void *dst = s_at(a.u_top, (size_t)c * a.lv[0].plane, a.sf);
    for (int q = tid; q < a.lv[0].plane; q += kTailThreads) s_st(dst, q, t.u[q], a.sf);
  }
}

// ------------------------------------------------------------------ setup, divergence, finalize

// Order-independent 64-bit digest of the factor (sum of mixed words), so a
// cached factor is only trusted if its contents are intact.
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

__device__ unsigned long long digest(const double *A, int n2) {
  __shared__ unsigned long long acc;
  if (threadIdx.x == 0) acc = 0;
  __syncthreads();
  unsigned long long h = 0;
  for (int i = threadIdx.x; i < n2; i += blockDim.x)
    h += mix64((unsigned long long)__double_as_longlong(A[i]) ^ (0x9e3779b97f4a7c15ull * (i + 1)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&acc, h);  // one shared atomic per warp
  __syncthreads();
  return acc;
}

// Builds and inverts M = -L + 11^T / n of the coarsest grid in FP64 (SPD, so
// Gauss-Jordan without pivoting is stable), unless the cached one in the
// workspace matches both the grid (tag) and its own digest.
// The power of two s with s * rms(r) in [0.5, 1): cycle k works on s_k r_k.
__device__ __forceinline__ float residual_scale(double rnorm2, long long cells) {
  const double rms = sqrt(rnorm2 / (double)(cells > 0 ? cells : 1));
  if (!(rms > 0.0) || !(rms < 1e300)) return 1.f;
  int e = 0;
  frexp(rms, &e);
  e = max(-120, min(120, e));
  return ldexpf(1.f, -e);
}

__global__ void __launch_bounds__(1024)
coarse_setup_kernel(LevelGeom g, double *A, CoarseTag *tag, CoarseTag want, Ctrl *ctrl, int C,
                    long long npx, Ctrl *sub) {
  griddep_enter();
  __shared__ int match;
  __shared__ double fcol[260];
  const int n = g.H * g.W;
  if (threadIdx.x == 0) {  // ||rho - mean(rho)||^2 and the means, from the divergence sums
    double r2 = 0.0;
    for (int c = 0; c < C; ++c) {
      const double m = ctrl->rho_sum[c] / (double)npx;
      ctrl->rho_mean[c] = (float)m;
      r2 += fmax(ctrl->rho_sq[c] - ctrl->rho_sum[c] * m, 0.0);
    }
    ctrl->rnorm2[0] = r2;
    ctrl->escale[0] = residual_scale(r2, (long long)C * npx);
    ctrl->split = sub ? 1 : 0;
  }
  if (sub) {  // the per-channel control blocks of a channel-split solve
    int *w = reinterpret_cast<int *>(sub);
    const int nw = (int)(sizeof(Ctrl) / sizeof(int)) * C;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) w[i] = 0;
    __syncthreads();
    if (threadIdx.x < C) {
      const int c = threadIdx.x;
      Ctrl *sc = sub + c;
      const double m = ctrl->rho_sum[c] / (double)npx;
      const double r2 = fmax(ctrl->rho_sq[c] - ctrl->rho_sum[c] * m, 0.0);
      sc->rtol = ctrl->rtol;
      sc->max_cycles = ctrl->max_cycles;
      sc->channels = 1;
      sc->rho_mean[0] = (float)m;
      sc->rho_sum[0] = ctrl->rho_sum[c];
      sc->rho_sq[0] = ctrl->rho_sq[c];
      sc->rnorm2[0] = r2;
      sc->escale[0] = residual_scale(r2, npx);
    }
  }
  if (threadIdx.x == 0) {
    const CoarseTag t = *tag;
    match = t.magic == want.magic && t.H0 == want.H0 && t.W0 == want.W0 &&
            t.levels == want.levels && t.Hc == want.Hc && t.Wc == want.Wc && t.nc == want.nc &&
            t.version == want.version;
  }
  __syncthreads();
  if (match) {
    const unsigned long long d = digest(A, n * n);
    if (d == tag->hash) return;  // uniform: every thread reads the same values
  }
  const double inv_n = 1.0 / n;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    const int I = i / g.W, J = i - I * g.W;
    const Coef cf = coef(g, I, J);
    double v = inv_n;
    if (j == i) v += (double)cf.e + cf.w + cf.s + cf.n;
    else if (j == i + 1 && J + 1 < g.W) v -= cf.e;
    else if (j == i - 1 && J > 0) v -= cf.w;
    else if (j == i + g.W && I + 1 < g.H) v -= cf.s;
    else if (j == i - g.W && I > 0) v -= cf.n;
    A[idx] = v;
  }
  __syncthreads();
  for (int p = 0; p < n; ++p) {
    const double piv = A[(size_t)p * n + p];
    for (int i = threadIdx.x; i < n; i += blockDim.x) fcol[i] = A[(size_t)i * n + p];
    __syncthreads();
    const double ip = 1.0 / piv;
    for (int j = threadIdx.x; j < n; j += blockDim.x)
      A[(size_t)p * n + j] = (j == p ? 1.0 : A[(size_t)p * n + j]) * ip;
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int i = idx / n, j = idx - i * n;
      if (i == p) continue;
      const double cur = (j == p) ? 0.0 : A[idx];
      A[idx] = cur - fcol[i] * A[(size_t)p * n + j];
    }
    __syncthreads();
  }
  const unsigned long long d = digest(A, n * n);
  if (threadIdx.x == 0) {
    CoarseTag t = want;
    t.magic = 0;
    t.hash = d;
    *tag = t;
    __threadfence();
    tag->magic = want.magic;
  }
}

struct DivArgs {
  const float *maps;
  const uint8_t *mask;
  int input_is_rho;
  float threshold;
  int C, H, W, tiles_x;
  float *rho;
  float rtol;
  int max_cycles;
};

__device__ __forceinline__ bool tile_on(const uint8_t *mask, int tiles_x, int i, int j) {
  return !mask || mask[(i / kTile) * tiles_x + (j / kTile)];
}

// rho(i,j) = [j<W-1] gx(i,j) - [j>=1] gx(i,j-1) + [i<H-1] gy(i,j) - [i>=1] gy(i-1,j),
// with gradients of tiles whose mask is 0 read as zero (or rho read directly for
// Laplacian fields); then the hard threshold T of Eq. thresh when t > 0; ||rho||^2.
__global__ void __launch_bounds__(256) divergence_kernel(DivArgs a, Ctrl *ctrl) {
  griddep_enter();
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    ctrl->rtol = a.rtol;
    ctrl->max_cycles = a.max_cycles;
    ctrl->channels = a.C;
  }
  const int c = blockIdx.y;
  const size_t plane = (size_t)a.H * a.W;
  const float *gxp = a.maps + (size_t)(a.input_is_rho ? c : 2 * c) * plane;
  const float *gyp = gxp + plane;
  bool bad = false;
  float n2 = 0.f, s1 = 0.f;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < plane;
       p += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(p / a.W), j = (int)(p - (size_t)i * a.W);
    float r = 0.f;
    if (a.input_is_rho) {
      if (tile_on(a.mask, a.tiles_x, i, j)) r = gxp[p];
    } else {
      if (j + 1 < a.W && tile_on(a.mask, a.tiles_x, i, j)) r += gxp[p];
      if (j >= 1 && tile_on(a.mask, a.tiles_x, i, j - 1)) r -= gxp[p - 1];
      if (i + 1 < a.H && tile_on(a.mask, a.tiles_x, i, j)) r += gyp[p];
      if (i >= 1 && tile_on(a.mask, a.tiles_x, i - 1, j)) r -= gyp[p - a.W];
    }
    bad |= !isfinite(r);
    if (a.threshold > 0.f && !(fabsf(r) >= a.threshold)) r = 0.f;
    a.rho[(size_t)c * plane + p] = r;
    n2 = fmaf(r, r, n2);
    s1 += r;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) set_status(ctrl, GDGS_ERR_NONFINITE);
  n2 = block_sum(n2);
  s1 = block_sum(s1);
  if (threadIdx.x == 0) {
    atomicAdd(&ctrl->rho_sq[c], (double)n2);
    atomicAdd(&ctrl->rho_sum[c], (double)s1);
  }
}

// The same divergence on four pixels of one row per thread (W % 4 == 0 and
// 16-byte aligned planes): 16-byte loads and stores, one 32-bit division per
// four pixels. A quad lies in one 16-pixel tile; only its left neighbour and
// the row above can sit in other tiles. Each pixel's terms are added in the
// order of the scalar kernel, so rho is bit-identical to it.
__device__ __forceinline__ float4 ld_f4(const float *p) {
  return __ldg(reinterpret_cast<const float4 *>(p));
}

__global__ void __launch_bounds__(256) divergence4_kernel(DivArgs a, Ctrl *ctrl) {
  griddep_enter();
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    ctrl->rtol = a.rtol;
    ctrl->max_cycles = a.max_cycles;
    ctrl->channels = a.C;
  }
  const int c = blockIdx.y, W = a.W, H = a.H, Wq = W >> 2, nq = H * Wq;
  const size_t plane = (size_t)H * W;
  const float *gxp = a.maps + (size_t)(a.input_is_rho ? c : 2 * c) * plane;
  const float *gyp = gxp + plane;
  float *rp = a.rho + (size_t)c * plane;
  bool bad = false;
  float n2 = 0.f, s1 = 0.f;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    const int i = q / Wq, j0 = (q - i * Wq) << 2;
    const size_t p = (size_t)i * W + j0;
    const bool on = tile_on(a.mask, a.tiles_x, i, j0);
    float r[4];
    if (a.input_is_rho) {
      const float4 v = on ? ld_f4(gxp + p) : make_float4(0.f, 0.f, 0.f, 0.f);
      r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
    } else {
      const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 gx = on ? ld_f4(gxp + p) : z;
      const float4 gy = on && i + 1 < H ? ld_f4(gyp + p) : z;
      const float4 gu = i >= 1 && tile_on(a.mask, a.tiles_x, i - 1, j0) ? ld_f4(gyp + p - W) : z;
      const float gl = j0 >= 1 && tile_on(a.mask, a.tiles_x, i, j0 - 1) ? gxp[p - 1] : 0.f;
      const float x[4] = {gx.x, gx.y, gx.z, gx.w}, y[4] = {gy.x, gy.y, gy.z, gy.w};
      const float u[4] = {gu.x, gu.y, gu.z, gu.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float v = 0.f;
        v += j0 + k + 1 < W ? x[k] : 0.f;
        v -= k > 0 ? x[k - 1] : gl;
        v += y[k];
        v -= u[k];
        r[k] = v;
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      bad |= !isfinite(r[k]);
      if (a.threshold > 0.f && !(fabsf(r[k]) >= a.threshold)) r[k] = 0.f;
      n2 = fmaf(r[k], r[k], n2);
      s1 += r[k];
    }
    *reinterpret_cast<float4 *>(rp + p) = make_float4(r[0], r[1], r[2], r[3]);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) set_status(ctrl, GDGS_ERR_NONFINITE);
  n2 = block_sum(n2);
  s1 = block_sum(s1);
  if (threadIdx.x == 0) {
    atomicAdd(&ctrl->rho_sq[c], (double)n2);
    atomicAdd(&ctrl->rho_sum[c], (double)s1);
  }
}

struct FinArgs {
  LevelGeom g0;
  const float *rho, *uhi, *ulo;
  float *image;
  float mean[GDGS_MAX_CHANNELS];
};

// m_c - mean(u_c), evaluated by one thread of the block (FP64 issues slowly on
// this GPU, so per-thread FP64 divides would dominate the kernel).
__device__ __forceinline__ float block_shift(float m, double sum_u, size_t plane) {
  __shared__ float s_shift;
  if (threadIdx.x == 0) s_shift = (float)((double)m - sum_u / (double)plane);
  __syncthreads();
  return s_shift;
}

// The supplied mean of channel c (a select over the parameter array, so the
// array is not copied to local memory for a dynamic index).
__device__ __forceinline__ float channel_mean(const float (&mean)[GDGS_MAX_CHANNELS], int c) {
  float m = mean[0];
#pragma unroll
  for (int i = 1; i < GDGS_MAX_CHANNELS; ++i)
    if (i == c) m = mean[i];
  return m;
}

// image = u + (m_c - mean(u_c)) for the iterate the cycle loop stopped at, and
// the residual rho - L u of that iterate in float-float arithmetic.
__global__ void __launch_bounds__(256) finalize_kernel(FinArgs a, Ctrl *ctrl) {
  griddep_enter();
  const int stopped = ctrl->stopped;
  const int c = blockIdx.y;
  const int kf = ctrl->split ? ctrl->kf_c[c] : (stopped ? ctrl->cycles : ctrl->max_cycles);
  const LevelGeom &g = a.g0;
  const size_t plane = (size_t)g.H * g.W;
  const float mc = channel_mean(a.mean, c);
  const float shift = block_shift(mc, ctrl->sum_u[kf][c], plane);
  const size_t cb = (size_t)c * plane;
  const float *uh = a.uhi + cb, *ul = a.ulo + cb;
  float r2 = 0.f;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < plane;
       p += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(p / g.W), j = (int)(p - (size_t)i * g.W);
    float r = a.rho[cb + p] - ctrl->rho_mean[c];
    float hi = 0.f, lo = 0.f;
    if (kf > 0) {
      hi = uh[p];
      lo = ul[p];
      float sh = 0.f, sl = 0.f;
      if (j + 1 < g.W) { sh += uh[p + 1] - hi; sl += ul[p + 1] - lo; }
      if (j > 0) { sh += uh[p - 1] - hi; sl += ul[p - 1] - lo; }
      if (i + 1 < g.H) { sh += uh[p + g.W] - hi; sl += ul[p + g.W] - lo; }
      if (i > 0) { sh += uh[p - g.W] - hi; sl += ul[p - g.W] - lo; }
      r -= sh + sl;
    }
    a.image[cb + p] = hi + (lo + shift);
    r2 = fmaf(r, r, r2);
  }
  r2 = block_sum(r2);
  if (threadIdx.x == 0) atomicAdd(&ctrl->final_rnorm2, (double)r2);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctrl->mean_set[c] = mc;
    if (c == 0 && !stopped && !ctrl->split) ctrl->cycles = kf;
  }
}

// L u of one pixel in float-float parts (sh + sl), neighbours east, west,
// south, north in that order, as in finalize_kernel.
__device__ __forceinline__ float fin_px(float h, float l, float eh, float el, float wh, float wl,
                                        float sh_, float sl_, float nh, float nl, bool E, bool Wst,
                                        bool S_, bool N_) {
  float sh = 0.f, sl = 0.f;
  if (E) { sh += eh - h; sl += el - l; }
  if (Wst) { sh += wh - h; sl += wl - l; }
  if (S_) { sh += sh_ - h; sl += sl_ - l; }
  if (N_) { sh += nh - h; sl += nl - l; }
  return sh + sl;
}

// The same finalisation on four pixels of one row per thread (W % 4 == 0,
// 16-byte aligned planes); per pixel the same operations in the same order as
// the scalar kernel.
__global__ void __launch_bounds__(256) finalize4_kernel(FinArgs a, Ctrl *ctrl) {
  griddep_enter();
  const int stopped = ctrl->stopped;
  const int c = blockIdx.y;
  const int kf = ctrl->split ? ctrl->kf_c[c] : (stopped ? ctrl->cycles : ctrl->max_cycles);
  const LevelGeom &g = a.g0;
  const int W = g.W, H = g.H, Wq = W >> 2, nq = H * Wq;
  const size_t plane = (size_t)H * W;
  const float mc = channel_mean(a.mean, c);
  const float shift = block_shift(mc, ctrl->sum_u[kf][c], plane);
  const float rm = ctrl->rho_mean[c];
  const size_t cb = (size_t)c * plane;
  const float *uh = a.uhi + cb, *ul = a.ulo + cb;
  float r2 = 0.f;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    const int i = q / Wq, j0 = (q - i * Wq) << 2;
    const size_t p = (size_t)i * W + j0;
    const float4 rv = ld_f4(a.rho + cb + p);
    float r[4] = {rv.x - rm, rv.y - rm, rv.z - rm, rv.w - rm};
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    if (kf > 0) {
      const float4 h4 = ld_f4(uh + p), l4 = ld_f4(ul + p);
      const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 hs = i + 1 < H ? ld_f4(uh + p + W) : z, ls = i + 1 < H ? ld_f4(ul + p + W) : z;
      const float4 hn = i > 0 ? ld_f4(uh + p - W) : z, ln = i > 0 ? ld_f4(ul + p - W) : z;
      const float hw = j0 > 0 ? uh[p - 1] : 0.f, lw = j0 > 0 ? ul[p - 1] : 0.f;
      const float he = j0 + 4 < W ? uh[p + 4] : 0.f, le = j0 + 4 < W ? ul[p + 4] : 0.f;
      const bool s_ = i + 1 < H, n_ = i > 0, w_ = j0 > 0, e_ = j0 + 4 < W;
      r[0] -= fin_px(h4.x, l4.x, h4.y, l4.y, hw, lw, hs.x, ls.x, hn.x, ln.x, true, w_, s_, n_);
      r[1] -= fin_px(h4.y, l4.y, h4.z, l4.z, h4.x, l4.x, hs.y, ls.y, hn.y, ln.y, true, true, s_, n_);
      r[2] -= fin_px(h4.z, l4.z, h4.w, l4.w, h4.y, l4.y, hs.z, ls.z, hn.z, ln.z, true, true, s_, n_);
      r[3] -= fin_px(h4.w, l4.w, he, le, h4.z, l4.z, hs.w, ls.w, hn.w, ln.w, e_, true, s_, n_);
      hi[0] = h4.x; hi[1] = h4.y; hi[2] = h4.z; hi[3] = h4.w;
      lo[0] = l4.x; lo[1] = l4.y; lo[2] = l4.z; lo[3] = l4.w;
    }
    *reinterpret_cast<float4 *>(a.image + cb + p) =
        make_float4(hi[0] + (lo[0] + shift), hi[1] + (lo[1] + shift), hi[2] + (lo[2] + shift),
                    hi[3] + (lo[3] + shift));
#pragma unroll
    for (int k = 0; k < 4; ++k) r2 = fmaf(r[k], r[k], r2);
  }
  r2 = block_sum(r2);
  if (threadIdx.x == 0) atomicAdd(&ctrl->final_rnorm2, (double)r2);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctrl->mean_set[c] = mc;
    if (c == 0 && !stopped && !ctrl->split) ctrl->cycles = kf;
  }
}

// Kernels executed inside graph-launched cycle loops (read by the diagnostics).
__device__ unsigned long long g_graph_kernels = 0;

// End of cycle k: stop once ||r_{k+1}|| <= rtol ||rho||, advance the cycle
// index, and (inside a graph) set the loop condition.
__global__ void advance_kernel(Ctrl *ctrl, int k_in, cudaGraphConditionalHandle h, int in_graph,
                               unsigned kernels_per_cycle, long long cells) {
  griddep_enter();
  const int k = k_in >= 0 ? k_in : ctrl->iter;
  if (k + 1 <= kMaxCycles) ctrl->escale[k + 1] = residual_scale(ctrl->rnorm2[k + 1], cells);
  if (!ctrl->stopped) {
    const double thr = ctrl->rtol * ctrl->rtol * ctrl->rnorm2[0];
    const double rk = ctrl->rnorm2[k + 1];
    if (!(rk == rk) || !(ctrl->rnorm2[0] == ctrl->rnorm2[0])) {  // NaN: stop and report
      set_status(ctrl, GDGS_ERR_NONFINITE);
      ctrl->stopped = 1;
      ctrl->cycles = k + 1;
    } else if (rk <= thr) {
      ctrl->stopped = 1;
      ctrl->cycles = k + 1;
    }
  }
  ctrl->iter = k + 1;
  if (in_graph) {
    atomicAdd(&g_graph_kernels, (unsigned long long)kernels_per_cycle);
    cudaGraphSetConditional(h, (!ctrl->stopped && k + 1 < ctrl->max_cycles) ? 1u : 0u);
  }
}

// After channel-split cycle loops: the all-channel state the finalize kernel and
// gdgs_sync_status read. A channel's iterate is the one its own loop stopped at
// (or its last, if it did not converge).
__global__ void merge_channels_kernel(Ctrl *ctrl, const Ctrl *sub, int C) {
  griddep_enter();
  if (threadIdx.x != 0) return;
  int all = 1, kmax = 0;
  for (int c = 0; c < C; ++c) {
    const Ctrl &s = sub[c];
    const int kc = s.stopped ? s.cycles : s.max_cycles;
    ctrl->kf_c[c] = kc;
    ctrl->sum_u[kc][c] = s.sum_u[kc][0];
    all &= s.stopped;
    kmax = max(kmax, kc);
    if (s.status != GDGS_OK) set_status(ctrl, s.status);
  }
  ctrl->stopped = all;
  ctrl->cycles = kmax;
}

// ------------------------------------------------------------------ host side

// Opt a kernel in to large dynamic shared memory, once per kernel and device,
// at the device's per-block maximum (launches then request what they need).
template <auto Kern>
cudaError_t set_smem(size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, Kern);
  if (e != cudaSuccess) return e;
  const int mx = optin - (int)fa.sharedSizeBytes;
  if (mx < (int)bytes) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// Launch names per level (the diagnostics keep the pointer).
const char *const kDownName[kMaxLevels] = {"mg0_down", "mg1_down", "mg2_down", "mg3_down", "mg4_down", "mg5_down", "mg6_down", "mg7_down", "mg8_down", "mg9_down", "mg10_down", "mg11_down", "mg12_down", "mg13_down", "mg14_down", "mg15_down", "mg16_down", "mg17_down", "mg18_down", "mg19_down", "mg20_down", "mg21_down", "mg22_down", "mg23_down"};
const char *const kUpName[kMaxLevels] = {"mg0_up", "mg1_up", "mg2_up", "mg3_up", "mg4_up", "mg5_up", "mg6_up", "mg7_up", "mg8_up", "mg9_up", "mg10_up", "mg11_up", "mg12_up", "mg13_up", "mg14_up", "mg15_up", "mg16_up", "mg17_up", "mg18_up", "mg19_up", "mg20_up", "mg21_up", "mg22_up", "mg23_up"};

template <int NU, int TY_, int TX_>
cudaError_t launch_mg_down_t(const LvArgs &a, Ctrl *ctrl, int k, int first, int C, cudaStream_t st) {
  using G = Geo<NU, TY_, TX_>;
  const size_t sm = DownShape<G>::smem;
  cudaError_t e = set_smem<mg_down_kernel<NU, TY_, TX_>>(sm);
  if (e != cudaSuccess) return e;
  const dim3 grid((a.g.W + TX_ - 1) / TX_, (a.g.H + TY_ - 1) / TY_, C);
  {
    LaunchScope ls_(kDownName[a.g.shift], st);
    launch_k(mg_down_kernel<NU, TY_, TX_>, grid, dim3(kBX, kBY), sm, st, a, ctrl, k, first);
  }
  return cudaGetLastError();
}

template <int NU, int TY_, int TX_>
cudaError_t launch_mg_up_t(const LvArgs &a, Ctrl *ctrl, int k, int C, cudaStream_t st) {
  using G = Geo<NU, TY_, TX_>;
  const size_t sm = UpShape<G>::smem;
  cudaError_t e = set_smem<mg_up_kernel<NU, TY_, TX_>>(sm);
  if (e != cudaSuccess) return e;
  const dim3 grid((a.g.W + TX_ - 1) / TX_, (a.g.H + TY_ - 1) / TY_, C);
  {
    LaunchScope ls_(kUpName[a.g.shift], st);
    launch_k(mg_up_kernel<NU, TY_, TX_>, grid, dim3(kBX, kBY), sm, st, a, ctrl, k);
  }
  return cudaGetLastError();
}

inline bool small_level(const LevelGeom &g) { return g.plane < kSmallLevel; }

// Streaming passes (even widths, V(2, 1)); GDGS_STREAM=0 keeps the tiles on every level.
bool stream_enabled() {
  static const bool on = [] {
    const char *v = getenv("GDGS_STREAM");
    return !(v && v[0] == '0');
  }();
  return on;
}

// Output rows per segment forced by GDGS_STREAM_ROWS (rounded up to a multiple of 8), or 0.
int stream_rows_env() {
  static const int rows = [] {
    const char *v = getenv("GDGS_STREAM_ROWS");
    const int r = v ? atoi(v) : 0;
    return r >= 1 ? (r + 7) & ~7 : 0;
  }();
  return rows;
}

// Levels 0 .. n-1 stream their down passes (GDGS_STREAM_DOWN_LEVELS, else 1) and
// their up passes (GDGS_STREAM_UP_LEVELS, else 3), each if its width is even.
int stream_levels(bool down) {
  static const int nd = [] {
    const char *v = getenv("GDGS_STREAM_DOWN_LEVELS");
    return v ? std::max(1, atoi(v)) : 1;
  }();
  static const int nu = [] {
    const char *v = getenv("GDGS_STREAM_UP_LEVELS");
    return v ? std::max(1, atoi(v)) : 3;
  }();
  return down ? nd : nu;
}

inline bool use_stream(const LvArgs &a, bool down) {
  return a.g.W % 2 == 0 && a.g.shift < stream_levels(down) && stream_enabled();
}

// Segments: the shortest height (a multiple of 8, at least 16 rows) that gives one launch at
// most ~10.5 warps per SM. Each segment recomputes a few halo rows and starts
// with a latency it cannot hide, so segments should be long; each warp runs its
// rows in order, so there should be enough of them to switch between. Measured
// best: 24 rows at 1080p (1575 warps per channel), 96 at 2160p (1587).
StreamGrid stream_grid(const LevelGeom &g, int C) {
  static const int sms = [] {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 0;
    return n > 0 ? n : 152;
  }();
  StreamGrid sg;
  sg.nstrips = (g.W + kStripOut - 1) / kStripOut;
  const int hev = (g.H + 1) & ~1;
  sg.S = stream_rows_env();
  if (sg.S == 0) {
    const long long target = (long long)sms * 21 / 2;
    const long long nseg = std::max(1LL, target / ((long long)sg.nstrips * std::max(C, 1)));
    const long long S = (hev + nseg - 1) / nseg;
    sg.S = (int)std::max(16LL, (S + 7) & ~7LL);
  }
  sg.nseg = (hev + sg.S - 1) / sg.S;
  return sg;
}

template <int SF>
cudaError_t launch_stream_t(bool down, const LvArgs &a, Ctrl *ctrl, int k, int first, int C, cudaStream_t st) {
  const StreamGrid sg = stream_grid(a.g, C);
  const int warps = sg.nstrips * sg.nseg;
  const dim3 grid((warps + kStreamThreads / 32 - 1) / (kStreamThreads / 32), 1, C);
  const dim3 block(kStreamThreads);
  if (down) {
    LaunchScope ls_(kDownName[a.g.shift], st);
    if (a.level0) launch_k(mg_down_stream_kernel<SF, true>, grid, block, 0, st, a, ctrl, k, first, sg);
    else launch_k(mg_down_stream_kernel<SF, false>, grid, block, 0, st, a, ctrl, k, first, sg);
  } else {
    LaunchScope ls_(kUpName[a.g.shift], st);
    if (a.level0) launch_k(mg0_up_stream_kernel<SF>, grid, block, 0, st, a, ctrl, k, sg);
    else launch_k(mg_upc_stream_kernel<SF>, grid, block, 0, st, a, ctrl, k, sg);
  }
  return cudaGetLastError();
}

cudaError_t launch_stream(bool down, const LvArgs &a, Ctrl *ctrl, int k, int first, int C, cudaStream_t st) {
  switch (a.sf) {
    case GDGS_STORAGE_BF16: return launch_stream_t<GDGS_STORAGE_BF16>(down, a, ctrl, k, first, C, st);
    case GDGS_STORAGE_F16: return launch_stream_t<GDGS_STORAGE_F16>(down, a, ctrl, k, first, C, st);
    default: return launch_stream_t<GDGS_STORAGE_F32>(down, a, ctrl, k, first, C, st);
  }
}

template <int NU>
cudaError_t launch_mg_down(const LvArgs &a, Ctrl *ctrl, int k, int first, int C, cudaStream_t st) {
  if (NU == 2 && use_stream(a, true)) return launch_stream(true, a, ctrl, k, first, C, st);
  return small_level(a.g) ? launch_mg_down_t<NU, 16, 64>(a, ctrl, k, first, C, st)
                          : launch_mg_down_t<NU, 32, 128>(a, ctrl, k, first, C, st);
}

template <int NU>
cudaError_t launch_mg_up(const LvArgs &a, Ctrl *ctrl, int k, int C, cudaStream_t st) {
  if (NU == 1 && use_stream(a, false)) return launch_stream(false, a, ctrl, k, 0, C, st);
  return small_level(a.g) ? launch_mg_up_t<NU, 16, 64>(a, ctrl, k, C, st)
                          : launch_mg_up_t<NU, 32, 128>(a, ctrl, k, C, st);
}

inline size_t tail_smem(const Plan &p, int t) {
  return tail_layout(p.lv + t, p.levels - t, nullptr) * sizeof(float);
}

// First level of the tail kernel: the first level >= 1 with at most kTailCells
// cells per channel whose tail fits kTailSmemMax bytes of shared memory (only
// very elongated grids need a later one; the coarsest alone always fits).
constexpr size_t kTailSmemMax = 200 * 1024;

inline int tail_level(const Plan &p) {
  int t = 1;
  while (t < p.levels - 1 && (p.lv[t].plane > kTailCells || tail_smem(p, t) > kTailSmemMax)) ++t;
  return t;
}

// Everything one V-cycle launches, for workspace `ws` laid out by `p`: the
// tiled levels 0 .. t-1 down, the tail (levels t .. L), the tiled levels up.
struct Cycle {
  const Plan *p;
  char *ws;
  Ctrl *ctrl;
  int C, nu1, nu2;
  float omega;
  int storage;
  const double *Minv;

  int chan = 0;  // channel-split loop: the one channel it solves (C == 1, pointers offset)

  // level-l array at byte offset off (storage format), FP32 finest-level array
  char *lvl(size_t off, int l) const {
    return ws + off + (size_t)chan * (size_t)p->lv[l].plane * (storage == GDGS_STORAGE_F32 ? 4 : 2);
  }
  char *fin0(size_t off) const { return ws + off + (size_t)chan * (size_t)p->lv[0].plane * 4; }

  LvArgs level(int l) const {
    LvArgs a{};
    a.g = p->lv[l];
    a.gc = p->lv[l + 1];
    a.f = l > 0 ? (const void *)lvl(p->off_lf[l], l) : nullptr;
    a.u = l > 0 ? lvl(p->off_lu[l], l) : lvl(p->off_e0, 0);
    a.uo = l > 0 ? (void *)lvl(p->off_luo[l], l) : nullptr;
    a.fc = lvl(p->off_lf[l + 1], l + 1);
    a.uc = lvl(p->off_luo[l + 1], l + 1);
    a.sf = storage;
    a.fin = ldexpf(1.f, 2 * l);
    a.fout = ldexpf(1.f, -2 * (l + 1));
    a.level0 = l == 0;
    a.rho = (const float *)fin0(p->off_rho);
    a.rb[0] = (float *)fin0(p->off_r[0]);
    a.rb[1] = (float *)fin0(p->off_r[1]);
    a.uhi = (float *)fin0(p->off_uhi);
    a.ulo = (float *)fin0(p->off_ulo);
    a.omega = omega;
    return a;
  }
  int T() const { return tail_level(*p); }
  unsigned kernels() const { return 2u * (unsigned)T() + 2u; }

  TailArgs tail() const {
    TailArgs a{};
    const int t = T();
    a.n = p->levels - t;
    for (int i = 0; i < a.n; ++i) a.lv[i] = p->lv[t + i];
    tail_layout(a.lv, a.n, &a);
    a.f_top = lvl(p->off_lf[t], t);
    a.u_top = lvl(p->off_luo[t], t);
    a.sf = storage;
    a.fin = ldexpf(1.f, 2 * t);
    a.Minv = Minv;
    a.nu1 = nu1;
    a.nu2 = nu2;
    a.omega = omega;
    return a;
  }

  // Opt-in to large dynamic shared memory for every kernel of the cycle; done
  // before any capture (attributes are set once per kernel and device).
  template <int A, int B>
  cudaError_t prepare_t() const {
    cudaError_t e = set_smem<mg_down_kernel<A, 32, 128>>(DownShape<Geo<A, 32, 128>>::smem);
    if (e == cudaSuccess) e = set_smem<mg_down_kernel<A, 16, 64>>(DownShape<Geo<A, 16, 64>>::smem);
    if (e == cudaSuccess) e = set_smem<mg_up_kernel<B, 32, 128>>(UpShape<Geo<B, 32, 128>>::smem);
    if (e == cudaSuccess) e = set_smem<mg_up_kernel<B, 16, 64>>(UpShape<Geo<B, 16, 64>>::smem);
    if (e == cudaSuccess) e = set_smem<mg_tail_kernel>(tail_smem(*p, T()));
    return e;
  }
  cudaError_t prepare() const {
#define GDGS_PREP(A, B) \
  if (nu1 == A && nu2 == B) return prepare_t<A, B>();
    GDGS_PREP(1, 1) GDGS_PREP(1, 2) GDGS_PREP(1, 3)
    GDGS_PREP(2, 1) GDGS_PREP(2, 2) GDGS_PREP(2, 3)
    GDGS_PREP(3, 1) GDGS_PREP(3, 2) GDGS_PREP(3, 3)
#undef GDGS_PREP
    return cudaErrorInvalidValue;
  }

  // k >= 0: explicit cycle index; k < 0: read from ctrl->iter (graph body).
  cudaError_t launch(int k, cudaGraphConditionalHandle h, int in_graph, cudaStream_t st) const {
    cudaError_t e = cudaSuccess;
    const int t = T();
    for (int l = 0; l < t; ++l) {
      const LvArgs la = level(l);
      const int first = (l == 1);
      e = nu1 == 1 ? launch_mg_down<1>(la, ctrl, k, first, C, st)
          : nu1 == 2 ? launch_mg_down<2>(la, ctrl, k, first, C, st)
                     : launch_mg_down<3>(la, ctrl, k, first, C, st);
      if (e != cudaSuccess) return e;
    }
    {
      LaunchScope ls_("mg_tail", st);
      launch_k(mg_tail_kernel, C, kTailThreads, tail_smem(*p, t), st, tail(), ctrl, k, t == 1 ? 1 : 0);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    for (int l = t - 1; l >= 0; --l) {
      const LvArgs la = level(l);
      e = nu2 == 1 ? launch_mg_up<1>(la, ctrl, k, C, st)
          : nu2 == 2 ? launch_mg_up<2>(la, ctrl, k, C, st)
                     : launch_mg_up<3>(la, ctrl, k, C, st);
      if (e != cudaSuccess) return e;
    }
    {
      LaunchScope ls_("mg_advance", st);
      launch_k(advance_kernel, 1, 1, 0, st, ctrl, k, h, in_graph, kernels(),
                                      (long long)C * p->lv[0].plane);
    }
    return cudaGetLastError();
  }
};

// ---- graph executor: the cycle loop as a CUDA graph with a WHILE node whose
// body is one V-cycle; the advance kernel ends the loop on convergence, so no
// launch is spent after it. Kernel parameters reference the workspace only, so
// one graph serves every call on the same workspace, shape and options.

// The key pins every pointer the graph bakes in: the workspace base and the
// layout of the solver's regions inside it (which depends on n and the pair
// capacity as well as on the image shape).
struct GraphKey {
  int dev;
  const void *ws;
  const void *ctrl;  // the loop's control block (one per channel in a split solve)
  int chan;
  int C, H, W, nu1, nu2, max_cycles, levels, storage;
  float omega;
  size_t off_rho, off_coarse, total;
  bool operator<(const GraphKey &o) const {
    return std::tie(dev, ws, ctrl, chan, C, H, W, nu1, nu2, max_cycles, levels, storage, omega,
                    off_rho, off_coarse, total) <
           std::tie(o.dev, o.ws, o.ctrl, o.chan, o.C, o.H, o.W, o.nu1, o.nu2, o.max_cycles,
                    o.levels, o.storage, o.omega, o.off_rho, o.off_coarse, o.total);
  }
};

struct GraphEntry {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned long long last_use = 0;
};

std::mutex g_graph_mu;
std::map<GraphKey, GraphEntry> g_graphs;
unsigned long long g_graph_clock = 0;
constexpr size_t kMaxGraphs = 64;

bool graphs_enabled() {
  static const bool on = [] {
    const char *v = getenv("GDGS_GRAPHS");
    return !(v && v[0] == '0');
  }();
  return on;
}

cudaError_t build_cycle_graph(const Cycle &cy, GraphEntry *out) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
  cudaStream_t cs = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      diag_set_capturing(true);
      const cudaError_t le = cy.launch(-1, h, 1, cs);
      diag_set_capturing(false);
      e = cudaStreamEndCapture(cs, &body);
      if (le != cudaSuccess) e = le;
    }
  }
  if (cs) cudaStreamDestroy(cs);
  cudaGraphExec_t x = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return e;
  }
  out->graph = g;
  out->exec = x;
  return cudaSuccess;
}

cudaError_t launch_cycle_graph(const Cycle &cy, const GraphKey &key, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_graph_mu);
  auto it = g_graphs.find(key);
  if (it == g_graphs.end()) {
    if (g_graphs.size() >= kMaxGraphs) {  // evict the least recently used
      auto lru = g_graphs.begin();
      for (auto jt = g_graphs.begin(); jt != g_graphs.end(); ++jt)
        if (jt->second.last_use < lru->second.last_use) lru = jt;
      cudaDeviceSynchronize();
      cudaGraphExecDestroy(lru->second.exec);
      cudaGraphDestroy(lru->second.graph);
      g_graphs.erase(lru);
    }
    GraphEntry ent;
    cudaError_t e = build_cycle_graph(cy, &ent);
    if (e != cudaSuccess) return e;
    it = g_graphs.emplace(key, ent).first;
  }
  it->second.last_use = ++g_graph_clock;
  return cudaGraphLaunch(it->second.exec, st);
}

// While `st` is being captured into a graph (a caller recording a whole view):
// add the cycle loop to that graph as a conditional WHILE node whose body is one
// V-cycle, recorded on a helper stream, and make the rest of the capture depend
// on it. The loop then runs exactly as many cycles as it needs at replay.
cudaError_t capture_cycle_loop(const Cycle &cy, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  const cudaGraphEdgeData *edges = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &edges, &nd);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive || !g) return cudaErrorStreamCaptureInvalidated;
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, deps, edges, nd, &np);
  if (e != cudaSuccess) return e;
  static thread_local cudaStream_t helper = nullptr;
  if (!helper && (e = cudaStreamCreateWithFlags(&helper, cudaStreamNonBlocking)) != cudaSuccess) {
    helper = nullptr;
    return e;
  }
  cudaGraph_t body = np.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(helper, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return e;
  const cudaError_t le = cy.launch(-1, h, 1, helper);
  e = cudaStreamEndCapture(helper, &body);
  if (le != cudaSuccess) return le;
  if (e != cudaSuccess) return e;
  return cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

}  // namespace

unsigned long long graph_kernel_count() {
  unsigned long long v = 0;
  if (cudaMemcpyFromSymbol(&v, g_graph_kernels, sizeof(v)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return v;
}

// Four-pixel kernels: rows of a multiple of 4 floats and 16-byte aligned planes.
inline bool quad_path(int W, const void *p0, const void *p1) {
  return W % 4 == 0 && ((uintptr_t)p0 % 16) == 0 && ((uintptr_t)p1 % 16) == 0;
}

bool split_enabled() {
  static const bool on = [] {
    const char *v = getenv("GDGS_SPLIT");
    return !(v && v[0] == '0');
  }();
  return on;
}

// Helper streams and events of channel-split solves, one set per (device,
// caller stream), so that calls on different caller streams never share a
// helper stream; at most kMaxForkSets sets, the least recently used replaced.
struct ForkSet {
  cudaStream_t s[GDGS_MAX_CHANNELS] = {};
  cudaEvent_t ev[GDGS_MAX_CHANNELS] = {};
  unsigned long long last_use = 0;
};
constexpr size_t kMaxForkSets = 32;

cudaError_t fork_set(cudaStream_t st, ForkSet **out) {
  static std::mutex mu;
  static std::map<std::pair<int, cudaStream_t>, ForkSet> sets;
  static unsigned long long clock = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(dev, st);
  auto it = sets.find(key);
  if (it == sets.end()) {
    if (sets.size() >= kMaxForkSets) {
      auto lru = sets.begin();
      for (auto jt = sets.begin(); jt != sets.end(); ++jt)
        if (jt->second.last_use < lru->second.last_use) lru = jt;
      for (int c = 0; c < GDGS_MAX_CHANNELS; ++c) {
        if (lru->second.s[c]) cudaStreamDestroy(lru->second.s[c]);
        if (lru->second.ev[c]) cudaEventDestroy(lru->second.ev[c]);
      }
      sets.erase(lru);
    }
    ForkSet f;
    for (int c = 0; c < GDGS_MAX_CHANNELS && e == cudaSuccess; ++c) {
      if (c > 0) e = cudaStreamCreateWithFlags(&f.s[c], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f.ev[c], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
      for (int c = 0; c < GDGS_MAX_CHANNELS; ++c) {
        if (f.s[c]) cudaStreamDestroy(f.s[c]);
        if (f.ev[c]) cudaEventDestroy(f.ev[c]);
      }
      return e;
    }
    it = sets.emplace(key, f).first;
  }
  it->second.last_use = ++clock;
  *out = &it->second;
  return cudaSuccess;
}

// Blocks per channel of the four-pixel passes (256 threads, a grid-stride loop
// over quads): a fixed count, 8/3 per SM (eight CTAs per SM for three channels).
// Each block ends in FP64 atomics on per-channel (or one) addresses, so a block
// per 256 quads (thousands of atomics on one address) serialised at the end; and
// the count does not depend on the number of channels, so a channel's sums (and
// with them its solve) come out the same bits whether it is solved alone or with
// others.
int pixel_blocks(size_t quads) {
  static const int sms = [] {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 0;
    return n > 0 ? n : 152;
  }();
  const size_t need = (quads + 255) / 256;
  const size_t want = std::max<size_t>(1, (size_t)(8 * sms) / 3);
  return (int)std::max<size_t>(1, std::min(need, want));
}

cudaError_t run_poisson(const PoissonArgs &a, cudaStream_t st) {
  const Plan &p = *a.plan;
  char *ws = a.ws;
  Ctrl *ctrl = a.ctrl;
  float *rho = (float *)(ws + p.off_rho);
  float *uhi = (float *)(ws + p.off_uhi);
  float *ulo = (float *)(ws + p.off_ulo);
  cudaError_t e;

  DivArgs d{a.maps, a.mask, a.input_is_rho, a.threshold, a.C, a.H, a.W, a.tiles_x, rho, a.rtol,
            a.max_cycles};
  {
    const size_t plane = (size_t)a.H * a.W;
    if (quad_path(a.W, a.maps, rho)) {
      const int bx = pixel_blocks(plane / 4);
      LaunchScope ls_("divergence", st);
      launch_k(divergence4_kernel, dim3(bx, a.C), 256, 0, st, d, ctrl);
    } else {
      int bx = (int)((plane + 255) / 256);
      if (bx > 4096) bx = 4096;
      LaunchScope ls_("divergence", st);
      launch_k(divergence_kernel, dim3(bx, a.C), 256, 0, st, d, ctrl);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }

  // coarse factor (cached in the workspace)
  const LevelGeom &gcoarse = p.lv[p.levels - 1];
  CoarseTag want{};
  want.magic = 0x4744475343303031ull;  // "GDGSC001"
  want.H0 = a.H;
  want.W0 = a.W;
  want.levels = p.levels;
  want.Hc = gcoarse.H;
  want.Wc = gcoarse.W;
  want.nc = p.nc;
  want.version = 1;
  CoarseTag *tag = (CoarseTag *)(ws + p.off_coarse);
  double *Minv = (double *)(ws + p.off_coarse + kCoarseTagBytes);
  const bool split = a.C > 1 && split_enabled();
  Ctrl *sub = split ? (Ctrl *)(ws + p.off_sub) : nullptr;
  {
    LaunchScope ls_("coarse_setup", st);
    launch_k(coarse_setup_kernel, 1, 1024, 0, st, gcoarse, Minv, tag, want, ctrl, a.C,
                                            (long long)a.H * a.W, sub);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;

  Cycle cy{};
  cy.p = &p;
  cy.ws = ws;
  cy.ctrl = ctrl;
  cy.C = a.C;
  cy.nu1 = a.nu1;
  cy.nu2 = a.nu2;
  cy.omega = a.omega;
  cy.storage = a.storage;
  cy.Minv = Minv;
  if ((e = cy.prepare()) != cudaSuccess) return e;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cap);

  // The cycle loop of one Cycle on stream s: a WHILE node recorded into the
  // caller's capture, a cached graph, or direct launches.
  auto run_loop = [&](const Cycle &c, cudaStream_t s) -> cudaError_t {
    if (cap == cudaStreamCaptureStatusActive && graphs_enabled() && !diag_profiling())
      return capture_cycle_loop(c, s);
    if (graphs_enabled() && !diag_profiling() && cap == cudaStreamCaptureStatusNone) {
      int dev = 0;
      cudaGetDevice(&dev);
      const GraphKey key{dev,          ws,       c.ctrl,   c.chan,  c.C,       a.H,
                         a.W,          a.nu1,    a.nu2,    a.max_cycles, p.levels, a.storage,
                         a.omega,      p.off_rho, p.off_coarse, p.total};
      return launch_cycle_graph(c, key, s);
    }
    // direct launches: every cycle is enqueued; once the advance kernel has
    // recorded convergence the remaining ones return at their first check
    for (int k = 0; k < a.max_cycles; ++k) {
      const cudaError_t e2 = c.launch(k, 0, 0, s);
      if (e2 != cudaSuccess) return e2;
    }
    return cudaSuccess;
  };

  if (!split) {
    if ((e = run_loop(cy, st)) != cudaSuccess) return e;
  } else {
    // Channel split: each channel's cycle loop on a stream of its own (channel 0
    // on the caller's stream), so the latency-bound small levels of one channel
    // overlap the bandwidth-bound large levels of the others. A channel stops
    // when its own relative residual reaches rtol, which implies the
    // all-channel criterion. Forked from and joined back to the caller's stream
    // by events, so the call keeps plain stream order (and is capturable).
    // While the per-kernel profiler records, the channels' loops run one after
    // another on the caller's stream, so that each launch is timed alone.
    const bool fork = !diag_profiling();
    ForkSet *fk = nullptr;
    if (fork) {
      if ((e = fork_set(st, &fk)) != cudaSuccess) return e;
      if ((e = cudaEventRecord(fk->ev[0], st)) != cudaSuccess) return e;
      for (int c = 1; c < a.C; ++c)
        if ((e = cudaStreamWaitEvent(fk->s[c], fk->ev[0], 0)) != cudaSuccess) return e;
    }
    for (int c = 0; c < a.C; ++c) {
      Cycle cc = cy;
      cc.C = 1;
      cc.chan = c;
      cc.ctrl = sub + c;
      if ((e = run_loop(cc, (c == 0 || !fork) ? st : fk->s[c])) != cudaSuccess) return e;
    }
    for (int c = 1; fork && c < a.C; ++c) {
      if ((e = cudaEventRecord(fk->ev[c], fk->s[c])) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(st, fk->ev[c], 0)) != cudaSuccess) return e;
    }
    {
      LaunchScope ls_("merge_channels", st);
      launch_k(merge_channels_kernel, 1, 32, 0, st, ctrl, (const Ctrl *)sub, a.C);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }

  FinArgs fa{};
  fa.g0 = p.lv[0];
  fa.rho = rho;
  fa.uhi = uhi;
  fa.ulo = ulo;
  fa.image = a.image;
  for (int c = 0; c < GDGS_MAX_CHANNELS; ++c) fa.mean[c] = a.mean[c];
  {
    const size_t plane = (size_t)a.H * a.W;
    if (quad_path(a.W, a.image, rho)) {
      const int bx = pixel_blocks(plane / 4);
      LaunchScope ls_("finalize", st);
      launch_k(finalize4_kernel, dim3(bx, a.C), 256, 0, st, fa, ctrl);
    } else {
      int bx = (int)((plane + 255) / 256);
      if (bx > 2048) bx = 2048;
      LaunchScope ls_("finalize", st);
      launch_k(finalize_kernel, dim3(bx, a.C), 256, 0, st, fa, ctrl);
    }
  }
  return cudaGetLastError();
}

}  // namespace gdgs
