// Binning of splats into 16x16 tiles in front-to-back order (K2-K4).
//
// The composite of Eq. color / Eq. gdgs2d visits splats "sorted from the view
// direction". The path orders them in two stable sorts instead of one wide key:
//   1. sort the Gaussians by their camera depth, held as a float-float pair
//      (hi, lo): one pass over an 8-bit digit of lo in units of ulp(hi) / 256,
//      then four passes over the float bits of hi (positive floats sort as
//      unsigned integers). Pairs with equal hi are thereby ordered by lo, which
//      resolves the depth to 2^-31 relative instead of float32's 2^-24 (N items);
//   2. walk them in that order, emit one (tile, Gaussian) pair per touched tile,
//      so pairs come out depth-ordered;
//   3. stable-sort the pairs by tile id only (ceil(log2 T) bits, 2 passes at
//      1080p). Stability keeps depth order inside each tile, ties by index.
// Compared with a 64-bit (tile | depth) key this sorts 13 instead of 45 bits per
// pair and moves 8 instead of 12 bytes per pair and pass.
//
// The radix sort is a classic LSD pass in three kernels (block histograms, one
// scan over digit-major histograms, stable scatter, which also scans the 256
// digit totals into the digit bases). Ranking inside a block is
// stable: items are taken in rounds of 256 consecutive keys; within a warp peers
// of a digit are found with __match_any_sync and ranked by lane; warps are
// ranked in order through a shared-memory prefix per digit.
#include <algorithm>

#include "gdgs_internal.cuh"

namespace gdgs {

namespace {

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ unsigned item_count(const unsigned long long *n_dev, unsigned cap) {
  if (!n_dev) return cap;
  const unsigned long long n = *n_dev;
  return n < cap ? (unsigned)n : cap;
}

template <int ITEMS>
__global__ void __launch_bounds__(kRadixThreads)
radix_hist_kernel(const uint32_t *keys, const unsigned long long *n_dev, unsigned cap,
                  int shift, unsigned mask, uint32_t *hist) {
  griddep_enter();
  __shared__ unsigned sh[256];
  const unsigned n = item_count(n_dev, cap);
  const unsigned nb = (n + kRadixThreads * ITEMS - 1) / (kRadixThreads * ITEMS);
  if (blockIdx.x >= nb) return;
  sh[threadIdx.x] = 0;
  __syncthreads();
  const unsigned base = blockIdx.x * (kRadixThreads * ITEMS);
#pragma unroll 4
  for (int r = 0; r < ITEMS; ++r) {
    const unsigned i = base + r * kRadixThreads + threadIdx.x;
    if (i < n) atomicAdd(&sh[(keys[i] >> shift) & mask], 1u);
  }
  __syncthreads();
  if (threadIdx.x <= mask) hist[threadIdx.x * nb + blockIdx.x] = sh[threadIdx.x];
}

// Block-wide exclusive scan of 32-bit values for 256 threads; *total = sum.
__device__ __forceinline__ unsigned scan256(unsigned v, unsigned *total) {
  __shared__ unsigned wt[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wt[w] = x;
  __syncthreads();
  unsigned before = 0, all = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k < w) before += wt[k];
    all += wt[k];
  }
  __syncthreads();
  *total = all;
  return x - v + before;
}

// Per digit d (one CTA each): exclusive scan of the block counts hist[d nb ..]
// in place; the digit's total goes to tot[d].
template <int ITEMS>
__global__ void __launch_bounds__(256)
radix_scan_digit_kernel(uint32_t *hist, uint32_t *tot, const unsigned long long *n_dev, unsigned cap) {
  griddep_enter();
  const unsigned n = item_count(n_dev, cap);
  const unsigned nb = (n + kRadixThreads * ITEMS - 1) / (kRadixThreads * ITEMS);
  uint32_t *h = hist + (size_t)blockIdx.x * nb;
  unsigned run = 0;
  for (unsigned base = 0; base < nb; base += 256) {
    const unsigned i = base + threadIdx.x;
    const unsigned v = i < nb ? h[i] : 0u;
    unsigned t;
    const unsigned ex = scan256(v, &t);
    if (i < nb) h[i] = run + ex;
    run += t;
  }
  if (threadIdx.x == 0) tot[blockIdx.x] = run;
}

// keys_next (nullable): the key written out for element i is keys_next[i]
// instead of the key ranked on, so a first pass over a secondary key leaves the
// primary keys in its order for the passes that follow. dtot: the digit totals;
// every block scans them into the digit bases itself (256 values: cheaper than a
// launch).
template <int ITEMS>
__global__ void __launch_bounds__(kRadixThreads)
radix_scatter_kernel(const uint32_t *keys_in, const uint32_t *vals_in, uint32_t *keys_out,
                     uint32_t *vals_out, const unsigned long long *n_dev, unsigned cap, int shift,
                     unsigned mask, const uint32_t *hist, const uint32_t *dtot,
                     const uint32_t *keys_next) {
  griddep_enter();
  constexpr int kWarps = kRadixThreads / 32;
  __shared__ unsigned run[256];
  __shared__ unsigned wcnt[kWarps][256];
  const unsigned n = item_count(n_dev, cap);
  const unsigned nb = (n + kRadixThreads * ITEMS - 1) / (kRadixThreads * ITEMS);
  if (blockIdx.x >= nb) return;
  const int w = threadIdx.x >> 5;
  {
    unsigned all;
    const unsigned dbase = scan256(threadIdx.x <= mask ? dtot[threadIdx.x] : 0u, &all);
    if (threadIdx.x <= mask) run[threadIdx.x] = dbase + hist[threadIdx.x * nb + blockIdx.x];
  }
  const unsigned base = blockIdx.x * (kRadixThreads * ITEMS);
  for (int r = 0; r < ITEMS; ++r) {
    const unsigned i = base + r * kRadixThreads + threadIdx.x;
    if (base + r * kRadixThreads >= n) break;  // uniform across the block
    const bool valid = i < n;
    const uint32_t key = valid ? keys_in[i] : 0u;
    const uint32_t val = valid ? (vals_in ? vals_in[i] : i) : 0u;
    const unsigned d = valid ? ((key >> shift) & mask) : 0x1000u;
    for (int t = threadIdx.x; t < kWarps * 256; t += kRadixThreads) (&wcnt[0][0])[t] = 0u;
    __syncthreads();
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned rank = __popc(peers & lanemask_lt());
    if (valid && rank == 0) wcnt[w][d] = __popc(peers);
    __syncthreads();
    if (threadIdx.x <= mask) {
      unsigned b2 = run[threadIdx.x];
#pragma unroll
      for (int k = 0; k < kWarps; ++k) {
        const unsigned c = wcnt[k][threadIdx.x];
        wcnt[k][threadIdx.x] = b2;
        b2 += c;
      }
      run[threadIdx.x] = b2;
    }
    __syncthreads();
    if (valid) {
      const unsigned pos = wcnt[w][d] + rank;
      keys_out[pos] = keys_next ? keys_next[i] : key;
      vals_out[pos] = val;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- pair emission

__device__ __forceinline__ unsigned rect_tiles(uint2 r) {
  const unsigned x0 = r.x & 0xffffu, x1 = r.x >> 16, y0 = r.y & 0xffffu, y1 = r.y >> 16;
  return (x1 - x0) * (y1 - y0);
}

// Block-wide exclusive scan of 64-bit values for 256 threads.
__device__ unsigned long long block_exclusive_scan(unsigned long long v, unsigned long long *total) {
  __shared__ unsigned long long wt[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wt[w] = x;
  __syncthreads();
  unsigned long long before = 0, all = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k < w) before += wt[k];
    all += wt[k];
  }
  __syncthreads();
  *total = all;
  return x - v + before;
}

// Sum of tile counts per block of kBinBlock depth-ordered Gaussians.
// The tiles a splat reaches: per row of tiles of its footprint box, the run of
// tiles whose box of pixel centres meets the ellipse p <= cut', where p = A dx^2
// + B dx dy + C dy^2 is the splat's exponent (conic with k log2 e folded in) and
// cut' the rasteriser's cut log2(opacity / alpha_min) + 1e-3 with a further
// 0.1 % + 0.01 of margin, so a dropped tile never holds a pixel where
// a >= alpha_min. The ellipse cut by a band of rows is convex, so its x-extent
// is one interval: on the right, the ellipse's rightmost point if that point's
// y lies in the band, else the larger value of the (concave) boundary function
// x = mx - B/(2A) dy + sqrt(cut'/A - D/(4A^2) dy^2), D = 4AC - B^2, at the
// band's ends; the left side likewise. A tile meets the ellipse iff its
// pixel-centre interval meets that extent.
struct Footprint {
  float mx, my, bx, cutA, dA, ry, rx, yr, yl;
  unsigned x0, x1, y0, y1;  // the box, in tiles (half open)
};

__device__ __forceinline__ Footprint footprint(const BinArgs &a, uint32_t g, uint2 rc) {
  Footprint f;
  const float4 m = a.smean[g], k = a.sconic[g];
  const float A = k.x, B = k.y, C = k.z;
  const float cut = (log2f(k.w / a.alpha_min) + 1e-3f) * 1.001f + 0.01f;
  const float D = fmaxf(4.f * A * C - B * B, 1e-30f);
  f.mx = m.x + m.z;
  f.my = m.y + m.w;
  f.bx = B / (2.f * A);         // x of the centre line: mx - bx dy
  f.cutA = cut / A;
  f.dA = D / (4.f * A * A);
  f.ry = sqrtf(cut * 4.f * A / D) * 1.0001f + 1e-3f;  // half extents
  f.rx = sqrtf(cut * 4.f * C / D) * 1.0001f + 1e-3f;
  const float by = B / (2.f * C);
  f.yr = f.my - by * f.rx;      // y of the rightmost point
  f.yl = f.my + by * f.rx;      // y of the leftmost point
  f.x0 = rc.x & 0xffffu;
  f.x1 = rc.x >> 16;
  f.y0 = rc.y & 0xffffu;
  f.y1 = rc.y >> 16;
  return f;
}

// Tiles [*lo, *hi) of row ty that the ellipse reaches (within the box).
__device__ __forceinline__ void row_span(const Footprint &f, unsigned ty, unsigned *lo,
                                         unsigned *hi) {
  *lo = *hi = f.x0;
  const float ya = fmaxf((float)(ty * kTile) + 0.5f, f.my - f.ry);
  const float yb = fminf((float)(ty * kTile) + (kTile - 0.5f), f.my + f.ry);
  if (ya > yb) return;
  auto hw = [&](float y) {
    const float d = y - f.my;
    return sqrtf(fmaxf(f.cutA - f.dA * d * d, 0.f));
  };
  const float ca = f.mx - f.bx * (ya - f.my), cb = f.mx - f.bx * (yb - f.my);
  const float wa = hw(ya), wb = hw(yb);
  const float xr = (f.yr >= ya && f.yr <= yb) ? f.mx + f.rx : fmaxf(ca + wa, cb + wb);
  const float xl = (f.yl >= ya && f.yl <= yb) ? f.mx - f.rx : fminf(ca - wa, cb - wb);
  // tile tx covers pixel centres [16 tx + 0.5, 16 tx + 15.5]
  const float tl = ceilf((xl - 1e-3f - (kTile - 0.5f)) / kTile);
  const float th = floorf((xr + 1e-3f - 0.5f) / kTile) + 1.f;
  const float l = fmaxf(tl, (float)f.x0), h = fminf(th, (float)f.x1);
  if (h > l) {
    *lo = (unsigned)l;
    *hi = (unsigned)h;
  }
}

__device__ __forceinline__ unsigned tiles_hit(const BinArgs &a, uint32_t g, uint2 rc) {
  const Footprint f = footprint(a, g, rc);
  unsigned c = 0;
  for (unsigned ty = f.y0; ty < f.y1; ++ty) {
    unsigned lo, hi;
    row_span(f, ty, &lo, &hi);
    c += hi - lo;
  }
  return c;
}

// One Gaussian per thread (kBinBlock per block): the block's sum of tile counts.
__global__ void __launch_bounds__(kBinBlock) count_kernel(BinArgs a) {
  griddep_enter();
  const int64_t i = (int64_t)blockIdx.x * kBinBlock + threadIdx.x;
  unsigned long long s = 0;
  if (i < a.n) {
    const uint32_t g = a.order[i];
    const uint2 rc = a.rect[g];
    if (rect_tiles(rc)) s = tiles_hit(a, g, rc);
    a.tiles[i] = (uint32_t)s;
  }
  unsigned long long tot;
  block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) a.blocksum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) blocksum_scan_kernel(BinArgs a, int nb) {
  griddep_enter();
  __shared__ unsigned long long wt[32];
  const int per = (nb + 1023) / 1024;
  const int b = threadIdx.x * per, e = min(b + per, nb);
  unsigned long long s = 0;
  for (int i = b; i < e; ++i) s += a.blocksum[i];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wt[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned long long t = wt[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    wt[lane] = t;
  }
  __syncthreads();
  unsigned long long run = x - s + (w > 0 ? wt[w - 1] : 0ull);
  for (int i = b; i < e; ++i) {
    const unsigned long long v = a.blocksum[i];
    a.blocksum[i] = run;
    run += v;
  }
  if (threadIdx.x == 1023) {
    const unsigned long long total = wt[31];
    a.ctrl->n_pairs = total;
    if (total > a.pair_cap) set_status(a.ctrl, GDGS_ERR_CAPACITY);
  }
}

// Pairs of one Gaussian per thread, at the offset its block's scan gives.
__global__ void __launch_bounds__(kBinBlock) emit_kernel(BinArgs a) {
  griddep_enter();
  const int64_t i = (int64_t)blockIdx.x * kBinBlock + threadIdx.x;
  const bool in = i < a.n;
  uint32_t g = 0;
  uint2 rc = make_uint2(0, 0);
  unsigned cnt = 0u;
  if (in) {
    g = a.order[i];
    rc = a.rect[g];
    cnt = a.tiles[i];  // as counted by count_kernel
  }
  unsigned long long tot;
  const unsigned long long my = a.blocksum[blockIdx.x] + block_exclusive_scan(cnt, &tot);
  if (cnt) {
    const Footprint f = footprint(a, g, rc);
    unsigned long long p = my;
    for (unsigned ty = f.y0; ty < f.y1; ++ty) {
      unsigned lo, hi;
      row_span(f, ty, &lo, &hi);
      for (unsigned tx = lo; tx < hi; ++tx, ++p)
        if (p < a.pair_cap) {
          a.pkey[p] = ty * (unsigned)a.tiles_x + tx;
          a.pval[p] = g;
        }
    }
  }
}

// Tile ranges from the boundaries in the tile-sorted keys, one pass over the
// pairs: pair i starts its tile's run when key[i-1] differs and ends it when
// key[i+1] differs. Ranges and mask are zeroed beforehand, so tiles without
// pairs read (0, 0) and 0. A run's first pair also appends its tile to
// `active` (order irrelevant: tiles are independent).
__global__ void __launch_bounds__(256)
ranges_kernel(const uint32_t *keys, Ctrl *ctrl, unsigned cap, uint2 *range, uint32_t *active,
              uint8_t *mask) {
  griddep_enter();
  const unsigned long long np = ctrl->n_pairs;
  const unsigned n = np < cap ? (unsigned)np : cap;
  unsigned *rw = reinterpret_cast<unsigned *>(range);
  const int lane = threadIdx.x & 31;
  const unsigned stride = gridDim.x * blockDim.x;
  for (unsigned i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {  // uniform per warp
    const unsigned i = i0 + threadIdx.x;
    const bool in = i < n;
    const uint32_t k = in ? keys[i] : 0u;
    const bool start = in && (i == 0 || keys[i - 1] != k);
    const bool end = in && (i + 1 == n || keys[i + 1] != k);
    if (start) {
      rw[2 * (size_t)k] = i;
      mask[k] = 1;
    }
    if (end) rw[2 * (size_t)k + 1] = i + 1;
    const unsigned ball = __ballot_sync(0xffffffffu, start);
    unsigned base = 0;
    if (lane == 0 && ball) base = atomicAdd(&ctrl->n_active, __popc(ball));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (start) active[base + __popc(ball & ((1u << lane) - 1u))] = k;
  }
}

}  // namespace

template <int ITEMS>
cudaError_t radix_pass(const uint32_t *ki, const uint32_t *vi, uint32_t *ko, uint32_t *vo,
                       const uint32_t *knext, const unsigned long long *n_dev, unsigned cap,
                       int shift, unsigned mask, uint32_t *hist, unsigned blocks,
                       cudaStream_t st) {
  { LaunchScope ls_("radix_hist", st); launch_k(radix_hist_kernel<ITEMS>, blocks, kRadixThreads, 0, st, ki, n_dev, cap, shift, mask, hist); }
  uint32_t *dtot = hist + (size_t)256 * blocks;
  { LaunchScope ls_("radix_scan", st); launch_k(radix_scan_digit_kernel<ITEMS>, mask + 1, 256, 0, st, hist, dtot, n_dev, cap); }
  {
    LaunchScope ls_("radix_scatter", st);
    launch_k(radix_scatter_kernel<ITEMS>, blocks, kRadixThreads, 0, st, ki, vi, ko, vo, n_dev, cap,
             shift, mask, (const uint32_t *)hist, (const uint32_t *)dtot, knext);
  }
  return cudaGetLastError();
}

template <int ITEMS>
cudaError_t radix_sort_t(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                         bool implicit_vals, const uint32_t *lo_keys,
                         const unsigned long long *n_dev, unsigned cap, int nbits,
                         uint32_t *hist, int max_blocks, bool *out_is_alt, cudaStream_t st) {
  uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
  bool alt = false;
  bool first = true;
  const unsigned blocks = (unsigned)max_blocks;
  if (blocks == 0) {
    *out_is_alt = false;
    return cudaSuccess;
  }
  if (lo_keys) {  // secondary key first (LSD): its low 8 bits, carrying the primary keys
    cudaError_t e = radix_pass<ITEMS>(lo_keys, implicit_vals ? nullptr : vi, ko, vo, ki, n_dev,
                                      cap, 0, 0xffu, hist, blocks, st);
    if (e != cudaSuccess) return e;
    first = false;
    uint32_t *t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
    alt = !alt;
  }
  for (int shift = 0; shift < nbits; shift += 8) {
    const int bits = nbits - shift < 8 ? nbits - shift : 8;
    const unsigned mask = (1u << bits) - 1u;
    cudaError_t e = radix_pass<ITEMS>(ki, (first && implicit_vals) ? nullptr : vi, ko, vo, nullptr,
                                      n_dev, cap, shift, mask, hist, blocks, st);
    if (e != cudaSuccess) return e;
    first = false;
    uint32_t *t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
    alt = !alt;
  }
  *out_is_alt = alt;
  return cudaGetLastError();
}

cudaError_t radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt,
                             uint32_t *vals_alt, bool implicit_vals, const uint32_t *lo_keys,
                             const unsigned long long *n_dev, unsigned cap, int nbits,
                             uint32_t *hist, int items, int max_blocks, bool *out_is_alt,
                             cudaStream_t st) {
  if (items == kRadixItemsSmall)
    return radix_sort_t<kRadixItemsSmall>(keys, vals, keys_alt, vals_alt, implicit_vals, lo_keys,
                                          n_dev, cap, nbits, hist, max_blocks, out_is_alt, st);
  if (items == kRadixItems)
    return radix_sort_t<kRadixItems>(keys, vals, keys_alt, vals_alt, implicit_vals, lo_keys, n_dev,
                                     cap, nbits, hist, max_blocks, out_is_alt, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_emit_pairs(const BinArgs &a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  const int nb = (int)((a.n + kBinBlock - 1) / kBinBlock);
  { LaunchScope ls_("pair_count", st); launch_k(count_kernel, nb, kBinBlock, 0, st, a); }
  { LaunchScope ls_("pair_scan", st); launch_k(blocksum_scan_kernel, 1, 1024, 0, st, a, nb); }
  { LaunchScope ls_("pair_emit", st); launch_k(emit_kernel, nb, kBinBlock, 0, st, a); }
  return cudaGetLastError();
}

cudaError_t launch_tile_ranges(const uint32_t *sorted_keys, Ctrl *ctrl, unsigned pair_cap,
                               int T, uint2 *range, uint32_t *active, uint8_t *mask,
                               cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(range, 0, 8 * (size_t)T, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(mask, 0, (size_t)T, st);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)std::min<unsigned long long>((pair_cap + 255ull) / 256, 2048);
  if (blocks == 0) return cudaSuccess;
  { LaunchScope ls_("tile_ranges", st); launch_k(ranges_kernel, blocks, 256, 0, st, sorted_keys, ctrl, pair_cap, range, active, mask); }
  return cudaGetLastError();
}

}  // namespace gdgs
