// Tile rasteriser of the per-Gaussian attribute (K5): the gradient (gx, gy per
// channel) or, in the paper-literal form, the Laplacian value per channel.
//
// One CTA of 256 threads per non-empty 16x16 tile, one pixel per thread. The
// tile's splats are already in front-to-back order (sort.cu); they are staged in
// batches of 256 into shared memory and every pixel composites them as in
// Eq. gdgs2d (Eq. color with the gradient attribute):
//   G = exp(-k d^T conic d), a = min(alpha_max, alpha G), skip a < alpha_min,
//   acc += g a T, T -= a T, stop once T < t_min.
// Tiles no splat reaches are never launched (the field is sparse, Sec. 2.2).
//
// The splat is staged relative to the tile origin (stage_splat): its centre's
// (hi, lo) pair becomes a grid part that pixel centres subtract exactly and a
// remainder folded into the expanded exponent, so alpha keeps FP32 relative
// precision anywhere in the image. alpha = 2^(L - p2) with L = log2(opacity)
// (ex2.approx; k log2 e is folded into the conic at projection); splats whose
// exponent already puts them below alpha_min (with a 1e-3 margin in the
// exponent) are skipped without the exponential.
//
// A warp holds a 4 x 8 pixel block of the tile (warp w: rows 4 (w >> 1) .. +3,
// columns 8 (w & 1) .. +7). When a batch is staged, every splat also gets the
// mask of the warps whose blocks its ellipse's bounding box can reach (closed
// form, with the binning's margins), and each warp compacts the batch into a
// list of its own in front-to-back order, so a warp never evaluates a splat that
// cannot reach its block (it would have been skipped by the exponent test at
// every pixel there). A compact block is reached by fewer of the small splats
// than a strip of two full rows.
#include "gdgs_internal.cuh"

namespace gdgs {

namespace {

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int Q>
__global__ void __launch_bounds__(256) raster_kernel(RasterArgs a) {
  griddep_enter();
  constexpr int QV = (Q + 3) / 4;  // float4 slots of the gradient attribute
  // splat batch, packed so that one pixel-splat evaluation reads 2 broadcast
  // 16-byte words (plus QV more when the splat contributes)
  __shared__ float4 s_geo[256];   // h_x, h_y (tile-relative grid part), conic A, B'
  __shared__ float4 s_geo2[256];  // conic C, L, linear terms a, b (see StagedSplat)
  __shared__ float4 s_g[QV][256];
  __shared__ uint8_t s_wmask[256];         // warps (row pairs) each splat of the batch can reach
  __shared__ uint8_t s_list[8][256];       // per warp: the batch's splats that can reach it
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned ntiles = a.use_active ? a.ctrl->n_active : (unsigned)a.T;
  if (blockIdx.x >= ntiles) return;
  const int tile = a.use_active ? (int)a.active[blockIdx.x] : (int)blockIdx.x;
  const int tyi = tile / a.tiles_x, txi = tile - tyi * a.tiles_x;
  const int x0 = txi * kTile, y0 = tyi * kTile;
  const int lx = 8 * (warp & 1) + (lane & 7), ly = 4 * (warp >> 1) + (lane >> 3);
  const int px = x0 + lx, py = y0 + ly;
  const bool inside = px < a.W && py < a.H;
  const float fpx = lx + 0.5f, fpy = ly + 0.5f;
  const float x0f = (float)x0, y0f = (float)y0;
  const uint2 rg = a.range[tile];
  const float amin = a.alpha_min, amax = a.alpha_max, tmin = a.t_min;
  const float cut = log2f(amin) - 1e-3f;  // skip when L - p2 < cut

  float acc[QV * 4];
#pragma unroll
  for (int q = 0; q < QV * 4; ++q) acc[q] = 0.f;
  float T = 1.f;
  bool done = !inside;

  for (unsigned s = rg.x; s < rg.y; s += 256) {
    if (__syncthreads_and(done)) break;
    const unsigned j = s + threadIdx.x;
    if (j < rg.y) {
      const uint32_t g = a.pval[j];
      const float4 kc = a.sconic[g];
      const StagedSplat st = stage_splat(a.smean[g], kc, x0f, y0f);
      s_geo[threadIdx.x] = st.geo;
      s_geo2[threadIdx.x] = st.geo2;
      s_wmask[threadIdx.x] = warp_block_mask(st, kc, amin);
      const float *gp = a.grad + (size_t)g * Q;
      float gv[QV * 4];
#pragma unroll
      for (int q = 0; q < QV * 4; ++q) gv[q] = 0.f;
      if (Q % 2 == 0 && a.grad_pairs) {  // 8-byte aligned rows: one 8-byte load per two floats
#pragma unroll
        for (int q = 0; q < Q; q += 2) {
          const float2 v2 = __ldg(reinterpret_cast<const float2 *>(gp + q));
          gv[q] = v2.x;
          gv[q + 1] = v2.y;
        }
      } else {
#pragma unroll
        for (int q = 0; q < Q; ++q) gv[q] = __ldg(gp + q);
      }
#pragma unroll
      for (int v = 0; v < QV; ++v)
        s_g[v][threadIdx.x] = make_float4(gv[4 * v], gv[4 * v + 1], gv[4 * v + 2], gv[4 * v + 3]);
    }
    __syncthreads();
    const int cnt = min(256u, rg.y - s);
    const int nl = warp_list(s_wmask, cnt, s_list[warp], warp, lane);  // this warp's list
    if (!done) {
      for (int i = 0; i < nl; ++i) {
        const int k = s_list[warp][i];
        const float4 ge = s_geo[k];
        const float4 ge2 = s_geo2[k];
        float X, Y;
        const float t = ge2.y - staged_exponent(ge, ge2, fpx, fpy, X, Y);
        if (t < cut) continue;
        const float al = fminf(amax, ex2_approx(t));
        if (al < amin) continue;
        const float w = __fmul_rn(al, T);
#pragma unroll
        for (int v = 0; v < QV; ++v) {
          const float4 gg = s_g[v][k];
          const float gq[4] = {gg.x, gg.y, gg.z, gg.w};
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (4 * v + c < Q) acc[4 * v + c] = fmaf(gq[c], w, acc[4 * v + c]);
        }
        T = __fsub_rn(T, w);  // T (1 - a), reusing the weight (the backward replays this)
        if (T < tmin) {
          done = true;
          break;
        }
      }
    }
  }
  if (inside) {
    const size_t plane = (size_t)a.H * a.W;
    const size_t o = (size_t)py * a.W + px;
#pragma unroll
    for (int q = 0; q < Q; ++q) a.maps[q * plane + o] = acc[q];
  }
}

}  // namespace

cudaError_t launch_raster(const RasterArgs &a_in, cudaStream_t st) {
  if (a_in.T == 0) return cudaSuccess;
  RasterArgs a = a_in;
  a.grad_pairs = (a.Q % 2 == 0 && (reinterpret_cast<uintptr_t>(a.grad) & 7u) == 0) ? 1 : 0;
  LaunchScope ls_("raster", st);
  switch (a.Q) {
    case 1: launch_k(raster_kernel<1>, a.T, 256, 0, st, a); break;
    case 2: launch_k(raster_kernel<2>, a.T, 256, 0, st, a); break;
    case 3: launch_k(raster_kernel<3>, a.T, 256, 0, st, a); break;
    case 4: launch_k(raster_kernel<4>, a.T, 256, 0, st, a); break;
    case 6: launch_k(raster_kernel<6>, a.T, 256, 0, st, a); break;
    case 8: launch_k(raster_kernel<8>, a.T, 256, 0, st, a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace gdgs
