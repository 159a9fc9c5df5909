// Backward of the render path: d(loss)/d(image) -> d(loss)/d(Gaussian parameters).
//
// The render is image = S(T(D(M(theta)))): M the front-to-back composite of the
// projected splats (Eq. gdgs2d), D the divergence (gradient attribute) or the
// identity (Laplacian attribute, Eq. gdgs), T the hard threshold (Eq. thresh),
// S the Neumann solve with the mean of rho removed and the supplied mean added
// (Eq. p2d). Backwards:
//   S^T  L is symmetric on zero-mean fields, so d rho = the same zero-mean solve
//        of d image (run by the caller's solver call into a second workspace);
//   T^T  d rho_raw = d rho where the threshold kept rho (rho != 0), else 0;
//   D^T  the transpose of the zero-flux divergence: d gx(i,j) = d rho(i,j) -
//        d rho(i,j+1) for j < W-1 (a negative forward difference), same for gy;
//        tiles the forward masked contribute nothing;
//   M^T  per tile, every pixel recomputes its forward pass (final transmittance
//        and last splat visited), then walks its splats back to front keeping
//        the transmittance before each splat (T / (1 - a)) and the attribute
//        composited behind it (B <- c a + (1 - a) B): dM/dc = a T_before,
//        dM/da = T_before (c - B); a = min(alpha_max, opacity 2^-p) gives the
//        opacity, centre and conic terms. Per-splat sums over a warp's pixels
//        go to global memory with one atomic per warp;
//   projection^T per Gaussian, from (d centre, d conic, d opacity) through
//        conic = Sigma2D^-1, Sigma2D = T Sigma T^T + dil I, T = J(t) W,
//        t = W mu + w, Sigma = R(q) S S^T R(q)^T and the quaternion's
//        normalisation. Alpha-test, stop and cull decisions have zero derivative.
#include <math.h>

#include "gdgs_internal.cuh"

namespace gdgs {

namespace {

__device__ __forceinline__ float ex2_approx_b(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ bool on_tile(const uint8_t *mask, int tiles_x, int i, int j) {
  return !mask || mask[(i / kTile) * tiles_x + (j / kTile)];
}

__global__ void __launch_bounds__(256) divergence_adjoint_kernel(DivAdjArgs a) {
  griddep_enter();
  const size_t plane = (size_t)a.H * a.W;
  const size_t total = plane * a.C;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < total;
       p += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(p / plane);
    const size_t q = p - (size_t)c * plane;
    const int i = (int)(q / a.W), j = (int)(q - (size_t)i * a.W);
    const float *rb = a.rbar + (size_t)c * plane;
    const float *rf = a.rho_fwd ? a.rho_fwd + (size_t)c * plane : nullptr;
    auto r = [&](size_t o) { return (rf && rf[o] == 0.f) ? 0.f : rb[o]; };
    const bool on = on_tile(a.mask, a.tiles_x, i, j);
    if (a.input_is_rho) {
      a.mbar[(size_t)c * plane + q] = on ? r(q) : 0.f;
    } else {
      const float r0 = r(q);
      a.mbar[(size_t)(2 * c) * plane + q] = (on && j + 1 < a.W) ? r0 - r(q + 1) : 0.f;
      a.mbar[(size_t)(2 * c + 1) * plane + q] = (on && i + 1 < a.H) ? r0 - r(q + a.W) : 0.f;
    }
  }
}

template <int N>
__device__ __forceinline__ void warp_sum(float (&v)[N]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
}

template <int Q>
__global__ void __launch_bounds__(256) raster_backward_kernel(RasterBwdArgs a) {
  griddep_enter();
  __shared__ float4 s_geo[256];   // as the forward rasteriser (StagedSplat)
  __shared__ float4 s_geo2[256];
  __shared__ float2 s_l[256];     // the centre's remainder l (offsets dx = X - l_x, ...)
  __shared__ float s_opa[256];
  __shared__ float s_g[Q][256];
  __shared__ uint32_t s_id[256];
  __shared__ uint8_t s_wmask[256];    // warps each staged splat can reach (as the forward)
  __shared__ uint8_t s_list[8][256];  // per warp: the batch's splats that can reach it
  __shared__ int s_last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned ntiles = a.ctrl->n_active;
  if (blockIdx.x >= ntiles) return;
  const int tile = (int)a.active[blockIdx.x];
  const int tyi = tile / a.tiles_x, txi = tile - tyi * a.tiles_x;
  const int x0 = txi * kTile, y0 = tyi * kTile;
  const int lx = 8 * (warp & 1) + (lane & 7), ly = 4 * (warp >> 1) + (lane >> 3);  // 4 x 8 blocks
  const int px = x0 + lx, py = y0 + ly;
  const bool inside = px < a.W && py < a.H;
  const float fpx = lx + 0.5f, fpy = ly + 0.5f;
  const float x0f = (float)x0, y0f = (float)y0;
  const uint2 rg = a.range[tile];
  const float amin = a.alpha_min, amax = a.alpha_max, tmin = a.t_min;
  const float cut = log2f(amin) - 1e-3f;
  const size_t plane = (size_t)a.H * a.W;
  const size_t po = (size_t)py * a.W + px;
  if (threadIdx.x == 0) s_last = -1;

  auto stage = [&](unsigned s) {
    const unsigned j = s + threadIdx.x;
    if (j < rg.y) {
      const uint32_t g = a.pval[j];
      const float4 k = a.sconic[g];
      const StagedSplat st = stage_splat(a.smean[g], k, x0f, y0f);
      s_geo[threadIdx.x] = st.geo;
      s_geo2[threadIdx.x] = st.geo2;
      s_l[threadIdx.x] = make_float2(st.lx, st.ly);
      s_opa[threadIdx.x] = k.w;
      s_id[threadIdx.x] = g;
      s_wmask[threadIdx.x] = warp_block_mask(st, k, amin);
#pragma unroll
      for (int q = 0; q < Q; ++q) s_g[q][threadIdx.x] = a.attr[(size_t)g * Q + q];
    }
  };

  // 1. the forward pass again: final transmittance and the last splat visited
  float T = 1.f;
  int last = -1;
  bool done = !inside;
  for (unsigned s = rg.x; s < rg.y; s += 256) {
    if (__syncthreads_and(done)) break;
    stage(s);
    __syncthreads();
    const int cnt = min(256u, rg.y - s);
    const int nl = warp_list(s_wmask, cnt, s_list[warp], warp, lane);
    if (!done) {
      for (int i = 0; i < nl; ++i) {
        const int k = s_list[warp][i];
        const float4 ge = s_geo[k];
        const float4 ge2 = s_geo2[k];
        float X, Y;
        const float t = ge2.y - staged_exponent(ge, ge2, fpx, fpy, X, Y);
        if (t < cut) continue;
        const float al = fminf(amax, ex2_approx_b(t));
        if (al < amin) continue;
        T = __fsub_rn(T, __fmul_rn(al, T));  // exactly as the forward rasteriser
        last = (int)(s + k);
        if (T < tmin) {
          done = true;
          break;
        }
      }
    }
  }
  __syncthreads();
  if (last >= 0) atomicMax(&s_last, last);
  float mbar[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) mbar[q] = inside ? a.mbar[q * plane + po] : 0.f;
  __syncthreads();
  const int jmax = s_last;
  if (jmax < 0) return;  // uniform

  // 2. back to front
  float B[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) B[q] = 0.f;
  const unsigned first_batch = rg.x + (unsigned)(jmax - (int)rg.x) / 256u * 256u;
  for (int s = (int)first_batch; s >= (int)rg.x; s -= 256) {
    __syncthreads();
    stage((unsigned)s);
    __syncthreads();
    const int cnt = min(256, (int)rg.y - s);
    const int nl = warp_list(s_wmask, cnt, s_list[warp], warp, lane);
    for (int i = nl - 1; i >= 0; --i) {
      const int k = s_list[warp][i];
      if (k > jmax - s) continue;  // after the tile's last contributing splat
      const int j = s + k;
      float v[6 + Q];
#pragma unroll
      for (int t = 0; t < 6 + Q; ++t) v[t] = 0.f;
      bool any = false;
      if (inside && j <= last) {
        const float4 ge = s_geo[k];
        const float4 ge2 = s_geo2[k];
        float X, Y;
        const float t = ge2.y - staged_exponent(ge, ge2, fpx, fpy, X, Y);
        if (t >= cut) {
          const float araw = ex2_approx_b(t);  // opacity 2^-p2
          const float al = fminf(amax, araw);
          if (al >= amin) {
            const float Tb = T / (1.f - al);
            float dal = 0.f;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
              const float c = s_g[q][k];
              v[6 + q] = mbar[q] * al * Tb;
              dal = fmaf(mbar[q], Tb * (c - B[q]), dal);
              B[q] = fmaf(c, al, (1.f - al) * B[q]);
            }
            if (araw < amax) {  // not clamped: the opacity and the exponent move a
              const float gp = -dal * araw * 0.6931471805599453f;  // d loss / d p2
              const float2 l = s_l[k];
              const float dx = X - l.x, dy = Y - l.y;
              v[0] = -gp * (2.f * ge.z * dx + ge.w * dy);
              v[1] = -gp * (ge.w * dx + 2.f * ge2.x * dy);
              v[2] = gp * dx * dx;
              v[3] = gp * dx * dy;
              v[4] = gp * dy * dy;
              v[5] = dal * (araw / s_opa[k]);  // d alpha / d opacity = 2^-p2
            }
            T = Tb;
            any = true;
          }
        }
      }
      if (!__any_sync(0xffffffffu, any)) continue;
      warp_sum(v);
      if (lane == 0) {
        const uint32_t g = s_id[k];
#pragma unroll
        for (int t = 0; t < 6; ++t) atomicAdd(&a.dsplat[(size_t)g * 6 + t], v[t]);
#pragma unroll
        for (int q = 0; q < Q; ++q) atomicAdd(&a.dattr[(size_t)g * Q + q], v[6 + q]);
      }
    }
  }
}

__global__ void __launch_bounds__(256) project_backward_kernel(ProjBwdArgs a) {
  griddep_enter();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const float *ds = a.dsplat + (size_t)i * 6;
  float dmx = ds[0], dmy = ds[1], dA = ds[2], dB = ds[3], dC = ds[4], dopa = ds[5];
  float gm[3] = {0.f, 0.f, 0.f}, gs[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f};
  const bool any = dmx != 0.f || dmy != 0.f || dA != 0.f || dB != 0.f || dC != 0.f || dopa != 0.f;
  if (any) {
    const float *w = a.w2c;
    const float mx = a.mean[3 * i], my = a.mean[3 * i + 1], mz = a.mean[3 * i + 2];
    const float s0 = a.scale[3 * i], s1 = a.scale[3 * i + 1], s2 = a.scale[3 * i + 2];
    float qr[4] = {a.quat[4 * i], a.quat[4 * i + 1], a.quat[4 * i + 2], a.quat[4 * i + 3]};
    const float qlen = sqrtf(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
    const float qw = qr[0] / qlen, qx = qr[1] / qlen, qy = qr[2] / qlen, qz = qr[3] / qlen;
    float R[3][3] = {{1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy)},
                     {2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx)},
                     {2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)}};
    const float sv[3] = {s0, s1, s2};
    float M[3][3], Sig[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) M[r][c] = R[r][c] * sv[c];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) Sig[r][c] = M[r][0] * M[c][0] + M[r][1] * M[c][1] + M[r][2] * M[c][2];
    const float tx = w[0] * mx + w[1] * my + w[2] * mz + w[3];
    const float ty = w[4] * mx + w[5] * my + w[6] * mz + w[7];
    const float tz = w[8] * mx + w[9] * my + w[10] * mz + w[11];
    const float iz = 1.f / tz;
    float J[2][3] = {{a.fx * iz, 0.f, -a.fx * tx * iz * iz}, {0.f, a.fy * iz, -a.fy * ty * iz * iz}};
    float Tm[2][3];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 3; ++c) Tm[r][c] = J[r][0] * w[c] + J[r][1] * w[4 + c] + J[r][2] * w[8 + c];
    float TS[2][3];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 3; ++c) TS[r][c] = Tm[r][0] * Sig[0][c] + Tm[r][1] * Sig[1][c] + Tm[r][2] * Sig[2][c];
    const float sxx = TS[0][0] * Tm[0][0] + TS[0][1] * Tm[0][1] + TS[0][2] * Tm[0][2] + a.dilation;
    const float sxy = TS[0][0] * Tm[1][0] + TS[0][1] * Tm[1][1] + TS[0][2] * Tm[1][2];
    const float syy = TS[1][0] * Tm[1][0] + TS[1][1] * Tm[1][1] + TS[1][2] * Tm[1][2] + a.dilation;
    const float det = sxx * syy - sxy * sxy;
    const float ca = syy / det, cb = -sxy / det, cc = sxx / det;
    // d conic from the stored (A, B, C) = k2 (ca, 2 cb, cc)
    const float k2 = a.exp_coef * 1.4426950408889634f;
    const float g00 = dA * k2, g01 = dB * k2, g11 = dC * k2;  // dL/dC as a symmetric matrix
    // d Sigma2D = -C dC C
    const float c00 = ca, c01 = cb, c11 = cc;
    const float X00 = c00 * g00 + c01 * g01, X01 = c00 * g01 + c01 * g11;
    const float X10 = c01 * g00 + c11 * g01, X11 = c01 * g01 + c11 * g11;
    const float S00b = -(X00 * c00 + X01 * c01), S01b = -(X00 * c01 + X01 * c11);
    const float S10b = -(X10 * c00 + X11 * c01), S11b = -(X10 * c01 + X11 * c11);
    const float Sb[2][2] = {{S00b, 0.5f * (S01b + S10b)}, {0.5f * (S01b + S10b), S11b}};
    // d Sigma = T^T Sb T, d T = 2 Sb T Sigma
    float Sigb[3][3], Tb[2][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        Sigb[r][c] = Tm[0][r] * (Sb[0][0] * Tm[0][c] + Sb[0][1] * Tm[1][c]) +
                     Tm[1][r] * (Sb[1][0] * Tm[0][c] + Sb[1][1] * Tm[1][c]);
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 3; ++c) Tb[r][c] = 2.f * (Sb[r][0] * TS[0][c] + Sb[r][1] * TS[1][c]);
    // d J = d T W_R^T
    float Jb[2][3];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 3; ++c) Jb[r][c] = Tb[r][0] * w[4 * c] + Tb[r][1] * w[4 * c + 1] + Tb[r][2] * w[4 * c + 2];
    float tb[3];
    tb[0] = dmx * a.fx * iz + Jb[0][2] * (-a.fx * iz * iz);
    tb[1] = dmy * a.fy * iz + Jb[1][2] * (-a.fy * iz * iz);
    tb[2] = dmx * (-a.fx * tx * iz * iz) + dmy * (-a.fy * ty * iz * iz) +
            Jb[0][0] * (-a.fx * iz * iz) + Jb[0][2] * (2.f * a.fx * tx * iz * iz * iz) +
            Jb[1][1] * (-a.fy * iz * iz) + Jb[1][2] * (2.f * a.fy * ty * iz * iz * iz);
    for (int c = 0; c < 3; ++c) gm[c] = w[c] * tb[0] + w[4 + c] * tb[1] + w[8 + c] * tb[2];
    // Sigma = M M^T: d M = 2 d Sigma M (d Sigma symmetric)
    float Rb[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        const float Mb = 2.f * (Sigb[r][0] * M[0][c] + Sigb[r][1] * M[1][c] + Sigb[r][2] * M[2][c]);
        gs[c] += Mb * R[r][c];
        Rb[r][c] = Mb * sv[c];
      }
    // R(q) for the normalised q
    float qb[4];
    qb[0] = 2.f * (-qz * Rb[0][1] + qy * Rb[0][2] + qz * Rb[1][0] - qx * Rb[1][2] - qy * Rb[2][0] + qx * Rb[2][1]);
    qb[1] = 2.f * (qy * Rb[0][1] + qz * Rb[0][2] + qy * Rb[1][0] - 2.f * qx * Rb[1][1] - qw * Rb[1][2] +
                   qz * Rb[2][0] + qw * Rb[2][1] - 2.f * qx * Rb[2][2]);
    qb[2] = 2.f * (-2.f * qy * Rb[0][0] + qx * Rb[0][1] + qw * Rb[0][2] + qx * Rb[1][0] + qz * Rb[1][2] -
                   qw * Rb[2][0] + qz * Rb[2][1] - 2.f * qy * Rb[2][2]);
    qb[3] = 2.f * (-2.f * qz * Rb[0][0] - qw * Rb[0][1] + qx * Rb[0][2] + qw * Rb[1][0] - 2.f * qz * Rb[1][1] +
                   qy * Rb[1][2] + qx * Rb[2][0] + qy * Rb[2][1]);
    const float qn[4] = {qw, qx, qy, qz};
    const float dot = qn[0] * qb[0] + qn[1] * qb[1] + qn[2] * qb[2] + qn[3] * qb[3];
    for (int c = 0; c < 4; ++c) gq[c] = (qb[c] - qn[c] * dot) / qlen;
  }
  for (int c = 0; c < 3; ++c) a.d_mean[3 * i + c] = gm[c];
  for (int c = 0; c < 3; ++c) a.d_scale[3 * i + c] = gs[c];
  for (int c = 0; c < 4; ++c) a.d_quat[4 * i + c] = gq[c];
  a.d_opacity[i] = dopa;
}

}  // namespace

cudaError_t launch_divergence_adjoint(const DivAdjArgs &a, cudaStream_t st) {
  const size_t total = (size_t)a.C * a.H * a.W;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 8192) blocks = 8192;
  { LaunchScope ls_("divergence_adjoint", st); launch_k(divergence_adjoint_kernel, blocks, 256, 0, st, a); }
  return cudaGetLastError();
}

cudaError_t launch_raster_backward(const RasterBwdArgs &a, cudaStream_t st) {
  if (a.T == 0) return cudaSuccess;
  LaunchScope ls_("raster_backward", st);
  switch (a.Q) {
    case 1: launch_k(raster_backward_kernel<1>, a.T, 256, 0, st, a); break;
    case 2: launch_k(raster_backward_kernel<2>, a.T, 256, 0, st, a); break;
    case 3: launch_k(raster_backward_kernel<3>, a.T, 256, 0, st, a); break;
    case 4: launch_k(raster_backward_kernel<4>, a.T, 256, 0, st, a); break;
    case 6: launch_k(raster_backward_kernel<6>, a.T, 256, 0, st, a); break;
    case 8: launch_k(raster_backward_kernel<8>, a.T, 256, 0, st, a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_project_backward(const ProjBwdArgs &a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((a.n + 255) / 256);
  { LaunchScope ls_("project_backward", st); launch_k(project_backward_kernel, blocks, 256, 0, st, a); }
  return cudaGetLastError();
}

}  // namespace gdgs
