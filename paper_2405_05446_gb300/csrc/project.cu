// Projection of gradient Gaussians onto the image plane (K1).
//
// Per Gaussian: Sigma = R S S^T R^T from the quaternion and scales (Eq. 3dgs,
// the same kernel that carries the field in Eq. gdgs); camera transform;
// Sigma2D = J W Sigma W^T J^T with W the world-to-camera rotation and J the
// Jacobian of the pinhole map at the camera-space centre (Eq. sig2d, Sec. 2.2
// "Projection"); a low-pass dilation on the diagonal; conic = Sigma2D^-1; the
// exact footprint box of {alpha exp(-k d^T conic d) >= alpha_min}, widened by a
// relative 1e-4 plus 1e-3 px so binning never drops a pixel the composite uses;
// and the 16x16 tile rectangle it covers.
//
// Precision: the camera transform and the projected centre are computed in
// float-float arithmetic (about 44 bits) and stored as a (hi, lo) float pair. In FP32 the centre of a splat 1000 px from
// the origin carries ~1e-4 px of rounding, which moves alpha by ~1e-4 relative;
// the pair keeps the later per-pixel offset accurate to FP32 relative precision.
// The camera depth is a float-float pair (hi, lo) as well. The near cull compares
// the pair with the near plane, and the view-depth sort orders by hi and then by
// an 8-bit digit of lo in units of ulp(hi) / 256, so two depths are ordered as in
// exact arithmetic whenever they differ by more than 2^-31 relative (an FP32 key
// alone merges depths within 2^-24 and leaves their order to the index).
#include <math.h>

#include "gdgs_internal.cuh"

namespace gdgs {

namespace {

// Float-float numbers (value = hi + lo, |lo| <= ulp(hi) / 2) from error-free
// transformations: Knuth's TwoSum and the exact product by FMA. The _rn
// intrinsics keep the compiler from contracting or reassociating them. About
// 44 bits of precision, with FP32 instructions only (FP64 issues slowly here).
struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ FF ff_fast_sum(float a, float b) {  // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ FF ff_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ FF ff_add(FF x, FF y) {
  const FF s = ff_two_sum(x.hi, y.hi), t = ff_two_sum(x.lo, y.lo);
  const FF u = ff_fast_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return ff_fast_sum(u.hi, __fadd_rn(u.lo, t.lo));
}

__device__ __forceinline__ FF ff_mul(FF x, float y) {
  const FF p = ff_prod(x.hi, y);
  return ff_fast_sum(p.hi, __fmaf_rn(x.lo, y, p.lo));
}

__device__ __forceinline__ FF ff_div(FF x, FF y) {
  const float q1 = __fdiv_rn(x.hi, y.hi);
  const FF r = ff_add(x, ff_mul({-y.hi, -y.lo}, q1));
  return ff_fast_sum(q1, __fdiv_rn(r.hi, y.hi));
}

// w[0] x + w[1] y + w[2] z + w[3] as a float-float.
__device__ __forceinline__ FF ff_affine(const float *w, float x, float y, float z) {
  return ff_add(ff_add(ff_prod(w[0], x), ff_prod(w[1], y)), ff_add(ff_prod(w[2], z), FF{w[3], 0.f}));
}

// The 8-bit digit floor(lo / ulp(hi) * 256) + 128 of a normalised pair with
// hi > 0 (|lo| <= ulp(hi) / 2, so the digit lies in [0, 256]; 256 is clamped).
// For equal hi it is monotone in lo. The scaling by 2^(158 - e), e the biased
// exponent of hi, is exact (ldexpf of a power of two), and |lo| 2^(158 - e)
// <= 128. Very small depths (e < 31) get the middle digit.
__device__ __forceinline__ uint32_t depth_lo_digit(FF t) {
  const int e = (int)((__float_as_uint(t.hi) >> 23) & 0xffu);
  if (e < 31 || e == 255) return 128u;
  const float q = floorf(ldexpf(t.lo, 158 - e)) + 128.f;
  return (uint32_t)fminf(fmaxf(q, 0.f), 255.f);
}

__global__ void __launch_bounds__(256) project_kernel(ProjectArgs a) {
  griddep_enter();
  if (a.cam_dev) {  // camera from device memory (a graph replays for any camera)
    const gdgs_camera *cd = a.cam_dev;
#pragma unroll
    for (int j = 0; j < 12; ++j) a.w2c[j] = __ldg(&cd->world_to_cam[j]);
    a.fx = __ldg(&cd->fx);
    a.fy = __ldg(&cd->fy);
    a.cx = __ldg(&cd->cx);
    a.cy = __ldg(&cd->cy);
    // not validated on the host: a negative or NaN near plane reads as 0, so the
    // depth keys of visible Gaussians stay positive floats (their bits sort)
    a.znear = fmaxf(__ldg(&cd->near_plane), 0.f);
  }
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool visible = false;
  if (i < a.n) {
    const float mx = a.mean[3 * i], my = a.mean[3 * i + 1], mz = a.mean[3 * i + 2];
    const float s0 = a.scale[3 * i], s1 = a.scale[3 * i + 1], s2 = a.scale[3 * i + 2];
    float qw = a.quat[4 * i], qx = a.quat[4 * i + 1], qy = a.quat[4 * i + 2],
          qz = a.quat[4 * i + 3];
    const float opa = a.opacity[i];
    bool finite = isfinite(mx) && isfinite(my) && isfinite(mz) && isfinite(s0) &&
                  isfinite(s1) && isfinite(s2) && isfinite(qw) && isfinite(qx) &&
                  isfinite(qy) && isfinite(qz) && isfinite(opa);
    for (int q = 0; q < a.Q; ++q) finite = finite && isfinite(a.grad[i * a.Q + q]);
    if (!finite) set_status(a.ctrl, GDGS_ERR_NONFINITE);

    // camera depth t_z as a float-float pair; culled unless t_z > near
    const FF t2 = ff_affine(a.w2c + 8, mx, my, mz);
    const bool in_front = t2.hi > a.znear || (t2.hi == a.znear && t2.lo > 0.f);
    const float qn = qw * qw + qx * qx + qy * qy + qz * qz;
    bool ok = finite && qn > 1e-20f && in_front && opa >= a.alpha_min;

    float u_f = 0.f, v_f = 0.f, ca = 0.f, cb = 0.f, cc = 0.f, sxx = 0.f, sxy = 0.f, syy = 0.f;
    int tx0 = 0, tx1 = 0, ty0 = 0, ty1 = 0;
    if (ok) {
      const float inv = 1.0f / sqrtf(qn);
      qw *= inv; qx *= inv; qy *= inv; qz *= inv;
      // rotation (w, x, y, z) and M = R S
      const float R00 = 1.f - 2.f * (qy * qy + qz * qz), R01 = 2.f * (qx * qy - qw * qz),
                  R02 = 2.f * (qx * qz + qw * qy);
      const float R10 = 2.f * (qx * qy + qw * qz), R11 = 1.f - 2.f * (qx * qx + qz * qz),
                  R12 = 2.f * (qy * qz - qw * qx);
      const float R20 = 2.f * (qx * qz - qw * qy), R21 = 2.f * (qy * qz + qw * qx),
                  R22 = 1.f - 2.f * (qx * qx + qy * qy);
      const float M00 = R00 * s0, M01 = R01 * s1, M02 = R02 * s2;
      const float M10 = R10 * s0, M11 = R11 * s1, M12 = R12 * s2;
      const float M20 = R20 * s0, M21 = R21 * s1, M22 = R22 * s2;
      // Sigma = M M^T (symmetric)
      const float S00 = M00 * M00 + M01 * M01 + M02 * M02;
      const float S01 = M00 * M10 + M01 * M11 + M02 * M12;
      const float S02 = M00 * M20 + M01 * M21 + M02 * M22;
      const float S11 = M10 * M10 + M11 * M11 + M12 * M12;
      const float S12 = M10 * M20 + M11 * M21 + M12 * M22;
      const float S22 = M20 * M20 + M21 * M21 + M22 * M22;

      // camera-space centre and projected centre in float-float
      const FF t0 = ff_affine(a.w2c, mx, my, mz), t1 = ff_affine(a.w2c + 4, mx, my, mz);
      const FF u = ff_add(ff_mul(ff_div(t0, t2), a.fx), FF{a.cx, 0.f});
      const FF v = ff_add(ff_mul(ff_div(t1, t2), a.fy), FF{a.cy, 0.f});
      const float u_hi = u.hi, v_hi = v.hi, u_lo = u.lo, v_lo = v.lo;
      u_f = u_hi;
      v_f = v_hi;

      // J (2x3) at t, T = J W (2x3)
      const float tx = t0.hi, ty = t1.hi, tz = t2.hi;
      const float izf = 1.0f / tz;
      const float J00 = a.fx * izf, J02 = -a.fx * tx * izf * izf;
      const float J11 = a.fy * izf, J12 = -a.fy * ty * izf * izf;
      const float T00 = J00 * a.w2c[0] + J02 * a.w2c[8];
      const float T01 = J00 * a.w2c[1] + J02 * a.w2c[9];
      const float T02 = J00 * a.w2c[2] + J02 * a.w2c[10];
      const float T10 = J11 * a.w2c[4] + J12 * a.w2c[8];
      const float T11 = J11 * a.w2c[5] + J12 * a.w2c[9];
      const float T12 = J11 * a.w2c[6] + J12 * a.w2c[10];
      // (T Sigma)
      const float A00 = T00 * S00 + T01 * S01 + T02 * S02;
      const float A01 = T00 * S01 + T01 * S11 + T02 * S12;
      const float A02 = T00 * S02 + T01 * S12 + T02 * S22;
      const float A10 = T10 * S00 + T11 * S01 + T12 * S02;
      const float A11 = T10 * S01 + T11 * S11 + T12 * S12;
      const float A12 = T10 * S02 + T11 * S12 + T12 * S22;
      sxx = A00 * T00 + A01 * T01 + A02 * T02 + a.dilation;
      sxy = A00 * T10 + A01 * T11 + A02 * T12;
      syy = A10 * T10 + A11 * T11 + A12 * T12 + a.dilation;
      const float det = sxx * syy - sxy * sxy;
      ok = det > 0.f && isfinite(det) && isfinite(u_hi) && isfinite(v_hi);
      if (ok) {
        const float idet = 1.0f / det;
        ca = syy * idet;
        cb = -sxy * idet;
        cc = sxx * idet;
        const float lev = logf(opa / a.alpha_min);
        const float rx = sqrtf(sxx * lev / a.exp_coef) * 1.0001f + 1e-3f;
        const float ry = sqrtf(syy * lev / a.exp_coef) * 1.0001f + 1e-3f;
        // pixel j is in the box iff u - rx <= j + 0.5 <= u + rx
        const float inv_t = 1.0f / kTile;
        float fx0 = floorf((u_hi - rx - 0.5f) * inv_t);
        float fx1 = floorf((u_hi + rx - 0.5f) * inv_t) + 1.f;
        float fy0 = floorf((v_hi - ry - 0.5f) * inv_t);
        float fy1 = floorf((v_hi + ry - 0.5f) * inv_t) + 1.f;
        fx0 = fminf(fmaxf(fx0, 0.f), (float)a.tiles_x);
        fx1 = fminf(fmaxf(fx1, 0.f), (float)a.tiles_x);
        fy0 = fminf(fmaxf(fy0, 0.f), (float)a.tiles_y);
        fy1 = fminf(fmaxf(fy1, 0.f), (float)a.tiles_y);
        tx0 = (int)fx0; tx1 = (int)fx1; ty0 = (int)fy0; ty1 = (int)fy1;
        visible = tx1 > tx0 && ty1 > ty0;
        if (visible) {
          const float k2 = a.exp_coef * 1.4426950408889634f;  // exp(-x) = 2^(-x log2 e)
          a.smean[i] = make_float4(u_hi, v_hi, u_lo, v_lo);
          a.sconic[i] = make_float4(ca * k2, 2.f * cb * k2, cc * k2, opa);
        }
      }
    }
    if (!visible) { tx0 = tx1 = ty0 = ty1 = 0; }
    const float key = t2.hi;
    a.key[i] = visible ? __float_as_uint(key) : kInvalidKey;
    a.key_lo[i] = visible ? depth_lo_digit(t2) : 0u;
    a.rect[i] = make_uint2((unsigned)tx0 | ((unsigned)tx1 << 16), (unsigned)ty0 | ((unsigned)ty1 << 16));
    if (a.o_mean2d) {
      a.o_mean2d[2 * i] = visible ? u_f : 0.f;
      a.o_mean2d[2 * i + 1] = visible ? v_f : 0.f;
    }
    if (a.o_cov2d) {
      a.o_cov2d[3 * i] = visible ? sxx : 0.f;
      a.o_cov2d[3 * i + 1] = visible ? sxy : 0.f;
      a.o_cov2d[3 * i + 2] = visible ? syy : 0.f;
    }
    if (a.o_depth) a.o_depth[i] = visible ? key : 0.f;
    if (a.o_rect) {
      a.o_rect[4 * i] = tx0; a.o_rect[4 * i + 1] = ty0;
      a.o_rect[4 * i + 2] = tx1; a.o_rect[4 * i + 3] = ty1;
    }
  }
  const unsigned ball = __ballot_sync(0xffffffffu, visible);
  if ((threadIdx.x & 31) == 0 && ball) atomicAdd(&a.ctrl->n_visible, __popc(ball));
}

}  // namespace

cudaError_t launch_project(const ProjectArgs &a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = (unsigned)((a.n + threads - 1) / threads);
  { LaunchScope ls_("project", st); launch_k(project_kernel, blocks, threads, 0, st, a); }
  return cudaGetLastError();
}

}  // namespace gdgs
