/*
 * FP64 oracle: projection and front-to-back compositing of gradient Gaussians.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow reference that the CUDA
 * path is checked against. It shares no code with the CUDA path; only tests,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.
 *
 * Everything is computed in double precision from float inputs, straight from
 * the paper's definitions:
 *   - Sigma = R S S^T R^T for the anisotropic 3D Gaussian (Sec. 1.2, Eq. 3dgs;
 *     the same kernel carries the Laplacian/gradient field in Eq. gdgs);
 *   - Sigma2D = J W Sigma W^T J^T with W the world-to-camera rotation and J the
 *     Jacobian of the pinhole projection at the camera-space centre
 *     (Eq. sig2d, repeated in Sec. 2.2 "Projection");
 *   - the front-to-back alpha composite in view-depth order of Eq. color, applied
 *     to the gradient attribute as in Eq. gdgs2d.
 * Readings where the paper is silent (dilation, clamps, stop threshold, footprint,
 * pixel centres, tie-break) are the options passed in; they are listed with the
 * design notes of the repository.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* One projected Gaussian is a row of ORC_STRIDE doubles. */
enum {
  ORC_VALID = 0, /* 1.0 if the Gaussian survives the culls, else 0.0 */
  ORC_DEPTH,     /* camera-space z */
  ORC_MX, ORC_MY, /* projected centre in pixels (x = column, y = row) */
  ORC_CA, ORC_CB, ORC_CC, /* conic = inverse of Sigma2D: [[CA, CB], [CB, CC]] */
  ORC_OPA,
  ORC_XMIN, ORC_XMAX, ORC_YMIN, ORC_YMAX, /* exact footprint box (pixel coords) */
  ORC_S00, ORC_S01, ORC_S11, /* Sigma2D including the dilation */
  ORC_KEY,       /* float32 depth key that decides the order (exact in double) */
  ORC_STRIDE
};

/* cam: w2c[12] (row-major 3x4), fx, fy, cx, cy, near  -> 17 doubles
 * opt: dilation, exp_coef, alpha_min                  -> 3 doubles */
void oracle_project(int64_t n, const float *mean, const float *scale,
                    const float *quat, const float *opacity, const double *cam,
                    const double *opt, double *out) {
  const double *w = cam; /* w2c */
  const double fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
  const double znear = cam[16];
  const double dil = opt[0], kexp = opt[1], amin = opt[2];
  float w32[12];
  for (int i = 0; i < 12; ++i) w32[i] = (float)w[i];
  for (int64_t k = 0; k < n; ++k) {
    double *o = out + k * ORC_STRIDE;
    memset(o, 0, sizeof(double) * ORC_STRIDE);
    /* rotation from the (w, x, y, z) quaternion, normalised first */
    double qw = quat[4 * k + 0], qx = quat[4 * k + 1], qy = quat[4 * k + 2],
           qz = quat[4 * k + 3];
    double qn = qw * qw + qx * qx + qy * qy + qz * qz;
    if (!(qn > 1e-20)) continue;
    qn = 1.0 / sqrt(qn);
    qw *= qn; qx *= qn; qy *= qn; qz *= qn;
    double R[3][3] = {
        {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)},
        {2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)},
        {2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)}};
    double s[3] = {scale[3 * k], scale[3 * k + 1], scale[3 * k + 2]};
    /* Sigma = R S S^T R^T */
    double Sig[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double acc = 0;
        for (int m = 0; m < 3; ++m) acc += R[i][m] * s[m] * s[m] * R[j][m];
        Sig[i][j] = acc;
      }
    /* camera-space centre t = W mu + w_t */
    double t[3];
    for (int i = 0; i < 3; ++i)
      t[i] = w[4 * i] * mean[3 * k] + w[4 * i + 1] * mean[3 * k + 1] +
             w[4 * i + 2] * mean[3 * k + 2] + w[4 * i + 3];
    /* The view-depth order ("sorted from the view direction", Eq. color) and the
     * near cull are integer decisions; they are taken on the float32 key
     *   key = fma(w20, mx, fma(w21, my, fma(w22, mz, w23)))
     * (single-rounding IEEE fmaf), the precision the GPU path sorts in. */
    float key = fmaf(w32[8], mean[3 * k],
                     fmaf(w32[9], mean[3 * k + 1],
                          fmaf(w32[10], mean[3 * k + 2], w32[11])));
    if (!(key > (float)znear)) continue;
    /* J: Jacobian of (fx x/z + cx, fy y/z + cy) at t */
    double J[2][3] = {{fx / t[2], 0.0, -fx * t[0] / (t[2] * t[2])},
                      {0.0, fy / t[2], -fy * t[1] / (t[2] * t[2])}};
    /* T = J W (2x3), Sigma2D = T Sigma T^T */
    double T[2][3];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 3; ++j)
        T[i][j] = J[i][0] * w[j] + J[i][1] * w[4 + j] + J[i][2] * w[8 + j];
    double S2[2][2];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        double acc = 0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) acc += T[i][a] * Sig[a][b] * T[j][b];
        S2[i][j] = acc;
      }
    S2[0][0] += dil;
    S2[1][1] += dil;
    double det = S2[0][0] * S2[1][1] - S2[0][1] * S2[1][0];
    if (!(det > 0)) continue;
    double opa = opacity[k];
    if (!(opa >= amin)) continue; /* can never reach alpha_min */
    /* footprint: {d : kexp * d^T conic d <= ln(opa / alpha_min)} */
    double lev = log(opa / amin);
    double rx = sqrt(S2[0][0] * lev / kexp), ry = sqrt(S2[1][1] * lev / kexp);
    double mx = fx * t[0] / t[2] + cx, my = fy * t[1] / t[2] + cy;
    o[ORC_VALID] = 1.0;
    o[ORC_DEPTH] = t[2];
    o[ORC_KEY] = (double)key;
    o[ORC_MX] = mx;
    o[ORC_MY] = my;
    o[ORC_CA] = S2[1][1] / det;
    o[ORC_CB] = -S2[0][1] / det;
    o[ORC_CC] = S2[0][0] / det;
    o[ORC_OPA] = opa;
    o[ORC_XMIN] = mx - rx;
    o[ORC_XMAX] = mx + rx;
    o[ORC_YMIN] = my - ry;
    o[ORC_YMAX] = my + ry;
    o[ORC_S00] = S2[0][0];
    o[ORC_S01] = S2[0][1];
    o[ORC_S11] = S2[1][1];
  }
}

typedef struct {
  double kexp, amin, amax, tmin, amb_rel, depth_rel;
} orc_opts;

/* Composite one pixel centre (px, py) over the candidates `cand` (already in
 * ascending depth, ties by index). With check_box, candidates whose footprint
 * box does not contain the pixel centre are skipped first; this never changes
 * the result because the box contains every point where alpha >= alpha_min.
 * Returns the ambiguity flag: set when a discontinuous decision (alpha vs
 * alpha_min, T vs T_min, the order of two nearly equal depths) is taken within
 * a relative margin of its threshold. */
static int composite_pixel(double px, double py, const int64_t *cand, int64_t m,
                           int check_box, const double *proj, const float *grad,
                           int Q, const orc_opts *o, double *acc) {
  double T = 1.0;
  int amb = 0;
  double last_depth = -1.0;
  for (int q = 0; q < Q; ++q) acc[q] = 0.0;
  for (int64_t i = 0; i < m; ++i) {
    int64_t g = cand[i];
    const double *r = proj + g * ORC_STRIDE;
    if (check_box && (px < r[ORC_XMIN] || px > r[ORC_XMAX] || py < r[ORC_YMIN] ||
                      py > r[ORC_YMAX]))
      continue;
    double dx = px - r[ORC_MX], dy = py - r[ORC_MY];
    double power = o->kexp * (r[ORC_CA] * dx * dx + 2.0 * r[ORC_CB] * dx * dy +
                              r[ORC_CC] * dy * dy);
    double a = r[ORC_OPA] * exp(-power);
    if (a > o->amax) a = o->amax;
    if (fabs(a - o->amin) <= o->amb_rel * o->amin) amb = 1;
    if (a < o->amin) continue;
    /* The order is taken on the float32 key, ties by index, as on the GPU; a
     * nonzero depth_rel additionally flags near-ties of the key. */
    if (last_depth >= 0.0 && r[ORC_KEY] != last_depth &&
        fabs(r[ORC_KEY] - last_depth) <= o->depth_rel * r[ORC_KEY])
      amb = 1;
    last_depth = r[ORC_KEY];
    double wgt = a * T;
    for (int q = 0; q < Q; ++q) acc[q] += (double)grad[g * Q + q] * wgt;
    T *= (1.0 - a);
    if (fabs(T - o->tmin) <= o->amb_rel * o->tmin) amb = 1;
    if (T < o->tmin) break;
  }
  return amb;
}

/* opt: exp_coef, alpha_min, alpha_max, t_min, amb_rel, depth_rel.
 * order: the valid Gaussians sorted by (depth, index).
 * Q: attribute floats per Gaussian (2 per channel for gradients, 1 per channel
 * for the Laplacian field of Eq. gdgs).
 * Full image (pixels == NULL): out is [H*W][Q] in raster order, amb [H*W].
 * Pixel list: out is [n_pixels][Q], amb [n_pixels]; pixel id = row*W + col.
 * use_box = 0 composites every candidate at every pixel (the plain definition);
 * use_box = 1 pre-filters by the footprint box (same result, faster). */
void oracle_composite(const double *proj, const float *grad, int Q,
                      const int64_t *order, int64_t n_order, int W, int H,
                      int use_box, const double *opt, const int64_t *pixels,
                      int64_t n_pixels, int nthreads, double *out,
                      uint8_t *amb) {
  orc_opts o = {opt[0], opt[1], opt[2], opt[3], opt[4], opt[5]};
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  if (pixels) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < n_pixels; ++p) {
      int64_t row = pixels[p] / W, col = pixels[p] % W;
      amb[p] = (uint8_t)composite_pixel(col + 0.5, row + 0.5, order, n_order,
                                        use_box, proj, grad, Q, &o,
                                        out + p * Q);
    }
    return;
  }
#pragma omp parallel
  {
    int64_t *rowc = (int64_t *)malloc(sizeof(int64_t) * (n_order > 0 ? n_order : 1));
#pragma omp for schedule(dynamic, 1)
    for (int row = 0; row < H; ++row) {
      double py = row + 0.5;
      int64_t m = 0;
      if (use_box) {
        for (int64_t i = 0; i < n_order; ++i) {
          const double *r = proj + order[i] * ORC_STRIDE;
          if (py >= r[ORC_YMIN] && py <= r[ORC_YMAX]) rowc[m++] = order[i];
        }
      } else {
        memcpy(rowc, order, sizeof(int64_t) * n_order);
        m = n_order;
      }
      for (int col = 0; col < W; ++col) {
        int64_t p = (int64_t)row * W + col;
        amb[p] = (uint8_t)composite_pixel(col + 0.5, py, rowc, m, use_box, proj,
                                          grad, Q, &o, out + p * Q);
      }
    }
    free(rowc);
  }
}
