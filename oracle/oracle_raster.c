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
 *
 * Ambiguity. The method's result jumps at a few discrete decisions: whether a
 * Gaussian passes the near cull, the view-depth order of two Gaussians, whether
 * alpha reaches alpha_min, and whether T has fallen below T_min. A float32
 * evaluation of the same definitions can take such a decision the other way when
 * the FP64 quantity lies within the float32 rounding error of its threshold. For
 * each decision this file carries an a-priori bound on that error (first-order
 * float32 error analysis, unit roundoff u = 2^-24, stated where it is used) and
 * flags the pixel as ambiguous when the FP64 value lies within it. Only the flag
 * depends on these bounds; the composite itself is the plain FP64 definition.
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
  ORC_DERR,      /* float32 error bound of the camera depth (see oracle_project) */
  ORC_KAPPA,     /* condition number of Sigma2D (largest / smallest eigenvalue) */
  ORC_GHOST,     /* 1.0 if culled by the near plane only within ORC_DERR of it */
  ORC_NEARAMB,   /* 1.0 if the depth lies within ORC_DERR of the near plane */
  ORC_BOXW,      /* widening factor of the box for the ambiguity checks (>= 1) */
  ORC_TZ0, ORC_TZ1, ORC_TZ2, /* the depth's terms w20 x, w21 y, w22 z (exact in FP64) */
  ORC_LMAX,      /* largest eigenvalue of Sigma2D */
  ORC_STRIDE
};

/* unit roundoff of float32 */
#define ORC_U (1.0 / 16777216.0)

/* Float32 error model of the exponent p = k d^T Sigma2D^-1 d at a pixel (first
 * order, u = 2^-24), as an absolute error in p:
 *  - Sigma2D = J W Sigma W^T J^T evaluated in float32 is off by dSigma with
 *    ||dSigma|| <= C_SIGMA u lmax (about a dozen roundings along the longest
 *    chain, each relative to entries of size up to the largest eigenvalue lmax);
 *    since d(Sigma^-1) = -Sigma^-1 dSigma Sigma^-1, the form moves by at most
 *    ||dSigma|| |Sigma^-1 d|^2. Along the major axis of an elongated splat this
 *    is u p, along the minor axis u p kappa.
 *  - the float32 form A dx^2 + 2B dx dy + C dy^2 itself: C_F u times the sum of
 *    the magnitudes of its terms (large where the terms cancel);
 *  - the offset d from the pixel centre to the projected centre, rounded to
 *    float32 once per coordinate (|dd| <= u |d|): the form moves by
 *    2 |Sigma^-1 d| |dd|, so C_D u |Sigma^-1 d| |d|;
 *  - the exponent's own rounding and its scaling: C_P u max(p, 1).
 * A further C_EXP u (relative) covers the exponential, to a few ulp, and the
 * opacity's log or product. An absolute error e in p moves alpha by e of
 * itself, so the relative alpha error is the sum. An evaluation that rounds
 * the projected centre itself to float32 (an offset error of u times the pixel
 * coordinate, ~1e-4 px at x ~ 1000) is not covered. err_scale multiplies the
 * whole bound (1 by default; 0 turns the ambiguity flags off). */
#define ORC_C_SIGMA 16.0
#define ORC_C_F 3.0
#define ORC_C_D 4.0
#define ORC_C_P 8.0
#define ORC_C_EXP 8.0

/* row r of a projected Gaussian (see the enum) */
static double alpha_err_at(const double *r, double dx, double dy, double kexp,
                           double p, double err_scale) {
  double cdx = r[ORC_CA] * dx + r[ORC_CB] * dy, cdy = r[ORC_CB] * dx + r[ORC_CC] * dy;
  double lmax = r[ORC_LMAX];
  double form_abs = fabs(r[ORC_CA]) * dx * dx + 2.0 * fabs(r[ORC_CB] * dx * dy) +
                    fabs(r[ORC_CC]) * dy * dy;
  double cd = sqrt(cdx * cdx + cdy * cdy), dd = sqrt(dx * dx + dy * dy);
  double ep = kexp * (ORC_C_SIGMA * lmax * cd * cd + ORC_C_F * form_abs + ORC_C_D * cd * dd) +
              ORC_C_P * fmax(p, 1.0);
  return err_scale * ORC_U * (ep + ORC_C_EXP);
}

/* The largest relative alpha error on the alpha_min level of a Gaussian whose
 * exponent there is lev (minor-axis direction; the form's terms and the offset
 * term at most 2 kappa lev each). */
static double alpha_err_max(double lev, double kappa) {
  return ORC_U * ((ORC_C_SIGMA + 2.0 * ORC_C_F + 2.0 * ORC_C_D) * kappa * fmax(lev, 1.0) +
                  ORC_C_P * fmax(lev, 1.0) + ORC_C_EXP);
}

/* cam: w2c[12] (row-major 3x4), fx, fy, cx, cy, near  -> 17 doubles
 * opt: dilation, exp_coef, alpha_min, depth_rel       -> 4 doubles */
void oracle_project(int64_t n, const float *mean, const float *scale,
                    const float *quat, const float *opacity, const double *cam,
                    const double *opt, double *out) {
  const double *w = cam; /* w2c */
  const double fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
  const double znear = cam[16];
  const double dil = opt[0], kexp = opt[1], amin = opt[2], depth_rel = opt[3];
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
     * near cull are taken on the FP64 camera depth t_z. An implementation that
     * evaluates the depth with relative precision depth_rel (error at most
     * depth_rel * S, S the sum of the magnitudes of the affine form's terms
     * w20 x, w21 y, w22 z, w23) may order two depths closer than the sum of
     * their bounds either way, and may cull one within its bound of the near
     * plane either way. A plain float32 evaluation (three multiplies and three
     * adds, or three fused multiply-adds) has depth_rel = gamma_4 = 4u / (1 - 4u)
     * (Higham, Accuracy and Stability of Numerical Algorithms, Sec. 3.1). */
    double dsum = fabs(w[8] * mean[3 * k]) + fabs(w[9] * mean[3 * k + 1]) +
                  fabs(w[10] * mean[3 * k + 2]) + fabs(w[11]);
    double derr = depth_rel * dsum;
    int near_amb = fabs(t[2] - znear) <= derr;
    int ghost = 0;
    if (!(t[2] > znear)) {
      /* culled; kept as a ghost (no contribution, only the ambiguity flag) when
       * a float32 depth could still pass the cull */
      if (!(near_amb && t[2] > 0.0)) continue;
      ghost = 1;
    }
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
    o[ORC_VALID] = ghost ? 0.0 : 1.0;
    o[ORC_GHOST] = ghost ? 1.0 : 0.0;
    o[ORC_NEARAMB] = near_amb ? 1.0 : 0.0;
    o[ORC_DEPTH] = t[2];
    o[ORC_DERR] = derr;
    o[ORC_TZ0] = w[8] * mean[3 * k];
    o[ORC_TZ1] = w[9] * mean[3 * k + 1];
    o[ORC_TZ2] = w[10] * mean[3 * k + 2];
    {
      double tr = S2[0][0] + S2[1][1];
      double disc = sqrt(fmax(0.25 * (S2[0][0] - S2[1][1]) * (S2[0][0] - S2[1][1]) +
                              S2[0][1] * S2[0][1], 0.0));
      double lmax = 0.5 * tr + disc, lmin = det / lmax;
      o[ORC_KAPPA] = lmax / lmin;
      o[ORC_LMAX] = lmax;
    }
    /* the widened box reaches the level where alpha = alpha_min (1 - 2 e), e the
     * largest alpha error bound at the cut (with err_scale up to 1) */
    {
      double e = alpha_err_max(lev, o[ORC_KAPPA]);
      o[ORC_BOXW] = lev > 1e-12 ? sqrt((lev - log1p(-fmin(2.0 * e, 0.5))) / lev) * (1.0 + 1e-9)
                                : 1.0;
    }
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
  double kexp, amin, amax, tmin, err_scale;
} orc_opts;

/* A pixel centre lies in a Gaussian's footprint box widened by the factor
 * ORC_BOXW about its centre; the widening covers the pixels where alpha is
 * within alpha_err of alpha_min, whose decisions are checked for ambiguity. */
static int in_box(const double *r, double px, double py) {
  double wx = (r[ORC_MX] - r[ORC_XMIN]) * r[ORC_BOXW];
  double wy = (r[ORC_MY] - r[ORC_YMIN]) * r[ORC_BOXW];
  return px >= r[ORC_MX] - wx && px <= r[ORC_MX] + wx && py >= r[ORC_MY] - wy &&
         py <= r[ORC_MY] + wy;
}

/* exponent p and its relative alpha error at pixel centre (px, py) */
static double exponent_at(const double *r, double px, double py, const orc_opts *o,
                          double *err) {
  double dx = px - r[ORC_MX], dy = py - r[ORC_MY];
  double p = o->kexp * (r[ORC_CA] * dx * dx + 2.0 * r[ORC_CB] * dx * dy + r[ORC_CC] * dy * dy);
  *err = alpha_err_at(r, dx, dy, o->kexp, p, o->err_scale);
  return p;
}

/* Two Gaussians whose FP64 depths lie within the sum of their float32 depth
 * error bounds may be ordered either way by a float32 sort. The exception is a
 * pair whose depth terms w20 x, w21 y, w22 z are equal one by one (the same mean,
 * or means that differ only along axes the depth does not see): any evaluation
 * of the depth then gets the same inputs and the same value, so both sides keep
 * ascending index. */
static int depth_tie(const double *r, const double *s) {
  if (r[ORC_TZ0] == s[ORC_TZ0] && r[ORC_TZ1] == s[ORC_TZ1] && r[ORC_TZ2] == s[ORC_TZ2])
    return 0;
  return fabs(r[ORC_DEPTH] - s[ORC_DEPTH]) <= r[ORC_DERR] + s[ORC_DERR];
}

/* Composite one pixel centre (px, py) over the candidates `cand` (ascending FP64
 * depth, ties by ascending index; ghosts included, see oracle_project). With
 * check_box, candidates whose widened footprint box does not contain the pixel
 * centre are skipped first; this never changes the result because the exact box
 * already contains every point where alpha >= alpha_min.
 *   acc += c_k a T, T *= (1 - a), stop once T < T_min (Eq. gdgs2d).
 * Returns the ambiguity flag: set when one of the discontinuous decisions (near
 * cull, depth order of two contributing Gaussians, alpha vs alpha_min, T vs
 * T_min) is taken within its float32 error bound of the threshold. */
static int composite_pixel(double px, double py, const int64_t *cand, int64_t m,
                           int check_box, const double *proj, const float *grad,
                           int Q, const orc_opts *o, double *acc) {
  double T = 1.0, t_err = 0.0; /* transmittance and its relative float32 error bound */
  int amb = 0;
  const double *last = NULL; /* the last Gaussian that contributed */
  int64_t i = 0;
  for (int q = 0; q < Q; ++q) acc[q] = 0.0;
  for (; i < m; ++i) {
    int64_t g = cand[i];
    const double *r = proj + g * ORC_STRIDE;
    if (check_box && !in_box(r, px, py)) continue;
    double e;
    double p = exponent_at(r, px, py, o, &e);
    double a = r[ORC_OPA] * exp(-p);
    int clamped = a > o->amax * exp(e);
    /* alpha vs alpha_min: an exponent error of e moves alpha by a factor exp(+-e) */
    int near_cut = fabs(log(a / o->amin)) <= e;
    if (a > o->amax) a = o->amax;
    if (near_cut) amb = 1;
    if (a < o->amin) continue;
    if (o->err_scale > 0.0 && r[ORC_NEARAMB] != 0.0) amb = 1;
    if (r[ORC_GHOST] != 0.0) continue; /* culled: flags only */
    if (last && o->err_scale > 0.0 && depth_tie(last, r)) amb = 1;
    last = r;
    double wgt = a * T;
    for (int q = 0; q < Q; ++q) acc[q] += (double)grad[g * Q + q] * wgt;
    T *= (1.0 - a);
    t_err += (clamped ? 0.0 : fmin(e, 1.0) * a / (1.0 - a)) + 2.0 * o->err_scale * ORC_U;
    if (fabs(T - o->tmin) <= t_err * o->tmin) amb = 1;
    if (T < o->tmin) break;
  }
  /* After the stop: a contributing Gaussian within the depth bound of the last
   * one could have been composited before it. */
  if (i < m && last && o->err_scale > 0.0) {
    for (++i; i < m; ++i) {
      const double *r = proj + cand[i] * ORC_STRIDE;
      if (r[ORC_DEPTH] - last[ORC_DEPTH] > 4.0 * last[ORC_DERR] + r[ORC_DERR]) break;
      if (check_box && !in_box(r, px, py)) continue;
      double e;
      double p = exponent_at(r, px, py, o, &e);
      if (log(r[ORC_OPA] / o->amin) - p >= -e && depth_tie(last, r)) {
        amb = 1;
        break;
      }
    }
  }
  return amb;
}

/* opt: exp_coef, alpha_min, alpha_max, t_min, err_scale.
 * order: the valid Gaussians and the ghosts, sorted by (FP64 depth, index).
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
  orc_opts o = {opt[0], opt[1], opt[2], opt[3], opt[4]};
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
          double wy = (r[ORC_MY] - r[ORC_YMIN]) * r[ORC_BOXW];
          if (py >= r[ORC_MY] - wy && py <= r[ORC_MY] + wy) rowc[m++] = order[i];
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
