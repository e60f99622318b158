/*
 * dic_oracle.c -- plain, slow FP64 CPU oracle of the DIC hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg call this file.  The CUDA library never links,
 * includes or calls it, and it shares no code with the CUDA path.
 *
 * What it computes (Thoma & Ravi, "Significance of parallel computing on the
 * performance of Digital Image Correlation algorithms in MATLAB"):
 *
 *  - ZNCC of a (2M+1)^2 reference subset and a target subset, Eq. 1
 *    (Section 2 / 2.1), evaluated from exact 64-bit integer sums of 8-bit
 *    grey levels.  With N = (2M+1)^2:
 *        num = N*Sfg - Sf*Sg,  Df = N*Sff - Sf^2,  Dg = N*Sgg - Sg^2,
 *        C   = num / sqrt(Df*Dg)
 *    which is Eq. 1 with the means multiplied out.
 *  - Brute-force search (Section 2.1): every integer offset of the search
 *    window is evaluated and the largest C wins.  Candidates are compared
 *    exactly (sign of num, then num_a^2*Dg_b against num_b^2*Dg_a in 128-bit
 *    integers); ties keep the lowest linear index (dv+R)(2R+1)+(du+R).
 *  - Sub-pixel refinement (Section 2.2) by the inverse-compositional
 *    Gauss-Newton algorithm with a first-order (affine) warp, and by the
 *    forward-additive Newton-Raphson algorithm in its Gauss-Newton form
 *    (Table 2).  Grey levels between pixels come from bicubic interpolation
 *    (Section 2.2) with the Keys cubic-convolution kernel, a = -0.5, on the
 *    4x4 neighbourhood, evaluated straight from the pixels (no look-up table),
 *    or from the bilinear interpolation of Eq. 5.
 *  - The summed ZNSSD of every subset at given shape parameters and its
 *    gradient with respect to the deformed-image pixels and the parameters
 *    (hand-derived adjoint, FP64).
 *  - Sub-pixel refinement with a second-order (12-parameter) subset shape
 *    function, by both methods (an extension; readings at that section).
 *  - Integer search by particle swarm optimisation (Section 2.1, Eqs. 2-4)
 *    and by the modified swarm with one star-search step per generation
 *    (Sections 3, 5); the swarm's random numbers are inputs.  Readings are
 *    stated at that section below.
 *
 * The paper leaves the shape function, the update rules, the bicubic kernel,
 * the gradient operator, the convergence norm and the POI grid unstated; the
 * readings used here are the standard first-order IC-GN / FA-NR forms:
 *
 *   warp      W(xi; p) = (x0 + dx + u + ux*dx + uy*dy, y0 + dy + v + vx*dx + vy*dy),
 *             p = (u, ux, uy, v, vx, vy)
 *   IC-GN     SD_i = [fx, fx dx, fx dy, fy, fy dx, fy dy], H = sum SD_i^T SD_i,
 *             r_i = (f_i - fbar) - (df/dg)(g_i - gbar),
 *             dp = -H^-1 sum SD_i^T r_i,  W(p) <- W(p) W(dp)^-1
 *   FA-NR     J_i = grad g(W(xi_i;p)) dW/dp,
 *             dp = (sum J^T J)^-1 sum J_i^T [(dg/df)(f_i - fbar) - (g_i - gbar)],
 *             p <- p + dp
 *   stop      |dp|_c = sqrt(du^2 + dv^2 + M^2 (dux^2+duy^2+dvx^2+dvy^2)) < tol,
 *             or max_iter solves
 *   gradients of f: central differences at integer pixels (equal to the
 *             derivative of the Keys a=-0.5 interpolant at the nodes)
 *   POI grid  x0 = B + k*step, B = M + R + 2, while x0 <= W-1-B (same in y)
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC (no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum {
  ST_OK = 0,
  ST_ZERO_VAR_REF = 1,
  ST_OUT_OF_BOUNDS = 2,
  ST_MAX_ITER = 3,
  ST_NONFINITE = 4,
  ST_SINGULAR = 5,
  ST_ZERO_VAR_DEF = 6
};

/* ------------------------------------------------------------------ grid */
int dico_grid(int W, int H, int subset, int step, int R, int *nx, int *ny) {
  if (subset < 3 || (subset & 1) == 0 || step < 1 || R < 0 || W < 1 || H < 1)
    return -1;
  int M = subset / 2, B = M + R + 2;
  int ax = W - 1 - 2 * B, ay = H - 1 - 2 * B;
  *nx = ax >= 0 ? ax / step + 1 : 0;
  *ny = ay >= 0 ? ay / step + 1 : 0;
  return 0;
}

static void poi_centre(int64_t poi, int nx, int M, int R, int step, int *x0, int *y0) {
  int B = M + R + 2;
  *x0 = B + (int)(poi % nx) * step;
  *y0 = B + (int)(poi / nx) * step;
}

/* ------------------------------------------------------- integer search */
/* 1 if C_a > C_b strictly, where C = n / sqrt(Df * d) with the same Df > 0. */
static int zncc_greater(int64_t na, int64_t da, int64_t nb, int64_t db) {
  if (na >= 0 && nb < 0) return 1;
  if (na < 0 && nb >= 0) return 0;
  __int128 lhs = (__int128)na * (__int128)na * (__int128)db;
  __int128 rhs = (__int128)nb * (__int128)nb * (__int128)da;
  if (na >= 0) return lhs > rhs;
  return lhs < rhs; /* both negative: smaller |C| is the larger C */
}

static void search_one(const uint8_t *f, const uint8_t *g, int pitch, int x0, int y0,
                       int M, int R, int32_t *u0, int32_t *v0, double *zncc,
                       uint8_t *status) {
  const int64_t N = (int64_t)(2 * M + 1) * (2 * M + 1);
  int64_t Sf = 0, Sff = 0;
  for (int dy = -M; dy <= M; ++dy)
    for (int dx = -M; dx <= M; ++dx) {
      int64_t a = f[(int64_t)(y0 + dy) * pitch + (x0 + dx)];
      Sf += a;
      Sff += a * a;
    }
  const int64_t Df = N * Sff - Sf * Sf;
  if (Df == 0) {
    *u0 = 0; *v0 = 0; *zncc = 0.0; *status = ST_ZERO_VAR_REF;
    return;
  }
  int have = 0;
  int64_t bn = 0, bd = 1;
  int bu = -R, bv = -R;
  for (int dv = -R; dv <= R; ++dv)
    for (int du = -R; du <= R; ++du) {
      int64_t Sg = 0, Sgg = 0, Sfg = 0;
      for (int dy = -M; dy <= M; ++dy)
        for (int dx = -M; dx <= M; ++dx) {
          int64_t a = f[(int64_t)(y0 + dy) * pitch + (x0 + dx)];
          int64_t b = g[(int64_t)(y0 + dy + dv) * pitch + (x0 + dx + du)];
          Sg += b;
          Sgg += b * b;
          Sfg += a * b;
        }
      int64_t Dg = N * Sgg - Sg * Sg;
      if (Dg == 0) continue; /* undefined correlation: never preferred */
      int64_t num = N * Sfg - Sf * Sg;
      if (!have || zncc_greater(num, Dg, bn, bd)) {
        have = 1; bn = num; bd = Dg; bu = du; bv = dv;
      }
    }
  if (!have) {
    *u0 = -R; *v0 = -R; *zncc = 0.0; *status = ST_ZERO_VAR_DEF;
    return;
  }
  *u0 = bu; *v0 = bv;
  *zncc = (double)bn / sqrt((double)Df * (double)bd);
  *status = ST_OK;
}

int dico_integer_search(const uint8_t *f, const uint8_t *g, int W, int H, int pitch,
                        int subset, int step, int R, const int64_t *poi_idx,
                        int64_t n_idx, int nthreads, int32_t *u0, int32_t *v0,
                        double *zncc, uint8_t *status) {
  int nx, ny;
  if (dico_grid(W, H, subset, step, R, &nx, &ny)) return -1;
  const int M = subset / 2;
  const int64_t total = (int64_t)nx * ny;
  const int64_t n = poi_idx ? n_idx : total;
  if (nthreads <= 0) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
  for (int64_t k = 0; k < n; ++k) {
    int64_t poi = poi_idx ? poi_idx[k] : k;
    int x0, y0;
    poi_centre(poi, nx, M, R, step, &x0, &y0);
    search_one(f, g, pitch, x0, y0, M, R, &u0[k], &v0[k], &zncc[k], &status[k]);
  }
  return 0;
}

/* -------------------------------------------------- bicubic (Keys a=-0.5) */
/* Keys cubic-convolution kernel with a = -1/2 and its derivative. */
static double keys(double s) {
  double t = fabs(s);
  if (t <= 1.0) return 1.5 * t * t * t - 2.5 * t * t + 1.0;
  if (t < 2.0) return -0.5 * t * t * t + 2.5 * t * t - 4.0 * t + 2.0;
  return 0.0;
}
static double keys_d(double s) {
  double t = fabs(s), sg = s < 0 ? -1.0 : 1.0;
  if (t <= 1.0) return sg * (4.5 * t * t - 5.0 * t);
  if (t < 2.0) return sg * (-1.5 * t * t + 5.0 * t - 4.0);
  return 0.0;
}

/* Value (and optionally the x/y derivatives) of the bicubic interpolant at
 * (x, y); the caller guarantees 1 <= x < W-2 and 1 <= y < H-2. */
static double interp(const double *img, int pitch, double x, double y, double *gx,
                     double *gy) {
  double fx0 = floor(x), fy0 = floor(y);
  int ix = (int)fx0, iy = (int)fy0;
  double tx = x - fx0, ty = y - fy0;
  double wx[4], wy[4], dwx[4], dwy[4];
  for (int k = 0; k < 4; ++k) {
    wx[k] = keys(tx - (k - 1));
    wy[k] = keys(ty - (k - 1));
    dwx[k] = keys_d(tx - (k - 1));
    dwy[k] = keys_d(ty - (k - 1));
  }
  double v = 0, vx = 0, vy = 0;
  for (int l = 0; l < 4; ++l)
    for (int k = 0; k < 4; ++k) {
      double p = img[(int64_t)(iy + l - 1) * pitch + (ix + k - 1)];
      v += wy[l] * wx[k] * p;
      vx += wy[l] * dwx[k] * p;
      vy += dwy[l] * wx[k] * p;
    }
  if (gx) *gx = vx;
  if (gy) *gy = vy;
  return v;
}

double dico_bicubic(const double *img, int W, int H, int pitch, double x, double y,
                    double *gx, double *gy) {
  if (!(x >= 1.0 && x < W - 2.0 && y >= 1.0 && y < H - 2.0)) return NAN;
  return interp(img, pitch, x, y, gx, gy);
}

/* ------------------------------------------------------ bilinear (Eq. 5) */
/* G(x*, y*) = a00 + a10 x' + a01 y' + a11 x'y' (Eq. 5, Section 2.2), with
 * x', y' the offsets along x and y from the integer pixel (floor x*,
 * floor y*) and the four coefficients from the linear system that makes G
 * equal the grey levels of the four surrounding pixels, G(0,0) = g00,
 * G(1,0) = g10, G(0,1) = g01, G(1,1) = g11, solved by substitution.  The
 * gradient is that of the same patch. */
static double interp_bilinear(const double *img, int pitch, double x, double y, double *gx,
                              double *gy) {
  double fx0 = floor(x), fy0 = floor(y);
  int ix = (int)fx0, iy = (int)fy0;
  double xp = x - fx0, yp = y - fy0;
  const double *r = img + (int64_t)iy * pitch + ix;
  double g00 = r[0], g10 = r[1], g01 = r[pitch], g11 = r[pitch + 1];
  double a00 = g00;
  double a10 = g10 - a00;
  double a01 = g01 - a00;
  double a11 = g11 - a00 - a10 - a01;
  if (gx) *gx = a10 + a11 * yp;
  if (gy) *gy = a01 + a11 * xp;
  return a00 + a10 * xp + a01 * yp + a11 * xp * yp;
}

double dico_bilinear(const double *img, int W, int H, int pitch, double x, double y,
                     double *gx, double *gy) {
  if (!(x >= 0.0 && x < W - 1.0 && y >= 0.0 && y < H - 1.0)) return NAN;
  return interp_bilinear(img, pitch, x, y, gx, gy);
}

/* interpolation of g: 0 bicubic (Keys), 1 bilinear (Eq. 5) */
static double interp_g(int mode, const double *img, int pitch, double x, double y,
                       double *gx, double *gy) {
  return mode ? interp_bilinear(img, pitch, x, y, gx, gy) : interp(img, pitch, x, y, gx, gy);
}

/* ------------------------------------------------------------ 6x6 solve */
/* Cholesky factorisation of a symmetric 6x6 matrix in place (lower). */
static int chol6(double A[6][6]) {
  for (int j = 0; j < 6; ++j) {
    double d = A[j][j];
    for (int k = 0; k < j; ++k) d -= A[j][k] * A[j][k];
    if (!(d > 0.0) || !isfinite(d)) return -1;
    d = sqrt(d);
    A[j][j] = d;
    for (int i = j + 1; i < 6; ++i) {
      double s = A[i][j];
      for (int k = 0; k < j; ++k) s -= A[i][k] * A[j][k];
      A[i][j] = s / d;
    }
  }
  return 0;
}
static void chol6_solve(double L[6][6], const double b[6], double x[6]) {
  double y[6];
  for (int i = 0; i < 6; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
    y[i] = s / L[i][i];
  }
  for (int i = 5; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < 6; ++k) s -= L[k][i] * x[k];
    x[i] = s / L[i][i];
  }
}

/* ----------------------------------------------------------- warp helpers */
/* p = (u, ux, uy, v, vx, vy) */
static void warp_pt(const double p[6], int x0, int y0, int dx, int dy, double *x,
                    double *y) {
  *x = x0 + dx + p[0] + p[1] * dx + p[2] * dy;
  *y = y0 + dy + p[3] + p[4] * dx + p[5] * dy;
}

static int in_bounds(const double p[6], int x0, int y0, int M, int W, int H) {
  for (int cy = -1; cy <= 1; cy += 2)
    for (int cx = -1; cx <= 1; cx += 2) {
      double x, y;
      warp_pt(p, x0, y0, cx * M, cy * M, &x, &y);
      if (!(x >= 1.0 && x < W - 2.0 && y >= 1.0 && y < H - 2.0)) return 0;
    }
  return 1;
}

/* W(p) <- W(p) * W(dp)^-1 with W(q) = [[1+ux, uy, u], [vx, 1+vy, v], [0, 0, 1]]. */
static void compose_inverse(const double p[6], const double dp[6], double out[6]) {
  double a = 1 + dp[1], b = dp[2], c = dp[4], d = 1 + dp[5];
  double det = a * d - b * c;
  double ia = d / det, ib = -b / det, ic = -c / det, id = a / det;
  double itx = -(ia * dp[0] + ib * dp[3]);
  double ity = -(ic * dp[0] + id * dp[3]);
  double P00 = 1 + p[1], P01 = p[2], P02 = p[0];
  double P10 = p[4], P11 = 1 + p[5], P12 = p[3];
  double n00 = P00 * ia + P01 * ic, n01 = P00 * ib + P01 * id;
  double n02 = P00 * itx + P01 * ity + P02;
  double n10 = P10 * ia + P11 * ic, n11 = P10 * ib + P11 * id;
  double n12 = P10 * itx + P11 * ity + P12;
  out[0] = n02; out[1] = n00 - 1; out[2] = n01;
  out[3] = n12; out[4] = n10; out[5] = n11 - 1;
}

static double dp_norm(const double dp[6], int M) {
  double m2 = (double)M * M;
  return sqrt(dp[0] * dp[0] + dp[3] * dp[3] +
              m2 * (dp[1] * dp[1] + dp[2] * dp[2] + dp[4] * dp[4] + dp[5] * dp[5]));
}

/* g at every warped subset point; returns mean and sqrt(sum (g-gbar)^2).
 * Optional derivative outputs. */
static void sample_subset(const double *g, int pitch, const double p[6], int x0, int y0,
                          int M, int mode, double *gv, double *gxv, double *gyv,
                          double *gbar, double *dg) {
  int S = 2 * M + 1, N = S * S;
  double s = 0;
  for (int i = 0; i < N; ++i) {
    int dx = i % S - M, dy = i / S - M;
    double x, y;
    warp_pt(p, x0, y0, dx, dy, &x, &y);
    gv[i] = interp_g(mode, g, pitch, x, y, gxv ? &gxv[i] : NULL, gyv ? &gyv[i] : NULL);
    s += gv[i];
  }
  double m = s / N, q = 0;
  for (int i = 0; i < N; ++i) q += (gv[i] - m) * (gv[i] - m);
  *gbar = m;
  *dg = sqrt(q);
}

/* ------------------------------------------------------------- sub-pixel */
static void subpixel_one(const double *f, const double *g, int W, int H, int pitch,
                         int x0, int y0, int M, int method, int mode, double tol, int max_iter,
                         int32_t iu0, int32_t iv0, uint8_t st0, double *pout,
                         double *zncc, int32_t *iters, uint8_t *status, double *traj) {
  const int S = 2 * M + 1, N = S * S;
  double p[6] = {(double)iu0, 0, 0, (double)iv0, 0, 0};
  for (int k = 0; k < 6; ++k) pout[k] = p[k];
  *iters = 0;
  if (traj)
    for (int k = 0; k < (max_iter + 1) * 6; ++k) traj[k] = NAN;
  if (traj)
    for (int k = 0; k < 6; ++k) traj[k] = p[k];
  if (st0 != ST_OK) {
    *zncc = 0.0;
    *status = st0;
    return;
  }
  double *fc = malloc(sizeof(double) * N * 6);
  double *fx = fc + N, *fy = fx + N, *gv = fy + N, *gxv = gv + N, *gyv = gxv + N;
  double fs = 0;
  for (int i = 0; i < N; ++i) {
    int dx = i % S - M, dy = i / S - M;
    int64_t o = (int64_t)(y0 + dy) * pitch + (x0 + dx);
    fc[i] = f[o];
    fx[i] = 0.5 * (f[o + 1] - f[o - 1]);
    fy[i] = 0.5 * (f[o + pitch] - f[o - pitch]);
    fs += fc[i];
  }
  double fbar = fs / N, q = 0;
  for (int i = 0; i < N; ++i) {
    fc[i] -= fbar;
    q += fc[i] * fc[i];
  }
  const double df = sqrt(q);
  uint8_t st = ST_MAX_ITER;
  int it_done = 0;
  if (df == 0.0) {
    st = ST_ZERO_VAR_REF;
    goto final;
  }

  if (method == 0) {
    /* ---------------- IC-GN: Hessian from the reference subset, once ---- */
    double Hm[6][6] = {{0}};
    for (int i = 0; i < N; ++i) {
      int dx = i % S - M, dy = i / S - M;
      double sd[6] = {fx[i], fx[i] * dx, fx[i] * dy, fy[i], fy[i] * dx, fy[i] * dy};
      for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) Hm[a][b] += sd[a] * sd[b];
    }
    if (chol6(Hm)) {
      st = ST_SINGULAR;
      goto final;
    }
    for (int it = 1; it <= max_iter; ++it) {
      double gbar, dg;
      sample_subset(g, pitch, p, x0, y0, M, mode, gv, NULL, NULL, &gbar, &dg);
      if (!(dg > 0.0) || !isfinite(dg)) {
        st = ST_NONFINITE;
        break;
      }
      double b[6] = {0};
      for (int i = 0; i < N; ++i) {
        int dx = i % S - M, dy = i / S - M;
        double r = fc[i] - (df / dg) * (gv[i] - gbar);
        double sd[6] = {fx[i], fx[i] * dx, fx[i] * dy, fy[i], fy[i] * dx, fy[i] * dy};
        for (int a = 0; a < 6; ++a) b[a] += sd[a] * r;
      }
      double dp[6];
      chol6_solve(Hm, b, dp);
      for (int a = 0; a < 6; ++a) dp[a] = -dp[a];
      it_done = it;
      int fin = 1;
      for (int a = 0; a < 6; ++a) fin &= isfinite(dp[a]);
      if (!fin) {
        st = ST_NONFINITE;
        break;
      }
      double pn[6];
      compose_inverse(p, dp, pn);
      if (!in_bounds(pn, x0, y0, M, W, H)) {
        st = ST_OUT_OF_BOUNDS;
        break;
      }
      memcpy(p, pn, sizeof p);
      if (traj)
        for (int k = 0; k < 6; ++k) traj[it * 6 + k] = p[k];
      if (dp_norm(dp, M) < tol) {
        st = ST_OK;
        break;
      }
    }
  } else {
    /* ---------------- FA-NR (Gauss-Newton Hessian, rebuilt each step) --- */
    for (int it = 1; it <= max_iter; ++it) {
      double gbar, dg;
      sample_subset(g, pitch, p, x0, y0, M, mode, gv, gxv, gyv, &gbar, &dg);
      if (!(dg > 0.0) || !isfinite(dg)) {
        st = ST_NONFINITE;
        break;
      }
      double Hm[6][6] = {{0}}, b[6] = {0};
      for (int i = 0; i < N; ++i) {
        int dx = i % S - M, dy = i / S - M;
        double J[6] = {gxv[i], gxv[i] * dx, gxv[i] * dy, gyv[i], gyv[i] * dx,
                       gyv[i] * dy};
        double r = (dg / df) * fc[i] - (gv[i] - gbar);
        for (int a = 0; a < 6; ++a) {
          b[a] += J[a] * r;
          for (int c = 0; c < 6; ++c) Hm[a][c] += J[a] * J[c];
        }
      }
      it_done = it;
      if (chol6(Hm)) {
        st = ST_SINGULAR;
        break;
      }
      double dp[6];
      chol6_solve(Hm, b, dp);
      int fin = 1;
      for (int a = 0; a < 6; ++a) fin &= isfinite(dp[a]);
      if (!fin) {
        st = ST_NONFINITE;
        break;
      }
      double pn[6];
      for (int a = 0; a < 6; ++a) pn[a] = p[a] + dp[a];
      if (!in_bounds(pn, x0, y0, M, W, H)) {
        st = ST_OUT_OF_BOUNDS;
        break;
      }
      memcpy(p, pn, sizeof p);
      if (traj)
        for (int k = 0; k < 6; ++k) traj[it * 6 + k] = p[k];
      if (dp_norm(dp, M) < tol) {
        st = ST_OK;
        break;
      }
    }
  }

final:
  for (int k = 0; k < 6; ++k) pout[k] = p[k];
  *iters = it_done;
  *status = st;
  if (st == ST_ZERO_VAR_REF) {
    *zncc = 0.0;
  } else {
    /* Eq. 1 at the returned shape, interpolated target grey levels */
    double gbar, dg;
    sample_subset(g, pitch, p, x0, y0, M, mode, gv, NULL, NULL, &gbar, &dg);
    double s = 0;
    for (int i = 0; i < N; ++i) s += fc[i] * (gv[i] - gbar);
    *zncc = (dg > 0.0) ? s / (df * dg) : 0.0;
  }
  free(fc);
}

int dico_subpixel_interp(const double *f, const double *g, int W, int H, int pitch,
                         int subset, int step, int R, int method, int mode, double tol,
                         int max_iter, const int64_t *poi_idx, int64_t n_idx,
                         const int32_t *u0, const int32_t *v0, const uint8_t *st0,
                         int nthreads, double *p_out, double *zncc, int32_t *iters,
                         uint8_t *status, double *traj) {
  int nx, ny;
  if (dico_grid(W, H, subset, step, R, &nx, &ny)) return -1;
  if (method != 0 && method != 1) return -1;
  if (mode != 0 && mode != 1) return -1;
  if (max_iter < 1) return -1;
  const int M = subset / 2;
  const int64_t n = poi_idx ? n_idx : (int64_t)nx * ny;
  if (nthreads <= 0) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
  for (int64_t k = 0; k < n; ++k) {
    int64_t poi = poi_idx ? poi_idx[k] : k;
    int x0, y0;
    poi_centre(poi, nx, M, R, step, &x0, &y0);
    subpixel_one(f, g, W, H, pitch, x0, y0, M, method, mode, tol, max_iter, u0[k], v0[k],
                 st0[k], &p_out[k * 6], &zncc[k], &iters[k], &status[k],
                 traj ? &traj[k * (int64_t)(max_iter + 1) * 6] : NULL);
  }
  return 0;
}

/* ------------------------------------------------ second-order shape */
/* Second-order subset shape function, p = (u, ux, uy, uxx, uxy, uyy,
 * v, vx, vy, vxx, vxy, vyy):
 *   x = x0 + dx + u + ux dx + uy dy + uxx dx^2/2 + uxy dx dy + uyy dy^2/2
 * (and y with the v terms), i.e. p . (1, dx, dy, dx^2/2, dx dy, dy^2/2) per
 * direction.  The paper uses first-order shapes only; this extension keeps
 * the first-order readings and adds:
 *   - IC-GN: SD_i = [fx e_i, fy e_i] with e = (1, dx, dy, dx^2/2, dx dy,
 *     dy^2/2), H = sum SD^T SD (12x12, Cholesky), dp = -H^-1 sum SD^T r;
 *     W(p) <- W(p) W(dp)^-1 in the 6x6 representation of a quadratic warp
 *     acting on w = (xi^2, xi eta, eta^2, xi, eta, 1), whose rows are the
 *     warped (xi'^2, xi' eta', eta'^2, xi', eta', 1) with terms above second
 *     order dropped; the new p is read from rows 4 and 5 of the product;
 *   - FA-NR: J = [gx e, gy e], dp = (J^T J)^-1 J^T r, p <- p + dp;
 *   - stop: |dp|^2 = du^2 + dv^2 + M^2 (first derivatives^2) + (M^2/2)^2
 *     (dxx^2 + dyy^2 terms) + M^4 (dxy^2 terms): each term weighted by the
 *     largest change of the displacement it causes over the subset;
 *   - bounds: every warped subset point must stay inside [1, W-2) x
 *     [1, H-2) (a quadratic warp need not reach its extremes at corners). */
static void basis2(int dx, int dy, double e[6]) {
  e[0] = 1.0; e[1] = dx; e[2] = dy;
  e[3] = 0.5 * dx * dx; e[4] = (double)dx * dy; e[5] = 0.5 * dy * dy;
}

static void warp2_pt(const double p[12], int x0, int y0, int dx, int dy, double *x, double *y) {
  double e[6];
  basis2(dx, dy, e);
  double lx = 0, ly = 0;
  for (int k = 0; k < 6; ++k) {
    lx += p[k] * e[k];
    ly += p[6 + k] * e[k];
  }
  *x = x0 + dx + lx;
  *y = y0 + dy + ly;
}

static int in_bounds2(const double p[12], int x0, int y0, int M, int W, int H) {
  for (int dy = -M; dy <= M; ++dy)
    for (int dx = -M; dx <= M; ++dx) {
      double x, y;
      warp2_pt(p, x0, y0, dx, dy, &x, &y);
      if (!(x >= 1.0 && x < W - 2.0 && y >= 1.0 && y < H - 2.0)) return 0;
    }
  return 1;
}

/* 6x6 representation of the quadratic warp p (rows: xi'^2, xi' eta',
 * eta'^2, xi', eta', 1 over the columns xi^2, xi eta, eta^2, xi, eta, 1). */
void dico_warp2_matrix(const double p[12], double Mx[36]) {
  const double A1 = 0.5 * p[3], A2 = p[4], A3 = 0.5 * p[5], A4 = 1.0 + p[1], A5 = p[2],
               A6 = p[0];
  const double B1 = 0.5 * p[9], B2 = p[10], B3 = 0.5 * p[11], B4 = p[7], B5 = 1.0 + p[8],
               B6 = p[6];
  const double r[36] = {
      A4 * A4 + 2 * A1 * A6, 2 * A4 * A5 + 2 * A2 * A6, A5 * A5 + 2 * A3 * A6, 2 * A4 * A6,
      2 * A5 * A6, A6 * A6,
      A4 * B4 + A1 * B6 + A6 * B1, A4 * B5 + A5 * B4 + A2 * B6 + A6 * B2,
      A5 * B5 + A3 * B6 + A6 * B3, A4 * B6 + A6 * B4, A5 * B6 + A6 * B5, A6 * B6,
      B4 * B4 + 2 * B1 * B6, 2 * B4 * B5 + 2 * B2 * B6, B5 * B5 + 2 * B3 * B6, 2 * B4 * B6,
      2 * B5 * B6, B6 * B6,
      A1, A2, A3, A4, A5, A6,
      B1, B2, B3, B4, B5, B6,
      0, 0, 0, 0, 0, 1};
  memcpy(Mx, r, sizeof r);
}

/* Inverse of a 6x6 matrix by Gauss-Jordan elimination with partial
 * pivoting; -1 if singular. */
static int inv6(const double A[36], double X[36]) {
  double a[6][12];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 12; ++j) a[i][j] = j < 6 ? A[i * 6 + j] : (j - 6 == i ? 1.0 : 0.0);
  for (int c = 0; c < 6; ++c) {
    int piv = c;
    for (int i = c + 1; i < 6; ++i)
      if (fabs(a[i][c]) > fabs(a[piv][c])) piv = i;
    if (!(fabs(a[piv][c]) > 0.0)) return -1;
    if (piv != c)
      for (int j = 0; j < 12; ++j) {
        double t = a[c][j]; a[c][j] = a[piv][j]; a[piv][j] = t;
      }
    double d = a[c][c];
    for (int j = 0; j < 12; ++j) a[c][j] /= d;
    for (int i = 0; i < 6; ++i)
      if (i != c) {
        double m = a[i][c];
        for (int j = 0; j < 12; ++j) a[i][j] -= m * a[c][j];
      }
  }
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) X[i * 6 + j] = a[i][6 + j];
  return 0;
}

/* W(p) <- W(p) W(dp)^-1 for quadratic warps (see above); -1 if W(dp)'s
 * matrix is singular. */
int dico_compose2(const double p[12], const double dp[12], double out[12]) {
  double Mp[36], Md[36], Mi[36], P[36];
  dico_warp2_matrix(p, Mp);
  dico_warp2_matrix(dp, Md);
  if (inv6(Md, Mi)) return -1;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double s = 0;
      for (int k = 0; k < 6; ++k) s += Mp[i * 6 + k] * Mi[k * 6 + j];
      P[i * 6 + j] = s;
    }
  out[3] = 2.0 * P[18]; out[4] = P[19]; out[5] = 2.0 * P[20];
  out[1] = P[21] - 1.0; out[2] = P[22]; out[0] = P[23];
  out[9] = 2.0 * P[24]; out[10] = P[25]; out[11] = 2.0 * P[26];
  out[7] = P[27]; out[8] = P[28] - 1.0; out[6] = P[29];
  return 0;
}

static double dp_norm2(const double dp[12], int M) {
  const double m2 = (double)M * M, q2 = 0.25 * m2 * m2, m4 = m2 * m2;
  return sqrt(dp[0] * dp[0] + dp[6] * dp[6] +
              m2 * (dp[1] * dp[1] + dp[2] * dp[2] + dp[7] * dp[7] + dp[8] * dp[8]) +
              q2 * (dp[3] * dp[3] + dp[5] * dp[5] + dp[9] * dp[9] + dp[11] * dp[11]) +
              m4 * (dp[4] * dp[4] + dp[10] * dp[10]));
}

/* Cholesky of a symmetric n x n matrix in place (lower), n <= 12. */
static int choln(double *A, int n) {
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
    if (!(d > 0.0) || !isfinite(d)) return -1;
    d = sqrt(d);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = A[i * n + j];
      for (int k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = s / d;
    }
  }
  return 0;
}
static void choln_solve(const double *L, int n, const double *b, double *x) {
  double y[12];
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
    y[i] = s / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
    x[i] = s / L[i * n + i];
  }
}

/* g at every warped point of a quadratic shape (bicubic), mean and spread. */
static void sample_subset2(const double *g, int pitch, const double p[12], int x0, int y0,
                           int M, double *gv, double *gxv, double *gyv, double *gbar,
                           double *dg) {
  int S = 2 * M + 1, N = S * S;
  double s = 0;
  for (int i = 0; i < N; ++i) {
    int dx = i % S - M, dy = i / S - M;
    double x, y;
    warp2_pt(p, x0, y0, dx, dy, &x, &y);
    gv[i] = interp(g, pitch, x, y, gxv ? &gxv[i] : NULL, gyv ? &gyv[i] : NULL);
    s += gv[i];
  }
  double m = s / N, q = 0;
  for (int i = 0; i < N; ++i) q += (gv[i] - m) * (gv[i] - m);
  *gbar = m;
  *dg = sqrt(q);
}

static void subpixel2_one(const double *f, const double *g, int W, int H, int pitch, int x0,
                          int y0, int M, int method, double tol, int max_iter, int32_t iu0,
                          int32_t iv0, uint8_t st0, double *pout, double *zncc,
                          int32_t *iters, uint8_t *status, double *traj) {
  const int S = 2 * M + 1, N = S * S;
  double p[12] = {0};
  p[0] = iu0;
  p[6] = iv0;
  memcpy(pout, p, sizeof p);
  *iters = 0;
  if (traj) {
    for (int k = 0; k < (max_iter + 1) * 12; ++k) traj[k] = NAN;
    memcpy(traj, p, sizeof p);
  }
  if (st0 != ST_OK) {
    *zncc = 0.0;
    *status = st0;
    return;
  }
  double *fc = malloc(sizeof(double) * N * 6);
  double *fx = fc + N, *fy = fx + N, *gv = fy + N, *gxv = gv + N, *gyv = gxv + N;
  double fs = 0;
  for (int i = 0; i < N; ++i) {
    int dx = i % S - M, dy = i / S - M;
    int64_t o = (int64_t)(y0 + dy) * pitch + (x0 + dx);
    fc[i] = f[o];
    fx[i] = 0.5 * (f[o + 1] - f[o - 1]);
    fy[i] = 0.5 * (f[o + pitch] - f[o - pitch]);
    fs += fc[i];
  }
  double fbar = fs / N, q = 0;
  for (int i = 0; i < N; ++i) {
    fc[i] -= fbar;
    q += fc[i] * fc[i];
  }
  const double df = sqrt(q);
  uint8_t st = ST_MAX_ITER;
  int it_done = 0;
  double Hm[144];
  if (df == 0.0) {
    st = ST_ZERO_VAR_REF;
    goto final2;
  }
  if (method == 0) {
    memset(Hm, 0, sizeof Hm);
    for (int i = 0; i < N; ++i) {
      double e[6], sd[12];
      basis2(i % S - M, i / S - M, e);
      for (int k = 0; k < 6; ++k) { sd[k] = fx[i] * e[k]; sd[6 + k] = fy[i] * e[k]; }
      for (int a = 0; a < 12; ++a)
        for (int b = 0; b < 12; ++b) Hm[a * 12 + b] += sd[a] * sd[b];
    }
    if (choln(Hm, 12)) {
      st = ST_SINGULAR;
      goto final2;
    }
  }
  for (int it = 1; it <= max_iter; ++it) {
    double gbar, dg;
    sample_subset2(g, pitch, p, x0, y0, M, gv, method ? gxv : NULL, method ? gyv : NULL, &gbar,
                   &dg);
    if (!(dg > 0.0) || !isfinite(dg)) {
      st = ST_NONFINITE;
      break;
    }
    double b[12] = {0}, dp[12];
    if (method == 0) {
      for (int i = 0; i < N; ++i) {
        double e[6];
        basis2(i % S - M, i / S - M, e);
        double r = fc[i] - (df / dg) * (gv[i] - gbar);
        for (int k = 0; k < 6; ++k) {
          b[k] += fx[i] * e[k] * r;
          b[6 + k] += fy[i] * e[k] * r;
        }
      }
      choln_solve(Hm, 12, b, dp);
      for (int a = 0; a < 12; ++a) dp[a] = -dp[a];
    } else {
      memset(Hm, 0, sizeof Hm);
      for (int i = 0; i < N; ++i) {
        double e[6], J[12];
        basis2(i % S - M, i / S - M, e);
        for (int k = 0; k < 6; ++k) { J[k] = gxv[i] * e[k]; J[6 + k] = gyv[i] * e[k]; }
        double r = (dg / df) * fc[i] - (gv[i] - gbar);
        for (int a = 0; a < 12; ++a) {
          b[a] += J[a] * r;
          for (int c = 0; c < 12; ++c) Hm[a * 12 + c] += J[a] * J[c];
        }
      }
      it_done = it;
      if (choln(Hm, 12)) {
        st = ST_SINGULAR;
        break;
      }
      choln_solve(Hm, 12, b, dp);
    }
    it_done = it;
    int fin = 1;
    for (int a = 0; a < 12; ++a) fin &= isfinite(dp[a]);
    if (!fin) {
      st = ST_NONFINITE;
      break;
    }
    double pn[12];
    if (method == 0) {
      if (dico_compose2(p, dp, pn)) {
        st = ST_NONFINITE;
        break;
      }
    } else {
      for (int a = 0; a < 12; ++a) pn[a] = p[a] + dp[a];
    }
    if (!in_bounds2(pn, x0, y0, M, W, H)) {
      st = ST_OUT_OF_BOUNDS;
      break;
    }
    memcpy(p, pn, sizeof p);
    if (traj) memcpy(traj + it * 12, p, sizeof p);
    if (dp_norm2(dp, M) < tol) {
      st = ST_OK;
      break;
    }
  }
final2:
  memcpy(pout, p, sizeof p);
  *iters = it_done;
  *status = st;
  if (st == ST_ZERO_VAR_REF) {
    *zncc = 0.0;
  } else {
    double gbar, dg;
    sample_subset2(g, pitch, p, x0, y0, M, gv, NULL, NULL, &gbar, &dg);
    double s2 = 0;
    for (int i = 0; i < N; ++i) s2 += fc[i] * (gv[i] - gbar);
    *zncc = (dg > 0.0) ? s2 / (df * dg) : 0.0;
  }
  free(fc);
}

/* Eq. 1 at given second-order shapes p[k][12] (bicubic); NAN where a warped
 * point leaves [1, W-2) x [1, H-2) or a subset is flat. */
int dico_zncc_at2(const double *f, const double *g, int W, int H, int pitch, int subset,
                  int step, int R, const int64_t *poi_idx, int64_t n_idx, const double *p,
                  int nthreads, double *zncc) {
  int nx, ny;
  if (dico_grid(W, H, subset, step, R, &nx, &ny)) return -1;
  const int M = subset / 2, S = subset, N = S * S;
  const int64_t n = poi_idx ? n_idx : (int64_t)nx * ny;
  if (nthreads <= 0) nthreads = 1;
#pragma omp parallel num_threads(nthreads)
  {
    double *fc = malloc(sizeof(double) * N * 2);
    double *gv = fc + N;
#pragma omp for schedule(dynamic, 16)
    for (int64_t k = 0; k < n; ++k) {
      int64_t poi = poi_idx ? poi_idx[k] : k;
      int x0, y0;
      poi_centre(poi, nx, M, R, step, &x0, &y0);
      const double *pk = &p[k * 12];
      zncc[k] = NAN;
      if (!in_bounds2(pk, x0, y0, M, W, H)) continue;
      double fs = 0;
      for (int i = 0; i < N; ++i) {
        int dx = i % S - M, dy = i / S - M;
        fc[i] = f[(int64_t)(y0 + dy) * pitch + (x0 + dx)];
        fs += fc[i];
      }
      double fbar = fs / N, q = 0;
      for (int i = 0; i < N; ++i) {
        fc[i] -= fbar;
        q += fc[i] * fc[i];
      }
      double df = sqrt(q), gbar, dg;
      sample_subset2(g, pitch, pk, x0, y0, M, gv, NULL, NULL, &gbar, &dg);
      if (!(df > 0.0) || !(dg > 0.0)) continue;
      double c = 0;
      for (int i = 0; i < N; ++i) c += fc[i] * (gv[i] - gbar);
      zncc[k] = c / (df * dg);
    }
    free(fc);
  }
  return 0;
}

int dico_subpixel2(const double *f, const double *g, int W, int H, int pitch, int subset,
                   int step, int R, int method, double tol, int max_iter,
                   const int64_t *poi_idx, int64_t n_idx, const int32_t *u0, const int32_t *v0,
                   const uint8_t *st0, int nthreads, double *p_out, double *zncc,
                   int32_t *iters, uint8_t *status, double *traj) {
  int nx, ny;
  if (dico_grid(W, H, subset, step, R, &nx, &ny)) return -1;
  if (method != 0 && method != 1) return -1;
  if (max_iter < 1) return -1;
  const int M = subset / 2;
  const int64_t n = poi_idx ? n_idx : (int64_t)nx * ny;
  if (nthreads <= 0) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
  for (int64_t k = 0; k < n; ++k) {
    int64_t poi = poi_idx ? poi_idx[k] : k;
    int x0, y0;
    poi_centre(poi, nx, M, R, step, &x0, &y0);
    subpixel2_one(f, g, W, H, pitch, x0, y0, M, method, tol, max_iter, u0[k], v0[k], st0[k],
                  &p_out[k * 12], &zncc[k], &iters[k], &status[k],
                  traj ? &traj[k * (int64_t)(max_iter + 1) * 12] : NULL);
  }
  return 0;
}

/* Eq. 1 at given shapes: for POI k, the ZNCC of the reference subset and the
 * target grey levels interpolated (mode 0 bicubic, 1 bilinear) at the warped
 * subset points W(xi; p_k), C = sum (f_i - fbar)(g_i - gbar) / (df dg).
 * A POI whose warped subset leaves [1, W-2) x [1, H-2), or whose reference
 * or target subset is flat, gets NAN. */
int dico_zncc_at(const double *f, const double *g, int W, int H, int pitch, int subset,
                 int step, int R, int mode, const int64_t *poi_idx, int64_t n_idx,
                 const double *p, int nthreads, double *zncc) {
  int nx, ny;
  if (dico_grid(W, H, subset, step, R, &nx, &ny)) return -1;
  if (mode != 0 && mode != 1) return -1;
  const int M = subset / 2, S = subset, N = S * S;
  const int64_t n = poi_idx ? n_idx : (int64_t)nx * ny;
  if (nthreads <= 0) nthreads = 1;
#pragma omp parallel num_threads(nthreads)
  {
    double *fc = malloc(sizeof(double) * N * 2);
    double *gv = fc + N;
#pragma omp for schedule(dynamic, 16)
    for (int64_t k = 0; k < n; ++k) {
      int64_t poi = poi_idx ? poi_idx[k] : k;
      int x0, y0;
      poi_centre(poi, nx, M, R, step, &x0, &y0);
      const double *pk = &p[k * 6];
      zncc[k] = NAN;
      if (!in_bounds(pk, x0, y0, M, W, H)) continue;
      double fs = 0;
      for (int i = 0; i < N; ++i) {
        int dx = i % S - M, dy = i / S - M;
        fc[i] = f[(int64_t)(y0 + dy) * pitch + (x0 + dx)];
        fs += fc[i];
      }
      double fbar = fs / N, q = 0;
      for (int i = 0; i < N; ++i) {
        fc[i] -= fbar;
        q += fc[i] * fc[i];
      }
      double df = sqrt(q), gbar, dg;
      sample_subset(g, pitch, pk, x0, y0, M, mode, gv, NULL, NULL, &gbar, &dg);
      if (!(df > 0.0) || !(dg > 0.0)) continue;
      double c = 0;
      for (int i = 0; i < N; ++i) c += fc[i] * (gv[i] - gbar);
      zncc[k] = c / (df * dg);
    }
    free(fc);
  }
  return 0;
}

int dico_subpixel(const double *f, const double *g, int W, int H, int pitch, int subset,
                  int step, int R, int method, double tol, int max_iter,
                  const int64_t *poi_idx, int64_t n_idx, const int32_t *u0,
                  const int32_t *v0, const uint8_t *st0, int nthreads, double *p_out,
                  double *zncc, int32_t *iters, uint8_t *status, double *traj) {
  return dico_subpixel_interp(f, g, W, H, pitch, subset, step, R, method, 0, tol, max_iter,
                              poi_idx, n_idx, u0, v0, st0, nthreads, p_out, zncc, iters,
                              status, traj);
}

/* ------------------------------------------------------- ZNSSD + adjoint */
/* L = sum over POIs k and subset points i of
 *       [ (f_i - fbar)/df - (g(W(xi_i; p_k)) - gbar)/dg ]^2
 * and, if requested, dL/dg (H x pitch, accumulated) and dL/dp (n x 6).
 * With ft_i = (f_i-fbar)/df, gt_i = (g_i-gbar)/dg and C = sum ft_i gt_i:
 *   dL/dg_i = (2/dg) (C gt_i - ft_i),  dL/dp = sum_i dL/dg_i * grad g_i dW/dp,
 * and dL/dg_i is spread onto the 4x4 pixels with the bicubic weights. */
int dico_znssd(const double *f, const double *g, int W, int H, int pitch, int subset,
               int step, int R, const int64_t *poi_idx, int64_t n_idx,
               const double *p, double *loss, double *loss_poi, double *dL_dg,
               double *dL_dp) {
  int nx, ny;
  if (dico_grid(W, H, subset, step, R, &nx, &ny)) return -1;
  const int M = subset / 2, S = subset, N = S * S;
  const int64_t n = poi_idx ? n_idx : (int64_t)nx * ny;
  double *buf = malloc(sizeof(double) * N * 4);
  double *fc = buf, *gv = buf + N, *gxv = gv + N, *gyv = gxv + N;
  double total = 0;
  for (int64_t k = 0; k < n; ++k) {
    int64_t poi = poi_idx ? poi_idx[k] : k;
    int x0, y0;
    poi_centre(poi, nx, M, R, step, &x0, &y0);
    const double *pk = &p[k * 6];
    if (dL_dp)
      for (int a = 0; a < 6; ++a) dL_dp[k * 6 + a] = 0.0;
    if (loss_poi) loss_poi[k] = 0.0;
    if (!in_bounds(pk, x0, y0, M, W, H)) continue;
    double fs = 0;
    for (int i = 0; i < N; ++i) {
      int dx = i % S - M, dy = i / S - M;
      fc[i] = f[(int64_t)(y0 + dy) * pitch + (x0 + dx)];
      fs += fc[i];
    }
    double fbar = fs / N, q = 0;
    for (int i = 0; i < N; ++i) {
      fc[i] -= fbar;
      q += fc[i] * fc[i];
    }
    double df = sqrt(q), gbar, dg;
    sample_subset(g, pitch, pk, x0, y0, M, 0, gv, gxv, gyv, &gbar, &dg);
    if (!(df > 0) || !(dg > 0)) continue;
    double C = 0, Lk = 0;
    for (int i = 0; i < N; ++i) {
      double e = fc[i] / df - (gv[i] - gbar) / dg;
      Lk += e * e;
      C += (fc[i] / df) * ((gv[i] - gbar) / dg);
    }
    total += Lk;
    if (loss_poi) loss_poi[k] = Lk;
    if (!dL_dg && !dL_dp) continue;
    for (int i = 0; i < N; ++i) {
      int dx = i % S - M, dy = i / S - M;
      double gi = (2.0 / dg) * (C * (gv[i] - gbar) / dg - fc[i] / df);
      if (dL_dp) {
        double J[6] = {gxv[i], gxv[i] * dx, gxv[i] * dy, gyv[i], gyv[i] * dx,
                       gyv[i] * dy};
        for (int a = 0; a < 6; ++a) dL_dp[k * 6 + a] += gi * J[a];
      }
      if (dL_dg) {
        double x, y;
        warp_pt(pk, x0, y0, dx, dy, &x, &y);
        double fx0 = floor(x), fy0 = floor(y);
        int ix = (int)fx0, iy = (int)fy0;
        double tx = x - fx0, ty = y - fy0;
        for (int l = 0; l < 4; ++l)
          for (int c = 0; c < 4; ++c)
            dL_dg[(int64_t)(iy + l - 1) * pitch + (ix + c - 1)] +=
                gi * keys(ty - (l - 1)) * keys(tx - (c - 1));
      }
    }
  }
  free(buf);
  *loss = total;
  return 0;
}

/* ------------------------------------------- particle swarm integer search */
/* Integer search by particle swarm optimisation (Section 2.1, Eqs. 2-4) and
 * by the modified swarm whose particles also look at the four pixels around
 * them, the star search folded into the swarm (Sections 3 and 5).
 *
 * Per POI, with the swarm's random numbers passed in as
 * rand[k][t][i][0..3] (uniforms in [0,1); k the POI, t the generation, i the
 * particle):
 *   t = 0   p_i = R (2 u_0 - 1, 2 u_1 - 1),  v_i = vinit (2 u_2 - 1, 2 u_3 - 1)
 *   t >= 1  Eq. 2 with w = w(t-1) of Eq. 4, r1 = (u_0, u_1), r2 = (u_2, u_3)
 *           per direction, evaluated as ((w v) + (c1 r1)(pbest - p)) +
 *           (c2 r2)(gbest - p); then Eq. 3, p clamped to [-R, R] per
 *           direction (the velocity is kept).
 *   every generation, each particle evaluates Eq. 1 at its nearest pixel
 *   q = floor(p + 1/2); the modified swarm also evaluates q +- (1,0) and
 *   q +- (0,1) inside the window, keeps the best of the five (ties: centre,
 *   +x, -x, +y, -y) and moves onto it.  pbest takes the evaluated pixel if it
 *   is strictly better (at t = 0 unconditionally); after all particles,
 *   gbest takes the first strictly better pbest in particle order.
 *   The swarm stops after `gmax` generations, or after the first generation
 *   whose gbest reaches C >= stop_num / stop_den (tested exactly).
 * Each pixel is evaluated at most once per POI (a look-up table, as the
 * paper's implementation keeps); `evals` counts the distinct pixels.
 * Candidates compare exactly as in the brute-force search; a pixel whose
 * target subset is flat has no correlation and ranks below every other. */
typedef struct {
  int64_t num, den; /* C = num / sqrt(Df * den) */
  int def;          /* den != 0 */
} zc_t;

static int zc_greater(zc_t a, zc_t b) {
  if (!a.def) return 0;
  if (!b.def) return 1;
  return zncc_greater(a.num, a.den, b.num, b.den);
}

/* C >= sn / sd, exactly (0 <= sn, 1 <= sd <= 2^20). */
static int zc_at_least(zc_t a, int64_t Df, int64_t sn, int64_t sd) {
  if (!a.def || a.num < 0) return 0;
  __int128 lhs = (__int128)a.num * (__int128)a.num * ((__int128)sd * (__int128)sd);
  __int128 rhs = ((__int128)sn * (__int128)sn) * ((__int128)Df * (__int128)a.den);
  return lhs >= rhs;
}

typedef struct {
  const uint8_t *f, *g;
  int pitch, x0, y0, M, R;
  int64_t N, Sf;
  uint8_t *seen;
  zc_t *memo;
  int evals;
} pso_ctx;

static zc_t pso_eval(pso_ctx *c, int du, int dv) {
  int64_t slot = (int64_t)(dv + c->R) * (2 * c->R + 1) + (du + c->R);
  if (c->seen[slot]) return c->memo[slot];
  int64_t Sg = 0, Sgg = 0, Sfg = 0;
  for (int dy = -c->M; dy <= c->M; ++dy)
    for (int dx = -c->M; dx <= c->M; ++dx) {
      int64_t a = c->f[(int64_t)(c->y0 + dy) * c->pitch + (c->x0 + dx)];
      int64_t b = c->g[(int64_t)(c->y0 + dy + dv) * c->pitch + (c->x0 + dx + du)];
      Sg += b;
      Sgg += b * b;
      Sfg += a * b;
    }
  zc_t z;
  z.den = c->N * Sgg - Sg * Sg;
  z.num = c->N * Sfg - c->Sf * Sg;
  z.def = z.den != 0;
  c->seen[slot] = 1;
  c->memo[slot] = z;
  c->evals++;
  return z;
}

static void pso_one(pso_ctx *c, int modified, int P, int gmax, double c1, double c2,
                    double vinit, int64_t sn, int64_t sd, const double *rand,
                    double *trace, double (*p)[2], double (*v)[2], int (*pb)[2],
                    zc_t *pbc, int32_t *u0, int32_t *v0, double *zncc, uint8_t *status,
                    int32_t *gens) {
  const int M = c->M, R = c->R;
  int64_t Sff = 0;
  c->Sf = 0;
  for (int dy = -M; dy <= M; ++dy)
    for (int dx = -M; dx <= M; ++dx) {
      int64_t a = c->f[(int64_t)(c->y0 + dy) * c->pitch + (c->x0 + dx)];
      c->Sf += a;
      Sff += a * a;
    }
  const int64_t Df = c->N * Sff - c->Sf * c->Sf;
  *gens = 0;
  if (Df == 0) {
    *u0 = 0; *v0 = 0; *zncc = 0.0; *status = ST_ZERO_VAR_REF;
    return;
  }
  static const int star[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
  int gb[2] = {0, 0};
  zc_t gc = {0, 0, 0};
  for (int t = 0; t < gmax; ++t) {
    const double *rt = rand + (int64_t)t * P * 4;
    if (t == 0) {
      for (int i = 0; i < P; ++i)
        for (int d = 0; d < 2; ++d) {
          p[i][d] = (double)R * (2.0 * rt[i * 4 + d] - 1.0);
          v[i][d] = vinit * (2.0 * rt[i * 4 + 2 + d] - 1.0);
        }
    } else {
      const double w = 0.9 - (double)(t - 1) / (2.0 * (double)gmax); /* Eq. 4 */
      for (int i = 0; i < P; ++i)
        for (int d = 0; d < 2; ++d) {
          double r1 = rt[i * 4 + d], r2 = rt[i * 4 + 2 + d];
          double inert = w * v[i][d];
          double cogn = (c1 * r1) * ((double)pb[i][d] - p[i][d]);
          double soc = (c2 * r2) * ((double)gb[d] - p[i][d]);
          v[i][d] = (inert + cogn) + soc; /* Eq. 2 */
          double np = p[i][d] + v[i][d];  /* Eq. 3 */
          p[i][d] = np < -R ? (double)-R : (np > R ? (double)R : np);
        }
    }
    for (int i = 0; i < P; ++i) {
      double *tr = trace ? trace + ((int64_t)t * P + i) * 8 : NULL;
      if (tr) { tr[0] = p[i][0]; tr[1] = p[i][1]; tr[2] = v[i][0]; tr[3] = v[i][1]; }
      int q[2] = {(int)floor(p[i][0] + 0.5), (int)floor(p[i][1] + 0.5)};
      int best[2] = {q[0], q[1]};
      zc_t bc = pso_eval(c, q[0], q[1]);
      if (modified) {
        for (int s = 0; s < 4; ++s) {
          int nx = q[0] + star[s][0], ny = q[1] + star[s][1];
          if (nx < -R || nx > R || ny < -R || ny > R) continue;
          zc_t z = pso_eval(c, nx, ny);
          if (zc_greater(z, bc)) { best[0] = nx; best[1] = ny; bc = z; }
        }
        p[i][0] = best[0];
        p[i][1] = best[1];
      }
      if (t == 0 || zc_greater(bc, pbc[i])) {
        pb[i][0] = best[0]; pb[i][1] = best[1]; pbc[i] = bc;
      }
      if (tr) { tr[4] = q[0]; tr[5] = q[1]; tr[6] = pb[i][0]; tr[7] = pb[i][1]; }
    }
    for (int i = 0; i < P; ++i)
      if ((t == 0 && i == 0) || zc_greater(pbc[i], gc)) {
        gb[0] = pb[i][0]; gb[1] = pb[i][1]; gc = pbc[i];
      }
    *gens = t + 1;
    if (zc_at_least(gc, Df, sn, sd)) break;
  }
  *u0 = gb[0]; *v0 = gb[1];
  if (!gc.def) {
    *zncc = 0.0; *status = ST_ZERO_VAR_DEF;
    return;
  }
  *zncc = (double)gc.num / sqrt((double)Df * (double)gc.den);
  *status = ST_OK;
}

int dico_pso_search(const uint8_t *f, const uint8_t *g, int W, int H, int pitch, int subset,
                    int step, int R, const int64_t *poi_idx, int64_t n_idx, int modified,
                    int particles, int gmax, double c1, double c2, double vinit,
                    int64_t stop_num, int64_t stop_den, const double *rand, int nthreads,
                    int32_t *u0, int32_t *v0, double *zncc, uint8_t *status, int32_t *gens,
                    int32_t *evals, double *trace) {
  int nx, ny;
  if (dico_grid(W, H, subset, step, R, &nx, &ny)) return -1;
  if (particles < 1 || particles > 4096 || gmax < 1 || gmax > 1000 || stop_num < 0 ||
      stop_den < 1 || stop_den > (1 << 20) || subset > 127 || !rand)
    return -1;
  const int M = subset / 2;
  const int64_t total = (int64_t)nx * ny;
  const int64_t n = poi_idx ? n_idx : total;
  const int64_t win = (int64_t)(2 * R + 1) * (2 * R + 1);
  const int64_t per_poi = (int64_t)gmax * particles * 4;
  if (poi_idx)
    for (int64_t k = 0; k < n; ++k)
      if (poi_idx[k] < 0 || poi_idx[k] >= total) return -1;
  if (nthreads <= 0) nthreads = 1;
  int failed = 0;
#pragma omp parallel num_threads(nthreads)
  {
    uint8_t *seen = malloc((size_t)win);
    zc_t *memo = malloc(sizeof(zc_t) * (size_t)win);
    double (*p)[2] = malloc(sizeof(double[2]) * (size_t)particles);
    double (*v)[2] = malloc(sizeof(double[2]) * (size_t)particles);
    int (*pb)[2] = malloc(sizeof(int[2]) * (size_t)particles);
    zc_t *pbc = malloc(sizeof(zc_t) * (size_t)particles);
    int ok = seen && memo && p && v && pb && pbc;
    if (!ok) {
#pragma omp atomic write
      failed = 1;
    }
#pragma omp for schedule(dynamic, 4)
    for (int64_t k = 0; k < n; ++k) {
      if (!ok) continue;
      int64_t poi = poi_idx ? poi_idx[k] : k;
      pso_ctx c;
      c.f = f; c.g = g; c.pitch = pitch; c.M = M; c.R = R;
      c.N = (int64_t)subset * subset;
      c.seen = seen; c.memo = memo; c.evals = 0;
      memset(seen, 0, (size_t)win);
      poi_centre(poi, nx, M, R, step, &c.x0, &c.y0);
      pso_one(&c, modified, particles, gmax, c1, c2, vinit, stop_num, stop_den,
              rand + k * per_poi, trace ? trace + k * per_poi * 2 : NULL, p, v, pb, pbc,
              &u0[k], &v0[k], &zncc[k], &status[k], &gens[k]);
      evals[k] = c.evals;
    }
    free(seen); free(memo); free(p); free(v); free(pb); free(pbc);
  }
  return failed ? -2 : 0;
}
