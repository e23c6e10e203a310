/*
 * CPU FP64 oracle core: the unaccelerated Chebyshev boundary-integral (CBIE)
 * kernel rows of Paul & Sideris, "Accelerated 3D Maxwell Integral Equation
 * Solver using the Interpolated Factored Green Function Method".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the GPU product path may call,
 * link or load this file; it exists so tests, smoke() and the benchmark's
 * CPU-baseline leg can check the CUDA library against a plain, slow,
 * independent implementation.  It shares no code with the CUDA library.
 *
 * For each requested target x_l this fills four dense rows K_s[l][m]
 * (s = S_e, S_i, D_e, D_i) such that S_s[phi](x_l) = sum_m K_s[l][m] phi_m
 * and D_s[phi](x_l) likewise, where
 *   - for patches p in the regular set R_l (Eq. patch_reg): the Fejer rule
 *     of Sec. III-C, K = G(x_l, x_m) * omega_m, omega_m = J w_i w_j;
 *   - for patches p in the singular set S_l (Eq. patch_sing): the
 *     precomputed-moment rule of Sec. III-D: beta_mn (Eq. int_moments) by
 *     the clustering change of variables (Eqs. mk_cov_1, mk_cov_2, cov) and
 *     an N_beta-point Fejer rule (Eq. int_moments_cov), then
 *     S_p(x_l) = sum_mn a_mn beta_mn (Eq. rp_exp) with a_mn the Chebyshev
 *     coefficients of phi on the patch (Eq. phi_cheby), i.e. the row entry
 *     for node (i', j') of p is sum_mn beta_mn A[m][i'] A[n][j'].
 * The normal-derivative kernel is dG/dn(x) = n(x).(x-y)(i k r - 1) e^{ikr}/(4 pi r^3).
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC cbie_core.c -o libcbie_oracle.so -lm
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef double _Complex cplx;

/* Chebyshev polynomials T_0..T_{n-1} at t by the three-term recurrence. */
static void cheb_T(double t, int n, double *T) {
  if (n > 0) T[0] = 1.0;
  if (n > 1) T[1] = t;
  for (int k = 2; k < n; ++k) T[k] = 2.0 * t * T[k - 1] - T[k - 2];
}

/* Patch geometry as the Chebyshev interpolant of its oversampled samples:
 * coef is [ng][ng][9] (x, x_u, x_v), value(u,v) = sum_mn coef[m][n] T_m(u) T_n(v). */
typedef struct {
  const double *coef;
  int ng;
} patch_geom;

static void geom_eval(const patch_geom *g, double u, double v, int nch, double *out) {
  double Tu[64], Tv[64];
  cheb_T(u, g->ng, Tu);
  cheb_T(v, g->ng, Tv);
  for (int c = 0; c < nch; ++c) out[c] = 0.0;
  for (int m = 0; m < g->ng; ++m) {
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int n = 0; n < g->ng; ++n) {
      const double *cf = g->coef + ((size_t)m * g->ng + n) * 9;
      for (int c = 0; c < nch; ++c) acc[c] += cf[c] * Tv[n];
    }
    for (int c = 0; c < nch; ++c) out[c] += acc[c] * Tu[m];
  }
}

/* ---------------- closest point (Eq. dist_min): golden-section search ---------------- */
static const double GOLD = 0.6180339887498948482;

typedef struct {
  const patch_geom *g;
  const double *x;
  double u;
} inner_ctx;

static double dist2_uv(const patch_geom *g, const double *x, double u, double v) {
  double y[3];
  geom_eval(g, u, v, 3, y);
  double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
  return dx * dx + dy * dy + dz * dz;
}

/* min over v in [a, b] of |x - eta(u, v)|^2 by golden section, fixed iteration count */
static double golden_v(const patch_geom *g, const double *x, double u, double a, double b,
                       int iters, double *vbest) {
  double c = b - GOLD * (b - a), d = a + GOLD * (b - a);
  double fc = dist2_uv(g, x, u, c), fd = dist2_uv(g, x, u, d);
  for (int it = 0; it < iters; ++it) {
    if (fc < fd) {
      b = d; d = c; fd = fc; c = b - GOLD * (b - a); fc = dist2_uv(g, x, u, c);
    } else {
      a = c; c = d; fc = fd; d = a + GOLD * (b - a); fd = dist2_uv(g, x, u, d);
    }
  }
  *vbest = 0.5 * (a + b);
  return dist2_uv(g, x, u, *vbest);
}

static double golden_uv(const patch_geom *g, const double *x, double ua, double ub, double va,
                        double vb, int iters, double *ubest, double *vbest) {
  double a = ua, b = ub;
  double vt;
  double c = b - GOLD * (b - a), d = a + GOLD * (b - a);
  double fc = golden_v(g, x, c, va, vb, iters, &vt), fd = golden_v(g, x, d, va, vb, iters, &vt);
  for (int it = 0; it < iters; ++it) {
    if (fc < fd) {
      b = d; d = c; fd = fc; c = b - GOLD * (b - a); fc = golden_v(g, x, c, va, vb, iters, &vt);
    } else {
      a = c; c = d; fc = fd; d = a + GOLD * (b - a); fd = golden_v(g, x, d, va, vb, iters, &vt);
    }
  }
  *ubest = 0.5 * (a + b);
  double f = golden_v(g, x, *ubest, va, vb, iters, vbest);
  return f;
}

/* Edge snap after the search (reading R15): a parameter within tol of +-1 is put on the edge,
 * where the polish below holds it.  tol is the larger of 1e-9 and twice the width the search's
 * bracket shrinks to, w GOLD^iters for an initial bracket of width w: a shorter search leaves a
 * minimum on an edge farther from it than 1e-9.  At 60 steps the bracket term is below 2e-12
 * (w <= 2), so tol is 1e-9. */
static double snap_tol(double w, int iters) {
  const double t = 2.0 * w * pow(GOLD, iters);
  return t > 1e-9 ? t : 1e-9;
}

static double snap_edge(double t, double tol) {
  if (t > 1.0 - tol) return 1.0;
  if (t < -1.0 + tol) return -1.0;
  return t;
}

/* Position, first and second parametric derivatives of the interpolant (channels 0..2):
 * out = [x, x_u, x_v, x_uu, x_uv, x_vv] (3 each).  T'' by differentiating the recurrence twice. */
static void geom_eval_d2(const patch_geom *g, double u, double v, double *out) {
  double T[2][64], dT[2][64], ddT[2][64];
  double xs[2] = {u, v};
  for (int a = 0; a < 2; ++a) {
    double t = xs[a];
    for (int k = 0; k < g->ng; ++k) {
      if (k == 0) { T[a][0] = 1; dT[a][0] = 0; ddT[a][0] = 0; }
      else if (k == 1) { T[a][1] = t; dT[a][1] = 1; ddT[a][1] = 0; }
      else {
        T[a][k] = 2 * t * T[a][k - 1] - T[a][k - 2];
        dT[a][k] = 2 * T[a][k - 1] + 2 * t * dT[a][k - 1] - dT[a][k - 2];
        ddT[a][k] = 4 * dT[a][k - 1] + 2 * t * ddT[a][k - 1] - ddT[a][k - 2];
      }
    }
  }
  for (int c = 0; c < 18; ++c) out[c] = 0;
  for (int m = 0; m < g->ng; ++m)
    for (int n = 0; n < g->ng; ++n) {
      const double *cf = g->coef + ((size_t)m * g->ng + n) * 9;
      double w[6] = {T[0][m] * T[1][n], dT[0][m] * T[1][n], T[0][m] * dT[1][n],
                     ddT[0][m] * T[1][n], dT[0][m] * dT[1][n], T[0][m] * ddT[1][n]};
      for (int q = 0; q < 6; ++q)
        for (int c = 0; c < 3; ++c) out[3 * q + c] += cf[c] * w[q];
    }
}

/* Newton steps on the stationarity conditions (x - eta).eta_u = (x - eta).eta_v = 0 after the
 * golden-section search: the search only resolves a flat minimum to ~sqrt(eps); these steps
 * make the closest point reproducible to rounding (reading R15).  Coordinates on an edge
 * (|t| = 1 after snapping) stay fixed; a step is taken only where the Hessian is positive. */
static void newton_polish(const patch_geom *g, const double *x, double *u, double *v, int iters) {
  const int fu = (*u == 1.0 || *u == -1.0), fv = (*v == 1.0 || *v == -1.0);
  if (fu && fv) return;
  for (int it = 0; it < iters; ++it) {
    double o[18];
    geom_eval_d2(g, *u, *v, o);
    double r[3] = {x[0] - o[0], x[1] - o[1], x[2] - o[2]};
    double gu = -(r[0] * o[3] + r[1] * o[4] + r[2] * o[5]);
    double gv = -(r[0] * o[6] + r[1] * o[7] + r[2] * o[8]);
    double Huu = o[3] * o[3] + o[4] * o[4] + o[5] * o[5] - (r[0] * o[9] + r[1] * o[10] + r[2] * o[11]);
    double Huv = o[3] * o[6] + o[4] * o[7] + o[5] * o[8] - (r[0] * o[12] + r[1] * o[13] + r[2] * o[14]);
    double Hvv = o[6] * o[6] + o[7] * o[7] + o[8] * o[8] - (r[0] * o[15] + r[1] * o[16] + r[2] * o[17]);
    double du = 0, dv = 0;
    if (fu) {
      if (Hvv > 0) dv = -gv / Hvv;
    } else if (fv) {
      if (Huu > 0) du = -gu / Huu;
    } else {
      double det = Huu * Hvv - Huv * Huv;
      if (Huu > 0 && det > 0) {
        du = -(Hvv * gu - Huv * gv) / det;
        dv = -(Huu * gv - Huv * gu) / det;
      }
    }
    *u = fmin(1.0, fmax(-1.0, *u + du));
    *v = fmin(1.0, fmax(-1.0, *v + dv));
  }
}

/* ---------------- clustering change of variables (Eqs. mk_cov_1, mk_cov_2, cov) ---------------- */
static double nu_f(double t, double d) {
  double a = (M_PI - t) / M_PI;
  return (1.0 / d - 0.5) * a * a * a + (1.0 / d) * ((t - M_PI) / M_PI) + 0.5;
}
static double nu_df(double t, double d) {
  double a = (M_PI - t) / M_PI;
  return -(1.0 / d - 0.5) * 3.0 * a * a / M_PI + 1.0 / (d * M_PI);
}
/* w(t) = 2 pi nu(t)^d / (nu(t)^d + nu(2pi - t)^d) and its derivative */
static void w_f(double t, double d, double *w, double *dw) {
  double n1 = nu_f(t, d), n2 = nu_f(2.0 * M_PI - t, d);
  double a = pow(n1, d), b = pow(n2, d);
  double da = d * pow(n1, d - 1.0) * nu_df(t, d);
  double db = -d * pow(n2, d - 1.0) * nu_df(2.0 * M_PI - t, d);
  *w = 2.0 * M_PI * a / (a + b);
  *dw = 2.0 * M_PI * (da * b - a * db) / ((a + b) * (a + b));
}
/* xi_alpha(tau), d xi_alpha / d tau and the displacement xi_alpha(tau) - alpha on tau in [-1, 1] */
static void xi_f(double alpha, double tau, double d, double *xi, double *mu, double *dxi) {
  double w, dw;
  if (alpha == 1.0) {
    w_f(M_PI * fabs((tau - 1.0) * 0.5), d, &w, &dw);
    *dxi = -((1.0 + alpha) / M_PI) * w;
    *mu = dw;
  } else if (alpha == -1.0) {
    w_f(M_PI * fabs((tau + 1.0) * 0.5), d, &w, &dw);
    *dxi = ((1.0 - alpha) / M_PI) * w;
    *mu = dw;
  } else {
    double s = (tau > 0) ? 1.0 : ((tau < 0) ? -1.0 : 0.0);
    w_f(M_PI * fabs(tau), d, &w, &dw);
    *dxi = ((s - alpha) / M_PI) * w;
    *mu = (s - alpha) * s * dw;
    if (s == 0.0) *mu = 0.0;
  }
  *xi = alpha + *dxi;
}

/* T_k(a) and the differences T_k(a + delta) - T_k(a), k < n, without cancellation:
 * D_{k+1} = 2 delta T_k(a + delta) + 2 a D_k - D_{k-1}, D_0 = 0, D_1 = delta. */
static void cheb_T_diff(double a, double delta, int n, double *Ta, double *Dk) {
  cheb_T(a, n, Ta);
  if (n > 0) Dk[0] = 0.0;
  if (n > 1) Dk[1] = delta;
  for (int k = 1; k + 1 < n; ++k) Dk[k + 1] = 2.0 * delta * (Ta[k] + Dk[k]) + 2.0 * a * Dk[k] - Dk[k - 1];
}

/* Second differences E_k = T_k(a + delta) - T_k(a) - delta T_k'(a), k < n:
 * E_{k+1} = 2 delta D_k + 2 a E_k - E_{k-1}, E_0 = E_1 = 0 (D_k as above). */
static void cheb_T_diff2(double a, double delta, int n, const double *Dk, double *Ek) {
  if (n > 0) Ek[0] = 0.0;
  if (n > 1) Ek[1] = 0.0;
  for (int k = 1; k + 1 < n; ++k) Ek[k + 1] = 2.0 * delta * Dk[k] + 2.0 * a * Ek[k] - Ek[k - 1];
}

/* Displacement e = eta(a + du, b + dv) - eta(a, b) of the patch interpolant and its
 * component along the target normal nrm, both without cancellation:
 *   e = sum_mn c_mn [D_m(u) (T_n(b) + D_n(v)) + T_m(a) D_n(v)],
 *   nrm.e = nrm.R,  R = sum_mn c_mn [D_m D_n + T_n(b) E_m + T_m(a) E_n]
 * (E the second differences).  nrm.e is second order in the distance while e is first
 * order, so it must not be formed from e.  The first-order part du nrm.eta_u + dv nrm.eta_v
 * vanishes on the surface (the normal is orthogonal to the tangent plane); on the
 * interpolant it is the derivative of the interpolation error, which differentiation
 * near an edge inflates to ~ng^2 times the coefficient rounding, so it is left out
 * (reading R21). */
static void geom_disp(const patch_geom *g, double a, double du, double b, double dv, const double *nrm,
                      double *e, double *ne) {
  double Ta[64], Da[64], Ea[64], Tb[64], Db[64], Eb[64];
  cheb_T_diff(a, du, g->ng, Ta, Da);
  cheb_T_diff(b, dv, g->ng, Tb, Db);
  cheb_T_diff2(a, du, g->ng, Da, Ea);
  cheb_T_diff2(b, dv, g->ng, Db, Eb);
  double R[3] = {0, 0, 0};
  e[0] = e[1] = e[2] = 0.0;
  for (int m = 0; m < g->ng; ++m)
    for (int n = 0; n < g->ng; ++n) {
      const double *cf = g->coef + ((size_t)m * g->ng + n) * 9;
      double f = Da[m] * (Tb[n] + Db[n]) + Ta[m] * Db[n];
      double r2 = Da[m] * Db[n] + Tb[n] * Ea[m] + Ta[m] * Eb[n];
      for (int c = 0; c < 3; ++c) {
        e[c] += cf[c] * f;
        R[c] += cf[c] * r2;
      }
    }
  *ne = nrm[0] * R[0] + nrm[1] * R[1] + nrm[2] * R[2];
}

/* The four kernels for the separation d = x - y, its component nd = n_x.d along the
 * target normal, and the wavenumbers: G_e, G_i, dG_e/dn_x, dG_i/dn_x.  r == 0 -> zeros. */
static void kernels4n(const double *dv, double nd, double ke, double ki, cplx *K) {
  double d0 = dv[0], d1 = dv[1], d2 = dv[2];
  double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  if (r == 0.0) {
    K[0] = K[1] = K[2] = K[3] = 0.0;
    return;
  }
  double kk[2] = {ke, ki};
  for (int s = 0; s < 2; ++s) {
    cplx g = cexp(I * kk[s] * r) / (4.0 * M_PI * r);
    K[s] = g;
    K[2 + s] = nd * (I * kk[s] * r - 1.0) * g / (r * r);
  }
}

static void kernels4_xy(const double *x, const double *nx, const double *y, double ke, double ki, cplx *K) {
  double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
  kernels4n(d, nx[0] * d[0] + nx[1] * d[1] + nx[2] * d[2], ke, ki, K);
}

/*
 * Four kernel rows for the targets rows[0..nrows-1].
 *   nodes, normals: [N][3]; qw: [N] Fejer-times-Jacobian weights omega_m;
 *   fine_coef: [P][ng][ng][9] Chebyshev coefficients of (x, x_u, x_v) per patch;
 *   gap: [P] margin added to delta before a patch is ruled regular from its
 *        node distances alone (the node-grid covering radius);
 *   u_nodes: [nc] open Chebyshev nodes; A: [nc][nc] values-to-coefficients map;
 *   t_beta, w_beta: [nbeta] Fejer nodes and weights for the moment rule.
 * Output K: [4][nrows][N] complex (interleaved re, im), sing: [nrows] |S_l|.
 */
int ora_kernel_rows(int P, int nc, int ng, const double *nodes, const double *normals,
                    const double *qw, const double *fine_coef, const double *gap,
                    const double *u_nodes, const double *A, double ke, double ki, double delta,
                    int nbeta, const double *t_beta, const double *w_beta, double cov_d,
                    int gs_iters, int nrows, const int *rows, double *K_out, int *sing) {
  const int npp = nc * nc;
  const size_t N = (size_t)P * npp;
  if (ng > 64 || nc > 64 || nbeta > 256) return -1;
  cplx *K = (cplx *)K_out;
  memset(K_out, 0, sizeof(cplx) * 4 * (size_t)nrows * N);

#pragma omp parallel for schedule(dynamic, 1)
  for (int r = 0; r < nrows; ++r) {
    const int l = rows[r];
    const double *x = nodes + 3 * (size_t)l;
    const double *nx = normals + 3 * (size_t)l;
    const int pl = l / npp;
    int nsing = 0;
    double *ub = malloc(sizeof(double) * nbeta * 2);
    double *vb = malloc(sizeof(double) * nbeta * 2);
    double *Tu = malloc(sizeof(double) * nbeta * nc);
    double *Tv = malloc(sizeof(double) * nbeta * nc);
    cplx *f = malloc(sizeof(cplx) * 4 * nbeta * nbeta);
    cplx *tmp = malloc(sizeof(cplx) * 4 * nbeta * nc);
    cplx *beta = malloc(sizeof(cplx) * 4 * nc * nc);
    cplx *tmp2 = malloc(sizeof(cplx) * 4 * nc * nc);
    for (int p = 0; p < P; ++p) {
      patch_geom g = {fine_coef + (size_t)p * ng * ng * 9, ng};
      double uc, vc;
      int singular = 0;
      if (p == pl) {
        /* target is a node of this patch: its own parameters are the closest point */
        int il = (l % npp) / nc, jl = l % nc;
        uc = u_nodes[il];
        vc = u_nodes[jl];
        singular = 1;
      } else {
        double dmin = INFINITY;
        int im = 0, jm = 0;
        for (int i = 0; i < nc; ++i)
          for (int j = 0; j < nc; ++j) {
            const double *y = nodes + 3 * ((size_t)p * npp + i * nc + j);
            double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
            double dd = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            if (dd < dmin) { dmin = dd; im = i; jm = j; }
          }
        if (dmin <= delta + gap[p]) {
          /* bracket from the neighbouring nodes (the grid is descending in u) */
          double ua = (im == nc - 1) ? -1.0 : u_nodes[im + 1];
          double uz = (im == 0) ? 1.0 : u_nodes[im - 1];
          double va = (jm == nc - 1) ? -1.0 : u_nodes[jm + 1];
          double vz = (jm == 0) ? 1.0 : u_nodes[jm - 1];
          double d2 = golden_uv(&g, x, ua, uz, va, vz, gs_iters, &uc, &vc);
          uc = snap_edge(uc, snap_tol(uz - ua, gs_iters));
          vc = snap_edge(vc, snap_tol(vz - va, gs_iters));
          newton_polish(&g, x, &uc, &vc, 4);
          (void)d2;
          double dist = sqrt(dist2_uv(&g, x, uc, vc));
          singular = dist <= delta;
        }
      }
      const size_t m0 = (size_t)p * npp;
      if (!singular) {
        for (int mm = 0; mm < npp; ++mm) {
          cplx k4[4];
          kernels4_xy(x, nx, nodes + 3 * (m0 + mm), ke, ki, k4);
          for (int s = 0; s < 4; ++s) K[((size_t)s * nrows + r) * N + m0 + mm] = k4[s] * qw[m0 + mm];
        }
        continue;
      }
      ++nsing;
      /* clustered nodes, their Jacobians mu (Eq. int_moments_1) and displacements */
      double dub[256], dvb[256];
      for (int i = 0; i < nbeta; ++i) {
        xi_f(uc, t_beta[i], cov_d, &ub[2 * i], &ub[2 * i + 1], &dub[i]);
        xi_f(vc, t_beta[i], cov_d, &vb[2 * i], &vb[2 * i + 1], &dvb[i]);
        cheb_T(ub[2 * i], nc, Tu + (size_t)i * nc);
        cheb_T(vb[2 * i], nc, Tv + (size_t)i * nc);
      }
      /* integrand samples f_ij = K(x, eta(u_i, v_j)) J mu_i mu_j w_i w_j (Eq. int_moments_cov) */
      for (int i = 0; i < nbeta; ++i)
        for (int j = 0; j < nbeta; ++j) {
          double gv[9];
          geom_eval(&g, ub[2 * i], vb[2 * j], 9, gv);
          double cx = gv[4] * gv[8] - gv[5] * gv[7];
          double cy = gv[5] * gv[6] - gv[3] * gv[8];
          double cz = gv[3] * gv[7] - gv[4] * gv[6];
          double J = sqrt(cx * cx + cy * cy + cz * cz);
          double wt = J * ub[2 * i + 1] * vb[2 * j + 1] * w_beta[i] * w_beta[j];
          cplx k4[4];
          if (p == pl) {
            /* Target on this patch: it is the interpolated surface point eta_p(u_i', v_j')
             * (reading R12); x - y = -(eta(u, v) - eta(uc, vc)) and its normal component are
             * formed from Chebyshev differences so that no cancellation occurs near the target. */
            double e[3], ne;
            geom_disp(&g, uc, dub[i], vc, dvb[j], nx, e, &ne);
            double dneg[3] = {-e[0], -e[1], -e[2]};
            kernels4n(dneg, -ne, ke, ki, k4);
          } else {
            kernels4_xy(x, nx, gv, ke, ki, k4);
          }
          for (int s = 0; s < 4; ++s) f[((size_t)s * nbeta + i) * nbeta + j] = k4[s] * wt;
        }
      /* beta_mn = sum_ij f_ij T_m(u_i) T_n(v_j) */
      for (int s = 0; s < 4; ++s) {
        for (int i = 0; i < nbeta; ++i)
          for (int n = 0; n < nc; ++n) {
            cplx acc = 0;
            for (int j = 0; j < nbeta; ++j) acc += f[((size_t)s * nbeta + i) * nbeta + j] * Tv[(size_t)j * nc + n];
            tmp[((size_t)s * nbeta + i) * nc + n] = acc;
          }
        for (int m = 0; m < nc; ++m)
          for (int n = 0; n < nc; ++n) {
            cplx acc = 0;
            for (int i = 0; i < nbeta; ++i) acc += Tu[(size_t)i * nc + m] * tmp[((size_t)s * nbeta + i) * nc + n];
            beta[((size_t)s * nc + m) * nc + n] = acc;
          }
        /* node weights W[i'][j'] = sum_mn beta_mn A[m][i'] A[n][j'] */
        for (int m = 0; m < nc; ++m)
          for (int jp = 0; jp < nc; ++jp) {
            cplx acc = 0;
            for (int n = 0; n < nc; ++n) acc += beta[((size_t)s * nc + m) * nc + n] * A[n * nc + jp];
            tmp2[((size_t)s * nc + m) * nc + jp] = acc;
          }
        for (int ip = 0; ip < nc; ++ip)
          for (int jp = 0; jp < nc; ++jp) {
            cplx acc = 0;
            for (int m = 0; m < nc; ++m) acc += A[m * nc + ip] * tmp2[((size_t)s * nc + m) * nc + jp];
            K[((size_t)s * nrows + r) * N + m0 + (size_t)ip * nc + jp] = acc;
          }
      }
    }
    sing[r] = nsing;
    free(ub); free(vb); free(Tu); free(Tv); free(f); free(tmp); free(beta); free(tmp2);
  }
  return 0;
}

/* Closest point of x to patch p (exposed for tests): returns dist, writes (u, v). */
double ora_closest_point(int nc, int ng, const double *patch_nodes, const double *coef,
                         const double *u_nodes, const double *x, int gs_iters, double *uv) {
  patch_geom g = {coef, ng};
  double dmin = INFINITY;
  int im = 0, jm = 0;
  for (int i = 0; i < nc; ++i)
    for (int j = 0; j < nc; ++j) {
      const double *y = patch_nodes + 3 * (i * nc + j);
      double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
      double dd = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      if (dd < dmin) { dmin = dd; im = i; jm = j; }
    }
  double ua = (im == nc - 1) ? -1.0 : u_nodes[im + 1];
  double uz = (im == 0) ? 1.0 : u_nodes[im - 1];
  double va = (jm == nc - 1) ? -1.0 : u_nodes[jm + 1];
  double vz = (jm == 0) ? 1.0 : u_nodes[jm - 1];
  double uc, vc;
  golden_uv(&g, x, ua, uz, va, vz, gs_iters, &uc, &vc);
  uv[0] = snap_edge(uc, snap_tol(uz - ua, gs_iters));
  uv[1] = snap_edge(vc, snap_tol(vz - va, gs_iters));
  newton_polish(&g, x, &uv[0], &uv[1], 4);
  return sqrt(dist2_uv(&g, x, uv[0], uv[1]));
}

/* The change of variables itself (exposed for tests). */
void ora_cov(double alpha, int n, const double *tau, double d, double *xi, double *mu) {
  double dx;
  for (int i = 0; i < n; ++i) xi_f(alpha, tau[i], d, &xi[i], &mu[i], &dx);
}
