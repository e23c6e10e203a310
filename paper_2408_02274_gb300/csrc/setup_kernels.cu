// Device setup kernels (FP64): node geometry and quadrature weights
// (Sec. III-A/C), closest points (Eq. dist_min), singular moments
// (Sec. III-D) and the near-field matrix with local corrections (Sec. III-H).
#include "kernels.h"

namespace ifgf {

// ---------------------------------------------------------------- small tables
// fejer[n]: Fejer weights (Eq. fejer_weighs); A[n][n]: values -> Chebyshev
// coefficients on the open grid (a_0 with factor 1/n, a_i with 2/n);
// Dm[n][n]: derivative of the interpolant at the nodes.
__global__ void k_cheb_tables(int n, double* fejer, double* A, double* Dm) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n && fejer) {
    double s = 0;
    for (int m = 1; m <= n / 2; ++m) s += cos(m * kPi * (2 * t + 1) / n) / (4.0 * m * m - 1.0);
    fejer[t] = (2.0 / n) * (1.0 - 2.0 * s);
  }
  if (t < n * n) {
    int i = t / n, j = t % n;
    if (A) A[t] = (i == 0 ? 1.0 : 2.0) / n * cos(i * (j + 0.5) * kPi / n);
    if (Dm) {
      // D[i][j] = sum_k T_k'(x_i) A[k][j], T_k'(cos th) = k sin(k th)/sin th
      double th = (i + 0.5) * kPi / n;
      double acc = 0;
      for (int k = 1; k < n; ++k)
        acc += k * sin(k * th) / sin(th) * (2.0 / n) * cos(k * (j + 0.5) * kPi / n);
      Dm[t] = acc;
    }
  }
}

// Per-node geometry from the sampled tangents: J, n, t1, t2, inverse metric, omega = J w_i w_j.
__global__ void k_node_geom(int N, int nc, const double* fejer, NodeGeom g) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= N) return;
  const double* u = g.xu + 3 * (size_t)l;
  const double* v = g.xv + 3 * (size_t)l;
  double c0 = u[1] * v[2] - u[2] * v[1], c1 = u[2] * v[0] - u[0] * v[2], c2 = u[0] * v[1] - u[1] * v[0];
  double J = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
  double n0 = c0 / J, n1 = c1 / J, n2 = c2 / J;
  double lu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  double a0 = u[0] / lu, a1 = u[1] / lu, a2 = u[2] / lu;
  double E = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  double F = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
  double G = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  double det = E * G - F * F;
  g.J[l] = J;
  g.n[3 * l] = n0; g.n[3 * l + 1] = n1; g.n[3 * l + 2] = n2;
  g.t1[3 * l] = a0; g.t1[3 * l + 1] = a1; g.t1[3 * l + 2] = a2;
  g.t2[3 * l] = n1 * a2 - n2 * a1;
  g.t2[3 * l + 1] = n2 * a0 - n0 * a2;
  g.t2[3 * l + 2] = n0 * a1 - n1 * a0;
  g.g[3 * l] = G / det;
  g.g[3 * l + 1] = -F / det;
  g.g[3 * l + 2] = E / det;
  int i = (l % (nc * nc)) / nc, j = l % nc;
  g.w[l] = J * fejer[i] * fejer[j];
}

// 2D Chebyshev coefficients of the oversampled patch geometry: coef = A (x) A applied to samples.
__global__ void k_fine_coefs(int ng, const double* A, const double* fine, double* coef) {
  int p = blockIdx.x;
  const double* f = fine + (size_t)p * ng * ng * 9;
  double* c = coef + (size_t)p * ng * ng * 9;
  for (int t = threadIdx.x; t < ng * ng * 9; t += blockDim.x) {
    int ch = t % 9, mn = t / 9, m = mn / ng, n = mn % ng;
    double acc = 0;
    for (int i = 0; i < ng; ++i) {
      double ai = A[m * ng + i];
      double row = 0;
      for (int j = 0; j < ng; ++j) row += A[n * ng + j] * f[((size_t)i * ng + j) * 9 + ch];
      acc += ai * row;
    }
    c[t] = acc;
  }
}

// ---------------------------------------------------------------- patch interpolant
struct PatchCoef {
  const double* c;  // [ng][ng][9]
  int ng;
};

__device__ inline void geom_at(const PatchCoef& pc, double u, double v, int nch, double* out) {
  double Tu0 = 1, Tu1 = u;
  for (int c = 0; c < nch; ++c) out[c] = 0;
  for (int m = 0; m < pc.ng; ++m) {
    double Tum = (m == 0) ? 1.0 : (m == 1 ? u : 0);
    if (m >= 2) {
      Tum = 2 * u * Tu1 - Tu0;
      Tu0 = Tu1;
      Tu1 = Tum;
    }
    double acc[9];
    for (int c = 0; c < nch; ++c) acc[c] = 0;
    double Tv0 = 1, Tv1 = v;
    for (int n = 0; n < pc.ng; ++n) {
      double Tvn = (n == 0) ? 1.0 : (n == 1 ? v : 0);
      if (n >= 2) {
        Tvn = 2 * v * Tv1 - Tv0;
        Tv0 = Tv1;
        Tv1 = Tvn;
      }
      const double* cf = pc.c + ((size_t)m * pc.ng + n) * 9;
      for (int c = 0; c < nch; ++c) acc[c] += cf[c] * Tvn;
    }
    for (int c = 0; c < nch; ++c) out[c] += acc[c] * Tum;
  }
}

__device__ inline double dist2_at(const PatchCoef& pc, const double* x, double u, double v) {
  double y[3];
  geom_at(pc, u, v, 3, y);
  double a = x[0] - y[0], b = x[1] - y[1], c = x[2] - y[2];
  return a * a + b * b + c * c;
}

// ---------------------------------------------------------------- closest point (Eq. dist_min)
__device__ const double kGold = 0.6180339887498948482;

// Geometry contracted along u at a fixed u: cu[n][c] = sum_m coef[m][n][c] T_m(u), c < 3.
__device__ inline void contract_u(const PatchCoef& pc, double u, double* cu) {
  for (int t = 0; t < pc.ng * 3; ++t) cu[t] = 0;
  double T0 = 1, T1 = u;
  for (int m = 0; m < pc.ng; ++m) {
    double Tm = (m == 0) ? 1.0 : (m == 1 ? u : 0);
    if (m >= 2) {
      Tm = 2 * u * T1 - T0;
      T0 = T1;
      T1 = Tm;
    }
    for (int n = 0; n < pc.ng; ++n) {
      const double* cf = pc.c + ((size_t)m * pc.ng + n) * 9;
      cu[3 * n] += cf[0] * Tm;
      cu[3 * n + 1] += cf[1] * Tm;
      cu[3 * n + 2] += cf[2] * Tm;
    }
  }
}

__device__ inline double dist2_v(const double* cu, int ng, const double* x, double v) {
  double y0 = 0, y1 = 0, y2 = 0, T0 = 1, T1 = v;
  for (int n = 0; n < ng; ++n) {
    double Tn = (n == 0) ? 1.0 : (n == 1 ? v : 0);
    if (n >= 2) {
      Tn = 2 * v * T1 - T0;
      T0 = T1;
      T1 = Tn;
    }
    y0 += cu[3 * n] * Tn;
    y1 += cu[3 * n + 1] * Tn;
    y2 += cu[3 * n + 2] * Tn;
  }
  double a = x[0] - y0, b = x[1] - y1, c = x[2] - y2;
  return a * a + b * b + c * c;
}

// min over v in [a, b] of |x - eta(u, v)|^2 by golden section (fixed iteration count);
// the interpolant is contracted along u once and then evaluated in v only.
__device__ double golden_inner(const PatchCoef& pc, const double* x, double u, double a, double b,
                               int iters, double* vbest) {
  double cu[3 * 48];
  contract_u(pc, u, cu);
  double c = b - kGold * (b - a), d = a + kGold * (b - a);
  double fc = dist2_v(cu, pc.ng, x, c), fd = dist2_v(cu, pc.ng, x, d);
  for (int it = 0; it < iters; ++it) {
    if (fc < fd) {
      b = d; d = c; fd = fc; c = b - kGold * (b - a); fc = dist2_v(cu, pc.ng, x, c);
    } else {
      a = c; c = d; fc = fd; d = a + kGold * (b - a); fd = dist2_v(cu, pc.ng, x, d);
    }
  }
  *vbest = 0.5 * (a + b);
  return dist2_v(cu, pc.ng, x, *vbest);
}

// Edge snap after the search (reading R15): a parameter within tol of +-1 goes on the edge,
// where the Newton polish holds it.  tol is the larger of 1e-9 and twice the width the search's
// bracket shrinks to (w kGold^iters for an initial width w), so that a shorter search still puts
// a minimum that lies on an edge there; at 60 steps the bracket term is below 2e-12 (w <= 2) and
// tol is 1e-9.
__device__ inline double snap_tol(double w, int iters) {
  const double t = 2.0 * w * pow(kGold, (double)iters);
  return t > 1e-9 ? t : 1e-9;
}

__device__ inline double snap_edge(double t, double tol) {
  if (t > 1.0 - tol) return 1.0;
  if (t < -1.0 + tol) return -1.0;
  return t;
}

// Position, first and second parametric derivatives of the interpolant (channels 0..2):
// out = [x, x_u, x_v, x_uu, x_uv, x_vv], T'' by differentiating the recurrence twice.
__device__ void geom_d2(const PatchCoef& pc, double u, double v, double* out) {
  for (int c = 0; c < 18; ++c) out[c] = 0;
  double Tu0 = 1, Tu1 = u, dTu0 = 0, dTu1 = 1, ddTu0 = 0, ddTu1 = 0;
  for (int m = 0; m < pc.ng; ++m) {
    double Tm, dTm, ddTm;
    if (m == 0) { Tm = 1; dTm = 0; ddTm = 0; }
    else if (m == 1) { Tm = u; dTm = 1; ddTm = 0; }
    else {
      Tm = 2 * u * Tu1 - Tu0;
      dTm = 2 * Tu1 + 2 * u * dTu1 - dTu0;
      ddTm = 4 * dTu1 + 2 * u * ddTu1 - ddTu0;
      Tu0 = Tu1; Tu1 = Tm; dTu0 = dTu1; dTu1 = dTm; ddTu0 = ddTu1; ddTu1 = ddTm;
    }
    double a[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};   // sum_n c_mn {T_n, T_n', T_n''}(v)
    double Tv0 = 1, Tv1 = v, dTv0 = 0, dTv1 = 1, ddTv0 = 0, ddTv1 = 0;
    for (int n = 0; n < pc.ng; ++n) {
      double Tn, dTn, ddTn;
      if (n == 0) { Tn = 1; dTn = 0; ddTn = 0; }
      else if (n == 1) { Tn = v; dTn = 1; ddTn = 0; }
      else {
        Tn = 2 * v * Tv1 - Tv0;
        dTn = 2 * Tv1 + 2 * v * dTv1 - dTv0;
        ddTn = 4 * dTv1 + 2 * v * ddTv1 - ddTv0;
        Tv0 = Tv1; Tv1 = Tn; dTv0 = dTv1; dTv1 = dTn; ddTv0 = ddTv1; ddTv1 = ddTn;
      }
      const double* cf = pc.c + ((size_t)m * pc.ng + n) * 9;
      for (int c = 0; c < 3; ++c) {
        a[0][c] += cf[c] * Tn;
        a[1][c] += cf[c] * dTn;
        a[2][c] += cf[c] * ddTn;
      }
    }
    for (int c = 0; c < 3; ++c) {
      out[c] += a[0][c] * Tm;
      out[3 + c] += a[0][c] * dTm;
      out[6 + c] += a[1][c] * Tm;
      out[9 + c] += a[0][c] * ddTm;
      out[12 + c] += a[1][c] * dTm;
      out[15 + c] += a[2][c] * Tm;
    }
  }
}

// Newton steps on the stationarity conditions (x - eta).eta_u = (x - eta).eta_v = 0 after
// the golden-section search, which resolves a flat minimum only to ~sqrt(eps): they make
// the closest point reproducible to rounding (reading R15).  Edge coordinates (|t| = 1
// after snapping) stay fixed; a step is taken only where the Hessian is positive.
__device__ void newton_polish(const PatchCoef& pc, const double* x, double* u, double* v, int iters) {
  const bool fu = (*u == 1.0 || *u == -1.0), fv = (*v == 1.0 || *v == -1.0);
  if (fu && fv) return;
  for (int it = 0; it < iters; ++it) {
    double o[18];
    geom_d2(pc, *u, *v, o);
    const double r0 = x[0] - o[0], r1 = x[1] - o[1], r2 = x[2] - o[2];
    const double gu = -(r0 * o[3] + r1 * o[4] + r2 * o[5]);
    const double gv = -(r0 * o[6] + r1 * o[7] + r2 * o[8]);
    const double Huu = o[3] * o[3] + o[4] * o[4] + o[5] * o[5] - (r0 * o[9] + r1 * o[10] + r2 * o[11]);
    const double Huv = o[3] * o[6] + o[4] * o[7] + o[5] * o[8] - (r0 * o[12] + r1 * o[13] + r2 * o[14]);
    const double Hvv = o[6] * o[6] + o[7] * o[7] + o[8] * o[8] - (r0 * o[15] + r1 * o[16] + r2 * o[17]);
    double du = 0, dv = 0;
    if (fu) {
      if (Hvv > 0) dv = -gv / Hvv;
    } else if (fv) {
      if (Huu > 0) du = -gu / Huu;
    } else {
      const double det = Huu * Hvv - Huv * Huv;
      if (Huu > 0 && det > 0) {
        du = -(Hvv * gu - Huv * gv) / det;
        dv = -(Huu * gv - Huv * gu) / det;
      }
    }
    *u = fmin(1.0, fmax(-1.0, *u + du));
    *v = fmin(1.0, fmax(-1.0, *v + dv));
  }
}

// One thread per candidate (target, patch) pair: closest parameters and the
// singular-set decision dist(x_l, Gamma_p) <= delta (Eq. patch_sing).
__global__ void k_closest(int npairs, int nc, int ng, int iters, double delta, const int* pair_tgt,
                          const int* pair_patch, const double* x, const double* coef,
                          const double* unodes, double* uv, uint8_t* singular) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npairs) return;
  const int l = pair_tgt[e], p = pair_patch[e];
  const int npp = nc * nc;
  const double* xl = x + 3 * (size_t)l;
  if (l / npp == p) {
    int i = (l % npp) / nc, j = l % nc;
    uv[2 * e] = unodes[i];
    uv[2 * e + 1] = unodes[j];
    singular[e] = 1;
    return;
  }
  // bracket from the nearest node and its grid neighbours
  double dmin = 1e300;
  int im = 0, jm = 0;
  for (int i = 0; i < nc; ++i)
    for (int j = 0; j < nc; ++j) {
      const double* y = x + 3 * ((size_t)p * npp + i * nc + j);
      double a = xl[0] - y[0], b = xl[1] - y[1], c = xl[2] - y[2];
      double dd = sqrt(a * a + b * b + c * c);
      if (dd < dmin) { dmin = dd; im = i; jm = j; }
    }
  double ua = (im == nc - 1) ? -1.0 : unodes[im + 1];
  double ub = (im == 0) ? 1.0 : unodes[im - 1];
  double va = (jm == nc - 1) ? -1.0 : unodes[jm + 1];
  double vb = (jm == 0) ? 1.0 : unodes[jm - 1];
  PatchCoef pc{coef + (size_t)p * ng * ng * 9, ng};
  double a = ua, b = ub, vt;
  double c = b - kGold * (b - a), d = a + kGold * (b - a);
  double fc = golden_inner(pc, xl, c, va, vb, iters, &vt);
  double fd = golden_inner(pc, xl, d, va, vb, iters, &vt);
  for (int it = 0; it < iters; ++it) {
    if (fc < fd) {
      b = d; d = c; fd = fc; c = b - kGold * (b - a); fc = golden_inner(pc, xl, c, va, vb, iters, &vt);
    } else {
      a = c; c = d; fc = fd; d = a + kGold * (b - a); fd = golden_inner(pc, xl, d, va, vb, iters, &vt);
    }
  }
  double uc = 0.5 * (a + b), vc;
  golden_inner(pc, xl, uc, va, vb, iters, &vc);
  uc = snap_edge(uc, snap_tol(ub - ua, iters));
  vc = snap_edge(vc, snap_tol(vb - va, iters));
  newton_polish(pc, xl, &uc, &vc, 4);
  uv[2 * e] = uc;
  uv[2 * e + 1] = vc;
  singular[e] = sqrt(dist2_at(pc, xl, uc, vc)) <= delta ? 1 : 0;
}

// ---------------------------------------------------------------- change of variables
__device__ inline double nu_f(double t, double d) {
  double a = (kPi - t) / kPi;
  return (1.0 / d - 0.5) * a * a * a + (1.0 / d) * ((t - kPi) / kPi) + 0.5;
}
__device__ inline double nu_df(double t, double d) {
  double a = (kPi - t) / kPi;
  return -(1.0 / d - 0.5) * 3.0 * a * a / kPi + 1.0 / (d * kPi);
}
// w(t) of Eq. mk_cov_1 (with nu of Eq. mk_cov_2) and its derivative
__device__ inline void w_f(double t, double d, double* w, double* dw) {
  double n1 = nu_f(t, d), n2 = nu_f(2.0 * kPi - t, d);
  double a = pow(n1, d), b = pow(n2, d);
  double da = d * pow(n1, d - 1.0) * nu_df(t, d);
  double db = -d * pow(n2, d - 1.0) * nu_df(2.0 * kPi - t, d);
  *w = 2.0 * kPi * a / (a + b);
  *dw = 2.0 * kPi * (da * b - a * db) / ((a + b) * (a + b));
}
// xi_alpha(tau) (Eq. cov), d xi / d tau and the displacement xi - alpha
__device__ inline void xi_f(double alpha, double tau, double d, double* xi, double* mu, double* dxi) {
  double w, dw;
  if (alpha == 1.0) {
    w_f(kPi * fabs((tau - 1.0) * 0.5), d, &w, &dw);
    *dxi = -(2.0 / kPi) * w;
    *mu = dw;
  } else if (alpha == -1.0) {
    w_f(kPi * fabs((tau + 1.0) * 0.5), d, &w, &dw);
    *dxi = (2.0 / kPi) * w;
    *mu = dw;
  } else {
    double s = (tau > 0) ? 1.0 : ((tau < 0) ? -1.0 : 0.0);
    w_f(kPi * fabs(tau), d, &w, &dw);
    *dxi = ((s - alpha) / kPi) * w;
    *mu = (s == 0.0) ? 0.0 : (s - alpha) * s * dw;
  }
  *xi = alpha + *dxi;
}

// T_k(a + delta) - T_k(a) (first differences D_k) and T_k(a + delta) - T_k(a) - delta T_k'(a)
// (second differences E_k) for k = 0.. by the recurrences
//   D_{k+1} = 2 delta T_k(a + delta) + 2 a D_k - D_{k-1},  E_{k+1} = 2 delta D_k + 2 a E_k - E_{k-1},
// which do not cancel for small delta.
struct ChebDiff {
  double a, delta, T0, T1, D0, D1, E0, E1;
  int k;
  __device__ ChebDiff(double a_, double d_) : a(a_), delta(d_), T0(1), T1(a_), D0(0), D1(d_), E0(0), E1(0), k(0) {}
  // returns (T_k(a), D_k, E_k) and advances
  __device__ inline void next(double* Tk, double* Dk, double* Ek) {
    if (k == 0) {
      *Tk = 1.0; *Dk = 0.0; *Ek = 0.0;
    } else if (k == 1) {
      *Tk = a; *Dk = delta; *Ek = 0.0;
    } else {
      double T2 = 2 * a * T1 - T0;
      double D2 = 2 * delta * (T1 + D1) + 2 * a * D1 - D0;
      double E2 = 2 * delta * D1 + 2 * a * E1 - E0;
      T0 = T1; T1 = T2; D0 = D1; D1 = D2; E0 = E1; E1 = E2;
      *Tk = T2; *Dk = D2; *Ek = E2;
    }
    ++k;
  }
};

// ---------------------------------------------------------------- singular weights
// One warp per singular (target, patch) pair.  With the clustered Fejer
// nodes (u_i, v_j) of Eq. int_moments_1 and f_ij = K(x, eta(u_i, v_j)) J
// mu_i mu_j w_i w_j (Eq. int_moments_cov), the moments beta_mn = sum_ij f_ij
// T_m(u_i) T_n(v_j) are mapped to node weights W = A^T beta A, computed here
// as W[i'][j'] = sum_ij L[i][i'] f_ij L[j][j'] with L[i][i'] = sum_m T_m(u_i)
// A[m][i'] (the same sum, regrouped).  Kernels: G_e, G_i, dG_e/dn, dG_i/dn.
__global__ void k_moments(int nsp, const int* sp_pair, const int* pair_tgt, const int* pair_patch,
                          const double* uvc, int nc, int ng, int nbeta, double cov_d,
                          const double* tb, const double* wb, const double* A, const double* x,
                          const double* nrm, const double* coef, double ke, double ki, double* W) {
  extern __shared__ double sm[];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int nw = blockDim.x / 32;
  const int sp = blockIdx.x * nw + warp;
  // per-warp shared layout
  const int nb = nbeta, npp = nc * nc;
  size_t per = 6 * (size_t)nb + (size_t)ng * 9 + 8 * (size_t)nb + (size_t)nb * nc + 8 * (size_t)nc +
               (size_t)nc + 8 * (size_t)npp + 9 * (size_t)ng;
  double* base = sm + per * warp;
  double* ub = base;                 // [nb] u_i
  double* mub = ub + nb;             // [nb]
  double* vb = mub + nb;             // [nb]
  double* mvb = vb + nb;             // [nb]
  double* cu = mvb + nb;             // [ng][9] geometry contracted at u_i
  double* f = cu + (size_t)ng * 9;   // [4][nb][2] integrand row i
  double* Lv = f + 8 * (size_t)nb;   // [nb][nc] Lagrange weights of v_j
  double* tmp = Lv + (size_t)nb * nc;  // [4][nc][2]
  double* Lu = tmp + 8 * (size_t)nc;   // [nc] Lagrange weights of u_i
  double* Wacc = Lu + nc;              // [4][npp][2]
  double* dub = Wacc + 8 * (size_t)npp;  // [nb] u_i - uc
  double* dvb = dub + nb;                // [nb] v_j - vc
  double* cua = dvb + nb;                // [ng][3] geometry contracted at uc
  double* cud = cua + 3 * (size_t)ng;    // [ng][3] contracted with T_m(u_i) - T_m(uc)
  double* cuE = cud + 3 * (size_t)ng;    // [ng][3] contracted with the second differences at u_i
  if (sp >= nsp) return;
  const int e = sp_pair[sp];
  const int l = pair_tgt[e], p = pair_patch[e];
  const double uc = uvc[2 * e], vc = uvc[2 * e + 1];
  PatchCoef pc{coef + (size_t)p * ng * ng * 9, ng};
  const double xs[3] = {x[3 * (size_t)l], x[3 * (size_t)l + 1], x[3 * (size_t)l + 2]};
  // Target on this patch: it is the interpolated surface point at its own parameters
  // (reading R12), and x - y = -(eta(u, v) - eta(uc, vc)) is formed from Chebyshev
  // differences so that no cancellation occurs next to the target.
  const bool self = (l / npp == p);
  const double nx0 = nrm[3 * (size_t)l], nx1 = nrm[3 * (size_t)l + 1], nx2 = nrm[3 * (size_t)l + 2];
  for (int i = lane; i < nb; i += 32) {
    xi_f(uc, tb[i], cov_d, &ub[i], &mub[i], &dub[i]);
    xi_f(vc, tb[i], cov_d, &vb[i], &mvb[i], &dvb[i]);
  }
  if (self)
    for (int t = lane; t < ng * 3; t += 32) {
      int n = t / 3, ch = t % 3;
      double T0 = 1, T1 = uc, acc = 0;
      for (int m = 0; m < ng; ++m) {
        double Tm = (m == 0) ? 1.0 : (m == 1 ? uc : 0);
        if (m >= 2) {
          Tm = 2 * uc * T1 - T0;
          T0 = T1;
          T1 = Tm;
        }
        acc += pc.c[((size_t)m * ng + n) * 9 + ch] * Tm;
      }
      cua[t] = acc;
    }
  __syncwarp();
  for (int t = lane; t < nb * nc; t += 32) {
    int j = t / nc, jp = t % nc;
    double v = vb[j], T0 = 1, T1 = v, acc = A[jp];   // m = 0 term
    if (nc > 1) acc += v * A[nc + jp];
    for (int m = 2; m < nc; ++m) {
      double T2 = 2 * v * T1 - T0;
      acc += T2 * A[m * nc + jp];
      T0 = T1;
      T1 = T2;
    }
    Lv[t] = acc;
  }
  for (int t = lane; t < 8 * npp; t += 32) Wacc[t] = 0;
  __syncwarp();
  const double kk[2] = {ke, ki};
  for (int i = 0; i < nb; ++i) {
    const double u = ub[i];
    // geometry contracted along u at u_i: cu[n][ch] = sum_m coef[m][n][ch] T_m(u)
    for (int t = lane; t < ng * 9; t += 32) {
      int n = t / 9, ch = t % 9;
      double T0 = 1, T1 = u, acc = 0;
      for (int m = 0; m < ng; ++m) {
        double Tm = (m == 0) ? 1.0 : (m == 1 ? u : 0);
        if (m >= 2) {
          Tm = 2 * u * T1 - T0;
          T0 = T1;
          T1 = Tm;
        }
        acc += pc.c[((size_t)m * ng + n) * 9 + ch] * Tm;
      }
      cu[t] = acc;
    }
    if (self)
      for (int t = lane; t < ng * 3; t += 32) {
        int n = t / 3, ch = t % 3;
        ChebDiff cd(uc, dub[i]);
        double acc = 0, acce = 0;
        for (int m = 0; m < ng; ++m) {
          double Tm, Dm, Em;
          cd.next(&Tm, &Dm, &Em);
          acc += pc.c[((size_t)m * ng + n) * 9 + ch] * Dm;
          acce += pc.c[((size_t)m * ng + n) * 9 + ch] * Em;
        }
        cud[t] = acc;
        cuE[t] = acce;
      }
    if (lane < nc) {
      double T0 = 1, T1 = u, acc = A[lane];
      if (nc > 1) acc += u * A[nc + lane];
      for (int m = 2; m < nc; ++m) {
        double T2 = 2 * u * T1 - T0;
        acc += T2 * A[m * nc + lane];
        T0 = T1;
        T1 = T2;
      }
      Lu[lane] = acc;
    }
    __syncwarp();
    for (int j = lane; j < nb; j += 32) {
      const double v = vb[j];
      double gv[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      double T0 = 1, T1 = v;
      for (int n = 0; n < ng; ++n) {
        double Tn = (n == 0) ? 1.0 : (n == 1 ? v : 0);
        if (n >= 2) {
          Tn = 2 * v * T1 - T0;
          T0 = T1;
          T1 = Tn;
        }
        for (int ch = 0; ch < 9; ++ch) gv[ch] += cu[n * 9 + ch] * Tn;
      }
      double c0 = gv[4] * gv[8] - gv[5] * gv[7];
      double c1 = gv[5] * gv[6] - gv[3] * gv[8];
      double c2 = gv[3] * gv[7] - gv[4] * gv[6];
      double J = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
      double wt = J * mub[i] * mvb[j] * wb[i] * wb[j];
      double d0 = xs[0] - gv[0], d1 = xs[1] - gv[1], d2 = xs[2] - gv[2];
      double ndn = nx0 * d0 + nx1 * d1 + nx2 * d2;
      if (self) {
        // e = eta(u, v) - eta(uc, vc) and, separately, its normal component from the
        // second-order remainder (n.e is second order in the distance, e first order).
        // The first-order part du n.eta_u + dv n.eta_v vanishes on the surface; on the
        // interpolant it is the derivative of the interpolation error, which near an edge
        // carries ~ng^2 times the coefficient rounding, so it is left out (reading R21).
        ChebDiff cd(vc, dvb[j]);
        double e0 = 0, e1 = 0, e2 = 0, R0 = 0, R1 = 0, R2 = 0;
        for (int n = 0; n < ng; ++n) {
          double Tn, Dn, En;
          cd.next(&Tn, &Dn, &En);
          const double tv = Tn + Dn;   // T_n(v_j)
          e0 += cud[3 * n] * tv + cua[3 * n] * Dn;
          e1 += cud[3 * n + 1] * tv + cua[3 * n + 1] * Dn;
          e2 += cud[3 * n + 2] * tv + cua[3 * n + 2] * Dn;
          R0 += cud[3 * n] * Dn + cuE[3 * n] * Tn + cua[3 * n] * En;
          R1 += cud[3 * n + 1] * Dn + cuE[3 * n + 1] * Tn + cua[3 * n + 1] * En;
          R2 += cud[3 * n + 2] * Dn + cuE[3 * n + 2] * Tn + cua[3 * n + 2] * En;
        }
        d0 = -e0; d1 = -e1; d2 = -e2;
        ndn = -(nx0 * R0 + nx1 * R1 + nx2 * R2);
      }
      double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      for (int s = 0; s < 2; ++s) {
        double fr = 0, fi = 0, dr = 0, di = 0;
        if (r > 0.0) {
          double sn, cs;
          sincos(kk[s] * r, &sn, &cs);
          double g = wt / (4.0 * kPi * r);
          fr = g * cs;
          fi = g * sn;
          double nd = ndn / (r * r);
          // (i k r - 1) * (fr + i fi) * nd
          dr = nd * (-fr - kk[s] * r * fi);
          di = nd * (-fi + kk[s] * r * fr);
        }
        f[((size_t)s * nb + j) * 2] = fr;
        f[((size_t)s * nb + j) * 2 + 1] = fi;
        f[((size_t)(2 + s) * nb + j) * 2] = dr;
        f[((size_t)(2 + s) * nb + j) * 2 + 1] = di;
      }
    }
    __syncwarp();
    // tmp[s][j'] = sum_j f[s][j] Lv[j][j']
    for (int t = lane; t < 4 * nc; t += 32) {
      int s = t / nc, jp = t % nc;
      double ar = 0, ai = 0;
      for (int j = 0; j < nb; ++j) {
        double L = Lv[j * nc + jp];
        ar += f[((size_t)s * nb + j) * 2] * L;
        ai += f[((size_t)s * nb + j) * 2 + 1] * L;
      }
      tmp[2 * t] = ar;
      tmp[2 * t + 1] = ai;
    }
    __syncwarp();
    // W[s][i'][j'] += Lu[i'] tmp[s][j']
    for (int t = lane; t < 4 * npp; t += 32) {
      int s = t / npp, r2 = t % npp, ip = r2 / nc, jp = r2 % nc;
      Wacc[2 * t] += Lu[ip] * tmp[2 * (s * nc + jp)];
      Wacc[2 * t + 1] += Lu[ip] * tmp[2 * (s * nc + jp) + 1];
    }
    __syncwarp();
  }
  double* out = W + (size_t)sp * 8 * npp;
  for (int t = lane; t < 8 * npp; t += 32) out[t] = Wacc[t];
}

size_t moments_smem_per_warp(int nc, int ng, int nbeta) {
  int npp = nc * nc;
  return sizeof(double) * (6 * (size_t)nbeta + (size_t)ng * 9 + 8 * (size_t)nbeta + (size_t)nbeta * nc +
                           8 * (size_t)nc + (size_t)nc + 8 * (size_t)npp + 9 * (size_t)ng);
}

// ---------------------------------------------------------------- near-field matrix values
// Either output may be null (the plan keeps the values in its own precision only).
// Row l (Sec. III-H, reading R12): for columns on singular patches the
// singular weight minus the plain Fejer term wherever the far algorithm also
// counts the pair (column outside the neighbour boxes of x_l); for neighbour
// points on regular patches the plain Fejer term.
__global__ void k_near_values(int N, int nc, const int64_t* row_ptr, const int* col, const int* pair,
                              const int* sp_of_pair, const double* W, const double* x,
                              const double* nrm, const double* qw, const int* leafc, double ke,
                              double ki, double* val64, float* val32) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
  if (warp >= N) return;
  const int l = warp, npp = nc * nc;
  const double x0 = x[3 * (size_t)l], x1 = x[3 * (size_t)l + 1], x2 = x[3 * (size_t)l + 2];
  const double n0 = nrm[3 * (size_t)l], n1 = nrm[3 * (size_t)l + 1], n2 = nrm[3 * (size_t)l + 2];
  const int c0 = leafc[3 * l], c1 = leafc[3 * l + 1], c2 = leafc[3 * l + 2];
  const double kk[2] = {ke, ki};
  for (int64_t e = row_ptr[l] + lane; e < row_ptr[l + 1]; e += 32) {
    const int m = col[e];
    const int pr = pair[e];
    bool inU = abs(leafc[3 * m] - c0) <= 1 && abs(leafc[3 * m + 1] - c1) <= 1 && abs(leafc[3 * m + 2] - c2) <= 1;
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    bool fejer = (pr < 0) || !inU;
    if (fejer) {
      double d0 = x0 - x[3 * (size_t)m], d1 = x1 - x[3 * (size_t)m + 1], d2 = x2 - x[3 * (size_t)m + 2];
      double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      double nd = (n0 * d0 + n1 * d1 + n2 * d2) / (r * r);
      double sgn = (pr < 0) ? 1.0 : -1.0;
      for (int s = 0; s < 2; ++s) {
        double sn, cs;
        sincos(kk[s] * r, &sn, &cs);
        double g = sgn * qw[m] / (4.0 * kPi * r);
        double fr = g * cs, fi = g * sn;
        v[2 * s] = fr;
        v[2 * s + 1] = fi;
        v[4 + 2 * s] = nd * (-fr - kk[s] * r * fi);
        v[4 + 2 * s + 1] = nd * (-fi + kk[s] * r * fr);
      }
    }
    if (pr >= 0) {
      const double* w = W + (size_t)sp_of_pair[pr] * 8 * npp;
      int lm = m % npp;
      for (int s = 0; s < 4; ++s) {
        v[2 * s] += w[2 * (s * npp + lm)];
        v[2 * s + 1] += w[2 * (s * npp + lm) + 1];
      }
    }
    for (int t = 0; t < 8; ++t) {
      if (val64) val64[8 * e + t] = v[t];
      if (val32) val32[8 * e + t] = (float)v[t];
    }
  }
}

}  // namespace ifgf
