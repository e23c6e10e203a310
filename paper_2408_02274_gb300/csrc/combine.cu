// Density preparation (step a0) and the N-Mueller combination (step c-post), FP64.
//
// a0: the tangential densities y = (m.t1, m.t2, j.t1, j.t2) become the eight
// scalar densities of Sec. III (first paragraph): Cartesian m, j and their
// surface divergences, div = J^{-1} [(J V^u)_u + (J V^v)_v] with per-patch
// Chebyshev differentiation (the "Chebyshev recurrence relations" of Sec. III).
// c-post: the vector operators R, K, T (Eqs. potential_r, potential_k,
// potential_t) are rebuilt from S and D = dS/dn at the nodes:
//   K_s[V] = sum_c n_c grad_G S_s[V_c] - P_T D_s[V],  R_s[V] = n x S_s[V],
//   T_s[V] = n x grad_G S_s[div_G V]      (reading R6)
// and combined into the two rows of Eq. n_muller with Eqs. k_delta, r_delta,
// t_delta, projected on (t1, t2).
#include "kernels.h"

namespace ifgf {

namespace {

struct c64 {
  double r, i;
};
__device__ inline c64 operator+(c64 a, c64 b) { return {a.r + b.r, a.i + b.i}; }
__device__ inline c64 operator-(c64 a, c64 b) { return {a.r - b.r, a.i - b.i}; }
__device__ inline c64 operator*(double s, c64 a) { return {s * a.r, s * a.i}; }
__device__ inline c64 mul_i(c64 a) { return {-a.i, a.r}; }   // i * a

struct cv3 {
  c64 v[3];
};
__device__ inline cv3 cross_rn(const double* n, const cv3& a) {   // n x a (n real)
  cv3 r;
  r.v[0] = n[1] * a.v[2] - n[2] * a.v[1];
  r.v[1] = n[2] * a.v[0] - n[0] * a.v[2];
  r.v[2] = n[0] * a.v[1] - n[1] * a.v[0];
  return r;
}
__device__ inline c64 operator*(c64 a, double s) { return {s * a.r, s * a.i}; }

// T: storage of the densities phi and weighted densities a (original order); TS: the weighted
// densities in octree order, read by the IFGF kernels (FP32 in the mixed-precision plan).
template <typename T, typename TS = T>
__global__ void k_density_prep(int nc, const double* __restrict__ y, NodeGeom g,
                               const double* __restrict__ Dm, const int* __restrict__ iperm,
                               int N, T* __restrict__ phi, TS* __restrict__ a_sorted,
                               T* __restrict__ a_orig, double* __restrict__ phi64) {
  extern __shared__ double sm[];
  const int npp = nc * nc;
  double* JV = sm;   // [4][npp][2]: J m^u, J m^v, J j^u, J j^v
  const size_t rb = blockIdx.y;   // right-hand side of a batched call
  y += rb * 8 * (size_t)N;
  phi += rb * 16 * (size_t)N;
  a_sorted += rb * 16 * (size_t)N;
  a_orig += rb * 16 * (size_t)N;
  phi64 += rb * 16 * (size_t)N;
  const int p = blockIdx.x, t = threadIdx.x;
  const int l = p * npp + t;
  double vals[16];
  if (t < npp) {
    const double* t1 = g.t1 + 3 * (size_t)l;
    const double* t2 = g.t2 + 3 * (size_t)l;
    const double* xu = g.xu + 3 * (size_t)l;
    const double* xv = g.xv + 3 * (size_t)l;
    const double J = g.J[l], guu = g.g[3 * l], guv = g.g[3 * l + 1], gvv = g.g[3 * l + 2];
    for (int q = 0; q < 2; ++q) {       // q = 0: m, q = 1: j
      double ar = y[2 * ((size_t)(2 * q) * N + l)], ai = y[2 * ((size_t)(2 * q) * N + l) + 1];
      double br = y[2 * ((size_t)(2 * q + 1) * N + l)], bi = y[2 * ((size_t)(2 * q + 1) * N + l) + 1];
      double Vr[3], Vi[3];
      for (int c = 0; c < 3; ++c) {
        Vr[c] = ar * t1[c] + br * t2[c];
        Vi[c] = ai * t1[c] + bi * t2[c];
        vals[2 * (3 * q + c)] = Vr[c];
        vals[2 * (3 * q + c) + 1] = Vi[c];
      }
      double pur = Vr[0] * xu[0] + Vr[1] * xu[1] + Vr[2] * xu[2];
      double pui = Vi[0] * xu[0] + Vi[1] * xu[1] + Vi[2] * xu[2];
      double pvr = Vr[0] * xv[0] + Vr[1] * xv[1] + Vr[2] * xv[2];
      double pvi = Vi[0] * xv[0] + Vi[1] * xv[1] + Vi[2] * xv[2];
      JV[2 * ((2 * q) * npp + t)] = J * (guu * pur + guv * pvr);
      JV[2 * ((2 * q) * npp + t) + 1] = J * (guu * pui + guv * pvi);
      JV[2 * ((2 * q + 1) * npp + t)] = J * (guv * pur + gvv * pvr);
      JV[2 * ((2 * q + 1) * npp + t) + 1] = J * (guv * pui + gvv * pvi);
    }
  }
  __syncthreads();
  if (t >= npp) return;
  const int i = t / nc, j = t % nc;
  const double J = g.J[l];
  for (int q = 0; q < 2; ++q) {
    double dr = 0, di = 0;
    for (int k = 0; k < nc; ++k) {
      double a = Dm[i * nc + k], b = Dm[j * nc + k];
      dr += a * JV[2 * ((2 * q) * npp + k * nc + j)] + b * JV[2 * ((2 * q + 1) * npp + i * nc + k)];
      di += a * JV[2 * ((2 * q) * npp + k * nc + j) + 1] + b * JV[2 * ((2 * q + 1) * npp + i * nc + k) + 1];
    }
    vals[2 * (6 + q)] = dr / J;
    vals[2 * (6 + q) + 1] = di / J;
  }
  const double w = g.w[l];
  const int ls = iperm[l];
  for (int k = 0; k < 16; ++k) {
    phi[16 * (size_t)l + k] = (T)vals[k];
    phi64[16 * (size_t)l + k] = vals[k];
    a_orig[16 * (size_t)l + k] = (T)(vals[k] * w);
    a_sorted[16 * (size_t)ls + k] = (TS)(vals[k] * w);
  }
}

// Raw densities given by the caller (fields entry point): convert and weight.
template <typename T, typename TS = T>
__global__ void k_phi_input(int N, const double* __restrict__ phi_in, const double* __restrict__ w,
                            const int* __restrict__ iperm, T* phi, TS* a_sorted, T* a_orig,
                            double* phi64) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 16 * N) return;
  int l = t / 16, k = t % 16;
  double v = phi_in[t];
  phi[t] = (T)v;
  phi64[t] = v;
  a_orig[t] = (T)(v * w[l]);
  a_sorted[16 * (size_t)iperm[l] + k] = (TS)(v * w[l]);
}

template <typename T>
__global__ void k_combine(int nc, int N, const T* __restrict__ f28, const double* __restrict__ y,
                          NodeGeom g, const double* __restrict__ Dm, Materials M,
                          double* __restrict__ out) {
  extern __shared__ double sm[];
  const int npp = nc * nc;
  double* S = sm;   // [16][npp][2] the S fields of this patch
  const size_t rb = blockIdx.y;   // right-hand side of a batched call
  f28 += rb * 56 * (size_t)N;
  y += rb * 8 * (size_t)N;
  out += rb * 8 * (size_t)N;
  const int p = blockIdx.x, t = threadIdx.x;
  const int l = p * npp + t;
  for (int e = t; e < 16 * npp; e += blockDim.x) {
    int k = e / npp, q = e % npp;
    S[2 * e] = (double)f28[56 * ((size_t)p * npp + q) + 2 * k];
    S[2 * e + 1] = (double)f28[56 * ((size_t)p * npp + q) + 2 * k + 1];
  }
  __syncthreads();
  if (t >= npp) return;
  const int i = t / nc, j = t % nc;
  const double* xu = g.xu + 3 * (size_t)l;
  const double* xv = g.xv + 3 * (size_t)l;
  const double* n = g.n + 3 * (size_t)l;
  const double* t1 = g.t1 + 3 * (size_t)l;
  const double* t2 = g.t2 + 3 * (size_t)l;
  const double guu = g.g[3 * l], guv = g.g[3 * l + 1], gvv = g.g[3 * l + 2];
  // tangential densities at this node
  cv3 mv, jv;
  for (int c = 0; c < 3; ++c) {
    mv.v[c] = c64{y[2 * l] * t1[c] + y[2 * ((size_t)N + l)] * t2[c],
                  y[2 * l + 1] * t1[c] + y[2 * ((size_t)N + l) + 1] * t2[c]};
    jv.v[c] = c64{y[2 * (2 * (size_t)N + l)] * t1[c] + y[2 * (3 * (size_t)N + l)] * t2[c],
                  y[2 * (2 * (size_t)N + l) + 1] * t1[c] + y[2 * (3 * (size_t)N + l) + 1] * t2[c]};
  }
  const double kk[2] = {M.ke, M.ki};
  const double mu[2] = {M.mu_e, M.mu_i}, ep[2] = {M.eps_e, M.eps_i};
  cv3 row1, row2, RTm, RTj;
  for (int c = 0; c < 3; ++c) {
    row1.v[c] = 0.5 * (M.mu_e + M.mu_i) * mv.v[c];
    row2.v[c] = 0.5 * (M.eps_e + M.eps_i) * jv.v[c];
    RTm.v[c] = c64{0, 0};
    RTj.v[c] = c64{0, 0};
  }
  for (int s = 0; s < 2; ++s) {
    const double sg = (s == 0) ? 1.0 : -1.0;
    cv3 grad[8];
    for (int k = 0; k < 8; ++k) {
      const double* Sk = S + 2 * (size_t)(8 * s + k) * npp;
      double fur = 0, fui = 0, fvr = 0, fvi = 0;
      for (int q = 0; q < nc; ++q) {
        double a = Dm[i * nc + q], b = Dm[j * nc + q];
        fur += a * Sk[2 * (q * nc + j)];
        fui += a * Sk[2 * (q * nc + j) + 1];
        fvr += b * Sk[2 * (i * nc + q)];
        fvi += b * Sk[2 * (i * nc + q) + 1];
      }
      double cur = guu * fur + guv * fvr, cui = guu * fui + guv * fvi;
      double cvr = guv * fur + gvv * fvr, cvi = guv * fui + gvv * fvi;
      for (int c = 0; c < 3; ++c) grad[k].v[c] = c64{cur * xu[c] + cvr * xv[c], cui * xu[c] + cvi * xv[c]};
    }
    // D fields of this kernel (Cartesian m then j), tangential projection
    cv3 Dm3, Dj3;
    const T* fd = f28 + 56 * (size_t)l + 2 * (16 + 6 * s);
    for (int c = 0; c < 3; ++c) {
      Dm3.v[c] = c64{(double)fd[2 * c], (double)fd[2 * c + 1]};
      Dj3.v[c] = c64{(double)fd[2 * (3 + c)], (double)fd[2 * (3 + c) + 1]};
    }
    c64 dmn = Dm3.v[0] * n[0] + Dm3.v[1] * n[1] + Dm3.v[2] * n[2];
    c64 djn = Dj3.v[0] * n[0] + Dj3.v[1] * n[1] + Dj3.v[2] * n[2];
    cv3 Km, Kj, Sm, Sj;
    for (int c = 0; c < 3; ++c) {
      Km.v[c] = n[0] * grad[0].v[c] + n[1] * grad[1].v[c] + n[2] * grad[2].v[c] - (Dm3.v[c] - n[c] * dmn);
      Kj.v[c] = n[0] * grad[3].v[c] + n[1] * grad[4].v[c] + n[2] * grad[5].v[c] - (Dj3.v[c] - n[c] * djn);
      const double* fs = S + 2 * (size_t)(8 * s) * npp;
      Sm.v[c] = c64{fs[2 * (c * npp + t)], fs[2 * (c * npp + t) + 1]};
      Sj.v[c] = c64{fs[2 * ((3 + c) * npp + t)], fs[2 * ((3 + c) * npp + t) + 1]};
    }
    cv3 Rm = cross_rn(n, Sm), Rj = cross_rn(n, Sj);
    cv3 Tm = cross_rn(n, grad[6]), Tj = cross_rn(n, grad[7]);
    for (int c = 0; c < 3; ++c) {
      row1.v[c] = row1.v[c] + (sg * mu[s]) * Km.v[c];
      row2.v[c] = row2.v[c] + (sg * ep[s]) * Kj.v[c];
      RTj.v[c] = RTj.v[c] + sg * ((kk[s] * kk[s]) * Rj.v[c] + Tj.v[c]);
      RTm.v[c] = RTm.v[c] + sg * ((kk[s] * kk[s]) * Rm.v[c] + Tm.v[c]);
    }
  }
  const double iw = 1.0 / M.omega;
  for (int c = 0; c < 3; ++c) {
    row1.v[c] = row1.v[c] + iw * mul_i(RTj.v[c]);        // + (i/omega) (R^D-like sum) j
    row2.v[c] = row2.v[c] - iw * mul_i(RTm.v[c]);        // + (-i/omega) (...) m
  }
  c64 o[4];
  o[0] = row1.v[0] * t1[0] + row1.v[1] * t1[1] + row1.v[2] * t1[2];
  o[1] = row1.v[0] * t2[0] + row1.v[1] * t2[1] + row1.v[2] * t2[2];
  o[2] = row2.v[0] * t1[0] + row2.v[1] * t1[1] + row2.v[2] * t1[2];
  o[3] = row2.v[0] * t2[0] + row2.v[1] * t2[1] + row2.v[2] * t2[2];
  for (int q = 0; q < 4; ++q) {
    out[2 * ((size_t)q * N + l)] = o[q].r;
    out[2 * ((size_t)q * N + l) + 1] = o[q].i;
  }
}

template <typename T>
__global__ void k_zero(size_t n, T* a) {
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t < n) a[t] = T(0);
}

template <typename T>
__global__ void k_export(size_t n, const T* a, double* b) {
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t < n) b[t] = (double)a[t];
}

}  // namespace

cudaError_t launch_density_prep(const ifgf_plan_t* p, const double* y, const double* phi_in,
                                cudaStream_t s, int nrhs) {
  const int npp = p->nc * p->nc;
  const int* iperm = p->perm + p->N;   // second half of the perm buffer holds original -> sorted
  const int prec = p->desc.precision;
  if (phi_in) {
    int nt = 16 * p->N;
    if (prec == IFGF_FP64)
      k_phi_input<double><<<(nt + 255) / 256, 256, 0, s>>>(p->N, phi_in, p->geo.w, iperm,
          (double*)p->phi, (double*)p->a_sorted, (double*)p->a_orig, p->phi64);
    else if (prec == IFGF_MIXED)
      k_phi_input<double, float><<<(nt + 255) / 256, 256, 0, s>>>(p->N, phi_in, p->geo.w, iperm,
          (double*)p->phi, (float*)p->a_sorted, (double*)p->a_orig, p->phi64);
    else
      k_phi_input<float><<<(nt + 255) / 256, 256, 0, s>>>(p->N, phi_in, p->geo.w, iperm,
          (float*)p->phi, (float*)p->a_sorted, (float*)p->a_orig, p->phi64);
    return cudaGetLastError();
  }
  size_t smem = sizeof(double) * 8 * npp;
  int threads = ((npp + 31) / 32) * 32;
  if (prec == IFGF_FP64)
    k_density_prep<double><<<dim3(p->P, nrhs), threads, smem, s>>>(p->nc, y, p->geo, p->tab_D, iperm, p->N,
        (double*)p->phi, (double*)p->a_sorted, (double*)p->a_orig, p->phi64);
  else if (prec == IFGF_MIXED)
    k_density_prep<double, float><<<dim3(p->P, nrhs), threads, smem, s>>>(p->nc, y, p->geo, p->tab_D, iperm,
        p->N, (double*)p->phi, (float*)p->a_sorted, (double*)p->a_orig, p->phi64);
  else
    k_density_prep<float><<<dim3(p->P, nrhs), threads, smem, s>>>(p->nc, y, p->geo, p->tab_D, iperm, p->N,
        (float*)p->phi, (float*)p->a_sorted, (float*)p->a_orig, p->phi64);
  return cudaGetLastError();
}

// Opt the patch-wise kernels into the dynamic shared memory their largest
// patch (nc = 24) needs: k_combine keeps 16 complex FP64 fields per node.
cudaError_t setup_combine_kernels() {
  const int smax = (int)(sizeof(double) * 32 * 24 * 24);
  cudaError_t e = cudaFuncSetAttribute(k_combine<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_combine<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  return e;
}

cudaError_t launch_combine(const ifgf_plan_t* p, const double* y, double* out, cudaStream_t s, int nrhs) {
  const int npp = p->nc * p->nc;
  size_t smem = sizeof(double) * 32 * npp;
  int threads = ((npp + 31) / 32) * 32;
  Materials M{p->desc.k_ext, p->desc.k_int, p->desc.eps_ext, p->desc.eps_int,
              p->desc.mu_ext, p->desc.mu_int, p->omega};
  if (store64(p->desc))
    k_combine<double><<<dim3(p->P, nrhs), threads, smem, s>>>(p->nc, p->N, (const double*)p->f28, y, p->geo,
                                                    p->tab_D, M, out);
  else
    k_combine<float><<<dim3(p->P, nrhs), threads, smem, s>>>(p->nc, p->N, (const float*)p->f28, y, p->geo,
                                                   p->tab_D, M, out);
  return cudaGetLastError();
}

__global__ void k_block_scale(size_t n, size_t N, double cm, double cj, const double* in,
                              double* out) {   // in == out allowed: each entry is read then written by one thread
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;   // complex entry
  if (i >= n) return;
  const double c = ((i / N) & 3) < 2 ? cm : cj;
  out[2 * i] = c * in[2 * i];
  out[2 * i + 1] = c * in[2 * i + 1];
}

cudaError_t launch_block_scale(int N, int nrhs, double cm, double cj, const double* in, double* out,
                               cudaStream_t s) {
  const size_t n = 4 * (size_t)N * nrhs;
  k_block_scale<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, (size_t)N, cm, cj, in, out);
  return cudaGetLastError();
}

cudaError_t launch_zero_f28(const ifgf_plan_t* p, cudaStream_t s) {
  size_t n = (size_t)p->N * 56;
  if (store64(p->desc))
    k_zero<double><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, (double*)p->f28);
  else
    k_zero<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, (float*)p->f28);
  return cudaGetLastError();
}

cudaError_t launch_f28_export(const ifgf_plan_t* p, double* out, cudaStream_t s) {
  size_t n = (size_t)p->N * 56;
  if (store64(p->desc))
    k_export<double><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, (const double*)p->f28, out);
  else
    k_export<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, (const float*)p->f28, out);
  return cudaGetLastError();
}

}  // namespace ifgf
