// (e) Device GMRES for A y = b (Eq. lin_system), FP64 Arnoldi with classical
// Gram-Schmidt applied twice, Givens rotations on the device, y0 = 0, no
// restart.  The right-hand side is omega^{-1}(n x E^inc, n x H^inc) projected
// on (t1, t2) (right side of Eq. n_muller).
#include "gmres.h"

namespace ifgf {

namespace {

constexpr int kDotThreads = 256;
constexpr int kDotItems = 4;

__global__ void k_rhs(int N, const double* __restrict__ inc, NodeGeom g, double iw, double* __restrict__ b) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= N) return;
  const double* n = g.n + 3 * (size_t)l;
  const double* t1 = g.t1 + 3 * (size_t)l;
  const double* t2 = g.t2 + 3 * (size_t)l;
  for (int f = 0; f < 2; ++f) {          // f = 0: E, f = 1: H
    double vr[3], vi[3];
    for (int c = 0; c < 3; ++c) {
      vr[c] = inc[2 * ((size_t)(3 * f + c) * N + l)];
      vi[c] = inc[2 * ((size_t)(3 * f + c) * N + l) + 1];
    }
    double cr[3] = {n[1] * vr[2] - n[2] * vr[1], n[2] * vr[0] - n[0] * vr[2], n[0] * vr[1] - n[1] * vr[0]};
    double ci[3] = {n[1] * vi[2] - n[2] * vi[1], n[2] * vi[0] - n[0] * vi[2], n[0] * vi[1] - n[1] * vi[0]};
    double p1r = cr[0] * t1[0] + cr[1] * t1[1] + cr[2] * t1[2];
    double p1i = ci[0] * t1[0] + ci[1] * t1[1] + ci[2] * t1[2];
    double p2r = cr[0] * t2[0] + cr[1] * t2[1] + cr[2] * t2[2];
    double p2i = ci[0] * t2[0] + ci[1] * t2[1] + ci[2] * t2[2];
    b[2 * ((size_t)(2 * f) * N + l)] = iw * p1r;
    b[2 * ((size_t)(2 * f) * N + l) + 1] = iw * p1i;
    b[2 * ((size_t)(2 * f + 1) * N + l)] = iw * p2r;
    b[2 * ((size_t)(2 * f + 1) * N + l) + 1] = iw * p2i;
  }
}

// part[chunk][j] = sum over the chunk of conj(V_j) w for j = 0..k1-1 (complex).  Grid:
// (chunks of kDotThreads * kDotItems elements) x (groups of kDotJ vectors); w is read once
// per block and the kDotJ sums are reduced together.
constexpr int kDotJ = 8;
__global__ void __launch_bounds__(kDotThreads) k_dots(int64_t n, int k1, const double* __restrict__ V,
                                                      const double* __restrict__ w, double* __restrict__ part) {
  __shared__ double red[kDotThreads / 32][2 * kDotJ];
  const int64_t base = (int64_t)blockIdx.x * kDotThreads * kDotItems;
  const int j0 = blockIdx.y * kDotJ;
  double wr[kDotItems], wi[kDotItems];
  int64_t idx[kDotItems];
#pragma unroll
  for (int it = 0; it < kDotItems; ++it) {
    idx[it] = base + it * kDotThreads + threadIdx.x;
    wr[it] = idx[it] < n ? w[2 * idx[it]] : 0.0;
    wi[it] = idx[it] < n ? w[2 * idx[it] + 1] : 0.0;
  }
  double acc[2 * kDotJ];
#pragma unroll
  for (int jj = 0; jj < kDotJ; ++jj) {
    double ar = 0, ai = 0;
    const int j = j0 + jj;
    if (j < k1) {
      const double* v = V + 2 * (size_t)j * n;
#pragma unroll
      for (int it = 0; it < kDotItems; ++it)
        if (idx[it] < n) {
          const double vr = v[2 * idx[it]], vi = v[2 * idx[it] + 1];
          ar += vr * wr[it] + vi * wi[it];
          ai += vr * wi[it] - vi * wr[it];
        }
    }
    acc[2 * jj] = ar;
    acc[2 * jj + 1] = ai;
  }
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll
  for (int q = 0; q < 2 * kDotJ; ++q)
    for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 2 * kDotJ; ++q) red[warp][q] = acc[q];
  __syncthreads();
  if (threadIdx.x < 2 * kDotJ) {
    const int q = threadIdx.x, j = j0 + q / 2;
    if (j < k1) {
      double sum = 0;
      for (int ww = 0; ww < kDotThreads / 32; ++ww) sum += red[ww][q];
      part[2 * ((size_t)blockIdx.x * k1 + j) + (q & 1)] = sum;
    }
  }
}

// h[j] (+)= sum_blk part[blk][j]
__global__ void k_reduce_parts(int nblk, int k1, const double* __restrict__ part, double* __restrict__ h,
                               int accumulate) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k1) return;
  double sr = 0, si = 0;
  for (int b = 0; b < nblk; ++b) {
    sr += part[2 * ((size_t)b * k1 + j)];
    si += part[2 * ((size_t)b * k1 + j) + 1];
  }
  if (accumulate) {
    h[2 * j] += sr;
    h[2 * j + 1] += si;
  } else {
    h[2 * j] = sr;
    h[2 * j + 1] = si;
  }
}

// w -= sum_j V_j c_j (sign = -1) or y = sum_j V_j c_j (sign = +1, overwrite)
__global__ void k_combo(int64_t n, int k1, const double* __restrict__ V, const double* __restrict__ c,
                        double* __restrict__ w, int overwrite) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double ar = 0, ai = 0;
  for (int j = 0; j < k1; ++j) {
    double vr = V[2 * ((size_t)j * n + i)], vi = V[2 * ((size_t)j * n + i) + 1];
    double cr = c[2 * j], ci = c[2 * j + 1];
    ar += vr * cr - vi * ci;
    ai += vr * ci + vi * cr;
  }
  if (overwrite) {
    w[2 * i] = ar;
    w[2 * i + 1] = ai;
  } else {
    w[2 * i] -= ar;
    w[2 * i + 1] -= ai;
  }
}

__global__ void k_scale_copy(int64_t n, const double* __restrict__ src, const double* __restrict__ sc,
                             int inv, double* __restrict__ dst) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double f = inv ? (sc[0] != 0.0 ? 1.0 / sc[0] : 0.0) : sc[0];
  dst[2 * i] = src[2 * i] * f;
  dst[2 * i + 1] = src[2 * i + 1] * f;
}

// |w|^2 partials (reuses the dot kernel with V = w) -> scal[0] = |w|
__global__ void k_norm_final(int nblk, const double* __restrict__ part, double* __restrict__ out) {
  double s = 0;
  for (int b = 0; b < nblk; ++b) s += part[2 * (size_t)b];
  out[0] = sqrt(s);
}

// Arnoldi column k: Hcol[0..k] = h, Hcol[k+1] = beta; apply the previous
// rotations, form the new one, update g; res[0] = |g_{k+1}| / |b|.
__global__ void k_givens(int k, int ldh, double* __restrict__ H, const double* __restrict__ h,
                         const double* __restrict__ beta, double* __restrict__ cs, double* __restrict__ sn,
                         double* __restrict__ g, const double* __restrict__ bnorm, double* __restrict__ res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* col = H + 2 * (size_t)k * ldh;   // column k, rows 0..k+1
  for (int i = 0; i <= k; ++i) {
    col[2 * i] = h[2 * i];
    col[2 * i + 1] = h[2 * i + 1];
  }
  col[2 * (k + 1)] = beta[0];
  col[2 * (k + 1) + 1] = 0.0;
  for (int i = 0; i < k; ++i) {
    // [a; b] <- [conj(c) conj(s); -s c] [a; b]
    double ar = col[2 * i], ai = col[2 * i + 1], br = col[2 * (i + 1)], bi = col[2 * (i + 1) + 1];
    double cr = cs[2 * i], ci = cs[2 * i + 1], sr = sn[2 * i], si = sn[2 * i + 1];
    double tr = (cr * ar + ci * ai) + (sr * br + si * bi);
    double ti = (cr * ai - ci * ar) + (sr * bi - si * br);
    double ur = -(sr * ar - si * ai) + (cr * br - ci * bi);
    double ui = -(sr * ai + si * ar) + (cr * bi + ci * br);
    col[2 * i] = tr;
    col[2 * i + 1] = ti;
    col[2 * (i + 1)] = ur;
    col[2 * (i + 1) + 1] = ui;
  }
  double ar = col[2 * k], ai = col[2 * k + 1], br = col[2 * (k + 1)], bi = col[2 * (k + 1) + 1];
  double den = sqrt(ar * ar + ai * ai + br * br + bi * bi);
  double cr = 1, ci = 0, sr = 0, si = 0;
  if (den > 0) {
    cr = ar / den; ci = ai / den; sr = br / den; si = bi / den;
  }
  cs[2 * k] = cr; cs[2 * k + 1] = ci;
  sn[2 * k] = sr; sn[2 * k + 1] = si;
  col[2 * k] = (cr * ar + ci * ai) + (sr * br + si * bi);
  col[2 * k + 1] = (cr * ai - ci * ar) + (sr * bi - si * br);
  col[2 * (k + 1)] = 0;
  col[2 * (k + 1) + 1] = 0;
  double gr = g[2 * k], gi = g[2 * k + 1];
  g[2 * (k + 1)] = -(sr * gr - si * gi);
  g[2 * (k + 1) + 1] = -(sr * gi + si * gr);
  g[2 * k] = cr * gr + ci * gi;
  g[2 * k + 1] = cr * gi - ci * gr;
  res[0] = sqrt(g[2 * (k + 1)] * g[2 * (k + 1)] + g[2 * (k + 1) + 1] * g[2 * (k + 1) + 1]) / bnorm[0];
}

__global__ void k_init_g(const double* __restrict__ bnorm, double* __restrict__ g, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 2 * n) g[i] = 0;
  if (i == 0) g[0] = bnorm[0];
}

// back substitution R z = g[0..k-1] (R upper triangular in H), z into c
__global__ void k_backsub(int k, int ldh, const double* __restrict__ H, const double* __restrict__ g,
                          double* __restrict__ z) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double sr = g[2 * i], si = g[2 * i + 1];
    for (int j = i + 1; j < k; ++j) {
      double hr = H[2 * ((size_t)j * ldh + i)], hi = H[2 * ((size_t)j * ldh + i) + 1];
      sr -= hr * z[2 * j] - hi * z[2 * j + 1];
      si -= hr * z[2 * j + 1] + hi * z[2 * j];
    }
    double dr = H[2 * ((size_t)i * ldh + i)], di = H[2 * ((size_t)i * ldh + i) + 1];
    double den = dr * dr + di * di;
    z[2 * i] = (sr * dr + si * di) / den;
    z[2 * i + 1] = (si * dr - sr * di) / den;
  }
}

}  // namespace

cudaError_t launch_rhs(const ifgf_plan_t* p, const double* inc, double* b, cudaStream_t s) {
  k_rhs<<<(p->N + 127) / 128, 128, 0, s>>>(p->N, inc, p->geo, 1.0 / p->omega, b);
  return cudaGetLastError();
}

int dots_blocks(int64_t n) { return (int)((n + kDotThreads * kDotItems - 1) / (kDotThreads * kDotItems)); }

// Gram-Schmidt projection h (+)= V[0..k1)^H w and w -= V h_pass.
static cudaError_t project(GmresWork& G, int64_t n, int k1, double* hpass, double* htot, int first,
                           cudaStream_t s) {
  int nb = dots_blocks(n);
  k_dots<<<dim3(nb, (k1 + kDotJ - 1) / kDotJ), kDotThreads, 0, s>>>(n, k1, G.V, G.w, G.part);
  k_reduce_parts<<<(k1 + 127) / 128, 128, 0, s>>>(nb, k1, G.part, hpass, 0);
  k_combo<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, k1, G.V, hpass, G.w, 0);
  k_reduce_parts<<<(k1 + 127) / 128, 128, 0, s>>>(nb, k1, G.part, htot, first ? 0 : 1);
  return cudaGetLastError();
}

cudaError_t gmres_run(ifgf_plan_t* p, const MatvecFn& matvec, double tol, int max_iter, int* iters,
                      double* relres, cudaStream_t s) {
  GmresWork& G = p->gm;
  const int64_t n = 4 * (int64_t)p->N;
  const int ldh = G.max_iter + 1;
  const int nb = dots_blocks(n);
  cudaError_t err;
  // |b|
  k_dots<<<nb, kDotThreads, 0, s>>>(n, 1, G.b, G.b, G.part);
  k_norm_final<<<1, 1, 0, s>>>(nb, G.part, G.scal + 0);          // scal[0] = |b|
  k_init_g<<<(2 * (G.max_iter + 1) + 127) / 128, 128, 0, s>>>(G.scal + 0, G.g, G.max_iter + 1);
  k_scale_copy<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, G.b, G.scal + 0, 1, G.V);   // v0 = b/|b|
  p->launches += 4;
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if ((err = cudaMemcpyAsync(G.hres, G.scal, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return err;
  if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return err;
  const double bnorm = G.hres[0];
  int k = 0;
  double res = 1.0;
  if (bnorm == 0.0) {
    cudaMemsetAsync(G.y, 0, sizeof(double) * 2 * n, s);
    *iters = 0;
    *relres = 0.0;
    return cudaGetLastError();
  }
  for (k = 0; k < max_iter; ++k) {
    double* vk = G.V + 2 * (size_t)k * n;
    if ((err = matvec(vk, G.w, s)) != cudaSuccess) return err;
    const int rec = timer_begin(p, TK_GMRES, s);
    // CGS2: two projection passes, h = h1 + h2
    if ((err = project(G, n, k + 1, G.h + 2 * (size_t)(G.max_iter + 1), G.h, 1, s)) != cudaSuccess) return err;
    if ((err = project(G, n, k + 1, G.h + 2 * (size_t)(G.max_iter + 1), G.h, 0, s)) != cudaSuccess) return err;
    k_dots<<<nb, kDotThreads, 0, s>>>(n, 1, G.w, G.w, G.part);
    k_norm_final<<<1, 1, 0, s>>>(nb, G.part, G.scal + 1);         // scal[1] = beta
    k_givens<<<1, 1, 0, s>>>(k, ldh, G.H, G.h, G.scal + 1, G.cs, G.sn, G.g, G.scal + 0, G.scal + 2);
    k_scale_copy<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, G.w, G.scal + 1, 1, G.V + 2 * (size_t)(k + 1) * n);
    timer_end(p, rec, s);
    p->launches += 12;   // 2 x (dots, reduce, combo, reduce), dots, norm, givens, scale
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if ((err = cudaMemcpyAsync(G.hres, G.scal + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return err;
    if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return err;
    res = G.hres[1];
    if (res <= tol || G.hres[0] == 0.0) {
      ++k;
      break;
    }
  }
  if (k > max_iter) k = max_iter;
  k_backsub<<<1, 1, 0, s>>>(k, ldh, G.H, G.g, G.h);
  k_combo<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, k, G.V, G.h, G.y, 1);
  p->launches += 2;
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  *iters = k;
  *relres = res;
  return cudaSuccess;
}

}  // namespace ifgf
