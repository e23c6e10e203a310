// (e) Device GMRES for A y = b (Eq. lin_system), FP64 Arnoldi with classical
// Gram-Schmidt applied twice, Givens rotations on the device, y0 = 0, no
// restart.  The right-hand side is omega^{-1}(n x E^inc, n x H^inc) projected
// on (t1, t2) (right side of Eq. n_muller).
//
// nrhs independent solves run side by side and share every forward map: the
// Krylov basis is stored [k][rhs][4N], so the k-th vectors of all right-hand
// sides form one contiguous [nrhs][4N] block, the input of one batched
// forward map.  Every small kernel takes the right-hand side from its grid.
// A right-hand side whose residual estimate reached the tolerance is frozen
// (its Givens rotations, Hessenberg column and residual stop changing) while
// the others continue.
#include "gmres.h"

namespace ifgf {

namespace {

constexpr int kDotThreads = 256;
constexpr int kDotItems = 4;
constexpr int kDotJ = 8;
constexpr int kScal = 8;   // scalars per right-hand side: |b|, beta, residual estimate

__global__ void k_rhs(int N, const double* __restrict__ inc, NodeGeom g, double iw, double* __restrict__ b) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= N) return;
  const size_t rb = blockIdx.y;   // right-hand side
  inc += rb * 12 * (size_t)N;
  b += rb * 8 * (size_t)N;
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

// part[rb][chunk][j] = sum over the chunk of conj(V_{j,rb}) w_rb for j = 0..k1-1 (complex),
// V_{j,rb} = V + 2 (j ldv + rb n), w_rb = w + 2 rb n.  Grid: (chunks of kDotThreads *
// kDotItems elements) x (groups of kDotJ vectors) x (right-hand sides); w is read once per
// block and the kDotJ sums are reduced together.
__global__ void __launch_bounds__(kDotThreads) k_dots(int64_t n, int k1, const double* __restrict__ V,
                                                      size_t ldv, const double* __restrict__ w,
                                                      double* __restrict__ part, size_t pstride) {
  __shared__ double red[kDotThreads / 32][2 * kDotJ];
  const size_t rb = blockIdx.z;
  V += 2 * rb * (size_t)n;
  w += 2 * rb * (size_t)n;
  part += rb * pstride;
  const int64_t base = (int64_t)blockIdx.x * kDotThreads * kDotItems;
  const int j0 = blockIdx.y * kDotJ;
  double wr[kDotItems], wi[kDotItems];
  int64_t idx[kDotItems];
  const double2* w2 = reinterpret_cast<const double2*>(w);   // complex values: 16-byte loads
#pragma unroll
  for (int it = 0; it < kDotItems; ++it) {
    idx[it] = base + it * kDotThreads + threadIdx.x;
    const double2 x = idx[it] < n ? w2[idx[it]] : make_double2(0.0, 0.0);
    wr[it] = x.x;
    wi[it] = x.y;
  }
  double acc[2 * kDotJ];
#pragma unroll
  for (int jj = 0; jj < kDotJ; ++jj) {
    double ar = 0, ai = 0;
    const int j = j0 + jj;
    if (j < k1) {
      const double2* v = reinterpret_cast<const double2*>(V + 2 * (size_t)j * ldv);
#pragma unroll
      for (int it = 0; it < kDotItems; ++it)
        if (idx[it] < n) {
          const double2 x = v[idx[it]];
          ar += x.x * wr[it] + x.y * wi[it];
          ai += x.x * wi[it] - x.y * wr[it];
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

// h_rb[j] (+)= sum_blk part_rb[blk][j]: one warp per j, lanes over the chunks, then a warp
// reduction in a fixed order (the sums do not depend on timing)
constexpr int kReduceWarps = 4;
__global__ void __launch_bounds__(32 * kReduceWarps) k_reduce_parts(int nblk, int k1, const double* __restrict__ part,
                                                                    size_t pstride, double* __restrict__ h,
                                                                    size_t hstride, int accumulate) {
  const int j = blockIdx.x * kReduceWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (j >= k1) return;
  part += blockIdx.y * pstride;
  h += blockIdx.y * hstride;
  double sr = 0, si = 0;
  for (int b = lane; b < nblk; b += 32) {
    sr += part[2 * ((size_t)b * k1 + j)];
    si += part[2 * ((size_t)b * k1 + j) + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if (lane != 0) return;
  if (accumulate) {
    h[2 * j] += sr;
    h[2 * j + 1] += si;
  } else {
    h[2 * j] = sr;
    h[2 * j + 1] = si;
  }
}

// w_rb -= sum_j V_{j,rb} c_rb[j] (overwrite = 0) or w_rb = sum_j V_{j,rb} c_rb[j] (overwrite = 1),
// j < k1, or j < kvec[rb] when kvec is given
__global__ void k_combo(int64_t n, int k1, const int* __restrict__ kvec, const double* __restrict__ V,
                        size_t ldv, const double* __restrict__ c, size_t cstride, double* __restrict__ w,
                        int overwrite) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t rb = blockIdx.y;
  if (kvec) k1 = kvec[rb];
  V += 2 * rb * (size_t)n;
  c += rb * cstride;
  w += 2 * rb * (size_t)n;
  double ar = 0, ai = 0;
  const double2* V2 = reinterpret_cast<const double2*>(V) + i;   // complex values: 16-byte loads
  const double2* c2 = reinterpret_cast<const double2*>(c);
#pragma unroll 4
  for (int j = 0; j < k1; ++j) {
    const double2 v = V2[(size_t)j * ldv], cc = c2[j];
    ar += v.x * cc.x - v.y * cc.y;
    ai += v.x * cc.y + v.y * cc.x;
  }
  if (overwrite) {
    w[2 * i] = ar;
    w[2 * i + 1] = ai;
  } else {
    w[2 * i] -= ar;
    w[2 * i + 1] -= ai;
  }
}

// dst_rb = src_rb * f, f = 1 / sc_rb[0] (inv; 0 when sc_rb[0] = 0) or sc_rb[0]
__global__ void k_scale_copy(int64_t n, const double* __restrict__ src, const double* __restrict__ sc,
                             int inv, double* __restrict__ dst) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t rb = blockIdx.y;
  src += 2 * rb * (size_t)n;
  dst += 2 * rb * (size_t)n;
  const double s0 = sc[rb * kScal];
  double f = inv ? (s0 != 0.0 ? 1.0 / s0 : 0.0) : s0;
  dst[2 * i] = src[2 * i] * f;
  dst[2 * i + 1] = src[2 * i + 1] * f;
}

// r_rb = b_rb - w_rb (sub = 1) or r_rb += w_rb (sub = 0), n2 doubles per right-hand side; b and r
// may be the same array
__global__ void k_sub_add(int64_t n2, const double* b, const double* w, double* r, int sub) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n2) return;
  const size_t o = blockIdx.y * (size_t)n2 + i;
  r[o] = sub ? b[o] - w[o] : r[o] + w[o];
}

// |w_rb|^2 partials -> out_rb = |w_rb|; one block per right-hand side
__global__ void k_norm_final(int nblk, const double* __restrict__ part, size_t pstride, double* __restrict__ out) {
  const size_t rb = blockIdx.x;   // one warp per right-hand side, fixed summation order
  const int lane = threadIdx.x & 31;
  part += rb * pstride;
  double s = 0;
  for (int b = lane; b < nblk; b += 32) s += part[2 * (size_t)b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[rb * kScal] = sqrt(s);
}

struct Arnoldi {                  // per-right-hand-side arrays and their strides (doubles)
  double *H, *h, *cs, *sn, *g, *scal;
  size_t sH, sh, sv;              // H: (max_iter + 1) ldh x 2; h, cs, sn, g: (max_iter + 1) x 2
};

// Arnoldi column k of right-hand side rb (one block each; frozen ones return): Hcol[0..k] = h,
// Hcol[k+1] = beta; apply the previous rotations, form the new one, update g;
// scal[2] = |g_{k+1}| / |b|.
__global__ void k_givens(int k, int ldh, Arnoldi R, const int* __restrict__ active) {
  if (threadIdx.x != 0) return;
  const size_t rb = blockIdx.x;
  if (!active[rb]) return;
  double* H = R.H + rb * R.sH;
  const double* h = R.h + rb * R.sh;
  double* cs = R.cs + rb * R.sv;
  double* sn = R.sn + rb * R.sv;
  double* g = R.g + rb * R.sv;
  double* scal = R.scal + rb * kScal;
  double* col = H + 2 * (size_t)k * ldh;   // column k, rows 0..k+1
  for (int i = 0; i <= k; ++i) {
    col[2 * i] = h[2 * i];
    col[2 * i + 1] = h[2 * i + 1];
  }
  col[2 * (k + 1)] = scal[1];
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
  scal[2] = sqrt(g[2 * (k + 1)] * g[2 * (k + 1)] + g[2 * (k + 1) + 1] * g[2 * (k + 1) + 1]) / scal[0];
}

__global__ void k_init_g(Arnoldi R, int n) {
  const size_t rb = blockIdx.y;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double* g = R.g + rb * R.sv;
  if (i < 2 * n) g[i] = 0;
  if (i == 0) g[0] = R.scal[rb * kScal];
}

// back substitution R z = g[0..k_rb-1] (R upper triangular in H), z into h; one block per rhs
__global__ void k_backsub(const int* __restrict__ kvec, int ldh, Arnoldi R) {
  if (threadIdx.x != 0) return;
  const size_t rb = blockIdx.x;
  const int k = kvec[rb];
  const double* H = R.H + rb * R.sH;
  const double* g = R.g + rb * R.sv;
  double* z = R.h + rb * R.sh;
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

cudaError_t launch_rhs(const ifgf_plan_t* p, const double* inc, double* b, cudaStream_t s, int nrhs) {
  k_rhs<<<dim3((p->N + 127) / 128, nrhs), 128, 0, s>>>(p->N, inc, p->geo, 1.0 / p->omega, b);
  return cudaGetLastError();
}

int dots_blocks(int64_t n) { return (int)((n + kDotThreads * kDotItems - 1) / (kDotThreads * kDotItems)); }

namespace {

struct Batch {
  int nrhs;
  int64_t n;        // 4N
  int nb;           // dot-product chunks
  size_t ldv;       // doubles / 2 between consecutive Krylov vectors of one right-hand side
  size_t pstride;   // doubles of partial sums per right-hand side
};

// Gram-Schmidt projection of w against V[0..k1): h_pass = V^H w (per rhs), w -= V h_pass,
// h_tot (+)= h_pass.
cudaError_t project(GmresWork& G, const Batch& B, const Arnoldi& R, int k1, int first, cudaStream_t s) {
  double* hpass = R.h + 2 * (size_t)(G.max_iter + 1);   // second half of each rhs's h block
  k_dots<<<dim3(B.nb, (k1 + kDotJ - 1) / kDotJ, B.nrhs), kDotThreads, 0, s>>>(B.n, k1, G.V, B.ldv, G.w, G.part,
                                                                              B.pstride);
  k_reduce_parts<<<dim3((k1 + kReduceWarps - 1) / kReduceWarps, B.nrhs), 32 * kReduceWarps, 0, s>>>(
      B.nb, k1, G.part, B.pstride, hpass, R.sh, 0);
  k_combo<<<dim3((unsigned)((B.n + 255) / 256), B.nrhs), 256, 0, s>>>(B.n, k1, nullptr, G.V, B.ldv, hpass, R.sh,
                                                                        G.w, 0);
  k_reduce_parts<<<dim3((k1 + kReduceWarps - 1) / kReduceWarps, B.nrhs), 32 * kReduceWarps, 0, s>>>(
      B.nb, k1, G.part, B.pstride, R.h, R.sh,
                                                                  first ? 0 : 1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t gmres_residual(ifgf_plan_t* p, int nrhs, const double* b, const double* w, double* r,
                           cudaStream_t s) {
  GmresWork& G = p->gm;
  const int64_t n = 4 * (int64_t)p->N;
  const int nb = dots_blocks(n);
  const size_t pstride = 2 * (size_t)nb * (G.max_iter + 1);
  k_sub_add<<<dim3((unsigned)((2 * n + 255) / 256), nrhs), 256, 0, s>>>(2 * n, b, w, r, 1);
  k_dots<<<dim3(nb, 1, nrhs), kDotThreads, 0, s>>>(n, 1, r, 0, r, G.part, pstride);
  k_norm_final<<<nrhs, 32, 0, s>>>(nb, G.part, pstride, G.scal + 3);
  k_dots<<<dim3(nb, 1, nrhs), kDotThreads, 0, s>>>(n, 1, b, 0, b, G.part, pstride);
  k_norm_final<<<nrhs, 32, 0, s>>>(nb, G.part, pstride, G.scal + 4);
  p->launches += 5;
  return cudaGetLastError();
}

cudaError_t gmres_accumulate(ifgf_plan_t* p, int nrhs, const double* d, double* y, cudaStream_t s, bool subtract) {
  const int64_t n2 = 8 * (int64_t)p->N;
  k_sub_add<<<dim3((unsigned)((n2 + 255) / 256), nrhs), 256, 0, s>>>(n2, y, d, y, subtract ? 1 : 0);
  ++p->launches;
  return cudaGetLastError();
}

cudaError_t gmres_run(ifgf_plan_t* p, const MatvecFn& matvec, int nrhs, double tol, int max_iter, int* iters,
                      double* relres, cudaStream_t s, const MatvecFn* precond) {
  GmresWork& G = p->gm;
  const int64_t n = 4 * (int64_t)p->N;
  const int ldh = G.max_iter + 1;
  Batch B{nrhs, n, dots_blocks(n), (size_t)nrhs * (size_t)n, 2 * (size_t)dots_blocks(n) * (G.max_iter + 1)};
  const size_t sv = 2 * (size_t)(G.max_iter + 1);
  Arnoldi R{G.H, G.h, G.cs, G.sn, G.g, G.scal, 2 * (size_t)(G.max_iter + 1) * ldh, 2 * sv, sv};
  const unsigned vblocks = (unsigned)((n + 255) / 256);
  cudaError_t err;
  // |b_rb|, g_rb = |b_rb| e_1, v_{0,rb} = b_rb / |b_rb|
  k_dots<<<dim3(B.nb, 1, nrhs), kDotThreads, 0, s>>>(n, 1, G.b, 0, G.b, G.part, B.pstride);
  k_norm_final<<<nrhs, 32, 0, s>>>(B.nb, G.part, B.pstride, G.scal + 0);
  k_init_g<<<dim3((2 * (G.max_iter + 1) + 127) / 128, nrhs), 128, 0, s>>>(R, G.max_iter + 1);
  k_scale_copy<<<dim3(vblocks, nrhs), 256, 0, s>>>(n, G.b, G.scal + 0, 1, G.V);
  p->launches += 4;
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if ((err = cudaMemcpyAsync(G.hres, G.scal, sizeof(double) * kScal * nrhs, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return err;
  if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return err;
  int nactive = 0;
  for (int r = 0; r < nrhs; ++r) {
    const bool a = G.hres[r * kScal] != 0.0;   // b = 0: y = 0 after zero iterations
    G.hactive[r] = a ? 1 : 0;
    G.hk[r] = 0;
    relres[r] = a ? 1.0 : 0.0;
    nactive += a;
  }
  if ((err = cudaMemcpyAsync(G.active, G.hactive, sizeof(int) * nrhs, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return err;
  int k = 0;
  for (k = 0; k < max_iter && nactive > 0; ++k) {
    // w_rb = A v_{k,rb} (flexible: w_rb = A z_{k,rb}, z = M v) for all right-hand sides in one
    // batched forward map
    const double* vk = G.V + 2 * (size_t)k * B.ldv;
    if (precond) {
      double* zk = p->pc.Z + 2 * (size_t)k * B.ldv;
      if ((err = (*precond)(vk, zk, s)) != cudaSuccess) return err;
      vk = zk;
      ++p->launches;
    }
    if ((err = matvec(vk, G.w, s)) != cudaSuccess) return err;
    const int rec = timer_begin(p, TK_GMRES, s);
    // CGS2: two projection passes, h = h1 + h2
    if ((err = project(G, B, R, k + 1, 1, s)) != cudaSuccess) return err;
    if ((err = project(G, B, R, k + 1, 0, s)) != cudaSuccess) return err;
    k_dots<<<dim3(B.nb, 1, nrhs), kDotThreads, 0, s>>>(n, 1, G.w, 0, G.w, G.part, B.pstride);
    k_norm_final<<<nrhs, 32, 0, s>>>(B.nb, G.part, B.pstride, G.scal + 1);   // scal[1] = beta
    k_givens<<<nrhs, 32, 0, s>>>(k, ldh, R, G.active);
    k_scale_copy<<<dim3(vblocks, nrhs), 256, 0, s>>>(n, G.w, G.scal + 1, 1, G.V + 2 * (size_t)(k + 1) * B.ldv);
    timer_end(p, rec, s);
    p->launches += 12;   // 2 x (dots, reduce, combo, reduce), dots, norm, givens, scale
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if ((err = cudaMemcpyAsync(G.hres, G.scal, sizeof(double) * kScal * nrhs, cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
      return err;
    if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return err;
    bool changed = false;
    for (int r = 0; r < nrhs; ++r) {
      if (!G.hactive[r]) continue;
      relres[r] = G.hres[r * kScal + 2];
      G.hk[r] = k + 1;
      if (relres[r] <= tol || G.hres[r * kScal + 1] == 0.0) {
        G.hactive[r] = 0;
        --nactive;
        changed = true;
      }
    }
    if (changed && nactive > 0 &&
        (err = cudaMemcpyAsync(G.active, G.hactive, sizeof(int) * nrhs, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return err;
  }
  if ((err = cudaMemcpyAsync(G.kfin, G.hk, sizeof(int) * nrhs, cudaMemcpyHostToDevice, s)) != cudaSuccess) return err;
  k_backsub<<<nrhs, 32, 0, s>>>(G.kfin, ldh, R);
  k_combo<<<dim3(vblocks, nrhs), 256, 0, s>>>(n, 0, G.kfin, precond ? p->pc.Z : G.V, B.ldv, R.h, R.sh, G.y, 1);
  p->launches += 2;
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  for (int r = 0; r < nrhs; ++r) iters[r] = G.hk[r];
  return cudaSuccess;
}

}  // namespace ifgf
