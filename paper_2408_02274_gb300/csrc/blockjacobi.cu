// Block-Jacobi right preconditioner (this library's addition; the paper solves with plain
// GMRES): per patch p the exact inverse of A's diagonal block A_pp, the operator restricted to
// the 4 Nc^2 unknowns of the patch's nodes (rows and columns), applied as z_p = A_pp^{-1} v_p.
//
// Assembly: the operator restricted to self-patch sources (the near matvec and the direct far
// sum, each keeping only sources in the target's own patch, between the plan's own density
// preparation and N-Mueller combination, both local to a patch) maps a vector that is the unit
// vector e_c on every patch at once to the c-th columns of all diagonal blocks, without
// crosstalk between patches; 4 Nc^2 such probes, up to the plan's batch per call, give every
// block.  For an IFGF plan the block's far part is the direct sum (the IFGF approximates it).
// Inversion: in-place Gauss-Jordan with partial (row) pivoting in FP64, one block of threads per
// patch, the pivot row and column staged in shared memory, the row interchanges undone on the
// columns at the end.
#include <algorithm>

#include "kernels.h"

namespace ifgf {

namespace {

constexpr int kGjThreads = 512;

// y[r][k][p npp + i] = 1 if c0 + r = k npp + i else 0, for every patch p (complex128)
__global__ void k_probe_set(int N, int npp, int c0, int nb, double* __restrict__ y) {
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t per = 4 * (size_t)N;
  if (idx >= per * nb) return;
  const int r = (int)(idx / per);
  const size_t kn = idx - (size_t)r * per;
  const int k = (int)(kn / N), l = (int)(kn - (size_t)k * N), i = l % npp;
  y[2 * idx] = (c0 + r == k * npp + i) ? 1.0 : 0.0;
  y[2 * idx + 1] = 0.0;
}

// B[p][k npp + i][c0 + r] = out[r][k][p npp + i]: column c0 + r of every diagonal block
__global__ void k_probe_gather(int N, int npp, int m, int c0, int nb, const double* __restrict__ out,
                               double* __restrict__ B) {
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t per = 4 * (size_t)N;
  if (idx >= per * nb) return;
  const int r = (int)(idx / per);
  const size_t kn = idx - (size_t)r * per;
  const int k = (int)(kn / N), l = (int)(kn - (size_t)k * N), p = l / npp, i = l - p * npp;
  const size_t dst = ((size_t)p * m + (size_t)(k * npp + i)) * m + (size_t)(c0 + r);
  B[2 * dst] = out[2 * idx];
  B[2 * dst + 1] = out[2 * idx + 1];
}

__device__ inline double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ inline double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// In-place inverse of the m x m complex block of patch blockIdx.x (row-major, double2): Gauss-
// Jordan with partial pivoting.  A zero pivot column sets bit 1 of *err and leaves the block.
__global__ void __launch_bounds__(kGjThreads) k_gj_inverse(int m, double2* __restrict__ Ball, int* __restrict__ ipiv_all,
                                                           int* __restrict__ err) {
  extern __shared__ double2 gj_smem[];   // [m] pivot column, [m] pivot row
  __shared__ double red_v[kGjThreads / 32];
  __shared__ int red_i[kGjThreads / 32];
  __shared__ int piv_s;
  __shared__ double2 inv_s;
  double2* colk = gj_smem;
  double2* rowk = gj_smem + m;
  double2* A = Ball + (size_t)blockIdx.x * m * m;
  int* ipiv = ipiv_all + (size_t)blockIdx.x * m;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int k = 0; k < m; ++k) {
    // pivot: the largest |A[i][k]|, i >= k (smallest i on ties)
    double best = -1.0;
    int bi = k;
    for (int i = k + t; i < m; i += blockDim.x) {
      const double v = cabs2(A[(size_t)i * m + k]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      red_v[warp] = best;
      red_i[warp] = bi;
    }
    __syncthreads();
    if (t == 0) {
      double bv = red_v[0];
      int b = red_i[0];
      for (int w = 1; w < (int)(blockDim.x / 32); ++w)
        if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < b)) {
          bv = red_v[w];
          b = red_i[w];
        }
      piv_s = bv > 0.0 ? b : -1;
      ipiv[k] = b;
    }
    __syncthreads();
    const int piv = piv_s;
    if (piv < 0) {
      if (t == 0) atomicOr(err, 2);
      return;
    }
    if (piv != k)
      for (int j = t; j < m; j += blockDim.x) {
        const double2 a = A[(size_t)k * m + j];
        A[(size_t)k * m + j] = A[(size_t)piv * m + j];
        A[(size_t)piv * m + j] = a;
      }
    __syncthreads();
    if (t == 0) {
      const double2 pv = A[(size_t)k * m + k];
      const double d = cabs2(pv);
      inv_s = make_double2(pv.x / d, -pv.y / d);
    }
    __syncthreads();
    const double2 inv = inv_s;
    for (int i = t; i < m; i += blockDim.x) colk[i] = A[(size_t)i * m + k];
    for (int j = t; j < m; j += blockDim.x) rowk[j] = j == k ? inv : cmul(A[(size_t)k * m + j], inv);
    __syncthreads();
    // A[i][j] -= A[i][k] * row_k[j] (i != k, j != k); column k: -A[i][k] / pivot; row k: row_k
    const int nwarps = blockDim.x >> 5;
    for (int i = warp; i < m; i += nwarps) {
      double2* Ai = A + (size_t)i * m;
      const double2 c = colk[i];
      for (int j = lane; j < m; j += 32) {
        if (i == k) {
          Ai[j] = rowk[j];
        } else if (j == k) {
          Ai[j] = make_double2(-(c.x * inv.x - c.y * inv.y), -(c.x * inv.y + c.y * inv.x));
        } else {
          const double2 r = rowk[j], a = Ai[j];
          Ai[j] = make_double2(a.x - (c.x * r.x - c.y * r.y), a.y - (c.x * r.y + c.y * r.x));
        }
      }
    }
    __syncthreads();
  }
  // undo the row interchanges: swap columns k and ipiv[k], last interchange first
  for (int k = m - 1; k >= 0; --k) {
    const int q = ipiv[k];
    if (q != k)
      for (int i = t; i < m; i += blockDim.x) {
        const double2 a = A[(size_t)i * m + k];
        A[(size_t)i * m + k] = A[(size_t)i * m + q];
        A[(size_t)i * m + q] = a;
      }
    __syncthreads();
  }
}

// z_p = Binv_p v_p for every patch, right-hand side blockIdx.z; a warp per output row, v_p staged
// in shared memory ([nrhs][4][N] complex128 in and out)
constexpr int kBjRows = 8;
__global__ void __launch_bounds__(32 * kBjRows) k_bj_apply(int N, int npp, int m, const double2* __restrict__ Binv,
                                                           const double2* __restrict__ v, double2* __restrict__ z) {
  extern __shared__ double2 vp[];   // [m]
  const int p = blockIdx.x;
  const size_t rb = blockIdx.z;
  v += rb * 4 * (size_t)N;
  z += rb * 4 * (size_t)N;
  for (int c = threadIdx.x; c < m; c += blockDim.x) vp[c] = v[(size_t)(c / npp) * N + (size_t)p * npp + c % npp];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.y * kBjRows + warp;
  if (row >= m) return;
  const double2* R = Binv + ((size_t)p * m + row) * m;
  double sr = 0.0, si = 0.0;
  for (int c = lane; c < m; c += 32) {
    const double2 a = R[c], b = vp[c];
    sr += a.x * b.x - a.y * b.y;
    si += a.x * b.y + a.y * b.x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if (lane == 0) z[(size_t)(row / npp) * N + (size_t)p * npp + row % npp] = make_double2(sr, si);
}

}  // namespace

cudaError_t setup_bj_kernels() {
  // the Gauss-Jordan pivot row and column of the largest block (N_c = 24: m = 2304)
  return cudaFuncSetAttribute(k_gj_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(2 * sizeof(double2) * 4 * 24 * 24));
}

cudaError_t launch_bj_apply(const ifgf_plan_t* p, int nrhs, const double* v, double* z, cudaStream_t s) {
  const BlockJacobi& J = p->bj;
  const int npp = p->nc * p->nc;
  k_bj_apply<<<dim3((unsigned)p->P, (unsigned)((J.m + kBjRows - 1) / kBjRows), (unsigned)nrhs), 32 * kBjRows,
               sizeof(double2) * J.m, s>>>(p->N, npp, J.m, reinterpret_cast<const double2*>(J.inv),
                                           reinterpret_cast<const double2*>(v), reinterpret_cast<double2*>(z));
  return cudaGetLastError();
}

// Assembles and inverts every diagonal block into p->bj.inv (allocated by the caller, [P][m][m]
// complex128), using yb and ob ([batch][4][N] complex128 each) as probe buffers and ipiv ([P][m])
// as scratch.  Synchronous on s; bit 1 of *err_dev set means a singular block.
cudaError_t bj_build(ifgf_plan_t* p, double* yb, double* ob, int* ipiv, int* err_dev, cudaStream_t s) {
  const int npp = p->nc * p->nc, m = 4 * npp;
  cudaError_t e = cudaSuccess;
  const size_t per = 4 * (size_t)p->N;
  for (int c0 = 0; c0 < m && e == cudaSuccess; c0 += p->batch) {
    const int nb = std::min(p->batch, m - c0);
    const unsigned g = (unsigned)((per * nb + 255) / 256);
    k_probe_set<<<g, 256, 0, s>>>(p->N, npp, c0, nb, yb);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_density_prep(p, yb, nullptr, s, nb);
    if (e == cudaSuccess) e = launch_near_self(p, s, nb);
    if (e == cudaSuccess) e = launch_far_self(p, s, nb);
    if (e == cudaSuccess) e = launch_combine(p, yb, ob, s, nb);
    if (e == cudaSuccess) {
      k_probe_gather<<<g, 256, 0, s>>>(p->N, npp, m, c0, nb, ob, p->bj.inv);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) {
    k_gj_inverse<<<(unsigned)p->P, kGjThreads, 2 * sizeof(double2) * m, s>>>(
        m, reinterpret_cast<double2*>(p->bj.inv), ipiv, err_dev);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace ifgf
