// (d) Near-field correction matvec and the plain direct far sum.
//
// Near: f28[l] = sum_m N_s[l][m] phi_m for the four precomputed complex
// matrices N = (S_e, S_i, D_e, D_i) (singular weights of Sec. III-D with the
// local corrections of Sec. III-H); S acts on all 8 densities, D on the 6
// Cartesian ones.  One warp per target row; the weights stream once from HBM.
//
// Direct far: the sum of Eq. ifgf_sum_em written out, over all sources
// outside the target's neighbour boxes (the pairs the IFGF approximates),
// for G_e, G_i and their normal derivatives at the target.
#include "kernels.h"

namespace ifgf {

namespace {

template <typename T>
__device__ inline T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// n values of type T from a 16-byte aligned address as 16-byte vector loads
template <typename T, int n>
__device__ __forceinline__ void ldg_vec(const T* __restrict__ src, T* dst) {
  static_assert((n * sizeof(T)) % 16 == 0, "whole 16-byte vectors");
  const float4* s4 = reinterpret_cast<const float4*>(src);
  float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int i = 0; i < (int)(n * sizeof(T) / 16); ++i) d4[i] = __ldg(s4 + i);
}

template <typename T>
__device__ __forceinline__ void near_madd(const T* w, const T* ph, T* acc) {
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const T wr = w[2 * s], wi = w[2 * s + 1];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      acc[2 * (8 * s + k)] += wr * ph[2 * k] - wi * ph[2 * k + 1];
      acc[2 * (8 * s + k) + 1] += wr * ph[2 * k + 1] + wi * ph[2 * k];
    }
    const T dr = w[4 + 2 * s], di = w[4 + 2 * s + 1];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      acc[2 * (16 + 6 * s + k)] += dr * ph[2 * k] - di * ph[2 * k + 1];
      acc[2 * (16 + 6 * s + k) + 1] += dr * ph[2 * k + 1] + di * ph[2 * k];
    }
  }
}

// One warp per target row, lanes strided over the row's nonzeros.  Software pipeline per lane:
// while the multiply-adds of nonzero e run, the weights and densities of e + 32 are in flight
// and the column index of e + 64 is being loaded, so neither the column -> density gather
// dependence nor the HBM latency of the weights sits between two steps.
template <typename T>
__global__ void __launch_bounds__(256) k_near(int N, const int64_t* __restrict__ row_ptr,
                                              const int* __restrict__ col, const T* __restrict__ val,
                                              const T* __restrict__ phi, T* __restrict__ f28) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= N) return;
  const size_t rb = blockIdx.y;   // right-hand side of a batched call
  phi += rb * 16 * (size_t)N;
  f28 += rb * 56 * (size_t)N;
  T acc[56];
#pragma unroll
  for (int k = 0; k < 56; ++k) acc[k] = T(0);
  const int64_t e0 = row_ptr[row], e1 = row_ptr[row + 1];
  int64_t e = e0 + lane;
  if constexpr (sizeof(T) == 8) {   // FP64: twice the registers per nonzero, one nonzero per step
    for (; e < e1; e += 32) {
      alignas(16) T w0[8], p0[16];
      ldg_vec<T, 8>(val + 8 * e, w0);
      ldg_vec<T, 16>(phi + 16 * (size_t)__ldg(col + e), p0);
      near_madd(w0, p0, acc);
    }
    e = e1;
  }
  alignas(16) T w[8], p[16];
  if (e < e1) {
    ldg_vec<T, 8>(val + 8 * e, w);
    ldg_vec<T, 16>(phi + 16 * (size_t)__ldg(col + e), p);
  }
  int m1 = (e + 32 < e1) ? __ldg(col + e + 32) : 0;   // column of the next step
  for (; e < e1; e += 32) {
    const int64_t e1n = e + 32, e2n = e + 64;
    const int m2 = (e2n < e1) ? __ldg(col + e2n) : 0;   // column two steps ahead
    alignas(16) T wn[8], pn[16];
    if (e1n < e1) {
      ldg_vec<T, 8>(val + 8 * e1n, wn);
      ldg_vec<T, 16>(phi + 16 * (size_t)m1, pn);
    }
    near_madd(w, p, acc);
#pragma unroll
    for (int k = 0; k < 8; ++k) w[k] = wn[k];
#pragma unroll
    for (int k = 0; k < 16; ++k) p[k] = pn[k];
    m1 = m2;
  }
#pragma unroll
  for (int k = 0; k < 56; ++k) acc[k] = warp_sum(acc[k]);
  T* out = f28 + 56 * (size_t)row;
#pragma unroll
  for (int k = 0; k < 56; ++k)
    if ((k & 31) == lane) out[k] = acc[k];
}

template <typename T>
struct SrcTile {
  T x[3];
  int c[3];
  T a[16];
};

// T: storage type of the densities and fields (the plan's precision); A: arithmetic type
// (T, or FP64 for the sampled reference of an FP32 plan).
template <typename T, typename A = T>
__global__ void __launch_bounds__(128) k_far_direct(int N, const double* __restrict__ x,
                                                    const double* __restrict__ nrm,
                                                    const int* __restrict__ leafc,
                                                    const T* __restrict__ a, A ke, A ki,
                                                    T* __restrict__ f28, const int* __restrict__ blocks,
                                                    int npp, int self_patch = 0) {
  __shared__ SrcTile<A> tile[128];
  const size_t rb = blockIdx.y;   // right-hand side of a batched call
  a += rb * 16 * (size_t)N;
  f28 += rb * 56 * (size_t)N;
  // targets: thread t takes node l0 + t when lo <= l0 + t < hi; node l0 is the block's origin.
  // Without a block list, a block is a chunk of up to 128 nodes of one patch (npp = N_c^2) or
  // 128 consecutive nodes (npp = 128); a block list gives (l0, lo, hi) per block explicitly.
  int l0, lo, hi;
  if (blocks) {
    l0 = blocks[3 * blockIdx.x];
    lo = blocks[3 * blockIdx.x + 1];
    hi = blocks[3 * blockIdx.x + 2];
  } else {
    const int cpp = (npp + 127) / 128, chunk = blockIdx.x % cpp;
    l0 = lo = (int)(blockIdx.x / cpp) * npp + chunk * 128;
    hi = min(l0 + min(128, npp - chunk * 128), N);
  }
  const int lt = l0 + (int)threadIdx.x;
  const bool act = lt >= lo && lt < hi;
  const int l = act ? lt : lo;
  // coordinates relative to the block origin, formed in FP64: the differences of
  // nearby points keep their digits whatever the body's size
  const double o0 = x[3 * (size_t)l0], o1 = x[3 * (size_t)l0 + 1], o2 = x[3 * (size_t)l0 + 2];
  A xl[3] = {0, 0, 0}, nl[3] = {0, 0, 0};
  int cl[3] = {0, 0, 0};
  if (act) {
    xl[0] = (A)(x[3 * (size_t)l] - o0);
    xl[1] = (A)(x[3 * (size_t)l + 1] - o1);
    xl[2] = (A)(x[3 * (size_t)l + 2] - o2);
    for (int k = 0; k < 3; ++k) {
      nl[k] = (A)nrm[3 * (size_t)l + k];
      cl[k] = leafc[3 * l + k];
    }
  }
  A acc[56];
#pragma unroll
  for (int k = 0; k < 56; ++k) acc[k] = A(0);
  const A kk[2] = {ke, ki};
  const A inv4pi = A(1.0 / (4.0 * kPi));
  // sources: all nodes, or (self_patch, blocks of one patch) only the block's own patch
  const int sb = self_patch ? l0 / npp * npp : 0, se = self_patch ? min(sb + npp, N) : N;
  for (int base = sb; base < se; base += 128) {
    __syncthreads();
    int m = base + threadIdx.x;
    if (m < se) {
      tile[threadIdx.x].x[0] = (A)(x[3 * (size_t)m] - o0);
      tile[threadIdx.x].x[1] = (A)(x[3 * (size_t)m + 1] - o1);
      tile[threadIdx.x].x[2] = (A)(x[3 * (size_t)m + 2] - o2);
      for (int k = 0; k < 3; ++k) tile[threadIdx.x].c[k] = leafc[3 * m + k];
      for (int k = 0; k < 16; ++k) tile[threadIdx.x].a[k] = (A)a[16 * (size_t)m + k];
    }
    __syncthreads();
    const int nt = min(128, se - base);
    if (!act) continue;
    for (int q = 0; q < nt; ++q) {
      const SrcTile<A>& s = tile[q];
      if (abs(s.c[0] - cl[0]) <= 1 && abs(s.c[1] - cl[1]) <= 1 && abs(s.c[2] - cl[2]) <= 1) continue;
      A d0 = xl[0] - s.x[0], d1 = xl[1] - s.x[1], d2 = xl[2] - s.x[2];
      A r2 = d0 * d0 + d1 * d1 + d2 * d2;
      A r = sqrt_t(r2);
      A ir = A(1) / r;
      A nd = (nl[0] * d0 + nl[1] * d1 + nl[2] * d2) * ir * ir;
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        A sn, cs;
        sincos_t(kk[ks] * r, &sn, &cs);
        A g = inv4pi * ir;
        A gr = g * cs, gi = g * sn;
        A dr = nd * (-gr - kk[ks] * r * gi), di = nd * (-gi + kk[ks] * r * gr);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          acc[2 * (8 * ks + k)] += gr * s.a[2 * k] - gi * s.a[2 * k + 1];
          acc[2 * (8 * ks + k) + 1] += gr * s.a[2 * k + 1] + gi * s.a[2 * k];
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          acc[2 * (16 + 6 * ks + k)] += dr * s.a[2 * k] - di * s.a[2 * k + 1];
          acc[2 * (16 + 6 * ks + k) + 1] += dr * s.a[2 * k + 1] + di * s.a[2 * k];
        }
      }
    }
  }
  if (act)
    for (int k = 0; k < 56; ++k) f28[56 * (size_t)l + k] += (T)acc[k];
}

// The near matvec restricted to sources in the target's own patch (nodes are patch-major,
// npp per patch): one warp per target row; for the diagonal blocks of the block-Jacobi
// preconditioner.  Overwrites f28 like k_near.
template <typename T>
__global__ void __launch_bounds__(256) k_near_self(int N, int npp, const int64_t* __restrict__ row_ptr,
                                                   const int* __restrict__ col, const T* __restrict__ val,
                                                   const T* __restrict__ phi, T* __restrict__ f28) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= N) return;
  const size_t rb = blockIdx.y;
  phi += rb * 16 * (size_t)N;
  f28 += rb * 56 * (size_t)N;
  T acc[56];
#pragma unroll
  for (int k = 0; k < 56; ++k) acc[k] = T(0);
  const int patch = row / npp;
  for (int64_t e = row_ptr[row] + lane; e < row_ptr[row + 1]; e += 32) {
    const int c = __ldg(col + e);
    if (c / npp != patch) continue;
    alignas(16) T w[8], pc[16];
    ldg_vec<T, 8>(val + 8 * e, w);
    ldg_vec<T, 16>(phi + 16 * (size_t)c, pc);
    near_madd(w, pc, acc);
  }
#pragma unroll
  for (int k = 0; k < 56; ++k) acc[k] = warp_sum(acc[k]);
  T* out = f28 + 56 * (size_t)row;
#pragma unroll
  for (int k = 0; k < 56; ++k)
    if ((k & 31) == lane) out[k] = acc[k];
}

}  // namespace

cudaError_t launch_near_self(const ifgf_plan_t* p, cudaStream_t s, int nrhs) {
  const int npp = p->desc.nc * p->desc.nc;
  const unsigned blocks = (unsigned)(((size_t)p->N * 32 + 255) / 256);
  if (store64(p->desc))
    k_near_self<double><<<dim3(blocks, nrhs), 256, 0, s>>>(p->N, npp, p->near.row_ptr, p->near.col,
        p->near.val64, (const double*)p->phi, (double*)p->f28);
  else
    k_near_self<float><<<dim3(blocks, nrhs), 256, 0, s>>>(p->N, npp, p->near.row_ptr, p->near.col,
        p->near.val32, (const float*)p->phi, (float*)p->f28);
  return cudaGetLastError();
}

// The direct far sum restricted to sources in the target's own patch (blocks are chunks of one
// patch in both precisions); accumulates into f28.
cudaError_t launch_far_self(const ifgf_plan_t* p, cudaStream_t s, int nrhs) {
  const int npp = p->desc.nc * p->desc.nc;
  const unsigned blocks = (unsigned)(p->P * ((npp + 127) / 128));
  if (store64(p->desc))
    k_far_direct<double><<<dim3(blocks, nrhs), 128, 0, s>>>(p->N, p->geo.x, p->geo.n, p->leafc,
        (const double*)p->a_orig, p->desc.k_ext, p->desc.k_int, (double*)p->f28, nullptr, npp, 1);
  else
    k_far_direct<float><<<dim3(blocks, nrhs), 128, 0, s>>>(p->N, p->geo.x, p->geo.n, p->leafc,
        (const float*)p->a_orig, (float)p->desc.k_ext, (float)p->desc.k_int, (float*)p->f28, nullptr, npp, 1);
  return cudaGetLastError();
}

cudaError_t launch_near(const ifgf_plan_t* p, cudaStream_t s, int nrhs) {
  const int threads = p->near_threads;   // 128 or 256 (the kernel's launch bound)
  const unsigned blocks = (unsigned)(((size_t)p->N * 32 + threads - 1) / threads);
  if (store64(p->desc))
    k_near<double><<<dim3(blocks, nrhs), threads, 0, s>>>(p->N, p->near.row_ptr, p->near.col,
        p->near.val64, (const double*)p->phi, (double*)p->f28);
  else
    k_near<float><<<dim3(blocks, nrhs), threads, 0, s>>>(p->N, p->near.row_ptr, p->near.col,
        p->near.val32, (const float*)p->phi, (float*)p->f28);
  return cudaGetLastError();
}

cudaError_t launch_far_direct(const ifgf_plan_t* p, cudaStream_t s, int nrhs) {
  const int npp = p->desc.nc * p->desc.nc;
  if (store64(p->desc)) {
    // FP64 keeps the digits of nearby differences without patch-local origins: every block
    // takes 128 consecutive nodes (no idle lanes when N_c^2 is not a multiple of 128)
    k_far_direct<double><<<dim3((unsigned)((p->N + 127) / 128), nrhs), 128, 0, s>>>(p->N, p->geo.x, p->geo.n,
        p->leafc, (const double*)p->a_orig, p->desc.k_ext, p->desc.k_int, (double*)p->f28, nullptr, 128);
  } else {
    // FP32: a block takes a chunk of one patch, a compact group around its origin
    const unsigned blocks = (unsigned)(p->P * ((npp + 127) / 128));
    k_far_direct<float><<<dim3(blocks, nrhs), 128, 0, s>>>(p->N, p->geo.x, p->geo.n, p->leafc,
        (const float*)p->a_orig, (float)p->desc.k_ext, (float)p->desc.k_int, (float*)p->f28, nullptr, npp);
  }
  return cudaGetLastError();
}

// The FP64 direct far sum on listed target ranges (the sampled reference): blocks [nblocks][3] =
// (origin, lo, hi) with origin = 128 * j, the start of the FP64 full map's j-th block, so that
// the listed rows see the same origin, tile order and summation order as in that map.
cudaError_t launch_far_direct_blocks(const ifgf_plan_t* p, cudaStream_t s, const int* blocks, int nblocks) {
  if (store64(p->desc))
    k_far_direct<double><<<dim3((unsigned)nblocks, 1), 128, 0, s>>>(p->N, p->geo.x, p->geo.n, p->leafc,
        (const double*)p->a_orig, p->desc.k_ext, p->desc.k_int, (double*)p->f28, blocks, 128);
  else
    k_far_direct<float, double><<<dim3((unsigned)nblocks, 1), 128, 0, s>>>(p->N, p->geo.x, p->geo.n,
        p->leafc, (const float*)p->a_orig, p->desc.k_ext, p->desc.k_int, (float*)p->f28, blocks, 128);
  return cudaGetLastError();
}

// The same direct far-sum kernel on caller-provided arrays (used by the
// allocation-free entry point): a [N][8] weighted densities and f28 [N][28]
// accumulators in the given precision; f28 must be zeroed by the caller.  Without a
// patch structure the target groups are runs of 128 consecutive nodes.
cudaError_t launch_far_direct_raw(int N, const double* x, const double* nrm, const int* leafc, const void* a,
                                  double ke, double ki, int precision, void* f28, cudaStream_t s) {
  const unsigned blocks = (unsigned)((N + 127) / 128);
  if (precision == IFGF_FP64)
    k_far_direct<double><<<blocks, 128, 0, s>>>(N, x, nrm, leafc, (const double*)a, ke, ki, (double*)f28,
                                                 nullptr, 128);
  else
    k_far_direct<float><<<blocks, 128, 0, s>>>(N, x, nrm, leafc, (const float*)a, (float)ke, (float)ki,
                                                (float*)f28, nullptr, 128);
  return cudaGetLastError();
}

}  // namespace ifgf
