// Learned right preconditioner for flexible GMRES (this library's addition; the
// paper solves with plain GMRES).  Per patch p, with v_p the 4 Nc^2 complex
// unknowns of the patch (the (m.t1, m.t2, j.t1, j.t2) components of its nodes)
// read as 8 Nc^2 reals x and s_p = |x|:
//   z_p = v_p + s_p (W2^T relu(W1^T (x / s_p) + b1) + b2)
// (or, with the block-Jacobi preconditioner built, z_p = (A_pp^{-1} v)_p + the same correction),
// a two-layer network shared by all patches, BF16 weights with FP32
// accumulation.  Zero output weights give z = v (plain GMRES).  The network
// is trained on pairs (v, e) with v = A e: per patch the input x = v_p / s_p and
// the target (e_p - v_p) / s_p, mean squared error, Adam, all on the device.
#include <cuda_bf16.h>

#include "kernels.h"

namespace ifgf {

namespace {

constexpr int kMlpThreads = 256;

// feature f = (c Nc^2 + q) 2 + ri of patch p of right-hand side rb in a [nrhs][4][N] complex128
// vector: component c, node l = p Nc^2 + q, real (ri = 0) or imaginary part
__device__ inline size_t feat_index(int f, int p, int npp, int N) {
  const int ri = f & 1, cq = f >> 1, c = cq / npp, q = cq % npp;
  return 2 * ((size_t)c * N + (size_t)p * npp + q) + ri;
}

__device__ inline float block_sum(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float s = 0;
  for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
  return s;
}

// z = M v, one block per (patch, right-hand side); x and the hidden layer live in shared memory
__global__ void __launch_bounds__(kMlpThreads) k_mlp_apply(int N, int npp, int in, int hid,
                                                           const __nv_bfloat16* __restrict__ W1,
                                                           const float* __restrict__ b1,
                                                           const __nv_bfloat16* __restrict__ W2,
                                                           const float* __restrict__ b2, const double* __restrict__ v,
                                                           const double* base, double* z) {
  extern __shared__ float sx[];   // [in] features, then [hid] hidden
  __shared__ float red[kMlpThreads / 32];
  float* sh = sx + in;
  const int p = blockIdx.x;
  const size_t rb = blockIdx.y;
  v += rb * 8 * (size_t)N;
  base += rb * 8 * (size_t)N;
  z += rb * 8 * (size_t)N;
  float ss = 0;
  for (int f = threadIdx.x; f < in; f += blockDim.x) {
    const float x = (float)v[feat_index(f, p, npp, N)];
    sx[f] = x;
    ss += x * x;
  }
  const float s = sqrtf(block_sum(ss, red));
  const float is = s > 0.f ? 1.f / s : 0.f;
  for (int h = threadIdx.x; h < hid; h += blockDim.x) {
    float a = b1[h];
    for (int f = 0; f < in; ++f) a += __bfloat162float(W1[(size_t)f * hid + h]) * sx[f] * is;
    sh[h] = fmaxf(a, 0.f);
  }
  __syncthreads();
  for (int f = threadIdx.x; f < in; f += blockDim.x) {
    float a = b2[f];
    for (int h = 0; h < hid; ++h) a += __bfloat162float(W2[(size_t)h * in + f]) * sh[h];
    const size_t i = feat_index(f, p, npp, N);
    z[i] = base[i] + (s > 0.f ? (double)(s * a) : 0.0);   // base may be z itself (same element)
  }
}

// training pairs: rows rb P + p of X = v_p / s_p and T = (e_p - v_p) / s_p (zero rows when s_p = 0)
__global__ void __launch_bounds__(kMlpThreads) k_mlp_features(int N, int npp, int in, int P,
                                                              const double* __restrict__ v,
                                                              const double* __restrict__ e,
                                                              const double* __restrict__ base, float* __restrict__ X,
                                                              float* __restrict__ T) {
  __shared__ float red[kMlpThreads / 32];
  const int p = blockIdx.x;
  const size_t rb = blockIdx.y;
  v += rb * 8 * (size_t)N;
  e += rb * 8 * (size_t)N;
  base += rb * 8 * (size_t)N;
  const size_t row = (rb * P + p) * (size_t)in;
  float ss = 0;
  for (int f = threadIdx.x; f < in; f += blockDim.x) {
    const float x = (float)v[feat_index(f, p, npp, N)];
    ss += x * x;
  }
  const float s = sqrtf(block_sum(ss, red));
  const float is = s > 0.f ? 1.f / s : 0.f;
  for (int f = threadIdx.x; f < in; f += blockDim.x) {
    const size_t i = feat_index(f, p, npp, N);
    X[row + f] = (float)v[i] * is;
    T[row + f] = (float)(e[i] - base[i]) * is;
  }
}

// C[M][N] = sum_k op(A)[m][k] op(B)[k][n] (+ bias[n]) with op = identity or transpose of a
// row-major matrix; 16 x 16 tiles through shared memory, FP32
constexpr int kTile = 16;
__global__ void k_gemm(int M, int Nn, int K, const float* __restrict__ A, int ta, const float* __restrict__ B,
                       int tb, const float* __restrict__ bias, float* __restrict__ C) {
  __shared__ float As[kTile][kTile + 1], Bs[kTile][kTile + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int m = blockIdx.y * kTile + ty, n = blockIdx.x * kTile + tx;
  float acc = 0.f;
  for (int k0 = 0; k0 < K; k0 += kTile) {
    const int ka = k0 + tx, kb = k0 + ty;
    // A tile: row m, column ka
    float a = 0.f;
    if (m < M && ka < K) a = ta ? A[(size_t)ka * M + m] : A[(size_t)m * K + ka];
    As[ty][tx] = a;
    float b = 0.f;
    if (kb < K && n < Nn) b = tb ? B[(size_t)n * K + kb] : B[(size_t)kb * Nn + n];
    Bs[ty][tx] = b;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kTile; ++k) acc += As[ty][k] * Bs[k][tx];
    __syncthreads();
  }
  if (m < M && n < Nn) C[(size_t)m * Nn + n] = acc + (bias ? bias[n] : 0.f);
}

// counter-based sample index: the SplitMix64 finaliser of (seed, step, i)
__device__ inline uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void k_gather(int64_t nsamples, int in, int B, uint64_t seed, int step, const float* __restrict__ X,
                         const float* __restrict__ T, float* __restrict__ Xb, float* __restrict__ Tb) {
  const int b = blockIdx.x;
  const uint64_t r = mix64(seed ^ mix64(((uint64_t)step << 32) | (uint64_t)b));
  const int64_t row = (int64_t)(r % (uint64_t)nsamples);
  for (int f = threadIdx.x; f < in; f += blockDim.x) {
    Xb[(size_t)b * in + f] = X[(size_t)row * in + f];
    Tb[(size_t)b * in + f] = T[(size_t)row * in + f];
  }
}

__global__ void k_relu(size_t n, const float* __restrict__ pre, float* __restrict__ h) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) h[i] = fmaxf(pre[i], 0.f);
}

// dY = 2 (Y - T) / count, loss partial sums of (Y - T)^2 / count
__global__ void k_mse_grad(size_t n, const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ dY,
                           float* __restrict__ loss) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < n) {
    const float d = Y[i] - T[i];
    dY[i] = 2.f * d / (float)n;
    l = d * d / (float)n;
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
}

__global__ void k_relu_back(size_t n, const float* __restrict__ pre, float* __restrict__ dH) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n && pre[i] <= 0.f) dH[i] = 0.f;
}

// db[j] = sum_b d[b][j]
__global__ void k_colsum(int B, int n, const float* __restrict__ d, float* __restrict__ db) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += d[(size_t)b * n + j];
  db[j] = s;
}

__global__ void k_adam(size_t n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float c1, float c2) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  m[i] = b1 * m[i] + (1.f - b1) * gi;
  v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
  w[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + 1e-8f);
}

__global__ void k_to_bf16(size_t n, const float* __restrict__ a, __nv_bfloat16* __restrict__ b) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16(a[i]);
}

unsigned blocks_of(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

cudaError_t gemm(int M, int Nn, int K, const float* A, int ta, const float* B, int tb, const float* bias, float* C,
                 cudaStream_t s) {
  dim3 g((Nn + kTile - 1) / kTile, (M + kTile - 1) / kTile);
  k_gemm<<<g, dim3(kTile, kTile), 0, s>>>(M, Nn, K, A, ta, B, tb, bias, C);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mlp_apply(const ifgf_plan_t* p, int nrhs, const double* v, double* z, cudaStream_t s,
                             const double* base) {
  const Precond& M = p->pc;
  const size_t smem = sizeof(float) * (M.in + M.hidden);
  k_mlp_apply<<<dim3(p->P, nrhs), kMlpThreads, smem, s>>>(p->N, p->nc * p->nc, M.in, M.hidden,
      (const __nv_bfloat16*)M.W1h, M.b1, (const __nv_bfloat16*)M.W2h, M.b2, v, base ? base : v, z);
  return cudaGetLastError();
}

cudaError_t launch_mlp_features(const ifgf_plan_t* p, int nrhs, const double* v, const double* e, float* X, float* T,
                                cudaStream_t s, const double* base) {
  k_mlp_features<<<dim3(p->P, nrhs), kMlpThreads, 0, s>>>(p->N, p->nc * p->nc, p->pc.in, p->P, v, e,
                                                           base ? base : v, X, T);
  return cudaGetLastError();
}

cudaError_t mlp_refresh_bf16(ifgf_plan_t* p, cudaStream_t s) {
  Precond& M = p->pc;
  const size_t n1 = (size_t)M.in * M.hidden;
  k_to_bf16<<<blocks_of(n1), 256, 0, s>>>(n1, M.W1, (__nv_bfloat16*)M.W1h);
  k_to_bf16<<<blocks_of(n1), 256, 0, s>>>(n1, M.W2, (__nv_bfloat16*)M.W2h);
  return cudaGetLastError();
}

// steps of Adam on minibatches drawn with the counter-based generator; loss[step] (device) gets
// the minibatch mean squared error before the step
cudaError_t mlp_train(ifgf_plan_t* p, int64_t nsamples, const float* X, const float* T, int steps, int B, float lr,
                      uint64_t seed, float* loss, cudaStream_t s) {
  Precond& M = p->pc;
  TrainWork& W = M.tw;
  const int in = M.in, H = M.hidden;
  const size_t n1 = (size_t)in * H;
  cudaError_t e;
  for (int it = 0; it < steps; ++it) {
    const int t = ++M.adam_t;
    const float c1 = 1.f - powf(0.9f, (float)t), c2 = 1.f - powf(0.999f, (float)t);
    k_gather<<<B, 256, 0, s>>>(nsamples, in, B, seed, t, X, T, W.Xb, W.Tb);
    if ((e = gemm(B, H, in, W.Xb, 0, M.W1, 0, M.b1, W.Hpre, s)) != cudaSuccess) return e;   // [B][H]
    k_relu<<<blocks_of((size_t)B * H), 256, 0, s>>>((size_t)B * H, W.Hpre, W.H1);
    if ((e = gemm(B, in, H, W.H1, 0, M.W2, 0, M.b2, W.Y, s)) != cudaSuccess) return e;      // [B][in]
    k_mse_grad<<<blocks_of((size_t)B * in), 256, 0, s>>>((size_t)B * in, W.Y, W.Tb, W.dY, loss + it);
    if ((e = gemm(H, in, B, W.H1, 1, W.dY, 0, nullptr, W.gW2, s)) != cudaSuccess) return e;  // H1^T dY
    k_colsum<<<blocks_of(in), 256, 0, s>>>(B, in, W.dY, W.gb2);
    if ((e = gemm(B, H, in, W.dY, 0, M.W2, 1, nullptr, W.dH, s)) != cudaSuccess) return e;   // dY W2^T
    k_relu_back<<<blocks_of((size_t)B * H), 256, 0, s>>>((size_t)B * H, W.Hpre, W.dH);
    if ((e = gemm(in, H, B, W.Xb, 1, W.dH, 0, nullptr, W.gW1, s)) != cudaSuccess) return e;  // Xb^T dH
    k_colsum<<<blocks_of(H), 256, 0, s>>>(B, H, W.dH, W.gb1);
    k_adam<<<blocks_of(n1), 256, 0, s>>>(n1, M.W1, W.gW1, W.mW1, W.vW1, lr, 0.9f, 0.999f, c1, c2);
    k_adam<<<blocks_of(H), 256, 0, s>>>(H, M.b1, W.gb1, W.mb1, W.vb1, lr, 0.9f, 0.999f, c1, c2);
    k_adam<<<blocks_of(n1), 256, 0, s>>>(n1, M.W2, W.gW2, W.mW2, W.vW2, lr, 0.9f, 0.999f, c1, c2);
    k_adam<<<blocks_of(in), 256, 0, s>>>(in, M.b2, W.gb2, W.mb2, W.vb2, lr, 0.9f, 0.999f, c1, c2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return mlp_refresh_bf16(p, s);
}

}  // namespace ifgf
