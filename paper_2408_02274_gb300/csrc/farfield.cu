// Far-field pattern of the scattered electric field from a solution of Eq. n_muller.
//
// With the exterior representation E^sc = -omega mu_e curl S_e[m] - i (k^2 S_e[j] + grad S_e[div j])
// (k = kappa_e) and G(x, y) -> e^{i k r}/(4 pi r) e^{-i k d.y} along a direction d as r -> infinity
// (grad_x -> i k d), E^sc(r d) = e^{i k r}/r E_inf(d) + O(1/r^2) with
//   E_inf(d) = -i k omega mu_e (d x F[m]) - i k^2 F[j] + k d F[div j],
//   F[f] = (1/4 pi) sum_l f(x_l) e^{-i k d.x_l} omega_l   (the Nystrom nodes and weights).
// One block per (direction, right-hand side) sums the seven complex moments over the nodes in
// FP64 (the phase k d.x is formed and reduced in FP64); the densities come from the density
// preparation of step a0.
#include "kernels.h"

namespace ifgf {

namespace {

constexpr int kFfThreads = 256;

__global__ void __launch_bounds__(kFfThreads) k_far_field(int N, const double* __restrict__ x,
                                                          const double* __restrict__ w,
                                                          const double* __restrict__ phi64,
                                                          const double* __restrict__ dirs, int ndirs, double k,
                                                          double omega_mu, double* __restrict__ out) {
  __shared__ double red[kFfThreads / 32][14];
  const int q = blockIdx.x;
  const size_t r = blockIdx.y;   // right-hand side
  phi64 += r * 16 * (size_t)N;
  const double d0 = dirs[3 * q], d1 = dirs[3 * q + 1], d2 = dirs[3 * q + 2];
  double acc[14];
#pragma unroll
  for (int f = 0; f < 14; ++f) acc[f] = 0.0;
  for (int l = threadIdx.x; l < N; l += blockDim.x) {
    double s, c;
    sincos(-k * (d0 * x[3 * (size_t)l] + d1 * x[3 * (size_t)l + 1] + d2 * x[3 * (size_t)l + 2]), &s, &c);
    const double wr = w[l] * c, wi = w[l] * s;
    const double* p = phi64 + 16 * (size_t)l;
#pragma unroll
    for (int f = 0; f < 6; ++f) {   // m_xyz, j_xyz
      const double pr = p[2 * f], pi = p[2 * f + 1];
      acc[2 * f] += wr * pr - wi * pi;
      acc[2 * f + 1] += wr * pi + wi * pr;
    }
    const double qr = p[14], qi = p[15];   // div j
    acc[12] += wr * qr - wi * qi;
    acc[13] += wr * qi + wi * qr;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int f = 0; f < 14; ++f) {
    double v = acc[f];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][f] = v;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double F[14];
  for (int f = 0; f < 14; ++f) {
    double v = 0;
    for (int wi = 0; wi < kFfThreads / 32; ++wi) v += red[wi][f];
    F[f] = v / (4.0 * kPi);
  }
  // d x F[m] (complex, component-wise on real and imaginary parts)
  const double dd[3] = {d0, d1, d2};
  double* o = out + (r * (size_t)ndirs + q) * 6;
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    const double cr = dd[b] * F[2 * (c)] - dd[c] * F[2 * (b)];           // Re (d x F[m])_a
    const double ci = dd[b] * F[2 * (c) + 1] - dd[c] * F[2 * (b) + 1];   // Im (d x F[m])_a
    const double jr = F[2 * (3 + a)], ji = F[2 * (3 + a) + 1];
    // -i k omega mu (cr + i ci) - i k^2 (jr + i ji) + k d_a (F12 + i F13)
    o[2 * a] = k * omega_mu * ci + k * k * ji + k * dd[a] * F[12];
    o[2 * a + 1] = -k * omega_mu * cr - k * k * jr + k * dd[a] * F[13];
  }
}

}  // namespace

cudaError_t launch_far_field(const ifgf_plan_t* p, int nrhs, int ndirs, const double* dirs, double* out,
                             cudaStream_t s) {
  k_far_field<<<dim3((unsigned)ndirs, (unsigned)nrhs), kFfThreads, 0, s>>>(
      p->N, p->geo.x, p->geo.w, p->phi64, dirs, ndirs, p->desc.k_ext, p->omega * p->desc.mu_ext, out);
  return cudaGetLastError();
}

}  // namespace ifgf
