// Shared device/host helpers of the CBIE-IFGF library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace ifgf {

constexpr double kPi = 3.14159265358979323846;
constexpr double kEta = 0.57735026918962576451;   // sqrt(3)/3: upper bound of s on cousins (Sec. III-E)
constexpr int kPs = 3;                            // radial interpolation points per cone (Remark 2)
constexpr int kPa = 5;                            // angular interpolation points per cone
constexpr int kQ = kPs * kPa * kPa;               // 75 interpolation points per cone segment
constexpr int kF = 16;                            // complex fields carried by the IFGF: 8 densities x 2 kernels
constexpr int kFR = 2 * kF;                       // real components (re, im interleaved)
constexpr int kNearFields = 28;                   // S_e[8], S_i[8], D_e[6], D_i[6]
constexpr int kUpRunMax = 32;                     // parent points per upward-pass run (<= 32: one per lane)
constexpr int kUpGroups = 4;                      // disjoint parent-point groups, one per warp of the upward block
constexpr int kTcBoxes = 4;                       // parent slots per tensor-core upward tile (M = 4 x 32 rows)
constexpr int kTcMaxUnits = 192;                  // most (octant, child cone) units of one parent cone on that path
constexpr size_t kImgFloatsHost = 2 * 32 * 80;     // tensor-core operand image (hi, lo) of one cone segment

// Complex helpers on plain real pairs (the library keeps complex data interleaved).
template <typename T>
struct cplx {
  T re, im;
};

template <typename T>
__host__ __device__ inline cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

template <typename T>
__device__ inline void sincos_t(T x, T* s, T* c);
template <>
__device__ inline void sincos_t<float>(float x, float* s, float* c) { sincosf(x, s, c); }
template <>
__device__ inline void sincos_t<double>(double x, double* s, double* c) { sincos(x, s, c); }

template <typename T>
__device__ inline T sqrt_t(T x);
template <>
__device__ inline float sqrt_t<float>(float x) { return sqrtf(x); }
template <>
__device__ inline double sqrt_t<double>(double x) { return sqrt(x); }

#if defined(__CUDACC__)
template <typename T>
__device__ inline T cospi_t(T x);
template <>
__device__ inline float cospi_t<float>(float x) { return cospif(x); }
template <>
__device__ inline double cospi_t<double>(double x) { return cospi(x); }
#endif

template <typename T>
__device__ inline T atan2_t(T y, T x);
template <>
__device__ inline float atan2_t<float>(float y, float x) { return atan2f(y, x); }
template <>
__device__ inline double atan2_t<double>(double y, double x) { return atan2(y, x); }

// T_0..T_{n-1}(t) and derivatives by the three-term recurrences.
template <typename T, int N>
__device__ __forceinline__ void cheb_vals(T t, T* v) {
  v[0] = T(1);
  if (N > 1) v[1] = t;
#pragma unroll
  for (int k = 2; k < N; ++k) v[k] = T(2) * t * v[k - 1] - v[k - 2];
}
// T_k'(t) = k U_{k-1}(t)
template <typename T, int N>
__device__ __forceinline__ void cheb_dvals(T t, T* d) {
  T u0 = T(1), u1 = T(2) * t;
  d[0] = T(0);
  if (N > 1) d[1] = T(1);
  if (N > 2) d[2] = T(2) * u1;
#pragma unroll
  for (int k = 3; k < N; ++k) {
    T u2 = T(2) * t * u1 - u0;
    d[k] = T(k) * u2;
    u0 = u1;
    u1 = u2;
  }
}

// Cone-segment geometry of one level (Sec. III-E, Eq. cone_dom):
// s in [0, eta) split in ns intervals, theta in [0, pi] in na, phi in [0, 2 pi) in 2 na.
struct ConeGeom {
  double h;      // box radius sqrt(3)/2 H
  int ns, na;
  __host__ __device__ double ds() const { return kEta / ns; }
  __host__ __device__ double dth() const { return kPi / na; }
};

// The same geometry in the arithmetic type of a kernel, with the spacings and their
// reciprocals formed once on the host (no FP64 division inside the FP32 kernels).
template <typename T>
struct ConeGeomT {
  T h, ds, dth, ids, idth;
  int ns, na;
};
template <typename T>
inline ConeGeomT<T> cone_geom_t(const ConeGeom& g) {
  return ConeGeomT<T>{(T)g.h, (T)g.ds(), (T)g.dth(), (T)(1.0 / g.ds()), (T)(1.0 / g.dth()), g.ns, g.na};
}

// A cone segment (g1, g2, g3) of a level (s-, theta-, phi-cell indices) as a key: three
// 21-bit fields with g1 most significant, so keys order like (g1, g2, g3) and stay unique
// for any level (ns, na < 2^20; the product ns * na * 2na may exceed 32 bits on deep trees).
typedef int64_t cone_key;
constexpr int kConeBits = 21;
constexpr int64_t kConeMask = (int64_t(1) << kConeBits) - 1;
__host__ __device__ inline void cone_decode(cone_key id, int* g1, int* g2, int* g3) {
  *g3 = (int)(id & kConeMask);
  *g2 = (int)((id >> kConeBits) & kConeMask);
  *g1 = (int)(id >> (2 * kConeBits));
}
__host__ __device__ inline cone_key cone_encode(int g1, int g2, int g3) {
  return ((cone_key)g1 << (2 * kConeBits)) | ((cone_key)g2 << kConeBits) | (cone_key)g3;
}

// Open Chebyshev node k of n on [-1, 1] (Eq. cheby_nodes).
__host__ __device__ inline double cheb_node(int k, int n) { return cos((k + 0.5) * kPi / n); }

}  // namespace ifgf

#define IFGF_CUDA_TRY(expr)                                   \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) {                                  \
      ::ifgf::set_last_cuda_error(_e, #expr, __FILE__, __LINE__); \
      return IFGF_ECUDA;                                      \
    }                                                         \
  } while (0)

namespace ifgf {
void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);
// records the message ifgf_status_string(status) returns for EUNSUPPORTED and EINTERNAL
void set_status_detail(int status, const char* msg);
}
