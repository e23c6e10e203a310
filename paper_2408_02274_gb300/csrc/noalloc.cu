// Allocation-free evaluation of the plain direct far-field sums.
//
// Who needs this: a caller that cannot create device allocations of its own
// at the point where it needs the sums -- for example a solver embedded in a
// larger application that hands this library only device buffers it already
// owns (its own memory pool), or a latency-critical loop where cudaMalloc's
// implicit device synchronisation and cost are not acceptable.  Such a
// caller cannot build an ifgf_plan (plan creation allocates), so this entry
// point takes raw arrays and keeps its working arrays (the weighted densities
// and the field accumulators) in one fixed, file-scope device array instead
// of allocating them.
//
// The array is shared by every call in the process and keeps the last call's
// contents; each call clears what must start at zero.  Calls that overlap on
// the GPU (different streams, or host threads without ordering) race on it.
#include <exception>
#include <mutex>

#include "kernels.h"

namespace ifgf {

namespace {

// Fixed working storage: per node 16 reals of weighted densities and 56 reals
// of field accumulators, in FP64, for up to kNoAllocMaxNodes nodes (~55 MiB).
constexpr int kNoAllocMaxNodes = 100000;
constexpr size_t kNoAllocBytes = (size_t)kNoAllocMaxNodes * (16 + 56) * sizeof(double);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the array, resolved once per device (host code cannot use
// the symbol itself as a device pointer).
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

template <typename T>
__global__ void k_weight_densities(int N, const double* __restrict__ phi, const double* __restrict__ w,
                                   T* __restrict__ a, T* __restrict__ f28) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t < 16 * (size_t)N) a[t] = (T)(phi[t] * w[t / 16]);
  if (t < 56 * (size_t)N) f28[t] = T(0);
}

template <typename T>
__global__ void k_fields_out(size_t n, const T* __restrict__ f, double* __restrict__ out) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t < n) out[t] = (double)f[t];
}

}  // namespace
}  // namespace ifgf

using namespace ifgf;

static ifgf_status noalloc_impl(int32_t n, const double* nodes, const double* normals, const double* weights,
                                const int32_t* leaf_coords, const void* phi, double k_ext, double k_int,
                                int32_t precision, void* f28, ifgf_stream stream) {
  if (n < 1 || !nodes || !normals || !weights || !leaf_coords || !phi || !f28) return IFGF_EINVAL;
  if (!(k_ext > 0) || !(k_int > 0)) return IFGF_EINVAL;
  if (precision != IFGF_FP64 && precision != IFGF_FP32) return IFGF_EINVAL;
  if (n > kNoAllocMaxNodes) {
    set_status_detail(IFGF_EUNSUPPORTED,
                      "ifgf_far_direct_noalloc: n exceeds the fixed working array (at most 100000 nodes)");
    return IFGF_EUNSUPPORTED;
  }
  int dev = 0;
  IFGF_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_status_detail(IFGF_EUNSUPPORTED, "ifgf_far_direct_noalloc: device ordinal beyond 63");
    return IFGF_EUNSUPPORTED;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* ptr = nullptr;
      IFGF_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
      g_scratch_addr[dev] = ptr;
    }
    base = g_scratch_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t el = (precision == IFGF_FP64) ? sizeof(double) : sizeof(float);
  void* a = base;
  void* acc = static_cast<unsigned char*>(base) + 16 * (size_t)n * el;
  const unsigned blocks = (unsigned)((56 * (size_t)n + 255) / 256);
  if (precision == IFGF_FP64)
    k_weight_densities<double><<<blocks, 256, 0, s>>>(n, (const double*)phi, weights, (double*)a, (double*)acc);
  else
    k_weight_densities<float><<<blocks, 256, 0, s>>>(n, (const double*)phi, weights, (float*)a, (float*)acc);
  IFGF_CUDA_TRY(cudaGetLastError());
  IFGF_CUDA_TRY(launch_far_direct_raw(n, nodes, normals, leaf_coords, a, k_ext, k_int, precision, acc, s));
  if (precision == IFGF_FP64)
    k_fields_out<double><<<blocks, 256, 0, s>>>(56 * (size_t)n, (const double*)acc, (double*)f28);
  else
    k_fields_out<float><<<blocks, 256, 0, s>>>(56 * (size_t)n, (const float*)acc, (double*)f28);
  IFGF_CUDA_TRY(cudaGetLastError());
  return IFGF_OK;
}

// No C++ exception leaves the C ABI: the lock can throw std::system_error, reported as
// IFGF_EINTERNAL with its message.
extern "C" ifgf_status ifgf_far_direct_noalloc(int32_t n, const double* nodes, const double* normals,
                                               const double* weights, const int32_t* leaf_coords,
                                               const void* phi, double k_ext, double k_int, int32_t precision,
                                               void* f28, ifgf_stream stream) {
  try {
    return noalloc_impl(n, nodes, normals, weights, leaf_coords, phi, k_ext, k_int, precision, f28, stream);
  } catch (const std::exception& e) {
    set_status_detail(IFGF_EINTERNAL, e.what());
    return IFGF_EINTERNAL;
  } catch (...) {
    set_status_detail(IFGF_EINTERNAL, "ifgf_far_direct_noalloc: unknown exception");
    return IFGF_EINTERNAL;
  }
}
