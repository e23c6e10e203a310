// Kernel declarations and launch-argument structs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "plan.h"

namespace ifgf {

// ---- setup (setup_kernels.cu)
__global__ void k_cheb_tables(int n, double* fejer, double* A, double* Dm);
__global__ void k_node_geom(int N, int nc, const double* fejer, NodeGeom g);
__global__ void k_fine_coefs(int ng, const double* A, const double* fine, double* coef);
__global__ void k_closest(int npairs, int nc, int ng, int iters, double delta, const int* pair_tgt,
                          const int* pair_patch, const double* x, const double* coef,
                          const double* unodes, double* uv, uint8_t* singular);
__global__ void k_moments(int nsp, const int* sp_pair, const int* pair_tgt, const int* pair_patch,
                          const double* uvc, int nc, int ng, int nbeta, double cov_d,
                          const double* tb, const double* wb, const double* A, const double* x,
                          const double* nrm, const double* coef, double ke, double ki, double* W);
size_t moments_smem_per_warp(int nc, int ng, int nbeta);
__global__ void k_near_values(int N, int nc, const int64_t* row_ptr, const int* col, const int* pair,
                              const int* sp_of_pair, const double* W, const double* x,
                              const double* nrm, const double* qw, const int* leafc, double ke,
                              double ki, double* val64, float* val32);

// ---- per-apply launchers (return cudaGetLastError of the launches)
struct Materials {
  double ke, ki, eps_e, eps_i, mu_e, mu_i, omega;
};

// a0: y [4][N] complex128 -> phi (orig, plan precision), a_sorted, a_orig (phi * omega)
// (every per-apply launcher takes nrhs right-hand sides as a grid dimension; buffers are
//  [nrhs][...] with the per-right-hand-side strides of the plan)
cudaError_t launch_density_prep(const ifgf_plan_t* p, const double* y, const double* phi_in,
                                cudaStream_t s, int nrhs = 1);
// c-post: f28 + y -> out [4][N] complex128
cudaError_t launch_combine(const ifgf_plan_t* p, const double* y, double* out, cudaStream_t s, int nrhs = 1);
cudaError_t setup_combine_kernels();
// (d): f28 = near * phi   (overwrites f28)
cudaError_t launch_near(const ifgf_plan_t* p, cudaStream_t s, int nrhs = 1);
// far field by the plain direct sum (accumulates into f28)
cudaError_t launch_far_direct(const ifgf_plan_t* p, cudaStream_t s, int nrhs = 1);
// the same sum in FP64 (also for an FP32 plan; densities and fields stay in the plan's
// precision) on listed target ranges: blocks (device, [nblocks][3]) = (origin, lo, hi) with
// origin a multiple of 128 and origin <= lo < hi <= min(origin + 128, N)
cudaError_t launch_far_direct_blocks(const ifgf_plan_t* p, cudaStream_t s, const int* blocks, int nblocks);
cudaError_t launch_far_direct_raw(int N, const double* x, const double* nrm, const int* leafc, const void* a,
                                  double ke, double ki, int precision, void* f28, cudaStream_t s);
// the FP32 target step of level d alone, warp per target (mode 0) or per box chunk (mode 1)
cudaError_t launch_target_level(ifgf_plan_t* p, int d, int mode, cudaStream_t s);
cudaError_t launch_up_level(ifgf_plan_t* p, int d, int mode, cudaStream_t s);
cudaError_t launch_leaf_level(ifgf_plan_t* p, int mode, cudaStream_t s);
// opt the IFGF kernels into the dynamic shared memory they use (once per device)
cudaError_t setup_ifgf_kernels();
// far field by IFGF: (a), then per level (c) and (b) (accumulates into f28)
cudaError_t launch_far_ifgf(ifgf_plan_t* p, cudaStream_t s, int nrhs = 1);
// the same with fields_per_pass 1 or 8: one traversal per group of fields (ifgf_pass.cu)
cudaError_t launch_far_ifgf_pass(ifgf_plan_t* p, cudaStream_t s, int nrhs = 1);
// far-field pattern E_inf [nrhs][ndirs][3] complex128 (out) of the scattered field from the densities
// of the last density preparation (phi64); dirs: device [ndirs][3] unit vectors
cudaError_t launch_far_field(const ifgf_plan_t* p, int nrhs, int ndirs, const double* dirs, double* out,
                             cudaStream_t s);
// zero f28
cudaError_t launch_zero_f28(const ifgf_plan_t* p, cudaStream_t s);
// f28 (plan precision) -> complex128 [N][28]
cudaError_t launch_f28_export(const ifgf_plan_t* p, double* out, cudaStream_t s);

// ---- optional event timing (api.cu)
int timer_begin(ifgf_plan_t* p, int kind, cudaStream_t s);   // -1 when timing is off
void timer_end(ifgf_plan_t* p, int rec, cudaStream_t s);
cudaError_t timer_flush(ifgf_plan_t* p);

// ---- self-patch parts of the operator (near_direct.cu), block-Jacobi preconditioner (blockjacobi.cu)
cudaError_t launch_near_self(const ifgf_plan_t* p, cudaStream_t s, int nrhs = 1);
cudaError_t launch_far_self(const ifgf_plan_t* p, cudaStream_t s, int nrhs = 1);
cudaError_t setup_bj_kernels();
cudaError_t launch_bj_apply(const ifgf_plan_t* p, int nrhs, const double* v, double* z, cudaStream_t s);
cudaError_t bj_build(ifgf_plan_t* p, double* yb, double* ob, int* ipiv, int* err_dev, cudaStream_t s);

// ---- learned preconditioner (precond.cu)
// z = base + s MLP(v / s) per patch (base = v when null; base may equal z)
cudaError_t launch_mlp_apply(const ifgf_plan_t* p, int nrhs, const double* v, double* z, cudaStream_t s,
                             const double* base = nullptr);
// X = v / s, T = (e - base) / s per patch (base = v when null)
cudaError_t launch_mlp_features(const ifgf_plan_t* p, int nrhs, const double* v, const double* e, float* X, float* T,
                                cudaStream_t s, const double* base = nullptr);
cudaError_t mlp_refresh_bf16(ifgf_plan_t* p, cudaStream_t s);
cudaError_t mlp_train(ifgf_plan_t* p, int64_t nsamples, const float* X, const float* T, int steps, int batch, float lr,
                      uint64_t seed, float* loss, cudaStream_t s);

// ---- GMRES helpers (gmres.cu)
cudaError_t launch_rhs(const ifgf_plan_t* p, const double* inc, double* b, cudaStream_t s, int nrhs = 1);
// out = D in for nrhs blocks [4][N] complex128: the first two components (m) times cm, the
// last two (j) times cj; in == out allowed.
cudaError_t launch_block_scale(int N, int nrhs, double cm, double cj, const double* in, double* out,
                               cudaStream_t s);

}  // namespace ifgf
