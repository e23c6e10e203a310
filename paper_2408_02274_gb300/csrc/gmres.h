// Device GMRES driver (see gmres.cu).
#pragma once
#include <functional>

#include "kernels.h"

namespace ifgf {

// matvec(v, w, stream): w_r = A v_r for the right-hand sides of the solve, device
// [nrhs][4N] complex128 blocks.
using MatvecFn = std::function<cudaError_t(const double*, double*, cudaStream_t)>;

// Solves A y_r = b_r, r < nrhs, with b in p->gm.b [nrhs][4N]; solutions to p->gm.y [nrhs][4N];
// iters[r], relres[r] (host arrays) receive the Krylov dimension and the residual estimate.
// With `precond` (flexible GMRES): z_k = M v_k is stored in p->pc.Z, w = A z_k, and y = Z (H^-1 g).
cudaError_t gmres_run(ifgf_plan_t* p, const MatvecFn& matvec, int nrhs, double tol, int max_iter, int* iters,
                      double* relres, cudaStream_t s, const MatvecFn* precond = nullptr);
int dots_blocks(int64_t n);
// Residual refinement helpers (device [nrhs][4N] complex128 blocks): r = b - w with
// p->gm.scal[rb * 8 + 3] = |r_rb| and p->gm.scal[rb * 8 + 4] = |b_rb| (r may alias w); y += d
// (y -= d with subtract).
cudaError_t gmres_residual(ifgf_plan_t* p, int nrhs, const double* b, const double* w, double* r,
                           cudaStream_t s);
cudaError_t gmres_accumulate(ifgf_plan_t* p, int nrhs, const double* d, double* y, cudaStream_t s, bool subtract);

}  // namespace ifgf
