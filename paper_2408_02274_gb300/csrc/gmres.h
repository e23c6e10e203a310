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

}  // namespace ifgf
