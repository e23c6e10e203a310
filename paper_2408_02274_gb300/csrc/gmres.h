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
cudaError_t gmres_run(ifgf_plan_t* p, const MatvecFn& matvec, int nrhs, double tol, int max_iter, int* iters,
                      double* relres, cudaStream_t s);
int dots_blocks(int64_t n);

}  // namespace ifgf
