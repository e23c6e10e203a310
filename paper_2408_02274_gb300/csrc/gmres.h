// Device GMRES driver (see gmres.cu).
#pragma once
#include <functional>

#include "kernels.h"

namespace ifgf {

// matvec(v, w, stream): w = A v for device [4][N] complex128 vectors.
using MatvecFn = std::function<cudaError_t(const double*, double*, cudaStream_t)>;

// Solves A y = b with b in p->gm.b; the solution is written to p->gm.y.
cudaError_t gmres_run(ifgf_plan_t* p, const MatvecFn& matvec, double tol, int max_iter, int* iters,
                      double* relres, cudaStream_t s);
int dots_blocks(int64_t n);

}  // namespace ifgf
