/*
 * ifgf.h -- C ABI of the GB300 (sm_103a) CBIE-IFGF N-Mueller library.
 *
 * The library evaluates the forward map of the discretised indirect
 * N-Mueller boundary integral equation for a dielectric scatterer and solves
 * it with GMRES on the device (Paul & Sideris, "Accelerated 3D Maxwell
 * Integral Equation Solver using the Interpolated Factored Green Function
 * Method": Eq. n_muller with Eqs. k_delta, r_delta, t_delta; the linear
 * system Eq. lin_system).  The far interactions are accelerated with the
 * IFGF method (Sec. III-E to III-I), the near interactions use precomputed
 * singular weights (Sec. III-D) with the local corrections of Sec. III-H.
 *
 * Conventions used by every entry point:
 *  - All sizes are int32 unless stated; N = num_patches * nc * nc nodes.
 *  - Node order is l = j + nc*i + p*nc^2 (Eq. mesh_pts_l): node l of patch p
 *    sits at the parameter point (u_i, u_j), u_k = cos((k + 1/2) pi / nc)
 *    (Eq. cheby_nodes).  The caller samples the surface there.
 *  - Complex numbers are interleaved (re, im) doubles (C99 double _Complex /
 *    std::complex<double> / torch.complex128 layout).
 *  - "device pointer" means memory of the current CUDA device; "host or
 *    device" entry points accept either (detected per call).
 *  - Every function returns an ifgf_status; 0 is success.  No C++ exception
 *    crosses this boundary.  A CUDA error inside apply or solve poisons the
 *    plan: later calls on it return IFGF_ECUDA.
 *  - Time dependence e^{-i omega t}; kappa_s = omega sqrt(eps_s mu_s).
 */
#ifndef IFGF_H
#define IFGF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ifgf_status;
enum {
  IFGF_OK = 0,
  IFGF_EINVAL = 1,        /* a descriptor field or argument is invalid */
  IFGF_ENOMEM = 2,        /* a host or device allocation failed (plan_create only) */
  IFGF_ECUDA = 3,         /* a CUDA call failed; the plan is poisoned */
  IFGF_ENOCONV = 4,       /* GMRES reached max_iter above the tolerance (y still written) */
  IFGF_ETIMEOUT = 5,      /* a bounded device wait expired (ifgf_plan_check, the solves) */
  IFGF_EUNSUPPORTED = 6,  /* the combination of options is not implemented */
  IFGF_EINTERNAL = 7      /* an internal consistency check failed */
};

/* arithmetic of the per-apply work: IFGF_FP64 everything in FP64; IFGF_FP32 everything in FP32
 * (densities, near matrix, fields, IFGF kernels); IFGF_MIXED the IFGF kernels (a)-(c) in FP32 and
 * the densities, near-field weights and matvec, fields and N-Mueller combination in FP64 */
enum { IFGF_FP64 = 0, IFGF_FP32 = 1, IFGF_MIXED = 2 };
enum { IFGF_FAR_IFGF = 0, IFGF_FAR_DIRECT = 1 }; /* far-field algorithm */

typedef struct ifgf_plan_t* ifgf_plan;
typedef void* ifgf_stream;                       /* a cudaStream_t (NULL = legacy default stream) */

/*
 * Plan descriptor.  All pointers are HOST pointers; plan_create copies what
 * it needs, the caller keeps ownership.
 */
typedef struct {
  int32_t num_patches;     /* P >= 1 */
  int32_t nc;              /* Chebyshev nodes per patch direction, 2..24 */
  const double* nodes;     /* [N][3] surface points eta_p(u_i, u_j) */
  const double* dxdu;      /* [N][3] d eta_p / du at the nodes */
  const double* dxdv;      /* [N][3] d eta_p / dv at the nodes; dxdu x dxdv points outward */
  int32_t ng;              /* oversampled geometry grid per direction, nc..48 */
  const double* fine;      /* [P][ng][ng][9]: (eta, d eta/du, d eta/dv) on the ng open Chebyshev
                              grid; the patch between nodes is the Chebyshev interpolant of these
                              samples (used by the singular quadrature of Sec. III-D) */
  double k_ext, k_int;     /* kappa_e, kappa_i > 0 */
  double eps_ext, eps_int; /* permittivities > 0 */
  double mu_ext, mu_int;   /* permeabilities > 0; omega = k_ext / sqrt(eps_ext mu_ext) */
  int32_t ps, pa;          /* interpolation points per cone segment, radial and angular
                              (Remark 2: the paper uses 3 and 5; only 3, 5 is built) */
  int32_t ns0, na0;        /* n_{s;D+1}, n_{a;D+1} (paper: 1, 2), >= 1 */
  double leaf_size;        /* upper bound on the leaf box side H_D; 0 -> 0.25 * 2 pi / k_ext */
  int32_t min_levels;      /* lower bound on D (>= 3; 0 -> 3) */
  double delta;            /* singular-set distance threshold of Eq. patch_sing; must be > 0 */
  int32_t n_beta;          /* Fejer points per direction of the moment rule (Eq. int_moments_cov), 4..96 */
  double cov_d;            /* change-of-variables order d >= 2 (Eq. mk_cov_1) */
  int32_t gs_iters;        /* golden-section iterations per direction (Eq. dist_min); 0 -> 20.
                              The edge snap follows the final bracket, so 10-20 steps find the
                              same closest points after the Newton polish (kernel rows within
                              3e-14 of 60 steps) */
  int32_t precision;       /* IFGF_FP64, IFGF_FP32 or IFGF_MIXED: arithmetic of steps (a)-(d) per apply */
  int32_t far_mode;        /* IFGF_FAR_IFGF or IFGF_FAR_DIRECT (plain O(N^2) far sum) */
  int32_t max_krylov;      /* GMRES basis capacity allocated by plan_create (0 -> 300, <= 1000) */
  int32_t batch;           /* right-hand sides one batched call may carry (ifgf_apply_batch,
                              bie_solve_batch): the per-apply buffers, cone coefficients and GMRES
                              workspace are allocated this many times (0 -> 1, <= 1024) */
  int32_t max_leaf_pts;    /* point-count leaf rule: deepen the octree until no leaf box holds
                              more nodes (0 -> off; thin bodies need it); <= 1e6 */
  int32_t gmres_scaling;   /* 0: GMRES on Eq. n_muller as written; 1: GMRES on A D with D =
                              diag(2/(mu_e+mu_i) on m, 2/(eps_e+eps_i) on j) and y = D z, so the
                              identity parts of both block rows become 1 (a constant right
                              scaling: same solution, residuals of the unscaled system) */
  int32_t upward_tc;       /* 1: the upward step (b) of the FP32 IFGF kernels as TF32 contractions on
                              the tensor cores (tcgen05; same results to FP32 rounding); 0: FP32 SIMT
                              contractions (default: faster here, see the header of k_up_tc) */
  int32_t refine;          /* residual refinement of the solves (bie_solve*), 0..20 sweeps: after
                              GMRES, r = b - A_r y is formed in FP64, A_r the map of the residual
                              plan (ifgf_plan_set_residual; this plan's own map without one), and
                              while |r| / |b| > tol and still falling, GMRES with this plan's map
                              (cold start) solves A d = r to the relative accuracy that brings |r|
                              to tol |b| and y += d.  The solves then report the formed residual,
                              not the Arnoldi estimate, and iters sums the sweeps.  0: GMRES alone.
                              Two more [batch][4N] complex vectors are allocated */
  int32_t fields_per_pass; /* IFGF fields carried per octree traversal (Sec. III, "IFGF for Multiple
                              Densities: Speed-vs-Memory Trade-off", and the Remark "On selection of
                              IFGF approach"); of the 16 sums of Eq. ifgf_sum_em (8 densities x 2
                              kernels): 0 or 16: all in one traversal (IFGF_Vec, the default);
                              8: one kernel per traversal (two traversals, half the interpolation
                              coefficients' memory); 1: one (density, kernel) sum per traversal
                              (IFGF_Seq: sixteen traversals, 1/16 of that memory).  1 and 8 need
                              far_mode IFGF_FAR_IFGF, FP32 IFGF kernels (precision IFGF_FP32 or
                              IFGF_MIXED) and upward_tc 0, else IFGF_EUNSUPPORTED; other values
                              IFGF_EINVAL.  Same sums to FP32 rounding; the autotuner leaves the
                              far-field kernels of such a plan untuned */
} ifgf_plan_desc;

/*
 * Device memory of a plan before it is created (Remark "On selection of IFGF approach": the
 * memory of the interpolation data follows from the relevant cone segments, so it can be known
 * before the run).  Host work only: the octree, cone tables and near-field candidates are
 * built as ifgf_plan_create builds them; no GPU call is made.  The near matrix is bounded by
 * counting every candidate patch of every target as singular (ifgf_plan_create keeps the
 * candidates whose closest point lies within delta), so near_nnz_max, bytes_near_max and the
 * totals are upper bounds; everything else is exact: bytes_plan_max - ifgf_plan_stats'
 * device_bytes = (near_nnz_max - near_nnz) * (8 * sizeof(plan precision) + 4).
 */
typedef struct {
  int32_t levels;                /* D */
  int64_t cones[24];             /* relevant cone segments per level d (index d) */
  int64_t candidate_pairs;       /* (target, candidate patch) pairs: bounds the singular pairs */
  int64_t near_nnz_max;          /* near-matrix nonzeros if every candidate were singular */
  int64_t bytes_geometry;        /* node geometry, sorted copies, permutations, leaf coordinates */
  int64_t bytes_near_max;        /* near values in the plan's precision, columns, row pointers */
  int64_t bytes_tables;          /* per-level octree and cone-segment tables */
  int64_t bytes_coefs;           /* the two cone-coefficient buffers, times batch */
  int64_t bytes_apply;           /* per-apply densities and fields, times batch */
  int64_t bytes_gmres;           /* Krylov basis and GMRES work, times batch */
  int64_t bytes_plan_max;        /* the created plan's device_bytes, upper bound */
  int64_t bytes_setup_peak_max;  /* largest device use during ifgf_plan_create (temporaries
                                    included), upper bound */
} ifgf_plan_estimate_t;

ifgf_status ifgf_plan_estimate(const ifgf_plan_desc* desc, ifgf_plan_estimate_t* out);

/* Counts describing a plan (ifgf_plan_stats). */
typedef struct {
  int32_t n;                 /* nodes */
  int32_t levels;            /* D */
  int32_t boxes[24];         /* relevant boxes per level d = 1..D (index d) */
  int32_t cones[24];         /* relevant cone segments per level */
  int32_t ns[24], na[24];    /* cone counts per level */
  int64_t interactions[24];  /* (target, cousin box) pairs evaluated per level */
  int64_t leaf_pairs;        /* (interpolation point, source) pairs of the leaf step */
  int64_t up_pairs;          /* (parent point, child box) pairs of the upward steps */
  int64_t near_nnz;          /* nonzeros of the near-field matrix (per kernel) */
  int64_t singular_pairs;    /* (target, patch) pairs treated with the moment rule */
  int64_t device_bytes;      /* device memory held by the plan */
  double setup_seconds;      /* wall time of plan_create, and its parts: */
  double setup_tree_s;       /*   host octree, cone segments and their tables */
  double setup_geometry_s;   /*   node geometry and interpolant coefficients (device) */
  double setup_near_host_s;  /*   near-field candidates and matrix structure (host) */
  double setup_closest_s;    /*   closest points (device) */
  double setup_moments_s;    /*   singular moments (device) */
  double setup_near_values_s;/*   near-matrix values (device) */
} ifgf_stats;

/*
 * Build a plan: octree, cone segments and interaction lists on the host
 * (Sec. III-F, steps "determine relevant boxes and cones"), then on the
 * device the node geometry, closest points and singular moments (Sec. III-D)
 * and the near-field matrix with local corrections (Sec. III-H).  The plan
 * owns all device memory it uses; apply and solve allocate nothing.  Runs on
 * the current device, synchronously.  The host part runs on all cores, or on
 * at most IFGF_HOST_THREADS threads when that environment variable holds a
 * positive number; the tables built do not depend on the thread count.
 * Errors: IFGF_EINVAL (descriptor), IFGF_ENOMEM, IFGF_ECUDA,
 * IFGF_EUNSUPPORTED.  On error *out is NULL.
 */
ifgf_status ifgf_plan_create(const ifgf_plan_desc* desc, ifgf_plan* out);

/* Release a plan (NULL is allowed). Synchronises the device. */
ifgf_status ifgf_plan_destroy(ifgf_plan plan);

/*
 * Forward map out = A y, the left-hand side of Eq. n_muller (Sec. IV-A,
 * "forward map").  y and out are DEVICE pointers to [4][N] complex128:
 * the components (m.t1, m.t2, j.t1, j.t2) on the orthonormal frame
 * t1 = eta_u/|eta_u|, t2 = n x t1 at every node; out uses the same layout
 * (projections of the two rows of Eq. n_muller on t1, t2).  Asynchronous on
 * `stream`; y and out must not alias.  Allocates nothing.
 */
ifgf_status ifgf_apply(ifgf_plan plan, const void* y, void* out, ifgf_stream stream);

/*
 * Batched forward map: out_r = A y_r for r = 0 .. nrhs-1 with one launch per kernel (the
 * right-hand side is a grid dimension of every per-apply kernel; the near-field matrix,
 * octree and cone tables are shared).  y, out: DEVICE [nrhs][4][N] complex128,
 * 1 <= nrhs <= the plan's batch, not aliased.  Each out_r equals ifgf_apply on y_r bit for
 * bit.  Asynchronous on `stream`; allocates nothing.  Errors as ifgf_apply, and
 * IFGF_EINVAL for nrhs outside [1, batch].
 */
ifgf_status ifgf_apply_batch(ifgf_plan plan, int32_t nrhs, const void* y, void* out, ifgf_stream stream);

/*
 * Sampled direct reference: the forward map with the far field taken by the plain
 * O(N) sum per target (the sum of Eq. ifgf_sum_em written out, as IFGF_FAR_DIRECT) at the
 * nodes of the listed patches only, and the plan's own near matrix.  For accuracy spot
 * checks of the IFGF forward map at sizes where the full O(N^2) direct sum is too slow.
 * Whole patches are the unit because the N-Mueller combination differentiates the
 * potentials tangentially across each patch (Sec. III, surface divergence and curl).
 * y and out: DEVICE [4][N] complex128 as ifgf_apply; only the entries of out at the nodes
 * p Nc^2 .. (p+1) Nc^2 - 1 of each listed patch p (in all 4 components) are defined.
 * patches: HOST int32 [npatches], distinct patch indices in [0, P), 1 <= npatches <= P.
 * The far sum is computed in FP64 whatever the plan's precision (an FP32 sum over all N
 * sources carries ~sqrt(N) FP32 roundings, 1e-4 at N ~ 3e5: too coarse a reference); the
 * densities, near matrix and fields are the plan's own, so against ifgf_apply on the same
 * plan only the far algorithm differs.  For an FP64 plan the entries equal those of
 * ifgf_apply with far_mode IFGF_FAR_DIRECT bit for bit (each target keeps the full map's
 * coordinate origin, the first node of its aligned run of 128 nodes, and its summation
 * order).  Allocates a device list of target blocks per call and returns after `stream` has
 * finished.  IFGF_EINVAL on a null pointer, y == out, npatches out of range, a patch out of
 * range or repeated; IFGF_ENOMEM if the block list cannot be allocated; IFGF_ECUDA poisons
 * the plan.
 */
ifgf_status ifgf_apply_direct_patches(ifgf_plan plan, const void* y, void* out, const int32_t* patches,
                                      int32_t npatches, ifgf_stream stream);

/*
 * Raw scalar sums for tests: given the eight densities phi (DEVICE [N][8]
 * complex128, order m_x m_y m_z j_x j_y j_z div m div j; Sec. III first
 * paragraph), write f28 (DEVICE [N][28] complex128): S_e[phi_k] (k=0..7),
 * S_i[phi_k], dS_e/dn[phi_k] (k=0..5), dS_i/dn[phi_k] at every node, where
 * `which` selects the part:  IFGF_PART_NEAR (near matrix only),
 * IFGF_PART_FAR (the plan's far algorithm only: the sum of Eq. ifgf_sum_em
 * over sources outside the target's neighbour boxes, with a = phi * omega),
 * IFGF_PART_ALL (both).  Arithmetic in the plan's precision.
 */
enum { IFGF_PART_NEAR = 1, IFGF_PART_FAR = 2, IFGF_PART_ALL = 3 };
ifgf_status ifgf_apply_fields(ifgf_plan plan, const void* phi, void* f28, int32_t which,
                              ifgf_stream stream);

/*
 * Solve A y = b with GMRES (Eq. lin_system; no restart, CGS2 Arnoldi in FP64,
 * y0 = 0), where b = omega^{-1} (n x E^inc, n x H^inc) projected on (t1, t2)
 * (right-hand side of Eq. n_muller).  inc: HOST or DEVICE [6][N] complex128
 * (E_x, E_y, E_z, H_x, H_y, H_z of the incident field at the nodes).
 * y: HOST or DEVICE [4][N] complex128 output.  Stops when the Arnoldi
 * residual estimate |b - A y| / |b| <= tol or after max_iter iterations
 * (<= 1000).  iters / relres (host pointers, may be NULL) receive the
 * iteration count and the final relative residual estimate.  Returns
 * IFGF_ENOCONV if tol was not reached (y holds the last iterate).
 * With the plan's refine > 0, GMRES is followed by residual refinement:
 * relres is then |b - A y| / |b| formed from the map, iters the Krylov
 * dimensions summed over the sweeps, max_iter the bound of each sweep.
 * Synchronises `stream` (one scalar is read back per iteration).
 */
ifgf_status bie_solve(ifgf_plan plan, const void* inc, double tol, int32_t max_iter, void* y,
                      int32_t* iters, double* relres, ifgf_stream stream);

/*
 * nrhs independent solves of Eq. lin_system (as bie_solve) that share every forward map:
 * each GMRES iteration applies A to the current Krylov vectors of all right-hand sides with
 * one batched forward map.  inc: HOST or DEVICE [nrhs][6][N] complex128; y: HOST or DEVICE
 * [nrhs][4][N] complex128; iters, relres: HOST arrays [nrhs] (may be NULL).  A right-hand
 * side whose residual estimate reaches tol keeps its iterate (its Arnoldi state is frozen)
 * while the others continue, up to max_iter.  1 <= nrhs <= the plan's batch.  Returns
 * IFGF_ENOCONV if any right-hand side did not reach tol.  Synchronises `stream` (nrhs x 8
 * scalars are read back per iteration).  No C++ exception leaves the call: a failed host
 * allocation is IFGF_ENOMEM, any other host failure IFGF_EINTERNAL with its message.
 */
ifgf_status bie_solve_batch(ifgf_plan plan, int32_t nrhs, const void* inc, double tol, int32_t max_iter,
                            void* y, int32_t* iters, double* relres, ifgf_stream stream);

/*
 * Uneven batch: independent solves on several plans (different bodies) at once.  Solve i is
 * bie_solve_batch(plans[i], nrhs[i], incs[i], tol, max_iter, ys[i], iters[i], relres[i],
 * streams[i]), each run from its own host thread so that the kernels of all solves share the
 * device concurrently.  All arrays have nplans entries; iters[i] / relres[i] may be NULL (the
 * outer arrays too).  The plans must be distinct and belong to the current device; streams[i]
 * must be distinct, and a NULL entry (or a NULL streams array) makes the call create a
 * non-blocking stream for that solve and destroy it before returning.  status[i] (HOST array,
 * may be NULL) receives each solve's status.  Returns IFGF_OK if every solve reached tol,
 * otherwise the first status other than IFGF_OK and IFGF_ENOCONV, otherwise IFGF_ENOCONV.
 * The message of the first failed solve (plan order) is handed to the calling thread, so that
 * ifgf_status_string of that status shows it.  Returns when all solves have finished.
 */
ifgf_status bie_solve_many(int32_t nplans, const ifgf_plan* plans, const int32_t* nrhs,
                           const void* const* incs, double tol, int32_t max_iter, void* const* ys,
                           int32_t* const* iters, double* const* relres, ifgf_status* status,
                           const ifgf_stream* streams);

/*
 * Device status of a plan.  The one device-side wait of the library, the tensor-core upward
 * step (upward_tc = 1) waiting for its MMAs, gives up after 1 s, records the timeout in the
 * plan's device status word, releases its tensor memory and leaves the step's output unwritten;
 * the context stays usable.  ifgf_plan_check synchronises `stream`, reads and clears that word
 * and returns IFGF_ETIMEOUT (with a message) if a wait expired in work queued on the plan since
 * the last check (the results of those applies are then not valid), else IFGF_OK.  The solves
 * (bie_solve*) check it before they return and report IFGF_ETIMEOUT in the same way.
 */
ifgf_status ifgf_plan_check(ifgf_plan plan, ifgf_stream stream);

/*
 * Residual plan of the refinement (plan field refine): mixed-precision iterative refinement
 * forms r = b - A_r y with `residual`'s map (e.g. an FP64 IFGF plan, or the plain FP64 direct
 * sum, IFGF_FAR_DIRECT, of the same body) while GMRES runs on `plan`'s (FP32) map.  The
 * residual then falls below the FP32 map's own rounding floor, down to tol against A_r.
 * `residual` must have the same nodes (N) and a batch at least `plan`'s, must not itself have a
 * residual plan, must outlive the link (NULL unlinks) and must not be applied by another solve
 * at the same time (bie_solve_many refuses plans that share one).  IFGF_EINVAL otherwise.
 */
ifgf_status ifgf_plan_set_residual(ifgf_plan plan, ifgf_plan residual);

/*
 * Fault injection for the timeout path (no GPU fault involved).  which = 1: the tensor-core
 * upward step issues no MMA for the first unit of each block, so the wait for it expires (the
 * waits of this plan then give up after 1 ms instead of 1 s); which = 0: off.  Applies made
 * while it is on give invalid results and set the status word that ifgf_plan_check reports.
 */
ifgf_status ifgf_plan_inject(ifgf_plan plan, int32_t which);

/*
 * Right-hand side of Eq. lin_system: b_r = omega^{-1} (n x E^inc_r, n x H^inc_r) projected on
 * (t1, t2) for r < nrhs.  inc: DEVICE [nrhs][6][N] complex128, b: DEVICE [nrhs][4][N]
 * complex128 (the vector bie_solve solves for).  Asynchronous on `stream`.
 */
ifgf_status bie_rhs(ifgf_plan plan, int32_t nrhs, const void* inc, void* b, ifgf_stream stream);

/*
 * Learned right preconditioner for flexible GMRES (this library's addition; the paper
 * solves with plain GMRES).  A two-layer network shared by all patches acts on each
 * patch's unknowns: with v_p the 4 Nc^2 complex values of patch p (components
 * m.t1, m.t2, j.t1, j.t2 of its nodes), read as in = 8 Nc^2 reals x (feature
 * f = (c Nc^2 + q) 2 + ri: component c, node q of the patch, real/imaginary part) and
 * s_p = |x|,   z_p = v_p + s_p (W2^T relu(W1^T x / s_p + b1) + b2).
 * W1 [in][hidden], b1 [hidden], W2 [hidden][in], b2 [in] (row-major FP32 on the host);
 * the device keeps FP32 master weights and BF16 copies, and the apply kernel accumulates
 * in FP32.  All-zero W2 and b2 give z = v.
 *
 * ifgf_precond_attach: set (or replace) the weights, hidden in [1, 512]; the first call
 *   allocates the weights and the flexible-GMRES basis (the plan's batch x its Krylov
 *   capacity), a later call must keep `hidden`.  Synchronous.  It also restarts Adam.
 * ifgf_precond_get: copy the FP32 master weights back (HOST arrays; any may be NULL).
 * ifgf_precond_apply: z = M v for DEVICE [nrhs][4][N] complex128 v, z (not aliased).
 * ifgf_precond_features: training pairs from DEVICE [nrhs][4][N] complex128 v and e
 *   (v = A e): rows r P + p of the DEVICE FP32 arrays X, T [nrhs P][in] receive
 *   x / s_p and (e_p - v_p) / s_p (zero rows for s_p = 0).
 * ifgf_precond_train: `steps` Adam steps (beta 0.9, 0.999) on the mean squared error of
 *   the network output against T over minibatches of `batch` rows of (X, T) (DEVICE FP32
 *   [nsamples][in]) drawn with a counter-based generator from `seed`; the minibatch loss
 *   before each step goes to `loss` (HOST [steps], may be NULL).  Allocates its scratch on
 *   the first call (and when `batch` grows).  Synchronises `stream`.
 * bie_solve_precond: as bie_solve_batch with flexible GMRES: z_k = M v_k, w = A z_k,
 *   y = Z (H^-1 g); needs an attached network or a built block-Jacobi preconditioner.
 *
 * Block-Jacobi preconditioner (ifgf_precond_block_jacobi): per patch the exact inverse of
 * the operator's diagonal block A_pp (the 4 Nc^2 unknowns of the patch's nodes, rows and
 * columns; for an IFGF plan its far part is the direct sum that the IFGF approximates),
 * assembled on the device by probing the operator restricted to self-patch sources and
 * inverted by Gauss-Jordan with partial pivoting in FP64; stored as P (4 Nc^2)^2 complex128
 * (allocated with the plan on the first call; also the flexible basis if no network was
 * attached).  Once built, M = A_pp^{-1} per patch, and with a network attached as well
 *   z_p = (A_pp^{-1} v)_p + s_p (W2^T relu(W1^T x / s_p + b1) + b2),
 * a learned correction of the block-Jacobi product, whose training targets
 * (ifgf_precond_features) become (e_p - (A_pp^{-1} v)_p) / s_p.  Synchronises `stream`;
 * IFGF_EINTERNAL (with a message) if a block is singular, IFGF_ENOMEM if it does not fit.
 */
ifgf_status ifgf_precond_block_jacobi(ifgf_plan plan, ifgf_stream stream);
ifgf_status ifgf_precond_attach(ifgf_plan plan, int32_t hidden, const float* W1, const float* b1, const float* W2,
                                const float* b2);
ifgf_status ifgf_precond_get(ifgf_plan plan, float* W1, float* b1, float* W2, float* b2);
ifgf_status ifgf_precond_apply(ifgf_plan plan, int32_t nrhs, const void* v, void* z, ifgf_stream stream);
ifgf_status ifgf_precond_features(ifgf_plan plan, int32_t nrhs, const void* v, const void* e, float* X, float* T,
                                  ifgf_stream stream);
ifgf_status ifgf_precond_train(ifgf_plan plan, int64_t nsamples, const float* X, const float* T, int32_t steps,
                               int32_t batch, float lr, uint64_t seed, float* loss, ifgf_stream stream);
ifgf_status bie_solve_precond(ifgf_plan plan, int32_t nrhs, const void* inc, double tol, int32_t max_iter,
                              void* y, int32_t* iters, double* relres, ifgf_stream stream);

/* Counts and sizes of a plan. */
ifgf_status ifgf_plan_stats(ifgf_plan plan, ifgf_stats* st);

/*
 * Optional CUDA-event timing of the library's kernels, for profiling.
 * ifgf_set_timing(plan, 1) resets the counters and records an event pair
 * around every timed launch on the launch stream from then on (0 stops).
 * ifgf_get_timing synchronises on the recorded events and returns, per kind
 * k = 0 density prep (a0), 1 near matrix (d), 2 leaf step (a), 3 upward
 * step (b), 4 target evaluation (c), 5 combination, 6 direct far sum,
 * 7 GMRES orthogonalisation (per iteration), the summed time ms[k] and the
 * number of timed records calls[k] (arrays of 8), and the number of kernels
 * launched by apply/solve since the reset.  Any pointer may be NULL.
 */
ifgf_status ifgf_set_timing(ifgf_plan plan, int32_t enable);
ifgf_status ifgf_get_timing(ifgf_plan plan, double* ms, int64_t* calls, int64_t* launches);

/*
 * Allocation-free direct far-field sums (this library's own addition; the
 * paper has no counterpart).  For callers that cannot create device
 * allocations where they need the sums -- a solver embedded in an
 * application that owns all device memory through its own pool, or a
 * latency-critical loop that cannot afford cudaMalloc's implicit device
 * synchronisation -- and therefore cannot create a plan.
 *
 * Computes the same scalar far sums as ifgf_apply_fields(plan, phi, f28,
 * IFGF_PART_FAR, ...) of a plan with far_mode = IFGF_FAR_DIRECT: for every
 * node l, the sums over all nodes m whose integer leaf box differs from that
 * of l by more than 1 in some coordinate (outside the neighbour boxes) of
 * G_e, G_i (fields k = 0..7) and dG_e/dn, dG_i/dn at l (k = 0..5) times
 * a_m = phi_m * weights_m.  All pointers are DEVICE pointers:
 *   nodes, normals [n][3] double; weights [n] double (quadrature weights);
 *   leaf_coords [n][3] int32 (e.g. from ifgf_tree_perm); phi [n][8]
 *   complex128; f28 [n][28] complex128 output (same layout as
 *   ifgf_apply_fields).  precision: IFGF_FP64 or IFGF_FP32 arithmetic.
 * The working arrays live in one fixed device array compiled into the
 * library (~55 MiB, held by every device that loads the library until the
 * process exits); n is limited to 100000 nodes: larger n returns
 * IFGF_EUNSUPPORTED, whose ifgf_status_string message names the limit.
 * No cudaMalloc, cudaFree or allocating library routine is called.
 * Targets are taken in runs of 128 consecutive nodes whose first node is
 * the coordinate origin of the run; with IFGF_FP32 the node differences
 * keep their digits only if consecutive nodes are close together (grouped
 * by patch, or in ifgf_tree_perm order): nodes in random order lose up to
 * FP32 epsilon times (body size / leaf size) in relative accuracy.
 * IFGF_EINTERNAL (with a message) if a host lock fails.
 * The first call on a device looks up the array's device address (this call
 * should come before any stream capture).  Every call shares the array and
 * clears what must start at zero; calls that overlap on the GPU race.
 * Asynchronous on `stream`.
 */
ifgf_status ifgf_far_direct_noalloc(int32_t n, const double* nodes, const double* normals,
                                    const double* weights, const int32_t* leaf_coords, const void* phi,
                                    double k_ext, double k_int, int32_t precision, void* f28,
                                    ifgf_stream stream);

/*
 * Far-field pattern of the scattered electric field of a solution (the quantity of the
 * scattering experiments of Sec. IV; the reciprocity check of the batched incidences): with the
 * exterior field representation E^sc = -omega mu_e curl S_e[m] - i (k^2 S_e[j] + grad S_e[div j])
 * (k = kappa_e, e^{-i omega t}), E^sc(r d) = e^{i k r}/r E_inf(d) + O(1/r^2) and
 *   E_inf(d) = -i k omega mu_e (d x F[m]) - i k^2 F[j] + k d F[div j],
 *   F[f] = (1/4 pi) sum_l f(x_l) e^{-i k d.x_l} omega_l  (Nystrom nodes and weights, FP64).
 * y: DEVICE [nrhs][4][N] complex128 solution (the layout of ifgf_apply); dirs: DEVICE [ndirs][3]
 * double unit directions; out: DEVICE [nrhs][ndirs][3] complex128.  1 <= nrhs <= batch,
 * 1 <= ndirs <= 2^24.  Uses the plan's per-apply density buffers (do not overlap with an apply on
 * another stream); asynchronous on `stream`; allocates nothing.  IFGF_EINVAL on invalid
 * arguments; IFGF_ECUDA poisons the plan.
 */
ifgf_status ifgf_far_field(ifgf_plan plan, int32_t nrhs, const void* y, int32_t ndirs, const double* dirs, void* out,
                           ifgf_stream stream);

/*
 * Autotuner (this library's own; the paper runs on CPUs): times, on the plan's own tables and
 * buffers, the launch shapes whose choice changes the forward map's time, and keeps the faster
 * one in the plan for later applies and solves:
 *   - per octree level d of an FP32 or mixed IFGF plan, the target step (c) as a warp per target
 *     or a warp per chunk of 32 targets of one box (choices[d]: 0 or 1; times_ms[2d], [2d+1]:
 *     ms per launch of each);
 *   - the near-field matvec's block size, 128 or 256 threads (choices[25]; times_ms[50], [51]);
 *   - for an FP32 or mixed IFGF plan, the leaf step (a) with SIMT or tensor-pipe (TF32 mma)
 *     density products (choices[30]: 0 or 1; times_ms[60], [61]);
 *   - per parent level d of an FP32 or mixed IFGF plan without the tensor-core option, the
 *     upward step (b) into d by runs of point groups with a block per parent slot, by a warp per
 *     parent slot, or by runs with a block per item of up to four slots of one parent cone
 *     (choices[32 + d]: 0, 1 or 2; times_ms[64 + 2d], [65 + 2d], [100 + d]).
 * reps: timed launches per candidate (after one warm-up), 1..1000.  choices: host int32 [64]
 * or NULL (-1 where not applicable); times_ms: host float [128] or NULL.  Results of later
 * applies are unchanged up to summation order (the target step's grouping differs between its
 * two shapes; the upward step's two shapes sum each parent value in a different order).  Synchronises `stream`; overwrites the plan's per-apply buffers (call it between
 * applies, not during a capture).  IFGF_EINVAL for reps out of range; IFGF_ECUDA poisons the plan.
 */
ifgf_status ifgf_plan_tune(ifgf_plan plan, int32_t reps, int32_t* choices, float* times_ms, ifgf_stream stream);

/* Human-readable message for a status code (static storage). */
const char* ifgf_status_string(ifgf_status s);

/*
 * Host-only octree and cone-segment tables (no GPU work): the setup of
 * Sec. III-F (relevant boxes Eq. rele_boxes, neighbours and cousins Eqs.
 * box_neighbor / box_cousin, cone counts of Remark 2, relevant cone segments
 * Eq. rele_cone_d) for a point set, exposed for inspection and tests.
 * nodes: host [n][3]; k_max: the largest wavenumber the cones must resolve;
 * max_leaf_pts: the point-count leaf rule of the plan descriptor (0 -> off).
 * A tree from ifgf_tree_create is released with ifgf_tree_destroy; the tree
 * of a plan (ifgf_plan_tree) is borrowed and lives as long as the plan.
 * IFGF_EINVAL (here, and from ifgf_plan_create / ifgf_plan_estimate, which
 * build the same tree) also for node coordinates that are not finite, fewer
 * than two distinct points, min_levels above 21 (the octree's depth limit,
 * 21 bits per Morton coordinate) and cone-segment counts that do not fit the
 * cone key's 21-bit fields (n_s or 2 n_a above 2^21: k_max times the body
 * size too large for ns0, na0).
 * Output arrays are caller-owned host arrays; pass NULL to query sizes.
 */
typedef struct ifgf_tree_t* ifgf_tree;
ifgf_status ifgf_tree_create(const double* nodes, int32_t n, double leaf_size, int32_t min_levels,
                             double k_max, int32_t ns0, int32_t na0, int32_t max_leaf_pts, ifgf_tree* out);
ifgf_status ifgf_tree_destroy(ifgf_tree tree);
ifgf_status ifgf_plan_tree(ifgf_plan plan, ifgf_tree* out);
/* levels D, level-1 cube corner [3] and side H_1 */
ifgf_status ifgf_tree_info(ifgf_tree tree, int32_t* levels, double* corner, double* h1);
/* perm [n]: sorted position -> node; leaf_coords [n][3]: integer leaf box of each node */
ifgf_status ifgf_tree_perm(ifgf_tree tree, int32_t* perm, int32_t* leaf_coords);
/* level d (1..D): box count, relevant-cone count, (n_s, n_a), integer box coordinates [nb][3],
 * relevant cones CSR per box (box_slot_ptr [nb+1], slot_cone [nslots] cone keys
 * g1 << 42 | g2 << 21 | g3 for the s-, theta- and phi-cell indices, sorted within a box) */
ifgf_status ifgf_tree_level(ifgf_tree tree, int32_t d, int32_t* nboxes, int32_t* nslots, int32_t* ns,
                            int32_t* na, int32_t* box_coords, int32_t* box_slot_ptr, int64_t* slot_cone);
/* level d (3..D-1) as the parent of level d+1: the upward tables.  ncompact distinct relevant
 * cone keys of level d; up_cc [ncompact][8][75] the child cone (compact index at level d+1, -1
 * where no child box holds it) of each interpolation point and octant; up_order
 * [ncompact][8][75] the points ranked by (warp group, child cone); up_task [ntask] the runs
 * start | len << 8 | octant << 16 per (compact cone, group), up_task_ptr [ncompact*4+1]. */
ifgf_status ifgf_tree_upward(ifgf_tree tree, int32_t d, int64_t* ncompact, int32_t* up_cc, int32_t* up_order,
                             int64_t* ntask, int32_t* up_task, int32_t* up_task_ptr);
/* level d (3..D-1) as the parent of level d+1: the items of the upward step (Sec. III-G step 3;
 * the FP32 step per item and the tensor-core step take one item per block): groups of up to 4
 * slots of level d with one cone key, whose interpolation geometry is therefore shared, taken in
 * the order (set of child octants, slot), so that slots with equal sets of children tend to share
 * an item (a block skips the absent children of each slot); items [nitems][4] slot indices, -1
 * after the last slot of a short item, listed in the order of their first slot.  items may be
 * NULL (count only). */
ifgf_status ifgf_tree_items(ifgf_tree tree, int32_t d, int64_t* nitems, int32_t* items);
/* level d (3..D): per sorted target, the relevant cones (slots of level d) it is evaluated from:
 * tgt_ptr [n+1] (int64), tgt_slot [ninter]; slot_box [nslots] box of each slot */
ifgf_status ifgf_tree_targets(ifgf_tree tree, int32_t d, int64_t* ninter, int64_t* tgt_ptr,
                              int32_t* tgt_slot, int32_t* slot_box);

#ifdef __cplusplus
}
#endif
#endif /* IFGF_H */
