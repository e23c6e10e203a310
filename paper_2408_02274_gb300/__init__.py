"""GB300 (sm_103a) CBIE-IFGF N-Mueller library: Python binding of the C ABI.

The functions here carry the names of the C entry points in include/ifgf.h
and only marshal arguments: every step of the forward map and the solver
runs in the CUDA library ``libifgf.so`` built in-tree by ``build.py``.
There is no CPU fallback: importing the binding without the library raises.
PyTorch provides device memory and the current stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libifgf.so")

IFGF_OK, IFGF_EINVAL, IFGF_ENOMEM, IFGF_ECUDA, IFGF_ENOCONV, IFGF_ETIMEOUT, IFGF_EUNSUPPORTED, IFGF_EINTERNAL = range(8)
IFGF_FP64, IFGF_FP32, IFGF_MIXED = 0, 1, 2
IFGF_FAR_IFGF, IFGF_FAR_DIRECT = 0, 1
IFGF_PART_NEAR, IFGF_PART_FAR, IFGF_PART_ALL = 1, 2, 3

EXPORTS = ["ifgf_plan_create", "ifgf_plan_destroy", "ifgf_apply", "ifgf_apply_batch", "ifgf_apply_fields",
           "ifgf_apply_direct_patches",
           "bie_solve", "bie_solve_batch", "bie_solve_many", "bie_solve_precond", "bie_rhs", "ifgf_precond_attach",
           "ifgf_precond_get", "ifgf_precond_apply", "ifgf_precond_features", "ifgf_precond_train",
           "ifgf_plan_stats", "ifgf_plan_estimate", "ifgf_set_timing", "ifgf_get_timing", "ifgf_status_string",
           "ifgf_tree_create", "ifgf_tree_destroy", "ifgf_plan_tree", "ifgf_tree_info", "ifgf_tree_perm",
           "ifgf_tree_level", "ifgf_tree_targets", "ifgf_tree_upward", "ifgf_tree_items", "ifgf_far_direct_noalloc", "ifgf_far_field",
           "ifgf_plan_tune", "ifgf_plan_check", "ifgf_plan_inject", "ifgf_plan_set_residual",
           "ifgf_precond_block_jacobi"]


class ifgf_plan_desc(ctypes.Structure):
    _fields_ = [
        ("num_patches", ctypes.c_int32), ("nc", ctypes.c_int32),
        ("nodes", ctypes.POINTER(ctypes.c_double)), ("dxdu", ctypes.POINTER(ctypes.c_double)),
        ("dxdv", ctypes.POINTER(ctypes.c_double)),
        ("ng", ctypes.c_int32), ("fine", ctypes.POINTER(ctypes.c_double)),
        ("k_ext", ctypes.c_double), ("k_int", ctypes.c_double),
        ("eps_ext", ctypes.c_double), ("eps_int", ctypes.c_double),
        ("mu_ext", ctypes.c_double), ("mu_int", ctypes.c_double),
        ("ps", ctypes.c_int32), ("pa", ctypes.c_int32), ("ns0", ctypes.c_int32), ("na0", ctypes.c_int32),
        ("leaf_size", ctypes.c_double), ("min_levels", ctypes.c_int32),
        ("delta", ctypes.c_double), ("n_beta", ctypes.c_int32), ("cov_d", ctypes.c_double),
        ("gs_iters", ctypes.c_int32), ("precision", ctypes.c_int32), ("far_mode", ctypes.c_int32),
        ("max_krylov", ctypes.c_int32), ("batch", ctypes.c_int32), ("max_leaf_pts", ctypes.c_int32),
        ("gmres_scaling", ctypes.c_int32), ("upward_tc", ctypes.c_int32), ("refine", ctypes.c_int32),
        ("fields_per_pass", ctypes.c_int32),
    ]


class ifgf_stats(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("levels", ctypes.c_int32),
        ("boxes", ctypes.c_int32 * 24), ("cones", ctypes.c_int32 * 24),
        ("ns", ctypes.c_int32 * 24), ("na", ctypes.c_int32 * 24),
        ("interactions", ctypes.c_int64 * 24),
        ("leaf_pairs", ctypes.c_int64), ("up_pairs", ctypes.c_int64), ("near_nnz", ctypes.c_int64),
        ("singular_pairs", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
        ("setup_seconds", ctypes.c_double), ("setup_tree_s", ctypes.c_double),
        ("setup_geometry_s", ctypes.c_double), ("setup_near_host_s", ctypes.c_double),
        ("setup_closest_s", ctypes.c_double), ("setup_moments_s", ctypes.c_double),
        ("setup_near_values_s", ctypes.c_double),
    ]


class ifgf_plan_estimate_t(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int32), ("cones", ctypes.c_int64 * 24),
        ("candidate_pairs", ctypes.c_int64), ("near_nnz_max", ctypes.c_int64),
        ("bytes_geometry", ctypes.c_int64), ("bytes_near_max", ctypes.c_int64),
        ("bytes_tables", ctypes.c_int64), ("bytes_coefs", ctypes.c_int64),
        ("bytes_apply", ctypes.c_int64), ("bytes_gmres", ctypes.c_int64),
        ("bytes_plan_max", ctypes.c_int64), ("bytes_setup_peak_max", ctypes.c_int64),
    ]


class IfgfError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = load().ifgf_status_string(status).decode()
        super().__init__(f"{where}: status {status} ({msg})")


_lib = None


def load(path: str = LIB_PATH):
    """Load libifgf.so (raises if it was not built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    lib.ifgf_plan_create.argtypes = [ctypes.POINTER(ifgf_plan_desc), ctypes.POINTER(vp)]
    lib.ifgf_plan_estimate.argtypes = [ctypes.POINTER(ifgf_plan_desc), ctypes.POINTER(ifgf_plan_estimate_t)]
    lib.ifgf_plan_destroy.argtypes = [vp]
    lib.ifgf_apply.argtypes = [vp, vp, vp, vp]
    lib.ifgf_apply_batch.argtypes = [vp, i32, vp, vp, vp]
    lib.ifgf_apply_fields.argtypes = [vp, vp, vp, i32, vp]
    lib.ifgf_apply_direct_patches.argtypes = [vp, vp, vp, ctypes.POINTER(i32), i32, vp]
    lib.bie_solve.argtypes = [vp, vp, ctypes.c_double, i32, vp, ctypes.POINTER(i32),
                              ctypes.POINTER(ctypes.c_double), vp]
    lib.bie_solve_batch.argtypes = [vp, i32, vp, ctypes.c_double, i32, vp, ctypes.POINTER(i32),
                                    ctypes.POINTER(ctypes.c_double), vp]
    fp = ctypes.POINTER(ctypes.c_float)
    lib.bie_solve_precond.argtypes = [vp, i32, vp, ctypes.c_double, i32, vp, ctypes.POINTER(i32),
                                      ctypes.POINTER(ctypes.c_double), vp]
    lib.ifgf_precond_attach.argtypes = [vp, i32, fp, fp, fp, fp]
    lib.bie_rhs.argtypes = [vp, i32, vp, vp, vp]
    lib.ifgf_precond_get.argtypes = [vp, fp, fp, fp, fp]
    lib.ifgf_precond_apply.argtypes = [vp, i32, vp, vp, vp]
    lib.ifgf_precond_features.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    lib.ifgf_precond_train.argtypes = [vp, ctypes.c_int64, vp, vp, i32, i32, ctypes.c_float, ctypes.c_uint64, fp, vp]
    lib.bie_solve_many.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(i32), ctypes.POINTER(vp), ctypes.c_double,
                                   i32, ctypes.POINTER(vp), ctypes.POINTER(ctypes.POINTER(i32)),
                                   ctypes.POINTER(ctypes.POINTER(ctypes.c_double)), ctypes.POINTER(i32),
                                   ctypes.POINTER(vp)]
    lib.ifgf_plan_stats.argtypes = [vp, ctypes.POINTER(ifgf_stats)]
    lib.ifgf_set_timing.argtypes = [vp, i32]
    lib.ifgf_get_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(ctypes.c_int64)]
    lib.ifgf_status_string.argtypes = [i32]
    lib.ifgf_status_string.restype = ctypes.c_char_p
    lib.ifgf_tree_create.argtypes = [vp, i32, ctypes.c_double, i32, ctypes.c_double, i32, i32, i32,
                                     ctypes.POINTER(vp)]
    lib.ifgf_tree_destroy.argtypes = [vp]
    lib.ifgf_plan_tree.argtypes = [vp, ctypes.POINTER(vp)]
    lib.ifgf_tree_info.argtypes = [vp, ctypes.POINTER(i32), vp, ctypes.POINTER(ctypes.c_double)]
    lib.ifgf_tree_perm.argtypes = [vp, vp, vp]
    lib.ifgf_tree_level.argtypes = [vp, i32] + [ctypes.POINTER(i32)] * 4 + [vp, vp, vp]
    lib.ifgf_tree_targets.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_int64), vp, vp, vp]
    lib.ifgf_tree_upward.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_int64), vp, vp, ctypes.POINTER(ctypes.c_int64), vp, vp]
    lib.ifgf_tree_items.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_int64), vp]
    lib.ifgf_far_direct_noalloc.argtypes = [i32, vp, vp, vp, vp, vp, ctypes.c_double, ctypes.c_double, i32, vp, vp]
    lib.ifgf_far_field.argtypes = [vp, i32, vp, i32, vp, vp, vp]
    lib.ifgf_plan_tune.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float), vp]
    lib.ifgf_plan_check.argtypes = [vp, vp]
    lib.ifgf_plan_inject.argtypes = [vp, i32]
    lib.ifgf_plan_set_residual.argtypes = [vp, vp]
    lib.ifgf_precond_block_jacobi.argtypes = [vp, vp]
    for name in EXPORTS:
        if name != "ifgf_status_string":
            getattr(lib, name).restype = ctypes.c_int32
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(int(stream))


def _check(st: int, where: str):
    if st != IFGF_OK:
        raise IfgfError(st, where)


def _plan_n(plan) -> int:
    """Node count N of a plan handle (host-side read of the plan's statistics)."""
    st = ifgf_stats()
    _check(load().ifgf_plan_stats(plan, ctypes.byref(st)), "ifgf_plan_stats")
    return int(st.n)


def _arg(a, dtype: str, numel: int, name: str, cuda: bool = True):
    """Address of `a` once the checks the C ABI cannot make hold: a contiguous array of `dtype`
    ("complex128", "float64", "float32", "int32") with `numel` elements; a tensor on the current
    CUDA device when `cuda`, else a numpy array or a tensor in host or device memory.  Reads
    metadata only (no device work), so it is safe inside CUDA graph capture."""
    if hasattr(a, "data_ptr"):
        if str(a.dtype) != "torch." + dtype:
            raise TypeError(f"{name}: dtype {a.dtype}, expected torch.{dtype}")
        if cuda:
            import torch
            if a.device.type != "cuda" or a.device.index != torch.cuda.current_device():
                raise ValueError(f"{name}: a tensor on the current CUDA device is required, got {a.device}")
        if not a.is_contiguous():
            raise ValueError(f"{name}: the tensor must be contiguous")
        if a.numel() != numel:
            raise ValueError(f"{name}: {a.numel()} elements, expected {numel}")
        return ctypes.c_void_p(a.data_ptr())
    if cuda:
        raise TypeError(f"{name}: a torch CUDA tensor is required, got {type(a).__name__}")
    if not isinstance(a, np.ndarray) or a.dtype != np.dtype(dtype) or not a.flags.c_contiguous:
        raise TypeError(f"{name}: a C-contiguous numpy {dtype} array or a torch tensor is required")
    if a.size != numel:
        raise ValueError(f"{name}: {a.size} elements, expected {numel}")
    return ctypes.c_void_p(a.ctypes.data)


def _nrhs(a, name: str) -> int:
    if len(a.shape) < 1:
        raise ValueError(f"{name}: a leading batch dimension is required")
    return int(a.shape[0])


def ifgf_plan_create(nodes, dxdu, dxdv, fine, num_patches: int, nc: int, k_ext: float, k_int: float,
                     eps_ext: float, eps_int: float, mu_ext: float = 1.0, mu_int: float = 1.0, *,
                     delta: float, ps: int = 3, pa: int = 5, ns0: int = 1, na0: int = 2,
                     leaf_size: float = 0.0, min_levels: int = 0, n_beta: int = 48, cov_d: float = 4.0,
                     gs_iters: int = 20, precision: int = IFGF_FP64, far_mode: int = IFGF_FAR_IFGF,
                     max_krylov: int = 0, batch: int = 0, max_leaf_pts: int = 0,
                     gmres_scaling: int = 0, upward_tc: int = 0, refine: int = 0, fields_per_pass: int = 0):
    """ifgf_plan_create: host arrays in, opaque plan handle (c_void_p) out."""
    lib = load()
    arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in (nodes, dxdu, dxdv, fine)]
    d = _desc(arrs, num_patches, nc, k_ext, k_int, eps_ext, eps_int, mu_ext, mu_int, delta, ps, pa, ns0, na0,
              leaf_size, min_levels, n_beta, cov_d, gs_iters, precision, far_mode, max_krylov, batch,
              max_leaf_pts, gmres_scaling, upward_tc, refine, fields_per_pass)
    h = ctypes.c_void_p()
    _check(lib.ifgf_plan_create(ctypes.byref(d), ctypes.byref(h)), "ifgf_plan_create")
    return h


def _desc(arrs, num_patches, nc, k_ext, k_int, eps_ext, eps_int, mu_ext, mu_int, delta, ps, pa, ns0, na0,
          leaf_size, min_levels, n_beta, cov_d, gs_iters, precision, far_mode, max_krylov, batch, max_leaf_pts,
          gmres_scaling, upward_tc=0, refine=0, fields_per_pass=0):
    ng = int(arrs[3].shape[1])
    return ifgf_plan_desc(num_patches, nc, _dptr(arrs[0]), _dptr(arrs[1]), _dptr(arrs[2]), ng, _dptr(arrs[3]),
                          k_ext, k_int, eps_ext, eps_int, mu_ext, mu_int, ps, pa, ns0, na0, leaf_size,
                          min_levels, delta, n_beta, cov_d, gs_iters, precision, far_mode, max_krylov, batch,
                          max_leaf_pts, gmres_scaling, upward_tc, refine, fields_per_pass)


def ifgf_plan_estimate(nodes, dxdu, dxdv, fine, num_patches: int, nc: int, k_ext: float, k_int: float,
                       eps_ext: float, eps_int: float, mu_ext: float = 1.0, mu_int: float = 1.0, *,
                       delta: float, ps: int = 3, pa: int = 5, ns0: int = 1, na0: int = 2,
                       leaf_size: float = 0.0, min_levels: int = 0, n_beta: int = 48, cov_d: float = 4.0,
                       gs_iters: int = 20, precision: int = IFGF_FP64, far_mode: int = IFGF_FAR_IFGF,
                       max_krylov: int = 0, batch: int = 0, max_leaf_pts: int = 0, gmres_scaling: int = 0,
                       upward_tc: int = 0, refine: int = 0, fields_per_pass: int = 0) -> dict:
    """ifgf_plan_estimate: the device memory ifgf_plan_create would allocate for the same
    arguments (host work only; near-matrix figures are upper bounds)."""
    arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in (nodes, dxdu, dxdv, fine)]
    d = _desc(arrs, num_patches, nc, k_ext, k_int, eps_ext, eps_int, mu_ext, mu_int, delta, ps, pa, ns0, na0,
              leaf_size, min_levels, n_beta, cov_d, gs_iters, precision, far_mode, max_krylov, batch,
              max_leaf_pts, gmres_scaling, upward_tc, refine, fields_per_pass)
    e = ifgf_plan_estimate_t()
    _check(load().ifgf_plan_estimate(ctypes.byref(d), ctypes.byref(e)), "ifgf_plan_estimate")
    out = {name: getattr(e, name) for name, _ in ifgf_plan_estimate_t._fields_ if name != "cones"}
    out["cones"] = list(e.cones[:e.levels + 1])
    return out


def ifgf_plan_destroy(plan):
    _check(load().ifgf_plan_destroy(plan), "ifgf_plan_destroy")


def ifgf_apply(plan, y, out, stream=None):
    """out = A y for torch complex128 CUDA tensors y, out of shape [4, N]."""
    n4 = 4 * _plan_n(plan)
    _check(load().ifgf_apply(plan, _arg(y, "complex128", n4, "y"), _arg(out, "complex128", n4, "out"),
                             _stream(stream)), "ifgf_apply")


def ifgf_apply_batch(plan, y, out, stream=None):
    """out[r] = A y[r] for torch complex128 CUDA tensors y, out of shape [nrhs, 4, N]."""
    nrhs, n4 = _nrhs(y, "y"), 4 * _plan_n(plan)
    _check(load().ifgf_apply_batch(plan, nrhs, _arg(y, "complex128", nrhs * n4, "y"),
                                   _arg(out, "complex128", nrhs * n4, "out"), _stream(stream)), "ifgf_apply_batch")


def ifgf_plan_tune(plan, reps: int = 5, stream=None):
    """Autotune the plan's launch shapes; returns (choices [64] int32, times_ms [128] float32)."""
    ch = np.zeros(64, dtype=np.int32)
    tm = np.zeros(128, dtype=np.float32)
    _check(load().ifgf_plan_tune(plan, int(reps), ch.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 tm.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _stream(stream)),
           "ifgf_plan_tune")
    return ch, tm


def ifgf_plan_check(plan, stream=None):
    """Synchronise the stream and raise IfgfError (IFGF_ETIMEOUT) if a bounded device wait of the
    plan expired since the last check (its device status word is cleared)."""
    _check(load().ifgf_plan_check(plan, _stream(stream)), "ifgf_plan_check")


def ifgf_plan_set_residual(plan, residual):
    """Residual plan of the refinement (None unlinks): the solves form b - A y with its map."""
    _check(load().ifgf_plan_set_residual(plan, residual), "ifgf_plan_set_residual")


def ifgf_precond_block_jacobi(plan, stream=None):
    """Build the block-Jacobi right preconditioner (inverse diagonal blocks) of the plan."""
    _check(load().ifgf_precond_block_jacobi(plan, _stream(stream)), "ifgf_precond_block_jacobi")


def ifgf_plan_inject(plan, which: int):
    """Fault injection for the timeout path: 1 makes the tensor-core upward step skip its first
    MMAs so that its (1 ms) wait expires; 0 turns it off."""
    _check(load().ifgf_plan_inject(plan, int(which)), "ifgf_plan_inject")


def ifgf_far_field(plan, y, dirs, out, stream=None):
    """Far-field pattern E_inf of the scattered field of solutions y (complex128 CUDA tensor
    [nrhs, 4, N] or [4, N]) at unit directions dirs (float64 CUDA tensor [ndirs, 3]) into out
    (complex128 CUDA tensor [nrhs, ndirs, 3] or [ndirs, 3])."""
    n = _plan_n(plan)
    nrhs = 1 if y.dim() == 2 else int(y.shape[0])
    ndirs = int(dirs.shape[0])
    _check(load().ifgf_far_field(plan, nrhs, _arg(y, "complex128", nrhs * 4 * n, "y"), ndirs,
                                 _arg(dirs, "float64", 3 * ndirs, "dirs"),
                                 _arg(out, "complex128", nrhs * ndirs * 3, "out"), _stream(stream)),
           "ifgf_far_field")


def ifgf_apply_direct_patches(plan, y, out, patches, stream=None):
    """out = A y with a direct far sum at the nodes of the listed patches only (torch
    complex128 CUDA tensors [4, N]; patches: distinct patch indices).  Only the columns of
    out at those patches' nodes are defined."""
    q = np.ascontiguousarray(np.asarray(patches, dtype=np.int32))
    n4 = 4 * _plan_n(plan)
    _check(load().ifgf_apply_direct_patches(plan, _arg(y, "complex128", n4, "y"), _arg(out, "complex128", n4, "out"),
                                            q.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(q.size),
                                            _stream(stream)), "ifgf_apply_direct_patches")


def ifgf_apply_fields(plan, phi, f28, which: int = IFGF_PART_ALL, stream=None):
    """Scalar S/D sums: phi [N, 8] complex128 CUDA -> f28 [N, 28] complex128 CUDA."""
    n = _plan_n(plan)
    _check(load().ifgf_apply_fields(plan, _arg(phi, "complex128", 8 * n, "phi"), _arg(f28, "complex128", 28 * n, "f28"),
                                    int(which), _stream(stream)), "ifgf_apply_fields")


def bie_solve(plan, inc, tol: float, max_iter: int, y, stream=None, raise_on_noconv: bool = False):
    """GMRES solve; inc [6, N] and y [4, N] complex128, host (numpy) or CUDA (torch).

    Returns (iterations, relative residual estimate, status)."""
    n = _plan_n(plan)
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    st = load().bie_solve(plan, _arg(inc, "complex128", 6 * n, "inc", cuda=False), float(tol), int(max_iter),
                          _arg(y, "complex128", 4 * n, "y", cuda=False), ctypes.byref(it), ctypes.byref(rr),
                          _stream(stream))
    if st not in (IFGF_OK, IFGF_ENOCONV) or (raise_on_noconv and st == IFGF_ENOCONV):
        raise IfgfError(st, "bie_solve")
    return it.value, rr.value, st


def bie_solve_batch(plan, inc, tol: float, max_iter: int, y, stream=None):
    """Batched GMRES solves; inc [nrhs, 6, N] and y [nrhs, 4, N] complex128, host (numpy) or
    CUDA (torch).  Returns (iterations [nrhs], relative residual estimates [nrhs], status)."""
    nrhs, n = _nrhs(inc, "inc"), _plan_n(plan)
    it = (ctypes.c_int32 * nrhs)()
    rr = (ctypes.c_double * nrhs)()
    st = load().bie_solve_batch(plan, nrhs, _arg(inc, "complex128", nrhs * 6 * n, "inc", cuda=False), float(tol),
                                int(max_iter), _arg(y, "complex128", nrhs * 4 * n, "y", cuda=False), it, rr,
                                _stream(stream))
    if st not in (IFGF_OK, IFGF_ENOCONV):
        raise IfgfError(st, "bie_solve_batch")
    return list(it), list(rr), st


def bie_solve_many(plans, incs, ys, tol: float, max_iter: int, streams=None):
    """Uneven batch: concurrent solves on several plans.  incs[i] [nrhs_i, 6, N_i] and
    ys[i] [nrhs_i, 4, N_i] complex128 (host numpy or CUDA torch); streams: optional list of
    distinct CUDA streams.  Returns (iterations per plan, residuals per plan, statuses, status)."""
    n = len(plans)
    vp = ctypes.c_void_p
    if len(incs) != n or len(ys) != n:
        raise ValueError("bie_solve_many: one inc and one y per plan")
    handles = [p.handle if hasattr(p, "handle") else p for p in plans]
    nr = [_nrhs(a, f"incs[{i}]") for i, a in enumerate(incs)]
    ns = [_plan_n(h) for h in handles]
    inc_p = [_arg(a, "complex128", nr[i] * 6 * ns[i], f"incs[{i}]", cuda=False) for i, a in enumerate(incs)]
    y_p = [_arg(a, "complex128", nr[i] * 4 * ns[i], f"ys[{i}]", cuda=False) for i, a in enumerate(ys)]
    its = [(ctypes.c_int32 * k)() for k in nr]
    rrs = [(ctypes.c_double * k)() for k in nr]
    st = (ctypes.c_int32 * n)()
    it_ptrs = (ctypes.POINTER(ctypes.c_int32) * n)(*[ctypes.cast(a, ctypes.POINTER(ctypes.c_int32)) for a in its])
    rr_ptrs = (ctypes.POINTER(ctypes.c_double) * n)(*[ctypes.cast(a, ctypes.POINTER(ctypes.c_double)) for a in rrs])
    strm = None
    if streams is not None:
        strm = (vp * n)(*[vp(int(getattr(s, "cuda_stream", s))) for s in streams])
    status = load().bie_solve_many(n, (vp * n)(*handles), (ctypes.c_int32 * n)(*nr), (vp * n)(*inc_p), float(tol),
                                   int(max_iter), (vp * n)(*y_p), it_ptrs, rr_ptrs, st, strm)
    if status not in (IFGF_OK, IFGF_ENOCONV):
        raise IfgfError(status, "bie_solve_many")
    return [list(a) for a in its], [list(a) for a in rrs], list(st), status


def _f32(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class Preconditioner:
    """The learned right preconditioner of a plan (ifgf_precond_*): per-patch two-layer
    network, in = 8 Nc^2 features, `hidden` units."""

    def __init__(self, plan, hidden=128, weights=None, seed=0):
        self.plan = plan
        self.hidden = hidden
        self.n_in = 8 * plan.nc * plan.nc
        if weights is None:   # small random first layer, zero output layer: z = v to start
            rng = np.random.default_rng(seed)
            weights = (rng.standard_normal((self.n_in, hidden)) * np.sqrt(2.0 / self.n_in),
                       np.zeros(hidden), np.zeros((hidden, self.n_in)), np.zeros(self.n_in))
        self.set(*weights)

    def set(self, W1, b1, W2, b2):
        arrs = [_f32(a) for a in (W1, b1, W2, b2)]
        _check(load().ifgf_precond_attach(self.plan.handle, int(self.hidden), *[p for _, p in arrs]),
               "ifgf_precond_attach")

    def get(self):
        W1 = np.zeros((self.n_in, self.hidden), np.float32)
        b1 = np.zeros(self.hidden, np.float32)
        W2 = np.zeros((self.hidden, self.n_in), np.float32)
        b2 = np.zeros(self.n_in, np.float32)
        ptrs = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) for a in (W1, b1, W2, b2)]
        _check(load().ifgf_precond_get(self.plan.handle, *ptrs), "ifgf_precond_get")
        return W1, b1, W2, b2

    def apply(self, v, z, stream=None):
        """z = M v for torch complex128 CUDA tensors [nrhs, 4, N]."""
        nrhs, n4 = _nrhs(v, "v"), 4 * self.plan.N
        _check(load().ifgf_precond_apply(self.plan.handle, nrhs, _arg(v, "complex128", nrhs * n4, "v"),
                                         _arg(z, "complex128", nrhs * n4, "z"), _stream(stream)), "ifgf_precond_apply")

    def features(self, v, e, X, T, stream=None):
        """Per-patch training pairs from v = A e ([nrhs, 4, N] complex128 CUDA) into float32 CUDA
        tensors X, T [nrhs * P, in]."""
        nrhs, n4 = _nrhs(v, "v"), 4 * self.plan.N
        nx = nrhs * self.plan.P * self.n_in
        _check(load().ifgf_precond_features(self.plan.handle, nrhs, _arg(v, "complex128", nrhs * n4, "v"),
                                            _arg(e, "complex128", nrhs * n4, "e"), _arg(X, "float32", nx, "X"),
                                            _arg(T, "float32", nx, "T"), _stream(stream)), "ifgf_precond_features")

    def train(self, X, T, steps, batch=256, lr=1e-3, seed=1, stream=None):
        """Adam on float32 CUDA tensors X, T [n, in]; returns the minibatch losses."""
        loss = np.zeros(steps, np.float32)
        nx = _nrhs(X, "X")
        _check(load().ifgf_precond_train(self.plan.handle, nx, _arg(X, "float32", nx * self.n_in, "X"),
                                         _arg(T, "float32", nx * self.n_in, "T"), int(steps), int(batch), float(lr),
                                         int(seed), loss.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                         _stream(stream)), "ifgf_precond_train")
        return loss


def bie_solve_precond(plan, inc, tol: float, max_iter: int, y, stream=None):
    """Flexible GMRES with the attached preconditioner; as bie_solve_batch."""
    nrhs, n = _nrhs(inc, "inc"), _plan_n(plan)
    it = (ctypes.c_int32 * nrhs)()
    rr = (ctypes.c_double * nrhs)()
    st = load().bie_solve_precond(plan, nrhs, _arg(inc, "complex128", nrhs * 6 * n, "inc", cuda=False), float(tol),
                                  int(max_iter), _arg(y, "complex128", nrhs * 4 * n, "y", cuda=False), it, rr,
                                  _stream(stream))
    if st not in (IFGF_OK, IFGF_ENOCONV):
        raise IfgfError(st, "bie_solve_precond")
    return list(it), list(rr), st


def ifgf_plan_stats(plan) -> dict:
    s = ifgf_stats()
    _check(load().ifgf_plan_stats(plan, ctypes.byref(s)), "ifgf_plan_stats")
    D = s.levels
    return {
        "n": s.n, "levels": D,
        "boxes": list(s.boxes[:D + 1]), "cones": list(s.cones[:D + 1]),
        "ns": list(s.ns[:D + 1]), "na": list(s.na[:D + 1]),
        "interactions": list(s.interactions[:D + 1]),
        "leaf_pairs": s.leaf_pairs, "up_pairs": s.up_pairs, "near_nnz": s.near_nnz,
        "singular_pairs": s.singular_pairs, "device_bytes": s.device_bytes,
        "setup_seconds": s.setup_seconds,
        "setup_parts_s": {"tree": s.setup_tree_s, "geometry": s.setup_geometry_s, "near_host": s.setup_near_host_s,
                          "closest": s.setup_closest_s, "moments": s.setup_moments_s,
                          "near_values": s.setup_near_values_s},
    }


def ifgf_set_timing(plan, enable: bool = True):
    _check(load().ifgf_set_timing(plan, int(enable)), "ifgf_set_timing")


TIMED_KINDS = ["prep", "near", "leaf", "up", "target", "combine", "far_direct", "gmres"]


def ifgf_get_timing(plan):
    """{kind: (total ms, timed records)} and the kernel launch count since ifgf_set_timing."""
    ms = (ctypes.c_double * 8)()
    calls = (ctypes.c_int64 * 8)()
    nl = ctypes.c_int64(0)
    _check(load().ifgf_get_timing(plan, ms, calls, ctypes.byref(nl)), "ifgf_get_timing")
    return {k: (ms[i], calls[i]) for i, k in enumerate(TIMED_KINDS)}, nl.value


def ifgf_far_direct_noalloc(nodes, normals, weights, leaf_coords, phi, k_ext: float, k_int: float, f28,
                            precision: int = IFGF_FP64, stream=None):
    """Direct far-field sums without any device allocation (CUDA tensors in, f28 out).

    For callers that cannot allocate device memory where they need the sums
    (an application that owns all device memory, a latency-critical loop): the
    library keeps its working arrays in one fixed device array instead.
    nodes, normals [n, 3] float64; weights [n] float64; leaf_coords [n, 3]
    int32; phi [n, 8] and f28 [n, 28] complex128; n <= 100000.
    """
    n = _nrhs(nodes, "nodes")
    _check(load().ifgf_far_direct_noalloc(n, _arg(nodes, "float64", 3 * n, "nodes"),
                                          _arg(normals, "float64", 3 * n, "normals"),
                                          _arg(weights, "float64", n, "weights"),
                                          _arg(leaf_coords, "int32", 3 * n, "leaf_coords"),
                                          _arg(phi, "complex128", 8 * n, "phi"), float(k_ext), float(k_int),
                                          int(precision), _arg(f28, "complex128", 28 * n, "f28"), _stream(stream)),
           "ifgf_far_direct_noalloc")


class Tree:
    """Host-only octree and cone-segment tables (ifgf_tree_*); no GPU is used."""

    def __init__(self, nodes=None, leaf_size=None, k_max=None, min_levels=0, ns0=1, na0=2, handle=None,
                 owned=True, max_leaf_pts=0):
        lib = load()
        if handle is None:
            x = np.ascontiguousarray(np.asarray(nodes, dtype=np.float64))
            h = ctypes.c_void_p()
            _check(lib.ifgf_tree_create(ctypes.c_void_p(x.ctypes.data), x.shape[0], float(leaf_size),
                                        int(min_levels), float(k_max), int(ns0), int(na0), int(max_leaf_pts),
                                        ctypes.byref(h)),
                   "ifgf_tree_create")
            handle = h
            self.n = x.shape[0]
        self.handle, self.owned = handle, owned
        lv = ctypes.c_int32(0)
        corner = np.zeros(3)
        h1 = ctypes.c_double(0)
        _check(lib.ifgf_tree_info(self.handle, ctypes.byref(lv), ctypes.c_void_p(corner.ctypes.data),
                                  ctypes.byref(h1)), "ifgf_tree_info")
        self.levels, self.corner, self.h1 = lv.value, corner, h1.value

    @classmethod
    def of_plan(cls, plan_handle, n):
        h = ctypes.c_void_p()
        _check(load().ifgf_plan_tree(plan_handle, ctypes.byref(h)), "ifgf_plan_tree")
        t = cls(handle=h, owned=False)
        t.n = n
        return t

    def perm(self):
        perm = np.zeros(self.n, dtype=np.int32)
        lc = np.zeros((self.n, 3), dtype=np.int32)
        _check(load().ifgf_tree_perm(self.handle, ctypes.c_void_p(perm.ctypes.data),
                                     ctypes.c_void_p(lc.ctypes.data)), "ifgf_tree_perm")
        return perm, lc

    def level(self, d: int):
        """(box_coords [nb,3], box_slot_ptr [nb+1], slot_cone [nslots], ns, na)."""
        lib = load()
        nb, nsl, ns, na = (ctypes.c_int32(0) for _ in range(4))
        _check(lib.ifgf_tree_level(self.handle, d, ctypes.byref(nb), ctypes.byref(nsl), ctypes.byref(ns),
                                   ctypes.byref(na), None, None, None), "ifgf_tree_level")
        coords = np.zeros((nb.value, 3), dtype=np.int32)
        ptr = np.zeros(nb.value + 1, dtype=np.int32)
        cones = np.zeros(max(nsl.value, 1), dtype=np.int64)
        _check(lib.ifgf_tree_level(self.handle, d, ctypes.byref(nb), ctypes.byref(nsl), ctypes.byref(ns),
                                   ctypes.byref(na), ctypes.c_void_p(coords.ctypes.data),
                                   ctypes.c_void_p(ptr.ctypes.data), ctypes.c_void_p(cones.ctypes.data)),
               "ifgf_tree_level")
        return coords, ptr, cones[:nsl.value], ns.value, na.value

    def targets(self, d: int):
        """(tgt_ptr [n+1] int64, tgt_slot [ninter], slot_box [nslots]) of level d >= 3."""
        lib = load()
        ni = ctypes.c_int64(0)
        _check(lib.ifgf_tree_targets(self.handle, d, ctypes.byref(ni), None, None, None), "ifgf_tree_targets")
        _, ptr, cones, _, _ = self.level(d)
        tp = np.zeros(self.n + 1, dtype=np.int64)
        ts = np.zeros(max(ni.value, 1), dtype=np.int32)
        sb = np.zeros(max(cones.size, 1), dtype=np.int32)
        _check(lib.ifgf_tree_targets(self.handle, d, ctypes.byref(ni), ctypes.c_void_p(tp.ctypes.data),
                                     ctypes.c_void_p(ts.ctypes.data), ctypes.c_void_p(sb.ctypes.data)),
               "ifgf_tree_targets")
        return tp, ts[:ni.value], sb[:cones.size]

    def upward(self, d: int):
        """(up_cc [ncompact,8,75], up_order [ncompact,8,75], up_task [ntask], up_task_ptr) of
        parent level d (3..D-1)."""
        lib = load()
        nc, nt = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(lib.ifgf_tree_upward(self.handle, d, ctypes.byref(nc), None, None, ctypes.byref(nt), None, None),
               "ifgf_tree_upward")
        cc = np.zeros((max(nc.value, 1), 8, 75), dtype=np.int32)
        order = np.zeros_like(cc)
        task = np.zeros(max(nt.value, 1), dtype=np.int32)
        ptr = np.zeros(nc.value * 4 + 1, dtype=np.int32)
        _check(lib.ifgf_tree_upward(self.handle, d, ctypes.byref(nc), ctypes.c_void_p(cc.ctypes.data),
                                    ctypes.c_void_p(order.ctypes.data), ctypes.byref(nt),
                                    ctypes.c_void_p(task.ctypes.data), ctypes.c_void_p(ptr.ctypes.data)),
               "ifgf_tree_upward")
        return cc[:nc.value], order[:nc.value], task[:nt.value], ptr

    def items(self, d: int):
        """items [nitems, 4] of parent level d (3..D-1): slots of one cone and child set, -1 padded."""
        lib = load()
        ni = ctypes.c_int64(0)
        _check(lib.ifgf_tree_items(self.handle, d, ctypes.byref(ni), None), "ifgf_tree_items")
        it = np.zeros((max(ni.value, 1), 4), dtype=np.int32)
        _check(lib.ifgf_tree_items(self.handle, d, ctypes.byref(ni), ctypes.c_void_p(it.ctypes.data)),
               "ifgf_tree_items")
        return it[:ni.value]

    def close(self):
        if self.handle and self.owned:
            load().ifgf_tree_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Owning wrapper around an ifgf_plan for one Problem-like description."""

    def __init__(self, nodes, dxdu, dxdv, fine, num_patches, nc, k_ext, k_int, eps_ext, eps_int,
                 mu_ext=1.0, mu_int=1.0, **kw):
        self.N = num_patches * nc * nc
        self.nc, self.P = nc, num_patches
        self.handle = ifgf_plan_create(nodes, dxdu, dxdv, fine, num_patches, nc, k_ext, k_int, eps_ext,
                                       eps_int, mu_ext, mu_int, **kw)

    @staticmethod
    def estimate(problem, **kw) -> dict:
        """The device memory a plan for `problem` with these options would take (no GPU work)."""
        x, xu, xv = problem.nodes()
        return ifgf_plan_estimate(x, xu, xv, problem.fine(), problem.num_patches, problem.nc, problem.k_ext,
                                  problem.k_int, problem.eps_ext, problem.eps_int, problem.mu_ext, problem.mu_int,
                                  **kw)

    @classmethod
    def from_problem(cls, problem, **kw):
        x, xu, xv = problem.nodes()
        return cls(x, xu, xv, problem.fine(), problem.num_patches, problem.nc, problem.k_ext, problem.k_int,
                   problem.eps_ext, problem.eps_int, problem.mu_ext, problem.mu_int, **kw)

    def apply(self, y, out, stream=None):
        ifgf_apply(self.handle, y, out, stream)

    def apply_batch(self, y, out, stream=None):
        ifgf_apply_batch(self.handle, y, out, stream)

    def tune(self, reps: int = 5, stream=None):
        return ifgf_plan_tune(self.handle, reps, stream)

    def check(self, stream=None):
        ifgf_plan_check(self.handle, stream)

    def inject(self, which: int):
        ifgf_plan_inject(self.handle, which)

    def block_jacobi(self, stream=None):
        ifgf_precond_block_jacobi(self.handle, stream)

    def precond_apply(self, v, z, stream=None):
        """z = M v (block Jacobi and/or the attached network) for complex128 CUDA tensors [nrhs, 4, N]."""
        nrhs, n4 = _nrhs(v, "v"), 4 * self.N
        _check(load().ifgf_precond_apply(self.handle, nrhs, _arg(v, "complex128", nrhs * n4, "v"),
                                         _arg(z, "complex128", nrhs * n4, "z"), _stream(stream)), "ifgf_precond_apply")

    def set_residual(self, other):
        """Form the refinement residual with `other`'s map (a Plan of the same body, or None);
        `other` is kept alive while linked."""
        ifgf_plan_set_residual(self.handle, other.handle if other is not None else None)
        self._resid = other

    def far_field(self, y, dirs, out, stream=None):
        ifgf_far_field(self.handle, y, dirs, out, stream)

    def apply_direct_patches(self, y, out, patches, stream=None):
        ifgf_apply_direct_patches(self.handle, y, out, patches, stream)

    def solve_batch(self, inc, y, tol=1e-6, max_iter=300, stream=None):
        return bie_solve_batch(self.handle, inc, tol, max_iter, y, stream)

    def solve_precond(self, inc, y, tol=1e-6, max_iter=300, stream=None):
        return bie_solve_precond(self.handle, inc, tol, max_iter, y, stream)

    def rhs(self, inc, b, stream=None):
        """b = right-hand side of the solve for CUDA tensors inc [nrhs, 6, N], b [nrhs, 4, N]."""
        nrhs = _nrhs(inc, "inc")
        _check(load().bie_rhs(self.handle, nrhs, _arg(inc, "complex128", nrhs * 6 * self.N, "inc"),
                              _arg(b, "complex128", nrhs * 4 * self.N, "b"), _stream(stream)), "bie_rhs")

    def fields(self, phi, f28, which=IFGF_PART_ALL, stream=None):
        ifgf_apply_fields(self.handle, phi, f28, which, stream)

    def solve(self, inc, y, tol=1e-6, max_iter=300, stream=None):
        return bie_solve(self.handle, inc, tol, max_iter, y, stream)

    def stats(self):
        return ifgf_plan_stats(self.handle)

    def close(self):
        if self.handle:
            ifgf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
