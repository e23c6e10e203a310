"""The Python binding checks what the C ABI cannot (dtype, device, contiguity, element count)
before it passes a pointer on, so that a host tensor, a complex64 or a transposed view never
reaches a kernel.  Runs without a GPU: the library is replaced by a recorder and the CUDA
tensors by stand-ins that report a CUDA device."""
import ctypes
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2408_02274_gb300 as lib  # noqa: E402

N = 40        # nodes of the fake plan
P = 10        # patches of the fake plan (nc = 2)


class FakeCuda:
    """A CPU tensor that reports device cuda:0 (metadata only; never read on a device)."""

    def __init__(self, t):
        self.t = t
        self.dtype, self.shape = t.dtype, t.shape
        self.device = torch.device("cuda", 0)

    def is_contiguous(self):
        return self.t.is_contiguous()

    def numel(self):
        return self.t.numel()

    def data_ptr(self):
        return self.t.data_ptr()


class Recorder:
    def __init__(self):
        self.calls = []

    def ifgf_plan_stats(self, plan, ref):
        ref._obj.n = N
        return lib.IFGF_OK

    def __getattr__(self, name):
        def fn(*args):
            self.calls.append((name, args))
            return lib.IFGF_OK
        return fn


@pytest.fixture
def rec(monkeypatch):
    r = Recorder()
    monkeypatch.setattr(lib, "load", lambda *a, **k: r)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    return r


def c128(*shape):
    return FakeCuda(torch.zeros(shape, dtype=torch.complex128))


def test_valid_arguments_reach_the_library(rec):
    plan = ctypes.c_void_p(1)
    y, out = c128(4, N), c128(4, N)
    lib.ifgf_apply(plan, y, out, stream=0)
    lib.ifgf_apply_batch(plan, c128(3, 4, N), c128(3, 4, N), stream=0)
    lib.ifgf_apply_direct_patches(plan, y, out, [0, 2], stream=0)
    lib.ifgf_apply_fields(plan, c128(N, 8), c128(N, 28), stream=0)
    lib.bie_solve(plan, np.zeros((6, N), np.complex128), 1e-6, 10, np.zeros((4, N), np.complex128), stream=0)
    lib.bie_solve(plan, c128(6, N), 1e-6, 10, c128(4, N), stream=0)
    lib.bie_solve_batch(plan, c128(2, 6, N), 1e-6, 10, np.zeros((2, 4, N), np.complex128), stream=0)
    lib.bie_solve_precond(plan, c128(1, 6, N), 1e-6, 10, c128(1, 4, N), stream=0)
    lib.bie_solve_many([plan, plan], [c128(1, 6, N), c128(2, 6, N)], [c128(1, 4, N), c128(2, 4, N)], 1e-6, 10)
    x = FakeCuda(torch.zeros((N, 3), dtype=torch.float64))
    lc = FakeCuda(torch.zeros((N, 3), dtype=torch.int32))
    w = FakeCuda(torch.zeros(N, dtype=torch.float64))
    lib.ifgf_far_direct_noalloc(x, x, w, lc, c128(N, 8), 1.0, 2.0, c128(N, 28), stream=0)
    names = [c[0] for c in rec.calls]
    assert names == ["ifgf_apply", "ifgf_apply_batch", "ifgf_apply_direct_patches", "ifgf_apply_fields",
                     "bie_solve", "bie_solve", "bie_solve_batch", "bie_solve_precond", "bie_solve_many",
                     "ifgf_far_direct_noalloc"]
    assert rec.calls[0][1][1].value == y.data_ptr() and rec.calls[0][1][2].value == out.data_ptr()
    assert rec.calls[1][1][1] == 3                        # nrhs from the leading dimension
    assert list(rec.calls[8][1][2]) == [1, 2]             # per-plan right-hand-side counts
    assert rec.calls[9][1][0] == N


def test_plan_and_preconditioner_methods(rec):
    plan = types.SimpleNamespace(handle=ctypes.c_void_p(1), N=N, P=P, nc=2)   # no destructor
    lib.Plan.rhs(plan, c128(2, 6, N), c128(2, 4, N), stream=0)
    with pytest.raises(ValueError):
        lib.Plan.rhs(plan, c128(2, 6, N), c128(1, 4, N), stream=0)
    pc = lib.Preconditioner.__new__(lib.Preconditioner)
    pc.plan, pc.hidden, pc.n_in = plan, 8, 8 * 4
    pc.apply(c128(2, 4, N), c128(2, 4, N), stream=0)
    X = FakeCuda(torch.zeros((2 * P, pc.n_in), dtype=torch.float32))
    pc.features(c128(2, 4, N), c128(2, 4, N), X, X, stream=0)
    with pytest.raises(TypeError):
        pc.features(c128(2, 4, N), c128(2, 4, N), FakeCuda(torch.zeros((2 * P, pc.n_in), dtype=torch.float64)), X, stream=0)
    pc.train(X, X, steps=3, stream=0)
    assert [c[0] for c in rec.calls] == ["bie_rhs", "ifgf_precond_apply", "ifgf_precond_features",
                                         "ifgf_precond_train"]


@pytest.mark.parametrize("bad,err", [
    (lambda: torch.zeros((4, N), dtype=torch.complex128), ValueError),           # host tensor
    (lambda: np.zeros((4, N), np.complex128), TypeError),                       # numpy array
    (lambda: c128(4, N + 1), ValueError),                                       # wrong size
    (lambda: FakeCuda(torch.zeros((4, N), dtype=torch.complex64)), TypeError),  # complex64
    (lambda: FakeCuda(torch.zeros((N, 4), dtype=torch.complex128).T), ValueError),   # transposed view
])
def test_device_entry_points_reject_bad_arrays(rec, bad, err):
    plan = ctypes.c_void_p(1)
    with pytest.raises(err):
        lib.ifgf_apply(plan, bad(), c128(4, N), stream=0)
    with pytest.raises(err):
        lib.ifgf_apply(plan, c128(4, N), bad(), stream=0)
    assert rec.calls == []                                # nothing reached the library


def test_solve_entry_points_check_host_arrays_too(rec):
    plan = ctypes.c_void_p(1)
    inc = np.zeros((6, N), np.complex128)
    with pytest.raises(TypeError):
        lib.bie_solve(plan, inc.astype(np.complex64), 1e-6, 10, np.zeros((4, N), np.complex128), stream=0)
    with pytest.raises(TypeError):
        lib.bie_solve(plan, np.asfortranarray(np.zeros((6, N), np.complex128)), 1e-6, 10,
                      np.zeros((4, N), np.complex128), stream=0)
    with pytest.raises(ValueError):
        lib.bie_solve(plan, inc, 1e-6, 10, np.zeros((4, N - 1), np.complex128), stream=0)
    with pytest.raises(ValueError):
        lib.bie_solve_batch(plan, np.zeros((2, 6, N), np.complex128), 1e-6, 10,
                            np.zeros((3, 4, N), np.complex128), stream=0)
    with pytest.raises(ValueError):
        lib.bie_solve_many([plan], [c128(1, 6, N)], [], 1e-6, 10)
    assert rec.calls == []
