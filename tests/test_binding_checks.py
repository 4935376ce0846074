"""The binding's checks of the tensors whose raw pointers go to the library.

A tensor on the wrong device, of the wrong dtype or too small for what the
library reads or writes through its pointer must raise ValueError before any
library call. These run without a GPU: the checker is exercised on CPU
tensors against a CPU device, and the Context methods on a context object
that has no library handle (a call that got past the checks would fail on
it with a different error)."""
import numpy as np
import pytest
import torch

from paper_2302_07084_gb300 import lne

CPU = torch.device("cpu")


def test_check_tensor_accepts_a_matching_tensor():
    t = torch.zeros((5, 3), dtype=torch.float32)
    assert lne._check_tensor("t", t, CPU, torch.float32, shape=(5, 3), min_rows=5, cols=3, min_numel=15) is t
    assert lne._check_tensor("t", t, CPU, (torch.float64, torch.float32)) is t
    lne._check_tensor("empty", torch.zeros((0, 3)), CPU, cols=3)


@pytest.mark.parametrize("case", ["device", "contiguous", "dtype", "shape", "rows", "cols", "numel", "type"])
def test_check_tensor_rejects(case):
    t = torch.zeros((5, 3), dtype=torch.float32)
    args = dict(device=CPU)
    if case == "device":
        args["device"] = torch.device("cuda", 0)
    elif case == "contiguous":
        t = t.t()
    elif case == "dtype":
        args["dtype"] = torch.int32
    elif case == "shape":
        args["shape"] = (3, 5)
    elif case == "rows":
        args["min_rows"] = 6
    elif case == "cols":
        args["cols"] = 4
    elif case == "numel":
        args["min_numel"] = 16
    else:
        t = np.zeros((5, 3), np.float32)
    with pytest.raises(ValueError):
        lne._check_tensor("t", t, **args)


@pytest.fixture
def ctx():
    """A Context with no library behind it: only the binding's own checks run."""
    c = lne.Context.__new__(lne.Context)
    c.lib = None
    c.h = None
    c.device = 0
    return c


def _csr(n=6, nnz=8):
    return dict(n=n, nnz=nnz, indptr=torch.zeros(n + 1, dtype=torch.int64),
                indices=torch.zeros(nnz, dtype=torch.int32), data=torch.zeros(nnz, dtype=torch.float32))


def _graph():
    return lne.DeviceGraph(np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32), device="cpu")


def test_host_tensors_are_refused_before_the_library_is_called(ctx):
    p = lne.Params(T=1, s=[1.0], samples=10.0, d=4)
    X = torch.zeros((6, 4))
    calls = [
        lambda: ctx.spmm(_csr(), X),
        lambda: ctx.rsvd(_csr(), p),
        lambda: ctx.sparse_sign_spmm(_csr(), 4, 2, 1),
        lambda: ctx.very_sparse_spmm(_csr(), 4, 2.0, 1),
        lambda: ctx.cholqr2(X),
        lambda: ctx.svd_small(torch.eye(4, dtype=torch.float64)),
        lambda: ctx.sparsifier_counts(_graph(), p),
        lambda: ctx.sparsifier_csr(_graph(), p),
        lambda: ctx.propagate(_graph(), p, torch.zeros((2, 4))),
        lambda: ctx.embed(_graph(), p),
        lambda: ctx.macro_f1(torch.zeros((4, 3)), torch.zeros((4, 2), dtype=torch.uint8),
                             torch.arange(2, dtype=torch.int32), torch.arange(2, dtype=torch.int32)),
        lambda: ctx.surrogate_predict(torch.zeros((3, lne.SURROGATE_INPUTS))),
        lambda: ctx.surrogate_fit_scaling(torch.zeros((3, lne.SURROGATE_INPUTS))),
        lambda: ctx.surrogate_grad(torch.zeros((3, lne.SURROGATE_INPUTS)), torch.zeros(3)),
    ]
    for call in calls:
        with pytest.raises(ValueError, match="needs it on cuda"):
            call()


def test_shape_errors_are_refused(ctx):
    with pytest.raises(ValueError, match="square"):
        ctx.svd_small(torch.zeros((3, 4), dtype=torch.float64))
    with pytest.raises(ValueError, match="2-D"):
        ctx.spmm(_csr(), torch.zeros(6))


def test_graph_arrays_are_checked_against_n_and_nnz():
    g = _graph()
    g._c(CPU)                      # consistent arrays pass on their own device
    g.nnz = 3                      # more arcs than indices holds
    with pytest.raises(ValueError, match="indices"):
        g._c(CPU)
    g = _graph()
    g.n = 3                        # indptr too short for n
    with pytest.raises(ValueError, match="indptr"):
        g._c(CPU)
    g = _graph()
    g.indptr = g.indptr.to(torch.int32)
    with pytest.raises(ValueError, match="int64"):
        g._c(CPU)
    with pytest.raises(ValueError):
        _graph()._c(torch.device("cuda", 0))
