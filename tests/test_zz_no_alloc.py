"""The allocation-free objective entry point (hpc_objective_noalloc).

Some callers cannot allocate device memory when they need the objective, for
instance code running while a stream is captured into a CUDA graph.  This
entry point takes no context and keeps its scratch in a fixed array inside
the library.  The test calls it through the C ABI twice in a row, on
different inputs, and compares each result with hpc_objective's (labels
equal, objective within the 1e-6 relative tolerance of the other GPU tests).
It runs last and on its own: nothing here depends on earlier tests.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2311_04517_gb300 import hpclust as H

pytestmark = pytest.mark.gpu
RTOL = 1e-6


def _noalloc(lib):
    fn = lib.hpc_objective_noalloc
    P = ctypes.c_void_p
    fn.argtypes = [P, ctypes.c_int64, ctypes.c_int32, P, ctypes.c_int32, P, P, P, P, P]
    fn.restype = ctypes.c_int
    return fn


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _case(seed, n, d, k):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-10, 10, (k, d))
    X = (mu[rng.integers(0, k, n)] + rng.standard_normal((n, d))).astype(np.float32)
    C = (X[rng.choice(n, k, replace=False)] + 0.1).astype(np.float32)
    deg = np.zeros(k, np.uint8)
    deg[k // 2] = 1
    return torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda(), torch.from_numpy(deg).cuda()


def test_noalloc_objective_matches_hpc_objective_twice():
    ctx = H.Context(0)
    ctx.set_tensor_cores(0)       # compare with the same (CUDA-core) search
    fn = _noalloc(ctx.lib)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed, (n, d, k) in enumerate([(200_003, 16, 25), (70_001, 32, 40)]):
        X, C, deg = _case(seed, n, d, k)
        lab_ref = torch.empty(n, dtype=torch.int32, device="cuda")
        f_ref = H.hpc_objective(ctx, X, C, deg, labels_out=lab_ref)
        ctx.check_status()
        f = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        lab = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
        rc = fn(_ptr(X), n, d, _ptr(C), k, _ptr(deg), _ptr(f), _ptr(lab), _ptr(status), stream)
        assert rc == H.HPC_OK
        torch.cuda.synchronize()
        assert int(status.item()) == H.HPC_OK
        assert float(f.item()) == pytest.approx(float(f_ref.item()), rel=RTOL)
        assert torch.equal(lab, lab_ref)
    ctx.close()


def test_noalloc_rejects_bad_sizes():
    lib = H.load()
    fn = _noalloc(lib)
    C = torch.zeros((2, 200), device="cuda")
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    X = torch.zeros((4, 200), device="cuda")
    assert fn(_ptr(X), 4, 200, _ptr(C), 2, None, _ptr(f), None, _ptr(st), None) == H.HPC_ERR_ARG
