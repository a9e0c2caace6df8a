"""The allocation-free objective entry point (hpc_objective_noalloc).

Some callers cannot allocate device memory when they need the objective, for
instance code running while a stream is captured into a CUDA graph.  This
entry point takes no context and keeps its scratch in a fixed array inside
the library.  The test calls it through the C ABI twice in a row, on
different inputs, and compares each result with hpc_objective's (labels
equal, objective within the 1e-6 relative tolerance of the other GPU tests)
and with the CPU oracle's.  It runs last and on its own: nothing here
depends on earlier tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as orc
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
        # and against the oracle directly (Eq. 1 in double precision)
        f_o, lab_o = orc.objective(X.cpu().numpy(), C.cpu().numpy(), deg.cpu().numpy(),
                                   want_labels=True)
        assert float(f.item()) == pytest.approx(f_o, rel=RTOL)
        diff = np.flatnonzero(lab.cpu().numpy() != lab_o)
        if diff.size:
            _, d1, d2, _ = orc.assign(X.cpu().numpy()[diff], C.cpu().numpy(), deg.cpu().numpy())
            assert ((d2 - d1) <= 1e-6 * d1).all()
    ctx.close()


def test_noalloc_objective_inside_a_cuda_graph():
    # the use the entry point serves: a call recorded while a stream is
    # captured (no allocation is allowed there), replayed after the rows
    # changed in place; one uncaptured call first, same padded d and k class
    lib = H.load()
    fn = _noalloc(lib)
    n, d, k = 50_001, 32, 40
    X, C, deg = _case(7, n, d, k)
    X2, _, _ = _case(8, n, d, k)
    X1 = X.clone()
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    lab = torch.zeros(n, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    cur = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert fn(_ptr(X), n, d, _ptr(C), k, _ptr(deg), _ptr(f), _ptr(lab), _ptr(st), cur) == H.HPC_OK
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        rc = fn(_ptr(X), n, d, _ptr(C), k, _ptr(deg), _ptr(f), _ptr(lab), _ptr(st),
                ctypes.c_void_p(side.cuda_stream))
    assert rc == H.HPC_OK
    ctx = H.Context(0)
    ctx.set_tensor_cores(0)
    try:
        for src in (X2, X1):
            X.copy_(src)
            f.fill_(-1.0)
            g.replay()
            torch.cuda.synchronize()
            assert int(st.item()) == H.HPC_OK
            lab_ref = torch.empty(n, dtype=torch.int32, device="cuda")
            f_ref = H.hpc_objective(ctx, X, C, deg, labels_out=lab_ref)
            ctx.check_status()
            assert float(f.item()) == pytest.approx(float(f_ref.item()), rel=RTOL)
            assert torch.equal(lab, lab_ref)
            f_o = orc.objective(X.cpu().numpy(), C.cpu().numpy(), deg.cpu().numpy())
            assert float(f.item()) == pytest.approx(f_o, rel=RTOL)
    finally:
        ctx.close()


def test_noalloc_rejects_bad_sizes():
    lib = H.load()
    fn = _noalloc(lib)
    C = torch.zeros((2, 200), device="cuda")
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    X = torch.zeros((4, 200), device="cuda")
    assert fn(_ptr(X), 4, 200, _ptr(C), 2, None, _ptr(f), None, _ptr(st), None) == H.HPC_ERR_ARG
    # each rejected case returns before any launch
    X = torch.zeros((64, 16), device="cuda")
    C = torch.zeros((4, 16), device="cuda")
    base = ctypes.c_void_p(X.data_ptr())
    odd = ctypes.c_void_p(X.data_ptr() + 4)          # not 16-byte aligned
    cases = [
        (odd, 63, 16, _ptr(C), 4, _ptr(f), _ptr(st)),                       # unaligned X
        (base, 64, 16, ctypes.c_void_p(C.data_ptr() + 4), 3, _ptr(f), _ptr(st)),  # unaligned C
        (base, 64, 16, _ptr(C), 0, _ptr(f), _ptr(st)),                      # k < 1
        (base, -1, 16, _ptr(C), 4, _ptr(f), _ptr(st)),                      # n < 0
        (base, 64, 16, _ptr(C), 4, _ptr(f), None),                          # no status_out
        (base, 64, 16, _ptr(C), 4, None, _ptr(st)),                         # no f_out
        (base, 64, 0, _ptr(C), 4, _ptr(f), _ptr(st)),                       # d < 1
    ]
    for Xp, n, d, Cp, k, fp, sp in cases:
        assert fn(Xp, n, d, Cp, k, None, fp, None, sp, None) == H.HPC_ERR_ARG
