"""Shared checks of a GPU Lloyd run against the oracle (Algorithm 1 with the
Section 6.5 stop rule), for the GPU parity tests.

Two runs from the same start follow the same trajectory until a row sits at
a near tie (its two nearest centroids within 1e-6 relative in FP64), where
the contract lets the labels differ; after that the runs may part.  A run
that differs from the oracle is therefore accepted only when a lock-step
replay (one update at a time from the oracle's state) finds that the first
difference is such a tie, or a stop test whose relative improvement lies
within 1e-6 of the 1e-4 threshold, and the two runs agree up to that step.
"""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_2311_04517_gb300 import hpclust as H

RTOL = 1e-6
TIE = 1e-6
ATOL_REL = 1e-9


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy()


def assert_centroids(Cg, Co, what=""):
    """Per coordinate: |Cg - Co| <= 1e-6 |Co| + 1e-9 max(1, max |Co|)."""
    Co64 = np.asarray(Co, np.float64)
    Cg64 = np.asarray(Cg, np.float64)
    scale = max(1.0, float(np.abs(Co64).max())) if Co64.size else 1.0
    tol = RTOL * np.abs(Co64) + ATOL_REL * scale
    bad = np.abs(Cg64 - Co64) > tol
    if bad.any():
        i = np.unravel_index(np.argmax(np.abs(Cg64 - Co64) - tol), Co64.shape)
        raise AssertionError(f"{what}: {int(bad.sum())} centroid coordinates off, worst at {i}: "
                             f"{Cg64[i]} vs {Co64[i]}")


def gpu_lloyd(ctx, S, C0, deg0, **kw):
    Sd = S if isinstance(S, torch.Tensor) else dev(S)
    Cg, dg = dev(C0), dev(deg0)
    lab = torch.empty(Sd.shape[0], dtype=torch.int32, device="cuda")
    f, it = H.hpc_lloyd(ctx, Sd, Cg, dg, labels_out=lab, **kw)
    ctx.check_status()
    return dict(C=host(Cg), degenerate=host(dg), labels=host(lab), f=float(host(f)[0]),
                iters=int(host(it)[0]))


def lockstep_divergence(ctx, S, C0, deg0, iters):
    """Steps the oracle and the GPU one update at a time from the same state.
    Returns the first step where the labels differ (only near ties allowed),
    or None; any centroid difference beyond tolerance fails."""
    C, deg = C0.copy(), deg0.copy()
    Sd = dev(S)
    for it in range(iters + 1):
        lab_o, d1, d2, _ = orc.assign(S, C, deg)
        lab = torch.empty(S.shape[0], dtype=torch.int32, device="cuda")
        H.hpc_objective(ctx, Sd, dev(C), dev(deg), labels_out=lab)
        ctx.check_status()
        diff = np.flatnonzero(host(lab) != lab_o)
        if diff.size:
            assert ((d2[diff] - d1[diff]) <= TIE * d1[diff]).all(), "labels differ away from ties"
            return it
        Co, dego = orc.update(S, lab_o, C, deg)
        g = gpu_lloyd(ctx, Sd, C, deg, max_iter=1, rel_tol=0.0)
        assert_centroids(g["C"], Co, f"lockstep step {it}")
        np.testing.assert_array_equal(g["degenerate"], dego)
        C, deg = Co, dego
    return None


def check_parted_run(ctx, S, C0, deg0, g, o):
    """A GPU run g and the oracle's run o from (C0, deg0) that do not agree:
    the first difference must be a near tie, and up to it the runs agree."""
    step = lockstep_divergence(ctx, S, C0, deg0, max(g["iters"], o["iters"]))
    if step is None:
        tr = o["f_trace"]
        it = min(g["iters"], o["iters"])
        ratio = (tr[it - 1] - tr[it]) / tr[it - 1]
        assert abs(ratio - 1e-4) <= 1e-6, "trajectories differ without a near tie"
        step = it
    if step > 0:
        gs = gpu_lloyd(ctx, S, C0, deg0, max_iter=step, rel_tol=0.0)
        os_ = orc.lloyd(S, C0, deg0, max_iter=step, rel_tol=0.0)
        assert gs["iters"] == os_["iters"] == step
        assert_centroids(gs["C"], os_["C"], f"lloyd up to step {step}")
        np.testing.assert_array_equal(gs["degenerate"], os_["degenerate"])
        assert gs["f"] == pytest.approx(os_["f"], rel=RTOL)
    return step
