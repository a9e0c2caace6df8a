"""Host logic of the batched split-BF16 Lloyd launch's CTA plan
(hpc_lloyd_cta_plan, the same code the launch's one-thread planner runs on
the device before every launch): every worker runs exactly once, either on
a contiguous group of CTAs of its own or alone from the list; the list is
largest first; the groups' CTAs per worker follow round(work / (0.85
mean)); the launch's CTAs are all used."""
import numpy as np
import pytest

from paper_2311_04517_gb300 import hpclust as H
from paper_2311_04517_gb300 import synth


def work_of(s, k, u):
    uc = np.clip(np.asarray(u, np.int64), 0, 1000)
    return np.maximum(np.asarray(s, np.float64), 1) * np.asarray(k, np.float64) * (uc + 1)


def check_plan(s, k, u, ctas):
    W = len(s)
    p = H.lloyd_cta_plan(s, k, u, ctas)
    ct, lst, nb = p["cta_task"], p["list"], p["nblocks"]
    work = work_of(s, k, u)
    assert len(ct) == ctas and ((ct >= 0) | (ct == -2)).all()
    runs = np.zeros(W, np.int64)
    for w in range(W):
        cs = np.flatnonzero(ct == w)
        if cs.size:  # a group: contiguous CTAs, as many as nblocks
            assert cs.size == nb[w] and (np.diff(cs) == 1).all()
            assert nb[w] <= -(-int(s[w]) // 128)
            runs[w] += 1
    for w in lst:
        assert nb[w] == 1 and not (ct == w).any()
        runs[w] += 1
    assert (runs == 1).all(), "every worker exactly once"
    assert (np.diff(work[lst]) <= 0).all(), "the list is largest first"
    M = 0.85 * work.sum() / ctas
    grouped = [w for w in range(W) if (ct == w).any()]
    for w in grouped:
        assert work[w] >= M
        assert nb[w] <= max(1, int(np.floor(work[w] / M + 0.5)))
    if len(lst):  # listed workers are below M, or were dropped as the smallest groups
        assert work[lst].max() <= max(work[grouped].min() if grouped else np.inf, M)
    # CTAs not in a group take from the list
    assert ((ct == -2).sum() > 0) or len(lst) == 0 or (ct >= 0).sum() == ctas
    return p


def test_large_workload_plan():
    wl = synth.WORKLOADS["large"]
    ws = synth.worker_setup(wl)
    rng = np.random.default_rng(7)
    for _ in range(20):
        u = rng.integers(4, 18, len(ws.s))
        p = check_plan(ws.s, ws.k, u, 152)
        assert len(p["list"]) > 0 and (p["cta_task"] >= 0).sum() > 0


@pytest.mark.parametrize("W,ctas", [(1, 152), (2, 3), (128, 152), (128, 40), (64, 304), (5, 5)])
def test_plan_shapes(W, ctas):
    rng = np.random.default_rng(W * 1000 + ctas)
    s = rng.integers(1, 2_000_000, W)
    k = rng.integers(1, 512, W)
    u = rng.integers(-3, 3000, W)   # out-of-range updates are clamped
    check_plan(s, k, u, ctas)


def test_one_worker_takes_every_cta_it_can_use():
    p = check_plan([10_000_000], [500], [7], 152)
    assert (p["cta_task"] == 0).sum() == 152 and len(p["list"]) == 0
    p = check_plan([1000], [500], [7], 152)   # eight 128-row tiles: at most 8 CTAs
    assert p["nblocks"][0] == 8


def test_bad_arguments():
    with pytest.raises(H.HPCError):
        H.lloyd_cta_plan([], [], [], 10)
    with pytest.raises(H.HPCError):
        H.lloyd_cta_plan([10] * 129, [5] * 129, [0] * 129, 152)
    with pytest.raises(H.HPCError):
        H.lloyd_cta_plan([0], [5], [0], 152)
    with pytest.raises(H.HPCError):
        H.lloyd_cta_plan([10], [5], [0], 0)
