"""Host logic of the batched split-BF16 Lloyd launch's CTA plan
(hpc_lloyd_cta_plan, the same code the launch's one-thread planner runs on
the device before every launch): workers of fewer than 16 tiles wait in a
largest-first list that keeps CTAs in proportion to its work; the others
are dealt, largest first, to the set with the least work; every set gets a
contiguous range of CTAs, one each and then one at a time to the set with
the most work per CTA (at most its smallest worker's tiles); a set runs its
workers one after another through the next links; every worker runs
exactly once."""
import numpy as np
import pytest

from paper_2311_04517_gb300 import hpclust as H
from paper_2311_04517_gb300 import synth

SET_CTAS = 16


def work_of(s, k, u):
    uc = np.clip(np.asarray(u, np.int64), 0, 1000)
    return np.maximum(np.asarray(s, np.float64), 1) * np.asarray(k, np.float64) * (uc + 1)


def candidate(work, tiles, ctas, tiny):
    """One candidate plan restated: workers of fewer than `tiny` tiles in the
    list, the greedy deal of the others, greedy CTAs; and its estimate."""
    W = len(work)
    order = sorted(range(W), key=lambda w: (-work[w], w))
    listed = [w for w in order if tiles[w] < tiny]
    rest = [w for w in order if tiles[w] >= tiny]
    lc = 0
    if listed:
        lc = int(np.floor(ctas * sum(work[w] for w in listed) / sum(work) + 0.5))
        lc = min(max(lc, 1), len(listed))
        lc = ctas if not rest else min(lc, ctas - 1)
    tset = ctas - lc
    ns = min(max(1, tset // SET_CTAS), len(rest))
    sums, members = [0.0] * ns, [[] for _ in range(ns)]
    for w in rest:
        b = min(range(ns), key=lambda j: (sums[j], j))
        sums[b] += work[w]
        members[b].append(w)
    gmax = [min(min(tiles[w] for w in m), tset) for m in members]
    g = [1] * ns
    used = ns
    while used < tset:
        cand = [j for j in range(ns) if g[j] < gmax[j]]
        if not cand:
            break
        b = cand[0]
        for j in cand[1:]:
            if sums[j] / g[j] > sums[b] / g[b]:
                b = j
        g[b] += 1
        used += 1
    # the estimate: sets' times, the list to the CTA free first
    free = [sums[j] / g[j] for j in range(ns) for _ in range(g[j])] + [0.0] * (ctas - used)
    mk = max([sums[j] / g[j] for j in range(ns)] + [0.0])
    for w in listed:
        i = int(np.argmin(free))
        free[i] += work[w]
        mk = max(mk, free[i])
    return members, g, listed, mk


def expected_sets(work, tiles, ctas):
    """The plan restated: all in sets, or the small workers in the list,
    whichever has the smaller estimate."""
    a = candidate(work, tiles, ctas, 0)
    if any(t < SET_CTAS for t in tiles):
        b = candidate(work, tiles, ctas, SET_CTAS)
        if b[3] < a[3]:
            return b[:3]
    return a[:3]


def check_plan(s, k, u, ctas):
    W = len(s)
    p = H.lloyd_cta_plan(s, k, u, ctas)
    ct, lst, nxt, nb = p["cta_task"], p["list"], p["next"], p["nblocks"]
    work = work_of(s, k, u)
    tiles = [-(-int(x) // 128) for x in s]
    assert len(ct) == ctas and ((ct >= 0) | (ct == -2)).all()
    members, g, listed = expected_sets(work, tiles, ctas)
    assert lst.tolist() == listed, "the list: the workers of fewer tiles, largest first"
    assert all(tiles[w] < SET_CTAS for w in listed)
    runs = np.zeros(W, np.int64)
    c = 0
    for m, gj in zip(members, g):
        # a contiguous range of CTAs, all starting with the set's first worker
        assert (ct[c:c + gj] == m[0]).all()
        seq, w = [], m[0]
        while w >= 0:
            assert len(seq) <= W, "no cycle"
            seq.append(w)
            w = int(nxt[w])
        assert seq == m, "the set runs its workers in the order dealt"
        for w in seq:
            assert nb[w] == gj and gj <= max(1, tiles[w])
            runs[w] += 1
        c += gj
    assert (ct[c:] == -2).all()
    if listed:
        assert (ct == -2).sum() >= 1, "the list keeps a CTA"
    for w in listed:
        assert nb[w] == 1 and nxt[w] == -1 and not (ct == w).any()
        runs[w] += 1
    assert (runs == 1).all(), "every worker exactly once"
    return p


def test_large_workload_plan_is_near_balanced():
    import bench
    wl = synth.WORKLOADS["large"]
    ws = synth.worker_setup(wl)
    s = np.asarray(ws.s, np.int64)
    k = np.asarray(ws.k, np.int32)
    rng = np.random.default_rng(7)
    for _ in range(10):
        u = np.clip(np.round(14 - 7 * s / s.max() + rng.normal(0, 1, len(s))), 3, 20).astype(np.int32)
        p = check_plan(s, k, u, 152)
        assert len({int(t) for t in p["cta_task"]}) == 152 // SET_CTAS
        # with the counts the plan was made from: within 12% of an even spread
        assert bench.plan_balance(s, k, u, u, 152)["makespan_over_balanced"] < 1.12


@pytest.mark.parametrize("W,ctas", [(1, 152), (2, 3), (128, 152), (128, 40), (64, 304), (5, 5),
                                    (128, 1216), (1, 1), (40, 152)])
def test_plan_shapes(W, ctas):
    rng = np.random.default_rng(W * 1000 + ctas)
    s = rng.integers(1, 2_000_000, W)
    k = rng.integers(1, 512, W)
    u = rng.integers(-3, 3000, W)   # out-of-range updates are clamped
    check_plan(s, k, u, ctas)


def test_one_worker_takes_every_cta_it_can_use():
    p = check_plan([10_000_000], [500], [7], 152)
    assert (p["cta_task"] == 0).sum() == 152 and p["next"][0] == -1
    p = check_plan([1000], [500], [7], 152)   # eight 128-row tiles: at most 8 CTAs
    assert p["nblocks"][0] == 8 and (p["cta_task"] == -2).sum() == 144


def test_small_samples_cap_their_set():
    # a set is held to its smallest worker's tiles (here 20); the CTAs left
    # over go to the other sets
    s = [100_000] * 16 + [2560]
    p = check_plan(s, [100] * 17, [5] * 17, 64)
    assert p["nblocks"][16] <= 20 and len(p["list"]) == 0


def test_tiny_samples_wait_in_the_list():
    # beside large workers, workers of fewer than 16 tiles would hold their
    # sets to eight CTAs: they run alone from the list, which keeps CTAs in
    # proportion to its work, and the sets keep the rest
    s = [200_000] * 30 + [1000] * 10   # eight tiles each
    p = check_plan(s, [100] * 40, [5] * 40, 152)
    assert sorted(p["list"].tolist()) == list(range(30, 40))
    assert (p["cta_task"] == -2).sum() >= 1
    # only small workers: sets of up to eight CTAs each beat one CTA each
    p = check_plan([1000] * 50, [100] * 50, [5] * 50, 152)
    assert len(p["list"]) == 0 and p["nblocks"].max() == 8
    # the list where it is better: many small workers, a few CTAs
    p = check_plan([1000] * 50, [100] * 50, [5] * 50, 40)


def test_bad_arguments():
    with pytest.raises(H.HPCError):
        H.lloyd_cta_plan([], [], [], 10)
    with pytest.raises(H.HPCError):
        H.lloyd_cta_plan([10] * 129, [5] * 129, [0] * 129, 152)
    with pytest.raises(H.HPCError):
        H.lloyd_cta_plan([0], [5], [0], 152)
    with pytest.raises(H.HPCError):
        H.lloyd_cta_plan([10], [5], [0], 0)


def test_plan_balance_even_work_is_balanced():
    # eight equal workers on sixteen CTAs: one set, every worker on its 16
    # CTAs one after another, the balanced time exactly
    import bench
    s = np.full(8, 100_000, np.int64)
    k = np.full(8, 500, np.int32)
    u = np.full(8, 9, np.int32)
    r = bench.plan_balance(s, k, u, u, 16)
    assert r["sets"] == 1 and r["set_ctas"] == 16 and r["list"] == 0
    assert r["makespan_over_balanced"] == pytest.approx(1.0, rel=1e-12)


def test_plan_balance_sees_a_wrong_prediction():
    # a worker that takes more updates than predicted lengthens its set
    import bench
    ws = synth.worker_setup(synth.WORKLOADS["large"])
    s = np.asarray(ws.s, np.int64)
    k = np.asarray(ws.k, np.int32)
    u = np.clip(np.round(14 - 7 * s / s.max()), 3, 15).astype(np.int32)
    r = bench.plan_balance(s, k, u, u, 152)
    assert r["sets"] == 9 and r["set_ctas"] == 152 and r["list"] == 0
    assert 1.0 <= r["makespan_over_balanced"] < 1.12
    late = u.copy()
    w = int(np.argmax(s))
    late[w] = 3 * u[w]
    assert bench.plan_balance(s, k, u, late, 152)["makespan_over_balanced"] > \
        r["makespan_over_balanced"]


def test_plan_balance_with_a_list():
    # sets and a list: the listed workers go to the CTAs free first, so the
    # makespan is at least the largest listed worker and the sets' times
    import bench
    s = np.array([200_000] * 30 + [1000] * 10, np.int64)
    k = np.full(40, 100, np.int32)
    u = np.full(40, 5, np.int32)
    r = bench.plan_balance(s, k, u, u, 152)
    assert r["list"] == 10 and r["sets"] >= 1
    work = s * 100.0 * 6
    assert r["makespan_over_balanced"] * work.sum() / 152 >= work[30:].max() - 1e-6
    assert 1.0 <= r["makespan_over_balanced"] < 1.5
