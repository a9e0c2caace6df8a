"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test names what fixes the expected value: a library run (numpy's Philox,
scipy's distance routine), a closed form, a brute-force optimum, a textbook
dynamic programme, an invariant, or a statistical law.  They are chosen so a
plausible slip in the oracle (a dropped term, a wrong sign or index, a
transposed operand, an off-by-one in a draw) fails at least one of them.
"""
import itertools
import json
from pathlib import Path

import numpy as np
import pytest
from scipy.spatial.distance import cdist
from scipy.stats import chisquare

GOLDEN = Path(__file__).resolve().parent / "golden"
M64 = (1 << 64) - 1


# --------------------------------------------------------------------------
# Philox4x64-10 and the stream layout (parallel random numbers, §5.3)
# --------------------------------------------------------------------------
def _numpy_philox_block(key, ctr):
    """numpy's Philox advances its 256-bit counter before each block, so the
    block for counter c comes from numpy state c - 1."""
    c = sum(int(v) << (64 * i) for i, v in enumerate(ctr))
    c = (c - 1) % (1 << 256)
    prev = np.array([(c >> (64 * i)) & M64 for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=prev)
    return [int(v) for v in bg.random_raw(4)]


def test_philox_matches_numpy(orc):
    rng = np.random.default_rng(123)
    cases = [([0, 0], [0, 0, 0, 0]), ([M64, M64], [M64, M64, M64, M64]),
             ([1, 2], [0, 7, 0, 0])]
    for _ in range(20):
        cases.append((list(rng.integers(0, 2**63, 2)), list(rng.integers(0, 2**63, 4))))
    for key, ctr in cases:
        got = [int(v) for v in orc.philox4x64_10(ctr, key)]
        assert got == _numpy_philox_block(key, ctr), (key, ctr)


def test_draw_stream_layout(orc):
    # draw j of (seed, worker, round, tag) = word j%4 of the block at
    # counter (j//4, round, tag, 0) under key (seed, worker)
    for seed, w, r, tag in [(0, 0, 0, 0), (7, 3, 11, 1), (2**40 + 5, 63, 29, 0)]:
        for j in [0, 1, 2, 3, 4, 9, 1023]:
            blk = _numpy_philox_block([seed, w], [j // 4, r, tag, 0])
            assert orc.draw(seed, w, r, tag, j) == blk[j % 4]


def test_sample_rows_and_indices(orc):
    rng = np.random.default_rng(5)
    n, d, s = 1000, 3, 257
    X = rng.standard_normal((n, d)).astype(np.float32)
    S, idx = orc.draw_sample(X, seed=9, worker=2, round_=4, s=s)
    for i in range(s):
        blk = _numpy_philox_block([9, 2], [i // 4, 4, orc.TAG_SAMPLE, 0])
        assert idx[i] == (blk[i % 4] * n) >> 64
    np.testing.assert_array_equal(S, X[idx])


def test_sample_indices_uniform(orc):
    n, s = 7, 70000
    X = np.arange(n, dtype=np.float32).reshape(n, 1)
    _, idx = orc.draw_sample(X, seed=1, worker=0, round_=0, s=s)
    counts = np.bincount(idx, minlength=n)
    assert chisquare(counts).pvalue > 1e-4


# --------------------------------------------------------------------------
# Nearest-centroid assignment (Eq. 1, Algorithm 1)
# --------------------------------------------------------------------------
def test_assign_matches_scipy(orc):
    rng = np.random.default_rng(0)
    for s, d, k in [(500, 2, 5), (300, 16, 25), (64, 7, 1), (50, 3, 4)]:
        S = (rng.standard_normal((s, d)) * 4).astype(np.float32)
        C = (rng.standard_normal((k, d)) * 4).astype(np.float32)
        deg = np.zeros(k, np.uint8)
        if k >= 4:
            deg[[1, k - 1]] = 1
        D = cdist(S.astype(np.float64), C.astype(np.float64), "sqeuclidean")
        D[:, deg.astype(bool)] = np.inf
        lab, d1, d2, f = orc.assign(S, C, deg)
        np.testing.assert_array_equal(lab, np.argmin(D, axis=1))
        np.testing.assert_allclose(d1, D.min(axis=1), rtol=1e-12, atol=1e-12)
        if (~deg.astype(bool)).sum() > 1:
            np.testing.assert_allclose(d2, np.sort(D, axis=1)[:, 1], rtol=1e-12, atol=1e-12)
        assert f == pytest.approx(D.min(axis=1).sum(), rel=1e-12)


def test_assign_ties_go_to_lowest_index(orc):
    S = np.array([[0.0, 0.0], [2.0, 0.0]], np.float32)
    C = np.array([[1.0, 0.0], [1.0, 0.0], [-1.0, 0.0]], np.float32)
    lab, _, _, _ = orc.assign(S, C)
    assert list(lab) == [0, 0]
    lab, _, _, _ = orc.assign(S, C, np.array([1, 0, 0], np.uint8))
    assert list(lab) == [1, 1]


def test_sse_decomposition_identity(orc):
    # f(C,X) = sum_j [ sum_{i in j} ||x_i - m_j||^2 + n_j ||m_j - c_j||^2 ]
    rng = np.random.default_rng(2)
    X = (rng.standard_normal((2000, 5)) * 3 + 1).astype(np.float32)
    C = (rng.standard_normal((6, 5)) * 3).astype(np.float32)
    f, lab = orc.objective(X, C, want_labels=True)
    Xd = X.astype(np.float64)
    total = 0.0
    for j in range(6):
        m = lab == j
        if not m.any():
            continue
        mj = Xd[m].mean(axis=0)
        total += ((Xd[m] - mj) ** 2).sum() + m.sum() * ((mj - C[j].astype(np.float64)) ** 2).sum()
    assert f == pytest.approx(total, rel=1e-11)


def test_objective_empty_and_excludes_degenerate(orc):
    C = np.array([[0.0, 0.0], [10.0, 10.0]], np.float32)
    assert orc.objective(np.zeros((0, 2), np.float32), C) == 0.0
    X = np.array([[9.0, 9.0]], np.float32)
    assert orc.objective(X, C) == pytest.approx(2.0)
    assert orc.objective(X, C, np.array([0, 1], np.uint8)) == pytest.approx(162.0)


# --------------------------------------------------------------------------
# Lloyd (Algorithm 1) with the stop rule of §6.5
# --------------------------------------------------------------------------
def _brute_force_optimum(X, k):
    """Minimum of Eq. 1 over every assignment of n points to k labels."""
    n = X.shape[0]
    labs = np.array(list(itertools.product(range(k), repeat=n)), dtype=np.int64)
    Xd = X.astype(np.float64)
    onehot = np.eye(k)[labs]                      # (M, n, k)
    counts = onehot.sum(axis=1)                   # (M, k)
    sums = np.einsum("mnk,nd->mkd", onehot, Xd)   # (M, k, d)
    means = sums / np.maximum(counts, 1)[:, :, None]
    resid = Xd[None, :, :] - np.take_along_axis(means, labs[:, :, None], axis=1)
    obj = (resid ** 2).sum(axis=(1, 2))
    b = int(np.argmin(obj))
    return obj[b], labs[b], means[b]


@pytest.mark.parametrize("n,k,d,seed", [(9, 2, 2, 0), (10, 3, 2, 1), (12, 3, 1, 2), (11, 2, 3, 3)])
def test_lloyd_against_brute_force(orc, n, k, d, seed):
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((n, d)) * 2 + rng.integers(-3, 4, (n, 1))).astype(np.float32)
    fstar, labs, means = _brute_force_optimum(X, k)
    # the optimal partition's means are a Lloyd fixed point with objective f*
    r = orc.lloyd(X, means.astype(np.float32))
    assert r["rc"] == 0
    assert r["f"] == pytest.approx(fstar, rel=1e-9)
    np.testing.assert_array_equal(r["labels"], labs)
    # no Lloyd run, from any K-means++ start, goes below the optimum
    for sd in range(25):
        init = orc.kmeanspp(X, np.zeros((k, d), np.float32), np.ones(k, np.uint8), L=3, seed=sd)
        r = orc.lloyd(X, init["C"], init["degenerate"])
        assert r["f"] >= fstar * (1 - 1e-12)


def test_lloyd_k1_closed_form(orc):
    rng = np.random.default_rng(7)
    X = (rng.standard_normal((5000, 6)) * 2 + 5).astype(np.float32)
    r = orc.lloyd(X, X[:1].copy())
    mean = X.astype(np.float64).mean(axis=0)
    scatter = ((X.astype(np.float64) - mean) ** 2).sum()
    np.testing.assert_array_equal(r["C"][0], mean.astype(np.float32))
    assert r["f"] == pytest.approx(scatter, rel=1e-10)
    # update 1 reaches the mean; update 2 changes nothing, so the assignment
    # after it shows a zero improvement and stops
    assert r["iters"] == 2


def test_lloyd_objective_never_increases(orc):
    rng = np.random.default_rng(11)
    for trial in range(6):
        k = [3, 5, 10, 25, 7, 2][trial]
        X = (rng.standard_normal((3000, 4)) * rng.uniform(0.5, 2)
             + rng.uniform(-10, 10, (3000 // 100 + 1, 4)).repeat(100, axis=0)[:3000]).astype(np.float32)
        init = orc.kmeanspp(X, np.zeros((k, 4), np.float32), np.ones(k, np.uint8), seed=trial)
        r = orc.lloyd(X, init["C"], init["degenerate"], rel_tol=0.0, max_iter=60)
        tr = r["f_trace"]
        assert np.all(np.diff(tr) <= 1e-9 * tr[:-1])


def test_lloyd_update_is_mean_of_members(orc):
    rng = np.random.default_rng(3)
    X = (rng.standard_normal((4000, 8)) * 3).astype(np.float32)
    C0 = X[:12].copy()
    lab0, _, _, _ = orc.assign(X, C0)
    r = orc.lloyd(X, C0, max_iter=1)
    assert r["iters"] == 1
    for j in range(12):
        m = lab0 == j
        want = X[m].astype(np.float64).mean(axis=0).astype(np.float32)
        np.testing.assert_array_equal(r["C"][j], want)


def test_lloyd_empty_cluster_goes_degenerate(orc):
    X = np.array([[0, 0], [0.1, 0], [5, 5], [5.1, 5]], np.float32)
    C0 = np.array([[0, 0], [5, 5], [100, 100]], np.float32)
    r = orc.lloyd(X, C0)
    assert list(r["degenerate"]) == [0, 0, 1]
    np.testing.assert_array_equal(r["C"][2], C0[2])     # keeps its value, excluded
    assert set(r["labels"]) == {0, 1}


def test_lloyd_stop_rule_and_cap(orc):
    rng = np.random.default_rng(4)
    X = (rng.standard_normal((2000, 2)) * 5).astype(np.float32)
    C0 = X[:8].copy()
    r = orc.lloyd(X, C0, rel_tol=1e-4)
    tr = r["f_trace"]
    it = r["iters"]
    # stopped at the first assignment whose relative improvement fell below 1e-4
    assert (tr[it - 1] - tr[it]) < 1e-4 * tr[it - 1]
    assert all((tr[i - 1] - tr[i]) >= 1e-4 * tr[i - 1] for i in range(1, it))
    r3 = orc.lloyd(X, C0, rel_tol=0.0, max_iter=3)
    assert r3["iters"] == 3
    r0 = orc.lloyd(X, C0, max_iter=0)
    assert r0["iters"] == 0
    np.testing.assert_array_equal(r0["C"], C0)


def test_lloyd_all_degenerate_is_an_error(orc):
    X = np.zeros((4, 2), np.float32)
    r = orc.lloyd(X, np.zeros((2, 2), np.float32), np.ones(2, np.uint8))
    assert r["rc"] == orc.ERR_DEGENERATE_ALL


def _dp_1d_optimum(x, k):
    """Textbook O(k n^2) dynamic programme: on the line an optimal k-partition
    of sorted points is contiguous."""
    x = np.sort(x.astype(np.float64))
    n = len(x)
    p1 = np.concatenate([[0.0], np.cumsum(x)])
    p2 = np.concatenate([[0.0], np.cumsum(x * x)])

    def cost(a, b):  # scatter of x[a:b]
        m = b - a
        s = p1[b] - p1[a]
        return (p2[b] - p2[a]) - s * s / m

    INF = np.inf
    D = np.full((k + 1, n + 1), INF)
    arg = np.zeros((k + 1, n + 1), dtype=int)
    D[0, 0] = 0.0
    for j in range(1, k + 1):
        for i in range(j, n + 1):
            for m in range(j - 1, i):
                v = D[j - 1, m] + cost(m, i)
                if v < D[j, i]:
                    D[j, i] = v
                    arg[j, i] = m
    bounds = []
    i = n
    for j in range(k, 0, -1):
        m = arg[j, i]
        bounds.append((m, i))
        i = m
    means = np.array([x[a:b].mean() for a, b in reversed(bounds)])
    return D[k, n], means


def test_dp_matches_brute_force_on_the_line():
    rng = np.random.default_rng(8)
    x = rng.standard_normal(10).astype(np.float32) * 3
    f_dp, _ = _dp_1d_optimum(x, 3)
    f_bf, _, _ = _brute_force_optimum(x.reshape(-1, 1), 3)
    assert f_dp == pytest.approx(f_bf, rel=1e-10)


def test_lloyd_against_1d_dynamic_programme(orc):
    rng = np.random.default_rng(9)
    x = np.concatenate([rng.normal(-6, 1, 30), rng.normal(0, 0.7, 25), rng.normal(5, 1.5, 35)])
    x = x.astype(np.float32)
    X = x.reshape(-1, 1)
    fstar, means = _dp_1d_optimum(x, 3)
    r = orc.lloyd(X, means.astype(np.float32).reshape(-1, 1))
    assert r["f"] == pytest.approx(fstar, rel=1e-9)
    for sd in range(20):
        init = orc.kmeanspp(X, np.zeros((3, 1), np.float32), np.ones(3, np.uint8), seed=sd)
        r = orc.lloyd(X, init["C"], init["degenerate"])
        assert r["f"] >= fstar * (1 - 1e-12)


# --------------------------------------------------------------------------
# K-means++ (§3, §6.5): D^2 draw, greedy candidates, partial reseeding
# --------------------------------------------------------------------------
def test_fixed_point_grid(orc):
    assert orc.fixed_scale(1.0, 1) == 60          # 1 = 0.5*2^1, bit_length(1)=1
    assert orc.quant(1.0, 60) == 2**60
    assert orc.quant(0.75, 3) == 6
    assert orc.quant(0.74, 3) == 5                # floor, not round
    # the largest sum stays below 2^62 even at the extremes
    for M, s in [(3.0e38, 2**40), (1e-40, 3), (7.5, 1_048_576)]:
        F = orc.fixed_scale(M, s)
        assert s * orc.quant(M, F) < 2**62


def test_d2_draw_interval_boundaries(orc):
    # weights 1,2,3,4: row i is drawn iff r lies in
    # [ceil(P_{i-1} 2^64 / Q), ceil(P_i 2^64 / Q)), P = running sum, Q = 10 units
    w = np.array([1, 2, 3, 4], np.float32)
    P = [0, 1, 3, 6, 10]
    for i in range(4):
        lo = -(-(P[i] << 64) // 10)
        hi = -(-(P[i + 1] << 64) // 10)
        assert orc.d2_pick(w, lo) == i
        assert orc.d2_pick(w, hi - 1) == i
    assert orc.d2_pick(np.zeros(3, np.float32), 12345) == -1


def test_d2_draw_frequencies_chi_square(orc):
    w = np.array([0, 1.5, 3, 0.25, 7, 2, 0, 4.5, 1, 9], np.float32)
    rng = np.random.default_rng(1)
    N = 200_000
    r = rng.integers(0, 2**63, size=N, dtype=np.int64).astype(np.uint64) * np.uint64(2) \
        + rng.integers(0, 2, size=N).astype(np.uint64)
    picks = np.array([orc.d2_pick(w, int(v)) for v in r])
    counts = np.bincount(picks, minlength=len(w))
    assert counts[0] == 0 and counts[6] == 0        # zero weight: never drawn
    nz = w > 0
    exp = w[nz].astype(np.float64) / w[nz].sum() * N
    assert chisquare(counts[nz], exp).pvalue > 1e-4


def _fp64_d2(S, C):
    return cdist(S.astype(np.float64), C.astype(np.float64), "sqeuclidean").min(axis=1)


def test_kmeanspp_greedy_picks_smallest_potential(orc):
    rng = np.random.default_rng(12)
    S = np.concatenate([rng.normal(c, 1.0, (200, 3)) for c in (-8, -2, 3, 9)]).astype(np.float32)
    k, L = 6, 3
    res = orc.kmeanspp(S, np.zeros((k, 3), np.float32), np.ones(k, np.uint8), L=L, seed=4)
    assert res["rc"] == 0 and not res["degenerate"].any()
    C = res["C"]
    # every centroid is a sample row
    for j in range(k):
        assert (S == C[j]).all(axis=1).any()
    live = [0]
    for j in range(1, k):
        cands = res["cand"][j]
        assert (cands >= 0).all()
        D2 = _fp64_d2(S, C[live])
        assert (D2[cands] > 0).all()                 # a zero-weight row is never drawn
        phi = [np.minimum(D2, ((S.astype(np.float64) - S[c].astype(np.float64)) ** 2).sum(1)).sum()
               for c in cands]
        best = int(np.argmin(phi))
        srt = np.sort(phi)
        if srt[1] - srt[0] > 1e-6 * srt[0]:
            np.testing.assert_array_equal(C[j], S[cands[best]])
        # the fixed-point potentials order the candidates like the exact ones
        order_fx = np.argsort(res["phi"][j], kind="stable")
        order_64 = np.argsort(phi, kind="stable")
        if np.all(np.diff(np.sort(phi)) > 1e-6 * srt[0]):
            np.testing.assert_array_equal(order_fx, order_64)
        live.append(j)


def test_kmeanspp_second_centroid_distribution(orc):
    # with L = 1 and one live centroid, the new centroid is row i with
    # probability D(x_i)^2 / sum D^2 (classic K-means++)
    S = np.array([[0.0], [1.0], [2.0], [4.0], [7.0]], np.float32)
    C0 = np.array([[0.0], [0.0]], np.float32)
    deg = np.array([0, 1], np.uint8)
    N = 20000
    counts = np.zeros(5, int)
    for sd in range(N):
        res = orc.kmeanspp(S, C0, deg, L=1, seed=sd)
        counts[int(np.flatnonzero(S[:, 0] == res["C"][1, 0])[0])] += 1
    w = (S[:, 0].astype(np.float64) - 0.0) ** 2
    assert counts[0] == 0
    assert chisquare(counts[1:], w[1:] / w.sum() * N).pvalue > 1e-4


def test_kmeanspp_first_pick_uniform(orc):
    S = np.arange(6, dtype=np.float32).reshape(6, 1)
    N = 12000
    counts = np.zeros(6, int)
    for sd in range(N):
        res = orc.kmeanspp(S, np.zeros((1, 1), np.float32), np.ones(1, np.uint8), seed=sd)
        counts[int(res["C"][0, 0])] += 1
    assert chisquare(counts).pvalue > 1e-4


def test_kmeanspp_only_touches_degenerate_slots(orc):
    rng = np.random.default_rng(13)
    S = rng.standard_normal((300, 4)).astype(np.float32)
    C0 = rng.standard_normal((5, 4)).astype(np.float32)
    deg = np.array([0, 1, 0, 1, 1], np.uint8)
    res = orc.kmeanspp(S, C0, deg, seed=3)
    for j in (0, 2):
        np.testing.assert_array_equal(res["C"][j], C0[j])
    assert not res["degenerate"].any()
    assert (res["cand"][[0, 2]] == -1).all()


def test_kmeanspp_runs_out_of_distinct_points(orc):
    S = np.array([[0, 0], [0, 0], [1, 1], [1, 1]], np.float32)
    res = orc.kmeanspp(S, np.zeros((4, 2), np.float32), np.ones(4, np.uint8), seed=0)
    assert res["rc"] == 0
    assert list(res["degenerate"]) == [0, 0, 1, 1]
    assert {tuple(res["C"][0]), tuple(res["C"][1])} == {(0.0, 0.0), (1.0, 1.0)}


# --------------------------------------------------------------------------
# Rounds (Algorithms 3 and 4)
# --------------------------------------------------------------------------
def _composed_round(orc, X, st, strategy, seed, rnd, L=3):
    """One round rebuilt from the separately pinned primitives."""
    W = len(st.s)
    snap = [st.centroids(w) for w in range(W)]
    fsnap = st.fhat.copy()
    out = []
    for w in range(W):
        S, _ = orc.draw_sample(X, seed, w, rnd, int(st.s[w]))
        b = w
        if strategy == orc.COOPERATIVE:
            cands = [v for v in range(W) if st.group[v] == st.group[w] and st.k[v] == st.k[w]]
            b = min(cands, key=lambda v: (fsnap[v], v))
        C, deg = snap[b]
        seeded = orc.kmeanspp(S, C, deg, L=L, seed=seed, worker=w, round_=rnd)
        r = orc.lloyd(S, seeded["C"], seeded["degenerate"])
        per = r["f"] / st.s[w]
        acc = per < st.fhat[w]
        out.append((r, per, acc))
    for w, (r, per, acc) in enumerate(out):
        if acc:
            k = int(st.k[w])
            st.C_pool[st.C_off[w]: st.C_off[w] + k * st.d] = r["C"].ravel()
            st.deg_pool[st.K_off[w]: st.K_off[w] + k] = r["degenerate"]
            st.fhat[w] = per
    return out


@pytest.mark.parametrize("strategy", [0, 1])
def test_round_matches_composed_primitives(orc, strategy):
    rng = np.random.default_rng(21)
    X = np.concatenate([rng.normal(c, 0.8, (40, 2)) for c in (-5, 0, 6)]).astype(np.float32)
    s, k = [16, 24, 16], [3, 3, 4]
    group = [0, 0, 1]
    a = orc.RoundState(2, s, k, group)
    b = orc.RoundState(2, s, k, group)
    for rnd in range(3):
        res = orc.round_(X, a, strategy, seed=5, round_idx=rnd)
        comp = _composed_round(orc, X, b, strategy, 5, rnd)
        np.testing.assert_array_equal(a.C_pool, b.C_pool)
        np.testing.assert_array_equal(a.deg_pool, b.deg_pool)
        np.testing.assert_array_equal(a.fhat, b.fhat)
        assert list(res["accepted"]) == [c[2] for c in comp]
        assert list(res["iters"]) == [c[0]["iters"] for c in comp]


def test_round_incumbents_never_worsen_and_coop_shares(orc):
    rng = np.random.default_rng(22)
    X = np.concatenate([rng.normal(c, 1.0, (300, 3)) for c in (-6, -1, 4, 9)]).astype(np.float32)
    st = orc.RoundState(3, [64, 64, 64, 64], [4, 4, 4, 4])
    prev = st.fhat.copy()
    for rnd in range(5):
        orc.round_(X, st, orc.COMPETITIVE if rnd < 2 else orc.COOPERATIVE, seed=1, round_idx=rnd)
        assert np.all(st.fhat <= prev)
        prev = st.fhat.copy()
    # in a cooperative round every worker starts from the best incumbent: after
    # it, any accepted worker's centroids derive from that base, so a worker
    # that was accepted reached an objective no worse than its own incumbent
    assert np.isfinite(st.fhat).all()


@pytest.mark.parametrize("n1", [0, 2, 99])
def test_hybrid_is_competitive_then_cooperative(orc, n1):
    # Algorithm 5: rounds below N1 run the competitive phase, the rest the
    # cooperative one; N1 = 0 is Algorithm 4 throughout, N1 >= rounds is
    # Algorithm 3 throughout
    rng = np.random.default_rng(23)
    X = np.concatenate([rng.normal(c, 0.9, (120, 3)) for c in (-7, -2, 3, 8)]).astype(np.float32)
    s, k, group = [40, 56, 40, 48], [3, 3, 3, 4], [0, 0, 0, 0]
    hyb = orc.RoundState(3, s, k, group)
    ref = orc.RoundState(3, s, k, group)
    for rnd in range(4):
        a = orc.round_(X, hyb, orc.HYBRID, seed=9, round_idx=rnd, n_competitive=n1)
        b = orc.round_(X, ref, orc.COMPETITIVE if rnd < n1 else orc.COOPERATIVE, seed=9,
                       round_idx=rnd)
        np.testing.assert_array_equal(hyb.C_pool, ref.C_pool)
        np.testing.assert_array_equal(hyb.fhat, ref.fhat)
        assert list(a["iters"]) == list(b["iters"])
    if n1 == 2:
        # the cooperative phase really shares: a fresh competitive-only run
        # from the same state differs in at least one worker's base
        comp = orc.RoundState(3, s, k, group)
        for rnd in range(4):
            orc.round_(X, comp, orc.COMPETITIVE, seed=9, round_idx=rnd)
        assert not np.array_equal(comp.C_pool, hyb.C_pool)


def test_paper_hyperparameters_fixture(orc):
    hp = json.loads((GOLDEN / "paper_hyperparameters.json").read_text())
    assert hp["lloyd_max_iter"] == 300 and hp["lloyd_rel_tol"] == 1e-4
    assert hp["kmeanspp_candidates"] == 3
    # the oracle's Python defaults follow the paper's stated values
    import inspect
    sig = inspect.signature(orc.lloyd)
    assert sig.parameters["max_iter"].default == hp["lloyd_max_iter"]
    assert sig.parameters["rel_tol"].default == hp["lloyd_rel_tol"]
    assert inspect.signature(orc.kmeanspp).parameters["L"].default == hp["kmeanspp_candidates"]
