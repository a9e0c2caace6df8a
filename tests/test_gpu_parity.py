"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bars (from the arithmetic, see each test):
  * sample rows / indices and K-means++ seeding: bit-exact (integer and
    exact-fixed-point decisions taken in the same precision on both sides);
  * labels: equal, except rows whose two nearest double-precision distances
    differ by less than 1e-6 relative (a near tie);
  * objectives: within 1e-6 relative; centroids: per coordinate within 1e-6
    relative plus an absolute floor of 1e-9 of the largest coordinate (the
    GPU sums coordinates exactly on a fixed-point grid 2^-F with
    F = 62 - bitlen(s) - e(max|x|), so each mean carries at most
    2^(bitlen(s) + e - 63) <= 2^-42 max|x| of grid rounding for s <= 2^20,
    and both sides round the mean to float once).
"""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_2311_04517_gb300 import hpclust as H
from paper_2311_04517_gb300 import synth

from lloyd_replay import (RTOL, TIE, assert_centroids, check_parted_run, dev, gpu_lloyd, host,
                          lockstep_divergence)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = H.Context(0)
    yield c
    c.close()


def mixture(n, d, comps, seed, spread=10.0, sd=1.0):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-spread, spread, (comps, d))
    z = rng.integers(0, comps, n)
    return (mu[z] + sd * rng.standard_normal((n, d))).astype(np.float32)


def assert_labels(lab_g, S, C, deg, what=""):
    lab_o, d1, d2, _ = orc.assign(S, C, deg)
    diff = np.flatnonzero(lab_g != lab_o)
    if diff.size:
        near = (d2[diff] - d1[diff]) <= TIE * d1[diff]
        assert near.all(), f"{what}: {np.count_nonzero(~near)} labels differ away from ties"
        # the GPU's pick is then as near as the oracle's within the tie bound
        Cd = C.astype(np.float64)
        dg = ((S[diff].astype(np.float64) - Cd[lab_g[diff]]) ** 2).sum(1)
        assert np.all(dg <= d1[diff] * (1 + TIE))
    return diff.size


# ---------------------------------------------------------------------------
# Sampling (Section 3)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,d,s", [(1000, 16, 777), (5, 3, 64), (1, 2, 10), (12345, 128, 3001),
                                   (70000, 1, 5000), (1000, 5, 0)])
def test_draw_sample_bit_exact(ctx, n, d, s):
    X = mixture(n, d, 3, 1)
    S_o, idx_o = orc.draw_sample(X, seed=77, worker=5, round_=3, s=s)
    idx = torch.empty(s, dtype=torch.int64, device="cuda")
    S_g, _ = H.hpc_draw_sample(ctx, dev(X), 77, 5, 3, s, idx_out=idx)
    ctx.check_status()
    np.testing.assert_array_equal(host(idx), idx_o)
    np.testing.assert_array_equal(host(S_g), S_o)


# ---------------------------------------------------------------------------
# Full-data objective (Eq. 1) and assignment
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,d,k", [(20000, 2, 5), (100003, 16, 25), (4099, 1, 3), (3001, 3, 7),
                                   (50001, 32, 50), (20011, 64, 100), (9001, 128, 100),
                                   (7777, 17, 9), (2048, 5, 1)])
def test_objective_parity(ctx, n, d, k):
    X = mixture(n, d, max(k, 2), seed=n + d)
    rng = np.random.default_rng(k)
    C = X[rng.choice(n, k, replace=False)] + 0.1 * rng.standard_normal((k, d)).astype(np.float32)
    C = C.astype(np.float32)
    deg = np.zeros(k, np.uint8)
    if k >= 5:
        deg[[1, k // 2]] = 1
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    f_g = H.hpc_objective(ctx, dev(X), dev(C), dev(deg), labels_out=lab)
    ctx.check_status()
    f_o = orc.objective(X, C, deg)
    assert float(host(f_g)[0]) == pytest.approx(f_o, rel=RTOL)
    assert_labels(host(lab), X, C, deg, "objective")
    # deterministic: a second run gives the same bits
    f_g2 = H.hpc_objective(ctx, dev(X), dev(C), dev(deg))
    ctx.check_status()
    assert float(host(f_g2)[0]) == float(host(f_g)[0])


def test_objective_edge_cases(ctx):
    C = dev(np.array([[0, 0], [1, 0], [1, 0], [-1, 0]], np.float32))
    # empty input
    f = H.hpc_objective(ctx, torch.empty((0, 2), dtype=torch.float32, device="cuda"), C)
    ctx.check_status()
    assert float(host(f)[0]) == 0.0
    # exact ties go to the lowest index (centroids 1 and 2 coincide)
    X = dev(np.array([[2, 0], [0.5, 0], [-0.5, 0], [3, 0]], np.float32))
    lab = torch.empty(4, dtype=torch.int32, device="cuda")
    H.hpc_objective(ctx, X, C, labels_out=lab)
    ctx.check_status()
    assert list(host(lab)) == [1, 0, 0, 1]
    # no live centroid
    H.hpc_objective(ctx, X, C, dev(np.ones(4, np.uint8)))
    assert ctx.sync_status() == H.HPC_ERR_DEGENERATE_ALL
    # non-finite row
    Xn = np.array([[1, 1], [np.nan, 0]], np.float32)
    H.hpc_objective(ctx, dev(Xn), C)
    assert ctx.sync_status() == H.HPC_ERR_NONFINITE
    # host-side argument errors
    with pytest.raises(H.HPCError):
        H.hpc_objective(ctx, torch.zeros((4, 129), device="cuda"), torch.zeros((2, 129), device="cuda"))
    with pytest.raises(H.HPCError):
        H.hpc_objective(ctx, X, C, prec=H.HPC_BF16)


def test_objective_near_ties_are_resolved_exactly(ctx):
    # rows placed (almost) on the bisector of two centroids far from the
    # origin: the FP32 expanded form cannot separate them, rescoring must
    rng = np.random.default_rng(3)
    d = 16
    c0 = rng.uniform(50, 60, d)
    c1 = c0 + rng.uniform(-1, 1, d) * 0.5
    mid = (c0 + c1) / 2
    n = 4096
    X = (mid + rng.standard_normal((n, d)) * 1e-4 + np.outer(rng.uniform(-1e-3, 1e-3, n), c1 - c0))
    X = X.astype(np.float32)
    C = np.stack([c0, c1]).astype(np.float32)
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    H.hpc_objective(ctx, dev(X), dev(C), labels_out=lab)
    ctx.check_status()
    lab_o, d1, d2, _ = orc.assign(X, C)
    g = host(lab)
    # double-precision rescoring: equal wherever the FP64 distances differ at all
    strict = (d2 - d1) > 1e-12 * d1
    np.testing.assert_array_equal(g[strict], lab_o[strict])


@pytest.mark.parametrize("n", [2**25 + 3])
def test_objective_large_index_range(ctx, n):
    # n * d > 2^31 elements: 64-bit row addressing
    d, k = 64, 8
    g = torch.Generator(device="cuda").manual_seed(5)
    X = torch.randn((n, d), generator=g, device="cuda") * 3
    Cn = np.random.default_rng(1).standard_normal((k, d)).astype(np.float32) * 3
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    f = H.hpc_objective(ctx, X, dev(Cn), labels_out=lab)
    ctx.check_status()
    idx = np.concatenate([np.arange(1000), np.arange(n - 5000, n),
                          np.random.default_rng(2).integers(0, n, 20000)])
    Xs = host(X[torch.from_numpy(idx).cuda()])
    assert_labels(host(lab)[idx], Xs, Cn, None, "large")
    f_o = orc.objective(host(X), Cn)
    assert float(host(f)[0]) == pytest.approx(f_o, rel=RTOL)
    del X


# ---------------------------------------------------------------------------
# K-means++ seeding: bit-exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("s,d,k,L,seed", [(2000, 2, 5, 3, 0), (100000, 16, 25, 3, 1),
                                          (3001, 17, 12, 1, 2), (5000, 128, 20, 3, 3),
                                          (777, 3, 40, 8, 4), (1, 4, 1, 3, 5)])
def test_kmeanspp_bit_exact(ctx, s, d, k, L, seed):
    S = mixture(s, d, max(2, k // 2), seed)
    C0 = np.zeros((k, d), np.float32)
    deg0 = np.ones(k, np.uint8)
    o = orc.kmeanspp(S, C0, deg0, L=L, seed=seed, worker=2, round_=7)
    Cg, dg = dev(C0), dev(deg0)
    H.hpc_kmeanspp(ctx, dev(S), Cg, dg, n_candidates=L, seed=seed, worker=2, round_=7)
    ctx.check_status()
    np.testing.assert_array_equal(host(dg), o["degenerate"])
    np.testing.assert_array_equal(host(Cg), o["C"])


def test_kmeanspp_partial_reseed_and_exhaustion(ctx):
    rng = np.random.default_rng(9)
    S = mixture(4000, 8, 6, 9)
    C0 = rng.standard_normal((10, 8)).astype(np.float32)
    deg0 = np.array([0, 1, 1, 0, 0, 1, 0, 1, 1, 0], np.uint8)
    o = orc.kmeanspp(S, C0, deg0, seed=11, worker=1, round_=2)
    Cg, dg = dev(C0), dev(deg0)
    H.hpc_kmeanspp(ctx, dev(S), Cg, dg, seed=11, worker=1, round_=2)
    ctx.check_status()
    np.testing.assert_array_equal(host(Cg), o["C"])
    np.testing.assert_array_equal(host(dg), o["degenerate"])
    # fewer distinct rows than centroids: the rest stay degenerate
    S2 = np.repeat(np.array([[0, 0], [1, 1], [5, 5]], np.float32), 50, axis=0)
    o2 = orc.kmeanspp(S2, np.zeros((6, 2), np.float32), np.ones(6, np.uint8), seed=3)
    Cg, dg = dev(np.zeros((6, 2), np.float32)), dev(np.ones(6, np.uint8))
    H.hpc_kmeanspp(ctx, dev(S2), Cg, dg, seed=3)
    ctx.check_status()
    np.testing.assert_array_equal(host(dg), o2["degenerate"])
    np.testing.assert_array_equal(host(Cg), o2["C"])
    # nothing to seed: untouched
    Cg = dev(C0)
    dg = dev(np.zeros(10, np.uint8))
    H.hpc_kmeanspp(ctx, dev(S), Cg, dg, seed=3)
    ctx.check_status()
    np.testing.assert_array_equal(host(Cg), C0)


# ---------------------------------------------------------------------------
# Lloyd (Algorithm 1, Section 6.5 stop rule)
# ---------------------------------------------------------------------------
def lloyd_case(ctx, S, k, seed):
    d = S.shape[1]
    init = orc.kmeanspp(S, np.zeros((k, d), np.float32), np.ones(k, np.uint8), seed=seed)
    C0, deg0 = init["C"], init["degenerate"]
    o = orc.lloyd(S, C0, deg0)
    g = gpu_lloyd(ctx, S, C0, deg0)
    same = (g["iters"] == o["iters"] and (g["degenerate"] == o["degenerate"]).all()
            and abs(g["f"] - o["f"]) <= RTOL * o["f"])
    if same:
        assert_centroids(g["C"], o["C"], "lloyd")
        assert_labels(g["labels"], S, o["C"], o["degenerate"], "lloyd")
    else:
        # only a near tie (in a label or in the stop test) may explain it;
        # up to the step where they part, the two runs agree
        check_parted_run(ctx, S, C0, deg0, g, o)
    # the reported objective is the objective of the returned centroids
    assert g["f"] == pytest.approx(orc.objective(S, g["C"], g["degenerate"]), rel=RTOL)
    return g, o


@pytest.mark.parametrize("s,d,k,seed", [(2000, 2, 5, 0), (100000, 16, 25, 1), (20000, 32, 50, 2),
                                        (9001, 64, 30, 3), (5000, 128, 10, 4), (30011, 5, 8, 5),
                                        # d in (64, 128]: the d = 128 kernel, and at d = 100
                                        # its rows padded with zeros
                                        (30011, 128, 40, 6), (7001, 100, 17, 7)])
def test_lloyd_parity(ctx, s, d, k, seed):
    S = mixture(s, d, k, seed, sd=1.5)
    lloyd_case(ctx, S, k, seed)


def zipf_mixture(s, d, comps, seed):
    """A Zipf-weighted mixture like the large workload's (several centroids
    share the heavy components, light ones get few rows)."""
    rng = np.random.default_rng(seed)
    mu = 4.0 * rng.standard_normal((comps, d))
    w = np.arange(1, comps + 1, dtype=np.float64) ** -1.1
    z = rng.choice(comps, s, p=w / w.sum())
    sd = rng.uniform(0.5, 2.0, comps)
    return (mu[z] + sd[z, None] * rng.standard_normal((s, d))).astype(np.float32)


@pytest.mark.parametrize("s,d,k,seed", [(20000, 64, 500, 11), (5000, 128, 256, 12),
                                        (65536, 64, 500, 13)])
def test_lloyd_parity_global_sums(ctx, s, d, k, seed):
    # CUDA-core Lloyd with k x d x 8 bytes of per-block sums above what a
    # block's shared memory holds (the large workload's k = 500 at d = 64):
    # every block adds its rows' fixed-point coordinates straight into the
    # global sums
    ctx.set_tensor_cores(0)
    try:
        sched = ctx.lloyd_schedule(s, d, k)
        assert not sched["smem_sums"] and sched["form"] == "simt", sched
        lloyd_case(ctx, zipf_mixture(s, d, k, seed), k, seed)
    finally:
        ctx.set_tensor_cores(2)


# ---------------------------------------------------------------------------
# Lloyd with the x.c contraction on the tensor cores (split BF16, d = 64 /
# 128): incremental fixed-point sums of the rows whose label changed
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("s,d,k,seed", [(20000, 64, 500, 21), (65613, 64, 500, 22),
                                        (5000, 128, 256, 23), (30011, 128, 100, 24),
                                        (9001, 64, 130, 25), (3001, 64, 64, 26),
                                        (129, 64, 60, 27), (1000, 128, 200, 28),
                                        (40000, 64, 256, 29), (7000, 64, 33, 30)])
def test_lloyd_parity_tensor_cores(ctx, s, d, k, seed):
    ctx.set_tensor_cores(1)
    try:
        assert ctx.lloyd_schedule(s, d, k)["form"] == "split_bf16"
        S = zipf_mixture(s, d, k, seed) if k >= 256 else mixture(s, d, k, seed, sd=1.5)
        lloyd_case(ctx, S, k, seed)
    finally:
        ctx.set_tensor_cores(2)


@pytest.mark.parametrize("d,k", [(64, 500), (128, 100)])
def test_lloyd_tensor_cores_match_cuda_cores(ctx, d, k):
    # the same run on both searches: the same labels away from near ties,
    # centroids and objective within the contract, the same iteration count
    S = zipf_mixture(30000, d, k, 31)
    init = orc.kmeanspp(S, np.zeros((k, d), np.float32), np.ones(k, np.uint8), seed=31)
    out = {}
    for mode in (0, 1):
        ctx.set_tensor_cores(mode)
        out[mode] = gpu_lloyd(ctx, S, init["C"], init["degenerate"])
    ctx.set_tensor_cores(2)
    a, b = out[0], out[1]
    if a["iters"] == b["iters"]:
        assert_centroids(b["C"], a["C"], "tensor vs CUDA cores")
        np.testing.assert_array_equal(a["degenerate"], b["degenerate"])
        assert b["f"] == pytest.approx(a["f"], rel=RTOL)
        assert_labels(b["labels"], S, a["C"], a["degenerate"], "tensor cores")
    else:   # only a near tie may part the runs
        lockstep_divergence(ctx, S, init["C"], init["degenerate"], max(a["iters"], b["iters"]))


def test_lloyd_tensor_cores_edge_cases(ctx):
    ctx.set_tensor_cores(1)
    try:
        d = 64
        # one row, and fewer rows than a tile
        S = mixture(77, d, 5, 41)
        C0 = S[:5].copy()
        o = orc.lloyd(S, C0, np.zeros(5, np.uint8))
        g = gpu_lloyd(ctx, S, C0, np.zeros(5, np.uint8))
        assert g["iters"] == o["iters"]
        assert_centroids(g["C"], o["C"], "77 rows")
        assert g["f"] == pytest.approx(o["f"], rel=RTOL)
        g = gpu_lloyd(ctx, S[:1], C0[:1], np.zeros(1, np.uint8))
        assert g["f"] == 0.0 and g["iters"] == 1
        # centroids that lose every row become degenerate and keep their values
        S2 = np.concatenate([np.zeros((100, d)), np.full((100, d), 5.0)]).astype(np.float32)
        C2 = np.stack([np.zeros(d), np.full(d, 5.0), np.full(d, 100.0),
                       np.full(d, 2.4)]).astype(np.float32)
        o = orc.lloyd(S2, C2, np.zeros(4, np.uint8))
        g = gpu_lloyd(ctx, S2, C2, np.zeros(4, np.uint8))
        np.testing.assert_array_equal(g["degenerate"], o["degenerate"])
        assert_centroids(g["C"], o["C"], "emptied clusters")
        # zero iterations: only the assignment
        g = gpu_lloyd(ctx, S, C0, np.zeros(5, np.uint8), max_iter=0)
        assert g["iters"] == 0
        np.testing.assert_array_equal(g["C"], C0)
        # every centroid degenerate; a non-finite row
        Cg, dg = dev(C0), dev(np.ones(5, np.uint8))
        H.hpc_lloyd(ctx, dev(S), Cg, dg)
        assert ctx.sync_status() == H.HPC_ERR_DEGENERATE_ALL
        Sn = S.copy()
        Sn[30, 7] = np.nan
        H.hpc_lloyd(ctx, dev(Sn), dev(C0), dev(np.zeros(5, np.uint8)))
        assert ctx.sync_status() == H.HPC_ERR_NONFINITE
        # the context stays usable, and runs are deterministic
        S3 = zipf_mixture(20000, d, 300, 42)
        a = gpu_lloyd(ctx, S3, S3[:300].copy(), np.zeros(300, np.uint8))
        b = gpu_lloyd(ctx, S3, S3[:300].copy(), np.zeros(300, np.uint8))
        np.testing.assert_array_equal(a["C"], b["C"])
        np.testing.assert_array_equal(a["labels"], b["labels"])
        assert a["f"] == b["f"] and a["iters"] == b["iters"]
    finally:
        ctx.set_tensor_cores(2)


def test_lloyd_tensor_cores_near_ties(ctx):
    # rows on the bisector of two far centroids: the split-BF16 values
    # cannot separate them; the exact stages must give the oracle's labels
    rng = np.random.default_rng(43)
    d = 64
    c0 = rng.uniform(50, 60, d)
    c1 = c0 + rng.uniform(-1, 1, d) * 0.5
    mid = (c0 + c1) / 2
    n = 4096
    S = (mid + rng.standard_normal((n, d)) * 1e-3 +
         np.outer(rng.uniform(-1e-2, 1e-2, n), c1 - c0)).astype(np.float32)
    C = np.stack([c0, c1] + [c0 + 30 * rng.standard_normal(d) for _ in range(126)]).astype(np.float32)
    ctx.set_tensor_cores(1)
    try:
        g = gpu_lloyd(ctx, S, C, np.zeros(128, np.uint8), max_iter=0)
    finally:
        ctx.set_tensor_cores(2)
    lab_o, d1, d2, _ = orc.assign(S, C)
    strict = (d2 - d1) > 1e-12 * d1
    np.testing.assert_array_equal(g["labels"][strict], lab_o[strict])


@pytest.mark.parametrize("d,k", [(64, 128), (64, 300), (128, 200)])
def test_lloyd_tensor_cores_three_way_ties(ctx, d, k):
    # rows at the centre of three centroids at equal distance (up to the
    # rounding of the FP32 rows and centroids): every row has a third
    # candidate inside the split-BF16 window, so it is settled against every
    # centroid, and FP32 cannot order the three, so FP64 decides.  One update
    # must equal the oracle's update on the oracle's labels.
    rng = np.random.default_rng(44 + d + k)
    m = rng.uniform(50, 60, d)
    Q, _ = np.linalg.qr(rng.standard_normal((d, 3)))
    near = [m + 5.0 * Q[:, j] for j in range(3)]
    far = [m + 30.0 * rng.standard_normal(d) for _ in range(k - 3)]
    C = np.stack(near + far).astype(np.float32)
    n = 4096
    S = (m + 2e-6 * rng.standard_normal((n, d))).astype(np.float32)
    deg = np.zeros(k, np.uint8)
    lab_o, d1, d2, _ = orc.assign(S, C, deg)
    assert ((d2 - d1) > 1e-12 * d1).all()     # strict in FP64
    Co, dego = orc.update(S, lab_o, C, deg)
    ctx.set_tensor_cores(1)
    ctx.set_search_stats(True)
    ctx.search_stats(reset=True)
    try:
        assert ctx.lloyd_schedule(n, d, k)["form"] == "split_bf16"
        g = gpu_lloyd(ctx, S, C, deg, max_iter=1, rel_tol=0.0)
        st = ctx.search_stats(reset=True)
    finally:
        ctx.set_search_stats(False)
        ctx.set_tensor_cores(2)
    assert st["all_centroids"] > 0 and st["fp64"] > 0, st
    np.testing.assert_array_equal(g["degenerate"], dego)
    assert_centroids(g["C"], Co, "one update")


def test_lloyd_edge_cases(ctx):
    # k > distinct rows: empty clusters become degenerate, keep their values
    S = np.array([[0, 0], [0.1, 0], [5, 5], [5.1, 5]], np.float32)
    C0 = np.array([[0, 0], [5, 5], [100, 100]], np.float32)
    o = orc.lloyd(S, C0, np.zeros(3, np.uint8))
    g = gpu_lloyd(ctx, S, C0, np.zeros(3, np.uint8))
    np.testing.assert_array_equal(g["degenerate"], o["degenerate"])
    assert_centroids(g["C"], o["C"])
    assert g["iters"] == o["iters"]
    # one row
    g = gpu_lloyd(ctx, S[:1], C0[:1], np.zeros(1, np.uint8))
    assert g["f"] == 0.0 and g["iters"] == 1
    # zero iterations: only the assignment
    S2 = mixture(3000, 4, 3, 8)
    g = gpu_lloyd(ctx, S2, S2[:3].copy(), np.zeros(3, np.uint8), max_iter=0)
    assert g["iters"] == 0
    np.testing.assert_array_equal(g["C"], S2[:3])
    assert g["f"] == pytest.approx(orc.objective(S2, S2[:3]), rel=RTOL)
    # every centroid degenerate
    Cg, dg = dev(C0), dev(np.ones(3, np.uint8))
    H.hpc_lloyd(ctx, dev(S), Cg, dg)
    assert ctx.sync_status() == H.HPC_ERR_DEGENERATE_ALL
    # non-finite sample
    Sn = S.copy()
    Sn[2, 1] = np.inf
    H.hpc_lloyd(ctx, dev(Sn), dev(C0), dev(np.zeros(3, np.uint8)))
    assert ctx.sync_status() == H.HPC_ERR_NONFINITE


def test_lloyd_is_deterministic(ctx):
    S = mixture(50000, 16, 20, 12, sd=2.0)
    C0 = S[:20].copy()
    a = gpu_lloyd(ctx, S, C0, np.zeros(20, np.uint8))
    b = gpu_lloyd(ctx, S, C0, np.zeros(20, np.uint8))
    np.testing.assert_array_equal(a["C"], b["C"])
    np.testing.assert_array_equal(a["labels"], b["labels"])
    assert a["f"] == b["f"] and a["iters"] == b["iters"]


# ---------------------------------------------------------------------------
# Rounds (Algorithms 3 and 4), re-synchronised to the GPU state every round
# ---------------------------------------------------------------------------
def oracle_state_from(batch):
    st = orc.RoundState(batch.d, batch.s, batch.k, batch.group)
    for w in range(batch.W):
        k = int(batch.k[w])
        C, deg = batch.centroids(w)
        st.C_pool[st.C_off[w]: st.C_off[w] + k * batch.d] = host(C).ravel()
        st.deg_pool[st.K_off[w]: st.K_off[w] + k] = host(deg)
    st.fhat[:] = host(batch.fhat)
    return st


def check_round(ctx, X, Xd, batch, strategy, seed, rnd):
    st = oracle_state_from(batch)
    res = orc.round_(X, st, strategy, seed, rnd, n_competitive=batch.n_competitive)
    H.hpc_round(ctx, Xd, batch, strategy, seed, rnd)
    ctx.check_status()
    for w in range(batch.W):
        C, deg = batch.centroids(w)
        Co, dego = st.centroids(w)
        np.testing.assert_array_equal(host(deg), dego)
        assert_centroids(host(C), Co, f"round {rnd} worker {w}")
        assert int(host(batch.iters)[w]) == res["iters"][w]
        assert float(host(batch.f_new)[w]) == pytest.approx(res["f_new"][w], rel=RTOL)
    np.testing.assert_allclose(host(batch.fhat), st.fhat, rtol=RTOL)
    np.testing.assert_array_equal(host(batch.accepted).astype(bool), res["accepted"])


def test_round_tiny_workload_20_rounds(ctx):
    wl = synth.WORKLOADS["tiny"]
    X = host(synth.make_data(wl))
    Xd = dev(X)
    ws = synth.worker_setup(wl)
    batch = H.Batch(wl.d, ws.s, ws.k, ws.group)
    for rnd in range(wl.rounds):
        check_round(ctx, X, Xd, batch, H.HPC_COMPETITIVE, wl.seed, rnd)
        f = H.hpc_objective(ctx, Xd, batch.centroids(0)[0], batch.centroids(0)[1])
        ctx.check_status()
        C, deg = batch.centroids(0)
        assert float(host(f)[0]) == pytest.approx(orc.objective(X, host(C), host(deg)), rel=RTOL)


@pytest.mark.parametrize("strategy", [0, 1])
def test_round_several_workers(ctx, strategy):
    X = mixture(30000, 8, 12, 21, sd=1.2)
    Xd = dev(X)
    batch = H.Batch(8, [3000, 5000, 4000, 2500], [6, 6, 9, 6], [0, 0, 1, 0])
    for rnd in range(4):
        check_round(ctx, X, Xd, batch, strategy, 3, rnd)


@pytest.mark.parametrize("strategy", [0, 1])
def test_round_mixed_k_batch(ctx, strategy):
    # batching-workload shape at test size: 16 workers, k_w = (10, 25, 50, 100)[w mod 4],
    # uneven samples, cooperative sharing only among equal k; one launch per phase
    X = mixture(60000, 32, 50, 5, sd=2.0)
    Xd = dev(X)
    rng = np.random.default_rng(9)
    W = 16
    s = rng.integers(1500, 6000, W).tolist()
    k = [(10, 25, 50, 100)[w % 4] for w in range(W)]
    batch = H.Batch(32, s, k, [0] * W)
    for rnd in range(3):
        check_round(ctx, X, Xd, batch, strategy, 17, rnd)


@pytest.mark.parametrize("strategy", [0, 1])
def test_round_tensor_core_lloyd(ctx, strategy):
    # d = 64 workers with k up to 500 (the large workload's shape at test
    # size): the split-BF16 tensor-core Lloyd inside the batched round
    X = zipf_mixture(80000, 64, 300, 45)
    Xd = dev(X)
    rng = np.random.default_rng(46)
    W = 8
    s = rng.integers(3000, 12000, W).tolist()
    k = [(100, 300, 500)[w % 3] for w in range(W)]
    batch = H.Batch(64, s, k, [0] * W)
    assert ctx.lloyd_schedule(max(s), 64, 500)["form"] == "split_bf16"
    for rnd in range(3):
        check_round(ctx, X, Xd, batch, strategy, 19, rnd)


def test_round_tensor_core_lloyd_sets(ctx):
    # 36 workers on the launch's CTAs: nine sets of four, each set running
    # its workers one after another on all of its CTAs (every worker's
    # barriers and sums over the set), the plan remade on the device before
    # every launch from the previous round's updates
    X = zipf_mixture(60000, 64, 200, 47)
    Xd = dev(X)
    rng = np.random.default_rng(48)
    W = 36
    s = rng.integers(2500, 6000, W).tolist()
    k = [(60, 120, 200)[w % 3] for w in range(W)]
    plan = H.lloyd_cta_plan(s, k, [0] * W, 152)
    firsts = {int(t) for t in plan["cta_task"] if t >= 0}
    assert len(firsts) == 9 and (plan["next"] >= 0).sum() == W - 9
    batch = H.Batch(64, s, k, [0] * W)
    assert ctx.lloyd_schedule(max(s), 64, 200)["form"] == "split_bf16"
    for rnd in range(3):
        check_round(ctx, X, Xd, batch, 0, 23, rnd)


def test_round_hybrid_switches_phase(ctx):
    # Algorithm 5 with N1 = 2: two competitive rounds, then cooperative ones
    X = mixture(20000, 6, 8, 31, sd=1.1)
    Xd = dev(X)
    batch = H.Batch(6, [2000, 3000, 2500, 2000], [5, 5, 5, 7], [0, 0, 0, 0], n_competitive=2)
    for rnd in range(4):
        check_round(ctx, X, Xd, batch, H.HPC_HYBRID, 41, rnd)


def test_round_more_workers_than_one_launch_takes(ctx):
    # 300 workers: the persistent kernels run in chunks of workers
    X = mixture(5000, 4, 6, 8)
    Xd = dev(X)
    W = 300
    s = [200 + 7 * (w % 13) for w in range(W)]
    k = [3 + (w % 3) for w in range(W)]
    batch = H.Batch(4, s, k, [w % 2 for w in range(W)])
    for rnd in range(2):
        check_round(ctx, X, Xd, batch, 1, 23, rnd)


@pytest.mark.parametrize("i", [0, 1, 2])
@pytest.mark.parametrize("strategy", [0, 1, 2])
def test_round_scaling_workload(ctx, i, strategy):
    # the Section 6.8 scaling set (10 blobs + uniform noise, k = 10,
    # s = min(5000, m - 1000), eight workers), three rounds of each strategy
    wl = synth.workload(f"scaling{i}")
    X = host(synth.make_data(wl))
    Xd = dev(X)
    ws = synth.worker_setup(wl)
    batch = H.Batch(wl.d, ws.s, ws.k, ws.group, n_competitive=1)
    for rnd in range(3):
        check_round(ctx, X, Xd, batch, strategy, 7 + i, rnd)


def test_baseline_convergence_time(ctx):
    # Section 6.4: the baseline convergence time is the time until any worker
    # first reaches a given sample objective.  Every worker's run end is
    # stamped on the device; with the oracle's per-round objectives the
    # first (round, worker) below a threshold is known exactly.
    X = mixture(30000, 8, 12, 71, sd=1.2)
    Xd = dev(X)
    S, K, G = [3000, 5000, 4000, 2500], [6, 6, 6, 6], [0, 0, 0, 0]
    R = 5
    st = orc.RoundState(8, S, K, G)
    vals = []
    for r in range(R):
        res = orc.round_(X, st, H.HPC_COMPETITIVE, 9, r)
        vals.append(res["f_new"] / np.asarray(S, np.float64))
    vals = np.array(vals)
    # the threshold: the best sample objective of round 1, with room for the
    # 1e-6 parity of the GPU's objectives; no other value near it
    v = float(vals[1].min())
    target = v * (1 + 1e-7)
    others = vals[np.abs(vals - v) > 1e-12 * v]
    assert np.all(np.abs(others - v) > 2e-6 * v)
    first = min((r, w) for r in range(R) for w in range(len(S)) if vals[r, w] <= target)
    batch = H.Batch(8, S, K, G)
    t0 = ctx.timestamp()
    stamps, fs, bounds = [], [], []
    for r in range(R):
        before = ctx.timestamp()
        H.hpc_round(ctx, Xd, batch, H.HPC_COMPETITIVE, 9, r)
        after = ctx.timestamp()
        ctx.check_status()
        stamps.append(host(batch.t_done).copy())
        fs.append(host(batch.f_new) / np.asarray(S, np.float64))
        bounds.append((int(before.item()), int(after.item())))
    hits = [(int(stamps[r][w]), r, w) for r in range(R) for w in range(len(S))
            if fs[r][w] <= target]
    tbar_ns, r1, w1 = min(hits)
    assert (r1, w1) == first or (r1 == first[0])
    lo, hi = bounds[r1]
    assert lo <= tbar_ns <= hi            # stamped inside its round
    assert tbar_ns - int(t0.item()) > 0


# ---------------------------------------------------------------------------
# Failure detection: a bounded device wait that runs out reports an error
# ---------------------------------------------------------------------------
def test_bounded_wait_reports_timeout(ctx):
    ctx.selftest_wait_timeout(20_000_000)     # 20 ms
    assert ctx.sync_status() == H.HPC_ERR_TIMEOUT
    # the context stays usable afterwards
    X = mixture(1000, 4, 3, 1)
    f = H.hpc_objective(ctx, dev(X), dev(X[:3].copy()))
    ctx.check_status()
    assert float(host(f)[0]) == pytest.approx(orc.objective(X, X[:3]), rel=RTOL)


def test_round_with_non_finite_rows_reports_and_recovers(ctx):
    # 1% of the rows non-finite: every worker's sample draws some, so every
    # Lloyd task stops at its first barrier and the round ends with
    # HPC_ERR_NONFINITE (no wait runs out); the incumbents stay as they were
    # and the next round on finite data matches the oracle
    X = mixture(20000, 8, 6, 31, sd=1.0)
    Xd = dev(X)
    batch = H.Batch(8, [3000, 5000, 4000, 2500], [6, 6, 9, 6], [0, 0, 1, 0])
    check_round(ctx, X, Xd, batch, H.HPC_COMPETITIVE, 5, 0)
    before = (host(batch.C).copy(), host(batch.degenerate).copy(), host(batch.fhat).copy())
    Xn = X.copy()
    Xn[::100, 3] = np.nan
    H.hpc_round(ctx, dev(Xn), batch, H.HPC_COMPETITIVE, 5, 1)
    assert ctx.sync_status() == H.HPC_ERR_NONFINITE
    np.testing.assert_array_equal(host(batch.C), before[0])
    np.testing.assert_array_equal(host(batch.degenerate), before[1])
    np.testing.assert_array_equal(host(batch.fhat), before[2])
    check_round(ctx, X, Xd, batch, H.HPC_COMPETITIVE, 5, 1)
