"""Checkpoint and resume of an HPClust run (hpc_batch_save / hpc_batch_load).

Every random draw of round r is a function of (seed, worker, r) and the
workers keep no state between rounds but their incumbents (Algorithms 3-5),
so a run saved after round r and resumed into a fresh batch must end
bit-identical to the uninterrupted run.  Corrupted, foreign and mismatched
checkpoints are refused.
"""
import struct

import numpy as np
import pytest
import torch

from paper_2311_04517_gb300 import hpclust as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = H.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def data():
    rng = np.random.default_rng(7)
    d, comps, n = 16, 12, 200_000
    mu = rng.uniform(-10, 10, (comps, d))
    z = rng.integers(0, comps, n)
    X = (mu[z] + rng.uniform(0.5, 2.0, comps)[z, None] * rng.standard_normal((n, d)))
    return torch.from_numpy(X.astype(np.float32)).cuda()


WORKERS = dict(s=[4000, 9000, 6000, 12000, 5000, 7000], k=[5, 10, 5, 10, 12, 12],
               group=[0, 1, 0, 1, 2, 2])


def new_batch(d, n_competitive=0):
    return H.Batch(d, WORKERS["s"], WORKERS["k"], WORKERS["group"], n_competitive=n_competitive)


def state(b):
    return (b.C.clone(), b.degenerate.clone(), b.fhat.clone())


def same(a, b):
    return all(torch.equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("strategy,n_comp", [(H.HPC_COMPETITIVE, 0), (H.HPC_COOPERATIVE, 0),
                                             (H.HPC_HYBRID, 2)])
def test_resume_equals_uninterrupted_run(ctx, data, tmp_path, strategy, n_comp):
    d, seed, R, cut = data.shape[1], 11, 6, 3
    straight = new_batch(d, n_comp)
    for r in range(R):
        H.hpc_round(ctx, data, straight, strategy, seed, r)
    ctx.check_status()
    first = new_batch(d, n_comp)
    for r in range(cut):
        H.hpc_round(ctx, data, first, strategy, seed, r)
    path = tmp_path / "run.hpcb"
    first.save(ctx, path, cut, seed, strategy)
    resumed = new_batch(d, n_comp)
    r0, seed0, strat0 = resumed.load(ctx, path)
    assert (r0, seed0, strat0) == (cut, seed, strategy)
    assert same(state(resumed), state(first))
    for r in range(r0, R):
        H.hpc_round(ctx, data, resumed, strat0, seed0, r)
    ctx.check_status()
    assert same(state(resumed), state(straight))


def test_resume_into_a_prepared_round(ctx, data):
    d, seed, R, cut = data.shape[1], 5, 5, 2
    straight = new_batch(d)
    for r in range(R):
        H.hpc_round(ctx, data, straight, H.HPC_COOPERATIVE, seed, r)
    first = new_batch(d)
    for r in range(cut):
        H.hpc_round(ctx, data, first, H.HPC_COOPERATIVE, seed, r)
    blob = H.hpc_batch_save(ctx, first, cut, seed, H.HPC_COOPERATIVE)
    resumed = new_batch(d)
    r0, seed0, strat0 = H.hpc_batch_load(ctx, resumed, blob)
    H.hpc_round_prepare(ctx, data, resumed, strat0, seed0, r0)
    for _ in range(r0, R):
        H.hpc_round_enqueue(ctx)
    ctx.check_status()
    assert same(state(resumed), state(straight))


def test_checkpoint_layout(ctx, data):
    d = data.shape[1]
    b = new_batch(d)
    H.hpc_round(ctx, data, b, H.HPC_COMPETITIVE, 3, 0)
    blob = H.hpc_batch_save(ctx, b, 1, 3, H.HPC_COMPETITIVE)
    W = b.W
    floats = sum(int(k) * d for k in b.k)
    flags = sum(int(k) for k in b.k)
    assert len(blob) == 64 + 16 * W + 4 * floats + flags + 8 * W
    magic, version, W_, d_, strat, nxt, ncomp, seed, fl, fg = struct.unpack_from("<8sIiiiIiQqq", blob)
    assert (magic, version, W_, d_, strat, nxt, seed, fl, fg) == (
        b"HPCBATCH", 1, W, d, H.HPC_COMPETITIVE, 1, 3, floats, flags)
    off = 64 + 16 * W
    C0 = np.frombuffer(blob, np.float32, int(b.k[0]) * d, off)
    np.testing.assert_array_equal(C0, b.centroids(0)[0].cpu().numpy().ravel())
    fh = np.frombuffer(blob, np.float64, W, len(blob) - 8 * W)
    np.testing.assert_array_equal(fh, b.fhat.cpu().numpy())


def test_bad_checkpoints_are_refused(ctx, data):
    d = data.shape[1]
    b = new_batch(d)
    H.hpc_round(ctx, data, b, H.HPC_COMPETITIVE, 3, 0)
    blob = bytearray(H.hpc_batch_save(ctx, b, 1, 3, H.HPC_COMPETITIVE))
    before = state(b)
    target = new_batch(d)
    bad = bytearray(blob)
    bad[200] ^= 0x40                                   # payload bit flip
    for broken in (bytes(bad), bytes(blob[:-1]), b"NOTACKPT" + bytes(blob[8:])):
        with pytest.raises(H.HPCError) as e:
            H.hpc_batch_load(ctx, target, broken)
        assert e.value.code == H.HPC_ERR_ARG
    other = H.Batch(d, WORKERS["s"], [5, 10, 5, 10, 12, 11], WORKERS["group"])
    with pytest.raises(H.HPCError):
        H.hpc_batch_load(ctx, other, bytes(blob))       # another batch's shape
    other_d = H.Batch(8, WORKERS["s"], WORKERS["k"], WORKERS["group"])
    with pytest.raises(H.HPCError):
        H.hpc_batch_load(ctx, other_d, bytes(blob))
    assert same(state(b), before)
    # refused loads leave the target untouched
    assert torch.all(target.degenerate == 1) and torch.all(torch.isinf(target.fhat))
