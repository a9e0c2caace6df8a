"""One HPClust job split over two ranks (gloo, CPU): workers in contiguous
ranges per rank, the cooperative share as an all-gather of (f-hat, index)
and a broadcast of the best incumbent, the objective of Eq. 1 as a sum of
row shards.  Each rank's compute is the CPU oracle; the split run must equal
the one-process oracle run of all workers bit for bit (competitive,
cooperative and hybrid rounds), and the sharded objective the whole one
within FP64 summation order."""
import os
import socket
import sys
from pathlib import Path

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = Path(__file__).resolve().parents[1]
S = [900, 1300, 700, 1100, 1000, 800]
K = [5, 5, 7, 5, 7, 5]
G = [0, 0, 1, 0, 1, 0]
D = 6
ROUNDS = 4
SEED = 13


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _data():
    rng = np.random.default_rng(5)
    mu = rng.uniform(-10, 10, (8, D))
    z = rng.integers(0, 8, 6000)
    return (mu[z] + 1.2 * rng.standard_normal((6000, D))).astype(np.float32)


class OracleBackend:
    """The CPU oracle as one rank's compute (test infrastructure)."""

    def __init__(self, orc, X, w0, w1):
        self.orc, self.X, self.w0 = orc, X, w0
        self.st = orc.RoundState(D, S[w0:w1], K[w0:w1], G[w0:w1])
        self.acc = None

    def pools(self):
        return (torch.from_numpy(self.st.C_pool), torch.from_numpy(self.st.deg_pool),
                torch.from_numpy(self.st.fhat))

    def offsets(self):
        return self.st.C_off, self.st.K_off

    def run_round(self, seed, rnd):
        res = self.orc.round_(self.X, self.st, self.orc.COMPETITIVE, seed, rnd, worker0=self.w0)
        self.acc = res["accepted"]

    def accepted(self):
        return self.acc

    def objective(self, rows, C, deg):
        return torch.tensor(self.orc.objective(rows.numpy(), C.numpy().reshape(-1, D),
                                               deg.numpy()), dtype=torch.float64)


def _rank(rank, world, port, strategy, out_dir):
    sys.path.insert(0, str(ROOT))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as orc
    from paper_2311_04517_gb300 import multirank as MR
    X = _data()
    ranges = MR.worker_ranges(S, K, world)
    w0, w1 = ranges[rank]
    run = MR.RankedRun(OracleBackend(orc, X, w0, w1), S, K, G, D, w0, w1)
    for r in range(ROUNDS):
        run.round(strategy, SEED, r, ranges, n_competitive=2)
    C, deg, fhat = run.b.pools()
    np.savez(Path(out_dir) / f"rank{rank}.npz", C=C.numpy(), deg=deg.numpy(),
             fhat=fhat.numpy(), w0=w0, w1=w1)
    # the objective of group 0's best incumbent, over row shards
    wb, fb, Cb, db = run.best(ranges, key=0)
    a, b = MR.row_range(X.shape[0], world, rank)
    f = run.objective(torch.from_numpy(X[a:b]), Cb, db)
    np.savez(Path(out_dir) / f"best{rank}.npz", wb=wb, fb=fb, C=Cb.numpy(), deg=db.numpy(),
             f=float(f.item()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("strategy", [0, 1, 2])
def test_two_ranks_equal_one_process(strategy, tmp_path, orc):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), strategy, str(tmp_path)), nprocs=world,
             join=True)
    X = _data()
    ref = orc.RoundState(D, S, K, G)
    for r in range(ROUNDS):
        orc.round_(X, ref, strategy, SEED, r, n_competitive=2)
    for rank in range(world):
        z = np.load(tmp_path / f"rank{rank}.npz")
        w0, w1 = int(z["w0"]), int(z["w1"])
        assert w1 > w0
        for i, w in enumerate(range(w0, w1)):
            Co, do = ref.centroids(w)
            st = orc.RoundState(D, S[w0:w1], K[w0:w1], G[w0:w1])
            a, kk = int(st.C_off[i]), K[w]
            np.testing.assert_array_equal(z["C"][a:a + kk * D].reshape(kk, D), Co)
            np.testing.assert_array_equal(z["deg"][int(st.K_off[i]):int(st.K_off[i]) + kk], do)
            assert z["fhat"][i] == ref.fhat[w]
    # the global best of group 0 and its objective over the row shards
    g0 = [w for w in range(len(S)) if G[w] == 0]
    wb = min(g0, key=lambda w: (ref.fhat[w], w))
    Co, do = ref.centroids(wb)
    f_ref = orc.objective(X, Co, do)
    for rank in range(world):
        b = np.load(tmp_path / f"best{rank}.npz")
        assert int(b["wb"]) == wb and float(b["fb"]) == ref.fhat[wb]
        np.testing.assert_array_equal(b["C"].reshape(-1, D), Co)
        np.testing.assert_array_equal(b["deg"], do)
        assert float(b["f"]) == pytest.approx(f_ref, rel=1e-12)


def test_worker_and_row_ranges():
    sys.path.insert(0, str(ROOT))
    from paper_2311_04517_gb300 import multirank as MR
    for W, world in [(10, 3), (4, 2), (2, 4), (1, 1), (128, 8), (7, 7)]:
        s = np.random.default_rng(W).integers(100, 1000, W)
        k = np.full(W, 5)
        rr = MR.worker_ranges(s, k, world)
        assert rr[0][0] == 0 and rr[-1][1] == W and len(rr) == world
        assert all(a <= b for a, b in rr) and all(rr[i][1] == rr[i + 1][0] for i in range(world - 1))
        if W >= world:
            assert all(b > a for a, b in rr)
        if W >= 8 * world:   # balanced to within one worker's work
            work = [float((s[a:b] * k[a:b]).sum()) for a, b in rr]
            assert max(work) - min(work) <= 2 * float((s * k).max())
    for n, world in [(10, 3), (7, 7), (1000003, 8), (2, 4)]:
        rs = [MR.row_range(n, world, r) for r in range(world)]
        assert rs[0][0] == 0 and rs[-1][1] == n
        assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
