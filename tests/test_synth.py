"""The seeded input recipes (no GPU): the workloads' shapes and the Section
6.8 scaling set's structure, and that a seed fixes the data."""
import numpy as np
import torch

from paper_2311_04517_gb300 import synth


def test_workload_table_shapes():
    w = synth.WORKLOADS
    assert (w["tiny"].n, w["tiny"].d, w["tiny"].k, w["tiny"].W) == (20_000, 2, (5,), 1)
    assert (w["fp32"].n, w["fp32"].d, w["fp32"].k, w["fp32"].s) == (10_000_000, 16, (25,),
                                                                   ("const", 100_000))
    assert (w["precision"].n, w["precision"].d, w["precision"].k) == (20_000_000, 128, (100,))
    b = w["batching"]
    assert (b.n, b.d, b.W, b.k, b.s) == (50_000_000, 32, 64, (10, 25, 50, 100),
                                         ("uniform", 16_384, 262_144))
    g = w["large"]
    assert (g.n, g.d, g.W, g.k, g.weights) == (200_000_000, 64, 128, (500,), "zipf1.1")


def test_worker_setup_groups_equal_k():
    ws = synth.worker_setup("batching")
    assert len(ws.s) == 64 and ws.s.min() >= 16_384 and ws.s.max() <= 262_144
    for g in set(ws.group.tolist()):
        assert len(set(ws.k[ws.group == g].tolist())) == 1


def test_mixture_is_seeded():
    a = synth.make_data("tiny")
    b = synth.make_data("tiny")
    c = synth.make_data("tiny", seed=1)
    assert torch.equal(a, b) and not torch.equal(a, c)
    assert a.shape == (20_000, 2) and a.dtype == torch.float32


def test_scaling_set_structure():
    for i in (0, 2):
        wl = synth.workload(f"scaling{i}")
        m = 3 ** (i + 7)
        X = synth.make_data(wl).numpy()
        assert X.shape == (m + 500, 10)
        noise = X[m:]
        assert np.all(np.abs(noise) <= 50.0)
        ws = synth.worker_setup(wl)
        assert np.all(ws.s == min(5000, m - 1000)) and np.all(ws.k == 10)
    # blob means inside (-40, 40)^10: every blob row is within a few sd of one
    X = synth.make_data(synth.workload("scaling2")).numpy()[: 3 ** 9]
    assert np.abs(X).max() < 40 + 10 * 8
