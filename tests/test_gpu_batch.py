"""Batched rand_cholQR (randqr_factor_batched): uneven matrices in one autotuned CUDA graph.

Each item's result meets the orthogonality and residual targets and equals the single-call
result within the parity tolerance; a graph replay reproduces it; a failing item is
reported on its own while the others succeed."""
import numpy as np
import pytest

import oracle
import synthetic
from gpu_util import parity_tolerance

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rq():
    import paper_2309_05868_gb300 as rq
    return rq


def _batch(count, seed=0):
    rng = np.random.default_rng(seed)
    shapes = []
    for i in range(count):
        m = int(np.exp(rng.uniform(np.log(3000), np.log(60000))))
        n = int(rng.choice([8, 16, 32, 64]))
        m = max(m, 4 * n)
        kappa = float(10 ** rng.uniform(0, 12))
        shapes.append((m, n, kappa))
    Vh = [synthetic.make_v(m, n, k, seed=i) for i, (m, n, k) in enumerate(shapes)]
    Vs = [torch.from_numpy(v).cuda() for v in Vh]
    Qs = [torch.empty_like(v) for v in Vs]
    Rs = [torch.empty((v.shape[1], v.shape[1]), dtype=torch.float64, device="cuda") for v in Vs]
    return shapes, Vh, Vs, Qs, Rs


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_matches_single_calls(rq, prec):
    shapes, Vh, Vs, Qs, Rs = _batch(40, seed=prec)
    ctx = rq.Context(0)
    items = rq.batch_items(Vs, Qs, Rs, seeds=list(range(40)))
    sts = rq.randqr_factor_batched(ctx, items, prec=prec)
    assert all(s == 0 for s in sts)
    lanes, ms = rq.randqr_batch_plan_info(ctx, items, prec=prec)
    assert lanes in (4, 8, 16, 32) and ms > 0
    first = [(q.cpu().numpy(), r.cpu().numpy()) for q, r in zip(Qs, Rs)]
    for q in Qs:
        q.zero_()
    assert all(s == 0 for s in rq.randqr_factor_batched(ctx, items, prec=prec))  # graph replay
    for i in range(0, 40, 3):
        Q, R = Qs[i].cpu().numpy(), Rs[i].cpu().numpy()
        m, n, k = shapes[i]
        s1, s2 = synthetic.default_sketch_sizes(n)
        tq, tr = parity_tolerance(Vh[i], s1, s2)
        scale = 64 if prec == 1 else 1
        # a replay differs from the first run only by the order of atomic additions
        assert np.abs(Q - first[i][0]).max() <= scale * tq
        assert oracle.orth_err(Q)[0] <= 1e-12 and oracle.resid(Vh[i], Q, R) <= 1e-13
        Qs1, Rs1, _ = rq.randqr_factor(Vs[i], seed=i, prec=prec)
        assert np.abs(Q - Qs1.cpu().numpy()).max() <= scale * tq
        assert np.abs(R - Rs1.cpu().numpy()).max() / np.abs(R).max() <= scale * tr
        # and against the oracle itself (its own S2 for seed + 1: the device's Gaussian
        # entries agree with the host's to a few ulp, and Q, R are the unique QR factors of
        # V whatever the sketch, within the parity tolerance)
        Qo, Ro = oracle.rand_cholqr(Vh[i], s1, s2, seed=i)
        assert np.abs(Q - Qo).max() <= scale * tq
        assert np.abs(R - Ro).max() / np.abs(Ro).max() <= scale * tr
    ctx.close()


def test_batched_failing_item_is_isolated(rq):
    shapes, Vh, Vs, Qs, Rs = _batch(12, seed=5)
    Vs[4][:, 2] = 0.0  # rank deficient: R_s has a zero diagonal
    ctx = rq.Context(0)
    items = rq.batch_items(Vs, Qs, Rs)
    sts = rq.randqr_factor_batched(ctx, items)
    assert sts[4] == -3
    assert all(s == 0 for i, s in enumerate(sts) if i != 4)
    ctx.close()
