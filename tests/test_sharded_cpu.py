"""Row-sharded rand_cholQR (Sec. 4.1) on the CPU: the orchestration in
``paper_2309_05868_gb300.sharded`` driven by oracle stages, as logical shards in one process
and as two gloo ranks.  No GPU."""
import os
import socket

import numpy as np
import pytest

import oracle
import synthetic
from paper_2309_05868_gb300 import sharded
from shard_worker import OracleStages, rank_main


class Recording(OracleStages):
    """Oracle stages that also keep the summed sketch and Gram the driver hands on."""

    def __init__(self, as_torch=False):
        super().__init__(as_torch)
        self.Ws = None
        self.G = None

    def sketch_r(self, Ws):
        self.Ws = np.array(self._np(Ws))
        return super().sketch_r(Ws)

    def finish(self, Q, G, Rs):
        self.G = np.array(self._np(G))
        return super().finish(Q, G, Rs)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_even_cuts():
    assert sharded.even_cuts(10, 3) == [0, 4, 7, 10]
    assert sharded.even_cuts(2, 4) == [0, 1, 2, 2, 2]
    for m, p in ((1000, 7), (5, 5), (1 << 20, 8)):
        c = sharded.even_cuts(m, p)
        assert c[0] == 0 and c[-1] == m and len(c) == p + 1
        assert max(np.diff(c)) - min(np.diff(c)) <= 1


def test_shard_sketches_sum_to_the_global_sketch_exactly():
    # Integer V and a +-1 S2 keep every product and sum exact, so the summed shard sketches
    # equal the unsharded Ws bit for bit (and a wrong row offset would not).
    m, n = 4000, 6
    s1, s2 = 2 * (n * n + n), 4 * n
    V = synthetic.integer_matrix(m, n, bound=2 ** 10, seed=4)
    S2 = np.where(synthetic.rng(5).random((s2, s1)) < 0.5, -1.0, 1.0)
    Ws_global = oracle.randqr(V, s1, s2, 3, S2=S2)[3]
    rec = Recording()
    Q = np.empty_like(V)
    sharded.factor_logical_shards(V, [0, 3, 1000, 1001, 4000], s1, s2, seed=3, S2=S2, Q=Q,
                                  stages=rec)
    np.testing.assert_array_equal(rec.Ws, Ws_global)
    # the same shards with every offset taken as 0 give another sketch
    wrong = sum(oracle.gemm(S2, oracle.countsketch_rows(V[a:b], s1, 3, 0))
                for a, b in ((0, 3), (3, 1000), (1000, 1001), (1001, 4000)))
    assert np.abs(wrong - Ws_global).max() > 0


@pytest.mark.parametrize("cuts", [[0, 2500], [0, 5, 1200, 1201, 2500], [0, 1, 2, 3, 2500]])
def test_logical_shards_match_the_unsharded_oracle(cuts):
    m, n, kappa = 2500, 12, 1e4
    V = synthetic.make_v(m, n, kappa, seed=6)
    Q_ref, R_ref = oracle.rand_cholqr(V, 2 * (n * n + n), 4 * n, 0)
    Q = np.empty_like(V)
    Q, R = sharded.factor_logical_shards(V, cuts, seed=0, Q=Q, stages=OracleStages(False))
    # the shards change only the order of the two sums: both results are the unique QR
    # factors of V to O(u kappa)
    assert _rel(R, R_ref) <= 1e-12
    assert _rel(Q, Q_ref) <= 1e-11
    if len(cuts) == 2:
        np.testing.assert_array_equal(Q, Q_ref)
        np.testing.assert_array_equal(R, R_ref)


def test_logical_shards_ill_conditioned():
    m, n, kappa = 3000, 10, 1e13
    V = synthetic.make_v(m, n, kappa, seed=7)
    Q = np.empty_like(V)
    Q, R = sharded.factor_logical_shards(V, sharded.even_cuts(m, 4), seed=1, Q=Q,
                                         stages=OracleStages(False))
    e2, _ = oracle.orth_err(Q)
    assert e2 <= 1e-13
    assert oracle.resid(V, Q, R) <= 1e-14
    assert (np.diag(R) > 0).all() and np.array_equal(R, np.triu(R))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_match_logical_shards(tmp_path):
    import torch.multiprocessing as mp
    oracle._load()  # build the oracle once, before the ranks start
    m, n, kappa, seed = 2001, 9, 1e6, 2
    cuts = [0, 1100, m]
    mp.start_processes(rank_main, args=(2, _free_port(), m, n, kappa, seed, cuts, str(tmp_path)),
                       nprocs=2, join=True, start_method="spawn")
    parts = [np.load(tmp_path / f"rank{r}.npz") for r in range(2)]
    # every rank holds the same R
    np.testing.assert_array_equal(parts[0]["R"], parts[1]["R"])
    V = synthetic.make_v(m, n, kappa, seed=seed)
    Q_log = np.empty_like(V)
    Q_log, R_log = sharded.factor_logical_shards(V, cuts, seed=seed, Q=Q_log,
                                                 stages=OracleStages(False))
    Q = np.concatenate([p["Q"] for p in parts])
    # a two-term allreduce adds in either order: the result is the fixed-order sum
    np.testing.assert_array_equal(parts[0]["R"], R_log)
    np.testing.assert_array_equal(Q, Q_log)
    Q_ref, R_ref = oracle.rand_cholqr(V, 2 * (n * n + n), 4 * n, seed)
    assert _rel(R_log, R_ref) <= 1e-11 and _rel(Q_log, Q_ref) <= 1e-9
