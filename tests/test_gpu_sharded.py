"""Row-sharded rand_cholQR (Sec. 4.1) on one GPU: logical shards through the C ABI's stage
entry points (randqr_shard_sketch, randqr_sketch_r, randqr_shard_gram, randqr_shard_finish),
their partial sketches and Grams summed in shard order, against the CPU oracle and the
unsharded randqr_factor.

The shard sketch is checked bit for bit with integer V and a +-1 S2 (every product and sum
exact); the factorization to the stated tolerances (orthogonality <= 1e-12, residual <=
1e-13, Q and R within max(1e-10, 10 x the oracle's spread) of the oracle)."""
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


def _orth(Q):
    n = Q.shape[1]
    return torch.linalg.matrix_norm(Q.T @ Q - torch.eye(n, dtype=Q.dtype, device=Q.device),
                                    ord=2).item()


def _resid(V, Q, R):
    return (torch.linalg.norm(V - Q @ R) / torch.linalg.norm(V)).item()


@pytest.mark.parametrize("m,n,cuts", [
    (5000, 8, [0, 1, 2, 3, 4999, 5000]),
    (20000, 16, [0, 7000, 7001, 20000]),
    (130000, 64, [0, 127, 128, 65536, 130000]),
])
def test_shard_sketch_bit_exact(rq, m, n, cuts):
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = synthetic.integer_matrix(m, n, bound=2 ** 12, seed=n)
    S2 = np.where(synthetic.rng(n + 1).random((s2, s1)) < 0.5, -1.0, 1.0)
    Vd, S2d = torch.from_numpy(V).cuda(), torch.from_numpy(S2).cuda()
    total = torch.zeros((s2, n), dtype=torch.float64, device="cuda")
    for r0, r1 in zip(cuts[:-1], cuts[1:]):
        Wk = rq.randqr_shard_sketch(Vd[r0:r1], r0, s1, s2, seed=7, S2=S2d)
        ref = oracle.gemm(S2, oracle.countsketch_rows(V[r0:r1], s1, 7, r0))
        np.testing.assert_array_equal(Wk.cpu().numpy(), ref)
        total += Wk
    Ws_ref = oracle.randqr(V, s1, s2, 7, S2=S2)[3]
    np.testing.assert_array_equal(total.cpu().numpy(), Ws_ref)


@pytest.mark.parametrize("m,n,kappa,cuts", [
    (20000, 16, 1e10, [0, 5000, 10000, 15000, 20000]),
    (12001, 33, 1e8, [0, 3, 6000, 12001]),
    (20000, 64, 1e14, [0, 1, 19999, 20000]),
    (20000, 128, 1e12, [0, 10000, 20000]),
])
def test_logical_shards_parity_with_oracle(rq, m, n, kappa, cuts):
    from paper_2309_05868_gb300 import sharded
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = synthetic.make_v(m, n, kappa, seed=m % 89)
    S2 = oracle.gauss_sketch(1, s2, s1)
    Vd = torch.from_numpy(V).cuda()
    Q, R = sharded.factor_logical_shards(Vd, cuts, s1, s2, seed=0, S2=torch.from_numpy(S2).cuda())
    assert _orth(Q) <= 1e-12
    assert _resid(Vd, Q, R) <= 1e-13
    Rh = R.cpu().numpy()
    assert np.array_equal(Rh, np.triu(Rh)) and (np.diag(Rh) > 0).all()
    Q_ref, R_ref = oracle.rand_cholqr(V, s1, s2, 0, S2=S2)
    tq, tr = parity_tolerance(V, s1, s2)
    assert np.abs(Q.cpu().numpy() - Q_ref).max() <= tq
    assert np.abs(Rh - R_ref).max() / np.abs(R_ref).max() <= tr


@pytest.mark.parametrize("shards", [1, 3, 8])
def test_logical_shards_match_unsharded_at_scale(rq, shards):
    from paper_2309_05868_gb300 import sharded
    m, n = (1 << 21) + 37, 64
    s1, s2 = synthetic.default_sketch_sizes(n)
    cuts = sharded.even_cuts(m, shards)
    # kappa = 1e4: both results are the unique QR factors of V to O(u kappa) = 1e-12
    V = synthetic.make_v_torch(m, n, 1e4, seed=3)
    Q0, R0, _ = rq.randqr_factor(V, s1, s2, seed=0)
    Q, R = sharded.factor_logical_shards(V, cuts, s1, s2, seed=0)
    assert (Q - Q0).abs().max().item() <= 1e-11
    assert ((R - R0).abs().max() / R0.abs().max()).item() <= 1e-11
    del V, Q, Q0
    # kappa = 1e12: the accuracy bars
    V = synthetic.make_v_torch(m, n, 1e12, seed=4)
    Q, R = sharded.factor_logical_shards(V, cuts, s1, s2, seed=0)
    assert _orth(Q) <= 1e-12 and _resid(V, Q, R) <= 1e-13
    del V, Q


def test_in_place_shards(rq):
    from paper_2309_05868_gb300 import sharded
    m, n = 50000, 32
    V = synthetic.make_v_torch(m, n, 1e8, seed=5)
    Vc = V.clone()
    Q, R = sharded.factor_logical_shards(V, sharded.even_cuts(m, 4), seed=2, Q=V)
    assert Q.data_ptr() == V.data_ptr()
    assert _orth(Q) <= 1e-12 and _resid(Vc, Q, R) <= 1e-13


def test_stage_argument_errors(rq):
    V = torch.zeros((100, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(rq.RandQRError) as e:
        rq.randqr_shard_sketch(V, -1, 144, 32)
    assert e.value.name == "ERR_ARG"
    with pytest.raises(rq.RandQRError):
        rq.randqr_shard_sketch(V, 0, 144, 4)      # s2 < n
    Ws = torch.zeros((4, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(rq.RandQRError):
        rq.randqr_sketch_r(Ws)                    # s2 < n
    G = torch.eye(8, dtype=torch.float64, device="cuda")
    with pytest.raises(rq.RandQRError):
        rq.randqr_shard_gram(V, G, Q=V[:, :8], G=V[:8])   # G overlaps Q
    # a rank-deficient sketch reports through the status
    Ws = torch.zeros((32, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(rq.RandQRError) as e:
        rq.randqr_sketch_r(Ws)
    assert e.value.name in ("ERR_RANK", "ERR_NONFINITE")
    # an indefinite Gram is reported by the finish stage
    Gbad = -torch.eye(8, dtype=torch.float64, device="cuda")
    Q = torch.ones((10, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(rq.RandQRError) as e:
        rq.randqr_shard_finish(Q, Gbad, torch.eye(8, dtype=torch.float64, device="cuda"))
    assert e.value.name == "ERR_NOT_SPD"
