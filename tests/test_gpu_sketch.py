"""GPU parity of Algorithm 1 step 1 (the multisketch) against the CPU oracle, through the
C ABI: the CountSketch hash is bit-exact, W1 = S1 V is bit-exact on integer-valued V,
S2 agrees to a few ulp, and Ws = S2 S1 V is within the FP64 product bound."""
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


@pytest.mark.parametrize("seed,m,s1", [(0, 1, 1), (0, 1000, 544), (7, 300_001, 2112),
                                       (2**64 - 1, 100_000, 33024), (12345, 2**23, 8320),
                                       (3, 50_000, 2**31 - 1)])
def test_hash_bit_exact(rq, seed, m, s1):
    b, s = rq.randqr_cs_hash(seed, m, s1)
    bo, so = oracle.cs_hash(seed, m, s1)
    np.testing.assert_array_equal(b.cpu().numpy(), bo)
    np.testing.assert_array_equal(s.cpu().numpy(), so)


def test_hash_empty(rq):
    b, s = rq.randqr_cs_hash(0, 0, 10)
    assert b.numel() == 0 and s.numel() == 0


@pytest.mark.parametrize("seed,s2,s1", [(1, 64, 544), (99, 3, 7), (5, 256, 8320)])
def test_gauss_sketch_matches_oracle(rq, seed, s2, s1):
    S2 = rq.randqr_gauss_sketch(seed, s2, s1).cpu().numpy()
    So = oracle.gauss_sketch(seed, s2, s1)
    # same Philox integers; sqrt/log/cos from CUDA vs the host libm differ by a few ulp
    scale = 1 / np.sqrt(s2)
    assert np.abs(S2 - So).max() <= 64 * np.finfo(float).eps * scale * 8


@pytest.mark.parametrize("m,n,s1", [(1000, 1, 4), (3001, 7, 97), (20000, 16, 544),
                                    (50_000, 33, 2244), (40_000, 64, 8320), (10_000, 128, 33024)])
def test_countsketch_integer_bit_exact(rq, m, n, s1):
    # Integer entries: every partial sum is exact in FP64, so the atomics' order does not
    # matter and W1 must equal the oracle's bit for bit.  With S2 = I, Ws = W1 exactly.
    V = synthetic.integer_matrix(m, n, seed=m + n)
    Vd = torch.from_numpy(V).cuda()
    eye = torch.eye(s1, dtype=torch.float64, device="cuda") if s1 <= 9000 else None
    if eye is None:
        pytest.skip("identity S2 too large for this size")
    Ws = rq.randqr_sketch(Vd, s1, s1, seed=11, S2=eye).cpu().numpy()
    np.testing.assert_array_equal(Ws, oracle.countsketch(V, s1, 11))


@pytest.mark.parametrize("m,n,kappa,ld_pad", [(20000, 16, 1e10, 0), (12345, 33, 1e4, 3),
                                              (30000, 64, 1e14, 0), (9000, 128, 1e8, 1)])
def test_sketch_within_product_bound(rq, m, n, kappa, ld_pad):
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = synthetic.make_v(m, n, kappa, seed=4)
    S2 = oracle.gauss_sketch(9, s2, s1)
    Vbuf = torch.zeros((m, n + ld_pad), dtype=torch.float64, device="cuda")
    Vbuf[:, :n] = torch.from_numpy(V).cuda()
    Vd = Vbuf[:, :n]
    Ws = rq.randqr_sketch(Vd, s1, s2, seed=3, S2=torch.from_numpy(S2).cuda()).cpu().numpy()
    W1 = oracle.countsketch(V, s1, 3)
    Wo = oracle.gemm(S2, W1)
    b, sg = oracle.cs_hash(3, m, s1)
    absW1 = np.zeros((s1, n))
    np.add.at(absW1, b, np.abs(V))
    bound = 2 * (s1 + m / s1 + 8) * 2**-53 * (np.abs(S2) @ absW1)
    assert (np.abs(Ws - Wo) <= bound).all()


def test_sketch_uses_cached_seeded_s2(rq):
    m, n = 5000, 8
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = synthetic.make_v(m, n, 1e3, seed=2)
    Vd = torch.from_numpy(V).cuda()
    a = rq.randqr_sketch(Vd, s1, s2, seed=21).cpu().numpy()
    b = rq.randqr_sketch(Vd, s1, s2, seed=21,
                         S2=rq.randqr_gauss_sketch(22, s2, s1)).cpu().numpy()
    Wo = oracle.gemm(oracle.gauss_sketch(22, s2, s1), oracle.countsketch(V, s1, 21))
    assert np.abs(a - b).max() < 1e-13 and np.abs(a - Wo).max() < 1e-12


@pytest.mark.parametrize("s2,s1", [(1, 1), (64, 544), (256, 8320), (37, 1001), (776, 34279)])
def test_rademacher_sketch_bit_exact(rq, s2, s1):
    S2 = rq.randqr_rademacher_sketch(11, s2, s1).cpu().numpy()
    np.testing.assert_array_equal(S2, oracle.rademacher_sketch(11, s2, s1))


def test_rand_cholqr_with_rademacher_sketch_kind(rq):
    # the context's generated S2 (seed + 1) is the Rademacher sketch: same factors as the
    # explicit sketch, and parity with the oracle run on that sketch
    m, n = 20000, 16
    s1, s2 = synthetic.default_sketch_sizes(n)
    # kappa = 1e6: run-to-run differences (FP64 atomics in the scatter and the Gram) stay far
    # below the comparison bars
    V = synthetic.make_v(m, n, 1e6, seed=2)
    Vd = torch.from_numpy(V).cuda()
    ctx = rq.Context(0)
    ctx.set_sketch_kind(rq.SKETCH_RADEMACHER)
    Q, R, _ = rq.randqr_factor(Vd, s1, s2, seed=5, ctx=ctx)
    S2 = oracle.rademacher_sketch(6, s2, s1)
    Q2, R2, _ = rq.randqr_factor(Vd, s1, s2, seed=5, S2=torch.from_numpy(S2).cuda(), ctx=ctx)
    assert (Q - Q2).abs().max().item() <= 1e-12
    Q_ref, R_ref = oracle.rand_cholqr(V, s1, s2, 5, S2=S2)
    tq, tr = parity_tolerance(V, s1, s2)
    assert np.abs(Q.cpu().numpy() - Q_ref).max() <= tq
    assert np.abs(R.cpu().numpy() - R_ref).max() / np.abs(R_ref).max() <= tr
    ctx.set_sketch_kind(rq.SKETCH_GAUSSIAN)
    Qg, _, _ = rq.randqr_factor(Vd, s1, s2, seed=5, ctx=ctx)
    Qg2, _, _ = rq.randqr_factor(Vd, s1, s2, seed=5, S2=rq.randqr_gauss_sketch(6, s2, s1), ctx=ctx)
    assert (Qg - Qg2).abs().max().item() <= 1e-12
    with pytest.raises(rq.RandQRError):
        ctx.set_sketch_kind(7)
