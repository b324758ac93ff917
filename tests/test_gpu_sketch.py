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
                                    (50_000, 33, 2244), (40_000, 64, 8320), (10_000, 128, 33024),
                                    (30_001, 100, 3000), (40_000, 128, 4000), (5000, 97, 1000)])
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


# ---- the Gaussian sketch GEMM as split products on the tensor cores (n <= 64) ------------

def _gaussian_only_ctx(rq, tensor_cores=True):
    ctx = rq.Context(0)
    ctx.set_sketch_kind(rq.SKETCH_GAUSSIAN_ONLY)  # Ws = S2 V: the GEMM alone, K = m
    ctx.set_tensor_cores(tensor_cores)
    return ctx


@pytest.mark.parametrize("m,n,s2", [(64, 1, 1), (1037, 5, 130), (4099, 33, 257), (20000, 64, 64),
                                    (70001, 64, 300)])
def test_sketch_gemm_exact_on_integers(rq, m, n, s2):
    # +-1 S2 and integer V: every digit product and every sum is an exact integer, so the
    # split product equals S2 V bit for bit (ragged chunks of K, ragged 128-row tiles)
    V = synthetic.integer_matrix(m, n, bound=2 ** 12, seed=m % 97)
    S2 = np.where(synthetic.rng(s2 + 5).random((s2, m)) < 0.5, -1.0, 1.0)
    ctx = _gaussian_only_ctx(rq)
    Ws = rq.randqr_sketch(torch.from_numpy(V).cuda(), m, s2, S2=torch.from_numpy(S2).cuda(), ctx=ctx)
    np.testing.assert_array_equal(Ws.cpu().numpy(), S2 @ V)  # integer sums below 2^53: exact


def _split_product_bound(S2, V, chunk=64):
    # The split product's error for chunk c of K: each term is cut relative to the chunk's
    # largest |a_ik| and |b_kj| (scales 2^E < 2 max), truncation 2^-54 of the scale on each
    # factor and the dropped digit pairs below 2^-58 of the product of the scales; then one
    # rounding per chunk and the FP64 sum of the chunks.
    s2, m = S2.shape
    bound = np.zeros((s2, V.shape[1]))
    for c0 in range(0, m, chunk):
        a = np.abs(S2[:, c0:c0 + chunk]).max(axis=1)
        b = np.abs(V[c0:c0 + chunk]).max(axis=0)
        L = min(chunk, m - c0)
        bound += np.outer(2 * a, 2 * b) * L * (2 * 2.0 ** -54 + 2.0 ** -58)
    nchunks = -(-m // chunk)
    return bound + (nchunks + 1) * 2.0 ** -52 * (np.abs(S2) @ np.abs(V))


@pytest.mark.parametrize("m,n,s2", [(3000, 16, 64), (9001, 64, 130)])
def test_sketch_gemm_within_split_bound(rq, m, n, s2):
    # rows of V spread over 2^-60 .. 2^60 and a Gaussian S2: the result against S2 V in
    # extended precision, within the split product's bound, for the tensor-core and the
    # CUDA-core GEMM alike
    rng = synthetic.rng(m)
    V = rng.standard_normal((m, n)) * np.exp2(rng.integers(-60, 61, size=(m, 1)).astype(float))
    S2 = oracle.gauss_sketch(3, s2, m)
    exact = (S2.astype(np.longdouble) @ V.astype(np.longdouble)).astype(np.float64)
    bound = _split_product_bound(S2, V)
    for tc in (True, False):
        ctx = _gaussian_only_ctx(rq, tc)
        Ws = rq.randqr_sketch(torch.from_numpy(V).cuda(), m, s2, S2=torch.from_numpy(S2).cuda(), ctx=ctx)
        err = np.abs(Ws.cpu().numpy() - exact)
        assert (err <= bound).all(), (tc, (err / bound).max())


@pytest.mark.parametrize("n", [8, 64])
def test_sketch_at_paper_sizes_within_product_bound(rq, n):
    # the paper's multisketch sizes (Sec. 6.2): s1 odd for n = 64 (34279), so the rows of S2
    # start at every alignment
    m = 60000
    s1, s2 = synthetic.paper_multisketch_sizes(n)
    V = synthetic.make_v(m, n, 1e8, seed=n)
    S2 = oracle.gauss_sketch(4, s2, s1)
    Ws = rq.randqr_sketch(torch.from_numpy(V).cuda(), s1, s2, seed=5, S2=torch.from_numpy(S2).cuda()).cpu().numpy()
    W1 = oracle.countsketch(V, s1, 5)
    Wo = oracle.gemm(S2, W1)
    b, _ = oracle.cs_hash(5, m, s1)
    absW1 = np.zeros((s1, n))
    np.add.at(absW1, b, np.abs(V))
    bound = _split_product_bound(S2, W1) + 2 * (s1 + m / s1 + 8) * 2.0 ** -53 * (np.abs(S2) @ absW1)
    assert (np.abs(Ws - Wo) <= bound).all()


def test_rademacher_generated_inside_the_sketch_gemm(rq):
    """With the Rademacher kind and no S2 passed, the tensor-core sketch GEMM draws the signs
    itself (Sec. 7's dense alternative, generated on the fly): no S2 buffer is held, and Ws is
    what the materialised Rademacher S2 gives -- bit for bit on integer V with s2 = 64 (entries
    +-1/8, every product exact), within the FP64 atomics' reordering otherwise."""
    m, n = 50000, 16
    s1, s2 = synthetic.default_sketch_sizes(n)
    Vi = torch.from_numpy(synthetic.integer_matrix(m, n, seed=4)).cuda()
    ctx = rq.Context(0)
    ctx.set_sketch_kind(rq.SKETCH_RADEMACHER)
    fly = rq.randqr_sketch(Vi, s1, s2, seed=5, ctx=ctx)
    assert ctx.workspace_bytes() < 8 * s1 * s2  # the sketch matrix was never materialised
    S2 = rq.randqr_rademacher_sketch(6, s2, s1)
    mat = rq.randqr_sketch(Vi, s1, s2, seed=5, S2=S2, ctx=ctx)
    assert torch.equal(fly, mat)
    np.testing.assert_array_equal(fly.cpu().numpy(),
                                  oracle.gemm(oracle.rademacher_sketch(6, s2, s1),
                                              oracle.countsketch(Vi.cpu().numpy(), s1, 5)))
    m, n = 40000, 64
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = torch.from_numpy(synthetic.make_v(m, n, 1e10, seed=6)).cuda()
    fly = rq.randqr_sketch(V, s1, s2, seed=7, ctx=ctx)
    mat = rq.randqr_sketch(V, s1, s2, seed=7, S2=rq.randqr_rademacher_sketch(8, s2, s1), ctx=ctx)
    assert (fly - mat).abs().max().item() <= 1e-13 * mat.abs().max().item()
    Q, R, _ = rq.randqr_factor(V, s1, s2, seed=7, ctx=ctx)
    Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
    assert oracle.orth_err(Qh)[0] <= 1e-12 and oracle.resid(V.cpu().numpy(), Qh, Rh) <= 1e-13
    ctx.close()
