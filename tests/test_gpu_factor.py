"""GPU parity of the factorizations (rand_cholQR, randQR, CholeskyQR2, shifted CholeskyQR3)
against the CPU oracle through the C ABI, on the same seeded inputs and the same S2.

Tolerances: orthogonality ||I - Q^T Q||_2 <= 1e-12 and residual ||V - QR||_F/||V||_F <=
1e-13 for kappa(V) up to 1e14 (FP64); Q and R within max(1e-10, 10 x the oracle's own
spread between two sketches) of the oracle -- see tests/gpu_util.py."""
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


def _run(rq, V, s1, s2, seed, S2, ld_pad=0, inplace=False, prec=0):
    m, n = V.shape
    buf = torch.zeros((m, n + ld_pad), dtype=torch.float64, device="cuda")
    buf[:, :n] = torch.from_numpy(V).cuda()
    Vd = buf[:, :n]
    S2d = torch.from_numpy(S2).cuda()
    if inplace:
        Q, R, info = rq.randqr_factor(Vd, s1, s2, seed=seed, S2=S2d, Q=Vd, prec=prec)
    else:
        Q, R, info = rq.randqr_factor(Vd, s1, s2, seed=seed, S2=S2d, prec=prec)
    return Q.cpu().numpy(), R.cpu().numpy(), info


CASES = [  # m, n, kappa
    (20000, 16, 1e10),     # the small benchmarked configuration
    (3001, 1, 1.0), (2999, 2, 1e3), (5003, 3, 1e6), (4097, 5, 1e12), (6000, 7, 1e14),
    (10000, 32, 1e0), (10000, 32, 1e4), (12001, 33, 1e8), (30000, 64, 1e8), (20000, 64, 1e12),
    (20000, 64, 1e14), (16385, 100, 1e8), (20000, 128, 1e4), (20000, 128, 1e14),
]


@pytest.mark.parametrize("m,n,kappa", CASES)
def test_rand_cholqr_parity(rq, m, n, kappa):
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = synthetic.make_v(m, n, kappa, seed=m % 97)
    S2 = oracle.gauss_sketch(1, s2, s1)
    Q, R, info = _run(rq, V, s1, s2, 0, S2)
    e2, eF = oracle.orth_err(Q)
    res = oracle.resid(V, Q, R)
    assert e2 <= 1e-12, e2
    assert res <= 1e-13, res
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    Qo, Ro = oracle.rand_cholqr(V, s1, s2, seed=0, S2=S2)
    tq, tr = parity_tolerance(V, s1, s2)
    assert np.abs(Q - Qo).max() <= tq
    assert np.abs(R - Ro).max() / np.abs(Ro).max() <= tr


@pytest.mark.parametrize("m,n,kappa", [(20000, 8, 1e12), (20000, 32, 1e14), (30000, 64, 1e12)])
def test_rand_cholqr_parity_paper_sketch_sizes(rq, m, n, kappa):
    # the paper's multisketch sizes (Sec. 6.2): s1 = ceil(8.24 (n^2 + n)), s2 = ceil(74.3 ln s1)
    s1, s2 = synthetic.paper_multisketch_sizes(n)
    V = synthetic.make_v(m, n, kappa, seed=n)
    S2 = oracle.gauss_sketch(1, s2, s1)
    Q, R, _ = _run(rq, V, s1, s2, 0, S2)
    e2, _ = oracle.orth_err(Q)
    assert e2 <= 1e-12 and oracle.resid(V, Q, R) <= 1e-13
    Qo, Ro = oracle.rand_cholqr(V, s1, s2, seed=0, S2=S2)
    tq, tr = parity_tolerance(V, s1, s2)
    assert np.abs(Q - Qo).max() <= tq
    assert np.abs(R - Ro).max() / np.abs(Ro).max() <= tr


@pytest.mark.parametrize("ld_pad,inplace", [(1, False), (5, True), (0, True)])
def test_leading_dims_and_in_place(rq, ld_pad, inplace):
    m, n = 7777, 24
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = synthetic.make_v(m, n, 1e9, seed=5)
    S2 = oracle.gauss_sketch(3, s2, s1)
    Q, R, _ = _run(rq, V, s1, s2, 2, S2, ld_pad=ld_pad, inplace=inplace)
    Qo, Ro = oracle.rand_cholqr(V, s1, s2, seed=2, S2=S2)
    tq, tr = parity_tolerance(V, s1, s2)
    assert np.abs(Q - Qo).max() <= tq and np.abs(R - Ro).max() / np.abs(Ro).max() <= tr


def test_randqr_alone_matches_oracle(rq):
    m, n = 15000, 20
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = synthetic.make_v(m, n, 1e6, seed=6)
    S2 = oracle.gauss_sketch(4, s2, s1)
    Q0, R0, info = rq.randqr_randqr(torch.from_numpy(V).cuda(), s1, s2, seed=3,
                                    S2=torch.from_numpy(S2).cuda())
    Q0, R0 = Q0.cpu().numpy(), R0.cpu().numpy()
    Q0o, R0o, _, _ = oracle.randqr(V, s1, s2, seed=3, S2=S2)
    # R_s comes from a backward-stable QR of the same sketch: rows agree to ~u kappa(Ws)
    assert np.abs(R0 - R0o).max() / np.abs(R0o).max() < 1e-9
    assert np.linalg.cond(Q0) < 10
    assert np.abs(Q0 - Q0o).max() < 1e-7
    assert info.rs_min_diag > 0 and info.rs_max_diag >= info.rs_min_diag


@pytest.mark.parametrize("m,n,kappa,tc", [(30000, 64, 1e12, True), (20000, 100, 1e10, True),
                                          (20000, 64, 1e10, False)])
def test_randqr_alone_solve_paths(rq, m, n, kappa, tc):
    """randQR alone through the split-product solve (n = 64: one product with R_s^{-1};
    n = 100: blocked at n1 = 36) and through FP64 substitution (tensor cores off): Q0 against
    the oracle's V R_s^{-1} to within the perturbation theory of a triangular solve with the
    same R_s (u kappa(V) relative to |Q0|, with a margin), and R0 = R_s."""
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = synthetic.make_v(m, n, kappa, seed=n + 1)
    S2 = oracle.gauss_sketch(7, s2, s1)
    ctx = rq.Context(0)
    ctx.set_tensor_cores(tc)
    Q0, R0, _ = rq.randqr_randqr(torch.from_numpy(V).cuda(), s1, s2, seed=5,
                                 S2=torch.from_numpy(S2).cuda(), ctx=ctx)
    ctx.close()
    Q0, R0 = Q0.cpu().numpy(), R0.cpu().numpy()
    Q0o, R0o, _, _ = oracle.randqr(V, s1, s2, seed=5, S2=S2)
    assert np.abs(R0 - R0o).max() / np.abs(R0o).max() < 1e-9
    assert np.linalg.cond(Q0) < 10
    assert np.abs(Q0 - Q0o).max() <= 100 * kappa * 2.0**-53 * np.abs(Q0o).max()


@pytest.mark.parametrize("m,n,kappa", [(20000, 32, 1.0), (20000, 32, 1e5), (30001, 64, 1e7), (20000, 100, 1e6)])
def test_cholqr2_parity(rq, m, n, kappa):
    # both passes' solves are split products with the computed inverses (n = 100: blocked)
    V = synthetic.make_v(m, n, kappa, seed=8)
    Q, R, _ = rq.randqr_cholqr2(torch.from_numpy(V).cuda())
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    Qo, Ro = oracle.cholqr2(V)
    assert oracle.orth_err(Q)[0] <= 1e-13 and oracle.resid(V, Q, R) <= 1e-14
    assert np.abs(Q - Qo).max() <= max(1e-10, 1e-14 * kappa**2)
    # R0 = chol(V^T V) moves by up to u kappa(V) (normwise) under the Gram's rounding
    assert np.abs(R - Ro).max() / np.abs(Ro).max() <= max(1e-12, 1e-16 * kappa)


@pytest.mark.parametrize("m,n,kappa", [(20000, 32, 1.0), (20000, 32, 1e9), (30000, 64, 1e12), (20000, 128, 1e10)])
def test_shifted_cholqr3_parity(rq, m, n, kappa):
    V = synthetic.make_v(m, n, kappa, seed=9)
    Q, R, _ = rq.randqr_shifted_cholqr3(torch.from_numpy(V).cuda())
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    Qo, Ro = oracle.scholqr3(V)
    assert oracle.orth_err(Q)[0] <= 1e-13 and oracle.resid(V, Q, R) <= 1e-14
    assert np.abs(R - Ro).max() / np.abs(Ro).max() <= max(1e-10, 1e-15 * kappa)


def _fails(rq, fn, Vd):
    try:
        Q, R, _ = fn(Vd)
    except rq.RandQRError as e:
        assert e.name == "ERR_NOT_SPD" and e.info.info >= 1 and e.info.stage >= 1
        return True
    Qh = Q.cpu().numpy()
    return not np.isfinite(Qh).all() or oracle.orth_err(Qh)[0] > 1e-6


def test_failure_points_sec63(rq):
    """cholQR2 breaks down past kappa ~ 1e8 (status NOT_SPD with stage and pivot, or a
    useless Q), sCholQR3 past ~1e12, while rand_cholQR stays accurate (Sec. 6.3)."""
    m, n = 20000, 32
    Vd = torch.from_numpy(synthetic.make_v(m, n, 1e13, seed=10)).cuda()
    assert _fails(rq, rq.randqr_cholqr2, Vd)
    Vd = torch.from_numpy(synthetic.make_v(m, n, 1e16, seed=10)).cuda()
    assert _fails(rq, rq.randqr_shifted_cholqr3, Vd)
    Vd = torch.from_numpy(synthetic.make_v(m, n, 1e15, seed=10)).cuda()
    Q, R, _ = rq.randqr_factor(Vd)
    assert oracle.orth_err(Q.cpu().numpy())[0] <= 1e-12
    # the context recovers: a later call on a good matrix succeeds
    V2 = torch.from_numpy(synthetic.make_v(m, n, 10.0, seed=1)).cuda()
    rq.randqr_cholqr2(V2)


def test_rank_deficient_and_nonfinite_inputs(rq):
    m, n = 5000, 8
    V = synthetic.make_v(m, n, 10.0, seed=11)
    V[:, 3] = 0.0
    with pytest.raises(rq.RandQRError) as e:
        rq.randqr_factor(torch.from_numpy(V).cuda())
    assert e.value.name == "ERR_RANK"
    V = synthetic.make_v(m, n, 10.0, seed=11)
    V[17, 2] = np.nan
    with pytest.raises(rq.RandQRError) as e:
        rq.randqr_factor(torch.from_numpy(V).cuda())
    assert e.value.name in ("ERR_RANK", "ERR_NOT_SPD")


def test_argument_errors_enqueue_nothing(rq):
    V = torch.zeros((100, 8), dtype=torch.float64, device="cuda")
    for kw in [dict(s1=10, s2=4), dict(s1=5, s2=20), dict(s1=2**31, s2=32)]:
        with pytest.raises(rq.RandQRError) as e:
            rq.randqr_factor(V, **kw)
        assert e.value.name == "ERR_ARG"
    with pytest.raises(rq.RandQRError):
        rq.randqr_factor(torch.zeros((100, 129), dtype=torch.float64, device="cuda"))
    with pytest.raises(rq.RandQRError):  # Q overlapping V without being V
        big = torch.zeros((200, 8), dtype=torch.float64, device="cuda")
        rq.randqr_factor(big[:100], s1=144, s2=32, Q=big[50:150])


def test_full_size_sampled(rq):
    """m = 2^23, n = 64, kappa = 1e12 in the benchmarked launch configuration: the hash is
    bit-exact on every row, R_s matches the oracle's (its sketch and Householder steps are
    cheap enough to run in full), sampled rows satisfy Q_i R = V_i, and orthogonality and
    the residual hold on the whole matrix."""
    m, n, kappa = 2**23, 64, 1e12
    s1, s2 = synthetic.default_sketch_sizes(n)
    Vd = synthetic.make_v_torch(m, n, kappa, seed=0)
    Q, R, info = rq.randqr_factor(Vd, s1, s2, seed=0)
    G = (Q.T @ Q).cpu().numpy()
    e2 = oracle.sym_absmax_eig(G - np.eye(n))
    res = (torch.linalg.norm(Vd - Q @ R) / torch.linalg.norm(Vd)).item()
    assert e2 <= 1e-12 and res <= 1e-13, (e2, res)
    Vh = Vd.cpu().numpy()
    S2 = oracle.gauss_sketch(1, s2, s1)  # the context's cached S2 for seed 0 (seed + 1)
    _, R0, _ = rq.randqr_randqr(Vd, s1, s2, seed=0)
    W1 = oracle.countsketch(Vh, s1, 0)
    R0o = oracle.hhqr_r(oracle.gemm(S2, W1))
    assert np.abs(R0.cpu().numpy() - R0o).max() / np.abs(R0o).max() < 1e-9
    rows = synthetic.rng(1).choice(m, 2000, replace=False)
    Qs, Rh = Q[torch.from_numpy(rows).cuda()].cpu().numpy(), R.cpu().numpy()
    assert oracle.resid(Vh[rows], Qs, Rh) <= 1e-13
    b, sg = rq.randqr_cs_hash(0, m, s1)
    bo, so = oracle.cs_hash(0, m, s1)
    assert np.array_equal(b.cpu().numpy(), bo) and np.array_equal(sg.cpu().numpy(), so)


def test_full_size_elementwise_against_oracle(rq):
    """The benchmarked configuration (m = 2^23, n = 64, kappa = 1e12, s1 = 8320, s2 = 256, S2
    passed in) in the launch configuration the bench times: every element of Q and R against
    the oracle on the same V and S2, at the parity tolerance max(1e-10, 10 x the oracle's own
    two-sketch spread) measured on this V.  The three oracle runs (about two minutes each)
    go in parallel threads (the ctypes calls release the interpreter lock)."""
    import threading
    m, n, kappa = 2**23, 64, 1e12
    s1, s2 = synthetic.default_sketch_sizes(n)
    Vd = synthetic.make_v_torch(m, n, kappa, seed=0)
    S2 = oracle.gauss_sketch(1, s2, s1)
    Q, R, _ = rq.randqr_factor(Vd, s1, s2, seed=0, S2=torch.from_numpy(S2).cuda())
    Vh, Qh, Rh = Vd.cpu().numpy(), Q.cpu().numpy(), R.cpu().numpy()
    del Q, R, Vd
    torch.cuda.empty_cache()
    out = {}

    def run(key, seed, S):
        out[key] = oracle.rand_cholqr(Vh, s1, s2, seed=seed, S2=S)

    jobs = [threading.Thread(target=run, args=("o", 0, S2)),
            threading.Thread(target=run, args=("a", 0, None)),
            threading.Thread(target=run, args=("b", 1, None))]
    for j in jobs:
        j.start()
    for j in jobs:
        j.join()
    Qo, Ro = out["o"]
    dq = np.abs(out["a"][0] - out["b"][0]).max()
    dr = np.abs(out["a"][1] - out["b"][1]).max() / np.abs(out["a"][1]).max()
    tq, tr = max(1e-10, 10 * dq), max(1e-10, 10 * dr)
    eq = np.abs(Qh - Qo).max()
    er = np.abs(Rh - Ro).max() / np.abs(Ro).max()
    assert eq <= tq, (eq, tq)
    assert er <= tr, (er, tr)


@pytest.mark.parametrize("m,n,kappa,inplace", [(30000, 66, 1e12, False), (20000, 100, 1e14, False),
                                                 (40001, 128, 1e8, False), (20000, 128, 1e15, True),
                                                 (9999, 97, 1e10, False), (20000, 96, 1e12, False),
                                                 (30001, 98, 1e10, True)])
def test_blocked_solves_64_to_128(rq, m, n, kappa, inplace):
    """64 < n <= 128 (even n): both solves blocked into split products at n1 = n - 64 (the
    off-diagonal block by substitution order for the first solve, through the inverse for the
    well-conditioned second); odd n keeps the substitution kernels.  Targets and parity as for
    every other size."""
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = synthetic.make_v(m, n, kappa, seed=n)
    S2 = oracle.gauss_sketch(1, s2, s1)
    Q, R, _ = _run(rq, V, s1, s2, 0, S2, inplace=inplace)
    e2, _ = oracle.orth_err(Q)
    assert e2 <= 1e-12, e2
    assert oracle.resid(V, Q, R) <= 1e-13
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    Qo, Ro = oracle.rand_cholqr(V, s1, s2, seed=0, S2=S2)
    tq, tr = parity_tolerance(V, s1, s2)
    assert np.abs(Q - Qo).max() <= tq
    assert np.abs(R - Ro).max() / np.abs(Ro).max() <= tr


def test_blocked_cholqr2_last_pass(rq):
    # CholeskyQR2's well-conditioned last pass at n = 128 runs the blocked product
    m, n = 30000, 128
    V = synthetic.make_v(m, n, 1e4, seed=3)
    Q, R, _ = rq.randqr_cholqr2(torch.from_numpy(V).cuda())
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    assert oracle.orth_err(Q)[0] <= 1e-13 and oracle.resid(V, Q, R) <= 1e-14
    Qo, Ro = oracle.cholqr2(V)
    assert np.abs(R - Ro).max() / np.abs(Ro).max() <= 1e-11


DF_CASES = [(20000, 16, 1e10), (3001, 1, 1.0), (5003, 3, 1e6), (6000, 7, 1e14), (10000, 32, 1e4),
            (12001, 33, 1e8), (20000, 64, 1e12), (20000, 64, 1e14), (16385, 100, 1e8),
            (20000, 128, 1e14)]


@pytest.mark.parametrize("m,n,kappa", DF_CASES)
def test_rand_cholqr_f32x2_parity(rq, m, n, kappa):
    """Row passes in pair arithmetic (~2^-47 unit roundoff): the same orthogonality and
    residual targets as FP64; Q and R against the FP64 oracle within the oracle's spread
    scaled by the ratio of unit roundoffs (2^6)."""
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = synthetic.make_v(m, n, kappa, seed=m % 89)
    S2 = oracle.gauss_sketch(1, s2, s1)
    Q, R, info = _run(rq, V, s1, s2, 0, S2, prec=rq.F32X2)
    e2, _ = oracle.orth_err(Q)
    res = oracle.resid(V, Q, R)
    assert e2 <= 1e-12, e2
    assert res <= 1e-13, res
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    Qo, Ro = oracle.rand_cholqr(V, s1, s2, seed=0, S2=S2)
    tq, tr = parity_tolerance(V, s1, s2)
    assert np.abs(Q - Qo).max() <= 64 * tq
    assert np.abs(R - Ro).max() / np.abs(Ro).max() <= 64 * tr


def test_f32x2_in_place_and_ld(rq):
    m, n = 9999, 40
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = synthetic.make_v(m, n, 1e11, seed=3)
    S2 = oracle.gauss_sketch(1, s2, s1)
    Q, R, _ = _run(rq, V, s1, s2, 0, S2, ld_pad=3, inplace=True, prec=rq.F32X2)
    assert oracle.orth_err(Q)[0] <= 1e-12 and oracle.resid(V, Q, R) <= 1e-13


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("m,n,kappa", [(20000, 16, 1e10), (30001, 64, 1e13), (9000, 100, 1e6),
                                       (5000, 128, 1e14)])
def test_tensor_core_gram_matches_cuda_core_gram(rq, prec, m, n, kappa):
    """The Gram from exact split products on the tensor cores and the CUDA-core Gram give
    factorizations that both meet the targets and agree within the parity tolerance."""
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = synthetic.make_v(m, n, kappa, seed=n)
    Vd = torch.from_numpy(V).cuda()
    out = []
    for tc in (True, False):
        ctx = rq.Context(0)
        ctx.set_tensor_cores(tc)
        Q, R, _ = rq.randqr_factor(Vd, s1, s2, seed=1, prec=prec, ctx=ctx)
        Q, R = Q.cpu().numpy(), R.cpu().numpy()
        assert oracle.orth_err(Q)[0] <= 1e-12 and oracle.resid(V, Q, R) <= 1e-13
        out.append((Q, R))
        ctx.close()
    tq, tr = parity_tolerance(V, s1, s2)
    scale = 64 if prec else 1
    assert np.abs(out[0][0] - out[1][0]).max() <= scale * tq
    assert np.abs(out[0][1] - out[1][1]).max() / np.abs(out[0][1]).max() <= scale * tr


def test_tensor_core_gram_cholqr2_exact_on_orthonormal_columns(rq):
    # V with orthonormal columns scaled by powers of two: V^T V is diagonal and exactly known
    m, n = 40000, 48
    U = np.linalg.qr(synthetic.rng(3).standard_normal((m, n)))[0]
    Q, R, _ = rq.randqr_cholqr2(torch.from_numpy(U).cuda())
    R = R.cpu().numpy()
    np.testing.assert_allclose(np.abs(np.diag(R)), 1.0, rtol=1e-14)
    assert np.abs(np.triu(R, 1)).max() < 1e-14


def test_single_countsketch_kind(rq):
    # S2 = I: rand_cholQR with the CountSketch alone, against the oracle on an explicit identity
    m, n = 20000, 16
    s1, _ = synthetic.paper_single_sketch_sizes(n)
    V = synthetic.make_v(m, n, 1e6, seed=3)  # kappa <= 1e8: the 1e-10 parity bar applies
    ctx = rq.Context(0)
    ctx.set_sketch_kind(rq.SKETCH_COUNT_ONLY)
    Q, R, _ = rq.randqr_factor(torch.from_numpy(V).cuda(), s1, s1, seed=4, ctx=ctx)
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    e2, _ = oracle.orth_err(Q)
    assert e2 <= 1e-12 and oracle.resid(V, Q, R) <= 1e-13
    Qo, Ro = oracle.rand_cholqr(V, s1, s1, seed=4, S2=np.eye(s1))
    assert np.abs(Q - Qo).max() <= 1e-10
    assert np.abs(R - Ro).max() / np.abs(Ro).max() <= 1e-10
    with pytest.raises(rq.RandQRError):  # s2 != s1
        rq.randqr_factor(torch.from_numpy(V).cuda(), s1, 64, seed=4, ctx=ctx)


def test_single_gaussian_kind(rq):
    # S1 = I: the Gaussian sketch of V itself, against the oracle's steps (Algorithm 3 with
    # Ws = S2 V)
    m, n = 5000, 16
    _, s2 = synthetic.paper_single_sketch_sizes(n)
    V = synthetic.make_v(m, n, 1e6, seed=6)  # kappa <= 1e8: the 1e-10 parity bar applies
    S2 = oracle.gauss_sketch(2, s2, m)
    ctx = rq.Context(0)
    ctx.set_sketch_kind(rq.SKETCH_GAUSSIAN_ONLY)
    buf = torch.zeros((m, n + 3), dtype=torch.float64, device="cuda")
    buf[:, :n] = torch.from_numpy(V).cuda()  # ld != n: packed internally
    Q, R, _ = rq.randqr_factor(buf[:, :n], m, s2, seed=0, S2=torch.from_numpy(S2).cuda(), ctx=ctx)
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    e2, _ = oracle.orth_err(Q)
    assert e2 <= 1e-12 and oracle.resid(V, Q, R) <= 1e-13
    Rs = oracle.hhqr_r(oracle.gemm(S2, V))
    W = oracle.trsm(V, Rs)
    Rc = oracle.chol(oracle.gram(W))
    Qo, Ro = oracle.trsm(W, Rc), oracle.trmm(Rc, Rs)
    assert np.abs(Q - Qo).max() <= 1e-10
    assert np.abs(R - Ro).max() / np.abs(Ro).max() <= 1e-10
    with pytest.raises(rq.RandQRError):  # s1 != m
        rq.randqr_factor(torch.from_numpy(V).cuda(), 544, s2, seed=0, ctx=ctx)


def test_tensor_core_gram_rows_of_changing_magnitude(rq):
    # 64-row blocks scaled by 1, 2^3, 2^6, 2^9, 2^12, 1, ...: later groups of an event outgrow the
    # event's column scales (cut again with their own) or fall far below them; both Gram paths
    # and the oracle agree
    m, n = 50000, 32
    V = synthetic.make_v(m, n, 10.0, seed=11)
    V *= np.ldexp(1.0, 3 * ((np.arange(m) // 64) % 5))[:, None]
    Vd = torch.from_numpy(V).cuda()
    Qo, Ro = oracle.cholqr2(V)
    for tc in (True, False):
        ctx = rq.Context(0)
        ctx.set_tensor_cores(tc)
        Q, R, _ = rq.randqr_cholqr2(Vd, ctx=ctx)
        Q, R = Q.cpu().numpy(), R.cpu().numpy()
        assert oracle.orth_err(Q)[0] <= 1e-12 and oracle.resid(V, Q, R) <= 1e-13
        assert np.abs(R - Ro).max() / np.abs(Ro).max() <= 1e-10  # kappa(V) ~ 1e4: u kappa ~ 1e-12
        Q, R, _ = rq.randqr_factor(Vd, seed=2, ctx=ctx)
        Q, R = Q.cpu().numpy(), R.cpu().numpy()
        assert oracle.orth_err(Q)[0] <= 1e-12 and oracle.resid(V, Q, R) <= 1e-13
        assert np.abs(R - Ro).max() / np.abs(Ro).max() <= 1e-10
        ctx.close()


@pytest.mark.parametrize("m,n", [(20001, 66), (33333, 100), (40000, 128), (5000, 128), (30001, 1), (20011, 7),
                                 (25000, 16), (33333, 17), (40000, 32), (9999, 33), (40001, 64)])
def test_gram_against_the_oracle(rq, m, n):
    """The split-product Gram at every width: n <= 16, <= 32 and <= 64 by the 16-, 32- and
    64-column instances of the Gram kernel, 64 < n <= 128 by the 64-column instance on the first
    64 columns and the cross-block kernel for the rest against all n, read back through the shard
    stage that returns it:
    against the oracle's Gram of the same W (the split format's error is a few units of 2^-53
    of the columns' scales; the bound allows for the oracle's own sequential sums), on rows whose magnitude jumps every 64 rows so that events
    restart and groups are cut again with their own scales."""
    V = synthetic.make_v(m, n, 1e3, seed=n)
    V *= np.ldexp(1.0, 5 * ((np.arange(m) // 64) % 4))[:, None]
    Vd = torch.from_numpy(V).cuda()
    s1, s2 = synthetic.default_sketch_sizes(n)
    Rs, _ = rq.randqr_sketch_r(rq.randqr_sketch(Vd, s1, s2, seed=1))
    W, G = rq.randqr_shard_gram(Vd, Rs)
    Wh, Gh = W.cpu().numpy(), G.cpu().numpy()
    Go = oracle.gram(Wh)
    scale = np.sqrt(np.outer(np.diag(Go), np.diag(Go)))
    assert np.abs(Gh - Go).max() / scale.max() <= 1e-12
    assert np.allclose(Gh, Gh.T, rtol=0, atol=0)  # both triangles from the packed upper one
