"""The fused first row pass of rand_cholQR at n = 64 (Algorithm 3's W = V R_s^{-1} together with
the Gram G = W^T W of Algorithm 2 step 1): one launch on pairs of CTAs of a cluster, the solve in
one and the Gram of the stored rows in the other (randqr_set_fused_first_pass; off by default).  Checked against the oracle, against the two-pass
path on the same inputs (W is the same product row by row, so it must match bit for bit; G is
the same split-product Gram over a different row partition, so it matches to rounding), and on
row counts that leave a pair a single partial tile, a pair with no rows, a ragged tail, or many
tiles."""
import numpy as np
import pytest

import oracle
import synthetic
from gpu_util import parity_tolerance

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = 64


@pytest.fixture(scope="module")
def rq():
    import paper_2309_05868_gb300 as rq
    return rq


def _factor(rq, ctx, Vd, s1, s2, S2d, prec=0, Q=None):
    ctx.set_profiling(True)
    Q, R, _ = rq.randqr_factor(Vd, s1, s2, seed=0, S2=S2d, prec=prec, ctx=ctx, Q=Q)
    torch.cuda.synchronize()
    kt = ctx.kernel_times()
    ctx.set_profiling(False)
    return Q.cpu().numpy(), R.cpu().numpy(), kt


@pytest.mark.parametrize("m,kappa", [(256, 1e2), (300, 1e6), (20037, 1e12), (30000, 1e8), (131077, 1e14)])
def test_fused_first_pass_against_oracle_and_two_passes(rq, m, kappa):
    s1, s2 = synthetic.default_sketch_sizes(N)
    V = synthetic.make_v(m, N, kappa, seed=m % 89)
    S2 = oracle.gauss_sketch(1, s2, s1)
    Vd, S2d = torch.from_numpy(V).cuda(), torch.from_numpy(S2).cuda()
    ctx = rq.Context(0)
    ctx.set_fused_first_pass(True)
    Qf, Rf, kf = _factor(rq, ctx, Vd, s1, s2, S2d)
    # one fused launch, then only the second solve (no separate Gram pass)
    assert kf["solve_gram"][1] == 1 and kf["trsm_tc"][1] == 1 and "gram_tc" not in kf, kf
    ctx.set_fused_first_pass(False)
    Qu, Ru, ku = _factor(rq, ctx, Vd, s1, s2, S2d)
    assert "solve_gram" not in ku and ku["trsm_tc"][1] == 2 and ku["gram_tc"][1] == 1, ku
    ctx.close()
    Qo, Ro = oracle.rand_cholqr(V, s1, s2, seed=0, S2=S2)
    tq, tr = parity_tolerance(V, s1, s2)
    for Q, R in ((Qf, Rf), (Qu, Ru)):
        assert oracle.orth_err(Q)[0] <= 1e-12
        assert oracle.resid(V, Q, R) <= 1e-13
        assert np.abs(Q - Qo).max() <= tq
        assert np.abs(R - Ro).max() / np.abs(Ro).max() <= tr
    # the two paths differ only in the Gram's rounding (its row partition), which moves Q and R
    # by no more than the spread between two correct results
    assert np.abs(Rf - Ru).max() / np.abs(Ru).max() <= tr
    assert np.abs(Qf - Qu).max() <= tq


def test_fused_first_pass_f32x2_and_in_place(rq):
    m, kappa = 50001, 1e12
    s1, s2 = synthetic.default_sketch_sizes(N)
    V = synthetic.make_v(m, N, kappa, seed=5)
    S2 = oracle.gauss_sketch(1, s2, s1)
    S2d = torch.from_numpy(S2).cuda()
    ctx = rq.Context(0)
    ctx.set_fused_first_pass(True)
    Q, R, kt = _factor(rq, ctx, torch.from_numpy(V).cuda(), s1, s2, S2d, prec=1)
    assert kt["solve_gram"][1] == 1, kt
    assert oracle.orth_err(Q)[0] <= 1e-12 and oracle.resid(V, Q, R) <= 1e-12
    Vd = torch.from_numpy(V).cuda()
    Q2, R2, kt = _factor(rq, ctx, Vd, s1, s2, S2d, Q=Vd)  # Q overwrites V
    assert kt["solve_gram"][1] == 1, kt
    ctx.close()
    Qo, Ro = oracle.rand_cholqr(V, s1, s2, seed=0, S2=S2)
    tq, tr = parity_tolerance(V, s1, s2)
    assert np.abs(Q2 - Qo).max() <= tq
    assert np.abs(R2 - Ro).max() / np.abs(Ro).max() <= tr


@pytest.mark.parametrize("m", [40001, 1200007])
def test_fused_shard_gram_matches_two_passes(rq, m):
    """W and G of the shard stage, fused and not, on rows whose magnitude jumps every 64 rows
    (the Gram's events restart and its groups are cut again); at 1.2e6 rows every pair runs
    dozens of tiles, the Gram CTA trailing its solve CTA through the whole range."""
    V = synthetic.make_v(m, N, 1e6, seed=11)
    V *= np.ldexp(1.0, 5 * ((np.arange(m) // 64) % 4))[:, None]
    Vd = torch.from_numpy(V).cuda()
    s1, s2 = synthetic.default_sketch_sizes(N)
    ctx = rq.Context(0)
    Rs, _ = rq.randqr_sketch_r(rq.randqr_sketch(Vd, s1, s2, seed=1, ctx=ctx), ctx=ctx)
    ctx.set_fused_first_pass(True)
    ctx.set_profiling(True)
    Wf, Gf = rq.randqr_shard_gram(Vd, Rs, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.kernel_times()["solve_gram"][1] == 1
    ctx.set_fused_first_pass(False)
    Wu, Gu = rq.randqr_shard_gram(Vd, Rs, ctx=ctx)
    torch.cuda.synchronize()
    assert "solve_gram" not in ctx.kernel_times()
    ctx.close()
    assert torch.equal(Wf, Wu)  # the same product, row by row
    Gfh, Guh = Gf.cpu().numpy(), Gu.cpu().numpy()
    scale = np.sqrt(np.outer(np.diag(Guh), np.diag(Guh))).max()
    assert np.abs(Gfh - Guh).max() / scale <= 1e-14
    assert np.allclose(Gfh, Gfh.T, rtol=0, atol=0)
    if m <= 100000:
        Go = oracle.gram(Wf.cpu().numpy())
        assert np.abs(Gfh - Go).max() / scale <= 1e-12


def test_fused_pass_gives_up_on_its_waits_and_recovers(rq):
    """With a wait bound of 0 polls both roles give up at their first wait (the solver on its
    pipeline barriers, the Gram CTA on the solver's progress words), the shard stage reports
    RANDQR_ERR_TIMEOUT at once, and the same context then computes the right W and G."""
    import time
    m = 40000
    s1, s2 = synthetic.default_sketch_sizes(N)
    Vd = torch.from_numpy(synthetic.make_v(m, N, 1e8, seed=3)).cuda()
    good = rq.Context(0)
    Rs, _ = rq.randqr_sketch_r(rq.randqr_sketch(Vd, s1, s2, seed=1, ctx=good), ctx=good)
    ctx = rq.Context(0)
    ctx.set_fused_first_pass(True)
    ctx.set_wait_limit(0)
    t0 = time.time()
    rq.randqr_shard_gram(Vd, Rs, ctx=ctx)
    torch.cuda.synchronize()
    st, _ = rq.get_status(ctx)
    assert st == -7 and time.time() - t0 < 30.0
    ctx.set_wait_limit(-1)
    W, G = rq.randqr_shard_gram(Vd, Rs, ctx=ctx)
    Wg, Gg = rq.randqr_shard_gram(Vd, Rs, ctx=good)  # two passes
    torch.cuda.synchronize()
    assert rq.get_status(ctx)[0] == 0
    assert torch.equal(W, Wg)
    assert (G - Gg).abs().max().item() <= 1e-14 * Gg.abs().max().item()
    ctx.close()
    good.close()
