"""Failure detection on the device, without faulting the GPU.

Every wait inside the library's kernels is bounded; a context's wait bound can be set to 0
polls (randqr_set_wait_limit), after which any kernel that has to wait gives up at once,
records RANDQR_ERR_TIMEOUT in the status word, drains its own copies and products, frees its
tensor memory and returns.  These tests make exactly that happen in each kind of waiting
kernel and check that the status comes back, that the call ends quickly, and that the context
is usable afterwards."""
import time

import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rq():
    import paper_2309_05868_gb300 as rq
    return rq


def _expect_timeout(rq, fn):
    t0 = time.time()
    with pytest.raises(rq.RandQRError) as e:
        fn()
    torch.cuda.synchronize()
    assert e.value.name == "ERR_TIMEOUT", e.value.name
    assert time.time() - t0 < 30.0


def test_timeouts_in_each_waiting_kernel_and_recovery(rq):
    m, n = 40000, 64
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = synthetic.make_v(m, n, 1e8, seed=3)
    Vd = torch.from_numpy(V).cuda()
    ctx = rq.Context(0)
    good = rq.Context(0)
    Rs, _ = rq.randqr_sketch_r(rq.randqr_sketch(Vd, s1, s2, seed=1, ctx=good), ctx=good)
    ctx.set_wait_limit(0)
    # the split-product sketch GEMM (the first kernel of rand_cholQR that waits)
    _expect_timeout(rq, lambda: rq.randqr_factor(Vd, seed=1, ctx=ctx))
    # the cluster Householder QR of the sketch (flag waits across the cluster's CTAs)
    Ws = rq.randqr_sketch(Vd, s1, s2, seed=1, ctx=good)
    _expect_timeout(rq, lambda: rq.randqr_sketch_r(Ws, ctx=ctx))
    # the split-product triangular solve (mbarrier pipeline) through the shard stage
    rq.randqr_shard_gram(Vd, Rs, ctx=ctx)
    st, _ = rq.get_status(ctx)
    assert st == -7
    # the split-product Gram (first kernel of CholeskyQR2)
    _expect_timeout(rq, lambda: rq.randqr_cholqr2(Vd, ctx=ctx))
    # back to the default bound: the same context factors correctly
    ctx.set_wait_limit(-1)
    Q, R, _ = rq.randqr_factor(Vd, seed=1, ctx=ctx)
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    assert oracle.orth_err(Q)[0] <= 1e-12 and oracle.resid(V, Q, R) <= 1e-13
    Qg, Rg, _ = rq.randqr_factor(Vd, seed=1, ctx=good)
    # same kernels on the same input: equal up to the order of the FP64 atomics
    assert np.abs(Q - Qg.cpu().numpy()).max() <= 1e-8
    ctx.close()
    good.close()


def test_timeout_above_64_columns(rq):
    # 64 < n <= 128: the Gram of the first 64 columns is the first kernel to wait and gives up;
    # the cross-block Gram and the blocked solves after it return at once on the failed status
    m, n = 20000, 100
    Vd = torch.from_numpy(synthetic.make_v(m, n, 1e3, seed=4)).cuda()
    ctx = rq.Context(0)
    ctx.set_wait_limit(0)
    _expect_timeout(rq, lambda: rq.randqr_cholqr2(Vd, ctx=ctx))
    ctx.set_wait_limit(-1)
    Q, R, _ = rq.randqr_cholqr2(Vd, ctx=ctx)
    assert oracle.orth_err(Q.cpu().numpy())[0] <= 1e-13
    ctx.close()
