"""Serving path (randqr_submit / randqr_poll): continuous batching over the context's slots.

Checked through the C ABI: every request of a mixed stream completes with the accuracy the
direct call has; a request's result is the same alone and inside a mix; admission keeps the
bytes in flight under the HBM budget and refuses requests that can never fit; a failing
request does not disturb the others; tickets retire once."""
import time

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


def _V(m, n, kappa, seed):
    return torch.from_numpy(synthetic.make_v(m, n, kappa, seed=seed)).cuda()


def _drain(rq, ctx, tickets, timeout=120.0):
    out, t0 = {}, time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t in out:
                continue
            st, info = rq.randqr_poll(ctx, t)
            if st != rq.PENDING:
                out[t] = (st, info)
        assert time.time() - t0 < timeout, "requests did not finish"
    return out


MIX = [  # m, n, kappa, algo, prec, max_orth_err
    (20000, 16, 1e10, 0, 0, 0.0), (5000, 4, 1e3, 0, 0, 0.0), (60000, 64, 1e12, 0, 0, 0.0),
    (30000, 32, 1e6, 1, 0, 0.0), (30000, 32, 1e9, 2, 0, 0.0), (12345, 8, 1e14, 0, 0, 0.0),
    (40000, 64, 1e8, 0, 1, 0.0), (25000, 16, 1e4, 0, 0, 1e-12), (7000, 128, 1e6, 0, 0, 0.0),
    (50000, 8, 1e2, 1, 0, 0.0), (20000, 33, 1e11, 0, 0, 1e-12), (9000, 5, 1.0, 2, 0, 0.0),
]


def test_mixed_stream_completes_accurately(rq):
    ctx = rq.Context(0)
    rq.randqr_serve_config(ctx, slots=4)
    subs = []
    for i, (m, n, kappa, algo, prec, tol) in enumerate(MIX):
        V = _V(m, n, kappa, seed=i)
        t, keep = rq.randqr_submit(ctx, V, algo=algo, prec=prec, seed=i, max_orth_err=tol)
        subs.append((t, keep))
    res = _drain(rq, ctx, [t for t, _ in subs])
    for (t, (V, Q, R)), (m, n, kappa, algo, prec, tol) in zip(subs, MIX):
        st, _ = res[t]
        assert st == 0, (m, n, kappa, algo, st)
        Vh, Qh, Rh = V.cpu().numpy(), Q.cpu().numpy(), R.cpu().numpy()
        assert oracle.orth_err(Qh)[0] <= 1e-12
        assert oracle.resid(Vh, Qh, Rh) <= 1e-13
    stats = rq.randqr_serve_stats_get(ctx)
    assert stats["completed"] == len(MIX) and stats["queued"] == 0 and stats["running"] == 0
    ctx.close()


def test_result_alone_equals_result_in_mix(rq):
    m, n, kappa = 30000, 24, 1e7
    s1, s2 = synthetic.default_sketch_sizes(n)
    Vh = synthetic.make_v(m, n, kappa, seed=42)
    V = torch.from_numpy(Vh).cuda()
    ctx = rq.Context(0)
    rq.randqr_serve_config(ctx, slots=6)
    t, (_, Qa, Ra) = rq.randqr_submit(ctx, V, seed=5)
    assert rq.randqr_wait(ctx, t)[0] == 0
    others = [rq.randqr_submit(ctx, _V(40000, nn, 1e9, seed=nn), seed=nn)
              for nn in (8, 16, 32, 64, 4, 48)]
    t2, (_, Qb, Rb) = rq.randqr_submit(ctx, V, seed=5)
    others += [rq.randqr_submit(ctx, _V(20000, nn, 1e3, seed=nn + 1), seed=nn)
               for nn in (12, 20, 64)]
    res = _drain(rq, ctx, [t2] + [o[0] for o in others])
    assert all(st == 0 for st, _ in res.values())
    tq, tr = parity_tolerance(Vh, s1, s2)
    Qa, Qb, Ra, Rb = Qa.cpu().numpy(), Qb.cpu().numpy(), Ra.cpu().numpy(), Rb.cpu().numpy()
    assert np.abs(Qa - Qb).max() <= tq
    assert np.abs(Ra - Rb).max() / np.abs(Ra).max() <= tr
    ctx.close()


def test_admission_respects_budget(rq):
    budget = 64 << 20
    ctx = rq.Context(0)
    rq.randqr_serve_config(ctx, slots=8, hbm_budget_bytes=budget)
    subs = [rq.randqr_submit(ctx, _V(150000, 8, 1e4, seed=i), seed=i) for i in range(10)]
    # each request holds ~19.2 MB (V, Q, R, workspace): at most 3 fit in 64 MiB
    peak, done = 0, {}
    t0 = time.time()
    while len(done) < len(subs):
        s = rq.randqr_serve_stats_get(ctx)
        peak = max(peak, s["bytes_in_flight"])
        assert s["running"] <= 3
        for t, _ in subs:
            if t not in done:
                st, _ = rq.randqr_poll(ctx, t)
                if st != rq.PENDING:
                    done[t] = st
        assert time.time() - t0 < 120
    assert all(st == 0 for st in done.values())
    assert 0 < peak <= budget
    big = torch.zeros((2_000_000, 8), dtype=torch.float64, device="cuda")  # 128 MB > budget
    with pytest.raises(rq.RandQRError) as e:
        rq.randqr_submit(ctx, big)
    assert e.value.name == "ERR_ADMISSION"
    ctx.close()


def test_failure_is_isolated_and_tickets_retire(rq):
    ctx = rq.Context(0)
    bad = _V(30000, 32, 1e13, seed=1)
    good = [_V(30000, 32, 1e3, seed=s) for s in range(3)]
    tb, _ = rq.randqr_submit(ctx, bad, algo=rq.ALGO_CHOLQR2)
    tg = [rq.randqr_submit(ctx, g, seed=i)[0] for i, g in enumerate(good)]
    st, info = rq.randqr_wait(ctx, tb)
    if st != 0:
        assert st == -2 and info.info >= 1
    for t in tg:
        assert rq.randqr_wait(ctx, t)[0] == 0
    assert rq.randqr_poll(ctx, tg[0])[0] == -9  # retired
    assert rq.randqr_poll(ctx, 123456789)[0] == -9
    ctx.close()


def test_tensor_core_kernels_under_concurrent_load(rq):
    """Many large factorizations on eight slots at once (the row-pass kernels of different
    requests then share the GPU's SMs and memory bandwidth, which stretches load latencies
    inside each kernel's pipeline): every result matches the same call made alone on one
    stream (up to the order of the Gram's final FP64 atomics: well-conditioned V, so 1e-13)."""
    shapes = [(1 << 20, 64), (1 << 19, 4), (700001, 16), (1 << 20, 32), (300000, 64), (1 << 20, 8)]
    Vs = [torch.randn(m, n, dtype=torch.float64, device="cuda") / 1e3 for (m, n) in shapes]
    alone = []
    ctx1 = rq.Context(0)
    for i, V in enumerate(Vs):
        Q, R, _ = rq.randqr_factor(V, seed=i, ctx=ctx1)
        alone.append((Q.clone(), R.clone()))
    ctx1.close()
    ctx = rq.Context(0)
    rq.randqr_serve_config(ctx, slots=8)
    for rep in range(3):
        outs, subs = [], []
        for i, V in enumerate(Vs * 2):
            Q = torch.empty_like(V)
            R = torch.empty((V.shape[1], V.shape[1]), dtype=torch.float64, device="cuda")
            t, keep = rq.randqr_submit(ctx, V, Q=Q, R=R, seed=i % len(Vs))
            subs.append(t)
            outs.append((i % len(Vs), Q, R, keep))
        res = _drain(rq, ctx, subs)
        assert all(st == 0 for st, _ in res.values()), res
        for i, Q, R, _ in outs:
            dq = (Q - alone[i][0]).abs().max().item()
            dr = ((R - alone[i][1]).abs().max() / alone[i][1].abs().max()).item()
            assert dq <= 1e-13 and dr <= 1e-13, (rep, i, dq, dr)
    ctx.close()


def test_corrupted_descriptors_are_refused_while_others_run(rq):
    """Failure detection for the request path: descriptors with a bad field (unknown algorithm
    or precision, sizes or leading dimensions out of range, NULL or overlapping buffers, sketch
    sizes that do not fit, a nonzero reserved word) are refused at submit with RANDQR_ERR_ARG
    and queue nothing, a batch holding one of them queues none, and the requests already in
    flight finish correctly."""
    import ctypes
    ctx = rq.Context(0)
    good = [_V(200_000, 32, 1e6, seed=s) for s in range(4)]
    tickets = [rq.randqr_submit(ctx, g, seed=i)[0] for i, g in enumerate(good)]
    V = _V(20_000, 16, 1e3, seed=9)
    base, keep = rq.make_request(V)
    L = rq._serve_sigs(rq._load())

    def corrupt(**kw):
        r = rq.Request.from_buffer_copy(base)
        for k, v in kw.items():
            setattr(r, k, v)
        return r

    bad = [corrupt(algo=7), corrupt(algo=-1), corrupt(prec=5), corrupt(n=0), corrupt(n=129),
           corrupt(m=8), corrupt(ldv=8), corrupt(ldq=8), corrupt(ldr=8), corrupt(V=None),
           corrupt(Q=None), corrupt(R=None), corrupt(reserved=1),
           corrupt(R=base.V + 8 * 1000),                # R inside V
           corrupt(Q=base.V + 8 * 16, ldq=base.ldv),  # Q overlapping V without being V
           corrupt(Q=base.V, ldq=base.ldv + 2),       # in place with another leading dimension
           corrupt(s1=100, s2=200),                   # s1 < s2
           corrupt(s1=600, s2=8)]                     # s2 < n
    for r in bad:
        t = ctypes.c_uint64(0)
        assert L.randqr_submit(ctx.handle, ctypes.byref(r), ctypes.byref(t)) == -1
    arr = (rq.Request * 3)(base, bad[0], base)
    tk = (ctypes.c_uint64 * 3)()
    assert L.randqr_submit_batch(ctx.handle, arr, 3, tk) == -1
    assert rq.randqr_serve_stats_get(ctx)["submitted"] == len(tickets)
    for t, g in zip(tickets, good):
        st, _ = rq.randqr_wait(ctx, t)
        assert st == 0
    ctx.close()
    del keep


def test_slow_producer(rq):
    """A producer that submits with gaps (the server drains to empty at one point and new work
    arrives after it) and stalls for half a second mid-stream: every request completes once,
    with the direct call's accuracy, and the server's counters come back to nothing queued,
    running or in flight."""
    ctx = rq.Context(0)
    rq.randqr_serve_config(ctx, slots=4)
    rng = np.random.default_rng(7)
    shapes = [(int(rng.integers(5000, 60000)), int(rng.choice([4, 8, 16, 32, 64])), 10.0 ** rng.uniform(0, 12))
              for _ in range(24)]
    pending, finished, keep = set(), {}, {}

    def poll_all():
        for t in list(pending):
            st, _ = rq.randqr_poll(ctx, t)
            if st != rq.PENDING:
                finished[t] = st
                pending.discard(t)

    for i, (m, n, kappa) in enumerate(shapes):
        t, k = rq.randqr_submit(ctx, _V(m, n, kappa, seed=100 + i))
        pending.add(t)
        keep[t] = k
        if i == 6:  # let the server run dry before the next arrival
            t0 = time.time()
            while pending:
                poll_all()
                assert time.time() - t0 < 60.0
            s = rq.randqr_serve_stats_get(ctx)
            assert s["queued"] == 0 and s["running"] == 0 and s["bytes_in_flight"] == 0, s
        time.sleep(0.5 if i == 12 else float(rng.uniform(0.0, 0.02)))
        poll_all()
    t0 = time.time()
    while pending:
        poll_all()
        assert time.time() - t0 < 120.0, "requests did not finish"
    assert len(finished) == len(shapes) and all(st == 0 for st in finished.values()), finished
    s = rq.randqr_serve_stats_get(ctx)
    assert s["submitted"] == s["completed"] == len(shapes), s
    assert s["queued"] == 0 and s["running"] == 0 and s["bytes_in_flight"] == 0, s
    for t, (V, Q, R) in keep.items():
        Vh, Qh, Rh = V.cpu().numpy(), Q.cpu().numpy(), R.cpu().numpy()
        assert oracle.orth_err(Qh)[0] <= 1e-12
        assert oracle.resid(Vh, Qh, Rh) <= 1e-13
    ctx.close()


def test_served_requests_take_the_wait_bound(rq):
    """The server's slot contexts run under the serving context's wait bound: with 0 polls a
    served request gives up at its first wait and retires with RANDQR_ERR_TIMEOUT; with the
    default restored the next request on the same server completes."""
    ctx = rq.Context(0)
    rq.randqr_serve_config(ctx, slots=2)
    V = _V(30000, 64, 1e6, seed=5)
    ctx.set_wait_limit(0)
    t, _ = rq.randqr_submit(ctx, V)
    st, _ = rq.randqr_wait(ctx, t)
    assert st == -7, st
    ctx.set_wait_limit(-1)
    t, (Vk, Q, R) = rq.randqr_submit(ctx, V)
    st, _ = rq.randqr_wait(ctx, t)
    assert st == 0, st
    Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
    assert oracle.orth_err(Qh)[0] <= 1e-12 and oracle.resid(V.cpu().numpy(), Qh, Rh) <= 1e-13
    ctx.close()
