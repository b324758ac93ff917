"""rand_cholQR of a matrix in host memory (randqr_factor_host): the C ABI call uploads V into
the context's staging area, factors it there and downloads Q and R.  Checked against the
device-memory call on the same matrix, with padded leading dimensions, in place on the host,
with pageable host memory, asynchronously on a stream, and for its argument errors."""
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


def _orth(Q):
    Q = torch.as_tensor(Q, dtype=torch.float64)
    n = Q.shape[1]
    return torch.linalg.matrix_norm(Q.T @ Q - torch.eye(n, dtype=torch.float64), ord=2).item()


@pytest.mark.parametrize("m,n,kappa", [(20000, 16, 1e10), (100003, 64, 1e12), (30000, 100, 1e8)])
def test_host_call_matches_device_call(rq, m, n, kappa):
    V = synthetic.make_v(m, n, kappa, seed=m % 31)
    Vh = torch.from_numpy(V).pin_memory()
    Q, R, info = rq.randqr_factor_host(Vh, seed=3)
    assert Q.device.type == "cpu" and R.device.type == "cpu"
    assert _orth(Q) <= 1e-12
    assert oracle.resid(V, Q.numpy(), R.numpy()) <= 1e-13
    assert np.array_equal(R.numpy(), np.triu(R.numpy())) and (np.diag(R.numpy()) > 0).all()
    assert info.info == 0
    # against the device call: the same kernels on the same values, only the order of the
    # atomic sums differs, so at kappa = 1e3 the two agree to O(u kappa)
    V = synthetic.make_v(m, n, 1e3, seed=m % 29)
    Q, R, _ = rq.randqr_factor_host(torch.from_numpy(V).pin_memory(), seed=3)
    Qd, Rd, _ = rq.randqr_factor(torch.from_numpy(V).cuda(), seed=3)
    assert (Q - Qd.cpu()).abs().max().item() <= 1e-11
    assert ((R - Rd.cpu()).abs().max() / Rd.abs().max().cpu()).item() <= 1e-11


def test_host_call_padded_in_place_and_pageable(rq):
    m, n = 50001, 32
    V = synthetic.make_v(m, n, 1e3, seed=2)  # results of separate runs agree to O(u kappa)
    Qref, Rref, _ = rq.randqr_factor(torch.from_numpy(V).cuda(), seed=1)
    Qref, Rref = Qref.cpu(), Rref.cpu()
    # leading dimensions larger than n on every host matrix, pinned
    Vb = torch.zeros((m, n + 5), dtype=torch.float64).pin_memory()
    Vb[:, :n] = torch.from_numpy(V)
    Qb = torch.full((m, n + 3), 7.0, dtype=torch.float64).pin_memory()
    Rb = torch.full((n, n + 1), 7.0, dtype=torch.float64).pin_memory()
    rq.randqr_factor_host(Vb[:, :n], seed=1, Q=Qb[:, :n], R=Rb[:, :n])
    assert (Qb[:, :n] - Qref).abs().max().item() <= 1e-11
    assert (Qb[:, n:] == 7.0).all() and (Rb[:, n:] == 7.0).all()  # padding untouched
    assert ((Rb[:, :n] - Rref).abs().max() / Rref.abs().max()).item() <= 1e-11
    # in place on the host: Q = V
    Vi = torch.from_numpy(V.copy()).pin_memory()
    Q, R, _ = rq.randqr_factor_host(Vi, seed=1, Q=Vi)
    assert Q.data_ptr() == Vi.data_ptr()
    assert (Vi - Qref).abs().max().item() <= 1e-11
    # pageable host memory (copies block the host, same result)
    Vp = torch.from_numpy(V.copy())
    Qp = torch.empty_like(Vp)
    Rp = torch.empty((n, n), dtype=torch.float64)
    rq.randqr_factor_host(Vp, seed=1, Q=Qp, R=Rp)
    assert (Qp - Qref).abs().max().item() <= 1e-11


def test_host_calls_on_two_streams(rq):
    # two contexts on two streams, several calls each without waiting: the pipelined use
    m, n = 200000, 64
    Vs = [torch.from_numpy(synthetic.make_v(m, n, 1e3, seed=10 + k)).pin_memory() for k in range(2)]
    ctxs = [rq.Context(0) for _ in range(2)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    outs = []
    for rep in range(3):
        for b in range(2):
            Q = torch.empty((m, n), dtype=torch.float64).pin_memory()
            R = torch.empty((n, n), dtype=torch.float64).pin_memory()
            rq.randqr_factor_host(Vs[b], seed=rep, Q=Q, R=R, ctx=ctxs[b], stream=streams[b], sync=False)
            outs.append((b, rep, Q, R))
    torch.cuda.synchronize()
    for c, st in zip(ctxs, streams):
        assert rq.get_status(c, st)[0] == 0
    for b, rep, Q, R in outs:
        assert _orth(Q) <= 1e-12
        assert oracle.resid(Vs[b].numpy(), Q.numpy(), R.numpy()) <= 1e-13
        Qd, _, _ = rq.randqr_factor(Vs[b].cuda(), seed=rep)
        assert (Q - Qd.cpu()).abs().max().item() <= 1e-11


def test_host_call_argument_errors(rq):
    V = torch.zeros((100, 8), dtype=torch.float64)
    with pytest.raises(ValueError):
        rq.randqr_factor_host(V.cuda())  # device tensors go to randqr_factor
    with pytest.raises(rq.RandQRError) as e:
        rq.randqr_factor_host(V, s1=144, s2=4)  # s2 < n
    assert e.value.name == "ERR_ARG"
    buf = torch.zeros((100, 8), dtype=torch.float64)
    with pytest.raises(rq.RandQRError) as e:  # R inside V
        rq.randqr_factor_host(buf, R=buf[92:100])
    assert e.value.name == "ERR_ARG"
