"""Each result states its own accuracy (randqr_info.want_accuracy): ||I - Q^T Q||_2 and
||V - QR||_F / ||V||_F measured on the device after the factorization, checked against the
same measures computed on the host from the returned Q and R (numpy's blocked products and
symmetric eigensolver: the reference numbers carry rounding of a few units of sqrt(m) u, so
the comparison allows that much), and the same for a power-of-two multiple of V."""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

U = 2.0 ** -53


@pytest.fixture(scope="module")
def rq():
    import paper_2309_05868_gb300 as rq
    return rq


def _host_measures(V, Q, R):
    n = Q.shape[1]
    e2 = np.abs(np.linalg.eigvalsh(Q.T @ Q - np.eye(n))).max()
    res = np.linalg.norm(V - Q @ R) / np.linalg.norm(V)
    return e2, res


def _close(a, b, m):
    return abs(a - b) <= 0.5 * max(a, b) + 8 * np.sqrt(m) * U


@pytest.mark.parametrize("m,n,kappa,tc", [(20000, 16, 1e10, True), (30000, 64, 1e12, True),
                                          (20000, 100, 1e8, True), (20000, 16, 1e10, False),
                                          (5000, 3, 1e6, True)])
def test_factor_states_its_accuracy(rq, m, n, kappa, tc):
    V = synthetic.make_v(m, n, kappa, seed=n)
    Vd = torch.from_numpy(V).cuda()
    ctx = rq.Context(0)
    ctx.set_tensor_cores(tc)
    Q, R, info = rq.randqr_factor(Vd, seed=2, ctx=ctx, accuracy=True)
    Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
    e2, res = _host_measures(V, Qh, Rh)
    assert 0 <= info.orth_err2 <= 1e-12 and 0 <= info.resid_relF <= 1e-13
    assert _close(info.orth_err2, e2, m), (info.orth_err2, e2)
    assert _close(info.resid_relF, res, m), (info.resid_relF, res)
    # a power-of-two multiple of V: the relative measures come out the same (up to the order
    # of the sketch's FP64 atomics)
    _, _, info2 = rq.randqr_factor(Vd * 8.0, seed=2, ctx=ctx, accuracy=True)
    assert _close(info2.orth_err2, info.orth_err2, m) and _close(info2.resid_relF, info.resid_relF, m)
    # without the request the fields stay unmeasured
    _, _, info3 = rq.randqr_factor(Vd, seed=2, ctx=ctx)
    assert info3.orth_err2 == -1.0 and info3.resid_relF == -1.0
    ctx.close()


def test_in_place_states_orthogonality_only(rq):
    m, n = 20000, 32
    V = synthetic.make_v(m, n, 1e6, seed=1)
    Vd = torch.from_numpy(V).cuda()
    Q, R, info = rq.randqr_factor(Vd, seed=0, Q=Vd, accuracy=True)
    assert info.resid_relF == -1.0
    e2, _ = _host_measures(V, Q.cpu().numpy(), R.cpu().numpy())
    assert _close(info.orth_err2, e2, m)


@pytest.mark.parametrize("algo", ["cholqr2", "scholqr3"])
def test_baselines_state_their_accuracy(rq, algo):
    m, n = 20000, 32
    V = synthetic.make_v(m, n, 1e5, seed=2)
    fn = rq.randqr_cholqr2 if algo == "cholqr2" else rq.randqr_shifted_cholqr3
    Q, R, info = fn(torch.from_numpy(V).cuda(), accuracy=True)
    e2, res = _host_measures(V, Q.cpu().numpy(), R.cpu().numpy())
    assert _close(info.orth_err2, e2, m) and _close(info.resid_relF, res, m)


def test_served_request_states_its_accuracy(rq):
    m, n = 50000, 48
    V = synthetic.make_v(m, n, 1e9, seed=5)
    Vd = torch.from_numpy(V).cuda()
    ctx = rq.Context(0)
    t, (_, Q, R) = rq.randqr_submit(ctx, Vd, seed=3, accuracy=True)
    t2, _ = rq.randqr_submit(ctx, Vd, seed=3)
    st, info = rq.randqr_wait(ctx, t)
    assert st == 0
    e2, res = _host_measures(V, Q.cpu().numpy(), R.cpu().numpy())
    assert _close(info.orth_err2, e2, m) and _close(info.resid_relF, res, m)
    st, info2 = rq.randqr_wait(ctx, t2)
    assert st == 0 and info2.orth_err2 == -1.0
    ctx.close()


def test_host_entry_point_states_orthogonality(rq):
    m, n = 30000, 24
    V = synthetic.make_v(m, n, 1e7, seed=6)
    Vh = torch.from_numpy(V).pin_memory()
    Q, R, info = rq.randqr_factor_host(Vh, seed=1, accuracy=True)
    assert info.resid_relF == -1.0  # factored in place in the staging area
    e2, _ = _host_measures(V, Q.numpy(), R.numpy())
    assert _close(info.orth_err2, e2, m)
    assert oracle.resid(V, Q.numpy(), R.numpy()) <= 1e-13
