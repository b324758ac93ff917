"""Guard zones around the caller's buffers (the out-of-bounds check that stands in for a memory
sanitizer): a factorization writes Q (n of the ldq values of each row) and R (n of the ldr
values of each row) and nothing else, and reads V without writing it unless Q is V.

Each buffer sits inside a larger allocation filled with a bit pattern that no kernel produces
(a signalling-NaN payload); after the call the zones before and after the buffer, and the
padding columns past n in every row, must still hold it bit for bit.  The shapes cover every
solve path: one column, odd widths with odd leading dimensions (element stores), the
half-width and full-width split-product instances, the fused first pass, the blocked solves
above 64 columns and the substitution path of an odd width above 64, and the baselines."""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CANARY = 0x7FF4DEADBEEF1234  # a signalling NaN as FP64; positive as int64
ZONE = 4096  # elements before and after each buffer


@pytest.fixture(scope="module")
def rq():
    import paper_2309_05868_gb300 as rq
    return rq


class Guarded:
    """A rows x cols FP64 matrix with leading dimension ld inside a canary-filled allocation."""

    def __init__(self, rows, cols, ld, init=None):
        self.rows, self.cols, self.ld = rows, cols, ld
        self.raw = torch.full((ZONE + rows * ld + ZONE,), CANARY, dtype=torch.int64, device="cuda")
        self.mat = self.raw[ZONE:ZONE + rows * ld].view(torch.float64).view(rows, ld)[:, :cols]
        if init is not None:
            self.mat.copy_(torch.from_numpy(init).cuda())

    def intact(self):
        torch.cuda.synchronize()
        raw = self.raw.cpu().numpy()
        body = raw[ZONE:ZONE + self.rows * self.ld].reshape(self.rows, self.ld)
        zones = np.concatenate([raw[:ZONE], raw[ZONE + self.rows * self.ld:], body[:, self.cols:].ravel()])
        return bool(np.all(zones == CANARY))


CASES = [  # m, n, ldv, ldq, ldr
    (3001, 1, 1, 3, 2), (20011, 7, 9, 8, 7), (40000, 16, 16, 17, 16), (30002, 32, 32, 32, 33),
    (30007, 33, 35, 34, 40), (50001, 64, 64, 64, 64), (50001, 64, 66, 67, 65), (20001, 100, 100, 102, 101),
    (20003, 97, 97, 97, 99), (20000, 128, 128, 130, 128),
]


@pytest.mark.parametrize("m,n,ldv,ldq,ldr", CASES)
def test_rand_cholqr_writes_only_its_outputs(rq, m, n, ldv, ldq, ldr):
    V0 = synthetic.make_v(m, n, 1e8, seed=n)
    V, Q, R = Guarded(m, n, ldv, V0), Guarded(m, n, ldq), Guarded(n, n, ldr)
    before = V.raw.clone()
    rq.randqr_factor(V.mat, Q=Q.mat, R=R.mat)
    assert Q.intact() and R.intact()
    assert torch.equal(V.raw, before)  # V read only
    Qh, Rh = Q.mat.cpu().numpy(), R.mat.cpu().numpy()
    assert oracle.orth_err(Qh)[0] <= 1e-12 and oracle.resid(V0, Qh, Rh) <= 1e-13


@pytest.mark.parametrize("fused", [False, True])
def test_in_place_and_fused_write_only_their_outputs(rq, fused):
    m, n = 70001, 64
    V0 = synthetic.make_v(m, n, 1e12, seed=2)
    V, R = Guarded(m, n, n, V0), Guarded(n, n, n)
    ctx = rq.Context(0)
    ctx.set_fused_first_pass(fused)
    rq.randqr_factor(V.mat, Q=V.mat, R=R.mat, ctx=ctx)  # Q overwrites V
    assert V.intact() and R.intact()
    Qh, Rh = V.mat.cpu().numpy(), R.mat.cpu().numpy()
    assert oracle.orth_err(Qh)[0] <= 1e-12 and oracle.resid(V0, Qh, Rh) <= 1e-13
    W, G = Guarded(m, n, n), Guarded(n, n, n)
    Vs = Guarded(m, n, n, V0)
    Rs, _ = rq.randqr_sketch_r(rq.randqr_sketch(Vs.mat, 8320, 256, seed=1, ctx=ctx), ctx=ctx)
    rq.randqr_shard_gram(Vs.mat, Rs, Q=W.mat, G=G.mat, ctx=ctx)
    assert W.intact() and G.intact()
    ctx.close()


@pytest.mark.parametrize("algo", ["randqr", "cholqr2", "scholqr3", "f32x2"])
def test_other_entry_points_write_only_their_outputs(rq, algo):
    m, n, ldv, ldq, ldr = 30001, 48, 50, 49, 51
    V0 = synthetic.make_v(m, n, 1e6, seed=9)
    V, Q, R = Guarded(m, n, ldv, V0), Guarded(m, n, ldq), Guarded(n, n, ldr)
    if algo == "randqr":
        rq.randqr_randqr(V.mat, Q=Q.mat, R=R.mat)
    elif algo == "cholqr2":
        rq.randqr_cholqr2(V.mat, Q=Q.mat, R=R.mat)
    elif algo == "scholqr3":
        rq.randqr_shifted_cholqr3(V.mat, Q=Q.mat, R=R.mat)
    else:
        rq.randqr_factor(V.mat, Q=Q.mat, R=R.mat, prec=rq.F32X2)
    assert Q.intact() and R.intact()
    Qh, Rh = Q.mat.cpu().numpy(), R.mat.cpu().numpy()
    assert oracle.resid(V0, Qh, Rh) <= 1e-12
