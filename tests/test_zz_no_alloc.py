"""The allocation-free sketch entry point (randqr_sketch_static).

Some callers cannot allocate device memory where they need a sketch (a framework that owns
every allocation through its own pool, a host callback, a latency-critical path where an
allocation's implicit synchronisation is not allowed).  randqr_sketch_static serves them:
no context, no cudaMalloc, scratch in a fixed device array.  This file checks, through the
C ABI, that two calls in a row give the same Ws as the context-based randqr_sketch (bit for
bit on integer-valued V, within the sketch's FP64 product bound otherwise), and that sizes
beyond the scratch limit are refused.  It is collected last on purpose."""
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


def test_static_sketch_matches_context_sketch_twice(rq):
    m, n = 40_000, 64
    s1, s2 = synthetic.default_sketch_sizes(n)  # s1 * n = 532,480 <= 2^20
    S2 = torch.from_numpy(oracle.gauss_sketch(5, s2, s1)).cuda()
    # integer-valued V and S2 = I: Ws = W1 = S1 V, every sum exact whatever the order of
    # the atomics, so both entry points must agree bit for bit
    Vi = torch.from_numpy(synthetic.integer_matrix(m, n, seed=3)).cuda()
    eye = torch.eye(s1, dtype=torch.float64, device="cuda")
    ref = rq.randqr_sketch(Vi, s1, s1, seed=9, S2=eye)
    for _ in range(2):  # the second call must not see the first call's W1
        Ws = torch.full((s1, n), float("nan"), dtype=torch.float64, device="cuda")
        rq.randqr_sketch_static(Vi, s1, s1, eye, Ws, seed=9)
        torch.cuda.synchronize()
        assert torch.equal(Ws, ref)
    del eye
    # a general matrix: within the FP64 product bound of the sketch
    V = synthetic.make_v(m, n, 1e8, seed=4)
    Vd = torch.from_numpy(V).cuda()
    ref = rq.randqr_sketch(Vd, s1, s2, seed=2, S2=S2).cpu().numpy()
    S2h = S2.cpu().numpy()
    b, _ = oracle.cs_hash(2, m, s1)
    absW1 = np.zeros((s1, n))
    np.add.at(absW1, b, np.abs(V))
    bound = 2 * (s1 + m / s1 + 8) * 2.0**-53 * (np.abs(S2h) @ absW1)
    for _ in range(2):
        Ws = torch.empty((s2, n), dtype=torch.float64, device="cuda")
        rq.randqr_sketch_static(Vd, s1, s2, S2, Ws, seed=2)
        assert (np.abs(Ws.cpu().numpy() - ref) <= bound).all()


def test_static_sketch_rejects_oversize_and_missing_s2(rq):
    n = 128
    s1, s2 = synthetic.default_sketch_sizes(n)  # s1 * n = 4,227,072 > 2^20
    V = torch.zeros((1000, n), dtype=torch.float64, device="cuda")
    S2 = torch.zeros((s2, s1), dtype=torch.float64, device="cuda")
    Ws = torch.zeros((s2, n), dtype=torch.float64, device="cuda")
    with pytest.raises(rq.RandQRError) as e:
        rq.randqr_sketch_static(V, s1, s2, S2, Ws)
    assert e.value.name == "ERR_ARG"
    L = rq._load()
    import ctypes
    st = L.randqr_sketch_static(ctypes.c_void_p(V.data_ptr()), 1000, 8, n, 144, 32, 0, None,
                                ctypes.c_void_p(Ws.data_ptr()), None)
    assert st == -1


def test_static_sketch_allocates_nothing(rq):
    # after a first call (which looks up the array's device address once), further calls
    # leave the device's free memory exactly as it was
    m, n = 20_000, 32
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = torch.from_numpy(synthetic.make_v(m, n, 1e4, seed=8)).cuda()
    S2 = torch.from_numpy(oracle.gauss_sketch(2, s2, s1)).cuda()
    Ws = torch.empty((s2, n), dtype=torch.float64, device="cuda")
    rq.randqr_sketch_static(V, s1, s2, S2, Ws, seed=1)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        rq.randqr_sketch_static(V, s1, s2, S2, Ws, seed=1)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_sketch_reports_its_status(rq):
    # the status word of the fixed scratch comes back through randqr_sketch_static_status:
    # OK normally, RANDQR_ERR_TIMEOUT when the sketch kernel's bounded wait gives up (a wait
    # bound of 0 polls makes it give up at once); the next call clears it
    m, n = 20_000, 64
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = torch.from_numpy(synthetic.make_v(m, n, 1e4, seed=9)).cuda()
    S2 = torch.from_numpy(oracle.gauss_sketch(3, s2, s1)).cuda()
    ref = rq.randqr_sketch(V, s1, s2, seed=4, S2=S2)
    Ws = torch.empty((s2, n), dtype=torch.float64, device="cuda")
    rq.randqr_sketch_static(V, s1, s2, S2, Ws, seed=4)
    st, _ = rq.randqr_sketch_static_status()
    assert st == 0
    try:
        rq.randqr_set_wait_limit(None, 0)
        rq.randqr_sketch_static(V, s1, s2, S2, Ws, seed=4)
        st, _ = rq.randqr_sketch_static_status()
        assert st == -7
    finally:
        rq.randqr_set_wait_limit(None, -1)
    rq.randqr_sketch_static(V, s1, s2, S2, Ws, seed=4)
    st, _ = rq.randqr_sketch_static_status()
    assert st == 0
    assert torch.allclose(Ws, ref, rtol=0, atol=1e-12 * ref.abs().max().item())
