"""The served stream of the measurement script as a test: 200 requests (m log-uniform in
[1e4, 4e6], n in {4, 8, 16, 32, 64}, kappa up to 1e12, each the leading rows of a pre-built
matrix) first one after another, then Poisson arrivals into 8 slots in FP64 and with the
pair-arithmetic row passes.  Every request must finish with status OK and orthonormal Q: this
mix, with up to eight factorizations overlapping on the device, caught a failure that the
smaller serving tests did not."""
import pytest

import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_bench_served_stream_completes():
    import bench
    import paper_2309_05868_gb300 as rq
    r = bench.serve_bench(rq, synthetic, torch, torch.device("cuda", 0), n_req=200, loads=(0.8,))
    for mode in ("served_fp64", "served_mixed"):
        assert r[mode]["max_orth_err_2"] <= 1e-12, (mode, r[mode])
    assert r["requests"] == 200
