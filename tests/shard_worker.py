"""Stages of the row-sharded rand_cholQR (Sec. 4.1) computed by the CPU oracle, and the rank
body of the multi-process test.  Test infrastructure: the orchestration under test is
``paper_2309_05868_gb300.sharded``; only the stages are swapped for the oracle's."""
import os

import numpy as np


class OracleStages:
    """Sec. 4.1 stages with the oracle's FP64 steps; arrays are torch CPU tensors (so that a
    torch.distributed allreduce can sum them) or numpy arrays."""

    def __init__(self, as_torch):
        self.as_torch = as_torch

    def _out(self, a):
        if self.as_torch:
            import torch
            return torch.from_numpy(np.ascontiguousarray(a))
        return a

    @staticmethod
    def _np(a):
        return a.numpy() if hasattr(a, "numpy") else a

    def sketch(self, V, row0, s1, s2, seed, S2):
        import oracle
        S2 = oracle.gauss_sketch(seed + 1, s2, s1) if S2 is None else self._np(S2)
        return self._out(oracle.gemm(S2, oracle.countsketch_rows(self._np(V), s1, seed, row0)))

    def sketch_r(self, Ws):
        import oracle
        return self._out(oracle.hhqr_r(self._np(Ws)))

    def gram(self, V, Rs, Q):
        import oracle
        W = oracle.trsm(self._np(V), self._np(Rs))
        Qn = self._np(Q)
        Qn[...] = W
        return Q, self._out(oracle.gram(W))

    def finish(self, Q, G, Rs):
        import oracle
        Rc = oracle.chol(self._np(G))
        Qn = self._np(Q)
        Qn[...] = oracle.trsm(Qn.copy(), Rc)
        return Q, self._out(oracle.trmm(Rc, self._np(Rs)))


def rank_main(rank, world, port, m, n, kappa, seed, cuts, out_dir):
    """One rank: its row block of the seeded V, the sharded driver over gloo, results to
    out_dir/rank{r}.npz."""
    import torch
    import torch.distributed as dist

    import synthetic
    from paper_2309_05868_gb300 import sharded

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        V = synthetic.make_v(m, n, kappa, seed=seed)
        r0, r1 = cuts[rank], cuts[rank + 1]
        Vk = torch.from_numpy(np.ascontiguousarray(V[r0:r1]))
        Qk = torch.empty_like(Vk)
        Qk, R = sharded.factor_row_sharded(Vk, r0, sharded.dist_allreduce(), seed=seed, Q=Qk,
                                           stages=OracleStages(as_torch=True))
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), Q=Qk.numpy(), R=R.numpy())
    finally:
        dist.destroy_process_group()
