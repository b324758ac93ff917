"""Row-sharded rand_cholQR (Sec. 4.1, the distributed form of the sketch).

V (M x n) is split by rows; shard k holds V_k = V[row0_k : row0_k + m_k].  Everything the
method does to V is either row-local (the CountSketch scatter, W = V R_s^{-1}, Q = W R_c^{-1})
or a sum over rows (S2 S1 V and W^T W), and the CountSketch hash is a function of the global
row index, so

    Ws = sum_k S2 S1_k V_k        (s2 x n)
    G  = sum_k W_k^T W_k          (n x n)

and the method needs exactly two cross-shard sums of small buffers.  The Householder QR of
Ws and the Cholesky of G are replicated: every shard computes the same R_s and R_c.

The four stages run in the library's kernels (``DeviceStages``); the sums are the caller's
(``torch.distributed.all_reduce`` across ranks, or a fixed-order sum of logical shards held
by one process).  The stage object is pluggable so that the orchestration itself can be
exercised with other implementations of the stages.
"""
from . import (default_sketch_sizes, randqr_shard_finish, randqr_shard_gram, randqr_shard_sketch,
               randqr_sketch_r)

__all__ = ["DeviceStages", "factor_row_sharded", "factor_logical_shards", "dist_allreduce",
           "even_cuts"]


class DeviceStages:
    """The stages through the C ABI, on one context and stream.  ``gram`` writes W_k into the
    Q it is given and ``finish`` overwrites that Q in place.  With sync=False the R_s and
    finish stages only enqueue work (no host wait inside a factorization); their status is
    then read afterwards with ``get_status``."""

    def __init__(self, ctx=None, stream=None, sync=True):
        self.ctx = ctx
        self.stream = stream
        self.sync = sync

    def sketch(self, V, row0, s1, s2, seed, S2):
        return randqr_shard_sketch(V, row0, s1, s2, seed=seed, S2=S2, ctx=self.ctx,
                                   stream=self.stream)

    def sketch_r(self, Ws):
        return randqr_sketch_r(Ws, ctx=self.ctx, stream=self.stream, sync=self.sync)[0]

    def gram(self, V, Rs, Q):
        return randqr_shard_gram(V, Rs, Q=Q, ctx=self.ctx, stream=self.stream)

    def finish(self, Q, G, Rs):
        Q, R, _ = randqr_shard_finish(Q, G, Rs, ctx=self.ctx, stream=self.stream, sync=self.sync)
        return Q, R


def dist_allreduce(group=None):
    """In-place sum over the ranks of ``group`` (torch.distributed, any backend)."""
    import torch.distributed as dist

    def allreduce(t):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)

    return allreduce


def factor_row_sharded(V, row0, allreduce, s1=None, s2=None, seed=0, S2=None, Q=None,
                       stages=None):
    """rand_cholQR of the global matrix of which V is the row block starting at global row
    ``row0``.  ``allreduce(t)`` sums t in place over all shards.  Returns (Q_k, R): this
    shard's rows of Q and the (replicated) n x n R."""
    n = V.shape[1]
    d1, d2 = default_sketch_sizes(n)
    s1 = d1 if s1 is None else s1
    s2 = d2 if s2 is None else s2
    st = stages if stages is not None else DeviceStages()
    Ws = st.sketch(V, row0, s1, s2, seed, S2)
    allreduce(Ws)
    Rs = st.sketch_r(Ws)
    Q, G = st.gram(V, Rs, Q)
    allreduce(G)
    return st.finish(Q, G, Rs)


def even_cuts(m, shards):
    """Row boundaries of ``shards`` near-equal blocks of m rows (first blocks one longer)."""
    base, extra = divmod(m, shards)
    cuts = [0]
    for k in range(shards):
        cuts.append(cuts[-1] + base + (1 if k < extra else 0))
    return cuts


def factor_logical_shards(V, cuts, s1=None, s2=None, seed=0, S2=None, Q=None, stages=None):
    """The sharded decomposition on one process: shards V[cuts[k]:cuts[k+1]], their partial
    sketches and Grams summed in shard order (what an allreduce over ranks would give, up to
    its summation order).  Q may be V (in place).  Returns (Q, R)."""
    import torch
    n = V.shape[1]
    d1, d2 = default_sketch_sizes(n)
    s1 = d1 if s1 is None else s1
    s2 = d2 if s2 is None else s2
    st = stages if stages is not None else DeviceStages()
    if Q is None:
        Q = torch.empty_like(V)
    blocks = [(r0, r1) for r0, r1 in zip(cuts[:-1], cuts[1:]) if r1 > r0]
    Ws = None
    for r0, r1 in blocks:
        Wk = st.sketch(V[r0:r1], r0, s1, s2, seed, S2)
        Ws = Wk if Ws is None else Ws + Wk
    Rs = st.sketch_r(Ws)
    G = None
    for r0, r1 in blocks:
        _, Gk = st.gram(V[r0:r1], Rs, Q[r0:r1])
        G = Gk if G is None else G + Gk
    R = None
    for r0, r1 in blocks:
        _, Rk = st.finish(Q[r0:r1], G, Rs)
        R = Rk if R is None else R
    return Q, R
