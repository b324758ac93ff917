"""Helpers shared by the GPU parity tests (tolerances and reference spreads)."""
import numpy as np

import oracle

U = 2.0 ** -53


def oracle_spread(V, s1, s2, seeds=(0, 1)):
    """Intrinsic floor of the Q/R comparison: two runs of the oracle that differ only in
    the random sketch are both correct rand_cholQR results; how far apart they land is
    the sensitivity of the unique QR factor of V to rounding (about kappa(V) u)."""
    a = oracle.rand_cholqr(V, s1, s2, seed=seeds[0])
    b = oracle.rand_cholqr(V, s1, s2, seed=seeds[1])
    dq = np.abs(a[0] - b[0]).max()
    dr = np.abs(a[1] - b[1]).max() / np.abs(a[1]).max()
    return dq, dr


def parity_tolerance(V, s1, s2):
    """max(1e-10, 10 x the oracle's own spread) for Q (absolute) and R (relative to
    max|R|): the stated 1e-10 wherever the problem is conditioned to allow it."""
    dq, dr = oracle_spread(V, s1, s2)
    return max(1e-10, 10 * dq), max(1e-10, 10 * dr)
