"""Comparison of the CUDA path's kNN output with the oracle's.

The bar: neighbour index lists identical to the oracle's (ties broken by the
lower index), except where the oracle's k-th and (k+1)-th distances agree to
within 1e-6 relative (a true near-tie at the boundary; then only the members
of that tie group may differ and must still lie in it), and distances within
1e-5 relative of the float64 distance (absolute floor 1e-30 for duplicates).
"""
import numpy as np

TIE_REL = 1e-6
DIST_REL = 1e-5


def compare(gpu_idx, gpu_dist, or_idx, or_d2, k):
    """gpu_idx / gpu_dist: (n, k); or_idx / or_d2: oracle lists with k or k+1
    columns.  Returns a dict of counts; raises AssertionError on a violation."""
    gpu_idx = np.asarray(gpu_idx)
    gpu_dist = np.asarray(gpu_dist, dtype=np.float64)
    od = np.sqrt(np.asarray(or_d2, dtype=np.float64))
    oi = np.asarray(or_idx)
    n = gpu_idx.shape[0]
    assert gpu_idx.shape == (n, k) and oi.shape[0] == n
    exact = np.all(gpu_idx == oi[:, :k], axis=1)
    exempt = 0
    for q in np.nonzero(~exact)[0]:
        if oi.shape[1] <= k:
            raise AssertionError(f"query {q}: {gpu_idx[q].tolist()} != {oi[q, :k].tolist()}")
        dk, dk1 = od[q, k - 1], od[q, k]
        if not (dk1 - dk <= TIE_REL * max(dk1, 1e-300)):
            raise AssertionError(f"query {q}: {gpu_idx[q].tolist()} != {oi[q, :k].tolist()} "
                                 f"(d_k={dk!r}, d_k+1={dk1!r})")
        lo = dk * (1 - TIE_REL)
        strict = od[q, :k] < lo
        assert set(gpu_idx[q][gpu_dist[q] < lo * (1 - DIST_REL)]) <= set(oi[q, :k][strict]) | set(oi[q, :k]), q
        assert np.all(gpu_dist[q][~strict[: k]] >= lo * (1 - DIST_REL)), q
        exempt += 1
    ref = od[:, :k]
    err = np.abs(gpu_dist - ref)
    assert np.all(err <= DIST_REL * ref + 1e-30), float(np.max(err / np.maximum(ref, 1e-30)))
    assert np.all(np.diff(gpu_dist, axis=1) >= 0)
    return {"queries": n, "exact": int(exact.sum()), "exempt": exempt}
