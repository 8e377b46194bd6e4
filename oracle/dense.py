"""Dense definition of the selected results (Alg. 4, Sec. II-C2), complex128.

G^R = A^{-1} and G^< = A^{-1} B A^{-H} computed from one full LU of the
N x N matrix (N = n*b + a), then restricted to the BTA pattern (Sec. II-A:
only the entries matching the pattern of A and B are wanted).  O(N^3) time and
O(N^2) memory, so only for small N.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def _offsets(sizes):
    o = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
    return [slice(o[i], o[i + 1]) for i in range(len(sizes))], int(o[-1])


def to_dense(m: dict) -> np.ndarray:
    """Scatter the BTA blocks into a dense N x N matrix (zero off the pattern).
    The tip occupies the last a rows/columns (Sec. III-A).  Blocks may differ
    in size (lists of blocks): block i spans rows/columns sum_{j<i} b_j ..."""
    sizes = [int(x.shape[0]) for x in m["diag"]]
    n = len(sizes)
    a = m["tip"].shape[0]
    sl, nb = _offsets(sizes)
    N = nb + a
    d = np.zeros((N, N), dtype=np.complex128)
    for i in range(n):
        s = sl[i]
        d[s, s] = m["diag"][i]
        d[s, nb:] = m["arrow_r"][i]
        d[nb:, s] = m["arrow_b"][i]
        if i < n - 1:
            s1 = sl[i + 1]
            d[s, s1] = m["upper"][i]
            d[s1, s] = m["lower"][i]
    d[nb:, nb:] = m["tip"]
    return d


def from_dense_sizes(d: np.ndarray, sizes, a: int) -> dict:
    """Gather the BTA-pattern blocks of a dense matrix with block sizes
    `sizes` into lists of blocks."""
    sl, nb = _offsets(sizes)
    n = len(sizes)
    return {"diag": [d[sl[i], sl[i]].copy() for i in range(n)],
            "upper": [d[sl[i], sl[i + 1]].copy() for i in range(n - 1)],
            "lower": [d[sl[i + 1], sl[i]].copy() for i in range(n - 1)],
            "arrow_r": [d[sl[i], nb:].copy() for i in range(n)],
            "arrow_b": [d[nb:, sl[i]].copy() for i in range(n)],
            "tip": d[nb:, nb:].copy()}


def from_dense(d: np.ndarray, n: int, b: int, a: int) -> dict:
    """Gather the BTA-pattern blocks of a dense matrix."""
    out = {
        "diag": np.stack([d[i * b:(i + 1) * b, i * b:(i + 1) * b] for i in range(n)]),
        "upper": np.zeros((n - 1, b, b), complex),
        "lower": np.zeros((n - 1, b, b), complex),
        "arrow_r": np.stack([d[i * b:(i + 1) * b, n * b:] for i in range(n)]),
        "arrow_b": np.stack([d[n * b:, i * b:(i + 1) * b] for i in range(n)]),
        "tip": d[n * b:, n * b:].copy(),
    }
    for i in range(n - 1):
        out["upper"][i] = d[i * b:(i + 1) * b, (i + 1) * b:(i + 2) * b]
        out["lower"][i] = d[(i + 1) * b:(i + 2) * b, i * b:(i + 1) * b]
    return {k: np.ascontiguousarray(v) for k, v in out.items()}


def dense_solve(A: dict, B: dict | None = None):
    """Alg. 4: L, U <- getrf(A); G^R = U \\ (L / I); Y = U \\ (L / B);
    X = Y A^{-H} (formed as (A^{-1} Y^H)^H with the same LU).
    Returns (GR, GL) restricted to the pattern (GL is None without B)."""
    a = A["tip"].shape[0]
    if isinstance(A["diag"], list):
        sizes = [int(x.shape[0]) for x in A["diag"]]
        gather = lambda d: from_dense_sizes(d, sizes, a)
    else:
        n, b, _ = A["diag"].shape
        gather = lambda d: from_dense(d, n, b, a)
    Ad = to_dense(A)
    lu = sla.lu_factor(Ad)
    N = Ad.shape[0]
    G = sla.lu_solve(lu, np.eye(N, dtype=np.complex128))
    GR = gather(G)
    if B is None:
        return GR, None
    Y = sla.lu_solve(lu, to_dense(B))
    X = np.conj(sla.lu_solve(lu, np.conj(Y.T)).T)
    return GR, gather(X)
