"""Error measure and algorithmic work model for BTA selected inversion / quadratic solve.

Error: per-block relative Frobenius error ||X - X_ref||_F / ||X_ref||_F, maximised
over every output block of the BTA pattern (diagonal, upper, lower, both arrows,
tip).  Where ||X_ref||_F < 1e-300 the absolute error is used.

Work model: complex multiply-adds (cMAC) of the executed formulation, counted
per block step of the forward pass (Alg. 1 with the arrow terms of Sec. III-A)
and of the backward pass (Alg. 2 with the compound trailing block, width
w = b + a).  Real flops = 8 x cMAC.  The paper's Table 4 op counts are not used:
they disagree with its own algorithms and text, so work is counted from the
formulas actually executed.
"""
from __future__ import annotations

import numpy as np

BLOCK_KEYS = ("diag", "upper", "lower", "arrow_r", "arrow_b", "tip")


def _blocks(arr: np.ndarray):
    if arr.ndim == 2:
        yield arr
    else:
        for x in arr:
            yield x


def max_block_rel_err(x: dict, ref: dict, keys=BLOCK_KEYS) -> float:
    """Max over pattern blocks of ||X - X_ref||_F / ||X_ref||_F; a block whose
    error is not finite (a NaN or inf anywhere in it) makes the result inf."""
    worst = 0.0
    for k in keys:
        if isinstance(ref[k], list):  # non-uniform blocks: lists of blocks
            if len(x[k]) != len(ref[k]):
                raise ValueError(f"block count mismatch in {k}")
            pairs = [(np.asarray(xb), np.asarray(rb)) for xb, rb in zip(x[k], ref[k])]
            for xb, rb in pairs:
                if xb.shape != rb.shape:
                    raise ValueError(f"shape mismatch in {k}: {xb.shape} vs {rb.shape}")
        else:
            xa = np.asarray(x[k])
            ra = np.asarray(ref[k])
            if xa.shape != ra.shape:
                raise ValueError(f"shape mismatch in {k}: {xa.shape} vs {ra.shape}")
            if ra.size == 0:
                continue
            pairs = zip(_blocks(xa), _blocks(ra))
        for xb, rb in pairs:
            if rb.size == 0:
                continue
            nr = np.linalg.norm(rb)
            e = np.linalg.norm(xb - rb)
            r = e / nr if nr >= 1e-300 else e
            if not np.isfinite(r):  # max() would drop a NaN
                return float("inf")
            worst = max(worst, r)
    return float(worst)


def cmac_forward(n: int, b: int, a: int, quad: bool = True, antihermitian: bool = False) -> float:
    """cMAC of the forward pass: per block the inversion (b^3, Gauss-Jordan or
    getrf+getri), the SI update 2b^3 + 3ab^2 + a^2 b for blocks with a
    successor, and the SQ update 6b^3 + 7ab^2 + 3a^2 b; the tip inversion a^3
    and, with B, S_B,tt = S_tt B_tt S_tt^H (2a^3).  antihermitian: B-hat_{t,i+1}
    is the mirror of B-hat_{i+1,t} (its three a b^2 products are not formed)."""
    inv = n * b ** 3
    # S_A B S_A^H on every block: 2 b^3
    sq_diag = n * 2 * b ** 3 if quad else 0
    # Lt = A_ti S_A on every block: a b^2 ; tip A update: a^2 b
    si_arrow_all = n * (a * b * b + a * a * b)
    # blocks with a successor: L1 (b^3), A_{i+1,i+1} (b^3), 2 arrow updates (2 a b^2)
    si_next = (n - 1) * (2 * b ** 3 + 2 * a * b * b)
    sq = 0
    if quad:
        # every block: A_ti S_B (a b^2), tip B update (3 a^2 b)
        sq += n * (a * b * b + 3 * a * a * b)
        # with successor: Q (b^3), 3 b^3 diag update, 6 a b^2 arrow updates
        # (3 a b^2 when the bottom arrow is mirrored)
        sq += (n - 1) * (4 * b ** 3 + (3 if antihermitian else 6) * a * b * b)
    tip = a ** 3 + (2 * a ** 3 if quad else 0)
    return float(inv + sq_diag + si_arrow_all + si_next + sq + tip)


def cmac_backward(n: int, b: int, a: int, quad: bool = True, antihermitian: bool = False) -> float:
    """cMAC of the backward pass: per block with trailing width w (b + a, or a
    for the last block): SI 2 b w^2 + 3 w b^2, SQ 4 b w^2 + 7 w b^2.
    antihermitian: X_R rho (b w^2), Y21 (2 w b^2) and Y_{R,i} (b w^2) are
    mirrors of products already formed: SQ 2 b w^2 + 5 w b^2."""
    total = 0.0
    for i in range(n):
        w = a if i == n - 1 else b + a
        total += 2 * b * w * w + 3 * w * b * b
        if quad:
            total += (2 * b * w * w + 5 * w * b * b) if antihermitian else (4 * b * w * w + 7 * w * b * b)
    return total


def flops_selquad(n: int, b: int, a: int, antihermitian: bool = False) -> float:
    """Real flops of one fused SI+SQ solve (8 per complex multiply-add);
    antihermitian: without the products that mirroring replaces."""
    return 8.0 * (cmac_forward(n, b, a, True, antihermitian) + cmac_backward(n, b, a, True, antihermitian))


def flops_selinv(n: int, b: int, a: int) -> float:
    return 8.0 * (cmac_forward(n, b, a, False) + cmac_backward(n, b, a, False))


def bytes_bta(n: int, b: int, a: int) -> int:
    """Bytes of one complex128 BTA matrix."""
    elems = n * b * b + 2 * (n - 1) * b * b + 2 * n * a * b + a * a
    return 16 * elems


def flops_products(n: int, b: int, a: int, quad: bool = True, antihermitian: bool = False) -> float:
    """Real flops of the block products of one solve: the whole work model
    minus the block inversions (n b^3 and the tip a^3 cMAC), i.e. the
    contractions of the forward and backward sweeps."""
    total = cmac_forward(n, b, a, quad, antihermitian) + cmac_backward(n, b, a, quad, antihermitian)
    return 8.0 * (total - n * b ** 3 - a ** 3)
