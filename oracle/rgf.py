"""Recursive Green's function (RGF) selected inversion + selected quadratic solve
for block-tridiagonal-with-arrowhead (BTA) matrices, complex128, plain numpy.

Notation follows the paper: blocks i = 0..n-1 of size b, arrow tip t of size a,
hat = value after forward (Schur complement) updates, ^H = conjugate transpose
(the paper's dagger).  Inputs and outputs are dicts with keys
diag (n,b,b), upper (n-1,b,b) = X_{i,i+1}, lower (n-1,b,b) = X_{i+1,i},
arrow_r (n,b,a) = X_{i,t}, arrow_b (n,a,b) = X_{t,i}, tip (a,a) = X_{t,t}.
Non-uniform block sizes b_i (the matrices of Sec. II-A need not have equal
blocks): the same keys hold Python lists of blocks, diag[i] b_i x b_i,
upper[i] b_i x b_{i+1}, lower[i] b_{i+1} x b_i, arrow_r[i] b_i x a,
arrow_b[i] a x b_i; every step below is per block and reads the sizes from
the blocks themselves.

Readings of the paper taken here (the BTA equations themselves are in a figure
that is not printed, Fig. 5):
* Alg. 1 loops over "n_i" but its body uses i; the loop index is i.
* The arrow tip is the last block row/column (bottom right), Sec. III-A.
* Forward BTA step: eliminating block i updates block i+1, the arrow blocks
  (i+1, t), (t, i+1) and the tip (t, t); these are the only nonzero products
  (Sec. III-A, Fig. 5(b)).  The formulas are the block LDU elimination of the
  trailing matrix, A_R <- A_R - r S c, and B_R <- B_R + r S_B r^H - rho (r S)^H
  - (r S) gamma, with r, c, rho, gamma the coupling column/row of A and B.
* Backward BTA step: the trailing set R = {i+1, t} (or {t} for the last block)
  is treated as one compound block, mirroring Alg. 2 with T1A = S c, T2A = X_R r.
"""
from __future__ import annotations

import numpy as np


def _h(x: np.ndarray) -> np.ndarray:
    """Conjugate transpose of one block."""
    return np.conj(x.T)


def _inv(x: np.ndarray) -> np.ndarray:
    """Inverse of one diagonal block (LAPACK getrf + getri, partial pivoting
    inside the block only, as in Sec. II-B)."""
    if x.shape[0] == 0:
        return x.copy()
    return np.linalg.inv(x)


def shape_of(m: dict):
    """(n, b, a); b is None for non-uniform blocks (lists of blocks)."""
    a = m["tip"].shape[0]
    if isinstance(m["diag"], list):
        return len(m["diag"]), None, a
    n, b, _ = m["diag"].shape
    return n, b, a


def block_sizes(m: dict) -> list[int]:
    return [int(d.shape[0]) for d in m["diag"]]


def _copy(x):
    """Working copy of one block array (stacked array or list of blocks)."""
    return [y.copy() for y in x] if isinstance(x, list) else x.copy()


def _like(x):
    """Uninitialised array of the same blocks (stacked) or n empty slots (list)."""
    return [None] * len(x) if isinstance(x, list) else np.empty_like(x)


# ---------------------------------------------------------------------------
# a0: system matrix of Sec. I: A = (E + i eta) I - H - Sigma^R
# ---------------------------------------------------------------------------
def assemble_a(h: dict, energy: float, eta: float, gamma: float) -> dict:
    """A = (E + i*eta) I - H - Sigma^R with the contact self-energy
    Sigma^R = -i*gamma*I on the first and last diagonal blocks (Sec. I: the
    open-boundary contacts couple only to the source and drain ends); the tip is
    not a contact block.  All pattern blocks of A are -H except the diagonal."""
    n, _, a = shape_of(h)
    z = complex(energy, eta)
    out = {k: ([-x for x in v] if isinstance(v, list) else -v.copy()) for k, v in h.items()}
    for i in range(n):
        out["diag"][i] += z * np.eye(out["diag"][i].shape[0])
    for i in sorted({0, n - 1}):
        out["diag"][i] += 1j * gamma * np.eye(out["diag"][i].shape[0])
    if a:
        out["tip"] += z * np.eye(a)
    return out


# ---------------------------------------------------------------------------
# Forward pass: Alg. 1 extended to the arrowhead (Sec. III-A)
# ---------------------------------------------------------------------------
def forward(A: dict, B: dict | None = None) -> dict:
    """Schur-complement sweep over the diagonal blocks, then the tip.

    Returns the factor: S_A[i] = (A_hat_ii)^{-1}, S_B[i] = S_A[i] B_hat_ii S_A[i]^H,
    the arrow blocks as they were when block i was eliminated, and the tip
    quantities S_tt = (A_hat_tt)^{-1}, S_B,tt = S_tt B_hat_tt S_tt^H.
    """
    n, b, a = shape_of(A)
    quad = B is not None
    Ad = _copy(A["diag"])          # A_hat_ii
    Ar = _copy(A["arrow_r"])       # A_hat_{i,t}
    Ab = _copy(A["arrow_b"])       # A_hat_{t,i}
    Att = A["tip"].copy()          # A_hat_tt
    SA = _like(Ad)
    if quad:
        Bd = _copy(B["diag"])
        Br = _copy(B["arrow_r"])
        Bb = _copy(B["arrow_b"])
        Btt = B["tip"].copy()
        SB = _like(Bd)

    for i in range(n):
        # Alg. 1 line 2 (line 7 for the last block): S_A,ii <- A_ii^{-1}
        SA[i] = _inv(Ad[i])
        # Alg. 1 line 3 (line 8): S_B,ii <- S_A,ii B_ii S_A,ii^H
        if quad:
            SB[i] = SA[i] @ Bd[i] @ _h(SA[i])
        # arrow row of the lower factor: Lt = A_hat_{t,i} S_A,ii
        Lt = Ab[i] @ SA[i]
        if i < n - 1:
            # Alg. 1 line 4: T1A <- A_{i+1,i} S_A,ii
            T1A = A["lower"][i] @ SA[i]
            # Alg. 1 line 5: A_{i+1,i+1} <- A_{i+1,i+1} - T1A A_{i,i+1}
            Ad[i + 1] = Ad[i + 1] - T1A @ A["upper"][i]
            # Sec. III-A: arrow blocks of the next column/row
            Ar[i + 1] = Ar[i + 1] - T1A @ Ar[i]
            Ab[i + 1] = Ab[i + 1] - Lt @ A["upper"][i]
            if quad:
                # Alg. 1 line 6
                Bd[i + 1] = (Bd[i + 1]
                             + A["lower"][i] @ SB[i] @ _h(A["lower"][i])
                             - B["lower"][i] @ _h(T1A)
                             - T1A @ B["upper"][i])
                # Sec. III-A: B arrow blocks of the next column/row
                Br[i + 1] = (Br[i + 1]
                             + A["lower"][i] @ SB[i] @ _h(Ab[i])
                             - T1A @ Br[i]
                             - B["lower"][i] @ _h(Lt))
                Bb[i + 1] = (Bb[i + 1]
                             + Ab[i] @ SB[i] @ _h(A["lower"][i])
                             - Lt @ B["upper"][i]
                             - Bb[i] @ _h(T1A))
        # Sec. III-A: tip updates from block i
        if quad:
            Btt = Btt + Ab[i] @ SB[i] @ _h(Ab[i]) - Lt @ Br[i] - Bb[i] @ _h(Lt)
        Att = Att - Lt @ Ar[i]

    f = {"n": n, "b": b, "a": a, "SA": SA, "Ar": Ar, "Ab": Ab,
         "Stt": _inv(Att), "quad": quad}
    if quad:
        f.update({"SB": SB, "Br": Br, "Bb": Bb})
        f["SBtt"] = f["Stt"] @ Btt @ _h(f["Stt"])
    return f


# ---------------------------------------------------------------------------
# Backward pass: Alg. 2 with the compound trailing block R = {i+1, t}
# ---------------------------------------------------------------------------
def _cat_rows(top, bot):
    return np.concatenate([top, bot], axis=0)


def _cat_cols(left, right):
    return np.concatenate([left, right], axis=1)


def backward(A: dict, f: dict, B: dict | None = None) -> tuple[dict, dict | None]:
    """Selected inversion (G^R) and, if B is given, selected quadratic solve
    (G^<) from the forward factor ``f``.  Returns (GR, GL)."""
    n, b, a = f["n"], f["b"], f["a"]
    quad = B is not None
    if quad and not f["quad"]:
        raise ValueError("factor was computed without B")
    if b is None:  # non-uniform blocks: lists filled block by block
        GR = {"diag": [None] * n, "upper": [None] * (n - 1), "lower": [None] * (n - 1),
              "arrow_r": [None] * n, "arrow_b": [None] * n, "tip": f["Stt"].copy()}
    else:
        GR = {"diag": np.empty((n, b, b), complex), "upper": np.empty((n - 1, b, b), complex),
              "lower": np.empty((n - 1, b, b), complex), "arrow_r": np.empty((n, b, a), complex),
              "arrow_b": np.empty((n, a, b), complex), "tip": f["Stt"].copy()}
    GL = None
    if quad:
        GL = {k: _like(v) for k, v in GR.items()}
        GL["tip"] = f["SBtt"].copy()

    # Alg. 2 lines 1-2 (arrow version): X_tt <- S_tt, Y_tt <- S_B,tt
    for i in range(n - 1, -1, -1):
        S = f["SA"][i]
        if i == n - 1:
            # trailing set R = {t}
            XR = GR["tip"]
            r = f["Ab"][i]                       # A_hat_{t,i}
            c = f["Ar"][i]                       # A_hat_{i,t}
            if quad:
                YR = GL["tip"]
                rho = f["Bb"][i]                 # B_hat_{t,i}
                gam = f["Br"][i]                 # B_hat_{i,t}
        else:
            # trailing set R = {i+1, t}: compound 2x2 block
            XR = np.block([[GR["diag"][i + 1], GR["arrow_r"][i + 1]],
                           [GR["arrow_b"][i + 1], GR["tip"]]])
            r = _cat_rows(A["lower"][i], f["Ab"][i])     # [A_{i+1,i}; A_hat_{t,i}]
            c = _cat_cols(A["upper"][i], f["Ar"][i])     # [A_{i,i+1}, A_hat_{i,t}]
            if quad:
                YR = np.block([[GL["diag"][i + 1], GL["arrow_r"][i + 1]],
                               [GL["arrow_b"][i + 1], GL["tip"]]])
                rho = _cat_rows(B["lower"][i], f["Bb"][i])
                gam = _cat_cols(B["upper"][i], f["Br"][i])

        # Alg. 2 line 4: T1A <- S_A,ii c ; T2A <- X_R r
        T1A = S @ c
        T2A = XR @ r
        # Alg. 2 line 5: X_{R,i} <- -T2A S_A,ii
        X_Ri = -T2A @ S
        # Alg. 2 line 6: X_{i,R} <- -T1A X_R
        X_iR = -T1A @ XR
        # Alg. 2 line 7: X_ii <- S_A,ii - T1A X_{R,i}
        X_ii = S - T1A @ X_Ri

        if quad:
            SBi = f["SB"][i]
            # Alg. 2 lines 8-9 grouped: Y12 = T4B - T2B, Y21 = T5B - T3B
            Y12 = S @ gam @ _h(XR) - SBi @ _h(T2A)
            Y21 = XR @ rho @ _h(S) - T2A @ SBi
            # Alg. 2 lines 10-12
            Y_iR = Y12 - T1A @ YR
            Y_Ri = Y21 - YR @ _h(T1A)
            Y_ii = SBi - T1A @ Y21 - Y12 @ _h(T1A) + T1A @ YR @ _h(T1A)

        GR["diag"][i] = X_ii
        if i == n - 1:
            GR["arrow_r"][i] = X_iR
            GR["arrow_b"][i] = X_Ri
        else:
            k = A["upper"][i].shape[1]  # b_{i+1}: the R = {i+1, t} split
            GR["upper"][i] = X_iR[:, :k]
            GR["arrow_r"][i] = X_iR[:, k:]
            GR["lower"][i] = X_Ri[:k, :]
            GR["arrow_b"][i] = X_Ri[k:, :]
        if quad:
            GL["diag"][i] = Y_ii
            if i == n - 1:
                GL["arrow_r"][i] = Y_iR
                GL["arrow_b"][i] = Y_Ri
            else:
                GL["upper"][i] = Y_iR[:, :k]
                GL["arrow_r"][i] = Y_iR[:, k:]
                GL["lower"][i] = Y_Ri[:k, :]
                GL["arrow_b"][i] = Y_Ri[k:, :]
    return GR, GL


def selinv(A: dict) -> dict:
    """G^R = A^{-1} on the BTA pattern (SI)."""
    return backward(A, forward(A))[0]


def selquad(A: dict, B: dict) -> tuple[dict, dict]:
    """Fused SI + SQ: (G^R, G^< = A^{-1} B A^{-H}) on the BTA pattern."""
    return backward(A, forward(A, B), B)


# ---------------------------------------------------------------------------
# Alg. 1 / Alg. 2 exactly as printed, block-tridiagonal only (a = 0)
# ---------------------------------------------------------------------------
def rgf_bt_printed(A: dict, B: dict) -> tuple[dict, dict]:
    """The literal BT form of Alg. 1 and Alg. 2 (no arrowhead, a = 0), kept as a
    second path that shares no grouping with ``forward``/``backward``."""
    n, b, a = shape_of(A)
    if a != 0:
        raise ValueError("printed Alg. 1/2 is for block-tridiagonal matrices (a = 0)")
    Ad = A["diag"].copy()
    Bd = B["diag"].copy()
    SA = np.empty_like(Ad)
    SB = np.empty_like(Bd)
    # Alg. 1
    for i in range(n - 1):
        SA[i] = np.linalg.inv(Ad[i])
        SB[i] = SA[i] @ Bd[i] @ _h(SA[i])
        T1A = A["lower"][i] @ SA[i]
        Ad[i + 1] = Ad[i + 1] - T1A @ A["upper"][i]
        Bd[i + 1] = (Bd[i + 1] + A["lower"][i] @ SB[i] @ _h(A["lower"][i])
                     - B["lower"][i] @ _h(T1A) - T1A @ B["upper"][i])
    SA[n - 1] = np.linalg.inv(Ad[n - 1])
    SB[n - 1] = SA[n - 1] @ Bd[n - 1] @ _h(SA[n - 1])
    # Alg. 2
    XA = {"diag": np.empty_like(Ad), "upper": np.empty_like(A["upper"]),
          "lower": np.empty_like(A["lower"])}
    XB = {"diag": np.empty_like(Ad), "upper": np.empty_like(A["upper"]),
          "lower": np.empty_like(A["lower"])}
    XA["diag"][n - 1] = SA[n - 1]
    XB["diag"][n - 1] = SB[n - 1]
    for i in range(n - 2, -1, -1):
        T1A = SA[i] @ A["upper"][i]
        T2A = XA["diag"][i + 1] @ A["lower"][i]
        XA["lower"][i] = -T2A @ SA[i]
        XA["upper"][i] = -T1A @ XA["diag"][i + 1]
        XA["diag"][i] = SA[i] - T1A @ XA["lower"][i]
        T1B = XB["diag"][i + 1] @ _h(T1A)
        T2B = SB[i] @ _h(T2A)
        T3B = T2A @ SB[i]
        T4B = SA[i] @ B["upper"][i] @ _h(XA["diag"][i + 1])
        T5B = XA["diag"][i + 1] @ B["lower"][i] @ _h(SA[i])
        XB["upper"][i] = -T1A @ XB["diag"][i + 1] - T2B + T4B
        XB["lower"][i] = -T1B - T3B + T5B
        XB["diag"][i] = (SB[i] + T1A @ T1B + T1A @ T3B + T2B @ _h(T1A)
                         - T1A @ T5B - T4B @ _h(T1A))
    for X in (XA, XB):
        X["arrow_r"] = np.zeros((n, b, 0), complex)
        X["arrow_b"] = np.zeros((n, 0, b), complex)
        X["tip"] = np.zeros((0, 0), complex)
    return XA, XB
