"""Host logic of the partitioned solve (Sec. III-B on one GPU), without a GPU.

The library's move plan (qsi_partition_plan) is executed here in numpy. The
partitions' partial sweeps are restated from Alg. 1/2 in their compound-arrow
form, and the oracle solves the reduced system.  The assembled G^R and G^< must
equal the oracle's unpartitioned solve of the same matrix.  This pins the
plan: the interior layout with identity padding, the permuted top separator
in the arrow, the reduced-system assembly, the boundary hand-off and the
scatter.  The phases' disjointness, which the single-launch execution of each
phase relies on, is checked element by element.

Accuracy: the partitions' pivots are Schur complements of interior sub-chains,
which lack the contact self-energy of blocks 0 and n-1 that keeps RGF's
leading pivots well conditioned.  At the recipe's broadening eta = 1e-3 their
condition numbers run 10-50 times RGF's, and G^< (two factors of every
pivot) loses accordingly: 1e-9 against 1e-14 for RGF on the same matrix.  At
eta = 0.1 both agree with the dense definition to 1e-14.  The parity bar of
1e-10 is therefore applied at eta = 0.1, and a bound from the measured pivot
conditioning at eta = 1e-3."""
import numpy as np
import pytest

from conftest import make_problem
from oracle import rgf
from paper_2601_04904_gb300 import inputs
from paper_2601_04904_gb300.metrics import max_block_rel_err

qsi = pytest.importorskip("paper_2601_04904_gb300.qsi")

MAXF = 1 + qsi.MAX_RHS
K_IN, K_LOC, K_RED, K_RED_OUT, K_LOC_OUT, K_OUT = range(6)
H = lambda x: np.conj(np.swapaxes(x, -1, -2))


def aid(kind, fam, k):
    return (kind * MAXF + fam) * 6 + k


def run_moves(arrs, moves, lo, hi):
    for x in moves[lo:hi]:
        out = np.eye(x.rows, dtype=np.complex128) if x.fill == 1 else np.zeros((x.rows, x.cols), np.complex128)
        for s in range(3):
            if x.src[s] < 0:
                continue
            for j in range(x.cnt[s]):
                o = x.off[s] + j * x.stride[s]
                src = arrs[x.src[s]]
                out = out + np.stack([src[o + r * x.lds[s]: o + r * x.lds[s] + x.cols] for r in range(x.rows)])
        d = arrs[x.dst]
        for r in range(x.rows):
            d[x.dst_off + r * x.ldd: x.dst_off + r * x.ldd + x.cols] = out[r]


def blocks(v, cnt, rows, cols):
    return v[: cnt * rows * cols].reshape(cnt, rows, cols)


def local_views(arrs, f, p, m, b, w, sD, sR, kind):
    """Views of partition p's arrays (m+1 blocks, arrow width w)."""
    sU = m * b * b
    d = blocks(arrs[aid(kind, f, 0)][p * sD:], m + 1, b, b)
    u = blocks(arrs[aid(kind, f, 1)][p * sU:], m, b, b)
    lo = blocks(arrs[aid(kind, f, 2)][p * sU:], m, b, b)
    r = blocks(arrs[aid(kind, f, 3)][p * sR:], m + 1, b, w)
    bt = blocks(arrs[aid(kind, f, 4)][p * sR:], m + 1, w, b)
    t = arrs[aid(kind, f, 5)][p * w * w:(p + 1) * w * w].reshape(w, w)
    return d, u, lo, r, bt, t


def partial_forward(A, Bs, m):
    """Alg. 1 (arrow form of Sec. III-A) over blocks 0..m-1 of an (m+1)-block
    BTA: block m and the tip receive their updates but are not inverted.
    In place: A[0][i] becomes S_i, every B[0][i] becomes S_B,i."""
    D, U, Lo, Ar, Ab, T = A
    for i in range(m):
        S = np.linalg.inv(D[i])
        D[i] = S
        L1, Lt = Lo[i] @ S, Ab[i] @ S
        for (SB, Bu, Bl, Br, Bb, Bt) in Bs:
            SBi = S @ SB[i] @ H(S)
            SB[i] = SBi
            Q, W = Lo[i] @ SBi, Ab[i] @ SBi
            SB[i + 1] += Q @ H(Lo[i]) - Bl[i] @ H(L1) - L1 @ Bu[i]
            Br[i + 1] += Q @ H(Ab[i]) - L1 @ Br[i] - Bl[i] @ H(Lt)
            Bb[i + 1] += W @ H(Lo[i]) - Lt @ Bu[i] - Bb[i] @ H(L1)
            Bt += W @ H(Ab[i]) - Lt @ Br[i] - Bb[i] @ H(Lt)
        D[i + 1] -= L1 @ U[i]
        Ar[i + 1] -= L1 @ Ar[i]
        Ab[i + 1] -= Lt @ U[i]
        T -= Lt @ Ar[i]


def partial_backward(A, Bs, X, Ys, m, b):
    """Alg. 2 with the trailing set R = {i+1, arrow}, i = m-1..0, started from
    the block-m and tip outputs already in X, Ys."""
    S_, U, Lo, Ar, Ab, _ = A
    Xd, Xu, Xl, Xr, Xb, Xt = X
    for i in range(m - 1, -1, -1):
        S = S_[i]
        XR = np.block([[Xd[i + 1], Xr[i + 1]], [Xb[i + 1], Xt]])
        r = np.concatenate([Lo[i], Ab[i]], axis=0)
        c = np.concatenate([U[i], Ar[i]], axis=1)
        Uc, Pr = S @ c, XR @ r
        XRi, XiR = -Pr @ S, -Uc @ XR
        for (SB, Bu, Bl, Br, Bb, _), Y in zip(Bs, Ys):
            Yd, Yu, Yl, Yr, Yb, Yt = Y
            YR = np.block([[Yd[i + 1], Yr[i + 1]], [Yb[i + 1], Yt]])
            rho = np.concatenate([Bl[i], Bb[i]], axis=0)
            gam = np.concatenate([Bu[i], Br[i]], axis=1)
            Y12 = S @ gam @ H(XR) - SB[i] @ H(Pr)
            Y21 = XR @ rho @ H(S) - Pr @ SB[i]
            YiR, YRi = Y12 - Uc @ YR, Y21 - YR @ H(Uc)
            Yd[i] = SB[i] - Uc @ Y21 - Y12 @ H(Uc) + Uc @ YR @ H(Uc)
            Yu[i], Yr[i] = YiR[:, :b], YiR[:, b:]
            Yl[i], Yb[i] = YRi[:b], YRi[b:]
        Xd[i] = S - Uc @ XRi
        Xu[i], Xr[i] = XiR[:, :b], XiR[:, b:]
        Xl[i], Xb[i] = XRi[:b], XRi[b:]


def reduced_dict(arrs, kind, f, nr, b, a):
    d = {"diag": blocks(arrs[aid(kind, f, 0)], nr, b, b), "upper": blocks(arrs[aid(kind, f, 1)], nr - 1, b, b),
         "lower": blocks(arrs[aid(kind, f, 2)], nr - 1, b, b), "arrow_r": blocks(arrs[aid(kind, f, 3)], nr, b, a),
         "arrow_b": blocks(arrs[aid(kind, f, 4)], nr, a, b), "tip": arrs[aid(kind, f, 5)][: a * a].reshape(a, a)}
    return d


def partitioned_solve(A, Bs, P, diag_only=False):
    n, b, a = rgf.shape_of(A)
    plan = qsi.partition_plan(n, b, a, P, len(Bs), diag_only)
    assert plan is not None
    moves, sizes, pe, (P_, m, w, nr, sD, sR) = plan
    assert P_ == P and w == (a if P == 2 else b + a) and nr == P - 1  # P = 2: the twisted split
    arrs = {i: np.zeros(int(sizes[i]), np.complex128) for i in range(qsi.PLAN_ARRAYS)}
    for f, M in enumerate([A] + Bs):
        for k, key in enumerate(qsi.KEYS):
            if sizes[aid(K_IN, f, k)]:
                arrs[aid(K_IN, f, k)][:] = M[key].ravel()
    run_moves(arrs, moves, 0, pe[0])
    nf = 1 + len(Bs)
    for p in range(P):
        Aloc = local_views(arrs, 0, p, m, b, w, sD, sR, K_LOC)
        Bloc = [local_views(arrs, f, p, m, b, w, sD, sR, K_LOC) for f in range(1, nf)]
        partial_forward(Aloc, Bloc, m)
    run_moves(arrs, moves, pe[0], pe[1])
    Ar = reduced_dict(arrs, K_RED, 0, nr, b, a)
    outs = [rgf.selinv(Ar)] + [rgf.selquad(Ar, reduced_dict(arrs, K_RED, f, nr, b, a))[1] for f in range(1, nf)]
    for f, o in enumerate(outs):
        for k, key in enumerate(qsi.KEYS):
            arrs[aid(K_RED_OUT, f, k)][:] = o[key].ravel()
    run_moves(arrs, moves, pe[1], pe[2])
    for p in range(P):
        Aloc = local_views(arrs, 0, p, m, b, w, sD, sR, K_LOC)
        Bloc = [local_views(arrs, f, p, m, b, w, sD, sR, K_LOC) for f in range(1, nf)]
        X = local_views(arrs, 0, p, m, b, w, sD, sR, K_LOC_OUT)
        Ys = [local_views(arrs, f, p, m, b, w, sD, sR, K_LOC_OUT) for f in range(1, nf)]
        partial_backward(Aloc, Bloc, X, Ys, m, b)
    run_moves(arrs, moves, pe[2], pe[3])
    res = []
    for f in range(nf):
        d = {"diag": blocks(arrs[aid(K_OUT, f, 0)], n, b, b), "arrow_r": blocks(arrs[aid(K_OUT, f, 3)], n, b, a),
             "arrow_b": blocks(arrs[aid(K_OUT, f, 4)], n, a, b), "tip": arrs[aid(K_OUT, f, 5)].reshape(a, a)}
        if not diag_only:
            d["upper"] = blocks(arrs[aid(K_OUT, f, 1)], n - 1, b, b)
            d["lower"] = blocks(arrs[aid(K_OUT, f, 2)], n - 1, b, b)
        res.append(d)
    return res, plan


def _rel(x, y, keys):
    return max_block_rel_err(x, y, keys)


@pytest.mark.parametrize("n,b,a,P,k", [(3, 2, 1, 2, 1), (5, 3, 2, 2, 1), (9, 3, 2, 3, 1), (10, 2, 0, 3, 1),
                                       (17, 4, 3, 5, 2), (7, 1, 1, 4, 1), (12, 3, 2, 4, 0), (11, 2, 5, 3, 1),
                                       (14, 3, 2, 3, 1)])
def test_partitioned_plan_matches_oracle(n, b, a, P, k):
    _, A, B = make_problem(n, b, a, seed=60 + n, eta=0.1)
    Bs = [B] + [inputs.lesser_rhs(n, b, a, seed=inputs.BASE_SEED + 500 + r) for r in range(1, k)]
    res, _ = partitioned_solve(A, Bs[:k], P)
    keys = qsi.KEYS if n > 1 else ("diag", "arrow_r", "arrow_b", "tip")
    assert _rel(res[0], rgf.selinv(A), keys) < 1e-10
    for r in range(k):
        assert _rel(res[1 + r], rgf.selquad(A, Bs[r])[1], keys) < 1e-10, r


def test_partitioned_plan_diagonal_only():
    n, b, a, P = 11, 3, 2, 3
    _, A, B = make_problem(n, b, a, seed=71, eta=0.1)
    res, _ = partitioned_solve(A, [B], P, diag_only=True)
    keys = ("diag", "arrow_r", "arrow_b", "tip")
    assert _rel(res[0], rgf.selinv(A), keys) < 1e-10
    assert _rel(res[1], rgf.selquad(A, B)[1], keys) < 1e-10


def partition_pivot_kappa(A, P, frobenius=False):
    """Largest 2-norm condition number among the partitions' pivots, formed
    exactly as the partial forward sweeps of the library's plan form them
    (interiors with the top separator permuted into the arrow).  frobenius:
    ||S||_F ||S^-1||_F instead, the upper bound of it that the automatic
    partition choice estimates on the device."""
    n, b, a = rgf.shape_of(A)
    moves, sizes, pe, (_, m, w, _, sD, sR) = qsi.partition_plan(n, b, a, P, 1, False)
    arrs = {i: np.zeros(int(sizes[i]), np.complex128) for i in range(qsi.PLAN_ARRAYS)}
    for kk, key in enumerate(qsi.KEYS):
        arrs[aid(K_IN, 0, kk)][:] = A[key].ravel()
    run_moves(arrs, [x for x in moves[:pe[0]] if x.dst // 6 == aid(K_LOC, 0, 0) // 6], 0, None)
    kappa = 0.0
    for p in range(P):
        D, U, Lo, Ar, Ab, T = local_views(arrs, 0, p, m, b, w, sD, sR, K_LOC)
        for i in range(m):
            S = np.linalg.inv(D[i])
            k = np.linalg.norm(D[i]) * np.linalg.norm(S) if frobenius else np.linalg.cond(D[i])
            kappa = max(kappa, k)
            D[i + 1] -= Lo[i] @ S @ U[i]
            Ar[i + 1] -= Lo[i] @ S @ Ar[i]
            Ab[i + 1] -= Ab[i] @ S @ U[i]
    return kappa


@pytest.mark.parametrize("n,b,a,P,seed", [(14, 3, 2, 3, 1), (30, 4, 2, 5, 90), (64, 8, 4, 8, 3)])
def test_partitioned_small_broadening_within_conditioning_bound(n, b, a, P, seed):
    """eta = 1e-3: the error follows the interior pivots' conditioning kappa
    (G^< carries two factors of every pivot): within 1e-13 * kappa^2."""
    _, A, B = make_problem(n, b, a, seed=seed)
    res, plan = partitioned_solve(A, [B], P)
    bound = 1e-13 * partition_pivot_kappa(A, P) ** 2
    assert max_block_rel_err(res[0], rgf.selinv(A)) < bound
    assert max_block_rel_err(res[1], rgf.selquad(A, B)[1]) < bound


@pytest.mark.parametrize("n,b,a,P,k,diag", [(9, 3, 2, 3, 1, False), (17, 4, 3, 5, 2, False), (10, 2, 0, 3, 1, True)])
def test_partition_phases_write_disjoint_elements(n, b, a, P, k, diag):
    """Within a phase no element is written twice, and none is read that the
    same phase writes: one kernel launch can run a phase's moves in any order."""
    moves, _, pe, _ = qsi.partition_plan(n, b, a, P, k, diag)
    lo = 0
    for hi in pe:
        written, read = set(), set()
        for x in moves[lo:hi]:
            for r in range(x.rows):
                for c in range(x.cols):
                    e = (x.dst, x.dst_off + r * x.ldd + c)
                    assert e not in written
                    written.add(e)
                    for s in range(3):
                        if x.src[s] >= 0:
                            for j in range(x.cnt[s]):
                                read.add((x.src[s], x.off[s] + j * x.stride[s] + r * x.lds[s] + c))
        assert not (written & read)
        lo = hi


def test_partition_layout_and_invalid_counts():
    # interiors as equal as possible, the longer ones first; m = the longest
    _, _, pe, meta = qsi.partition_plan(14, 2, 1, 3, 1)
    assert meta[:4] == (3, 4, 3, 2)  # 12 interior blocks over 3 partitions; arrow width b + a; 2 separators
    _, _, _, meta = qsi.partition_plan(15, 2, 1, 3, 1)
    assert meta[1] == 5  # 13 interior blocks: 5, 4, 4
    assert qsi.partition_plan(7, 2, 1, 4, 1) is not None  # 2P - 1 = n: one interior block each
    assert qsi.partition_plan(6, 2, 1, 4, 1) is None
    assert qsi.partition_plan(6, 2, 1, 1, 1) is None  # P = 1 has no plan (the plain solve)
    assert qsi.partition_plan(6, 2, 1, 2, qsi.MAX_RHS + 1) is None


@pytest.mark.parametrize("n,b,a,P,k,diag", [(3, 2, 1, 2, 1, False), (11, 2, 3, 3, 2, False), (16, 1, 2, 5, 1, True),
                                            (25, 2, 0, 7, 1, False), (9, 3, 2, 5, 0, False)])
def test_partition_plan_covers_every_output_and_input(n, b, a, P, k, diag):
    """Every element of the caller's outputs is written exactly once (phase 3),
    every element of the caller's inputs is read (phases 0 and 1), and every
    partition / reduced array element a sweep reads as input is written first."""
    moves, sizes, pe, _ = qsi.partition_plan(n, b, a, P, k, diag)
    written = {}
    read = set()
    for ph, (lo, hi) in enumerate(zip([0] + pe[:-1], pe)):
        for x in moves[lo:hi]:
            for r in range(x.rows):
                for c in range(x.cols):
                    e = (x.dst, x.dst_off + r * x.ldd + c)
                    written.setdefault(e, []).append(ph)
                    for s in range(3):
                        if x.src[s] >= 0:
                            for j in range(x.cnt[s]):
                                read.add((x.src[s], x.off[s] + j * x.stride[s] + r * x.lds[s] + c))
    for f in range(1 + k):
        for kk in range(6):
            out_id, in_id = aid(K_OUT, f, kk), aid(K_IN, f, kk)
            for e in range(int(sizes[out_id])):
                assert written.get((out_id, e)) == [3], (f, kk, e)
            for e in range(int(sizes[in_id])):
                assert (in_id, e) in read, (f, kk, e)
            # the reduced system's inputs are all assembled in phase 1
            red = aid(K_RED, f, kk)
            for e in range(int(sizes[red])):
                assert written.get((red, e)) == [1], ("reduced", f, kk, e)


@pytest.mark.parametrize("n,b,a,P,seed,eta", [(16, 8, 4, 4, 2, 2.0), (14, 3, 2, 3, 1, 1e-3), (9, 16, 8, 3, 89, 0.1)])
def test_frobenius_kappa_bounds_the_2norm_kappa(n, b, a, P, seed, eta):
    """The estimate of the automatic partition choice: kappa_2 <= kappa_F <=
    b * kappa_2 on the plan's pivots (||X||_2 <= ||X||_F <= sqrt(b) ||X||_2)."""
    _, A, _ = make_problem(n, b, a, seed=seed, eta=eta)
    k2, kf = partition_pivot_kappa(A, P), partition_pivot_kappa(A, P, frobenius=True)
    assert k2 <= kf * (1 + 1e-12) and kf <= b * k2 * (1 + 1e-12)


@pytest.mark.parametrize("n,b,a,k,diag", [(3, 2, 1, 1, False), (4, 3, 2, 1, False), (9, 3, 2, 2, False),
                                          (10, 4, 0, 1, False), (15, 3, 2, 1, True), (64, 4, 2, 1, False),
                                          (30, 5, 3, 3, False)])
def test_twisted_split_at_recipe_broadening(n, b, a, k, diag):
    """P = 2 is the twisted split: the top interior eliminated from block 0
    down, the bottom one from block n-1 up (stored reversed), meeting at one
    separator.  Both start at a contact block, so the pivots are the plain
    sweep's own (top half) or the reversed matrix's (bottom half): at the
    recipe's eta = 1e-3, where the general partitions miss 1e-10, the result
    matches the oracle's dense definition (Alg. 4) at 1e-10.  (There, on one
    of these right-hand sides, the oracle's own sweep is 2.3e-10 from the
    dense result and the twisted split 1e-11: the reference is the dense one.)"""
    from oracle.dense import dense_solve

    _, A, B = make_problem(n, b, a, seed=120 + n)
    Bs = ([B] + [inputs.lesser_rhs(n, b, a, seed=inputs.BASE_SEED + 700 + r) for r in range(1, k)])[:k]
    res, (_, _, _, (P_, m, w, nr, _, _)) = partitioned_solve(A, Bs, 2, diag_only=diag)
    assert (w, nr, m) == (a, 1, (n - 1 + 1) // 2)
    keys = ("diag", "arrow_r", "arrow_b", "tip") if diag else qsi.KEYS
    assert _rel(res[0], dense_solve(A)[0], keys) < 1e-10
    for r in range(k):
        assert _rel(res[1 + r], dense_solve(A, Bs[r])[1], keys) < 1e-10, r


def test_twisted_split_pivots_conditioned_like_the_plain_sweep():
    """The twisted halves' pivots are Schur complements grown from a contact
    block: their largest condition number stays within a small factor of the
    plain sweep's, while the general three-way split's interior pivots do not."""
    n, b, a = 64, 8, 4
    _, A, _ = make_problem(n, b, a, seed=3)
    D = [A["diag"][i].copy() for i in range(n)]
    k_plain = 0.0
    for i in range(n):
        k_plain = max(k_plain, np.linalg.cond(D[i]))
        if i + 1 < n:
            D[i + 1] = D[i + 1] - A["lower"][i] @ np.linalg.inv(D[i]) @ A["upper"][i]
    k2, k3 = partition_pivot_kappa(A, 2), partition_pivot_kappa(A, 3)
    assert k2 <= 2 * k_plain, (k2, k_plain)
    assert k3 > 2 * k_plain, (k3, k_plain)


@pytest.mark.parametrize("n,b,a,k,diag", [(3, 2, 1, 1, False), (8, 3, 2, 1, True), (9, 2, 0, 0, False),
                                          (12, 4, 3, 1, False), (13, 1, 2, 1, True), (6, 2, 3, 2, False)])
def test_twisted_plan_host_io_mapping(n, b, a, k, diag):
    """The twisted split's host entry replaces phases 0 and 3 by one copy per
    block between the host arrays and the partition slots, and phase 1's reads
    of the caller's arrays by a staging area.  That holds when (i) phase 0 is
    the identity padding plus exactly these contiguous block copies: slot j of
    the top half <- block j - j0, slot j of the bottom half <- block
    n - 1 - (j - j0) with its couplings' upper and lower swapped; (ii) phase 3
    is their reverse (off-diagonal blocks only for full outputs) plus the
    separator's and the tip's outputs; (iii) phase 1 reads of the caller's
    inputs exactly the separator's diagonal and arrow blocks and the tip."""
    A_D, A_U, A_L, A_R, A_B, A_T = range(6)
    moves, _, pe, meta = qsi.partition_plan(n, b, a, 2, k, diag)
    P, m, w = meta[0], meta[1], meta[2]
    assert P == 2 and w == a
    bb, ba = b * b, b * a
    sig = n // 2  # the separator: the top interior holds blocks 0 .. sig - 1
    assert m == sig
    lens = [sig, n - 1 - sig]
    j0 = [m - ln for ln in lens]
    sD, sU, sR = (m + 1) * bb, m * bb, (m + 1) * ba

    def orig(p, j):
        return j - j0[p] if p == 0 else n - 1 - (j - j0[p])

    exp_in, exp_out, exp_fill = [], [], []
    for f in range(1 + k):
        full = not diag
        for p in range(2):
            for j in range(j0[p]):
                if f == 0:
                    exp_fill.append((aid(K_LOC, 0, A_D), p * sD + j * bb, b))
            for j in range(j0[p], m):
                kk = orig(p, j)
                c = kk if p == 0 else kk - 1
                up, lo = (A_U, A_L) if p == 0 else (A_L, A_U)
                pairs = [(A_D, p * sD + j * bb, A_D, kk * bb, b, b), (A_U, p * sU + j * bb, up, c * bb, b, b),
                         (A_L, p * sU + j * bb, lo, c * bb, b, b)]
                if a > 0:
                    pairs += [(A_R, p * sR + j * ba, A_R, kk * ba, b, a), (A_B, p * sR + j * ba, A_B, kk * ba, a, b)]
                for (lk, loff, hk, hoff, rows, cols) in pairs:
                    exp_in.append((aid(K_LOC, f, lk), loff, aid(K_IN, f, hk), hoff, rows, cols))
                    if full or lk not in (A_U, A_L):
                        exp_out.append((aid(K_OUT, f, hk), hoff, aid(K_LOC_OUT, f, lk), loff, rows, cols))
        sig_out = [(A_D, sig * bb, b, b)]
        if a > 0:
            sig_out += [(A_R, sig * ba, b, a), (A_B, sig * ba, a, b), (A_T, 0, a, a)]
        for (kk, off, rows, cols) in sig_out:
            exp_out.append((aid(K_OUT, f, kk), off, aid(K_RED_OUT, f, kk), 0, rows, cols))

    def copies(lo, hi):
        got, fills = [], []
        for x in moves[lo:hi]:
            if x.fill == 1 and x.src[0] < 0:
                fills.append((x.dst, x.dst_off, x.rows))
                continue
            # one contiguous block, one source
            assert x.src[1] < 0 and x.src[2] < 0 and x.cnt[0] == 1
            assert x.ldd == x.cols and x.lds[0] == x.cols
            got.append((x.dst, x.dst_off, x.src[0], x.off[0], x.rows, x.cols))
        return sorted(got), sorted(fills)

    got_in, fills = copies(0, pe[0])
    assert got_in == sorted(exp_in)
    assert fills == sorted(exp_fill)
    got_out, fills3 = copies(pe[2], pe[3])
    assert got_out == sorted(exp_out) and not fills3
    # phase 1: the caller's inputs read are the separator's blocks and the tip, nothing else
    reads = set()
    for x in moves[pe[0]:pe[1]]:
        for s in range(3):
            if x.src[s] >= 0 and x.src[s] // (6 * MAXF) == K_IN:
                assert x.cnt[s] == 1
                reads.add((x.src[s], x.off[s], x.lds[s], x.rows, x.cols))
    exp_reads = set()
    for f in range(1 + k):
        exp_reads.add((aid(K_IN, f, A_D), sig * bb, b, b, b))
        if a > 0:
            exp_reads |= {(aid(K_IN, f, A_R), sig * ba, a, b, a), (aid(K_IN, f, A_B), sig * ba, b, a, b),
                          (aid(K_IN, f, A_T), 0, a, a, a)}
    assert reads == exp_reads
