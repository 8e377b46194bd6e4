"""GPU parity of the partitioned solve (qsi_bta_solve_partitioned; Sec. III-B
run on one GPU, the partitions as batch entries of the sweeps) against the
oracle's unpartitioned solve.

The 1e-10 bar applies at broadening eta = 0.1.  At the recipe's eta = 1e-3 the
partitions' interior pivots lack the contact self-energy.  Their conditioning
kappa then bounds the error at 1e-13 * kappa^2 (see test_partition_plan)."""
import numpy as np
import pytest

from conftest import make_problem
from oracle import rgf
from paper_2601_04904_gb300 import inputs
from paper_2601_04904_gb300.metrics import max_block_rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-10
# checked partition count: general partitions only while 1e-13 kappa_F^2 <= 1e-10
KAPPA_LIMIT = (1e-10 / 1e-13) ** 0.5
DIAG_KEYS = ("diag", "arrow_r", "arrow_b", "tip")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04904_gb300 import qsi

    return torch, qsi


def _solve(qsi, ctx, A, Bs, P, prec, diag_only=False):
    n, b, a = rgf.shape_of(A)
    GR = qsi.device_zeros(n, b, a, off_diagonal=not diag_only)
    GX = [qsi.device_zeros(n, b, a, off_diagonal=not diag_only) for _ in Bs]
    ctx.solve_partitioned(qsi.to_device(A), [qsi.to_device(B) for B in Bs], P, GR, GX, prec)
    ctx.synchronize()
    return GR, GX


def _host(qsi, m):
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in m.items()}


@pytest.mark.parametrize("prec_name", ["FP64", "FP64_EMU"])
@pytest.mark.parametrize("n,b,a,P,k", [(9, 16, 8, 3, 1), (10, 32, 0, 3, 1), (17, 24, 12, 5, 2), (7, 40, 16, 4, 1),
                                       (12, 64, 32, 2, 1), (31, 48, 20, 4, 0), (40, 16, 72, 8, 1)])
def test_partitioned_matches_oracle(env, prec_name, n, b, a, P, k):
    torch, qsi = env
    _, A, B = make_problem(n, b, a, seed=80 + n, eta=0.1)
    Bs = ([B] + [inputs.lesser_rhs(n, b, a, seed=inputs.BASE_SEED + 600 + r) for r in range(1, k)])[:k]
    ctx = qsi.Context(0)
    GR, GX = _solve(qsi, ctx, A, Bs, P, getattr(qsi, prec_name))
    assert max_block_rel_err(_host(qsi, GR), rgf.selinv(A)) < TOL
    for r in range(k):
        assert max_block_rel_err(_host(qsi, GX[r]), rgf.selquad(A, Bs[r])[1]) < TOL, r
    ctx.close()


@pytest.mark.parametrize("prec_name", ["FP64", "FP64_EMU"])
@pytest.mark.parametrize("n,b,a,P,seed", [(64, 32, 16, 8, 3), (30, 24, 8, 5, 90), (14, 40, 0, 3, 1)])
def test_partitioned_recipe_broadening_vs_oracle(env, prec_name, n, b, a, P, seed):
    """The recipe's broadening eta = 1e-3 against the oracle's unpartitioned
    solve: every block within 1e-13 * kappa^2, kappa the largest condition
    number of the partitions' pivots (formed by the library's plan in numpy),
    the bound the elimination's conditioning gives (G^< carries two factors of
    every pivot)."""
    torch, qsi = env
    from test_partition_plan import partition_pivot_kappa

    _, A, B = make_problem(n, b, a, seed=seed)
    ctx = qsi.Context(0)
    GR, GX = _solve(qsi, ctx, A, [B], P, getattr(qsi, prec_name))
    ref_R, ref_L = rgf.selquad(A, B)
    kappa = partition_pivot_kappa(A, P)
    bound = 1e-13 * kappa ** 2
    eR, eL = max_block_rel_err(_host(qsi, GR), ref_R), max_block_rel_err(_host(qsi, GX[0]), ref_L)
    print(f"partitioned eta=1e-3 ({n},{b},{a}) P={P}: kappa {kappa:.3g} bound {bound:.3g} G^R {eR:.3g} G^< {eL:.3g}")
    assert eR < bound and eL < bound
    ctx.close()


def test_partitioned_recipe_broadening_within_conditioning_bound(env):
    torch, qsi = env
    from test_partition_plan import partitioned_solve  # the same plan run in numpy, for the pivots' conditioning

    n, b, a, P = 64, 32, 16, 8
    _, A, B = make_problem(n, b, a, seed=3)
    ctx = qsi.Context(0)
    GR, GX = _solve(qsi, ctx, A, [B], P, qsi.FP64)
    ref_R, ref_L = rgf.selquad(A, B)
    # kappa of the partitions' pivots: the inverses the numpy run of the plan forms
    res, plan = partitioned_solve(A, [B], P)
    e_np = max(max_block_rel_err(res[0], ref_R), max_block_rel_err(res[1], ref_L))
    e_gpu = max(max_block_rel_err(_host(qsi, GR), ref_R), max_block_rel_err(_host(qsi, GX[0]), ref_L))
    # the GPU result is as accurate as the same elimination in numpy (both bounded by the conditioning)
    assert e_gpu < max(10 * e_np, 1e-12)
    ctx.close()


def test_partitioned_diagonal_only_and_single_partition(env):
    torch, qsi = env
    n, b, a, P = 13, 24, 8, 3
    _, A, B = make_problem(n, b, a, seed=90, eta=0.1)
    ctx = qsi.Context(0)
    GRf, GXf = _solve(qsi, ctx, A, [B], P, qsi.FP64_EMU)
    GRd, GXd = _solve(qsi, ctx, A, [B], P, qsi.FP64_EMU, diag_only=True)
    for key in DIAG_KEYS:
        assert np.array_equal(GRd[key].cpu().numpy(), GRf[key].cpu().numpy()), key
        assert np.array_equal(GXd[0][key].cpu().numpy(), GXf[0][key].cpu().numpy()), key
    # P = 1 is the plain solve: the same bits as qsi_bta_solve
    G1, X1 = _solve(qsi, ctx, A, [B], 1, qsi.FP64_EMU)
    G0, X0 = ctx.solve(qsi.to_device(A), [qsi.to_device(B)], precision=qsi.FP64_EMU)
    ctx.synchronize()
    for key in qsi.KEYS:
        assert np.array_equal(G1[key].cpu().numpy(), G0[key].cpu().numpy()), key
        assert np.array_equal(X1[0][key].cpu().numpy(), X0[0][key].cpu().numpy()), key
    ctx.close()


def test_partitioned_repeat_bitwise_and_argument_errors(env):
    torch, qsi = env
    n, b, a = 9, 16, 8
    _, A, B = make_problem(n, b, a, seed=91, eta=0.1)
    ctx = qsi.Context(0)
    R1, X1 = _solve(qsi, ctx, A, [B], 4, qsi.FP64)
    R2, X2 = _solve(qsi, ctx, A, [B], 4, qsi.FP64)
    for key in qsi.KEYS:
        assert np.array_equal(R1[key].cpu().numpy(), R2[key].cpu().numpy()), key
        assert np.array_equal(X1[0][key].cpu().numpy(), X2[0][key].cpu().numpy()), key
    # partitions = 0: the twisted split, the bits of P = 2; partitions = -1:
    # round(sqrt(9)) = 3 partitions, whose pivots at eta = 0.1 exceed the
    # conditioning limit, so the twisted split's bits too
    from test_partition_plan import partition_pivot_kappa

    assert partition_pivot_kappa(A, 3, frobenius=True) > KAPPA_LIMIT
    R2, X2 = _solve(qsi, ctx, A, [B], 2, qsi.FP64)
    for P in (0, -1):
        RA, XA = _solve(qsi, ctx, A, [B], P, qsi.FP64)
        for key in qsi.KEYS:
            assert np.array_equal(RA[key].cpu().numpy(), R2[key].cpu().numpy()), (P, key)
            assert np.array_equal(XA[0][key].cpu().numpy(), X2[0][key].cpu().numpy()), (P, key)
    for P in (-2, 6):  # (n + 1) / 2 = 5 partitions at most
        with pytest.raises(qsi.QsiError) as ei:
            _solve(qsi, ctx, A, [B], P, qsi.FP64)
        assert ei.value.status == qsi.ERR_ARG
    ctx.close()


def test_partitioned_mixed_precision(env):
    torch, qsi = env
    n, b, a, P = 17, 64, 32, 4
    _, A, B = make_problem(n, b, a, seed=92, eta=0.1)
    ctx = qsi.Context(0)
    GR, GX = _solve(qsi, ctx, A, [B], P, qsi.MIXED)
    assert max_block_rel_err(_host(qsi, GR), rgf.selinv(A)) < 1e-6
    assert max_block_rel_err(_host(qsi, GX[0]), rgf.selquad(A, B)[1]) < 1e-6
    ctx.close()


def test_partitioned_graph_replays_match_direct(env):
    """On a stream context the partitioned run is captured once and replayed;
    every replay (also after the inputs changed in place) is bitwise equal to
    the direct run on the legacy default stream."""
    torch, qsi = env
    n, b, a, P = 21, 32, 16, 4
    _, A, B = make_problem(n, b, a, seed=93, eta=0.1)
    stream = torch.cuda.Stream()
    ctx = qsi.Context(0, stream=stream)
    ctx0 = qsi.Context(0)
    Ad, Bd = qsi.to_device(A), qsi.to_device(B)
    GR, GX = qsi.device_zeros(n, b, a), [qsi.device_zeros(n, b, a)]
    torch.cuda.synchronize()
    for call in range(3):
        if call == 2:
            _, A2, _ = make_problem(n, b, a, seed=94, eta=0.1)
            Ad["diag"].copy_(torch.from_numpy(A2["diag"]).to(Ad["diag"].device))
            Bd["tip"].mul_(0.5)
            torch.cuda.synchronize()
        ctx.solve_partitioned(Ad, [Bd], P, GR, GX, qsi.FP64_EMU)
        ctx.synchronize()
        R0, X0 = ctx0.solve_partitioned(Ad, [Bd], P, precision=qsi.FP64_EMU)
        ctx0.synchronize()
        for key in qsi.KEYS:
            assert np.array_equal(GR[key].cpu().numpy(), R0[key].cpu().numpy()), (call, key)
            assert np.array_equal(GX[0][key].cpu().numpy(), X0[0][key].cpu().numpy()), (call, key)
    Ah, Bh = qsi.to_host(Ad), qsi.to_host(Bd)
    assert max_block_rel_err(qsi.to_host(GR), rgf.selinv(Ah)) < TOL
    assert max_block_rel_err(qsi.to_host(GX[0]), rgf.selquad(Ah, Bh)[1]) < TOL
    ctx.close()
    ctx0.close()


@pytest.mark.parametrize("prec_name", ["FP64", "FP64_EMU"])
@pytest.mark.parametrize("graph", [False, True])
def test_partitioned_checked_choice(env, prec_name, graph):
    """partitions = -1 (Sec. III-B with the conditioning rule): round(sqrt(16))
    = 4 partitions when the largest kappa_F of their pivots keeps 1e-13
    kappa_F^2 within 1e-10 (eta = 2: the explicit P = 4 bits), the twisted
    split otherwise (the recipe's eta = 1e-3: the bits of P = 2).  The device
    estimate equals the plan's pivots' kappa_F formed in numpy; both results
    match the oracle at 1e-10.  On a stream context the checked run is two
    replayed graphs."""
    torch, qsi = env
    from test_partition_plan import partition_pivot_kappa

    n, b, a, P = 16, 8, 4, 4
    prec = getattr(qsi, prec_name)
    stream = torch.cuda.Stream() if graph else None
    ctx = qsi.Context(0, stream=stream)
    for eta, keep in ((2.0, True), (1e-3, False)):
        _, A, B = make_problem(n, b, a, seed=2, eta=eta)
        kf = partition_pivot_kappa(A, P, frobenius=True)
        assert (kf <= KAPPA_LIMIT) == keep, kf
        Ad, Bd = qsi.to_device(A), [qsi.to_device(B)]
        GR, GX = qsi.device_zeros(n, b, a), [qsi.device_zeros(n, b, a)]
        ER, EX = qsi.device_zeros(n, b, a), [qsi.device_zeros(n, b, a)]
        torch.cuda.synchronize()
        ctx.solve_partitioned(Ad, Bd, P if keep else 2, ER, EX, prec)
        ctx.synchronize()
        expect = (qsi.to_host(ER), qsi.to_host(EX[0]))
        st0 = ctx.stats()
        reps = 3 if graph else 1
        for _ in range(reps):
            ctx.solve_partitioned(Ad, Bd, -1, GR, GX, prec)
            ctx.synchronize()
            got = (qsi.to_host(GR), qsi.to_host(GX[0]))
            for key in qsi.KEYS:
                assert np.array_equal(got[0][key], expect[0][key]), (eta, key)
                assert np.array_equal(got[1][key], expect[1][key]), (eta, key)
        st1 = ctx.stats()
        assert abs(st1["partition_kappa"] - kf) <= 1e-6 * kf, (st1["partition_kappa"], kf)
        assert st1["partition_fallbacks"] - st0["partition_fallbacks"] == (0 if keep else reps)
        if graph and keep:  # the first call runs directly; each later one replays both stages
            assert st1["graph_launches"] - st0["graph_launches"] == 2 * (reps - 1)
        ref_R, ref_L = rgf.selquad(A, B)
        assert max_block_rel_err(got[0], ref_R) < TOL and max_block_rel_err(got[1], ref_L) < TOL
    ctx.close()


@pytest.mark.parametrize("prec_name", ["FP64", "FP64_EMU"])
@pytest.mark.parametrize("n,b,a,k,seed", [(64, 32, 16, 1, 3), (31, 48, 20, 2, 7), (14, 40, 0, 1, 1), (9, 16, 8, 1, 5)])
def test_twisted_split_at_recipe_broadening(env, prec_name, n, b, a, k, seed):
    """partitions = 2 is the twisted split (the top interior eliminated from
    block 0 down, the bottom one from block n-1 up, meeting at one separator):
    its pivots are the plain sweep's own Schur complements from either contact,
    so at the recipe's eta = 1e-3 it matches the oracle's dense definition
    (Alg. 4) at 1e-10 where the general partitions do not."""
    torch, qsi = env
    from oracle.dense import dense_solve

    _, A, B = make_problem(n, b, a, seed=seed)
    Bs = ([B] + [inputs.lesser_rhs(n, b, a, seed=inputs.BASE_SEED + 800 + r) for r in range(1, k)])[:k]
    ctx = qsi.Context(0)
    GR, GX = _solve(qsi, ctx, A, Bs, 2, getattr(qsi, prec_name))
    assert max_block_rel_err(_host(qsi, GR), dense_solve(A)[0]) < TOL
    for r in range(k):
        assert max_block_rel_err(_host(qsi, GX[r]), dense_solve(A, Bs[r])[1]) < TOL, r
    ctx.close()
