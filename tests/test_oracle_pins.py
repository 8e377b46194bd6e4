"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* dense definition (Alg. 4): G^R = A^{-1}, G^< = A^{-1} B A^{-H} on the pattern;
  the dense reference is itself pinned by its residuals A G = I, A X A^H = B;
* exact rational arithmetic (sympy) on tiny Gaussian-integer matrices;
* Usmani's continuant closed form for the inverse of a tridiagonal matrix
  (1x1-block chains, b = 1, a = 0);
* the exact inverse of tridiag(-1, 2, -1) (golden fixture) and its block
  Kronecker extension;
* n = 1, b = 1, a = 0: G = 1/A, G^< = B/|A|^2;
* the literal Alg. 1/2 (a = 0) as a second formula path;
* invariants that use only pattern blocks: (A G^R)_{ii} = I, (G^R A)_{ii} = I,
  (A G^R)_{i,t} = 0, (A G^R)_{tt} = I, (A G^<)_{ii} = (B G^{R H})_{ii}, and
  G^< anti-Hermitian when B is.
"""
import os

import numpy as np
import pytest

from conftest import make_problem
from oracle import dense, rgf
from paper_2601_04904_gb300 import inputs
from paper_2601_04904_gb300.metrics import max_block_rel_err

SHAPES = [(1, 1, 0), (2, 1, 0), (5, 1, 0), (4, 3, 0), (4, 3, 2), (8, 32, 16), (1, 4, 3),
          (6, 8, 0), (3, 5, 7), (2, 2, 1), (1, 1, 1), (7, 6, 9)]
TOL = 1e-11


@pytest.mark.parametrize("n,b,a", SHAPES)
def test_rgf_matches_dense_definition(n, b, a):
    _, A, B = make_problem(n, b, a)
    GR, GL = rgf.selquad(A, B)
    dR, dL = dense.dense_solve(A, B)
    assert max_block_rel_err(GR, dR) < TOL
    assert max_block_rel_err(GL, dL) < TOL
    # SI-only path gives the same G^R
    assert max_block_rel_err(rgf.selinv(A), dR) < TOL


@pytest.mark.parametrize("n,b,a", [(3, 4, 2), (5, 3, 0), (2, 6, 5)])
def test_rgf_unstructured_inputs(n, b, a):
    """No Hermitian structure at all: catches conj/transposition slips that a
    symmetric input could hide."""
    A = inputs.random_bta(n, b, a, seed=99)
    for i in range(n):
        A["diag"][i] += 4.0 * np.eye(b)
    if a:
        A["tip"] += 4.0 * np.eye(a)
    B = inputs.random_bta(n, b, a, seed=100)
    GR, GL = rgf.selquad(A, B)
    dR, dL = dense.dense_solve(A, B)
    assert max_block_rel_err(GR, dR) < TOL
    assert max_block_rel_err(GL, dL) < TOL


@pytest.mark.parametrize("n,b,a", [(4, 3, 2), (3, 2, 0), (8, 32, 16)])
def test_dense_reference_residuals(n, b, a):
    """The dense reference itself satisfies A G = I and A X A^H = B on the full
    matrix (small N), so it is not trusted on faith."""
    _, A, B = make_problem(n, b, a)
    Ad, Bd = dense.to_dense(A), dense.to_dense(B)
    N = Ad.shape[0]
    import scipy.linalg as sla
    lu = sla.lu_factor(Ad)
    G = sla.lu_solve(lu, np.eye(N))
    X = G @ Bd @ np.conj(G.T)
    assert np.linalg.norm(Ad @ G - np.eye(N)) < 1e-12 * N
    assert np.linalg.norm(Ad @ X @ np.conj(Ad.T) - Bd) < 1e-12 * np.linalg.norm(Bd)
    GR, GL = dense.dense_solve(A, B)
    assert max_block_rel_err(GR, dense.from_dense(G, n, b, a)) < 1e-13
    assert max_block_rel_err(GL, dense.from_dense(X, n, b, a)) < 1e-12


def _gaussian_int_bta(n, b, a, seed, dominant):
    r = np.random.default_rng(seed)
    m = {}
    for k, s in inputs.block_shapes(n, b, a).items():
        m[k] = (r.integers(-3, 4, size=s) + 1j * r.integers(-3, 4, size=s)).astype(complex)
    if dominant:
        for i in range(n):
            m["diag"][i] += 20 * np.eye(b)
        if a:
            m["tip"] += 20 * np.eye(a)
    return m


@pytest.mark.parametrize("n,b,a", [(2, 2, 1), (3, 1, 2), (1, 2, 2), (3, 2, 0)])
def test_exact_rational(n, b, a):
    """Exact G and G^< by rational arithmetic on Gaussian-integer matrices."""
    sympy = pytest.importorskip("sympy")
    A = _gaussian_int_bta(n, b, a, seed=7 + n, dominant=True)
    B = _gaussian_int_bta(n, b, a, seed=17 + n, dominant=False)
    to_sym = lambda d: sympy.Matrix([[sympy.Integer(int(z.real)) + sympy.I * sympy.Integer(int(z.imag))
                                      for z in row] for row in d])
    As, Bs = to_sym(dense.to_dense(A)), to_sym(dense.to_dense(B))
    Gs = As.inv()
    Xs = Gs * Bs * Gs.H
    to_np = lambda M: np.array([[complex(sympy.N(M[i, j], 30)) for j in range(M.shape[1])]
                                for i in range(M.shape[0])])
    G_exact = dense.from_dense(to_np(Gs), n, b, a)
    X_exact = dense.from_dense(to_np(Xs), n, b, a)
    GR, GL = rgf.selquad(A, B)
    assert max_block_rel_err(GR, G_exact) < 1e-14
    assert max_block_rel_err(GL, X_exact) < 1e-13


def _usmani_inverse(diag, sup, sub):
    """Usmani (1994): inverse of a tridiagonal matrix from the continuants
    theta (leading) and phi (trailing)."""
    n = len(diag)
    th = np.zeros(n + 1, complex)
    th[0] = 1
    th[1] = diag[0]
    for i in range(2, n + 1):
        th[i] = diag[i - 1] * th[i - 1] - sup[i - 2] * sub[i - 2] * th[i - 2]
    ph = np.zeros(n + 2, complex)
    ph[n + 1] = 1
    ph[n] = diag[n - 1]
    for i in range(n - 1, 0, -1):
        ph[i] = diag[i - 1] * ph[i + 1] - sup[i - 1] * sub[i - 1] * ph[i + 2]
    G = np.zeros((n, n), complex)
    for i in range(1, n + 1):
        for j in range(1, n + 1):
            if i == j:
                G[i - 1, j - 1] = th[i - 1] * ph[j + 1] / th[n]
            elif i < j:
                G[i - 1, j - 1] = ((-1) ** (i + j) * np.prod(sup[i - 1:j - 1])
                                   * th[i - 1] * ph[j + 1] / th[n])
            else:
                G[i - 1, j - 1] = ((-1) ** (i + j) * np.prod(sub[j - 1:i - 1])
                                   * th[j - 1] * ph[i + 1] / th[n])
    return G


@pytest.mark.parametrize("n", [1, 2, 3, 6, 11])
def test_usmani_chain(n):
    _, A, B = make_problem(n, 1, 0, seed=n)
    G = _usmani_inverse(A["diag"][:, 0, 0], A["upper"][:, 0, 0], A["lower"][:, 0, 0])
    X = G @ dense.to_dense(B) @ np.conj(G.T)
    GR, GL = rgf.selquad(A, B)
    assert max_block_rel_err(GR, dense.from_dense(G, n, 1, 0)) < 1e-12
    assert max_block_rel_err(GL, dense.from_dense(X, n, 1, 0)) < 1e-12


def _golden_laplacian():
    path = os.path.join(os.path.dirname(__file__), "golden", "laplacian_chain_inverse_n4.txt")
    rows = [list(map(float, ln.split())) for ln in open(path) if ln.strip() and not ln.startswith("#")]
    return np.array(rows) / 5.0


@pytest.mark.parametrize("b", [1, 3])
def test_laplacian_chain_golden(b):
    Tinv = _golden_laplacian()
    n = Tinv.shape[0]
    A = inputs.zeros(n, b, 0)
    A["diag"][:] = 2 * np.eye(b)
    A["upper"][:] = -np.eye(b)
    A["lower"][:] = -np.eye(b)
    expect = dense.from_dense(np.kron(Tinv, np.eye(b)).astype(complex), n, b, 0)
    assert max_block_rel_err(rgf.selinv(A), expect) < 1e-15


def test_scalar_case():
    A = inputs.zeros(1, 1, 0)
    B = inputs.zeros(1, 1, 0)
    A["diag"][0, 0, 0] = 0.3 - 2.0j
    B["diag"][0, 0, 0] = 1.5j
    GR, GL = rgf.selquad(A, B)
    assert abs(GR["diag"][0, 0, 0] - 1 / (0.3 - 2.0j)) < 1e-16
    assert abs(GL["diag"][0, 0, 0] - 1.5j / abs(0.3 - 2.0j) ** 2) < 1e-16


@pytest.mark.parametrize("n,b", [(2, 1), (5, 4), (6, 8)])
def test_printed_alg_equals_bta_form(n, b):
    _, A, B = make_problem(n, b, 0)
    pR, pL = rgf.rgf_bt_printed(A, B)
    GR, GL = rgf.selquad(A, B)
    assert max_block_rel_err(GR, pR) < 1e-12
    assert max_block_rel_err(GL, pL) < 1e-12


def _mm(x, y):
    return x @ y


@pytest.mark.parametrize("n,b,a", [(6, 5, 3), (8, 32, 16), (3, 4, 0)])
def test_pattern_invariants(n, b, a):
    _, A, B = make_problem(n, b, a)
    G, X = rgf.selquad(A, B)
    I_b = np.eye(b)
    for i in range(n):
        ag = A["diag"][i] @ G["diag"][i] + A["arrow_r"][i] @ G["arrow_b"][i]
        ga = G["diag"][i] @ A["diag"][i] + G["arrow_r"][i] @ A["arrow_b"][i]
        ait = A["diag"][i] @ G["arrow_r"][i] + A["arrow_r"][i] @ G["tip"]
        ax = A["diag"][i] @ X["diag"][i] + A["arrow_r"][i] @ X["arrow_b"][i]
        bg = B["diag"][i] @ np.conj(G["diag"][i].T) + B["arrow_r"][i] @ np.conj(G["arrow_r"][i].T)
        if i > 0:
            ag += A["lower"][i - 1] @ G["upper"][i - 1]
            ga += G["lower"][i - 1] @ A["upper"][i - 1]
            ait += A["lower"][i - 1] @ G["arrow_r"][i - 1]
            ax += A["lower"][i - 1] @ X["upper"][i - 1]
            bg += B["lower"][i - 1] @ np.conj(G["lower"][i - 1].T)
        if i < n - 1:
            ag += A["upper"][i] @ G["lower"][i]
            ga += G["upper"][i] @ A["lower"][i]
            ait += A["upper"][i] @ G["arrow_r"][i + 1]
            ax += A["upper"][i] @ X["lower"][i]
            bg += B["upper"][i] @ np.conj(G["upper"][i].T)
        assert np.linalg.norm(ag - I_b) < 1e-12
        assert np.linalg.norm(ga - I_b) < 1e-12
        assert np.linalg.norm(ait) < 1e-12
        assert np.linalg.norm(ax - bg) < 1e-11 * max(1.0, np.linalg.norm(bg))
    if a:
        att = A["tip"] @ G["tip"] + sum(A["arrow_b"][i] @ G["arrow_r"][i] for i in range(n))
        assert np.linalg.norm(att - np.eye(a)) < 1e-12
    # G^< is anti-Hermitian because B is
    h = lambda z: np.conj(np.swapaxes(z, -1, -2))
    assert np.abs(X["diag"] + h(X["diag"])).max() < 1e-11 * np.abs(X["diag"]).max()
    assert np.abs(X["upper"] + h(X["lower"])).max() < 1e-11 * np.abs(X["upper"]).max()
    if a:
        assert np.abs(X["arrow_r"] + h(X["arrow_b"])).max() < 1e-11 * np.abs(X["arrow_r"]).max()
        assert np.abs(X["tip"] + h(X["tip"])).max() < 1e-11 * np.abs(X["tip"]).max()


def test_assembly_definition():
    """A = (E + i eta) I - H - Sigma^R with Sigma^R = -i gamma I on blocks 0, n-1."""
    n, b, a = 4, 3, 2
    h = inputs.hamiltonian(n, b, a)
    A = rgf.assemble_a(h, 0.25, 0.01, 0.4)
    Hd, Ad = dense.to_dense(h), dense.to_dense(A)
    sig = np.zeros(n * b + a, complex)
    sig[:b] = -0.4j
    sig[(n - 1) * b:n * b] = -0.4j
    expect = (0.25 + 0.01j) * np.eye(n * b + a) - Hd - np.diag(sig)
    assert np.array_equal(Ad, expect)
    # single block: contact self-energy applied once
    h1 = inputs.hamiltonian(1, 2, 0)
    A1 = rgf.assemble_a(h1, 0.0, 0.0, 0.5)
    assert np.allclose(np.diag(A1["diag"][0]), -np.diag(h1["diag"][0]) + 0.5j)


def test_rgf_matches_dense_definition_random_shapes():
    """The oracle's sweep against the dense definition (Alg. 4) over random
    shapes and unstructured inputs (hypothesis): 1-7 blocks of 1-5, arrow 0-4,
    with and without Hermitian structure."""
    pytest.importorskip("hypothesis")
    from hypothesis import given, settings
    from hypothesis import strategies as st

    @settings(max_examples=60, deadline=None)
    @given(st.integers(1, 7), st.integers(1, 5), st.integers(0, 4), st.booleans(), st.integers(0, 10 ** 6))
    def check(n, b, a, structured, seed):
        if structured:
            _, A, B = make_problem(n, b, a, seed=seed % 1000, eta=0.1)
        else:
            A = inputs.random_bta(n, b, a, seed=seed)
            for i in range(n):
                A["diag"][i] += 4.0 * np.eye(b)
            if a:
                A["tip"] += 4.0 * np.eye(a)
            B = inputs.random_bta(n, b, a, seed=seed + 1)
        GR, GL = rgf.selquad(A, B)
        dR, dL = dense.dense_solve(A, B)
        assert max_block_rel_err(GR, dR) < TOL
        assert max_block_rel_err(GL, dL) < TOL

    check()
