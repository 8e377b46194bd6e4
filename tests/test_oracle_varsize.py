"""Pins of the oracle on non-uniform block sizes (block i of size b_i; the BTA
pattern of Sec. II-A does not need equal blocks).

* against the dense definition (Alg. 4) on ragged block sizes, with and without
  an arrow, for G^R and G^<;
* against the dense definition on unstructured (non-Hermitian) ragged inputs,
  which catch transposition or conjugation slips;
* the dense reference's own residuals A G = I and A X A^H = B;
* uniform sizes given as lists of blocks reproduce the stacked-array oracle
  bit for bit (the generalisation only changes how blocks are held);
* G^< anti-Hermitian when B is."""
import numpy as np
import pytest

from oracle import dense, rgf
from paper_2601_04904_gb300 import inputs
from paper_2601_04904_gb300.metrics import max_block_rel_err

TOL = 1e-11
SIZES = [([3, 5, 2, 4], 3), ([1, 4, 1], 0), ([6], 2), ([2, 3], 5), ([7, 3, 5, 2, 8, 4], 4), ([1, 1, 9, 1], 2),
         ([5, 4, 3, 2, 1], 0)]


def _problem(sizes, a, seed=0):
    h = inputs.hamiltonian_sizes(sizes, a, seed=inputs.BASE_SEED + 40 + seed)
    B = inputs.lesser_rhs_sizes(sizes, a, seed=inputs.BASE_SEED + 50 + seed)
    return rgf.assemble_a(h, 0.3, 1e-3, 0.5), B


@pytest.mark.parametrize("sizes,a", SIZES)
def test_ragged_rgf_matches_dense(sizes, a):
    A, B = _problem(sizes, a)
    GR, GL = rgf.selquad(A, B)
    dR, dL = dense.dense_solve(A, B)
    assert max_block_rel_err(GR, dR) < TOL
    assert max_block_rel_err(GL, dL) < TOL
    assert max_block_rel_err(rgf.selinv(A), dR) < TOL
    for i, s in enumerate(sizes):
        assert GR["diag"][i].shape == (s, s) and GL["arrow_r"][i].shape == (s, a)


@pytest.mark.parametrize("sizes,a", [([3, 5, 2], 2), ([4, 1, 6, 2], 0)])
def test_ragged_unstructured_inputs(sizes, a):
    rng = np.random.default_rng(7)
    cn = lambda r, c: rng.standard_normal((r, c)) + 1j * rng.standard_normal((r, c))
    n = len(sizes)

    def rand():
        return {"diag": [cn(s, s) + 4.0 * np.eye(s) for s in sizes],
                "upper": [cn(sizes[i], sizes[i + 1]) for i in range(n - 1)],
                "lower": [cn(sizes[i + 1], sizes[i]) for i in range(n - 1)],
                "arrow_r": [cn(s, a) for s in sizes], "arrow_b": [cn(a, s) for s in sizes],
                "tip": cn(a, a) + 4.0 * np.eye(a)}
    A, B = rand(), rand()
    GR, GL = rgf.selquad(A, B)
    dR, dL = dense.dense_solve(A, B)
    assert max_block_rel_err(GR, dR) < TOL
    assert max_block_rel_err(GL, dL) < TOL


def test_ragged_dense_reference_residuals():
    sizes, a = [3, 5, 2, 4], 3
    A, B = _problem(sizes, a, seed=1)
    Ad, Bd = dense.to_dense(A), dense.to_dense(B)
    N = Ad.shape[0]
    assert N == sum(sizes) + a
    G = np.linalg.inv(Ad)
    X = G @ Bd @ G.conj().T
    assert np.linalg.norm(Ad @ G - np.eye(N)) < 1e-10
    assert np.linalg.norm(Ad @ X @ Ad.conj().T - Bd) < 1e-9 * np.linalg.norm(Bd)
    dR, dL = dense.dense_solve(A, B)
    got = dense.from_dense_sizes(G, sizes, a)
    assert max_block_rel_err(dR, got) < 1e-12


def test_uniform_sizes_as_lists_equal_stacked_oracle():
    n, b, a = 5, 4, 3
    h = inputs.hamiltonian(n, b, a, seed=inputs.BASE_SEED + 61)
    B = inputs.lesser_rhs(n, b, a, seed=inputs.BASE_SEED + 62)
    A = rgf.assemble_a(h, 0.3, 1e-3, 0.5)
    as_list = lambda m: {k: (list(v) if v.ndim == 3 else v) for k, v in m.items()}
    R1, L1 = rgf.selquad(A, B)
    R2, L2 = rgf.selquad(as_list(A), as_list(B))
    for X1, X2 in ((R1, R2), (L1, L2)):
        for k in X1:
            got = X2[k] if not isinstance(X2[k], list) else (np.stack(X2[k]) if X2[k] else np.zeros_like(X1[k]))
            assert np.array_equal(X1[k], got), k


def test_ragged_lesser_is_antihermitian():
    sizes, a = [4, 2, 6, 3], 2
    A, B = _problem(sizes, a, seed=2)
    _, GL = rgf.selquad(A, B)
    H = lambda x: np.conj(x.T)
    for i in range(len(sizes)):
        assert np.allclose(GL["diag"][i], -H(GL["diag"][i]), atol=1e-10 * np.linalg.norm(GL["diag"][i]))
        assert np.allclose(GL["arrow_r"][i], -H(GL["arrow_b"][i]), atol=1e-10 * max(1, np.linalg.norm(GL["arrow_r"][i])))
    for i in range(len(sizes) - 1):
        assert np.allclose(GL["upper"][i], -H(GL["lower"][i]), atol=1e-10 * np.linalg.norm(GL["upper"][i]))


def test_pack_unpack_roundtrip():
    sizes, a = [3, 1, 4], 2
    h = inputs.hamiltonian_sizes(sizes, a, seed=3)
    flat = inputs.pack_sizes(h)
    assert flat["diag"].size == sum(s * s for s in sizes)
    assert flat["upper"].size == 3 * 1 + 1 * 4
    back = inputs.unpack_sizes(flat, sizes, a)
    for k in inputs.KEYS:
        if isinstance(h[k], list):
            for x, y in zip(h[k], back[k]):
                assert np.array_equal(x, y)
        else:
            assert np.array_equal(h[k], back[k])
