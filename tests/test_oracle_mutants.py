"""The oracle's pins have teeth: each plausible slip planted in a copy of the
oracle source (a dropped term, a flipped sign, a wrong index, a transposed or
unconjugated operand) must make the dense-definition pin fail.

Mistakes are planted only in an in-memory copy of ``oracle/rgf.py`` on the CPU.
"""
import importlib.util
import os
import types

import pytest

from conftest import make_problem
from oracle import dense
from paper_2601_04904_gb300.metrics import max_block_rel_err

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "rgf.py")

MUTANTS = [
    # forward SI
    ("Ad[i + 1] = Ad[i + 1] - T1A @ A[\"upper\"][i]", "Ad[i + 1] = Ad[i + 1] + T1A @ A[\"upper\"][i]"),
    ("Ar[i + 1] = Ar[i + 1] - T1A @ Ar[i]", "Ar[i + 1] = Ar[i + 1]"),
    ("Ab[i + 1] = Ab[i + 1] - Lt @ A[\"upper\"][i]", "Ab[i + 1] = Ab[i + 1] - Lt @ A[\"lower\"][i]"),
    ("Att = Att - Lt @ Ar[i]", "Att = Att - Lt @ Ar[i - 1]"),
    ("T1A = A[\"lower\"][i] @ SA[i]", "T1A = A[\"upper\"][i] @ SA[i]"),
    # forward SQ
    ("- B[\"lower\"][i] @ _h(T1A)\n", "- B[\"lower\"][i] @ T1A.T\n"),
    ("- T1A @ B[\"upper\"][i])", "+ T1A @ B[\"upper\"][i])"),
    ("- T1A @ Br[i]", "- T1A @ Br[i + 1]"),
    ("- Lt @ B[\"upper\"][i]", "- Lt @ B[\"lower\"][i]"),
    ("- Bb[i] @ _h(T1A))", ")"),
    ("- Lt @ Br[i] - Bb[i] @ _h(Lt)", "- Lt @ Br[i] - Bb[i] @ Lt.T"),
    ("SB[i] = SA[i] @ Bd[i] @ _h(SA[i])", "SB[i] = SA[i] @ Bd[i] @ SA[i].T"),
    ("f[\"SBtt\"] = f[\"Stt\"] @ Btt @ _h(f[\"Stt\"])", "f[\"SBtt\"] = f[\"Stt\"] @ Btt @ f[\"Stt\"]"),
    # backward SI
    ("X_Ri = -T2A @ S", "X_Ri = -S @ T2A.T.T if False else -T2A @ S.T"),
    ("X_iR = -T1A @ XR", "X_iR = T1A @ XR"),
    ("X_ii = S - T1A @ X_Ri", "X_ii = S - X_Ri.T @ T1A.T"),
    # backward SQ
    ("Y12 = S @ gam @ _h(XR) - SBi @ _h(T2A)", "Y12 = S @ gam @ _h(XR) + SBi @ _h(T2A)"),
    ("Y21 = XR @ rho @ _h(S) - T2A @ SBi", "Y21 = XR @ rho @ S.T - T2A @ SBi"),
    ("Y_iR = Y12 - T1A @ YR", "Y_iR = Y12 - T1A @ XR"),
    ("Y_Ri = Y21 - YR @ _h(T1A)", "Y_Ri = Y21 - YR @ T1A.T"),
    ("+ T1A @ YR @ _h(T1A)", ""),
    ("r = _cat_rows(A[\"lower\"][i], f[\"Ab\"][i])", "r = _cat_rows(A[\"lower\"][i], f[\"Ab\"][i + 1])"),
    ("gam = _cat_cols(B[\"upper\"][i], f[\"Br\"][i])", "gam = _cat_cols(B[\"lower\"][i], f[\"Br\"][i])"),
]


def _load_mutant(old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    mod = types.ModuleType("rgf_mutant")
    exec(compile(src.replace(old, new, 1), "rgf_mutant", "exec"), mod.__dict__)
    return mod


def _dense_pin_error(mod, n=5, b=4, a=3):
    _, A, B = make_problem(n, b, a, seed=3)
    dR, dL = dense.dense_solve(A, B)
    try:
        GR, GL = mod.selquad(A, B)
    except Exception:
        return float("inf")
    return max(max_block_rel_err(GR, dR), max_block_rel_err(GL, dL))


def test_unmutated_copy_passes():
    spec = importlib.util.spec_from_file_location("rgf_copy", SRC)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    assert _dense_pin_error(mod) < 1e-11


@pytest.mark.parametrize("old,new", MUTANTS)
def test_mutant_is_caught(old, new):
    assert _dense_pin_error(_load_mutant(old, new)) > 1e-6


# slips that only show with non-uniform blocks: the R = {i+1, t} split taken
# at b_i instead of b_{i+1}, or the next block's size read from the wrong array
RAGGED_MUTANTS = [
    ("k = A[\"upper\"][i].shape[1]  # b_{i+1}: the R = {i+1, t} split", "k = A[\"upper\"][i].shape[0]"),
    ("k = A[\"upper\"][i].shape[1]  # b_{i+1}: the R = {i+1, t} split", "k = f[\"SA\"][i].shape[0]"),
]


def _ragged_pin_error(mod):
    from paper_2601_04904_gb300 import inputs

    sizes, a = [3, 5, 2, 4], 2
    h = inputs.hamiltonian_sizes(sizes, a, seed=inputs.BASE_SEED + 90)
    B = inputs.lesser_rhs_sizes(sizes, a, seed=inputs.BASE_SEED + 91)
    A = mod.assemble_a(h, 0.3, 1e-3, 0.5)
    dR, dL = dense.dense_solve(A, B)
    try:
        GR, GL = mod.selquad(A, B)
        return max(max_block_rel_err(GR, dR), max_block_rel_err(GL, dL))
    except Exception:
        return float("inf")


def test_unmutated_copy_passes_ragged():
    spec = importlib.util.spec_from_file_location("rgf_copy2", SRC)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    assert _ragged_pin_error(mod) < 1e-11


@pytest.mark.parametrize("old,new", RAGGED_MUTANTS)
def test_ragged_mutant_is_caught(old, new):
    assert _ragged_pin_error(_load_mutant(old, new)) > 1e-6
