"""The per-block error measure used by every parity test and the bench."""
import numpy as np

from paper_2601_04904_gb300.metrics import max_block_rel_err


def _pair(n=3, b=2, a=1, seed=0):
    rng = np.random.default_rng(seed)
    c = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    ref = {"diag": c(n, b, b), "upper": c(n - 1, b, b), "lower": c(n - 1, b, b), "arrow_r": c(n, b, a),
           "arrow_b": c(n, a, b), "tip": c(a, a)}
    return {k: v.copy() for k, v in ref.items()}, ref


def test_error_of_a_perturbed_block():
    x, ref = _pair()
    x["upper"][1] += 1e-7 * ref["upper"][1]
    assert abs(max_block_rel_err(x, ref) - 1e-7) < 1e-15
    assert max_block_rel_err(ref, ref) == 0.0


def test_non_finite_output_is_an_infinite_error():
    # a NaN must not read as zero error (Python's max drops it)
    for bad in (np.nan, np.inf):
        x, ref = _pair()
        x["lower"][0][1, 0] = bad
        assert max_block_rel_err(x, ref) == float("inf")
        x, ref = _pair()
        x["tip"][0, 0] = complex(0.0, bad)
        assert max_block_rel_err(x, ref) == float("inf")
