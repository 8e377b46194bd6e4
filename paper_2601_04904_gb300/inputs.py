"""Seeded synthetic inputs for the BTA selected-inversion / quadratic-solve path.

This module only draws random numbers and lays them out on the block-tridiagonal
with arrowhead (BTA) pattern of Sec. II-A (n square diagonal blocks of size b,
arrow blocks of width a, tip a x a; N = n*b + a).  It contains none of the
method's arithmetic: no Schur complements, no inversions, no assembly of the
system matrix A from H.  Both the CPU oracle and the CUDA path are fed from the
arrays it returns.

Block container (a plain ``dict`` of complex128 numpy arrays, all row-major):

====== ================== ==========================================
key    shape              block
====== ================== ==========================================
diag   (n, b, b)          M_{i,i}
upper  (n-1, b, b)        M_{i,i+1}
lower  (n-1, b, b)        M_{i+1,i}
arrow_r (n, b, a)         M_{i,t}   (right arrow column)
arrow_b (n, a, b)         M_{t,i}   (bottom arrow row)
tip    (a, a)             M_{t,t}
====== ================== ==========================================

Recipe (the paper's datasets NR_3408 and SD of Table 6 are not available; these
synthetic matrices stand in for them):

* ``hamiltonian``: M has Re and Im i.i.d. N(0,1)/sqrt(b) on every pattern block,
  H = (M + M^H)/2 taken blockwise, so H is Hermitian and zero off the pattern.
* ``lesser_rhs``: C has Re and Im i.i.d. N(0,1) on every pattern block and
  B = C - C^H blockwise, so B is anti-Hermitian on the same pattern, as the
  lesser self-energy Sigma^< of Sec. I is.
* ``energy_grid``: energies uniform in [-1, 1] and the contact broadening
  gamma(E) = 0.5 + 0.3 E, which maps [-1, 1] onto [0.2, 0.8].
"""
from __future__ import annotations

import numpy as np

KEYS = ("diag", "upper", "lower", "arrow_r", "arrow_b", "tip")

# Base seed of every synthetic workload.
BASE_SEED = 20260104


def block_shapes(n: int, b: int, a: int) -> dict:
    """Shapes of the six block arrays of an (n, b, a) BTA matrix."""
    if n < 1 or b < 1 or a < 0:
        raise ValueError(f"invalid BTA shape n={n} b={b} a={a}")
    return {
        "diag": (n, b, b),
        "upper": (n - 1, b, b),
        "lower": (n - 1, b, b),
        "arrow_r": (n, b, a),
        "arrow_b": (n, a, b),
        "tip": (a, a),
    }


def zeros(n: int, b: int, a: int) -> dict:
    return {k: np.zeros(s, dtype=np.complex128) for k, s in block_shapes(n, b, a).items()}


def _cnormal(rng: np.random.Generator, shape, scale: float) -> np.ndarray:
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im) * scale


def _random_pattern(n: int, b: int, a: int, seed: int, scale: float) -> dict:
    rng = np.random.default_rng(seed)
    return {k: _cnormal(rng, s, scale) for k, s in block_shapes(n, b, a).items()}


def _conj_t(x: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(x, -1, -2))


def hamiltonian(n: int, b: int, a: int, seed: int = BASE_SEED) -> dict:
    """Hermitian H on the BTA pattern: H = (M + M^H)/2, M ~ CN(0,1)/sqrt(b)."""
    m = _random_pattern(n, b, a, seed, 1.0 / np.sqrt(b))
    h = {
        "diag": 0.5 * (m["diag"] + _conj_t(m["diag"])),
        "upper": 0.5 * (m["upper"] + _conj_t(m["lower"])),
        "arrow_r": 0.5 * (m["arrow_r"] + _conj_t(m["arrow_b"])),
        "tip": 0.5 * (m["tip"] + _conj_t(m["tip"])),
    }
    h["lower"] = _conj_t(h["upper"]).copy()
    h["arrow_b"] = _conj_t(h["arrow_r"]).copy()
    return {k: np.ascontiguousarray(h[k]) for k in KEYS}


def lesser_rhs(n: int, b: int, a: int, seed: int = BASE_SEED + 7) -> dict:
    """Anti-Hermitian B on the BTA pattern: B = C - C^H, C ~ CN(0,1)."""
    c = _random_pattern(n, b, a, seed, 1.0)
    bb = {
        "diag": c["diag"] - _conj_t(c["diag"]),
        "upper": c["upper"] - _conj_t(c["lower"]),
        "arrow_r": c["arrow_r"] - _conj_t(c["arrow_b"]),
        "tip": c["tip"] - _conj_t(c["tip"]),
    }
    bb["lower"] = -_conj_t(bb["upper"])
    bb["arrow_b"] = -_conj_t(bb["arrow_r"])
    return {k: np.ascontiguousarray(bb[k]) for k in KEYS}


def random_bta(n: int, b: int, a: int, seed: int, scale: float = 1.0) -> dict:
    """Unstructured complex BTA matrix (no symmetry), used for edge-case tests."""
    return _random_pattern(n, b, a, seed, scale)


def energy_grid(count: int, seed: int = BASE_SEED + 1):
    """Energies E ~ U[-1, 1] and contact broadenings gamma(E) = 0.5 + 0.3 E."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(-1.0, 1.0, size=count)
    return e, 0.5 + 0.3 * e


def workload(name: str) -> dict:
    """Named synthetic workloads (sizes of the five benchmark settings)."""
    table = {
        # single solve, small: n=8 blocks of 32, arrow 16
        "bta_n8_b32_a16": dict(n=8, b=32, a=16, E=0.3, eta=1e-3, gamma=0.5),
        # single solve at device scale: n=64 blocks of 512, arrow 256
        "bta_n64_b512_a256": dict(n=64, b=512, a=256, E=0.3, eta=1e-3, gamma=0.5),
        # energy batch: 256 points sharing H, n=32 blocks of 256, arrow 128
        "bta_n32_b256_a128_x256E": dict(n=32, b=256, a=128, eta=1e-3, points=256),
        # large single solve for the split-precision mode
        "bta_n128_b1024_a512": dict(n=128, b=1024, a=512, E=0.3, eta=1e-3, gamma=0.5),
    }
    return dict(table[name])


def _ragged_pattern(sizes, a: int, seed: int, scale) -> dict:
    """Lists of blocks with block i of size sizes[i]; scale(b_i, b_j) per block."""
    rng = np.random.default_rng(seed)
    n = len(sizes)
    return {"diag": [_cnormal(rng, (sizes[i], sizes[i]), scale(sizes[i], sizes[i])) for i in range(n)],
            "upper": [_cnormal(rng, (sizes[i], sizes[i + 1]), scale(sizes[i], sizes[i + 1])) for i in range(n - 1)],
            "lower": [_cnormal(rng, (sizes[i + 1], sizes[i]), scale(sizes[i + 1], sizes[i])) for i in range(n - 1)],
            "arrow_r": [_cnormal(rng, (sizes[i], a), scale(sizes[i], a)) for i in range(n)],
            "arrow_b": [_cnormal(rng, (a, sizes[i]), scale(a, sizes[i])) for i in range(n)],
            "tip": _cnormal(rng, (a, a), scale(a, a))}


def hamiltonian_sizes(sizes, a: int, seed: int = BASE_SEED) -> dict:
    """Hermitian H with non-uniform blocks (lists of blocks, block i of size
    sizes[i]): H = (M + M^H)/2 blockwise, M ~ CN(0,1)/sqrt(max b_i)."""
    s = 1.0 / np.sqrt(max(sizes))
    m = _ragged_pattern(list(sizes), a, seed, lambda r, c: s)
    h = {"diag": [0.5 * (x + _conj_t(x)) for x in m["diag"]],
         "upper": [0.5 * (u + _conj_t(l)) for u, l in zip(m["upper"], m["lower"])],
         "arrow_r": [0.5 * (r + _conj_t(bt)) for r, bt in zip(m["arrow_r"], m["arrow_b"])],
         "tip": 0.5 * (m["tip"] + _conj_t(m["tip"]))}
    h["lower"] = [_conj_t(u).copy() for u in h["upper"]]
    h["arrow_b"] = [_conj_t(r).copy() for r in h["arrow_r"]]
    return {k: ([np.ascontiguousarray(x) for x in h[k]] if isinstance(h[k], list) else np.ascontiguousarray(h[k]))
            for k in KEYS}


def lesser_rhs_sizes(sizes, a: int, seed: int = BASE_SEED + 7) -> dict:
    """Anti-Hermitian B with non-uniform blocks: B = C - C^H blockwise."""
    c = _ragged_pattern(list(sizes), a, seed, lambda r, cc: 1.0)
    out = {"diag": [x - _conj_t(x) for x in c["diag"]],
           "upper": [u - _conj_t(l) for u, l in zip(c["upper"], c["lower"])],
           "arrow_r": [r - _conj_t(bt) for r, bt in zip(c["arrow_r"], c["arrow_b"])],
           "tip": c["tip"] - _conj_t(c["tip"])}
    out["lower"] = [-_conj_t(u) for u in out["upper"]]
    out["arrow_b"] = [-_conj_t(r) for r in out["arrow_r"]]
    return {k: ([np.ascontiguousarray(x) for x in out[k]] if isinstance(out[k], list)
                else np.ascontiguousarray(out[k])) for k in KEYS}


def pack_sizes(m: dict) -> dict:
    """Lists of blocks -> one flat complex128 array per key (blocks one after
    the other, each row-major): the device layout of non-uniform matrices."""
    return {k: (np.concatenate([x.ravel() for x in m[k]]) if isinstance(m[k], list) and len(m[k])
                else (np.zeros(0, np.complex128) if isinstance(m[k], list) else m[k].ravel().copy()))
            for k in KEYS}


def unpack_sizes(flat: dict, sizes, a: int) -> dict:
    """Inverse of pack_sizes for block sizes `sizes` and arrow a."""
    n = len(sizes)
    shapes = {"diag": [(sizes[i], sizes[i]) for i in range(n)],
              "upper": [(sizes[i], sizes[i + 1]) for i in range(n - 1)],
              "lower": [(sizes[i + 1], sizes[i]) for i in range(n - 1)],
              "arrow_r": [(sizes[i], a) for i in range(n)], "arrow_b": [(a, sizes[i]) for i in range(n)]}
    out = {}
    for k, shp in shapes.items():
        v, o, blocks = np.asarray(flat[k]).ravel(), 0, []
        for r, c in shp:
            blocks.append(v[o:o + r * c].reshape(r, c))
            o += r * c
        out[k] = blocks
    out["tip"] = np.asarray(flat["tip"]).reshape(a, a)
    return out
