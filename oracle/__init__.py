"""CPU oracle for selected inversion (SI) and the selected quadratic solve (SQ).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package.  The CUDA library never calls it and shares no code
with it; both sides receive the same arrays from the seeded input generator.

Everything here is complex128 numpy, written in the order of the paper's
algorithms so that it can be checked against the text by eye:

* ``rgf``   - RGF for BTA matrices (Alg. 1 forward Schur complement, Alg. 2
  backward SI/SQ, extended to the arrowhead as described in Sec. III-A), and the
  literal block-tridiagonal form of Alg. 1/2 (a = 0) as an independent path.
* ``dense`` - the dense definition (Alg. 4): G^R = A^{-1} and
  G^< = A^{-1} B A^{-H} from a full LU, restricted to the BTA pattern.

Library primitives used as single steps: ``numpy.matmul``, ``numpy.linalg.inv``
(LAPACK getrf + getri) and ``scipy.linalg.lu_factor/lu_solve``.

Pinning (see ``tests/test_oracle_*.py``): dense definition, exact rational
arithmetic on tiny integer inputs, closed forms for 1x1-block chains, and the
invariants A G^R = I on the pattern and G^< = -(G^<)^H.  Every function here is
pinned; none is "parity unpinned".
"""
from . import dense, rgf  # noqa: F401
