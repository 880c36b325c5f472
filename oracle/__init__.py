"""Oracle: a plain, slow, dense FP64 CPU reference of the Hermitian-symmetric CTMRG.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or execute anything in this
package. The library (``paper_2410_11596_gb300``) never imports it, and this
package imports nothing from the library: the two share no code. Inputs come
from the seeded generators in ``paper_2410_11596_gb300.inputs`` (a module with
no arithmetic of the method) and are passed in as arrays.

Everything here is numpy/scipy in float64 / complex128, written for a reader to
check against the paper by eye:

* ``basis``        -- bra-ket swap S, its eigenbasis U, sector dimensions and the
                      real/imaginary grading with the tensor f (Sec. II.B, II.C,
                      Eqs. (1)-(3)).
* ``doublelayer``  -- the double-layer tensor a = sum_s A_s (x) conj(A_s)
                      (Sec. II.A, Fig. 1(b)) and its rotation into the eigenbasis
                      of S (Sec. II.B).
* ``ctmrg``        -- dense C4v CTMRG (Sec. II.A, Fig. 1(d)): traced-boundary
                      initialisation, enlarged corner, eigenvalue truncation
                      (complex-symmetric eigenvectors for complex tensors), renormalisation
                      and max-abs normalisation.
* ``observables``  -- one-site environment eps and the Hermitian symmetry error
                      S_err (Sec. III.A, Eq. (4)), two-site reduced density
                      matrix and bond energy, normalised corner spectrum,
                      per-site free energy, correlation length.
* ``hotrg``        -- dense HOTRG (Sec. II.A) and its symmetry-error probe built
                      from the tensor b (Sec. III.A).

Parity pins (tests/test_oracle_*.py) tie each function to something other than
itself: the D=2 basis printed in Sec. II.B, closed forms, Onsager's solution of
the 2D Ising model, brute-force contraction of finite patches and complex
arithmetic. Functions without such a pin say "parity unpinned" in their
docstring.
"""
