"""FP64 CPU oracle of the PURIFY SDMM-SARA hot path (arXiv:1307.4370).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, complex128
restatement of what the method computes, written to check the CUDA library
against.  Only the tests, the smoke check of ``__graft_entry__`` and the CPU
baseline leg of ``bench.py`` may import it.  The product path (the C-ABI
library and its Python binding) never calls, imports or links anything here,
and this package imports nothing from the product path.

Modules and the passages they follow:

* ``kaiser_bessel`` -- the interpolation kernel of G and its Fourier
  transform (the reciprocal of which is D), §5 eq. opmodel.
* ``measurement``  -- Phi = G F D Z (B = I) and its adjoint, §5 eq. opmodel,
  plus the direct non-uniform DFT of §3.1 eq. ri4 used to pin it.
* ``daubechies``   -- Daubechies-p filters by spectral factorisation
  (the db1..db8 bases named in §3.3).
* ``sara``         -- the SARA dictionary Psi = [Dirac, db1..db8] and its
  adjoint, §3.3, normalised to a Parseval frame as §4.4 requires.
* ``prox``         -- the proximity operators of §4.4 eqs. prox1, prox2,
  prox3.
* ``cg``           -- conjugate gradient on Q = Phi^H Phi + 2I, §4.4.
* ``sdmm``         -- Algorithm 1 with the stopping quantities of §4.4,
  the penalty gamma of §4.4 and the reweighting of §3.3.
* ``simulate``     -- visibilities and the l2 bound of §6.

Pins (tests that do not use this package to check itself) are in
``tests/test_oracle_*.py``.  Parts without an independent pin are marked
"parity unpinned" in their module docstring.
"""
