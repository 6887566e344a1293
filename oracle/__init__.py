"""FP64 CPU oracle for the CT-HYB local trace (arXiv 2010.08482).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls, links or
executes this package.  Its only users are the tests under ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``.

The oracle computes the plain definitions, slowly and in float64, so that a
reader can check each step against the paper by eye:

* ``oracle.atom``  -- Fock space and fermion operators (Sec. 3.3.1,
  "Computing the local impurity trace"), the local Hamiltonian
  (Eq. ImpurityHamiltonian) with Kanamori / Slater-Condon interactions,
  spin-orbit coupling and crystal fields, the sector decomposition by abelian
  quantum numbers, ``numpy.linalg.eigh`` per sector and the operator blocks
  F_alpha(q) in the eigenbasis.
* ``oracle.trace`` -- the sector-string trace (the sum over q0 of the trace of
  propagators and blocks along the string q0 -> q1 -> ... -> q0, Sec. 3.3.1),
  the full-Fock-space brute-force trace with matrix exponentials, the
  lazy-trace norm bounds (Sec. 3.3.1, last paragraphs), the Metropolis
  decision (Eqs. MHratio, decide), and the atomic Green function.
* ``oracle.observables`` -- the reduced-density-matrix estimator of one
  configuration (Eq. ImpurityDensityMatrix: the projector |v><u| inserted at
  every time, integrated analytically over each propagation interval), and
  its brute-force counterpart by quadrature over the full Fock space.
* ``oracle.improved`` -- the static part of the improved estimator for the
  self-energy (Eq. PImprovedEstimatorStatic): the Bulla operators [c_f, U]
  from the interaction terms alone, in the occupation basis and then the
  eigenbasis, and the ratio of the trace with one annihilator replaced to
  the plain trace.

It shares no code with the GPU path (``paper_2010_08482_gb300``) and imports
nothing from it.  Every function is pinned by a ``-m "not gpu"`` test against
closed forms, textbook values, brute force or library routines; see the test
files ``tests/test_oracle_*.py``.
"""
