"""FP64 CPU oracle for the Hierarchical Subspace Iteration Method.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the paper's method (Nasikun & Hildebrandt, "The Hierarchical
Subspace Iteration Method for Laplace-Beltrami Eigenproblems"): NumPy/SciPy in
float64 plus one small C file for Dijkstra.  Only the tests, the smoke check
and the benchmark's CPU-baseline leg may import it; the library in
``paper_2111_09039_gb300`` never does, and this package never imports the
library.  The two share nothing but the seeded mesh generators in ``synth``.

Modules
-------
assembly   cotan stiffness S and lumped mass M (Sec. 3.1, eq. massStiffMatrices)
hierarchy  level sizes (eqs. nT-1, growthRate), farthest-point sampling
           (Alg. 2), prolongations U (eqs. radius, basis and normalisation)
galerkin   S^tau = U^T S U, M^tau = U^T M U (Alg. 3, restriction step)
sim        subspace iteration (Alg. 1) with the HSIM refinements, and the
           coarse-to-fine driver (Alg. 3)

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py``; nothing here is "parity unpinned" except what the
header of ``sim.py`` lists.
"""
