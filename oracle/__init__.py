"""CPU oracle for the Wilson-clover AMA hot path (plain numpy, FP64).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library and its Python binding never call into it, and it
shares no code with them: the only common module is the seeded input
generator ``paper_1605_00564_gb300.synth``, which holds none of the method's
arithmetic.

Every function is written for a reader checking it against the paper
(arXiv:1605.00564, von Hippel, Rae, Shintani, Wittig), section 2:

* ``dirac``    - the O(a)-improved Wilson-clover operator of the Dirac
                 equation D psi = eta (Sec. 2.2), clover term from plaquette
                 leaves.
* ``solve``    - plain unpreconditioned GCR and CG on the normal equations,
                 dense inverse for tiny lattices.
* ``sap``      - block decomposition, D = D_Omega + D_Omega* + D_dOmega +
                 D_dOmega*, the SAP cycle and kernel K, M_SAP (Sec. 2.2).
* ``nucleon``  - nucleon interpolator N = eps (u^T C g5 d) u (eq. Nop), its
                 two-point function with P+- projections, the AMA estimator
                 (eqs. caa1, caa2).
* ``deflation``- deflation projector P_L, little Dirac operator A (eq. little),
                 deflated solution (eq. deflsoln).
"""
