"""Plain FP64 CPU oracle for the multiple Arnoldi method (Hoshi et al., arXiv:1202.0098).

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import, call or run
anything in this package: only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it. It shares
no code with the CUDA library; both take their inputs (atom positions and
parameter sets) from the ``synth`` package, which holds no method arithmetic.

It follows the paper's steps in its order and notation, slowly and densely:

* ``sk``       the model: Slater-Koster sp blocks, the periodic H and S, and the
               real-space projection onto a cluster (Sec. 3).
* ``mka``      per column j: inner CG for s_j = S^{-1} e_j (Sec. 2), the
               S-orthonormal multiple Krylov basis (Eqs. EQ-REC-UN, EQ-KN-HUN,
               EQ-MGram-Schmidt, EQ-CALC-S-INV), the Galerkin reduced problem
               (Eq. EQ-SUB-EIG-VEC), the density matrix (Eq. EQ-DM), the subspace
               Green's function (Eq. EQ-SOLUTION-SUB-GZ), the band energy
               (Eq. EQ-ENE) and mu by bisection.
* ``rounding`` FP32 / BF16 storage rounding of H and S values, so that mixed
               precision forms are checked against the oracle run on the very
               values they store.
* ``mlp``      FP64 forward/backward of the warm-start network, for gradient checks.

Every function cites the passage it follows. Pins that tie each part to
something other than itself live in ``tests/test_oracle_*.py``.
"""
