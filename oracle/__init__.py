"""CPU FP64 oracle for the adaptive Hessian-sketch ridge solver (Lacotte & Pilanci,
"Effective Dimension Adaptive Sketching Methods for Faster Regularized
Least-Squares Optimization", NeurIPS 2020).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never calls it, and it shares no code with the CUDA
sources: the two sides meet only through the seeded input generators in
``paper_2006_05874_gb300.problems`` (which hold none of the method's arithmetic)
and through the random-number specification, which each side implements on its
own from the published Philox4x32-10 definition.

Everything here is plain numpy in float64 (FP32 inputs are promoted exactly).
Each function cites the passage of the paper it restates.  Modules:

* ``philox``   - Philox4x32-10 counter-based generator (Salmon et al., SC'11).
* ``rng``      - the seeded draws the method needs: Rademacher signs, the SRHT
                 row subset, Gaussian sketch entries.
* ``hadamard`` - explicit Walsh-Hadamard matrix and a plain FWHT.
* ``sketch``   - SRHT and Gaussian embeddings applied to A (Sec. 1, App. C).
* ``linalg``   - objective, gradient, direct solve, Woodbury inverse of the
                 sketched Hessian, sketched Newton decrement, effective dimension.
* ``params``   - step sizes, momentum and rates (Thm 2.1, 2.2, Def 3.1, 3.2).
* ``ihs``      - Algorithm 1 and its gradient-only variant.
* ``cg``       - CG and sketch-preconditioned CG comparators (Sec. 5).
* ``warmstart`` - probe features, the warm-start network, its gradient and
                 the Adam step (an addition: no counterpart in the paper).

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, library routines, published known-answer vectors or invariants
the paper states; none is "parity unpinned".
"""
