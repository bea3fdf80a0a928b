"""Oracle: plain, slow CPU reference for the BFP multigrid hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package may import this
package.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

Modules
-------
bfp      exact block-floating-point arithmetic (paper Sec. 2, Sec. 4,
         Alg. qcomp, Alg. nnqcomp, App. B) in Python/numpy integers.
mg       FP64 multigrid and the BFP multigrid schedule (V(2,2), FMG, IR;
         App. C algorithms adapted to damped Jacobi) built from ``bfp``.
"""
