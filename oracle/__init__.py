"""CPU FP64 oracle for the current-flow closeness hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.
The product path (``paper_1607_02955_gb300``) never imports it, and this
package never imports the product path.  The two share no code; the only
common dependency is the seeded input generators in ``synth/``, which hold
none of the method's arithmetic.

Everything here is plain, slow and FP64: numpy / scipy library primitives
(dense inverse, sparse mat-vec, connected components) serve as single steps;
there is no blocking, fusion or reordering beyond what the paper states.

Modules and the passages they follow (Bergamini et al., "Estimating
Current-Flow Closeness Centrality with a Multigrid Laplacian Solver"):

* ``philox``   -- Philox4x64-10 counter-based generator (Salmon et al., SC'11),
                  the random source for the JL matrix Q (Sec. 5.2) and the
                  sampled pivots (Sec. 5.1).  Pinned against numpy's own
                  Philox bit generator.
* ``graph``    -- G = (V, E, w) and L = D - A (Sec. 2), incidence matrix B and
                  W (Sec. 5.2).
* ``dense``    -- L^+ and the grounded inverse (Sec. 4), effective resistance
                  d_ER (Sec. 4), electrical farness and c_ER (Eq. closeness2).
* ``cg``       -- conjugate gradient for L x = b with the null space removed
                  (Sec. 2 rank n-1, Sec. 3.1 CG and relative residual).
* ``jl``       -- the projection estimator, Algorithm 1 (Sec. 5.2).
* ``sampling`` -- the pivot-sampling estimator and Proposition 1 (Sec. 5.1).

Every function is pinned by a ``-m "not gpu"`` test against closed forms,
identities, a library routine or brute force; the exceptions are named
"parity unpinned" in the function's docstring.
"""
