"""Plain FP64 CPU oracle for symmetric block-sparse contraction.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_1203_2222_gb300``) never imports it and
shares no code with it; the two meet only in the seeded input generators of
``paper_1203_2222_gb300/synthetic.py``, which hold none of the method's
arithmetic.

What the oracle computes is the plain definition of each operation of
S. Singh, "Tensor Network States and Algorithms in the presence of Abelian and
non-Abelian Symmetries" (arXiv:1203.2222):

* ``cg``        Clebsch-Gordan coefficients (Ch. 5, Eq. cg, Racah's closed form)
                and recoupling coefficients F by explicit CG contraction
                (Ch. 5, Eq. f, with the reading noted there).
* ``u1``        U(1)-symmetric tensors: sector enumeration, dense embedding,
                extraction (charge conservation, Ch. 4 general statements).
* ``su2``       SU(2)-invariant tensors in a tree decomposition: sector
                enumeration, dense embedding through explicit CG trees and
                cups (Ch. 6, tree decompositions), extraction by projection,
                generator-based invariance residual (Ch. 5, Eq. Tinv).
* ``contract``  Dense brute-force contraction (Ch. 5, Eq. tensormult) and the
                dense gradient, extracted back to blocks.
* ``z2f``       Fermion-parity tensors (the thesis's conclusion): parity
                labels, swap signs of permutations and contractions.
* ``svd``       Blockwise singular value decomposition (Ch. 5, Eq. svd0 and
                svd1): block-diagonal form, SVD of every block, truncation,
                factors recast as tensors.
* ``eig``       Blockwise symmetric eigendecomposition (Ch. 5, Eq. spectral,
                by blocks as after Eq. svd1): the same block-diagonal form,
                numpy's eigh of every block, truncation by |lambda|, factors.
* ``sample``    Single dense elements of a contraction and of its gradients
                (Ch. 5, Eq. tensormult at one index) for tensors too large to
                embed.

Every function works in float64 with no blocking, fusion or reordering beyond
what the definition states.

Pins (tests/test_oracle_*.py, ``-m "not gpu"``) tie each part to values the
paper prints or to mathematics: printed CG values and omega matrices, CG
orthogonality, ladder-operator relations, 6j closed forms / orthogonality /
tetrahedral symmetry, generator invariance of embedded tensors, charge
conservation of dense products, printed storage counts and bond dimensions,
the dense SVD's spectrum and the Eckart-Young optimum of a truncation.
"""
