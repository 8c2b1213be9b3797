"""Plain, slow FP64 CPU oracle of the implicit-randomized-SVD PEPS contraction.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or runs
anything in this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA
library: the only common dependency is the seeded input generator ``synth``,
which holds none of the method's arithmetic.

Modules and the passages they follow (arXiv:2006.15234):
  philox      -- Philox4x64-10 counter-based generator (Salmon et al., SC'11)
                 drawing the sketch of Algorithm 4 and the gauge vector.
  implicit    -- the implicit operator A of one zip-up einsumsvd step
                 (Algorithm 3, einsumsvd line; Sec. IV-A implicit application)
                 applied as A X and A^H Y without forming A.
  rsvd        -- Algorithm 4 (randomized SVD of an implicit operator), with
                 Householder QR as "orthogonalize".
  bmps        -- Algorithm 2 (boundary MPS) and Algorithm 3 (zip-up
                 ApproxApply), one- and two-layer (Sec. III-B).
  bruteforce  -- exact contraction used to pin the above on tiny lattices.
  expectation -- Eq. 6 with the cached-environment strips of Sec. IV-B.
  grad        -- central finite differences of the expectation energy.
  qrsvd       -- operator application by QR-SVD (Algorithm 1) with the
                 einsumsvd of G, R1, R2 (Eq. 5), and one TEBD layer over all
                 nearest-neighbour bonds (one-site operators by Eq. 4).
  ite         -- imaginary-time evolution (Sec. II-D): TEBD steps with the
                 Rayleigh quotient after each.

Parity status: the final scalars of the larger lattices (8x8 and 16x16
norms) have no closed form; they are pinned only through the checks of each
building block ("parity unpinned" beyond the oracle's replay of the
algorithm).  Every other function is pinned by tests/test_oracle_*.py.
"""
