"""CPU FP64 oracle for the TNVAN hot path (arXiv 2504.12037).

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain, independent
statement of what the GPU path must compute.  Only the test suite, the smoke
check and the CPU-baseline / reference arm of the benchmark may import it; the
product library never does, and it shares no code with the CUDA kernels.

Modules and the passages they restate:
  philox     Philox4x32-10 counter-based generator (Salmon et al., SC'11), the
             uniforms behind the Bernoulli draws of Eq. 8.
  ising      Eq. 1-2 (energy, brute-force Z) and Eq. 3-4 (log Z_R by plain
             enumeration of the leftover spins).
  transfer   Eq. 2 contracted row by row: dense 2^w transfer matrices for
             lattice strips, whole-lattice row and single-site (helical)
             transfer matrices, and Kaufman's closed form for the torus.
  dense      Eq. 4 for a fully connected leftover block: plain 2^|R| sum.
  general    Eq. 4 for general leftover components: enumeration, or variable
             elimination in its own min-degree order.
  slicing    Sec. 2 width sets: the width of an elimination order, exact
             treewidth and smallest width sets of small graphs.
  made       Eq. 6-8 (MADE conditionals, log q, ancestral sampling).
  estimators Eq. 5, 9, 10 (F_q, importance-sampled log Z, REINFORCE weights
             and gradient, exact enumeration of F_q) and the Adam update.
  kacward    the Kac-Ward determinant: exact ln Z of an open planar lattice
             (the ferromagnet of Sec. 4, Fig. 2).
  magnetisation  Sec. 3 observables: conditional magnetisation moments from
             a uniform-field derivative of any contraction above, and their
             importance-weighted averages (magnetisation, susceptibility).

Parity status: every function is pinned by a `-m "not gpu"` test against a
closed form, brute force, or an invariant, except where its docstring says
"parity unpinned".
"""
