"""Plain, slow FP64 CPU oracle for the disconnected-loop noise-subtraction method
(Baral, Whyte, Wilcox, Morgan, "Disconnected Loop Subtraction Methods in Lattice QCD").

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The product path
(the CUDA library behind ``include/lqcd.h`` and its Python binding) never imports, links or
executes anything here, and nothing here imports the product.

Every routine is written directly from the paper's definitions (equations and sections are
cited in each docstring), in numpy/scipy FP64, with no blocking, fusion or reordering beyond
what the definition states.  Library primitives (matrix products, QR, LU, eigen-solvers) are
used as single steps.

Modules
  lattice   -- site indexing, gamma matrices, the Wilson hopping matrix P and M = 1 - kappa P (Eq. xyz556)
  rng       -- Philox-4x32-10 counter generator and Z(4) noise (Sec. 2)
  krylov    -- GMRES-DR, MINRES-DR (Hermitian form), GMRES-Proj deflated solves (Sec. 5.3, 7, 8)
  subtract  -- PS / POLY / ES / HFES / HFPS / HFPOLY subtraction vectors and trace add-backs (Sec. 5)
  evenodd   -- even/odd reduced Wilson system, reconstruction, full eigenpairs from reduced ones (Sec. 7)
  operators -- the nine loop operators of Table Table903 and their per-site contractions (Sec. 6)
  estimate  -- noise estimators, error bars, relative efficiency (Sec. 5, 7)
  exact     -- dense-matrix exact traces and the exact Z(4) variance of Eq. xyz255 (Sec. 3)

Parity status: every function is pinned by a `-m "not gpu"` test in ``tests/test_oracle_*.py``
except the Min-Res polynomial values of Table xyz520 (their gauge configuration is not
published): parity unpinned for those printed values; the polynomial routine itself is
pinned by its least-squares optimality conditions.
"""
