"""CPU FP64 oracle for compressed H / UH / H^2 matrix-vector products.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It
shares no code with the GPU library (``paper_2405_03456_gb300``) and imports
nothing from it; both take their inputs from ``synth``.

Every function follows the paper (Kriemann, "Floating Point Compression of
Hierarchical Matrix Formats and its Impact on Matrix-Vector Multiplication")
in its own plain code: section and equation numbers are cited in each
docstring.  Arithmetic is IEEE FP64 throughout.

Modules
  codec    -- AFLP, FPX (Sec. 4.1) and VALR bit widths (Sec. 4.2)
  kernels  -- matrix entries of the model problems (Sec. 2.1 stand-in)
  trees    -- cluster tree (Def. Cluster Tree), block tree (Def. Block Tree)
  hmatrix  -- H(T, eps) construction by truncated SVD (eqn. epsilon)
  nested   -- shared (UH, Sec. 2.3) and nested (H^2, Sec. 2.4) cluster bases
  compress -- direct and VALR compression of a built matrix (Sec. 4.1-4.2)
  matvec   -- Alg. 1, Alg. 4 + 5, Alg. 6 + 7, with Alg. 8 decompression
  hlu      -- H-LU factors on the block tree and their triangular solves (Sec. 5, Conclusion)
  baseline -- the timed CPU run used as the benchmark's CPU baseline

Parity status: every function is pinned by ``tests/test_oracle_*.py`` except
the exact bit layout of AFLP codes, which the paper does not print ("parity
unpinned" for the layout; the codec's stated properties are pinned).
"""
