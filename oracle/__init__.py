"""Oracle for the butterfly-factorisation apply: plain, slow, obviously correct.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything from this package.  The
product library (``paper_1803_04128_gb300``) never imports, links or executes
it, and this package never imports the product.  The two share no code; only
the seeded input generators (``paper_1803_04128_gb300/inputs.py``, which holds
none of the method's arithmetic) feed both sides, through the tests.

Modules
  direct     -- the plain definition g = K f in FP64 (C, OpenMP), plus a long
                double brute-force variant and single entries of K.
  lowrank    -- Alg. 1 (randomised sampling rank-r SVD) for the amplitude split.
  recovery   -- Algs. 3, 4, 5: a low-rank phase Psi (e^{2 pi i Psi} = e^{2 pi i Phi})
                recovered from kernel entries alone (Scenario 1 of Table sc).
  special    -- the Hankel-function transform of Sec. 5 (Eq. HK): entries, direct sums.
  decide     -- Alg. 6 of Sec. 3: may r-dimensional NUFFTs after dimension lifting
                evaluate the transform, or does it need the butterfly?
  nufft      -- Eq. (tg3) of Sec. 3 by 1-D NUFFTs (Gaussian gridding) for phases
                that are rank 1 on each column half (the split of Eq. FIOwq2).
  butterfly  -- the butterfly algorithm of Sec. 4 (Algorithm 4.1) in FP64,
                on the fly, in the paper's step order; and the IBF apply of
                Eq. (tg): g = sum_k a_k * BF(b_k * f).

Parity status of each function is listed in its docstring; every function
here is pinned by tests/test_oracle_pins.py.
"""
