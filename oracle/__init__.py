"""CPU FP64 oracle for the multidimensional butterfly factorization (BF) apply.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or execute
this package: only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg
of `bench.py` use it.  It shares no code with the CUDA library; the only common
dependency is `mbf_synth`, which draws seeded random inputs and holds none of
the method's arithmetic.

Contents, each function citing the passage of Li, Yang & Ying,
"Multidimensional Butterfly Factorization" (arXiv 1509.07925) it follows:

* `problem`  -- kernels K(x, xi) (2-D/3-D DFT, the FIO of Example 1 and its
               isotropic special case), point sets X and Omega (§1.1), Z-order
               quadtrees/octrees (§2.2, Fig. 1), the polar map (§3.1) and the
               corona split (§4.1).
* `direct`   -- the direct sum u(x) = sum_xi K(x,xi) g(xi) (eq. kernel), the
               closed-form DFT special case, and the relative error e (§3.3).
* `lowrank`  -- the three low-rank forms (eqs. lowrank1-3), SVD via random
               sampling and via random matvec (§2.1).
* `bf`       -- construction (middle level §2.3, recursive factorization §2.4)
               into a padded factor set, assembly of every factor as an explicit
               sparse matrix exactly as §2.3-2.4 draw them, and the apply of
               eq. (gbf) and its adjoint by multiplying those matrices in order.
* `msbf`     -- the multiscale sum of eqs. (msumd) and (f1).

Pins (tests/test_oracle_*.py, run with -m "not gpu") tie every function to
something other than itself: the closed-form DFT, exactness of the BF when the
rank is at least every block dimension, the adjoint identity, brute force on
tiny inputs, structural patterns of Figs. 2-3, and the paper's Table 2 error.
"""
