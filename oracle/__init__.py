"""Plain, slow, FP64 CPU oracle for the immersed-FE multigrid-preconditioned CG solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or runs this
package: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` do.  It shares no code with the CUDA library.

It follows de Prenter et al., "Scalable multigrid methods for immersed finite element
methods and immersed isogeometric analysis" step by step:

* ``geometry``    -- level sets and cell classification (Sec. 2, Fig. 1)
* ``basis``       -- uniform open-knot B-splines and equispaced Lagrange bases (Sec. 2)
* ``quadrature``  -- bisect / triangulate / clip cut-cell quadrature (Sec. 2, Fig. 1)
* ``discretize``  -- assembly of A x = b (Eqs. weakMulti, operatorsMulti, systemMulti)
* ``multigrid``   -- two-scale restriction (Eq. coarsening), Galerkin coarse operators
                     (Remark 3.1), Schwarz blocks with encapsulating supports and the
                     tiny-eigenvalue rule (Sec. 3.4, Remark 3.3), the V-cycle
                     (Algorithm 1) and multigrid-preconditioned CG (Sec. 3.2)

Every function states the passage it follows.  Where the paper is silent or ambiguous
the reading taken is stated in the docstring.
"""
