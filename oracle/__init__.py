"""CPU FP64 oracle for the multilevel BLUP hot path (arXiv:1701.00285).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package.
The GPU library never calls it and shares no code with it; the one module both
sides use is ``workloads`` (seeded input generators, no method arithmetic).

What it computes, in the paper's order and notation:

* ``matern``   -- the Matern covariance (Def. "Matern covariance function"):
                  closed forms at nu = 1/2, 3/2, 5/2, the definition with the
                  library K_nu for any other nu; the Gaussian kernel of the
                  accuracy study (Sec. 8.2); the anisotropic distance r(theta)
                  (Sec. 3); derivatives in log(rho).
* ``design``   -- the total-degree monomial design matrix X (Sec. 2, Q^d_w).
* ``tree``     -- the kd-tree (Algorithms 1-3: Rule, InitialTree, MakeTree).
* ``basis``    -- the multilevel basis W, L (Sec. 3.1, steps 1-5 and the
                  operator W = [W_t; ...; W_0]).
* ``pattern``  -- the distance criterion tau_{i,j} and tree search (Sec. 4.1,
                  Algorithms 4-6).
* ``assemble`` -- the sparse multilevel covariance C~_W (Algorithm 7).
* ``pcg``      -- diagonally preconditioned CG stopped on the unpreconditioned
                  residual (Sec. 6.2).
* ``dense``    -- the classic GLS/BLUP formulae (eqs. GLSbeta, KrigBLUP) and the
                  saddle-point system (eq. Spatial:problem).
* ``dense_mp`` -- the saddle-point system solved at 100 digits (mpmath) for
                  the ill-conditioned accuracy study of Sec. 8.2 (Table 5).
* ``mlblup``   -- the multilevel predictor (eqs. Spatial:eqn1-3, Spatial).
* ``grad``     -- gradient of a held-out prediction loss in log(rho) and
                  log(nugget) by the adjoint of the saddle-point system (the
                  paper has no gradient; this is the plain adjoint of its
                  BLUP equations).
* ``loglik``   -- the multilevel log-likelihood of the full transform (Sec.
                  5.1) and a stochastic Lanczos quadrature estimate of its
                  log-determinant; the kriging MSE is ``dense.mse_at`` (the
                  formula after eq. Spatial).

Readings of points where the paper is silent or garbled are stated in each
function's docstring.
"""
