"""Oracle: a plain, slow, FP64, single-threaded CPU restatement of the method of
Zambrano, Serrano, Lazarov & Galvis, "Fast multiscale contrast independent
preconditioners for linear elastic topology optimization problems" (arXiv
2006.13387).

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import or run this
package.  The product path (the CUDA library and its Python binding) never
imports it and shares no code with it.

Modules:
  fem      -- Q4/Hex8 element stiffness (Eq. 5 discretised), SIMP (Eq. 4),
              global assembly of K(rho) (Eq. 2), Dirichlet elimination, direct solve.
  schwarz  -- overlapping subdomains (Sec. 2, Eq. 6), the heat-operator coarse
              space with rotation enrichment (Sec. 4.1-4.3, Eqs. for V_{0,H}),
              the Galerkin coarse matrix K_0 = R_0 K R_0^T (Sec. 2.1) and the
              two-level additive preconditioner M_EH(+Rot) (Sec. 4.3).
  pcg      -- preconditioned CG (Sec. 2, Sec. 5), Lanczos condition estimate
              (Sec. 5, Saad ch. 6), energy-error estimate.

Readings of passages the paper leaves open are listed where they are used.
"""
