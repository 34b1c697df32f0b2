"""FP64 CPU oracle for the spectral boundary-integral method for N rigid spheres
in Stokes flow (Corona & Veerapaneni, arXiv:1707.06551).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, numpy restatement of
the paper's definitions and algorithm steps, used to check the CUDA path.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it.  It shares no code with the CUDA library and never
imports the product package.

Modules
  quadrature  Gauss-Legendre nodes, the sphere grid and smooth weights (Sec. 4, Eqs. 4.2-4.4)
  sph         scalar and vector spherical harmonics (Sec. 2.1, Eqs. 2.1, 2.4-2.6)
  vsh         VSH analysis and synthesis on the grid (Sec. 2.1, Eqs. 2.12-2.17)
  signatures  eigenvalues of S, D+-, K+- (Theorem 2, Eq. 3.12)
  kernels     Stokeslet / stresslet smooth-quadrature sums (Eqs. 2.19-2.22, 4.4)
  dual        forward-mode dual numbers (used for the traction of an expansion)
  offsurface  exterior evaluation of S, D and the traction K (Eqs. 3.6-3.11, 3.18)
  operators   the discrete operators and BIEs (Sec. 4.1, 4.3, Eqs. 5.8, 5.19)
  gmres       plain restarted GMRES with modified Gram-Schmidt
  solve       mobility and resistance drivers (Sec. 5, Problems 2 and 5)

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py``; none is "parity unpinned".
"""
