"""Plain, slow FP64 CPU oracle of the multigrid Rayleigh-quotient eigensolver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package may import, call or
execute anything under ``oracle/``; only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` do.  It shares no code with the CUDA
path: its inputs come from ``synth`` (random numbers only) and every piece of
arithmetic here is written out from the paper (arXiv:1509.06865, Bali et al.,
"(Approximate) Low-Mode Averaging with a new Multigrid Eigensolver"):

  dirac    the clover-improved Wilson operator D, Q = gamma5 D, D_sigma (Sec. 2, Eq. 2.1)
  dense    dense matrices of D / Q for small lattices, eigh-based reference spectra
  mg       aggregation interpolation P (Eq. 2.4), coarse operator P^dag D P (Eq. 2.5,
           2.6), SAP smoother, GMRES smoother, the two-grid cycle (Eq. 2.3)
  krylov   restarted GMRES and flexible GMRES (Sec. 2.2: double precision FGMRES
           preconditioned by the multigrid method)
  rqi      the multigrid setup and Rayleigh quotient iteration (Algorithm 1)

Floating point is complex128 throughout.  Field layouts follow ``synth``:
gauge U[t, z, y, x, mu, a, b], spinor psi[..., t, z, y, x, spin, colour].
"""
