"""CPU FP64 oracle for finite-temperature TD-DMRG carrier mobility.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
Python binding) may import, call or link anything in this package.  Only the
test-suite, the package smoke check and the CPU-baseline leg of the benchmark
use it.

The oracle is written from the paper (Li, Ren & Shuai, "Finite temperature
TD-DMRG for the carrier mobility of organic semiconductors"):

* ``model``  -- multi-mode Holstein(-Peierls) chain, Eq. 1 and Eq. 10, the current
  operator (Eq. 3), their MPOs and an independent dense construction.
* ``ed``     -- exact diagonalisation in the one-carrier sector: C(t) of Eq. 6
  through the eigenbasis, Z, <H>, the Kubo mobility of Eq. 2.
* ``tdvp``   -- a plain FP64 purified-MPS TD-DMRG (Eq. 4-6, Eq. S1) with the
  one-site projector-splitting integrator the paper uses for both imaginary
  and real time.
* ``kubo``   -- quadrature of Eq. 2 and the hopping-limit closed form of Eq. 7.
* ``gradient`` -- exact dC(t)/dtheta and dmu/dtheta (theta = omega_m, g_m, V) and the
  isotope derivative, by Frechet derivatives of the matrix exponential in the
  one-carrier sector: the reference for an adjoint of the TDVP step.
* ``adjoint`` -- vector-Jacobian products of the TDVP building blocks (the H_eff and
  bond products, the environment updates, the Krylov exponential with its Frechet
  integral by Gauss-Legendre quadrature, the full-rank gauge QR) and the discrete
  adjoint of one projector-splitting step recorded on a tape, with the parameter
  gradient through the MPO; the reverse pass of the real-time correlation (steps of
  both states and the j overlaps, recomputed from stored states) and of the
  imaginary-time preparation (d log Z / dtheta), completed gauge columns included.

Every function is slow and literal on purpose.  It shares no code, tables or
helpers with the CUDA path.
"""
