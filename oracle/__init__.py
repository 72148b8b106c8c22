"""FP64 CPU oracle for HP2SPH (Drake & Wright, "A Fast and Accurate Algorithm for
Spherical Harmonic Analysis on HEALPix Grids", arXiv:1904.10514).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
leg of ``bench.py`` use it.  It shares no code with the CUDA library.

Every function follows the paper's definition of a step, written out plainly in
float64 with NumPy (direct sums, dense least squares, exact Gauss-Legendre
quadrature).  There is no blocking, fusion or fast algorithm beyond what the
definition states.  Readings of points where the paper is silent or garbled are
stated where they are used:

* p = 2*Nside (the printed "p = Nside/2" of Sec. 3.3 contradicts m = 4*Nside+1 of
  Sec. 3.2.2 and the 4*Nside longitude modes); lmax <= p.
* Nyquist term of a ring expansion (Eq. trig_expansion vs Eq. interp_cond): the
  real-symmetric split, half of the n = -nphi/2 coefficient at each of +-nphi/2.
* Pole values (Sec. 3.2.1): unit-weight least squares fit of a full quadratic in
  the tangent-plane coordinates (x, y) = (sin t cos l, sin t sin l) over the 24
  samples of the three rings nearest the pole; the value is the constant term.
* Inverse NUFFT-II (Sec. 3.2.2): the exact least-squares solution with
  m = 4*Nside+1 latitude modes over the 8*Nside DFS nodes.
* FSHT (Sec. 3.3): the L2(S^2) projection of the bivariate Fourier series onto
  Y_l^m, l <= lmax, which is what a change of basis by orthogonal connection
  matrices computes in exact arithmetic.
* Y_l^m with the Condon-Shortley phase and Y_l^{-m} = (-1)^m conj(Y_l^m)
  (Appendix A prints the relation without the conjugate).

Modules
-------
geometry   HEALPix rings, Eq. (healpts)
legendre   orthonormal associated Legendre functions and Y_l^m (Appendix A)
hp2sph     Algorithm 1 step by step, C_l (Eq. APS)
dense      dense analysis matrix A and its transpose at small Nside
healpix    the HEALPix software analysis of Sec. 2.2 (equal weights, Jacobi iteration)
"""

from . import geometry, legendre, hp2sph, dense, healpix  # noqa: F401
