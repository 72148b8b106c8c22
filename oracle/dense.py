"""Dense analysis matrix A of HP2SPH at small Nside and its transpose with respect
to the real inner products used by the adjoint (test infrastructure).

HP2SPH is linear over the reals in the map (every step of Algorithm 1 is), so
A e_i for the unit maps e_i gives its columns.  With
  <f, g>_map = sum_i f_i g_i,
  <a, b>_alm = sum_l [Re(a_l0 conj b_l0) + 2 sum_{m>0} Re(a_lm conj b_lm)],
the transpose is (A^T a)_i = <A e_i, a>_alm.
"""

import numpy as np

from . import geometry, hp2sph


def alm_weights(lmax):
    """1 for m = 0, 2 for m > 0, in packed order."""
    w = np.empty(hp2sph.n_alm(lmax))
    for m in range(lmax + 1):
        i0 = hp2sph.alm_index(m, m, lmax)
        w[i0:i0 + lmax - m + 1] = 1.0 if m == 0 else 2.0
    return w


def analysis_matrix(nside, lmax=None):
    """Complex (n_alm, N) matrix with A[:, i] = analyze(e_i)."""
    n = geometry.npix(nside)
    eye = np.eye(n)
    return hp2sph.analyze(eye, nside, lmax).T


def transpose_apply(A, a, lmax):
    """A^T a for packed alm ``a`` (any leading batch dims flattened to (B, n_alm))."""
    a = np.atleast_2d(a)
    w = alm_weights(lmax)
    return np.real((A.T[None, :, :] * np.conj(a)[:, None, :] * w[None, None, :]).sum(-1))


def alm_dot(a, b, lmax):
    w = alm_weights(lmax)
    return float(np.sum(w * np.real(a * np.conj(b))))
