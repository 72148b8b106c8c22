"""Orthonormal associated Legendre functions and spherical harmonics, Appendix A
(test infrastructure; see package doc).

Pbar_l^m(x) = sqrt((2l+1)/2 * (l-m)!/(l+m)!) P_l^m(x), with the Condon-Shortley
phase in P_l^m, so that  int_{-1}^{1} Pbar_l^m(x)^2 dx = 1  and
Y_l^m(lambda, theta) = Pbar_l^m(cos theta) e^{i m lambda} / sqrt(2 pi)
is Eq. (ssph).  For m < 0, Y_l^m = (-1)^m conj(Y_l^{|m|}).

The values come from the standard three-term recurrence in l at fixed m.  The
starting value Pbar_m^m = (-1)^m sqrt((2m+1)/2 * (2m-1)!!/(2m)!!) sin^m(theta)
underflows float64 for large m near the poles, so the recurrence runs on a
mantissa with a separate power-of-two exponent, which is only applied at the end.
"""

import numpy as np

_BIG = 2.0 ** 400
_LOG2_BIG = 400


def _log2_pmm(m, sin_t):
    """log2 |Pbar_m^m| and its sign, elementwise in sin_t (> 0)."""
    k = np.arange(1, m + 1, dtype=np.float64)
    log2c = 0.5 * np.log2((2 * m + 1) / 2.0) + 0.5 * np.sum(np.log2((2 * k - 1) / (2 * k)))
    with np.errstate(divide="ignore"):
        l2 = log2c + m * np.log2(sin_t)
    return l2, (-1.0) ** m


def pbar_table(m, lmax, x, sin_t=None):
    """Pbar_l^m(x) for l = m..lmax, shape (lmax - m + 1, len(x)), float64.

    x must lie in [-1, 1]; values that are below the float64 range come out 0.
    ``sin_t`` = sqrt(1 - x^2) may be passed when it is known more accurately
    than it can be recovered from x (near the poles).
    """
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros((max(lmax - m + 1, 0), x.size))
    if lmax < m:
        return out
    if sin_t is None:
        sin_t = np.sqrt(np.maximum(0.0, (1.0 - x) * (1.0 + x)))
    else:
        sin_t = np.asarray(sin_t, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        if m == 0:
            l2 = np.full(x.size, np.log2(np.sqrt(0.5)))
            sgn = 1.0
        else:
            l2, sgn = _log2_pmm(m, sin_t)
    zero = ~np.isfinite(l2)           # sin theta == 0 and m > 0: exactly zero
    l2 = np.where(zero, 0.0, l2)
    e = np.floor(l2)                  # value = mant * 2**e
    mant = sgn * np.exp2(l2 - e)
    mant = np.where(zero, 0.0, mant)
    # p_{l-1} (prev) and p_l (cur) share the exponent e.
    prev = np.zeros_like(mant)
    cur = mant
    out[0] = np.ldexp(cur, np.clip(e, -2000, 2000).astype(np.int64))
    for l in range(m + 1, lmax + 1):
        a = np.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
        if l == m + 1:
            nxt = a * x * cur
        else:
            b = np.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
            nxt = a * (x * cur - b * prev)
        prev, cur = cur, nxt
        # renormalise mantissas that grew large while their exponent is negative
        big = (np.abs(cur) > _BIG) & (e < 0)
        if np.any(big):
            cur = np.where(big, cur / _BIG, cur)
            prev = np.where(big, prev / _BIG, prev)
            e = np.where(big, e + _LOG2_BIG, e)
        out[l - m] = np.ldexp(cur, np.clip(e, -2000, 2000).astype(np.int64))
    return out


def pbar(l, m, x, sin_t=None):
    """Pbar_l^m(x) for a single (l, m), m >= 0 (zero when l < m)."""
    if l < m:
        return np.zeros(np.size(x))
    return pbar_table(m, l, x, sin_t)[-1]


def ylm(l, m, lam, theta):
    """Y_l^m(lambda, theta) of Eq. (ssph), any sign of m."""
    lam = np.asarray(lam, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    ma = abs(m)
    val = pbar(l, ma, np.cos(theta).ravel(), np.abs(np.sin(theta)).ravel()).reshape(np.shape(theta)) \
        * np.exp(1j * ma * lam) / np.sqrt(2.0 * np.pi)
    if m < 0:
        val = (-1.0) ** ma * np.conj(val)
    return val
