"""HEALPix point set, Eq. (healpts) of Sec. 2.1 (test infrastructure; see package doc).

Rings are numbered i = 0 .. 4*Nside-2 from north to south; pixels are stored in
RING order (north to south, increasing longitude within a ring).
"""

import numpy as np


def ring_table(nside):
    """Return a list of dicts, one per ring, north to south.

    Keys: ``z`` (cos theta), ``theta``, ``nphi``, ``phi0`` (longitude of the first
    pixel), ``shifted`` (True when the ring's longitudes are offset by half a
    pixel), ``start`` (offset of the ring's first pixel in RING order).

    Eq. (healpts): north cap j = 1..Nside-1 has 4j points at
    lambda = pi (k + 1/2) / (2j), z = 1 - j^2 / (3 Nside^2); equatorial rings
    j = Nside..3 Nside have 4 Nside points at lambda = pi (k + ((j+1) mod 2)/2) /
    (2 Nside), z = 2 (2 Nside - j) / (3 Nside); the south cap mirrors the north.
    """
    ns = int(nside)
    rings = []
    start = 0
    for j in range(1, 4 * ns):
        if j < ns:
            jj = j
            z = 1.0 - jj * jj / (3.0 * ns * ns)
            # theta = 2 asin(j / (sqrt(6) Nside)) is the same angle without the
            # cancellation of arccos near 1.
            theta = 2.0 * np.arcsin(jj / (np.sqrt(6.0) * ns))
            nphi = 4 * jj
            shifted = True
        elif j <= 3 * ns:
            z = 2.0 * (2 * ns - j) / (3.0 * ns)
            theta = np.arccos(z)
            nphi = 4 * ns
            shifted = ((j + 1) % 2) == 1
        else:
            jj = 4 * ns - j
            z = -(1.0 - jj * jj / (3.0 * ns * ns))
            theta = np.pi - 2.0 * np.arcsin(jj / (np.sqrt(6.0) * ns))
            nphi = 4 * jj
            shifted = True
        phi0 = (np.pi / nphi) if shifted else 0.0
        rings.append(dict(z=z, theta=theta, nphi=nphi, phi0=phi0,
                          shifted=shifted, start=start))
        start += nphi
    return rings


def npix(nside):
    return 12 * int(nside) ** 2


def pixel_angles(nside):
    """(theta, lambda) of every pixel centre in RING order (float64 arrays)."""
    th = []
    ph = []
    for r in ring_table(nside):
        k = np.arange(r["nphi"])
        th.append(np.full(r["nphi"], r["theta"]))
        ph.append(r["phi0"] + 2.0 * np.pi * k / r["nphi"])
    return np.concatenate(th), np.concatenate(ph)


def latitude_nodes(nside):
    """The 4*Nside+1 latitudes on [0, pi]: north pole, the rings, south pole
    (Sec. 3.2.1: the poles are added to close the gap over the caps)."""
    rings = ring_table(nside)
    return np.concatenate([[0.0], [r["theta"] for r in rings], [np.pi]])
