"""Image-source sums for a shoebox room (oracle, test infrastructure).

Eq. (an2): psi(r,k) = G_k(r, r_s) + sum_j A_j G_k(r, r_j), with the images of
Allen & Berkley (1979) for the room [0,lx]x[0,ly]x[0,lz]: per axis the image
coordinate is 2 q L + (1 - 2u) s (q integer, u in {0,1}); it has |q - u|
reflections off the wall at 0 and |q| off the wall at L.  A_j is the product
of the wall reflection coefficients over those reflections (A_j = R^{n_j}
for a uniform R).  Images are dropped when A_j < A_th (Sec. 4 uses 1e-7) or,
with complex k, when exp(-Im k |r - r_j|) falls below ``decay_tol``.

For rigid walls (R = 1) with complex k the sum is the exact Neumann Green's
function of the box.  For absorbing walls it is the paper's approximate
analytical model.
"""
from __future__ import annotations

import numpy as np


def _axis_images(s, L, qmax):
    out = []
    for q in range(-qmax, qmax + 1):
        for u in (0, 1):
            out.append((2 * q * L + (1 - 2 * u) * s, abs(q - u), abs(q)))
    return out


def image_field(xr, xs, room, k, R_walls=(1, 1, 1, 1, 1, 1), a_th=1e-7,
                decay_tol=1e-12, qmax=None, include_direct=True):
    """psi at points xr[n,3] for a source xs in the shoebox ``room``.

    R_walls: reflection coefficients of walls (x=0, x=lx, y=0, y=ly, z=0, z=lz).
    qmax: image order per axis; by default enough for the decay tolerance
    (complex k) or for A_th (|R| < 1).
    """
    xr = np.atleast_2d(np.asarray(xr, float))
    lx, ly, lz = room
    Rw = np.asarray(R_walls, dtype=np.complex128)
    kim = float(np.imag(k))
    if qmax is None:
        if kim > 0:
            rmax = -np.log(decay_tol) / kim
            qmax = int(np.ceil(rmax / (2 * min(room)))) + 1
        else:
            rmax_abs = float(np.max(np.abs(Rw)))
            qmax = int(np.ceil(np.log(a_th) / np.log(rmax_abs) / 2)) + 1 if rmax_abs < 1 else 20
    axes = []
    for s, L, r0, r1 in ((xs[0], lx, Rw[0], Rw[1]), (xs[1], ly, Rw[2], Rw[3]),
                         (xs[2], lz, Rw[4], Rw[5])):
        pos, amp, nref = [], [], []
        for q in range(-qmax, qmax + 1):
            for u in (0, 1):
                pos.append(2 * q * L + (1 - 2 * u) * s)
                amp.append(r0 ** abs(q - u) * r1 ** abs(q))
                nref.append(abs(q - u) + abs(q))
        axes.append((np.array(pos), np.array(amp), np.array(nref)))
    (X, ax, nx), (Y, ay, ny), (Z, az, nz) = axes
    A = ax[:, None, None] * ay[None, :, None] * az[None, None, :]
    nrefl = nx[:, None, None] + ny[None, :, None] + nz[None, None, :]
    P = np.stack(np.meshgrid(X, Y, Z, indexing="ij"), -1)
    keep = (np.abs(A) >= a_th) | (nrefl == 0)
    if not include_direct:
        keep &= nrefl != 0
    P = P[keep]
    A = A[keep]
    out = np.zeros(xr.shape[0], np.complex128)
    for s in range(0, P.shape[0], 20000):
        d = np.linalg.norm(xr[:, None, :] - P[None, s:s + 20000, :], axis=-1)
        out += np.sum(A[None, s:s + 20000] * np.exp(1j * k * d) / (4 * np.pi * d), axis=1)
    return out


def reflection_from_admittance(beta):
    """Normal-incidence reflection coefficient R = (zeta-1)/(zeta+1) = (1-beta)/(1+beta),
    inverted from Eq. (sp4)."""
    beta = np.asarray(beta, dtype=np.complex128)
    return (1 - beta) / (1 + beta)
