"""Indirect boundary-element formulation with two unknowns per element
(Sec. 2.3, Eqs. ibem1-ibem5) -- oracle, test infrastructure.

The unknowns are the scattered field on the two sides of every element,
psi+ and psi-; the element normal points from the - side to the + side (out
of the room on the walls).  With a = k/(i zeta) = -i k beta on each side
(beta the admittance of that side):

    mu    = psi+ - psi-                                           (ibem4)
    sigma = gamma- + gamma+ - a- psi- - a+ psi+
    boundary conditions:  d psi-/dn + a- psi- = gamma-,
                         -d psi+/dn + a+ psi+ = gamma+
    for an incident field psi_in:  gamma- = -d psi_in/dn - a- psi_in,
                                   gamma+ =  d psi_in/dn - a+ psi_in

and Eq. (ibem5), collocated at the centroids:

    (psi- + psi+)/2 - M[psi+ - psi-] + L[a- psi- + a+ psi+] = L[gamma- + gamma+]
    -M'[psi+ - psi-] + (a+ psi+ - a- psi-)/2 + L'[a- psi- + a+ psi+]
                              = (gamma+ - gamma-)/2 + L'[gamma- + gamma+]

The scattered field off the surface is psi_sc = L[sigma] + M[mu]   (ibem1).
L, M, L' are the dense matrices of ``bem.dense_operators`` and M' that of
``hypersingular.dense_mp`` (same quadrature rules as the GPU path).
"""
from __future__ import annotations

import numpy as np

from . import bem


def _a(k, beta):
    return -1j * k * np.asarray(beta, dtype=np.complex128)


def system(L, M, LP, MP, k, beta_p, beta_m):
    """The 2N x 2N matrix of Eq. (ibem5); unknown vector [psi+, psi-]."""
    n = L.shape[0]
    ap = np.broadcast_to(_a(k, beta_p), (n,))
    am = np.broadcast_to(_a(k, beta_m), (n,))
    A = np.empty((2 * n, 2 * n), np.complex128)
    A[:n, :n] = -M + L * ap[None, :]
    A[:n, n:] = M + L * am[None, :]
    A[n:, :n] = -MP + LP * ap[None, :]
    A[n:, n:] = MP + LP * am[None, :]
    d = np.arange(n)
    A[d, d] += 0.5
    A[d, n + d] += 0.5
    A[n + d, d] += 0.5 * ap
    A[n + d, n + d] -= 0.5 * am
    return A


def gammas_incident(k, beta_p, beta_m, u, dudn):
    """(gamma+, gamma-) for an incident field with values u and normal
    derivatives dudn at the centroids (ibem4)."""
    return dudn - _a(k, beta_p) * u, -dudn - _a(k, beta_m) * u


def gammas_two_sided(k, beta_p, beta_m, vp, dvp, vm, dvm):
    """(gamma+, gamma-) for which the scattered field is vm on the - side and
    vp on the + side (values and normal derivatives at the centroids): the
    boundary conditions of (ibem4) applied to those fields."""
    return -dvp + _a(k, beta_p) * vp, dvm + _a(k, beta_m) * vm


def rhs(L, LP, gamma_p, gamma_m):
    """Right-hand side of Eq. (ibem5)."""
    s = gamma_m + gamma_p
    return np.concatenate([L @ s, 0.5 * (gamma_p - gamma_m) + LP @ s])


def densities(k, beta_p, beta_m, psi_p, psi_m, gamma_p, gamma_m):
    """(sigma, mu) of Eq. (ibem4)."""
    mu = psi_p - psi_m
    sigma = gamma_m + gamma_p - _a(k, beta_m) * psi_m - _a(k, beta_p) * psi_p
    return sigma, mu


def field(mesh, k, sigma, mu, xr, chunk=64):
    """psi_sc = L[sigma] + M[mu] at points off the surface (Eq. ibem1)."""
    xr = np.asarray(xr, float)
    out = np.empty(xr.shape[0], np.complex128)
    nz = np.zeros_like(xr)
    for s in range(0, xr.shape[0], chunk):
        e = min(xr.shape[0], s + chunk)
        L, M, _ = bem.operator_rows(mesh, k, xr[s:e], nz[s:e], -np.ones(e - s, int))
        out[s:e] = L @ sigma + M @ mu
    return out
