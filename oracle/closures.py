"""Discrete SMM closures (oracle).

Sec. "Transport Discretization", Eqs. correction_tensor_disc,
bdr_correction_factor_disc, eb0_disc and broken_Tdiv:

    T(x)    = sum_d w_d Omega_d (x) Omega_d psi_d(x) - 1/3 I sum_d w_d psi_d(x)
    beta(x) = sum_d w_d |Omega_d . n| psi_d(x) - E_b0 sum_d w_d psi_d(x)
    E_b0    = sum_d w_d |Omega_d . n| / 4 pi
    J_in(x) = sum_{Omega_d . n < 0} w_d (Omega_d . n) psibar_d(x)

The paper prints J_in with "w_d Omega_d psibar" (no ". n"); J_in is a
scalar partial current (Sec. "Derivation of Moment System"), so this oracle
reads it with the normal component.  E_b0 is taken pointwise (with the
local unit normal) on curved boundary faces.  psi_d(x) on a boundary face
is the element's own DG trace (the finite element interpolant).

T and phi are represented in the nodal basis of Y_p as linear combinations
of the psi_d nodal values (exact), and the broken divergence of T is taken
from the basis derivatives (Eq. broken_Tdiv).
"""
from __future__ import annotations

import math

import numpy as np


def nodal_moments(disc, psi):
    """phi, Jx, Jy, Txx, Txy, Tyy nodal values [6][ne][n] from psi [nd][ne][n]."""
    w, om = disc.wq, disc.omega
    phi = np.einsum("d,den->en", w, psi)
    jx = np.einsum("d,den->en", w * om[:, 0], psi)
    jy = np.einsum("d,den->en", w * om[:, 1], psi)
    pxx = np.einsum("d,den->en", w * om[:, 0] * om[:, 0], psi)
    pxy = np.einsum("d,den->en", w * om[:, 0] * om[:, 1], psi)
    pyy = np.einsum("d,den->en", w * om[:, 1] * om[:, 1], psi)
    return np.stack([phi, jx, jy, pxx - phi / 3.0, pxy, pyy - phi / 3.0])


def eb0(disc, nhat):
    """E_b0 at unit normals nhat [k][2] (Eq. eb0_disc)."""
    return np.abs(nhat @ disc.omega.T) @ disc.wq / (4.0 * math.pi)


def boundary_sums(disc, psi):
    """B(x_q) = sum_d w_d |Omega_d . n| psi_d(x_q) at the quadrature points of
    every boundary face: [n_bface][nfq]."""
    out = []
    for (e, f) in disc.bfaces:
        fd = disc.faces[e][f]
        nhat = fd["nds"] / np.linalg.norm(fd["nds"], axis=1)[:, None]
        a = np.abs(nhat @ disc.omega.T)              # [nfq][nd]
        vals = fd["V"] @ psi[:, e, :].T              # [nfq][nd]
        out.append(np.sum(a * vals * disc.wq[None, :], axis=1))
    return np.array(out)


def beta(disc, psi):
    """beta at boundary face quadrature points [n_bface][nfq]."""
    B = boundary_sums(disc, psi)
    phi = np.einsum("d,den->en", disc.wq, psi)
    out = np.zeros_like(B)
    for b, (e, f) in enumerate(disc.bfaces):
        fd = disc.faces[e][f]
        nhat = fd["nds"] / np.linalg.norm(fd["nds"], axis=1)[:, None]
        out[b] = B[b] - eb0(disc, nhat) * (fd["V"] @ phi[e])
    return out


def j_in(disc, psibar):
    """Incoming partial current at boundary face quadrature points
    [n_bface][nfq]; psibar: None or [nd][n_bface][p+1] face-node values."""
    nf = len(disc.elems[0].fq_s) if disc.ne else 0
    out = np.zeros((len(disc.bfaces), nf))
    if psibar is None:
        return out
    for b, (e, f) in enumerate(disc.bfaces):
        fd = disc.faces[e][f]
        nhat = fd["nds"] / np.linalg.norm(fd["nds"], axis=1)[:, None]
        on = nhat @ disc.omega.T                      # [nfq][nd]
        vals = np.stack([disc.L1 @ psibar[d][b] for d in range(disc.nd)], axis=1)
        out[b] = np.sum(np.where(on < 0.0, on, 0.0) * vals * disc.wq[None, :], axis=1)
    return out


def source_moments(disc, q):
    """Q_0 = sum_d w_d q_d and Q_1 = sum_d w_d Omega_d q_d, nodal [3][ne][n]."""
    q = np.asarray(q, float)
    if q.ndim == 2:
        q = np.broadcast_to(q, (disc.nd,) + q.shape)
    return np.stack([np.einsum("d,den->en", disc.wq, q),
                     np.einsum("d,den->en", disc.wq * disc.omega[:, 0], q),
                     np.einsum("d,den->en", disc.wq * disc.omega[:, 1], q)])
