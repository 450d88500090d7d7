"""The SMM fixed-point map and its iteration (oracle).

Eq. moment:smm_fp: G(varphi) = D^{-1} b(L^{-1}(sigma_s/(4 pi) varphi + q)),
applied in two stages (a sweep, then the moment solve with closures from
that sweep), and Eq. fixed-point: varphi^{k+1} = G(varphi^k), stopped when
the max norm of the difference between successive iterates is below the
tolerance (Sec. "Results": the KINSOL criterion).  The initial guess is
unstated in the paper; zero is used.

Also: plain source iteration for the S_N equations (the transport fixed
point the SMM solution approaches as the mesh is refined, Sec. "Spatial
Convergence to S_N Solution"), and a dense solve of the coupled linear
transport + SMM system on tiny meshes.
"""
from __future__ import annotations

import numpy as np

from . import closures, ipsmm
from .transport import Discretization


class SMMProblem:
    """A discretization plus its data: q (per steradian, isotropic [ne][n]
    or angular [nd][ne][n]) and inflow psibar ([nd][n_bface][p+1] or None)."""

    def __init__(self, disc: Discretization, q, psibar=None, kappa_scale=1.0, fixup=False, tiles=1):
        self.disc = disc
        self.q = np.asarray(q, float)
        self.psibar = psibar
        self.fixup = fixup
        # parallel block Jacobi sweep: tile ids; the previous sweep's psi (zero at first) feeds
        # lagged inflow (between tiles, or closing a cycle)
        self.block = disc.element_tiles(tiles) if tiles > 1 else None
        self.psi_prev = np.zeros((disc.nd, disc.ne, disc.n))
        self.A = ipsmm.assemble_lhs(disc, kappa_scale)
        self.Q = closures.source_moments(disc, self.q)
        self.jin = closures.j_in(disc, psibar)

    def rhs_from_psi(self, psi):
        T = closures.nodal_moments(self.disc, psi)[3:6]
        beta = closures.beta(self.disc, psi)
        return ipsmm.assemble_rhs(self.disc, self.Q, T, self.jin, beta)

    def G(self, varphi):
        """One application of the fixed-point map; returns (varphi_new, psi)."""
        psi = self.disc.sweep(varphi, self.q, self.psibar, self.fixup, self.block, self.psi_prev)
        self.psi_prev = psi
        b = self.rhs_from_psi(psi)
        x = ipsmm.solve(self.A, b)
        return x.reshape(self.disc.ne, self.disc.n), psi

    def iterate(self, tol=1e-6, max_outer=200, relative=False, varphi0=None):
        """Fixed-point iteration; returns (varphi, iterations, history)."""
        ne, n = self.disc.ne, self.disc.n
        phi = np.zeros((ne, n)) if varphi0 is None else np.array(varphi0, float)
        hist = []
        for k in range(1, max_outer + 1):
            new, _ = self.G(phi)
            diff = float(np.max(np.abs(new - phi)))
            if relative:
                diff /= max(float(np.max(np.abs(new))), 1e-300)
            hist.append(diff)
            phi = new
            if diff < tol:
                return phi, k, hist
        return phi, max_outer, hist


def source_iteration(disc: Discretization, q, psibar=None, tol=1e-10, max_iter=10000):
    """S_N source iteration phi^{k+1} = sum_d w_d [L^{-1}(sigma_s/4pi phi^k + q)]_d."""
    phi = np.zeros((disc.ne, disc.n))
    for k in range(1, max_iter + 1):
        psi = disc.sweep(phi, q, psibar)
        new = np.einsum("d,den->en", disc.wq, psi)
        diff = float(np.max(np.abs(new - phi)))
        phi = new
        if diff < tol:
            return phi, k
    return phi, max_iter


def coupled_dense_solve(prob: SMMProblem):
    """Solve the coupled linear system {L psi = sigma_s/(4pi) varphi + q,
    D varphi = b(psi)} in one dense LU.  The maps varphi -> L^{-1}(...)
    (each ordinate's whole DG system solved at once, so cycles of the upwind
    graph need no lagging) and psi -> b(psi) are affine; their matrices are
    built column by column from unit vectors.  Tiny meshes only."""
    disc = prob.disc
    ne, n, nd = disc.ne, disc.n, disc.nd
    npsi, nphi = nd * ne * n, ne * n
    # affine transport map: psi = S varphi + s0
    zero_q = np.zeros_like(prob.q)
    s0 = disc.solve_global(None, prob.q, prob.psibar).ravel()
    S = np.zeros((npsi, nphi))
    for j in range(nphi):
        e_j = np.zeros(nphi)
        e_j[j] = 1.0
        S[:, j] = disc.solve_global(e_j.reshape(ne, n), zero_q, None).ravel()
    # affine closure map: b = R psi + r0
    r0 = prob.rhs_from_psi(np.zeros((nd, ne, n)))
    R = np.zeros((nphi, npsi))
    saved_q, saved_jin = prob.Q, prob.jin
    prob.Q = np.zeros_like(saved_q)
    prob.jin = np.zeros_like(saved_jin)
    for j in range(npsi):
        e_j = np.zeros(npsi)
        e_j[j] = 1.0
        R[:, j] = prob.rhs_from_psi(e_j.reshape(nd, ne, n))
    prob.Q, prob.jin = saved_q, saved_jin
    # D varphi = R (S varphi + s0) + r0
    Dm = prob.A.toarray()
    phi = np.linalg.solve(Dm - R @ S, R @ s0 + r0)
    return phi.reshape(ne, n)
