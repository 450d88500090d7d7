"""Mapped Q_p finite elements on curved quadrilaterals (oracle).

Follows Sec. "Finite Element Preliminaries":

* the element map x(xi) = sum_i x_{K,i} l_i(xi) with l_i the Lagrange
  polynomials on the (m+1)^2 Gauss-Lobatto points of [0,1]^2 ("Description
  of the Mesh");
* F = dx/dxi, J = det F, grad u = F^{-T} grad_hat u, int_K = int_Khat (.) J
  ("Integration Transformations");
* Y_p: mapped Q_p with a nodal basis, discontinuous across elements
  ("Discontinuous Galerkin").  The paper is silent on the DG nodes; this
  oracle uses Gauss-Lobatto nodes so a face trace is p+1 nodal values.

Quadrature: n_q = p + m + 1 Gauss-Legendre points per direction in volume
and on faces.
"""
from __future__ import annotations

import numpy as np

from .quadrature import gauss_legendre, gauss_lobatto


def lagrange(nodes: np.ndarray, x: np.ndarray):
    """Values V[len(x)][len(nodes)] and derivatives D of the Lagrange
    polynomials through ``nodes`` at points ``x`` (product formula)."""
    nodes = np.asarray(nodes, float)
    x = np.atleast_1d(np.asarray(x, float))
    k = len(nodes)
    V = np.ones((len(x), k))
    D = np.zeros((len(x), k))
    for a in range(k):
        for b in range(k):
            if b == a:
                continue
            V[:, a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
        # derivative: sum over the dropped factor
        for c in range(k):
            if c == a:
                continue
            term = np.full(len(x), 1.0 / (nodes[a] - nodes[c]))
            for b in range(k):
                if b == a or b == c:
                    continue
                term *= (x - nodes[b]) / (nodes[a] - nodes[b])
            D[:, a] += term
    return V, D


def tensor_basis(nodes1d, xi, eta):
    """Q_k nodal basis on [0,1]^2 at points (xi, eta): values [npts][(k+1)^2]
    and reference gradients [npts][(k+1)^2][2]; index i = iy*(k+1)+ix."""
    Vx, Dx = lagrange(nodes1d, xi)
    Vy, Dy = lagrange(nodes1d, eta)
    k1 = len(nodes1d)
    n = k1 * k1
    npts = len(np.atleast_1d(xi))
    V = np.empty((npts, n))
    G = np.empty((npts, n, 2))
    for iy in range(k1):
        for ix in range(k1):
            i = iy * k1 + ix
            V[:, i] = Vx[:, ix] * Vy[:, iy]
            G[:, i, 0] = Dx[:, ix] * Vy[:, iy]
            G[:, i, 1] = Vx[:, ix] * Dy[:, iy]
    return V, G


# face f: reference point of parameter s
def face_point(f: int, s):
    s = np.asarray(s, float)
    if f == 0:
        return s, np.zeros_like(s)
    if f == 1:
        return np.ones_like(s), s
    if f == 2:
        return s, np.ones_like(s)
    if f == 3:
        return np.zeros_like(s), s
    raise ValueError(f)


def face_nodes(p: int, f: int) -> np.ndarray:
    """Indices of the p+1 nodal points on face f, in increasing s."""
    a = np.arange(p + 1)
    q = p + 1
    return {0: a, 1: a * q + p, 2: p * q + a, 3: a * q}[f]


# corner control-point indices of face f (s=0 end, s=1 end) for geometry order m
def face_corners(m: int, f: int):
    q = m + 1
    c00, c10, c01, c11 = 0, m, m * q, m * q + m
    return {0: (c00, c10), 1: (c10, c11), 2: (c01, c11), 3: (c00, c01)}[f]


class Element:
    """Geometry and quadrature data of one curved element."""

    def __init__(self, ctrl: np.ndarray, m: int, p: int):
        self.m, self.p = m, p
        self.ctrl = np.asarray(ctrl, float)  # [(m+1)^2][2]
        self.gm, _ = gauss_lobatto(m + 1)
        self.gp, _ = gauss_lobatto(p + 1)
        nq = p + m + 1
        self.nq = nq
        qx, qw = gauss_legendre(nq)
        self.fq_s, self.fq_w = qx, qw
        XI, ETA = np.meshgrid(qx, qx, indexing="xy")
        W = np.outer(qw, qw)
        self.xi, self.eta, self.w = XI.ravel(), ETA.ravel(), W.ravel()
        # geometry at volume points
        self.x, self.F = self.map(self.xi, self.eta)
        self.J = self.F[:, 0, 0] * self.F[:, 1, 1] - self.F[:, 0, 1] * self.F[:, 1, 0]
        # basis at volume points
        self.V, Gh = tensor_basis(self.gp, self.xi, self.eta)
        self.G = self.phys_grad(self.F, Gh)         # [nqv][n][2]

    def map(self, xi, eta):
        """Physical points [npts][2] and Jacobians F [npts][2][2]."""
        Vg, Gg = tensor_basis(self.gm, np.atleast_1d(xi), np.atleast_1d(eta))
        x = Vg @ self.ctrl
        # F_{cd} = sum_i x_{i,c} d l_i / d xi_d
        F = np.einsum("ic,qid->qcd", self.ctrl, Gg)
        return x, F

    @staticmethod
    def phys_grad(F, Gh):
        """grad u = F^{-T} grad_hat u at each point."""
        Finv = np.linalg.inv(F)                      # [npts][2][2]
        return np.einsum("qdc,qid->qic", Finv, Gh)   # (F^{-T})_{cd} = Finv_{dc}

    def face(self, f: int):
        """Face data at the face quadrature points of face f: reference
        points, physical points, scaled outward normals n |dx/ds| w, basis
        values [nfq][n] and physical gradients [nfq][n][2]."""
        s = self.fq_s
        xi, eta = face_point(f, s)
        x, F = self.map(xi, eta)
        # tangent dx/ds along the face
        t = F[:, :, 0] if f in (0, 2) else F[:, :, 1]
        if f in (0, 1):
            nvec = np.stack([t[:, 1], -t[:, 0]], axis=1)
        else:
            nvec = np.stack([-t[:, 1], t[:, 0]], axis=1)
        nds = nvec * self.fq_w[:, None]
        V, Gh = tensor_basis(self.gp, xi, eta)
        G = self.phys_grad(F, Gh)
        return dict(xi=xi, eta=eta, x=x, nds=nds, V=V, G=G)

    # element matrices (angle independent)
    def mass(self):
        """M_ij = int_K phi_i phi_j."""
        wJ = self.w * self.J
        return np.einsum("q,qi,qj->ij", wJ, self.V, self.V)

    def stream(self):
        """Gx_ij = int_K phi_j dphi_i/dx, Gy_ij likewise (i test, j trial)."""
        wJ = self.w * self.J
        Gx = np.einsum("q,qi,qj->ij", wJ, self.G[:, :, 0], self.V)
        Gy = np.einsum("q,qi,qj->ij", wJ, self.G[:, :, 1], self.V)
        return Gx, Gy

    def stiffness(self):
        """K^{ab}_ij = int_K dphi_i/da dphi_j/db for a, b in {x, y}."""
        wJ = self.w * self.J
        return np.einsum("q,qia,qjb->abij", wJ, self.G, self.G)

    def area(self):
        return float(np.sum(self.w * self.J))
