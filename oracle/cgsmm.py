"""Continuous finite element SMM moment system (oracle, test infrastructure).

Sec. 5.1 extracts a continuous Galerkin (CG) SMM method from Eq. ipsmm by
taking test and trial functions in V_p, the degree-p continuous space: jumps
of V_p functions vanish on interior faces and broken gradients are gradients,
so the penalty and the [u]-weighted face terms drop out.  Find varphi in V_p
such that for all u in V_p

  int_Gb E_b0 u varphi + int grad u . D grad varphi + int sigma_a u varphi
 = int u Q_0 + int grad u . Q_1/sigma_t - int_Gb u (2 J_in + beta)
   + int_G0 {grad u/sigma_t} . [T n] - int grad u . (1/sigma_t) div_h T

with D = 1/(3 sigma_t), [T n] = T_1 n - T_2 n (n pointing from K1 to K2).  The
correction tensor T is still discontinuous (it comes from the DG transport
solution), so the face term stays.

V_p is built on the DG elements' own Gauss-Lobatto nodal basis: a global node
is a class of element nodes identified across interior faces (the p+1 nodes
of a face with the matching nodes of the neighbour's face), so a V_p function
is a DG function whose values agree at identified nodes, and the injection
P: V_p -> Y_p copies the value of each global node to its element nodes.  The
scalar flux that drives the next sweep is P varphi.

The system is assembled element by element and face by face in scipy.sparse
and solved directly; every function here writes out the integrals above.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import closures
from .closures import eb0
from .fem import face_nodes
from .ipsmm import _div_T, _nbr_face_grad, interior_faces


def continuous_numbering(disc):
    """Global V_p node of every element node: (gid [ne][n], number of nodes).
    Element nodes are joined across every interior face, node a of face f of
    K1 with node a (or p - a if the face runs the other way) of the shared
    face of K2; global ids follow the first appearance in element order."""
    ne, n, p = disc.ne, disc.n, disc.p
    parent = list(range(ne * n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for e in range(ne):
        for f in range(4):
            nb = disc.nbr[e][f]
            if nb is None:
                continue
            e2, f2, flip = nb
            a1 = face_nodes(p, f)
            a2 = face_nodes(p, f2)
            for a in range(p + 1):
                r1 = find(e * n + int(a1[a]))
                r2 = find(e2 * n + int(a2[p - a if flip else a]))
                if r1 != r2:
                    parent[max(r1, r2)] = min(r1, r2)
    root_id = {}
    gid = np.empty((ne, n), dtype=np.int64)
    for k in range(ne * n):
        r = find(k)
        if r not in root_id:
            root_id[r] = len(root_id)
        gid[k // n, k % n] = root_id[r]
    return gid, len(root_id)


def injection(gid, nglob):
    """P: V_p -> Y_p as a sparse (ne n) x nglob 0/1 matrix."""
    ne, n = gid.shape
    return sp.csr_matrix((np.ones(ne * n), (np.arange(ne * n), gid.ravel())), shape=(ne * n, nglob))


def _scatter_matrix(blocks, gid, nglob):
    rows, cols, vals = [], [], []
    for e, B in blocks:
        g = gid[e]
        r, c = np.meshgrid(g, g, indexing="ij")
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(B.ravel())
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(nglob, nglob)).tocsr()


def assemble_lhs(disc, gid, nglob):
    """int_Gb E_b0 u varphi + int grad u . D grad varphi + int sigma_a u varphi on V_p."""
    st, ss = disc.sigma_t, disc.sigma_s
    blocks = []
    for e, el in enumerate(disc.elems):
        K = el.stiffness()
        blocks.append((e, (K[0, 0] + K[1, 1]) / (3.0 * st[e]) + (st[e] - ss[e]) * disc.M[e]))
    for (e, f) in disc.bfaces:
        fd = disc.faces[e][f]
        ds = np.linalg.norm(fd["nds"], axis=1)
        E = eb0(disc, fd["nds"] / ds[:, None])
        blocks.append((e, fd["V"].T @ ((E * ds)[:, None] * fd["V"])))
    return _scatter_matrix(blocks, gid, nglob)


def assemble_rhs(disc, gid, nglob, Q, T, jin, beta):
    """Right-hand side on V_p.  Q: [3][ne][n] nodal (Q_0, Q_1x, Q_1y); T: [3][ne][n]
    nodal (Txx, Txy, Tyy); jin, beta: [n_bface][nfq] at face quadrature points."""
    n = disc.n
    st = disc.sigma_t
    b = np.zeros(nglob)
    for e, el in enumerate(disc.elems):
        wJ = el.w * el.J
        q1 = np.stack([el.V @ Q[1][e], el.V @ Q[2][e]], axis=1)
        dT = _div_T(el.G, (T[0][e], T[1][e], T[2][e]))
        be = disc.M[e] @ Q[0][e] + np.einsum("q,qic,qc->i", wJ, el.G, (q1 - dT) / st[e])
        np.add.at(b, gid[e], be)
    for (e, f) in interior_faces(disc):
        e2 = disc.nbr[e][f][0]
        fd = disc.faces[e][f]
        nds = fd["nds"]
        V1, G1 = fd["V"], fd["G"]
        V2, G2 = _nbr_face_grad(disc, e, f)
        t1 = [V1 @ T[k][e] for k in range(3)]
        t2 = [V2 @ T[k][e2] for k in range(3)]
        # [T n] ds with n from K1 to K2: (T_1 - T_2) n ds
        jx = (t1[0] - t2[0]) * nds[:, 0] + (t1[1] - t2[1]) * nds[:, 1]
        jy = (t1[1] - t2[1]) * nds[:, 0] + (t1[2] - t2[2]) * nds[:, 1]
        tj = np.stack([jx, jy], axis=1)
        # {grad u / sigma_t} . [T n]: half from each side
        np.add.at(b, gid[e], 0.5 * np.einsum("qic,qc->i", G1, tj) / st[e])
        np.add.at(b, gid[e2], 0.5 * np.einsum("qic,qc->i", G2, tj) / st[e2])
    for bi, (e, f) in enumerate(disc.bfaces):
        fd = disc.faces[e][f]
        ds = np.linalg.norm(fd["nds"], axis=1)
        np.add.at(b, gid[e], -(fd["V"].T @ (ds * (2.0 * jin[bi] + beta[bi]))))
    return b


class SMMProblemCG:
    """The SMM fixed point with the CG moment system (same interface as
    oracle.smm.SMMProblem: varphi is carried as DG nodal values P varphi)."""

    def __init__(self, disc, q, psibar=None):
        self.disc = disc
        self.q = np.asarray(q, float)
        self.psibar = psibar
        self.gid, self.nglob = continuous_numbering(disc)
        self.P = injection(self.gid, self.nglob)
        self.A = assemble_lhs(disc, self.gid, self.nglob)
        self.Q = closures.source_moments(disc, self.q)
        self.jin = closures.j_in(disc, psibar)

    def rhs_from_psi(self, psi):
        T = closures.nodal_moments(self.disc, psi)[3:6]
        beta = closures.beta(self.disc, psi)
        return assemble_rhs(self.disc, self.gid, self.nglob, self.Q, T, self.jin, beta)

    def G(self, varphi):
        """One application of the fixed-point map; returns (P varphi_new as [ne][n], psi)."""
        psi = self.disc.sweep(varphi, self.q, self.psibar)
        x = spla.spsolve(self.A.tocsc(), self.rhs_from_psi(psi))
        return (self.P @ x).reshape(self.disc.ne, self.disc.n), psi

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
