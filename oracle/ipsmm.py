"""Interior penalty SMM moment system (oracle), Eq. ipsmm.

Find varphi in Y_p such that for all u in Y_p

  int_Gb E_b0 u varphi + int_G0 kappa [u][varphi] - int_G0 [u]{D grad varphi . n}
  - int_G0 {D grad u . n}[varphi] + int grad u . D grad varphi + int sigma_a u varphi
 = int u Q_0 + int grad u . Q_1/sigma_t - int_G0 [u]{Q_1 . n/sigma_t}
  - int_Gb u (2 J_in + beta) + int_G0 [u]{(1/sigma_t) div_h T . n}
  + int_G0 {grad u/sigma_t} . [T n] - int grad u . (1/sigma_t) div_h T

with D = 1/(3 sigma_t), sigma_a = sigma_t - sigma_s, n pointing from K1 to
K2 on interior faces, [u] = u1 - u2, {u} = (u1 + u2)/2 (Sec. "Description of
the Mesh").  The penalty is kappa = {(p+1)^2 / (sigma_t h)} (Sec. "Results");
the paper does not define h: this oracle takes h_K = |K| / (longest face of
K).  ``kappa_scale`` multiplies kappa (the paper uses 169 on its triple
point mesh).

The matrix is assembled face by face in scipy.sparse and solved directly.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .closures import eb0
from .fem import face_point, tensor_basis


def _nbr_face_grad(disc, e, f):
    """Physical gradients of the neighbour's basis at this face's points."""
    e2, f2, flip = disc.nbr[e][f]
    el2 = disc.elems[e2]
    s = disc.elems[e].fq_s
    s2 = 1.0 - s if flip else s
    xi2, eta2 = face_point(f2, s2)
    _, F2 = el2.map(xi2, eta2)
    V2, Gh2 = tensor_basis(el2.gp, xi2, eta2)
    return V2, el2.phys_grad(F2, Gh2)


def element_h(disc, e):
    el = disc.elems[e]
    longest = max(float(np.sum(np.linalg.norm(disc.faces[e][f]["nds"], axis=1))) for f in range(4))
    return el.area() / longest


def interior_faces(disc):
    """Unique interior faces as (e1, f1): the element with the smaller
    index owns the face and its outward normal is n."""
    out = []
    for e in range(disc.ne):
        for f in range(4):
            nb = disc.nbr[e][f]
            if nb is not None and e < nb[0]:
                out.append((e, f))
    return out


def assemble_lhs(disc, kappa_scale=1.0):
    n, ne, p = disc.n, disc.ne, disc.p
    rows, cols, vals = [], [], []

    def add(block, r0, c0):
        r, c = np.meshgrid(np.arange(block.shape[0]) + 0, np.arange(block.shape[1]) + 0, indexing="ij")
        rows.append((r + r0).ravel())
        cols.append((c + c0).ravel())
        vals.append(block.ravel())

    st, ss = disc.sigma_t, disc.sigma_s
    for e, el in enumerate(disc.elems):
        K = el.stiffness()
        D = 1.0 / (3.0 * st[e])
        add(D * (K[0, 0] + K[1, 1]) + (st[e] - ss[e]) * disc.M[e], e * n, e * n)
    hK = [element_h(disc, e) for e in range(ne)]
    for (e, f) in interior_faces(disc):
        e2 = disc.nbr[e][f][0]
        fd = disc.faces[e][f]
        nds = fd["nds"]
        ds = np.linalg.norm(nds, axis=1)
        V1, G1 = fd["V"], fd["G"]
        V2, G2 = _nbr_face_grad(disc, e, f)
        D1, D2 = 1.0 / (3.0 * st[e]), 1.0 / (3.0 * st[e2])
        U = np.concatenate([V1, -V2], axis=1)
        Gn = np.concatenate([0.5 * D1 * np.einsum("qjc,qc->qj", G1, nds),
                             0.5 * D2 * np.einsum("qjc,qc->qj", G2, nds)], axis=1)
        kappa = kappa_scale * 0.5 * ((p + 1) ** 2 / (st[e] * hK[e]) + (p + 1) ** 2 / (st[e2] * hK[e2]))
        Af = kappa * U.T @ (ds[:, None] * U) - U.T @ Gn - Gn.T @ U
        idx = np.concatenate([np.arange(n) + e * n, np.arange(n) + e2 * n])
        r, c = np.meshgrid(idx, idx, indexing="ij")
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(Af.ravel())
    for (e, f) in disc.bfaces:
        fd = disc.faces[e][f]
        ds = np.linalg.norm(fd["nds"], axis=1)
        nhat = fd["nds"] / ds[:, None]
        E = eb0(disc, nhat)
        add(fd["V"].T @ ((E * ds)[:, None] * fd["V"]), e * n, e * n)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(ne * n, ne * n)).tocsr()
    return A


def _div_T(G, T):
    """div T at points from nodal T = (Txx, Txy, Tyy) and gradients G [q][n][2]."""
    txx, txy, tyy = T
    dx = G[:, :, 0] @ txx + G[:, :, 1] @ txy
    dy = G[:, :, 0] @ txy + G[:, :, 1] @ tyy
    return np.stack([dx, dy], axis=1)


def assemble_rhs(disc, Q, T, jin, beta):
    """Q: [3][ne][n] nodal (Q_0, Q_1x, Q_1y); T: [3][ne][n] nodal
    (Txx, Txy, Tyy); jin, beta: [n_bface][nfq] at face quadrature points."""
    n, ne = disc.n, disc.ne
    st = disc.sigma_t
    b = np.zeros(ne * n)
    for e, el in enumerate(disc.elems):
        wJ = el.w * el.J
        q1 = np.stack([el.V @ Q[1][e], el.V @ Q[2][e]], axis=1)
        dT = _div_T(el.G, (T[0][e], T[1][e], T[2][e]))
        b[e * n:(e + 1) * n] += disc.M[e] @ Q[0][e]
        b[e * n:(e + 1) * n] += np.einsum("q,qic,qc->i", wJ, el.G, (q1 - dT) / st[e])
    for (e, f) in interior_faces(disc):
        e2 = disc.nbr[e][f][0]
        fd = disc.faces[e][f]
        nds = fd["nds"]
        V1, G1 = fd["V"], fd["G"]
        V2, G2 = _nbr_face_grad(disc, e, f)
        T1 = (T[0][e], T[1][e], T[2][e])
        T2 = (T[0][e2], T[1][e2], T[2][e2])
        v1 = (np.stack([_div_T(G1, T1)[:, 0] - V1 @ Q[1][e], _div_T(G1, T1)[:, 1] - V1 @ Q[2][e]], axis=1)) / st[e]
        v2 = (np.stack([_div_T(G2, T2)[:, 0] - V2 @ Q[1][e2], _div_T(G2, T2)[:, 1] - V2 @ Q[2][e2]], axis=1)) / st[e2]
        g = 0.5 * np.sum((v1 + v2) * nds, axis=1)                       # {(divT - Q1).n/sigma_t} ds
        t1 = [V1 @ t for t in T1]
        t2 = [V2 @ t for t in T2]
        jx = (t1[0] - t2[0]) * nds[:, 0] + (t1[1] - t2[1]) * nds[:, 1]  # [T n] ds, x
        jy = (t1[1] - t2[1]) * nds[:, 0] + (t1[2] - t2[2]) * nds[:, 1]
        tj = np.stack([jx, jy], axis=1)
        b[e * n:(e + 1) * n] += V1.T @ g + 0.5 * np.einsum("qic,qc->i", G1, tj) / st[e]
        b[e2 * n:(e2 + 1) * n] += -V2.T @ g + 0.5 * np.einsum("qic,qc->i", G2, tj) / st[e2]
    for bi, (e, f) in enumerate(disc.bfaces):
        fd = disc.faces[e][f]
        ds = np.linalg.norm(fd["nds"], axis=1)
        b[e * n:(e + 1) * n] -= fd["V"].T @ (ds * (2.0 * jin[bi] + beta[bi]))
    return b


def solve(A, b):
    """Direct solution of the assembled SPD system."""
    return spla.spsolve(A.tocsc(), b)
