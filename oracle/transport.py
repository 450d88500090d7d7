"""Upwind DG S_N transport discretization and sweep (oracle).

Sec. "Transport Discretization": each discrete-ordinate flux psi_d lies in
Y_p and the streaming + collision operator L is inverted by a transport
sweep.  The paper defers the DG transport scheme to the solvers it cites,
so this oracle states the standard upwind DG weak form: for ordinate d and
element K find psi in Q_p(K) such that for all v in Q_p(K)

    - int_K psi Omega_d . grad v + int_K sigma_t psi v
    + sum_F int_F max(Omega_d . n, 0) psi v
  = int_K s_d v - sum_F int_F min(Omega_d . n, 0) psi^up v,

with n the outward normal of K, the sign taken pointwise at face
quadrature points, psi^up the upwind neighbour's trace or the inflow
function psibar on the domain boundary (Eq. inflow), and
s_d = sigma_s/(4 pi) varphi + q_d (Eq. moment_coupled, first line).

Elements are visited in a topological order of each ordinate's upwind
graph (a neighbour is upwind if Omega_d . n < 0 at any point of the shared
face, so a face that is inflow at some points and outflow at others makes
its two elements depend on each other).  Cycles are lagged, as Sec. 6.2
does on its distorted mesh: whenever no element is left whose upwind
neighbours are all done, the lowest-numbered remaining element is taken
next and its inflow from the neighbours not yet done comes from the
previous sweep (psi_lag; zero if none is given).  Each local system is
solved by dense LU with partial pivoting.
"""
from __future__ import annotations

import heapq
import math

import numpy as np

from .fem import Element, face_corners, face_nodes, face_point, lagrange, tensor_basis
from .quadrature import gauss_lobatto, level_symmetric_2d


def zero_and_scale(A, x):
    """Zero and scale negative flux fixup of one element solution (the fixup
    Sec. 6.3 uses inside the sweep, cited there, not printed): negative nodal
    values are set to zero and the rest scaled so that the element's particle
    balance -- the local system tested with v = 1, sum_i (A x)_i, i.e.
    outflow + collisions -- keeps its value; if that value is not positive
    the element flux is set to zero."""
    if np.all(x >= 0.0):
        return x
    c = A.sum(axis=0)                 # balance functional 1^T A
    pos = np.maximum(x, 0.0)
    t, tp = float(c @ x), float(c @ pos)
    if t <= 0.0 or tp <= 0.0:
        return np.zeros_like(x)
    return (t / tp) * pos


class CycleError(RuntimeError):
    pass


class Discretization:
    """Mesh, finite elements, quadrature and per-element matrices."""

    def __init__(self, nodes, elem_nodes, m: int, p: int, sn: int, sigma_t, sigma_s):
        nodes = np.asarray(nodes, float)
        elem_nodes = np.asarray(elem_nodes)
        self.m, self.p, self.sn = m, p, sn
        self.n = (p + 1) ** 2
        self.ne = len(elem_nodes)
        self.sigma_t = np.asarray(sigma_t, float)
        self.sigma_s = np.asarray(sigma_s, float)
        self.omega, self.wq = level_symmetric_2d(sn)
        self.nd = len(self.wq)
        self.elems = [Element(nodes[elem_nodes[e]], m, p) for e in range(self.ne)]
        self.faces = [[el.face(f) for f in range(4)] for el in self.elems]
        self.M = [el.mass() for el in self.elems]
        st = [el.stream() for el in self.elems]
        self.Gx = [g[0] for g in st]
        self.Gy = [g[1] for g in st]
        # connectivity from shared corner control points
        owner = {}
        for e in range(self.ne):
            for f in range(4):
                c0, c1 = face_corners(m, f)
                key = frozenset((int(elem_nodes[e, c0]), int(elem_nodes[e, c1])))
                owner.setdefault(key, []).append((e, f))
        self.nbr = [[None] * 4 for _ in range(self.ne)]
        for key, lst in owner.items():
            if len(lst) == 2:
                (e1, f1), (e2, f2) = lst
                a1 = int(elem_nodes[e1, face_corners(m, f1)[0]])
                a2 = int(elem_nodes[e2, face_corners(m, f2)[0]])
                flip = a1 != a2
                self.nbr[e1][f1] = (e2, f2, flip)
                self.nbr[e2][f2] = (e1, f1, flip)
            elif len(lst) > 2:
                raise ValueError("non-manifold face")
        self.bfaces = [(e, f) for e in range(self.ne) for f in range(4) if self.nbr[e][f] is None]
        self.bindex = {ef: b for b, ef in enumerate(self.bfaces)}
        # neighbour basis at this face's quadrature points (matching points)
        self.Vnb = [[None] * 4 for _ in range(self.ne)]
        gp, _ = gauss_lobatto(p + 1)
        for e in range(self.ne):
            for f in range(4):
                if self.nbr[e][f] is None:
                    continue
                e2, f2, flip = self.nbr[e][f]
                s = self.elems[e].fq_s
                s2 = 1.0 - s if flip else s
                xi2, eta2 = face_point(f2, s2)
                V2, _ = tensor_basis(gp, xi2, eta2)
                self.Vnb[e][f] = V2
        # 1D Lagrange (face nodes) at face quadrature points, for inflow data
        self.L1, _ = lagrange(gp, self.elems[0].fq_s) if self.ne else (None, None)

    # -- upwind graph -------------------------------------------------------
    def element_tiles(self, tiles: int):
        """Tile of every element for the parallel block Jacobi sweep: the
        mesh's bounding box cut into tiles x tiles equal rectangles, an
        element belonging to the rectangle holding the mean of its four
        corner control points (ids by * tiles + bx)."""
        ctrl = np.array([el.ctrl for el in self.elems])          # [ne][(m+1)^2][2]
        m = self.m
        corners = ctrl[:, [0, m, m * (m + 1), m * (m + 1) + m], :].mean(axis=1)
        allp = ctrl.reshape(-1, 2)
        lo, hi = allp.min(axis=0), allp.max(axis=0)
        t = np.minimum(((corners - lo) / (hi - lo) * tiles).astype(int), tiles - 1)
        return t[:, 1] * tiles + t[:, 0]

    def upwind_order(self, d: int, block=None, lag_cycles=True):
        """(order, lagged): a topological order of the elements for ordinate
        d (smallest index first among ready elements) and the set of (e, f)
        whose inflow is lagged.  With a tile array, upwind neighbours in
        another tile are not dependencies (their values are lagged).  A cycle
        is broken by taking the lowest-numbered remaining element and lagging
        its pending inflow faces; with lag_cycles=False it raises CycleError."""
        if not hasattr(self, "_orders"):
            self._orders = {}
        key = (d, None if block is None else tuple(block), lag_cycles)
        if key not in self._orders:
            self._orders[key] = self._topological_order(d, block, lag_cycles)
        return self._orders[key]

    def upwind_faces(self, e: int, d: int):
        """Faces of element e through which ordinate d enters at some point
        from a neighbour (the element's upwind dependencies)."""
        out = []
        for f in range(4):
            nb = self.nbr[e][f]
            if nb is not None and np.any(self.faces[e][f]["nds"] @ self.omega[d] < 0.0):
                out.append((f, nb[0]))
        return out

    def _topological_order(self, d: int, block=None, lag_cycles=True):
        lagged = set()
        deps = [{} for _ in range(self.ne)]      # upwind neighbour -> faces of e toward it
        for e in range(self.ne):
            for f, u in self.upwind_faces(e, d):
                if block is not None and block[u] != block[e]:
                    lagged.add((e, f))
                    continue
                deps[e].setdefault(u, []).append(f)
        indeg = [len(s) for s in deps]
        down = [[] for _ in range(self.ne)]
        for e in range(self.ne):
            for u in deps[e]:
                down[u].append(e)
        ready = [e for e in range(self.ne) if indeg[e] == 0]
        heapq.heapify(ready)
        order, done = [], [False] * self.ne
        while len(order) < self.ne:
            if not ready:
                if not lag_cycles:
                    raise CycleError(f"upwind graph of ordinate {d} has a cycle")
                v = min(e for e in range(self.ne) if not done[e])
                for u, faces in deps[v].items():
                    if not done[u]:
                        lagged.update((v, f) for f in faces)
                        down[u].remove(v)
                indeg[v] = 0
                heapq.heappush(ready, v)
            u = heapq.heappop(ready)
            done[u] = True
            order.append(u)
            for v in down[u]:
                indeg[v] -= 1
                if indeg[v] == 0:
                    heapq.heappush(ready, v)
        return order, lagged
        om = self.omega[d]
        deps = [set() for _ in range(self.ne)]
        for e in range(self.ne):
            for f in range(4):
                nb = self.nbr[e][f]
                if nb is None:
                    continue
                if block is not None and block[nb[0]] != block[e]:
                    continue
                a = self.faces[e][f]["nds"] @ om
                if np.any(a < 0.0):
                    deps[e].add(nb[0])
        indeg = [len(s) for s in deps]
        down = [[] for _ in range(self.ne)]
        for e in range(self.ne):
            for u in deps[e]:
                down[u].append(e)
        ready = [e for e in range(self.ne) if indeg[e] == 0]
        heapq.heapify(ready)
        order = []
        while ready:
            u = heapq.heappop(ready)
            order.append(u)
            for v in down[u]:
                indeg[v] -= 1
                if indeg[v] == 0:
                    heapq.heappush(ready, v)
        if len(order) != self.ne:
            raise CycleError(f"upwind graph of ordinate {d} has a cycle")
        return order

    # -- local system -------------------------------------------------------
    def local_matrix(self, e: int, d: int):
        """A_{K,d}: streaming + collision + outflow face terms."""
        ox, oy = self.omega[d]
        A = self.sigma_t[e] * self.M[e] - ox * self.Gx[e] - oy * self.Gy[e]
        for f in range(4):
            fd = self.faces[e][f]
            a = fd["nds"] @ self.omega[d]
            A = A + fd["V"].T @ (np.maximum(a, 0.0)[:, None] * fd["V"])
        return A

    def upwind_values(self, e, f, d, psi, psibar):
        """psi^up at the quadrature points of face f of element e."""
        nb = self.nbr[e][f]
        if nb is not None:
            return self.Vnb[e][f] @ psi[nb[0]]
        if psibar is None:
            return np.zeros(len(self.elems[e].fq_s))
        return self.L1 @ psibar[d][self.bindex[(e, f)]]

    def sweep_ordinate(self, d: int, src, psibar=None, fixup=False, block=None, psi_lag=None):
        """Solve L psi_d = src_d with inflow psibar; src: [ne][n] nodal
        values of the total source for this ordinate; psibar: None (vacuum)
        or [nd][n_bface][p+1] face-node values.  fixup: apply the zero and
        scale negative flux fixup to every element solution before it is
        passed downwind.  psi_lag [ne][n] (the previous sweep; zero if None)
        feeds the lagged faces: those that close a cycle, and, with a tile
        array (parallel block Jacobi sweep, Sec. 6.5), those from another
        tile."""
        psi = np.zeros((self.ne, self.n))
        order, lagset = self.upwind_order(d, block)
        if psi_lag is None:
            psi_lag = np.zeros((self.ne, self.n))
        for e in order:
            A = self.local_matrix(e, d)
            b = self.M[e] @ src[e]
            for f in range(4):
                fd = self.faces[e][f]
                a = fd["nds"] @ self.omega[d]
                neg = np.minimum(a, 0.0)
                if np.any(neg < 0.0):
                    up = self.upwind_values(e, f, d, psi_lag if (e, f) in lagset else psi, psibar)
                    b = b - fd["V"].T @ (neg * up)
            psi[e] = np.linalg.solve(A, b)
            if fixup:
                psi[e] = zero_and_scale(A, psi[e])
        return psi

    def scattering_source(self, varphi):
        """sigma_s/(4 pi) varphi per element node (zero for varphi None)."""
        if varphi is None:
            return np.zeros((self.ne, self.n))
        return (self.sigma_s / (4.0 * math.pi))[:, None] * np.asarray(varphi, float)

    def sweep(self, varphi, q, psibar=None, fixup=False, block=None, psi_lag=None):
        """psi = L^{-1}(sigma_s/(4 pi) varphi + q) for all ordinates.

        varphi: [ne][n] nodal scalar flux (or None for zero);
        q: [ne][n] isotropic or [nd][ne][n] angular source per steradian.
        Returns psi [nd][ne][n]."""
        q = np.asarray(q, float)
        out = np.zeros((self.nd, self.ne, self.n))
        scat = self.scattering_source(varphi)
        for d in range(self.nd):
            qd = q if q.ndim == 2 else q[d]
            out[d] = self.sweep_ordinate(d, scat + qd, psibar, fixup, block,
                                         None if psi_lag is None else psi_lag[d])
        return out

    # -- global assembly of one ordinate's DG system (brute force check) ------
    def global_ordinate_matrix(self, d: int):
        """Dense matrix of the whole single-ordinate DG system (all elements
        coupled through upwind face terms): row block e, column block of the
        upwind neighbour holds + int_F min(Omega.n,0) psi_nb v."""
        n, ne = self.n, self.ne
        A = np.zeros((ne * n, ne * n))
        for e in range(ne):
            A[e * n:(e + 1) * n, e * n:(e + 1) * n] = self.local_matrix(e, d)
            for f in range(4):
                nb = self.nbr[e][f]
                if nb is None:
                    continue
                fd = self.faces[e][f]
                neg = np.minimum(fd["nds"] @ self.omega[d], 0.0)
                A[e * n:(e + 1) * n, nb[0] * n:(nb[0] + 1) * n] += fd["V"].T @ (neg[:, None] * self.Vnb[e][f])
        return A

    def global_ordinate_rhs(self, d: int, src, psibar=None):
        n, ne = self.n, self.ne
        b = np.zeros(ne * n)
        zero = np.zeros((ne, n))
        for e in range(ne):
            b[e * n:(e + 1) * n] = self.M[e] @ src[e]
            for f in range(4):
                if self.nbr[e][f] is not None:
                    continue
                fd = self.faces[e][f]
                neg = np.minimum(fd["nds"] @ self.omega[d], 0.0)
                up = self.upwind_values(e, f, d, zero, psibar)
                b[e * n:(e + 1) * n] -= fd["V"].T @ (neg * up)
        return b

    def solve_global(self, varphi, q, psibar=None):
        """psi = L^{-1}(sigma_s/(4 pi) varphi + q) with each ordinate's whole
        DG system (global_ordinate_matrix) solved by dense LU: the transport
        solution the sweep computes when no inflow is lagged, and the fixed
        point of lagged sweeps otherwise.  Tiny meshes only."""
        q = np.asarray(q, float)
        out = np.zeros((self.nd, self.ne, self.n))
        scat = self.scattering_source(varphi)
        for d in range(self.nd):
            src = scat + (q if q.ndim == 2 else q[d])
            A = self.global_ordinate_matrix(d)
            out[d] = np.linalg.solve(A, self.global_ordinate_rhs(d, src, psibar)).reshape(self.ne, self.n)
        return out

    # -- helpers --------------------------------------------------------------
    def interpolate(self, func):
        """Nodal values [ne][n] of func(x, y) at the physical nodal points
        (element map applied to the Gauss-Lobatto reference nodes)."""
        gp, _ = gauss_lobatto(self.p + 1)
        XI, ETA = np.meshgrid(gp, gp, indexing="xy")
        out = np.zeros((self.ne, self.n))
        for e, el in enumerate(self.elems):
            x, _ = el.map(XI.ravel(), ETA.ravel())
            out[e] = func(x[:, 0], x[:, 1])
        return out

    def l2_error(self, u, func):
        """|| u - func ||_{L2(D)} with the element quadrature."""
        s = 0.0
        for e, el in enumerate(self.elems):
            uq = el.V @ u[e]
            ex = func(el.x[:, 0], el.x[:, 1])
            s += np.sum(el.w * el.J * (uq - ex) ** 2)
        return math.sqrt(s)

    def integrate(self, u):
        return float(sum(np.sum(el.w * el.J * (el.V @ u[e])) for e, el in enumerate(self.elems)))

    def max_h(self):
        return max(math.sqrt(el.area()) for el in self.elems)
