"""Problem builders for oracle tests (inputs from smm_workloads only)."""
import math

import numpy as np

import smm_workloads as W
from oracle.transport import Discretization


def disc_for(mesh, p, sn, sigt, sigs):
    ne = mesh.n_elem
    st = np.broadcast_to(np.asarray(sigt, float), (ne,)).copy()
    ss = np.broadcast_to(np.asarray(sigs, float), (ne,)).copy()
    return Discretization(mesh.nodes, mesh.elem_nodes, mesh.m, p, sn, st, ss)


def angular_source(disc, func):
    """[nd][ne][n] nodal values of func(x, y, ox, oy)."""
    return np.stack([disc.interpolate(lambda x, y, o=o: func(x, y, o[0], o[1])) for o in disc.omega])


def inflow(mesh, disc, func):
    bf = W.boundary_faces(mesh)
    fp = W.face_node_positions(mesh, disc.p, bf)
    return np.stack([func(fp[:, :, 0], fp[:, :, 1], o[0], o[1]) for o in disc.omega])


def mms_problem(nx, m, p, sn, seed, sigt=1.0, sigs=0.9):
    mesh = W.structured_mesh(nx, m=m, perturb_seed=seed)
    disc = disc_for(mesh, p, sn, sigt, sigs)
    q = angular_source(disc, lambda x, y, ox, oy: W.mms_source(x, y, ox, oy, sigt, sigs))
    pb = inflow(mesh, disc, W.mms_psi)
    return mesh, disc, q, pb


def linear_problem(nx, m, p, sn, seed=None, sigt=1.0, sigs=0.5):
    mesh = W.structured_mesh(nx, m=m, perturb_seed=seed)
    disc = disc_for(mesh, p, sn, sigt, sigs)

    def qf(x, y, ox, oy):
        gx, gy = W.linear_aniso_grad_psi(x, y, ox, oy)
        phi = W.LIN_A + W.LIN_B * x + W.LIN_C * y
        return ox * gx + oy * gy + sigt * W.linear_aniso_psi(x, y, ox, oy) - sigs / (4 * math.pi) * phi

    q = angular_source(disc, qf)
    pb = inflow(mesh, disc, W.linear_aniso_psi)
    phi_ex = disc.interpolate(lambda x, y: W.LIN_A + W.LIN_B * x + W.LIN_C * y)
    return mesh, disc, q, pb, phi_ex
