"""Shared seeded inputs for GPU-vs-oracle parity tests.

Every array here comes from smm_workloads (the input generators); the
ordinate-dependent inputs are evaluated at the directions of whichever side
consumes them (the library's own quadrature for the GPU, the oracle's for the
oracle)."""
import math

import numpy as np

import smm_workloads as W


def problem(nx, ny=None, m=1, p=1, sn=4, seed=None, sigt=1.0, c=0.5, kind="mms", domain=(0.0, 1.0, 0.0, 1.0),
            fan=0.0):
    ny = nx if ny is None else ny
    mesh = W.structured_mesh(nx, ny, m=m, perturb_seed=seed, domain=domain, fan=fan)
    ne = mesh.n_elem
    st = np.broadcast_to(np.asarray(sigt, float), (ne,)).copy()
    ss = st * c
    pos = W.dg_node_positions(mesh, p)
    bf = W.boundary_faces(mesh)
    fpos = W.face_node_positions(mesh, p, bf)
    return dict(mesh=mesh, p=p, sn=sn, sigma_t=st, sigma_s=ss, pos=pos, bfaces=bf, fpos=fpos, kind=kind)


def sources(prob, omega):
    """(q, inflow) for directions omega [nd][2]."""
    pos, fpos = prob["pos"], prob["fpos"]
    st, ss = prob["sigma_t"], prob["sigma_s"]
    kind = prob["kind"]
    if kind == "mms":
        q = np.stack([W.mms_source(pos[:, :, 0], pos[:, :, 1], o[0], o[1], st[:, None], ss[:, None]) for o in omega])
        inflow = np.stack([W.mms_psi(fpos[:, :, 0], fpos[:, :, 1], o[0], o[1]) for o in omega])
        return q, inflow
    if kind == "linear":
        def qf(x, y, ox, oy):
            gx, gy = W.linear_aniso_grad_psi(x, y, ox, oy)
            phi = W.LIN_A + W.LIN_B * x + W.LIN_C * y
            return ox * gx + oy * gy + st[:, None] * W.linear_aniso_psi(x, y, ox, oy) - ss[:, None] / (4 * math.pi) * phi
        q = np.stack([qf(pos[:, :, 0], pos[:, :, 1], o[0], o[1]) for o in omega])
        inflow = np.stack([W.linear_aniso_psi(fpos[:, :, 0], fpos[:, :, 1], o[0], o[1]) for o in omega])
        return q, inflow
    if kind == "iso":
        return np.ones(pos.shape[:2]), None
    raise ValueError(kind)


def oracle_disc(prob):
    from oracle.transport import Discretization
    mesh = prob["mesh"]
    return Discretization(mesh.nodes, mesh.elem_nodes, mesh.m, prob["p"], prob["sn"], prob["sigma_t"], prob["sigma_s"])
