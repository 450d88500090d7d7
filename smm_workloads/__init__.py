"""Seeded synthetic inputs for the SMM transport hot path.

This module is the only code shared by the CPU oracle (``oracle/``) and the
CUDA path (``paper_2304_07386_gb300``).  It produces *inputs* only: mesh
control points and connectivity, piecewise-constant cross sections, nodal
source values and inflow traces, and the manufactured solution of the
paper's MMS study (Sec. "Method of Manufactured Solutions", Eq. mms_psi).
It holds none of the method's arithmetic: no quadrature, no element
matrices, no sweep, no moments, no moment system.

Conventions shared by every consumer (they define the input format):

* Reference element [0,1]^2.  Nodal points of an order-k Lagrange element
  sit on the tensor product of the k+1 Gauss-Lobatto points of [0,1],
  numbered lexicographically with the x-index fastest: i = iy*(k+1) + ix.
* Structured meshes number elements e = j*nx + i (i along x, j along y).
* Faces of an element: 0 bottom (eta=0), 1 right (xi=1), 2 top (eta=1),
  3 left (xi=0).  Along each face the parameter s increases with the
  reference coordinate that varies on it.
* Boundary faces are enumerated by ascending (element, face).
* Discrete ordinates are numbered quadrant-major: quadrants (+,+), (-,+),
  (-,-), (+,-) in that order; inside a quadrant by the octant level
  triple (i, j, k), i ascending then j ascending.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "gauss_lobatto_points",
    "StructuredMesh",
    "structured_mesh",
    "dg_node_positions",
    "boundary_faces",
    "face_node_positions",
    "block_materials",
    "gaussian_random_field",
    "mms_psi",
    "mms_grad_psi",
    "mms_phi",
    "mms_source",
    "linear_aniso_psi",
    "linear_aniso_grad_psi",
]


# ---------------------------------------------------------------------------
# Node positions (where nodal input values live)
# ---------------------------------------------------------------------------

def gauss_lobatto_points(npts: int) -> np.ndarray:
    """The ``npts`` Gauss-Lobatto points on [0, 1] (endpoints included).

    Interior points are the roots of P'_{npts-1}; used here only to place
    mesh control points and nodal input values.
    """
    if npts < 2:
        raise ValueError("Gauss-Lobatto rule needs at least 2 points")
    if npts == 2:
        return np.array([0.0, 1.0])
    c = np.zeros(npts)
    c[-1] = 1.0
    inner = np.polynomial.legendre.Legendre(c).deriv().roots()
    inner = np.sort(np.real(inner))
    # polish the roots by Newton on P'_{n-1}
    leg = np.polynomial.legendre.Legendre(c)
    d1, d2 = leg.deriv(1), leg.deriv(2)
    for _ in range(3):
        inner = inner - d1(inner) / d2(inner)
    x = np.concatenate(([-1.0], inner, [1.0]))
    return 0.5 * (x + 1.0)


@dataclass
class StructuredMesh:
    """A structured nx*ny quad mesh of geometry order m on [x0,x1]x[y0,y1]."""

    nx: int
    ny: int
    m: int
    x0: float
    x1: float
    y0: float
    y1: float
    nodes: np.ndarray            # [n_nodes][2] float64
    elem_nodes: np.ndarray       # [n_elem][(m+1)^2] int32
    perturb: tuple = field(default=())  # ((ax,k1,k2),(ay,k3,k4)) or ()
    fan: float = 0.0             # x spread factor at the top edge (see structured_mesh)

    @property
    def n_elem(self) -> int:
        return self.nx * self.ny

    def map(self, x: np.ndarray, y: np.ndarray):
        """The analytic node map applied to straight-grid positions."""
        xt = (x - self.x0) / (self.x1 - self.x0)
        yt = (y - self.y0) / (self.y1 - self.y0)
        if self.perturb:
            (ax, k1, k2), (ay, k3, k4) = self.perturb
            xm = x + ax * np.sin(math.pi * k1 * xt) * np.sin(math.pi * k2 * yt)
            ym = y + ay * np.sin(math.pi * k3 * xt) * np.sin(math.pi * k4 * yt)
        else:
            xm, ym = x, y
        if self.fan:
            xc = 0.5 * (self.x0 + self.x1)
            xm = xc + (xm - xc) * (1.0 + self.fan * yt)
        return xm, ym


def _perturbation(seed: int, lx: float, ly: float, amplitude: float, wave_max: int = 2, scale_by_k: bool = True):
    """Seeded sinusoidal perturbation parameters.

    Wave numbers are drawn from {1, ..., wave_max}; the amplitude of each
    component is ``amplitude * L / max(k)`` (scale_by_k, so that the largest
    face tilt stays at about ``amplitude * pi`` radians whatever the draw) or
    ``amplitude * L``, with a random sign.
    """
    rng = np.random.default_rng(seed)
    k = rng.integers(1, wave_max + 1, size=4)
    s = rng.choice([-1.0, 1.0], size=2)
    ax = s[0] * amplitude * lx / (max(k[0], k[1]) if scale_by_k else 1)
    ay = s[1] * amplitude * ly / (max(k[2], k[3]) if scale_by_k else 1)
    return ((float(ax), int(k[0]), int(k[1])), (float(ay), int(k[2]), int(k[3])))


def structured_mesh(nx: int, ny: int | None = None, m: int = 1,
                    domain=(0.0, 1.0, 0.0, 1.0), *, perturb_seed: int | None = None,
                    amplitude: float = 0.05, wave_max: int = 2, scale_by_k: bool = True,
                    fan: float = 0.0) -> StructuredMesh:
    """Structured quad mesh with control points on GLL nodes of order ``m``.

    With ``perturb_seed`` the straight grid is moved by the seeded
    sinusoidal map x' = x + a_x sin(pi k1 x~) sin(pi k2 y~),
    y' = y + a_y sin(pi k3 x~) sin(pi k4 y~) (x~, y~ scaled to [0,1]), which
    leaves the domain boundary in place.  Shared control points make the
    mesh continuous.  wave_max = 3, scale_by_k = False gives wave numbers in
    {1, 2, 3} at amplitude a_x = amplitude * (x1 - x0), whose tilted faces can
    be inflow at some points and outflow at others for grazing ordinates.
    fan > 0 then spreads the columns as y grows, x' = x_c + (x - x_c)(1 + fan y~)
    (x_c the centre; bilinear, so exact at any geometry order): the elements
    become trapezoids that widen upwards, and an ordinate pointing up enters
    them through three straight faces.
    """
    ny = nx if ny is None else ny
    x0, x1, y0, y1 = map(float, domain)
    g = gauss_lobatto_points(m + 1)
    nxn, nyn = nx * m + 1, ny * m + 1
    hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
    # straight positions of the global control-point grid
    ix = np.arange(nxn)
    iy = np.arange(nyn)
    ex, ax_ = np.minimum(ix // m, nx - 1), ix - np.minimum(ix // m, nx - 1) * m
    ey, ay_ = np.minimum(iy // m, ny - 1), iy - np.minimum(iy // m, ny - 1) * m
    xs = x0 + (ex + g[ax_]) * hx
    ys = y0 + (ey + g[ay_]) * hy
    xs[-1], ys[-1] = x1, y1
    X, Y = np.meshgrid(xs, ys, indexing="xy")  # [nyn][nxn]
    pert = (_perturbation(perturb_seed, x1 - x0, y1 - y0, amplitude, wave_max, scale_by_k)
            if perturb_seed is not None else ())
    mesh = StructuredMesh(nx, ny, m, x0, x1, y0, y1, np.zeros((0, 2)), np.zeros((0, 0), np.int32), pert, float(fan))
    Xm, Ym = mesh.map(X, Y)
    nodes = np.stack([Xm.ravel(), Ym.ravel()], axis=1).astype(np.float64)
    en = np.empty((nx * ny, (m + 1) ** 2), dtype=np.int32)
    for j in range(ny):
        for i in range(nx):
            e = j * nx + i
            for b in range(m + 1):
                for a in range(m + 1):
                    en[e, b * (m + 1) + a] = (j * m + b) * nxn + (i * m + a)
    mesh.nodes = nodes
    mesh.elem_nodes = en
    return mesh


def dg_node_positions(mesh: StructuredMesh, p: int) -> np.ndarray:
    """Physical positions [n_elem][(p+1)^2][2] of the order-p nodal points,
    obtained by applying the analytic node map to the straight grid."""
    g = gauss_lobatto_points(p + 1)
    hx = (mesh.x1 - mesh.x0) / mesh.nx
    hy = (mesh.y1 - mesh.y0) / mesh.ny
    out = np.empty((mesh.n_elem, (p + 1) ** 2, 2))
    gx, gy = np.meshgrid(g, g, indexing="xy")
    gx, gy = gx.ravel(), gy.ravel()
    for j in range(mesh.ny):
        for i in range(mesh.nx):
            e = j * mesh.nx + i
            xs = mesh.x0 + (i + gx) * hx
            ys = mesh.y0 + (j + gy) * hy
            xm, ym = mesh.map(xs, ys)
            out[e, :, 0], out[e, :, 1] = xm, ym
    return out


def boundary_faces(mesh: StructuredMesh):
    """List of (element, face) on the domain boundary, ascending."""
    out = []
    for e in range(mesh.n_elem):
        i, j = e % mesh.nx, e // mesh.nx
        for f, on in enumerate((j == 0, i == mesh.nx - 1, j == mesh.ny - 1, i == 0)):
            if on:
                out.append((e, f))
    return out


def face_node_positions(mesh: StructuredMesh, p: int, bfaces) -> np.ndarray:
    """Positions [n_bface][p+1][2] of the nodal points along boundary faces,
    in increasing face parameter s."""
    pos = dg_node_positions(mesh, p)
    q = p + 1
    out = np.empty((len(bfaces), q, 2))
    for b, (e, f) in enumerate(bfaces):
        a = np.arange(q)
        if f == 0:
            idx = a
        elif f == 1:
            idx = a * q + p
        elif f == 2:
            idx = p * q + a
        else:
            idx = a * q
        out[b] = pos[e, idx]
    return out


# ---------------------------------------------------------------------------
# Materials
# ---------------------------------------------------------------------------

def block_materials(nx: int, blocks: int, seed: int, thick=(200.0, 0.999), thin=(0.2, 0.5)):
    """Random thick/thin block layout on an nx*nx grid split in blocks*blocks
    equal blocks; each block is thick or thin by a fair coin (seeded).

    Returns (sigma_t[n_elem], sigma_s[n_elem], block_of_elem[n_elem],
    is_thick[blocks*blocks]).
    """
    rng = np.random.default_rng(seed)
    thick_blk = rng.random(blocks * blocks) < 0.5
    per = nx // blocks
    e = np.arange(nx * nx)
    bi, bj = (e % nx) // per, (e // nx) // per
    blk = bj * blocks + bi
    st = np.where(thick_blk[blk], thick[0], thin[0])
    ss = np.where(thick_blk[blk], thick[0] * thick[1], thin[0] * thin[1])
    return st.astype(np.float64), ss.astype(np.float64), blk, thick_blk


def gaussian_random_field(n: int, corr_len: float, seed: int) -> np.ndarray:
    """Unit-variance Gaussian random field with Gaussian covariance of
    correlation length ``corr_len`` (domain units, domain [0,1]^2) on an
    n*n cell grid, sampled by FFT filtering of white noise; returns [n*n]
    in element order."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((n, n))
    k = np.fft.fftfreq(n, d=1.0 / n) * 2 * math.pi  # angular wave numbers on [0,1]
    kx, ky = np.meshgrid(k, k, indexing="xy")
    spec = np.exp(-0.25 * (corr_len ** 2) * (kx ** 2 + ky ** 2))
    f = np.real(np.fft.ifft2(np.fft.fft2(white) * np.sqrt(spec)))
    f = (f - f.mean()) / f.std()
    return f.ravel()


# ---------------------------------------------------------------------------
# Manufactured solutions (Sec. "Method of Manufactured Solutions")
# ---------------------------------------------------------------------------

MMS_DELTA, MMS_ZETA, MMS_OMEGA = 1.25, 0.1, 0.05


def _mms_fields(x, y):
    """alpha, beta-vector, Theta and their gradients at points (x, y)."""
    pi = math.pi
    d, z, w = MMS_DELTA, MMS_ZETA, MMS_OMEGA
    al = np.sin(pi * x) * np.sin(pi * y) + d
    al_x = pi * np.cos(pi * x) * np.sin(pi * y)
    al_y = pi * np.sin(pi * x) * np.cos(pi * y)
    c2 = 2 * pi / (1 + 2 * w)
    s2 = np.sin(c2 * (x + w)) * np.sin(c2 * (y + w))
    s2_x = c2 * np.cos(c2 * (x + w)) * np.sin(c2 * (y + w))
    s2_y = c2 * np.sin(c2 * (x + w)) * np.cos(c2 * (y + w))
    c3 = 3 * pi / (1 + 2 * z)
    s3 = np.sin(c3 * (x + z)) * np.sin(c3 * (y + z))
    s3_x = c3 * np.cos(c3 * (x + z)) * np.sin(c3 * (y + z))
    s3_y = c3 * np.sin(c3 * (x + z)) * np.cos(c3 * (y + z))
    # beta = (s2, s2); Theta = [[s3/2, s2], [s2, s3/4]]  (both read literally)
    return dict(al=al, al_x=al_x, al_y=al_y, s2=s2, s2_x=s2_x, s2_y=s2_y,
                s3=s3, s3_x=s3_x, s3_y=s3_y)


def mms_psi(x, y, ox, oy):
    """psi = (alpha + Omega.beta + Omega(x)Omega : Theta) / (4 pi)."""
    F = _mms_fields(x, y)
    val = (F["al"] + (ox + oy) * F["s2"] + ox * ox * 0.5 * F["s3"]
           + 2 * ox * oy * F["s2"] + oy * oy * 0.25 * F["s3"])
    return val / (4 * math.pi)


def mms_grad_psi(x, y, ox, oy):
    F = _mms_fields(x, y)
    gx = (F["al_x"] + (ox + oy) * F["s2_x"] + ox * ox * 0.5 * F["s3_x"]
          + 2 * ox * oy * F["s2_x"] + oy * oy * 0.25 * F["s3_x"])
    gy = (F["al_y"] + (ox + oy) * F["s2_y"] + ox * ox * 0.5 * F["s3_y"]
          + 2 * ox * oy * F["s2_y"] + oy * oy * 0.25 * F["s3_y"])
    return gx / (4 * math.pi), gy / (4 * math.pi)


def mms_phi(x, y):
    """Scalar flux of the MMS angular flux: alpha + tr(Theta)/3."""
    F = _mms_fields(x, y)
    return F["al"] + (0.5 * F["s3"] + 0.25 * F["s3"]) / 3.0


def mms_source(x, y, ox, oy, sigma_t, sigma_s):
    """Angular source q = Omega.grad(psi) + sigma_t psi - sigma_s/(4 pi) phi
    that makes the MMS angular flux an exact solution of the transport
    equation (with the scalar flux of the continuous MMS solution)."""
    gx, gy = mms_grad_psi(x, y, ox, oy)
    return (ox * gx + oy * gy + sigma_t * mms_psi(x, y, ox, oy)
            - sigma_s / (4 * math.pi) * mms_phi(x, y))


# A linearly anisotropic angular flux that is linear in space:
# psi = (phi + 3 Omega.J) / (4 pi) with phi = a + b x + c y, J constant.
LIN_A, LIN_B, LIN_C, LIN_JX, LIN_JY = 2.0, 0.7, -0.4, 0.15, -0.1


def linear_aniso_psi(x, y, ox, oy):
    phi = LIN_A + LIN_B * x + LIN_C * y
    return (phi + 3.0 * (ox * LIN_JX + oy * LIN_JY)) / (4 * math.pi)


def linear_aniso_grad_psi(x, y, ox, oy):
    z = np.zeros_like(np.asarray(x, dtype=float))
    return z + LIN_B / (4 * math.pi), z + LIN_C / (4 * math.pi)


# ---------------------------------------------------------------------------
# Learned-guess workload: log-normal cross sections, piecewise-constant sources
# ---------------------------------------------------------------------------

def learned_guess_problem(nx: int, seed: int, blocks: int = 8):
    """Straight nx*nx mesh of [0,1]^2 with sigma_t = 10 exp(1.5 g) (g a unit
    Gaussian random field, correlation length 0.1), sigma_s = c sigma_t with a
    smooth scattering ratio field c in [0.5, 0.99], and an isotropic source
    that is piecewise constant (0 or 1 per steradian) on a random
    blocks*blocks map.  Returns (mesh, sigma_t, sigma_s, q_elem) with q_elem
    the per-element source value."""
    mesh = structured_mesh(nx, m=1)
    g = gaussian_random_field(nx, 0.1, 2 * seed)
    h = gaussian_random_field(nx, 0.2, 2 * seed + 1)
    st = 10.0 * np.exp(1.5 * g)
    c = 0.5 + 0.49 / (1.0 + np.exp(-1.5 * h))
    rng = np.random.default_rng(10_000 + seed)
    bmap = (rng.random((blocks, blocks)) < 0.5).astype(float)
    e = np.arange(nx * nx)
    bi = np.minimum((e % nx) * blocks // nx, blocks - 1)
    bj = np.minimum((e // nx) * blocks // nx, blocks - 1)
    q = bmap[bj, bi]
    return mesh, st, c * st, q
