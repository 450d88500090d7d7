"""Quadrature rules (oracle).

* Gauss-Legendre and Gauss-Lobatto rules on [0, 1] (the paper's mesh control
  points and nodal basis sit on Gauss-Lobatto points, Sec. "Description of
  the Mesh").
* Level-symmetric LQ_N angular quadrature (the paper names "Level Symmetric
  S_N" for every experiment but does not print it).  Construction: the
  standard direction-cosine recursion mu_i^2 = mu_1^2 + (i-1) 2(1-3 mu_1^2)/(N-2)
  from the published mu_1 of each N; point weights solve the even-moment
  conditions sum w mu^{2k} = 1/(2k+1) (k = 0, 2, 3, ...; k = 1 holds by
  symmetry); the 2D set keeps the upper hemisphere with doubled weights and
  is normalized to sum 4 pi.
"""
from __future__ import annotations

import math

import numpy as np

# Published first direction cosine of the LQ_N sets.  For N = 4 the value is
# fixed by the mu^4 condition (one weight class): mu_1^2 = (4 - sqrt(6.4))/12.
LQ_MU1 = {
    2: 1.0 / math.sqrt(3.0),
    4: math.sqrt((4.0 - math.sqrt(6.4)) / 12.0),
    6: 0.2666355,
    8: 0.2182179,
    10: 0.1893213,
    12: 0.1672126,
}


def gauss_legendre(n: int):
    """n-point Gauss-Legendre rule on [0, 1] (exact to degree 2n-1)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def gauss_lobatto(n: int):
    """n-point Gauss-Lobatto rule on [0, 1] (exact to degree 2n-3).

    Interior nodes: roots of P'_{n-1}; weights 2 / (n (n-1) P_{n-1}(x)^2) on
    [-1, 1], halved for [0, 1].
    """
    if n < 2:
        raise ValueError("n >= 2")
    c = np.zeros(n)
    c[-1] = 1.0
    P = np.polynomial.legendre.Legendre(c)
    if n == 2:
        x = np.array([-1.0, 1.0])
    else:
        r = np.sort(np.real(P.deriv().roots()))
        d1, d2 = P.deriv(1), P.deriv(2)
        for _ in range(3):  # Newton polish
            r = r - d1(r) / d2(r)
        x = np.concatenate(([-1.0], r, [1.0]))
    w = 2.0 / (n * (n - 1) * P(x) ** 2)
    return 0.5 * (x + 1.0), 0.5 * w


def level_symmetric_octant(N: int):
    """Points of one octant of LQ_N: (cosines [npts][3], weights summing to 1).

    Point order: level triples (i, j, k), i + j + k = N/2 - 1 (0-based),
    i ascending then j ascending; cosines (mu_i, mu_j, mu_k).
    """
    if N not in LQ_MU1:
        raise ValueError(f"unsupported S_N order {N}")
    mu1 = LQ_MU1[N]
    L = N // 2
    if N == 2:
        mu = np.array([mu1])
    else:
        step = 2.0 * (1.0 - 3.0 * mu1 * mu1) / (N - 2)
        mu = np.sqrt(mu1 * mu1 + np.arange(L) * step)
    pts = [(i, j, L - 1 - i - j) for i in range(L) for j in range(L - i)]
    classes = sorted({tuple(sorted(t)) for t in pts})
    cls = [classes.index(tuple(sorted(t))) for t in pts]
    nc = len(classes)
    ks = [0] + list(range(2, nc + 1))
    A = np.zeros((nc, nc))
    rhs = np.zeros(nc)
    for r, k in enumerate(ks):
        for t, c in zip(pts, cls):
            A[r, c] += mu[t[0]] ** (2 * k)
        rhs[r] = 1.0 / (2 * k + 1)
    wc = np.linalg.solve(A, rhs)
    cos = np.array([[mu[t[0]], mu[t[1]], mu[t[2]]] for t in pts])
    w = np.array([wc[c] for c in cls])
    return cos, w


def level_symmetric_2d(N: int):
    """2D LQ_N set: ordinates Omega_d = (Omega_x, Omega_y) [N(N+2)/2][2] and
    weights [N(N+2)/2] summing to 4 pi; quadrant-major order
    (+,+), (-,+), (-,-), (+,-)."""
    cos, w = level_symmetric_octant(N)
    signs = [(1.0, 1.0), (-1.0, 1.0), (-1.0, -1.0), (1.0, -1.0)]
    om, ww = [], []
    for sx, sy in signs:
        for c, wi in zip(cos, w):
            om.append((sx * c[0], sy * c[1]))
            # 8 octants of total weight 1 each -> 4 pi; the two hemispheres
            # (+/- z) project onto the same 2D ordinate
            ww.append(2.0 * wi * (4.0 * math.pi / 8.0))
    return np.array(om), np.array(ww)
