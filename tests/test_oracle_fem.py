"""Pins for the oracle's mapped finite elements (geometry, basis, element matrices)."""
import numpy as np
import pytest

import smm_workloads as W
from oracle.fem import Element, lagrange
from oracle.quadrature import gauss_lobatto
from tests.oracle_problems import disc_for


def test_lagrange_partition_and_interpolation():
    g, _ = gauss_lobatto(5)
    V, D = lagrange(g, g)
    assert np.allclose(V, np.eye(5), atol=1e-14)
    x = np.linspace(0, 1, 17)
    V, D = lagrange(g, x)
    assert np.allclose(V.sum(1), 1.0, atol=1e-14) and np.allclose(D.sum(1), 0.0, atol=1e-12)
    # exact derivative of x^3 from its nodal values
    assert np.allclose(D @ g ** 3, 3 * x ** 2, atol=1e-12)


@pytest.mark.parametrize("m,seed", [(1, None), (2, 4), (3, 9)])
def test_geometry_area_and_jacobian(m, seed):
    mesh = W.structured_mesh(5, m=m, perturb_seed=seed)
    disc = disc_for(mesh, 2, 4, 1.0, 0.5)
    assert min(el.J.min() for el in disc.elems) > 0
    assert abs(sum(el.area() for el in disc.elems) - 1.0) < 1e-13
    # neighbouring faces: same physical points, opposite normals
    for e in range(disc.ne):
        for f in range(4):
            nb = disc.nbr[e][f]
            if nb is None:
                continue
            e2, f2, flip = nb
            a, b = disc.faces[e][f], disc.faces[e2][f2]
            xb, nb_ = (b["x"][::-1], b["nds"][::-1]) if flip else (b["x"], b["nds"])
            assert np.allclose(a["x"], xb, atol=1e-14)
            assert np.allclose(a["nds"], -nb_, atol=1e-14)
    # boundary normals integrate to zero over the closed boundary of each element
    for e in range(disc.ne):
        tot = sum(disc.faces[e][f]["nds"].sum(0) for f in range(4))
        assert np.allclose(tot, 0.0, atol=1e-14)


def test_element_matrices_against_exact_integrals():
    sympy = pytest.importorskip("sympy")
    X, Y = sympy.symbols("x y")
    # rectangle [0,2]x[0,1], p = 1, straight map
    ctrl = np.array([[0, 0], [2, 0], [0, 1], [2, 1]], float)
    el = Element(ctrl, 1, 1)
    lx = [1 - X / 2, X / 2]
    ly = [1 - Y, Y]
    phi = [lx[i % 2] * ly[i // 2] for i in range(4)]
    M = np.array([[float(sympy.integrate(phi[i] * phi[j], (X, 0, 2), (Y, 0, 1))) for j in range(4)] for i in range(4)])
    Gx = np.array([[float(sympy.integrate(phi[j] * sympy.diff(phi[i], X), (X, 0, 2), (Y, 0, 1))) for j in range(4)] for i in range(4)])
    Gy = np.array([[float(sympy.integrate(phi[j] * sympy.diff(phi[i], Y), (X, 0, 2), (Y, 0, 1))) for j in range(4)] for i in range(4)])
    gx, gy = el.stream()
    assert np.allclose(el.mass(), M, atol=1e-14)
    assert np.allclose(gx, Gx, atol=1e-14) and np.allclose(gy, Gy, atol=1e-14)


def test_element_matrix_identities_curved():
    mesh = W.structured_mesh(3, m=3, perturb_seed=2)
    disc = disc_for(mesh, 3, 4, 1.0, 0.5)
    for e, el in enumerate(disc.elems):
        one = np.ones(disc.n)
        assert abs(one @ disc.M[e] @ one - el.area()) < 1e-14
        # sum_i dphi_i/dx = 0 => column sums of Gx, Gy vanish
        assert np.allclose(one @ disc.Gx[e], 0.0, atol=1e-13)
        assert np.allclose(one @ disc.Gy[e], 0.0, atol=1e-13)
        # int_K d(x)/dx = |K|: Gx applied to the nodal values of x, tested with v = 1 ... via K: sum_ij Kxx x_j
        K = el.stiffness()
        xs = el.V  # unused; check symmetry of stiffness blocks
        assert np.allclose(K[0, 1], K[1, 0].T, atol=1e-14)


@pytest.mark.parametrize("m,p,seed", [(2, 2, 4), (3, 3, 9), (2, 4, 1)])
def test_physical_gradients_on_curved_elements(m, p, seed):
    """Isoparametric reproduction: with p >= m a physical linear function
    a . x + c lies in Q_p of every curved element (x(xi) has degree m), so its
    nodal interpolant's gradient is exactly a at every volume and face point;
    and the divergence theorem int_K dphi_i/dx_c = oint phi_i n_c ds holds
    for every basis function (both exact under the element's quadrature)."""
    from oracle.quadrature import gauss_lobatto
    mesh = W.structured_mesh(3, 2, m=m, perturb_seed=seed)
    disc = disc_for(mesh, p, 4, 1.0, 0.5)
    g, _ = gauss_lobatto(p + 1)
    XI, ETA = np.meshgrid(g, g, indexing="xy")
    a = np.array([1.7, -0.6])
    for e, el in enumerate(disc.elems):
        xn, _ = el.map(XI.ravel(), ETA.ravel())  # physical DG node positions, x fastest
        u = xn @ a + 0.3
        assert np.max(np.abs(el.G.transpose(0, 2, 1) @ u - a)) < 1e-12
        for f in range(4):
            Gf = disc.faces[e][f]["G"]
            assert np.max(np.abs(Gf.transpose(0, 2, 1) @ u - a)) < 1e-12
        vol = np.einsum("q,qic->ic", el.w * el.J, el.G)
        surf = sum(disc.faces[e][f]["V"].T @ disc.faces[e][f]["nds"] for f in range(4))
        assert np.max(np.abs(vol - surf)) < 1e-13
