"""CPU checks of the host setup of the CUDA path (setup.cpp) against the oracle.

A driver compiled against setup.cpp writes the element operators it builds
for seeded curved meshes, and each must equal the oracle's own quadrature or
assembled system:

- the sweep's ordering: ordinates, the inflow/outflow direction of every face
  (the sign of Omega . n at the face quadrature points), the upwind level of
  every (element, ordinate) and the task list the sweep kernel walks;
- the sweep's mass and streaming matrices (Sec. "Transport Discretization");
- the IP-SMM operator's diagonal and neighbour blocks and their inverses (LHS
  of Eq. ipsmm), and the source part of its right-hand side;
- the operators the right-hand-side kernels stream: three T-divergence blocks
  per element (K_xx, K_xy + K_yx, K_yy of the volume term
  -int grad u . (1/sigma_t) div_h T of Eq. ipsmm) and the physical basis
  gradients at the face quadrature points.

The right-hand-side kernels also rely on the last two annihilating constants
(their rows sum to zero because the nodal basis is a partition of unity) when
they shift T by its value at an element's first node; that is checked too.

A second driver builds the multigrid hierarchy of the moment solve's
preconditioner (amg.cpp; the project's replacement for the AMG-based subspace
correction of Sec. "Results"), which is checked against its definitions:
Galerkin products, the vertex-bilinear level, smoothed aggregation, the
damping estimates and the coarsest inverse.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import smm_workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2304_07386_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path_factory.mktemp("setup") / "setup_dump"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, os.path.join(ROOT, "tests", "setup_dump.cpp"),
                    os.path.join(CSRC, "setup.cpp"), "-o", str(exe)], check=True)
    return str(exe)


CASES = [(4, 3, 3, 4, 2), (3, 3, 2, 2, 5), (2, 3, 1, 1, None), (2, 2, 6, 3, 7)]


def write_inputs(tmp_path, mesh, p):
    ne, n = mesh.n_elem, (p + 1) ** 2
    st = 1.0 + 0.25 * (np.arange(ne) % 4)
    q = np.random.default_rng(3).uniform(0.5, 1.5, (ne, n))
    np.asarray(mesh.nodes, np.float64).tofile(tmp_path / "nodes.f64")
    np.asarray(mesh.elem_nodes, np.int32).tofile(tmp_path / "elem.i32")
    st.tofile(tmp_path / "sigma_t.f64")
    q.tofile(tmp_path / "q.f64")
    return st, q


def run_setup(driver, tmp_path, case, strong=False):
    """Run the host setup on a seeded curved mesh (strong: wave numbers up to 3
    at amplitude 0.05, whose upwind graphs have cycles); returns (mesh,
    sigma_t, q, loader, dims)."""
    nx, ny, m, p, seed = case
    mesh = (W.structured_mesh(nx, ny, m=m, perturb_seed=seed, wave_max=3, scale_by_k=False) if strong
            else W.structured_mesh(nx, ny, m=m, perturb_seed=seed))
    st, q = write_inputs(tmp_path, mesh, p)
    subprocess.run([driver, str(tmp_path), str(mesh.n_elem), str(len(mesh.nodes)), str(m), str(p)], check=True)
    n, nfq, nd, nlevels = map(int, open(tmp_path / "dims.txt").read().split())
    assert n == (p + 1) ** 2

    def load(name, shape, dtype=np.float64):
        ext = {np.float64: ".f64", np.int32: ".i32", np.int8: ".i8"}[dtype]
        return np.fromfile(tmp_path / (name + ext), dtype=dtype).reshape(shape)

    return mesh, st, q, load, dict(n=n, nfq=nfq, nd=nd, nlevels=nlevels)


@pytest.mark.parametrize("case", CASES, ids=lambda c: "nx%d_ny%d_m%d_p%d" % c[:4])
def test_rhs_operators_match_oracle_quadrature(driver, tmp_path, case):
    from oracle.transport import Discretization
    m, p = case[2], case[3]
    mesh, st, _, load, dims = run_setup(driver, tmp_path, case)
    ne, n, nfq = mesh.n_elem, dims["n"], dims["nfq"]
    Kxx, Ks, Kyy = (load(k, (ne, n, n)) for k in ("Kxx", "Ks", "Kyy"))
    Dfx, Dfy = (load(k, (ne, 4, nfq, n)) for k in ("Dfx", "Dfy"))
    nds = load("nds", (ne, 4, nfq, 2))

    disc = Discretization(mesh.nodes, mesh.elem_nodes, m, p, 4, st, 0.5 * st)
    assert nfq == len(disc.elems[0].fq_s)
    for e in range(ne):
        K = disc.elems[e].stiffness()  # [a][b][i][j] = int dphi_i/da dphi_j/db
        scale = np.max(np.abs(K))
        for got, want in ((Kxx[e], -K[0, 0] / st[e]), (Ks[e], -(K[0, 1] + K[1, 0]) / st[e]),
                          (Kyy[e], -K[1, 1] / st[e])):
            assert np.max(np.abs(got - want)) <= 1e-12 * scale, e
            assert np.max(np.abs(got - got.T)) <= 1e-13 * scale, e
            # rows annihilate constants
            assert np.max(np.abs(got.sum(axis=1))) <= 1e-13 * scale, e
        for f in range(4):
            fd = disc.faces[e][f]
            gscale = np.max(np.abs(fd["G"]))
            assert np.max(np.abs(Dfx[e, f] - fd["G"][:, :, 0])) <= 1e-12 * gscale, (e, f)
            assert np.max(np.abs(Dfy[e, f] - fd["G"][:, :, 1])) <= 1e-12 * gscale, (e, f)
            assert np.max(np.abs(Dfx[e, f].sum(axis=1))) <= 1e-13 * gscale, (e, f)
            assert np.max(np.abs(Dfy[e, f].sum(axis=1))) <= 1e-13 * gscale, (e, f)
            assert np.max(np.abs(nds[e, f] - fd["nds"])) <= 1e-13 * np.max(np.abs(fd["nds"])), (e, f)


@pytest.mark.parametrize("case", CASES, ids=lambda c: "nx%d_ny%d_m%d_p%d" % c[:4])
def test_sweep_and_moment_operators_match_oracle(driver, tmp_path, case):
    from oracle import closures, ipsmm
    from oracle.transport import Discretization
    m, p = case[2], case[3]
    mesh, st, q, load, dims = run_setup(driver, tmp_path, case)
    ne, n = mesh.n_elem, dims["n"]
    M, Gx, Gy, Ad, Pinv = (load(k, (ne, n, n)) for k in ("M", "Gx", "Gy", "Adiag", "Pinv"))
    Aoff = load("Aoff", (ne, 4, n, n))
    nbr = load("nbr", (ne, 4), np.int32)
    bfixed = load("bfixed", (ne, n))
    disc = Discretization(mesh.nodes, mesh.elem_nodes, m, p, 4, st, 0.5 * st)
    A = ipsmm.assemble_lhs(disc).tocsr()
    for e in range(ne):
        ms = np.max(np.abs(disc.M[e]))
        assert np.max(np.abs(M[e] - disc.M[e])) <= 1e-13 * ms, e
        gs = max(np.max(np.abs(disc.Gx[e])), np.max(np.abs(disc.Gy[e])))
        assert np.max(np.abs(Gx[e] - disc.Gx[e])) <= 1e-12 * gs, e
        assert np.max(np.abs(Gy[e] - disc.Gy[e])) <= 1e-12 * gs, e
        rows = slice(e * n, (e + 1) * n)
        blk = A[rows, rows].toarray()
        scale = np.max(np.abs(blk))
        assert np.max(np.abs(Ad[e] - blk)) <= 1e-12 * scale, e
        assert np.max(np.abs(Pinv[e] @ blk - np.eye(n))) <= 1e-9, e
        for f in range(4):
            nb = disc.nbr[e][f]
            if nb is None:
                assert nbr[e, f] < 0
                continue
            assert nbr[e, f] == nb[0]
            want = A[rows, nb[0] * n:(nb[0] + 1) * n].toarray()
            assert np.max(np.abs(Aoff[e, f] - want)) <= 1e-12 * scale, (e, f)
    # source part of the right-hand side: isotropic q per steradian, vacuum inflow, T = 0, beta = 0
    Q = closures.source_moments(disc, np.broadcast_to(q, (disc.nd,) + q.shape))
    jin = closures.j_in(disc, None)
    b = ipsmm.assemble_rhs(disc, Q, np.zeros((3, ne, n)), jin, np.zeros_like(jin))
    assert np.max(np.abs(bfixed.ravel() - b)) <= 1e-12 * np.max(np.abs(b))


@pytest.mark.parametrize("case,strong", [(c, False) for c in CASES + [(6, 5, 2, 1, 9)]] +
                         [((5, 5, 2, 1, 1), True), ((6, 4, 2, 2, 4), True)],
                         ids=lambda c: "nx%d_ny%d_m%d_p%d" % c[:4] if isinstance(c, tuple) else ("cycles" if c else "dag"))
def test_sweep_ordering_matches_oracle_upwind_graph(driver, tmp_path, case, strong):
    """Face directions from the sign of Omega_d . n at every face point (1
    outflow, -1 inflow, 2 both; -2 and 3 when the inflow is lagged); the
    faces lagged to break cycles are the oracle's (the same rule, stated in
    oracle/transport.py); level of (e, d) = 0 without unlagged upwind
    neighbours, else 1 + the largest level of those (longest path, unique);
    tasks = all (e, d) sorted by (level, e, d), level_start the first task of
    each level."""
    from oracle.transport import Discretization
    m, p = case[2], case[3]
    mesh, st, _, load, dims = run_setup(driver, tmp_path, case, strong)
    ne, nd, nfq, nlev = mesh.n_elem, dims["nd"], dims["nfq"], dims["nlevels"]
    disc = Discretization(mesh.nodes, mesh.elem_nodes, m, p, 4, st, 0.5 * st)
    assert nd == disc.nd
    om = np.stack([load("ox", (nd,)), load("oy", (nd,))], axis=1)
    assert np.array_equal(om, disc.omega)
    fdir = load("fdir", (ne, nd, 4), np.int8)
    level = load("level", (nd, ne), np.int32)
    tasks = load("tasks", (ne * nd,), np.int32)
    start = load("level_start", (nlev + 1,), np.int32)
    n_lagged = 0
    for d in range(nd):
        order, lagged = disc.upwind_order(d)
        n_lagged += len(lagged)
        deps = [[] for _ in range(ne)]
        for e in range(ne):
            for f in range(4):
                a = disc.faces[e][f]["nds"] @ disc.omega[d]
                pos, neg = np.any(a > 0), np.any(a < 0)
                want = 2 if pos and neg else (1 if pos else (-1 if neg else 0))
                if (e, f) in lagged:
                    want = {-1: -2, 2: 3}[want]
                assert fdir[e, d, f] == want, (e, d, f)
                if disc.nbr[e][f] is not None and neg and (e, f) not in lagged:
                    deps[e].append(disc.nbr[e][f][0])
        for e in order:  # unlagged upwind neighbours first
            want = 1 + max(level[d, u] for u in deps[e]) if deps[e] else 0
            assert level[d, e] == want, (e, d)
    assert (n_lagged > 0) == strong
    assert nlev == level.max() + 1
    assert np.array_equal(np.sort(tasks), np.arange(ne * nd))
    e_of, d_of = tasks // nd, tasks % nd
    key = np.stack([level[d_of, e_of], e_of, d_of], axis=1)
    assert all(tuple(key[i]) < tuple(key[i + 1]) for i in range(len(key) - 1))
    assert start[0] == 0 and start[-1] == ne * nd
    for lv in range(nlev):
        assert np.all(key[start[lv]:start[lv + 1], 0] == lv)


def test_sign_indefinite_face_is_rejected_without_lagging(driver, tmp_path):
    """Two elements sharing a bowed quadratic face: its normal turns through
    the direction of some S4 ordinate, which then flows in at some face points
    and out at others.  With cycle lagging off (the driver's fourth mode
    argument) setup fails with that error, and the oracle's ordering without
    lagging rejects it too."""
    nodes = np.array([[0, 0], [0.5, 0], [1, 0], [0, 0.5], [0.5, 0.5], [1, 0.5], [0, 1], [0.5, 1], [1, 1],
                      [1.5, 0], [2, 0], [1.5, 0.5], [2, 0.5], [1.5, 1], [2, 1]], float)
    nodes[5] = [1.25, 0.5]  # middle node of the shared face, pushed to the right
    elem = np.array([[0, 1, 2, 3, 4, 5, 6, 7, 8], [2, 9, 10, 5, 11, 12, 8, 13, 14]], np.int32)

    class Mesh:
        n_elem = 2

    mesh = Mesh()
    mesh.nodes, mesh.elem_nodes = nodes, elem
    write_inputs(tmp_path, mesh, 1)
    r = subprocess.run([driver, str(tmp_path), "2", str(len(nodes)), "2", "1", "nolag"], capture_output=True, text=True)
    assert r.returncode == 4
    assert "inflow at some quadrature points and outflow at others" in r.stderr
    # the oracle rejects it too without lagging: across a mixed face each element is upwind of the other
    from oracle.transport import CycleError, Discretization
    disc = Discretization(nodes, elem, 2, 1, 4, np.ones(2), 0.5 * np.ones(2))
    with pytest.raises(CycleError):
        for d in range(disc.nd):
            disc.upwind_order(d, lag_cycles=False)
    # with lagging both accept it
    r = subprocess.run([driver, str(tmp_path), "2", str(len(nodes)), "2", "1"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert sum(len(disc.upwind_order(d)[1]) for d in range(disc.nd)) > 0


@pytest.mark.parametrize("ne,m,p,sn", [
    (2**31 // 40 + 1, 1, 1, 8),   # (element, ordinate) task ids: 40 ordinates
    (2**31 // 49 + 1, 6, 1, 2),   # control point slots: 49 per element at geometry order 6
    (2**31 // 25 + 1, 1, 4, 2),   # unknown ids: 25 dofs per element at p = 4
])
def test_sizes_beyond_32_bit_indexes_are_rejected(driver, ne, m, p, sn):
    """Task ids, control point slots and unknown ids are 32-bit integers on the
    host and in the kernels: a mesh whose element count times any of them
    passes 2^31 - 1 is rejected before its arrays are read."""
    r = subprocess.run([driver, "--size-check", str(ne), str(m), str(p), str(sn)], capture_output=True, text=True,
                       timeout=60)
    assert r.returncode == 4, (r.returncode, r.stderr)
    assert "mesh too large" in r.stderr


# ---------------------------------------------------------------------------
# multigrid hierarchy of the moment-system preconditioner (amg.cpp)

@pytest.fixture(scope="module")
def mg_driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path_factory.mktemp("mg") / "mg_dump"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, os.path.join(ROOT, "tests", "mg_dump.cpp"),
                    os.path.join(CSRC, "setup.cpp"), os.path.join(CSRC, "amg.cpp"), "-o", str(exe)], check=True)
    return str(exe)


def _csr(tmp_path, stem, nrow, ncol):
    import scipy.sparse as sp
    rp = np.fromfile(tmp_path / (stem + "_rp.i32"), dtype=np.int32)
    ci = np.fromfile(tmp_path / (stem + "_ci.i32"), dtype=np.int32)
    v = np.fromfile(tmp_path / (stem + "_v.f64"))
    return sp.csr_matrix((v, ci, rp), shape=(nrow, ncol)).toarray()


# Gauss-Lobatto points of [0, 1], closed forms
GLL01 = {1: [0.0, 1.0], 2: [0.0, 0.5, 1.0],
         3: [0.0, (1 - 5 ** -0.5) / 2, (1 + 5 ** -0.5) / 2, 1.0],
         4: [0.0, (1 - (3 / 7) ** 0.5) / 2, 0.5, (1 + (3 / 7) ** 0.5) / 2, 1.0]}


# (nx, ny, m, p, seed, coarse_max): the last two build two aggregation levels
MG_CASES = [(8, 8, 2, 2, 4, 20), (10, 9, 3, 3, 6, 40), (5, 4, 3, 4, 2, 8), (16, 16, 1, 1, 5, 8), (14, 12, 2, 1, 3, 6)]


@pytest.mark.parametrize("case", MG_CASES, ids=lambda c: "nx%d_ny%d_m%d_p%d" % c[:4])
def test_multigrid_hierarchy(mg_driver, tmp_path, case):
    """Level 1 is the Galerkin product P1^T A P1 of the DG operator with the
    continuous bilinear functions on the mesh vertices (a DG node takes the
    bilinear interpolant of its element's corner values); each further level
    is R A P with R = P^T and P = (I - w D^-1 A) T, T a piecewise-constant
    aggregation (one 1 per row); the damping factors come from Rayleigh
    estimates that never exceed the largest eigenvalue of the Jacobi (or
    element-block Jacobi) preconditioned operator; the coarsest level is
    inverted."""
    import scipy.linalg as sla
    nx, ny, m, p, seed, coarse_max = case
    mesh = W.structured_mesh(nx, ny, m=m, perturb_seed=seed)
    ne, n, p1 = mesh.n_elem, (p + 1) ** 2, p + 1
    write_inputs(tmp_path, mesh, p)
    subprocess.run([mg_driver, str(tmp_path), str(ne), str(len(mesh.nodes)), str(m), str(p), str(coarse_max)],
                   check=True)
    lines = open(tmp_path / "mg.txt").read().split("\n")
    nvert, ncoarse, nlev, omega0 = lines[0].split()
    nvert, ncoarse, nlev, omega0 = int(nvert), int(ncoarse), int(nlev), float(omega0)
    levels = [dict(zip(("nrow", "omega", "hasP"), (int(a), float(b), int(c))))
              for a, b, c in (l.split() for l in lines[1:1 + nlev])]
    f64 = lambda name: np.fromfile(tmp_path / (name + ".f64"))
    i32 = lambda name: np.fromfile(tmp_path / (name + ".i32"), dtype=np.int32)
    Ad, Aoff, Pinv = f64("Adiag").reshape(ne, n, n), f64("Aoff").reshape(ne, 4, n, n), f64("Pinv").reshape(ne, n, n)
    nbr = i32("nbr").reshape(ne, 4)
    N = ne * n
    A0 = np.zeros((N, N))
    for e in range(ne):
        A0[e * n:(e + 1) * n, e * n:(e + 1) * n] = Ad[e]
        for f in range(4):
            if nbr[e, f] >= 0:
                A0[e * n:(e + 1) * n, nbr[e, f] * n:(nbr[e, f] + 1) * n] += Aoff[e, f]
    # vertices: the distinct corner control points, numbered in increasing id order
    cidx = [0, m, m * (m + 1), m * (m + 1) + m]
    corner_ids = np.asarray(mesh.elem_nodes)[:, cidx]
    uniq = np.unique(corner_ids)
    vid = i32("vid").reshape(ne, 4)
    assert nvert == len(uniq) == (nx + 1) * (ny + 1)
    assert np.array_equal(vid, np.searchsorted(uniq, corner_ids))
    vrp, vinc = i32("vrp"), i32("vinc")
    for v in range(nvert):
        assert list(vinc[vrp[v]:vrp[v + 1]]) == list(np.flatnonzero(vid.ravel() == v))
    # bilinear weights of the DG nodes (x fastest)
    g = np.asarray(GLL01[p])
    w4 = f64("w4").reshape(n, 4)
    X, Y = np.meshgrid(g, g, indexing="xy")
    X, Y = X.ravel(), Y.ravel()
    want = np.stack([(1 - X) * (1 - Y), X * (1 - Y), (1 - X) * Y, X * Y], axis=1)
    assert np.max(np.abs(w4 - want)) < 1e-15
    P1 = np.zeros((N, nvert))
    for e in range(ne):
        for c in range(4):
            P1[e * n:(e + 1) * n, vid[e, c]] += w4[:, c]
    # level-0 block-Jacobi damping from a Rayleigh estimate of lambda_max(Pinv A)
    Bd = sla.block_diag(*Ad)
    assert np.max(np.abs(sla.block_diag(*Pinv) @ Bd - np.eye(N))) < 1e-9
    lam0 = sla.eigh(A0, Bd, eigvals_only=True)[-1]
    est0 = (4.0 / 3.0) / (1.05 * omega0)
    assert 0.7 * lam0 <= est0 <= lam0 * (1 + 1e-9), (est0, lam0)
    A_prev = P1.T @ A0 @ P1
    for l, L in enumerate(levels, start=1):
        A = _csr(tmp_path, "L%d_A" % l, L["nrow"], L["nrow"])
        scale = np.max(np.abs(A))
        assert np.max(np.abs(A - A_prev)) <= 1e-12 * scale, l
        assert np.max(np.abs(A - A.T)) <= 1e-12 * scale, l
        assert np.linalg.eigvalsh(A)[0] > 0, l
        dinv = f64("L%d_dinv" % l)
        assert np.array_equal(dinv, 1.0 / np.diag(A)), l
        lam = np.linalg.eigvalsh(np.sqrt(dinv)[:, None] * A * np.sqrt(dinv)[None, :])[-1]
        est = (4.0 / 3.0) / (1.05 * L["omega"])
        assert 0.7 * lam <= est <= lam * (1 + 1e-9), (l, est, lam)
        if not L["hasP"]:
            assert l == nlev
            break
        nc = levels[l]["nrow"]
        P = _csr(tmp_path, "L%d_P" % l, L["nrow"], nc)
        R = _csr(tmp_path, "L%d_R" % l, nc, L["nrow"])
        assert np.array_equal(R, P.T), l
        # P = (I - w D^-1 A) T: w from P 1 = 1 - w D^-1 A 1, then T must be an aggregation
        u = dinv * A.sum(axis=1)
        k = np.argmax(np.abs(u))
        w = (1.0 - P.sum(axis=1)[k]) / u[k]
        S = np.eye(L["nrow"]) - w * dinv[:, None] * A
        T = np.linalg.solve(S, P)
        assert np.max(np.abs(T - np.round(T))) < 1e-8, l
        T = np.round(T)
        assert set(np.unique(T)) <= {0.0, 1.0} and np.all(T.sum(axis=1) == 1) and np.all(T.sum(axis=0) >= 1), l
        # the prolongator's damping is a Rayleigh estimate of lambda_max(D^-1 A) too
        assert 0.7 * lam <= (4.0 / 3.0) / w <= lam * (1 + 1e-9), (l, w, lam)
        A_prev = R @ A @ P
    assert ncoarse == levels[-1]["nrow"]
    assert ncoarse <= coarse_max or nlev >= 2
    Cinv = f64("coarse_inv").reshape(ncoarse, ncoarse)
    assert np.max(np.abs(Cinv @ A_prev - np.eye(ncoarse))) < 1e-9
