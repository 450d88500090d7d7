"""CPU checks of the host setup of the CUDA path (setup.cpp) against the oracle.

A driver compiled against setup.cpp writes the element operators it builds
for seeded curved meshes, and each must equal the oracle's own quadrature or
assembled system:

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


def run_setup(driver, tmp_path, case):
    """Run the host setup on a seeded curved mesh; returns (mesh, sigma_t, q, loader, n, nfq)."""
    nx, ny, m, p, seed = case
    mesh = W.structured_mesh(nx, ny, m=m, perturb_seed=seed)
    ne, n = mesh.n_elem, (p + 1) ** 2
    st = 1.0 + 0.25 * (np.arange(ne) % 4)
    q = np.random.default_rng(3).uniform(0.5, 1.5, (ne, n))
    np.asarray(mesh.nodes, np.float64).tofile(tmp_path / "nodes.f64")
    np.asarray(mesh.elem_nodes, np.int32).tofile(tmp_path / "elem.i32")
    st.tofile(tmp_path / "sigma_t.f64")
    q.tofile(tmp_path / "q.f64")
    subprocess.run([driver, str(tmp_path), str(ne), str(len(mesh.nodes)), str(m), str(p)], check=True)
    n_out, nfq = map(int, open(tmp_path / "dims.txt").read().split())
    assert n_out == n

    def load(name, shape, dtype=np.float64):
        ext = ".i32" if dtype == np.int32 else ".f64"
        return np.fromfile(tmp_path / (name + ext), dtype=dtype).reshape(shape)

    return mesh, st, q, load, n, nfq


@pytest.mark.parametrize("case", CASES, ids=lambda c: "nx%d_ny%d_m%d_p%d" % c[:4])
def test_rhs_operators_match_oracle_quadrature(driver, tmp_path, case):
    from oracle.transport import Discretization
    m, p = case[2], case[3]
    mesh, st, _, load, n, nfq = run_setup(driver, tmp_path, case)
    ne = mesh.n_elem
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
    mesh, st, q, load, n, nfq = run_setup(driver, tmp_path, case)
    ne = mesh.n_elem
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
