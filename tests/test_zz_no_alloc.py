"""The allocation-free PCG entry point (smm_block_pcg_noalloc) through the C ABI.

It serves callers that cannot call cudaMalloc: it keeps its CG temporaries
in a fixed device array of the library.  Two calls in a row (different
right-hand sides, the second from a non-zero guess) must give the same
solution as the existing handle-based moment solve (smm_moment_solve) of the
same IP-SMM system, within the 1e-9 tolerance of the other moment-solve
parity tests.  The operator blocks are taken from the oracle's assembled
matrix, which matches the library's to rounding.
"""
import numpy as np
import pytest

import smm_workloads as W
from tests.parity_inputs import oracle_disc, problem, sources

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _blocks(disc, A):
    """Column-major n x n blocks of the oracle's IP-SMM matrix."""
    n, ne = disc.n, disc.ne
    A = A.toarray()
    diag = np.zeros((ne, n, n))
    off = np.zeros((ne, 4, n, n))
    nbr = -np.ones((ne, 4), dtype=np.int32)
    for e in range(ne):
        diag[e] = A[e * n:(e + 1) * n, e * n:(e + 1) * n]
        for f in range(4):
            nb = disc.nbr[e][f]
            if nb is not None:
                nbr[e, f] = nb[0]
                off[e, f] = A[e * n:(e + 1) * n, nb[0] * n:(nb[0] + 1) * n]
    pinv = np.linalg.inv(diag)
    colmajor = lambda a: np.ascontiguousarray(np.swapaxes(a, -1, -2))
    return colmajor(diag), colmajor(off), nbr, colmajor(pinv)


def test_noalloc_pcg_matches_moment_solve_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_07386_gb300 as P
    from oracle import ipsmm
    from oracle.smm import SMMProblem
    from paper_2304_07386_gb300 import build as B

    B.build()
    prob = problem(5, 4, m=2, p=2, sn=4, seed=3, kind="mms", c=0.6)
    mesh = prob["mesh"]
    om, _ = P.smm_quadrature(prob["sn"])
    q, inflow = sources(prob, om)
    opt = P.smm_default_options()
    opt.tol_cg = 1e-13
    h = P.smm_create(mesh.nodes, mesh.elem_nodes, mesh.m, prob["p"], prob["sn"], prob["sigma_t"],
                     prob["sigma_s"], q, inflow=inflow, options=opt)
    info = h.info()
    ne, n = info.n_elem, info.n_dof_elem
    disc = oracle_disc(prob)
    qo, io = sources(prob, disc.omega)
    op = SMMProblem(disc, qo, io)
    d_diag, d_off, d_nbr, d_pinv = (torch.as_tensor(a, device="cuda") for a in _blocks(disc, op.A))

    rng = np.random.default_rng(1)
    for call in range(2):
        # closures given as data: zero in the first call, random T and beta in the second
        T = np.zeros((3, ne, n)) if call == 0 else rng.standard_normal((3, ne, n))
        beta = np.zeros((info.n_bface, info.n_fq)) if call == 0 else rng.standard_normal((info.n_bface, info.n_fq))
        mom = np.concatenate([np.zeros((3, ne, n)), T])
        P.smm_set_moments(h, torch.as_tensor(mom.ravel(), device="cuda"), torch.as_tensor(beta.ravel(), device="cuda"))
        ref = torch.zeros(ne * n, dtype=torch.float64, device="cuda")
        P.smm_moment_solve(h, ref)
        b = ipsmm.assemble_rhs(disc, op.Q, T, op.jin, beta)
        x = torch.zeros(ne * n, dtype=torch.float64, device="cuda")
        if call == 1:
            x += torch.as_tensor(rng.standard_normal(ne * n), device="cuda")
        iters = P.smm.smm_block_pcg_noalloc(d_diag, d_off, d_nbr, d_pinv, torch.as_tensor(b, device="cuda"), x,
                                             tol=1e-13)
        torch.cuda.synchronize()
        assert iters > 0
        r, xx = ref.cpu().numpy(), x.cpu().numpy()
        assert np.max(np.abs(xx - r)) < 1e-9 * np.max(np.abs(r)), call


def test_noalloc_pcg_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_07386_gb300 as P

    P.load_library()
    n, ne = 16, (1 << 19) // 16 + 1
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    nbr = torch.zeros((1, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(P.SMMError) as ei:
        # sizes are checked before any pointer is used
        lib = P.load_library()
        import ctypes as C
        rc = lib.smm_block_pcg_noalloc(ne, n, C.c_void_p(z.data_ptr()), C.c_void_p(z.data_ptr()),
                                       C.c_void_p(nbr.data_ptr()), C.c_void_p(z.data_ptr()), C.c_void_p(z.data_ptr()),
                                       C.c_void_p(z.data_ptr()), 1e-10, 10, None, None)
        P.smm._check(rc)
    assert ei.value.status == 1
