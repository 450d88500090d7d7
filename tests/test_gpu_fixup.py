"""GPU zero and scale negative flux fixup (inside the sweep, Sec. 6.3) vs the
oracle: a strip of thick absorbing cells lit from the left, whose DG solution
dips below zero; both local solvers, sweep to 1e-11 and converged SMM flux to
1e-9."""
import numpy as np
import pytest

import smm_workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_07386_gb300 import build as B
    B.build()


def strip(nx=6, sig=30.0, c=0.0, p=2, sn=4):
    mesh = W.structured_mesh(nx, 1, m=1)
    st = np.full(mesh.n_elem, sig)
    ss = c * st
    bf = W.boundary_faces(mesh)
    nd = sn * (sn + 2) // 2
    pb = np.zeros((nd, len(bf), p + 1))
    for b, (e, f) in enumerate(bf):
        if f == 3:
            pb[:, b, :] = 1.0
    return mesh, st, ss, pb


def gpu(mesh, st, ss, pb, p, sn, fixup, solver):
    import paper_2304_07386_gb300 as P
    opt = P.smm_default_options()
    opt.negative_flux_fixup = fixup
    opt.sweep_solver = solver
    opt.tol_cg = 1e-13
    q = np.zeros((mesh.n_elem, (p + 1) ** 2))
    return P.smm_create(mesh.nodes, mesh.elem_nodes, 1, p, sn, st, ss, q, inflow=pb, options=opt)


@pytest.mark.parametrize("solver", [0, 1], ids=["lu", "cached_inverse"])
def test_sweep_with_fixup_matches_oracle(solver):
    import paper_2304_07386_gb300 as P
    from tests.oracle_problems import disc_for
    p, sn = 2, 4
    mesh, st, ss, pb = strip()
    disc = disc_for(mesh, p, sn, st, ss)
    q = np.zeros((disc.ne, disc.n))
    for fixup in (0, 1):
        h = gpu(mesh, st, ss, pb, p, sn, fixup, solver)
        info = h.info()
        P.smm_sweep(h, torch.zeros(info.n_elem * info.n_dof_elem, dtype=torch.float64, device="cuda"))
        psi = torch.zeros(info.n_elem * info.n_ord * info.n_dof_elem, dtype=torch.float64, device="cuda")
        P.smm_get_psi(h, psi)
        h.destroy()
        psi_g = psi.cpu().numpy().reshape(info.n_elem, info.n_ord, info.n_dof_elem).transpose(1, 0, 2)
        psi_o = disc.sweep(None, q, pb, fixup=bool(fixup))
        assert np.max(np.abs(psi_g - psi_o)) <= 1e-11 * np.max(np.abs(psi_o))
        if fixup:
            assert psi_g.min() >= 0.0
        else:
            assert psi_g.min() < -1e-3


def test_iterate_with_fixup_matches_oracle():
    import paper_2304_07386_gb300 as P
    from oracle.smm import SMMProblem
    from tests.oracle_problems import disc_for
    p, sn = 2, 4
    mesh, st, ss, pb = strip(8, 50.0, 0.9)
    disc = disc_for(mesh, p, sn, st, ss)
    phi_o, k_o, _ = SMMProblem(disc, np.zeros((disc.ne, disc.n)), pb, fixup=True).iterate(tol=1e-12, relative=True)
    h = gpu(mesh, st, ss, pb, p, sn, 1, 1)
    x = torch.zeros(disc.ne * disc.n, dtype=torch.float64, device="cuda")
    rc, stats = P.smm_iterate(h, x, 1e-12, 100, relative=True)
    h.destroy()
    assert rc == 0 and abs(stats["outer_iterations"] - k_o) <= 1
    assert np.max(np.abs(x.cpu().numpy().reshape(disc.ne, disc.n) - phi_o)) <= 1e-9 * np.max(np.abs(phi_o))


def test_fixup_rejected_with_fp32_refined_sweep():
    import paper_2304_07386_gb300 as P
    mesh, st, ss, pb = strip()
    opt = P.smm_default_options()
    opt.negative_flux_fixup = 1
    opt.sweep_precision = P.SMM_SWEEP_FP32_REFINED
    with pytest.raises(P.SMMError):
        P.smm_create(mesh.nodes, mesh.elem_nodes, 1, 2, 4, st, ss, np.zeros((mesh.n_elem, 9)), inflow=pb, options=opt)
