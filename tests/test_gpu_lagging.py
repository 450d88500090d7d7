"""Cycle lagging on the GPU (Sec. 6.2 lags the cycles of its distorted
mesh's upwind graphs): meshes whose faces turn enough that grazing ordinates
enter some faces at some points and leave them at others.

Tolerances as in test_gpu_parity.py: 1e-11 relative per sweep, 1e-9 on
converged scalar fluxes.
"""
import numpy as np
import pytest

import smm_workloads as W
from tests.parity_inputs import sources

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_07386_gb300 import build as B
    B.build()


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def cyclic_problem(nx, m, p, sn, seed, kind="mms", c=0.6):
    mesh = W.structured_mesh(nx, m=m, perturb_seed=seed, wave_max=3, scale_by_k=False)
    ne = mesh.n_elem
    st = 1.0 + 0.5 * (np.arange(ne) % 3)
    pos = W.dg_node_positions(mesh, p)
    bf = W.boundary_faces(mesh)
    return dict(mesh=mesh, p=p, sn=sn, sigma_t=st, sigma_s=c * st, pos=pos, bfaces=bf,
                fpos=W.face_node_positions(mesh, p, bf), kind=kind)


def make_gpu(prob, **kw):
    import paper_2304_07386_gb300 as P
    om, _ = P.smm_quadrature(prob["sn"])
    q, inflow = sources(prob, om)
    opt = P.smm_default_options()
    for k, v in kw.items():
        setattr(opt, k, v)
    mesh = prob["mesh"]
    return P.smm_create(mesh.nodes, mesh.elem_nodes, mesh.m, prob["p"], prob["sn"], prob["sigma_t"],
                        prob["sigma_s"], q, inflow=inflow, options=opt)


def oracle(prob):
    from oracle.smm import SMMProblem
    from oracle.transport import Discretization
    mesh = prob["mesh"]
    disc = Discretization(mesh.nodes, mesh.elem_nodes, mesh.m, prob["p"], prob["sn"], prob["sigma_t"],
                          prob["sigma_s"])
    q, inflow = sources(prob, disc.omega)
    return disc, q, inflow, SMMProblem


CASES = [(5, 2, 1, 8, 1), (4, 2, 2, 12, 5), (4, 3, 3, 8, 2), (3, 2, 4, 8, 1)]


@pytest.mark.parametrize("solver", [0, 1], ids=["lu", "cached_inverse"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "nx%d_m%d_p%d_S%d" % c[:4])
def test_consecutive_lagged_sweeps_match_oracle(case, solver):
    """Two sweeps in a row: the first lags zero inflow (no previous sweep),
    the second the first's flux, as the oracle's sweeps given the same
    previous flux; moments of the second against the oracle's closures."""
    import paper_2304_07386_gb300 as P
    from oracle import closures
    prob = cyclic_problem(*case)
    h = make_gpu(prob, sweep_solver=solver)
    info = h.info()
    assert info.n_lagged > 0
    disc, q, inflow, _ = oracle(prob)
    assert info.n_lagged == sum(len(disc.upwind_order(d)[1]) for d in range(disc.nd))
    phi = W.mms_phi(prob["pos"][:, :, 0], prob["pos"][:, :, 1])
    prev = None
    for _ in range(2):
        P.smm_sweep(h, torch.as_tensor(phi.ravel(), device="cuda"))
        psi = torch.zeros(info.n_angular, dtype=torch.float64, device="cuda")
        P.smm_get_psi(h, psi)
        got = psi.cpu().numpy().reshape(info.n_elem, info.n_ord, info.n_dof_elem).transpose(1, 0, 2)
        ref = disc.sweep(phi, q, inflow, psi_lag=prev)
        assert rel(got, ref) < 1e-11
        prev = ref
    mom = torch.zeros(6 * info.n_elem * info.n_dof_elem, dtype=torch.float64, device="cuda")
    P.smm_moments(h, mom)
    mom_o = closures.nodal_moments(disc, prev)
    for c in range(6):
        assert np.max(np.abs(mom.cpu().numpy().reshape(6, info.n_elem, -1)[c] - mom_o[c])) <= \
            1e-11 * np.max(np.abs(mom_o[0]))


@pytest.mark.parametrize("solver", [0, 1], ids=["lu", "cached_inverse"])
def test_lagged_iteration_reaches_the_coupled_solution(solver):
    """With lagged sweeps the SMM iteration converges to the dense solution of
    the coupled transport + moment system (each ordinate's whole DG system
    solved at once), in about the oracle's number of outer steps."""
    import paper_2304_07386_gb300 as P
    from oracle.smm import coupled_dense_solve
    prob = cyclic_problem(4, 2, 1, 4, 1, c=0.9)
    disc, q, inflow, SMMProblem = oracle(prob)
    ref = coupled_dense_solve(SMMProblem(disc, q, inflow))
    _, k_o, _ = SMMProblem(disc, q, inflow).iterate(tol=1e-12, max_outer=300)
    h = make_gpu(prob, sweep_solver=solver, tol_cg=1e-14)
    x = torch.zeros(disc.ne * disc.n, dtype=torch.float64, device="cuda")
    rc, st = P.smm_iterate(h, x, 1e-12, 300)
    assert rel(x.cpu().numpy(), ref.ravel()) < 1e-9
    assert abs(st["outer_iterations"] - k_o) <= 1


def test_cycles_rejected_without_lagging_or_in_fp32_mode():
    import paper_2304_07386_gb300 as P
    prob = cyclic_problem(5, 2, 1, 8, 1)
    for kw in (dict(cycle_lagging=0), dict(sweep_precision=1), dict(negative_flux_fixup=1)):
        with pytest.raises(P.SMMError) as ei:
            make_gpu(prob, **kw)
        assert ei.value.status == 5, kw
