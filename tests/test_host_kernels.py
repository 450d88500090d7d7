"""The IP-SMM right-hand-side kernels of moments.cu, run on the CPU, against
the oracle's right-hand side (Eq. ipsmm); the angular-moment and boundary
correction kernels of the same file against the oracle's closures (Eqs.
correction_tensor_disc, bdr_correction_factor_disc); and the wavefront sweep
kernel of sweep.cu, in both FP64 local-solve forms, with the negative flux
fixup, in the FP32-refined form (FP64 residual, FP32 correction), and as the
batched kernel over several problems, against the oracle's upwind DG sweep
(Sec. 4); and the flexible-CG operator product and the level-0 smoothing step
of the moment solve (first, inner and last steps, with the CG update and dot
products folded into the first and last, and the residual restricted to the
element corners) against the oracle's IP-SMM matrix (Eq. ipsmm).

The kernel source (rhs_trace_kernel, rhs_assemble_kernel, the T staging
helper and the FP32-pair arithmetic of dfloat.cuh) is taken from the CUDA
files as text and compiled for the host with host_kernel_shim.h, which runs
every CUDA thread of a block as a std::thread with a barrier for
__syncthreads; rhs_emu.cpp feeds it the operators of the library's host
setup in the library's device layouts and launch shapes.  This checks the
kernels' indexing, shared-memory phases and pair arithmetic without a GPU;
the GPU parity tests check the same kernels on the device.  T carries jumps
across faces (smooth plus seeded noise) so that every face term counts.
"""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

import smm_workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2304_07386_gb300", "csrc")


def extract(src, signature):
    """The definition starting at `signature` (with a template line just above
    it), through its closing brace."""
    i = src.index(signature)
    line_start = src.rfind("\n", 0, i - 1) + 1
    if src.startswith("template", line_start):
        i = line_start
    depth, k = 0, src.index("{", i)
    while True:
        depth += {"{": 1, "}": -1}.get(src[k], 0)
        if depth == 0:
            return src[i:k + 1]
        k += 1


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("rhs_emu")
    moments = open(os.path.join(CSRC, "moments.cu")).read()
    dfloat = open(os.path.join(CSRC, "dfloat.cuh")).read()
    body = dfloat[dfloat.index("namespace smm {") + len("namespace smm {"):dfloat.rindex("}")]
    parts = [body,
             extract(moments, "__device__ __forceinline__ void stage_T("),
             extract(moments, "__global__ void rhs_trace_kernel("),
             extract(moments, "__global__ void rhs_assemble_kernel(")]
    inc = "\n".join(parts)
    n_shared = len(re.findall(r"extern __shared__ float2 (\w+)\[\];", inc))
    assert n_shared == 2
    inc = re.sub(r"extern __shared__ float2 (\w+)\[\];", r"float2* \1 = (float2*)emu_dynamic_smem;", inc)
    (d / "rhs_kernels.inc").write_text(inc)
    exe = d / "rhs_emu"
    subprocess.run([cxx, "-std=c++20", "-O1", "-ffp-contract=off", "-pthread", "-I", str(d), "-I",
                    os.path.join(ROOT, "tests"), "-I", CSRC, os.path.join(ROOT, "tests", "rhs_emu.cpp"),
                    os.path.join(CSRC, "setup.cpp"), "-o", str(exe)], check=True)
    return str(exe)


# (nx, ny, m, p, seed, noise): every element size the kernels are compiled for, curved maps, a
# one-element mesh, and a finer mesh with smooth T (where the pair products cancel most)
CASES = [(3, 2, 1, 1, None, 0.1), (3, 3, 2, 2, 4, 0.1), (2, 3, 3, 3, 7, 0.1), (3, 2, 3, 4, 2, 0.1),
         (1, 1, 1, 2, None, 0.1), (2, 2, 6, 4, 5, 0.1), (8, 8, 3, 4, 3, 0.0)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "nx%d_ny%d_m%d_p%d" % c[:4])
def test_rhs_kernels_match_oracle(emu, tmp_path, case):
    from oracle import closures, ipsmm
    from oracle.transport import Discretization
    nx, ny, m, p, seed, noise = case
    mesh = W.structured_mesh(nx, ny, m=m, perturb_seed=seed)
    ne, n = mesh.n_elem, (p + 1) ** 2
    st = 1.0 + 0.25 * (np.arange(ne) % 4)
    rng = np.random.default_rng(17)
    q = rng.uniform(0.5, 1.5, (ne, n))
    pos = W.dg_node_positions(mesh, p)
    x, y = pos[:, :, 0], pos[:, :, 1]
    T = np.stack([np.sin(2 * x + 1) * np.cos(1.5 * y), 0.5 * np.cos(2 * x - y), 0.8 * np.sin(x + 2 * y) + 0.3])
    T = T + noise * rng.standard_normal(T.shape)
    mom = np.concatenate([rng.uniform(0.5, 1.5, (3, ne, n)), T])
    disc = Discretization(mesh.nodes, mesh.elem_nodes, m, p, 4, st, 0.5 * st)
    nfq = len(disc.elems[0].fq_s)
    beta = rng.uniform(-0.2, 0.2, (len(disc.bfaces), nfq))
    np.asarray(mesh.nodes, np.float64).tofile(tmp_path / "nodes.f64")
    np.asarray(mesh.elem_nodes, np.int32).tofile(tmp_path / "elem.i32")
    st.tofile(tmp_path / "sigma_t.f64")
    q.tofile(tmp_path / "q.f64")
    mom.tofile(tmp_path / "mom.f64")
    beta.tofile(tmp_path / "beta.f64")
    subprocess.run([emu, str(tmp_path), str(ne), str(len(mesh.nodes)), str(m), str(p)], check=True, timeout=300)
    n_out, nfq_out, nb_out = map(int, open(tmp_path / "dims.txt").read().split())
    assert (n_out, nfq_out, nb_out) == (n, nfq, len(disc.bfaces))
    rhs = np.fromfile(tmp_path / "rhs.f64")
    Q = closures.source_moments(disc, np.broadcast_to(q, (disc.nd,) + q.shape))
    jin = closures.j_in(disc, None)
    b = ipsmm.assemble_rhs(disc, Q, T, jin, beta)
    assert np.max(np.abs(rhs - b)) <= 1e-12 * np.max(np.abs(b)), np.max(np.abs(rhs - b)) / np.max(np.abs(b))


# ---------------------------------------------------------------------------
# angular moments and the boundary correction (the sweep kernel's epilogue,
# element_moments, from the FP64 flux and from its pair copy) against the
# oracle's closures

@pytest.fixture(scope="module")
def moments_emu(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("moments_emu")
    sweep = open(os.path.join(CSRC, "sweep.cu")).read()
    kcuh = open(os.path.join(CSRC, "kernels.cuh")).read()
    dfloat = open(os.path.join(CSRC, "dfloat.cuh")).read()
    body = dfloat[dfloat.index("namespace smm {") + len("namespace smm {"):dfloat.rindex("}")]
    enums = re.findall(r"enum : int \{[^}]*\};", kcuh)
    parts = enums + [extract(kcuh, "struct SweepArgs {") + ";", body,
                     extract(sweep, "__device__ __noinline__ void element_moments(")]
    (d / "moments_kernels.inc").write_text("\n".join(parts))
    exe = d / "moments_emu"
    subprocess.run([cxx, "-std=c++20", "-O1", "-ffp-contract=off", "-pthread", "-I", str(d), "-I",
                    os.path.join(ROOT, "tests"), "-I", CSRC, os.path.join(ROOT, "tests", "moments_emu.cpp"),
                    os.path.join(CSRC, "setup.cpp"), "-o", str(exe)], check=True)
    return str(exe)


# (nx, ny, m, p, S_N, seed): every element size, S2 to S12 (fewer and more
# ordinates than a warp's lanes), curved maps, a one-element mesh
MOMENT_CASES = [(3, 2, 1, 1, 4, None), (2, 3, 2, 2, 8, 4), (3, 3, 3, 3, 12, 7), (2, 2, 3, 4, 8, 2),
                (1, 1, 1, 2, 2, None)]


@pytest.mark.parametrize("case", MOMENT_CASES, ids=lambda c: "nx%d_ny%d_m%d_p%d_S%d" % c[:5])
def test_moment_kernels_match_oracle(moments_emu, tmp_path, case):
    from oracle import closures
    from oracle.transport import Discretization
    nx, ny, m, p, sn, seed = case
    mesh = W.structured_mesh(nx, ny, m=m, perturb_seed=seed)
    ne, n = mesh.n_elem, (p + 1) ** 2
    st = np.ones(ne)
    disc = Discretization(mesh.nodes, mesh.elem_nodes, m, p, sn, st, 0.5 * st)
    rng = np.random.default_rng(23)
    pos = W.dg_node_positions(mesh, p)
    # an anisotropic, spatially varying psi [nd][ne][n] with seeded noise, so that
    # every moment and every boundary sum is nonzero
    om = disc.omega
    psi = (1.0 + 0.5 * om[:, 0, None, None] * np.sin(2 * pos[None, :, :, 0])
           + 0.3 * om[:, 1, None, None] ** 2 * np.cos(pos[None, :, :, 1])
           + 0.2 * rng.uniform(0.0, 1.0, (disc.nd, ne, n)))
    np.asarray(mesh.nodes, np.float64).tofile(tmp_path / "nodes.f64")
    np.asarray(mesh.elem_nodes, np.int32).tofile(tmp_path / "elem.i32")
    st.tofile(tmp_path / "sigma_t.f64")
    np.ones((ne, n)).tofile(tmp_path / "q.f64")
    np.ascontiguousarray(psi.transpose(1, 0, 2)).tofile(tmp_path / "psi.f64")
    subprocess.run([moments_emu, str(tmp_path), str(ne), str(len(mesh.nodes)), str(m), str(p), str(sn)],
                   check=True, timeout=300)
    n_o, nd_o, nfq_o, nb_o = map(int, open(tmp_path / "dims.txt").read().split())
    mom_ref = closures.nodal_moments(disc, psi)
    beta_ref = closures.beta(disc, psi)
    assert (n_o, nd_o, nb_o) == (n, disc.nd, len(disc.bfaces)) and beta_ref.shape == (nb_o, nfq_o)
    scale = np.max(np.abs(mom_ref))
    # FP64 sums: rounding only.  Pair sums: each of the nd pair multiply-adds
    # leaves the float correction term an error of about 2^-48 of the sum
    # (and the pair copy of psi differs from it by 2^-48).
    for name, tol in (("mom", 1e-13), ("mom_df", 4 * disc.nd * 2.0 ** -48)):
        got = np.fromfile(tmp_path / f"{name}.f64").reshape(6, ne, n)
        assert np.max(np.abs(got - mom_ref)) <= tol * scale, (name, np.max(np.abs(got - mom_ref)) / scale)
    # beta is a difference of terms of the size of phi (zero for S2, whose
    # ordinates all have the same |Omega.n| on the straight boundary)
    for name in ("beta", "beta_df"):
        beta = np.fromfile(tmp_path / f"{name}.f64").reshape(nb_o, nfq_o)
        assert np.max(np.abs(beta - beta_ref)) <= 1e-13 * scale, name
    if sn == 2:
        assert np.max(np.abs(beta_ref)) <= 1e-13 * scale
    else:
        assert np.max(np.abs(beta_ref)) > 1e-3 * scale


# ---------------------------------------------------------------------------
# the wavefront sweep kernel (sweep_kernel with the in-register LU and with
# cached pair inverses, after invert_kernel / source_kernel / mass_apply_kernel)
# against the oracle's sweep

@pytest.fixture(scope="module")
def sweep_emu(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("sweep_emu")
    sweep = open(os.path.join(CSRC, "sweep.cu")).read()
    kcuh = open(os.path.join(CSRC, "kernels.cuh")).read()
    dfloat = open(os.path.join(CSRC, "dfloat.cuh")).read()
    body = dfloat[dfloat.index("namespace smm {") + len("namespace smm {"):dfloat.rindex("}")]
    enums = re.findall(r"enum : int \{[^}]*\};", kcuh)
    assert len(enums) == 2
    parts = enums + [extract(kcuh, "struct SweepArgs {") + ";", extract(kcuh, "struct ResidualArgs {") + ";", body,
                     extract(sweep, "__device__ bool wait_epoch("),
                     extract(sweep, "__device__ __forceinline__ int face_node("),
                     extract(sweep, "template <typename T> __device__ __forceinline__ T ldg_cg("),
                     extract(sweep, "__device__ __noinline__ void element_moments("),
                     extract(sweep, "__device__ bool sweep_gate("),
                     extract(sweep, "__device__ __forceinline__ bool sweep_task("),
                     extract(sweep, "__global__ void __launch_bounds__(256, INV ? (P <= 3 ? 5 : 3) : 1) sweep_kernel("),
                     extract(sweep, "__global__ void __launch_bounds__(256, INV ? (PMAX <= 3 ? 5 : 3) : 1) batch_sweep_kernel("),
                     extract(sweep, "__global__ void __launch_bounds__(256) invert_kernel("),
                     extract(sweep, "__global__ void __launch_bounds__(256) residual_kernel("),
                     extract(sweep, "__global__ void mass_apply_kernel("),
                     extract(sweep, "__global__ void source_kernel(")]
    (d / "sweep_kernels.inc").write_text("\n".join(parts))
    exe = d / "sweep_emu"
    subprocess.run([cxx, "-std=c++20", "-O1", "-ffp-contract=off", "-pthread", "-I", str(d), "-I",
                    os.path.join(ROOT, "tests"), "-I", CSRC, os.path.join(ROOT, "tests", "sweep_emu.cpp"),
                    os.path.join(CSRC, "setup.cpp"), "-o", str(exe)], check=True)
    return str(exe)


# (nx, ny, m, p, S_N, seed, kind): every p, straight and curved maps, isotropic
# source with vacuum boundaries or the manufactured angular source with its
# inflow, a one-element mesh and a ragged strip
SWEEP_CASES = [(3, 2, 1, 1, 4, None, "iso"), (2, 3, 2, 2, 4, 4, "mms"), (3, 3, 3, 3, 4, 7, "mms"),
               (2, 2, 3, 4, 4, 2, "mms"), (1, 1, 1, 2, 8, None, "iso"), (5, 1, 2, 1, 8, 3, "mms")]


def _sweep_problem(case, sig=None, strip_light=False, strong=False, fan=0.0):
    """Mesh, cross sections, the oracle's discretization, varphi, q and inflow
    of one sweep case (isotropic q with vacuum boundaries, or the manufactured
    angular source with its inflow, or a strip lit from the left face)."""
    from oracle.transport import Discretization
    nx, ny, m, p, sn, seed, kind = case
    mesh = (W.structured_mesh(nx, ny, m=m, perturb_seed=seed, wave_max=3, scale_by_k=False) if strong
            else W.structured_mesh(nx, ny, m=m, perturb_seed=seed, fan=fan))
    ne, n = mesh.n_elem, (p + 1) ** 2
    st = np.full(ne, sig) if sig is not None else 1.0 + 0.5 * (np.arange(ne) % 3)
    ss = (0.0 if strip_light else 0.6) * st
    disc = Discretization(mesh.nodes, mesh.elem_nodes, m, p, sn, st, ss)
    rng = np.random.default_rng(31)
    phi = rng.uniform(0.5, 2.0, (ne, n))
    pos = W.dg_node_positions(mesh, p)
    if kind == "mms":
        fpos = W.face_node_positions(mesh, p, W.boundary_faces(mesh))
        q = np.stack([W.mms_source(pos[:, :, 0], pos[:, :, 1], o[0], o[1], st[:, None], ss[:, None])
                      for o in disc.omega])
        inflow = np.stack([W.mms_psi(fpos[:, :, 0], fpos[:, :, 1], o[0], o[1]) for o in disc.omega])
    elif kind == "strip":
        q = np.zeros((ne, n))
        inflow = np.zeros((disc.nd, len(disc.bfaces), p + 1))
        for b, (e, f) in enumerate(W.boundary_faces(mesh)):
            if f == 3:
                inflow[:, b, :] = 1.0
    else:
        q, inflow = rng.uniform(0.0, 1.0, (ne, n)), None
    return mesh, st, ss, disc, phi, q, inflow


def _run_sweep_emu(exe, tmp_path, case, mode="plain", K=0, psi_lag=None, **kw):
    nx, ny, m, p, sn, seed, kind = case
    mesh, st, ss, disc, phi, q, inflow = _sweep_problem(case, **kw)
    ne, n = mesh.n_elem, (p + 1) ** 2
    if psi_lag is not None:
        np.ascontiguousarray(psi_lag(disc).transpose(1, 0, 2), np.float64).tofile(tmp_path / "psi_lag.f64")
    for name, arr in (("nodes", mesh.nodes), ("sigma_t", st), ("sigma_s", ss), ("phi", phi), ("q", q)):
        np.ascontiguousarray(arr, np.float64).tofile(tmp_path / f"{name}.f64")
    np.asarray(mesh.elem_nodes, np.int32).tofile(tmp_path / "elem.i32")
    if inflow is not None:
        np.ascontiguousarray(inflow, np.float64).tofile(tmp_path / "inflow.f64")
    (tmp_path / "nbface.txt").write_text(str(len(disc.bfaces)))
    subprocess.run([exe, str(tmp_path), str(ne), str(len(mesh.nodes)), str(m), str(p), str(sn),
                    str(int(q.ndim == 3)), str(int(inflow is not None)), mode, str(K)], check=True, timeout=600)
    n_o, nd_o, nb_o, nlev = map(int, open(tmp_path / "dims.txt").read().split())
    assert (n_o, nd_o, nb_o) == (n, disc.nd, len(disc.bfaces))
    assert open(tmp_path / "err.txt").read().split() == ["0", "0"]
    names = ("psi_lu", "psi_inv") + (("psi2_inv",) if mode != "refine" else ())
    got = {k: np.fromfile(tmp_path / f"{k}.f64").reshape(ne, disc.nd, n) for k in names}
    got_mom = {k: np.fromfile(tmp_path / f"mom_{k}.f64").reshape(6, ne, n) for k in ("lu", "inv")}
    got_beta = {k: np.fromfile(tmp_path / f"beta_{k}.f64").reshape(len(disc.bfaces), -1) for k in ("lu", "inv")}
    _run_sweep_emu.moments = (got_mom, got_beta)
    return disc, phi, q, inflow, got


def _check_fused_moments(disc, psi_nd, tol=1e-12):
    """The moments and beta the last emulated sweep formed in its epilogue
    (each element's last task in list order, after the element's other
    ordinates) against the oracle's closures of psi_nd ([nd][ne][n])."""
    from oracle import closures
    got_mom, got_beta = _run_sweep_emu.moments
    mom_ref = closures.nodal_moments(disc, psi_nd)
    beta_ref = closures.beta(disc, psi_nd)
    scale = np.max(np.abs(mom_ref))
    for k in ("lu", "inv"):
        assert np.max(np.abs(got_mom[k] - mom_ref)) <= tol * scale, (k, np.max(np.abs(got_mom[k] - mom_ref)) / scale)
        assert np.max(np.abs(got_beta[k] - beta_ref)) <= tol * scale, k


@pytest.mark.parametrize("case", SWEEP_CASES, ids=lambda c: "nx%d_ny%d_m%d_p%d_S%d_%s" % (c[:5] + c[6:]))
def test_sweep_kernel_matches_oracle(sweep_emu, tmp_path, case):
    disc, phi, q, inflow, got = _run_sweep_emu(sweep_emu, tmp_path, case)
    ref_nd = disc.sweep(phi, q, inflow)
    ref = ref_nd.transpose(1, 0, 2)   # [ne][nd][n], the device layout
    scale = np.max(np.abs(ref))
    for name, psi in got.items():
        assert np.max(np.abs(psi - ref)) <= 1e-12 * scale, (name, np.max(np.abs(psi - ref)) / scale)
    _check_fused_moments(disc, ref_nd)


@pytest.mark.parametrize("case", [(4, 3, 1, 1, 8, None, "mms"), (3, 3, 2, 2, 12, None, "mms"),
                                  (4, 2, 1, 3, 8, None, "iso")], ids=lambda c: "nx%d_ny%d_m%d_p%d_S%d_%s" % (c[:5] + c[6:]))
def test_sweep_kernel_takes_three_inflow_faces(sweep_emu, tmp_path, case):
    """On a fan mesh (trapezoids that widen upwards) an ordinate pointing up
    enters some elements through three straight faces (two is the rule on
    meshes of nearly parallel faces); the sweep and its moments must still
    equal the oracle's."""
    disc, phi, q, inflow, got = _run_sweep_emu(sweep_emu, tmp_path, case, fan=1.5)
    three = sum(1 for e in range(disc.ne) for d in range(disc.nd)
                if sum(bool(np.all(disc.faces[e][f]["nds"] @ disc.omega[d] < 0.0)) for f in range(4)) == 3)
    assert three > 0
    ref_nd = disc.sweep(phi, q, inflow)
    ref = ref_nd.transpose(1, 0, 2)
    scale = np.max(np.abs(ref))
    for name, psi in got.items():
        assert np.max(np.abs(psi - ref)) <= 1e-12 * scale, (name, np.max(np.abs(psi - ref)) / scale)
    _check_fused_moments(disc, ref_nd)


def test_sweep_kernel_wait_expires_and_the_next_sweep_is_exact(sweep_emu, tmp_path):
    """The bounded dependency wait: with the first task of the list never run,
    its flag is never published and the tasks downwind of it give up after the
    timeout (20 ms here).  Each form of the kernel must then return with the
    device error word at DEV_TIMEOUT (every warp stopping, or the launch would
    not end), and the following sweep on the same flags -- error word cleared,
    next epoch, whole list, as the library's next call runs it -- must equal
    the oracle's sweep: flags left at the old epoch are harmless."""
    import re as _re
    kcuh = open(os.path.join(CSRC, "kernels.cuh")).read()
    dev_timeout = int(_re.search(r"DEV_TIMEOUT = (\d+)", kcuh).group(1))
    case = (3, 3, 2, 2, 4, 4, "mms")
    disc, phi, q, inflow, got = _run_sweep_emu(sweep_emu, tmp_path, case, "timeout")
    e1_lu, e2_lu, e1_inv, e2_inv = map(int, open(tmp_path / "timeout_err.txt").read().split())
    assert (e1_lu, e1_inv) == (dev_timeout, dev_timeout)
    assert (e2_lu, e2_inv) == (0, 0)
    ref = disc.sweep(phi, q, inflow).transpose(1, 0, 2)
    scale = np.max(np.abs(ref))
    for name, psi in got.items():
        assert np.max(np.abs(psi - ref)) <= 1e-12 * scale, (name, np.max(np.abs(psi - ref)) / scale)


@pytest.mark.parametrize("case", [(5, 5, 2, 1, 8, 1, "mms"), (4, 4, 2, 2, 12, 5, "iso"), (4, 3, 3, 3, 8, 2, "mms")],
                         ids=lambda c: "nx%d_ny%d_m%d_p%d_S%d" % c[:5])
def test_sweep_kernel_lags_cycles_like_the_oracle(sweep_emu, tmp_path, case):
    """Meshes whose faces turn enough (wave numbers up to 3, amplitude 0.05)
    that grazing ordinates enter some faces at some points and leave them at
    others: the upwind graphs have cycles.  The kernels with their optional
    parts (the LU and the cached pair inverses, built with the pointwise face
    matrices) sweep with the faces the setup lagged reading a given previous
    flux, as the oracle's lagged sweep does with the same previous flux; the
    moments formed after the sweep match the oracle's closures."""
    rng = np.random.default_rng(9)

    def lag(disc):
        return rng.uniform(0.2, 1.2, (disc.nd, disc.ne, disc.n))
    store = {}

    def lag_keep(disc):
        store["lag"] = lag(disc)
        return store["lag"]
    disc, phi, q, inflow, got = _run_sweep_emu(sweep_emu, tmp_path, case, "lag", psi_lag=lag_keep, strong=True)
    assert sum(len(disc.upwind_order(d)[1]) for d in range(disc.nd)) > 0
    ref_nd = disc.sweep(phi, q, inflow, psi_lag=store["lag"])
    ref = ref_nd.transpose(1, 0, 2)
    scale = np.max(np.abs(ref))
    for name, psi in got.items():
        assert np.max(np.abs(psi - ref)) <= 1e-12 * scale, (name, np.max(np.abs(psi - ref)) / scale)
    _check_fused_moments(disc, ref_nd)


def test_batched_sweep_kernel_matches_oracle(sweep_emu, tmp_path):
    """Problems of different p, S_N, size, geometry and source kind swept by
    one batch_sweep_kernel launch over their merged level-by-level task list
    (each task dispatching on its problem's p), with the LU and with cached
    inverses, each against the oracle's sweep of that problem."""
    cases = [(3, 2, 1, 1, 4, None, "iso"), (2, 3, 2, 2, 8, 4, "mms"), (2, 2, 3, 4, 4, 2, "mms"),
             (1, 1, 1, 3, 2, None, "iso")]
    refs = []
    for k, case in enumerate(cases):
        nx, ny, m, p, sn, seed, kind = case
        mesh, st, ss, disc, phi, q, inflow = _sweep_problem(case)
        d = tmp_path / str(k)
        d.mkdir()
        for name, arr in (("nodes", mesh.nodes), ("sigma_t", st), ("sigma_s", ss), ("phi", phi), ("q", q)):
            np.ascontiguousarray(arr, np.float64).tofile(d / f"{name}.f64")
        np.asarray(mesh.elem_nodes, np.int32).tofile(d / "elem.i32")
        if inflow is not None:
            np.ascontiguousarray(inflow, np.float64).tofile(d / "inflow.f64")
        (d / "nbface.txt").write_text(str(len(disc.bfaces)))
        (d / "args.txt").write_text("%d %d %d %d %d %d %d" % (mesh.n_elem, len(mesh.nodes), m, p, sn, int(q.ndim == 3),
                                                           int(inflow is not None)))
        refs.append(disc.sweep(phi, q, inflow).transpose(1, 0, 2))
    subprocess.run([sweep_emu, "--batch", str(tmp_path), str(len(cases))], check=True, timeout=600)
    for k, ref in enumerate(refs):
        d = tmp_path / str(k)
        assert open(d / "err.txt").read().split() == ["0", "0"]
        scale = np.max(np.abs(ref))
        for name in ("psi_lu", "psi_inv", "psi2_inv"):
            got = np.fromfile(d / f"{name}.f64").reshape(ref.shape)
            assert np.max(np.abs(got - ref)) <= 1e-12 * scale, (k, name, np.max(np.abs(got - ref)) / scale)
        # the moments each problem's own last tasks formed inside the batched launch
        from oracle import closures
        disc = _sweep_problem(cases[k])[3]
        ref_nd = ref.transpose(1, 0, 2)
        mom_ref, beta_ref = closures.nodal_moments(disc, ref_nd), closures.beta(disc, ref_nd)
        mscale = np.max(np.abs(mom_ref))
        for form in ("lu", "inv"):
            mom = np.fromfile(d / f"mom_{form}.f64").reshape(mom_ref.shape)
            beta = np.fromfile(d / f"beta_{form}.f64").reshape(beta_ref.shape)
            assert np.max(np.abs(mom - mom_ref)) <= 1e-12 * mscale, (k, form)
            assert np.max(np.abs(beta - beta_ref)) <= 1e-12 * mscale, (k, form)


def test_sweep_kernel_fixup_matches_oracle(sweep_emu, tmp_path):
    """The kernels with their optional parts compiled in and the zero-and-scale
    fixup on, on a thick absorbing strip lit from the left whose DG solution
    dips below zero (Sec. 6.3), against the oracle's sweep with its fixup."""
    case = (6, 1, 1, 2, 4, None, "strip")
    disc, phi, q, inflow, got = _run_sweep_emu(sweep_emu, tmp_path, case, "fixup", sig=30.0, strip_light=True)
    plain = disc.sweep(phi, q, inflow)
    assert plain.min() < 0.0            # the case needs the fixup
    ref = disc.sweep(phi, q, inflow, fixup=True).transpose(1, 0, 2)
    assert ref.min() >= 0.0
    scale = np.max(np.abs(ref))
    for name, psi in got.items():
        assert np.max(np.abs(psi - ref)) <= 1e-12 * scale, (name, np.max(np.abs(psi - ref)) / scale)
    _check_fused_moments(disc, ref.transpose(1, 0, 2))


@pytest.mark.parametrize("case", [SWEEP_CASES[1], SWEEP_CASES[3]], ids=["p2_curved", "p4_curved"])
def test_fp32_refined_sweeps_converge_to_the_fp64_sweep(sweep_emu, tmp_path, case):
    """The FP32-refined form: one sweep is FP32-accurate, and repeated residual
    sweeps (FP64 residual, FP32 correction) reach the FP64 sweep."""
    errs = {}
    for K in (1, 4):
        disc, phi, q, inflow, got = _run_sweep_emu(sweep_emu, tmp_path, case, "refine", K)
        ref = disc.sweep(phi, q, inflow).transpose(1, 0, 2)
        scale = np.max(np.abs(ref))
        errs[K] = {k: np.max(np.abs(v - ref)) / scale for k, v in got.items()}
    for name in ("psi_lu", "psi_inv"):
        assert 1e-10 < errs[1][name] < 1e-5, (name, errs)
        assert errs[4][name] < 1e-12, (name, errs)
    # the moments formed inside the last correction sweep, from the accumulated FP64 flux
    _check_fused_moments(disc, ref.transpose(1, 0, 2), tol=1e-11)


# ---------------------------------------------------------------------------
# the flexible-CG operator product (cgx_spmv_kernel: q = A p on the
# face-factored IP-SMM operator in FP32-pair arithmetic, p.q by the last-block
# reduction) against the oracle's assembled IP-SMM matrix

def _operator_helpers():
    """The operator structs of kernels.cuh, the pair arithmetic and the row and
    reduction helpers of blockops.cuh, its cache-policy loads (inline
    assembly) made plain loads."""
    kcuh = open(os.path.join(CSRC, "kernels.cuh")).read()
    dfloat = open(os.path.join(CSRC, "dfloat.cuh")).read()
    blockops = open(os.path.join(CSRC, "blockops.cuh")).read()
    body = dfloat[dfloat.index("namespace smm {") + len("namespace smm {"):dfloat.rindex("}")]
    ops = blockops[blockops.index("namespace smm {") + len("namespace smm {"):blockops.rindex("}")]
    # the cache-policy loads (inline assembly) become plain loads
    host = {"__device__ __forceinline__ unsigned long long l2_keep(": "inline unsigned long long l2_keep() { return 0; }",
            "__device__ __forceinline__ unsigned long long l2_stream(":
                "inline unsigned long long l2_stream() { return 0; }",
            "__device__ __forceinline__ float ld_hint(const float* a":
                "inline float ld_hint(const float* a, unsigned long long) { return *a; }",
            "__device__ __forceinline__ float2 ld_hint(const float2* a":
                "inline float2 ld_hint(const float2* a, unsigned long long) { return *a; }"}
    for sig, repl in host.items():
        ops = ops.replace(extract(ops, sig), repl)
    assert "asm" not in ops
    return [extract(kcuh, "struct FaceOp {") + ";", extract(kcuh, "struct FaceOpDF {") + ";",
            extract(kcuh, "struct CGArgs {") + ";", body, ops]


@pytest.fixture(scope="module")
def cg_emu(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("cg_emu")
    moments = open(os.path.join(CSRC, "moments.cu")).read()
    parts = _operator_helpers() + [extract(moments, "__global__ void __launch_bounds__(256) cgx_spmv_kernel(")]
    (d / "cg_kernels.inc").write_text("\n".join(parts))
    exe = d / "cg_emu"
    subprocess.run([cxx, "-std=c++20", "-O1", "-ffp-contract=off", "-pthread", "-I", str(d), "-I",
                    os.path.join(ROOT, "tests"), "-I", CSRC, os.path.join(ROOT, "tests", "cg_emu.cpp"),
                    os.path.join(CSRC, "setup.cpp"), "-o", str(exe)], check=True)
    return str(exe)


# (nx, ny, m, p, seed): every element size, curved maps, a one-element mesh, and
# meshes with more elements than one block's slots (several blocks and the
# last-block reduction), ragged against the two-elements-per-thread tiling
# (a block holds 2 x 64 / 28 / 16 / 10 elements for p = 1 / 2 / 3 / 4)
CG_CASES = [(3, 2, 1, 1, None), (4, 3, 2, 2, 4), (3, 3, 3, 3, 7), (3, 2, 3, 4, 2), (1, 1, 1, 2, None),
            (12, 11, 1, 1, 5), (8, 8, 2, 2, 3), (7, 5, 3, 3, 6), (5, 5, 3, 4, 2)]


@pytest.mark.parametrize("case", CG_CASES, ids=lambda c: "nx%d_ny%d_m%d_p%d" % c[:4])
def test_cg_operator_product_matches_oracle(cg_emu, tmp_path, case):
    from oracle import ipsmm
    from oracle.transport import Discretization
    nx, ny, m, p, seed = case
    mesh = W.structured_mesh(nx, ny, m=m, perturb_seed=seed)
    ne, n = mesh.n_elem, (p + 1) ** 2
    st = 1.0 + 0.5 * (np.arange(ne) % 3)
    ss = 0.7 * st
    rng = np.random.default_rng(41)
    pv = rng.standard_normal((ne, n))
    for name, arr in (("nodes", mesh.nodes), ("sigma_t", st), ("sigma_s", ss), ("q", np.ones((ne, n))), ("p", pv)):
        np.ascontiguousarray(arr, np.float64).tofile(tmp_path / f"{name}.f64")
    np.asarray(mesh.elem_nodes, np.int32).tofile(tmp_path / "elem.i32")
    subprocess.run([cg_emu, str(tmp_path), str(ne), str(len(mesh.nodes)), str(m), str(p)], check=True, timeout=600)
    disc = Discretization(mesh.nodes, mesh.elem_nodes, m, p, 4, st, ss)
    A = ipsmm.assemble_lhs(disc).tocsr()
    ref = A @ pv.ravel()
    scale = np.max(abs(A) @ np.abs(pv.ravel()))
    q = np.fromfile(tmp_path / "q_out.f64")
    assert np.max(np.abs(q - ref)) <= 1e-12 * scale, np.max(np.abs(q - ref)) / scale
    scal = np.fromfile(tmp_path / "scal.f64")
    pq = float(pv.ravel() @ q)
    assert abs(scal[1] - pq) <= 1e-12 * float(np.abs(pv.ravel()) @ np.abs(q))
    assert scal[5] == pytest.approx(1.0 / scal[1], rel=1e-15)


# ---------------------------------------------------------------------------
# one level-0 smoothing step of the multigrid preconditioner (bj_smooth_kernel,
# FP32) against the same step formed from the oracle's IP-SMM matrix

@pytest.fixture(scope="module")
def smooth_emu(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("smooth_emu")
    mg = open(os.path.join(CSRC, "mg.cu")).read()
    kcuh = open(os.path.join(CSRC, "kernels.cuh")).read()
    # the L2 prefetch (inline assembly) of the residual kernel is a no-op here
    parts = _operator_helpers() + [extract(kcuh, "struct L2Chunk {") + ";",
                                   "inline void prefetch_l2(const void*, unsigned) {}",
                                   extract(mg, "__device__ __forceinline__ bool mg_skip("),
                                   extract(mg, "__global__ void __launch_bounds__(256) bj_residual_kernel("),
                                   extract(mg, "__global__ void __launch_bounds__(256) bj_smooth_kernel("),
                                   extract(mg, "__global__ void __launch_bounds__(256) bj_last_dots_kernel("),
                                   extract(mg, "__global__ void __launch_bounds__(256) bj_first_update_kernel(")]
    (d / "smooth_kernels.inc").write_text("\n".join(parts))
    exe = d / "smooth_emu"
    subprocess.run([cxx, "-std=c++20", "-O1", "-ffp-contract=off", "-pthread", "-I", str(d), "-I",
                    os.path.join(ROOT, "tests"), "-I", CSRC, os.path.join(ROOT, "tests", "smooth_emu.cpp"),
                    os.path.join(CSRC, "setup.cpp"), "-o", str(exe)], check=True)
    return str(exe)


@pytest.mark.parametrize("case", CG_CASES, ids=lambda c: "nx%d_ny%d_m%d_p%d" % c[:4])
def test_level0_smoothing_step_matches_oracle(smooth_emu, tmp_path, case):
    """xout = xin + c2 A_d^{-1} (b - A xin) + c1 (xin - xprev) (a Chebyshev
    step; the first step of a V-cycle has xin = xprev = 0)."""
    from oracle import ipsmm
    from oracle.transport import Discretization
    nx, ny, m, p, seed = case
    mesh = W.structured_mesh(nx, ny, m=m, perturb_seed=seed)
    ne, n = mesh.n_elem, (p + 1) ** 2
    st = 1.0 + 0.5 * (np.arange(ne) % 3)
    ss = 0.7 * st
    rng = np.random.default_rng(43)
    b = rng.standard_normal(ne * n)
    xin = rng.standard_normal(ne * n).astype(np.float32)
    xprev = rng.standard_normal(ne * n).astype(np.float32)
    for name, arr in (("nodes", mesh.nodes), ("sigma_t", st), ("sigma_s", ss), ("q", np.ones((ne, n))), ("b", b)):
        np.ascontiguousarray(arr, np.float64).tofile(tmp_path / f"{name}.f64")
    np.asarray(mesh.elem_nodes, np.int32).tofile(tmp_path / "elem.i32")
    xin.tofile(tmp_path / "xin.f32")
    xprev.tofile(tmp_path / "xprev.f32")
    disc = Discretization(mesh.nodes, mesh.elem_nodes, m, p, 4, st, ss)
    A = ipsmm.assemble_lhs(disc).toarray()
    Pinv = np.zeros_like(A)
    for e in range(ne):
        sl = slice(e * n, (e + 1) * n)
        Pinv[sl, sl] = np.linalg.inv(A[sl, sl])
    c1, c2 = 0.375, 0.8125            # exactly representable in FP32
    for first in (1, 0):
        subprocess.run([smooth_emu, str(tmp_path), str(ne), str(len(mesh.nodes)), str(m), str(p), str(c1), str(c2),
                        str(first)], check=True, timeout=600)
        got = np.fromfile(tmp_path / "xout.f32", dtype=np.float32).astype(np.float64)
        x0 = np.zeros(ne * n) if first else xin.astype(np.float64)
        xp = np.zeros(ne * n) if first else xprev.astype(np.float64)
        ref = x0 + c2 * (Pinv @ (b - A @ x0)) + c1 * (x0 - xp)
        scale = np.max(np.abs(x0)) + c2 * np.max(np.abs(Pinv) @ (np.abs(b) + np.abs(A) @ np.abs(x0))) + \
            c1 * np.max(np.abs(x0) + np.abs(xp))
        assert np.max(np.abs(got - ref)) <= 1e-5 * scale, (first, np.max(np.abs(got - ref)) / scale)


@pytest.mark.parametrize("case", CG_CASES, ids=lambda c: "nx%d_ny%d_m%d_p%d" % c[:4])
def test_last_smoothing_step_and_cg_dots_match_oracle(smooth_emu, tmp_path, case):
    """The last level-0 step inside the flexible CG: z (FP64 output of the
    FP32 step with b = r), and from the last block beta = (r - r_old).z /
    rz_old, rz = r.z, rr = the sum of the first step's partials, the iteration
    count and the convergence flag (blocks with a partial last warp for p = 2, 4)."""
    from oracle import ipsmm
    from oracle.transport import Discretization
    nx, ny, m, p, seed = case
    mesh = W.structured_mesh(nx, ny, m=m, perturb_seed=seed)
    ne, n = mesh.n_elem, (p + 1) ** 2
    st = 1.0 + 0.5 * (np.arange(ne) % 3)
    ss = 0.7 * st
    rng = np.random.default_rng(47)
    r = rng.standard_normal(ne * n)
    rold = rng.standard_normal(ne * n)
    xin = rng.standard_normal(ne * n).astype(np.float32)
    xprev = rng.standard_normal(ne * n).astype(np.float32)
    epb = 256 // n
    grid = (ne + 2 * epb - 1) // (2 * epb)
    rr_parts = rng.uniform(0.5, 1.5, grid)
    rz_old, thresh = 2.5, float(rr_parts.sum()) * 1.001        # rr just below the threshold: converged
    for name, arr in (("nodes", mesh.nodes), ("sigma_t", st), ("sigma_s", ss), ("q", np.ones((ne, n))), ("b", r),
                      ("rold", rold), ("cg", np.concatenate([[rz_old, thresh], rr_parts]))):
        np.ascontiguousarray(arr, np.float64).tofile(tmp_path / f"{name}.f64")
    np.asarray(mesh.elem_nodes, np.int32).tofile(tmp_path / "elem.i32")
    xin.tofile(tmp_path / "xin.f32")
    xprev.tofile(tmp_path / "xprev.f32")
    c1, c2 = 0.375, 0.8125
    subprocess.run([smooth_emu, str(tmp_path), str(ne), str(len(mesh.nodes)), str(m), str(p), str(c1), str(c2), "2"],
                   check=True, timeout=600)
    z = np.fromfile(tmp_path / "z.f64")
    scal = np.fromfile(tmp_path / "scal.f64")
    ctl = np.fromfile(tmp_path / "ctl.i32", dtype=np.int32)
    disc = Discretization(mesh.nodes, mesh.elem_nodes, m, p, 4, st, ss)
    A = ipsmm.assemble_lhs(disc).toarray()
    Pinv = np.zeros_like(A)
    for e in range(ne):
        sl = slice(e * n, (e + 1) * n)
        Pinv[sl, sl] = np.linalg.inv(A[sl, sl])
    x0, xp = xin.astype(np.float64), xprev.astype(np.float64)
    ref = x0 + c2 * (Pinv @ (r - A @ x0)) + c1 * (x0 - xp)
    scale = np.max(np.abs(x0)) + c2 * np.max(np.abs(Pinv) @ (np.abs(r) + np.abs(A) @ np.abs(x0))) + \
        c1 * np.max(np.abs(x0) + np.abs(xp))
    assert np.max(np.abs(z - ref)) <= 1e-5 * scale
    # the dots of the kernel's own z, in FP64: every row counted once
    assert scal[0] == pytest.approx(float(r @ z), rel=1e-12, abs=1e-12 * float(np.abs(r) @ np.abs(z)))
    dz = float((r - rold) @ z)
    assert scal[6] * rz_old == pytest.approx(dz, rel=1e-12, abs=1e-12 * float(np.abs(r - rold) @ np.abs(z)))
    assert scal[2] == pytest.approx(float(rr_parts.sum()), rel=1e-14)
    assert ctl[1] == 6 and ctl[0] == 1 and ctl[3] == 0 and ctl[6] == 0


@pytest.mark.parametrize("case", CG_CASES, ids=lambda c: "nx%d_ny%d_m%d_p%d" % c[:4])
def test_first_smoothing_step_with_cg_update_matches_oracle(smooth_emu, tmp_path, case):
    """The first level-0 step inside the flexible CG: x += alpha p, r_old = r,
    r -= alpha q (FP64), xout = c2 A_d^{-1} r (FP32), and per-block partials of
    r.r that add up to the new r.r (blocks with a partial last warp for p = 2, 4)."""
    from oracle import ipsmm
    from oracle.transport import Discretization
    nx, ny, m, p, seed = case
    mesh = W.structured_mesh(nx, ny, m=m, perturb_seed=seed)
    ne, n = mesh.n_elem, (p + 1) ** 2
    st = 1.0 + 0.5 * (np.arange(ne) % 3)
    ss = 0.7 * st
    rng = np.random.default_rng(53)
    r, x, pv, q = (rng.standard_normal(ne * n) for _ in range(4))
    alpha = 0.7071
    for name, arr in (("nodes", mesh.nodes), ("sigma_t", st), ("sigma_s", ss), ("q", q), ("b", r), ("x", x),
                      ("p", pv), ("cg", np.array([alpha]))):
        np.ascontiguousarray(arr, np.float64).tofile(tmp_path / f"{name}.f64")
    np.asarray(mesh.elem_nodes, np.int32).tofile(tmp_path / "elem.i32")
    c2 = 0.8125
    subprocess.run([smooth_emu, str(tmp_path), str(ne), str(len(mesh.nodes)), str(m), str(p), "0", str(c2), "3"],
                   check=True, timeout=600)
    rn = r - alpha * q
    assert np.array_equal(np.fromfile(tmp_path / "x_out.f64"), x + alpha * pv)
    assert np.array_equal(np.fromfile(tmp_path / "r_out.f64"), rn)
    assert np.array_equal(np.fromfile(tmp_path / "rold_out.f64"), r)
    assert np.fromfile(tmp_path / "rr.f64").sum() == pytest.approx(float(rn @ rn), rel=1e-13)
    disc = Discretization(mesh.nodes, mesh.elem_nodes, m, p, 4, st, ss)
    A = ipsmm.assemble_lhs(disc).toarray()
    ref = np.concatenate([c2 * np.linalg.solve(A[e * n:(e + 1) * n, e * n:(e + 1) * n], rn[e * n:(e + 1) * n])
                          for e in range(ne)])
    got = np.fromfile(tmp_path / "xout.f32", dtype=np.float32).astype(np.float64)
    # FP32 block inverses and residual: rounding of a few parts in 1e7, amplified by the blocks' conditioning
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))


@pytest.mark.parametrize("case", CG_CASES, ids=lambda c: "nx%d_ny%d_m%d_p%d" % c[:4])
def test_level0_residual_corner_sums_match_oracle(smooth_emu, tmp_path, case):
    """The level-0 residual restricted to the element corners, w4^T (b - A x)
    per element, with the diagonal blocks entering as W = w4^T A_d (any
    weights w4 [n][4]; the library's are the bilinear ones)."""
    from oracle import ipsmm
    from oracle.transport import Discretization
    nx, ny, m, p, seed = case
    mesh = W.structured_mesh(nx, ny, m=m, perturb_seed=seed)
    ne, n = mesh.n_elem, (p + 1) ** 2
    st = 1.0 + 0.5 * (np.arange(ne) % 3)
    ss = 0.7 * st
    rng = np.random.default_rng(59)
    b = rng.standard_normal(ne * n)
    x = rng.standard_normal(ne * n).astype(np.float32)
    w4 = rng.uniform(0.0, 1.0, (n, 4))
    for name, arr in (("nodes", mesh.nodes), ("sigma_t", st), ("sigma_s", ss), ("q", np.ones((ne, n))), ("b", b),
                      ("w4", w4)):
        np.ascontiguousarray(arr, np.float64).tofile(tmp_path / f"{name}.f64")
    np.asarray(mesh.elem_nodes, np.int32).tofile(tmp_path / "elem.i32")
    x.tofile(tmp_path / "xin.f32")
    subprocess.run([smooth_emu, str(tmp_path), str(ne), str(len(mesh.nodes)), str(m), str(p), "0", "0", "4"],
                   check=True, timeout=600)
    got = np.fromfile(tmp_path / "cres.f32", dtype=np.float32).astype(np.float64).reshape(ne, 4)
    disc = Discretization(mesh.nodes, mesh.elem_nodes, m, p, 4, st, ss)
    A = ipsmm.assemble_lhs(disc).toarray()
    res = (b - A @ x.astype(np.float64)).reshape(ne, n)
    ref = res @ w4
    scale = np.max((np.abs(b) + np.abs(A) @ np.abs(x.astype(np.float64))).reshape(ne, n) @ w4)
    assert np.max(np.abs(got - ref)) <= 1e-5 * scale, np.max(np.abs(got - ref)) / scale
