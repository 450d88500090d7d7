"""The oracle's pins catch plausible mistakes.

Each case plants one mistake -- a dropped term, a wrong sign, factor or
index, a transposed operand, the wrong neighbour -- in a copy of `oracle/`
(only the copy; on the CPU) and runs the pins that must catch it in a
subprocess that imports the copy.  The planted copy must fail them; an
unmodified copy must pass, so a failure comes from the planted mistake.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

Q, FEM, TR, CL, IP, SMM, CNN, CG = ("quadrature.py", "fem.py", "transport.py", "closures.py", "ipsmm.py", "smm.py",
                                   "cnn.py", "cgsmm.py")
T_QUAD = ["tests/test_oracle_quadrature.py"]
T_FEM = ["tests/test_oracle_fem.py"]
T_SWEEP = ["tests/test_oracle_sweep.py"]
T_CLOS = ["tests/test_oracle_closures.py"]
T_IP = ["tests/test_oracle_ipsmm.py"]

# (id, file, planted from, planted to, pins)
MUTATIONS = [
    ("lq_weights_2pi", Q, "ww.append(2.0 * wi * (4.0 * math.pi / 8.0))", "ww.append(2.0 * wi * (2.0 * math.pi / 8.0))",
     T_QUAD),
    ("lq_cosine_step", Q, "step = 2.0 * (1.0 - 3.0 * mu1 * mu1) / (N - 2)",
     "step = 2.0 * (1.0 - 3.0 * mu1 * mu1) / (N - 1)", T_QUAD),
    ("lq_moment_condition", Q, "rhs[r] = 1.0 / (2 * k + 1)", "rhs[r] = 1.0 / (2 * k + 2)", T_QUAD),
    ("gll_weight", Q, "w = 2.0 / (n * (n - 1) * P(x) ** 2)", "w = 2.0 / (n * (n + 1) * P(x) ** 2)", T_QUAD),
    ("basis_gradient_direction", FEM, "G[:, i, 0] = Dx[:, ix] * Vy[:, iy]", "G[:, i, 0] = Vx[:, ix] * Dy[:, iy]", T_FEM),
    ("physical_gradient_transposed", FEM, '"qdc,qid->qic"', '"qcd,qid->qic"', T_FEM),
    ("mass_without_jacobian", FEM, 'return np.einsum("q,qi,qj->ij", wJ, self.V, self.V)',
     'return np.einsum("q,qi,qj->ij", self.w, self.V, self.V)', T_FEM),
    ("face_normals_flipped", FEM, "if f in (0, 1):", "if f in (0, 3):", T_FEM + T_SWEEP),
    ("streaming_sign", TR, "A = self.sigma_t[e] * self.M[e] - ox * self.Gx[e] - oy * self.Gy[e]",
     "A = self.sigma_t[e] * self.M[e] - ox * self.Gx[e] + oy * self.Gy[e]", T_SWEEP),
    ("outflow_term_min", TR, 'A = A + fd["V"].T @ (np.maximum(a, 0.0)[:, None] * fd["V"])',
     'A = A + fd["V"].T @ (np.minimum(a, 0.0)[:, None] * fd["V"])', T_SWEEP),
    ("upwind_trace_of_own_element", TR, "return self.Vnb[e][f] @ psi[nb[0]]", "return self.Vnb[e][f] @ psi[e]",
     T_SWEEP),
    ("scattering_over_2pi", TR, "return (self.sigma_s / (4.0 * math.pi))", "return (self.sigma_s / (2.0 * math.pi))",
     ["tests/test_oracle_smm.py::test_linear_fixed_point_on_curved_mesh",
      "tests/test_oracle_smm.py::test_iteration_converges_to_coupled_dense_solution"]),
    ("fixup_without_rescale", TR, "return (t / tp) * pos", "return pos", ["tests/test_oracle_fixup.py"]),
    ("lagged_inflow_not_lagged", TR, "up = self.upwind_values(e, f, d, psi_lag if (e, f) in lagset else psi, psibar)",
     "up = self.upwind_values(e, f, d, psi, psibar)",
     ["tests/test_oracle_block_jacobi.py", "tests/test_oracle_lagging.py"]),
    ("cycle_lagging_wrong_faces", TR, "lagged.update((v, f) for f in faces)", "lagged.update((u, f) for f in faces)",
     ["tests/test_oracle_lagging.py"]),
    ("tensor_trace_half", CL, "pxx - phi / 3.0, pxy", "pxx - phi / 2.0, pxy", T_CLOS),
    ("beta_sign", CL, 'out[b] = B[b] - eb0(disc, nhat) * (fd["V"] @ phi[e])',
     'out[b] = B[b] + eb0(disc, nhat) * (fd["V"] @ phi[e])', T_CLOS),
    ("partial_current_outgoing", CL, "np.where(on < 0.0, on, 0.0)", "np.where(on > 0.0, on, 0.0)", T_CLOS),
    ("eb0_over_2pi", CL, "@ disc.wq / (4.0 * math.pi)", "@ disc.wq / (2.0 * math.pi)", T_CLOS),
    ("ip_symmetry_term_dropped", IP, "Af = kappa * U.T @ (ds[:, None] * U) - U.T @ Gn - Gn.T @ U",
     "Af = kappa * U.T @ (ds[:, None] * U) - U.T @ Gn", T_IP),
    ("ip_absorption_sign", IP, "(st[e] - ss[e]) * disc.M[e], e * n, e * n)",
     "(st[e] + ss[e]) * disc.M[e], e * n, e * n)", T_IP),
    ("ip_rhs_tensor_jump_dropped", IP,
     'b[e * n:(e + 1) * n] += V1.T @ g + 0.5 * np.einsum("qic,qc->i", G1, tj) / st[e]',
     "b[e * n:(e + 1) * n] += V1.T @ g", T_IP),
    ("ip_div_T_index", IP, "dx = G[:, :, 0] @ txx + G[:, :, 1] @ txy", "dx = G[:, :, 0] @ txx + G[:, :, 0] @ txy",
     T_IP + ["tests/test_oracle_smm.py"]),
    ("ip_rhs_divT_average_sign", IP, "g = 0.5 * np.sum((v1 + v2) * nds, axis=1)",
     "g = 0.5 * np.sum((v1 - v2) * nds, axis=1)", T_IP),
    ("ip_rhs_tensor_jump_other_side", IP,
     'b[e2 * n:(e2 + 1) * n] += -V2.T @ g + 0.5 * np.einsum("qic,qc->i", G2, tj) / st[e2]',
     'b[e2 * n:(e2 + 1) * n] += -V2.T @ g - 0.5 * np.einsum("qic,qc->i", G2, tj) / st[e2]', T_IP),
    ("fixed_point_moment_slice", SMM, "T = closures.nodal_moments(self.disc, psi)[3:6]",
     "T = closures.nodal_moments(self.disc, psi)[2:5]",
     ["tests/test_oracle_smm.py::test_smm_approaches_sn_at_order_p_plus_1"]),
    ("ip_marshak_term_halved", IP, 'add(fd["V"].T @ ((E * ds)[:, None] * fd["V"]), e * n, e * n)',
     'add(fd["V"].T @ ((0.5 * ds)[:, None] * fd["V"]), e * n, e * n)', T_IP),
    ("boundary_sum_without_abs", CL, "a = np.abs(nhat @ disc.omega.T)", "a = nhat @ disc.omega.T", T_CLOS),
    ("gauss_legendre_weights", Q, "leggauss(n)\n    return 0.5 * (x + 1.0), 0.5 * w",
     "leggauss(n)\n    return 0.5 * (x + 1.0), w", T_QUAD),
    ("source_current_components_swapped", CL, 'np.einsum("d,den->en", disc.wq * disc.omega[:, 0], q)',
     'np.einsum("d,den->en", disc.wq * disc.omega[:, 1], q)', T_IP + ["tests/test_oracle_smm.py"]),
    ("cnn_upsampling_adjoint", CNN, ".sum(axis=(3, 5))", ".mean(axis=(3, 5))", ["tests/test_oracle_cnn.py"]),
    ("cnn_relu_mask", CNN, 'g5 = q(gu5 * (c["a5"] > 0))', 'g5 = q(gu5 * (c["a4"].mean() > 0))',
     ["tests/test_oracle_cnn.py"]),
    ("cg_rhs_wrong_element_sigma", CG, 'np.add.at(b, gid[e2], 0.5 * np.einsum("qic,qc->i", G2, tj) / st[e2])',
     'np.add.at(b, gid[e2], 0.5 * np.einsum("qic,qc->i", G2, tj) / st[e])', ["tests/test_oracle_cgsmm.py"]),
]


def run_pins(copy_root, tests):
    """Run the pins with the oracle imported from copy_root; returns (exit status, output)."""
    code = ("import sys; sys.path.insert(0, %r); sys.path.append(%r)\n"
            "import oracle\n"
            "assert oracle.__file__.startswith(%r), oracle.__file__\n"
            "import pytest\n"
            "args = ['-x', '-q', '-p', 'no:cacheprovider', '--import-mode=append', '-m', 'not gpu']\n"
            "sys.exit(pytest.main(args + %r))"
            % (str(copy_root), ROOT, str(copy_root), list(tests)))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout + r.stderr


def planted_copy(root, fname=None, old=None, new=None):
    dst = root / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), dst, ignore=shutil.ignore_patterns("__pycache__"))
    if fname is not None:
        path = dst / fname
        src = path.read_text()
        assert src.count(old) == 1, (fname, old)
        path.write_text(src.replace(old, new))
    return root


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    """Every case's (exit status, output), the subprocesses run concurrently;
    key None is the unmodified copy."""
    from concurrent.futures import ThreadPoolExecutor
    cases = [(None, None, None, None, T_QUAD + T_CLOS + T_SWEEP)] + MUTATIONS
    roots = [planted_copy(tmp_path_factory.mktemp("copy"), *c[1:4]) for c in cases]
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as pool:
        outs = list(pool.map(run_pins, roots, [c[4] for c in cases]))
    return {c[0]: o for c, o in zip(cases, outs)}


def test_unmodified_copy_passes(results):
    rc, out = results[None]
    assert rc == 0, out[-2000:]


@pytest.mark.parametrize("name", [m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(results, name):
    rc, out = results[name]
    # 1: some pin failed (not 0: all passed; not 2..5: the copy did not even load or collect)
    assert rc == 1, (name, rc, out[-2000:])
