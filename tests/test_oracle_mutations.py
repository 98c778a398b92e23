"""Mutation check of the oracle's pins (CPU only).

Each case plants one plausible mistake in a private copy of the oracle package (a
dropped term or weight, a wrong sign, index or sub-step, a transposed operand) and
runs, against that copy, the pin tests that should notice it.  The case passes when
those pins fail, i.e. when pytest exits with status 1 (failed tests; a copy that no
longer imports would exit 2 and does not count).  The unmodified copy must pass the
same pins first.  Mistakes are planted in the copy only: the oracle the rest of the
suite imports is never touched.

The copies run as separate pytest processes, several at a time.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
THIS = os.path.basename(__file__)

Q, G, T, MO, S, R = ("quadrature.py", "dg.py", "transport.py", "models.py", "scheme.py", "source.py")

# (id, oracle file, text, replacement, pin files), the text occurring once in the file
MUTATIONS = [
    # Gauss-Lobatto rule and Lagrange basis (Section 3.1, eq. (3.3) and (3.4))
    ("gl_weight_square_dropped", Q, "w = 2.0 / (d * (d + 1) * pd * pd)", "w = 2.0 / (d * (d + 1) * pd)",
     ["test_oracle_quadrature.py"]),
    ("gl_inner_nodes_of_lower_polynomial", Q, "_leg.legroots(_leg.legder(c))", "_leg.legroots(c[1:])",
     ["test_oracle_quadrature.py"]),
    ("derivative_matrix_transposed", Q, "D[j, i] = s", "D[i, j] = s", ["test_oracle_quadrature.py"]),
    ("derivative_product_wrong_index", Q, "p *= (x[j] - x[m]) / (x[i] - x[m])",
     "p *= (x[j] - x[m]) / (x[k] - x[m])", ["test_oracle_quadrature.py"]),
    # DG transport matrix, eq. (3.7)
    ("dg_downwind_flux", G, "vp, vm = max(vn, 0.0), min(vn, 0.0)", "vm, vp = max(vn, 0.0), min(vn, 0.0)",
     ["test_oracle_dg.py"]),
    ("dg_normal_sign_dropped", G, "vn = s * v[a] * cof[a]", "vn = v[a] * cof[a]", ["test_oracle_dg.py"]),
    ("dg_neighbour_point_wrong_end", G, "ip[a] = 0 if s > 0 else n - 1", "ip[a] = n - 1 if s > 0 else 0",
     ["test_oracle_dg.py"]),
    ("dg_volume_gradient_transposed", G, "grad[a] = Dm[j[a], i[a]] if others else 0.0",
     "grad[a] = Dm[i[a], j[a]] if others else 0.0", ["test_oracle_dg.py"]),
    ("dg_volume_weight_dropped", G, "coef * omega_j / omega_Li", "coef / omega_Li", ["test_oracle_dg.py"]),
    ("dg_face_weight_dropped", G, "mu = float(np.prod([w1[i[b]] for b in range(D) if b != a]))", "mu = 1.0",
     ["test_oracle_dg.py"]),
    ("dg_cofactor_inverted", G, "cof = np.array([det * 2.0 / mesh.h[a] for a in range(D)])",
     "cof = np.array([det * mesh.h[a] / 2.0 for a in range(D)])", ["test_oracle_dg.py"]),
    ("dg_volume_couples_all_nodes", G, "others = all(i[b] == j[b] for b in range(D) if b != a)", "others = True",
     ["test_oracle_dg.py"]),
    ("dg_inflow_cell_test_off_by_one", G, "inside = (cells[a] + s >= 0) & (cells[a] + s < mesh.N[a])",
     "inside = (cells[a] + s >= 0) & (cells[a] + s <= mesh.N[a])", ["test_oracle_boundary.py"]),
    # theta transport step, eq. (3.11), and its Fourier forms
    ("theta_weights_swapped", T, "self.A = (I - theta * delta * L).tocsc()",
     "self.A = (I - (1.0 - theta) * delta * L).tocsc()", ["test_oracle_transport.py"]),
    ("inflow_term_sign", T, "rhs = rhs + self.delta * (self.bcoef", "rhs = rhs - self.delta * (self.bcoef",
     ["test_oracle_boundary.py"]),
    ("line_lifting_at_wrong_end", T, "K[0, 0] += 1.0 / w[0]", "K[-1, -1] += 1.0 / w[0]",
     ["test_oracle_transport.py"]),
    ("line_mode_phase_sign", T, "Kk = K[None, :, :] - np.exp(-1j * kappa)", "Kk = K[None, :, :] - np.exp(1j * kappa)",
     ["test_oracle_transport.py"]),
    ("plane_kronecker_transposed", T, "nuy * np.kron(Ky[jy], I)[None])", "nuy * np.kron(I, Ky[jy])[None])",
     ["test_oracle_d2q9.py"]),
    ("planes_wrong_numpy_axis", T, "npc = 2 - c ", "npc = c ", ["test_oracle_d3q19.py"]),
    ("box_kronecker_y_on_z", T, "np.kron(np.kron(I, Ky[i]), I)", "np.kron(np.kron(Ky[i], I), I)",
     ["test_oracle_d3q27.py"]),
    ("explicit_half_weight", T, "self.B = (I + (1.0 - theta) * delta * L).tocsr()",
     "self.B = (I + theta * delta * L).tocsr()", ["test_oracle_transport.py"]),
    ("line_mirror_missing_on_input", T, "    if sign < 0:\n        f = f[..., ::-1]\n", "",
     ["test_oracle_transport.py"]),
    ("line_explicit_part_theta", T, "Bm = I - (1.0 - theta) * nu * Kk", "Bm = I - theta * nu * Kk",
     ["test_oracle_transport.py"]),
    ("plane_mode_phase_sign", T, "Kx = K[None] - np.exp(-1j * kx)", "Kx = K[None] - np.exp(1j * kx)",
     ["test_oracle_d2q9.py"]),
    ("box_courant_of_wrong_axis", T, "nu = [2.0 * abs(v[a]) * delta / h[a] for a in range(3)]",
     "nu = [2.0 * abs(v[a]) * delta / h[0] for a in range(3)]", ["test_oracle_d3q27.py"]),
    # kinetic models (Section 2)
    ("dnq2n_equilibrium_lambda_square_dropped", MO, "vq / (2.0 * self.lam ** 2)", "vq / (2.0 * self.lam)",
     ["test_oracle_models.py"]),
    ("shallow_water_pressure_half_dropped", MO, "p = 0.5 * self.gravity * h * h", "p = self.gravity * h * h",
     ["test_oracle_models.py"]),
    ("euler_energy_flux_pressure_dropped", MO, "comps.append((E + p) * u[a])", "comps.append(E * u[a])",
     ["test_oracle_models.py"]),
    ("lattice_equilibrium_quadratic_term", MO, "uv * uv / (2.0 * c2 * c2)", "uv * uv / (2.0 * c2)",
     ["test_oracle_d2q9.py"]),
    ("lattice_momentum_wrong_component", MO, "np.tensordot(V[:, a], g, axes=(0, 0))",
     "np.tensordot(V[:, 0], g, axes=(0, 0))", ["test_oracle_d2q9.py"]),
    ("d3q27_corner_weight", MO, "[1 / 54] * 12 + [1 / 216] * 8", "[1 / 54] * 12 + [1 / 108] * 8",
     ["test_oracle_d3q27.py"]),
    ("d3q15_axis_weight", MO, "[2 / 9] + [1 / 9] * 6 + [1 / 72] * 8", "[2 / 9] + [1 / 18] * 6 + [1 / 72] * 8",
     ["test_oracle_d3q27.py"]),
    ("lattice_equilibrium_kinetic_term_dropped", MO, " - uu / (2.0 * c2))", ")", ["test_oracle_d2q9.py"]),
    ("d3q19_edge_weight", MO, "[1 / 3] + [1 / 18] * 6 + [1 / 36] * 12", "[1 / 3] + [1 / 36] * 6 + [1 / 18] * 12",
     ["test_oracle_d3q19.py"]),
    ("lattice_sound_speed", MO, "return self.lam / np.sqrt(3.0)", "return self.lam / 3.0", ["test_oracle_d2q9.py"]),
    # collision and palindromic compositions (Section 3.2, Section 5.1)
    ("collision_weights_swapped", S, "return omega * model.feq(w) + (1.0 - omega) * f",
     "return (1.0 - omega) * model.feq(w) + omega * f", ["test_oracle_scheme.py"]),
    ("m2_full_first_substep", S, "f = transporter(f, 0.5 * dt)\n    f = source_collision",
     "f = transporter(f, dt)\n    f = source_collision", ["test_oracle_scheme.py"]),
    ("collapsed_last_half_step", S, "f = transporter(f, dt if s < nsteps - 1 else 0.5 * dt)",
     "f = transporter(f, dt)", ["test_oracle_scheme.py"]),
    ("m2kin_middle_substep", S, "f = transporter(f, 0.5 * dt)\n    f = collision(f, model, omega)\n    return",
     "f = transporter(f, 0.25 * dt)\n    f = collision(f, model, omega)\n    return", ["test_oracle_scheme.py"]),
    ("triple_jump_coefficient_sign", S, "g1 = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))",
     "g1 = 1.0 / (2.0 + 2.0 ** (1.0 / 3.0))", ["test_oracle_scheme.py"]),
    ("triple_jump_not_palindromic", S, "for g in (g1, g2, g1):", "for g in (g1, g1, g2):",
     ["test_oracle_scheme.py"]),
    ("m2kin_first_substep", S, "f = transporter(f, 0.25 * dt)\n    f = collision", "f = transporter(f, 0.5 * dt)\n    f = collision",
     ["test_oracle_scheme.py"]),
    ("m2kin_one_collision", S, "f = collision(f, model, omega)\n    f = transporter(f, 0.5 * dt)",
     "f = transporter(f, 0.5 * dt)", ["test_oracle_scheme.py"]),
    # source step (Section 3.2, Section 5.1, Section 5.2)
    ("penalisation_sign", R, "A[k, k] = -K", "A[k, k] = K", ["test_oracle_source.py"]),
    ("gravity_wrong_component", R, "A[2, 0] += self.g[1]", "A[2, 0] += self.g[0]", ["test_oracle_source.py"]),
    ("source_theta_dropped", R, "lhs = I - th * delta * Am", "lhs = I - delta * Am", ["test_oracle_source.py"]),
    ("source_equilibrium_part_not_replaced", R, "return f + model.feq(wn) - model.feq(w)",
     "return f + model.feq(wn) - model.feq(wn)", ["test_oracle_source.py"]),
    ("penalisation_profile_sign", R, "np.exp(-self.kappa", "np.exp(self.kappa", ["test_oracle_source.py"]),
    ("source_half_steps_asymmetric", S, "return source_step(f, model, transporter.mesh, source, 0.5 * dt)",
     "return source_step(f, model, transporter.mesh, source, dt)", ["test_oracle_source.py"]),
]

PIN_FILES = sorted({f for m in MUTATIONS for f in m[4]})


def _copy(dst):
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(dst, "tests"),
                    ignore=shutil.ignore_patterns("__pycache__", THIS, "test_gpu_*", "test_abi_*",
                                                  "test_multirank_*", "test_zz_*"))


def _pytest(dst, files):
    # the seeded input generators (which hold none of the method's arithmetic) come from
    # the repository; the oracle and the pins from the copy, which is first on the path
    path = os.pathsep.join([dst, ROOT] + [p for p in os.environ.get("PYTHONPATH", "").split(os.pathsep) if p])
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1", PYTHONPATH=path)
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]
    cmd += [os.path.join("tests", f) for f in files]
    r = subprocess.run(cmd, cwd=dst, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, (r.stdout + r.stderr)[-1500:]


def _run(base, case):
    name, fname, old, new, files = case
    dst = os.path.join(base, name)
    _copy(dst)
    path = os.path.join(dst, "oracle", fname)
    with open(path) as fh:
        src = fh.read()
    count = src.count(old)
    if count != 1:
        return name, ("text", count)
    with open(path, "w") as fh:
        fh.write(src.replace(old, new))
    return name, _pytest(dst, files)


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    base = str(tmp_path_factory.mktemp("oracle_mutants"))
    clean = os.path.join(base, "_unmodified")
    _copy(clean)
    jobs = MUTATIONS
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        unmodified = ex.submit(_pytest, clean, PIN_FILES)
        res = dict(ex.map(lambda c: _run(base, c), jobs))
    return unmodified.result(), res


def test_unmodified_copy_passes_the_pins(outcomes):
    rc, tail = outcomes[0]
    assert rc == 0, tail


@pytest.mark.parametrize("case", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(outcomes, case):
    out = outcomes[1][case[0]]
    assert out[0] != "text", f"the text to mutate occurs {out[1]} times in oracle/{case[1]}"
    rc, tail = out
    assert rc == 1, f"planted mistake not caught (pytest exit {rc}):\n{tail}"
