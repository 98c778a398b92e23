"""Mutation check of the CPU tests of the library's host logic (no GPU).

Two parts of the library run on the host and are checked through the C ABI without a GPU:
the planner (csrc/pdg_plan.cpp: Gauss-Lobatto rule, derivative matrix, per-cell line
coefficients, windows, the tile and box cell inverses and their truncation widths), checked
by `tests/test_abi_host.py` and `tests/test_sweep_algorithms.py`, and the pass schedule of
the palindromic compositions (csrc/pdg_schedule.cu), checked by `tests/test_schedule_host.py`.
Each case plants one plausible mistake in a copy of one source file, compiles that copy,
links it with the library's other objects into a private library, and runs the checking
test files against it; the case passes when they fail (pytest exit 1).  The unmodified
sources, linked the same way, must pass them first.  Nothing of the repository's own
library or sources is modified.

The line plan (coefficients, ratio (1-theta)/theta, windows, composed-step coupling) is
visible through pdg_plan_line and the tile / box plans through pdg_plan_sweep.  What only
the kernels see (the squared matrix E^2 of the composed step, the float-pair splits) is
covered by the GPU parity tests instead, and is not planted here.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_1702_00169_gb300"
PLAN, API = "pdg_plan.cpp", "pdg_schedule.cu"
PINS = {PLAN: ["test_abi_host.py", "test_sweep_algorithms.py"], API: ["test_schedule_host.py"]}

# (id, text, replacement[, file]), the text occurring once in the file (default pdg_plan.cpp)
MUTATIONS = [
    ("legendre_recurrence_denominator", "(j - 1.0) * p0) / j;", "(j - 1.0) * p0) / (j + 1.0);"),
    ("gl_weight_square_dropped", "w[j] = 2.0 / (d * (d + 1.0) * p * p);", "w[j] = 2.0 / (d * (d + 1.0) * p);"),
    ("gl_nodes_reversed", "x[j] = -s; x[d - j] = s;", "x[j] = s; x[d - j] = -s;"),
    ("derivative_matrix_transposed", "Dm[j * n + i] = v;", "Dm[i * n + j] = v;"),
    ("line_lifting_at_wrong_end", "K[0] += 1.0 / w[0];\n  // A = B", "K[n * n - 1] += 1.0 / w[0];\n  // A = B"),
    ("line_explicit_weight", "R[r * k + j] = id - (1.0 - theta) * nu * K[r * n + j];",
     "R[r * k + j] = id - theta * nu * K[r * n + j];"),
    ("line_inflow_theta_dropped", "R[r * k + n] = (r == 0) ? theta * nu / w[0] : 0.0;",
     "R[r * k + n] = (r == 0) ? nu / w[0] : 0.0;"),
    ("tile_courant_numbers_swapped", "if (iy == jy) k2 += nux * K[ix * n + jx];",
     "if (iy == jy) k2 += nuy * K[ix * n + jx];"),
    ("box_z_courant_number", "if (iy == jy && ix == jx) k3 += nuz * K[iz * n + jz];",
     "if (iy == jy && ix == jx) k3 += nuy * K[iz * n + jz];"),
    ("tile_width_tolerance", "const double tol = std::ldexp(1.0, -57);\n  for (int W = 1; W <= 128",
     "const double tol = std::ldexp(1.0, -27);\n  for (int W = 1; W <= 128"),
    ("box_width_tolerance", "const double tol = std::ldexp(1.0, -57);\n  // acc",
     "const double tol = std::ldexp(1.0, -27);\n  // acc"),
    ("box_width_cubic_shortcut_always", "const bool cubic = nux == nuy && nuy == nuz;", "const bool cubic = true;"),
    ("tile_width_edge_roles", "const double* X = edge == 0 ? A : B;", "const double* X = A;"),
    ("line_ratio_inverted", "c->zb = (1.0 - theta) / theta;", "c->zb = theta / (1.0 - theta);"),
    ("line_window_tolerance", "std::ceil(-60.0 * std::log(2.0) / std::log(a))",
     "std::ceil(-30.0 * std::log(2.0) / std::log(a))"),
    ("composed_coupling_term_dropped", "c->gamma1 = c->Eq[n - 1] * c->za + c->q[n - 1] * c->zb;",
     "c->gamma1 = c->Eq[n - 1] * c->za;"),
    ("composed_window_ignores_coupling", "if (bK <= tol && (double)K * g * bk <= tol) return K;",
     "if (bK <= tol) return K;"),
    # pass schedule of the compositions (Section 3.2, Section 5.1)
    ("m2_next_leading_half_step_dropped", "if (a != L) put(spec(a, 2, o2, z2, &half[a], 1));",
     "if (a != L) put(spec(a, 1, o2, z2, &half[a], 1));", API),
    ("m2_collision_dropped_from_last_axis_pass", "put(spec(L, 3, ottc, z3, &half[L], 1));",
     "put(spec(L, 2, ottc, z3, &half[L], 1));", API),
    ("collapsed_interior_step_half", "const int ops[2] = {T, C}, ci[2] = {s == 0 ? 0 : 1, 0};",
     "const int ops[2] = {T, C}, ci[2] = {0, 0};", API),
    ("m2kin_segment_coefficients_swapped", "auto seg_ci = [&](long long j) { return (j % 2 == 1) ? 1 : 0; };",
     "auto seg_ci = [&](long long j) { return (j % 2 == 0) ? 1 : 0; };", API),
    ("m2kin_first_pass_trailing_quarter", "ci[3] = {seg_ci(0), 0, seg_ci(1)};", "ci[3] = {seg_ci(0), 0, seg_ci(0)};", API),
    ("m4kin_not_palindromic", "for (double g : {g1, g2, g1}) {", "for (double g : {g1, g1, g2}) {", API),
    ("diagonal_collapsed_interior_half", "dl[0] = end ? h : dt;", "dl[0] = h;", API),
    ("diagonal_home_copy_condition", "if (slot != Lat.diag) {", "if (slot == Lat.diag) {", API),
    ("source_substep_full", "sp.sdelta = c->src.flags ? 0.5 * dt : 0.0;", "sp.sdelta = c->src.flags ? dt : 0.0;", API),
]


def _objects(B, skip=None):
    objs = [os.path.join(B.OBJDIR, f) for f in sorted(os.listdir(B.OBJDIR)) if f.endswith(".o")]
    return [o for o in objs if os.path.basename(o) != skip]


def _prepare(dst):
    for sub in ("oracle", "include"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(dst, sub), ignore=shutil.ignore_patterns("__pycache__"))
    os.makedirs(os.path.join(dst, PKG, "lib"))
    for f in ("__init__.py", "pdg.py", "build.py", "workloads.py"):
        shutil.copy(os.path.join(ROOT, PKG, f), os.path.join(dst, PKG, f))
    shutil.copytree(os.path.join(ROOT, PKG, "csrc"), os.path.join(dst, PKG, "csrc"))   # read by source checks
    os.makedirs(os.path.join(dst, "tests"))
    for f in ["conftest.py", "golden_util.py"] + sorted({p for v in PINS.values() for p in v}):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))


def _build_and_test(B, dst, fname, src_text):
    src = os.path.join(dst, fname)
    with open(src, "w") as fh:
        fh.write(src_text)
    stem = os.path.splitext(fname)[0]
    obj = os.path.join(dst, stem + ".o")
    inc = ["-I", B.CSRC]                              # the headers beside the original
    if fname.endswith(".cpp"):
        cmd = [B.nvcc()] + B.COMMON + inc + ["-x", "c++", "-c", src, "-o", obj]
    else:
        cmd = [B.nvcc()] + B.ARCH + B.COMMON + inc + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        return "compile", r.stderr[-1500:]
    lib = os.path.join(dst, PKG, "lib", "libpdg.so")
    r = subprocess.run([B.nvcc()] + B.ARCH + ["-shared", "-o", lib] + _objects(B, stem + ".o") + [obj] +
                       ["-lcudart_static", "-lrt", "-lpthread", "-ldl"], capture_output=True, text=True)
    if r.returncode != 0:
        return "link", r.stderr[-1500:]
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1", PYTHONPATH=dst)
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]
    cmd += [os.path.join("tests", f) for f in PINS[fname]]
    r = subprocess.run(cmd, cwd=dst, env=env, capture_output=True, text=True, timeout=900)
    shutil.rmtree(os.path.join(dst, PKG, "lib"))      # about 55 MB each
    return r.returncode, (r.stdout + r.stderr)[-1500:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    from paper_1702_00169_gb300 import build as B
    if not os.path.exists(B.LIB) or not os.path.isdir(B.OBJDIR) or len(_objects(B)) < 10:
        B.build()
    original = {}
    for f in PINS:
        with open(os.path.join(B.CSRC, f)) as fh:
            original[f] = fh.read()
    base = str(tmp_path_factory.mktemp("host_mutants"))

    def job(case):
        name, old, new = case[:3]
        fname = case[3] if len(case) > 3 else PLAN
        dst = os.path.join(base, name)
        _prepare(dst)
        if name.startswith("_unmodified"):
            return name, _build_and_test(B, dst, fname, original[fname])
        count = original[fname].count(old)
        if count != 1:
            return name, ("text", count)
        return name, _build_and_test(B, dst, fname, original[fname].replace(old, new))

    cases = [("_unmodified_plan", "", "", PLAN), ("_unmodified_api", "", "", API)] + MUTATIONS
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        return dict(ex.map(job, cases))


@pytest.mark.parametrize("name", ["_unmodified_plan", "_unmodified_api"])
def test_unmodified_sources_pass(outcomes, name):
    rc, tail = outcomes[name]
    assert rc == 0, tail


@pytest.mark.parametrize("case", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_host_mistake_is_caught(outcomes, case):
    rc, tail = outcomes[case[0]]
    assert rc != "text", f"the text to mutate occurs {tail} times in {case[3] if len(case) > 3 else PLAN}"
    assert rc == 1, f"planted mistake not caught ({rc}):\n{tail}"
