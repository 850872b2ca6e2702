"""The CPU checks of the library's host setup catch plausible mistakes planted in it.

Each row plants one mistake in a copy of `csrc/setup.cpp` (the C++ host
setup: basis, spacetree quadrature, partition, time step, load vector,
implicit system, factorisation), compiles it, links it with the library's
other object files (as built by `paper_2310_14712_gb300/build.py`) into a
library in a temporary folder, and runs there, in its own Python process, the
host test it names, which must then fail.  The repository's library is not
touched.  A control run of every named test against the unchanged source
must pass first (it fails, for instance, when the object files are older
than `setup.h`: rebuild).  No GPU is used.

Not listed, because nothing the setup returns changes: a box test that
sends cells lying inside a hole to the spacetree (their fill ratio is zero,
so the fill-ratio rule drops them all the same).
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2310_14712_gb300")
OBJS = [os.path.join(PKG, "_build", "imex.o"), os.path.join(PKG, "_build", "probe.o")]

H = "tests/test_host_setup.py::"
E = "tests/test_host_element_matrices.py::"

# (text as written in setup.cpp, planted mistake, host test that must fail)
MISTAKES = [
    ("w[j] = 2.0 / (p * (p + 1.0) * pn * pn);", "w[j] = 2.0 / (p * (p - 1.0) * pn * pn);",
     H + "test_host_gll_and_gauss_match_oracle"),
    ("if (k != i) d *= (xn[i] - xn[k]);", "if (k != i) d *= (xn[k] - xn[i]);",
     H + "test_host_setup_3d_box_matches_oracle"),
    ("if (j != i && j != k) t *= (x - nodes[j]);", "if (j != i) t *= (x - nodes[j]);",
     E + "test_plate16_cut_and_uncut_cells"),
    ("if (s <= 1.0) return false;", "if (s <= 0.9) return false;", E + "test_plate16_cut_and_uncut_cells"),
    ("double nearest = (l > 0.0) ? l : ((u < 0.0) ? u : 0.0);", "double nearest = (l > 0.0) ? l : 0.0;",
     E + "test_3d_box_with_a_void"),
    ("if (dmin < 1.0) cut = true;", "if (dmin < 0.81) cut = true;", H + "test_host_setup_plate16_matches_oracle"),
    ("if (level < depth && geo.classify(plo, phi) == CELL_CUT)",
     "if (level <= depth && geo.classify(plo, phi) == CELL_CUT)", E + "test_plate16_cut_and_uncut_cells"),
    ("          double w = vol;\n", "          double w = 1.0;\n", E + "test_plate16_cut_and_uncut_cells"),
    ("for (int d = 0; d < dim; ++d) xp[d] = clo[d] + (pt.xr[d] + 1.0) * 0.5 * g.h[d];",
     "for (int d = 0; d < dim; ++d) xp[d] = clo[d] + (pt.xr[d] + 1.0) * g.h[d];", E + "test_plate16_cut_and_uncut_cells"),
    ("const double al = q.phys ? 1.0 : pb.alpha;", "const double al = q.phys ? pb.alpha : 1.0;",
     E + "test_plate16_cut_and_uncut_cells"),
    ("kwB[j] = wq * pb.rho * c * c;", "kwB[j] = wq * pb.rho * c;", E + "test_per_cell_wave_speed"),
    ("double t = jac * (2.0 / g.h[gd]) * (2.0 / g.h[gd]);", "double t = jac * (2.0 / g.h[gd]);",
     E + "test_plate16_cut_and_uncut_cells"),
    ("for (int d = 0; d < dim; ++d) { m *= hs.gll_w[r % P]; r /= P; }",
     "for (int d = 0; d < dim; ++d) { m *= hs.gll_w[(r + 1) % P]; r /= P; }", E + "test_plate16_cut_and_uncut_cells"),
    ("if (cut_fill[k] < kEmptyFill) {", "if (cut_fill[k] < 1e-2) {",
     H + "test_host_setup_small_perforated_plate_matches_oracle"),
    ("else if (nc == NODE_INACTIVE) nc = NODE_D;", "else nc = NODE_D;", H + "test_host_setup_plate16_matches_oracle"),
    ("hs.dt_crit_uncut = 2.0 / std::sqrt(lam);", "hs.dt_crit_uncut = 1.0 / std::sqrt(lam);",
     H + "test_host_setup_plate16_matches_oracle"),
    ("if (hs.cell_type[cid] == CELL_UNCUT) cmax = std::max(cmax, cell_speed(cid));",
     "if (hs.cell_type[cid] == CELL_UNCUT) cmax = pb.c0;", H + "test_host_setup_per_cell_wave_speed_matches_oracle"),
    ("double fv = source_value(pb, xp, col) * Wt[q] * jac;", "double fv = source_value(pb, xp, col) * Wt[q];",
     H + "test_host_setup_plate16_matches_oracle"),
    ("for (int d = 0; d < dim; ++d) xp[d] = g.lo[d] + ci[d] * g.h[d] + (Xr[q * 3 + d] + 1.0) * 0.5 * g.h[d];",
     "for (int d = 0; d < dim; ++d) xp[d] = g.lo[d] + ci[d] * g.h[d] + (Xr[q * 3 + d] + 1.0) * g.h[d];",
     H + "test_host_setup_plate16_matches_oracle"),
    ("fe[(size_t)col * Pd + bcol] += wq * fv[col] * N[bcol];", "fe[(size_t)col * Pd + bcol] += q.w * fv[col] * N[bcol];",
     H + "test_host_setup_plate16_matches_oracle"),
    ("constexpr double kBeta = 0.25;", "constexpr double kBeta = 0.5;", H + "test_host_implicit_system_matches_oracle"),
    ("es.emplace_back(key, mv + bdt2 * kv);", "es.emplace_back(key, mv + kv);",
     H + "test_host_implicit_system_matches_oracle"),
    ("            s0 -= x * C0[q];", "            s0 += x * C0[q];", H + "test_host_setup_plate16_matches_oracle"),
    ("      for (int q = j0; q < j; ++q) d -= Rj[q] * Rj[q];", "      for (int q = j0; q < j; ++q) d -= Rj[q];",
     H + "test_host_setup_plate16_matches_oracle"),
]


def _tools():
    from paper_2310_14712_gb300 import build
    nvcc = build._nvcc()
    if shutil.which("g++") is None or shutil.which(nvcc) is None or not all(map(os.path.exists, OBJS)):
        pytest.skip("needs g++, nvcc and the library's object files (python -m paper_2310_14712_gb300.build)")
    return nvcc, build.ARCH


def _prepare(base):
    ignore = shutil.ignore_patterns("__pycache__", "*.pyc")
    for d in ("oracle", "tests", "include"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(base, d), ignore=ignore)
    pkg = os.path.join(base, "paper_2310_14712_gb300")
    os.makedirs(pkg)
    for name in os.listdir(PKG):
        if name.endswith(".py"):
            shutil.copy(os.path.join(PKG, name), pkg)


def _run(nvcc, arch, src, tests):
    """Build a library from `src` (setup.cpp's text) in a fresh folder and run `tests` there."""
    base = tempfile.mkdtemp(prefix="host_mistake_")
    try:
        _prepare(base)
        cpp = os.path.join(base, "setup.cpp")
        with open(cpp, "w") as f:
            f.write(src)
        obj = os.path.join(base, "setup.o")
        lib = os.path.join(base, "paper_2310_14712_gb300", "libimex.so")
        for cmd in (["g++", "-O1", "-std=c++17", "-fPIC", "-pthread", "-I", os.path.join(PKG, "csrc"), "-c", cpp,
                     "-o", obj],
                    [nvcc, *arch, "-shared", *OBJS, obj, "-o", lib, "-lpthread"]):
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
            if r.returncode != 0:
                return None, r.stdout + r.stderr
        env = {k: v for k, v in os.environ.items() if k != "PYTHONPATH"}
        env["PYTHONDONTWRITEBYTECODE"] = "1"
        r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", *tests],
                           cwd=base, env=env, capture_output=True, text=True, timeout=600)
        return r.returncode, r.stdout + r.stderr
    finally:
        shutil.rmtree(base, ignore_errors=True)


def test_every_planted_host_mistake_fails_its_check():
    nvcc, arch = _tools()
    with open(os.path.join(PKG, "csrc", "setup.cpp")) as f:
        src = f.read()
    rc, out = _run(nvcc, arch, src, sorted({m[2] for m in MISTAKES}))
    assert rc == 0, "the host checks fail on the unchanged setup:\n" + out[-2000:]

    def planted(k):
        before, after, test = MISTAKES[k]
        if src.count(before) != 1:
            return k, None, f"the text to change occurs {src.count(before)} times"
        return (k, *_run(nvcc, arch, src.replace(before, after), [test]))

    missed = []
    with cf.ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1))) as ex:
        for k, rc, out in ex.map(planted, range(len(MISTAKES))):
            if rc != 1 or "failed" not in out.splitlines()[-1]:
                missed.append(f"{MISTAKES[k][1]!r} -> {MISTAKES[k][2]} (exit {rc})\n{out[-600:]}")
    assert not missed, "planted host mistakes that no check caught:\n" + "\n".join(missed)


def test_host_mistake_table_names_existing_checks():
    with open(os.path.join(PKG, "csrc", "setup.cpp")) as f:
        src = f.read()
    for before, after, test in MISTAKES:
        path, name = test.split("::")
        with open(os.path.join(ROOT, path)) as f:
            assert f"def {name}(" in f.read(), test
        assert src.count(before) == 1, before
        assert before != after
