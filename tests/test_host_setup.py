"""The C-ABI library on the CPU: it loads, exports every symbol include/imex.h
declares, and its host setup (partition, load vector, counts) agrees with the
oracle.  No GPU is used here."""
import os
import re

import numpy as np
import pytest

from oracle import basis, pipeline
from oracle.geometry import UNCUT, CUT, EMPTY
from paper_2310_14712_gb300 import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

imex = pytest.importorskip("paper_2310_14712_gb300.imex",
                           reason="libimex.so not built (python -m paper_2310_14712_gb300.build)")


def test_library_exports_every_declared_symbol():
    header = open(os.path.join(ROOT, "include", "imex.h")).read()
    declared = set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(imex_\w+)\s*\(", header, re.M))
    assert declared, "no declarations parsed"
    assert declared == set(imex.EXPORTS)
    for name in declared:
        assert hasattr(imex._lib, name), name


@pytest.mark.parametrize("p", range(1, 9))
def test_host_gll_and_gauss_match_oracle(p):
    x, w = imex.gll_points(p)
    xo, wo = basis.gll_points(p)
    assert np.allclose(x, xo, atol=2e-15, rtol=0) and np.allclose(w, wo, atol=2e-15, rtol=0)
    x, w = imex.gauss_points(p + 1)
    xo, wo = basis.gauss_points(p + 1)
    assert np.allclose(x, xo, atol=2e-15, rtol=0) and np.allclose(w, wo, atol=2e-15, rtol=0)


def _compare_partition(w):
    cls, fx, st = imex.host_setup_export(**w.kwargs())
    s = pipeline.setup(**w.kwargs())
    d = s.disc
    ocls = np.zeros(len(cls), dtype=np.uint8)
    ocls[d.is_d] = 1
    ocls[d.is_c] = 2
    assert np.array_equal(cls, ocls)                                  # index work: bit-exact
    assert st["n_d"] == d.is_d.sum() and st["n_c"] == d.is_c.sum()
    assert st["n_cut"] == (d.cell_type == CUT).sum()
    assert st["n_uncut"] == (d.cell_type == UNCUT).sum()
    assert st["n_empty"] == (d.cell_type == EMPTY).sum()
    assert st["dt"] == pytest.approx(s.dt, rel=1e-14)
    scale = np.abs(d.fx).max()
    assert np.abs(fx - d.fx).max() <= 1e-13 * scale
    return st


def test_host_setup_plate16_matches_oracle():
    st = _compare_partition(workloads.plate16())
    assert st["n_components"] >= 1 and st["nnz_L"] > 0


def test_host_setup_small_perforated_plate_matches_oracle():
    w = workloads.plate256()
    w.ncells = (32, 16)                      # same holes, coarse grid: fast on the CPU
    w.p = 3
    _compare_partition(w)


def test_host_setup_rejects_bad_arguments():
    w = workloads.plate16()
    kw = w.kwargs()
    kw["p"] = 0
    with pytest.raises(imex.ImexError) as e:
        imex.host_setup_export(**kw)
    assert e.value.code == -1
    kw = w.kwargs()
    kw["alpha"] = 0.0
    with pytest.raises(imex.ImexError):
        imex.host_setup_export(**kw)


def test_setup_statistics_log_line():
    # IMEX_LOG=1: one JSON line of setup statistics on stderr (a child process,
    # so that the variable is read by a fresh library).
    import json
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2310_14712_gb300 import imex, workloads\n"
            "imex.host_setup_export(**workloads.plate16().kwargs())\n") % ROOT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       env=dict(os.environ, IMEX_LOG="1"), timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [json.loads(l) for l in r.stderr.splitlines() if l.startswith('{"imex_setup"')]
    assert len(lines) == 1
    st = imex.host_setup_export(**workloads.plate16().kwargs())[2]
    rec = lines[0]
    assert rec["imex_setup"] == "host"
    for k in ("n_d", "n_c", "n_cut", "n_uncut", "n_empty", "nnz_L"):
        assert rec[k] == st[k], k
    assert rec["dt"] == st["dt"] and rec["factorized"] == 1


def test_host_setup_per_cell_wave_speed_matches_oracle():
    # The adjoint's workload: a wave speed per cell in [0.8, 1.2].  The time
    # step follows the fastest uncut cell, so it differs from the c0 rule.
    w = workloads.adjoint()
    st = _compare_partition(w)
    c_uncut = np.asarray(w.cell_c)[pipeline.setup(**w.kwargs()).disc.cell_type == UNCUT].max()
    assert c_uncut > 1.05 and st["dt"] < 0.95 * imex.host_setup_export(**{**w.kwargs(), "cell_c": None})[2]["dt"]


def _box3d(p):
    return workloads.Workload("box3d", 3, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (4, 4, 4), p, 1e-5, 2,
                              np.array([[0.5, 0.45, 0.55, 0.3, 0.25, 0.2]]), np.array([[0.2, 0.3, 0.3]]),
                              3.0, 0.08, 0)


@pytest.mark.parametrize("p", [2, 3])
def test_host_setup_3d_box_matches_oracle(p):
    st = _compare_partition(_box3d(p))
    assert st["n_cut"] > 0 and st["n_d"] > 0


@pytest.mark.parametrize("make", [workloads.plate16, lambda: _box3d(3)], ids=["plate16", "box3d_p3"])
def test_host_implicit_system_matches_oracle(make):
    # S = M^cc + beta dt^2 K^cc as the library factorises it (Fig.
    # TrapCDMIMEX) against the oracle's assembled M and K restricted to I_c,
    # entry by entry in the library's c-order; the two assemble the same
    # quadrature sums in different orders (roundoff, 1e-12 of the largest entry).
    import scipy.sparse as sp
    w = make()
    c_node, ptr, col, sv, mv = imex.host_implicit_system(**w.kwargs())
    s = pipeline.setup(**w.kwargs())
    d = s.disc
    assert np.array_equal(np.sort(c_node), np.flatnonzero(d.is_c))        # the c-set, any order
    n = len(c_node)
    S_lib = sp.csr_matrix((sv, col, ptr), shape=(n, n))
    M_lib = sp.csr_matrix((mv, col, ptr), shape=(n, n))
    M_ref = sp.csr_matrix(d.M)[c_node][:, c_node]
    S_ref = M_ref + 0.25 * s.dt * s.dt * sp.csr_matrix(d.K)[c_node][:, c_node]
    for lib, ref in ((S_lib, S_ref), (M_lib, M_ref)):
        scale = abs(ref).max()
        assert abs(lib - ref).max() <= 1e-12 * scale
    # the pattern: columns ascending in every row and symmetric
    assert all(np.all(np.diff(col[ptr[r]:ptr[r + 1]]) > 0) for r in range(n))
    assert abs(S_lib - S_lib.T).max() <= 1e-14 * abs(S_lib).max()
