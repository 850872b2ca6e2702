"""Independent source columns (imex_setup_batch) against the oracle.

Column k of a batched context must be the whole method run with source k
alone: checked against the oracle column by column (same gates as the
single-source parity tests), and bit for bit against a single-column
context on the same source (the kernels take the same path for every
column), and under a permutation of the sources.
"""
import numpy as np
import pytest

from oracle import pipeline
from paper_2310_14712_gb300 import workloads

from parity_util import check_state

pytestmark = pytest.mark.gpu


def _imex():
    from paper_2310_14712_gb300 import imex
    return imex


def _state(g):
    n = g.n_nodes
    return {k: g.fields(k, out=np.zeros(g.field_len)).reshape(g.ncols, n)
            for k in ("u", "u_prev_d", "v_c", "a_c")}


def _run_batch(w, nsteps):
    imex = _imex()
    with imex.Imex.from_workload(w, ncols=len(w.src_pos)) as g:
        g.step(nsteps)
        st = _state(g)
        info = g.info()
    assert info["ncols"] == len(w.src_pos) and info["step"] == nsteps
    return st


def _col(st, k):
    return {name: v[k] for name, v in st.items()}


@pytest.mark.parametrize("ncols", [3, 8])
def test_batched_columns_match_oracle(ncols):
    w = workloads.multisource(nsrc=ncols)
    nsteps = 200
    st = _run_batch(w, nsteps)
    kw = w.kwargs()
    pos = kw.pop("src_pos")
    for k, s in enumerate(pipeline.setup_columns(pos, **kw)):
        ref = s.imex.run(nsteps)
        check_state(s, ref, _col(st, k), w.holes, w.alpha, nsteps)


def test_batched_column_equals_single_source_context():
    w = workloads.multisource(nsrc=5)
    nsteps = 60
    st = _run_batch(w, nsteps)
    imex = _imex()
    for k in (0, 4):
        w1 = workloads.multisource(nsrc=5)
        w1.src_pos = w.src_pos[k:k + 1]
        with imex.Imex.from_workload(w1) as g:
            g.step(nsteps)
            one = {n: g.fields(n, out=np.zeros(g.n_nodes)) for n in ("u", "u_prev_d", "v_c", "a_c")}
        for name in one:
            assert np.array_equal(st[name][k], one[name]), (k, name)


def test_batched_permuted_sources_permute_columns():
    w = workloads.multisource(nsrc=6)
    nsteps = 40
    st = _run_batch(w, nsteps)
    perm = np.array([3, 0, 5, 1, 4, 2])
    w2 = workloads.multisource(nsrc=6)
    w2.src_pos = w.src_pos[perm]
    st2 = _run_batch(w2, nsteps)
    for name in st:
        assert np.array_equal(st2[name], st[name][perm]), name


def test_batched_full_size_sampled():
    # The 64-column workload at its full 2000 steps; three columns against the oracle.
    w = workloads.multisource()
    st = _run_batch(w, w.steps)
    kw = w.kwargs()
    pos = kw.pop("src_pos")
    for k in (0, 31, 63):
        s = pipeline.setup(src_pos=pos[k:k + 1], **kw)
        ref = s.imex.run(w.steps)
        check_state(s, ref, _col(st, k), w.holes, w.alpha, w.steps)


def test_batched_rejects_source_count_mismatch():
    imex = _imex()
    w = workloads.multisource(nsrc=4)
    with pytest.raises(imex.ImexError):
        imex.Imex.from_workload(w, ncols=3)


@pytest.mark.parametrize("make", [lambda: workloads.plate16(), lambda: workloads.multisource(nsrc=4)])
def test_explicit_variants_agree_bitwise(make, monkeypatch):
    # The autotuner picks one of eight explicit variants (two tile sizes, the
    # persistent strip sweep in long or short chunks, the split launch: the
    # tiles the solve reads first, the others on a second stream beside the
    # solve, with a few CTAs per SM); all must give the same numbers (per
    # node the same contractions and vertex sums in the same order), so the
    # choice never changes a result.  Each sweep runs twice: one CTA per
    # unit, and a few CTAs whose unit ranges cross strips.
    imex = _imex()
    out = {}
    for tile, ctas in (("large", None), ("small", None), ("sweep", None), ("sweep", "7"),
                       ("sweep_short", None), ("sweep_short", "5"), ("large_split1", None),
                       ("large_split2", None), ("small_split2", None), ("small_split4", None)):
        monkeypatch.setenv("IMEX_EXPLICIT_TILE", tile)
        if ctas:
            monkeypatch.setenv("IMEX_SWEEP_CTAS", ctas)
        w = make()
        with imex.Imex.from_workload(w, ncols=len(w.src_pos) if w.name == "multisource" else 1) as g:
            g.step(50)
            info = g.info()
            out[(tile, ctas)] = (g.fields("u", out=np.zeros(g.field_len)), info["explicit_variant"])
    assert [v[1] for v in out.values()] == [0, 1, 2, 2, 3, 3, 4, 5, 6, 7]
    ref = out[("large", None)][0]
    for key, (u, _) in out.items():
        assert np.array_equal(u, ref), key


def test_column_blocks_agree_bitwise(monkeypatch):
    # A walk / dense-top CTA takes a block of independent columns (the factor
    # blocks staged once for all of them); per column the arithmetic is the
    # same, so every block size (here 1, 3 with a ragged last block, 4 and
    # all 10 columns) gives the same numbers bit for bit.
    imex = _imex()
    w = workloads.multisource(nsrc=10)
    out = {}
    for cb in (1, 3, 4, 10):
        monkeypatch.setenv("IMEX_COL_BLOCK", str(cb))
        with imex.Imex.from_workload(w, ncols=10) as g:
            g.step(60)
            assert g.info()["solve_col_block"] == cb
            out[cb] = _state(g)
    assert np.abs(out[1]["a_c"]).max() > 0
    for cb in (3, 4, 10):
        for k in out[1]:
            assert np.array_equal(out[cb][k], out[1][k]), (cb, k)
