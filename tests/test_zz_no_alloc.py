"""The allocation-free stepping entry point (imex_step_noalloc) against imex_step.

imex_step_noalloc serves callers that must not allocate device memory while
stepping (a device budget fixed at start-up, or code regions where allocation
calls are not allowed): the factorised solve's scratch comes from a fixed
array inside the library.  Two identical problems are advanced side by side,
one through each entry point, over two calls in a row (the second call reuses
the array with whatever the first left in it).  Both run the same kernels in
the same order on the same stream, only with other scratch addresses, so the
fields must be bit-identical.  Contexts the entry point cannot serve (set to
a PCG solver, or needing more scratch than the array holds) are rejected
before anything is launched.
"""
import numpy as np
import pytest

from paper_2310_14712_gb300 import workloads

pytestmark = pytest.mark.gpu

FIELDS = ("u", "u_prev_d", "v_c", "a_c")


def _imex():
    from paper_2310_14712_gb300 import imex
    return imex


def _side_by_side(w, calls=(17, 23), **kw):
    imex = _imex()
    with imex.Imex.from_workload(w, **kw) as ref, imex.Imex.from_workload(w, **kw) as na:
        for n in calls:
            ref.step(n)
            na.step_noalloc(n)
            assert na.info()["step"] == ref.info()["step"]
            for field in FIELDS:
                a = na.fields(field, out=np.zeros(na.field_len))
                b = ref.fields(field, out=np.zeros(ref.field_len))
                assert np.isfinite(a).all()
                assert np.array_equal(a, b), (field, n, float(np.abs(a - b).max()))


def test_noalloc_step_matches_step_over_two_calls():
    _side_by_side(workloads.plate16())


def test_noalloc_batched_columns_match_step():
    w = workloads.multisource(nsrc=4, steps=40)
    _side_by_side(w, ncols=4)


def test_noalloc_cdm_scheme_matches_step():
    _side_by_side(workloads.plate16(), scheme="cdm")


def test_noalloc_large_supernodes_match_step():
    # A 3D solid whose factor has supernodes of more than 256 rows: the
    # array also holds the backward products of their row chunks.
    w = workloads.voids3d(ncells=(8, 8, 4), steps=40)
    imex = _imex()
    with imex.Imex.from_workload(w) as g:
        assert g.info()["large_supernodes"] > 0
    _side_by_side(w, calls=(5, 7))


def test_noalloc_rejects_pcg_context_and_oversized_problem():
    imex = _imex()
    with imex.Imex.from_workload(workloads.plate16()) as g:
        g.set_solver("pcg_jacobi", 1e-10, 500)
        with pytest.raises(imex.ImexError) as ei:
            g.step_noalloc(2)
        assert ei.value.code == -1          # IMEX_ERR_ARG
        assert g.info()["step"] == 0         # nothing launched
        g.set_solver("direct")
        g.step_noalloc(2)
        assert g.info()["step"] == 2
    # 8 columns of the 256x128 plate: 8 x 2 x n_c alone exceeds 262,144 doubles.
    w = workloads.plate256()
    w.src_pos = np.repeat(w.src_pos, 8, axis=0)
    with imex.Imex.from_workload(w, ncols=8) as g:
        assert 8 * 2 * g.info()["n_c"] > 262144
        with pytest.raises(imex.ImexError) as ei:
            g.step_noalloc(1)
        assert ei.value.code == -1
        assert g.info()["step"] == 0
