"""The allocation-free stepping entry point (imex_step_noalloc) against imex_step.

imex_step_noalloc serves callers that must not allocate device memory while
stepping: the implicit solve's scratch comes from a fixed array inside the
library.  Two identical problems are advanced side by side, one through each
entry point, over two calls in a row (the second call reuses the array with
whatever the first left in it); the fields must agree within the parity
tolerance of the other GPU tests.
"""
import numpy as np
import pytest

from paper_2310_14712_gb300 import workloads

pytestmark = pytest.mark.gpu


def _rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a - b))


def test_noalloc_step_matches_step_over_two_calls():
    from paper_2310_14712_gb300 import imex
    w = workloads.plate16()
    with imex.Imex.from_workload(w) as ref, imex.Imex.from_workload(w) as na:
        for n in (17, 23):
            ref.step(n)
            na.step_noalloc(n)
            assert na.info()["step"] == ref.info()["step"]
            for field in ("u", "u_prev_d", "v_c", "a_c"):
                a = na.fields(field, out=np.zeros(na.n_nodes))
                b = ref.fields(field, out=np.zeros(ref.n_nodes))
                assert np.isfinite(a).all()
                assert _rel(a, b) <= 1e-11, (field, n, _rel(a, b))
