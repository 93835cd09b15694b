"""collage_uniform_term_noalloc against the regular entry point.

The allocation-free call serves callers that must not call cudaMalloc (their device memory belongs
to another allocator, or their loop cannot afford cudaMalloc's synchronisation).  It must give the
distribution loss that collage_loss_backward reports for the same image and container, call after
call, even though every call reuses one built-in scratch array.  This file is collected last so
that a failure here comes after every other test has run.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2406_04008_gb300 import workloads as W
from tests import _util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2406_04008_gb300 import build
    build.build()
    from paper_2406_04008_gb300 import _lib as L
    assert torch.cuda.is_available()
    return L


def _reference_and_inputs(prob, res):
    """L_u from collage_loss_backward, the rendered image, and the container coverage rendered as
    an element (the disk container's ring as a polygon about its centre)."""
    from paper_2406_04008_gb300.collage import Collage
    g, _ = U.paired()
    col = Collage(prob, level_res=[res], **g)
    terms, _ = col.loss_backward()
    ihat, _ = col.render()
    ring = prob["ring_pts"].reshape(-1, 2).astype(np.float64)
    cont = W.make_problem([(1, ring - (0.5, 0.5), 0.0)], [ring], [(0.5, 0.5, 0.0, 1.0)], res)
    ccol = Collage(cont, level_res=[res], **g)
    cbw, _ = ccol.render()
    torch.cuda.synchronize()
    ref = float(terms[0, 2].item())
    col.close()
    ccol.close()
    return ref, ihat, (1.0 - cbw).contiguous()


def _call(L, res, ihat, cov, weights=(1.0, 2.0, 3.0, 4.0)):
    w = (C.c_float * len(weights))(*weights)
    loss = torch.zeros(1, device="cuda", dtype=torch.float32)
    grad = torch.empty(res * res, device="cuda", dtype=torch.float32)
    st = L.load().collage_uniform_term_noalloc(
        C.c_void_p(torch.cuda.current_stream().cuda_stream), res, len(weights), w,
        C.c_void_p(ihat.data_ptr()), C.c_void_p(cov.data_ptr()), C.c_void_p(loss.data_ptr()),
        C.c_void_p(grad.data_ptr()))
    return st, loss, grad


def test_noalloc_matches_loss_backward_on_consecutive_calls(lib):
    # two different problems and sizes back to back: the second call must not see the first's
    # leftovers in the shared scratch
    cases = [(W.config_problem(1, n_elems=16, grid=256), 256),
             (W.config_problem(1, collage_index=5, n_elems=9, grid=128), 128)]
    results = []
    for prob, res in cases:
        ref, ihat, cov = _reference_and_inputs(prob, res)
        st, loss, grad = _call(lib, res, ihat, cov)
        assert st == 0
        torch.cuda.synchronize()
        got = float(loss.item())
        assert ref > 0
        assert abs(got - ref) <= U.LOSS_RTOL * abs(ref) + U.COV_ATOL, (got, ref)
        assert torch.isfinite(grad).all()
        results.append((got, grad.clone()))
    # the first case again: same answer as its first call
    prob, res = cases[0]
    ref, ihat, cov = _reference_and_inputs(prob, res)
    st, loss, grad = _call(lib, res, ihat, cov)
    torch.cuda.synchronize()
    assert st == 0 and float(loss.item()) == results[0][0]
    assert torch.equal(grad, results[0][1])


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    x = torch.zeros(1, device="cuda", dtype=torch.float32)
    st, _, _ = _call(lib, 1025, x, x)
    assert st == -1  # COLLAGE_ERR_INVALID_ARG: 1025^2 pixels exceed COLLAGE_NOALLOC_MAX_PIXELS
    st, _, _ = _call(lib, 0, x, x)
    assert st == -1
