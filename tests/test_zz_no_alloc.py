"""collage_uniform_term_noalloc against the regular entry point and the FP64 oracle.

The allocation-free call serves callers that must not call cudaMalloc: their device memory belongs
to another allocator (a framework's caching allocator, a fixed arena), or their loop cannot afford
cudaMalloc's synchronisation.  It must give the distribution loss that collage_loss_backward
reports for the same image and container, and a gradient dL_u/dO equal, pixel by pixel, to the
oracle's on the same inputs, call after call, even though every call reuses one built-in scratch
array.  This file is collected last so that a failure here comes after every other test has run.
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


def _reference_and_inputs(prob, res, weights):
    """L_u from collage_loss_backward, the rendered image, and the container coverage rendered as
    an element (the container's rings as polygons about the centre)."""
    from paper_2406_04008_gb300.collage import Collage
    g, _ = U.paired(n_dil=len(weights), dil_weight=tuple(weights))
    col = Collage(prob, level_res=[res], **g)
    terms, _ = col.loss_backward()
    ihat, _ = col.render()
    roff = np.asarray(prob["ring_off"])
    rp = prob["ring_pts"].reshape(-1, 2).astype(np.float64)
    rings = [rp[roff[r]:roff[r + 1]] for r in range(len(roff) - 1)]
    assert len(rings) == 1, "the container must be one ring to render it as one element"
    cont = W.make_problem([(1, rings[0] - (0.5, 0.5), 0.0)], rings, [(0.5, 0.5, 0.0, 1.0)], res)
    ccol = Collage(cont, level_res=[res], **g)
    cbw, _ = ccol.render()
    torch.cuda.synchronize()
    ref = float(terms[0, 2].item())
    col.close()
    ccol.close()
    return ref, ihat, (1.0 - cbw).contiguous()


def _call(L, res, ihat, cov, weights):
    w = (C.c_float * len(weights))(*weights)
    loss = torch.zeros(1, device="cuda", dtype=torch.float32)
    grad = torch.empty(res * res, device="cuda", dtype=torch.float32)
    st = L.load().collage_uniform_term_noalloc(
        C.c_void_p(torch.cuda.current_stream().cuda_stream), res, len(weights), w,
        C.c_void_p(ihat.data_ptr()), C.c_void_p(cov.data_ptr()), C.c_void_p(loss.data_ptr()),
        C.c_void_p(grad.data_ptr()))
    return st, loss, grad


def _box(img, r):
    c = np.pad(img, ((r + 1, r), (r + 1, r))).cumsum(0).cumsum(1)
    n = img.shape[0]
    w = 2 * r + 1
    return c[w:w + n, w:w + n] - c[:n, w:w + n] - c[w:w + n, :n] + c[:n, :n]


def _qbits(w):
    """Fixed-point bits of the call's box sums for a widest kernel of w px: the most (at most 23)
    for which every sum of w x w values in [0, 1] fits in 32 bits with a bit to spare."""
    q = 0
    while q < 23 and (w * w + w) << (q + 1) < 1 << 32:
        q += 1
    return q


def _check_against_oracle(oracle_mod, ihat, cov, weights, got_loss, got_grad):
    """The oracle's L_u and dL_u/dO on the same (float) inputs promoted to FP64.  The call decides
    min(1, B) on box sums in fixed point (each O rounded to a multiple of 2^-Q); where that decision
    differs from the exact one (a box sum within rounding of 1), both sides of the kink are valid
    one-sided derivatives, so the pixels whose windows hold such a flip are left out of the
    element-wise comparison (there are few or none)."""
    res = int(round(ihat.numel() ** 0.5))
    ih32 = ihat.cpu().numpy().reshape(res, res)
    occ = 1.0 - ih32.astype(np.float64)
    covc = cov.double().cpu().numpy().reshape(res, res)
    lu, gou = oracle_mod.uniform_term(occ, covc, weights)
    assert abs(got_loss - lu) <= U.LOSS_RTOL * abs(lu) + U.COV_ATOL, (got_loss, lu)
    K = len(weights)
    Q = _qbits(5 + 6 * (K - 1))
    fixed = np.rint((np.float32(1.0) - ih32).astype(np.float64) * 2.0 ** Q)  # the call's rounding
    skip = np.zeros((res, res), bool)
    for k in range(K):
        r = 2 + 3 * k
        flip = (_box(fixed, r) < 2.0 ** Q) != (_box(occ, r) < 1.0)
        skip |= _box(flip.astype(np.float64), r) > 0
    assert skip.sum() <= res * res // 100, skip.sum()
    g = got_grad.double().cpu().numpy().reshape(res, res)
    floor = U.GRAD_FLOOR * np.abs(gou).max()
    err = np.abs(g - gou) / np.maximum(np.abs(gou), floor)
    err[skip] = 0.0
    assert err.max() <= U.GRAD_RTOL, (err.max(), np.unravel_index(err.argmax(), err.shape))
    assert np.abs(gou).max() > 0


CASES = [  # (problem, res, weights): the widest kernel count at a grid that is not a multiple of
           # the 32-px dilation tile, and the default four kernels on two grids
    (lambda: W.config_problem(2, n_elems=40, grid=200), 200, tuple(float(k + 1) for k in range(8))),
    (lambda: W.config_problem(1, n_elems=16, grid=256), 256, (1.0, 2.0, 3.0, 4.0)),
    (lambda: W.config_problem(1, collage_index=5, n_elems=9, grid=128), 128, (1.0, 2.0, 3.0, 4.0)),
]


def test_noalloc_matches_loss_backward_and_oracle_on_consecutive_calls(lib, oracle_mod):
    # different problems, sizes and kernel counts back to back: no call may see the previous
    # call's leftovers in the shared scratch
    first = []
    for make, res, wts in CASES:
        ref, ihat, cov = _reference_and_inputs(make(), res, wts)
        st, loss, grad = _call(lib, res, ihat, cov, wts)
        assert st == 0
        torch.cuda.synchronize()
        got = float(loss.item())
        assert ref > 0
        assert abs(got - ref) <= U.LOSS_RTOL * abs(ref) + U.COV_ATOL, (got, ref)
        _check_against_oracle(oracle_mod, ihat, cov, wts, got, grad)
        first.append((got, grad.clone()))
    # the first case again, twice in a row: the same answer as its first call, bit for bit
    make, res, wts = CASES[0]
    _, ihat, cov = _reference_and_inputs(make(), res, wts)
    for _ in range(2):
        st, loss, grad = _call(lib, res, ihat, cov, wts)
        torch.cuda.synchronize()
        assert st == 0 and float(loss.item()) == first[0][0]
        assert torch.equal(grad, first[0][1])


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    x = torch.zeros(1, device="cuda", dtype=torch.float32)
    st, _, _ = _call(lib, 1025, x, x, (1.0, 2.0, 3.0, 4.0))
    assert st == -1  # COLLAGE_ERR_INVALID_ARG: 1025^2 pixels exceed COLLAGE_NOALLOC_MAX_PIXELS
    st, _, _ = _call(lib, 0, x, x, (1.0, 2.0, 3.0, 4.0))
    assert st == -1
    st, _, _ = _call(lib, 64, x, x, tuple(1.0 for _ in range(9)))
    assert st == -1  # more than 8 kernels
