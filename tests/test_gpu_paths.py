"""Parity on inputs that drive the raster kernels down their rarely taken paths.

Each case is built so that one path must run, and the library's path counters (collage_get_info)
prove that it did:
  - a comb whose pixel rows cross the outline more than 16 times inside one tile: the winding
    number of those rows is taken over every segment; its 523 segments are more than the 512
    the emission stages in shared memory, so its tiles read the outline from global memory;
  - 40 small disks stacked at one spot: tiles that list more than 32 elements, ranked by the
    composite from their element ids staged in shared memory; 300 of them: lists longer than that
    staging (256), ranked from global memory;
  - a disk container of 3000 segments: the container raster stages its ring in chunks;
  - a solid disk wider than the widest dilation kernel: full boxes, whose fixed-point sums pass
    2^31 (the distribution term's unsigned arithmetic).
Per-pixel Ihat / A_tau are compared with the FP64 oracle at 1e-5, the loss terms at 1e-5 relative
and every gradient component at 1e-3 (atomic and deterministic modes): nonzero winding and the
composites of Sec. 3-4.2.
"""
import numpy as np
import pytest
import torch

from paper_2406_04008_gb300 import workloads as W
from tests import _util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(oracle_mod):
    from paper_2406_04008_gb300 import build
    build.build()
    from paper_2406_04008_gb300.collage import Collage
    assert torch.cuda.is_available()
    return oracle_mod, Collage


def comb(width_px, teeth, tooth_px, body_px, res):
    """A closed polygon: a body of width_px x body_px with `teeth` triangular teeth of height
    tooth_px along its top edge (period width_px / teeth), centred on the origin, unit coords."""
    p = width_px / teeth
    v = [(0.0, 0.0), (width_px, 0.0), (width_px, body_px)]
    for k in range(teeth):
        v.append((width_px - (k + 0.5) * p, body_px + tooth_px))
        v.append((width_px - (k + 1) * p, body_px))
    v = np.asarray(v[:-1] + [(0.0, body_px)])
    v -= (width_px / 2, (body_px + tooth_px) / 2)
    return v / res


def comb_problem(res):
    els = [(1, comb(48.0, 260, 6.0, 5.0, res), 0.0)]
    params = [(0.5, 0.5, 0.12, 1.0)]
    rng = np.random.default_rng(3)
    for _ in range(6):  # ordinary elements beside it
        els.append((1, W.regular_polygon(rng.uniform(0.02, 0.05), 16), 0.0))
        a = rng.uniform(0, 2 * np.pi)
        params.append((0.5 + 0.25 * np.cos(a), 0.5 + 0.25 * np.sin(a), 0.0, 1.0))
    return W.make_problem(els, W.disk_container(), params, res)


def stack_problem(res):
    rng = np.random.default_rng(5)
    els, params = [], []
    for _ in range(40):
        els.append((1, W.regular_polygon(rng.uniform(2.0, 3.0) / res, 12), 0.0))
        params.append((0.5 + rng.uniform(-0.6, 0.6) / res, 0.5 + rng.uniform(-0.6, 0.6) / res,
                       rng.uniform(0, 1), 1.0))
    return W.make_problem(els, W.disk_container(), params, res)


def big_ring_problem(res):
    prob = W.config_problem(1, n_elems=16, grid=res)
    ring = W.disk_container(n=3000)
    return W.make_problem(
        [(int(prob["kind"][e]),
          prob["pts"][2 * prob["pt_off"][e]:2 * prob["pt_off"][e + 1]].reshape(-1, 2).astype(np.float64),
          0.0) for e in range(len(prob["kind"]))],
        ring, prob["params0"].reshape(-1, 4).astype(np.float64), res)


def _check_case(env, prob, res, tile, det=0, opts=None):
    O, Collage = env
    g, o = U.paired(**(opts or {}))
    col = Collage(prob, level_res=[res], tile=tile, deterministic=det, **g)
    bw, tau = col.render()
    terms, grad = col.loss_backward()
    torch.cuda.synchronize()
    info = col.info()
    sc = O.Scene(prob)
    q = prob["params0"].astype(np.float64)
    ihat, atau, _ = sc.render(q, res, o)
    assert np.abs(bw.cpu().numpy().reshape(res, res) - ihat).max() <= U.COV_ATOL
    assert np.abs(tau.cpu().numpy().reshape(res, res) - atau).max() <= U.COV_ATOL
    ref = sc.eval(q, res, o)
    U.check_terms(terms.cpu().numpy()[0], ref["terms"], res, (o.alpha, o.beta, o.gamma, o.delta),
                  use_u=o.gamma != 0)
    U.check_grad(grad.cpu().numpy(), ref["grad_a"])
    col.close()
    return info


@pytest.mark.parametrize("tile,det", [(8, 0), (16, 0), (16, 1)])
def test_comb_rows_over_the_crossing_list(env, tile, det):
    info = _check_case(env, comb_problem(128), 128, tile, det)
    assert info["path_row_fallback"] > 0, info
    assert info["path_long_near"] > 0, info


@pytest.mark.parametrize("tile,det", [(8, 0), (8, 1), (16, 0)])
def test_tiles_with_more_than_32_elements(env, tile, det):
    info = _check_case(env, stack_problem(128), 128, tile, det, dict(pad_px=1.0))
    assert info["path_wide_tile"] > 0, info


@pytest.mark.parametrize("tile", [8, 16])
def test_container_ring_longer_than_one_chunk(env, tile):
    info = _check_case(env, big_ring_problem(160), 160, tile)
    assert info["path_ring_chunk"] > 0, info


def test_ordinary_case_takes_none_of_these_paths(env):
    # the counters count: a plain small case leaves them at zero
    info = _check_case(env, W.config_problem(1), 128, 16, 0, dict(gamma=0.0))
    assert info["path_row_fallback"] == info["path_wide_tile"] == info["path_ring_chunk"] == 0, info


def solid_problem(res):
    """One large irregular polygon over the middle of the container: the occupancy is 1 over whole
    boxes of the widest kernel, whose fixed-point sums then pass 2^31.  Placed off both axes with
    a blob beside it, so that no gradient component vanishes by symmetry."""
    rng = W.PCG32(17)
    els = [(1, W.convex_polygon(rng, 0.28, 24), 0.0), (0, W.blob_controls(rng, 0.05), 0.0)]
    params = [(0.47, 0.52, 0.3, 1.0), (0.62, 0.86, 0.0, 1.0)]
    return W.make_problem(els, W.disk_container(), params, res)


@pytest.mark.parametrize("n_dil", [4, 8])
def test_solid_occupancy_box_sums_past_2_31(env, n_dil):
    # the fixed-point precision Q is the largest with (w^2 + w) 2^(Q+1) < 2^32, w the widest
    # kernel, so a full box holds w^2 2^Q, which is 2^31 or more for both kernel counts here
    w, q = 5 + 6 * (n_dil - 1), 0
    while q < 23 and ((w * w + w) << (q + 1)) < (1 << 32):
        q += 1
    assert (w * w) << q >= 1 << 31
    _check_case(env, solid_problem(128), 128, 8, 0,
                dict(n_dil=n_dil, dil_weight=tuple(float(k + 1) for k in range(n_dil))))


def deep_stack_problem(res, n=300):
    rng = np.random.default_rng(7)
    els, params = [], []
    for _ in range(n):
        els.append((1, W.regular_polygon(rng.uniform(1.5, 2.5) / res, 8), 0.0))
        params.append((0.5 + rng.uniform(-0.8, 0.8) / res, 0.5 + rng.uniform(-0.8, 0.8) / res,
                       rng.uniform(0, 1), 1.0))
    return W.make_problem(els, W.disk_container(), params, res)


def test_tiles_with_more_than_256_elements(env):
    # lists longer than the composite ranks in shared memory: ranked from global memory
    O, _ = env
    prob = deep_stack_problem(128)
    t, _ = O.Scene(prob).bins(prob["params0"], 128, 8, 1.0, 1.0)
    assert np.bincount(t).max() > 256  # the case reaches that path
    info = _check_case(env, prob, 128, 8, 1, dict(pad_px=1.0))
    assert info["path_wide_tile"] > 0, info
