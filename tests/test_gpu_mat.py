"""Skeleton-based initialisation (Sec. 4.1) through the C ABI against the FP64 oracle: the medial
width, the ridge axis and the placements are integer or float32 decisions taken the same way on both
sides, so they are compared exactly."""
import numpy as np
import pytest
import torch

from paper_2406_04008_gb300 import workloads as W
from tests import _util as U

pytestmark = pytest.mark.gpu

# the inside test is coverage >= 1/2; a pixel whose coverage lies this close to 1/2 could fall
# either way between FP32 and FP64, so the cases are checked to have none
AMBIGUOUS = 1e-4


@pytest.fixture(scope="module")
def env(oracle_mod):
    from paper_2406_04008_gb300 import build
    build.build()
    from paper_2406_04008_gb300.collage import Collage
    assert torch.cuda.is_available()
    return oracle_mod, Collage


def _check(env, probs, grids, **gpu):
    O, Collage = env
    g, o = U.paired()
    g.update(gpu)
    col = Collage(probs, **g)
    axis, width = col.mat_init(want_maps=True)
    q = col.get_params().cpu().numpy()
    axis, width = axis.cpu().numpy(), width.cpu().numpy()
    col.close()
    pix = e0 = 0
    for prob, R in zip(probs, grids):
        _, _, covc = O.Scene(prob).render(prob["params0"].astype(np.float64), R, o)
        assert np.abs(covc - 0.5).min() > AMBIGUOUS
        qr, D2, ax = O.mat_init(prob, prob["params0"], R, o)
        n = len(prob["kind"])
        assert np.array_equal(axis[pix:pix + R * R].reshape(R, R), ax.astype(np.int32))
        assert np.array_equal(width[pix:pix + R * R].reshape(R, R), np.sqrt(D2.astype(np.float32)))
        assert np.array_equal(q[e0:e0 + n], qr)
        pix += R * R
        e0 += n


def test_mat_init_mixed_annulus(env):
    _check(env, [W.config_problem(3, n_elems=120, grid=256)], [256], level_res=[256], tile=8)


def test_mat_init_open_rect_ragged(env):
    # the open top: the rows above the image count as outside
    _check(env, [W.config_problem(5, n_elems=150, grid=240)], [240], level_res=[240], tile=16)


def test_mat_init_batch(env):
    probs = [W.config_problem(4, i) for i in range(3)]
    _check(env, probs, [int(p["grid"]) for p in probs], n_levels=1, level_res=[1], tile=8)


def test_mat_init_headline_size(env):
    # the 1000-element workload's container at its 1024^2 level, in the benchmark's configuration
    _check(env, [W.config_problem(3)], [1024], level_res=[1024], tile=8, persistent=1, use_graphs=1)


def test_mat_init_empty_container_keeps_params(env):
    # a container smaller than a pixel has no inside pixel at 64^2: nothing moves, no axis
    O, Collage = env
    rng = W.PCG32(3)
    els = [(1, W.regular_polygon(0.05, 6), 0.0), (0, W.blob_controls(rng, 0.04), 0.0)]
    params = [(0.3, 0.4, 0.5, 1.0), (0.6, 0.7, 1.0, 1.2)]
    prob = W.make_problem(els, [W.regular_polygon(0.002, 8) + (0.5, 0.5)], params, 64)
    g, o = U.paired()
    col = Collage(prob, level_res=[64], tile=8, **g)
    axis, width = col.mat_init(want_maps=True)
    assert not axis.any().item() and not width.any().item()
    assert np.array_equal(col.get_params().cpu().numpy().reshape(-1), prob["params0"])
    col.close()


def test_mat_init_more_elements_than_ranked(env):
    # past 4096 elements the placement takes the largest remaining element by a reduction per step
    # instead of a precomputed order: the same rule, the same result
    rng = W.PCG32(8)
    els, params = [], []
    for _ in range(4200):
        els.append((1, W.regular_polygon(0.002 + 0.004 * rng.uniform(), 5), 0.0))
        params.append((0.5, 0.5, 0.0, 0.6 + 0.8 * rng.uniform()))
    prob = W.make_problem(els, W.annulus_container(), params, 256)
    _check(env, [prob], [256], level_res=[256], tile=16)


def test_mat_init_few_axis_pixels(env):
    # a container a few pixels wide: fewer axis pixels than the placement's cluster has blocks,
    # so most blocks hold no candidate and the choice comes from the others' partials; more
    # elements than axis pixels, so the later ones take the pixel of largest clearance
    O, Collage = env
    rng = W.PCG32(7)
    els = [(1, W.regular_polygon(0.01 + 0.005 * k, 6), 0.0) for k in range(5)] + \
          [(0, W.blob_controls(rng, 0.012), 0.0) for _ in range(4)]
    params = [(0.2 + 0.07 * k, 0.3, 0.1 * k, 1.0) for k in range(len(els))]
    for side in (0.018, 0.035):  # 4 and 16 axis pixels
        ring = W.regular_polygon(side, 24) + (0.5, 0.5)
        prob = W.make_problem(els, [ring], params, 64)
        _check(env, [prob], [64], level_res=[64], tile=8)
