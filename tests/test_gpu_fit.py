"""Outline fitting (Sec. 3, Vector Representation) through the C ABI against the FP64 oracle: loss
terms and dL/d(points), the device flattening after collage_set_controls, and Adam steps on the
points with the transforms held fixed."""
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


def _case(name):
    """(problem, loss kwargs, grid, tile)"""
    if name == "star20_128":
        return W.fit_problem(0, n_cubics=20, grid=128), dict(W.FIT_LOSS), 128, 8
    if name == "star20_200_t16":  # ragged: 200 is no multiple of the 16-px tile
        return W.fit_problem(1, n_cubics=20, grid=200), dict(W.FIT_LOSS), 200, 16
    if name == "mixed60_full":  # every element kind, the full loss of Eq. 8 with padding and force
        return W.config_problem(3, n_elems=60, grid=192), dict(pad_px=2.0, delta=100.0), 192, 8
    raise KeyError(name)


def _point_err(g, gr):
    """Per coordinate, relative to max(|g_ref|, 1e-2 max |g_ref|) (near-zero entries)."""
    floor = U.GRAD_FLOOR * np.abs(gr).max()
    return np.abs(g - gr) / np.maximum(np.abs(gr), floor)


def _pts(prob):
    return np.asarray(prob["pts"], np.float32).reshape(-1, 2)


@pytest.mark.parametrize("name", ["star20_128", "star20_200_t16", "mixed60_full"])
def test_fit_terms_and_point_gradient_match_oracle(env, name):
    O, Collage = env
    prob, kw, grid, tile = _case(name)
    g, o = U.paired(**kw)
    col = Collage(prob, level_res=[grid], tile=tile, fit_controls=1, **g)
    terms, _ = col.loss_backward()
    dp = col.control_grad().cpu().numpy()
    ref, rterms = O.control_grad(prob, prob["params0"], grid, o)
    U.check_terms(terms.cpu().numpy()[0], rterms, grid, (o.alpha, o.beta, o.gamma, o.delta),
                  use_u=o.gamma != 0)
    err = _point_err(dp, ref)
    assert err.max() <= U.GRAD_RTOL, (err.max(), np.unravel_index(err.argmax(), err.shape))
    # the points themselves are untouched by a backward pass
    assert np.array_equal(col.get_controls().cpu().numpy(), _pts(prob))
    col.close()


def test_set_controls_flattens_on_the_device(env):
    O, Collage = env
    prob, kw, grid, tile = _case("mixed60_full")
    g, o = U.paired(**kw)
    col = Collage(prob, level_res=[grid], tile=tile, **g)  # any mode: points are settable
    rng = np.random.default_rng(3)
    P = _pts(prob)
    P2 = (P * (1.0 + 0.3 * rng.uniform(-1, 1, size=P.shape))).astype(np.float32)  # bigger and smaller
    col.set_controls(torch.from_numpy(P2).cuda())
    assert np.array_equal(col.get_controls().cpu().numpy(), P2)
    bw, _ = col.render()
    prob2 = dict(prob)
    prob2["pts"] = P2.reshape(-1)
    ihat, _, _ = O.Scene(prob2).render(prob["params0"].astype(np.float64), grid, o)
    assert np.abs(bw.cpu().numpy().reshape(grid, grid) - ihat).max() <= U.COV_ATOL
    # without fit_controls the point gradient stays zero
    col.loss_backward()
    assert not col.control_grad().abs().max().item()
    col.close()


@pytest.mark.parametrize("deterministic", [0, 1])
def test_fit_adam_steps(env, deterministic):
    O, Collage = env
    prob, kw, grid, tile = _case("star20_128")
    g, o = U.paired(**kw)
    col = Collage(prob, level_res=[grid], tile=tile, fit_controls=1, deterministic=deterministic,
                  **g)
    P0 = _pts(prob).astype(np.float64)
    gref, t0 = O.control_grad(prob, prob["params0"], grid, o)
    col.step(1)
    P1 = col.get_controls().cpu().numpy().astype(np.float64)
    r1, _, _ = O.adam_points(P0, np.zeros_like(P0), np.zeros_like(P0), gref, 1)
    # the first Adam step moves a coordinate by lr g / (|g| + eps): where the gradient is clearly
    # nonzero the two agree to rounding, elsewhere the move is at most lr
    big = np.abs(gref) > U.GRAD_FLOOR * np.abs(gref).max()
    assert np.abs(P1 - r1)[big].max() <= 1e-6
    assert np.abs(P1 - P0).max() <= 1e-2 + 1e-6
    # many steps: the transforms stay put, the GPU loss is the oracle's loss at the GPU's points,
    # and the fit improves
    col.step(60)
    P = col.get_controls().cpu().numpy()
    terms = col.loss().cpu().numpy()[0]
    prob2 = dict(prob)
    prob2["pts"] = P.reshape(-1)
    assert np.array_equal(col.get_params().cpu().numpy().reshape(-1), prob["params0"])
    col.loss_backward()  # the loss at the current points (step reports the previous iteration's)
    now = col.loss().cpu().numpy()[0]
    ref = O.Scene(prob2).eval(prob["params0"].astype(np.float64), grid, o, grad=False)["terms"]
    U.check_terms(now, ref, grid, (o.alpha, o.beta, o.gamma, o.delta), use_u=False)
    assert ref[0] < 0.5 * t0[0], (t0[0], ref[0], terms[0])
    col.close()


def test_fit_step_host_moves_points_not_transforms(env):
    # the host-buffer step in fitting mode: the transforms it returns are the fixed ones, the points
    # move, and the loss it returns is the iteration's
    O, Collage = env
    prob, kw, grid, tile = _case("star20_128")
    g, o = U.paired(**kw)
    col = Collage(prob, level_res=[grid], tile=tile, fit_controls=1, **g)
    p0 = np.asarray(prob["params0"], np.float32)
    for _ in range(3):
        pout, lout = col.step_host(1, params_in=p0)
        assert np.array_equal(pout, p0)
    assert not np.array_equal(col.get_controls().cpu().numpy(), _pts(prob))
    assert np.array_equal(lout, col.loss().cpu().numpy().reshape(-1))
    col.close()
