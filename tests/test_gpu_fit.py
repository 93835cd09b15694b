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


def _point_bound(O, prob, R, o, ref):
    """The bound for the point gradients: the gradient bound plus twice what moving every float32
    vertex by one ulp does to the oracle's point gradients.  A point's gradient sums few pixels and
    can react to geometry at that scale by several 1e-3 (measured with the oracle: 7.6e-3 for 8
    cubics at 128^2); the device's vertex transform (float-float) differs from the oracle's (double)
    at that scale, so a bound below this reaction would test rounding, not the method."""
    moved, _ = _ref_grad(O, prob, R, o, nudge=True)
    return U.GRAD_RTOL + 2.0 * _point_err(moved, ref).max()


def _pts(prob):
    return np.asarray(prob["pts"], np.float32).reshape(-1, 2)


def _ref_grad(O, prob, R, o, spc=16, nudge=False):
    """The oracle's dL/d(points) for the outlines as the device holds them: the flattened vertices
    are float32 (one rounding of the double flattening), so every cubic path enters the oracle as
    the polygon of its rounded vertices, and the vertex gradients go back to the control points by
    the Bernstein weights.  A point's gradient sums few pixels: that rounding alone moves it by up
    to ~4e-3 of its size (the oracle on rounded against unrounded vertices), more than the bound."""
    sc = O.Scene(prob, spc)
    kind = np.asarray(prob["kind"])
    off = np.asarray(prob["pt_off"])
    pts, koff, kk = [], [0], []
    rng = np.random.default_rng(0)
    for e in range(len(kind)):
        v = sc.local_vertices(e).astype(np.float32) if kind[e] == 0 else \
            np.asarray(prob["pts"], np.float32).reshape(-1, 2)[off[e]:off[e + 1]]
        if nudge:  # every coordinate moved to a float32 neighbour, up or down at random
            v = np.nextafter(v, np.where(rng.uniform(size=v.shape) < 0.5, -np.inf, np.inf).astype(np.float32))
        pts.append(v)
        koff.append(koff[-1] + len(v))
        kk.append(1 if kind[e] == 0 else kind[e])
    flat = dict(prob, kind=np.array(kk, np.int32), pt_off=np.array(koff, np.int32),
                pts=np.concatenate(pts).reshape(-1))
    gv, terms = O.control_grad(flat, prob["params0"], R, o, spc)
    w = O.bernstein_weights(spc)
    out = np.zeros((int(off[-1]), 2))
    for e in range(len(kind)):
        ge = gv[koff[e]:koff[e + 1]]
        if kind[e] != 0:
            out[off[e]:off[e + 1]] = ge
            continue
        npt = int(off[e + 1] - off[e])
        for c in range(npt // 3):
            for r in range(4):
                out[off[e] + (3 * c + r) % npt] += w[:, r] @ ge[c * spc:(c + 1) * spc]
    return out, terms


@pytest.mark.parametrize("name", ["star20_128", "star20_200_t16", "mixed60_full"])
def test_fit_terms_and_point_gradient_match_oracle(env, name):
    O, Collage = env
    prob, kw, grid, tile = _case(name)
    g, o = U.paired(**kw)
    col = Collage(prob, level_res=[grid], tile=tile, fit_controls=1, **g)
    terms, _ = col.loss_backward()
    dp = col.control_grad().cpu().numpy()
    ref, rterms = _ref_grad(O, prob, grid, o)
    U.check_terms(terms.cpu().numpy()[0], rterms, grid, (o.alpha, o.beta, o.gamma, o.delta),
                  use_u=o.gamma != 0)
    err = _point_err(dp, ref)
    assert err.max() <= _point_bound(O, prob, grid, o, ref), (err.max(), np.unravel_index(err.argmax(), err.shape))
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
    gref, t0 = _ref_grad(O, prob, grid, o)
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


def test_fit_batch_of_uneven_problems(env):
    # three outlines on different grids in one handle: every problem's points and their gradient
    O, Collage = env
    probs = [W.fit_problem(2, n_cubics=12, grid=96), W.fit_problem(3, n_cubics=20, grid=160),
             W.fit_problem(4, n_cubics=8, grid=128)]
    g, o = U.paired(**W.FIT_LOSS)
    col = Collage(probs, n_levels=1, level_res=[1], tile=8, fit_controls=1, **g)
    terms, _ = col.loss_backward()
    dp = col.control_grad().cpu().numpy()
    k = 0
    for i, prob in enumerate(probs):
        R = int(prob["grid"])
        ref, rterms = _ref_grad(O, prob, R, o)
        U.check_terms(terms.cpu().numpy()[i], rterms, R, (o.alpha, o.beta, o.gamma, o.delta), use_u=False)
        n = len(ref)
        err = _point_err(dp[k:k + n], ref)
        assert err.max() <= _point_bound(O, prob, R, o, ref), (i, err.max())
        k += n
    assert k == len(dp)
    col.close()
