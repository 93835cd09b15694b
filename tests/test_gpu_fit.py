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


def _generic(prob, grid, k=0):
    """The fitting workload's circle starts centred on the grid, so its flattening is symmetric
    about the grid diagonals: a pixel centre on a diagonal is exactly equidistant from the two
    segments meeting at the vertex there, where the gradient is set-valued (reading A15: any
    choice is a valid one-sided derivative, and float rounding decides which side a kernel takes).
    The parity cases move the (fixed) transform by a fraction of a pixel and rotate it slightly, so
    that no pixel sits on such a tie; _assert_tie_free checks it."""
    q = np.asarray(prob["params0"], np.float64).reshape(-1, 4).copy()
    q[:, 0] += (0.29 + 0.07 * k) / grid
    q[:, 1] += (0.41 - 0.05 * k) / grid
    q[:, 2] += 0.0137 * (1 + k)
    out = dict(prob)
    out["params0"] = q.astype(np.float32).reshape(-1)
    return out


def _case(name):
    """(problem, loss kwargs, grid, tile)"""
    if name == "star20_128":
        return _generic(W.fit_problem(0, n_cubics=20, grid=128), 128, 5), dict(W.FIT_LOSS), 128, 8
    if name == "star20_200_t16":  # ragged: 200 is no multiple of the 16-px tile
        return _generic(W.fit_problem(1, n_cubics=20, grid=200), 200, 0), dict(W.FIT_LOSS), 200, 16
    if name == "mixed60_full":  # every element kind, the full loss of Eq. 8 with padding and force
        return W.config_problem(3, n_elems=60, grid=192), dict(pad_px=2.0, delta=100.0), 192, 8
    raise KeyError(name)


TIE_PX = 1e-5  # the device's distances are good to ~1e-6 px


def _assert_tie_free(O, prob, R, o):
    """No pixel whose coverage carries a gradient (|sd| < rho + pad (+ hw), in px) has two closest
    segments, with different closest points, whose distances differ by less than TIE_PX."""
    sc = O.Scene(prob)
    q = np.asarray(prob["params0"], np.float64)
    kind = np.asarray(prob["kind"])
    hw = np.asarray(prob["hw"], np.float64)
    ys, xs = np.mgrid[0:R, 0:R]
    P = np.stack([(xs.ravel() + 0.5), (ys.ravel() + 0.5)], 1)  # px
    for e in range(len(kind)):
        v = sc.world_vertices(q, e) * R
        a = v if kind[e] != 2 else v[:-1]
        b = np.roll(v, -1, 0) if kind[e] != 2 else v[1:]
        lo, hi = v.min(0) - 4 - hw[e] * R, v.max(0) + 4 + hw[e] * R
        sel = np.all((P >= lo) & (P <= hi), 1)
        p = P[sel]
        ab = b - a
        t = np.clip(((p[:, None, :] - a[None]) * ab[None]).sum(2) / np.maximum((ab * ab).sum(1), 1e-300), 0, 1)
        cp = a[None] + t[:, :, None] * ab[None]
        d = np.hypot(*(p[:, None, :] - cp).transpose(2, 0, 1))
        j = d.argmin(1)
        d1 = d[np.arange(len(p)), j]
        sd = d1 if kind[e] == 2 else d1  # |sd| for closed kinds; hw - d for strokes
        band = (np.abs(hw[e] * R - d1) if kind[e] == 2 else d1) < o.rho_px + o.pad_px
        same = np.hypot(*(cp - cp[np.arange(len(p)), j][:, None, :]).transpose(2, 0, 1)) < 1e-6
        d2 = np.where(same, np.inf, d).min(1)
        ties = band & (d2 - d1 < TIE_PX)
        assert not ties.any(), (e, p[ties][:4], (d2 - d1)[ties][:4], sd[ties][:4])


def _point_err(g, gr):
    """Per coordinate, relative to max(|g_ref|, 1e-2 max |g_ref|) (near-zero entries)."""
    floor = U.GRAD_FLOOR * np.abs(gr).max()
    return np.abs(g - gr) / np.maximum(np.abs(gr), floor)


def _pts(prob):
    return np.asarray(prob["pts"], np.float32).reshape(-1, 2)


def _ref_grad(O, prob, R, o, spc=16, tie_free=True):
    """The oracle's dL/d(points) at the problem's control points (FP64 flattening, Sec. 3), after
    checking (tie_free) that the case has no closest-segment near-tie."""
    if tie_free:
        _assert_tie_free(O, prob, R, o)
    return O.control_grad(prob, prob["params0"], R, o, spc)


@pytest.mark.parametrize("name", ["star20_128", "star20_200_t16", "mixed60_full"])
def test_fit_terms_and_point_gradient_match_oracle(env, name):
    O, Collage = env
    prob, kw, grid, tile = _case(name)
    g, o = U.paired(**kw)
    col = Collage(prob, level_res=[grid], tile=tile, fit_controls=1, **g)
    terms, _ = col.loss_backward()
    dp = col.control_grad().cpu().numpy()
    # the 60-element case holds near-ties inside its small blobs (128 segments of ~0.1 px: an
    # interior pixel has many nearly equal distances) where the two candidates' normals differ
    # by 0.05 rad; the star fits are tie-free
    ref, rterms = _ref_grad(O, prob, grid, o, tie_free=name != "mixed60_full")
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
    probs = [_generic(W.fit_problem(2, n_cubics=12, grid=96), 96, 1),
             _generic(W.fit_problem(3, n_cubics=20, grid=160), 160, 0),
             _generic(W.fit_problem(4, n_cubics=8, grid=128), 128, 0)]
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
        assert err.max() <= U.GRAD_RTOL, (i, err.max())
        k += n
    assert k == len(dp)
    col.close()
