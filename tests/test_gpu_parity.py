"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded inputs."""
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


def _run(env, prob, grid, opts, **gpu_extra):
    O, Collage = env
    g, o = U.paired(**opts)
    g.update(gpu_extra)
    g.setdefault("level_res", [grid])
    col = Collage(prob, **g)
    terms, grad = col.loss_backward()
    torch.cuda.synchronize()
    ref = O.Scene(prob).eval(prob["params0"].astype(np.float64), grid, o)
    return col, terms.cpu().numpy()[0], grad.cpu().numpy(), ref, g, o


CASES = ["disks16", "blobs40_ragged", "mixed120_pad2", "open150_force", "mixed120_point_force"]


@pytest.mark.parametrize("name", CASES)
def test_loss_and_gradient_match_oracle(env, name):
    prob, opts, grid = U.small_case(name)
    col, terms, grad, ref, g, o = _run(env, prob, grid, opts)
    weights = (o.alpha, o.beta, o.gamma, o.delta)
    U.check_terms(terms, ref["terms"], grid, weights, use_u=o.gamma != 0)
    U.check_grad(grad, ref["grad_a"])
    col.close()


@pytest.mark.parametrize("tile", [8])
def test_other_tile_sizes_match_oracle(env, tile):
    prob, opts, grid = U.small_case("mixed120_pad2")
    col, terms, grad, ref, g, o = _run(env, prob, grid, opts, tile=tile)
    U.check_terms(terms, ref["terms"], grid, (o.alpha, o.beta, o.gamma, o.delta))
    U.check_grad(grad, ref["grad_a"])
    col.close()


@pytest.mark.parametrize("name", ["disks16", "mixed120_pad2", "open150_force"])
def test_render_matches_oracle_per_pixel(env, name):
    O, Collage = env
    prob, opts, grid = U.small_case(name)
    g, o = U.paired(**opts)
    col = Collage(prob, level_res=[grid], **g)
    bw, tau = col.render()
    ihat, atau, _ = O.Scene(prob).render(prob["params0"].astype(np.float64), grid, o)
    bw = bw.cpu().numpy().reshape(grid, grid)
    tau = tau.cpu().numpy().reshape(grid, grid)
    assert np.abs(bw - ihat).max() <= U.COV_ATOL
    assert np.abs(tau - atau).max() <= U.COV_ATOL
    assert (ihat < 1).sum() > 100  # the case is not trivially empty
    col.close()


@pytest.mark.parametrize("name,tile", [("mixed120_pad2", 16), ("open150_force", 8),
                                       ("blobs40_ragged", 8)])
def test_bins_are_bit_exact(env, name, tile):
    O, Collage = env
    prob, opts, grid = U.small_case(name)
    g, o = U.paired(**opts)
    col = Collage(prob, level_res=[grid], tile=tile, **g)
    col.loss_backward()
    t, e = col.bins()
    rt, re_ = O.Scene(prob).bins(prob["params0"], grid, tile, 1.0, float(o.pad_px))
    assert np.array_equal(t, rt) and np.array_equal(e, re_)
    col.close()


def test_batched_problems_match_oracle_and_bins(env):
    O, Collage = env
    probs = [W.config_problem(4, i, n_elems=n) for i, n in ((0, 60), (1, 25), (2, 90))]
    g, o = U.paired()
    col = Collage(probs, level_res=[1], **g)
    assert col.info()["n_probs"] == 3
    terms, grad = col.loss_backward()
    terms, grad = terms.cpu().numpy(), grad.cpu().numpy()
    t, e = col.bins()
    off, tile_base = 0, 0
    for i, p in enumerate(probs):
        n, res = len(p["kind"]), p["grid"]
        ref = O.Scene(p).eval(p["params0"].astype(np.float64), res, o)
        U.check_terms(terms[i], ref["terms"], res, (o.alpha, o.beta, o.gamma, o.delta))
        U.check_grad(grad[off:off + n], ref["grad_a"])
        rt, re_ = O.Scene(p).bins(p["params0"], res, 16, 1.0, 0.0)
        sel = (e >= off) & (e < off + n)
        assert np.array_equal(t[sel] - tile_base, rt) and np.array_equal(e[sel] - off, re_)
        off += n
        tile_base += ((res + 15) // 16) ** 2
    col.close()


def test_deterministic_mode_is_bitwise_reproducible(env):
    O, Collage = env
    prob, opts, grid = U.small_case("mixed120_pad2")
    g, o = U.paired(**opts)
    outs = []
    for _ in range(2):
        col = Collage(prob, level_res=[grid], deterministic=1, **g)
        terms, grad = col.loss_backward()
        outs.append((terms.cpu().numpy().copy(), grad.cpu().numpy().copy()))
        col.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    col = Collage(prob, level_res=[grid], deterministic=0, **g)
    terms, grad = col.loss_backward()
    assert np.array_equal(terms.cpu().numpy(), outs[0][0])
    np.testing.assert_allclose(grad.cpu().numpy(), outs[0][1], rtol=1e-4,
                               atol=1e-5 * np.abs(outs[0][1]).max())
    col.close()


def test_graph_replay_equals_eager_launches(env):
    O, Collage = env
    prob, opts, grid = U.small_case("mixed120_pad2")
    g, o = U.paired(**opts)
    res = []
    for graphs in (0, 1):
        col = Collage(prob, level_res=[grid], deterministic=1, use_graphs=graphs, **g)
        col.step(7)
        res.append((col.get_params().cpu().numpy().copy(), col.loss().cpu().numpy().copy()))
        col.close()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


@pytest.mark.parametrize("graphs", [0, 1])
def test_overlapped_launches_equal_serialised_launches(env, graphs):
    O, Collage = env
    prob, opts, grid = U.small_case("mixed120_pad2")
    g, o = U.paired(**opts)
    res = []
    for pdl in (0, 1):
        col = Collage(prob, level_res=[grid], deterministic=1, use_graphs=graphs,
                      overlap_launches=pdl, **g)
        col.step(5)
        terms, grad = col.loss_backward()
        res.append((col.get_params().cpu().numpy().copy(), terms.cpu().numpy().copy(),
                    grad.cpu().numpy().copy()))
        col.close()
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)


def test_async_steps_equal_synchronous_steps(env):
    O, Collage = env
    prob, opts, grid = U.small_case("mixed120_pad2")
    g, o = U.paired(**opts)
    res = []
    for mode in ("sync", "async"):
        col = Collage(prob, level_res=[grid], deterministic=1, **g)
        if mode == "sync":
            col.step(6)
        else:
            for _ in range(6):
                col.step_async(1)
            col.sync()
        _, step, _ = col.get_state()
        assert step == 6
        res.append((col.get_params().cpu().numpy().copy(), col.loss().cpu().numpy().copy()))
        col.close()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_batched_equals_sequential_bitwise(env):
    O, Collage = env
    probs = [W.config_problem(4, i, n_elems=n) for i, n in ((3, 40), (4, 70))]
    g, o = U.paired()
    kw = dict(level_res=[1], deterministic=1, **g)
    col = Collage(probs, **kw)
    col.step(3)
    pb, lb = col.get_params().cpu().numpy(), col.loss().cpu().numpy()
    col.close()
    off = 0
    for i, p in enumerate(probs):
        c1 = Collage(p, **kw)
        c1.step(3)
        n = len(p["kind"])
        assert np.array_equal(c1.get_params().cpu().numpy(), pb[off:off + n])
        assert np.array_equal(c1.loss().cpu().numpy()[0], lb[i])
        off += n
        c1.close()


def test_one_adam_step_matches_oracle(env):
    O, Collage = env
    prob, opts, grid = U.small_case("disks16")
    g, o = U.paired(**opts)
    col = Collage(prob, level_res=[grid], **g)
    col.step(1)
    p1 = col.get_params().cpu().numpy().reshape(-1)
    q0 = prob["params0"].astype(np.float64)
    gr = O.Scene(prob).eval(q0, grid, o)["grad_a"]
    ref, _, _ = O.adam(q0, np.zeros_like(q0), np.zeros_like(q0), gr, 1)
    big = np.abs(gr) > 1e-2 * np.abs(gr).max()
    np.testing.assert_allclose(p1[big], ref[big], atol=2e-6)
    assert np.all(np.abs(p1 - ref) <= 2e-2 + 1e-6)  # first Adam step is at most lr per entry
    col.close()


def test_autograd_function_matches_central_differences(env):
    """Adjoint of the library (through torch.autograd) against FP64 central differences of the
    oracle loss on 20 random elements of a 200-blob star collage.

    With h = 1e-4 (unit coordinates, 0.026 px on this 256^2 grid) a third of the difference
    quotients straddle kinks of the loss (the min(1, B) of the distribution term, the relu of the
    overlap surrogate), and the oracle's own analytic gradient misses them by the same amounts as
    the GPU's; with h = 1e-7 the quotient resolves the local derivative (the oracle's analytic
    gradient meets it to 2e-5) and every component must agree to 1e-3."""
    O, Collage = env
    from paper_2406_04008_gb300.collage import collage_loss
    prob = W.config_problem(2, grid=256)
    g, o = U.paired()
    col = Collage(prob, level_res=[256], **g)
    params = torch.tensor(prob["params0"], device="cuda").view(-1, 4).requires_grad_(True)
    loss = collage_loss(params, col)
    loss.backward()
    grad = params.grad.cpu().numpy()
    sc = O.Scene(prob)
    q0 = prob["params0"].astype(np.float64)
    ref = sc.eval(q0, 256, o)["grad_a"].reshape(-1, 4)
    rng = np.random.default_rng(3)
    picks = rng.choice(len(prob["kind"]), 20, replace=False)
    scale = np.abs(ref).max(0)

    def fd(h):
        out = np.zeros((20, 4))
        for i, e in enumerate(picks):
            for c in range(4):
                qp, qm = q0.copy(), q0.copy()
                qp[4 * e + c] += h
                qm[4 * e + c] -= h
                out[i, c] = (sc.eval(qp, 256, o, grad=False)["terms"][4] -
                             sc.eval(qm, 256, o, grad=False)["terms"][4]) / (2 * h)
        return out

    def rel(a, b):
        return np.abs(a - b) / np.maximum(np.abs(b), 1e-2 * scale)

    gsel, rsel = grad[picks], ref[picks]
    f4 = fd(1e-4)
    assert np.median(rel(gsel, f4)) < 1e-3
    # where the h = 1e-4 quotient disagrees, it disagrees with the oracle's gradient just as much
    np.testing.assert_allclose(rel(gsel, f4), rel(rsel, f4), rtol=1e-2, atol=1e-3)
    assert rel(gsel, fd(1e-7)).max() < 1e-3
    col.close()


@pytest.mark.slow
def test_full_size_headline_level_matches_oracle(env):
    """1000 mixed elements at the 1024^2 level, in the launch configuration the benchmark times
    (persistent grid, CUDA graph): loss terms, every gradient component, and sampled pixels."""
    O, Collage = env
    prob = W.config_problem(3)
    g, o = U.paired(pad_px=2.0)
    col = Collage(prob, level_res=[128, 256, 512, 1024], n_levels=4, **g)
    col.set_level(3)
    terms, grad = col.loss_backward()
    bw, tau = col.render()
    sc = O.Scene(prob)
    q0 = prob["params0"].astype(np.float64)
    ref = sc.eval(q0, 1024, o)
    U.check_terms(terms.cpu().numpy()[0], ref["terms"], 1024, (o.alpha, o.beta, o.gamma, o.delta))
    U.check_grad(grad.cpu().numpy(), ref["grad_a"])
    ihat, atau, _ = sc.render(q0, 1024, o)
    assert np.abs(bw.cpu().numpy().reshape(1024, 1024) - ihat).max() <= U.COV_ATOL
    assert np.abs(tau.cpu().numpy().reshape(1024, 1024) - atau).max() <= U.COV_ATOL
    col.close()


def _timed_form(Collage, prob, g, grid):
    """A handle in the benchmark's launch configuration (persistent grids, CUDA graph, autotuned
    tile) at one level of `grid`."""
    col = Collage(prob, level_res=[grid], use_graphs=1, persistent=1, tile=0, **g)
    col.autotune()
    return col


@pytest.mark.slow
@pytest.mark.parametrize("cfg,grid,opts", [(1, 128, dict(gamma=0.0)), (2, 512, dict()),
                                           (5, 2048, dict(pad_px=1.0, delta=1e3))])
def test_full_size_configs_match_oracle(env, cfg, grid, opts):
    """The 16-disk, 200-blob and 5000-element open-packing workloads at their full sizes: loss
    terms, every gradient component (atomic and deterministic modes) and the bins."""
    O, Collage = env
    prob = W.config_problem(cfg)
    g, o = U.paired(**opts)
    sc = O.Scene(prob)
    q0 = prob["params0"].astype(np.float64)
    ref = sc.eval(q0, grid, o)
    weights = (o.alpha, o.beta, o.gamma, o.delta)
    for det in (0, 1):
        col = _timed_form(Collage, prob, dict(g, deterministic=det), grid)
        terms, grad = col.loss_backward()
        U.check_terms(terms.cpu().numpy()[0], ref["terms"], grid, weights, use_u=o.gamma != 0)
        U.check_grad(grad.cpu().numpy(), ref["grad_a"])
        if det == 0:
            t, e = col.bins()
            rt, re_ = sc.bins(prob["params0"], grid, col.info()["tile"], 1.0, float(o.pad_px))
            assert np.array_equal(t, rt) and np.array_equal(e, re_)
        col.close()


@pytest.mark.slow
def test_full_batch_of_64_collages_matches_oracle(env):
    """The 64-collage batch (uneven element counts and grids) in one batched handle: per-collage
    loss terms and gradients for a sample of collages including the largest, bins of the whole
    batch against the oracle's rule per collage."""
    O, Collage = env
    probs = [W.config_problem(4, i) for i in range(64)]
    g, o = U.paired()
    col = Collage(probs, level_res=[1], use_graphs=1, persistent=1, tile=0, **g)
    tile, _ = col.autotune()
    terms, grad = col.loss_backward()
    terms, grad = terms.cpu().numpy(), grad.cpu().numpy()
    t, e = col.bins()
    sizes = [len(p["kind"]) * p["grid"] ** 2 for p in probs]
    sample = sorted({0, 17, 40, 63, int(np.argmax(sizes)), int(np.argmin(sizes))})
    off, tile_base = 0, 0
    for i, p in enumerate(probs):
        n, res = len(p["kind"]), p["grid"]
        sc = O.Scene(p)
        rt, re_ = sc.bins(p["params0"], res, tile, 1.0, 0.0)
        sel = (e >= off) & (e < off + n)
        assert np.array_equal(t[sel] - tile_base, rt) and np.array_equal(e[sel] - off, re_)
        if i in sample:
            ref = sc.eval(p["params0"].astype(np.float64), res, o)
            try:
                U.check_terms(terms[i], ref["terms"], res, (o.alpha, o.beta, o.gamma, o.delta))
                U.check_grad(grad[off:off + n], ref["grad_a"])
            except AssertionError as ex:
                raise AssertionError(f"collage {i} (n={n}, grid {res}): {ex}") from None
        off += n
        tile_base += ((res + tile - 1) // tile) ** 2
    col.close()


def _check_metrics(m, ref, amb):
    """GPU metrics against the oracle's: pixel counts may differ only where the oracle's value
    sits within rounding of a threshold (amb such pixels, plus two for overlap decisions)."""
    tol = amb + 2
    for k in range(4):
        assert abs(m[k] - ref[k]) <= tol, (k, m[k], ref[k], tol)
    for k in range(4, 7):
        assert abs(m[k] - ref[k]) <= tol / max(ref[1], 1.0) + 1e-15, (k, m[k], ref[k])
    if np.array_equal(m[:4], ref[:4]):
        assert abs(m[7] - ref[7]) <= 1e-9 * ref[7] + 1e-15, (m[7], ref[7])
    else:
        assert abs(m[7] - ref[7]) <= 1e-3 * ref[7], (m[7], ref[7])


@pytest.mark.parametrize("name", ["disks16", "mixed120_pad2", "open150_force"])
def test_quality_metrics_match_oracle(env, name):
    O, Collage = env
    prob, opts, grid = U.small_case(name)
    g, o = U.paired(**opts)
    col = Collage(prob, level_res=[grid], **g)
    m = col.metrics()[0]
    sc = O.Scene(prob)
    q0 = prob["params0"].astype(np.float64)
    ref = sc.metrics(q0, grid, o)
    ihat, _, covc = sc.render(q0, grid, o)
    amb = int(((np.abs(ihat - 0.5) < 1e-5) | (np.abs(covc - 0.5) < 1e-5)).sum())
    _check_metrics(m, ref, amb)
    assert ref[0] > 0 and ref[1] > 0
    col.close()


@pytest.mark.slow
def test_quality_metrics_full_size(env):
    """The headline level (1000 elements at 1024^2) after a few steps, in the benchmark's launch
    configuration, and the 64-collage batch (every collage)."""
    O, Collage = env
    prob = W.config_problem(3)
    g, o = U.paired(pad_px=2.0)
    col = Collage(prob, level_res=[1024], use_graphs=1, persistent=1, tile=0, **g)
    col.autotune()
    col.step(5)
    q = col.get_params().cpu().numpy().astype(np.float64).reshape(-1)
    m = col.metrics()[0]
    sc = O.Scene(prob)
    ref = sc.metrics(q, 1024, o)
    ihat, _, covc = sc.render(q, 1024, o)
    amb = int(((np.abs(ihat - 0.5) < 1e-5) | (np.abs(covc - 0.5) < 1e-5)).sum())
    _check_metrics(m, ref, amb)
    col.close()
    probs = [W.config_problem(4, i) for i in range(64)]
    gb, ob = U.paired()
    col = Collage(probs, level_res=[1], use_graphs=1, persistent=1, tile=0, **gb)
    mb = col.metrics()
    for i in (0, 23, 63):
        p = probs[i]
        sc = O.Scene(p)
        q0 = p["params0"].astype(np.float64)
        ref = sc.metrics(q0, p["grid"], ob)
        ihat, _, covc = sc.render(q0, p["grid"], ob)
        amb = int(((np.abs(ihat - 0.5) < 1e-5) | (np.abs(covc - 0.5) < 1e-5)).sum())
        _check_metrics(mb[i], ref, amb)
    col.close()
