"""The autotuner (collage_autotune / collage_get_tuning) through the C ABI: it picks one of its
candidates, never slower than the defaults it timed, changes no params, gives the same results as a
handle configured by hand the same way, and a second handle with the same key takes the cached
choice without a search."""
import numpy as np
import pytest
import torch

from paper_2406_04008_gb300 import workloads as W
from tests import _util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Collage():
    from paper_2406_04008_gb300 import build
    build.build()
    from paper_2406_04008_gb300.collage import Collage as C
    return C


def _kw():
    g, _ = U.paired(pad_px=2.0)
    g.update(level_res=[512], deterministic=1, persistent=1, use_graphs=1)
    return g


def test_autotune_choice_cache_and_results(Collage, oracle_mod):
    # blobs of 10-30 px radius: their gradients are well conditioned (a blob of a few pixels, whose
    # 128 segments are ~0.1 px long, has pixels within rounding of a closest-segment tie, where the
    # derivative is set-valued (reading A15) and its rotation gradient nearly cancels)
    prob = W.config_problem(2, collage_index=9, n_elems=150, grid=512)
    a = Collage(prob, tile=0, **_kw())
    p0 = a.get_params().clone()
    tile, best = a.autotune()
    t = a.tuning()
    assert t["tile"] == tile and tile in (8, 16)
    assert t["emit_threads"] in (128, 256) and t["chunk_px"] in (32, 64)
    for k in ("fwd_grid", "bwd_grid", "comp_grid"):
        assert t[k] in (0.5, 1.0, 2.0)
    assert t["from_cache"] == 0 and t["trials"] >= 8
    assert 0 < t["best_ms"] <= t["default_ms"]
    assert best == pytest.approx(t["best_ms"])
    assert torch.equal(a.get_params(), p0)  # the search steps nothing
    ta, ga = a.loss_backward()
    # a second handle of the same key: the cached choice, no search
    b = Collage(prob, tile=0, **_kw())
    b.autotune()
    tb = b.tuning()
    assert tb["from_cache"] == 1 and tb["trials"] == 0
    for k in ("tile", "emit_threads", "chunk_px", "fwd_grid", "bwd_grid", "comp_grid"):
        assert tb[k] == t[k]
    tb_, gb = b.loss_backward()
    assert torch.equal(ta, tb_) and torch.equal(ga, gb)
    # a handle with the chosen tile and the default launch parameters: the same numbers (the grids
    # and block sizes change no result in deterministic mode)
    c = Collage(prob, tile=tile, **_kw())
    tc, gc = c.loss_backward()
    assert torch.equal(ta, tc) and torch.equal(ga, gc)
    # and they are the oracle's
    o = U.paired(pad_px=2.0)[1]
    ref = oracle_mod.Scene(prob).eval(prob["params0"].astype(np.float64), 512, o)
    U.check_terms(ta.cpu().numpy()[0], ref["terms"], 512, (o.alpha, o.beta, o.gamma, o.delta))
    U.check_grad(ga.cpu().numpy(), ref["grad_a"])
    for h in (a, b, c):
        h.close()


def test_set_tuning_applies_a_saved_choice(Collage):
    # in deterministic mode the launch parameters change no result at a given tile (the tile sets
    # the order of the per-tile loss sums); values outside the search are refused and leave the
    # handle as it was
    prob = W.config_problem(2, collage_index=4, n_elems=60, grid=256)
    kw = _kw()
    kw["level_res"] = [256]
    ref = {}
    for T in (8, 16):
        h = Collage(prob, tile=T, **kw)
        ref[T] = h.loss_backward()
        h.close()
    a = Collage(prob, tile=16, **kw)
    for choice in (dict(tile=8, emit_threads=256, chunk_px=32, fwd_grid=0.5, bwd_grid=2.0, comp_grid=2.0),
                   dict(tile=16, emit_threads=256, chunk_px=64, fwd_grid=2.0, bwd_grid=0.5, comp_grid=0.5),
                   dict(tile=8, emit_threads=128, chunk_px=64, fwd_grid=1.0, bwd_grid=1.0, comp_grid=1.0),
                   dict(tile=16, emit_threads=128, chunk_px=32, fwd_grid=0.5, bwd_grid=1.0, comp_grid=2.0)):
        a.set_tuning(**choice)
        t = a.tuning()
        for k, v in choice.items():
            assert t[k] == v, (k, t[k], v)
        assert t["best_ms"] == 0 and t["trials"] == 0
        tc, gc = a.loss_backward()
        t0, g0 = ref[choice["tile"]]
        assert torch.equal(t0, tc) and torch.equal(g0, gc), choice
    before = a.tuning()
    for bad in (dict(tile=12), dict(emit_threads=192), dict(chunk_px=48), dict(fwd_grid=3.0)):
        with pytest.raises(Exception):
            a.set_tuning(**bad)
        assert a.tuning() == before
    a.close()
