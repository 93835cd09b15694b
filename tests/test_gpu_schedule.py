"""The level schedule (Sec. 4.3, coarse to fine) captured as one CUDA graph, through the C ABI.

collage_run_schedule with use_graphs = 1 runs every level's switch and iterations from one graph
whose loops are decided on the device; with use_graphs = 0 the host sets each level and steps it.
In deterministic mode the two must agree bit for bit, also when the graph meets a bin overflow
part-way (provoked from the host: params enlarged behind the captured capacity) and the run
resumes on the host path from the iteration that did not complete."""
import numpy as np
import pytest
import torch

from paper_2406_04008_gb300 import workloads as W
from tests import _util as U

pytestmark = pytest.mark.gpu

LEVELS = dict(n_levels=3, level_res=[64, 128, 256], level_iters=[6, 5, 4])


@pytest.fixture(scope="module")
def Collage():
    from paper_2406_04008_gb300 import build
    build.build()
    from paper_2406_04008_gb300.collage import Collage as C
    return C


def _kw(**extra):
    g, _ = U.paired(pad_px=2.0)
    g.update(LEVELS)
    g.update(deterministic=1, tile=8)
    g.update(extra)
    return g


def _prob():
    return W.config_problem(3, n_elems=120, grid=256)


def test_graph_schedule_equals_host_schedule(Collage):
    prob = _prob()
    a = Collage(prob, use_graphs=1, **_kw())
    b = Collage(prob, use_graphs=0, **_kw())
    for _ in range(2):  # the second run replays the cached graph from level 0 again
        a.set_level(0)
        b.set_level(0)
        a.run_schedule()
        b.run_schedule()
        assert a.info()["level"] == b.info()["level"] == 2
        sa, stepa, _ = a.get_state()
        sb, stepb, _ = b.get_state()
        assert stepa == stepb
        assert torch.equal(sa, sb)
        assert torch.equal(a.loss(), b.loss())
    assert stepa == 30
    # stepping on after the schedule (the last level's one-iteration graph)
    a.step(2)
    b.step(2)
    assert torch.equal(a.get_params(), b.get_params())
    a.close()
    b.close()


def test_graph_schedule_from_a_later_level(Collage):
    prob = _prob()
    a = Collage(prob, use_graphs=1, **_kw())
    b = Collage(prob, use_graphs=0, **_kw())
    for c in (a, b):
        c.set_level(1)
        c.run_schedule()
    _, step, _ = a.get_state()
    assert step == 9
    assert torch.equal(a.get_state()[0], b.get_state()[0])
    a.close()
    b.close()


def test_overflow_inside_the_graph_resumes_exactly(Collage):
    prob = _prob()
    q6 = torch.tensor(prob["params0"], device="cuda").view(-1, 4).clone()
    q6[:, 3] *= 6.0  # elements 6x larger: far more (tile, element) pairs than captured for
    n = q6.shape[0]
    state = torch.cat([q6.reshape(-1), torch.zeros(8 * n, device="cuda")])
    a = Collage(prob, use_graphs=1, **_kw())
    a.run_schedule()  # captures the schedule for the original sizes
    cap0 = a.info()["pair_capacity"]
    a.set_state(state, 0, 0)  # level 0, step 0, enlarged params: the cached graph is replayed
    a.run_schedule()
    assert a.info()["pair_capacity"] > cap0  # an overflow was met and the buffers regrown
    _, step, level = a.get_state()
    assert step == 15 and level == 2
    prob6 = dict(prob)
    prob6["params0"] = q6.reshape(-1).cpu().numpy()
    b = Collage(prob6, use_graphs=0, **_kw())
    b.run_schedule()
    assert torch.equal(a.get_state()[0], b.get_state()[0])
    assert torch.equal(a.loss(), b.loss())
    a.close()
    b.close()


def test_schedule_with_a_level_of_zero_iterations(Collage):
    prob = _prob()
    kw = _kw()
    kw["level_iters"] = [3, 0, 2]
    a = Collage(prob, use_graphs=1, **kw)
    b = Collage(prob, use_graphs=0, **kw)
    a.run_schedule()
    b.run_schedule()
    _, step, level = a.get_state()
    assert step == 5 and level == 2
    assert torch.equal(a.get_state()[0], b.get_state()[0])
    a.close()
    b.close()


def test_schedule_bodies_of_several_iterations(Collage):
    # 12 iterations: two passes of a 6-iteration body; 11 (prime): eleven passes of one; 4: one pass
    prob = _prob()
    kw = _kw()
    kw["level_iters"] = [12, 11, 4]
    a = Collage(prob, use_graphs=1, **kw)
    b = Collage(prob, use_graphs=0, **kw)
    a.run_schedule()
    b.run_schedule()
    _, step, level = a.get_state()
    assert step == 27 and level == 2
    assert torch.equal(a.get_state()[0], b.get_state()[0])
    assert torch.equal(a.loss(), b.loss())
    a.close()
    b.close()
