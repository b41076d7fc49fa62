"""tt_step replayed as a captured CUDA graph (tt_context_set_graphs) against eager steps: the same
kernels run in the same order, so states must agree bit for bit, across changes of the step's
arguments, of the TSQR kernel table and of the precision, with launch counters that count each
replay, and with kernel timing (which runs eagerly)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_00290_gb300.workloads import cube_config, plane_config1, slab_config0  # noqa: E402


@pytest.fixture(scope="module")
def tt():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2602_00290_gb300 as mod
    return mod


def _pair(tt, wl, dtype, ranks):
    out = []
    for graphs in (False, True):
        ctx = tt.Context(0)
        ctx.set_graphs(graphs)
        plan = tt.Plan(ctx, wl)
        out.append((ctx, plan, tt.initial_state(plan, ranks, dtype)))
    return out


def _same(a, b):
    assert a.ranks() == b.ranks()
    for ca, cb in zip(a.to_cores(), b.to_cores()):
        assert np.array_equal(ca, cb)


def _close(pair):
    for ctx, plan, _ in pair:
        plan.close()
        ctx.close()


PLANE = plane_config1(nx=12, ny=10, G=5, ntheta=4, nphi=8, rmax=8, tol=1e-6)


@pytest.mark.parametrize("wl,prec,dtype", [(PLANE, "mixed", "f32"), (PLANE, "mixed", "f64"), (PLANE, "fp64", "f64"),
                                           (slab_config0(), "fp64", "f64"), (slab_config0(), "mixed", "f32"),
                                           (cube_config(), "mixed", "f32")],
                         ids=["plane-mixed-f32", "plane-mixed-f64", "plane-fp64", "slab-fp64", "slab-mixed",
                              "cube-mixed"])
def test_graph_steps_equal_eager_steps(tt, wl, prec, dtype):
    ranks = [wl.rmax] if wl.ndim == 1 else [wl.rmax, wl.rmax]
    pair = _pair(tt, wl, dtype, ranks)
    for s in range(6):
        for ctx, plan, x in pair:
            tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, prec)
        for ctx, _, _ in pair:
            ctx.sync()
        _same(pair[0][2], pair[1][2])
    # the first step ran eagerly, the second captured the graph, every later one replayed it
    d = pair[1][0].diagnostics()
    assert (d["graph_captures"], d["graph_failures"], d["graph_replays"]) == (1, 0, 5)
    d0 = pair[0][0].diagnostics()
    assert (d0["graph_captures"], d0["graph_replays"]) == (0, 0)
    _close(pair)


def test_graph_follows_argument_and_table_changes(tt):
    wl = PLANE
    pair = _pair(tt, wl, "f32", [wl.rmax, wl.rmax])
    K1 = wl.rmax
    plan_of_steps = [(1e-6, 8, "mixed")] * 3 + [(1e-4, 8, "mixed")] * 2 + [(1e-6, 6, "mixed")] * 2
    for i, (tol, rmax, prec) in enumerate(plan_of_steps):
        if i == 5:  # a new TSQR choice for the transport sum: the graph is captured again
            for ctx, _, _ in pair:
                ctx.set_tsqr(prec, 5 * K1, "rowsplit", 0)
        for ctx, plan, x in pair:
            tt.tt_step(ctx, plan, x, tol, rmax, prec)
        for ctx, _, _ in pair:
            ctx.sync()
        _same(pair[0][2], pair[1][2])
    _close(pair)


def test_graph_replays_are_counted_and_timing_runs_eagerly(tt):
    wl = PLANE
    pair = _pair(tt, wl, "f32", [wl.rmax, wl.rmax])
    counts = []
    for ctx, plan, x in pair:
        ctx.counters(reset=True)
        for _ in range(4):
            tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, "mixed")
        ctx.sync()
        _, launches = ctx.counters(reset=True)
        counts.append(sum(launches.values()))
    assert counts[0] == counts[1] > 0
    # with kernel timing on, the graph context steps eagerly and reports kernel times
    ctx, plan, x = pair[1]
    ctx.set_timing(True)
    tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, "mixed")
    ctx.sync()
    ms, _ = ctx.counters(reset=True)
    ctx.set_timing(False)
    assert ms["tsqr_leaf"] > 0.0
    c0, p0, x0 = pair[0]
    tt.tt_step(c0, p0, x0, wl.tol, wl.rmax, "mixed")
    c0.sync()
    _same(x0, x)
    # and back to replays
    for ctx, plan, x in pair:
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, "mixed")
        ctx.sync()
    _same(pair[0][2], pair[1][2])
    _close(pair)


def test_graph_off_releases_and_steps_eagerly(tt):
    wl = PLANE
    pair = _pair(tt, wl, "f32", [wl.rmax, wl.rmax])
    for k in range(4):
        if k == 2:
            pair[1][0].set_graphs(False)
        for ctx, plan, x in pair:
            tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, "mixed")
            ctx.sync()
        _same(pair[0][2], pair[1][2])
    _close(pair)
