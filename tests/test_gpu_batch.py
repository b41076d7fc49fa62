"""Batched stepping (tt_batch_*) of independent, unevenly shaped problems: against the same
problems stepped one by one through tt_step, against the CPU oracle, and graph replay.

Shapes follow the batched workload (Nx = Ny, G, ordinates and r_max drawn per problem, Planck
inflow on the x- face at T_b ~ U[0.1, 1]) scaled down 8x so that the oracle runs in seconds.
Tolerances: FP64 as the single-problem parity tests (1e-10, identical ranks unless the oracle's
tail is within 1e-9 of the threshold); mixed 1e-6 in energy density.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import naive_tt as nt, problem  # noqa: E402
from paper_2602_00290_gb300.workloads import batch_config3  # noqa: E402
from tie import STEP_KEYS, assert_tie_free  # noqa: E402



@pytest.fixture(scope="module")
def tt():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2602_00290_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def ctx(tt):
    return tt.Context(0)


@pytest.fixture
def batches():
    made = []
    yield made
    for b in made:
        b.close()


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) / max(float(np.max(np.abs(np.asarray(b)))), 1e-300)


def _setup(tt, ctx, wls, dtype):
    plans = [tt.Plan(ctx, wl) for wl in wls]
    states = [tt.initial_state(p, [wl.rmax, wl.rmax], dtype) for p, wl in zip(plans, wls)]
    return plans, states


def test_batch_fp64_matches_single_steps_and_oracle(tt, ctx, batches):
    wls = batch_config3(8, seed=3, scale=8)
    plans, states = _setup(tt, ctx, wls, "f64")
    batch = tt.Batch(ctx, plans, states, [w.tol for w in wls], [w.rmax for w in wls], "fp64", nstreams=4)
    batches.append(batch)
    singles = [tt.initial_state(p, [w.rmax, w.rmax], "f64") for p, w in zip(plans, wls)]
    coefs = [problem.build(w) for w in wls]
    refs = [nt.initial_tt(problem.initial_rows(w, c), c) for w, c in zip(wls, coefs)]
    for step in range(3):
        batch.step(1)
        assert batch.sync() == [0] * len(wls)
        for i, (p, w, c) in enumerate(zip(plans, wls, coefs)):
            tt.tt_step(ctx, p, singles[i], w.tol, w.rmax, "fp64")
            info = {}
            refs[i] = nt.step(refs[i], c, w.tol, w.rmax, info)
            ctx.sync()
            xb = nt.to_dense_rows(states[i].to_cores())
            assert states[i].ranks() == singles[i].ranks(), (step, i)
            assert rel(xb, nt.to_dense_rows(singles[i].to_cores())) < 1e-12, (step, i)
            assert_tie_free(info, STEP_KEYS, where=f"step {step}, problem {i}")
            assert states[i].ranks() == nt.ranks(refs[i]), (step, i)
            assert rel(xb, nt.to_dense_rows(refs[i])) < 1e-10, (step, i)
    assert batch.info()["launches_per_step"] > 0
    batch.close()


def test_batch_mixed_energy_within_1e6(tt, ctx, batches):
    wls = batch_config3(6, seed=5, scale=8)
    for dtype in ("f32", "f64"):
        plans, states = _setup(tt, ctx, wls, dtype)
        batch = tt.Batch(ctx, plans, states, [w.tol for w in wls], [w.rmax for w in wls], "mixed")
        batches.append(batch)
        coefs = [problem.build(w) for w in wls]
        refs = [nt.initial_tt(problem.initial_rows(w, c), c) for w, c in zip(wls, coefs)]
        for step in range(3):
            batch.step(1)
            batch.sync()
            for i, (p, w, c) in enumerate(zip(plans, wls, coefs)):
                refs[i] = nt.step(refs[i], c, w.tol, w.rmax)
                E = tt.tt_energy_density(ctx, p, states[i]).cpu().numpy()
                Er = nt.energy_density_rows(refs[i], c)
                assert np.linalg.norm(E - Er) <= 1e-6 * np.linalg.norm(Er), (dtype, step, i)
        batch.close()


def test_batch_graph_replay_is_deterministic(tt, ctx, batches):
    """nsteps replays in one call give bit-identical states to one-step calls."""
    wls = batch_config3(5, seed=7, scale=8)
    out = []
    for calls in ([3], [1, 1, 1]):
        plans, states = _setup(tt, ctx, wls, "f32")
        batch = tt.Batch(ctx, plans, states, [w.tol for w in wls], [w.rmax for w in wls], "mixed", nstreams=3)
        batches.append(batch)
        for n in calls:
            batch.step(n)
        batch.sync()
        out.append([(s.ranks(), [c.cpu().numpy().copy() for c in s.cores]) for s in states])
        batch.close()
    for (ra, ca), (rb, cb) in zip(*out):
        assert ra == rb
        for a, b in zip(ca, cb):
            assert np.array_equal(a, b)


def test_batch_rejects_bad_arguments(tt, ctx):
    wls = batch_config3(2, seed=9, scale=8)
    plans, states = _setup(tt, ctx, wls, "f64")
    with pytest.raises(tt.TTError) as e:
        tt.Batch(ctx, plans, states, [w.tol for w in wls], [w.rmax + 1 for w in wls], "fp64")
    assert e.value.status == tt.TT_ERR_CAPACITY
    with pytest.raises(tt.TTError) as e:
        tt.Batch(ctx, plans[::-1], states, [w.tol for w in wls], [w.rmax for w in wls], "fp64")
    assert e.value.status == tt.TT_ERR_SHAPE
