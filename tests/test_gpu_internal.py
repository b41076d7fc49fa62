"""Internal delta-ranks of the merged core on the GPU (tt_internal_ranks, Sec. 5.2) against the
oracle's SVDs of the two reshapes, on rounded states of the plane workload.  Singular values
agree to 1e-8 relative to the largest (the GPU takes them from FP64 Gram matrices); ranks agree
wherever the oracle's tail is not within 1e-3 (relative) of the threshold."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import naive_tt as nt, problem  # noqa: E402
from paper_2602_00290_gb300.workloads import plane_config1  # noqa: E402


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


def _tail_gap(S, delta):
    S = np.asarray(S)
    tot = np.sqrt(np.sum(S ** 2))
    t = np.sqrt(np.cumsum((S ** 2)[::-1])[::-1])
    return np.min(np.abs(t - delta * tot)) / (delta * tot)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_internal_ranks_match_oracle(tt, ctx, dtype):
    wl = plane_config1(nx=16, ny=12, G=8, ntheta=4, nphi=8, rmax=10, tol=1e-6)
    coef = problem.build(wl)
    plan = tt.Plan(ctx, wl)
    x = tt.initial_state(plan, [wl.rmax, wl.rmax], dtype)
    for _ in range(4):
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, "fp64" if dtype == "f64" else "mixed")
    ctx.sync()
    cores = x.to_cores()
    Z = cores[0][0]
    for delta in (1e-2, 1e-4, 1e-6):
        r1, r1x, snu, sx = tt.tt_internal_ranks(ctx, plan, x, delta)
        o1, o1x, onu, ox = nt.internal_ranks(Z, wl.ngroup, delta)
        assert np.allclose(snu[:len(onu)], onu, rtol=0, atol=1e-8 * onu[0])
        k = min(len(sx), len(ox))
        assert np.allclose(sx[:k], ox[:k], rtol=0, atol=1e-8 * ox[0])
        if _tail_gap(onu, delta) > 1e-3:
            assert r1 == o1, (delta, r1, o1)
        if _tail_gap(ox, delta) > 1e-3:
            assert r1x == o1x, (delta, r1x, o1x)
