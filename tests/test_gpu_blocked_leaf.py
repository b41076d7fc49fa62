"""The blocked TSQR leaf (TSQR variant 3: 256-row blocks held in tensor memory, 32-column panels,
compact-WY trailing updates; FP32) forced for every pass, against the FP64 oracle.

Bars as for the other mixed kernels: energy density within 1e-6 of the oracle after every step
(FP32 and FP64 storage of the merged core), tt_round reconstruction within 1e-6 with the oracle's
ranks (the cases keep the oracle's tail far from the threshold).  Shapes cover passes of 9 to 224
columns (the widest the kernel takes: a 3-D transport sum at rank 32), row counts that are not
multiples of the 256-row block, fewer rows than columns, and leaf caps below the SM count (so
that a leaf takes several blocks)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import naive_tt as nt, problem  # noqa: E402
from paper_2602_00290_gb300.workloads import cube_config, plane_config1, random_tt  # noqa: E402
from tie import assert_tie_free  # noqa: E402


@pytest.fixture(scope="module")
def tt():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2602_00290_gb300 as mod
    return mod


def fro_rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _force(ctx, leaves, prec="mixed"):
    for n in range(1, 257):
        ctx.set_tsqr(prec, n, "blocked", leaves)


def _plane(**kw):
    args = dict(nx=12, ny=10, G=5, ntheta=4, nphi=8, rmax=8, tol=1e-6)
    args.update(kw)
    return plane_config1(**args)


CASES = {
    "plane_r8": (_plane(), 0),
    "plane_r16_inflow_3_leaves": (_plane(nx=14, ny=12, G=6, ntheta=8, nphi=16, rmax=16).with_(
        inflow_temperature=(0.9, None, 0.6, None, None, None)), 3),
    "plane_r32": (_plane(nx=20, ny=16, G=8, ntheta=8, nphi=16, rmax=32), 0),
    "rusanov_r12": (_plane(rmax=12).with_(flux="rusanov"), 2),
    "tiny_2x2_g2": (plane_config1(nx=2, ny=2, G=2, ntheta=4, nphi=8, rmax=8, tol=1e-6), 0),
    "cube_r8_inflow": (cube_config().with_(inflow_temperature=(0.9, None, None, None, 0.6, None)), 0),
    "cube_r32_224_columns": (cube_config(nx=6, ny=5, nz=4, G=3, ntheta=6, nphi=12, rmax=32), 1),
}


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("name", list(CASES))
def test_blocked_leaf_steps_match_oracle(tt, name, dtype):
    wl, leaves = CASES[name]
    ctx = tt.Context(0)
    _force(ctx, leaves)
    coef = problem.build(wl)
    plan = tt.Plan(ctx, wl)
    x = tt.initial_state(plan, [wl.rmax, wl.rmax], dtype)
    ref = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    errs = []
    for _ in range(5):
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, "mixed")
        ref = nt.step(ref, coef, wl.tol, wl.rmax)
        ctx.sync()
        E = tt.tt_energy_density(ctx, plan, x).cpu().numpy()
        errs.append(fro_rel(E, nt.energy_density_rows(ref, coef)))
    assert max(errs) <= 1e-6, errs
    R1 = (wl.ndim * 2 + 1) * wl.rmax + (0 if name.find("inflow") < 0 else 2)
    assert ctx.get_tsqr("mixed", R1)[0] == "blocked"
    plan.close()
    ctx.close()


@pytest.mark.parametrize("n,r,leaves", [([2333, 5, 9], [6, 4], 0), ([700, 6, 9], [5, 4], 2), ([300, 16, 32], [20, 12], 1)])
def test_blocked_leaf_round_matches_oracle(tt, n, r, leaves):
    a = nt.add_many([nt.scale(random_tt(n, r, seed=50 + i), 10.0 ** -i) for i in range(3)])
    info = {}
    want = nt.round_tt(a, 1e-5, 40, info)
    assert_tie_free(info, tie=0.01)
    ctx = tt.Context(0)
    _force(ctx, leaves)
    x = tt.TT.from_cores(a, rcap=[max(40, 3 * r[0]), max(40, 3 * r[1])], dtype="f32")
    tt.tt_round(ctx, x, 1e-5, 40, "mixed")
    ctx.sync()
    assert x.ranks() == nt.ranks(want)
    assert fro_rel(nt.full(x.to_cores()), nt.full(want)) < 1e-5
    ctx.close()
