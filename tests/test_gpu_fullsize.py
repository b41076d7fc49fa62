"""One tt_step at the full bench size (128 x 128 cells, G = 64, 16 x 32 ordinates, r <= 32,
tol 1e-6: N_Z = 1,048,576 rows, a 160-column transport sum) with the TSQR kernels the bench
runs (pinned to the autotuner's choice for this workload), against one step of the oracle from
the same state.

The state is a seeded random rank-32 TT (not produced by the CUDA path) whose bonds are graded
geometrically, so that the singular values at every bond are well separated; the new ranks reach
the cap r = 32 as in the bench's saturated steps (the oracle's relative gap at the cut is 0.03).
The oracle step (explicit transport sum, LAPACK QR and SVD) takes tens of seconds on the host,
so it runs once for all cases.  Compared: the new ranks, every row's energy density, and the
full angular rows I[k, :] at 2048 sampled rows k.  Tolerances: FP64 1e-10 relative; mixed 1e-6
in energy density (FP32 state or FP64 state).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import naive_tt as nt, problem  # noqa: E402
from paper_2602_00290_gb300.workloads import plane_config1, random_tt  # noqa: E402

TIE = 1e-9
PINNED = {"fp64": {"transport": ("column", 304), "source": ("rowsplit", 304)},
          "mixed": {"transport": ("column_dense", 608), "source": ("rowsplit", 456)},
          "mixed_3xtf32": {"transport": ("column_dense", 608), "source": ("rowsplit", 456)},
          "mixed_blocked": {"transport": ("blocked", 152), "source": ("blocked", 152)}}


@pytest.fixture(scope="module")
def tt():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2602_00290_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def case():
    wl = plane_config1()
    coef = problem.build(wl)
    a = random_tt([wl.nrow, wl.ntheta, wl.nphi], [wl.rmax, wl.rmax], seed=21)
    a[0] = a[0] * (0.55 ** np.arange(wl.rmax))[None, None, :]
    a[1] = a[1] * (0.7 ** np.arange(wl.rmax))[None, None, :]
    info = {}
    ref = nt.step(a, coef, wl.tol, wl.rmax, info)
    rows = np.sort(np.random.default_rng(5).choice(wl.nrow, 2048, replace=False))
    return wl, coef, a, ref, info, rows


def sampled_rows(cores, rows):
    """I[k, :] for the sampled rows k: Z[k, :] times the right part of the angular cores."""
    z = np.asarray(cores[0])[0][rows]                        # (len(rows), r1)
    right = np.einsum("alb,bp->alp", np.asarray(cores[1]), np.asarray(cores[2])[:, :, 0])
    return z @ right.reshape(right.shape[0], -1)


@pytest.mark.parametrize("prec,dtype", [("fp64", "f64"), ("mixed", "f32"), ("mixed", "f64"), ("mixed_3xtf32", "f32"),
                                        ("mixed_blocked", "f32")])
def test_full_size_step_matches_oracle(tt, case, prec, dtype):
    wl, coef, a, ref, info, rows = case
    ctx = tt.Context(0)
    K1 = wl.rmax
    pins = PINNED[prec]
    if prec == "mixed_blocked":  # the mixed step with the blocked TSQR leaf over both sums
        prec = "mixed"
    for role, ncap in (("transport", 5 * K1), ("source", K1 + 1)):
        variant, leaves = pins[role]
        ctx.set_tsqr(prec, ncap, variant, leaves)
    plan = tt.Plan(ctx, wl)
    x = tt.TT.from_cores(a, rcap=[K1, K1], dtype=dtype)
    tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, prec)
    ctx.sync()
    E = tt.tt_energy_density(ctx, plan, x).cpu().numpy()
    Er = nt.energy_density_rows(ref, coef)
    if prec == "fp64":
        gaps = [b["gap"] for k in ("transport_round", "source_round") for b in info[k]["bonds"]]
        assert min(gaps) > TIE  # the graded state leaves no rank decision near a tie
        assert x.ranks() == nt.ranks(ref)
        got = sampled_rows(x.to_cores(), rows)
        want = sampled_rows(ref, rows)
        assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want))
        assert np.max(np.abs(E - Er)) <= 1e-10 * np.max(np.abs(Er))
    else:
        assert np.linalg.norm(E - Er) <= 1e-6 * np.linalg.norm(Er)
    plan.close()
    ctx.close()
