"""tt_dot_noalloc (the allocation-free inner product over a fixed device scratch array) against
tt_dot through the C ABI, on two calls in a row, with the 1e-13 relative tolerance the other
exact-operation parity tests use.  Collected last so that it also runs after every other
test has used the library on this device."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_00290_gb300.workloads import random_tt  # noqa: E402

TOL = 1e-13


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


CASES = [
    # modes, ranks of x, ranks of y, capacities of x, capacities of y, storage dtype
    ([50, 6, 7], [3, 4], [2, 5], [5, 6], [3, 5], "f64"),
    ([37, 9], [4], [3], [6], [4], "f64"),
    ([4100, 16, 32], [9, 7], [12, 5], [12, 8], [16, 6], "f32"),
    # 2^16 merged rows at capacity 128 x 128: the default chunking (64 chunks of 1024 rows)
    # needs more partials than the scratch holds, so the call uses 29 longer chunks
    ([65536, 8], [100], [90], [128], [128], "f64"),
]


def make(tt, n, r, rcap, seed, dtype):
    return tt.TT.from_cores(random_tt(n, r, seed=seed), rcap=rcap, dtype=dtype)


@pytest.mark.parametrize("n,rx,ry,cx,cy,dtype", CASES)
def test_noalloc_dot_matches_tt_dot_twice(tt, ctx, n, rx, ry, cx, cy, dtype):
    x = make(tt, n, rx, cx, 11, dtype)
    y = make(tt, n, ry, cy, 12, dtype)
    want = tt.tt_dot(ctx, x, y).item()
    scale = max(abs(want), float(torch.sqrt(tt.tt_dot(ctx, x, x) * tt.tt_dot(ctx, y, y)).item()))
    stream = torch.cuda.current_stream()
    for _ in range(2):
        out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        tt.tt_dot_noalloc(stream, x, y, out)
        got = out.item()
        assert abs(got - want) <= TOL * scale, (got, want)


def test_noalloc_dot_after_a_different_shape(tt, ctx):
    # the shared scratch keeps the previous call's contents: a call with another shape in
    # between must not change the result of the next one
    a = make(tt, [300, 5, 6], [3, 2], [4, 3], 21, "f64")
    b = make(tt, [300, 5, 6], [2, 3], [2, 4], 22, "f64")
    big_x = make(tt, [2000, 24], [20], [20], 23, "f64")
    big_y = make(tt, [2000, 24], [19], [20], 24, "f64")
    want = tt.tt_dot(ctx, a, b).item()
    stream = torch.cuda.current_stream()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    tt.tt_dot_noalloc(stream, a, b, out)
    first = out.item()
    tt.tt_dot_noalloc(stream, big_x, big_y, out)
    tt.tt_dot_noalloc(stream, a, b, out)
    second = out.item()
    scale = max(abs(want), 1.0)
    assert abs(first - want) <= TOL * scale and abs(second - want) <= TOL * scale


def test_noalloc_dot_rejects_oversized_ranks(tt):
    # capacity 512 x 512 needs more than 3 * 512^2 doubles of scratch: above the 2^19 it has
    x = make(tt, [3, 4], [512], [512], 31, "f64")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(tt.TTError) as e:
        tt.tt_dot_noalloc(torch.cuda.current_stream(), x, x, out)
    assert e.value.status == tt.TT_ERR_WORKSPACE
    assert out.item() == 0.0
