"""Launch geometry of the TSQR over the merged core (tt_tsqr_geometry, a host computation made by
the same functions the launches use) checked on the CPU against the buffers a step sizes and the
shared memory a launch asks for.

Every index the leaf and merge kernels form is restated here from the kernels' own expressions
(packed upper-triangular R, the double-buffered reflector, the two or four reflector scalars, the
row flags), independently of the library's size formulas, and checked to stay inside:
  * leaves x ncap^2 doubles written by the leaves into the first R buffer;
  * every merge level: inputs 2m, 2m+1 < n read from one buffer, outputs m < ceil(n/2) written to the
    other, alternating, for every level of the tree (odd levels copy their last factor);
  * the dynamic shared memory of the leaf and merge launches, with 16-byte vector accesses aligned.
The resident-CTA count per SM is swept over every value the shared memory admits (what the
occupancy query can report), for the bench shapes, ragged and tiny row counts, odd SM counts and
leaf caps.  No GPU is used."""
import math

import pytest

SMEM_PER_SM = 228 * 1024  # shared memory of one SM; each resident CTA also reserves 1 KB


@pytest.fixture(scope="module")
def tt():
    from paper_2602_00290_gb300 import _build
    _build.build()
    import paper_2602_00290_gb300 as mod
    return mod


def tri_elems(n):
    """Packed upper triangle of an n x n factor, padded to a multiple of 4 elements."""
    return (n * (n + 1) // 2 + 3) // 4 * 4


# Column descriptor of the stencil source (int kind, q, ax, w, b; double lam; float lamf; long s):
# 20 bytes of ints, padded to 24, the double to 32, the float to 36, padded to 40, the long to 48.
STENCIL_COL_BYTES = 48


def blocked_touch(ncap):
    """(end byte, vector accesses) of the blocked leaf: column descriptors, packed R, U and C-chunk
    tiles [256][36], W/Y [32][ncap], T [32][33], norm [8] + dot [8][32] + per-warp [8][32] partials,
    row flags [256]; 16-byte vectors on the U and C-chunk rows."""
    off = (STENCIL_COL_BYTES * ncap + 15) // 16 * 16
    R = off
    off += 4 * tri_elems(ncap)
    U = off
    off += 4 * 256 * 36
    C = off
    off += 4 * 256 * 36
    off += 4 * 32 * ncap + 4 * 32 * 33 + 4 * (8 + 8 * 32 + 8 * 32) + 4 * 256
    vec = [(U + 4 * (t * 36 + c), 16) for t in range(256) for c in range(0, 32, 4)]
    vec += [(C + 4 * (t * 36 + c), 16) for t in range(256) for c in range(0, 32, 4)]
    assert R % 16 == 0
    return off, vec


def leaf_touch(prec, variant, ncap, br):
    """(end byte, list of (offset, width) vector accesses) of the leaf kernel's shared memory."""
    sz = 8 if prec == "fp64" else 4
    R4 = tri_elems(ncap)
    vec = []
    if variant == 3:
        return blocked_touch(ncap)
    if variant == 1:  # row-split: QS = 4 lanes per column, lane q holds RPT rows at stride SS
        QS, RPT = 4, br // 4
        SS = RPT + 4
        for buf in (0, 1):
            for q in range(QS):
                for i in range(0, RPT, 4):
                    vec.append((sz * (R4 + buf * QS * SS + q * SS + i), 16))
        # highest reflector element, taub[3], then BR row flags (unsigned)
        assert (1 * QS * SS + (QS - 1) * SS + RPT - 1) < 2 * QS * SS
        end = sz * (R4 + 2 * QS * SS + 4) + 4 * br
    else:  # column owner: thread c owns column c, reflector of BR rows, double-buffered
        step = 4 if sz == 4 else 2
        for buf in (0, 1):
            for i in range(0, br, step):
                vec.append((sz * (R4 + buf * br + i), 16))
        end = sz * (R4 + 2 * br + 4) + 4 * br
    # R itself: tri_off(j, n) + (c - j) for j <= c < n reaches n (n + 1) / 2 - 1
    last_r = (ncap - 1) * ncap - ((ncap - 1) * (ncap - 2)) // 2 + 0
    assert last_r == ncap * (ncap + 1) // 2 - 1
    return end, vec


def merge_touch(prec, ncap, threads, rows):
    sz = 8 if prec == "fp64" else 4
    R4 = tri_elems(ncap)
    if threads >= 4 * ncap:  # row-split merge: 64 rows of the second factor at a time, FP32 160
        # from 65 to 160 columns (one block at 160 columns)
        assert rows == (160 if sz == 4 and 64 < ncap <= 160 else 64)
        QS, RPT = 4, rows // 4
        SS = RPT + 4
        vec = [(sz * (R4 + buf * QS * SS + q * SS + i), 16) for buf in (0, 1) for q in range(QS)
               for i in range(0, RPT, 4)]
        return sz * (R4 + 2 * QS * SS + 4), vec
    mbr = 64 if sz == 4 else 32
    return sz * (R4 + 2 * mbr + 4), []


def check(g, prec, variant, ncap, nrows):
    nn = ncap * ncap
    L, rpc, br = g["leaves"], g["rows_per_leaf"], g["block_rows"]
    # every leaf owns whole blocks of rows, the last one the ragged rest, and no leaf is empty
    assert rpc % br == 0 and rpc >= br
    assert L >= 1 and (L - 1) * rpc < nrows <= L * rpc
    # the leaves write L R factors of ncap^2 doubles into the first buffer
    assert L * nn <= g["ws_a_doubles"]
    # merge tree: alternate buffers, read 2m and 2m + 1 < n, write m < ceil(n / 2)
    caps = [g["ws_a_doubles"], g["ws_b_doubles"]]
    n, src, levels = L, 0, 0
    while n > 1:
        m = (n + 1) // 2
        reads_end = n * nn  # input a = 2m (copied alone when 2m + 1 = n) and b = 2m + 1 < n
        writes_end = m * nn
        assert reads_end <= caps[src], (levels, n)
        assert writes_end <= caps[1 - src], (levels, n, m)
        src, n, levels = 1 - src, m, levels + 1
    assert levels == g["merge_levels"] == (math.ceil(math.log2(L)) if L > 1 else 0)
    # threads: a column per thread (column owner) or per four lanes (row-split), whole warps
    t = g["leaf_threads"]
    assert t % 32 == 0
    if g["variant"] == 3:  # blocked: a row per thread, one CTA per SM (the block's tensor memory)
        assert t == 256 and br == 256 and prec == "mixed" and ncap <= 224
        assert L <= g["leaves_cap_sms"]
    else:
        want = 4 * ncap if g["variant"] == 1 else ncap
        assert want <= t < want + 32
    if g["variant"] == 2:
        assert t <= 160 and prec == "mixed"
    # shared memory: every restated access inside the launch's dynamic shared memory, vectors aligned
    end, vec = leaf_touch(prec, g["variant"], ncap, br)
    assert end <= g["leaf_smem"] <= 227 * 1024
    for off, width in vec:
        assert off % width == 0 and off + width <= g["leaf_smem"]
    mend, mvec = merge_touch(prec, ncap, g["merge_threads"], g["merge_rows"])
    assert mend <= g["merge_smem"] <= 227 * 1024
    for off, width in mvec:
        assert off % width == 0 and off + width <= g["merge_smem"]


SHAPES = [
    ("mixed", 160, 1048576),  # bench transport sum: 128 x 128 x 64 rows, (2 d_X + 1) r = 5 x 32 columns
    ("mixed", 33, 1048576),   # bench source sum: r + 1 columns
    ("fp64", 160, 1048576),
    ("fp64", 33, 1048576),
    ("mixed", 160, 589824),   # 96 x 96 x 64 rows
    ("mixed", 224, 7 * 9 * 3),  # 3-D sum wider than the rows
    ("fp64", 24, 1024),       # slab: 64 cells x 16 groups, 3 x 8 columns
    ("mixed", 40, 8),         # 2 x 2 cells, 2 groups: fewer rows than columns
    ("fp64", 40, 1),
    ("mixed", 160, 1048577),  # one ragged row beyond the bench size
    ("fp64", 160, 64 * 152 * 2 + 1),
    ("mixed", 256, 123457),   # the widest pass the TSQR takes
    ("fp64", 224, 4099),      # FP64 R factors of 224 columns still fit a CTA's shared memory
]


@pytest.mark.parametrize("prec,ncap,nrows", SHAPES)
@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("num_sms,max_leaves", [(152, 0), (152, 912), (152, 608), (152, 456), (152, 8), (7, 0),
                                                (3, 5)])
def test_tsqr_geometry_stays_inside_its_buffers(tt, prec, ncap, nrows, variant, num_sms, max_leaves):
    g0 = tt.tsqr_geometry(prec, variant, ncap, nrows, num_sms, 1, max_leaves)
    most = SMEM_PER_SM // (g0["leaf_smem"] + 1024)  # resident CTAs the leaf's shared memory admits
    assert most >= 1
    for per_sm in range(1, min(most, 32) + 1):
        g = tt.tsqr_geometry(prec, variant, ncap, nrows, num_sms, per_sm, max_leaves)
        g["leaves_cap_sms"] = num_sms
        check(g, prec, variant, ncap, nrows)
        if max_leaves > 0:
            assert g["leaves"] <= max_leaves


def test_tsqr_geometry_refuses_what_no_kernel_takes(tt):
    with pytest.raises(tt.TTError) as e:
        tt.tsqr_geometry("mixed", 0, 288, 1000, 152, 1)  # one thread per column: at most 256
    assert e.value.status == tt.TT_ERR_UNSUPPORTED
    with pytest.raises(tt.TTError) as e:
        tt.tsqr_geometry("fp64", 1, 100, 1000, 152, 0)  # row-split leaf with no resident CTA
    assert e.value.status == tt.TT_ERR_UNSUPPORTED
    # variants that cannot take the shape report the kernels that run
    assert tt.tsqr_geometry("fp64", 2, 160, 1000, 152, 1)["variant"] == 0  # dense leaf is FP32 only
    assert tt.tsqr_geometry("mixed", 2, 192, 1000, 152, 1)["variant"] == 0  # more than 160 threads
    assert tt.tsqr_geometry("mixed", 1, 256, 1000, 152, 1)["variant"] == 1  # 1024 lanes: still row-split
    assert tt.tsqr_geometry("mixed", 3, 224, 1000, 152, 1)["variant"] == 3  # blocked: up to 224 columns
    assert tt.tsqr_geometry("mixed", 3, 232, 1000, 152, 1)["variant"] == 0
    assert tt.tsqr_geometry("fp64", 3, 160, 1000, 152, 1)["variant"] == 0  # blocked leaf is FP32 only
    with pytest.raises(tt.TTError) as e:
        tt.tsqr_geometry("fp64", 0, 256, 1000, 152, 1)  # 256 FP64 columns: R beyond 227 KB
    assert e.value.status == tt.TT_ERR_UNSUPPORTED
