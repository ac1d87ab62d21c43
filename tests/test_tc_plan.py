"""Host-side launch plans of the tensor-core variants (no GPU): the work list
every CTA role walks — classic units dealt round-robin, then a stream-K tail
of contiguous chunk ranges — covers every K block of every tile exactly once,
a CTA holds at most two pieces, a tile has at most five contributors, and
stream-K is used where it pays (a partial last wave of long-K tiles) and not
where its fixup would cost more than it saves."""
import itertools

import pytest

import paper_2311_03543_b300 as cp

P = 148
TC = [cp.V_TC_TF32, cp.V_TC_BF16, cp.V_TC_FP8, cp.V_SPLIT3, cp.V_SPLIT6, cp.V_SPLIT3_TF32,
      cp.V_SPLIT3_FUSED]


def _items(b, grid, pl):
    """The CTA's work list as the kernel builds it (model of the device code):
    (tile, kb_begin, kb_end, piece)."""
    splits = pl["splits"]
    dp = pl["sk_tile0"] if pl["sk_q"] else pl["tiles"] * splits
    out, i = [], 0
    while True:
        u = b + i * grid
        if u < dp:
            s = u % splits
            out.append((u // splits, s * pl["kb_per_split"],
                        min(pl["num_kb"], (s + 1) * pl["kb_per_split"]), -1))
            i += 1
            continue
        if not pl["sk_q"] or b >= pl["sk_ctas"]:
            return out
        n_dp = (dp - 1 - b) // grid + 1 if b < dp else 0
        k = i - n_dp
        q0 = b * pl["sk_q"] // pl["sk_ctas"]
        q1 = (b + 1) * pl["sk_q"] // pl["sk_ctas"]
        cpt, ch = pl["sk_cpt"], pl["sk_chunk_kb"]
        q = q0 if k == 0 else (q0 // cpt + 1) * cpt
        if k > 1 or q >= q1:
            return out
        t = q // cpt
        qe = min(q1, (t + 1) * cpt)
        out.append((pl["sk_tile0"] + t, (q - t * cpt) * ch, min(pl["num_kb"], (qe - t * cpt) * ch), k))
        i += 1


def _check(v, m, n, k, pairs=None):
    slots = P if pairs is None else pairs
    pl = cp.Context.tc_plan(v, m, n, k, P, pairs=pairs)
    tiles = pl["tiles"]
    tm = 128 if pairs is None else 256
    assert tiles == -(-m // tm) * -(-n // 256)
    if pairs is not None:
        assert pl["splits"] == 1
    grid = min(tiles * pl["splits"], slots)
    if pl["sk_q"]:
        grid = slots if pl["sk_tile0"] > 0 else pl["sk_ctas"]
    cover = {}
    for b in range(grid):
        its = _items(b, grid, pl)
        assert sum(1 for it in its if it[3] >= 0) <= 2
        for t, kb0, kb1, piece in its:
            assert 0 <= kb0 < kb1 <= pl["num_kb"]
            cover.setdefault(t, []).append((kb0, kb1))
    assert sorted(cover) == list(range(tiles))
    for t, segs in cover.items():
        if pl["splits"] > 1:
            assert len(segs) == pl["splits"]
            continue
        assert len(segs) <= 5
        pos = 0
        for kb0, kb1 in sorted(segs):
            assert kb0 == pos
            pos = kb1
        assert pos == pl["num_kb"]
    return pl


@pytest.mark.parametrize("v", TC)
def test_work_lists_cover_every_k_block_once(v):
    for m, n, k in itertools.product([128, 1000, 2048, 2560, 4096, 5120, 333],
                                     [256, 2048, 4096, 100], [32, 300, 1024, 4096, 8200]):
        _check(v, m, n, k)


def test_stream_k_where_it_pays():
    # 4096^3: 512 tiles = 3 full waves + 68 tiles; long K
    for v in (cp.V_SPLIT3, cp.V_SPLIT6, cp.V_TC_BF16, cp.V_TC_TF32, cp.V_SPLIT3_FUSED):
        pl = _check(v, 4096, 4096, 4096)
        assert pl["sk_tile0"] == 444 and pl["sk_q"] > 0, v
    # FP8 tiles are too short for the fixup to pay; 8192^3 has a full last
    # wave in effect (2048 tiles, 13.8 waves); 2048^3 one wave of 128 tiles
    assert _check(cp.V_TC_FP8, 4096, 4096, 4096)["sk_q"] == 0
    assert _check(cp.V_SPLIT3, 8192, 8192, 8192)["sk_q"] == 0
    assert _check(cp.V_SPLIT3, 2048, 2048, 2048)["sk_q"] == 0
    # few tiles, long K: split-K with a reduce instead
    pl = _check(cp.V_SPLIT3, 256, 1024, 4096)
    assert pl["splits"] > 1 and pl["sk_q"] == 0


def test_plan_arguments_are_validated():
    assert cp.compar_tc_plan(cp.V_GROUPED, 64, 64, 64, P, (cp._i64 * 9)()) == cp.ERR_INVALID
    assert cp.compar_tc_plan(cp.V_SIMT, 64, 64, 64, P, (cp._i64 * 9)()) == cp.ERR_INVALID
    assert cp.compar_tc_plan(cp.V_SPLIT3, 0, 64, 64, P, (cp._i64 * 9)()) == cp.ERR_INVALID


PAIR = [cp.V_TC_TF32, cp.V_TC_BF16, cp.V_TC_FP8, cp.V_SPLIT3]


@pytest.mark.parametrize("v", PAIR)
@pytest.mark.parametrize("pairs", [74, 71, 1])
def test_pair_work_lists_cover_every_k_block_once(v, pairs):
    """CTA-pair plans (256 x 256 tiles, the work list walked per pair): the
    same coverage rules, for the pair count of a full B300 and for fewer
    resident pairs."""
    for m, n, k in itertools.product([256, 1000, 2560, 4096, 5120, 333],
                                     [256, 2048, 4096, 100], [32, 300, 4096, 8200]):
        _check(v, m, n, k, pairs=pairs)


def test_pair_plan_stream_k_and_validation():
    # 4096^3 on 74 pairs: 256 tiles = 3 waves + 34 tiles; the tail is cut
    pl = _check(cp.V_SPLIT3, 4096, 4096, 4096, pairs=74)
    assert pl["tiles"] == 256 and pl["sk_tile0"] == 222 and pl["sk_q"] > 0
    out = (cp._i64 * 9)()
    for v in (cp.V_SPLIT3_FUSED, cp.V_SPLIT6, cp.V_SPLIT3_TF32):   # no pair kernels
        assert cp.compar_tc_pair_plan(v, 512, 512, 512, 74, out) == cp.ERR_INVALID
    assert cp.compar_tc_pair_plan(cp.V_SPLIT3, 512, 512, 512, 0, out) == cp.ERR_INVALID
    assert cp.compar_tc_pair_plan(cp.V_SIMT, 512, 512, 512, 74, out) == cp.ERR_INVALID
