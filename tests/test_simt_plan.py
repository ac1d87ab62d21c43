"""Host-side launch plans of the SIMT variant (no GPU).

Short-M shapes with a wide, deep B (rows of B readable 4 elements at a time)
take the skinny kernel: K chunks of at most 512 (multiples of 8) cover K, at
most one cluster's worth of trailing chunks is empty, clusters hold 1, 2, 4
or 8 CTAs, and the grid fills the GPU (three CTAs per SM) without a second
wave unless K needs more chunks.  Other shapes take the tiled kernel.  The
parity tests' skinny shapes cover every branch of the plan."""
import pytest

import paper_2311_03543_b300 as cp

P = 148


@pytest.mark.parametrize("m", [1, 7, 8, 9, 16, 33, 48, 64])
@pytest.mark.parametrize("n,k", [(256, 8), (512, 64), (1000, 3000), (4096, 4096), (8192, 1024),
                                 (65536, 1030), (300, 20), (16384, 100000)])
def test_skinny_plan_covers_k(m, n, k):
    p = cp.Context.simt_plan(m, n, k, num_sms=P)
    if n % 4:
        assert p["skinny"] == 0
        return
    assert p["skinny"] == 1
    assert p["rows"] == (8 if m <= 8 else 16) and p["cols"] == 512
    cl, kp = p["cluster"], p["k_per"]
    assert cl in (1, 2, 4, 8) and p["rows"] % cl == 0
    assert 8 <= kp <= 512 and kp % 8 == 0
    chunks = p["splits"] * cl
    assert kp * chunks >= k                 # K covered
    assert kp * (chunks - cl) < k           # fewer than one cluster of empty chunks
    ctas = -(-m // p["rows"]) * -(-n // 512) * chunks
    if -(-k // 512) * -(-m // p["rows"]) * -(-n // 512) <= 3 * P:
        assert ctas <= max(3 * P, -(-m // p["rows"]) * -(-n // 512) * cl)


@pytest.mark.parametrize("m,n,k,ldb", [(65, 4096, 4096, 4096), (16, 128, 4096, 128),
                                       (16, 4098, 4096, 4098), (16, 4096, 4096, 4097),
                                       (256, 4096, 4096, 4096)])
def test_tiled_plan_elsewhere(m, n, k, ldb):
    p = cp.Context.simt_plan(m, n, k, ldb=ldb, num_sms=P)
    assert p["skinny"] == 0 and p["cluster"] == 1
    assert p["rows"] == (32 if m <= 48 else 128) and p["cols"] == 128
    assert p["k_per"] * p["splits"] >= k


def test_dtype_sets_the_vector_rule():
    # 4 bf16 or E4M3 elements are 8 or 4 bytes: any ldb % 4 == 0 row start aligns
    for dt in (cp.F32, cp.BF16, cp.F8E4M3):
        assert cp.Context.simt_plan(16, 4096, 4096, dtype=dt)["skinny"] == 1
        assert cp.Context.simt_plan(16, 4096, 4096, dtype=dt, ldb=4098)["skinny"] == 0


def test_parity_shapes_cover_every_branch():
    import importlib.util, os
    spec = importlib.util.spec_from_file_location(
        "parity", os.path.join(os.path.dirname(__file__), "test_gemm_parity.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    seen = set()
    for m, n, k in mod.SKINNY:
        p = cp.Context.simt_plan(m, n, k, num_sms=P)
        assert p["skinny"] == 1
        seen.add((p["cluster"], p["splits"] > 1))
    assert seen == {(c, r) for c in (1, 2, 4, 8) for r in (False, True)}


def test_bad_arguments():
    with pytest.raises(cp.ComparError):
        cp.Context.simt_plan(0, 4, 4)
    with pytest.raises(cp.ComparError):
        cp.Context.simt_plan(4, 8, 4, ldb=4)
