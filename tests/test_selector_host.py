"""Host logic of the runtime, on host-only contexts (no GPU): eligibility by
dtype and error model, history-table selection and its nearest-neighbour
lookup, the roofline prior, forced variants, decision caching, and selector
files (round trip, corruption, version checks)."""
import os

import pytest

import paper_2311_03543_b300 as cp


@pytest.fixture
def hctx():
    c = cp.Context.host()
    yield c
    c.close()


def _rec(m, n, k, dtype, v, t, batch=1, tol=1e-5):
    r = cp.compar_record_t()
    r.m, r.n, r.k, r.dtype, r.variant, r.batch = m, n, k, dtype, v, batch
    r.tol, r.time_ms, r.rel_err = tol, t, -1.0
    return r


def test_compute_calls_are_refused_without_a_device(hctx):
    assert cp.compar_gemm(hctx.handle, 4, 4, 4, cp.F32, 0.0, 16, 16, 16, None) == cp.ERR_UNSUPPORTED
    assert cp.compar_selftest_timeout(hctx.handle, None) == cp.ERR_UNSUPPORTED


def test_eligibility_by_tolerance(hctx):
    # FP32 inputs at 1e-5: only FP32-accurate variants (naive, simt, 3xbf16)
    assert hctx.select(4096, 4096, 4096, cp.F32, 1e-5) in (cp.V_NAIVE, cp.V_SIMT, cp.V_SPLIT3,
                                                            cp.V_SPLIT3_TF32, cp.V_SPLIT6,
                                                            cp.V_SPLIT3_FUSED)
    # at 1e-1 the fp8 variant is the fastest by the roofline prior for big shapes
    assert hctx.select(8192, 8192, 8192, cp.F32, 1e-1) == cp.V_TC_FP8
    # BF16 inputs can never run the f32-only variants
    assert hctx.select(2048, 2048, 2048, cp.BF16, 1e-3) in (cp.V_NAIVE, cp.V_SIMT, cp.V_TC_BF16)


def test_tolerance_below_3xbf16(hctx):
    # tol 1e-6 on float32: 3xBF16 (~4e-6) no longer qualifies; a big square
    # goes to the 6-product split, the only tensor-core variant left
    assert hctx.select(4096, 4096, 4096, cp.F32, 1e-6) == cp.V_SPLIT6
    # SIMT's error follows its longest FMA chain: a 32 x 32 x 4096 product is
    # split 16 ways along K (256-term chains), so SIMT qualifies there, while
    # the naive variant's 4096-term chain does not
    assert hctx.predict_error(cp.V_NAIVE, cp.F32, 4096) * 1.25 > 1e-6
    assert hctx.select(32, 32, 4096, cp.F32, 1e-6) in (cp.V_SIMT, cp.V_SPLIT6)


def test_no_variant_meets_impossible_tolerance(hctx):
    assert cp.compar_select(hctx.handle, 64, 64, 64, cp.F32, 1e-12, 1) == cp.ERR_NO_VARIANT


def test_history_table_overrides_prior(hctx):
    m = n = k = 1024
    first = hctx.select(m, n, k, cp.F32, 1e-5)
    other = cp.V_SIMT if first != cp.V_SIMT else cp.V_SPLIT3
    hctx.record_add([_rec(m, n, k, cp.F32, other, 0.001), _rec(m, n, k, cp.F32, first, 5.0)])
    hctx.clear_decisions()
    assert hctx.select(m, n, k, cp.F32, 1e-5) == other
    # a nearby shape (within the quarter-log2 grid distance) follows the table
    hctx.clear_decisions()
    assert hctx.select(1100, 1024, 1000, cp.F32, 1e-5) == other


def test_decision_cache_is_sticky_until_cleared(hctx):
    m = n = k = 512
    v0 = hctx.select(m, n, k, cp.F32, 1e-5)
    other = cp.V_SIMT if v0 != cp.V_SIMT else cp.V_NAIVE
    hctx.record_add([_rec(m, n, k, cp.F32, other, 1e-6)])
    assert hctx.select(m, n, k, cp.F32, 1e-5) == v0          # cached
    hctx.clear_decisions()
    assert hctx.select(m, n, k, cp.F32, 1e-5) == other


def test_forced_variant(hctx):
    hctx.force_variant(cp.V_NAIVE)
    assert hctx.select(4096, 4096, 4096, cp.F32, 1e-5) == cp.V_NAIVE
    hctx.force_variant(cp.V_SPLIT3)
    assert cp.compar_select(hctx.handle, 64, 64, 64, cp.BF16, 1e-3, 1) == cp.ERR_UNSUPPORTED
    hctx.force_variant(None)
    with pytest.raises(cp.ComparError):
        hctx.force_variant(17)


def test_error_model_get_set_predict(hctx):
    c0, c1, c2 = hctx.error_model(cp.V_SPLIT3, cp.F32)
    assert c0 > 0
    assert hctx.error_model(cp.V_SPLIT3, cp.BF16)[0] == float("inf")
    hctx.set_error_model(cp.V_SPLIT3, cp.F32, 1e-3, 0.0, 0.0)
    assert hctx.predict_error(cp.V_SPLIT3, cp.F32, 4096) == pytest.approx(1e-3, rel=1e-6)
    # with a pessimistic model the 3xBF16 variant drops out at 1e-5
    assert hctx.select(4096, 4096, 4096, cp.F32, 1e-5) != cp.V_SPLIT3
    hctx.set_error_model(cp.V_SPLIT3, cp.F32, 0.0, 0.0, 1.0)
    u = 2.0 ** -24
    assert hctx.predict_error(cp.V_SPLIT3, cp.F32, 1000) == pytest.approx(1000 * u, rel=1e-6)
    with pytest.raises(cp.ComparError):
        hctx.set_error_margin(0.5)


def test_selector_file_round_trip(hctx, tmp_path):
    recs = [_rec(256 * i, 256 * i, 256 * i, cp.F32, v, 0.01 * i * (v + 1))
            for i in range(1, 8) for v in (0, 1, 5)]
    hctx.record_add(recs)
    hctx.set_error_model(cp.V_TC_TF32, cp.F32, 2e-4, 0.5, 0.01)
    path = str(tmp_path / "sel.bin")
    hctx.selector_save(path)
    other = cp.Context.host()
    try:
        other.selector_load(path)
        assert other.error_model(cp.V_TC_TF32, cp.F32) == pytest.approx((2e-4, 0.5, 0.01))
        for i in range(1, 8):
            s = 256 * i
            assert other.select(s, s, s, cp.F32, 1e-5) == hctx.select(s, s, s, cp.F32, 1e-5)
    finally:
        other.close()


def test_rehearsal_sample_is_saved_capped_and_reloaded(tmp_path):
    """A selector file carries a uniform sample of at most 16384 timing
    records (48 bytes each): with 20000 records held the file is exactly
    16384 records larger than with the same models and none held, and a
    context that loaded the file and records nothing more writes the same
    sample size again."""
    import os
    recs = []
    for i in range(20000):
        r = cp.compar_record_t()
        r.m, r.n, r.k = 64 + i % 512, 32 + i % 256, 16 + i % 1024
        r.dtype, r.variant, r.batch = cp.F32, i % cp.NUM_VARIANTS, 1
        if r.variant == cp.V_GROUPED:
            r.variant = cp.V_SIMT
        r.tol, r.time_ms, r.rel_err = 1e-5, 0.01 + 1e-6 * i, -1.0
        recs.append(r)
    h = cp.Context.host()
    h.record_add(recs)                  # records and history observations
    p1 = str(tmp_path / "with.bin")
    h.selector_save(p1)
    assert cp.compar_record_clear(h.handle) == cp.OK   # history kept, records gone
    p0 = str(tmp_path / "none.bin")
    h.selector_save(p0)
    assert os.path.getsize(p1) - os.path.getsize(p0) == 16384 * 48
    h2 = cp.Context.host()
    h2.selector_load(p1)
    p2 = str(tmp_path / "again.bin")
    h2.selector_save(p2)
    assert os.path.getsize(p2) == os.path.getsize(p1)
    for c in (h, h2):
        c.close()


def test_corrupted_selector_file_is_rejected_and_model_kept(hctx, tmp_path):
    hctx.record_add([_rec(2048, 2048, 2048, cp.F32, cp.V_SIMT, 1e-6)])
    path = str(tmp_path / "sel.bin")
    hctx.selector_save(path)
    data = bytearray(open(path, "rb").read())
    fresh = cp.Context.host()
    try:
        fresh.record_add([_rec(2048, 2048, 2048, cp.F32, cp.V_NAIVE, 1e-7)])
        before = fresh.select(2048, 2048, 2048, cp.F32, 1e-5)
        bad = bytearray(data); bad[40] ^= 0xFF                     # payload flip -> checksum
        for name, blob in [("flip", bad), ("magic", b"XXXXXXXX" + data[8:]),
                           ("version", data[:8] + b"\x09\x00\x00\x00" + data[12:]),
                           ("truncated", data[:-9]), ("empty", b"")]:
            p = str(tmp_path / f"{name}.bin")
            open(p, "wb").write(bytes(blob))
            assert cp.compar_selector_load(fresh.handle, os.fsencode(p)) == cp.ERR_IO, name
        fresh.clear_decisions()
        assert fresh.select(2048, 2048, 2048, cp.F32, 1e-5) == before
        assert cp.compar_selector_load(fresh.handle, b"/nonexistent/file") == cp.ERR_IO
    finally:
        fresh.close()


def test_records_ring_and_validation(hctx):
    hctx.record_add([_rec(8, 8, 8, cp.F32, 1, 0.5)])
    assert len(hctx.records()) == 1
    bad = _rec(8, 8, 8, cp.F32, 42, 0.5)
    with pytest.raises(cp.ComparError):
        hctx.record_add([bad])
    hctx.record_clear()
    assert hctx.records() == []


def test_online_exploration_stays_within_eligible_variants(hctx):
    # epsilon = 1: every decision-cache miss explores; picks vary, are never
    # cached, and never leave the variants that meet the tolerance
    hctx.set_online(epsilon=1.0)
    seen = set()
    for _ in range(200):
        v = hctx.select(2048, 2048, 2048, cp.F32, 1e-5)
        assert v in (cp.V_NAIVE, cp.V_SIMT, cp.V_SPLIT3, cp.V_SPLIT6, cp.V_SPLIT3_TF32,
                     cp.V_SPLIT3_FUSED)
        seen.add(v)
    assert len(seen) >= 2
    explored, retrains, _ = hctx.online_stats()
    assert explored == 200 and retrains == 0
    hctx.set_online(epsilon=0.0)
    first = hctx.select(2048, 2048, 2048, cp.F32, 1e-5)
    assert all(hctx.select(2048, 2048, 2048, cp.F32, 1e-5) == first for _ in range(20))
    with pytest.raises(cp.ComparError):
        hctx.set_online(epsilon=1.5)


def test_stencil_selection_on_host_context(hctx):
    # roofline prior only: a long run on a big grid goes to temporal blocking,
    # a single step to the one-launch-per-step variant; forcing overrides
    assert hctx.stencil_select(8192, 8192, 100) in (cp.S_TILED, cp.S_TMA)
    assert hctx.stencil_select(8192, 8192, 1) == cp.S_NAIVE
    assert hctx.stencil_select(64, 62, 100) != cp.S_TMA          # rows not 16-byte multiples
    hctx.stencil_force_variant(cp.S_NAIVE)
    try:
        assert hctx.stencil_select(8192, 8192, 100) == cp.S_NAIVE
    finally:
        hctx.stencil_force_variant(None)
    assert cp.compar_stencil_select(hctx.handle, 0, 8, 1) == cp.ERR_INVALID
    assert cp.compar_stencil_force_variant(hctx.handle, cp.NUM_STENCIL_VARIANTS) == cp.ERR_INVALID
    assert [cp.compar_stencil_variant_name(v).decode() for v in range(cp.NUM_STENCIL_VARIANTS)] \
        == cp.STENCIL_NAMES
    assert cp.compar_stencil_variant_name(3) is None


def test_stencil_history_round_trips_through_selector_file(hctx, tmp_path):
    # the shipped selector file carries a stencil history table; saving and
    # loading it on a host context keeps the choices
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_2311_03543_b300", "selector_default.bin")
    hctx.selector_load(path)
    picks = [hctx.stencil_select(r, c, i) for r, c, i in [(8192, 8192, 100), (512, 512, 1000),
                                                            (128, 128, 10), (4096, 256, 1)]]
    out = str(tmp_path / "sel.bin")
    hctx.selector_save(out)
    h2 = cp.Context.host()
    try:
        h2.selector_load(out)
        assert [h2.stencil_select(r, c, i) for r, c, i in [(8192, 8192, 100), (512, 512, 1000),
                                                             (128, 128, 10), (4096, 256, 1)]] \
            == picks
    finally:
        h2.close()


def test_context_loads_a_selector_file_at_creation(tmp_path):
    """`selector=` loads a file as selector_load does (the shipped selector
    here, the default of a device context); a missing file is an error."""
    a = cp.Context(host_only=True, selector=cp.DEFAULT_SELECTOR)
    b = cp.Context.host()
    try:
        b.selector_load(cp.DEFAULT_SELECTOR)
        for m, n, k, dt, tol in [(4096, 4096, 4096, cp.F32, 1e-5), (512, 512, 512, cp.F32, 1e-5),
                                 (16, 4096, 4096, cp.F32, 1e-5), (2048, 64, 2048, cp.BF16, 1e-3),
                                 (1000, 1000, 1000, cp.F8E4M3, 1e-1)]:
            assert a.select(m, n, k, dt, tol) == b.select(m, n, k, dt, tol)
    finally:
        a.close()
        b.close()
    with pytest.raises(cp.ComparError):
        cp.Context(host_only=True, selector=str(tmp_path / "missing.bin"))
