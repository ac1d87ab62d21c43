"""C-ABI boundary checks that need no GPU: the library loads, exports every
function the public headers declare, and answers its host-only queries."""
import ctypes
import glob
import os
import re

import pytest

import paper_2311_03543_b300 as cp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(compar_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary_calls():
    names = _declared_functions()
    for required in ["compar_init", "compar_terminate", "compar_gemm", "compar_gemm_batched",
                     "compar_force_variant", "compar_selector_load"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(cp.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert _declared_functions() == set(cp.SIGNATURES)


def test_host_only_queries():
    assert cp.compar_variant_count() == cp.NUM_VARIANTS
    names = [cp.compar_variant_name(i).decode() for i in range(cp.NUM_VARIANTS)]
    assert names == cp.VARIANT_NAMES
    assert cp.compar_variant_name(99) is None
    assert cp.compar_status_string(cp.ERR_NO_VARIANT).decode() == "no variant meets the tolerance"
    assert cp.compar_status_string(12345).decode() == "unknown status"


def test_variant_ids_are_stable():
    # ids 0-5 and 6 (grouped, batched only) as first assigned; later variants
    # take new ids
    assert [cp.compar_variant_name(i).decode() for i in range(7)] == [
        "naive-f32", "simt-f32", "tc-tf32", "tc-bf16", "tc-fp8", "split-3xbf16", "grouped"]
    assert cp.compar_variant_name(7).decode() == "split-6xbf16"
    assert cp.compar_variant_name(8).decode() == "split-3xtf32"
    assert cp.compar_variant_name(9).decode() == "split-3xbf16-fused"
    assert (cp.V_GROUPED, cp.V_SPLIT6, cp.V_SPLIT3_TF32, cp.V_SPLIT3_FUSED) == (6, 7, 8, 9)
    h = cp.Context.host()
    try:
        assert not h.supported(cp.V_GROUPED, 64, 64, 64, cp.F32)   # never a single call
        assert h.supported(cp.V_SPLIT6, 64, 64, 64, cp.F32)
        assert cp.compar_force_variant(h.handle, cp.V_GROUPED) == cp.OK
        assert cp.compar_force_variant(h.handle, cp.NUM_VARIANTS) == cp.ERR_INVALID
        assert cp.compar_force_variant(h.handle, -1) == cp.OK
    finally:
        h.close()


def test_null_context_is_rejected():
    assert cp.compar_gemm(None, 1, 1, 1, cp.F32, 0.0, None, None, None, None) == cp.ERR_INVALID
    assert cp.compar_force_variant(None, 1) == cp.ERR_INVALID
    assert cp.compar_terminate(None) == cp.OK
    assert cp.compar_init(None, 0) == cp.ERR_INVALID


def test_selector_load_missing_file_without_context():
    assert cp.compar_selector_load(None, b"/nonexistent") == cp.ERR_INVALID
