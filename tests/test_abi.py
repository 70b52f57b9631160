"""The C ABI library builds for sm_103a, loads without a GPU, and exports every
entry point that include/rr.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(rr_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = _declared()
    for must in ("rr_load_index", "rr_range_search", "rr_result_free", "rr_last_error", "rr_brute_force"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_2502_13245_gb300 as rr
    path = rr.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(rr.EXPORTS) == sorted(_declared())


def test_params_defaults_without_gpu():
    import paper_2502_13245_gb300 as rr
    p = rr.rr_params_init()
    assert p.beam == 64 and p.b_max == 32768 and p.es_visit_limit == 20
    assert p.max_results_total == 1 << 28
    q = rr.rr_params_init(beam=16, collect_stats=1)
    assert q.beam == 16 and q.collect_stats == 1


def test_errors_are_statuses_not_crashes():
    import paper_2502_13245_gb300 as rr
    L = rr.load_library()
    h = ctypes.c_void_p()
    assert L.rr_load_index(b"/nonexistent/file.rrx", 0, ctypes.byref(h)) == rr.RR_EINVAL
    assert "cannot open" in rr.rr_last_error()
    assert L.rr_create_index(None, 10, 4, 0, 0, None, 4, 0, 0, 1, ctypes.byref(h)) == rr.RR_EINVAL
    res = rr.Result()
    assert L.rr_range_search(None, None, 0, None, 1.0, 0, None, None, 0, ctypes.byref(res)) == rr.RR_EINVAL


def test_rrx_reader_rejects_corrupt_file(tmp_path):
    import numpy as np
    import paper_2502_13245_gb300 as rr
    import rrsynth
    X = np.arange(64, dtype=np.uint8).reshape(8, 8)
    adj = np.full((8, 2), 0xFFFFFFFF, np.uint32)
    p = tmp_path / "x.rrx"
    rrsynth.write_rrx(str(p), X, adj, 0, 0)
    raw = bytearray(p.read_bytes())
    raw[70] ^= 0xFF
    (tmp_path / "bad.rrx").write_bytes(bytes(raw))
    L = rr.load_library()
    h = ctypes.c_void_p()
    assert L.rr_load_index(str(tmp_path / "bad.rrx").encode(), 0, ctypes.byref(h)) == rr.RR_EFORMAT
    assert "checksum" in rr.rr_last_error()
    (tmp_path / "short.rrx").write_bytes(bytes(raw[:100]))
    assert L.rr_load_index(str(tmp_path / "short.rrx").encode(), 0, ctypes.byref(h)) == rr.RR_EFORMAT


def test_binding_struct_layouts_match_the_library():
    # every ctypes mirror of a public struct has the size the C compiler gave it
    import paper_2502_13245_gb300 as rr
    rr.build()
    sizes = rr.rr_abi_sizes()
    mirror = {"rr_params": rr.Params, "rr_query_stats": rr.QueryStats, "rr_result": rr.Result,
              "rr_index_info": rr.IndexInfo, "rr_profile": rr.Profile, "rr_serve_cfg": rr.ServeCfg,
              "rr_serve_stats_t": rr.ServeStats, "rr_build_info": rr.BuildInfo}
    for name, cls in mirror.items():
        assert ctypes.sizeof(cls) == sizes[name], (name, ctypes.sizeof(cls), sizes[name])
    assert rr.STATS_DTYPE.itemsize == sizes["rr_query_stats"]


def test_graph_builder_arguments_are_checked_without_gpu():
    import numpy as np
    import paper_2502_13245_gb300 as rr
    L = rr.load_library()
    X = np.zeros((10, 4), np.float32)
    adj = np.zeros((10, 4), np.uint32)
    assert L.rr_build_graph(X.ctypes.data, 10, 4, rr.RR_F32, rr.RR_L2, 4, 8, 1.2, 2, 0, 0, 0, adj.ctypes.data,
                            None) == rr.RR_EINVAL
    assert "8-bit" in rr.rr_last_error()
    Xu = np.zeros((10, 4), np.uint8)
    assert L.rr_build_graph(Xu.ctypes.data, 10, 4, rr.RR_U8, rr.RR_L2, 4, 8, 0.5, 2, 0, 0, 0, adj.ctypes.data,
                            None) == rr.RR_EINVAL
    assert L.rr_build_graph(Xu.ctypes.data, 10, 4, rr.RR_U8, rr.RR_L2, 4, 8, 1.2, 2, 0, 10, 0, adj.ctypes.data,
                            None) == rr.RR_EINVAL
    assert L.rr_build_graph(None, 10, 4, rr.RR_U8, rr.RR_L2, 4, 8, 1.2, 2, 0, 0, 0, adj.ctypes.data,
                            None) == rr.RR_EINVAL
