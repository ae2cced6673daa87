"""C ABI checks that need no GPU: the library builds and loads, exports every
function include/grand.h declares, validates arguments before touching the
device, and its host-only polar helper agrees with the oracle's construction."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


@pytest.fixture(scope="module")
def glib():
    import paper_2405_01808_gb300 as g

    g.build()
    return g


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w]+\s*\**\s+(grand_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for must in ("grand_code_create", "grand_demod", "grand_decode_batch", "grand_polar_H",
                 "grand_decode_symbols", "grand_decode_mixed", "grand_code_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(glib):
    from paper_2405_01808_gb300 import _build

    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    L = glib.lib()
    for n in declared_functions():
        assert getattr(L, n) is not None


def test_version_and_status(glib):
    L = glib.lib()
    assert L.grand_version() == 10000
    assert L.grand_status_string(0) == b"ok"
    assert b"rank" in L.grand_status_string(-2)


@pytest.mark.parametrize("N", [32, 64, 128, 256, 512, 1024])
def test_polar_helper_matches_oracle(glib, oracle_lib, N):
    H, frozen = glib.polar_H(N, N // 2)
    assert frozen.tolist() == oracle_lib.frozen_set(N, N // 2).tolist()
    dense = oracle_lib.parity_H(N, N // 2)
    assert np.array_equal(H, glib.H_from_dense(dense))


def test_argument_validation_without_gpu(glib):
    L = glib.lib()
    H = np.zeros((16, 1), dtype=np.uint32)
    h = ctypes.c_void_p()
    assert L.grand_polar_H(33, 16, 0.0, H.ctypes.data, None) == -1
    assert L.grand_polar_H(32, 32, 0.0, H.ctypes.data, None) == -1
    assert L.grand_polar_H(32, 16, 0.0, None, None) == -1
    assert L.grand_code_create(H.ctypes.data, 48, 16, ctypes.byref(h)) == -1
    assert L.grand_code_create(None, 32, 16, ctypes.byref(h)) == -1
    # rank deficient H is refused before any device work
    assert L.grand_code_create(H.ctypes.data, 32, 16, ctypes.byref(h)) == -2
    p = glib.Params.make(S=13)
    assert L.grand_decode_symbols(None, ctypes.byref(p), None, 1, ctypes.c_float(1.0), None, None, None, None,
                                  None) == -1
    assert L.grand_demod(None, 1, 32, 16, ctypes.c_float(1.0), 0, None, None, None, None, None, 128, None) == -1
    assert L.grand_code_destroy(None) == 0


def test_server_and_plan_validation_without_gpu(glib):
    L = glib.lib()
    h = ctypes.c_void_p()
    assert L.grand_server_create(None, ctypes.byref(h)) == -1
    assert L.grand_plan_launch(None, None) == -1
    assert L.grand_plan_destroy(None) == 0
    assert L.grand_server_destroy(None) == 0
    assert L.grand_clock_ns() > 0


def test_params_layout_matches_header(glib):
    """grand_params as the binding lays it out: the header's field order,
    natural alignment, 56 bytes (membership fills the slot before the 8-byte
    deadline)."""
    P = glib.Params
    assert ctypes.sizeof(P) == 56
    offsets = {name: getattr(P, name).offset for name, _ in P._fields_}
    assert offsets == {"order": 0, "M": 4, "S": 8, "max_weight": 12, "query_cap": 16, "lik_variant": 24,
                       "tiles": 28, "membership": 44, "deadline_ns": 48}
    text = open(os.path.join(ROOT, "include", "grand.h")).read()
    body = text[text.index("typedef struct grand_params {"):text.index("} grand_params;")]
    fields = re.findall(r"^\s*\w+\s+(\w+)(?:\[\d+\])?;", body, flags=re.M)
    assert fields == [n for n, _ in P._fields_]
    for name, value in (("GRAND_ORDER_QAM_NEARER", glib.ORDER_QAM_NEARER), ("GRAND_ORDER_QAM_NNE5", glib.ORDER_QAM_NNE5),
                        ("GRAND_MEMBERSHIP_DELTA", glib.MEMBERSHIP_DELTA),
                        ("GRAND_MEMBERSHIP_ROW_PARITY", glib.MEMBERSHIP_ROW_PARITY),
                        ("GRAND_MEMBERSHIP_HASH", glib.MEMBERSHIP_HASH),
                        ("GRAND_MEMBERSHIP_FASTEST", glib.MEMBERSHIP_FASTEST),
                        ("GRAND_MEMBERSHIP_SOLVE", glib.MEMBERSHIP_SOLVE),
                        ("GRAND_E_UNSUPPORTED", glib.E_UNSUPPORTED),
                        ("GRAND_ABANDON_SUSPENDED", glib.ABANDON_SUSPENDED),
                        ("GRAND_CURSOR_BYTES", glib.CURSOR_BYTES)):
        assert re.search(rf"{name}(\s*=\s*|\s+){value}\b", text), name


# Every struct of the ABI as a C compiler lays it out (gcc on include/grand.h,
# host only) against the binding's ctypes structures and numpy record types.
_LAYOUT_C = r"""
#include <stddef.h>
#include <stdio.h>
#include "grand.h"
#define F(T, f) printf("%s %s %zu\n", #T, #f, offsetof(T, f));
#define Z(T) printf("%s sizeof %zu\n", #T, sizeof(T));
int main(void) {
  Z(grand_params) F(grand_params, order) F(grand_params, M) F(grand_params, S) F(grand_params, max_weight)
  F(grand_params, query_cap) F(grand_params, lik_variant) F(grand_params, tiles) F(grand_params, membership)
  F(grand_params, deadline_ns)
  Z(grand_frame_desc) F(grand_frame_desc, code) F(grand_frame_desc, M) F(grand_frame_desc, sym_offset)
  F(grand_frame_desc, cw_offset)
  Z(grand_stats) F(grand_stats, evaluated_checks) F(grand_stats, hard_frames) F(grand_stats, search_useful)
  F(grand_stats, prep_ms) F(grand_stats, search_ms)
  Z(grand_tune_result) F(grand_tune_result, best_ms) F(grand_tune_result, candidates) F(grand_tune_result, from_cache)
  F(grand_tune_result, membership)
  Z(grand_server_cfg) F(grand_server_cfg, codes) F(grand_server_cfg, n_codes) F(grand_server_cfg, params)
  F(grand_server_cfg, N0) F(grand_server_cfg, max_slots) F(grand_server_cfg, max_device_bytes)
  F(grand_server_cfg, max_batch) F(grand_server_cfg, n_streams) F(grand_server_cfg, resume_weight_step)
  Z(grand_request) F(grand_request, code) F(grand_request, M) F(grand_request, symbols) F(grand_request, tag)
  F(grand_request, arrival_ns)
  Z(grand_result) F(grand_result, tag) F(grand_result, arrival_ns) F(grand_result, done_ns) F(grand_result, queries)
  F(grand_result, abandon) F(grand_result, continued) F(grand_result, pad) F(grand_result, cw)
  Z(grand_server_stats) F(grand_server_stats, admitted) F(grand_server_stats, max_launch_ns)
  F(grand_server_stats, long_frames) F(grand_server_stats, resume_launches) F(grand_server_stats, long_live)
  return 0;
}
"""


def test_struct_layouts_match_the_compiler(glib, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(_LAYOUT_C)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    c = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        t, f, v = line.split()
        c[(t, f)] = int(v)
    g = glib
    ctypes_structs = {"grand_params": g.Params, "grand_stats": g.Stats, "grand_tune_result": g.TuneResult,
                      "grand_server_cfg": g.ServerCfg, "grand_server_stats": g.ServerStats}
    for t, S in ctypes_structs.items():
        assert ctypes.sizeof(S) == c[(t, "sizeof")], t
        for name, _ in S._fields_:
            if (t, name) in c:
                assert getattr(S, name).offset == c[(t, name)], (t, name)
    records = {"grand_frame_desc": g.FRAME_DESC_DTYPE, "grand_request": g.REQUEST_DTYPE, "grand_result": g.RESULT_DTYPE}
    for t, dt in records.items():
        assert dt.itemsize == c[(t, "sizeof")], t
        for name in dt.names:
            key = (t, name)
            assert key in c, key
            assert dt.fields[name][1] == c[key], key
