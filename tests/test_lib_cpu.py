"""libhc.so on the CPU: it loads, exports every entry point include/hc.h
declares, and rejects bad arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1908_05936_gb300 import build
    build.build()
    from paper_1908_05936_gb300 import _lib
    return _lib.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hc.h")).read()
    return sorted(set(re.findall(r"^HC_API\s+[\w\s\*]+?\b(hc_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    from paper_1908_05936_gb300 import _lib
    assert sorted(_lib.EXPORTS) == names


def test_abi_version(lib):
    assert lib.hc_abi_version() == 2


def test_argument_errors_before_any_launch(lib):
    from paper_1908_05936_gb300 import _lib as L
    h = ctypes.c_void_p()
    assert lib.hc_create(None, 0, 16, None, None) == L.ERR_ARG
    assert lib.hc_create(ctypes.byref(h), 9, 16, None, None) == L.ERR_ARG
    assert b"kind" in lib.hc_last_error()
    assert lib.hc_create(ctypes.byref(h), 0, 0, None, None) == L.ERR_ARG
    bad = L.Config(48, 0, 0)
    assert lib.hc_create(ctypes.byref(h), 0, 16, ctypes.byref(bad), None) == L.ERR_ARG
    tes = L.Config(32, L.HASH_TESCHNER, 0)
    assert lib.hc_create(ctypes.byref(h), L.SET_U64, 16, ctypes.byref(tes), None) == L.ERR_ARG
    assert lib.hc_insert(None, None, None, 1, None, None) == L.ERR_ARG
    assert lib.hc_find(None, None, 1, None, None, None) == L.ERR_ARG
    assert lib.hc_erase(None, None, 1, None, None) == L.ERR_ARG
    assert lib.hc_destroy(None) == L.OK
    assert lib.hc_batch_create(None, None, 0, None, None) == L.ERR_ARG
    assert lib.hc_ordered_scratch_bytes(-1) == -1
    assert lib.hc_ordered_scratch_bytes(1000) >= 2048 * 16 + 1000 * 9      # 16-byte entries, leaders, skip flags
    assert lib.hc_insert_ordered(None, None, None, 1, None, None, 0, None) == L.ERR_ARG
    assert lib.hc_erase_ordered(None, None, 1, None, None, 0, None) == L.ERR_ARG
    assert lib.hc_apply_mixed(None, None, None, None, 1, None, None, None) == L.ERR_ARG
    assert lib.hc_pack_short3(None, -1, None, None) == L.ERR_ARG
    assert lib.hc_pack_short3(None, 0, None, None) == L.OK
    assert lib.hc_unpack_short3(None, 1, None, None) == L.ERR_ARG
    s3 = L.Config(32, L.HASH_TESCHNER_SHORT3, 0)
    assert lib.hc_create(ctypes.byref(h), L.SET_U64, 16, ctypes.byref(s3), None) == L.ERR_ARG
    assert lib.hc_create(ctypes.byref(h), L.MAP_I64_I32, 16, ctypes.byref(L.Config(32, 3, 0)), None) == L.ERR_ARG
    pred = L.Predicate(L.PRED_ALL, 0, 0, 0)
    assert lib.hc_select(None, ctypes.byref(pred), None, None, 0, None, None) == L.ERR_ARG
    assert lib.hc_batch_destroy(None) == L.OK


def test_served_calls_refuse_bad_handles(lib):
    """The served loop's entry points check their handle and arguments before
    touching the device (no GPU needed)."""
    from paper_1908_05936_gb300 import _lib as L
    req = L.Request(0, 0, None, None, 0, None, None, 0.0, 0.0, -1.0, -1, 0)
    st = L.ServeStats()
    assert lib.hc_server_create(None, None, 0, None) == L.ERR_ARG
    h = ctypes.c_void_p()
    assert lib.hc_server_create(ctypes.byref(h), None, 0, None) == L.ERR_ARG
    assert lib.hc_server_start(None) == L.ERR_ARG
    assert lib.hc_server_submit(None, ctypes.byref(req)) == L.ERR_ARG
    assert lib.hc_server_wait(None, ctypes.byref(req), 1.0) == L.ERR_ARG
    assert lib.hc_server_stop(None, ctypes.byref(st)) == L.ERR_ARG
    assert lib.hc_server_run(None, ctypes.byref(req), 1, 0, 1.0, ctypes.byref(st)) == L.ERR_ARG
    assert lib.hc_server_destroy(None) == L.OK
    assert L.RC_NAMES[L.ERR_TIMEOUT] == "HC_ERR_TIMEOUT"


def test_table_bytes(lib):
    from paper_1908_05936_gb300 import _lib as L
    b = ctypes.c_int64()
    # header (256) + whole buckets of slots, rounded to 256 bytes
    assert lib.hc_table_bytes(L.MAP_U64_U64, 1 << 28, None, ctypes.byref(b)) == L.OK
    assert b.value == 256 + (1 << 28) * 16
    assert lib.hc_table_bytes(L.SET_U32, 1, None, ctypes.byref(b)) == L.OK
    assert b.value == 256 + 256          # one 32-byte bucket, rounded up
    cfg = L.Config(128, 0, 0)
    assert lib.hc_table_bytes(L.SET_U64, 17, ctypes.byref(cfg), ctypes.byref(b)) == L.OK
    assert b.value == 256 + 256           # two 128-byte buckets
    assert lib.hc_table_bytes(L.SET_U64, 0, None, ctypes.byref(b)) == L.ERR_ARG


def test_examples_library_exports_and_argument_errors(lib):
    """libhc_examples.so (user kernels on include/hc_device.cuh) builds against
    the public headers alone, loads, and rejects bad arguments before any
    launch; hc_device_view_get rejects a NULL table."""
    from paper_1908_05936_gb300 import _lib as L
    from paper_1908_05936_gb300 import build
    from paper_1908_05936_gb300 import device_api as D
    build.build_examples()
    ex = D.load_examples()
    for name in ("hcx_apply", "hcx_update_set"):
        assert hasattr(ex, name), name
    dv = L.DeviceView()
    assert lib.hc_device_view_get(None, ctypes.byref(dv), None) == L.ERR_ARG
    assert ex.hcx_apply(None, None, 0, None, None, 1, None, None, None, 128, None) == L.ERR_ARG
    dv.kind = 9
    assert ex.hcx_apply(ctypes.byref(dv), None, 0, None, None, 0, None, None, None, 128, None) == L.OK
    assert ex.hcx_apply(ctypes.byref(dv), None, 3, None, None, 1, None, None, None, 128, None) == L.ERR_ARG
    assert ex.hcx_apply(ctypes.byref(dv), None, 0, None, None, 1, None, None, None, 100, None) == L.ERR_ARG
    assert ex.hcx_update_set(ctypes.byref(dv), ctypes.byref(dv), None, 1, None) == L.ERR_ARG


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct the binding passes by pointer has the header's size and
    field offsets (compiled here with the system C compiler)."""
    import shutil
    import subprocess
    from paper_1908_05936_gb300 import _lib as L
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    checks = {"hc_config": (L.Config, []), "hc_launch": (L.Launch, []), "hc_stats_t": (L.Stats, []),
              "hc_batch_item": (L.BatchItem, ["d_keys", "n", "d_vals_out"]),
              "hc_batch_config": (L.BatchConfig, ["use_graph"]),
              "hc_device_view": (L.DeviceView, ["nb", "kind", "pad_from"]),
              "hc_predicate": (L.Predicate, ["lo", "box"]),
              "hc_serve_config": (L.ServeConfig, ["slot_bytes", "batch"]),
              "hc_request": (L.Request, ["h_keys", "n", "arrival", "deadline", "done", "rc"]),
              "hc_serve_stats": (L.ServeStats, ["timed_out", "wall_s", "max_ms"])}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hc.h"', "int main(void) {"]
    for name, (_, fields) in checks.items():
        lines.append(f'    printf("%zu\\n", sizeof({name}));')
        for f in fields:
            lines.append(f'    printf("%zu\\n", offsetof({name}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = []
    for name, (cls, fields) in checks.items():
        want.append(ctypes.sizeof(cls))
        want += [getattr(cls, f).offset for f in fields]
    assert got == want


def test_random_read_probe_argument_errors(lib):
    """hc_measure_random_reads refuses bad arguments before any launch."""
    from paper_1908_05936_gb300 import _lib as L
    ms = ctypes.c_float()
    assert lib.hc_measure_random_reads(None, 1 << 20, 1, 1, ctypes.byref(ms), None) == L.ERR_ARG
    assert lib.hc_measure_random_reads(ctypes.c_void_p(1 << 20), 32, 1, 1, ctypes.byref(ms), None) == L.ERR_ARG
    assert lib.hc_measure_random_reads(ctypes.c_void_p(1 << 20), 1 << 20, 0, 1, ctypes.byref(ms), None) == L.ERR_ARG
    assert lib.hc_measure_random_reads(ctypes.c_void_p((1 << 20) + 16), 1 << 20, 1, 1, ctypes.byref(ms),
                                       None) == L.ERR_ARG


def test_batch_tuner_candidates_and_cache(tmp_path, monkeypatch):
    """The batched-form tuner's candidate list and cache lookup (no GPU)."""
    import json
    from paper_1908_05936_gb300 import tune
    c32, c64 = tune.batch_candidates(32), tune.batch_candidates(64)
    assert all(c["lane_bytes"] == 0 for c in c32)              # a 32-byte bucket is one 32-byte lane
    assert len(c64) == len(c32) + 18 and {c["keys_per_group"] for c in c64} == {1, 2, 4}
    assert all(c["block"] in (64, 128, 256) and c["tile"] in (0, 1024, 4096) for c in c64)
    cache = tmp_path / "tuned.json"
    monkeypatch.setattr(tune, "CACHE", str(cache))
    monkeypatch.setattr(tune, "device_key", lambda: "dev/1SM")
    assert tune.batch_config() is None
    best = dict(bucket_bytes=32, lane_bytes=0, keys_per_group=1, block=128, tile=1024, ms=5.0, mops=1.0)
    cache.write_text(json.dumps({"dev/1SM": {"batch/set_u64": best}}))
    assert tune.batch_config() == dict(bucket_bytes=32, lane_bytes=0, keys_per_group=1, block=128, tile=1024)
