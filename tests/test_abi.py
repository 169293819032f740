"""The C-ABI library builds, loads and exports every symbol include/pifu.h
declares; host-side argument checks need no GPU."""
import ctypes
import os
import re
import struct

import numpy as np
import pytest

from paper_2007_13988_gb300 import pifu, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*[A-Za-z_][\w \t\*]*?\b(pifu_\w+)\s*\(", src, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    lib = pifu.load()
    names = declared_functions()
    assert {"pifu_create", "pifu_localize", "pifu_render", "pifu_query"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(pifu.EXPORTS) == names


def test_binding_constants_match_the_header():
    # every enumerator or #define of the header that the binding names
    # carries the same value there
    src = open(os.path.join(ROOT, "include", "pifu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    pairs = re.findall(r"\b(PIFU_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)
    pairs += re.findall(r"#define\s+(PIFU_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", src)
    checked = 0
    for name, value in pairs:
        if hasattr(pifu, name):
            assert getattr(pifu, name) == int(value), name
            checked += 1
    assert checked >= 10
    for name in ("PIFU_SCHED_PER_LAYER", "PIFU_SCHED_CHAINED", "PIFU_PREC_MIXED", "PIFU_ERR_ARG"):
        assert name in dict(pairs), name
    # the profiler classes: the binding's names in the header's order
    classes = {n[len("PIFU_K_"):].lower(): int(v) for n, v in pairs if n.startswith("PIFU_K_")}
    assert len(pifu.KERNEL_CLASSES) == classes.pop("count")
    for name, idx in classes.items():
        assert pifu.KERNEL_CLASSES[idx] == name, (name, idx)


def test_status_strings():
    assert pifu.pifu_status_string(0) == "ok"
    assert "converge" in pifu.pifu_status_string(pifu.PIFU_ERR_NOT_CONVERGED)


def test_create_rejects_malformed_blobs_without_a_gpu():
    lib = pifu.load()
    ctx = ctypes.c_void_p()
    for blob in (b"", b"XXXX" + struct.pack("<II", 1, 2), b"PIFU" + struct.pack("<II", 2, 2),
                 b"PIFU" + struct.pack("<II", 1, 2) + b"\x00" * 7):
        buf = ctypes.create_string_buffer(blob, max(1, len(blob)))
        st = lib.pifu_create(buf, len(blob), ctypes.byref(ctx))
        # malformed headers are rejected before any device work
        assert st == pifu.PIFU_ERR_FORMAT, (blob, st)
    assert lib.pifu_create(None, 0, ctypes.byref(ctx)) == pifu.PIFU_ERR_ARG
    assert lib.pifu_create(None, 0, None) == pifu.PIFU_ERR_ARG


def test_blob_layout_matches_header_description():
    w = synth.tiny(0)
    blob = pifu.blob_from_nets(w.occ_net, w.col_net)
    assert blob[:4] == b"PIFU"
    version, n_nets = struct.unpack_from("<II", blob, 4)
    assert (version, n_nets) == (1, 2)
    kind, d_in, L, slope = struct.unpack_from("<IIIf", blob, 12)
    assert (kind, d_in, L) == (0, 33, 3) and abs(slope - 0.01) < 1e-9
    widths = struct.unpack_from("<3I", blob, 28)
    assert widths == (128, 64, 1)
    n_params = sum(W.size + b.size for W, b in zip(w.occ_net.W, w.occ_net.b))
    n_params_c = sum(W.size + b.size for W, b in zip(w.col_net.W, w.col_net.b))
    header = 12 + 2 * (16 + 3 * 4 + 4)
    assert len(blob) == header + 4 * (n_params + n_params_c)


def test_null_arguments_are_rejected_on_the_host():
    lib = pifu.load()
    calib = (ctypes.c_float * 12)()
    assert lib.pifu_query(None, None, calib, None, 1, None, None) == pifu.PIFU_ERR_ARG
    assert lib.pifu_localize(None, None, calib, None, None, None) == pifu.PIFU_ERR_ARG
    assert lib.pifu_render(None, None, None, None, calib, None, None, None, None) == pifu.PIFU_ERR_ARG
    assert lib.pifu_sync_stats(None, None) == pifu.PIFU_ERR_ARG
    codes = (ctypes.c_int32 * 1)(256)
    assert lib.pifu_set_tiles(None, codes, 1) == pifu.PIFU_ERR_ARG
    assert lib.pifu_set_schedule(None, pifu.PIFU_SCHED_CHAINED) == pifu.PIFU_ERR_ARG
    assert lib.pifu_set_recheck(None, pifu.PIFU_RECHECK_SIMT) == pifu.PIFU_ERR_ARG
    assert lib.pifu_test_starve_wait(None, 1) == pifu.PIFU_ERR_ARG
    lib.pifu_destroy(None)


def test_unpack_bits_row_layout():
    n = 40
    rw = (n + 1 + 31) // 32
    rng = np.random.default_rng(0)
    ref = rng.random((n + 1, n + 1, n + 1)) < 0.3
    words = np.zeros((n + 1, n + 1, rw), dtype=np.uint32)
    for i in range(n + 1):
        words[:, :, i >> 5] |= ref[:, :, i].astype(np.uint32) << np.uint32(i & 31)
    np.testing.assert_array_equal(pifu.unpack_bits(words.view(np.int32).ravel(), n, rw), ref)
