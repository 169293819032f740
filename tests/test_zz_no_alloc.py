"""pifu_query_noalloc: the context-free, allocation-free occupancy query for
callers that cannot call cudaMalloc (its activation scratch is a fixed
device array inside the library).  Called through the C ABI and compared
with pifu_query on the same inputs, twice in a row, so that the second call
also shows that the shared scratch's leftovers from the first do not leak
into the result.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2007_13988_gb300 import pifu, synth

from gpu_common import OCC_TOL, to_dev

pytestmark = pytest.mark.gpu


def call_noalloc(lib, blob, blob_dev, occ, calib, pts, out):
    buf = ctypes.create_string_buffer(blob, len(blob))
    fm = pifu.fmap(occ)
    c = (ctypes.c_float * 12)(*np.asarray(calib, np.float32).ravel().tolist())
    return lib.pifu_query_noalloc(buf, len(blob), ctypes.c_void_p(blob_dev.data_ptr()),
                                  ctypes.byref(fm), c, ctypes.c_void_p(pts.data_ptr()),
                                  pts.shape[0], ctypes.c_void_p(out.data_ptr()), None)


def m_max(net):
    # the fixed scratch holds 4194304 floats: one gather row (d_in rounded
    # up to 8) and two rows of the widest hidden layer per point
    ldx = (net.d_in + 7) // 8 * 8
    h = max(8, max(net.widths[:-1]))
    return 4194304 // (ldx + 2 * h)


@pytest.mark.parametrize("which", ["tiny", "full"])
def test_noalloc_query_matches_pifu_query(which):
    import torch
    w = synth.tiny(0) if which == "tiny" else synth.full(0)
    m = m_max(w.occ_net)
    assert m == {"tiny": 14169, "full": 1814}[which]
    lib = pifu.load()
    blob = pifu.blob_from_nets(w.occ_net, w.col_net)
    # the caller owns every device buffer, the weights' device copy included
    blob_dev = torch.frombuffer(bytearray(blob), dtype=torch.uint8).cuda()
    occ = to_dev(w.occ_map)
    ctx = pifu.pifu_create(blob)
    try:
        # two calls in a row: the largest allowed batch, then a ragged one
        for call, (seed, n) in enumerate(((11, m), (12, m // 3 + 7))):
            P = synth.query_points(n, seed=seed) * np.float32(1.1)
            pts = to_dev(P)
            ref = torch.empty(n, dtype=torch.float32, device="cuda")
            pifu.pifu_query(ctx, occ, w.calib, pts, ref)
            out = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
            st = call_noalloc(lib, blob, blob_dev, occ, w.calib, pts, out)
            assert st == pifu.PIFU_OK, (call, st)
            torch.cuda.synchronize()
            err = float(torch.max(torch.abs(out - ref)).item())
            assert err <= OCC_TOL, (call, err)
    finally:
        pifu.pifu_destroy(ctx)


def test_noalloc_rejects_batches_beyond_the_scratch():
    import torch
    w = synth.full(0)
    blob = pifu.blob_from_nets(w.occ_net, w.col_net)
    blob_dev = torch.frombuffer(bytearray(blob), dtype=torch.uint8).cuda()
    occ = to_dev(w.occ_map)
    n = m_max(w.occ_net) + 1
    pts = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    out = torch.zeros(n, dtype=torch.float32, device="cuda")
    st = call_noalloc(pifu.load(), blob, blob_dev, occ, w.calib, pts, out)
    assert st == pifu.PIFU_ERR_ARG
    assert float(out.abs().max().item()) == 0.0   # nothing was written
