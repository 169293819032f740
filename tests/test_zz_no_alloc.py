"""pifu_query_noalloc: the context-free, allocation-free occupancy query for
callers that cannot call cudaMalloc (an application whose own allocator
owns the device memory, or code where device allocation is not permitted).
Its activation scratch is a fixed device array inside the library.

Called through the C ABI and compared, twice in a row, with the FP64 oracle
and with pifu_query on the same inputs, so that the second call also shows
that the shared scratch's leftovers from the first do not leak into the
result; the device's free memory is the same before and after the second
call.  A network with odd hidden widths and another skip pattern (which
pifu_create refuses) is compared with the oracle alone, and the first call
of a fresh process under lazy module loading is checked on its own.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from oracle import field
from paper_2007_13988_gb300 import pifu, synth

from gpu_common import OCC_TOL, to_dev

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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
def test_noalloc_query_matches_oracle_and_pifu_query(which):
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
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            st = call_noalloc(lib, blob, blob_dev, occ, w.calib, pts, out)
            assert st == pifu.PIFU_OK, (call, st)
            torch.cuda.synchronize()
            free1 = torch.cuda.mem_get_info()[0]
            if call == 1:
                assert free1 == free0, (free0, free1)   # nothing allocated
            got = out.cpu().numpy().astype(np.float64)
            want = field.occupancy(w.occ_net, w.occ_map, w.calib, P)
            assert np.max(np.abs(got - want)) <= OCC_TOL, (call, np.max(np.abs(got - want)))
            err = float(torch.max(torch.abs(out - ref)).item())
            assert err <= OCC_TOL, (call, err)
    finally:
        pifu.pifu_destroy(ctx)


def odd_net(d_in, seed):
    """An occupancy MLP d_in -> 37 -> 19 -> 1 with the input re-read by the
    last layer only: hidden widths that are not multiples of 4 (so the second
    scratch row block starts off a 16-byte boundary for odd m) and a skip
    pattern the synthetic networks do not have."""
    rng = np.random.default_rng(seed)
    widths, skip = (37, 19, 1), (2,)
    Ws, bs = [], []
    for l, n_out in enumerate(widths):
        fan = (d_in if l == 0 else widths[l - 1]) + (d_in if l in skip else 0)
        Ws.append(rng.uniform(-1, 1, (n_out, fan)).astype(np.float32) * np.float32(np.sqrt(3.0 / fan)))
        bs.append(rng.uniform(-0.1, 0.1, n_out).astype(np.float32))
    return synth.Net(d_in=d_in, widths=widths, skip=skip, W=Ws, b=bs, out_act="sigmoid")


def test_noalloc_odd_widths_and_skip_mask():
    import torch
    w = synth.tiny(0)
    net = odd_net(w.occ_net.d_in, 5)
    m = m_max(net)
    # with m - 1 points the second hidden block starts off a 16-byte boundary
    assert (m - 1) * (40 + 37) % 4 != 0
    lib = pifu.load()
    blob = pifu.blob_from_nets(net, w.col_net)
    blob_dev = torch.frombuffer(bytearray(blob), dtype=torch.uint8).cuda()
    occ = to_dev(w.occ_map)
    for n in (m - 1, m):
        P = synth.query_points(n, seed=40 + n) * np.float32(1.1)
        pts = to_dev(P)
        out = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        assert call_noalloc(lib, blob, blob_dev, occ, w.calib, pts, out) == pifu.PIFU_OK
        torch.cuda.synchronize()
        want = field.occupancy(net, w.occ_map, w.calib, P)
        assert np.max(np.abs(out.cpu().numpy() - want)) <= OCC_TOL
    pts = torch.zeros((m + 1, 3), dtype=torch.float32, device="cuda")
    out = torch.zeros(m + 1, dtype=torch.float32, device="cuda")
    assert call_noalloc(lib, blob, blob_dev, occ, w.calib, pts, out) == pifu.PIFU_ERR_ARG


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


def test_noalloc_first_call_of_a_fresh_process():
    """With lazy module loading, the first call of a process loads the
    library's device code and scratch array itself: made before any other
    call of the library, it still gives the oracle's occupancies, twice."""
    script = textwrap.dedent("""
        import ctypes, sys
        sys.path.insert(0, %r)
        sys.path.insert(0, %r)
        import numpy as np, torch
        from oracle import field
        from paper_2007_13988_gb300 import pifu, synth
        from test_zz_no_alloc import call_noalloc
        w = synth.tiny(0)
        blob = pifu.blob_from_nets(w.occ_net, w.col_net)
        blob_dev = torch.frombuffer(bytearray(blob), dtype=torch.uint8).cuda()
        occ = torch.from_numpy(w.occ_map).cuda()
        lib = pifu.load()
        for seed, n in ((3, 5000), (4, 777)):
            P = synth.query_points(n, seed=seed)
            pts = torch.from_numpy(P).cuda()
            out = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
            st = call_noalloc(lib, blob, blob_dev, occ, w.calib, pts, out)
            assert st == pifu.PIFU_OK, st
            torch.cuda.synchronize()
            want = field.occupancy(w.occ_net, w.occ_map, w.calib, P)
            err = float(np.max(np.abs(out.cpu().numpy() - want)))
            assert err <= %r, err
        print("fresh-process noalloc ok")
    """) % (ROOT, os.path.join(ROOT, "tests"), OCC_TOL)
    env = dict(os.environ, CUDA_MODULE_LOADING="LAZY")
    r = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "fresh-process noalloc ok" in r.stdout
