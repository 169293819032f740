"""Asynchronous frames (pifu_frame_async / pifu_frame_wait): the same graph as
pifu_frame, enqueued without the host waiting.  Checked for equality with the
synchronous call bit for bit, for stream order across frames with new
inputs, against the FP64 oracle, and for the latched device-side error and
the context's recovery after it."""
import numpy as np
import pytest

from oracle import field, localize, metrics
from paper_2007_13988_gb300 import pifu, synth

from gpu_common import Ctx

pytestmark = pytest.mark.gpu

R = 64


def outputs():
    import torch
    return (torch.empty((R, R), dtype=torch.float32, device="cuda"),
            torch.empty((R, R, 3), dtype=torch.float32, device="cuda"),
            torch.empty((R, R), dtype=torch.uint8, device="cuda"))


def host(t):
    return t.cpu().numpy()


def same(a, b):
    return np.array_equal(np.nan_to_num(a, nan=-7.0), np.nan_to_num(b, nan=-7.0))


@pytest.fixture(scope="module")
def tiny():
    c = Ctx(synth.tiny(0))
    yield c
    c.close()


def frame_args(c, depth, rgb, mask, **kw):
    w = c.w
    return (c.ctx, c.occ, c.col, w.calib, w.n0, w.num_levels, R, R, depth, rgb, mask), kw


def test_async_frames_follow_stream_order_and_equal_sync_frames(tiny):
    import torch
    c, w = tiny, tiny.w
    w5 = synth.tiny(5)
    map_a = c.occ.clone()
    map_b = torch.from_numpy(w5.occ_map).cuda()
    depth, rgb, mask = outputs()
    a, kw = frame_args(c, depth, rgb, mask, precision=pifu.PIFU_PREC_MIXED)
    # the synchronous frame on each map
    ref = []
    for m in (map_a, map_b):
        c.occ.copy_(m)
        vol = pifu.pifu_frame(*a, **kw)
        torch.cuda.synchronize()
        ref.append((host(depth), host(rgb), host(mask), c.volume_host(vol), int(vol.n_eval)))
    # two asynchronous frames, the map replaced in between on the same
    # stream, frame 1's outputs copied aside before frame 2 overwrites them
    s = torch.cuda.current_stream()
    side = [t.clone() for t in (depth, rgb, mask)]
    c.occ.copy_(map_a)
    pifu.pifu_frame_async(*a, **kw)
    for dst, src in zip(side, (depth, rgb, mask)):
        dst.copy_(src)
    c.occ.copy_(map_b)
    pifu.pifu_frame_async(*a, **kw)
    vol = pifu.pifu_frame_wait(c.ctx, s)
    got_a = [host(t) for t in side]
    for g, r in zip(got_a, ref[0][:3]):
        assert same(g, r)
    for g, r in zip((host(depth), host(rgb), host(mask)), ref[1][:3]):
        assert same(g, r)
    b, e, v = c.volume_host(vol)
    rb, re_, rv = ref[1][3]
    assert np.array_equal(b, rb) and np.array_equal(e, re_)
    assert np.array_equal(v[e], rv[e])
    assert int(vol.n_eval) == ref[1][4]
    # and frame 2 is the method's result on map b (oracle, FP64)
    lv = localize.hierarchical(lambda P: field.occupancy(w.occ_net, w5.occ_map, w.calib, P),
                               w.n0, w.num_levels)
    assert metrics.iou(b, lv[-1].binary) >= 0.99
    c.occ.copy_(map_a)


def test_async_error_is_latched_and_the_context_recovers(tiny):
    import torch
    c = tiny
    depth, rgb, mask = outputs()
    a, kw = frame_args(c, depth, rgb, mask, precision=pifu.PIFU_PREC_MIXED)
    vol = pifu.pifu_frame(*a, **kw)
    torch.cuda.synchronize()
    ref = (host(depth), host(rgb), host(mask), int(vol.n_eval))
    s = torch.cuda.current_stream()
    with pytest.raises(pifu.PifuError) as ei:
        pifu.pifu_frame_wait(c.ctx, s)             # nothing pending
    assert ei.value.status == pifu.PIFU_ERR_STATE
    # a round cap the frame exceeds: the call returns, the wait reports it,
    # also when a good frame ran after the failing one
    pifu.pifu_frame_async(*a, max_rounds=1, **kw)
    pifu.pifu_frame_async(*a, **kw)
    with pytest.raises(pifu.PifuError) as ei:
        pifu.pifu_frame(*a, **kw)                  # frames pending: refused, nothing enqueued
    assert ei.value.status == pifu.PIFU_ERR_STATE
    with pytest.raises(pifu.PifuError) as ei:
        pifu.pifu_frame_wait(c.ctx, s)
    assert ei.value.status == pifu.PIFU_ERR_NOT_CONVERGED
    # cleared: the next frames run and equal the synchronous one
    pifu.pifu_frame_async(*a, **kw)
    pifu.pifu_frame_async(*a, **kw)
    vol = pifu.pifu_frame_wait(c.ctx, s)
    assert int(vol.n_eval) == ref[3]
    for g, r in zip((host(depth), host(rgb), host(mask)), ref[:3]):
        assert same(g, r)
    vol = pifu.pifu_frame(*a, **kw)                # and the synchronous call again
    torch.cuda.synchronize()
    assert int(vol.n_eval) == ref[3]


def test_async_host_errors_enqueue_nothing(tiny):
    import torch
    c = tiny
    depth, rgb, mask = outputs()
    a, kw = frame_args(c, depth, rgb, mask, precision=pifu.PIFU_PREC_FP32)
    with pytest.raises(pifu.PifuError) as ei:
        pifu.pifu_frame_async(*a, **kw)            # the graph has no FP32 form
    assert ei.value.status == pifu.PIFU_ERR_UNSUPPORTED
    with pytest.raises(pifu.PifuError) as ei:
        pifu.pifu_frame_wait(c.ctx, torch.cuda.current_stream())
    assert ei.value.status == pifu.PIFU_ERR_STATE


def test_destroy_with_frames_pending():
    # pifu_destroy waits for the frames still in flight before it releases
    # their graph and buffers; a context made afterwards works as before
    import torch
    w = synth.tiny(0)
    c = Ctx(w)
    depth, rgb, mask = outputs()
    a, kw = frame_args(c, depth, rgb, mask, precision=pifu.PIFU_PREC_MIXED)
    vol = pifu.pifu_frame(*a, **kw)
    torch.cuda.synchronize()
    ref = (host(depth), host(mask), int(vol.n_eval))
    for _ in range(3):
        pifu.pifu_frame_async(*a, **kw)
    c.close()                                      # frames pending
    torch.cuda.synchronize()
    for g, r in zip((host(depth), host(mask)), ref[:2]):
        assert same(g, r)                          # the frames ran to the end
    c2 = Ctx(w)
    try:
        a2, kw2 = frame_args(c2, depth, rgb, mask, precision=pifu.PIFU_PREC_MIXED)
        vol = pifu.pifu_frame(*a2, **kw2)
        torch.cuda.synchronize()
        assert int(vol.n_eval) == ref[2]
        assert same(host(depth), ref[0])
    finally:
        c2.close()

