"""The library's graph API (mcc_graph_begin / end / launch / destroy): a
batch of fields with uneven bounds, compressed and decompressed, recorded
once and replayed as one graph, gives the eager batch's streams and values
bit for bit on every replay; misuse is reported, not faulted."""
import numpy as np
import pytest
import torch

import paper_2501_06910_gb300 as mcc
import synth

pytestmark = pytest.mark.gpu


def _setup():
    coords, cells = synth.mesh2d_jittered(nside=60, seed=3)
    dev = torch.device("cuda", 0)
    plan = mcc.plan_create(torch.from_numpy(coords).to(dev), torch.from_numpy(cells).to(dev),
                           (48, 40))
    xs = [torch.from_numpy(synth.field_sincos(coords, seed=10 + k)).to(dev) for k in range(3)]
    prms = [mcc.params_default(dtype=mcc.F64, eb=eb, grid_fraction=0.5)
            for eb in (1e-5, 1e-3, 1e-2)]
    return plan, xs, prms


def _buffers(plan, prms, xs):
    cws = max(mcc.workspace_size(plan, p)[0] for p in prms)
    dws = max(mcc.workspace_size(plan, p)[1] for p in prms)
    slot = (max(mcc.compress_bound(plan, p) for p in prms) + 7) // 8 * 8
    n = len(xs)
    dev = xs[0].device
    return (slot, torch.zeros(slot * n, dtype=torch.uint8, device=dev),
            torch.empty(cws * n, dtype=torch.uint8, device=dev),
            torch.empty(dws * n, dtype=torch.uint8, device=dev),
            [torch.empty_like(x) for x in xs])


def test_graph_replays_a_batch_bit_exactly():
    plan, xs, prms = _setup()
    slot, out, wsc, wsd, ys = _buffers(plan, prms, xs)
    sizes = mcc.compress_batch(plan, xs, prms, wsc, out, slot)
    mcc.decompress_batch(plan, out, slot, sizes, ys, wsd)
    ref_out = out.clone()
    ref_ys = [y.clone() for y in ys]
    for x, y, p in zip(xs, ys, prms):
        tau = p.eb * float(x.max() - x.min())
        assert float((y - x).abs().max()) <= tau
    slot2, out2, wsc2, wsd2, ys2 = _buffers(plan, prms, xs)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())

    def record():
        mcc.compress_batch(plan, xs, prms, wsc2, out2, slot2, sync=False, stream=s)
        mcc.decompress_batch(plan, out2, slot2, [slot2] * len(xs), ys2, wsd2, sync=False,
                             stream=s)

    g = mcc.graph_capture(record, s)
    try:
        for _ in range(2):  # every replay gives the same result
            out2.zero_()
            for y in ys2:
                y.fill_(float("nan"))
            g.launch(s)
            s.synchronize()
            for f, size in enumerate(sizes):
                assert torch.equal(out2[f * slot2:f * slot2 + size], ref_out[f * slot:f * slot + size])
                assert torch.equal(ys2[f], ref_ys[f])
    finally:
        g.close()
        plan.close()


def test_graph_misuse_is_an_error():
    with pytest.raises(mcc.MCCError) as e:
        mcc.graph_begin(torch.cuda.default_stream())  # the legacy default stream
    assert e.value.status == mcc.INVALID_ARG
    s = torch.cuda.Stream()
    with pytest.raises(mcc.MCCError) as e:
        mcc.graph_end(s)  # nothing recorded
    assert e.value.status == mcc.INVALID_ARG
    mcc.graph_begin(s)
    with pytest.raises(mcc.MCCError) as e:
        mcc.graph_begin(s)  # no nested recording
    assert e.value.status == mcc.INVALID_ARG
    g = mcc.graph_end(s)  # an empty recording is a valid (empty) graph
    g.launch(s)
    s.synchronize()
    g.close()
