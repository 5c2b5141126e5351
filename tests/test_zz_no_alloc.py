"""gs_tile_queue_static: the tile queue for callers that cannot allocate
device memory (a fixed pool owned by a host application, a latency-critical
thread where cudaMalloc would synchronise the device, a path that must not
allocate).  It runs in a scratch array the library keeps in device memory,
so it must give exactly what gs_tile_queue gives with a caller workspace,
call after call, even though every call reuses the same array.

This file is collected last so that a run stopping at the first failure has
run every other test before it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _ranges(lengths, seed):
    """Per-tile [start, end) ranges with the given list lengths, in a random
    tile order (as a pair sort produces them)."""
    rng = np.random.default_rng(seed)
    T = len(lengths)
    perm = rng.permutation(T)
    starts = np.zeros(T, np.int64)
    starts[perm] = np.concatenate([[0], np.cumsum(lengths[perm])[:-1]])
    r = np.stack([starts, starts + lengths], 1).astype(np.uint32).view(np.int32)
    return torch.as_tensor(r).cuda().contiguous()


def _queue(gs, ranges, T):
    ws = torch.empty(gs.gs_tile_queue_workspace_size(T), dtype=torch.uint8, device="cuda")
    out = torch.empty(T, dtype=torch.int32, device="cuda")
    gs.gs_tile_queue(ranges, T, out, ws)
    return out


@pytest.mark.parametrize("T", [4056, 65536])
def test_static_queue_matches_workspace_queue_on_consecutive_calls(T):
    from paper_2603_09277_gb300 import gs
    rng = np.random.default_rng(T)
    outs = []
    for call in range(2):
        # many equal lengths so that the tie order (by tile id) is exercised
        lengths = rng.integers(0, 40 if call == 0 else 2000, T)
        ranges = _ranges(lengths, seed=T + call)
        ref = _queue(gs, ranges, T)
        got = torch.full((T,), -1, dtype=torch.int32, device="cuda")
        assert gs.gs_tile_queue_static(ranges, T, got) == gs.GS_OK
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
        ln = lengths[got.cpu().numpy()]
        assert (np.diff(ln) <= 0).all()
        outs.append(got.cpu().numpy())
    assert not np.array_equal(outs[0], outs[1])


def test_static_queue_rejects_more_tiles_than_its_scratch_holds():
    from paper_2603_09277_gb300 import gs
    T = 65537
    ranges = torch.zeros(T, 2, dtype=torch.int32, device="cuda")
    out = torch.zeros(T, dtype=torch.int32, device="cuda")
    assert gs.gs_tile_queue_static(ranges, T, out) == gs.GS_ERR_INVALID_ARG
    assert "65536" in gs.gs_last_error_string()
    torch.cuda.synchronize()
    assert int(out.abs().sum().item()) == 0


def test_static_queue_allocates_nothing_and_follows_its_stream():
    """After a first call (which looks up the scratch address), a call leaves
    the device's free memory unchanged; a call enqueued on a non-default
    stream, ordered after the inputs by an event, gives the same order."""
    from paper_2603_09277_gb300 import gs
    T = 4056
    lengths = np.random.default_rng(7).integers(0, 300, T)
    ranges = _ranges(lengths, seed=7)
    ref = _queue(gs, ranges, T)
    got = torch.full((T,), -1, dtype=torch.int32, device="cuda")
    assert gs.gs_tile_queue_static(ranges, T, got) == gs.GS_OK  # warm-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert gs.gs_tile_queue_static(ranges, T, got) == gs.GS_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(got, ref)
    # on a side stream, after an event that follows the inputs' writes
    s = torch.cuda.Stream()
    side = torch.full((T,), -1, dtype=torch.int32, device="cuda")
    ranges2 = ranges.clone()
    ready = torch.cuda.Event()
    ready.record()
    s.wait_event(ready)
    assert gs.gs_tile_queue_static(ranges2, T, side, stream=s) == gs.GS_OK
    done = torch.cuda.Event()
    done.record(s)
    torch.cuda.current_stream().wait_event(done)
    assert torch.equal(side, ref)
