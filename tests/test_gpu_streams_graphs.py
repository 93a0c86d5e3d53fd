"""The entry points on a non-default stream and captured into a CUDA graph: the same bytes as
eager launches on the default stream (the library synchronises nothing and allocates nothing,
so every call can be captured and replayed)."""
import numpy as np
import pytest

from paper_1308_1419_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1308_1419_gb300 import td  # noqa: E402


def _calls():
    N, n = 3000, 2500
    x3 = torch.from_numpy(synth.uniform_points(n, 3, 61)).cuda()
    x64 = torch.from_numpy(synth.uniform_points(700, 64, 62)).cuda()
    c, r = synth.spheres(2000, seed=63, coord_bits=12, rmin=0, rmax=300)
    ct, rt = torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda()
    probe = torch.empty(N * (N + 1) // 2, dtype=torch.int32, device="cuda")
    e_chunk = torch.empty(n * (n + 1) // 2, dtype=torch.float32, device="cuda")
    e_tile = torch.empty(700 * 701 // 2, dtype=torch.float32, device="cuda")
    e_strict = torch.empty(n * (n - 1) // 2, dtype=torch.float32, device="cuda")
    table = torch.empty(td.td_collide_words(2000), dtype=torch.int32, device="cuda")
    xg = torch.from_numpy(synth.uniform_points(600, 128, 64)).cuda()
    e_gram = torch.empty(600 * 601 // 2, dtype=torch.float32, device="cuda")
    ws = torch.empty(td.td_edm_gram_workspace(600, 128) + 1024, dtype=torch.uint8, device="cuda")
    outs = [probe, e_chunk, e_tile, e_strict, table, e_gram]

    def run(stream=None):
        td.td_map_probe("LTM", "chunked", N, 16, probe, stream=stream)
        td.td_edm("LTM", "chunked", x3, 16, e_chunk, stream=stream)
        td.td_edm("UTM-BLOCK", "persistent", x64, 128, e_tile, stream=stream)
        td.td_edm_strict(x3, e_strict, stream=stream)
        td.td_collide("LTM", "grid", ct, rt, table, stream=stream)
        td.td_edm_gram(xg, e_gram, ws, stream=stream)
    return run, outs


def test_side_stream_matches_default_stream():
    run, outs = _calls()
    run()
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs]
    for o in outs:
        o.fill_(-1)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    run(stream=side)
    side.synchronize()
    for a, b in zip(outs, ref):
        assert torch.equal(a, b)


def test_graph_capture_replays_the_same_bytes():
    run, outs = _calls()
    run()
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        run()
    for o in outs:
        o.fill_(-1)
    graph.replay()
    torch.cuda.synchronize()
    for a, b in zip(outs, ref):
        assert torch.equal(a, b)
