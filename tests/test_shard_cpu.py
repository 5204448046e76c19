"""The multi-GPU split of a query, on CPU: two gloo ranks each hold one
shard's exact top-k (computed here by the oracle restricted to the
triangles the shard owns), exchange them with one all-gather and merge them
with the library's host merge (wtri_merge_topk).  The merged answer must
equal the oracle's top-k of the whole graph."""
import math
import os
import socket

import numpy as np
import pytest

import oracle
import synth

PS = [-math.inf, 1.0, 2.0, math.inf]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_shards_partition_the_triangles():
    g = synth.tiny_graph(0)
    for nsh in (1, 2, 3, 5):
        total = sum(oracle.topk_shard(g.n, g.u, g.v, g.w, 1.0, 10, s, nsh)["ntri"] for s in range(nsh))
        assert total == oracle.count_triangles(g.n, g.u, g.v)


def test_shard_rule_hand_built():
    """The ownership rule itself, on a graph whose per-shard triangles are
    written out by hand (tests/shard_pin.py)."""
    import shard_pin
    n, u, v, w = shard_pin.graph()
    for nsh, want in shard_pin.EXPECTED.items():
        for sh in range(nsh):
            r = oracle.topk_shard(n, u, v, w, 1.0, 100, sh, nsh)
            got = sorted(tuple(int(x) for x in t) for t in r["tri"])
            assert got == sorted(want[sh]), (nsh, sh, got)


def test_host_merge():
    wt = pytest.importorskip("paper_1910_00692_gb300")
    from paper_1910_00692_gb300 import build_lib
    build_lib.build()
    a = (np.array([[0, 1, 2], [3, 4, 5]]), np.array([5.0, 3.0]), np.array([15, 9], dtype=np.uint64))
    b = (np.array([[1, 2, 3], [0, 4, 6]]), np.array([5.0, 4.0]), np.array([15, 12], dtype=np.uint64))
    t, w, k = wt.merge_topk([a, b], 3)
    assert t.tolist() == [[0, 1, 2], [1, 2, 3], [0, 4, 6]]
    assert k.tolist() == [15, 15, 12]
    t, w, k = wt.merge_topk([a, b, (np.zeros((0, 3)), np.zeros(0), np.zeros(0, np.uint64))], 10)
    assert t.shape[0] == 4
    with pytest.raises(wt.WtriError):
        wt.merge_topk([a, a], 3)  # a triangle in two parts


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    from paper_1910_00692_gb300 import distributed
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    g = synth.tiny_graph(0)
    ok = True
    for p in PS:
        for k in (1, 100, 999):
            r = oracle.topk_shard(g.n, g.u, g.v, g.w, p, k, rank, world)
            merged = distributed.merge_across_ranks((r["tri"], r["value"], r["key"]), k)
            want = oracle.topk(g.n, g.u, g.v, g.w, p, k)
            same = (np.array_equal(merged[0], want["tri"]) and np.array_equal(merged[1], want["value"])
                    and np.array_equal(merged[2], want["key"]))
            ok = ok and same
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write("ok" if ok else "mismatch")
    dist.destroy_process_group()


def test_gloo_two_ranks(tmp_path):
    pytest.importorskip("torch.distributed")
    import torch.multiprocessing as mp
    from paper_1910_00692_gb300 import build_lib
    build_lib.build()
    oracle.build()
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    for r in range(2):
        assert (tmp_path / f"rank{r}.txt").read_text() == "ok"


def test_pack_roundtrip():
    """The fixed-size exchange buffer carries counts, triples, fp64 weights
    and 64-bit keys bit for bit, short parts padded."""
    from paper_1910_00692_gb300 import distributed
    t = np.array([[0, 1, 2], [5, 6, 7]], np.int32)
    w = np.array([1.0 / 3.0, 2.0 ** -1074], np.float64)
    kk = np.array([2 ** 64 - 1, 12], np.uint64)
    buf = distributed.pack_part((t, w, kk), 4)
    assert buf.shape == (21,) and buf.dtype == np.int64
    t2, w2, k2 = distributed.unpack_part(buf, 4)
    assert np.array_equal(t2, t) and np.array_equal(w2.view(np.int64), w.view(np.int64))
    assert np.array_equal(k2, kk)
    t3, w3, k3 = distributed.unpack_part(distributed.pack_part((t[:0], w[:0], kk[:0]), 4), 4)
    assert t3.shape == (0, 3) and w3.shape == (0,) and k3.shape == (0,)
