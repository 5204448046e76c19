"""GPU shards of one query (the multi-GPU split, run here one after another
on one GPU): each shard equals the oracle's top-k of the triangles it owns,
and the merged shards equal the whole query."""
import math

import numpy as np
import pytest

import oracle
import synth
from wtri_testutil import PS, assert_topk_equal

pytestmark = pytest.mark.gpu

wt = pytest.importorskip("paper_1910_00692_gb300")


@pytest.mark.parametrize("n,m,seed", [(2000, 20000, 0), (100000, 1000000, 12)])
@pytest.mark.parametrize("nshards", [2, 3])
def test_shards(n, m, seed, nshards):
    g = synth.tiny_graph(0) if n == 2000 else synth.scaled_mid_graph(n, m, seed=seed)
    d = wt.build_csr(g.n, g.u, g.v, g.w)
    try:
        for p in PS:
            k = 500
            parts = []
            for sh in range(nshards):
                t, w, kk = wt.topk_shard(d, p, k, sh, nshards)
                want = oracle.topk_shard(g.n, g.u, g.v, g.w, p, k, sh, nshards)
                assert_topk_equal(t, w, want, p, f"shard {sh}/{nshards} p={p}")
                assert np.array_equal(kk, want["key"])
                parts.append((t, w, kk))
            mt, mw, mk = wt.merge_topk(parts, k)
            ft, fw = d.topk(p, k)
            assert np.array_equal(mt, ft) and np.array_equal(mw, fw)
    finally:
        d.free()


def test_shard_rule_hand_built():
    """wtri_topk_shard gives each shard exactly the triangles the hand-built
    pin lists (ownership by the first edge's 1024-position chunk)."""
    import shard_pin
    n, u, v, w = shard_pin.graph()
    d = wt.build_csr(n, u, v, w)
    try:
        for nsh, want in shard_pin.EXPECTED.items():
            for sh in range(nsh):
                for p in PS:
                    t, _, _ = wt.topk_shard(d, p, 100, sh, nsh)
                    got = sorted(tuple(int(x) for x in row) for row in t)
                    assert got == sorted(want[sh]), (nsh, sh, p, got)
    finally:
        d.free()


def _dist_rank(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    import paper_1910_00692_gb300 as wt_
    from paper_1910_00692_gb300 import distributed
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    g = synth.tiny_graph(0)
    d = wt_.build_csr(g.n, g.u, g.v, g.w)
    ok = True
    for p in PS:
        for k in (1, 300, 5000):
            t, w, kk = distributed.topk_distributed(d, p, k)
            want = oracle.topk(g.n, g.u, g.v, g.w, p, k)
            ok = ok and np.array_equal(t, want["tri"]) and np.array_equal(kk, want["key"])
            ok = ok and np.allclose(w, want["value"], rtol=1e-12, atol=0.0)
    d.free()
    with open(f"{out_dir}/rank{rank}.txt", "w") as f:
        f.write("ok" if ok else "mismatch")
    dist.destroy_process_group()


def test_topk_distributed_two_ranks(tmp_path):
    """The multi-GPU path end to end (each rank its own replica and shard,
    the fixed-size all-gather, the host merge), as two processes sharing the
    one GPU over a gloo group: the ranks' kernels never wait on one another,
    only the host-side gather does."""
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mp.start_processes(_dist_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    for r in range(2):
        assert (tmp_path / f"rank{r}.txt").read_text() == "ok"
