"""Multi-rank logic on CPU ranks (gloo, world size 2): the equal-work row-block partition
of one set (the shard a rank would take) and the bench's aggregation over ranks.  Each
rank computes its block with the oracle; the union of the blocks must equal the
single-rank result, and the aggregate must be the max time and the summed units."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import bench
    from oracle import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ps = synth.families_1k().subset(np.arange(160))
    mat = synth.blosum62()
    codes = O.encode(ps.ascii)
    rp, code, pos = O.kmers(codes, ps.offsets, 6)
    cands = O.candidates(rp, code, pos, 6, 0, mat, 1)
    blocks = bench.row_blocks(ps.n, world)
    i0, i1 = blocks[rank]
    mine = cands[(cands["i"] >= i0) & (cands["i"] < i1)]
    alns, _ = O.align_pairs(codes, ps.offsets, mine, mat)
    edges = O.filter_edges(ps.offsets, mine, alns)
    gathered = [None] * world
    dist.all_gather_object(gathered, edges.tobytes())
    ms, units = bench.combine_ranks(10.0 * (rank + 1), len(edges), world, dist)
    if rank == 0:
        allb = b"".join(gathered)
        ref = O.run(ps.ascii, ps.offsets, mat)["edges"].tobytes()
        sizes = [len(g) for g in gathered]
        with open(os.path.join(out_dir, "result.txt"), "w") as f:
            f.write(f"{int(allb == ref)} {ms} {units} {sum(sizes) // 20} {len(ref) // 20}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_row_blocks_equal_work_and_cover():
    import bench
    for n, b in ((10, 3), (1000, 8), (100_000, 8), (5, 5), (1, 1)):
        blocks = bench.row_blocks(n, b)
        assert blocks[0][0] == 0 and blocks[-1][1] == n
        assert all(blocks[k][1] == blocks[k + 1][0] for k in range(b - 1))
        work = [sum(n - 1 - i for i in range(a, c)) for a, c in blocks]
        if n >= 1000:
            assert max(work) - min(work) <= 2 * n   # a boundary moves by at most one row


def test_two_gloo_ranks_partition_the_job(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    ok, ms, units, got, want = open(tmp_path / "result.txt").read().split()
    assert ok == "1"
    assert float(ms) == 20.0
    assert int(float(units)) == int(got) == int(want)
