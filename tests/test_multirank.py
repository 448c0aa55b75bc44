"""Multi-rank logic on CPU ranks (gloo, world size 2): the bench's split of one job into
equal-work row blocks and its assignment of blocks to ranks (bench.rank_blocks), and the
bench's aggregation over ranks.  Each rank computes its blocks with the oracle; the
blocks in order must equal the single-rank result, and the aggregate must be the max
time and the summed units."""
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
    # the bench's own split: equal-work row blocks of one job, rank r taking blocks
    # r, r + world, ... in step order
    batches = 5
    blocks = bench.row_blocks(ps.n, batches)
    parts = []
    for b in bench.rank_blocks(batches, world, rank):
        i0, i1 = blocks[b]
        mine = cands[(cands["i"] >= i0) & (cands["i"] < i1)]
        alns, _ = O.align_pairs(codes, ps.offsets, mine, mat)
        parts.append((b, O.filter_edges(ps.offsets, mine, alns)))
    n_edges = sum(len(e) for _, e in parts)
    gathered = [None] * world
    dist.all_gather_object(gathered, [(b, e.tobytes()) for b, e in parts])
    ms, units = bench.combine_ranks(10.0 * (rank + 1), n_edges, world, dist)
    if rank == 0:
        by_block = sorted(x for g in gathered for x in g)
        assert [b for b, _ in by_block] == list(range(batches))     # every block exactly once
        allb = b"".join(e for _, e in by_block)
        ref = O.run(ps.ascii, ps.offsets, mat)["edges"].tobytes()
        sizes = [len(e) for _, e in by_block]
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


def test_rank_blocks_cover_each_block_once():
    import bench
    for batches, world in ((8, 1), (8, 2), (8, 3), (64, 8), (5, 2)):
        got = sorted(b for r in range(world) for b in bench.rank_blocks(batches, world, r))
        assert got == list(range(batches))


def test_two_gloo_ranks_partition_the_job(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    ok, ms, units, got, want = open(tmp_path / "result.txt").read().split()
    assert ok == "1"
    assert float(ms) == 20.0
    assert int(float(units)) == int(got) == int(want)
