"""The exchange plan of a population spread over several GPUs
(pa_shard_plan, host code of the C library; no GPU needed) and the exchange
itself between two CPU ranks over gloo, with the oracle doing each rank's
arithmetic (Sec. 2 of the paper: the replicas are independent between
resampling steps, which couple them only through Q_i and the copy-number
offsets)."""
import math
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _pa():
    from paper_1704_01888_gb300 import build

    try:
        build.build()
    except (OSError, RuntimeError) as e:
        pytest.skip(f"cannot build the CUDA library here: {e}")
    import paper_1704_01888_gb300 as pa

    return pa


@pytest.mark.parametrize("totals", [[5, 7], [0, 9], [9, 0], [3, 3, 3], [10, 0, 0, 2], [1, 1, 1, 1, 1],
                                    [2500, 2499, 2502, 2499], [17]])
def test_plan_is_a_consistent_partition(totals):
    pa = _pa()
    world = len(totals)
    R = sum(totals)
    plans = [pa.shard_plan(totals, world, g) for g in range(world)]
    bounds = [plans[g][1] for g in range(world)] + [plans[-1][2]]
    assert bounds[0] == 0 and bounds[-1] == R
    assert all(plans[g][2] == bounds[g + 1] for g in range(world))
    assert all(plans[g][0] == R for g in range(world))
    # ranges as even as integers allow
    sizes = np.diff(bounds)
    assert sizes.max() - sizes.min() <= 1
    for g in range(world):
        send, recv = plans[g][3], plans[g][4]
        assert send.sum() == totals[g]                    # every child goes somewhere
        assert recv.sum() == bounds[g + 1] - bounds[g]    # every new slot is filled
        for d in range(world):
            assert send[d] == plans[d][4][g]              # what g sends d is what d receives from g
    # rank g's children are the new slots [O_g, O_g + T_g): a slot's owner is
    # the rank whose range holds it
    O = np.concatenate([[0], np.cumsum(totals)])
    for g in range(world):
        for d in range(world):
            want = len(set(range(O[g], O[g + 1])) & set(range(bounds[d], bounds[d + 1])))
            assert plans[g][3][d] == want


def test_plan_rejects_bad_input():
    pa = _pa()
    for totals, world, rank in (([1, 2], 2, 2), ([1, 2], 2, -1), ([1, -2], 2, 0)):
        with pytest.raises(pa.PAError) as e:
            pa.shard_plan(totals, world, rank)
        assert e.value.status == pa.PA_ERR_INVALID
    with pytest.raises(pa.PAError) as e:
        pa.shard_plan([0, 0], 2, 0)
    assert e.value.status == pa.PA_ERR_CAPACITY


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q, L, R, seed, theta, betas, result_path):
    """One CPU rank: its slice of the population, resampled from the whole
    population's energies, its children sent over gloo as runs (parent
    replica and child count) placed by the library's plan, swept by the
    oracle with global slot keys."""
    import sys

    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle
    import paper_1704_01888_gb300 as pa

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    N = L * L
    lo, hi = rank * R // world, (rank + 1) * R // world
    spins = oracle.init_random(q, L, lo, hi - lo, seed)
    E = np.array([oracle.energy(s) for s in spins], dtype=np.int32)
    lnZ = N * math.log(q)
    records = []
    for i in range(1, len(betas)):
        dbeta = betas[i] - betas[i - 1]
        # the histogram summed over the ranks is the whole population's
        h = torch.from_numpy(np.bincount(E + 2 * N, minlength=2 * N + 1).astype(np.int32))
        dist.all_reduce(h)
        parts = [None] * world
        dist.all_gather_object(parts, E)
        E_all = np.concatenate(parts)
        assert np.array_equal(np.bincount(E_all + 2 * N, minlength=2 * N + 1), h.numpy())
        r, lnq, R_new, _ = oracle.copy_numbers(E_all, dbeta, R, oracle.NEAREST_INT, i, seed)
        T = torch.tensor([int(r[lo:hi].sum())], dtype=torch.int64)
        totals = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(totals, T)
        totals = [int(t.item()) for t in totals]
        Rn, lo2, hi2, send_children, recv_children = pa.shard_plan(totals, world, rank)
        assert Rn == R_new
        # runs of this rank's children for each destination (consecutive
        # children of one parent), sent as the parent replica and a count
        parent_of = np.repeat(np.arange(hi - lo), r[lo:hi])
        O = sum(totals[:rank])
        bounds = [min(max(pa.shard_plan(totals, world, d)[1] - O, 0), len(parent_of)) for d in range(world)]
        bounds.append(len(parent_of))
        run_parent, run_count, send = [], [], []
        for d in range(world):
            seg = parent_of[bounds[d]:bounds[d + 1]]
            heads = np.flatnonzero(np.diff(seg, prepend=-1) != 0)
            run_parent.append(seg[heads])
            run_count.append(np.diff(np.append(heads, seg.size)))
            send.append(heads.size)
            assert run_count[-1].sum() == send_children[d]
        run_parent, run_count = np.concatenate(run_parent), np.concatenate(run_count).astype(np.int32)
        recv = torch.zeros(world, dtype=torch.int64)
        dist.all_to_all_single(recv, torch.tensor(send, dtype=torch.int64))
        recv = recv.tolist()
        words = N // 4
        out = torch.zeros(sum(recv) * words, dtype=torch.int32)
        inp = torch.from_numpy(np.ascontiguousarray(spins[run_parent]).view(np.int32).reshape(-1).copy())
        dist.all_to_all_single(out, inp, [x * words for x in recv], [x * words for x in send])
        cnt = torch.zeros(sum(recv), dtype=torch.int32)
        dist.all_to_all_single(cnt, torch.from_numpy(run_count), recv, send)
        runs = out.numpy().view(np.uint8).reshape(-1, L, L)
        spins = np.repeat(runs, cnt.numpy(), axis=0).copy()
        assert spins.shape[0] == hi2 - lo2 == recv_children.sum()
        lo, hi = lo2, hi2
        spins = np.array([oracle.sweep_replica(q, s, betas[i], theta, i, lo + k, seed) for k, s in enumerate(spins)],
                         dtype=np.uint8).reshape(-1, L, L)
        E = np.array([oracle.energy(s) for s in spins], dtype=np.int32)
        sums = torch.tensor([int(E.astype(np.int64).sum()), int((E.astype(np.int64) ** 2).sum())], dtype=torch.int64)
        dist.all_reduce(sums)
        lnZ += lnq
        records.append((int(sums[0]), int(sums[1]), float(lnZ), Rn))
    parts = [None] * world
    dist.all_gather_object(parts, spins)
    if rank == 0:
        np.savez(result_path, spins=np.concatenate(parts), records=np.array(records, dtype=object))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,K", [(2, 6), (3, 3)])
def test_cpu_ranks_reproduce_the_single_population_run(tmp_path, world, K):
    """world_size 2 (and 3, with steps large enough that a few replicas take
    most children, whose runs then span several ranks) over gloo: the gathered
    population, the integer sums and ln Z equal the oracle's unsharded run bit
    for bit (ln Z exactly: both sum the same ln Q values in the same order)."""
    _pa()
    import oracle
    import torch.multiprocessing as mp

    q, L, R, seed, theta = 6, 8, 300, 5, 2
    betas = np.linspace(0.0, 1.2, K + 1)
    path = str(tmp_path / "shard.npz")
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, q, L, R, seed, theta, betas, path), nprocs=world, join=True,
                       start_method="spawn")
    got = np.load(path, allow_pickle=True)
    ref = oracle.run(q, L, R, seed, theta, betas)
    assert np.array_equal(got["spins"], ref["spins"])
    for i, (sE, sE2, lnZ, Rn) in enumerate(got["records"], start=1):
        assert (sE, sE2, Rn) == (ref["sumE"][i], ref["sumE2"][i], ref["R"][i])
        assert lnZ == ref["lnZ"][i]
