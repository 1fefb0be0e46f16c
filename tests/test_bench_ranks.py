"""The multi-rank path of bench.py on CPU: two gloo ranks reduce their
timings (max) and attempts (sum) as the GPU ranks do over NCCL."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = 10.0 + 5.0 * rank
    attempts = 1000 * (rank + 1)
    t, a = bench.reduce_over_ranks(elapsed, attempts, "cpu")
    out.put((rank, t, a))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    assert [r[2] for r in res] == [3000.0, 3000.0]


def test_bench_helpers_and_global_names():
    """The benchmark's layout and roofline helpers give the documented figures,
    and every global name its functions read exists (a code path that only runs
    on a GPU machine must not fail there on a missing helper)."""
    import builtins
    import dis
    import types

    sys.path.insert(0, ROOT)
    import bench

    assert bench.replica_bytes(10, 64) == 2048
    assert bench.replica_bytes(10, 16) == 128
    assert bench.replica_bytes(20, 256) == 40960
    assert bench.replica_bytes(2, 8) == 16        # 2 words padded to 4
    assert bench.replica_bytes(10, 48) == 1152    # banded: 36 words per colour
    assert bench.replica_bytes(10, 24) == 768     # padded rows: 24 words per colour
    # q = 10 (B = 4), 6 acceptance planes, theta = 10: Philox 50 + 1.5 counter
    # words, shift 4, proposal 32, dE class 49, acceptance 18, merge 5,
    # measurements (28 + 80) / 20 = 5.4
    assert bench.ops_per_word(10, 6.0, 10) == pytest.approx(164.9)
    w = bench.wl.C2
    A, src = bench.acceptance_planes(w, 6, 25)
    assert src is not None and 5.5 < A < 6.5
    A5, src5 = bench.acceptance_planes(bench.wl.C5, 6, 25)
    assert src5 is not None and 4.5 < A5 < 6.0
    # no count for the small case; a count holds only for the schedule it was taken on
    assert bench.acceptance_planes(bench.wl.C1, 6, 25) == (bench.ACC_PLANES, None)
    other = bench.wl.scaled(bench.wl.C2, K=100, name="c2-K100")
    assert bench.acceptance_planes(other, 6, 25) == (bench.ACC_PLANES, None)

    missing = set()

    def visit(code):
        for ins in dis.get_instructions(code):
            if ins.opname == "LOAD_GLOBAL":
                name = ins.argval if isinstance(ins.argval, str) else str(ins.argval)
                name = name.split(" + ")[-1].replace("NULL + ", "")
                if not hasattr(bench, name) and not hasattr(builtins, name):
                    missing.add((code.co_name, name))
        for c in code.co_consts:
            if isinstance(c, types.CodeType):
                visit(c)

    for obj in vars(bench).values():
        if isinstance(obj, types.FunctionType) and obj.__module__ == "bench":
            visit(obj.__code__)
    assert not missing, sorted(missing)
