"""Multi-rank slice distribution on CPU (gloo, world size 2 and 3).

The per-rank solver here is the FP64 oracle (this is a CPU test of the
distribution logic); the gathered result must equal the single-rank result
bit for bit, since slices are independent and every replica of the matrix is
identical."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2003_12677_b300.distributed import rank_slices, slice_plan


def test_plan_covers_every_slice_once():
    for n in range(0, 40):
        for w in (1, 2, 3, 5, 8):
            for chunk in (None, 1, 2, 3, 7):
                plan = slice_plan(n, w, chunk)
                got = sorted(s for ranges in plan for b, e in ranges for s in range(b, e))
                assert got == list(range(n))


def test_plan_last_loop_uneven_rule():
    # 10 slices, 4 ranks, at most 2 per loop: loop 1 = 2+2+2+2, loop 2 = 1+1+0+0
    plan = slice_plan(10, 4, 2)
    sizes = [[e - b for b, e in r] for r in plan]
    assert sizes == [[2, 1], [2, 1], [2], [2]]
    # one loop: 7 slices on 3 ranks -> 3, 2, 2 (the last ranks get one less)
    assert [[e - b for b, e in r] for r in slice_plan(7, 3)] == [[3], [2], [2]]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n_z, chunk, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2003_12677_b300 import inputs
    from paper_2003_12677_b300.distributed import gather_slices

    g = oracle.Geometry(24, 24, 24, 30)
    A = oracle.build_matrix(g)
    AT = A.transpose()
    case = inputs.make_case(24, 30, n_z, seed=9, phantom="ellipsoids3d", noise="poisson", level=1e4)
    mine = rank_slices(n_z, world, rank, chunk)
    local = oracle.sirt(A, AT, case.sino[mine].reshape(len(mine), -1), 15) if mine else np.zeros((0, A.cols))
    full = gather_slices(torch.from_numpy(np.ascontiguousarray(local)), n_z, chunk)
    if rank == 0:
        np.save(out_path, full.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,n_z,chunk", [(2, 7, None), (3, 8, 2)])
def test_gathered_equals_single_rank(tmp_path, world, n_z, chunk):
    import oracle
    from paper_2003_12677_b300 import inputs

    out = str(tmp_path / "full.npy")
    mp.start_processes(_worker, args=(world, _free_port(), n_z, chunk, out), nprocs=world, join=True,
                       start_method="spawn")
    got = np.load(out)
    g = oracle.Geometry(24, 24, 24, 30)
    A = oracle.build_matrix(g)
    case = inputs.make_case(24, 30, n_z, seed=9, phantom="ellipsoids3d", noise="poisson", level=1e4)
    ref = oracle.sirt(A, A.transpose(), case.sino.reshape(n_z, -1), 15)
    np.testing.assert_array_equal(got, ref)


def _worker_sharded(rank, world, port, n_z, chunk, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2003_12677_b300 import inputs
    from paper_2003_12677_b300.distributed import solve_sharded

    g = oracle.Geometry(24, 24, 24, 30)
    A = oracle.build_matrix(g)
    AT = A.transpose()
    case = inputs.make_case(24, 30, n_z, seed=9, phantom="ellipsoids3d", noise="poisson", level=1e4)
    calls = []

    def solve(sino):          # the per-rank solver (here the oracle's CGLS, on the CPU)
        calls.append(sino.shape[0])
        x, _ = oracle.cgls(A, AT, sino.reshape(sino.shape[0], -1).numpy(), 6)
        return torch.from_numpy(x.reshape(sino.shape[0], 24, 24))

    full = solve_sharded(solve, torch.from_numpy(case.sino), chunk)
    counts = [None] * world
    dist.all_gather_object(counts, calls)
    if rank == 0:
        np.save(out_path, full.numpy())
        np.save(out_path + ".calls.npy", np.array([sum(c) for c in counts]))
    else:
        assert full is None
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,n_z,chunk", [(2, 5, None), (3, 10, 2), (3, 2, None)])
def test_solve_sharded_equals_single_rank(tmp_path, world, n_z, chunk):
    """The product's sharded solve: each rank solves exactly its plan's slices
    (loop by loop, the last loop uneven; a rank with none contributes nothing),
    and the gathered stack equals the single-rank solve bit for bit."""
    import oracle
    from paper_2003_12677_b300 import inputs

    out = str(tmp_path / "sharded.npy")
    mp.start_processes(_worker_sharded, args=(world, _free_port(), n_z, chunk, out), nprocs=world, join=True,
                       start_method="spawn")
    got = np.load(out)
    per_rank = np.load(out + ".calls.npy")
    plan = slice_plan(n_z, world, chunk)
    own = [sum(e - b for b, e in r) for r in plan]
    assert [int(c) if o else 0 for c, o in zip(per_rank, own)] == own
    g = oracle.Geometry(24, 24, 24, 30)
    A = oracle.build_matrix(g)
    case = inputs.make_case(24, 30, n_z, seed=9, phantom="ellipsoids3d", noise="poisson", level=1e4)
    ref, _ = oracle.cgls(A, A.transpose(), case.sino.reshape(n_z, -1), 6)
    np.testing.assert_array_equal(got.reshape(n_z, -1), ref)


def test_solve_sharded_single_process():
    """Without a process group (one process) the sharded solve is the plain
    solve over the plan's loops, in stack order."""
    import torch
    from paper_2003_12677_b300 import distributed as dd
    assert not torch.distributed.is_initialized()
    sino = torch.arange(7 * 3, dtype=torch.float32).reshape(7, 3)
    calls = []

    def solve(s):
        calls.append(s.shape[0])
        return 2 * s
    out = dd.solve_sharded(solve, sino, chunk=3)
    assert torch.equal(out, 2 * sino)
    assert calls == [3, 3, 1]
    assert dd.world_rank() == (1, 0)
