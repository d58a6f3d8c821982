"""The N > 1 host path of bench.py on CPU ranks (gloo, world size 2): every rank
gets the same channels, meshes and energies and its own parameter samples
(rank 0's are the single-GPU workload's), the step time is the maximum over
ranks, the barrier returns on every rank, and the oracle leg runs on rank 0
alone.  No GPU: the ranks only exercise the host logic (there is no data-path
collective to test: the shards never exchange data)."""
import os
import socket
import sys
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    try:
        args = types.SimpleNamespace(impl="reference", samples=6, gpus=ws, steps=1, warmup=0, cpu_samples=1,
                                     ref_samples=1, workload="config4")
        got_ws, r, _ = bench.dist_init(args)  # the oracle leg's backend: gloo
        wl = bench.rank_workload(6, r)
        step_max = bench.max_over_ranks(got_ws, 10.0 + 5.0 * r)
        bench.barrier(got_ws)
        skipped = None
        if r != 0:
            skipped = bench.run_reference(args, got_ws, r)  # returns at once, prints nothing
        q.put((r, got_ws, step_max, wl.nwp, wl.coeffs.tolist(), wl.e_lab.tolist(), skipped))
    except Exception as e:  # noqa: BLE001 - reported to the parent
        q.put(("error", rank, repr(e)))
    finally:
        if dist.is_initialized():
            dist.destroy_process_group()


def test_two_cpu_ranks_shard_by_sample():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    from paper_2106_00454_gb300 import inputs as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = [q.get(timeout=180) for _ in range(2)]
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    errors = [x for x in res if x[0] == "error"]
    assert not errors, errors
    res = sorted(res, key=lambda x: x[0])
    (r0, ws0, m0, nwp0, c0, e0, _), (r1, ws1, m1, nwp1, c1, e1, skipped) = res
    assert (r0, r1) == (0, 1) and ws0 == ws1 == 2
    assert m0 == m1 == 15.0                    # the maximum over ranks, on every rank
    assert nwp0 == nwp1 and e0 == e1           # the same channel set and energies
    assert not np.allclose(np.array(c0), np.array(c1))  # different parameter samples
    single = W.workload_mixed(n_samples=6)
    assert nwp0 == single.nwp and np.array_equal(np.array(c0), single.coeffs)
    assert skipped is None
