"""World-size-2 gloo run of the multi-GPU host logic on CPU.

Each rank owns its range of mocks, computes their correlation functions
(here with the CPU oracle standing in for the GPU path) and the rows are
gathered before the LC covariance; the result must equal the single-process
computation over all mocks.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth

N_D, PER_RANK, WORLD = 300, 4, 2


def _xi_rows(mocks):
    b = oracle.Binning(np.linspace(0, 60.0, 7), 2, oracle.PERIODIC, 300.0)
    rows = {k: [] for k in ("a1", "a2", "b")}
    for m in mocks:
        mk = synth.SMALL.make_mock(m, n_d=N_D, M=2)
        c = oracle.count_mock(mk.data, mk.randoms, b)
        for k, sel in (("a1", [0]), ("a2", [1]), ("b", [0, 1])):
            rows[k].append(oracle.ls(c["DD"], c["DR"], c["RR"], N_D, [N_D, N_D], sel))
    return {k: torch.tensor(np.array(v)) for k, v in rows.items()}


def _worker(rank, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    from paper_2205_11852_gb300 import multi  # noqa: import inside the spawned process
    local = _xi_rows(multi.mock_range(rank, PER_RANK))
    full = {k: multi.gather_rows(v, WORLD) for k, v in local.items()}
    if rank == 0:
        q.put({k: v.numpy() for k, v in full.items()})
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_sharded_gather_equals_single_process():
    pytest.importorskip("torch.distributed")
    import __graft_entry__
    __graft_entry__.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    ref = _xi_rows(range(WORLD * PER_RANK))
    for k in ref:
        assert np.array_equal(got[k], ref[k].numpy())
    a = oracle.lc_cov(got["a1"], got["a2"], got["b"], 1, 50.0)
    r = oracle.lc_cov(ref["a1"].numpy(), ref["a2"].numpy(), ref["b"].numpy(), 1, 50.0)
    assert np.array_equal(a["C_lc"], r["C_lc"])
