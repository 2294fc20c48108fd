"""Data-parallel training's gradient all-reduce on CPU ranks (gloo, world size 2, 127.0.0.1).

Each rank takes its equal shard of a seeded batch (train.shard_rows), computes the gradients of
Eq. 5 on it, and the ranks average them in place (train.allreduce_mean_, one all-reduce per
buffer). The gradient computation here is the oracle's FP64 backward (oracle/mlp.py) standing in
for the device's mlp_train_grads, which needs a GPU. Checked: the mean of the shard gradients
equals the whole batch's gradient (Eq. 5 is a mean over the batch), both ranks hold the same
values, and one Adam step from them leaves identical parameters on both ranks, equal to the
single-process step on the whole batch."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WIDTHS = [32, 48, 40, 24, 29]
B = 64


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem():
    from oracle import mlp as M
    rng = np.random.default_rng(7101)
    layers = M.init_params(WIDTHS, 7102)
    z = rng.normal(size=(B, WIDTHS[0]))
    target = rng.normal(size=(B, WIDTHS[-1]))
    return M, layers, z, target


def _grads(M, layers, z, target):
    out, cache = M.forward(layers, z)
    _, dout = M.l1_loss(out, target)
    return M.backward(layers, cache, dout)


def _flat(grads):
    return np.concatenate([np.concatenate([g["W"].ravel(), g["b"]]) for g in grads])


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2312_05800_gb300 import train
    M, layers, z, target = _problem()
    rows = np.arange(B)
    mine = train.shard_rows(rows, rank, world)
    g = _grads(M, layers, z[mine], target[mine])
    tensors = [torch.from_numpy(np.ascontiguousarray(x)) for gl in g for x in (gl["W"], gl["b"])]
    train.allreduce_mean_(tensors, world)
    reduced = [{"W": tensors[2 * i].numpy(), "b": tensors[2 * i + 1].numpy()} for i in range(len(g))]
    state = M.adam_init(layers)
    M.adam_step(layers, reduced, state, 1e-3)
    q.put((rank, _flat(reduced), np.concatenate([np.concatenate([L["W"].ravel(), L["b"]]) for L in layers])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_average_shard_gradients():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=120) for _ in range(2)), key=lambda o: o[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    M, layers, z, target = _problem()
    full = _flat(_grads(M, layers, z, target))
    for _, g, _ in out:
        assert np.allclose(g, full, rtol=1e-12, atol=1e-15)
    assert np.array_equal(out[0][1], out[1][1])
    state = M.adam_init(layers)
    M.adam_step(layers, _grads(M, layers, z, target), state, 1e-3)
    ref = np.concatenate([np.concatenate([L["W"].ravel(), L["b"]]) for L in layers])
    assert np.array_equal(out[0][2], out[1][2])
    assert np.allclose(out[0][2], ref, rtol=1e-12, atol=1e-15)


def test_shards_split_the_batch():
    sys.path.insert(0, ROOT)
    import pytest
    from paper_2312_05800_gb300 import train
    rows = np.arange(24)
    parts = [train.shard_rows(rows, r, 3) for r in range(3)]
    assert np.array_equal(np.concatenate(parts), rows)
    with pytest.raises(ValueError):
        train.shard_rows(np.arange(10), 0, 3)
