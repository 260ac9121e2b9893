"""The Gaussian-partitioned operator on the CUDA kernels (gpair_forward_shard,
gpair_adjoint_shard and the ShardedOperator wrapper).

In one process: the shards' partial signals add up to gpair_forward's signals and the shards'
gradient rows are gpair_adjoint's rows, for even and ragged splits of the lattice rows (slab
boundaries that do not fall on the kernels' own brick or cube boundaries).  Across two
processes on one GPU: each rank computes its slab with the kernels, a gloo all-reduce of host
copies completes the signals, and the result matches the FP64 oracle (relative L2 1e-5 plus the
window-ambiguity bound) and the single-call forward; no kernel waits on another process."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest
import torch

import oracle
from gpair_testutil import TAU, assert_signal_parity, device_inputs, oracle_gaussians, rel_l2
from paper_2602_03893_gb300 import _lib, synth

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _workload():
    g = synth.centred_grid(24, 20, 22, 0.1e-3)
    A = (np.random.default_rng(17).uniform(0.0, 1.0, g.M) ** 2).astype(np.float32)
    return synth.Workload("shard", g, synth.cap_sensors(96, 30e-3, 140.0), 2048, A=A)


@pytest.mark.parametrize("n", [2, 3, 5])
def test_shards_sum_to_the_full_operators(n):
    w = _workload()
    gs, arr = device_inputs(w)
    y_full = torch.empty((w.Nd, w.Nt), device="cuda")
    _lib.gpair_forward(gs, arr, y_full)
    y_sum = torch.zeros_like(y_full)
    y_s = torch.empty_like(y_full)
    rows = []
    for s in range(n):
        _lib.gpair_forward_shard(gs, arr, s, n, y_s)
        y_sum += y_s
        rows.append(_lib.gpair_shard_range(gs.grid, s, n))
    assert rows[0][0] == 0 and rows[-1][1] == w.grid.nz
    assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
    d = torch.randn((w.Nd, w.Nt), device="cuda", generator=torch.Generator(device="cuda").manual_seed(2))
    g_full = torch.empty(w.M, device="cuda")
    _lib.gpair_adjoint(gs, arr, d, g_full)
    g_sh = torch.full((w.M,), float("nan"), device="cuda")
    for s in range(n):
        _lib.gpair_adjoint_shard(gs, arr, s, n, d, g_sh)
    torch.cuda.synchronize()
    assert _lib.gpair_last_device_status() == 0
    # A slab boundary off the kernels' own tiling changes the FP32 reference of every pair near
    # it by ~1e-10 m, which can move a term lying within that distance of its window edge in or
    # out: the two signals agree to FP32 rounding plus (twice) the weight of those terms.
    oracle.set_threads(os.cpu_count() or 1)
    y_ora, amb = oracle.forward(oracle_gaussians(w), w.sensors, w.v, w.fs, w.t0, w.Nt, k=w.k, tau=TAU, want_amb=True)
    ys, yf = y_sum.cpu().numpy().astype(np.float64), y_full.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(ys - yf) <= 1e-6 * np.linalg.norm(yf) + 2 * np.linalg.norm(amb)
    assert_signal_parity(ys, y_ora, amb)
    assert torch.isfinite(g_sh).all()
    assert rel_l2(g_sh.cpu().numpy(), g_full.cpu().numpy()) < 1e-6


def test_shard_arguments():
    w = _workload()
    gs, arr = device_inputs(w)
    y = torch.empty((w.Nd, w.Nt), device="cuda")
    for bad in [(2, 2), (-1, 2), (0, 0)]:
        with pytest.raises(_lib.GpairError) as e:
            _lib.gpair_forward_shard(gs, arr, bad[0], bad[1], y)
        assert e.value.code == 1
    # more shards than rows: the empty shards give zero signals and leave the gradient alone
    n = w.grid.nz + 3
    _lib.gpair_forward_shard(gs, arr, n - 1, n, y)
    g = torch.full((w.M,), 7.0, device="cuda")
    _lib.gpair_adjoint_shard(gs, arr, n - 1, n, y, g)
    torch.cuda.synchronize()
    assert float(y.abs().max()) == 0.0 and float((g - 7.0).abs().max()) == 0.0
    free = synth.free_gaussians(w.grid, 1)
    wf = synth.Workload("free", w.grid, w.sensors, 64, free=free)
    gf, af = device_inputs(wf)
    with pytest.raises(_lib.GpairError) as e:
        _lib.gpair_forward_shard(gf, af, 0, 2, torch.empty((wf.Nd, wf.Nt), device="cuda"))
    assert e.value.code == 5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    try:
        sys.path.insert(0, ROOT)
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        import torch.distributed as dist

        from gpair_testutil import device_inputs as dev_in
        from paper_2602_03893_gb300 import sharded

        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
        dist.init_process_group("gloo", rank=rank, world_size=world)
        torch.cuda.set_device(0)
        w = _workload()
        gs, arr = dev_in(w)
        op = sharded.ShardedOperator(gs, arr)
        y = torch.empty((w.Nd, w.Nt), device="cuda")
        op.forward(y)                       # this rank's slab on the GPU, then the all-reduce
        d = torch.randn((w.Nd, w.Nt), device="cuda", generator=torch.Generator(device="cuda").manual_seed(2))
        gA = torch.zeros(w.M, device="cuda")
        op.adjoint(d, gA)
        torch.cuda.synchronize()
        gh = gA.cpu()
        dist.all_reduce(gh)                 # rows are disjoint: the sum assembles the gradient
        dist.destroy_process_group()
        q.put((rank, y.cpu().numpy() if rank == 0 else None, gh.numpy() if rank == 0 else None, (op.z_begin, op.z_end),
               None))
    except Exception as e:
        q.put((rank, None, None, None, repr(e)))


def test_two_processes_on_one_gpu_match_the_oracle():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=300) for _ in procs], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in out:
        assert r[4] is None, r[4]
    assert out[0][3][1] == out[1][3][0]
    y, gA = out[0][1], out[0][2]
    w = _workload()
    gs, arr = device_inputs(w)
    y1 = torch.empty((w.Nd, w.Nt), device="cuda")
    _lib.gpair_forward(gs, arr, y1)
    d = torch.randn((w.Nd, w.Nt), device="cuda", generator=torch.Generator(device="cuda").manual_seed(2))
    g1 = torch.empty(w.M, device="cuda")
    _lib.gpair_adjoint(gs, arr, d, g1)
    assert rel_l2(y, y1.cpu().numpy()) < 1e-6
    assert rel_l2(gA, g1.cpu().numpy()) < 1e-6
    oracle.set_threads(os.cpu_count() or 1)
    idx = np.arange(0, w.Nd, 8)
    y_ora, amb = oracle.forward(oracle_gaussians(w), w.sensors[idx], w.v, w.fs, w.t0, w.Nt, k=w.k, tau=TAU,
                                want_amb=True)
    assert_signal_parity(y[idx], y_ora, amb)
