"""Multi-rank paths on CPU (gloo, world size 2, 127.0.0.1).

The GPU path is run as independent replicas (one GPU per process; no collective on the data
path).  What would shard it -- Gaussians split into z-slabs, partial signals summed over ranks,
the residual replicated so that each rank's adjoint and Adam step stay local -- is checked here
on the FP64 oracle: the all-reduced partial forwards equal the full forward and the per-rank
adjoints are the full adjoint's slices (both operators are sums over Gaussians).  The bench's
rank helpers and its reference arm under torchrun are exercised the same way.
"""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _shard_worker(rank, world, port, q):
    os.environ["CUDA_VISIBLE_DEVICES"] = ""      # CPU ranks, gloo
    try:
        sys.path.insert(0, ROOT)
        import torch

        import oracle
        from paper_2602_03893_gb300 import synth

        dist = _init(rank, world, port)
        oracle.set_threads(1)
        g = synth.centred_grid(6, 5, 8, 0.2e-3)
        A = np.random.default_rng(3).uniform(0.2, 1.0, g.M)
        sens = synth.cap_sensors(9, 8e-3, 160.0)
        v, fs, t0, Nt, k = 1500.0, 40e6, 0.0, 256, 3.0
        # z-slab of this rank (x fastest, so a z range is a contiguous index range)
        z0, z1 = rank * g.nz // world, (rank + 1) * g.nz // world
        lo, hi = z0 * g.nx * g.ny, z1 * g.nx * g.ny
        G = oracle.gaussians_from_grid(g.nx, g.ny, g.nz, g.ox, g.oy, g.oz, g.h, g.sigma, A)
        Gs = oracle.Gaussians(G.c[lo:hi], G.sigma[lo:hi], G.A[lo:hi])
        y_part = torch.as_tensor(oracle.forward(Gs, sens, v, fs, t0, Nt, k=k))
        dist.all_reduce(y_part)                      # the one exchange per forward
        y_full = oracle.forward(G, sens, v, fs, t0, Nt, k=k)
        delta = np.random.default_rng(4).normal(size=y_full.shape)   # replicated residual
        gA_part = torch.as_tensor(oracle.adjoint(Gs, sens, v, fs, t0, Nt, delta, k=k, want=("A",))["A"])
        parts = [torch.zeros(((r + 1) * g.nz // world - r * g.nz // world) * g.nx * g.ny, dtype=torch.float64)
                 for r in range(world)]
        dist.all_gather(parts, gA_part)
        gA_full = oracle.adjoint(G, sens, v, fs, t0, Nt, delta, k=k, want=("A",))["A"]
        fwd_err = float(np.linalg.norm(y_part.numpy() - y_full) / np.linalg.norm(y_full))
        adj_err = float(np.linalg.norm(torch.cat(parts).numpy() - gA_full) / np.linalg.norm(gA_full))
        dist.destroy_process_group()
        q.put((rank, fwd_err, adj_err, None))
    except Exception as e:   # reported to the parent
        q.put((rank, None, None, repr(e)))


def _helpers_worker(rank, world, port, q):
    os.environ["CUDA_VISIBLE_DEVICES"] = ""      # CPU ranks: dist_setup picks gloo
    try:
        sys.path.insert(0, ROOT)
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                          LOCAL_RANK=str(rank))
        import bench

        r, w, local = bench.dist_setup(world)
        bench.barrier(w)
        m = bench.max_over_ranks(1.5 + r, w)
        import torch.distributed as dist

        dist.destroy_process_group()
        q.put((rank, (r, w, local, m), None))
    except Exception as e:
        q.put((rank, None, repr(e)))


def _run(target, world=2, timeout=240):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=timeout) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out)


def test_gaussian_sharded_operators_match_full_operators():
    for rank, fwd_err, adj_err, err in _run(_shard_worker):
        assert err is None, err
        assert fwd_err < 1e-13 and adj_err < 1e-13, (rank, fwd_err, adj_err)


def test_bench_rank_helpers():
    out = _run(_helpers_worker)
    for rank, res, err in out:
        assert err is None, err
        r, w, local, m = res
        assert (r, w, local) == (rank, 2, rank)
        assert m == 2.5          # max over ranks of 1.5 + rank


def test_bench_reference_arm_under_torchrun():
    """Rank 0 alone runs the oracle and prints one JSON line; rank 1 exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference", "--gpus", "2",
           "--workload", "tiny", "--steps", "1", "--warmup", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="2", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
