"""Multi-rank paths on CPU (gloo, world sizes 2 and 3, 127.0.0.1).

The Gaussian-partitioned operator (paper_2602_03893_gb300.sharded: z-slabs from the library's
gpair_shard_range, partial signals summed by one all-reduce, the residual replicated so that
each rank's adjoint stays local) is checked here with the FP64 oracle standing in for each
rank's slab forward: the all-reduced partial forwards equal the full forward and the per-rank
adjoints over the rank's rows are the full adjoint's slices (both operators are sums over
Gaussians).  The CUDA kernels behind the same wrapper are checked in tests/test_sharded_gpu.py.
The bench's rank helpers and its reference arm under torchrun are exercised the same way.
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
        from paper_2602_03893_gb300 import _lib, sharded, synth

        dist = _init(rank, world, port)
        oracle.set_threads(1)
        g = synth.centred_grid(6, 5, 8, 0.2e-3)
        A = np.random.default_rng(3).uniform(0.2, 1.0, g.M)
        sens = synth.cap_sensors(9, 8e-3, 160.0)
        v, fs, t0, Nt, k = 1500.0, 40e6, 0.0, 256, 3.0
        grid = _lib.Grid(g.nx, g.ny, g.nz, g.ox, g.oy, g.oz, g.h, g.sigma)
        gs = _lib.Gaussians(A=torch.as_tensor(A, dtype=torch.float32), grid=grid)
        arr = _lib.SensorArray(xyz=torch.as_tensor(sens), sound_speed=v, fs=fs, n_samples=Nt, t0=t0, window_k=k)
        G = oracle.gaussians_from_grid(g.nx, g.ny, g.nz, g.ox, g.oy, g.oz, g.h, g.sigma, A)

        def slab(op):
            r = op.rows
            return oracle.Gaussians(G.c[r], G.sigma[r], G.A[r])

        def local_forward(y):
            y.copy_(torch.as_tensor(oracle.forward(slab(op), sens, v, fs, t0, Nt, k=k)))

        op = sharded.ShardedOperator(gs, arr, local_forward=local_forward)
        y = torch.zeros((len(sens), Nt), dtype=torch.float64)
        op.forward(y)                                # partial forward + the one all-reduce
        y_full = oracle.forward(G, sens, v, fs, t0, Nt, k=k)
        delta = np.random.default_rng(4).normal(size=y_full.shape)   # replicated residual
        gA_part = torch.as_tensor(oracle.adjoint(slab(op), sens, v, fs, t0, Nt, delta, k=k, want=("A",))["A"])
        sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(sizes, torch.tensor([gA_part.numel()]))
        nmax = int(max(sizes))          # gloo gathers equal sizes: pad, then trim
        parts = [torch.zeros(nmax, dtype=torch.float64) for _ in sizes]
        dist.all_gather(parts, torch.cat([gA_part, torch.zeros(nmax - gA_part.numel(), dtype=torch.float64)]))
        parts = [p[:int(n)] for p, n in zip(parts, sizes)]
        gA_full = oracle.adjoint(G, sens, v, fs, t0, Nt, delta, k=k, want=("A",))["A"]
        fwd_err = float(np.linalg.norm(y.numpy() - y_full) / np.linalg.norm(y_full))
        adj_err = float(np.linalg.norm(torch.cat(parts).numpy() - gA_full) / np.linalg.norm(gA_full))
        rows = (op.z_begin, op.z_end)
        dist.destroy_process_group()
        q.put((rank, fwd_err, adj_err, rows, None))
    except Exception as e:   # reported to the parent
        q.put((rank, None, None, None, repr(e)))


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


@pytest.mark.parametrize("world", [2, 3])
def test_gaussian_sharded_operators_match_full_operators(world):
    out = _run(_shard_worker, world=world)
    spans = []
    for rank, fwd_err, adj_err, rows, err in out:
        assert err is None, err
        assert fwd_err < 1e-13 and adj_err < 1e-13, (rank, fwd_err, adj_err)
        spans.append(rows)
    # the slabs tile the 8 lattice rows in order, the first 8 % world ranks one row longer
    assert spans[0][0] == 0 and spans[-1][1] == 8
    assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
    assert sorted((e - b for b, e in spans), reverse=True) == [e - b for b, e in spans]
    assert max(e - b for b, e in spans) - min(e - b for b, e in spans) <= 1


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
