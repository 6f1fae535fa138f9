"""Multi-rank paths on CPU (gloo, world size 2) and the row-block partition
design check.

The solver itself runs one system per GPU; with N GPUs the benchmark runs N
independent replicas and reports the slowest (max over ranks).  Sharding one
system across GPUs (a row-block partition with a halo exchange of p and two
all-reduces per iteration) is design-only; the emulation below checks that the
partition reproduces the unpartitioned product bitwise and the CG iteration.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import femgen
import oracle


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        vals = bench.max_over_ranks([10.0 + rank, 5.0 - rank, float(rank)], dist, "cpu")
        out[rank] = vals
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_timing_is_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        assert out[0] == out[1] == [11.0, 5.0, 1.0]
    assert bench.max_over_ranks([3.0], None, "cpu") == [3.0]


# ------------------------------------------------ row-block partition emulation
def partition(n, P):
    cuts = np.linspace(0, n, P + 1).astype(int)
    return [(cuts[i], cuts[i + 1]) for i in range(P)]


def halo_plan(ptr, idx, parts):
    """For each part: the sorted off-part columns it reads (what a neighbour must send)."""
    plans = []
    for (a, b) in parts:
        cols = idx[ptr[a]:ptr[b]]
        plans.append(np.unique(cols[(cols < a) | (cols >= b)]))
    return plans


def partitioned_spmv(ptr, idx, val, x, parts, plans):
    y = np.empty_like(x)
    for (a, b), halo in zip(parts, plans):
        # explicit exchange buffer: the halo values as another rank would send them
        xloc = {int(c): x[c] for c in halo}
        for i in range(a, b):
            s = 0.0
            for k in range(ptr[i], ptr[i + 1]):
                c = idx[k]
                s += val[k] * (x[c] if a <= c < b else xloc[int(c)])
            y[i] = s
    return y


@pytest.mark.parametrize("P", [2, 3, 5])
def test_row_block_partition_reproduces_the_product(P):
    s = femgen.build_system(femgen.Grid(9, 8, 10))
    x = femgen.random_vector(s.n, 4)
    parts = partition(s.n, P)
    plans = halo_plan(s.ptr, s.idx, parts)
    # with natural ordering only the neighbouring blocks exchange halos
    for p, ((a, b), halo) in enumerate(zip(parts, plans)):
        owners = {q for q, (c0, c1) in enumerate(parts) if np.any((halo >= c0) & (halo < c1))}
        assert owners <= {p - 1, p + 1}
    y = partitioned_spmv(s.ptr, s.idx, s.val, x, parts, plans)
    assert np.array_equal(y, oracle.spmv("csr", s.ptr, s.idx, s.val, x))


def test_row_block_partition_cg_matches_oracle():
    # CG with per-part partial dot products summed in a fixed order (the two
    # all-reduces per iteration) and the halo exchange of p before each product
    s = femgen.build_system(femgen.Grid(8, 8, 8))
    parts = partition(s.n, 3)
    plans = halo_plan(s.ptr, s.idx, parts)

    def pdot(u, v):
        return sum(float(np.dot(u[a:b], v[a:b])) for a, b in parts)

    x = np.zeros(s.n)
    r = s.b.copy()
    p = r.copy()
    rr = pdot(r, r)
    nb = np.sqrt(pdot(s.b, s.b))
    k = 0
    while np.sqrt(rr) / nb > 1e-10 and k < 10 * s.n:
        q = partitioned_spmv(s.ptr, s.idx, s.val, p, parts, plans)
        alpha = rr / pdot(p, q)
        x += alpha * p
        r -= alpha * q
        rr_new = pdot(r, r)
        k += 1
        p = r + (rr_new / rr) * p
        rr = rr_new
    ref = oracle.cg("csr", s.ptr, s.idx, s.val, s.b, tol=1e-10, maxit=10 * s.n)
    assert abs(k - ref.iterations) <= 0.05 * ref.iterations + 5
    assert np.linalg.norm(x - ref.x) <= 1e-6 * np.linalg.norm(ref.x)
