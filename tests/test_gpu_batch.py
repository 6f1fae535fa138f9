"""Batched multi-right-hand-side solver (one persistent launch of
thread-block clusters, replayed as a CUDA graph) against the CPU oracle, which
solves every system and right-hand side on its own, through the C ABI.

Gates per system and right-hand side, as for the single-system solves (each
summation order gives a different but equally valid CG run):
  - true relative residual ||b - A x|| / ||b||, recomputed by the oracle's
    double-precision product, <= tol, and the same status as the oracle;
  - iteration count within 5% + 5 of the oracle's in double precision; for
    the single-precision inner CG within 10% + 10 (float rounding makes two
    valid runs differ more: a 486-row instance took 625 and 671 inner
    iterations with double and with pairwise-float dot accumulation);
    refinement passes within one;
  - solved to 1e-12 on both sides, ||x - x_oracle|| / ||x_oracle|| <= 1e-8.
"""
import numpy as np
import pytest

import femgen
import oracle
import paper_1010_4639_gb300 as gb

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def torch():
    import torch
    gb.build()
    assert torch.cuda.is_available()
    return torch


def small_grids(count=10, seed=5):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nx, ny, nz = (int(v) for v in rng.integers(4, 12, 3))
        out.append(femgen.Grid(nx, ny, nz, contrast=float(10 ** rng.uniform(1, 4)), seed_mesh=100 + 2 * i,
                               seed_x=101 + 2 * i))
    out.append(femgen.Grid(3, 5, 5, seed_mesh=90, seed_x=91))
    return out


def with_edge_cases(bs, empty_at=3, zero=(2, 5)):
    """An empty instance inserted at position empty_at and a zero right-hand
    side (instance zero[0], column zero[1])."""
    row_off = np.insert(bs.row_off, empty_at, bs.row_off[empty_at])
    grids = list(bs.grids)
    grids.insert(empty_at, None)
    B = bs.B.copy()
    Xs = bs.Xstar.copy()
    i, k = zero
    r0, r1 = row_off[i], row_off[i + 1]
    B[r0:r1, k] = 0.0
    Xs[r0:r1, k] = 0.0
    return femgen.BatchSystem(grids, row_off, bs.ptr, bs.idx, bs.val, B, Xs)


@pytest.fixture(scope="module")
def small():
    return with_edge_cases(femgen.build_batch(small_grids(), nrhs=8))


def instance(bs, i):
    r0, r1 = int(bs.row_off[i]), int(bs.row_off[i + 1])
    k0, k1 = int(bs.ptr[r0]), int(bs.ptr[r1])
    return r0, r1, (bs.ptr[r0:r1 + 1] - k0).astype(np.int32), (bs.idx[k0:k1] - r0).astype(np.int32), bs.val[k0:k1]


def true_rel_res(bs, X):
    """(count, nrhs) true relative residuals in double precision (oracle product); 0 where b = 0."""
    out = np.zeros((bs.count, bs.B.shape[1]))
    for i in range(bs.count):
        r0, r1, p, j, v = instance(bs, i)
        for k in range(bs.B.shape[1]):
            b = bs.B[r0:r1, k]
            nb = np.linalg.norm(b)
            if r1 > r0 and nb > 0:
                out[i, k] = np.linalg.norm(b - oracle.spmv("csr", p, j, v, X[r0:r1, k])) / nb
    return out


def gpu_batch_solve(torch, bs, **kw):
    with gb.Batch(bs.row_off, bs.ptr, bs.idx, bs.val, nrhs=bs.B.shape[1], tune=kw.pop("tune", False)) as Bt:
        if "tuning" in kw:
            Bt.set_tuning(kw.get("precision", "fp32_ir"), *kw.pop("tuning"))
        b = torch.from_numpy(bs.B).cuda()
        x, infos, rep = Bt.solve(b, **kw)
        return x.cpu().numpy(), infos, rep


@pytest.mark.parametrize("precision", ["fp32_ir", "fp64", "fp32_ru"])
def test_batch_matches_oracle(torch, small, precision):
    maxit = 50 * int(np.diff(small.row_off).max())
    X, infos, rep = gpu_batch_solve(torch, small, tol=TOL, maxit=maxit, precision=precision)
    assert rep["status"] == "OK" and rep["graph"] == 1 and rep["launches"] == 1
    Xo, res = oracle.batch_solve(small.row_off, small.ptr, small.idx, small.val, small.B, tol=TOL, maxit=maxit,
                                 precision=precision)
    rr = true_rel_res(small, X)
    assert rr.max() <= TOL, rr.max()
    for i in range(small.count):
        for k in range(small.B.shape[1]):
            g, o = infos[i, k], res[i][k]
            assert oracle.STATUS[int(g["status"])] == o.status == "OK", (i, k)
            rel, add = (0.05, 5) if precision == "fp64" else (0.10, 10)
            assert abs(int(g["iterations"]) - o.iterations) <= rel * o.iterations + add, (i, k, g, o.iterations)
            # refinement passes (IR) vs the oracle's passes; for double precision
            # the passes are the first run plus its restarts; a reliable update
            # of an instance serves all its right-hand sides, so the batch makes
            # at least the oracle's updates of one right-hand side
            if precision == "fp32_ru":
                assert int(g["outer"]) >= o.restarts - 2, (i, k, g, o.restarts)
            else:
                passes = o.restarts if precision == "fp32_ir" else o.restarts + (1 if o.iterations else 0)
                assert abs(int(g["outer"]) - passes) <= 1, (i, k, g, o.restarts)
            assert g["rel_res_true"] <= TOL
    # the empty instance and the zero right-hand side: x = 0 after no iteration
    assert np.all(infos[3]["iterations"] == 0)
    r0, r1 = small.row_off[2], small.row_off[3]
    assert np.all(X[r0:r1, 5] == 0.0) and infos[2, 5]["iterations"] == 0


def test_batch_solution_parity_at_1e12(torch, small):
    maxit = 50 * int(np.diff(small.row_off).max())
    Xo, res = oracle.batch_solve(small.row_off, small.ptr, small.idx, small.val, small.B, tol=1e-12, maxit=maxit,
                                 precision="fp64")
    for precision in ("fp32_ir", "fp64", "fp32_ru"):
        X, infos, rep = gpu_batch_solve(torch, small, tol=1e-12, maxit=maxit, precision=precision)
        assert rep["status"] == "OK", precision
        for i in range(small.count):
            r0, r1 = small.row_off[i], small.row_off[i + 1]
            for k in range(small.B.shape[1]):
                xo = Xo[r0:r1, k]
                if r1 > r0 and np.linalg.norm(xo) > 0:
                    assert np.linalg.norm(X[r0:r1, k] - xo) <= 1e-8 * np.linalg.norm(xo), (precision, i, k)


def launch_configs():
    for threads in (256, 512):
        for cluster in (1, 2, 4, 8, 16):
            for rpw in (1, 2, 4, 8, 16):
                yield threads, cluster, rpw


def test_every_launch_configuration(torch, small):
    """Each CTA size, cluster size and rows-per-warp variant of the kernel
    (both precisions; rows per warp 16 only in single precision) converges."""
    maxit = 50 * int(np.diff(small.row_off).max())
    ran = 0
    with gb.Batch(small.row_off, small.ptr, small.idx, small.val, nrhs=8, tune=False) as Bt:
        b = torch.from_numpy(small.B).cuda()
        for threads, cluster, rpw in launch_configs():
            for precision in ("fp32_ir", "fp64"):
                if precision == "fp64" and rpw == 16:
                    continue
                Bt.set_tuning(precision, threads, cluster, rpw)
                try:
                    x, infos, rep = Bt.solve(b, tol=TOL, maxit=maxit, precision=precision)
                except gb.GbcgError as e:  # a cluster shape this device cannot co-schedule
                    assert "cannot be launched" in str(e), str(e)
                    continue
                ran += 1
                assert rep["status"] == "OK" and rep["threads"] == threads and rep["cluster"] == cluster
                rr = true_rel_res(small, x.cpu().numpy())
                assert rr.max() <= TOL, (threads, cluster, rpw, precision, rr.max())
    assert ran >= 60


@pytest.mark.parametrize("G", [2, 4, 8])
def test_instances_spanning_several_clusters(torch, small, G):
    """Every instance split over G clusters (global-memory sums and bounded
    group barriers): same gates against the oracle, and the same bits on a
    repeated solve with the same schedule."""
    maxit = 50 * int(np.diff(small.row_off).max())
    Xo, res = oracle.batch_solve(small.row_off, small.ptr, small.idx, small.val, small.B, tol=TOL, maxit=maxit,
                                 precision="fp32_ir")
    with gb.Batch(small.row_off, small.ptr, small.idx, small.val, nrhs=8, tune=False) as Bt:
        b = torch.from_numpy(small.B).cuda()
        x1, infos, rep = Bt.solve(b, tol=TOL, maxit=maxit, force_group=G, fixed_order=True)
        x2, infos2, rep2 = Bt.solve(b, tol=TOL, maxit=maxit, force_group=G, fixed_order=True)
    assert rep["status"] == "OK", rep
    assert rep["max_group"] == min(G, rep["clusters"]) and rep["groups"] == small.count
    assert torch.equal(x1, x2) and np.array_equal(infos, infos2)
    assert true_rel_res(small, x1.cpu().numpy()).max() <= TOL
    for i in range(small.count):
        for k in range(8):
            o = res[i][k]
            assert abs(int(infos[i, k]["iterations"]) - o.iterations) <= 0.10 * o.iterations + 10, (i, k)


def test_group_wait_times_out_cleanly(torch, small):
    """A group member that never arrives: the waiting cluster gives up after
    the bound, the launch ends with GBCG_ERR_TIMEOUT and the context stays
    usable for the next solve."""
    maxit = 50 * int(np.diff(small.row_off).max())
    with gb.Batch(small.row_off, small.ptr, small.idx, small.val, nrhs=8, tune=False) as Bt:
        assert Bt.selftest_group_timeout(50) == 5
        b = torch.from_numpy(small.B).cuda()
        x, infos, rep = Bt.solve(b, tol=TOL, maxit=maxit)
    assert rep["status"] == "OK"
    assert true_rel_res(small, x.cpu().numpy()).max() <= TOL


def test_result_is_independent_of_the_schedule(torch, small):
    """The second solve runs with the queue reordered by the first one's
    measured times; with single-cluster instances every result is
    bit-identical (which cluster runs an instance, and when, does not enter
    its arithmetic)."""
    with gb.Batch(small.row_off, small.ptr, small.idx, small.val, nrhs=8, tune=False) as Bt:
        b = torch.from_numpy(small.B).cuda()
        x1, i1, r1 = Bt.solve(b, tol=TOL, maxit=100000, max_group=1)
        t1, p1, _ = Bt.instance_times()
        x2, i2, r2 = Bt.solve(b, tol=TOL, maxit=100000, max_group=1)
        t2, p2, _ = Bt.instance_times()
    assert torch.equal(x1, x2)
    assert np.array_equal(i1, i2) and np.array_equal(p1, p2)
    # the longest instance of the first run is among the first the second run started
    longest = int(np.argmax(t1[:, 1] - t1[:, 0]))
    started = np.argsort(t2[:, 0], kind="stable")[:max(1, r2["clusters"])]
    assert longest in started


def test_fewer_right_hand_sides_host_memory(torch):
    bs = femgen.build_batch(small_grids(6, seed=9), nrhs=3)
    maxit = 50 * int(np.diff(bs.row_off).max())
    with gb.Batch(bs.row_off, bs.ptr, bs.idx, bs.val, nrhs=3, tune=False) as Bt:
        x = np.zeros_like(bs.B)
        x, infos, rep = Bt.solve(bs.B.copy(), x, tol=TOL, maxit=maxit)
    assert rep["status"] == "OK"
    assert true_rel_res(bs, x).max() <= TOL
    assert infos.shape == (bs.count, 3)


def test_initial_guess_is_used(torch, small):
    maxit = 50 * int(np.diff(small.row_off).max())
    with gb.Batch(small.row_off, small.ptr, small.idx, small.val, nrhs=8, tune=False) as Bt:
        b = torch.from_numpy(small.B).cuda()
        x = torch.from_numpy(small.Xstar).cuda().clone()  # x0 = the exact solution
        x, infos, rep = Bt.solve(b, x, tol=1e-8, maxit=maxit)
    assert rep["status"] == "OK"
    assert int(infos["iterations"].max()) == 0


def test_maxit_reported_per_system(torch, small):
    X, infos, rep = gpu_batch_solve(torch, small, tol=TOL, maxit=5)
    assert rep["status"] == "MAXIT"
    nonempty = np.diff(small.row_off) > 0
    st = infos["status"][nonempty]
    assert np.all((st == 3) | (st == 0))
    assert int(infos["iterations"].max()) <= 5


def test_indefinite_instance_matches_the_oracle_status(torch):
    """An instance whose mesh has an inverted element (indefinite matrix):
    double precision stops with NOT_SPD where the oracle's CG meets p'Ap <= 0,
    mixed precision runs out of refinement passes like the oracle's; the
    healthy instance beside it converges."""
    bad = femgen.Grid(34, 21, 27, contrast=2238.12, seed_mesh=318, seed_x=319)
    good = femgen.Grid(9, 8, 10, seed_mesh=3, seed_x=4)
    bs = femgen.build_batch([good, bad], nrhs=2)
    for precision, want in (("fp64", "NOT_SPD"), ("fp32_ir", "MAXIT")):
        X, infos, rep = gpu_batch_solve(torch, bs, tol=TOL, maxit=100000, precision=precision)
        Xo, res = oracle.batch_solve(bs.row_off, bs.ptr, bs.idx, bs.val, bs.B, tol=TOL, maxit=100000,
                                     precision=precision)
        assert rep["status"] == want, (precision, rep["status"])
        for k in range(2):
            assert res[0][k].status == "OK" and infos[0, k]["status"] == 0
            assert res[1][k].status == want
            assert oracle.STATUS[int(infos[1, k]["status"])] == want, (precision, k, infos[1, k])


def test_autotune_picks_a_valid_configuration_and_caches_it(torch, small):
    with gb.Batch(small.row_off, small.ptr, small.idx, small.val, nrhs=8, tune=True) as Bt:
        st = Bt.stats()
        assert st["threads"][1] in (256, 512) and st["cluster"][1] in (1, 2, 4, 8, 16)
        assert all(r in (1, 2, 4, 8, 16) for r in st["rows_per_warp"][1])
        t = Bt.autotune("fp32_ir")
        assert t["from_cache"]
        t64 = Bt.autotune("fp64")
        assert t64["candidates"] > 0 and all(r <= 8 for r in t64["rows_per_warp"])
        b = torch.from_numpy(small.B).cuda()
        x, infos, rep = Bt.solve(b, tol=TOL, maxit=100000, precision="fp64")
        assert rep["status"] == "OK"


def test_full_size_uneven_batch(torch):
    """256 instances with grid edges in [12, 40], contrasts in [10, 1e4], eight
    right-hand sides each: every system reaches 1e-10 in the true residual;
    sampled systems match the oracle's iteration counts."""
    bs = femgen.build_batch(femgen.batched_instances(256), nrhs=8)
    with gb.Batch(bs.row_off, bs.ptr, bs.idx, bs.val, nrhs=8, tune=True) as Bt:
        b = torch.from_numpy(bs.B).cuda()
        x, infos, rep = Bt.solve(b, tol=TOL, maxit=100000, precision="fp32_ir")
        xu, infu, repu = Bt.solve(b, tol=TOL, maxit=100000, precision="fp32_ru")
    assert rep["status"] == "OK", rep
    assert repu["status"] == "OK", repu
    assert true_rel_res(bs, xu.cpu().numpy()).max() <= TOL
    # reliable updates keep the Krylov space: fewer products than the refinement
    assert repu["products"] < rep["products"]
    X = x.cpu().numpy()
    rr = true_rel_res(bs, X)
    assert rr.max() <= TOL, rr.max()
    assert np.all(infos["status"] == 0)
    sizes = np.diff(bs.row_off)
    for i in (int(np.argmin(sizes)), int(np.argsort(sizes)[len(sizes) // 2])):
        r0, r1, p, j, v = instance(bs, i)
        o = oracle.cg_ir("csr", p, j, v, bs.B[r0:r1, 0], tol=TOL, maxit=100000)
        assert o.status == "OK"
        assert abs(int(infos[i, 0]["iterations"]) - o.iterations) <= 0.10 * o.iterations + 10
