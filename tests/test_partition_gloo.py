"""The multi-device partitions of the pair sums (paper_2110_10749_gb300/
parallel.py), run as two gloo ranks on the CPU with the FP64 oracle standing
in for each rank's device work: row blocks of one operator application
(all-reduce of the zero-filled blocks) and surfaces of a batch (no exchange
until the gather).  The assembled results equal the oracle's whole
application exactly."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2110_10749_gb300 import parallel as par  # noqa: E402


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_row_blocks_cover_and_align():
    for n, world in ((1062, 2), (17070, 3), (138830, 8), (600, 4), (5, 2)):
        blocks = par.row_blocks(n, world)
        assert blocks[0][0] == 0 and blocks[-1][1] == n and len(blocks) == world
        for (b0, e0), (b1, e1) in zip(blocks, blocks[1:]):
            assert e0 == b1
        for b, e in blocks[1:]:
            assert b % par.ROW_ALIGN == 0 or b == n
        sizes = [e - b for b, e in blocks]
        assert max(sizes) - min(sizes) <= 2 * par.ROW_ALIGN   # each cut within half a tile of r n / world


def test_surface_blocks_balance():
    sizes = [4302, 1062, 17070, 2392, 6902, 1742, 4302]
    out = par.surface_blocks(sizes, 3)
    assert sorted(s for v in out for s in v) == list(range(len(sizes)))
    load = [sum(sizes[s] ** 2 for s in v) for v in out]
    assert max(load) == 17070 ** 2       # the largest surface alone bounds the makespan
    assert par.surface_blocks(sizes, 1) == [list(range(len(sizes)))]


def _spatial_order(xyz):
    # any fixed permutation serves as the layout order; a coarse spatial sort
    q = np.floor((xyz + 2.0) * 4.0).astype(np.int64)
    return np.lexsort((q[2], q[1], q[0])).astype(np.int64)


def _rows_rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import oracle
    from oracle import quadrature as Q
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    h = 1 / 8
    p = Q.ellipsoid_points((1.0, 0.8, 0.6), h)
    n = p["w"].size
    order = _spatial_order(p["xyz"])
    rng = np.random.default_rng(3)
    dens = {"laplace_DL": rng.normal(size=n), "stokes_DL": rng.normal(size=(3, n))}
    res = {}
    for name, fn in (("laplace_DL", oracle.laplace_dl), ("stokes_DL", oracle.stokes_dl)):
        d = dens[name]

        def rows(b, e, d=d, fn=fn):
            out = np.zeros_like(d)
            if e > b:
                out[..., order[b:e]] = fn(p, 3 * h, d, rows=order[b:e])
            return torch.from_numpy(out)

        def reduce(x):
            dist.all_reduce(x)
        res[name] = par.sharded_apply(rows, n, rank, world, reduce, align=128).numpy()
    q.put((rank, res))
    dist.destroy_process_group()


def test_row_block_apply_two_gloo_ranks():
    import oracle
    from oracle import quadrature as Q
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_rows_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    got = dict(q.get(timeout=300) for _ in range(2))
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    h = 1 / 8
    p = Q.ellipsoid_points((1.0, 0.8, 0.6), h)
    rng = np.random.default_rng(3)
    n = p["w"].size
    ref = {"laplace_DL": oracle.laplace_dl(p, 3 * h, rng.normal(size=n)),
           "stokes_DL": oracle.stokes_dl(p, 3 * h, rng.normal(size=(3, n)))}
    for rank in (0, 1):
        for k, v in ref.items():
            assert np.array_equal(got[rank][k], v), (rank, k)


def _surfaces():
    from oracle import quadrature as Q
    return [Q.sphere_points(1.0, 1 / 6), Q.ellipsoid_points((1.0, 0.8, 0.6), 1 / 8),
            Q.sphere_points(0.7, 1 / 10), Q.ellipsoid_points((1.0, 0.6, 0.4), 1 / 10),
            Q.sphere_points(1.2, 1 / 5)]


def _surf_rank(rank, world, port, q):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    surfs = _surfaces()
    mine = par.surface_blocks([s["w"].size for s in surfs], world)[rank]
    local = {}
    for k in mine:
        s = surfs[k]
        g = np.cos(3.0 * s["xyz"][0]) + s["xyz"][2]
        local[k] = oracle.laplace_dl(s, 3.0 / 8, g)
    gathered = [None] * world
    dist.all_gather_object(gathered, local)
    q.put((rank, {k: v for part in gathered for k, v in part.items()}, mine))
    dist.destroy_process_group()


def test_surface_split_two_gloo_ranks():
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_surf_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    got = [q.get(timeout=300) for _ in range(2)]
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    surfs = _surfaces()
    owned = sorted(k for _, _, mine in got for k in mine)
    assert owned == list(range(len(surfs)))
    for _, res, _ in got:
        for k, s in enumerate(surfs):
            g = np.cos(3.0 * s["xyz"][0]) + s["xyz"][2]
            assert np.array_equal(res[k], oracle.laplace_dl(s, 3.0 / 8, g))
