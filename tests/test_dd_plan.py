"""Slab decomposition of the multigrid hierarchy (mg_dd_make_plan), on the CPU.

The plan is host-only library code.  Checked here without a GPU:
  - invariants: every cut level is split into equal slabs of an even number (>= 2) of planes,
    the switch level is not the coarsest, the whole-grid levels follow the oracle's level rule;
  - with the gloo backend at 2 and 4 ranks, the halo exchange and the gather of the coarse
    levels that the plan prescribes: each rank holds its slab of a seeded whole-grid field on
    every cut level (coarse levels by the oracle's 8:1 restriction), swaps its boundary planes
    with its neighbours, and must find bitwise the whole grid's planes in its ghost planes; the
    restriction of its own planes must be bitwise its planes of the next level (pairs never
    straddle two slabs); and the slabs' restrictions gathered on rank 0 at the switch level
    must be bitwise the whole-grid coarse array;
  - for the mixed decomposition's FP32 storage, with 2 and 4 gloo ranks: slabs of 4k planes
    keep the whole grid's colours in their own colour-split storage, a per-colour exchange
    fills each colour half's ghost planes with bitwise the whole grid's split planes, and a
    slab's view of the whole coarse level starts at an even plane (the same colours).
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _plan(dims, coarsest, ranks, max_dec=0):
    sys.path.insert(0, ROOT)
    from paper_2605_30082_gb300 import _lib as L

    return L.mg_dd_make_plan(dims, coarsest, ranks, max_dec)


@pytest.mark.parametrize("dims,coarsest,ranks,max_dec", [((64, 64, 64), 4, 2, 0), ((64, 64, 64), 4, 4, 0),
                                                         ((64, 48, 128), 8, 8, 0), ((64, 64, 32), 4, 4, 0),
                                                         ((96, 80, 64), 8, 2, 2), ((32, 32, 256), 4, 16, 0)])
def test_plan_invariants(dims, coarsest, ranks, max_dec):
    import oracle as O
    from paper_2605_30082_gb300 import _lib as L

    st, pl = _plan(dims, coarsest, ranks, max_dec)
    assert st == L.MG_OK
    nx, ny, nz = dims
    assert pl.ranks == ranks and pl.levels == O.num_levels(nx, ny, nz, coarsest)
    assert 1 <= pl.switch_level < pl.levels
    if max_dec:
        assert pl.switch_level <= max_dec
    for l in range(pl.levels):
        assert (pl.nx[l], pl.ny[l], pl.nz[l]) == (nx >> l, ny >> l, nz >> l)
        if l < pl.switch_level:
            assert pl.planes[l] * ranks == pl.nz[l] and pl.planes[l] >= 2 and pl.planes[l] % 2 == 0
        else:
            assert pl.planes[l] == 0
    # the cut stops only where the rule stops it (or at max_dec)
    s = pl.switch_level
    if s < pl.levels - 1 and (not max_dec or s < max_dec):
        assert pl.nz[s] % ranks or (pl.nz[s] // ranks) % 2 or pl.nz[s] // ranks < 2


def test_plan_rejects_what_cannot_be_cut():
    from paper_2605_30082_gb300 import _lib as L

    assert _plan((64, 64, 60), 4, 8)[0] == L.MG_ERR_ARG    # 60 / 8 is no whole number of planes
    assert _plan((64, 64, 64), 4, 64)[0] == L.MG_ERR_ARG   # one plane per slab: pairs would straddle
    assert _plan((64, 64, 64), 4, 0)[0] == L.MG_ERR_ARG
    assert _plan((64, 64, 64), 4, 65)[0] == L.MG_ERR_ARG   # beyond MG_DD_MAX_RANKS
    assert _plan((4, 4, 4), 4, 2)[0] == L.MG_ERR_ARG       # a single level


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, dims, coarsest, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle as O

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        st, pl = _plan(dims, coarsest, world)
        assert st == 0
        nx, ny, nz = dims
        g = [np.random.default_rng(7).standard_normal((nz, ny, nx))]
        for _ in range(pl.switch_level):
            g.append(O.restrict(g[-1]))
        checks = 0
        for l in range(pl.switch_level):
            m = pl.planes[l]
            z0 = rank * m
            slab = np.zeros((m + 2, pl.ny[l], pl.nx[l]))
            slab[1:-1] = g[l][z0:z0 + m]
            t = torch.from_numpy(slab)  # shares memory with slab
            reqs = []
            if rank > 0:  # first own plane down, ghost below from the rank below
                reqs.append(dist.isend(t[1].clone(), rank - 1, tag=2 * l))
                reqs.append(dist.irecv(t[0], rank - 1, tag=2 * l + 1))
            if rank + 1 < world:  # last own plane up, ghost above from the rank above
                reqs.append(dist.isend(t[m].clone(), rank + 1, tag=2 * l + 1))
                reqs.append(dist.irecv(t[m + 1], rank + 1, tag=2 * l))
            for r in reqs:
                r.wait()
            if rank > 0:
                assert np.array_equal(slab[0], g[l][z0 - 1]), (rank, l, "ghost below")
                checks += 1
            if rank + 1 < world:
                assert np.array_equal(slab[m + 1], g[l][z0 + m]), (rank, l, "ghost above")
                checks += 1
            # the slab's restriction is its part of the next level, bitwise
            rc = O.restrict(np.ascontiguousarray(slab[1:-1]))
            assert np.array_equal(rc, g[l + 1][z0 // 2:(z0 + m) // 2]), (rank, l, "restriction")
            checks += 1
        # the gather onto rank 0 at the switch level
        s = pl.switch_level
        m = pl.planes[s - 1]
        z0 = rank * m
        part = torch.from_numpy(O.restrict(np.ascontiguousarray(g[s - 1][z0:z0 + m])))
        parts = [torch.empty_like(part) for _ in range(world)] if rank == 0 else None
        dist.gather(part, parts, dst=0)
        if rank == 0:
            whole = torch.cat(parts, 0).numpy()
            assert np.array_equal(whole, g[s]), "gathered switch level"
            checks += 1
        q.put((rank, checks, None))
    except Exception as e:  # report, do not hang the others
        q.put((rank, -1, repr(e)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,dims,coarsest", [(2, (32, 24, 64), 4), (4, (32, 16, 64), 4), (4, (16, 16, 32), 4)])
def test_halo_exchange_and_gather_follow_the_plan_gloo(world, dims, coarsest):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, dims, coarsest, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, checks, err in res:
        assert err is None, (rank, err)
        assert checks > 0


def _split(a):
    """Colour-split storage of a whole-grid (or slab) array whose first plane is even: all cells
    with (x + y + z) even, then the odd ones, each colour row by row with cell x at k = x // 2."""
    nz, ny, nx = a.shape
    out = np.zeros((2, nz, ny, nx // 2))
    z, y, x = np.meshgrid(range(nz), range(ny), range(nx), indexing="ij")
    c = (x + y + z) % 2
    out[c, z, y, x // 2] = a
    return out


def _worker_split(rank, world, port, dims, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nx, ny, nz = dims
        m = nz // world
        assert m % 4 == 0  # slabs of 4k planes: even first planes on this level and the next
        g = np.random.default_rng(11).standard_normal((nz, ny, nx))
        whole = _split(g)
        z0 = rank * m
        # the slab's own planes in its own split storage: the whole grid's colours (z0 even)
        own = _split(g[z0:z0 + m])
        assert np.array_equal(own, whole[:, z0:z0 + m]), "slab colours"
        slab = np.zeros((2, m + 2, ny, nx // 2))  # each colour half: ghost below, own planes, ghost above
        slab[:, 1:-1] = own
        checks = 0
        for c in (0, 1):  # one colour per exchange, as after a half sweep of that colour
            t = torch.from_numpy(slab[c])
            reqs = []
            if rank > 0:
                reqs.append(dist.isend(t[1].clone(), rank - 1, tag=10 + 2 * c))
                reqs.append(dist.irecv(t[0], rank - 1, tag=11 + 2 * c))
            if rank + 1 < world:
                reqs.append(dist.isend(t[m].clone(), rank + 1, tag=11 + 2 * c))
                reqs.append(dist.irecv(t[m + 1], rank + 1, tag=10 + 2 * c))
            for r in reqs:
                r.wait()
            if rank > 0:
                assert np.array_equal(slab[c, 0], whole[c, z0 - 1]), (rank, c, "ghost below")
                checks += 1
            if rank + 1 < world:
                assert np.array_equal(slab[c, m + 1], whole[c, z0 + m]), (rank, c, "ghost above")
                checks += 1
        # the coarse view: the slab's coarse planes start at an even whole-grid plane, so their
        # colours in the whole coarse level's storage are the slab's own
        zc0 = z0 // 2
        gc = np.random.default_rng(12).standard_normal((nz // 2, ny // 2, nx // 2))
        assert zc0 % 2 == 0
        assert np.array_equal(_split(gc[zc0:zc0 + m // 2]), _split(gc)[:, zc0:zc0 + m // 2]), "coarse view"
        q.put((rank, checks + 1, None))
    except Exception as e:
        q.put((rank, -1, repr(e)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,dims", [(2, (16, 12, 16)), (4, (16, 8, 32))])
def test_split_layout_exchange_per_colour_gloo(world, dims):
    """The mixed decomposition's layout: each rank's colour-split slab (ghost plane below and
    above in each colour half) receives its neighbours' boundary planes one colour at a time
    and must find bitwise the whole grid's split planes in its ghosts."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_split, args=(r, world, port, dims, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, checks, err in res:
        assert err is None, (rank, err)
        assert checks > 0
