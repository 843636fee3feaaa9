"""Host-side bookkeeping of the x-slab decomposition (no GPU): the slab plan, the electron
exchange rules, and a two-rank exchange over gloo in which each rank holds one slab of a
synthetic window and trades its boundary electrons with the other through send/recv."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1912_04674_gb300 import slabs


@pytest.mark.parametrize("nx,nslab,halo", [(96, 2, 8), (96, 3, 8), (2048, 4, 13), (50, 1, 8), (257, 3, 9)])
def test_plan_partitions_the_window(nx, nslab, halo):
    plan = slabs.plan_slabs(nx, nslab, halo)
    assert [s.index for s in plan] == list(range(nslab))
    assert plan[0].own_lo == 0 and plan[-1].own_hi == nx
    assert all(a.own_hi == b.own_lo for a, b in zip(plan, plan[1:]))
    assert [s.front for s in plan] == [False] * (nslab - 1) + [True]
    for a, b in zip(plan, plan[1:]):
        B = b.own_lo
        assert b.x0 == B - halo and a.x0 + a.nx == B + halo      # the exchange's geometry
    for s in plan:
        assert s.own_hi - s.own_lo >= 2 * halo and s.nx >= 2 * halo
        assert s.x0 >= 0 and s.x0 + s.nx <= nx
    # node columns of the whole-window arrays: each taken from exactly one slab
    cols = np.concatenate([np.arange(*slabs.owned_nodes(s, nx)) for s in plan])
    assert np.array_equal(cols, np.arange(nx + 1))


def test_plan_refuses_slabs_narrower_than_two_halos():
    with pytest.raises(ValueError):
        slabs.plan_slabs(40, 3, 8)
    assert slabs.min_halo() == 8 and slabs.min_halo(7) == 15


def test_exchange_rules():
    plan = slabs.plan_slabs(64, 2, 8)
    L, R = plan
    B = R.own_lo
    cl = np.arange(L.x0, L.x0 + L.nx)              # one electron per cell of each local window
    cr = np.arange(R.x0, R.x0 + R.nx)
    e = slabs.exchange_sets(L, cl, R, cr, 8)
    assert np.array_equal(cl[e["keep_left"]], np.arange(0, B))
    assert np.array_equal(cr[e["keep_right"]], np.arange(B, R.x0 + R.nx))
    assert np.array_equal(cr[e["right_to_left"]], np.arange(B, B + 8))
    assert np.array_equal(cl[e["left_to_right"]], np.arange(B - 8, B))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _window_electrons(nx, seed=3):
    """A synthetic window: 4 electrons per cell, ids 0..4nx-1, cells after one step of drift
    (less than a cell either way) and one window shift."""
    rng = np.random.default_rng(seed)
    ids = np.arange(4 * nx)
    x = ids // 4 + rng.uniform(0, 1, ids.size)
    x = x + rng.uniform(-0.9, 0.9, ids.size) - 1.0
    return ids, np.floor(x).astype(np.int64)


def _rank(rank, port, q, nx, halo):
    import sys
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2")
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist

    from paper_1912_04674_gb300 import slabs as S
    dist.init_process_group("gloo", rank=rank, world_size=2)
    plan = S.plan_slabs(nx, 2, halo)
    me, other = plan[rank], plan[1 - rank]
    ids, cells = _window_electrons(nx)
    # before the step this rank held its local window (owned cells and halo copies); the
    # step moved them; electrons that left the local window were dropped by the position push
    held = (ids // 4 >= me.x0) & (ids // 4 < me.x0 + me.nx)
    ids, cells = ids[held], cells[held]
    inside = (cells >= me.x0) & (cells < me.x0 + me.nx) & (cells >= 0)
    ids, cells = ids[inside], cells[inside]
    # the exchange: each side computes its own half of the rules
    n_mine = torch.tensor([cells.size])
    n_other = torch.zeros(1, dtype=torch.int64)
    req = [dist.isend(n_mine, 1 - rank), dist.irecv(n_other, 1 - rank)]
    for r in req:
        r.wait()
    B = plan[1].own_lo
    if rank == 0:
        keep = cells < B
        send = keep & (cells >= B - halo)
    else:
        keep = cells >= B
        send = keep & (cells < B + halo)
    out = torch.from_numpy(np.stack([ids[send], cells[send]]).astype(np.int64))
    cnt = torch.tensor([out.shape[1]])
    got_cnt = torch.zeros(1, dtype=torch.int64)
    for r in [dist.isend(cnt, 1 - rank), dist.irecv(got_cnt, 1 - rank)]:
        r.wait()
    got = torch.zeros((2, int(got_cnt.item())), dtype=torch.int64)
    for r in [dist.isend(out.contiguous(), 1 - rank), dist.irecv(got, 1 - rank)]:
        r.wait()
    new_ids = np.concatenate([ids[keep], got[0].numpy()])
    new_cells = np.concatenate([cells[keep], got[1].numpy()])
    dist.barrier()
    q.put((rank, new_ids, new_cells, me))
    dist.destroy_process_group()


def test_two_rank_exchange_over_gloo():
    nx, halo = 64, 8
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q, nx, halo)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r, i, c, sl = q.get(timeout=120)
        res[r] = (i, c, sl)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ids, cells = _window_electrons(nx)
    alive = (cells >= 0) & (cells < nx)
    owned = []
    for r, (i, c, sl) in res.items():
        assert len(np.unique(i)) == len(i)                  # no electron twice on a rank
        lo, hi = sl.x0, sl.x0 + sl.nx
        assert np.all((c >= lo) & (c < hi))                  # within the local window
        own = (c >= sl.own_lo) & (c < sl.own_hi)
        owned.append(i[own])
        # every electron of the whole window that lies in this rank's local window is held
        want = set(ids[alive & (cells >= lo) & (cells < hi)].tolist())
        assert set(i.tolist()) == want
    allown = np.concatenate(owned)
    assert np.array_equal(np.sort(allown), np.sort(ids[alive]))   # each electron owned once
