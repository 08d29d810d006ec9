"""Slab decomposition of the block grid (the multi-GPU sharding of the method: x slabs,
one-block halo for WCSPH, two for PCISPH's 2-ring search, migration after re-binning),
checked with gloo ranks on the CPU: after migration every rank owns exactly the
particles of its slab, each particle once; after the halo exchange every neighbour of an
owned particle (brute force over the whole scene) is owned or a ghost on that rank; the
fields travel with their particles unchanged."""
import json
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _scene(pcisph):
    from paper_2009_14514_gb300 import scenes
    if pcisph:
        return scenes.pool_drop((16, 12, 4), 4, 0.02, 0.01, (0.16, 0.12, 0.12), 3.5e-4,
                                jitter=2e-3, seed=5)
    return scenes.dam_break((16, 6, 6), 0.02, (0.4, 0.2, 0.2), 1e-4, jitter=3e-3, seed=9)


def _rank_main(rank, world, port, out_dir, pcisph):
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    import oracle as O
    from paper_2009_14514_gb300 import slabs
    sc = _scene(pcisph)
    halo = slabs.halo_layers(sc.params)
    part = slabs.SlabPartition(sc.params, world, halo=halo)
    assert slabs.halo_reach_ok(part, sc.params)
    x = sc.x.astype(np.float64)
    n = len(x)
    ids = np.arange(n)
    vel = np.random.default_rng(1).normal(size=(n, 3))
    # start from the owners of positions shifted by a third of a block: after the move
    # each rank hands the particles that crossed into a neighbour's slab to it
    x_old = x.copy()
    x_old[:, 0] -= part.edge / 3
    mine = part.owner(x_old) == rank
    oid, ox, (ov,) = slabs.migrate(part, ids[mine], x[mine], (vel[mine],))
    res = {"owned": oid.tolist(),
           "owner_ok": bool(np.all(part.owner(ox) == rank)),
           "fields_ok": bool(np.array_equal(ov, vel[oid]) and np.array_equal(ox, x[oid]))}
    gid, gx, (gv,) = slabs.halo_exchange(part, oid, ox, (ov,))
    res["ghosts"] = gid.tolist()
    res["ghost_fields_ok"] = bool(np.array_equal(gv, vel[gid]) and np.array_equal(gx, x[gid]))
    # every neighbour (the whole scene, brute force) of an owned particle is here; the
    # 2-ring search of PCISPH region 1 reaches up to two blocks: all particles within
    # two block edges must be here as well
    off, idx = O.neighbors_brute(x, np.zeros((0, 3)), float(sc.params["support_r"]))
    here = set(oid.tolist()) | set(gid.tolist())
    res["neighbours_ok"] = all(int(j) in here for i in oid for j in idx[off[i]:off[i + 1]])
    reach = halo * part.edge
    col = part.column(x)
    lo, hi = part.lo[rank], part.lo[rank + 1]
    need = np.nonzero((col >= lo - halo) & (col < hi + halo))[0]
    res["reach_ok"] = set(need.tolist()) <= here
    res["reach"] = reach
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world, pcisph", [(2, False), (3, False), (2, True)])
def test_slab_migration_and_halo_exchange(tmp_path, world, pcisph):
    port = _free_port()
    mp.spawn(_rank_main, args=(world, port, str(tmp_path), pcisph), nprocs=world, join=True)
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(world)]
    n = len(_scene(pcisph).x)
    owned = sorted(i for rr in r for i in rr["owned"])
    assert owned == list(range(n))                     # every particle owned exactly once
    for rr in r:
        assert rr["owner_ok"] and rr["fields_ok"] and rr["ghost_fields_ok"]
        assert rr["neighbours_ok"] and rr["reach_ok"]
        assert len(rr["ghosts"]) > 0 and not set(rr["ghosts"]) & set(rr["owned"])


def test_slab_bounds_balance_particle_counts():
    sys.path.insert(0, ROOT)
    from paper_2009_14514_gb300 import slabs
    sc = _scene(False)
    part = slabs.SlabPartition(sc.params, 4)
    assert part.lo[0] == 0 and part.lo[-1] == part.nx and part.lo == sorted(part.lo)
    counts = np.bincount(part.column(sc.x), minlength=part.nx)
    bal = slabs.SlabPartition(sc.params, 2, weights=counts)
    own = bal.owner(sc.x)
    assert abs(int((own == 0).sum()) - int((own == 1).sum())) <= counts.max()
    with pytest.raises(ValueError):
        slabs.SlabPartition(sc.params, part.nx + 1)
