"""Spatial domain decomposition of the block grid into x slabs, one per rank.

The regional-time-stepping path shards by space: the block grid (Section 3) is cut along
x into contiguous slabs of whole blocks, rank k owning slab k.  Every step that needs
neighbours (density, forces, R_min, the PCISPH region expansion and 2-ring search) reads
only blocks within a fixed reach of its own, so a rank needs, besides its own particles,
copies of the particles in the `halo` block layers just outside its slab (one layer for
WCSPH; two for the PCISPH 2-ring search of R_1).  After each re-binning, particles whose
block moved into another slab migrate to its owner.

This module holds the host side of that decomposition over torch.distributed: the slab
bounds (equal widths, or balanced by per-column particle counts), the owner of each
particle, the halo exchange and the migration, with point-to-point send/recv between
neighbouring ranks on host tensors (gloo).  Every exchanged row is copied into the
receiving rank's own memory; nothing reads another rank's memory directly.  It moves
arrays only: stepping a slab with ghost particles on each rank's GPU is not built (every
machine of this build has one GPU), so the multi-GPU benchmark runs replicas.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


class SlabPartition:
    """x slabs of the block grid: rank k owns block columns [lo[k], lo[k + 1])."""

    def __init__(self, params: dict, world: int, halo: int = 1, weights=None):
        if world < 1:
            raise ValueError("world must be >= 1")
        self.origin = float(params["domain_min"][0])
        self.edge = float(params["block_edge"])
        self.nx = int(params["grid_dim"][0])
        if world > self.nx:
            raise ValueError(f"{world} slabs of a grid {self.nx} blocks wide")
        self.world = world
        self.halo = int(halo)
        if weights is None:   # equal numbers of block columns
            self.lo = [int(round(k * self.nx / world)) for k in range(world + 1)]
        else:                 # balance the given per-column weights (e.g. particle counts)
            w = np.asarray(weights, np.float64)
            if w.shape != (self.nx,):
                raise ValueError("weights: one value per block column")
            c = np.concatenate([[0.0], np.cumsum(w)])
            tot = c[-1]
            self.lo = [0]
            for k in range(1, world):
                b = int(np.searchsorted(c, tot * k / world))
                self.lo.append(min(max(b, self.lo[-1] + 1), self.nx - (world - k)))
            self.lo.append(self.nx)
        if min(self.lo[k + 1] - self.lo[k] for k in range(world)) < max(1, self.halo):
            raise ValueError("every slab must be at least as wide as the halo")

    def column(self, x) -> np.ndarray:
        """Block column (x index) of each position, clamped to the grid."""
        x = np.asarray(x, np.float64)
        c = np.floor((x[:, 0] - self.origin) / self.edge).astype(np.int64)
        return np.clip(c, 0, self.nx - 1)

    def owner(self, x) -> np.ndarray:
        """Rank owning each position's block."""
        return np.searchsorted(np.asarray(self.lo[1:-1]), self.column(x), side="right")

    def halo_for(self, x, rank: int):
        """Masks of the positions (owned by `rank`) that the left and right neighbours
        need: those in the halo block layers just outside the neighbours' slabs."""
        c = self.column(x)
        left = (c >= self.lo[rank]) & (c < self.lo[rank] + self.halo) if rank > 0 else np.zeros(len(c), bool)
        right = ((c >= self.lo[rank + 1] - self.halo) & (c < self.lo[rank + 1])
                 if rank + 1 < self.world else np.zeros(len(c), bool))
        return left, right


def _exchange(send_left, send_right, rank, world, like):
    """Send one tensor to each neighbour and receive theirs (row counts first).  Even
    ranks send first and odd ranks receive first, so the blocking point-to-point calls
    never wait on each other in a cycle.  Returns the tensors received from the left and
    the right (empty at the ends of the row of slabs)."""
    def sendrecv(peer, out_t, width):
        n_out = torch.tensor([out_t.shape[0]], dtype=torch.int64, device=like.device)
        n_in = torch.zeros(1, dtype=torch.int64, device=like.device)
        if rank % 2 == 0:
            dist.send(n_out, peer)
            dist.recv(n_in, peer)
        else:
            dist.recv(n_in, peer)
            dist.send(n_out, peer)
        inp = torch.empty((int(n_in.item()), width), dtype=like.dtype, device=like.device)
        if rank % 2 == 0:
            if out_t.shape[0]:
                dist.send(out_t.contiguous(), peer)
            if inp.shape[0]:
                dist.recv(inp, peer)
        else:
            if inp.shape[0]:
                dist.recv(inp, peer)
            if out_t.shape[0]:
                dist.send(out_t.contiguous(), peer)
        return inp

    width = like.shape[1]
    empty = torch.empty((0, width), dtype=like.dtype, device=like.device)
    got_left = sendrecv(rank - 1, send_left, width) if rank > 0 else empty
    got_right = sendrecv(rank + 1, send_right, width) if rank + 1 < world else empty
    return got_left, got_right


def pack(ids, fields):
    """One float64 row per particle: id, then the fields' columns (float64 holds the ids
    and FP32 values exactly)."""
    cols = [torch.as_tensor(np.asarray(ids, np.float64)).reshape(-1, 1)]
    for f in fields:
        t = torch.as_tensor(np.asarray(f, np.float64))
        cols.append(t.reshape(t.shape[0], -1))
    return torch.cat(cols, dim=1)


def unpack(rows, widths):
    """Inverse of pack: ids (int64) and the fields (float64 arrays of the given widths)."""
    r = rows.cpu().numpy()
    ids = r[:, 0].astype(np.int64)
    out, k = [], 1
    for w in widths:
        out.append(r[:, k:k + w] if w > 1 else r[:, k])
        k += w
    return ids, out


def halo_exchange(part: SlabPartition, ids, x, fields=(), rank=None, world=None):
    """Ghost copies for this rank: the particles of the neighbours' slabs that lie in the
    `halo` block layers just outside this rank's slab, with their fields.  Returns
    (ghost ids, ghost x, ghost fields)."""
    rank = dist.get_rank() if rank is None else rank
    world = dist.get_world_size() if world is None else world
    x = np.asarray(x, np.float64)
    rows = pack(ids, (x,) + tuple(fields))
    left, right = part.halo_for(x, rank)
    got_l, got_r = _exchange(rows[torch.as_tensor(left)], rows[torch.as_tensor(right)], rank, world, rows)
    widths = [3] + [int(np.asarray(f).reshape(len(x), -1).shape[1]) for f in fields]
    gid, g = unpack(torch.cat([got_l, got_r]), widths)
    return gid, g[0], g[1:]


def migrate(part: SlabPartition, ids, x, fields=(), rank=None, world=None):
    """Move the particles whose block left this rank's slab to the neighbour that owns it
    (particles move less than a slab between re-binnings, so only neighbours exchange;
    a particle owned further away is an error).  Returns (ids, x, fields) owned here."""
    rank = dist.get_rank() if rank is None else rank
    world = dist.get_world_size() if world is None else world
    x = np.asarray(x, np.float64)
    own = part.owner(x)
    if np.any(np.abs(own - rank) > 1):
        raise ValueError("a particle moved further than the neighbouring slab")
    rows = pack(ids, (x,) + tuple(fields))
    stay = own == rank
    got_l, got_r = _exchange(rows[torch.as_tensor(own == rank - 1)],
                             rows[torch.as_tensor(own == rank + 1)], rank, world, rows)
    widths = [3] + [int(np.asarray(f).reshape(len(x), -1).shape[1]) for f in fields]
    nid, nf = unpack(torch.cat([rows[torch.as_tensor(stay)], got_l, got_r]), widths)
    order = np.argsort(nid, kind="stable")     # a canonical order: by caller id
    return nid[order], nf[0][order], [f[order] for f in nf[1:]]


def halo_layers(params: dict) -> int:
    """Block layers of halo the method needs: 1 for WCSPH (27-block stencil, R_min); for
    PCISPH the 2-ring search of R_1 (r1_search_rings) reaches further, and the region
    expansion by expand_layers is recomputed redundantly inside the halo."""
    if int(params["scheme"]) == 0:
        return 1
    return max(1, int(params.get("r1_search_rings", 2)), int(params.get("r2_search_rings", 1)))


def halo_reach_ok(part: SlabPartition, params: dict) -> bool:
    """The halo covers every block the method reads around an owned block: at least
    halo_layers blocks (the block edge is at least the support radius)."""
    return part.halo >= halo_layers(params) and part.edge >= float(params["support_r"])
