"""One instance split into r* slabs with halo rows (Sec. 4's decomposition
of the grid work into independent pieces, here along r*).

A slab of the global grid (rows 0 .. Nr-1 at r*_i = r*_min + i dr*) owns the
interior rows [a, b) and carries h halo rows on each side that touches
another slab.  It is an ordinary context over its own r* range, so its
coefficients, source patch and extraction node are those of the global grid
at the same r*.  The step treats the first and last rows of a context as
grid boundary rows: the implicit angular stage (row-local) skips them and
the Lax-Wendroff stages (one row of reach per stage pair) zero them.  A
slab's outermost halo row therefore misses the angular stage in the first
step, which spoils the next row inward, and every further step spoils one
more row.  With h halo rows, h - 1 steps leave every owned row exactly what
the whole grid computes; the global boundary rows are the outer rows of the
first and last slab.  Stepping h - 1 steps, then copying each slab's
outermost h owned rows into the neighbour's halo, repeats that.

halo_plan gives the row ranges of every copy; SlabStepper runs the slabs of
one grid in one process (the neighbours' rows copied on the device), and
exchange_halos_dist moves the same rows between ranks that hold one slab
each (torch.distributed point-to-point).
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class SlabGeom:
    a: int          # first interior (owned) global row
    b: int          # one past the last owned global row
    hl: int         # halo rows below a (0 for the first slab)
    hr: int         # halo rows above b-1 (0 for the last slab)

    @property
    def rows(self) -> int:
        return self.b - self.a + self.hl + self.hr

    @property
    def g0(self) -> int:
        """Global row of local row 0."""
        return self.a - self.hl


def slab_bounds(Nr: int, nslabs: int, halo: int) -> list[SlabGeom]:
    """nslabs contiguous slabs of near-equal size covering rows 0 .. Nr-1,
    each with `halo` rows on the sides that touch another slab."""
    if nslabs < 1 or halo < 1:
        raise ValueError("need nslabs >= 1 and halo >= 1")
    if Nr < nslabs * max(halo, 3):
        raise ValueError("slabs must own at least max(halo, 3) rows each")
    out = []
    for k in range(nslabs):
        a = (Nr * k) // nslabs
        b = (Nr * (k + 1)) // nslabs
        out.append(SlabGeom(a, b, 0 if k == 0 else halo, 0 if k == nslabs - 1 else halo))
    return out


def halo_plan(geoms: list[SlabGeom], halo: int) -> list[tuple[int, slice, int, slice]]:
    """Copies (src slab, src local rows, dst slab, dst local rows) that
    refresh every halo row from its owner after `halo` steps."""
    plan = []
    for k in range(len(geoms) - 1):
        L, R = geoms[k], geoms[k + 1]
        # L's top `halo` owned rows -> R's lower halo; R's bottom owned rows -> L's upper halo
        plan.append((k, slice(L.rows - L.hr - halo, L.rows - L.hr), k + 1, slice(0, halo)))
        plan.append((k + 1, slice(R.hl, R.hl + halo), k, slice(L.rows - halo, L.rows)))
    return plan


def steps_per_exchange(halo: int) -> int:
    """Steps between halo refreshes that h halo rows allow."""
    if halo < 2:
        raise ValueError("halo exchange needs at least two halo rows")
    return halo - 1


def local_rows(geom: SlabGeom) -> slice:
    """Local rows of the owned (interior) part of a slab."""
    return slice(geom.hl, geom.hl + geom.b - geom.a)


class SlabStepper:
    """One grid stepped as `nslabs` slab contexts on one device, with the
    `halo` halo rows copied between them every halo - 1 steps.  Keyword
    arguments are those of teuk.Stepper for the whole grid."""

    def __init__(self, nslabs: int, halo: int = 3, **kw):
        from . import teuk
        self.Nr, self.Ntheta = int(kw["Nr"]), int(kw["Ntheta"])
        rs_min, rs_max = float(kw["rstar_min"]), float(kw["rstar_max"])
        drs = (rs_max - rs_min) / (self.Nr - 1)
        kw.setdefault("dt", 0.5 * drs)
        self.halo = int(halo)
        self.chunk = steps_per_exchange(self.halo)
        self.geoms = slab_bounds(self.Nr, nslabs, self.halo)
        self.plan = halo_plan(self.geoms, self.halo)
        self.slabs = []
        for g in self.geoms:
            sk = dict(kw, Nr=g.rows, rstar_min=rs_min + g.g0 * drs, rstar_max=rs_min + (g.g0 + g.rows - 1) * drs)
            self.slabs.append(teuk.Stepper(**sk))
        i_ext = int(round((float(kw["rstar_extract"]) - rs_min) / drs))
        i_ext = min(max(i_ext, 0), self.Nr - 1)
        self.owner = next(k for k, g in enumerate(self.geoms) if g.a <= i_ext < g.b)

    def set_source(self, *args, **kwargs):
        for st in self.slabs:
            st.set_source(*args, **kwargs)

    def set_state(self, u, step: int = 0):
        """u: the whole grid's [2, Nr, Ntheta] complex state."""
        for g, st in zip(self.geoms, self.slabs):
            st.set_state(u[:, g.g0:g.g0 + g.rows, :], step)

    def _exchange(self):
        views = []
        for st in self.slabs:
            st.synchronize()
            views.append(st.level_view()[0])
        for src, srows, dst, drows in self.plan:
            views[dst][:, drows, :].copy_(views[src][:, srows, :])
        import torch
        torch.cuda.synchronize(self.slabs[0].device)

    def step(self, n: int):
        """Advance n steps in chunks of halo - 1 steps (the last chunk may be
        shorter), refreshing the halos after each chunk."""
        left = int(n)
        while left > 0:
            k = min(self.chunk, left)
            for st in self.slabs:
                st.step(k)
            self._exchange()
            left -= k

    def get_state(self):
        """The whole grid's physical state, assembled from the owned rows."""
        import numpy as np
        parts = [st.get_state()[:, local_rows(g), :] for g, st in zip(self.geoms, self.slabs)]
        return np.concatenate(parts, axis=1)

    def waveform(self, first: int, count: int):
        """Samples at the extraction radius, from the slab that owns it."""
        return self.slabs[self.owner].waveform(first, count)

    @property
    def current_step(self) -> int:
        return self.slabs[0].current_step

    def close(self):
        for st in self.slabs:
            st.close()


def exchange_halos_dist(level, geom: SlabGeom, halo: int, rank: int, world: int, group=None):
    """Refresh the halo rows of this rank's slab (level: its [2, rows, Ntheta]
    state) from the neighbouring ranks' slabs, by point-to-point sends of the
    rows halo_plan names.  Rank k holds slab k."""
    import torch.distributed as dist
    ops = []
    bufs = []
    if rank + 1 < world:   # upper neighbour
        up = level[:, geom.rows - geom.hr - halo:geom.rows - geom.hr, :].contiguous()
        rx = level[:, geom.rows - halo:geom.rows, :].clone()
        ops.append(dist.isend(up, rank + 1, group=group))
        ops.append(dist.irecv(rx, rank + 1, group=group))
        bufs.append((slice(geom.rows - halo, geom.rows), rx))
    if rank > 0:           # lower neighbour
        dn = level[:, geom.hl:geom.hl + halo, :].contiguous()
        rx = level[:, 0:halo, :].clone()
        ops.append(dist.isend(dn, rank - 1, group=group))
        ops.append(dist.irecv(rx, rank - 1, group=group))
        bufs.append((slice(0, halo), rx))
    for op in ops:
        op.wait()
    for rows, rx in bufs:
        level[:, rows, :] = rx
