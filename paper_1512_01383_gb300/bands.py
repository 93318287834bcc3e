"""Spatial decomposition of one image problem into bands of rows.

The operator of Sec. 4 couples a pixel only to its forward-difference
neighbours (x+1, y+1 in the gradient, x-1, y-1 in the divergence).  So an
image split into bands of consecutive rows, one band per GPU (or several on
one GPU), needs one row of a neighbouring band per half-step and nothing
else: before the dual step the first own row's primal records (x, xbar) go to
the band above, before the primal step the last own row's dual records (y) go
to the band below.  Each band's own rows then evolve exactly as in a single
solve of the whole image.  The energies of the image are the sums of the
bands' energies (an FP64 allreduce across ranks).

Every step runs in the library's kernels (``lift_create_band``,
``lift_band_export`` / ``lift_band_import``, ``lift_dual_step`` /
``lift_primal_step`` on a band handle); this module orders the half-steps and
moves the halo rows between bands: by device copies between handles on one
device (:class:`LocalBands`), or by point-to-point ``torch.distributed``
messages between ranks (:class:`DistributedBand`, NCCL between GPUs).
"""
from __future__ import annotations

from . import lift as G

PRIMAL, DUAL = G.LIFT_HALO_PRIMAL, G.LIFT_HALO_DUAL


def band_rows(H: int, nbands: int) -> list[tuple[int, int]]:
    """Rows [row0, row1) of each of `nbands` bands of an H-row image, as equal
    as whole rows allow (every band at least one row)."""
    if not 1 <= nbands <= H:
        raise ValueError(f"{nbands} bands of a {H}-row image")
    cuts = [H * j // nbands for j in range(nbands + 1)]
    return [(cuts[j], cuts[j + 1]) for j in range(nbands)]


class HandleBand:
    """One band of the image as a library handle on the current device: the
    operations the exchange schedule needs."""

    def __init__(self, spec: G.lift_spec, row0: int, row1: int, stream: int | None = None):
        self.row0, self.row1 = row0, row1
        self.first, self.last = row0 == 0, row1 == spec.H
        self.h = G.lift_create_band(spec, row0, row1, stream)
        self.W, self.k = spec.W, spec.L - 1

    def halo_bytes(self, which: int) -> int:
        return G.lift_band_halo_bytes(self.h, which)

    def export(self, which: int, buf) -> None:
        G.lift_band_export(self.h, which, buf)

    def import_(self, which: int, buf) -> None:
        G.lift_band_import(self.h, which, buf)

    def dual_step(self) -> None:
        G.lift_dual_step(self.h)

    def primal_step(self) -> None:
        G.lift_primal_step(self.h)

    def energy(self) -> tuple[float, float, float]:
        return G.lift_energy(self.h)

    def unlift(self, out=None):
        return G.lift_unlift(self.h, out) if out is not None else self._unlift_host()

    def _unlift_host(self):
        import numpy as np
        out = np.empty((self.row1 - self.row0, self.W), dtype=np.float32)
        G.lift_unlift(self.h, out)
        return out

    def close(self) -> None:
        if self.h:
            G.lift_destroy(self.h)
            self.h = 0


class LocalBands:
    """All bands of one image on the current device, on one stream; the halos
    move by device-to-device copies through a staging buffer per boundary."""

    def __init__(self, spec: G.lift_spec, nbands: int, stream: int | None = None):
        import torch
        self.bands = [HandleBand(spec, r0, r1, stream) for r0, r1 in band_rows(spec.H, nbands)]
        dev = torch.device("cuda", torch.cuda.current_device())
        nb = lambda w: self.bands[0].halo_bytes(w)
        self.buf = {w: [torch.empty(nb(w), dtype=torch.uint8, device=dev) for _ in self.bands]
                    for w in (PRIMAL, DUAL)}

    def _exchange_primal(self) -> None:
        for j in range(1, len(self.bands)):           # first own row -> band above
            self.bands[j].export(PRIMAL, self.buf[PRIMAL][j])
            self.bands[j - 1].import_(PRIMAL, self.buf[PRIMAL][j])

    def _exchange_dual(self) -> None:
        for j in range(len(self.bands) - 1):          # last own row -> band below
            self.bands[j].export(DUAL, self.buf[DUAL][j])
            self.bands[j + 1].import_(DUAL, self.buf[DUAL][j])

    def iterate(self, iters: int) -> None:
        for _ in range(iters):
            self._exchange_primal()
            for b in self.bands:
                b.dual_step()
            self._exchange_dual()
            for b in self.bands:
                b.primal_step()

    def energy(self) -> tuple[float, float, float]:
        """(P, D, E_nc) of the whole image: the bands' sums (after bringing
        the halo rows below up to date)."""
        self._exchange_primal()
        tot = [0.0, 0.0, 0.0]
        for b in self.bands:
            for i, v in enumerate(b.energy()):
                tot[i] += v
        return tot[0], tot[1], tot[2]

    def unlift(self):
        import numpy as np
        return np.concatenate([b.unlift() for b in self.bands], axis=0)

    def close(self) -> None:
        for b in self.bands:
            b.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class DistributedBand:
    """The band of this rank in a ``torch.distributed`` group of world_size
    bands (rank r owns band r of band_rows(H, world_size)).  ``band`` is any
    object with the HandleBand operations (halo_bytes, export, import_,
    dual_step, primal_step, energy); ``alloc(nbytes)`` returns a staging
    tensor on the device the process group communicates from (CUDA for NCCL,
    CPU for gloo).  Halo rows travel by isend / irecv between neighbouring
    ranks; the energies are summed by an FP64 all_reduce."""

    def __init__(self, band, rank: int, world: int, alloc, group=None):
        self.band, self.rank, self.world, self.group = band, rank, world, group
        self.send = {w: alloc(band.halo_bytes(w)) for w in (PRIMAL, DUAL)}
        self.recv = {w: alloc(band.halo_bytes(w)) for w in (PRIMAL, DUAL)}

    def _exchange(self, which: int) -> None:
        import torch.distributed as dist
        # PRIMAL goes up (to rank - 1), DUAL goes down (to rank + 1)
        to = self.rank - 1 if which == PRIMAL else self.rank + 1
        frm = self.rank + 1 if which == PRIMAL else self.rank - 1
        ops = []
        if 0 <= to < self.world:
            self.band.export(which, self.send[which])
            ops.append(dist.P2POp(dist.isend, self.send[which], to, self.group))
        if 0 <= frm < self.world:
            ops.append(dist.P2POp(dist.irecv, self.recv[which], frm, self.group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        if 0 <= frm < self.world:
            self.band.import_(which, self.recv[which])

    def iterate(self, iters: int) -> None:
        for _ in range(iters):
            self._exchange(PRIMAL)
            self.band.dual_step()
            self._exchange(DUAL)
            self.band.primal_step()

    def energy(self, device) -> tuple[float, float, float]:
        import torch
        import torch.distributed as dist
        self._exchange(PRIMAL)
        e = torch.tensor(self.band.energy(), dtype=torch.float64, device=device)
        if self.world > 1:
            dist.all_reduce(e, op=dist.ReduceOp.SUM, group=self.group)
        return float(e[0]), float(e[1]), float(e[2])
