"""The band decomposition of one image (paper_1512_01383_gb300.bands) at world
size 2 and 3 on CPU (gloo): each rank runs the FP64 oracle on its band of
rows plus one halo row on each side, the package's exchange schedule
(DistributedBand) moves the halo rows between ranks by point-to-point
messages, and the own rows after the iterations must equal, bit for bit,
those of the oracle run on the whole image; the energies summed by the
schedule's all_reduce must equal the whole image's (up to the order of the
FP64 sums)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.dirname(os.path.abspath(__file__))

FIELDS = ("u", "s", "ubar", "sbar", "v", "z", "px", "py")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleBand:
    """A band of the image as an oracle problem: the own rows [row0, row1)
    and the halo rows around them, with the operations of the schedule.  The
    halo formats are this class's own (FP64 arrays); the oracle runs its
    half-steps over the whole local image, and the halo rows' own updates,
    which no own row reads, are overwritten by the next import."""

    def __init__(self, c, row0, row1):
        import oracle as O
        from _cases import crop, oracle_problem
        self.O = O
        H, W = c["H"], c["W"]
        self.up, self.dn = int(row0 > 0), int(row1 < H)
        self.n, self.W, self.k = row1 - row0, W, c["L"] - 1
        self.row0, self.row1 = row0, row1
        loc = crop(c, row0 - self.up, row1 + self.dn, 0, W)
        self.P = oracle_problem(loc)
        self.X = O.State(self.P)
        self.rec = W * self.k

    def rows(self, r):
        return slice(r * self.W, (r + 1) * self.W)

    def halo_bytes(self, which):
        return 4 * self.rec * 8

    def export(self, which, buf):
        a = buf.numpy().view(np.float64).reshape(4, self.W, self.k)
        if which == 0:        # first own row's primal records
            r = self.rows(self.up)
            for j, n in enumerate(("u", "s", "ubar", "sbar")):
                a[j] = getattr(self.X, n)[r]
        else:                 # last own row's dual records
            r = self.rows(self.up + self.n - 1)
            for j, n in enumerate(("v", "z", "px", "py")):
                a[j] = getattr(self.X, n)[r]

    def import_(self, which, buf):
        a = buf.numpy().view(np.float64).reshape(4, self.W, self.k)
        if which == 0:        # into the halo row below
            r = self.rows(self.up + self.n)
            for j, n in enumerate(("u", "s", "ubar", "sbar")):
                getattr(self.X, n)[r] = a[j]
        else:                 # into the halo row above
            r = self.rows(0)
            for j, n in enumerate(("v", "z", "px", "py")):
                getattr(self.X, n)[r] = a[j]

    def dual_step(self):
        self.O.half_step(self.P, self.X, 0)

    def primal_step(self):
        self.O.half_step(self.P, self.X, 1)

    def own(self):
        r = slice(self.up * self.W, (self.up + self.n) * self.W)
        return {n: getattr(self.X, n)[r].copy() for n in FIELDS} | {"q": self.X.q[r].copy()}

    def energy(self):
        """Markers of this band (its first and last own row and a count):
        the test checks that the schedule's all_reduce sums them over the
        ranks (the energies' per-band sums are checked on the GPU)."""
        return (float(self.row0), float(self.row1), 1.0)


def _worker(rank, world, port, c, iters, out):
    import torch.distributed as dist
    sys.path[:0] = [ROOT, TESTS]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1512_01383_gb300.bands import DistributedBand, band_rows
        r0, r1 = band_rows(c["H"], world)[rank]
        band = OracleBand(c, r0, r1)
        sched = DistributedBand(band, rank, world, lambda n: torch.empty(n, dtype=torch.uint8))
        sched.iterate(iters)
        e = sched.energy("cpu")      # runs the halo exchange and the FP64 all_reduce
        out.put((rank, r0, r1, band.own(), e))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _run(world, c, iters):
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, c, iters, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=300) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(res, key=lambda t: t[0])


@pytest.mark.parametrize("world,kind,H,W,L", [(2, 1, 11, 9, 5), (3, 2, 13, 7, 4), (2, 0, 6, 10, 3)])
def test_bands_over_ranks_equal_the_whole_image(world, kind, H, W, L):
    sys.path[:0] = [ROOT, TESTS]
    import oracle as O
    from _cases import case, oracle_run
    c = case(kind, H, W, L, 4100 + H, ndisp=9) if kind == 2 else case(kind, H, W, L, 4100 + H)
    iters = 25
    res = _run(world, c, iters)
    P, X = oracle_run(c, iters)
    rows = []
    for rank, r0, r1, own, e in res:
        rows.append((r0, r1))
        sl = slice(r0 * W, r1 * W)
        for n in FIELDS:
            np.testing.assert_array_equal(own[n], getattr(X, n)[sl], err_msg=f"{n} rank {rank}")
        np.testing.assert_array_equal(own["q"], X.q[sl])
    assert rows[0][0] == 0 and rows[-1][1] == H
    assert all(rows[j][1] == rows[j + 1][0] for j in range(len(rows) - 1))
    # every rank got the sums over all ranks
    want = (float(sum(r[0] for r in rows)), float(sum(r[1] for r in rows)), float(world))
    for *_, e in res:
        assert tuple(e) == want
