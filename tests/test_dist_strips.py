"""Row-strip decomposition across processes on the CPU (gloo): the host side
(paper_1101_0876_gb300.strips: the split of the rows, the halo-row exchange
between neighbouring ranks, the sum of the partial records) driven with the
oracle's band pass as the strip's colour pass.  World sizes 2 and 3 must
reproduce the whole-lattice oracle's spins and every record; a strip object
that hands out the wrong rows for the exchange must be caught.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


class OracleBand:
    """A strip held as (nrows + 2) x L row-major bytes (halo rows first and
    last), swept by oracle.band_pass; the exchange moves whole rows, which
    is more than the colour pass needs and changes nothing it reads."""

    def __init__(self, L, q, seed, row0, own_rows, update, swap_rows=False):
        self.L, self.q, self.seed, self.row0 = L, q, seed, row0
        self.update = update
        n = own_rows.shape[0]
        self.buf = np.zeros((n + 2, L), np.uint8)
        self.buf[1:n + 1] = own_rows
        self.t = 0
        self.n = n
        self.swap = swap_rows
        self.view = torch.from_numpy(self.buf)

    def rows(self, colour):
        first, last = self.view[1], self.view[self.n]
        if self.swap:                      # planted mistake
            first, last = last, first
        return first, last, self.view[0], self.view[self.n + 1]

    def new_record(self):
        return torch.zeros(1 + self.q, dtype=torch.int64)

    def pass_(self, beta, colour, record):
        import oracle
        part = np.zeros(1 + self.q, np.uint64)
        oracle.band_pass(self.buf, self.L, self.q, self.row0, self.seed,
                         self.t, colour, beta, part, self.update)
        record += torch.from_numpy(part.astype(np.int64))
        if colour == 1:
            self.t += 1


def _worker(rank, world, port, L, q, seed, beta, K, update, swap, outdir):
    import torch.distributed as dist

    import oracle
    from paper_1101_0876_gb300 import strips
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        row0, n = strips.partition(L, world)[rank]
        start = oracle.Lattice(L, q, 1, seed).spins()
        band = OracleBand(L, q, seed, row0, start[row0:row0 + n], update,
                          swap_rows=swap)
        sw = strips.StripSweeper(band, rank, world)
        recs = [sw.sweep(beta).numpy().copy() for _ in range(K)]
        own = torch.from_numpy(band.buf[1:n + 1].copy())
        parts = [None] * world
        dist.all_gather_object(parts, (row0, own.numpy()))
        if rank == 0:
            spins = np.zeros((L, L), np.uint8)
            for r0, rows in parts:
                spins[r0:r0 + rows.shape[0]] = rows
            np.save(os.path.join(outdir, "spins.npy"), spins)
            np.save(os.path.join(outdir, "recs.npy"), np.array(recs))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(world, L, q, update, swap, tmp_path):
    import torch.multiprocessing as mp
    seed, K = 7, 4
    beta = float(np.log1p(np.sqrt(q)))
    mp.start_processes(_worker, args=(world, _free_port(), L, q, seed, beta,
                                      K, update, swap, str(tmp_path)),
                       nprocs=world, join=True, start_method="spawn")
    import oracle
    ref = oracle.Lattice(L, q, 1, seed)
    want = ref.sweep(beta, K, update=update)
    got = np.load(tmp_path / "recs.npy").astype(np.uint64)
    spins = np.load(tmp_path / "spins.npy")
    return (np.array_equal(got, want), np.array_equal(spins, ref.spins()))


@pytest.mark.parametrize("world,L,q,update", [(2, 32, 9, 0), (3, 32, 24, 0),
                                              (2, 64, 9, 1)])
def test_strips_over_ranks_equal_whole_lattice(world, L, q, update, tmp_path):
    recs_ok, spins_ok = _run(world, L, q, update, False, tmp_path)
    assert recs_ok and spins_ok


def test_wrong_exchange_rows_are_caught(tmp_path):
    recs_ok, spins_ok = _run(2, 32, 9, 0, True, tmp_path)
    assert not (recs_ok and spins_ok)


def test_partition():
    from paper_1101_0876_gb300 import strips
    for L in (32, 64, 96, 32768):
        for world in (1, 2, 3, 5, 8, 16):
            parts = strips.partition(L, world)
            assert len(parts) == world
            assert parts[0][0] == 0
            assert sum(n for _, n in parts) == L
            for (r0, n), (r1, _) in zip(parts, parts[1:] + [(L, 0)]):
                assert n >= 2 and n % 2 == 0 and r0 % 2 == 0 and r0 + n == r1
            sizes = [n for _, n in parts]
            assert max(sizes) - min(sizes) <= 2
    assert strips.neighbours(0, 4) == (3, 1)
    assert strips.neighbours(3, 4) == (2, 0)
    with pytest.raises(ValueError):
        strips.partition(32, 17)
