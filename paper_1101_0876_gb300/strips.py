"""Row-strip decomposition of one lattice over processes, one strip per rank
(the multi-GPU extension Sec. 7 proposes, on the colour-packed planes of
Sec. 3.3).

This module holds the host side of it: the split of the L rows into strips,
the exchange of halo rows between neighbouring ranks before each colour
pass, and the sum of the strips' partial records after each sweep.  The
colour pass itself belongs to the strip object handed in: on a GPU a
`StripBand` around the CUDA strip handle (potts_strip_*), whose passes run
in the library's kernels.

A strip object provides
    rows(colour) -> (first own row, last own row, halo above, halo below),
        four 1-D uint8 tensors aliasing that plane's rows;
    pass_(beta, colour, record) -> None: the colour pass over its own rows,
        adding its partial counts {B, hist} to `record` (int64 tensor of
        1 + q on the strip's device);
    new_record() -> a zeroed record tensor.
Before the pass of colour c every strip needs the halo rows of plane 1 - c
as the neighbours hold them after their pass of colour 1 - c; the black
pass's partial records summed over all strips are the sweep's record.
"""
from __future__ import annotations


def partition(L: int, world: int):
    """(row0, nrows) of each strip: even row counts as equal as possible,
    strip 0 first (the split potts_create_sharded uses)."""
    L, world = int(L), int(world)
    if L % 2 or world < 1 or world > L // 2:
        raise ValueError(f"cannot split {L} rows into {world} even strips")
    pairs = L // 2
    base, extra = divmod(pairs, world)
    out, row0 = [], 0
    for s in range(world):
        n = 2 * (base + (1 if s < extra else 0))
        out.append((row0, n))
        row0 += n
    return out


def neighbours(rank: int, world: int):
    """Ranks holding the strips just above and just below (periodic)."""
    return (rank - 1) % world, (rank + 1) % world


# Tags of the two directions (gloo matches on them; NCCL on posting order,
# which is the same on every rank).
TAG_UP, TAG_DOWN = 17, 18


class StripSweeper:
    """Sweeps one strip of a lattice whose other strips live on the other
    ranks of `group` (torch.distributed), rank r holding strip r."""

    def __init__(self, strip, rank: int, world: int, group=None):
        self.strip, self.rank, self.world, self.group = strip, rank, world, group
        self.prev, self.next = neighbours(rank, world)

    def exchange(self, plane: int) -> None:
        """Halo rows of `plane` from the neighbours' own rows."""
        first, last, above, below = self.strip.rows(plane)
        if self.world == 1:          # the lattice is one periodic strip
            above.copy_(last)
            below.copy_(first)
            return
        import torch.distributed as dist
        ops = [dist.P2POp(dist.isend, first, self.prev, self.group, TAG_UP),
               dist.P2POp(dist.irecv, below, self.next, self.group, TAG_UP),
               dist.P2POp(dist.isend, last, self.next, self.group, TAG_DOWN),
               dist.P2POp(dist.irecv, above, self.prev, self.group, TAG_DOWN)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()

    def sweep(self, beta: float, record=None, reduce: bool = True):
        """One sweep: black halo rows, white pass, white halo rows, black
        pass; then the record summed over the ranks (if `reduce`).  Returns
        the record tensor (int64, 1 + q)."""
        rec = self.strip.new_record() if record is None else record
        self.exchange(1)
        self.strip.pass_(beta, 0, rec)
        self.exchange(0)
        self.strip.pass_(beta, 1, rec)
        if reduce and self.world > 1:
            import torch.distributed as dist
            dist.all_reduce(rec, group=self.group)
        return rec


class _CudaRows:
    """A device byte range as a torch tensor (no copy)."""

    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {
            "shape": (int(nbytes),), "typestr": "|u1",
            "data": (int(ptr), False), "version": 2}


class StripBand:
    """A CUDA row strip (paper_1101_0876_gb300.potts.Strip) with the strip
    interface of this module, its passes on torch's current stream of
    `device` so that they order with the halo exchange."""

    def __init__(self, L: int, q: int, start: int, seed: int, row0: int,
                 nrows: int, device=None, layout: int = 0):
        import torch

        from . import potts
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device()
                                   if device is None else device)
        self.q = int(q)
        with torch.cuda.device(self.device):
            self.h = potts.Strip(L, q, start, seed, row0, nrows, layout)
            self.h.set_stream(torch.cuda.current_stream().cuda_stream)
        self._rows = {}
        for c in (0, 1):
            ptrs, nbytes = self.h.rows(c)
            self._rows[c] = tuple(
                torch.as_tensor(_CudaRows(p, nbytes), device=self.device)
                for p in ptrs)

    def rows(self, colour: int):
        return self._rows[colour]

    def new_record(self):
        return self.torch.zeros(1 + self.q, dtype=self.torch.int64,
                                device=self.device)

    def pass_(self, beta: float, colour: int, record) -> None:
        self.h.pass_(beta, colour, record.data_ptr())

    def close(self) -> None:
        self.h.close()
