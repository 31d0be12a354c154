"""Slab decomposition of one 2D FS grid over R ranks (include/fs_slab.h).

Algorithm 1's step splits into a row pass (x transforms and the pointwise
stage, local to rows) and a column pass (y transforms and the per-mode solve
of Eqs. (A-C_discrete_fft_c) / (A-C_discrete_fft_eta), local to kx columns).
Rank r holds rows [r rows, (r + 1) rows) for the first and packed kx columns
[r cols, (r + 1) cols) for the second (rows = ny / R, cols = nx / (2R)); a
transpose of the spectra joins them, one forward and one back per step.

This module holds the host side of that transpose, the part that is the same
on every transport:
  * `SlabLayout` -- who owns which rows and columns, block shapes;
  * `exchange_forward` / `exchange_back` -- the blocks of one transpose as
    point-to-point messages of torch.distributed (NCCL between GPUs, gloo
    between CPU processes), one batch per direction;
  * `exchange_local_forward` / `exchange_local_back` -- the same block moves
    between several ranks held by one process (device copies on one stream,
    no rank ever waits on another);
and the drivers over the library's slab calls: `Slab` (one rank), `LocalSlabs`
(R ranks on one GPU) and `DistributedSlab` (one rank per process).

Exchanged arrays are real tensors with a trailing (re, im) axis:
  send    [R][slots_fwd][rows][cols][2]   row-pass output by destination
  colspec [slots_fwd][ny][cols][2]        the column pass's spectra
  recv    [R][slots_back][rows][cols][2]  column-pass results by source
"""
from __future__ import annotations

from dataclasses import dataclass

from . import fs as F


@dataclass(frozen=True)
class SlabLayout:
    nx: int
    ny: int
    p: int
    nranks: int
    rank: int

    def __post_init__(self):
        R = self.nranks
        if R < 1 or R & (R - 1) or not 0 <= self.rank < R:
            raise ValueError("nranks must be a power of two and 0 <= rank < nranks")
        if self.ny % R or self.nx % (2 * R) or self.ny // R < 8 or self.nx // R < 8:
            raise ValueError("ny / nranks and nx / nranks must be whole and >= 8")

    @property
    def rows(self) -> int:
        return self.ny // self.nranks

    @property
    def cols(self) -> int:
        return self.nx // (2 * self.nranks)

    @property
    def slots_fwd(self) -> int:  # c, g_1 .. g_p, df/dc
        return self.p + 2

    @property
    def slots_back(self) -> int:  # c, eta_1 .. eta_p
        return self.p + 1

    def row_range(self, q: int | None = None) -> slice:
        """Rows y of rank q (default: this rank) in the row pass."""
        q = self.rank if q is None else q
        return slice(q * self.rows, (q + 1) * self.rows)

    def col_range(self, q: int | None = None) -> slice:
        """Packed kx columns of rank q in the column pass (column 0 holds
        kx = 0 and kx = nx/2 as real and imaginary parts)."""
        q = self.rank if q is None else q
        return slice(q * self.cols, (q + 1) * self.cols)

    def peers(self):
        return [q for q in range(self.nranks) if q != self.rank]

    def exchange_bytes(self, elem_bytes: int) -> tuple[int, int]:
        """Bytes this rank sends in the forward and in the back transpose."""
        blk = self.rows * self.cols * elem_bytes
        return (self.nranks - 1) * self.slots_fwd * blk, (self.nranks - 1) * self.slots_back * blk


def _run(dist, ops):
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


def exchange_forward(lay: SlabLayout, send, colspec, dist, group=None):
    """After the row pass: send[q][s] goes to rank q, which receives it at
    colspec[s][rank rows ..].  Every message is one contiguous block."""
    ops = []
    for q in lay.peers():
        for s in range(lay.slots_fwd):
            ops.append(dist.P2POp(dist.isend, send[q, s], q, group))
            ops.append(dist.P2POp(dist.irecv, colspec[s, lay.row_range(q)], q, group))
    _run(dist, ops)


def exchange_back(lay: SlabLayout, colspec, recv, dist, group=None):
    """After the column pass: colspec[s][q rows ..] goes back to rank q, which
    receives it at recv[rank][s]."""
    ops = []
    for q in lay.peers():
        for s in range(lay.slots_back):
            ops.append(dist.P2POp(dist.isend, colspec[s, lay.row_range(q)], q, group))
            ops.append(dist.P2POp(dist.irecv, recv[q, s], q, group))
    _run(dist, ops)


def exchange_local_forward(lays, sends, colspecs):
    """exchange_forward for ranks held by one process (copies)."""
    for r, lay in enumerate(lays):
        for q in lay.peers():
            for s in range(lay.slots_fwd):
                colspecs[q][s, lay.row_range()].copy_(sends[r][q, s])


def exchange_local_back(lays, colspecs, recvs):
    for r, lay in enumerate(lays):
        for q in lay.peers():
            for s in range(lay.slots_back):
                recvs[q][r, s].copy_(colspecs[r][s, lay.row_range(q)])


class _DeviceBuffer:
    """A view of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2}


class Slab:
    """One rank's share of a 2D FS grid on the current CUDA device and stream."""

    def __init__(self, prob, precision: str, rank: int, nranks: int, stream=None):
        import torch
        if len(prob.n) != 2:
            raise ValueError("slabs are 2D")
        self.layout = SlabLayout(prob.n[0], prob.n[1], prob.p, nranks, rank)
        self.prob = prob
        self.nf = prob.p + 1
        self.dtype = torch.float64 if precision == "f64" else torch.float32
        self.h = F.fs_slab_create(F.make_params(prob, precision), rank, nranks, stream)
        info = F.fs_slab_info_get(self.h)
        lay, ts = self.layout, "<f8" if precision == "f64" else "<f4"
        assert (info.rows, info.cols) == (lay.rows, lay.cols)

        def view(ptr, shape):
            return torch.as_tensor(_DeviceBuffer(ptr, shape, ts), device="cuda")
        self.send = view(info.send, (nranks, lay.slots_fwd, lay.rows, lay.cols, 2))
        self.recv = view(info.recv, (nranks, lay.slots_back, lay.rows, lay.cols, 2))
        self.colspec = view(info.colspec, (lay.slots_fwd, lay.ny, lay.cols, 2))

    def set_fields(self, rows) -> float:
        """rows: (nf, rows, nx) tensor of this rank's rows; returns its FP64 c sum."""
        return F.fs_slab_set_fields(self.h, [rows[f] for f in range(self.nf)])

    def set_c_sum(self, total: float):
        F.fs_slab_set_c_sum(self.h, total)

    def row_pass(self):
        F.fs_slab_row_pass(self.h)

    def col_pass(self):
        F.fs_slab_col_pass(self.h)

    def get_fields(self):
        import torch
        out = torch.empty((self.nf, self.layout.rows, self.layout.nx), dtype=self.dtype, device="cuda")
        F.fs_slab_get_fields(self.h, [out[f] for f in range(self.nf)])
        return out

    def sync(self):
        F.fs_slab_sync(self.h)

    def close(self):
        # the views alias the slab's device memory: drop them before it is freed
        self.send = self.recv = self.colspec = None
        if self.h is not None and self.h.value:
            F.fs_slab_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LocalSlabs:
    """R slabs of one grid held by one process on one GPU: the decomposed
    step with the transposes as device copies.  Every launch is independent
    (no kernel waits for another rank), so this runs on one GPU safely."""

    def __init__(self, prob, precision: str, nranks: int):
        self.slabs = [Slab(prob, precision, r, nranks) for r in range(nranks)]
        self.lays = [s.layout for s in self.slabs]

    def set_fields(self, fields):
        """fields: (nf, ny, nx) tensor of the whole grid."""
        total = sum(s.set_fields(fields[:, s.layout.row_range()].contiguous()) for s in self.slabs)
        for s in self.slabs:
            s.set_c_sum(total)

    def step(self, n: int = 1):
        for _ in range(n):
            for s in self.slabs:
                s.row_pass()
            exchange_local_forward(self.lays, [s.send for s in self.slabs], [s.colspec for s in self.slabs])
            for s in self.slabs:
                s.col_pass()
            exchange_local_back(self.lays, [s.colspec for s in self.slabs], [s.recv for s in self.slabs])

    def get_fields(self):
        import torch
        return torch.cat([s.get_fields() for s in self.slabs], dim=1)

    def sync(self):
        for s in self.slabs:
            s.sync()

    def close(self):
        for s in self.slabs:
            s.close()


class DistributedSlab:
    """This process's rank of a grid decomposed over a torch.distributed
    process group (one GPU per rank; NCCL point-to-point transposes)."""

    def __init__(self, prob, precision: str, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.slab = Slab(prob, precision, dist.get_rank(group), dist.get_world_size(group))
        self.layout = self.slab.layout

    def set_fields(self, rows):
        import torch
        local = self.slab.set_fields(rows)
        t = torch.tensor([local], dtype=torch.float64, device="cuda")
        self.dist.all_reduce(t, group=self.group)
        self.slab.set_c_sum(float(t.item()))

    def step(self, n: int = 1):
        s = self.slab
        for _ in range(n):
            s.row_pass()
            exchange_forward(self.layout, s.send, s.colspec, self.dist, self.group)
            s.col_pass()
            exchange_back(self.layout, s.colspec, s.recv, self.dist, self.group)

    def get_fields(self):
        return self.slab.get_fields()

    def sync(self):
        self.slab.sync()

    def close(self):
        self.slab.close()
