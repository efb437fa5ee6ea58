"""Latitude-band sharding of one sphere mesh: one band of contiguous latitude
rows per rank (or several bands in one process), with one exchange of
boundary rows between neighbouring bands before every Runge-Kutta stage.

The paper (Sec. 5.1) names the Rusanov-flux phase as the only one that
exchanges data between neighbouring elements (an element needs its four
neighbours' traces, Eq. rusanov).  Longitude stays whole inside a band, so
the periodic lambda neighbours are local; the rows just south and north of a
band belong to the neighbouring bands and arrive as ghost rows.  What crosses
between bands before a stage is the stage's input on the boundary row: u^n and
the stage's increment (the library's stages read base + increment), so every
band computes exactly the bits the whole mesh would.

This module is argument marshalling and message passing only: the stages run
in the library (dgswe.Solver.band), and any object with the same methods
(halo_len, pack, unpack, stage) can stand in for a band.

Transports: DistExchange (torch.distributed point-to-point messages, one band
per rank; NCCL with device buffers or gloo through host buffers) and
LocalExchange (every band in this process, device-to-device copies on one
stream).
"""
from __future__ import annotations

import numpy as np

SOUTH, NORTH = 0, 1


def band_rows(nlat: int, nbands: int, k: int):
    """Rows [j_begin, j_end) of band k of nbands: contiguous, sizes differing
    by at most one row."""
    if not 0 <= k < nbands or nbands > nlat:
        raise ValueError(f"band {k} of {nbands} on {nlat} rows")
    return k * nlat // nbands, (k + 1) * nlat // nbands


def stages_per_step(rk_order: int) -> int:
    """Stages of the RK schemes of Table "Butcher" (orders 1-4)."""
    if rk_order not in (1, 2, 3, 4):
        raise ValueError("RK order must be 1..4")
    return rk_order


def sequential_sum(values, start: float = 0.0) -> float:
    """start + v0 + v1 + ... added one at a time, left to right, in FP64 (the
    order the library uses for its reference depth; numpy's sum is pairwise,
    its cumulative sum is sequential)."""
    v = np.concatenate([[float(start)], np.asarray(values, dtype=np.float64).ravel()])
    return float(np.cumsum(v)[-1])


def two_sum_merge(pairs):
    """Merge compensated (sum, err) pairs in the given order: the sums with an
    error-free two-sum, the errors added (the merge of the library's own
    fixed-order mass reduction)."""
    s, c = 0.0, 0.0
    for a, b in pairs:
        t = s + a
        bp = t - s
        c = c + ((s - (t - bp)) + (a - bp))
        c = c + b
        s = t
    return s, c


def bind_stream(band, stream):
    """Make the band's library calls run on the torch stream `stream` (an
    explicit, non-default stream: the library reads stream 0 as "its own
    stream", which the exchange's copies would not be ordered with)."""
    from . import dgswe

    if stream.cuda_stream == 0:
        raise ValueError("use a non-default torch.cuda.Stream for the bands")
    band.set_option(dgswe.OPT_STREAM, stream.cuda_stream)


class LocalExchange:
    """Every band in this process, in band order (south to north), on one
    device; messages are device tensors copied in place.  Every band is bound
    to `stream`, so the packs, unpacks and stages of all bands run in one
    order."""

    def __init__(self, bands, torch, dtype, stream):
        self.bands = bands
        for b in bands:
            bind_stream(b, stream)
        n = bands[0].halo_len
        with torch.cuda.stream(stream):
            self.out = [[torch.empty(n, dtype=dtype, device="cuda") for _ in range(2)] for _ in bands]

    def exchange(self):
        nb = len(self.bands)
        for k, b in enumerate(self.bands):
            if k > 0:
                b.pack(SOUTH, self.out[k][SOUTH])
            if k < nb - 1:
                b.pack(NORTH, self.out[k][NORTH])
        for k, b in enumerate(self.bands):
            if k > 0:
                b.unpack(SOUTH, self.out[k - 1][NORTH])
            if k < nb - 1:
                b.unpack(NORTH, self.out[k + 1][SOUTH])


class DistExchange:
    """One band per rank, rank order = band order (rank 0 the southernmost).
    Each exchange sends the band's boundary rows to the ranks below and above
    and receives theirs, with torch.distributed point-to-point messages.  The
    band's buffers live on `device`; `wire` is where the messages travel from
    ("cuda" for NCCL, "cpu" for gloo; host copies are made when they differ).
    A GPU band is bound to `stream` and the exchange's copies and messages
    are issued on it (NCCL orders its work after the current stream)."""

    def __init__(self, band, dist, rank, world, torch, dtype, device="cuda", wire="cuda", stream=None):
        self.band, self.dist, self.rank, self.world, self.torch = band, dist, rank, world, torch
        self.stream = stream
        if device != "cpu":
            if stream is None:
                raise ValueError("a GPU band needs an explicit stream")
            bind_stream(band, stream)
        n = band.halo_len
        self.dev = [torch.empty(n, dtype=dtype, device=device) for _ in range(4)]   # out S, out N, in S, in N
        self.wire = [t if wire == device else torch.empty(n, dtype=dtype, device=wire) for t in self.dev]
        self.has = (rank > 0, rank < world - 1)

    def exchange(self):
        if self.stream is None:
            self._exchange()
        else:
            with self.torch.cuda.stream(self.stream):
                self._exchange()

    def _exchange(self):
        b, d, w = self.band, self.dev, self.wire
        for side in (SOUTH, NORTH):
            if self.has[side]:
                b.pack(side, d[side])
                if w[side] is not d[side]:
                    w[side].copy_(d[side])
        ops = []
        for side, peer in ((SOUTH, self.rank - 1), (NORTH, self.rank + 1)):
            if self.has[side]:
                ops.append(self.dist.isend(w[side], peer))
                ops.append(self.dist.irecv(w[2 + side], peer))
        for op in ops:
            op.wait()
        for side in (SOUTH, NORTH):
            if self.has[side]:
                if w[2 + side] is not d[2 + side]:
                    d[2 + side].copy_(w[2 + side])
                b.unpack(side, d[2 + side])


def advance(bands, exchange, nsteps: int, dt: float, rk_order: int = 3):
    """nsteps RK steps of every band in `bands` (the bands this process owns):
    before each stage the boundary rows are exchanged, then every band runs
    the stage."""
    ns = stages_per_step(rk_order)
    for _ in range(nsteps):
        for _ in range(ns):
            exchange.exchange()
            for b in bands:
                b.stage(dt)


def global_min(dist, value: float, torch) -> float:
    """Minimum over ranks."""
    if dist is None:
        return float(value)
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    return float(t.item())


def global_dt(dist, terms, cfl: float, degree: int, torch) -> float:
    """The whole mesh's CFL step cfl * H / (max(p, 1) c) from every rank's
    terms (H, c) (dg_band_cfl_terms): H = the smallest, c = the largest over
    the bands, so the step equals the one the whole-mesh solver computes.
    terms: this rank's (H, c), or a list of the (H, c) of the bands in this
    process when dist is None."""
    if dist is None:
        pairs = terms if isinstance(terms, list) else [terms]
        H, c = min(h for h, _ in pairs), max(v for _, v in pairs)
    else:
        H = global_min(dist, terms[0], torch)
        c = -global_min(dist, -terms[1], torch)
    return cfl * H / (max(degree, 1) * c)


def global_mass(dist, pair, radius: float, torch) -> float:
    """Whole-mesh mass from every rank's compensated pair: gathered, merged in
    rank order, scaled by R^2 (one all-gather of two doubles per rank)."""
    if dist is None:
        pairs = [pair]
    else:
        t = torch.tensor(list(pair), dtype=torch.float64)
        out = [torch.empty(2, dtype=torch.float64) for _ in range(dist.get_world_size())]
        dist.all_gather(out, t)
        pairs = [(float(x[0]), float(x[1])) for x in out]
    s, c = two_sum_merge(pairs)
    return radius * radius * (s + c)


def reference_depth(dist, h_mode0, rank: int, world: int, torch) -> float:
    """The whole mesh's reference depth 0.5 * sum_e h_e / nel, summed in
    element order across the bands (rank r continues rank r - 1's running
    sum), so every band stores h relative to exactly the value the whole-mesh
    solver would use.  h_mode0: this band's mode-0 h coefficients in element
    order."""
    h_mode0 = np.asarray(h_mode0, dtype=np.float64).ravel()
    if dist is None or world == 1:
        return 0.5 * sequential_sum(h_mode0) / h_mode0.size
    run = torch.zeros(2, dtype=torch.float64)            # running sum, element count
    if rank > 0:
        dist.recv(run, rank - 1)
    s = sequential_sum(h_mode0, float(run[0]))
    run = torch.tensor([s, float(run[1]) + h_mode0.size], dtype=torch.float64)
    if rank < world - 1:
        dist.send(run, rank + 1)
    dist.broadcast(run, world - 1)
    return 0.5 * float(run[0]) / float(run[1])
