"""Latitude-band sharding on the CPU: two (and three) gloo ranks, each owning
one latitude band of a mesh, exchange their boundary rows through
paper_2303_11767_gb300.bands before every stage of a CPU stand-in of the
stage, and together reproduce the single-rank run bit for bit; the
reference depth and the mass merge of the module are checked too.

The stand-in is the degree-0 case of the method (a first-order finite-volume
Rusanov scheme for the shallow water equations on the sphere, FP64) held in
the same form as the library's bands: ghost rows around the own rows, the
stage input = u^n + increment, the increment form of SSP-RK3, and halo
messages [u^n row | increment row].  It tests the decomposition and the
exchange schedule, not the kernels (the GPU tests do that).
"""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2303_11767_gb300 import bands

R, G, OMEGA = 6.37122e6, 9.80616, 7.292e-5
NLON, NLAT, NSTEPS, DT = 12, 7, 6, 400.0


class StandInBand:
    """Rows [jb, je) of an NLON x NLAT mesh, p = 0, FP64, SSP-RK3 in
    increment form: stage 1 inc0 = dt k; stage 2 inc1 = (inc0 + dt k)/4;
    stage 3 u^{n+1} = u^n + 2/3 (inc1 + dt k)."""

    PLAN = [(-1, 0, 0.0, 1.0, False), (0, 1, 0.25, 0.25, False), (1, -1, 2.0 / 3.0, 2.0 / 3.0, True)]

    def __init__(self, jb, je):
        self.jb, self.je, self.nb = jb, je, je - jb
        shape = (self.nb + 2, NLON, 3)           # ghost south, own rows, ghost north
        self.base = [np.zeros(shape), np.zeros(shape)]
        self.inc = [np.zeros(shape), np.zeros(shape)]
        self.cur, self.stage_i = 0, 0
        self.halo_len = 2 * NLON * 3

    def set_state(self, u):
        self.base[self.cur][1:-1] = u

    def state(self):
        return self.base[self.cur][1:-1].copy()

    def _inputs(self):
        ii = self.PLAN[self.stage_i][0]
        return self.base[self.cur], (self.inc[ii] if ii >= 0 else None)

    def pack(self, side, t):
        b, inc = self._inputs()
        row = 1 if side == bands.SOUTH else self.nb
        n = NLON * 3
        out = t.numpy()
        out[:n] = b[row].ravel()
        out[n:] = inc[row].ravel() if inc is not None else 0.0

    def unpack(self, side, t):
        b, inc = self._inputs()
        row = 0 if side == bands.SOUTH else self.nb + 1
        n = NLON * 3
        src = t.numpy()
        b[row] = src[:n].reshape(NLON, 3)
        if inc is not None:
            inc[row] = src[n:].reshape(NLON, 3)

    def _rhs(self, u):
        """First-order finite volume on the own rows: cell values, exact
        cos(theta)-weighted cell areas, Rusanov fluxes at edge midpoints, zero
        flux through a pole edge, midpoint sources."""
        dl, dth = 2 * math.pi / NLON, math.pi / NLAT
        k = np.zeros((self.nb, NLON, 3))

        def F(s):
            h, hu, hv = s[..., 0], s[..., 1], s[..., 2]
            return np.stack([hu, hu * hu / h + 0.5 * G * h * h, hu * hv / h], -1) / R

        def Gf(s, th):
            h, hu, hv = s[..., 0], s[..., 1], s[..., 2]
            return math.cos(th) * np.stack([hv, hu * hv / h, hv * hv / h + 0.5 * G * h * h], -1) / R

        def spd(s, c):
            return np.abs(s[..., c] / s[..., 0]) + np.sqrt(G * s[..., 0])

        for r in range(self.nb):
            j = self.jb + r
            tb = -math.pi / 2 + j * dth
            tc, tt = tb + 0.5 * dth, tb + dth
            c = u[r + 1]
            E, W = np.roll(c, -1, axis=0), np.roll(c, 1, axis=0)
            fe = 0.5 * (F(c) + F(E)) - 0.5 * (np.maximum(spd(c, 1), spd(E, 1)) / R)[:, None] * (E - c)
            fw = 0.5 * (F(W) + F(c)) - 0.5 * (np.maximum(spd(W, 1), spd(c, 1)) / R)[:, None] * (c - W)
            gn = np.zeros_like(c)
            gs = np.zeros_like(c)
            if j < NLAT - 1:
                N = u[r + 2]
                gn = 0.5 * (Gf(c, tt) + Gf(N, tt)) - 0.5 * math.cos(tt) * (
                    np.maximum(spd(c, 2), spd(N, 2)) / R)[:, None] * (N - c)
            if j > 0:
                S = u[r]
                gs = 0.5 * (Gf(S, tb) + Gf(c, tb)) - 0.5 * math.cos(tb) * (
                    np.maximum(spd(S, 2), spd(c, 2)) / R)[:, None] * (c - S)
            h, hu, hv = c[:, 0], c[:, 1], c[:, 2]
            cor = 2 * OMEGA * math.sin(tc) * math.cos(tc) + (hu / h) * math.sin(tc) / R
            src = np.stack([0 * h, cor * hv, -G * h * h * math.sin(tc) / (2 * R) - cor * hu], -1)
            area = dl * (math.sin(tt) - math.sin(tb))
            k[r] = (dl * dth * src - dth * (fe - fw) - dl * (gn - gs)) / area
        return k

    def stage(self, dt):
        ii, io, ci, cc, fin = self.PLAN[self.stage_i]
        b = self.base[self.cur]
        u = b + self.inc[ii] if ii >= 0 else b.copy()
        k = self._rhs(u)
        prev = self.inc[ii][1:-1] if ii >= 0 else 0.0
        if fin:
            self.base[self.cur ^ 1][1:-1] = b[1:-1] + (ci * prev + cc * dt * k)
            self.cur ^= 1
            self.stage_i = 0
        else:
            self.inc[io][1:-1] = ci * prev + cc * dt * k
            self.stage_i += 1


class NoExchange:
    def exchange(self):
        pass


def initial_state():
    rng = np.random.default_rng(7)
    u = np.zeros((NLAT, NLON, 3))
    u[..., 0] = 5960.0 + 50.0 * rng.normal(size=(NLAT, NLON))
    u[..., 1] = u[..., 0] * 10.0 * rng.normal(size=(NLAT, NLON))
    u[..., 2] = u[..., 0] * 10.0 * rng.normal(size=(NLAT, NLON))
    return u


def single_rank():
    b = StandInBand(0, NLAT)
    b.set_state(initial_state())
    bands.advance([b], NoExchange(), NSTEPS, DT)
    return b.state()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        jb, je = bands.band_rows(NLAT, world, rank)
        b = StandInBand(jb, je)
        u0 = initial_state()
        b.set_state(u0[jb:je])
        ex = bands.DistExchange(b, dist, rank, world, torch, torch.float64, device="cpu", wire="cpu")
        bands.advance([b], ex, NSTEPS, DT)
        href = bands.reference_depth(dist, u0[jb:je, :, 0], rank, world, torch)
        pair = (float(np.sum(u0[jb:je, :, 0])), 1e-9 * (rank + 1))
        mass = bands.global_mass(dist, pair, 1.0, torch)
        dmin = bands.global_min(dist, 100.0 + rank, torch)
        dglob = bands.global_dt(dist, (10.0 - rank, 3.0 + rank), 0.5, 2, torch)
        np.save(os.path.join(out_dir, f"band{rank}.npy"), b.state())
        np.save(os.path.join(out_dir, f"scalars{rank}.npy"), np.array([jb, je, href, mass, dmin, dglob]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_band_split_matches_single_rank_bitwise(world, tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    want = single_rank()
    got = np.concatenate([np.load(tmp_path / f"band{r}.npy") for r in range(world)], axis=0)
    assert got.shape == want.shape
    assert np.array_equal(got, want)            # bit for bit
    assert not np.array_equal(want, initial_state())
    # the reference depth is the whole mesh's, summed in element order
    u0 = initial_state()
    href_single = 0.5 * float(np.cumsum(u0[..., 0].ravel())[-1]) / (NLAT * NLON)
    pairs = []
    for r in range(world):
        jb, je, href, mass, dmin, dglob = np.load(tmp_path / f"scalars{r}.npy")
        assert href == href_single
        assert dmin == 100.0
        # smallest H and largest c of all ranks: 0.5 (10 - (world - 1)) / (2 (3 + world - 1))
        assert dglob == 0.5 * (10.0 - (world - 1)) / (2 * (3.0 + world - 1))
        pairs.append((float(np.sum(u0[int(jb):int(je), :, 0])), 1e-9 * (r + 1)))
    # mass: the pairs merged in rank order with the error-free two-sum
    want_mass = math.fsum([a for a, _ in pairs]) + sum(b for _, b in pairs)
    assert abs(mass - want_mass) <= 1e-15 * abs(want_mass)


def test_band_rows_cover_the_mesh():
    for nlat in (2, 7, 90, 720):
        for nb in range(1, min(nlat, 9) + 1):
            rows = [bands.band_rows(nlat, nb, k) for k in range(nb)]
            assert rows[0][0] == 0 and rows[-1][1] == nlat
            assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
            sizes = [e - b for b, e in rows]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        bands.band_rows(3, 4, 0)


def test_sequential_sum_and_two_sum_merge():
    rng = np.random.default_rng(3)
    v = rng.normal(size=1000) * 1e3 + 5000.0
    s = 0.0
    for x in v:
        s += float(x)
    assert bands.sequential_sum(v) == s
    assert bands.sequential_sum(v[500:], bands.sequential_sum(v[:500])) == s
    # the merge is exact for sums the two-sum can represent
    pairs = [(1e16, 0.0), (1.0, 0.0), (-1e16, 0.0)]
    S, C = bands.two_sum_merge(pairs)
    assert S + C == 1.0
