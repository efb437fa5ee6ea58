"""Latitude-band sharding through the C ABI on one GPU: the mesh split into
2-4 bands (dg_create_band), their boundary rows exchanged before every stage
(paper_2303_11767_gb300.bands.LocalExchange: device copies on one stream),
every band advanced by dg_band_stage.  The bands together must equal the
whole-mesh solver bit for bit (same kernels, same reference depth) and the
FP64 oracle within the state tolerances (1e-12 FP64, 1e-5 FP32)."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2303_11767_gb300 import bands, dgswe, synth

pytestmark = pytest.mark.gpu

R, G, OMEGA = synth.EARTH_RADIUS, 9.80616, 7.292e-5
TOL = {"fp64": 1e-12, "fp32": 1e-5}
NTHREADS = os.cpu_count() or 1


def _run_bands(u0, nlon, nlat, p, prec, nb, nsteps, dt, rk, torch, wb=0):
    stream = torch.cuda.Stream()
    rows = [bands.band_rows(nlat, nb, k) for k in range(nb)]
    bs = [dgswe.Solver.band(nlon, nlat, jb, je, p, R, G, OMEGA, precision=prec, rk_order=rk) for jb, je in rows]
    ex = bands.LocalExchange(bs, torch, torch.float64 if prec == "fp64" else torch.float32, stream)
    href = bands.reference_depth(None, u0[:, :, 0, 0], 0, 1, torch)
    for b, (jb, je) in zip(bs, rows):
        b.set_option(dgswe.OPT_WELL_BALANCED, wb)
        if prec != "fp64" or wb:
            b.set_reference_depth(href)
        b.set_state(u0[jb:je])
    bands.advance(bs, ex, nsteps, dt, rk)
    out = np.concatenate([b.get_state() for b in bs], axis=0)
    mass = bands.global_mass(None, bands.two_sum_merge([b.mass_pair() for b in bs]), R, torch)
    dt_glob = bands.global_dt(None, [b.cfl_terms() for b in bs], 0.1, p, torch)
    for b in bs:
        assert b.get_time() == pytest.approx(nsteps * dt, rel=1e-15)
        b.close()
    return out, mass, dt_glob


def _whole(u0, nlon, nlat, p, prec, nsteps, dt, rk, torch, wb=0):
    with dgswe.Solver(nlon, nlat, p, R, G, OMEGA, precision=prec, rk_order=rk) as s:
        s.set_option(dgswe.OPT_WELL_BALANCED, wb)
        s.set_state(u0)
        s.step(nsteps, dt)
        return s.get_state(), s.total_mass(), s.max_dt(0.1)   # the step of the final state, as for the bands


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nlon,nlat,p,nb", [(20, 10, 1, 2), (44, 14, 3, 3), (15, 19, 4, 4), (35, 19, 2, 2)])
def test_bands_equal_whole_mesh_and_oracle(nlon, nlat, p, nb, prec):
    torch = pytest.importorskip("torch")
    o = O.Oracle.sphere(nlon, nlat, p, R, G, OMEGA)
    o.set_threads(NTHREADS)
    u0 = o.project_tensor(synth.SmoothField(17).fields_grid)
    dt = o.max_dt(u0, 0.1)
    nsteps = 12
    got, mass, dt_bands = _run_bands(u0, nlon, nlat, p, prec, nb, nsteps, dt, 3, torch)
    want, mass_whole, dt_whole = _whole(u0, nlon, nlat, p, prec, nsteps, dt, 3, torch)
    assert np.array_equal(got, want), np.abs(got - want).max()          # bit for bit
    assert dt_bands == dt_whole
    assert abs(mass / mass_whole - 1) < 1e-14
    ref = o.step(u0, nsteps, dt, 3)
    for f in range(3):
        d = got[..., f, :] - ref[..., f, :]
        assert np.linalg.norm(d) / np.linalg.norm(ref[..., f, :]) <= TOL[prec]
        assert np.abs(d).max() / np.abs(ref[..., f, :]).max() <= TOL[prec]


@pytest.mark.parametrize("rk", [1, 2, 4])
def test_bands_every_rk_order(rk):
    torch = pytest.importorskip("torch")
    nlon, nlat, p = 24, 12, 2
    o = O.Oracle.sphere(nlon, nlat, p, R, G, OMEGA)
    u0 = o.project_tensor(synth.SmoothField(19).fields_grid)
    dt = o.max_dt(u0, 0.05)
    for prec in ("fp64", "fp32"):
        got, _, _ = _run_bands(u0, nlon, nlat, p, prec, 3, 5, dt, rk, torch)
        want, _, _ = _whole(u0, nlon, nlat, p, prec, 5, dt, rk, torch)
        assert np.array_equal(got, want), (prec, rk)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_bands_well_balanced_equal_whole_mesh(prec):
    """The well-balanced option on bands: every band removes the rest-state
    tendency of the same reference depth (the whole mesh's, given to each band),
    so the bands still equal the whole mesh bit for bit."""
    torch = pytest.importorskip("torch")
    nlon, nlat, p = 24, 12, 2
    o = O.Oracle.sphere(nlon, nlat, p, R, G, OMEGA)
    u0 = o.project_tensor(synth.SmoothField(23).fields_grid)
    dt = o.max_dt(u0, 0.1)
    got, _, _ = _run_bands(u0, nlon, nlat, p, prec, 3, 6, dt, 3, torch, wb=1)
    want, _, _ = _whole(u0, nlon, nlat, p, prec, 6, dt, 3, torch, wb=1)
    assert np.array_equal(got, want), np.abs(got - want).max()


def test_band_refuses_what_needs_the_whole_mesh():
    torch = pytest.importorskip("torch")
    b = dgswe.Solver.band(20, 10, 3, 7, 1, R, G, OMEGA)
    u = np.zeros((4, 20, 3, 4))
    u[..., 0, 0] = 2 * 5000.0
    b.set_state(u)
    for call in (lambda: b.step(1, 1.0), lambda: b.rhs(u),
                 lambda: b.set_option(dgswe.OPT_PRECISION, dgswe.PREC["fp32_tc_bf16"]),
                 lambda: b.set_option(dgswe.OPT_ALPHA_MODE, 1)):
        with pytest.raises(dgswe.DGError) as e:
            call()
        assert e.value.status == dgswe.DG_EUNSUPPORTED
    with pytest.raises(ValueError):                  # the library's own stream is not ordered with torch's
        bands.LocalExchange([b], torch, torch.float64, torch.cuda.default_stream())
    # the pole side of a polar band has no ghost row
    s = dgswe.Solver.band(20, 10, 0, 5, 1, R, G, OMEGA)
    s.set_state(np.concatenate([u, u[:1]], axis=0))
    t = torch.zeros(s.halo_len, dtype=torch.float64, device="cuda")
    with pytest.raises(dgswe.DGError):
        s.unpack(bands.SOUTH, t)
    s.unpack(bands.NORTH, t)
    with pytest.raises(dgswe.DGError):
        dgswe.Solver.band(20, 10, 5, 5, 1)
    b.close()
    s.close()
