"""Parity of the CUDA path (through the C-ABI) with the FP64 CPU oracle.

Tolerances, per field:
* States (projection, time stepping): relative to the reference field,
  ||x - y||_2 / ||y||_2 and max|x - y| / max|y|, 1e-12 (FP64) / 1e-5 (FP32).
* Tendencies (dg_rhs): relative to the oracle's magnitude bound
  S = |M^-1| sum |terms| (pinned against a closed form and a brute force in
  the oracle's own tests).  FP64: 3e-14, twice the summation bound
  gamma_N = N u / (1 - N u) (u = 2^-53) with N ~ 3 n^2 + 5 n ~ 100 terms per
  tendency entry at degree 4, once for each of the two evaluations compared;
  the observed errors are ~1e-16 over a whole mesh and up to 1.1e-14 for
  single elements.  FP32: 1e-6, below that bound (1.2e-5) and ~20x above the
  observed ~5e-8.  The
  tendency of this mesh is a small difference of large terms (flux
  divergences of a nearly non-divergent flow, amplified by 1/cos(theta) in
  the polar rows), so any floating-point evaluation of it is only determined
  up to a few units of roundoff times S.  The plain relative error
  ||k - k_oracle||_2 / ||k_oracle||_2 of every tendency check is recorded
  and printed at the end of the run.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2303_11767_gb300 import dgswe, synth
from _records import record_tendency

pytestmark = pytest.mark.gpu

R, G, OMEGA = synth.EARTH_RADIUS, 9.80616, 7.292e-5
TOL = {"fp64": 1e-12, "fp32": 1e-5}
TEND_TOL = {"fp64": 3e-14, "fp32": 1e-6,
            # split FP16 operands: 8 u^2 of the pair plus the FP16-pair subnormal floor (tests/test_tc_gpu.py)
            "fp32_tc_fp16x3": 8 * 2.0 ** -24 + 4e-6}
NTHREADS = os.cpu_count() or 1


def oracle_sphere(nlon, nlat, p):
    o = O.Oracle.sphere(nlon, nlat, p, R, G, OMEGA)
    o.set_threads(NTHREADS)
    return o


_cache = {}


def case(nlon, nlat, p, seed):
    """Oracle and the oracle-projected seeded state (cached)."""
    key = (nlon, nlat, p, seed)
    if key not in _cache:
        o = oracle_sphere(nlon, nlat, p)
        _cache[key] = (o, o.project_tensor(synth.SmoothField(seed).fields_grid))
    return _cache[key]


def state_err(x, y):
    x = np.asarray(x).reshape(y.shape)
    out = []
    for f in range(3):
        d = x[..., f, :] - y[..., f, :]
        out.append((np.linalg.norm(d) / np.linalg.norm(y[..., f, :]), np.abs(d).max() / np.abs(y[..., f, :]).max()))
    return out


def tend_err(x, y, S, what=""):
    x = np.asarray(x).reshape(y.shape)
    if what:
        record_tendency(what, x, y, S)
    out = []
    for f in range(3):
        d = x[..., f, :] - y[..., f, :]
        out.append((np.linalg.norm(d) / np.linalg.norm(S[..., f, :]), np.abs(d).max() / S[..., f, :].max()))
    return out


def assert_within(errs, tol, what):
    for f, (l2, mx) in enumerate(errs):
        assert l2 <= tol and mx <= tol, f"{what}: field {f} l2={l2:.3e} max={mx:.3e} tol={tol:g}"


def solver(nlon, nlat, p, prec, **kw):
    return dgswe.Solver(nlon, nlat, p, R, G, OMEGA, precision=prec, **kw)


# -------------------------------------------------------------- tendencies --

# meshes spanning several tiles (a warp holds 32/(p+1) elements of a row, a
# block 8 rows) with ragged last tiles, and degenerate tiny meshes
SMALL = [(p, nlon, 19) for p, nlon in ((0, 67), (1, 35), (2, 23), (3, 19), (4, 15))] + \
        [(p, 4, 2) for p in range(5)] + [(2, 1, 3), (3, 2, 9)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p,nlon,nlat", SMALL)
def test_rhs_parity_small_meshes(p, nlon, nlat, prec):
    o, u = case(nlon, nlat, p, 11)
    with solver(nlon, nlat, p, prec) as s:
        k = s.rhs(u)
    what = f"rhs p={p} {nlon}x{nlat} {prec}"
    assert_within(tend_err(k, o.rhs(u), o.rhs_magnitude(u), what), TEND_TOL[prec], what)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nlon,nlat,p,seed", [(20, 10, 1, 1), (180, 90, 3, 2), (360, 180, 4, 3)])
def test_rhs_parity_configs(nlon, nlat, p, seed, prec):
    o, u = case(nlon, nlat, p, seed)
    with solver(nlon, nlat, p, prec) as s:
        k = s.rhs(u)
    what = f"rhs {nlon}x{nlat} p={p} {prec}"
    assert_within(tend_err(k, o.rhs(u), o.rhs_magnitude(u), what), TEND_TOL[prec], what)


# -------------------------------------------------------------- time steps --

def _oracle_run(nlon, nlat, p, seed, nsteps, order=3, cfl=0.1):
    key = ("run", nlon, nlat, p, seed, nsteps, order, cfl)
    if key not in _cache:
        o, u = case(nlon, nlat, p, seed)
        dt = o.max_dt(u, cfl)
        _cache[key] = (dt, o.total_mass(u), o.step(u, nsteps, dt, order))
    return _cache[key]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nlon,nlat,p,seed,nsteps", [(20, 10, 1, 1, 100), (180, 90, 3, 2, 1000)])
def test_step_parity_and_mass(nlon, nlat, p, seed, nsteps, prec):
    o, u = case(nlon, nlat, p, seed)
    dt, m0, want = _oracle_run(nlon, nlat, p, seed, nsteps)
    with solver(nlon, nlat, p, prec) as s:
        s.set_state(u)
        gm0 = s.total_mass()
        s.step(nsteps, dt)
        got = s.get_state()
        gm1 = s.total_mass()
        assert s.get_time() == pytest.approx(nsteps * dt, rel=1e-15)
    assert_within(state_err(got, want), TOL[prec], f"{nsteps} steps {nlon}x{nlat} {prec}")
    assert abs(gm0 / m0 - 1) < (1e-14 if prec == "fp64" else 1e-7)
    assert abs(gm1 / gm0 - 1) < (1e-13 if prec == "fp64" else 1e-9), (gm0, gm1)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p,nlon,nlat", SMALL)
def test_step_parity_small_meshes(p, nlon, nlat, prec):
    """Five SSP-RK3 steps on every degree and ragged / degenerate mesh: from
    the second stage on each tile also stages its halo ring's increment
    (16-, 8- or 4-byte pieces, by the size of an element's modes)."""
    nsteps = 5
    o, u = case(nlon, nlat, p, 11)
    dt, m0, want = _oracle_run(nlon, nlat, p, 11, nsteps)
    with solver(nlon, nlat, p, prec) as s:
        s.set_state(u)
        s.step(nsteps, dt)
        got = s.get_state()
    assert_within(state_err(got, want), TOL[prec], f"{nsteps} steps p={p} {nlon}x{nlat} {prec}")


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_rk_orders(order):
    nlon, nlat, p = 16, 8, 2
    o, u = case(nlon, nlat, p, 5)
    dt = o.max_dt(u, 0.1)
    want = o.step(u, 13, dt, order)
    with solver(nlon, nlat, p, "fp64", rk_order=order) as s:
        s.set_option(dgswe.OPT_STEPS_PER_GRAPH, 4)   # graphs of 4 steps plus a remainder
        s.set_state(u)
        s.step(13, dt)
        assert_within(state_err(s.get_state(), want), 1e-12, f"RK{order}")


# ---------------------------------------------------- global Rusanov alpha --

@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5), ("fp32_tc_fp16", 8 * 2.0 ** -12),
                                      ("fp32_tc_fp16x3", 1e-5)])
def test_global_alpha_mode_matches_oracle(prec, tol):
    nlon, nlat, p = 44, 14, 3
    o = oracle_sphere(nlon, nlat, p)
    o.set_alpha_mode(1)
    u = o.project_tensor(synth.SmoothField(13).fields_grid)
    dt = o.max_dt(u, 0.1)
    want = o.step(u, 12, dt, 3)
    with solver(nlon, nlat, p, prec) as s:
        k_local = s.rhs(u)
        s.set_option(dgswe.OPT_ALPHA_MODE, 1)
        k = s.rhs(u)
        S = o.rhs_magnitude(u)
        assert_within(tend_err(k, o.rhs(u), S, f"global-alpha rhs {prec}"), TEND_TOL.get(prec, tol),
                      f"global-alpha rhs {prec}")
        if prec == "fp64":   # the switch changes the tendency as it does in the oracle
            o_loc = oracle_sphere(nlon, nlat, p)
            d_or = o.rhs(u) - o_loc.rhs(u)
            assert np.abs((k - k_local) - d_or).max() <= 0.05 * np.abs(d_or).max()
        s.set_option(dgswe.OPT_STEPS_PER_GRAPH, 4)
        s.set_state(u)
        m0 = s.total_mass()
        s.step(12, dt)
        got = s.get_state()
        assert abs(s.total_mass() / m0 - 1) < (1e-13 if prec == "fp64" else 1e-9)
    if prec == "fp32_tc_fp16":
        for f in range(3):
            d = np.abs(got[..., f, :] - want[..., f, :]).max()
            assert d <= 12 * dt * tol * S[..., f, :].max() + 1e-5 * np.abs(want[..., f, :]).max()
    else:
        assert_within(state_err(got, want), tol, f"global-alpha 12 steps {prec}")


# ------------------------------------------------------------- diagnostics --

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_max_dt_and_mass_match_oracle(prec):
    nlon, nlat, p = 36, 18, 3
    o, u = case(nlon, nlat, p, 6)
    with solver(nlon, nlat, p, prec) as s:
        s.set_state(u)
        assert s.max_dt(0.1) == pytest.approx(o.max_dt(u, 0.1), rel=1e-12 if prec == "fp64" else 1e-6)
        assert s.total_mass() == pytest.approx(o.total_mass(u), rel=1e-14 if prec == "fp64" else 1e-8)


@pytest.mark.parametrize("nlon,nlat,p", [(20, 10, 1), (12, 7, 4)])
def test_project_nodal_matches_oracle(nlon, nlat, p):
    o = oracle_sphere(nlon, nlat, p)
    f = synth.SmoothField(9)
    want = o.project_tensor(f.fields_grid)
    with solver(nlon, nlat, p, "fp64") as s:
        got = s.project_grid(f.fields_grid)
    assert_within(state_err(got, want), 1e-13, "projection")


# -------------------------------------------------------- API and failures --

def test_roundtrip_resume_and_determinism_fp64():
    nlon, nlat, p = 24, 12, 2
    o, u = case(nlon, nlat, p, 7)
    dt = o.max_dt(u, 0.1)
    with solver(nlon, nlat, p, "fp64") as s:
        s.set_state(u)
        np.testing.assert_array_equal(s.get_state(), u)     # FP64 resident state is the input
        s.step(20, dt)
        a = s.get_state()
        s.set_state(u)
        s.step(10, dt)
        mid = s.get_state()
        s.set_state(mid)
        s.step(10, dt)
        np.testing.assert_array_equal(s.get_state(), a)     # bitwise resume
        launches = s.stage_launches()
    assert launches == 3 * 40 + 1 * 0


def test_determinism_fp32():
    nlon, nlat, p = 40, 20, 3
    _, u = case(nlon, nlat, p, 8)
    outs = []
    for _ in range(2):
        with solver(nlon, nlat, p, "fp32") as s:
            s.set_state(u)
            s.step(25, 1.0)
            outs.append((s.get_state(), s.total_mass()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nonphysical_and_nonfinite_are_reported(prec):
    nlon, nlat, p = 16, 8, 1
    _, u = case(nlon, nlat, p, 4)
    bad = u.copy()
    bad[3, 5, 0, 0] = -100.0                  # negative depth in one element
    with solver(nlon, nlat, p, prec) as s:
        with pytest.raises(dgswe.DGError) as e:
            s.rhs(bad)
        assert e.value.status == dgswe.DG_ENONPHYSICAL
        nan = u.copy()
        nan[2, 2, 1, 1] = np.nan              # NaN in a momentum mode
        with pytest.raises(dgswe.DGError) as e:
            s.rhs(nan)
        assert e.value.status == dgswe.DG_ENONFINITE
        s.set_state(nan)
        with pytest.raises(dgswe.DGError) as e:
            s.step(1, 1.0)
        assert e.value.status == dgswe.DG_ENONFINITE
        # the solver stays usable after a reported failure
        s.set_state(u)
        s.step(2, 1.0)
        assert np.isfinite(s.get_state()).all()


def test_option_errors():
    with solver(8, 4, 1, "fp64") as s:
        for key, val, status in [(dgswe.OPT_PRECISION, 7, dgswe.DG_EINVAL),
                                 (dgswe.OPT_ALPHA_MODE, 2, dgswe.DG_EINVAL),
                                 (dgswe.OPT_RK_ORDER, 5, dgswe.DG_EINVAL),
                                 (99, 0, dgswe.DG_EINVAL)]:
            with pytest.raises(dgswe.DGError) as e:
                s.set_option(key, val)
            assert e.value.status == status
        with pytest.raises(dgswe.DGError):
            s.step(1, 1.0)                    # no state yet
        with pytest.raises(ValueError):
            s.set_state(np.zeros(5))


def test_precision_switch_keeps_state():
    nlon, nlat, p = 20, 10, 1
    _, u = case(nlon, nlat, p, 1)
    with solver(nlon, nlat, p, "fp64") as s:
        s.set_state(u)
        s.set_option(dgswe.OPT_PRECISION, dgswe.PREC["fp32"])
        assert_within(state_err(s.get_state(), u), 1e-7, "to fp32")
        s.set_option(dgswe.OPT_PRECISION, dgswe.PREC["fp64"])
        assert_within(state_err(s.get_state(), u), 1e-7, "back to fp64")


# --------------------------------------------- the largest mesh, sampled --

def _large_state(nlon, nlat, p, seed):
    """A seeded modal state for a mesh too large to project: element means of
    the smooth field (mode 0) plus small seeded higher modes (any modal
    coefficients are a valid DG state; the depth stays positive)."""
    field = synth.SmoothField(seed)
    lam = (np.arange(nlon) + 0.5) * (2 * math.pi / nlon)
    th = -0.5 * math.pi + (np.arange(nlat) + 0.5) * (math.pi / nlat)
    u = np.zeros((nlat, nlon, 3, (p + 1) ** 2))
    rng = np.random.default_rng(seed)
    for f, v in enumerate(field.fields_grid(lam, th)):
        u[:, :, f, 0] = 2.0 * v
        u[:, :, f, 1:] = rng.normal(size=(nlat, nlon, (p + 1) ** 2 - 1)) * (1e-3 * np.abs(v).max())
    return u


def test_rhs_parity_largest_mesh_sampled():
    """1440 x 720, degree 4 (the largest bench mesh, 1.04 M elements): the
    whole-mesh tendency of the FP64, FP32 and BF16 tensor-core stages against
    the oracle's element-by-element tendency on sampled elements (pole rows,
    the periodic seam, tile boundaries and random ones), each relative to the
    element's own magnitude bound."""
    nlon, nlat, p = 1440, 720, 4
    u = _large_state(nlon, nlat, p, 3)
    o = oracle_sphere(nlon, nlat, p)
    rng = np.random.default_rng(0)
    picks = {(0, 0), (0, nlon - 1), (nlat - 1, 0), (nlat - 1, nlon - 1), (nlat // 2, 0), (1, 719), (2, 720),
             (3, 29), (4, 30), (7, 31), (8, 32), (nlat // 2 + 1, 47), (nlat - 2, 1)}
    picks |= {(int(j), int(i)) for j, i in zip(rng.integers(0, nlat, 120), rng.integers(0, nlon, 120))}
    want = {(j, i): (o.rhs_element(u, j, i), o.rhs_magnitude_element(u, j, i)) for j, i in sorted(picks)}
    # per element, relative to its own bound: FP64 3e-14 as everywhere; FP32
    # 1e-5, the summation bound 2 gamma_N of FP32 (the whole-mesh 1e-6 is
    # taken against the mesh's largest bound)
    for prec, tol in (("fp64", TEND_TOL["fp64"]), ("fp32", 1e-5), ("fp32_tc_bf16", 8 * 2.0 ** -9)):
        with solver(nlon, nlat, p, prec) as s:
            k = s.rhs(u)
        for (j, i), (kw, Sw) in want.items():
            for f in range(3):
                err = np.abs(k[j, i, f] - kw[f]).max() / Sw[f].max()
                assert err <= tol, (prec, j, i, f, err)



@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_tc_fp16"])
def test_zero_steps_change_nothing(prec):
    nlon, nlat, p = 12, 6, 2
    _, u = case(nlon, nlat, p, 9)
    with solver(nlon, nlat, p, prec) as s:
        s.set_state(u)
        before = s.get_state()
        s.step(0, 1.0)
        np.testing.assert_array_equal(s.get_state(), before)
        assert s.stage_launches() == 0 and s.get_time() == 0.0


# --------------------------------------------------------- well-balanced option --

@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5), ("fp32_tc_fp16", 8 * 2.0 ** -12),
                                      ("fp32_tc_fp16x3", 1e-5)])
def test_well_balanced_option_matches_oracle(prec, tol):
    nlon, nlat, p = 44, 14, 3
    u = case(nlon, nlat, p, 15)[1]
    href = 0.5 * u[..., 0, 0].mean()          # the library's reference depth: the mean element depth
    o = oracle_sphere(nlon, nlat, p)
    o.set_well_balanced(href)
    dt = o.max_dt(u, 0.1)
    with solver(nlon, nlat, p, prec) as s:
        s.set_state(u)
        s.set_option(dgswe.OPT_WELL_BALANCED, 1)       # toggled with a resident state: kept
        assert_within(state_err(s.get_state(), u), 1e-7 if prec != "fp64" else 1e-15, "state kept")
        S = o.rhs_magnitude(u)
        assert_within(tend_err(s.rhs(u), o.rhs(u), S, f"well-balanced rhs {prec}"), TEND_TOL.get(prec, tol),
                      f"well-balanced rhs {prec}")
        rest = np.zeros_like(u)
        rest[..., 0, 0] = 2.0 * 5000.0
        assert np.abs(s.rhs(rest)).max() == 0.0       # the rest state is exactly steady
        s.set_option(dgswe.OPT_STEPS_PER_GRAPH, 4)
        s.set_state(u)
        s.step(10, dt)
        got = s.get_state()
    want = o.step(u, 10, dt, 3)
    if prec == "fp32_tc_fp16":
        for f in range(3):
            d = np.abs(got[..., f, :] - want[..., f, :]).max()
            assert d <= 10 * dt * tol * S[..., f, :].max() + 1e-5 * np.abs(want[..., f, :]).max()
    else:
        assert_within(state_err(got, want), tol, f"well-balanced 10 steps {prec}")
