"""The planar validation problem on the GPU (linear advection on the periodic
unit square, FP64): parity with the oracle's planar mode, and the paper's
printed convergence tables reproduced through the CUDA path."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2303_11767_gb300 import dgswe, synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "linear_advection_tables.txt")


def _golden():
    rows = {}
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            t, p, k, e = line.split()
            rows[(t, int(p), int(k))] = float(e)
    return rows


def _u0(x, y):
    return [np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)]


@pytest.mark.parametrize("alpha_speed", [False, True])
@pytest.mark.parametrize("p,nx,ny", [(0, 7, 5), (1, 9, 4), (2, 6, 7), (3, 5, 3), (4, 4, 6)])
def test_planar_rhs_and_steps_match_oracle(p, nx, ny, alpha_speed):
    o = O.Oracle.plane_advection(nx, ny, p, 0.7, -1.3, alpha_speed)
    rng = np.random.default_rng(p)
    u = rng.normal(size=o.shape)
    want = o.rhs(u)
    S = o.rhs_magnitude(u)
    with dgswe.Solver.plane_advection(nx, ny, p, 0.7, -1.3, alpha_speed) as s:
        k = s.rhs(u)
        assert np.abs(k - want).max() <= 1e-12 * S.max()
        s.set_option(dgswe.OPT_STEPS_PER_GRAPH, 4)
        s.set_state(u)
        s.step(10, 1e-3)
        got = s.get_state()
    ref = o.step(u, 10, 1e-3, 4)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def _advect_gpu(k, p, alpha_speed, dt):
    o = O.Oracle.plane_advection(k, k, p, 1.0, 1.0, alpha_speed)
    u = o.project_fn(_u0)
    with dgswe.Solver.plane_advection(k, k, p, 1.0, 1.0, alpha_speed, rk_order=4) as s:
        s.set_option(dgswe.OPT_STEPS_PER_GRAPH, 200)
        s.set_state(u)
        s.step(int(round(1.0 / dt)), dt)   # T = 1: one full period
        u1 = s.get_state()
    x, y = o.projection_points()
    return o.l2_error(u1, np.stack(_u0(x, y), axis=2), 0)


@pytest.mark.parametrize("p,k,alpha_speed,tol", [
    (1, 40, True, 0.02), (2, 20, True, 0.01), (2, 40, True, 0.01), (3, 20, False, 0.01), (3, 40, False, 0.01),
])
def test_gpu_reproduces_paper_tables(p, k, alpha_speed, tol):
    """Table sine_conv of the paper (GT4Py), through the CUDA path."""
    want = _golden()[("gt4py", p, k)]
    got = _advect_gpu(k, p, alpha_speed, 1e-3 if p < 3 else 5e-4)
    assert abs(got / want - 1) < tol, (got, want)


def test_gpu_convergence_rates():
    for p, alpha_speed in ((1, True), (2, True), (3, False)):
        e = [_advect_gpu(k, p, alpha_speed, 1e-3 if p < 3 else 5e-4) for k in (20, 40, 80)]
        rates = [math.log2(e[i] / e[i + 1]) for i in range(2)]
        assert all(abs(r - (p + 1)) < 0.3 for r in rates), (p, e, rates)


def test_planar_sphere_only_calls_are_rejected():
    with dgswe.Solver.plane_advection(4, 4, 1) as s:
        s.set_state(np.zeros(s.shape))
        for call in (s.total_mass, lambda: s.max_dt(0.1),
                     lambda: s.set_option(dgswe.OPT_PRECISION, dgswe.PREC["fp32"]),
                     lambda: s.set_option(dgswe.OPT_ALPHA_MODE, 1)):
            with pytest.raises(dgswe.DGError) as e:
                call()
            assert e.value.status == dgswe.DG_EUNSUPPORTED


# ------------------------------------------------ shallow water on the f-plane --

L_DOM, G_PL, F_PL = 1.0e7, 9.80616, 1.0e-4


@pytest.mark.parametrize("p,nx,ny", [(0, 6, 5), (1, 7, 4), (2, 5, 6), (3, 4, 5), (4, 3, 4)])
def test_plane_swe_rhs_and_steps_match_oracle(p, nx, ny):
    o = O.Oracle.plane_swe(nx, ny, p, L_DOM, G_PL, F_PL)
    rng = np.random.default_rng(10 + p)
    u = np.zeros(o.shape)
    u[..., 0, 0] = 2.0 * 1000.0
    u[..., :, 1:] = rng.normal(size=u[..., :, 1:].shape) * np.array([5.0, 200.0, 200.0])[:, None]
    u[..., 1:, 0] = rng.normal(size=u[..., 1:, 0].shape) * 500.0
    want = o.rhs(u)
    S = o.rhs_magnitude(u)
    with dgswe.Solver.plane_swe(nx, ny, p, L_DOM, G_PL, F_PL) as s:
        k = s.rhs(u)
        for f in range(3):
            assert np.abs(k[..., f, :] - want[..., f, :]).max() <= 1e-12 * S[..., f, :].max()
        s.set_option(dgswe.OPT_STEPS_PER_GRAPH, 4)
        s.set_state(u)
        m0 = s.total_mass()
        s.step(10, 100.0)
        got = s.get_state()
        m1 = s.total_mass()
    ref = o.step(u, 10, 100.0, 4)
    for f in range(3):
        assert np.abs(got[..., f, :] - ref[..., f, :]).max() <= 1e-12 * np.abs(ref[..., f, :]).max()
    assert m0 == pytest.approx(o.total_mass(u), rel=1e-14)
    assert abs(m1 / m0 - 1) < 1e-14


def test_geostrophic_adjustment_run_matches_oracle():
    """The paper's set-up (Sec. 4.3): 50x50 elements, degree 3, RK4, dt = 100 s,
    T = 36000 s, Gaussian hump on a fluid at rest, f = 1e-4; the initial state
    is projected by the library and by the oracle, and both runs agree."""
    nx = ny = 50
    p = 3
    o = O.Oracle.plane_swe(nx, ny, p, L_DOM, G_PL, F_PL)
    o.set_threads(os.cpu_count() or 1)
    fn = synth.geostrophic_adjustment_grid(L_DOM)

    with dgswe.Solver.plane_swe(nx, ny, p, L_DOM, G_PL, F_PL) as s:
        u0 = s.project_grid(fn)
        want0 = o.project_fn(lambda xx, yy: [1000.0 + 5.0 * np.exp(-((xx - L_DOM / 2) ** 2 + (yy - L_DOM / 2) ** 2)
                                                                   / (2 * (L_DOM / 20) ** 2)), 0 * xx, 0 * xx])
        np.testing.assert_allclose(u0, want0, rtol=0, atol=1e-12 * np.abs(want0).max())
        s.set_option(dgswe.OPT_STEPS_PER_GRAPH, 120)
        s.set_state(u0)
        m0 = s.total_mass()
        s.step(360, 100.0)
        got = s.get_state()
        m1 = s.total_mass()
    want = o.step(u0, 360, 100.0, 4)
    for f in range(3):
        assert np.abs(got[..., f, :] - want[..., f, :]).max() <= 1e-11 * np.abs(want[..., f, :]).max(), f
    assert abs(m1 / m0 - 1) < 1e-13
    # the hump has adjusted: flow in geostrophic rotation, mass unchanged
    assert np.abs(got[..., 1:, :]).max() > 1.0
