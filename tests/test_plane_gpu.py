"""The planar validation problem on the GPU (linear advection on the periodic
unit square, FP64): parity with the oracle's planar mode, and the paper's
printed convergence tables reproduced through the CUDA path."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2303_11767_gb300 import dgswe

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
