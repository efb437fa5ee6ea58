"""The tensor-core precisions (BF16 / FP16 operands, FP32 accumulation)
against the FP64 oracle, through the C-ABI.

Tolerances, from the arithmetic.  Rounding an FP32 value to the operand type
has relative error at most u = 2^-9 (BF16) or 2^-12 (FP16).  Every term of the
tendency is a product of a rounded basis entry and a rounded point value
(a flux, a source or an edge flux) computed from rounded modal coefficients;
a flux is at most quadratic in the state, so each term carries a relative
error of a few u.  With C = 8 units the tendency therefore stays within
C * u * S, S = |M^-1| sum |terms| the oracle's magnitude bound (the same
measure as the FP32 / FP64 parity tests).  A state after K steps of size dt
stays within K dt C u |S| of the oracle's, plus the FP32 state tolerance.
The contraction itself (exact products of rounded operands, FP32 sums of at
most 32 terms) matches an FP64 product of the rounded operands to 1e-5.

Split operands (precisions fp32_tc_bf16x3, fp32_tc_fp16x3): each operand is
a pair hi + lo of the 16-bit type, which represents it to u^2, and each
product is A_hi B_hi + A_lo B_hi + A_hi B_lo; the neglected A_lo B_lo is of
order u^2 too.  Their tendencies are held to C u^2 S plus the FP32
tendency tolerance (1e-6 S), and their states to the plain per-field FP32
tolerance 1e-5 (relative L2 and max), with no derived allowance.  FP16 pairs
also have an absolute floor: a residual below FP16's smallest normal (6.1e-5)
is subnormal, spaced 2^-24, so an operand x is held to about 3e-8 / |x|; the
smallest fluxes of a coarse degree-0 mesh (~0.03) put that near 1e-6, and the
FP16-pair tendency bound gets 4e-6 S on top.
"""
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import oracle as O
from paper_2303_11767_gb300 import dgswe, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

R, G, OMEGA = synth.EARTH_RADIUS, 9.80616, 7.292e-5
OPS = {"fp32_tc_bf16": (0, 2.0 ** -9, torch.bfloat16), "fp32_tc_fp16": (1, 2.0 ** -12, torch.float16)}
SPLIT = {"fp32_tc_bf16x3": 2.0 ** -18, "fp32_tc_fp16x3": 2.0 ** -24}   # u^2 of the pair
SPLIT_FLOOR = {"fp32_tc_bf16x3": 1e-6, "fp32_tc_fp16x3": 4e-6}        # + FP32 rounding / FP16 subnormals
C = 8.0
_cache = {}


def case(nlon, nlat, p, seed):
    key = (nlon, nlat, p, seed)
    if key not in _cache:
        o = O.Oracle.sphere(nlon, nlat, p, R, G, OMEGA)
        _cache[key] = (o, o.project_tensor(synth.SmoothField(seed).fields_grid))
    return _cache[key]


def tend_err(x, y, S):
    x = np.asarray(x).reshape(y.shape)
    return [(np.linalg.norm(x[..., f, :] - y[..., f, :]) / np.linalg.norm(S[..., f, :]),
             np.abs(x[..., f, :] - y[..., f, :]).max() / S[..., f, :].max()) for f in range(3)]


def _orthonormal(k, x):
    c = np.zeros(k + 1)
    c[k] = 1.0
    return np.sqrt((2 * k + 1) / 2.0) * npleg.legval(x, c)


def eval_trace_matrix(n, n1, k1):
    """B1 written out from its definition: rows = Gauss points (padded to 8),
    then the S, N, W, E edge points; columns = modes m = b n + a."""
    x, _ = npleg.leggauss(n)
    npts = n * n
    nc = 8 * ((npts + 7) // 8)
    B = np.zeros((n1, k1))
    for m in range(npts):
        a, b = m % n, m // n
        for q in range(npts):
            B[q, m] = _orthonormal(a, x[q % n]) * _orthonormal(b, x[q // n])
        for k in range(n):
            B[nc + k, m] = _orthonormal(a, x[k]) * _orthonormal(b, -1.0)
            B[nc + n + k, m] = _orthonormal(a, x[k]) * _orthonormal(b, 1.0)
            B[nc + 2 * n + k, m] = _orthonormal(a, -1.0) * _orthonormal(b, x[k])
            B[nc + 3 * n + k, m] = _orthonormal(a, 1.0) * _orthonormal(b, x[k])
    return B


@pytest.mark.parametrize("prec", list(OPS))
@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_contraction_on_tensor_cores(p, prec):
    op, _, tdt = OPS[prec]
    n1, k1 = dgswe.tc_contraction_shape(p, op)
    rng = np.random.default_rng(p)
    a = rng.normal(size=(128, k1)) * 10.0 ** rng.uniform(-2, 2, size=(128, 1))
    a[:, (p + 1) ** 2:] = 0.0
    da = torch.tensor(a, dtype=torch.float32, device="cuda")
    out = torch.empty((128, n1), dtype=torch.float32, device="cuda")
    dgswe.tc_check_contraction(p, op, da, out)
    ar = da.to(tdt).double().cpu().numpy()
    Br = torch.tensor(eval_trace_matrix(p + 1, n1, k1), dtype=torch.float32).to(tdt).double().numpy()
    want = ar @ Br.T
    got = out.double().cpu().numpy()
    scale = np.abs(ar) @ np.abs(Br).T
    assert np.all(np.abs(got - want) <= 1e-5 * scale + 1e-30), np.abs(got - want).max()


# meshes with ragged tiles in both directions (30 elements per warp row,
# 8 rows per CTA for p <= 3 and 4 for p = 4) and a tiny one
MESHES = [(44, 14), (7, 3)]


@pytest.mark.parametrize("prec", list(OPS))
@pytest.mark.parametrize("nlon,nlat", MESHES)
@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_rhs_matches_oracle(p, nlon, nlat, prec):
    o, u = case(nlon, nlat, p, 21)
    with dgswe.Solver(nlon, nlat, p, R, G, OMEGA, precision=prec) as s:
        k = s.rhs(u)
    tol = C * OPS[prec][1]
    for f, (l2, mx) in enumerate(tend_err(k, o.rhs(u), o.rhs_magnitude(u))):
        assert l2 <= tol and mx <= tol, (f, l2, mx, tol)


@pytest.mark.parametrize("prec", list(OPS))
@pytest.mark.parametrize("nlon,nlat,p,seed", [(180, 90, 3, 2), (360, 180, 4, 3)])
def test_rhs_matches_oracle_full_size(nlon, nlat, p, seed, prec):
    o, u = case(nlon, nlat, p, seed)
    with dgswe.Solver(nlon, nlat, p, R, G, OMEGA, precision=prec) as s:
        k = s.rhs(u)
    errs = tend_err(k, o.rhs(u), o.rhs_magnitude(u))
    tol = C * OPS[prec][1]
    print(prec, nlon, nlat, p, ["%.2e/%.2e" % e for e in errs])
    for f, (l2, mx) in enumerate(errs):
        assert l2 <= tol and mx <= tol, (f, l2, mx, tol)


@pytest.mark.parametrize("prec", list(OPS))
def test_rest_state_equals_fp32_path(prec):
    """h constant, u = v = 0: every rounded operand is zero, so the tendency is
    the rest-state pressure term alone, as on the FP32 path."""
    nlon, nlat, p = 36, 18, 3
    u = np.zeros((nlat, nlon, 3, (p + 1) ** 2))
    u[..., 0, 0] = 2.0 * 5000.0                 # mode 0 of the orthonormal basis: 2 x mean
    out = {}
    for pr in ("fp32", prec):
        with dgswe.Solver(nlon, nlat, p, R, G, OMEGA, precision=pr) as s:
            out[pr] = s.rhs(u)
    np.testing.assert_allclose(out[prec], out["fp32"], rtol=0, atol=1e-6 * np.abs(out["fp32"]).max())


@pytest.mark.parametrize("prec", list(OPS))
@pytest.mark.parametrize("nlon,nlat,p,seed,nsteps", [(20, 10, 1, 1, 100), (64, 32, 4, 4, 60)])
def test_steps_match_oracle_and_keep_mass(nlon, nlat, p, seed, nsteps, prec):
    o, u = case(nlon, nlat, p, seed)
    dt = o.max_dt(u, 0.1)
    want = o.step(u, nsteps, dt, 3)
    S = o.rhs_magnitude(u)
    with dgswe.Solver(nlon, nlat, p, R, G, OMEGA, precision=prec) as s:
        s.set_option(dgswe.OPT_STEPS_PER_GRAPH, 16)
        s.set_state(u)
        m0 = s.total_mass()
        s.step(nsteps, dt)
        got = s.get_state()
        m1 = s.total_mass()
    tol = C * OPS[prec][1]
    for f in range(3):
        d = np.abs(got[..., f, :] - want[..., f, :]).max()
        bound = nsteps * dt * tol * S[..., f, :].max() + 1e-5 * np.abs(want[..., f, :]).max()
        assert d <= bound, (f, d, bound)
    assert abs(m1 / m0 - 1) < 1e-9, (m0, m1)


def test_tc_precisions_agree_with_each_other_and_fp32():
    """FP16 (3 more mantissa bits) is closer to the FP32 path than BF16."""
    nlon, nlat, p = 60, 30, 3
    o, u = case(nlon, nlat, p, 12)
    ks = {}
    for pr in ("fp32", "fp32_tc_bf16", "fp32_tc_fp16"):
        with dgswe.Solver(nlon, nlat, p, R, G, OMEGA, precision=pr) as s:
            ks[pr] = s.rhs(u)
    S = o.rhs_magnitude(u)
    e_bf = max(m for _, m in tend_err(ks["fp32_tc_bf16"], ks["fp32"], S))
    e_fp = max(m for _, m in tend_err(ks["fp32_tc_fp16"], ks["fp32"], S))
    assert e_fp < e_bf


def test_precision_switch_to_tc_keeps_state():
    nlon, nlat, p = 20, 10, 2
    _, u = case(nlon, nlat, p, 1)
    with dgswe.Solver(nlon, nlat, p, R, G, OMEGA, precision="fp64") as s:
        s.set_state(u)
        for pr in ("fp32_tc_bf16", "fp32_tc_fp16", "fp64"):
            s.set_option(dgswe.OPT_PRECISION, dgswe.PREC[pr])
            got = s.get_state()
            for f in range(3):
                assert np.abs(got[..., f, :] - u[..., f, :]).max() <= 1e-7 * np.abs(u[..., f, :]).max()


def test_tc_determinism_and_launch_count():
    nlon, nlat, p = 40, 20, 4
    _, u = case(nlon, nlat, p, 8)
    outs = []
    for _ in range(2):
        with dgswe.Solver(nlon, nlat, p, R, G, OMEGA, precision="fp32_tc_bf16") as s:
            s.set_option(dgswe.OPT_STEPS_PER_GRAPH, 4)
            s.set_state(u)
            s.step(9, 1.0)
            outs.append(s.get_state())
            assert s.stage_launches() == 27
    np.testing.assert_array_equal(outs[0], outs[1])


def test_first_use_is_a_captured_step():
    """A fresh process whose first tensor-core stage is recorded into a CUDA
    graph: everything that allocates happens when the precision is chosen."""
    import subprocess
    import sys
    code = ("import numpy as np\n"
            "from paper_2303_11767_gb300 import dgswe, synth\n"
            "s = dgswe.Solver(40, 20, 3, precision='fp32_tc_fp16')\n"
            "s.set_option(dgswe.OPT_STEPS_PER_GRAPH, 8)\n"
            "s.set_state(s.project_grid(synth.SmoothField(3).fields_grid))\n"
            "s.step(16, s.max_dt(0.1))\n"
            "assert np.isfinite(s.get_state()).all()\n"
            "print('ok', s.stage_launches())\n")
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.split() == ["ok", "48"]


@pytest.mark.parametrize("prec", ["fp32", "fp32_tc_bf16", "fp32_tc_fp16", "fp32_tc_bf16x3", "fp32_tc_fp16x3"])
def test_precision_config_360x180_p4_500_steps(prec):
    """The precision configuration: 360x180, degree 4, 500 SSP-RK3 steps at
    CFL 0.1, per-field relative L2 and max error against the FP64 oracle.
    FP32 and the split tensor-core precisions: within the plain 1e-5;
    the single-pass ones: within their derived allowance."""
    nlon, nlat, p, seed, nsteps = 360, 180, 4, 3, 500
    key = ("run500", nlon, nlat, p, seed)
    o, u = case(nlon, nlat, p, seed)
    if key not in _cache:
        o.set_threads(os.cpu_count() or 1)
        dt = o.max_dt(u, 0.1)
        _cache[key] = (dt, o.step(u, nsteps, dt, 3), o.rhs_magnitude(u))
    dt, want, S = _cache[key]
    with dgswe.Solver(nlon, nlat, p, R, G, OMEGA, precision=prec) as s:
        s.set_option(dgswe.OPT_STEPS_PER_GRAPH, 100)
        s.set_state(u)
        m0 = s.total_mass()
        s.step(nsteps, dt)
        got = s.get_state()
        m1 = s.total_mass()
    errs = []
    for f in range(3):
        d = got[..., f, :] - want[..., f, :]
        errs.append((np.linalg.norm(d) / np.linalg.norm(want[..., f, :]), np.abs(d).max() / np.abs(want[..., f, :]).max()))
    print(f"\n{prec} 360x180 p=4, 500 steps: rel L2 / max per field (h, hu, hv):",
          " ".join("%.2e/%.2e" % e for e in errs), "mass drift %.1e" % (m1 / m0 - 1))
    if prec == "fp32" or prec in SPLIT:
        for f, (l2, mx) in enumerate(errs):
            assert l2 <= 1e-5 and mx <= 1e-5, (prec, f, l2, mx)
    else:
        tol = C * OPS[prec][1]
        for f in range(3):
            d = np.abs(got[..., f, :] - want[..., f, :]).max()
            bound = nsteps * dt * tol * S[..., f, :].max() + 1e-5 * np.abs(want[..., f, :]).max()
            assert d <= bound, (f, d, bound)
    assert abs(m1 / m0 - 1) < 1e-9


# ------------------------------------------------------------ split operands --

def state_errs(got, want):
    out = []
    for f in range(3):
        d = got[..., f, :] - want[..., f, :]
        out.append((np.linalg.norm(d) / np.linalg.norm(want[..., f, :]), np.abs(d).max() / np.abs(want[..., f, :]).max()))
    return out


@pytest.mark.parametrize("prec", list(SPLIT))
@pytest.mark.parametrize("nlon,nlat", MESHES)
@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_split_rhs_matches_oracle(p, nlon, nlat, prec):
    o, u = case(nlon, nlat, p, 21)
    with dgswe.Solver(nlon, nlat, p, R, G, OMEGA, precision=prec) as s:
        k = s.rhs(u)
    tol = C * SPLIT[prec] + SPLIT_FLOOR[prec]
    for f, (l2, mx) in enumerate(tend_err(k, o.rhs(u), o.rhs_magnitude(u))):
        assert l2 <= tol and mx <= tol, (f, l2, mx, tol)


@pytest.mark.parametrize("prec", list(SPLIT))
@pytest.mark.parametrize("nlon,nlat,p,seed", [(180, 90, 3, 2), (360, 180, 4, 3)])
def test_split_rhs_matches_oracle_full_size(nlon, nlat, p, seed, prec):
    o, u = case(nlon, nlat, p, seed)
    with dgswe.Solver(nlon, nlat, p, R, G, OMEGA, precision=prec) as s:
        k = s.rhs(u)
    errs = tend_err(k, o.rhs(u), o.rhs_magnitude(u))
    print(prec, nlon, nlat, p, ["%.2e/%.2e" % e for e in errs])
    tol = C * SPLIT[prec] + SPLIT_FLOOR[prec]
    for f, (l2, mx) in enumerate(errs):
        assert l2 <= tol and mx <= tol, (f, l2, mx, tol)


@pytest.mark.parametrize("prec", list(SPLIT))
@pytest.mark.parametrize("nlon,nlat,p,seed,nsteps", [(20, 10, 1, 1, 100), (64, 32, 4, 4, 60), (180, 90, 3, 2, 1000)])
def test_split_steps_match_oracle_within_fp32_tolerance(nlon, nlat, p, seed, nsteps, prec):
    """States after 100 (20x10, degree 1), 60 (64x32, degree 4) and 1000
    (180x90, degree 3) SSP-RK3 steps: plain per-field 1e-5, mass to 1e-9."""
    key = ("run", nlon, nlat, p, seed, nsteps)
    o, u = case(nlon, nlat, p, seed)
    if key not in _cache:
        o.set_threads(os.cpu_count() or 1)
        dt = o.max_dt(u, 0.1)
        _cache[key] = (dt, o.step(u, nsteps, dt, 3))
    dt, want = _cache[key]
    with dgswe.Solver(nlon, nlat, p, R, G, OMEGA, precision=prec) as s:
        s.set_option(dgswe.OPT_STEPS_PER_GRAPH, 50)
        s.set_state(u)
        m0 = s.total_mass()
        s.step(nsteps, dt)
        got = s.get_state()
        m1 = s.total_mass()
    errs = state_errs(got, want)
    print(f"\n{prec} {nlon}x{nlat} p={p}, {nsteps} steps: rel L2 / max (h, hu, hv):",
          " ".join("%.2e/%.2e" % e for e in errs))
    for f, (l2, mx) in enumerate(errs):
        assert l2 <= 1e-5 and mx <= 1e-5, (prec, f, l2, mx)
    assert abs(m1 / m0 - 1) < 1e-9, (m0, m1)


def test_split_is_closer_to_fp32_than_single_pass():
    nlon, nlat, p = 60, 30, 3
    o, u = case(nlon, nlat, p, 12)
    ks = {}
    for pr in ("fp32", "fp32_tc_fp16", "fp32_tc_bf16x3", "fp32_tc_fp16x3"):
        with dgswe.Solver(nlon, nlat, p, R, G, OMEGA, precision=pr) as s:
            ks[pr] = s.rhs(u)
    S = o.rhs_magnitude(u)
    e = {pr: max(m for _, m in tend_err(ks[pr], ks["fp32"], S)) for pr in ks if pr != "fp32"}
    assert e["fp32_tc_fp16x3"] < e["fp32_tc_bf16x3"] < e["fp32_tc_fp16"], e
