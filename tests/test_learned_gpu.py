"""Learned correction on the GPU: the network kernels against the FP64
reference (forward, gradients), training, the nested projection, and the
learned source term inside the degree-1 solver."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlp_oracle as M
from paper_2303_11767_gb300 import dgswe, learned, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
R, G, OMEGA = synth.EARTH_RADIUS, 9.80616, 7.292e-5


def _norm(rng, n_in=60, n_out=12):
    return (rng.normal(size=n_in).astype(np.float32), (1 + rng.random(n_in)).astype(np.float32),
            rng.normal(size=n_out).astype(np.float32), (1 + rng.random(n_out)).astype(np.float32))


def test_forward_and_gradients_match_fp64_reference():
    rng = np.random.default_rng(1)
    mlp = dgswe.MLP(60, 128, 12, seed=3)
    norm = _norm(rng)
    mlp.set_normalization(*norm)
    batch = 300                                   # not a multiple of the 64-row tiles
    x = (rng.normal(size=(batch, 60)) * norm[1] + norm[0]).astype(np.float32)
    t = (rng.normal(size=(batch, 12)) * norm[3] + norm[2]).astype(np.float32)
    dx, dt = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    y = torch.empty(batch, 12, dtype=torch.float32, device="cuda")
    mlp.forward(dx, y)
    p = mlp.get_params().astype(np.float64)
    nrm = tuple(a.astype(np.float64) for a in norm)
    want_y, _ = M.forward(p, x, nrm, 60, 128, 12)
    assert np.abs(y.cpu().numpy() - want_y).max() < 1e-5 * np.abs(want_y).max()
    g, loss = mlp.gradients(dx, dt)
    want_loss, want_g = M.loss_and_grad(p, x, t, nrm, 60, 128, 12)
    assert abs(loss / want_loss - 1) < 1e-5
    assert np.abs(g - want_g).max() < 1e-4 * np.abs(want_g).max()


def test_training_reduces_the_loss():
    rng = np.random.default_rng(2)
    mlp = dgswe.MLP(60, 128, 12, seed=4)
    A = rng.normal(size=(60, 12)) / 8
    x = rng.normal(size=(8192, 60)).astype(np.float32)
    t = (np.tanh(x @ A) + 0.01 * rng.normal(size=(8192, 12))).astype(np.float32)
    dx, dt = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    first = mlp.train_step(dx[:1024], dt[:1024], 1e-3)
    for k in range(300):
        b = (k % 8) * 1024
        last = mlp.train_step(dx[b:b + 1024], dt[b:b + 1024], 1e-3)
    assert last < 0.5 * first, (first, last)


def test_restriction_is_exact_for_coarse_polynomials():
    nlonc, nlatc, r = 4, 2, 5
    rng = np.random.default_rng(5)
    coef = rng.normal(size=(nlatc, nlonc, 3, 4))
    coef[..., 0, 0] = 5000 + 100 * rng.random((nlatc, nlonc))
    dl, dth = 2 * math.pi / nlonc, math.pi / nlatc

    def f(lam, th):
        I = np.minimum((lam / dl).astype(int), nlonc - 1)
        J = np.minimum(((th + math.pi / 2) / dth).astype(int), nlatc - 1)
        x = lam - (I + 0.5) * dl
        y = th - (-math.pi / 2 + (J + 0.5) * dth)
        c = coef[J, I]
        return [c[..., k, 0] + c[..., k, 1] * x + c[..., k, 2] * y + 10 * c[..., k, 3] * x * y for k in range(3)]

    fine = O.Oracle.sphere(nlonc * r, nlatc * r, 4, R, G, OMEGA)
    coarse = O.Oracle.sphere(nlonc, nlatc, 1, R, G, OMEGA)
    uf, want = fine.project_fn(f), coarse.project_fn(f)
    with dgswe.Solver(nlonc * r, nlatc * r, 4, R, G, OMEGA, precision="fp64") as sf, \
            dgswe.Solver(nlonc, nlatc, 1, R, G, OMEGA, precision="fp64") as sc:
        sf.set_state(uf)
        sc.restrict_from(sf)
        got = sc.get_state()
    for k in range(3):
        assert np.abs(got[..., k, :] - want[..., k, :]).max() < 1e-11 * np.abs(want[..., k, :]).max()


def _coarse_state():
    o = O.Oracle.sphere(72, 36, 1, R, G, OMEGA)
    u = o.project_tensor(synth.SmoothField(7).fields_grid)
    return o, u


def test_zero_network_leaves_the_solver_unchanged():
    o, u = _coarse_state()
    mlp = dgswe.MLP(60, 128, 12, seed=1)
    p = mlp.get_params()
    p[-(12 * 128 + 12):] = 0.0                    # W3 = 0, b3 = 0
    mlp.set_params(p)
    rng = np.random.default_rng(0)
    norm = _norm(rng)
    mlp.set_normalization(norm[0], norm[1], np.zeros(12, np.float32), norm[3])
    dt = o.max_dt(u, 0.1)
    out = []
    for attach in (False, True):
        with dgswe.Solver(72, 36, 1, R, G, OMEGA, precision="fp32") as s:
            s.set_state(u)
            if attach:
                s.attach_mlp(mlp)
            s.step(10, dt)
            out.append(s.get_state())
    np.testing.assert_array_equal(out[0], out[1])


def test_learned_source_matches_reference_and_keeps_mass():
    o, u = _coarse_state()
    mlp = dgswe.MLP(60, 128, 12, seed=2)
    X = learned.gather_inputs(u)
    mlp.set_normalization(X.mean(0), X.std(0) + 1e-6, np.zeros(12, np.float32), np.full(12, 1e-3, np.float32))
    with dgswe.Solver(72, 36, 1, R, G, OMEGA, precision="fp32") as s:
        k0 = s.rhs(u)
        s.attach_mlp(mlp)
        k1 = s.rhs(u)
        # reference: network output (denormalised), then the mass shift of mode 0 of h
        p = mlp.get_params().astype(np.float64)
        nrm = (X.mean(0).astype(np.float32).astype(np.float64), (X.std(0) + 1e-6).astype(np.float32).astype(np.float64),
               np.zeros(12), np.full(12, 1e-3, np.float32).astype(np.float64))
        y, _ = M.forward(p, X, nrm, 60, 128, 12)
        src = (y * nrm[3] + nrm[2]).reshape(36, 72, 3, 4)
        c0 = np.array([[o.mass_matrix(j)[0, 0], o.mass_matrix(j)[0, 2]] for j in range(36)])
        mass = (c0[:, None, 0] * src[..., 0, 0] + c0[:, None, 1] * src[..., 0, 2]).sum()
        src[..., 0, 0] -= mass / (c0[:, 0].sum() * 72)
        d = (k1 - k0) - src
        assert np.abs(d).max() < 1e-3 * np.abs(src).max()
        # mass is kept while stepping with the source
        s.set_state(u)
        m0 = s.total_mass()
        s.step(50, o.max_dt(u, 0.1))
        assert abs(s.total_mass() / m0 - 1) < 1e-8


def test_row_normalised_source_matches_reference():
    o, u = _coarse_state()
    mlp = dgswe.MLP(60, 128, 12, seed=3)
    X = learned.gather_inputs(u)
    mlp.set_normalization(X.mean(0), X.std(0) + 1e-6, np.zeros(12, np.float32), np.ones(12, np.float32))
    rng = np.random.default_rng(4)
    om = (rng.normal(size=(36, 12)) * 1e-4).astype(np.float32)
    osd = (1e-3 * (1 + rng.random((36, 12)))).astype(np.float32)
    mlp.set_row_normalization(om, osd)
    with dgswe.Solver(72, 36, 1, R, G, OMEGA, precision="fp32") as s:
        k0 = s.rhs(u)
        s.attach_mlp(mlp)
        k1 = s.rhs(u)
    p = mlp.get_params().astype(np.float64)
    nrm = (X.mean(0).astype(np.float32).astype(np.float64), (X.std(0) + 1e-6).astype(np.float32).astype(np.float64),
           np.zeros(12), np.ones(12))
    y, _ = M.forward(p, X, nrm, 60, 128, 12)
    rows = np.arange(36 * 72) // 72
    src = (y * osd[rows] + om[rows]).reshape(36, 72, 3, 4)
    c0 = np.array([[o.mass_matrix(j)[0, 0], o.mass_matrix(j)[0, 2]] for j in range(36)])
    mass = (c0[:, None, 0] * src[..., 0, 0] + c0[:, None, 1] * src[..., 0, 2]).sum()
    src[..., 0, 0] -= mass / (c0[:, 0].sum() * 72)
    assert np.abs((k1 - k0) - src).max() < 1e-3 * np.abs(src).max()
    # statistics of another mesh are refused when the source runs
    mlp.set_row_normalization(om[:20], osd[:20])
    with dgswe.Solver(72, 36, 1, R, G, OMEGA, precision="fp32") as s:
        s.attach_mlp(mlp)
        with pytest.raises(dgswe.DGError) as e:
            s.rhs(u)
        assert e.value.status == dgswe.DG_EINVAL


def test_pipeline_end_to_end_reports_plain_vs_learned(capsys):
    """Reduced pipeline (64 pairs of one training run, 2 epochs, 1 h on a
    held-out seed): it runs on the library kernels end to end, the learned
    solver keeps mass, and the comparison with plain coarse DG is reported.
    The full-size comparison is recorded with its numbers in
    profiles/learned_correction_c5.md."""
    X, T = learned.generate(64, [5000], spinup_s=600.0, stride=8, target_steps=8, log=lambda s: None)
    assert X.shape == (64 * 2592, 60) and T.shape == (64 * 2592, 12)
    assert np.isfinite(X).all() and np.isfinite(T).all()
    mlp, norm, hist = learned.train(X, T, epochs=2, batch=4096, log=lambda s: None)
    assert hist[-1] < hist[0]
    ev = learned.evaluate(mlp, 6000, 3600.0, checkpoints=1, spinup_s=600.0, log=lambda s: None)[-1]
    assert all(np.isfinite(ev["plain"])) and all(np.isfinite(ev["learned"]))
    assert abs(ev["mass_drift_learned"]) < 1e-9
    with capsys.disabled():
        print("\nlearned correction (reduced), 1 h, relative L2 (h, hu, hv): plain",
              ["%.2e" % v for v in ev["plain"]], "learned", ["%.2e" % v for v in ev["learned"]])


def test_learned_source_gains_over_plain_dg(capsys):
    """What the trained network gains over the method without it: 300 pairs
    of two training runs (targets over 8 coarse steps), 8 epochs; the
    shrinkage of the learned source chosen on a validation seed (6001, 2 h)
    among 0.5, 0.25, 0.1; then, on the held-out test seed 6000 after 3 h,
    the learned coarse solver's relative L2 error against the projected fine
    run is below plain coarse DG's in every field."""
    X, T = learned.generate(300, [5000, 5001], stride=8, target_steps=8, log=lambda s: None)
    mlp, norm, hist = learned.train(X, T, epochs=8, log=lambda s: None)
    alpha, val = learned.select_alpha(mlp, norm, [0.5, 0.25, 0.1], 6001, 2.0, log=lambda s: None)
    net = learned.scaled_copy(mlp, norm, alpha)
    row = learned.evaluate_many({"learned": net}, 6000, 3 * 3600.0, checkpoint_hours=[3.0], log=lambda s: None)[-1]
    with capsys.disabled():
        print(f"\nlearned correction, alpha {alpha} (validation scores {val['score']}), 3 h on the test seed, "
              "relative L2 (h, hu, hv): plain", ["%.2e" % v for v in row["plain"]],
              "learned", ["%.2e" % v for v in row["learned"]])
    assert abs(row["mass_drift_learned"]) < 1e-9
    assert all(l < p for l, p in zip(row["learned"], row["plain"])), (row["learned"], row["plain"])
