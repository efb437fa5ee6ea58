"""Learned correction of a coarse degree-1 DG solver.

A per-element network (60 -> 128 -> 128 -> 12, GELU, BF16 weights, FP32
accumulation; the library's own kernels) learns the modal tendency that the
coarse 72 x 36 degree-1 mesh misses, from pairs the method itself generates
with the degree-4 360 x 180 mesh:

    target = [P(u_fine(t + tau)) - Phi_coarse^tau(P(u_fine(t)))] / tau,

P the nested cos(theta)-weighted L2 projection (5 x 5 fine elements per
coarse element), Phi_coarse^tau one coarse SSP-RK3 step of size tau.  Inputs:
the 3 fields x 4 modes of the element and of its W, E, S, N neighbours (zeros
across a pole), normalised per feature with training statistics.  At run time
the network's output is added as a modal source in every stage (its h mode-0
part shifted to keep the total mass), and plain DG is the fallback.

Usage: python -m paper_2303_11767_gb300.learned --pairs 2000 --out result.json
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import dgswe, synth

COARSE = (72, 36, 1)
FINE = (360, 180, 4)
CFL_COARSE = 0.1
CFL_FINE = 0.3


def gather_inputs(u):
    """[nlat, nlon, 3, 4] coarse modal state -> [nlat*nlon, 60] network inputs
    (element, W, E, S, N; zeros across a pole)."""
    nlat, nlon = u.shape[:2]
    e = u.reshape(nlat, nlon, 12)
    w = np.roll(e, 1, axis=1)
    ea = np.roll(e, -1, axis=1)
    s = np.zeros_like(e)
    s[1:] = e[:-1]
    n = np.zeros_like(e)
    n[:-1] = e[1:]
    return np.concatenate([e, w, ea, s, n], axis=2).reshape(nlat * nlon, 60)


class Pair:
    def __init__(self, seed, spinup_s):
        self.fine = dgswe.Solver(*FINE, precision="fp32", check_finite=True)
        self.coarse = dgswe.Solver(*COARSE, precision="fp32", check_finite=True)
        self.fine.set_option(dgswe.OPT_STEPS_PER_GRAPH, 64)
        u0 = self.fine.project_grid(synth.SmoothField(seed).fields_grid)
        self.fine.set_state(u0)
        self.coarse.restrict_from(self.fine)
        self.tau = self.coarse.max_dt(CFL_COARSE)
        self.m = int(math.ceil(self.tau / self.fine.max_dt(CFL_FINE)))
        self.dt_fine = self.tau / self.m
        self.advance_fine(int(round(spinup_s / self.tau)))

    def advance_fine(self, coarse_steps):
        if coarse_steps > 0:
            self.fine.step(coarse_steps * self.m, self.dt_fine)

    def projected(self):
        self.coarse.restrict_from(self.fine)
        return self.coarse.get_state()

    def sample(self, k=1):
        """(inputs, target) of one pair starting at the current fine time:
        the mean tendency the coarse mesh misses over k coarse steps,
        [P(u_fine(t + k tau)) - Phi^k(P(u_fine(t)))] / (k tau)."""
        self.coarse.restrict_from(self.fine)
        u0 = self.coarse.get_state()
        self.coarse.step(k, self.tau)
        phi = self.coarse.get_state()
        self.advance_fine(k)
        u1 = self.projected()
        return gather_inputs(u0), ((u1 - phi) / (k * self.tau)).reshape(-1, 12)

    def close(self):
        self.fine.close()
        self.coarse.close()


def generate(n_pairs, seeds, spinup_s=1800.0, stride=4, target_steps=1, log=print):
    X, T = [], []
    per = int(math.ceil(n_pairs / len(seeds)))
    t0 = time.time()
    for seed in seeds:
        p = Pair(seed, spinup_s)
        for k in range(per):
            if len(X) >= n_pairs:
                break
            x, t = p.sample(target_steps)
            X.append(x)
            T.append(t)
            p.advance_fine(max(0, stride - target_steps))   # decorrelate consecutive pairs
        log(f"seed {seed}: {len(X)} pairs, tau {p.tau:.3f} s, {p.m} fine steps per tau, {time.time() - t0:.0f} s")
        p.close()
    return np.concatenate(X).astype(np.float32), np.concatenate(T).astype(np.float32)


def prolong(u, r, nf):
    """The modal state, on the mesh refined r x r with nf points per
    direction, of the same piecewise polynomial as the coarse state u
    [nlat, nlon, 3, nc^2] (nested meshes: a coarse polynomial restricted to a
    sub-element is one of degree nc - 1 <= nf - 1 there, so this is exact):
    per direction T[s][a_f][a_c] = int L_af(x) L_ac((x + 2s + 1)/r - 1) dx,
    exact with max(nf, nc) + 1 Gauss points."""
    from numpy.polynomial import legendre as npleg

    nlat, nlon, nfld, ncp = u.shape
    nc = int(round(math.sqrt(ncp)))
    x, w = npleg.leggauss(max(nf, nc) + 1)

    def L(k, t):
        c = np.zeros(k + 1)
        c[k] = 1.0
        return math.sqrt((2 * k + 1) / 2.0) * npleg.legval(t, c)

    T = np.array([[[np.sum(w * L(af, x) * L(ac, (x + 2 * sub + 1) / r - 1)) for ac in range(nc)] for af in range(nf)]
                  for sub in range(r)])
    uf = np.einsum("yBb,xAa,jifba->jyixfBA", T, T, u.reshape(nlat, nlon, nfld, nc, nc))
    return np.ascontiguousarray(uf.reshape(nlat * r, nlon * r, nfld, nf * nf))


def generate_local(n_pairs, seeds, spinup_s=1800.0, stride=8, target_steps=8, log=print):
    """Pairs whose inputs are states of the plain coarse trajectory and whose
    targets are the coarse scheme's own error over k coarse steps at that
    state: the fine mesh starts from the same piecewise polynomial (exact
    prolongation, `prolong`), both meshes advance k coarse steps and
        target = [P(Phi_fine^k(L u_c)) - Phi_coarse^k(u_c)] / (k tau).
    The network then sees at training the states it meets at run time (the
    coarse run's, not projections of the fine run's)."""
    X, T = [], []
    per = int(math.ceil(n_pairs / len(seeds)))
    t0 = time.time()
    r = FINE[0] // COARSE[0]
    for seed in seeds:
        p = Pair(seed, spinup_s)
        traj = dgswe.Solver(*COARSE, precision="fp32", check_finite=True)
        probe = dgswe.Solver(*COARSE, precision="fp32", check_finite=True)
        traj.set_state(p.projected())
        for _ in range(per):
            if len(X) >= n_pairs:
                break
            uc = traj.get_state()
            p.fine.set_state(prolong(uc, r, FINE[2] + 1))
            p.advance_fine(target_steps)
            u1 = p.projected()
            probe.set_state(uc)
            probe.step(target_steps, p.tau)
            X.append(gather_inputs(uc))
            T.append(((u1 - probe.get_state()) / (target_steps * p.tau)).reshape(-1, 12))
            traj.step(stride, p.tau)
        log(f"seed {seed}: {len(X)} pairs (coarse trajectory), {time.time() - t0:.0f} s")
        for x in (traj, probe):
            x.close()
        p.close()
    return np.concatenate(X).astype(np.float32), np.concatenate(T).astype(np.float32)


def row_statistics(T, nlon, nlat):
    """Per latitude row mean and std of the targets [n_samples, 12] (samples
    are whole coarse meshes in element order); stds floored at 1e-6 of the
    output's largest row std."""
    rows = (np.arange(T.shape[0]) % (nlon * nlat)) // nlon
    om = np.stack([T[rows == j].mean(0) for j in range(nlat)])
    sd = np.stack([T[rows == j].std(0) for j in range(nlat)])
    sd = np.maximum(sd, 1e-6 * sd.max(axis=0, keepdims=True) + 1e-30)
    return rows, om.astype(np.float32), sd.astype(np.float32)


def train(X, T, epochs=8, batch=4096, lr=1e-3, seed=0, log=print, row_norm=False, input_noise=0.0):
    """row_norm: targets normalised per latitude row (the coarse mesh's error
    depends on latitude, which the 60 inputs do not carry); the library then
    denormalises the network output with the row statistics.
    input_noise: every batch's inputs get fresh Gaussian noise of this many
    standard deviations per feature (targets unchanged), so the network also
    sees states off the projected-fine ones the corrected coarse run drifts
    into, and its output varies slowly across them."""
    import torch

    mlp = dgswe.MLP(60, 128, 12, seed=seed)
    in_mean, in_std = X.mean(0), X.std(0) + 1e-12
    rowstats = None
    if row_norm:
        rows, om, osd = row_statistics(T, COARSE[0], COARSE[1])
        T = ((T - om[rows]) / osd[rows]).astype(np.float32)
        out_mean, out_std = np.zeros(12, np.float32), np.ones(12, np.float32)
        rowstats = (om, osd)
    else:
        out_mean, out_std = T.mean(0), T.std(0) + 1e-30
    mlp.set_normalization(in_mean, in_std, out_mean, out_std)
    dX = torch.from_numpy(X).cuda()
    dT = torch.from_numpy(T).cuda()
    dstd = torch.from_numpy(in_std.astype(np.float32)).cuda()
    n = X.shape[0]
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    history = []
    steps = 0
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=g)
        losses = []
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            xb = dX.index_select(0, idx).contiguous()
            if input_noise > 0:
                xb = (xb + input_noise * dstd * torch.randn(xb.shape, device="cuda", generator=g)).contiguous()
            tb = dT.index_select(0, idx).contiguous()
            lr_k = lr * 0.5 * (1 + math.cos(math.pi * steps / max(1, epochs * (n // batch))))
            losses.append(mlp.train_step(xb, tb, lr_k))
            steps += 1
        history.append(float(np.mean(losses)))
        log(f"epoch {ep}: mean normalised MSE {history[-1]:.4f}")
    norm = {"in_mean": in_mean, "in_std": in_std, "out_mean": out_mean, "out_std": out_std}
    if rowstats is not None:
        mlp.set_row_normalization(*rowstats)
        norm.update(row_mean=rowstats[0], row_std=rowstats[1])
    return mlp, norm, history


def rel_l2(x, y):
    return [float(np.linalg.norm(x[..., f, :] - y[..., f, :]) / np.linalg.norm(y[..., f, :])) for f in range(3)]


def evaluate(mlp, seed, horizon_s, checkpoints=4, spinup_s=1800.0, log=print):
    """Plain and learned coarse runs from the projected fine state at the end
    of the spin-up, both compared with the projected fine run."""
    p = Pair(seed, spinup_s)
    u0 = p.projected()
    plain = dgswe.Solver(*COARSE, precision="fp32")
    learned = dgswe.Solver(*COARSE, precision="fp32")
    for s in (plain, learned):
        s.set_state(u0)
        s.set_option(dgswe.OPT_STEPS_PER_GRAPH, 64)
    learned.attach_mlp(mlp)
    nsteps = int(round(horizon_s / p.tau))
    out = []
    done = 0
    for c in range(1, checkpoints + 1):
        k = nsteps * c // checkpoints - done
        p.advance_fine(k)
        plain.step(k, p.tau)
        learned.step(k, p.tau)
        done += k
        ref = p.projected()
        row = {"hours": done * p.tau / 3600.0, "plain": rel_l2(plain.get_state(), ref),
               "learned": rel_l2(learned.get_state(), ref),
               "mass_drift_learned": (learned.total_mass() - plain.total_mass()) / plain.total_mass()}
        log(json.dumps(row))
        out.append(row)
    p.close()
    return out


def scaled_copy(mlp, norm, alpha):
    """A copy of a trained network whose learned source is alpha times the
    original (the output statistics scaled; same weights): shrinking a
    correction that overshoots."""
    c = dgswe.MLP(60, 128, 12, seed=0)
    c.set_params(mlp.get_params())
    c.set_normalization(norm["in_mean"], norm["in_std"], alpha * norm["out_mean"], alpha * norm["out_std"])
    if "row_mean" in norm:
        c.set_row_normalization(alpha * norm["row_mean"], alpha * norm["row_std"])
    return c


def parse_variant(spec):
    """'name[:key=value,...]' with keys noise (input noise), row_norm (0/1),
    alpha (shrinkage of the learned source), epochs."""
    name, _, rest = spec.partition(":")
    kw = {"noise": 0.0, "row_norm": 0, "alpha": 1.0, "epochs": None}
    for item in filter(None, rest.split(",")):
        k, v = item.split("=")
        if k not in kw:
            raise ValueError(f"unknown variant key {k}")
        kw[k] = float(v)
    return name, kw


def evaluate_many(mlps, seed, horizon_s, checkpoints=4, spinup_s=1800.0, log=print, checkpoint_hours=None):
    """evaluate() for several networks at once ({name: network}), against
    one fine reference run: plain coarse DG and one learned coarse solver per
    network, all from the projected fine state at the end of the spin-up.
    checkpoint_hours: explicit evaluation times (hours, increasing) instead
    of `checkpoints` equal intervals."""
    p = Pair(seed, spinup_s)
    u0 = p.projected()
    solvers = {"plain": dgswe.Solver(*COARSE, precision="fp32")}
    for name in mlps:
        solvers[name] = dgswe.Solver(*COARSE, precision="fp32")
    for name, s in solvers.items():
        s.set_state(u0)
        s.set_option(dgswe.OPT_STEPS_PER_GRAPH, 64)
        if name != "plain":
            s.attach_mlp(mlps[name])
    nsteps = int(round(horizon_s / p.tau))
    if checkpoint_hours:
        marks = [int(round(h * 3600.0 / p.tau)) for h in checkpoint_hours]
    else:
        marks = [nsteps * c // checkpoints for c in range(1, checkpoints + 1)]
    out = []
    done = 0
    diverged = set()   # learned solvers whose state stopped being physical (h <= 0 or non-finite)
    for mark in marks:
        k = mark - done
        p.advance_fine(k)
        for name, s in solvers.items():
            if name in diverged:
                continue
            try:
                s.step(k, p.tau)
            except dgswe.DGError:
                if name == "plain":
                    raise
                diverged.add(name)
        done += k
        ref = p.projected()
        m_plain = solvers["plain"].total_mass()
        row = {"hours": done * p.tau / 3600.0}
        for name, s in solvers.items():
            if name in diverged:
                row[name] = [float("nan")] * 3
                continue
            row[name] = rel_l2(s.get_state(), ref)
            if name != "plain":
                row["mass_drift_" + name] = (s.total_mass() - m_plain) / m_plain
        log(json.dumps(row))
        out.append(row)
    for s in solvers.values():
        s.close()
    p.close()
    return out


def select_alpha(mlp, norm, alphas, seed, hours, log=print):
    """The shrinkage of the learned source chosen on a validation seed: every
    alpha is evaluated against one fine reference run of `seed` at `hours`,
    and the alpha with the smallest mean log ratio of its relative L2 error
    to plain coarse DG over the three fields wins (ratios below 1 = a gain).
    Returns (alpha, the validation row)."""
    nets = {f"a{a}": (mlp if a == 1.0 else scaled_copy(mlp, norm, a)) for a in alphas}
    row = evaluate_many(nets, seed, hours * 3600.0, checkpoint_hours=[hours], log=log)[-1]
    score = {a: float(np.mean([math.log(e / p) for e, p in zip(row[f"a{a}"], row["plain"])])) for a in alphas}
    best = min(alphas, key=lambda a: score[a])
    return best, {"row": row, "score": score}


def main_alpha(args):
    """Train one network, choose the shrinkage alpha on the validation seed,
    then evaluate every alpha (the chosen one marked) on the held-out test
    seed against one fine reference run, at the checkpoint times."""
    t0 = time.time()
    gen = generate_local if args.local_targets else generate
    X, T = gen(args.pairs, args.train_seeds, stride=args.stride, target_steps=args.target_steps)
    t_gen = time.time() - t0
    mlp, norm, hist = train(X, T, epochs=args.epochs, row_norm=args.row_norm)
    t_train = time.time() - t0 - t_gen
    alphas = [float(a) for a in args.alphas.split(",")]
    best, val = select_alpha(mlp, norm, alphas, args.val_seed, args.val_hours)
    print(f"validation seed {args.val_seed}, {args.val_hours} h: alpha = {best}", json.dumps(val["score"]), flush=True)
    t_val = time.time() - t0 - t_gen - t_train
    nets = {f"a{a}": (mlp if a == 1.0 else scaled_copy(mlp, norm, a)) for a in alphas}
    hours = [float(h) for h in args.checkpoint_hours.split(",")] if args.checkpoint_hours else None
    ev = evaluate_many(nets, args.test_seed, args.horizon_hours * 3600.0, checkpoint_hours=hours)
    res = {"pairs": args.pairs, "samples": int(X.shape[0]), "train_seeds": args.train_seeds,
           "target_steps": args.target_steps, "stride": args.stride, "epochs": args.epochs,
           "targets": "coarse-trajectory local error" if args.local_targets else "projected fine run",
           "alphas": alphas, "val_seed": args.val_seed, "val_hours": args.val_hours, "alpha_selected": best,
           "validation": val, "test_seed": args.test_seed, "loss_history": hist, "evaluation": ev,
           "seconds": {"generate": t_gen, "train": t_train, "validate": t_val,
                       "evaluate": time.time() - t0 - t_gen - t_train - t_val}}
    with open(args.out, "w") as fh:
        json.dump(res, fh, indent=1)
    if args.params_out:
        np.savez(args.params_out, params=mlp.get_params(), alpha=best, **norm)
    print(json.dumps(res["evaluation"][-1]))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=2000)
    ap.add_argument("--train-seeds", type=int, nargs="+", default=[5000, 5001, 5002, 5003])
    ap.add_argument("--test-seed", type=int, default=6000)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--target-steps", type=int, default=1, help="coarse steps the target averages over")
    ap.add_argument("--stride", type=int, default=4, help="coarse steps between pairs")
    ap.add_argument("--horizon-hours", type=float, default=12.0)
    ap.add_argument("--out", default="learned_result.json")
    ap.add_argument("--params-out", default="")
    ap.add_argument("--row-norm", action="store_true", help="normalise the targets per latitude row")
    ap.add_argument("--variant", action="append", default=[],
                    help="name[:noise=s,row_norm=0|1,alpha=a,epochs=e]; several variants are trained on the "
                         "same pairs and evaluated against one fine reference run")
    ap.add_argument("--alphas", default="", help="comma-separated shrinkages of the learned source; the one "
                                                  "used is chosen on --val-seed")
    ap.add_argument("--val-seed", type=int, default=6001)
    ap.add_argument("--val-hours", type=float, default=3.0)
    ap.add_argument("--checkpoint-hours", default="", help="comma-separated evaluation times (hours)")
    ap.add_argument("--local-targets", action="store_true",
                    help="inputs from the plain coarse trajectory, targets its own k-step error (generate_local)")
    args = ap.parse_args()
    if args.variant:
        return main_variants(args)
    if args.alphas:
        return main_alpha(args)
    t0 = time.time()
    X, T = generate(args.pairs, args.train_seeds, stride=args.stride, target_steps=args.target_steps)
    t_gen = time.time() - t0
    mlp, norm, hist = train(X, T, epochs=args.epochs, row_norm=args.row_norm)
    t_train = time.time() - t0 - t_gen
    ev = evaluate(mlp, args.test_seed, args.horizon_hours * 3600.0)
    res = {"pairs": args.pairs, "samples": int(X.shape[0]), "train_seeds": args.train_seeds,
           "target_steps": args.target_steps, "stride": args.stride, "row_norm": args.row_norm,
           "test_seed": args.test_seed, "epochs": args.epochs, "loss_history": hist, "evaluation": ev,
           "seconds": {"generate": t_gen, "train": t_train, "evaluate": time.time() - t0 - t_gen - t_train}}
    with open(args.out, "w") as fh:
        json.dump(res, fh, indent=1)
    if args.params_out:
        np.savez(args.params_out, params=mlp.get_params(), **norm)
    print(json.dumps(res["evaluation"][-1]))


def main_variants(args):
    """Train every --variant on one set of pairs and evaluate them all
    against one fine reference run (evaluate_many)."""
    t0 = time.time()
    X, T = generate(args.pairs, args.train_seeds, stride=args.stride, target_steps=args.target_steps)
    t_gen = time.time() - t0
    trained, mlps, hist = {}, {}, {}
    for spec in args.variant:
        name, kw = parse_variant(spec)
        key = (kw["noise"], kw["row_norm"], kw["epochs"])
        if key not in trained:     # variants that differ only in alpha share one network
            trained[key] = train(X, T, epochs=int(kw["epochs"] or args.epochs), row_norm=bool(kw["row_norm"]),
                                 input_noise=kw["noise"], log=lambda s: None)
        mlp, norm, h = trained[key]
        mlps[name] = mlp if kw["alpha"] == 1.0 else scaled_copy(mlp, norm, kw["alpha"])
        hist[name] = h
        print(name, kw, "loss", ["%.4f" % v for v in h], flush=True)
    t_train = time.time() - t0 - t_gen
    ev = evaluate_many(mlps, args.test_seed, args.horizon_hours * 3600.0)
    res = {"pairs": args.pairs, "samples": int(X.shape[0]), "train_seeds": args.train_seeds,
           "target_steps": args.target_steps, "stride": args.stride, "test_seed": args.test_seed,
           "variants": args.variant, "loss_history": hist, "evaluation": ev,
           "seconds": {"generate": t_gen, "train": t_train, "evaluate": time.time() - t0 - t_gen - t_train}}
    with open(args.out, "w") as fh:
        json.dump(res, fh, indent=1)
    print(json.dumps(res["evaluation"][-1]))


if __name__ == "__main__":
    main()
