"""Design-space exploration with a learned surrogate.

Simulating every candidate RANC configuration exactly is what makes design
sweeps take hours to weeks (Sec. I); here a small network predicts, from a
configuration's parameters, two outcomes measured by the exact simulator:

* spike traffic: packets delivered per sample, relative to the nominal design;
* output agreement: the fraction of samples whose output-bus class (argmax of
  the output counts, lowest id on ties) equals the nominal design's class.

Flow: simulate a seeded training set of design points on the GPU, many at
once in one multi-network handle (ranc_create_multi: the design-sweep runner,
one tick launch for every point of a chunk), train the surrogate with the
library's own kernels (include/ranc_mlp.h: tensor-core products, bf16
weights, fp32 accumulation, Adam), score many seeded candidates with it, and
simulate only the best-ranked ones exactly, again side by side.  The exact simulator has the
last word: reported gains compare re-simulated results of the surrogate's choice
with an equally sized random choice.  PyTorch only holds device buffers.
"""

import time

import numpy as np

from ranc_workloads import dse as D

from . import ranc
from .mlp import MLP

TRAFFIC_WEIGHT = 0.2
HIDDEN = (128, 128, 128)


def argmax_lowest(counts):
    return np.argmax(counts, axis=1)  # numpy returns the first maximum: the lowest id


def objective(agreement, rel_traffic):
    """Higher is better: agree with the nominal design while sending fewer packets."""
    return agreement - TRAFFIC_WEIGHT * rel_traffic


class Evaluator:
    """Exact simulation of design points on fixed seeded inputs, up to
    `chunk_cores` cores of points at a time in one multi-network handle."""

    def __init__(self, n_samples=256, window=32, seed=0x5EEDD5E, chunk_cores=12000):
        self.master = D.Master(seed)
        self.x = D.prototype_inputs(seed, n_samples, 16)
        self.window = window
        self.n = n_samples
        self.chunk_cores = chunk_cores
        self.sim_seconds = 0.0
        self.n_sims = 0
        self.launches = 0
        (counts, packets), = self.simulate([D.NOMINAL])
        self.ref_class = argmax_lowest(counts)
        self.ref_packets = max(packets, 1.0)

    def simulate(self, points):
        """[(output counts [S, 10], packets per sample)] of every point."""
        res = []
        k = 0
        while k < len(points):
            nets, cores = [], 0
            while k < len(points) and (not nets or cores + 20 * points[k].replicas <= self.chunk_cores):
                nets.append(D.build(self.master, points[k]))
                cores += nets[-1].n_cores
                k += 1
            sim = ranc.MultiSim(nets, self.n)
            l0 = ranc.ranc_launch_count(sim.h)
            counts = sim.run_samples(self.x, self.window)
            self.launches += ranc.ranc_launch_count(sim.h) - l0
            packets = sim.counters()[:, 1].astype(np.float64) / self.n
            sim.close()
            res.extend(zip(counts, packets))
        return res

    def targets(self, points):
        """[n, 2]: (agreement, relative traffic) per point."""
        out = np.zeros((len(points), 2), np.float64)
        t0 = time.perf_counter()
        for k, (counts, packets) in enumerate(self.simulate(points)):
            out[k, 0] = float(np.mean(argmax_lowest(counts) == self.ref_class))
            out[k, 1] = packets / self.ref_packets
        self.sim_seconds += time.perf_counter() - t0
        self.n_sims += len(points)
        return out


def features(points):
    """[n, N_FEATURES] float32, row i = points[i].features() (formed column by column)."""
    col = lambda name: np.array([getattr(p, name) for p in points], dtype=np.float64)
    rep, neu, wb, nt = col("replicas"), col("neurons"), col("weight_bits"), col("n_types")
    cols = [rep / D.R_MAX, neu == 256, wb == 4, wb == 6, wb == 9, nt == 4, col("density"),
            np.log2(col("thr_scale")) / 2 + 0.5, col("leak_max") / 8, col("delay_max") / 15]
    out = np.stack([np.asarray(c, dtype=np.float64).astype(np.float32) for c in cols], axis=1)
    return out.reshape(len(points), D.N_FEATURES)


class Surrogate:
    def __init__(self, seed=1, max_batch=256):
        self.mlp = MLP((D.N_FEATURES,) + HIDDEN + (2,), max_batch, seed=seed)
        self.max_batch = max_batch
        self.mu = np.zeros(2)
        self.sd = np.ones(2)

    def fit(self, X, Y, steps=3000, lr=2e-3, seed=2):
        import torch
        self.mu, self.sd = Y.mean(axis=0), Y.std(axis=0) + 1e-6
        Yn = ((Y - self.mu) / self.sd).astype(np.float32)
        dx = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        dy = torch.from_numpy(np.ascontiguousarray(Yn)).cuda()
        g = np.random.default_rng(seed)
        n = X.shape[0]
        bs = min(self.max_batch, n)
        losses = []
        for s in range(steps):
            idx = torch.from_numpy(g.choice(n, size=bs, replace=False)).cuda()
            xb, yb = dx[idx].contiguous(), dy[idx].contiguous()
            want = s % 100 == 0 or s == steps - 1
            loss, _ = self.mlp.loss_backward(xb.data_ptr(), yb.data_ptr(), bs) if want else (None, None)
            if not want:
                self.mlp.loss_backward(xb.data_ptr(), yb.data_ptr(), bs)
            else:
                losses.append(loss)
            self.mlp.adam_step(lr=lr * (0.1 ** (s / steps)))
        torch.cuda.synchronize()
        return losses

    def predict(self, X):
        """One copy of all rows to the device, forward passes of max_batch
        rows on consecutive slices, one copy back."""
        import torch
        n, f = X.shape
        dx = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
        dy = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        for a in range(0, n, self.max_batch):
            b = min(self.max_batch, n - a)
            self.mlp.forward(dx.data_ptr() + a * f * 4, b, dy.data_ptr() + a * 2 * 4)
        torch.cuda.synchronize()
        return dy.cpu().numpy() * self.sd + self.mu


def spearman(a, b):
    from scipy.stats import spearmanr
    return float(spearmanr(a, b).correlation)


def explore(n_train=512, n_val=128, n_candidates=20000, top_k=64, seed=11, steps=3000, n_samples=256,
            evaluator=None, rounds=1, surrogate=None):
    """Train on simulated points, rank candidates, re-simulate the top_k and
    a random top_k; returns a report dict.

    With rounds > 1 the search is refined: after each round the re-simulated
    candidates join the training set, a new surrogate is trained on all of
    them and the top_k candidates not simulated yet are simulated next.  The
    random baseline then gets the same budget (rounds * top_k exact
    simulations).  `evaluator` (an Evaluator) and `surrogate` (a factory
    taking a seed, default Surrogate) can be replaced."""
    ev = evaluator or Evaluator(n_samples=n_samples)
    make = surrogate or (lambda sd: Surrogate(seed=sd))
    pts = D.sample_points(seed, n_train + n_val)
    Y = ev.targets(pts)
    X = features(pts)
    sur = make(1)
    t0 = time.perf_counter()
    losses = sur.fit(X[:n_train], Y[:n_train], steps=steps)
    train_s = time.perf_counter() - t0
    Yv = sur.predict(X[n_train:])
    mae = np.abs(Yv - Y[n_train:]).mean(axis=0)
    rho_val = spearman(objective(Yv[:, 0], Yv[:, 1]), objective(Y[n_train:, 0], Y[n_train:, 1]))
    cand = D.sample_points(seed + 1, n_candidates)
    Xc = features(cand)
    t0 = time.perf_counter()
    pred = sur.predict(Xc)
    rank_s = time.perf_counter() - t0
    score = objective(pred[:, 0], pred[:, 1])
    top = np.argsort(-score, kind="stable")[:top_k]
    rnd_all = np.random.default_rng(seed + 2).choice(n_candidates, size=min(n_candidates, rounds * top_k),
                                                     replace=False)
    rnd = rnd_all[:top_k]
    Yt = ev.targets([cand[i] for i in top])
    Yr = ev.targets([cand[i] for i in rnd])
    true_top, true_rnd = objective(Yt[:, 0], Yt[:, 1]), objective(Yr[:, 0], Yr[:, 1])
    history = [dict(mean=float(true_top.mean()), best=float(true_top.max()),
                    spearman_pred_vs_true=spearman(score[top], true_top))]
    chosen, Ych = list(top), [Yt]
    for r in range(1, rounds):
        Xr = np.concatenate([X[:n_train], Xc[chosen]])
        Yrr = np.concatenate([Y[:n_train]] + Ych)
        sur_r = make(1 + r)
        sur_r.fit(Xr, Yrr, steps=steps)
        pr = sur_r.predict(Xc)
        sc = objective(pr[:, 0], pr[:, 1])
        sc[chosen] = -np.inf  # simulated already
        nxt = np.argsort(-sc, kind="stable")[:top_k]
        Yn = ev.targets([cand[i] for i in nxt])
        tn = objective(Yn[:, 0], Yn[:, 1])
        history.append(dict(mean=float(tn.mean()), best=float(tn.max()), spearman_pred_vs_true=spearman(sc[nxt], tn)))
        chosen += list(nxt)
        Ych.append(Yn)
    rep = dict(
        n_train=n_train, n_val=n_val, n_candidates=n_candidates, top_k=top_k, train_steps=steps,
        final_train_loss=losses[-1], val_mae_agreement=float(mae[0]), val_mae_rel_traffic=float(mae[1]),
        val_spearman_objective=rho_val,
        top_true_objective_mean=float(true_top.mean()), random_true_objective_mean=float(true_rnd.mean()),
        top_true_objective_best=float(true_top.max()), random_true_objective_best=float(true_rnd.max()),
        gain_mean=float(true_top.mean() - true_rnd.mean()),
        spearman_top_pred_vs_true=history[0]["spearman_pred_vs_true"],
        rounds=rounds)
    if rounds > 1:
        Ya = ev.targets([cand[i] for i in rnd_all[top_k:]])
        true_all = np.concatenate([true_rnd, objective(Ya[:, 0], Ya[:, 1])])
        found = objective(np.concatenate(Ych)[:, 0], np.concatenate(Ych)[:, 1])
        rep.update(round_history=history, refined_best=float(found.max()),
                   refined_top_mean=float(np.sort(found)[-top_k:].mean()),
                   random_best_same_budget=float(true_all.max()),
                   random_top_mean_same_budget=float(np.sort(true_all)[-top_k:].mean()),
                   exact_sims_by_search=rounds * top_k)
    rep.update(sims=ev.n_sims, sim_seconds=ev.sim_seconds, seconds_per_sim=ev.sim_seconds / max(ev.n_sims, 1),
               sim_kernel_launches=ev.launches, train_seconds=train_s, rank_seconds=rank_s,
               exact_sims_saved=n_candidates - rounds * top_k)
    return rep
