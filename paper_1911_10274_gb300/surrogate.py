"""Surrogate-screened morphology search for actuated voxel robots.

The paper's asynchronous design exists so that optimisation (topology and
actuation, Sec. III-F; many agents in parallel, Sec. I) can run alongside the
simulation.  This module closes that loop on the GPU:

* morphologies: an 8 x 8 x 8 voxel grid, Bernoulli(0.6) occupancy, largest
  26-connected component, one mass per voxel, 26-neighbourhood springs; each
  voxel carries a phase and every spring the mean of its two voxels'
  sinusoidal signals (amplitude 0.1, 2 Hz);
* fitness: the robot's centroid x-displacement after a rollout on the ground,
  simulated by the batched persistent kernels (``titan.Batch``);
* surrogate: an MLP on the tcgen05 tensor cores (``titan.MLP``) mapping the
  1024 features (occupancy bits, then per-voxel phases scaled to [-1, 1), 0
  where empty) to the standardised fitness, trained with Adam on simulated
  rollouts;
* search: a (mu + lambda) mutation search.  The plain form simulates every
  mutant; the screened form lets the surrogate rank all mutants and simulates
  only the top few, whose simulated fitness (the simulator has the final say)
  decides who survives; those simulated mutants also refine the network
  (online fine-tuning on a window of the latest simulated mutants, or all of
  them, mirror-augmented), because a network trained only on random robots
  ranks nearby mutants poorly.  A random pick of the same size is the
  ablation.

Python here only orchestrates: every rollout and every network product runs
in the library's kernels.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Tuple

import numpy as np

from . import inputs
from . import titan as T

GRID = 8
N_FEATURES = 2 * GRID ** 3


@dataclasses.dataclass
class Morph:
    occ: np.ndarray      # (8, 8, 8) bool, (z, y, x)
    phase: np.ndarray    # (8, 8, 8) float, radians (only occupied voxels matter)


def random_morph(rng: np.random.Generator, p: float = 0.6) -> Morph:
    occ = inputs.voxel_morphology(rng, GRID, p)
    return Morph(occ=occ, phase=rng.uniform(0.0, 2.0 * np.pi, (GRID,) * 3))


def robot(m: Morph, freq: float = 2.0) -> inputs.System:
    return inputs.voxel_robot(m.occ, m.phase, amp=0.1, freq=freq)


def encode(morphs: List[Morph]) -> np.ndarray:
    """(n, 1024) float32: occupancy bits, then phases scaled to [-1, 1) (0 where empty)."""
    X = np.zeros((len(morphs), N_FEATURES), np.float32)
    for i, m in enumerate(morphs):
        o = m.occ.ravel()
        X[i, :GRID ** 3] = o
        X[i, GRID ** 3:] = np.where(o, m.phase.ravel() / np.pi - 1.0, 0.0)
    return X


def mirrored(morphs: List[Morph], y: np.ndarray):
    """Exact symmetries of the task: reflecting a robot through x -> -x negates
    its centroid x-displacement (ground, gravity and friction are symmetric);
    reflecting y -> -y leaves it unchanged.  Returns the 4x augmented set."""
    out_m, out_y = [], []
    for m, f in zip(morphs, y):
        for fx in (False, True):
            for fy in (False, True):
                occ, ph = m.occ, m.phase
                if fx:
                    occ, ph = occ[:, :, ::-1], ph[:, :, ::-1]
                if fy:
                    occ, ph = occ[:, ::-1, :], ph[:, ::-1, :]
                out_m.append(Morph(occ=np.ascontiguousarray(occ), phase=np.ascontiguousarray(ph)))
                out_y.append(-f if fx else f)
    return out_m, np.array(out_y)


def mirrored_encoded(X: np.ndarray, y: np.ndarray):
    """encode(mirrored(morphs, y)) from encode(morphs): the same four
    reflections, rows in the same order (for each robot: as is, y -> -y,
    x -> -x, both), formed on the encoded grids instead of re-encoding."""
    n = len(X)
    V = X.reshape(n, 2, GRID, GRID, GRID)          # (occupancy, phase) blocks, (z, y, x)
    out = np.empty((n, 4) + V.shape[1:], X.dtype)
    out[:, 0] = V
    out[:, 1] = V[:, :, :, ::-1, :]
    out[:, 2] = V[:, :, :, :, ::-1]
    out[:, 3] = V[:, :, :, ::-1, ::-1]
    yy = np.repeat(np.asarray(y, np.float64), 4).reshape(n, 4)
    yy[:, 2:] *= -1.0
    return out.reshape(4 * n, X.shape[1]), yy.ravel()


def fitness(morphs: List[Morph], steps: int, freq: float = 2.0, chunk: int = 4096,
            device: int = 0) -> np.ndarray:
    """Centroid x-displacement of each robot after `steps` steps (simulated)."""
    out = np.empty(len(morphs))
    for s in range(0, len(morphs), chunk):
        robots = [robot(m, freq) for m in morphs[s:s + chunk]]
        x0 = np.array([r.pos[:, 0].mean() for r in robots])
        with T.Batch(robots, device=device) as b:
            b.rollout(steps)
            c = b.centroids()
        out[s:s + chunk] = c[:, 0].astype(np.float64) - x0
    return out


def mutate(rng: np.random.Generator, m: Morph, flip_mean: float = 1.5, phase_prob: float = 0.15,
           phase_sigma: float = 1.0) -> Morph:
    """Toggles 1 + Poisson(flip_mean) voxels, perturbs some phases, keeps the
    largest connected component (at least 8 voxels)."""
    for _ in range(20):
        occ = m.occ.copy()
        phase = m.phase.copy()
        for _ in range(1 + rng.poisson(flip_mean)):
            z, y, x = rng.integers(0, GRID, 3)
            if not occ[z, y, x]:
                phase[z, y, x] = rng.uniform(0.0, 2.0 * np.pi)
            occ[z, y, x] = not occ[z, y, x]
        jig = rng.random((GRID,) * 3) < phase_prob
        phase = np.where(jig, np.mod(phase + rng.normal(0.0, phase_sigma, phase.shape), 2.0 * np.pi), phase)
        occ = inputs.largest_component(occ)
        if occ.sum() >= 8:
            return Morph(occ=occ, phase=phase)
    return m


class Surrogate:
    """The tensor-core MLP plus target standardisation."""

    def __init__(self, hidden: int = 512, seed: int = 0, device: int = 0):
        import torch
        self.torch = torch
        self.net = T.MLP(N_FEATURES, hidden, seed=seed, device=device)
        self.device = device
        self.mu, self.sd = 0.0, 1.0

    def _x(self, X):
        """BF16 features on the device (a tensor already there is taken as is)."""
        if isinstance(X, self.torch.Tensor):
            return X
        return self.torch.as_tensor(X, dtype=self.torch.float32, device=f"cuda:{self.device}").bfloat16()

    def fit(self, X: np.ndarray, y: np.ndarray, epochs: int = 20, batch: int = 4096, lr: float = 1e-3,
            seed: int = 0) -> List[float]:
        torch = self.torch
        self.mu, self.sd = float(y.mean()), float(y.std() + 1e-12)
        yt = (y - self.mu) / self.sd
        n = (len(X) // 128) * 128
        batch = min(batch, n)
        batch -= batch % 128
        rng = np.random.default_rng(seed)
        Xd = self._x(X)
        yd = torch.as_tensor(yt, dtype=torch.float32, device=f"cuda:{self.device}")
        loss = torch.empty(1, device=f"cuda:{self.device}")
        hist = []
        for _ in range(epochs):
            perm = torch.as_tensor(rng.permutation(len(X)), device=f"cuda:{self.device}")
            for s in range(0, n - batch + 1, batch):
                idx = perm[s:s + batch]
                self.net.train_step(Xd[idx].contiguous(), yd[idx].contiguous(), lr, loss)
            self.net.sync()
            hist.append(float(loss))
        return hist

    def refine(self, X: np.ndarray, y: np.ndarray, epochs: int = 3, batch: int = 1024, lr: float = 5e-4,
               seed: int = 0) -> None:
        """Continues training on (X, y) keeping the target standardisation."""
        torch = self.torch
        n = (len(X) // 128) * 128
        if n == 0:
            return
        batch = max(128, min(batch, n) - min(batch, n) % 128)
        rng = np.random.default_rng(seed)
        Xd = self._x(X)
        yd = torch.as_tensor((y - self.mu) / self.sd, dtype=torch.float32, device=f"cuda:{self.device}")
        loss = torch.empty(1, device=f"cuda:{self.device}")
        for _ in range(epochs):
            perm = torch.as_tensor(rng.permutation(len(X)), device=f"cuda:{self.device}")
            for s in range(0, n - batch + 1, batch):
                idx = perm[s:s + batch]
                self.net.train_step(Xd[idx].contiguous(), yd[idx].contiguous(), lr, loss)
        self.net.sync()

    def predict(self, X: np.ndarray) -> np.ndarray:
        torch = self.torch
        n = len(X)
        pad = (-n) % 128
        Xp = np.concatenate([X, np.zeros((pad, X.shape[1]), X.dtype)]) if pad else X
        x = self._x(Xp)
        y = torch.empty(len(Xp), device=f"cuda:{self.device}")
        self.net.forward(x, y)
        return y.cpu().numpy()[:n].astype(np.float64) * self.sd + self.mu


class Ensemble:
    """Several surrogates that differ in their initial weights and each see
    their own bootstrap resample of the training set.  Their spread measures
    how far a candidate lies from anything they were trained on, which a
    single network's point prediction cannot show; predict() returns the
    screening score mean + kappa * std (an upper confidence bound), so a
    mutant the members disagree on is simulated rather than discarded."""

    def __init__(self, members: int = 5, hidden: int = 512, seed: int = 0, device: int = 0, kappa: float = 1.0):
        self.members = [Surrogate(hidden=hidden, seed=seed * 1000 + k, device=device) for k in range(members)]
        self.kappa = float(kappa)
        self.seed = seed

    def _boot(self, n: int, k: int, salt: int) -> np.ndarray:
        return np.random.default_rng([self.seed, k, salt]).integers(0, n, n)

    def fit(self, X: np.ndarray, y: np.ndarray, epochs: int = 20, batch: int = 4096, lr: float = 1e-3,
            seed: int = 0) -> List[float]:
        out = []
        for k, m in enumerate(self.members):
            idx = self._boot(len(X), k, seed)
            out.append(m.fit(X[idx], y[idx], epochs=epochs, batch=batch, lr=lr, seed=seed + k)[-1])
        return out

    def refine(self, X: np.ndarray, y: np.ndarray, epochs: int = 3, batch: int = 1024, lr: float = 5e-4,
               seed: int = 0) -> None:
        Xd = self.members[0]._x(X)               # uploaded once, each member's resample taken on the device
        for k, m in enumerate(self.members):
            idx = self._boot(len(X), k, 7919 + seed)
            sel = m.torch.as_tensor(idx, device=Xd.device)
            m.refine(Xd[sel], y[idx], epochs=epochs, batch=batch, lr=lr, seed=seed + k)

    def predict_stats(self, X: np.ndarray):
        P = np.stack([m.predict(X) for m in self.members])
        return P.mean(axis=0), P.std(axis=0)

    def predict(self, X: np.ndarray) -> np.ndarray:
        mu, sd = self.predict_stats(X)
        return mu + self.kappa * sd

    def get_state(self):
        return [(m.net.get_params(), m.mu, m.sd) for m in self.members]

    def set_state(self, state) -> None:
        for m, (p, mu, sd) in zip(self.members, state):
            m.net.set_params(p)
            m.mu, m.sd = mu, sd


def spearman(a, b) -> float:
    ra = np.argsort(np.argsort(a))
    rb = np.argsort(np.argsort(b))
    return float(np.corrcoef(ra, rb)[0, 1])


def search(mode: str, start: List[Morph], start_fit: np.ndarray, generations: int, mutants: int, screened: int,
           steps: int, seed: int = 0, surrogate: Optional[Surrogate] = None, parents: int = 16,
           freq: float = 2.0, refine_epochs: int = 2, target: Optional[float] = None,
           max_rollouts: Optional[int] = None, refine_window: int = 8192) -> dict:
    """(mu + lambda) search from a simulated starting population.

    mode 'plain': simulate all mutants; 'surrogate': simulate the `screened`
    mutants the surrogate ranks highest, then refine the surrogate on the last
    `refine_window` mutants simulated (0: all of them; mirror-augmented); 'random': simulate
    `screened` random mutants.  Stops after `generations`, or once the best simulated
    fitness reaches `target`, or when `max_rollouts` would be exceeded.
    Returns the best fitness after each generation with the simulator rollouts
    spent so far (the starting population is not counted)."""
    rng = np.random.default_rng(seed)
    order = np.argsort(-start_fit)[:parents]
    pop = [start[i] for i in order]
    pop_fit = start_fit[order].copy()
    best, used, hist = float(pop_fit[0]), 0, []
    seen_X, seen_y = np.zeros((0, N_FEATURES), np.float32), np.zeros(0)   # encoded, mirrored
    gains = []
    for g in range(generations):
        if target is not None and best >= target:
            break
        n_sim = mutants if mode == "plain" else screened
        if max_rollouts is not None and used + n_sim > max_rollouts:
            break
        kids = [mutate(rng, pop[k % len(pop)]) for k in range(mutants)]
        if mode == "plain":
            chosen = kids
        elif mode == "surrogate":
            pred = surrogate.predict(encode(kids))
            chosen = [kids[i] for i in np.argsort(-pred)[:screened]]
        else:
            chosen = [kids[i] for i in rng.choice(len(kids), screened, replace=False)]
        f = fitness(chosen, steps, freq)
        used += len(chosen)
        gains.append(float(f.mean() - pop_fit.mean()))
        if mode == "surrogate":
            # each simulated mutant is encoded (and mirrored) once, when simulated
            Xn, yn = mirrored_encoded(encode(chosen), f)
            seen_X = np.concatenate([seen_X, Xn])
            seen_y = np.concatenate([seen_y, yn])
            if refine_window > 0:
                seen_X, seen_y = seen_X[-4 * refine_window:], seen_y[-4 * refine_window:]
            surrogate.refine(seen_X, seen_y, epochs=refine_epochs, batch=512, seed=g)
        allm = pop + chosen
        allf = np.concatenate([pop_fit, f])
        keep = np.argsort(-allf)[:parents]
        pop = [allm[i] for i in keep]
        pop_fit = allf[keep]
        best = max(best, float(pop_fit[0]))
        hist.append((used, best))
    return {"history": hist, "best": best, "rollouts": used, "generations": len(hist),
            "mean_offspring_gain": float(np.mean(gains)) if gains else None}


def best_at(history, rollouts: int) -> Optional[float]:
    """Best fitness a search had found once it had spent at most `rollouts`."""
    got = [b for used, b in history if used <= rollouts]
    return got[-1] if got else None


def thin(history, points: int = 40):
    """At most `points` evenly spaced (rollouts, best) pairs of a history."""
    if len(history) <= points:
        return [list(h) for h in history]
    idx = np.unique(np.linspace(0, len(history) - 1, points).round().astype(int))
    return [list(history[i]) for i in idx]


def rollouts_to_reach(history, target: float) -> Optional[int]:
    for used, best in history:
        if best >= target:
            return used
    return None


def main(argv=None):
    """Full-scale run: python -m paper_1911_10274_gb300.surrogate [--train N] [--steps S] ...

    Trains on N random robots, runs the plain search for --generations, then
    runs the screened search and its random-screening ablation until each
    reaches the plain search's best fitness, within the plain search's rollout
    budget; prints the rollouts each needed."""
    import argparse
    import json
    import os
    import time
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=200_000)
    ap.add_argument("--steps", type=int, default=10_000)
    ap.add_argument("--generations", type=int, default=100)
    ap.add_argument("--mutants", type=int, default=1024)
    ap.add_argument("--screened", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--search-seed", type=int, default=None, help="seed of the searches (default: seed + 1)")
    ap.add_argument("--refine-epochs", type=int, default=2)
    ap.add_argument("--refine-window", type=int, default=8192, help="simulated mutants refined on; 0: all")
    ap.add_argument("--no-random", action="store_true", help="skip the random-screening ablation")
    ap.add_argument("--screened-budget", type=int, default=0,
                    help="rollout cap of the screened searches; 0: the plain search's own rollouts")
    ap.add_argument("--fitness-cache", default=None,
                    help="npz file holding the training robots' simulated fitness (written if absent)")
    ap.add_argument("--search-seeds", default=None,
                    help="comma-separated search seeds: run every arm once per seed from the same trained "
                         "networks and report rollouts-to-plain-best per seed (one JSON line per seed, then a summary)")
    ap.add_argument("--ensemble", type=int, default=0, help="also run the ensemble-screened arm with this many members")
    ap.add_argument("--kappa", type=float, default=1.0, help="ensemble screening score: mean + kappa * std")
    ap.add_argument("--no-single", action="store_true", help="skip the single-network screened arm")
    a = ap.parse_args(argv)
    if a.search_seeds:
        return multi_seed(a)
    rng = np.random.default_rng(a.seed)
    t0 = time.time()
    morphs = [random_morph(rng) for _ in range(a.train)]
    key = f"{a.seed}-{a.train}-{a.steps}"
    y = None
    if a.fitness_cache and os.path.exists(a.fitness_cache):
        d = np.load(a.fitness_cache)
        if str(d["key"]) == key:
            y = d["y"]
    cached = y is not None
    if y is None:
        y = fitness(morphs, a.steps)
        if a.fitness_cache:
            np.savez(a.fitness_cache, key=key, y=y)
    t_sim = time.time() - t0
    n_val = max(128, a.train // 10)
    sur = Surrogate(seed=a.seed)
    t1 = time.time()
    am, ay = mirrored(morphs[:-n_val], y[:-n_val])
    sur.fit(encode(am), ay, epochs=a.epochs)
    t_fit = time.time() - t1
    val_corr = spearman(sur.predict(encode(morphs[-n_val:])), y[-n_val:])
    start, start_fit = morphs[-n_val:], y[-n_val:]
    t2 = time.time()
    sseed = a.seed + 1 if a.search_seed is None else a.search_seed
    plain = search("plain", start, start_fit, a.generations, a.mutants, a.screened, a.steps, seed=sseed)
    target = plain["best"]
    budget = plain["rollouts"] if a.screened_budget <= 0 else min(plain["rollouts"], a.screened_budget)
    t3 = time.time()
    big = 10 ** 9
    scr = search("surrogate", start, start_fit, big, a.mutants, a.screened, a.steps, seed=sseed,
                 surrogate=sur, target=target, max_rollouts=budget, refine_epochs=a.refine_epochs,
                 refine_window=a.refine_window)
    t4 = time.time()
    rnd = {"history": [], "best": None, "rollouts": 0, "generations": 0, "mean_offspring_gain": None}
    if not a.no_random:
        rnd = search("random", start, start_fit, big, a.mutants, a.screened, a.steps, seed=sseed,
                     target=target, max_rollouts=budget)
    t5 = time.time()
    out = {"train_rollouts": a.train, "steps": a.steps, "fitness_cached": cached, "simulate_s": t_sim,
           "search_seed": sseed, "refine_epochs": a.refine_epochs, "refine_window": a.refine_window,
           "fit_s": t_fit, "val_spearman": val_corr,
           "plain": {"best": target, "rollouts": plain["rollouts"], "generations": plain["generations"],
                     "s": t3 - t2},
           "screened_budget": budget,
           "surrogate": {"best": scr["best"], "rollouts_to_plain_best": rollouts_to_reach(scr["history"], target),
                         "rollouts": scr["rollouts"], "generations": scr["generations"],
                         "mean_offspring_gain": scr["mean_offspring_gain"], "s": t4 - t3,
                         "plain_best_at_same_rollouts": best_at(plain["history"], scr["rollouts"]),
                         "plain_rollouts_to_this_best": rollouts_to_reach(plain["history"], scr["best"])},
           "random": {"best": rnd["best"], "rollouts_to_plain_best": rollouts_to_reach(rnd["history"], target),
                      "rollouts": rnd["rollouts"], "generations": rnd["generations"],
                      "mean_offspring_gain": rnd["mean_offspring_gain"], "s": t5 - t4,
                      "plain_best_at_same_rollouts": best_at(plain["history"], rnd["rollouts"]),
                      "plain_rollouts_to_this_best": rollouts_to_reach(plain["history"], rnd["best"])
                      if rnd["best"] is not None else None},
           "curves": {k: thin(v["history"]) for k, v in (("plain", plain), ("surrogate", scr), ("random", rnd))}}
    print(json.dumps(out))
    return out


def _train_set(a):
    """The random training robots, their simulated fitness (cached in
    a.fitness_cache when given) and the wall time spent simulating."""
    import os
    import time
    rng = np.random.default_rng(a.seed)
    t0 = time.time()
    morphs = [random_morph(rng) for _ in range(a.train)]
    key = f"{a.seed}-{a.train}-{a.steps}"
    y = None
    if a.fitness_cache and os.path.exists(a.fitness_cache):
        d = np.load(a.fitness_cache)
        if str(d["key"]) == key:
            y = d["y"]
    if y is None:
        y = fitness(morphs, a.steps)
        if a.fitness_cache:
            np.savez(a.fitness_cache, key=key, y=y)
    return morphs, y, time.time() - t0


def multi_seed(a):
    """Every arm (plain, single-network screened, ensemble screened, random
    pick) once per search seed, all from the same trained networks (their
    parameters restored before each search), each screened arm capped at the
    plain search's rollouts.  Prints one JSON line per seed and a summary with
    the median rollouts-to-plain-best of each arm (None counts as not reached)."""
    import json
    import time
    morphs, y, t_sim = _train_set(a)
    n_val = max(128, a.train // 10)
    am, ay = mirrored(morphs[:-n_val], y[:-n_val])
    Xtr = encode(am)
    start, start_fit = morphs[-n_val:], y[-n_val:]
    t1 = time.time()
    single = None
    if not a.no_single:
        single = Surrogate(seed=a.seed)
        single.fit(Xtr, ay, epochs=a.epochs)
        single_state = (single.net.get_params(), single.mu, single.sd)
    ens = None
    if a.ensemble > 0:
        ens = Ensemble(members=a.ensemble, seed=a.seed, kappa=a.kappa)
        ens.fit(Xtr, ay, epochs=a.epochs)
        ens_state = ens.get_state()
    t_fit = time.time() - t1
    val = {}
    Xval = encode(start)
    if single is not None:
        val["single_spearman"] = spearman(single.predict(Xval), start_fit)
    if ens is not None:
        mu, sd = ens.predict_stats(Xval)
        val["ensemble_mean_spearman"] = spearman(mu, start_fit)
        val["ensemble_ucb_spearman"] = spearman(mu + a.kappa * sd, start_fit)
    big = 10 ** 9
    rows = []
    for sseed in [int(x) for x in a.search_seeds.split(",")]:
        t2 = time.time()
        plain = search("plain", start, start_fit, a.generations, a.mutants, a.screened, a.steps, seed=sseed)
        target, budget = plain["best"], plain["rollouts"]
        arms = {"plain": {"best": target, "rollouts": budget, "rollouts_to_plain_best":
                          rollouts_to_reach(plain["history"], target), "s": time.time() - t2}}
        todo = []
        if single is not None:
            todo.append(("single", single, single_state))
        if ens is not None:
            todo.append(("ensemble", ens, ens_state))
        todo.append(("random", None, None))
        for name, model, state in todo:
            t3 = time.time()
            if name == "single":
                model.net.set_params(state[0])
                model.mu, model.sd = state[1], state[2]
            elif name == "ensemble":
                model.set_state(state)
            r = search("random" if model is None else "surrogate", start, start_fit, big, a.mutants, a.screened,
                       a.steps, seed=sseed, surrogate=model, target=target, max_rollouts=budget,
                       refine_epochs=a.refine_epochs, refine_window=a.refine_window)
            arms[name] = {"best": r["best"], "rollouts": r["rollouts"],
                          "rollouts_to_plain_best": rollouts_to_reach(r["history"], target),
                          "plain_best_at_same_rollouts": best_at(plain["history"], r["rollouts"]),
                          "s": time.time() - t3}
        row = {"search_seed": sseed, "arms": arms}
        rows.append(row)
        print(json.dumps(row), flush=True)

    def med(name):
        v = [r["arms"][name]["rollouts_to_plain_best"] for r in rows if name in r["arms"]]
        v = [x if x is not None else float("inf") for x in v]
        return float(np.median(v)) if v else None

    summary = {"summary": True, "train_rollouts": a.train, "steps": a.steps, "simulate_s": t_sim, "fit_s": t_fit,
               "mutants": a.mutants, "screened": a.screened, "generations": a.generations,
               "ensemble": a.ensemble, "kappa": a.kappa, "refine_window": a.refine_window,
               "validation": val, "seeds": [r["search_seed"] for r in rows],
               "median_rollouts_to_plain_best": {k: med(k) for k in rows[0]["arms"]} if rows else {}}
    print(json.dumps(summary), flush=True)
    return {"rows": rows, "summary": summary}


if __name__ == "__main__":
    main()
