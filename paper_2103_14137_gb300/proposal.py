"""Learned candidate proposal: score every candidate lamp position with the
BF16 perceptron (uvc_mlp_*) on its features, keep the best fraction
(uvc_select_top), and evaluate the irradiance matrix only there.

Features per candidate (IN_DIM = 114): the 66 scene features of
uvc_candidate_features (distance histogram to the patches, clearance, height)
and the 48-cell visibility sketch of uvc_probe_features, taken from the
irradiance of all candidates on one half of a probe sample of PROBE of the
patches.  The other half of the probe is the fallback check: if the kept
candidates leave more than LOST_MAX of the area lit there dark
(uvc_probe_lost), the job runs on all candidates.  Whatever the scores, the
best source of every sketch patch is kept, and every source of a sketch
patch that at most a fraction RARE_FRAC of the candidates light (uvc_mark_best).

The scorer learns which candidates the relaxed LP of Sec. IV-D (Eq. (9))
gives a non-zero dwell time; the plain method - every candidate, exact matrix,
the same LP - stays the fallback and the referee.  Training and the evaluation are
host orchestration of library calls plus the host LP (lp.py).
"""
from __future__ import annotations

import math
import os

import numpy as np
import torch

from . import uvc
from .lp import MU_MIN, T_MAX, patch_sample, solve_job, support

KEEP = 0.2              # fraction of candidates kept
PROBE = 0.01            # fraction of patches in the probe (half sketch, half fallback check)
LOST_MAX = 0.0025       # check area lit by all candidates but dark for the kept ones -> fallback
RARE_FRAC = 0.01        # sketch patches lit by at most this fraction of the candidates keep all their sources
GROUP = 1               # > 1: also keep the best of every GROUP consecutive (neighbouring) candidates
HIDDEN = 256
IN_DIM = uvc.FEATURES + uvc.PROBE_FEATURES
LP_PATCHES = 1000       # initial LP rows; row generation adds the violated patches
LP_ADD = 1500           # violated patches added per round
LP_ROUNDS = 4
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "scorer.npz")


def rare_count(nc: int) -> int:
    return max(3, int(math.ceil(RARE_FRAC * nc)))


def keep_count(nc: int, keep: float = KEEP) -> int:
    return min(nc, max(1, int(math.ceil(keep * nc)))) if nc > 0 else 0


def probe_columns(np_: int, seed: int, frac: float = PROBE):
    """Probe patch indices ordered (sketch half, check half): a seeded sample of
    frac of the patches, alternate members going to each half."""
    s = patch_sample(np_, max(2, int(round(frac * np_))), seed)
    return np.concatenate([s[0::2], s[1::2]]), (s.size + 1) // 2


def features(scene, cand, A_sketch, area_sketch, feat=None, work=None, stream=None):
    """(nc, IN_DIM) scorer input in one row-major buffer."""
    nc = cand.shape[0]
    if feat is None:
        feat = torch.empty((nc, IN_DIM), dtype=torch.float32, device=cand.device)
    uvc.candidate_features(scene, cand, feat=feat[:, :uvc.FEATURES], stream=stream)
    uvc.probe_features(A_sketch, area_sketch, feat=feat[:, uvc.FEATURES:], work=work, stream=stream)
    return feat


def fold_standardisation(flat, mean, std, in_dim, hidden):
    """Parameters that take raw features: W1'[r] = W1[r] / std_r,
    b1' = b1 - sum_r mean_r / std_r W1[r]."""
    P = (in_dim + 15) // 16 * 16
    f = np.asarray(flat, np.float64).copy()
    W1 = f[:P * hidden].reshape(P, hidden)
    b1 = f[P * hidden:P * hidden + hidden]
    W1[:in_dim] /= std[:, None]
    b1 -= mean @ W1[:in_dim]
    return f.astype(np.float32)


class Scorer:
    """The trained perceptron with its input standardisation folded in."""

    def __init__(self, flat, in_dim=IN_DIM, hidden=HIDDEN, max_batch=1 << 16):
        self.flat = np.asarray(flat, np.float32)
        self.in_dim, self.hidden = in_dim, hidden
        self.mlp = uvc.Mlp(in_dim, hidden, max_batch=max_batch)
        self.mlp.set_params(self.flat)

    @classmethod
    def load(cls, path=WEIGHTS, max_batch=1 << 16):
        z = np.load(path)
        return cls(z["params"], int(z["in_dim"]), int(z["hidden"]), max_batch=max_batch)

    def close(self):
        self.mlp.close()

    def scores(self, feat, out=None, stream=None):
        return self.mlp.forward(feat, logit=out, stream=stream)

    def select(self, feat, cand, A_sketch=None, keep: float = KEEP, score=None, stream=None):
        """(idx, kept candidates): the best source of every sketch patch
        (A_sketch, if given), then the best-scoring candidate of every group
        of GROUP neighbours, then the best scores, keep-fraction in all,
        ascending index."""
        score = self.scores(feat, out=score, stream=stream)
        if GROUP > 1:
            uvc.group_boost(score, GROUP, stream=stream)
        if A_sketch is not None:
            uvc.mark_best(A_sketch, score, rare=rare_count(cand.shape[0]), stream=stream)
        return uvc.select_top(score, keep_count(cand.shape[0], keep), cand=cand, stream=stream)


def label_of(eta, t):
    """Training target in [0, 1]: the LP efficiency eta (1 on the dwell-time
    support), sharpened so that near-substitutes of the chosen candidates
    stand out from the bulk: y = clip(eta, 0, 1)^8, and 1 where t_k > 0."""
    y = np.clip(np.asarray(eta, np.float64), 0.0, 1.0) ** 8
    y[support(t)] = 1.0
    return y.astype(np.float32)


def train(X, y, hidden=HIDDEN, steps=3000, lr=1e-3, batch=4096, seed=0, device="cuda"):
    """Fit the scorer to features X (N, d) and targets y (N,) in [0, 1]
    (cross-entropy with soft targets, the two ends weighted to balance);
    returns (folded parameters, history of losses)."""
    X = np.asarray(X, np.float64)
    y = np.asarray(y, np.float32)
    mean, std = X.mean(0), X.std(0)
    std = np.where(std > 1e-12, std, 1.0)
    Xs = ((X - mean) / std).astype(np.float32)
    pi = float(np.clip(y.mean(), 1e-6, 1 - 1e-6))
    cpos, cneg = 0.5 / pi, 0.5 / (1 - pi)          # weight w = y cpos + (1 - y) cneg
    B = min(batch, X.shape[0])
    m = uvc.Mlp(X.shape[1], hidden, max_batch=B, seed=seed)
    Xd = torch.from_numpy(Xs).to(device)
    yd = torch.from_numpy(y).to(device)
    wd = torch.from_numpy((y * cpos + (1 - y) * cneg).astype(np.float32) / B).to(device)
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    for s in range(steps):
        idx = torch.randint(0, X.shape[0], (B,), generator=g).to(device)
        loss = m.train_step(Xd[idx].contiguous(), yd[idx].contiguous(), wd[idx].contiguous(),
                            lr * (0.1 ** (s / steps)))
        if s % 100 == 0 or s == steps - 1:
            hist.append(float(loss.item()))
    flat = m.params()
    m.close()
    return fold_standardisation(flat, mean, std, X.shape[1], hidden), hist


def save(path, flat, in_dim=IN_DIM, hidden=HIDDEN, **meta):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    np.savez(path, params=np.asarray(flat, np.float32), in_dim=in_dim, hidden=hidden,
             **{k: np.asarray(v) for k, v in meta.items()})


def solve_many(jobs, workers: int):
    """Solve LP jobs [(A_rows, area)] in `workers` spawned processes."""
    args = [(A, a, MU_MIN, T_MAX) for A, a in jobs]
    if workers <= 1 or len(args) <= 1:
        return [solve_job(x) for x in args]
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(solve_job, args, chunksize=1)


def dwell_rowgen(problems, workers: int, rounds: int = LP_ROUNDS, add: int = LP_ADD, log=None):
    """Eq. (9) over every patch by row generation.  problems: dicts with the
    device matrix `A` (nc, np), `rows` (candidate indices used, or None for
    all), `area` (np,) device, `seed`.  Each round solves the LP on the current
    patch rows, computes the fluence of every patch with the exact matrix, and
    adds the most under-dosed patches that the rows can light.  Returns, per
    problem, (t over the rows, the fluence, LP seconds, rounds, rows, eta
    over the rows: the efficiency at the final LP's dual prices)."""
    state = []
    for p in problems:
        A = p["A"] if p.get("rows") is None else p["A"].index_select(
            0, torch.as_tensor(p["rows"], device=p["A"].device).long())
        lit = (A > 0).any(0)
        cols = patch_sample(A.shape[1], LP_PATCHES, p["seed"])
        state.append({"A": A.contiguous(), "lit": lit, "cols": cols, "secs": 0.0, "rounds": 0, "done": False,
                      "scene": p["scene"]})
    area_h = [p["area"].double().cpu().numpy() for p in problems]
    for r in range(rounds):
        todo = [k for k, s in enumerate(state) if not s["done"]]
        if not todo:
            break
        jobs = []
        for k in todo:
            s = state[k]
            ci = torch.from_numpy(s["cols"]).to(s["A"].device)
            jobs.append((s["A"].index_select(1, ci).double().cpu().numpy(), area_h[k][s["cols"]]))
        sols = solve_many(jobs, workers)
        for k, (t, secs, eta) in zip(todo, sols):
            s = state[k]
            s["t"], s["eta"], s["secs"], s["rounds"] = t, eta, s["secs"] + secs, r + 1
            tt = torch.from_numpy(t.astype(np.float32)).to(s["A"].device)[None, :].contiguous()
            s["mu"] = uvc.fluence(s["scene"], s["A"], tt)[0]
            short = (s["mu"] < MU_MIN * (1 - 1e-4)) & s["lit"]
            short[torch.from_numpy(s["cols"]).to(short.device).long()] = False
            n_short = int(short.sum().item())
            if n_short == 0 or r == rounds - 1:
                s["done"] = True
                s["short_left"] = n_short
                continue
            ratio = torch.where(short, s["mu"] / MU_MIN, torch.full_like(s["mu"], 2.0))
            newc = torch.topk(ratio, min(add, n_short), largest=False).indices.cpu().numpy()
            s["cols"] = np.union1d(s["cols"], newc)
        if log:
            log(f"row generation round {r + 1}: {len(todo)} LPs, "
                f"{sum(1 for s in state if not s['done'])} still short")
    return [(s["t"], s["mu"], s["secs"], s["rounds"], int(s["cols"].size), s["eta"]) for s in state]


def coverage_of(area, mu, lit=None):
    """Area fraction with fluence >= MU_MIN (of all patches, or of `lit`)."""
    ok = (mu >= MU_MIN)
    a = area.double()
    if lit is not None:
        return float((a * ok).sum().item() / max((a * lit).sum().item(), 1e-30))
    return float((a * ok).sum().item() / a.sum().item())


__all__ = ["KEEP", "PROBE", "LOST_MAX", "HIDDEN", "IN_DIM", "LP_PATCHES", "WEIGHTS", "Scorer", "train", "save",
           "keep_count", "rare_count", "probe_columns", "features", "label_of", "fold_standardisation", "solve_many", "dwell_rowgen",
           "coverage_of", "support"]
