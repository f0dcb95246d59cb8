"""Train the candidate scorer on LP dwell-time labels from seeded procedural
rooms, then evaluate the proposal against the plain method on held-out rooms.

Run from the repository root (it uses the seeded room generator in synth/):
    python -m paper_2103_14137_gb300.train_scorer --rooms 48 --eval-rooms 8 \
        --out paper_2103_14137_gb300/data/scorer.npz --report scorer_report.json

Training jobs: rooms 10000 + r of the uneven-room generator, three random
lamp designs each, at most --cap candidates; targets from the relaxed LP (Eq. (9))
over every patch, solved by row generation: the efficiency of each candidate
at the LP's dual prices (label_of).
Evaluation: rooms 100 + r (the batched benchmark's rooms), designs 1, 5 and 9, all
their candidates.  For each job the plain LP (all candidates) and the reduced
LP (the kept candidates) give dwell times whose coverage at MU_MIN is
measured over every patch with the exact matrix; lost coverage is the drop,
added dwell the relative increase of sum t.  A job whose fallback probe loses
more than LOST_MAX of its lit area runs on all candidates.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np
import torch

from . import _build, uvc
from .lp import MU_MIN, support
from .proposal import (KEEP, LOST_MAX, LP_PATCHES, PROBE, Scorer, coverage_of, dwell_rowgen, features, label_of,
                       probe_columns, save, train)


def _synth():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from synth.batched import POWER, batched_room, design_candidates, designs
    from synth.scenes import line_lamp
    return batched_room, design_candidates, designs, line_lamp, POWER


def _scene(room, dev):
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    return uvc.build_scene(T(room.verts), T(room.tris), T(room.centroid), T(room.normal), T(room.area),
                           T(room.excl)), T


def _job(sc, T, room, cand, lamp, seed):
    """Exact matrix, probe split and scorer features of one (room, design)."""
    cd = T(cand)
    A, _ = uvc.irradiance_matrix(sc, cd, uvc.Lamp(lamp.offsets, lamp.weights, lamp.power))
    area = T(np.asarray(room.area, np.float32))
    probe, half = probe_columns(room.np_, seed)
    pi = torch.from_numpy(probe).to(A.device)
    Ap = A.index_select(1, pi).contiguous()
    ap = area.index_select(0, pi).contiguous()
    feat = features(sc, cd, Ap[:, :half], ap[:half])
    return {"scene": sc, "A": A, "area": area, "seed": seed, "cand": cd, "feat": feat,
            "check": (Ap[:, half:], ap[half:]), "sketch": Ap[:, :half]}


def _label_settings(cap):
    """Everything a chunk's features and labels depend on besides its rooms:
    the settings, and the source of the room generator, the proposal and the
    LP (any edit there invalidates the cache)."""
    import hashlib
    from . import proposal as prop
    from .lp import T_MAX
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    h = hashlib.sha256()
    for rel in ("synth/batched.py", "synth/mesh.py", "synth/scenes.py", "paper_2103_14137_gb300/proposal.py",
                "paper_2103_14137_gb300/lp.py"):
        with open(os.path.join(root, rel), "rb") as f:
            h.update(f.read())
    return {"cap": int(cap), "probe": prop.PROBE, "lp_patches": prop.LP_PATCHES, "lp_add": prop.LP_ADD,
            "lp_rounds": prop.LP_ROUNDS, "mu_min": MU_MIN, "t_max": T_MAX, "features": int(uvc.FEATURES),
            "probe_features": int(uvc.PROBE_FEATURES), "code": h.hexdigest()[:16]}


def _chunk_path(cache, r0, r1):
    return os.path.join(cache, f"train_rooms_{10000 + r0}-{10000 + r1 - 1}.npz")


def save_chunk(cache, r0, r1, cap, feats, ys, etas, sups, lp_s):
    """Write one chunk of solved training jobs (rooms r0..r1-1) to the cache
    directory, atomically, with the settings they were made under."""
    os.makedirs(cache, exist_ok=True)
    n = np.array([len(f) for f in feats], np.int64)
    path = _chunk_path(cache, r0, r1)
    tmp = f"{path}.{os.getpid()}.tmp.npz"
    np.savez_compressed(tmp, settings=json.dumps(_label_settings(cap)), n=n,
                        feat=np.concatenate(feats).astype(np.float32), y=np.concatenate(ys).astype(np.float32),
                        eta=np.concatenate(etas).astype(np.float32), support=np.concatenate(sups).astype(bool),
                        lp_s=np.asarray(lp_s, np.float64))
    os.replace(tmp, path)


def load_chunk(cache, r0, r1, cap):
    """The cached chunk of rooms r0..r1-1 as per-job lists, or None when it is
    missing or was made under other settings."""
    path = _chunk_path(cache, r0, r1) if cache else None
    if not path or not os.path.exists(path):
        return None
    z = np.load(path)
    if json.loads(str(z["settings"])) != _label_settings(cap):
        return None
    cut = np.cumsum(z["n"])[:-1]
    split = lambda a: list(np.split(a, cut))  # noqa: E731
    return split(z["feat"]), split(z["y"]), split(z["eta"]), split(z["support"]), list(z["lp_s"])


def training_data(n_rooms, cap, dev, workers, log, chunk=12, cache=None):
    """Features and LP labels of the training jobs, chunk by chunk of rooms.
    With `cache` (a directory) every solved chunk is written there and a
    chunk found there under the same settings is read instead of solved, so an
    interrupted run resumes at its first unsolved chunk."""
    batched_room, design_candidates, designs, line_lamp, POWER = _synth()
    D = designs()
    feats, ys, lp_s, etas, sups = [], [], [], [], []
    for c0 in range(0, n_rooms, chunk):
        c1 = min(n_rooms, c0 + chunk)
        hit = load_chunk(cache, c0, c1, cap)
        if hit is not None:
            f, y, e, sp, ls = hit
            feats += f
            ys += y
            etas += e
            sups += sp
            lp_s += ls
            log(f"training rooms {c0}..{c1 - 1}: {len(f)} jobs read from {cache}")
            continue
        n_before = len(feats)
        jobs, scenes = [], []
        for r in range(c0, min(n_rooms, c0 + chunk)):
            seed = 10000 + r
            room = batched_room(seed)
            sc, T = _scene(room, dev)
            scenes.append(sc)
            rng = np.random.default_rng(seed)
            for d in rng.choice(len(D), 3, replace=False):
                h, L, K = D[d]
                cand = design_candidates(room, h, L, min(room.info["targets"][2], cap), seed=seed * 16 + int(d))
                jobs.append(_job(sc, T, room, cand, line_lamp(L, K, POWER), seed * 16 + int(d)))
                feats.append(jobs[-1]["feat"].cpu().numpy())
        t0 = time.perf_counter()
        sols = dwell_rowgen(jobs, workers, log=log)
        for t, mu, secs, rounds, rows, eta in sols:
            ys.append(label_of(eta, t))
            etas.append(eta.astype(np.float32))
            sups.append(support(t))
            lp_s.append(secs)
        log(f"training rooms {c0}..{c0 + len(scenes) - 1}: {len(jobs)} jobs, LPs {time.perf_counter() - t0:.1f} s, "
            f"rows {np.mean([x[4] for x in sols]):.0f} mean")
        if cache:
            save_chunk(cache, c0, c1, cap, feats[n_before:], ys[n_before:], etas[n_before:], sups[n_before:],
                       lp_s[n_before:])
        del jobs, sols
        for sc in scenes:
            sc.free()
        torch.cuda.empty_cache()
    return feats, ys, lp_s, etas, sups


def evaluate(scorer, n_rooms, dev, workers, log, design_ids=(1, 5, 9), mark=True):
    batched_room, design_candidates, designs, line_lamp, POWER = _synth()
    D = designs()
    jobs, scenes, meta = [], [], []
    for r in range(n_rooms):
        seed = 100 + r
        room = batched_room(seed)
        sc, T = _scene(room, dev)
        scenes.append(sc)
        for d in design_ids:
            h, L, K = D[d]
            cand = design_candidates(room, h, L, room.info["targets"][2], seed=seed * 16 + d)
            j = _job(sc, T, room, cand, line_lamp(L, K, POWER), seed * 16 + d)
            idx, _ = scorer.select(j["feat"], j["cand"], A_sketch=j["sketch"] if mark else None)
            lost = float(uvc.probe_lost(j["check"][0], idx, j["check"][1]).item())
            keep = idx.cpu().numpy()
            jobs.append(j)
            meta.append({"room": seed, "design": d, "nc": int(cand.shape[0]), "np": int(room.np_),
                         "kept": int(keep.size), "probe_lost": lost, "fallback": bool(lost > LOST_MAX),
                         "_keep": keep})
        log(f"evaluation room {r}: nt={room.nt} np={room.np_}")
    full = [dict(j, rows=None) for j in jobs]
    red = [dict(j, rows=m["_keep"]) for j, m in zip(jobs, meta)]
    t0 = time.perf_counter()
    sols = dwell_rowgen(full + red, workers, log=log)
    log(f"evaluation LPs {time.perf_counter() - t0:.1f} s")
    n = len(jobs)
    for k, (j, m) in enumerate(zip(jobs, meta)):
        t_full, mu_full, s_full, r_full, rows_full, eta_full = sols[k]
        t_red, mu_red, s_red, r_red, rows_red, _ = sols[n + k]
        if m["fallback"]:
            t_red, mu_red = t_full, mu_full
        lit = (j["A"] > 0).any(0)
        cf, cr = coverage_of(j["area"], mu_full), coverage_of(j["area"], mu_red)
        supp = support(t_full)
        m.update({"coverable": coverage_of(j["area"], lit.float() * MU_MIN), "cov_full": cf, "cov_kept": cr,
                  "lost_coverage": max(0.0, cf - cr), "dwell_full": float(t_full.sum()),
                  "dwell_kept": float(t_red.sum()),
                  "added_dwell": float(t_red.sum() / max(t_full.sum(), 1e-30) - 1.0), "support": int(supp.sum()),
                  "support_recall": float(np.isin(np.flatnonzero(supp), m["_keep"]).mean()) if supp.any() else 1.0,
                  "eta_kept_mean": float(np.clip(eta_full, 0, 1)[m["_keep"]].mean()),
                  "eta_top_mean": float(np.sort(np.clip(eta_full, 0, 1))[::-1][:len(m["_keep"])].mean()),
                  "lp_s": [round(s_full, 2), round(s_red, 2)], "lp_rows": [rows_full, rows_red],
                  "lp_rounds": [r_full, r_red]})
        m.pop("_keep")
    del jobs, full, red, sols
    for sc in scenes:
        sc.free()
    return meta


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--rooms", type=int, default=48)
    ap.add_argument("--eval-rooms", type=int, default=8)
    ap.add_argument("--cap", type=int, default=1200, help="candidates per training job at most")
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--out", default=None)
    ap.add_argument("--load", default=None, help="evaluate these weights instead of training")
    ap.add_argument("--report", default=None)
    ap.add_argument("--save-data", default=None, help="write the training features and labels (.npz)")
    ap.add_argument("--no-mark", action="store_true", help="select by score alone (no best-source marking)")
    ap.add_argument("--cache", default=None,
                    help="directory for solved training chunks (written as they finish, reused on a rerun)")
    a = ap.parse_args(argv)
    dev = torch.device("cuda", 0)
    _build.build()
    t_start = time.perf_counter()
    log = lambda m: print(f"[{time.perf_counter() - t_start:7.1f}s] {m}", flush=True)  # noqa: E731
    report = {"keep": KEEP, "probe": PROBE, "lost_max": LOST_MAX, "lp_patches": LP_PATCHES}
    if a.load:
        scorer = Scorer.load(a.load)
    else:
        feats, ys, lp_s, etas, sups = training_data(a.rooms, a.cap, dev, a.workers, log, cache=a.cache)
        X, y = np.concatenate(feats), np.concatenate(ys)
        if a.save_data:
            np.savez_compressed(a.save_data, X=X.astype(np.float32), y=y, eta=np.concatenate(etas),
                                support=np.concatenate(sups),
                                job=np.concatenate([np.full(len(f), i) for i, f in enumerate(feats)]))
        flat, hist = train(X, y, steps=a.steps, lr=a.lr)
        log(f"trained on {X.shape[0]} candidates (target mean {y.mean():.4f}): loss {hist[0]:.4f} -> {hist[-1]:.4f}")
        report.update({"train_rooms": a.rooms, "train_candidates": int(X.shape[0]),
                       "train_support": int(np.concatenate(sups).sum()),
                       "loss_first": hist[0], "loss_last": hist[-1], "train_lp_s_mean": float(np.mean(lp_s))})
        if a.out:
            save(a.out, flat, rooms=a.rooms, steps=a.steps)
        scorer = Scorer(flat)
    jobs = evaluate(scorer, a.eval_rooms, dev, a.workers, log, mark=not a.no_mark)
    report["mark_best"] = not a.no_mark
    lost = np.array([j["lost_coverage"] for j in jobs])
    added = np.array([j["added_dwell"] for j in jobs])
    report.update({"eval_jobs": len(jobs), "lost_coverage_mean": float(lost.mean()), "lost_coverage_max": float(lost.max()),
                   "added_dwell_mean": float(added.mean()), "added_dwell_max": float(added.max()),
                   "fallback_rate": float(np.mean([j["fallback"] for j in jobs])),
                   "support_recall_mean": float(np.mean([j["support_recall"] for j in jobs])), "jobs": jobs})
    summary = {k: v for k, v in report.items() if k != "jobs"}
    print(json.dumps(summary), flush=True)
    if a.report:
        with open(a.report, "w") as f:
            json.dump(report, f, indent=1)
    scorer.close()


if __name__ == "__main__":
    main()
