"""Parameter sweep of the 2D buoyant bubble rise on the batched solver.

Each sweep point (Eo, Bi, channel width W, elasticity E0, bulk
concentration C0; D = 32) is one instance of a batch.  The batch is stepped
for a fixed number of steps; every `sample_every` steps the diagnostics of
every instance are read: the rise velocity U_v of the red region (Eqs. 33-34)
and its aspect ratio (horizontal over vertical extent from the second
moments).  The terminal values are the means over the last `window` fraction
of the samples, and their relative spread over that window is kept as a
steadiness measure.  Terminal Reynolds number: Re = rho^B0 |U_v| D_eff /
mu^B0 with D_eff the diameter of the red region's area (Sec. 3.4 scales).

The surrogate (paper_2311_15242_gb300.surrogate) is trained on these
results; plain single-instance solves (`plain=True`) are its judge and its
fallback.

  python -m paper_2311_15242_gb300.sweep --n 512 --seed 1 --steps 30000 --out train.npz
"""
import argparse
import os
import sys
import time

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)
import workloads as W  # noqa: E402  (seeded sweep points and initial fields)

FEATURES = ("Eo", "Bi", "W_over_D", "E0", "C0")
TARGETS = ("Re", "AR")


def features(pt, D_b=32.0):
    return [pt["Eo"], pt["Bi"], pt["width"] / D_b, pt["E0"], pt["C0"]]


def _terminal(series, window):
    s = np.asarray(series, dtype=np.float64)
    k = max(1, int(round(len(s) * window)))
    w = s[-k:]
    mean = float(np.mean(w))
    spread = float(np.std(w) / max(abs(mean), 1e-30))
    return mean, spread


def summarise(history, window):
    """Terminal (Re, AR) and their spreads from per-sample diagnostics."""
    re, re_s = _terminal([h["Re"] for h in history], window)
    ar, ar_s = _terminal([h["aspect_ratio"] for h in history], window)
    return re, ar, re_s, ar_s


def run_batch(cfgs, steps, sample_every, storage="f32", window=0.25, seed=0, log=None):
    """Step the instances as one batch; returns per-instance (Re, AR,
    spreads) and the device throughput (MLUPS, excluding diagnostics).  An
    instance whose solve diverges is taken out of the batch and reported as
    NaN."""
    from . import Batch, autotune
    from .lbs import LBS_EDIVERGED
    import torch
    b = Batch(cfgs, storage=storage)
    for k, c in enumerate(cfgs):
        f = W.initial_fields(c, seed=seed + k)
        b.init_fields(k, f["phi"], f["psi"], f["C"], f["u"])
    autotune.tune(b, [c["nx"] for c in cfgs])
    hist = [[] for _ in cfgs]
    failed = set()
    noconv = 0
    cells = sum(c["nx"] * c["ny"] for c in cfgs)
    dev_ms = 0.0
    done = 0
    while done < steps:
        n = min(sample_every, steps - done)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        b.step(n)
        e1.record(b.stream)
        e1.synchronize()
        dev_ms += e0.elapsed_time(e1)
        done += n
        for k, code in enumerate(b.status()):
            if code == LBS_EDIVERGED and k not in failed:
                failed.add(k)
                b.set_active(k, False)
            elif code:
                noconv += 1  # a solve that hit the SOR round limit (kept)
        for k, d in enumerate(b.diagnostics()):
            hist[k].append(d)
        if log:
            log(f"batch of {len(cfgs)}: step {done}/{steps}, {len(failed)} diverged, "
                f"{noconv} SOR round limits")
    b.close()
    nan = (float("nan"),) * 4
    out = [nan if k in failed else summarise(h, window) for k, h in enumerate(hist)]
    return out, cells * steps / (dev_ms / 1e3) / 1e6


def run_plain(cfg, steps, sample_every, storage="f32", window=0.25, seed=0):
    """One plain single-instance solve of a sweep point."""
    from . import Solver
    from .lbs import LBS_EDIVERGED, LBS_ENOCONV, LbsError
    s = Solver(cfg, storage=storage)
    f = W.initial_fields(cfg, seed=seed)
    s.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    hist = []
    done = 0
    try:
        while done < steps:
            n = min(sample_every, steps - done)
            s.step(n)
            done += n
            try:
                d = s.diagnostics()
            except LbsError as e:
                if e.code != LBS_ENOCONV:  # (SOR round limit: reported, state kept)
                    raise
                d = s.diagnostics()
            hist.append(d)
    except LbsError as e:
        if e.code != LBS_EDIVERGED:
            raise
        return (float("nan"),) * 4
    finally:
        s.close()
    return summarise(hist, window)


def generate(n, seed, steps, sample_every=500, batch_size=64, plain=False, storage="f32",
             window=0.25, log=print):
    """Sweep n seeded points (workloads.bubble_sweep_2d) and return arrays
    X (n x 5 features), Y (n x 2: Re, AR), S (n x 2 spreads)."""
    cfgs = W.bubble_sweep_2d(n, seed=seed)
    X = np.array([features(c["sweep_point"]) for c in cfgs])
    Y = np.zeros((n, 2))
    S = np.zeros((n, 2))
    t0 = time.time()
    mlups = []
    secs = np.zeros(n)
    if plain:
        for k, c in enumerate(cfgs):
            t1 = time.time()
            re, ar, rs, as_ = run_plain(c, steps, sample_every, storage, window, seed=1000 + k)
            secs[k] = time.time() - t1
            Y[k] = (re, ar)
            S[k] = (rs, as_)
            log(f"plain {k + 1}/{n} Re {re:.3f} AR {ar:.3f} ({time.time() - t0:.0f} s)")
    else:
        for i in range(0, n, batch_size):
            part = cfgs[i:i + batch_size]
            res, m = run_batch(part, steps, sample_every, storage, window, seed=1000 + i,
                               log=log if sample_every * 10 >= steps else None)
            mlups.append(m)
            for j, (re, ar, rs, as_) in enumerate(res):
                Y[i + j] = (re, ar)
                S[i + j] = (rs, as_)
            log(f"batch {i // batch_size + 1}: {m:.0f} MLUPS ({time.time() - t0:.0f} s)")
    ok = np.isfinite(Y).all(axis=1)
    log(f"{int(ok.sum())} of {n} solves finished ({n - int(ok.sum())} diverged)")
    return dict(X=X, Y=Y, S=S, ok=ok, seed=seed, steps=steps, plain=plain, solve_seconds=secs,
                mlups=np.array(mlups), features=np.array(FEATURES), targets=np.array(TARGETS))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30000)
    ap.add_argument("--sample-every", type=int, default=500)
    ap.add_argument("--plain", action="store_true")
    ap.add_argument("--storage", default="f32")
    ap.add_argument("--out", required=True)
    a = ap.parse_args()
    r = generate(a.n, a.seed, a.steps, a.sample_every, plain=a.plain, storage=a.storage)
    np.savez(a.out, **r)
    print("wrote", a.out)


if __name__ == "__main__":
    main()
