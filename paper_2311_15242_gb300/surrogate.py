"""Surrogate of the bubble-rise sweep: terminal Reynolds number and aspect
ratio from (Eo, Bi, W/D, E0, C0), with the plain solver as fallback.

An ensemble of five networks 5 -> 128 -> 128 -> 128 -> 2 (SiLU), trained
on the GPU by the library's kernels (lbs_mlp_*) on sweep results, evaluated
with bfloat16 weights.  Inputs are encoded as (log Eo, log Bi, W/D, E0, C0)
and standardised; targets are log Re and log AR, standardised, so that the
ensemble's standard deviation of a log target is the relative uncertainty
(std / |mean|) of that output to first order.  The spread of an ensemble
trained on the same data understates its error, so it is calibrated: a
fifth of the training points is held back, the ensemble trained on the rest
predicts them, and for each output the factor k that makes k * spread
cover 90 % of their errors scales every later uncertainty of that output
(the final ensemble is then trained on all points).  A query whose calibrated relative uncertainty exceeds the
tolerance (3 %) on either output is not answered by the network: the plain
solver runs it (`query`).  The most uncertain candidates are where a sweep
should refine next (`suggest`).
"""
import numpy as np

N_IN, N_OUT = 5, 2


def encode(X):
    """Network inputs from raw features (Eo, Bi, W/D, E0, C0)."""
    X = np.asarray(X, np.float64)
    return np.stack([np.log(X[:, 0]), np.log(X[:, 1]), X[:, 2], X[:, 3], X[:, 4]], axis=1)


class Surrogate:
    def __init__(self, members=5, width=128, depth=3, max_batch=1024):
        from . import Mlp
        self.net = Mlp(members, N_IN, width, depth, N_OUT, max_batch=max_batch)
        self.mx = self.sx = self.my = self.sy = None

    def close(self):
        self.net.close()

    def _train(self, X, Y, iters, batch, lr, seed):
        Z = encode(X)
        T = np.log(np.asarray(Y, np.float64))
        self.mx, self.sx = Z.mean(0), Z.std(0) + 1e-12
        self.my, self.sy = T.mean(0), T.std(0) + 1e-12
        self.net.init(seed)
        self.net.set_data(((Z - self.mx) / self.sx).astype(np.float32),
                          ((T - self.my) / self.sy).astype(np.float32))
        b = min(batch, self.net.max_batch)
        loss = None
        # the learning rate steps down by 3 twice (at 1/2 and 3/4 of the run)
        for frac, scale in ((0.5, 1.0), (0.25, 1.0 / 3.0), (0.25, 1.0 / 9.0)):
            loss = self.net.train(int(iters * frac), b, lr * scale, seed=seed + 1)
        return loss

    def fit(self, X, Y, iters=6000, batch=256, lr=2e-3, seed=0, calib_frac=0.2, cover=0.9):
        """Train on features X [n][5] and targets Y [n][2] = (Re, AR) and
        calibrate the uncertainty (see the module notes).  Returns the last
        minibatch loss of every member of the final ensemble."""
        X = np.asarray(X, np.float64)
        Y = np.asarray(Y, np.float64)
        rng = np.random.default_rng(seed)
        perm = rng.permutation(len(X))
        nc = max(1, int(round(calib_frac * len(X))))
        cal, fit = perm[:nc], perm[nc:]
        self.k = np.ones(N_OUT)
        self._train(X[fit], Y[fit], iters, batch, lr, seed)
        mean, unc = self.predict(X[cal])
        err = np.abs(np.log(mean / Y[cal]))
        self.k = np.quantile(err / np.maximum(unc, 1e-12), cover, axis=0)
        return self._train(X, Y, iters, batch, lr, seed)

    def predict(self, X, bf16=True):
        """(mean [n][2] in physical units, calibrated relative uncertainty
        [n][2])."""
        Z = ((encode(X) - self.mx) / self.sx).astype(np.float32)
        mu, sd = self.net.predict(Z, bf16=bf16)
        logm = mu.astype(np.float64) * self.sy + self.my
        k = getattr(self, "k", np.ones(N_OUT))
        return np.exp(logm), k * sd.astype(np.float64) * self.sy

    def query(self, X, solve, tol=0.03, bf16=True):
        """Answer every query: the network where its relative uncertainty is
        within tol on both outputs, else solve(i) -> (Re, AR) (the plain
        solver).  Returns (Y, served) with served[i] True where the network
        answered."""
        mean, unc = self.predict(X, bf16=bf16)
        served = unc.max(axis=1) <= tol
        Y = mean.copy()
        for i in np.flatnonzero(~served):
            Y[i] = solve(i)
        return Y, served

    def suggest(self, candidates, k, bf16=True):
        """Indices of the k candidates with the largest relative uncertainty
        (the points where the sweep should run next)."""
        _, unc = self.predict(candidates, bf16=bf16)
        return np.argsort(-unc.max(axis=1))[:k]
