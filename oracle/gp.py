"""Dense FP64 Gaussian-process oracle (numpy).

TEST INFRASTRUCTURE ONLY: tests/, the smoke check and bench.py's CPU-baseline
leg may import this module; the product package never does.

Follows the paper's Sec. 2.2 and 2.3:
  - Eq. quadraticKernelEq: K(x_i, x_j) = sf2 * exp(-d_ij^2 / (2 l2));
  - Eq. d2Eq: d_ij^2 = sum_k ((x_ik - x_jk) / Dbar_k)^2, with Dbar_k the mean
    separation between database inputs along dimension k (reading: the mean of
    |x_ik - x_jk| over all pairs i < j; recomputed whenever the database
    changes; a fallback scale when fewer than two entries or a zero spread);
  - Eq. covarianceEq: C = K(X, X) + sn2 I;
  - Eq. predMeanEq: mean = mu(X*) + K(X*, X) C^-1 (y - mu(X));
  - Eq. predVarEq: var = diag(K(X*, X*) - K(X*, X) C^-1 K(X, X*)), the latent
    variance with no noise term, clamped at zero;
  - Eq. evidenceEq: log marginal likelihood;
  - App. B, Eq. periodicKernel: K(t, t') = sf2 exp(-2 sin^2(pi |t - t'| / T) / l2)
    on a single input (time), no Eq. d2Eq scaling, for filtering a periodic
    flow-rate time series (period > 0 selects it).
The Cholesky factorisation and triangular solves are numpy/scipy library
primitives used as single steps.
"""
import math

import numpy as np
import scipy.linalg as sla


def scales(X, fallback=1.0):
    """Dbar_k: mean over all pairs i < j of |x_ik - x_jk| (Eq. d2Eq reading)."""
    X = np.asarray(X, dtype=np.float64)
    M, D = X.shape
    fb = np.broadcast_to(np.asarray(fallback, dtype=np.float64), (D,))
    out = np.array(fb, dtype=np.float64)
    if M < 2:
        return out
    for k in range(D):
        tot = 0.0
        for i in range(M):
            tot += np.abs(X[i + 1:, k] - X[i, k]).sum()
        mean = tot / (M * (M - 1) / 2)
        if mean > 0.0:
            out[k] = mean
    return out


def sq_dist(A, B, dbar):
    """Normalised squared distances d_ij^2 between rows of A and B (Eq. d2Eq)."""
    A = np.asarray(A, dtype=np.float64) / dbar
    B = np.asarray(B, dtype=np.float64) / dbar
    diff = A[:, None, :] - B[None, :, :]
    return (diff * diff).sum(axis=2)


def kernel(A, B, dbar, sf2, l2):
    """Squared-exponential covariance (Eq. quadraticKernelEq)."""
    return sf2 * np.exp(-sq_dist(A, B, dbar) / (2.0 * l2))


def periodic_kernel(A, B, period, sf2, l2):
    """App. B Eq. periodicKernel on one input: sf2 exp(-2 sin^2(pi |t - t'| / T) / l2)."""
    a = np.asarray(A, dtype=np.float64).reshape(-1)
    b = np.asarray(B, dtype=np.float64).reshape(-1)
    s = np.sin(np.pi * np.abs(a[:, None] - b[None, :]) / period)
    return sf2 * np.exp(-2.0 * s * s / l2)


class GP:
    """Fit on (X, y) with hyperparameters (sf2, l2, sn2) and an optional prior
    mean function mu (callable on an (n, D) array; zero by default)."""

    def __init__(self, X, y, sf2, l2, sn2, mu=None, dbar=None, fallback=1.0, period=0.0):
        self.X = np.asarray(X, dtype=np.float64).reshape(len(y), -1) if len(y) else np.zeros((0, 1))
        self.y = np.asarray(y, dtype=np.float64)
        self.sf2, self.l2, self.sn2 = float(sf2), float(l2), float(sn2)
        self.mu = mu
        self.period = float(period)
        self.M = len(self.y)
        if self.M == 0:
            self.dbar = None
            return
        if self.period > 0.0:
            self.dbar = None
        else:
            self.dbar = scales(self.X, fallback) if dbar is None else np.asarray(dbar, dtype=np.float64)
        C = self._k(self.X, self.X) + self.sn2 * np.eye(self.M)
        self.C = C
        self.L = np.linalg.cholesky(C)                              # C = L L^T
        r = self.y - self._mu(self.X)
        self.alpha = sla.cho_solve((self.L, True), r)               # C^-1 (y - mu(X))

    def _k(self, A, B):
        if self.period > 0.0:
            return periodic_kernel(A, B, self.period, self.sf2, self.l2)
        return kernel(A, B, self.dbar, self.sf2, self.l2)

    def _mu(self, X):
        if self.mu is None:
            return np.zeros(len(X))
        return np.asarray(self.mu(X), dtype=np.float64).reshape(len(X))

    def predict(self, Xs):
        """Posterior mean and latent variance at the rows of Xs."""
        Xs = np.asarray(Xs, dtype=np.float64).reshape(len(Xs), -1)
        m0 = self._mu(Xs)
        if self.M == 0:
            return m0, np.full(len(Xs), self.sf2)
        Ks = self._k(Xs, self.X)                                    # K(X*, X)
        mean = m0 + Ks @ self.alpha
        V = sla.solve_triangular(self.L, Ks.T, lower=True)          # L^-1 K(X, X*)
        var = self.sf2 - (V * V).sum(axis=0)
        return mean, np.maximum(var, 0.0)

    def log_marginal_likelihood(self):
        """Eq. evidenceEq with y replaced by y - mu(X)."""
        r = self.y - self._mu(self.X)
        return (-0.5 * r @ self.alpha - np.log(np.diag(self.L)).sum()
                - 0.5 * self.M * np.log(2.0 * np.pi))


def gate(sd, sigma_t):
    """Alg. 1: an MD run is requested when the predicted standard deviation
    exceeds the threshold (strict inequality)."""
    return np.asarray(sd) > sigma_t


def optimize(X, y, sf2, l2, sn2, mu=None, fallback=1.0, max_evals=200, period=0.0, hold=0):
    """Hyperparameters by maximum evidence (Sec. 2.3, Eq. evidenceEq): a
    pattern search over (sf2, l2, sn2).  Each coordinate in turn tries
    value * step and value / step and keeps the better log marginal
    likelihood when it gains more than 1e-9 relative (+1e-12); a pass with no
    move takes the square root of the step, from 4 while it exceeds 1.05, or
    until max_evals evaluations.  A covariance that is not positive definite
    scores -inf.  hold is a bit mask of the values kept fixed (1 sf2, 2 l2,
    4 sn2; App. B keeps sf2).  Returns (sf2, l2, sn2, lml)."""
    def lml(h):
        try:
            return GP(X, y, h[0], h[1], h[2], mu=mu, fallback=fallback, period=period).log_marginal_likelihood()
        except np.linalg.LinAlgError:
            return -np.inf
    cur = [float(sf2), float(l2), float(sn2)]
    f = lml(cur)
    evals, step = 1, 4.0
    while step > 1.05 and evals < max_evals:
        moved = False
        for k in range(3):
            if evals >= max_evals:
                break
            if hold & (1 << k):
                continue
            v0 = cur[k]
            bestv, bestf = v0, f
            for v in (v0 * step, v0 / step):
                if evals >= max_evals:
                    break
                cur[k] = v
                ft = lml(cur)
                evals += 1
                if ft > bestf + 1e-9 * abs(bestf) + 1e-12:
                    bestf, bestv = ft, v
            cur[k] = bestv
            if bestv != v0:
                f, moved = bestf, True
        if not moved:
            step = math.sqrt(step)
    return cur[0], cur[1], cur[2], f


def periodic_filter(t, q, period, sf2, l2, sn2, fit_until=None, max_evals=200):
    """App. B: filter the noise out of a periodic flow-rate time series q(t).
    The length scale and the noise variance maximise the log marginal
    likelihood (Sec. 2.3) of the samples up to fit_until (the paper: the
    first peak), with sf2 held; then GP regression with zero prior mean over
    the whole series (Eqs. predMeanEq, predVarEq).  Returns (mean, var, l2, sn2)."""
    t = np.asarray(t, dtype=np.float64).reshape(-1, 1)
    q = np.asarray(q, dtype=np.float64)
    sel = slice(None) if fit_until is None else (t[:, 0] <= fit_until)
    _, l2, sn2, _ = optimize(t[sel], q[sel], sf2, l2, sn2, period=period, hold=1, max_evals=max_evals)
    g = GP(t, q, sf2, l2, sn2, period=period)
    mean, var = g.predict(t)
    return mean, var, l2, sn2
