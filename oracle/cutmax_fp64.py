"""FP64 CutMax: Alg. 1 exactly, and the FP64 mirror of the HE circuit (Alg. 2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

``cutmax_exact``   Alg. 1 (Sect. 3.1): T iterations of mean, population
                   variance, z = (y - mu)/(c*sigma) + 1, y <- z^p; then Z = Y/sum(Y).
                   Reading: the normalisation uses the last iterate.
``cutmax_circuit`` the same polynomial steps the encrypted circuit evaluates
                   (Alg. 2, Sect. 3.2): integer-centred D = n*Y - S, the
                   rotate-and-sum sums, the coupled Goldschmidt inverse square
                   root (App. B.1, after Panda 2022; with a plan's relaxation
                   constants each step's 3/2 becomes that step's alpha, the
                   over-relaxed form App. B cites) and the Goldschmidt inverse
                   prod_{i<=d} (1 + (1-x)^(2^i)) (equation in App. B.1).
Also: the convergence bound and T_min of Theorem 1 / App. E table, the Beta
cut-noise exponent of Lemma 2 / Observation 1 and the Gumbel noise of Def. 3.1.
"""
import math

import numpy as np


def _per_iter(v, T):
    if np.isscalar(v):
        return [v] * T
    v = list(v)
    assert len(v) == T
    return v


def cutmax_exact(x, T, p, c, return_iterates=False):
    """Alg. 1 in float64."""
    y = np.asarray(x, dtype=np.float64).copy()
    ps, cs = _per_iter(p, T), _per_iter(c, T)
    its = [y.copy()]
    for t in range(T):
        mu = y.mean()
        var = ((y - mu) ** 2).mean()
        z = (y - mu) / (cs[t] * math.sqrt(var)) + 1.0
        y = z ** ps[t]
        its.append(y.copy())
    Z = y / y.sum()
    return (Z, its) if return_iterates else Z


def semi_standardize(y, c):
    """S_c of Def. (c-semi-standardisation), App. E.1."""
    y = np.asarray(y, dtype=np.float64)
    mu = y.mean()
    sd = math.sqrt(((y - mu) ** 2).mean())
    return (y - mu) / (c * sd) + 1.0


def gap_ratio(y):
    """Gamma(y) = y_(i*) / y_(i**) (Def. Gap Ratio, App. E.1)."""
    s = np.sort(np.asarray(y, dtype=np.float64))
    return s[-1] / s[-2]


def is_delta_gap_bounded(x, delta):
    s = np.sort(np.asarray(x, dtype=np.float64))
    return s[-1] - s[-2] >= delta * np.asarray(x).std()


def gap_growth_bound(delta, c, n, p):
    """(1 + delta/(c + sqrt n))^p, Lemma 4 / Lemma 5 (App. E.2)."""
    return (1.0 + delta / (c + math.sqrt(n))) ** p


def t_min(k, delta, c, n, p, gamma0=1.0):
    """Theorem 1: T >= ceil((ln k - ln Gamma0) / (p ln(1 + delta/(c + sqrt n))))."""
    return math.ceil((math.log(k) - math.log(gamma0)) / (p * math.log(1.0 + delta / (c + math.sqrt(n)))))


def goldschmidt_inv(x, d):
    """prod_{i=0}^{d} (1 + (1-x)^(2^i)), App. B.1; converges to 1/x on (0, 2)."""
    a = 1.0 - np.asarray(x, dtype=np.float64)
    f = 1.0 + a
    sq = a
    for _ in range(d):
        sq = sq * sq
        f = f * (1.0 + sq)
    return f


def goldschmidt_invsqrt(x, k, y0, alphas=None):
    """Coupled Goldschmidt iteration for 1/sqrt(x) (k >= 1 iterations).

    g0 = x*y0, h0 = y0/2; repeat: r = 1/2 - g*h, g <- g*(1+r), h <- h*(1+r);
    return 2*h.  Written with the same grouping as the encrypted circuit.
    alphas: step i's 1 + r is alphas[i-1] - g*h instead of 3/2 - g*h (the
    over-relaxed form; 3/2 is Newton's step).
    """
    x = np.asarray(x, dtype=np.float64)
    al = [1.5] * max(k, 1) if alphas is None else list(alphas)
    a = al[0] - (y0 * y0 / 2.0) * x
    h = (y0 / 2.0) * a
    g = (x * y0) * a
    for i in range(2, k + 1):
        a = al[i - 1] - g * h
        if i < k:
            g = g * a
        h = h * a
    return 2.0 * h


def power_by_squaring(u, p):
    """u^p with the squaring / multiplication order of the encrypted circuit."""
    sq = u
    acc = None
    pp = int(p)
    while True:
        if pp & 1:
            acc = sq if acc is None else acc * sq
        pp >>= 1
        if pp == 0:
            break
        sq = sq * sq
    return acc


def relax_constants(plan, t):
    """The additive constant of each Goldschmidt step of iteration t: 3/2
    (Newton's step for x^(-1/2)) unless the plan carries relaxation constants
    (plan.relax[t], one per step)."""
    k = plan.k[t]
    r = getattr(plan, "relax", None)
    if r is None or r[t] is None or len(r[t]) == 0:
        return [1.5] * max(k, 1)
    assert len(r[t]) == k
    return [float(v) for v in r[t]]


def cutmax_circuit(x, plan, return_trace=False):
    """FP64 mirror of the encrypted circuit, on the n real entries.

    The padded slots of the ciphertext hold zero and are left out of every
    sum by construction (variance correction and mask), so the mirror works on
    the real entries only.
    """
    y = np.asarray(x, dtype=np.float64).copy()
    n = plan.n
    boot = bool(getattr(plan, "bootstrap", False))
    trace = {"V": [], "S_final": None}
    for t in range(plan.T):
        S = y.sum()
        D = n * y - S
        V = (D * D).sum()
        trace["V"].append(V)
        kap, y0, k = plan.kappa[t], plan.y0[t], plan.k[t]
        al = relax_constants(plan, t)
        rn = plan.norm[t] ** (1.0 / plan.p[t]) if boot else 1.0
        if k == 0:                    # learned quadratic (A x^2 + B x + C)/2 of x = kappa V
            A, B, C = plan.lq[t]
            xx = kap * V
            h = (A * xx * xx + B * xx + C) / 2.0
        elif boot:                    # bootstrapped circuit: x = kappa V first
            xx = kap * V
            a = al[0] - (y0 * y0 / 2.0) * xx
            h = (y0 / 2.0) * a
            g = (xx * y0) * a
        else:
            a = al[0] - (kap * y0 * y0 / 2.0) * V
            h = (y0 / 2.0) * a
            g = (kap * y0 * V) * a
        for i in range(2, k + 1) if k else ():
            a = al[i - 1] - g * h
            if i < k:
                g = g * a
            h = h * a
        Dp = D * (2.0 * math.sqrt(kap * n) / plan.c[t] * rn)
        u = Dp * h + rn
        y = power_by_squaring(u, plan.p[t])
    S = y.sum()
    trace["S_final"] = S
    a = 1.0 - plan.kappa_f * S
    F = 1.0 + a
    sq = a
    for _ in range(plan.d):
        sq = sq * sq
        F = F * (1.0 + sq)
    Z = (y * plan.kappa_f) * F
    return (Z, trace) if return_trace else Z


# ---------------------------------------------------------------- sampling
def beta_alpha(p, q=None):
    """alpha of Lemma 2 (q = p) and Observation 1: ln(1-q)/ln(p)."""
    q = p if q is None else q
    return math.log(1.0 - q) / math.log(p)


def beta_noise(u, alpha):
    """Inverse CDF of Beta(alpha, 1): F(x) = x^alpha, so G = U^(1/alpha) (Alg. 3)."""
    return np.asarray(u, dtype=np.float64) ** (1.0 / alpha)


def gumbel_noise(u):
    """G = -log(-log U), Def. 3.1 (Gumbel(0,1))."""
    return -np.log(-np.log(np.asarray(u, dtype=np.float64)))


def nucleus_set(x, p):
    """Smallest top-ranked set with softmax mass >= p (nucleus / top-p)."""
    x = np.asarray(x, dtype=np.float64)
    pr = np.exp(x - x.max())
    pr /= pr.sum()
    order = np.argsort(-pr, kind="stable")
    cum = np.cumsum(pr[order])
    k = int(np.searchsorted(cum, p) + 1)
    return set(order[:k].tolist())
