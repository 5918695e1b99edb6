"""Synthetic analogues of the paper's plaintext experiments (Sect. 4), on
seeded synthetic logits instead of the LLM logits of arXiv abstracts, at sizes
that run in seconds (`tests/synthetic_experiments.py` runs them at the paper's
vocabulary sizes):

- convergence of Alg. 1 against T (Table empirical_T): for every T some odd
  p in 7..19 and odd c in 3..39 recovers the argmax of every input, and the
  best mean of max Z grows with T to one-hot;
- the violation rate of nucleus sampling (Fig. 5, p = 0.9): Gumbel-max draws
  fall outside the top-p nucleus with probability exactly 1 - (nucleus mass),
  the Beta cut of Alg. 3 (alpha of Lemma 2) never does;
- the fraction of entries below the mean per iteration (Fig. 3, (p, c) =
  (19, 27), T = 3) grows with t.
"""
import numpy as np

from oracle import cutmax_fp64 as F
from paper_2509_08383_gb300 import synth

GAPS = (0.05, 0.2, 1.0)


def _cutmax_rows(X, T, p, c):
    """Alg. 1 on every row of X (the rows are independent inputs)."""
    Y = X.copy()
    for _ in range(T):
        mu = Y.mean(1, keepdims=True)
        sd = Y.std(1, keepdims=True)
        Y = ((Y - mu) / (c * sd) + 1.0) ** p
    return Y / Y.sum(1, keepdims=True)


def convergence_table(n, seeds, Ts=(2, 3, 4, 5)):
    """Per T: (best mean max Z, its max over inputs, p, c) over the paper's grid,
    among the (p, c) that recover every input's argmax."""
    X = np.stack([synth.logits_heavy_tail(s, n=n, gap=GAPS[s % 3]) for s in seeds])
    am = X.argmax(1)
    out = {}
    for T in Ts:
        best = None
        for p in range(7, 20, 2):
            for c in range(3, 40, 2):
                with np.errstate(all="ignore"):
                    Z = _cutmax_rows(X, T, p, c)
                if not np.isfinite(Z).all() or not (Z.argmax(1) == am).all():
                    continue
                mz = Z.max(1)
                if best is None or mz.mean() > best[0]:
                    best = (float(mz.mean()), float(mz.max()), p, c)
        out[T] = best
    # the single exact routine on one input, to tie the batched rows to it
    T, (_, _, p, c) = max(out), out[max(out)]
    assert np.allclose(_cutmax_rows(X[:1], T, p, c)[0], F.cutmax_exact(X[0], T, p, c))
    return out


def violation_rates(n, seeds, draws, p=0.9, sd=2.0):
    """Per input: (Gumbel-max violation rate, Beta-cut violation rate, 1 - nucleus mass)."""
    alpha = F.beta_alpha(p)
    rows = []
    for s in seeds:
        x = synth.logits_gaussian(s, n=n, sd=sd, gap=0.5)
        nuc = np.zeros(n, dtype=bool)
        nuc[list(F.nucleus_set(x, p))] = True
        pr = np.exp(x - x.max())
        pr /= pr.sum()
        u = synth.uniforms(10_000 + s, draws * n).reshape(draws, n)
        g = (x[None, :] + F.gumbel_noise(u)).argmax(1)
        b = (x[None, :] + F.beta_noise(u, alpha)).argmax(1)
        rows.append((1.0 - nuc[g].mean(), 1.0 - nuc[b].mean(), 1.0 - pr[nuc].sum()))
    return np.asarray(rows)


def below_mean_fractions(n, seeds, T=3, p=19, c=27):
    """[inputs, T] fractions of entries below the mean of each iterate."""
    fr = []
    for s in seeds:
        x = synth.logits_heavy_tail(s, n=n, gap=GAPS[s % 3])
        _, its = F.cutmax_exact(x, T, p, c, return_iterates=True)
        fr.append([float((y < y.mean()).mean()) for y in its[1:]])
    return np.asarray(fr)


def test_convergence_against_T():
    tab = convergence_table(8192, range(1000, 1009), Ts=(2, 3, 4))
    assert all(tab[T] is not None for T in tab)            # full recovery reachable at every T
    means = [tab[T][0] for T in sorted(tab)]
    assert means == sorted(means)                           # more iterations concentrate more mass
    assert tab[4][0] > 0.999                                # near one-hot by T = 4 (Table empirical_T)


def test_nucleus_violation_rates():
    v = violation_rates(1024, range(3000, 3020), draws=500)
    assert (v[:, 1] == 0).all()                             # the Beta cut never leaves the nucleus
    # Gumbel-max samples softmax(x) exactly: it leaves the nucleus with
    # probability 1 - (nucleus mass), within sampling error
    se = np.sqrt(v[:, 2] * (1 - v[:, 2]) / 500)
    assert abs(v[:, 0].mean() - v[:, 2].mean()) < 4 * np.sqrt((se ** 2).sum()) / len(v)
    assert 0.05 < v[:, 2].mean() <= 0.1                     # the nucleus holds at least p of the mass


def test_below_mean_fraction_grows():
    fr = below_mean_fractions(8192, range(2000, 2010))
    m = fr.mean(0)
    assert (np.diff(m) > 0).all()
    assert m[-1] > 0.99
