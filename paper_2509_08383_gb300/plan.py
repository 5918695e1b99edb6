"""CutMax circuit plan: the constants that make Alg. 2 polynomial and in range.

Sect. 3.2 of the paper requires two obligations of any encrypted CutMax:
(i) no intermediate exceeds the scheme bound and (ii) the inputs of the
inverse-square-root and inverse approximations stay inside their convergence
ranges, which is achieved by range scaling x -> x/b with a known bound b.
This module picks those constants from FP64 statistics of the input
distribution (client side, never on encrypted data):

  kappa[t]  range scale of the iteration-t variance sum V_t = sum (n*y - S)^2
            (= n^3 sigma_t^2); the Goldschmidt input is kappa[t] * V_t
  y0[t]     Goldschmidt initial guess for 1/sqrt(kappa[t] V_t)
  k[t]      Goldschmidt inverse-square-root iterations (2 levels each)
  kappa_f   range scale of the final sum S_T for the Goldschmidt inverse
  d         degree of the Goldschmidt inverse (product of d+1 factors)
  norm[t]   positive factor applied to Y_(t+1) (folded as norm^(1/p) into the
            standardisation constants) so that max Y stays near 1 where a
            ciphertext may be bootstrapped; 1 for leveled plans

The statistics are those of the polynomial circuit itself (its Goldschmidt
iterates, not the exact Alg. 1), taken iteration by iteration, since an
approximate inverse square root changes every later statistic.

S_c is scale invariant (Def. of c-semi-standardisation, App. E.1) and so is
the final normalisation, so only the spread of V_t and S_T across inputs
matters, not their absolute size.
"""
import math
from dataclasses import dataclass, field, asdict
from typing import List

import numpy as np


@dataclass
class CutMaxPlan:
    n: int                      # real entries (vocabulary size) per stream
    slots: int                  # N/2
    packing: str                # "replicate" (n | slots, n power of two) or "pad"
    T: int
    p: List[int]
    c: List[float]
    k: List[int]
    kappa: List[float]
    y0: List[float]
    d: int
    kappa_f: float
    bootstrap: bool = False
    norm: List[float] = None
    extra: dict = field(default_factory=dict)
    cts: int = 1                # ciphertexts per stream (n > slots spreads over several)
    shared: bool = False        # batched streams share the scalar chains (bootstrapped plans)
    lq: List = None             # per iteration [A, B, C] of a learned quadratic (used where k[t] == 0)
    relax: List = None          # per iteration the k[t] Goldschmidt steps' additive constants (None: 3/2)

    def __post_init__(self):
        if self.norm is None:
            self.norm = [1.0] * self.T

    @property
    def rotsum_steps(self) -> int:
        m = self.n if self.packing == "replicate" else self.slots
        return int(round(math.log2(m)))

    @property
    def pad(self) -> int:
        return 0 if self.packing == "replicate" else self.cts * self.slots - self.n

    def depth(self) -> int:
        """Levels consumed without bootstrapping (see the circuit description;
        a learned iteration counts 2 levels for the quadratic and 3 for x)."""
        dep = 0
        for t in range(self.T):
            dep += 2 + (2 * self.k[t] if self.k[t] else 5) + power_depth(self.p[t])
        return dep + self.d + 3

    def to_dict(self):
        return asdict(self)


def power_depth(p: int) -> int:
    """Depth of y^p by square-and-multiply: ceil(log2 p)."""
    p = int(p)
    if p <= 1:
        return 0
    return (p - 1).bit_length()


def cts_for(n: int, slots: int) -> int:
    """Ciphertexts a stream of n entries fills."""
    return -(-int(n) // int(slots))


def packing_for(n: int, slots: int) -> str:
    if n <= slots and slots % n == 0 and (n & (n - 1)) == 0:
        return "replicate"
    return "pad"


def pack(x, slots: int, packing: str) -> np.ndarray:
    """Slot vector for one ciphertext (n <= slots)."""
    x = np.asarray(x, dtype=np.float64)
    if len(x) > slots:
        raise ValueError("n > slots: use pack_cts")
    out = np.zeros(slots)
    if packing == "replicate":
        out[:] = np.tile(x, slots // len(x))
    else:
        out[: len(x)] = x
    return out


def pack_cts(x, slots: int) -> List[np.ndarray]:
    """Slot vectors of the ciphertexts of one zero-padded stream: ciphertext c
    holds entries c*slots .. (c+1)*slots - 1, the last one zero-padded."""
    x = np.asarray(x, dtype=np.float64)
    k = cts_for(len(x), slots)
    out = np.zeros(k * slots)
    out[: len(x)] = x
    return [out[c * slots:(c + 1) * slots].copy() for c in range(k)]


def _exact_stats(x, T, p, c):
    """V_t = sum (n y - S)^2 for t < T and S_T = sum y_T under Alg. 1."""
    y = np.asarray(x, dtype=np.float64).copy()
    n = len(y)
    Vs = []
    for t in range(T):
        S = y.sum()
        D = n * y - S
        V = float((D * D).sum())
        Vs.append(V)
        mu = S / n
        sig = math.sqrt(V / n ** 3)
        y = ((y - mu) / (c[t] * sig) + 1.0) ** p[t]
    return Vs, float(y.sum())


def _invsqrt_half(x, k, y0, alphas=None):
    """The circuit's Goldschmidt output h ~ 1/(2 sqrt(x)) (k iterations; step i
    multiplies by alpha_i - g h, alpha_i = 3/2 unless relaxation constants are
    given)."""
    al = [1.5] * max(k, 1) if alphas is None else alphas
    a = al[0] - (y0 * y0 / 2.0) * x
    h = (y0 / 2.0) * a
    g = (x * y0) * a
    for i in range(2, k + 1):
        a = al[i - 1] - g * h
        if i < k:
            g = g * a
        h = h * a
    return h


def invsqrt_half_at(plan_k, plan_y0, lq, t, x, relax=None):
    """h of iteration t of the circuit: Goldschmidt (k[t] >= 1, with the
    plan's relaxation constants if any) or the learned quadratic
    (A x^2 + B x + C)/2 (k[t] == 0)."""
    if plan_k[t] == 0:
        A, B, C = lq[t]
        return (A * x * x + B * x + C) / 2.0
    al = relax[t] if relax is not None and relax[t] else None
    return _invsqrt_half(x, plan_k[t], plan_y0[t], al)


def _invsqrt_err(x, k, y0, alphas=None):
    return np.abs(2.0 * _invsqrt_half(x, k, y0, alphas) * np.sqrt(x) - 1.0).max()


def _relaxed_steps(xs, k_max, tol, c_maxes=(2.0, 2.5)):
    """Fewest relaxed Goldschmidt steps reaching tol on xs, and their start.

    With u = x y^2 a step maps u to u (alpha - u/2)^2: alpha = 3/2 is Newton's
    step (quadratic convergence at u = 1), a larger alpha multiplies a small u
    by alpha^2 instead of 9/4, so a wide range climbs to 1 in fewer steps.
    Only the additive constant changes, so a relaxed step costs the levels of
    a plain one.  Greedy per step: while u_min < 1/4 take the alpha that lifts
    u_min most with every image in (0, c_max]; after that the one with the
    least error.  Starts put x_max y0^2 in [0.3, c_max]; the plan keeps the
    start with the fewest steps (then the least error), checked with the
    circuit's own iteration."""
    grid = np.linspace(1.5, 3.5, 201)
    best = None
    for cmax in c_maxes:
        for c in np.linspace(0.3, cmax, 40):
            y0 = math.sqrt(c / xs[-1])
            u = xs * y0 * y0
            al = []
            while np.abs(np.sqrt(u) - 1.0).max() >= tol and len(al) < k_max:
                key_best, a_best = None, 1.5
                for a in grid:
                    v = u * (a - 0.5 * u) ** 2
                    if v.max() > cmax or v.min() <= 0.0:
                        continue
                    key = -v.min() if u.min() < 0.25 else np.abs(np.sqrt(v) - 1.0).max()
                    if key_best is None or key < key_best:
                        key_best, a_best = key, float(a)
                al.append(a_best)
                u = u * (a_best - 0.5 * u) ** 2
            if not al:
                continue
            err = _invsqrt_err(xs, len(al), y0, al)
            if err < tol and (best is None or (len(al), err) < (len(best[1]), best[2])):
                best = (y0, al, err)
    return None if best is None else (best[0], best[1])


def _fewest_iterations(xs, k_max, tol, y0_default):
    """Smallest k (and a constant start y0 reaching it) with the circuit's
    Goldschmidt error below tol on xs.  The iteration needs 0 < x y0^2 < 3;
    candidates put x_max y0^2 between 0.5 and 2.5 (headroom below 3 for inputs
    beyond the calibrated range)."""
    cands = [y0_default] + [math.sqrt(u / xs[-1]) for u in np.linspace(0.5, 2.5, 50)]
    best_k, best_y0 = k_max, y0_default
    for kk in range(1, k_max + 1):
        ok = [y for y in cands if _invsqrt_err(xs, kk, y) < tol]
        if ok:
            # among the starts that reach tol in kk steps, the one with the least error
            errs = [_invsqrt_err(xs, kk, y) for y in ok]
            return kk, ok[int(np.argmin(errs))]
    return best_k, best_y0


def _inv_err(x, d):
    a = 1.0 - x
    f = 1.0 + a
    sq = a
    for _ in range(d):
        sq = sq * sq
        f = f * (1.0 + sq)
    return np.abs(x * f - 1.0).max()


def _power(u, p):
    sq, acc, pp = u, None, int(p)
    while True:
        if pp & 1:
            acc = sq if acc is None else acc * sq
        pp >>= 1
        if pp == 0:
            break
        sq = sq * sq
    return acc


def calibrate(sample, n_cal, n, slots, T, p, c, margin=1.25, tol_k=1e-7, tol_d=1e-7,
              k_max=8, d_max=12, k_fixed=None, d_fixed=None, bootstrap=False, norm_margin=1.25, learn=None,
              relax=False):
    """Pick kappa/y0/k per iteration and kappa_f/d from `n_cal` draws of ``sample(i)``,
    following the circuit's own iterates; with bootstrap=True also the
    normalisers norm[t] that keep max Y_(t+1) at about 1/norm_margin.
    learn(t, kappa_t, xs, (a, b)) -> [A, B, C] or None: offered the iteration-t
    range scale, the inputs x of the calibration draws and the margin range; a
    quadratic it returns replaces that iteration's Goldschmidt steps (k[t] = 0).
    relax=True: where relaxation constants (one per Goldschmidt step) reach
    tol_k in fewer steps than Newton's 3/2, the iteration takes them."""
    p = [int(v) for v in (p if not np.isscalar(p) else [p] * T)]
    c = [float(v) for v in (c if not np.isscalar(c) else [c] * T)]
    ys = [np.asarray(sample(i), dtype=np.float64).copy() for i in range(n_cal)]
    kappa, y0s, ks, norms, vr, lqs, rels = [], [], [], [], [], [], []
    for t in range(T):
        Vs, Ds = [], []
        for y in ys:
            S = y.sum()
            D = n * y - S
            Ds.append(D)
            Vs.append(float((D * D).sum()))
        Vs = np.asarray(Vs)
        vr.append([float(Vs.min()), float(Vs.max())])
        a, b = Vs.min() / margin, Vs.max() * margin
        kap = 1.0 / math.sqrt(a * b)
        xs = np.geomspace(a * kap, b * kap, 2001)
        y0 = 1.0 if xs[-1] < 2.5 else math.sqrt(2.5 / xs[-1])
        if k_fixed is not None:
            k = int(k_fixed if np.isscalar(k_fixed) else k_fixed[t])
        else:
            k, y0 = _fewest_iterations(xs, k_max, tol_k, y0)
        al = [1.5] * k
        if relax and k_fixed is None:
            r = _relaxed_steps(xs, k_max, tol_k)
            if r is not None and len(r[1]) < k:
                y0, al = r
                k = len(al)
        q = learn(t, kap, kap * Vs, (a * kap, b * kap)) if learn is not None else None
        lqs.append(list(q) if q is not None else [0.0, 0.0, 0.0])
        if q is not None:
            k, al = 0, []
        rels.append(al)
        new = []
        for D, V in zip(Ds, Vs):
            h = invsqrt_half_at([k], [y0], [q], 0, kap * V, [al])
            u = D * (2.0 * math.sqrt(kap * n) / c[t]) * h + 1.0
            new.append(_power(u, p[t]))
        nm = 1.0
        if bootstrap:
            nm = 1.0 / (norm_margin * max(float(np.abs(v).max()) for v in new))
        ys = [v * nm for v in new]
        kappa.append(kap)
        y0s.append(y0)
        ks.append(k)
        norms.append(nm)
    Ss = np.asarray([float(y.sum()) for y in ys])
    af, bf = Ss.min() / margin, Ss.max() * margin
    kf = 2.0 / (af + bf)
    xs = np.linspace(af * kf, bf * kf, 2001)
    if d_fixed is not None:
        d = int(d_fixed)
    else:
        d = d_max
        for dd in range(1, d_max + 1):
            if _inv_err(xs, dd) < tol_d:
                d = dd
                break
    return CutMaxPlan(n=n, slots=slots, packing=packing_for(n, slots), T=T, p=p, c=c, k=ks,
                      kappa=kappa, y0=y0s, d=d, kappa_f=kf, bootstrap=bootstrap, norm=norms, cts=cts_for(n, slots),
                      lq=lqs if any(kk == 0 for kk in ks) else None, relax=rels if relax else None,
                      extra={"V_range": vr, "S_range": [float(Ss.min()), float(Ss.max())], "margin": margin,
                             "n_cal": n_cal})
