"""Alg. 2 (HE CutMax) and Alg. 3 (one-shot nucleus sampling) on oracle CKKS ops.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Scale rule.  Every ciphertext carries its exact scale.  A multiplication by a
real constant c at level l (prime q = q_l) towards a target scale `target`
encodes E = (target*q)/scale, multiplies by K = rint(c*E), sets the scale to
scale*E and rescales (scale/q).  Adding a constant c adds rint(c*scale) to
the constant coefficient.  Ciphertext products multiply scales, rescale
divides by q_l.  These float64 steps are written in exactly this order on both
implementations.

Circuit (iteration t; Y at level l):
  S  = rotsum(Y)                       sum_i Y_i in every slot (App. D)
  D  = n*Y - S                         n*(Y - mu), no level
  E  = rescale(D*D)
  V  = rotsum(E) [- m*rescale(S*S)]    n^3 sigma^2 (m zero-padded slots)
  h  = Goldschmidt 1/(2 sqrt(kappa V)) in k iterations, 2 levels each
  D' = D * 2 sqrt(kappa n)/c           (times the 0/1 slot mask when padded)
  u  = D' * h + 1 (+ mask when padded) = (Y - mu)/(c sigma) + 1     (Alg. 2)
  Y  = u^p                             square and multiply
Final (Alg. 2 last step): S = rotsum(Y); a = 1 - kappa_f S;
  F = prod_{i<=d} (1 + a^(2^i)); Z = (kappa_f Y) * F.

A vocabulary longer than the slot count spreads over plan.cts ciphertexts
(entries c*slots .. in ciphertext c, the last zero-padded): every sum over
the vocabulary adds the ciphertexts before the rotate-and-sum, and S, h and F
then serve every ciphertext of the stream.
"""
import math

import numpy as np

from . import encoding as enc
from .cutmax_fp64 import relax_constants


ROTSUM_LOG_RADIX = 3


def rotsum_stages(steps, log_radix=ROTSUM_LOG_RADIX):
    """The rotate-and-sum over 2^steps slots as hoisted stages: stage i covers
    the doublings [i L, min((i+1) L, steps)) and adds the rotations by
    r 2^(i L), 0 < r < 2^len (L = log_radix)."""
    out = []
    for start in range(0, steps, log_radix):
        ln = min(log_radix, steps - start)
        out.append([r << start for r in range(1, 1 << ln)])
    return out


class HE:
    """Helpers implementing the scale rule over an oracle Context."""

    def __init__(self, ctx, delta, rotsum_log_radix=ROTSUM_LOG_RADIX):
        self.ctx = ctx
        self.delta = float(delta)
        self.rotsum_log_radix = rotsum_log_radix

    def q(self, level):
        return self.ctx.primes[level]

    def mcr(self, ct, c, target=None):
        target = self.delta if target is None else target
        q = float(self.q(ct.level))
        E = (target * q) / ct.scale
        K = float(np.rint(c * E))
        t = self.ctx.mul_intd(ct, K, ct.scale * E)
        return self.ctx.rescale(t)

    def mcr_bits(self, ct, c, target, min_bits):
        """c * ct with K = rint(c E) of at least min_bits bits: E spans as many
        primes r <= 3 (rescales) as that takes, E = target q_l..q_(l-r+1)/scale."""
        target = self.delta if target is None else target
        r = 1
        E = (target * float(self.q(ct.level))) / ct.scale
        while abs(c * E) < 2.0 ** min_bits and r < 3 and ct.level - r >= 1:
            E *= float(self.q(ct.level - r))
            r += 1
        K = float(np.rint(c * E))
        t = self.ctx.mul_intd(ct, K, ct.scale * E)
        for _ in range(r):
            t = self.ctx.rescale(t)
        return t

    def add_const(self, ct, c):
        return self.ctx.add_intd(ct, float(np.rint(c * ct.scale)))

    def neg(self, ct):
        return self.ctx.mul_int(ct, -1)

    def mul_rescale(self, a, b):
        """Product, relinearisation and rescale in one rounded division by q_l P."""
        ctx = self.ctx
        l = min(a.level, b.level)
        if a.level > l:
            a = ctx.drop(a, l)
        if b.level > l:
            b = ctx.drop(b, l)
        return ctx.mul_rescale(a, b)

    def mul_plain_rescale(self, ct, vec, target=None):
        target = self.delta if target is None else target
        q = float(self.q(ct.level))
        E = (target * q) / ct.scale
        pt = None if getattr(self.ctx, "dry", False) else enc.encode(vec, self.ctx.log_n, E)
        t = self.ctx.mul_plain(ct, pt, ct.scale * E)
        return self.ctx.rescale(t)

    def add_plain_vec(self, ct, vec):
        pt = None if getattr(self.ctx, "dry", False) else enc.encode(vec, self.ctx.log_n, ct.scale)
        return self.ctx.add_plain(ct, pt)

    def rotsum(self, ct, steps):
        """Every slot i gets the sum of slots i .. i + 2^steps - 1 (App. D), in
        hoisted stages (each x + sum_r rot(x, r) through one ModUp and one
        ModDown)."""
        for rots in rotsum_stages(steps, self.rotsum_log_radix):
            ct = self.ctx.rotsum_stage(ct, rots)
        return ct

    def power(self, u, p):
        sq, acc, pp = u, None, int(p)
        while True:
            if pp & 1:
                acc = sq if acc is None else self.mul_rescale(acc, sq)
            pp >>= 1
            if pp == 0:
                break
            sq = self.mul_rescale(sq, sq)
        return acc


def required_rotations(plan, log_radix=ROTSUM_LOG_RADIX):
    return sorted({r for rots in rotsum_stages(plan.rotsum_steps, log_radix) for r in rots})


def invsqrt_goldschmidt(he, V, kappa, y0, k, alphas=None):
    """h ~ 1/(2 sqrt(kappa V)), coupled Goldschmidt, 2k levels.  Step i
    multiplies by a = alpha_i - g h (alpha_i = 3/2 for Newton's step; other
    values are relaxation constants of the over-relaxed form App. B cites)."""
    al = [1.5] * max(k, 1) if alphas is None else list(alphas)
    a = he.add_const(he.mcr(V, -kappa * y0 * y0 / 2.0), al[0])
    h = he.mcr(a, y0 / 2.0)
    g = he.mul_rescale(he.mcr(V, kappa * y0), a) if k >= 2 else None
    for i in range(2, k + 1):
        a = he.add_const(he.neg(he.mul_rescale(g, h)), al[i - 1])
        if i < k:
            g = he.mul_rescale(g, a)
        h = he.mul_rescale(h, a)
    return h


def learned_half(he, x, abc):
    """(A x^2 + B x + C)/2: the learned inverse square root, two levels."""
    A, B, C = abc
    t2 = he.mcr_bits(he.mul_rescale(x, x), A / 2.0, None, 24)
    t1 = he.mcr_bits(x, B / 2.0, None, 24)
    l = min(t2.level, t1.level)
    t2 = he.ctx.drop(t2, l) if t2.level > l else t2
    t1 = he.ctx.drop(t1, l) if t1.level > l else t1
    return he.add_const(he.ctx.add(t2, t1), C / 2.0)


def inverse_goldschmidt(he, S, kappa_f, d):
    """F ~ 1/(kappa_f S) by prod_{i<=d}(1 + (1 - kappa_f S)^(2^i)); d + 2 levels."""
    a = he.add_const(he.mcr(S, -kappa_f), 1.0)
    F = he.add_const(a, 1.0)
    sq = a
    for _ in range(d):
        sq = he.mul_rescale(sq, sq)
        F = he.mul_rescale(F, he.add_const(sq, 1.0))
    return F


def _masks(plan):
    """Per-ciphertext 0/1 slot masks of a zero-padded stream (None if unpadded)."""
    if not plan.pad:
        return None
    k = getattr(plan, "cts", 1)
    flat = np.zeros(k * plan.slots)
    flat[:plan.n] = 1.0
    return [flat[c * plan.slots:(c + 1) * plan.slots] for c in range(k)]


def _vsum(ctx, cts):
    """Sum of the stream's ciphertexts (Y_0 + Y_1 + ...)."""
    acc = cts[0]
    for c in cts[1:]:
        acc = ctx.add(acc, c)
    return acc


def cutmax_he(he, ct, plan, bootstrap=None):
    """Alg. 2 over one stream: one ciphertext packed by ``plan.packing``, or a
    list of plan.cts zero-padded ciphertexts (the result is then a list)."""
    ctx = he.ctx
    many = isinstance(ct, (list, tuple))
    Ys = list(ct) if many else [ct]
    n, steps, m = plan.n, plan.rotsum_steps, plan.pad
    masks = _masks(plan)
    for t in range(plan.T):
        S = he.rotsum(_vsum(ctx, Ys), steps)
        Ds = [ctx.sub(ctx.mul_int(Y, n), S) for Y in Ys]
        Es = [he.mul_rescale(D, D) for D in Ds]
        V = he.rotsum(_vsum(ctx, Es), steps)
        if m:
            V = ctx.sub(V, ctx.mul_int(he.mul_rescale(S, S), m))
        if plan.k[t]:
            h = invsqrt_goldschmidt(he, V, plan.kappa[t], plan.y0[t], plan.k[t], relax_constants(plan, t))
        else:
            h = learned_half(he, he.mcr_bits(V, plan.kappa[t], None, 30), plan.lq[t])
        coef = 2.0 * math.sqrt(plan.kappa[t] * n) / plan.c[t]
        new = []
        for c, D in enumerate(Ds):
            # the 0/1 mask as a plaintext, coef as an integer multiplier (a
            # plaintext of coef-sized values would round to ~1e-5 relative)
            Dp = he.mcr(he.mul_plain_rescale(D, masks[c]) if m else D, coef)
            u = he.mul_rescale(Dp, h)
            u = he.add_plain_vec(u, masks[c]) if m else he.add_const(u, 1.0)
            new.append(he.power(u, plan.p[t]))
        Ys = new
    S = he.rotsum(_vsum(ctx, Ys), steps)
    F = inverse_goldschmidt(he, S, plan.kappa_f, plan.d)
    Z = [he.mul_rescale(he.mcr(Y, plan.kappa_f), F) for Y in Ys]
    return Z if many else Z[0]


# ------------------------------------------------------------------ bootstrapped form
class _SimCt:
    """Level and scale of a ciphertext, nothing else (see LevelSim)."""
    __slots__ = ("level", "scale")

    def __init__(self, level, scale):
        self.level, self.scale = level, float(scale)

    def set_scale(self, s):
        self.scale = float(s)


class LevelSim:
    """A Context that keeps only the level and scale of every ciphertext
    (each operation updates them exactly as the real one does) and counts key
    switches by level: one per product, one per rotation or conjugation.  The
    refresh schedule plays the circuit on it."""
    dry = True

    def __init__(self, primes, nq, log_n):
        self.primes, self.nq, self.log_n = list(primes), nq, log_n
        self.n, self.slots, self.top_level = 1 << log_n, 1 << (log_n - 1), nq - 1
        self.ks = {}

    def _ks(self, level):
        self.ks[level] = self.ks.get(level, 0) + 1

    def mul_intd(self, a, K, scale_out):
        return _SimCt(a.level, scale_out)

    def mul_plain(self, a, pt, scale_out):
        return _SimCt(a.level, scale_out)

    def mul_int(self, a, k):
        return _SimCt(a.level, a.scale)

    def add_intd(self, a, K):
        return _SimCt(a.level, a.scale)

    def add_plain(self, a, pt):
        return _SimCt(a.level, a.scale)

    def mul_monomial(self, a, e):
        return _SimCt(a.level, a.scale)

    def rescale(self, a):
        if a.level < 1:
            raise ValueError("rescale at level 0")
        return _SimCt(a.level - 1, a.scale / float(self.primes[a.level]))

    def drop(self, a, level):
        return _SimCt(level, a.scale)

    def add(self, a, b):
        return _SimCt(min(a.level, b.level), a.scale)

    sub = add

    def mul(self, a, b):
        l = min(a.level, b.level)
        self._ks(l)
        return _SimCt(l, a.scale * b.scale)

    def mul_rescale(self, a, b):
        return self.rescale(self.mul(a, b))

    def automorphism(self, a, g):
        self._ks(a.level)
        return _SimCt(a.level, a.scale)

    def rotate(self, a, r):
        return self.automorphism(a, 0)

    def rotsum_stage(self, a, rots):
        self.ks[a.level] = self.ks.get(a.level, 0) + len(rots)
        return _SimCt(a.level, a.scale)

    def conj(self, a):
        return self.automorphism(a, 0)


class _DryBoot:
    """Bootstrapping stand-in for LevelSim: output level, input scale, counts."""

    def __init__(self, out_level):
        self._out = out_level
        self.general = self.const = 0

    def out_level(self):
        return self._out

    def bootstrap(self, ct):
        self.general += 1
        return _SimCt(self._out, ct.scale)

    def bootstrap_const(self, ct):
        self.const += 1
        return _SimCt(self._out, ct.scale)


class CountingBoot:
    """Wraps a Bootstrapper and counts its general and constant refreshes."""

    def __init__(self, boot):
        self.boot = boot
        self.general = self.const = 0

    def out_level(self):
        return self.boot.out_level()

    def bootstrap(self, ct):
        self.general += 1
        return self.boot.bootstrap(ct)

    def bootstrap_const(self, ct):
        self.const += 1
        return self.boot.bootstrap_const(ct)


class CountingCtx:
    """Forwards to a Context and counts the circuit's own key switches by
    level (the bootstrapper keeps the bare Context, so its rotations are not
    counted here)."""

    def __init__(self, ctx):
        self._ctx = ctx
        self.ks = {}

    def __getattr__(self, name):
        return getattr(self._ctx, name)

    def _ks(self, level):
        self.ks[level] = self.ks.get(level, 0) + 1

    def mul(self, a, b):
        self._ks(min(a.level, b.level))
        return self._ctx.mul(a, b)

    def mul_rescale(self, a, b):
        self._ks(min(a.level, b.level))
        return self._ctx.mul_rescale(a, b)

    def automorphism(self, a, g):
        self._ks(a.level)
        return self._ctx.automorphism(a, g)

    def rotate(self, a, r):
        self._ks(a.level)
        return self._ctx.rotate(a, r)

    def rotsum_stage(self, a, rots):
        self.ks[a.level] = self.ks.get(a.level, 0) + len(rots)
        return self._ctx.rotsum_stage(a, rots)

    def conj(self, a):
        self._ks(a.level)
        return self._ctx.conj(a)


def _imag2(ctx, a):
    """2 Im(a) of a complex constant a, as a real constant: (a - conj a)(-i),
    -i being the monomial X^(3N/2)."""
    return ctx.mul_monomial(ctx.sub(a, ctx.conj(a)), 3 * ctx.n // 2)


def _boot_circuit(he, ct, plan, boot, h_refresh, y_boot, tally):
    """The bootstrapped CutMax of one stream: Alg. 2 with refreshes, the
    Goldschmidt input x = kappa V, Y_(t+1) scaled by norm[t] through
    u' = norm^(1/p) u.  The stream is one ciphertext, or a list of plan.cts
    zero-padded ones (a vocabulary longer than the slot count; the sums add
    the ciphertexts before the rotate-and-sum, the scalars serve all of them,
    and the result is then a list).  The vectors (Y, D', u) take the general
    bootstrap (all of a stream's ciphertexts at once: tally['vector'] counts
    these refreshes, one per event); the scalars (x, the Goldschmidt pair, h,
    the final sum), which hold one value in every slot, the constant
    bootstrap.  The Goldschmidt
    pair (g, h) travels as one complex constant z = g + i h/4: one product z^2,
    one conjugation (2 Im(z^2) = g h, the 1/4 keeping the scale of every step
    at s^3/(q q')), then z <- z (1.5 - g h); h = 4 Im z.  Each refresh inside
    the iteration is followed by a multiplication by 1 that lands on Delta.
    Refreshes: Y before the statistics when it has fewer than 5 levels (V
    needs up to 3 rescales to reach x ~ 1 with a 30-bit multiplier) or when
    y_boot[t] asks; x when it has fewer than 2 (tally['x'] counts these); z
    between steps when it has fewer than 2 and before h is read when it has
    none; h when it has none, or when h_refresh[t] asks and h sits below D';
    D' and h before their product (1), u before the power (ceil log2 p), Y
    before the final sum (2), the final sum before the inverse (d + 3)."""
    ctx = he.ctx
    many = isinstance(ct, (list, tuple))
    cts = list(ct) if many else [ct]
    n, steps, m = plan.n, plan.rotsum_steps, plan.pad
    masks = _masks(plan)

    def ensure(c, need):
        return boot.bootstrap(c) if c.level < need else c

    def vrefresh(cs):
        tally["vector"] = tally.get("vector", 0) + 1
        return [boot.bootstrap(c) for c in cs]

    def vensure(cs, need):
        return vrefresh(cs) if cs[0].level < need else cs

    out = boot.out_level()
    Y = [ctx.drop(c, out) if c.level > out else c for c in cts]
    for t in range(plan.T):
        p, k, kap, y0 = plan.p[t], plan.k[t], plan.kappa[t], plan.y0[t]
        rn = plan.norm[t] ** (1.0 / p)
        if Y[0].level < 5 or y_boot[t]:
            Y = vrefresh(Y)
        S = he.rotsum(_vsum(ctx, Y), steps)
        D = [ctx.sub(ctx.mul_int(y, n), S) for y in Y]
        V = he.rotsum(_vsum(ctx, [he.mul_rescale(d, d) for d in D]), steps)
        if m:
            V = ctx.sub(V, ctx.mul_int(he.mul_rescale(S, S), m))
        x = he.mcr_bits(V, kap, None, 30)
        if x.level < 2:
            tally["x"] = tally.get("x", 0) + 1
            x = boot.bootstrap_const(x)
        coef = 2.0 * math.sqrt(kap * n) / plan.c[t] * rn
        Dp = [he.mcr(he.mul_plain_rescale(d, masks[c]), coef) if m else he.mcr(d, coef) for c, d in enumerate(D)]
        if k == 0:
            h = learned_half(he, x, plan.lq[t])
        else:
            al = relax_constants(plan, t)
            a = he.add_const(he.mcr(x, -y0 * y0 / 2.0), al[0])
            z = he.add_plain_vec(he.mcr(x, y0), np.full(plan.slots, 1j * y0 / 8.0))
            z = he.mul_rescale(z, a)
            for i in range(2, k + 1):
                if z.level < 2:
                    z = he.mcr(boot.bootstrap_const(z), 1.0)
                gh = _imag2(ctx, he.mul_rescale(z, z))
                z = he.mul_rescale(z, he.add_const(he.neg(gh), al[i - 1]))
            if z.level < 1:
                z = boot.bootstrap_const(z)
            h = ctx.mul_int(_imag2(ctx, z), 2)
        if (h_refresh[t] and h.level < Dp[0].level) or h.level < 1:
            h = boot.bootstrap_const(h)
        h, Dp = ensure(h, 1), vensure(Dp, 1)
        u = [he.mul_rescale(d, h) for d in Dp]
        u = [he.add_plain_vec(uu, rn * masks[c]) if m else he.add_const(uu, rn) for c, uu in enumerate(u)]
        u = vensure(u, (p - 1).bit_length())
        Y = [he.power(uu, p) for uu in u]
    Y = vensure(Y, 2)
    S = he.rotsum(_vsum(ctx, Y), steps)
    if S.level < plan.d + 3:
        S = boot.bootstrap_const(S)
    F = inverse_goldschmidt(he, S, plan.kappa_f, plan.d)
    Z = [he.mul_rescale(he.mcr(y, plan.kappa_f), F) for y in Y]
    return Z if many else Z[0]


def refresh_schedule(he, ct, plan, out_level):
    """The optional refreshes of the bootstrapped circuit, chosen by playing
    every combination on LevelSim: per iteration t, refresh h when it sits
    below D' (h_refresh[t]), and bootstrap Y before the statistics although it
    has the levels they need (y_boot[t]); 4^T combinations for T <= 6, 2^T
    (h only) for 6 < T <= 16, none beyond.  The cheapest counts a general
    bootstrap 7, a constant one 3 (their cost ratio on the GPU the circuit
    targets) and a refresh of x 3000 (x reaches tens,
    beyond what a refresh of a constant keeps accurate); ties go to fewer
    bootstraps, then to the first combination (t = 0 the least significant
    digit, bit 0 h_refresh, bit 1 y_boot)."""
    T = plan.T
    if T > 16:
        return [0] * T, [0] * T
    per = 4 if T <= 6 else 2
    ctx = he.ctx
    primes = list(ctx.primes)
    many = isinstance(ct, (list, tuple))
    start = [_SimCt(min(c.level, out_level), c.scale) for c in ct] if many else _SimCt(min(ct.level, out_level),
                                                                                       ct.scale)
    best, best_key = None, None
    for combo in range(per ** T):
        cc, hr, yb = combo, [], []
        for _ in range(T):
            ch = cc % per
            cc //= per
            hr.append(ch & 1)
            yb.append(1 if ch & 2 else 0)
        sim = LevelSim(primes, ctx.nq, ctx.log_n)
        dry = _DryBoot(out_level)
        tally = {}
        _boot_circuit(HE(sim, he.delta, he.rotsum_log_radix), start, plan, dry, hr, yb, tally)
        general = tally.get("vector", 0)          # a stream's vector refresh is one event
        cost = 7 * general + 3 * dry.const + 3000 * tally.get("x", 0)
        key = (cost, general + dry.const)
        if best_key is None or key < best_key:
            best, best_key = (hr, yb), key
    return best


def cutmax_he_boot(he, ct, plan, boot, stats=None):
    """Alg. 2 with bootstrapping (see _boot_circuit), the optional refreshes
    picked by refresh_schedule.  boot: a Bootstrapper (oracle/bootstrap.py).
    stats (a dict, optional) receives the schedule, the general and constant
    refreshes made and the circuit's own key switches by level."""
    many = isinstance(ct, (list, tuple))
    if (len(ct) if many else 1) != getattr(plan, "cts", 1):
        raise ValueError("a stream is plan.cts ciphertexts (a list when more than one)")
    hr, yb = refresh_schedule(he, ct, plan, boot.out_level())
    cctx, cboot = CountingCtx(he.ctx), CountingBoot(boot)
    tally = {}
    out = _boot_circuit(HE(cctx, he.delta, he.rotsum_log_radix), ct, plan, cboot, hr, yb, tally)
    if stats is not None:
        stats.update(h_refresh=hr, y_boot=yb, general=cboot.general, const=cboot.const, x_refresh=tally.get("x", 0),
                     vector_refreshes=tally.get("vector", 0), ks=dict(cctx.ks))
    return out


def chebyshev_interpolant(f, d):
    """c_0..c_d with f(t) ~ sum_k c_k T_k(t) on [-1, 1]: the interpolant of f
    at the d + 1 Chebyshev nodes t_j = cos(pi (j + 1/2) / (d + 1)), whose
    coefficients follow from the discrete orthogonality of T_0..T_d there."""
    j = np.arange(d + 1)
    th = np.pi * (j + 0.5) / (d + 1)
    fx = f(np.cos(th))
    c = np.array([2.0 / (d + 1) * np.sum(fx * np.cos(k * th)) for k in range(d + 1)])
    c[0] /= 2
    return c


def chebyshev_sum(he, x, c, target):
    """sum_k c_k T_k(x) of a ciphertext whose slots lie in [-1, 1]: every T_k
    by T_(a+b) = 2 T_a T_b - T_(a-b) with a = ceil(k/2), b = floor(k/2)
    (depth ceil(log2 k)), each term c_k T_k multiplied towards `target`, the
    terms summed on the lowest level, then c_0 added."""
    ctx = he.ctx
    T = {1: x}
    for k in range(2, len(c)):
        a, b = (k + 1) // 2, k // 2
        P2 = ctx.mul_int(he.mul_rescale(T[a], T[b]), 2)
        if a == b:
            T[k] = he.add_const(P2, -1.0)
        else:
            xm = he.mcr(T[1], 1.0, P2.scale)
            T[k] = ctx.sub(P2, ctx.drop(xm, P2.level) if xm.level > P2.level else xm)
    terms = [he.mcr(T[k], float(c[k]), target) for k in range(1, len(c)) if c[k] != 0.0]
    low = min(t.level for t in terms)
    acc = None
    for t in terms:
        t = ctx.drop(t, low) if t.level > low else t
        acc = t if acc is None else ctx.add(acc, t)
    return he.add_const(acc, float(c[0]))


def beta_noise_he(he, u, alpha, d):
    """Alg. 3's cut noise G = U^(1/alpha) (the inverse CDF of Beta(alpha, 1),
    Lemma 2 / Observation 1) evaluated on encrypted uniforms U in [0, 1]:
    t = 2U - 1 at U's own scale, then the degree-d Chebyshev interpolant of
    ((t + 1)/2)^(1/alpha), landing on he.delta.  (The paper fixes no scale for
    this step; working at U's scale lets uniforms encrypted on large primes keep
    their scale through the products.)"""
    if not alpha > 0 or not 2 <= d <= 127:
        raise ValueError("alpha must be positive and the degree in 2..127")
    c = chebyshev_interpolant(lambda t: ((t + 1.0) / 2.0) ** (1.0 / alpha), d)
    t = he.add_const(he.mcr(u, 2.0, u.scale), -1.0)
    return chebyshev_sum(he, t, c, he.delta)


def nucleus_alpha(top_p, q=0.0):
    """alpha = ln(1 - q) / ln(p), so that P(G > p) = q for G ~ Beta(alpha, 1)
    (Lemma 2 with q = p, Observation 1 for any q; q = 0 reads as q = p)."""
    q = top_p if not q else q
    return math.log(1.0 - q) / math.log(top_p)


def nucleus_he(he, ct_logits, ct_rand, plan, top_p=None, q=0.0, kind="beta", degree=31):
    """Alg. 3: X~ = X + G, then CutMax.  kind "beta": ct_rand encrypts G
    itself; "uniform": ct_rand encrypts uniforms U and G = U^(1/alpha) is
    evaluated here (beta_noise_he, alpha from top_p and q)."""
    G = ct_rand
    if kind == "uniform":
        G = beta_noise_he(he, ct_rand, nucleus_alpha(top_p, q), degree)
    return cutmax_he(he, he.ctx.add(ct_logits, G), plan)


def _shared_circuit(he, cts, plan, boot, h_refresh, y_boot):
    """The bootstrapped CutMax of S streams (S >= 2) with the scalar chains
    shared; cts[s] is stream s: one ciphertext, or a list of plan.cts
    zero-padded ones (its sums add them before the rotate-and-sum, its
    scalars serve all of them; the result per stream then is a list).  The
    scalars that every stream holds in all of its slots (x, the Goldschmidt
    pair and h, the final sum and its inverse) are packed into one ciphertext,
    stream s in the slot class i = s (mod S'), S' = S rounded up to a power of
    two (a 0/1 class mask per stream, then the sum over the streams: 1 level);
    one chain serves them all, and each stream takes its value back (its class
    mask, then a log2 S'-step rotate-and-sum: 1 level).  The packed Goldschmidt
    pair lies in the slot halves, g = x y0 in [0, s/2) and h = y0/2 in
    [s/2, s); a rotation by s/2 lines the halves up for g h.  Every refresh is
    the general bootstrap: the vectors' (one per ciphertext of every stream),
    the packed chain's (one), a stream's x before packing (one per stream).
    Engineering beyond the paper (which evaluates one stream at a time); the
    steps are those of cutmax_he_boot otherwise (Alg. 2, Sect. 3.2; App. B's
    Goldschmidt steps with the plan's relaxation constants).
    Refreshes: Y before the statistics when it has fewer than 5 levels or
    y_boot[t] asks; each stream's x when it has none, the packed x when it has
    fewer than 2; the pair between steps when it has fewer than 2 (then
    multiplied by 1 to land on Delta) and when it has none before h is read;
    the packed h before unpacking when it has none, or when h_refresh[t] asks
    and it would arrive below D'; an unpacked h and D' before their product
    (1); u before the power (ceil log2 p); Y before the final sum (2); the
    packed final sum before the inverse (d + 3); the inverse after it (2) and
    once unpacked (1)."""
    ctx = he.ctx
    S = len(cts)
    many = isinstance(cts[0], (list, tuple))
    Ys = [list(c) if many else [c] for c in cts]
    n, steps, m = plan.n, plan.rotsum_steps, plan.pad
    slots, half = plan.slots, plan.slots // 2
    masks = _masks(plan)
    Sp, lsp = 1, 0
    while Sp < S:
        Sp, lsp = 2 * Sp, lsp + 1
    cls = []
    for s in range(S):
        c = np.zeros(slots)
        c[s::Sp] = 1.0
        cls.append(c)

    def ensure(c, need):
        return boot.bootstrap(c) if c.level < need else c

    def ensure_all(cs, need):
        return [ensure(c, need) for c in cs]

    def ensure_streams(streams, need):
        return [ensure_all(cs, need) for cs in streams]

    def pack(cs):
        acc = None
        for s, c in enumerate(cs):
            t = he.mul_plain_rescale(c, cls[s])
            acc = t if acc is None else ctx.add(acc, t)
        return acc

    def unpack(c):
        return [he.rotsum(he.mul_plain_rescale(c, cls[s]), lsp) for s in range(S)]

    out = boot.out_level()
    Y = [[ctx.drop(c, out) if c.level > out else c for c in cs] for cs in Ys]
    for t in range(plan.T):
        p, k, kap, y0 = plan.p[t], plan.k[t], plan.kappa[t], plan.y0[t]
        rn = plan.norm[t] ** (1.0 / p)
        if Y[0][0].level < 5 or y_boot[t]:
            Y = [[boot.bootstrap(y) for y in cs] for cs in Y]
        Ssum = [he.rotsum(_vsum(ctx, cs), steps) for cs in Y]
        D = [[ctx.sub(ctx.mul_int(y, n), Ssum[s]) for y in cs] for s, cs in enumerate(Y)]
        V = [he.rotsum(_vsum(ctx, [he.mul_rescale(d, d) for d in ds]), steps) for ds in D]
        if m:
            V = [ctx.sub(v, ctx.mul_int(he.mul_rescale(s_, s_), m)) for v, s_ in zip(V, Ssum)]
        x = pack(ensure_all([he.mcr_bits(v, kap, None, 30) for v in V], 1))
        if x.level < 2:
            x = boot.bootstrap(x)
        coef = 2.0 * math.sqrt(kap * n) / plan.c[t] * rn
        Dp = [[he.mcr(he.mul_plain_rescale(d, masks[c]), coef) if m else he.mcr(d, coef) for c, d in enumerate(ds)]
              for ds in D]
        if k == 0:
            hp = learned_half(he, x, plan.lq[t])
        else:
            al = relax_constants(plan, t)
            vlo, vhi = np.zeros(slots), np.zeros(slots)
            vlo[:half], vhi[half:] = y0, y0 / 2.0
            a = he.add_const(he.mcr(x, -y0 * y0 / 2.0), al[0])
            P = he.mul_rescale(he.add_plain_vec(he.mul_plain_rescale(x, vlo), vhi), a)
            for i in range(2, k + 1):
                if P.level < 2:
                    P = he.mcr(boot.bootstrap(P), 1.0)
                Q = he.mul_rescale(P, ctx.rotate(P, half))
                P = he.mul_rescale(P, he.add_const(he.neg(Q), al[i - 1]))
            P = ensure(P, 1)
            hi = np.zeros(slots)
            hi[half:] = 1.0
            hm = he.mul_plain_rescale(P, hi)
            hp = ctx.add(hm, ctx.rotate(hm, half))
        if h_refresh[t] and hp.level - 1 < Dp[0][0].level:
            hp = boot.bootstrap(hp)
        h = ensure_all(unpack(ensure(hp, 1)), 1)
        Dp = ensure_streams(Dp, 1)
        u = [[he.mul_rescale(d, h[s]) for d in ds] for s, ds in enumerate(Dp)]
        u = [[he.add_plain_vec(uu, rn * masks[c]) if m else he.add_const(uu, rn) for c, uu in enumerate(us)]
             for us in u]
        u = ensure_streams(u, (p - 1).bit_length())
        Y = [[he.power(uu, p) for uu in us] for us in u]
    Y = ensure_streams(Y, 2)
    Sp_ct = ensure(pack(ensure_all([he.rotsum(_vsum(ctx, cs), steps) for cs in Y], 1)), plan.d + 3)
    Fp = ensure(inverse_goldschmidt(he, Sp_ct, plan.kappa_f, plan.d), 2)
    F = ensure_all(unpack(Fp), 1)
    Y = ensure_streams(Y, 2)
    Z = [[he.mul_rescale(he.mcr(y, plan.kappa_f), F[s]) for y in cs] for s, cs in enumerate(Y)]
    return Z if many else [z[0] for z in Z]


def refresh_schedule_shared(he, cts, plan, out_level):
    """The optional refreshes of the shared-chain circuit, chosen by playing
    every combination of (h_refresh[t], y_boot[t]) on LevelSim (4^T for
    T <= 6, 2^T beyond, none past 16): the one that bootstraps the fewest
    ciphertexts wins (a refresh of the vectors counts one per stream, of the
    packed chain one); ties go to the first combination (t = 0 the least
    significant digit, bit 0 h_refresh, bit 1 y_boot)."""
    T = plan.T
    if T > 16:
        return [0] * T, [0] * T
    per = 4 if T <= 6 else 2
    ctx = he.ctx
    many = isinstance(cts[0], (list, tuple))
    start = [[_SimCt(min(c.level, out_level), c.scale) for c in cs] if many else _SimCt(min(cs.level, out_level),
                                                                                          cs.scale) for cs in cts]
    best, best_cost = None, None
    for combo in range(per ** T):
        cc, hr, yb = combo, [], []
        for _ in range(T):
            ch = cc % per
            cc //= per
            hr.append(ch & 1)
            yb.append(1 if ch & 2 else 0)
        dry = _DryBoot(out_level)
        _shared_circuit(HE(LevelSim(ctx.primes, ctx.nq, ctx.log_n), he.delta, he.rotsum_log_radix), start, plan,
                        dry, hr, yb)
        cost = dry.general + dry.const
        if best_cost is None or cost < best_cost:
            best, best_cost = (hr, yb), cost
    return best


def cutmax_he_boot_shared(he, cts, plan, boot, stats=None):
    """_shared_circuit with the refreshes refresh_schedule_shared picks; returns
    one output per stream (a ciphertext, or a list for multi-ciphertext streams).  stats (a dict, optional) receives the
    schedule and the number of ciphertexts bootstrapped."""
    many = isinstance(cts[0], (list, tuple))
    if len(cts) < 2 or any((len(c) if many else 1) != getattr(plan, "cts", 1) for c in cts):
        raise ValueError("the shared circuit takes two or more streams of plan.cts ciphertexts each")
    hr, yb = refresh_schedule_shared(he, cts, plan, boot.out_level())
    cboot = CountingBoot(boot)
    out = _shared_circuit(he, cts, plan, cboot, hr, yb)
    if stats is not None:
        stats.update(h_refresh=hr, y_boot=yb, bootstrapped=cboot.general + cboot.const)
    return out
