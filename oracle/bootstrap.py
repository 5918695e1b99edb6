"""CKKS bootstrapping on oracle operations (plain, by definition).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper refreshes ciphertexts whose levels run out "via bootstrap" (App.
B.1, "Multiplication Depth"); this is the textbook full-slot procedure for
real messages:

  ModRaise   level-0 ciphertext lifted to the top modulus: decrypts to
             t = m + q0*I with a small integer polynomial I.
  CoeffToSlot  slots <- w(t)/(q0 (K+1)), w_k = t_k + i t_(k+h), as the dense
             matrix V^H (V[j,k] = xi_j^k, xi_j the slot roots; V^-1 = V^H / h
             since V V^H = h I) evaluated by baby-step giant-step over its h
             diagonals, then the scalar S/(h q0 (K+1)) with the scale taking
             up the rounding of that scalar exactly; one more level is dropped
             so the level count matches the factored form.
  split      Re and Im parts with one conjugation (the factor 1/2 is taken
             into the scale); multiplying by -i is X^(3N/2).
  EvalMod    x -> cos(2 pi ((K+1) x - 1/4) / 2^r) by its Chebyshev series
             of degree d (T_k by T_(a+b) = 2 T_a T_b - T_(a-b)), then r double
             angles c <- 2c^2 - 1, giving sin(2 pi t/q0) ~ 2 pi (t/q0 - I).
  SlotToCoeff  slots <- (q0/(2 pi S)) V w', dense, BSGS, two levels dropped.
The output encrypts the input message at a known scale.

For a ciphertext whose slots all hold one complex value (the plaintext
a + b X^(N/2), a scalar of the CutMax circuit), `bootstrap_const` replaces
CoeffToSlot by the trace over the automorphisms X -> X^(5^k), k < N/2, which
keeps exactly the coefficients of 1 and X^(N/2) of t, puts their real and
imaginary parts into the two slot halves for one EvalMod, corrects the sine
by one Taylor step of arcsin (a constant's value sits whole in coefficient 0),
and puts the value back in every slot.
"""
import math

import numpy as np

from . import encoding as enc
from .circuit import HE


def slot_roots_matrix(log_n):
    """V[j, k] = xi_j^k, xi_j = exp(i pi (5^j mod 2N) / N), j, k < N/2."""
    n = 1 << log_n
    h = n // 2
    e = np.empty(h, dtype=np.int64)
    g = 1
    for j in range(h):
        e[j] = g
        g = (g * 5) % (2 * n)
    k = np.arange(h)
    return np.exp(1j * np.pi * ((np.outer(e, k)) % (2 * n)) / n)


def chebyshev_coeffs(f, d):
    """Interpolation at the d+1 Chebyshev nodes: f(x) ~ sum_k c_k T_k(x)."""
    j = np.arange(d + 1)
    th = np.pi * (j + 0.5) / (d + 1)
    fx = f(np.cos(th))
    c = np.array([2.0 / (d + 1) * np.sum(fx * np.cos(k * th)) for k in range(d + 1)])
    c[0] /= 2
    return c


def trace(ctx, ct):
    """Sum over k < N/2 of the automorphism X -> X^(5^k) applied to ct, as
    the doubling sum x <- x + rot(x, 2^i), i < log2(N/2) (5 has order N/2 mod
    2N).  Its plaintext is (N/2) (t_0 + t_(N/2) X^(N/2)): the orbit sum of any
    other monomial vanishes at every root of X^N + 1."""
    x, r = ct, 1
    while r < ctx.n // 2:
        x = ctx.add(x, ctx.rotate(x, r))
        r *= 2
    return x


def evalmod_function(K, r):
    return lambda x: np.cos(2 * np.pi * ((K + 1) * x - 0.25) / (2 ** r))


class Bootstrapper:
    """Dense-matrix bootstrapping for small ring degrees (h <= 2048 slots)."""

    def __init__(self, ctx, K, r, d, s_fix=2.0 ** 40, target=2.0 ** 60, out_scale=2.0 ** 40):
        self.ctx, self.K, self.r, self.d = ctx, K, r, d
        self.s_fix, self.target, self.out_scale = s_fix, target, out_scale
        self.he = HE(ctx, target)
        n = ctx.n
        self.h = n // 2
        q0 = ctx.primes[0]
        V = slot_roots_matrix(ctx.log_n)
        self.vh = V.conj().T
        self.cts_scalar = s_fix / (self.h * q0 * (K + 1))
        self.stc = (q0 / (2 * np.pi * s_fix)) * V
        self.cheb = chebyshev_coeffs(evalmod_function(K, r), d)
        self.bs = 1 << int(math.ceil(math.log2(math.sqrt(self.h))))

    def out_level(self):
        """Level of a bootstrapped ciphertext: 3 + ceil(log2(d+1)) + 1 + r + 3 below the top."""
        return self.ctx.nq - 1 - 6 - (math.ceil(math.log2(self.d + 1)) + 1 + self.r)

    def rotations(self):
        h, bs = self.h, self.bs
        rots = set(range(1, bs)) | set(range(bs, h, bs))
        return sorted(rots)

    def gen_keys(self):
        self.ctx.gen_relin_key()
        for r in self.rotations():
            self.ctx.gen_rot_key(r)
        self.ctx.gen_galois_key(self.ctx.conj_galois())

    def _diag(self, M, r):
        h = self.h
        i = np.arange(h)
        return M[i, (i + r) % h]

    def linear(self, ct, M, target):
        """sum_r diag_r(M) * rot(ct, r) by baby-step giant-step, one rescale."""
        ctx, h, bs = self.ctx, self.h, self.bs
        q = float(ctx.primes[ct.level])
        E = (target * q) / ct.scale
        baby = [ct] + [ctx.rotate(ct, b) for b in range(1, bs)]
        acc = None
        for G in range(0, h, bs):
            inner = None
            for b in range(bs):
                dg = np.roll(self._diag(M, G + b), G)       # diag'[i] = diag[i - G]
                if np.abs(dg).max() == 0:
                    continue
                t = ctx.mul_plain(baby[b], enc.encode(dg, ctx.log_n, E), ct.scale * E)
                inner = t if inner is None else ctx.add(inner, t)
            if inner is None:
                continue
            if G:
                inner = ctx.rotate(inner, G)
            acc = inner if acc is None else ctx.add(acc, inner)
        return ctx.rescale(acc)

    def exact_scalar(self, ct, c, target):
        """ct * c, rescaled, with the scale taking up the rounding of c exactly."""
        ctx = self.ctx
        q = float(ctx.primes[ct.level])
        E = (target * q) / ct.scale
        K = float(np.rint(c * E))
        return ctx.rescale(ctx.mul_intd(ct, K, ct.scale * (K / c)))

    def evalmod(self, x):
        he, ctx = self.he, self.ctx
        T = {1: x}
        for k in range(2, self.d + 1):
            a, b = (k + 1) // 2, k // 2
            P2 = ctx.mul_int(he.mul_rescale(T[a], T[b]), 2)
            if a == b:
                T[k] = he.add_const(P2, -1.0)
            else:
                xm = ctx.drop(he.mcr(T[1], 1.0, P2.scale), P2.level)
                T[k] = ctx.sub(P2, xm)
        terms = [he.mcr(T[k], float(self.cheb[k]), self.target) for k in range(1, self.d + 1)]
        low = min(t.level for t in terms)
        acc = None
        for t in terms:
            t = ctx.drop(t, low) if t.level > low else t
            acc = t if acc is None else ctx.add(acc, t)
        c = he.add_const(acc, float(self.cheb[0]))
        for _ in range(self.r):
            c = he.add_const(ctx.mul_int(he.mul_rescale(c, c), 2), -1.0)
        return c

    def bootstrap(self, ct):
        ctx = self.ctx
        ratio = ct.scale / self.s_fix
        low = ctx.drop(ct, 0) if ct.level else ct
        up = ctx.mod_raise(low)
        up.set_scale(self.s_fix)
        # the Re/Im split doubles the declared scale, so aim CoeffToSlot at half
        # the EvalMod scale: EvalMod then squares ciphertexts whose scale is
        # close to its primes and the scale stays put
        y = self.linear(up, self.vh, 2.0 ** 40)
        x = self.exact_scalar(y, self.cts_scalar, self.target / 2)
        x = ctx.drop(x, x.level - 1)
        xc = ctx.conj(x)
        re = ctx.add(x, xc)
        re.set_scale(2 * re.scale)
        im = ctx.mul_monomial(ctx.sub(x, xc), 3 * ctx.n // 2)
        im.set_scale(2 * im.scale)
        re, im = self.evalmod(re), self.evalmod(im)
        w = ctx.add(re, ctx.mul_monomial(im, ctx.n // 2))
        out = self.linear(w, self.stc, self.out_scale)
        out = ctx.drop(out, out.level - 2)
        # the slots read m / s_fix = (message) * ratio: declaring the scale
        # ratio times larger reads the message
        out.set_scale(out.scale * ratio)
        return out

    def gen_const_keys(self):
        """Rotation keys of the trace (1, 2, ..., N/4)."""
        r = 1
        while r < self.h:
            self.ctx.gen_rot_key(r)
            r *= 2

    def bootstrap_const(self, ct):
        """Refresh of one complex value in every slot; output at out_level()
        and at the input's scale."""
        ctx, he = self.ctx, self.he
        q0 = ctx.primes[0]
        ratio = ct.scale / self.s_fix
        low = ctx.drop(ct, 0) if ct.level else ct
        up = ctx.mod_raise(low, ctx.nq - 3)
        up.set_scale(q0 * (self.K + 1))
        x = trace(ctx, up)
        x.set_scale(x.scale * self.h)           # slots: (t_0 + i t_(N/2)) / (q0 (K+1))
        xc = ctx.conj(x)
        re = ctx.add(x, xc)
        re.set_scale(2 * re.scale)
        im = ctx.mul_monomial(ctx.sub(x, xc), 3 * ctx.n // 2)
        im.set_scale(2 * im.scale)
        half = self.h // 2
        lo = np.concatenate([np.ones(half), np.zeros(half)])
        y = ctx.add(he.mul_plain_rescale(re, lo, self.target), he.mul_plain_rescale(im, 1.0 - lo, self.target))
        y = self.evalmod(y)                     # sin(theta), theta = 2 pi m / q0
        y2 = he.mul_rescale(y, y)
        y2.set_scale(6 * y2.scale)
        y = he.mul_rescale(y, he.add_const(y2, 1.0))   # arcsin to third order
        w = ctx.add(y, ctx.mul_monomial(ctx.rotate(y, half), ctx.n // 2))
        w = he.mul_plain_rescale(w, lo, q0 / (2 * np.pi))
        w = ctx.add(w, ctx.rotate(w, half))
        w.set_scale(w.scale * 2 * np.pi * self.s_fix / q0 * ratio)
        out = self.out_level()
        return ctx.drop(w, out) if w.level > out else w
