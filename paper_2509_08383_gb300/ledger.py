"""Operation-count model of the encrypted CutMax circuit.

Replays the level bookkeeping of the library's circuits (leveled Alg. 2, the
bootstrapped variant and bootstrapping itself) without any arithmetic and
counts the hybrid key switches at each level: one per ciphertext product
(relinearisation) and one per rotation or conjugation.  The counts say where
the time goes (key switching dominates every step of Alg. 2) and scale
per-operation timings to a whole decode.
"""
import math
from collections import Counter


def _stage_offsets(h, len_):
    return {0, (len_ // 2) % h, (-len_ // 2) % h}


def _group_offsets(h, lens):
    offs = {0}
    for L in lens:
        offs = {(a + b) % h for a in offs for b in _stage_offsets(h, L)}
    return offs


def _bsgs_counts(h, offs):
    """(used baby rotations, nonzero giant rotations) of one transform level."""
    so = [r - h if r > h // 2 else r for r in offs]
    u = 0
    for r in so:
        u = math.gcd(u, abs(r))
    u = u or 1
    ms = [r // u for r in so]
    mmin, mmax = min(ms), max(ms)
    span = mmax - mmin + 1
    bs = 1
    while bs * bs < 4 * span:              # babies are cheap (hoisted ModUp and ModDown)
        bs <<= 1
    babies, giants = set(), set()
    for m in ms:
        g, b = divmod(m - mmin, bs)
        if b:
            babies.add(b)
        G = (mmin + g * bs) * u
        if G % h:
            giants.add(g)
    return len(babies), len(giants)


def transform_rotations(log_n):
    """Key switches of the three CoeffToSlot and three SlotToCoeff levels."""
    h = 1 << (log_n - 1)
    s = log_n - 1
    g3 = s // 3
    g2 = (s - g3) // 2
    g1 = s - g3 - g2
    sizes = [g1, g2, g3]
    stc, cts = [], []
    st = 1
    for sz in sizes:
        lens = [1 << (st + k) for k in range(sz)]
        st += sz
        stc.append(sum(_bsgs_counts(h, _group_offsets(h, lens))))
    st = s
    for sz in sizes:
        lens = [1 << (st - k) for k in range(sz)]
        st -= sz
        cts.append(sum(_bsgs_counts(h, _group_offsets(h, lens))))
    return cts, stc


ROTSUM_LOG_RADIX = 3


def rotsum_keys(steps, log_radix=ROTSUM_LOG_RADIX):
    """Key applications of a rotate-and-sum over 2^steps slots in hoisted
    stages of radix 2^log_radix (the library's he_rotsum): 2^len - 1 per stage."""
    return sum((1 << min(log_radix, steps - s)) - 1 for s in range(0, steps, log_radix))


class Sim:
    """Level-only stand-in for a ciphertext context."""

    def __init__(self, nq, log_n, boot=None, log_radix=ROTSUM_LOG_RADIX):
        self.nq, self.log_n, self.boot = nq, log_n, boot
        self.log_radix = log_radix
        self.ks = Counter()
        self.n_boot = 0
        self.n_boot_const = 0             # of which constant bootstraps

    def mul(self, a, b):
        l = min(a, b)
        self.ks[l] += 1
        return l - 1                      # relinearise + rescale

    def rot(self, a):
        self.ks[a] += 1
        return a

    def _evalmod(self, lvl, d, r):
        """Baby-step giant-step Chebyshev series of degree d, then r double angles."""
        m = 1
        while m * m <= d + 1:
            m *= 2
        top = m
        while 2 * top <= d:
            top *= 2
        T = {1: lvl}

        def make(k):
            T[k] = self.mul(T[(k + 1) // 2], T[k // 2])

        for k in range(2, m):
            make(k)
        g = m
        while g <= top:
            make(g)
            g *= 2

        def ev(deg):
            if deg < m:
                return min(T[k] for k in range(1, deg + 1)) - 1
            G = m
            while 2 * G <= deg:
                G *= 2
            if deg == G:                  # constant quotient: a constant multiplication
                P = T[G] - 1
            else:
                P = self.mul(ev(deg - G), T[G])
            ev(G - 1)
            return P

        c = ev(d)
        for _ in range(r):
            c = self.mul(c, c)
        return c

    def bootstrap(self, a):
        K, r, d = self.boot
        self.n_boot += 1
        L = self.nq - 1
        cts, stc = transform_rotations(self.log_n)
        for i in range(3):
            self.ks[L - i] += cts[i]
        lvl = L - 3
        self.ks[lvl] += 1                 # conjugation
        for _ in range(2):                # EvalMod of the real and imaginary parts
            c = self._evalmod(lvl, d, r)
        for i in range(3):
            self.ks[c - i] += stc[i]
        return c - 3

    def bootstrap_const(self, a):
        """Bootstrapping of one complex value in every slot: trace, one EvalMod
        on the packed real and imaginary parts, unpacking; handed back at the
        general bootstrap's output level."""
        K, r, d = self.boot
        out = Sim(self.nq, self.log_n, self.boot).bootstrap(0)
        self.n_boot += 1
        self.n_boot_const += 1
        L = self.nq - 3                   # raised 2 levels below the top
        self.ks[L] += rotsum_keys(self.log_n - 1, self.log_radix) + 1  # trace, conjugation
        c = self._evalmod(L - 1, d, r)    # after the packing mask
        c = self.mul(c, c)                # arcsine step y (1 + y^2/6)
        c = self.mul(c + 1, c)
        self.ks[c] += 1                   # rotation by N/4 lining up the halves
        self.ks[c - 1] += 1               # replication after the mask
        return min(c - 1, out)


def refresh_schedule(plan, qb, y_level, out, padded):
    """The library's refresh schedule of a bootstrapped plan with per-stream
    scalar chains: per iteration, (refresh h by a constant bootstrap when it
    sits below D', bootstrap Y early), the combination of least cost (general
    bootstrap 7, constant 3; then fewer bootstraps; then the first) on the
    circuit's level bookkeeping (plans of more than 16 iterations: none)."""
    T = plan.T
    if T > 16:                            # no search: no optional refresh
        return [False] * T, [False] * T
    per = 4 if T <= 6 else 2

    def mcr_bits_level(a, c):
        r, e = 1, qb[a]
        while abs(c) * 2.0 ** e < 2.0 ** 30 and r < 3 and a - r >= 1:
            e += qb[a - r]
            r += 1
        return a - r

    best, best_key = 0, None
    for combo in range(per ** T):
        cc, Y, g, c = combo, y_level, 0, 0
        for t in range(T):
            ch = cc % per
            cc //= per
            hr, yb = ch & 1, ch & 2
            k, lp = plan.k[t], (int(plan.p[t]) - 1).bit_length()
            if Y < 5 or yb:
                Y, g = out, g + 1
            x = mcr_bits_level(Y - 1, plan.kappa[t])
            if x < 2:                           # x is too large to refresh well
                x, c = out, c + 1000
            if k == 0:
                h = x - 2
            else:
                z = x - 2
                for _ in range(2, k + 1):
                    if z < 2:
                        z, c = out - 1, c + 1
                    z -= 2
                if z < 1:
                    z, c = out, c + 1
                h = z
            Dp = Y - (2 if padded else 1)
            if hr and h < Dp:
                h, c = out, c + 1
            if h < 1:
                h, c = out, c + 1
            if Dp < 1:
                Dp, g = out, g + 1
            u = min(Dp, h) - 1
            if u < lp:
                u, g = out, g + 1
            Y = u - lp
        if Y < 2:
            Y, g = out, g + 1
        if Y < plan.d + 3:
            c += 1
        key = (7 * g + 3 * c, g + c)
        if best_key is None or key < best_key:
            best, best_key = combo, key
    hr, yb = [], []
    for t in range(T):
        ch = best % per
        best //= per
        hr.append(bool(ch & 1))
        yb.append(bool(ch & 2))
    return hr, yb


def refresh_schedule_shared(plan, qb, y_level, out, padded, members, streams):
    """The library's refresh schedule of a bootstrapped plan whose batch of
    `streams` streams (`members` ciphertexts) shares its scalar chains: per
    iteration, (refresh the packed h before unpacking it when it would arrive
    below D', bootstrap Y early), the combination that bootstraps the fewest
    ciphertexts (a vector refresh counts one per member, a stream's x before
    packing one per stream, the packed chain one; then the first).  Returns
    (h_refresh, y_boot, bootstrapped ciphertexts)."""
    T = plan.T
    if T > 16:
        return [False] * T, [False] * T, None
    per = 4 if T <= 6 else 2

    def mcr_bits_level(a, c):
        r, e = 1, qb[a]
        while abs(c) * 2.0 ** e < 2.0 ** 30 and r < 3 and a - r >= 1:
            e += qb[a - r]
            r += 1
        return a - r

    best, best_cost = 0, None
    for combo in range(per ** T):
        cc, Y, cost = combo, y_level, 0
        for t in range(T):
            ch = cc % per
            cc //= per
            hr, yb = ch & 1, ch & 2
            k, lp = plan.k[t], (int(plan.p[t]) - 1).bit_length()
            if Y < 5 or yb:
                Y, cost = out, cost + members
            x = mcr_bits_level(Y - 1, plan.kappa[t])
            if x < 1:
                x, cost = out, cost + streams
            x -= 1                                  # pack: the class mask
            if x < 2:
                x, cost = out, cost + 1
            if k == 0:
                h = x - 2
            else:
                z = x - 2                           # the pair after its start
                for _ in range(2, k + 1):
                    if z < 2:
                        z, cost = out - 1, cost + 1
                    z -= 2
                if z < 1:
                    z, cost = out, cost + 1
                h = z - 1                           # h's half of the pair
            Dp = Y - (2 if padded else 1)
            if hr and h - 1 < Dp:
                h, cost = out, cost + 1
            if h < 1:
                h, cost = out, cost + 1
            h -= 1                                  # unpack: the class mask
            if h < 1:
                h, cost = out, cost + streams
            if Dp < 1:
                Dp, cost = out, cost + members
            u = min(Dp, h) - 1
            if u < lp:
                u, cost = out, cost + members
            Y = u - lp
        if Y < 2:
            Y, cost = out, cost + members
        if Y - 1 < plan.d + 3:
            cost += 1                               # the packed final sum before the inverse
        if best_cost is None or cost < best_cost:
            best, best_cost = combo, cost
    hr, yb = [], []
    for t in range(T):
        ch = best % per
        best //= per
        hr.append(bool(ch & 1))
        yb.append(bool(ch & 2))
    return hr, yb, best_cost


def cutmax_ledger(plan, nq, log_n, boot=None, start_level=None, qbits=None, detail=False):
    """Key switches per level and bootstraps of one CutMax (library circuit).
    qbits: bit sizes of the Q primes (default 40 each), for the number of
    rescales the range-scale multiplication x = kappa V takes."""
    sim = Sim(nq, log_n, boot)
    qb = list(qbits) if qbits is not None else [40] * nq
    steps = plan.rotsum_steps
    m = plan.pad

    def rotsum(a):
        sim.ks[a] += rotsum_keys(steps, sim.log_radix)
        return a

    def mcr(a):
        return a - 1

    def mcr_bits(a, c, min_bits=30):
        # the integer multiplier c * q_a * ... (scale ~ target) keeps min_bits bits
        r, e = 1, qb[a]
        while abs(c) * 2.0 ** e < 2.0 ** min_bits and r < 3 and a - r >= 1:
            e += qb[a - r]
            r += 1
        return a - r

    def power(u, p):
        sq, acc, pp = u, None, int(p)
        while True:
            if pp & 1:
                acc = sq if acc is None else sim.mul(acc, sq)
            pp >>= 1
            if pp == 0:
                break
            sq = sim.mul(sq, sq)
        return acc

    def ensure(a, need):
        return sim.bootstrap(a) if a < need else a

    Y = nq - 1 if start_level is None else start_level
    if plan.bootstrap:                    # the circuit computes on the bootstrap's output levels
        out = Sim(nq, log_n, boot).bootstrap(0)
        Y = min(Y, out)
        h_refresh, y_boot = refresh_schedule(plan, qb, Y, out, m != 0)
    for t in range(plan.T):
        p, k = plan.p[t], plan.k[t]
        if plan.bootstrap and (Y < 5 or y_boot[t]):
            Y = sim.bootstrap(Y)
        rotsum(Y)
        D = Y
        E = sim.mul(D, D)
        V = rotsum(E)
        if m:
            sim.mul(Y, Y)
        if plan.bootstrap:
            x = mcr_bits(V, plan.kappa[t])
            if x < 2:                         # scalars take the constant bootstrap
                x = sim.bootstrap_const(x)
            Dp = mcr(mcr(D)) if m else mcr(D)
            if k == 0:                        # learned quadratic: x^2, then constants
                h = mcr(sim.mul(x, x))
            else:
                a = mcr(x)
                z = sim.mul(mcr(x), a)        # complex pair z = g + i h/4
                for i in range(2, k + 1):
                    if z < 2:
                        z = mcr(sim.bootstrap_const(z))
                    Q = sim.rot(sim.mul(z, z))    # z^2, conjugated for g h
                    z = sim.mul(z, Q)
                if z < 1:
                    z = sim.bootstrap_const(z)
                h = sim.rot(z)                # h = 4 Im z by one conjugation
            if (h_refresh[t] and h < Dp) or h < 1:
                h = sim.bootstrap_const(h)
            Dp = ensure(Dp, 1)
            u = sim.mul(Dp, h)
            u = ensure(u, (p - 1).bit_length())
        elif k == 0:
            h = mcr(sim.mul(mcr_bits(V, plan.kappa[t]), mcr_bits(V, plan.kappa[t])))
            Dp = mcr(mcr(D)) if m else mcr(D)
            u = sim.mul(Dp, h)
        else:
            a = mcr(V)
            h = mcr(a)
            g = sim.mul(mcr(V), a) if k >= 2 else None
            for i in range(2, k + 1):
                a = sim.mul(g, h)
                if i < k:
                    g = sim.mul(g, a)
                h = sim.mul(h, a)
            Dp = mcr(mcr(D)) if m else mcr(D)
            u = sim.mul(Dp, h)
        Y = power(u, p)
    if plan.bootstrap:
        Y = ensure(Y, 2)
    S = rotsum(Y)
    if plan.bootstrap and S < plan.d + 3:  # the inverse's d + 2 levels, on the scalar
        S = sim.bootstrap_const(S)
    a = mcr(S)
    F = a
    sq = a
    for _ in range(plan.d):
        sq = sim.mul(sq, sq)
        F = sim.mul(F, sq)
    sim.mul(mcr(Y), F)
    if detail:                            # (key switches, bootstraps, constant bootstraps among them)
        return dict(sim.ks), sim.n_boot, sim.n_boot_const
    return dict(sim.ks), sim.n_boot
