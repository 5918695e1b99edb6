"""ctypes wrapper of the C oracle (ckks_oracle.c): RNS-CKKS by definition.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
import ctypes as C
import numpy as np

from .build import build_oracle

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build_oracle())
        u64, i64, u32, dbl, vp, ip = C.c_uint64, C.c_int64, C.c_uint32, C.c_double, C.c_void_p, C.c_int
        P = np.ctypeslib.ndpointer
        pu64 = P(np.uint64, flags="C")
        pdbl = P(np.float64, flags="C")
        sig = {
            "or_powmod": (u64, [u64, u64, u64]),
            "or_set_threads": (ip, [ip]),
            "or_get_threads": (ip, []),
            "or_invmod": (u64, [u64, u64]),
            "or_is_prime": (ip, [u64]),
            "or_gen_primes": (ip, [ip, P(np.int32, flags="C"), ip, pu64]),
            "or_find_psi": (u64, [u64, ip]),
            "or_ntt_def": (None, [pu64, pu64, ip, u64, u64]),
            "or_ntt": (None, [pu64, ip, u64]),
            "or_intt": (None, [pu64, ip, u64]),
            "or_negacyclic_schoolbook": (None, [pu64, pu64, pu64, ip, u64]),
            "or_philox": (None, [P(np.uint32, flags="C"), P(np.uint32, flags="C"), P(np.uint32, flags="C")]),
            "or_gauss_cdt": (None, [dbl, pu64]),
            "or_sample_gauss": (None, [u64, u32, u32, dbl, ip, P(np.int64, flags="C")]),
            "or_sample_secret": (None, [u64, ip, ip, P(np.int8, flags="C")]),
            "or_ctx_create": (vp, [ip, ip, ip, P(np.int32, flags="C"), P(np.int32, flags="C"), ip, ip, dbl, u64]),
            "or_ctx_free": (None, [vp]),
            "or_ctx_info": (None, [vp, pu64, P(np.int32, flags="C")]),
            "or_ctx_secret": (None, [vp, P(np.int8, flags="C")]),
            "or_ctx_psi": (u64, [vp, ip]),
            "or_gen_relin_key": (None, [vp]),
            "or_gen_galois_key": (None, [vp, u64]),
            "or_key_export": (ip, [vp, u64, ip, ip, pu64]),
            "or_ct_new": (vp, [vp, ip, dbl]),
            "or_ct_free": (None, [vp]),
            "or_ct_level": (ip, [vp]),
            "or_ct_scale": (dbl, [vp]),
            "or_ct_set_scale": (None, [vp, dbl]),
            "or_ct_export": (None, [vp, vp, pu64]),
            "or_ct_import": (vp, [vp, pu64, ip, dbl]),
            "or_encrypt": (vp, [vp, pdbl, dbl, u32, ip]),
            "or_decrypt": (None, [vp, vp, pdbl]),
            "or_drop": (vp, [vp, vp, ip]),
            "or_add": (vp, [vp, vp, vp, ip]),
            "or_mul_int": (vp, [vp, vp, i64]),
            "or_mul_intd": (vp, [vp, vp, dbl, dbl]),
            "or_add_intd": (vp, [vp, vp, dbl]),
            "or_add_plain": (vp, [vp, vp, pdbl]),
            "or_mul_plain": (vp, [vp, vp, pdbl, dbl]),
            "or_keyswitch": (ip, [vp, pu64, ip, u64, pu64, pu64]),
            "or_moddown": (None, [vp, pu64, pu64, ip, pu64, pu64]),
            "or_mul": (vp, [vp, vp, vp]),
            "or_mul_rescale": (vp, [vp, vp, vp]),
            "or_rescale": (vp, [vp, vp]),
            "or_automorphism": (vp, [vp, vp, u64]),
            "or_rotsum_stage": (vp, [vp, vp, P(np.int64, flags="C"), ip]),
            "or_rot_galois": (u64, [ip, i64]),
            "or_mod_raise": (vp, [vp, vp, ip]),
            "or_mul_monomial": (vp, [vp, vp, u64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


# ----------------------------------------------------------------- helpers
def set_threads(n):
    """Threads for the per-limb loops (0 = all cores of this process's affinity)."""
    return lib().or_set_threads(int(n))


def get_threads():
    return lib().or_get_threads()


def gen_primes(log_n, bits):
    b = np.asarray(bits, dtype=np.int32)
    out = np.zeros(len(b), dtype=np.uint64)
    rc = lib().or_gen_primes(log_n, b, len(b), out)
    if rc != 0:
        raise ValueError(f"prime generation failed ({rc})")
    return out


def ntt(a, log_n, q):
    x = np.ascontiguousarray(a, dtype=np.uint64).copy()
    lib().or_ntt(x, log_n, int(q))
    return x


def intt(a, log_n, q):
    x = np.ascontiguousarray(a, dtype=np.uint64).copy()
    lib().or_intt(x, log_n, int(q))
    return x


def ntt_def(a, log_n, q, psi):
    x = np.ascontiguousarray(a, dtype=np.uint64)
    out = np.zeros_like(x)
    lib().or_ntt_def(x, out, log_n, int(q), int(psi))
    return out


def schoolbook(a, b, log_n, q):
    out = np.zeros(1 << log_n, dtype=np.uint64)
    lib().or_negacyclic_schoolbook(np.ascontiguousarray(a, dtype=np.uint64),
                                   np.ascontiguousarray(b, dtype=np.uint64), out, log_n, int(q))
    return out


def philox(ctr, key):
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox(np.asarray(ctr, dtype=np.uint32), np.asarray(key, dtype=np.uint32), out)
    return out


def gauss_cdt(sigma):
    """The sampler's 19 thresholds: floor(2^64 P(|e| <= k)), k = 0..18."""
    out = np.zeros(19, dtype=np.uint64)
    lib().or_gauss_cdt(float(sigma), out)
    return out


def sample_secret(seed, log_n, h):
    out = np.zeros(1 << log_n, dtype=np.int8)
    lib().or_sample_secret(seed, log_n, h, out)
    return out


def sample_gauss(seed, obj, domain, sigma, log_n):
    out = np.zeros(1 << log_n, dtype=np.int64)
    lib().or_sample_gauss(seed, obj, domain, sigma, log_n, out)
    return out


def rot_galois(log_n, r):
    return int(lib().or_rot_galois(log_n, int(r)))


# ----------------------------------------------------------------- objects
class Ciphertext:
    __slots__ = ("ctx", "ptr")

    def __init__(self, ctx, ptr):
        if not ptr:
            raise RuntimeError("oracle operation failed (missing key?)")
        self.ctx = ctx
        self.ptr = ptr

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.or_ct_free(self.ptr)
            self.ptr = None

    @property
    def level(self):
        return lib().or_ct_level(self.ptr)

    @property
    def scale(self):
        return lib().or_ct_scale(self.ptr)

    def set_scale(self, s):
        lib().or_ct_set_scale(self.ptr, float(s))

    def export(self):
        """(2, level+1, N) uint64, coefficient form."""
        L = self.level
        out = np.zeros(2 * (L + 1) * self.ctx.n, dtype=np.uint64)
        lib().or_ct_export(self.ctx.ptr, self.ptr, out)
        return out.reshape(2, L + 1, self.ctx.n)


class Context:
    """RNS-CKKS context: primes, secret, keys (all derived from `seed`)."""

    def __init__(self, log_n, qbits, pbits, dnum, h=0, sigma=3.2, seed=0):
        self.log_n = log_n
        self.n = 1 << log_n
        self.slots = self.n // 2
        self.nq = len(qbits)
        self.np_ = len(pbits)
        self.dnum = dnum
        self.h = h
        self.seed = seed
        qb = np.asarray(qbits, dtype=np.int32)
        pb = np.asarray(pbits, dtype=np.int32)
        self.ptr = lib().or_ctx_create(log_n, len(qb), len(pb), qb, pb, dnum, h, sigma, seed)
        if not self.ptr:
            raise ValueError("oracle context creation failed")
        primes = np.zeros(self.nq + self.np_, dtype=np.uint64)
        ab = np.zeros(2, dtype=np.int32)
        lib().or_ctx_info(self.ptr, primes, ab)
        self.primes = [int(p) for p in primes]
        self.alpha, self.beta = int(ab[0]), int(ab[1])
        self.top_level = self.nq - 1

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.or_ctx_free(self.ptr)
            self.ptr = None

    def secret(self):
        out = np.zeros(self.n, dtype=np.int8)
        lib().or_ctx_secret(self.ptr, out)
        return out

    def psi(self, i):
        return int(lib().or_ctx_psi(self.ptr, i))

    # keys
    def gen_relin_key(self):
        lib().or_gen_relin_key(self.ptr)

    def gen_galois_key(self, g):
        lib().or_gen_galois_key(self.ptr, int(g))

    def gen_rot_key(self, r):
        self.gen_galois_key(rot_galois(self.log_n, r))

    def conj_galois(self):
        return 2 * self.n - 1

    def key_export(self, g, digit, which):
        out = np.zeros((self.nq + self.np_) * self.n, dtype=np.uint64)
        if lib().or_key_export(self.ptr, int(g), digit, which, out) != 0:
            raise KeyError(g)
        return out.reshape(self.nq + self.np_, self.n)

    # encryption
    def encrypt(self, pt, scale, ctr, level=None):
        pt = np.ascontiguousarray(pt, dtype=np.float64)
        assert pt.shape == (self.n,)
        lvl = self.top_level if level is None else level
        return Ciphertext(self, lib().or_encrypt(self.ptr, pt, float(scale), int(ctr), lvl))

    def decrypt(self, ct):
        out = np.zeros(self.n, dtype=np.float64)
        lib().or_decrypt(self.ptr, ct.ptr, out)
        return out

    def import_ct(self, arr, level, scale):
        a = np.ascontiguousarray(arr, dtype=np.uint64).reshape(-1)
        return Ciphertext(self, lib().or_ct_import(self.ptr, a, level, float(scale)))

    # operations (each returns a new ciphertext)
    def add(self, a, b):
        return Ciphertext(self, lib().or_add(self.ptr, a.ptr, b.ptr, 0))

    def sub(self, a, b):
        return Ciphertext(self, lib().or_add(self.ptr, a.ptr, b.ptr, 1))

    def drop(self, a, level):
        return Ciphertext(self, lib().or_drop(self.ptr, a.ptr, level))

    def mul_int(self, a, k):
        return Ciphertext(self, lib().or_mul_int(self.ptr, a.ptr, int(k)))

    def mul_intd(self, a, K, scale_out):
        return Ciphertext(self, lib().or_mul_intd(self.ptr, a.ptr, float(K), float(scale_out)))

    def add_intd(self, a, K):
        return Ciphertext(self, lib().or_add_intd(self.ptr, a.ptr, float(K)))

    def add_plain(self, a, pt):
        return Ciphertext(self, lib().or_add_plain(self.ptr, a.ptr, np.ascontiguousarray(pt, dtype=np.float64)))

    def mul_plain(self, a, pt, scale_out):
        return Ciphertext(self, lib().or_mul_plain(self.ptr, a.ptr, np.ascontiguousarray(pt, dtype=np.float64),
                                                   float(scale_out)))

    def mul(self, a, b):
        return Ciphertext(self, lib().or_mul(self.ptr, a.ptr, b.ptr))

    def rescale(self, a):
        return Ciphertext(self, lib().or_rescale(self.ptr, a.ptr))

    def mul_rescale(self, a, b):
        """Product, relinearisation and rescale with one rounded division by q_l P."""
        return Ciphertext(self, lib().or_mul_rescale(self.ptr, a.ptr, b.ptr))

    def automorphism(self, a, g):
        return Ciphertext(self, lib().or_automorphism(self.ptr, a.ptr, int(g)))

    def rotsum_stage(self, a, rots):
        """a + sum_r rot(a, r) as one hoisted stage (one ModUp of c1, the key
        products of every rotation summed, one ModDown)."""
        arr = np.ascontiguousarray(rots, dtype=np.int64)
        return Ciphertext(self, lib().or_rotsum_stage(self.ptr, a.ptr, arr, len(arr)))

    def rotate(self, a, r):
        return self.automorphism(a, rot_galois(self.log_n, r))

    def conj(self, a):
        return self.automorphism(a, self.conj_galois())

    def mod_raise(self, a, level=None):
        lvl = self.top_level if level is None else level
        return Ciphertext(self, lib().or_mod_raise(self.ptr, a.ptr, lvl))

    def mul_monomial(self, a, e):
        return Ciphertext(self, lib().or_mul_monomial(self.ptr, a.ptr, int(e)))

    def moddown(self, acc0, acc1, level):
        """round(acc / P) mod q_0..q_level of two polynomials given over
        q_0..q_level, p_0..p_(K-1) ([(level+1+K)][N] residues each)."""
        a0 = np.ascontiguousarray(acc0, dtype=np.uint64).reshape(-1)
        a1 = np.ascontiguousarray(acc1, dtype=np.uint64).reshape(-1)
        assert a0.size == a1.size == (level + 1 + self.np_) * self.n
        o0 = np.zeros((level + 1) * self.n, dtype=np.uint64)
        o1 = np.zeros_like(o0)
        lib().or_moddown(self.ptr, a0, a1, level, o0, o1)
        return o0.reshape(level + 1, self.n), o1.reshape(level + 1, self.n)

    def keyswitch(self, d, level, g):
        d = np.ascontiguousarray(d, dtype=np.uint64).reshape(-1)
        o0 = np.zeros_like(d)
        o1 = np.zeros_like(d)
        if lib().or_keyswitch(self.ptr, d, level, int(g), o0, o1) != 0:
            raise KeyError(g)
        return o0.reshape(level + 1, self.n), o1.reshape(level + 1, self.n)
