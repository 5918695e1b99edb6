"""Thin ctypes binding of libhecutmax.so (the C ABI in include/he_cutmax.h).

Argument marshalling only: every step of every operation runs in the CUDA
library.  Device memory for the library's arena comes from PyTorch's caching
allocator, and the library issues its kernels on PyTorch's current stream.
If the compiled library is missing, loading raises; there is no fallback.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhecutmax.so")

HE_OK, HE_EINVAL, HE_ENOMEM, HE_ELEVEL, HE_ERANGE, HE_ECUDA, HE_ETIMEOUT, HE_ENOKEY = range(8)
HE_RAND_BETA, HE_RAND_UNIFORM = 0, 1
HE_NUCLEUS_DEGREE = 31
_NAMES = {0: "HE_OK", 1: "HE_EINVAL", 2: "HE_ENOMEM", 3: "HE_ELEVEL", 4: "HE_ERANGE", 5: "HE_ECUDA",
          6: "HE_ETIMEOUT", 7: "HE_ENOKEY"}


class HeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("log_n", C.c_uint32), ("n_q", C.c_uint32), ("n_p", C.c_uint32), ("dnum", C.c_uint32),
                ("q_bits", C.POINTER(C.c_int32)), ("p_bits", C.POINTER(C.c_int32)), ("log_scale", C.c_double),
                ("sigma", C.c_double), ("secret_hw", C.c_uint32), ("seed", C.c_uint64),
                ("enable_bootstrap", C.c_int32)]


class CPlan(C.Structure):
    _fields_ = [("n", C.c_uint32), ("packing", C.c_uint32), ("T", C.c_uint32), ("power", C.POINTER(C.c_uint32)),
                ("c", C.POINTER(C.c_double)), ("k", C.POINTER(C.c_uint32)), ("kappa", C.POINTER(C.c_double)),
                ("y0", C.POINTER(C.c_double)), ("d", C.c_uint32), ("kappa_f", C.c_double),
                ("norm", C.POINTER(C.c_double)), ("bootstrap", C.c_int32), ("cts", C.c_uint32),
                ("shared", C.c_uint32), ("learned", C.POINTER(C.c_double)), ("relax", C.POINTER(C.c_double))]


_lib = None
VP = C.c_void_p
PP = C.POINTER(C.c_void_p)


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run paper_2509_08383_gb300.build)")
        L = C.CDLL(LIB_PATH)
        u64, u32, i32, i64, dbl, sz = C.c_uint64, C.c_uint32, C.c_int32, C.c_int64, C.c_double, C.c_size_t
        pd, pu64 = C.POINTER(C.c_double), C.POINTER(C.c_uint64)
        sig = {
            "he_ctx_create": [C.POINTER(Params), VP, sz, PP],
            "he_ctx_destroy": [VP],
            "he_ctx_set_stream": [VP, VP],
            "he_ctx_primes": [VP, pu64],
            "he_ctx_memory": [VP, C.POINTER(sz), C.POINTER(sz)],
            "he_last_error": [VP],
            "he_launch_count": [],
            "he_profile_enable": [i32],
            "he_ledger_read": [VP, pu64, pu64, i32],
            "he_ledger_ops": [VP, u32, pu64],
            "he_profile_read": [i32, C.POINTER(u64), pd, pd],
            "he_keygen_relin": [VP],
            "he_keygen_galois": [VP, u64],
            "he_keygen_rotations": [VP, C.POINTER(i32), sz],
            "he_export_secret": [VP, C.POINTER(C.c_int8)],
            "he_export_key": [VP, u64, u32, i32, pu64],
            "he_encode": [VP, pd, pd, sz, dbl, pd],
            "he_encrypt": [VP, pd, pd, sz, dbl, u32, i32, PP],
            "he_encrypt_poly": [VP, pd, dbl, u32, i32, PP],
            "he_decrypt": [VP, VP, pd, pd, sz],
            "he_decrypt_poly": [VP, VP, pd],
            "he_ct_export": [VP, VP, pu64, sz],
            "he_ct_import": [VP, pu64, u32, dbl, PP],
            "he_ct_info": [VP, C.POINTER(u32), pd],
            "he_ct_device": [VP, C.POINTER(pu64), C.POINTER(sz)],
            "he_ct_free": [VP],
            "he_batch_pack": [VP, PP, sz, PP],
            "he_batch_member": [VP, VP, u32, PP],
            "he_batch_size": [VP, C.POINTER(u32)],
            "he_add": [VP, VP, VP, PP],
            "he_sub": [VP, VP, VP, PP],
            "he_mul_int": [VP, VP, i64, PP],
            "he_mul_const": [VP, VP, dbl, dbl, PP],
            "he_add_const": [VP, VP, dbl, PP],
            "he_mul": [VP, VP, VP, PP],
            "he_mul_rescale": [VP, VP, VP, PP],
            "he_rescale": [VP, VP, PP],
            "he_drop": [VP, VP, u32, PP],
            "he_rotate": [VP, VP, i32, PP],
            "he_conjugate": [VP, VP, PP],
            "he_automorphism": [VP, VP, u64, PP],
            "he_mul_monomial": [VP, VP, u64, PP],
            "he_rotsum": [VP, VP, u32, PP],
            "he_rotsum_stage": [VP, VP, C.POINTER(i32), sz, PP],
            "he_ctx_set_rotsum_radix": [VP, u32],
            "he_keyswitch_raw": [VP, pu64, u32, u64, pu64, pu64],
            "he_moddown_raw": [VP, pu64, pu64, u32, pu64, pu64],
            "he_ntt_device": [VP, VP, u32, u32, i32],
            "he_keyswitch_noalloc": [VP, VP, u32, u64, VP],
            "he_bootstrap_prepare": [VP, u32, u32, u32],
            "he_bootstrap": [VP, VP, PP],
            "he_bootstrap_stage": [VP, VP, i32, PP],
            "he_bootstrap_const": [VP, VP, PP],
            "he_cutmax_prepare": [VP, C.POINTER(CPlan)],
            "he_learn_invsqrt": [VP, C.POINTER(C.c_float), sz, u32, C.c_float, u64, pd, pd],
            "cutmax": [VP, VP, C.POINTER(CPlan), PP],
            "he_cutmax_graph": [VP, VP, C.POINTER(CPlan), PP],
            "he_cutmax_graph_stats": [VP, pu64, pu64, pu64],
            "he_cutmax_graph_clear": [VP],
            "he_ctx_set_graphs": [VP, i32],
            "nucleus_sample": [VP, VP, dbl, dbl, VP, i32, C.POINTER(CPlan), PP],
            "nucleus_sample_groups": [VP, VP, pd, u32, dbl, VP, i32, C.POINTER(CPlan), PP],
            "he_beta_noise": [VP, VP, dbl, u32, PP],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = None if name in ("he_ctx_destroy", "he_ct_free") else C.c_int
        L.he_last_error.restype = C.c_char_p
        L.he_launch_count.restype = C.c_uint64
        _lib = L
    return _lib


def launch_count():
    return int(lib().he_launch_count())


PROF_NTT_FWD, PROF_NTT_INV, PROF_KS_INNER, PROF_BCONV = 0, 1, 2, 3


def profile_enable(kernel_class):
    if lib().he_profile_enable(int(kernel_class)) != 0:
        raise ValueError(kernel_class)


def profile_read(kernel_class):
    n, ms, b = C.c_uint64(), C.c_double(), C.c_double()
    lib().he_profile_read(int(kernel_class), C.byref(n), C.byref(ms), C.byref(b))
    return int(n.value), float(ms.value), float(b.value)


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _u64ptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint64))


class Ciphertext:
    __slots__ = ("ctx", "ptr")

    def __init__(self, ctx, ptr):
        self.ctx = ctx
        self.ptr = ptr

    def __del__(self):
        if self.ptr and _lib is not None:
            _lib.he_ct_free(self.ptr)
            self.ptr = None

    def _info(self):
        lv, sc = C.c_uint32(), C.c_double()
        lib().he_ct_info(self.ptr, C.byref(lv), C.byref(sc))
        return lv.value, sc.value

    @property
    def level(self):
        return self._info()[0]

    @property
    def scale(self):
        return self._info()[1]

    @property
    def batch(self):
        n = C.c_uint32()
        lib().he_batch_size(self.ptr, C.byref(n))
        return n.value

    def export(self):
        """(2, level+1, N) uint64, coefficient form."""
        L = self.level
        out = np.zeros(2 * (L + 1) * self.ctx.n, dtype=np.uint64)
        self.ctx._chk(lib().he_ct_export(self.ctx.ptr, self.ptr, _u64ptr(out), out.size))
        return out.reshape(2, L + 1, self.ctx.n)


def plan_struct(plan):
    """Package CutMaxPlan -> (ctypes struct, keep-alive arrays)."""
    T = plan.T
    norm = list(plan.norm) if getattr(plan, "norm", None) is not None else [1.0] * T
    arrs = dict(power=(C.c_uint32 * T)(*plan.p), c=(C.c_double * T)(*plan.c), k=(C.c_uint32 * T)(*plan.k),
                kappa=(C.c_double * T)(*plan.kappa), y0=(C.c_double * T)(*plan.y0), norm=(C.c_double * T)(*norm))
    lq = getattr(plan, "lq", None)
    arrs["learned"] = (C.c_double * (3 * T))(*[float(v) for row in lq for v in row]) if lq else None
    rel = getattr(plan, "relax", None)
    if rel is not None:
        flat = []
        for t in range(T):
            row = list(rel[t]) if rel[t] else []
            if row and len(row) != int(plan.k[t]):
                raise ValueError(f"iteration {t}: {len(row)} relaxation constants for {plan.k[t]} Goldschmidt steps")
            flat += row if row else [1.5] * int(plan.k[t])
        arrs["relax"] = (C.c_double * max(1, len(flat)))(*flat)
    else:
        arrs["relax"] = None
    s = CPlan(n=plan.n, packing=0 if plan.packing == "replicate" else 1, T=T, power=arrs["power"], c=arrs["c"],
              k=arrs["k"], kappa=arrs["kappa"], y0=arrs["y0"], d=plan.d, kappa_f=plan.kappa_f,
              norm=arrs["norm"], bootstrap=int(bool(getattr(plan, "bootstrap", False))),
              cts=int(getattr(plan, "cts", 1)), shared=int(bool(getattr(plan, "shared", False))),
              learned=arrs["learned"], relax=arrs["relax"])
    return s, arrs


class Context:
    """A CKKS context on the current CUDA device (see he_ctx_create)."""

    def __init__(self, log_n, qbits, pbits, dnum, log_scale=40.0, sigma=3.2, h=0, seed=0, bootstrap=False,
                 arena_bytes=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.log_n, self.n, self.slots = log_n, 1 << log_n, 1 << (log_n - 1)
        self.nq, self.np_ = len(qbits), len(pbits)
        self.delta = 2.0 ** log_scale
        qb = (C.c_int32 * len(qbits))(*qbits)
        pb = (C.c_int32 * len(pbits))(*pbits)
        prm = Params(log_n=log_n, n_q=len(qbits), n_p=len(pbits), dnum=dnum, q_bits=qb, p_bits=pb,
                     log_scale=log_scale, sigma=sigma, secret_hw=h, seed=seed, enable_bootstrap=int(bootstrap))
        if arena_bytes is None:
            alpha = -(-len(qbits) // dnum)
            beta = -(-len(qbits) // alpha)
            key = beta * 2 * (len(qbits) + len(pbits)) * self.n * 8
            ct = 2 * len(qbits) * self.n * 8
            arena_bytes = 128 * key + 512 * ct + (64 << 20)
        self._arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device="cuda")
        self.ptr = C.c_void_p()
        rc = lib().he_ctx_create(C.byref(prm), C.c_void_p(self._arena.data_ptr()), int(arena_bytes),
                                 C.byref(self.ptr))
        if rc != 0:
            raise HeError(rc, "context creation failed")
        self._chk(lib().he_ctx_set_stream(self.ptr, C.c_void_p(torch.cuda.current_stream().cuda_stream)))
        pr = np.zeros(self.nq + self.np_, dtype=np.uint64)
        lib().he_ctx_primes(self.ptr, _u64ptr(pr))
        self.primes = [int(p) for p in pr]
        self.top_level = self.nq - 1

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.he_ctx_destroy(self.ptr)
            self.ptr = None

    def _chk(self, rc):
        if rc != 0:
            raise HeError(rc, lib().he_last_error(self.ptr).decode())

    def _ct(self, fn, *args):
        out = C.c_void_p()
        self._chk(fn(self.ptr, *args, C.byref(out)))
        return Ciphertext(self, out)

    def ledger(self, reset=False):
        """(key switches per level [n_q], bootstraps) since creation / last reset."""
        ks = np.zeros(self.nq, dtype=np.uint64)
        nb = np.zeros(1, dtype=np.uint64)
        self._chk(lib().he_ledger_read(self.ptr, _u64ptr(ks), _u64ptr(nb), int(bool(reset))))
        return ks.astype(np.int64), int(nb[0])

    LEDGER_KINDS = ("rescale", "tensor", "plain_mul", "add")

    def ledger_ops(self):
        """{kind: operations per level [n_q]} since the last ledger reset, for
        kind in rescale, tensor, plain_mul, add (read before ledger(reset=True))."""
        out = {}
        for i, name in enumerate(self.LEDGER_KINDS):
            v = np.zeros(self.nq, dtype=np.uint64)
            self._chk(lib().he_ledger_ops(self.ptr, i, _u64ptr(v)))
            out[name] = v.astype(np.int64)
        return out

    def memory(self):
        a, b = C.c_size_t(), C.c_size_t()
        lib().he_ctx_memory(self.ptr, C.byref(a), C.byref(b))
        return a.value, b.value

    # keys
    def secret(self):
        out = np.zeros(self.n, dtype=np.int8)
        self._chk(lib().he_export_secret(self.ptr, out.ctypes.data_as(C.POINTER(C.c_int8))))
        return out

    def gen_relin_key(self):
        self._chk(lib().he_keygen_relin(self.ptr))

    def gen_galois_key(self, g):
        self._chk(lib().he_keygen_galois(self.ptr, int(g)))

    def gen_rot_keys(self, steps):
        arr = (C.c_int32 * len(steps))(*steps)
        self._chk(lib().he_keygen_rotations(self.ptr, arr, len(steps)))

    def key_export(self, g, digit, which):
        out = np.zeros((self.nq + self.np_) * self.n, dtype=np.uint64)
        self._chk(lib().he_export_key(self.ptr, int(g), digit, which, _u64ptr(out)))
        return out.reshape(self.nq + self.np_, self.n)

    # encoding / encryption
    def encode(self, z, scale):
        z = np.asarray(z)
        re = np.ascontiguousarray(z.real, dtype=np.float64)
        im = np.ascontiguousarray(z.imag, dtype=np.float64) if np.iscomplexobj(z) else None
        out = np.zeros(self.n)
        self._chk(lib().he_encode(self.ptr, _dptr(re), _dptr(im) if im is not None else None, len(re), float(scale),
                                  _dptr(out)))
        return out

    def encrypt(self, z, scale, ctr, level=-1):
        z = np.asarray(z)
        re = np.ascontiguousarray(z.real, dtype=np.float64)
        im = np.ascontiguousarray(z.imag, dtype=np.float64) if np.iscomplexobj(z) else None
        return self._ct(lib().he_encrypt, _dptr(re), _dptr(im) if im is not None else None, len(re), float(scale),
                        int(ctr), int(level))

    def encrypt_poly(self, m, scale, ctr, level=-1):
        m = np.ascontiguousarray(m, dtype=np.float64)
        return self._ct(lib().he_encrypt_poly, _dptr(m), float(scale), int(ctr), int(level))

    def decrypt(self, ct, n_slots=None, complex_out=False):
        n_slots = self.slots if n_slots is None else n_slots
        re = np.zeros(n_slots)
        im = np.zeros(n_slots) if complex_out else None
        self._chk(lib().he_decrypt(self.ptr, ct.ptr, _dptr(re), _dptr(im) if im is not None else None, n_slots))
        return re + 1j * im if complex_out else re

    def decrypt_poly(self, ct):
        out = np.zeros(self.n)
        self._chk(lib().he_decrypt_poly(self.ptr, ct.ptr, _dptr(out)))
        return out

    # batches
    def batch_pack(self, cts):
        """One batch holding the members of `cts` (ciphertexts or batches), in order."""
        arr = (C.c_void_p * len(cts))(*[c.ptr for c in cts])
        return self._ct(lib().he_batch_pack, arr, len(cts))

    def batch_member(self, batch, i):
        return self._ct(lib().he_batch_member, batch.ptr, int(i))

    def import_ct(self, arr, level, scale):
        a = np.ascontiguousarray(arr, dtype=np.uint64).reshape(-1)
        return self._ct(lib().he_ct_import, _u64ptr(a), int(level), float(scale))

    # operations
    def add(self, a, b):
        return self._ct(lib().he_add, a.ptr, b.ptr)

    def sub(self, a, b):
        return self._ct(lib().he_sub, a.ptr, b.ptr)

    def mul_int(self, a, k):
        return self._ct(lib().he_mul_int, a.ptr, int(k))

    def mul_const(self, a, c, target):
        return self._ct(lib().he_mul_const, a.ptr, float(c), float(target))

    def add_const(self, a, c):
        return self._ct(lib().he_add_const, a.ptr, float(c))

    def mul(self, a, b):
        return self._ct(lib().he_mul, a.ptr, b.ptr)

    def rescale(self, a):
        return self._ct(lib().he_rescale, a.ptr)

    def mul_rescale(self, a, b):
        """Product, relinearisation and rescale with one rounding (by q_l P)."""
        return self._ct(lib().he_mul_rescale, a.ptr, b.ptr)

    def drop(self, a, level):
        return self._ct(lib().he_drop, a.ptr, int(level))

    def rotate(self, a, r):
        return self._ct(lib().he_rotate, a.ptr, int(r))

    def conj(self, a):
        return self._ct(lib().he_conjugate, a.ptr)

    def automorphism(self, a, g):
        return self._ct(lib().he_automorphism, a.ptr, int(g))

    def mul_monomial(self, a, e):
        return self._ct(lib().he_mul_monomial, a.ptr, int(e))

    def rotsum(self, a, steps):
        return self._ct(lib().he_rotsum, a.ptr, int(steps))

    def rotsum_stage(self, a, rots):
        """a + sum_r rot(a, r): one hoisted stage (one ModUp, one ModDown)."""
        arr = (C.c_int32 * len(rots))(*[int(r) for r in rots])
        return self._ct(lib().he_rotsum_stage, a.ptr, arr, len(rots))

    def set_rotsum_radix(self, log2_radix):
        """Radix 2^log2_radix of the rotate-and-sum stages (default 8); set before
        generating keys with cutmax_prepare / bootstrap_prepare."""
        self._chk(lib().he_ctx_set_rotsum_radix(self.ptr, int(log2_radix)))

    def keyswitch(self, d, level, g):
        d = np.ascontiguousarray(d, dtype=np.uint64).reshape(-1)
        o0, o1 = np.zeros_like(d), np.zeros_like(d)
        self._chk(lib().he_keyswitch_raw(self.ptr, _u64ptr(d), int(level), int(g), _u64ptr(o0), _u64ptr(o1)))
        return o0.reshape(level + 1, self.n), o1.reshape(level + 1, self.n)

    def moddown(self, acc0, acc1, level):
        """round(acc / P) mod q_0..q_level of two polynomials given in coefficient
        form over q_0..q_level, p_0..p_(K-1) ([(level+1+K)][N] each)."""
        a0 = np.ascontiguousarray(acc0, dtype=np.uint64).reshape(-1)
        a1 = np.ascontiguousarray(acc1, dtype=np.uint64).reshape(-1)
        assert a0.size == a1.size == (level + 1 + self.np_) * self.n
        o0 = np.zeros((level + 1) * self.n, dtype=np.uint64)
        o1 = np.zeros_like(o0)
        self._chk(lib().he_moddown_raw(self.ptr, _u64ptr(a0), _u64ptr(a1), int(level), _u64ptr(o0), _u64ptr(o1)))
        return o0.reshape(level + 1, self.n), o1.reshape(level + 1, self.n)

    def keyswitch_noalloc(self, d_tensor, level, g, out_tensor):
        """Key switch on device tensors with the library's static scratch (no allocation):
        d (level+1, N) NTT form -> out (2, level+1, N) NTT form."""
        assert d_tensor.is_cuda and out_tensor.is_cuda
        self._chk(lib().he_keyswitch_noalloc(self.ptr, C.c_void_p(d_tensor.data_ptr()), int(level), int(g),
                                             C.c_void_p(out_tensor.data_ptr())))

    def ntt_device(self, tensor, prime_idx0, inverse=False):
        """In-place (I)NTT of a CUDA uint64/int64 tensor of shape (limbs, N)."""
        assert tensor.is_cuda and tensor.is_contiguous() and tensor.shape[-1] == self.n
        limbs = tensor.numel() // self.n
        self._chk(lib().he_ntt_device(self.ptr, C.c_void_p(tensor.data_ptr()), limbs, int(prime_idx0),
                                      int(bool(inverse))))

    # bootstrapping
    def bootstrap_prepare(self, K, r, d):
        self._chk(lib().he_bootstrap_prepare(self.ptr, int(K), int(r), int(d)))

    def bootstrap(self, ct):
        return self._ct(lib().he_bootstrap, ct.ptr)

    def bootstrap_stage(self, ct, stage):
        return self._ct(lib().he_bootstrap_stage, ct.ptr, int(stage))

    def bootstrap_const(self, ct):
        """Refresh a ciphertext holding one complex value in every slot."""
        return self._ct(lib().he_bootstrap_const, ct.ptr)

    def learn_invsqrt(self, xs, steps=3000, lr=1e-2, seed=0):
        """Train the learned inverse-square-root network on the GPU (FP32): returns
        ([A, B, C], final mean squared relative error) of f(x) = A x^2 + B x + C ~ 1/sqrt(x)."""
        x = np.ascontiguousarray(xs, dtype=np.float32)
        abc = np.zeros(3)
        loss = C.c_double()
        self._chk(lib().he_learn_invsqrt(self.ptr, x.ctypes.data_as(C.POINTER(C.c_float)), x.size, int(steps),
                                         float(lr), int(seed), _dptr(abc), C.byref(loss)))
        return [float(v) for v in abc], float(loss.value)

    # CutMax / nucleus
    def cutmax_prepare(self, plan):
        s, keep = plan_struct(plan)
        self._chk(lib().he_cutmax_prepare(self.ptr, C.byref(s)))

    def cutmax(self, ct, plan):
        s, keep = plan_struct(plan)
        return self._ct(lib().cutmax, ct.ptr, C.byref(s))

    def cutmax_graph(self, ct, plan):
        """cutmax through a CUDA graph captured per plan and input shape."""
        s, keep = plan_struct(plan)
        return self._ct(lib().he_cutmax_graph, ct.ptr, C.byref(s))

    def graph_stats(self):
        """(graphs captured, graph launches, direct runs) of cutmax_graph."""
        v = [C.c_uint64(0) for _ in range(3)]
        self._chk(lib().he_cutmax_graph_stats(self.ptr, *[C.byref(x) for x in v]))
        return tuple(int(x.value) for x in v)

    def graph_clear(self):
        self._chk(lib().he_cutmax_graph_clear(self.ptr))

    def set_graphs(self, on):
        """cutmax and nucleus_sample through CUDA graphs (on) or directly."""
        self._chk(lib().he_ctx_set_graphs(self.ptr, int(bool(on))))

    def beta_noise(self, u_ct, alpha, degree=31):
        """G = U^(1/alpha) of encrypted uniforms (Chebyshev interpolant)."""
        return self._ct(lib().he_beta_noise, u_ct.ptr, float(alpha), int(degree))

    def nucleus_sample(self, ct, rand_ct, plan, top_p, q=0.0, kind="beta"):
        """Alg. 3: CutMax(ct + G), P(G_i > top_p) = q (q = 0: q = top_p).  kind
        "beta": rand_ct encrypts G itself; "uniform": rand_ct encrypts uniforms U
        and the library evaluates G = U^(1/alpha)."""
        s, keep = plan_struct(plan)
        k = {"beta": HE_RAND_BETA, "uniform": HE_RAND_UNIFORM}[kind]
        return self._ct(lib().nucleus_sample, ct.ptr, float(top_p), float(q), rand_ct.ptr, k, C.byref(s))

    def nucleus_sample_groups(self, ct, rand_ct, plan, top_ps, q=0.0, kind="beta"):
        """Alg. 3 for a batch split into len(top_ps) equal groups of streams,
        group j at top-p mass top_ps[j]; one CutMax for the whole batch."""
        s, keep = plan_struct(plan)
        k = {"beta": HE_RAND_BETA, "uniform": HE_RAND_UNIFORM}[kind]
        tp = (C.c_double * len(top_ps))(*[float(x) for x in top_ps])
        return self._ct(lib().nucleus_sample_groups, ct.ptr, tp, len(top_ps), float(q), rand_ct.ptr, k, C.byref(s))
