// Device-side arithmetic and addressing shared by the kernels of the library.
//
// Residues are 64-bit words modulo primes q < 2^62 (so 4q fits a word, which
// the lazy NTT butterflies rely on).  Three reductions are used:
//   Shoup    w*x mod q for a constant w with precomputed w' = floor(w 2^64/q):
//            hi = floor(x w' / 2^64), r = x w - hi q in [0, 2q) for any x < 2^64.
//   Barrett  x mod q for x < 2^(2b+1), b = bit length of q, with
//            mu = floor(2^(2b+1) / q): qhat = ((x >> (b-1)) * mu) >> (b+2),
//            r = x - qhat q in [0, 3q), then at most two subtractions.
//   plain    a +- b mod q with one conditional correction.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

typedef uint64_t u64;
typedef uint32_t u32;
typedef int64_t i64;

#define HE_MAX_PRIMES 64
#define HE_MAX_CTX 8     // contexts alive at once (one constant-memory slot each)

struct ModQ {
    u64 q;
    u64 mu;      // floor(2^(2b+1)/q)
    u32 b;       // bit length of q
    u32 pad;
};

// Per-context constants, one constant-memory slot per live context (filled
// by he::upload_constants); kernels find their slot in Rows::slot.
struct PrimeConsts {
    ModQ m[HE_MAX_PRIMES];
    u64 n_inv[HE_MAX_PRIMES];
    u64 n_inv_shoup[HE_MAX_PRIMES];
    u64 r64[HE_MAX_PRIMES];  // 2^64 mod q
    u64 mont_qinv[HE_MAX_PRIMES];  // -q^-1 mod 2^64 (Montgomery reduction)
    u64 cdt[24];             // rounded-Gaussian CDT thresholds
    int ncdt;
    int pad;
};

namespace he {
// context slot used by make_rows(); set by the host entry points
extern thread_local int t_slot;
}

__device__ __forceinline__ u64 shoup_mul_lazy(u64 x, u64 w, u64 w_shoup, u64 q) {
    u64 hi = __umul64hi(x, w_shoup);
    return x * w - hi * q;  // in [0, 2q)
}
__device__ __forceinline__ u64 shoup_mul(u64 x, u64 w, u64 w_shoup, u64 q) {
    u64 r = shoup_mul_lazy(x, w, w_shoup, q);
    return r >= q ? r - q : r;
}

__device__ __forceinline__ u64 barrett_reduce(u64 lo, u64 hi, const ModQ &m) {
    u64 x1 = (lo >> (m.b - 1)) | (hi << (65 - m.b));
    u64 plo = x1 * m.mu, phi = __umul64hi(x1, m.mu);
    u64 qhat = (plo >> (m.b + 2)) | (phi << (62 - m.b));
    u64 r = lo - qhat * m.q;
    if (r >= m.q) r -= m.q;
    if (r >= m.q) r -= m.q;
    return r;
}
// (hi 2^64 + lo) 2^-64 mod q, fully reduced, for any hi < 2^63 - q (the
// Montgomery quotient step leaves a value < hi + q, which Barrett reduces)
__device__ __forceinline__ u64 mont_reduce_wide(u64 lo, u64 hi, const ModQ &m, u64 qinv_neg) {
    u64 mm = lo * qinv_neg;
    u64 t = hi + __umul64hi(mm, m.q) + (lo != 0 ? 1ull : 0ull);
    return barrett_reduce(t, 0, m);
}
__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, const ModQ &m) {
    return barrett_reduce(a * b, __umul64hi(a, b), m);
}
// a*b + c*d mod q (each operand < q): the 128-bit sum is < 2q^2 < 2^(2b+1)
__device__ __forceinline__ u64 mul_add_mod(u64 a, u64 b, u64 c, u64 d, const ModQ &m) {
    u64 lo1 = a * b, hi1 = __umul64hi(a, b);
    u64 lo2 = c * d, hi2 = __umul64hi(c, d);
    u64 lo = lo1 + lo2;
    u64 hi = hi1 + hi2 + (lo < lo1 ? 1ull : 0ull);
    return barrett_reduce(lo, hi, m);
}
// Montgomery reduction of T = hi*2^64 + lo < q 2^64: T / 2^64 mod q in [0, q)
__device__ __forceinline__ u64 mont_reduce(u64 lo, u64 hi, u64 q, u64 qinv_neg) {
    u64 m = lo * qinv_neg;
    u64 t = hi + __umul64hi(m, q) + (lo != 0 ? 1ull : 0ull);
    return t >= q ? t - q : t;
}

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) {
    u64 s = a + b;
    return s >= q ? s - q : s;
}
__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) {
    return a >= b ? a - b : a + q - b;
}

// A batch of limb rows.  Row r belongs to polynomial r / lpp, limb t = r % lpp.
// Default addressing: the limb sits at base + poly*poly_stride + t*N and uses
// prime prime0 + t when t < l1, else prime nq + (t - l1) (the special primes
// of the key-switching basis).  Descriptor addressing (desc != nullptr): limb
// t of every polynomial sits at base + poly*poly_stride + desc[t].x*N and uses
// prime desc[t].y.  pmod > 0 takes the polynomial index modulo pmod, so that
// one operand (a plaintext, say) serves every member of a batch.
struct Rows {
    u64 *base;
    size_t poly_stride;  // elements between consecutive polynomials
    int lpp;             // limbs per polynomial
    int l1;              // leading limbs on the Q chain
    int nq;              // index of the first special prime
    int prime0;          // offset added to Q-chain limb indices
    int slot;            // constant-memory slot of the owning context
    int pmod;            // > 0: polynomial index modulo pmod
    const int2 *desc;
    __host__ __device__ __forceinline__ u64 *row(int r, int log_n) const {
        int poly = r / lpp, t = r - poly * lpp;
        if (pmod) poly %= pmod;
        const size_t off = desc ? (size_t)desc[t].x : (size_t)t;
        return base + (size_t)poly * poly_stride + (off << log_n);
    }
    __host__ __device__ __forceinline__ int prime(int r) const {
        int t = r % lpp;
        if (desc) return desc[t].y;
        return t < l1 ? prime0 + t : nq + (t - l1);
    }
};

static inline Rows make_rows(u64 *base, size_t poly_stride, int lpp, int l1, int nq, int prime0 = 0) {
    Rows r;
    r.base = base; r.poly_stride = poly_stride; r.lpp = lpp; r.l1 = l1; r.nq = nq; r.prime0 = prime0;
    r.slot = he::t_slot;
    r.pmod = 0;
    r.desc = nullptr;
    return r;
}
// n_desc descriptor rows per polynomial, polynomials poly_stride apart
static inline Rows desc_rows(u64 *base, const int2 *desc, int n_desc, size_t poly_stride = 0) {
    Rows r = make_rows(base, poly_stride, n_desc, n_desc, 0, 0);
    r.desc = desc;
    return r;
}
static inline Rows shared_rows(Rows r, int pmod) {
    r.pmod = pmod;
    return r;
}
