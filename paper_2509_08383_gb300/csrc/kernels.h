// Host-callable launchers of the library's CUDA kernels (kernels.cu).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace he {

struct NttTables {
    const ulonglong2 *fwd, *inv;  // [prime][N] pairs (twiddle, Shoup companion)
};

// Residues of one constant for every prime (value and Shoup companion).
struct ScalarTab {
    u64 v[HE_MAX_PRIMES];
    u64 s[HE_MAX_PRIMES];
};

// Basis-conversion table: for input a < n_in and output row t < n_out,
// qhat[a*stride + t] and its Montgomery form qhat * 2^64 mod p_t, and
// qhinv[a] (+ Shoup), device memory.
struct BConvTab {
    const u64 *qhinv = nullptr, *qhinv_sh = nullptr;  // [n_in]
    const u64 *qhat = nullptr, *qhat_mont = nullptr;  // [n_in][stride]
    int n_in = 0, n_out = 0, stride = 0;
    // rounding mode (ModDown): floor(2^128 / q_a) as (low, high) words [n_in][2]
    // and (-Q mod p_t) 2^64 mod p_t [stride], Q the product of the input
    // primes; null: approximate conversion
    const u64 *inv_fix = nullptr;
    const u64 *negq_mont = nullptr;
    // exact rounding where the fixed-point estimate cannot decide (x within
    // ~1e-13 Q of Q/2): q_j^-1 mod q_i at [i*n_in + j] (j < i) and the
    // mixed-radix digits of (Q-1)/2 [n_in]
    const u64 *mr_inv = nullptr;
    const u64 *mr_half = nullptr;
};

// number of kernels launched by this library so far (all contexts)
unsigned long long launch_count();
void launches_add(long long n);  // launches made (or, negative, taken back) around CUDA graphs

// CUDA-event timing of one kernel class at a time (see he_profile_enable)
enum ProfClass { PROF_NTT_FWD = 0, PROF_NTT_INV = 1, PROF_KS_INNER = 2, PROF_BCONV = 3 };
void prof_enable(int cls);
bool prof_any();  // some kernel class is instrumented
void prof_begin(int cls, cudaStream_t s);
void prof_end(int cls, cudaStream_t s, double bytes);
void prof_read(int cls, unsigned long long *launches, double *ms, double *bytes);

void upload_constants(int slot, const PrimeConsts &pc, const u64 *cdt, int n_cdt, cudaStream_t s);

// NTT / INTT of n_rows limb rows in place.
void ntt_forward(const Rows &rows, int n_rows, const NttTables &tw, int log_n, cudaStream_t s);
void ntt_inverse(const Rows &rows, int n_rows, const NttTables &tw, int log_n, cudaStream_t s);
// out-of-place INTT: dst <- INTT(src) (src rows read once, by the first pass)
void ntt_inverse_from(const Rows &dst, const Rows &src, int n_rows, const NttTables &tw, int log_n, cudaStream_t s);

// out = a + b / a - b (sub != 0) / -a (b ignored when neg != 0)
void ew_add(const Rows &out, const Rows &a, const Rows &b, int n_rows, int sub, int log_n, cudaStream_t s);
void ew_neg(const Rows &out, const Rows &a, int n_rows, int log_n, cudaStream_t s);
void ew_copy(const Rows &out, const Rows &a, int n_rows, int log_n, cudaStream_t s);
// out = a * K (per prime residue of K)
void ew_mul_scalar(const Rows &out, const Rows &a, const ScalarTab &k, int n_rows, int log_n, cudaStream_t s);
// out = a + K in every position (NTT form of a constant polynomial)
void ew_add_scalar(const Rows &out, const Rows &a, const ScalarTab &k, int n_rows, int log_n, cudaStream_t s);
// out = a (*) b pointwise
// Plaintext-diagonal multiply-accumulate of one baby-step giant-step group:
// out0/out1 = sum_{b < n} c0[b]/c1[b] * pt[b], limb-major rows 0..n_rows-1
// (row r uses prime r for r < l1, special prime nq + r - l1 after), plaintexts
// in Montgomery form (x 2^64).
constexpr int DIAG_MAC_MAX = 64;
// Batch members (grid z) read c0/c1 at + member * c_stride and write out at +
// member * out_stride; the plaintexts are shared.
struct DiagMac {
    const u64 *c0[DIAG_MAC_MAX], *c1[DIAG_MAC_MAX], *pt[DIAG_MAC_MAX];
    u64 *out0, *out1;
    int n, slot, l1, nq;
    int batch = 1;
    size_t c_stride = 0, out_stride = 0;
};
// QP lift of `batch` members (member m at out + m*out_stride, src + m*src_stride)
void ew_qp_lift(u64 *out, const u64 *src, int l1, int n_rows, u64 g, int add, const ScalarTab &pm, int slot,
                int log_n, cudaStream_t s, int batch = 1, size_t out_stride = 0, size_t src_stride = 0);
// Batch-member group sum (sum != 0: out member s = sum_{c<g} in member s*g+c)
// or broadcast (out member b = in member b/g), both polynomials, limbs 0..l1-1
// (limb t on prime t); member m at + m*stride, polynomial k at + k*poly.
void ew_group(u64 *out, const u64 *in, int n_out_members, int g, int sum, int l1, size_t out_stride, size_t in_stride,
              size_t in_poly, size_t out_poly, int slot, int log_n, cudaStream_t s);
void ew_diag_mac(const DiagMac &dm, int n_rows, int log_n, cudaStream_t s);
void ew_mul(const Rows &out, const Rows &a, const Rows &b, int n_rows, int log_n, cudaStream_t s);
// out = out + a (*) b pointwise
void ew_mul_acc(const Rows &out, const Rows &a, const Rows &b, int n_rows, int log_n, cudaStream_t s);
// out = a0 - a1 (*) b  (decryption / encryption building block)
void ew_tensor(const Rows &d0, const Rows &d1, const Rows &d2, const Rows &a0, const Rows &a1,
               const Rows &b0, const Rows &b1, int n_rows, int log_n, cudaStream_t s);
// in place: x -> x 2^64 mod q (back = 0) or x 2^-64 mod q (back = 1)
void ew_mont(const Rows &rows, int n_rows, int back, int log_n, cudaStream_t s);
// out = a * X^e (e < 2N) in NTT form
void ew_monomial(const Rows &out, const Rows &a, int n_rows, u64 e, const NttTables &tw, int log_n, cudaStream_t s);
// automorphism X -> X^g in NTT form (permutation of positions)
void ew_automorph_ntt(const Rows &out, const Rows &a, int n_rows, u64 g, int log_n, cudaStream_t s);

// Key-switch pieces
// out row (poly*n_out + t) = sum_a [in_a * qhinv_a] * qhat[a][t], in row (poly*n_in + a)
void bconv(const Rows &out, const Rows &in, const BConvTab &tab, int n_polys, int log_n, cudaStream_t s);
// up to BCONV_SET_MAX conversions without rounding in one launch (out[j] <- in[j]
// by tab[j], n_polys polynomials each)
constexpr int BCONV_SET_MAX = 8;
struct BConvSet {
    Rows out[BCONV_SET_MAX], in[BCONV_SET_MAX];
    BConvTab tab[BCONV_SET_MAX];
    int n = 0;
};
void bconv_set(const BConvSet &set, int n_polys, int log_n, cudaStream_t s);
// acc0/acc1 rows t < n_rows: sum_j x_j[t] * key_j[t], x_j = (t in digit j) ? d[t] : ext_j[t],
// for `batch` members (member m's d, ext and acc at + m * the stride)
struct KeyIP {
    const u64 *d_ntt;     // level limbs of the input polynomial (NTT form)
    const u64 *ext;       // [beta][n_rows][N] extended digits (rows inside the digit unused)
    const u64 *key;       // [beta][2][nq+np][N]
    u64 *acc;             // [2][n_rows][N]
    int n_rows, l1, nq, np, alpha, beta, key_limbs;
    int slot;
    u64 galois;           // 0: read x_j at position i; else at the source of i under X -> X^galois
    int batch = 1;
    size_t d_stride = 0, ext_stride = 0, acc_stride = 0;
};
// + P * d_k on the Q rows (t < l1) of output polynomial k of one member: the
// addend rows d_k at d + k * poly_stride, P mod q_i in pmod
struct KeyLift {
    const u64 *d = nullptr;
    size_t poly_stride = 0;
    ScalarTab pmod;
};
void keyswitch_inner(const KeyIP &k, int log_n, cudaStream_t s, const KeyLift *lift = nullptr);
// Hoisted rotate-and-sum stage: the sum over n_keys rotations r of the key
// inner products of sigma_r(ext) (one shared ModUp of c1, read through
// X -> X^gal[r] in NTT form), plus P * (c0 + sum_r sigma_r(c0)) on the Q rows,
// for `batch` members; acc = [2][n_rows][N] per member.  Products are summed
// per key in 128 bits (keys in Montgomery form), reduced, then added mod q.
constexpr int ROTSUM_MAX_KEYS = 15;
struct KeyIPMulti {
    const u64 *d_ntt;     // c1, level limbs (NTT form)
    const u64 *ext;       // [beta][n_rows][N] hoisted digits (rows inside the digit unused)
    const u64 *c0;        // c0, level limbs (NTT form)
    u64 *acc;             // [2][n_rows][N]
    int n_rows, l1, nq, np, alpha, beta, key_limbs;
    int slot;
    int n_keys;
    const u64 *keys[ROTSUM_MAX_KEYS];  // [beta][2][nq+np][N] each, Montgomery form
    u64 gal[ROTSUM_MAX_KEYS];
    ScalarTab pmod;       // P mod q_i
    int batch = 1;
    size_t d_stride = 0, ext_stride = 0, acc_stride = 0, c0_stride = 0;
};
void keyswitch_inner_multi(const KeyIPMulti &k, int log_n, cudaStream_t s);
// out_i = (acc_i - conv_i) * pinv_i; polynomial p of the batch (row / lpp)
// also adds add_to's row when bit p of add_mask is set.
void moddown_finish(const Rows &out, const Rows &acc, const Rows &conv, const ScalarTab &pinv, int n_rows,
                    const Rows &add_to, int add_mask, int log_n, cudaStream_t s);
// rescale: from coefficient-form last limbs (n_polys rows at last + poly*N,
// prime ql) write the centred lift into rows of `lift` (n_polys*l targets,
// row r: polynomial r / l, prime r % l)
// (kmul: rescale K a instead of a, K mod q_i in kmul, limbs 0..l)
void rescale_lift(const Rows &lift, const u64 *last, int n_polys, u64 ql, int l, int log_n, cudaStream_t s,
                  const ScalarTab *kmul = nullptr);
void rescale_finish(const Rows &out, const Rows &in, const Rows &lift, const ScalarTab &qlinv, int n_rows,
                    int log_n, cudaStream_t s, const ScalarTab *kmul = nullptr);
// mod-raise: from coefficient-form level-0 limbs (prime q0; polynomial p's at
// src + p*N) write the centred lift into the rows of out (coefficient form)
void modraise_lift(const Rows &out, const u64 *src, u64 q0, int n_rows, int log_n, cudaStream_t s);

// Sampling (Philox4x32-10, counter = (index, limb, object, domain))
void sample_uniform(const Rows &out, int n_rows, u64 seed, u32 object, u32 domain, int log_n, cudaStream_t s);
// e_k for every row: rounded Gaussian by CDT, optional plaintext add (integer
// valued doubles, may be null)
void sample_error_plus(const Rows &out, int n_rows, u64 seed, u32 object, u32 domain, const double *pt,
                       int log_n, cudaStream_t s);
// small signed integers (secret) -> rows
void load_small(const Rows &out, int n_rows, const int8_t *v, int log_n, cudaStream_t s);
// integer-valued doubles -> rows
void load_intd(const Rows &out, int n_rows, const double *v, int log_n, cudaStream_t s);

// Encoding (float64 canonical embedding)
struct Cplx { double re, im; };
void encode_slots(double *out_coeff, const double *re, const double *im, int n_slots, double scale,
                  const int *slot_l, Cplx *work, int log_n, cudaStream_t s);
void decode_coeffs(double *re, double *im, const double *coeff, double scale, const int *slot_l, Cplx *work,
                   int log_n, cudaStream_t s);
// centred CRT of rows 0 (and 1 when two) in coefficient form -> doubles
void crt_to_double(double *out, const u64 *r0, const u64 *r1, u64 q0, u64 q1, u64 q0inv_mod_q1, int two,
                   int log_n, cudaStream_t s);
// pointwise out[k] = a[k]*b[k] + c[k] for decryption (rows 0..n_rows-1)
void decrypt_rows(const Rows &out, const Rows &c0, const Rows &c1, const Rows &sk, int n_rows, int log_n,
                  cudaStream_t s);

}  // namespace he
