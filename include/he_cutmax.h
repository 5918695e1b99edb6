/*
 * he_cutmax.h -- C ABI of the GB300 (sm_103a) homomorphic CutMax library.
 *
 * What it computes.  CutMax (arXiv 2509.08383, Alg. 1) is a comparison-free
 * argmax: T iterations of mean and variance, an inverse square root, an
 * elementwise power, then a final normalisation.  Alg. 2 ("CutMax_HE") runs
 * it over CKKS ciphertexts with rotate-and-sum reductions (App. D) and
 * Goldschmidt inverse / inverse-square-root polynomials (App. B.1).  Alg. 3
 * (Sect. 3.3, "Nucleus One-Shot Sampling") adds Beta(alpha,1) cut noise to the
 * logits and calls CutMax once.  The HE interface itself (Enc, Dec, add,
 * mult, rotate) is the one assumed in Sect. 2.1 ("HE Preliminaries").
 *
 * Conventions for every call.
 *  - Every function returns int: HE_OK (0) or one of the HE_E* codes below.
 *    On error, he_last_error(ctx) gives a one-line message; outputs are not
 *    written and no object is leaked.
 *  - he_ctx and he_ct are opaque, library-owned.  The caller owns every he_ct*
 *    it receives and frees it with he_ct_free.  Input ciphertexts are never
 *    modified.
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *    global memory of the current device.  All GPU work is issued on the
 *    context's stream (he_ctx_set_stream); calls that return host data
 *    synchronise that stream before returning.
 *  - Ring degree N = 2^log_n, slots = N/2.  Ring elements are RNS vectors of
 *    64-bit words, limb-major: limb i holds the residues modulo prime i.
 *    Exported ciphertexts are in COEFFICIENT form, natural order, layout
 *    [2][level+1][N] (c0 then c1), residues in [0, q_i).
 *  - Integer plaintexts are passed as float64 arrays of N integer values.
 */
#ifndef HE_CUTMAX_H
#define HE_CUTMAX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    HE_OK = 0,
    HE_EINVAL = 1,   /* bad argument, shape or parameter */
    HE_ENOMEM = 2,   /* device arena or host allocation exhausted */
    HE_ELEVEL = 3,   /* not enough levels left and bootstrapping disabled */
    HE_ERANGE = 4,   /* plan constants out of the approximations' range */
    HE_ECUDA = 5,    /* a CUDA call failed */
    HE_ETIMEOUT = 6, /* a bounded device wait gave up */
    HE_ENOKEY = 7    /* a needed evaluation key has not been generated */
};

typedef struct he_ctx he_ctx;
typedef struct he_ct he_ct;

/* Scheme parameters.  Primes: q_bits[i] (i < n_q) for the ciphertext chain
 * q_0..q_{n_q-1}, p_bits[k] for the key-switching primes.  Primes of b bits
 * are the NTT-friendly q = k*2N+1 < 2^b in decreasing order, one cursor per
 * bit size, assigned in request order (Q first, then P).  dnum = number of
 * key-switching digits at the top level; alpha = ceil(n_q/dnum) primes per
 * digit.  secret_hw = 0 selects a dense ternary secret, h > 0 a ternary
 * secret of Hamming weight h.  sigma is the rounded-Gaussian error width.
 * log_scale is log2 of the default encoding / target scale Delta. */
typedef struct {
    uint32_t log_n, n_q, n_p, dnum;
    const int32_t *q_bits;
    const int32_t *p_bits;
    double log_scale;
    double sigma;
    uint32_t secret_hw;
    uint64_t seed;
    int32_t enable_bootstrap;
} he_params;

/* Create a context on the current CUDA device.  dev_arena/arena_bytes: a
 * caller-owned device buffer the library sub-allocates for keys, tables and
 * ciphertexts (must outlive the context); pass NULL/0 to let the library
 * cudaMalloc its own arena of arena_bytes (0 -> a size derived from the
 * parameters).  Generates the secret (from seed) and all static tables. */
int he_ctx_create(const he_params *params, void *dev_arena, size_t arena_bytes, he_ctx **out);
void he_ctx_destroy(he_ctx *ctx);
/* stream: a cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream). */
int he_ctx_set_stream(he_ctx *ctx, void *stream);
/* host out[n_q + n_p]: the prime chain. */
int he_ctx_primes(const he_ctx *ctx, uint64_t *out);
/* bytes of the arena in use / high-water mark. */
int he_ctx_memory(const he_ctx *ctx, size_t *in_use, size_t *peak);
const char *he_last_error(const he_ctx *ctx);
/* Number of CUDA kernels this library has launched since it was loaded
 * (all contexts); used to count launches inside a timed region. */
uint64_t he_launch_count(void);
/* Time one kernel class with CUDA events around each of its launches (on
 * the launch stream): 0 forward NTT, 1 inverse NTT, 2 key-switch inner
 * product, 3 basis conversion; -1 turns timing off.  Enabling resets the
 * counters.  he_profile_read synchronises the recorded events and returns
 * the launch count, the summed device time (ms) and the summed algorithmic
 * bytes of those launches (NTT: 16 bytes per coefficient per limb; inner
 * product: (3*beta + 2) words per coefficient per row; conversion: one
 * word per input and output coefficient). */
int he_profile_enable(int32_t kernel_class);
/* Operation ledger of a context since creation (or the last reset): host
 * ks_by_level[n_q] = key switches performed at each level, *n_boot = number of
 * bootstraps.  reset != 0 zeroes the ledger after reading. */
int he_ledger_read(he_ctx *ctx, uint64_t *ks_by_level, uint64_t *n_boot, int32_t reset);
/* The rest of the ledger, read without resetting (he_ledger_read resets all of
 * it): host by_level[n_q] = operations of one kind performed at each level,
 * counting every member of a batch: kind 0 rescales, 1 ciphertext (tensor)
 * products, 2 plaintext products (a bootstrap's transform diagonals
 * included), 3 additions and subtractions of ciphertexts.  HE_EINVAL for
 * another kind. */
int he_ledger_ops(const he_ctx *ctx, uint32_t kind, uint64_t *by_level);
int he_profile_read(int32_t kernel_class, uint64_t *launches, double *ms, double *bytes);

/* ---- keys (Sect. 2.1 rotations; hybrid key switching) ---------------- */
int he_keygen_relin(he_ctx *ctx);
/* Galois key for X -> X^g (g odd, < 2N); rotation by r uses g = 5^r mod 2N,
 * conjugation g = 2N-1. */
int he_keygen_galois(he_ctx *ctx, uint64_t g);
int he_keygen_rotations(he_ctx *ctx, const int32_t *steps, size_t n_steps);
/* host out[N]: the secret's coefficients in {-1,0,1}. */
int he_export_secret(const he_ctx *ctx, int8_t *out);
/* host out[(n_q+n_p)*N]: digit `digit` of key g (g = 0: relinearisation),
 * which = 0 -> b part, 1 -> a part, coefficient form. */
int he_export_key(he_ctx *ctx, uint64_t g, uint32_t digit, int32_t which, uint64_t *out);

/* ---- encode / encrypt / decrypt (Sect. 2.1) ---------------------------- */
/* Canonical-embedding encoding on the GPU (float64 FFT): host re/im[n_slots]
 * (im may be NULL; missing slots are zero) -> host out[N] integer values
 * round(scale * coefficient). */
int he_encode(he_ctx *ctx, const double *re, const double *im, size_t n_slots, double scale, double *out);
/* Secret-key encryption c1 = a, c0 = -a*s + e + m at `level` (-1 = top).
 * ctr: 32-bit counter naming this encryption's randomness. */
int he_encrypt(he_ctx *ctx, const double *re, const double *im, size_t n_slots, double scale,
               uint32_t ctr, int32_t level, he_ct **out);
/* Same with an integer plaintext polynomial host m[N]. */
int he_encrypt_poly(he_ctx *ctx, const double *m, double scale, uint32_t ctr, int32_t level, he_ct **out);
/* Decrypt and decode: host re/im[n_slots] (im may be NULL). */
int he_decrypt(he_ctx *ctx, const he_ct *ct, double *re, double *im, size_t n_slots);
/* Decrypt to the centred integer plaintext (modulo q0*q1, or q0 at level 0):
 * host out[N]. */
int he_decrypt_poly(he_ctx *ctx, const he_ct *ct, double *out);

/* ---- ciphertext objects ------------------------------------------------ */
/* host out[cap >= 2*(level+1)*N], coefficient form. */
int he_ct_export(he_ctx *ctx, const he_ct *ct, uint64_t *out, size_t cap);
int he_ct_import(he_ctx *ctx, const uint64_t *in, uint32_t level, double scale, he_ct **out);
int he_ct_info(const he_ct *ct, uint32_t *level, double *scale);
/* device pointer of c0 limb 0 (NTT form) and the element stride between
 * c0 and c1, for zero-copy inspection. */
int he_ct_device(const he_ct *ct, uint64_t **dev, size_t *poly_stride);
void he_ct_free(he_ct *ct);
/* ---- batches (engineering: the paper evaluates one ciphertext at a time) -
 * A batch holds several ciphertexts of one level and scale back to back; every
 * operation on a batch acts on all members with one kernel launch per step.
 * he_batch_pack copies n ciphertexts (batches allowed: their members are
 * concatenated) at the lowest of their levels into a new batch; members must
 * share the scale (HE_EINVAL otherwise).  he_batch_member copies member i
 * into a new single ciphertext.  he_batch_size reports the member count. */
int he_batch_pack(he_ctx *ctx, const he_ct *const *cts, size_t n, he_ct **out);
int he_batch_member(he_ctx *ctx, const he_ct *batch, uint32_t i, he_ct **out);
int he_batch_size(const he_ct *ct, uint32_t *n);

/* ---- homomorphic operations ------------------------------------------ */
int he_add(he_ctx *ctx, const he_ct *a, const he_ct *b, he_ct **out);
int he_sub(he_ctx *ctx, const he_ct *a, const he_ct *b, he_ct **out);
/* multiply by an integer (scale unchanged) */
int he_mul_int(he_ctx *ctx, const he_ct *a, int64_t k, he_ct **out);
/* multiply by a real constant c towards scale `target` and rescale:
 * E = target*q_l/scale, K = rint(c*E), scale -> (scale*E)/q_l. */
int he_mul_const(he_ctx *ctx, const he_ct *a, double c, double target, he_ct **out);
/* add a real constant to every slot: + rint(c*scale) */
int he_add_const(he_ctx *ctx, const he_ct *a, double c, he_ct **out);
/* tensor product and relinearisation, no rescale */
int he_mul(he_ctx *ctx, const he_ct *a, const he_ct *b, he_ct **out);
int he_rescale(he_ctx *ctx, const he_ct *a, he_ct **out);
/* Product, relinearisation and rescale with ONE rounding: for the tensor
 * product (d0, d1, d2) at level l and the key products acc of d2 over the
 * key-switching basis, out_k = round((P d_k + acc_k) / (q_l P)) at level l-1,
 * scale(a) scale(b) / q_l: the message of he_rescale(he_mul(a, b)), without the
 * separate rescale's transforms (the ciphertexts differ by that rounding).
 * HE_ELEVEL at level 0; with more than 15 special primes it falls back to
 * he_mul then he_rescale. */
int he_mul_rescale(he_ctx *ctx, const he_ct *a, const he_ct *b, he_ct **out);
int he_drop(he_ctx *ctx, const he_ct *a, uint32_t level, he_ct **out);
/* left slot rotation by r (g = 5^r mod 2N); conjugation; general X -> X^g */
int he_rotate(he_ctx *ctx, const he_ct *a, int32_t r, he_ct **out);
int he_conjugate(he_ctx *ctx, const he_ct *a, he_ct **out);
int he_automorphism(he_ctx *ctx, const he_ct *a, uint64_t g, he_ct **out);
/* multiplication by the monomial X^e (e taken mod 2N; X^N = -1), exact and
 * without a key: X^(N/2) is i in every slot, so e = N/2 multiplies the
 * message by i and e = 3N/2 by -i */
int he_mul_monomial(he_ctx *ctx, const he_ct *a, uint64_t e, he_ct **out);
/* rotate-and-sum over 2^steps consecutive slots (App. D): every slot i gets
 * the sum of slots i .. i + 2^steps - 1 (cyclically).  Computed in hoisted
 * stages of radix R = 2^L (he_ctx_set_rotsum_radix, default L = 3): stage s
 * covers the doublings [s L, min((s+1) L, steps)) and adds to x its
 * rotations by r 2^(s L), 0 < r < 2^len (he_rotsum_stage), which needs the
 * rotation keys of those amounts (he_cutmax_prepare generates them).  With
 * L = 1 its stages are the textbook doublings x += rot(x, 2^i), each hoisted. */
int he_rotsum(he_ctx *ctx, const he_ct *a, uint32_t steps, he_ct **out);
/* One hoisted stage: out = a + sum_r rot(a, rots[r]) for n_rots (1..15)
 * rotation amounts, with ONE ModUp of a's c1 shared by every rotation (the
 * digits read through each automorphism), the key inner products of all of
 * them and P (c0 + sum_r sigma_r(c0)) summed in the key-switching basis,
 * and ONE ModDown (hoisting: Halevi-Shoup).  It encrypts the same message as
 * the rotations and additions one by one, with key-switching noise of the
 * same size; the ciphertexts differ (the automorphism meets the approximate
 * basis conversion after it instead of before it, and one ModDown rounds
 * the summed products).  HE_ENOKEY when a rotation key is missing. */
int he_rotsum_stage(he_ctx *ctx, const he_ct *a, const int32_t *rots, size_t n_rots, he_ct **out);
/* log2 of the rotate-and-sum radix (1..4: radix 2, 4, 8, 16) used by
 * he_rotsum, cutmax, nucleus_sample and the constant bootstrap's trace; set
 * it before he_cutmax_prepare / he_bootstrap_prepare, which generate the
 * rotation keys its stages need.  HE_EINVAL outside 1..4. */
int he_ctx_set_rotsum_radix(he_ctx *ctx, uint32_t log2_radix);
/* Hybrid key switch of a raw polynomial: host d[(level+1)*N] coefficient
 * form -> host out0/out1[(level+1)*N] coefficient form, with key g. */
int he_keyswitch_raw(he_ctx *ctx, const uint64_t *d, uint32_t level, uint64_t g, uint64_t *out0, uint64_t *out1);
/* ModDown of hybrid key switching alone: the rounded division
 * out = round(acc / P) mod q_0..q_level of two polynomials given over the
 * key-switching basis, P the product of the special primes.  Host
 * acc0/acc1[(level+1+n_p)*N] in coefficient form (rows q_0..q_level, then
 * p_0..p_(n_p-1), residues in [0, prime)) -> host out0/out1[(level+1)*N] in
 * coefficient form.  Exact for every input, including x within one unit of
 * +-P/2 (the float64 estimate of the rounding is replaced by an exact
 * mixed-radix comparison where it cannot decide). */
int he_moddown_raw(he_ctx *ctx, const uint64_t *acc0, const uint64_t *acc1, uint32_t level, uint64_t *out0,
                   uint64_t *out1);
/* Key switch that allocates nothing, for callers that cannot allocate device
 * memory on demand: cudaMalloc/cudaFree synchronise the device and can fail
 * under fragmentation, so latency-critical serving code, or a process whose
 * device memory is entirely reserved by another allocator, cannot get
 * scratch space per call.  The paper has no counterpart.
 * Computes the same hybrid key switch as he_keyswitch_raw, on DEVICE data:
 * d[(level+1)*N] in NTT form -> out[2][level+1][N] in NTT form (key g, g = 0:
 * relinearisation).  Scratch comes from one file-scope device array of 2^22
 * 64-bit words (32 MiB) that every GPU loading the library holds until exit;
 * a key switch needing more (words = (level+1)N + beta*n_ext*N + 2 n_ext N +
 * 2 (level+1) N, n_ext = level+1+n_p) is rejected with HE_EINVAL.  The first
 * call on a device looks the array's address up (cudaGetSymbolAddress with
 * that device current), so make that first call before any stream capture.
 * All calls share the array and nothing in it needs clearing (every word is
 * written before it is read); calls whose GPU work overlaps race on it.
 * During the call the context's own key-switch scratch is pointed at the
 * array (and restored before return), so no other host thread may use the
 * same context meanwhile (contexts are not thread-safe in any case). */
int he_keyswitch_noalloc(he_ctx *ctx, const uint64_t *d, uint32_t level, uint64_t g, uint64_t *out);
/* Negacyclic NTT (inverse != 0: INTT) in place on DEVICE data[n_limbs][N];
 * limb t uses prime prime_idx0 + t.  NTT form: position i holds
 * a(psi^(2 brv(i) + 1)), psi the canonical 2N-th root of that prime. */
int he_ntt_device(he_ctx *ctx, uint64_t *data, uint32_t n_limbs, uint32_t prime_idx0, int32_t inverse);

/* ---- bootstrapping (App. B.1: ciphertexts are refreshed when their
 * multiplicative depth runs out) ------------------------------------------- */
/* Build the bootstrapping tables and keys.  K bounds |I| in the ModRaise
 * plaintext t = m + q0*I (about 6 standard deviations of the secret's
 * contribution, sqrt(h/12) for Hamming weight h); the modular reduction is
 * cos(2 pi((K+1)x - 1/4)/2^r) by a Chebyshev series of degree d (d < 64),
 * followed by r double angles.  Needs n_q >= 18: the transforms take 3 + 3
 * levels and EvalMod ceil(log2 d) + 1 + r levels, all from the top of the
 * chain; a bootstrapped ciphertext comes out at level n_q - 1 - that many.
 * Level-consuming steps use the chain from the top down, so the top
 * primes should be the large (about 60-bit) ones. */
int he_bootstrap_prepare(he_ctx *ctx, uint32_t K, uint32_t r, uint32_t d);
/* Refresh a ciphertext (any level, any scale; only limb q0 is used) to a high
 * level, encrypting the same message at the input's scale, up to the
 * bootstrapping error. */
int he_bootstrap(he_ctx *ctx, const he_ct *in, he_ct **out);
/* The ciphertext after one stage of he_bootstrap, for inspection: 0 ModRaise
 * (scale declared q0 (K+1)), 1..3 after each CoeffToSlot level, 4 / 5 the
 * real / imaginary part, 6 / 7 those after EvalMod, 8 recombined, 9 / 10 after
 * the first two SlotToCoeff levels, 11 the result. */
int he_bootstrap_stage(he_ctx *ctx, const he_ct *in, int32_t stage, he_ct **out);
/* Refresh a ciphertext whose slots all hold one complex value a + i b (the
 * plaintext polynomial a + b X^(N/2), e.g. a scalar of the CutMax circuit),
 * at about half the cost of he_bootstrap: after ModRaise, the trace over the
 * automorphisms X -> X^(5^k) (a log2(N/2)-step rotate-and-sum with the
 * rotation keys of 1, 2, ..., N/4, which he_cutmax_prepare of a bootstrapped
 * plan generates) keeps the coefficients of 1 and X^(N/2) only; both go
 * through one EvalMod, packed into the two halves of the slots, followed by
 * one Taylor step of arcsin (a constant's value sits whole in coefficient 0,
 * where the sine's curvature would otherwise show: relative error ~4e-7 v^4
 * for a value v at q0 / Delta = 2^7).  Output at he_bootstrap's output level
 * and at the input's scale.  Slots that do not hold one common value come
 * out as their average (the trace is a projection): the result is then not
 * the input's message, and no error is raised.  HE_EINVAL without
 * he_bootstrap_prepare; HE_EKEY (or the missing-key error) without the keys. */
int he_bootstrap_const(he_ctx *ctx, const he_ct *in, he_ct **out);

/* ---- CutMax (Alg. 2) and nucleus sampling (Alg. 3) ------------------- */
/* Circuit plan: the range-scaling constants of Sect. 3.2's obligations.
 * n real entries (the vocabulary) per stream, spread over cts ciphertexts
 * (0 is read as 1): ciphertext c of a stream holds entries c*N/2 .. in its
 * slots, the last one zero-padded.  packing 0 = replicate (one ciphertext, n
 * a power of two dividing N/2, slot j = x[j mod n]), 1 = zero-pad.
 * Per iteration t < T: power[t] (p), c[t], k[t] Goldschmidt inverse-sqrt
 * iterations, kappa[t] range scale of V_t = sum (n y - S)^2, y0[t] initial
 * guess.  Final normalisation: Goldschmidt inverse of degree d on
 * kappa_f * sum(Y).  bootstrap != 0 selects the bootstrapped circuit (needs
 * he_bootstrap_prepare): the Goldschmidt input is x = kappa V, Y_(t+1) is
 * scaled by norm[t] (NULL = all 1) and a ciphertext is bootstrapped before
 * any phase that needs more levels than it has (Y before the statistics: 5,
 * since V = sum (n y - S)^2 is scaled to x = kappa V by up to 3 rescales that
 * keep a 30-bit multiplier, and V itself is too large to refresh;
 * x: 2; the Goldschmidt pair z = g + i h, one complex constant refreshed
 * by he_bootstrap_const, between steps: 2; D' and h: 1; u before the
 * power: ceil(log2 p); Y before the final normalisation: d + 3).
 * shared != 0 (bootstrapped plans, batches of S > 1 streams): the per-stream
 * scalar chains (the Goldschmidt inverse square root and the final inverse,
 * whose inputs are replicated in every slot) run once for the batch, packed
 * into one ciphertext (slot i carries stream i mod S', S' = S rounded up to a
 * power of two, S' <= N/4), and are handed back to the streams by a slot mask
 * and a log2(S')-step rotate-and-sum; engineering beyond the paper, which
 * evaluates one stream at a time.
 * learned: NULL, or [T][3] coefficients {A, B, C} of learned quadratics
 * (he_learn_invsqrt); at an iteration with k[t] = 0 the inverse square root is
 * h = (A x^2 + B x + C) / 2 of x = kappa V (two levels after x) instead of the
 * Goldschmidt iteration.  k[t] = 0 without `learned` is HE_ERANGE.
 * relax: NULL, or the additive constant of every Goldschmidt step, k[0] +
 * ... + k[T-1] doubles in iteration order (none for k[t] = 0): step i of
 * iteration t multiplies the running estimate by a = relax[...] - g h instead
 * of Newton's 3/2 - g h (App. B's inverse square root with the per-step
 * over-relaxation of the implementation it cites; a relaxed step costs the
 * levels of a plain one).  NULL is 3/2 for every step; a constant outside
 * [1, 4] is HE_ERANGE. */
typedef struct {
    uint32_t n, packing, T;
    const uint32_t *power;
    const double *c;
    const uint32_t *k;
    const double *kappa;
    const double *y0;
    uint32_t d;
    double kappa_f;
    const double *norm;
    int32_t bootstrap;
    uint32_t cts;
    uint32_t shared;
    const double *learned;
    const double *relax;
} he_cutmax_plan;

/* Learned inverse-square-root stand-in (engineering on top of Sect. 3.2,
 * whose inverse square root is the generic approximation of App. B): trains
 * a 1 -> 16 -> 1 network with square activations in FP32 on the GPU
 * (full-batch Adam, `steps` steps from rate lr decayed by a half cosine,
 * initial weights from seed) to
 * minimise mean (f(x) sqrt(x) - 1)^2 over the n host values x (> 0, the
 * range-scaled variances kappa V of the circuit), and returns its quadratic
 * form abc = {A, B, C}: f(x) = A x^2 + B x + C; loss (may be NULL) is the final
 * mean squared relative error.  HE_ERANGE for a non-positive x. */
int he_learn_invsqrt(he_ctx *ctx, const float *x, size_t n, uint32_t steps, float lr, uint64_t seed,
                     double *abc, double *loss);

/* Generate every key the plan needs (rotations 2^i, relinearisation and,
 * with bootstrapping, its rotations and conjugation). */
int he_cutmax_prepare(he_ctx *ctx, const he_cutmax_plan *plan);
/* CutMax_HE (Alg. 2): out = encrypted near-one-hot of argmax(in).  `in` may
 * be a batch (he_batch_pack) of S streams of plan->cts ciphertexts each,
 * stream-major; every step then runs once for the whole batch, and the
 * output is the batch of the streams' results in the same order. */
int cutmax(he_ctx *ctx, const he_ct *in, const he_cutmax_plan *plan, he_ct **out);
/* cutmax through a CUDA graph (engineering; the paper evaluates Alg. 2 op by
 * op).  Same arguments, result and errors as cutmax, bit for bit.  The first
 * call with a given plan and input shape (level, scale, batch size, the
 * context's rotate-and-sum radix) runs directly and then captures the whole
 * call -- every iteration, refresh and the final normalisation -- as one CUDA
 * graph; every buffer of the graph comes from a block of the context's arena
 * that the graph keeps until he_cutmax_graph_clear or he_ctx_destroy (about
 * 1.25x the device memory one call takes).  Later calls with the same key copy
 * `in` into the graph's input buffer, launch the graph on the context's stream
 * and copy its output into *out (owned by the caller).  Ledger counts and the
 * launch count advance as for a direct call.  Where a call cannot be captured
 * (or while a kernel class is being profiled) it runs directly.  Calls on one
 * context must not overlap (the graph's buffers are shared); graphs that hold
 * bootstrap tables or rotation choices that have since changed are retired,
 * and a context keeps at most 16 graphs (the least recently used one goes). */
int he_cutmax_graph(he_ctx *ctx, const he_ct *in, const he_cutmax_plan *plan, he_ct **out);
/* Calls of he_cutmax_graph so far: graphs captured, graph launches, direct
 * runs after a capture that failed or under profiling (any pointer may be NULL). */
int he_cutmax_graph_stats(he_ctx *ctx, uint64_t *captured, uint64_t *replayed, uint64_t *direct);
/* Frees every captured graph and its arena block (waits for the context's stream). */
int he_cutmax_graph_clear(he_ctx *ctx);
/* on != 0: cutmax and nucleus_sample run their CutMax as he_cutmax_graph does
 * (same results, bit for bit); 0 (the default): directly. */
int he_ctx_set_graphs(he_ctx *ctx, int32_t on);
/* Cut noise drawn by the server from encrypted uniforms (Alg. 3 with
 * Lemma 2 / Observation 1): out = G = U^(1/alpha) slot by slot, U in [0, 1]
 * encrypted by the client, by the degree-`degree` Chebyshev interpolant of
 * ((t+1)/2)^(1/alpha) on t = 2U - 1 (1 + about log2(degree) + 1 levels).
 * Accurate to ~1e-2 for U >= 1e-3 at degree 31 (alpha ~ 22); the interpolant
 * cannot follow the cusp of U^(1/alpha) at U = 0.  The series runs at U's own
 * scale and G comes out at the context's scale Delta: uniforms encrypted on
 * large primes (e.g. at scale 2^60 on the 60-bit bootstrapping primes, 7
 * levels above the bootstrap output level) keep their scale through the
 * products, and G lands on the circuit's levels with all of them left.
 * HE_EINVAL for alpha <= 0 or degree outside 2..127.  Works on batches. */
int he_beta_noise(he_ctx *ctx, const he_ct *u, double alpha, uint32_t degree, he_ct **out);

/* Kinds of the randomness handed to nucleus_sample. */
#define HE_RAND_BETA 0    /* rand_ct encrypts the cut noise G = U^(1/alpha) itself (client-side draw) */
#define HE_RAND_UNIFORM 1 /* rand_ct encrypts uniforms U in [0, 1]; the library evaluates G = U^(1/alpha) */
/* Chebyshev degree of the library's U^(1/alpha) for HE_RAND_UNIFORM (7 levels) */
#define HE_NUCLEUS_DEGREE 31

/* Nucleus one-shot sampling (Alg. 3, Sect. 3.3): out = CutMax(logits + G),
 * an encrypted near-one-hot vector at the sampled token, where G_i are
 * Beta(alpha, 1) cut variables with alpha = ln(1-q)/ln(top_p), so that
 * P(G_i > top_p) = q (Lemma 2 for q = top_p, Observation 1 for any q); q = 0
 * reads as q = top_p.  rand_kind HE_RAND_BETA: rand_ct already encrypts G
 * (drawn by the client for this top_p and q; 0 levels).  HE_RAND_UNIFORM:
 * rand_ct encrypts uniforms U and the library evaluates G = U^(1/alpha) by
 * he_beta_noise of degree HE_NUCLEUS_DEGREE (7 levels, taken from rand_ct's
 * level before the addition; G at the context's scale Delta, see
 * he_beta_noise).  logits and rand_ct follow the layout of the plan (one
 * ciphertext or a batch, as for cutmax); logits and G must share one scale.
 * HE_EINVAL for top_p outside (0, 1), q outside [0, 1), an unknown kind or
 * operands of different scales. */
int nucleus_sample(he_ctx *ctx, const he_ct *logits, double top_p, double q, const he_ct *rand_ct,
                   int32_t rand_kind, const he_cutmax_plan *plan, he_ct **out);
/* Nucleus sampling for a batch whose streams use different top-p masses (Alg. 3
 * per stream, one CutMax for all): logits and rand_ct are batches split into
 * n_groups equal runs of members, group j taking top_p[j] (alpha_j =
 * ln(1-q)/ln(top_p[j]); q = 0 reads as q = top_p[j]).  Each group's cut noise is
 * drawn as nucleus_sample draws it, the noisy logits of every group are joined
 * into one batch, and CutMax runs once over it (shared scalar chains then serve
 * every stream of the batch).  The output is the batch of all streams' results
 * in order.  With one group this is nucleus_sample.  HE_EINVAL as for
 * nucleus_sample, for n_groups < 1, a batch not divisible into n_groups whole
 * groups of streams, or a null top_p. */
int nucleus_sample_groups(he_ctx *ctx, const he_ct *logits, const double *top_p, uint32_t n_groups, double q,
                          const he_ct *rand_ct, int32_t rand_kind, const he_cutmax_plan *plan, he_ct **out);

#ifdef __cplusplus
}
#endif
#endif /* HE_CUTMAX_H */
