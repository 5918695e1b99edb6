/*
 * Plain CPU reference of RNS-CKKS for the homomorphic CutMax path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code with the CUDA library: every
 * routine here is written from its textbook definition, deliberately slow.
 *
 * Conventions (all of them restated independently on the CUDA side):
 *   - Ring R_q = Z_q[X]/(X^N+1); primes q = 1 mod 2N, all < 2^62.
 *   - Polynomials are kept in COEFFICIENT form here, natural order.  The
 *     "NTT form" is defined as NTT(a)[i] = a(psi^(2*brv(i)+1)) mod q,
 *     bit-reversed evaluation order, psi the canonical primitive 2N-th root
 *     (first x = 2,3,... with x^((q-1)/2N) of order 2N).
 *   - Modular products use (unsigned __int128) % q, a different arithmetic
 *     path from the Shoup / Barrett / Montgomery forms of the CUDA kernels.
 *   - Randomness: Philox4x32-10 (Salmon et al., SC'11) keyed by the context
 *     seed, counter = (index, limb, object, domain).
 *
 * The paper (arXiv 2509.08383) assumes an abstract CKKS API with Enc, Dec,
 * add, mult and rotate (Sect. 2.1 "HE Preliminaries"); this file is that API.
 */
#define _GNU_SOURCE
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>
#include <sched.h>

typedef uint64_t u64;
typedef int64_t i64;
typedef uint32_t u32;
typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* parallel loop over independent limbs (pthreads; the arithmetic of  */
/* each iteration does not depend on the thread count)               */
/* ------------------------------------------------------------------ */
typedef void (*pf_body)(void *arg, int i);
typedef struct { pf_body fn; void *arg; int n, next; pthread_mutex_t mu; } pf_state;
static int g_threads = 0;

int or_set_threads(int n) { g_threads = n; return n; }
int or_get_threads(void) {
    if (g_threads > 0) return g_threads;
    const char *e = getenv("OR_THREADS");
    if (e && atoi(e) > 0) return atoi(e);
    cpu_set_t cs;
    if (sched_getaffinity(0, sizeof(cs), &cs) == 0) return CPU_COUNT(&cs);
    return 1;
}
static void *pf_worker(void *p) {
    pf_state *s = (pf_state *)p;
    for (;;) {
        pthread_mutex_lock(&s->mu);
        int i = s->next++;
        pthread_mutex_unlock(&s->mu);
        if (i >= s->n) break;
        s->fn(s->arg, i);
    }
    return NULL;
}
static void parallel_for(int n, pf_body fn, void *arg) {
    int T = or_get_threads();
    if (T > n) T = n;
    if (T > 64) T = 64;
    if (T <= 1) { for (int i = 0; i < n; i++) fn(arg, i); return; }
    pf_state s; s.fn = fn; s.arg = arg; s.n = n; s.next = 0;
    pthread_mutex_init(&s.mu, NULL);
    pthread_t th[64];
    for (int t = 1; t < T; t++) pthread_create(&th[t], NULL, pf_worker, &s);
    pf_worker(&s);
    for (int t = 1; t < T; t++) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&s.mu);
}

/* ------------------------------------------------------------------ */
/* modular arithmetic by definition                                    */
/* ------------------------------------------------------------------ */
static inline u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static inline u64 addmod(u64 a, u64 b, u64 q) { u64 s = a + b; return s >= q ? s - q : s; }
static inline u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

u64 or_powmod(u64 a, u64 e, u64 q) {
    u64 r = 1 % q; a %= q;
    while (e) { if (e & 1) r = mulmod(r, a, q); a = mulmod(a, a, q); e >>= 1; }
    return r;
}
u64 or_invmod(u64 a, u64 q) { return or_powmod(a, q - 2, q); } /* q prime */

/* Deterministic Miller-Rabin for n < 2^64 with the first 12 prime bases. */
int or_is_prime(u64 n) {
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) { if (n % bases[i] == 0) return n == bases[i]; }
    u64 d = n - 1; int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        u64 x = or_powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int comp = 1;
        for (int r = 1; r < s; r++) { x = mulmod(x, x, n); if (x == n - 1) { comp = 0; break; } }
        if (comp) return 0;
    }
    return 1;
}

/* Prime chain rule: primes of b bits are q = k*2N+1 < 2^b taken in
 * decreasing order, one cursor per bit size, in request order. */
int or_gen_primes(int log_n, const int *bits, int count, u64 *out) {
    u64 two_n = 2ull << log_n;
    int used_bits[64]; u64 cursor[64]; int nb = 0;
    for (int i = 0; i < count; i++) {
        int b = bits[i], c = -1;
        if (b < 20 || b > 61) return -1;
        for (int j = 0; j < nb; j++) if (used_bits[j] == b) c = j;
        if (c < 0) { c = nb++; used_bits[c] = b; cursor[c] = ((1ull << b) - 1) / two_n; }
        for (;;) {
            u64 k = cursor[c]--;
            u64 q = k * two_n + 1;
            if (q < (1ull << (b - 1))) return -2;
            if (or_is_prime(q)) { out[i] = q; break; }
        }
    }
    return 0;
}

/* Canonical psi: first x = 2,3,... such that x^((q-1)/2N) has order 2N. */
u64 or_find_psi(u64 q, int log_n) {
    u64 two_n = 2ull << log_n, n = 1ull << log_n;
    for (u64 x = 2;; x++) {
        u64 c = or_powmod(x, (q - 1) / two_n, q);
        if (or_powmod(c, n, q) == q - 1) return c;
    }
}

static inline u32 brv(u32 x, int bits) {
    u32 r = 0;
    for (int i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

/* NTT straight from the definition, O(N^2), for tiny N. */
void or_ntt_def(const u64 *a, u64 *out, int log_n, u64 q, u64 psi) {
    u64 n = 1ull << log_n;
    for (u64 i = 0; i < n; i++) {
        u64 e = 2 * (u64)brv((u32)i, log_n) + 1;
        u64 x = or_powmod(psi, e, q), acc = 0, p = 1;
        for (u64 k = 0; k < n; k++) { acc = addmod(acc, mulmod(a[k], p, q), q); p = mulmod(p, x, q); }
        out[i] = acc;
    }
}

/* Negacyclic product by schoolbook, O(N^2), for tiny N. */
void or_negacyclic_schoolbook(const u64 *a, const u64 *b, u64 *out, int log_n, u64 q) {
    u64 n = 1ull << log_n;
    for (u64 k = 0; k < n; k++) out[k] = 0;
    for (u64 i = 0; i < n; i++)
        for (u64 j = 0; j < n; j++) {
            u64 p = mulmod(a[i], b[j], q);
            u64 k = i + j;
            if (k < n) out[k] = addmod(out[k], p, q);
            else out[k - n] = submod(out[k - n], p, q);
        }
}

/* ------------------------------------------------------------------ */
/* per-prime tables for the textbook radix-2 transform                 */
/* ------------------------------------------------------------------ */
typedef struct {
    u64 q, psi, psi_inv, n_inv;
    u64 *psi_pow, *psi_inv_pow; /* psi^k, psi^-k, k < N */
    u64 *w_pow, *w_inv_pow;     /* w^k, w^-k with w = psi^2, k < N/2 */
} prime_tab;

static void tab_init(prime_tab *t, u64 q, int log_n) {
    u64 n = 1ull << log_n;
    t->q = q; t->psi = or_find_psi(q, log_n); t->psi_inv = or_invmod(t->psi, q);
    t->n_inv = or_invmod(n % q, q);
    t->psi_pow = malloc(n * 8); t->psi_inv_pow = malloc(n * 8);
    t->w_pow = malloc(n / 2 * 8); t->w_inv_pow = malloc(n / 2 * 8);
    u64 w = mulmod(t->psi, t->psi, q), wi = mulmod(t->psi_inv, t->psi_inv, q);
    t->psi_pow[0] = 1; t->psi_inv_pow[0] = 1;
    for (u64 k = 1; k < n; k++) {
        t->psi_pow[k] = mulmod(t->psi_pow[k - 1], t->psi, q);
        t->psi_inv_pow[k] = mulmod(t->psi_inv_pow[k - 1], t->psi_inv, q);
    }
    t->w_pow[0] = 1; t->w_inv_pow[0] = 1;
    for (u64 k = 1; k < n / 2; k++) {
        t->w_pow[k] = mulmod(t->w_pow[k - 1], w, q);
        t->w_inv_pow[k] = mulmod(t->w_inv_pow[k - 1], wi, q);
    }
}
static void tab_free(prime_tab *t) { free(t->psi_pow); free(t->psi_inv_pow); free(t->w_pow); free(t->w_inv_pow); }

/* Cyclic DFT of length N over Z_q with root table wp (w^k, k<N/2), textbook
 * iterative radix-2 decimation in time: bit-reversal copy, then butterflies. */
static void cyclic_dft(u64 *x, int log_n, u64 q, const u64 *wp) {
    u64 n = 1ull << log_n;
    for (u64 i = 0; i < n; i++) {
        u64 j = brv((u32)i, log_n);
        if (j > i) { u64 t = x[i]; x[i] = x[j]; x[j] = t; }
    }
    for (u64 len = 2; len <= n; len <<= 1) {
        u64 half = len >> 1, step = n / len;
        for (u64 i = 0; i < n; i += len)
            for (u64 k = 0; k < half; k++) {
                u64 u = x[i + k], v = mulmod(x[i + k + half], wp[k * step], q);
                x[i + k] = addmod(u, v, q);
                x[i + k + half] = submod(u, v, q);
            }
    }
}

/* NTT: twist by psi^k, cyclic DFT with w = psi^2 (natural order result
 * A_j = a(psi^(2j+1))), then store A_brv(i) at position i. */
static void ntt_tab(u64 *a, int log_n, const prime_tab *t, u64 *tmp) {
    u64 n = 1ull << log_n;
    for (u64 k = 0; k < n; k++) tmp[k] = mulmod(a[k], t->psi_pow[k], t->q);
    cyclic_dft(tmp, log_n, t->q, t->w_pow);
    for (u64 i = 0; i < n; i++) a[i] = tmp[brv((u32)i, log_n)];
}
static void intt_tab(u64 *a, int log_n, const prime_tab *t, u64 *tmp) {
    u64 n = 1ull << log_n;
    for (u64 j = 0; j < n; j++) tmp[j] = a[brv((u32)j, log_n)];
    cyclic_dft(tmp, log_n, t->q, t->w_inv_pow);
    for (u64 k = 0; k < n; k++) a[k] = mulmod(mulmod(tmp[k], t->n_inv, t->q), t->psi_inv_pow[k], t->q);
}

void or_ntt(u64 *a, int log_n, u64 q) {
    prime_tab t; tab_init(&t, q, log_n);
    u64 *tmp = malloc((8ull << log_n)); ntt_tab(a, log_n, &t, tmp); free(tmp); tab_free(&t);
}
void or_intt(u64 *a, int log_n, u64 q) {
    prime_tab t; tab_init(&t, q, log_n);
    u64 *tmp = malloc((8ull << log_n)); intt_tab(a, log_n, &t, tmp); free(tmp); tab_free(&t);
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and samplers      */
/* ------------------------------------------------------------------ */
void or_philox(const u32 ctr_in[4], const u32 key_in[2], u32 out[4]) {
    const u32 M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    u32 c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    u32 k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        if (r) { k0 += W0; k1 += W1; }
        u64 p0 = (u64)M0 * c0, p1 = (u64)M1 * c2;
        u32 n0 = (u32)(p1 >> 32) ^ c1 ^ k0, n1 = (u32)p1;
        u32 n2 = (u32)(p0 >> 32) ^ c3 ^ k1, n3 = (u32)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static inline void philox_block(u64 seed, u32 index, u32 limb, u32 object, u32 domain, u32 out[4]) {
    u32 ctr[4] = {index, limb, object, domain};
    u32 key[2] = {(u32)seed, (u32)(seed >> 32)};
    or_philox(ctr, key, out);
}

enum { DOM_SECRET = 1, DOM_ERROR = 2, DOM_UNIFORM = 3, DOM_KEY_A = 4, DOM_KEY_E = 5, DOM_SPARSE = 6 };

/* uniform residue: one Philox block -> 128-bit integer -> mod q */
static inline u64 uniform_mod(u64 seed, u32 index, u32 limb, u32 object, u32 domain, u64 q) {
    u32 w[4]; philox_block(seed, index, limb, object, domain, w);
    u128 v = ((u128)(((u64)w[3] << 32) | w[2]) << 64) | (((u64)w[1] << 32) | w[0]);
    return (u64)(v % q);
}

/* CDT for the rounded Gaussian of width sigma on |x| <= bound. */
#define GAUSS_BOUND 19
void or_gauss_cdt(double sigma, u64 *table /* GAUSS_BOUND entries */) {
    double rho[GAUSS_BOUND + 1], z = 0.0;
    for (int k = 0; k <= GAUSS_BOUND; k++) {
        rho[k] = exp(-((double)k * (double)k) / (2.0 * sigma * sigma));
        z += (k == 0 ? 1.0 : 2.0) * rho[k];
    }
    double cdf = 0.0;
    for (int k = 0; k < GAUSS_BOUND; k++) {
        cdf += (k == 0 ? 1.0 : 2.0) * rho[k] / z;
        table[k] = (u64)ldexp(cdf, 64);
    }
}
static inline i64 gauss_sample(u64 seed, u32 index, u32 object, u32 domain, const u64 *cdt) {
    u32 w[4]; philox_block(seed, index, 0, object, domain, w);
    u64 u = ((u64)w[1] << 32) | w[0];
    i64 mag = 0;
    for (int k = 0; k < GAUSS_BOUND; k++) mag += (cdt[k] <= u);
    return (w[2] & 1) ? -mag : mag;
}

void or_sample_gauss(u64 seed, u32 object, u32 domain, double sigma, int log_n, i64 *out) {
    u64 cdt[GAUSS_BOUND]; or_gauss_cdt(sigma, cdt);
    for (u64 k = 0; k < (1ull << log_n); k++) out[k] = gauss_sample(seed, (u32)k, object, domain, cdt);
}

/* Dense ternary secret: s_k = floor(3*w/2^32) - 1. Sparse: Fisher-Yates. */
void or_sample_secret(u64 seed, int log_n, int h, int8_t *s) {
    u64 n = 1ull << log_n;
    if (h == 0) {
        for (u64 k = 0; k < n; k++) {
            u32 w[4]; philox_block(seed, (u32)k, 0, 0, DOM_SECRET, w);
            s[k] = (int8_t)((int)(((u64)w[0] * 3) >> 32) - 1);
        }
        return;
    }
    u32 *perm = malloc(n * 4);
    for (u64 k = 0; k < n; k++) { perm[k] = (u32)k; s[k] = 0; }
    for (int i = 0; i < h; i++) {
        u32 w[4]; philox_block(seed, (u32)i, 0, 0, DOM_SPARSE, w);
        u64 j = (u64)i + (((u64)w[0] * (n - (u64)i)) >> 32);
        u32 t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        s[perm[i]] = (w[1] & 1) ? -1 : 1;
    }
    free(perm);
}

/* ------------------------------------------------------------------ */
/* context, keys, ciphertexts                                          */
/* ------------------------------------------------------------------ */
typedef struct {
    u64 g;          /* Galois element; 0 marks the relinearisation key */
    u64 **b, **a;   /* [digit] -> [(nq+np) * N], NTT form */
} or_key;

typedef struct {
    int log_n, nq, np, dnum, alpha, beta, h;
    u64 n, seed;
    double sigma;
    u64 *primes;
    prime_tab *tab;
    int8_t *sk;
    u64 *sk_ntt;     /* [(nq+np) * N] */
    or_key *keys; int nkeys, capkeys;
} or_ctx;

typedef struct {
    int level;       /* limbs 0..level of the Q chain */
    double scale;
    u64 *c[2];       /* coefficient form, [(level+1) * N] each */
} or_ct;

static void poly_ntt(or_ctx *cx, u64 *p, int limb_prime) {
    u64 *tmp = malloc(cx->n * 8); ntt_tab(p, cx->log_n, &cx->tab[limb_prime], tmp); free(tmp);
}
static void poly_intt(or_ctx *cx, u64 *p, int limb_prime) {
    u64 *tmp = malloc(cx->n * 8); intt_tab(p, cx->log_n, &cx->tab[limb_prime], tmp); free(tmp);
}

/* signed integer -> residue */
static inline u64 smod(i64 v, u64 q) { i64 r = v % (i64)q; return r < 0 ? (u64)(r + (i64)q) : (u64)r; }

/* integer-valued double -> residue mod q, exact for any magnitude */
static u64 dmod(double x, u64 q) {
    if (fabs(x) < 9.2e18) return smod((i64)x, q);
    int e; double m = frexp(x, &e);           /* x = m * 2^e, 0.5 <= |m| < 1 */
    i64 mi = (i64)ldexp(m, 53); e -= 53;       /* x = mi * 2^e exactly */
    u64 r = smod(mi, q);
    return mulmod(r, or_powmod(2, (u64)e, q), q);
}

typedef struct { or_ctx *cx; or_key *k; int j; u32 obj; const i64 *e; const u64 *sp; } bk_args;
static void bk_body(void *vp, int i) {
    bk_args *A = (bk_args *)vp;
    or_ctx *cx = A->cx; u64 n = cx->n; int j = A->j;
    u64 q = cx->primes[i];
    u64 *a = A->k->a[j] + (u64)i * n, *b = A->k->b[j] + (u64)i * n;
    for (u64 c = 0; c < n; c++) a[c] = uniform_mod(cx->seed, (u32)c, (u32)i, A->obj, DOM_KEY_A, q);
    for (u64 c = 0; c < n; c++) b[c] = smod(A->e[c], q);
    poly_ntt(cx, b, i);
    u64 pmod = 1;
    for (int p = 0; p < cx->np; p++) pmod = mulmod(pmod, cx->primes[cx->nq + p] % q, q);
    int in_digit = (i < cx->nq) && (i / cx->alpha == j);
    const u64 *s = cx->sk_ntt + (u64)i * n, *s2 = A->sp + (u64)i * n;
    for (u64 c = 0; c < n; c++) {
        u64 v = submod(b[c], mulmod(a[c], s[c], q), q);
        if (in_digit) v = addmod(v, mulmod(pmod, s2[c], q), q);
        b[c] = v;
    }
}

static void build_key(or_ctx *cx, or_key *k, const u64 *s_prime_ntt /*[(nq+np)*N]*/, u32 key_id) {
    u64 n = cx->n; int tot = cx->nq + cx->np;
    u64 cdt[GAUSS_BOUND]; or_gauss_cdt(cx->sigma, cdt);
    k->b = malloc(sizeof(u64 *) * cx->beta); k->a = malloc(sizeof(u64 *) * cx->beta);
    for (int j = 0; j < cx->beta; j++) {
        u32 obj = (key_id << 8) | (u32)j;
        k->b[j] = malloc(tot * n * 8); k->a[j] = malloc(tot * n * 8);
        i64 *e = malloc(n * 8);
        for (u64 c = 0; c < n; c++) e[c] = gauss_sample(cx->seed, (u32)c, obj, DOM_KEY_E, cdt);
        bk_args A = {cx, k, j, obj, e, s_prime_ntt};
        parallel_for(tot, bk_body, &A);
        free(e);
    }
}

static void tab_body(void *vp, int i) {
    or_ctx *cx = (or_ctx *)vp;
    tab_init(&cx->tab[i], cx->primes[i], cx->log_n);
}
static void sk_body(void *vp, int i) {
    or_ctx *cx = (or_ctx *)vp;
    u64 *p = cx->sk_ntt + (u64)i * cx->n;
    for (u64 c = 0; c < cx->n; c++) p[c] = smod(cx->sk[c], cx->primes[i]);
    poly_ntt(cx, p, i);
}

or_ctx *or_ctx_create(int log_n, int nq, int np, const int *qbits, const int *pbits,
                      int dnum, int h, double sigma, u64 seed) {
    or_ctx *cx = calloc(1, sizeof(or_ctx));
    cx->log_n = log_n; cx->n = 1ull << log_n; cx->nq = nq; cx->np = np; cx->dnum = dnum;
    cx->alpha = (nq + dnum - 1) / dnum; cx->beta = (nq + cx->alpha - 1) / cx->alpha;
    cx->h = h; cx->sigma = sigma; cx->seed = seed;
    int tot = nq + np;
    int *bits = malloc(sizeof(int) * tot);
    for (int i = 0; i < nq; i++) bits[i] = qbits[i];
    for (int i = 0; i < np; i++) bits[nq + i] = pbits[i];
    cx->primes = malloc(8 * tot);
    if (or_gen_primes(log_n, bits, tot, cx->primes) != 0) { free(bits); free(cx->primes); free(cx); return NULL; }
    free(bits);
    cx->tab = malloc(sizeof(prime_tab) * tot);
    parallel_for(tot, tab_body, cx);
    cx->sk = malloc(cx->n);
    or_sample_secret(seed, log_n, h, cx->sk);
    cx->sk_ntt = malloc(tot * cx->n * 8);
    parallel_for(tot, sk_body, cx);
    return cx;
}

void or_ctx_free(or_ctx *cx) {
    int tot = cx->nq + cx->np;
    for (int k = 0; k < cx->nkeys; k++) {
        for (int j = 0; j < cx->beta; j++) { free(cx->keys[k].b[j]); free(cx->keys[k].a[j]); }
        free(cx->keys[k].b); free(cx->keys[k].a);
    }
    free(cx->keys);
    for (int i = 0; i < tot; i++) tab_free(&cx->tab[i]);
    free(cx->tab); free(cx->primes); free(cx->sk); free(cx->sk_ntt); free(cx);
}

void or_ctx_info(const or_ctx *cx, u64 *primes, int *alpha_beta) {
    memcpy(primes, cx->primes, 8 * (cx->nq + cx->np));
    alpha_beta[0] = cx->alpha; alpha_beta[1] = cx->beta;
}
void or_ctx_secret(const or_ctx *cx, int8_t *out) { memcpy(out, cx->sk, cx->n); }
u64 or_ctx_psi(const or_ctx *cx, int i) { return cx->tab[i].psi; }

static or_key *find_key(or_ctx *cx, u64 g) {
    for (int k = 0; k < cx->nkeys; k++) if (cx->keys[k].g == g) return &cx->keys[k];
    return NULL;
}
static or_key *new_key(or_ctx *cx, u64 g) {
    if (cx->nkeys == cx->capkeys) {
        cx->capkeys = cx->capkeys ? 2 * cx->capkeys : 8;
        cx->keys = realloc(cx->keys, sizeof(or_key) * cx->capkeys);
    }
    or_key *k = &cx->keys[cx->nkeys++]; k->g = g; return k;
}

/* automorphism X -> X^g on a coefficient-form polynomial mod q */
static void automorph(const u64 *a, u64 *out, u64 n, u64 g, u64 q) {
    u64 two_n = 2 * n;
    for (u64 k = 0; k < n; k++) {
        u64 e = (k * g) % two_n;
        if (e < n) out[e] = a[k]; else out[e - n] = a[k] ? q - a[k] : 0;
    }
}

/* relinearisation key: encrypts P*s^2 digit-wise (hybrid key switching) */
void or_gen_relin_key(or_ctx *cx) {
    if (find_key(cx, 0)) return;
    int tot = cx->nq + cx->np; u64 n = cx->n;
    u64 *s2 = malloc(tot * n * 8);
    for (u64 i = 0; i < (u64)tot * n; i++) s2[i] = mulmod(cx->sk_ntt[i], cx->sk_ntt[i], cx->primes[i / n]);
    or_key *k = new_key(cx, 0);
    build_key(cx, k, s2, 0);
    free(s2);
}

/* Galois key for X -> X^g: encrypts P*s(X^g) */
void or_gen_galois_key(or_ctx *cx, u64 g) {
    if (find_key(cx, g)) return;
    int tot = cx->nq + cx->np; u64 n = cx->n;
    u64 *sg = malloc(tot * n * 8);
    u64 *sc = malloc(n * 8);
    for (int i = 0; i < tot; i++) {
        u64 q = cx->primes[i];
        for (u64 c = 0; c < n; c++) sc[c] = smod(cx->sk[c], q);
        automorph(sc, sg + (u64)i * n, n, g, q);
        poly_ntt(cx, sg + (u64)i * n, i);
    }
    free(sc);
    or_key *k = new_key(cx, g);
    build_key(cx, k, sg, (u32)g);
    free(sg);
}

/* export a key digit in coefficient form: which=0 -> b, 1 -> a */
int or_key_export(or_ctx *cx, u64 g, int digit, int which, u64 *out) {
    or_key *k = find_key(cx, g);
    if (!k || digit >= cx->beta) return -1;
    int tot = cx->nq + cx->np; u64 n = cx->n;
    memcpy(out, which ? k->a[digit] : k->b[digit], tot * n * 8);
    for (int i = 0; i < tot; i++) poly_intt(cx, out + (u64)i * n, i);
    return 0;
}

or_ct *or_ct_new(or_ctx *cx, int level, double scale) {
    or_ct *ct = malloc(sizeof(or_ct));
    ct->level = level; ct->scale = scale;
    ct->c[0] = calloc((level + 1) * cx->n, 8); ct->c[1] = calloc((level + 1) * cx->n, 8);
    return ct;
}
void or_ct_free(or_ct *ct) { if (!ct) return; free(ct->c[0]); free(ct->c[1]); free(ct); }
int or_ct_level(const or_ct *ct) { return ct->level; }
double or_ct_scale(const or_ct *ct) { return ct->scale; }
void or_ct_set_scale(or_ct *ct, double s) { ct->scale = s; }
void or_ct_export(or_ctx *cx, const or_ct *ct, u64 *out) {
    u64 m = (ct->level + 1) * cx->n;
    memcpy(out, ct->c[0], m * 8); memcpy(out + m, ct->c[1], m * 8);
}
or_ct *or_ct_import(or_ctx *cx, const u64 *in, int level, double scale) {
    or_ct *ct = or_ct_new(cx, level, scale);
    u64 m = (level + 1) * cx->n;
    memcpy(ct->c[0], in, m * 8); memcpy(ct->c[1], in + m, m * 8);
    return ct;
}

/* Secret-key encryption of an integer plaintext polynomial (coefficients
 * given as integer-valued doubles): c1 = a, c0 = -a*s + e + m, at `level`.
 * a is uniform in the NTT domain; e is the rounded Gaussian. */
typedef struct { or_ctx *cx; or_ct *ct; u32 ctr; const i64 *e; const double *m; } enc_args;
static void enc_body(void *vp, int i) {
    enc_args *A = (enc_args *)vp;
    or_ctx *cx = A->cx; u64 n = cx->n, q = cx->primes[i];
    u64 *c0 = A->ct->c[0] + (u64)i * n, *c1 = A->ct->c[1] + (u64)i * n;
    for (u64 c = 0; c < n; c++) c1[c] = uniform_mod(cx->seed, (u32)c, (u32)i, A->ctr, DOM_UNIFORM, q);
    for (u64 c = 0; c < n; c++) c0[c] = addmod(smod(A->e[c], q), dmod(A->m[c], q), q);
    poly_ntt(cx, c0, i);
    const u64 *s = cx->sk_ntt + (u64)i * n;
    for (u64 c = 0; c < n; c++) c0[c] = submod(c0[c], mulmod(c1[c], s[c], q), q);
    poly_intt(cx, c0, i);
    poly_intt(cx, c1, i);
}

or_ct *or_encrypt(or_ctx *cx, const double *m, double scale, u32 ctr, int level) {
    if (level < 0 || level >= cx->nq) return NULL;  /* no such level: the caller raises */
    u64 n = cx->n;
    or_ct *ct = or_ct_new(cx, level, scale);
    u64 cdt[GAUSS_BOUND]; or_gauss_cdt(cx->sigma, cdt);
    i64 *e = malloc(n * 8);
    for (u64 c = 0; c < n; c++) e[c] = gauss_sample(cx->seed, (u32)c, ctr, DOM_ERROR, cdt);
    enc_args A = {cx, ct, ctr, e, m};
    parallel_for(level + 1, enc_body, &A);
    free(e);
    return ct;
}

/* Decryption: m = c0 + c1*s; returns the centred integer value of m mod
 * q0*q1 (or q0 at level 0) as a double, coefficient by coefficient. */
void or_decrypt(or_ctx *cx, const or_ct *ct, double *out) {
    u64 n = cx->n; int nl = ct->level >= 1 ? 2 : 1;
    u64 *m = malloc(nl * n * 8);
    for (int i = 0; i < nl; i++) {
        u64 q = cx->primes[i];
        u64 *mi = m + (u64)i * n, *t = malloc(n * 8);
        memcpy(t, ct->c[1] + (u64)i * n, n * 8);
        poly_ntt(cx, t, i);
        const u64 *s = cx->sk_ntt + (u64)i * n;
        for (u64 c = 0; c < n; c++) t[c] = mulmod(t[c], s[c], q);
        poly_intt(cx, t, i);
        for (u64 c = 0; c < n; c++) mi[c] = addmod(ct->c[0][(u64)i * n + c], t[c], q);
        free(t);
    }
    u64 q0 = cx->primes[0];
    if (nl == 1) {
        for (u64 c = 0; c < n; c++) out[c] = m[c] > q0 / 2 ? -(double)(q0 - m[c]) : (double)m[c];
    } else {
        u64 q1 = cx->primes[1], q0inv = or_invmod(q0 % q1, q1);
        u128 Q = (u128)q0 * q1;
        for (u64 c = 0; c < n; c++) {
            u64 x0 = m[c], x1 = m[n + c];
            u64 k = mulmod(submod(x1, x0 % q1, q1), q0inv, q1);
            u128 v = (u128)x0 + (u128)q0 * k;       /* CRT value in [0, q0 q1) */
            if (v > Q / 2) out[c] = -(double)(Q - v); else out[c] = (double)v;
        }
    }
    free(m);
}

/* ---------------- elementary homomorphic operations ---------------- */
static or_ct *ct_copy_to_level(or_ctx *cx, const or_ct *a, int level) {
    or_ct *r = or_ct_new(cx, level, a->scale);
    u64 m = (level + 1) * cx->n;
    memcpy(r->c[0], a->c[0], m * 8); memcpy(r->c[1], a->c[1], m * 8);
    return r;
}
or_ct *or_drop(or_ctx *cx, const or_ct *a, int level) { return ct_copy_to_level(cx, a, level); }

or_ct *or_add(or_ctx *cx, const or_ct *a, const or_ct *b, int negate_b) {
    int l = a->level < b->level ? a->level : b->level;
    or_ct *r = or_ct_new(cx, l, a->scale);
    for (int k = 0; k < 2; k++)
        for (int i = 0; i <= l; i++) {
            u64 q = cx->primes[i];
            for (u64 c = 0; c < cx->n; c++) {
                u64 x = a->c[k][(u64)i * cx->n + c], y = b->c[k][(u64)i * cx->n + c];
                r->c[k][(u64)i * cx->n + c] = negate_b ? submod(x, y, q) : addmod(x, y, q);
            }
        }
    return r;
}

/* multiply by the integer k (any sign); the scale is unchanged */
or_ct *or_mul_int(or_ctx *cx, const or_ct *a, i64 k) {
    or_ct *r = or_ct_new(cx, a->level, a->scale);
    for (int j = 0; j < 2; j++)
        for (int i = 0; i <= a->level; i++) {
            u64 q = cx->primes[i], km = smod(k, q);
            for (u64 c = 0; c < cx->n; c++) r->c[j][(u64)i * cx->n + c] = mulmod(a->c[j][(u64)i * cx->n + c], km, q);
        }
    return r;
}

/* multiply by the integer-valued double K; the scale becomes scale * new_scale_factor */
or_ct *or_mul_intd(or_ctx *cx, const or_ct *a, double K, double scale_out) {
    or_ct *r = or_ct_new(cx, a->level, scale_out);
    for (int j = 0; j < 2; j++)
        for (int i = 0; i <= a->level; i++) {
            u64 q = cx->primes[i], km = dmod(K, q);
            for (u64 c = 0; c < cx->n; c++) r->c[j][(u64)i * cx->n + c] = mulmod(a->c[j][(u64)i * cx->n + c], km, q);
        }
    return r;
}

/* add the integer-valued double K to every slot's plaintext (coefficient 0) */
or_ct *or_add_intd(or_ctx *cx, const or_ct *a, double K) {
    or_ct *r = ct_copy_to_level(cx, a, a->level);
    for (int i = 0; i <= a->level; i++) {
        u64 q = cx->primes[i];
        r->c[0][(u64)i * cx->n] = addmod(r->c[0][(u64)i * cx->n], dmod(K, q), q);
    }
    return r;
}

/* add an integer plaintext polynomial (integer-valued doubles) */
or_ct *or_add_plain(or_ctx *cx, const or_ct *a, const double *pt) {
    or_ct *r = ct_copy_to_level(cx, a, a->level);
    for (int i = 0; i <= a->level; i++) {
        u64 q = cx->primes[i];
        for (u64 c = 0; c < cx->n; c++)
            r->c[0][(u64)i * cx->n + c] = addmod(r->c[0][(u64)i * cx->n + c], dmod(pt[c], q), q);
    }
    return r;
}

/* multiply by an integer plaintext polynomial; scale becomes scale_out */
typedef struct { or_ctx *cx; const or_ct *a; or_ct *r; const double *pt; } mp_args;
static void mp_body(void *vp, int i) {
    mp_args *A = (mp_args *)vp;
    or_ctx *cx = A->cx; u64 n = cx->n, q = cx->primes[i];
    u64 *p = malloc(n * 8), *t = malloc(n * 8);
    for (u64 c = 0; c < n; c++) p[c] = dmod(A->pt[c], q);
    poly_ntt(cx, p, i);
    for (int j = 0; j < 2; j++) {
        memcpy(t, A->a->c[j] + (u64)i * n, n * 8);
        poly_ntt(cx, t, i);
        for (u64 c = 0; c < n; c++) t[c] = mulmod(t[c], p[c], q);
        poly_intt(cx, t, i);
        memcpy(A->r->c[j] + (u64)i * n, t, n * 8);
    }
    free(p); free(t);
}

or_ct *or_mul_plain(or_ctx *cx, const or_ct *a, const double *pt, double scale_out) {
    or_ct *r = or_ct_new(cx, a->level, scale_out);
    mp_args A = {cx, a, r, pt};
    parallel_for(a->level + 1, mp_body, &A);
    return r;
}

/* ModUp of one digit: the approximate basis conversion
 *   [x]_t = sum_{i in D_j} [x_i * (Qhat_i)^-1]_{q_i} * Qhat_i  mod t
 * (its overflow, a small multiple of the digit modulus, is divided away by
 * P with the key's error), then the product with the key, accumulated. */
typedef struct {
    or_ctx *cx; const u64 *d; const or_key *key; int j, lo, hi, cnt; const u64 *qhinv; const int *pidx;
    u64 *acc0, *acc1;
} mu_args;
static void mu_body(void *vp, int t) {
    mu_args *A = (mu_args *)vp;
    or_ctx *cx = A->cx; u64 n = cx->n;
    int pt = A->pidx[t], lo = A->lo, hi = A->hi, cnt = A->cnt;
    u64 qt = cx->primes[pt];
    u64 *e = malloc(n * 8);
    if (pt >= lo && pt < hi) {
        memcpy(e, A->d + (u64)pt * n, n * 8);
    } else {
        u64 *qh = malloc(8 * cnt);
        for (int a = 0; a < cnt; a++) {
            u64 v = 1;
            for (int b = 0; b < cnt; b++) if (b != a) v = mulmod(v, cx->primes[lo + b] % qt, qt);
            qh[a] = v;
        }
        for (u64 c = 0; c < n; c++) {
            u64 s = 0;
            for (int a = 0; a < cnt; a++) {
                u64 qa = cx->primes[lo + a];
                u64 y = mulmod(A->d[(u64)(lo + a) * n + c], A->qhinv[a], qa);
                s = addmod(s, mulmod(y % qt, qh[a], qt), qt);
            }
            e[c] = s;
        }
        free(qh);
    }
    poly_ntt(cx, e, pt);
    const u64 *kb = A->key->b[A->j] + (u64)pt * n, *ka = A->key->a[A->j] + (u64)pt * n;
    u64 *a0 = A->acc0 + (u64)t * n, *a1 = A->acc1 + (u64)t * n;
    for (u64 c = 0; c < n; c++) {
        a0[c] = addmod(a0[c], mulmod(e[c], kb[c], qt), qt);
        a1[c] = addmod(a1[c], mulmod(e[c], ka[c], qt), qt);
    }
    free(e);
}
typedef struct { or_ctx *cx; u64 *acc0, *acc1; int ext; const int *pidx; } it_args;
static void it_body(void *vp, int t) {
    it_args *A = (it_args *)vp;
    u64 *p = (t < A->ext ? A->acc0 + (u64)t * A->cx->n : A->acc1 + (u64)(t - A->ext) * A->cx->n);
    poly_intt(A->cx, p, A->pidx[t % A->ext]);
}
/* Rounded division by a product M of some of the basis primes: ModDown
 * divides by P (the special primes), the product with its rescale by P q_l.
 * The rows d0 .. d0+K-1 of the accumulators hold x mod the divisor primes
 * dp[0..K-1]; for every coefficient Garner's algorithm gives the mixed-radix
 * digits x mod M = m_0 + m_1 dp_0 + m_2 dp_0 dp_1 + ... (m_k < dp_k);
 * comparing them, most significant first, with the digits of (M-1)/2 picks
 * the centred representative x_c = x mod M, or that minus M; then for the
 * output rows i < n_out
 *   out_i = (acc_i - x_c) * M^-1 mod q_i = round(x / M) mod q_i,
 * exact, with x_c reduced mod q_i from its digits. */
typedef struct {
    or_ctx *cx; const u64 *acc0, *acc1; int d0, K, chunk; const u64 *dp; u64 *dig0, *dig1;
    unsigned char *hi0, *hi1; const u64 *pjinv, *hdig;
} gd_args;
static void gd_body(void *vp, int job) {
    gd_args *A = (gd_args *)vp;
    or_ctx *cx = A->cx; u64 n = cx->n; int K = A->K;
    int nch = (int)((n + A->chunk - 1) / A->chunk), w = job / nch;
    u64 c0 = (u64)(job % nch) * A->chunk, c1 = c0 + A->chunk < n ? c0 + A->chunk : n;
    const u64 *acc = w ? A->acc1 : A->acc0;
    u64 *dig = w ? A->dig1 : A->dig0;
    unsigned char *hi = w ? A->hi1 : A->hi0;
    for (u64 c = c0; c < c1; c++) {
        for (int k = 0; k < K; k++) {
            u64 pk = A->dp[k], t = acc[(u64)(A->d0 + k) * n + c];
            for (int j = 0; j < k; j++) t = mulmod(submod(t, dig[(u64)j * n + c] % pk, pk), A->pjinv[j * K + k], pk);
            dig[(u64)k * n + c] = t;
        }
        int above = 0;
        for (int k = K - 1; k >= 0; k--) {
            u64 m = dig[(u64)k * n + c];
            if (m != A->hdig[k]) { above = m > A->hdig[k]; break; }
        }
        hi[c] = (unsigned char)above;
    }
}
typedef struct {
    or_ctx *cx; const u64 *acc0, *acc1; u64 *out0, *out1; int K; const u64 *dp; const u64 *dig0, *dig1;
    const unsigned char *hi0, *hi1;
} md_args;
static void md_body(void *vp, int i) {
    md_args *A = (md_args *)vp;
    or_ctx *cx = A->cx; u64 n = cx->n; int K = A->K;
    u64 qi = cx->primes[i], pm = 1, *radix = malloc(8 * K);
    for (int a = 0; a < K; a++) {  /* radix[a] = dp_0 ... dp_(a-1) mod q_i */
        radix[a] = pm;
        pm = mulmod(pm, A->dp[a] % qi, qi);
    }
    u64 pinv = or_invmod(pm, qi);
    for (int w = 0; w < 2; w++) {
        const u64 *acc = w ? A->acc1 : A->acc0, *dig = w ? A->dig1 : A->dig0;
        const unsigned char *hi = w ? A->hi1 : A->hi0;
        u64 *out = w ? A->out1 : A->out0;
        for (u64 c = 0; c < n; c++) {
            u64 xc = 0;
            for (int a = 0; a < K; a++) xc = addmod(xc, mulmod(dig[(u64)a * n + c] % qi, radix[a], qi), qi);
            if (hi[c]) xc = submod(xc, pm, qi);
            out[(u64)i * n + c] = mulmod(submod(acc[(u64)i * n + c], xc, qi), pinv, qi);
        }
    }
    free(radix);
}

/* mixed-radix digits of (M-1)/2 (residues (dp_k - 1)/2) and dp_j^-1 mod dp_k */
static void divide_consts(const u64 *dp, int K, u64 *pjinv, u64 *hdig) {
    for (int j = 0; j < K; j++)
        for (int k = 0; k < K; k++) pjinv[j * K + k] = j == k ? 0 : or_invmod(dp[j] % dp[k], dp[k]);
    for (int k = 0; k < K; k++) {
        u64 pk = dp[k], t = (pk - 1) / 2;
        for (int j = 0; j < k; j++) t = mulmod(submod(t, hdig[j] % pk, pk), pjinv[j * K + k], pk);
        hdig[k] = t;
    }
}

static void divide_round_exact(or_ctx *cx, const u64 *acc0, const u64 *acc1, int d0, const u64 *dp, int K,
                               int n_out, u64 *out0, u64 *out1) {
    u64 n = cx->n; int chunk = 1024;
    u64 *pjinv = malloc(8 * K * K), *hdig = malloc(8 * K);
    divide_consts(dp, K, pjinv, hdig);
    u64 *dig0 = malloc((u64)K * n * 8), *dig1 = malloc((u64)K * n * 8);
    unsigned char *hi0 = malloc(n), *hi1 = malloc(n);
    gd_args G = {cx, acc0, acc1, d0, K, chunk, dp, dig0, dig1, hi0, hi1, pjinv, hdig};
    parallel_for(2 * (int)((n + chunk - 1) / chunk), gd_body, &G);
    md_args M = {cx, acc0, acc1, out0, out1, K, dp, dig0, dig1, hi0, hi1};
    parallel_for(n_out, md_body, &M);
    free(pjinv); free(hdig); free(dig0); free(dig1); free(hi0); free(hi1);
}

/* ModDown: the rounded division by P of accumulators over q_0..q_l, p_0..p_(K-1) */
static void moddown_exact(or_ctx *cx, const u64 *acc0, const u64 *acc1, int l, u64 *out0, u64 *out1) {
    divide_round_exact(cx, acc0, acc1, l + 1, cx->primes + cx->nq, cx->np, l + 1, out0, out1);
}

/* Hybrid key switching of the coefficient-form polynomial d at level l.
 * ModUp per digit by the approximate basis conversion
 *   [x]_t = sum_{i in D_j} [x_i * (Qhat_i)^-1]_{q_i} * Qhat_i  mod t,
 * inner product with the key over Q_l u P, then ModDown, the rounded
 * division by P (moddown_exact). */
/* The key products of hybrid key switching, before ModDown: acc0/acc1
 * [(l+1+K)][N] in coefficient form over q_0..q_l, p_0..p_(K-1) (caller's
 * buffers, zeroed here). */
static void ks_accumulate(or_ctx *cx, const u64 *d, int l, const or_key *key, u64 *acc0, u64 *acc1) {
    u64 n = cx->n; int K = cx->np, ext = l + 1 + K;
    int beta = (l + 1 + cx->alpha - 1) / cx->alpha;
    int *pidx = malloc(sizeof(int) * ext);
    for (int t = 0; t <= l; t++) pidx[t] = t;
    for (int t = 0; t < K; t++) pidx[l + 1 + t] = cx->nq + t;
    memset(acc0, 0, (u64)ext * n * 8);
    memset(acc1, 0, (u64)ext * n * 8);
    for (int j = 0; j < beta; j++) {
        int lo = j * cx->alpha, hi = lo + cx->alpha; if (hi > l + 1) hi = l + 1;
        int cnt = hi - lo;
        u64 *qhinv = malloc(8 * cnt);
        for (int a = 0; a < cnt; a++) {
            u64 q = cx->primes[lo + a], v = 1;
            for (int b = 0; b < cnt; b++) if (b != a) v = mulmod(v, cx->primes[lo + b] % q, q);
            qhinv[a] = or_invmod(v, q);
        }
        mu_args A = {cx, d, key, j, lo, hi, cnt, qhinv, pidx, acc0, acc1};
        parallel_for(ext, mu_body, &A);
        free(qhinv);
    }
    it_args B = {cx, acc0, acc1, ext, pidx};
    parallel_for(2 * ext, it_body, &B);
    free(pidx);
}

static void keyswitch(or_ctx *cx, const u64 *d, int l, const or_key *key, u64 *out0, u64 *out1) {
    u64 ext = (u64)(l + 1 + cx->np) * cx->n;
    u64 *acc0 = malloc(ext * 8), *acc1 = malloc(ext * 8);
    ks_accumulate(cx, d, l, key, acc0, acc1);
    moddown_exact(cx, acc0, acc1, l, out0, out1);
    free(acc0); free(acc1);
}

/* ModDown exposed for tests: acc0/acc1 coefficient form over q_0..q_l then
 * p_0..p_(K-1), [(l+1+K)][N] each; out0/out1 [(l+1)][N] */
void or_moddown(or_ctx *cx, const u64 *acc0, const u64 *acc1, int l, u64 *out0, u64 *out1) {
    moddown_exact(cx, acc0, acc1, l, out0, out1);
}

/* key switch exposed for tests: d coefficient form at level l */
int or_keyswitch(or_ctx *cx, const u64 *d, int l, u64 g, u64 *out0, u64 *out1) {
    or_key *k = find_key(cx, g);
    if (!k) return -1;
    keyswitch(cx, d, l, k, out0, out1);
    return 0;
}

typedef struct { or_ctx *cx; const or_ct *a, *b; or_ct *r; u64 *d2; } tp_args;
static void tp_body(void *vp, int i) {
    tp_args *A = (tp_args *)vp;
    or_ctx *cx = A->cx; u64 n = cx->n, q = cx->primes[i];
    u64 *a0 = malloc(n * 8), *a1 = malloc(n * 8), *b0 = malloc(n * 8), *b1 = malloc(n * 8);
    memcpy(a0, A->a->c[0] + (u64)i * n, n * 8); memcpy(a1, A->a->c[1] + (u64)i * n, n * 8);
    memcpy(b0, A->b->c[0] + (u64)i * n, n * 8); memcpy(b1, A->b->c[1] + (u64)i * n, n * 8);
    poly_ntt(cx, a0, i); poly_ntt(cx, a1, i); poly_ntt(cx, b0, i); poly_ntt(cx, b1, i);
    u64 *d0 = A->r->c[0] + (u64)i * n, *d1 = A->r->c[1] + (u64)i * n, *e2 = A->d2 + (u64)i * n;
    for (u64 c = 0; c < n; c++) {
        d0[c] = mulmod(a0[c], b0[c], q);
        d1[c] = addmod(mulmod(a0[c], b1[c], q), mulmod(a1[c], b0[c], q), q);
        e2[c] = mulmod(a1[c], b1[c], q);
    }
    poly_intt(cx, d0, i); poly_intt(cx, d1, i); poly_intt(cx, e2, i);
    free(a0); free(a1); free(b0); free(b1);
}

/* tensor product + relinearisation (no rescale); scale = a.scale * b.scale */
or_ct *or_mul(or_ctx *cx, const or_ct *a, const or_ct *b) {
    or_key *rk = find_key(cx, 0);
    if (!rk) return NULL;
    int l = a->level < b->level ? a->level : b->level;
    u64 n = cx->n;
    or_ct *r = or_ct_new(cx, l, a->scale * b->scale);
    u64 *d2 = malloc((l + 1) * n * 8);
    tp_args A = {cx, a, b, r, d2};
    parallel_for(l + 1, tp_body, &A);
    u64 *o0 = malloc((l + 1) * n * 8), *o1 = malloc((l + 1) * n * 8);
    keyswitch(cx, d2, l, rk, o0, o1);
    for (int i = 0; i <= l; i++) {
        u64 q = cx->primes[i];
        for (u64 c = 0; c < n; c++) {
            u64 x = (u64)i * n + c;
            r->c[0][x] = addmod(r->c[0][x], o0[x], q);
            r->c[1][x] = addmod(r->c[1][x], o1[x], q);
        }
    }
    free(d2); free(o0); free(o1);
    return r;
}

/* Product, relinearisation and rescale with ONE rounding: the tensor product
 * (d0, d1, d2) at level l, the key products acc of d2 over Q_l u P, then
 *   out_k = round((P d_k + acc_k) / (P q_l))  mod q_0..q_(l-1),
 * the exact rounded division by P q_l (q_l's row and the special rows are the
 * divisor; divide_round_exact).  The message is that of rescale(mul(a, b))
 * at the same level and scale; the ciphertext differs by that rounding. */
or_ct *or_mul_rescale(or_ctx *cx, const or_ct *a, const or_ct *b) {
    or_key *rk = find_key(cx, 0);
    int l = a->level < b->level ? a->level : b->level;
    if (!rk || l < 1) return NULL;
    u64 n = cx->n; int K = cx->np; u64 ext = (u64)(l + 1 + K) * n;
    or_ct *t = or_ct_new(cx, l, a->scale * b->scale);
    u64 *d2 = malloc((l + 1) * n * 8);
    tp_args A = {cx, a, b, t, d2};
    parallel_for(l + 1, tp_body, &A);
    u64 *acc0 = malloc(ext * 8), *acc1 = malloc(ext * 8);
    ks_accumulate(cx, d2, l, rk, acc0, acc1);
    for (int i = 0; i <= l; i++) {
        u64 q = cx->primes[i], pm = 1;
        for (int p = 0; p < K; p++) pm = mulmod(pm, cx->primes[cx->nq + p] % q, q);
        for (u64 c = 0; c < n; c++) {
            u64 x = (u64)i * n + c;
            acc0[x] = addmod(acc0[x], mulmod(t->c[0][x], pm, q), q);
            acc1[x] = addmod(acc1[x], mulmod(t->c[1][x], pm, q), q);
        }
    }
    u64 *dp = malloc(8 * (K + 1));
    dp[0] = cx->primes[l];
    for (int p = 0; p < K; p++) dp[1 + p] = cx->primes[cx->nq + p];
    or_ct *r = or_ct_new(cx, l - 1, a->scale * b->scale / (double)cx->primes[l]);
    divide_round_exact(cx, acc0, acc1, l, dp, K + 1, l, r->c[0], r->c[1]);
    free(dp); free(d2); free(acc0); free(acc1); or_ct_free(t);
    return r;
}

/* Rescale: divide by the last prime q_l with rounding, i.e. subtract the
 * centred representative of the last limb and multiply by q_l^-1. */
or_ct *or_rescale(or_ctx *cx, const or_ct *a) {
    int l = a->level; u64 n = cx->n, ql = cx->primes[l];
    or_ct *r = or_ct_new(cx, l - 1, a->scale / (double)ql);
    for (int k = 0; k < 2; k++)
        for (int i = 0; i < l; i++) {
            u64 q = cx->primes[i], qlinv = or_invmod(ql % q, q);
            for (u64 c = 0; c < n; c++) {
                u64 v = a->c[k][(u64)l * n + c];
                u64 vm = v <= (ql - 1) / 2 ? v % q : submod(v % q, ql % q, q);
                r->c[k][(u64)i * n + c] = mulmod(submod(a->c[k][(u64)i * n + c], vm, q), qlinv, q);
            }
        }
    return r;
}

/* Apply X -> X^g and key-switch back to s. */
or_ct *or_automorphism(or_ctx *cx, const or_ct *a, u64 g) {
    or_key *k = find_key(cx, g);
    if (!k) return NULL;
    int l = a->level; u64 n = cx->n;
    or_ct *r = or_ct_new(cx, l, a->scale);
    u64 *c1g = malloc((l + 1) * n * 8), *o0 = malloc((l + 1) * n * 8);
    for (int i = 0; i <= l; i++) {
        automorph(a->c[0] + (u64)i * n, r->c[0] + (u64)i * n, n, g, cx->primes[i]);
        automorph(a->c[1] + (u64)i * n, c1g + (u64)i * n, n, g, cx->primes[i]);
    }
    keyswitch(cx, c1g, l, k, o0, r->c[1]);
    for (int i = 0; i <= l; i++) {
        u64 q = cx->primes[i];
        for (u64 c = 0; c < n; c++) r->c[0][(u64)i * n + c] = addmod(r->c[0][(u64)i * n + c], o0[(u64)i * n + c], q);
    }
    free(c1g); free(o0);
    return r;
}

/* Galois element of a left slot rotation by r: 5^r mod 2N */
u64 or_rot_galois(int log_n, i64 r) {
    u64 two_n = 2ull << log_n, slots = 1ull << (log_n - 1);
    i64 rr = r % (i64)slots; if (rr < 0) rr += (i64)slots;
    u64 g = 1;
    for (i64 i = 0; i < rr; i++) g = (g * 5) % two_n;
    return g;
}

/* One hoisted rotate-and-sum stage (App. D's rotate-and-sum, hoisted as by
 * Halevi and Shoup): out = a + sum_r rot(a, rots[r]).
 *   ext_j = ModUp of c1 for digit j (coefficient form; the digit's own rows
 *           are c1 itself), computed ONCE;
 *   acc   = sum_r sum_j NTT(sigma_r(ext_j)) * key_r,j  over Q_l u P, plus
 *           P * (c0 + sum_r sigma_r(c0)) on the Q rows;
 *   out   = (ModDown(acc_0), ModDown(acc_1) + c1).
 * sigma_r is X -> X^g_r applied to each row's coefficients mod its prime.
 * Returns NULL when a rotation key is missing. */
typedef struct {
    or_ctx *cx; const or_ct *a; int l, ext, beta, nr; const u64 *gal; or_key *const *keys; const int *pidx;
    const u64 *ecoef; u64 *acc0, *acc1;
} rs_args;
static void rs_ext_body(void *vp, int t) {
    /* ext rows of every digit for target row t (coefficient form) */
    rs_args *A = (rs_args *)vp;
    or_ctx *cx = A->cx; u64 n = cx->n; int pt = A->pidx[t]; u64 qt = cx->primes[pt];
    const u64 *d = A->a->c[1];
    u64 *ec = (u64 *)A->ecoef;
    for (int j = 0; j < A->beta; j++) {
        int lo = j * cx->alpha, hi = lo + cx->alpha; if (hi > A->l + 1) hi = A->l + 1;
        int cnt = hi - lo;
        u64 *e = ec + ((u64)j * A->ext + t) * n;
        if (pt >= lo && pt < hi) { memcpy(e, d + (u64)pt * n, n * 8); continue; }
        u64 *qhinv = malloc(8 * cnt), *qh = malloc(8 * cnt);
        for (int a = 0; a < cnt; a++) {
            u64 q = cx->primes[lo + a], v = 1, w = 1;
            for (int b = 0; b < cnt; b++)
                if (b != a) { v = mulmod(v, cx->primes[lo + b] % q, q); w = mulmod(w, cx->primes[lo + b] % qt, qt); }
            qhinv[a] = or_invmod(v, q);
            qh[a] = w;
        }
        for (u64 c = 0; c < n; c++) {
            u64 sum = 0;
            for (int a = 0; a < cnt; a++) {
                u64 qa = cx->primes[lo + a];
                u64 y = mulmod(d[(u64)(lo + a) * n + c], qhinv[a], qa);
                sum = addmod(sum, mulmod(y % qt, qh[a], qt), qt);
            }
            e[c] = sum;
        }
        free(qhinv); free(qh);
    }
}
static void rs_acc_body(void *vp, int t) {
    rs_args *A = (rs_args *)vp;
    or_ctx *cx = A->cx; u64 n = cx->n; int pt = A->pidx[t]; u64 q = cx->primes[pt];
    u64 *e = malloc(n * 8), *y = malloc(n * 8);
    u64 *a0 = A->acc0 + (u64)t * n, *a1 = A->acc1 + (u64)t * n;
    for (int r = 0; r < A->nr; r++)
        for (int j = 0; j < A->beta; j++) {
            automorph(A->ecoef + ((u64)j * A->ext + t) * n, e, n, A->gal[r], q);
            poly_ntt(cx, e, pt);
            const u64 *kb = A->keys[r]->b[j] + (u64)pt * n, *ka = A->keys[r]->a[j] + (u64)pt * n;
            for (u64 c = 0; c < n; c++) {
                a0[c] = addmod(a0[c], mulmod(e[c], kb[c], q), q);
                a1[c] = addmod(a1[c], mulmod(e[c], ka[c], q), q);
            }
        }
    if (t <= A->l) {
        const u64 *c0 = A->a->c[0] + (u64)t * n;
        memcpy(y, c0, n * 8);
        for (int r = 0; r < A->nr; r++) {
            automorph(c0, e, n, A->gal[r], q);
            for (u64 c = 0; c < n; c++) y[c] = addmod(y[c], e[c], q);
        }
        u64 pm = 1;
        for (int p = 0; p < cx->np; p++) pm = mulmod(pm, cx->primes[cx->nq + p] % q, q);
        for (u64 c = 0; c < n; c++) y[c] = mulmod(y[c], pm, q);
        poly_ntt(cx, y, pt);
        for (u64 c = 0; c < n; c++) a0[c] = addmod(a0[c], y[c], q);
    }
    free(e); free(y);
}
or_ct *or_rotsum_stage(or_ctx *cx, const or_ct *a, const i64 *rots, int n_rots) {
    if (n_rots < 1) return NULL;
    int l = a->level, K = cx->np, ext = l + 1 + K; u64 n = cx->n;
    int beta = (l + 1 + cx->alpha - 1) / cx->alpha;
    u64 *gal = malloc(8 * n_rots);
    or_key **keys = malloc(sizeof(or_key *) * n_rots);
    for (int r = 0; r < n_rots; r++) {
        gal[r] = or_rot_galois(cx->log_n, rots[r]);
        keys[r] = find_key(cx, gal[r]);
        if (!keys[r]) { free(gal); free(keys); return NULL; }
    }
    int *pidx = malloc(sizeof(int) * ext);
    for (int t = 0; t <= l; t++) pidx[t] = t;
    for (int t = 0; t < K; t++) pidx[l + 1 + t] = cx->nq + t;
    u64 *ecoef = malloc((u64)beta * ext * n * 8);
    u64 *acc0 = calloc((u64)ext * n, 8), *acc1 = calloc((u64)ext * n, 8);
    rs_args A = {cx, a, l, ext, beta, n_rots, gal, keys, pidx, ecoef, acc0, acc1};
    parallel_for(ext, rs_ext_body, &A);
    parallel_for(ext, rs_acc_body, &A);
    it_args B = {cx, acc0, acc1, ext, pidx};
    parallel_for(2 * ext, it_body, &B);
    or_ct *r = or_ct_new(cx, l, a->scale);
    moddown_exact(cx, acc0, acc1, l, r->c[0], r->c[1]);
    for (int i = 0; i <= l; i++) {
        u64 q = cx->primes[i];
        for (u64 c = 0; c < n; c++)
            r->c[1][(u64)i * n + c] = addmod(r->c[1][(u64)i * n + c], a->c[1][(u64)i * n + c], q);
    }
    free(gal); free(keys); free(pidx); free(ecoef); free(acc0); free(acc1);
    return r;
}

/* Raise a level-0 ciphertext to the top level: centred lift of each
 * coefficient of both polynomials modulo q0, reduced modulo every q_i. */
or_ct *or_mod_raise(or_ctx *cx, const or_ct *a, int level) {
    u64 n = cx->n, q0 = cx->primes[0];
    or_ct *r = or_ct_new(cx, level, a->scale);
    for (int k = 0; k < 2; k++)
        for (int i = 0; i <= level; i++) {
            u64 q = cx->primes[i];
            for (u64 c = 0; c < n; c++) {
                u64 v = a->c[k][c];
                r->c[k][(u64)i * n + c] = v <= (q0 - 1) / 2 ? v % q : submod(v % q, q0 % q, q);
            }
        }
    return r;
}

/* Multiply by the monomial X^e (e < 2N), i.e. each slot by zeta^(e*5^j). */
or_ct *or_mul_monomial(or_ctx *cx, const or_ct *a, u64 e) {
    u64 n = cx->n, two_n = 2 * n;
    or_ct *r = or_ct_new(cx, a->level, a->scale);
    for (int k = 0; k < 2; k++)
        for (int i = 0; i <= a->level; i++) {
            u64 q = cx->primes[i];
            for (u64 c = 0; c < n; c++) {
                u64 t = (c + e) % two_n, v = a->c[k][(u64)i * n + c];
                if (t < n) r->c[k][(u64)i * n + t] = v; else r->c[k][(u64)i * n + t - n] = v ? q - v : 0;
            }
        }
    return r;
}
