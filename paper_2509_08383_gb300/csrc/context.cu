// Host side of the CKKS context: prime chain, tables, device arena, keys,
// encryption and the elementary homomorphic operations.  Every operation on
// ring data is a launch of a kernel from kernels.cu on the context stream.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "context.h"

namespace he {

typedef unsigned __int128 u128;

static std::mutex g_slot_mu;
static bool g_slot_used[HE_MAX_CTX];

static int take_slot() {
    std::lock_guard<std::mutex> lk(g_slot_mu);
    for (int i = 0; i < HE_MAX_CTX; i++)
        if (!g_slot_used[i]) { g_slot_used[i] = true; return i; }
    throw Error{HE_ENOMEM, "too many live contexts (at most 8)"};
}
static void give_slot(int i) {
    std::lock_guard<std::mutex> lk(g_slot_mu);
    if (i >= 0 && i < HE_MAX_CTX) g_slot_used[i] = false;
}
void release_slot(int i) { give_slot(i); }

void check_cuda(cudaError_t e, const char *what) {
    if (e != cudaSuccess) throw Error{HE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e)};
}

// ---------------------------------------------------------------- arena
u64 mulmod_host(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
u64 powmod_host(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod_host(r, a, q);
        a = mulmod_host(a, a, q);
        e >>= 1;
    }
    return r;
}
static u64 invmod_host(u64 a, u64 q) { return powmod_host(a, q - 2, q); }
u64 shoup_host(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

static bool is_prime_host(u64 n) {
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 b : bases)
        if (n % b == 0) return n == b;
    u64 d = n - 1;
    int s = 0;
    while (!(d & 1)) { d >>= 1; s++; }
    for (u64 b : bases) {
        u64 x = powmod_host(b, d, n);
        if (x == 1 || x == n - 1) continue;
        bool composite = true;
        for (int r = 1; r < s && composite; r++) {
            x = mulmod_host(x, x, n);
            if (x == n - 1) composite = false;
        }
        if (composite) return false;
    }
    return true;
}

// Primes of b bits: q = k*2N+1 < 2^b, decreasing, one cursor per bit size.
static std::vector<u64> make_primes(int log_n, const std::vector<int> &bits) {
    u64 two_n = 2ull << log_n;
    std::map<int, u64> cursor;
    std::vector<u64> out;
    for (int b : bits) {
        if (b < 31 || b > 61) throw Error{HE_EINVAL, "prime bit sizes must lie in [31, 61]"};
        if (!cursor.count(b)) cursor[b] = ((1ull << b) - 1) / two_n;
        for (;;) {
            u64 k = cursor[b]--;
            u64 q = k * two_n + 1;
            if (q < (1ull << (b - 1))) throw Error{HE_EINVAL, "ran out of NTT-friendly primes"};
            if (is_prime_host(q)) { out.push_back(q); break; }
        }
    }
    return out;
}

static u64 find_psi(u64 q, int log_n) {
    u64 two_n = 2ull << log_n, n = 1ull << log_n;
    for (u64 x = 2;; x++) {
        u64 c = powmod_host(x, (q - 1) / two_n, q);
        if (powmod_host(c, n, q) == q - 1) return c;
    }
}

static inline u32 brv_host(u32 x, int bits) {
    u32 r = 0;
    for (int i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

u64 intd_mod_host(double x, u64 q) {
    if (std::fabs(x) < 9.2e18) {
        i64 v = (i64)x;
        i64 r = v % (i64)q;
        return r < 0 ? (u64)(r + (i64)q) : (u64)r;
    }
    int e;
    double m = std::frexp(x, &e);
    i64 mi = (i64)std::ldexp(m, 53);
    e -= 53;
    i64 r0 = mi % (i64)q;
    u64 r = r0 < 0 ? (u64)(r0 + (i64)q) : (u64)r0;
    return mulmod_host(r, powmod_host(2, (u64)e, q), q);
}

ScalarTab scalar_int(he_ctx *cx, i64 k, int n_limbs) {
    ScalarTab t;
    memset(&t, 0, sizeof(t));
    int tot = cx->nq + cx->np;
    for (int i = 0; i < tot && i < HE_MAX_PRIMES; i++) {
        u64 q = cx->primes[i];
        i64 r = k % (i64)q;
        t.v[i] = r < 0 ? (u64)(r + (i64)q) : (u64)r;
        t.s[i] = shoup_host(t.v[i], q);
    }
    (void)n_limbs;
    return t;
}
ScalarTab scalar_intd(he_ctx *cx, double K, int n_limbs) {
    ScalarTab t;
    memset(&t, 0, sizeof(t));
    int tot = cx->nq + cx->np;
    for (int i = 0; i < tot; i++) {
        u64 q = cx->primes[i];
        t.v[i] = intd_mod_host(K, q);
        t.s[i] = shoup_host(t.v[i], q);
    }
    (void)n_limbs;
    return t;
}

// ---------------------------------------------------------------- ciphertexts
void CtDel::operator()(he_ct *c) const { ct_release(c); }

he_ct *ct_alloc(he_ctx *cx, int level, double scale, int batch) {
    if (batch < 1) throw Error{HE_EINVAL, "batch size must be positive"};
    he_ct *ct = new he_ct;
    ct->ctx = cx;
    ct->level = level;
    ct->scale = scale;
    ct->cap = level + 1;
    ct->batch = batch;
    ct->bytes = (size_t)2 * batch * ct->cap * cx->N() * 8;
    try {
        ct->d = (u64 *)cx->arena.alloc(ct->bytes);
        cx->live.insert(ct);
    } catch (...) {
        delete ct;
        throw;
    }
    return ct;
}
void ct_release(he_ct *ct) {
    if (!ct) return;
    if (ct->ctx) {  // an orphan's memory went away with its context's arena
        ct->ctx->arena.release(ct->d, ct->bytes);
        ct->ctx->live.erase(ct);
    }
    delete ct;
}
Rows ct_rows(const he_ct *ct, int level) {
    int l = level < 0 ? ct->level : level;
    return make_rows(ct->d, (size_t)ct->cap * ct->ctx->N(), l + 1, l + 1, ct->ctx->nq);
}
u64 *ct_poly(const he_ct *ct, int k) { return ct->d + (size_t)k * ct->cap * ct->ctx->N(); }
Rows ct_polys(const he_ct *ct, int k, int level) {
    int l = level < 0 ? ct->level : level;
    return make_rows(ct_poly(ct, k), (size_t)2 * ct->cap * ct->ctx->N(), l + 1, l + 1, ct->ctx->nq);
}
size_t ct_member_stride(const he_ct *ct) { return (size_t)2 * ct->cap * ct->ctx->N(); }

u64 *Scratch::get(size_t words) {
    u64 *p = (u64 *)cx->arena.alloc(words * 8);
    v.emplace_back(p, words * 8);
    return p;
}
Scratch::~Scratch() {
    for (auto &pb : v) cx->arena.release(pb.first, pb.second);
}


// ---------------------------------------------------------------- setup
static void gauss_cdt(double sigma, u64 *table) {
    const int B = 19;
    double rho[B + 1], z = 0.0;
    for (int k = 0; k <= B; k++) {
        rho[k] = std::exp(-((double)k * (double)k) / (2.0 * sigma * sigma));
        z += (k == 0 ? 1.0 : 2.0) * rho[k];
    }
    double cdf = 0.0;
    for (int k = 0; k < B; k++) {
        cdf += (k == 0 ? 1.0 : 2.0) * rho[k] / z;
        table[k] = (u64)std::ldexp(cdf, 64);
    }
}

// Philox4x32-10 (host copy for the sparse secret's Fisher-Yates draws)
static void philox_host(u32 c[4], u32 k0, u32 k1) {
    const u32 M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    for (int r = 0; r < 10; r++) {
        if (r) { k0 += W0; k1 += W1; }
        u64 p0 = (u64)M0 * c[0], p1 = (u64)M1 * c[2];
        u32 n0 = (u32)(p1 >> 32) ^ c[1] ^ k0, n2 = (u32)(p0 >> 32) ^ c[3] ^ k1;
        c[0] = n0; c[1] = (u32)p1; c[2] = n2; c[3] = (u32)p0;
    }
}

static void make_secret(he_ctx *cx) {
    size_t n = cx->N();
    cx->sk_host.assign(n, 0);
    u32 k0 = (u32)cx->seed, k1 = (u32)(cx->seed >> 32);
    if (cx->h == 0) {
        for (size_t k = 0; k < n; k++) {
            u32 c[4] = {(u32)k, 0, 0, DOM_SECRET};
            philox_host(c, k0, k1);
            cx->sk_host[k] = (int8_t)((int)(((u64)c[0] * 3) >> 32) - 1);
        }
        return;
    }
    std::vector<u32> perm(n);
    for (size_t k = 0; k < n; k++) perm[k] = (u32)k;
    for (int i = 0; i < cx->h; i++) {
        u32 c[4] = {(u32)i, 0, 0, DOM_SPARSE};
        philox_host(c, k0, k1);
        u64 j = (u64)i + (((u64)c[0] * (n - (u64)i)) >> 32);
        std::swap(perm[i], perm[j]);
        cx->sk_host[perm[i]] = (c[1] & 1) ? -1 : 1;
    }
}

void ctx_init(he_ctx *cx, const he_params *p, void *arena, size_t arena_bytes) {
    if (!p || p->log_n < 10 || p->log_n > 16 || p->n_q < 2 || p->n_p < 1 || p->dnum < 1 ||
        p->n_q + p->n_p > HE_MAX_PRIMES || !p->q_bits || !p->p_bits)
        throw Error{HE_EINVAL, "invalid parameters (log_n in [10,16], n_q >= 2, n_p >= 1, n_q+n_p <= 64)"};
    cx->log_n = p->log_n;
    cx->n = 1 << p->log_n;
    cx->nq = p->n_q;
    cx->np = p->n_p;
    cx->dnum = p->dnum;
    cx->alpha = (cx->nq + cx->dnum - 1) / cx->dnum;
    cx->beta = (cx->nq + cx->alpha - 1) / cx->alpha;
    if (cx->alpha > 16 || cx->np > 16) throw Error{HE_EINVAL, "at most 16 primes per digit and 16 special primes"};
    cx->h = (int)p->secret_hw;
    cx->sigma = p->sigma > 0 ? p->sigma : 3.2;
    cx->delta = std::ldexp(1.0, 0) * std::pow(2.0, p->log_scale);
    cx->seed = p->seed;
    cx->boot = p->enable_bootstrap != 0;
    std::vector<int> bits;
    for (uint32_t i = 0; i < p->n_q; i++) bits.push_back(p->q_bits[i]);
    for (uint32_t i = 0; i < p->n_p; i++) bits.push_back(p->p_bits[i]);
    cx->primes = make_primes(cx->log_n, bits);
    const int tot = cx->nq + cx->np;
    for (u64 q : cx->primes)  // the key-switch inner product sums beta products below q 2^64
        if ((unsigned __int128)cx->beta * q >= ((unsigned __int128)1 << 64))
            throw Error{HE_EINVAL, "dnum too large for the prime sizes (beta * q must stay below 2^64)"};
    const size_t N = cx->N();

    // arena
    size_t key_bytes = (size_t)cx->beta * 2 * tot * N * 8;
    size_t ct_bytes = (size_t)2 * cx->nq * N * 8;
    if (arena) {
        cx->arena.base = (char *)arena;
        cx->arena.cap = arena_bytes;
    } else {
        size_t want = arena_bytes ? arena_bytes : (key_bytes * 48 + ct_bytes * 256 + ((size_t)64 << 20));
        size_t fr = 0, totm = 0;
        check_cuda(cudaMemGetInfo(&fr, &totm), "cudaMemGetInfo");
        if (!arena_bytes && want > fr * 7 / 10) want = fr * 7 / 10;
        check_cuda(cudaMalloc(&cx->arena.base, want), "cudaMalloc(arena)");
        cx->arena.cap = want;
        cx->arena.owned = true;
    }

    // per-prime constants
    memset(&cx->pc, 0, sizeof(cx->pc));
    for (int i = 0; i < tot; i++) {
        u64 q = cx->primes[i];
        int b = 64 - __builtin_clzll(q);
        cx->pc.m[i].q = q;
        cx->pc.m[i].b = (u32)b;
        cx->pc.m[i].mu = (u64)(((u128)1 << (2 * b + 1)) / q);
        u64 ni = invmod_host(N % q, q);
        cx->pc.n_inv[i] = ni;
        cx->pc.n_inv_shoup[i] = shoup_host(ni, q);
    }
    gauss_cdt(cx->sigma, cx->cdt);
    cx->slot = take_slot();
    t_slot = cx->slot;
    upload_constants(cx->slot, cx->pc, cx->cdt, cx->n_cdt, cx->stream);

    // twiddles: fwd[k] = psi^brv(k), inv[k] = psi^-brv(k)
    cx->d_tw = (u64 *)cx->arena.alloc((size_t)4 * tot * N * 8);
    {
        std::vector<u64> h((size_t)4 * tot * N);
        std::vector<u64> pw(N), ipw(N);
        for (int i = 0; i < tot; i++) {
            u64 q = cx->primes[i], psi = find_psi(q, cx->log_n), ipsi = invmod_host(psi, q);
            pw[0] = ipw[0] = 1;
            for (size_t k = 1; k < N; k++) {
                pw[k] = mulmod_host(pw[k - 1], psi, q);
                ipw[k] = mulmod_host(ipw[k - 1], ipsi, q);
            }
            u64 *f = &h[(size_t)2 * i * N], *v = &h[(size_t)2 * (tot + i) * N];  // (value, Shoup) pairs
            for (size_t k = 0; k < N; k++) {
                u32 b = brv_host((u32)k, cx->log_n);
                f[2 * k] = pw[b];
                f[2 * k + 1] = shoup_host(pw[b], q);
                v[2 * k] = ipw[b];
                v[2 * k + 1] = shoup_host(ipw[b], q);
            }
        }
        check_cuda(cudaMemcpy(cx->d_tw, h.data(), h.size() * 8, cudaMemcpyHostToDevice), "upload twiddles");
        cx->tw.fwd = reinterpret_cast<const ulonglong2 *>(cx->d_tw);
        cx->tw.inv = reinterpret_cast<const ulonglong2 *>(cx->d_tw + (size_t)2 * tot * N);
    }

    // scratch
    cx->ks_coef = (u64 *)cx->arena.alloc((size_t)cx->nq * N * 8);
    cx->ks_ext = (u64 *)cx->arena.alloc((size_t)cx->beta * tot * N * 8);
    cx->ks_acc = (u64 *)cx->arena.alloc((size_t)2 * tot * N * 8);
    cx->ks_conv = (u64 *)cx->arena.alloc((size_t)2 * cx->nq * N * 8);
    cx->sc_a = (u64 *)cx->arena.alloc((size_t)2 * tot * N * 8);
    cx->sc_b = (u64 *)cx->arena.alloc((size_t)2 * tot * N * 8);
    cx->d_fft = (Cplx *)cx->arena.alloc(N / 2 * sizeof(Cplx));
    cx->d_dbl = (double *)cx->arena.alloc(3 * N * sizeof(double));
    cx->d_slot_l = (int *)cx->arena.alloc(N / 2 * sizeof(int));
    {
        std::vector<int> sl(N / 2);
        u64 g = 1, two_n = 2 * N;
        for (size_t j = 0; j < N / 2; j++) {
            sl[j] = (int)((g - 1) / 4);
            g = (g * 5) % two_n;
        }
        check_cuda(cudaMemcpy(cx->d_slot_l, sl.data(), sl.size() * sizeof(int), cudaMemcpyHostToDevice),
                   "upload slot map");
    }

    // basis-conversion tables, per level
    std::vector<u64> tab;  // host staging
    struct Pending { int l, j; size_t qhinv, qhat; int n_in, n_out; };
    std::vector<Pending> pend;
    std::vector<int2> desc_all;
    std::vector<size_t> desc_off(cx->nq);
    cx->lv.resize(cx->nq);
    const int K = cx->np;
    for (int l = 0; l < cx->nq; l++) {
        LevelTabs &T = cx->lv[l];
        T.n_ext = l + 1 + K;
        T.beta = (l + 1 + cx->alpha - 1) / cx->alpha;
        desc_off[l] = desc_all.size();
        for (int j = 0; j < T.beta; j++) {
            int lo = j * cx->alpha, cnt = std::min(cx->alpha, l + 1 - lo);
            T.digit_lo.push_back(lo);
            T.digit_cnt.push_back(cnt);
            T.digit_off.push_back((int)(desc_all.size() - desc_off[l]));
            std::vector<int> targets;
            for (int t = 0; t < T.n_ext; t++)
                if (t < lo || t >= lo + cnt) targets.push_back(t);
            T.digit_nout.push_back((int)targets.size());
            for (int t : targets) {
                int pt = t <= l ? t : cx->nq + (t - l - 1);
                desc_all.push_back(make_int2(j * T.n_ext + t, pt));
            }
            Pending pd{l, j, tab.size(), 0, cnt, (int)targets.size()};
            for (int a = 0; a < cnt; a++) {
                u64 qa = cx->primes[lo + a], v = 1;
                for (int b = 0; b < cnt; b++)
                    if (b != a) v = mulmod_host(v, cx->primes[lo + b] % qa, qa);
                u64 inv = invmod_host(v, qa);
                tab.push_back(inv);
            }
            for (int a = 0; a < cnt; a++) tab.push_back(shoup_host(tab[pd.qhinv + a], cx->primes[lo + a]));
            pd.qhat = tab.size();
            std::vector<u64> qh((size_t)cnt * targets.size());
            for (int a = 0; a < cnt; a++)
                for (size_t u = 0; u < targets.size(); u++) {
                    int t = targets[u];
                    u64 pt = cx->primes[t <= l ? t : cx->nq + (t - l - 1)], v = 1;
                    for (int b = 0; b < cnt; b++)
                        if (b != a) v = mulmod_host(v, cx->primes[lo + b] % pt, pt);
                    qh[(size_t)a * targets.size() + u] = v;
                }
            for (u64 v : qh) tab.push_back(v);
            for (int a = 0; a < cnt; a++)
                for (size_t u = 0; u < targets.size(); u++) {
                    int t = targets[u];
                    u64 pt = cx->primes[t <= l ? t : cx->nq + (t - l - 1)];
                    tab.push_back((u64)(((u128)qh[(size_t)a * targets.size() + u] << 64) % pt));  // Montgomery form
                }
            pend.push_back(pd);
        }
        T.n_desc = (int)(desc_all.size() - desc_off[l]);
        if (l >= 1) {
            memset(&T.ql_inv, 0, sizeof(T.ql_inv));
            u64 ql = cx->primes[l];
            for (int i = 0; i < l; i++) {
                u64 q = cx->primes[i];
                T.ql_inv.v[i] = invmod_host(ql % q, q);
                T.ql_inv.s[i] = shoup_host(T.ql_inv.v[i], q);
            }
        }
    }
    // ModDown: P -> Q
    size_t md_off = tab.size();
    for (int a = 0; a < K; a++) {
        u64 pa = cx->primes[cx->nq + a], v = 1;
        for (int b = 0; b < K; b++)
            if (b != a) v = mulmod_host(v, cx->primes[cx->nq + b] % pa, pa);
        tab.push_back(invmod_host(v, pa));
    }
    for (int a = 0; a < K; a++) tab.push_back(shoup_host(tab[md_off + a], cx->primes[cx->nq + a]));
    size_t md_qhat = tab.size();
    for (int a = 0; a < K; a++)
        for (int i = 0; i < cx->nq; i++) {
            u64 q = cx->primes[i], v = 1;
            for (int b = 0; b < K; b++)
                if (b != a) v = mulmod_host(v, cx->primes[cx->nq + b] % q, q);
            tab.push_back(v);
        }
    for (int a = 0; a < K; a++)
        for (int i = 0; i < cx->nq; i++)  // Montgomery form
            tab.push_back((u64)(((u128)tab[md_qhat + (size_t)a * cx->nq + i] << 64) % cx->primes[i]));
    // rounding: floor(2^128 / p_a) (low, high words), and (-P mod q_i) in Montgomery form
    size_t md_inv = tab.size();
    for (int a = 0; a < K; a++) {
        const u128 m = ~(u128)0 / cx->primes[cx->nq + a];  // = floor(2^128 / p_a): p_a is odd
        tab.push_back((u64)m);
        tab.push_back((u64)(m >> 64));
    }
    size_t md_negp = tab.size();
    for (int i = 0; i < cx->nq; i++) {
        u64 q = cx->primes[i], P = 1;
        for (int b = 0; b < K; b++) P = mulmod_host(P, cx->primes[cx->nq + b] % q, q);
        tab.push_back((u64)(((u128)((q - P) % q) << 64) % q));
    }
    // exact rounding where the float64 estimate cannot decide: p_j^-1 mod p_i
    // (j < i) and the mixed-radix digits of (P-1)/2, whose residue mod p_i is
    // (p_i - 1)/2 (twice it is P - 1 = -1 mod p_i)
    size_t md_mrinv = tab.size();
    for (int i = 0; i < K; i++)
        for (int j = 0; j < K; j++) {
            u64 pi = cx->primes[cx->nq + i];
            tab.push_back(j < i ? invmod_host(cx->primes[cx->nq + j] % pi, pi) : 0);
        }
    size_t md_half = tab.size();
    for (int i = 0; i < K; i++) {
        u64 pi = cx->primes[cx->nq + i], t = (pi - 1) / 2;
        for (int j = 0; j < i; j++)
            t = mulmod_host((t + pi - tab[md_half + j] % pi) % pi, tab[md_mrinv + (size_t)i * K + j], pi);
        tab.push_back(t);
    }
    memset(&cx->p_inv, 0, sizeof(cx->p_inv));
    memset(&cx->p_mod, 0, sizeof(cx->p_mod));
    for (int i = 0; i < cx->nq; i++) {
        u64 q = cx->primes[i], P = 1;
        for (int b = 0; b < K; b++) P = mulmod_host(P, cx->primes[cx->nq + b] % q, q);
        cx->p_mod.v[i] = P;
        cx->p_mod.s[i] = shoup_host(P, q);
        cx->p_inv.v[i] = invmod_host(P, q);
        cx->p_inv.s[i] = shoup_host(cx->p_inv.v[i], q);
    }
    // product with its rescale: division by M = q_l P, inputs {q_l, p_0..p_(K-1)}
    // (the rows l .. l+K of a key-switch accumulator), outputs q_0..q_(l-1)
    struct MulRes { size_t qhinv, qhat, inv, negm, mrinv, half; };
    std::vector<MulRes> mres(cx->nq);
    const int KM = K + 1;
    const bool have_mres = KM <= 16;
    for (int l = 1; have_mres && l < cx->nq; l++) {
        std::vector<u64> m(KM);
        m[0] = cx->primes[l];
        for (int a = 0; a < K; a++) m[1 + a] = cx->primes[cx->nq + a];
        MulRes &R = mres[l];
        R.qhinv = tab.size();
        for (int a = 0; a < KM; a++) {  // (M / m_a)^-1 mod m_a
            u64 v = 1;
            for (int b = 0; b < KM; b++)
                if (b != a) v = mulmod_host(v, m[b] % m[a], m[a]);
            tab.push_back(invmod_host(v, m[a]));
        }
        for (int a = 0; a < KM; a++) tab.push_back(shoup_host(tab[R.qhinv + a], m[a]));
        R.qhat = tab.size();
        std::vector<u64> qh((size_t)KM * l);
        for (int a = 0; a < KM; a++)
            for (int t = 0; t < l; t++) {  // M / m_a mod q_t
                u64 q = cx->primes[t], v = 1;
                for (int b = 0; b < KM; b++)
                    if (b != a) v = mulmod_host(v, m[b] % q, q);
                qh[(size_t)a * l + t] = v;
            }
        for (u64 v : qh) tab.push_back(v);
        for (int a = 0; a < KM; a++)
            for (int t = 0; t < l; t++) tab.push_back((u64)(((u128)qh[(size_t)a * l + t] << 64) % cx->primes[t]));
        R.inv = tab.size();
        for (int a = 0; a < KM; a++) {
            const u128 f = ~(u128)0 / m[a];
            tab.push_back((u64)f);
            tab.push_back((u64)(f >> 64));
        }
        R.negm = tab.size();
        ScalarTab &mi = cx->lv[l].mulres_inv;
        memset(&mi, 0, sizeof(mi));
        for (int t = 0; t < l; t++) {
            u64 q = cx->primes[t], M = 1;
            for (int b = 0; b < KM; b++) M = mulmod_host(M, m[b] % q, q);
            tab.push_back((u64)(((u128)((q - M) % q) << 64) % q));
            mi.v[t] = invmod_host(M, q);
            mi.s[t] = shoup_host(mi.v[t], q);
        }
        R.mrinv = tab.size();
        for (int i = 0; i < KM; i++)
            for (int j = 0; j < KM; j++) tab.push_back(j < i ? invmod_host(m[j] % m[i], m[i]) : 0);
        R.half = tab.size();
        for (int i = 0; i < KM; i++) {  // mixed-radix digits of (M - 1)/2, whose residue mod m_i is (m_i - 1)/2
            u64 t = (m[i] - 1) / 2;
            for (int j = 0; j < i; j++)
                t = mulmod_host((t + m[i] - tab[R.half + j] % m[i]) % m[i], tab[R.mrinv + (size_t)i * KM + j], m[i]);
            tab.push_back(t);
        }
    }
    size_t desc_bytes = desc_all.size() * sizeof(int2);
    cx->d_tabs = (u64 *)cx->arena.alloc(tab.size() * 8 + desc_bytes + 16);
    check_cuda(cudaMemcpy(cx->d_tabs, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice), "upload tables");
    int2 *d_desc = (int2 *)(cx->d_tabs + tab.size());
    check_cuda(cudaMemcpy(d_desc, desc_all.data(), desc_bytes, cudaMemcpyHostToDevice), "upload descriptors");
    for (auto &pd : pend) {
        LevelTabs &T = cx->lv[pd.l];
        BConvTab bt;
        bt.qhinv = cx->d_tabs + pd.qhinv;
        bt.qhinv_sh = cx->d_tabs + pd.qhinv + pd.n_in;
        bt.qhat = cx->d_tabs + pd.qhat;
        bt.qhat_mont = cx->d_tabs + pd.qhat + (size_t)pd.n_in * pd.n_out;
        bt.n_in = pd.n_in;
        bt.n_out = pd.n_out;
        bt.stride = pd.n_out;
        T.modup.push_back(bt);
    }
    for (int l = 0; l < cx->nq; l++) cx->lv[l].desc = d_desc + desc_off[l];
    cx->moddown.qhinv = cx->d_tabs + md_off;
    cx->moddown.qhinv_sh = cx->d_tabs + md_off + K;
    cx->moddown.qhat = cx->d_tabs + md_qhat;
    cx->moddown.qhat_mont = cx->d_tabs + md_qhat + (size_t)K * cx->nq;
    cx->moddown.n_in = K;
    cx->moddown.n_out = cx->nq;
    cx->moddown.stride = cx->nq;
    cx->moddown.inv_fix = cx->d_tabs + md_inv;
    cx->moddown.negq_mont = cx->d_tabs + md_negp;
    cx->moddown.mr_inv = cx->d_tabs + md_mrinv;
    cx->moddown.mr_half = cx->d_tabs + md_half;
    for (int l = 1; have_mres && l < cx->nq; l++) {
        const MulRes &R = mres[l];
        BConvTab &bt = cx->lv[l].mulres;
        bt.qhinv = cx->d_tabs + R.qhinv;
        bt.qhinv_sh = cx->d_tabs + R.qhinv + KM;
        bt.qhat = cx->d_tabs + R.qhat;
        bt.qhat_mont = cx->d_tabs + R.qhat + (size_t)KM * l;
        bt.n_in = KM;
        bt.n_out = l;
        bt.stride = l;
        bt.inv_fix = cx->d_tabs + R.inv;
        bt.negq_mont = cx->d_tabs + R.negm;
        bt.mr_inv = cx->d_tabs + R.mrinv;
        bt.mr_half = cx->d_tabs + R.half;
    }

    // secret
    make_secret(cx);
    cx->d_sk_small = (int8_t *)cx->arena.alloc(N);
    check_cuda(cudaMemcpy(cx->d_sk_small, cx->sk_host.data(), N, cudaMemcpyHostToDevice), "upload secret");
    cx->d_sk_ntt = (u64 *)cx->arena.alloc((size_t)tot * N * 8);
    Rows sk = make_rows(cx->d_sk_ntt, 0, tot, cx->nq, cx->nq);
    load_small(sk, tot, cx->d_sk_small, cx->log_n, cx->stream);
    ntt_forward(sk, tot, cx->tw, cx->log_n, cx->stream);
    check_cuda(cudaStreamSynchronize(cx->stream), "context setup");
}

// ---------------------------------------------------------------- keys
const KeyDev *find_key(he_ctx *cx, u64 g) {
    for (auto &k : cx->keys)
        if (k.g == g) return &k;
    return nullptr;
}

// b_j = -a_j s + e_j + [i in digit j] P s'  (all primes of Q and P, NTT form)
static void build_key(he_ctx *cx, u64 g, const u64 *d_sp /*[(nq+np)][N] NTT*/) {
    const int tot = cx->nq + cx->np;
    const size_t N = cx->N();
    KeyDev k;
    k.g = g;
    k.bytes = (size_t)cx->beta * 2 * tot * N * 8;
    k.data = (u64 *)cx->arena.alloc(k.bytes);
    cudaStream_t s = cx->stream;
    for (int j = 0; j < cx->beta; j++) {
        u32 obj = ((u32)g << 8) | (u32)j;
        u64 *b = k.data + (size_t)(2 * j) * tot * N, *a = k.data + (size_t)(2 * j + 1) * tot * N;
        Rows rb = make_rows(b, 0, tot, cx->nq, cx->nq), ra = make_rows(a, 0, tot, cx->nq, cx->nq);
        Rows sk = make_rows(cx->d_sk_ntt, 0, tot, cx->nq, cx->nq);
        Rows tmp = make_rows(cx->sc_a, 0, tot, cx->nq, cx->nq);
        sample_uniform(ra, tot, cx->seed, obj, DOM_KEY_A, cx->log_n, s);
        sample_error_plus(rb, tot, cx->seed, obj, DOM_KEY_E, nullptr, cx->log_n, s);
        ntt_forward(rb, tot, cx->tw, cx->log_n, s);
        ew_mul(tmp, ra, sk, tot, cx->log_n, s);
        ew_add(rb, rb, tmp, tot, 1, cx->log_n, s);
        int lo = j * cx->alpha, cnt = std::min(cx->alpha, cx->nq - lo);
        Rows dig = make_rows(b + (size_t)lo * N, 0, cnt, cnt, cx->nq, lo);
        Rows sp = make_rows((u64 *)d_sp + (size_t)lo * N, 0, cnt, cnt, cx->nq, lo);
        Rows t2 = make_rows(cx->sc_a, 0, cnt, cnt, cx->nq, lo);
        ew_mul_scalar(t2, sp, cx->p_mod, cnt, cx->log_n, s);
        ew_add(dig, dig, t2, cnt, 0, cx->log_n, s);
    }
    // stored in Montgomery form for the key-switch inner product
    ew_mont(make_rows(k.data, (size_t)tot * N, tot, cx->nq, cx->nq), 2 * cx->beta * tot, 0, cx->log_n, s);
    check_cuda(cudaGetLastError(), "key generation");
    cx->keys.push_back(k);
}

void gen_relin_key(he_ctx *cx) {
    if (find_key(cx, 0)) return;
    const int tot = cx->nq + cx->np;
    Rows sk = make_rows(cx->d_sk_ntt, 0, tot, cx->nq, cx->nq);
    Rows s2 = make_rows(cx->sc_b, 0, tot, cx->nq, cx->nq);
    ew_mul(s2, sk, sk, tot, cx->log_n, cx->stream);
    build_key(cx, 0, cx->sc_b);
}

void gen_galois_key(he_ctx *cx, u64 g) {
    if (g == 0 || (g & 1) == 0 || g >= 2 * cx->N()) throw Error{HE_EINVAL, "Galois element must be odd and < 2N"};
    if (find_key(cx, g)) return;
    const int tot = cx->nq + cx->np;
    Rows sk = make_rows(cx->d_sk_ntt, 0, tot, cx->nq, cx->nq);
    Rows sg = make_rows(cx->sc_b, 0, tot, cx->nq, cx->nq);
    ew_automorph_ntt(sg, sk, tot, g, cx->log_n, cx->stream);
    build_key(cx, g, cx->sc_b);
}

u64 rot_galois(he_ctx *cx, i64 r) {
    u64 two_n = 2 * cx->N(), slots = cx->N() / 2;
    i64 rr = r % (i64)slots;
    if (rr < 0) rr += (i64)slots;
    return powmod_host(5, (u64)rr, two_n);
}

// ---------------------------------------------------------------- encryption
he_ct *encrypt_dev(he_ctx *cx, const double *d_pt, double scale, u32 ctr, int level) {
    if (level < 0) level = cx->nq - 1;
    if (level >= cx->nq) throw Error{HE_EINVAL, "level out of range"};
    he_ct *ct = ct_alloc(cx, level, scale);
    cudaStream_t s = cx->stream;
    Rows c0 = make_rows(ct_poly(ct, 0), 0, level + 1, level + 1, cx->nq);
    Rows c1 = make_rows(ct_poly(ct, 1), 0, level + 1, level + 1, cx->nq);
    Rows sk = make_rows(cx->d_sk_ntt, 0, level + 1, level + 1, cx->nq);
    Rows tmp = make_rows(cx->sc_a, 0, level + 1, level + 1, cx->nq);
    sample_uniform(c1, level + 1, cx->seed, ctr, DOM_UNIFORM, cx->log_n, s);
    sample_error_plus(c0, level + 1, cx->seed, ctr, DOM_ERROR, d_pt, cx->log_n, s);
    ntt_forward(c0, level + 1, cx->tw, cx->log_n, s);
    ew_mul(tmp, c1, sk, level + 1, cx->log_n, s);
    ew_add(c0, c0, tmp, level + 1, 1, cx->log_n, s);
    return ct;
}

void decrypt_dev(he_ctx *cx, const he_ct *ct, double *d_out) {
    int nl = ct->level >= 1 ? 2 : 1;
    cudaStream_t s = cx->stream;
    Rows m = make_rows(cx->sc_a, 0, nl, nl, cx->nq);
    Rows c0 = make_rows(ct_poly(ct, 0), 0, nl, nl, cx->nq);
    Rows c1 = make_rows(ct_poly(ct, 1), 0, nl, nl, cx->nq);
    Rows sk = make_rows(cx->d_sk_ntt, 0, nl, nl, cx->nq);
    decrypt_rows(m, c0, c1, sk, nl, cx->log_n, s);
    ntt_inverse(m, nl, cx->tw, cx->log_n, s);
    u64 q0 = cx->primes[0], q1 = cx->primes[1];
    u64 q0inv = invmod_host(q0 % q1, q1);
    crt_to_double(d_out, cx->sc_a, cx->sc_a + cx->N(), q0, q1, q0inv, nl == 2, cx->log_n, s);
}

void encode_dev(he_ctx *cx, const double *d_re, const double *d_im, int n_slots, double scale, double *d_out) {
    encode_slots(d_out, d_re, d_im, n_slots, scale, cx->d_slot_l, cx->d_fft, cx->log_n, cx->stream);
}
void decode_dev(he_ctx *cx, const double *d_coeff, double scale, double *d_re, double *d_im) {
    decode_coeffs(d_re, d_im, d_coeff, scale, cx->d_slot_l, cx->d_fft, cx->log_n, cx->stream);
}

// ---------------------------------------------------------------- evaluator
// Every operation acts on all `batch` members of its operands (member m's
// polynomial k at d + (2m + k) cap N): one launch per kernel for the batch.
static inline int nrows(const he_ct *ct, int l) { return 2 * ct->batch * (l + 1); }
static void same_batch(const he_ct *a, const he_ct *b) {
    if (a->batch != b->batch) throw Error{HE_EINVAL, "operands hold different numbers of ciphertexts"};
}

Ct op_copy(he_ctx *cx, const he_ct *a) {
    Ct out(ct_alloc(cx, a->level, a->scale, a->batch));
    ew_copy(ct_rows(out.get()), ct_rows(a), nrows(a, a->level), cx->log_n, cx->stream);
    return out;
}

// Operands of an addition must encrypt their messages at one scale: the sum
// of m_a s_a and m_b s_b read at s_a is m_a + m_b s_b / s_a.  Scales that the
// circuits line up agree to float64 rounding (~1e-15 relative); 1e-9 leaves
// room for that and rejects a ciphertext one rescale apart (~1e-5 and more).
static void same_scale(const he_ct *a, const he_ct *b) {
    if (!(std::fabs(a->scale - b->scale) <= 1e-9 * std::fabs(a->scale)))
        throw Error{HE_EINVAL, "operands of an addition have different scales (" + std::to_string(a->scale) +
                                   " and " + std::to_string(b->scale) + ")"};
}

Ct op_add(he_ctx *cx, const he_ct *a, const he_ct *b, bool sub) {
    same_batch(a, b);
    same_scale(a, b);
    int l = std::min(a->level, b->level);
    cx->ops_by_level[3][l] += (uint64_t)a->batch;
    Ct out(ct_alloc(cx, l, a->scale, a->batch));
    ew_add(ct_rows(out.get()), ct_rows(a, l), ct_rows(b, l), nrows(a, l), sub ? 1 : 0, cx->log_n, cx->stream);
    return out;
}

Ct op_mul_int(he_ctx *cx, const he_ct *a, i64 k) {
    Ct out(ct_alloc(cx, a->level, a->scale, a->batch));
    ew_mul_scalar(ct_rows(out.get()), ct_rows(a), scalar_int(cx, k, a->level + 1), nrows(a, a->level), cx->log_n,
                  cx->stream);
    return out;
}

Ct op_mul_intd(he_ctx *cx, const he_ct *a, double K, double scale_out) {
    Ct out(ct_alloc(cx, a->level, scale_out, a->batch));
    ew_mul_scalar(ct_rows(out.get()), ct_rows(a), scalar_intd(cx, K, a->level + 1), nrows(a, a->level), cx->log_n,
                  cx->stream);
    return out;
}

Ct op_add_intd(he_ctx *cx, const he_ct *a, double K) {
    Ct out(ct_alloc(cx, a->level, a->scale, a->batch));
    const int l = a->level, nr = a->batch * (l + 1);
    ew_add_scalar(ct_polys(out.get(), 0), ct_polys(a, 0), scalar_intd(cx, K, l + 1), nr, cx->log_n, cx->stream);
    ew_copy(ct_polys(out.get(), 1), ct_polys(a, 1), nr, cx->log_n, cx->stream);
    return out;
}

// n_pt integer plaintexts (device doubles, n_pt x N) -> NTT rows; member m of
// a batch uses plaintext m % n_pt
static Rows plain_rows(he_ctx *cx, Scratch &sc, const double *d_pt, int n_pt, int l) {
    const size_t N = cx->N();
    u64 *buf = n_pt == 1 ? cx->sc_b : sc.get((size_t)n_pt * (l + 1) * N);
    for (int i = 0; i < n_pt; i++) {
        Rows pt = make_rows(buf + (size_t)i * (l + 1) * N, 0, l + 1, l + 1, cx->nq);
        load_intd(pt, l + 1, d_pt + (size_t)i * N, cx->log_n, cx->stream);
    }
    Rows all = make_rows(buf, (size_t)(l + 1) * N, l + 1, l + 1, cx->nq);
    ntt_forward(all, n_pt * (l + 1), cx->tw, cx->log_n, cx->stream);
    return shared_rows(all, n_pt);
}

static Ct mul_plain_rows(he_ctx *cx, const he_ct *a, const Rows &pt, double scale_out) {
    int l = a->level;
    cx->ops_by_level[2][l] += (uint64_t)a->batch;
    Ct out(ct_alloc(cx, l, scale_out, a->batch));
    for (int k = 0; k < 2; k++) ew_mul(ct_polys(out.get(), k), ct_polys(a, k), pt, a->batch * (l + 1), cx->log_n, cx->stream);
    return out;
}
// c0 + pt into the output directly, c1 copied
static Ct add_plain_rows(he_ctx *cx, const he_ct *a, const Rows &pt) {
    int l = a->level;
    Ct out(ct_alloc(cx, l, a->scale, a->batch));
    ew_add(ct_polys(out.get(), 0), ct_polys(a, 0, l), pt, a->batch * (l + 1), 0, cx->log_n, cx->stream);
    ew_copy(ct_polys(out.get(), 1), ct_polys(a, 1, l), a->batch * (l + 1), cx->log_n, cx->stream);
    return out;
}
static Rows ntt_plain_rows(he_ctx *cx, const u64 *pt, int n_pt, int l) {
    return shared_rows(make_rows(const_cast<u64 *>(pt), (size_t)(l + 1) * cx->N(), l + 1, l + 1, cx->nq), n_pt);
}

Ct op_mul_plain(he_ctx *cx, const he_ct *a, const double *d_pt, double scale_out, int n_pt) {
    Scratch sc{cx, {}};
    return mul_plain_rows(cx, a, plain_rows(cx, sc, d_pt, n_pt, a->level), scale_out);
}
Ct op_add_plain(he_ctx *cx, const he_ct *a, const double *d_pt, int n_pt) {
    Scratch sc{cx, {}};
    return add_plain_rows(cx, a, plain_rows(cx, sc, d_pt, n_pt, a->level));
}
Ct op_mul_plain_ntt(he_ctx *cx, const he_ct *a, const u64 *pt, double scale_out, int n_pt) {
    return mul_plain_rows(cx, a, ntt_plain_rows(cx, pt, n_pt, a->level), scale_out);
}
Ct op_add_plain_ntt(he_ctx *cx, const he_ct *a, const u64 *pt, int n_pt) {
    return add_plain_rows(cx, a, ntt_plain_rows(cx, pt, n_pt, a->level));
}

// Encoded plaintexts of the circuits' constant vectors, kept on the device
// per (vector, encoding scale, level): the same masks and constants are
// encoded at the same scales on every call.  Only vectors that device_const
// holds qualify (their addresses stay theirs); nothing is added during a graph
// capture (capture runs nothing, so the entry would stay unwritten).  Above
// 512 entries the cache starts over, which retires the captured graphs.
const u64 *encoded_plain(he_ctx *cx, const double *re, const double *im, int n_slots, int n_pt, double E, int l) {
    for (const auto &e : cx->plain_cache)
        if (e.re == re && e.im == im && e.n_slots == n_slots && e.n_pt == n_pt && e.E == E && e.level == l) return e.d;
    if (cx->capturing || !cx->const_ptrs.count(re)) return nullptr;
    if (cx->plain_cache.size() >= 512) {
        for (auto &e : cx->plain_cache) cx->arena.release(e.d, e.bytes);
        cx->plain_cache.clear();
        cx->gen++;
    }
    const size_t N = cx->N(), bytes = (size_t)n_pt * (l + 1) * N * 8;
    u64 *d = (u64 *)cx->arena.alloc(bytes);
    double *tmp = cx->d_dbl + N;
    for (int i = 0; i < n_pt; i++) {
        encode_dev(cx, re + (size_t)i * n_slots, im ? im + (size_t)i * n_slots : nullptr, n_slots, E, tmp);
        load_intd(make_rows(d + (size_t)i * (l + 1) * N, 0, l + 1, l + 1, cx->nq), l + 1, tmp, cx->log_n, cx->stream);
    }
    ntt_forward(make_rows(d, (l + 1) * N, l + 1, l + 1, cx->nq), n_pt * (l + 1), cx->tw, cx->log_n, cx->stream);
    cx->plain_cache.push_back(he_ctx::PlainVec{re, im, n_slots, n_pt, l, E, d, bytes});
    return d;
}

// ModUp of B members (member m's limbs 0..l at d_ntt + m*d_stride, NTT form)
// into ext (member m at ext + m*beta*n_ext*N, [beta][n_ext][N] NTT form, rows
// inside each digit left unused): INTT, basis conversion per digit, NTT.
void modup(he_ctx *cx, const u64 *d_ntt, int l, u64 *ext, int B, size_t d_stride) {
    const int log_n = cx->log_n;
    const size_t N = cx->N();
    const LevelTabs &T = cx->lv[l];
    const size_t ext_w = (size_t)T.beta * T.n_ext * N;
    cudaStream_t s = cx->stream;
    Scratch sc{cx, {}};
    u64 *coef = B == 1 ? cx->ks_coef : sc.get((size_t)B * (l + 1) * N);
    if (B == 1) d_stride = 0;
    Rows crow = make_rows(coef, (size_t)(l + 1) * N, l + 1, l + 1, cx->nq);
    ntt_inverse_from(crow, make_rows((u64 *)d_ntt, d_stride, l + 1, l + 1, cx->nq), B * (l + 1), cx->tw, log_n, s);
    // every digit's conversion in one launch (at most BCONV_SET_MAX at a time)
    for (int j0 = 0; j0 < T.beta; j0 += BCONV_SET_MAX) {
        BConvSet set;
        for (int j = j0; j < std::min(T.beta, j0 + BCONV_SET_MAX); j++, set.n++) {
            int lo = T.digit_lo[j], cnt = T.digit_cnt[j];
            set.in[set.n] = make_rows(coef + (size_t)lo * N, (size_t)(l + 1) * N, cnt, cnt, cx->nq, lo);
            set.out[set.n] = desc_rows(ext, T.desc + T.digit_off[j], T.digit_nout[j], ext_w);
            set.tab[set.n] = T.modup[j];
        }
        bconv_set(set, B, log_n, s);
    }
    ntt_forward(desc_rows(ext, T.desc, T.n_desc, ext_w), B * T.n_desc, cx->tw, log_n, s);
}

// Inner product with the key, reading the digits through X -> X^galois when
// galois != 0: acc = (sum_j ext_j * b_j, sum_j ext_j * a_j) over QP, two
// polynomials of n_ext rows each (Q limbs 0..l, then the special primes), for
// B members (member m's acc at + m*2*n_ext*N).
void ks_inner(he_ctx *cx, const u64 *d_ntt, const u64 *ext, int l, const KeyDev &key, u64 galois, u64 *acc, int B,
              size_t d_stride, const u64 *lift, size_t lift_poly) {
    const LevelTabs &T = cx->lv[l];
    const size_t N = cx->N();
    cx->ks_by_level[l] += (uint64_t)B;
    KeyIP kp;
    kp.d_ntt = d_ntt;
    kp.ext = ext;
    kp.key = key.data;
    kp.acc = acc;
    kp.n_rows = T.n_ext;
    kp.l1 = l + 1;
    kp.nq = cx->nq;
    kp.np = cx->np;
    kp.alpha = cx->alpha;
    kp.beta = T.beta;
    kp.key_limbs = cx->nq + cx->np;
    kp.slot = cx->slot;
    kp.galois = galois;
    kp.batch = B;
    kp.d_stride = B == 1 ? 0 : d_stride;
    kp.ext_stride = (size_t)T.beta * T.n_ext * N;
    kp.acc_stride = (size_t)2 * T.n_ext * N;
    if (lift) {
        KeyLift lf;
        lf.d = lift;
        lf.poly_stride = lift_poly;
        lf.pmod = cx->p_mod;
        keyswitch_inner(kp, cx->log_n, cx->stream, &lf);
    } else {
        keyswitch_inner(kp, cx->log_n, cx->stream);
    }
}

// ModDown of B two-polynomial QP accumulators (destroys their special-prime
// rows): out = (acc_Q - conv(acc_P)) * P^-1 (+ add where add_mask bit k
// selects polynomial k); out and add cover the 2B polynomials.
void moddown(he_ctx *cx, u64 *acc, int l, const Rows &out, const Rows &add, int add_mask, int B) {
    const int K = cx->np, log_n = cx->log_n;
    const size_t N = cx->N();
    const LevelTabs &T = cx->lv[l];
    cudaStream_t s = cx->stream;
    Scratch sc{cx, {}};
    Rows accP = make_rows(acc + (size_t)(l + 1) * N, (size_t)T.n_ext * N, K, 0, cx->nq);
    ntt_inverse(accP, 2 * B * K, cx->tw, log_n, s);
    BConvTab md = cx->moddown;
    md.n_out = l + 1;
    u64 *cv = B == 1 ? cx->ks_conv : sc.get((size_t)2 * B * (l + 1) * N);
    Rows conv = make_rows(cv, (size_t)(l + 1) * N, l + 1, l + 1, cx->nq);
    bconv(conv, accP, md, 2 * B, log_n, s);
    ntt_forward(conv, 2 * B * (l + 1), cx->tw, log_n, s);
    Rows accQ = make_rows(acc, (size_t)T.n_ext * N, l + 1, l + 1, cx->nq);
    moddown_finish(out, accQ, conv, cx->p_inv, 2 * B * (l + 1), add, add_mask, log_n, s);
}

size_t ks_ext_words(he_ctx *cx, int l) { return (size_t)cx->lv[l].beta * cx->lv[l].n_ext * cx->N(); }
size_t ks_acc_words(he_ctx *cx, int l) { return (size_t)2 * cx->lv[l].n_ext * cx->N(); }

// Inner product with the key and ModDown: out = ModDown(acc) (+ add).
void keyswitch_ext(he_ctx *cx, const u64 *d_ntt, const u64 *ext, int l, const KeyDev &key, u64 galois,
                   const Rows &out, const Rows &add, int add_mask, int B, size_t d_stride) {
    Scratch sc{cx, {}};
    u64 *acc = B == 1 ? cx->ks_acc : sc.get((size_t)B * ks_acc_words(cx, l));
    ks_inner(cx, d_ntt, ext, l, key, galois, acc, B, d_stride);
    moddown(cx, acc, l, out, add, add_mask, B);
}

void keyswitch(he_ctx *cx, const u64 *d_ntt, int l, const KeyDev &key, const Rows &out, const Rows &add, int add_mask,
               int B, size_t d_stride) {
    Scratch sc{cx, {}};
    u64 *ext = B == 1 ? cx->ks_ext : sc.get((size_t)B * ks_ext_words(cx, l));
    modup(cx, d_ntt, l, ext, B, d_stride);
    keyswitch_ext(cx, d_ntt, ext, l, key, 0, out, add, add_mask, B, d_stride);
}

std::vector<std::vector<i64>> rotsum_stages(int steps, int log_radix) {
    if (log_radix < 1 || log_radix > 4) throw Error{HE_EINVAL, "rotate-and-sum radix must be 2, 4, 8 or 16"};
    std::vector<std::vector<i64>> st;
    for (int start = 0; start < steps; start += log_radix) {
        const int len = std::min(log_radix, steps - start);
        std::vector<i64> rots;
        for (i64 r = 1; r < ((i64)1 << len); r++) rots.push_back(r << start);
        st.push_back(rots);
    }
    return st;
}

// x + sum_r rot(x, r): the rotations share one ModUp of c1; the key inner
// products of all of them (digits read through each automorphism) and
// P (c0 + sum_r sigma_r(c0)) are summed in the QP basis; one ModDown, then
// + c1 on the second polynomial.  The same message as the rotations and
// additions one by one, with key-switching noise of the same size (the
// automorphism acts after the approximate basis conversion instead of before
// it, and one ModDown rounds the summed products).
Ct op_rotsum_stage(he_ctx *cx, const he_ct *a, const std::vector<i64> &rots) {
    const int n_keys = (int)rots.size();
    if (n_keys < 1 || n_keys > ROTSUM_MAX_KEYS) throw Error{HE_EINVAL, "a hoisted stage takes 1..15 rotations"};
    const int l = a->level, B = a->batch;
    const LevelTabs &T = cx->lv[l];
    const size_t N = cx->N(), ms = ct_member_stride(a);
    KeyIPMulti kp;
    for (int r = 0; r < n_keys; r++) {
        const u64 g = rot_galois(cx, rots[r]);
        const KeyDev *key = find_key(cx, g);
        if (!key) throw Error{HE_ENOKEY, "rotation key for " + std::to_string(rots[r]) + " not generated"};
        kp.keys[r] = key->data;
        kp.gal[r] = g;
    }
    Scratch sc{cx, {}};
    u64 *ext = B == 1 ? cx->ks_ext : sc.get((size_t)B * ks_ext_words(cx, l));
    u64 *acc = B == 1 ? cx->ks_acc : sc.get((size_t)B * ks_acc_words(cx, l));
    modup(cx, ct_poly(a, 1), l, ext, B, ms);
    kp.d_ntt = ct_poly(a, 1);
    kp.ext = ext;
    kp.c0 = ct_poly(a, 0);
    kp.acc = acc;
    kp.n_rows = T.n_ext;
    kp.l1 = l + 1;
    kp.nq = cx->nq;
    kp.np = cx->np;
    kp.alpha = cx->alpha;
    kp.beta = T.beta;
    kp.key_limbs = cx->nq + cx->np;
    kp.slot = cx->slot;
    kp.n_keys = n_keys;
    kp.pmod = cx->p_mod;
    kp.batch = B;
    kp.d_stride = kp.c0_stride = B == 1 ? 0 : ms;
    kp.ext_stride = ks_ext_words(cx, l);
    kp.acc_stride = ks_acc_words(cx, l);
    keyswitch_inner_multi(kp, cx->log_n, cx->stream);
    cx->ks_by_level[l] += (uint64_t)n_keys * (uint64_t)B;
    Ct out(ct_alloc(cx, l, a->scale, B));
    moddown(cx, acc, l, ct_rows(out.get()), ct_rows(a), 2, B);
    return out;
}

Ct op_rotsum(he_ctx *cx, const he_ct *a, int steps) {
    Ct cur;
    for (const auto &rots : rotsum_stages(steps, cx->rotsum_log_radix))
        cur = op_rotsum_stage(cx, cur ? cur.get() : a, rots);
    return cur ? std::move(cur) : op_copy(cx, a);
}

Ct op_mul(he_ctx *cx, const he_ct *a, const he_ct *b) {
    same_batch(a, b);
    const KeyDev *rk = find_key(cx, 0);
    if (!rk) throw Error{HE_ENOKEY, "relinearisation key not generated"};
    const int l = std::min(a->level, b->level), B = a->batch;
    const size_t N = cx->N();
    cx->ops_by_level[1][l] += (uint64_t)B;
    Ct out(ct_alloc(cx, l, a->scale * b->scale, B));
    Scratch sc{cx, {}};
    u64 *d2 = B == 1 ? cx->sc_a : sc.get((size_t)B * (l + 1) * N);
    Rows r2 = make_rows(d2, (size_t)(l + 1) * N, l + 1, l + 1, cx->nq);
    ew_tensor(ct_polys(out.get(), 0), ct_polys(out.get(), 1), r2, ct_polys(a, 0, l), ct_polys(a, 1, l),
              ct_polys(b, 0, l), ct_polys(b, 1, l), B * (l + 1), cx->log_n, cx->stream);
    Rows o = ct_rows(out.get());
    keyswitch(cx, d2, l, *rk, o, o, 3, B, (size_t)(l + 1) * N);
    return out;
}

// Product, relinearisation and rescale with one rounding.  The tensor
// product (d0, d1, d2) at level l; the key products acc of d2 (ModUp, inner
// product) over Q_l u P; P d_k added on the Q rows; then the rounded
// division by M = q_l P: INTT of the rows of q_l and the special primes,
// basis conversion from them (exact rounding) to q_0..q_(l-1), NTT, and
// out_i = (acc_i - conv_i) M^-1.  The same message, level and scale as
// rescale(mul(a, b)), without the rescale's own INTT, lift and NTT.
Ct op_mul_rescale(he_ctx *cx, const he_ct *a, const he_ct *b) {
    same_batch(a, b);
    const int l = std::min(a->level, b->level), B = a->batch;
    if (l < 1) throw Error{HE_ELEVEL, "cannot rescale a level-0 product"};
    const LevelTabs &T = cx->lv[l];
    if (T.mulres.n_in == 0) return op_rescale(cx, op_mul(cx, a, b).get());
    const KeyDev *rk = find_key(cx, 0);
    if (!rk) throw Error{HE_ENOKEY, "relinearisation key not generated"};
    const size_t N = cx->N(), ne = (size_t)T.n_ext, qp_w = 2 * ne * N;
    const int K = cx->np, log_n = cx->log_n;
    cudaStream_t s = cx->stream;
    cx->ops_by_level[1][l] += (uint64_t)B;
    cx->ops_by_level[0][l] += (uint64_t)B;
    Scratch sc{cx, {}};
    Ct t(ct_alloc(cx, l, a->scale * b->scale, B));
    u64 *d2 = B == 1 ? cx->sc_a : sc.get((size_t)B * (l + 1) * N);
    Rows r2 = make_rows(d2, (size_t)(l + 1) * N, l + 1, l + 1, cx->nq);
    ew_tensor(ct_polys(t.get(), 0), ct_polys(t.get(), 1), r2, ct_polys(a, 0, l), ct_polys(a, 1, l), ct_polys(b, 0, l),
              ct_polys(b, 1, l), B * (l + 1), log_n, s);
    u64 *ext = B == 1 ? cx->ks_ext : sc.get((size_t)B * ks_ext_words(cx, l));
    u64 *acc = B == 1 ? cx->ks_acc : sc.get((size_t)B * ks_acc_words(cx, l));
    modup(cx, d2, l, ext, B, (size_t)(l + 1) * N);
    // + P d_k on the Q rows of output polynomial k: inside the inner product
    // for one member, as its own pass for a batch (where the extra registers
    // would halve the batched kernel's occupancy)
    const size_t ts = ct_member_stride(t.get());
    if (B == 1) {
        ks_inner(cx, d2, ext, l, *rk, 0, acc, B, (size_t)(l + 1) * N, ct_poly(t.get(), 0),
                 (size_t)(ct_poly(t.get(), 1) - ct_poly(t.get(), 0)));
    } else {
        ks_inner(cx, d2, ext, l, *rk, 0, acc, B, (size_t)(l + 1) * N);
        for (int k = 0; k < 2; k++)
            ew_qp_lift(acc + (size_t)k * ne * N, ct_poly(t.get(), k), l + 1, (int)ne, 0, 1, cx->p_mod, cx->slot, log_n,
                       s, B, qp_w, ts);
    }
    // rows l .. l+K of each polynomial: q_l, then the special primes
    Rows div = make_rows(acc + (size_t)l * N, ne * N, K + 1, 1, cx->nq, l);
    ntt_inverse(div, 2 * B * (K + 1), cx->tw, log_n, s);
    u64 *cv = B == 1 ? cx->ks_conv : sc.get((size_t)2 * B * l * N);
    Rows conv = make_rows(cv, (size_t)l * N, l, l, cx->nq);
    bconv(conv, div, T.mulres, 2 * B, log_n, s);
    ntt_forward(conv, 2 * B * l, cx->tw, log_n, s);
    Ct out(ct_alloc(cx, l - 1, a->scale * b->scale / (double)cx->primes[l], B));
    Rows accQ = make_rows(acc, ne * N, l, l, cx->nq);
    moddown_finish(ct_rows(out.get()), accQ, conv, T.mulres_inv, 2 * B * l, accQ, 0, log_n, s);
    return out;
}

// rescale of K a (kmul: K mod q_i; null: K = 1) whose scale is `scale`
static Ct rescale_times(he_ctx *cx, const he_ct *a, const ScalarTab *kmul, double scale) {
    int l = a->level;
    if (l < 1) throw Error{HE_ELEVEL, "cannot rescale a level-0 ciphertext"};
    cx->ops_by_level[0][l] += (uint64_t)a->batch;
    const size_t N = cx->N();
    const int np2 = 2 * a->batch;
    cudaStream_t s = cx->stream;
    u64 ql = cx->primes[l];
    Ct out(ct_alloc(cx, l - 1, scale / (double)ql, a->batch));
    Scratch sc{cx, {}};
    u64 *lastb = a->batch == 1 ? cx->sc_a : sc.get((size_t)np2 * N);
    u64 *liftb = a->batch == 1 ? cx->sc_b : sc.get((size_t)np2 * l * N);
    // last limbs of every polynomial -> coefficient form
    Rows last = make_rows(lastb, N, 1, 1, cx->nq, l);
    Rows src = make_rows(ct_poly(a, 0) + (size_t)l * N, (size_t)a->cap * N, 1, 1, cx->nq, l);
    ntt_inverse_from(last, src, np2, cx->tw, cx->log_n, s);
    Rows lift = make_rows(liftb, (size_t)l * N, l, l, cx->nq);
    rescale_lift(lift, lastb, np2, ql, l, cx->log_n, s, kmul);
    ntt_forward(lift, np2 * l, cx->tw, cx->log_n, s);
    rescale_finish(ct_rows(out.get()), ct_rows(a, l - 1), lift, cx->lv[l].ql_inv, np2 * l, cx->log_n, s, kmul);
    return out;
}
Ct op_rescale(he_ctx *cx, const he_ct *a) { return rescale_times(cx, a, nullptr, a->scale); }
Ct op_mul_intd_rescale(he_ctx *cx, const he_ct *a, double K, double scale_mid) {
    const ScalarTab k = scalar_intd(cx, K, a->level + 1);
    return rescale_times(cx, a, &k, scale_mid);
}

Ct op_drop(he_ctx *cx, const he_ct *a, int level) {
    if (level > a->level || level < 0) throw Error{HE_EINVAL, "drop to an invalid level"};
    Ct out(ct_alloc(cx, level, a->scale, a->batch));
    ew_copy(ct_rows(out.get()), ct_rows(a, level), nrows(a, level), cx->log_n, cx->stream);
    return out;
}

Ct op_automorph(he_ctx *cx, const he_ct *a, u64 g) {
    const KeyDev *k = find_key(cx, g);
    if (!k) throw Error{HE_ENOKEY, "Galois key not generated for element " + std::to_string(g)};
    const int l = a->level, B = a->batch;
    const size_t N = cx->N();
    Ct out(ct_alloc(cx, l, a->scale, B));
    // sigma(c0) -> out polynomial 0 (added in place by the ModDown), sigma(c1) -> scratch
    Scratch sc{cx, {}};
    u64 *sb = B == 1 ? cx->sc_b : sc.get((size_t)B * (l + 1) * N);
    ew_automorph_ntt(ct_polys(out.get(), 0), ct_polys(a, 0), B * (l + 1), g, cx->log_n, cx->stream);
    ew_automorph_ntt(make_rows(sb, (size_t)(l + 1) * N, l + 1, l + 1, cx->nq), ct_polys(a, 1), B * (l + 1), g,
                     cx->log_n, cx->stream);
    Rows o = ct_rows(out.get());
    keyswitch(cx, sb, l, *k, o, o, 1, B, (size_t)(l + 1) * N);
    return out;
}

Ct op_mul_monomial(he_ctx *cx, const he_ct *a, u64 e) {
    Ct out(ct_alloc(cx, a->level, a->scale, a->batch));
    ew_monomial(ct_rows(out.get()), ct_rows(a), nrows(a, a->level), e % (2 * cx->N()), cx->tw, cx->log_n, cx->stream);
    return out;
}

Ct op_mod_raise(he_ctx *cx, const he_ct *a, int level) {
    if (a->level != 0) throw Error{HE_EINVAL, "mod raise expects a level-0 ciphertext"};
    const size_t N = cx->N();
    const int np2 = 2 * a->batch;
    cudaStream_t s = cx->stream;
    Scratch sc{cx, {}};
    u64 *lastb = a->batch == 1 ? cx->sc_a : sc.get((size_t)np2 * N);
    Rows last = make_rows(lastb, N, 1, 1, cx->nq, 0);
    ew_copy(last, make_rows(ct_poly(a, 0), (size_t)a->cap * N, 1, 1, cx->nq, 0), np2, cx->log_n, s);
    ntt_inverse(last, np2, cx->tw, cx->log_n, s);
    Ct out(ct_alloc(cx, level, a->scale, a->batch));
    Rows o = ct_rows(out.get());
    modraise_lift(o, lastb, cx->primes[0], np2 * (level + 1), cx->log_n, s);
    ntt_forward(o, np2 * (level + 1), cx->tw, cx->log_n, s);
    return out;
}

// ---- batches
Ct op_batch_pack(he_ctx *cx, const he_ct *const *cts, int n) {
    if (n < 1) throw Error{HE_EINVAL, "empty batch"};
    int l = cts[0]->level;
    for (int i = 0; i < n; i++) {
        if (cts[i]->ctx != cx) throw Error{HE_EINVAL, "ciphertext from another context"};
        if (std::fabs(cts[i]->scale - cts[0]->scale) > 1e-9 * cts[0]->scale)
            throw Error{HE_EINVAL, "batch members must share one scale"};
        l = std::min(l, cts[i]->level);
    }
    int total = 0;
    for (int i = 0; i < n; i++) total += cts[i]->batch;
    Ct out(ct_alloc(cx, l, cts[0]->scale, total));
    const size_t ms = ct_member_stride(out.get());
    int m = 0;
    for (int i = 0; i < n; i++) {
        Rows dst = make_rows(out->d + (size_t)m * ms, (size_t)out->cap * cx->N(), l + 1, l + 1, cx->nq);
        ew_copy(dst, ct_rows(cts[i], l), nrows(cts[i], l), cx->log_n, cx->stream);
        m += cts[i]->batch;
    }
    return out;
}

Ct op_batch_member(he_ctx *cx, const he_ct *a, int i, int count) {
    if (i < 0 || count < 1 || i + count > a->batch) throw Error{HE_EINVAL, "batch member out of range"};
    Ct out(ct_alloc(cx, a->level, a->scale, count));
    Rows src = make_rows(a->d + (size_t)i * ct_member_stride(a), (size_t)a->cap * cx->N(), a->level + 1,
                         a->level + 1, cx->nq);
    ew_copy(ct_rows(out.get()), src, nrows(out.get(), a->level), cx->log_n, cx->stream);
    return out;
}

// groups of g consecutive members: summed (sum) into one member each, or each
// member repeated g times (broadcast)
Ct op_group(he_ctx *cx, const he_ct *a, int g, bool sum) {
    if (g < 1 || (sum && a->batch % g)) throw Error{HE_EINVAL, "batch is not a whole number of groups"};
    const int l = a->level, nb = sum ? a->batch / g : a->batch * g;
    Ct out(ct_alloc(cx, l, a->scale, nb));
    const size_t N = cx->N();
    ew_group(out->d, a->d, nb, g, sum ? 1 : 0, l + 1, ct_member_stride(out.get()), ct_member_stride(a),
             (size_t)a->cap * N, (size_t)out->cap * N, cx->slot, cx->log_n, cx->stream);
    return out;
}

}  // namespace he

he_ctx::~he_ctx() {
    he::graphs_release(this);
    for (he_ct *c : live) c->ctx = nullptr;
    he::release_slot(slot);
    for (auto &k : keys) arena.release(k.data, k.bytes);
    if (arena.owned && arena.base) cudaFree(arena.base);
}
