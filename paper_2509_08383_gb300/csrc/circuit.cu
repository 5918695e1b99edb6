// CutMax_HE (Alg. 2) and nucleus one-shot sampling (Alg. 3) on the GPU
// evaluator.
//
// Scale rule: every ciphertext carries its exact scale.  A multiplication by
// a real constant c at level l towards `target` encodes E = (target*q_l)/scale,
// multiplies by K = rint(c*E), sets the scale to scale*E and rescales
// (scale/q_l).  Adding a constant c adds rint(c*scale).  Products multiply
// scales, rescale divides by q_l.
//
// Iteration t of Alg. 2 (Y at level l):
//   S = rotsum(Y); D = n*Y - S (= n(Y - mu)); E = rescale(D*D)
//   V = rotsum(E) [- m * rescale(S*S) when m slots are zero padding] = n^3 sigma^2
//   h = 1/(2 sqrt(kappa V)) by k coupled Goldschmidt iterations (2 levels each)
//   D' = D * 2 sqrt(kappa n)/c (times the slot mask when padded)
//   u = D' h + 1 (+ mask when padded) = (Y - mu)/(c sigma) + 1
//   Y = u^p by square-and-multiply
// Final: S = rotsum(Y); a = 1 - kappa_f S; F = prod_{i<=d}(1 + a^(2^i));
//   Z = (kappa_f Y) F   (Goldschmidt inverse, App. B.1)
#include <algorithm>
#include <cmath>
#include <string_view>

#include "context.h"

namespace he {

// Device copy of a constant slot vector, uploaded on first use and kept for
// the context's life (keyed by content): the circuits use the same masks and
// constants on every call, and a CUDA graph capture cannot upload from
// pageable host memory.  Above 4096 vectors the cache starts over, which
// retires the captured graphs that point into it.
const double *device_const(he_ctx *cx, const std::vector<double> &v) {
    const size_t bytes = v.size() * sizeof(double);
    const uint64_t h = std::hash<std::string_view>{}(std::string_view(reinterpret_cast<const char *>(v.data()), bytes));
    auto r = cx->const_cache.equal_range(h);
    for (auto it = r.first; it != r.second; ++it)
        if (it->second.host == v) return it->second.d;
    if (cx->capturing) throw Error{HE_EINVAL, "a constant vector first seen during a graph capture"};
    if (cx->const_cache.size() >= 4096) {  // the encodings keyed by these vectors go too
        for (auto &e : cx->const_cache) cx->arena.release(e.second.d, e.second.host.size() * sizeof(double));
        for (auto &e : cx->plain_cache) cx->arena.release(e.d, e.bytes);
        cx->const_cache.clear();
        cx->const_ptrs.clear();
        cx->plain_cache.clear();
        cx->gen++;
    }
    double *d = (double *)cx->arena.alloc(bytes);
    // a pageable source is staged before the call returns
    check_cuda(cudaMemcpyAsync(d, v.data(), bytes, cudaMemcpyHostToDevice, cx->stream), "constant vector");
    cx->const_cache.emplace(h, he_ctx::ConstVec{d, v});
    cx->const_ptrs.insert(d);
    return d;
}

namespace {

struct HE {
    he_ctx *cx;
    double delta;

    u64 q(int level) const { return cx->primes[level]; }

    Ct mcr(const he_ct *ct, double c, double target = -1) {
        if (target < 0) target = delta;
        double E = (target * (double)q(ct->level)) / ct->scale;
        double K = std::rint(c * E);
        return op_mul_intd_rescale(cx, ct, K, ct->scale * E);
    }
    // c * ct with the integer multiplier K = rint(c E) carrying at least
    // min_bits bits: a tiny c against a large scale (the range scale kappa of
    // a variance sum of tens of thousands of terms) is spread over as many
    // rescales r <= 3 as that takes, E = target q_l ... q_(l-r+1) / scale.
    Ct mcr_bits(const he_ct *ct, double c, double target, int min_bits) {
        if (target < 0) target = delta;
        int r = 1;
        double E = (target * (double)q(ct->level)) / ct->scale;
        while (std::fabs(c * E) < std::ldexp(1.0, min_bits) && r < 3 && ct->level - r >= 1) {
            E *= (double)q(ct->level - r);
            r++;
        }
        double K = std::rint(c * E);
        Ct t = op_mul_intd_rescale(cx, ct, K, ct->scale * E);
        for (int i = 1; i < r; i++) t = op_rescale(cx, t.get());
        return t;
    }
    Ct add_const(const he_ct *ct, double c) { return op_add_intd(cx, ct, std::rint(c * ct->scale)); }
    Ct neg(const he_ct *ct) { return op_mul_int(cx, ct, -1); }
    // learned inverse square root: (A x^2 + B x + C) / 2, two levels
    Ct learned_half(const he_ct *x, const double *abc) {
        Ct x2 = mul_rescale(x, x);
        Ct t2 = mcr_bits(x2.get(), abc[0] / 2.0, -1, 24), t1 = mcr_bits(x, abc[1] / 2.0, -1, 24);
        return add_const(op_add(cx, t2.get(), t1.get(), false).get(), abc[2] / 2.0);
    }
    // product, relinearisation and rescale in one rounded division by q_l P
    Ct mul_rescale(const he_ct *a, const he_ct *b) { return op_mul_rescale(cx, a, b); }
    // n_pt device slot vectors (n_pt x n_slots doubles; member m of a batch
    // uses vector m % n_pt) encoded at scale E, multiply, rescale
    Ct mul_plain_rescale(const he_ct *ct, const double *d_vec, int n_slots, double target = -1, int n_pt = 1) {
        if (target < 0) target = delta;
        double E = (target * (double)q(ct->level)) / ct->scale;
        if (const u64 *pt = encoded_plain(cx, d_vec, nullptr, n_slots, n_pt, E, ct->level))
            return op_rescale(cx, op_mul_plain_ntt(cx, ct, pt, ct->scale * E, n_pt).get());
        Scratch sc{cx, {}};
        double *d_pt = n_pt == 1 ? cx->d_dbl + cx->N() : (double *)sc.get((size_t)n_pt * cx->N());
        for (int i = 0; i < n_pt; i++) encode_dev(cx, d_vec + (size_t)i * n_slots, nullptr, n_slots, E, d_pt + i * cx->N());
        Ct t = op_mul_plain(cx, ct, d_pt, ct->scale * E, n_pt);
        return op_rescale(cx, t.get());
    }
    // ct + (re + i im) in every slot
    Ct add_complex_const(const he_ct *ct, double re, double im) {
        const int slots = cx->n / 2;
        std::vector<double> v(2 * (size_t)slots);
        for (int i = 0; i < slots; i++) v[i] = re, v[slots + i] = im;
        const double *d_v = device_const(cx, v);
        if (const u64 *pt = encoded_plain(cx, d_v, d_v + slots, slots, 1, ct->scale, ct->level))
            return op_add_plain_ntt(cx, ct, pt);
        double *d_pt = cx->d_dbl + cx->N();
        encode_dev(cx, d_v, d_v + slots, slots, ct->scale, d_pt);
        return op_add_plain(cx, ct, d_pt);
    }
    Ct add_plain_vec(const he_ct *ct, const double *d_vec, int n_slots, int n_pt = 1) {
        if (const u64 *pt = encoded_plain(cx, d_vec, nullptr, n_slots, n_pt, ct->scale, ct->level))
            return op_add_plain_ntt(cx, ct, pt, n_pt);
        Scratch sc{cx, {}};
        double *d_pt = n_pt == 1 ? cx->d_dbl + cx->N() : (double *)sc.get((size_t)n_pt * cx->N());
        for (int i = 0; i < n_pt; i++)
            encode_dev(cx, d_vec + (size_t)i * n_slots, nullptr, n_slots, ct->scale, d_pt + i * cx->N());
        return op_add_plain(cx, ct, d_pt, n_pt);
    }
    // rotate-and-sum in hoisted stages of the context's radix (op_rotsum)
    Ct rotsum(const he_ct *ct, int steps) { return op_rotsum(cx, ct, steps); }
    Ct power(const he_ct *u, int p) {
        Ct sq = op_copy(cx, u), acc;
        int pp = p;
        for (;;) {
            if (pp & 1) acc = acc ? mul_rescale(acc.get(), sq.get()) : op_copy(cx, sq.get());
            pp >>= 1;
            if (!pp) break;
            sq = mul_rescale(sq.get(), sq.get());
        }
        return acc;
    }
};

// step i multiplies by a = alpha[i-1] - g h (3/2: Newton's step; larger
// values over-relax the steps where x y^2 is still small)
Ct invsqrt_goldschmidt(HE &he, const he_ct *V, double kappa, double y0, int k, const double *alpha) {
    Ct a = he.add_const(he.mcr(V, -kappa * y0 * y0 / 2.0).get(), alpha[0]);
    Ct h = he.mcr(a.get(), y0 / 2.0);
    Ct g;
    if (k >= 2) g = he.mul_rescale(he.mcr(V, kappa * y0).get(), a.get());
    for (int i = 2; i <= k; i++) {
        a = he.add_const(he.neg(he.mul_rescale(g.get(), h.get()).get()).get(), alpha[i - 1]);
        if (i < k) g = he.mul_rescale(g.get(), a.get());
        h = he.mul_rescale(h.get(), a.get());
    }
    return h;
}

Ct inverse_goldschmidt(HE &he, const he_ct *S, double kappa_f, int d) {
    Ct a = he.add_const(he.mcr(S, -kappa_f).get(), 1.0);
    Ct F = he.add_const(a.get(), 1.0);
    Ct sq = op_copy(he.cx, a.get());
    for (int i = 0; i < d; i++) {
        sq = he.mul_rescale(sq.get(), sq.get());
        F = he.mul_rescale(F.get(), he.add_const(sq.get(), 1.0).get());
    }
    return F;
}

int rotsum_steps(const Plan &pl, int slots) {
    int m = pl.packing == 0 ? pl.n : slots;
    int s = 0;
    while ((1 << s) < m) s++;
    return s;
}

}  // namespace

int Plan::pad(int slots) const { return packing == 0 ? 0 : cps * slots - n; }

Plan plan_from(const he_cutmax_plan *p) {
    if (!p || p->T < 1 || p->T > 64 || !p->power || !p->c || !p->k || !p->kappa || !p->y0 || p->n < 2)
        throw Error{HE_EINVAL, "invalid CutMax plan"};
    Plan pl;
    pl.n = (int)p->n;
    pl.packing = (int)p->packing;
    pl.T = (int)p->T;
    for (uint32_t t = 0; t < p->T; t++) {
        if (p->power[t] < 1 || (p->k[t] < 1 && !p->learned) || !(p->c[t] > 0) || !(p->kappa[t] > 0) ||
            !(p->y0[t] > 0))
            throw Error{HE_ERANGE, "plan constants out of range"};
        if (p->k[t] == 0)
            for (int i = 0; i < 3; i++)
                if (!std::isfinite(p->learned[3 * t + i])) throw Error{HE_ERANGE, "learned coefficients must be finite"};
        pl.p.push_back((int)p->power[t]);
        pl.c.push_back(p->c[t]);
        pl.k.push_back((int)p->k[t]);
        pl.kappa.push_back(p->kappa[t]);
        pl.y0.push_back(p->y0[t]);
        double nm = p->norm ? p->norm[t] : 1.0;
        if (!(nm > 0)) throw Error{HE_ERANGE, "plan normalisers must be positive"};
        pl.norm.push_back(nm);
    }
    pl.bootstrap = p->bootstrap != 0;
    pl.cps = p->cts ? (int)p->cts : 1;
    pl.shared = p->shared != 0;
    if (p->learned) pl.lq.assign(p->learned, p->learned + 3 * p->T);
    for (uint32_t t = 0; t < p->T; t++) {
        pl.relax_at.push_back((int)pl.relax.size());
        for (uint32_t i = 0; i < p->k[t]; i++) {
            const double a = p->relax ? p->relax[pl.relax.size()] : 1.5;
            if (!(a >= 1.0 && a <= 4.0)) throw Error{HE_ERANGE, "relaxation constants must lie in [1, 4]"};
            pl.relax.push_back(a);
        }
    }
    if (pl.cps > 64) throw Error{HE_EINVAL, "more than 64 ciphertexts per stream"};
    pl.d = (int)p->d;
    pl.kappa_f = p->kappa_f;
    if (!(pl.kappa_f > 0)) throw Error{HE_ERANGE, "kappa_f must be positive"};
    return pl;
}

static int power_depth(int p) {
    int d = 0;
    while ((1 << d) < p) d++;
    return d;
}

void plan_keys(he_ctx *cx, const Plan &pl, std::vector<u64> &galois) {
    // the rotate-and-sum stages; with bootstrapping also those of the constant
    // bootstrap's trace (every slot) and the rotation by N/4
    std::vector<int> all_steps = {rotsum_steps(pl, cx->n / 2)};
    if (pl.bootstrap) all_steps.push_back(cx->log_n - 1);
    for (int steps : all_steps)
        for (const auto &rots : rotsum_stages(steps, cx->rotsum_log_radix))
            for (i64 r : rots) galois.push_back(rot_galois(cx, r));
    if (pl.bootstrap) galois.push_back(rot_galois(cx, cx->n / 4));  // packed Goldschmidt pair
    std::sort(galois.begin(), galois.end());
    galois.erase(std::unique(galois.begin(), galois.end()), galois.end());
}

static Ct cutmax_boot(he_ctx *cx, const he_ct *in, const Plan &pl);
int boot_out_level(he_ctx *cx);
Ct bootstrap_stage(he_ctx *cx, const he_ct *in, int stage);

// Streams of pl.cps ciphertexts each, stream-major in the batch.  Checks the
// shape and builds the per-position slot masks (1 on real entries) that the
// zero-padded packing needs.
struct StreamShape {
    int cps, S, slots, steps, m;
    std::vector<double> mask;  // [cps][slots]
};
static StreamShape stream_shape(he_ctx *cx, const he_ct *in, const Plan &pl) {
    StreamShape sh;
    sh.slots = cx->n / 2;
    sh.cps = pl.cps;
    if (in->batch % sh.cps) throw Error{HE_EINVAL, "batch is not a whole number of streams"};
    sh.S = in->batch / sh.cps;
    if (pl.n > sh.cps * sh.slots) throw Error{HE_EINVAL, "plan n exceeds the slots of its ciphertexts"};
    if (sh.cps > 1 && pl.n <= (sh.cps - 1) * sh.slots) throw Error{HE_EINVAL, "plan uses more ciphertexts than n needs"};
    if (pl.packing == 0 && (sh.cps != 1 || sh.slots % pl.n != 0 || (pl.n & (pl.n - 1))))
        throw Error{HE_EINVAL, "replicated packing needs one ciphertext and n a power of two dividing N/2"};
    sh.steps = rotsum_steps(pl, sh.slots);
    sh.m = pl.pad(sh.slots);
    if (sh.m) {
        sh.mask.assign((size_t)sh.cps * sh.slots, 0.0);
        for (int i = 0; i < pl.n; i++) sh.mask[i] = 1.0;
    }
    return sh;
}
// per-stream sum of a batch and the broadcast of a per-stream batch back to
// the streams' ciphertexts.  With one ciphertext per stream both are the
// identity: the view then points at the input itself (no copy), and an owned
// ciphertext is passed through.
struct CtView {
    Ct own;
    const he_ct *p;
};
static CtView stream_group_view(he_ctx *cx, const he_ct *a, int cps, bool sum) {
    if (cps == 1) return {nullptr, a};
    Ct g = op_group(cx, a, cps, sum);
    const he_ct *p = g.get();
    return {std::move(g), p};
}
static CtView stream_sum(he_ctx *cx, const he_ct *a, int cps) { return stream_group_view(cx, a, cps, true); }
static CtView stream_bcast(he_ctx *cx, const he_ct *a, int cps) { return stream_group_view(cx, a, cps, false); }
static Ct stream_bcast(he_ctx *cx, Ct a, int cps) { return cps > 1 ? op_group(cx, a.get(), cps, false) : std::move(a); }
// device copy of `vals` scaled by c (see device_const)
static const double *upload_scaled(he_ctx *cx, Scratch &, const std::vector<double> &vals, double c) {
    std::vector<double> v(vals);
    for (double &x : v) x *= c;
    return device_const(cx, v);
}

Ct cutmax_ct(he_ctx *cx, const he_ct *in, const Plan &pl) {
    if (pl.bootstrap) return cutmax_boot(cx, in, pl);
    StreamShape sh = stream_shape(cx, in, pl);
    int depth = pl.d + 3;
    for (int t = 0; t < pl.T; t++) depth += 2 + (pl.k[t] ? 2 * pl.k[t] : 5) + power_depth(pl.p[t]);
    if (depth > in->level) throw Error{HE_ELEVEL, "circuit depth " + std::to_string(depth) + " exceeds level " +
                                                   std::to_string(in->level)};
    HE he{cx, cx->delta};
    const int cps = sh.cps, m = sh.m;
    Scratch sc{cx, {}};
    const double *d_mask = m ? upload_scaled(cx, sc, sh.mask, 1.0) : nullptr;
    Ct Y = op_copy(cx, in);
    for (int t = 0; t < pl.T; t++) {
        Ct S = he.rotsum(stream_sum(cx, Y.get(), cps).p, sh.steps);
        Ct D = op_add(cx, op_mul_int(cx, Y.get(), pl.n).get(), stream_bcast(cx, S.get(), cps).p, true);
        Ct E = he.mul_rescale(D.get(), D.get());
        Ct V = he.rotsum(stream_sum(cx, E.get(), cps).p, sh.steps);
        if (m) {
            Ct S2 = he.mul_rescale(S.get(), S.get());
            V = op_add(cx, V.get(), op_mul_int(cx, S2.get(), m).get(), true);
        }
        Ct h = stream_bcast(cx,
                            pl.k[t] ? invsqrt_goldschmidt(he, V.get(), pl.kappa[t], pl.y0[t], pl.k[t],
                                                              pl.relax.data() + pl.relax_at[t])
                                    : he.learned_half(he.mcr_bits(V.get(), pl.kappa[t], -1, 30).get(), &pl.lq[3 * t]),
                            cps);
        double coef = 2.0 * std::sqrt(pl.kappa[t] * pl.n) / pl.c[t];
        // D' = D * coef (times the 0/1 slot mask when padded): the mask is a
        // plaintext of O(1) slot values and coef (~1e-5 for tens of thousands of
        // logits) an integer multiplier, each exact to ~1e-7 or better; one
        // plaintext of coef-sized slot values would round to ~1e-5 relative.
        // D' has spare levels (h's path is longer), so the split costs no depth.
        Ct Dp = m ? he.mul_plain_rescale(D.get(), d_mask, sh.slots, -1, cps) : op_copy(cx, D.get());
        Dp = he.mcr(Dp.get(), coef);
        Ct u = he.mul_rescale(Dp.get(), h.get());
        u = m ? he.add_plain_vec(u.get(), d_mask, sh.slots, cps) : he.add_const(u.get(), 1.0);
        Y = he.power(u.get(), pl.p[t]);
    }
    Ct S = he.rotsum(stream_sum(cx, Y.get(), cps).p, sh.steps);
    Ct F = stream_bcast(cx, inverse_goldschmidt(he, S.get(), pl.kappa_f, pl.d), cps);
    return he.mul_rescale(he.mcr(Y.get(), pl.kappa_f).get(), F.get());
}

}  // namespace he

// ======================================================================
// Bootstrapping (full-slot, real messages).  The paper refreshes
// ciphertexts whose levels run out by bootstrapping (App. B.1); the steps:
//   ModRaise   level-0 ciphertext -> top modulus; the plaintext becomes
//              t = m + q0*I.  Its scale is declared q0*(K+1), so its slots
//              read decode(t)/(q0 (K+1)).
//   CoeffToSlot  slots <- BR(w(t))/(q0 (K+1)), w_k = t_k + i t_(k+h): the
//              inverse of the slot-domain special FFT V = S_h ... S_2 BR
//              (S_len: radix-2 stage of block length len with twiddles
//              exp(2 pi i (5^j mod 4 len)/(4 len))), its stages grouped into
//              three levels, each a baby-step giant-step sum of rotations.
//   split      Re / Im by one conjugation (factor 1/2 in the scale; -i is
//              X^(3N/2)).
//   EvalMod    cos(2 pi ((K+1)x - 1/4)/2^r) by its Chebyshev series, then r
//              double angles: sin(2 pi t/q0).
//   SlotToCoeff  the stages of V in three levels; the factor q0/(2 pi S)
//              is taken into the scale, so the result encrypts the message.
// Bit-reversed slot order between the two transforms is harmless because
// EvalMod acts slot by slot.
// ======================================================================
#include <complex>
#include <functional>
#include <numeric>

namespace he {

using cplx = std::complex<double>;
using Diag = std::map<int, std::vector<cplx>>;  // offset (mod h) -> diagonal

struct LinLevel {
    Diag diag;
    std::vector<int> baby, giant;          // rotation amounts (signed slots)
    std::vector<std::vector<int>> idx;     // [g][b] -> index into pts, or -1
    std::vector<int> offs;                 // per plaintext: its diagonal offset
    std::vector<int> pg;                   // per plaintext: its giant amount
    u64 *pts = nullptr;                    // [n_pt][level+1][N] NTT form
    size_t pts_bytes = 0;
    int level = -1;
    double scale_in = 0, E = 0, target = 0;
};

struct Boot {
    int K = 0, r = 0, d = 0;
    double s_fix = 0, em_scale = 0;
    std::vector<double> cheb;
    LinLevel cts[3], stc[3];
    std::vector<u64> galois;
};

static Diag stage_diag(int h, int len, bool inverse) {
    Diag D;
    std::vector<cplx> d0(h), dp(h), dm(h);
    for (int i = 0; i < h; i++) {
        int j = i % len, half = len / 2;
        int jj = j < half ? j : j - half;
        u64 e = powmod_host(5, (u64)jj, 4ull * len);
        cplx tau = std::polar(1.0, 2.0 * M_PI * (double)e / (4.0 * len));
        if (!inverse) {
            if (j < half) { d0[i] = 1.0; dp[i] = tau; }
            else { dm[i] = 1.0; d0[i] = -tau; }
        } else {
            if (j < half) { d0[i] = 0.5; dp[i] = 0.5; }
            else { d0[i] = -0.5 / tau; dm[i] = 0.5 / tau; }
        }
    }
    auto put = [&](int off, std::vector<cplx> &v) {
        off = ((off % h) + h) % h;
        auto it = D.find(off);
        if (it == D.end()) D[off] = v;
        else for (int i = 0; i < h; i++) it->second[i] += v[i];
    };
    put(0, d0);
    put(len / 2, dp);
    put(-len / 2, dm);
    return D;
}

// (A B) x = A (B x): diag_{r+s} += dA_r * rot(dB_s, r), rot(v, r)[i] = v[i+r]
static Diag diag_mul(const Diag &A, const Diag &B, int h) {
    Diag C;
    for (auto &a : A)
        for (auto &b : B) {
            int off = (a.first + b.first) % h;
            auto &dst = C[off];
            if (dst.empty()) dst.assign(h, 0.0);
            for (int i = 0; i < h; i++) dst[i] += a.second[i] * b.second[(i + a.first) % h];
        }
    for (auto it = C.begin(); it != C.end();) {
        double mx = 0;
        for (auto &v : it->second) mx = std::max(mx, std::abs(v));
        if (mx < 1e-300) it = C.erase(it);
        else ++it;
    }
    return C;
}

static void bsgs_layout(LinLevel &L, int h) {
    std::vector<int> so;
    for (auto &d : L.diag) {
        int r = d.first;
        if (r > h / 2) r -= h;
        so.push_back(r);
    }
    int u = 0;
    for (int r : so) u = std::gcd(u, std::abs(r));
    if (u == 0) u = 1;
    int mmin = 1 << 30, mmax = -(1 << 30);
    for (int r : so) { mmin = std::min(mmin, r / u); mmax = std::max(mmax, r / u); }
    // baby steps only cost an inner product (their ModDown is hoisted), giant
    // steps a full key switch: take bs^2 >= 4 span (more babies, fewer giants)
    int span = mmax - mmin + 1, bs = 1;
    while ((long)bs * bs < 4L * span) bs <<= 1;
    int ng = (span + bs - 1) / bs;
    L.baby.clear();
    L.giant.clear();
    for (int b = 0; b < bs; b++) L.baby.push_back(b * u);
    for (int g = 0; g < ng; g++) L.giant.push_back((mmin + g * bs) * u);
    L.idx.assign(ng, std::vector<int>(bs, -1));
    L.offs.clear();
    L.pg.clear();
    for (int r : so) {
        int m = r / u - mmin, g = m / bs, b = m % bs;
        L.idx[g][b] = (int)L.offs.size();
        L.offs.push_back(((r % h) + h) % h);
        L.pg.push_back(L.giant[g]);
    }
}

static std::vector<double> chebyshev_coeffs(int K, int r, int d) {
    std::vector<double> c(d + 1), fx(d + 1), th(d + 1);
    for (int j = 0; j <= d; j++) {
        th[j] = M_PI * (j + 0.5) / (d + 1);
        double x = std::cos(th[j]);
        fx[j] = std::cos(2.0 * M_PI * ((K + 1) * x - 0.25) / std::ldexp(1.0, r));
    }
    for (int k = 0; k <= d; k++) {
        double s = 0;
        for (int j = 0; j <= d; j++) s += fx[j] * std::cos(k * th[j]);
        c[k] = 2.0 / (d + 1) * s;
    }
    c[0] /= 2;
    return c;
}

// Plaintexts of one transform level for a ciphertext at `level` and `scale`.
static void build_level(he_ctx *cx, LinLevel &L, int level, double scale_in, double target) {
    if (L.pts && L.level == level && L.scale_in == scale_in && L.target == target) return;
    const int h = cx->n / 2;
    const size_t N = cx->N();
    if (L.pts) cx->arena.release(L.pts, L.pts_bytes);
    L.level = level;
    L.scale_in = scale_in;
    L.target = target;
    L.E = (target * (double)cx->primes[level]) / scale_in;
    const int npt = (int)L.offs.size();
    const int ne = cx->lv[level].n_ext;  // plaintexts live in the QP basis
    L.pts_bytes = (size_t)npt * ne * N * 8;
    L.pts = (u64 *)cx->arena.alloc(L.pts_bytes);
    std::vector<double> re(h), im(h);
    for (int p = 0; p < npt; p++) {
        const std::vector<cplx> &dg = L.diag.at(L.offs[p]);
        int G = ((L.pg[p] % h) + h) % h;
        for (int i = 0; i < h; i++) {  // v'[i] = diag[i - G]
            cplx v = dg[((i - G) % h + h) % h];
            re[i] = v.real();
            im[i] = v.imag();
        }
        double *d_re = cx->d_dbl, *d_im = cx->d_dbl + N / 2, *d_pt = cx->d_dbl + N;
        check_cuda(cudaMemcpyAsync(d_re, re.data(), h * 8, cudaMemcpyHostToDevice, cx->stream), "H2D");
        check_cuda(cudaMemcpyAsync(d_im, im.data(), h * 8, cudaMemcpyHostToDevice, cx->stream), "H2D");
        encode_dev(cx, d_re, d_im, h, L.E, d_pt);
        Rows pr = make_rows(L.pts + (size_t)p * ne * N, 0, ne, level + 1, cx->nq);
        load_intd(pr, ne, d_pt, cx->log_n, cx->stream);
        ntt_forward(pr, ne, cx->tw, cx->log_n, cx->stream);
        ew_mont(pr, ne, 0, cx->log_n, cx->stream);  // Montgomery form for ew_diag_mac
        check_cuda(cudaStreamSynchronize(cx->stream), "build transform plaintexts");
    }
}

// sum_g rot_G( sum_b pt[g][b] * rot_b(x) ), one rescale, with both key-switch
// halves hoisted: one ModUp of c1 serves every baby step; the baby-step
// rotations stay in the QP basis as P rot_b(x) (inner product with the key
// plus P sigma_b(c0), no ModDown), the plaintext diagonals are applied there,
// and each giant group pays one ModDown before its giant rotation, whose own
// result is again accumulated in QP; one ModDown at the end.
static Ct apply_level(he_ctx *cx, const he_ct *x, LinLevel &L, double target) {
    build_level(cx, L, x->level, x->scale, target);
    const int l = x->level, h = cx->n / 2, B = x->batch;
    const size_t N = cx->N();
    const LevelTabs &LT = cx->lv[l];
    const int ne = LT.n_ext;
    // per member: a QP-basis ciphertext of 2 ne rows; members back to back
    const size_t qp_w = (size_t)2 * ne * N, xs = ct_member_stride(x);
    cudaStream_t s = cx->stream;
    Scratch bufs{cx, {}};
    auto qp = [&](u64 *base) { return make_rows(base, (size_t)ne * N, ne, l + 1, cx->nq); };
    // baby steps in QP
    std::vector<u64 *> baby(L.baby.size(), nullptr);
    u64 *ext = nullptr;
    for (size_t b = 0; b < L.baby.size(); b++) {
        bool used = false;
        for (auto &row : L.idx) used |= row[b] >= 0;
        if (!used) continue;
        baby[b] = bufs.get((size_t)B * qp_w);
        if (b == 0) {
            ew_qp_lift(baby[b], ct_poly(x, 0), l + 1, ne, 0, 0, cx->p_mod, cx->slot, cx->log_n, s, B, qp_w, xs);
            ew_qp_lift(baby[b] + (size_t)ne * N, ct_poly(x, 1), l + 1, ne, 0, 0, cx->p_mod, cx->slot, cx->log_n, s, B,
                       qp_w, xs);
            continue;
        }
        u64 g = rot_galois(cx, L.baby[b]);
        const KeyDev *key = find_key(cx, g);
        if (!key) throw Error{HE_ENOKEY, "bootstrapping rotation key missing"};
        if (!ext) {
            ext = bufs.get((size_t)B * ks_ext_words(cx, l));
            modup(cx, ct_poly(x, 1), l, ext, B, xs);
        }
        ks_inner(cx, ct_poly(x, 1), ext, l, *key, g, baby[b], B, xs);
        ew_qp_lift(baby[b], ct_poly(x, 0), l + 1, ne, g, 1, cx->p_mod, cx->slot, cx->log_n, s, B, qp_w, xs);
    }
    // giant groups
    u64 *tot = bufs.get((size_t)B * qp_w), *inner = bufs.get((size_t)B * qp_w);
    u64 *gext = nullptr, *gacc = nullptr;
    bool have = false;
    for (size_t g = 0; g < L.giant.size(); g++) {
        DiagMac dm;
        dm.n = 0;
        dm.slot = cx->slot;
        dm.l1 = l + 1;
        dm.nq = cx->nq;
        dm.batch = B;
        dm.c_stride = qp_w;
        dm.out_stride = qp_w;
        for (size_t b = 0; b < L.baby.size(); b++) {
            int p = L.idx[g][b];
            if (p < 0) continue;
            if (dm.n == DIAG_MAC_MAX) throw Error{HE_EINVAL, "too many diagonals in one giant step"};
            dm.c0[dm.n] = baby[b];
            dm.c1[dm.n] = baby[b] + (size_t)ne * N;
            dm.pt[dm.n] = L.pts + (size_t)p * ne * N;
            dm.n++;
        }
        if (!dm.n) continue;
        const bool rot = L.giant[g] % h != 0;
        u64 *dst = (!rot && !have) ? tot : inner;
        dm.out0 = dst;
        dm.out1 = dst + (size_t)ne * N;
        ew_diag_mac(dm, ne, cx->log_n, s);
        cx->ops_by_level[2][l] += (uint64_t)dm.n * (uint64_t)B;
        if (!rot) {
            if (have) ew_add(qp(tot), qp(tot), qp(inner), 2 * B * ne, 0, cx->log_n, s);
            have = true;
            continue;
        }
        // ModDown of the group, then its giant rotation, accumulated in QP
        Ct y(ct_alloc(cx, l, x->scale * L.E, B));
        moddown(cx, inner, l, ct_rows(y.get()), ct_rows(y.get()), 0, B);
        u64 gg = rot_galois(cx, L.giant[g]);
        const KeyDev *key = find_key(cx, gg);
        if (!key) throw Error{HE_ENOKEY, "bootstrapping rotation key missing"};
        if (!gext) gext = B == 1 ? cx->ks_ext : bufs.get((size_t)B * ks_ext_words(cx, l));
        const size_t ys = ct_member_stride(y.get());
        modup(cx, ct_poly(y.get(), 1), l, gext, B, ys);
        u64 *acc = tot;
        if (have) {
            if (!gacc) gacc = B == 1 ? cx->ks_acc : bufs.get((size_t)B * qp_w);
            acc = gacc;
        }
        ks_inner(cx, ct_poly(y.get(), 1), gext, l, *key, gg, acc, B, ys);
        ew_qp_lift(acc, ct_poly(y.get(), 0), l + 1, ne, gg, 1, cx->p_mod, cx->slot, cx->log_n, s, B, qp_w, ys);
        if (have) ew_add(qp(tot), qp(tot), qp(acc), 2 * B * ne, 0, cx->log_n, s);
        have = true;
    }
    if (!have) throw Error{HE_EINVAL, "empty linear transform level"};
    Ct out(ct_alloc(cx, l, x->scale * L.E, B));
    moddown(cx, tot, l, ct_rows(out.get()), ct_rows(out.get()), 0, B);
    return op_rescale(cx, out.get());
}

// Chebyshev series sum_k c_k T_k(x) by baby steps T_1..T_(m-1) and giant
// steps T_m, T_2m, T_4m, ...: a series of degree >= m is split by the largest
// giant G <= degree as q T_G + r (T_G T_j = (T_(G+j) + T_(|G-j|))/2 gives
// q_0 = c_G, q_j = 2 c_(G+j), r_(G-j) = c_(G-j) - c_(G+j)).  Every call
// lands on the scale it is asked for: q is aimed at target q_lp / scale(T_G),
// q_lp the prime that rescales the product q T_G, so that the product comes
// out at the target, and r is aimed at the product's scale.  (Two summands
// whose declared scales differ by a relative e add with an error e |value|,
// which the double-angle steps and the 1/(2 pi) read-out of bootstrapping
// amplify by several orders of magnitude.)
struct ChebEval {
    HE &he;
    std::vector<Ct> T;   // T_1..T_(m-1) and the giants (index k)
    int m;

    int giant(int deg) const {
        int G = m;
        while (2 * G <= deg) G *= 2;
        return G;
    }

    // level of eval()'s result for a series of degree deg
    int out_level(int deg) const {
        if (deg < m) {
            int lo = 1 << 30;
            for (int k = 1; k <= deg; k++) lo = std::min(lo, T[k]->level);
            return lo - 1;
        }
        int G = giant(deg);
        if (deg == G) return T[G]->level - 1;
        return std::min(out_level(deg - G), T[G]->level) - 1;
    }

    // sum_k c_k T_k + c_0 with one rescale for all terms: every T_k is
    // dropped to the lowest level l among them and multiplied by the integer
    // K_k = rint(c_k E_k), E_k = target q_l / scale(T_k), so that every term
    // sits at the scale target q_l; the sum is rescaled once, onto target
    Ct baby_sum(const std::vector<double> &c, double target) {
        he_ctx *cx = he.cx;
        int low = 1 << 30;
        for (size_t k = 1; k < c.size(); k++)
            if (c[k] != 0.0) low = std::min(low, T[k]->level);
        if (low == (1 << 30)) throw Error{HE_EINVAL, "empty Chebyshev series"};
        const double sc = target * (double)he.q(low);
        Ct acc;
        for (size_t k = 1; k < c.size(); k++) {
            if (c[k] == 0.0) continue;
            Ct dropped;
            const he_ct *t = T[k].get();
            if (t->level > low) {
                dropped = op_drop(cx, t, low);
                t = dropped.get();
            }
            Ct u = op_mul_intd(cx, t, std::rint(c[k] * (sc / t->scale)), sc);
            acc = acc ? op_add(cx, acc.get(), u.get(), false) : std::move(u);
        }
        acc = op_rescale(cx, acc.get());
        return he.add_const(acc.get(), c[0]);
    }

    Ct eval(const std::vector<double> &c, double target) {
        he_ctx *cx = he.cx;
        int deg = (int)c.size() - 1;
        if (deg < m) return baby_sum(c, target);
        int G = giant(deg);
        std::vector<double> q(deg - G + 1), r(c.begin(), c.begin() + G);
        q[0] = c[G];
        for (int j = 1; j <= deg - G; j++) {
            q[j] = 2.0 * c[G + j];
            r[G - j] -= c[G + j];
        }
        Ct P;
        if (deg == G) {  // constant quotient: one constant multiplication of T_G
            P = he.mcr(T[G].get(), q[0], target);
        } else {
            const int lp = std::min(out_level(deg - G), T[G]->level);
            Ct Q = eval(q, target * (double)cx->primes[lp] / T[G]->scale);
            P = he.mul_rescale(Q.get(), T[G].get());
        }
        Ct R = eval(r, P->scale);
        if (R->level > P->level) R = op_drop(cx, R.get(), P->level);
        return op_add(cx, P.get(), R.get(), false);
    }
};

// Chebyshev series sum_k c_k T_k(x) of a ciphertext x with slots in [-1, 1]
// (baby steps T_1..T_(m-1), giants T_m, T_2m, ...), landing on `target`.
static Ct cheb_series(HE &he, const he_ct *x, const std::vector<double> &cheb, double target);

static Ct evalmod(HE &he, const he_ct *x, const Boot &B) {
    Ct c = cheb_series(he, x, B.cheb, B.em_scale);
    for (int i = 0; i < B.r; i++)
        c = he.add_const(op_mul_int(he.cx, he.mul_rescale(c.get(), c.get()).get(), 2).get(), -1.0);
    return c;
}

static Ct cheb_series(HE &he, const he_ct *x, const std::vector<double> &cheb, double target) {
    he_ctx *cx = he.cx;
    const int d = (int)cheb.size() - 1;
    int m = 1;
    while (m * m <= d + 1) m *= 2;  // baby steps T_1..T_(m-1)
    int top = m;
    while (2 * top <= d) top *= 2;  // largest giant step
    ChebEval ce{he, std::vector<Ct>(std::max(m, top) + 1), m};
    ce.T[1] = op_copy(cx, x);
    auto make = [&](int k) {  // T_k = 2 T_a T_b - T_(a-b), a = ceil(k/2), b = floor(k/2)
        int a = (k + 1) / 2, b = k / 2;
        Ct P2 = op_mul_int(cx, he.mul_rescale(ce.T[a].get(), ce.T[b].get()).get(), 2);
        if (a == b) {
            ce.T[k] = he.add_const(P2.get(), -1.0);
        } else {
            Ct xm = he.mcr(ce.T[1].get(), 1.0, P2->scale);
            if (xm->level > P2->level) xm = op_drop(cx, xm.get(), P2->level);
            ce.T[k] = op_add(cx, P2.get(), xm.get(), true);
        }
    };
    for (int k = 2; k < m; k++) make(k);
    for (int g = m; g <= top; g *= 2) make(g);
    return ce.eval(cheb, target);
}

// Beta(alpha, 1) cut noise of Alg. 3 from an encrypted uniform (Lemma 2 /
// Observation 1: G = U^(1/alpha), alpha = ln(1-q)/ln(p)): the degree-d
// Chebyshev interpolant (Chebyshev nodes) of f(t) = ((t + 1)/2)^(1/alpha) on
// t = 2U - 1, so that the server draws the noise from the client's uniforms.
// The interpolant follows U^(1/alpha) to ~1e-2 for U >= 1e-3 at d = 31; it
// cannot follow the cusp at U = 0.  The series works at U's own scale (t =
// 2U - 1 keeps it), so uniforms encrypted above the circuit's levels at the
// size of the primes there keep that scale through the products, and the
// noise lands on the context's scale Delta, d's depth plus one below U.
Ct beta_noise(he_ctx *cx, const he_ct *u, double alpha, int d) {
    if (!(alpha > 0) || d < 2 || d > 127) throw Error{HE_EINVAL, "noise needs alpha > 0 and degree 2..127"};
    HE he{cx, cx->delta};
    std::vector<double> c(d + 1), fx(d + 1), th(d + 1);
    for (int j = 0; j <= d; j++) {
        th[j] = M_PI * (j + 0.5) / (d + 1);
        fx[j] = std::pow((std::cos(th[j]) + 1.0) / 2.0, 1.0 / alpha);
    }
    for (int k = 0; k <= d; k++) {
        double acc = 0;
        for (int j = 0; j <= d; j++) acc += fx[j] * std::cos(k * th[j]);
        c[k] = 2.0 / (d + 1) * acc;
    }
    c[0] /= 2;
    Ct t = he.add_const(he.mcr(u, 2.0, u->scale).get(), -1.0);
    return cheb_series(he, t.get(), c, cx->delta);
}

// Level bookkeeping of evalmod(): the baby-step giant-step series can use
// one level less than ceil(log2(d+1)) + 1 for some degrees, so the output
// level is found by replaying it.
static int evalmod_out_level(int l0, int d, int r) {
    int m = 1;
    while (m * m <= d + 1) m *= 2;
    int top = m;
    while (2 * top <= d) top *= 2;
    std::vector<int> T(std::max(m, top) + 1, 0);
    T[1] = l0;
    auto make = [&](int k) { T[k] = std::min(T[(k + 1) / 2], T[k / 2]) - 1; };
    for (int k = 2; k < m; k++) make(k);
    for (int g = m; g <= top; g *= 2) make(g);
    std::function<int(int)> ev = [&](int deg) -> int {
        if (deg < m) {
            int lo = 1 << 30;
            for (int k = 1; k <= deg; k++) lo = std::min(lo, T[k]);
            return lo - 1;
        }
        int G = m;
        while (2 * G <= deg) G *= 2;
        if (deg == G) return T[G] - 1;
        int Q = ev(deg - G);
        return std::min(Q, T[G]) - 1;
    };
    return ev(d) - r;
}

// level of a bootstrapped ciphertext: 3 (CoeffToSlot) + EvalMod + 3 (SlotToCoeff) below the top
int boot_out_level(he_ctx *cx) {
    const Boot &B = *cx->boot_state;
    return evalmod_out_level(cx->nq - 1 - 3, B.d, B.r) - 3;
}

void boot_prepare(he_ctx *cx, int K, int r, int d) {
    if (d < 2 || d > 63 || r < 0 || r > 8 || K < 1) throw Error{HE_EINVAL, "bootstrap parameters out of range"};
    if (cx->nq < 18) throw Error{HE_ELEVEL, "bootstrapping needs at least 17 levels above q0"};
    auto B = std::make_shared<Boot>();
    B->K = K;
    B->r = r;
    B->d = d;
    B->s_fix = cx->delta;
    B->em_scale = std::ldexp(1.0, 60);
    B->cheb = chebyshev_coeffs(K, r, d);
    const int h = cx->n / 2, s = cx->log_n - 1;
    int g3 = s / 3, g2 = (s - g3) / 2, g1 = s - g3 - g2;  // g1 >= g2 >= g3
    int sizes[3] = {g1, g2, g3};
    // SlotToCoeff: stages len = 2, 4, ..., applied in that order, grouped
    int st = 1;
    for (int lv = 0; lv < 3; lv++) {
        Diag M;
        for (int k = 0; k < sizes[lv]; k++, st++) {
            Diag S = stage_diag(h, 1 << st, false);
            M = M.empty() ? S : diag_mul(S, M, h);
        }
        B->stc[lv].diag = M;
        bsgs_layout(B->stc[lv], h);
    }
    // CoeffToSlot: inverse stages len = h, h/2, ..., grouped
    st = s;
    for (int lv = 0; lv < 3; lv++) {
        Diag M;
        for (int k = 0; k < sizes[lv]; k++, st--) {
            Diag S = stage_diag(h, 1 << st, true);
            M = M.empty() ? S : diag_mul(S, M, h);
        }
        B->cts[lv].diag = M;
        bsgs_layout(B->cts[lv], h);
    }
    std::vector<u64> gs;
    for (auto *Ls : {B->cts, B->stc})
        for (int lv = 0; lv < 3; lv++) {
            for (int b : Ls[lv].baby)
                if (b % h) gs.push_back(rot_galois(cx, b));
            for (int g : Ls[lv].giant)
                if (g % h) gs.push_back(rot_galois(cx, g));
        }
    gs.push_back(2 * cx->N() - 1);
    // the constant bootstrap's trace: a rotate-and-sum over every slot
    for (const auto &rots : rotsum_stages(cx->log_n - 1, cx->rotsum_log_radix))
        for (i64 r : rots) gs.push_back(rot_galois(cx, r));
    gs.push_back(rot_galois(cx, h / 2));
    std::sort(gs.begin(), gs.end());
    gs.erase(std::unique(gs.begin(), gs.end()), gs.end());
    B->galois = gs;
    gen_relin_key(cx);
    for (u64 g : gs) gen_galois_key(cx, g);
    cx->boot_state = B;
    cx->gen++;  // graphs that point into the previous tables retire
}

Ct bootstrap_ct(he_ctx *cx, const he_ct *in) { return bootstrap_stage(cx, in, 100); }

// stage: 0 ModRaise, 1..3 after CoeffToSlot level, 4 real part, 5 imaginary
// part, 6 real part after EvalMod, 7 imaginary part after EvalMod, 8 combined,
// 9..11 after SlotToCoeff level (11 = the bootstrapped result)
Ct bootstrap_stage(he_ctx *cx, const he_ct *in, int stage) {
    auto B = cx->boot_state;
    if (!B) throw Error{HE_EINVAL, "bootstrapping not prepared"};
    HE he{cx, B->em_scale};
    cx->n_boot += (uint64_t)in->batch;
    const u64 q0 = cx->primes[0];
    const double ratio = in->scale / B->s_fix;
    Ct low = in->level ? op_drop(cx, in, 0) : op_copy(cx, in);
    Ct x = op_mod_raise(cx, low.get(), cx->nq - 1);
    x->scale = (double)q0 * (double)(B->K + 1);
    if (stage == 0) return x;
    // CoeffToSlot, aimed at half the EvalMod scale (the split doubles it)
    for (int lv = 0; lv < 3; lv++) {
        x = apply_level(cx, x.get(), B->cts[lv], B->em_scale / 2);
        if (stage == 1 + lv) return x;
    }
    Ct xc = op_automorph(cx, x.get(), 2 * cx->N() - 1);
    Ct re = op_add(cx, x.get(), xc.get(), false);
    re->scale *= 2;
    if (stage == 4) return re;
    Ct im = op_mul_monomial(cx, op_add(cx, x.get(), xc.get(), true).get(), 3 * cx->N() / 2);
    im->scale *= 2;
    if (stage == 5) return im;
    if (in->batch <= 2) {
        // both parts as one batch: every launch carries twice the rows and
        // every key word read serves both (members are bit-identical to
        // separate evaluations); larger batches fill the GPU by themselves
        const he_ct *parts[2] = {re.get(), im.get()};
        Ct both = evalmod(he, op_batch_pack(cx, parts, 2).get(), *B);
        re = op_batch_member(cx, both.get(), 0, in->batch);
        im = op_batch_member(cx, both.get(), in->batch, in->batch);
    } else {
        re = evalmod(he, re.get(), *B);
        im = evalmod(he, im.get(), *B);
    }
    if (stage == 6) return re;
    if (stage == 7) return im;
    Ct w = op_add(cx, re.get(), op_mul_monomial(cx, im.get(), cx->N() / 2).get(), false);
    // values sin(2 pi t/q0) ~ 2 pi m/q0: read them as m / s_fix
    w->scale = w->scale * (2.0 * M_PI * B->s_fix) / (double)q0;
    if (stage == 8) return w;
    const double tg[3] = {std::ldexp(1.0, 50), std::ldexp(1.0, 45), cx->delta};
    for (int lv = 0; lv < 3; lv++) {
        w = apply_level(cx, w.get(), B->stc[lv], tg[lv]);
        if (stage == 9 + lv && lv < 2) return w;
    }
    // the slots read m / s_fix = (message) * ratio: declaring the scale ratio
    // times larger reads the message
    w->scale = w->scale * ratio;
    return w;
}

// Bootstrapping of a ciphertext whose slots all hold one complex value z (the
// polynomial a + b X^(N/2)), at about half the cost of bootstrap_stage: after
// ModRaise, t = m + q0 I is projected onto {1, X^(N/2)} by the trace over the
// automorphisms X -> X^(5^k) (a log2(N/2)-step rotate-and-sum, exact: every
// other monomial's orbit sums to 0) instead of CoeffToSlot; its two
// coefficients, scaled, become the real and the imaginary part of every
// slot, are packed into the two slot halves for one EvalMod (followed by one
// arcsine step), and are put back as a complex constant, in place of the
// second EvalMod and of SlotToCoeff.  Returns the refreshed ciphertext at the
// bootstrap output level and the input's scale.
Ct bootstrap_const(he_ctx *cx, const he_ct *in) {
    auto B = cx->boot_state;
    if (!B) throw Error{HE_EINVAL, "bootstrapping not prepared"};
    HE he{cx, B->em_scale};
    cx->n_boot += (uint64_t)in->batch;
    const u64 q0 = cx->primes[0];
    const int slots = cx->n / 2, half = slots / 2;
    const double ratio = in->scale / B->s_fix;
    Ct low = in->level ? op_drop(cx, in, 0) : op_copy(cx, in);
    // raised to 2 levels below the top, so that the packing mask lands the
    // EvalMod input on the level (and scale) where bootstrap_stage has it
    Ct x = op_mod_raise(cx, low.get(), cx->nq - 3);
    x->scale = (double)q0 * (double)(B->K + 1);
    x = op_rotsum(cx, x.get(), cx->log_n - 1);  // trace: N/2 (t_0 + t_(N/2) X^(N/2))
    x->scale *= (double)slots;
    // slots read (t_0 + i t_(N/2)) / (q0 (K+1)): real and imaginary parts, packed
    Ct xc = op_automorph(cx, x.get(), 2 * cx->N() - 1);
    Ct re = op_add(cx, x.get(), xc.get(), false);
    re->scale *= 2;
    Ct im = op_mul_monomial(cx, op_add(cx, x.get(), xc.get(), true).get(), 3 * cx->N() / 2);
    im->scale *= 2;
    std::vector<double> lo(slots, 0.0), hi(slots, 0.0);
    for (int i = 0; i < half; i++) lo[i] = 1.0, hi[half + i] = 1.0;
    Scratch sc{cx, {}};
    const double *d_lo = upload_scaled(cx, sc, lo, 1.0), *d_hi = upload_scaled(cx, sc, hi, 1.0);
    Ct y = op_add(cx, he.mul_plain_rescale(re.get(), d_lo, slots, B->em_scale).get(),
                  he.mul_plain_rescale(im.get(), d_hi, slots, B->em_scale).get(), false);
    y = evalmod(he, y.get(), *B);
    // A constant's whole value sits in coefficient 0 (a vector's spreads over
    // N coefficients), so sin(theta), theta = 2 pi m / q0, is read at angles
    // where its curvature shows (theta^2 / 6 ~ 4e-4 for a value 1 at q0 = 2^47
    // against Delta = 2^40). One Taylor step of arcsin, sin + sin^3 / 6, takes
    // the error to 3 theta^4 / 40; the 1/6 is a scale declaration.
    {
        Ct y2 = he.mul_rescale(y.get(), y.get());
        y2->scale *= 6.0;
        y = he.mul_rescale(y.get(), he.add_const(y2.get(), 1.0).get());
    }
    // w = y + i rot(y, s/2): the lower half holds re + i im; keep it, spread it
    Ct w = op_add(cx, y.get(), op_mul_monomial(cx, op_automorph(cx, y.get(), rot_galois(cx, half)).get(),
                                                 cx->N() / 2).get(), false);
    // the mask aims at q0 / (2 pi), so that the read-out below lands on the
    // input's scale
    w = he.mul_plain_rescale(w.get(), d_lo, slots, (double)q0 / (2.0 * M_PI));
    w = op_add(cx, w.get(), op_automorph(cx, w.get(), rot_galois(cx, half)).get(), false);
    // values sin(2 pi t/q0) ~ 2 pi m/q0: read them as m / s_fix, then as m / scale(in)
    w->scale = w->scale * (2.0 * M_PI * B->s_fix) / (double)q0 * ratio;
    const int out = boot_out_level(cx);
    return w->level > out ? op_drop(cx, w.get(), out) : std::move(w);
}

// Refresh schedule of the bootstrapped circuit with per-stream scalar chains.
// The scalars (x, h and the final sum) hold one value in every slot and are
// refreshed by the constant bootstrap; the vector Y, D', u by the general one
// (7/3 of the cost: 33.2 against 14.3 ms at N = 2^16, 30 + 10 primes, on a
// GB300). Per iteration two choices are open: refresh h when
// it sits below D' (so that u keeps D's levels for the power), and bootstrap
// Y before the statistics although it has the 5 levels they need. Every
// combination is played on the circuit's level bookkeeping (integer multipliers
// sized from the primes' bit lengths, as the rescale rule does) and the one
// costing least (general 7, constant 3; then fewer bootstraps; then the first)
// is kept.  Plans of more than 16 iterations make no optional refresh.
struct RefreshSched {
    std::vector<uint8_t> h_refresh, y_boot;
};
static RefreshSched refresh_schedule(he_ctx *cx, const Plan &pl, int y_level, int out, bool padded) {
    auto bits = [&](int l) { return (double)std::lround(std::log2((double)cx->primes[l])); };
    auto mcr_bits_level = [&](int a, double c) {
        int r = 1;
        double e = bits(a);
        while (std::fabs(c) * std::exp2(e) < std::exp2(30.0) && r < 3 && a - r >= 1) e += bits(a - r), r++;
        return a - r;
    };
    const int T = pl.T, per = T <= 6 ? 4 : 2;  // choices per iteration (early Y bootstraps only up to T = 6)
    if (T > 16) return RefreshSched{std::vector<uint8_t>(T, 0), std::vector<uint8_t>(T, 0)};  // no search
    long total = 1;
    for (int t = 0; t < T; t++) total *= per;
    long best = -1;
    int best_cost = 1 << 30, best_n = 1 << 30;
    for (long combo = 0; combo < total; combo++) {
        long cc = combo;
        int Y = y_level, g = 0, c = 0;
        for (int t = 0; t < T; t++) {
            const int ch = (int)(cc % per);
            cc /= per;
            const bool hr = ch & 1, yb = ch & 2;
            const int k = pl.k[t], lp = power_depth(pl.p[t]);
            if (Y < 5 || yb) Y = out, g++;
            int x = mcr_bits_level(Y - 1, pl.kappa[t]);
            if (x < 2) x = out, c += 1000;  // x (up to ~sqrt of the range ratio) is too large to refresh well
            int h;
            if (k == 0) {
                h = x - 2;
            } else {
                int z = x - 2;
                for (int i = 2; i <= k; i++) {
                    if (z < 2) z = out - 1, c++;
                    z -= 2;
                }
                if (z < 1) z = out, c++;
                h = z;
            }
            int Dp = Y - (padded ? 2 : 1);
            if (hr && h < Dp) h = out, c++;
            if (h < 1) h = out, c++;
            if (Dp < 1) Dp = out, g++;
            int u = std::min(Dp, h) - 1;
            if (u < lp) u = out, g++;
            Y = u - lp;
        }
        if (Y < 2) Y = out, g++;
        if (Y < pl.d + 3) c++;
        const int cost = 7 * g + 3 * c;
        if (cost < best_cost || (cost == best_cost && g + c < best_n)) best = combo, best_cost = cost, best_n = g + c;
    }
    RefreshSched rs{std::vector<uint8_t>(T, 0), std::vector<uint8_t>(T, 0)};
    for (int t = 0; t < T; t++) {
        const int ch = (int)(best % per);
        best /= per;
        rs.h_refresh[t] = ch & 1;
        rs.y_boot[t] = (ch & 2) ? 1 : 0;
    }
    return rs;
}

// Refresh schedule of the bootstrapped circuit with scalar chains shared by the
// batch's streams.  A refresh of a vector (Y, D', u) bootstraps every one of
// the batch's `members` ciphertexts, one of a per-stream scalar (x before
// packing, h after unpacking) one ciphertext per stream, one of the packed
// chain a single ciphertext.  Per iteration two choices
// are open: refresh the packed h before unpacking it when it would arrive
// below D' (u then keeps D's levels for the power), and bootstrap Y before the
// statistics although it has the levels they need.  Every combination is
// played on the shared circuit's level bookkeeping and the one that
// bootstraps fewest ciphertexts is kept (then the first).
static RefreshSched refresh_schedule_shared(he_ctx *cx, const Plan &pl, int y_level, int out, bool padded,
                                            int members, int streams) {
    auto bits = [&](int l) { return (double)std::lround(std::log2((double)cx->primes[l])); };
    auto mcr_bits_level = [&](int a, double c) {
        int r = 1;
        double e = bits(a);
        while (std::fabs(c) * std::exp2(e) < std::exp2(30.0) && r < 3 && a - r >= 1) e += bits(a - r), r++;
        return a - r;
    };
    const int T = pl.T, per = T <= 6 ? 4 : 2;
    if (T > 16) return RefreshSched{std::vector<uint8_t>(T, 0), std::vector<uint8_t>(T, 0)};
    long total = 1;
    for (int t = 0; t < T; t++) total *= per;
    long best = -1, best_cost = 1L << 40;
    for (long combo = 0; combo < total; combo++) {
        long cc = combo, cost = 0;
        int Y = y_level;
        for (int t = 0; t < T; t++) {
            const int ch = (int)(cc % per);
            cc /= per;
            const bool hr = ch & 1, yb = ch & 2;
            const int k = pl.k[t], lp = power_depth(pl.p[t]);
            if (Y < 5 || yb) Y = out, cost += members;
            int x = mcr_bits_level(Y - 1, pl.kappa[t]);
            if (x < 1) x = out, cost += streams;
            x -= 1;                                   // pack: the class mask
            if (x < 2) x = out, cost += 1;
            int h;
            if (k == 0) {
                h = x - 2;
            } else {
                int P = x - 2;                        // start: constant products, then P a
                for (int i = 2; i <= k; i++) {
                    if (P < 2) P = out - 1, cost += 1;
                    P -= 2;
                }
                if (P < 1) P = out, cost += 1;
                h = P - 1;                            // h's half of the pair
            }
            const int Dp = Y - (padded ? 2 : 1);
            if (hr && h - 1 < Dp) h = out, cost += 1;  // refresh the packed h
            if (h < 1) h = out, cost += 1;
            h -= 1;                                   // unpack: the class mask
            if (h < 1) h = out, cost += streams;
            int d = Dp;
            if (d < 1) d = out, cost += members;
            int u = std::min(d, h) - 1;
            if (u < lp) u = out, cost += members;
            Y = u - lp;
        }
        if (Y < 2) Y = out, cost += members;           // the final mcr and product
        if (Y - 1 < pl.d + 3) cost += 1;              // the packed final sum before the inverse
        if (cost < best_cost) best = combo, best_cost = cost;
    }
    RefreshSched rs{std::vector<uint8_t>(T, 0), std::vector<uint8_t>(T, 0)};
    for (int t = 0; t < T; t++) {
        const int ch = (int)(best % per);
        best /= per;
        rs.h_refresh[t] = ch & 1;
        rs.y_boot[t] = (ch & 2) ? 1 : 0;
    }
    return rs;
}

// Alg. 2 with bootstrapping when levels run out (same steps as cutmax_ct;
// the Goldschmidt input is x = kappa V and Y_(t+1) is scaled by norm[t]
// through u' = norm^(1/p) u, so that every refreshed ciphertext is bounded).
static Ct cutmax_boot(he_ctx *cx, const he_ct *in, const Plan &pl) {
    if (!cx->boot_state) throw Error{HE_EINVAL, "bootstrapped plan needs he_bootstrap_prepare"};
    StreamShape sh = stream_shape(cx, in, pl);
    const int slots = sh.slots, cps = sh.cps, m = sh.m;
    HE he{cx, cx->delta};
    auto ensure = [&](Ct c, int need) -> Ct { return c->level < need ? bootstrap_ct(cx, c.get()) : std::move(c); };
    // compute only on the levels a bootstrap hands back: the primes above are
    // the bootstrapping primes, where products of Delta-scale ciphertexts
    // would shrink the scale
    const int out_level = boot_out_level(cx);
    Ct Y = in->level > out_level ? op_drop(cx, in, out_level) : op_copy(cx, in);
    // shared scalar chains: the Goldschmidt pair packed in one ciphertext,
    // slots [0, s/2) holding g, slots [s/2, s) h; one rotation by s/2 lines
    // them up for g*h (per-stream chains carry it as one complex constant)
    const int half = slots / 2;
    const u64 g_half = rot_galois(cx, half);
    // scalar chains shared by the batch's streams: stream s owns the slots
    // i = s (mod Sp); packing costs one level, unpacking one level and a
    // log2(Sp)-step rotate-and-sum
    const int n_streams = sh.S;
    const bool shared = pl.shared && n_streams > 1;
    const RefreshSched rs = shared ? refresh_schedule_shared(cx, pl, Y->level, out_level, m != 0, in->batch, sh.S)
                                   : refresh_schedule(cx, pl, Y->level, out_level, m != 0);
    int Sp = 1, lsp = 0;
    while (Sp < n_streams) Sp *= 2, lsp++;
    if (shared && (Sp > slots / 2 || lsp > sh.steps))
        throw Error{HE_EINVAL, "too many streams to share the scalar chains"};
    Scratch smask{cx, {}};
    const double *d_cls = nullptr;
    if (shared) {
        std::vector<double> cls((size_t)n_streams * slots, 0.0);
        for (int st = 0; st < n_streams; st++)
            for (int i = st; i < slots; i += Sp) cls[(size_t)st * slots + i] = 1.0;
        d_cls = upload_scaled(cx, smask, cls, 1.0);
    }
    auto pack = [&](const he_ct *a) -> Ct {  // S members, replicated scalars -> one ciphertext
        Ct mk = he.mul_plain_rescale(a, d_cls, slots, -1, n_streams);
        return op_group(cx, mk.get(), n_streams, true);
    };
    auto unpack = [&](const he_ct *a) -> Ct {  // one packed ciphertext -> S members, replicated
        Ct b = op_group(cx, a, n_streams, false);
        Ct mk = he.mul_plain_rescale(b.get(), d_cls, slots, -1, n_streams);
        return he.rotsum(mk.get(), lsp);
    };
    for (int t = 0; t < pl.T; t++) {
        const int p = pl.p[t], k = pl.k[t];
        const double kap = pl.kappa[t], y0 = pl.y0[t], rn = std::pow(pl.norm[t], 1.0 / p);
        if (Y->level < 5 || rs.y_boot[t]) Y = bootstrap_ct(cx, Y.get());
        Ct S = he.rotsum(stream_sum(cx, Y.get(), cps).p, sh.steps);
        Ct D = op_add(cx, op_mul_int(cx, Y.get(), pl.n).get(), stream_bcast(cx, S.get(), cps).p, true);
        Ct E = he.mul_rescale(D.get(), D.get());
        Ct V = he.rotsum(stream_sum(cx, E.get(), cps).p, sh.steps);
        if (m) {
            Ct S2 = he.mul_rescale(S.get(), S.get());
            V = op_add(cx, V.get(), op_mul_int(cx, S2.get(), m).get(), true);
        }
        // V (about n^3 sigma^2, far beyond what a bootstrap can refresh) keeps
        // the 4 levels that Y brought: up to 3 rescales scale it to x ~ 1
        Ct x = he.mcr_bits(V.get(), kap, -1, 30);
        if (shared) x = pack(ensure(std::move(x), 1).get());
        if (x->level < 2) x = shared ? bootstrap_ct(cx, x.get()) : bootstrap_const(cx, x.get());
        const double coef = 2.0 * std::sqrt(kap * pl.n) / pl.c[t] * rn;
        // D' = D * coef (times the 0/1 slot mask when padded), mask and scalar
        // applied separately for precision (see cutmax_ct)
        Ct Dp;
        if (m) {
            Scratch s2{cx, {}};
            Dp = he.mul_plain_rescale(D.get(), upload_scaled(cx, s2, sh.mask, 1.0), slots, -1, cps);
            Dp = he.mcr(Dp.get(), coef);
        } else {
            Dp = he.mcr(D.get(), coef);
        }
        // shared chains: the packed h, refreshed first when the schedule says so
        // and it would arrive below D', back to the streams
        auto unpack_h = [&](Ct hp) -> Ct {
            if (rs.h_refresh[t] && hp->level - 1 < Dp->level) hp = bootstrap_ct(cx, hp.get());
            return unpack(ensure(std::move(hp), 1).get());
        };
        Ct h;
        if (k == 0) {  // learned quadratic in place of the Goldschmidt iteration
            h = he.learned_half(x.get(), &pl.lq[3 * t]);
            if (shared) h = unpack_h(std::move(h));
        } else if (!shared) {
            // Goldschmidt pair as one complex constant z = g + i h/4 in every
            // slot (the polynomial g + (h/4) X^(N/2)): 2 Im(z^2) = g h by one
            // conjugation, z <- z (1.5 - g h), h = 4 Im(z); the 1/4 keeps
            // every step's scale at s^3 / (q q'), as for a real pair.
            // Refreshed by the constant bootstrap (bootstrap_const), then
            // landed on Delta.
            const u64 g_conj = 2 * cx->N() - 1, e_mi = 3 * cx->N() / 2;  // X -> X^-1; X^(3N/2) = -i
            auto imag2 = [&](const he_ct *a) {  // 2 Im(a) as a real constant: (a - conj a)(-i)
                return op_mul_monomial(cx, op_add(cx, a, op_automorph(cx, a, g_conj).get(), true).get(), e_mi);
            };
            Ct a = he.add_const(he.mcr(x.get(), -y0 * y0 / 2.0).get(), pl.alpha(t, 0));
            Ct z = he.add_complex_const(he.mcr(x.get(), y0).get(), 0.0, y0 / 8.0);
            z = he.mul_rescale(z.get(), a.get());
            for (int i = 2; i <= k; i++) {
                if (z->level < 2) z = he.mcr(bootstrap_const(cx, z.get()).get(), 1.0);
                Ct gh = imag2(he.mul_rescale(z.get(), z.get()).get());
                z = he.mul_rescale(z.get(), he.add_const(he.neg(gh.get()).get(), pl.alpha(t, i - 1)).get());
            }
            if (z->level < 1) z = bootstrap_const(cx, z.get());
            // on z's level: no level spent on reading h out
            h = op_mul_int(cx, imag2(z.get()).get(), 2);
        } else {
        std::vector<double> vlo(slots, 0.0), vhi(slots, 0.0);
        for (int i = 0; i < half; i++) vlo[i] = y0;
        for (int i = half; i < slots; i++) vhi[i] = y0 / 2.0;
        Scratch sv{cx, {}};
        const double *d_vlo = upload_scaled(cx, sv, vlo, 1.0), *d_vhi = upload_scaled(cx, sv, vhi, 1.0);
        Ct a = he.add_const(he.mcr(x.get(), -y0 * y0 / 2.0).get(), pl.alpha(t, 0));
        Ct P = he.mul_plain_rescale(x.get(), d_vlo, slots);
        P = he.add_plain_vec(P.get(), d_vhi, slots);
        P = he.mul_rescale(P.get(), a.get());
        // one step maps the pair's scale s to s^3 / (q q'): a deviation from
        // Delta triples every step and a bootstrap keeps it, so each refresh
        // is followed by a multiplication by 1 that lands exactly on Delta
        // (the spare 13th level of a refresh: 6 steps still fit)
        for (int i = 2; i <= k; i++) {
            if (P->level < 2) P = he.mcr(bootstrap_ct(cx, P.get()).get(), 1.0);
            Ct Q = he.mul_rescale(P.get(), op_automorph(cx, P.get(), g_half).get());
            P = he.mul_rescale(P.get(), he.add_const(he.neg(Q.get()).get(), pl.alpha(t, i - 1)).get());
        }
        P = ensure(std::move(P), 1);
        for (int i = 0; i < slots; i++) vhi[i] = i < half ? 0.0 : 1.0;
        Ct hm = he.mul_plain_rescale(P.get(), upload_scaled(cx, sv, vhi, 1.0), slots);
        h = op_add(cx, hm.get(), op_automorph(cx, hm.get(), g_half).get(), false);
        if (shared) h = unpack_h(std::move(h));
        }
        if (!shared && ((rs.h_refresh[t] && h->level < Dp->level) || h->level < 1)) h = bootstrap_const(cx, h.get());
        h = ensure(std::move(h), 1);
        Dp = ensure(std::move(Dp), 1);
        Ct u = he.mul_rescale(Dp.get(), stream_bcast(cx, h.get(), cps).p);
        if (m) {
            Scratch s3{cx, {}};
            u = he.add_plain_vec(u.get(), upload_scaled(cx, s3, sh.mask, rn), slots, cps);
        } else {
            u = he.add_const(u.get(), rn);
        }
        u = ensure(std::move(u), power_depth(p));
        Y = he.power(u.get(), p);
    }
    Y = ensure(std::move(Y), 2);
    Ct Ssum = he.rotsum(stream_sum(cx, Y.get(), cps).p, sh.steps);
    if (!shared && Ssum->level < pl.d + 3) Ssum = bootstrap_const(cx, Ssum.get());  // the inverse's d + 2 levels
    Ct F;
    if (shared) {
        Ct Sp_ct = ensure(pack(ensure(std::move(Ssum), 1).get()), pl.d + 3);
        Ct Fp = ensure(inverse_goldschmidt(he, Sp_ct.get(), pl.kappa_f, pl.d), 2);
        F = ensure(unpack(Fp.get()), 1);
        Y = ensure(std::move(Y), 2);
    } else {
        F = inverse_goldschmidt(he, Ssum.get(), pl.kappa_f, pl.d);
    }
    F = stream_bcast(cx, std::move(F), cps);
    return he.mul_rescale(he.mcr(Y.get(), pl.kappa_f).get(), F.get());
}

}  // namespace he
