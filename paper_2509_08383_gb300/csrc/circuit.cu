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
#include <cmath>

#include "context.h"

namespace he {

namespace {

struct HE {
    he_ctx *cx;
    double delta;

    u64 q(int level) const { return cx->primes[level]; }

    Ct mcr(const he_ct *ct, double c, double target = -1) {
        if (target < 0) target = delta;
        double E = (target * (double)q(ct->level)) / ct->scale;
        double K = std::rint(c * E);
        Ct t = op_mul_intd(cx, ct, K, ct->scale * E);
        return op_rescale(cx, t.get());
    }
    Ct add_const(const he_ct *ct, double c) { return op_add_intd(cx, ct, std::rint(c * ct->scale)); }
    Ct neg(const he_ct *ct) { return op_mul_int(cx, ct, -1); }
    Ct mul_rescale(const he_ct *a, const he_ct *b) {
        Ct t = op_mul(cx, a, b);
        return op_rescale(cx, t.get());
    }
    // device slot vector (n_slots doubles) encoded at scale E, multiply, rescale
    Ct mul_plain_rescale(const he_ct *ct, const double *d_vec, int n_slots, double target = -1) {
        if (target < 0) target = delta;
        double E = (target * (double)q(ct->level)) / ct->scale;
        double *d_pt = cx->d_dbl + cx->N();
        encode_dev(cx, d_vec, nullptr, n_slots, E, d_pt);
        Ct t = op_mul_plain(cx, ct, d_pt, ct->scale * E);
        return op_rescale(cx, t.get());
    }
    Ct add_plain_vec(const he_ct *ct, const double *d_vec, int n_slots) {
        double *d_pt = cx->d_dbl + cx->N();
        encode_dev(cx, d_vec, nullptr, n_slots, ct->scale, d_pt);
        return op_add_plain(cx, ct, d_pt);
    }
    Ct rotsum(const he_ct *ct, int steps) {
        Ct cur = op_copy(cx, ct);
        for (int i = 0; i < steps; i++) {
            Ct r = op_automorph(cx, cur.get(), rot_galois(cx, (i64)1 << i));
            cur = op_add(cx, cur.get(), r.get(), false);
        }
        return cur;
    }
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

Ct invsqrt_goldschmidt(HE &he, const he_ct *V, double kappa, double y0, int k) {
    Ct a = he.add_const(he.mcr(V, -kappa * y0 * y0 / 2.0).get(), 1.5);
    Ct h = he.mcr(a.get(), y0 / 2.0);
    Ct g;
    if (k >= 2) g = he.mul_rescale(he.mcr(V, kappa * y0).get(), a.get());
    for (int i = 2; i <= k; i++) {
        a = he.add_const(he.neg(he.mul_rescale(g.get(), h.get()).get()).get(), 1.5);
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

int Plan::pad(int slots) const { return packing == 0 ? 0 : slots - n; }

Plan plan_from(const he_cutmax_plan *p) {
    if (!p || p->T < 1 || p->T > 64 || !p->power || !p->c || !p->k || !p->kappa || !p->y0 || p->n < 2)
        throw Error{HE_EINVAL, "invalid CutMax plan"};
    Plan pl;
    pl.n = (int)p->n;
    pl.packing = (int)p->packing;
    pl.T = (int)p->T;
    for (uint32_t t = 0; t < p->T; t++) {
        if (p->power[t] < 1 || p->k[t] < 1 || !(p->c[t] > 0) || !(p->kappa[t] > 0) || !(p->y0[t] > 0))
            throw Error{HE_ERANGE, "plan constants out of range"};
        pl.p.push_back((int)p->power[t]);
        pl.c.push_back(p->c[t]);
        pl.k.push_back((int)p->k[t]);
        pl.kappa.push_back(p->kappa[t]);
        pl.y0.push_back(p->y0[t]);
    }
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
    int steps = rotsum_steps(pl, cx->n / 2);
    for (int i = 0; i < steps; i++) galois.push_back(rot_galois(cx, (i64)1 << i));
}

Ct cutmax_ct(he_ctx *cx, const he_ct *in, const Plan &pl) {
    const int slots = cx->n / 2;
    if (pl.n > slots) throw Error{HE_EINVAL, "plan n exceeds the slot count"};
    if (pl.packing == 0 && (slots % pl.n != 0 || (pl.n & (pl.n - 1))))
        throw Error{HE_EINVAL, "replicated packing needs n a power of two dividing N/2"};
    int depth = pl.d + 3;
    for (int t = 0; t < pl.T; t++) depth += 2 + 2 * pl.k[t] + power_depth(pl.p[t]);
    if (depth > in->level) throw Error{HE_ELEVEL, "circuit depth " + std::to_string(depth) + " exceeds level " +
                                                   std::to_string(in->level)};
    HE he{cx, cx->delta};
    const int steps = rotsum_steps(pl, slots);
    const int m = pl.pad(slots);
    double *d_mask = nullptr;
    std::vector<double> mask;
    if (m) {
        // slot masks live in the third N-double scratch block: [mask | coef*mask]
        mask.assign(slots, 0.0);
        for (int i = 0; i < pl.n; i++) mask[i] = 1.0;
        d_mask = cx->d_dbl + 2 * cx->N();
        check_cuda(cudaMemcpyAsync(d_mask, mask.data(), slots * sizeof(double), cudaMemcpyHostToDevice, cx->stream),
                   "upload mask");
    }
    Ct Y = op_copy(cx, in);
    for (int t = 0; t < pl.T; t++) {
        Ct S = he.rotsum(Y.get(), steps);
        Ct D = op_add(cx, op_mul_int(cx, Y.get(), pl.n).get(), S.get(), true);
        Ct E = he.mul_rescale(D.get(), D.get());
        Ct V = he.rotsum(E.get(), steps);
        if (m) {
            Ct S2 = he.mul_rescale(S.get(), S.get());
            V = op_add(cx, V.get(), op_mul_int(cx, S2.get(), m).get(), true);
        }
        Ct h = invsqrt_goldschmidt(he, V.get(), pl.kappa[t], pl.y0[t], pl.k[t]);
        double coef = 2.0 * std::sqrt(pl.kappa[t] * pl.n) / pl.c[t];
        Ct Dp;
        if (m) {
            for (int i = 0; i < pl.n; i++) mask[i] = coef;
            double *d_cm = cx->d_dbl + 2 * cx->N() + slots;
            check_cuda(cudaMemcpyAsync(d_cm, mask.data(), slots * sizeof(double), cudaMemcpyHostToDevice, cx->stream),
                       "upload scaled mask");
            Dp = he.mul_plain_rescale(D.get(), d_cm, slots);
        } else {
            Dp = he.mcr(D.get(), coef);
        }
        Ct u = he.mul_rescale(Dp.get(), h.get());
        u = m ? he.add_plain_vec(u.get(), d_mask, slots) : he.add_const(u.get(), 1.0);
        Y = he.power(u.get(), pl.p[t]);
    }
    Ct S = he.rotsum(Y.get(), steps);
    Ct F = inverse_goldschmidt(he, S.get(), pl.kappa_f, pl.d);
    return he.mul_rescale(he.mcr(Y.get(), pl.kappa_f).get(), F.get());
}

}  // namespace he
