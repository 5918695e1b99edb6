// extern "C" entry points declared in include/he_cutmax.h.
#include <cmath>
#include <cstring>
#include <new>

#include "context.h"

using namespace he;

#define API_TRY \
    he::t_slot = cx->slot; \
    try {
#define API_CATCH(cx)                                                   \
    }                                                                   \
    catch (const Error &e) {                                            \
        if (cx) const_cast<he_ctx *>(cx)->err = e.msg;                  \
        return e.code;                                                  \
    }                                                                   \
    catch (const std::bad_alloc &) {                                    \
        if (cx) const_cast<he_ctx *>(cx)->err = "host allocation failed"; \
        return HE_ENOMEM;                                               \
    }                                                                   \
    return HE_OK;

static void sync(he_ctx *cx, const char *what) {
    check_cuda(cudaGetLastError(), what);
    check_cuda(cudaStreamSynchronize(cx->stream), what);
}
static void need(bool ok, const char *msg) {
    if (!ok) throw Error{HE_EINVAL, msg};
}
static void launched(he_ctx *cx, const char *what) { check_cuda(cudaGetLastError(), what); }
// every ciphertext argument must belong to the context it is used with
static void own(const he_ctx *cx, const he_ct *ct) {
    if (ct && ct->ctx != cx) throw Error{HE_EINVAL, "ciphertext does not belong to this context"};
}
// entry points that read or write one ciphertext's data refuse batches
static void single(const he_ct *ct) {
    if (ct && ct->batch != 1) throw Error{HE_EINVAL, "a batch here: take its members with he_batch_member"};
}

extern "C" {

int he_ctx_create(const he_params *params, void *dev_arena, size_t arena_bytes, he_ctx **out) {
    if (!out) return HE_EINVAL;
    he_ctx *cx = nullptr;
    try {
        cx = new he_ctx();
        ctx_init(cx, params, dev_arena, arena_bytes);
        *out = cx;
        return HE_OK;
    } catch (const Error &e) {
        delete cx;
        return e.code;
    } catch (const std::bad_alloc &) {
        delete cx;
        return HE_ENOMEM;
    }
}

void he_ctx_destroy(he_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    delete ctx;
}

int he_ctx_set_stream(he_ctx *cx, void *stream) {
    if (!cx) return HE_EINVAL;
    API_TRY
    sync(cx, "stream switch");
    cx->stream = (cudaStream_t)stream;
    upload_constants(cx->slot, cx->pc, cx->cdt, cx->n_cdt, cx->stream);
    sync(cx, "stream switch");
    API_CATCH(cx)
}

int he_ctx_primes(const he_ctx *cx, uint64_t *out) {
    if (!cx || !out) return HE_EINVAL;
    memcpy(out, cx->primes.data(), cx->primes.size() * 8);
    return HE_OK;
}

int he_ctx_memory(const he_ctx *cx, size_t *in_use, size_t *peak) {
    if (!cx) return HE_EINVAL;
    if (in_use) *in_use = cx->arena.in_use;
    if (peak) *peak = cx->arena.peak;
    return HE_OK;
}

const char *he_last_error(const he_ctx *cx) { return cx ? cx->err.c_str() : "null context"; }

uint64_t he_launch_count(void) { return (uint64_t)launch_count(); }

int he_profile_enable(int32_t kernel_class) {
    if (kernel_class < -1 || kernel_class > 3) return HE_EINVAL;
    prof_enable(kernel_class);
    return HE_OK;
}

int he_ledger_read(he_ctx *cx, uint64_t *ks_by_level, uint64_t *n_boot, int32_t reset) {
    if (!cx) return HE_EINVAL;
    if (ks_by_level) memcpy(ks_by_level, cx->ks_by_level, sizeof(uint64_t) * cx->nq);
    if (n_boot) *n_boot = cx->n_boot;
    if (reset) {
        memset(cx->ks_by_level, 0, sizeof(cx->ks_by_level));
        memset(cx->ops_by_level, 0, sizeof(cx->ops_by_level));
        cx->n_boot = 0;
    }
    return HE_OK;
}

int he_ledger_ops(const he_ctx *cx, uint32_t kind, uint64_t *by_level) {
    if (!cx || !by_level || kind > 3) return HE_EINVAL;
    memcpy(by_level, cx->ops_by_level[kind], sizeof(uint64_t) * cx->nq);
    return HE_OK;
}

int he_profile_read(int32_t kernel_class, uint64_t *launches, double *ms, double *bytes) {
    if (!launches || !ms || !bytes) return HE_EINVAL;
    unsigned long long l = 0;
    prof_read(kernel_class, &l, ms, bytes);
    *launches = l;
    return HE_OK;
}

int he_keygen_relin(he_ctx *cx) {
    if (!cx) return HE_EINVAL;
    API_TRY
    gen_relin_key(cx);
    sync(cx, "relinearisation key");
    API_CATCH(cx)
}

int he_keygen_galois(he_ctx *cx, uint64_t g) {
    if (!cx) return HE_EINVAL;
    API_TRY
    gen_galois_key(cx, g);
    sync(cx, "Galois key");
    API_CATCH(cx)
}

int he_keygen_rotations(he_ctx *cx, const int32_t *steps, size_t n) {
    if (!cx || (n && !steps)) return HE_EINVAL;
    API_TRY
    for (size_t i = 0; i < n; i++) gen_galois_key(cx, rot_galois(cx, steps[i]));
    sync(cx, "rotation keys");
    API_CATCH(cx)
}

int he_export_secret(const he_ctx *cx, int8_t *out) {
    if (!cx || !out) return HE_EINVAL;
    memcpy(out, cx->sk_host.data(), cx->N());
    return HE_OK;
}

int he_export_key(he_ctx *cx, uint64_t g, uint32_t digit, int32_t which, uint64_t *out) {
    if (!cx || !out) return HE_EINVAL;
    API_TRY
    const KeyDev *k = find_key(cx, g);
    if (!k) throw Error{HE_ENOKEY, "key not generated"};
    need((int)digit < cx->beta && (which == 0 || which == 1), "bad key digit / part");
    const int tot = cx->nq + cx->np;
    const size_t N = cx->N();
    Rows tmp = make_rows(cx->ks_acc, 0, tot, cx->nq, cx->nq);
    Rows src = make_rows(k->data + (size_t)(2 * digit + which) * tot * N, 0, tot, cx->nq, cx->nq);
    ew_copy(tmp, src, tot, cx->log_n, cx->stream);
    ew_mont(tmp, tot, 1, cx->log_n, cx->stream);  // keys are stored in Montgomery form
    ntt_inverse(tmp, tot, cx->tw, cx->log_n, cx->stream);
    check_cuda(cudaMemcpyAsync(out, cx->ks_acc, (size_t)tot * N * 8, cudaMemcpyDeviceToHost, cx->stream), "D2H");
    sync(cx, "export key");
    API_CATCH(cx)
}

int he_encode(he_ctx *cx, const double *re, const double *im, size_t n_slots, double scale, double *out) {
    if (!cx || !re || !out) return HE_EINVAL;
    API_TRY
    const size_t N = cx->N();
    need(n_slots <= N / 2, "more values than slots");
    double *d_re = cx->d_dbl, *d_im = im ? cx->d_dbl + N / 2 : nullptr, *d_out = cx->d_dbl + N;
    check_cuda(cudaMemcpyAsync(d_re, re, n_slots * 8, cudaMemcpyHostToDevice, cx->stream), "H2D");
    if (im) check_cuda(cudaMemcpyAsync(d_im, im, n_slots * 8, cudaMemcpyHostToDevice, cx->stream), "H2D");
    encode_dev(cx, d_re, d_im, (int)n_slots, scale, d_out);
    check_cuda(cudaMemcpyAsync(out, d_out, N * 8, cudaMemcpyDeviceToHost, cx->stream), "D2H");
    sync(cx, "encode");
    API_CATCH(cx)
}

int he_encrypt(he_ctx *cx, const double *re, const double *im, size_t n_slots, double scale, uint32_t ctr,
               int32_t level, he_ct **out) {
    if (!cx || !re || !out) return HE_EINVAL;
    API_TRY
    const size_t N = cx->N();
    need(n_slots <= N / 2, "more values than slots");
    double *d_re = cx->d_dbl, *d_im = im ? cx->d_dbl + N / 2 : nullptr, *d_pt = cx->d_dbl + N;
    check_cuda(cudaMemcpyAsync(d_re, re, n_slots * 8, cudaMemcpyHostToDevice, cx->stream), "H2D");
    if (im) check_cuda(cudaMemcpyAsync(d_im, im, n_slots * 8, cudaMemcpyHostToDevice, cx->stream), "H2D");
    encode_dev(cx, d_re, d_im, (int)n_slots, scale, d_pt);
    Ct ct(encrypt_dev(cx, d_pt, scale, ctr, level));
    sync(cx, "encrypt");
    *out = ct.release();
    API_CATCH(cx)
}

int he_encrypt_poly(he_ctx *cx, const double *m, double scale, uint32_t ctr, int32_t level, he_ct **out) {
    if (!cx || !m || !out) return HE_EINVAL;
    API_TRY
    double *d_pt = cx->d_dbl + cx->N();
    check_cuda(cudaMemcpyAsync(d_pt, m, cx->N() * 8, cudaMemcpyHostToDevice, cx->stream), "H2D");
    Ct ct(encrypt_dev(cx, d_pt, scale, ctr, level));
    sync(cx, "encrypt");
    *out = ct.release();
    API_CATCH(cx)
}

int he_decrypt(he_ctx *cx, const he_ct *ct, double *re, double *im, size_t n_slots) {
    if (!cx || !ct || !re) return HE_EINVAL;
    API_TRY
    own(cx, ct);
    single(ct);
    const size_t N = cx->N();
    need(n_slots <= N / 2, "more values than slots");
    double *d_c = cx->d_dbl + N, *d_re = cx->d_dbl, *d_im = cx->d_dbl + N / 2;
    decrypt_dev(cx, ct, d_c);
    decode_dev(cx, d_c, ct->scale, d_re, d_im);
    check_cuda(cudaMemcpyAsync(re, d_re, n_slots * 8, cudaMemcpyDeviceToHost, cx->stream), "D2H");
    if (im) check_cuda(cudaMemcpyAsync(im, d_im, n_slots * 8, cudaMemcpyDeviceToHost, cx->stream), "D2H");
    sync(cx, "decrypt");
    API_CATCH(cx)
}

int he_decrypt_poly(he_ctx *cx, const he_ct *ct, double *out) {
    if (!cx || !ct || !out) return HE_EINVAL;
    API_TRY
    own(cx, ct);
    single(ct);
    double *d_c = cx->d_dbl + cx->N();
    decrypt_dev(cx, ct, d_c);
    check_cuda(cudaMemcpyAsync(out, d_c, cx->N() * 8, cudaMemcpyDeviceToHost, cx->stream), "D2H");
    sync(cx, "decrypt");
    API_CATCH(cx)
}

int he_ct_export(he_ctx *cx, const he_ct *ct, uint64_t *out, size_t cap) {
    if (!cx || !ct || !out) return HE_EINVAL;
    API_TRY
    own(cx, ct);
    single(ct);
    const size_t N = cx->N(), m = (size_t)(ct->level + 1) * N;
    need(cap >= 2 * m, "export buffer too small");
    u64 *tmp = (u64 *)cx->arena.alloc(2 * m * 8);
    try {
        Rows t = make_rows(tmp, m, ct->level + 1, ct->level + 1, cx->nq);
        ew_copy(t, ct_rows(ct), 2 * (ct->level + 1), cx->log_n, cx->stream);
        ntt_inverse(t, 2 * (ct->level + 1), cx->tw, cx->log_n, cx->stream);
        check_cuda(cudaMemcpyAsync(out, tmp, 2 * m * 8, cudaMemcpyDeviceToHost, cx->stream), "D2H");
        sync(cx, "export");
    } catch (...) {
        cx->arena.release(tmp, 2 * m * 8);
        throw;
    }
    cx->arena.release(tmp, 2 * m * 8);
    API_CATCH(cx)
}

int he_ct_import(he_ctx *cx, const uint64_t *in, uint32_t level, double scale, he_ct **out) {
    if (!cx || !in || !out) return HE_EINVAL;
    API_TRY
    need((int)level < cx->nq, "level out of range");
    Ct ct(ct_alloc(cx, (int)level, scale));
    size_t m = (size_t)(level + 1) * cx->N();
    check_cuda(cudaMemcpyAsync(ct->d, in, 2 * m * 8, cudaMemcpyHostToDevice, cx->stream), "H2D");
    ntt_forward(ct_rows(ct.get()), 2 * (level + 1), cx->tw, cx->log_n, cx->stream);
    sync(cx, "import");
    *out = ct.release();
    API_CATCH(cx)
}

int he_ct_info(const he_ct *ct, uint32_t *level, double *scale) {
    if (!ct) return HE_EINVAL;
    if (level) *level = (uint32_t)ct->level;
    if (scale) *scale = ct->scale;
    return HE_OK;
}

int he_ct_device(const he_ct *ct, uint64_t **dev, size_t *poly_stride) {
    if (!ct || !ct->ctx) return HE_EINVAL;
    if (dev) *dev = ct->d;
    if (poly_stride) *poly_stride = (size_t)ct->cap * ct->ctx->N();
    return HE_OK;
}

void he_ct_free(he_ct *ct) { ct_release(ct); }

int he_batch_pack(he_ctx *cx, const he_ct *const *cts, size_t n, he_ct **out) {
    if (!cx || !cts || !out || n == 0) return HE_EINVAL;
    API_TRY
    for (size_t i = 0; i < n; i++) {
        need(cts[i] != nullptr, "null ciphertext");
        own(cx, cts[i]);
    }
    need(n <= 65536, "too many ciphertexts");
    Ct r = op_batch_pack(cx, cts, (int)n);
    launched(cx, "batch pack");
    *out = r.release();
    API_CATCH(cx)
}

int he_batch_member(he_ctx *cx, const he_ct *batch, uint32_t i, he_ct **out) {
    if (!cx || !batch || !out) return HE_EINVAL;
    API_TRY
    own(cx, batch);
    Ct r = op_batch_member(cx, batch, (int)i);
    launched(cx, "batch member");
    *out = r.release();
    API_CATCH(cx)
}

int he_batch_size(const he_ct *ct, uint32_t *n) {
    if (!ct || !n) return HE_EINVAL;
    *n = (uint32_t)ct->batch;
    return HE_OK;
}

#define UNARY_OP(name, expr)                                     \
    int name {                                                   \
        if (!cx || !a || !out) return HE_EINVAL;                 \
        API_TRY                                                  \
        own(cx, a);                                              \
        Ct res_ = expr;                                          \
        launched(cx, #name);                                     \
        *out = res_.release();                                   \
        API_CATCH(cx)                                            \
    }

UNARY_OP(he_add(he_ctx *cx, const he_ct *a, const he_ct *b, he_ct **out), (need(b, "null b"), own(cx, b), op_add(cx, a, b, false)))
UNARY_OP(he_sub(he_ctx *cx, const he_ct *a, const he_ct *b, he_ct **out), (need(b, "null b"), own(cx, b), op_add(cx, a, b, true)))
UNARY_OP(he_mul_int(he_ctx *cx, const he_ct *a, int64_t k, he_ct **out), op_mul_int(cx, a, k))
UNARY_OP(he_mul(he_ctx *cx, const he_ct *a, const he_ct *b, he_ct **out), (need(b, "null b"), own(cx, b), op_mul(cx, a, b)))
UNARY_OP(he_mul_rescale(he_ctx *cx, const he_ct *a, const he_ct *b, he_ct **out), (need(b, "null b"), own(cx, b), op_mul_rescale(cx, a, b)))
UNARY_OP(he_rescale(he_ctx *cx, const he_ct *a, he_ct **out), op_rescale(cx, a))
UNARY_OP(he_drop(he_ctx *cx, const he_ct *a, uint32_t level, he_ct **out), op_drop(cx, a, (int)level))
UNARY_OP(he_rotate(he_ctx *cx, const he_ct *a, int32_t r, he_ct **out), op_automorph(cx, a, rot_galois(cx, r)))
UNARY_OP(he_conjugate(he_ctx *cx, const he_ct *a, he_ct **out), op_automorph(cx, a, 2 * cx->N() - 1))
UNARY_OP(he_automorphism(he_ctx *cx, const he_ct *a, uint64_t g, he_ct **out), op_automorph(cx, a, g))
UNARY_OP(he_mul_monomial(he_ctx *cx, const he_ct *a, uint64_t e, he_ct **out), op_mul_monomial(cx, a, e))

int he_mul_const(he_ctx *cx, const he_ct *a, double c, double target, he_ct **out) {
    if (!cx || !a || !out) return HE_EINVAL;
    API_TRY
    own(cx, a);
    double E = (target * (double)cx->primes[a->level]) / a->scale;
    double K = std::rint(c * E);
    Ct t = op_mul_intd(cx, a, K, a->scale * E);
    Ct r = op_rescale(cx, t.get());
    launched(cx, "mul_const");
    *out = r.release();
    API_CATCH(cx)
}

int he_add_const(he_ctx *cx, const he_ct *a, double c, he_ct **out) {
    if (!cx || !a || !out) return HE_EINVAL;
    API_TRY
    own(cx, a);
    Ct r = op_add_intd(cx, a, std::rint(c * a->scale));
    launched(cx, "add_const");
    *out = r.release();
    API_CATCH(cx)
}

int he_rotsum(he_ctx *cx, const he_ct *a, uint32_t steps, he_ct **out) {
    if (!cx || !a || !out) return HE_EINVAL;
    API_TRY
    own(cx, a);
    need(steps < 32, "too many rotate-and-sum steps");
    Ct cur = op_rotsum(cx, a, (int)steps);
    launched(cx, "rotsum");
    *out = cur.release();
    API_CATCH(cx)
}

int he_rotsum_stage(he_ctx *cx, const he_ct *a, const int32_t *rots, size_t n_rots, he_ct **out) {
    if (!cx || !a || !rots || !out) return HE_EINVAL;
    API_TRY
    own(cx, a);
    need(n_rots >= 1 && n_rots <= 15, "a hoisted stage takes 1..15 rotations");
    std::vector<i64> r(rots, rots + n_rots);
    Ct res = op_rotsum_stage(cx, a, r);
    launched(cx, "rotsum stage");
    *out = res.release();
    API_CATCH(cx)
}

int he_ctx_set_rotsum_radix(he_ctx *cx, uint32_t log2_radix) {
    if (!cx) return HE_EINVAL;
    if (log2_radix < 1 || log2_radix > 4) {
        cx->err = "rotate-and-sum radix must be 2, 4, 8 or 16 (log2 1..4)";
        return HE_EINVAL;
    }
    if (cx->rotsum_log_radix != (int)log2_radix) cx->gen++;
    cx->rotsum_log_radix = (int)log2_radix;
    return HE_OK;
}

int he_keyswitch_raw(he_ctx *cx, const uint64_t *d, uint32_t level, uint64_t g, uint64_t *out0, uint64_t *out1) {
    if (!cx || !d || !out0 || !out1) return HE_EINVAL;
    API_TRY
    need((int)level < cx->nq, "level out of range");
    const KeyDev *k = find_key(cx, g);
    if (!k) throw Error{HE_ENOKEY, "key not generated"};
    const size_t N = cx->N(), m = (size_t)(level + 1) * N;
    int l = (int)level;
    check_cuda(cudaMemcpyAsync(cx->sc_a, d, m * 8, cudaMemcpyHostToDevice, cx->stream), "H2D");
    Rows in = make_rows(cx->sc_a, 0, l + 1, l + 1, cx->nq);
    ntt_forward(in, l + 1, cx->tw, cx->log_n, cx->stream);
    Rows o = make_rows(cx->sc_b, m, l + 1, l + 1, cx->nq);
    keyswitch(cx, cx->sc_a, l, *k, o, o, 0);
    ntt_inverse(o, 2 * (l + 1), cx->tw, cx->log_n, cx->stream);
    check_cuda(cudaMemcpyAsync(out0, cx->sc_b, m * 8, cudaMemcpyDeviceToHost, cx->stream), "D2H");
    check_cuda(cudaMemcpyAsync(out1, cx->sc_b + m, m * 8, cudaMemcpyDeviceToHost, cx->stream), "D2H");
    sync(cx, "keyswitch");
    API_CATCH(cx)
}

int he_moddown_raw(he_ctx *cx, const uint64_t *acc0, const uint64_t *acc1, uint32_t level, uint64_t *out0,
                   uint64_t *out1) {
    if (!cx || !acc0 || !acc1 || !out0 || !out1) return HE_EINVAL;
    API_TRY
    need((int)level < cx->nq, "level out of range");
    const int l = (int)level, ne = cx->lv[l].n_ext;
    const size_t N = cx->N(), m = (size_t)(l + 1) * N, me = (size_t)ne * N;
    check_cuda(cudaMemcpyAsync(cx->ks_acc, acc0, me * 8, cudaMemcpyHostToDevice, cx->stream), "H2D");
    check_cuda(cudaMemcpyAsync(cx->ks_acc + me, acc1, me * 8, cudaMemcpyHostToDevice, cx->stream), "H2D");
    ntt_forward(make_rows(cx->ks_acc, me, ne, l + 1, cx->nq), 2 * ne, cx->tw, cx->log_n, cx->stream);
    Rows o = make_rows(cx->sc_b, m, l + 1, l + 1, cx->nq);
    moddown(cx, cx->ks_acc, l, o, o, 0);
    ntt_inverse(o, 2 * (l + 1), cx->tw, cx->log_n, cx->stream);
    check_cuda(cudaMemcpyAsync(out0, cx->sc_b, m * 8, cudaMemcpyDeviceToHost, cx->stream), "D2H");
    check_cuda(cudaMemcpyAsync(out1, cx->sc_b + m, m * 8, cudaMemcpyDeviceToHost, cx->stream), "D2H");
    sync(cx, "moddown");
    API_CATCH(cx)
}

int he_ntt_device(he_ctx *cx, uint64_t *data, uint32_t n_limbs, uint32_t prime_idx0, int32_t inverse) {
    if (!cx || !data) return HE_EINVAL;
    API_TRY
    need(prime_idx0 + n_limbs <= (uint32_t)(cx->nq + cx->np), "prime range out of bounds");
    Rows r = make_rows(data, 0, (int)n_limbs, (int)n_limbs, cx->nq, (int)prime_idx0);
    if (inverse) ntt_inverse(r, (int)n_limbs, cx->tw, cx->log_n, cx->stream);
    else ntt_forward(r, (int)n_limbs, cx->tw, cx->log_n, cx->stream);
    launched(cx, "ntt");
    API_CATCH(cx)
}

int he_bootstrap_prepare(he_ctx *cx, uint32_t K, uint32_t r, uint32_t d) {
    if (!cx) return HE_EINVAL;
    API_TRY
    boot_prepare(cx, (int)K, (int)r, (int)d);
    sync(cx, "bootstrap keys");
    API_CATCH(cx)
}

int he_bootstrap(he_ctx *cx, const he_ct *in, he_ct **out) {
    if (!cx || !in || !out) return HE_EINVAL;
    API_TRY
    own(cx, in);
    Ct r = bootstrap_ct(cx, in);
    launched(cx, "bootstrap");
    *out = r.release();
    API_CATCH(cx)
}

int he_bootstrap_stage(he_ctx *cx, const he_ct *in, int32_t stage, he_ct **out) {
    if (!cx || !in || !out) return HE_EINVAL;
    API_TRY
    own(cx, in);
    Ct r = bootstrap_stage(cx, in, stage);
    launched(cx, "bootstrap stage");
    *out = r.release();
    API_CATCH(cx)
}

int he_bootstrap_const(he_ctx *cx, const he_ct *in, he_ct **out) {
    if (!cx || !in || !out) return HE_EINVAL;
    API_TRY
    own(cx, in);
    Ct r = bootstrap_const(cx, in);
    launched(cx, "constant bootstrap");
    *out = r.release();
    API_CATCH(cx)
}

int he_learn_invsqrt(he_ctx *cx, const float *x, size_t n, uint32_t steps, float lr, uint64_t seed, double *abc,
                     double *loss) {
    if (!cx || !x || !abc) return HE_EINVAL;
    API_TRY
    need(lr > 0.f && std::isfinite(lr), "learning rate must be positive");
    learn_invsqrt(cx, x, n, (int)steps, lr, seed, abc, loss);
    launched(cx, "invsqrt training");
    API_CATCH(cx)
}

int he_cutmax_prepare(he_ctx *cx, const he_cutmax_plan *plan) {
    if (!cx) return HE_EINVAL;
    API_TRY
    Plan pl = plan_from(plan);
    std::vector<u64> gs;
    plan_keys(cx, pl, gs);
    gen_relin_key(cx);
    for (u64 g : gs) gen_galois_key(cx, g);
    sync(cx, "cutmax keys");
    API_CATCH(cx)
}

int cutmax(he_ctx *cx, const he_ct *in, const he_cutmax_plan *plan, he_ct **out) {
    if (!cx || !in || !out) return HE_EINVAL;
    API_TRY
    own(cx, in);
    Plan pl = plan_from(plan);
    Ct r = cx->use_graphs ? cutmax_graph(cx, in, pl) : cutmax_ct(cx, in, pl);
    launched(cx, "cutmax");
    *out = r.release();
    API_CATCH(cx)
}

int he_cutmax_graph(he_ctx *cx, const he_ct *in, const he_cutmax_plan *plan, he_ct **out) {
    if (!cx || !in || !out) return HE_EINVAL;
    API_TRY
    own(cx, in);
    Plan pl = plan_from(plan);
    Ct r = cutmax_graph(cx, in, pl);
    launched(cx, "cutmax graph");
    *out = r.release();
    API_CATCH(cx)
}

int he_cutmax_graph_stats(he_ctx *cx, uint64_t *captured, uint64_t *replayed, uint64_t *direct) {
    if (!cx) return HE_EINVAL;
    if (captured) *captured = cx->graph_stats[0];
    if (replayed) *replayed = cx->graph_stats[1];
    if (direct) *direct = cx->graph_stats[2];
    return HE_OK;
}

int he_ctx_set_graphs(he_ctx *cx, int32_t on) {
    if (!cx) return HE_EINVAL;
    cx->use_graphs = on != 0;
    return HE_OK;
}

int he_cutmax_graph_clear(he_ctx *cx) {
    if (!cx) return HE_EINVAL;
    API_TRY
    graphs_release(cx);
    API_CATCH(cx)
}

int he_beta_noise(he_ctx *cx, const he_ct *u, double alpha, uint32_t degree, he_ct **out) {
    if (!cx || !u || !out) return HE_EINVAL;
    API_TRY
    own(cx, u);
    Ct r = beta_noise(cx, u, alpha, (int)degree);
    launched(cx, "beta noise");
    *out = r.release();
    API_CATCH(cx)
}

// alpha = ln(1-q)/ln(top_p) (Lemma 2 / Observation 1; q = 0 reads as q = top_p)
static double nucleus_alpha(double top_p, double q) {
    need(top_p > 0.0 && top_p < 1.0, "top-p mass must lie in (0, 1)");
    need(q >= 0.0 && q < 1.0, "q must lie in [0, 1) (0: q = top_p)");
    const double qq = q > 0.0 ? q : top_p;
    const double alpha = std::log(1.0 - qq) / std::log(top_p);
    need(std::isfinite(alpha) && alpha > 0.0, "alpha = ln(1-q)/ln(p) must be positive");
    return alpha;
}

int nucleus_sample_groups(he_ctx *cx, const he_ct *logits, const double *top_p, uint32_t n_groups, double q,
                          const he_ct *rand_ct, int32_t rand_kind, const he_cutmax_plan *plan, he_ct **out) {
    if (!cx || !logits || !rand_ct || !out || !top_p) return HE_EINVAL;
    API_TRY
    own(cx, logits);
    own(cx, rand_ct);
    need(n_groups >= 1, "at least one group");
    need(rand_kind == HE_RAND_BETA || rand_kind == HE_RAND_UNIFORM, "unknown noise kind");
    Plan pl = plan_from(plan);
    const int B = logits->batch, G = (int)n_groups;
    need(rand_ct->batch == B, "logits and noise batches differ in size");
    need(B % G == 0 && (B / G) % pl.cps == 0, "the batch does not split into whole groups of streams");
    std::vector<double> alpha(G);
    for (int j = 0; j < G; j++) alpha[j] = nucleus_alpha(top_p[j], q);
    Ct noise;
    if (rand_kind == HE_RAND_UNIFORM) {
        const int per = B / G;
        std::vector<Ct> parts;
        std::vector<const he_ct *> ptrs;
        for (int j = 0; j < G; j++) {
            Ct u = G == 1 ? Ct() : op_batch_member(cx, rand_ct, j * per, per);
            parts.push_back(beta_noise(cx, u ? u.get() : rand_ct, alpha[j], HE_NUCLEUS_DEGREE));
            ptrs.push_back(parts.back().get());
        }
        noise = G == 1 ? std::move(parts[0]) : op_batch_pack(cx, ptrs.data(), G);
    }
    Ct x = op_add(cx, logits, noise ? noise.get() : rand_ct, false);
    Ct r = cx->use_graphs ? cutmax_graph(cx, x.get(), pl) : cutmax_ct(cx, x.get(), pl);
    launched(cx, "nucleus_sample_groups");
    *out = r.release();
    API_CATCH(cx)
}

int nucleus_sample(he_ctx *cx, const he_ct *logits, double top_p, double q, const he_ct *rand_ct, int32_t rand_kind,
                   const he_cutmax_plan *plan, he_ct **out) {
    return nucleus_sample_groups(cx, logits, &top_p, 1, q, rand_ct, rand_kind, plan, out);
}

}  // extern "C"
