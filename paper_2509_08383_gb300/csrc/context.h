// Host-side state of a CKKS context and the homomorphic evaluator.
#pragma once
#include <map>
#include <memory>
#include <string>
#include <unordered_set>
#include <vector>

#include "../../include/he_cutmax.h"
#include "kernels.h"

namespace he {
struct Boot;

// Sub-allocator over one device buffer; exact-size reuse of freed blocks.
struct Arena {
    char *base = nullptr;
    size_t cap = 0, top = 0, in_use = 0, peak = 0;
    bool owned = false;
    std::multimap<size_t, size_t> free_blocks;  // size -> offset
    void *alloc(size_t bytes);
    void release(void *p, size_t bytes);
};

struct KeyDev {
    u64 g;       // Galois element, 0 = relinearisation
    u64 *data;   // [beta][2][nq+np][N], NTT form
    size_t bytes;
};

enum Domain : u32 { DOM_SECRET = 1, DOM_ERROR = 2, DOM_UNIFORM = 3, DOM_KEY_A = 4, DOM_KEY_E = 5, DOM_SPARSE = 6 };

struct LevelTabs {
    // key-switch basis at this level: n_ext = l+1+K rows per polynomial
    int n_ext = 0, beta = 0;
    std::vector<int> digit_lo, digit_cnt, digit_off, digit_nout;  // per digit
    int2 *desc = nullptr;         // all digits' extension rows (device)
    int n_desc = 0;
    std::vector<BConvTab> modup;  // per digit
    ScalarTab ql_inv;             // q_l^-1 mod q_i, i < l (for rescale)
};

}  // namespace he

struct he_ct {
    he_ctx *ctx;    // null once the owning context has been destroyed
    int level;
    double scale;
    u64 *d;     // c0 limbs then c1 limbs
    int cap;        // limbs allocated per polynomial
    size_t bytes;
};

struct he_ctx {
    int slot = -1;  // constant-memory slot (see PrimeConsts)
    int log_n = 0, n = 0, nq = 0, np = 0, dnum = 0, alpha = 0, beta = 0, h = 0;
    double delta = 0, sigma = 0;
    u64 seed = 0;
    bool boot = false;
    std::vector<u64> primes;
    PrimeConsts pc;
    u64 cdt[19];
    int n_cdt = 19;
    cudaStream_t stream = 0;
    he::Arena arena;
    std::string err;
    // tables
    u64 *d_tw = nullptr;
    he::NttTables tw;
    std::vector<int8_t> sk_host;
    int8_t *d_sk_small = nullptr;
    u64 *d_sk_ntt = nullptr;           // [(nq+np)][N]
    std::vector<he::LevelTabs> lv;         // per level l
    u64 *d_tabs = nullptr;             // storage of all BConv tables
    he::BConvTab moddown;                  // n_in = np, stride = nq
    he::ScalarTab p_inv;                   // P^-1 mod q_i
    he::ScalarTab p_mod;                   // P mod q_i
    int *d_slot_l = nullptr;
    he::Cplx *d_fft = nullptr;
    double *d_dbl = nullptr;               // 3 * N doubles of scratch
    // key-switch scratch
    u64 *ks_coef = nullptr, *ks_ext = nullptr, *ks_acc = nullptr, *ks_conv = nullptr;
    u64 *sc_a = nullptr, *sc_b = nullptr;  // 2*(nq+np) rows each, general scratch
    std::vector<he::KeyDev> keys;
    std::unordered_set<he_ct *> live;      // ciphertexts handed out and not yet freed
    std::shared_ptr<he::Boot> boot_state;  // bootstrapping tables, when prepared
    // operation ledger: key switches by level, bootstraps
    uint64_t ks_by_level[HE_MAX_PRIMES] = {0};
    uint64_t n_boot = 0;

    ~he_ctx();
    size_t N() const { return (size_t)n; }
};

namespace he {

// RAII owner of a ciphertext
struct CtDel { void operator()(he_ct *c) const; };
using Ct = std::unique_ptr<he_ct, CtDel>;

struct Error { int code; std::string msg; };

// ---- context / memory
void ctx_init(he_ctx *cx, const he_params *p, void *arena, size_t arena_bytes);  // throws Error
he_ct *ct_alloc(he_ctx *cx, int level, double scale);
void ct_release(he_ct *ct);
Rows ct_rows(const he_ct *ct, int level = -1);  // both polynomials, limbs 0..level
u64 *ct_poly(const he_ct *ct, int k);
ScalarTab scalar_int(he_ctx *cx, i64 k, int n_limbs);
ScalarTab scalar_intd(he_ctx *cx, double K, int n_limbs);
u64 intd_mod_host(double x, u64 q);
u64 mulmod_host(u64 a, u64 b, u64 q);
u64 powmod_host(u64 a, u64 e, u64 q);
u64 shoup_host(u64 w, u64 q);

// ---- keys
const KeyDev *find_key(he_ctx *cx, u64 g);
void gen_relin_key(he_ctx *cx);
void gen_galois_key(he_ctx *cx, u64 g);
u64 rot_galois(he_ctx *cx, i64 r);

// ---- encryption
he_ct *encrypt_dev(he_ctx *cx, const double *d_pt, double scale, u32 ctr, int level);
void decrypt_dev(he_ctx *cx, const he_ct *ct, double *d_out);   // N centred values on device
void encode_dev(he_ctx *cx, const double *d_re, const double *d_im, int n_slots, double scale, double *d_out);
void decode_dev(he_ctx *cx, const double *d_coeff, double scale, double *d_re, double *d_im);

// ---- evaluator (all inputs are NTT form, outputs new ciphertexts)
Ct op_add(he_ctx *cx, const he_ct *a, const he_ct *b, bool sub);
Ct op_mul_int(he_ctx *cx, const he_ct *a, i64 k);
Ct op_mul_intd(he_ctx *cx, const he_ct *a, double K, double scale_out);
Ct op_add_intd(he_ctx *cx, const he_ct *a, double K);
Ct op_mul_plain(he_ctx *cx, const he_ct *a, const double *d_pt, double scale_out);
Ct op_add_plain(he_ctx *cx, const he_ct *a, const double *d_pt);
Ct op_mul(he_ctx *cx, const he_ct *a, const he_ct *b);
Ct op_rescale(he_ctx *cx, const he_ct *a);
Ct op_drop(he_ctx *cx, const he_ct *a, int level);
Ct op_automorph(he_ctx *cx, const he_ct *a, u64 g);
Ct op_mod_raise(he_ctx *cx, const he_ct *a, int level);
Ct op_mul_monomial(he_ctx *cx, const he_ct *a, u64 e);
Ct op_copy(he_ctx *cx, const he_ct *a);
// raw hybrid key switch: d (NTT form, limbs 0..l) -> out (2 polys, NTT form),
// add_mask bit k: out poly k += add poly k
void keyswitch(he_ctx *cx, const u64 *d_ntt, int l, const KeyDev &key, const Rows &out, const Rows &add, int add_mask);
// the two halves of a key switch, for rotations that share one ModUp
void modup(he_ctx *cx, const u64 *d_ntt, int l, u64 *ext);
void ks_inner(he_ctx *cx, const u64 *d_ntt, const u64 *ext, int l, const KeyDev &key, u64 galois, u64 *acc);
void moddown(he_ctx *cx, u64 *acc, int l, const Rows &out, const Rows &add, int add_mask);
void keyswitch_ext(he_ctx *cx, const u64 *d_ntt, const u64 *ext, int l, const KeyDev &key, u64 galois,
                   const Rows &out, const Rows &add, int add_mask);

// ---- circuits (circuit.cu)
struct Plan {
    int n, packing, T;
    std::vector<int> p, k;
    std::vector<double> c, kappa, y0, norm;
    int d;
    double kappa_f;
    bool bootstrap;
    int pad(int slots) const;
};
Plan plan_from(const he_cutmax_plan *p);
void plan_keys(he_ctx *cx, const Plan &pl, std::vector<u64> &galois);
Ct cutmax_ct(he_ctx *cx, const he_ct *in, const Plan &pl);
void boot_prepare(he_ctx *cx, int K, int r, int d);
Ct bootstrap_ct(he_ctx *cx, const he_ct *in);
Ct bootstrap_stage(he_ctx *cx, const he_ct *in, int stage);

void check_cuda(cudaError_t e, const char *what);
void release_slot(int slot);

}  // namespace he
