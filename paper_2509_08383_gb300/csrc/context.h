// Host-side state of a CKKS context and the homomorphic evaluator.
#pragma once
#include <map>
#include <memory>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/he_cutmax.h"
#include "arena.h"
#include "kernels.h"

namespace he {
struct Boot;
struct CutmaxGraph;

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
    // product with its rescale: rounded division by M = q_l P, from the basis
    // {q_l, p_0..p_(K-1)} to q_0..q_(l-1) (l >= 1; n_in = 0: not available)
    BConvTab mulres;
    ScalarTab mulres_inv;         // M^-1 mod q_i, i < l
};

}  // namespace he

// `batch` ciphertexts of one level and scale stored back to back: member m's
// polynomial k (c0, c1) holds its limbs at d + (2m + k) cap N.
struct he_ct {
    he_ctx *ctx;    // null once the owning context has been destroyed
    int level;
    double scale;
    u64 *d;
    int cap;        // limbs allocated per polynomial
    int batch = 1;  // ciphertexts held
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
    // operation ledger: key switches by level, bootstraps, and the other
    // ciphertext operations by level (he_ledger_ops)
    uint64_t ks_by_level[HE_MAX_PRIMES] = {0};
    uint64_t n_boot = 0;
    uint64_t ops_by_level[4][HE_MAX_PRIMES] = {{0}};  // rescales, tensor products, plaintext products, additions
    int rotsum_log_radix = 3;              // rotate-and-sum stages of 2^this slots (he_ctx_set_rotsum_radix)
    // device copies of the circuits' constant slot vectors (masks, constants),
    // keyed by content; they live as long as the context
    struct ConstVec { double *d; std::vector<double> host; };
    std::unordered_multimap<uint64_t, ConstVec> const_cache;
    std::unordered_set<const double *> const_ptrs;  // the device vectors of const_cache
    // their encodings (encoded_plain): vector, scale E, level -> NTT-form rows
    struct PlainVec {
        const double *re, *im;
        int n_slots, n_pt, level;
        double E;
        u64 *d;
        size_t bytes;
    };
    std::vector<PlainVec> plain_cache;
    // CutMax calls captured as CUDA graphs (graph.cu); `gen` changes whenever
    // something a graph holds by address may change (bootstrap tables,
    // rotate-and-sum radix), which retires every graph
    std::vector<std::shared_ptr<he::CutmaxGraph>> graphs;
    uint64_t gen = 0;
    bool capturing = false;                // a CUDA graph capture is under way
    bool use_graphs = false;               // cutmax and nucleus_sample go through cutmax_graph
    uint64_t graph_stats[3] = {0, 0, 0};   // captured, replayed, run directly after a failed capture
    uint64_t graph_calls = 0;              // calls of cutmax_graph (the graphs' use clock)

    ~he_ctx();
    size_t N() const { return (size_t)n; }
};

namespace he {

// RAII owner of a ciphertext
struct CtDel { void operator()(he_ct *c) const; };
using Ct = std::unique_ptr<he_ct, CtDel>;

// arena buffers released on every exit path
struct Scratch {
    he_ctx *cx;
    std::vector<std::pair<u64 *, size_t>> v;
    u64 *get(size_t words);
    ~Scratch();
};

// ---- context / memory
void ctx_init(he_ctx *cx, const he_params *p, void *arena, size_t arena_bytes);  // throws Error
he_ct *ct_alloc(he_ctx *cx, int level, double scale, int batch = 1);
void ct_release(he_ct *ct);
Rows ct_rows(const he_ct *ct, int level = -1);  // every polynomial of every member, limbs 0..level
u64 *ct_poly(const he_ct *ct, int k);           // member 0's polynomial k
Rows ct_polys(const he_ct *ct, int k, int level = -1);  // polynomial k of every member
size_t ct_member_stride(const he_ct *ct);
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
// n_pt plaintexts (n_pt x N integer-valued doubles); member m uses plaintext m % n_pt
Ct op_mul_plain(he_ctx *cx, const he_ct *a, const double *d_pt, double scale_out, int n_pt = 1);
Ct op_add_plain(he_ctx *cx, const he_ct *a, const double *d_pt, int n_pt = 1);
// the same with a plaintext already in NTT form on limbs 0..level of `a`
// (n_pt of them back to back, member m takes m % n_pt)
Ct op_mul_plain_ntt(he_ctx *cx, const he_ct *a, const u64 *pt, double scale_out, int n_pt = 1);
Ct op_add_plain_ntt(he_ctx *cx, const he_ct *a, const u64 *pt, int n_pt = 1);
// NTT-form plaintext of device_const slot vectors encoded at scale E on limbs
// 0..l, cached per context; nullptr when it cannot be cached (see context.cu)
const u64 *encoded_plain(he_ctx *cx, const double *re, const double *im, int n_slots, int n_pt, double E, int l);
Ct op_mul(he_ctx *cx, const he_ct *a, const he_ct *b);
// product, relinearisation and rescale with one rounding: round((P d + acc) / (q_l P))
Ct op_mul_rescale(he_ctx *cx, const he_ct *a, const he_ct *b);
Ct op_rescale(he_ctx *cx, const he_ct *a);
// rescale(K a) in one pass: the product by the integer K (rint of a double,
// any size) folded into the rescale's lift and finish; scale_mid = a's scale
// times K's encoding scale
Ct op_mul_intd_rescale(he_ctx *cx, const he_ct *a, double K, double scale_mid);
Ct op_drop(he_ctx *cx, const he_ct *a, int level);
Ct op_automorph(he_ctx *cx, const he_ct *a, u64 g);
Ct op_mod_raise(he_ctx *cx, const he_ct *a, int level);
Ct op_mul_monomial(he_ctx *cx, const he_ct *a, u64 e);
Ct op_copy(he_ctx *cx, const he_ct *a);
// batches: members of several ciphertexts packed back to back; members
// [i, i+count) of a batch; groups of g consecutive members summed, or every
// member repeated g times
Ct op_batch_pack(he_ctx *cx, const he_ct *const *cts, int n);
Ct op_batch_member(he_ctx *cx, const he_ct *a, int i, int count = 1);
Ct op_group(he_ctx *cx, const he_ct *a, int g, bool sum);
// raw hybrid key switch of B polynomials (member m's limbs 0..l at d_ntt +
// m*d_stride, NTT form) -> out (2B polys, NTT form); add_mask bit k: out
// polynomial k of every member += the matching add polynomial
void keyswitch(he_ctx *cx, const u64 *d_ntt, int l, const KeyDev &key, const Rows &out, const Rows &add, int add_mask,
               int B = 1, size_t d_stride = 0);
// the pieces of a key switch, for rotations that share one ModUp; ext holds
// ks_ext_words(l) and acc ks_acc_words(l) words per member
size_t ks_ext_words(he_ctx *cx, int l);
size_t ks_acc_words(he_ctx *cx, int l);
void modup(he_ctx *cx, const u64 *d_ntt, int l, u64 *ext, int B = 1, size_t d_stride = 0);
// (lift, one member only: + P * d_k on the Q rows of output polynomial k, d_k
// at lift + k lift_poly)
void ks_inner(he_ctx *cx, const u64 *d_ntt, const u64 *ext, int l, const KeyDev &key, u64 galois, u64 *acc,
              int B = 1, size_t d_stride = 0, const u64 *lift = nullptr, size_t lift_poly = 0);
void moddown(he_ctx *cx, u64 *acc, int l, const Rows &out, const Rows &add, int add_mask, int B = 1);
void keyswitch_ext(he_ctx *cx, const u64 *d_ntt, const u64 *ext, int l, const KeyDev &key, u64 galois,
                   const Rows &out, const Rows &add, int add_mask, int B = 1, size_t d_stride = 0);
// rotate-and-sum (App. D) over 2^steps consecutive slots in hoisted stages:
// stage i covers doublings [i L, min((i+1) L, steps)) (L = the context's
// log2 radix) and adds to x its rotations by r 2^(i L), 0 < r < 2^len, all
// through one ModUp of c1 and one ModDown of the summed inner products
std::vector<std::vector<i64>> rotsum_stages(int steps, int log_radix);
Ct op_rotsum_stage(he_ctx *cx, const he_ct *a, const std::vector<i64> &rots);
Ct op_rotsum(he_ctx *cx, const he_ct *a, int steps);

// ---- circuits (circuit.cu)
struct Plan {
    int n, packing, T;
    std::vector<int> p, k;
    std::vector<double> c, kappa, y0, norm;
    int d;
    double kappa_f;
    bool bootstrap;
    int cps = 1;  // ciphertexts per stream
    bool shared = false;  // batched streams share the scalar chains (see he_cutmax_plan)
    std::vector<double> lq;  // [T][3] learned quadratics (used where k[t] == 0)
    // additive constant of each Goldschmidt step (3/2 unless the plan relaxes
    // them): iteration t's k[t] steps start at relax_at[t]
    std::vector<double> relax;
    std::vector<int> relax_at;
    double alpha(int t, int i) const { return relax[(size_t)relax_at[t] + i]; }
    int pad(int slots) const;
};
Plan plan_from(const he_cutmax_plan *p);
void plan_keys(he_ctx *cx, const Plan &pl, std::vector<u64> &galois);
Ct cutmax_ct(he_ctx *cx, const he_ct *in, const Plan &pl);
// CutMax through a CUDA graph captured per plan and input shape (graph.cu)
Ct cutmax_graph(he_ctx *cx, const he_ct *in, const Plan &pl);
void graphs_release(he_ctx *cx);
const double *device_const(he_ctx *cx, const std::vector<double> &v);
void boot_prepare(he_ctx *cx, int K, int r, int d);
Ct bootstrap_ct(he_ctx *cx, const he_ct *in);
Ct bootstrap_stage(he_ctx *cx, const he_ct *in, int stage);
Ct bootstrap_const(he_ctx *cx, const he_ct *in);  // one complex value in every slot
Ct beta_noise(he_ctx *cx, const he_ct *u, double alpha, int d);

// learned inverse-square-root stand-in (learn.cu): trains the 1 -> 16 -> 1
// square-activation network on host variances x (> 0) and returns its
// quadratic form A x^2 + B x + C
void learn_invsqrt(he_ctx *cx, const float *x_host, size_t n, int steps, float lr, u64 seed, double *abc,
                   double *loss);

void check_cuda(cudaError_t e, const char *what);
void release_slot(int slot);

}  // namespace he
