// CUDA kernels of the homomorphic CutMax library (sm_103a).
//
// Everything that touches ring data runs here: negacyclic NTT / INTT,
// pointwise modular arithmetic, the hybrid key-switching pieces (basis
// conversion, key inner product, ModDown), rescale, automorphisms, the
// Philox samplers and the float64 canonical-embedding FFT.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <vector>

#include "context.h"
#include "kernels.h"

namespace he {

thread_local int t_slot = 0;
__constant__ PrimeConsts c_pcs[HE_MAX_CTX];

void upload_constants(int slot, const PrimeConsts &pc_in, const u64 *cdt, int n_cdt, cudaStream_t s) {
    PrimeConsts pc = pc_in;
    for (int i = 0; i < HE_MAX_PRIMES; i++) {
        u64 q = pc.m[i].q;
        pc.r64[i] = q ? (u64)(((unsigned __int128)1 << 64) % q) : 0;
        u64 inv = 1;  // q^-1 mod 2^64 by Newton iteration (q odd)
        for (int it = 0; it < 6; it++) inv *= 2 - q * inv;
        pc.mont_qinv[i] = q ? (u64)0 - inv : 0;
    }
    for (int i = 0; i < n_cdt && i < 24; i++) pc.cdt[i] = cdt[i];
    pc.ncdt = n_cdt;
    cudaMemcpyToSymbolAsync(c_pcs, &pc, sizeof(pc), sizeof(PrimeConsts) * slot, cudaMemcpyHostToDevice, s);
}

static std::atomic<unsigned long long> g_launches{0};
unsigned long long launch_count() { return g_launches.load(); }
void launches_add(long long n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

// ---------------------------------------------------------------- profiling
// When a kernel class is enabled, its launchers bracket each launch with a
// pair of CUDA events on the launch stream; prof_read sums the durations.
namespace {
struct ProfState {
    int cls = -1;
    std::vector<cudaEvent_t> ev;  // pairs
    std::vector<double> bytes;
    size_t used = 0;
    double total_bytes = 0;
};
ProfState g_prof;
}  // namespace

void prof_enable(int cls) {
    g_prof.cls = cls;
    g_prof.used = 0;
    g_prof.total_bytes = 0;
    g_prof.bytes.clear();
}
bool prof_on(int cls) { return cls == g_prof.cls; }
bool prof_any() { return g_prof.cls >= 0; }
void prof_begin(int cls, cudaStream_t s) {
    if (cls != g_prof.cls) return;
    if (g_prof.used * 2 + 2 > g_prof.ev.size()) {
        size_t grow = g_prof.ev.size() ? g_prof.ev.size() : 1024;
        for (size_t i = 0; i < grow; i++) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            g_prof.ev.push_back(e);
        }
    }
    cudaEventRecord(g_prof.ev[2 * g_prof.used], s);
}
void prof_end(int cls, cudaStream_t s, double bytes) {
    if (cls != g_prof.cls) return;
    cudaEventRecord(g_prof.ev[2 * g_prof.used + 1], s);
    g_prof.used++;
    g_prof.total_bytes += bytes;
}
void prof_read(int cls, unsigned long long *launches, double *ms, double *bytes) {
    *launches = 0;
    *ms = 0;
    *bytes = 0;
    if (cls != g_prof.cls) return;
    double t = 0;
    for (size_t i = 0; i < g_prof.used; i++) {
        cudaEventSynchronize(g_prof.ev[2 * i + 1]);
        float f = 0;
        cudaEventElapsedTime(&f, g_prof.ev[2 * i], g_prof.ev[2 * i + 1]);
        t += f;
    }
    *launches = g_prof.used;
    *ms = t;
    *bytes = g_prof.total_bytes;
}

static inline unsigned grid_for(size_t total, int per_block) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    size_t g = (total + per_block - 1) / per_block;
    return (unsigned)(g > 0x7fffffff ? 0x7fffffff : g);
}

// ------------------------------------------------------------------ NTT
// N = R*C with R = 2^LOGR, C = 2^LOGC.  Forward (Cooley-Tukey with the
// psi twist merged, Harvey lazy butterflies in [0,4q)): stages 0..LOGR-1
// pair rows of one column (column pass), the rest pair entries of one row
// (row pass).  Stage with m groups uses twiddle psi^brv(m + j/(2t)).
// Inverse (Gentleman-Sande, [0,2q)) runs the same stages in reverse, then
// multiplies by N^-1.
// Each CTA transforms a tile of 16 independent sub-transforms of size
// M = 2^LOGM (16 columns of R rows in the column pass, 16 rows of C entries in
// the row pass) with M threads; every thread holds 16 entries in registers.
// Round A covers the sub-transform's first four stages (distances M/2 ..
// M/16): thread j owns entries j + (M/16) i.  Round B covers the remaining
// LOGM - 4 stages (distances < 16): thread j owns entries 16 j + i.
// Local stage s of a sub-transform is global stage s (column pass) or
// LOGR + s (row pass); its twiddle index is 2^s + grp (column) or
// 2^s (R + row) + grp (row), grp < 2^s.
// The CTA stages its tile and the twiddle pairs (value, Shoup companion) in
// shared memory with asynchronous 16-byte copies: the column pass shares the
// R - 1 twiddles of its stages among all columns; the row pass needs, for
// stage s, the 16 * 2^s consecutive table entries starting at 2^s (R + first
// row).  The butterflies then read only shared memory.  The row pass stages
// round A's twiddles with the tile, and round B's (15/16 of them) only once
// the tile sits in registers, into the same buffer: 65 KB instead of 102 KB
// per CTA at C = 256, so that three CTAs share an SM.  Row-pass tiles carry
// two pad words per 16 entries, which keeps 16-byte alignment and spreads
// round B's 16-byte reads over the banks.
constexpr int NTT_TILE = 16;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <int LOGR, int LOGC, bool COLS>
struct NttShape {
    static constexpr int LOGM = COLS ? LOGR : LOGC, M = 1 << LOGM;
    static constexpr int DATA = COLS ? 16 * M : 18 * M;       // u64 words
    // twiddle pairs: column pass all M - 1 (one per group, shared by the
    // columns); row pass, round A (stages 0..3) 16 * 15, round B 16 * (M - 16)
    static constexpr int TWA = COLS ? M : 16 * 15;
    static constexpr int TWB = COLS ? 0 : 16 * (M - 16);
    // row pass: the tile and round B's twiddles share the first region
    static constexpr size_t U = COLS ? (size_t)DATA * 8
                                     : ((size_t)DATA * 8 > (size_t)TWB * 16 ? (size_t)DATA * 8 : (size_t)TWB * 16);
    static constexpr size_t SMEM = U + (size_t)TWA * 16;
};

template <bool FWD>
__device__ __forceinline__ void bfly(u64 &X, u64 &Y, ulonglong2 w, u64 q, u64 q2) {
    if (FWD) {  // Harvey CT, values in [0, 4q)
        if (X >= q2) X -= q2;
        u64 T = shoup_mul_lazy(Y, w.x, w.y, q);
        Y = X - T + q2;
        X = X + T;
    } else {    // Harvey GS, values in [0, 2q)
        u64 S = X + Y;
        if (S >= q2) S -= q2;
        Y = shoup_mul_lazy(X - Y + q2, w.x, w.y, q);
        X = S;
    }
}

// One tile of one pass: tile `tile` (16 sub-transforms) of limb row `rb`;
// smem holds the pass's NttShape::SMEM bytes.
template <int LOGR, int LOGC, bool FWD, bool COLS>
__device__ __forceinline__ void ntt_tile(const Rows &rows, const Rows &src, const NttTables &tw, const int tile,
                                         const int rb, unsigned char *ntt_smem) {
    using S = NttShape<LOGR, LOGC, COLS>;
    constexpr int LOGN = LOGR + LOGC, R = 1 << LOGR, C = 1 << LOGC;
    constexpr int LOGM = S::LOGM, M = S::M, TPS = M / 16;
    u64 *sm = reinterpret_cast<u64 *>(ntt_smem);
    ulonglong2 *stw = reinterpret_cast<ulonglong2 *>(ntt_smem + S::U);       // column pass; row pass round A
    ulonglong2 *stwb = reinterpret_cast<ulonglong2 *>(ntt_smem);             // row pass round B (over the tile)
    const PrimeConsts &pc = c_pcs[rows.slot];
    u64 *x = rows.row(rb, LOGN);
    const u64 *xin = src.base ? src.row(rb, LOGN) : x;  // out-of-place first pass
    const int p = rows.prime(rb);
    const u64 q = pc.m[p].q, q2 = 2 * q;
    const ulonglong2 *W = (FWD ? tw.fwd : tw.inv) + ((size_t)p << LOGN);
    const int tid = threadIdx.x;
    // smem word of entry e of sub-transform `sub`
    auto sidx = [&](int sub, int e) -> int {
        if (COLS) return e * 16 + sub;
        int a = sub * M + e;
        return a + 2 * (a >> 4);
    };
    // thread -> (sub-transform, position)
    const int sub = COLS ? (tid & 15) : (tid / TPS);
    const int j = COLS ? (tid >> 4) : (tid % TPS);
    // the inverse row pass starts with round B, whose 16 entries per thread
    // are consecutive words: it reads them straight into registers and stages
    // round B's twiddles at once, in the buffer the tile would otherwise take
    constexpr bool direct_b = !FWD && !COLS;
    // row pass, round B's twiddles: group j G + g of row `sub` stored at g TPS + j,
    // stage s at 16 (2^s - 16)
    auto issue_b = [&]() {
        const size_t r0 = (size_t)tile * 16;
        constexpr int LT = LOGM - 4;  // log2 TPS
#pragma unroll
        for (int s = 4; s < LOGM; s++) {
            const ulonglong2 *ws = W + ((R + r0) << s);
            ulonglong2 *ds = stwb + 16 * ((1 << s) - 16);
            for (int k = tid; k < (16 << s); k += M) {
                const int sub_k = k >> s, grp = k & ((1 << s) - 1);
                const int jj = grp >> (s - LT), g = grp & ((1 << (s - LT)) - 1);
                cp_async16(ds + (sub_k << s) + (g << LT) + jj, ws + k);
            }
        }
    };
    u64 v[16];
    if (COLS) {
        const int c0 = tile * 16;
#pragma unroll 4
        for (int idx = tid; idx < 8 * M; idx += M) {  // row r of the tile: 16 words at xin[r C + c0]
            int r = idx >> 3, h = idx & 7;
            cp_async16(sm + r * 16 + 2 * h, xin + (size_t)r * C + c0 + 2 * h);
        }
        if (tid + 1 < M) cp_async16(stw + tid, W + tid + 1);
    } else {
        const u64 *xr = xin + (size_t)tile * 16 * C;
        if (!direct_b) {
#pragma unroll 4
            for (int idx = tid; idx < 8 * M; idx += M) {
                int a = 2 * idx;
                cp_async16(sm + a + 2 * (a >> 4), xr + a);
            }
        }
        const size_t r0 = (size_t)tile * 16;
#pragma unroll
        for (int s = 0; s < 4; s++) {  // round A: one group per thread group of a row (broadcast reads)
            const ulonglong2 *ws = W + ((R + r0) << s);
            ulonglong2 *ds = stw + 16 * ((1 << s) - 1);
            for (int k = tid; k < (16 << s); k += M) cp_async16(ds + k, ws + k);
        }
        if (direct_b) {
            issue_b();
            const ulonglong2 *p2 = reinterpret_cast<const ulonglong2 *>(xr + (size_t)sub * M + 16 * j);
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const ulonglong2 t2 = p2[i];
                v[2 * i] = t2.x;
                v[2 * i + 1] = t2.y;
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();
    // forward row pass: round B's twiddles once the tile is in registers
    auto stage_b = [&]() {
        if (COLS || direct_b) return;
        __syncthreads();  // every thread has read its entries of the tile
        issue_b();
        cp_async_wait_all();
        __syncthreads();
    };
    auto release_b = [&]() {  // round B done with its twiddles: the tile may return
        if (!COLS) __syncthreads();
    };
    auto twl = [&](int s, int grp) -> ulonglong2 {  // local stage s, group grp
        if (COLS) return stw[(1 << s) - 1 + grp];
        return stw[16 * ((1 << s) - 1) + (sub << s) + grp];
    };
    // row pass, round B: group j G + g (G = 2^s / TPS), stored transposed
    auto twl_b = [&](int s, int g) -> ulonglong2 {
        if (COLS) return stw[(1 << s) - 1 + j * ((1 << s) / TPS) + g];
        return stwb[16 * ((1 << s) - 16) + (sub << s) + g * TPS + j];
    };
    auto round_a = [&]() {  // stages 0..3, entries j + TPS i
#pragma unroll
        for (int st = 0; st < 4; st++) {
            const int s = FWD ? st : 3 - st;
            const int d = 8 >> s;  // distance in i
#pragma unroll
            for (int i = 0; i < 16; i++)
                if ((i & d) == 0) bfly<FWD>(v[i], v[i + d], twl(s, i >> (4 - s)), q, q2);
        }
    };
    auto round_b = [&]() {  // stages 4..LOGM-1, entries 16 j + i
#pragma unroll
        for (int st = 0; st < LOGM - 4; st++) {
            const int s = FWD ? 4 + st : LOGM - 1 - st;
            const int t = M >> (s + 1);  // distance (< 16)
#pragma unroll
            for (int i = 0; i < 16; i++)
                if ((i & t) == 0) bfly<FWD>(v[i], v[i + t], twl_b(s, i / (2 * t)), q, q2);
        }
    };
    auto load_a = [&]() {
#pragma unroll
        for (int i = 0; i < 16; i++) v[i] = sm[sidx(sub, j + TPS * i)];
    };
    auto store_a = [&]() {
#pragma unroll
        for (int i = 0; i < 16; i++) sm[sidx(sub, j + TPS * i)] = v[i];
    };
    auto load_b = [&]() {
        if (COLS) {
#pragma unroll
            for (int i = 0; i < 16; i++) v[i] = sm[sidx(sub, 16 * j + i)];
        } else {
            const ulonglong2 *p2 = reinterpret_cast<const ulonglong2 *>(sm + sidx(sub, 16 * j));
#pragma unroll
            for (int i = 0; i < 8; i++) {
                ulonglong2 t2 = p2[i];
                v[2 * i] = t2.x;
                v[2 * i + 1] = t2.y;
            }
        }
    };
    auto store_b = [&]() {
        if (COLS) {
#pragma unroll
            for (int i = 0; i < 16; i++) sm[sidx(sub, 16 * j + i)] = v[i];
        } else {
            ulonglong2 *p2 = reinterpret_cast<ulonglong2 *>(sm + sidx(sub, 16 * j));
#pragma unroll
            for (int i = 0; i < 8; i++) p2[i] = make_ulonglong2(v[2 * i], v[2 * i + 1]);
        }
    };
    if (FWD) {
        load_a();
        round_a();
        store_a();
        __syncthreads();
        load_b();
        stage_b();
        round_b();
        if (!COLS) {  // last stage of the forward transform: reduce to [0, q)
#pragma unroll
            for (int i = 0; i < 16; i++) {
                u64 t = v[i];
                if (t >= q2) t -= q2;
                if (t >= q) t -= q;
                v[i] = t;
            }
        }
        release_b();
        store_b();
    } else {
        if (!direct_b) load_b();
        stage_b();
        round_b();
        release_b();
        store_b();
        __syncthreads();
        load_a();
        round_a();
        if (COLS) {  // end of the inverse transform: times N^-1, reduce to [0, q)
            const u64 ni = pc.n_inv[p], nis = pc.n_inv_shoup[p];
#pragma unroll
            for (int i = 0; i < 16; i++) v[i] = shoup_mul(v[i], ni, nis, q);
        }
        store_a();
    }
    __syncthreads();
    if (COLS) {
        const int c0 = tile * 16;
#pragma unroll 4
        for (int idx = tid; idx < 8 * M; idx += M) {
            int r = idx >> 3, h = idx & 7;
            *reinterpret_cast<ulonglong2 *>(x + (size_t)r * C + c0 + 2 * h) =
                *reinterpret_cast<const ulonglong2 *>(sm + r * 16 + 2 * h);
        }
    } else {
        u64 *xr = x + (size_t)tile * 16 * C;
#pragma unroll 4
        for (int idx = tid; idx < 8 * M; idx += M) {
            int a = 2 * idx;
            *reinterpret_cast<ulonglong2 *>(xr + a) = *reinterpret_cast<const ulonglong2 *>(sm + a + 2 * (a >> 4));
        }
    }
}

template <int LOGR, int LOGC, bool FWD, bool COLS>
__global__ void __launch_bounds__(1 << (COLS ? LOGR : LOGC), 3) k_ntt(Rows rows, Rows src, NttTables tw) {
    extern __shared__ __align__(16) unsigned char ntt_smem[];
    ntt_tile<LOGR, LOGC, FWD, COLS>(rows, src, tw, blockIdx.x, blockIdx.y, ntt_smem);
}

// dynamic shared memory above 48 KB is an opt-in attribute, set once per device
template <typename K>
static void ntt_smem_attr(K kern, size_t bytes, std::atomic<unsigned long long> &done) {
    int dev = 0;
    cudaGetDevice(&dev);
    unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return;
    check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes),
               "NTT shared memory attribute");
    done.fetch_or(bit, std::memory_order_release);
}

template <int LOGR, int LOGC>
static void ntt_launch(const Rows &rows, const Rows &src, int n_rows, const NttTables &tw, bool fwd, cudaStream_t s) {
    constexpr int R = 1 << LOGR, C = 1 << LOGC;
    using SC = NttShape<LOGR, LOGC, true>;
    using SR = NttShape<LOGR, LOGC, false>;
    static std::atomic<unsigned long long> done[4];
    dim3 gc(C / NTT_TILE, n_rows), gr(R / NTT_TILE, n_rows);
    Rows none = rows;
    none.base = nullptr;
    g_launches.fetch_add(2, std::memory_order_relaxed);
    if (fwd) {
        ntt_smem_attr(k_ntt<LOGR, LOGC, true, true>, SC::SMEM, done[0]);
        ntt_smem_attr(k_ntt<LOGR, LOGC, true, false>, SR::SMEM, done[1]);
        k_ntt<LOGR, LOGC, true, true><<<gc, R, SC::SMEM, s>>>(rows, src, tw);
        k_ntt<LOGR, LOGC, true, false><<<gr, C, SR::SMEM, s>>>(rows, none, tw);
    } else {
        ntt_smem_attr(k_ntt<LOGR, LOGC, false, false>, SR::SMEM, done[2]);
        ntt_smem_attr(k_ntt<LOGR, LOGC, false, true>, SC::SMEM, done[3]);
        k_ntt<LOGR, LOGC, false, false><<<gr, C, SR::SMEM, s>>>(rows, src, tw);
        k_ntt<LOGR, LOGC, false, true><<<gc, R, SC::SMEM, s>>>(rows, none, tw);
    }
}

static void ntt_dispatch(const Rows &rows, const Rows &src, int n_rows, const NttTables &tw, int log_n, bool fwd,
                         cudaStream_t s) {
    if (n_rows <= 0) return;
    if ((reinterpret_cast<uintptr_t>(rows.base) & 15) || (reinterpret_cast<uintptr_t>(src.base) & 15))
        throw Error{HE_EINVAL, "NTT data must start on a 16-byte boundary"};
    const int cls = fwd ? PROF_NTT_FWD : PROF_NTT_INV;
    prof_begin(cls, s);
    switch (log_n) {
        case 10: ntt_launch<5, 5>(rows, src, n_rows, tw, fwd, s); break;
        case 11: ntt_launch<5, 6>(rows, src, n_rows, tw, fwd, s); break;
        case 12: ntt_launch<6, 6>(rows, src, n_rows, tw, fwd, s); break;
        case 13: ntt_launch<6, 7>(rows, src, n_rows, tw, fwd, s); break;
        case 14: ntt_launch<7, 7>(rows, src, n_rows, tw, fwd, s); break;
        case 15: ntt_launch<7, 8>(rows, src, n_rows, tw, fwd, s); break;
        case 16: ntt_launch<8, 8>(rows, src, n_rows, tw, fwd, s); break;
        default: break;
    }
    prof_end(cls, s, 16.0 * (double)n_rows * (double)(1 << log_n));
}
static Rows no_src(const Rows &r) {
    Rows n = r;
    n.base = nullptr;
    return n;
}
void ntt_forward(const Rows &rows, int n_rows, const NttTables &tw, int log_n, cudaStream_t s) {
    ntt_dispatch(rows, no_src(rows), n_rows, tw, log_n, true, s);
}
void ntt_inverse(const Rows &rows, int n_rows, const NttTables &tw, int log_n, cudaStream_t s) {
    ntt_dispatch(rows, no_src(rows), n_rows, tw, log_n, false, s);
}
void ntt_inverse_from(const Rows &dst, const Rows &src, int n_rows, const NttTables &tw, int log_n, cudaStream_t s) {
    ntt_dispatch(dst, src, n_rows, tw, log_n, false, s);
}

// ------------------------------------------------------------------ elementwise
// Row-parallel layout: blockIdx.y selects the limb row and every thread of
// an EW_T-thread block handles EW_PAIRS pairs of consecutive coefficients
// (one 16-byte access per operand and pair; pairs EW_T apart, so each warp
// access is one contiguous 512-byte span).  A row's addresses and prime are
// resolved once per thread.  Every row must start on a 16-byte boundary
// (the launchers check the base pointers; rows are N >= 2 words apart).
constexpr int EW_T = 256, EW_PAIRS = 4;

static inline dim3 ew_grid(int n_rows, int log_n) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (n_rows > 65535) throw Error{HE_EINVAL, "too many rows for one elementwise launch"};
    const size_t per_block = (size_t)EW_T * 2 * EW_PAIRS;
    return dim3((unsigned)((((size_t)1 << log_n) + per_block - 1) / per_block), (unsigned)n_rows);
}
static inline void need16(const void *p) {
    if (reinterpret_cast<uintptr_t>(p) & 15) throw Error{HE_EINVAL, "device rows must start on a 16-byte boundary"};
}
static inline void need16(const Rows &r) { need16(r.base); }

// k runs over the first coefficient of each pair this thread owns in its row
#define EW_PAIRS_FOR(k, log_n)                                                                 \
    _Pragma("unroll") for (int ew_i = 0; ew_i < EW_PAIRS; ew_i++)                              \
        if (const size_t k = 2 * (((size_t)blockIdx.x * EW_PAIRS + ew_i) * EW_T + threadIdx.x); \
            k < ((size_t)1 << (log_n)))

__device__ __forceinline__ ulonglong2 ld2(const u64 *p) { return *reinterpret_cast<const ulonglong2 *>(p); }
__device__ __forceinline__ void st2(u64 *p, u64 a, u64 b) {
    *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(a, b);
}

__global__ void __launch_bounds__(EW_T) k_add(Rows out, Rows a, Rows b, int sub, int log_n) {
    const int r = blockIdx.y;
    const u64 q = c_pcs[out.slot].m[out.prime(r)].q;
    u64 *o = out.row(r, log_n);
    const u64 *x = a.row(r, log_n), *y = b.row(r, log_n);
    EW_PAIRS_FOR(k, log_n) {
        ulonglong2 u = ld2(x + k), v = ld2(y + k);
        if (sub) st2(o + k, sub_mod(u.x, v.x, q), sub_mod(u.y, v.y, q));
        else st2(o + k, add_mod(u.x, v.x, q), add_mod(u.y, v.y, q));
    }
}
__global__ void __launch_bounds__(EW_T) k_neg(Rows out, Rows a, int log_n) {
    const int r = blockIdx.y;
    const u64 q = c_pcs[out.slot].m[out.prime(r)].q;
    u64 *o = out.row(r, log_n);
    const u64 *x = a.row(r, log_n);
    EW_PAIRS_FOR(k, log_n) {
        ulonglong2 u = ld2(x + k);
        st2(o + k, u.x ? q - u.x : 0, u.y ? q - u.y : 0);
    }
}
__global__ void __launch_bounds__(EW_T) k_copy(Rows out, Rows a, int log_n) {
    const int r = blockIdx.y;
    u64 *o = out.row(r, log_n);
    const u64 *x = a.row(r, log_n);
    EW_PAIRS_FOR(k, log_n) {
        ulonglong2 u = ld2(x + k);
        st2(o + k, u.x, u.y);
    }
}
__global__ void __launch_bounds__(EW_T) k_mul_scalar(Rows out, Rows a, ScalarTab kt, int log_n) {
    const int r = blockIdx.y, p = out.prime(r);
    const u64 q = c_pcs[out.slot].m[p].q, w = kt.v[p], ws = kt.s[p];
    u64 *o = out.row(r, log_n);
    const u64 *x = a.row(r, log_n);
    EW_PAIRS_FOR(k, log_n) {
        ulonglong2 u = ld2(x + k);
        st2(o + k, shoup_mul(u.x, w, ws, q), shoup_mul(u.y, w, ws, q));
    }
}
__global__ void __launch_bounds__(EW_T) k_add_scalar(Rows out, Rows a, ScalarTab kt, int log_n) {
    const int r = blockIdx.y, p = out.prime(r);
    const u64 q = c_pcs[out.slot].m[p].q, w = kt.v[p];
    u64 *o = out.row(r, log_n);
    const u64 *x = a.row(r, log_n);
    EW_PAIRS_FOR(k, log_n) {
        ulonglong2 u = ld2(x + k);
        st2(o + k, add_mod(u.x, w, q), add_mod(u.y, w, q));
    }
}
__global__ void __launch_bounds__(EW_T) k_mul(Rows out, Rows a, Rows b, int acc, int log_n) {
    const int r = blockIdx.y;
    const ModQ m = c_pcs[out.slot].m[out.prime(r)];
    u64 *o = out.row(r, log_n);
    const u64 *x = a.row(r, log_n), *y = b.row(r, log_n);
    EW_PAIRS_FOR(k, log_n) {
        ulonglong2 u = ld2(x + k), v = ld2(y + k);
        u64 p0 = mul_mod(u.x, v.x, m), p1 = mul_mod(u.y, v.y, m);
        if (acc) {
            ulonglong2 c = ld2(o + k);
            p0 = add_mod(c.x, p0, m.q);
            p1 = add_mod(c.y, p1, m.q);
        }
        st2(o + k, p0, p1);
    }
}
// out_k = sum_b src_b,k * pt_b (k = 0, 1: both polynomials of a ciphertext),
// plaintexts in Montgomery form: the products are summed in 128 bits and each
// output is reduced once.
__device__ __forceinline__ void mac128(u64 &lo, u64 &hi, u64 x, u64 w) {
    const u64 pl = x * w, ph = __umul64hi(x, w);
    lo += pl;
    hi += ph + (lo < pl ? 1ull : 0ull);
}
__global__ void __launch_bounds__(EW_T) k_diag_mac(DiagMac dm, int log_n) {
    const PrimeConsts &pc = c_pcs[dm.slot];
    const int r = blockIdx.y;
    const int pr = r < dm.l1 ? r : dm.nq + (r - dm.l1);
    const ModQ m = pc.m[pr];
    const u64 qn = pc.mont_qinv[pr];
    const size_t row = (size_t)r << log_n, mo = (size_t)blockIdx.z * dm.c_stride, oo = (size_t)blockIdx.z * dm.out_stride;
    EW_PAIRS_FOR(k, log_n) {
        const size_t off = row + k;
        u64 s00 = 0, s01 = 0, s10 = 0, s11 = 0;
        for (int b0 = 0; b0 < dm.n; b0 += 16) {  // at most 16 products (< 2^126) per 128-bit sum
            u64 l00 = 0, h00 = 0, l01 = 0, h01 = 0, l10 = 0, h10 = 0, l11 = 0, h11 = 0;
            const int b1 = min(dm.n, b0 + 16);
            for (int b = b0; b < b1; b++) {
                const ulonglong2 w = ld2(dm.pt[b] + off);
                const ulonglong2 x0 = ld2(dm.c0[b] + mo + off), x1 = ld2(dm.c1[b] + mo + off);
                mac128(l00, h00, x0.x, w.x);
                mac128(l01, h01, x0.y, w.y);
                mac128(l10, h10, x1.x, w.x);
                mac128(l11, h11, x1.y, w.y);
            }
            s00 = add_mod(s00, mont_reduce_wide(l00, h00, m, qn), m.q);
            s01 = add_mod(s01, mont_reduce_wide(l01, h01, m, qn), m.q);
            s10 = add_mod(s10, mont_reduce_wide(l10, h10, m, qn), m.q);
            s11 = add_mod(s11, mont_reduce_wide(l11, h11, m, qn), m.q);
        }
        st2(dm.out0 + oo + off, s00, s01);
        st2(dm.out1 + oo + off, s10, s11);
    }
}
void ew_diag_mac(const DiagMac &dm, int n_rows, int log_n, cudaStream_t s) {
    need16(dm.out0);
    need16(dm.out1);
    for (int b = 0; b < dm.n; b++) {
        need16(dm.c0[b]);
        need16(dm.c1[b]);
        need16(dm.pt[b]);
    }
    if (dm.batch < 1 || (dm.batch > 1 && ((dm.c_stride | dm.out_stride) & 1)))
        throw Error{HE_EINVAL, "diagonal multiply-accumulate: bad batch layout"};
    dim3 grid = ew_grid(n_rows, log_n);
    grid.z = (unsigned)dm.batch;
    k_diag_mac<<<grid, EW_T, 0, s>>>(dm, log_n);
}

// Members of a batch of ciphertexts (both polynomials, limbs 0..l, member m
// at base + m*stride): out member s = sum of in members s*g .. s*g+g-1
// (group sum), or out member b = in member b / g (broadcast).
__global__ void __launch_bounds__(EW_T) k_group(u64 *out, const u64 *in, int g, int sum, int l1, size_t out_stride,
                                                size_t in_stride, size_t in_poly, size_t out_poly, int slot,
                                                int log_n) {
    const int r = blockIdx.y, poly = r / l1, t = r % l1;
    const u64 q = c_pcs[slot].m[t].q;
    const size_t m = blockIdx.z;
    u64 *o = out + m * out_stride + poly * out_poly + ((size_t)t << log_n);
    if (sum) {
        const u64 *x = in + m * g * in_stride + poly * in_poly + ((size_t)t << log_n);
        EW_PAIRS_FOR(k, log_n) {
            ulonglong2 a = ld2(x + k);
            for (int c = 1; c < g; c++) {
                const ulonglong2 b = ld2(x + c * in_stride + k);
                a.x = add_mod(a.x, b.x, q);
                a.y = add_mod(a.y, b.y, q);
            }
            st2(o + k, a.x, a.y);
        }
    } else {
        const u64 *x = in + (m / g) * in_stride + poly * in_poly + ((size_t)t << log_n);
        EW_PAIRS_FOR(k, log_n) {
            const ulonglong2 a = ld2(x + k);
            st2(o + k, a.x, a.y);
        }
    }
}
void ew_group(u64 *out, const u64 *in, int n_out_members, int g, int sum, int l1, size_t out_stride, size_t in_stride,
              size_t in_poly, size_t out_poly, int slot, int log_n, cudaStream_t s) {
    need16(out);
    need16(in);
    if (((out_stride | in_stride | in_poly | out_poly) & 1) || g < 1) throw Error{HE_EINVAL, "group op: bad layout"};
    dim3 grid = ew_grid(2 * l1, log_n);
    grid.z = (unsigned)n_out_members;
    k_group<<<grid, EW_T, 0, s>>>(out, in, g, sum, l1, out_stride, in_stride, in_poly, out_poly, slot, log_n);
}

// source position of NTT-form position i under X -> X^g (g odd < 2N)
__device__ __forceinline__ u32 automorph_src(u32 i, u64 g, int log_n) {
    const u64 two_n_mask = (2ull << log_n) - 1;
    const u64 e = 2ull * (__brev(i) >> (32 - log_n)) + 1;
    const u64 e2 = (e * g) & two_n_mask;
    return __brev((u32)((e2 - 1) >> 1)) >> (32 - log_n);
}

// One polynomial in the QP basis, times P: out_r = (add ? out_r : 0) +
// (P mod q_r) * src_r read through X -> X^g (g = 0: identity) for the Q rows
// r < l1 of an n_rows-row block; the special-prime rows are 0 (P = 0 mod p_i)
// and are left unchanged when adding.
__global__ void __launch_bounds__(EW_T) k_qp_lift(u64 *out, const u64 *src, int l1, u64 g, int add, ScalarTab pm,
                                                  int slot, size_t out_stride, size_t src_stride, int log_n) {
    const int r = blockIdx.y;
    out += blockIdx.z * out_stride;
    src += blockIdx.z * src_stride;
    u64 *o = out + ((size_t)r << log_n);
    if (r >= l1) {
        EW_PAIRS_FOR(k, log_n) st2(o + k, 0, 0);
        return;
    }
    const u64 q = c_pcs[slot].m[r].q, w = pm.v[r], ws = pm.s[r];
    const u64 *x = src + ((size_t)r << log_n);
    EW_PAIRS_FOR(k, log_n) {
        u64 a, b;
        if (g) {
            a = x[automorph_src((u32)k, g, log_n)];
            b = x[automorph_src((u32)k + 1, g, log_n)];
        } else {
            ulonglong2 u = ld2(x + k);
            a = u.x;
            b = u.y;
        }
        a = shoup_mul(a, w, ws, q);
        b = shoup_mul(b, w, ws, q);
        if (add) {
            ulonglong2 c = ld2(o + k);
            a = add_mod(c.x, a, q);
            b = add_mod(c.y, b, q);
        }
        st2(o + k, a, b);
    }
}
void ew_qp_lift(u64 *out, const u64 *src, int l1, int n_rows, u64 g, int add, const ScalarTab &pm, int slot,
                int log_n, cudaStream_t s, int batch, size_t out_stride, size_t src_stride) {
    need16(out);
    need16(src);
    if (batch > 1 && ((out_stride | src_stride) & 1)) throw Error{HE_EINVAL, "QP lift: bad batch layout"};
    dim3 grid = ew_grid(add ? l1 : n_rows, log_n);
    grid.z = (unsigned)batch;
    k_qp_lift<<<grid, EW_T, 0, s>>>(out, src, l1, g, add, pm, slot, out_stride, src_stride, log_n);
}

__global__ void __launch_bounds__(EW_T) k_tensor(Rows d0, Rows d1, Rows d2, Rows a0, Rows a1, Rows b0, Rows b1,
                                                 int log_n) {
    const int r = blockIdx.y;
    const ModQ m = c_pcs[d0.slot].m[d0.prime(r)];
    u64 *o0 = d0.row(r, log_n), *o1 = d1.row(r, log_n), *o2 = d2.row(r, log_n);
    const u64 *pa0 = a0.row(r, log_n), *pa1 = a1.row(r, log_n), *pb0 = b0.row(r, log_n), *pb1 = b1.row(r, log_n);
    EW_PAIRS_FOR(k, log_n) {
        const ulonglong2 x0 = ld2(pa0 + k), x1 = ld2(pa1 + k), y0 = ld2(pb0 + k), y1 = ld2(pb1 + k);
        st2(o0 + k, mul_mod(x0.x, y0.x, m), mul_mod(x0.y, y0.y, m));
        st2(o1 + k, mul_add_mod(x0.x, y1.x, x1.x, y0.x, m), mul_add_mod(x0.y, y1.y, x1.y, y0.y, m));
        st2(o2 + k, mul_mod(x1.x, y1.x, m), mul_mod(x1.y, y1.y, m));
    }
}
__global__ void __launch_bounds__(EW_T) k_automorph(Rows out, Rows a, u64 g, int log_n) {
    const int r = blockIdx.y;
    u64 *o = out.row(r, log_n);
    const u64 *x = a.row(r, log_n);
    EW_PAIRS_FOR(k, log_n) st2(o + k, x[automorph_src((u32)k, g, log_n)], x[automorph_src((u32)k + 1, g, log_n)]);
}

// out = a * X^e: in NTT form position i is multiplied by psi^((2 brv(i)+1) e),
// read from the forward table (psi^j = fwd[brv(j)], psi^(j+N) = -psi^j).
__global__ void __launch_bounds__(EW_T) k_monomial(Rows out, Rows a, u64 e, NttTables tw, int log_n) {
    const int r = blockIdx.y, p = out.prime(r);
    const ModQ m = c_pcs[out.slot].m[p];
    const u64 n = 1ull << log_n, two_n_mask = 2 * n - 1;
    const ulonglong2 *fw = tw.fwd + ((size_t)p << log_n);
    u64 *o = out.row(r, log_n);
    const u64 *x = a.row(r, log_n);
    auto factor = [&](u32 i) -> u64 {
        const u64 t = ((2ull * (__brev(i) >> (32 - log_n)) + 1) * e) & two_n_mask;
        return t < n ? fw[__brev((u32)t) >> (32 - log_n)].x : m.q - fw[__brev((u32)(t - n)) >> (32 - log_n)].x;
    };
    EW_PAIRS_FOR(k, log_n) {
        const ulonglong2 u = ld2(x + k);
        st2(o + k, mul_mod(u.x, factor((u32)k), m), mul_mod(u.y, factor((u32)k + 1), m));
    }
}
// x -> x * 2^64 mod q (to Montgomery form) or x * 2^-64 mod q (back)
__global__ void __launch_bounds__(EW_T) k_to_mont(Rows out, int back, int log_n) {
    const int r = blockIdx.y, p = out.prime(r);
    const PrimeConsts &pc = c_pcs[out.slot];
    const ModQ m = pc.m[p];
    const u64 qn = pc.mont_qinv[p], r64 = pc.r64[p];
    u64 *o = out.row(r, log_n);
    EW_PAIRS_FOR(k, log_n) {
        const ulonglong2 u = ld2(o + k);
        if (back) st2(o + k, mont_reduce(u.x, 0, m.q, qn), mont_reduce(u.y, 0, m.q, qn));
        else st2(o + k, mul_mod(u.x, r64, m), mul_mod(u.y, r64, m));
    }
}
void ew_mont(const Rows &rows, int n_rows, int back, int log_n, cudaStream_t s) {
    need16(rows);
    k_to_mont<<<ew_grid(n_rows, log_n), EW_T, 0, s>>>(rows, back, log_n);
}
void ew_monomial(const Rows &out, const Rows &a, int n_rows, u64 e, const NttTables &tw, int log_n, cudaStream_t s) {
    need16(out);
    need16(a);
    k_monomial<<<ew_grid(n_rows, log_n), EW_T, 0, s>>>(out, a, e, tw, log_n);
}
void ew_add(const Rows &out, const Rows &a, const Rows &b, int n_rows, int sub, int log_n, cudaStream_t s) {
    need16(out);
    need16(a);
    need16(b);
    k_add<<<ew_grid(n_rows, log_n), EW_T, 0, s>>>(out, a, b, sub, log_n);
}
void ew_neg(const Rows &out, const Rows &a, int n_rows, int log_n, cudaStream_t s) {
    need16(out);
    need16(a);
    k_neg<<<ew_grid(n_rows, log_n), EW_T, 0, s>>>(out, a, log_n);
}
void ew_copy(const Rows &out, const Rows &a, int n_rows, int log_n, cudaStream_t s) {
    need16(out);
    need16(a);
    k_copy<<<ew_grid(n_rows, log_n), EW_T, 0, s>>>(out, a, log_n);
}
void ew_mul_scalar(const Rows &out, const Rows &a, const ScalarTab &k, int n_rows, int log_n, cudaStream_t s) {
    need16(out);
    need16(a);
    k_mul_scalar<<<ew_grid(n_rows, log_n), EW_T, 0, s>>>(out, a, k, log_n);
}
void ew_add_scalar(const Rows &out, const Rows &a, const ScalarTab &k, int n_rows, int log_n, cudaStream_t s) {
    need16(out);
    need16(a);
    k_add_scalar<<<ew_grid(n_rows, log_n), EW_T, 0, s>>>(out, a, k, log_n);
}
void ew_mul(const Rows &out, const Rows &a, const Rows &b, int n_rows, int log_n, cudaStream_t s) {
    need16(out);
    need16(a);
    need16(b);
    k_mul<<<ew_grid(n_rows, log_n), EW_T, 0, s>>>(out, a, b, 0, log_n);
}
void ew_mul_acc(const Rows &out, const Rows &a, const Rows &b, int n_rows, int log_n, cudaStream_t s) {
    need16(out);
    need16(a);
    need16(b);
    k_mul<<<ew_grid(n_rows, log_n), EW_T, 0, s>>>(out, a, b, 1, log_n);
}
void ew_tensor(const Rows &d0, const Rows &d1, const Rows &d2, const Rows &a0, const Rows &a1, const Rows &b0,
               const Rows &b1, int n_rows, int log_n, cudaStream_t s) {
    for (const Rows *r : {&d0, &d1, &d2, &a0, &a1, &b0, &b1}) need16(*r);
    k_tensor<<<ew_grid(n_rows, log_n), EW_T, 0, s>>>(d0, d1, d2, a0, a1, b0, b1, log_n);
}
void ew_automorph_ntt(const Rows &out, const Rows &a, int n_rows, u64 g, int log_n, cudaStream_t s) {
    need16(out);
    need16(a);
    k_automorph<<<ew_grid(n_rows, log_n), EW_T, 0, s>>>(out, a, g, log_n);
}

// ------------------------------------------------------------------ key switching
// Approximate basis conversion: for every coefficient, y_a = [x_a*qhinv_a]_{q_a},
// out_t = sum_a y_a * qhat[a][t] mod p_t  (= x + v Q for some 0 <= v < n_in).
// Rounding mode (tab.inv_fix set, used by ModDown): v = round(sum_a y_a / q_a)
// = round(S / Q), S = sum_a y_a Qhat_a, so that out_t - v Q mod p_t is the
// centred representative of x mod Q (|.| <= Q/2) and ModDown's (acc - out) / Q
// is the rounded division.  The sum is estimated in 64-bit fixed point with
// integer multiplies: each term floor(y_a m_a / 2^64), m_a = floor(2^128 / q_a),
// is (y_a / q_a) 2^64 less at most 2 units, the carries out of the 64-bit sum
// count the integer part.  Where the fraction lies within 2^20 units
// (~6e-14) of 1/2, the decision is taken exactly instead: the integer part is
// still right, and whether x mod Q exceeds (Q-1)/2 follows from the
// mixed-radix digits of x (Garner's algorithm), compared with those of
// (Q-1)/2 from the most significant down.
// One thread per (coefficient, chunk of BCONV_CHUNK output rows).  The
// products y_a * w_a,t with w = qhat[a][t] 2^64 mod p_t are summed exactly in
// a 128-bit accumulator of four 32-bit words (n_in <= 16 terms below 2^122
// each), one schoolbook 64x64-bit product per term folded in by a PTX carry
// chain of 32-bit multiply-adds; each output is reduced once, by a Montgomery
// step and a Barrett correction.  The chunk's constants sit in shared memory
// (every thread reads the same word: broadcasts).
constexpr int BCONV_CHUNK = 8, BCONV_MAX_IN = 16;
// each thread converts BCONV_CPT coefficients, one after another (1: looping
// over more, to share the block's table set-up, measured slower)
constexpr int BCONV_CPT = 1;
// (a3:a2:a1:a0) += (y1:y0) * (w1:w0)  (no carry out of a3: the caller's sums stay below 2^128)
__device__ __forceinline__ void mac128_words(u32 &a0, u32 &a1, u32 &a2, u32 &a3, u32 y0, u32 y1, u32 w0, u32 w1) {
    asm("mad.lo.cc.u32 %0, %4, %6, %0;\n\t"
        "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"
        "madc.lo.cc.u32 %2, %5, %7, %2;\n\t"
        "madc.hi.u32 %3, %5, %7, %3;\n\t"
        "mad.lo.cc.u32 %1, %4, %7, %1;\n\t"
        "madc.hi.cc.u32 %2, %4, %7, %2;\n\t"
        "addc.u32 %3, %3, 0;\n\t"
        "mad.lo.cc.u32 %1, %5, %6, %1;\n\t"
        "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"
        "addc.u32 %3, %3, 0;"
        : "+r"(a0), "+r"(a1), "+r"(a2), "+r"(a3)
        : "r"(y0), "r"(y1), "r"(w0), "r"(w1));
}
// 1 if the integer x with residues x_a = s_in[a][k] (a < n_in, primes
// s_pidx[a]) exceeds (Q-1)/2 as an element of [0, Q), else 0: mixed-radix
// digits m_i = (((x_i - m_0) q_0^-1 - m_1) q_1^-1 - ...) mod q_i, compared
// from m_(n_in-1) down with the digits of (Q-1)/2.
__device__ __noinline__ u32 bconv_above_half(const u64 *const *s_in, const int *s_pidx, size_t k, int n_in,
                                             const BConvTab &tab, const PrimeConsts &pc) {
    u64 m[BCONV_MAX_IN];
    for (int i = 0; i < n_in; i++) {
        const ModQ mi = pc.m[s_pidx[i]];
        u64 t = s_in[i][k];
        for (int j = 0; j < i; j++)
            t = mul_mod(sub_mod(t, barrett_reduce(m[j], 0, mi), mi.q), tab.mr_inv[i * n_in + j], mi);
        m[i] = t;
    }
    for (int i = n_in - 1; i >= 0; i--)
        if (m[i] != tab.mr_half[i]) return m[i] > tab.mr_half[i] ? 1u : 0u;
    return 0u;  // x = (Q-1)/2 itself rounds down
}
// One block of a conversion: 128 coefficients of polynomial by / n_chunks,
// output chunk by % n_chunks.
template <bool RND>
__device__ __forceinline__ void bconv_block(const Rows &out, const Rows &in, const BConvTab &tab, int n_polys,
                                            int log_n, int by) {
    __shared__ u64 s_w[BCONV_MAX_IN * BCONV_CHUNK];
    __shared__ u64 s_qi[BCONV_MAX_IN], s_qis[BCONV_MAX_IN], s_q[BCONV_MAX_IN];
    __shared__ const u64 *s_in[BCONV_MAX_IN];
    __shared__ int s_pidx[BCONV_MAX_IN];
    __shared__ u64 *s_out[BCONV_CHUNK];
    __shared__ int s_p[BCONV_CHUNK];
    __shared__ u64 s_mlo[BCONV_MAX_IN], s_mhi[BCONV_MAX_IN];
    __shared__ u64 s_wn[BCONV_CHUNK];
    constexpr bool rnd = RND;
    const PrimeConsts &pc = c_pcs[out.slot];
    const size_t n = (size_t)1 << log_n;
    const int n_chunks = (tab.n_out + BCONV_CHUNK - 1) / BCONV_CHUNK;
    const int chunk = by % n_chunks, poly = by / n_chunks;
    const int t0 = chunk * BCONV_CHUNK, nt = min(BCONV_CHUNK, tab.n_out - t0);
    for (int i = threadIdx.x; i < BCONV_MAX_IN * BCONV_CHUNK; i += blockDim.x) {
        const int a = i / BCONV_CHUNK, c = i % BCONV_CHUNK;
        s_w[i] = (a < tab.n_in && c < nt) ? tab.qhat_mont[a * tab.stride + t0 + c] : 0;
    }
    if (threadIdx.x < BCONV_MAX_IN) {
        const int a = threadIdx.x;
        const bool ok = a < tab.n_in && poly < n_polys;
        s_qi[a] = ok ? tab.qhinv[a] : 0;
        s_qis[a] = ok ? tab.qhinv_sh[a] : 0;
        s_q[a] = ok ? pc.m[in.prime(poly * tab.n_in + a)].q : 1;
        s_in[a] = ok ? in.row(poly * tab.n_in + a, log_n) : nullptr;
        s_pidx[a] = ok ? in.prime(poly * tab.n_in + a) : 0;
        s_mlo[a] = ok && rnd ? tab.inv_fix[2 * a] : 0;
        s_mhi[a] = ok && rnd ? tab.inv_fix[2 * a + 1] : 0;
    }
    if (threadIdx.x < BCONV_CHUNK) {
        const int c = threadIdx.x, r = poly * tab.n_out + t0 + c;
        const bool ok = c < nt && poly < n_polys;
        s_out[c] = ok ? out.row(r, log_n) : nullptr;
        s_p[c] = ok ? out.prime(r) : 0;
        s_wn[c] = ok && rnd ? tab.negq_mont[t0 + c] : 0;
    }
    __syncthreads();
    if (poly >= n_polys) return;
    for (int ci = 0; ci < BCONV_CPT; ci++) {
        const size_t k = ((size_t)blockIdx.x * BCONV_CPT + ci) * blockDim.x + threadIdx.x;
        if (k >= n) return;
        u32 acc[BCONV_CHUNK][4];
#pragma unroll
        for (int c = 0; c < BCONV_CHUNK; c++) acc[c][0] = acc[c][1] = acc[c][2] = acc[c][3] = 0;
        u64 flo = 0;  // fraction of sum_a y_a / q_a in units of 2^-64
        u32 fhi = 0;  // its integer part
#pragma unroll 2
        for (int a = 0; a < tab.n_in; a++) {
            const u64 y = shoup_mul(s_in[a][k], s_qi[a], s_qis[a], s_q[a]);
            if (RND) {  // floor(y m / 2^64) with m = floor(2^128 / q_a) < 2^128: (y / q_a) 2^64 - [0, 2)
                const u64 t = __umul64hi(y, s_mlo[a]) + y * s_mhi[a];
                flo += t;
                fhi += flo < t ? 1u : 0u;
            }
            const u32 y0 = (u32)y, y1 = (u32)(y >> 32);
#pragma unroll
            for (int c = 0; c < BCONV_CHUNK; c++) {
                const u64 w = s_w[a * BCONV_CHUNK + c];
                mac128_words(acc[c][0], acc[c][1], acc[c][2], acc[c][3], y0, y1, (u32)w, (u32)(w >> 32));
            }
        }
        if (RND) {  // + v (-Q): v <= n_in, one more term below 2^66
            constexpr u64 half = 1ull << 63, win = 1ull << 20;
            u32 v = fhi + (flo > half ? 1u : 0u);
            if ((flo > half ? flo - half : half - flo) < win)
                v = fhi + bconv_above_half(s_in, s_pidx, k, tab.n_in, tab, pc);
#pragma unroll
            for (int c = 0; c < BCONV_CHUNK; c++)
                mac128_words(acc[c][0], acc[c][1], acc[c][2], acc[c][3], v, 0u, (u32)s_wn[c], (u32)(s_wn[c] >> 32));
        }
#pragma unroll
        for (int c = 0; c < BCONV_CHUNK; c++) {
            if (c < nt) {
                const int p = s_p[c];
                const u64 lo = ((u64)acc[c][1] << 32) | acc[c][0], hi = ((u64)acc[c][3] << 32) | acc[c][2];
                s_out[c][k] = mont_reduce_wide(lo, hi, pc.m[p], pc.mont_qinv[p]);
            }
        }
    }
}
// the rounding variant at seven blocks per SM (72 registers instead of 88)
template <bool RND>
__global__ void __launch_bounds__(128, RND ? 7 : 4) k_bconv(Rows out, Rows in, BConvTab tab, int n_polys, int log_n) {
    bconv_block<RND>(out, in, tab, n_polys, log_n, blockIdx.y);
}
// several conversions of one shape in one launch (blockIdx.z selects one):
// the digits of a ModUp
__global__ void __launch_bounds__(128, 7) k_bconv_set(BConvSet set, int n_polys, int log_n) {
    const int j = blockIdx.z;
    const int n_chunks = (set.tab[j].n_out + BCONV_CHUNK - 1) / BCONV_CHUNK;
    if ((int)blockIdx.y >= n_chunks * n_polys) return;  // this conversion has fewer output chunks
    bconv_block<false>(set.out[j], set.in[j], set.tab[j], n_polys, log_n, blockIdx.y);
}
void bconv_set(const BConvSet &set, int n_polys, int log_n, cudaStream_t s) {
    if (set.n < 1 || set.n > BCONV_SET_MAX) throw Error{HE_EINVAL, "basis conversion set: 1..8 conversions"};
    int max_chunks = 0;
    double bytes = 0;
    for (int j = 0; j < set.n; j++) {
        if (set.tab[j].n_in > BCONV_MAX_IN || set.tab[j].inv_fix)
            throw Error{HE_EINVAL, "basis conversion set: more than 16 primes or a rounding table"};
        max_chunks = std::max(max_chunks, (set.tab[j].n_out + BCONV_CHUNK - 1) / BCONV_CHUNK);
        bytes += 8.0 * (set.tab[j].n_in + set.tab[j].n_out) * (double)n_polys * (double)(1 << log_n);
    }
    const size_t n = (size_t)1 << log_n;
    dim3 grid((unsigned)((n + 127) / 128), (unsigned)(max_chunks * n_polys), (unsigned)set.n);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    prof_begin(PROF_BCONV, s);
    k_bconv_set<<<grid, 128, 0, s>>>(set, n_polys, log_n);
    prof_end(PROF_BCONV, s, bytes);
}
void bconv(const Rows &out, const Rows &in, const BConvTab &tab, int n_polys, int log_n, cudaStream_t s) {
    if (tab.n_in > BCONV_MAX_IN) throw Error{HE_EINVAL, "basis conversion from more than 16 primes"};
    const size_t n = (size_t)1 << log_n;
    const int n_chunks = (tab.n_out + BCONV_CHUNK - 1) / BCONV_CHUNK;
    dim3 grid((unsigned)((n + 128 * BCONV_CPT - 1) / (128 * BCONV_CPT)), (unsigned)(n_chunks * n_polys));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    prof_begin(PROF_BCONV, s);
    if (tab.inv_fix) k_bconv<true><<<grid, 128, 0, s>>>(out, in, tab, n_polys, log_n);
    else k_bconv<false><<<grid, 128, 0, s>>>(out, in, tab, n_polys, log_n);
    prof_end(PROF_BCONV, s, 8.0 * (tab.n_in + tab.n_out) * (double)n_polys * (double)n);
}

// Batch members are processed KS_MB at a time per thread, so that every key
// word loaded serves KS_MB members from registers (KS_MB = 1 for one member).
template <int KS_MB, bool LIFT>
__global__ void __launch_bounds__(EW_T) k_keyswitch_inner(KeyIP kp, int log_n, KeyLift lf) {
    const PrimeConsts &pc = c_pcs[kp.slot];
    const int t = blockIdx.y, b0 = blockIdx.z * KS_MB, nb = min(KS_MB, kp.batch - b0);
    const int p = t < kp.l1 ? t : kp.nq + (t - kp.l1);
    const u64 q = pc.m[p].q, qn = pc.mont_qinv[p];
    const int jt = t < kp.l1 ? t / kp.alpha : -1;
    const size_t row = (size_t)t << log_n;
    EW_PAIRS_FOR(k, log_n) {
        size_t s0 = k, s1 = k + 1;
        if (kp.galois) {  // hoisted rotation: position k reads the automorphism's source position
            s0 = automorph_src((u32)k, kp.galois, log_n);
            s1 = automorph_src((u32)k + 1, kp.galois, log_n);
        }
        // keys are in Montgomery form (times 2^64): the beta products are summed
        // in 128 bits (< beta q^2 < q 2^64) and reduced once
        u64 acc[KS_MB][8];
#pragma unroll
        for (int m = 0; m < KS_MB; m++)
#pragma unroll
            for (int i = 0; i < 8; i++) acc[m][i] = 0;
        for (int j = 0; j < kp.beta; j++) {
            const ulonglong2 kb = ld2(kp.key + ((((size_t)(2 * j) * kp.key_limbs + p)) << log_n) + k);
            const ulonglong2 ka = ld2(kp.key + ((((size_t)(2 * j + 1) * kp.key_limbs + p)) << log_n) + k);
#pragma unroll
            for (int m = 0; m < KS_MB; m++) {
                if (m >= nb) break;
                const size_t mb = (size_t)(b0 + m);
                const u64 *xs = (j == jt) ? kp.d_ntt + mb * kp.d_stride + row
                                          : kp.ext + mb * kp.ext_stride + (((size_t)j * kp.n_rows + t) << log_n);
                u64 x0, x1;
                if (kp.galois) {
                    x0 = xs[s0];
                    x1 = xs[s1];
                } else {
                    const ulonglong2 xv = ld2(xs + k);
                    x0 = xv.x;
                    x1 = xv.y;
                }
                mac128(acc[m][0], acc[m][1], x0, kb.x);
                mac128(acc[m][2], acc[m][3], x1, kb.y);
                mac128(acc[m][4], acc[m][5], x0, ka.x);
                mac128(acc[m][6], acc[m][7], x1, ka.y);
            }
        }
#pragma unroll
        for (int m = 0; m < KS_MB; m++) {
            if (m >= nb) break;
            u64 *acc_m = kp.acc + (size_t)(b0 + m) * kp.acc_stride;
            if constexpr (!LIFT) {
                st2(acc_m + row + k, mont_reduce(acc[m][0], acc[m][1], q, qn), mont_reduce(acc[m][2], acc[m][3], q, qn));
                st2(acc_m + (((size_t)kp.n_rows + t) << log_n) + k, mont_reduce(acc[m][4], acc[m][5], q, qn),
                    mont_reduce(acc[m][6], acc[m][7], q, qn));
            } else {
                u64 r0 = mont_reduce(acc[m][0], acc[m][1], q, qn), r1 = mont_reduce(acc[m][2], acc[m][3], q, qn);
                u64 r2 = mont_reduce(acc[m][4], acc[m][5], q, qn), r3 = mont_reduce(acc[m][6], acc[m][7], q, qn);
                if (t < kp.l1) {  // + P d_k (P = 0 mod the special primes)
                    const u64 w = lf.pmod.v[p], ws = lf.pmod.s[p];
                    const u64 *dk = lf.d + row;
                    const ulonglong2 u0 = ld2(dk + k), u1 = ld2(dk + lf.poly_stride + k);
                    r0 = add_mod(r0, shoup_mul(u0.x, w, ws, q), q);
                    r1 = add_mod(r1, shoup_mul(u0.y, w, ws, q), q);
                    r2 = add_mod(r2, shoup_mul(u1.x, w, ws, q), q);
                    r3 = add_mod(r3, shoup_mul(u1.y, w, ws, q), q);
                }
                st2(acc_m + row + k, r0, r1);
                st2(acc_m + (((size_t)kp.n_rows + t) << log_n) + k, r2, r3);
            }
        }
    }
}
void keyswitch_inner(const KeyIP &k, int log_n, cudaStream_t s, const KeyLift *lift) {
    need16(k.d_ntt);
    need16(k.ext);
    need16(k.key);
    need16(k.acc);
    if (lift) {
        need16(lift->d);
        if ((lift->poly_stride & 1) || k.batch != 1) throw Error{HE_EINVAL, "key inner product: bad lift"};
    }
    if (k.batch < 1 || (k.batch > 1 && ((k.d_stride | k.ext_stride | k.acc_stride) & 1)))
        throw Error{HE_EINVAL, "key inner product: bad batch layout"};
    constexpr int MB = 4;
    dim3 grid = ew_grid(k.n_rows, log_n);
    grid.z = (unsigned)(k.batch == 1 ? 1 : (k.batch + MB - 1) / MB);
    prof_begin(PROF_KS_INNER, s);
    static const KeyLift none{};
    if (lift) k_keyswitch_inner<1, true><<<grid, EW_T, 0, s>>>(k, log_n, *lift);
    else if (k.batch == 1) k_keyswitch_inner<1, false><<<grid, EW_T, 0, s>>>(k, log_n, none);
    else k_keyswitch_inner<MB, false><<<grid, EW_T, 0, s>>>(k, log_n, none);
    // algorithmic bytes: the beta key digits (b and a) once, then per member the
    // beta input digits and the two outputs (and the two lifted polynomials)
    prof_end(PROF_KS_INNER, s,
             8.0 * (double)(1 << log_n) *
                 ((2.0 * k.beta + (k.beta + 2.0) * k.batch) * (double)k.n_rows + (lift ? 2.0 * k.l1 : 0.0)));
}

// Hoisted rotate-and-sum stage (see KeyIPMulti): for each key r the beta
// digit products (read through the automorphism's permutation) are summed in
// 128 bits and reduced once, then added mod q across keys; the Q rows take
// P * (c0 + sum_r sigma_r(c0)) on top, so that ModDown returns the rotations'
// c0 parts exactly.  MB members per thread share every key word loaded.
template <int MB>
__global__ void __launch_bounds__(EW_T) k_keyswitch_inner_multi(KeyIPMulti kp, int log_n) {
    const PrimeConsts &pc = c_pcs[kp.slot];
    const int t = blockIdx.y, b0 = blockIdx.z * MB, nb = min(MB, kp.batch - b0);
    const bool q_row = t < kp.l1;
    const int p = q_row ? t : kp.nq + (t - kp.l1);
    const u64 q = pc.m[p].q, qn = pc.mont_qinv[p];
    const int jt = q_row ? t / kp.alpha : -1;
    const size_t row = (size_t)t << log_n;
    EW_PAIRS_FOR(k, log_n) {
        u64 sum[MB][4];  // (b part at k, k+1; a part at k, k+1)
#pragma unroll
        for (int m = 0; m < MB; m++)
#pragma unroll
            for (int i = 0; i < 4; i++) sum[m][i] = 0;
        for (int r = 0; r < kp.n_keys; r++) {
            const size_t s0 = automorph_src((u32)k, kp.gal[r], log_n), s1 = automorph_src((u32)k + 1, kp.gal[r], log_n);
            const u64 *key = kp.keys[r];
            u64 acc[MB][8];
#pragma unroll
            for (int m = 0; m < MB; m++)
#pragma unroll
                for (int i = 0; i < 8; i++) acc[m][i] = 0;
            for (int j = 0; j < kp.beta; j++) {
                const ulonglong2 kb = ld2(key + ((((size_t)(2 * j) * kp.key_limbs + p)) << log_n) + k);
                const ulonglong2 ka = ld2(key + ((((size_t)(2 * j + 1) * kp.key_limbs + p)) << log_n) + k);
#pragma unroll
                for (int m = 0; m < MB; m++) {
                    if (m >= nb) break;
                    const size_t mb = (size_t)(b0 + m);
                    const u64 *xs = (j == jt) ? kp.d_ntt + mb * kp.d_stride + row
                                              : kp.ext + mb * kp.ext_stride + (((size_t)j * kp.n_rows + t) << log_n);
                    const u64 x0 = xs[s0], x1 = xs[s1];
                    mac128(acc[m][0], acc[m][1], x0, kb.x);
                    mac128(acc[m][2], acc[m][3], x1, kb.y);
                    mac128(acc[m][4], acc[m][5], x0, ka.x);
                    mac128(acc[m][6], acc[m][7], x1, ka.y);
                }
            }
#pragma unroll
            for (int m = 0; m < MB; m++)
#pragma unroll
                for (int i = 0; i < 4; i++) sum[m][i] = add_mod(sum[m][i], mont_reduce(acc[m][2 * i], acc[m][2 * i + 1], q, qn), q);
        }
        if (q_row) {  // + P (c0 + sum_r sigma_r(c0)); P = 0 on the special rows
            const u64 w = kp.pmod.v[p], ws = kp.pmod.s[p];
#pragma unroll
            for (int m = 0; m < MB; m++) {
                if (m >= nb) break;
                const u64 *c = kp.c0 + (size_t)(b0 + m) * kp.c0_stride + row;
                const ulonglong2 cv = ld2(c + k);
                u64 y0 = cv.x, y1 = cv.y;
                for (int r = 0; r < kp.n_keys; r++) {
                    y0 = add_mod(y0, c[automorph_src((u32)k, kp.gal[r], log_n)], q);
                    y1 = add_mod(y1, c[automorph_src((u32)k + 1, kp.gal[r], log_n)], q);
                }
                sum[m][0] = add_mod(sum[m][0], shoup_mul(y0, w, ws, q), q);
                sum[m][1] = add_mod(sum[m][1], shoup_mul(y1, w, ws, q), q);
            }
        }
#pragma unroll
        for (int m = 0; m < MB; m++) {
            if (m >= nb) break;
            u64 *acc_m = kp.acc + (size_t)(b0 + m) * kp.acc_stride;
            st2(acc_m + row + k, sum[m][0], sum[m][1]);
            st2(acc_m + (((size_t)kp.n_rows + t) << log_n) + k, sum[m][2], sum[m][3]);
        }
    }
}
void keyswitch_inner_multi(const KeyIPMulti &k, int log_n, cudaStream_t s) {
    need16(k.d_ntt);
    need16(k.ext);
    need16(k.c0);
    need16(k.acc);
    if (k.n_keys < 1 || k.n_keys > ROTSUM_MAX_KEYS) throw Error{HE_EINVAL, "hoisted stage: 1..15 keys"};
    for (int r = 0; r < k.n_keys; r++) need16(k.keys[r]);
    if (k.batch < 1 || (k.batch > 1 && ((k.d_stride | k.ext_stride | k.acc_stride | k.c0_stride) & 1)))
        throw Error{HE_EINVAL, "hoisted stage: bad batch layout"};
    constexpr int MB = 2;
    dim3 grid = ew_grid(k.n_rows, log_n);
    grid.z = (unsigned)(k.batch == 1 ? 1 : (k.batch + MB - 1) / MB);
    prof_begin(PROF_KS_INNER, s);
    if (k.batch == 1) k_keyswitch_inner_multi<1><<<grid, EW_T, 0, s>>>(k, log_n);
    else k_keyswitch_inner_multi<MB><<<grid, EW_T, 0, s>>>(k, log_n);
    // algorithmic bytes: every key digit (b and a) once, per member the beta
    // input digits, c0 on the Q rows and the two outputs
    prof_end(PROF_KS_INNER, s,
             8.0 * (double)(1 << log_n) *
                 ((2.0 * k.beta * k.n_keys + (k.beta + 2.0) * k.batch) * (double)k.n_rows + (double)k.batch * k.l1));
}

__global__ void __launch_bounds__(EW_T) k_moddown_finish(Rows out, Rows acc, Rows conv, ScalarTab pinv,
                                                         Rows add_to, int add_mask, int log_n) {
    const int r = blockIdx.y, p = out.prime(r);
    const u64 q = c_pcs[out.slot].m[p].q, w = pinv.v[p], ws = pinv.s[p];
    const bool add = (add_mask >> ((r / out.lpp) & 1)) & 1;  // bit k: polynomial k of every member
    u64 *o = out.row(r, log_n);
    const u64 *pa = acc.row(r, log_n), *pc = conv.row(r, log_n);
    const u64 *pd = add ? add_to.row(r, log_n) : nullptr;
    EW_PAIRS_FOR(k, log_n) {
        const ulonglong2 a = ld2(pa + k), c = ld2(pc + k);
        u64 v0 = shoup_mul(sub_mod(a.x, c.x, q), w, ws, q), v1 = shoup_mul(sub_mod(a.y, c.y, q), w, ws, q);
        if (add) {
            const ulonglong2 d = ld2(pd + k);
            v0 = add_mod(v0, d.x, q);
            v1 = add_mod(v1, d.y, q);
        }
        st2(o + k, v0, v1);
    }
}
void moddown_finish(const Rows &out, const Rows &acc, const Rows &conv, const ScalarTab &pinv, int n_rows,
                    const Rows &add_to, int add_mask, int log_n, cudaStream_t s) {
    need16(out);
    need16(acc);
    need16(conv);
    if (add_mask) need16(add_to);
    k_moddown_finish<<<ew_grid(n_rows, log_n), EW_T, 0, s>>>(out, acc, conv, pinv, add_to, add_mask, log_n);
}

// ------------------------------------------------------------------ rescale / mod raise
// centred representative of v mod q_src (v in [0, q_src)) reduced mod m
__device__ __forceinline__ u64 centred_mod(u64 v, u64 q_src, u64 q_src_mod_m, const ModQ &m) {
    u64 vm = barrett_reduce(v, 0, m);
    if (v > (q_src - 1) / 2) vm = sub_mod(vm, q_src_mod_m, m.q);
    return vm;
}
// MUL: the rescaled ciphertext is K a (K mod q_l in kl, its Shoup companion
// kls): the last limb's coefficients are multiplied by K before the lift
// (the INTT is linear, so K INTT(a_l) = INTT(K a_l) mod q_l)
template <bool MUL>
__global__ void __launch_bounds__(EW_T) k_rescale_lift(Rows lift, const u64 *last, u64 ql, int l, u64 kl, u64 kls,
                                                       int log_n) {
    const int r = blockIdx.y;  // polynomial r / l, target prime r % l
    const int poly = r / l, i = r % l;
    const ModQ m = c_pcs[lift.slot].m[i];
    const u64 qlm = barrett_reduce(ql, 0, m);
    const u64 *src = last + ((size_t)poly << log_n);
    u64 *o = lift.row(r, log_n);
    EW_PAIRS_FOR(k, log_n) {
        ulonglong2 v = ld2(src + k);
        if (MUL) {
            v.x = shoup_mul(v.x, kl, kls, ql);
            v.y = shoup_mul(v.y, kl, kls, ql);
        }
        st2(o + k, centred_mod(v.x, ql, qlm, m), centred_mod(v.y, ql, qlm, m));
    }
}
void rescale_lift(const Rows &lift, const u64 *last, int n_polys, u64 ql, int l, int log_n, cudaStream_t s,
                  const ScalarTab *kmul) {
    need16(lift);
    need16(last);
    if (kmul)
        k_rescale_lift<true><<<ew_grid(n_polys * l, log_n), EW_T, 0, s>>>(lift, last, ql, l, kmul->v[l], kmul->s[l],
                                                                          log_n);
    else
        k_rescale_lift<false><<<ew_grid(n_polys * l, log_n), EW_T, 0, s>>>(lift, last, ql, l, 0, 0, log_n);
}
// out = (K a - lift) q_l^-1 (MUL; else K = 1)
template <bool MUL>
__global__ void __launch_bounds__(EW_T) k_rescale_finish(Rows out, Rows in, Rows lift, ScalarTab qlinv, ScalarTab kmul,
                                                         int log_n) {
    const int r = blockIdx.y, p = out.prime(r);
    const u64 q = c_pcs[out.slot].m[p].q, w = qlinv.v[p], ws = qlinv.s[p];
    u64 *o = out.row(r, log_n);
    const u64 *x = in.row(r, log_n), *y = lift.row(r, log_n);
    EW_PAIRS_FOR(k, log_n) {
        ulonglong2 a = ld2(x + k);
        const ulonglong2 b = ld2(y + k);
        if (MUL) {
            a.x = shoup_mul(a.x, kmul.v[p], kmul.s[p], q);
            a.y = shoup_mul(a.y, kmul.v[p], kmul.s[p], q);
        }
        st2(o + k, shoup_mul(sub_mod(a.x, b.x, q), w, ws, q), shoup_mul(sub_mod(a.y, b.y, q), w, ws, q));
    }
}
void rescale_finish(const Rows &out, const Rows &in, const Rows &lift, const ScalarTab &qlinv, int n_rows,
                    int log_n, cudaStream_t s, const ScalarTab *kmul) {
    need16(out);
    need16(in);
    need16(lift);
    if (kmul)
        k_rescale_finish<true><<<ew_grid(n_rows, log_n), EW_T, 0, s>>>(out, in, lift, qlinv, *kmul, log_n);
    else
        k_rescale_finish<false><<<ew_grid(n_rows, log_n), EW_T, 0, s>>>(out, in, lift, qlinv, qlinv, log_n);
}
__global__ void __launch_bounds__(EW_T) k_modraise_lift(Rows out, const u64 *src0, u64 q0, int log_n) {
    const int r = blockIdx.y;
    const ModQ m = c_pcs[out.slot].m[out.prime(r)];
    const u64 q0m = barrett_reduce(q0, 0, m);
    const u64 *src = src0 + ((size_t)(r / out.lpp) << log_n);
    u64 *o = out.row(r, log_n);
    EW_PAIRS_FOR(k, log_n) {
        const ulonglong2 v = ld2(src + k);
        st2(o + k, centred_mod(v.x, q0, q0m, m), centred_mod(v.y, q0, q0m, m));
    }
}
void modraise_lift(const Rows &out, const u64 *src, u64 q0, int n_rows, int log_n, cudaStream_t s) {
    need16(out);
    need16(src);
    k_modraise_lift<<<ew_grid(n_rows, log_n), EW_T, 0, s>>>(out, src, q0, log_n);
}

// ------------------------------------------------------------------ sampling
// (grid-stride loops over flat element indices: these kernels run once per
// encryption, decryption or key generation)
#define EW_LOOP(total)                                                                 \
    for (size_t gi = (size_t)blockIdx.x * blockDim.x + threadIdx.x; gi < (total);      \
         gi += (size_t)gridDim.x * blockDim.x)

__device__ __forceinline__ void philox4x32_10(u32 c[4], u32 k0, u32 k1) {
    const u32 M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r) { k0 += W0; k1 += W1; }
        u32 hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
        u32 hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
        u32 n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

__global__ void k_sample_uniform(Rows out, int n_rows, u64 seed, u32 object, u32 domain, int log_n) {
    const PrimeConsts &pc = c_pcs[out.slot];
    const size_t total = (size_t)n_rows << log_n, mask = ((size_t)1 << log_n) - 1;
    EW_LOOP(total) {
        int r = (int)(gi >> log_n);
        u32 k = (u32)(gi & mask);
        int p = out.prime(r);
        u32 c[4] = {k, (u32)p, object, domain};
        philox4x32_10(c, (u32)seed, (u32)(seed >> 32));
        const ModQ &m = pc.m[p];
        u64 lo = ((u64)c[1] << 32) | c[0], hi = ((u64)c[3] << 32) | c[2];
        u64 h = mul_mod(barrett_reduce(hi, 0, m), pc.r64[p], m);
        out.row(r, log_n)[k] = add_mod(h, barrett_reduce(lo, 0, m), m.q);
    }
}
void sample_uniform(const Rows &out, int n_rows, u64 seed, u32 object, u32 domain, int log_n, cudaStream_t s) {
    size_t t = (size_t)n_rows << log_n;
    k_sample_uniform<<<grid_for(t, 256), 256, 0, s>>>(out, n_rows, seed, object, domain, log_n);
}

__device__ __forceinline__ u64 intd_mod(double x, const ModQ &m) {
    // x integer-valued; exact residue for any magnitude
    if (fabs(x) < 9.2e18) {
        i64 v = (i64)x;
        u64 a = v < 0 ? (u64)(-v) : (u64)v;
        u64 r = barrett_reduce(a, 0, m);
        return (v < 0 && r) ? m.q - r : r;
    }
    int e;
    double mant = frexp(x, &e);
    i64 mi = (i64)ldexp(mant, 53);
    e -= 53;
    u64 a = mi < 0 ? (u64)(-mi) : (u64)mi;
    u64 r = barrett_reduce(a, 0, m);
    // r * 2^e mod q by repeated doubling (e < 1024)
    for (int i = 0; i < e; i++) r = add_mod(r, r, m.q);
    return (mi < 0 && r) ? m.q - r : r;
}

__global__ void k_sample_error_plus(Rows out, int n_rows, u64 seed, u32 object, u32 domain, const double *pt,
                                    int log_n) {
    const PrimeConsts &pc = c_pcs[out.slot];
    const size_t n = (size_t)1 << log_n;
    EW_LOOP(n) {
        u32 k = (u32)gi;
        u32 c[4] = {k, 0u, object, domain};
        philox4x32_10(c, (u32)seed, (u32)(seed >> 32));
        u64 u = ((u64)c[1] << 32) | c[0];
        i64 mag = 0;
        for (int i = 0; i < pc.ncdt; i++) mag += (pc.cdt[i] <= u);
        i64 e = (c[2] & 1) ? -mag : mag;
        double mv = pt ? pt[k] : 0.0;
        for (int r = 0; r < n_rows; r++) {
            const ModQ &m = pc.m[out.prime(r)];
            u64 em = e < 0 ? (e == 0 ? 0 : m.q - (u64)(-e)) : (u64)e;
            u64 v = pt ? add_mod(em, intd_mod(mv, m), m.q) : em;
            out.row(r, log_n)[k] = v;
        }
    }
}
void sample_error_plus(const Rows &out, int n_rows, u64 seed, u32 object, u32 domain, const double *pt, int log_n,
                       cudaStream_t s) {
    size_t t = (size_t)1 << log_n;
    k_sample_error_plus<<<grid_for(t, 256), 256, 0, s>>>(out, n_rows, seed, object, domain, pt, log_n);
}

__global__ void k_load_small(Rows out, int n_rows, const int8_t *v, int log_n) {
    const PrimeConsts &pc = c_pcs[out.slot];
    const size_t total = (size_t)n_rows << log_n, mask = ((size_t)1 << log_n) - 1;
    EW_LOOP(total) {
        int r = (int)(gi >> log_n);
        size_t k = gi & mask;
        u64 q = pc.m[out.prime(r)].q;
        int x = v[k];
        out.row(r, log_n)[k] = x < 0 ? q - (u64)(-x) : (u64)x;
    }
}
void load_small(const Rows &out, int n_rows, const int8_t *v, int log_n, cudaStream_t s) {
    size_t t = (size_t)n_rows << log_n;
    k_load_small<<<grid_for(t, 256), 256, 0, s>>>(out, n_rows, v, log_n);
}
__global__ void k_load_intd(Rows out, int n_rows, const double *v, int log_n) {
    const PrimeConsts &pc = c_pcs[out.slot];
    const size_t total = (size_t)n_rows << log_n, mask = ((size_t)1 << log_n) - 1;
    EW_LOOP(total) {
        int r = (int)(gi >> log_n);
        size_t k = gi & mask;
        out.row(r, log_n)[k] = intd_mod(v[k], pc.m[out.prime(r)]);
    }
}
void load_intd(const Rows &out, int n_rows, const double *v, int log_n, cudaStream_t s) {
    size_t t = (size_t)n_rows << log_n;
    k_load_intd<<<grid_for(t, 256), 256, 0, s>>>(out, n_rows, v, log_n);
}

// ------------------------------------------------------------------ encoding (float64)
// Slot j sits at DFT index l(j) = (5^j mod 2N - 1)/4 of the length-h (= N/2)
// transform of the twisted coefficients b_k = (m_k + i m_{k+h}) zeta^k.
__device__ __forceinline__ u32 brv_bits(u32 x, int bits) { return __brev(x) >> (32 - bits); }

__global__ void k_enc_scatter(Cplx *A, const double *re, const double *im, int n_slots, const int *slot_l,
                              int log_h) {
    const size_t h = (size_t)1 << log_h;
    EW_LOOP(h) {
        int j = (int)gi;
        Cplx z = {0.0, 0.0};
        if (j < n_slots) { z.re = re[j]; z.im = im ? im[j] : 0.0; }
        A[brv_bits((u32)slot_l[j], log_h)] = z;  // bit-reversed for the DIT stages
    }
}
// one radix-2 decimation-in-time stage; sign = -1 forward (e^{-2 pi i}), +1 backward
__global__ void k_fft_stage(Cplx *a, int log_h, int len, int sign) {
    const size_t h = (size_t)1 << log_h;
    const int half = len >> 1;
    EW_LOOP(h / 2) {
        size_t blk = gi / half, k = gi % half;
        size_t i0 = blk * len + k, i1 = i0 + half;
        double sn, cs;
        sincospi((double)sign * 2.0 * (double)k / (double)len, &sn, &cs);
        Cplx u = a[i0], v = a[i1];
        double vr = v.re * cs - v.im * sn, vi = v.re * sn + v.im * cs;
        a[i0] = {u.re + vr, u.im + vi};
        a[i1] = {u.re - vr, u.im - vi};
    }
}
__global__ void k_enc_untwist(double *out, const Cplx *b, double scale, int log_n) {
    const size_t n = (size_t)1 << log_n, h = n / 2;
    EW_LOOP(h) {
        size_t k = gi;
        double sn, cs;
        sincospi(-(double)k / (double)n, &sn, &cs);
        double f = scale / (double)h;
        double wr = (b[k].re * cs - b[k].im * sn) * f;
        double wi = (b[k].re * sn + b[k].im * cs) * f;
        out[k] = rint(wr);
        out[k + h] = rint(wi);
    }
}
void encode_slots(double *out_coeff, const double *re, const double *im, int n_slots, double scale,
                  const int *slot_l, Cplx *work, int log_n, cudaStream_t s) {
    int log_h = log_n - 1;
    size_t h = (size_t)1 << log_h;
    k_enc_scatter<<<grid_for(h, 256), 256, 0, s>>>(work, re, im, n_slots, slot_l, log_h);
    for (int len = 2; len <= (int)h; len <<= 1)
        k_fft_stage<<<grid_for(h / 2, 256), 256, 0, s>>>(work, log_h, len, -1);
    k_enc_untwist<<<grid_for(h, 256), 256, 0, s>>>(out_coeff, work, scale, log_n);
}

__global__ void k_dec_twist(Cplx *A, const double *m, int log_n) {
    const size_t n = (size_t)1 << log_n, h = n / 2;
    EW_LOOP(h) {
        size_t k = gi;
        double sn, cs;
        sincospi((double)k / (double)n, &sn, &cs);
        double wr = m[k], wi = m[k + h];
        A[brv_bits((u32)k, log_n - 1)] = {wr * cs - wi * sn, wr * sn + wi * cs};
    }
}
__global__ void k_dec_gather(double *re, double *im, const Cplx *A, double scale, const int *slot_l, int log_n) {
    const size_t h = (size_t)1 << (log_n - 1);
    EW_LOOP(h) {
        Cplx v = A[slot_l[gi]];
        re[gi] = v.re / scale;
        if (im) im[gi] = v.im / scale;
    }
}
void decode_coeffs(double *re, double *im, const double *coeff, double scale, const int *slot_l, Cplx *work,
                   int log_n, cudaStream_t s) {
    size_t h = (size_t)1 << (log_n - 1);
    k_dec_twist<<<grid_for(h, 256), 256, 0, s>>>(work, coeff, log_n);
    for (int len = 2; len <= (int)h; len <<= 1)
        k_fft_stage<<<grid_for(h / 2, 256), 256, 0, s>>>(work, log_n - 1, len, +1);
    k_dec_gather<<<grid_for(h, 256), 256, 0, s>>>(re, im, work, scale, slot_l, log_n);
}

// correctly rounded unsigned 128-bit -> double
__device__ __forceinline__ double u128_to_double(u64 hi, u64 lo) {
    if (hi == 0) return __ull2double_rn(lo);
    int lz = __clzll(hi);
    int shift = 64 - lz;  // bits beyond the top 64
    u64 top, sticky;
    if (shift == 64) { top = hi; sticky = lo != 0; }
    else { top = (hi << lz) | (lo >> shift); sticky = (lo << (64 - shift)) != 0; }
    top |= sticky;
    return ldexp(__ull2double_rn(top), shift);
}
__global__ void k_crt2(double *out, const u64 *r0, const u64 *r1, u64 q0, u64 q1, u64 q0inv, int two, int log_n,
                       int slot) {
    const PrimeConsts &pc = c_pcs[slot];
    const size_t n = (size_t)1 << log_n;
    EW_LOOP(n) {
        u64 x0 = r0[gi];
        if (!two) {
            out[gi] = x0 > q0 / 2 ? -(double)(q0 - x0) : (double)x0;
            continue;
        }
        const ModQ &m1 = pc.m[1];
        u64 x1 = r1[gi];
        u64 k = mul_mod(sub_mod(x1, barrett_reduce(x0, 0, m1), q1), q0inv, m1);
        // v = x0 + q0*k < q0 q1
        u64 lo = q0 * k, hi = __umul64hi(q0, k);
        u64 lo2 = lo + x0;
        hi += (lo2 < lo);
        lo = lo2;
        // Q = q0 q1
        u64 Qlo = q0 * q1, Qhi = __umul64hi(q0, q1);
        // half = Q/2 (floor)
        u64 Hlo = (Qlo >> 1) | (Qhi << 63), Hhi = Qhi >> 1;
        bool neg = (hi > Hhi) || (hi == Hhi && lo > Hlo);
        if (neg) {
            u64 dlo = Qlo - lo, dhi = Qhi - hi - (Qlo < lo);
            out[gi] = -u128_to_double(dhi, dlo);
        } else {
            out[gi] = u128_to_double(hi, lo);
        }
    }
}
void crt_to_double(double *out, const u64 *r0, const u64 *r1, u64 q0, u64 q1, u64 q0inv_mod_q1, int two, int log_n,
                   cudaStream_t s) {
    size_t t = (size_t)1 << log_n;
    k_crt2<<<grid_for(t, 256), 256, 0, s>>>(out, r0, r1, q0, q1, q0inv_mod_q1, two, log_n, t_slot);
}

__global__ void k_decrypt_rows(Rows out, Rows c0, Rows c1, Rows sk, int n_rows, int log_n) {
    const PrimeConsts &pc = c_pcs[out.slot];
    const size_t total = (size_t)n_rows << log_n, mask = ((size_t)1 << log_n) - 1;
    EW_LOOP(total) {
        int r = (int)(gi >> log_n);
        size_t k = gi & mask;
        const ModQ &m = pc.m[out.prime(r)];
        out.row(r, log_n)[k] = add_mod(c0.row(r, log_n)[k], mul_mod(c1.row(r, log_n)[k], sk.row(r, log_n)[k], m), m.q);
    }
}
void decrypt_rows(const Rows &out, const Rows &c0, const Rows &c1, const Rows &sk, int n_rows, int log_n,
                  cudaStream_t s) {
    size_t t = (size_t)n_rows << log_n;
    k_decrypt_rows<<<grid_for(t, 256), 256, 0, s>>>(out, c0, c1, sk, n_rows, log_n);
}

}  // namespace he
