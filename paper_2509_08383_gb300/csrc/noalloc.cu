// A key-switch entry point that allocates nothing.
//
// cudaMalloc and cudaFree synchronise the whole device and can fail when
// memory is fragmented, so a caller on a latency-critical serving path, or one
// whose device memory is entirely reserved by another allocator (for example a
// process in which PyTorch's caching allocator owns the GPU), cannot obtain
// scratch memory on demand.  This entry point takes its scratch from one
// file-scope device array of HE_NOALLOC_SCRATCH_WORDS 64-bit words (32 MiB),
// which every GPU that loads the library holds until the process exits.  The
// paper has no counterpart; it is a deployment convenience.
#include <cstring>
#include <mutex>

#include "context.h"

#define HE_NOALLOC_SCRATCH_WORDS (1ull << 22)

static __device__ __align__(256) u64 g_noalloc_scratch[HE_NOALLOC_SCRATCH_WORDS];

namespace {
std::mutex g_noalloc_mu;
u64 *g_noalloc_ptr[64];  // device address of the array, per device (filled on first use)
}  // namespace

using namespace he;

extern "C" int he_keyswitch_noalloc(he_ctx *cx, const uint64_t *d, uint32_t level, uint64_t g, uint64_t *out) {
    if (!cx || !d || !out) return HE_EINVAL;
    t_slot = cx->slot;
    try {
        if ((int)level >= cx->nq) throw Error{HE_EINVAL, "level out of range"};
        const KeyDev *key = find_key(cx, g);
        if (!key) throw Error{HE_ENOKEY, "key not generated"};
        const int l = (int)level;
        const LevelTabs &T = cx->lv[l];
        const size_t N = cx->N();
        const size_t w_coef = (size_t)(l + 1) * N, w_ext = (size_t)T.beta * T.n_ext * N;
        const size_t w_acc = (size_t)2 * T.n_ext * N, w_conv = (size_t)2 * (l + 1) * N;
        const size_t need = w_coef + w_ext + w_acc + w_conv;
        if (need > HE_NOALLOC_SCRATCH_WORDS)
            throw Error{HE_EINVAL, "key switch at level " + std::to_string(l) + " needs " + std::to_string(need) +
                                       " scratch words; the no-allocation entry point holds " +
                                       std::to_string(HE_NOALLOC_SCRATCH_WORDS)};
        int dev = 0;
        check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
        if (dev < 0 || dev >= 64) throw Error{HE_EINVAL, "device index out of range"};
        u64 *base;
        {
            std::lock_guard<std::mutex> lk(g_noalloc_mu);
            if (!g_noalloc_ptr[dev]) {
                void *p = nullptr;
                check_cuda(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
                g_noalloc_ptr[dev] = (u64 *)p;
            }
            base = g_noalloc_ptr[dev];
        }
        // the context's key-switch scratch is swapped for the static array for
        // the duration of this call (restored on every exit path)
        struct Swap {
            he_ctx *cx;
            u64 *coef, *ext, *acc, *conv;
            ~Swap() { cx->ks_coef = coef; cx->ks_ext = ext; cx->ks_acc = acc; cx->ks_conv = conv; }
        } sw{cx, cx->ks_coef, cx->ks_ext, cx->ks_acc, cx->ks_conv};
        cx->ks_coef = base;
        cx->ks_ext = base + w_coef;
        cx->ks_acc = base + w_coef + w_ext;
        cx->ks_conv = base + w_coef + w_ext + w_acc;
        Rows o = make_rows(out, (size_t)(l + 1) * N, l + 1, l + 1, cx->nq);
        keyswitch(cx, d, l, *key, o, o, 0);
        check_cuda(cudaGetLastError(), "key switch (no allocation)");
    } catch (const Error &e) {
        cx->err = e.msg;
        return e.code;
    }
    return HE_OK;
}
