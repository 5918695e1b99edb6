// CutMax (Alg. 2) as one CUDA graph per plan and input shape.
//
// A decode is about ten thousand kernel launches whose order, grids and
// arguments depend only on the plan, the input's level, scale and batch size,
// the context's keys and tables, and the addresses of the buffers it uses.
// The first call with a new (plan, shape) runs directly and records how much
// device memory it takes.  The same call then captures the whole circuit
// (its T iterations with their refreshes and the final normalisation) on a
// capture stream into one graph, every buffer drawn from a block of the
// context's arena reserved for that graph, so that the addresses baked into
// the graph stay its own.  Later calls copy the input into the graph's input
// buffer, launch the graph on the context's stream and copy its output into a
// new ciphertext: the same kernels in the same order on the same data, hence
// the same bits as a direct call.  A capture that fails (a call that is not
// capturable, an arena too small) leaves that key to direct calls.  Capture
// runs nothing, so the ledger counts recorded during it are taken back and
// added again at every launch.
#include <cstring>

#include "context.h"

namespace he {

struct CutmaxGraph {
    std::vector<double> key;
    uint64_t gen = 0;
    cudaGraphExec_t exec = nullptr;
    char *block = nullptr;  // the graph's arena: one block of the context's arena
    size_t block_bytes = 0;
    he_ct xin{}, zout{};    // input and output buffers inside the block
    uint64_t ks[HE_MAX_PRIMES] = {0}, ops[4][HE_MAX_PRIMES] = {{0}}, boots = 0;
    unsigned long long launches = 0;
    bool failed = false;
    uint64_t last_use = 0;  // call counter at the graph's last launch (least recently used goes first)
};

// graphs a context keeps at once (each holds its own arena block)
constexpr size_t GRAPHS_MAX = 16;

static std::vector<double> graph_key(he_ctx *cx, const he_ct *in, const Plan &pl) {
    std::vector<double> k = {(double)pl.n,         (double)pl.packing, (double)pl.T,      (double)pl.d,
                             pl.kappa_f,           (double)pl.bootstrap, (double)pl.cps,  (double)pl.shared,
                             (double)in->level,    in->scale,          (double)in->batch, (double)cx->rotsum_log_radix};
    auto add = [&](const auto &v) {
        k.push_back((double)v.size());
        for (auto x : v) k.push_back((double)x);
    };
    add(pl.p);
    add(pl.k);
    add(pl.c);
    add(pl.kappa);
    add(pl.y0);
    add(pl.norm);
    add(pl.lq);
    add(pl.relax);
    return k;
}

static void copy_ct(he_ctx *cx, he_ct *dst, const he_ct *src, cudaStream_t s) {
    const size_t row = (size_t)(src->level + 1) * cx->N() * 8;
    check_cuda(cudaMemcpy2DAsync(dst->d, (size_t)dst->cap * cx->N() * 8, src->d, (size_t)src->cap * cx->N() * 8, row,
                                 (size_t)2 * src->batch, cudaMemcpyDeviceToDevice, s),
               "graph input/output copy");
}

static void graph_free(he_ctx *cx, CutmaxGraph &g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    if (g.block) cx->arena.release(g.block, g.block_bytes);
    g.block = nullptr;
}

void graphs_release(he_ctx *cx) {
    if (cx->graphs.empty()) return;
    cudaStreamSynchronize(cx->stream);  // no launch of a graph may still read its block
    for (auto &g : cx->graphs) graph_free(cx, *g);
    cx->graphs.clear();
}

// Capture cutmax_ct(in-shaped input) into g; false when it cannot be captured.
static bool capture(he_ctx *cx, const he_ct *in, const Plan &pl, size_t need, CutmaxGraph &g) {
    const size_t in_bytes = (size_t)2 * in->batch * (in->level + 1) * cx->N() * 8;
    g.block_bytes = need + need / 4 + in_bytes + ((size_t)16 << 20);
    try {
        g.block = (char *)cx->arena.alloc(g.block_bytes);
    } catch (const Error &) {
        g.block = nullptr;
        return false;
    }
    Arena ga;
    ga.base = g.block;
    ga.cap = g.block_bytes;
    // saved state: the ledger and the launch counter move during capture
    uint64_t ks0[HE_MAX_PRIMES], ops0[4][HE_MAX_PRIMES];
    std::memcpy(ks0, cx->ks_by_level, sizeof(ks0));
    std::memcpy(ops0, cx->ops_by_level, sizeof(ops0));
    const uint64_t boots0 = cx->n_boot;
    const unsigned long long l0 = launch_count();
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const cudaStream_t s0 = cx->stream;
    std::swap(cx->arena, ga);  // every allocation below comes from the graph's block
    cx->stream = cs;
    cx->capturing = true;
    bool ok = true;
    cudaGraph_t graph = nullptr;
    he_ct *x = nullptr, *z = nullptr;
    try {
        x = ct_alloc(cx, in->level, in->scale, in->batch);
    } catch (const Error &) {
        ok = false;
    }
    if (ok && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        try {
            z = cutmax_ct(cx, x, pl).release();
        } catch (const Error &) {
            ok = false;
        }
        if (cudaStreamEndCapture(cs, &graph) != cudaSuccess || !graph) ok = false;
    } else {
        ok = false;
    }
    cudaGetLastError();  // a refused capture leaves its error here
    cx->capturing = false;
    cx->stream = s0;
    std::swap(cx->arena, ga);
    cudaStreamDestroy(cs);
    // the buffers belong to the block from now on: no ciphertext handles
    for (he_ct *c : {x, z})
        if (c) {
            cx->live.erase(c);
            if (c == x) g.xin = *c;
            else g.zout = *c;
            delete c;
        }
    g.launches = launch_count() - l0;
    for (int i = 0; i < HE_MAX_PRIMES; i++) {
        g.ks[i] = cx->ks_by_level[i] - ks0[i];
        for (int k = 0; k < 4; k++) g.ops[k][i] = cx->ops_by_level[k][i] - ops0[k][i];
    }
    g.boots = cx->n_boot - boots0;
    std::memcpy(cx->ks_by_level, ks0, sizeof(ks0));  // nothing ran
    std::memcpy(cx->ops_by_level, ops0, sizeof(ops0));
    cx->n_boot = boots0;
    launches_add(-(long long)g.launches);
    if (ok && !z) ok = false;
    if (ok && cudaGraphInstantiate(&g.exec, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        g.exec = nullptr;
        ok = false;
    }
    if (graph) cudaGraphDestroy(graph);
    return ok;
}

Ct cutmax_graph(he_ctx *cx, const he_ct *in, const Plan &pl) {
    if (prof_any()) {  // instrumented launches are timed one by one: run directly
        cx->graph_stats[2]++;
        return cutmax_ct(cx, in, pl);
    }
    // graphs that point at retired tables go
    for (size_t i = 0; i < cx->graphs.size();)
        if (cx->graphs[i]->gen != cx->gen) {
            cudaStreamSynchronize(cx->stream);
            graph_free(cx, *cx->graphs[i]);
            cx->graphs.erase(cx->graphs.begin() + (long)i);
        } else {
            i++;
        }
    const std::vector<double> key = graph_key(cx, in, pl);
    const uint64_t now = ++cx->graph_calls;
    for (auto &gp : cx->graphs) {
        CutmaxGraph &g = *gp;
        if (g.key != key) continue;
        g.last_use = now;
        if (g.failed) {
            cx->graph_stats[2]++;
            return cutmax_ct(cx, in, pl);
        }
        copy_ct(cx, &g.xin, in, cx->stream);
        check_cuda(cudaGraphLaunch(g.exec, cx->stream), "graph launch");
        Ct out(ct_alloc(cx, g.zout.level, g.zout.scale, g.zout.batch));
        copy_ct(cx, out.get(), &g.zout, cx->stream);
        for (int i = 0; i < HE_MAX_PRIMES; i++) {
            cx->ks_by_level[i] += g.ks[i];
            for (int k = 0; k < 4; k++) cx->ops_by_level[k][i] += g.ops[k][i];
        }
        cx->n_boot += g.boots;
        launches_add((long long)g.launches);
        cx->graph_stats[1]++;
        return out;
    }
    // a new key: the least recently used graph gives way when the context holds
    // GRAPHS_MAX of them
    if (cx->graphs.size() >= GRAPHS_MAX) {
        size_t lru = 0;
        for (size_t i = 1; i < cx->graphs.size(); i++)
            if (cx->graphs[i]->last_use < cx->graphs[lru]->last_use) lru = i;
        cudaStreamSynchronize(cx->stream);  // no launch of it may still read its block
        graph_free(cx, *cx->graphs[lru]);
        cx->graphs.erase(cx->graphs.begin() + (long)lru);
    }
    // first call with this key: run directly, measuring the memory it takes,
    // then capture the graph for the calls after it
    const size_t base = cx->arena.in_use, peak0 = cx->arena.peak;
    cx->arena.peak = base;
    Ct r = cutmax_ct(cx, in, pl);
    const size_t need = cx->arena.peak - base;
    cx->arena.peak = std::max(peak0, cx->arena.peak);
    auto g = std::make_shared<CutmaxGraph>();
    g->key = key;
    g->gen = cx->gen;
    g->last_use = now;
    if (capture(cx, in, pl, need, *g)) {
        cx->graph_stats[0]++;
    } else {
        graph_free(cx, *g);
        g->failed = true;
        cx->graph_stats[2]++;
    }
    cx->graphs.push_back(std::move(g));
    return r;
}

}  // namespace he
