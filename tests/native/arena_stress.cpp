// Random allocate/release sequences against the context's device-memory
// sub-allocator (host logic only; no device memory is touched: the base is a
// fake address).  Checks after every step batch that live blocks never
// overlap, that in_use counts the live bytes, that free and live blocks tile
// [0, top) with no two free blocks adjacent, and that releasing everything
// returns the allocator to empty.  Exit code 0 on success.
#include <cstdio>
#include <random>
#include <vector>

#include "arena.h"

int main(int argc, char **argv) {
    const unsigned long long seed = argc > 1 ? std::stoull(argv[1]) : 1;
    he::Arena A;
    A.base = reinterpret_cast<char *>(size_t(1) << 40);
    A.cap = size_t(1) << 40;
    std::mt19937_64 rng(seed);
    std::vector<std::pair<size_t, size_t>> live;  // offset, rounded size
    for (int it = 0; it < 100000; it++) {
        if (live.empty() || rng() % 3) {
            // sizes spanning granules to tens of MB, as ciphertext batches do
            size_t b = 1 + rng() % ((rng() % 4 == 0) ? (64u << 20) : (1u << 16));
            size_t off = (size_t)((char *)A.alloc(b) - A.base);
            size_t rb = (b + 255) & ~(size_t)255;
            if (off % 256) { std::printf("misaligned block\n"); return 1; }
            for (auto &l : live)
                if (off < l.first + l.second && l.first < off + rb) { std::printf("overlap\n"); return 1; }
            live.push_back({off, rb});
        } else {
            size_t i = rng() % live.size();
            A.release(A.base + live[i].first, live[i].second);
            live[i] = live.back();
            live.pop_back();
        }
        if (it % 5000 == 0) {
            size_t s = 0, f = 0;
            for (auto &l : live) s += l.second;
            for (auto &kv : A.by_off) f += kv.second;
            if (s != A.in_use) { std::printf("in_use mismatch\n"); return 1; }
            if (f + s != A.top) { std::printf("free and live blocks do not tile the used range\n"); return 1; }
            if (A.by_off.size() != A.by_size.size()) { std::printf("free indexes disagree\n"); return 1; }
            for (auto i = A.by_off.begin(); i != A.by_off.end(); ++i) {
                auto nx = std::next(i);
                if (nx != A.by_off.end() && i->first + i->second == nx->first) { std::printf("adjacent free blocks\n"); return 1; }
                if (i->first + i->second == A.top) { std::printf("free block at the top\n"); return 1; }
            }
        }
    }
    // exhaustion raises HE_ENOMEM and leaves the state unchanged
    he::Arena B;
    B.base = A.base;
    B.cap = 1 << 20;
    B.alloc(1 << 19);
    try {
        B.alloc(1 << 20);
        std::printf("no exhaustion error\n");
        return 1;
    } catch (const he::Error &e) {
        if (e.code != HE_ENOMEM || B.in_use != (1u << 19)) { std::printf("bad exhaustion error\n"); return 1; }
    }
    for (auto &l : live) A.release(A.base + l.first, l.second);
    if (A.top || A.in_use || !A.by_off.empty()) { std::printf("not empty after releasing everything\n"); return 1; }
    std::printf("ok peak %zu\n", A.peak);
    return 0;
}
