// Device-memory sub-allocator of a context (host code only).
//
// A context draws every ciphertext, key, table and scratch buffer from one
// device buffer supplied by the caller.  Blocks are 256-byte granules; a
// request takes the best-fitting free block (the remainder stays free) or
// extends the top; a freed block merges with free neighbours and, when it
// ends at the top, lowers the top.  Batches of many sizes (every batch size
// has its own temporaries) therefore do not fragment the buffer.
#pragma once
#include <algorithm>
#include <cstddef>
#include <map>
#include <string>

#include "../../include/he_cutmax.h"

namespace he {

struct Error { int code; std::string msg; };

struct Arena {
    char *base = nullptr;
    size_t cap = 0, top = 0, in_use = 0, peak = 0;
    bool owned = false;
    std::map<size_t, size_t> by_off;          // free blocks: offset -> size
    std::multimap<size_t, size_t> by_size;    // free blocks: size -> offset
    void *alloc(size_t bytes);                // throws Error{HE_ENOMEM} when full
    void release(void *p, size_t bytes);

   private:
    void erase_free(size_t off, size_t sz);
};

// Best fit among the free blocks (split, remainder kept free), else from the
// top; freed blocks merge with free neighbours and with the top.
inline void *Arena::alloc(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    size_t off;
    auto it = by_size.lower_bound(bytes);
    if (it != by_size.end()) {
        const size_t sz = it->first;
        off = it->second;
        by_size.erase(it);
        by_off.erase(off);
        if (sz > bytes) {
            by_off[off + bytes] = sz - bytes;
            by_size.emplace(sz - bytes, off + bytes);
        }
    } else {
        if (top + bytes > cap) throw Error{HE_ENOMEM, "device arena exhausted"};
        off = top;
        top += bytes;
    }
    in_use += bytes;
    peak = std::max(peak, in_use);
    return base + off;
}
inline void Arena::erase_free(size_t off, size_t sz) {
    by_off.erase(off);
    auto r = by_size.equal_range(sz);
    for (auto i = r.first; i != r.second; ++i)
        if (i->second == off) {
            by_size.erase(i);
            break;
        }
}
inline void Arena::release(void *p, size_t bytes) {
    if (!p) return;
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    size_t off = (size_t)((char *)p - base);
    in_use -= bytes;
    auto next = by_off.lower_bound(off);
    if (next != by_off.end() && next->first == off + bytes) {  // merge the following free block
        size_t nsz = next->second;
        erase_free(next->first, nsz);
        bytes += nsz;
    }
    auto prev = by_off.lower_bound(off);
    if (prev != by_off.begin()) {
        --prev;
        if (prev->first + prev->second == off) {  // merge into the preceding free block
            size_t poff = prev->first, psz = prev->second;
            erase_free(poff, psz);
            off = poff;
            bytes += psz;
        }
    }
    if (off + bytes == top) {  // give the tail back to the top
        top = off;
        return;
    }
    by_off[off] = bytes;
    by_size.emplace(bytes, off);
}

}  // namespace he
