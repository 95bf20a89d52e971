// sv_pool.cpp -- a buddy allocator for state vectors inside one device arena.
//
// A state of n qubits occupies 2^n amplitudes, a power of two of bytes, so a
// buddy system places states without waste: every block is a power of two
// aligned to its own size, a free block's buddy is found by flipping one
// offset bit, and freeing merges buddies back up. The arena is device memory
// the caller allocated once (the library's relaxed memory model, Sec. II-A:
// the caller owns state memory); this file only does offset arithmetic on the
// host and never touches the memory or calls CUDA. An arena that is not a
// power of two is cut into maximal aligned power-of-two roots, each a buddy
// tree of its own. Admission of a request then asks exactly whether its state
// fits (sv_pool_alloc) instead of comparing byte counts that ignore
// fragmentation.
#include <cstdint>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <vector>

#include "sv.h"

struct sv_pool_ctx {
    uintptr_t base = 0;
    uint64_t capacity = 0;
    int min_order = 0;
    std::map<uint64_t, int> roots;            // root offset -> order
    std::vector<std::set<uint64_t>> free_at;  // order -> free block offsets
    std::map<uint64_t, int> used;             // allocated offset -> order
    uint64_t in_use = 0;
    std::mutex mu;
};

namespace {

constexpr int kMaxOrder = 62;

int order_of(uint64_t bytes, int min_order) {
    int o = min_order;
    while (o < kMaxOrder && (1ull << o) < bytes) ++o;
    return o;
}

// the root containing offset `off`
std::map<uint64_t, int>::const_iterator root_of(const sv_pool_ctx *p, uint64_t off) {
    auto it = p->roots.upper_bound(off);
    --it;
    return it;
}

}  // namespace

extern "C" {

SV_API sv_status_t sv_pool_create(void *d_base, uint64_t bytes, uint64_t min_block_bytes, sv_pool_t *out) {
    if (!out || !d_base || (reinterpret_cast<uintptr_t>(d_base) & 255u) || min_block_bytes < 256 ||
        (min_block_bytes & (min_block_bytes - 1)) || bytes < min_block_bytes)
        return SV_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    sv_pool_ctx *p = new (std::nothrow) sv_pool_ctx();
    if (!p) return SV_ERR_ALLOC;
    p->base = reinterpret_cast<uintptr_t>(d_base);
    p->min_order = order_of(min_block_bytes, 0);
    p->free_at.resize(kMaxOrder + 1);
    // maximal power-of-two roots, each aligned (relative to the base) to its size
    uint64_t off = 0;
    while (bytes - off >= min_block_bytes) {
        int o = kMaxOrder;
        while (o > p->min_order && (((1ull << o) > bytes - off) || (off & ((1ull << o) - 1)))) --o;
        p->roots[off] = o;
        p->free_at[o].insert(off);
        off += 1ull << o;
    }
    p->capacity = off;
    *out = p;
    return SV_OK;
}

SV_API sv_status_t sv_pool_destroy(sv_pool_t p) {
    if (!p) return SV_ERR_INVALID_ARGUMENT;
    delete p;
    return SV_OK;
}

SV_API sv_status_t sv_pool_alloc(sv_pool_t p, uint64_t bytes, void **d_out) {
    if (!p || !d_out || bytes == 0) return SV_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> lock(p->mu);
    const int want = order_of(bytes, p->min_order);
    if ((1ull << want) < bytes) return SV_ERR_INSUFFICIENT_WORKSPACE;
    int o = want;
    while (o <= kMaxOrder && p->free_at[o].empty()) ++o;
    if (o > kMaxOrder) return SV_ERR_INSUFFICIENT_WORKSPACE;
    // the lowest free block of the smallest order that fits, split down to size
    const uint64_t off = *p->free_at[o].begin();
    p->free_at[o].erase(p->free_at[o].begin());
    while (o > want) {
        --o;
        p->free_at[o].insert(off + (1ull << o));
    }
    p->used[off] = want;
    p->in_use += 1ull << want;
    *d_out = reinterpret_cast<void *>(p->base + off);
    return SV_OK;
}

SV_API sv_status_t sv_pool_free(sv_pool_t p, void *d_ptr) {
    if (!p || !d_ptr) return SV_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> lock(p->mu);
    const uintptr_t a = reinterpret_cast<uintptr_t>(d_ptr);
    if (a < p->base) return SV_ERR_INVALID_ARGUMENT;
    uint64_t off = a - p->base;
    auto u = p->used.find(off);
    if (u == p->used.end()) return SV_ERR_INVALID_ARGUMENT;
    int o = u->second;
    p->used.erase(u);
    p->in_use -= 1ull << o;
    const auto r = root_of(p, off);
    const uint64_t root_off = r->first;
    const int root_order = r->second;
    while (o < root_order) {
        const uint64_t buddy = root_off + ((off - root_off) ^ (1ull << o));
        auto f = p->free_at[o].find(buddy);
        if (f == p->free_at[o].end()) break;
        p->free_at[o].erase(f);
        if (buddy < off) off = buddy;
        ++o;
    }
    p->free_at[o].insert(off);
    return SV_OK;
}

SV_API sv_status_t sv_pool_stats(sv_pool_t p, uint64_t *bytes_in_use, uint64_t *largest_free_block,
                                 uint64_t *capacity) {
    if (!p) return SV_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> lock(p->mu);
    if (bytes_in_use) *bytes_in_use = p->in_use;
    if (largest_free_block) {
        uint64_t big = 0;
        for (int o = kMaxOrder; o >= 0; --o)
            if (!p->free_at[o].empty()) {
                big = 1ull << o;
                break;
            }
        *largest_free_block = big;
    }
    if (capacity) *capacity = p->capacity;
    return SV_OK;
}

}  // extern "C"
