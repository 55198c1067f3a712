// Device-memory pool of the working arenas of pooled hierarchies
// (mg_params.pooled = 1), one per device.
//
// A pooled hierarchy keeps only its plan and a small persistent part; the
// working arena (level vectors, FP64 u and r: nearly all of its bytes) is
// taken from this pool when a solve is admitted and handed back when it
// completes.  The pool holds device memory in chunks obtained with cudaMalloc,
// never more than its budget in total, and sub-allocates blocks from them:
//
//   - a block handed back stays assigned to its last hierarchy ("cached"):
//     when that hierarchy is admitted again and the block is still there, it
//     gets the same address with its contents, so its launch plan and CUDA
//     graphs stay valid and nothing is re-zeroed;
//   - a request that does not fit in the free space evicts cached blocks,
//     least recently used first, coalescing free neighbours, until a free
//     range is large enough; then, while the budget allows, a new chunk is
//     allocated; otherwise the request does not fit now (the serving engine
//     keeps it queued) -- blocks in use are never moved or taken.
//
// So the budget bounds the device memory the pool holds (`reserved`), and
// with it the working memory of everything admitted.  All functions are
// thread-safe (one mutex per pool).
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "mg_host.h"

namespace mgi {
namespace {

constexpr size_t kBlockAlign = 4096;
constexpr size_t kChunkMin = size_t(256) << 20;  // chunks of at least 256 MiB (fewer, larger cudaMallocs)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Block {
    size_t off = 0, size = 0;
    mgi_hier* owner = nullptr;  // nullptr: free
    bool in_use = false;
    unsigned long long stamp = 0;  // last hand-back (LRU order of cached blocks)
};

struct Chunk {
    char* base = nullptr;
    size_t size = 0;
    std::vector<Block> blocks;  // tile [0, size) in address order
};

struct Pool {
    std::mutex mu;
    int device = 0;
    size_t budget = 0;  // 0: not yet set (default taken at the first use)
    size_t reserved = 0, in_use = 0, peak_in_use = 0, peak_reserved = 0;
    unsigned long long tick = 0, acquires = 0, reuses = 0, evictions = 0;
    std::vector<Chunk> chunks;

    void ensure_budget() {
        if (budget) return;
        size_t fr = 0, tot = 0;
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            fr = size_t(8) << 30;
        }
        cudaSetDevice(cur);
        budget = fr / 10 * 8;
    }
    // merges block i of chunk c with free neighbours
    static void coalesce(Chunk& c, size_t i) {
        if (i + 1 < c.blocks.size() && !c.blocks[i + 1].owner && !c.blocks[i].owner) {
            c.blocks[i].size += c.blocks[i + 1].size;
            c.blocks.erase(c.blocks.begin() + (long)i + 1);
        }
        if (i > 0 && !c.blocks[i - 1].owner && !c.blocks[i].owner) {
            c.blocks[i - 1].size += c.blocks[i].size;
            c.blocks.erase(c.blocks.begin() + (long)i);
        }
    }
    Block* find(mgi_hier* h, Chunk** ch) {
        for (Chunk& c : chunks)
            for (Block& b : c.blocks)
                if (b.owner == h) {
                    if (ch) *ch = &c;
                    return &b;
                }
        return nullptr;
    }
    // best fit among free ranges; assigns it to h (in use)
    bool take_free(mgi_hier* h, size_t bytes, char** base) {
        Chunk* bc = nullptr;
        size_t bi = 0, best = ~size_t(0);
        for (Chunk& c : chunks)
            for (size_t i = 0; i < c.blocks.size(); ++i) {
                const Block& b = c.blocks[i];
                if (!b.owner && b.size >= bytes && b.size < best) { best = b.size; bc = &c; bi = i; }
            }
        if (!bc) return false;
        Block& b = bc->blocks[bi];
        if (b.size > bytes) {  // split: the remainder stays free after it
            Block rest;
            rest.off = b.off + bytes;
            rest.size = b.size - bytes;
            b.size = bytes;
            bc->blocks.insert(bc->blocks.begin() + (long)bi + 1, rest);
        }
        Block& t = bc->blocks[bi];
        t.owner = h;
        t.in_use = true;
        *base = bc->base + t.off;
        return true;
    }
    // frees the least recently handed-back cached block; false if there is none
    bool evict_one() {
        Chunk* bc = nullptr;
        size_t bi = 0;
        unsigned long long oldest = ~0ull;
        for (Chunk& c : chunks)
            for (size_t i = 0; i < c.blocks.size(); ++i) {
                const Block& b = c.blocks[i];
                if (b.owner && !b.in_use && b.stamp < oldest) { oldest = b.stamp; bc = &c; bi = i; }
            }
        if (!bc) return false;
        bc->blocks[bi].owner = nullptr;
        ++evictions;
        coalesce(*bc, bi);
        return true;
    }
    // gives one chunk that holds no block back to the device; false if none
    bool free_empty_chunk() {
        for (size_t k = chunks.size(); k-- > 0;) {
            Chunk& c = chunks[k];
            if (c.blocks.size() == 1 && !c.blocks[0].owner) {
                int cur = 0;
                cudaGetDevice(&cur);
                cudaSetDevice(device);
                cudaFree(c.base);
                cudaSetDevice(cur);
                reserved -= c.size;
                chunks.erase(chunks.begin() + (long)k);
                return true;
            }
        }
        return false;
    }
    // releases empty chunks while more than the budget is held
    void trim() {
        while (reserved > budget && free_empty_chunk()) {
        }
    }
};

std::mutex g_pools_mu;
std::map<int, Pool*> g_pools;

Pool& pool(int device) {
    std::lock_guard<std::mutex> lk(g_pools_mu);
    Pool*& p = g_pools[device];
    if (!p) {
        p = new Pool();  // lives for the process (hierarchies may outlive any scope)
        p->device = device;
    }
    return *p;
}

}  // namespace

int pool_acquire(int device, mgi_hier* h, size_t bytes, char** base, bool* kept) {
    Pool& P = pool(device);
    std::lock_guard<std::mutex> lk(P.mu);
    P.ensure_budget();
    bytes = align_up(bytes, kBlockAlign);
    *kept = false;
    if (bytes > P.budget) return 2;
    ++P.acquires;
    Chunk* c = nullptr;
    if (Block* b = P.find(h, &c)) {
        if (b->in_use) return 3;  // a hierarchy holds at most one arena
        if (b->size >= bytes) {   // its cached block is still there: same address, contents intact
            b->in_use = true;
            *base = c->base + b->off;
            *kept = true;
            P.in_use += b->size;
            P.peak_in_use = std::max(P.peak_in_use, P.in_use);
            ++P.reuses;
            return 0;
        }
        b->owner = nullptr;  // too small (cannot happen for a fixed layout): give it up
        Pool::coalesce(*c, (size_t)(b - c->blocks.data()));
    }
    for (;;) {
        if (P.take_free(h, bytes, base)) break;
        // grow while the budget allows, else make room from cached blocks
        if (P.reserved + bytes <= P.budget) {
            const size_t sz = std::max(bytes, std::min(kChunkMin, P.budget - P.reserved));
            void* mem = nullptr;
            int cur = 0;
            cudaGetDevice(&cur);
            cudaSetDevice(device);
            cudaError_t e = mgi_fault_take(MG_FAULT_ARENA) ? cudaErrorMemoryAllocation : cudaMalloc(&mem, sz);
            cudaSetDevice(cur);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return 3;
            }
            Chunk nc;
            nc.base = static_cast<char*>(mem);
            nc.size = sz;
            Block fb;
            fb.size = sz;
            nc.blocks.push_back(fb);
            P.chunks.push_back(nc);
            P.reserved += sz;
            P.peak_reserved = std::max(P.peak_reserved, P.reserved);
            continue;
        }
        // no range fits and the budget is held: first return an empty chunk to the
        // device (so a larger one can be made), then evict cached blocks
        if (P.free_empty_chunk()) continue;
        if (!P.evict_one()) return 1;
    }
    P.in_use += bytes;
    P.peak_in_use = std::max(P.peak_in_use, P.in_use);
    return 0;
}

void pool_release(int device, mgi_hier* h) {
    Pool& P = pool(device);
    std::lock_guard<std::mutex> lk(P.mu);
    if (Block* b = P.find(h, nullptr)) {
        if (b->in_use) {
            b->in_use = false;
            P.in_use -= b->size;
        }
        b->stamp = ++P.tick;
    }
}

void pool_drop(int device, mgi_hier* h) {
    Pool& P = pool(device);
    std::lock_guard<std::mutex> lk(P.mu);
    Chunk* c = nullptr;
    if (Block* b = P.find(h, &c)) {
        if (b->in_use) P.in_use -= b->size;
        b->in_use = false;
        b->owner = nullptr;
        Pool::coalesce(*c, (size_t)(b - c->blocks.data()));
    }
    P.trim();
}

size_t pool_budget(int device) {
    Pool& P = pool(device);
    std::lock_guard<std::mutex> lk(P.mu);
    P.ensure_budget();
    return P.budget;
}

void pool_set_budget(int device, size_t bytes) {
    Pool& P = pool(device);
    std::lock_guard<std::mutex> lk(P.mu);
    P.budget = bytes;
    if (bytes) {
        while (P.reserved > P.budget) {  // empty chunks first, then cached arenas
            if (P.free_empty_chunk()) continue;
            if (!P.evict_one()) break;
        }
    }
    P.peak_in_use = P.in_use;  // the peaks restart with the new budget
    P.peak_reserved = P.reserved;
}

PoolStats pool_stats(int device) {
    Pool& P = pool(device);
    std::lock_guard<std::mutex> lk(P.mu);
    PoolStats s{};
    s.budget = P.budget;
    s.reserved = P.reserved;
    s.in_use = P.in_use;
    s.peak_in_use = P.peak_in_use;
    s.peak_reserved = P.peak_reserved;
    s.acquires = P.acquires;
    s.reuses = P.reuses;
    s.evictions = P.evictions;
    s.chunks = P.chunks.size();
    return s;
}

}  // namespace mgi
