// arena.h - best-fit sub-allocator over one reserved device range.
//
// The serving engine reserves its HBM budget once and places every resident
// graph, input copy and build workspace inside it, so admission is exact
// (a request is admitted only when its blocks fit) and the steady state makes
// no cudaMalloc/cudaFree calls (cudaFree waits for the whole device). Offsets
// and sizes are multiples of ALIGN; free neighbours are merged. Host-only
// code with no CUDA dependency, so it is tested on its own.
#pragma once
#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>

namespace bb {

class Arena {
public:
    static constexpr size_t ALIGN = 256;

    Arena() = default;
    explicit Arena(size_t capacity) { reset(capacity); }

    void reset(size_t capacity) {
        cap_ = capacity / ALIGN * ALIGN;
        used_ = 0;
        by_off_.clear();
        by_size_.clear();
        if (cap_) insert(0, cap_);
    }

    static size_t round(size_t bytes) { return (bytes + ALIGN - 1) / ALIGN * ALIGN; }

    // smallest free block that fits; false when none does
    bool alloc(size_t bytes, size_t *off) {
        const size_t need = round(bytes ? bytes : 1);
        auto it = by_size_.lower_bound(need);
        if (it == by_size_.end()) return false;
        const size_t o = it->second, sz = it->first;
        erase(o, sz);
        if (sz > need) insert(o + need, sz - need);
        used_ += need;
        *off = o;
        return true;
    }

    void free(size_t off, size_t bytes) {
        size_t sz = round(bytes ? bytes : 1);
        used_ -= sz;
        auto next = by_off_.lower_bound(off);
        if (next != by_off_.end() && off + sz == next->first) {  // merge with the block after
            const size_t nsz = next->second;
            erase(next->first, nsz);
            sz += nsz;
        }
        auto after = by_off_.lower_bound(off);
        if (after != by_off_.begin()) {  // merge with the block before
            auto prev = std::prev(after);
            if (prev->first + prev->second == off) {
                const size_t po = prev->first, psz = prev->second;
                erase(po, psz);
                off = po;
                sz += psz;
            }
        }
        insert(off, sz);
    }

    size_t capacity() const { return cap_; }
    size_t used() const { return used_; }
    size_t free_bytes() const { return cap_ - used_; }
    size_t largest_free() const { return by_size_.empty() ? 0 : by_size_.rbegin()->first; }
    size_t free_blocks() const { return by_off_.size(); }

    // walks the free list; true when it tiles [0, cap) with used blocks
    // without overlap and no two free blocks touch
    bool consistent() const {
        size_t free_sum = 0, end = 0;
        bool first = true;
        for (const auto &b : by_off_) {
            if (!first && b.first <= end) return false;  // touching or overlapping
            if (b.first + b.second > cap_) return false;
            end = b.first + b.second;
            free_sum += b.second;
            first = false;
        }
        if (free_sum != cap_ - used_) return false;
        return by_size_.size() == by_off_.size();
    }

private:
    void insert(size_t off, size_t sz) {
        by_off_[off] = sz;
        by_size_.emplace(sz, off);
    }
    void erase(size_t off, size_t sz) {
        by_off_.erase(off);
        auto range = by_size_.equal_range(sz);
        for (auto it = range.first; it != range.second; ++it)
            if (it->second == off) { by_size_.erase(it); break; }
    }

    size_t cap_ = 0, used_ = 0;
    std::map<size_t, size_t> by_off_;        // free: offset -> size
    std::multimap<size_t, size_t> by_size_;  // free: size -> offset
};

}  // namespace bb
