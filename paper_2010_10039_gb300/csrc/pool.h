// Host-side bookkeeping of one device memory region: address-ordered
// first-fit allocation of aligned blocks with coalescing on free.  No CUDA
// here (the server owns the region); the CPU tests compile this header alone.
#pragma once

#include <cstdint>
#include <iterator>
#include <map>

namespace huff {

class RegionAllocator {
public:
    explicit RegionAllocator(uint64_t capacity = 0, uint64_t align = 256) { reset(capacity, align); }

    void reset(uint64_t capacity, uint64_t align) {
        cap_ = capacity;
        align_ = align ? align : 1;
        free_.clear();
        if (cap_) free_[0] = cap_;
        used_ = 0;
        peak_ = 0;
    }

    // Rounds a request up to the alignment (every block starts aligned).
    uint64_t block_size(uint64_t bytes) const { return (bytes + align_ - 1) / align_ * align_; }

    // First block (lowest offset) of at least `bytes`; false if none is free.
    bool alloc(uint64_t bytes, uint64_t *offset) {
        const uint64_t need = block_size(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need) continue;
            const uint64_t off = it->first, size = it->second;
            free_.erase(it);
            if (size > need) free_[off + need] = size - need;
            used_ += need;
            if (used_ > peak_) peak_ = used_;
            *offset = off;
            return true;
        }
        return false;
    }

    // Returns a block obtained from alloc(bytes) and merges it with free neighbours.
    void release(uint64_t offset, uint64_t bytes) {
        uint64_t size = block_size(bytes ? bytes : 1);
        used_ -= size;
        auto next = free_.lower_bound(offset);
        if (next != free_.end() && offset + size == next->first) {
            size += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == offset) {
                prev->second += size;
                return;
            }
        }
        free_[offset] = size;
    }

    bool fits_ever(uint64_t bytes) const { return block_size(bytes ? bytes : 1) <= cap_; }
    uint64_t capacity() const { return cap_; }
    uint64_t used() const { return used_; }
    uint64_t peak() const { return peak_; }
    uint64_t free_blocks() const { return free_.size(); }
    uint64_t largest_free() const {
        uint64_t m = 0;
        for (const auto &kv : free_) m = kv.second > m ? kv.second : m;
        return m;
    }

private:
    uint64_t cap_ = 0, align_ = 256, used_ = 0, peak_ = 0;
    std::map<uint64_t, uint64_t> free_;    // offset -> size
};

}  // namespace huff
