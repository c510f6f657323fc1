// mtb_arena.h -- the serving path's device-memory arena: offsets within one
// device allocation handed out first-fit.  Plain C++ (no CUDA), so that the
// allocator can be checked on the host alone.
#pragma once

#include <cstddef>

namespace mtb {

constexpr size_t kArenaAlign = 256;

inline size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// First-fit allocator over [0, size), in kArenaAlign units.  The free blocks
// are kept sorted by offset and merged with their neighbours, so an allocated
// block lies between any two of them: with at most kMaxHolders blocks allocated
// at once there are at most kMaxHolders + 1 free blocks.  The list is therefore
// a fixed array, and nothing is allocated on the heap while blocks come and go
// (the server releases a job's memory in a CUDA completion callback).
template <int kMaxHolders>
class Arena {
  public:
    explicit Arena(size_t size) {
        if (size) blk_[n_++] = Block{0, size};
    }
    bool alloc(size_t bytes, size_t *off) {
        bytes = round_up(bytes, kArenaAlign);
        for (int i = 0; i < n_; ++i) {
            if (blk_[i].size < bytes) continue;
            *off = blk_[i].off;
            blk_[i].off += bytes;
            blk_[i].size -= bytes;
            if (blk_[i].size == 0) erase(i);
            in_use_ += bytes;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = round_up(bytes, kArenaAlign);
        in_use_ -= bytes;
        int i = 0;  // the first free block after `off`
        while (i < n_ && blk_[i].off < off) ++i;
        const bool prev = i > 0 && blk_[i - 1].off + blk_[i - 1].size == off;
        const bool next = i < n_ && off + bytes == blk_[i].off;
        if (prev && next) {
            blk_[i - 1].size += bytes + blk_[i].size;
            erase(i);
        } else if (prev) {
            blk_[i - 1].size += bytes;
        } else if (next) {
            blk_[i].off = off;
            blk_[i].size += bytes;
        } else {  // n_ < kCap by the bound above
            for (int k = n_; k > i; --k) blk_[k] = blk_[k - 1];
            blk_[i] = Block{off, bytes};
            ++n_;
        }
    }
    size_t in_use() const { return in_use_; }
    // the free list, for checks: block i's offset and size, i < free_blocks()
    int free_blocks() const { return n_; }
    size_t free_offset(int i) const { return blk_[i].off; }
    size_t free_size(int i) const { return blk_[i].size; }

  private:
    struct Block {
        size_t off, size;
    };
    static constexpr int kCap = kMaxHolders + 1;
    void erase(int i) {
        for (int k = i; k + 1 < n_; ++k) blk_[k] = blk_[k + 1];
        --n_;
    }
    Block blk_[kCap] = {};
    int n_ = 0;
    size_t in_use_ = 0;
};

}  // namespace mtb
