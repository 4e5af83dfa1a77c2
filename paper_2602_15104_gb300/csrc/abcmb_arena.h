// First-fit allocator over the offsets of one device arena (host code only;
// the spectrum server places each request's buffers with it).
#pragma once

#include <algorithm>
#include <cstddef>
#include <vector>

namespace abcmb {

struct Block {
    size_t off, len;
};

// first-fit allocator over [0, size) with 256-byte granules
class Arena {
  public:
    void init(size_t size)
    {
        size_ = size & ~(size_t)255;
        free_.assign(1, Block{0, size_});
    }
    bool alloc(size_t len, size_t *off)
    {
        len = (len + 255) & ~(size_t)255;
        for (size_t i = 0; i < free_.size(); i++) {
            if (free_[i].len >= len) {
                *off = free_[i].off;
                free_[i].off += len;
                free_[i].len -= len;
                if (free_[i].len == 0) free_.erase(free_.begin() + i);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t len)
    {
        len = (len + 255) & ~(size_t)255;
        auto it = std::lower_bound(free_.begin(), free_.end(), off,
                                   [](const Block &b, size_t o) { return b.off < o; });
        it = free_.insert(it, Block{off, len});
        // coalesce with neighbours
        if (it + 1 != free_.end() && it->off + it->len == (it + 1)->off) {
            it->len += (it + 1)->len;
            free_.erase(it + 1);
        }
        if (it != free_.begin() && (it - 1)->off + (it - 1)->len == it->off) {
            (it - 1)->len += it->len;
            free_.erase(it);
        }
    }
    size_t largest() const
    {
        size_t m = 0;
        for (const Block &b : free_) m = std::max(m, b.len);
        return m;
    }
    size_t size() const { return size_; }

  private:
    size_t size_ = 0;
    std::vector<Block> free_;
};

} // namespace abcmb
