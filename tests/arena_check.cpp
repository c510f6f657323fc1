// Host check of the serving arena (paper_2007_06483_gb300/csrc/mtb_arena.h)
// against a brute-force model: a map of 256-byte units, each free or taken.
// First fit over free blocks sorted by offset, with every free block merged
// with its neighbours, hands out the start of the lowest maximal free run that
// is long enough; the arena's free list must equal the model's maximal free
// runs after every step, and never hold more than holders + 1 blocks.
// Usage: arena_check <seed> <steps>; exit status 0 when every check holds.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <utility>
#include <vector>

#include "mtb_arena.h"

namespace {

constexpr int kHolders = 8;
using TestArena = mtb::Arena<kHolders>;

struct Model {
    std::vector<bool> taken;
    explicit Model(size_t units) : taken(units, false) {}
    // maximal free runs as (first unit, units)
    std::vector<std::pair<size_t, size_t>> runs() const {
        std::vector<std::pair<size_t, size_t>> r;
        size_t i = 0;
        while (i < taken.size()) {
            if (taken[i]) {
                ++i;
                continue;
            }
            size_t j = i;
            while (j < taken.size() && !taken[j]) ++j;
            r.emplace_back(i, j - i);
            i = j;
        }
        return r;
    }
    bool first_fit(size_t units, size_t *at) const {
        for (const auto &run : runs())
            if (run.second >= units) {
                *at = run.first;
                return true;
            }
        return false;
    }
    void mark(size_t first, size_t units, bool v) {
        for (size_t k = first; k < first + units; ++k) taken[k] = v;
    }
};

int fail(const char *what, long step) {
    std::fprintf(stderr, "arena check failed at step %ld: %s\n", step, what);
    return 1;
}

int compare(const TestArena &a, const Model &m, size_t held_bytes, long step) {
    const auto runs = m.runs();
    if (a.free_blocks() != (int)runs.size()) return fail("free block count differs from the model", step);
    if (a.free_blocks() > kHolders + 1) return fail("more than holders + 1 free blocks", step);
    for (int i = 0; i < a.free_blocks(); ++i)
        if (a.free_offset(i) != runs[i].first * mtb::kArenaAlign || a.free_size(i) != runs[i].second * mtb::kArenaAlign)
            return fail("free block differs from the model's free run", step);
    if (a.in_use() != held_bytes) return fail("bytes in use differ", step);
    return 0;
}

}  // namespace

int main(int argc, char **argv) {
    const unsigned seed = argc > 1 ? (unsigned)std::strtoul(argv[1], nullptr, 10) : 1u;
    const long steps = argc > 2 ? std::strtol(argv[2], nullptr, 10) : 20000;
    std::mt19937_64 rng(seed);
    const size_t units = 64 + rng() % 448;
    TestArena a(units * mtb::kArenaAlign);
    Model m(units);
    struct Held {
        size_t off, bytes, units;
    };
    std::vector<Held> held;
    size_t held_bytes = 0;
    if (compare(a, m, 0, -1)) return 1;
    for (long step = 0; step < steps; ++step) {
        const bool do_alloc = held.empty() || ((int)held.size() < kHolders && rng() % 2 == 0);
        if (do_alloc) {
            // sizes from one byte to half the arena; not all multiples of 256
            const size_t want_units = 1 + rng() % (units / 2);
            const size_t bytes = want_units * mtb::kArenaAlign - rng() % mtb::kArenaAlign;
            size_t off = 0, at = 0;
            const bool got = a.alloc(bytes, &off);
            const bool model_got = m.first_fit(want_units, &at);
            if (got != model_got) return fail("alloc success differs from the model", step);
            if (got) {
                if (off != at * mtb::kArenaAlign) return fail("alloc offset is not the first fit", step);
                m.mark(at, want_units, true);
                held.push_back(Held{off, bytes, want_units});
                held_bytes += want_units * mtb::kArenaAlign;
            }
        } else {
            const size_t k = rng() % held.size();
            const Held h = held[k];
            held.erase(held.begin() + (long)k);
            a.release(h.off, h.bytes);
            m.mark(h.off / mtb::kArenaAlign, h.units, false);
            held_bytes -= h.units * mtb::kArenaAlign;
        }
        if (compare(a, m, held_bytes, step)) return 1;
    }
    for (const Held &h : held) {
        a.release(h.off, h.bytes);
        m.mark(h.off / mtb::kArenaAlign, h.units, false);
    }
    if (compare(a, m, 0, steps)) return 1;
    if (a.free_blocks() != 1 || a.free_size(0) != units * mtb::kArenaAlign)
        return fail("the arena is not one block after everything is released", steps);
    return 0;
}
