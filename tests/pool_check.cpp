// Randomised check of the batch pool's first-fit allocator (lb_pool.h)
// against a brute-force model of the pool, one flag per ALIGN-byte unit:
// each allocation must take the lowest-addressed free run that holds it and
// fail only when no run does; after every operation the free byte count and
// the number of free ranges (every maximal run exactly one range: coalescing)
// must match the model.  Prints the number of failed checks; exit status 0
// when there are none.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <utility>
#include <vector>

#include "lb_pool.h"

constexpr size_t A = 256;

static uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

struct Model {
    std::vector<bool> used;
    explicit Model(size_t units) : used(units, false) {}
    // lowest start of a free run of at least n units, or -1
    long first_fit(size_t n) const {
        size_t run = 0;
        for (size_t u = 0; u < used.size(); ++u) {
            run = used[u] ? 0 : run + 1;
            if (run == n) return (long)(u + 1 - n);
        }
        return -1;
    }
    size_t free_units() const {
        size_t f = 0;
        for (bool b : used) f += !b;
        return f;
    }
    size_t runs() const {
        size_t r = 0;
        for (size_t u = 0; u < used.size(); ++u)
            if (!used[u] && (u == 0 || used[u - 1])) ++r;
        return r;
    }
};

int main(int argc, char** argv) {
    const int rounds = argc > 1 ? atoi(argv[1]) : 200;
    uint64_t s = 16781;
    long bad = 0;
    for (int r = 0; r < rounds; ++r) {
        const size_t units = 1 + splitmix(s) % 400;
        lbgb::Pool<A> pool;
        pool.reset(units * A);
        Model m(units);
        std::vector<std::pair<size_t, size_t>> live;  // (offset, bytes as requested)
        for (int op = 0; op < 600; ++op) {
            if (live.empty() || splitmix(s) % 100 < 55) {
                // request sizes: not multiples of A, sometimes exactly A, sometimes large
                const size_t bytes = 1 + splitmix(s) % (splitmix(s) % 4 == 0 ? units * A : 8 * A);
                const size_t need = (bytes + A - 1) / A;
                const long want = m.first_fit(need);
                size_t off = 0;
                const bool ok = pool.alloc(bytes, &off);
                if (ok != (want >= 0)) {
                    ++bad;
                } else if (ok) {
                    if (off % A || off != (size_t)want * A) ++bad;
                    for (size_t u = 0; u < need; ++u) m.used[off / A + u] = true;
                    live.push_back({off, bytes});
                }
            } else {
                const size_t k = splitmix(s) % live.size();
                const auto [off, bytes] = live[k];
                live.erase(live.begin() + (long)k);
                pool.release(off, bytes);
                for (size_t u = 0; u < (bytes + A - 1) / A; ++u) m.used[off / A + u] = false;
            }
            if (pool.free_bytes() != m.free_units() * A) ++bad;
            if (pool.free_ranges() != m.runs()) ++bad;
        }
        for (auto [off, bytes] : live) pool.release(off, bytes);
        if (pool.free_bytes() != units * A || pool.free_ranges() != 1) ++bad;
    }
    std::printf("pool checks failed: %ld\n", bad);
    return bad ? 1 : 0;
}
