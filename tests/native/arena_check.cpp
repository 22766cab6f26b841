// Randomised check of the serving arena's sub-allocator against a plain
// model (one flag per 256-byte unit): blocks never overlap or leave the
// range, the free lists stay merged and consistent, best fit is taken, and
// freeing everything restores one block of the full capacity.
// Usage: arena_check <seed> <ops>; prints "ok" or the first failure.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "arena.h"

int main(int argc, char **argv) {
    const unsigned seed = argc > 1 ? (unsigned)atoi(argv[1]) : 1u;
    const int ops = argc > 2 ? atoi(argv[2]) : 20000;
    std::mt19937_64 rng(seed);
    const size_t units = 4096, A = bb::Arena::ALIGN;
    bb::Arena arena(units * A + 100);  // capacity rounds down to whole units
    if (arena.capacity() != units * A) { puts("capacity not rounded"); return 1; }
    std::vector<int> owner(units, -1);
    struct Live { size_t off, bytes; int id; };
    std::vector<Live> live;
    int next_id = 0;
    for (int k = 0; k < ops; k++) {
        const bool do_alloc = live.empty() || rng() % 100 < 55;
        if (do_alloc) {
            size_t bytes = 1 + rng() % (rng() % 8 == 0 ? 64 * A : 4 * A);
            // what a best fit must find: the smallest free run that holds the request
            const size_t need = (bytes + A - 1) / A;
            size_t best = 0, run = 0;
            for (size_t u = 0; u <= units; u++) {
                if (u < units && owner[u] < 0) { run++; continue; }
                if (run >= need && (best == 0 || run < best)) best = run;
                run = 0;
            }
            size_t off;
            const bool ok = arena.alloc(bytes, &off);
            if (ok != (best != 0)) { printf("alloc %zu: got %d, model says %d\n", bytes, ok, best != 0); return 1; }
            if (!ok) continue;
            if (off % A) { puts("unaligned offset"); return 1; }
            // the chosen block must be a free run of exactly the best size
            size_t lo = off / A, hi = lo;
            while (lo > 0 && owner[lo - 1] < 0) lo--;
            while (hi < units && owner[hi] < 0) hi++;
            if (hi - lo != best) { printf("not best fit: run %zu, best %zu\n", hi - lo, best); return 1; }
            for (size_t u = off / A; u < off / A + need; u++) {
                if (u >= units || owner[u] >= 0) { puts("overlap or out of range"); return 1; }
                owner[u] = next_id;
            }
            live.push_back({off, bytes, next_id++});
        } else {
            const size_t i = rng() % live.size();
            const Live L = live[i];
            live[i] = live.back();
            live.pop_back();
            arena.free(L.off, L.bytes);
            for (size_t u = L.off / A; u < L.off / A + (L.bytes + A - 1) / A; u++) {
                if (owner[u] != L.id) { puts("freed a unit it did not own"); return 1; }
                owner[u] = -1;
            }
        }
        size_t used = 0;
        for (int o : owner) used += o >= 0;
        if (arena.used() != used * A) { printf("used %zu, model %zu\n", arena.used(), used * A); return 1; }
        if (!arena.consistent()) { puts("free lists inconsistent"); return 1; }
    }
    for (const Live &L : live) arena.free(L.off, L.bytes);
    if (arena.used() != 0 || arena.largest_free() != arena.capacity() || arena.free_blocks() != 1) {
        puts("free everything: not one full block");
        return 1;
    }
    puts("ok");
    return 0;
}
