/*
 * CPU context baseline, not the oracle: the oracle's order (bytes as
 * unsigned, a string that is a proper prefix of another first, equal strings
 * by ascending input index) produced by libstdc++'s parallel-mode stable sort
 * (__gnu_parallel::stable_sort, OpenMP threads) with a memcmp comparator,
 * then the naive LCP of neighbours in an OpenMP loop.  A library sort on all
 * host cores, for comparison with the GPU; only the benchmark's CPU leg runs
 * it, and the tests check its output against orc_sort.
 *
 * String model as in oracle.c: string i starts at chars[offsets[i]]; it has
 * lengths[i] bytes if lengths != NULL, else fixed_len bytes if fixed_len != 0,
 * else it ends at the first 0 byte.
 */
#include <omp.h>
#include <stdint.h>
#include <string.h>

#include <parallel/algorithm>
#include <vector>

extern "C" int orc_sort_parallel(const uint8_t *chars, const uint64_t *offsets, const uint32_t *lengths,
                                 uint32_t fixed_len, uint64_t n, uint32_t *perm, uint32_t *lcp, int threads) {
    if (threads > 0) omp_set_num_threads(threads);
    std::vector<uint64_t> len(n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; i++)
        len[i] = lengths ? lengths[i] : fixed_len ? fixed_len : strlen((const char *)chars + offsets[i]);
    std::vector<uint32_t> idx(n);
    for (uint64_t i = 0; i < n; i++) idx[i] = (uint32_t)i;
    auto less = [&](uint32_t a, uint32_t b) {
        const uint64_t la = len[a], lb = len[b];
        const int c = memcmp(chars + offsets[a], chars + offsets[b], la < lb ? la : lb);
        return c != 0 ? c < 0 : la < lb;   // equal strings: the stable sort keeps input order
    };
    __gnu_parallel::stable_sort(idx.begin(), idx.end(), less);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < (int64_t)n; k++) {
        perm[k] = idx[k];
        if (k == 0) {
            lcp[0] = 0;
            continue;
        }
        const uint32_t a = idx[k - 1], b = idx[k];
        const uint64_t m = len[a] < len[b] ? len[a] : len[b];
        const uint8_t *pa = chars + offsets[a], *pb = chars + offsets[b];
        uint64_t h = 0;
        while (h < m && pa[h] == pb[h]) h++;
        lcp[k] = (uint32_t)h;
    }
    return omp_get_max_threads();
}
