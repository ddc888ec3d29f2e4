// K-way LCP merge of sorted runs in one pass (Section 5.2: the LCP-aware
// tournament tree of Algorithm 4; Section 5.3: splitting the merge into
// independent jobs; Section 5.4: caching the distinguishing characters).
//
// The output is cut into jobs at splitter strings taken from the runs
// themselves: every kKwDense-th string of every run is a splitter.  A
// splitter's place in every other run is found by binary search (the order
// of equal strings from different runs is the run order), which gives its
// rank in the merged output; a job is the stretch of outputs from one
// splitter's rank to the next splitter's.  The searches are narrowed in two
// steps: sparse splitters (every kKwSparse-th string) are searched over whole
// runs, dense ones only between the places of the sparse splitters around
// them, comparing from the characters those two sparse splitters share.
//
// Each job is merged by one thread with an LCP loser tree over the runs: a
// node keeps the losing run of its last game and that string's LCP with the
// winner that passed; when the winner is output and its run's next string
// (whose LCP with the winner is the run's own LCP entry) enters at the leaf,
// every game on the way up is decided by LCP-Compare (Algorithm 2): unequal
// LCPs decide without looking at characters, equal ones first compare the
// cached characters and only then read the strings.  The LCP of every output
// with the one before is the winner's LCP at the time it wins.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ss_internal.cuh"

namespace ss {

constexpr uint32_t kKwMaxRuns = kKwayMaxRuns;   // runs merged by one pass
constexpr uint32_t kKwSparse = 4096;      // strings of a run between sparse splitters
#ifndef SS_KW_DENSE
#define SS_KW_DENSE 128
#endif
constexpr uint32_t kKwDense = SS_KW_DENSE;   // strings of a run between dense splitters (jobs)
static_assert(kKwSparse % kKwDense == 0, "dense splitters refine the sparse ones");

// run tables of one merge, passed by value
struct KwRuns {
    uint32_t R;                        // runs (<= kKwMaxRuns), all non-empty
    uint32_t rb[kKwMaxRuns + 1];       // run k holds entries rb[k] .. rb[k+1]
    uint32_t base[kKwMaxRuns];         // string index = run entry + base[k]
    uint32_t sp[kKwMaxRuns + 1];       // sparse splitters of run k: sp[k] .. sp[k+1]
    uint32_t dn[kKwMaxRuns + 1];       // dense splitters of run k: dn[k] .. dn[k+1]
};

struct KwData {
    ReqDesc S;                         // the string set
    const uint32_t *perm;              // run entries (string indices without the base)
    const uint32_t *lcp;               // run LCP arrays
    const uint64_t *off;               // string offset of every run entry
    const uint64_t *ck;                // 8 characters of every entry at its run LCP
    const uint32_t *ckd;               // that depth
};

__device__ __forceinline__ uint32_t kw_run_of(const KwRuns &T, uint32_t e) {
    uint32_t r = 0;
#pragma unroll
    for (uint32_t k = 1; k < kKwMaxRuns; k++) r += (k < T.R && T.rb[k] <= e) ? 1u : 0u;
    return r;
}

// full comparison of strings a and b from depth h (both share h characters),
// 16 characters per round; -1/0/+1 and the lcp in *l
__device__ __forceinline__ int kw_cmp(const ReqDesc &S, uint32_t a, uint64_t oa, uint32_t b, uint64_t ob, uint32_t h,
                                      uint32_t *l) {
    for (;;) {
        uint64_t a0, a1, b0, b1;
        load_key2_o(S, a, oa, h, a0, a1);
        load_key2_o(S, b, ob, h, b0, b1);
        if (a0 != b0) { *l = h + lcp8(a0, b0); return a0 < b0 ? -1 : 1; }
        if (has_zero(a0)) { *l = h + nulpos(a0); return 0; }
        if (a1 != b1) { *l = h + 8 + lcp8(a1, b1); return a1 < b1 ? -1 : 1; }
        if (has_zero(a1)) { *l = h + 8 + nulpos(a1); return 0; }
        h += 16;
    }
}

// place of string (id, o) of run r in run k: the entries of run k that
// precede it in the merged order (equal strings: the lower run first),
// searched in entries [lo, hi) of run k, comparing from depth h
__device__ __forceinline__ uint32_t kw_place(const KwData &D, const KwRuns &T, uint32_t k, uint32_t r, uint32_t id,
                                             uint64_t o, uint32_t lo, uint32_t hi, uint32_t h) {
    const uint32_t a0 = T.rb[k];
    while (lo < hi) {
        const uint32_t mid = (lo + hi) / 2;
        const uint32_t e = a0 + mid;
        uint32_t l;
        const int c = kw_cmp(D.S, D.perm[e] + T.base[k], D.off[e], id, o, h, &l);
        const bool before = c < 0 || (c == 0 && k < r);
        if (before) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Sparse splitters: one thread per (splitter, run); the splitter's own run
// gives its place directly.  Also, per splitter, the characters it shares
// with the next sparse splitter of its run (the minimum of the run's LCPs
// between them), one warp per splitter, in k_kw_sparse_lcp.
__global__ void k_kw_sparse(KwData D, KwRuns T, uint32_t *spos) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t c = g / kKwMaxRuns, k = g % kKwMaxRuns;
    if (c >= T.sp[T.R] || k >= T.R) return;
    uint32_t r = 0;
    while (r + 1 < T.R && T.sp[r + 1] <= c) r++;
    const uint32_t i = (c - T.sp[r]) * kKwSparse;   // entry of the splitter inside run r
    const uint32_t e = T.rb[r] + i;
    uint32_t p;
    if (k == r) p = i;
    else p = kw_place(D, T, k, r, D.perm[e] + T.base[r], D.off[e], 0, T.rb[k + 1] - T.rb[k], 0);
    spos[c * kKwMaxRuns + k] = p;
}

__global__ void k_kw_sparse_lcp(KwData D, KwRuns T, uint32_t *splcp) {
    const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= T.sp[T.R]) return;
    uint32_t r = 0;
    while (r + 1 < T.R && T.sp[r + 1] <= w) r++;
    const uint32_t i = (w - T.sp[r]) * kKwSparse;
    const uint32_t n = T.rb[r + 1] - T.rb[r];
    const uint32_t j = min(n, i + kKwSparse);   // entry of the next sparse splitter (or the run's end)
    uint32_t m = 0xFFFFFFFFu;
    for (uint32_t x = i + 1 + lane; x <= j && x < n; x += 32) m = min(m, D.lcp[T.rb[r] + x]);
    m = __reduce_min_sync(0xffffffffu, m);
    if (lane == 0) splcp[w] = j < n ? m : 0u;   // no next splitter: nothing shared is known
}

// Dense splitters: one thread per (splitter, run).  A dense splitter lies
// between the sparse splitters sa and sa + 1 of its run, so its place in run
// k lies between theirs, and every string there shares the characters sa and
// sa + 1 share (any string between two strings in sorted order shares their
// LCP).  Its rank in the merged output is the sum of its places.
__global__ void k_kw_dense(KwData D, KwRuns T, const uint32_t *spos, const uint32_t *splcp, uint32_t *dpos) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t c = g / kKwMaxRuns, k = g % kKwMaxRuns;
    if (c >= T.dn[T.R] || k >= T.R) return;
    uint32_t r = 0;
    while (r + 1 < T.R && T.dn[r + 1] <= c) r++;
    const uint32_t i = (c - T.dn[r]) * kKwDense;   // entry inside run r
    const uint32_t sa = T.sp[r] + i / kKwSparse;   // the sparse splitter at or before it
    const bool exact = i % kKwSparse == 0;
    uint32_t p;
    if (k == r) {
        p = i;
    } else if (exact) {
        p = spos[sa * kKwMaxRuns + k];
    } else {
        const uint32_t nk = T.rb[k + 1] - T.rb[k];
        const bool last = sa + 1 >= T.sp[r + 1];   // no sparse splitter after it in run r
        const uint32_t lo = spos[sa * kKwMaxRuns + k];
        const uint32_t hi = last ? nk : spos[(sa + 1) * kKwMaxRuns + k];
        const uint32_t h = last ? 0u : splcp[sa];
        const uint32_t e = T.rb[r] + i;
        p = kw_place(D, T, k, r, D.perm[e] + T.base[r], D.off[e], lo, hi, h);
    }
    dpos[c * kKwMaxRuns + k] = p;
}

// rank of every dense splitter, and the rank where its job ends (the next
// splitter's, or the total): dense splitters of one run have increasing
// ranks, so the next one of run k is found by a binary search over them
__global__ void k_kw_rank(KwRuns T, const uint32_t *dpos, uint32_t *drank) {
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= T.dn[T.R]) return;
    uint32_t s = 0;
    for (uint32_t k = 0; k < T.R; k++) s += dpos[c * kKwMaxRuns + k];
    drank[c] = s;
}

// Also the splitter's place among all splitters in rank order (the jobs run
// in that order, so the threads of a warp merge neighbouring stretches of
// every run and of the output)
__global__ void k_kw_ends(KwRuns T, const uint32_t *drank, uint32_t total, uint32_t *dend, uint32_t *order) {
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= T.dn[T.R]) return;
    const uint32_t g = drank[c];
    uint32_t nxt = total, before = 0;
    for (uint32_t k = 0; k < T.R; k++) {
        uint32_t lo = T.dn[k], hi = T.dn[k + 1];   // first splitter of run k ranked after g
        while (lo < hi) {
            const uint32_t mid = (lo + hi) / 2;
            if (drank[mid] <= g) lo = mid + 1; else hi = mid;
        }
        if (lo < T.dn[k + 1]) nxt = min(nxt, drank[lo]);
        before += (c >= T.dn[k] && c < T.dn[k + 1]) ? c - T.dn[k] : lo - T.dn[k];
    }
    dend[c] = nxt;
    order[before] = c;
}

// A run's front in shared memory: its entry, string index and offset, the
// LCP with the string it last met, and its cached characters (8 at depth d).
struct KwFront {
    uint32_t e, id, h, d;   // e = ~0: run exhausted
    uint64_t o, k;
};

// LCP-Compare (Algorithm 2) of fronts x (run rx) and y (run ry), both with
// their LCP with the same earlier string.  Returns true if x goes first; *hl =
// LCP of the loser with the winner.  Exhausted fronts always lose.  Equal
// LCPs compare the cached characters where they cover the depth, then the
// strings.
__device__ __forceinline__ bool kw_game(const ReqDesc &S, uint32_t rx, const KwFront &x, uint32_t ry, const KwFront &y,
                                        uint32_t *hl) {
    if (y.e == ~0u) { *hl = y.h; return true; }
    if (x.e == ~0u) { *hl = x.h; return false; }
    if (x.h > y.h) { *hl = y.h; return true; }    // x shares more with the earlier string: x is smaller
    if (x.h < y.h) { *hl = x.h; return false; }
    const uint32_t h = x.h;
    if (x.d <= h && y.d <= h && h - x.d < 8 && h - y.d < 8) {
        const uint32_t sa = h - x.d, sb = h - y.d;
        const uint64_t wa = x.k << (8 * sa), wb = y.k << (8 * sb);
        const uint32_t nk = 8 - max(sa, sb);   // bytes known for both from depth h on
        const uint64_t mask = ~0ull << (64 - 8 * nk);
        const uint64_t v = (wa ^ wb) & mask;
        if (v) {
            *hl = h + (uint32_t)(__clzll((long long)v) >> 3);
            return (wa & mask) < (wb & mask);
        }
        const uint64_t z = zero_bytes(wa) & mask;   // both end inside the overlap: equal strings
        if (z) {
            *hl = h + (uint32_t)(__clzll((long long)z) >> 3);
            return rx < ry;
        }
    }
    const int c = kw_cmp(S, x.id, x.o, y.id, y.o, h, hl);
    return c < 0 || (c == 0 && rx < ry);
}

// threads per CTA of the merge: the fronts of all runs of every thread fit in
// 48 KB of static shared memory
__host__ __device__ constexpr uint32_t kw_threads(uint32_t KP) { return KP >= 8 ? 64u : 128u; }

// One job per thread: the outputs [drank[c], dend[c]) from the places
// dpos[c][*] in every run.  The tree of KP leaves (runs R .. KP-1 empty)
// lives in shared memory, one column per thread: node i holds the loser of
// its last game, whose front keeps its LCP with that game's winner.  Each
// run's next entry is read one output ahead (into its `next` slot), so the
// reads of a front that enters overlap the games before it.
template <uint32_t KP, uint32_t NT = kw_threads(KP)>
__global__ void __launch_bounds__(NT) k_kw_merge(KwData D, KwRuns T, const uint32_t *dpos, const uint32_t *drank,
                                                         const uint32_t *dend, const uint32_t *order, uint32_t njobs,
                                                         uint32_t *out_perm, uint32_t *out_lcp) {
    __shared__ KwFront s_f[KP][NT];      // each run's front
    __shared__ KwFront s_n[KP][NT];      // each run's next entry (h = its run LCP)
    __shared__ uint8_t s_lose[KP][NT];   // node i: run of its loser
    const uint32_t t = threadIdx.x;
    const uint32_t q = blockIdx.x * blockDim.x + t;
    if (q >= njobs) return;
    const uint32_t c = order[q];
    const uint32_t g0 = drank[c], g1 = dend[c];
    auto entry = [&](uint32_t k, uint32_t e, uint32_t h) {
        KwFront f;
        if (k < T.R && e < T.rb[k + 1]) {
            f.e = e;
            f.id = D.perm[e] + T.base[k];
            f.o = D.off[e];
            f.h = h;
            f.k = D.ck[e];
            f.d = D.ckd[e];
        } else {
            f.e = ~0u; f.id = 0; f.o = 0; f.h = 0; f.k = 0; f.d = ~0u;
        }
        return f;
    };
    const uint32_t r0 = [&] {   // run of the splitter that starts the job
        uint32_t r = 0;
        while (r + 1 < T.R && T.dn[r + 1] <= c) r++;
        return r;
    }();
    const uint32_t e0 = T.rb[r0] + dpos[c * kKwMaxRuns + r0];
    // the job's first output: its LCP with the string before it is the largest
    // of its LCPs with every run's string before its place
    uint32_t first_lcp = 0;
    for (uint32_t k = 0; k < KP; k++) {
        const uint32_t p = k < T.R ? dpos[c * kKwMaxRuns + k] : 0u;
        const uint32_t e = k < T.R ? T.rb[k] + p : ~0u;
        s_f[k][t] = entry(k, e, 0u);
        s_n[k][t] = entry(k, e + 1, (k < T.R && e + 1 < T.rb[k + 1]) ? D.lcp[e + 1] : 0u);
        if (g0 > 0 && k < T.R && p > 0) {
            uint32_t l;
            if (k == r0) l = D.lcp[e0];
            else {
                const uint32_t ep = e - 1;
                kw_cmp(D.S, D.perm[ep] + T.base[k], D.off[ep], D.perm[e0] + T.base[r0], D.off[e0], 0, &l);
            }
            first_lcp = max(first_lcp, l);
        }
    }
    // build: games bottom-up, every front's LCP taken against the empty string
    uint32_t win[KP];
#pragma unroll
    for (int i = KP - 1; i >= 1; i--) {
        const uint32_t a = (2 * i >= (int)KP) ? (2 * i - KP) : win[2 * i];
        const uint32_t b = (2 * i + 1 >= (int)KP) ? (2 * i + 1 - KP) : win[2 * i + 1];
        uint32_t hl;
        const bool a_first = kw_game(D.S, a, s_f[a][t], b, s_f[b][t], &hl);
        const uint32_t w = a_first ? a : b, l = a_first ? b : a;
        win[i] = w;
        s_lose[i][t] = (uint8_t)l;
        s_f[l][t].h = hl;
    }
    uint32_t w = win[1];
    for (uint32_t o = g0; o < g1; o++) {
        const KwFront fw = s_f[w][t];
        if (fw.e == ~0u) break;   // cannot happen for a consistent job; leaves the rest unwritten
        out_perm[o] = fw.id;
        out_lcp[o] = o == g0 ? first_lcp : fw.h;
        // the run's next entry enters (its LCP with the string just output is its
        // run LCP); the one after it is read now, used one output later
        s_f[w][t] = s_n[w][t];
        const uint32_t e2 = fw.e + 2;
        const KwFront nn = entry(w, e2, (e2 < T.rb[w + 1]) ? D.lcp[e2] : 0u);
        uint32_t x = w;
        for (uint32_t i = (KP + w) / 2; i >= 1; i /= 2) {
            const uint32_t y = s_lose[i][t];
            uint32_t hl;
            const bool x_first = kw_game(D.S, x, s_f[x][t], y, s_f[y][t], &hl);
            if (!x_first) {
                s_lose[i][t] = (uint8_t)x;
                s_f[x][t].h = hl;
                x = y;
            } else {
                s_f[y][t].h = hl;
            }
        }
        s_n[w][t] = nn;
        w = x;
    }
}

// string offset and cached characters (8 at the run LCP) of every run entry
__global__ void k_kw_prep(KwData D, KwRuns T, uint32_t total, uint64_t *off, uint64_t *ck, uint32_t *ckd) {
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const uint32_t r = kw_run_of(T, e);
        const uint32_t id = D.perm[e] + T.base[r];
        const uint64_t o = __ldg(D.S.offsets + id);
        const uint32_t d = e == T.rb[r] ? 0u : D.lcp[e];
        off[e] = o;
        ck[e] = load_key_o(D.S, id, o, d);
        ckd[e] = d;
    }
}

static int kw_check(cudaError_t e, const char *what) { return e == cudaSuccess ? SS_OK : cuda_fail(e, what); }

size_t merge_kway_scratch(uint32_t total, uint32_t R, const uint32_t *rb) {
    size_t nsp = 0, nde = 0;
    for (uint32_t k = 0; k < R; k++) {
        const uint32_t n = rb[k + 1] - rb[k];
        nsp += (n + kKwSparse - 1) / kKwSparse;
        nde += (n + kKwDense - 1) / kKwDense;
    }
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return al(8ull * total) * 2 + al(4ull * total) + al(4ull * kKwMaxRuns * nsp) + al(4ull * nsp) +
           al(4ull * kKwMaxRuns * nde) + 3 * al(4ull * nde) + 256;
}

// Merges R (2..kKwMaxRuns) non-empty runs in one pass; rb / base are host
// arrays (run k = entries rb[k] .. rb[k+1] of run_perm / run_lcp, string index
// = entry + base[k]).  Returns when the merge is complete.
int merge_kway(const ReqDesc &set, const uint32_t *run_perm, const uint32_t *run_lcp, const uint32_t *rb,
               const uint32_t *base, uint32_t R, uint32_t *perm_out, uint32_t *lcp_out, cudaStream_t st) {
    KwRuns T;
    memset(&T, 0, sizeof(T));
    T.R = R;
    for (uint32_t k = 0; k <= R; k++) T.rb[k] = rb[k];
    for (uint32_t k = R + 1; k <= kKwMaxRuns; k++) T.rb[k] = rb[R];
    T.sp[0] = T.dn[0] = 0;
    for (uint32_t k = 0; k < kKwMaxRuns; k++) {
        const uint32_t n = k < R ? rb[k + 1] - rb[k] : 0u;
        T.base[k] = k < R ? base[k] : 0u;
        T.sp[k + 1] = T.sp[k] + (n + kKwSparse - 1) / kKwSparse;
        T.dn[k + 1] = T.dn[k] + (n + kKwDense - 1) / kKwDense;
    }
    const uint32_t total = rb[R], nsp = T.sp[R], nde = T.dn[R];
    const size_t bytes = merge_kway_scratch(total, R, rb);
    void *block = nullptr;
    cudaError_t e = scratch_alloc(&block, bytes, st);
    if (e) {
        cudaGetLastError();
        set_error_detail("ss_merge: scratch allocation of %zu bytes failed", bytes);
        return SS_ERR_OOM;
    }
    char *p = (char *)block;
    auto take = [&](size_t b) { char *q = p; p += (b + 255) & ~(size_t)255; return q; };
    uint64_t *off = (uint64_t *)take(8ull * total);
    uint64_t *ck = (uint64_t *)take(8ull * total);
    uint32_t *ckd = (uint32_t *)take(4ull * total);
    uint32_t *spos = (uint32_t *)take(4ull * kKwMaxRuns * nsp);
    uint32_t *splcp = (uint32_t *)take(4ull * nsp);
    uint32_t *dpos = (uint32_t *)take(4ull * kKwMaxRuns * nde);
    uint32_t *drank = (uint32_t *)take(4ull * nde);
    uint32_t *dend = (uint32_t *)take(4ull * nde);
    uint32_t *order = (uint32_t *)take(4ull * nde);
    KwData D{set, run_perm, run_lcp, off, ck, ckd};
    int rc = SS_OK;
    do {
        const uint32_t pg = std::min<uint32_t>((total + 255) / 256, 8192);
        SS_LAUNCH_U("run_prep", st, total, k_kw_prep<<<pg, 256, 0, st>>>(D, T, total, off, ck, ckd));
        SS_LAUNCH_U("kway_sparse", st, nsp, k_kw_sparse<<<(nsp * kKwMaxRuns + 127) / 128, 128, 0, st>>>(D, T, spos));
        SS_LAUNCH_U("kway_sparse_lcp", st, nsp, k_kw_sparse_lcp<<<(nsp * 32 + 255) / 256, 256, 0, st>>>(D, T, splcp));
        SS_LAUNCH_U("kway_dense", st, nde, k_kw_dense<<<(nde * kKwMaxRuns + 127) / 128, 128, 0, st>>>(D, T, spos, splcp,
                                                                                                   dpos));
        SS_LAUNCH_U("kway_rank", st, nde, k_kw_rank<<<(nde + 255) / 256, 256, 0, st>>>(T, dpos, drank));
        SS_LAUNCH_U("kway_ends", st, nde, k_kw_ends<<<(nde + 255) / 256, 256, 0, st>>>(T, drank, total, dend, order));
        if (R <= 2)
            SS_LAUNCH_U("merge_kway", st, total, (k_kw_merge<2><<<(nde + kw_threads(2) - 1) / kw_threads(2), kw_threads(2), 0,
                                                               st>>>(D, T, dpos, drank, dend, order, nde, perm_out, lcp_out)));
        else if (R <= 4)
            SS_LAUNCH_U("merge_kway", st, total, (k_kw_merge<4><<<(nde + kw_threads(4) - 1) / kw_threads(4), kw_threads(4), 0,
                                                               st>>>(D, T, dpos, drank, dend, order, nde, perm_out, lcp_out)));
        else
            SS_LAUNCH_U("merge_kway", st, total, (k_kw_merge<8><<<(nde + kw_threads(8) - 1) / kw_threads(8), kw_threads(8), 0,
                                                               st>>>(D, T, dpos, drank, dend, order, nde, perm_out, lcp_out)));
        if ((rc = kw_check(cudaGetLastError(), "ss_merge launch")) != SS_OK) break;
        rc = kw_check(cudaStreamSynchronize(st), "ss_merge");
    } while (0);
    scratch_free(block, st);
    return rc;
}

}  // namespace ss
