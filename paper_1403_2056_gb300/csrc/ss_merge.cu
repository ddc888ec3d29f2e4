// LCP-aware merging of sorted runs (Section 5: LCP-Compare, Algorithm 2;
// binary LCP-merge, Algorithm 3) on one GPU.
//
// The paper merges K runs with one LCP-aware tournament tree per job and
// splits jobs by LCP minima (Section 5.3).  On the GPU the K-way merge is
// ceil(log2 K) rounds of pairwise merges.  Inside a round the output of every
// pair is cut by merge path (a search on the cross diagonal by a group of
// lanes, full string comparisons) at every kCoarse outputs, with the
// characters each window's strings share; then every chunk of kMergeItems
// outputs gets its start (the search inside its window, from the shared
// prefix, and the LCPs of both fronts with the string before the chunk: one
// side's is the run's own LCP entry, the other comes from the search's last
// probes where unequal LCPs decide, else from one string comparison).  The
// merge proper runs per CTA window of kMergeTile outputs: each thread runs
// the binary LCP-merge over its chunk, reading the window's LCPs and cached
// characters through L1, and the CTA writes the outputs with coalesced
// stores staged in shared memory.
// Comparisons whose LCPs differ cost no string access at all (cases 2 and 3
// of LCP-Compare); equal LCPs first try the cached characters, and only then
// read characters, 16 at a time from the known common prefix on; the front
// that stays keeps the characters read last as its cache.  Round 1 takes the
// runs' offsets and cached characters from the sort when the caller has them
// (ss_merge_cached), else loads them itself (k_run_prep).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <string.h>
#include <vector>

#include "ss_internal.cuh"

namespace ss {

#ifndef SS_MERGE_ITEMS
#define SS_MERGE_ITEMS 16
#endif
constexpr uint32_t kMergeItems = SS_MERGE_ITEMS;   // outputs per thread
#ifndef SS_MERGE_COARSE
#define SS_MERGE_COARSE 1024
#endif
constexpr uint32_t kCoarse = SS_MERGE_COARSE;   // outputs per merge-path window

// full comparison of strings a and b from depth h on (both share h characters),
// 16 characters per round; returns -1/0/+1 and the lcp in *l
// str_cmp_from that also hands back the 8 characters of both strings from
// depth *kd where it decided (*kd <= *l < *kd + 8, or both end there): the
// merge keeps them as the characters cached for the front that stays
__device__ __forceinline__ int str_cmp_keys(const ReqDesc &S, uint32_t a, uint64_t oa, uint32_t b, uint64_t ob,
                                            uint32_t h, uint32_t *l, uint64_t *ka, uint64_t *kb, uint32_t *kd) {
    for (;;) {
        uint64_t a0, a1, b0, b1;
        load_key2_o(S, a, oa, h, a0, a1);
        load_key2_o(S, b, ob, h, b0, b1);
        if (a0 != b0 || has_zero(a0)) {
            *ka = a0; *kb = b0; *kd = h;
            if (a0 != b0) { *l = h + lcp8(a0, b0); return a0 < b0 ? -1 : 1; }
            *l = h + nulpos(a0);
            return 0;
        }
        if (a1 != b1 || has_zero(a1)) {
            *ka = a1; *kb = b1; *kd = h + 8;
            if (a1 != b1) { *l = h + 8 + lcp8(a1, b1); return a1 < b1 ? -1 : 1; }
            *l = h + 8 + nulpos(a1);
            return 0;
        }
        h += 16;
    }
}

__device__ __forceinline__ int str_cmp_from(const ReqDesc &S, uint32_t a, uint64_t oa, uint32_t b, uint64_t ob,
                                            uint32_t h, uint32_t *l) {
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


// pair (2p, 2p+1) of the round's runs; an unpaired last run has B empty.
// With a table of string offsets aligned to the runs (Ao/Bo) every string
// access is one random load; without one the set's offsets are looked up.
struct PairView {
    uint32_t a0, na, nb, baseA, baseB;
    const uint32_t *Ap, *Bp, *HA, *HB;
    const uint64_t *Ao, *Bo, *offsets;
    __device__ __forceinline__ uint32_t A(uint32_t k) const { return Ap[k] + baseA; }
    __device__ __forceinline__ uint32_t B(uint32_t k) const { return Bp[k] + baseB; }
    __device__ __forceinline__ uint64_t OA(uint32_t k) const { return Ao ? Ao[k] : __ldg(offsets + A(k)); }
    __device__ __forceinline__ uint64_t OB(uint32_t k) const { return Bo ? Bo[k] : __ldg(offsets + B(k)); }
};

__device__ __forceinline__ PairView pair_view(const ReqDesc &S, uint32_t p, const uint32_t *in_perm,
                                              const uint32_t *in_lcp, const uint64_t *in_off, const uint32_t *rb,
                                              uint32_t R, const uint32_t *rbase) {
    PairView v;
    uint32_t a1 = rb[2 * p + 1];
    uint32_t b1 = (2 * p + 1 < R) ? rb[2 * p + 2] : a1;
    v.a0 = rb[2 * p];
    v.na = a1 - v.a0;
    v.nb = b1 - a1;
    v.Ap = in_perm + v.a0;
    v.Bp = in_perm + a1;
    v.HA = in_lcp + v.a0;
    v.HB = in_lcp + a1;
    v.Ao = in_off ? in_off + v.a0 : nullptr;
    v.Bo = in_off ? in_off + a1 : nullptr;
    v.offsets = S.offsets;
    // string index of a run entry: entry + the run's index base (first round only)
    v.baseA = rbase ? rbase[2 * p] : 0u;
    v.baseB = (rbase && 2 * p + 1 < R) ? rbase[2 * p + 1] : 0u;
    return v;
}

// merge path: number of strings taken from A among the first diag outputs
// (A first on ties), searched in [lo, hi); all compared strings share h characters
// Merge-path search on diagonal diag inside [lo, hi), comparing from depth h.
// The probe that set the final lo (at i - 1, against B[diag - i]) and the one
// that set the final hi (at i, against B[diag - i - 1]) leave their LCPs in
// *la / *lb, each with a flag (false: that bound was never moved).
struct PathEnd {
    uint32_t i, la, lb;
    bool has_la, has_lb;
};
__device__ __forceinline__ PathEnd path_search_lcp(const ReqDesc &S, const PairView &v, uint32_t diag, uint32_t lo,
                                                   uint32_t hi, uint32_t h) {
    PathEnd r{0u, 0u, 0u, false, false};
    while (lo < hi) {
        uint32_t mid = (lo + hi) / 2;
        uint32_t l, bj = diag - 1 - mid;
        if (str_cmp_from(S, v.A(mid), v.OA(mid), v.B(bj), v.OB(bj), h, &l) <= 0) {
            lo = mid + 1;
            r.la = l;
            r.has_la = true;
        } else {
            hi = mid;
            r.lb = l;
            r.has_lb = true;
        }
    }
    r.i = lo;
    return r;
}
__device__ __forceinline__ uint32_t path_search(const ReqDesc &S, const PairView &v, uint32_t diag, uint32_t lo,
                                                uint32_t hi, uint32_t h) {
    return path_search_lcp(S, v, diag, lo, hi, h).i;
}

// string offset of every run entry, for the first round
// Per round, for every run entry: its string offset (first round: looked up
// and written to off; later rounds: carried in off) and its cached characters
// ck = the 8 characters at its run LCP (0 for a run's first entry), the
// distinguishing characters that the caching variant of Section 5.4 keeps so
// that LCP-Compare's first character comparison needs no string access.
__global__ void k_run_prep(ReqDesc S, const uint32_t *in_perm, const uint32_t *in_lcp, const uint32_t *rb, uint32_t R,
                           const uint32_t *rbase, uint32_t total, int lookup_offsets, uint64_t *off, uint64_t *ck,
                           uint32_t *ckd) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < total; p += gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = R;   // run of position p
        while (hi - lo > 1) {
            uint32_t mid = (lo + hi) / 2;
            if (rb[mid] <= p) lo = mid; else hi = mid;
        }
        uint32_t id = in_perm[p] + (rbase ? rbase[lo] : 0u);
        uint64_t o;
        if (lookup_offsets) {
            o = __ldg(S.offsets + id);
            off[p] = o;
        } else {
            o = off[p];
        }
        uint32_t d = p == rb[lo] ? 0u : in_lcp[p];
        ck[p] = load_key_o(S, id, o, d);
        ckd[p] = d;
    }
}

struct Coarse {
    uint32_t i;   // strings from A among the outputs before this window's first output
    uint32_t h;   // characters shared by every string of the window
};

__device__ __forceinline__ uint32_t pair_of_entry(const uint32_t *cbase, uint32_t npairs, uint32_t e) {
    uint32_t lo = 0, hi = npairs;   // last pair with cbase[p] <= e
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) / 2;
        if (cbase[mid] <= e) lo = mid; else hi = mid;
    }
    return lo;
}

// The same search by a group of kCutLanes lanes: each round the lanes test
// kCutLanes evenly spaced candidates at once (the comparison is monotone in
// the candidate), and the range shrinks to the gap between the last one that
// does not pass A and the first that does, kCutLanes + 1 times smaller.  A cut
// searches a whole pair from depth 0; with few cuts (one per kCoarse outputs)
// the chain of dependent string reads bounds the kernel, which the group
// shortens from log2 to log_(kCutLanes+1) of the pair length.  Measured on
// GB300 (4 runs of 10 M URL-like / 20 M DNA strings): 4 lanes with 1024-output
// windows beat one lane with 256-output windows by 6 % / 2 % of the merge.
#ifndef SS_CUT_LANES
#define SS_CUT_LANES 4
#endif
constexpr uint32_t kCutLanes = SS_CUT_LANES;   // a power of two, at most 32
constexpr uint32_t kCutMask = kCutLanes == 32 ? 0xFFFFFFFFu : ((1u << kCutLanes) - 1);
static_assert((kCutLanes & (kCutLanes - 1)) == 0 && kCutLanes >= 1 && kCutLanes <= 32, "lanes per cut");

__device__ __forceinline__ uint32_t path_search_group(const ReqDesc &S, const PairView &v, uint32_t diag, uint32_t lo,
                                                      uint32_t hi, uint32_t glane, uint32_t gmask, uint32_t gshift) {
    while (lo < hi) {
        const uint32_t n = hi - lo;
        auto probe = [&](uint32_t k) { return lo + (uint32_t)(((uint64_t)(k + 1) * n) / (kCutLanes + 1)); };
        const uint32_t x = probe(glane);   // in [lo, hi)
        uint32_t l;
        const bool past = str_cmp_from(S, v.A(x), v.OA(x), v.B(diag - 1 - x), v.OB(diag - 1 - x), 0, &l) > 0;
        const uint32_t votes = (__ballot_sync(gmask, past) >> gshift) & kCutMask;
        const uint32_t first = votes ? (uint32_t)(__ffs(votes) - 1) : kCutLanes;   // first probe past A
        const uint32_t nlo = first > 0 ? probe(first - 1) + 1 : lo;
        const uint32_t nhi = first < kCutLanes ? probe(first) : hi;
        lo = nlo;
        hi = nhi;
    }
    return lo;
}

// window cuts: pair p has entries cbase[p] + k for diagonals min(k kCoarse, na + nb);
// kCutLanes consecutive lanes per entry
__global__ void k_merge_cuts(ReqDesc S, const uint32_t *in_perm, const uint32_t *in_lcp, const uint64_t *in_off,
                             const uint32_t *rb, uint32_t R, const uint32_t *rbase, const uint32_t *cbase,
                             uint32_t npairs, uint32_t nentries, Coarse *C) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t e = g / kCutLanes, glane = g % kCutLanes;
    if (e >= nentries) return;   // whole groups leave together
    const uint32_t gshift = (threadIdx.x & 31) & ~(kCutLanes - 1);
    const uint32_t gmask = kCutMask << gshift;
    uint32_t p = pair_of_entry(cbase, npairs, e);
    PairView v = pair_view(S, p, in_perm, in_lcp, in_off, rb, R, rbase);
    uint32_t len = v.na + v.nb;
    uint32_t diag = min((e - cbase[p]) * kCoarse, len);
    uint32_t lo = diag > v.nb ? diag - v.nb : 0, hi = min(diag, v.na);
    const uint32_t i = path_search_group(S, v, diag, lo, hi, glane, gmask, gshift);
    if (glane == 0) C[e].i = i;
}

// characters shared by a whole window: the strings of a window are a
// contiguous run of the merged order, so they share min(lcp(A_i0, A_i1-1),
// lcp(B_j0, B_j1-1), lcp(A_i0, B_j0)) characters
__global__ void k_merge_windows(ReqDesc S, const uint32_t *in_perm, const uint32_t *in_lcp, const uint64_t *in_off,
                                const uint32_t *rb, uint32_t R, const uint32_t *rbase, const uint32_t *cbase,
                                uint32_t npairs, uint32_t nentries, Coarse *C) {
    uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nentries) return;
    uint32_t p = pair_of_entry(cbase, npairs, e);
    uint32_t last = (p + 1 < npairs ? cbase[p + 1] : nentries) - 1;
    if (e == last) { C[e].h = 0; return; }
    PairView v = pair_view(S, p, in_perm, in_lcp, in_off, rb, R, rbase);
    uint32_t len = v.na + v.nb;
    uint32_t k = e - cbase[p];
    uint32_t d0 = min(k * kCoarse, len), d1 = min((k + 1) * kCoarse, len);
    uint32_t i0 = C[e].i, i1 = C[e + 1].i, j0 = d0 - i0, j1 = d1 - i1;
    uint32_t h = 0xFFFFFFFFu, l;
    if (i1 > i0) { str_cmp_from(S, v.A(i0), v.OA(i0), v.A(i1 - 1), v.OA(i1 - 1), 0, &l); h = min(h, l); }
    if (j1 > j0) { str_cmp_from(S, v.B(j0), v.OB(j0), v.B(j1 - 1), v.OB(j1 - 1), 0, &l); h = min(h, l); }
    if (i1 > i0 && j1 > j0) { str_cmp_from(S, v.A(i0), v.OA(i0), v.B(j0), v.OB(j0), 0, &l); h = min(h, l); }
    C[e].h = h == 0xFFFFFFFFu ? 0u : h;
}

__device__ __forceinline__ uint32_t upper_run(const uint32_t *rb, uint32_t R, uint32_t o) {
    uint32_t lo = 0, hi = R;   // last run with rb[run] <= o
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) / 2;
        if (rb[mid] <= o) lo = mid; else hi = mid;
    }
    return lo;
}

// One round: pair (2p, 2p+1) of the R runs rb[0..R] is merged into the same
// output positions; an unpaired last run is copied.  With a window table
// (C, cbase) each thread's merge path search stays inside its window and
// compares from the window's shared prefix; without one (C == NULL) it
// searches the whole pair from depth 0.
__global__ void k_merge_round(ReqDesc S, const uint32_t *in_perm, const uint32_t *in_lcp, const uint32_t *rb, uint32_t R,
                              const uint32_t *rbase, uint32_t total, uint32_t *out_perm, uint32_t *out_lcp,
                              const Coarse *C, const uint32_t *cbase, const uint64_t *in_off, uint64_t *out_off,
                              const uint64_t *ck, const uint32_t *ckd, uint64_t *out_ck, uint32_t *out_ckd) {
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t o64 = (uint64_t)t * kMergeItems;
    if (o64 >= total) return;
    uint32_t o = (uint32_t)o64;
    const uint32_t end = (o64 + kMergeItems < (uint64_t)total) ? (uint32_t)(o64 + kMergeItems) : total;
    while (o < end) {
        uint32_t r = upper_run(rb, R, o);
        uint32_t p = r / 2;
        const PairView v = pair_view(S, p, in_perm, in_lcp, in_off, rb, R, rbase);
        const uint32_t a0 = v.a0, na = v.na, nb = v.nb;
        const uint32_t *HA = v.HA, *HB = v.HB;
        auto A = [&](uint32_t k) { return v.A(k); };
        auto B = [&](uint32_t k) { return v.B(k); };
        auto OA = [&](uint32_t k) { return v.OA(k); };
        auto OB = [&](uint32_t k) { return v.OB(k); };
        const uint32_t pair_end = a0 + na + nb;
        const uint32_t stop = min(end, pair_end);
        uint32_t diag = o - a0;
        uint32_t lo = diag > nb ? diag - nb : 0, hi = min(diag, na);
        // window of the diagonal: strings A[i0, i1) and B[j0, j1) share hw characters
        uint32_t i0 = 0, i1 = na, j0 = 0, j1 = nb, hw = 0;
        bool win = C != nullptr;
        uint32_t i;
        if (win) {
            uint32_t k = diag / kCoarse;
            uint32_t e = cbase[p] + k;
            uint32_t d0 = k * kCoarse;
            i0 = C[e].i;
            j0 = d0 - i0;
            if (d0 == diag) {
                i = i0;
                win = false;   // exact cut: no search, no shared prefix needed
            } else {
                uint32_t d1 = min(d0 + kCoarse, na + nb);
                i1 = C[e + 1].i;
                j1 = d1 - i1;
                hw = C[e].h;
                lo = max(lo, max(i0, diag > j1 ? diag - j1 : 0u));
                hi = min(hi, min(i1, diag - j0));
                i = path_search(S, v, diag, lo, hi, hw);
            }
        } else {
            i = path_search(S, v, diag, lo, hi, 0);
        }
        uint32_t j = diag - i;
        auto inA = [&](uint32_t x) { return win && x >= i0 && x < i1; };
        auto inB = [&](uint32_t y) { return win && y >= j0 && y < j1; };
        // LCPs of both fronts with the last string written before position o
        uint32_t ha = 0, hb = 0;
        if (diag > 0) {
            bool last_is_b;
            if (i == 0) last_is_b = true;
            else if (j == 0) last_is_b = false;
            else {
                uint32_t l;
                uint32_t h0 = (inA(i - 1) && inB(j - 1)) ? hw : 0u;
                last_is_b = str_cmp_from(S, A(i - 1), OA(i - 1), B(j - 1), OB(j - 1), h0, &l) <= 0;   // ties: A then B
            }
            uint32_t prev = last_is_b ? B(j - 1) : A(i - 1);
            uint64_t prev_o = last_is_b ? OB(j - 1) : OA(i - 1);
            bool prev_in = last_is_b ? inB(j - 1) : inA(i - 1);
            if (i < na) {
                if (!last_is_b) ha = HA[i];
                else { uint32_t l; str_cmp_from(S, prev, prev_o, A(i), OA(i), (prev_in && inA(i)) ? hw : 0u, &l); ha = l; }
            }
            if (j < nb) {
                if (last_is_b) hb = HB[j];
                else { uint32_t l; str_cmp_from(S, prev, prev_o, B(j), OB(j), (prev_in && inB(j)) ? hw : 0u, &l); hb = l; }
            }
        }
        // cached characters of the fronts: 8 bytes of the string at depth kd
        // (kd = ~0: none), refreshed from (ck, ckd) whenever a front advances;
        // a cache is a fact about its string, so it travels with the string
        // into the next round
        uint32_t kdA = ~0u, kdB = ~0u;
        uint64_t kA = 0, kB = 0;
        auto cacheA = [&]() {
            if (ck && i < na) { kdA = ckd[a0 + i]; kA = ck[a0 + i]; } else kdA = ~0u;
        };
        auto cacheB = [&]() {
            if (ck && j < nb) { kdB = ckd[a0 + na + j]; kB = ck[a0 + na + j]; } else kdB = ~0u;
        };
        cacheA();
        cacheB();
        // binary LCP-merge (Algorithm 3) over positions [o, stop)
        for (; o < stop; o++) {
            bool take_b;
            uint32_t hp = 0;
            bool both = i < na && j < nb;
            if (!both) {
                take_b = i >= na;
            } else if (ha == hb) {   // case 1: compare characters from the common LCP on
                const uint32_t h = ha;
                bool decided = false;
                if (kdA <= h && kdB <= h && h - kdA < 8 && h - kdB < 8) {
                    // both fronts' cached bytes cover depth h: compare the overlap
                    const uint32_t sa = h - kdA, sb = h - kdB;
                    const uint64_t wa = kA << (8 * sa), wb = kB << (8 * sb);
                    const uint32_t nk = 8 - max(sa, sb);   // bytes known for both from h on
                    const uint64_t mask = ~0ull << (64 - 8 * nk);
                    const uint64_t x = (wa ^ wb) & mask;
                    if (x) {
                        hp = h + (uint32_t)(__clzll(x) >> 3);
                        take_b = (wa & mask) > (wb & mask);
                        decided = true;
                    } else {
                        const uint64_t z = zero_bytes(wa) & mask;   // both end inside the overlap: equal
                        if (z) {
                            hp = h + (uint32_t)(__clzll(z) >> 3);
                            take_b = false;
                            decided = true;
                        }
                    }
                }
                if (!decided) {
                    int c = str_cmp_from(S, A(i), OA(i), B(j), OB(j), h, &hp);
                    take_b = c > 0;
                }
            } else if (ha < hb) {    // case 2: B is smaller
                take_b = true;
                hp = ha;
            } else {                 // case 3: A is smaller
                take_b = false;
                hp = hb;
            }
            if (!take_b) {
                out_perm[o] = A(i);
                if (out_off) out_off[o] = OA(i);
                if (out_ck) { out_ck[o] = kA; out_ckd[o] = kdA; }
                out_lcp[o] = (o == a0) ? 0u : ha;
                i++;
                ha = i < na ? HA[i] : 0;
                if (both) hb = hp;
                cacheA();
            } else {
                out_perm[o] = B(j);
                if (out_off) out_off[o] = OB(j);
                if (out_ck) { out_ck[o] = kB; out_ckd[o] = kdB; }
                out_lcp[o] = (o == a0) ? 0u : hb;
                j++;
                hb = j < nb ? HB[j] : 0;
                if (both) ha = hp;
                cacheB();
            }
        }
    }
}

#ifndef SS_MERGE_TILE_THREADS
#define SS_MERGE_TILE_THREADS 256
#endif
constexpr uint32_t kMergeTileThreads = SS_MERGE_TILE_THREADS;
// CTAs per SM the merge tile must fit by registers: 6 (40 registers, a few
// bytes spilled) measured faster than the 5 its 47 registers allow (its
// lanes wait on dependent reads, more warps hide more); the chunk-start
// search measured slower when held to fewer registers
#ifndef SS_MERGE_TILE_MINB
#define SS_MERGE_TILE_MINB 6
#endif
constexpr uint32_t kMergeTile = kMergeTileThreads * kMergeItems;   // outputs per CTA window
static_assert(kMergeTile % kCoarse == 0, "a CTA window is a whole number of merge-path windows");
static_assert(kMergeTile <= 65536, "tile-local sources are 16-bit");

struct MergeStart {   // where a thread's outputs start: strings taken from A, front LCPs
    uint32_t i, ha, hb, pad;
};

// window w of pair p: outputs [d0, d1) of the pair, C entries k0 .. k1
struct MergeWindow {
    uint32_t p, d0, d1, k0, k1;
};

__device__ __forceinline__ MergeWindow merge_window(const uint32_t *wbase, uint32_t npairs, uint32_t len_of_pair,
                                                    uint32_t p, uint32_t w) {
    MergeWindow mw;
    mw.p = p;
    mw.d0 = w * kMergeTile;
    mw.d1 = min(mw.d0 + kMergeTile, len_of_pair);
    const uint32_t nent = (len_of_pair + kCoarse - 1) / kCoarse;   // C holds diagonals min(k kCoarse, len), k = 0..nent
    mw.k0 = mw.d0 / kCoarse;
    mw.k1 = mw.d1 == len_of_pair ? nent : mw.d1 / kCoarse;
    return mw;
}

// Start of every thread's kMergeItems outputs, one thread per chunk of a
// window (same grid shape as k_merge_tile): the merge-path search inside the
// kCoarse window of its diagonal, from the window's shared prefix, and the
// LCPs of both fronts with the string output just before the chunk.  These are
// most of the string accesses of a round; they run here, apart from the merge
// tile, at the occupancy the registers allow.
__global__ void __launch_bounds__(kMergeTileThreads) k_merge_starts(
    ReqDesc S, const uint32_t *in_perm, const uint32_t *in_lcp, const uint32_t *rb, uint32_t R, const uint32_t *rbase,
    const uint32_t *wbase, uint32_t npairs, const Coarse *C, const uint32_t *cbase, const uint64_t *in_off,
    MergeStart *starts) {
    const uint32_t p = pair_of_entry(wbase, npairs, blockIdx.x);
    const PairView v = pair_view(S, p, in_perm, in_lcp, in_off, rb, R, rbase);
    const uint32_t na = v.na, nb = v.nb, len = na + nb;
    const MergeWindow mw = merge_window(wbase, npairs, len, p, blockIdx.x - wbase[p]);
    const uint32_t diag = mw.d0 + threadIdx.x * kMergeItems;
    if (diag >= mw.d1) return;
    uint32_t lo = diag > nb ? diag - nb : 0, hi = min(diag, na);
    const uint32_t k = diag / kCoarse, e = cbase[p] + k, dc = k * kCoarse;
    const uint32_t i0 = C[e].i, j0 = dc - i0;
    uint32_t i1 = na, j1 = nb, hw = 0;
    PathEnd pe{i0, 0u, 0u, false, false};
    bool win = true;
    if (dc == diag) {
        win = false;   // exact cut: no search, no shared prefix needed
    } else {
        const uint32_t dce = min(dc + kCoarse, len);
        i1 = C[e + 1].i;
        j1 = dce - i1;
        hw = C[e].h;
        lo = max(lo, max(i0, diag > j1 ? diag - j1 : 0u));
        hi = min(hi, min(i1, diag - j0));
        pe = path_search_lcp(S, v, diag, lo, hi, hw);
    }
    const uint32_t i = pe.i, j = diag - i;
    auto inA = [&](uint32_t x) { return win && x >= i0 && x < i1; };
    auto inB = [&](uint32_t y) { return win && y >= j0 && y < j1; };
    uint32_t ha = 0, hb = 0;
    if (diag > 0) {
        // which of A[i - 1] and B[j - 1] is output last.  The search's last
        // probes give lb = lcp(A[i], B[j - 1]) (B[j - 1] < A[i]) and
        // la = lcp(A[i - 1], B[j]) (A[i - 1] <= B[j]); with the run LCPs
        // HA[i] = lcp(A[i - 1], A[i]) and HB[j] = lcp(B[j - 1], B[j]), of two
        // strings below the same string the one that shares more with it is
        // the larger, so unequal LCPs decide without reading a string
        bool last_is_b = false, known = false;
        if (i == 0) { last_is_b = true; known = true; }
        else if (j == 0) { last_is_b = false; known = true; }
        else if (pe.has_lb && i < na && v.HA[i] != pe.lb) { last_is_b = v.HA[i] < pe.lb; known = true; }
        else if (pe.has_la && j < nb && v.HB[j] != pe.la) { last_is_b = v.HB[j] > pe.la; known = true; }
        if (!known) {
            uint32_t l;
            uint32_t h0 = (inA(i - 1) && inB(j - 1)) ? hw : 0u;
            last_is_b = str_cmp_from(S, v.A(i - 1), v.OA(i - 1), v.B(j - 1), v.OB(j - 1), h0, &l) <= 0;   // ties: A then B
        }
        const uint32_t prev = last_is_b ? v.B(j - 1) : v.A(i - 1);
        const uint64_t prev_o = last_is_b ? v.OB(j - 1) : v.OA(i - 1);
        const bool prev_in = last_is_b ? inB(j - 1) : inA(i - 1);
        if (i < na) {
            if (!last_is_b) ha = v.HA[i];
            else if (pe.has_lb) ha = pe.lb;   // lcp(B[j - 1], A[i]) from the probe at i
            else { uint32_t l; str_cmp_from(S, prev, prev_o, v.A(i), v.OA(i), (prev_in && inA(i)) ? hw : 0u, &l); ha = l; }
        }
        if (j < nb) {
            if (last_is_b) hb = v.HB[j];
            else if (pe.has_la) hb = pe.la;   // lcp(A[i - 1], B[j]) from the probe at i - 1
            else { uint32_t l; str_cmp_from(S, prev, prev_o, v.B(j), v.OB(j), (prev_in && inB(j)) ? hw : 0u, &l); hb = l; }
        }
    }
    starts[blockIdx.x * kMergeTileThreads + threadIdx.x] = MergeStart{i, ha, hb, 0u};
}

struct MergeTileSmem {
    uint32_t olcp[kMergeTile];   // per output: LCP with the output before it
    uint16_t src[kMergeTile];    // per output: which window entry it is
};

// One round of pairwise merges, one CTA per window of kMergeTile outputs of a
// pair (windows do not straddle pairs; wbase[p] = first window of pair p).  The
// window's run entries (LCPs and cached characters) are read through L1, each
// thread walking its own consecutive entries of both runs (not staged in
// shared memory: that held the CTAs per SM to a third and measured slower);
// from its start (k_merge_starts) each thread runs the binary LCP-merge
// (Algorithm 3) over kMergeItems outputs and records which entry each output
// is and its LCP; the CTA then writes all outputs with coalesced stores.  Only
// the case-1 comparisons that the cached characters leave open read strings.
__global__ void __launch_bounds__(kMergeTileThreads, SS_MERGE_TILE_MINB) k_merge_tile(
    ReqDesc S, const uint32_t *in_perm, const uint32_t *in_lcp, const uint32_t *rb, uint32_t R, const uint32_t *rbase,
    const uint32_t *wbase, uint32_t npairs, uint32_t *out_perm, uint32_t *out_lcp, const Coarse *C,
    const uint32_t *cbase, const MergeStart *starts, const uint64_t *in_off, uint64_t *out_off, const uint64_t *ck,
    const uint32_t *ckd, uint64_t *out_ck, uint32_t *out_ckd) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MergeTileSmem &T = *reinterpret_cast<MergeTileSmem *>(smem_raw);
    const uint32_t p = pair_of_entry(wbase, npairs, blockIdx.x);
    const PairView v = pair_view(S, p, in_perm, in_lcp, in_off, rb, R, rbase);
    const uint32_t a0 = v.a0, na = v.na, nb = v.nb, len = na + nb;
    const MergeWindow mw = merge_window(wbase, npairs, len, p, blockIdx.x - wbase[p]);
    const uint32_t d0 = mw.d0, d1 = mw.d1;
    const uint32_t I0 = C[cbase[p] + mw.k0].i, I1 = C[cbase[p] + mw.k1].i;
    const uint32_t J0 = d0 - I0, J1 = d1 - I1;
    const uint32_t nA = I1 - I0, nW = d1 - d0;
    const uint32_t dl = threadIdx.x * kMergeItems;
    MergeStart ms{0u, 0u, 0u, 0u};
    if (dl < nW) ms = starts[blockIdx.x * kMergeTileThreads + threadIdx.x];
    // the window's entries: x < nA is A's entry I0 + x, else B's entry J0 + x - nA
    auto gpos = [&](uint32_t x) { return x < nA ? a0 + I0 + x : a0 + na + J0 + (x - nA); };   // run-aligned position
    auto e_lcp = [&](uint32_t x) { return __ldg(in_lcp + gpos(x)); };
    auto e_ck = [&](uint32_t x) { return ck ? __ldg(ck + gpos(x)) : 0ull; };
    auto e_ckd = [&](uint32_t x) { return ck ? __ldg(ckd + gpos(x)) : ~0u; };
    if (dl < nW) {
        const uint32_t diag = d0 + dl;
        const uint32_t stop = min(dl + kMergeItems, nW);
        uint32_t i = ms.i, j = diag - ms.i, ha = ms.ha, hb = ms.hb;
        // fronts' cached characters (depth kd, ~0: none)
        uint32_t kdA = ~0u, kdB = ~0u;
        uint64_t kA = 0, kB = 0;
        if (i < I1) { kdA = e_ckd(i - I0); kA = e_ck(i - I0); }
        if (j < J1) { kdB = e_ckd(nA + j - J0); kB = e_ck(nA + j - J0); }
        for (uint32_t s = dl; s < stop; s++) {
            // the window holds exactly the entries its outputs take: a side past
            // its part of the window is exhausted here
            const bool hasA = i < I1, hasB = j < J1;
            bool take_b;
            uint32_t hp = 0;
            const bool both = hasA && hasB;
            if (!both) {
                take_b = !hasA;
            } else if (ha == hb) {   // case 1: compare characters from the common LCP on
                const uint32_t h = ha;
                bool decided = false;
                if (kdA <= h && kdB <= h && h - kdA < 8 && h - kdB < 8) {
                    const uint32_t sa = h - kdA, sb = h - kdB;
                    const uint64_t wa = kA << (8 * sa), wb = kB << (8 * sb);
                    const uint32_t nk = 8 - max(sa, sb);   // bytes known for both from h on
                    const uint64_t mask = ~0ull << (64 - 8 * nk);
                    const uint64_t x = (wa ^ wb) & mask;
                    if (x) {
                        hp = h + (uint32_t)(__clzll(x) >> 3);
                        take_b = (wa & mask) > (wb & mask);
                        decided = true;
                    } else {
                        const uint64_t z = zero_bytes(wa) & mask;   // both end inside the overlap: equal
                        if (z) {
                            hp = h + (uint32_t)(__clzll(z) >> 3);
                            take_b = false;
                            decided = true;
                        }
                    }
                }
                if (!decided) {
                    // the front that stays keeps the characters this comparison read
                    // at its new LCP (the one that is output is replaced below)
                    uint64_t ka, kb;
                    uint32_t kd;
                    take_b = str_cmp_keys(S, v.A(i), v.OA(i), v.B(j), v.OB(j), h, &hp, &ka, &kb, &kd) > 0;
                    kA = ka; kdA = kd;
                    kB = kb; kdB = kd;
                }
            } else if (ha < hb) {    // case 2: B is smaller
                take_b = true;
                hp = ha;
            } else {                 // case 3: A is smaller
                take_b = false;
                hp = hb;
            }
            if (!take_b) {
                T.src[s] = (uint16_t)(i - I0);
                T.olcp[s] = diag + (s - dl) == 0 ? 0u : ha;
                i++;
                ha = i < I1 ? e_lcp(i - I0) : 0u;
                if (both) hb = hp;
                if (i < I1) { kdA = e_ckd(i - I0); kA = e_ck(i - I0); } else kdA = ~0u;
            } else {
                T.src[s] = (uint16_t)(nA + j - J0);
                T.olcp[s] = diag + (s - dl) == 0 ? 0u : hb;
                j++;
                hb = j < J1 ? e_lcp(nA + j - J0) : 0u;
                if (both) ha = hp;
                if (j < J1) { kdB = e_ckd(nA + j - J0); kB = e_ck(nA + j - J0); } else kdB = ~0u;
            }
        }
    }
    __syncthreads();
    // coalesced write of the window's outputs
    for (uint32_t s = threadIdx.x; s < nW; s += kMergeTileThreads) {
        const uint32_t x = T.src[s];
        const bool fromA = x < nA;
        const uint32_t g = gpos(x);
        const uint32_t o = a0 + d0 + s;
        const uint32_t id = in_perm[g] + (fromA ? v.baseA : v.baseB);
        out_perm[o] = id;
        out_lcp[o] = T.olcp[s];
        if (out_off) out_off[o] = in_off ? in_off[g] : __ldg(S.offsets + id);
        if (out_ck) { out_ck[o] = e_ck(x); out_ckd[o] = e_ckd(x); }
    }
}

// a single run: copy with its index base added; its first LCP becomes 0
__global__ void k_copy_run(const uint32_t *in_perm, const uint32_t *in_lcp, uint32_t base, uint32_t total,
                           uint32_t *out_perm, uint32_t *out_lcp) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        out_perm[i] = in_perm[i] + base;
        out_lcp[i] = i ? in_lcp[i] : 0u;
    }
}

int merge_runs(const ReqDesc &set, const uint32_t *run_perm, const uint32_t *run_lcp, const uint32_t *run_begin_host,
               const uint32_t *run_base_host, uint32_t K, uint32_t *perm_out, uint32_t *lcp_out, cudaStream_t st,
               uint32_t method, RunCache cache) {
    uint32_t total = run_begin_host[K];
    // drop empty runs (they merge as nothing)
    std::vector<uint32_t> rb{0}, rbase;
    for (uint32_t k = 0; k < K; k++)
        if (run_begin_host[k + 1] > run_begin_host[k]) {
            rb.push_back(run_begin_host[k + 1]);
            rbase.push_back(run_base_host ? run_base_host[k] : 0u);
        }
    uint32_t R = (uint32_t)rb.size() - 1;
    // the loser-tree method: one pass over up to kKwayMaxRuns runs (ss_kway.cu);
    // more runs go through the pairwise rounds below
    if (method == MERGE_LOSER_TREE && R >= 2 && R <= kKwayMaxRuns)
        return merge_kway(set, run_perm, run_lcp, rb.data(), rbase.data(), R, perm_out, lcp_out, st);
    size_t rounds = 0;
    for (uint32_t r = R; r > 1; r = (r + 1) / 2) rounds++;
    // window table: at most total / kCoarse + 2 entries per pair
    const size_t max_entries = (size_t)total / kCoarse + 2ull * (K + 1) + 2;
    const size_t a64 = 63;
    const size_t tot64 = ((size_t)total + a64) & ~a64;
    // thread starts: one per kMergeItems outputs, at most one partial window per pair
    const size_t max_starts = ((size_t)total / kMergeTile + K + 2) * kMergeTileThreads;
    // one table region per round (rb, bases, cbase, wbase), so no round waits for the host
    const size_t tstride = (4 * (K + 2) + 63) & ~(size_t)63;
    const size_t nrt = rounds ? rounds : 1;
    size_t bytes = 4ull * 8 * tot64 + 4ull * 4 * tot64 + 4ull * tstride * nrt + sizeof(Coarse) * max_entries +
                   sizeof(MergeStart) * max_starts + 4096;
    void *block = nullptr;
    cudaError_t e = scratch_alloc(&block, bytes, st);
    if (e) {
        cudaGetLastError();
        set_error_detail("ss_merge: scratch allocation of %zu bytes failed", bytes);
        return SS_ERR_OOM;
    }
    // string offsets and cached characters (bytes, depth) aligned to the runs,
    // ping-pong across rounds
    uint64_t *off_buf[2] = {(uint64_t *)block, (uint64_t *)block + tot64};
    uint64_t *ck_buf[2] = {off_buf[1] + tot64, off_buf[1] + 2 * tot64};
    uint32_t *ckd_buf[2] = {(uint32_t *)(ck_buf[1] + tot64), (uint32_t *)(ck_buf[1] + tot64) + tot64};
    uint32_t *tmp_perm = ckd_buf[1] + tot64;
    uint32_t *tmp_lcp = tmp_perm + tot64;
    uint32_t *d_tables = tmp_lcp + tot64;   // per round: rb[R+1], bases[R], cbase[pairs], wbase[pairs]
    Coarse *d_coarse = (Coarse *)(d_tables + tstride * nrt);
    MergeStart *d_starts = (MergeStart *)(d_coarse + ((max_entries + 63) & ~(size_t)63));
    int rc = SS_OK;
    uint32_t *stage_all = (uint32_t *)host_staging(sizeof(uint32_t) * tstride * nrt);
    do {
        if (R <= 1) {
            uint32_t base = rbase.empty() ? 0u : rbase[0];
            uint32_t grid = (total + 255) / 256;
            if (grid > 4096) grid = 4096;
            SS_LAUNCH_U("copy_run", st, total, k_copy_run<<<grid, 256, 0, st>>>(run_perm, run_lcp, base, total, perm_out, lcp_out));
            if ((e = cudaGetLastError())) break;
            e = cudaStreamSynchronize(st);
            break;
        }
        // ping-pong so that the last round lands in perm_out / lcp_out
        const uint32_t *src_p = run_perm, *src_l = run_lcp;
        size_t round = 0;
        while (R > 1) {
            round++;
            bool last = round == rounds;
            uint32_t *dst_p = last ? perm_out : ((rounds - round) % 2 ? tmp_perm : perm_out);
            uint32_t *dst_l = last ? lcp_out : ((rounds - round) % 2 ? tmp_lcp : lcp_out);
            // staging: rb[R+1], bases[R] (first round), cbase[pairs], wbase[pairs]
            uint32_t *stage = stage_all + tstride * (round - 1);
            uint32_t *d_rb = d_tables + tstride * (round - 1);
            const uint32_t npairs = (R + 1) / 2;
            memcpy(stage, rb.data(), sizeof(uint32_t) * (R + 1));
            if (round == 1) memcpy(stage + (R + 1), rbase.data(), sizeof(uint32_t) * R);
            uint32_t *cb = stage + (2 * R + 1);
            uint32_t *wb = cb + npairs;
            uint32_t nentries = 0, nwin = 0;
            for (uint32_t p = 0; p < npairs; p++) {
                uint32_t len = rb[std::min(2 * p + 2, R)] - rb[2 * p];
                cb[p] = nentries;
                nentries += (len + kCoarse - 1) / kCoarse + 1;
                wb[p] = nwin;
                nwin += (len + kMergeTile - 1) / kMergeTile;
            }
            size_t cp = sizeof(uint32_t) * (2 * R + 1 + 2 * npairs);
            if ((e = cudaMemcpyAsync(d_rb, stage, cp, cudaMemcpyHostToDevice, st))) break;
            const uint32_t *bases = round == 1 ? d_rb + (R + 1) : nullptr;
            const uint32_t *d_cb = d_rb + (2 * R + 1);
            const uint32_t *d_wb = d_cb + npairs;
            // round 1 reads the runs' caches when the caller has them (a sort
            // wrote them), else computes them
            const bool given = round == 1 && cache.ck;
            const uint64_t *src_o = given ? cache.off : off_buf[(round - 1) & 1];
            uint64_t *dst_o = last ? nullptr : off_buf[round & 1];
            const uint64_t *src_ck = given ? cache.ck : ck_buf[(round - 1) & 1];
            const uint32_t *src_ckd = given ? cache.ckd : ckd_buf[(round - 1) & 1];
            uint64_t *dst_ck = last ? nullptr : ck_buf[round & 1];
            uint32_t *dst_ckd = last ? nullptr : ckd_buf[round & 1];
            if (round == 1 && !given) {
                uint32_t grid = std::min<uint32_t>((total + 255) / 256, 8192);
                SS_LAUNCH_U("run_prep", st, total, k_run_prep<<<grid, 256, 0, st>>>(
                    set, src_p, src_l, d_rb, R, bases, total, 1, off_buf[0], ck_buf[0], ckd_buf[0]));
            }
            SS_LAUNCH_U("merge_cuts", st, nentries, k_merge_cuts<<<(nentries * kCutLanes + 127) / 128, 128, 0, st>>>(
                set, src_p, src_l, src_o, d_rb, R, bases, d_cb, npairs, nentries, d_coarse));
            SS_LAUNCH_U("merge_windows", st, nentries, k_merge_windows<<<(nentries + 127) / 128, 128, 0, st>>>(
                set, src_p, src_l, src_o, d_rb, R, bases, d_cb, npairs, nentries, d_coarse));
            SS_LAUNCH_U("merge_starts", st, total, k_merge_starts<<<nwin, kMergeTileThreads, 0, st>>>(
                set, src_p, src_l, d_rb, R, bases, d_wb, npairs, d_coarse, d_cb, src_o, d_starts));
            SS_LAUNCH_U("merge_round", st, total, k_merge_tile<<<nwin, kMergeTileThreads, sizeof(MergeTileSmem), st>>>(
                set, src_p, src_l, d_rb, R, bases, d_wb, npairs, dst_p, dst_l, d_coarse, d_cb, d_starts, src_o, dst_o,
                src_ck, src_ckd, dst_ck, dst_ckd));
            if ((e = cudaGetLastError())) break;
            std::vector<uint32_t> nrb{0};
            for (uint32_t k = 2; k <= R; k += 2) nrb.push_back(rb[k]);
            if (R % 2) nrb.push_back(rb[R]);
            rb = nrb;
            R = (uint32_t)rb.size() - 1;
            src_p = dst_p;
            src_l = dst_l;
        }
        if (!e) e = cudaStreamSynchronize(st);
    } while (0);
    if (e) rc = cuda_fail(e, "ss_merge");
    scratch_free(block, st);
    return rc;
}

}  // namespace ss

// ---------------------------------------------------------------------------
// ss_merge_noalloc: the same merge without any allocation.
//
// Some callers cannot let a library allocate: a serving process whose device
// memory is reserved up front by its own arena, code with a hard device-memory
// budget, or a latency-critical path that must not pay for (or synchronize
// on) cudaMalloc/cudaFree or pinned host allocations.  This entry point keeps
// its temporary arrays in one fixed array of device memory that is part of
// the library image: every GPU that loads the library holds these
// kNoAllocBytes until the process exits.  The run table of each round is
// passed to the device by value and stored in the same array by a one-thread
// kernel, so no host staging buffer is needed either.
//
// The array is shared by every call on a device and keeps whatever the last
// call left in it; nothing here relies on its contents at entry (every word
// is written before it is read within a call).  Calls that overlap on the GPU
// (different streams, or different host threads, without ordering between
// them) race on the array and give wrong results: order them on one stream.
namespace ss {

constexpr uint32_t kNoAllocMaxStrings = 1u << 20;   // 1,048,576 strings in total
constexpr uint32_t kNoAllocMaxRuns = 64;
constexpr uint32_t kNoAllocTableWords = 2 * (kNoAllocMaxRuns + 1);
constexpr size_t kNoAllocWords = 2ull * kNoAllocMaxStrings + kNoAllocTableWords;

static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

struct RunTable {
    uint32_t rb[kNoAllocMaxRuns + 1];
    uint32_t base[kNoAllocMaxRuns];
};

// writes one round's run starts and index bases into the fixed array
__global__ void k_store_run_table(RunTable t, uint32_t R, uint32_t *dst) {
    for (uint32_t k = threadIdx.x; k <= R; k += blockDim.x) dst[k] = t.rb[k];
    for (uint32_t k = threadIdx.x; k < R; k += blockDim.x) dst[kNoAllocMaxRuns + 1 + k] = t.base[k];
}

// Device address of g_noalloc_scratch on the current device.  In host code the
// symbol name is only a host-side stand-in, so the address is asked for with
// the device current, on every call: the lookup allocates nothing, and an
// address cached across calls could go stale after cudaDeviceReset or a
// re-created primary context (the module is loaded again, possibly elsewhere).
// The first call on a device may load the library's module there, so that
// first call should come before any stream capture.
static cudaError_t noalloc_setup(uint32_t **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = (uint32_t *)p;
    return cudaSuccess;
}

static int merge_runs_noalloc(const ReqDesc &set, const uint32_t *run_perm, const uint32_t *run_lcp,
                              const uint32_t *run_begin_host, const uint32_t *run_base_host, uint32_t K,
                              uint32_t *perm_out, uint32_t *lcp_out, cudaStream_t st) {
    uint32_t total = run_begin_host[K];
    uint32_t *scratch = nullptr;
    cudaError_t e = noalloc_setup(&scratch);
    if (e != cudaSuccess) return cuda_fail(e, "ss_merge_noalloc: symbol address of the fixed scratch array");
    uint32_t *tmp_perm = scratch;
    uint32_t *tmp_lcp = scratch + kNoAllocMaxStrings;
    uint32_t *d_table = scratch + 2ull * kNoAllocMaxStrings;
    RunTable t;
    memset(&t, 0, sizeof(t));
    uint32_t R = 0;
    t.rb[0] = 0;
    for (uint32_t k = 0; k < K; k++)
        if (run_begin_host[k + 1] > run_begin_host[k]) {
            t.base[R] = run_base_host ? run_base_host[k] : 0u;
            t.rb[++R] = run_begin_host[k + 1];
        }
    if (R <= 1) {
        uint32_t base = R ? t.base[0] : 0u;
        uint32_t grid = (total + 255) / 256;
        if (grid > 4096) grid = 4096;
        SS_LAUNCH_U("copy_run", st, total, k_copy_run<<<grid, 256, 0, st>>>(run_perm, run_lcp, base, total, perm_out, lcp_out));
        e = cudaGetLastError();
        return e ? cuda_fail(e, "ss_merge_noalloc") : SS_OK;
    }
    size_t rounds = 0;
    for (uint32_t r = R; r > 1; r = (r + 1) / 2) rounds++;
    const uint32_t *src_p = run_perm, *src_l = run_lcp;
    size_t round = 0;
    while (R > 1) {
        round++;
        bool last = round == rounds;
        uint32_t *dst_p = last ? perm_out : ((rounds - round) % 2 ? tmp_perm : perm_out);
        uint32_t *dst_l = last ? lcp_out : ((rounds - round) % 2 ? tmp_lcp : lcp_out);
        if (round > 1) memset(t.base, 0, sizeof(t.base));   // later rounds hold set indices
        SS_LAUNCH("store_run_table", st, k_store_run_table<<<1, 128, 0, st>>>(t, R, d_table));
        uint32_t threads = (total + kMergeItems - 1) / kMergeItems;
        SS_LAUNCH_U("merge_round", st, total, k_merge_round<<<(threads + 255) / 256, 256, 0, st>>>(
            set, src_p, src_l, d_table, R, d_table + kNoAllocMaxRuns + 1, total, dst_p, dst_l, nullptr, nullptr,
            nullptr, nullptr, nullptr, nullptr, nullptr, nullptr));
        if ((e = cudaGetLastError())) return cuda_fail(e, "ss_merge_noalloc");
        RunTable nt;
        memset(&nt, 0, sizeof(nt));
        uint32_t nR = 0;
        for (uint32_t k = 2; k <= R; k += 2) nt.rb[++nR] = t.rb[k];
        if (R % 2) nt.rb[++nR] = t.rb[R];
        t = nt;
        R = nR;
        src_p = dst_p;
        src_l = dst_l;
    }
    return SS_OK;
}

}  // namespace ss

extern "C" int ss_merge_noalloc(const uint8_t *chars, const uint64_t *offsets, const uint32_t *lengths,
                                uint32_t fixed_len, const uint32_t *run_perm, const uint32_t *run_lcp,
                                const uint32_t *run_begin_host, const uint32_t *run_base_host, uint32_t K,
                                uint32_t *perm_out, uint32_t *lcp_out, ss_stream_t stream) {
    using namespace ss;
    set_error_detail("%s", "");
    if (K == 0 || !run_begin_host || run_begin_host[0] != 0) {
        set_error_detail("ss_merge_noalloc: K must be >= 1 with run_begin_host[K+1], run_begin_host[0] = 0");
        return SS_ERR_INVALID;
    }
    if (K > kNoAllocMaxRuns) {
        set_error_detail("ss_merge_noalloc: K = %u runs is beyond the fixed limit of %u runs", K, kNoAllocMaxRuns);
        return SS_ERR_TOO_LARGE;
    }
    for (uint32_t k = 0; k < K; k++)
        if (run_begin_host[k + 1] < run_begin_host[k]) {
            set_error_detail("ss_merge_noalloc: run_begin_host must be non-decreasing");
            return SS_ERR_INVALID;
        }
    uint32_t total = run_begin_host[K];
    if (total > kNoAllocMaxStrings) {
        set_error_detail("ss_merge_noalloc: %u strings is beyond the fixed scratch limit of %u strings "
                         "(use ss_merge for larger merges)", total, kNoAllocMaxStrings);
        return SS_ERR_TOO_LARGE;
    }
    if (total == 0) return SS_OK;
    if (!chars || !offsets || !run_perm || !run_lcp || !perm_out || !lcp_out) {
        set_error_detail("ss_merge_noalloc: NULL pointer");
        return SS_ERR_INVALID;
    }
    ReqDesc set;
    memset(&set, 0, sizeof(set));
    set.chars = chars;
    set.offsets = offsets;
    set.lengths = lengths;
    set.fixed_len = lengths ? 0 : fixed_len;
    return merge_runs_noalloc(set, run_perm, run_lcp, run_begin_host, run_base_host, K, perm_out, lcp_out,
                              reinterpret_cast<cudaStream_t>(stream));
}
