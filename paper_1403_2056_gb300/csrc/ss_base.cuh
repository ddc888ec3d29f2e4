// Base case of the recursion: segments of at most kSmallMax strings that
// share their first `depth` characters are sorted completely inside one CTA
// (or one warp), and their LCPs are written (the role LCP insertion sort,
// Algorithm 5, plays in the paper's pS5).
//
// A segment is sorted by its 8-character keys once: by one counting pass on
// a digit of the keys when no digit gets more than a few strings (then
// insertion sort inside each digit), else with a CTA merge sort (8 keys per
// thread sorted in registers, then merge-path passes through padded,
// bank-conflict-free shared memory).  Sorting is skipped when every group's
// keys are already equal.  Neighbours with different keys are split (LCP =
// depth + lcp of the keys); neighbours with equal keys that hold the end of
// the string are equal strings (LCP = their length); runs of equal keys
// without the end form groups that continue 8 characters deeper.  Groups of
// at most 32 strings are finished by the warp class (several groups packed
// into one warp); larger groups are re-sorted by the CTA, compacted, by
// (group, next key, position).  Equal strings keep their input order (input
// order inside a segment is index order).  An LCP belongs to a position:
// once two neighbouring positions are split, every later re-sort stays on one
// side of that boundary.  With sort caches requested, each position's 8
// characters are written where its LCP is decided and its string offset where
// its permutation entry is.
#pragma once

#include "ss_internal.cuh"

// (no namespace of its own: included by ss_kernels.cuh inside the includer's)

// ----------------------------------------------------------- warp finish
struct WElem {
    uint32_t g;    // group id: first lane of its group (0xFFFFFFFF: padding)
    uint32_t i;    // string index
    uint64_t o;    // byte offset of the string
    uint64_t k0;   // characters [depth, depth + 8)
    uint64_t k1;   // characters [depth + 8, depth + 16)
};

__device__ __forceinline__ bool welem_less(const WElem &a, const WElem &b) {
    if (a.g != b.g) return a.g < b.g;
    if (a.k0 != b.k0) return a.k0 < b.k0;
    if (a.k1 != b.k1) return a.k1 < b.k1;
    return a.i < b.i;   // inside a segment input order equals index order
}

__device__ __forceinline__ WElem shfl_xor_welem(const WElem &e, int m) {
    WElem r;
    r.g = __shfl_xor_sync(0xffffffffu, e.g, m);
    r.i = __shfl_xor_sync(0xffffffffu, e.i, m);
    r.o = __shfl_xor_sync(0xffffffffu, e.o, m);
    r.k0 = __shfl_xor_sync(0xffffffffu, e.k0, m);
    r.k1 = __shfl_xor_sync(0xffffffffu, e.k1, m);
    return r;
}

// Sort groups of at most W strings completely, W in {4, 8, 16, 32}: the warp
// holds 32 / W groups side by side, group s on lanes sW .. sW + W - 1, and
// sorts them all at once, 16 characters per round (a group of a few strings
// whose duplicates need many rounds no longer holds a whole warp).  Lane l
// with l % W < m holds string index `id` (string offset `off`) and its 16
// characters at `depth`; m, depth, out and R are its group's.  mmax, the
// largest m of the warp, bounds the sorting network (all lanes call this).
// Writes perm and lcp of R-local positions out .. out + m - 1 (not the lcp of
// position `out`, which the caller owns).
template <bool A>
__device__ __forceinline__ void warp_finish(const ReqDesc &R, uint32_t W, uint32_t m, uint32_t mmax, uint32_t depth,
                                            uint32_t id, uint64_t off, uint64_t k0, uint64_t k1, uint32_t out) {
    const uint32_t lane = threadIdx.x & 31, ls = lane & (W - 1);
    const uint32_t kc = key_chars(R);   // characters per key
    WElem e;
    if (ls < m) { e.g = 0; e.i = id; e.o = off; e.k0 = k0; e.k1 = k1; }
    else { e.g = 0xFFFFFFFFu; e.i = 0xFFFFFFFFu; e.o = 0; e.k0 = ~0ull; e.k1 = ~0ull; }
    uint32_t lcp = 0, ckd = 0;
    uint64_t ck = 0;   // the key the LCP was decided in, and its depth
    for (;;) {
        // bitonic network inside each group's lanes (xor partners below W stay
        // in the group); after the stage of size k >= mmax the first k lanes of
        // every group are ascending and hold all its strings
        for (uint32_t k = 2; k <= W; k <<= 1) {
            if ((k >> 1) >= mmax && k > 2) break;   // lanes >= m hold padding only
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                WElem o = shfl_xor_welem(e, (int)j);
                bool up = (ls & k) == 0;
                bool lower = (ls & j) == 0;
                bool take_o = lower == up ? welem_less(o, e) : welem_less(e, o);
                if (take_o) e = o;
            }
        }
        const int w = (int)W;
        uint32_t pg = __shfl_up_sync(0xffffffffu, e.g, 1, w);
        uint64_t p0 = __shfl_up_sync(0xffffffffu, e.k0, 1, w);
        uint64_t p1 = __shfl_up_sync(0xffffffffu, e.k1, 1, w);
        bool start = true;
        if (ls > 0 && ls < m && pg == e.g) {
            if (p0 != e.k0) { lcp = depth + key_lcp<A>(R, p0, e.k0); ck = e.k0; ckd = depth; }
            else if (key_ends<A>(R, e.k0, depth)) { lcp = depth + key_len<A>(R, e.k0, depth); ck = e.k0; ckd = depth; }
            else if (p1 != e.k1) { lcp = depth + kc + key_lcp<A>(R, p1, e.k1); ck = e.k1; ckd = depth + kc; }
            else if (key_ends<A>(R, e.k1, depth + kc)) {
                lcp = depth + kc + key_len<A>(R, e.k1, depth + kc);
                ck = e.k1;
                ckd = depth + kc;
            } else {
                start = false;
            }
        }
        if (ls >= m) start = true;
        uint32_t sg = start ? ls : 0;
        for (uint32_t o = 1; o < W; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, sg, o, w);
            if (ls >= o) sg = max(sg, y);
        }
        bool next_start = __shfl_down_sync(0xffffffffu, start, 1, w) || ls == W - 1;
        bool active = ls < m && !(start && next_start);
        if (ls < m) e.g = sg;
        if (!__any_sync(0xffffffffu, active)) break;
        depth += 2 * kc;
        if (active) key2_at<A>(R, e.i, e.o, depth, e.k0, e.k1);
    }
    if (ls < m) {
        R.perm_out[out + ls] = e.i;
        put_off(R, out + ls, e.o);
        if (ls > 0) {
            R.lcp_out[out + ls] = lcp;
            put_ck(R, out + ls, ck, ckd);
        }
    }
}

// Tiny base cases (2..32 strings).  The task count is read on the device: the
// CTA base cases below append groups to the same list.  A warp takes the tasks
// in slots of 8: the largest of a slot sets the lanes per group W (4, 8, 16 or
// 32), and the slot's tasks go through the warp 32 / W at a time.
template <bool A>
__global__ void __launch_bounds__(kThreads) k_small_warp(const SmallTask *tasks, const uint32_t *ntask_dev,
                                                         const ReqDesc *reqs, ElemBufs eb) {
    constexpr uint32_t kSlot = 8;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t ntask = *ntask_dev;
    for (uint32_t t0 = gw * kSlot; t0 < ntask; t0 += nw * kSlot) {
        const uint32_t nt = min(kSlot, ntask - t0);
        const uint32_t smax = __reduce_max_sync(0xffffffffu, lane < nt ? tasks[t0 + lane].size : 0u);
        const uint32_t W = smax <= 4 ? 4u : smax <= 8 ? 8u : smax <= 16 ? 16u : 32u;
        for (uint32_t b = 0; b < nt; b += 32 / W) {
            const uint32_t q = b + lane / W, ls = lane & (W - 1);
            SmallTask t{0u, 0u, 0u, 0u, 0u, 0u};
            if (q < nt) t = tasks[t0 + q];
            const uint32_t mmax = __reduce_max_sync(0xffffffffu, t.size);
            const uint32_t *idx = eb.idx[t.parity];
            const uint64_t *soff = eb.soff[t.parity];
            const uint64_t *key = eb.key[t.parity];
            const ReqDesc &R = reqs[t.req];
            uint32_t id = 0;
            uint64_t off = 0, k0 = 0, k1 = 0;
            if (ls < t.size) {
                id = idx[t.begin + ls];
                off = soff[t.begin + ls];
                if (t.gather) {
                    key2_at<A>(R, id, off, t.depth, k0, k1);
                } else {
                    k0 = key[t.begin + ls];
                    k1 = key_ends<A>(R, k0, t.depth) ? 0ull : key_at<A>(R, id, off, t.depth + key_chars(R));
                }
            }
            warp_finish<A>(R, W, t.size, mmax, t.depth, id, off, k0, k1, t.begin - R.base);
        }
    }
}

// -------------------------------------------------------- CTA merge sort
// element: 64-bit key k and g = group << 12 | original index (both < 4096);
// order (group, key, original index); padding g = 0xFFFFFFFF sorts last

__device__ __forceinline__ bool gk_less(uint64_t ka, uint32_t ga, uint64_t kb, uint32_t gb) {
    uint32_t xa = ga >> 12, xb = gb >> 12;
    if (xa != xb) return xa < xb;
    if (ka != kb) return ka < kb;
    return (ga & 0xFFFu) < (gb & 0xFFFu);
}

// Shared-memory slot index with one pad word per 8 slots: thread t's blocked
// slots t*8 .. t*8+7 then fall in distinct banks across a warp (9t + j is a
// bijection mod 32), so the blocked stores and loads below are conflict-free.
__device__ __forceinline__ uint32_t padx(uint32_t x) { return x + (x >> 3); }

// The order of the sort: (group, key, original index), or the key alone when
// every slot is in one group and the slots start in original-index order (the
// first sort of a segment): the sort below is stable, so equal keys keep that
// order and the result is the same.  The key-only order needs no group word in
// the comparisons.
template <bool KEYONLY>
__device__ __forceinline__ bool sort_less(uint64_t ka, uint32_t ga, uint64_t kb, uint32_t gb) {
    return KEYONLY ? ka < kb : gk_less(ka, ga, kb, gb);
}

template <int ITEMS, bool KEYONLY>
__device__ __forceinline__ void reg_sort(uint64_t (&k)[ITEMS], uint32_t (&g)[ITEMS]) {
    // odd-even transposition network, fully unrolled; it swaps only strictly
    // smaller neighbours forward, so it is stable
#pragma unroll
    for (int r = 0; r < ITEMS; r++) {
#pragma unroll
        for (int j = r & 1; j + 1 < ITEMS; j += 2) {
            if (sort_less<KEYONLY>(k[j + 1], g[j + 1], k[j], g[j])) {
                uint64_t tk = k[j]; k[j] = k[j + 1]; k[j + 1] = tk;
                uint32_t tg = g[j]; g[j] = g[j + 1]; g[j + 1] = tg;
            }
        }
    }
}

// Sort the P (power of two, >= ITEMS) slots held blocked in registers
// (thread t holds slots t*ITEMS ..) through the padded shared buffers MK / MG
// (sized for padx(P)).  On return each thread holds its ITEMS slots of the
// sorted sequence.
template <int NT, int ITEMS, bool KEYONLY>
__device__ __forceinline__ void block_merge_sort(uint64_t (&k)[ITEMS], uint32_t (&g)[ITEMS], uint32_t P, uint64_t *MK,
                                                 uint32_t *MG) {
    reg_sort<ITEMS, KEYONLY>(k, g);
    const uint32_t o = threadIdx.x * ITEMS;
    for (uint32_t L = ITEMS; L < P; L <<= 1) {
        if (o < P) {
#pragma unroll
            for (int j = 0; j < ITEMS; j++) { MK[padx(o + j)] = k[j]; MG[padx(o + j)] = g[j]; }
        }
        __syncthreads();
        if (o < P) {
            const uint32_t base = o & ~(2 * L - 1), d = o - base;
            const uint32_t a = base, b = base + L;
            uint32_t lo = d > L ? d - L : 0, hi = d < L ? d : L;
            while (lo < hi) {   // merge path: A[mid] goes first unless B[d-1-mid] < A[mid]
                uint32_t mid = (lo + hi) >> 1;
                uint32_t bi = padx(b + d - 1 - mid), ai = padx(a + mid);
                if (!sort_less<KEYONLY>(MK[bi], KEYONLY ? 0u : MG[bi], MK[ai], KEYONLY ? 0u : MG[ai])) lo = mid + 1;
                else hi = mid;
            }
            uint32_t i = lo, jj = d - lo;
            uint64_t ka = i < L ? MK[padx(a + i)] : 0, kb = jj < L ? MK[padx(b + jj)] : 0;
            uint32_t ga = i < L ? MG[padx(a + i)] : 0, gb = jj < L ? MG[padx(b + jj)] : 0;
#pragma unroll
            for (int q = 0; q < ITEMS; q++) {
                bool takeA = jj >= L || (i < L && !sort_less<KEYONLY>(kb, gb, ka, ga));
                if (takeA) {
                    k[q] = ka; g[q] = ga; i++;
                    if (i < L) { ka = MK[padx(a + i)]; ga = MG[padx(a + i)]; }
                } else {
                    k[q] = kb; g[q] = gb; jj++;
                    if (jj < L) { kb = MK[padx(b + jj)]; gb = MG[padx(b + jj)]; }
                }
            }
        }
        __syncthreads();
    }
}

// block-wide scan over slots [0, M) of v (blocked, ITEMS per thread):
// MAXSCAN: inclusive max; else exclusive sum (returns the total)
template <int NT, int ITEMS, bool MAXSCAN>
__device__ __forceinline__ uint32_t block_scan(uint32_t *v, uint32_t M, uint32_t *wsum) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = NT / 32;
    const uint32_t base = threadIdx.x * ITEMS;
    uint32_t loc[ITEMS];
    uint32_t run = 0;
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        uint32_t x = (base + j < M) ? v[base + j] : 0;
        if (MAXSCAN) { run = max(run, x); loc[j] = run; }
        else { loc[j] = run; run += x; }
    }
    uint32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl = MAXSCAN ? max(incl, y) : incl + y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t prev = 0, total = 0;
#pragma unroll
    for (int w = 0; w < NW; w++) {
        uint32_t x = wsum[w];
        if (w < (int)warp) prev = MAXSCAN ? max(prev, x) : prev + x;
        total = MAXSCAN ? max(total, x) : total + x;
    }
    uint32_t ex = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) ex = MAXSCAN ? 0u : 0u;
    ex = MAXSCAN ? max(ex, prev) : ex + prev;
#pragma unroll
    for (int j = 0; j < ITEMS; j++)
        if (base + j < M) v[base + j] = MAXSCAN ? max(loc[j], ex) : loc[j] + ex;
    __syncthreads();
    return total;
}

template <int NT, int ITEMS>
struct BaseSmem {
    static constexpr uint32_t CAP = NT * ITEMS;
    uint64_t SK[CAP + CAP / 8];   // key at the current depth by position; padded merge buffer while sorting
    uint32_t MG[CAP + CAP / 8];   // padded merge buffer; scan buffer between sorts
    uint32_t SI[CAP];        // string index by original index
    uint16_t SP[CAP];        // original index at each position
    uint16_t SG[CAP];        // first position of the group of each position
    uint16_t GS[CAP];        // size of the group that starts at a position
    uint16_t ACT[CAP];       // positions still being sorted, in order
    uint32_t WL[CAP / 2];    // groups of 2..32 strings for the warps: start << 16 | size
    uint64_t wlast[NT / 32]; // last key of each warp's slots (first round's neighbour test)
    uint64_t wmin[NT / 32], wmax[NT / 32];   // smallest and largest key of each warp's slots
    uint32_t wsum[NT / 32];
    uint32_t nwl, nws, wbase;   // small groups, their strings, first reserved list slot
    uint32_t sigma;          // first round: distinct bytes after the keys' common prefix
    uint32_t task, next;     // task taken from the queue, and the one after it
};

// First round by one counting pass (the adaptivity of Section 8.1: when the
// keys of a segment are spread, distribute by a digit as radix sort does).
// The digit has 2^B >= m values and is monotone in the key: the key's place
// in the segment's key range [kmin, kmax] (fixed point, below), or for keys
// of a small alphabet the ranks of its bytes (below).  Keys spread evenly over
// their range (a bucket between two splitters) fill the interpolation digits
// evenly wherever the range lies, where the bits after the keys' common prefix
// would leave most digits empty when the range straddles a power of two.
// One shared-memory histogram, scan and placement put the segment in
// digit order; each digit's strings (at most kRadixBucketMax, otherwise the
// merge sort below is used instead) are then put in (key, original index)
// order by insertion sort.  kin holds the keys of this thread's slots
// tid + r NT (SK holds all of them by position).  On success SK / SP hold the
// segment sorted by (key, original index) by position and true is returned;
// false leaves SK untouched and SP unset (all keys equal, or a digit too
// full).  Every thread of the CTA calls this.
constexpr uint32_t kRadixBucketMax = 8;
// 1: the rank digit for keys of a small alphabet, the interpolation digit
// otherwise; 0: keys of a small alphabet go to the merge sort; 2: always the
// rank digit
#ifndef SS_RADIX_RANK
#define SS_RADIX_RANK 1
#endif

template <int NT, int ITEMS>
__device__ __forceinline__ bool radix_first_round(BaseSmem<NT, ITEMS> &S, uint32_t m, const uint64_t (&kin)[ITEMS]) {
    constexpr int NW = NT / 32;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t k0 = S.SK[0];
    uint64_t k[ITEMS];
    uint64_t x = 0, kmn = ~0ull, kmx = 0;
#pragma unroll
    for (int r = 0; r < ITEMS; r++) {
        const uint32_t i = tid + r * NT;
        k[r] = i < m ? kin[r] : k0;
        x |= k[r] ^ k0;
        kmn = min(kmn, k[r]);
        kmx = max(kmx, k[r]);
    }
    const uint32_t xl = __reduce_or_sync(0xffffffffu, (uint32_t)x);
    const uint32_t xh = __reduce_or_sync(0xffffffffu, (uint32_t)(x >> 32));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kmn = min(kmn, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)kmn, o));
        kmx = max(kmx, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)kmx, o));
    }
    if (lane == 0) {
        S.wlast[warp] = ((uint64_t)xh << 32) | xl;
        S.wmin[warp] = kmn;
        S.wmax[warp] = kmx;
    }
    __syncthreads();
    x = 0;
#pragma unroll
    for (int w = 0; w < NW; w++) {
        x |= S.wlast[w];
        kmn = min(kmn, S.wmin[w]);
        kmx = max(kmx, S.wmax[w]);
    }
    if (x == 0) return false;   // every key equal: nothing to distribute
    const uint32_t cp = (uint32_t)__clzll((long long)x);
    uint32_t B = 1;
    while ((1u << B) < m) B++;
    const uint32_t nb = 1u << B;   // <= NT * ITEMS
    // Keys whose B bits after the common prefix nearly all vary get the
    // interpolation digit.  Keys of a small alphabet (some bits of every byte
    // fixed) would fill that digit space unevenly; they get a rank digit: each
    // byte from the first differing one on is replaced by its rank among the
    // byte values the segment's keys use there (b = ceil(log2 sigma) bits for
    // sigma values), and the ranks, concatenated, give the top B bits.  Ranks
    // keep the byte order, so the digit is monotone in the key.
    uint32_t d[ITEMS];
    const bool dense = (uint32_t)__popcll((x << cp) >> (64 - B)) + 1 >= B;
    if (dense && SS_RADIX_RANK != 2) {
        // the range normalised: span << L in [2^63, 2^64), sh its top 32 bits;
        // M = 2^44 / (sh + 1) * (1 - 2^-20 + 2^-22) at most (the float quotient
        // is within 2^-23 of the exact one), so ((t >> 32) * M) < 2^44 for
        // every t = (key - kmin) << L <= span << L, and M >= 4094 keeps the
        // digits even to 1 part in 4096
        const uint64_t span = kmx - kmn;   // > 0: the keys are not all equal
        const uint32_t L = (uint32_t)__clzll((long long)span);
        const uint32_t sh = (uint32_t)((span << L) >> 32);
        const uint32_t M = (uint32_t)__float2uint_rz(17592186044416.0f / (__uint2float_rn(sh) + 1.0f) *
                                                     (1.0f - 1.0f / 1048576.0f));
#pragma unroll
        for (int r = 0; r < ITEMS; r++) d[r] = (uint32_t)(((uint64_t)(uint32_t)(((k[r] - kmn) << L) >> 32) * M) >> (44 - B));
    } else {
        const uint32_t c0 = cp >> 3;   // bytes before c0 are the same in every key
        // an alphabet of at most 16 byte values varies in at most 4 bits of a
        // byte (e.g. A C G T: 4); text varies in more, and its first round is
        // left to the merge sort
        if (SS_RADIX_RANK == 0 || (SS_RADIX_RANK == 1 && (uint32_t)__popcll((long long)x) > 4 * (8 - c0) + 1))
            return false;
        uint16_t *rank = S.GS;   // free until the group rounds
        for (uint32_t v = tid; v < 256; v += NT) rank[v] = 0;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < ITEMS; r++)
            if (tid + r * NT < m)
                for (uint32_t j = c0; j < 8; j++) rank[(uint32_t)(k[r] >> (56 - 8 * j)) & 0xFFu] = 1;
        __syncthreads();
        if (warp == 0) {   // rank of a byte value: the used values below it
            uint32_t f[8], c = 0;
#pragma unroll
            for (int t = 0; t < 8; t++) { f[t] = rank[8 * lane + t]; c += f[t]; }
            uint32_t incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= (uint32_t)o) incl += y;
            }
            uint32_t base = incl - c;
#pragma unroll
            for (int t = 0; t < 8; t++) { rank[8 * lane + t] = (uint16_t)base; base += f[t]; }
            if (lane == 31) S.sigma = incl;
        }
        __syncthreads();
        uint32_t bw = 1;   // bits per rank; sigma >= 2 (the keys differ in byte c0)
        while ((1u << bw) < S.sigma) bw++;
#pragma unroll
        for (int r = 0; r < ITEMS; r++) {
            uint32_t dd = 0, nbits = 0;
            for (uint32_t j = c0; j < 8 && nbits < B; j++) {
                dd = (dd << bw) | rank[(uint32_t)(k[r] >> (56 - 8 * j)) & 0xFFu];
                nbits += bw;
            }
            d[r] = nbits >= B ? dd >> (nbits - B) : dd << (B - nbits);
        }
    }
    uint32_t *C = S.MG;
    for (uint32_t b = tid; b < nb; b += NT) C[b] = 0;
    __syncthreads();
    uint32_t rk[ITEMS];
#pragma unroll
    for (int r = 0; r < ITEMS; r++) {
        const uint32_t i = tid + r * NT;
        rk[r] = i < m ? atomicAdd(&C[d[r]], 1u) : 0u;
    }
    __syncthreads();
    bool full = false;
    for (uint32_t b = tid; b < nb; b += NT) full = full || C[b] > kRadixBucketMax;
    if (__syncthreads_or(full)) return false;
    block_scan<NT, ITEMS, false>(C, nb, S.wsum);
#pragma unroll
    for (int r = 0; r < ITEMS; r++) {
        const uint32_t i = tid + r * NT;
        if (i < m) {
            const uint32_t pos = C[d[r]] + rk[r];
            S.SK[pos] = k[r];
            S.SP[pos] = (uint16_t)i;
        }
    }
    __syncthreads();
    for (uint32_t b = tid; b < nb; b += NT) {
        const uint32_t st = C[b], en = b + 1 < nb ? C[b + 1] : m;
        for (uint32_t a = st + 1; a < en; a++) {
            const uint64_t kk = S.SK[a];
            const uint16_t pp = S.SP[a];
            uint32_t z = a;
            while (z > st && (S.SK[z - 1] > kk || (S.SK[z - 1] == kk && S.SP[z - 1] > pp))) {
                S.SK[z] = S.SK[z - 1];
                S.SP[z] = S.SP[z - 1];
                z--;
            }
            S.SK[z] = kk;
            S.SP[z] = pp;
        }
    }
    __syncthreads();
    return true;
}

// Small groups are handed to the warp kernel through the other parity's
// buffers: base cases run after the last level, so those positions of the
// task are free, and no other task reads them.
//
// Tasks come from a device work queue: each CTA takes the next task of its
// class list with one atomic on the queue head (`next_task`), so the grid is
// sized to the CTAs that fit on the device at once and segments of uneven
// size balance themselves.  The task count is read on the device.
//
// First round: the segment is sorted by its keys at the task's depth.  When
// every pair of neighbours is then decided (different keys, or equal keys
// that hold the end of the string), the sorted keys still in registers give
// every LCP and the task ends there; only segments with equal keys that
// continue past these 8 characters go through the group rounds below.
// CTAs per SM the register budget must allow: as many as the shared memory
// (228 KB per SM, 1 KB of it reserved per CTA) and the 2048 threads of an SM
// let in, but no fewer than 64 registers per thread
constexpr int base_min_ctas(int nt, size_t smem) {
    const int by_smem = (int)(233472 / (smem + 1024)), by_threads = 2048 / nt, by_regs = 65536 / (64 * nt);
    const int m = by_smem < by_threads ? by_smem : by_threads;
    return m < by_regs ? (m > 0 ? m : 1) : by_regs;
}

template <int NT, int ITEMS, bool A>
__global__ void __launch_bounds__(NT, base_min_ctas(NT, sizeof(BaseSmem<NT, ITEMS>))) k_base_cta(const SmallTask *tasks, const uint32_t *ntask_dev, uint32_t *next_task,
                                                 const ReqDesc *reqs, ElemBufs eb, SmallTask *tiny, uint32_t tiny_cap,
                                                 uint32_t *counters) {
    constexpr uint32_t CAP = NT * ITEMS;
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BaseSmem<NT, ITEMS> &S = *reinterpret_cast<BaseSmem<NT, ITEMS> *>(smem_raw);
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t ntask = *ntask_dev;
    if (tid == 0) S.task = atomicAdd(next_task, 1u);
    __syncthreads();
    for (;;) {
        const uint32_t tk = S.task;
        if (tk >= ntask) break;
        const SmallTask t = tasks[tk];
        const uint32_t *idx = eb.idx[t.parity];
        const uint64_t *soff = eb.soff[t.parity];
        const uint64_t *key = eb.key[t.parity];
        uint32_t *idx_hand = eb.idx[t.parity ^ 1];
        uint64_t *soff_hand = eb.soff[t.parity ^ 1];
        const ReqDesc &R = reqs[t.req];
        const uint32_t m = t.size <= CAP ? t.size : CAP;
        const uint32_t lbase = t.begin - R.base;
        // every load of the segment in flight at once (striped: slot tid + r NT)
        uint64_t kk[ITEMS];
        uint32_t ii[ITEMS];
#pragma unroll
        for (int r = 0; r < ITEMS; r++) {
            const uint32_t i = tid + r * NT;
            kk[r] = i < m ? key[t.begin + i] : 0ull;
            ii[r] = i < m ? idx[t.begin + i] : 0u;
        }
        // the next task is fetched while this one runs
        if (tid == 0) S.next = atomicAdd(next_task, 1u);
#pragma unroll
        for (int r = 0; r < ITEMS; r++) {
            const uint32_t i = tid + r * NT;
            if (i < m) { S.SI[i] = ii[r]; S.SK[i] = kk[r]; }
        }
        if (tid == 0) { S.nwl = 0; S.nws = 0; }
        uint32_t M = m, depth = t.depth;
        bool finished = false;   // the first round decided every neighbour pair
        __syncthreads();
        bool presorted = radix_first_round<NT, ITEMS>(S, m, kk);
        if (presorted) {
            bool open = false;   // some neighbours share all 8 characters and continue
            for (uint32_t s = tid + 1; s < m; s += NT) {
                const uint64_t a = S.SK[s - 1], b = S.SK[s];
                open = open || (a == b && !key_ends<A>(R, b, depth));
            }
            if (!__syncthreads_or(open)) {
                for (uint32_t s = tid; s < m; s += NT) {
                    R.perm_out[lbase + s] = S.SI[S.SP[s]];
                    put_off(R, lbase + s, soff[t.begin + S.SP[s]]);
                    if (s > 0) {
                        const uint64_t a = S.SK[s - 1], b = S.SK[s];
                        R.lcp_out[lbase + s] = a != b ? depth + key_lcp<A>(R, a, b) : depth + key_len<A>(R, b, depth);
                        put_ck(R, lbase + s, b, depth);
                    }
                }
                finished = true;
            }
        }
        if (!finished) {   // state of the group rounds: one group, positions in order
            for (uint32_t i = tid; i < m; i += NT) {
                if (!presorted) S.SP[i] = (uint16_t)i;
                S.SG[i] = 0;
                S.ACT[i] = (uint16_t)i;
            }
            if (tid == 0) S.GS[0] = (uint16_t)min(m, 0xFFFFu);
            __syncthreads();
        }
        while (!finished && M > 0) {
            const uint16_t *act = S.ACT;
            if (!presorted) {
            // load the active slots, sort them by (group, key, original index)
            uint64_t k[ITEMS];
            uint32_t g[ITEMS];
#pragma unroll
            for (int j = 0; j < ITEMS; j++) {
                uint32_t s = tid * ITEMS + j;
                if (s < M) {
                    uint32_t pos = act[s];
                    k[j] = S.SK[pos];
                    g[j] = ((uint32_t)S.SG[pos] << 12) | S.SP[pos];
                } else {
                    k[j] = ~0ull;
                    g[j] = 0xFFFFFFFFu;
                }
            }
            // groups whose keys are all equal need no sort (common when a whole
            // segment shares a long prefix): sort only if some neighbour differs
            bool differ = false;
#pragma unroll
            for (int j = 0; j < ITEMS; j++) {
                uint32_t s = tid * ITEMS + j;
                if (s > 0 && s < M) {
                    uint32_t pos = act[s], prv = act[s - 1];
                    if (S.SG[pos] == S.SG[prv] && S.SK[pos] != S.SK[prv]) differ = true;
                }
            }
            if (__syncthreads_or(differ)) {
                uint32_t P = ITEMS;
                while (P < M) P <<= 1;
                // first round: one group, slots in original order (key-only order)
                if (depth == t.depth) block_merge_sort<NT, ITEMS, true>(k, g, P, S.SK, S.MG);
                else block_merge_sort<NT, ITEMS, false>(k, g, P, S.SK, S.MG);
#pragma unroll
                for (int j = 0; j < ITEMS; j++) {
                    uint32_t s = tid * ITEMS + j;
                    if (s < M) {
                        uint32_t pos = act[s];
                        S.SK[pos] = k[j];
                        S.SP[pos] = (uint16_t)(g[j] & 0xFFFu);
                    }
                }
            }
            __syncthreads();
            if (depth == t.depth) {
                // one group in original-index order: slot s holds position s, and
                // (sorted or all equal) the registers hold the keys in position order
                if (lane == 31) S.wlast[warp] = k[ITEMS - 1];
                __syncthreads();
                uint64_t prev = __shfl_up_sync(0xffffffffu, k[ITEMS - 1], 1);
                if (lane == 0) prev = warp ? S.wlast[warp - 1] : 0ull;
                uint32_t lc[ITEMS];
                bool open = false;   // some neighbours share all 8 characters and continue
#pragma unroll
                for (int j = 0; j < ITEMS; j++) {
                    const uint32_t s = tid * ITEMS + j;
                    const uint64_t a = j ? k[j - 1] : prev, b = k[j];
                    lc[j] = 0;
                    if (s > 0 && s < M) {
                        if (a != b) lc[j] = depth + key_lcp<A>(R, a, b);
                        else if (key_ends<A>(R, b, depth)) lc[j] = depth + key_len<A>(R, b, depth);
                        else open = true;
                    }
                }
                if (!__syncthreads_or(open)) {
#pragma unroll
                    for (int j = 0; j < ITEMS; j++) {
                        const uint32_t s = tid * ITEMS + j;
                        if (s < M) {
                            R.perm_out[lbase + s] = S.SI[g[j] & 0xFFFu];
                            put_off(R, lbase + s, soff[t.begin + (g[j] & 0xFFFu)]);
                            if (s > 0) {
                                R.lcp_out[lbase + s] = lc[j];
                                put_ck(R, lbase + s, k[j], depth);
                            }
                        }
                    }
                    finished = true;
                    break;
                }
            }
            }   // !presorted
            presorted = false;
            // split groups: LCPs at new boundaries, new group starts (as positions, max-scanned)
            for (uint32_t s = tid; s < M; s += NT) {
                uint32_t pos = act[s];
                uint32_t st = 1;
                if (pos != S.SG[pos]) {   // not the first position of its group
                    uint64_t a = S.SK[pos - 1], b = S.SK[pos];
                    if (a != b) R.lcp_out[lbase + pos] = depth + key_lcp<A>(R, a, b);
                    else if (key_ends<A>(R, b, depth)) R.lcp_out[lbase + pos] = depth + key_len<A>(R, b, depth);
                    else st = 0;
                    if (st) put_ck(R, lbase + pos, b, depth);
                }
                S.MG[s] = st ? pos : 0u;
            }
            __syncthreads();
            block_scan<NT, ITEMS, true>(S.MG, M, S.wsum);
            // group sizes at each group's last slot; small groups to the warp list
            for (uint32_t s = tid; s < M; s += NT) {
                uint32_t pos = act[s];
                uint32_t ng = S.MG[s];
                bool last = (s + 1 == M) || S.MG[s + 1] != ng;
                S.SG[pos] = (uint16_t)ng;
                if (last) {
                    uint32_t size = pos - ng + 1;
                    S.GS[ng] = (uint16_t)size;
                    if (size >= 2 && size <= 32) {
                        uint32_t w = atomicAdd(&S.nwl, 1u);
                        atomicAdd(&S.nws, size);
                        S.WL[w] = (ng << 16) | size;
                    }
                }
            }
            __syncthreads();
            // positions in groups of more than 32 stay; they read the key 8 characters
            // deeper.  The list of positions is compacted in place: every thread
            // holds its slots in registers before any slot is overwritten.
            uint32_t spos[ITEMS];
            bool stays[ITEMS];
#pragma unroll
            for (int j = 0; j < ITEMS; j++) {
                uint32_t s = tid * ITEMS + j;
                stays[j] = false;
                spos[j] = 0;
                if (s < M) {
                    spos[j] = act[s];
                    stays[j] = S.GS[S.SG[spos[j]]] > 32;
                    S.MG[s] = stays[j] ? 1u : 0u;
                }
            }
            __syncthreads();
            uint32_t M2 = block_scan<NT, ITEMS, false>(S.MG, M, S.wsum);
#pragma unroll
            for (int j = 0; j < ITEMS; j++) {
                uint32_t s = tid * ITEMS + j;
                if (s < M && stays[j]) {
                    uint32_t pos = spos[j];
                    S.ACT[S.MG[s]] = (uint16_t)pos;
                    uint32_t orig = S.SP[pos];
                    S.SK[pos] = key_at<A>(R, S.SI[orig], soff[t.begin + orig], depth + key_chars(R));
                }
            }
            // groups of 2..32 strings go to the warp kernel: their string indices in
            // sorted order back to the index buffer, keys gathered there; one
            // reservation of list slots per CTA and iteration
            const uint32_t nwl = S.nwl;
            if (tid == 0 && nwl) {
                S.wbase = atomicAdd(counters + C_NTASK + 0, nwl);
                atomicAdd(counters + C_ETASK + 0, S.nws);
            }
            __syncthreads();
            for (uint32_t w = warp; w < nwl; w += NW) {
                uint32_t e = S.WL[w];
                uint32_t s0 = e >> 16, sz = e & 0xFFFFu;
                if (lane < sz) {
                    uint32_t orig = S.SP[s0 + lane];
                    idx_hand[t.begin + s0 + lane] = S.SI[orig];
                    soff_hand[t.begin + s0 + lane] = soff[t.begin + orig];
                }
                if (lane == 0) {
                    uint32_t k = S.wbase + w;
                    if (k < tiny_cap) tiny[k] = SmallTask{t.begin + s0, sz, depth + key_chars(R), t.req, t.parity ^ 1u, 1u};
                    else set_error(counters, E_SMALL_OVERFLOW, k);
                }
            }
            __syncthreads();
            if (tid == 0) { S.nwl = 0; S.nws = 0; }
            M = M2;
            depth += key_chars(R);
            __syncthreads();
        }
        // positions that ended as groups of one
        if (!finished)
            for (uint32_t i = tid; i < m; i += NT)
                if (S.GS[S.SG[i]] == 1) {
                    R.perm_out[lbase + i] = S.SI[S.SP[i]];
                    put_off(R, lbase + i, soff[t.begin + S.SP[i]]);
                }
        __syncthreads();
        if (tid == 0) S.task = S.next;
        __syncthreads();
    }
}
