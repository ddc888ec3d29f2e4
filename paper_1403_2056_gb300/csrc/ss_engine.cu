// Super scalar string sample sort (S5) on one GB300, level-synchronous.
//
// k_init gives every string its index, byte offset and first characters;
// a large request whose strings all share a prefix starts that deep
// (k_shared_prefix, k_skip_prefix).  Then every recursion level of the
// paper's S5 (Algorithm 1, applied recursively as in Section 4.5) runs as a
// handful of kernels over ALL segments that are still larger than the
// base-case threshold, whatever request they belong to:
//
//   k_build_trees  sample (alpha = 2), sort, pick splitters with the
//                  skip-equal-samples recursion (Section 4.4)      one CTA / segment
//   k_jump_tables  (jump-table classifier only) a table over the key bits
//                  after the splitters' shared prefix (Section 8.1)  one CTA / segment
//   k_classify     tree descent + equality test per 8-byte key (or the
//                  S5-Equal descent, or table + descent), bucket buffer,
//                  per-tile histogram (Alg. 1 loops)                 one CTA / tile
//   k_scan_*       exclusive prefix sum over the bucket-major
//                  (segment, bucket, tile) counters (Theorem 1)
//   k_scatter      stable out-of-place redistribution of (index, offset,
//                  next key) through shared memory, final placement of
//                  singletons and all-equal buckets
//   k_buckets      child segments: big ones to the next level, small ones to
//                  the base case; bucket boundaries recorded for LCPs
//
// Segments of at most kSmallMax strings are sorted completely by the base
// case (k_small_warp / k_base_cta in ss_base.cuh), which also emits their LCPs
// (the role of LCP insertion sort, Algorithm 5).  The LCP between the last
// string of one bucket and the first of the next is depth + lcp of their keys
// at that depth (Section 5.4, "LCPs for free"), computed in k_boundary once all
// strings are placed.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <type_traits>
#include <vector>

#include "ss_internal.cuh"
#include "ss_base.cuh"

namespace ss {

// --------------------------------------------------------------- helpers

__host__ __device__ __forceinline__ uint32_t choose_d(uint32_t size, uint32_t target) {
    // v + 1 = 2^d about size / target, d in [2, kLevelD]
    uint32_t q = (size + target - 1) / target;
    uint32_t d = 0;
    while ((1u << d) < q) d++;
    if (d < 2) d = 2;
    if (d > (uint32_t)kLevelD) d = kLevelD;
    return d;
}

// Depth step of the even bucket between splitters x_{r-1} and x_r: its strings
// share lcp(x_{r-1}, x_r) more characters (0 for the outer buckets).  A step of
// fewer than min_step characters is not taken: the bucket keeps its depth and
// the key it carries, which still holds at least 8 - min_step + 1 unresolved
// characters, and the random gather of a new key is saved.  Any depth up to
// the shared prefix gives the same result.
__device__ __forceinline__ uint32_t even_delta(const ReqDesc &R, uint64_t xl, uint64_t xr, uint32_t r, uint32_t v,
                                               uint32_t min_step) {
    if (r == 0 || r == v) return 0u;
    uint32_t l = key_lcp(R, xl, xr);
    return l >= min_step ? l : 0u;
}

__host__ __device__ __forceinline__ uint32_t tiles_of(uint32_t size) { return (size + kTile - 1) / kTile; }
__host__ __device__ __forceinline__ uint32_t buckets_of(uint32_t d) { return (2u << d) - 1u; }

__device__ __forceinline__ uint32_t find_req(const ReqDesc *reqs, uint32_t nreq, uint32_t g) {
    uint32_t lo = 0, hi = nreq;   // last request with base <= g
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) / 2;
        if (reqs[mid].base <= g) lo = mid; else hi = mid;
    }
    return lo;
}

// last segment whose field (prefix) <= t
template <typename F>
__device__ __forceinline__ uint32_t find_seg(const BigSeg *segs, uint32_t nseg, uint32_t t, F field) {
    uint32_t lo = 0, hi = nseg;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) / 2;
        if (field(segs[mid]) <= t) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ------------------------------------------------------------ k_init

// every element starts as (string index, string offset, key at depth 0); the
// offset travels with the index so later gathers need one random load, not two
template <bool A>
__global__ void k_init(const ReqDesc *reqs, uint32_t nreq, uint32_t N, uint32_t *idx0, uint64_t *soff0, uint64_t *key0,
                       uint64_t *next0) {
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < N; g += gridDim.x * blockDim.x) {
        uint32_t r = find_req(reqs, nreq, g);
        const ReqDesc &R = reqs[r];
        uint32_t i = g - R.base;
        uint64_t off = __ldg(R.offsets + i);
        idx0[g] = i;
        soff0[g] = off;
        // characters 0..15: the second word serves the shared-prefix step below
        // (it lives in the other parity's key buffer until the first scatter)
        uint64_t k0, k1 = 0;
        if (A && R.alpha) k0 = key_at<A>(R, i, off, 0);   // no shared-prefix step for compressed keys
        else load_key2_o(R, i, off, 0, k0, k1);
        key0[g] = k0;
        next0[g] = k1;
        if (i == 0) {
            R.lcp_out[0] = 0;
            if (R.n == 1) R.perm_out[0] = 0;
        }
    }
}

// ------------------------------------------------- shared prefix of a request
// The strings of a large request may all share their first characters (a
// common scheme or host prefix); the first level's splitters would spend
// those.  The characters all of them share are the minimum over its strings
// of the lcp with its first string (one coalesced pass over the depth-0 keys,
// per chunk of a request's segment); the request's segment then starts that
// deep, with its keys reloaded there in input order.

constexpr uint32_t kPrefChunk = 8192;   // strings per CTA of the two passes below

__global__ void __launch_bounds__(256) k_shared_prefix(const uint4 *chunks, const ReqDesc *reqs, const uint64_t *key0,
                                                       uint32_t *shared) {
    __shared__ uint32_t wmin[8];
    const uint4 c = chunks[blockIdx.x];   // begin, end, request
    const uint64_t first = key0[reqs[c.z].base];
    uint32_t b = 8;
    for (uint32_t g = c.x + threadIdx.x; g < c.y; g += blockDim.x) {
        const uint64_t key = key0[g];
        const uint32_t l = key == first ? (has_zero(key) ? nulpos(key) : 8u) : lcp8(key, first);
        b = min(b, l);
        if (b == 0) break;   // nothing shared: the rest cannot lower it
    }
    b = __reduce_min_sync(0xffffffffu, b);
    if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; w++) b = min(b, wmin[w]);
        if (b < ((volatile uint32_t *)shared)[c.z]) atomicMin(shared + c.z, b);
    }
}

__global__ void __launch_bounds__(256) k_skip_prefix(const uint4 *chunks, const uint64_t *next0, uint64_t *key0,
                                                     const uint32_t *shared) {
    const uint4 c = chunks[blockIdx.x];
    const uint32_t b = shared[c.z];
    if (b == 0 || b > 8) return;
    // the key at depth b from characters 0..15 (zero past the end of a string)
    for (uint32_t g = c.x + threadIdx.x; g < c.y; g += blockDim.x)
        key0[g] = b == 8 ? next0[g] : (key0[g] << (8 * b)) | (next0[g] >> (64 - 8 * b));
}

__global__ void k_start_depth(BigSeg *big, uint32_t nbig, const uint32_t *shared) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nbig; k += gridDim.x * blockDim.x) {
        const uint32_t b = shared[big[k].req];
        if (b > 0 && b <= 8) big[k].depth = b;
    }
}

// ------------------------------------------------------ k_setup_big
// Exclusive prefix sums over the big list: tile_base, cnt_base, bkt_base,
// scan_base, from each segment's tree depth as k_build_trees chose it.  The
// totals of counters and (segment, bucket) pairs go to totals[0..1].

__global__ void __launch_bounds__(1024) k_setup_big(BigSeg *segs, uint32_t nseg, uint32_t *totals) {
    __shared__ uint32_t wsum[4][32];
    __shared__ uint32_t carry[4];
    if (threadIdx.x < 4) carry[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t base = 0; base < nseg; base += 1024) {
        uint32_t i = base + threadIdx.x;
        uint32_t v[4] = {0, 0, 0, 0};
        if (i < nseg) {
            BigSeg s = segs[i];
            uint32_t d = s.d;
            uint32_t t = tiles_of(s.size);
            uint32_t B = buckets_of(d);
            v[0] = t;
            v[1] = B * t;
            v[2] = B;
            v[3] = s.size;
        }
        uint32_t incl[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            uint32_t x = v[k];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= (uint32_t)o) x += y;
            }
            incl[k] = x;
            if (lane == 31) wsum[k][warp] = x;
        }
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                uint32_t x = wsum[k][lane];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= (uint32_t)o) x += y;
                }
                wsum[k][lane] = x;   // inclusive over warps
            }
        }
        __syncthreads();
        uint32_t excl[4];
#pragma unroll
        for (int k = 0; k < 4; k++) excl[k] = carry[k] + (warp ? wsum[k][warp - 1] : 0) + incl[k] - v[k];
        if (i < nseg) {
            BigSeg s = segs[i];
            s.tiles = v[0];
            s.tile_base = excl[0];
            s.cnt_base = excl[1];
            s.bkt_base = excl[2];
            s.scan_base = excl[3];
            segs[i] = s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < 4; k++) carry[k] += wsum[k][31];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        totals[0] = carry[1];
        totals[1] = carry[2];
    }
}

// ------------------------------------------------------ k_build_trees

// bitonic sort of n (power of two) u64 keys in shared memory
__device__ void bitonic_u64(uint64_t *s, uint32_t n) {
    for (uint32_t k = 2; k <= n; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t t = threadIdx.x; t < n / 2; t += blockDim.x) {
                uint32_t i = 2 * t - (t & (j - 1));   // lower index of the pair
                uint32_t l = i + j;
                bool up = (i & k) == 0;
                uint64_t a = s[i], b = s[l];
                if ((a > b) == up) { s[i] = b; s[l] = a; }
            }
            __syncthreads();
        }
    }
}

// Splitter pick of Section 4.4 on a sorted sample s[0..a): breadth-first over
// the implicit tree; node state (lo, hi, has_right, right, left).
struct PickNode {
    uint32_t lo, hi, has_right, pad;
    uint64_t right, left;
};

__device__ void pick_splitters(const uint64_t *s, uint32_t a, uint32_t d, uint64_t *x, PickNode *cur, PickNode *nxt) {
    if (threadIdx.x == 0) cur[0] = PickNode{0, a, 0, 0, 0ull, 0ull};
    __syncthreads();
    for (uint32_t l = 0; l < d; l++) {
        uint32_t nodes = 1u << l;
        uint32_t span = 1u << (d - l);   // slots covered: span - 1
        for (uint32_t j = threadIdx.x; j < nodes; j += blockDim.x) {
            PickNode nd = cur[j];
            uint32_t xm = j * span + span / 2 - 1;
            PickNode L, R;
            if (nd.lo >= nd.hi) {
                uint64_t val = nd.has_right ? nd.right : nd.left;
                x[xm] = val;
                L = PickNode{0, 0, 1, 0, val, nd.left};
                R = PickNode{0, 0, nd.has_right, 0, nd.right, val};
            } else {
                uint32_t m = nd.lo + (nd.hi - nd.lo) / 2;
                uint64_t sv = s[m];
                uint32_t lo = nd.lo, hi = m;   // first index in [lo, m] equal to sv
                while (lo < hi) {
                    uint32_t mid = (lo + hi) / 2;
                    if (s[mid] < sv) lo = mid + 1; else hi = mid;
                }
                uint32_t b = lo;
                lo = m; hi = nd.hi;             // first index in [m, hi) greater than sv
                while (lo < hi) {
                    uint32_t mid = (lo + hi) / 2;
                    if (s[mid] <= sv) lo = mid + 1; else hi = mid;
                }
                uint32_t ap = lo;
                x[xm] = sv;
                L = PickNode{nd.lo, b, 1, 0, sv, nd.left};
                R = PickNode{ap, nd.hi, nd.has_right, 0, nd.right, sv};
            }
            if (l + 1 < d) {
                nxt[2 * j] = L;
                nxt[2 * j + 1] = R;
            }
        }
        __syncthreads();
        PickNode *t = cur; cur = nxt; nxt = t;
    }
}

struct TreeSmem {
    uint64_t s[2 * (kMaxV + 1)];
    PickNode n0[(kMaxV + 1) / 2], n1[(kMaxV + 1) / 2];
};

// The sample has alpha * v + alpha - 1 keys (alpha = 2) for the tree size the
// segment's length allows (choose_d); the tree actually built has just enough
// levels for the distinct keys of the sample (adaptivity, Section 8.1): a
// segment whose sample holds 27 distinct keys gets 31 splitters, not 1023.
// The chosen depth is stored in the segment record; k_setup_big lays out the
// counters from it.
__global__ void __launch_bounds__(kThreads) k_build_trees(BigSeg *segs, const ReqDesc *reqs, const uint64_t *key,
                                                           uint64_t *splitters) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TreeSmem &S = *reinterpret_cast<TreeSmem *>(smem_raw);
    __shared__ uint32_t distinct;
    BigSeg sg = segs[blockIdx.x];
    const uint32_t dmax = choose_d(sg.size, req_child_target(reqs[sg.req]));
    uint32_t v = (1u << dmax) - 1;
    uint32_t a = 2 * v + 1;            // alpha * v + alpha - 1 with alpha = 2
    uint32_t P = a + 1;
    if (threadIdx.x == 0) distinct = 0;
    uint64_t seed = ((uint64_t)sg.begin << 32) ^ (uint64_t)sg.depth * 0x9E3779B97F4A7C15ULL;
    for (uint32_t j = threadIdx.x; j < P; j += blockDim.x) {
        if (j < a) {
            uint32_t pos = (uint32_t)(mix64(seed + j) % sg.size);
            S.s[j] = key[sg.begin + pos];
        } else {
            S.s[j] = ~0ull;
        }
    }
    __syncthreads();
    bitonic_u64(S.s, P);
    uint32_t mine = 0;
    for (uint32_t j = threadIdx.x; j < a; j += blockDim.x) mine += (j == 0 || S.s[j] != S.s[j - 1]) ? 1u : 0u;
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&distinct, mine);
    __syncthreads();
    uint32_t d = 1;
    while (d < dmax && ((1u << d) - 1) < distinct) d++;
    if (threadIdx.x == 0) segs[blockIdx.x].d = d;
    uint64_t *x = splitters + (size_t)blockIdx.x * kMaxV;
    pick_splitters(S.s, a, d, x, S.n0, S.n1);
}

// stand-alone splitter pick (ss_splitters): sample given, a <= 2047
__global__ void __launch_bounds__(kThreads) k_pick_only(const uint64_t *sample, uint32_t a, uint32_t d, uint64_t *x) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TreeSmem &S = *reinterpret_cast<TreeSmem *>(smem_raw);
    uint32_t P = 1;
    while (P < a) P <<= 1;
    for (uint32_t j = threadIdx.x; j < P; j += blockDim.x) S.s[j] = j < a ? sample[j] : ~0ull;
    __syncthreads();
    bitonic_u64(S.s, P);
    pick_splitters(S.s, a, d, x, S.n0, S.n1);
}

// ------------------------------------------------------------ k_classify

template <int D>
struct ClassifySmem {
    uint64_t t[(1 << D)];   // level order, one-based (t[0] unused)
    uint64_t x[(1 << D)];   // in order, x[v] unused
    uint32_t cnt[(2 << D)];
    uint16_t j[1 << kJumpBits];   // jump table (CLS_JUMP segments only)
};

// load the in-order splitters and build the level-order tree (Figure 1):
// node i at level l, position j = i - 2^l holds x[(2j + 1) 2^(d-l-1) - 1]
__device__ __forceinline__ void load_tree(const uint64_t *xs, uint32_t d, uint64_t *t, uint64_t *x) {
    uint32_t v = (1u << d) - 1;
    for (uint32_t k = threadIdx.x; k < v; k += blockDim.x) x[k] = xs[k];
    __syncthreads();
    for (uint32_t i = threadIdx.x + 1; i <= v; i += blockDim.x) {
        uint32_t l = 31 - __clz(i);
        uint32_t j = i - (1u << l);
        t[i] = x[((2 * j + 1) << (d - l - 1)) - 1];
    }
}

// Jump tables.  All keys between the smallest and the largest splitter share
// the splitters' common prefix of s bits (s = clz(x_0 xor x_{v-1}), at most
// 64 - kJumpBits); a key whose top s bits are below that prefix lies below
// x_0 (leaf 2^d, bucket 0), above it lies above x_{v-1} (leaf 2^(d+1) - 1,
// bucket 2v).  Entry p covers the keys with the prefix followed by the
// kJumpBits bits p, an interval [lo, hi]; its descent is fixed while the node's
// splitter t is below lo (every key goes right) or at least hi (every key goes
// left), and the entry holds the first node where it is not, or the leaf.
__device__ __forceinline__ uint32_t jump_shift(uint64_t x0, uint64_t xl) {
    uint32_t s = x0 == xl ? 64u : (uint32_t)__clzll((long long)(x0 ^ xl));
    return min(s, 64u - (uint32_t)kJumpBits);
}
__device__ __forceinline__ uint64_t prefix_mask(uint32_t s) { return s ? ~0ull << (64 - s) : 0ull; }

// one table per segment whose request classifies with CLS_JUMP (all segments
// when reqs is NULL); one CTA per segment
__global__ void __launch_bounds__(kThreads) k_jump_tables(const BigSeg *__restrict__ segs, const ReqDesc *__restrict__ reqs,
                                                          const uint64_t *__restrict__ splitters, uint16_t *__restrict__ jt) {
    __shared__ uint64_t t[kMaxV + 1];
    const BigSeg sg = segs[blockIdx.x];
    if (reqs && req_classifier(reqs[sg.req]) != CLS_JUMP) return;
    const uint32_t d = sg.d, v = (1u << d) - 1;
    const uint64_t *x = splitters + (size_t)blockIdx.x * kMaxV;
    for (uint32_t i = threadIdx.x + 1; i <= v; i += blockDim.x) {
        uint32_t l = 31 - __clz(i);
        t[i] = x[((2 * (i - (1u << l)) + 1) << (d - l - 1)) - 1];
    }
    __syncthreads();
    const uint32_t s = jump_shift(x[0], x[v - 1]);
    const uint64_t pre = x[0] & prefix_mask(s);
    const uint32_t low = 64 - s - kJumpBits;   // key bits below an entry's range
    uint16_t *J = jt + (size_t)blockIdx.x * kJumpStride;
    for (uint32_t p = threadIdx.x; p < (1u << kJumpBits); p += blockDim.x) {
        const uint64_t lo = pre | ((uint64_t)p << low);
        const uint64_t hi = lo | ((1ull << low) - 1);
        uint32_t i = 1;
        while (i <= v) {
            const uint64_t ti = t[i];
            if (ti < lo) i = 2 * i + 1;
            else if (ti >= hi) i = 2 * i;
            else break;
        }
        J[p] = (uint16_t)i;
    }
    if (threadIdx.x == 0) J[1 << kJumpBits] = (uint16_t)s;
}

// Lanes of the warp whose value b agrees with this lane's in the low nbits
// bits: one vote per bit (nbits must be the same in the whole warp).  A bucket
// id of a tree of depth d has d + 1 bits and is at most 2^(d+1) - 2, so the
// marker 0xFFFF of an empty slot never agrees with a bucket.
__device__ __forceinline__ uint32_t peers_of(uint32_t b, uint32_t nbits) {
    uint32_t m = 0xFFFFFFFFu;
    for (uint32_t k = 0; k < nbits; k++) {
        const uint32_t bit = (b >> k) & 1u;
        const uint32_t vote = __ballot_sync(0xFFFFFFFFu, bit);
        m &= bit ? vote : ~vote;
    }
    return m;
}

// Tile histogram update: 1 = one shared atomic per element; 0 = lanes with
// equal buckets add once (warp match), slower on GB300 for every workload
// measured (the match costs more than the atomics it saves).
#ifndef SS_CLASSIFY_COUNT
#define SS_CLASSIFY_COUNT 1
#endif

// bucket b of element p into the bucket buffer and the tile histogram
__device__ __forceinline__ void emit_bucket(uint32_t *cnt, uint16_t *obuf, uint32_t p, bool ok, uint32_t b, uint32_t lane) {
    if (ok) obuf[p] = (uint16_t)b;
#if SS_CLASSIFY_COUNT == 1
    if (ok) atomicAdd(&cnt[b], 1u);
#else
    uint32_t key_b = ok ? b : 0xFFFFu;
    uint32_t peers = __match_any_sync(0xffffffffu, key_b);
    if (ok && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&cnt[b], (uint32_t)__popc(peers));
#endif
}

// The classifier is the segment's request's (or `cls` for all segments when
// reqs is NULL); jt holds the jump tables of CLS_JUMP segments.
template <int D>
__global__ void __launch_bounds__(kThreads) k_classify(const BigSeg *__restrict__ segs, uint32_t nseg,
                                                       const ReqDesc *__restrict__ reqs, uint32_t cls_all,
                                                       const uint64_t *__restrict__ key,
                                                       const uint64_t *__restrict__ splitters,
                                                       const uint16_t *__restrict__ jt,
                                                       uint16_t *__restrict__ obuf, uint32_t *__restrict__ counts) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ClassifySmem<D> &S = *reinterpret_cast<ClassifySmem<D> *>(smem_raw);
    const uint32_t tile = blockIdx.x;
    const uint32_t si = find_seg(segs, nseg, tile, [](const BigSeg &s) { return s.tile_base; });
    const BigSeg sg = segs[si];
    const uint32_t tl = tile - sg.tile_base;
    const uint32_t d = sg.d, v = (1u << d) - 1, B = 2 * v + 1;
    const uint32_t cls = reqs ? req_classifier(reqs[sg.req]) : cls_all;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t seg_end = sg.begin + sg.size;
    const uint32_t wbeg = sg.begin + tl * kTile + warp * kWarpSpan;
    // every key of this thread in flight while the tree is staged
    uint64_t c[kItems];
#pragma unroll
    for (int u = 0; u < kItems; u++) {
        uint32_t p = wbeg + u * 32 + lane;
        c[u] = p < seg_end ? key[p] : 0ull;
    }
    load_tree(splitters + (size_t)si * kMaxV, d, S.t, S.x);
    for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) S.cnt[b] = 0;
    uint32_t jshift = 0;
    if (cls == CLS_JUMP) {
        const uint16_t *J = jt + (size_t)si * kJumpStride;   // 16-byte aligned rows
        const uint4 *src = reinterpret_cast<const uint4 *>(J);
        uint4 *dst = reinterpret_cast<uint4 *>(S.j);
        for (uint32_t k = threadIdx.x; k < (1u << kJumpBits) / 8; k += blockDim.x) dst[k] = src[k];
        jshift = J[1 << kJumpBits];
    }
    __syncthreads();

    if (cls == CLS_EQUAL) {
        // one descent per key; the first splitter equal to the key ends it
#pragma unroll
        for (int u = 0; u < kItems; u++) {
            const uint32_t p = wbeg + u * 32 + lane;
            uint32_t i = 1, b = 0xFFFFFFFFu;
            for (uint32_t l = 0; l < d; l++) {
                const uint64_t tv = S.t[i];
                if (c[u] == tv) {   // node i of level l is in-order splitter k
                    b = 2 * ((((2 * (i - (1u << l)) + 1) << (d - l - 1)) - 1)) + 1;
                    break;
                }
                i = 2 * i + (c[u] > tv ? 1u : 0u);
            }
            if (b == 0xFFFFFFFFu) b = 2 * (i - (v + 1));
            emit_bucket(S.cnt, obuf, p, p < seg_end, b, lane);
        }
    } else {
        const uint64_t pm = prefix_mask(jshift);
        const uint64_t pre = S.x[0] & pm;
        // four interleaved descents per thread (Section 4.3: unrolled, interleaved loops)
#pragma unroll
        for (int it = 0; it < kItems; it += 4) {
            uint32_t p[4], node[4];
            bool ok[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                p[u] = wbeg + (it + u) * 32 + lane;
                ok[u] = p[u] < seg_end;
                node[u] = 1;
            }
            if (cls == CLS_JUMP) {
                uint32_t lmin = D;
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const uint64_t cu = c[it + u], cp = cu & pm;
                    node[u] = cp < pre ? v + 1 : cp > pre ? 2 * v + 1 : (uint32_t)S.j[(cu << jshift) >> (64 - kJumpBits)];
                    lmin = min(lmin, 31u - __clz(node[u]));
                }
                // finish the descents: nodes already at a leaf stay there
                for (uint32_t l = lmin; l < d; l++) {
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const bool in = node[u] <= v;
                        const uint64_t tv = S.t[in ? node[u] : 1u];
                        node[u] = in ? 2 * node[u] + (c[it + u] > tv ? 1u : 0u) : node[u];
                    }
                }
            } else {
                for (uint32_t l = 0; l < d; l++) {
#pragma unroll
                    for (int u = 0; u < 4; u++) node[u] = 2 * node[u] + (c[it + u] > S.t[node[u]] ? 1u : 0u);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                uint32_t r = node[u] - (v + 1);
                uint32_t b = 2 * r + ((r < v && S.x[r] == c[it + u]) ? 1u : 0u);
                emit_bucket(S.cnt, obuf, p[u], ok[u], b, lane);
            }
        }
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) counts[sg.cnt_base + b * sg.tiles + tl] = S.cnt[b];
}

// ------------------------------------------------------------ scan
constexpr int kScanItems = 16;
constexpr int kScanChunk = kThreads * kScanItems;   // 4096

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t *wsum, uint32_t *total) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kWarps ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= (uint32_t)o) w += y;
        }
        if (lane < kWarps) wsum[lane] = w;
    }
    __syncthreads();
    uint32_t r = (warp ? wsum[warp - 1] : 0) + incl - x;
    if (total) *total = wsum[kWarps - 1];
    __syncthreads();
    return r;
}

// The scans read their length n from device memory (the level's counter
// total is known only on the device); the grid is sized for an upper bound.
__global__ void __launch_bounds__(kThreads) k_scan_reduce(const uint32_t *a, const uint32_t *n_dev, uint32_t *partial) {
    __shared__ uint32_t wsum[32];
    const uint32_t n = *n_dev;
    uint32_t base = blockIdx.x * kScanChunk;
    if (base >= n) return;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        uint32_t i = base + k * kThreads + threadIdx.x;
        if (i < n) s += a[i];
    }
    uint32_t total;
    block_excl_scan(s, wsum, &total);
    if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_partials(uint32_t *partial, const uint32_t *n_dev) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    const uint32_t np = (*n_dev + kScanChunk - 1) / kScanChunk;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t base = 0; base < np; base += 1024) {
        uint32_t i = base + threadIdx.x;
        uint32_t x = i < np ? partial[i] : 0;
        uint32_t incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= (uint32_t)o) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        uint32_t ex = carry + (warp ? wsum[warp - 1] : 0) + incl - x;
        if (i < np) partial[i] = ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[31];
        __syncthreads();
    }
}

// in-place exclusive scan of a chunk plus its partial offset
__global__ void __launch_bounds__(kThreads) k_scan_down(uint32_t *a, const uint32_t *n_dev, const uint32_t *partial) {
    __shared__ uint32_t wsum[32];
    const uint32_t n = *n_dev;
    if (blockIdx.x * kScanChunk >= n) return;
    uint32_t base = blockIdx.x * kScanChunk + threadIdx.x * kScanItems;   // thread-contiguous
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        uint32_t i = base + k;
        v[k] = i < n ? a[i] : 0;
        s += v[k];
    }
    uint32_t off = block_excl_scan(s, wsum, nullptr) + partial[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        uint32_t i = base + k;
        if (i < n) a[i] = off;
        off += v[k];
    }
}

// ------------------------------------------------------------ k_scatter

template <int D>
struct ScatterSmem {
    static constexpr int MB = 2 * ((1 << D) - 1) + 1;   // buckets of a tree of depth D
    union {
        uint16_t wpos[kWarps][MB + 1];   // per warp: count, then running offset inside the tile's bucket
        uint64_t buf[kTile + 2];            // after the ranks: the tile's keys, then its string offsets
    } u;
    uint32_t sidx[kTile + 8];    // the tile's string indices (range rounded out to 16 bytes)
    uint32_t tbase[MB + 1];   // global position of each bucket's first string from this tile
    uint16_t lbase[MB + 1];   // tile-local start of each bucket (exclusive scan of the tile's counts)
    uint16_t binfo[MB + 1];   // delta | final << 6 | done << 7 | first tile << 8 | key length << 9
    uint16_t slot_b[kTile];      // bucket of each tile-local slot
    uint16_t src[kTile];         // tile element held by each slot
    uint32_t wcnt[kWarps];
    uint64_t bar[3];             // completion of the index, key and offset copies
};

static_assert(offsetof(ScatterSmem<kMaxD>, sidx) % 16 == 0 && offsetof(ScatterSmem<kLevelD>, sidx) % 16 == 0,
              "bulk copy targets 16-byte aligned");
static_assert(offsetof(ScatterSmem<kMaxD>, bar) % 8 == 0 && offsetof(ScatterSmem<kLevelD>, bar) % 8 == 0,
              "mbarriers 8-byte aligned");

enum { MODE_SORT = 0, MODE_CLASSIFY = 1 };

// bucket facts of the scatter (ScatterSmem::binfo): the depth step (up to the
// 32 characters of a compressed key), final (placed now), done (all equal and
// complete), the bucket's first tile, and the characters of the string in the
// equality bucket's key
constexpr uint32_t BI_DELTA = 0x3Fu, BI_FIN = 1u << 6, BI_DONE = 1u << 7, BI_FIRST = 1u << 8;
constexpr int BI_NP = 9;

// position of (bucket b, tile tl) from the scanned counters
__device__ __forceinline__ uint32_t tile_pos(const BigSeg &sg, const uint32_t *scan, uint32_t b, uint32_t tl) {
    return sg.begin + scan[sg.cnt_base + b * sg.tiles + tl] - sg.scan_base;
}

__device__ __forceinline__ uint32_t bucket_start(const BigSeg &sg, const uint32_t *scan, uint32_t b, uint32_t B) {
    return b < B ? tile_pos(sg, scan, b, 0) : sg.begin + sg.size;
}

#ifndef SS_SCATTER_MINB
#define SS_SCATTER_MINB 2
#endif

// Stable out-of-place redistribution of one tile (Section 4.3, the second hot
// loop).  Each element's rank inside the tile is fixed first (lanes in order
// inside a warp, warps in order inside the tile), giving every element its
// tile-local slot in bucket order.  The payload never passes through
// registers: the tile's string indices are copied into shared memory by one
// bulk copy issued at the start, its keys and then its string offsets by bulk
// copies into the space the per-warp counts leave once the ranks are known;
// each array is then written out slot by slot, so that consecutive threads
// write the consecutive positions of a bucket's run.  Strings whose bucket is
// final (one string, or all equal and complete) go straight to the output.
// Strings whose bucket continues deeper keep their carried key only if the
// depth stays; otherwise their next key is gathered afterwards (k_gather_new).
// Phase A's per-warp counts are one shared atomic per element; the rank
// inside a warp step comes from one vote per bucket bit (peers_of).
template <int MODE, int D>
__global__ void __launch_bounds__(kThreads, SS_SCATTER_MINB) k_scatter(const BigSeg *__restrict__ segs, uint32_t nseg,
                                                      const ReqDesc *__restrict__ reqs,
                                                      const uint32_t *__restrict__ idx_in,
                                                      const uint64_t *__restrict__ soff_in,
                                                      const uint64_t *__restrict__ key_in,
                                                      const uint16_t *__restrict__ obuf,
                                                      const uint32_t *__restrict__ scan,
                                                      const uint64_t *__restrict__ splitters,
                                                      uint32_t *__restrict__ idx_out, uint64_t *__restrict__ soff_out,
                                                      uint64_t *__restrict__ key_out, uint32_t *counters) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScatterSmem<D> &S = *reinterpret_cast<ScatterSmem<D> *>(smem_raw);
    constexpr int MB = ScatterSmem<D>::MB;
    const uint32_t tile = blockIdx.x;
    const uint32_t si = find_seg(segs, nseg, tile, [](const BigSeg &s) { return s.tile_base; });
    const BigSeg sg = segs[si];
    const uint32_t tl = tile - sg.tile_base;
    const uint32_t d = sg.d, v = (1u << d) - 1, B = 2 * v + 1;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t seg_end = sg.begin + sg.size;
    const uint32_t tbeg = sg.begin + tl * kTile;
    const uint32_t tcount = min((uint32_t)kTile, seg_end - tbeg);
    const uint32_t wbeg = tbeg + warp * kWarpSpan;
    const uint64_t *xs = splitters + (size_t)si * kMaxV;
    // the tile's ranges rounded out to 16 bytes (the arrays start 256-byte aligned
    // and are padded, so the rounded ranges stay inside the scratch block)
    const uint32_t i0 = tbeg & ~3u, ioff = tbeg - i0;
    const uint32_t ibytes = 4u * (((tbeg + tcount + 3u) & ~3u) - i0);
    const uint32_t k0 = tbeg & ~1u, koff = tbeg - k0;
    const uint32_t kbytes = 8u * (((tbeg + tcount + 1u) & ~1u) - k0);

    if (MODE == MODE_SORT && threadIdx.x == 0) {
        for (int k = 0; k < 3; k++) mbar_init(&S.bar[k], 1);
        fence_mbar_init();
        mbar_expect_tx(&S.bar[0], ibytes);
        bulk_to_smem(S.sidx, idx_in + i0, ibytes, &S.bar[0]);
    }
    // every bucket id of this thread in flight at once; kept in registers
    uint32_t bk[kItems];
#pragma unroll
    for (int u = 0; u < kItems; u++) {
        uint32_t p = wbeg + u * 32 + lane;
        bk[u] = p < seg_end ? (uint32_t)obuf[p] : 0xFFFFu;
    }
    for (uint32_t k = threadIdx.x; k < kWarps * (MB + 1) / 2; k += blockDim.x)
        reinterpret_cast<uint32_t *>(&S.u.wpos[0][0])[k] = 0;
    __syncthreads();
    // phase A: per-warp bucket counts of its contiguous span, one shared atomic
    // per element on the 32-bit word holding the 16-bit count (a warp's span has
    // 512 elements, so a count never carries into its neighbour)
#pragma unroll
    for (int u = 0; u < kItems; u++)
        if (bk[u] != 0xFFFFu)
            atomicAdd(reinterpret_cast<uint32_t *>(&S.u.wpos[warp][bk[u] & ~1u]), 1u << (16 * (bk[u] & 1u)));
    __syncthreads();
    // phase B: each warp's offset inside the tile's part of every bucket, the
    // tile's count of every bucket (in lbase for now) and the bucket facts.  The
    // counter and splitter reads of a half of this thread's buckets go out together.
    static_assert(MB + 1 >= kThreads, "at least one bucket slot per thread");
    constexpr int kPerT = (MB + 1) / kThreads;            // bucket slots per thread
    constexpr int kHalf = kPerT >= 2 ? kPerT / 2 : 1;
#pragma unroll
    for (int half = 0; half < kPerT / kHalf; half++) {
        uint32_t tb[kHalf], st[kHalf], en[kHalf];
        uint64_t xr[kHalf], xl[kHalf];
#pragma unroll
        for (int k = 0; k < kHalf; k++) {
            uint32_t b = threadIdx.x + (half * kHalf + k) * kThreads;
            bool in = b < B;
            tb[k] = in ? tile_pos(sg, scan, b, tl) : 0u;
            if (MODE == MODE_SORT) {
                uint32_t r = b >> 1;
                st[k] = in ? bucket_start(sg, scan, b, B) : 0u;
                en[k] = in ? bucket_start(sg, scan, b + 1, B) : 0u;
                xr[k] = (in && r < v) ? xs[r] : 0ull;
                xl[k] = (in && !(b & 1) && r > 0 && r < v) ? xs[r - 1] : 0ull;
            }
        }
#pragma unroll
        for (int k = 0; k < kHalf; k++) {
            uint32_t b = threadIdx.x + (half * kHalf + k) * kThreads;
            uint32_t run = 0;
            if (b < B) {
#pragma unroll
                for (int w = 0; w < kWarps; w++) {
                    uint32_t c = S.u.wpos[w][b];
                    S.u.wpos[w][b] = (uint16_t)run;
                    run += c;
                }
                S.tbase[b] = tb[k];
                if (MODE == MODE_SORT) {
                    const ReqDesc &RQ = reqs[sg.req];
                    uint32_t r = b >> 1;
                    uint32_t delta, done = 0, np = 0;
                    if (b & 1) {
                        np = key_len(RQ, xr[k], sg.depth);
                        done = key_ends(RQ, xr[k], sg.depth);   // equal keys that hold the end of the string: all equal
                        delta = key_chars(RQ);
                    } else {
                        delta = even_delta(RQ, xl[k], xr[k], r, v, req_min_step(RQ));
                    }
                    uint32_t fin = (en[k] - st[k] == 1) || done;
                    uint32_t first = tb[k] == st[k];
                    S.binfo[b] = (uint16_t)(delta | (fin ? BI_FIN : 0u) | (done ? BI_DONE : 0u) | (first ? BI_FIRST : 0u) |
                                            (np << BI_NP));
                }
            }
            S.lbase[b] = (uint16_t)run;
        }
    }
    __syncthreads();
    // tile-local bucket starts: exclusive scan of the counts, 8 contiguous buckets per thread
    {
        constexpr int kPer = (MB + 1) / kThreads;
        uint32_t c[kPer], sum = 0;
#pragma unroll
        for (int k = 0; k < kPer; k++) { c[k] = S.lbase[threadIdx.x * kPer + k]; sum += c[k]; }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        if (lane == 31) S.wcnt[warp] = incl;
        __syncthreads();
        uint32_t base = incl - sum;
        for (uint32_t w = 0; w < warp; w++) base += S.wcnt[w];
#pragma unroll
        for (int k = 0; k < kPer; k++) { S.lbase[threadIdx.x * kPer + k] = (uint16_t)base; base += c[k]; }
    }
    __syncthreads();
    // ranks: tile-local slot of every element, and the element of every slot
#pragma unroll
    for (int u = 0; u < kItems; u++) {
        const uint32_t b = bk[u];
        const bool ok = b != 0xFFFFu;
        uint32_t peers = peers_of(b, d + 1);
        uint32_t rank = __popc(peers & lanemask_lt());
        uint32_t off = ok ? S.u.wpos[warp][b] : 0u;
        const uint32_t lp = ok ? S.lbase[b] + off + rank : 0u;
        __syncwarp();
        if (ok && lane == (uint32_t)(__ffs(peers) - 1)) S.u.wpos[warp][b] = (uint16_t)(off + __popc(peers));
        __syncwarp();
        if (ok) {
            S.slot_b[lp] = (uint16_t)b;
            S.src[lp] = (uint16_t)(warp * kWarpSpan + u * 32 + lane);
        }
    }
    fence_proxy_async();   // this thread's accesses of the count space come before the key copy into it
    __syncthreads();       // wpos is dead from here: its space takes the keys, then the offsets
    if (MODE == MODE_CLASSIFY) {
        for (uint32_t s = threadIdx.x; s < tcount; s += kThreads) {
            const uint32_t b = S.slot_b[s];
            const uint32_t q = S.tbase[b] + (s - S.lbase[b]);
            if (q < sg.begin || q >= seg_end) { set_error(counters, E_BAD_POS, q); continue; }
            idx_out[q - sg.begin] = tl * kTile + S.src[s];
        }
        return;
    }
    if (threadIdx.x == 0) {
        mbar_expect_tx(&S.bar[1], kbytes);
        bulk_to_smem(S.u.buf, key_in + k0, kbytes, &S.bar[1]);
    }
    // string indices; strings whose bucket is final go straight to the output
    if (!__syncthreads_and(mbar_wait(&S.bar[0], 0))) {
        if (threadIdx.x == 0) set_error(counters, E_COPY_TIMEOUT, tile);
        mbar_wait(&S.bar[1], 0);
        return;
    }
    const ReqDesc &R = reqs[sg.req];
    for (uint32_t s = threadIdx.x; s < tcount; s += kThreads) {
        const uint32_t b = S.slot_b[s];
        const uint32_t lo = s - S.lbase[b];
        const uint32_t q = S.tbase[b] + lo;
        if (q < sg.begin || q >= seg_end) { set_error(counters, E_BAD_POS, q); continue; }
        const uint32_t id = S.sidx[ioff + S.src[s]];
        const uint32_t info = S.binfo[b];
        if (info & BI_FIN) {
            const uint32_t local = q - R.base;
            R.perm_out[local] = id;
            // all equal and complete: every string but the bucket's first has the whole key in common
            if ((info & BI_DONE) && (!(info & BI_FIRST) || lo > 0)) R.lcp_out[local] = sg.depth + (info >> BI_NP);
        } else {
            idx_out[q] = id;
        }
    }
    // keys: the carried key where the depth stays (others are gathered later)
    if (!__syncthreads_and(mbar_wait(&S.bar[1], 0))) {
        if (threadIdx.x == 0) set_error(counters, E_COPY_TIMEOUT, tile);
        return;
    }
    for (uint32_t s = threadIdx.x; s < tcount; s += kThreads) {
        const uint32_t b = S.slot_b[s];
        const uint32_t info = S.binfo[b];
        if (info & (BI_FIN | BI_DELTA)) continue;   // final, or a new depth
        const uint32_t q = S.tbase[b] + (s - S.lbase[b]);
        if (q < sg.begin || q >= seg_end) continue;
        key_out[q] = S.u.buf[koff + S.src[s]];
    }
    fence_proxy_async();
    __syncthreads();   // every key read from the buffer: it takes the offsets next
    if (threadIdx.x == 0) {
        mbar_expect_tx(&S.bar[2], kbytes);
        bulk_to_smem(S.u.buf, soff_in + k0, kbytes, &S.bar[2]);
    }
    if (!__syncthreads_and(mbar_wait(&S.bar[2], 0))) {
        if (threadIdx.x == 0) set_error(counters, E_COPY_TIMEOUT, tile);
        return;
    }
    for (uint32_t s = threadIdx.x; s < tcount; s += kThreads) {
        const uint32_t b = S.slot_b[s];
        if (S.binfo[b] & BI_FIN) continue;
        const uint32_t q = S.tbase[b] + (s - S.lbase[b]);
        if (q < sg.begin || q >= seg_end) continue;
        soff_out[q] = S.u.buf[koff + S.src[s]];
    }
}

// ------------------------------------------------------------ k_buckets

__device__ __forceinline__ void push_small(const TaskLists &tl, uint32_t *counters, SmallTask t) {
    const int c = class_of(t.size);
    uint32_t k = atomicAdd(counters + C_NTASK + c, 1u);
    atomicAdd(counters + C_ETASK + c, t.size);
    if (k < tl.cap[c]) tl.l[c][k] = t; else set_error(counters, E_SMALL_OVERFLOW, k);
}

// Child segments of every (segment, bucket) pair.  A bucket whose strings
// continue at a new depth needs their keys there: buckets of more than 32
// strings get gather chunks (k_gather_new loads the keys right after this
// level), smaller ones become warp tasks that load their own keys.
__global__ void __launch_bounds__(kThreads) k_buckets(const BigSeg *segs, uint32_t nseg, const ReqDesc *reqs,
                                                      const uint32_t *npairs_dev,
                                                      const uint32_t *scan, const uint64_t *splitters,
                                                      uint32_t next_parity, BigSeg *next_big, TaskLists tl,
                                                      Boundary *bounds, GatherChunk *gchunks, Caps caps,
                                                      uint32_t *counters) {
    uint32_t pr = blockIdx.x * blockDim.x + threadIdx.x;
    if (pr >= *npairs_dev) return;
    uint32_t si = find_seg(segs, nseg, pr, [](const BigSeg &s) { return s.bkt_base; });
    BigSeg sg = segs[si];
    uint32_t b = pr - sg.bkt_base;
    uint32_t v = (1u << sg.d) - 1, B = 2 * v + 1;
    if (b >= B) return;
    uint32_t st = bucket_start(sg, scan, b, B);
    uint32_t en = bucket_start(sg, scan, b + 1, B);
    if (en <= st) return;
    if (st > sg.begin) {
        uint32_t k = atomicAdd(counters + C_NBOUND, 1u);
        if (k < caps.bound) bounds[k] = Boundary{st, sg.depth, sg.req};
        else set_error(counters, E_BOUND_OVERFLOW, k);
    }
    uint32_t size = en - st;
    if (size == 1) return;
    const uint64_t *xs = splitters + (size_t)si * kMaxV;
    const ReqDesc &RQ = reqs[sg.req];
    uint32_t r = b >> 1, delta;
    if (b & 1) {
        if (key_ends(RQ, xs[r], sg.depth)) return;   // all equal and complete: placed by k_scatter
        delta = key_chars(RQ);
    } else {
        delta = even_delta(RQ, r > 0 ? xs[r - 1] : 0ull, r < v ? xs[r] : 0ull, r, v, req_min_step(RQ));
    }
    uint32_t depth = sg.depth + delta;
    const bool regather = delta != 0;
    if (regather && size > kTinyMax) {
        const uint32_t nch = (size + kGatherChunk - 1) / kGatherChunk;
        const uint32_t k = atomicAdd(counters + C_NGATHER, nch);
        if (k + nch <= caps.gather) {
            for (uint32_t j = 0; j < nch; j++)
                gchunks[k + j] = GatherChunk{st + j * kGatherChunk, min(en, st + (j + 1) * kGatherChunk), sg.req, depth};
        } else {
            set_error(counters, E_GATHER_OVERFLOW, k);
        }
    }
    if (size > kSmallMax) {
        uint32_t k = atomicAdd(counters + C_NBIG, 1u);
        if (k < caps.big) {
            BigSeg c{};
            c.begin = st; c.size = size; c.depth = depth; c.req = sg.req;
            next_big[k] = c;
            uint32_t d = choose_d(size, req_child_target(reqs[sg.req])), t = tiles_of(size), Bc = buckets_of(d);
            atomicAdd(counters + C_TILES, t);
            atomicAdd(counters + C_COUNTS, Bc * t);
            atomicAdd(counters + C_PAIRS, Bc);
            atomicAdd(counters + C_ELEMS, size);
        } else {
            set_error(counters, E_BIG_OVERFLOW, k);
        }
    } else {
        push_small(tl, counters, SmallTask{st, size, depth, sg.req, next_parity, (regather && size <= kTinyMax) ? 1u : 0u});
    }
}

// the next keys of every gather chunk of the level (a fixed grid walks the
// chunk list, whose length is read on the device)
template <bool A>
__global__ void __launch_bounds__(256) k_gather_new(const GatherChunk *__restrict__ gchunks, const uint32_t *nchunks_dev,
                                                    const ReqDesc *__restrict__ reqs, const uint32_t *__restrict__ idx,
                                                    const uint64_t *__restrict__ soff, uint64_t *__restrict__ key) {
    const uint32_t nch = *nchunks_dev;
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
        const GatherChunk g = gchunks[c];
        const ReqDesc &R = reqs[g.req];
        constexpr int U = kGatherChunk / 256;
        uint32_t id[U];
        uint64_t so[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint32_t p = g.begin + u * 256 + threadIdx.x;
            id[u] = p < g.end ? idx[p] : 0u;
            so[u] = p < g.end ? soff[p] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint32_t p = g.begin + u * 256 + threadIdx.x;
            if (p < g.end) key[p] = key_at<A>(R, id[u], so[u], g.depth);
        }
    }
}

// base case sorters: ss_base.cuh

// ------------------------------------------------------------ k_boundary

template <bool A>
__global__ void k_boundary(const Boundary *bounds, uint32_t nb, const ReqDesc *reqs) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x) {
        Boundary b = bounds[k];
        const ReqDesc &R = reqs[b.req];
        uint32_t lp = b.pos - R.base;
        uint32_t sa = R.perm_out[lp - 1], sb = R.perm_out[lp];
        uint64_t ka = key_at<A>(R, sa, __ldg(R.offsets + sa), b.depth), kb = key_at<A>(R, sb, __ldg(R.offsets + sb), b.depth);
        R.lcp_out[lp] = b.depth + key_lcp<A>(R, ka, kb);
    }
}

__global__ void k_status(const ReqDesc *reqs, uint32_t nreq, int32_t code) {
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nreq; r += gridDim.x * blockDim.x)
        if (reqs[r].status_out) *reqs[r].status_out = code;
}

__global__ void k_gather(ReqDesc R, const uint32_t *depth, uint64_t *keys) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < R.n; i += gridDim.x * blockDim.x)
        keys[i] = load_key(R, i, depth[i]);
}

__global__ void k_iota(uint32_t *a, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = i;
}

__global__ void k_bucket_begin(const BigSeg *seg, const uint32_t *scan, uint32_t *out) {
    uint32_t B = buckets_of(seg->d);
    for (uint32_t b = threadIdx.x; b <= B; b += blockDim.x) out[b] = bucket_start(*seg, scan, b, B) - seg->begin;
}

// ------------------------------------------------------------ host side

static int sm_count() {
    static const int n = [] {
        int dev = 0, c = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
        return c > 0 ? c : 1;
    }();
    return n;
}

#ifndef SS_C1_NT
#define SS_C1_NT 64     // threads of the CTA base case for 33..256 strings
#endif
#ifndef SS_C2_NT
#define SS_C2_NT 128    // .. for 257..1024 strings
#endif
#ifndef SS_C3_NT
#define SS_C3_NT 256    // .. for 1025..kSmallMax strings
#endif
#ifndef SS_BASE_CONCURRENT
#define SS_BASE_CONCURRENT 1
#endif

AuxStreams::AuxStreams() {
    ok = cudaStreamCreateWithFlags(&s[0], cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&s[1], cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; k < 3 && ok; k++) ok = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) cudaGetLastError();
}

AuxStreams &aux_streams() {
    static thread_local AuxStreams a;
    return a;
}

static std::atomic<bool> g_attrs_done[64];
static std::mutex g_attrs_mu;
// CTAs of each base-case class that are resident on the device at once
// (occupancy of its kernel times the SMs), set with the attributes
static uint32_t g_base_grid[2][kClasses];   // [some request compressed][class]

// runs f with std::true_type when some request of the call uses alphabet
// compression, with std::false_type otherwise (the kernels' template choice)
template <typename F>
static void with_alpha(bool any_alpha, F f) {
    if (any_alpha) f(std::true_type{});
    else f(std::false_type{});
}

template <bool A>
static cudaError_t base_attrs() {
    cudaError_t e;
    if ((e = set_smem_max(k_base_cta<SS_C1_NT, 256 / SS_C1_NT, A>, sizeof(BaseSmem<SS_C1_NT, 256 / SS_C1_NT>)))) return e;
    if ((e = set_smem_max(k_base_cta<SS_C2_NT, 1024 / SS_C2_NT, A>, sizeof(BaseSmem<SS_C2_NT, 1024 / SS_C2_NT>)))) return e;
    if ((e = set_smem_max(k_base_cta<SS_C3_NT, kSmallMax / SS_C3_NT, A>, sizeof(BaseSmem<SS_C3_NT, kSmallMax / SS_C3_NT>))))
        return e;
    g_base_grid[A][1] = resident_grid(k_base_cta<SS_C1_NT, 256 / SS_C1_NT, A>, SS_C1_NT, sizeof(BaseSmem<SS_C1_NT, 256 / SS_C1_NT>));
    g_base_grid[A][2] = resident_grid(k_base_cta<SS_C2_NT, 1024 / SS_C2_NT, A>, SS_C2_NT,
                                      sizeof(BaseSmem<SS_C2_NT, 1024 / SS_C2_NT>));
    g_base_grid[A][3] = resident_grid(k_base_cta<SS_C3_NT, kSmallMax / SS_C3_NT, A>, SS_C3_NT,
                                      sizeof(BaseSmem<SS_C3_NT, kSmallMax / SS_C3_NT>));
    return cudaSuccess;
}

template <typename K>
static uint32_t resident_grid(K kernel, int threads, size_t smem) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (uint32_t)per_sm * (uint32_t)(sms > 0 ? sms : 1);
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// kernels whose residency is limited by shared memory: the largest carveout
template <typename K>
static cudaError_t set_smem_max(K kernel, size_t bytes) {
    cudaError_t e = set_smem(kernel, bytes);
    if (e) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
}

static cudaError_t ensure_attrs() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && g_attrs_done[dev].load()) return cudaSuccess;
    std::lock_guard<std::mutex> lk(g_attrs_mu);
    cudaError_t e;
    if ((e = set_smem(k_build_trees, sizeof(TreeSmem)))) return e;
    if ((e = set_smem(k_pick_only, sizeof(TreeSmem)))) return e;
    if ((e = set_smem(k_classify<kLevelD>, sizeof(ClassifySmem<kLevelD>)))) return e;
    if ((e = set_smem(k_classify<kMaxD>, sizeof(ClassifySmem<kMaxD>)))) return e;
    if ((e = set_smem_max(k_scatter<MODE_SORT, kLevelD>, sizeof(ScatterSmem<kLevelD>)))) return e;
    if ((e = set_smem_max(k_scatter<MODE_CLASSIFY, kLevelD>, sizeof(ScatterSmem<kLevelD>)))) return e;
    if ((e = set_smem_max(k_scatter<MODE_CLASSIFY, kMaxD>, sizeof(ScatterSmem<kMaxD>)))) return e;
    if ((e = base_attrs<false>())) return e;
    if ((e = base_attrs<true>())) return e;
    if (dev < 64) g_attrs_done[dev] = true;
    return cudaSuccess;
}

// bump allocator over one scratch block
struct Carve {
    char *base;
    size_t off;
    template <typename T>
    T *take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T *p = reinterpret_cast<T *>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

static size_t carve_size(size_t N, uint32_t nreq, Caps &caps, size_t &np);

size_t engine_scratch_bytes(size_t N, uint32_t nreq) {
    Caps caps;
    size_t np;
    return carve_size(N, nreq, caps, np);
}

static size_t carve_size(size_t N, uint32_t nreq, Caps &caps, size_t &np) {
    caps.big = (uint32_t)(N / (kSmallMax + 1) + nreq + 1);
    for (int c = 0; c < kClasses; c++) {   // disjoint tasks of at least class_max(c - 1) + 1 strings
        size_t least = c == 0 ? 2 : class_max(c - 1) + 1;
        caps.small[c] = (uint32_t)(N / least + nreq + 1);
    }
    caps.bound = (uint32_t)(N + 1);
    // gather chunks of one level: buckets of more than kTinyMax strings, one
    // chunk per kGatherChunk of them
    caps.gather = (uint32_t)(N / (kTinyMax + 1) + N / kGatherChunk + nreq + 2);
    // sum over big segments of B * tiles <= 2047 (N / kTile + big) + 8 big
    caps.counts = (uint32_t)std::min<size_t>(0xFFFFFFF0ull, (size_t)kMaxB * ((size_t)N / kTile + caps.big) + (size_t)caps.big * 8 + 4096);
    np = caps.counts / kScanChunk + 2;
    Carve c{nullptr, 0};
    c.take<uint32_t>(N); c.take<uint32_t>(N);
    c.take<uint64_t>(N); c.take<uint64_t>(N);
    c.take<uint64_t>(N); c.take<uint64_t>(N);
    c.take<uint16_t>(N);
    c.take<uint32_t>(caps.counts);
    c.take<uint32_t>(np);
    c.take<uint64_t>((size_t)caps.big * kMaxV);
    c.take<uint16_t>((size_t)caps.big * kJumpStride);
    c.take<BigSeg>(caps.big); c.take<BigSeg>(caps.big);
    for (int k = 0; k < kClasses; k++) c.take<SmallTask>(caps.small[k]);
    c.take<Boundary>(caps.bound);
    c.take<GatherChunk>(caps.gather);
    c.take<uint32_t>(C_NUM);
    c.take<ReqDesc>(nreq);
    c.take<uint32_t>(nreq);
    c.take<uint4>(N / kPrefChunk + caps.big + 1);
    return c.off + 256;
}

static int check(cudaError_t e, const char *what) { return e == cudaSuccess ? SS_OK : cuda_fail(e, what); }

// exclusive scan of a[0 .. *n_dev), grid sized for n_bound >= *n_dev
static int launch_scan(uint32_t *a, uint32_t n_bound, const uint32_t *n_dev, uint32_t *partial, cudaStream_t st) {
    if (n_bound == 0) return SS_OK;
    uint32_t nb = (n_bound + kScanChunk - 1) / kScanChunk;
    SS_LAUNCH_U("scan_reduce", st, n_bound, k_scan_reduce<<<nb, kThreads, 0, st>>>(a, n_dev, partial));
    SS_LAUNCH_U("scan_partials", st, nb, k_scan_partials<<<1, 1024, 0, st>>>(partial, n_dev));
    SS_LAUNCH_U("scan_down", st, n_bound, k_scan_down<<<nb, kThreads, 0, st>>>(a, n_dev, partial));
    return check(cudaGetLastError(), "scan launch");
}

int engine_sort(const ReqDesc *reqs_in, uint32_t nreq, cudaStream_t st) {
    if (ensure_attrs() != cudaSuccess) return cuda_fail(cudaGetLastError(), "kernel attributes");
    std::vector<ReqDesc> reqs(reqs_in, reqs_in + nreq);
    uint64_t N64 = 0;
    for (auto &r : reqs) {
        r.base = (uint32_t)N64;
        N64 += r.n;
    }
    if (N64 > 0xFFFFFFFEull) {
        set_error_detail("total number of strings %llu exceeds 2^32 - 2", (unsigned long long)N64);
        return SS_ERR_TOO_LARGE;
    }
    const uint32_t N = (uint32_t)N64;
    if (N == 0) {
        for (auto &r : reqs)
            if (r.status_out) {
                int32_t ok = 0;
                cudaError_t e = cudaMemcpyAsync(r.status_out, &ok, 4, cudaMemcpyHostToDevice, st);
                if (e) return cuda_fail(e, "status write");
            }
        return check(cudaStreamSynchronize(st), "sync");
    }
    Caps caps;
    size_t np;
    size_t bytes = carve_size(N, nreq, caps, np);
    void *block = nullptr;
    cudaError_t e = scratch_alloc(&block, bytes, st);
    if (e != cudaSuccess) {
        set_error_detail("scratch allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        cudaGetLastError();
        return SS_ERR_OOM;
    }
    Carve c{(char *)block, 0};
    uint32_t *idx[2] = {c.take<uint32_t>(N), c.take<uint32_t>(N)};
    uint64_t *key[2] = {c.take<uint64_t>(N), c.take<uint64_t>(N)};
    uint64_t *soff[2] = {c.take<uint64_t>(N), c.take<uint64_t>(N)};
    ElemBufs eb;
    for (int p = 0; p < 2; p++) { eb.idx[p] = idx[p]; eb.soff[p] = soff[p]; eb.key[p] = key[p]; }
    uint16_t *obuf = c.take<uint16_t>(N);
    uint32_t *counts = c.take<uint32_t>(caps.counts);
    uint32_t *partial = c.take<uint32_t>(np);
    uint64_t *splitters = c.take<uint64_t>((size_t)caps.big * kMaxV);
    uint16_t *jt = c.take<uint16_t>((size_t)caps.big * kJumpStride);
    BigSeg *big[2] = {c.take<BigSeg>(caps.big), c.take<BigSeg>(caps.big)};
    TaskLists tl;
    for (int k = 0; k < kClasses; k++) {
        tl.l[k] = c.take<SmallTask>(caps.small[k]);
        tl.cap[k] = caps.small[k];
    }
    Boundary *bounds = c.take<Boundary>(caps.bound);
    GatherChunk *gchunks = c.take<GatherChunk>(caps.gather);
    uint32_t *counters = c.take<uint32_t>(C_NUM);
    ReqDesc *dreqs = c.take<ReqDesc>(nreq);
    uint32_t *shared = c.take<uint32_t>(nreq);   // characters shared by all strings of each large request
    uint4 *pchunks = c.take<uint4>(N / kPrefChunk + caps.big + 1);

    int rc = SS_OK;
    bool any_status = false;   // some request wants its status written on the device
    bool any_jump = false;     // some request classifies with jump tables
    bool any_alpha = false;    // some request uses alphabet compression
    for (const ReqDesc &q : reqs) {
        any_status = any_status || q.status_out;
        any_jump = any_jump || req_classifier(q) == CLS_JUMP;
        any_alpha = any_alpha || q.alpha;
    }
    // initial segments: one per request
    std::vector<BigSeg> big0;
    std::vector<SmallTask> s_task[kClasses];
    std::vector<uint4> pchunk_host;
    uint32_t tiles0 = 0, counts0 = 0, pairs0 = 0;
    for (uint32_t r = 0; r < nreq; r++) {
        const ReqDesc &q = reqs[r];
        if (q.n < 2) continue;
        if (q.n > kSmallMax) {
            BigSeg s{};
            s.begin = q.base; s.size = q.n; s.depth = 0; s.req = r;
            big0.push_back(s);
            uint32_t d = choose_d(q.n, req_child_target(q)), t = tiles_of(q.n), B = buckets_of(d);
            tiles0 += t; counts0 += B * t; pairs0 += B;
        } else {
            SmallTask t{q.base, q.n, 0, r, 0, 0};
            s_task[class_of(q.n)].push_back(t);
        }
    }
    uint32_t hcnt[C_NUM] = {0};
    uint32_t elems0 = 0;
    for (auto &s : big0) elems0 += s.size;
    for (int k = 0; k < kClasses; k++) {
        hcnt[C_NTASK + k] = (uint32_t)s_task[k].size();
        for (auto &t : s_task[k]) hcnt[C_ETASK + k] += t.size;
    }
#define TRY(x, what)                                     \
    do {                                                 \
        cudaError_t _e = (x);                            \
        if (_e != cudaSuccess) { rc = cuda_fail(_e, what); goto done; } \
    } while (0)
    for (const BigSeg &b : big0) {
        if (reqs[b.req].alpha) continue;   // compressed keys start at depth 0
        for (uint32_t x = 0; x < b.size; x += kPrefChunk)
            pchunk_host.push_back(make_uint4(b.begin + x, b.begin + std::min(b.size, x + kPrefChunk), b.req, 0));
    }
    // Everything the first launches read goes up from one pinned staging
    // buffer, asynchronously; the counter readbacks land in its own tail.
    uint32_t *hc;
    {
        size_t sz[4 + kClasses] = {sizeof(ReqDesc) * nreq, sizeof(hcnt), sizeof(BigSeg) * big0.size(),
                                   sizeof(uint4) * pchunk_host.size()};
        for (int k = 0; k < kClasses; k++) sz[4 + k] = sizeof(SmallTask) * s_task[k].size();
        size_t at[4 + kClasses + 1];
        at[0] = 0;
        for (int k = 0; k < 4 + kClasses; k++) at[k + 1] = at[k] + ((sz[k] + 15) & ~(size_t)15);
        char *up = (char *)host_staging(at[4 + kClasses] + sizeof(uint32_t) * C_NUM + 64);
        hc = (uint32_t *)(up + at[4 + kClasses]);
        memcpy(up + at[0], reqs.data(), sz[0]);
        memcpy(up + at[1], hcnt, sz[1]);
        if (sz[2]) memcpy(up + at[2], big0.data(), sz[2]);
        if (sz[3]) memcpy(up + at[3], pchunk_host.data(), sz[3]);
        for (int k = 0; k < kClasses; k++)
            if (sz[4 + k]) memcpy(up + at[4 + k], s_task[k].data(), sz[4 + k]);
        TRY(cudaMemcpyAsync(dreqs, up + at[0], sz[0], cudaMemcpyHostToDevice, st), "copy requests");
        TRY(cudaMemcpyAsync(counters, up + at[1], sz[1], cudaMemcpyHostToDevice, st), "copy counters");
        if (sz[2]) TRY(cudaMemcpyAsync(big[0], up + at[2], sz[2], cudaMemcpyHostToDevice, st), "copy big");
        if (sz[3]) TRY(cudaMemcpyAsync(pchunks, up + at[3], sz[3], cudaMemcpyHostToDevice, st), "copy chunks");
        for (int k = 0; k < kClasses; k++)
            if (sz[4 + k])
                TRY(cudaMemcpyAsync(tl.l[k], up + at[4 + k], sz[4 + k], cudaMemcpyHostToDevice, st), "copy base-case tasks");
    }
    {
        uint32_t grid = (uint32_t)std::min<uint64_t>((N + 255) / 256, (uint64_t)sm_count() * 8);
        with_alpha(any_alpha, [&](auto A) {
            SS_LAUNCH_U("init", st, N, k_init<decltype(A)::value><<<grid, 256, 0, st>>>(dreqs, nreq, N, idx[0], soff[0],
                                                                                        key[0], key[1]));
        });
        if (!pchunk_host.empty()) {
            const uint32_t nch = (uint32_t)pchunk_host.size();
            TRY(cudaMemsetAsync(shared, 0xFF, sizeof(uint32_t) * nreq, st), "reset shared prefix");
            SS_LAUNCH_U("shared_prefix", st, elems0, k_shared_prefix<<<nch, 256, 0, st>>>(pchunks, dreqs, key[0], shared));
            SS_LAUNCH_U("skip_prefix", st, elems0, k_skip_prefix<<<nch, 256, 0, st>>>(pchunks, key[1], key[0], shared));
            SS_LAUNCH_U("start_depth", st, big0.size(), k_start_depth<<<1, 256, 0, st>>>(big[0], (uint32_t)big0.size(), shared));
        }
        TRY(cudaGetLastError(), "init launch");
    }
    {
        uint32_t nbig = (uint32_t)big0.size(), ntiles = tiles0, ncounts = counts0, npairs = pairs0, nelems = elems0;
        uint32_t cur = 0;
        bool ran = false;
        while (nbig > 0) {
            ran = true;
            if (ncounts > caps.counts) {
                set_error_detail("internal: counters %u exceed capacity %u", ncounts, caps.counts);
                rc = SS_ERR_INTERNAL;
                goto done;
            }
            uint32_t nxt = cur ^ 1;
            // trees first: each chooses its depth; then the counter layout follows
            SS_LAUNCH_U("build_trees", st, nbig, k_build_trees<<<nbig, kThreads, sizeof(TreeSmem), st>>>(big[cur], dreqs, key[cur], splitters));
            SS_LAUNCH_U("setup_big", st, nbig, k_setup_big<<<1, 1024, 0, st>>>(big[cur], nbig, counters + C_LVL_COUNTS));
            if (any_jump)
                SS_LAUNCH_U("jump_tables", st, nbig, k_jump_tables<<<nbig, kThreads, 0, st>>>(big[cur], dreqs, splitters, jt));
            SS_LAUNCH_U("classify", st, nelems, k_classify<kLevelD><<<ntiles, kThreads, sizeof(ClassifySmem<kLevelD>), st>>>(
                big[cur], nbig, dreqs, 0u, key[cur], splitters, jt, obuf, counts));
            TRY(cudaGetLastError(), "classify launch");
            if ((rc = launch_scan(counts, ncounts, counters + C_LVL_COUNTS, partial, st)) != SS_OK) goto done;
            SS_LAUNCH_U("scatter", st, nelems, k_scatter<MODE_SORT, kLevelD><<<ntiles, kThreads, sizeof(ScatterSmem<kLevelD>), st>>>(
                big[cur], nbig, dreqs, idx[cur], soff[cur], key[cur], obuf, counts, splitters, idx[nxt], soff[nxt],
                key[nxt], counters));
            TRY(cudaMemsetAsync(counters + C_NBIG, 0, sizeof(uint32_t), st), "reset");
            TRY(cudaMemsetAsync(counters + C_TILES, 0, 3 * sizeof(uint32_t), st), "reset");
            TRY(cudaMemsetAsync(counters + C_ELEMS, 0, sizeof(uint32_t), st), "reset");
            TRY(cudaMemsetAsync(counters + C_NGATHER, 0, sizeof(uint32_t), st), "reset");
            SS_LAUNCH_U("buckets", st, npairs, k_buckets<<<(npairs + kThreads - 1) / kThreads, kThreads, 0, st>>>(
                big[cur], nbig, dreqs, counters + C_LVL_PAIRS, counts, splitters, nxt, big[nxt], tl, bounds, gchunks,
                caps, counters));
            with_alpha(any_alpha, [&](auto A) {
                SS_LAUNCH_U("gather_new", st, nelems, k_gather_new<decltype(A)::value><<<sm_count() * 8, 256, 0, st>>>(
                    gchunks, counters + C_NGATHER, dreqs, idx[nxt], soff[nxt], key[nxt]));
            });
            TRY(cudaGetLastError(), "level launch");
            TRY(cudaMemcpyAsync(hc, counters, sizeof(uint32_t) * C_NUM, cudaMemcpyDeviceToHost, st), "readback");
            TRY(cudaStreamSynchronize(st), "level sync");
            if (hc[C_ERROR]) break;
            nbig = hc[C_NBIG];
            ntiles = hc[C_TILES];
            ncounts = hc[C_COUNTS];
            npairs = hc[C_PAIRS];
            nelems = hc[C_ELEMS];
            cur = nxt;
        }
        // after a level the counters are fresh in hc; without one they are the host's own
        if (!ran) memcpy(hc, hcnt, sizeof(hcnt));
        if (hc[C_ERROR]) {
            set_error_detail("device-side check failed: code %u info %u", hc[C_ERROR], hc[C_ERRINFO]);
            rc = SS_ERR_INTERNAL;
            goto done;
        }
        uint32_t nb = hc[C_NBOUND];
        uint32_t sms = (uint32_t)sm_count();
        // CTA base cases first: they append their small equal-key groups to the
        // class-0 list, which the warp kernel then drains (count read on the device)
        SmallTask *const *L = tl.l;
        // the three CTA classes are independent: on side streams they overlap
        // each other's last waves; the warp kernel waits for all of them.  With
        // per-launch timing on they run one after another, so each kernel's time
        // is its own.
        AuxStreams &ax = aux_streams();
        const int nclasses = (hc[C_NTASK + 1] > 0) + (hc[C_NTASK + 2] > 0) + (hc[C_NTASK + 3] > 0);
        const bool fork = SS_BASE_CONCURRENT && nclasses > 1 && ax.ok && !prof_on();
        cudaStream_t s1 = fork ? ax.s[0] : st, s2 = fork ? ax.s[1] : st;
        if (fork) {
            TRY(cudaEventRecord(ax.ev[0], st), "fork");
            TRY(cudaStreamWaitEvent(s1, ax.ev[0], 0), "fork");
            TRY(cudaStreamWaitEvent(s2, ax.ev[0], 0), "fork");
        }
        // grids of the CTAs that fit on the device at once; each CTA takes its
        // tasks from the class's work queue (head in the counters)
        if (uint32_t n3 = hc[C_NTASK + 3]) {
            constexpr int NT = SS_C3_NT, IT = (int)(kSmallMax / SS_C3_NT);
            uint32_t grid = std::min<uint32_t>(n3, g_base_grid[any_alpha][3]);
            with_alpha(any_alpha, [&](auto A) {
                SS_LAUNCH_U("base_c3", st, hc[C_ETASK + 3],
                            (k_base_cta<NT, IT, decltype(A)::value><<<grid, NT, sizeof(BaseSmem<NT, IT>), st>>>(
                                L[3], counters + C_NTASK + 3, counters + C_QHEAD + 3, dreqs, eb, L[0], tl.cap[0],
                                counters)));
            });
        }
        if (uint32_t n2 = hc[C_NTASK + 2]) {
            constexpr int NT = SS_C2_NT, IT = (int)(1024 / SS_C2_NT);
            uint32_t grid = std::min<uint32_t>(n2, g_base_grid[any_alpha][2]);
            with_alpha(any_alpha, [&](auto A) {
                SS_LAUNCH_U("base_c2", s1, hc[C_ETASK + 2],
                            (k_base_cta<NT, IT, decltype(A)::value><<<grid, NT, sizeof(BaseSmem<NT, IT>), s1>>>(
                                L[2], counters + C_NTASK + 2, counters + C_QHEAD + 2, dreqs, eb, L[0], tl.cap[0],
                                counters)));
            });
        }
        if (uint32_t n1 = hc[C_NTASK + 1]) {
            constexpr int NT = SS_C1_NT, IT = (int)(256 / SS_C1_NT);
            uint32_t grid = std::min<uint32_t>(n1, g_base_grid[any_alpha][1]);
            with_alpha(any_alpha, [&](auto A) {
                SS_LAUNCH_U("base_c1", s2, hc[C_ETASK + 1],
                            (k_base_cta<NT, IT, decltype(A)::value><<<grid, NT, sizeof(BaseSmem<NT, IT>), s2>>>(
                                L[1], counters + C_NTASK + 1, counters + C_QHEAD + 1, dreqs, eb, L[0], tl.cap[0],
                                counters)));
            });
        }
        if (fork) {
            TRY(cudaEventRecord(ax.ev[1], s1), "join");
            TRY(cudaEventRecord(ax.ev[2], s2), "join");
            TRY(cudaStreamWaitEvent(st, ax.ev[1], 0), "join");
            TRY(cudaStreamWaitEvent(st, ax.ev[2], 0), "join");
        }
        if (hc[C_NTASK + 0] || hc[C_NTASK + 1] || hc[C_NTASK + 2] || hc[C_NTASK + 3]) {
            uint32_t grid = sms * 8;
            with_alpha(any_alpha, [&](auto A) {
                SS_LAUNCH_U("base_warp", st, hc[C_ETASK + 0], k_small_warp<decltype(A)::value><<<grid, kThreads, 0, st>>>(
                    L[0], counters + C_NTASK + 0, dreqs, eb));
            });
        }
        TRY(cudaGetLastError(), "base case launch");
        if (nb) {
            uint32_t grid = std::min<uint32_t>((nb + 255) / 256, sms * 8);
            with_alpha(any_alpha, [&](auto A) {
                SS_LAUNCH_U("boundary", st, nb, k_boundary<decltype(A)::value><<<grid, 256, 0, st>>>(bounds, nb, dreqs));
            });
            TRY(cudaGetLastError(), "boundary launch");
        }
        if (any_status) {
            SS_LAUNCH("status", st, k_status<<<(nreq + 255) / 256, 256, 0, st>>>(dreqs, nreq, 0));
            TRY(cudaGetLastError(), "status launch");
        }
        TRY(cudaMemcpyAsync(hc, counters, sizeof(uint32_t) * C_NUM, cudaMemcpyDeviceToHost, st), "readback");
        TRY(cudaStreamSynchronize(st), "final sync");
        if (hc[C_ERROR]) {
            set_error_detail("device-side check failed in the base case: code %u info %u", hc[C_ERROR], hc[C_ERRINFO]);
            rc = SS_ERR_INTERNAL;
            goto done;
        }
    }
done:
#undef TRY
    if (rc == SS_ERR_INTERNAL && any_status) {   // a device-side check failed: the requests learn it too
        k_status<<<(nreq + 255) / 256, 256, 0, st>>>(dreqs, nreq, rc);
        cudaStreamSynchronize(st);
    }
    scratch_free(block, st);
    return rc;
}

// ------------------------------------------------ single-step entry points

int engine_classify(const uint64_t *keys, uint32_t n, const uint64_t *x, uint32_t d, uint32_t classifier,
                    uint16_t *bucket_out, uint32_t *bucket_begin_out, uint32_t *order_out, cudaStream_t st) {
    if (ensure_attrs() != cudaSuccess) return cuda_fail(cudaGetLastError(), "kernel attributes");
    uint32_t v = (1u << d) - 1, B = 2 * v + 1;
    uint32_t tiles = tiles_of(n);
    uint32_t ncounts = B * tiles;
    uint32_t np = ncounts / kScanChunk + 2;
    size_t bytes = 0;
    Carve c0{nullptr, 0};
    c0.take<uint32_t>(ncounts); c0.take<uint32_t>(np); c0.take<uint64_t>(kMaxV); c0.take<uint16_t>(kJumpStride);
    c0.take<BigSeg>(1); c0.take<uint32_t>(C_NUM);
    bytes = c0.off + 256;
    void *block = nullptr;
    cudaError_t e = scratch_alloc(&block, bytes, st);
    if (e) { cudaGetLastError(); set_error_detail("scratch allocation failed"); return SS_ERR_OOM; }
    Carve c{(char *)block, 0};
    uint32_t *counts = c.take<uint32_t>(ncounts);
    uint32_t *partial = c.take<uint32_t>(np);
    uint64_t *spl = c.take<uint64_t>(kMaxV);
    uint16_t *jt = c.take<uint16_t>(kJumpStride);
    BigSeg *seg = c.take<BigSeg>(1);
    uint32_t *counters = c.take<uint32_t>(C_NUM);
    BigSeg s{};
    s.begin = 0; s.size = n; s.depth = 0; s.req = 0; s.d = d; s.tiles = tiles;
    s.tile_base = 0; s.cnt_base = 0; s.bkt_base = 0; s.scan_base = 0;
    int rc = SS_OK;
    uint32_t hcnt[C_NUM] = {0};
    hcnt[C_LVL_COUNTS] = ncounts;
    hcnt[C_LVL_PAIRS] = B;
    do {
        if ((e = cudaMemcpyAsync(seg, &s, sizeof(s), cudaMemcpyHostToDevice, st))) break;
        if ((e = cudaMemcpyAsync(spl, x, sizeof(uint64_t) * v, cudaMemcpyDeviceToDevice, st))) break;
        if ((e = cudaMemcpyAsync(counters, hcnt, sizeof(hcnt), cudaMemcpyHostToDevice, st))) break;
        if (n) {
            if (classifier == CLS_JUMP)
                SS_LAUNCH("jump_tables", st, k_jump_tables<<<1, kThreads, 0, st>>>(seg, nullptr, spl, jt));
            // the tree's depth picks the smallest kernel variant that holds it
            if (d <= (uint32_t)kLevelD) {
                SS_LAUNCH("classify", st, k_classify<kLevelD><<<tiles, kThreads, sizeof(ClassifySmem<kLevelD>), st>>>(
                    seg, 1, nullptr, classifier, keys, spl, jt, bucket_out, counts));
            } else {
                SS_LAUNCH("classify", st, k_classify<kMaxD><<<tiles, kThreads, sizeof(ClassifySmem<kMaxD>), st>>>(
                    seg, 1, nullptr, classifier, keys, spl, jt, bucket_out, counts));
            }
            if ((e = cudaGetLastError())) break;
            if ((rc = launch_scan(counts, ncounts, counters + C_LVL_COUNTS, partial, st)) != SS_OK) break;
            if (d <= (uint32_t)kLevelD) {
                SS_LAUNCH("scatter", st, k_scatter<MODE_CLASSIFY, kLevelD><<<tiles, kThreads, sizeof(ScatterSmem<kLevelD>), st>>>(
                    seg, 1, nullptr, nullptr, nullptr, nullptr, bucket_out, counts, spl, order_out, nullptr, nullptr, counters));
            } else {
                SS_LAUNCH("scatter", st, k_scatter<MODE_CLASSIFY, kMaxD><<<tiles, kThreads, sizeof(ScatterSmem<kMaxD>), st>>>(
                    seg, 1, nullptr, nullptr, nullptr, nullptr, bucket_out, counts, spl, order_out, nullptr, nullptr, counters));
            }
            if ((e = cudaGetLastError())) break;
            SS_LAUNCH("bucket_begin", st, k_bucket_begin<<<1, 256, 0, st>>>(seg, counts, bucket_begin_out));
        } else {
            if ((e = cudaMemsetAsync(bucket_begin_out, 0, sizeof(uint32_t) * (B + 1), st))) break;
        }
        if ((e = cudaGetLastError())) break;
        e = cudaStreamSynchronize(st);
    } while (0);
    if (e && rc == SS_OK) rc = cuda_fail(e, "classify");
    scratch_free(block, st);
    return rc;
}

int engine_splitters(const uint64_t *sample, uint32_t a, uint32_t d, uint64_t *x_out, cudaStream_t st) {
    if (ensure_attrs() != cudaSuccess) return cuda_fail(cudaGetLastError(), "kernel attributes");
    SS_LAUNCH("pick_only", st, k_pick_only<<<1, kThreads, sizeof(TreeSmem), st>>>(sample, a, d, x_out));
    cudaError_t e = cudaGetLastError();
    if (!e) e = cudaStreamSynchronize(st);
    return e ? cuda_fail(e, "splitters") : SS_OK;
}

int engine_gather(const ReqDesc &r, const uint32_t *depth, uint64_t *keys_out, cudaStream_t st) {
    if (r.n == 0) return SS_OK;
    uint32_t grid = std::min<uint32_t>((r.n + 255) / 256, (uint32_t)sm_count() * 8);
    SS_LAUNCH("gather", st, k_gather<<<grid, 256, 0, st>>>(r, depth, keys_out));
    cudaError_t e = cudaGetLastError();
    if (!e) e = cudaStreamSynchronize(st);
    return e ? cuda_fail(e, "gather") : SS_OK;
}

}  // namespace ss
