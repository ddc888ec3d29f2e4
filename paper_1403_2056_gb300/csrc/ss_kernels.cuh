// Device code of the GB300 string sample sorter: the per-level kernels, the
// base case (ss_base.cuh) and the device-driven level scheduler.  Included
// inside a namespace by two translation units: ss_engine.cu (whole-program
// compilation, the kernels the host launches) and ss_sched.cu (relocatable
// device code, SS_KERNELS_SCHEDULER = 1: the same kernels again plus the
// scheduler that launches them from the device).  The two copies share no
// device symbol.
#ifndef SS_KERNELS_SCHEDULER
#define SS_KERNELS_SCHEDULER 0
#endif

#include "ss_base.cuh"

// --------------------------------------------------------------- helpers

__host__ __device__ __forceinline__ uint32_t choose_d(uint32_t size, uint32_t target, uint32_t cap) {
    // v + 1 = 2^d about size / target, d in [2, cap], cap <= kLevelD
    uint32_t q = (size + target - 1) / target;
    uint32_t d = 0;
    while ((1u << d) < q) d++;
    if (d < 2) d = 2;
    if (d > cap) d = cap;
    return d;
}
__host__ __device__ __forceinline__ uint32_t req_choose_d(uint32_t size, const ReqDesc &r) {
    return choose_d(size, req_child_target(r), req_max_depth(r));
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
        if (!R.lvl1) {   // else the first level's scatter takes both from the request
            idx0[g] = i;
            soff0[g] = off;
        }
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

// The sample has alpha * v + alpha - 1 keys for the tree size the segment's
// length allows (choose_d), and every alpha-th sample key becomes a splitter.
// alpha = 2 while the tree can be as large as the segment asks for; when the
// depth cap holds the tree back (buckets of more than child_target strings on
// average) alpha grows to kAlphaCapped, so that the buckets are more even and
// fewer of them miss the base-case size by chance (a bucket of an alpha-sample
// splitter spans alpha sample gaps: its relative size has variance 1 / alpha).
// The tree actually built has just enough levels for the distinct keys of the
// sample (adaptivity, Section 8.1): a segment whose sample holds 27 distinct
// keys gets 31 splitters, not 1023.  The chosen depth is stored in the segment
// record; k_setup_big lays out the counters from it.
#ifndef SS_ALPHA_CAPPED
#define SS_ALPHA_CAPPED 8
#endif
constexpr uint32_t kAlphaCapped = SS_ALPHA_CAPPED;
static_assert(kAlphaCapped >= 2 && (kAlphaCapped & (kAlphaCapped - 1)) == 0 &&
                  kAlphaCapped * (1u << kLevelD) <= 2u * (kMaxV + 1),
              "the sample of a capped tree fits the tree builder's buffer");

__device__ __forceinline__ uint32_t sample_alpha(uint32_t size, uint32_t d, uint32_t target) {
    return size / target > (1u << d) ? kAlphaCapped : 2u;
}
__global__ void __launch_bounds__(kThreads) k_build_trees(BigSeg *segs, const ReqDesc *reqs, const uint64_t *key,
                                                           uint64_t *splitters) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TreeSmem &S = *reinterpret_cast<TreeSmem *>(smem_raw);
    __shared__ uint32_t distinct;
    BigSeg sg = segs[blockIdx.x];
    const uint32_t dmax = req_choose_d(sg.size, reqs[sg.req]);
    const uint32_t alpha = sample_alpha(sg.size, dmax, req_child_target(reqs[sg.req]));
    uint32_t v = (1u << dmax) - 1;
    uint32_t a = alpha * (v + 1) - 1;   // alpha * v + alpha - 1
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
// CTAs per SM the classifier's registers must allow: 4 (64 registers, the 16
// keys of a thread in flight) measured faster than the 2 that 95 registers
// leave room for
#ifndef SS_CLASSIFY_MINB
#define SS_CLASSIFY_MINB 4
#endif

template <int D>
__global__ void __launch_bounds__(kThreads, SS_CLASSIFY_MINB) k_classify(const BigSeg *__restrict__ segs, uint32_t nseg,
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

// SS_SCATTER_COMPACT = 1: the tile's string indices share the space the keys
// take later (about 16 KB less shared memory per CTA: with 64 registers 4
// CTAs fit per SM instead of 3), at the cost of issuing the key copy only
// once the indices are out; measured faster (no-LCP 64 Mi scatter 1.79 ->
// 1.67 ms, the others unchanged)
#ifndef SS_SCATTER_COMPACT
#define SS_SCATTER_COMPACT 1
#endif

template <int D>
struct ScatterSmem {
    static constexpr int MB = 2 * ((1 << D) - 1) + 1;   // buckets of a tree of depth D
#if SS_SCATTER_COMPACT
    union {
        struct {
            uint16_t wpos[kWarps][MB + 1];   // per warp: count, then running offset inside the tile's bucket
            alignas(16) uint32_t sidx[kTile + 8];   // the tile's string indices (range rounded out to 16 bytes)
        } r;
        uint64_t buf[kTile + 2];            // after the indices: the tile's keys, then its string offsets
    } u;
    __device__ uint16_t (*wpos())[MB + 1] { return u.r.wpos; }
    __device__ uint32_t *sidx() { return u.r.sidx; }
#else
    union {
        uint16_t wpos_[kWarps][MB + 1];   // per warp: count, then running offset inside the tile's bucket
        uint64_t buf[kTile + 2];            // after the ranks: the tile's keys, then its string offsets
    } u;
    uint32_t sidx_[kTile + 8];    // the tile's string indices (range rounded out to 16 bytes)
    __device__ uint16_t (*wpos())[MB + 1] { return u.wpos_; }
    __device__ uint32_t *sidx() { return sidx_; }
#endif
    uint32_t tbase[MB + 1];   // global position of each bucket's first string from this tile
    uint16_t lbase[MB + 1];   // tile-local start of each bucket (exclusive scan of the tile's counts)
    uint16_t binfo[MB + 1];   // delta | final << 6 | done << 7 | first tile << 8 | key length << 9
    uint16_t slot_b[kTile];      // bucket of each tile-local slot
    uint16_t src[kTile];         // tile element held by each slot
    uint32_t wcnt[kWarps];
    uint64_t bar[3];             // completion of the index, key and offset copies
};

#if SS_SCATTER_COMPACT
static_assert(offsetof(ScatterSmem<kMaxD>, u) % 16 == 0 && offsetof(ScatterSmem<kLevelD>, u) % 16 == 0 &&
                  alignof(ScatterSmem<kLevelD>) % 16 == 0,
              "bulk copy targets 16-byte aligned");
#else
static_assert(offsetof(ScatterSmem<kMaxD>, sidx_) % 16 == 0 && offsetof(ScatterSmem<kLevelD>, sidx_) % 16 == 0 &&
                  offsetof(ScatterSmem<kLevelD>, u) % 16 == 0,
              "bulk copy targets 16-byte aligned");
#endif
static_assert(offsetof(ScatterSmem<kMaxD>, bar) % 8 == 0 && offsetof(ScatterSmem<kLevelD>, bar) % 8 == 0,
              "mbarriers 8-byte aligned");

enum { MODE_SORT = 0, MODE_CLASSIFY = 1 };

// budget of every bulk-copy wait of the scatter (SM clock cycles); a test can
// shorten it and withhold the copies so that the waits run out
__device__ long long g_copy_wait_cycles = kCopyWaitCycles;
__device__ uint32_t g_copy_withheld;

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
#define SS_SCATTER_MINB (SS_SCATTER_COMPACT ? 4 : 2)
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
    // a request's first level: string index = position - base, offsets copied
    // from the request's 16-byte aligned array (tiles start at multiples of
    // kTile from its first string; the last 16-byte block is read whole)
    const bool lvl1 = MODE == MODE_SORT && sg.lvl1;

    const long long budget = g_copy_wait_cycles;
    const bool withheld = MODE == MODE_SORT && g_copy_withheld;   // test only: no copy is issued, the waits run out
    if (MODE == MODE_SORT && threadIdx.x == 0) {
        for (int k = 0; k < 3; k++) mbar_init(&S.bar[k], 1);
        fence_mbar_init();
        if (!withheld && !lvl1) {
            mbar_expect_tx(&S.bar[0], ibytes);
            bulk_to_smem(S.sidx(), idx_in + i0, ibytes, &S.bar[0]);
        }
    }
    // every bucket id of this thread in flight at once; kept in registers
    uint32_t bk[kItems];
#pragma unroll
    for (int u = 0; u < kItems; u++) {
        uint32_t p = wbeg + u * 32 + lane;
        bk[u] = p < seg_end ? (uint32_t)obuf[p] : 0xFFFFu;
    }
    for (uint32_t k = threadIdx.x; k < kWarps * (MB + 1) / 2; k += blockDim.x)
        reinterpret_cast<uint32_t *>(&S.wpos()[0][0])[k] = 0;
    __syncthreads();
    // phase A: per-warp bucket counts of its contiguous span, one shared atomic
    // per element on the 32-bit word holding the 16-bit count (a warp's span has
    // 512 elements, so a count never carries into its neighbour)
#pragma unroll
    for (int u = 0; u < kItems; u++)
        if (bk[u] != 0xFFFFu)
            atomicAdd(reinterpret_cast<uint32_t *>(&S.wpos()[warp][bk[u] & ~1u]), 1u << (16 * (bk[u] & 1u)));
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
                    uint32_t c = S.wpos()[w][b];
                    S.wpos()[w][b] = (uint16_t)run;
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
        uint32_t off = ok ? S.wpos()[warp][b] : 0u;
        const uint32_t lp = ok ? S.lbase[b] + off + rank : 0u;
        __syncwarp();
        if (ok && lane == (uint32_t)(__ffs(peers) - 1)) S.wpos()[warp][b] = (uint16_t)(off + __popc(peers));
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
    if (!SS_SCATTER_COMPACT && threadIdx.x == 0 && !withheld) {
        mbar_expect_tx(&S.bar[1], kbytes);
        bulk_to_smem(S.u.buf, key_in + k0, kbytes, &S.bar[1]);
    }
    // string indices; strings whose bucket is final go straight to the output
    if (!lvl1 && !__syncthreads_and(mbar_wait(&S.bar[0], 0, budget))) {
        if (threadIdx.x == 0) set_error(counters, E_COPY_TIMEOUT, tile);
        // the key copy in flight lands before the CTA leaves
        if (!SS_SCATTER_COMPACT && !withheld) mbar_wait(&S.bar[1], 0, budget);
        return;
    }
    const ReqDesc &R = reqs[sg.req];
    for (uint32_t s = threadIdx.x; s < tcount; s += kThreads) {
        const uint32_t b = S.slot_b[s];
        const uint32_t lo = s - S.lbase[b];
        const uint32_t q = S.tbase[b] + lo;
        if (q < sg.begin || q >= seg_end) { set_error(counters, E_BAD_POS, q); continue; }
        const uint32_t id = lvl1 ? tbeg - R.base + S.src[s] : S.sidx()[ioff + S.src[s]];
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
    if (SS_SCATTER_COMPACT) {   // the indices are out: their space takes the keys
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0 && !withheld) {
            mbar_expect_tx(&S.bar[1], kbytes);
            bulk_to_smem(S.u.buf, key_in + k0, kbytes, &S.bar[1]);
        }
    }
    // keys: the carried key where the depth stays (others are gathered later)
    if (!__syncthreads_and(mbar_wait(&S.bar[1], 0, budget))) {
        if (threadIdx.x == 0) set_error(counters, E_COPY_TIMEOUT, tile);
        return;
    }
    // a string of an all-equal complete bucket, not its first, has its LCP
    // from this key (a bucket's first gets its cache with its boundary LCP)
    auto done_not_first = [&](uint32_t info, uint32_t lo) {
        return (info & BI_DONE) && (!(info & BI_FIRST) || lo > 0);
    };
    for (uint32_t s = threadIdx.x; s < tcount; s += kThreads) {
        const uint32_t b = S.slot_b[s];
        const uint32_t info = S.binfo[b];
        const uint32_t q = S.tbase[b] + (s - S.lbase[b]);
        if (q < sg.begin || q >= seg_end) continue;
        if (info & BI_FIN) {
            if (done_not_first(info, s - S.lbase[b])) put_ck(R, q - R.base, S.u.buf[koff + S.src[s]], sg.depth);
            continue;
        }
        if (info & BI_DELTA) continue;   // a new depth: gathered later
        key_out[q] = S.u.buf[koff + S.src[s]];
    }
    fence_proxy_async();
    __syncthreads();   // every key read from the buffer: it takes the offsets next
    const uint32_t ooff = lvl1 ? 0u : koff;   // the offsets' place of the tile's first string in buf
    if (threadIdx.x == 0) {
        if (lvl1) {
            const uint32_t obytes = 8u * ((tcount + 1u) & ~1u);
            mbar_expect_tx(&S.bar[2], obytes);
            bulk_to_smem(S.u.buf, R.offsets + (tbeg - R.base), obytes, &S.bar[2]);
        } else {
            mbar_expect_tx(&S.bar[2], kbytes);
            bulk_to_smem(S.u.buf, soff_in + k0, kbytes, &S.bar[2]);
        }
    }
    if (!__syncthreads_and(mbar_wait(&S.bar[2], 0, budget))) {
        if (threadIdx.x == 0) set_error(counters, E_COPY_TIMEOUT, tile);
        return;
    }
    for (uint32_t s = threadIdx.x; s < tcount; s += kThreads) {
        const uint32_t b = S.slot_b[s];
        const uint32_t info = S.binfo[b];
        const uint32_t q = S.tbase[b] + (s - S.lbase[b]);
        if (q < sg.begin || q >= seg_end) continue;
        if (info & BI_FIN) {   // placed now: its string's offset
            put_off(R, q - R.base, S.u.buf[ooff + S.src[s]]);
            continue;
        }
        soff_out[q] = S.u.buf[ooff + S.src[s]];
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
    if (size > req_small_max(reqs[sg.req])) {
        uint32_t k = atomicAdd(counters + C_NBIG, 1u);
        if (k < caps.big) {
            BigSeg c{};
            c.begin = st; c.size = size; c.depth = depth; c.req = sg.req;
            next_big[k] = c;
            uint32_t d = req_choose_d(size, reqs[sg.req]), t = tiles_of(size), Bc = buckets_of(d);
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
                                                    const uint64_t *__restrict__ soff, uint64_t *__restrict__ key,
                                                    const uint32_t *counters) {
    // a failed scatter leaves positions unwritten: their indices must not be followed
    if (((volatile const uint32_t *)counters)[C_ERROR]) return;
    const uint32_t nch = *nchunks_dev;
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
        const GatherChunk g = gchunks[c];
        const ReqDesc &R = reqs[g.req];
        const bool by_index = R.lengths != nullptr;   // only explicit lengths need the string index
        constexpr int U = kGatherChunk / 256;
        uint32_t id[U];
        uint64_t so[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint32_t p = g.begin + u * 256 + threadIdx.x;
            id[u] = p < g.end && by_index ? idx[p] : 0u;
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
__global__ void k_boundary(const Boundary *bounds, uint32_t nb, const ReqDesc *reqs, uint32_t nfirst) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x) {
        Boundary b = bounds[k];
        const ReqDesc &R = reqs[b.req];
        uint32_t lp = b.pos - R.base;
        uint32_t sa = R.perm_out[lp - 1], sb = R.perm_out[lp];
        uint64_t ka = key_at<A>(R, sa, __ldg(R.offsets + sa), b.depth), kb = key_at<A>(R, sb, __ldg(R.offsets + sb), b.depth);
        R.lcp_out[lp] = b.depth + key_lcp<A>(R, ka, kb);
        put_ck(R, lp, kb, b.depth);
    }
    // with caches: the first position of every request (LCP 0), keys at depth 0
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nfirst; k += gridDim.x * blockDim.x) {
        const ReqDesc &R = reqs[k];
        if (!R.ck_out || R.n == 0) continue;
        const uint32_t s0 = R.perm_out[0];
        const uint64_t o0 = __ldg(R.offsets + s0);
        put_ck(R, 0, key_at<A>(R, s0, o0, 0), 0);
        put_off(R, 0, o0);
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


#if SS_KERNELS_SCHEDULER
// ------------------------------------------------------ device-driven levels
// A sort's recursion runs without the host: after the first launches, one
// single-thread scheduler grid reads the device counters of the level about
// to run, resets them for the level's own k_buckets, and tail-launches the
// level's kernels with grids sized from those counts, then itself for the
// next level (tail launches start in order, each after the grid before it
// and all work that grid launched).  When no big segment is left it launches
// the three CTA base-case classes side by side (fire-and-forget), then the
// warp class after all of them, the boundary LCPs and the status of every
// request.  The segment lists and the base-case task lists are the device
// work queue; the host only allocates, uploads the first lists and queues
// the first grids, so a sort call returns before the sort is done.



// first device-side failure of any sort (SS_* code), read and cleared by ss_device_error
__device__ int32_t g_device_error;
// kernels launched from the device, added to ss_launch_count
__device__ unsigned long long g_device_launches;

__device__ __forceinline__ int32_t status_of(uint32_t dev_error) {
    return dev_error == 0 ? SS_OK : dev_error == E_COPY_TIMEOUT ? SS_ERR_TIMEOUT : SS_ERR_INTERNAL;
}

// status of every request; the call's device error, if any, for ss_device_error
__global__ void k_finish(const ReqDesc *reqs, uint32_t nreq, const uint32_t *counters, uint32_t any_status) {
    const int32_t code = status_of(counters[C_ERROR]);
    if (any_status)
        for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nreq; r += gridDim.x * blockDim.x)
            if (reqs[r].status_out) *reqs[r].status_out = code;
    if (code != SS_OK && blockIdx.x == 0 && threadIdx.x == 0) atomicCAS((int *)&g_device_error, 0, code);
}

__device__ __forceinline__ void note_launch(uint32_t *counters) {
    atomicAdd(&g_device_launches, 1ull);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) set_error(counters, E_LAUNCH, (uint32_t)e);
}

template <bool A>
__global__ void k_sched(SortPlan P) {
    if (threadIdx.x != 0) return;
    uint32_t *c = P.counters;
    cudaStream_t TL = cudaStreamTailLaunch, FF = cudaStreamFireAndForget;
    const uint32_t fin_grid = (P.nreq + 255) / 256;
    if (c[C_ERROR] == 0 && c[C_NBIG] > 0) {
        const uint32_t nbig = c[C_NBIG], ntiles = c[C_TILES], ncounts = c[C_COUNTS], npairs = c[C_PAIRS],
                       nelems = c[C_ELEMS];
        if (ncounts > P.caps.counts || nbig > P.caps.big) {
            set_error(c, E_BIG_OVERFLOW, ncounts);
            k_finish<<<fin_grid, 256, 0, TL>>>(P.reqs, P.nreq, c, P.any_status);
            note_launch(c);
            return;
        }
        (void)nelems;
        // the level's counts are read: its k_buckets counts the next level from zero
        c[C_NBIG] = 0; c[C_TILES] = 0; c[C_COUNTS] = 0; c[C_PAIRS] = 0; c[C_ELEMS] = 0; c[C_NGATHER] = 0;
        const uint32_t cur = P.cur, nxt = cur ^ 1u;
        k_build_trees<<<nbig, kThreads, sizeof(TreeSmem), TL>>>(P.big[cur], P.reqs, P.eb.key[cur], P.splitters);
        note_launch(c);
        k_setup_big<<<1, 1024, 0, TL>>>(P.big[cur], nbig, c + C_LVL_COUNTS);
        note_launch(c);
        if (P.any_jump) {
            k_jump_tables<<<nbig, kThreads, 0, TL>>>(P.big[cur], P.reqs, P.splitters, P.jt);
            note_launch(c);
        }
        k_classify<kLevelD><<<ntiles, kThreads, sizeof(ClassifySmem<kLevelD>), TL>>>(
            P.big[cur], nbig, P.reqs, 0u, P.eb.key[cur], P.splitters, P.jt, P.obuf, P.counts);
        note_launch(c);
        const uint32_t nb = (ncounts + kScanChunk - 1) / kScanChunk;
        if (nb) {
            k_scan_reduce<<<nb, kThreads, 0, TL>>>(P.counts, c + C_LVL_COUNTS, P.partial);
            note_launch(c);
            k_scan_partials<<<1, 1024, 0, TL>>>(P.partial, c + C_LVL_COUNTS);
            note_launch(c);
            k_scan_down<<<nb, kThreads, 0, TL>>>(P.counts, c + C_LVL_COUNTS, P.partial);
            note_launch(c);
        }
        k_scatter<MODE_SORT, kLevelD><<<ntiles, kThreads, sizeof(ScatterSmem<kLevelD>), TL>>>(
            P.big[cur], nbig, P.reqs, P.eb.idx[cur], P.eb.soff[cur], P.eb.key[cur], P.obuf, P.counts, P.splitters,
            P.eb.idx[nxt], P.eb.soff[nxt], P.eb.key[nxt], c);
        note_launch(c);
        k_buckets<<<(npairs + kThreads - 1) / kThreads, kThreads, 0, TL>>>(
            P.big[cur], nbig, P.reqs, c + C_LVL_PAIRS, P.counts, P.splitters, nxt, P.big[nxt], P.tl, P.bounds, P.gchunks,
            P.caps, c);
        note_launch(c);
        k_gather_new<A><<<P.sms * 8, 256, 0, TL>>>(P.gchunks, c + C_NGATHER, P.reqs, P.eb.idx[nxt], P.eb.soff[nxt],
                                                  P.eb.key[nxt], c);
        note_launch(c);
        SortPlan Q = P;
        Q.cur = nxt;
        Q.levels = P.levels + 1;
        k_sched<A><<<1, 32, 0, TL>>>(Q);
        note_launch(c);
        return;
    }
    if (c[C_ERROR] == 0) {
        // base cases: the CTA classes side by side, each from its work queue
        if (const uint32_t n3 = c[C_NTASK + 3]) {
            constexpr int NT = SS_C3_NT, IT = (int)(kSmallMax / SS_C3_NT);
            k_base_cta<NT, IT, A><<<min(n3, P.base_grid[3]), NT, sizeof(BaseSmem<NT, IT>), FF>>>(
                P.tl.l[3], c + C_NTASK + 3, c + C_QHEAD + 3, P.reqs, P.eb, P.tl.l[0], P.tl.cap[0], c);
            note_launch(c);
        }
        if (const uint32_t n2 = c[C_NTASK + 2]) {
            constexpr int NT = SS_C2_NT, IT = (int)(1024 / SS_C2_NT);
            k_base_cta<NT, IT, A><<<min(n2, P.base_grid[2]), NT, sizeof(BaseSmem<NT, IT>), FF>>>(
                P.tl.l[2], c + C_NTASK + 2, c + C_QHEAD + 2, P.reqs, P.eb, P.tl.l[0], P.tl.cap[0], c);
            note_launch(c);
        }
        if (const uint32_t n1 = c[C_NTASK + 1]) {
            constexpr int NT = SS_C1_NT, IT = (int)(256 / SS_C1_NT);
            k_base_cta<NT, IT, A><<<min(n1, P.base_grid[1]), NT, sizeof(BaseSmem<NT, IT>), FF>>>(
                P.tl.l[1], c + C_NTASK + 1, c + C_QHEAD + 1, P.reqs, P.eb, P.tl.l[0], P.tl.cap[0], c);
            note_launch(c);
        }
        // after all three (and the groups they hand over): the warp class, then boundaries
        k_small_warp<A><<<P.sms * 8, kThreads, 0, TL>>>(P.tl.l[0], c + C_NTASK + 0, P.reqs, P.eb);
        note_launch(c);
        const uint32_t nbd = c[C_NBOUND], nfirst = P.any_cache ? P.nreq : 0u;
        if (nbd || nfirst) {
            k_boundary<A><<<min((max(nbd, nfirst) + 255) / 256, P.sms * 8), 256, 0, TL>>>(P.bounds, nbd, P.reqs, nfirst);
            note_launch(c);
        }
    }
    k_finish<<<fin_grid, 256, 0, TL>>>(P.reqs, P.nreq, c, P.any_status);
    note_launch(c);
}

#endif  // SS_KERNELS_SCHEDULER
