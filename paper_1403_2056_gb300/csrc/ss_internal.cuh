// Internal declarations of the GB300 string sample sorter.
//
// Layout in HBM during a sort (N = total strings of all requests):
//   idx[2][N]  u32  string index (request-local) per global position, double buffered
//   key[2][N]  u64  the 8 characters at the current depth of the element's segment
//   obuf[N]    u16  bucket of each element in the current level (the "oracle" array
//                   of Section 4.4; named bucket buffer here)
//   counts[]   u32  per (segment, bucket, tile) counters, bucket-major per segment
//   splitters  u64  in-order splitters of every big segment of the current level
//   lists      big segments (per level), small tasks and boundary records
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ss.h"

namespace ss {

// ---------------------------------------------------------------- tunables
constexpr int kThreads = 256;                  // CTA size of the tile kernels
constexpr int kWarps = kThreads / 32;
#ifndef SS_ITEMS
#define SS_ITEMS 16
#endif
#ifndef SS_MAX_D
#define SS_MAX_D 10
#endif
#ifndef SS_LEVEL_D
#define SS_LEVEL_D 8
#endif
constexpr int kItems = SS_ITEMS;               // elements per thread in a tile
constexpr int kTile = kThreads * kItems;       // 4096 elements per tile
constexpr int kWarpSpan = kTile / kWarps;      // 512 contiguous elements per warp
constexpr int kMaxD = SS_MAX_D;                // largest tree depth of any entry point: v = 2^d - 1 <= 1023
constexpr int kLevelD = SS_LEVEL_D;            // largest tree depth of a sort's levels: v <= 255
constexpr int kMaxV = (1 << kMaxD) - 1;
constexpr int kMaxB = 2 * kMaxV + 1;           // 2047 buckets
#ifndef SS_SMALL_MAX
#define SS_SMALL_MAX 2048
#endif
#ifndef SS_MIN_STEP
#define SS_MIN_STEP 5
#endif
#ifndef SS_CHILD_TARGET
#define SS_CHILD_TARGET 512
#endif
constexpr uint32_t kSmallMax = SS_SMALL_MAX;   // segments up to this size are base cases
constexpr uint32_t kChildTarget = SS_CHILD_TARGET;   // tree depth aims at children of about this size
constexpr uint32_t kTinyMax = 32;              // base cases handled by one warp
// base-case size classes: class 0 (2..32 strings) one warp; classes 1..3 one
// CTA each, holding up to 256, 1024 and kSmallMax strings
constexpr int kClasses = 4;
__host__ __device__ __forceinline__ uint32_t class_max(int c) {
    return c == 0 ? 32u : c == 1 ? 256u : c == 2 ? 1024u : kSmallMax;
}
__host__ __device__ __forceinline__ int class_of(uint32_t size) {
    return size <= 32u ? 0 : size <= 256u ? 1 : size <= 1024u ? 2 : 3;
}

// ------------------------------------------------------------ descriptors
struct ReqDesc {
    const uint8_t *chars;
    const uint64_t *offsets;
    const uint32_t *lengths;   // NULL: fixed_len or NUL-terminated
    uint32_t fixed_len;
    uint32_t n;
    uint32_t base;             // global position of the request's first element
    uint32_t tune;             // log2 child target (bits 0..7) | minimum depth step (bits 8..15) |
                               // classifier (bits 16..17) | largest tree depth of a level (bits 20..23) |
                               // log2 base-case threshold (bits 24..27); 0 fields: defaults
    uint32_t *perm_out;
    uint32_t *lcp_out;
    int32_t *status_out;
    uint32_t alpha;            // 0: keys of 8 bytes; else the sorted alphabet a0..a3 (bytes 0..3, a0 >= 1) of a
                               // fixed-length request: keys of 32 characters, 2 bits each (alphabet compression)
    uint64_t *off_out;         // NULL, or per sorted position: the string's offset,
    uint64_t *ck_out;          // 8 of its characters (byte keys) from depth ckd_out,
    uint32_t *ckd_out;         // where ckd_out <= its LCP < ckd_out + 8 (for a later LCP merge)
    uint32_t lvl1;             // set by the engine: the request's first level takes its string
                               // indices from the positions and its offsets from `offsets` itself
};

// The cache of R-local sorted position `local` (Section 5.4's distinguishing
// characters, handed to a later merge), written in two parts: put_ck where
// the position's LCP is decided (key = 8 characters from `depth`, depth <=
// LCP < depth + 8, or the string ends there; every string that can still end
// up at the position shares them), put_off where its string is (perm_out).
__device__ __forceinline__ void put_ck(const ReqDesc &R, uint32_t local, uint64_t key, uint32_t depth) {
    if (R.ck_out) {
        R.ck_out[local] = key;
        R.ckd_out[local] = depth;
    }
}
__device__ __forceinline__ void put_off(const ReqDesc &R, uint32_t local, uint64_t off) {
    if (R.off_out) R.off_out[local] = off;
}

// Per-request tuning: the segment size the tree depth aims at for children,
// and the smallest depth step an even bucket takes (0 fields: the defaults).
__host__ __device__ __forceinline__ uint32_t req_child_target(const ReqDesc &r) {
    const uint32_t s = r.tune & 0xFFu;
    return s ? (1u << s) : kChildTarget;
}
__host__ __device__ __forceinline__ uint32_t req_min_step(const ReqDesc &r) {
    const uint32_t m = (r.tune >> 8) & 0xFFu;
    return m ? m : (uint32_t)SS_MIN_STEP;
}
// Largest tree depth of a sort level (<= kLevelD) and the largest segment a
// base case takes (<= kSmallMax; larger segments get another level).
__host__ __device__ __forceinline__ uint32_t req_max_depth(const ReqDesc &r) {
    const uint32_t d = (r.tune >> 20) & 0xFu;
    return d ? d : (uint32_t)kLevelD;
}
__host__ __device__ __forceinline__ uint32_t req_small_max(const ReqDesc &r) {
    const uint32_t s = (r.tune >> 24) & 0xFu;
    return s ? (1u << s) : kSmallMax;
}

// How k_classify finds a key's bucket (every classifier gives the bucket of
// the closed form 2r + [x_r = c], r = #{j : x_j < c}, except that S5-Equal
// puts a key equal to a repeated splitter value into the equality bucket of
// the copy highest in the tree; the sorted result is the same):
//   CLS_UNROLL  descents with > only, four interleaved per thread, then one
//               equality test (S5-Unroll, Section 4.4's first alternative)
//   CLS_EQUAL   one descent per key with an equality test at every node,
//               leaving the tree at the first equal splitter (S5-Equal,
//               Section 4.4's fourth alternative)
//   CLS_JUMP    a table over the key bits that follow the splitters' shared
//               prefix gives the node where the descent starts to depend on
//               later bits (jump tables, Section 8.1), then as CLS_UNROLL
enum Classifier : uint32_t { CLS_UNROLL = 0, CLS_EQUAL = 1, CLS_JUMP = 2 };
__host__ __device__ __forceinline__ uint32_t req_classifier(const ReqDesc &r) { return (r.tune >> 16) & 0x3u; }
#ifndef SS_JUMP_BITS
#define SS_JUMP_BITS 10
#endif
constexpr int kJumpBits = SS_JUMP_BITS;            // 2^kJumpBits entries per jump table
constexpr int kJumpStride = (1 << kJumpBits) + 8;  // u16 per segment: the table, then the prefix length

struct BigSeg {                 // a segment sorted by one multi-CTA S5 step
    uint32_t begin, size, depth, req;
    uint32_t d, tiles;
    uint32_t tile_base, cnt_base, bkt_base, scan_base;
    uint32_t lvl1;              // 1: a request's first segment, positions are string indices and the
                                // string offsets are the request's own array (ReqDesc::lvl1)
    uint32_t pad1;
};

struct SmallTask {              // a base-case segment
    uint32_t begin, size, depth, req;
    uint32_t parity;            // which idx/key buffer holds it
    uint32_t gather;            // 1: the key buffer is stale, gather keys at `depth`
};

struct Boundary {               // lcp at global position pos is depth + lcp8(keys at depth)
    uint32_t pos, depth, req;
};

// device counters (one block of u32 per sort)
enum Counter : int {
    C_NBIG = 0,       // big segments emitted for the next level
    C_NBOUND = 1,     // boundary records
    C_ERROR = 2,      // first device-side error code (0 = none)
    C_TILES = 3,      // tiles of the next level's big segments
    C_COUNTS = 4,     // counters of the next level
    C_PAIRS = 5,      // (segment, bucket) pairs of the next level
    C_ERRINFO = 6,
    C_ELEMS = 7,      // strings in the next level's big segments
    C_LVL_COUNTS = 8, // counters of the current level (k_setup_big)
    C_LVL_PAIRS = 9,  // (segment, bucket) pairs of the current level
    C_NTASK = 10,     // base-case tasks of class c at C_NTASK + c
    C_ETASK = 14,     // their strings at C_ETASK + c
    C_QHEAD = 18,     // next task of class c's work queue at C_QHEAD + c
    C_NGATHER = 22,   // chunks of strings whose next key is gathered after the scatter
    C_NUM = 24
};

struct ElemBufs {               // per-position element arrays, double buffered by parity
    uint32_t *idx[2];           // string index (request-local)
    uint64_t *soff[2];          // byte offset of the string in its request's chars
    uint64_t *key[2];           // 8 characters at the segment's depth
};

struct TaskLists {              // base-case task lists by size class
    SmallTask *l[kClasses];
    uint32_t cap[kClasses];
};

enum DevError : uint32_t {
    E_NONE = 0,
    E_BIG_OVERFLOW = 1,
    E_SMALL_OVERFLOW = 2,
    E_BOUND_OVERFLOW = 3,
    E_BAD_BUCKET = 4,
    E_BAD_POS = 5,
    E_COPY_TIMEOUT = 6,   // a bulk copy into shared memory did not complete within its wait budget
    E_GATHER_OVERFLOW = 7,
    E_LAUNCH = 8,         // a launch from the device failed (info: the CUDA error)
};

struct Caps {                   // capacities of the scratch lists
    uint32_t big, bound, counts;
    uint32_t small[kClasses];
    uint32_t gather;            // gather chunks of one level
};

// a run of positions [begin, end) of one request whose keys are loaded anew at depth
struct GatherChunk {
    uint32_t begin, end, req, depth;
};
constexpr uint32_t kGatherChunk = 2048;   // positions per gather chunk

struct SortPlan {               // everything the scheduler launches with, by value
    const ReqDesc *reqs;
    uint32_t nreq, N;
    ElemBufs eb;
    uint16_t *obuf;
    uint32_t *counts, *partial;
    uint64_t *splitters;
    uint16_t *jt;
    BigSeg *big[2];
    TaskLists tl;
    Boundary *bounds;
    GatherChunk *gchunks;
    Caps caps;
    uint32_t *counters;
    uint32_t cur;               // parity of the level to run
    uint32_t levels;            // levels run so far
    uint32_t any_jump, any_status, sms;
    uint32_t any_cache;         // some request wants the caches of its sorted positions
    uint32_t base_grid[kClasses];
};

// ------------------------------------------------------------ device math
__device__ __forceinline__ uint64_t bswap64(uint64_t x) {
    uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
    uint32_t rlo = __byte_perm(lo, 0, 0x0123), rhi = __byte_perm(hi, 0, 0x0123);
    return ((uint64_t)rlo << 32) | rhi;
}

// per-byte zero flags (0x80 in each byte that is zero), exact (no carries)
__device__ __forceinline__ uint64_t zero_bytes(uint64_t x) {
    const uint64_t m = 0x7F7F7F7F7F7F7F7FULL;
    uint64_t t = (x & m) + m;
    return ~(t | x | m);
}

// number of leading non-zero bytes of a big-endian key (8 if none is zero)
__device__ __forceinline__ uint32_t nulpos(uint64_t key) {
    uint64_t z = zero_bytes(key);
    return z ? (uint32_t)(__clzll(z) >> 3) : 8u;
}

__device__ __forceinline__ bool has_zero(uint64_t key) { return zero_bytes(key) != 0; }

// common leading bytes of two keys (8 when equal)
__device__ __forceinline__ uint32_t lcp8(uint64_t a, uint64_t b) {
    uint64_t x = a ^ b;
    return x ? (uint32_t)(__clzll(x) >> 3) : 8u;
}

// 2-bit codes of 4 bytes (byte 0 = first character) against the sorted
// alphabet a0 <= a1 <= a2 (each replicated in 4 bytes): code = #{a_i < c},
// first character in bits 7..6
__device__ __forceinline__ uint32_t code8(uint32_t x, uint32_t a0, uint32_t a1, uint32_t a2) {
    const uint32_t m = (__vcmpgtu4(x, a0) & 0x01010101u) + (__vcmpgtu4(x, a1) & 0x01010101u) +
                       (__vcmpgtu4(x, a2) & 0x01010101u);
    return ((m & 3u) << 6) | ((m >> 4) & 0x30u) | ((m >> 14) & 0x0Cu) | ((m >> 24) & 0x03u);
}

// Alphabet-compressed key of a fixed-length string: characters [h, h + 32) as
// 2-bit codes, first character in the top bits; positions past the end get
// code 0, the same for every string of the request (all have the same length).
// Reads the aligned words that hold the characters, at most five.
__device__ __forceinline__ uint64_t load_key_packed(const ReqDesc &R, uint64_t off, uint32_t h) {
    const uint32_t L = R.fixed_len;
    if (h >= L) return 0ull;
    const uint32_t nb = min(32u, L - h);
    const uintptr_t a = (uintptr_t)(R.chars + off + h);
    const uint64_t *w = (const uint64_t *)(a & ~(uintptr_t)7);
    const uint32_t lead = (uint32_t)(a & 7), span = lead + nb, sh = 8 * lead;
    uint64_t W[5];
#pragma unroll
    for (int j = 0; j < 5; j++) W[j] = (uint32_t)(8 * j) < span ? __ldg(w + j) : 0ull;
    const uint32_t a0 = (R.alpha & 0xFFu) * 0x01010101u, a1 = ((R.alpha >> 8) & 0xFFu) * 0x01010101u,
                   a2 = ((R.alpha >> 16) & 0xFFu) * 0x01010101u;
    uint64_t key = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        uint64_t v = sh ? (W[i] >> sh) | (W[i + 1] << (64 - sh)) : W[i];   // bytes 8i .. 8i+7 of the window
        const int left = (int)nb - 8 * i;                                   // of which this many belong to the string
        if (left < 8) {
            const uint64_t keep = left <= 0 ? 0ull : (~0ull >> (64 - 8 * left));
            v = (v & keep) | ((uint64_t)a0 * 0x100000001ull & ~keep);      // past the end: code 0
        }
        key = (key << 16) | (code8((uint32_t)v, a0, a1, a2) << 8) | code8((uint32_t)(v >> 32), a0, a1, a2);
    }
    return key;
}

// chars_h: 8 bytes of string i (starting at byte `off` of chars) at depth h,
// big-endian, zero past the end.  Reads the aligned word holding byte h, and
// the next aligned word when the string continues into it.  For a terminated
// string that is known only once the first word has arrived, so the next word
// is read together with it whenever both lie in the same 4 KiB page (mapped
// whenever the first word is); bytes after the terminator are masked off.
__device__ __forceinline__ uint64_t load_key_o(const ReqDesc &R, uint32_t i, uint64_t off, uint32_t h) {
    uint64_t rem = ~0ULL;   // bytes of the string left from depth h (terminated: unknown)
    if (R.lengths) {
        uint32_t len = __ldg(R.lengths + i);
        if (h >= len) return 0;
        rem = len - h;
    } else if (R.fixed_len) {
        if (h >= R.fixed_len) return 0;
        rem = R.fixed_len - h;
    }
    const uint8_t *p = R.chars + off + h;
    uintptr_t a = (uintptr_t)p;
    const uint64_t *w = (const uint64_t *)(a & ~(uintptr_t)7);
    uint32_t sh = (uint32_t)(a & 7) * 8;
    // a known length decides the second word before the first arrives, and so
    // does a second word in the first one's page: both in flight
    const bool known = rem != ~0ULL;
    const bool same_page = ((uintptr_t)(w + 1) & 4095u) != 0;
    const bool ahead = sh && (known ? rem > (uint64_t)(8 - (a & 7)) : same_page);
    uint64_t w1 = ahead ? __ldg(w + 1) : 0ull;
    uint64_t w0 = __ldg(w);
    uint64_t v = w0 >> sh;   // memory bytes p[0 .. 8 - (a&7)) in the low bytes
    if (sh) {
        // terminated, second word in the next page: continue only if no 0 byte among the valid bytes
        if (!known && !same_page && !has_zero(v | (~0ULL << (64 - sh)))) w1 = __ldg(w + 1);
        v |= w1 << (64 - sh);
    }
    uint64_t key = bswap64(v);
    if (rem < 8) key &= ~0ULL << (8 * (8 - rem));
    uint64_t z = zero_bytes(key);
    if (z) {
        uint32_t k = (uint32_t)(__clzll(z) >> 3);   // first zero byte
        key &= k ? (~0ULL << (64 - 8 * k)) : 0ULL;
    }
    return key;
}

__device__ __forceinline__ uint64_t load_key(const ReqDesc &R, uint32_t i, uint32_t h) {
    return load_key_o(R, i, __ldg(R.offsets + i), h);
}

// keep the bytes of a big-endian key before byte k (k in 0..8)
__device__ __forceinline__ uint64_t keep_bytes(uint64_t key, uint32_t k) {
    return k >= 8 ? key : (k ? key & (~0ULL << (64 - 8 * k)) : 0ULL);
}

// chars_h for 16 characters: k0 = bytes [h, h+8), k1 = [h+8, h+16), zero past
// the end.  Each further aligned word is read when the string continues into
// it or, for a terminated string, ahead of that test when it lies in the first
// word's 4 KiB page, so no read touches a page the string does not.
__device__ __forceinline__ void load_key2_o(const ReqDesc &R, uint32_t i, uint64_t off, uint32_t h, uint64_t &k0,
                                            uint64_t &k1) {
    uint64_t rem = ~0ULL;
    if (R.lengths) {
        uint32_t len = __ldg(R.lengths + i);
        if (h >= len) { k0 = 0; k1 = 0; return; }
        rem = len - h;
    } else if (R.fixed_len) {
        if (h >= R.fixed_len) { k0 = 0; k1 = 0; return; }
        rem = R.fixed_len - h;
    }
    const uint8_t *p = R.chars + off + h;
    uintptr_t a = (uintptr_t)p;
    const uint64_t *w = (const uint64_t *)(a & ~(uintptr_t)7);
    const uint32_t sh = (uint32_t)(a & 7) * 8;
    const uint64_t avail0 = 8 - (a & 7);   // bytes of the string's window in the first word
    bool more1, more2;
    uint64_t w0, w1 = 0, w2 = 0;
    if (rem == ~0ULL) {
        const uintptr_t pg = (uintptr_t)w >> 12;
        const bool a1 = ((uintptr_t)(w + 1) >> 12) == pg;
        const bool a2 = sh && ((uintptr_t)(w + 2) >> 12) == pg;
        if (a1) w1 = __ldg(w + 1);
        if (a2) w2 = __ldg(w + 2);
        w0 = __ldg(w);
        more1 = !has_zero((w0 >> sh) | (sh ? (~0ULL << (64 - sh)) : 0ULL));
        if (more1 && !a1) w1 = __ldg(w + 1);
        more2 = more1 && sh && !has_zero(w1);
        if (more2 && !a2) w2 = __ldg(w + 2);
    } else {
        w0 = __ldg(w);
        more1 = rem > avail0;
        if (more1) w1 = __ldg(w + 1);
        more2 = sh && rem > avail0 + 8;
        if (more2) w2 = __ldg(w + 2);
    }
    uint64_t v0 = sh ? ((w0 >> sh) | (w1 << (64 - sh))) : w0;
    uint64_t v1 = sh ? ((w1 >> sh) | (w2 << (64 - sh))) : w1;
    k0 = bswap64(v0);
    k1 = bswap64(v1);
    if (rem < 16) {
        if (rem < 8) { k0 = keep_bytes(k0, (uint32_t)rem); k1 = 0; }
        else k1 = keep_bytes(k1, (uint32_t)(rem - 8));
    }
    uint64_t z0 = zero_bytes(k0);
    if (z0) {
        k0 = keep_bytes(k0, (uint32_t)(__clzll(z0) >> 3));
        k1 = 0;
    } else {
        uint64_t z1 = zero_bytes(k1);
        if (z1) k1 = keep_bytes(k1, (uint32_t)(__clzll(z1) >> 3));
    }
}

__device__ __forceinline__ void load_key2(const ReqDesc &R, uint32_t i, uint32_t h, uint64_t &k0, uint64_t &k1) {
    load_key2_o(R, i, __ldg(R.offsets + i), h, k0, k1);
}

// Keys of a request that may use alphabet compression.  Kernels that load keys
// take A = true only when some request of the call is compressed, so byte-key
// calls run code without the compressed path.
template <bool A>
__device__ __forceinline__ uint64_t key_at(const ReqDesc &R, uint32_t i, uint64_t off, uint32_t h) {
    if (A && R.alpha) return load_key_packed(R, off, h);
    return load_key_o(R, i, off, h);
}

// two consecutive keys: 16 bytes, or 64 compressed characters
template <bool A>
__device__ __forceinline__ void key2_at(const ReqDesc &R, uint32_t i, uint64_t off, uint32_t h, uint64_t &k0,
                                        uint64_t &k1) {
    if (A && R.alpha) {
        k0 = load_key_packed(R, off, h);
        k1 = load_key_packed(R, off, h + 32);
        return;
    }
    load_key2_o(R, i, off, h, k0, k1);
}

// ------------------------------------------------- key width of a request
// Characters per key: 8 bytes, or 32 two-bit codes for a request with an
// alphabet of at most four characters (alphabet compression, Section 8.1).
// Depths and LCPs stay in characters either way.
// With A = false the request is known to use byte keys (the kernel variant
// for calls without compressed requests), so no test of R.alpha is made.
template <bool A = true>
__host__ __device__ __forceinline__ uint32_t key_chars(const ReqDesc &R) { return (A && R.alpha) ? 32u : 8u; }

// characters two keys at the same depth have in common (key_chars if equal)
template <bool A = true>
__device__ __forceinline__ uint32_t key_lcp(const ReqDesc &R, uint64_t a, uint64_t b) {
    const uint64_t x = a ^ b;
    if (!x) return key_chars<A>(R);
    return (uint32_t)__clzll((long long)x) >> ((A && R.alpha) ? 1 : 3);
}

// the key of a string at `depth` reaches the string's end
template <bool A = true>
__device__ __forceinline__ bool key_ends(const ReqDesc &R, uint64_t key, uint32_t depth) {
    return (A && R.alpha) ? depth + 32u >= R.fixed_len : has_zero(key);
}

// characters of the string inside its key at `depth` (key_chars if it goes on)
template <bool A = true>
__device__ __forceinline__ uint32_t key_len(const ReqDesc &R, uint64_t key, uint32_t depth) {
    if (!(A && R.alpha)) return nulpos(key);
    return depth >= R.fixed_len ? 0u : min(32u, R.fixed_len - depth);
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {   // splitmix64 finaliser
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ void set_error(uint32_t *counters, uint32_t code, uint32_t info) {
    if (atomicCAS(counters + C_ERROR, 0u, code) == 0u) counters[C_ERRINFO] = info;
}

// ----------------------------------------- bulk copies into shared memory
// One-dimensional bulk copies (cp.async.bulk, the TMA unit's untiled form):
// global and shared addresses 16-byte aligned, size a multiple of 16, and
// completion counted in bytes on an mbarrier in shared memory.
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t arrivals) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(arrivals) : "memory");
}

// makes the initialisation of this thread's mbarriers visible to the bulk-copy unit
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// orders this thread's earlier shared-memory accesses before later bulk copies
// into shared memory (every thread that touched the space runs it, then a CTA
// barrier, then one thread issues the copy)
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// one arrival that also announces `bytes` of copies completing on the barrier
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_to_smem(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of the barrier to complete, for at most
// kCopyWaitCycles SM clock cycles (about a second); returns false when the
// budget ran out (the caller records E_COPY_TIMEOUT and skips the data).
constexpr long long kCopyWaitCycles = 2000000000ll;
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long budget = kCopyWaitCycles) {
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_test(bar, parity))
        if (clock64() - t0 > budget) return false;
    return true;
}

// ------------------------------------------------------- host-side helpers
void set_error_detail(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

// launch bookkeeping (profiling): begin/end around each library kernel launch
bool prof_on();   // per-launch timing is enabled

// Two side streams and three events per host thread (a server's workers each
// get their own), made on first use, for independent launches that may overlap.
struct AuxStreams {
    bool ok = false;
    cudaStream_t s[2] = {nullptr, nullptr};
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    AuxStreams();
};
AuxStreams &aux_streams();
void prof_begin(const char *name, cudaStream_t s);
void prof_end(const char *name, cudaStream_t s, uint64_t units);

// scratch memory from the library's stream-ordered pool
cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t s);
cudaError_t scratch_free(void *p, cudaStream_t s);

// pinned host staging buffer of the calling thread (at least `bytes`)
void *host_staging(size_t bytes);

// engine entry points (ss_engine.cu)
// async: levels driven by the device scheduler, the call returns at once
int engine_sort(const ReqDesc *reqs_host, uint32_t count, cudaStream_t stream, bool async = false);
size_t engine_scratch_bytes(size_t N, uint32_t nreq);
// the bytes of the first n strings of a fixed-length request, as a 256-bit
// set (mask[c / 32] bit c % 32); returns when done
int engine_byte_set(const ReqDesc &r, uint32_t n, uint32_t mask[8], cudaStream_t st);
int host_sort(const uint8_t *chars_host, uint64_t chars_len, const uint64_t *offsets_host, const uint32_t *lengths_host,
              uint32_t fixed_len, uint32_t n, uint32_t runs, uint32_t *perm_host, uint32_t *lcp_host, cudaStream_t st);
int engine_classify(const uint64_t *keys, uint32_t n, const uint64_t *x, uint32_t d, uint32_t classifier,
                    uint16_t *bucket_out, uint32_t *bucket_begin_out, uint32_t *order_out, cudaStream_t st);
int engine_splitters(const uint64_t *sample, uint32_t a, uint32_t d, uint64_t *x_out, cudaStream_t stream);
int engine_gather(const ReqDesc &r, const uint32_t *depth, uint64_t *keys_out, cudaStream_t stream);
// the device-driven level scheduler (ss_sched.cu): launches it for the sort the
// plan describes (its base_grid is filled there), and its device words
int sched_start(SortPlan plan, bool any_alpha, cudaStream_t stream);
uint64_t sched_device_launches();
void sched_reset_device_launches();
int32_t sched_take_device_error();
cudaError_t sched_copy_wait(long long budget_cycles, uint32_t withhold);
uint64_t engine_device_launches();        // kernels launched from the device so far
void engine_reset_device_launches();
int32_t engine_take_device_error();       // first device-side failure since the last take (0: none)
int engine_debug_copy_wait(long long budget_cycles, uint32_t withhold);
void *async_staging(size_t bytes, cudaStream_t stream, cudaEvent_t *done);

// merge methods (SS_MERGE_* of the C header)
enum MergeMethod : uint32_t { MERGE_PAIRWISE = 0, MERGE_LOSER_TREE = 1 };
constexpr uint32_t kKwayMaxRuns = 8;   // runs the loser-tree method merges in one pass
// one-pass K-way merge of 2..kKwayMaxRuns non-empty runs (ss_kway.cu)
int merge_kway(const ReqDesc &set, const uint32_t *run_perm, const uint32_t *run_lcp, const uint32_t *rb,
               const uint32_t *base, uint32_t R, uint32_t *perm_out, uint32_t *lcp_out, cudaStream_t stream);
size_t merge_kway_scratch(uint32_t total, uint32_t R, const uint32_t *rb);

// merge (ss_merge.cu)
// RunCache: the runs' string offsets and cached characters (run-aligned, as
// a sort writes them; see put_ck and put_off), or all NULL: computed by the merge
struct RunCache {
    const uint64_t *off;
    const uint64_t *ck;
    const uint32_t *ckd;
};
int merge_runs(const ReqDesc &set, const uint32_t *run_perm, const uint32_t *run_lcp, const uint32_t *run_begin_host,
               const uint32_t *run_base_host, uint32_t K, uint32_t *perm_out, uint32_t *lcp_out, cudaStream_t stream,
               uint32_t method = 0, RunCache cache = RunCache{nullptr, nullptr, nullptr});

}  // namespace ss

// launch with optional per-kernel timing; `units` = strings (or records)
// the launch processes, used to turn time into algorithmic bandwidth
#define SS_LAUNCH_U(name, stream, units, ...)    \
    do {                                         \
        ::ss::prof_begin(name, stream);          \
        __VA_ARGS__;                             \
        ::ss::prof_end(name, stream, (units));   \
    } while (0)
#define SS_LAUNCH(name, stream, ...) SS_LAUNCH_U(name, stream, 0, __VA_ARGS__)
