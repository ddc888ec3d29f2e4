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

namespace ss {

#include "ss_kernels.cuh"

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

static size_t carve_size(size_t N, uint32_t nreq, uint32_t min_small, Caps &caps, size_t &np);

size_t engine_scratch_bytes(size_t N, uint32_t nreq) {
    Caps caps;
    size_t np;
    return carve_size(N, nreq, kSmallMax, caps, np);
}

// min_small: the smallest base-case threshold of the requests (a big segment
// holds more strings than its request's threshold)
static size_t carve_size(size_t N, uint32_t nreq, uint32_t min_small, Caps &caps, size_t &np) {
    caps.big = (uint32_t)(N / (min_small + 1) + nreq + 1);
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

// Pinned staging for sorts the host does not wait for: a ring of slots per
// host thread, each reused only after the copies queued from it are done
// (an event per slot), so the host blocks only when it is a whole ring ahead.
struct StagingRing {
    static constexpr int kSlots = 8;
    void *buf[kSlots] = {};
    size_t cap[kSlots] = {};
    cudaEvent_t ev[kSlots] = {};
    bool used[kSlots] = {};
    int next = 0;
    ~StagingRing() {
        for (int k = 0; k < kSlots; k++) {
            if (buf[k]) cudaFreeHost(buf[k]);
            if (ev[k]) cudaEventDestroy(ev[k]);
        }
    }
};

void *async_staging(size_t bytes, cudaStream_t, cudaEvent_t *done) {
    static thread_local StagingRing ring;
    const int k = ring.next;
    ring.next = (ring.next + 1) % StagingRing::kSlots;
    if (!ring.ev[k] && cudaEventCreateWithFlags(&ring.ev[k], cudaEventDisableTiming) != cudaSuccess) return nullptr;
    if (ring.used[k] && cudaEventSynchronize(ring.ev[k]) != cudaSuccess) return nullptr;
    if (ring.cap[k] < bytes) {
        if (ring.buf[k]) cudaFreeHost(ring.buf[k]);
        ring.buf[k] = nullptr;
        ring.cap[k] = 0;
        size_t c = 1 << 16;
        while (c < bytes) c <<= 1;
        if (cudaHostAlloc(&ring.buf[k], c, cudaHostAllocDefault) != cudaSuccess) return nullptr;
        ring.cap[k] = c;
    }
    ring.used[k] = true;
    *done = ring.ev[k];
    return ring.buf[k];
}

int engine_sort(const ReqDesc *reqs_in, uint32_t nreq, cudaStream_t st, bool async) {
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
    uint32_t min_small = kSmallMax;
    for (const auto &r : reqs) min_small = std::min(min_small, req_small_max(r));
    size_t bytes = carve_size(N, nreq, min_small, caps, np);
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
    cudaEvent_t stage_done = nullptr;   // the staging ring slot's copies are done
    bool any_status = false;   // some request wants its status written on the device
    bool any_jump = false;     // some request classifies with jump tables
    bool any_alpha = false;    // some request uses alphabet compression
    bool any_cache = false;    // some request wants the caches of its sorted positions
    for (const ReqDesc &q : reqs) {
        any_status = any_status || q.status_out;
        any_jump = any_jump || req_classifier(q) == CLS_JUMP;
        any_alpha = any_alpha || q.alpha;
        any_cache = any_cache || q.ck_out;
    }
    // initial segments: one per request
    std::vector<BigSeg> big0;
    std::vector<SmallTask> s_task[kClasses];
    std::vector<uint4> pchunk_host;
    uint32_t tiles0 = 0, counts0 = 0, pairs0 = 0;
    for (uint32_t r = 0; r < nreq; r++) {
        ReqDesc &q = reqs[r];
        if (q.n < 2) continue;
        if (q.n > req_small_max(q)) {
            // a 16-byte aligned offsets array is copied straight into the first
            // level's scatter: k_init writes no index or offset for the request
            q.lvl1 = ((uintptr_t)q.offsets & 15u) == 0 ? 1u : 0u;
            BigSeg s{};
            s.begin = q.base; s.size = q.n; s.depth = 0; s.req = r; s.lvl1 = q.lvl1;
            big0.push_back(s);
            uint32_t d = req_choose_d(q.n, q), t = tiles_of(q.n), B = buckets_of(d);
            tiles0 += t; counts0 += B * t; pairs0 += B;
        } else {
            SmallTask t{q.base, q.n, 0, r, 0, 0};
            s_task[class_of(q.n)].push_back(t);
        }
    }
    uint32_t hcnt[C_NUM] = {0};
    uint32_t elems0 = 0;
    for (auto &s : big0) elems0 += s.size;
    // the first level's counts, where the device scheduler reads every level's
    hcnt[C_NBIG] = (uint32_t)big0.size();
    hcnt[C_TILES] = tiles0;
    hcnt[C_COUNTS] = counts0;
    hcnt[C_PAIRS] = pairs0;
    hcnt[C_ELEMS] = elems0;
    // Levels driven by the device scheduler when the caller asked for an
    // asynchronous sort: the call returns at once and no host round trip
    // separates the levels.  Otherwise the host drives them, queueing each
    // level's launches back to back, which measured faster on GB300 at every
    // size (grids launched from the device start about 12 us after the one
    // before and ran slower).  Per-launch timing (events recorded by the host
    // around every launch) also drives the levels from the host.
    const bool device_levels = async && !prof_on();
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
        // the host does not wait for a device-driven sort: its staging buffer is
        // taken from a ring whose slots are reused only once their copies are done
        const size_t stage_bytes = at[4 + kClasses] + sizeof(uint32_t) * C_NUM + 64;
        char *up = (char *)(device_levels ? async_staging(stage_bytes, st, &stage_done) : host_staging(stage_bytes));
        if (!up) { rc = cuda_fail(cudaGetLastError(), "pinned staging"); goto done; }
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
        if (stage_done) TRY(cudaEventRecord(stage_done, st), "staging event");
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
    if (device_levels) {
        SortPlan P;
        memset(&P, 0, sizeof(P));
        P.reqs = dreqs;
        P.nreq = nreq;
        P.N = N;
        P.eb = eb;
        P.obuf = obuf;
        P.counts = counts;
        P.partial = partial;
        P.splitters = splitters;
        P.jt = jt;
        P.big[0] = big[0];
        P.big[1] = big[1];
        P.tl = tl;
        P.bounds = bounds;
        P.gchunks = gchunks;
        P.caps = caps;
        P.counters = counters;
        P.cur = 0;
        P.any_jump = any_jump;
        P.any_status = any_status;
        P.any_cache = any_cache;
        P.sms = (uint32_t)sm_count();
        if ((rc = sched_start(P, any_alpha, st)) != SS_OK) goto done;
        scratch_free(block, st);   // stream-ordered: after the last grid the scheduler launches
        return SS_OK;
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
                    gchunks, counters + C_NGATHER, dreqs, idx[nxt], soff[nxt], key[nxt], counters));
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
            rc = hc[C_ERROR] == E_COPY_TIMEOUT ? SS_ERR_TIMEOUT : SS_ERR_INTERNAL;
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
        const uint32_t nfirst = any_cache ? nreq : 0u;
        if (nb || nfirst) {
            uint32_t grid = std::min<uint32_t>((std::max(nb, nfirst) + 255) / 256, sms * 8);
            with_alpha(any_alpha, [&](auto A) {
                SS_LAUNCH_U("boundary", st, nb, k_boundary<decltype(A)::value><<<grid, 256, 0, st>>>(bounds, nb, dreqs, nfirst));
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
    if ((rc == SS_ERR_INTERNAL || rc == SS_ERR_TIMEOUT) && any_status) {   // a device-side failure: the requests learn it too
        k_status<<<(nreq + 255) / 256, 256, 0, st>>>(dreqs, nreq, rc);
        cudaStreamSynchronize(st);
    }
    scratch_free(block, st);
    return rc;
}

// --------------------------------------------- device words of the engine

uint64_t engine_device_launches() { return sched_device_launches(); }

void engine_reset_device_launches() { sched_reset_device_launches(); }

int32_t engine_take_device_error() { return sched_take_device_error(); }

// the wait budget and the withheld copies, in both copies of the kernels
int engine_debug_copy_wait(long long budget, uint32_t withhold) {
    const long long b = budget > 0 ? budget : kCopyWaitCycles;
    cudaError_t e = cudaMemcpyToSymbol(g_copy_wait_cycles, &b, sizeof(b));
    if (!e) e = cudaMemcpyToSymbol(g_copy_withheld, &withhold, sizeof(withhold));
    if (!e) e = sched_copy_wait(b, withhold);
    return e ? cuda_fail(e, "ss_debug_copy_wait") : SS_OK;
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

// byte set of the first n strings of a fixed-length request (the autotuner's
// alphabet test): one string per thread, the warp's sets OR-ed together
__global__ void __launch_bounds__(256) k_byte_set(ReqDesc r, uint32_t n, uint32_t *mask) {
    uint32_t m[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint8_t *p = r.chars + r.offsets[i];
        for (uint32_t j = 0; j < r.fixed_len; j++) {
            const uint32_t c = p[j];
            m[c >> 5] |= 1u << (c & 31);
        }
    }
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const uint32_t v = __reduce_or_sync(0xffffffffu, m[k]);
        if ((threadIdx.x & 31) == 0 && v) atomicOr(mask + k, v);
    }
}

int engine_byte_set(const ReqDesc &r, uint32_t n, uint32_t mask[8], cudaStream_t st) {
    for (int k = 0; k < 8; k++) mask[k] = 0;
    if (n == 0 || r.fixed_len == 0 || r.lengths) return SS_OK;
    void *block = nullptr;
    cudaError_t e = scratch_alloc(&block, 256, st);
    if (e) {
        cudaGetLastError();
        set_error_detail("byte set: scratch allocation failed");
        return SS_ERR_OOM;
    }
    uint32_t *d_mask = (uint32_t *)block;
    uint32_t grid = std::min<uint32_t>((n + 255) / 256, (uint32_t)sm_count() * 8);
    do {
        if ((e = cudaMemsetAsync(d_mask, 0, 32, st))) break;
        SS_LAUNCH("byte_set", st, k_byte_set<<<grid, 256, 0, st>>>(r, n, d_mask));
        if ((e = cudaGetLastError())) break;
        if ((e = cudaMemcpyAsync(mask, d_mask, 32, cudaMemcpyDeviceToHost, st))) break;
        e = cudaStreamSynchronize(st);
    } while (0);
    scratch_free(block, st);
    return e ? cuda_fail(e, "byte set") : SS_OK;
}

}  // namespace ss
