// C ABI of the string sorter: argument checks, scratch pool, error detail,
// optional per-kernel timing.  Every entry point forwards to the kernels in
// ss_engine.cu / ss_merge.cu; nothing here computes on the host.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ss_internal.cuh"

namespace ss {

static thread_local std::string t_detail;

void set_error_detail(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_detail = buf;
}

int cuda_fail(cudaError_t e, const char *what) {
    set_error_detail("%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    return SS_ERR_CUDA;
}

// ---------------------------------------------------------- scratch pool
// One memory pool per device, owned by the library, keeping freed blocks
// for reuse (release threshold = unlimited).

static std::mutex g_pool_mu;
static std::map<int, cudaMemPool_t> g_pools;

static cudaMemPool_t pool_for_current() {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) return it->second;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    g_pools[dev] = pool;
    return pool;
}

// host-side allocation-failure injection (ss_debug_fail_allocs)
static std::atomic<uint32_t> g_inject_skip{0}, g_inject_fail{0};
static std::mutex g_inject_mu;

static bool inject_failure() {
    if (g_inject_fail.load(std::memory_order_relaxed) == 0) return false;
    std::lock_guard<std::mutex> lk(g_inject_mu);
    if (g_inject_fail.load() == 0) return false;
    if (g_inject_skip.load() > 0) {
        g_inject_skip.fetch_sub(1);
        return false;
    }
    g_inject_fail.fetch_sub(1);
    return true;
}

cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t s) {
    if (inject_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    cudaMemPool_t pool = pool_for_current();
    if (!pool) return cudaErrorMemoryAllocation;
    return cudaMallocFromPoolAsync(p, bytes ? bytes : 256, pool, s);
}

cudaError_t scratch_free(void *p, cudaStream_t s) {
    if (!p) return cudaSuccess;
    return cudaFreeAsync(p, s);
}

// ------------------------------------------------------ host staging
struct Staging {
    void *p = nullptr;
    size_t cap = 0;
    ~Staging() {
        if (p) cudaFreeHost(p);
    }
};
static thread_local Staging t_staging;

void *host_staging(size_t bytes) {
    if (t_staging.cap < bytes) {
        if (t_staging.p) cudaFreeHost(t_staging.p);
        t_staging.p = nullptr;
        size_t cap = bytes < 4096 ? 4096 : bytes;
        if (cudaMallocHost(&t_staging.p, cap) != cudaSuccess) {
            cudaGetLastError();
            t_staging.p = malloc(cap);   // pageable fallback for the counter readback only
        }
        t_staging.cap = cap;
    }
    return t_staging.p;
}

// ------------------------------------------------------------ profiling
static std::atomic<int> g_prof_on{0};
static std::atomic<uint64_t> g_launches{0};
struct ProfRec {
    uint64_t launches = 0;
    uint64_t units = 0;
    double ms = 0;
};
static std::mutex g_prof_mu;
static std::vector<std::pair<std::string, ProfRec>> g_prof;
struct PendingEv {
    std::string name;
    cudaEvent_t a, b;
    uint64_t units;
};
static thread_local std::vector<PendingEv> t_pending;
static thread_local cudaEvent_t t_open = nullptr;

static void prof_flush() {
    for (auto &pe : t_pending) {
        float ms = 0;
        cudaEventSynchronize(pe.b);
        cudaEventElapsedTime(&ms, pe.a, pe.b);
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
        std::lock_guard<std::mutex> lk(g_prof_mu);
        bool found = false;
        for (auto &r : g_prof)
            if (r.first == pe.name) { r.second.launches++; r.second.ms += ms; r.second.units += pe.units; found = true; break; }
        if (!found) {
            ProfRec r;
            r.launches = 1;
            r.ms = ms;
            r.units = pe.units;
            g_prof.emplace_back(pe.name, r);
        }
    }
    t_pending.clear();
}

bool prof_on() { return g_prof_on.load() != 0; }

void prof_begin(const char *name, cudaStream_t s) {
    (void)name;
    g_launches++;
    if (!g_prof_on.load()) return;
    cudaEventCreate(&t_open);
    cudaEventRecord(t_open, s);
}

void prof_end(const char *name, cudaStream_t s, uint64_t units) {
    if (!g_prof_on.load() || !t_open) return;
    cudaEvent_t b;
    cudaEventCreate(&b);
    cudaEventRecord(b, s);
    t_pending.push_back(PendingEv{name, t_open, b, units});
    t_open = nullptr;
    if (t_pending.size() > 4096) prof_flush();
}

}  // namespace ss

using namespace ss;

static cudaStream_t as_stream(ss_stream_t s) { return reinterpret_cast<cudaStream_t>(s); }

static ReqDesc make_req(const uint8_t *chars, const uint64_t *offsets, const uint32_t *lengths, uint32_t fixed_len,
                        uint32_t n, uint32_t *perm, uint32_t *lcp, int32_t *status) {
    ReqDesc r;
    memset(&r, 0, sizeof(r));
    r.chars = chars;
    r.offsets = offsets;
    r.lengths = lengths;
    r.fixed_len = lengths ? 0 : fixed_len;
    r.n = n;
    r.perm_out = perm;
    r.lcp_out = lcp;
    r.status_out = status;
    return r;
}

static int check_req(const ReqDesc &r, const char *who) {
    if (r.n == 0) return SS_OK;
    if (!r.chars || !r.offsets || !r.perm_out || !r.lcp_out) {
        set_error_detail("%s: NULL pointer with n = %u", who, r.n);
        return SS_ERR_INVALID;
    }
    if (r.n == 0xFFFFFFFFu) {
        set_error_detail("%s: n = 2^32 - 1 is beyond the limit 2^32 - 2", who);
        return SS_ERR_TOO_LARGE;
    }
    return SS_OK;
}

namespace ss {

// Host buffers in, host buffers out: copies, the sort (runs > 1: index-contiguous
// runs sorted together, then the LCP merge), copies back; returns when done.
int host_sort(const uint8_t *chars_host, uint64_t chars_len, const uint64_t *offsets_host, const uint32_t *lengths_host,
              uint32_t fixed_len, uint32_t n, uint32_t runs, uint32_t *perm_host, uint32_t *lcp_host, cudaStream_t st) {
    if (n == 0) return SS_OK;
    if (!chars_host || !offsets_host || !perm_host || !lcp_host || chars_len == 0) {
        set_error_detail("ss_sort_host: NULL pointer or empty chars with n = %u", n);
        return SS_ERR_INVALID;
    }
    if (n == 0xFFFFFFFFu) return SS_ERR_TOO_LARGE;
    if (runs == 0) runs = 1;
    if (runs > n) runs = n;
    const size_t A = 255;
    size_t cbytes = (chars_len + 15) & ~(size_t)15;   // aligned words past the end stay inside
    size_t nb4 = (4ull * n + A) & ~A, nb8 = (8ull * n + A) & ~A;
    size_t bytes = ((cbytes + A) & ~A) + nb8 + (lengths_host ? nb4 : 0) + 2 * nb4 + (runs > 1 ? 3 * nb4 + 2 * nb8 : 0) +
                   1024;
    void *block = nullptr;
    cudaError_t e = scratch_alloc(&block, bytes, st);
    if (e) {
        cudaGetLastError();
        set_error_detail("ss_sort_host: device allocation of %zu bytes failed", bytes);
        return SS_ERR_OOM;
    }
    char *p = (char *)block;
    uint8_t *d_chars = (uint8_t *)p;
    p += (cbytes + A) & ~A;
    uint64_t *d_off = (uint64_t *)p;
    p += nb8;
    uint32_t *d_len = nullptr;
    if (lengths_host) {
        d_len = (uint32_t *)p;
        p += nb4;
    }
    uint32_t *d_perm = (uint32_t *)p;
    p += nb4;
    uint32_t *d_lcp = (uint32_t *)p;
    p += nb4;
    uint32_t *d_rperm = runs > 1 ? (uint32_t *)p : nullptr;
    uint32_t *d_rlcp = runs > 1 ? (uint32_t *)(p + nb4) : nullptr;
    // the runs' caches, written by their sort and read by the merge
    uint64_t *d_roff = runs > 1 ? (uint64_t *)(p + 2 * nb4) : nullptr;
    uint64_t *d_rck = runs > 1 ? (uint64_t *)(p + 2 * nb4 + nb8) : nullptr;
    uint32_t *d_rckd = runs > 1 ? (uint32_t *)(p + 2 * nb4 + 2 * nb8) : nullptr;
    int rc = SS_OK;
    do {
        if (cbytes > chars_len && (e = cudaMemsetAsync(d_chars + chars_len, 0, cbytes - chars_len, st))) break;
        if ((e = cudaMemcpyAsync(d_chars, chars_host, chars_len, cudaMemcpyHostToDevice, st))) break;
        if ((e = cudaMemcpyAsync(d_off, offsets_host, 8ull * n, cudaMemcpyHostToDevice, st))) break;
        if (lengths_host && (e = cudaMemcpyAsync(d_len, lengths_host, 4ull * n, cudaMemcpyHostToDevice, st))) break;
        if (runs <= 1) {
            ReqDesc r = make_req(d_chars, d_off, d_len, fixed_len, n, d_perm, d_lcp, nullptr);
            rc = engine_sort(&r, 1, st);
        } else {
            // index-contiguous runs sorted together, then merged (Section 5)
            std::vector<ReqDesc> rq(runs);
            std::vector<uint32_t> rb(runs + 1);
            for (uint32_t k = 0; k <= runs; k++) rb[k] = (uint32_t)((uint64_t)n * k / runs);
            for (uint32_t k = 0; k < runs; k++) {
                rq[k] = make_req(d_chars, d_off + rb[k], d_len ? d_len + rb[k] : nullptr, fixed_len, rb[k + 1] - rb[k],
                                 d_rperm + rb[k], d_rlcp + rb[k], nullptr);
                rq[k].off_out = d_roff + rb[k];
                rq[k].ck_out = d_rck + rb[k];
                rq[k].ckd_out = d_rckd + rb[k];
            }
            rc = engine_sort(rq.data(), runs, st);
            if (rc == SS_OK) {
                ReqDesc set = make_req(d_chars, d_off, d_len, fixed_len, 0, nullptr, nullptr, nullptr);
                rc = merge_runs(set, d_rperm, d_rlcp, rb.data(), rb.data(), runs, d_perm, d_lcp, st, MERGE_PAIRWISE,
                                RunCache{d_roff, d_rck, d_rckd});
            }
        }
        if (rc != SS_OK) break;
        if ((e = cudaMemcpyAsync(perm_host, d_perm, 4ull * n, cudaMemcpyDeviceToHost, st))) break;
        if ((e = cudaMemcpyAsync(lcp_host, d_lcp, 4ull * n, cudaMemcpyDeviceToHost, st))) break;
        e = cudaStreamSynchronize(st);
        if (!e) {
            const int32_t dev = engine_take_device_error();
            if (dev != SS_OK) {
                set_error_detail("ss_sort_host: device-side failure %d", dev);
                rc = dev;
            }
        }
    } while (0);
    if (e && rc == SS_OK) rc = cuda_fail(e, "ss_sort_host");
    scratch_free(block, st);
    return rc;
}

}  // namespace ss

extern "C" {

int ss_version(void) { return 101; }

int ss_last_error_detail(char *buf, size_t len) {
    const std::string &d = t_detail;
    if (buf && len) {
        size_t k = d.size() < len - 1 ? d.size() : len - 1;
        memcpy(buf, d.data(), k);
        buf[k] = 0;
    }
    return (int)d.size();
}

int ss_sort_ex(const uint8_t *chars, const uint64_t *offsets, const uint32_t *lengths, uint32_t fixed_len, uint32_t n,
               uint32_t *perm_out, uint32_t *lcp_out, ss_stream_t stream) {
    t_detail.clear();
    ReqDesc r = make_req(chars, offsets, lengths, fixed_len, n, perm_out, lcp_out, nullptr);
    int rc = check_req(r, "ss_sort_ex");
    if (rc != SS_OK || n == 0) return rc;
    return engine_sort(&r, 1, as_stream(stream));
}

int ss_sort(const uint8_t *chars, const uint64_t *offsets, uint32_t n, uint32_t *perm_out, uint32_t *lcp_out,
            ss_stream_t stream) {
    return ss_sort_ex(chars, offsets, nullptr, 0, n, perm_out, lcp_out, stream);
}

int ss_sort_batch(const ss_request *reqs, uint32_t count, ss_stream_t stream) {
    t_detail.clear();
    if (count == 0) return SS_OK;
    if (!reqs) {
        set_error_detail("ss_sort_batch: NULL request array");
        return SS_ERR_INVALID;
    }
    std::vector<ReqDesc> v(count);
    for (uint32_t i = 0; i < count; i++) {
        const ss_request &q = reqs[i];
        v[i] = make_req(q.chars, q.offsets, q.lengths, q.fixed_len, q.n, q.perm_out, q.lcp_out, q.status_out);
        int rc = check_req(v[i], "ss_sort_batch");
        if (rc != SS_OK) return rc;
    }
    return engine_sort(v.data(), count, as_stream(stream));
}

// tuning of one request, packed as in ReqDesc::tune (and ReqDesc::alpha)
static int pack_tuning(const ss_tuning &t, ReqDesc &r, const char *who) {
    uint32_t &out = r.tune;
    if (t.alphabet) {
        const uint32_t a0 = t.alphabet & 0xFFu, a1 = (t.alphabet >> 8) & 0xFFu, a2 = (t.alphabet >> 16) & 0xFFu,
                       a3 = t.alphabet >> 24;
        if (!(a0 >= 1 && a0 <= a1 && a1 <= a2 && a2 <= a3)) {
            set_error_detail("%s: alphabet bytes must satisfy 1 <= a0 <= a1 <= a2 <= a3", who);
            return SS_ERR_INVALID;
        }
        if (r.lengths || r.fixed_len == 0) {
            set_error_detail("%s: alphabet compression needs fixed-length strings (lengths NULL, fixed_len > 0)", who);
            return SS_ERR_INVALID;
        }
        r.alpha = t.alphabet;
    }
    uint32_t s = 0;
    if (t.child_target) {
        if (t.child_target < 32 || t.child_target > 65536 || (t.child_target & (t.child_target - 1))) {
            set_error_detail("%s: child_target must be 0 or a power of two in [32, 65536], got %u", who, t.child_target);
            return SS_ERR_INVALID;
        }
        while ((1u << s) < t.child_target) s++;
    }
    if (t.min_step > 9) {
        set_error_detail("%s: min_step must be in [0, 9], got %u", who, t.min_step);
        return SS_ERR_INVALID;
    }
    if (t.classifier > CLS_JUMP) {
        set_error_detail("%s: classifier must be in [0, 2], got %u", who, t.classifier);
        return SS_ERR_INVALID;
    }
    if (t.max_depth && (t.max_depth < 2 || t.max_depth > (uint32_t)kLevelD)) {
        set_error_detail("%s: max_depth must be 0 or in [2, %d], got %u", who, kLevelD, t.max_depth);
        return SS_ERR_INVALID;
    }
    uint32_t sm = 0;
    if (t.small_max) {
        if (t.small_max < 64 || t.small_max > kSmallMax || (t.small_max & (t.small_max - 1))) {
            set_error_detail("%s: small_max must be 0 or a power of two in [64, %u], got %u", who, kSmallMax, t.small_max);
            return SS_ERR_INVALID;
        }
        while ((1u << sm) < t.small_max) sm++;
    }
    out = s | (t.min_step << 8) | (t.classifier << 16) | (t.max_depth << 20) | (sm << 24);
    return SS_OK;
}

int ss_sort_batch_async(const ss_request *reqs, const ss_tuning *tunings, uint32_t count, ss_stream_t stream) {
    t_detail.clear();
    if (count == 0) return SS_OK;
    if (!reqs) {
        set_error_detail("ss_sort_batch_async: NULL request array");
        return SS_ERR_INVALID;
    }
    std::vector<ReqDesc> v(count);
    for (uint32_t i = 0; i < count; i++) {
        const ss_request &q = reqs[i];
        v[i] = make_req(q.chars, q.offsets, q.lengths, q.fixed_len, q.n, q.perm_out, q.lcp_out, q.status_out);
        int rc = check_req(v[i], "ss_sort_batch_async");
        if (rc == SS_OK && tunings) rc = pack_tuning(tunings[i], v[i], "ss_sort_batch_async");
        if (rc != SS_OK) return rc;
    }
    return engine_sort(v.data(), count, as_stream(stream), true);
}

int ss_sort_batch_cached(const ss_request *reqs, const ss_tuning *tunings, const ss_sort_cache *caches,
                         uint32_t count, ss_stream_t stream) {
    t_detail.clear();
    if (count == 0) return SS_OK;
    if (!reqs) {
        set_error_detail("ss_sort_batch_cached: NULL request array");
        return SS_ERR_INVALID;
    }
    std::vector<ReqDesc> v(count);
    for (uint32_t i = 0; i < count; i++) {
        const ss_request &q = reqs[i];
        v[i] = make_req(q.chars, q.offsets, q.lengths, q.fixed_len, q.n, q.perm_out, q.lcp_out, q.status_out);
        int rc = check_req(v[i], "ss_sort_batch_cached");
        if (rc == SS_OK && tunings) rc = pack_tuning(tunings[i], v[i], "ss_sort_batch_cached");
        if (rc != SS_OK) return rc;
        if (!caches) continue;
        const ss_sort_cache &c = caches[i];
        const int given = (c.off_out != nullptr) + (c.ck_out != nullptr) + (c.ckd_out != nullptr);
        if (given == 0) continue;
        if (given != 3) {
            set_error_detail("ss_sort_batch_cached: request %u: give all of off_out, ck_out, ckd_out or none", i);
            return SS_ERR_INVALID;
        }
        if (v[i].alpha) {
            set_error_detail("ss_sort_batch_cached: request %u: caches hold bytes, not compressed characters", i);
            return SS_ERR_INVALID;
        }
        v[i].off_out = c.off_out;
        v[i].ck_out = c.ck_out;
        v[i].ckd_out = c.ckd_out;
    }
    return engine_sort(v.data(), count, as_stream(stream));
}

int ss_sort_batch_tuned(const ss_request *reqs, const ss_tuning *tunings, uint32_t count, ss_stream_t stream) {
    t_detail.clear();
    if (count == 0) return SS_OK;
    if (!reqs) {
        set_error_detail("ss_sort_batch_tuned: NULL request array");
        return SS_ERR_INVALID;
    }
    std::vector<ReqDesc> v(count);
    for (uint32_t i = 0; i < count; i++) {
        const ss_request &q = reqs[i];
        v[i] = make_req(q.chars, q.offsets, q.lengths, q.fixed_len, q.n, q.perm_out, q.lcp_out, q.status_out);
        int rc = check_req(v[i], "ss_sort_batch_tuned");
        if (rc == SS_OK && tunings) rc = pack_tuning(tunings[i], v[i], "ss_sort_batch_tuned");
        if (rc != SS_OK) return rc;
    }
    return engine_sort(v.data(), count, as_stream(stream));
}

int ss_autotune(const ss_request *req, uint32_t sample_n, ss_tuning *best_out, double *best_ms_out, ss_stream_t stream) {
    t_detail.clear();
    if (!req || !best_out) {
        set_error_detail("ss_autotune: NULL argument");
        return SS_ERR_INVALID;
    }
    ReqDesc r = make_req(req->chars, req->offsets, req->lengths, req->fixed_len, req->n, req->perm_out, req->lcp_out,
                         nullptr);
    int rc = check_req(r, "ss_autotune");
    if (rc != SS_OK) return rc;
    const uint32_t n = std::min<uint32_t>(req->n, sample_n ? sample_n : 2000000u);
    *best_out = ss_tuning{0, 0, 0, 0, 0, 0};
    if (best_ms_out) *best_ms_out = 0;
    if (n < 2) return SS_OK;
    cudaStream_t st = as_stream(stream);
    void *block = nullptr;
    const size_t nb = ((size_t)n * 4 + 255) & ~(size_t)255;
    cudaError_t e = scratch_alloc(&block, 2 * nb, st);
    if (e) {
        cudaGetLastError();
        set_error_detail("ss_autotune: scratch allocation failed");
        return SS_ERR_OOM;
    }
    r.n = n;
    r.perm_out = (uint32_t *)block;
    r.lcp_out = (uint32_t *)((char *)block + nb);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double best = -1;
    // one candidate: a warm sort (pool, caches), then a timed one
    auto try_one = [&](const ss_tuning &t) -> bool {
        if ((rc = pack_tuning(t, r, "ss_autotune")) != SS_OK) return false;
        if ((rc = engine_sort(&r, 1, st)) != SS_OK) return false;
        if ((e = cudaEventRecord(e0, st))) return false;
        if ((rc = engine_sort(&r, 1, st)) != SS_OK) return false;
        if ((e = cudaEventRecord(e1, st)) || (e = cudaEventSynchronize(e1))) return false;
        float msec = 0;
        if ((e = cudaEventElapsedTime(&msec, e0, e1))) return false;
        if (best < 0 || msec < best) {
            best = msec;
            *best_out = t;
        }
        return true;
    };
    const uint32_t targets[] = {256, 512, 1024, 2048};
    const uint32_t steps[] = {1, 3, 5, 9};
    do {
        if ((e = cudaEventCreate(&e0)) || (e = cudaEventCreate(&e1))) break;
        bool ok = true;
        for (uint32_t ct : targets)
            for (uint32_t ms : steps)
                if (ok) ok = try_one(ss_tuning{ct, ms, CLS_UNROLL, 0, 0, 0});
        // the other classifiers with the best tree shape
        const ss_tuning shape = *best_out;
        if (ok) ok = try_one(ss_tuning{shape.child_target, shape.min_step, CLS_EQUAL, 0, 0, 0});
        if (ok) ok = try_one(ss_tuning{shape.child_target, shape.min_step, CLS_JUMP, 0, 0, 0});
        // smaller trees per level, then smaller base cases, each on the best so far
        for (uint32_t md : {6u, 7u}) {
            ss_tuning t = *best_out;
            t.max_depth = md;
            if (ok) ok = try_one(t);
        }
        for (uint32_t sm : {512u, 1024u}) {
            ss_tuning t = *best_out;
            t.small_max = sm;
            if (ok) ok = try_one(t);
        }
        // key width: fixed-length strings over at most four bytes (none of
        // them 0) take keys of 32 two-bit characters (alphabet compression)
        if (ok && !r.lengths && r.fixed_len > 0) {
            uint32_t mask[8];
            if ((rc = engine_byte_set(r, n, mask, st)) != SS_OK) break;
            uint32_t a[4], na = 0;
            for (uint32_t c = 0; c < 256; c++)
                if (mask[c >> 5] >> (c & 31) & 1u) {
                    if (na < 4) a[na] = c;
                    na++;
                }
            if (na >= 1 && na <= 4 && a[0] != 0) {
                for (uint32_t k = na; k < 4; k++) a[k] = a[na - 1];
                ss_tuning t = *best_out;
                t.alphabet = a[0] | a[1] << 8 | a[2] << 16 | a[3] << 24;
                ok = try_one(t);
            }
        }
    } while (0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    scratch_free(block, st);
    if (e && rc == SS_OK) rc = cuda_fail(e, "ss_autotune");
    if (rc == SS_OK && best_ms_out) *best_ms_out = best;
    return rc;
}

int ss_sort_host(const uint8_t *chars_host, uint64_t chars_len, const uint64_t *offsets_host,
                 const uint32_t *lengths_host, uint32_t fixed_len, uint32_t n, uint32_t runs, uint32_t *perm_host,
                 uint32_t *lcp_host, ss_stream_t stream) {
    t_detail.clear();
    return host_sort(chars_host, chars_len, offsets_host, lengths_host, fixed_len, n, runs, perm_host, lcp_host,
                     as_stream(stream));
}

int ss_merge(const uint8_t *chars, const uint64_t *offsets, const uint32_t *lengths, uint32_t fixed_len,
             const uint32_t *run_perm, const uint32_t *run_lcp, const uint32_t *run_begin_host,
             const uint32_t *run_base_host, uint32_t K, uint32_t *perm_out, uint32_t *lcp_out, ss_stream_t stream) {
    return ss_merge_ex(chars, offsets, lengths, fixed_len, run_perm, run_lcp, run_begin_host, run_base_host, K,
                       SS_MERGE_PAIRWISE, perm_out, lcp_out, stream);
}

// argument checks shared by the merge entry points: SS_OK with *total set
// (0: nothing to merge), or the error
static int check_merge(const uint8_t *chars, const uint64_t *offsets, const uint32_t *run_perm, const uint32_t *run_lcp,
                       const uint32_t *run_begin_host, uint32_t K, const uint32_t *perm_out, const uint32_t *lcp_out,
                       uint32_t *total) {
    *total = 0;
    if (K == 0 || !run_begin_host) {
        set_error_detail("ss_merge: K must be >= 1 with run_begin_host[K+1]");
        return SS_ERR_INVALID;
    }
    if (run_begin_host[0] != 0) {
        set_error_detail("ss_merge: run_begin_host[0] must be 0");
        return SS_ERR_INVALID;
    }
    for (uint32_t k = 0; k < K; k++)
        if (run_begin_host[k + 1] < run_begin_host[k]) {
            set_error_detail("ss_merge: run_begin_host must be non-decreasing");
            return SS_ERR_INVALID;
        }
    const uint32_t t = run_begin_host[K];
    if (t == 0) return SS_OK;
    if (t == 0xFFFFFFFFu) return SS_ERR_TOO_LARGE;
    if (!chars || !offsets || !run_perm || !run_lcp || !perm_out || !lcp_out) {
        set_error_detail("ss_merge: NULL pointer");
        return SS_ERR_INVALID;
    }
    *total = t;
    return SS_OK;
}

int ss_merge_ex(const uint8_t *chars, const uint64_t *offsets, const uint32_t *lengths, uint32_t fixed_len,
                const uint32_t *run_perm, const uint32_t *run_lcp, const uint32_t *run_begin_host,
                const uint32_t *run_base_host, uint32_t K, uint32_t method, uint32_t *perm_out, uint32_t *lcp_out,
                ss_stream_t stream) {
    t_detail.clear();
    if (method != SS_MERGE_PAIRWISE && method != SS_MERGE_LOSER_TREE) {
        set_error_detail("ss_merge_ex: unknown merge method %u", method);
        return SS_ERR_INVALID;
    }
    uint32_t total = 0;
    int rc = check_merge(chars, offsets, run_perm, run_lcp, run_begin_host, K, perm_out, lcp_out, &total);
    if (rc != SS_OK || total == 0) return rc;
    ReqDesc set = make_req(chars, offsets, lengths, fixed_len, 0, nullptr, nullptr, nullptr);
    return merge_runs(set, run_perm, run_lcp, run_begin_host, run_base_host, K, perm_out, lcp_out, as_stream(stream),
                      method);
}

int ss_merge_cached(const uint8_t *chars, const uint64_t *offsets, const uint32_t *lengths, uint32_t fixed_len,
                    const uint32_t *run_perm, const uint32_t *run_lcp, const uint64_t *run_off, const uint64_t *run_ck,
                    const uint32_t *run_ckd, const uint32_t *run_begin_host, const uint32_t *run_base_host, uint32_t K,
                    uint32_t *perm_out, uint32_t *lcp_out, ss_stream_t stream) {
    t_detail.clear();
    uint32_t total = 0;
    int rc = check_merge(chars, offsets, run_perm, run_lcp, run_begin_host, K, perm_out, lcp_out, &total);
    if (rc != SS_OK || total == 0) return rc;
    if (!run_off || !run_ck || !run_ckd) {
        set_error_detail("ss_merge_cached: NULL cache array");
        return SS_ERR_INVALID;
    }
    ReqDesc set = make_req(chars, offsets, lengths, fixed_len, 0, nullptr, nullptr, nullptr);
    return merge_runs(set, run_perm, run_lcp, run_begin_host, run_base_host, K, perm_out, lcp_out, as_stream(stream),
                      MERGE_PAIRWISE, RunCache{run_off, run_ck, run_ckd});
}

int ss_gather_keys(const uint8_t *chars, const uint64_t *offsets, const uint32_t *lengths, uint32_t fixed_len,
                   uint32_t n, const uint32_t *depth, uint64_t *keys_out, ss_stream_t stream) {
    t_detail.clear();
    if (n == 0) return SS_OK;
    if (!chars || !offsets || !depth || !keys_out) {
        set_error_detail("ss_gather_keys: NULL pointer");
        return SS_ERR_INVALID;
    }
    ReqDesc r = make_req(chars, offsets, lengths, fixed_len, n, nullptr, nullptr, nullptr);
    return engine_gather(r, depth, keys_out, as_stream(stream));
}

int ss_splitters(const uint64_t *sample, uint32_t a, uint32_t d, uint64_t *x_out, ss_stream_t stream) {
    t_detail.clear();
    if (!sample || !x_out || a == 0 || a > 2047 || d < 1 || d > (uint32_t)kMaxD) {
        set_error_detail("ss_splitters: need 1 <= a <= 2047, 1 <= d <= %d and non-NULL pointers", kMaxD);
        return SS_ERR_INVALID;
    }
    return engine_splitters(sample, a, d, x_out, as_stream(stream));
}

int ss_classify(const uint64_t *keys, uint32_t n, const uint64_t *x, uint32_t d, uint16_t *bucket_out,
                uint32_t *bucket_begin_out, uint32_t *order_out, ss_stream_t stream) {
    t_detail.clear();
    if (d < 1 || d > (uint32_t)kMaxD || !x || !bucket_begin_out || (n && (!keys || !bucket_out || !order_out))) {
        set_error_detail("ss_classify: need 1 <= d <= %d and non-NULL pointers", kMaxD);
        return SS_ERR_INVALID;
    }
    if (n == 0xFFFFFFFFu) return SS_ERR_TOO_LARGE;
    return engine_classify(keys, n, x, d, CLS_UNROLL, bucket_out, bucket_begin_out, order_out, as_stream(stream));
}

int ss_classify_ex(const uint64_t *keys, uint32_t n, const uint64_t *x, uint32_t d, uint32_t classifier,
                   uint16_t *bucket_out, uint32_t *bucket_begin_out, uint32_t *order_out, ss_stream_t stream) {
    t_detail.clear();
    if (classifier > CLS_JUMP) {
        set_error_detail("ss_classify_ex: classifier must be in [0, 2], got %u", classifier);
        return SS_ERR_INVALID;
    }
    if (d < 1 || d > (uint32_t)kMaxD || !x || !bucket_begin_out || (n && (!keys || !bucket_out || !order_out))) {
        set_error_detail("ss_classify_ex: need 1 <= d <= %d and non-NULL pointers", kMaxD);
        return SS_ERR_INVALID;
    }
    if (n == 0xFFFFFFFFu) return SS_ERR_TOO_LARGE;
    return engine_classify(keys, n, x, d, classifier, bucket_out, bucket_begin_out, order_out, as_stream(stream));
}

int ss_profile_enable(int on) {
    g_prof_on.store(on ? 1 : 0);
    return SS_OK;
}

int ss_profile_reset(void) {
    prof_flush();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.clear();
    g_launches.store(0);
    engine_reset_device_launches();
    return SS_OK;
}

int ss_profile_read(char *names48, uint64_t *launches, double *total_ms, uint64_t *units, int cap) {
    prof_flush();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int k = 0;
    for (auto &r : g_prof) {
        if (k >= cap) break;
        if (names48) {
            memset(names48 + 48 * k, 0, 48);
            strncpy(names48 + 48 * k, r.first.c_str(), 47);
        }
        if (launches) launches[k] = r.second.launches;
        if (total_ms) total_ms[k] = r.second.ms;
        if (units) units[k] = r.second.units;
        k++;
    }
    return (int)g_prof.size();
}

uint64_t ss_launch_count(void) { return g_launches.load() + engine_device_launches(); }

int ss_device_error(int32_t *status_out) {
    t_detail.clear();
    if (!status_out) {
        set_error_detail("ss_device_error: NULL status_out");
        return SS_ERR_INVALID;
    }
    *status_out = engine_take_device_error();
    return SS_OK;
}

int ss_debug_copy_wait(uint64_t budget_cycles, uint32_t withhold) {
    t_detail.clear();
    return engine_debug_copy_wait((long long)std::min<uint64_t>(budget_cycles, (uint64_t)INT64_MAX), withhold ? 1u : 0u);
}

int ss_debug_fail_allocs(uint32_t skip, uint32_t count) {
    std::lock_guard<std::mutex> lk(g_inject_mu);
    g_inject_skip.store(count ? skip : 0u);
    g_inject_fail.store(count);
    return SS_OK;
}

}  // extern "C"
