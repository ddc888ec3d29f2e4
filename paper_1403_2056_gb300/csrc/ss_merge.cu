// LCP-aware merging of sorted runs (Section 4: LCP-Compare, Algorithm 2;
// binary LCP-merge, Algorithm 3) on one GPU.
//
// The paper merges K runs with one LCP-aware tournament tree per job and
// splits jobs by LCP minima (Section 4.3).  On the GPU the K-way merge is
// ceil(log2 K) rounds of pairwise merges; inside a round the output of every
// pair is cut into fixed chunks of kMergeItems strings by merge path (binary
// search on the cross diagonal, full string comparisons), and each thread
// runs the binary LCP-merge over its chunk.  The LCPs that start a chunk are
// recomputed at the cut: one side's is the run's own LCP entry, the other is
// one string comparison.  After that, comparisons whose LCPs differ cost no
// string access at all (cases 2 and 3 of LCP-Compare); only equal LCPs read
// characters, 8 at a time from the known common prefix on.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <string.h>
#include <vector>

#include "ss_internal.cuh"

namespace ss {

constexpr uint32_t kMergeItems = 64;

// full comparison of strings a and b from depth h on (both share h characters);
// returns -1/0/+1 and the lcp in *l
__device__ __forceinline__ int str_cmp_from(const ReqDesc &S, uint32_t a, uint32_t b, uint32_t h, uint32_t *l) {
    for (;;) {
        uint64_t ka = load_key(S, a, h), kb = load_key(S, b, h);
        if (ka != kb) {
            *l = h + lcp8(ka, kb);
            return ka < kb ? -1 : 1;
        }
        if (has_zero(ka)) {
            *l = h + nulpos(ka);
            return 0;
        }
        h += 8;
    }
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
// output positions; an unpaired last run is copied.
__global__ void k_merge_round(ReqDesc S, const uint32_t *in_perm, const uint32_t *in_lcp, const uint32_t *rb, uint32_t R,
                              const uint32_t *rbase, uint32_t total, uint32_t *out_perm, uint32_t *out_lcp) {
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t o64 = (uint64_t)t * kMergeItems;
    if (o64 >= total) return;
    uint32_t o = (uint32_t)o64;
    const uint32_t end = (o64 + kMergeItems < (uint64_t)total) ? (uint32_t)(o64 + kMergeItems) : total;
    while (o < end) {
        uint32_t r = upper_run(rb, R, o);
        uint32_t p = r / 2;
        uint32_t a0 = rb[2 * p], a1 = rb[2 * p + 1];
        uint32_t b1 = (2 * p + 1 < R) ? rb[2 * p + 2] : a1;   // unpaired last run: B empty
        const uint32_t na = a1 - a0, nb = b1 - a1;
        const uint32_t *Araw = in_perm + a0, *Braw = in_perm + a1;
        const uint32_t *HA = in_lcp + a0, *HB = in_lcp + a1;
        // string index of a run entry: entry + the run's index base (first round only)
        const uint32_t baseA = rbase ? rbase[2 * p] : 0u;
        const uint32_t baseB = (rbase && 2 * p + 1 < R) ? rbase[2 * p + 1] : 0u;
        auto A = [&](uint32_t k) { return Araw[k] + baseA; };
        auto B = [&](uint32_t k) { return Braw[k] + baseB; };
        const uint32_t pair_end = a0 + na + nb;
        const uint32_t stop = min(end, pair_end);
        uint32_t diag = o - a0;
        // merge path: i = strings taken from A among the first diag outputs (A first on ties)
        uint32_t lo = diag > nb ? diag - nb : 0, hi = min(diag, na);
        while (lo < hi) {
            uint32_t mid = (lo + hi) / 2;
            uint32_t l;
            if (str_cmp_from(S, A(mid), B(diag - 1 - mid), 0, &l) <= 0) lo = mid + 1; else hi = mid;
        }
        uint32_t i = lo, j = diag - lo;
        // LCPs of both fronts with the last string written before position o
        uint32_t ha = 0, hb = 0;
        if (diag > 0) {
            bool last_is_b;
            if (i == 0) last_is_b = true;
            else if (j == 0) last_is_b = false;
            else {
                uint32_t l;
                last_is_b = str_cmp_from(S, A(i - 1), B(j - 1), 0, &l) <= 0;   // ties: A then B
            }
            uint32_t prev = last_is_b ? B(j - 1) : A(i - 1);
            if (i < na) {
                if (!last_is_b) ha = HA[i];
                else { uint32_t l; str_cmp_from(S, prev, A(i), 0, &l); ha = l; }
            }
            if (j < nb) {
                if (last_is_b) hb = HB[j];
                else { uint32_t l; str_cmp_from(S, prev, B(j), 0, &l); hb = l; }
            }
        }
        // binary LCP-merge (Algorithm 3) over positions [o, stop)
        for (; o < stop; o++) {
            bool take_b;
            uint32_t hp = 0;
            bool both = i < na && j < nb;
            if (!both) {
                take_b = i >= na;
            } else if (ha == hb) {   // case 1: compare characters from the common LCP on
                int c = str_cmp_from(S, A(i), B(j), ha, &hp);
                take_b = c > 0;
            } else if (ha < hb) {    // case 2: B is smaller
                take_b = true;
                hp = ha;
            } else {                 // case 3: A is smaller
                take_b = false;
                hp = hb;
            }
            if (!take_b) {
                out_perm[o] = A(i);
                out_lcp[o] = (o == a0) ? 0u : ha;
                i++;
                ha = i < na ? HA[i] : 0;
                if (both) hb = hp;
            } else {
                out_perm[o] = B(j);
                out_lcp[o] = (o == a0) ? 0u : hb;
                j++;
                hb = j < nb ? HB[j] : 0;
                if (both) ha = hp;
            }
        }
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
               const uint32_t *run_base_host, uint32_t K, uint32_t *perm_out, uint32_t *lcp_out, cudaStream_t st) {
    uint32_t total = run_begin_host[K];
    // drop empty runs (they merge as nothing)
    std::vector<uint32_t> rb{0}, rbase;
    for (uint32_t k = 0; k < K; k++)
        if (run_begin_host[k + 1] > run_begin_host[k]) {
            rb.push_back(run_begin_host[k + 1]);
            rbase.push_back(run_base_host ? run_base_host[k] : 0u);
        }
    uint32_t R = (uint32_t)rb.size() - 1;
    size_t rounds = 0;
    for (uint32_t r = R; r > 1; r = (r + 1) / 2) rounds++;
    size_t bytes = 2ull * 4 * total + 8ull * (K + 2) + 2048;
    void *block = nullptr;
    cudaError_t e = scratch_alloc(&block, bytes, st);
    if (e) {
        cudaGetLastError();
        set_error_detail("ss_merge: scratch allocation of %zu bytes failed", bytes);
        return SS_ERR_OOM;
    }
    uint32_t *tmp_perm = (uint32_t *)block;
    uint32_t *tmp_lcp = tmp_perm + (((size_t)total + 63) & ~(size_t)63);
    uint32_t *d_rb = tmp_lcp + (((size_t)total + 63) & ~(size_t)63);
    uint32_t *d_base = d_rb + ((K + 2 + 63) & ~63u);
    int rc = SS_OK;
    uint32_t *stage = (uint32_t *)host_staging(sizeof(uint32_t) * 2 * (K + 2));
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
            memcpy(stage, rb.data(), sizeof(uint32_t) * (R + 1));
            if (round == 1) memcpy(stage + (R + 1), rbase.data(), sizeof(uint32_t) * R);
            size_t cp = sizeof(uint32_t) * ((R + 1) + (round == 1 ? R : 0));
            if ((e = cudaMemcpyAsync(d_rb, stage, cp, cudaMemcpyHostToDevice, st))) break;
            const uint32_t *bases = round == 1 ? d_rb + (R + 1) : nullptr;
            uint32_t threads = (total + kMergeItems - 1) / kMergeItems;
            SS_LAUNCH_U("merge_round", st, total, k_merge_round<<<(threads + 255) / 256, 256, 0, st>>>(
                set, src_p, src_l, d_rb, R, bases, total, dst_p, dst_l));
            if ((e = cudaGetLastError())) break;
            // the staging buffer is reused next round: wait for the copy
            if ((e = cudaStreamSynchronize(st))) break;
            std::vector<uint32_t> nrb{0};
            for (uint32_t k = 2; k <= R; k += 2) nrb.push_back(rb[k]);
            if (R % 2) nrb.push_back(rb[R]);
            rb = nrb;
            R = (uint32_t)rb.size() - 1;
            src_p = dst_p;
            src_l = dst_l;
        }
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

// device address of g_noalloc_scratch, looked up once per device with that
// device current (in host code the symbol name is only a host-side stand-in)
static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[128];

static cudaError_t noalloc_setup(uint32_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = (uint32_t *)g_noalloc_ptr[dev];
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
            set, src_p, src_l, d_table, R, d_table + kNoAllocMaxRuns + 1, total, dst_p, dst_l));
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
