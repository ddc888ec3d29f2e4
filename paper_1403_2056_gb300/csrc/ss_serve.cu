// Sort server: continuous batching of independent sort requests on one GPU.
//
// The paper's parallel sorter keeps a job queue of independent subproblems and
// lets idle threads take the next one (Section 4.5).  Serving many callers is
// the same problem one level up: requests arrive over time, each is an
// independent sort, and the device should be kept busy without letting a
// request wait behind a long queue.  The server admits requests in arrival
// order while their scratch memory fits a byte budget; an idle worker (one
// host thread driving one CUDA stream) takes every admitted request waiting
// at that moment as one batch (engine_sort over all of them, the same
// level-synchronous launches as ss_sort_batch), so batches formed while
// others run overlap on the device, and a lightly loaded server runs each
// request alone as soon as it arrives.  Results are those of one ss_sort_ex
// per request: batching changes where a request's segments sit, not the
// comparisons made for it.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ss_internal.cuh"

namespace ss {

struct HostArgs {      // a request on host buffers (ss_server_submit_host)
    const uint8_t *chars;
    uint64_t chars_len;
    const uint64_t *offsets;
    const uint32_t *lengths;
    uint32_t fixed_len, n, runs;
    uint32_t *perm, *lcp;
};

struct ServerJob {
    uint64_t ticket;
    bool host;           // host buffers: runs alone, with its copies, on the worker's stream
    HostArgs ha;
    ReqDesc req;
    size_t bytes;        // admission charge: scratch of the request alone
    double t_submit, t_start, t_done;
    int status;
    bool done;
};

struct Server {
    int device = 0;
    uint64_t budget = 0;
    uint64_t in_use = 0;          // bytes charged for admitted, unfinished jobs
    uint32_t max_batch = 0;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> waiting;                         // tickets in arrival order
    std::unordered_map<uint64_t, ServerJob> jobs;         // every unretrieved job
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;

    double now_ms() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }

    // under mu: the prefix of the waiting queue that fits the budget (at least
    // one job when nothing is in flight, so a job larger than the budget alone
    // is refused at submit time, never starved here)
    std::vector<uint64_t> take_batch() {
        std::vector<uint64_t> b;
        uint64_t used = in_use;
        while (!waiting.empty() && b.size() < max_batch) {
            ServerJob &j = jobs[waiting.front()];
            if (used + j.bytes > budget && !(used == 0 && b.empty())) break;
            // a host-buffer job runs alone (its copies overlap other workers' sorts)
            if (!b.empty() && (j.host || jobs[b.front()].host)) break;
            used += j.bytes;
            b.push_back(waiting.front());
            waiting.pop_front();
        }
        in_use = used;
        return b;
    }

    int enqueue(ServerJob &j, uint32_t n, uint64_t *ticket_out) {
        std::lock_guard<std::mutex> lk(mu);
        if (stop) {
            set_error_detail("ss_server_submit: the server is shutting down");
            return SS_ERR_INVALID;
        }
        if (j.bytes > budget) {
            set_error_detail("ss_server_submit: request of %u strings needs %zu bytes, above the budget %llu", n, j.bytes,
                             (unsigned long long)budget);
            return SS_ERR_TOO_LARGE;
        }
        j.ticket = next_ticket++;
        j.t_submit = now_ms();
        *ticket_out = j.ticket;
        jobs.emplace(j.ticket, j);
        waiting.push_back(j.ticket);
        cv_work.notify_one();
        return SS_OK;
    }

    void work(cudaStream_t st) {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            cv_work.wait(lk, [&] {
                if (stop && waiting.empty()) return true;
                if (waiting.empty()) return false;
                const ServerJob &j = jobs[waiting.front()];
                return in_use + j.bytes <= budget || in_use == 0;
            });
            if (stop && waiting.empty()) return;
            std::vector<uint64_t> batch = take_batch();
            if (batch.empty()) continue;
            std::vector<ReqDesc> reqs;
            uint64_t charged = 0;
            const double ts = now_ms();
            for (uint64_t t : batch) {
                ServerJob &j = jobs[t];
                j.t_start = ts;
                reqs.push_back(j.req);
                charged += j.bytes;
            }
            const bool host = jobs[batch.front()].host;
            const HostArgs ha = jobs[batch.front()].ha;
            lk.unlock();
            int rc = host ? host_sort(ha.chars, ha.chars_len, ha.offsets, ha.lengths, ha.fixed_len, ha.n, ha.runs, ha.perm,
                                      ha.lcp, st)
                          : engine_sort(reqs.data(), (uint32_t)reqs.size(), st);
            const double td = now_ms();
            lk.lock();
            in_use -= charged;
            for (uint64_t t : batch) {
                ServerJob &j = jobs[t];
                j.status = rc;
                j.t_done = td;
                j.done = true;
            }
            cv_done.notify_all();
            cv_work.notify_all();   // budget freed: another worker may admit now
        }
    }
};

}  // namespace ss

using namespace ss;

extern "C" {

uint64_t ss_scratch_bytes(uint32_t n) { return n ? (uint64_t)engine_scratch_bytes(n, 1) : 0; }

int ss_server_create(uint64_t budget_bytes, uint32_t workers, uint32_t max_batch, ss_server **out) {
    if (!out || workers == 0 || workers > 64 || budget_bytes == 0) {
        set_error_detail("ss_server_create: need out != NULL, 1 <= workers <= 64, budget > 0");
        return SS_ERR_INVALID;
    }
    Server *s = new Server();
    s->budget = budget_bytes;
    s->max_batch = max_batch ? max_batch : 0xFFFFFFFFu;
    s->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&s->device);
    for (uint32_t w = 0; w < workers; w++) {
        cudaStream_t st = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            delete s;
            return cuda_fail(e, "ss_server_create: stream");
        }
        s->streams.push_back(st);
    }
    for (uint32_t w = 0; w < workers; w++) s->workers.emplace_back([s, w] { s->work(s->streams[w]); });
    *out = reinterpret_cast<ss_server *>(s);
    return SS_OK;
}

int ss_server_submit(ss_server *server, const ss_request *q, uint64_t *ticket_out) {
    Server *s = reinterpret_cast<Server *>(server);
    if (!s || !q || !ticket_out) {
        set_error_detail("ss_server_submit: NULL argument");
        return SS_ERR_INVALID;
    }
    if (q->n && (!q->chars || !q->offsets || !q->perm_out || !q->lcp_out)) {
        set_error_detail("ss_server_submit: NULL pointer with n = %u", q->n);
        return SS_ERR_INVALID;
    }
    if (q->n == 0xFFFFFFFFu) {
        set_error_detail("ss_server_submit: n = 2^32 - 1 is beyond the limit 2^32 - 2");
        return SS_ERR_TOO_LARGE;
    }
    ServerJob j;
    j.host = false;
    memset(&j.ha, 0, sizeof(j.ha));
    memset(&j.req, 0, sizeof(j.req));
    j.req.chars = q->chars;
    j.req.offsets = q->offsets;
    j.req.lengths = q->lengths;
    j.req.fixed_len = q->lengths ? 0 : q->fixed_len;
    j.req.n = q->n;
    j.req.perm_out = q->perm_out;
    j.req.lcp_out = q->lcp_out;
    j.req.status_out = q->status_out;
    j.bytes = q->n ? engine_scratch_bytes(q->n, 1) : 0;
    j.t_start = j.t_done = 0;
    j.status = SS_OK;
    j.done = false;
    return s->enqueue(j, q->n, ticket_out);
}

int ss_server_submit_host(ss_server *server, const ss_host_request *q, uint64_t *ticket_out) {
    Server *s = reinterpret_cast<Server *>(server);
    if (!s || !q || !ticket_out) {
        set_error_detail("ss_server_submit_host: NULL argument");
        return SS_ERR_INVALID;
    }
    if (q->n && (!q->chars || !q->offsets || !q->perm_out || !q->lcp_out || q->chars_len == 0)) {
        set_error_detail("ss_server_submit_host: NULL pointer or empty chars with n = %u", q->n);
        return SS_ERR_INVALID;
    }
    if (q->n == 0xFFFFFFFFu) {
        set_error_detail("ss_server_submit_host: n = 2^32 - 1 is beyond the limit 2^32 - 2");
        return SS_ERR_TOO_LARGE;
    }
    ServerJob j;
    j.host = true;
    memset(&j.req, 0, sizeof(j.req));
    j.ha = HostArgs{q->chars, q->chars_len, q->offsets, q->lengths, q->lengths ? 0u : q->fixed_len, q->n,
                    q->runs ? q->runs : 1u, q->perm_out, q->lcp_out};
    // device copies of the input, the output, the runs and their caches, the
    // merge's buffers, and the sort's scratch
    const uint64_t n = q->n;
    j.bytes = q->n ? (size_t)(q->chars_len + 32 + 8 * n + (q->lengths ? 4 * n : 0) + 16 * n +
                              (j.ha.runs > 1 ? 8 * n + 20 * n + 56 * n : 0) + engine_scratch_bytes(q->n, j.ha.runs))
                   : 0;
    j.t_start = j.t_done = 0;
    j.status = SS_OK;
    j.done = false;
    return s->enqueue(j, q->n, ticket_out);
}

int ss_server_wait(ss_server *server, uint64_t ticket, int32_t *status_out, double *times_ms_out) {
    Server *s = reinterpret_cast<Server *>(server);
    if (!s) {
        set_error_detail("ss_server_wait: NULL server");
        return SS_ERR_INVALID;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) {
        set_error_detail("ss_server_wait: unknown ticket %llu", (unsigned long long)ticket);
        return SS_ERR_INVALID;
    }
    ServerJob &jr = it->second;   // element references survive rehashing
    s->cv_done.wait(lk, [&] { return jr.done; });
    ServerJob j = jr;
    s->jobs.erase(ticket);
    if (status_out) *status_out = j.status;
    if (times_ms_out) {
        times_ms_out[0] = j.t_submit;
        times_ms_out[1] = j.t_start;
        times_ms_out[2] = j.t_done;
    }
    return SS_OK;
}

int ss_server_cancel(ss_server *server, uint64_t ticket, int32_t *cancelled_out) {
    Server *s = reinterpret_cast<Server *>(server);
    if (!s) {
        set_error_detail("ss_server_cancel: NULL server");
        return SS_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) {
        set_error_detail("ss_server_cancel: unknown ticket %llu", (unsigned long long)ticket);
        return SS_ERR_INVALID;
    }
    // only a job still in the queue can be withdrawn; it holds no budget yet
    bool cancelled = false;
    for (auto w = s->waiting.begin(); w != s->waiting.end(); ++w) {
        if (*w == ticket) {
            s->waiting.erase(w);
            ServerJob &j = it->second;
            j.status = SS_ERR_CANCELLED;
            j.t_start = j.t_done = s->now_ms();
            j.done = true;
            cancelled = true;
            break;
        }
    }
    if (cancelled) {
        s->cv_done.notify_all();
        s->cv_work.notify_all();   // the queue's head may have changed
    }
    if (cancelled_out) *cancelled_out = cancelled ? 1 : 0;
    return SS_OK;
}

int ss_server_destroy(ss_server *server) {
    Server *s = reinterpret_cast<Server *>(server);
    if (!s) return SS_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    delete s;
    return SS_OK;
}

}  // extern "C"
