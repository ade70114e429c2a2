// Serving: continuous batching of single-query requests over several CUDA
// streams, admission by candidate-buffer bytes, latency statistics.  Host
// code only; every search runs through bbc_search_ex.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "bbc_internal.cuh"

namespace bbc {
int api_error(int code, const char* msg);
int64_t index_cap(const bbc_index* ix, int nprobe);
const DevIndex& index_dev(const bbc_index* ix);
int index_device(const bbc_index* ix);
int64_t index_kc(const bbc_index* ix, int k);
}

using namespace bbc;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
    uint64_t ticket;
    std::vector<float> q;
    int32_t k, nprobe;
    int64_t bytes;
    Clock::time_point t_submit;
};

struct Result {
    std::vector<int64_t> ids;
    std::vector<float> dists;
    bool done = false;
    int status = BBC_OK;
};

struct Slot {                       // one stream and its buffers
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<Request> reqs;
    int64_t bytes = 0;
    // pinned host staging and device buffers, grown on demand
    float* hq = nullptr; int64_t* hid = nullptr; float* hd = nullptr;
    float* dq = nullptr; int64_t* did = nullptr; float* dd = nullptr;
    int64_t cap_q = 0, cap_out = 0;
    int rc = BBC_OK;
};

}  // namespace

struct bbc_server {
    bbc_index* ix = nullptr;
    bbc_serve_config cfg{};
    int device = 0, d = 0;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> pending;
    std::map<uint64_t, Result> results;
    std::vector<Slot> slots;
    uint64_t next_ticket = 1;
    bool stopping = false;
    int64_t inflight_bytes = 0, inflight_peak = 0;
    int64_t submitted = 0, completed = 0, batches = 0, batched_reqs = 0;
    std::vector<double> lat_ms;
    Clock::time_point t0;
};

namespace {

int grow(Slot& s, int64_t nq, int64_t nout, int d) {
    if (nq > s.cap_q) {
        if (s.hq) cudaFreeHost(s.hq);
        if (s.dq) cudaFree(s.dq);
        s.hq = nullptr; s.dq = nullptr;
        const int64_t c = std::max<int64_t>(nq, 2 * s.cap_q);
        if (cudaMallocHost(&s.hq, (size_t)c * d * 4) != cudaSuccess || cudaMalloc(&s.dq, (size_t)c * d * 4) != cudaSuccess)
            return BBC_ERR_OOM;
        s.cap_q = c;
    }
    if (nout > s.cap_out) {
        if (s.hid) cudaFreeHost(s.hid);
        if (s.hd) cudaFreeHost(s.hd);
        if (s.did) cudaFree(s.did);
        if (s.dd) cudaFree(s.dd);
        s.hid = nullptr; s.hd = nullptr; s.did = nullptr; s.dd = nullptr;
        const int64_t c = std::max<int64_t>(nout, 2 * s.cap_out);
        if (cudaMallocHost(&s.hid, (size_t)c * 8) != cudaSuccess || cudaMallocHost(&s.hd, (size_t)c * 4) != cudaSuccess ||
            cudaMalloc(&s.did, (size_t)c * 8) != cudaSuccess || cudaMalloc(&s.dd, (size_t)c * 4) != cudaSuccess)
            return BBC_ERR_OOM;
        s.cap_out = c;
    }
    return BBC_OK;
}

// Launch one batch on slot s (worker thread, server mutex not held).
void launch(bbc_server* sv, Slot& s) {
    const int64_t nq = (int64_t)s.reqs.size();
    int64_t nout = 0;
    std::vector<int32_t> ks(nq), ps(nq);
    for (int64_t i = 0; i < nq; ++i) { ks[i] = s.reqs[i].k; ps[i] = s.reqs[i].nprobe; nout += ks[i]; }
    s.rc = grow(s, nq, nout, sv->d);
    if (s.rc) return;
    for (int64_t i = 0; i < nq; ++i) memcpy(s.hq + i * sv->d, s.reqs[i].q.data(), (size_t)sv->d * 4);
    if (cudaMemcpyAsync(s.dq, s.hq, (size_t)nq * sv->d * 4, cudaMemcpyHostToDevice, s.stream) != cudaSuccess) {
        s.rc = BBC_ERR_CUDA;
        return;
    }
    s.rc = bbc_search_ex(sv->ix, s.dq, nq, ks.data(), ps.data(), s.did, s.dd, s.stream);
    if (s.rc) return;
    if (cudaMemcpyAsync(s.hid, s.did, (size_t)nout * 8, cudaMemcpyDeviceToHost, s.stream) != cudaSuccess ||
        cudaMemcpyAsync(s.hd, s.dd, (size_t)nout * 4, cudaMemcpyDeviceToHost, s.stream) != cudaSuccess ||
        cudaEventRecord(s.done, s.stream) != cudaSuccess)
        s.rc = BBC_ERR_CUDA;
}

// Hand a finished slot's results to the waiting requests (mutex held).
void finish(bbc_server* sv, Slot& s) {
    const auto now = Clock::now();
    int64_t off = 0;
    for (auto& r : s.reqs) {
        Result& res = sv->results[r.ticket];
        res.status = s.rc;
        if (s.rc == BBC_OK) {
            res.ids.assign(s.hid + off, s.hid + off + r.k);
            res.dists.assign(s.hd + off, s.hd + off + r.k);
        }
        res.done = true;
        off += r.k;
        sv->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r.t_submit).count());
        ++sv->completed;
    }
    sv->inflight_bytes -= s.bytes;
    s.bytes = 0;
    s.reqs.clear();
    s.busy = false;
    sv->cv_done.notify_all();
}

void worker_loop(bbc_server* sv) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        // completions
        bool any_busy = false;
        for (auto& s : sv->slots) {
            if (!s.busy) continue;
            const cudaError_t q = s.rc ? cudaSuccess : cudaEventQuery(s.done);
            if (q == cudaSuccess) finish(sv, s);
            else if (q != cudaErrorNotReady) { s.rc = BBC_ERR_CUDA; finish(sv, s); }
            else any_busy = true;
        }
        // admissions: one batch per free stream, oldest requests first
        bool launched = false;
        for (auto& s : sv->slots) {
            if (s.busy || sv->pending.empty()) continue;
            while (!sv->pending.empty() && (int)s.reqs.size() < sv->cfg.max_batch) {
                const Request& r = sv->pending.front();
                const bool alone = sv->inflight_bytes == 0 && s.reqs.empty();
                if (!alone && sv->inflight_bytes + s.bytes + r.bytes > sv->cfg.cand_bytes_budget) break;
                s.bytes += r.bytes;
                s.reqs.push_back(std::move(sv->pending.front()));
                sv->pending.pop_front();
            }
            if (s.reqs.empty()) break;                   // budget full: wait for completions
            s.busy = true;
            sv->inflight_bytes += s.bytes;
            sv->inflight_peak = std::max(sv->inflight_peak, sv->inflight_bytes);
            ++sv->batches;
            sv->batched_reqs += (int64_t)s.reqs.size();
            lk.unlock();
            launch(sv, s);
            lk.lock();
            launched = true;
            any_busy = true;
        }
        if (sv->stopping && sv->pending.empty() && !any_busy) break;
        if (!launched) {
            if (any_busy) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            } else {
                sv->cv_work.wait(lk, [&] { return sv->stopping || !sv->pending.empty(); });
            }
        }
    }
}

}  // namespace

extern "C" {

int bbc_serve_start(bbc_index* ix, const bbc_serve_config* cfg, bbc_server** out) {
    if (!ix || !cfg || !out) return api_error(BBC_ERR_ARG, "null argument");
    if (cfg->max_batch < 1 || cfg->streams < 1 || cfg->streams > 16 || cfg->cand_bytes_budget < 1)
        return api_error(BBC_ERR_ARG, "serve config out of range");
    if (index_dev(ix).quant != 0) return api_error(BBC_ERR_UNSUPPORTED, "serving: not available on a sign-code index");
    auto* sv = new bbc_server();
    sv->ix = ix;
    sv->cfg = *cfg;
    sv->device = index_device(ix);
    sv->d = index_dev(ix).d;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(sv->device);
    sv->slots.resize(cfg->streams);
    for (auto& s : sv->slots) {
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) {
            if (prev >= 0) cudaSetDevice(prev);
            delete sv;
            return api_error(BBC_ERR_CUDA, "stream creation failed");
        }
    }
    if (prev >= 0) cudaSetDevice(prev);
    sv->t0 = Clock::now();
    sv->worker = std::thread(worker_loop, sv);
    *out = sv;
    return BBC_OK;
}

int bbc_serve_submit(bbc_server* sv, const float* host_query, int32_t k, int32_t nprobe, uint64_t* ticket) {
    if (!sv || !host_query || !ticket) return api_error(BBC_ERR_ARG, "null argument");
    const DevIndex& d = index_dev(sv->ix);
    if (k < 1) return api_error(BBC_ERR_ARG, "k must be >= 1");
    if (nprobe < 1 || nprobe > d.nlist || nprobe > 2048) return api_error(BBC_ERR_ARG, "nprobe out of range");
    Request r;
    r.q.assign(host_query, host_query + d.d);
    r.k = k;
    r.nprobe = nprobe;
    r.bytes = 8 * index_cap(sv->ix, nprobe) + 8 * index_kc(sv->ix, k);
    r.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stopping) return api_error(BBC_ERR_BUSY, "server is stopping");
        r.ticket = sv->next_ticket++;
        *ticket = r.ticket;
        sv->results[r.ticket] = Result{};
        sv->pending.push_back(std::move(r));
        ++sv->submitted;
    }
    sv->cv_work.notify_one();
    return BBC_OK;
}

int bbc_serve_poll(bbc_server* sv, uint64_t ticket, int64_t* ids, float* dists, int32_t timeout_ms) {
    if (!sv || !ids || !dists) return api_error(BBC_ERR_ARG, "null argument");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->results.find(ticket);
    if (it == sv->results.end()) return api_error(BBC_ERR_ARG, "unknown ticket");
    auto ready = [&] { return sv->results[ticket].done; };
    if (timeout_ms < 0) sv->cv_done.wait(lk, ready);
    else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return api_error(BBC_ERR_TIMEOUT, "result not ready");
    Result& r = sv->results[ticket];
    const int st = r.status;
    if (st == BBC_OK) {
        memcpy(ids, r.ids.data(), r.ids.size() * 8);
        memcpy(dists, r.dists.data(), r.dists.size() * 4);
    }
    sv->results.erase(ticket);
    return st == BBC_OK ? BBC_OK : api_error(st, "batch failed");
}

int bbc_serve_stats(bbc_server* sv, bbc_serve_stats_t* out) {
    if (!sv || !out) return api_error(BBC_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = sv->submitted;
    out->completed = sv->completed;
    out->batches = sv->batches;
    out->inflight_bytes_peak = sv->inflight_peak;
    out->mean_batch = sv->batches ? (double)sv->batched_reqs / sv->batches : 0.0;
    out->wall_s = std::chrono::duration<double>(Clock::now() - sv->t0).count();
    if (!sv->lat_ms.empty()) {
        std::vector<double> v = sv->lat_ms;
        auto pct = [&](double p) {
            const size_t i = std::min(v.size() - 1, (size_t)(p * (double)(v.size() - 1) + 0.5));
            std::nth_element(v.begin(), v.begin() + (long)i, v.end());
            return v[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
    }
    return BBC_OK;
}

int bbc_serve_stop(bbc_server* sv) {
    if (!sv) return api_error(BBC_ERR_ARG, "null server");
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(sv->device);
    for (auto& s : sv->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.hq) cudaFreeHost(s.hq);
        if (s.hid) cudaFreeHost(s.hid);
        if (s.hd) cudaFreeHost(s.hd);
        if (s.dq) cudaFree(s.dq);
        if (s.did) cudaFree(s.did);
        if (s.dd) cudaFree(s.dd);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
    }
    if (prev >= 0) cudaSetDevice(prev);
    delete sv;
    return BBC_OK;
}

}  // extern "C"
