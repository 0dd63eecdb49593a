// Serving loop: continuous batching of independent solve requests on one
// device (mrrr_serve_* in include/mrrr.h).  Host threads ("workers"), each
// with its own stream, repeatedly admit the oldest pending requests of one
// precision and mode within the device-byte budget and run them as one
// batched solve; requests that arrive meanwhile wait for the next free
// worker, so batches overlap on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mrrr.h"
#include "mrrr_entry.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

bool is_device(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct Req {
    long long ticket = 0;
    mrrr_request r{};
    size_t xs = 4;                 // bytes per value of the request's precision
    int k = 0;                     // eigenpairs asked for
    std::vector<char> d_host, e_host;  // host inputs, copied at submit
    bool in_dev = false, out_dev = false;
    size_t bytes = 0;              // device bytes charged while admitted
    Clock::time_point t_submit, t_admit, t_done;
    int status = 0, m = 0, batch = 0;
    bool done = false;
    cudaEvent_t ready = nullptr;   // recorded on the caller's stream at submit (device buffers)
    ~Req() {
        if (ready) cudaEventDestroy(ready);
    }
};

// Device bytes a request holds while it runs: its inputs (when copied in),
// device copies of host outputs, and the solver's per-matrix data -- the
// representation (4 n working-precision words plus its low copy), the
// scaled input, per-item records and lists, and the RQI scratch of 2 n
// working-precision words per eigenpair (bounded by the solver's 4 GiB wave).
size_t charge(const Req& q) {
    const size_t n = (size_t)q.r.n, k = (size_t)q.k, xs = q.xs;
    const size_t ys = (q.r.mode == MRRR_MIXED) ? 2 * xs : xs;
    size_t b = 0;
    if (!q.in_dev) b += 2 * n * xs;
    if (!q.out_dev) b += (n * k + k) * xs;
    b += n * (6 * ys + 32) + k * 256;
    b += std::min<size_t>(2 * n * k * ys, (size_t)4 << 30);
    return b + 4096;
}

}  // namespace

struct mrrr_server {
    mrrr_serve_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req*> pending;
    std::unordered_map<long long, Req*> live;
    size_t budget = 0, in_use = 0;
    long long next_ticket = 1;
    bool closing = false;
    std::vector<std::thread> workers;
    std::vector<double> latencies;
    long long eigenpairs = 0, batches = 0;
    std::atomic<int> alloc_failures{0};  // test hook: batches still to fail as out of memory
    bool started = false;
    Clock::time_point t_first, t_last;

    void worker_main();
    void run_batch(std::vector<Req*>& batch, cudaStream_t st, char*& pinned, size_t& pinned_cap);
};

void mrrr_server::run_batch(std::vector<Req*>& batch, cudaStream_t st, char*& pinned, size_t& pinned_cap) {
    const int nb = (int)batch.size();
    const bool dbl = batch[0]->r.precision == 1;
    const size_t xs = dbl ? 8 : 4;
    // one device block for the inputs given on the host and one for the
    // device copies of outputs that go back to the host
    size_t in_bytes = 0, out_bytes = 0;
    std::vector<size_t> in_off(nb), w_off(nb), z_off(nb);
    for (int p = 0; p < nb; ++p) {
        const Req& q = *batch[p];
        const size_t n = (size_t)q.r.n, k = (size_t)q.k;
        if (!q.in_dev) {
            in_off[p] = in_bytes;
            in_bytes += (2 * n * xs + 255) / 256 * 256;
        }
        if (!q.out_dev) {
            w_off[p] = out_bytes;
            out_bytes += (k * xs + 255) / 256 * 256;
            z_off[p] = out_bytes;
            out_bytes += (n * k * xs + 255) / 256 * 256;
        }
    }
    int rc = MRRR_OK;
    char* din = nullptr;
    char* dout = nullptr;
    // test hook: this batch fails as if its device allocation had
    if (alloc_failures.load() > 0 && alloc_failures.fetch_sub(1) > 0) rc = MRRR_ERR_NOMEM;
    // device buffers: after the caller's work queued before submit
    for (int p = 0; p < nb && rc == MRRR_OK; ++p)
        if (batch[p]->ready && cudaStreamWaitEvent(st, batch[p]->ready, 0) != cudaSuccess) rc = MRRR_ERR_CUDA;
    if (in_bytes && rc == MRRR_OK) {
        if (pinned_cap < in_bytes) {
            if (pinned) cudaFreeHost(pinned);
            pinned = nullptr;
            pinned_cap = 0;
            if (cudaHostAlloc((void**)&pinned, in_bytes, cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                pinned = nullptr;
                rc = MRRR_ERR_NOMEM;
            } else {
                pinned_cap = in_bytes;
            }
        }
        if (rc == MRRR_OK) {
            for (int p = 0; p < nb; ++p) {
                const Req& q = *batch[p];
                if (q.in_dev) continue;
                std::memcpy(pinned + in_off[p], q.d_host.data(), q.d_host.size());
                if (!q.e_host.empty()) std::memcpy(pinned + in_off[p] + q.r.n * xs, q.e_host.data(), q.e_host.size());
            }
            if (!(din = (char*)mrrr::dev_alloc(in_bytes, st))) rc = MRRR_ERR_NOMEM;
            else if (cudaMemcpyAsync(din, pinned, in_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
                rc = MRRR_ERR_CUDA;
        }
    }
    if (rc == MRRR_OK && out_bytes && !(dout = (char*)mrrr::dev_alloc(out_bytes, st))) rc = MRRR_ERR_NOMEM;
    std::vector<int> n(nb), il(nb), iu(nb), ldz(nb), m(nb, 0), status(nb, MRRR_OK);
    std::vector<const void*> d(nb), e(nb);
    std::vector<void*> W(nb), Z(nb);
    for (int p = 0; p < nb; ++p) {
        const Req& q = *batch[p];
        n[p] = q.r.n;
        il[p] = q.r.il > 0 ? q.r.il : 1;
        iu[p] = q.r.il > 0 ? q.r.iu : q.r.n;
        if (q.in_dev) {
            d[p] = q.r.d;
            e[p] = q.r.n > 1 ? q.r.e : nullptr;
        } else {
            d[p] = din + in_off[p];
            e[p] = q.r.n > 1 ? (const void*)(din + in_off[p] + q.r.n * xs) : nullptr;
        }
        if (q.out_dev) {
            W[p] = q.r.W;
            Z[p] = q.r.Z;
            ldz[p] = q.r.ldz;
        } else {
            W[p] = dout + w_off[p];
            Z[p] = dout + z_off[p];
            ldz[p] = q.r.n;
        }
    }
    const mrrr_mode mode = batch[0]->r.mode;
    if (rc == MRRR_OK) {
        if (dbl)
            rc = mrrr_solve_batch_d(nb, n.data(), (const double* const*)d.data(), (const double* const*)e.data(),
                                    il.data(), iu.data(), mode, nullptr, m.data(), (double* const*)W.data(),
                                    (double* const*)Z.data(), ldz.data(), status.data(), st);
        else
            rc = mrrr_solve_batch_s(nb, n.data(), (const float* const*)d.data(), (const float* const*)e.data(),
                                    il.data(), iu.data(), mode, nullptr, m.data(), (float* const*)W.data(),
                                    (float* const*)Z.data(), ldz.data(), status.data(), st);
    }
    // host outputs: W, then Z column by column into the caller's ldz
    bool copy_fail = false;
    if (rc != MRRR_ERR_CUDA && rc != MRRR_ERR_NOMEM && dout) {
        for (int p = 0; p < nb && !copy_fail; ++p) {
            const Req& q = *batch[p];
            if (q.out_dev || m[p] <= 0) continue;
            if (cudaMemcpyAsync(q.r.W, W[p], (size_t)m[p] * xs, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaMemcpy2DAsync(q.r.Z, (size_t)q.r.ldz * xs, Z[p], (size_t)q.r.n * xs, (size_t)q.r.n * xs,
                                  (size_t)m[p], cudaMemcpyDeviceToHost, st) != cudaSuccess)
                copy_fail = true;
        }
    }
    mrrr::dev_free(din, st);
    mrrr::dev_free(dout, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) copy_fail = true;
    if (copy_fail) cudaGetLastError();
    const auto t = Clock::now();
    std::lock_guard<std::mutex> lk(mu);
    for (int p = 0; p < nb; ++p) {
        Req& q = *batch[p];
        if (copy_fail || rc == MRRR_ERR_CUDA || rc == MRRR_ERR_NOMEM) q.status = copy_fail ? MRRR_ERR_CUDA : rc;
        else q.status = status[p];
        q.m = m[p];
        q.batch = nb;
        q.t_done = t;
        q.done = true;
        in_use -= q.bytes;
        latencies.push_back(ms_between(q.t_submit, t));
        eigenpairs += m[p];
    }
    ++batches;
    t_last = t;
}

void mrrr_server::worker_main() {
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        st = nullptr;
    }
    char* pinned = nullptr;
    size_t pinned_cap = 0;
    for (;;) {
        std::vector<Req*> batch;
        {
            std::unique_lock<std::mutex> lk(mu);
            // the oldest request is admitted when it fits, or alone when it is
            // larger than the whole budget and nothing else is admitted
            cv_work.wait(lk, [&] {
                if (pending.empty()) return closing;
                const Req* h = pending.front();
                return in_use + h->bytes <= budget || in_use == 0;
            });
            if (pending.empty()) break;  // closing and drained
            const int prec = pending.front()->r.precision;
            const mrrr_mode mode = pending.front()->r.mode;
            const auto t = Clock::now();
            for (auto it = pending.begin(); it != pending.end() && (int)batch.size() < cfg.max_batch;) {
                Req* q = *it;
                if (q->r.precision != prec || q->r.mode != mode) {
                    ++it;
                    continue;
                }
                if (!batch.empty() && in_use + q->bytes > budget) break;  // keep arrival order within the kind
                in_use += q->bytes;
                q->t_admit = t;
                batch.push_back(q);
                it = pending.erase(it);
            }
            if (!started) {
                started = true;
                t_first = t;
            }
        }
        if (st) {
            run_batch(batch, st, pinned, pinned_cap);
        } else {
            std::lock_guard<std::mutex> lk(mu);
            for (Req* q : batch) {
                q->status = MRRR_ERR_CUDA;
                q->done = true;
                q->t_done = Clock::now();
                in_use -= q->bytes;
            }
        }
        cv_done.notify_all();
        cv_work.notify_all();
    }
    if (pinned) cudaFreeHost(pinned);
    if (st) cudaStreamDestroy(st);
}

extern "C" int mrrr_serve_open(const mrrr_serve_config* cfg, mrrr_server** out) {
    if (!out) return MRRR_ERR_ARG;
    *out = nullptr;
    mrrr_serve_config c{};
    if (cfg) c = *cfg;
    if (c.workers < 0 || c.max_batch < 0 || c.hbm_budget < 0) return MRRR_ERR_ARG;
    if (c.workers == 0) c.workers = 2;
    if (c.max_batch == 0) c.max_batch = 512;
    int devs = 0, dev = 0;
    if (cudaGetDeviceCount(&devs) != cudaSuccess || devs == 0 || cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return MRRR_ERR_CUDA;
    }
    size_t fr = 0, tot = 0;
    if (c.hbm_budget == 0) {
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            return MRRR_ERR_CUDA;
        }
        c.hbm_budget = (long long)(fr / 2);
    }
    mrrr_server* s = new mrrr_server();
    s->cfg = c;
    s->device = dev;
    s->budget = (size_t)c.hbm_budget;
    s->alloc_failures = std::max(c.alloc_failures, 0);
    for (int w = 0; w < c.workers; ++w) s->workers.emplace_back([s] { s->worker_main(); });
    *out = s;
    return MRRR_OK;
}

extern "C" int mrrr_serve_submit(mrrr_server* s, const mrrr_request* req, long long* ticket) {
    if (!s || !req || !ticket) return MRRR_ERR_ARG;
    const mrrr_request& r = *req;
    if ((r.precision != 0 && r.precision != 1) || (r.mode != MRRR_MIXED && r.mode != MRRR_PLAIN)) return MRRR_ERR_ARG;
    if (r.n < 1 || !r.d || (r.n > 1 && !r.e) || !r.W || !r.Z || r.ldz < r.n) return MRRR_ERR_ARG;
    if (r.il != 0 && (r.il < 1 || r.iu > r.n || r.il > r.iu)) return MRRR_ERR_ARG;
    Req* q = new Req();
    q->r = r;
    q->xs = r.precision == 1 ? 8 : 4;
    q->k = r.il > 0 ? r.iu - r.il + 1 : r.n;
    const bool dd = is_device(r.d), de = r.n == 1 ? dd : is_device(r.e);
    const bool ow = is_device(r.W), oz = is_device(r.Z);
    if (dd != de || ow != oz) {
        delete q;
        return MRRR_ERR_ARG;  // inputs (and outputs) both on the device or both on the host
    }
    q->in_dev = dd;
    q->out_dev = ow;
    if (!dd) {
        q->d_host.assign((const char*)r.d, (const char*)r.d + r.n * q->xs);
        if (r.n > 1) q->e_host.assign((const char*)r.e, (const char*)r.e + (r.n - 1) * q->xs);
    }
    if (dd || ow) {
        if (cudaEventCreateWithFlags(&q->ready, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(q->ready, (cudaStream_t)r.stream) != cudaSuccess) {
            cudaGetLastError();
            delete q;
            return MRRR_ERR_CUDA;
        }
    }
    q->bytes = charge(*q);
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->closing) {
            delete q;
            return MRRR_ERR_ARG;
        }
        q->ticket = s->next_ticket++;
        s->live[q->ticket] = q;
        s->pending.push_back(q);
        *ticket = q->ticket;
    }
    s->cv_work.notify_one();
    return MRRR_OK;
}

extern "C" int mrrr_serve_poll(mrrr_server* s, long long ticket, int wait_ms, mrrr_serve_info* info) {
    if (!s) return MRRR_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->live.find(ticket);
    if (it == s->live.end()) return MRRR_ERR_ARG;
    Req* q = it->second;
    auto ready = [&] { return q->done; };
    if (wait_ms < 0) s->cv_done.wait(lk, ready);
    else if (wait_ms > 0) s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), ready);
    if (!q->done) return MRRR_PENDING;
    if (info) {
        info->status = q->status;
        info->m = q->m;
        info->batch = q->batch;
        info->queue_ms = ms_between(q->t_submit, q->t_admit);
        info->latency_ms = ms_between(q->t_submit, q->t_done);
    }
    int st = q->status;
    s->live.erase(it);
    delete q;
    return st;
}

extern "C" int mrrr_serve_cancel(mrrr_server* s, long long ticket) {
    if (!s) return MRRR_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->live.find(ticket);
        if (it == s->live.end()) return MRRR_ERR_ARG;
        Req* q = it->second;
        auto p = std::find(s->pending.begin(), s->pending.end(), q);
        if (p == s->pending.end()) return MRRR_PENDING;  // admitted or done: poll it
        s->pending.erase(p);
        q->status = MRRR_ERR_CANCELLED;
        q->t_admit = q->t_done = Clock::now();
        q->done = true;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
    return MRRR_OK;
}

extern "C" int mrrr_serve_stats_get(mrrr_server* s, mrrr_serve_stats* out) {
    if (!s || !out) return MRRR_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->completed = (long long)s->latencies.size();
    out->eigenpairs = s->eigenpairs;
    out->batches = s->batches;
    if (!s->latencies.empty()) {
        std::vector<double> v = s->latencies;
        std::sort(v.begin(), v.end());
        // nearest rank: the smallest value with at least a fraction p at or below it
        auto pct = [&](double p) {
            size_t r = (size_t)std::ceil(p * (double)v.size());
            return v[std::min(v.size(), std::max<size_t>(r, 1)) - 1];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = v.back();
        out->busy_s = std::chrono::duration<double>(s->t_last - s->t_first).count();
    }
    return MRRR_OK;
}

extern "C" int mrrr_serve_close(mrrr_server* s) {
    if (!s) return MRRR_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->closing = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->live) delete kv.second;
    delete s;
    return MRRR_OK;
}
