// Request serving: admission by a device-memory budget, concurrent worker
// streams, a cache of source-side plans, and batches of the queued requests that
// query one cached plan (include/slk_serve.h).
//
// The server uses the library's public calls (slk_plan_create, slk_sum,
// slk_plan_sync, slk_plan_destroy), one CUDA stream per worker thread.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "slk_serve.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

int64_t round8(int64_t v) { return (v + 7) / 8 * 8; }

struct CacheEntry {
    uint64_t key = 0;
    slk_plan plan = nullptr;
    int64_t bytes = 0;
    int refs = 0;
    bool ready = false;  // false while the request that builds it runs
    bool failed = false;
    uint64_t last_use = 0;
    std::mutex use;  // one call at a time on a plan
};

struct Request {
    uint64_t id = 0;
    slk_request req{};
    int64_t need = 0;  // reserved bytes while running
    bool cached = false;
    int batch = 1;  // requests served by the same launches (the cached plan's sum)
    bool done = false;
    slk_status status = SLK_OK;
    std::string message;
    Clock::time_point t_submit, t_start, t_done;
};

}  // namespace

struct slk_server_s {
    int device = 0;
    int64_t budget = 0, cache_cap = 0;
    int64_t in_use = 0, cache_bytes = 0;
    uint64_t next_id = 1, tick = 0;
    bool stop = false;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> pending;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> all;
    std::unordered_map<uint64_t, std::unique_ptr<CacheEntry>> cache;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;  // one per worker; destroyed after the cached plans

    void worker_loop(int index);
    bool waits_for_build(const Request* r) const;
    bool try_admit(Request* r);
    std::vector<Request*> take_batch(Request* first);
    void run_batch(const std::vector<Request*>& batch, CacheEntry* entry, cudaStream_t st);
    void evict_for(int64_t need);
    void finish(Request* r, CacheEntry* entry, slk_plan plan, bool keep_plan, int64_t plan_bytes);
};

extern "C" int64_t slk_request_bytes(const slk_plan_desc* desc, int64_t N, int64_t M) {
    if (!desc || N < 0 || M < 0) return -1;
    const int64_t e = desc->precision == SLK_PREC_F64 ? 8 : 4;
    const int64_t P = desc->P, d = desc->d;
    const int tc = desc->precision == SLK_PREC_BF16 ? 1 : (desc->precision == SLK_PREC_F16X3 ? 2 : 0);
    const int64_t ld16 = round8(d);
    int64_t base = P * d * 12 + 64 * d + (1 << 20);
    if (tc) base += P * ld16 * 2 * tc + d * round8(P) * 2;
    const int64_t stage_x = N * d * e + N * e;
    int64_t create = stage_x + P * N * e + (tc ? N * ld16 * 2 * tc : 0);
    int64_t persist = 0;
    if (desc->kernel != SLK_NEGDIST) {
        const int64_t grids = P * 16384 * e * 2;  // NFFT/NDFT plan state and scratch (bounded by the grid size)
        create += grids + P * e * 256 * (N / 32768 + 2);
        persist += grids;
    }
    if (desc->kernel == SLK_NEGDIST || desc->kernel == SLK_LAPLACIAN) {
        const int64_t NB = N / 4 + 2;  // the plan's bucket count: a power of two >= N / 8
        const int64_t sort = P * N * (e + 4) + 2 * P * N * e + P * N * 4 + P * 256 * (N / 4096 + 1) * 4;
        const int64_t keep = P * N * 2 * e + P * NB * 32;  // 32-byte bucket records
        create += sort + keep;
        persist += keep;
    }
    const int64_t sum = M * d * e + P * M * e * 2 + M * 8 + M * e + (tc ? M * ld16 * 2 * tc : 0);
    return base + std::max(create, persist + sum);
}

// A request whose sources' plan another request is building stays queued behind that build
// (so that it runs on the cached plan) without holding up the requests queued after it.
bool slk_server_s::waits_for_build(const Request* r) const {
    if (!r->req.source_key) return false;
    auto it = cache.find(r->req.source_key);
    return it != cache.end() && !it->second->ready && !it->second->failed;
}

bool slk_server_s::try_admit(Request* r) {
    const slk_request& q = r->req;
    CacheEntry* entry = nullptr;
    if (q.source_key) {
        auto it = cache.find(q.source_key);
        if (it != cache.end()) {
            entry = it->second.get();
            if (!entry->ready && !entry->failed) return false;  // another request is building it
            if (entry->failed) entry = nullptr;
        }
    }
    int64_t need = entry ? slk_request_bytes(&q.desc, 0, q.M) : slk_request_bytes(&q.desc, q.N, q.M);
    if (in_use + need > budget) evict_for(need);
    if (in_use + need > budget) return false;
    in_use += need;
    r->need = need;
    r->cached = entry != nullptr;
    if (entry) {
        entry->refs++;
        entry->last_use = ++tick;
    } else if (q.source_key) {
        auto e = std::make_unique<CacheEntry>();
        e->key = q.source_key;
        e->refs = 1;
        e->last_use = ++tick;
        cache[q.source_key] = std::move(e);
    }
    return true;
}

// Requests that query the same cached plan share its sum: after `first` (admitted on a ready
// cached plan) the queued requests with the same source key are admitted too, in order, as
// long as memory allows, up to kMaxBatch requests and kMaxBatchRows targets in all.
constexpr size_t kMaxBatch = 32;
constexpr int64_t kMaxBatchRows = int64_t(1) << 22;

std::vector<Request*> slk_server_s::take_batch(Request* first) {
    std::vector<Request*> batch{first};
    if (!first->cached) return batch;
    int64_t rows = first->req.M;
    for (auto it = pending.begin(); it != pending.end() && batch.size() < kMaxBatch;) {
        Request* q = *it;
        if (q->req.source_key != first->req.source_key || rows + q->req.M > kMaxBatchRows) {
            ++it;
            continue;
        }
        if (!try_admit(q)) break;
        q->t_start = first->t_start;
        rows += q->req.M;
        batch.push_back(q);
        it = pending.erase(it);
    }
    for (Request* q : batch) q->batch = static_cast<int>(batch.size());
    return batch;
}

// One sum over the concatenated targets of a batch on the cached plan: the targets are
// gathered into one array, summed, and each request's outputs copied back.
void slk_server_s::run_batch(const std::vector<Request*>& batch, CacheEntry* entry, cudaStream_t st) {
    const slk_plan_desc& desc = batch[0]->req.desc;
    const int64_t e = desc.precision == SLK_PREC_F64 ? 8 : 4, d = desc.d;
    int64_t rows = 0;
    for (Request* q : batch) rows += q->req.M;
    slk_status s = SLK_OK;
    std::string msg;
    void* ycat = nullptr;
    void* scat = nullptr;
    if (cudaMallocAsync(&ycat, static_cast<size_t>(rows * d * e), st) != cudaSuccess ||
        cudaMallocAsync(&scat, static_cast<size_t>(rows * e), st) != cudaSuccess) {
        cudaGetLastError();
        s = SLK_ERR_OOM;
        msg = "device allocation for a batch of requests failed";
    }
    int64_t off = 0;
    for (Request* q : batch) {
        if (s != SLK_OK) break;
        if (cudaMemcpy2DAsync(static_cast<char*>(ycat) + off * d * e, d * e, q->req.y, q->req.ldy * e, d * e,
                              q->req.M, cudaMemcpyDefault, st) != cudaSuccess) {
            cudaGetLastError();
            s = SLK_ERR_CUDA;
            msg = "gathering the targets of a batch failed";
        }
        off += q->req.M;
    }
    if (s == SLK_OK) {
        std::lock_guard<std::mutex> use(entry->use);
        s = slk_sum(entry->plan, ycat, rows, d, scat, st);
        if (s == SLK_OK) s = slk_plan_sync(entry->plan);
        if (s != SLK_OK) msg = slk_last_error();
    }
    off = 0;
    for (Request* q : batch) {
        if (s != SLK_OK) break;
        if (cudaMemcpyAsync(q->req.s, static_cast<char*>(scat) + off * e, static_cast<size_t>(q->req.M * e),
                            cudaMemcpyDefault, st) != cudaSuccess) {
            cudaGetLastError();
            s = SLK_ERR_CUDA;
            msg = "returning the outputs of a batch failed";
        }
        off += q->req.M;
    }
    if (ycat) cudaFreeAsync(ycat, st);
    if (scat) cudaFreeAsync(scat, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && s == SLK_OK) {
        cudaGetLastError();
        s = SLK_ERR_CUDA;
        msg = "a batch of requests failed on the device";
    }
    for (Request* q : batch) {
        q->status = s;
        q->message = msg;
        finish(q, entry, nullptr, false, 0);
    }
}

void slk_server_s::evict_for(int64_t need) {
    while (in_use + need > budget) {
        CacheEntry* victim = nullptr;
        for (auto& kv : cache) {
            CacheEntry* c = kv.second.get();
            if (c->ready && c->refs == 0 && (!victim || c->last_use < victim->last_use)) victim = c;
        }
        if (!victim) return;
        slk_plan_destroy(victim->plan);
        in_use -= victim->bytes;
        cache_bytes -= victim->bytes;
        cache.erase(victim->key);
    }
}

void slk_server_s::finish(Request* r, CacheEntry* entry, slk_plan plan, bool keep_plan, int64_t plan_bytes) {
    std::lock_guard<std::mutex> g(mu);
    in_use -= r->need;
    if (entry) {
        entry->refs--;
        if (!entry->ready) {
            if (keep_plan) {
                entry->plan = plan;
                entry->bytes = plan_bytes;
                entry->ready = true;
                in_use += plan_bytes;
                cache_bytes += plan_bytes;
            } else {
                cache.erase(entry->key);
            }
        }
    }
    r->t_done = Clock::now();
    r->done = true;
    cv.notify_all();
}

void slk_server_s::worker_loop(int index) {
    cudaSetDevice(device);
    cudaStream_t st = streams[index];
    for (;;) {
        Request* r = nullptr;
        std::vector<Request*> batch;
        {
            // admit the oldest admissible queued request as soon as memory allows: requests
            // waiting for a plan under construction are passed over (they stay queued), the
            // first one that does not fit the budget ends the scan (nothing overtakes it)
            std::unique_lock<std::mutex> lk(mu);
            for (;;) {
                for (auto it = pending.begin(); it != pending.end(); ++it) {
                    if (waits_for_build(*it)) continue;
                    if (try_admit(*it)) {
                        r = *it;
                        pending.erase(it);
                    }
                    break;
                }
                if (r) break;
                if (stop && pending.empty()) break;
                cv.wait(lk);  // woken by a submission, a finished request or shutdown
            }
            if (!r) break;
            r->t_start = Clock::now();
            batch = take_batch(r);
        }
        cv.notify_all();
        if (batch.size() > 1) {
            CacheEntry* entry = nullptr;
            {
                std::lock_guard<std::mutex> g(mu);
                entry = cache.find(r->req.source_key)->second.get();
            }
            run_batch(batch, entry, st);
            continue;
        }
        const slk_request& q = r->req;
        CacheEntry* entry = nullptr;
        if (q.source_key) {
            std::lock_guard<std::mutex> g(mu);
            auto it = cache.find(q.source_key);
            if (it != cache.end()) entry = it->second.get();
        }
        slk_plan plan = (entry && r->cached) ? entry->plan : nullptr;
        slk_status s = SLK_OK;
        std::string msg;
        bool keep = false;
        int64_t plan_bytes = 0;
        if (!plan) {
            s = slk_plan_create(&plan, &q.desc, q.x, q.N, q.ldx, q.w, st);
            if (s != SLK_OK) msg = slk_last_error();
        }
        if (s == SLK_OK) {
            std::unique_lock<std::mutex> use_lk;
            if (entry) use_lk = std::unique_lock<std::mutex>(entry->use);
            s = slk_sum(plan, q.y, q.M, q.ldy, q.s, st);
            if (s == SLK_OK) s = slk_plan_sync(plan);
            if (s != SLK_OK) msg = slk_last_error();
        }
        if (plan && !r->cached) {
            slk_plan_info info;
            if (entry && s == SLK_OK && slk_plan_get_info(plan, &info) == SLK_OK) {
                std::lock_guard<std::mutex> g(mu);
                plan_bytes = info.device_bytes;
                // room for the new plan: the least recently used cached plans no request holds go
                while (cache_bytes + plan_bytes > cache_cap && plan_bytes <= cache_cap) {
                    CacheEntry* victim = nullptr;
                    for (auto& kv : cache) {
                        CacheEntry* c = kv.second.get();
                        if (c->ready && c->refs == 0 && (!victim || c->last_use < victim->last_use)) victim = c;
                    }
                    if (!victim) break;
                    slk_plan_destroy(victim->plan);
                    in_use -= victim->bytes;
                    cache_bytes -= victim->bytes;
                    cache.erase(victim->key);
                }
                keep = cache_bytes + plan_bytes <= cache_cap;
            }
            if (!keep) slk_plan_destroy(plan);
        }
        r->status = s;
        r->message = msg;
        finish(r, entry, plan, keep, plan_bytes);
    }
    cudaStreamSynchronize(st);
}

using slk::Error;

namespace {
template <class Fn>
slk_status guarded_serve(Fn&& fn) {
    try {
        fn();
        return SLK_OK;
    } catch (const Error& e) {
        slk::set_last_error(e.msg);
        return e.status;
    } catch (const std::bad_alloc&) {
        slk::set_last_error("host allocation failed");
        return SLK_ERR_OOM;
    } catch (...) {
        slk::set_last_error("unexpected exception");
        return SLK_ERR_CUDA;
    }
}
}  // namespace

extern "C" {

slk_status slk_serve_create(slk_server* out, const slk_serve_desc* desc) {
    slk::set_last_error("");
    return guarded_serve([&] {
        SLK_REQUIRE(out, "server output pointer is NULL");
        *out = nullptr;
        slk_serve_desc dd{};
        if (desc) dd = *desc;
        SLK_REQUIRE(dd.workers >= 0 && dd.workers <= 64, "workers must be in [0, 64]");
        SLK_REQUIRE(dd.memory_budget >= 0 && dd.plan_cache_bytes >= 0, "budgets must be >= 0");
        auto srv = std::make_unique<slk_server_s>();
        SLK_CHECK_CUDA(cudaGetDevice(&srv->device));
        size_t free_b = 0, total_b = 0;
        SLK_CHECK_CUDA(cudaMemGetInfo(&free_b, &total_b));
        srv->budget = dd.memory_budget ? dd.memory_budget : static_cast<int64_t>(0.8 * static_cast<double>(free_b));
        srv->cache_cap = dd.plan_cache_bytes ? std::min(dd.plan_cache_bytes, srv->budget) : srv->budget / 4;
        const int nw = dd.workers ? dd.workers : 4;
        for (int i = 0; i < nw; ++i) {
            cudaStream_t st = nullptr;
            SLK_CHECK_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            srv->streams.push_back(st);
        }
        slk_server_s* raw = srv.get();
        for (int i = 0; i < nw; ++i) srv->workers.emplace_back([raw, i] { raw->worker_loop(i); });
        *out = srv.release();
    });
}

slk_status slk_serve_submit(slk_server srv, const slk_request* req, uint64_t* id) {
    slk::set_last_error("");
    return guarded_serve([&] {
        SLK_REQUIRE(srv && req && id, "server, request and id must not be NULL");
        SLK_REQUIRE(req->x && req->w && req->y && req->s, "request buffers must not be NULL");
        SLK_REQUIRE(req->N >= 1 && req->M >= 1 && req->ldx >= req->desc.d && req->ldy >= req->desc.d,
                    "bad request sizes");
        const int64_t need = slk_request_bytes(&req->desc, req->N, req->M);
        SLK_REQUIRE(need > 0, "bad request descriptor");
        if (need > srv->budget)
            slk::fail(SLK_ERR_OOM, "request needs about %lld bytes, more than the server budget of %lld",
                      static_cast<long long>(need), static_cast<long long>(srv->budget));
        auto r = std::make_unique<Request>();
        r->req = *req;
        r->t_submit = Clock::now();
        {
            std::lock_guard<std::mutex> g(srv->mu);
            SLK_REQUIRE(!srv->stop, "server is shutting down");
            r->id = srv->next_id++;
            *id = r->id;
            srv->pending.push_back(r.get());
            srv->all[r->id] = std::move(r);
        }
        srv->cv.notify_all();
    });
}

slk_status slk_serve_poll(slk_server srv, uint64_t id, int64_t timeout_us, slk_result* res) {
    slk::set_last_error("");
    if (!srv || !res) return SLK_ERR_INVALID;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->all.find(id);
    if (it == srv->all.end()) return SLK_ERR_NOT_FOUND;
    Request* r = it->second.get();
    if (!r->done) {
        if (timeout_us == 0) return SLK_ERR_TIMEOUT;
        if (timeout_us < 0) srv->cv.wait(lk, [&] { return r->done; });
        else if (!srv->cv.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->done; }))
            return SLK_ERR_TIMEOUT;
    }
    std::memset(res, 0, sizeof(*res));
    res->status = r->status;
    res->plan_cached = r->cached ? 1 : 0;
    res->batch_requests = r->batch;
    res->queue_ms = ms_between(r->t_submit, r->t_start);
    res->run_ms = ms_between(r->t_start, r->t_done);
    res->total_ms = ms_between(r->t_submit, r->t_done);
    std::strncpy(res->message, r->message.c_str(), sizeof(res->message) - 1);
    srv->all.erase(it);
    return SLK_OK;
}

slk_status slk_serve_destroy(slk_server srv) {
    if (!srv) return SLK_OK;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        srv->stop = true;
    }
    srv->cv.notify_all();
    for (auto& t : srv->workers) t.join();
    // cached plans free their memory on the streams that built them: before those streams go
    for (auto& kv : srv->cache)
        if (kv.second->plan) slk_plan_destroy(kv.second->plan);
    srv->cache.clear();
    for (cudaStream_t st : srv->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    delete srv;
    return SLK_OK;
}

}  // extern "C"
