// Request scheduler for serving many independent runs from one GPU with
// continuous batching: runs arrive at any time, wait in a FIFO queue until
// their device memory fits the budget, then advance together (each on a
// stream of its own, a few steps per scheduling round) and leave the GPU as
// soon as their results are collected, freeing room for the next ones.  The
// state of a running request stays on the device from admission to
// collection.  Host code only; the steps are the ordinary context steps.
//
// Nothing on the request path calls cudaMalloc or cudaFree (both can
// synchronise the device and stall the runs in flight): a request's context
// takes its arrays from the server's stream-ordered memory pool, whose
// release threshold is the budget (freed blocks stay reserved for the next
// requests), and streams and events are reused from a free list.  A request
// whose admission fails (a CUDA error, device memory short of the budget)
// is marked failed and leaves the queue, so it never blocks the requests
// behind it; its error code is returned when it is collected.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "sipf_internal.cuh"

namespace {

enum class ReqState { Queued, Running, Draining, Done, Failed };

struct Request {
    int64_t id = 0;
    sipf_grid grid{};
    int64_t N = 0;
    sipf_params params{};
    double dt = 0;
    int64_t steps = 0, remaining = 0;
    size_t bytes = 0;
    std::vector<float> x, v, m, w;   // host copy of the initial state until admission
    std::vector<double> mass;
    sipf_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;      // recorded after the last step was enqueued
    ReqState state = ReqState::Queued;
    bool reported = false;
    int error = SIPF_OK;             // failed requests: the code collect returns
    std::string message;
};

}  // namespace

struct sipf_server {
    size_t budget = 0, in_use = 0, peak = 0;
    int64_t next_id = 1;
    int32_t max_live = 0;                // 0: no limit besides the budget
    int inject = SIPF_OK;                // fault injection: code of the next admission
    int device = 0;
    cudaMemPool_t pool = nullptr;
    std::vector<cudaStream_t> free_streams;
    std::vector<cudaEvent_t> free_events;
    std::deque<Request*> queue;
    std::map<int64_t, Request*> live;    // admitted (or failed), not yet collected
    std::string last_error;
};

namespace {

// Returns the request's context, stream and event to the server (the
// context's arrays go back to the pool, stream-ordered).
void release(sipf_server* s, Request* r) {
    if (r->ctx) sipf_destroy(r->ctx);
    if (r->done) s->free_events.push_back(r->done);
    if (r->stream) s->free_streams.push_back(r->stream);
    r->ctx = nullptr;
    r->done = nullptr;
    r->stream = nullptr;
}

int live_running(const sipf_server* s) {
    int n = 0;
    for (const auto& kv : s->live)
        if (kv.second->state != ReqState::Failed) ++n;
    return n;
}

void mark_failed(sipf_server* s, Request* r, int code, const std::string& msg) {
    r->state = ReqState::Failed;
    r->error = code;
    r->message = msg;
    s->last_error = msg;
}

int fail(sipf_server* s, int code, const std::string& msg) {
    s->last_error = msg;
    return code;
}

// The pool of the requests' device memory, created on the first admission
// on the current device: blocks freed by collected requests stay reserved
// (up to the budget) for the next admissions.
int ensure_pool(sipf_server* s) {
    if (s->pool) return SIPF_OK;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        return SIPF_ECUDA;
    }
    props.location.id = s->device;
    uint64_t keep = static_cast<uint64_t>(s->budget);
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
        cudaGetLastError();
        s->pool = nullptr;
        return SIPF_ECUDA;
    }
    if (cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
        cudaGetLastError();
        cudaMemPoolDestroy(s->pool);
        s->pool = nullptr;
        return SIPF_ECUDA;
    }
    return SIPF_OK;
}

// Admits queued requests, in arrival order, while the next one fits (and,
// with a limit, while fewer than max_live requests are admitted).  A
// request whose admission fails is marked failed and leaves the queue.
void admit(sipf_server* s) {
    while (!s->queue.empty() && s->in_use + s->queue.front()->bytes <= s->budget &&
           (s->max_live <= 0 || live_running(s) < s->max_live)) {
        Request* r = s->queue.front();
        s->queue.pop_front();
        int rc = s->inject;
        s->inject = SIPF_OK;
        std::string what = "injected failure";
        if (rc == SIPF_OK) {
            if (!s->free_streams.empty()) {
                r->stream = s->free_streams.back();
                s->free_streams.pop_back();
            } else if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                r->stream = nullptr;
                rc = SIPF_ECUDA;
                what = "cudaStreamCreate";
            }
        }
        if (rc == SIPF_OK) {
            if (!s->free_events.empty()) {
                r->done = s->free_events.back();
                s->free_events.pop_back();
            } else if (cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                r->done = nullptr;
                rc = SIPF_ECUDA;
                what = "cudaEventCreate";
            }
        }
        if (rc == SIPF_OK) {
            rc = ensure_pool(s);
            what = "creating the memory pool";
        }
        if (rc == SIPF_OK) {
            rc = sipf::create_in_pool(&r->grid, r->N, &r->params, r->stream, s->pool, &r->ctx);
            what = "creating the context";
        }
        if (rc == SIPF_OK) {
            rc = sipf_set_state(r->ctx, r->x.data(), r->mass.data(), nullptr, r->v.data(),
                                r->m.data(), r->w.data(), SIPF_HOST);
            what = std::string("setting the state: ") + sipf_last_error(r->ctx);
        }
        std::vector<float>().swap(r->x);
        std::vector<float>().swap(r->v);
        std::vector<float>().swap(r->m);
        std::vector<float>().swap(r->w);
        std::vector<double>().swap(r->mass);
        s->live[r->id] = r;
        if (rc != SIPF_OK) {
            release(s, r);
            mark_failed(s, r, rc, "request " + std::to_string(r->id) + " not admitted: " + what);
            continue;
        }
        r->state = ReqState::Running;
        r->remaining = r->steps;
        s->in_use += r->bytes;
        s->peak = std::max(s->peak, s->in_use);
    }
}

}  // namespace

extern "C" {

int sipf_server_create(int64_t budget_bytes, sipf_server** out) {
    if (!out) return SIPF_EINVAL;
    *out = nullptr;
    if (budget_bytes <= 0) return SIPF_EINVAL;
    sipf_server* s = new (std::nothrow) sipf_server();
    if (!s) return SIPF_ENOMEM;
    s->budget = static_cast<size_t>(budget_bytes);
    *out = s;
    return SIPF_OK;
}

int sipf_server_set_limit(sipf_server* s, int32_t max_live) {
    if (!s || max_live < 0) return SIPF_EINVAL;
    s->max_live = max_live;
    return SIPF_OK;
}

int sipf_server_fail_next_admission(sipf_server* s, int code) {
    if (!s || code >= 0) return SIPF_EINVAL;
    s->inject = code;
    return SIPF_OK;
}

int sipf_server_submit(sipf_server* s, const sipf_grid* grid, int64_t N, const sipf_params* params,
                       const float* x, const double* mass, const float* v, const float* m,
                       const float* w, double dt, int64_t steps, int64_t* id) {
    if (!s) return SIPF_EINVAL;
    if (!grid || !params || !x || !mass || !v || !m || !w || !id)
        return fail(s, SIPF_EINVAL, "NULL argument");
    if (!(dt > 0.0 && dt <= 0.5) || steps < 0) return fail(s, SIPF_EINVAL, "bad dt or steps");
    const int64_t bytes = sipf_context_bytes(grid, N, params);
    if (bytes < 0) return fail(s, SIPF_EINVAL, "invalid grid, particle count or parameters");
    // the checks sipf_set_state makes, done here so that admission cannot fail on them
    for (int64_t i = 0; i < N; ++i)
        if (!(isfinite(mass[i]) && mass[i] >= 0.0))
            return fail(s, SIPF_EINVAL, "masses must be finite and >= 0");
    if (static_cast<size_t>(bytes) > s->budget)
        return fail(s, SIPF_EINVAL, "request needs " + std::to_string(bytes) +
                                        " device bytes, more than the budget");
    Request* r = new (std::nothrow) Request();
    if (!r) return SIPF_ENOMEM;
    const size_t H3 = static_cast<size_t>(grid->H) * grid->H * grid->H;
    try {
        r->x.assign(x, x + 3 * N);
        r->mass.assign(mass, mass + N);
        r->v.assign(v, v + H3);
        r->m.assign(m, m + H3);
        r->w.assign(w, w + H3);
    } catch (...) {
        delete r;
        return fail(s, SIPF_ENOMEM, "host copy of the request");
    }
    r->id = s->next_id++;
    r->grid = *grid;
    r->N = N;
    r->params = *params;
    r->dt = dt;
    r->steps = steps;
    r->bytes = static_cast<size_t>(bytes);
    s->queue.push_back(r);
    *id = r->id;
    return SIPF_OK;
}

int sipf_server_advance(sipf_server* s, int64_t quantum, int32_t* pending) {
    if (!s || quantum < 1) return SIPF_EINVAL;
    admit(s);
    // every running request gets up to `quantum` more steps, request after
    // request, so that their kernels overlap on the GPU; a request whose
    // steps fail is marked failed and the others go on
    for (auto& kv : s->live) {
        Request* r = kv.second;
        if (r->state != ReqState::Running) continue;
        const int64_t q = std::min<int64_t>(quantum, r->remaining);
        if (q > 0) {
            const int rc = sipf::run_steps_for(r->ctx, r->dt, q);
            if (rc != SIPF_OK) {
                mark_failed(s, r, rc, "request " + std::to_string(r->id) + ": " +
                                          sipf_last_error(r->ctx));
                continue;
            }
            r->remaining -= q;
        }
        if (r->remaining == 0) {
            if (cudaEventRecord(r->done, r->stream) != cudaSuccess) {
                cudaGetLastError();
                mark_failed(s, r, SIPF_ECUDA, "request " + std::to_string(r->id) +
                                                  ": cudaEventRecord");
                continue;
            }
            r->state = ReqState::Draining;
        }
    }
    // requests whose last step has finished on the device
    for (auto& kv : s->live) {
        Request* r = kv.second;
        if (r->state != ReqState::Draining) continue;
        const cudaError_t e = cudaEventQuery(r->done);
        if (e == cudaSuccess) {
            r->state = ReqState::Done;
        } else if (e != cudaErrorNotReady) {
            mark_failed(s, r, SIPF_ECUDA, std::string("request ") + std::to_string(r->id) + ": " +
                                              cudaGetErrorString(e));
        }
    }
    if (pending) {
        int32_t n = static_cast<int32_t>(s->queue.size());
        for (auto& kv : s->live)
            if (kv.second->state != ReqState::Done && kv.second->state != ReqState::Failed) ++n;
        *pending = n;
    }
    return SIPF_OK;
}

int sipf_server_poll(sipf_server* s, int64_t* ids, int32_t capacity, int32_t* count) {
    if (!s || !count || capacity < 0 || (capacity > 0 && !ids)) return SIPF_EINVAL;
    int32_t n = 0;
    for (auto& kv : s->live) {
        Request* r = kv.second;
        if (n >= capacity) break;
        if ((r->state == ReqState::Done || r->state == ReqState::Failed) && !r->reported) {
            ids[n++] = r->id;
            r->reported = true;
        }
    }
    *count = n;
    return SIPF_OK;
}

int sipf_server_collect(sipf_server* s, int64_t id, uint32_t mask, float* dst) {
    if (!s) return SIPF_EINVAL;
    auto it = s->live.find(id);
    if (it == s->live.end()) return fail(s, SIPF_EINVAL, "unknown or collected request");
    Request* r = it->second;
    if (r->state == ReqState::Failed) {
        // a failed request holds no device state beyond what release returns
        const int rc = r->error;
        s->last_error = r->message;
        const bool admitted = r->ctx != nullptr;
        if (r->stream) cudaStreamSynchronize(r->stream);
        release(s, r);
        if (admitted) s->in_use -= r->bytes;
        s->live.erase(it);
        delete r;
        return rc;
    }
    if (r->state != ReqState::Done) return fail(s, SIPF_EINVAL, "request not finished");
    int rc = SIPF_OK;
    if (mask) rc = sipf_fields(r->ctx, mask, dst, SIPF_HOST);
    if (rc == SIPF_OK) rc = sipf_sync(r->ctx);
    if (rc != SIPF_OK) s->last_error = sipf_last_error(r->ctx);
    release(s, r);
    s->in_use -= r->bytes;
    s->live.erase(it);
    delete r;
    return rc;
}

int sipf_server_stats(const sipf_server* s, int64_t* in_use, int64_t* peak, int32_t* queued,
                      int32_t* live) {
    if (!s) return SIPF_EINVAL;
    if (in_use) *in_use = static_cast<int64_t>(s->in_use);
    if (peak) *peak = static_cast<int64_t>(s->peak);
    if (queued) *queued = static_cast<int32_t>(s->queue.size());
    if (live) *live = static_cast<int32_t>(live_running(s));
    return SIPF_OK;
}

const char* sipf_server_last_error(const sipf_server* s) { return s ? s->last_error.c_str() : ""; }

void sipf_server_destroy(sipf_server* s) {
    if (!s) return;
    for (Request* r : s->queue) delete r;
    for (auto& kv : s->live) {
        if (kv.second->stream) cudaStreamSynchronize(kv.second->stream);
        release(s, kv.second);
        delete kv.second;
    }
    // the contexts' stream-ordered frees complete before the pool goes
    for (cudaStream_t st : s->free_streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (cudaEvent_t e : s->free_events) cudaEventDestroy(e);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
}

}  // extern "C"
