// server.cu -- the serving loop: independent FMM solves submitted at any time are admitted
// by device-memory footprint, batched into forests and run on several CUDA streams at once
// (continuous batching).  The paper has no counterpart; the solves themselves are the
// paper's method (dafmm_build_forest + dafmm_eval).
//
// One scheduler thread owns a pooled context (no cudaFree, so retiring a job never stalls
// the device).  Whenever a stream slot is free it forms a job from the queue
// (serve_policy.h), copies the job's inputs into one device array, builds the forest and
// evaluates it on the slot's stream, copies each result back into its caller's buffers and
// enqueues a host callback that stamps the completion time.  Requests that arrive meanwhile
// join the queue and are admitted as slots and memory come free; jobs on different slots
// overlap on the device.  Every request keeps its own tree inside the forest, so its result
// is the one a solve of it alone gives.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "api_types.h"
#include "dafmm.h"
#include "serve_policy.h"

using namespace dafmm;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct SReq {
    int64_t id = 0;
    const double* xyz = nullptr;
    const double* q = nullptr;
    int64_t n = 0;
    int order = 0, precision = 0, max_leaf = 0;
    double* phi = nullptr;
    double* field = nullptr;
    double t_submit = 0, t_start = 0, t_done = 0;
    int status = 1;  // 1 queued, 2 running, 0 done, < 0 failed
    int64_t cls() const { return ((int64_t)order * 4 + precision) * (1 << 20) + max_leaf; }
};

struct SJob {
    dafmm_server* srv = nullptr;
    std::vector<SReq*> reqs;
    int slot = -1;
    dafmm_tree* tree = nullptr;
    double* d_buf = nullptr;  // inputs (xyz, q) then outputs (phi, field), 8 doubles per particle
    size_t buf_bytes = 0;
    double t_done = 0;
    bool done = false;  // set by the stream callback, under the server's mutex
};

}  // namespace

struct dafmm_server {
    int device = 0;
    dafmm_ctx* ctx = nullptr;
    int slots = 1, max_batch = 1;
    int64_t max_particles = 0;
    std::vector<cudaStream_t> streams;
    std::vector<SJob*> running;
    std::deque<SReq*> queue;
    std::unordered_map<int64_t, SReq*> reqs;
    int64_t next_id = 1;
    std::mutex m;
    std::condition_variable cv_work, cv_done;
    bool wake = false, stop = false;
    std::thread th;
    std::string err;
    // counters
    int64_t completed = 0, failed = 0, jobs = 0, job_requests = 0;
    size_t peak_bytes = 0;
    int peak_running = 0;
};

namespace {

void CUDART_CB on_job_done(void* arg) {
    SJob* j = static_cast<SJob*>(arg);
    dafmm_server* s = j->srv;
    {
        std::lock_guard<std::mutex> lk(s->m);
        j->t_done = now_s();
        j->done = true;
        s->wake = true;
    }
    s->cv_work.notify_one();
}

// device bytes of one request inside a job: its share of the tree and expansions plus the
// job's staging buffers (the per-order tables are counted once, by the admission)
size_t request_estimate(const SReq* r) {
    const size_t with = dafmm_footprint(r->n, r->order, -1, r->max_leaf, r->precision);
    const size_t without = dafmm_footprint(0, r->order, -1, r->max_leaf, r->precision);
    return (with > without ? with - without : 0) + (size_t)r->n * 64 + ((size_t)1 << 20);
}

// the per-order tables (M2L matrices and their splits), when the order is not loaded yet
size_t tables_estimate(const dafmm_ctx* c, const SReq* r) {
    if (c->ord[r->order].k_ready) return 0;
    return 2 * dafmm_footprint(0, r->order, -1, r->max_leaf, r->precision);
}

// launch one job on its slot's stream; returns a DAFMM code (the job is not running on error)
int launch_job(dafmm_server* S, SJob* j) {
    dafmm_ctx* c = S->ctx;
    cudaStream_t st = S->streams[j->slot];
    const int nr = (int)j->reqs.size();
    std::vector<int64_t> offs(nr + 1, 0);
    for (int k = 0; k < nr; ++k) offs[k + 1] = offs[k] + j->reqs[k]->n;
    const int64_t n = offs[nr];
    j->buf_bytes = (size_t)std::max<int64_t>(n, 1) * 8 * sizeof(double);
    int rc = ctx_alloc(c, (void**)&j->d_buf, j->buf_bytes, "serving buffers");
    if (rc) return rc;
    double* d_xyz = j->d_buf;
    double* d_q = d_xyz + 3 * n;
    double* d_phi = d_q + n;
    double* d_field = d_phi + n;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < nr && e == cudaSuccess; ++k) {
        const SReq* r = j->reqs[k];
        if (r->n == 0) continue;
        e = cudaMemcpyAsync(d_xyz + 3 * offs[k], r->xyz, (size_t)r->n * 3 * sizeof(double), cudaMemcpyDefault, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_q + offs[k], r->q, (size_t)r->n * sizeof(double), cudaMemcpyDefault, st);
    }
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        c->err = std::string("serving input copy: ") + cudaGetErrorString(e);
        return DAFMM_ERR_CUDA;
    }
    const SReq* h = j->reqs[0];
    rc = dafmm_build_forest(c, d_xyz, d_q, offs.data(), nr, nullptr, h->max_leaf, st, &j->tree);
    if (!rc) rc = dafmm_eval(j->tree, h->order, 1.0, h->precision, d_phi, d_field, st);
    if (rc) {
        cudaStreamSynchronize(st);  // nothing of the job may still run when its memory is returned
        return rc;
    }
    for (int k = 0; k < nr && e == cudaSuccess; ++k) {
        const SReq* r = j->reqs[k];
        if (r->n == 0) continue;
        if (r->phi)
            e = cudaMemcpyAsync(r->phi, d_phi + offs[k], (size_t)r->n * sizeof(double), cudaMemcpyDefault, st);
        if (e == cudaSuccess && r->field)
            e = cudaMemcpyAsync(r->field, d_field + 3 * offs[k], (size_t)r->n * 3 * sizeof(double),
                                cudaMemcpyDefault, st);
    }
    if (e == cudaSuccess) e = cudaLaunchHostFunc(st, on_job_done, j);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        c->err = std::string("serving output copy: ") + cudaGetErrorString(e);
        return DAFMM_ERR_CUDA;
    }
    return DAFMM_OK;
}

void release_job(dafmm_server* S, SJob* j) {
    if (j->tree) dafmm_tree_free(j->tree);
    if (j->d_buf) ctx_free(S->ctx, j->d_buf, j->buf_bytes);
    j->tree = nullptr;
    j->d_buf = nullptr;
}

void finish(dafmm_server* S, SReq* r, int status, double t) {
    r->status = status;
    r->t_done = t;
    if (status == 0) ++S->completed;
    else ++S->failed;
}

void scheduler(dafmm_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->m);
    for (;;) {
        // retire finished jobs
        int nrun = 0;
        for (int k = 0; k < S->slots; ++k) {
            SJob* j = S->running[k];
            if (!j) continue;
            if (!j->done) {
                ++nrun;
                continue;
            }
            release_job(S, j);
            for (SReq* r : j->reqs) finish(S, r, 0, j->t_done);
            S->running[k] = nullptr;
            delete j;
            S->cv_done.notify_all();
        }
        // admit
        while (!S->stop && !S->queue.empty()) {
            int slot = -1;
            for (int k = 0; k < S->slots && slot < 0; ++k)
                if (!S->running[k]) slot = k;
            if (slot < 0) break;
            std::vector<PendingRequest> pend;
            const size_t scan = std::min<size_t>(S->queue.size(), 64 + 4 * (size_t)S->max_batch);
            for (size_t i = 0; i < scan; ++i) {
                SReq* r = S->queue[i];
                pend.push_back({r->cls(), r->n, request_estimate(r)});
            }
            const size_t in_use = S->ctx->in_use + tables_estimate(S->ctx, S->queue.front());
            const size_t pool = S->ctx->arena.size();
            const size_t free_b = pool > in_use ? pool - in_use : 0;
            std::vector<size_t> sel = select_batch(pend, free_b, S->max_batch, S->max_particles);
            if (sel.empty()) {
                if (nrun == 0) {  // the oldest request cannot fit even an idle pool
                    SReq* r = S->queue.front();
                    S->queue.pop_front();
                    finish(S, r, DAFMM_ERR_OVER_BUDGET, now_s());
                    S->cv_done.notify_all();
                    continue;
                }
                break;
            }
            SJob* j = new SJob();
            j->srv = S;
            j->slot = slot;
            for (size_t i : sel) j->reqs.push_back(S->queue[i]);
            for (size_t k = sel.size(); k-- > 0;) S->queue.erase(S->queue.begin() + (long)sel[k]);
            const double t0 = now_s();
            for (SReq* r : j->reqs) {
                r->status = 2;
                r->t_start = t0;
            }
            S->running[slot] = j;
            // the build synchronises this slot's stream: let submitters and callbacks proceed
            lk.unlock();
            const int rc = launch_job(S, j);
            lk.lock();
            if (rc) {
                release_job(S, j);
                S->running[slot] = nullptr;
                if (rc == DAFMM_ERR_OVER_BUDGET && nrun > 0) {
                    // the estimate was short: retry once running jobs have returned memory
                    for (size_t k = j->reqs.size(); k-- > 0;) {
                        j->reqs[k]->status = 1;
                        S->queue.push_front(j->reqs[k]);
                    }
                    delete j;
                    break;
                }
                S->err = S->ctx->err;
                for (SReq* r : j->reqs) finish(S, r, rc, now_s());
                delete j;
                S->cv_done.notify_all();
                continue;
            }
            ++S->jobs;
            S->job_requests += (int64_t)j->reqs.size();
            ++nrun;
            S->peak_running = std::max(S->peak_running, nrun);
            S->peak_bytes = std::max(S->peak_bytes, S->ctx->in_use);
        }
        if (S->stop && nrun == 0) break;
        S->cv_work.wait(lk, [S] { return S->wake || S->stop; });
        S->wake = false;
    }
    // stopping: whatever is still queued is cancelled
    for (SReq* r : S->queue) finish(S, r, DAFMM_ERR_CANCELLED, now_s());
    S->queue.clear();
    S->cv_done.notify_all();
}

}  // namespace

extern "C" {

int dafmm_server_create(int device, size_t pool_bytes, int slots, int max_batch, int64_t max_job_particles,
                        dafmm_server** out) {
    if (!out || slots < 1 || slots > 64 || max_batch < 1 || max_job_particles < 1) return DAFMM_ERR_INVALID_ARG;
    *out = nullptr;
    dafmm_ctx* c = nullptr;
    int rc = dafmm_create_pooled(&c, device, pool_bytes);
    if (rc) return rc;
    dafmm_server* S = new dafmm_server();
    S->device = device;
    S->ctx = c;
    S->slots = slots;
    S->max_batch = max_batch;
    S->max_particles = max_job_particles;
    S->running.assign(slots, nullptr);
    for (int k = 0; k < slots; ++k) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t x : S->streams) cudaStreamDestroy(x);
            dafmm_destroy(c);
            delete S;
            return DAFMM_ERR_CUDA;
        }
        S->streams.push_back(st);
    }
    S->th = std::thread(scheduler, S);
    *out = S;
    return DAFMM_OK;
}

int dafmm_server_submit(dafmm_server* S, const double* xyz, const double* q, int64_t n, int order, int precision,
                        int max_leaf, double* phi, double* field, int64_t* id) {
    if (!S || !id || n < 0 || (n > 0 && (!xyz || !q)) || max_leaf < 1) return DAFMM_ERR_INVALID_ARG;
    if (order < 0 || order > kMaxOrder) return DAFMM_ERR_UNSUPPORTED_ORDER;
    if (precision != DAFMM_FP64 && precision != DAFMM_MIXED && precision != DAFMM_FP32) return DAFMM_ERR_INVALID_ARG;
    SReq* r = new SReq();
    r->xyz = xyz;
    r->q = q;
    r->n = n;
    r->order = order;
    r->precision = precision;
    r->max_leaf = max_leaf;
    r->phi = phi;
    r->field = field;
    {
        std::lock_guard<std::mutex> lk(S->m);
        if (S->stop) {
            delete r;
            return DAFMM_ERR_CANCELLED;
        }
        r->id = S->next_id++;
        r->t_submit = now_s();
        S->reqs[r->id] = r;
        S->queue.push_back(r);
        S->wake = true;
        *id = r->id;
    }
    S->cv_work.notify_one();
    return DAFMM_OK;
}

int dafmm_server_wait(dafmm_server* S, int64_t id, double timeout_s, double* times3) {
    if (!S) return DAFMM_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->m);
    if (S->reqs.find(id) == S->reqs.end()) return DAFMM_ERR_INVALID_ARG;
    // the request is looked up afresh on every wake-up: another thread waiting for the same id
    // may have taken (and deleted) it meanwhile
    auto finished = [S, id] {
        auto f = S->reqs.find(id);
        return f == S->reqs.end() || f->second->status <= 0;
    };
    if (timeout_s < 0) S->cv_done.wait(lk, finished);
    else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), finished)) return DAFMM_ERR_TIMEOUT;
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return DAFMM_ERR_INVALID_ARG;  // another waiter took it
    SReq* r = it->second;
    if (times3) {
        times3[0] = (r->t_done - r->t_submit) * 1e3;  // latency
        times3[1] = (r->t_start - r->t_submit) * 1e3;  // waiting for admission
        times3[2] = (r->t_done - r->t_start) * 1e3;    // on the device (with its batch)
    }
    const int st = r->status;
    S->reqs.erase(it);
    delete r;
    return st;
}

int dafmm_server_stats(dafmm_server* S, double* out8) {
    if (!S || !out8) return DAFMM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->m);
    int nrun = 0;
    for (SJob* j : S->running) nrun += j != nullptr;
    out8[0] = (double)S->completed;
    out8[1] = (double)S->failed;
    out8[2] = (double)S->queue.size();
    out8[3] = (double)nrun;
    out8[4] = (double)S->jobs;
    out8[5] = S->jobs ? (double)S->job_requests / (double)S->jobs : 0.0;
    out8[6] = (double)S->peak_bytes;
    out8[7] = (double)S->peak_running;
    return DAFMM_OK;
}

const char* dafmm_server_last_error(dafmm_server* S) {
    if (!S) return "no server";
    // a copy per calling thread: the scheduler may replace the message at any time
    thread_local std::string copy;
    std::lock_guard<std::mutex> lk(S->m);
    copy = S->err;
    return copy.c_str();
}

int dafmm_server_destroy(dafmm_server* S) {
    if (!S) return DAFMM_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(S->m);
        S->stop = true;
        S->wake = true;
    }
    S->cv_work.notify_one();
    S->th.join();
    cudaSetDevice(S->device);
    for (cudaStream_t st : S->streams) cudaStreamDestroy(st);
    for (auto& kv : S->reqs) delete kv.second;
    dafmm_destroy(S->ctx);
    delete S;
    return DAFMM_OK;
}

}  // extern "C"
