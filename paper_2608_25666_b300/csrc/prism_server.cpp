// prism_server.cpp -- continuous-batching request loop for libprism_proj.
//
// Many MPC controllers (each a factored projector with its own J, H, N, dt and
// bounds) submit one projection request per control step.  A scheduler
// thread admits queued requests as soon as an execution slot (a CUDA stream)
// and device memory for the request's buffers are free, so requests that
// arrive while others run are launched immediately and their kernels overlap
// on the GPU.  Each controller's multiplier state stays on the device between
// its steps and is shifted along the receding horizon before the next solve
// (the paper warm-starts its sampling distribution the same way, Sec. III-B).
// Memory is admitted against a fixed budget: the controllers' resident state
// at registration, each request's staging buffers at launch.
//
// Scheduling rules:
//   * one request in flight per controller (its warm start depends on the
//     previous step's result);
//   * a controller's newer request supersedes its older queued one (an MPC
//     step whose successor has arrived is stale); the older is dropped and
//     counted as a deadline miss;
//   * otherwise first come, first served.
#include "prism_proj.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

// Records the thread-local error text of libprism_proj; device allocations of the
// library; the device word in which a handle's solves report a wait that ran
// out (all defined in prism_proj.cu).
prism_status prism_internal_fail(prism_status s, const char *msg);
cudaError_t prism_internal_dev_malloc(void **p, size_t bytes);
int *prism_internal_err_flag(prism_proj_t h);

struct Server;

namespace {

prism_status sfail(prism_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return prism_internal_fail(s, buf);
}

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum ReqState : int { Q_QUEUED = 0, Q_RUNNING = 1, Q_DONE = 2, Q_DROPPED = 3, Q_FAILED = 4 };

struct Request {
    unsigned long long ticket = 0;
    int ctrl = -1;
    const float *q0 = nullptr, *v0 = nullptr, *xi = nullptr;
    float *out = nullptr, *primal = nullptr;
    double t_submit = 0.0, t_done = 0.0;
    std::atomic<int> state{Q_QUEUED};
    bool retired = false;          // buffers released and statistics recorded
    prism_status fail_status = PRISM_OK;   // why a failed request failed
    size_t off = 0, bytes = 0;     // arena block of its staging buffers
    int slot = -1;
    struct Server *srv = nullptr;
};

struct Controller {
    prism_proj_t h = nullptr;
    int N = 0, J = 0, H = 0, D = 0, iters = 0;
    double rho = 1.0;
    bool warm = true, has_state = false, busy = false;
    size_t state_off = 0;
    std::shared_ptr<Request> queued;   // latest not-yet-launched request
};

// First-fit allocator over [0, size) of the device arena.
struct Arena {
    char *base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;   // offset -> length
    void init(char *b, size_t n)
    {
        base = b;
        size = n;
        free_.clear();
        free_[0] = n;
    }
    bool alloc(size_t n, size_t &off)
    {
        n = (n + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                off = it->first;
                const size_t rest = it->second - n;
                free_.erase(it);
                if (rest) free_[off + n] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = (n + 255) & ~size_t(255);
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t free_bytes() const
    {
        size_t s = 0;
        for (auto &kv : free_) s += kv.second;
        return s;
    }
};

}  // namespace

struct Server {
    int device = 0;
    double deadline_ms = 20.0;
    bool plain = false;               // PRISM_SERVER_PLAIN: every request on the plain comparator
    std::mutex mu;
    std::condition_variable cv;       // scheduler wake-ups
    std::condition_variable done_cv;  // waiters on tickets
    std::thread th;
    bool stop = false;
    Arena arena;
    size_t resident = 0;
    std::vector<Controller> ctrls;
    std::vector<cudaStream_t> streams;
    std::vector<std::shared_ptr<Request>> slot_req;
    int *slot_flag = nullptr;          // pinned host words: each slot's copy of its solve's timeout flag
    std::deque<std::shared_ptr<Request>> fifo;
    std::unordered_map<unsigned long long, std::shared_ptr<Request>> tickets;
    unsigned long long next_ticket = 1;
    // statistics
    std::vector<double> lat_ms;
    long long n_done = 0, n_dropped = 0, n_failed = 0, traj_done = 0;
    double t_first = 0.0, t_last = 0.0;
    std::string last_error;

    void run();
    bool enqueue(const std::shared_ptr<Request> &r, const Controller &c, bool warm_in);
    void retire(int slot);
};

struct prism_server_s {
    Server srv;
};

namespace {

void CUDART_CB on_request_done(void *arg)
{
    // runs on the CUDA callback thread: no CUDA calls and no locks here; the
    // scheduler polls at least every 200 microseconds.  Once the state is
    // stored the scheduler may retire the request and its waiter free it, so
    // nothing of the request is touched after the store (the server outlives
    // every callback: destroy synchronises the streams first).
    Request *r = static_cast<Request *>(arg);
    Server *srv = r->srv;
    r->t_done = now_s();
    r->state.store(Q_DONE);
    srv->cv.notify_all();
}

}  // namespace

// Enqueues one admitted request on its slot's stream: input copies, the
// warm-start shift, the solve, the result copies and the completion callback.
// Runs on the scheduler thread WITHOUT the server lock (a copy into pageable
// host memory blocks until the solve ends), on a snapshot of the controller.
bool Server::enqueue(const std::shared_ptr<Request> &r, const Controller &c, bool warm_in)
{
    cudaStream_t s = streams[r->slot];
    char *base = arena.base + r->off;
    const size_t seq = (size_t)c.N * c.H * c.J;
    float *d_xi = reinterpret_cast<float *>(base);
    float *d_out = d_xi + seq;
    float *d_pr = d_out + seq;
    float *d_q0 = d_pr + (size_t)c.N * c.J;
    float *d_v0 = d_q0 + c.J;
    float *d_state = reinterpret_cast<float *>(arena.base + c.state_off);
    bool ok = cudaMemcpyAsync(d_xi, r->xi, seq * sizeof(float), cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(d_q0, r->q0, c.J * sizeof(float), cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(d_v0, r->v0, c.J * sizeof(float), cudaMemcpyHostToDevice, s) == cudaSuccess;
    if (plain) {
        // the plain single-batch comparator: cold start, one thread per column
        if (ok)
            ok = prism_proj_solve_plain(c.h, c.N, d_q0, d_v0, d_xi, c.iters, c.rho, d_out, d_pr, nullptr, s) ==
                 PRISM_OK;
    } else {
        if (ok && warm_in) ok = prism_proj_shift_state(c.h, c.N, 1, nullptr, d_state, s) == PRISM_OK;
        prism_solve_opts o;
        o.x_init = nullptr;
        o.dual_init = warm_in ? d_state : nullptr;
        o.dual_out = c.warm ? d_state : nullptr;
        o.polish_iters = 0;
        o.init_layout = PRISM_INIT_SAMPLE_MAJOR;
        if (ok)
            ok = prism_proj_solve_ex(c.h, c.N, d_q0, d_v0, d_xi, c.iters, c.rho, &o, d_out, d_pr, nullptr, s) ==
                 PRISM_OK;
    }
    // the handle's timeout flag after this solve, read at retire without a host
    // sync, then cleared for the next launch of the handle
    int *d_flag = prism_internal_err_flag(c.h);
    slot_flag[r->slot] = 0;
    if (ok && d_flag)
        ok = cudaMemcpyAsync(&slot_flag[r->slot], d_flag, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
             cudaMemsetAsync(d_flag, 0, sizeof(int), s) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(r->out, d_out, seq * sizeof(float), cudaMemcpyDeviceToHost, s) == cudaSuccess;
    if (ok && r->primal)
        ok = cudaMemcpyAsync(r->primal, d_pr, (size_t)c.N * c.J * sizeof(float), cudaMemcpyDeviceToHost, s) ==
             cudaSuccess;
    if (ok) ok = cudaLaunchHostFunc(s, on_request_done, r.get()) == cudaSuccess;
    if (!ok) cudaStreamSynchronize(s);   // let whatever was enqueued finish before the buffers are reused
    return ok;
}

void Server::retire(int slot)
{
    std::shared_ptr<Request> r = slot_req[slot];
    slot_req[slot].reset();
    r->retired = true;
    Controller &c = ctrls[r->ctrl];
    c.busy = false;
    arena.release(r->off, r->bytes);
    if (r->state.load() == Q_DONE && slot_flag[slot] != 0) {
        // a bounded device-side wait of the solve ran out: the outputs and the
        // exported multiplier are invalid, so the controller starts cold next
        r->state.store(Q_FAILED);
        r->fail_status = PRISM_ERR_TIMEOUT;
        last_error = "a device-side wait of the solve ran out its bound";
        c.has_state = false;
    }
    const int st = r->state.load();
    if (st == Q_DONE) {
        const double ms = (r->t_done - r->t_submit) * 1e3;
        lat_ms.push_back(ms);
        ++n_done;
        traj_done += c.N;
        if (t_first == 0.0) t_first = r->t_submit;
        t_last = std::max(t_last, r->t_done);
    } else {
        ++n_failed;
    }
    done_cv.notify_all();
}

void Server::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    struct Job {
        std::shared_ptr<Request> r;
        Controller c;      // snapshot: the controller list may grow while unlocked
        bool warm_in;
    };
    std::vector<Job> jobs;
    while (!stop) {
        // retire finished requests
        for (size_t k = 0; k < slot_req.size(); ++k)
            if (slot_req[k] && (slot_req[k]->state.load() == Q_DONE || slot_req[k]->state.load() == Q_FAILED))
                retire((int)k);
        // admit queued requests in arrival order
        for (auto it = fifo.begin(); it != fifo.end();) {
            std::shared_ptr<Request> r = *it;
            if (r->state.load() != Q_QUEUED) { it = fifo.erase(it); continue; }
            Controller &c = ctrls[r->ctrl];
            if (c.busy) { ++it; continue; }
            int slot = -1;
            for (size_t k = 0; k < slot_req.size(); ++k)
                if (!slot_req[k]) { slot = (int)k; break; }
            if (slot < 0) break;
            const size_t bytes = (2 * (size_t)c.N * c.H * c.J + (size_t)c.N * c.J + 2 * (size_t)c.J + 64) * sizeof(float);
            size_t off;
            if (!arena.alloc(bytes, off)) { ++it; continue; }   // wait for memory to free up
            r->off = off;
            r->bytes = bytes;
            r->slot = slot;
            if (c.queued == r) c.queued.reset();
            it = fifo.erase(it);
            slot_req[slot] = r;
            c.busy = true;
            r->state.store(Q_RUNNING);
            Job j;
            j.r = r;
            j.c = c;
            j.c.queued.reset();
            j.warm_in = c.warm && c.has_state && !plain;
            jobs.push_back(std::move(j));
        }
        if (!jobs.empty()) {
            // enqueue outside the lock: submitters and waiters are never held up
            // by the copies (which block for pageable host buffers)
            lk.unlock();
            std::vector<bool> ok(jobs.size());
            for (size_t k = 0; k < jobs.size(); ++k) ok[k] = enqueue(jobs[k].r, jobs[k].c, jobs[k].warm_in);
            std::string err = prism_last_error();
            lk.lock();
            for (size_t k = 0; k < jobs.size(); ++k) {
                Request &r = *jobs[k].r;
                if (ok[k]) {
                    if (jobs[k].c.warm) ctrls[r.ctrl].has_state = true;
                } else {
                    // the multiplier may already be shifted or partly written:
                    // the controller's next request starts cold
                    ctrls[r.ctrl].has_state = false;
                    last_error = err;
                    r.fail_status = PRISM_ERR_CUDA;
                    r.t_done = now_s();
                    r.state.store(Q_FAILED);
                }
            }
            jobs.clear();
            continue;   // retire what finished meanwhile before sleeping
        }
        cv.wait_for(lk, std::chrono::microseconds(200));
    }
}

extern "C" {

prism_status prism_server_create(size_t mem_budget_bytes, int max_inflight, double deadline_ms, prism_server_t *out)
{
    return prism_server_create_ex(mem_budget_bytes, max_inflight, deadline_ms, 0, out);
}

prism_status prism_server_create_ex(size_t mem_budget_bytes, int max_inflight, double deadline_ms, int flags,
                                    prism_server_t *out)
{
    if (!out) return sfail(PRISM_ERR_INVALID_ARG, "out is NULL");
    if (flags & ~PRISM_SERVER_PLAIN) return sfail(PRISM_ERR_INVALID_ARG, "unknown server flags %d", flags);
    *out = nullptr;
    if (mem_budget_bytes < (1u << 20)) return sfail(PRISM_ERR_INVALID_ARG, "memory budget below 1 MiB");
    if (max_inflight < 1 || max_inflight > 256) return sfail(PRISM_ERR_INVALID_ARG, "max_inflight outside [1, 256]");
    if (!(deadline_ms > 0.0)) return sfail(PRISM_ERR_INVALID_ARG, "deadline must be positive");
    prism_server_t ps = new (std::nothrow) prism_server_s;
    if (!ps) return sfail(PRISM_ERR_OOM, "host allocation failed");
    Server &S = ps->srv;
    S.deadline_ms = deadline_ms;
    S.plain = (flags & PRISM_SERVER_PLAIN) != 0;
    cudaError_t e = cudaGetDevice(&S.device);
    char *base = nullptr;
    if (e == cudaSuccess) e = prism_internal_dev_malloc(reinterpret_cast<void **>(&base), mem_budget_bytes);
    if (e != cudaSuccess) {
        delete ps;
        return sfail(e == cudaErrorMemoryAllocation ? PRISM_ERR_OOM : PRISM_ERR_CUDA, "server arena: %s",
                     cudaGetErrorString(e));
    }
    S.arena.init(base, mem_budget_bytes);
    e = cudaHostAlloc(reinterpret_cast<void **>(&S.slot_flag), sizeof(int) * max_inflight, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaFree(base);
        delete ps;
        return sfail(PRISM_ERR_OOM, "server flags: %s", cudaGetErrorString(e));
    }
    std::memset(S.slot_flag, 0, sizeof(int) * max_inflight);
    S.streams.resize(max_inflight);
    S.slot_req.resize(max_inflight);
    for (int k = 0; k < max_inflight; ++k) {
        e = cudaStreamCreateWithFlags(&S.streams[k], cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (int q = 0; q < k; ++q) cudaStreamDestroy(S.streams[q]);
            cudaFreeHost(S.slot_flag);
            cudaFree(base);
            delete ps;
            return sfail(PRISM_ERR_CUDA, "server streams: %s", cudaGetErrorString(e));
        }
    }
    S.th = std::thread([&S] { S.run(); });
    *out = ps;
    return PRISM_OK;
}

prism_status prism_server_add_controller(prism_server_t ps, prism_proj_t h, int batch, int iters, int warm_start,
                                         int *id)
{
    if (!ps || !h || !id) return sfail(PRISM_ERR_INVALID_ARG, "null argument");
    if (batch < 1 || iters < 0) return sfail(PRISM_ERR_INVALID_ARG, "batch must be >= 1 and iters >= 0");
    int dims[6];
    double rho = 0.0;
    prism_status st = prism_proj_describe(h, dims, &rho);
    if (st) return st;
    if (!dims[5]) return sfail(PRISM_ERR_NOT_FACTORED, "controller handle is not factored");
    Server &S = ps->srv;
    std::lock_guard<std::mutex> lk(S.mu);
    Controller c;
    c.h = h;
    c.N = batch;
    c.J = dims[0];
    c.H = dims[1];
    c.D = dims[2];
    c.iters = iters;
    c.rho = rho;
    c.warm = warm_start != 0;
    const size_t state_bytes = c.warm ? (size_t)c.N * c.D * c.J * sizeof(float) : 256;
    const size_t req_bytes = (2 * (size_t)c.N * c.H * c.J + (size_t)c.N * c.J + 2 * (size_t)c.J + 64) * sizeof(float);
    // admission: the resident state plus one request's buffers must fit the budget
    if (S.resident + state_bytes + req_bytes > S.arena.size)
        return sfail(PRISM_ERR_OOM, "admission: controller needs %zu bytes, %zu of %zu in use", state_bytes + req_bytes,
                     S.resident, S.arena.size);
    if (!S.arena.alloc(state_bytes, c.state_off))
        return sfail(PRISM_ERR_OOM, "admission: no contiguous block of %zu bytes", state_bytes);
    S.resident += (state_bytes + 255) & ~size_t(255);
    S.ctrls.push_back(c);
    *id = (int)S.ctrls.size() - 1;
    return PRISM_OK;
}

prism_status prism_server_submit(prism_server_t ps, int id, const float *q0_host, const float *v0_host,
                                 const float *samples_host, float *out_host, float *primal_host,
                                 unsigned long long *ticket)
{
    if (!ps || !q0_host || !v0_host || !samples_host || !out_host || !ticket)
        return sfail(PRISM_ERR_INVALID_ARG, "null argument");
    Server &S = ps->srv;
    auto r = std::make_shared<Request>();
    r->q0 = q0_host;
    r->v0 = v0_host;
    r->xi = samples_host;
    r->out = out_host;
    r->primal = primal_host;
    r->srv = &S;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        if (id < 0 || id >= (int)S.ctrls.size()) return sfail(PRISM_ERR_INVALID_ARG, "unknown controller %d", id);
        r->ctrl = id;
        r->t_submit = now_s();
        r->ticket = S.next_ticket++;
        Controller &c = S.ctrls[id];
        if (c.queued && c.queued->state.load() == Q_QUEUED) {   // superseded MPC step
            c.queued->state.store(Q_DROPPED);
            c.queued->t_done = r->t_submit;
            ++S.n_dropped;
        }
        c.queued = r;
        S.fifo.push_back(r);
        S.tickets[r->ticket] = r;
        *ticket = r->ticket;
    }
    S.cv.notify_all();
    S.done_cv.notify_all();
    return PRISM_OK;
}

prism_status prism_server_wait(prism_server_t ps, unsigned long long ticket, double timeout_ms, int *state,
                               double *latency_ms)
{
    if (!ps) return sfail(PRISM_ERR_INVALID_ARG, "null server");
    Server &S = ps->srv;
    std::unique_lock<std::mutex> lk(S.mu);
    auto it = S.tickets.find(ticket);
    if (it == S.tickets.end()) return sfail(PRISM_ERR_INVALID_ARG, "unknown ticket %llu", ticket);
    std::shared_ptr<Request> r = it->second;
    const auto pred = [&] {
        const int s = r->state.load();
        return s == Q_DROPPED || ((s == Q_DONE || s == Q_FAILED) && r->retired);
    };
    if (timeout_ms < 0) S.done_cv.wait(lk, pred);
    else S.done_cv.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), pred);
    const int s = r->state.load();
    if (state) *state = s;
    if (latency_ms) *latency_ms = (s == Q_DONE || s == Q_DROPPED) ? (r->t_done - r->t_submit) * 1e3 : -1.0;
    if (pred()) S.tickets.erase(ticket);
    if (s == Q_FAILED)
        return sfail(r->fail_status == PRISM_ERR_TIMEOUT ? PRISM_ERR_TIMEOUT : PRISM_ERR_CUDA, "request failed: %s",
                     S.last_error.c_str());
    return PRISM_OK;
}

prism_status prism_server_stats(prism_server_t ps, double out[10])
{
    if (!ps || !out) return sfail(PRISM_ERR_INVALID_ARG, "null argument");
    Server &S = ps->srv;
    std::lock_guard<std::mutex> lk(S.mu);
    std::vector<double> v = S.lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {
        if (v.empty()) return -1.0;
        const size_t k = std::min(v.size() - 1, (size_t)std::ceil(p / 100.0 * v.size()) - (p > 0 ? 1 : 0));
        return v[k];
    };
    long long late = 0;
    for (double x : v)
        if (x > S.deadline_ms) ++late;
    out[0] = (double)S.n_done;
    out[1] = (double)S.n_dropped;
    out[2] = (double)S.n_failed;
    out[3] = pct(50.0);
    out[4] = pct(99.0);
    out[5] = v.empty() ? -1.0 : v.back();
    out[6] = (double)(late + S.n_dropped);
    out[7] = (double)S.traj_done;
    out[8] = (S.t_last > S.t_first) ? S.traj_done / (S.t_last - S.t_first) : 0.0;
    out[9] = (double)S.arena.free_bytes();
    return PRISM_OK;
}

prism_status prism_server_reset_stats(prism_server_t ps)
{
    if (!ps) return sfail(PRISM_ERR_INVALID_ARG, "null server");
    Server &S = ps->srv;
    std::lock_guard<std::mutex> lk(S.mu);
    S.lat_ms.clear();
    S.n_done = S.n_dropped = S.n_failed = S.traj_done = 0;
    S.t_first = S.t_last = 0.0;
    return PRISM_OK;
}

prism_status prism_server_destroy(prism_server_t ps)
{
    if (!ps) return sfail(PRISM_ERR_INVALID_ARG, "null server");
    Server &S = ps->srv;
    // stop the scheduler (no new work is enqueued after it returns), then let the
    // work in flight and its completion callbacks finish
    {
        std::lock_guard<std::mutex> lk(S.mu);
        S.stop = true;
    }
    S.cv.notify_all();
    if (S.th.joinable()) S.th.join();
    for (cudaStream_t s : S.streams) cudaStreamSynchronize(s);
    for (cudaStream_t s : S.streams) cudaStreamDestroy(s);
    cudaFreeHost(S.slot_flag);
    cudaFree(S.arena.base);
    delete ps;
    return PRISM_OK;
}

}  // extern "C"
