// Serving loop over the evaluator (the C ABI's exago_serve_*): concurrent solver instances on
// grids of different sizes submit evaluation requests; network data and states stay on the
// device (ExaGO's GPU mode keeps model evaluation on the device, Sec. II), and independent
// subproblems run side by side (EMPAR, Sec. V-A).
//
// Continuous batching: a scheduler thread admits queued requests whenever a slot and enough of
// the device arena are free -- not when a whole batch has drained -- and launches each admission
// on one of the server's streams, so requests that arrive while others run overlap with them on
// the GPU.  An admission takes the oldest queued request together with later queued requests for
// the same grid and the same outputs, up to a state budget, and evaluates all their states in one
// launch through a device table of per-state pointers (inputs and outputs stay where each client
// put them).  Each admission's scratch and table are carved from one arena allocated at creation,
// so serving allocates no device memory afterwards.  Completion is signalled by a host function
// queued behind the kernels (it only sets a flag; CUDA calls are not allowed there).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { RQ_QUEUED, RQ_RUNNING, RQ_DONE };

struct Group;

struct Request {
    uint64_t ticket = 0;
    int net_id = 0;
    exago_batch batch{};
    double *f = nullptr, *grad = nullptr, *gh = nullptr, *jval = nullptr, *hval = nullptr;
    size_t ws_bytes = 0;            // workspace of this request alone
    bool has_deadline = false;
    Clock::time_point submitted, deadline, finished;
    cudaEvent_t ready = nullptr;    // recorded on the caller's stream at submission
    ReqState state = RQ_QUEUED;
    exago_status status = EXAGO_OK;
    std::string err;
};

// One admission: the requests evaluated by one launch, its arena range and its stream.
struct Group {
    std::vector<Request *> members;
    size_t ws_off = 0, ws_bytes = 0;
    int stream = -1;
    struct exago_server *server = nullptr;
    std::atomic<int> gpu_done{0};   // set by the host function queued behind the kernels
};

// First-fit allocator over [0, size) with coalescing frees; offsets are 256-byte aligned.
class Arena {
  public:
    void reset(size_t size) {
        free_.clear();
        if (size) free_[0] = size;
    }
    bool alloc(size_t bytes, size_t *off) {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }

  private:
    std::map<size_t, size_t> free_;
};

}  // namespace

struct exago_server {
    size_t budget = 0;
    char *arena_base = nullptr;
    Arena arena;
    int max_slots = 1, running = 0;
    size_t max_queue = 4;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> all_events, free_events;   // one per queued or running request
    std::vector<exago_net_t> nets;
    std::vector<char> cart;        // per net id: evaluated in the cartesian formulation
    std::deque<Request *> queue;
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    std::vector<std::unique_ptr<Group>> running_groups;
    int max_merge = 32;            // states per launch when requests are merged (1: no merging)
    std::vector<double> latencies_ms;
    uint64_t next_ticket = 1;
    int next_stream = 0;
    int device = 0;
    std::mutex mu;                 // requests, queue, arena, slots (never held by on_done)
    std::condition_variable cv_done;
    // Wake-ups of the scheduler: submissions and completions bump `events` under wake_mu, which is
    // never held across a CUDA call (the completion host function takes it; a CUDA call that
    // waits for that function must not hold it).
    std::mutex wake_mu;
    std::condition_variable cv_wake;
    uint64_t events = 0;
    bool stop = false;
    std::thread worker;
};

namespace {

exago_status sfail(exago_status s, const std::string &m) {
    exago::set_last_error(s, m);
    return s;
}

void wake(exago_server *S) {
    {
        std::lock_guard<std::mutex> lk(S->wake_mu);
        S->events++;
    }
    S->cv_wake.notify_one();
}

// Host function behind an admission's kernels: flags completion and wakes the scheduler.  It
// takes only wake_mu, so a CUDA call that waits for it can never wait on the server's lock.
void CUDART_CB on_done(void *p) {
    Group *g = (Group *)p;
    g->gpu_done.store(1, std::memory_order_release);
    wake(g->server);
}

// Whether two requests can share a launch: same grid and the same outputs (the launch computes
// one set of outputs for all its states).
bool same_shape(const Request &a, const Request &b) {
    return a.net_id == b.net_id && !a.f == !b.f && !a.grad == !b.grad && !a.gh == !b.gh &&
           !a.jval == !b.jval && !a.hval == !b.hval;
}

size_t round256(size_t v) { return (v + 255) / 256 * 256; }

// The per-state table of a merged admission (host copy).
std::vector<exago::StateTab> state_table(exago_net_t net, const std::vector<Request *> &members) {
    const exago::HostPlan *p = nullptr;
    const exago::DevNet *d = nullptr;
    int dev = 0;
    exago::net_internal_view(net, &p, &d, &dev);
    std::vector<exago::StateTab> tab;
    for (const Request *r : members) {
        const exago_batch &bt = r->batch;
        for (int j = 0; j < bt.B; j++) {
            exago::StateTab e{};
            e.x = bt.x + (size_t)j * p->n;
            e.lam = bt.lambda ? bt.lambda + (size_t)j * p->m : nullptr;
            e.mask = bt.mask ? bt.mask + (size_t)j * p->nl : nullptr;
            e.gen_mask = bt.gen_mask ? bt.gen_mask + (size_t)j * p->ng : nullptr;
            e.pd_scale = bt.pd_scale ? bt.pd_scale + (size_t)j * p->nb : nullptr;
            e.obj_weight = bt.obj_weight ? bt.obj_weight + j : nullptr;
            e.sigma = bt.obj_factor;
            e.f = r->f ? r->f + j : nullptr;
            e.grad = r->grad ? r->grad + (size_t)j * p->n : nullptr;
            e.gh = r->gh ? r->gh + (size_t)j * p->m : nullptr;
            e.jval = r->jval ? r->jval + (size_t)j * p->nnzJ : nullptr;
            e.hval = r->hval ? r->hval + (size_t)j * p->nnzH : nullptr;
            tab.push_back(e);
        }
    }
    return tab;
}

// Caller holds S->mu.
void finish_locked(exago_server *S, Request *r, exago_status st, const std::string &err) {
    r->state = RQ_DONE;
    r->status = st;
    r->err = err;
    r->finished = Clock::now();
    if (r->ready) {
        S->free_events.push_back(r->ready);
        r->ready = nullptr;
    }
    if (st == EXAGO_OK)
        S->latencies_ms.push_back(
            std::chrono::duration<double, std::milli>(r->finished - r->submitted).count());
    S->cv_done.notify_all();
}

// Admits the oldest queued request, merged with later compatible ones when their states fit the
// merge budget and the arena.  Caller holds S->mu.  False when nothing could be admitted.
bool admit_locked(exago_server *S) {
    nvtxRangePushA("exago_serve_admit");
    struct Pop {
        ~Pop() { nvtxRangePop(); }
    } pop;
    Request *head = S->queue.front();
    exago_net_t net = S->nets[head->net_id];
    std::vector<Request *> members{head};
    int Btot = head->batch.B;
    const bool cart = S->cart[head->net_id] != 0;   // cartesian requests run alone
    if (S->max_merge > 1 && !cart)
        for (auto it = std::next(S->queue.begin()); it != S->queue.end(); ++it) {
            Request *q = *it;
            if (same_shape(*q, *head) && Btot + q->batch.B <= S->max_merge) {
                members.push_back(q);
                Btot += q->batch.B;
            }
        }
    // the merged admission if the arena holds it, else the oldest request alone
    size_t off = 0, bytes = 0, tab_bytes = 0;
    for (;;) {
        if (members.size() == 1) {
            bytes = head->ws_bytes;
            tab_bytes = 0;
        } else {
            size_t ws = 0;
            if (exago_eval_workspace_size(net, Btot, &ws) != EXAGO_OK) ws = (size_t)-1 / 2;
            tab_bytes = round256((size_t)Btot * sizeof(exago::StateTab));
            bytes = tab_bytes + round256(ws > 0 ? ws : 256);
        }
        if (S->arena.alloc(bytes, &off)) break;
        if (members.size() == 1) return false;     // memory-gated: wait for a release
        members.resize(1);
        Btot = head->batch.B;
    }
    for (Request *m : members) S->queue.erase(std::find(S->queue.begin(), S->queue.end(), m));
    std::unique_ptr<Group> g(new Group());
    g->members = members;
    g->ws_off = off;
    g->ws_bytes = bytes;
    g->server = S;
    g->stream = S->next_stream;
    S->next_stream = (S->next_stream + 1) % (int)S->streams.size();
    cudaStream_t st = S->streams[g->stream];
    // inputs produced on the callers' streams before submission are ready first
    exago_status rc = EXAGO_OK;
    for (Request *m : members) {
        cudaError_t ew = cudaStreamWaitEvent(st, m->ready, 0);
        if (ew != cudaSuccess) rc = exago::set_last_error(EXAGO_ECUDA, cudaGetErrorString(ew));
    }
    if (rc == EXAGO_OK) {
        exago_batch bt = head->batch;
        bt.stream = st;
        bt.workspace = S->arena_base + off + tab_bytes;
        bt.workspace_bytes = bytes - tab_bytes;
        if (cart) {
            rc = exago::eval_cart_direct(net, &bt, head->f, head->grad, head->gh, head->jval,
                                         head->hval);
        } else if (members.size() == 1) {
            rc = exago::eval_direct(net, &bt, head->f, head->grad, head->gh, head->jval, head->hval);
        } else {
            // per-state table: copied from pageable memory, so the host vector may go afterwards
            const std::vector<exago::StateTab> tab = state_table(net, members);
            exago::StateTab *dtab = (exago::StateTab *)(S->arena_base + off);
            cudaError_t ec = cudaMemcpyAsync(dtab, tab.data(), tab.size() * sizeof(tab[0]),
                                             cudaMemcpyHostToDevice, st);
            bt.B = Btot;
            rc = ec != cudaSuccess ? exago::set_last_error(EXAGO_ECUDA, cudaGetErrorString(ec))
                                   : exago::eval_direct(net, &bt, head->f, head->grad, head->gh,
                                                        head->jval, head->hval, dtab);
        }
    }
    cudaError_t e = rc == EXAGO_OK ? cudaLaunchHostFunc(st, on_done, g.get()) : cudaSuccess;
    if (rc != EXAGO_OK || e != cudaSuccess) {
        // nothing of this admission is queued behind the host function: release at once (the
        // stream may still read the arena range if a launch went out, so wait for it first)
        cudaStreamSynchronize(st);
        S->arena.release(off, bytes);
        const std::string msg = rc != EXAGO_OK ? exago_last_error() : cudaGetErrorString(e);
        for (Request *m : members) finish_locked(S, m, rc != EXAGO_OK ? rc : EXAGO_ECUDA, msg);
        return true;
    }
    for (Request *m : members) m->state = RQ_RUNNING;
    S->running++;
    S->running_groups.push_back(std::move(g));
    return true;
}

void worker_loop(exago_server *S) {
    cudaSetDevice(S->device);
    uint64_t seen = 0;
    for (;;) {
        bool progress = false;
        Clock::time_point until = Clock::now() + std::chrono::milliseconds(50);
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop) return;
            // retire finished admissions: free their slot and arena range
            for (auto it = S->running_groups.begin(); it != S->running_groups.end();) {
                Group *g = it->get();
                if (g->gpu_done.load(std::memory_order_acquire)) {
                    S->arena.release(g->ws_off, g->ws_bytes);
                    S->running--;
                    for (Request *m : g->members) finish_locked(S, m, EXAGO_OK, "");
                    it = S->running_groups.erase(it);
                    progress = true;
                } else {
                    ++it;
                }
            }
            // expire queued requests whose deadline passed
            const auto now = Clock::now();
            for (auto it = S->queue.begin(); it != S->queue.end();) {
                if ((*it)->has_deadline && now > (*it)->deadline) {
                    finish_locked(S, *it, EXAGO_ETIMEOUT, "deadline passed while queued");
                    it = S->queue.erase(it);
                    progress = true;
                } else {
                    ++it;
                }
            }
            // admit in arrival order while a slot and arena memory are free
            while (!S->queue.empty() && S->running < S->max_slots && admit_locked(S)) progress = true;
            for (Request *q : S->queue)
                if (q->has_deadline && q->deadline < until) until = q->deadline;
        }
        if (!progress) {
            // sleep until a submission, a completion, or the nearest deadline
            std::unique_lock<std::mutex> wl(S->wake_mu);
            S->cv_wake.wait_until(wl, until, [&] { return S->events != seen || S->stop; });
            seen = S->events;
        }
    }
}

Request *find_locked(exago_server *S, uint64_t ticket) {
    auto it = S->reqs.find(ticket);
    return it == S->reqs.end() ? nullptr : it->second.get();
}

}  // namespace

extern "C" {

exago_status exago_serve_create(size_t device_mem_budget, int max_slots, int n_streams,
                                exago_server_t *out) {
    if (!out) return sfail(EXAGO_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_slots < 1 || n_streams < 1 || device_mem_budget == 0)
        return sfail(EXAGO_EINVAL, "need max_slots >= 1, n_streams >= 1 and a non-zero budget");
    std::unique_ptr<exago_server> S(new (std::nothrow) exago_server());
    if (!S) return sfail(EXAGO_ENOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&S->device);
    if (e != cudaSuccess) return sfail(EXAGO_ECUDA, cudaGetErrorString(e));
    S->budget = (device_mem_budget + 255) / 256 * 256;
    e = exago::dev_malloc((void **)&S->arena_base, S->budget);
    if (e != cudaSuccess)
        return sfail(e == cudaErrorMemoryAllocation ? EXAGO_ENOMEM : EXAGO_ECUDA,
                     std::string("cudaMalloc (serve arena): ") + cudaGetErrorString(e));
    S->arena.reset(S->budget);
    S->max_slots = max_slots;
    S->max_queue = 4 * (size_t)max_slots;
    for (int i = 0; i < n_streams; i++) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (auto s2 : S->streams) cudaStreamDestroy(s2);
            cudaFree(S->arena_base);
            return sfail(EXAGO_ECUDA, cudaGetErrorString(e));
        }
        S->streams.push_back(st);
    }
    for (size_t i = 0; i < S->max_queue + (size_t)max_slots; i++) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (auto ev2 : S->all_events) cudaEventDestroy(ev2);
            for (auto s2 : S->streams) cudaStreamDestroy(s2);
            cudaFree(S->arena_base);
            return sfail(EXAGO_ECUDA, cudaGetErrorString(e));
        }
        S->all_events.push_back(ev);
    }
    S->free_events = S->all_events;
    exago_server *raw = S.release();
    raw->worker = std::thread(worker_loop, raw);
    *out = raw;
    return EXAGO_OK;
}

static exago_status register_net(exago_server_t S, exago_net_t net, int *net_id, bool cart) {
    if (!S || !net || !net_id) return sfail(EXAGO_EINVAL, "null argument");
    const exago::HostPlan *p = nullptr;
    const exago::DevNet *d = nullptr;
    int dev = 0;
    if (!exago::net_internal_view(net, &p, &d, &dev))
        return sfail(EXAGO_EINVAL, "invalid net (NULL or planned without a device)");
    std::lock_guard<std::mutex> lk(S->mu);
    S->nets.push_back(net);
    S->cart.push_back(cart ? 1 : 0);
    *net_id = (int)S->nets.size() - 1;
    return EXAGO_OK;
}

exago_status exago_serve_register(exago_server_t S, exago_net_t net, int *net_id) {
    return register_net(S, net, net_id, false);
}

exago_status exago_serve_register_cart(exago_server_t S, exago_net_t net, int *net_id) {
    return register_net(S, net, net_id, true);
}

exago_status exago_serve_submit(exago_server_t S, int net_id, const exago_batch *req, double *f,
                                double *grad, double *gh, double *jval, double *hval,
                                double deadline_ms, uint64_t *ticket) {
    if (!S || !req || !ticket) return sfail(EXAGO_EINVAL, "null argument");
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) return sfail(EXAGO_ENOMEM, "host allocation failed");
    exago_net_t net;
    bool cart;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (net_id < 0 || net_id >= (int)S->nets.size()) return sfail(EXAGO_EINVAL, "unknown net id");
        net = S->nets[net_id];
        cart = S->cart[net_id] != 0;
    }
    if (req->B < 1 || !req->x) return sfail(EXAGO_EINVAL, "request needs B >= 1 and x");
    if (hval && !req->lambda) return sfail(EXAGO_EINVAL, "the Hessian needs lambda");
    size_t ws = 0;
    exago_status st = cart ? exago_eval_cart_workspace_size(net, req->B, &ws)
                           : exago_eval_workspace_size(net, req->B, &ws);
    if (st != EXAGO_OK) return st;
    if ((ws + 255) / 256 * 256 > S->budget)
        return sfail(EXAGO_ENOMEM, "request needs more workspace than the server's whole budget");
    r->net_id = net_id;
    r->batch = *req;
    r->f = f; r->grad = grad; r->gh = gh; r->jval = jval; r->hval = hval;
    r->ws_bytes = round256(ws > 0 ? ws : 256);
    r->submitted = Clock::now();
    if (deadline_ms > 0) {
        r->has_deadline = true;
        r->deadline = r->submitted + std::chrono::microseconds((long long)(deadline_ms * 1000.0));
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->queue.size() >= S->max_queue || S->free_events.empty())
            return sfail(EXAGO_EBUSY, "serve queue full");
        cudaError_t e = cudaEventRecord(S->free_events.back(), (cudaStream_t)req->stream);
        if (e != cudaSuccess)
            return sfail(EXAGO_ECUDA, std::string("cudaEventRecord (request stream): ") + cudaGetErrorString(e));
        r->ready = S->free_events.back();
        S->free_events.pop_back();
        r->ticket = S->next_ticket++;
        *ticket = r->ticket;
        S->queue.push_back(r.get());
        S->reqs[r->ticket] = std::move(r);
    }
    wake(S);
    return EXAGO_OK;
}

exago_status exago_serve_set_merge(exago_server_t S, int max_states) {
    if (!S || max_states < 1) return sfail(EXAGO_EINVAL, "need a server and max_states >= 1");
    std::lock_guard<std::mutex> lk(S->mu);
    S->max_merge = max_states;
    return EXAGO_OK;
}

exago_status exago_serve_poll(exago_server_t S, uint64_t ticket, int *done) {
    if (!S || !done) return sfail(EXAGO_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    Request *r = find_locked(S, ticket);
    if (!r) return sfail(EXAGO_EINVAL, "unknown ticket");
    *done = r->state == RQ_DONE;
    return EXAGO_OK;
}

exago_status exago_serve_wait(exago_server_t S, uint64_t ticket, double timeout_ms) {
    if (!S) return sfail(EXAGO_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(S->mu);
    Request *r = find_locked(S, ticket);
    if (!r) return sfail(EXAGO_EINVAL, "unknown ticket");
    auto pred = [&] { return r->state == RQ_DONE; };
    if (timeout_ms > 0) {
        if (!S->cv_done.wait_for(lk, std::chrono::microseconds((long long)(timeout_ms * 1000.0)), pred))
            return sfail(EXAGO_EBUSY, "request still queued or running");
    } else {
        S->cv_done.wait(lk, pred);
    }
    const exago_status st = r->status;
    const std::string err = r->err;
    S->reqs.erase(ticket);
    if (st != EXAGO_OK) return sfail(st, err);
    return EXAGO_OK;
}

exago_status exago_serve_stats(exago_server_t S, double *p50_ms, double *p99_ms, uint64_t *completed) {
    if (!S) return sfail(EXAGO_EINVAL, "null server");
    std::vector<double> v;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        v = S->latencies_ms;
    }
    if (completed) *completed = v.size();
    std::sort(v.begin(), v.end());
    auto q = [&](double p) { return v.empty() ? 0.0 : v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
    if (p50_ms) *p50_ms = q(0.50);
    if (p99_ms) *p99_ms = q(0.99);
    return EXAGO_OK;
}

exago_status exago_serve_destroy(exago_server_t S) {
    if (!S) return EXAGO_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (Request *r : S->queue) finish_locked(S, r, EXAGO_ESTATE, "server destroyed");
        S->queue.clear();
    }
    {
        std::lock_guard<std::mutex> lk(S->wake_mu);
        S->stop = true;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_wake.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto st : S->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto ev : S->all_events) cudaEventDestroy(ev);
    cudaFree(S->arena_base);
    delete S;
    return EXAGO_OK;
}

}  // extern "C"

// ---- native load generator (exago_serve_drive) ------------------------------------------------
// The submission loop of a benchmark's simulated clients, in C++ so that the arrival process and
// the polling are not limited by an interpreter: closed loop, or Poisson arrivals with spin-timed
// submission.  Uses only the public serving calls.
#include <random>

extern "C" exago_status exago_serve_drive(exago_server_t S, const exago_serve_client *clients,
                                          const int *group, int n_clients, const double *weight,
                                          int n_groups, double rate, double seconds,
                                          uint64_t seed, double *result) {
    if (!S || !clients || !group || !weight || !result || n_clients < 1 || n_groups < 1 ||
        !(seconds > 0.0))
        return sfail(EXAGO_EINVAL, "exago_serve_drive: bad argument");
    std::vector<std::vector<int>> members(n_groups), free_c(n_groups);
    for (int i = 0; i < n_clients; i++) {
        if (group[i] < 0 || group[i] >= n_groups || !clients[i].batch)
            return sfail(EXAGO_EINVAL, "exago_serve_drive: bad client");
        members[group[i]].push_back(i);
    }
    double wsum = 0.0;
    for (int g = 0; g < n_groups; g++) {
        if (!(weight[g] >= 0.0)) return sfail(EXAGO_EINVAL, "exago_serve_drive: bad weight");
        if (members[g].empty() && weight[g] > 0.0)
            return sfail(EXAGO_EINVAL, "exago_serve_drive: a weighted group has no client");
        wsum += weight[g];
    }
    if (!(wsum > 0.0)) return sfail(EXAGO_EINVAL, "exago_serve_drive: weights sum to 0");
    std::vector<uint64_t> ticket(n_clients, 0);
    std::vector<char> busy(n_clients, 0);
    exago_status first = EXAGO_OK;
    auto note = [&](exago_status s) {
        if (s != EXAGO_OK && first == EXAGO_OK) first = s;
        return s;
    };
    auto submit = [&](int c) {
        const exago_serve_client &k = clients[c];
        exago_status s = note(exago_serve_submit(S, k.net_id, k.batch, k.f, k.grad, k.gh, k.jval,
                                                 k.hval, 0.0, &ticket[c]));
        busy[c] = s == EXAGO_OK;
        return s;
    };
    auto finish = [&](int c) {
        note(exago_serve_wait(S, ticket[c], 0.0));
        busy[c] = 0;
    };
    double deferred = 0.0;
    const auto t0 = Clock::now();
    auto elapsed = [&] { return std::chrono::duration<double>(Clock::now() - t0).count(); };
    if (rate <= 0.0) {
        for (int c = 0; c < n_clients && first == EXAGO_OK; c++) submit(c);
        for (int k = 0; elapsed() < seconds && first == EXAGO_OK; k++) {
            const int c = k % n_clients;
            if (busy[c]) finish(c);
            if (first == EXAGO_OK) submit(c);
        }
    } else {
        std::mt19937_64 rng(seed);
        std::exponential_distribution<double> gap(rate);
        std::discrete_distribution<int> pick(weight, weight + n_groups);
        for (int g = 0; g < n_groups; g++) free_c[g] = members[g];
        double t_next = 0.0;
        while (first == EXAGO_OK) {
            t_next += gap(rng);
            // the run ends at `seconds` of arrival time or of wall time, whichever comes first
            // (arrivals offered faster than they can be submitted fall behind the clock)
            if (t_next >= seconds || elapsed() >= seconds) break;
            while (elapsed() < t_next) {
            }
            const int g = pick(rng);
            if (free_c[g].empty()) {   // collect this group's finished requests
                for (int c : members[g]) {
                    int done = 0;
                    if (busy[c] && note(exago_serve_poll(S, ticket[c], &done)) == EXAGO_OK && done) {
                        finish(c);
                        free_c[g].push_back(c);
                    }
                }
            }
            if (free_c[g].empty()) {   // wait for the oldest outstanding one
                deferred += 1.0;
                int oldest = -1;
                for (int c : members[g])
                    if (busy[c] && (oldest < 0 || ticket[c] < ticket[oldest])) oldest = c;
                if (oldest < 0) break;
                finish(oldest);
                free_c[g].push_back(oldest);
            }
            const int c = free_c[g].back();
            free_c[g].pop_back();
            submit(c);
        }
    }
    for (int c = 0; c < n_clients; c++)
        if (busy[c]) finish(c);
    const double dt = elapsed();
    double p50 = 0.0, p99 = 0.0;
    uint64_t n = 0;
    note(exago_serve_stats(S, &p50, &p99, &n));
    result[0] = (double)n;
    result[1] = dt;
    result[2] = p50;
    result[3] = p99;
    result[4] = deferred;
    return first;
}
