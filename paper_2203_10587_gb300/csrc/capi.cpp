// C ABI of the evaluator (declared in include/exago.h): network lifetime, pattern queries and the
// evaluation entry points of the polar AC-OPF model (ExaGO, Sec. III, eqs. (7)-(10)).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

using namespace exago;

namespace exago {

// Testing hook: the next g_fail_allocs device allocations fail as if the device were out of
// memory (exago_test_fail_allocations).
std::atomic<int> g_fail_allocs{0};

// Every device allocation of a net goes through here.
cudaError_t dev_malloc(void **p, size_t bytes) {
    int left = g_fail_allocs.load();
    while (left > 0 && !g_fail_allocs.compare_exchange_weak(left, left - 1)) {
    }
    if (left > 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) cudaGetLastError();   // reported here; must not resurface at a launch
    return e;
}

}  // namespace exago

namespace {

thread_local std::string g_err;

// An NVTX range over one C-ABI call (visible to Nsight tools; free without them).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

exago_status fail(exago_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

exago_status cuda_fail(cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(e == cudaErrorMemoryAllocation ? EXAGO_ENOMEM : EXAGO_ECUDA, m);
}

}  // namespace

// One instantiated CUDA graph of the persistent schedule, keyed by every argument it bakes in.
struct GraphEntry {
    std::vector<uint64_t> key;
    cudaGraphExec_t exec = nullptr;
    uint64_t last_use = 0;
};

struct exago_net {
    HostPlan plan;
    bool on_device = false;
    int device = -1;
    int sm_count = 0;
    int smem_per_sm = 0;          // shared memory per SM (bytes)
    DevNet dev{};
    std::vector<void *> allocs;
    int *status_host = nullptr;   // host-mapped device status word
    void *ws = nullptr;           // internal workspace
    size_t ws_bytes = 0;
    // Stream order of the internal workspace's users: every uncaptured call that uses it records
    // ws_ev on its stream, and a call on another stream first waits for that event.  ws_captured:
    // some use was captured into a caller's graph, whose replays the event cannot see.
    cudaEvent_t ws_ev = nullptr;
    cudaStream_t ws_stream = nullptr;
    bool ws_captured = false;
    std::mutex mu;                // guards the workspace, the graph cache and the configuration
    exago_config cfg{};           // user configuration (zeros = automatic)
    std::map<int, exago_config> tuned;   // autotuned configuration per batch size
    std::vector<GraphEntry> graphs;
    uint64_t graph_clock = 0;
    std::vector<std::vector<uint64_t>> graph_seen;   // argument sets launched once, oldest first
    cudaStream_t cap_stream = nullptr;
    cudaStream_t side_stream = nullptr;   // pipelined schedule: bus kernels
    cudaEvent_t pipe_ev[18] = {};
    std::map<uint64_t, int> occ;  // resident CTAs per SM by (schedule, block, occupancy, shared memory)
    std::map<int, int> item_rows; // warp tiles: most row doubles of one bus item, by buses per item
};

namespace {

template <typename T>
exago_status upload(exago_net *net, const std::vector<T> &v, const T **out) {
    *out = nullptr;
    if (v.empty()) return EXAGO_OK;
    void *p = nullptr;
    cudaError_t e = dev_malloc(&p, v.size() * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (network arrays)");
    net->allocs.push_back(p);
    e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy (network arrays)");
    *out = (const T *)p;
    return EXAGO_OK;
}

exago_status alloc_dev(exago_net *net, size_t bytes, double **out) {
    *out = nullptr;
    if (bytes == 0) return EXAGO_OK;
    void *p = nullptr;
    cudaError_t e = dev_malloc(&p, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (admittances)");
    net->allocs.push_back(p);
    *out = (double *)p;
    return EXAGO_OK;
}

void free_device(exago_net *net) {
    if (!net->graphs.empty() || net->cap_stream || net->side_stream) cudaDeviceSynchronize();
    for (auto &g : net->graphs) cudaGraphExecDestroy(g.exec);
    net->graphs.clear();
    if (net->cap_stream) cudaStreamDestroy(net->cap_stream);
    net->cap_stream = nullptr;
    if (net->side_stream) {
        cudaStreamSynchronize(net->side_stream);
        cudaStreamDestroy(net->side_stream);
        for (auto &ev : net->pipe_ev)
            if (ev) cudaEventDestroy(ev);
    }
    net->side_stream = nullptr;
    for (void *p : net->allocs) cudaFree(p);
    net->allocs.clear();
    if (net->ws) cudaFree(net->ws);
    net->ws = nullptr;
    net->ws_bytes = 0;
    if (net->ws_ev) cudaEventDestroy(net->ws_ev);
    net->ws_ev = nullptr;
    if (net->status_host) cudaFreeHost(net->status_host);
    net->status_host = nullptr;
    net->on_device = false;
}

exago_status do_upload(exago_net *net) {
    const HostPlan &p = net->plan;
    DevNet &d = net->dev;
    exago_status s;
    cudaError_t e = cudaGetDevice(&net->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    e = cudaDeviceGetAttribute(&net->sm_count, cudaDevAttrMultiProcessorCount, net->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    e = cudaDeviceGetAttribute(&net->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                               net->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    d = DevNet{};
    d.nb = p.nb; d.nl = p.nl; d.ng = p.ng; d.n = p.n; d.m = p.m;
    d.nslot = p.nslot;
    d.chk_nslot = p.nslot;
    d.nnzJ = p.nnzJ; d.nnzJg = p.nnzJg; d.nnzH = p.nnzH;
    d.baseMVA = p.baseMVA;
    d.hpg = p.Hrowptr[2 * p.nb];
    d.jP_end = (int)p.Jrowptr[p.nb];
    d.jQ_end = (int)p.Jrowptr[2 * p.nb];
    d.hA_end = (int)p.Hrowptr[p.nb];
    d.hM_end = (int)p.Hrowptr[2 * p.nb];
    for (int t = 0; t < 4; t++) {   // largest bus tile's rows (and components), 32 to 256 buses
        const int T = 32 << t;
        int64_t rows = 0, all = 0, bulk = 0;
        for (int i0 = 0; i0 < p.nb; i0 += T) {
            const int i1 = i0 + T < p.nb ? i0 + T : p.nb;
            const int64_t r = 2 * (p.Jrowptr[i1] - p.Jrowptr[i0]) + (p.Hrowptr[i1] - p.Hrowptr[i0]) +
                              (p.Hrowptr[p.nb + i1] - p.Hrowptr[p.nb + i0]);
            const int64_t a = r + (int64_t)kDiagComps * (p.slot_ptr[i1] - p.slot_ptr[i0]);
            const int64_t k = r + (int64_t)NCOMP * (p.slot_ptr[i1] - p.slot_ptr[i0]);
            if (r > rows) rows = r;
            if (a > all) all = a;
            if (k > bulk) bulk = k;
        }
        d.stage_cap_rows[t] = (int)(rows < kStageMaxDoubles ? rows : kStageMaxDoubles);
        d.stage_cap_all[t] = (int)(all < kStageMaxDoubles ? all : kStageMaxDoubles);
        d.stage_cap_bulk[t] = (int)(bulk < kStageMaxDoubles ? bulk : kStageMaxDoubles);
    }
#define UP(field, vec) if ((s = upload(net, p.vec, &d.field)) != EXAGO_OK) return s
    UP(f, f); UP(t, t);
    UP(slot_ptr, slot_ptr); UP(slot_nbr, slot_nbr); UP(slot_ref, slot_ref); UP(br_slot, br_slot);
    UP(slot_bus, slot_bus); UP(slot_pos, slot_pos);
    UP(bus_jP, bus_jP); UP(bus_jQ, bus_jQ); UP(bus_hA, bus_hA); UP(bus_hM, bus_hM);
    UP(bus_k, bus_k); UP(bus_nlow, bus_nlow); UP(bus_perm, bus_perm);
    UP(Gs, Gs); UP(Bs, Bs); UP(Pd, Pd); UP(Qd, Qd);
    UP(gen_ptr, gen_ptr); UP(gen_ord, gen_ord);
    UP(c2, c2); UP(c1, c1); UP(c0, c0); UP(c2g, c2g); UP(c1g, c1g);
#undef UP
    // branch parameters, then the pi-model admittances evaluated on the device
    const double *r = nullptr, *x = nullptr, *b = nullptr, *tap = nullptr;
    if ((s = upload(net, p.r, &r)) != EXAGO_OK) return s;
    if ((s = upload(net, p.x, &x)) != EXAGO_OK) return s;
    if ((s = upload(net, p.b, &b)) != EXAGO_OK) return s;
    if ((s = upload(net, p.tap, &tap)) != EXAGO_OK) return s;
    const double *shift = nullptr;
    if ((s = upload(net, p.shift, &shift)) != EXAGO_OK) return s;   // empty: no phase shifters
    double *Y[13] = {};
    for (int k = 0; k < (shift ? 13 : 11); k++)
        if ((s = alloc_dev(net, (size_t)p.nl * sizeof(double), &Y[k])) != EXAGO_OK) return s;
    d.Gff = Y[0]; d.Bff = Y[1]; d.Gtt = Y[2]; d.Btt = Y[3]; d.Gft = Y[4]; d.Bft = Y[5];
    d.Gff2 = Y[6]; d.Bff2 = Y[7]; d.Gtt2 = Y[8]; d.Btt2 = Y[9]; d.Kft = Y[10];
    d.Gtf = Y[11]; d.Btf = Y[12];
    cudaStream_t st;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreate");
    int le = launch_admittance(r, x, b, tap, shift, p.nl, Y, st);
    e = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (le != 0) return cuda_fail((cudaError_t)le, "admittance kernel launch");
    if (e != cudaSuccess) return cuda_fail(e, "admittance kernel");
    e = cudaHostAlloc((void **)&net->status_host, sizeof(int), cudaHostAllocMapped);
    if (e != cudaSuccess) return cuda_fail(e, "cudaHostAlloc (status word)");
    *net->status_host = 0;
    e = cudaHostGetDevicePointer((void **)&d.status, net->status_host, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaHostGetDevicePointer (status word)");
    {   // once per device: let the staged bus kernels use more than 48 KB of shared memory
        static std::mutex mu;
        static bool done[64] = {false};
        std::lock_guard<std::mutex> lk(mu);
        if (net->device >= 0 && net->device < 64 && !done[net->device]) {
            int le2 = persist_allow_stage();
            if (le2 == 0) le2 = bus_allow_stage();
            if (le2 == 0) le2 = cart_allow_stage();
            if (le2 == 0) le2 = persist_w_allow_stage();
            if (le2 != 0) return cuda_fail((cudaError_t)le2, "cudaFuncSetAttribute");
            done[net->device] = true;
        }
    }
    net->on_device = true;
    return EXAGO_OK;
}

exago_status plan_only(int nb, const double *Gs, const double *Bs, const double *Pd,
                       const double *Qd, int nl, const int *f, const int *t, const double *r,
                       const double *x, const double *b, const double *tap, const double *rateA,
                       int ng, const int *gbus, const double *c2, const double *c1,
                       const double *c0, double baseMVA, const double *shift,
                       exago_net_t *out) {
    if (!out) return fail(EXAGO_EINVAL, "out is NULL");
    *out = nullptr;
    exago_net *net = new (std::nothrow) exago_net();
    if (!net) return fail(EXAGO_ENOMEM, "host allocation failed");
    std::string err;
    exago_status s;
    try {
        s = build_plan(net->plan, nb, Gs, Bs, Pd, Qd, nl, f, t, r, x, b, tap, rateA, ng, gbus,
                       c2, c1, c0, baseMVA, shift, err);
    } catch (const std::bad_alloc &) {
        s = EXAGO_ENOMEM;
        err = "host allocation failed while planning";
    }
    if (s != EXAGO_OK) {
        delete net;
        return fail(s, err);
    }
    *out = net;
    return EXAGO_OK;
}

// Launch settings of one call, resolved from the net's configuration and the batch size.
struct Resolved {
    int schedule;          // EXAGO_SCHED_KERNELS or EXAGO_SCHED_PERSISTENT
    int block, occ_warps, stage_recs, stage_cap, grid, lag, ring, use_graph, force_timeout;
    int group;             // persistent: tiles per work item
    int warp_tiles;        // persistent: warp-tiled kernel (a warp per branch or bus, a lane per
                           // state); lag and ring then count groups of 32 states
    int chunk, pipe_ring;  // pipelined schedule
    long long spin_limit;
};

constexpr long long kDefaultSpinLimit = 1ll << 22;   // polls of ~0.4 us: about 1.7 s

// Resident CTAs per SM of the persistent kernel (persistent) or of the bus kernel (otherwise)
// with `smem` bytes of dynamic shared memory, cached.
// warp: the warp-tiled persistent kernel (smem: its lanes' staging row in doubles).
int occupancy(exago_net *net, bool persistent, int block, int occ_warps, size_t smem,
              bool warp = false) {
    const uint64_t key = ((uint64_t)persistent << 62) | ((uint64_t)warp << 61) |
                         ((uint64_t)block << 48) | ((uint64_t)occ_warps << 40) | (uint64_t)smem;
    auto it = net->occ.find(key);
    if (it != net->occ.end()) return it->second;
    const int o = warp         ? persist_w_blocks_per_sm(block, occ_warps, (int)smem)
                  : persistent ? persist_blocks_per_sm(block, occ_warps, smem)
                               : bus_blocks_per_sm(smem);
    net->occ[key] = o;
    return o;
}

// Shared-memory doubles of one bus tile: its row segments (and, slot-parallel, its slots'
// diagonal components), but no more than keeps the register-limited number of resident CTAs per
// SM.  A tile that does not fit writes its rows straight to global memory (and walks its slots
// per bus).
int stage_cap(exago_net *net, bool persistent, int block, int occ_warps, int stage_recs) {
    const int t = stage_index(persistent ? block : 128);
    const int by_regs = occupancy(net, persistent, block, occ_warps, 0);
    const long budget = ((long)net->smem_per_sm / (by_regs > 0 ? by_regs : 1) - 4096) / 8;
    const int want = stage_recs == 2   ? net->dev.stage_cap_bulk[t]
                     : stage_recs == 1 ? net->dev.stage_cap_all[t]
                                       : net->dev.stage_cap_rows[t];
    return want > budget ? (int)(budget & ~1l) : want;
}

// The most row doubles (J rows P and Q, H rows Va and Vm) that one bus item of per_item
// consecutive buses writes, cached per per_item.
int item_rows_max(exago_net *net, int per_item) {
    auto it = net->item_rows.find(per_item);
    if (it != net->item_rows.end()) return it->second;
    const HostPlan &p = net->plan;
    const DevNet &d = net->dev;
    auto at = [&](const std::vector<int> &v, int i, int end) { return i < p.nb ? v[i] : end; };
    int mx = 0;
    for (int i0 = 0; i0 < p.nb; i0 += per_item) {
        const int i1 = std::min(p.nb, i0 + per_item);
        const int L = 2 * (at(p.bus_jP, i1, d.jP_end) - p.bus_jP[i0]) +
                      (at(p.bus_hA, i1, d.hA_end) - p.bus_hA[i0]) +
                      (at(p.bus_hM, i1, d.hM_end) - p.bus_hM[i0]);
        mx = std::max(mx, L);
    }
    net->item_rows[per_item] = mx;
    return mx;
}

Resolved resolve(exago_net *net, int B) {
    exago_config c = net->cfg;
    if (c.schedule == EXAGO_SCHED_AUTO) {
        auto it = net->tuned.find(B);
        if (it != net->tuned.end()) {
            exago_config t = it->second;
            t.spin_limit = c.spin_limit;
            t.test_force_timeout = c.test_force_timeout;
            c = t;
        }
    }
    Resolved r{};
    r.schedule = (c.schedule == EXAGO_SCHED_KERNELS || c.schedule == EXAGO_SCHED_PIPELINED)
                     ? c.schedule : EXAGO_SCHED_PERSISTENT;
    {   // pipelined: `ring` chunks of records within about 48 MB of L2
        const double per_state = (double)NCOMP * net->plan.nslot * sizeof(double);
        int pr = c.ring > 0 && c.schedule == EXAGO_SCHED_PIPELINED ? c.ring : 3;
        if (pr > 7) pr = 7;
        int ch = c.chunk > 0 ? c.chunk : (int)(48e6 / (pr * (per_state > 1 ? per_state : 1)));
        if (ch < 1) ch = 1;
        if (ch > B) ch = B;
        r.chunk = ch;
        r.pipe_ring = pr;
    }
    r.block = (c.block == 32 || c.block == 128 || c.block == 256) ? c.block : 64;
    r.occ_warps = (c.occupancy == 8 || c.occupancy == 24) ? c.occupancy : 16;
    const bool pers = r.schedule == EXAGO_SCHED_PERSISTENT;
    // bulk record copies only in the persistent kernel (others walk the records through L2)
    r.stage_recs = c.stage_records == EXAGO_STAGE_ON     ? 1
                   : c.stage_records == EXAGO_STAGE_BULK ? (pers ? 2 : 0)
                                                         : 0;
    r.use_graph = c.use_graph != EXAGO_GRAPH_OFF;
    r.spin_limit = c.spin_limit > 0 ? c.spin_limit : kDefaultSpinLimit;
    r.force_timeout = c.test_force_timeout ? 1 : 0;
    r.group = c.tile_group >= 1 && c.tile_group <= 4 ? c.tile_group : 1;
    if (pers && c.tiling == EXAGO_TILING_WARP) {
        // warp-tiled: blocks of 128 (default) or 64 threads, no record staging; the lag and the
        // ring count groups of 32 states.  By default bus items trail by the groups the resident
        // CTAs hold in branch work plus two, and the ring holds two lags (measured on 2000 buses
        // x 512, 128 threads: lag 3 and ring 6 take 0.469 ms, as do larger lags and rings up to
        // 6 / 12; lag 2 and ring 4 0.502 ms; lag 2 and ring 3 0.755 ms).
        r.warp_tiles = 1;
        r.block = c.block == 64 ? 64 : 128;
        r.occ_warps = c.occupancy == 8 ? 8 : 16;
        r.stage_recs = 0;
        const int G = (B + 31) / 32;
        const int per_item = (r.block / 32) * r.group;
        // Each lane stages its state's rows of one item in shared memory (odd row length: no bank
        // conflicts when the lanes write one position each): the longest bus item's rows, and the
        // branch items' 10 doubles per branch, within what keeps the register-limited residency.
        const int by_regs = occupancy(net, true, r.block, r.occ_warps, 0, true);
        const long budget = ((long)net->smem_per_sm / (by_regs > 0 ? by_regs : 1) - 1024) / (8 * 32);
        int want = item_rows_max(net, per_item);
        if (want < 10 * per_item) want = 10 * per_item;
        want |= 1;
        const int cap = (kStageMaxDoubles / 32 - 1) | 1;
        if (want > cap) want = cap;
        r.stage_cap = want <= budget ? want : (int)((budget - 1) | 1);
        if (r.stage_cap < 10 * per_item) r.stage_cap = 0;   // no staging at all
        r.grid = net->sm_count * occupancy(net, true, r.block, r.occ_warps, r.stage_cap, true);
        const int Tbr = (net->plan.nl + per_item - 1) / per_item;
        int lag = c.lag > 0 ? c.lag : (Tbr > 0 ? (r.grid + Tbr - 1) / Tbr : 1) + 2;
        if (lag > G) lag = G;
        if (lag < 1) lag = 1;
        int ring = c.ring > 0 ? c.ring : 2 * lag;
        if (ring <= lag) ring = lag + 1;
        if (ring > G + 1) ring = G + 1 > lag ? G + 1 : lag + 1;
        r.lag = lag;
        r.ring = ring;
        return r;
    }
    r.stage_cap = stage_cap(net, pers, r.block, r.occ_warps, r.stage_recs);
    r.grid = net->sm_count * occupancy(net, true, r.block, r.occ_warps,
                                       pers ? (size_t)r.stage_cap * sizeof(double) : 0);
    const int Tbr = (net->plan.nl + r.block * r.group - 1) / (r.block * r.group);
    // Bus tiles trail by 4/3 of the states the resident CTAs can hold in branch work, plus two,
    // and the ring holds three lags: bus tiles then seldom wait for branch tiles, nor branch
    // tiles for ring slots (measured on 2000 buses x 512: lag 40 and ring 122 take 0.43 ms, lag
    // 31 and ring 64 0.45 ms, lag 16 and ring 34 0.62 ms).
    int lag = c.lag > 0 ? c.lag : (Tbr > 0 ? (4 * r.grid + 3 * Tbr - 1) / (3 * Tbr) : 1) + 2;
    if (lag > B) lag = B;
    if (lag < 1) lag = 1;
    int ring = c.ring > 0 ? c.ring : 3 * lag + 2;
    if (ring <= lag) ring = lag + 1;
    if (ring > B + 1) ring = B + 1 > lag ? B + 1 : lag + 1;
    r.lag = lag;
    r.ring = ring;
    return r;
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// Branch-end records of one state.
size_t slot_bytes(const exago_net *net) {
    return (size_t)NCOMP * (size_t)net->dev.nslot * sizeof(double);
}

// One ring slot of the persistent schedule: a state's records, then its objective partials.
size_t persist_slot_bytes(const exago_net *net) {
    return slot_bytes(net) + (size_t)kObjLanes * sizeof(double);
}

// Ring scratch of a persistent launch: `ring` state slots, or group slots when warp-tiled.
size_t persist_ring_bytes(const exago_net *net, const Resolved &r) {
    if (r.warp_tiles) return round256(r.ring * persist_w_slot_doubles(net->dev.nslot) * sizeof(double));
    return round256(r.ring * persist_slot_bytes(net));
}

// Workspace of the persistent schedule: ring scratch, then counters.
size_t persist_bytes(const exago_net *net, const Resolved &r, int B) {
    return persist_ring_bytes(net, r) +
           round256((size_t)(1 + 2 * (size_t)B + 256) * sizeof(int));
}

size_t need_bytes(exago_net *net, int B) {
    size_t k = workspace_bytes(net->plan, B);
    if (!net->on_device) return k;
    Resolved r = resolve(net, B);
    size_t p = persist_bytes(net, r, B);
    size_t q = round256((size_t)r.pipe_ring * r.chunk * slot_bytes(net));
    return k > p ? (k > q ? k : q) : (p > q ? p : q);
}

exago_status check_batch(exago_net *net, const exago_batch *bt, bool need_lam) {
    if (!net) return fail(EXAGO_EINVAL, "net is NULL");
    if (!net->on_device) return fail(EXAGO_ESTATE, "net was planned without a device (exago_net_plan)");
    if (!bt) return fail(EXAGO_EINVAL, "batch is NULL");
    if (bt->B < 0) return fail(EXAGO_EINVAL, "batch B < 0");
    if (bt->B == 0) return EXAGO_OK;
    if (!bt->x) return fail(EXAGO_EINVAL, "batch x is NULL");
    if (need_lam && !bt->lambda) return fail(EXAGO_EINVAL, "batch lambda is NULL (needed by the Hessian)");
    if (bt->workspace) {
        if (((uintptr_t)bt->workspace & 255) != 0) return fail(EXAGO_EINVAL, "workspace not 256-byte aligned");
        std::lock_guard<std::mutex> lk(net->mu);
        if (bt->workspace_bytes < need_bytes(net, bt->B))
            return fail(EXAGO_EINVAL, "workspace smaller than exago_eval_workspace_size");
    }
    return EXAGO_OK;
}

// Caller holds net->mu.
exago_status ensure_workspace_locked(exago_net *net, size_t need) {
    if (net->ws_bytes >= need) return EXAGO_OK;
    if (net->ws) {
        // Earlier work may still use the old buffer.  Uncaptured uses are chained through ws_ev
        // (ws_acquire_locked), so its last record covers them all; a use captured into a
        // caller's graph is not, and then the whole device is drained.
        cudaError_t e = net->ws_captured || !net->ws_ev ? cudaDeviceSynchronize()
                                                        : cudaEventSynchronize(net->ws_ev);
        if (e != cudaSuccess) return cuda_fail(e, "synchronisation before workspace growth");
        cudaFree(net->ws);
        net->ws = nullptr;
        net->ws_bytes = 0;
    }
    cudaError_t e = dev_malloc(&net->ws, need);
    if (e != cudaSuccess) {
        net->ws = nullptr;
        return cuda_fail(e, "cudaMalloc (workspace)");
    }
    net->ws_bytes = need;
    return EXAGO_OK;
}

// Before a call queues work that uses the internal workspace on `st`: waits (on the device) for
// the last uncaptured use on another stream.  Caller holds net->mu.
exago_status ws_acquire_locked(exago_net *net, cudaStream_t st, bool capturing) {
    if (capturing) {
        net->ws_captured = true;
        return EXAGO_OK;
    }
    if (!net->ws_ev) {
        cudaError_t e = cudaEventCreateWithFlags(&net->ws_ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate (workspace order)");
        return EXAGO_OK;
    }
    if (net->ws_stream != st) {
        cudaError_t e = cudaStreamWaitEvent(st, net->ws_ev, 0);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent (workspace order)");
    }
    return EXAGO_OK;
}

// After a call has queued its work that uses the internal workspace on `st`.  Caller holds
// net->mu.
exago_status ws_release_locked(exago_net *net, cudaStream_t st, bool capturing) {
    if (capturing) return EXAGO_OK;
    cudaError_t e = cudaEventRecord(net->ws_ev, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord (workspace order)");
    net->ws_stream = st;
    return EXAGO_OK;
}

exago_status is_capturing(cudaStream_t st, bool *capturing) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
    *capturing = cap != cudaStreamCaptureStatusNone;
    return EXAGO_OK;
}

exago_status ensure_workspace(exago_net *net, int B) {
    std::lock_guard<std::mutex> lk(net->mu);
    return ensure_workspace_locked(net, need_bytes(net, B));
}

uint64_t bits(double v) {
    uint64_t u;
    std::memcpy(&u, &v, sizeof u);
    return u;
}

// Launches a schedule through a cached instantiated CUDA graph: `launch` queues the schedule's
// work on a capture stream once per distinct key (every argument the work bakes in).  Caller holds
// net->mu.
exago_status launch_graph_locked(exago_net *net, const std::vector<uint64_t> &key,
                                 const std::function<int(cudaStream_t)> &launch,
                                 cudaStream_t stream) {
    GraphEntry *hit = nullptr;
    for (auto &g : net->graphs)
        if (g.key == key) { hit = &g; break; }
    cudaError_t e;
    if (!hit) {
        // An argument set is captured on its second use among the last 32 uncached calls; a
        // one-off set (a caller cycling through many buffers) launches directly instead of paying
        // a capture and an instantiation on the host.
        auto seen = std::find(net->graph_seen.begin(), net->graph_seen.end(), key);
        if (seen == net->graph_seen.end()) {
            if (net->graph_seen.size() >= 32) net->graph_seen.erase(net->graph_seen.begin());
            net->graph_seen.push_back(key);
            const int le = launch(stream);
            if (le != 0) return cuda_fail((cudaError_t)le, "kernel launch");
            return EXAGO_OK;
        }
        net->graph_seen.erase(seen);
        if (!net->cap_stream) {
            e = cudaStreamCreateWithFlags(&net->cap_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate (graph capture)");
        }
        e = cudaStreamBeginCapture(net->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        int le = launch(net->cap_stream);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(net->cap_stream, &graph);
        if (le != 0) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail((cudaError_t)le, "kernel launch (capture)");
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        if (net->graphs.size() >= 8) {   // evict the least recently used graph
            size_t lru = 0;
            for (size_t i = 1; i < net->graphs.size(); i++)
                if (net->graphs[i].last_use < net->graphs[lru].last_use) lru = i;
            // no device synchronisation: an executable graph destroyed while a launch of it is
            // still in flight is freed by the runtime once that launch completes
            cudaGraphExecDestroy(net->graphs[lru].exec);
            net->graphs.erase(net->graphs.begin() + lru);
        }
        net->graphs.push_back(GraphEntry{key, exec, 0});
        hit = &net->graphs.back();
    }
    hit->last_use = ++net->graph_clock;
    e = cudaGraphLaunch(hit->exec, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return EXAGO_OK;
}

std::vector<uint64_t> req_key(const EvalReq &R, int schedule) {
    return {(uint64_t)schedule, (uint64_t)R.x, (uint64_t)R.lam, (uint64_t)R.mask, (uint64_t)R.gen_mask,
            (uint64_t)R.pd_scale, (uint64_t)R.obj_weight, (uint64_t)R.f, (uint64_t)R.grad,
            (uint64_t)R.gh, (uint64_t)R.jval, (uint64_t)R.hval, (uint64_t)R.scratch,
            (uint64_t)R.B, bits(R.sigma), (uint64_t)R.stage_recs, (uint64_t)R.stage_cap};
}

// The side stream (highest priority, so bus blocks are dispatched as soon as branch blocks retire)
// and the events of the pipelined schedule, created on first use.  Caller holds net->mu.
exago_status pipe_resources_locked(exago_net *net, PipeLaunch &pl) {
    if (!net->side_stream) {
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        cudaError_t e = cudaStreamCreateWithPriority(&net->side_stream, cudaStreamNonBlocking, hi);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithPriority");
        for (int i = 0; i < 18; i++) {
            e = cudaEventCreateWithFlags(&net->pipe_ev[i], cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate (pipeline)");
        }
    }
    pl.side = net->side_stream;
    pl.ev_fork = net->pipe_ev[16];
    pl.ev_join = net->pipe_ev[17];
    for (int i = 0; i < 8; i++) { pl.ev_br[i] = net->pipe_ev[i]; pl.ev_bu[i] = net->pipe_ev[8 + i]; }
    return EXAGO_OK;
}

exago_status eval_locked(exago_net *net, const exago_batch *bt, double *f, double *grad,
                         double *gh, double *jval, double *hval, ProfileHook *hook,
                         bool allow_graph, const StateTab *tab, const Resolved &rs, void *ws);

// One evaluation call.  With the internal workspace, the call is ordered after the last use of
// that workspace on any other stream (ws_acquire_locked).
exago_status eval(exago_net *net, const exago_batch *bt, double *f, double *grad, double *gh,
                  double *jval, double *hval, ProfileHook *hook = nullptr, bool allow_graph = true,
                  const StateTab *tab = nullptr) {
    exago_status s = check_batch(net, bt, hval != nullptr);
    if (s != EXAGO_OK || bt->B == 0) return s;
    std::lock_guard<std::mutex> lk(net->mu);
    const Resolved rs = resolve(net, bt->B);
    void *ws = bt->workspace;
    const bool needs_ws = gh || jval || hval || rs.schedule == EXAGO_SCHED_PERSISTENT;
    if (ws || !needs_ws) return eval_locked(net, bt, f, grad, gh, jval, hval, hook, allow_graph, tab, rs, ws);
    if ((s = ensure_workspace_locked(net, need_bytes(net, bt->B))) != EXAGO_OK) return s;
    const cudaStream_t st = (cudaStream_t)bt->stream;
    bool capturing = false;
    if ((s = is_capturing(st, &capturing)) != EXAGO_OK) return s;
    if ((s = ws_acquire_locked(net, st, capturing)) != EXAGO_OK) return s;
    s = eval_locked(net, bt, f, grad, gh, jval, hval, hook, allow_graph, tab, rs, net->ws);
    const exago_status r = ws_release_locked(net, st, capturing);
    return s != EXAGO_OK ? s : r;
}

exago_status eval_locked(exago_net *net, const exago_batch *bt, double *f, double *grad,
                         double *gh, double *jval, double *hval, ProfileHook *hook,
                         bool allow_graph, const StateTab *tab, const Resolved &rs, void *ws) {
    exago_status s = EXAGO_OK;
    EvalReq R{};
    R.B = bt->B;
    R.x = bt->x; R.lam = bt->lambda; R.mask = bt->mask; R.gen_mask = bt->gen_mask;
    R.pd_scale = bt->pd_scale; R.obj_weight = bt->obj_weight; R.sigma = bt->obj_factor;
    R.f = f; R.grad = grad; R.gh = gh; R.jval = jval; R.hval = hval;
    R.stage_recs = rs.stage_recs;
    R.stage_cap = rs.stage_cap;
    R.tab = tab;
    cudaStream_t stream = (cudaStream_t)bt->stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(stream, &cap);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamIsCapturing");
    const bool graph = allow_graph && !tab && rs.use_graph && !hook && cap == cudaStreamCaptureStatusNone;
    if (rs.schedule == EXAGO_SCHED_KERNELS) {
        R.scratch = (double *)ws;
        int e = launch_eval(net->dev, R, stream, hook);
        if (e != 0) return cuda_fail((cudaError_t)e, "evaluation kernel launch");
        return EXAGO_OK;
    }
    if (rs.schedule == EXAGO_SCHED_PIPELINED) {
        R.scratch = (double *)ws;
        PipeLaunch pl{};
        pl.chunk = rs.chunk;
        pl.ring = rs.pipe_ring;
        if ((s = pipe_resources_locked(net, pl)) != EXAGO_OK) return s;
        const DevNet &dn = net->dev;
        if (graph) {
            std::vector<uint64_t> key = req_key(R, EXAGO_SCHED_PIPELINED);
            key.push_back((uint64_t)pl.chunk);
            key.push_back((uint64_t)pl.ring);
            return launch_graph_locked(
                net, key, [&](cudaStream_t cs) { return launch_eval_pipelined(dn, R, pl, cs); }, stream);
        }
        int e = launch_eval_pipelined(dn, R, pl, stream, hook);
        if (e != 0) return cuda_fail((cudaError_t)e, "pipelined launch");
        return EXAGO_OK;
    }
    char *w = (char *)ws;
    R.scratch = (double *)w;
    w += persist_ring_bytes(net, rs);
    PersistLaunch pl;
    pl.block = rs.block; pl.occ_warps = rs.occ_warps; pl.grid = rs.grid; pl.lag = rs.lag;
    pl.ring = rs.ring;
    pl.group = rs.group;
    pl.spin_limit = rs.spin_limit; pl.force_timeout = rs.force_timeout;
    pl.counters = (int *)w;
    pl.sm_count = net->sm_count;
    if (graph) {
        std::vector<uint64_t> key = req_key(R, EXAGO_SCHED_PERSISTENT);
        for (uint64_t v : {(uint64_t)pl.counters, (uint64_t)pl.block, (uint64_t)pl.grid,
                           (uint64_t)pl.lag, (uint64_t)pl.ring, (uint64_t)pl.spin_limit,
                           (uint64_t)pl.occ_warps, (uint64_t)pl.force_timeout, (uint64_t)pl.group,
                           (uint64_t)rs.warp_tiles})
            key.push_back(v);
        const DevNet &dn = net->dev;
        if (rs.warp_tiles)
            return launch_graph_locked(
                net, key, [&](cudaStream_t cs) { return launch_eval_persistent_w(dn, R, pl, cs); }, stream);
        return launch_graph_locked(
            net, key, [&](cudaStream_t cs) { return launch_eval_persistent(dn, R, pl, cs); }, stream);
    }
    int e = rs.warp_tiles ? launch_eval_persistent_w(net->dev, R, pl, stream, hook)
                          : launch_eval_persistent(net->dev, R, pl, stream, hook);
    if (e != 0) return cuda_fail((cudaError_t)e, "persistent kernel launch");
    return EXAGO_OK;
}

}  // namespace

namespace exago {

bool net_plan_view(exago_net_t net, const HostPlan **plan) {
    if (!net) return false;
    *plan = &net->plan;
    return true;
}

bool net_internal_view(exago_net_t net, const HostPlan **plan, const DevNet **dev, int *device) {
    if (!net || !net->on_device) return false;
    *plan = &net->plan;
    *dev = &net->dev;
    *device = net->device;
    return true;
}

exago_status set_last_error(exago_status s, const std::string &msg) { return fail(s, msg); }

int multi_kernel_stage_cap(exago_net_t net) {
    std::lock_guard<std::mutex> lk(net->mu);
    return stage_cap(net, false, 128, 16, false);
}

exago_status with_net_workspace(exago_net_t net, void *caller_ws, size_t bytes, cudaStream_t st,
                                bool pipeline,
                                const std::function<exago_status(void *, const PipeLaunch *)> &fn) {
    std::lock_guard<std::mutex> lk(net->mu);
    PipeLaunch pl{};
    exago_status s = EXAGO_OK;
    if (pipeline && (s = pipe_resources_locked(net, pl)) != EXAGO_OK) return s;
    const PipeLaunch *plp = pipeline ? &pl : nullptr;
    if (caller_ws || bytes == 0) return fn(caller_ws, plp);
    if ((s = ensure_workspace_locked(net, bytes)) != EXAGO_OK) return s;
    bool capturing = false;
    if ((s = is_capturing(st, &capturing)) != EXAGO_OK) return s;
    if ((s = ws_acquire_locked(net, st, capturing)) != EXAGO_OK) return s;
    s = fn(net->ws, plp);
    const exago_status r = ws_release_locked(net, st, capturing);
    return s != EXAGO_OK ? s : r;
}

exago_config net_config(exago_net_t net) {
    std::lock_guard<std::mutex> lk(net->mu);
    return net->cfg;
}

exago_status net_graph_launch_locked(exago_net_t net, const std::vector<uint64_t> &key,
                                     const std::function<int(cudaStream_t)> &launch,
                                     cudaStream_t stream) {
    return launch_graph_locked(net, key, launch, stream);
}

exago_status eval_direct(exago_net_t net, const exago_batch *bt, double *f, double *grad,
                         double *gh, double *jval, double *hval, const StateTab *tab) {
    return eval(net, bt, f, grad, gh, jval, hval, nullptr, false, tab);
}

}  // namespace exago

extern "C" {

const char *exago_last_error(void) { return g_err.c_str(); }

void exago_test_fail_allocations(int n) { g_fail_allocs.store(n > 0 ? n : 0); }

const char *exago_status_name(exago_status s) {
    switch (s) {
        case EXAGO_OK: return "EXAGO_OK";
        case EXAGO_EINVAL: return "EXAGO_EINVAL";
        case EXAGO_ENOMEM: return "EXAGO_ENOMEM";
        case EXAGO_ECUDA: return "EXAGO_ECUDA";
        case EXAGO_ETIMEOUT: return "EXAGO_ETIMEOUT";
        case EXAGO_EBUSY: return "EXAGO_EBUSY";
        case EXAGO_ESTATE: return "EXAGO_ESTATE";
        case EXAGO_EDEVICE: return "EXAGO_EDEVICE";
    }
    return "EXAGO_UNKNOWN";
}

exago_status exago_net_plan(int nb, const double *Gs, const double *Bs, const double *Pd,
                            const double *Qd, int nl, const int *f, const int *t,
                            const double *r, const double *x, const double *b,
                            const double *tap, const double *rateA, int ng, const int *gbus,
                            const double *c2, const double *c1, const double *c0,
                            double baseMVA, exago_net_t *out) {
    return plan_only(nb, Gs, Bs, Pd, Qd, nl, f, t, r, x, b, tap, rateA, ng, gbus, c2, c1, c0,
                     baseMVA, nullptr, out);
}

exago_status exago_net_create(int nb, const double *Gs, const double *Bs, const double *Pd,
                              const double *Qd, int nl, const int *f, const int *t,
                              const double *r, const double *x, const double *b,
                              const double *tap, const double *rateA, int ng, const int *gbus,
                              const double *c2, const double *c1, const double *c0,
                              double baseMVA, exago_net_t *out) {
    return exago_net_create_shift(nb, Gs, Bs, Pd, Qd, nl, f, t, r, x, b, tap, nullptr, rateA, ng,
                                  gbus, c2, c1, c0, baseMVA, out);
}

exago_status exago_net_create_shift(int nb, const double *Gs, const double *Bs, const double *Pd,
                                    const double *Qd, int nl, const int *f, const int *t,
                                    const double *r, const double *x, const double *b,
                                    const double *tap, const double *shift,
                                    const double *rateA, int ng, const int *gbus,
                                    const double *c2, const double *c1, const double *c0,
                                    double baseMVA, exago_net_t *out) {
    Range range("exago_net_create");
    exago_status s = plan_only(nb, Gs, Bs, Pd, Qd, nl, f, t, r, x, b, tap, rateA, ng, gbus, c2,
                               c1, c0, baseMVA, shift, out);
    if (s != EXAGO_OK) return s;
    s = do_upload(*out);
    if (s != EXAGO_OK) {
        std::string keep = g_err;
        free_device(*out);
        delete *out;
        *out = nullptr;
        g_err = keep;
    }
    return s;
}

exago_status exago_net_destroy(exago_net_t net) {
    if (!net) return EXAGO_OK;
    free_device(net);
    delete net;
    return EXAGO_OK;
}

exago_status exago_net_dims(exago_net_t net, int *n, int *m_eq, int *m_ineq, int64_t *nnzJ,
                            int64_t *nnzH) {
    if (!net) return fail(EXAGO_EINVAL, "net is NULL");
    if (n) *n = net->plan.n;
    if (m_eq) *m_eq = 2 * net->plan.nb;
    if (m_ineq) *m_ineq = 2 * net->plan.nl;
    if (nnzJ) *nnzJ = net->plan.nnzJ;
    if (nnzH) *nnzH = net->plan.nnzH;
    return EXAGO_OK;
}

exago_status exago_net_jac_pattern(exago_net_t net, int64_t *rowptr, int *col) {
    if (!net || !rowptr || (!col && net->plan.nnzJ > 0)) return fail(EXAGO_EINVAL, "null argument");
    std::memcpy(rowptr, net->plan.Jrowptr.data(), net->plan.Jrowptr.size() * sizeof(int64_t));
    if (net->plan.nnzJ) std::memcpy(col, net->plan.Jcol.data(), net->plan.Jcol.size() * sizeof(int));
    return EXAGO_OK;
}

exago_status exago_net_hess_pattern(exago_net_t net, int64_t *rowptr, int *col) {
    if (!net || !rowptr || (!col && net->plan.nnzH > 0)) return fail(EXAGO_EINVAL, "null argument");
    std::memcpy(rowptr, net->plan.Hrowptr.data(), net->plan.Hrowptr.size() * sizeof(int64_t));
    if (net->plan.nnzH) std::memcpy(col, net->plan.Hcol.data(), net->plan.Hcol.size() * sizeof(int));
    return EXAGO_OK;
}

exago_status exago_net_ineq_bounds(exago_net_t net, double *hlo, double *hhi) {
    if (!net || (net->plan.nl > 0 && (!hlo || !hhi))) return fail(EXAGO_EINVAL, "null argument");
    const int nl = net->plan.nl;
    for (int l = 0; l < nl; l++) {
        double ra = net->plan.rateA[l];
        double hi = ra == 0.0 ? HUGE_VAL : ra * ra;
        hlo[l] = hlo[nl + l] = 0.0;
        hhi[l] = hhi[nl + l] = hi;
    }
    return EXAGO_OK;
}

exago_status exago_net_plan_array(exago_net_t net, const char *name, void *dst, size_t bytes,
                                  size_t *needed) {
    if (!net || !name) return fail(EXAGO_EINVAL, "null argument");
    const HostPlan &p = net->plan;
    const void *src = nullptr;
    size_t n = 0;
#define ARR(key, vec) if (!std::strcmp(name, key)) { src = p.vec.data(); n = p.vec.size() * sizeof(p.vec[0]); }
    ARR("slot_ptr", slot_ptr) else ARR("slot_nbr", slot_nbr) else ARR("slot_ref", slot_ref)
    else ARR("br_slot", br_slot) else ARR("slot_bus", slot_bus) else ARR("slot_pos", slot_pos)
    else ARR("bus_jP", bus_jP) else ARR("bus_jQ", bus_jQ) else ARR("bus_hA", bus_hA)
    else ARR("bus_hM", bus_hM) else ARR("bus_k", bus_k) else ARR("bus_nlow", bus_nlow)
    else ARR("bus_perm", bus_perm)
    else ARR("gen_ptr", gen_ptr) else ARR("gen_ord", gen_ord)
    else return fail(EXAGO_EINVAL, std::string("unknown plan array ") + name);
#undef ARR
    if (needed) *needed = n;
    if (dst) {
        if (bytes < n) return fail(EXAGO_EINVAL, "destination too small");
        if (n) std::memcpy(dst, src, n);
    }
    return EXAGO_OK;
}

exago_status exago_eval_workspace_size(exago_net_t net, int B, size_t *bytes) {
    if (!net || !bytes || B < 0) return fail(EXAGO_EINVAL, "bad argument");
    std::lock_guard<std::mutex> lk(net->mu);
    *bytes = need_bytes(net, B);
    return EXAGO_OK;
}

exago_status exago_net_reserve(exago_net_t net, int B) {
    if (!net || B < 0) return fail(EXAGO_EINVAL, "bad argument");
    if (!net->on_device) return fail(EXAGO_ESTATE, "net was planned without a device");
    return ensure_workspace(net, B);
}

exago_status exago_eval_obj(exago_net_t net, const exago_batch *bt, double *f) {
    Range range("exago_eval_obj");
    if (!f) return fail(EXAGO_EINVAL, "f is NULL");
    return eval(net, bt, f, nullptr, nullptr, nullptr, nullptr);
}

exago_status exago_eval_grad(exago_net_t net, const exago_batch *bt, double *grad) {
    Range range("exago_eval_grad");
    if (!grad) return fail(EXAGO_EINVAL, "grad is NULL");
    return eval(net, bt, nullptr, grad, nullptr, nullptr, nullptr);
}

exago_status exago_eval_cons(exago_net_t net, const exago_batch *bt, double *gh) {
    Range range("exago_eval_cons");
    if (!gh) return fail(EXAGO_EINVAL, "gh is NULL");
    return eval(net, bt, nullptr, nullptr, gh, nullptr, nullptr);
}

exago_status exago_eval_jac(exago_net_t net, const exago_batch *bt, double *jval) {
    Range range("exago_eval_jac");
    if (!jval) return fail(EXAGO_EINVAL, "jval is NULL");
    return eval(net, bt, nullptr, nullptr, nullptr, jval, nullptr);
}

exago_status exago_eval_hess(exago_net_t net, const exago_batch *bt, double *hval) {
    Range range("exago_eval_hess");
    if (!hval) return fail(EXAGO_EINVAL, "hval is NULL");
    return eval(net, bt, nullptr, nullptr, nullptr, nullptr, hval);
}

exago_status exago_eval_all(exago_net_t net, const exago_batch *bt, double *f, double *grad,
                            double *gh, double *jval, double *hval) {
    Range range("exago_eval_all");
    return eval(net, bt, f, grad, gh, jval, hval);
}

// Phase spans reported by exago_eval_profile for the persistent kernel, from the global-timer
// events of persist_kernel.cuh (PhaseSlot; the slot numbers are repeated here because that header
// is device code): from the earliest or latest time of event `from` to the earliest or latest
// time of event `to`.
constexpr int PHASE_N = 8;
struct PhaseSpan {
    const char *name;
    int from;
    bool from_latest;
    int to;
    bool to_latest;
};
constexpr PhaseSpan kPhaseSpan[] = {
    {"phase: first CTA entry to last CTA exit", 0, false, 7, true},
    {"phase: first CTA entry to first branch item start", 0, false, 1, false},
    {"phase: first to last branch item (start to end)", 1, false, 2, true},
    {"phase: last branch item end to first bus item start", 2, true, 3, false},
    {"phase: first to last bus item (start to end)", 3, false, 4, true},
    {"phase: objective (first start to last end)", 5, false, 6, true},
    {"phase: last bus item end to last CTA exit", 4, true, 7, true},
};
constexpr int kPhaseSpans = (int)(sizeof(kPhaseSpan) / sizeof(kPhaseSpan[0]));

exago_status exago_eval_profile(exago_net_t net, const exago_batch *bt, double *f, double *grad,
                                double *gh, double *jval, double *hval, int reps, int *nkernels,
                                const char **names, double *ms) {
    if (reps < 1 || !nkernels || !names || !ms) return fail(EXAGO_EINVAL, "bad profile arguments");
    exago_status s = check_batch(net, bt, hval != nullptr);
    if (s != EXAGO_OK) return s;
    *nkernels = 0;
    if (bt->B == 0) return EXAGO_OK;
    ProfileHook hk;
    for (int i = 0; i < ProfileHook::MAX; i++) {
        cudaError_t e = cudaEventCreate(&hk.ev[i]);
        if (e != cudaSuccess) {
            for (int j = 0; j < i; j++) cudaEventDestroy(hk.ev[j]);
            return cuda_fail(e, "cudaEventCreate");
        }
    }
    // the persistent kernel's phase timestamps: earliest (first 8) and latest (last 8) ns
    cudaError_t ea = dev_malloc((void **)&hk.phase, 2 * PHASE_N * sizeof(unsigned long long));
    if (ea != cudaSuccess) {
        for (int i = 0; i < ProfileHook::MAX; i++) cudaEventDestroy(hk.ev[i]);
        return cuda_fail(ea, "cudaMalloc (profile phases)");
    }
    const cudaStream_t st = (cudaStream_t)bt->stream;
    double acc[ProfileHook::MAX] = {0}, ph[kPhaseSpans] = {0};
    bool seen[kPhaseSpans];
    for (bool &v : seen) v = true;
    int nk = 0;
    bool phases = false;
    // reps evaluations timed by events with the phase marks off, then (for the persistent
    // schedule) reps more with them on, whose event times are not used
    unsigned long long *phase_buf = hk.phase;
    for (int r = 0; r < 2 * reps && s == EXAGO_OK; r++) {
        const bool timed = r < reps;
        if (!timed && !phases) break;
        hk.n = 0;
        hk.phase = timed ? nullptr : phase_buf;
        cudaError_t e = cudaMemsetAsync(phase_buf, 0xFF, PHASE_N * sizeof(unsigned long long), st);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(phase_buf + PHASE_N, 0, PHASE_N * sizeof(unsigned long long), st);
        if (e != cudaSuccess) { s = cuda_fail(e, "cudaMemsetAsync (profile phases)"); break; }
        s = eval(net, bt, f, grad, gh, jval, hval, &hk);
        if (s != EXAGO_OK) break;
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { s = cuda_fail(e, "cudaStreamSynchronize (profile)"); break; }
        if (timed) {
            nk = hk.n - 1;
            for (int k = 0; k < nk; k++) {
                float t = 0.f;
                cudaEventElapsedTime(&t, hk.ev[k], hk.ev[k + 1]);
                acc[k] += t;
                names[k] = hk.name[k];
            }
            phases = nk == 1 && std::strcmp(hk.name[0], "persistent") == 0;
        } else {
            unsigned long long T[2 * PHASE_N];
            e = cudaMemcpy(T, phase_buf, sizeof T, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) { s = cuda_fail(e, "cudaMemcpy (profile phases)"); break; }
            for (int k = 0; k < kPhaseSpans; k++) {
                const PhaseSpan &q = kPhaseSpan[k];
                const unsigned long long a = T[(q.from_latest ? PHASE_N : 0) + q.from];
                const unsigned long long b = T[(q.to_latest ? PHASE_N : 0) + q.to];
                // an event that never happened (no objective wanted) keeps its initial value
                if (T[q.from] == ~0ull || T[q.to] == ~0ull) seen[k] = false;
                ph[k] += ((double)b - (double)a) * 1e-6;   // ns -> ms (may be negative: overlap)
            }
        }
    }
    cudaFree(phase_buf);
    for (int i = 0; i < ProfileHook::MAX; i++) cudaEventDestroy(hk.ev[i]);
    if (s != EXAGO_OK) return s;
    for (int k = 0; k < nk; k++) ms[k] = acc[k] / reps;
    if (phases)
        for (int k = 0; k < kPhaseSpans && nk < ProfileHook::MAX; k++)
            if (seen[k]) {
                names[nk] = kPhaseSpan[k].name;
                ms[nk++] = ph[k] / reps;
            }
    *nkernels = nk;
    return EXAGO_OK;
}

namespace {

exago_status adjoint(exago_net *net, const exago_batch *bt, const double *v, double *out,
                     int mode) {
    exago_status s = check_batch(net, bt, mode == ADJ_HVP);
    if (s != EXAGO_OK || bt->B == 0) return s;
    if (!v || !out) return fail(EXAGO_EINVAL, "input or output vector is NULL");
    void *ws = bt->workspace;
    std::lock_guard<std::mutex> lk(net->mu);
    const cudaStream_t st = (cudaStream_t)bt->stream;
    bool capturing = false;
    const bool internal = ws == nullptr;
    if (internal) {
        if ((s = ensure_workspace_locked(net, need_bytes(net, bt->B))) != EXAGO_OK) return s;
        ws = net->ws;
        if ((s = is_capturing(st, &capturing)) != EXAGO_OK) return s;
        if ((s = ws_acquire_locked(net, st, capturing)) != EXAGO_OK) return s;
    }
    AdjReq A{};
    A.B = bt->B;
    A.x = bt->x; A.lam = bt->lambda; A.mask = bt->mask; A.gen_mask = bt->gen_mask;
    A.obj_weight = bt->obj_weight;
    A.sigma = bt->obj_factor;
    A.v = v; A.out = out;
    A.scratch = (double *)ws;
    int e = launch_adjoint(net->dev, A, mode, bt->stream);
    const exago_status r = internal ? ws_release_locked(net, st, capturing) : EXAGO_OK;
    if (e != 0) return cuda_fail((cudaError_t)e, "adjoint kernel launch");
    return r;
}

}  // namespace

exago_status exago_eval_jvp(exago_net_t net, const exago_batch *bt, const double *u, double *out) {
    Range range("exago_eval_jvp");
    return adjoint(net, bt, u, out, ADJ_JVP);
}

exago_status exago_eval_jtv(exago_net_t net, const exago_batch *bt, const double *v, double *out) {
    Range range("exago_eval_jtv");
    return adjoint(net, bt, v, out, ADJ_JTV);
}

exago_status exago_eval_hvp(exago_net_t net, const exago_batch *bt, const double *u, double *out) {
    Range range("exago_eval_hvp");
    return adjoint(net, bt, u, out, ADJ_HVP);
}

exago_status exago_net_set_config(exago_net_t net, const exago_config *cfg) {
    if (!net || !cfg) return fail(EXAGO_EINVAL, "null argument");
    if (cfg->schedule < EXAGO_SCHED_AUTO || cfg->schedule > EXAGO_SCHED_PIPELINED)
        return fail(EXAGO_EINVAL, "unknown schedule");
    if (cfg->chunk < 0) return fail(EXAGO_EINVAL, "negative chunk");
    if (cfg->schedule == EXAGO_SCHED_PIPELINED && cfg->ring > 7)
        return fail(EXAGO_EINVAL, "pipelined ring must be at most 7 chunks");
    if (cfg->block != 0 && cfg->block != 32 && cfg->block != 64 && cfg->block != 128 &&
        cfg->block != 256)
        return fail(EXAGO_EINVAL, "block must be 0, 32, 64, 128 or 256");
    if (cfg->occupancy != 0 && cfg->occupancy != 8 && cfg->occupancy != 16 && cfg->occupancy != 24)
        return fail(EXAGO_EINVAL, "occupancy must be 0, 8, 16 or 24");
    if (cfg->stage_records < EXAGO_STAGE_DEFAULT || cfg->stage_records > EXAGO_STAGE_BULK)
        return fail(EXAGO_EINVAL, "unknown stage_records value");
    if (cfg->lag < 0 || cfg->ring < 0 || cfg->spin_limit < 0)
        return fail(EXAGO_EINVAL, "negative lag, ring or spin limit");
    if (cfg->tile_group < 0 || cfg->tile_group > 4)
        return fail(EXAGO_EINVAL, "tile_group must be 0 to 4");
    if (cfg->schedule != EXAGO_SCHED_PIPELINED && cfg->ring > 0 && cfg->lag > 0 && cfg->ring <= cfg->lag)
        return fail(EXAGO_EINVAL, "ring must exceed lag");
    if (cfg->tiling < EXAGO_TILING_DEFAULT || cfg->tiling > EXAGO_TILING_WARP)
        return fail(EXAGO_EINVAL, "unknown tiling");
    if (cfg->tiling == EXAGO_TILING_WARP && cfg->block != 0 && cfg->block != 64 && cfg->block != 128)
        return fail(EXAGO_EINVAL, "warp tiling takes blocks of 64 or 128 threads");
    if (cfg->tiling == EXAGO_TILING_WARP && cfg->occupancy == 24)
        return fail(EXAGO_EINVAL, "warp tiling takes occupancy 0, 8 or 16");
    std::lock_guard<std::mutex> lk(net->mu);
    net->cfg = *cfg;
    return EXAGO_OK;
}

exago_status exago_net_get_config(exago_net_t net, int B, exago_config *cfg) {
    if (!net || !cfg || B < 0) return fail(EXAGO_EINVAL, "bad argument");
    if (!net->on_device) return fail(EXAGO_ESTATE, "net was planned without a device");
    std::lock_guard<std::mutex> lk(net->mu);
    const Resolved r = resolve(net, B > 0 ? B : 1);
    *cfg = net->cfg;
    cfg->schedule = r.schedule;
    cfg->stage_records = r.stage_recs == 2 ? EXAGO_STAGE_BULK
                         : r.stage_recs    ? EXAGO_STAGE_ON
                                           : EXAGO_STAGE_OFF;
    if (r.schedule == EXAGO_SCHED_PERSISTENT) {
        cfg->block = r.block;
        cfg->occupancy = r.occ_warps;
        cfg->lag = r.lag;
        cfg->ring = r.ring;
        cfg->use_graph = r.use_graph;
        cfg->tile_group = r.group;
        cfg->tiling = r.warp_tiles ? EXAGO_TILING_WARP : EXAGO_TILING_THREAD;
    }
    if (r.schedule == EXAGO_SCHED_PIPELINED) {
        cfg->chunk = r.chunk;
        cfg->ring = r.pipe_ring;
        cfg->use_graph = r.use_graph;
    }
    cfg->spin_limit = r.spin_limit;
    return EXAGO_OK;
}

exago_status exago_net_autotune(exago_net_t net, const exago_batch *bt, double *f, double *grad,
                                double *gh, double *jval, double *hval, int reps,
                                exago_config *best) {
    Range range("exago_net_autotune");
    if (reps < 1) return fail(EXAGO_EINVAL, "reps < 1");
    exago_status s = check_batch(net, bt, hval != nullptr);
    if (s != EXAGO_OK) return s;
    if (bt->B == 0) return EXAGO_OK;
    const exago_config saved = net->cfg;
    std::vector<exago_config> cands;
    {
        exago_config k{};
        k.schedule = EXAGO_SCHED_KERNELS;
        cands.push_back(k);
        for (int stage : {EXAGO_STAGE_OFF, EXAGO_STAGE_ON}) {
            exago_config k2 = k;
            k2.stage_records = stage;
            if (stage == EXAGO_STAGE_ON) cands.push_back(k2);
            const Resolved base = resolve(net, bt->B);
            for (int mul : {1, 2, 4}) {   // pipelined: derived chunk / 2, / 1 and x 2
                exago_config c{};
                c.schedule = EXAGO_SCHED_PIPELINED;
                c.stage_records = stage;
                c.use_graph = EXAGO_GRAPH_ON;
                c.chunk = base.chunk * mul / 2 > 0 ? base.chunk * mul / 2 : 1;
                cands.push_back(c);
            }
            for (int block : {32, 64, 128, 256})
                for (int occw : {8, 16, 24})
                    for (int group : {1, 2}) {
                        exago_config c{};
                        c.schedule = EXAGO_SCHED_PERSISTENT;
                        c.block = block;
                        c.occupancy = occw;
                        c.stage_records = stage;
                        c.tile_group = group;
                        c.use_graph = EXAGO_GRAPH_ON;
                        cands.push_back(c);
                    }
        }
        // persistent kernel with bus tiles' records in one bulk copy each
        for (int block : {64, 128})
            for (int occw : {8, 16}) {
                exago_config c{};
                c.schedule = EXAGO_SCHED_PERSISTENT;
                c.block = block;
                c.occupancy = occw;
                c.stage_records = EXAGO_STAGE_BULK;
                c.tile_group = 1;
                c.use_graph = EXAGO_GRAPH_ON;
                cands.push_back(c);
            }
        // warp-tiled persistent kernel: a warp per branch or bus, a lane per state
        for (int block : {64, 128})
            for (int occw : {8, 16})
                for (int group : {1, 2}) {
                    exago_config c{};
                    c.schedule = EXAGO_SCHED_PERSISTENT;
                    c.tiling = EXAGO_TILING_WARP;
                    c.block = block;
                    c.occupancy = occw;
                    c.tile_group = group;
                    c.use_graph = EXAGO_GRAPH_ON;
                    cands.push_back(c);
                }
    }
    cudaStream_t st = (cudaStream_t)bt->stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(EXAGO_ECUDA, "cudaEventCreate");
    float best_ms = 1e30f;
    exago_config best_cfg = cands[0];
    for (auto &c : cands) {
        c.spin_limit = saved.spin_limit;
        {
            std::lock_guard<std::mutex> lk(net->mu);
            net->cfg = c;
        }
        s = eval(net, bt, f, grad, gh, jval, hval);   // warm-up (and graph instantiation)
        if (s != EXAGO_OK) break;
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps && s == EXAGO_OK; r++) s = eval(net, bt, f, grad, gh, jval, hval);
        cudaEventRecord(e1, st);
        if (s != EXAGO_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) { s = fail(EXAGO_ECUDA, "autotune timing"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) { best_ms = ms; best_cfg = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(net->mu);
    net->cfg = saved;
    if (s != EXAGO_OK) return s;
    net->tuned[bt->B] = best_cfg;
    if (best) *best = best_cfg;
    return EXAGO_OK;
}

exago_status exago_net_check(exago_net_t net, void *stream) {
    if (!net) return fail(EXAGO_EINVAL, "net is NULL");
    if (!net->on_device) return fail(EXAGO_ESTATE, "net was planned without a device");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    int v = *(volatile int *)net->status_host;
    if (v != 0) {
        *(volatile int *)net->status_host = 0;
        char msg[128];
        if (v & ST_BOUNDS) {
            snprintf(msg, sizeof msg, "a device-side index check failed (status %d)", v);
            return fail(EXAGO_EDEVICE, msg);
        }
        snprintf(msg, sizeof msg, "a bounded device-side wait gave up (code %d)", v);
        return fail(EXAGO_ETIMEOUT, msg);
    }
    return EXAGO_OK;
}

exago_status exago_test_debug_bounds(exago_net_t net, int slots) {
    if (!net) return fail(EXAGO_EINVAL, "net is NULL");
    std::lock_guard<std::mutex> lk(net->mu);
    const int n = net->plan.nslot;
    net->dev.chk_nslot = slots < 0 ? n : std::min(slots, n);
    return EXAGO_OK;
}

}  // extern "C"
