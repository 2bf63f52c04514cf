// Served graph building with continuous batching (host C++ over the plan API).
//
// Events (requests) arrive at any time.  A dispatcher thread keeps, on each
// of the server's devices, `slots` regular slots and one spill slot; a slot
// is a plan with its own stream and its device memory reserved at creation,
// all of it within the per-device memory budget.  Whenever a slot is free it
// takes the requests that have arrived and not yet started, in arrival order,
// as many as fit its capacity in points, events and edges (a request's edges
// are estimated from the edges per point seen so far until a build has
// counted them exactly), and launches one batched build for them.  Slots run
// concurrently on their streams, so requests that arrive while earlier ones
// are on the GPU are admitted as soon as a slot frees up, and their work
// overlaps on the device.  When several devices have a free slot, the one
// with the fewest points in flight goes first.
//
// Edge overflow is handled per request, not per batch: the build counts every
// row before it fills any, so after a batch whose edges exceed its slot's
// capacity the requests whose edges fit (a prefix of the batch: edges are laid
// out in request order) are complete, and the others go back to the front of
// the queue with their exact edge counts, to a regular slot if they fit one,
// else alone to the spill slot (sized for a whole event of up to k edges per
// point, or for as many edges as the budget leaves).  Only a request whose
// edges exceed even the spill slot fails, with FRNN_ERR_OVERFLOW.
//
// A finished batch is copied back in two steps (row offsets first, then
// exactly the edges of its complete requests); a request's latency is the time
// from its arrival to the moment its rows are on the host.  The dispatcher
// holds the queue's lock only to take requests and to publish results, never
// across CUDA calls or row copies.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "frnn.h"
#include "frnn_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    const float* host = nullptr;  // caller's points (kept valid by the caller until done)
    int64_t n = 0;
    Clock::time_point arrival;
    int64_t edges_known = -1;     // exact edge count once a build has counted it
    bool solo = false;            // runs in a batch of its own (its first batch held a non-finite event)
    // results
    std::vector<int32_t> row_ptr;
    std::vector<int32_t> col;
    int status = FRNN_OK;
    int64_t n_edges = 0;
    double latency_s = 0.0;
    bool done = false;
    bool keep = true;  // keep the rows for frnn_server_wait
};

enum SlotState { kIdle, kBuilding, kCopying };

struct Slot {
    int device = 0;
    int group = 0;                         // index of the slot's device in the server's device list
    bool spill = false;
    int64_t cap_points = 0;
    int cap_events = 0;
    int64_t cap_edges = 0;
    frnn_plan* plan = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_build = nullptr, ev_copy = nullptr;
    float* d_in = nullptr;                 // device input of the batch
    int32_t* h_row_ptr = nullptr;          // pinned
    int32_t* h_edge_off = nullptr;         // pinned
    int32_t* h_col = nullptr;              // pinned
    unsigned* h_status = nullptr;          // pinned: the plan's status word after the batch's build
    SlotState state = kIdle;
    std::vector<Request*> reqs;
    std::vector<int64_t> ev_off;
    frnn_csr csr{};
    int build_status = FRNN_OK;
    int n_ok = 0;                          // leading requests whose rows are complete
    bool retry_solo = false;               // the batch held a non-finite event: rerun each request alone
};

struct Group {
    int device = 0;
    int64_t inflight_points = 0;
};

}  // namespace

struct frnn_server {
    frnn_server_params prm{};
    std::vector<Group> groups;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work;   // new request or shutdown
    std::condition_variable cv_done;   // a request finished
    std::deque<Request*> pending;
    std::unordered_map<uint64_t, Request*> all;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread dispatcher;
    uint64_t reserved_bytes = 0;
    int64_t reg_edges = 0;     // edge capacity of a regular slot
    int64_t spill_edges = 0;   // ... and of a spill slot
    frnn_server_stats stats{};
    // edges per point seen in finished requests (dispatcher thread only)
    double seen_points = 0.0, seen_edges = 0.0;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

void free_slot(Slot& s)
{
    DeviceGuard dg(s.device);
    if (s.plan) frnn_plan_destroy(s.plan);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.ev_build) cudaEventDestroy(s.ev_build);
    if (s.ev_copy) cudaEventDestroy(s.ev_copy);
    if (s.d_in) cudaFree(s.d_in);
    if (s.h_row_ptr) cudaFreeHost(s.h_row_ptr);
    if (s.h_edge_off) cudaFreeHost(s.h_edge_off);
    if (s.h_col) cudaFreeHost(s.h_col);
    if (s.h_status) cudaFreeHost(s.h_status);
    s = Slot{};
}

// Edges a request is expected to produce: exact once counted, else its
// points times the edges per point seen so far (with a margin), at least one.
int64_t edge_estimate(const frnn_server* srv, const Request* r)
{
    if (r->edges_known >= 0) return r->edges_known;
    const double epp = srv->seen_points > 0.0 ? 1.25 * srv->seen_edges / srv->seen_points : 0.0;
    return std::max<int64_t>(1, (int64_t)std::ceil(epp * (double)r->n));
}

// Fill a free slot from the queue (caller holds mu).  A regular slot takes
// queued requests in arrival order while they fit its points, events and
// edges; requests whose edges exceed a regular slot are passed over (they wait
// for a spill slot without blocking the requests behind them).  A spill slot
// takes the first such request, alone.
void take_requests(frnn_server* srv, Slot& s)
{
    if (s.spill) {
        for (auto it = srv->pending.begin(); it != srv->pending.end(); ++it)
            if (edge_estimate(srv, *it) > srv->reg_edges) {
                s.reqs.push_back(*it);
                srv->pending.erase(it);
                return;
            }
        return;
    }
    int64_t pts = 0, edges = 0;
    for (auto it = srv->pending.begin(); it != srv->pending.end() && (int)s.reqs.size() < s.cap_events;) {
        Request* r = *it;
        const int64_t e = edge_estimate(srv, r);
        if (e > s.cap_edges || (r->solo && !s.reqs.empty())) {
            ++it;
            continue;
        }
        if (pts + r->n > s.cap_points || edges + e > s.cap_edges) break;
        pts += r->n;
        edges += e;
        s.reqs.push_back(r);
        it = srv->pending.erase(it);
        if (r->solo) break;
    }
}

// Give queued requests to free slots (caller holds mu): each time, the free
// slot whose device has the fewest points in flight (counting this round's
// assignments), regular slots before spill slots.  Returns the slots that
// received work.
std::vector<Slot*> assign_batches(frnn_server* srv)
{
    std::vector<Slot*> started;
    std::vector<int64_t> load(srv->groups.size());
    for (size_t g = 0; g < load.size(); ++g) load[g] = srv->groups[g].inflight_points;
    std::vector<char> offered(srv->slots.size(), 0);
    while (!srv->pending.empty()) {
        int best = -1;
        for (size_t i = 0; i < srv->slots.size(); ++i) {
            const Slot& c = srv->slots[i];
            if (offered[i] || c.state != kIdle) continue;
            if (best >= 0) {
                const Slot& b = srv->slots[(size_t)best];
                const bool better = (c.spill != b.spill) ? !c.spill : load[(size_t)c.group] < load[(size_t)b.group];
                if (!better) continue;
            }
            best = (int)i;
        }
        if (best < 0) break;
        offered[(size_t)best] = 1;
        Slot& s = srv->slots[(size_t)best];
        take_requests(srv, s);
        if (s.reqs.empty()) continue;
        for (const Request* r : s.reqs) load[(size_t)s.group] += r->n;
        started.push_back(&s);
    }
    return started;
}

// Issue the copies and the build of a batch whose requests are in s.reqs
// (dispatcher thread, no lock held).
void launch_batch(frnn_server* srv, Slot& s)
{
    frnn::NvtxRange nvtx("frnn_server: launch a batch");
    DeviceGuard dg(s.device);
    const int d = srv->prm.d;
    s.ev_off.assign(1, 0);
    int64_t pts = 0;
    for (const Request* r : s.reqs) {
        pts += r->n;
        s.ev_off.push_back(pts);
    }
    for (size_t i = 0; i < s.reqs.size(); ++i) {
        const Request* r = s.reqs[i];
        if (r->n > 0)
            cudaMemcpyAsync(s.d_in + s.ev_off[i] * d, r->host, sizeof(float) * (size_t)(r->n * d),
                            cudaMemcpyHostToDevice, s.stream);
    }
    s.build_status = frnn_build_graph_batched(s.plan, s.d_in, s.ev_off.data(), (int)s.reqs.size(), d,
                                              srv->prm.r, srv->prm.k, s.stream, &s.csr);
    if (s.build_status == FRNN_OK) {
        cudaMemcpyAsync(s.h_row_ptr, s.csr.row_ptr, sizeof(int32_t) * (size_t)(pts + 1), cudaMemcpyDeviceToHost,
                        s.stream);
        cudaMemcpyAsync(s.h_edge_off, s.csr.edge_off, sizeof(int32_t) * (s.reqs.size() + 1),
                        cudaMemcpyDeviceToHost, s.stream);
        // the status word comes back with the offsets: no round trip when the build is done
        if (frnn::enqueue_status_read(s.plan, s.stream, s.h_status) != 0) s.build_status = FRNN_ERR_CUDA;
    }
    cudaEventRecord(s.ev_build, s.stream);
    srv->groups[(size_t)s.group].inflight_points += pts;
    s.state = kBuilding;
}

// The build of slot s is done: read its status bits and row offsets, decide
// which requests are complete, start the copy of their edges (dispatcher
// thread).  A non-finite event leaves the others' rows intact but the status
// word does not say which event it was, so a batch of several requests that
// latched it is rerun one request at a time.
void on_built(frnn_server* srv, Slot& s)
{
    frnn::NvtxRange nvtx("frnn_server: batch built");
    DeviceGuard dg(s.device);
    const int nb = (int)s.reqs.size();
    int st = s.build_status;
    unsigned bits = 0;
    if (st == FRNN_OK) {
        bits = *static_cast<volatile unsigned*>(s.h_status);  // landed: ev_build follows its copy
        if ((bits & frnn::kStTimeout) && frnn::recover_after_timeout(s.plan, s.stream) != FRNN_OK)
            st = FRNN_ERR_CUDA;
    }
    s.n_ok = 0;
    s.retry_solo = false;
    if (st == FRNN_OK) {
        if (bits & frnn::kStTimeout) {
            st = FRNN_ERR_TIMEOUT;
        } else if (bits & frnn::kStNonfinite) {
            if (nb > 1) s.retry_solo = true;
            else st = FRNN_ERR_NONFINITE_INPUT;
        } else {
            // rows are written for every request whose edges end within the
            // slot's capacity (with an overflow, a prefix of the batch)
            while (s.n_ok < nb && (int64_t)s.h_edge_off[s.n_ok + 1] <= s.cap_edges) ++s.n_ok;
            // every complete request's columns come to the host (also for a
            // trace replay, whose requests keep no copy of their own)
            const int64_t e_ok = s.h_edge_off[s.n_ok];
            if (e_ok > 0)
                cudaMemcpyAsync(s.h_col, s.csr.col, sizeof(int32_t) * (size_t)e_ok, cudaMemcpyDeviceToHost,
                                s.stream);
        }
    }
    s.build_status = st;
    cudaEventRecord(s.ev_copy, s.stream);
    s.state = kCopying;
}

// The copies of slot s are done: publish the complete requests, re-queue the
// ones that did not fit (dispatcher thread; takes mu only to publish).
void on_copied(frnn_server* srv, Slot& s)
{
    frnn::NvtxRange nvtx("frnn_server: batch copied");
    const int nb = (int)s.reqs.size();
    std::vector<Request*> requeue;
    const Clock::time_point now = Clock::now();
    for (int i = 0; i < nb; ++i) {
        Request* r = s.reqs[(size_t)i];
        if (s.build_status != FRNN_OK) {
            r->status = s.build_status;
        } else if (s.retry_solo) {
            r->solo = true;
            requeue.push_back(r);
            continue;
        } else if (i < s.n_ok) {
            const int64_t lo = s.ev_off[(size_t)i], hi = s.ev_off[(size_t)i + 1];
            const int32_t e0 = s.h_edge_off[i], e1 = s.h_edge_off[i + 1];
            r->status = FRNN_OK;
            r->n_edges = (int64_t)e1 - e0;
            if (r->keep) {
                r->row_ptr.resize((size_t)(hi - lo + 1));
                for (int64_t p = lo; p <= hi; ++p) r->row_ptr[(size_t)(p - lo)] = s.h_row_ptr[p] - e0;
                r->col.assign(s.h_col + e0, s.h_col + e1);
            }
            srv->seen_points += (double)r->n;
            srv->seen_edges += (double)r->n_edges;
        } else {
            // counted but not written: its exact edge count decides where it runs next
            r->edges_known = (int64_t)s.h_edge_off[i + 1] - s.h_edge_off[i];
            if (r->edges_known > std::max(srv->reg_edges, srv->spill_edges)) {
                r->status = FRNN_ERR_OVERFLOW;
                r->n_edges = r->edges_known;
            } else {
                requeue.push_back(r);
                continue;
            }
        }
        r->latency_s = std::chrono::duration<double>(now - r->arrival).count();
    }
    srv->groups[(size_t)s.group].inflight_points -= s.ev_off.back();
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        for (auto it = requeue.rbegin(); it != requeue.rend(); ++it) srv->pending.push_front(*it);
        for (Request* r : s.reqs)
            if (std::find(requeue.begin(), requeue.end(), r) == requeue.end()) r->done = true;
        srv->stats.batches += 1;
        if (s.spill) srv->stats.spill_batches += 1;
        srv->stats.readmitted += requeue.size();
        srv->stats.requests_done += (uint64_t)(nb - (int)requeue.size());
    }
    srv->cv_done.notify_all();
    s.reqs.clear();
    s.state = kIdle;
}

void dispatcher_loop(frnn_server* srv)
{
    std::unique_lock<std::mutex> lock(srv->mu);
    for (;;) {
        std::vector<Slot*> started = assign_batches(srv);
        srv->stats.max_queue = std::max<uint64_t>(srv->stats.max_queue, srv->pending.size());
        bool busy = !started.empty();
        for (const Slot& s : srv->slots) busy |= (s.state != kIdle);
        if (srv->stop && !busy && srv->pending.empty()) break;
        if (!busy) {
            srv->cv_work.wait(lock, [&] { return srv->stop || !srv->pending.empty(); });
            continue;
        }
        lock.unlock();
        for (Slot* s : started) launch_batch(srv, *s);
        bool progressed = !started.empty();
        for (Slot& s : srv->slots) {
            if (s.state == kIdle) continue;
            DeviceGuard dg(s.device);
            if (s.state == kBuilding && cudaEventQuery(s.ev_build) == cudaSuccess) {
                on_built(srv, s);
                progressed = true;
            }
            if (s.state == kCopying && cudaEventQuery(s.ev_copy) == cudaSuccess) {
                on_copied(srv, s);
                progressed = true;
            }
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
        lock.lock();
    }
}

int normalize(const frnn_server_params* p, std::vector<int>* devices)
{
    if (p->d < 1 || p->d > 64 || !(p->r > 0.f) || !std::isfinite(p->r) || p->k < 1 || p->k > 1024 ||
        p->batch_points < 1 || p->batch_events < 1 || p->slots < 1 || p->slots > 64 || p->edges_per_point < 0 ||
        p->n_devices < 0 || p->n_devices > 64 || (p->n_devices > 0 && !p->devices) ||
        p->batch_points * (int64_t)p->k >= (1ll << 31))
        return FRNN_ERR_INVALID_ARG;
    devices->clear();
    if (p->n_devices == 0) devices->push_back(p->device);
    for (int i = 0; i < p->n_devices; ++i) devices->push_back(p->devices[i]);
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess) {
        cudaGetLastError();
        return FRNN_ERR_CUDA;
    }
    for (int dv : *devices)
        if (dv < 0 || dv >= n_dev) return FRNN_ERR_INVALID_ARG;
    return FRNN_OK;
}

frnn_plan_params slot_plan_params(const frnn_server_params& p, int device, bool spill, int64_t edges)
{
    frnn_plan_params pp{};
    pp.device = device;
    pp.d_max = p.d;
    pp.n_max = p.batch_points;
    pp.events_max = spill ? 1 : p.batch_events;
    pp.k_max_cap = p.k;
    pp.edge_capacity = edges;
    pp.cells_per_point = 0;
    pp.flags = FRNN_USE_GRAPH;
    return pp;
}

uint64_t slot_device_bytes(const frnn_server_params& p, const frnn_plan_params& pp)
{
    uint64_t plan_bytes = 0;
    frnn_plan_bytes(&pp, &plan_bytes);
    return plan_bytes + sizeof(float) * (uint64_t)p.batch_points * (uint64_t)p.d;
}

int create_slot(frnn_server* srv, Slot& s, const frnn_plan_params& pp)
{
    const frnn_server_params& p = srv->prm;
    DeviceGuard dg(s.device);
    int rc = frnn_plan_create(&s.plan, &pp);
    if (rc != FRNN_OK) return rc;
    if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.ev_build, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.ev_copy, cudaEventDisableTiming) != cudaSuccess)
        return FRNN_ERR_CUDA;
    if (cudaMalloc(reinterpret_cast<void**>(&s.d_in), sizeof(float) * (size_t)(p.batch_points * p.d)) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&s.h_row_ptr), sizeof(int32_t) * (size_t)(p.batch_points + 1), 0) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&s.h_edge_off), sizeof(int32_t) * (size_t)(s.cap_events + 1), 0) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&s.h_col), sizeof(int32_t) * (size_t)pp.edge_capacity, 0) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&s.h_status), sizeof(unsigned), 0) != cudaSuccess) {
        cudaGetLastError();
        return FRNN_ERR_OOM;
    }
    // capture the slot's graph now, outside the serving loop
    std::vector<float> zero((size_t)p.d, 0.f);
    if (cudaMemcpy(s.d_in, zero.data(), sizeof(float) * (size_t)p.d, cudaMemcpyHostToDevice) != cudaSuccess)
        return FRNN_ERR_CUDA;
    const int64_t off[2] = {0, 1};
    if (frnn_build_graph_batched(s.plan, s.d_in, off, 1, p.d, p.r, p.k, s.stream, &s.csr) != FRNN_OK ||
        frnn_get_last_status(s.plan, s.stream) != FRNN_OK)
        return FRNN_ERR_CUDA;
    return FRNN_OK;
}

void destroy_all(frnn_server* srv)
{
    for (Slot& s : srv->slots) free_slot(s);
    for (auto& kv : srv->all) delete kv.second;
    delete srv;
}

Request* find_request(frnn_server* srv, uint64_t ticket)
{
    auto it = srv->all.find(ticket);
    return it == srv->all.end() ? nullptr : it->second;
}

}  // namespace

extern "C" {

int frnn_server_create(frnn_server** out, const frnn_server_params* p)
{
    frnn::NvtxRange nvtx("frnn_server_create");
    if (!out || !p) return FRNN_ERR_INVALID_ARG;
    *out = nullptr;
    std::vector<int> devices;
    int rc = normalize(p, &devices);
    if (rc != FRNN_OK) return rc;
    const int64_t epp = p->edges_per_point > 0 ? std::min(p->edges_per_point, p->k) : std::min(32, p->k);
    const int64_t reg_edges = std::max<int64_t>(1, p->batch_points * epp);
    const int64_t full_edges = p->batch_points * (int64_t)p->k;  // an event of batch_points points, k each
    // per device: the regular slots, then the spill slot with the edges the budget leaves
    const uint64_t reg_bytes = slot_device_bytes(*p, slot_plan_params(*p, 0, false, reg_edges));
    const uint64_t spill_fixed = slot_device_bytes(*p, slot_plan_params(*p, 0, true, 1));
    const uint64_t bytes_per_edge = slot_device_bytes(*p, slot_plan_params(*p, 0, true, 2)) - spill_fixed;
    uint64_t need = reg_bytes * (uint64_t)p->slots + spill_fixed + bytes_per_edge * (uint64_t)(reg_edges - 1);
    if (p->mem_budget_bytes > 0 && need > p->mem_budget_bytes) return FRNN_ERR_OOM;
    int64_t spill_edges = full_edges;
    if (p->mem_budget_bytes > 0) {
        const uint64_t left = p->mem_budget_bytes - (reg_bytes * (uint64_t)p->slots + spill_fixed);
        spill_edges = std::min<int64_t>(full_edges, (int64_t)(left / std::max<uint64_t>(bytes_per_edge, 1)));
    }
    spill_edges = std::max(spill_edges, reg_edges);
    frnn_server* srv = new (std::nothrow) frnn_server();
    if (!srv) return FRNN_ERR_OOM;
    srv->prm = *p;
    srv->prm.devices = nullptr;  // copied into groups; the caller's array need not outlive this call
    srv->prm.n_devices = (int)devices.size();
    srv->reg_edges = reg_edges;
    srv->spill_edges = spill_edges;
    for (int dv : devices) {
        Group g;
        g.device = dv;
        srv->groups.push_back(g);
    }
    // the regular slots of every device, then one spill slot per device
    for (size_t gi = 0; gi < devices.size(); ++gi)
        for (int i = 0; i < p->slots; ++i) {
            Slot s;
            s.device = devices[gi];
            s.group = (int)gi;
            s.cap_points = p->batch_points;
            s.cap_events = p->batch_events;
            s.cap_edges = reg_edges;
            srv->slots.push_back(s);
        }
    for (size_t gi = 0; gi < devices.size(); ++gi) {
        Slot s;
        s.device = devices[gi];
        s.group = (int)gi;
        s.spill = true;
        s.cap_points = p->batch_points;
        s.cap_events = 1;
        s.cap_edges = spill_edges;
        srv->slots.push_back(s);
    }
    for (Slot& s : srv->slots) {
        const frnn_plan_params pp = slot_plan_params(*p, s.device, s.spill, s.cap_edges);
        rc = create_slot(srv, s, pp);
        if (rc != FRNN_OK) break;
        srv->reserved_bytes += slot_device_bytes(*p, pp);
    }
    if (rc != FRNN_OK) {
        destroy_all(srv);
        return rc;
    }
    try {
        srv->dispatcher = std::thread(dispatcher_loop, srv);
    } catch (...) {
        destroy_all(srv);
        return FRNN_ERR_OOM;
    }
    *out = srv;
    return FRNN_OK;
}

int frnn_server_reserved_bytes(const frnn_server* srv, uint64_t* bytes)
{
    if (!srv || !bytes) return FRNN_ERR_INVALID_ARG;
    *bytes = srv->reserved_bytes;
    return FRNN_OK;
}

int frnn_server_get_stats(frnn_server* srv, frnn_server_stats* stats)
{
    if (!srv || !stats) return FRNN_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(srv->mu);
    *stats = srv->stats;
    stats->regular_edge_capacity = (uint64_t)srv->reg_edges;
    stats->spill_edge_capacity = (uint64_t)srv->spill_edges;
    return FRNN_OK;
}

int frnn_server_submit(frnn_server* srv, const float* host_emb, int64_t n, uint64_t* ticket)
{
    if (!srv || !ticket || n < 0 || (n > 0 && !host_emb)) return FRNN_ERR_INVALID_ARG;
    if (n > srv->prm.batch_points) return FRNN_ERR_CAPACITY;
    Request* r = new (std::nothrow) Request();
    if (!r) return FRNN_ERR_OOM;
    r->host = host_emb;
    r->n = n;
    r->arrival = Clock::now();
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        r->ticket = srv->next_ticket++;
        srv->all[r->ticket] = r;
        srv->pending.push_back(r);
    }
    srv->cv_work.notify_one();
    *ticket = r->ticket;
    return FRNN_OK;
}

int frnn_server_poll(frnn_server* srv, uint64_t ticket, int* done)
{
    if (!srv || !done) return FRNN_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(srv->mu);
    const Request* r = find_request(srv, ticket);
    if (!r) return FRNN_ERR_INVALID_ARG;
    *done = r->done ? 1 : 0;
    return FRNN_OK;
}

int frnn_server_wait(frnn_server* srv, uint64_t ticket, int32_t* row_ptr, int32_t* col, int64_t col_capacity,
                     int64_t* n_edges, double* latency_s)
{
    if (!srv) return FRNN_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(srv->mu);
    Request* r = find_request(srv, ticket);
    if (!r) return FRNN_ERR_INVALID_ARG;
    srv->cv_done.wait(lock, [&] { return r->done; });
    srv->all.erase(ticket);
    lock.unlock();
    int rc = r->status;
    if (n_edges) *n_edges = r->status == FRNN_OK ? (int64_t)r->col.size() : r->n_edges;
    if (latency_s) *latency_s = r->latency_s;
    if (rc == FRNN_OK) {
        if (row_ptr) std::memcpy(row_ptr, r->row_ptr.data(), sizeof(int32_t) * r->row_ptr.size());
        if ((int64_t)r->col.size() > col_capacity || (!col && !r->col.empty())) rc = FRNN_ERR_OVERFLOW;
        else if (col && !r->col.empty()) std::memcpy(col, r->col.data(), sizeof(int32_t) * r->col.size());
    }
    delete r;
    return rc;
}

int frnn_server_run_trace(frnn_server* srv, const float* host_emb, const int64_t* ev_start, const int64_t* ev_len,
                          const double* arrival_s, int n_events, double* latency_s, int64_t* n_edges, double* wall_s)
{
    frnn::NvtxRange nvtx("frnn_server_run_trace");
    if (!srv || !ev_start || !ev_len || !arrival_s || n_events < 0 || !latency_s) return FRNN_ERR_INVALID_ARG;
    const int d = srv->prm.d;
    for (int i = 0; i < n_events; ++i) {
        if (ev_start[i] < 0 || ev_len[i] < 0 || (ev_len[i] > 0 && !host_emb)) return FRNN_ERR_INVALID_ARG;
        if (ev_len[i] > srv->prm.batch_points) return FRNN_ERR_CAPACITY;
        if (i > 0 && arrival_s[i] < arrival_s[i - 1]) return FRNN_ERR_INVALID_ARG;
    }
    std::vector<Request*> reqs((size_t)n_events, nullptr);
    for (int i = 0; i < n_events; ++i) {
        reqs[(size_t)i] = new (std::nothrow) Request();
        if (!reqs[(size_t)i]) {
            for (Request* r : reqs) delete r;
            return FRNN_ERR_OOM;
        }
        reqs[(size_t)i]->host = host_emb + ev_start[i] * d;
        reqs[(size_t)i]->n = ev_len[i];
        reqs[(size_t)i]->keep = false;
    }
    const Clock::time_point t0 = Clock::now();
    for (int i = 0; i < n_events; ++i) {
        const Clock::time_point due = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival_s[i]));
        std::this_thread::sleep_until(due);
        Request* r = reqs[(size_t)i];
        r->arrival = Clock::now();
        {
            std::lock_guard<std::mutex> lock(srv->mu);
            srv->pending.push_back(r);
        }
        srv->cv_work.notify_one();
    }
    int rc = FRNN_OK;
    {
        std::unique_lock<std::mutex> lock(srv->mu);
        srv->cv_done.wait(lock, [&] {
            for (Request* r : reqs)
                if (!r->done) return false;
            return true;
        });
    }
    if (wall_s) *wall_s = std::chrono::duration<double>(Clock::now() - t0).count();
    for (int i = 0; i < n_events; ++i) {
        latency_s[i] = reqs[(size_t)i]->latency_s;
        if (n_edges) n_edges[i] = reqs[(size_t)i]->n_edges;
        if (reqs[(size_t)i]->status != FRNN_OK && rc == FRNN_OK) rc = reqs[(size_t)i]->status;
        delete reqs[(size_t)i];
    }
    return rc;
}

int frnn_server_destroy(frnn_server* srv)
{
    if (!srv) return FRNN_OK;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    if (srv->dispatcher.joinable()) srv->dispatcher.join();
    destroy_all(srv);
    return FRNN_OK;
}

}  // extern "C"
