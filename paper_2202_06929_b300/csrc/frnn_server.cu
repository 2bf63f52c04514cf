// Served graph building with continuous batching (host C++ over the plan API).
//
// Events (requests) arrive at any time.  A dispatcher thread keeps S slots,
// each a plan with its own stream and its own device memory reserved at
// creation within the server's memory budget.  Whenever a slot is free it
// takes the requests that have arrived and not yet started, in arrival order,
// as many as fit the slot (points, events), and launches one batched build
// for them; slots run concurrently on their streams, so requests that arrive
// while earlier ones are on the GPU are admitted as soon as a slot frees up
// and their work overlaps on the device.  A finished batch is copied back in
// two steps (row offsets first, then exactly the edges it produced), and each
// request's latency is the time from its arrival to the moment its rows are
// on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
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

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    const float* host = nullptr;  // caller's points (kept valid by the caller until done)
    int64_t n = 0;
    Clock::time_point arrival;
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
    frnn_plan* plan = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_build = nullptr, ev_copy = nullptr;
    float* d_in = nullptr;                 // device input of the batch
    int32_t* h_row_ptr = nullptr;          // pinned
    int32_t* h_edge_off = nullptr;         // pinned
    int32_t* h_col = nullptr;              // pinned
    SlotState state = kIdle;
    std::vector<Request*> reqs;
    std::vector<int64_t> ev_off;
    frnn_csr csr{};
    int build_status = FRNN_OK;
};

}  // namespace

struct frnn_server {
    frnn_server_params prm{};
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
};

namespace {

void free_slot(Slot& s)
{
    if (s.plan) frnn_plan_destroy(s.plan);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.ev_build) cudaEventDestroy(s.ev_build);
    if (s.ev_copy) cudaEventDestroy(s.ev_copy);
    if (s.d_in) cudaFree(s.d_in);
    if (s.h_row_ptr) cudaFreeHost(s.h_row_ptr);
    if (s.h_edge_off) cudaFreeHost(s.h_edge_off);
    if (s.h_col) cudaFreeHost(s.h_col);
    s = Slot{};
}

void finish_request(frnn_server* srv, Request* r, int status, const Slot* s, int idx)
{
    r->status = status;
    r->latency_s = std::chrono::duration<double>(Clock::now() - r->arrival).count();
    if (status == FRNN_OK && s) r->n_edges = (int64_t)s->h_edge_off[idx + 1] - s->h_edge_off[idx];
    if (status == FRNN_OK && r->keep && s) {
        const int64_t lo = s->ev_off[idx], hi = s->ev_off[idx + 1];
        const int32_t e0 = s->h_edge_off[idx], e1 = s->h_edge_off[idx + 1];
        r->row_ptr.resize((size_t)(hi - lo + 1));
        for (int64_t p = lo; p <= hi; ++p) r->row_ptr[(size_t)(p - lo)] = s->h_row_ptr[p] - e0;
        r->col.assign(s->h_col + e0, s->h_col + e1);
    }
    r->done = true;
    (void)srv;
}

// Launch one batch on a free slot from the pending queue (caller holds mu).
bool start_batch(frnn_server* srv, Slot& s)
{
    if (srv->pending.empty()) return false;
    s.reqs.clear();
    s.ev_off.assign(1, 0);
    int64_t pts = 0;
    while (!srv->pending.empty() && (int)s.reqs.size() < srv->prm.batch_events) {
        Request* r = srv->pending.front();
        if (pts + r->n > srv->prm.batch_points) break;
        srv->pending.pop_front();
        s.reqs.push_back(r);
        pts += r->n;
        s.ev_off.push_back(pts);
    }
    if (s.reqs.empty()) return false;
    const int d = srv->prm.d;
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
    }
    cudaEventRecord(s.ev_build, s.stream);
    s.state = kBuilding;
    return true;
}

void dispatcher_loop(frnn_server* srv)
{
    cudaSetDevice(srv->prm.device);
    std::unique_lock<std::mutex> lock(srv->mu);
    for (;;) {
        bool busy = false;
        for (Slot& s : srv->slots) {
            if (s.state == kBuilding && cudaEventQuery(s.ev_build) == cudaSuccess) {
                int st = s.build_status;
                if (st == FRNN_OK) st = frnn_get_last_status(s.plan, s.stream);
                const int64_t pts = s.ev_off.back();
                const int64_t e = (st == FRNN_OK) ? (int64_t)s.h_row_ptr[pts] : 0;
                if (st == FRNN_OK && e > 0) {
                    cudaMemcpyAsync(s.h_col, s.csr.col, sizeof(int32_t) * (size_t)e, cudaMemcpyDeviceToHost, s.stream);
                }
                s.build_status = st;
                cudaEventRecord(s.ev_copy, s.stream);
                s.state = kCopying;
            }
            if (s.state == kCopying && cudaEventQuery(s.ev_copy) == cudaSuccess) {
                for (size_t i = 0; i < s.reqs.size(); ++i) finish_request(srv, s.reqs[i], s.build_status, &s, (int)i);
                s.reqs.clear();
                s.state = kIdle;
                srv->cv_done.notify_all();
            }
            if (s.state == kIdle) start_batch(srv, s);
            busy |= (s.state != kIdle);
        }
        if (srv->stop && !busy && srv->pending.empty()) break;
        if (busy) {
            // poll the slots' events without holding the lock for long
            lock.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lock.lock();
        } else {
            srv->cv_work.wait(lock, [&] { return srv->stop || !srv->pending.empty(); });
        }
    }
}

uint64_t slot_device_bytes(const frnn_server_params& p, const frnn_plan_params& pp)
{
    uint64_t plan_bytes = 0;
    frnn_plan_bytes(&pp, &plan_bytes);
    return plan_bytes + sizeof(float) * (uint64_t)p.batch_points * (uint64_t)p.d;
}

}  // namespace

extern "C" {

int frnn_server_create(frnn_server** out, const frnn_server_params* p)
{
    if (!out || !p) return FRNN_ERR_INVALID_ARG;
    *out = nullptr;
    if (p->d < 1 || p->d > 64 || !(p->r > 0.f) || p->k < 1 || p->k > 1024 || p->batch_points < 1 ||
        p->batch_events < 1 || p->slots < 1 || p->slots > 64 || p->edges_per_point < 0 ||
        p->batch_points * (int64_t)p->k >= (1ll << 31))
        return FRNN_ERR_INVALID_ARG;
    const int64_t epp = p->edges_per_point > 0 ? std::min(p->edges_per_point, p->k) : std::min(32, p->k);
    frnn_plan_params pp{};
    pp.device = p->device;
    pp.d_max = p->d;
    pp.n_max = p->batch_points;
    pp.events_max = p->batch_events;
    pp.k_max_cap = p->k;
    pp.edge_capacity = p->batch_points * epp;
    pp.cells_per_point = 0;
    pp.flags = FRNN_USE_GRAPH;
    const uint64_t per_slot = slot_device_bytes(*p, pp);
    if (p->mem_budget_bytes > 0 && per_slot * (uint64_t)p->slots > p->mem_budget_bytes) return FRNN_ERR_OOM;
    frnn_server* srv = new (std::nothrow) frnn_server();
    if (!srv) return FRNN_ERR_OOM;
    srv->prm = *p;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(p->device) != cudaSuccess) {
        delete srv;
        return FRNN_ERR_CUDA;
    }
    int rc = FRNN_OK;
    srv->slots.resize((size_t)p->slots);
    for (Slot& s : srv->slots) {
        if (rc != FRNN_OK) break;
        rc = frnn_plan_create(&s.plan, &pp);
        if (rc != FRNN_OK) break;
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.ev_build, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.ev_copy, cudaEventDisableTiming) != cudaSuccess) {
            rc = FRNN_ERR_CUDA;
            break;
        }
        if (cudaMalloc(reinterpret_cast<void**>(&s.d_in), sizeof(float) * (size_t)(p->batch_points * p->d)) != cudaSuccess ||
            cudaHostAlloc(reinterpret_cast<void**>(&s.h_row_ptr), sizeof(int32_t) * (size_t)(p->batch_points + 1), 0) != cudaSuccess ||
            cudaHostAlloc(reinterpret_cast<void**>(&s.h_edge_off), sizeof(int32_t) * (size_t)(p->batch_events + 1), 0) != cudaSuccess ||
            cudaHostAlloc(reinterpret_cast<void**>(&s.h_col), sizeof(int32_t) * (size_t)pp.edge_capacity, 0) != cudaSuccess) {
            cudaGetLastError();
            rc = FRNN_ERR_OOM;
            break;
        }
        srv->reserved_bytes += per_slot;
    }
    if (rc == FRNN_OK) {
        // capture each slot's graph now, outside the serving loop
        for (Slot& s : srv->slots) {
            std::vector<float> zero((size_t)p->d, 0.f);
            cudaMemcpy(s.d_in, zero.data(), sizeof(float) * (size_t)p->d, cudaMemcpyHostToDevice);
            const int64_t off[2] = {0, 1};
            if (frnn_build_graph_batched(s.plan, s.d_in, off, 1, p->d, p->r, p->k, s.stream, &s.csr) != FRNN_OK ||
                frnn_get_last_status(s.plan, s.stream) != FRNN_OK) {
                rc = FRNN_ERR_CUDA;
                break;
            }
        }
    }
    cudaSetDevice(prev);
    if (rc != FRNN_OK) {
        for (Slot& s : srv->slots) free_slot(s);
        delete srv;
        return rc;
    }
    try {
        srv->dispatcher = std::thread(dispatcher_loop, srv);
    } catch (...) {
        for (Slot& s : srv->slots) free_slot(s);
        delete srv;
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

int frnn_server_wait(frnn_server* srv, uint64_t ticket, int32_t* row_ptr, int32_t* col, int64_t col_capacity,
                     int64_t* n_edges, double* latency_s)
{
    if (!srv) return FRNN_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(srv->mu);
    auto it = srv->all.find(ticket);
    if (it == srv->all.end()) return FRNN_ERR_INVALID_ARG;
    Request* r = it->second;
    srv->cv_done.wait(lock, [&] { return r->done; });
    srv->all.erase(it);
    lock.unlock();
    int rc = r->status;
    if (n_edges) *n_edges = (int64_t)r->col.size();
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
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(srv->prm.device);
    for (Slot& s : srv->slots) free_slot(s);
    cudaSetDevice(prev);
    for (auto& kv : srv->all) delete kv.second;
    delete srv;
    return FRNN_OK;
}

}  // extern "C"
