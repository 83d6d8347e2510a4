// cf_server.cpp -- serving loop with continuous batching.
//
// Requests (auto-correlation catalogues sharing one cf_params) are queued by cf_server_submit.
// Two worker threads, each with its own context and CUDA stream, take turns forming "waves": a
// worker admits every pending request that fits the memory budget and the slot limit left
// over by the wave in flight on the other worker, counts the wave with one batched call
// (one cell build over all its catalogues, one persistent pair kernel over their concatenated
// work list), writes each request's result and frees its share of memory and slots.  Requests
// that arrive while a wave is on the GPU are admitted by the other worker as soon as memory
// and slots allow, so its cell build overlaps the first wave's counting on the device.
//
// Waits are bounded: cf_server_poll takes a timeout, workers wake at least every 50 ms to
// notice a stop request.
//
// Failures: a wave whose batched count fails is counted again one request at a time, so that
// one bad catalogue fails only its own request.  A worker that cannot create its context
// records the error; once no worker is left, every pending and every later request fails with
// CF_ERR_CUDA instead of waiting.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "cf_api_internal.h"

namespace {

struct Request {
    uint64_t ticket = 0;
    cf_points pts;
    cf_result out;
    size_t mem = 0;
    int status = CF_ERR_BUSY;    // CF_ERR_BUSY while queued or running
    bool running = false;
};

struct Server {
    int device = 0;
    cf_params p;
    std::vector<double> edges;
    size_t budget = 0;
    int max_slots = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::map<uint64_t, Request *> all;
    uint64_t next_ticket = 1;
    size_t mem_in_flight = 0;
    int slots_in_flight = 0;
    bool stopping = false;
    int workers_alive = 0;       // workers whose context exists (set before they start)
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    std::string err;
    int fail(int st, const std::string &m)
    {
        err = m;
        return st;
    }
};

// device-memory estimate of one catalogue inside a wave: inputs (when copied), the packed
// layout, cell ids, ranks, original indices, cells and work items
size_t request_bytes(const cf_points &q)
{
    size_t es = q.dtype == CF_F64 ? 8 : 4;
    size_t n = (size_t)q.n;
    return n * (4 * es + 16 + 16 + 4 + 4 + 4 + 32 + 48 / 8) + (1u << 20);
}

void worker_main(Server *S, int wid)
{
    cudaSetDevice(S->device);
    void *ctxv = nullptr;
    if (cf_create(&ctxv, S->device, S->streams[wid]) != CF_OK) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->err = "a server worker could not create its CUDA context";
        if (--S->workers_alive == 0) {
            // nobody is left to serve: fail what waits instead of letting it time out
            for (auto *r : S->pending) r->status = CF_ERR_CUDA;
            S->pending.clear();
        }
        S->cv_done.notify_all();
        return;
    }
    CfCtx *C = (CfCtx *)ctxv;
    for (;;) {
        std::vector<Request *> wave;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            while (!S->stopping && S->pending.empty()) S->cv_work.wait_for(lk, std::chrono::milliseconds(50));
            if (S->stopping) break;
            size_t mem = 0;
            int slots = 0;
            while (!S->pending.empty()) {
                Request *r = S->pending.front();
                bool fits = S->mem_in_flight + mem + r->mem <= S->budget &&
                            S->slots_in_flight + slots + 1 <= S->max_slots;
                if (!fits && !wave.empty()) break;
                if (!fits && (S->mem_in_flight > 0 || S->slots_in_flight > 0)) break;   // wait for memory
                S->pending.pop_front();
                r->running = true;
                wave.push_back(r);
                mem += r->mem;
                slots += 1;
            }
            S->mem_in_flight += mem;
            S->slots_in_flight += slots;
            if (wave.empty()) {
                S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
                continue;
            }
        }
        std::vector<cf_points> cats(wave.size());
        std::vector<cf_result> outs(wave.size());
        for (size_t i = 0; i < wave.size(); i++) {
            cats[i] = wave[i]->pts;
            outs[i] = wave[i]->out;
        }
        int rc = cf_batch_count(C, &S->p, cats.data(), (int)cats.size(), outs.data());
        std::vector<int> st(wave.size(), rc);
        std::string msg = rc ? C->err : std::string();
        if (rc && wave.size() > 1) {
            // find the failing catalogue(s): count each request of the wave alone
            msg.clear();
            for (size_t i = 0; i < wave.size(); i++) {
                st[i] = cf_batch_count(C, &S->p, &cats[i], 1, &outs[i]);
                if (st[i] && msg.empty()) msg = C->err;
            }
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            size_t mem = 0;
            for (size_t i = 0; i < wave.size(); i++) {
                Request *r = wave[i];
                mem += r->mem;
                r->running = false;
                r->status = st[i];
            }
            if (!msg.empty()) S->err = msg;
            S->mem_in_flight -= mem;
            S->slots_in_flight -= (int)wave.size();
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
    cf_destroy(C);
}

}  // namespace

extern "C" {

cf_status cf_server_start(void **server_out, int device, const cf_params *params, size_t mem_budget_bytes,
                          int max_slots)
{
    if (!server_out || !params) return CF_ERR_ARG;
    *server_out = nullptr;
    std::string err;
    if (cfp_check_params(params, err) != CF_OK) return CF_ERR_ARG;
    if (!params->autocorr || max_slots < 1 || mem_budget_bytes == 0) return CF_ERR_ARG;
    Server *S = new Server();
    S->device = device;
    S->p = *params;
    S->edges.assign(params->edges, params->edges + params->nbins + 1);
    S->p.edges = S->edges.data();
    S->budget = mem_budget_bytes;
    S->max_slots = max_slots;
    DeviceGuard g(device);
    for (int w = 0; w < 2; w++) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (auto s : S->streams) cudaStreamDestroy(s);
            delete S;
            return CF_ERR_CUDA;
        }
        S->streams.push_back(st);
    }
    S->workers_alive = 2;
    for (int w = 0; w < 2; w++) S->workers.emplace_back(worker_main, S, w);
    *server_out = S;
    return CF_OK;
}

cf_status cf_server_submit(void *server, const cf_points *cat, cf_result *out, uint64_t *ticket)
{
    if (!server || !cat || !out || !ticket) return CF_ERR_ARG;
    Server *S = (Server *)server;
    if (cat->n < 0 || (cat->dtype != CF_F32 && cat->dtype != CF_F64))
        return (cf_status)S->fail(CF_ERR_ARG, "invalid catalogue");
    Request *r = new Request();
    r->pts = *cat;
    r->out = *out;
    r->mem = request_bytes(*cat);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) {
        delete r;
        return (cf_status)S->fail(CF_ERR_CANCELLED, "server is stopping");
    }
    if (S->workers_alive == 0) {
        delete r;
        return (cf_status)S->fail(CF_ERR_CUDA, "no server worker could create its CUDA context");
    }
    if (r->mem > S->budget) {
        delete r;
        return (cf_status)S->fail(CF_ERR_OOM, "request needs more device memory than the server's budget");
    }
    r->ticket = S->next_ticket++;
    S->all[r->ticket] = r;
    S->pending.push_back(r);
    *ticket = r->ticket;
    S->cv_work.notify_one();
    return CF_OK;
}

cf_status cf_server_poll(void *server, uint64_t ticket, int timeout_ms)
{
    if (!server) return CF_ERR_ARG;
    Server *S = (Server *)server;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return (cf_status)S->fail(CF_ERR_ARG, "unknown ticket");
    Request *r = it->second;
    auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
    while (r->status == CF_ERR_BUSY) {
        if (timeout_ms <= 0) return CF_ERR_BUSY;
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->status == CF_ERR_BUSY)
            return CF_ERR_TIMEOUT;
    }
    int st = r->status;
    S->all.erase(it);
    delete r;
    return (cf_status)st;
}

cf_status cf_server_cancel(void *server, uint64_t ticket)
{
    if (!server) return CF_ERR_ARG;
    Server *S = (Server *)server;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return (cf_status)S->fail(CF_ERR_ARG, "unknown ticket");
    Request *r = it->second;
    // a request in a wave on the GPU cannot be withdrawn: its inputs are still read and its result
    // will be written, so the caller keeps its buffers and polls for it
    if (r->running) return CF_ERR_BUSY;
    if (r->status == CF_ERR_BUSY) {
        auto q = std::find(S->pending.begin(), S->pending.end(), r);
        if (q != S->pending.end()) S->pending.erase(q);
        r->status = CF_ERR_CANCELLED;
    }
    S->cv_done.notify_all();
    return CF_OK;
}

cf_status cf_server_stop(void *server)
{
    if (!server) return CF_ERR_ARG;
    Server *S = (Server *)server;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        for (auto *r : S->pending) r->status = CF_ERR_CANCELLED;
        S->pending.clear();
    }
    S->cv_work.notify_all();
    for (auto &t : S->workers) t.join();
    {
        DeviceGuard g(S->device);
        for (auto s : S->streams) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    }
    for (auto &kv : S->all) delete kv.second;
    delete S;
    return CF_OK;
}

const char *cf_server_last_error(const void *server)
{
    if (!server) return "null server";
    // the workers assign err under the lock: copy it under the lock into this thread's buffer
    static thread_local std::string msg;
    Server *S = (Server *)server;
    std::lock_guard<std::mutex> lk(S->mu);
    msg = S->err;
    return msg.c_str();
}

}  // extern "C"
