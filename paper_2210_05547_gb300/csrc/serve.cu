// Serving: continuous batching of independent solves on one GPU (hyp_server_*).
//
// One worker thread owns a stream and a batch (batch.cu). Submissions go into a FIFO queue from
// any host thread. Between batch steps the worker admits queued requests while the device's free
// memory stays above the reserve after the request's footprint, advances the batch by as many
// steps as the nearest completion allows, and retires finished members. States stay resident on
// the device from admission to retirement; new requests join a running batch at a step boundary.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

constexpr int MAX_CHUNK = 8;   // steps between admission / retirement checks

// Device bytes of one admitted request per cell: the grid's scratch pool (about 216 doubles per
// cell for five species: centre, face and corner fields and six state-sized vectors), the
// line-sweep storage of its largest phase (about 54 doubles per cell), the two RK registers (16
// doubles) and the mask, rounded up; each further species adds about 29 doubles (nine centre
// fields, two artificial-diffusivity fields, six on each face family, six state-sized vectors);
// plus a fixed allowance for tables and plans.
constexpr long long BYTES_PER_CELL = 2400 + 240 * (NSP - 5);
constexpr long long BYTES_FIXED = 4LL << 20;

struct Request {
    hyp_request desc;
    std::vector<double> noise;
    hyp_request_stats stats;
    int remaining = 0;
    hyp_gas* gas = nullptr;
    hyp_state* st = nullptr;
    double* U = nullptr;
    double* dQ = nullptr;
    int64_t n = 0;
    std::vector<double> result;
};

double seconds_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

int64_t state_len(const hyp_grid_desc& g) {
    const int64_t nc = (int64_t)g.nx * g.ny;
    return (NSP + 1) * nc + (int64_t)(g.nx + 1) * g.ny + (int64_t)g.nx * (g.ny + 1);
}

}  // namespace

struct hyp_server {
    std::string table;
    int kind = HYP_GAS_CNEQ, precision = HYP_FP64, device = 0, max_members = 1;
    int64_t reserve = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::unique_ptr<Request>> reqs;
    std::deque<int64_t> pending;
    std::vector<int64_t> members;
    bool stop = false;
    std::thread worker;
    hyp_batch* batch = nullptr;
    cudaStream_t stream = nullptr;
    int64_t batch_steps = 0, member_steps = 0;
    double busy_s = 0.0;
    int32_t max_seen = 0;
};

namespace {

void release(Request& r) {
    if (r.st) hyp_state_free(r.st);
    if (r.gas) hyp_gas_free(r.gas);
    cudaFree(r.U);
    cudaFree(r.dQ);
    r.st = nullptr;
    r.gas = nullptr;
    r.U = r.dQ = nullptr;
}

// Build the request's gas, registers and state on the device and add it to the batch.
int admit(hyp_server* sv, Request& r) {
    int rc = hyp_gas_model_load(sv->table.c_str(), sv->kind, &r.desc.fs, &r.gas);
    if (rc) return rc;
    rc = hyp_state_size(r.gas, &r.desc.grid, &r.n);
    if (rc) return rc;
    cudaError_t e = cudaMalloc(&r.U, r.n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&r.dQ, r.n * sizeof(double));
    if (e != cudaSuccess) return hyp::cuda_fail(e, "cudaMalloc(request registers)");
    hyp_case cas = r.desc.cas;
    cas.noise = r.noise.empty() ? nullptr : r.noise.data();
    rc = hyp_state_init(r.gas, &r.desc.grid, &cas, r.U, r.dQ, sv->stream, &r.st);
    if (rc) return rc;
    return hyp_batch_add(sv->batch, r.st, r.desc.dt);
}

// Read the status, keep the result if asked, and free the request's device memory.
void retire(hyp_server* sv, Request& r) {
    uint32_t flags = 0;
    if (hyp_grid_status(hyp_state_grid(r.st), &flags, 1) != HYP_OK) r.stats.error = HYP_ERR_CUDA;
    r.stats.status = flags;
    if (r.desc.keep_result) {
        r.result.resize(r.n);
        if (cudaMemcpy(r.result.data(), r.U, r.n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            r.stats.error = HYP_ERR_CUDA;
    }
    hyp_batch_remove(sv->batch, r.st);
    release(r);
}

void worker_loop(hyp_server* sv) {
    cudaSetDevice(sv->device);
    for (;;) {
        // admission, in arrival order, while memory and member slots allow
        for (;;) {
            int64_t id;
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                if (sv->stop || sv->pending.empty() || (int)sv->members.size() >= sv->max_members) break;
                id = sv->pending.front();
            }
            Request& r = *sv->reqs[id];
            size_t free_b = 0, total_b = 0;
            cudaMemGetInfo(&free_b, &total_b);
            const int64_t need = BYTES_PER_CELL * r.stats.points + BYTES_FIXED;
            if ((int64_t)free_b < need + sv->reserve) {
                bool idle;
                {
                    std::lock_guard<std::mutex> lk(sv->mu);
                    idle = sv->members.empty();
                }
                if (!idle) break;                    // wait for members to retire
                // nothing will ever free memory: the request cannot be served
                std::lock_guard<std::mutex> lk(sv->mu);
                sv->pending.pop_front();
                r.stats.error = HYP_ERR_OOM;
                r.stats.done = 1;
                r.stats.t_finish = seconds_since(sv->t0);
                sv->cv_done.notify_all();
                continue;
            }
            const int rc = admit(sv, r);
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->pending.pop_front();
            r.stats.t_admit = seconds_since(sv->t0);
            r.stats.bytes = need;
            if (rc) {
                if (r.st) hyp_batch_remove(sv->batch, r.st);
                release(r);
                r.stats.error = rc;
                r.stats.done = 1;
                r.stats.t_finish = r.stats.t_admit;
                sv->cv_done.notify_all();
            } else {
                sv->members.push_back(id);
            }
        }
        int k = MAX_CHUNK;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            if (sv->members.empty()) {
                if (sv->stop) break;
                sv->cv_work.wait_for(lk, std::chrono::milliseconds(50));
                continue;
            }
            for (int64_t id : sv->members) k = std::min(k, sv->reqs[id]->remaining);
            sv->max_seen = std::max<int32_t>(sv->max_seen, (int32_t)sv->members.size());
        }
        const auto t_step = std::chrono::steady_clock::now();
        int rc = hyp_batch_step(sv->batch, k, sv->stream);
        if (rc == HYP_OK && cudaStreamSynchronize(sv->stream) != cudaSuccess) rc = HYP_ERR_CUDA;
        const double dt_step = seconds_since(t_step);
        std::vector<int64_t> finished;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->busy_s += dt_step;
            sv->batch_steps += k;
            sv->member_steps += (int64_t)k * sv->members.size();
            for (int64_t id : sv->members) {
                Request& r = *sv->reqs[id];
                r.remaining -= k;
                if (rc) r.stats.error = rc;
                if (r.remaining <= 0 || rc) finished.push_back(id);
            }
        }
        for (int64_t id : finished) retire(sv, *sv->reqs[id]);
        std::lock_guard<std::mutex> lk(sv->mu);
        for (int64_t id : finished) {
            Request& r = *sv->reqs[id];
            r.stats.done = 1;
            r.stats.t_finish = seconds_since(sv->t0);
            sv->members.erase(std::find(sv->members.begin(), sv->members.end(), id));
        }
        if (!finished.empty()) sv->cv_done.notify_all();
    }
}

}  // namespace

extern "C" int hyp_server_create(const char* table, int kind, int precision, int64_t reserve_bytes,
                                 int max_members, hyp_server** out) {
    if (!table || !out || max_members <= 0 || reserve_bytes < 0)
        return hyp::fail(HYP_ERR_ARG, "server needs a table, max_members > 0, reserve >= 0");
    hyp_server* sv = new hyp_server();
    sv->table = table;
    sv->kind = kind;
    sv->precision = precision;
    sv->reserve = reserve_bytes;
    sv->max_members = max_members;
    sv->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&sv->device);
    int rc = hyp_batch_create(precision, &sv->batch);
    if (rc == HYP_OK) rc = hyp_batch_configure(sv->batch, 1, 0);
    if (rc == HYP_OK) {
        const cudaError_t e = cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) rc = hyp::cuda_fail(e, "cudaStreamCreate");
    }
    if (rc) {
        if (sv->batch) hyp_batch_free(sv->batch);
        delete sv;
        return rc;
    }
    sv->worker = std::thread(worker_loop, sv);
    *out = sv;
    return HYP_OK;
}

extern "C" int hyp_server_submit(hyp_server* sv, const hyp_request* req, int64_t* id) {
    if (!sv || !req || !id) return hyp::fail(HYP_ERR_ARG, "null argument");
    const hyp_grid_desc& g = req->grid;
    if (g.nx < 8 || g.ny < 8 || (long long)g.nx * g.ny > (1LL << 28))
        return hyp::fail(HYP_ERR_ARG, "grid needs 8 to 2^28 cells per direction product");
    if (g.nz > 1) return hyp::fail(HYP_ERR_ARG, "the server takes two-dimensional grids");
    if (!(req->dt > 0.0) || req->nsteps <= 0) return hyp::fail(HYP_ERR_ARG, "request needs dt > 0 and nsteps > 0");
    auto r = std::make_unique<Request>();
    r->desc = *req;
    if (req->cas.noise) r->noise.assign(req->cas.noise, req->cas.noise + state_len(g));
    r->desc.cas.noise = nullptr;
    r->remaining = req->nsteps;
    memset(&r->stats, 0, sizeof(r->stats));
    r->stats.t_admit = r->stats.t_finish = -1.0;
    r->stats.points = (int64_t)g.nx * g.ny;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return hyp::fail(HYP_ERR_ARG, "server is stopping");
    r->stats.t_submit = seconds_since(sv->t0);
    *id = (int64_t)sv->reqs.size();
    sv->reqs.push_back(std::move(r));
    sv->pending.push_back(*id);
    sv->cv_work.notify_one();
    return HYP_OK;
}

extern "C" int hyp_server_wait(hyp_server* sv, int64_t id, double timeout_s) {
    if (!sv) return hyp::fail(HYP_ERR_ARG, "null server");
    std::unique_lock<std::mutex> lk(sv->mu);
    if (id >= (int64_t)sv->reqs.size()) return hyp::fail(HYP_ERR_ARG, "unknown request");
    const int64_t upto = (int64_t)sv->reqs.size();
    auto all_done = [&] {
        if (id >= 0) return sv->reqs[id]->stats.done != 0;
        for (int64_t k = 0; k < upto; ++k)
            if (!sv->reqs[k]->stats.done) return false;
        return true;
    };
    const bool ok = sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), all_done);
    return ok ? HYP_OK : hyp::fail(HYP_ERR_ARG, "timed out waiting for requests");
}

extern "C" int hyp_server_stats(hyp_server* sv, int64_t id, hyp_request_stats* out) {
    if (!sv || !out) return hyp::fail(HYP_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (id < 0 || id >= (int64_t)sv->reqs.size()) return hyp::fail(HYP_ERR_ARG, "unknown request");
    *out = sv->reqs[id]->stats;
    return HYP_OK;
}

extern "C" int hyp_server_result(hyp_server* sv, int64_t id, double* U_host) {
    if (!sv || !U_host) return hyp::fail(HYP_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (id < 0 || id >= (int64_t)sv->reqs.size()) return hyp::fail(HYP_ERR_ARG, "unknown request");
    Request& r = *sv->reqs[id];
    if (!r.stats.done || r.result.empty()) return hyp::fail(HYP_ERR_ARG, "no kept result for this request");
    memcpy(U_host, r.result.data(), r.result.size() * sizeof(double));
    std::vector<double>().swap(r.result);
    return HYP_OK;
}

extern "C" int hyp_server_counters(hyp_server* sv, int64_t* batch_steps, int64_t* member_steps,
                                   double* busy_s, int32_t* max_members) {
    if (!sv) return hyp::fail(HYP_ERR_ARG, "null server");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (batch_steps) *batch_steps = sv->batch_steps;
    if (member_steps) *member_steps = sv->member_steps;
    if (busy_s) *busy_s = sv->busy_s;
    if (max_members) *max_members = sv->max_seen;
    return HYP_OK;
}

extern "C" void hyp_server_free(hyp_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        for (int64_t id : sv->pending) {
            Request& r = *sv->reqs[id];
            r.stats.done = 1;
            r.stats.error = HYP_ERR_ARG;
            r.stats.t_finish = seconds_since(sv->t0);
        }
        sv->pending.clear();
        sv->cv_work.notify_all();
    }
    if (sv->worker.joinable()) sv->worker.join();
    hyp_batch_free(sv->batch);
    if (sv->stream) cudaStreamDestroy(sv->stream);
    delete sv;
}
