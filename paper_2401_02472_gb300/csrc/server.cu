// Serving: a request loop with continuous batching over resident graphs.
//
// The paper copies a graph to the device once and keeps it there while
// property arrays come and go (Section 4.1, host-device transfer analysis).
// The server takes that to many queries: graphs stay resident, and BC
// requests (a graph and a source multiset) arrive at any time.
//
//   admission  a request enters when its device footprint (its partial-BC
//              buffers plus the workspace of the batches it can run at once)
//              fits in what is left of the memory budget; otherwise it waits
//              in arrival order.
//   batching   an admitted request is cut into source batches fixed by the
//              request alone (its sources in order, `width` at a time).
//   slots      `max_slots` worker threads, each with its own CUDA stream and a
//              persistent grid of 1/max_slots of the GPU, take the next batch
//              of the oldest admitted request as soon as they are free, so a
//              new request starts while older ones are still running and the
//              batches of different requests overlap on the device.
//   completion the last batch of a request adds the request's partial BC
//              vectors in batch order into the caller's output and marks the
//              request done.
// A request's result therefore depends only on the request: alone or in a
// mix of other requests it is bit-identical.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace sp {

// Defined in api.cu.
sp_status bc_device_entry(Graph* g, const int32_t* d_src, int32_t nsrc, const sp_bc_opts& o, double* d_bc,
                          sp_bc_stats* stats, cudaStream_t st);
int default_batch_width(int32_t nsrc);
size_t batched_workspace_bytes(const Graph* g, int width, bool theta_f32);

static int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

__global__ void sum_partials_kernel(const double* __restrict__ part, int nb, int64_t n, double* __restrict__ out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[(int64_t)b * n + v];
        out[v] = s;
    }
}

struct Request {
    sp_request id = 0;
    Graph* g = nullptr;
    std::vector<int32_t> sources;
    sp_bc_opts opts{};
    double* bc_out = nullptr;
    int width = 0;
    int nbatches = 0;
    int next_batch = 0;   // next batch to hand to a slot
    int done_batches = 0;
    size_t footprint = 0;
    double* partials = nullptr;  // [nbatches][n] when nbatches > 1
    sp_status status = SP_NOT_READY;
    bool admitted = false, cancelled = false, finished = false;
    int64_t t_submit = 0, t_start = 0, t_done = 0;
    sp_bc_stats stats{};  // summed over the request's batches
};

struct Server {
    size_t budget = 0, used = 0;
    int slots = 1;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<Graph*> graphs;
    std::unordered_map<sp_request, std::shared_ptr<Request>> reqs;
    std::deque<std::shared_ptr<Request>> waiting;   // not yet admitted, arrival order
    std::deque<std::shared_ptr<Request>> admitted;  // admitted with batches left, arrival order
    std::vector<std::thread> workers;
    bool stopping = false;
    sp_request next_id = 1;
    cudaStream_t aux = nullptr;

    void admit_locked() {
        while (!waiting.empty()) {
            auto& r = waiting.front();
            if (r->cancelled) {
                r->status = SP_ERR_CANCELLED;
                r->finished = true;
                r->t_done = now_ns();
                waiting.pop_front();
                cv_done.notify_all();
                continue;
            }
            if (used + r->footprint > budget && used > 0) break;
            used += r->footprint;
            r->admitted = true;
            admitted.push_back(r);
            waiting.pop_front();
        }
    }

    void finish_locked(const std::shared_ptr<Request>& r, sp_status st) {
        r->status = st;
        r->finished = true;
        r->t_done = now_ns();
        used -= r->footprint;
        admit_locked();
        cv_done.notify_all();
        cv_work.notify_all();
    }

    void worker(int slot) {
        cudaSetDevice(device);
        cudaStream_t st;
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        int sms = device_sm_count(device);
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            cv_work.wait(lk, [&] {
                if (stopping) return true;
                for (auto& r : admitted)
                    if (r->next_batch < r->nbatches) return true;
                return false;
            });
            if (stopping) break;
            std::shared_ptr<Request> r;
            for (auto& x : admitted)
                if (x->next_batch < x->nbatches) { r = x; break; }
            if (!r) continue;
            const int b = r->next_batch++;
            if (r->next_batch == r->nbatches) {
                for (auto it = admitted.begin(); it != admitted.end(); ++it)
                    if (it->get() == r.get()) { admitted.erase(it); break; }
            }
            if (r->t_start == 0) r->t_start = now_ns();
            bool skip = r->cancelled || r->status != SP_NOT_READY;
            lk.unlock();

            sp_status rc = SP_OK;
            sp_bc_stats bst{};
            if (!skip) {
                if (r->partials == nullptr && r->nbatches > 1) rc = SP_ERR_OOM;
                const int lo = b * r->width;
                const int cnt = std::min<int>(r->width, (int)r->sources.size() - lo);
                int32_t* d_src = nullptr;
                if (rc == SP_OK) {
                    cudaError_t e = cudaMallocAsync((void**)&d_src, sizeof(int32_t) * cnt, st);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(d_src, r->sources.data() + lo, sizeof(int32_t) * cnt,
                                            cudaMemcpyHostToDevice, st);
                    if (e != cudaSuccess) rc = cuda_fail(e, "server batch sources");
                }
                if (rc == SP_OK) {
                    sp_bc_opts o = r->opts;
                    o.max_ctas = std::max(1, (sms * 4) / slots);
                    if (o.batch == 0 && o.form != SP_FORM_PLAIN) o.batch = r->width;
                    double* out = r->nbatches > 1 ? r->partials + (size_t)b * r->g->n : r->bc_out;
                    rc = bc_device_entry(r->g, d_src, cnt, o, out, &bst, st);
                }
                if (d_src) cudaFreeAsync(d_src, st);
                cudaStreamSynchronize(st);
            }

            lk.lock();
            if (rc != SP_OK && r->status == SP_NOT_READY) r->status = rc;
            if (rc == SP_OK && !skip) {
                r->stats.traversed_arcs += bst.traversed_arcs;
                r->stats.reached += bst.reached;
                r->stats.entries += bst.entries;
                r->stats.scanned_arcs += bst.scanned_arcs;
                r->stats.dag_arcs += bst.dag_arcs;
                r->stats.kernel_ms += bst.kernel_ms;
                r->stats.max_levels = std::max(r->stats.max_levels, bst.max_levels);
                r->stats.batches += 1;
                r->stats.batch = r->width;
                r->stats.form = bst.form;
                r->stats.promoted |= bst.promoted;
                r->stats.sigma_float |= bst.sigma_float;
                r->stats.launches += bst.launches;
            }
            r->done_batches++;
            if (r->done_batches == r->nbatches) {
                sp_status fin = r->cancelled ? SP_ERR_CANCELLED : r->status;
                if (fin == SP_NOT_READY) fin = SP_OK;
                if (fin == SP_OK && r->nbatches > 1) {
                    lk.unlock();
                    int64_t n = r->g->n;
                    int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
                    if (grid < 1) grid = 1;
                    sum_partials_kernel<<<grid, 256, 0, st>>>(r->partials, r->nbatches, n, r->bc_out);
                    cudaError_t e = cudaGetLastError();
                    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                    if (e != cudaSuccess) fin = cuda_fail(e, "server reduction");
                    lk.lock();
                }
                if (r->partials) {
                    cudaFreeAsync(r->partials, st);
                    r->partials = nullptr;
                }
                finish_locked(r, fin);
            }
        }
        lk.unlock();
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
};

}  // namespace sp

using namespace sp;

extern "C" {

sp_status sp_server_create(size_t hbm_budget_bytes, int32_t max_slots, sp_server* out) {
    set_last_error("");
    if (!out) return fail(SP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (max_slots < 1 || max_slots > 64) return fail(SP_ERR_INVALID_ARG, "max_slots must be in [1, 64]");
    if (hbm_budget_bytes == 0) return fail(SP_ERR_INVALID_ARG, "hbm_budget_bytes is 0");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(SP_ERR_NO_DEVICE, "no CUDA device");
    }
    Server* s = new Server();
    s->budget = hbm_budget_bytes;
    s->slots = max_slots;
    s->device = dev;
    for (int i = 0; i < max_slots; ++i) s->workers.emplace_back([s, i] { s->worker(i); });
    *out = reinterpret_cast<sp_server>(s);
    return SP_OK;
}

sp_status sp_server_add_graph(sp_server sh, sp_graph gh, int32_t* graph_id) {
    if (!sh || !gh || !graph_id) return fail(SP_ERR_INVALID_ARG, "NULL argument");
    Server* s = reinterpret_cast<Server*>(sh);
    std::lock_guard<std::mutex> lk(s->mu);
    s->graphs.push_back(reinterpret_cast<Graph*>(gh));
    *graph_id = (int32_t)s->graphs.size() - 1;
    return SP_OK;
}

sp_status sp_bc_submit(sp_server sh, int32_t graph_id, const int32_t* sources, int32_t nsrc, const sp_bc_opts* opts,
                       double* bc_out, sp_request* req) {
    set_last_error("");
    if (!sh || !req) return fail(SP_ERR_INVALID_ARG, "NULL argument");
    Server* s = reinterpret_cast<Server*>(sh);
    Graph* g = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (graph_id < 0 || graph_id >= (int32_t)s->graphs.size()) return fail(SP_ERR_INVALID_ARG, "graph_id");
        g = s->graphs[graph_id];
    }
    if (nsrc < 0 || (nsrc > 0 && !sources)) return fail(SP_ERR_INVALID_ARG, "sources");
    if (g->n > 0 && !bc_out) return fail(SP_ERR_INVALID_ARG, "bc_out is NULL");
    auto r = std::make_shared<Request>();
    r->g = g;
    r->bc_out = bc_out;
    sp_bc_opts_default(&r->opts);
    if (opts) r->opts = *opts;
    if (r->opts.precision != SP_FP64 && r->opts.precision != SP_FP32_DELTA)
        return fail(SP_ERR_INVALID_ARG, "precision");
    r->sources.resize(nsrc);
    if (nsrc > 0) {
        cudaPointerAttributes at{};
        bool dev = cudaPointerGetAttributes(&at, sources) == cudaSuccess && at.type == cudaMemoryTypeDevice;
        cudaGetLastError();
        if (dev) {
            if (cudaMemcpy(r->sources.data(), sources, sizeof(int32_t) * nsrc, cudaMemcpyDeviceToHost) != cudaSuccess)
                return cuda_fail(cudaGetLastError(), "copying request sources");
        } else {
            std::memcpy(r->sources.data(), sources, sizeof(int32_t) * nsrc);
        }
        for (int32_t i = 0; i < nsrc; ++i)
            if (r->sources[i] < 0 || r->sources[i] >= g->n)
                return fail(SP_ERR_INVALID_ARG, "source " + std::to_string(i) + " out of range");
    }
    const bool plain = r->opts.form == SP_FORM_PLAIN || (r->opts.form == SP_FORM_AUTO && nsrc < 2);
    r->width = plain ? std::max(1, nsrc) : (r->opts.batch > 0 ? r->opts.batch : default_batch_width(nsrc));
    r->nbatches = nsrc == 0 ? 1 : (nsrc + r->width - 1) / r->width;
    const bool theta32 = r->opts.precision == SP_FP32_DELTA;
    size_t ws = plain ? (size_t)g->n * 40 + (size_t)g->nnz : batched_workspace_bytes(g, r->width, theta32);
    r->footprint = (r->nbatches > 1 ? (size_t)r->nbatches * (size_t)g->n * sizeof(double) : 0) +
                   (size_t)std::min(r->nbatches, s->slots) * ws;
    r->t_submit = now_ns();
    if (r->nbatches > 1) {
        cudaError_t e = cudaMalloc((void**)&r->partials, (size_t)r->nbatches * (size_t)g->n * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(SP_ERR_OOM, "partial BC buffers");
        }
    }
    if (nsrc == 0) {
        if (g->n > 0 && cudaMemset(bc_out, 0, sizeof(double) * (size_t)g->n) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "zeroing bc_out");
    }
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    s->reqs[r->id] = r;
    if (nsrc == 0) {
        r->status = SP_OK;
        r->finished = true;
        r->t_start = r->t_done = now_ns();
    } else {
        s->waiting.push_back(r);
        s->admit_locked();
        s->cv_work.notify_all();
    }
    *req = r->id;
    return SP_OK;
}

sp_status sp_bc_poll(sp_server sh, sp_request req) {
    if (!sh) return fail(SP_ERR_INVALID_ARG, "server is NULL");
    Server* s = reinterpret_cast<Server*>(sh);
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req);
    if (it == s->reqs.end()) return fail(SP_ERR_INVALID_ARG, "unknown request");
    return it->second->finished ? it->second->status : SP_NOT_READY;
}

sp_status sp_bc_wait(sp_server sh, sp_request req, int64_t timeout_ns) {
    if (!sh) return fail(SP_ERR_INVALID_ARG, "server is NULL");
    Server* s = reinterpret_cast<Server*>(sh);
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req);
    if (it == s->reqs.end()) return fail(SP_ERR_INVALID_ARG, "unknown request");
    auto r = it->second;
    if (timeout_ns < 0) {
        s->cv_done.wait(lk, [&] { return r->finished; });
    } else if (!s->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), [&] { return r->finished; })) {
        return SP_NOT_READY;
    }
    return r->status;
}

sp_status sp_bc_cancel(sp_server sh, sp_request req) {
    if (!sh) return fail(SP_ERR_INVALID_ARG, "server is NULL");
    Server* s = reinterpret_cast<Server*>(sh);
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req);
    if (it == s->reqs.end()) return fail(SP_ERR_INVALID_ARG, "unknown request");
    auto r = it->second;
    if (r->finished) return r->status;
    r->cancelled = true;
    if (!r->admitted) s->admit_locked();  // drops it from the waiting queue
    s->cv_work.notify_all();
    return SP_OK;
}

sp_status sp_request_times(sp_server sh, sp_request req, int64_t* submit_ns, int64_t* start_ns, int64_t* done_ns) {
    if (!sh) return fail(SP_ERR_INVALID_ARG, "server is NULL");
    Server* s = reinterpret_cast<Server*>(sh);
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req);
    if (it == s->reqs.end()) return fail(SP_ERR_INVALID_ARG, "unknown request");
    if (submit_ns) *submit_ns = it->second->t_submit;
    if (start_ns) *start_ns = it->second->t_start;
    if (done_ns) *done_ns = it->second->t_done;
    return SP_OK;
}

sp_status sp_request_stats(sp_server sh, sp_request req, sp_bc_stats* out) {
    if (!sh || !out) return fail(SP_ERR_INVALID_ARG, "NULL argument");
    Server* s = reinterpret_cast<Server*>(sh);
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req);
    if (it == s->reqs.end()) return fail(SP_ERR_INVALID_ARG, "unknown request");
    *out = it->second->stats;
    return SP_OK;
}

sp_status sp_server_destroy(sp_server sh) {
    if (!sh) return fail(SP_ERR_INVALID_ARG, "server is NULL");
    Server* s = reinterpret_cast<Server*>(sh);
    {
        // wait for everything submitted to finish
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_done.wait(lk, [&] {
            for (auto& kv : s->reqs)
                if (!kv.second->finished) return false;
            return true;
        });
        s->stopping = true;
        s->cv_work.notify_all();
    }
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->reqs)
        if (kv.second->partials) cudaFree(kv.second->partials);
    delete s;
    return SP_OK;
}

}  // extern "C"
