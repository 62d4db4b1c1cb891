// Serving: a request loop with continuous batching over resident graphs.
//
// The paper copies a graph to the device once and keeps it there while
// property arrays come and go (Section 4.1, host-device transfer analysis).
// The server takes that to many queries: graphs stay resident, and BC
// requests (a graph and a source multiset) arrive at any time.
//
//   admission  a request enters when its device footprint (the workspace of
//              the batched launch it will run) fits in what is left of the
//              memory budget; otherwise it waits in arrival order.
//   slots      `max_slots` worker threads, each with its own CUDA stream, take
//              the oldest admitted request as soon as they are free; their
//              launches are sized for the whole GPU and overlap on the device
//              as SMs free up.  (Capping each slot's grid to its share of the
//              SMs made every launch slower than its share: 57 against 74
//              GTEPS at 200 requests/s with two slots.)
//   batching   a request the batched form serves takes along every admitted
//              request on the same graph with the same options (up to 1,024
//              sources in all): one persistent launch runs them together, each
//              request's sources regrouped among themselves and laid out in
//              32-lane words of its own.  The kernel keeps one partial BC
//              vector per word; each request's result is the sum of its words'
//              vectors in word order.  Other requests run alone.
// A request's words, the order of their lanes and the order in which its BC
// is added depend only on the request, so its result is bit-identical alone
// or in any mix of other requests.
//
// PageRank requests (the paper's second resident-graph workload, Section
// 3.3) share the queue, the admission budget and the slots; each runs alone
// in one persistent launch on its slot's stream.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace sp {

// Defined in api.cu.
sp_status bc_device_entry(Graph* g, const int32_t* d_src, int32_t nsrc, const sp_bc_opts& o, double* d_bc,
                          sp_bc_stats* stats, cudaStream_t st);
sp_status pagerank_device_entry(Graph* g, double damping, double tol, int32_t max_iter, double* d_pr,
                                PrResult* result, cudaStream_t st);
int default_batch_width(int32_t nsrc);
size_t batched_workspace_bytes(const Graph* g, int width, bool theta_f32);

static int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

enum class ReqKind : int { BC = 0, PAGERANK = 1 };

struct Request {
    sp_request id = 0;
    ReqKind kind = ReqKind::BC;
    Graph* g = nullptr;
    // PageRank requests: parameters and result
    double damping = 0.85, tol = 0.0;
    int32_t max_iter = 0;
    int32_t pr_iterations = 0;
    double pr_change = 0.0;
    std::vector<int32_t> sources;
    sp_bc_opts opts{};
    double* bc_out = nullptr;
    size_t footprint = 0;
    sp_status status = SP_NOT_READY;
    bool admitted = false, taken = false, cancelled = false, finished = false;
    std::string err_text;  // the worker's error description when status is an error
    int64_t t_submit = 0, t_start = 0, t_done = 0;
    sp_bc_stats stats{};
};

constexpr size_t kMergeSources = 1024;  // sources of all requests sharing one launch, at most

struct Server {
    size_t budget = 0, used = 0;
    int slots = 1;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<Graph*> graphs;
    std::unordered_map<sp_request, std::shared_ptr<Request>> reqs;
    std::deque<std::shared_ptr<Request>> waiting;   // not yet admitted, arrival order
    std::deque<std::shared_ptr<Request>> admitted;  // admitted, not yet taken by a slot, arrival order
    std::vector<std::thread> workers;
    bool stopping = false;
    bool live = true;  // batched requests run in live launches (sp_server_set_live)
    sp_request next_id = 1;

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
        if (st != SP_OK) r->err_text = sp_last_error();
        r->finished = true;
        r->t_done = now_ns();
        used -= r->footprint;
        admit_locked();
        cv_done.notify_all();
        cv_work.notify_all();
    }

    // Requests that can share r's launch: same graph, same options, batched.
    static bool compatible(const Request& r, const Request& x) {
        return x.kind == ReqKind::BC && r.kind == ReqKind::BC && x.g == r.g && !x.cancelled &&
               x.sources.size() >= 2 && x.opts.precision == r.opts.precision &&
               x.opts.form == r.opts.form && x.opts.flags == r.opts.flags && x.opts.max_ctas == r.opts.max_ctas &&
               x.opts.batch == r.opts.batch && x.opts.debug_flags == 0 && r.opts.debug_flags == 0;
    }

    // Host function enqueued after a live launch: wakes the slots.
    static void CUDART_CB wake(void* p) {
        Server* s = static_cast<Server*>(p);
        std::lock_guard<std::mutex> g(s->mu);
        s->cv_work.notify_all();
    }

    // Runs a group of compatible batched BC requests as one ordinary launch
    // (bc_requests) and finishes them.  Called and returns with lk unlocked.
    void run_group(const std::vector<std::shared_ptr<Request>>& group, const sp_bc_opts& o, cudaStream_t st,
                   std::unique_lock<std::mutex>& lk) {
        std::vector<RequestPart> parts(group.size());
        for (size_t i = 0; i < group.size(); ++i) {
            parts[i].h_sources = group[i]->sources.data();
            parts[i].nsrc = (int32_t)group[i]->sources.size();
            parts[i].d_out = group[i]->bc_out;
        }
        const sp_status rc = bc_requests(group[0]->g, parts.data(), (int)parts.size(), o, st);
        cudaStreamSynchronize(st);
        lk.lock();
        for (size_t i = 0; i < group.size(); ++i) {
            if (rc == SP_OK) {
                group[i]->stats = parts[i].stats;
                group[i]->stats.shared = (int32_t)group.size();
            }
            finish_locked(group[i], rc);
        }
        lk.unlock();
    }

    void worker(int slot) {
        (void)slot;
        cudaSetDevice(device);
        cudaStream_t st;
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        LiveFeed lf;  // this slot's live feed, reused launch after launch
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            cv_work.wait(lk, [&] { return stopping || !admitted.empty(); });
            if (stopping) break;
            std::shared_ptr<Request> r = admitted.front();
            admitted.pop_front();
            r->taken = true;
            r->t_start = now_ns();
            lk.unlock();
            sp_bc_opts o = r->opts;

            const bool batched = !r->cancelled && r->kind == ReqKind::BC &&
                                 request_is_batched(r->g, (int32_t)r->sources.size(), o, st);
            if (batched) {
                // continuous batching: admitted requests on the same graph join
                // this launch, each in words of its own
                std::vector<std::shared_ptr<Request>> group{r};
                lk.lock();
                size_t total = r->sources.size();
                for (auto it = admitted.begin(); it != admitted.end();) {
                    if (compatible(*r, **it) && total + (*it)->sources.size() <= kMergeSources) {
                        total += (*it)->sources.size();
                        (*it)->taken = true;
                        (*it)->t_start = now_ns();
                        group.push_back(*it);
                        it = admitted.erase(it);
                    } else {
                        ++it;
                    }
                }
                const bool use_live = live;
                lk.unlock();
                // a live launch keeps taking requests between its batches;
                // without a live feed, one ordinary launch
                if (!(o.debug_flags == 0 && use_live && serve_live(group, o, st, lf, lk))) run_group(group, o, st, lk);
                lk.lock();
                continue;
            }

            sp_status rc = SP_OK;
            sp_bc_stats sts{};
            if (!r->cancelled && r->kind == ReqKind::PAGERANK) {
                PrResult pr;
                rc = pagerank_device_entry(r->g, r->damping, r->tol, r->max_iter, r->bc_out, &pr, st);
                if (rc == SP_OK) {
                    r->pr_iterations = pr.iterations;
                    r->pr_change = pr.change;
                    sts.kernel_ms = pr.kernel_ms;
                    sts.launches = pr.launches;
                    sts.traversed_arcs = (int64_t)r->g->nnz * (int64_t)pr.iterations;
                }
            } else if (!r->cancelled) {
                const int cnt = (int)r->sources.size();
                int32_t* d_src = nullptr;
                cudaError_t e = cudaMallocAsync((void**)&d_src, sizeof(int32_t) * cnt, st);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(d_src, r->sources.data(), sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, st);
                if (e != cudaSuccess) rc = cuda_fail(e, "server request sources");
                if (rc == SP_OK) rc = bc_device_entry(r->g, d_src, cnt, o, r->bc_out, &sts, st);
                if (d_src) cudaFreeAsync(d_src, st);
            }
            cudaStreamSynchronize(st);

            lk.lock();
            if (rc == SP_OK && !r->cancelled) {
                r->stats = sts;
                r->stats.shared = 1;
            }
            finish_locked(r, r->cancelled ? SP_ERR_CANCELLED : rc);
        }
        lk.unlock();
        live_close(&lf, st);
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }

    // Runs `group` (compatible BC requests of the batched form, already taken)
    // in one live launch on stream st, admitting further compatible requests
    // between its batches, and finishes each request as soon as its words are
    // done.  Returns false, having changed nothing, when no live feed could be
    // set up (the caller then runs the group as one ordinary launch).  Called
    // and returns with lk unlocked.
    bool serve_live(const std::vector<std::shared_ptr<Request>>& group, const sp_bc_opts& o, cudaStream_t st,
                    LiveFeed& lf, std::unique_lock<std::mutex>& lk) {
        Graph* g = group[0]->g;
        size_t total = 0;
        for (auto& x : group) total += x->sources.size();
        if (live_open(g, o, (int64_t)total, &lf, st) != SP_OK) return false;
        struct Member {
            std::shared_ptr<Request> x;
            int64_t idx;
            bool joined, done;
        };
        std::vector<Member> mem;
        std::vector<std::shared_ptr<Request>> unplaced;
        for (auto& x : group) {
            const int64_t idx = live_append(&lf, x->sources.data(), (int32_t)x->sources.size(), x->bc_out);
            if (idx < 0) unplaced.push_back(x);
            else mem.push_back({x, idx, false, false});
        }
        if (mem.empty()) return false;
        live_publish(&lf);
        const int64_t t_launch = now_ns();
        // enqueued: the loop below polls the requests' done flags; the end of
        // the launch wakes it at once (a host function after the kernel)
        const sp_status run_rc = live_start(&lf, o, st, &Server::wake, this);
        LaunchResult res;
        bool ended = run_rc != SP_OK;
        auto finish_done = [&]() {  // with lk held
            for (auto& m : mem) {
                if (m.done || !live_done(&lf, m.idx)) continue;
                m.done = true;
                const FeedReq& fr = lf.req[m.idx % lf.req_cap];
                sp_bc_stats s{};
                s.traversed_arcs = (int64_t)fr.traversed;
                s.reached = (int64_t)fr.reached;
                s.kernel_ms = 1e-6 * (double)(now_ns() - std::max(t_launch, m.x->t_start));
                s.batch = lf.width;
                s.batches = (int32_t)((fr.nwords + lf.width / 32 - 1) / (lf.width / 32));
                s.form = SP_FORM_BATCHED;
                s.promoted = o.precision == SP_FP32_DELTA && !lf.theta_f32;
                s.sigma_float = lf.sigma_float ? 1 : 0;
                s.launches = 1;
                s.shared = (int32_t)lf.nreq;
                s.joined = m.joined ? 1 : 0;
                m.x->stats = s;
                finish_locked(m.x, SP_OK);
            }
            live_retire(&lf);
        };
        lk.lock();
        while (!ended) {
            finish_done();
            if (__atomic_load_n(&lf.ctl->closed, __ATOMIC_ACQUIRE) == 0) {
                // joins: the oldest admitted requests while they are compatible
                // (no request overtakes an older one on another graph)
                while (!admitted.empty() && compatible(*group[0], *admitted.front())) {
                    auto x = admitted.front();
                    const int64_t idx = live_append(&lf, x->sources.data(), (int32_t)x->sources.size(), x->bc_out);
                    if (idx < 0) break;  // full for now
                    x->taken = true;
                    x->t_start = now_ns();
                    mem.push_back({x, idx, true, false});
                    admitted.pop_front();
                }
                // joiners are published a whole batch of words at a time, so
                // that a join never adds a batch the launch would run part
                // empty; what is still held when the launch ends goes to the next
                if (lf.words - lf.pub_words >= lf.width / 32) live_publish(&lf);
            }
            cv_work.wait_for(lk, std::chrono::microseconds(50));
            ended = live_ended(&lf, &res);
        }
        finish_done();
        std::vector<std::shared_ptr<Request>> left;
        for (auto& m : mem)
            if (!m.done) left.push_back(m.x);
        const bool failed = run_rc != SP_OK || res.err != 0;
        if (!failed) {
            // requests the launch never reached (appended after its last look
            // at the feed) go back to the front of the queue, in order
            for (auto it = unplaced.rbegin(); it != unplaced.rend(); ++it) left.insert(left.begin(), *it);
            for (auto it = left.rbegin(); it != left.rend(); ++it) {
                (*it)->taken = false;
                admitted.push_front(*it);
            }
            if (!left.empty()) cv_work.notify_all();
            lk.unlock();
            return true;
        }
        lk.unlock();
        live_scrub(&lf, st);
        // the launch stopped on an error: the unfinished requests run as one
        // ordinary launch, which reruns with wider representations as needed
        for (auto& x : unplaced) left.push_back(x);
        if (!left.empty()) run_group(left, o, st, lk);
        return true;
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

sp_status sp_server_set_live(sp_server sh, int32_t on) {
    if (!sh) return fail(SP_ERR_INVALID_ARG, "server is NULL");
    Server* s = reinterpret_cast<Server*>(sh);
    std::lock_guard<std::mutex> lk(s->mu);
    s->live = on != 0;
    return SP_OK;
}

sp_status sp_server_add_graph(sp_server sh, sp_graph gh, int32_t* graph_id) {
    if (!sh || !gh || !graph_id) return fail(SP_ERR_INVALID_ARG, "NULL argument");
    Server* s = reinterpret_cast<Server*>(sh);
    {
        // the source keys live launches order requests with, made once per graph
        Graph* g = reinterpret_cast<Graph*>(gh);
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return cuda_fail(cudaGetLastError(), "stream");
        const sp_status rc = graph_host_keys(g, st);
        cudaStreamDestroy(st);
        if (rc != SP_OK) return rc;
    }
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
    if (g->n > 0) {
        // the kernels write bc_out directly: it must be memory this GPU can write
        cudaPointerAttributes at{};
        const bool ok = cudaPointerGetAttributes(&at, bc_out) == cudaSuccess &&
                        (at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == g->device));
        cudaGetLastError();
        if (!ok) return fail(SP_ERR_INVALID_ARG, "bc_out must be device memory of the graph's GPU");
    }
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
    const int width = r->opts.batch > 0 ? r->opts.batch : (nsrc >= 128 ? 256 : default_batch_width(nsrc));
    const bool theta32 = r->opts.precision == SP_FP32_DELTA;
    r->footprint = plain ? (size_t)g->n * 40 + (size_t)g->nnz : batched_workspace_bytes(g, width, theta32);
    r->t_submit = now_ns();
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

sp_status sp_pagerank_submit(sp_server sh, int32_t graph_id, double damping, double tol, int32_t max_iter,
                             double* pr_out, sp_request* req) {
    set_last_error("");
    if (!sh || !req) return fail(SP_ERR_INVALID_ARG, "NULL argument");
    Server* s = reinterpret_cast<Server*>(sh);
    Graph* g = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (graph_id < 0 || graph_id >= (int32_t)s->graphs.size()) return fail(SP_ERR_INVALID_ARG, "graph_id");
        g = s->graphs[graph_id];
    }
    if (!(damping >= 0.0 && damping <= 1.0)) return fail(SP_ERR_INVALID_ARG, "damping must be in [0, 1]");
    if (max_iter < 0) return fail(SP_ERR_INVALID_ARG, "max_iter < 0");
    if (g->n > 0) {
        if (!pr_out) return fail(SP_ERR_INVALID_ARG, "pr_out is NULL");
        cudaPointerAttributes at{};
        const bool ok = cudaPointerGetAttributes(&at, pr_out) == cudaSuccess &&
                        (at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == g->device));
        cudaGetLastError();
        if (!ok) return fail(SP_ERR_INVALID_ARG, "pr_out must be device memory of the graph's GPU");
    }
    auto r = std::make_shared<Request>();
    r->kind = ReqKind::PAGERANK;
    r->g = g;
    r->bc_out = pr_out;
    sp_bc_opts_default(&r->opts);
    r->damping = damping;
    r->tol = tol;
    r->max_iter = max_iter;
    // the launch's own vectors (two rank vectors, rank / out-degree, changes) and the hub plan
    r->footprint = (size_t)g->n * 32 + (size_t)g->knnz() / 64 + 4096;
    r->t_submit = now_ns();
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    s->reqs[r->id] = r;
    if (g->n == 0) {
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

sp_status sp_request_pagerank(sp_server sh, sp_request req, int32_t* iterations, double* change) {
    if (!sh) return fail(SP_ERR_INVALID_ARG, "server is NULL");
    Server* s = reinterpret_cast<Server*>(sh);
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req);
    if (it == s->reqs.end()) return fail(SP_ERR_INVALID_ARG, "unknown request");
    if (it->second->kind != ReqKind::PAGERANK) return fail(SP_ERR_INVALID_ARG, "not a PageRank request");
    if (!it->second->finished) return SP_NOT_READY;
    if (iterations) *iterations = it->second->pr_iterations;
    if (change) *change = it->second->pr_change;
    return it->second->status;
}

sp_status sp_bc_poll(sp_server sh, sp_request req) {
    if (!sh) return fail(SP_ERR_INVALID_ARG, "server is NULL");
    Server* s = reinterpret_cast<Server*>(sh);
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req);
    if (it == s->reqs.end()) return fail(SP_ERR_INVALID_ARG, "unknown request");
    if (!it->second->finished) return SP_NOT_READY;
    if (it->second->status != SP_OK) set_last_error(it->second->err_text);
    return it->second->status;
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
    if (r->status != SP_OK) set_last_error(r->err_text);
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
    delete s;
    return SP_OK;
}

}  // extern "C"
