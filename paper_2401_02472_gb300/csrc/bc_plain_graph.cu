// Plain form with the level loop driven by a CUDA graph instead of a
// persistent kernel.
//
// The paper's generated CUDA code runs the BFS and the reverse sweep as a host
// loop that launches one kernel per level and copies a `finished` flag back
// after each (Section 3.4, the iterateInBFS listing; Section 4.1 blames this loop and the grid
// synchronisation for the BC times).  Here the loop stays on the device but
// keeps the one-kernel-per-level shape: a graph holds one conditional WHILE
// node whose body is a chain of kUnroll launches of one step kernel.  In each
// launch every block of a full grid works through the current phase (a
// source's init, one forward level or one backward level) with the same
// per-entry code as the persistent form; the last block to finish (counted
// with an atomic, so no block ever waits on another) reads the level-stack
// fill, decides the next phase, prepares its bookkeeping and clears the loop
// condition once every source is done or an error is set.  The kernel
// boundary is the level barrier.  Launches that find the loop finished
// return at once, so a WHILE iteration may end part-way through its chain.
// One source runs at a time over the whole grid (no block groups).
// Results are bit-identical to the persistent form with one group: every
// per-vertex sum has the same order, and BC is added in source order.
//
// The loop cannot run away: the advance kernel counts phases and stops the
// loop with an error past the bound that a correct run never reaches
// (nsrc * (2n + 2) + 2 phases).
#include <algorithm>
#include <climits>
#include <cstring>
#include <string>

#include "bc_plain_kernel.cuh"

namespace sp {

enum StepStage : int { kStageInit = 0, kStageForward = 1, kStageBackward = 2, kStageDone = 3 };

// The loop's state between launches (device memory; one copy per graph).
struct StepState {
    int stage;
    int si;          // source index
    int d;           // current level
    int qb, qe;      // forward: level d's entries are q[qb, qe)
    int L;           // levels of the current source (after its forward pass)
    int hoff_d;      // first hub record of level d (forward)
    int bu;          // forward level d discovers bottom-up
    int levels_max;
    int pad;
    long long steps, step_limit;
};

// Kernel arguments and loop state live in one small device block owned by the
// graph object, so that an instantiated CUDA graph stays valid across calls:
// each call copies its arguments in and launches the cached graph.
struct StepBlock {
    PlainArgs args;
    alignas(16) StepState state;
    unsigned int arrived;  // blocks of the current launch that finished their work
};

constexpr int kUnroll = 4;  // step launches per WHILE iteration

// One thread of the last block: move the loop to its next phase.  Path-count
// and dependency types do not enter here (only the level bookkeeping);
// PlainKernel is instantiated for its index helpers.
static __device__ __noinline__ void step_advance(StepBlock* blk, cudaGraphConditionalHandle cond) {
    const PlainArgs& a = blk->args;
    StepState s = blk->state;
    PlainKernel<unsigned long long, double, false, false> K(a, 0);
    GroupCtl* gc = a.gctl;
    gc->work[0] = 0u;
    s.steps += 1;
    bool more = true;
    if (ld_volatile(&a.ctl->err) != 0 || s.stage == kStageDone) {
        more = false;
    } else if (s.steps > s.step_limit) {
        set_error(a.ctl, kErrCorrupt);
        more = false;
    } else {
        bool next_source = false;
        bool open = false;
        if (s.stage == kStageInit) {
            s.stage = kStageForward;
            s.d = 0;
            s.qb = 0;
            s.qe = 1;
            s.hoff_d = 0;
            open = true;
        } else if (s.stage == kStageForward) {
            const int nq = ld_volatile(&gc->qtail);
            s.hoff_d += (int)(ld_volatile(&K.hcnt()[s.d]) >> 32);
            if (nq == s.qe) {
                s.L = s.d + 1;
                s.levels_max = max(s.levels_max, s.L);
                if (s.L - 1 >= 1) {
                    s.stage = kStageBackward;
                    s.d = s.L - 1;
                } else {
                    next_source = true;
                }
            } else {
                s.qb = s.qe;
                s.qe = nq;
                s.d += 1;
                open = true;
            }
        } else if (s.stage == kStageBackward) {
            s.d -= 1;
            if (s.d < 1) next_source = true;
        }
        if (open) {
            if (s.d + 2 >= a.lcap) {
                set_error(a.ctl, kErrCapLevels);
                more = false;
            } else {
                K.d = s.d;
                K.hoff_d = s.hoff_d;
                K.open_level(s.qe);
                s.bu = a.bu_den > 0 && s.d > 0 && (int64_t)(s.qe - s.qb) * a.bu_den > (int64_t)a.n;
            }
        }
        if (next_source) {
            s.si += 1;
            if (s.si >= a.nsrc) {
                s.stage = kStageDone;
                more = false;
            } else {
                s.stage = kStageInit;
            }
        }
    }
    if (!more) {
        s.stage = kStageDone;
        atomicMax(&a.ctl->max_levels, s.levels_max);
    }
    blk->state = s;
    __threadfence();
    cudaGraphSetConditional(cond, more ? 1u : 0u);
}

// One forward or backward level of the current source, then the block's
// statistics.
template <typename SigT, typename ThT, bool kDir>
static __device__ __forceinline__ void step_work(PlainKernel<SigT, ThT, false, kDir>& K, const StepState& ss, int n) {
    constexpr bool kFloatSig = !std::is_integral<SigT>::value;
    const PlainArgs& sa = K.a;
    const int d = ss.d;
    K.d = d;
    const unsigned long long hc = ld_volatile(&K.hcnt()[d]);
    K.nrec_d = (int)(hc >> 32);
    K.nseg_d = (int)(hc & 0xFFFFFFFFull);
    if (ss.stage == kStageForward) {
        K.hoff_d = ss.hoff_d;
        K.hoff_next = K.hoff_d + K.nrec_d;
        if constexpr (kFloatSig) {
            K.cshift_prev = d > 0 ? K.shift_of(ld_volatile(&K.emax()[d - 1]), ld_volatile(&K.emin()[d - 1])) : 0;
            if (blockIdx.x == 0 && threadIdx.x == 0 && K.cshift_prev != 0) atomicAdd(&sa.ctl->recentred, 1ull);
        }
        K.discover = !ss.bu;
        K.template level_work<true>(0, ss.qb, ss.qe, false, ss.bu ? (n + 8 * kWarp - 1) / (8 * kWarp) : 0);
        if constexpr (kFloatSig) {
            int mx = warp_max_i32(K.my_emax), mn = warp_min_i32(K.my_emin);
            if (K.lane == 0 && mx >= mn) {
                atomicMax(&K.emax()[d], mx);
                atomicMin(&K.emin()[d], mn);
            }
        }
        if (K.ovf) set_error(sa.ctl, kErrSigmaOverflow);
    } else {
        const int qbd = ld_volatile(&K.qoff()[d]);
        const int qed = ld_volatile(&K.qoff()[d + 1]);
        K.hoff_d = ld_volatile(&K.hoff()[d]);
        if constexpr (kFloatSig) K.cshift_cur = K.shift_of(ld_volatile(&K.emax()[d]), ld_volatile(&K.emin()[d]));
        K.template level_work<false>(0, qbd, qed, d == ss.L - 1);
    }
    // statistics: block sums, one atomic per block and counter
    __shared__ unsigned long long s_st[4];
    if (threadIdx.x == 0) { s_st[0] = 0; s_st[1] = 0; s_st[2] = 0; s_st[3] = 0; }
    __syncthreads();
    if (K.st_arcs) atomicAdd(&s_st[0], K.st_arcs);
    if (K.st_reached) atomicAdd(&s_st[1], K.st_reached);
    if (K.st_scanned) atomicAdd(&s_st[2], K.st_scanned);
    if (K.st_dag) atomicAdd(&s_st[3], K.st_dag);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_st[0]) atomicAdd(&sa.ctl->traversed_arcs, s_st[0]);
        if (s_st[1]) atomicAdd(&sa.ctl->reached, s_st[1]);
        if (s_st[2]) atomicAdd(&sa.ctl->scanned_arcs, s_st[2]);
        if (s_st[3]) atomicAdd(&sa.ctl->dag_arcs, s_st[3]);
    }
}

template <typename SigT, typename ThT, bool kDir>
__global__ void __launch_bounds__(kPlainThreads, 2) plain_step_kernel(StepBlock* blk, cudaGraphConditionalHandle cond) {
    __shared__ PlainArgs sa;
    __shared__ StepState ss;
    if (threadIdx.x == 0) {
        sa = blk->args;
        ss = blk->state;
    }
    __syncthreads();
    if (ss.stage == kStageDone) return;  // the loop ended earlier in this iteration's chain
    if (ld_volatile(&sa.ctl->err) != 0) {
        // set before this launch (every launch's last block checks the flag, so
        // this is not expected); end the loop here rather than spin through it
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            blk->state.stage = kStageDone;
            cudaGraphSetConditional(cond, 0u);
        }
        return;
    }
    PlainKernel<SigT, ThT, false, kDir> K(sa, 0);
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = gridDim.x * blockDim.x;
    const int n = sa.n;
    if (ss.stage == kStageInit) {
        const int src = __ldg(&sa.sources[ss.si]);
        for (int i = tid; i < n; i += nthr) K.lv(i) = (i == src) ? 0 : -1;
        if (ss.si == 0)
            for (int i = tid; i < n; i += nthr) sa.bc[i] = 0.0;
        if (tid == 0) K.start_source(src);
    } else {
        step_work(K, ss, n);
    }
    // the last block to finish advances the loop
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&blk->arrived, 1u) == gridDim.x - 1;
        if (s_last) {
            __threadfence();
            blk->arrived = 0u;
            step_advance(blk, cond);
        }
    }
}

// Cached device block and instantiated graphs of one graph object.
struct StepCache {
    std::mutex mu;
    StepBlock* d_blk = nullptr;
    cudaGraphExec_t exec[4] = {};
    int grid[4] = {};
};

void destroy_step_cache(Graph* g) {
    auto* c = reinterpret_cast<StepCache*>(g->step_cache);
    if (!c) return;
    for (auto& e : c->exec)
        if (e) cudaGraphExecDestroy(e);
    if (c->d_blk) cudaFree(c->d_blk);
    delete c;
    g->step_cache = nullptr;
}

template <typename SigT, typename ThT>
static const void* step_fn(bool dir) {
    return dir ? reinterpret_cast<const void*>(&plain_step_kernel<SigT, ThT, true>)
               : reinterpret_cast<const void*>(&plain_step_kernel<SigT, ThT, false>);
}

// Build the graph: one WHILE node (condition 1 at every launch) whose body is
// a chain of kUnroll step launches.
static sp_status build_step_graph(const void* fn, int grid, StepBlock* d_blk, cudaGraphExec_t* out) {
    cudaGraph_t gr = nullptr;
    SP_CUDA(cudaGraphCreate(&gr, 0));
    struct Del {
        cudaGraph_t g;
        ~Del() { cudaGraphDestroy(g); }
    } del{gr};
    cudaGraphConditionalHandle cond;
    SP_CUDA(cudaGraphConditionalHandleCreate(&cond, gr, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    SP_CUDA(cudaGraphAddNode(&cnode, gr, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];

    StepBlock* blk = d_blk;
    void* kargs[] = {(void*)&blk, (void*)&cond};
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(fn);
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(kPlainThreads);
    kp.sharedMemBytes = 0;
    kp.kernelParams = kargs;
    cudaGraphNode_t prev = nullptr;
    for (int i = 0; i < kUnroll; ++i) {
        cudaGraphNode_t node;
        SP_CUDA(cudaGraphAddKernelNode(&node, body, prev ? &prev : nullptr, prev ? 1 : 0, &kp));
        prev = node;
    }
    SP_CUDA(cudaGraphInstantiate(out, gr, 0));
    return SP_OK;
}

sp_status run_plain_graph(const PlainLaunch& L, LaunchResult* result) {
    Graph* g = const_cast<Graph*>(L.g);
    const int64_t n = g->n;
    cudaStream_t st = L.stream;
    if (L.mode != PlainMode::BC) return fail(SP_ERR_INVALID_ARG, "graph-driven level loop: BC mode only");
    Tiers tiers{16, 4096, 4096};
    const int variant = (L.sigma_float ? 2 : 0) + (L.theta_f32 ? 1 : 0);
    const bool dir = g->directed;
    const void* fn = L.sigma_float ? (L.theta_f32 ? step_fn<double, float>(dir) : step_fn<double, double>(dir))
                                   : (L.theta_f32 ? step_fn<unsigned long long, float>(dir)
                                                  : step_fn<unsigned long long, double>(dir));
    int per_sm = 0;
    SP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPlainThreads, 0));
    if (per_sm < 1) return fail(SP_ERR_CUDA, "plain step kernel cannot be resident");
    int grid = per_sm * device_sm_count(g->device);
    if (L.max_ctas > 0 && L.max_ctas < grid) grid = L.max_ctas;

    const int64_t lcap = L.level_cap > 0 ? std::min<int64_t>(L.level_cap, n + 2) : n + 2;
    const int64_t hcap = g->knnz() / tiers.t_hub + 2;
    const int64_t segcap = g->knnz() / tiers.seg + hcap + 2;
    const PlainLayout lay = plain_layout(n, lcap, hcap, segcap, 1, grid, false);
    char* ws = nullptr;
    cudaError_t ce = cudaMallocAsync((void**)&ws, lay.bytes, st);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return fail(SP_ERR_OOM, "workspace allocation (plain form, graph-driven)");
    }
    struct FreeWs {
        char* p;
        cudaStream_t s;
        ~FreeWs() { cudaFreeAsync(p, s); }
    } free_ws{ws, st};
    SP_CUDA(cudaMemsetAsync(ws, 0, lay.zero_end, st));

    StepBlock hb{};
    PlainArgs& a = hb.args;
    a.rp = g->krp();
    a.ci = g->kci();
    a.directed = g->directed;
    a.odeg = g->d_odeg;
    a.n = (int32_t)n;
    a.sources = L.d_sources;
    a.nsrc = L.nsrc;
    a.bc = L.d_bc;
    plain_bind(a, ws, lay);
    a.gblocks = grid;
    a.ngroups = 1;
    a.hcap = (int32_t)hcap;
    a.segcap = (int32_t)segcap;
    a.lcap = (int32_t)lcap;
    a.pre_err = nullptr;
    a.gate = nullptr;
    a.mode = (int)PlainMode::BC;
    a.debug_flags = 0;
    a.timeout_ns = L.timeout_ns;
    a.t_thread = tiers.t_thread;
    a.t_hub = tiers.t_hub;
    a.seg = tiers.seg;
    a.bu_den = L.bottom_up_den;
    a.centre_bound = sigma_centre_bound(L.sigma_float, L.theta_f32, L.mode);
    a.trace = nullptr;
    hb.state.stage = kStageInit;
    hb.state.step_limit = (long long)L.nsrc * (2 * n + 2) + 2;

    StepCache* c;
    {
        std::lock_guard<std::mutex> lk(g->mu);
        if (!g->step_cache) g->step_cache = new StepCache();
        c = reinterpret_cast<StepCache*>(g->step_cache);
    }
    std::lock_guard<std::mutex> clk(c->mu);  // the device block is shared by calls on this graph
    if (!c->d_blk) {
        ce = cudaMalloc((void**)&c->d_blk, sizeof(StepBlock));
        if (ce != cudaSuccess) {
            cudaGetLastError();
            c->d_blk = nullptr;
            return fail(SP_ERR_OOM, "graph-driven loop state");
        }
    }
    if (!c->exec[variant] || c->grid[variant] != grid) {
        if (c->exec[variant]) cudaGraphExecDestroy(c->exec[variant]);
        c->exec[variant] = nullptr;
        sp_status rc = build_step_graph(fn, grid, c->d_blk, &c->exec[variant]);
        if (rc != SP_OK) return rc;
        c->grid[variant] = grid;
    }
    // hb is pageable: the copy has read it before cudaMemcpyAsync returns.
    SP_CUDA(cudaMemcpyAsync(c->d_blk, &hb, sizeof(StepBlock), cudaMemcpyHostToDevice, st));

    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, st);
    ce = cudaGraphLaunch(c->exec[variant], st);
    cudaEventRecord(ev1, st);
    static thread_local Ctl h;
    std::memset(&h, 0, sizeof(h));
    StepState fs{};
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h, ws + lay.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(&fs, &c->d_blk->state, sizeof(StepState), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    float ms = 0.0f;
    if (ce == cudaSuccess && cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess) result->kernel_ms = ms;
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (ce != cudaSuccess) return cuda_fail(ce, "graph-driven plain form");
    result->err = h.err;
    result->levels = h.max_levels;
    result->traversed_arcs = h.traversed_arcs;
    result->reached = h.reached;
    result->entries = h.reached;
    result->scanned_arcs = h.scanned_arcs;
    result->dag_arcs = h.dag_arcs;
    result->recentred = h.recentred;
    result->lcap = lcap;
    result->grid = grid;
    result->groups = 1;
    // every WHILE iteration launches the whole chain, finished or not
    result->launches = (int)std::min<long long>((fs.steps + kUnroll - 1) / kUnroll * kUnroll, INT_MAX);
    return SP_OK;
}

}  // namespace sp
