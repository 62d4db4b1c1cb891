// Plain form: one source at a time per group of blocks.
//
// Per source (paper Section 2, Fig. 1, ComputeBC; the level-synchronous BFS of
// Section 3.4) a group of blocks runs
//   init      level[] = -1, level[src] = 0, sigma[src] = 1
//   forward   for d = 0, 1, ...: every vertex v at level d pulls sigma from its
//             neighbours at level d-1 (the iterateInBFS sum over BFS parents)
//             and claims its unvisited neighbours for level d+1 in the same
//             adjacency scan; the level stack Q holds the levels in order
//   backward  for d = L-1 ... 1: v pulls theta(w) = (1 + delta(w)) / sigma(w)
//             from its neighbours at level d+1, then delta(v) = sigma(v) * sum,
//             BC(v) += delta(v) (the iterateInReverse sum over BFS children,
//             written so that no floating-point atomics are needed)
// with a timed barrier over the group's blocks between levels instead of the
// paper's host loop that copies a `finished` flag every level (Section 3.4;
// Section 4.1).
//
// Groups: the persistent launch is cut into `ngroups` groups of `gblocks`
// blocks.  Group g takes sources g, g + ngroups, ... in order, with its own
// level arrays, level stack, barrier and partial BC vector; the partial
// vectors are added in group order by a second kernel.  One group of every
// block suits graphs whose levels are wide (millions of arcs); many small
// groups suit high-diameter graphs, whose thousands of narrow levels would
// otherwise leave most of the GPU waiting at barriers.
//
// Work distribution inside a level: entries of Q are taken 32 at a time by a
// warp; rows of at most t_thread arcs are walked by one lane, longer rows by
// the whole warp, and rows longer than t_hub (hubs) are split into segments of
// `seg` arcs taken by different warps, whose partial sums the last segment to
// finish adds in segment order.  Every per-vertex sum therefore has an order
// fixed by the graph alone: results are bit-identical from run to run.
//
// Path counts: exact unsigned 64-bit integer sums (identical to FP64 sums while
// counts stay below 2^53), or, when counts overflow 64 bits, FP64 values with a
// power-of-two exponent per level (recentred when the level strays from 2^0).
#pragma once

#include <climits>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace sp {

// 512 threads, two blocks per SM: every variant fits in 64 registers, so the
// persistent grid (and the number of block groups) is the same for all.
constexpr int kPlainThreads = 512;

// Barrier and work counters of one block group (zeroed by the host).
struct GroupCtl {
    unsigned int bar_count;
    unsigned int bar_gen;
    unsigned int work[4];
    int qtail;
    int snap[2];
    int pad[7];
};

struct PlainArgs {
    const int32_t* rp;
    const int32_t* ci;
    int32_t n;
    const int32_t* sources;
    int32_t nsrc;
    double* bc;             // output; written directly when ngroups == 1
    double* bcpart;         // [ngroups][n] partial BC per group (ngroups > 1)
    double* sq;             // optional [n]: sum over the sources of delta_s(v)^2 (sampling bounds)
    double* sqpart;         // [ngroups][n] its partials per group (ngroups > 1)
    int32_t gblocks;        // blocks per group
    int32_t ngroups;
    // Per-group arrays: group g's copy starts at base + g * stride.
    int32_t* lvl;           // [n]
    void* sig;              // [n] 8-byte elements
    void* th;               // [n] 8-byte slots
    int32_t* q;             // [n] level stack
    int2* qrow;             // [n] row start and degree of each level-stack entry
    int32_t* qoff;          // [lcap]
    int32_t* hoff;          // [lcap]
    unsigned long long* hcnt;  // [lcap]: records << 32 | segments, per level
    int32_t* emax;          // [lcap] per-level exponent range of scaled sigma
    int32_t* emin;          // [lcap]
    long long* fexp;        // [lcap] cumulative exponent per level (sigma output)
    HubRec* hubs;           // [hcap]
    int32_t* hdone;         // [2*hcap]: forward / backward finish counters
    double* part;           // [segcap] per-segment partial sums (8-byte slots)
    int32_t hcap;
    int32_t segcap;
    int32_t lcap;
    Ctl* ctl;               // launch-wide: error, statistics
    GroupCtl* gctl;         // [ngroups]
    const int* pre_err;     // asynchronous calls: nonzero = the sources failed their check, do nothing
    const int* gate;        // asynchronous fallback launch: run only when *gate != 0 (null = always)
    int32_t* dist_out;
    double* mant_out;
    long long* exp_out;
    int mode;
    int debug_flags;
    unsigned long long timeout_ns;
    int t_thread, t_hub, seg;
    int bu_den;  // bottom-up discovery on levels with more than n / bu_den vertices (0 = never)
    // FP64 path counts: a level is recentred once its exponent range leaves
    // [-centre_bound, centre_bound] (0 = 512).  With FP32 theta the host passes
    // 64, so that theta-hat = (1 + delta) / sigma-hat stays in FP32 normals.
    int centre_bound;
    int directed;           // rp/ci: combined out- and in-arc rows (arc_in / arc_out); odeg: out-degrees
    const int32_t* odeg;
    int* trace;  // SP_TRACE builds: 8 ints per warp
};

// Barrier over the `nblocks` blocks of one group: as grid_sync (common.cuh),
// with the group's own counters; the last block to arrive snapshots the
// group's level-stack fill.  A group of one block needs only __syncthreads.
static __device__ __noinline__ bool group_sync(Ctl* ctl, GroupCtl* gc, unsigned nblocks, uint64_t timeout_ns,
                                               int phase, bool skip, int* qtail_snap, const int* block_qtail) {
    __shared__ int s_ok, s_snap;
    __syncthreads();
    if (nblocks == 1) {
        if (threadIdx.x == 0) {
            if (blockIdx.x < 1024) ctl->block_phase[blockIdx.x] = phase;
            s_snap = ld_volatile(block_qtail);
            s_ok = (ld_volatile(&ctl->err) == 0 && !skip) ? 1 : 0;
        }
        __syncthreads();
        *qtail_snap = s_snap;
        return s_ok != 0;
    }
    if (threadIdx.x < 32) {
        if (threadIdx.x == 0) {
            int ok = skip ? 0 : 1;
            int snapv = 0;
            if (!skip) {
                unsigned gen = ld_acquire_u32(&gc->bar_gen);
                if (blockIdx.x < 1024) ctl->block_phase[blockIdx.x] = phase;
                __threadfence();
                unsigned arrived = atomicAdd(&gc->bar_count, 1u);
                if (arrived == nblocks - 1) {
                    gc->snap[gen & 1u] = ld_volatile(&gc->qtail);
                    gc->bar_count = 0;
                    st_release_u32(&gc->bar_gen, gen + 1);
                } else {
                    uint64_t t0 = globaltimer();
                    unsigned ns = 32;
                    while (ld_acquire_u32(&gc->bar_gen) == gen) {
                        if (ld_volatile(&ctl->err) != 0) { ok = 0; break; }
                        if (globaltimer() - t0 > timeout_ns) {
                            if (atomicCAS(&ctl->err, 0, (int)SP_ERR_TIMEOUT) == 0) {
                                ctl->err_where = phase;
                                ctl->timeout_count = ld_volatile(&gc->bar_count);
                            }
                            ok = 0;
                            break;
                        }
                        __nanosleep(ns);
                        if (ns < 512) ns <<= 1;
                    }
                }
                __threadfence();
                snapv = ld_volatile(&gc->snap[gen & 1u]);
            }
            __threadfence();
            if (ld_volatile(&ctl->err) != 0) ok = 0;
            s_ok = ok;
            s_snap = snapv;
        }
        __syncwarp();
    }
    __syncthreads();
    *qtail_snap = s_snap;
    return s_ok != 0;
}

template <typename SigT>
struct SigOps;
template <>
struct SigOps<unsigned long long> {
    static __device__ __forceinline__ unsigned long long add(unsigned long long a, unsigned long long b, bool& ovf) {
        unsigned long long s = a + b;
        ovf |= s < a;
        return s;
    }
    static __device__ __forceinline__ unsigned long long warp_sum(unsigned long long v, bool& ovf) {
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long y = shfl_u64(kFull, v, lane_id() ^ o);
            v = add(v, y, ovf);
        }
        return v;
    }
};
template <>
struct SigOps<double> {
    static __device__ __forceinline__ double add(double a, double b, bool&) { return a + b; }
    static __device__ __forceinline__ double warp_sum(double v, bool&) { return warp_sum_f64(v); }
};

// kRec: the per-(group, vertex) state is one 32-byte record (level @0, BC
// partial @8, path count @16, theta @24) instead of separate arrays, so that a
// vertex's level test and its path count or theta share one DRAM sector; used
// when the groups' state is far larger than L2 and every access is a miss.
template <typename SigT, typename ThT, bool kRec, bool kDir>
struct PlainKernel {
    // Arcs of the rows this launch reads: for a directed graph the combined
    // rows (arc_in / arc_out); for an undirected one every arc serves both ways.
    static __device__ __forceinline__ int avtx(int raw) { return kDir ? arc_vertex(raw) : raw; }
    static __device__ __forceinline__ bool ain(int raw) { return !kDir || raw < 0; }
    static __device__ __forceinline__ bool aout(int raw) { return !kDir || raw >= 0; }
    const PlainArgs& a;
    Ctl* ctl;
    GroupCtl* gc;
    int lane;
    int* qtail;  // level-stack fill: shared memory for a one-block group, else the group's counter
    int grp;     // group index
    size_t gn;   // group offset into [n] arrays
    size_t gl;   // group offset into [lcap] arrays
    size_t gh;   // group offset into [hcap] arrays
    // per-level state (identical in every thread of the group)
    int d = 0;
    int hoff_d = 0, nrec_d = 0, nseg_d = 0;  // hub records of level d
    int hoff_next = 0;                       // first hub record of level d+1
    int cshift_prev = 0;                     // centring shift between level d-1 and d
    int cshift_cur = 0;                      // centring shift between level d and d+1 (backward)
    bool discover = true;                    // top-down discovery by the level's entries
    // per-thread accumulators
    int my_emax = INT_MIN, my_emin = INT_MAX;
    bool ovf = false;
    unsigned long long st_arcs = 0, st_reached = 0, st_scanned = 0, st_dag = 0;

    __device__ PlainKernel(const PlainArgs& args, int g)
        : a(args), ctl(args.ctl), gc(args.gctl + g), lane(lane_id()), qtail(&(args.gctl + g)->qtail), grp(g),
          gn((size_t)g * (size_t)args.n),
          gl((size_t)g * (size_t)args.lcap), gh((size_t)g * (size_t)args.hcap) {}

    static constexpr size_t kRecInts = 8;  // 32-byte vertex record
    __device__ __forceinline__ int32_t& lv(int v) const {
        if constexpr (kRec) return a.lvl[(gn + (size_t)v) * kRecInts];
        else return a.lvl[gn + (size_t)v];
    }
    __device__ __forceinline__ SigT& sg(int v) const {
        if constexpr (kRec) return *reinterpret_cast<SigT*>(a.lvl + (gn + (size_t)v) * kRecInts + 4);
        else return reinterpret_cast<SigT*>(a.sig)[gn + (size_t)v];
    }
    __device__ __forceinline__ ThT& tt(int v) const {
        if constexpr (kRec) return *reinterpret_cast<ThT*>(a.lvl + (gn + (size_t)v) * kRecInts + 6);
        else return reinterpret_cast<ThT*>(reinterpret_cast<double*>(a.th) + gn)[v];
    }
    // BC of v: the output itself for one group, else the group's partial
    __device__ __forceinline__ double& bb(int v) const {
        if constexpr (kRec) {
            if (a.ngroups > 1) return *reinterpret_cast<double*>(a.lvl + (gn + (size_t)v) * kRecInts + 2);
        }
        return a.ngroups == 1 ? a.bc[v] : a.bcpart[gn + (size_t)v];
    }
    // Power-of-two shift that centres a level of scaled path counts whose
    // exponents span [emin, emax] (X6 with the launch's bound).
    __device__ __forceinline__ int shift_of(int emax, int emin) const {
        return centre_shift(emax, emin, a.centre_bound > 0 ? a.centre_bound : 512);
    }
    __device__ __forceinline__ int32_t* q() const { return a.q + gn; }
    __device__ __forceinline__ int2* qrow() const { return a.qrow + gn; }
    __device__ __forceinline__ int32_t* qoff() const { return a.qoff + gl; }
    __device__ __forceinline__ int32_t* hoff() const { return a.hoff + gl; }
    __device__ __forceinline__ unsigned long long* hcnt() const { return a.hcnt + gl; }
    __device__ __forceinline__ int32_t* emax() const { return a.emax + gl; }
    __device__ __forceinline__ int32_t* emin() const { return a.emin + gl; }
    __device__ __forceinline__ long long* fexp() const { return a.fexp + gl; }
    __device__ __forceinline__ HubRec* hubs() const { return a.hubs + gh; }
    __device__ __forceinline__ int32_t* hdone() const { return a.hdone + 2 * gh; }
    __device__ __forceinline__ double* part() const { return a.part + (size_t)grp * (size_t)a.segcap; }

    // Level stack of a new source: src alone on level 0, sigma[src] = 1, and
    // src's hub record when its row is split into segments.  One thread.
    __device__ void start_source(int src) {
        const int rb = a.rp[src];
        int du = a.rp[src + 1] - rb;
        q()[0] = src;
        qrow()[0] = make_int2(rb, du);
        *qtail = 1;
        qoff()[0] = 0;
        hoff()[0] = 0;
        hcnt()[0] = 0ull;
        hcnt()[1] = 0ull;
        emax()[0] = 0;
        emin()[0] = 0;
        sg(src) = (SigT)1;
        if (du > a.t_hub) {
            int nseg = (du + a.seg - 1) / a.seg;
            if (a.hcap < 1 || nseg > a.segcap) {
                set_error(ctl, kErrCapacity);
            } else {
                q()[0] = (int)((unsigned)src | kHubFlag);
                HubRec h;
                h.v = src; h.qpos = 0; h.nseg = nseg; h.seg_base = 0;
                hubs()[0] = h;
                hdone()[0] = 0;
                hdone()[a.hcap] = 0;
                hcnt()[0] = (1ull << 32) | (unsigned long long)nseg;
            }
        }
    }

    // Bookkeeping before the forward pass over level d (entries end at qe):
    // level d+1 starts at qe; its hub counters and exponent range start empty.
    // One thread.
    __device__ void open_level(int qe) {
        qoff()[d + 1] = qe;
        hoff()[d] = hoff_d;
        hcnt()[d + 2] = 0ull;
        emax()[d + 1] = INT_MIN;
        emin()[d + 1] = INT_MAX;
    }

    // A vertex claimed for level `nl`: append to the level stack (and the hub list).
    __device__ void push(int u, int nl) {
        const int rb = __ldg(&a.rp[u]);
        push_row(u, nl, rb, __ldg(&a.rp[u + 1]) - rb);
    }
    // The same with u's row (start rb, degree du) already loaded.
    __device__ void push_row(int u, int nl, int rb, int du) {
        bool hub = du > a.t_hub;
        int pos = aggregated_slot(qtail);
        if (pos >= a.n) { set_error(ctl, kErrCapacity); return; }
        q()[pos] = hub ? (int)((unsigned)u | kHubFlag) : u;
        qrow()[pos] = make_int2(rb, du);
        if (hub) {
            int nseg = (du + a.seg - 1) / a.seg;
            unsigned long long old = atomicAdd(&hcnt()[nl], (1ull << 32) | (unsigned long long)(unsigned)nseg);
            int rec = hoff_next + (int)(old >> 32);
            int sb = (int)(old & 0xFFFFFFFFull);
            if (rec >= a.hcap || sb + nseg > a.segcap) { set_error(ctl, kErrCapacity); return; }
            HubRec h;
            h.v = u; h.qpos = pos; h.nseg = nseg; h.seg_base = sb;
            hubs()[rec] = h;
            hdone()[rec] = 0;
            hdone()[a.hcap + rec] = 0;
        }
    }

    // Forward visit of the arc `raw` of a vertex v at level d (its other end
    // u, u's level already loaded as lu): claim u for level d+1 over an arc
    // out of v, or return sigma[u] if u is a parent over an arc into v.
    __device__ __forceinline__ SigT fwd_visit(int raw, int lu) {
        const int u = avtx(raw);
        SigT c = 0;
        if (lu < 0) {
            if (discover && aout(raw) && atomicCAS(&lv(u), -1, d + 1) == -1) push(u, d + 1);
        } else if (lu == d - 1 && ain(raw)) {
            c = __ldcg(&sg(u));
            st_dag += 1;
        }
        return c;
    }
    __device__ __forceinline__ SigT fwd_arc(int raw) { return fwd_visit(raw, __ldcg(&lv(avtx(raw)))); }
    // Out-degree of v (traversed arcs); an undirected graph's row length.
    __device__ __forceinline__ int out_degree(int v, int row_len) const {
        return kDir ? __ldg(&a.odeg[v]) : row_len;
    }

    __device__ void fwd_finalize(int v, SigT acc, int deg) {
        st_arcs += (unsigned long long)deg;
        st_reached += 1;
        if (d == 0) return;  // sigma[src] = 1 was set by the init phase
        if constexpr (std::is_integral<SigT>::value) {  // integer path counts
            sg(v) = acc;
        } else {
            double val = scale2((double)acc, -cshift_prev);
            if (!normal_finite(val)) set_error(ctl, SP_ERR_RANGE);
            sg(v) = (SigT)val;
            int e = exp_field(val) - 1023;
            my_emax = max(my_emax, e);
            my_emin = min(my_emin, e);
        }
    }

    __device__ __forceinline__ double bwd_arc(int raw) {
        if (!aout(raw)) return 0.0;  // children: out-arcs only
        const int w = avtx(raw);
        int lw = __ldcg(&lv(w));
        return lw == d + 1 ? (double)__ldcg(&tt(w)) : 0.0;
    }

    __device__ void bwd_finalize(int v, double acc) {
        double sv = (double)__ldcg(&sg(v));
        double delta = sv * acc;
        if constexpr (!std::is_integral<SigT>::value) delta = scale2(delta, -cshift_cur);
        double t = (1.0 + delta) / sv;
        if constexpr (sizeof(ThT) == 4) {
            float tf = (float)t;
            if (!normal_finite_f(tf)) set_error(ctl, kErrThetaRange32);
            tt(v) = (ThT)tf;
        } else {
            if (!normal_finite(t)) set_error(ctl, SP_ERR_RANGE);
            tt(v) = (ThT)t;
        }
        double& b = bb(v);
        b = __ldcg(&b) + delta;
        if (a.sq != nullptr) {
            double& q = a.ngroups == 1 ? a.sq[v] : a.sqpart[gn + (size_t)v];
            q = __ldcg(&q) + delta * delta;
        }
    }

    // One chunk of level-stack entries [e0, qe), at most 32.
    template <bool FWD>
    __device__ void chunk(int e0, int qe, bool skip_arcs) {
        int e = e0 + lane;
        bool valid = e < qe;
        unsigned qv = kHubFlag;
        int2 rw = make_int2(0, 0);
        if (valid) {  // the entry and its row, stored together when it was pushed
            qv = (unsigned)__ldcg(&q()[e]);
            rw = __ldcg(&qrow()[e]);
        }
        bool hubent = (qv & kHubFlag) != 0;
        int v = (int)(qv & kVertexMask);
        if (valid && (v >= a.n || rw.x < 0 || rw.y < 0)) {
            set_error(ctl, kErrCorrupt);
            valid = false;
            hubent = true;
            v = 0;
        }
        int beg = 0, deg = 0;
        if (!hubent) {
            beg = rw.x;
            deg = rw.y;
        }
        int walk = skip_arcs ? 0 : deg;
        SigT sacc = 0;
        double tacc = 0.0;
        if (walk <= a.t_thread) {
            // one lane walks the row, four arcs at a time: their column ids,
            // then their levels, then their sigma / theta loads are issued
            // together; the sums still run in CSR order
            constexpr int G = 4;
            for (int k0 = 0; k0 < walk; k0 += G) {
                int u[G], lu[G];
                bool out[G], in[G];  // the arc leads out of v (claims, children) / into v (parents)
#pragma unroll
                for (int i = 0; i < G; ++i) {
                    const int raw = k0 + i < walk ? __ldg(&a.ci[beg + k0 + i]) : 0;
                    u[i] = k0 + i < walk ? avtx(raw) : -1;
                    out[i] = u[i] >= 0 && aout(raw);
                    in[i] = u[i] >= 0 && ain(raw);
                }
#pragma unroll
                for (int i = 0; i < G; ++i) lu[i] = u[i] >= 0 ? __ldcg(&lv(u[i])) : INT_MIN;
                if constexpr (FWD) {
                    // parents' path counts, the claims of unvisited
                    // neighbours, and the rows of the claimed ones are each
                    // issued for all G arcs before any result is used
                    SigT c[G];
                    bool claim[G];
#pragma unroll
                    for (int i = 0; i < G; ++i) {
                        c[i] = (SigT)0;
                        claim[i] = discover && out[i] && lu[i] < 0;
                        if (in[i] && lu[i] >= 0 && lu[i] == d - 1) {  // a parent (none on level 0)
                            c[i] = __ldcg(&sg(u[i]));
                            st_dag += 1;
                        }
                    }
#pragma unroll
                    for (int i = 0; i < G; ++i)
                        if (claim[i]) claim[i] = atomicCAS(&lv(u[i]), -1, d + 1) == -1;
                    int rb[G], re[G];
#pragma unroll
                    for (int i = 0; i < G; ++i) {
                        rb[i] = claim[i] ? __ldg(&a.rp[u[i]]) : 0;
                        re[i] = claim[i] ? __ldg(&a.rp[u[i] + 1]) : 0;
                    }
#pragma unroll
                    for (int i = 0; i < G; ++i)
                        if (claim[i]) push_row(u[i], d + 1, rb[i], re[i] - rb[i]);
#pragma unroll
                    for (int i = 0; i < G; ++i) sacc = SigOps<SigT>::add(sacc, c[i], ovf);
                } else {
                    double t[G];
#pragma unroll
                    for (int i = 0; i < G; ++i) t[i] = out[i] && lu[i] == d + 1 ? (double)__ldcg(&tt(u[i])) : 0.0;
#pragma unroll
                    for (int i = 0; i < G; ++i) tacc += t[i];
                }
            }
        }
        unsigned big = __ballot_sync(kFull, walk > a.t_thread);
        while (big) {
            int j = __ffs(big) - 1;
            big &= big - 1;
            int bj = __shfl_sync(kFull, beg, j), dj = __shfl_sync(kFull, deg, j);
            SigT sp_ = 0;
            double tp = 0.0;
            for (int k = lane; k < dj; k += kWarp) {
                const int raw = __ldg(&a.ci[bj + k]);
                if constexpr (FWD) sp_ = SigOps<SigT>::add(sp_, fwd_arc(raw), ovf);
                else tp += bwd_arc(raw);
            }
            if constexpr (FWD) {
                sp_ = SigOps<SigT>::warp_sum(sp_, ovf);
                if (lane == j) sacc = sp_;
            } else {
                tp = warp_sum_f64(tp);
                if (lane == j) tacc = tp;
            }
        }
        if (valid && !hubent) {
            st_scanned += (unsigned long long)walk;
            if constexpr (FWD) fwd_finalize(v, sacc, out_degree(v, deg));
            else bwd_finalize(v, tacc);
        }
    }

    // Segment g of the hubs of level d.
    template <bool FWD>
    __device__ void hub_segment(int g, bool skip_arcs) {
        int r = find_hub(hubs(), hoff_d, hoff_d + nrec_d, g);
        HubRec h;
        h.v = __ldcg(&hubs()[r].v);
        h.nseg = __ldcg(&hubs()[r].nseg);
        h.seg_base = __ldcg(&hubs()[r].seg_base);
        if (h.v < 0 || h.v >= a.n || h.nseg < 1 || h.seg_base < 0 || h.seg_base + h.nseg > a.segcap) {
            if (lane == 0) set_error(ctl, kErrCorrupt);
            return;
        }
        int s = g - h.seg_base;
        int rb = __ldg(&a.rp[h.v]), re = __ldg(&a.rp[h.v + 1]);
        int beg = rb + s * a.seg;
        int end = min(re, beg + a.seg);
        if (skip_arcs) end = beg;
        SigT sp_ = 0;
        double tp = 0.0;
        for (int k = beg + lane; k < end; k += kWarp) {
            const int raw = __ldg(&a.ci[k]);
            if constexpr (FWD) sp_ = SigOps<SigT>::add(sp_, fwd_arc(raw), ovf);
            else tp += bwd_arc(raw);
        }
        if (lane == 0) st_scanned += (unsigned long long)(end - beg);
        int* done = FWD ? &hdone()[r] : &hdone()[a.hcap + r];
        int old = 0;
        if constexpr (FWD) {
            sp_ = SigOps<SigT>::warp_sum(sp_, ovf);
            if (lane == 0) reinterpret_cast<SigT*>(part())[g] = sp_;
        } else {
            tp = warp_sum_f64(tp);
            if (lane == 0) part()[g] = tp;
        }
        if (lane == 0) {
            __threadfence();
            old = atomicAdd(done, 1);
        }
        old = __shfl_sync(kFull, old, 0);
        if (old != h.nseg - 1) return;
        __threadfence();
        // Last segment: add the partial sums in segment order.
        SigT st = 0;
        double tt = 0.0;
        for (int k = lane; k < h.nseg; k += kWarp) {
            if constexpr (FWD) st = SigOps<SigT>::add(st, __ldcg(&reinterpret_cast<SigT*>(part())[h.seg_base + k]), ovf);
            else tt += __ldcg(&part()[h.seg_base + k]);
        }
        if constexpr (FWD) {
            st = SigOps<SigT>::warp_sum(st, ovf);
            if (lane == 0) fwd_finalize(h.v, st, out_degree(h.v, re - rb));
        } else {
            tt = warp_sum_f64(tt);
            if (lane == 0) bwd_finalize(h.v, tt);
        }
    }

    // Bottom-up discovery of level d+1 (direction-optimising BFS, Beamer et
    // al., SC 2012): each still-unvisited vertex of a range of 256 scans its
    // row and stops at the first neighbour on level d.  Only the scanning
    // thread writes the vertex's level, so no atomic is needed; path counts
    // are pulled as usual when the vertex's level is processed.
    __device__ void bottom_up_range(int base) {
#pragma unroll 1
        for (int i = 0; i < 8; ++i) {
            const int u = base + i * kWarp + lane;
            if (u < a.n && __ldcg(&lv(u)) < 0) {
                const int b = __ldg(&a.rp[u]), e = __ldg(&a.rp[u + 1]);
                for (int k = b; k < e; ++k) {
                    st_scanned += 1;
                    const int raw = __ldg(&a.ci[k]);
                    if (!ain(raw)) continue;  // only an arc into u can reach it
                    if (__ldcg(&lv(avtx(raw))) == d) {
                        lv(u) = d + 1;
                        push(u, d + 1);
                        break;
                    }
                }
            }
        }
    }

    // Items of one level: hub segments, chunks of 32 entries, bottom-up
    // ranges.  Warp w of the group takes item w first and further items from
    // the group's counter, so a level with fewer items than warps costs no
    // atomics.
    template <bool FWD>
    __device__ void level_work(int phase, int qb, int qe, bool skip_arcs, int bu_items = 0) {
        const int nwarps = a.gblocks * (int)(blockDim.x / kWarp);
        const int c = entries_per_item(qe - qb, nwarps);
        int nchunks = (qe - qb + c - 1) / c;
        int total = nseg_d + nchunks + bu_items;
        int item = (int)(((blockIdx.x % a.gblocks) * blockDim.x + threadIdx.x) / kWarp);
        while (true) {
#ifdef SP_TRACE
            if (lane == 0 && a.trace) {
                int* t = a.trace + 8 * ((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
                t[0] = phase; t[1] = item; t[2] = total; t[3] = nseg_d; t[4] = qb; t[5] = qe; t[6] = d; t[7] += 1;
            }
#endif
            if (item >= total) break;
            if (item < nseg_d) hub_segment<FWD>(item, skip_arcs);
            else if (item < nseg_d + nchunks) {
                const int e0 = qb + (item - nseg_d) * c;
                chunk<FWD>(e0, min(e0 + c, qe), skip_arcs);
            }
            else bottom_up_range((item - nseg_d - nchunks) * (8 * kWarp));
            if (nwarps >= total) break;
            int next = 0;
            if (lane == 0) next = nwarps + (int)atomicAdd(&gc->work[phase & 3], 1u);
            item = __shfl_sync(kFull, next, 0);
        }
    }
};

// Whether an asynchronous launch skips its work: a fallback launch whose gate
// is closed, or a call whose sources failed their check on the device (the
// same words for every block, written before the launch).
static __device__ __forceinline__ bool plain_skip(const PlainArgs& a) {
    if (a.gate != nullptr && ld_volatile(a.gate) == 0) return true;
    if (a.pre_err != nullptr) {
        const int pe = ld_volatile(a.pre_err);
        if (pe != 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->err = pe;
            return true;
        }
    }
    return false;
}

template <typename SigT, typename ThT, bool kRec, bool kDir>
#ifndef SP_PLAIN_PER_SM
#define SP_PLAIN_PER_SM 2  // resident blocks per SM the registers are sized for
#endif
__global__ void __launch_bounds__(kPlainThreads, SP_PLAIN_PER_SM) plain_kernel(PlainArgs a) {
    if (plain_skip(a)) return;
    constexpr bool kFloatSig = !std::is_integral<SigT>::value;
    const int g = blockIdx.x / a.gblocks;
    if (g >= a.ngroups) return;  // the host sizes the grid to ngroups * gblocks
    PlainKernel<SigT, ThT, kRec, kDir> K(a, g);
    __shared__ int s_qtail;
    if (a.gblocks == 1) K.qtail = &s_qtail;  // the whole group is this block
    Ctl* ctl = a.ctl;
    GroupCtl* gc = K.gc;
    const int tid = (blockIdx.x % a.gblocks) * blockDim.x + threadIdx.x;  // rank in the group
    const int nthr = a.gblocks * blockDim.x;
    const int n = a.n;
    int phase = 0;
    int qsnap = 0;  // level-stack fill at the last barrier
    int levels_max = 0;
    // Barrier between phases; the work counter of phase p+2 is cleared in phase p.
    auto sync = [&]() -> bool {
        bool skip = (a.debug_flags & SP_DEBUG_SKIP_BARRIER) && blockIdx.x == 0 && phase == 1;
        bool ok = group_sync(ctl, gc, a.gblocks, a.timeout_ns, phase++, skip, &qsnap, K.qtail);
        if (tid == 0) gc->work[(phase + 2) & 3] = 0u;
        return ok;
    };

    if (a.mode == (int)PlainMode::BC) {
        for (int i = tid; i < n; i += nthr) K.bb(i) = 0.0;
        if (a.sq != nullptr) {
            double* q = a.ngroups == 1 ? a.sq : a.sqpart + K.gn;
            for (int i = tid; i < n; i += nthr) q[i] = 0.0;
        }
    }
    if (!sync()) goto out;

    for (int si = g; si < a.nsrc; si += a.ngroups) {
        const int src = __ldg(&a.sources[si]);
        // ---- init ----
        for (int i = tid; i < n; i += nthr) K.lv(i) = (i == src) ? 0 : -1;
        if (tid == 0) K.start_source(src);
        if (!sync()) goto out;

        // ---- forward ----
        int qb = 0, qe = 1;
        K.d = 0;
        K.hoff_d = 0;
        while (true) {
            const int d = K.d;
            if (d + 2 >= a.lcap) {
                if (tid == 0) set_error(ctl, kErrCapLevels);
                sync();
                goto out;
            }
            unsigned long long hc = ld_volatile(&K.hcnt()[d]);
            K.nrec_d = (int)(hc >> 32);
            K.nseg_d = (int)(hc & 0xFFFFFFFFull);
            K.hoff_next = K.hoff_d + K.nrec_d;
            if constexpr (kFloatSig) {
                K.cshift_prev = d > 0 ? K.shift_of(ld_volatile(&K.emax()[d - 1]), ld_volatile(&K.emin()[d - 1])) : 0;
                if (tid == 0 && K.cshift_prev != 0) atomicAdd(&ctl->recentred, 1ull);
            }
            if (tid == 0) K.open_level(qe);
            K.my_emax = INT_MIN;
            K.my_emin = INT_MAX;
            // Direction: fat levels discover bottom-up.
            const bool bu = a.bu_den > 0 && d > 0 && (int64_t)(qe - qb) * a.bu_den > (int64_t)n;
            K.discover = !bu;
            K.template level_work<true>(phase, qb, qe, false, bu ? (n + 8 * kWarp - 1) / (8 * kWarp) : 0);
            K.discover = true;
            if constexpr (kFloatSig) {
                int mx = warp_max_i32(K.my_emax), mn = warp_min_i32(K.my_emin);
                if (K.lane == 0 && mx >= mn) {
                    atomicMax(&K.emax()[d], mx);
                    atomicMin(&K.emin()[d], mn);
                }
            }
            if (K.ovf && a.mode != (int)PlainMode::BFS) set_error(ctl, kErrSigmaOverflow);
            if (!sync()) goto out;
            int nq = qsnap;
            K.hoff_d = K.hoff_next;
            if (nq == qe) break;
            qb = qe;
            qe = nq;
            K.d = d + 1;
        }
        const int L = K.d + 1;
        levels_max = max(levels_max, L);

        if (a.mode == (int)PlainMode::BFS) {
            int* row = a.dist_out + (size_t)si * (size_t)n;
            for (int i = tid; i < n; i += nthr) row[i] = __ldcg(&K.lv(i));
            if (!sync()) goto out;
            continue;
        }
        if (a.mode == (int)PlainMode::SIGMA) {
            if (tid == 0) {
                long long f = 0;
                for (int l = 0; l < L; ++l) {
                    K.fexp()[l] = f;
                    if constexpr (kFloatSig) f += K.shift_of(K.emax()[l], K.emin()[l]);
                }
            }
            if (!sync()) goto out;
            for (int i = tid; i < n; i += nthr) {
                int l = __ldcg(&K.lv(i));
                double m = 0.0;
                long long e2 = 0;
                if (l >= 0) {
                    double s = (double)__ldcg(&K.sg(i));
                    int e = exp_field(s) - 1023;
                    m = scale2(s, -e);
                    e2 = (long long)e + __ldcg(&K.fexp()[l]);
                }
                a.mant_out[i] = m;
                a.exp_out[i] = e2;
            }
            if (!sync()) goto out;
            continue;
        }

        // ---- backward ----
        for (int d = L - 1; d >= 1; --d) {
            K.d = d;
            int qbd = ld_volatile(&K.qoff()[d]);
            int qed = ld_volatile(&K.qoff()[d + 1]);
            unsigned long long hc = ld_volatile(&K.hcnt()[d]);
            K.hoff_d = ld_volatile(&K.hoff()[d]);
            K.nrec_d = (int)(hc >> 32);
            K.nseg_d = (int)(hc & 0xFFFFFFFFull);
            if constexpr (kFloatSig) K.cshift_cur = K.shift_of(ld_volatile(&K.emax()[d]), ld_volatile(&K.emin()[d]));
            K.template level_work<false>(phase, qbd, qed, d == L - 1);
            if (!sync()) goto out;
        }
    }

out:
    {
        // statistics: block-level then one atomic per block
        __shared__ unsigned long long s_st[4];
        if (threadIdx.x == 0) { s_st[0] = 0; s_st[1] = 0; s_st[2] = 0; s_st[3] = 0; }
        __syncthreads();
        atomicAdd(&s_st[0], K.st_arcs);
        atomicAdd(&s_st[1], K.st_reached);
        atomicAdd(&s_st[2], K.st_scanned);
        atomicAdd(&s_st[3], K.st_dag);
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicAdd(&ctl->traversed_arcs, s_st[0]);
            atomicAdd(&ctl->reached, s_st[1]);
            atomicAdd(&ctl->scanned_arcs, s_st[2]);
            atomicAdd(&ctl->dag_arcs, s_st[3]);
            atomicMax(&ctl->max_levels, levels_max);
        }
    }
}

// Offsets of the plain form's arrays inside its one workspace allocation
// (per-group copies of every per-source array, 256-byte aligned).
struct PlainLayout {
    size_t ctl, gctl, zero_end, lvl, sig, th, q, qrow, qoff, hoff, hcnt, emax, emin, fexp, hubs, hdone, part,
        bcpart, sqpart, trace, bytes;
};

// rec: one 32-byte record per (group, vertex) at `lvl` instead of the level,
// path-count, theta and partial-BC arrays.
inline PlainLayout plain_layout(int64_t n, int64_t lcap, int64_t hcap, int64_t segcap, int ngroups, int grid,
                                bool bcpart, bool rec = false, bool sqpart = false) {
    PlainLayout o{};
    const size_t G = (size_t)ngroups;
    size_t bytes = 0;
    auto take = [&](size_t b) { size_t at = bytes; bytes += (b + 255) & ~(size_t)255; return at; };
    o.ctl = take(sizeof(Ctl));
    o.gctl = take(sizeof(GroupCtl) * G);
    o.zero_end = bytes;
    o.lvl = take((rec ? 32 : sizeof(int32_t)) * (size_t)n * G);
    o.sig = take(rec ? 0 : 8 * (size_t)n * G);
    o.th = take(rec ? 0 : 8 * (size_t)n * G);
    o.q = take(sizeof(int32_t) * (size_t)n * G);
    o.qrow = take(sizeof(int2) * (size_t)n * G);
    o.qoff = take(sizeof(int32_t) * (size_t)lcap * G);
    o.hoff = take(sizeof(int32_t) * (size_t)lcap * G);
    o.hcnt = take(sizeof(unsigned long long) * (size_t)lcap * G);
    o.emax = take(sizeof(int32_t) * (size_t)lcap * G);
    o.emin = take(sizeof(int32_t) * (size_t)lcap * G);
    o.fexp = take(sizeof(long long) * (size_t)lcap * G);
    o.hubs = take(sizeof(HubRec) * (size_t)hcap * G);
    o.hdone = take(sizeof(int32_t) * 2 * (size_t)hcap * G);
    o.part = take(sizeof(double) * (size_t)segcap * G);
    o.bcpart = take(bcpart && !rec ? sizeof(double) * (size_t)n * G : 0);
    o.sqpart = take(sqpart && bcpart ? sizeof(double) * (size_t)n * G : 0);
    o.trace = take(sizeof(int) * 8 * (size_t)grid * (kPlainThreads / 32));
    o.bytes = bytes;
    return o;
}

inline void plain_bind(PlainArgs& a, char* ws, const PlainLayout& o) {
    a.bcpart = reinterpret_cast<double*>(ws + o.bcpart);
    a.sqpart = reinterpret_cast<double*>(ws + o.sqpart);
    a.lvl = reinterpret_cast<int32_t*>(ws + o.lvl);
    a.sig = ws + o.sig;
    a.th = ws + o.th;
    a.q = reinterpret_cast<int32_t*>(ws + o.q);
    a.qrow = reinterpret_cast<int2*>(ws + o.qrow);
    a.qoff = reinterpret_cast<int32_t*>(ws + o.qoff);
    a.hoff = reinterpret_cast<int32_t*>(ws + o.hoff);
    a.hcnt = reinterpret_cast<unsigned long long*>(ws + o.hcnt);
    a.emax = reinterpret_cast<int32_t*>(ws + o.emax);
    a.emin = reinterpret_cast<int32_t*>(ws + o.emin);
    a.fexp = reinterpret_cast<long long*>(ws + o.fexp);
    a.hubs = reinterpret_cast<HubRec*>(ws + o.hubs);
    a.hdone = reinterpret_cast<int32_t*>(ws + o.hdone);
    a.part = reinterpret_cast<double*>(ws + o.part);
    a.ctl = reinterpret_cast<Ctl*>(ws + o.ctl);
    a.gctl = reinterpret_cast<GroupCtl*>(ws + o.gctl);
    a.trace = reinterpret_cast<int*>(ws + o.trace);
}

// Sum of the groups' partial BC vectors, in group order.  Partial of group
// gi at vertex v: part[gi * n * vstride + v * vstride] (vstride 1 for the
// partial-BC arrays, 4 for the BC field of 32-byte vertex records).
static __global__ void sum_group_partials_kernel(const double* __restrict__ part, int ngroups, int64_t n,
                                                 int vstride, double* __restrict__ out, const int* gate) {
    if (gate != nullptr && ld_volatile(gate) == 0) return;  // a fallback launch that did not run
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int gi = 0; gi < ngroups; ++gi) s += part[((int64_t)gi * n + v) * vstride];
        out[v] = s;
    }
}

}  // namespace sp
