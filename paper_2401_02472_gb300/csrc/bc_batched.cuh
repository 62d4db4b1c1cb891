// Batched form: B = 32*W sources per batch traverse the graph together.
//
// Same method as the plain form (paper Section 2, Fig. 1, ComputeBC; level-
// synchronous BFS of Section 3.4), with many sources sharing each adjacency
// scan (the sourceSet loop of Fig. 1 run in parallel instead of in sequence):
//
//   per vertex v:          seen[v]    B-bit mask of sources that reached v
//   per level d:           F_d[v]     B-bit mask of sources with dist_s(v) = d
//                          (dense copies for the levels in use, a ring of 4)
//   per (vertex, source):  sig[v][s]  path counts, row-major so that a warp
//                          whose lane k*32+l is source k*32+l reads a row with
//                          coalesced loads
//                          th[v][s]   (1 + delta_s(v)) / sigma_s(v)
//   level stack:           entries (v, F_d[v]) for every vertex active at d
//
// Forward level d, for each entry (v, F) and each neighbour u of v:
//   sigma pull:   m = F & F_{d-1}[u];  sig[v][s] += sig[u][s] for s in m
//   discovery:    new = F & ~seen[u];  seen[u] |= new (atomic OR, the old value
//                 tells which bits are really new), F_{d+1}[u] |= new, and the
//                 first thread to give u bits at this level appends u
// Backward level d (L-1 .. 1), for each entry (v, F):
//   m = F & F_{d+1}[w] over neighbours w;  acc[s] += th[w][s] for s in m
//   delta_s(v) = sigma_s(v) * acc[s];  th[v][s] = (1 + delta) / sigma;
//   BC[v] += sum_s delta_s(v)
// The per-(vertex, source) sums walk v's row in CSR order (hubs: in segment
// order), so results are bit-identical from run to run.
#pragma once

#include <climits>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace sp {

#ifndef SP_BATCH_THREADS
#define SP_BATCH_THREADS 256  // threads per block
#endif
constexpr int kBatchThreads = SP_BATCH_THREADS;

#ifndef SP_BATCH_MINB
#define SP_BATCH_MINB 4  // resident blocks per SM the register budget is sized for
#endif

struct BatchArgs {
    const int32_t* rp;
    const int32_t* ci;
    int32_t n;
    const int32_t* sources;
    int32_t nsrc;
    double* bc;
    uint32_t* dense;          // [4][n][W]
    uint32_t* seen;           // [n][W]
    int32_t* ptag;            // [n] level stamp of the last append
    void* sig;                // [n][B]
    void* th;                 // [n][B]
    int32_t* ent;             // [ecap] level stack (vertex | hub flag)
    uint32_t* emask;          // [ecap][W]
    long long ecap;
    int32_t* eoff;            // [lcap+2]
    HubRec* hubs;
    int32_t hcap;
    int32_t* hoff;            // [lcap+2] first hub record of each level
    int32_t* soff;            // [lcap+2] first segment of each level in segrec
    int32_t* segrec;          // [scap] hub record of each segment
    int32_t scap;
    unsigned long long* hcnt; // [lcap+2] records << 32 | segments, per level
    int32_t* hdone;           // [2*hcap]
    void* part;               // [segcap][B] 8-byte slots
    int32_t segcap;
    int32_t* emax;            // [lcap][B]
    int32_t* emin;            // [lcap][B]
    int32_t lcap;
    Ctl* ctl;
    const int* pre_err;       // asynchronous calls: nonzero = the sources failed their check, do nothing
    int debug_flags;
    unsigned long long timeout_ns;
    int t_hub, seg;
    // Request mode (serving): sources are laid out in 32-lane words, each
    // word belonging to one request (-1 marks an empty lane); instead of one
    // BC vector the kernel keeps one partial BC vector per word and counts
    // traversed (arc, source) pairs and reached (vertex, source) pairs per
    // word, so that each request's result and statistics can be assembled
    // from its own words whatever else shares the launch.
    double* word_bc;                 // [nsrc / 32][n], zeroed by the host; null outside request mode
    unsigned long long* word_stats;  // [nsrc / 32][2]
    int bu_den;  // bottom-up discovery on levels with more than n / bu_den entries (0 = never)
    int centre_bound;  // FP64 path counts: recentre a level whose exponents leave [-bound, bound]
    int directed;      // rp/ci: combined out- and in-arc rows (arc_in / arc_out); odeg: out-degrees
    const int32_t* odeg;
    double* sq;        // optional [n]: sum over the call's sources of delta_s(v)^2 (sampling bounds)
    // Request mode: word_bc and word_stats hold word_cap word slots; word w
    // uses slot w % word_cap.  Live feed (serving): feed non-null; the words,
    // their lanes (sources, slot-indexed like word_bc) and the requests come
    // from the feed between batches instead of from nsrc.
    int32_t word_cap;
    FeedCtl* feed;
    FeedReq* feed_req;        // the feed's request records (host memory): done and counts are written here
    const int32_t* feed_lanes;  // the feed's lanes (host memory), copied into `sources` (device) as published
    FeedReq* req_dev;         // device copy of the published request records
    int32_t req_cap;
};

template <int W>
__device__ __forceinline__ void load_mask(const uint32_t* p, uint32_t (&m)[W]) {
    if constexpr (W == 1) {
        m[0] = __ldcg(p);
    } else if constexpr (W == 2) {
        uint2 x = __ldcg(reinterpret_cast<const uint2*>(p));
        m[0] = x.x; m[1] = x.y;
    } else {
#pragma unroll
        for (int k = 0; k < W; k += 4) {
            uint4 x = __ldcg(reinterpret_cast<const uint4*>(p + k));
            m[k] = x.x; m[k + 1] = x.y; m[k + 2] = x.z; m[k + 3] = x.w;
        }
    }
}
template <int W>
__device__ __forceinline__ void store_mask(uint32_t* p, const uint32_t (&m)[W]) {
    if constexpr (W == 1) {
        p[0] = m[0];
    } else if constexpr (W == 2) {
        *reinterpret_cast<uint2*>(p) = make_uint2(m[0], m[1]);
    } else {
#pragma unroll
        for (int k = 0; k < W; k += 4) *reinterpret_cast<uint4*>(p + k) = make_uint4(m[k], m[k + 1], m[k + 2], m[k + 3]);
    }
}
template <int W>
__device__ __forceinline__ void zero_mask(uint32_t* p) {
    uint32_t z[W];
#pragma unroll
    for (int k = 0; k < W; ++k) z[k] = 0u;
    store_mask<W>(p, z);
}

template <int W, typename SigT, typename ThT, bool kDir>
struct BatchKernel {
    static constexpr int B = 32 * W;
    // Arcs of the rows this launch reads: for a directed graph the combined
    // rows (arc_in / arc_out); for an undirected one every arc serves both ways.
    static __device__ __forceinline__ int avtx(int raw) { return kDir ? arc_vertex(raw) : raw; }
    static __device__ __forceinline__ bool ain(int raw) { return !kDir || raw < 0; }
    static __device__ __forceinline__ bool aout(int raw) { return !kDir || raw >= 0; }
    static constexpr bool kFloatSig = !std::is_integral<SigT>::value;
    static constexpr bool kTh32 = sizeof(ThT) == 4;
    // Path counts: stored rows are SigT (u32 exact counts, or FP64 with a
    // per-level exponent); sums and partial rows are 64-bit (a sum of at most
    // 2^31 u32 counts cannot wrap, so a count past 2^32 is caught exactly).
    using SigAcc = typename std::conditional<kFloatSig, double, unsigned long long>::type;
    // dependency accumulator: FP32 for FP32 dependencies, FP64 otherwise
    using AccT = typename std::conditional<kTh32, float, double>::type;

    const BatchArgs& a;
    Ctl* ctl;
    int lane;
    int d = 0;
    int word0 = 0;  // request mode: word slot of the current batch's first word
    bool discover_on = true;  // top-down discovery by the level's entries (off on bottom-up levels)
    uint32_t active[W];       // bits of the batch's sources (lanes with a source)
    unsigned long long* wst = nullptr;  // request mode: the block's per-word counts [W][2]
    int hoff_d = 0, nrec_d = 0, nseg_d = 0, hoff_next = 0;  // hub records of level d / d+1
    int soff_d = 0, soff_next = 0;                            // segments of level d / d+1
    int stamp_next = 0;
    bool backward = false;
    uint32_t* prev = nullptr;  // dense F_{d-1}
    uint32_t* cur = nullptr;   // dense F_d
    uint32_t* next = nullptr;  // dense F_{d+1}
    int cshift[W];             // per-source shift between level d-1 and d (forward) / d and d+1 (backward)
    int my_emax[W], my_emin[W];
    bool ovf = false;
    // Statistics live in this thread's slots of a shared-memory table (stride
    // kBatchThreads): 0 traversed (arc, source), 1 reached (vertex, source),
    // 2 entries, 3 scanned arcs, 4 DAG (arc, source) pairs.  Keeping them out
    // of registers leaves more registers to the pull's loads in flight.
    unsigned long long* sst = nullptr;
    __device__ __forceinline__ void stat(int i, unsigned long long x) { sst[i * kBatchThreads] += x; }
#ifdef SP_PROFILE
    // SM cycles by kind of work: 0-3 chunk / segment work (forward, backward),
    // 4 barrier, 5 other, 6 discovery, 7 parent/child pulls
    unsigned long long prof[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned long long prof_t = 0;
    __device__ __forceinline__ void mark(int cat) {
        const unsigned long long t = clock64();
        prof[cat] += t - prof_t;
        prof_t = t;
    }
#else
    __device__ __forceinline__ void mark(int) {}
#endif

    // Arcs whose row loads a warp issues together: chunks, and segments of long rows.
#ifndef SP_GCHUNK
#define SP_GCHUNK 8
#endif
    static constexpr int kGChunk = (SP_GCHUNK / W) > 0 ? SP_GCHUNK / W : 1;
#ifndef SP_GSEG
#define SP_GSEG 16
#endif
    static constexpr int kGSeg = (SP_GSEG / W) > 0 ? SP_GSEG / W : 1;

    __device__ BatchKernel(const BatchArgs& args) : a(args), ctl(args.ctl), lane(lane_id()) {
#pragma unroll
        for (int k = 0; k < W; ++k) { cshift[k] = 0; my_emax[k] = INT_MIN; my_emin[k] = INT_MAX; }
    }
    __device__ __forceinline__ SigT* sig() const { return reinterpret_cast<SigT*>(a.sig); }
    __device__ __forceinline__ ThT* th() const { return reinterpret_cast<ThT*>(a.th); }

    // Append vertex u to level nl of the stack; rows longer than t_hub also get
    // a hub record and one work item per segment of `seg` arcs.
    __device__ void push(int u, int nl) {
        int du = __ldg(&a.rp[u + 1]) - __ldg(&a.rp[u]);
        bool hub = du > a.t_hub;
        int pos = aggregated_slot(&ctl->qtail);
        if ((long long)pos >= a.ecap) { set_error(ctl, kErrCapEntries); return; }
        a.ent[pos] = hub ? (int)((unsigned)u | kHubFlag) : u;
        if (hub) {
            int nseg = (du + a.seg - 1) / a.seg;
            unsigned long long old = atomicAdd(&a.hcnt[nl], (1ull << 32) | (unsigned long long)(unsigned)nseg);
            int rec = hoff_next + (int)(old >> 32);
            int sb = (int)(old & 0xFFFFFFFFull);
            if (rec >= a.hcap || sb + nseg > a.segcap || (long long)soff_next + sb + nseg > a.scap) {
                set_error(ctl, kErrCapHubs);
                return;
            }
            HubRec h;
            h.v = u; h.qpos = pos; h.nseg = nseg; h.seg_base = sb;
            a.hubs[rec] = h;
            a.hdone[rec] = 0;
            a.hdone[a.hcap + rec] = 0;
            for (int q = 0; q < nseg; ++q) a.segrec[soff_next + sb + q] = rec;
        }
    }

    // Discovery of neighbour u by sources F (one lane, one arc).
    __device__ __forceinline__ void discover(int u, const uint32_t (&F)[W]) {
        uint32_t s[W];
        load_mask<W>(a.seen + (size_t)u * W, s);
        uint32_t any = 0;
        uint32_t nw[W];
#pragma unroll
        for (int k = 0; k < W; ++k) { nw[k] = F[k] & ~s[k]; any |= nw[k]; }
        if (!any) return;
        uint32_t anynew = 0;
        uint32_t* nx = next + (size_t)u * W;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            if (nw[k]) {
                uint32_t old = atomicOr(&a.seen[(size_t)u * W + k], nw[k]);
                uint32_t nb = nw[k] & ~old;
                if (nb) { atomicOr(&nx[k], nb); anynew |= nb; }
            }
        }
        if (anynew) {
            if (atomicMax(&a.ptag[u], stamp_next) < stamp_next) push(u, d + 1);
        }
    }

    // Pull over the pending arcs of one window, in lane (= CSR) order: for
    // pending lane j, every lane s with bit s of m_j set adds row[u_j][s].
    // Loads of G arcs are issued before any of them is added, so that a warp
    // keeps G*W row loads in flight.  on_owner(o) runs before the arcs of
    // entry o are added.
    template <int G, typename RowT, typename AccType, typename OnOwner>
    __device__ __forceinline__ void pull_window(const RowT* base, int u, int owner, const uint32_t (&m)[W],
                                                unsigned pend, AccType (&acc)[W], OnOwner&& on_owner) {
        // which of the lane's mask words are non-empty: words without bits
        // are skipped by the whole warp (regrouped sources leave most empty)
        uint32_t wm = 0;
#pragma unroll
        for (int k = 0; k < W; ++k) wm |= (m[k] != 0u ? 1u : 0u) << k;
        while (pend) {
            int jj[G];
#pragma unroll
            for (int i = 0; i < G; ++i) {
                jj[i] = pend ? __ffs(pend) - 1 : -1;
                pend &= pend - 1;
            }
            RowT x[G][W];
            int oi[G];
            uint32_t wi[G];
#pragma unroll
            for (int i = 0; i < G; ++i) {
                const int srcl = jj[i] >= 0 ? jj[i] : 0;
                const int ui = __shfl_sync(kFull, u, srcl);
                oi[i] = __shfl_sync(kFull, owner, srcl);
                wi[i] = __shfl_sync(kFull, wm, srcl);
                if (jj[i] < 0) wi[i] = 0u;
                const RowT* row = base + (size_t)ui * B + lane;
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    x[i][k] = (RowT)0;
                    if ((wi[i] >> k) & 1u) {
                        const uint32_t mk = __shfl_sync(kFull, m[k], srcl);
                        if ((mk >> lane) & 1u) x[i][k] = __ldcg(row + k * 32);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < G; ++i) {
                if (jj[i] < 0) break;
                on_owner(oi[i]);
#pragma unroll
                for (int k = 0; k < W; ++k)
                    if ((wi[i] >> k) & 1u) acc[k] += (AccType)x[i][k];
            }
        }
    }

    // Store the new path counts of entry (v, F) from the per-lane sums.
    __device__ __forceinline__ void sigma_flush(int v, const uint32_t (&F)[W], const SigAcc (&acc)[W]) {
#pragma unroll
        for (int k = 0; k < W; ++k) {
            if ((F[k] >> lane) & 1u) {
                size_t idx = (size_t)v * B + k * 32 + lane;
                if constexpr (kFloatSig) {
                    double val = scale2((double)acc[k], -cshift[k]);
                    if (!normal_finite(val)) set_error(ctl, SP_ERR_RANGE);
                    sig()[idx] = (SigT)val;
                    int e = exp_field(val) - 1023;
                    my_emax[k] = max(my_emax[k], e);
                    my_emin[k] = min(my_emin[k], e);
                } else {
                    if (acc[k] > 0xFFFFFFFFull) set_error(ctl, kErrSigmaOverflow);
                    sig()[idx] = (SigT)acc[k];
                }
            }
        }
    }

    // Backward: from the per-lane sums of theta over children, delta, theta(v), BC.
    // The entry's dependencies are added into BC in FP64 whatever their
    // storage precision: each lane's W values, then a fixed-order butterfly
    // over the warp.
    __device__ __forceinline__ void delta_flush(int v, const uint32_t (&F)[W], const AccT (&acc)[W]) {
        double bcsum = 0.0;
        AccT dk[W];
#pragma unroll
        for (int k = 0; k < W; ++k) {
            dk[k] = 0;
            if ((F[k] >> lane) & 1u) {
                size_t idx = (size_t)v * B + k * 32 + lane;
                SigT sv = __ldcg(&sig()[idx]);
                if constexpr (kTh32) {
                    float sf;
                    if constexpr (kFloatSig) {
                        sf = (float)sv;
                    } else {
                        sf = __uint2float_rn(sv);
                    }
                    float delta = sf * acc[k];
                    if constexpr (kFloatSig) delta = (float)scale2((double)delta, -cshift[k]);
                    float t = (1.0f + delta) / sf;
                    if (!normal_finite_f(t) || !normal_finite_f(sf)) set_error(ctl, kErrThetaRange32);
                    th()[idx] = t;
                    bcsum += (double)delta;
                    dk[k] = delta;
                } else {
                    double s = (double)sv;
                    double delta = s * acc[k];
                    if constexpr (kFloatSig) delta = scale2(delta, -cshift[k]);
                    double t = (1.0 + delta) / s;
                    if (!normal_finite(t)) set_error(ctl, SP_ERR_RANGE);
                    th()[idx] = t;
                    bcsum += delta;
                    dk[k] = delta;
                }
            }
        }
        if (a.word_bc != nullptr) {
            // request mode: each word's fixed-order sum into that word's vector
#pragma unroll
            for (int k = 0; k < W; ++k) {
                if (F[k] == 0u) continue;  // the entry's mask: the same in every lane
                const double x = warp_sum_f64((double)dk[k]);
                if (lane == 0) {
                    int ws = word0 + k;  // word0 is already a slot index
                    if (ws >= a.word_cap) ws -= a.word_cap;
                    double* p = a.word_bc + (size_t)ws * (size_t)a.n + v;
                    *p = __ldcg(p) + x;
                }
            }
            return;
        }
        // fixed-order reduction over the sources of this entry
        bcsum = warp_sum_f64(bcsum);
        if (lane == 0) a.bc[v] = __ldcg(&a.bc[v]) + bcsum;
        if (a.sq != nullptr) {  // squared dependencies (sampling bounds): only when asked for
            double sqsum = 0.0;
#pragma unroll
            for (int k = 0; k < W; ++k) sqsum += (double)dk[k] * (double)dk[k];
            sqsum = warp_sum_f64(sqsum);
            if (lane == 0) a.sq[v] = __ldcg(&a.sq[v]) + sqsum;
        }
    }

    // Request mode: per-word counts of traversed (arc, source) pairs and
    // reached (vertex, source) pairs for one entry of degree deg and mask F.
    __device__ __forceinline__ void count_words(unsigned long long deg, const uint32_t (&F)[W]) {
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const unsigned pc = __popc(F[k]);
            if (pc) {
                atomicAdd(&wst[2 * k], deg * pc);
                atomicAdd(&wst[2 * k + 1], (unsigned long long)pc);
            }
        }
    }

    // Owner lane of window position ai: the largest j with excl_j <= ai.
    __device__ __forceinline__ int owner_of(int excl, int ai) const {
        int j = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            int ex = __shfl_sync(kFull, excl, j + step < 32 ? j + step : 31);
            if (j + step < 32 && ex <= ai) j += step;
        }
        return j;
    }

    // Entry of lane (e0 + lane) if e0 + lane < qe; hub entries and entries
    // past the level come back with deg = 0.
    __device__ __forceinline__ void load_entry(int e, int qe, bool& valid, bool& hubent, int& v) const {
        valid = e < qe;
        unsigned qv = valid ? (unsigned)__ldcg(&a.ent[e]) : kHubFlag;
        hubent = (qv & kHubFlag) != 0;
        v = (int)(qv & kVertexMask);
        if (valid && v >= a.n) { set_error(ctl, kErrCorrupt); valid = false; hubent = true; v = 0; }
    }

    // ---------------- forward ----------------
    // Chunk of level-stack entries [e0, qe), at most 32.
    __device__ void fwd_chunk(int e0, int qe) {
        unsigned dag = 0;  // DAG (arc, source) pairs seen by this lane
        const int e = e0 + lane;
        bool valid, hubent;
        int v;
        load_entry(e, qe, valid, hubent, v);
        uint32_t F[W];
#pragma unroll
        for (int k = 0; k < W; ++k) F[k] = 0u;
        int beg = 0, deg = 0;
        if (valid) {
            load_mask<W>(cur + (size_t)v * W, F);
            store_mask<W>(a.emask + (size_t)e * W, F);
            stat(2, 1);
            if (!hubent) {
                beg = __ldg(&a.rp[v]);
                deg = __ldg(&a.rp[v + 1]) - beg;
                const int tdeg = kDir ? __ldg(&a.odeg[v]) : deg;  // traversed: out-arcs
                int pc = 0;
#pragma unroll
                for (int k = 0; k < W; ++k) pc += __popc(F[k]);
                stat(0, (unsigned long long)tdeg * (unsigned long long)pc);
                stat(1, (unsigned long long)pc);
                stat(3, (unsigned long long)deg);
                if (wst != nullptr) count_words((unsigned long long)tdeg, F);
            }
        }
        const int incl = warp_incl_scan(deg);
        const int excl = incl - deg;
        const int total = __shfl_sync(kFull, incl, 31);
        SigAcc acc[W];
#pragma unroll
        for (int k = 0; k < W; ++k) acc[k] = 0;
        int cur_e = -1;  // lane index of the entry whose sums are in acc
        auto flush_current = [&]() {
            if (cur_e >= 0) {
                uint32_t Fc[W];
#pragma unroll
                for (int k = 0; k < W; ++k) Fc[k] = __shfl_sync(kFull, F[k], cur_e);
                sigma_flush(__shfl_sync(kFull, v, cur_e), Fc, acc);
            }
        };
        for (int cb = 0; cb < total; cb += kWarp) {
            const int ai = cb + lane;
            const bool has = ai < total;
            const int j = owner_of(excl, ai);
            const int bj = __shfl_sync(kFull, beg, j);
            const int exj = __shfl_sync(kFull, excl, j);
            uint32_t Fj[W], m[W];
#pragma unroll
            for (int k = 0; k < W; ++k) { Fj[k] = __shfl_sync(kFull, F[k], j); m[k] = 0u; }
            int u = 0;
            if (has) {
                const int raw = __ldg(&a.ci[bj + (ai - exj)]);
                u = avtx(raw);
                if (d > 0 && ain(raw)) {
                    uint32_t p[W];
                    load_mask<W>(prev + (size_t)u * W, p);
#pragma unroll
                    for (int k = 0; k < W; ++k) { m[k] = Fj[k] & p[k]; dag += __popc(m[k]); }
                }
                mark(0);
                if (discover_on && aout(raw)) discover(u, Fj);
                mark(6);
            }
            if (d > 0) {
                uint32_t anym = 0;
#pragma unroll
                for (int k = 0; k < W; ++k) anym |= m[k];
                const unsigned pend = __ballot_sync(kFull, anym != 0u);
                mark(0);
                pull_window<kGChunk>(sig(), u, j, m, pend, acc, [&](int ej) {
                    if (ej != cur_e) {
                        flush_current();
                        cur_e = ej;
#pragma unroll
                        for (int k = 0; k < W; ++k) acc[k] = 0;
                    }
                });
                mark(7);
            }
        }
        flush_current();
        stat(4, dag);
    }

    // One segment of a long row (forward).  g: segment index within level d.
    __device__ void fwd_hub_segment(int g) {
        unsigned dag = 0;  // DAG (arc, source) pairs seen by this lane
        const int r = __ldcg(&a.segrec[soff_d + g]);
        if (r < hoff_d || r >= hoff_d + nrec_d) {
            if (lane == 0) set_error(ctl, kErrCorrupt);
            return;
        }
        const int hv = __ldcg(&a.hubs[r].v);
        const int nseg = __ldcg(&a.hubs[r].nseg);
        const int sb = __ldcg(&a.hubs[r].seg_base);
        if (hv < 0 || hv >= a.n || nseg < 1 || sb < 0 || sb + nseg > a.segcap || g < sb || g >= sb + nseg) {
            if (lane == 0) set_error(ctl, kErrCorrupt);
            return;
        }
        const int s = g - sb;
        const int rb = __ldg(&a.rp[hv]), re = __ldg(&a.rp[hv + 1]);
        const int beg = rb + s * a.seg;
        const int end = min(re, beg + a.seg);
        uint32_t F[W];
        load_mask<W>(cur + (size_t)hv * W, F);
        SigAcc acc[W];
#pragma unroll
        for (int k = 0; k < W; ++k) acc[k] = 0;
        for (int cb = beg; cb < end; cb += kWarp) {
            const int ai = cb + lane;
            const bool has = ai < end;
            uint32_t m[W];
#pragma unroll
            for (int k = 0; k < W; ++k) m[k] = 0u;
            int u = 0;
            if (has) {
                const int raw = __ldg(&a.ci[ai]);
                u = avtx(raw);
                if (d > 0 && ain(raw)) {
                    uint32_t p[W];
                    load_mask<W>(prev + (size_t)u * W, p);
#pragma unroll
                    for (int k = 0; k < W; ++k) { m[k] = F[k] & p[k]; dag += __popc(m[k]); }
                }
                mark(1);
                if (discover_on && aout(raw)) discover(u, F);
                mark(6);
            }
            if (d > 0) {
                uint32_t anym = 0;
#pragma unroll
                for (int k = 0; k < W; ++k) anym |= m[k];
                const unsigned pend = __ballot_sync(kFull, anym != 0u);
                mark(1);
                pull_window<kGSeg>(sig(), u, 0, m, pend, acc, [](int) {});
                mark(7);
            }
        }
        if (lane == 0) stat(3, (unsigned long long)(end - beg));
        stat(4, dag);
        auto count_entry = [&]() {
            if (lane == 0) {
                const int tdeg = kDir ? __ldg(&a.odeg[hv]) : re - rb;  // traversed: out-arcs
                int pc = 0;
#pragma unroll
                for (int k = 0; k < W; ++k) pc += __popc(F[k]);
                stat(0, (unsigned long long)tdeg * (unsigned long long)pc);
                stat(1, (unsigned long long)pc);
                if (wst != nullptr) count_words((unsigned long long)tdeg, F);
            }
        };
        if (nseg == 1) {  // the whole row in one segment: no partial sums
            count_entry();
            if (d > 0) sigma_flush(hv, F, acc);
            return;
        }
        SigAcc* prow = reinterpret_cast<SigAcc*>(a.part) + (size_t)g * B + lane;
#pragma unroll
        for (int k = 0; k < W; ++k) prow[k * 32] = acc[k];
        int old = 0;
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            old = atomicAdd(&a.hdone[r], 1);
        }
        old = __shfl_sync(kFull, old, 0);
        if (old != nseg - 1) return;
        __threadfence();
        // last segment: sum partial rows in segment order
        SigAcc tot[W];
#pragma unroll
        for (int k = 0; k < W; ++k) tot[k] = 0;
        for (int q = 0; q < nseg; ++q) {
            const SigAcc* pr = reinterpret_cast<const SigAcc*>(a.part) + (size_t)(sb + q) * B + lane;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                tot[k] += __ldcg(pr + k * 32);
            }
        }
        count_entry();
        if (d > 0) sigma_flush(hv, F, tot);
    }

    // Bottom-up discovery of level d+1 (direction-optimising BFS, Beamer et
    // al., SC 2012, on per-source bitmaps): each vertex of a range of 32 that
    // some source of the batch has not reached ORs the level-d masks of its
    // neighbours into its unseen bits, stopping once every unseen bit is
    // found; one lane owns the vertex (a warp for rows above 32 arcs), so its
    // seen bits, its level-(d+1) mask and its level-stack entry are written
    // without atomics.  Path counts are pulled as usual when level d+1 runs.
    __device__ void bottom_up_range(int base) {
        const int u = base + lane;
        uint32_t sn[W], unseen[W], got[W];
        uint32_t any = 0;
        int rb = 0, deg = 0;
#pragma unroll
        for (int k = 0; k < W; ++k) { sn[k] = 0u; unseen[k] = 0u; got[k] = 0u; }
        if (u < a.n) {
            load_mask<W>(a.seen + (size_t)u * W, sn);
#pragma unroll
            for (int k = 0; k < W; ++k) { unseen[k] = ~sn[k] & active[k]; any |= unseen[k]; }
            if (any) {
                rb = __ldg(&a.rp[u]);
                deg = __ldg(&a.rp[u + 1]) - rb;
            }
        }
        if (any && deg <= 32) {
            for (int e = 0; e < deg; ++e) {
                const int raw = __ldg(&a.ci[rb + e]);
                if (!ain(raw)) continue;  // only an arc into u can reach it
                uint32_t f[W];
                load_mask<W>(cur + (size_t)avtx(raw) * W, f);
                bool done = true;
#pragma unroll
                for (int k = 0; k < W; ++k) { got[k] |= f[k] & unseen[k]; done &= got[k] == unseen[k]; }
                if (done) break;
            }
        }
        unsigned big = __ballot_sync(kFull, any != 0u && deg > 32);
        while (big) {
            const int j = __ffs(big) - 1;
            big &= big - 1;
            const int bj = __shfl_sync(kFull, rb, j), dj = __shfl_sync(kFull, deg, j);
            uint32_t uns[W], g2[W];
#pragma unroll
            for (int k = 0; k < W; ++k) { uns[k] = __shfl_sync(kFull, unseen[k], j); g2[k] = 0u; }
            for (int e = lane; e < dj; e += kWarp) {
                const int raw = __ldg(&a.ci[bj + e]);
                if (!ain(raw)) continue;
                uint32_t f[W];
                load_mask<W>(cur + (size_t)avtx(raw) * W, f);
#pragma unroll
                for (int k = 0; k < W; ++k) g2[k] |= f[k] & uns[k];
            }
#pragma unroll
            for (int k = 0; k < W; ++k)
                for (int o = 16; o > 0; o >>= 1) g2[k] |= __shfl_xor_sync(kFull, g2[k], o);
            if (lane == j) {
#pragma unroll
                for (int k = 0; k < W; ++k) got[k] = g2[k];
            }
        }
        uint32_t anyg = 0;
#pragma unroll
        for (int k = 0; k < W; ++k) anyg |= got[k];
        if (anyg) {
            uint32_t ns[W];
#pragma unroll
            for (int k = 0; k < W; ++k) ns[k] = sn[k] | got[k];
            store_mask<W>(a.seen + (size_t)u * W, ns);
            store_mask<W>(next + (size_t)u * W, got);
            push(u, d + 1);
        }
    }

    // ---------------- backward ----------------
    __device__ void bwd_chunk(int e0, int qe, bool skip_arcs) {
        const int e = e0 + lane;
        bool valid, hubent;
        int v;
        load_entry(e, qe, valid, hubent, v);
        uint32_t F[W];
#pragma unroll
        for (int k = 0; k < W; ++k) F[k] = 0u;
        int beg = 0, deg = 0;
        if (valid && !hubent) {
            load_mask<W>(a.emask + (size_t)e * W, F);
            beg = __ldg(&a.rp[v]);
            deg = skip_arcs ? 0 : __ldg(&a.rp[v + 1]) - beg;
            stat(3, (unsigned long long)deg);
        }
        const int incl = warp_incl_scan(deg);
        const int excl = incl - deg;
        const int total = __shfl_sync(kFull, incl, 31);
        AccT acc[W];
#pragma unroll
        for (int k = 0; k < W; ++k) acc[k] = 0;
        // Entries are flushed in lane order; entries with no child arcs get acc = 0.
        int next_flush = 0;  // lanes below this index are flushed
        auto flush_upto = [&](int upto) {  // flush entries next_flush .. upto-1
            for (; next_flush < upto; ++next_flush) {
                const int c = next_flush;
                const bool cv = __shfl_sync(kFull, (int)(valid && !hubent), c) != 0;
                if (!cv) continue;
                uint32_t Fc[W];
#pragma unroll
                for (int k = 0; k < W; ++k) Fc[k] = __shfl_sync(kFull, F[k], c);
                delta_flush(__shfl_sync(kFull, v, c), Fc, acc);
#pragma unroll
                for (int k = 0; k < W; ++k) acc[k] = 0;
            }
        };
        for (int cb = 0; cb < total; cb += kWarp) {
            const int ai = cb + lane;
            const bool has = ai < total;
            const int j = owner_of(excl, ai);
            const int bj = __shfl_sync(kFull, beg, j);
            const int exj = __shfl_sync(kFull, excl, j);
            uint32_t m[W];
#pragma unroll
            for (int k = 0; k < W; ++k) m[k] = 0u;
            int w = 0;
            if (has) {
                const int raw = __ldg(&a.ci[bj + (ai - exj)]);
                w = avtx(raw);
                if (aout(raw)) load_mask<W>(next + (size_t)w * W, m);  // children: out-arcs
            }
            uint32_t anym = 0;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                m[k] &= __shfl_sync(kFull, F[k], j);
                anym |= m[k];
            }
            const unsigned pend = __ballot_sync(kFull, has && anym != 0u);
            mark(2);
            pull_window<kGChunk>(th(), w, j, m, pend, acc, [&](int ej) {
                if (ej > next_flush) flush_upto(ej);
            });
            mark(7);
        }
        flush_upto(32);
    }

    __device__ void bwd_hub_segment(int g, bool skip_arcs) {
        const int r = __ldcg(&a.segrec[soff_d + g]);
        if (r < hoff_d || r >= hoff_d + nrec_d) {
            if (lane == 0) set_error(ctl, kErrCorrupt);
            return;
        }
        const int hv = __ldcg(&a.hubs[r].v);
        const int qpos = __ldcg(&a.hubs[r].qpos);
        const int nseg = __ldcg(&a.hubs[r].nseg);
        const int sb = __ldcg(&a.hubs[r].seg_base);
        if (hv < 0 || hv >= a.n || nseg < 1 || sb < 0 || sb + nseg > a.segcap || qpos < 0 || qpos >= a.ecap ||
            g < sb || g >= sb + nseg) {
            if (lane == 0) set_error(ctl, kErrCorrupt);
            return;
        }
        const int s = g - sb;
        const int rb = __ldg(&a.rp[hv]), re = __ldg(&a.rp[hv + 1]);
        const int beg = rb + s * a.seg;
        const int end = skip_arcs ? beg : min(re, beg + a.seg);
        uint32_t F[W];
        load_mask<W>(a.emask + (size_t)qpos * W, F);
        AccT acc[W];
#pragma unroll
        for (int k = 0; k < W; ++k) acc[k] = 0;
        for (int cb = beg; cb < end; cb += kWarp) {
            const int ai = cb + lane;
            const bool has = ai < end;
            uint32_t m[W];
            uint32_t anym = 0;
            int w = 0;
#pragma unroll
            for (int k = 0; k < W; ++k) m[k] = 0u;
            if (has) {
                const int raw = __ldg(&a.ci[ai]);
                w = avtx(raw);
                if (aout(raw)) {  // children: out-arcs
                    uint32_t c[W];
                    load_mask<W>(next + (size_t)w * W, c);
#pragma unroll
                    for (int k = 0; k < W; ++k) { m[k] = c[k] & F[k]; anym |= m[k]; }
                }
            }
            const unsigned pend = __ballot_sync(kFull, anym != 0u);
            mark(3);
            pull_window<kGSeg>(th(), w, 0, m, pend, acc, [](int) {});
            mark(7);
        }
        if (lane == 0) stat(3, (unsigned long long)(end - beg));
        if (nseg == 1) {
            delta_flush(hv, F, acc);
            return;
        }
        AccT* prow = reinterpret_cast<AccT*>(a.part) + (size_t)g * B + lane;
#pragma unroll
        for (int k = 0; k < W; ++k) prow[k * 32] = acc[k];
        int old = 0;
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            old = atomicAdd(&a.hdone[a.hcap + r], 1);
        }
        old = __shfl_sync(kFull, old, 0);
        if (old != nseg - 1) return;
        __threadfence();
        AccT tot[W];
#pragma unroll
        for (int k = 0; k < W; ++k) tot[k] = 0;
        for (int q = 0; q < nseg; ++q) {
            const AccT* pr = reinterpret_cast<const AccT*>(a.part) + (size_t)(sb + q) * B + lane;
#pragma unroll
            for (int k = 0; k < W; ++k) tot[k] += __ldcg(pr + k * 32);
        }
        delta_flush(hv, F, tot);
    }

    // Per-block reduction of the level's sigma exponent range, then one
    // global atomic per source and block.
    __device__ void flush_exponents(int level) {
        if constexpr (kFloatSig) {
            __shared__ int s_max[B], s_min[B];
            for (int i = threadIdx.x; i < B; i += blockDim.x) { s_max[i] = INT_MIN; s_min[i] = INT_MAX; }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < W; ++k) {
                if (my_emax[k] >= my_emin[k]) {
                    atomicMax(&s_max[k * 32 + lane], my_emax[k]);
                    atomicMin(&s_min[k * 32 + lane], my_emin[k]);
                }
                my_emax[k] = INT_MIN;
                my_emin[k] = INT_MAX;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < B; i += blockDim.x) {
                if (s_max[i] >= s_min[i]) {
                    atomicMax(&a.emax[(size_t)level * B + i], s_max[i]);
                    atomicMin(&a.emin[(size_t)level * B + i], s_min[i]);
                }
            }
        }
    }
};

// Live feed (serving), kept out of line so that the batched kernel's register
// allocation does not see them.  live_ready: the requests from r0 on whose
// words all lie below word wend, [r0, result).  live_sum: each such request's
// BC as its words' partial vectors summed in word order, the slots cleared for
// the words that reuse them.  live_mark (one thread, after a grid barrier):
// the requests' counts, then done, and the launch's finished-request count.
// live_snapshot (every thread of block 0): the words and requests published
// since the last look, their lanes and records copied to device memory (so
// that the other blocks read no host memory), then the counts.
static __device__ __noinline__ void live_snapshot(const FeedCtl* feed, const int32_t* h_lanes, const FeedReq* h_req,
                                                  int32_t* lanes, FeedReq* req, int word_cap, int req_cap, Ctl* ctl) {
    __shared__ int s_w[2];
    if (threadIdx.x == 0) {
        s_w[0] = ld_acquire_sys_i32(&feed->words);
        s_w[1] = ld_volatile(&feed->nreq);
    }
    __syncthreads();
    const int w1 = s_w[0], r1 = s_w[1];
    const int w0 = ld_volatile(&ctl->live_words), r0 = ld_volatile(&ctl->live_nreq);
    for (int i = threadIdx.x; i < (w1 - w0) * 32; i += blockDim.x) {
        const size_t at = (size_t)((w0 + i / 32) % word_cap) * 32 + (size_t)(i & 31);
        lanes[at] = ld_volatile(&h_lanes[at]);
    }
    for (int r = r0 + (int)threadIdx.x; r < r1; r += blockDim.x) {
        const FeedReq* src = h_req + (r % req_cap);
        FeedReq* dst = req + (r % req_cap);
        dst->first_word = ld_volatile(&src->first_word);
        dst->nwords = ld_volatile(&src->nwords);
        dst->out = ld_volatile(&src->out);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl->live_words = w1;
        ctl->live_nreq = r1;
    }
}
static __device__ __noinline__ int live_ready(const FeedReq* req, int req_cap, int r0, int nreq, int wend) {
    int r1 = r0;
    while (r1 < nreq) {
        const FeedReq* fr = req + (r1 % req_cap);
        if (ld_volatile(&fr->first_word) + ld_volatile(&fr->nwords) > wend) break;
        ++r1;
    }
    return r1;
}
static __device__ __noinline__ void live_sum(const FeedReq* req, int req_cap, double* word_bc, int word_cap, int n,
                                             int r0, int r1, int tid, int nthr) {
    for (int r = r0; r < r1; ++r) {
        const FeedReq* fr = req + (r % req_cap);
        const int fw = ld_volatile(&fr->first_word), nw = ld_volatile(&fr->nwords);
        double* out = ld_volatile(&fr->out);
        const int s0 = fw % word_cap;
        for (int v = tid; v < n; v += nthr) {
            double sum = 0.0;
            for (int k = 0, ws = s0; k < nw; ++k, ws = ws + 1 == word_cap ? 0 : ws + 1) {
                double* p = word_bc + (size_t)ws * (size_t)n + v;
                sum += __ldcg(p);
                *p = 0.0;
            }
            out[v] = sum;
        }
    }
}
static __device__ __noinline__ void live_mark(const FeedReq* req, FeedReq* h_req, int req_cap,
                                              unsigned long long* word_stats, int word_cap, Ctl* ctl, int r0, int r1) {
    for (int r = r0; r < r1; ++r) {
        const FeedReq* dr = req + (r % req_cap);
        FeedReq* fr = h_req + (r % req_cap);
        const int fw = ld_volatile(&dr->first_word), nw = ld_volatile(&dr->nwords);
        unsigned long long tr = 0, re = 0;
        for (int k = 0; k < nw; ++k) {
            unsigned long long* q = word_stats + 2 * (size_t)((fw + k) % word_cap);
            tr += q[0];
            re += q[1];
            q[0] = 0ull;
            q[1] = 0ull;
        }
        fr->traversed = tr;
        fr->reached = re;
        __threadfence_system();
        st_release_sys_i32(&fr->done, 1);
    }
    ctl->live_req_done = r1;
}

template <int W, typename SigT, typename ThT, bool kDir>
__global__ void __launch_bounds__(kBatchThreads, SP_BATCH_MINB) batched_kernel(BatchArgs a) {
    if (a.pre_err != nullptr) {  // the same word for every block: all return, nothing is touched
        const int pe = ld_volatile(a.pre_err);
        if (pe != 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->err = pe;
            return;
        }
    }
    using K_t = BatchKernel<W, SigT, ThT, kDir>;
    constexpr int B = K_t::B;
    constexpr bool kFloatSig = K_t::kFloatSig;
    K_t K(a);
    __shared__ unsigned long long s_tstat[5 * kBatchThreads];
#pragma unroll
    for (int i = 0; i < 5; ++i) s_tstat[i * kBatchThreads + threadIdx.x] = 0ull;
    K.sst = s_tstat + threadIdx.x;
    __shared__ unsigned long long s_wst[2 * 8];
    if (a.word_stats != nullptr) {
        if (threadIdx.x < 2 * W) s_wst[threadIdx.x] = 0ull;
        K.wst = s_wst;
    }
    Ctl* ctl = a.ctl;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = gridDim.x * blockDim.x;
    const int lane = K.lane;
    const int n = a.n;
    int phase = 0;
    int qsnap = 0;  // level-stack fill at the last barrier
    int levels_max = 0;
    int stamp_base = 1;
#ifdef SP_PROFILE
    K.prof_t = clock64();
#endif
#define SP_PROF_MARK(cat) K.mark(cat)
    auto sync = [&]() -> bool {
        bool skip = (a.debug_flags & SP_DEBUG_SKIP_BARRIER) && blockIdx.x == 0 && phase == 1;
        SP_PROF_MARK(5);
        bool ok = grid_sync(ctl, gridDim.x, a.timeout_ns, phase++, skip, &qsnap);
        SP_PROF_MARK(4);
#ifdef SP_PROFILE
        if (tid == 0 && phase < 256) ctl->phase_ns[phase] = globaltimer();
#endif
        if (tid == 0) ctl->work[(phase + 2) & 3] = 0u;
        return ok;
    };
    // Work loop of one level: hub segments first, then chunks of 32 entries.
    // Warp w takes item w first and further items from a shared counter, so a
    // level with fewer items than warps costs no atomics.
    const int nwarps = nthr / kWarp;
    const int gwarp = tid / kWarp;
    auto work = [&](int nitems_hub, int qb, int qe, auto&& on_hub, auto&& on_chunk, int bu_items = 0) {
        const int c = entries_per_item(qe - qb, nwarps);
        const int nchunks = (qe - qb + c - 1) / c;
        const int total = nitems_hub + nchunks + bu_items;
        for (int item = gwarp; item < total;) {
            SP_PROF_MARK(5);
            if (item < nitems_hub) {
                on_hub(item);
                SP_PROF_MARK(K.d >= 0 && !K.backward ? 1 : 3);
            } else if (item < nitems_hub + nchunks) {
                const int e0 = qb + (item - nitems_hub) * c;
                on_chunk(e0, min(e0 + c, qe));
                SP_PROF_MARK(K.d >= 0 && !K.backward ? 0 : 2);
            } else {
                K.bottom_up_range((item - nitems_hub - nchunks) * kWarp);
                SP_PROF_MARK(6);
            }
            if (nwarps >= total) break;
            int next = 0;
            if (lane == 0) next = nwarps + (int)atomicAdd(&ctl->work[phase & 3], 1u);
            item = __shfl_sync(kFull, next, 0);
        }
    };

    if (a.word_bc == nullptr)
        for (int i = tid; i < n; i += nthr) a.bc[i] = 0.0;
    if (a.sq != nullptr)
        for (int i = tid; i < n; i += nthr) a.sq[i] = 0.0;
    if (a.feed != nullptr && blockIdx.x == 0)  // live feed: the words and requests there are now
        live_snapshot(a.feed, a.feed_lanes, a.feed_req, const_cast<int32_t*>(a.sources), a.req_dev, a.word_cap,
                      a.req_cap, ctl);
    if (!sync()) goto out;

    for (int b0 = 0, nb = 0;; b0 += nb) {
        if (a.feed != nullptr) {  // the next min(W, available) words
            const int avail = ld_volatile(&ctl->live_words);
            if ((b0 >> 5) >= avail) break;
            nb = min(W, avail - (b0 >> 5)) * 32;
        } else {
            if (b0 >= a.nsrc) break;
            nb = min(B, a.nsrc - b0);
        }
        // source of lane sl of this batch (-1: none); live feeds keep their
        // lanes in word slots that the host refills
        auto source_of = [&](int sl) -> int {
            if (a.feed == nullptr) return __ldg(&a.sources[b0 + sl]);
            const int w = (b0 + sl) >> 5;
            return __ldcg(&a.sources[(size_t)(w % a.word_cap) * 32 + (sl & 31)]);
        };
        // ---- init: sources of this batch at level 0 ----
        K.hoff_next = 0;
        K.soff_next = 0;
        K.stamp_next = stamp_base;
        K.d = -1;
        if (tid == 0) {
            a.hcnt[1] = 0ull;
            a.eoff[0] = 0;
            a.hoff[0] = 0;
            a.soff[0] = 0;
        }
        if constexpr (kFloatSig) {
            for (int i = tid; i < B; i += nthr) {
                a.emax[i] = 0;
                a.emin[i] = 0;
                a.emax[B + i] = INT_MIN;
                a.emin[B + i] = INT_MAX;
            }
        }
        K.word0 = a.word_cap > 0 ? (b0 >> 5) % a.word_cap : 0;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const int sl = k * 32 + lane;
            K.active[k] = __ballot_sync(kFull, sl < nb && source_of(sl) >= 0);
        }
        if (tid < nb && source_of(tid) >= 0) {  // request mode leaves empty lanes (-1)
            const int s = tid;
            const int x = source_of(s);
            const uint32_t bit = 1u << (s & 31);
            atomicOr(&a.seen[(size_t)x * W + (s >> 5)], bit);
            atomicOr(&a.dense[(size_t)x * W + (s >> 5)], bit);  // ring 0 = F_0
            K.sig()[(size_t)x * B + s] = (SigT)1;
            if (atomicMax(&a.ptag[x], stamp_base) < stamp_base) K.push(x, 0);
        }
        if (!sync()) goto out;

        // ---- forward ----
        int qb = 0, qe = qsnap;
        int hoff_d = 0, soff_d = 0;
        int d = 0;
        while (true) {
            K.d = d;
            K.prev = a.dense + (size_t)((d + 3) & 3) * n * W;
            K.cur = a.dense + (size_t)(d & 3) * n * W;
            K.next = a.dense + (size_t)((d + 1) & 3) * n * W;
            K.stamp_next = stamp_base + d + 1;
            unsigned long long hc = ld_volatile(&a.hcnt[d]);
            K.hoff_d = hoff_d;
            K.soff_d = soff_d;
            K.nrec_d = (int)(hc >> 32);
            K.nseg_d = (int)(hc & 0xFFFFFFFFull);
            K.hoff_next = hoff_d + K.nrec_d;
            K.soff_next = soff_d + K.nseg_d;
            if (d + 2 >= a.lcap) { set_error(ctl, kErrCapLevels); }
            if constexpr (kFloatSig) {
#pragma unroll
                for (int k = 0; k < W; ++k)
                    K.cshift[k] = d > 0 ? centre_shift(ld_volatile(&a.emax[(size_t)(d - 1) * B + k * 32 + lane]),
                                                       ld_volatile(&a.emin[(size_t)(d - 1) * B + k * 32 + lane]),
                                                       a.centre_bound)
                                        : 0;
                if (blockIdx.x == 0 && threadIdx.x < 32) {  // one warp counts the recentred (level, source) pairs
                    int nrec = 0;
#pragma unroll
                    for (int k = 0; k < W; ++k) nrec += __popc(__ballot_sync(kFull, K.cshift[k] != 0) & K.active[k]);
                    if (lane == 0 && nrec) atomicAdd(&ctl->recentred, (unsigned long long)nrec);
                }
                if (d + 1 < a.lcap)
                    for (int i = tid; i < B; i += nthr) {
                        a.emax[(size_t)(d + 1) * B + i] = INT_MIN;
                        a.emin[(size_t)(d + 1) * B + i] = INT_MAX;
                    }
            }
            if (tid == 0) {
                a.eoff[d + 1] = qe;
                a.hoff[d] = hoff_d;
                a.soff[d] = soff_d;
                if (d + 2 < a.lcap + 2) a.hcnt[d + 2] = 0ull;
            }
            // clear dense F_{d-2}
            if (d >= 2) {
                const int cb = ld_volatile(&a.eoff[d - 2]), ce = ld_volatile(&a.eoff[d - 1]);
                uint32_t* clr = a.dense + (size_t)((d + 2) & 3) * n * W;
                for (int i = cb + tid; i < ce; i += nthr) {
                    int v = (int)((unsigned)__ldcg(&a.ent[i]) & kVertexMask);
                    zero_mask<W>(clr + (size_t)v * W);
                }
            }
            // Direction: levels with many entries discover bottom-up.
            const bool bu = a.bu_den > 0 && d > 0 && (int64_t)(qe - qb) * a.bu_den > (int64_t)n;
            K.discover_on = !bu;
            work(K.nseg_d, qb, qe, [&](int g) { K.fwd_hub_segment(g); }, [&](int e0, int e1) { K.fwd_chunk(e0, e1); },
                 bu ? (n + kWarp - 1) / kWarp : 0);
            K.discover_on = true;
            K.flush_exponents(d);
            if (!sync()) goto out;
            const int nq = qsnap;
            hoff_d = K.hoff_next;
            soff_d = K.soff_next;
            if (nq == qe) break;
            qb = qe;
            qe = nq;
            ++d;
        }
        const int L = d + 1;
        levels_max = max(levels_max, L);

        // ---- backward ----
        K.backward = true;
        for (int dd = L - 1; dd >= 1; --dd) {
            K.d = dd;
            K.next = a.dense + (size_t)((dd + 1) & 3) * n * W;  // dense F_{dd+1}
            const int qbd = ld_volatile(&a.eoff[dd]), qed = ld_volatile(&a.eoff[dd + 1]);
            unsigned long long hc = ld_volatile(&a.hcnt[dd]);
            K.hoff_d = ld_volatile(&a.hoff[dd]);
            K.soff_d = ld_volatile(&a.soff[dd]);
            K.nrec_d = (int)(hc >> 32);
            K.nseg_d = (int)(hc & 0xFFFFFFFFull);
            if constexpr (kFloatSig) {
#pragma unroll
                for (int k = 0; k < W; ++k)
                    K.cshift[k] = centre_shift(ld_volatile(&a.emax[(size_t)dd * B + k * 32 + lane]),
                                               ld_volatile(&a.emin[(size_t)dd * B + k * 32 + lane]), a.centre_bound);
            }
            // scatter F_dd into its dense ring slot (read by level dd-1), clear F_{dd+2},
            // and clear seen of this level's vertices
            {
                uint32_t* dst = a.dense + (size_t)(dd & 3) * n * W;
                for (int i = qbd + tid; i < qed; i += nthr) {
                    int v = (int)((unsigned)__ldcg(&a.ent[i]) & kVertexMask);
                    uint32_t msk[W];
                    load_mask<W>(a.emask + (size_t)i * W, msk);
                    store_mask<W>(dst + (size_t)v * W, msk);
                    zero_mask<W>(a.seen + (size_t)v * W);
                }
                if (dd + 2 <= L - 1) {
                    const int cb = ld_volatile(&a.eoff[dd + 2]), ce = ld_volatile(&a.eoff[dd + 3]);
                    uint32_t* clr = a.dense + (size_t)((dd + 2) & 3) * n * W;
                    for (int i = cb + tid; i < ce; i += nthr) {
                        int v = (int)((unsigned)__ldcg(&a.ent[i]) & kVertexMask);
                        zero_mask<W>(clr + (size_t)v * W);
                    }
                }
            }
            const bool skip = dd == L - 1;
            work(K.nseg_d, qbd, qed, [&](int g) { K.bwd_hub_segment(g, skip); },
                 [&](int e0, int e1) { K.bwd_chunk(e0, e1, skip); });
            if (!sync()) goto out;
        }

        K.backward = false;
        if (a.word_stats != nullptr) {  // this batch's per-word counts
            __syncthreads();
            if (threadIdx.x < 2 * W) {
                int ws = K.word0 + (int)(threadIdx.x >> 1);
                if (ws >= a.word_cap) ws -= a.word_cap;
                if (s_wst[threadIdx.x]) atomicAdd(&a.word_stats[2 * (size_t)ws + (threadIdx.x & 1)], s_wst[threadIdx.x]);
                s_wst[threadIdx.x] = 0ull;
            }
            __syncthreads();
        }
        if (a.feed != nullptr && blockIdx.x == 0)  // what the feed holds now, for the next batch
            live_snapshot(a.feed, a.feed_lanes, a.feed_req, const_cast<int32_t*>(a.sources), a.req_dev, a.word_cap,
                          a.req_cap, ctl);
        // ---- cleanup: dense levels 0..2, seen of the sources; reset the stack ----
        for (int j = 0; j < 3 && j < L; ++j) {
            const int cb = ld_volatile(&a.eoff[j]), ce = ld_volatile(&a.eoff[j + 1]);
            uint32_t* clr = a.dense + (size_t)(j & 3) * n * W;
            for (int i = cb + tid; i < ce; i += nthr) {
                int v = (int)((unsigned)__ldcg(&a.ent[i]) & kVertexMask);
                zero_mask<W>(clr + (size_t)v * W);
                if (j == 0) zero_mask<W>(a.seen + (size_t)v * W);
            }
        }
        if (tid == 0) {
            ctl->qtail = 0;
            a.hcnt[0] = 0ull;
        }
        stamp_base += L + 1;
        if (!sync()) goto out;
        if (a.feed != nullptr) {
            // ---- live feed: finish the requests whose words are all done ----
            const int wend = (b0 + nb) >> 5;
            const int r0 = ld_volatile(&ctl->live_req_done);
            const int r1 = live_ready(a.req_dev, a.req_cap, r0, ld_volatile(&ctl->live_nreq), wend);
            if (r1 > r0) {
                live_sum(a.req_dev, a.req_cap, a.word_bc, a.word_cap, n, r0, r1, tid, nthr);
                if (!sync()) goto out;
                if (tid == 0) live_mark(a.req_dev, a.feed_req, a.req_cap, a.word_stats, a.word_cap, ctl, r0, r1);
            }
            if (tid == 0) st_release_sys_i32(&a.feed->ran_words, wend);
        }
    }
    if (a.feed != nullptr && tid == 0 && ld_volatile(&ctl->err) == 0) st_release_sys_i32(&a.feed->closed, 1);

out:
    {
        __shared__ unsigned long long s_st[5];
        if (threadIdx.x == 0) { s_st[0] = 0; s_st[1] = 0; s_st[2] = 0; s_st[3] = 0; s_st[4] = 0; }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 5; ++i) atomicAdd(&s_st[i], s_tstat[i * kBatchThreads + threadIdx.x]);
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicAdd(&ctl->traversed_arcs, s_st[0]);
            atomicAdd(&ctl->reached, s_st[1]);
            atomicAdd(&ctl->entries, s_st[2]);
            atomicAdd(&ctl->scanned_arcs, s_st[3]);
            atomicAdd(&ctl->dag_arcs, s_st[4]);
            atomicMax(&ctl->max_levels, levels_max);
        }
#ifdef SP_PROFILE
        if ((threadIdx.x & 31) == 0)
            for (int c = 0; c < 8; ++c) atomicAdd(&ctl->prof[c], K.prof[c]);
#endif
    }
}

// Host side: workspace layout and launch for one width.
template <int W>
sp_status launch_batched_w(const BatchedLaunch& L, LaunchResult* result);

}  // namespace sp
