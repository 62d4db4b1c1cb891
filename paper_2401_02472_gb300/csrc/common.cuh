// Shared device-side machinery of the starbc kernels: the launch control
// block, a grid barrier whose waits give up after a deadline, warp helpers and
// exact power-of-two scaling written from the IEEE-754 binary64 layout.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "starbc.h"

namespace sp {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kWarp = 32;
constexpr uint32_t kHubFlag = 0x80000000u;  // marks a level-stack entry processed in segments
constexpr uint32_t kVertexMask = 0x7FFFFFFFu;

// Internal error codes (never returned to callers as such).
constexpr int kErrSigmaOverflow = -100;   // exact integer path counts overflowed 64 bits
constexpr int kErrThetaRange32 = -101;    // a 1/sigma-scaled dependency left the FP32 normal range
constexpr int kErrCapacity = -102;        // a level-stack or hub buffer was too small
constexpr int kErrCapEntries = -103;      // batched level stack full
constexpr int kErrCapHubs = -104;         // batched hub list full
constexpr int kErrCapLevels = -105;       // more BFS levels than the batched form holds
constexpr int kErrCorrupt = -106;         // an index read from device state was out of range

// One per launch, in device memory, zeroed by the host before the launch.
struct Ctl {
    unsigned int bar_count;
    unsigned int bar_gen;
    int err;                         // first error (sp_status or internal code), 0 = none
    int err_where;                   // phase at which a barrier timed out
    unsigned int work[4];            // per-phase work counters, ring of 4
    int qtail;                       // level-stack fill (entries)
    int pad0;
    unsigned long long hctr[4];      // per-level hub counters (records << 32 | segments), ring of 4
    int levels_out;                  // L of the last source / batch
    int pad1;
    // statistics (accumulated over the launch)
    unsigned long long traversed_arcs;
    unsigned long long reached;
    unsigned long long entries;
    unsigned long long scanned_arcs;
    unsigned long long dag_arcs;     // (arc, source) pairs on shortest-path DAGs
    unsigned long long recentred;    // (level, source) pairs whose FP64 path counts were recentred
    int max_levels;
    unsigned int timeout_count;      // arrivals seen by the first wait that timed out
    int snap[2];                     // qtail as the last block found it, per barrier parity
    unsigned long long prof[8];      // SP_PROFILE builds: SM cycles by kind of work, summed over warps
    unsigned long long phase_ns[256];  // SP_PROFILE builds: %globaltimer at each of the first barriers
    int block_phase[1024];           // last barrier each block arrived at (diagnostics)
    // live feed (serving): the words and requests the launch may take, as
    // block 0 last read them from the feed; requests finished so far
    int live_words, live_nreq, live_req_done, pad2;
};

// Serving: a batched launch that keeps taking requests on its graph between
// batches.  Both structs live in mapped pinned host memory.  The host writes
// a request's lanes (one source per lane, -1 for empty lanes, in word slots
// word % word_cap) and its FeedReq (slot r % req_cap), then nreq, then words
// (release); the kernel reads words (acquire) and nreq at the end of each
// batch, runs the next batch of words, and finishes every request whose words
// are all done: its BC vector is the sum of its words' partial vectors in
// word order, written to out, and then done is set (release).
struct FeedReq {
    int32_t first_word;                 // host: global index of the request's first word
    int32_t nwords;                     // host
    double* out;                        // host: the request's BC vector (device memory, n doubles)
    unsigned long long traversed;       // device: (arc, source) pairs of the request's words
    unsigned long long reached;         // device: (vertex, source) pairs
    int32_t done;                       // device: 1 once out and the counts are complete
    int32_t pad;
};
struct FeedCtl {
    int32_t words;      // host: words appended so far
    int32_t nreq;       // host: requests appended so far (written before words)
    int32_t ran_words;  // device: words of the batches finished so far
    int32_t closed;     // device: 1 once the launch has taken its last batch
};
__device__ __forceinline__ int ld_acquire_sys_i32(const int* p) {
    int v;
    asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys_i32(int* p, int v) {
    asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Directed graphs: the kernels read a combined CSR whose row v lists v's
// out-arcs and then its in-arcs, an in-arc's column id tagged with the top
// bit.  arc_vertex strips the tag.  An untagged arc leads out of v (discovery
// and the backward sum over children); an arc leads into v (the forward sum
// over parents, bottom-up discovery) when it is tagged or when the graph is
// undirected, whose untagged arcs serve both ways.
constexpr int kArcVertex = 0x7FFFFFFF;
__device__ __forceinline__ int arc_vertex(int raw) { return raw & kArcVertex; }
__device__ __forceinline__ bool arc_out(int raw) { return raw >= 0; }
__device__ __forceinline__ bool arc_in(int raw, bool directed) { return !directed || raw < 0; }

struct HubRec {
    int32_t v;        // vertex id
    int32_t qpos;     // its index in the level stack
    int32_t nseg;     // number of adjacency segments
    int32_t seg_base; // first segment index of this hub within its level
};

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
template <typename T>
__device__ __forceinline__ T ld_volatile(const T* p) {
    return *const_cast<const volatile T*>(p);
}

__device__ __forceinline__ void set_error(Ctl* ctl, int code) { atomicCAS(&ctl->err, 0, code); }

// Grid-wide barrier for a co-resident (cooperative) grid.  Each wait gives up
// after timeout_ns and records SP_ERR_TIMEOUT; a block that sees an error
// anywhere leaves at once.  Returns false when the launch must stop.
// Lane 0 of warp 0 arrives and waits; the rest of warp 0 waits for it at
// __syncwarp() so that the warp is converged again before the block barrier
// (a block barrier reached by part of a warp does not hold the other lanes).
// The last block to arrive copies ctl->qtail into a snapshot before it
// releases the others: blocks that pass first start the next phase (and push
// to qtail) while slower ones are still leaving, so qtail itself must not be
// read after the barrier.  *qtail_snap receives the snapshot in every thread.
static __device__ __noinline__ bool grid_sync(Ctl* ctl, unsigned nblocks, uint64_t timeout_ns, int phase, bool skip,
                                              int* qtail_snap) {
    __shared__ int s_ok, s_snap;
    __syncthreads();
    if (threadIdx.x < 32) {
        if (threadIdx.x == 0) {
            int ok = skip ? 0 : 1;  // a skipping block (fault injection) leaves without arriving
            int snapv = 0;
            if (!skip) {
                unsigned gen = ld_acquire_u32(&ctl->bar_gen);
                if (blockIdx.x < 1024) ctl->block_phase[blockIdx.x] = phase;
                __threadfence();
                unsigned arrived = atomicAdd(&ctl->bar_count, 1u);
                if (arrived == nblocks - 1) {
                    ctl->snap[gen & 1u] = ld_volatile(&ctl->qtail);
                    ctl->bar_count = 0;
                    st_release_u32(&ctl->bar_gen, gen + 1);
                } else {
                    uint64_t t0 = globaltimer();
                    unsigned ns = 32;
                    while (ld_acquire_u32(&ctl->bar_gen) == gen) {
                        if (ld_volatile(&ctl->err) != 0) { ok = 0; break; }
                        if (globaltimer() - t0 > timeout_ns) {
                            if (atomicCAS(&ctl->err, 0, (int)SP_ERR_TIMEOUT) == 0) {
                                ctl->err_where = phase;
                                ctl->timeout_count = ld_volatile(&ctl->bar_count);
                            }
                            ok = 0;
                            break;
                        }
                        __nanosleep(ns);
                        if (ns < 512) ns <<= 1;
                    }
                }
                __threadfence();
                snapv = ld_volatile(&ctl->snap[gen & 1u]);
            }
            __threadfence();
            if (ld_volatile(&ctl->err) != 0) ok = 0;
            if (skip) ok = 0;
            s_ok = ok;
            s_snap = snapv;
        }
        __syncwarp();
    }
    __syncthreads();
    *qtail_snap = s_snap;
    return s_ok != 0;
}

// ---- exact power-of-two scaling (IEEE-754 binary64 exponent field) ----
__device__ __forceinline__ double pow2i(int k) {  // 2^k, -1022 <= k <= 1023
    return __longlong_as_double((long long)(k + 1023) << 52);
}
__device__ __forceinline__ double scale2(double x, int k) {  // x * 2^k, |k| <= 2044
    if (k > 1023) { x *= pow2i(1023); k -= 1023; }
    else if (k < -1022) { x *= pow2i(-1022); k += 1022; }
    return x * pow2i(k);
}
// Biased exponent field; 0 means zero/subnormal, 0x7FF infinity/NaN.
__device__ __forceinline__ int exp_field(double x) {
    return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}
__device__ __forceinline__ bool normal_finite(double x) {
    int f = exp_field(x);
    return f != 0 && f != 0x7FF;
}
__device__ __forceinline__ bool normal_finite_f(float x) {
    int f = (__float_as_int(x) >> 23) & 0xFF;
    return f != 0 && f != 0xFF;
}
// Per-level recentring of scaled path counts: with the level's largest and
// smallest unbiased exponents, shift only when the level strays from 2^0 by
// more than 2^bound, and then centre it.  0 shift keeps values bit-identical
// to unscaled FP64 arithmetic.
__device__ __forceinline__ int centre_shift(int emax, int emin, int bound) {
    if (emax < emin) return 0;  // empty level
    if (emax <= bound && emin >= -bound) return 0;
    return (emax + emin) >> 1;
}

// Unsigned 64-bit integer to float, round to nearest even, from the IEEE-754
// binary32 layout (integer pipe only).
__device__ __forceinline__ float u64_to_f32(unsigned long long x) {
    if (x == 0ull) return 0.0f;
    int lz = __clzll(x);
    int e = 63 - lz;                        // x in [2^e, 2^(e+1))
    unsigned long long norm = x << lz;      // leading one at bit 63
    unsigned mant = (unsigned)(norm >> 40); // 24 bits incl. the leading one
    unsigned long long rest = norm & ((1ull << 40) - 1);
    const unsigned long long half = 1ull << 39;
    if (rest > half || (rest == half && (mant & 1u))) {
        mant += 1u;
        if (mant == (1u << 24)) { mant >>= 1; e += 1; }
    }
    unsigned bits = ((unsigned)(e + 127) << 23) | (mant & 0x7FFFFFu);
    return __int_as_float((int)bits);
}

// ---- warp helpers ----
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ unsigned long long shfl_u64(unsigned mask, unsigned long long v, int src) {
    unsigned lo = __shfl_sync(mask, (unsigned)v, src), hi = __shfl_sync(mask, (unsigned)(v >> 32), src);
    return ((unsigned long long)hi << 32) | lo;
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += shfl_u64(kFull, v, lane_id() ^ o);
    return v;
}
// Butterfly sum: every lane ends with the same, order-fixed result.
__device__ __forceinline__ double warp_sum_f64(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum_f32(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ int warp_sum_i32(int v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ int warp_max_i32(int v) {
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ int warp_min_i32(int v) {
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
// Level-stack entries per work item: 32 (one per lane), or fewer when the
// level holds fewer than 32 entries per warp, so that a small level is spread
// over more warps and its slowest item (the level's critical path) is short.
__device__ __forceinline__ int entries_per_item(int entries, int nwarps) {
    const int c = (entries + nwarps - 1) / max(nwarps, 1);
    return c >= 32 ? 32 : (c < 1 ? 1 : c);
}

// Inclusive prefix sum over the warp.
__device__ __forceinline__ int warp_incl_scan(int v) {
    int lane = lane_id();
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Append the calling lanes' vertices to a list with one atomic per converged
// group of lanes.  Returns the slot index of the calling lane.
__device__ __forceinline__ int aggregated_slot(int* tail) {
    unsigned m = __activemask();
    int lane = lane_id();
    int leader = __ffs(m) - 1;
    int rank = __popc(m & ((1u << lane) - 1u));
    int base = 0;
    if (lane == leader) base = atomicAdd(tail, __popc(m));
    base = __shfl_sync(m, base, leader);
    return base + rank;
}

// Find the hub record whose segment range holds segment g (records sorted by
// seg_base).  Records [lo, hi).
__device__ __forceinline__ int find_hub(const HubRec* hubs, int lo, int hi, int g) {
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldcg(&hubs[mid].seg_base) <= g) lo = mid; else hi = mid;
    }
    return lo;
}

}  // namespace sp
