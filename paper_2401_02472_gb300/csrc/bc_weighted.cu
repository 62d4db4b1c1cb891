// Weighted form: BC under positive integer arc weights, one block per source.
//
// The ComputeBC program (paper Section 2, Fig. 1) with its BFS replaced by
// shortest distances under the weights, which the paper's SSSP program
// computes with the Min construct (Section 3.5: relax dist[nbr] through
// dist[v] + weight with atomicMin and mark the neighbour modified).  Per
// source a block runs, with __syncthreads as its only barrier:
//
//   distances  near-far frontier rounds (Davidson et al., IPDPS 2014): the
//              vertices whose distance fell below a threshold T in the last
//              round relax their arcs with atomicMin and join the next round
//              once (a round stamp); a vertex whose new distance is at least T
//              goes to a far pile instead (once, a flag).  When no near vertex
//              is left, T moves to the smallest far distance + delta (see
//              set_weights) and the far vertices below it become the
//              next near frontier.  A vertex is expanded at most once per
//              distance it takes; the first arrival at a vertex lists it as
//              reached
//   order      a counting sort of the reached vertices by distance, then the
//              boundaries of the runs of equal distance (the "levels")
//   sigma      level by level in increasing distance: sigma(v) = sum over
//              arcs (u, v) with dist(u) + w = dist(v) of sigma(u), in v's row
//              order (every such u lies on an earlier level: w >= 1)
//   delta      level by level in decreasing distance: theta(x) = (1 +
//              delta(x)) / sigma(x); delta(v) = sigma(v) * sum over arcs
//              (v, x) with dist(v) + w = dist(x) of theta(x); BC(v) += delta(v)
//
// Blocks take sources blockIdx.x, blockIdx.x + gridDim.x, ... and keep their
// own state and partial BC row in global memory; the rows are added in block
// order afterwards.  Every per-vertex sum has a fixed order, so results are
// bit-identical from run to run.  Path counts and dependencies are FP64;
// a count outside the FP64 range stops the call with SP_ERR_RANGE.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>

#include "common.cuh"
#include "internal.h"

namespace sp {
namespace {

#ifndef SP_W_THREADS
#define SP_W_THREADS 1024  // threads per block (one source per block)
#endif
constexpr int kWThreads = SP_W_THREADS;
#ifndef SP_W_DELTA_K
#define SP_W_DELTA_K 4.0  // near-far step = K x mean weight x n / nnz (sp_graph_set_weights)
#endif

#ifndef SP_W_PER_SM
#define SP_W_PER_SM 2  // resident blocks per SM the registers are sized for (32 registers)
#endif
constexpr int kWLane = 16;  // rows of at most this many arcs are walked by one lane
constexpr int kG = 4;       // arcs of a lane's row whose loads are in flight together
constexpr int kUnreached = INT_MAX;

struct WArgs {
    const int32_t* rp;
    const int32_t* ci;
    const int32_t* w;  // [nnz] arc weights, parallel to ci
    int32_t n;
    const int32_t* sources;
    int32_t nsrc;
    // per block (slot b at base + b * stride)
    int32_t* dist;    // [n]
    int32_t* stamp;   // [n] last round the vertex joined a frontier
    int32_t* front;   // [2][n] frontiers
    int32_t* reach;   // [n] reached vertices, arrival order
    int32_t* order;   // [n] reached vertices by distance
    int32_t* lstart;  // [hcap + 1] index of each distance among the nonempty ones
    int32_t* hist;    // [hcap + 1] counts, then offsets, of each distance
    double* sig;      // [n]
    double* th;       // [n]
    double* bcpart;   // [n]
    int32_t hcap;     // distances must stay below this
    Ctl* ctl;
    int32_t* dist_out;  // SSSP mode: [nsrc][n] distances (-1 unreachable), else null
    int32_t* far0;      // [n] far pile, two buffers
    int32_t* far1;      // [n]
    int32_t* infar;     // [n] 1 while the vertex is in the far pile
    int32_t* expd;      // [n] distance at which the vertex was last expanded (-1: never)
    int4* kids;         // [n] up to three shortest-path-DAG children in CSR order (x, y, z)
                        // and their count (w; -1: more than three), found by the sigma pass
    int32_t delta;      // near-far step
};

// Block-wide exclusive scan of cnt[0..m) in place (cnt[m] receives the total);
// the block's threads walk it in chunks of blockDim.x with a running carry.
__device__ void block_exclusive_scan(int32_t* cnt, int m) {
    __shared__ int s_w[kWThreads / kWarp];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = lane_id(), wid = threadIdx.x / kWarp, nw = blockDim.x / kWarp;
    for (int base = 0; base < m; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int x = i < m ? cnt[i] : 0;
        const int incl = warp_incl_scan(x);
        if (lane == 31) s_w[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const int t = lane < nw ? s_w[lane] : 0;
            const int ti = warp_incl_scan(t);
            if (lane < nw) s_w[lane] = ti - t;
        }
        __syncthreads();
        const int carry = s_carry;
        if (i < m) cnt[i] = carry + s_w[wid] + incl - x;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = carry + s_w[wid] + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) cnt[m] = s_carry;
    __syncthreads();
}

__global__ void __launch_bounds__(kWThreads, SP_W_PER_SM) weighted_kernel(WArgs a) {
    __shared__ int s_cnt[2];  // frontier fill (next), reached fill
    __shared__ int s_err;
    __shared__ int s_max;
    __shared__ int s_far, s_far2, s_min;  // far pile fill (current, next), its smallest distance
    __shared__ unsigned long long s_st[3];
    const int n = a.n;
    const int tid = threadIdx.x, lane = lane_id(), warp = tid / kWarp, nwarps = blockDim.x / kWarp;
    const size_t off = (size_t)blockIdx.x * (size_t)n;
    int32_t* dist = a.dist + off;
    int32_t* stamp = a.stamp + off;
    int32_t* f0 = a.front + 2 * off;
    int32_t* f1 = f0 + n;
    int32_t* reach = a.reach + off;
    int32_t* order = a.order + off;
    int32_t* lstart = a.lstart + (size_t)blockIdx.x * (size_t)(a.hcap + 1);
    int32_t* hist = a.hist + (size_t)blockIdx.x * (size_t)(a.hcap + 1);
    double* sig = a.sig + off;
    double* th = a.th + off;
    double* bcp = a.bcpart + off;
    int32_t* fcur = a.far0 + off;
    int32_t* fnxt = a.far1 + off;
    int32_t* infar = a.infar + off;
    int32_t* expd = a.expd + off;
    int4* kids = a.kids + off;
    unsigned long long st_arcs = 0, st_reached = 0, st_scanned = 0;
    int levels_max = 0;
    if (tid == 0) s_err = 0;
    for (int v = tid; v < n; v += blockDim.x) {
        dist[v] = kUnreached;
        stamp[v] = -1;
        infar[v] = 0;
        expd[v] = -1;
        if (a.dist_out == nullptr) bcp[v] = 0.0;
    }
    __syncthreads();
    int round = 0;
    for (int si = blockIdx.x; si < a.nsrc; si += gridDim.x) {
        const int s = __ldg(&a.sources[si]);
        if (tid == 0) {
            dist[s] = 0;
            stamp[s] = round;
            f0[0] = s;
            reach[0] = s;
            s_cnt[0] = 0;
            s_cnt[1] = 1;
            s_far = 0;
        }
        __syncthreads();
        // ---- distances: near-far frontier rounds ----
        int fsize = 1;
        int32_t* cur = f0;
        int32_t* nxt = f1;
        int thr = a.delta;  // near: distance below thr
        int splits = 0;
        while (true) {
            while (fsize > 0) {
                ++round;
                for (int i0 = warp * 32; i0 < fsize; i0 += nwarps * 32) {
                    const int i = i0 + lane;
                    int u = 0, beg = 0, deg = 0, du = 0;
                    if (i < fsize) {
                        u = cur[i];
                        du = ld_volatile(&dist[u]);
                        if (expd[u] != du) {  // not yet expanded at this distance
                            expd[u] = du;
                            beg = __ldg(&a.rp[u]);
                            deg = __ldg(&a.rp[u + 1]) - beg;
                            st_scanned += (unsigned long long)deg;
                        }
                    }
                    // a vertex whose distance fell: the next near round, or the far pile
                    auto improved = [&](int x, int nd, int old) {
                        if (old == kUnreached) reach[atomicAdd(&s_cnt[1], 1)] = x;
                        if (nd < thr) {
                            if (atomicExch(&stamp[x], round) != round) nxt[atomicAdd(&s_cnt[0], 1)] = x;
                        } else if (atomicExch(&infar[x], 1) == 0) {
                            fcur[atomicAdd(&s_far, 1)] = x;
                        }
                    };
                    // distances only fall, so a read that is not below the
                    // candidate proves the atomicMin would change nothing
                    auto relax = [&](int e, int d0) {
                        const int x = __ldg(&a.ci[e]);
                        const int nd = d0 + __ldg(&a.w[e]);
                        if (nd >= a.hcap) { atomicCAS(&s_err, 0, kErrCapLevels); return; }
                        if (__ldcg(&dist[x]) <= nd) return;
                        const int old = atomicMin(&dist[x], nd);
                        if (nd < old) improved(x, nd, old);
                    };
                    if (deg <= kWLane) {
                        // a lane's row, kG arcs at a time: their ids and weights,
                        // then their atomicMin, then the frontier updates, each
                        // issued for all kG arcs before any result is used
                        for (int k0 = 0; k0 < deg; k0 += kG) {
                            int x[kG], nd[kG], old[kG];
#pragma unroll
                            for (int q = 0; q < kG; ++q) {
                                const bool ok = k0 + q < deg;
                                x[q] = ok ? __ldg(&a.ci[beg + k0 + q]) : -1;
                                nd[q] = ok ? du + __ldg(&a.w[beg + k0 + q]) : 0;
                            }
                            int dc[kG];
#pragma unroll
                            for (int q = 0; q < kG; ++q) dc[q] = x[q] >= 0 ? __ldcg(&dist[x[q]]) : 0;
#pragma unroll
                            for (int q = 0; q < kG; ++q) {
                                old[q] = kUnreached;
                                if (x[q] >= 0) {
                                    if (nd[q] >= a.hcap) {
                                        atomicCAS(&s_err, 0, kErrCapLevels);
                                        x[q] = -1;
                                    } else if (nd[q] < dc[q]) {
                                        old[q] = atomicMin(&dist[x[q]], nd[q]);
                                    } else {
                                        x[q] = -1;  // no improvement possible
                                    }
                                }
                            }
#pragma unroll
                            for (int q = 0; q < kG; ++q)
                                if (x[q] >= 0 && nd[q] < old[q]) improved(x[q], nd[q], old[q]);
                        }
                    }
                    unsigned wide = __ballot_sync(kFull, i < fsize && deg > kWLane);
                    while (wide) {
                        const int j = __ffs(wide) - 1;
                        wide &= wide - 1;
                        const int bj = __shfl_sync(kFull, beg, j), dj = __shfl_sync(kFull, deg, j);
                        const int dj0 = __shfl_sync(kFull, du, j);
                        for (int k = lane; k < dj; k += kWarp) relax(bj + k, dj0);
                    }
                }
                __syncthreads();
                fsize = s_cnt[0];
                __syncthreads();
                if (tid == 0) s_cnt[0] = 0;
                int32_t* t = cur; cur = nxt; nxt = t;
                if (s_err != 0) break;
                __syncthreads();
            }
            if (s_err != 0) break;
            // no near vertex left: move the threshold to the far pile
            const int nf = s_far;
            if (nf == 0) break;
            if (++splits > n + 1) {  // each split takes at least one vertex out of the pile
                if (tid == 0) atomicCAS(&s_err, 0, kErrCorrupt);
                break;
            }
            if (tid == 0) { s_min = INT_MAX; s_far2 = 0; }
            __syncthreads();
            int mn = INT_MAX;
            for (int i = tid; i < nf; i += blockDim.x) mn = min(mn, dist[fcur[i]]);
            mn = warp_min_i32(mn);
            if (lane == 0) atomicMin(&s_min, mn);
            __syncthreads();
            thr = s_min + a.delta;
            ++round;
            for (int i = tid; i < nf; i += blockDim.x) {
                const int x = fcur[i];
                const int dx = dist[x];
                if (dx < thr) {
                    infar[x] = 0;
                    if (expd[x] != dx && atomicExch(&stamp[x], round) != round) cur[atomicAdd(&s_cnt[0], 1)] = x;
                } else {
                    fnxt[atomicAdd(&s_far2, 1)] = x;
                }
            }
            __syncthreads();
            fsize = s_cnt[0];
            __syncthreads();
            if (tid == 0) { s_cnt[0] = 0; s_far = s_far2; }
            int32_t* t = fcur; fcur = fnxt; fnxt = t;
            __syncthreads();
        }
        if (s_err != 0) break;
        const int nr = s_cnt[1];
        if (a.dist_out != nullptr) {  // SSSP mode: distances only
            int32_t* row = a.dist_out + (size_t)si * (size_t)n;
            for (int v = tid; v < n; v += blockDim.x) {
                const int d = dist[v];
                row[v] = d == kUnreached ? -1 : d;
            }
        } else {
            // ---- order: counting sort by distance, then level boundaries ----
            if (tid == 0) s_max = 0;
            __syncthreads();
            int mx = 0;
            for (int i = tid; i < nr; i += blockDim.x) mx = max(mx, dist[reach[i]]);
            mx = warp_max_i32(mx);
            if (lane == 0) atomicMax(&s_max, mx);
            __syncthreads();
            const int m = s_max + 1;
            for (int d = tid; d <= m; d += blockDim.x) hist[d] = 0;
            __syncthreads();
            for (int i = tid; i < nr; i += blockDim.x) atomicAdd(&hist[dist[reach[i]]], 1);
            __syncthreads();
            block_exclusive_scan(hist, m);
            // levels: the distances with a nonzero count, numbered in order
            for (int d = tid; d < m; d += blockDim.x) lstart[d] = hist[d + 1] > hist[d] ? 1 : 0;
            __syncthreads();
            block_exclusive_scan(lstart, m);  // lstart[d] = level number of distance d (if nonempty)
            const int nlev = lstart[m];
            // scatter into order (positions from the offsets; order within a level is free)
            for (int i = tid; i < nr; i += blockDim.x) {
                const int v = reach[i];
                order[atomicAdd(&hist[dist[v]], 1)] = v;
            }
            __syncthreads();
            // hist[d] now holds the end of distance d's run in order; reach[]
            // (no longer needed) receives the end of each level
            for (int d = tid; d < m; d += blockDim.x)
                if (lstart[d + 1] > lstart[d]) reach[lstart[d]] = hist[d];
            __syncthreads();
            levels_max = max(levels_max, nlev);
            // ---- sigma, level by level ----
            for (int l = 0; l < nlev; ++l) {
                const int b = l == 0 ? 0 : reach[l - 1], e = reach[l];
                for (int i0 = b + warp * 32; i0 < e; i0 += nwarps * 32) {
                    const int i = i0 + lane;
                    int v = 0, beg = 0, deg = 0, dv = 0;
                    if (i < e) {
                        v = order[i];
                        beg = __ldg(&a.rp[v]);
                        deg = __ldg(&a.rp[v + 1]) - beg;
                        dv = dist[v];
                        st_arcs += (unsigned long long)deg;
                        st_reached += 1;
                        st_scanned += (unsigned long long)deg;
                    }
                    double acc = 0.0;
                    // the row's arcs into the next distances are v's DAG children:
                    // the first three (CSR order) and their count are kept for
                    // the dependency pass
                    int kid[3] = {0, 0, 0}, nkid = 0;
                    if (deg <= kWLane)
                        for (int k0 = 0; k0 < deg; k0 += kG) {  // kG arcs in flight, summed in CSR order
                            int u[kG], wt[kG], du[kG];
                            double c[kG];
#pragma unroll
                            for (int q = 0; q < kG; ++q) {
                                const bool ok = k0 + q < deg;
                                u[q] = ok ? __ldg(&a.ci[beg + k0 + q]) : -1;
                                wt[q] = ok ? __ldg(&a.w[beg + k0 + q]) : 0;
                            }
#pragma unroll
                            for (int q = 0; q < kG; ++q) du[q] = u[q] >= 0 ? dist[u[q]] : kUnreached;
#pragma unroll
                            for (int q = 0; q < kG; ++q)
                                c[q] = du[q] != kUnreached && du[q] + wt[q] == dv ? sig[u[q]] : 0.0;
#pragma unroll
                            for (int q = 0; q < kG; ++q) {
                                if (k0 + q < deg && du[q] != kUnreached && du[q] + wt[q] == dv) acc += c[q];
                                if (u[q] >= 0 && du[q] != kUnreached && du[q] == dv + wt[q]) {
                                    if (nkid < 3) kid[nkid] = u[q];
                                    ++nkid;
                                }
                            }
                        }
                    if (i < e && deg <= kWLane) kids[v] = make_int4(kid[0], kid[1], kid[2], nkid > 3 ? -1 : nkid);
                    unsigned wide = __ballot_sync(kFull, i < e && deg > kWLane);
                    while (wide) {
                        const int j = __ffs(wide) - 1;
                        wide &= wide - 1;
                        const int bj = __shfl_sync(kFull, beg, j), dj = __shfl_sync(kFull, deg, j);
                        const int dvj = __shfl_sync(kFull, dv, j);
                        const int vj = __shfl_sync(kFull, v, j);
                        int* kj = reinterpret_cast<int*>(&kids[vj]);
                        int nk = 0;  // children so far (the same in every lane)
                        double p = 0.0;
                        for (int k0 = 0; k0 < dj; k0 += kWarp) {
                            const int k = k0 + lane;
                            bool child = false;
                            if (k < dj) {
                                const int u = __ldg(&a.ci[bj + k]);
                                const int du = dist[u];
                                const int wk = __ldg(&a.w[bj + k]);
                                if (du != kUnreached && du + wk == dvj) p += sig[u];
                                child = du != kUnreached && du == dvj + wk;
                            }
                            const unsigned cb = __ballot_sync(kFull, child);
                            if (child) {
                                const int rank = nk + __popc(cb & ((1u << lane) - 1u));
                                if (rank < 3) kj[rank] = __ldg(&a.ci[bj + k]);
                            }
                            nk += __popc(cb);
                        }
                        if (lane == 0) kj[3] = nk > 3 ? -1 : nk;
                        p = warp_sum_f64(p);
                        if (lane == j) acc = p;
                    }
                    if (i < e) {
                        const double sv = l == 0 ? 1.0 : acc;
                        if (!normal_finite(sv)) atomicCAS(&s_err, 0, (int)SP_ERR_RANGE);
                        sig[v] = sv;
                    }
                }
                __syncthreads();
            }
            if (s_err != 0) break;
            // ---- delta, level by level in reverse ----
            for (int l = nlev - 1; l >= 1; --l) {
                const int b = reach[l - 1], e = reach[l];
                for (int i0 = b + warp * 32; i0 < e; i0 += nwarps * 32) {
                    const int i = i0 + lane;
                    int v = 0, beg = 0, deg = 0, dv = 0;
                    int4 kd = make_int4(0, 0, 0, 0);
                    if (i < e) {
                        v = order[i];
                        kd = kids[v];
                        beg = __ldg(&a.rp[v]);
                        deg = __ldg(&a.rp[v + 1]) - beg;
                        dv = dist[v];
                    }
                    // at most three children: their slots, summed in CSR order;
                    // else the row is scanned again
                    const bool slots = kd.w >= 0;
                    if (slots) deg = 0;
                    if (i < e && !slots) st_scanned += (unsigned long long)deg;
                    double acc = 0.0;
                    if (i < e && slots && kd.w > 0) {
                        const double t0 = th[kd.x];
                        const double t1 = kd.w > 1 ? th[kd.y] : 0.0;
                        const double t2 = kd.w > 2 ? th[kd.z] : 0.0;
                        acc += t0;
                        if (kd.w > 1) acc += t1;
                        if (kd.w > 2) acc += t2;
                    }
                    if (deg <= kWLane)
                        for (int k0 = 0; k0 < deg; k0 += kG) {  // kG arcs in flight, summed in CSR order
                            int x[kG], wt[kG], dx[kG];
                            double c[kG];
#pragma unroll
                            for (int q = 0; q < kG; ++q) {
                                const bool ok = k0 + q < deg;
                                x[q] = ok ? __ldg(&a.ci[beg + k0 + q]) : -1;
                                wt[q] = ok ? __ldg(&a.w[beg + k0 + q]) : 0;
                            }
#pragma unroll
                            for (int q = 0; q < kG; ++q) dx[q] = x[q] >= 0 ? dist[x[q]] : kUnreached;
#pragma unroll
                            for (int q = 0; q < kG; ++q)
                                c[q] = dx[q] != kUnreached && dx[q] == dv + wt[q] ? th[x[q]] : 0.0;
#pragma unroll
                            for (int q = 0; q < kG; ++q)
                                if (x[q] >= 0 && dx[q] != kUnreached && dx[q] == dv + wt[q]) acc += c[q];
                        }
                    unsigned wide = __ballot_sync(kFull, i < e && deg > kWLane);
                    while (wide) {
                        const int j = __ffs(wide) - 1;
                        wide &= wide - 1;
                        const int bj = __shfl_sync(kFull, beg, j), dj = __shfl_sync(kFull, deg, j);
                        const int dvj = __shfl_sync(kFull, dv, j);
                        double p = 0.0;
                        for (int k = lane; k < dj; k += kWarp) {
                            const int x = __ldg(&a.ci[bj + k]);
                            const int dx = dist[x];
                            if (dx != kUnreached && dx == dvj + __ldg(&a.w[bj + k])) p += th[x];
                        }
                        p = warp_sum_f64(p);
                        if (lane == j) acc = p;
                    }
                    if (i < e) {
                        const double sv = sig[v];
                        const double delta = sv * acc;
                        const double t = (1.0 + delta) / sv;
                        if (!normal_finite(t)) atomicCAS(&s_err, 0, (int)SP_ERR_RANGE);
                        th[v] = t;
                        bcp[v] += delta;
                    }
                }
                __syncthreads();
            }
            if (s_err != 0) break;
        }
        // ---- reset the reached vertices for the next source: by distance
        // order in BC mode (reach[] then holds level ends), by arrival in SSSP mode ----
        __syncthreads();
        const int32_t* reached_list = a.dist_out != nullptr ? reach : order;
        for (int i = tid; i < nr; i += blockDim.x) {
            const int v = reached_list[i];
            dist[v] = kUnreached;
            expd[v] = -1;
        }
        __syncthreads();
    }
    if (tid == 0) { s_st[0] = 0; s_st[1] = 0; s_st[2] = 0; }
    __syncthreads();
    atomicAdd(&s_st[0], st_arcs);
    atomicAdd(&s_st[1], st_reached);
    atomicAdd(&s_st[2], st_scanned);
    __syncthreads();
    if (tid == 0) {
        atomicAdd(&a.ctl->traversed_arcs, s_st[0]);
        atomicAdd(&a.ctl->reached, s_st[1]);
        atomicAdd(&a.ctl->entries, s_st[1]);
        atomicAdd(&a.ctl->scanned_arcs, s_st[2]);
        atomicMax(&a.ctl->max_levels, levels_max);
        if (s_err != 0) set_error(a.ctl, s_err);
    }
}

// Sum of the blocks' partial BC rows, in block order.
__global__ void weighted_sum_kernel(const double* __restrict__ part, int nparts, int64_t n, double* __restrict__ out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += part[(int64_t)b * n + v];
        out[v] = s;
    }
}

// Arc weights: each in [1, kMaxWeight]; undirected graphs: the reverse arc
// carries the same weight (rows sorted, found by binary search).
__global__ void weights_check_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                     const int32_t* __restrict__ w, int32_t n, int32_t max_w, int* bad,
                                     unsigned long long* wsum) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    unsigned long long sum = 0;
    for (int v = warp; v < n; v += nwarp) {
        for (int e = rp[v] + lane; e < rp[v + 1]; e += 32) {
            const int x = ci[e], wt = w[e];
            sum += (unsigned long long)(unsigned)wt;
            if (wt < 1 || wt > max_w) { atomicMin(bad, e); continue; }
            int lo = rp[x], hi = rp[x + 1];
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (ci[mid] < v) lo = mid + 1; else hi = mid;
            }
            if (!(lo < rp[x + 1] && ci[lo] == v && w[lo] == wt)) atomicMin(bad, e);
        }
    }
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0 && sum != 0) atomicAdd(wsum, sum);
}

}  // namespace

sp_status set_weights(Graph* g, const int32_t* weights, bool device_src, cudaStream_t st) {
    if (g->directed) return fail(SP_ERR_INVALID_ARG, "weighted BC supports undirected graphs only");
    if (g->nnz > 0 && (g->info.sorted_rows != 1 || g->info.has_duplicates != 0))
        return fail(SP_ERR_INVALID_ARG, "weighted graphs need sorted rows without repeated arcs (SP_GRAPH_SORT_ROWS)");
    int32_t* d_w = nullptr;
    SP_CUDA(cudaMalloc((void**)&d_w, sizeof(int32_t) * (size_t)std::max<int64_t>(g->nnz, 1)));
    int* d_bad = nullptr;  // [0] the first bad arc (0x7F7F7F7F: none); then the weight sum (u64) at byte 8
    cudaError_t e = cudaSuccess;
    if (g->nnz > 0)
        e = cudaMemcpyAsync(d_w, weights, sizeof(int32_t) * (size_t)g->nnz,
                            device_src ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_bad, 16, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0x7F, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(reinterpret_cast<char*>(d_bad) + 8, 0, 8, st);
    int bad = 0x7F7F7F7F;
    unsigned long long wsum = 0;
    if (e == cudaSuccess && g->n > 0) {
        weights_check_kernel<<<device_sm_count(g->device) * 8, 256, 0, st>>>(
            g->d_rp, g->d_ci, d_w, g->n, kMaxWeight, d_bad,
            reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(d_bad) + 8));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&wsum, reinterpret_cast<char*>(d_bad) + 8, 8, cudaMemcpyDeviceToHost, st);
    if (d_bad) cudaFreeAsync(d_bad, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(d_w);
        return cuda_fail(e, "setting arc weights");
    }
    if (bad != 0x7F7F7F7F) {
        cudaFree(d_w);
        return fail(SP_ERR_BAD_GRAPH, "arc " + std::to_string(bad) + ": weight outside [1, " +
                                          std::to_string(kMaxWeight) + "] or unlike its reverse arc's");
    }
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->d_w) cudaFree(g->d_w);
    g->d_w = d_w;
    // near-far step of the weighted form: Delta ~ (largest weight) / (average
    // degree), the delta-stepping rule of Meyer and Sanders (2003), with the
    // largest weight of a uniform draw taken as twice the mean: 4 x mean
    // weight x n / nnz (about 7 for weights U[1, 100] at average degree 30)
    double delta = 1.0;
    if (g->nnz > 0 && g->n > 0) {
        const double mean_w = (double)wsum / (double)g->nnz;
        delta = std::floor(SP_W_DELTA_K * mean_w * (double)g->n / (double)g->nnz + 0.5);
    }
    g->w_delta = (int32_t)std::min(std::max(delta, 1.0), (double)kMaxWeight);
    return SP_OK;
}

sp_status run_weighted(const WeightedLaunch& L, LaunchResult* result) {
    const Graph* g = L.g;
    const int64_t n = g->n;
    cudaStream_t st = L.stream;
    int per_sm = 0;
    SP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)&weighted_kernel, kWThreads, 0));
    if (per_sm < 1) return fail(SP_ERR_CUDA, "weighted kernel cannot be resident");
    // one block per source at a time; per-block state of 80 bytes a vertex,
    // so the grid is also capped by a state budget (32 GiB)
    int grid = per_sm * device_sm_count(g->device);
    if (L.max_ctas > 0 && L.max_ctas < grid) grid = L.max_ctas;
    const int64_t hcap = L.dist_cap;
    const double per_block = 80.0 * (double)n + 8.0 * (double)(hcap + 2);
    grid = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)grid, (int64_t)L.nsrc,
                                                         (int64_t)((32.0 * (1ull << 30)) / per_block)}));
    size_t bytes = 0;
    auto take = [&](size_t b) { size_t o = bytes; bytes += (b + 255) & ~(size_t)255; return o; };
    const size_t G = (size_t)grid, N = (size_t)n;
    const size_t o_ctl = take(sizeof(Ctl));
    const size_t o_dist = take(4 * N * G), o_stamp = take(4 * N * G), o_front = take(8 * N * G);
    const size_t o_reach = take(4 * N * G), o_order = take(4 * N * G);
    const size_t o_lstart = take(4 * (size_t)(hcap + 1) * G);
    const size_t o_hist = take(4 * (size_t)(hcap + 1) * G);
    const size_t o_sig = take(8 * N * G), o_th = take(8 * N * G), o_part = take(8 * N * G);
    const size_t o_far0 = take(4 * N * G), o_far1 = take(4 * N * G), o_infar = take(4 * N * G),
                 o_expd = take(4 * N * G), o_kids = take(16 * N * G);
    char* ws = nullptr;
    if (workspace_alloc((void**)&ws, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(SP_ERR_OOM, "workspace allocation (weighted form, " + std::to_string(bytes >> 20) + " MiB)");
    }
    struct FreeWs {
        char* p;
        cudaStream_t s;
        ~FreeWs() { cudaFreeAsync(p, s); }
    } free_ws{ws, st};
    SP_CUDA(cudaMemsetAsync(ws, 0, sizeof(Ctl), st));
    WArgs a{};
    a.rp = g->d_rp;
    a.ci = g->d_ci;
    a.w = g->d_w;
    a.n = (int32_t)n;
    a.sources = L.d_sources;
    a.nsrc = L.nsrc;
    a.dist = reinterpret_cast<int32_t*>(ws + o_dist);
    a.stamp = reinterpret_cast<int32_t*>(ws + o_stamp);
    a.front = reinterpret_cast<int32_t*>(ws + o_front);
    a.reach = reinterpret_cast<int32_t*>(ws + o_reach);
    a.order = reinterpret_cast<int32_t*>(ws + o_order);
    a.lstart = reinterpret_cast<int32_t*>(ws + o_lstart);
    a.hist = reinterpret_cast<int32_t*>(ws + o_hist);
    a.sig = reinterpret_cast<double*>(ws + o_sig);
    a.th = reinterpret_cast<double*>(ws + o_th);
    a.bcpart = reinterpret_cast<double*>(ws + o_part);
    a.hcap = (int32_t)hcap;
    a.ctl = reinterpret_cast<Ctl*>(ws + o_ctl);
    a.dist_out = L.d_dist;
    a.far0 = reinterpret_cast<int32_t*>(ws + o_far0);
    a.far1 = reinterpret_cast<int32_t*>(ws + o_far1);
    a.infar = reinterpret_cast<int32_t*>(ws + o_infar);
    a.expd = reinterpret_cast<int32_t*>(ws + o_expd);
    a.kids = reinterpret_cast<int4*>(ws + o_kids);
    a.delta = std::max(1, g->w_delta);
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, st);
    void* args[] = {&a};
    cudaError_t ce = cudaLaunchKernel((const void*)&weighted_kernel, dim3(grid), dim3(kWThreads), args, 0, st);
    if (ce == cudaSuccess && L.d_dist == nullptr) {
        const int rgrid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)device_sm_count(g->device) * 8);
        weighted_sum_kernel<<<std::max(rgrid, 1), 256, 0, st>>>(a.bcpart, grid, n, L.d_bc);
        ce = cudaGetLastError();
    }
    cudaEventRecord(ev1, st);
    static thread_local Ctl h;
    std::memset(&h, 0, sizeof(h));
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h, ws + o_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    float ms = 0.0f;
    if (ce == cudaSuccess && cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess) result->kernel_ms = ms;
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (ce != cudaSuccess) return cuda_fail(ce, "weighted form");
    result->err = h.err;
    result->levels = h.max_levels;
    result->traversed_arcs = h.traversed_arcs;
    result->reached = h.reached;
    result->entries = h.entries;
    result->scanned_arcs = h.scanned_arcs;
    result->grid = grid;
    result->groups = grid;
    result->launches = L.d_dist == nullptr ? 2 : 1;
    result->lcap = hcap;
    return SP_OK;
}

}  // namespace sp
