// Host side of the batched form for one width: workspace layout and launch.
#pragma once

#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>

#include "bc_batched.cuh"

#ifndef SP_T_HUB
#define SP_T_HUB 64
#endif
#ifndef SP_SEG
#define SP_SEG 512
#endif

namespace sp {

template <int W>
sp_status launch_batched_w(const BatchedLaunch& L, LaunchResult* result) {
    constexpr int B = 32 * W;
    const Graph* g = L.g;
    const int64_t n = g->n;
    cudaStream_t st = L.stream;
    const int t_hub = SP_T_HUB, seg = SP_SEG;  // rows above t_hub arcs run in segments of seg arcs

    // path-count rows: exact u32 counts, or FP64 with per-level exponents once
    // a count passes 2^32
    const void* fn;
    auto pick = [&](auto dir) -> const void* {
        constexpr bool kDir = decltype(dir)::value;
        if (L.sigma_float)
            return L.theta_f32 ? (const void*)&batched_kernel<W, double, float, kDir>
                               : (const void*)&batched_kernel<W, double, double, kDir>;
        return L.theta_f32 ? (const void*)&batched_kernel<W, unsigned int, float, kDir>
                           : (const void*)&batched_kernel<W, unsigned int, double, kDir>;
    };
    fn = g->directed ? pick(std::true_type{}) : pick(std::false_type{});
    const size_t sig_size = L.sigma_float ? 8 : 4;
    int per_sm = 0;
    SP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBatchThreads, 0));
    if (per_sm < 1) return fail(SP_ERR_CUDA, "batched kernel cannot be resident");
    int grid = per_sm * device_sm_count(g->device);
    if (L.max_ctas > 0 && L.max_ctas < grid) grid = L.max_ctas;

    int64_t lcap = std::min<int64_t>(n + 2, L.level_cap > 0 ? L.level_cap : 16384);
    int64_t ecap_max = n * std::min<int64_t>(B, lcap);
    int64_t ecap = L.entry_cap > 0 ? L.entry_cap : std::max<int64_t>(8 * n, 1 << 16);
    ecap = std::max<int64_t>(1, std::min(ecap, ecap_max));
    const int64_t arcs = g->knnz();
    int64_t hcap = L.hub_cap > 0 ? L.hub_cap : (arcs / t_hub) * 4 + 1024;
    int64_t segcap = arcs / seg + arcs / t_hub + 2;              // segments of one level
    int64_t scap = L.hub_cap > 0 ? 2 * L.hub_cap + 4 * (arcs / seg) : 4 * (arcs / seg) + hcap;  // all levels
    if (hcap > INT32_MAX || segcap > INT32_MAX || ecap > INT32_MAX || scap > INT32_MAX)
        return fail(SP_ERR_TOO_LARGE, "batched workspace");
    const size_t th_size = L.theta_f32 ? 4 : 8;

    size_t bytes = 0;
    auto take = [&](size_t b) { size_t o = bytes; bytes += (b + 255) & ~(size_t)255; return o; };
    size_t o_ctl = take(sizeof(Ctl));
    size_t o_dense = take(sizeof(uint32_t) * 4 * (size_t)n * W);
    size_t o_seen = take(sizeof(uint32_t) * (size_t)n * W);
    size_t o_ptag = take(sizeof(int32_t) * (size_t)n);
    size_t zero_end = bytes;  // everything above starts at zero
    size_t o_sig = take(sig_size * (size_t)n * B);
    size_t o_th = take(th_size * (size_t)n * B);
    size_t o_ent = take(sizeof(int32_t) * (size_t)ecap);
    size_t o_emask = take(sizeof(uint32_t) * (size_t)ecap * W);
    size_t o_eoff = take(sizeof(int32_t) * (size_t)(lcap + 2));
    size_t o_hoff = take(sizeof(int32_t) * (size_t)(lcap + 2));
    size_t o_soff = take(sizeof(int32_t) * (size_t)(lcap + 2));
    size_t o_segrec = take(sizeof(int32_t) * (size_t)scap);
    size_t o_hcnt = take(sizeof(unsigned long long) * (size_t)(lcap + 2));
    size_t o_hubs = take(sizeof(HubRec) * (size_t)hcap);
    size_t o_hdone = take(sizeof(int32_t) * 2 * (size_t)hcap);
    size_t o_part = take(8 * (size_t)segcap * B);
    size_t o_emax = take(sizeof(int32_t) * (size_t)lcap * B);
    size_t o_emin = take(sizeof(int32_t) * (size_t)lcap * B);

    char* ws = nullptr;
    if (workspace_alloc((void**)&ws, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(SP_ERR_OOM, "workspace allocation (batched form, " + std::to_string(bytes >> 20) + " MiB)");
    }
    cudaError_t ce = cudaMemsetAsync(ws, 0, zero_end, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(ws + o_hcnt, 0, sizeof(unsigned long long) * (size_t)(lcap + 2), st);
    if (ce != cudaSuccess) { cudaFreeAsync(ws, st); return cuda_fail(ce, "cudaMemsetAsync"); }

    BatchArgs a{};
    a.rp = g->krp();
    a.ci = g->kci();
    a.directed = g->directed;
    a.odeg = g->d_odeg;
    a.n = (int32_t)n;
    a.sources = L.d_sources;
    a.nsrc = L.nsrc;
    a.bc = L.d_bc;
    a.dense = reinterpret_cast<uint32_t*>(ws + o_dense);
    a.seen = reinterpret_cast<uint32_t*>(ws + o_seen);
    a.ptag = reinterpret_cast<int32_t*>(ws + o_ptag);
    a.sig = ws + o_sig;
    a.th = ws + o_th;
    a.ent = reinterpret_cast<int32_t*>(ws + o_ent);
    a.emask = reinterpret_cast<uint32_t*>(ws + o_emask);
    a.ecap = ecap;
    a.eoff = reinterpret_cast<int32_t*>(ws + o_eoff);
    a.hubs = reinterpret_cast<HubRec*>(ws + o_hubs);
    a.hcap = (int32_t)hcap;
    a.hoff = reinterpret_cast<int32_t*>(ws + o_hoff);
    a.soff = reinterpret_cast<int32_t*>(ws + o_soff);
    a.segrec = reinterpret_cast<int32_t*>(ws + o_segrec);
    a.scap = (int32_t)scap;
    a.hcnt = reinterpret_cast<unsigned long long*>(ws + o_hcnt);
    a.hdone = reinterpret_cast<int32_t*>(ws + o_hdone);
    a.part = ws + o_part;
    a.segcap = (int32_t)segcap;
    a.emax = reinterpret_cast<int32_t*>(ws + o_emax);
    a.emin = reinterpret_cast<int32_t*>(ws + o_emin);
    a.lcap = (int32_t)lcap;
    a.ctl = reinterpret_cast<Ctl*>(ws + o_ctl);
    a.pre_err = L.async.pre_err;
    a.debug_flags = L.debug_flags;
    a.timeout_ns = L.timeout_ns;
    a.t_hub = t_hub;
    a.seg = seg;
    a.word_bc = L.d_word_bc;
    a.bu_den = L.bottom_up_den;
    a.word_stats = L.d_word_stats;
    a.centre_bound = sigma_centre_bound(L.sigma_float, L.theta_f32, PlainMode::BC);
    a.sq = L.d_sq;
    a.word_cap = L.word_cap;
    a.feed = L.feed;
    a.feed_req = L.feed_req;
    a.feed_lanes = L.feed_lanes;
    a.req_dev = L.req_dev;
    a.req_cap = L.req_cap;

    void* args[] = {&a};
    if (L.async.flags != nullptr) {  // enqueue only: the finish step moves the error word on
        ce = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBatchThreads), args, 0, st);
        if (ce != cudaSuccess) {
            cudaFreeAsync(ws, st);
            return cuda_fail(ce, "cudaLaunchCooperativeKernel (batched form)");
        }
        sp_status frc = enqueue_finish(a.ctl, L.async, st);
        cudaFreeAsync(ws, st);
        result->launches = 2;
        result->grid = grid;
        result->ecap = ecap;
        result->hcap = hcap;
        result->lcap = lcap;
        return frc;
    }
    if (L.ctl_out != nullptr) {  // enqueue only: the control block comes back with an event
        ce = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBatchThreads), args, 0, st);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(L.ctl_out, ws + o_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
        cudaFreeAsync(ws, st);
        if (ce == cudaSuccess && L.on_done != nullptr) ce = cudaLaunchHostFunc(st, L.on_done, L.on_done_arg);
        if (ce == cudaSuccess && L.done_ev != nullptr) ce = cudaEventRecord(L.done_ev, st);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaLaunchCooperativeKernel (batched form, live)");
        result->launches = 1;
        result->grid = grid;
        result->ecap = ecap;
        result->hcap = hcap;
        result->lcap = lcap;
        return SP_OK;
    }
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, st);
    ce = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBatchThreads), args, 0, st);
    cudaEventRecord(ev1, st);
    if (ce != cudaSuccess) {
        cudaFreeAsync(ws, st);
        return cuda_fail(ce, "cudaLaunchCooperativeKernel (batched form)");
    }
    static thread_local Ctl h;
    std::memset(&h, 0, sizeof(h));
    ce = cudaMemcpyAsync(&h, ws + o_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(ws, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return cuda_fail(ce, "reading the batched-form result");
    result->err = h.err;
    result->levels = h.max_levels;
    result->traversed_arcs = h.traversed_arcs;
    result->reached = h.reached;
    result->entries = h.entries;
    result->scanned_arcs = h.scanned_arcs;
    result->dag_arcs = h.dag_arcs;
    result->recentred = h.recentred;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess) result->kernel_ms = ms;
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    result->launches = 1;
    result->grid = grid;
#ifdef SP_PROFILE
    {
        const char* names[8] = {"fwd chunks", "fwd segments", "bwd chunks", "bwd segments", "barrier", "other",
                                "discovery", "pulls"};
        unsigned long long tot = 0;
        for (int c = 0; c < 8; ++c) tot += h.prof[c];
        fprintf(stderr, "profile W=%d grid=%d kernel %.3f ms, levels %d\n", W, grid, result->kernel_ms, h.max_levels);
        for (int c = 0; c < 8; ++c)
            fprintf(stderr, "  %-13s %6.2f%%\n", names[c], tot ? 100.0 * (double)h.prof[c] / (double)tot : 0.0);
        fprintf(stderr, "  phase ms:");
        for (int p = 2; p < 256 && h.phase_ns[p]; ++p)
            fprintf(stderr, " %.3f", (double)(h.phase_ns[p] - h.phase_ns[p - 1]) * 1e-6);
        fprintf(stderr, "\n");
    }
#endif
    if (h.err == SP_ERR_TIMEOUT) result->diag = barrier_diagnostic(h, grid);
    result->ecap = ecap;
    result->hcap = hcap;
    result->lcap = lcap;
    return SP_OK;
}

}  // namespace sp
