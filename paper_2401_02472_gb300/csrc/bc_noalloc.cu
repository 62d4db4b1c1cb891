// sp_bc_noalloc: betweenness centrality for callers that cannot allocate
// device memory.
//
// Some callers may not call cudaMalloc (or any allocator) at the point where
// they need BC: code that runs between the steps of a framework that owns all
// device memory and hands out fixed buffers, real-time or serving threads that
// must not block on the allocator or risk an out-of-memory failure mid-run, or
// embedded runtimes with a fixed memory plan.  For them this entry point runs
// the plain form (one source at a time, the kernel in bc_plain_kernel.cuh)
// with every byte of scratch taken from one file-scope device array, sized for
// graphs of up to kNoallocMaxN vertices and kNoallocMaxNnz arcs.  The caller
// passes the graph, the sources and the output buffer, all in device memory.
//
// The array is reserved on every GPU that loads this library, for as long as
// the process lives.  Every call shares it and it keeps the last call's
// contents, so each call clears what must start at zero (the launch control
// block and the check results); calls that overlap on the GPU (two streams,
// or two host threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <climits>
#include <cstring>
#include <mutex>
#include <string>

#include "bc_plain_kernel.cuh"

namespace sp {
namespace {

constexpr int64_t kNoallocMaxN = int64_t(1) << 18;    // 262,144 vertices
constexpr int64_t kNoallocMaxNnz = int64_t(1) << 24;  // 16,777,216 arcs (both directions counted)
constexpr int kTThread = 16, kTHub = 4096, kSeg = 4096;
constexpr int64_t kHcap = kNoallocMaxNnz / kTHub + 2;
constexpr int64_t kSegcap = kNoallocMaxNnz / kSeg + kHcap + 2;
constexpr int64_t kLevels = kNoallocMaxN + 2;

// Results of the argument check kernel (0x7F7F7F7F = nothing found).
struct NoallocCheck {
    int bad_rowptr;
    int bad_col;
    int bad_src;
    int pad;
};
constexpr int kNone = 0x7F7F7F7F;

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kOffCtl = 0;
constexpr size_t kOffGctl = kOffCtl + align256(sizeof(Ctl));
constexpr size_t kOffCheck = kOffGctl + align256(sizeof(GroupCtl));
constexpr size_t kOffLvl = kOffCheck + align256(sizeof(NoallocCheck));
constexpr size_t kOffSig = kOffLvl + align256(4 * kNoallocMaxN);
constexpr size_t kOffTh = kOffSig + align256(8 * kNoallocMaxN);
constexpr size_t kOffQ = kOffTh + align256(8 * kNoallocMaxN);
constexpr size_t kOffQrow = kOffQ + align256(4 * kNoallocMaxN);
constexpr size_t kOffQoff = kOffQrow + align256(8 * kNoallocMaxN);
constexpr size_t kOffHubs = kOffQoff + align256(4 * kLevels);
constexpr size_t kOffHoff = kOffHubs + align256(sizeof(HubRec) * kHcap);
constexpr size_t kOffHcnt = kOffHoff + align256(4 * kLevels);
constexpr size_t kOffHdone = kOffHcnt + align256(8 * kLevels);
constexpr size_t kOffPart = kOffHdone + align256(4 * 2 * kHcap);
constexpr size_t kOffEmax = kOffPart + align256(8 * kSegcap);
constexpr size_t kOffEmin = kOffEmax + align256(4 * kLevels);
constexpr size_t kOffFexp = kOffEmin + align256(4 * kLevels);
constexpr size_t kScratchBytes = kOffFexp + align256(8 * kLevels);  // about 18 MB

static_assert(kLevels < INT32_MAX, "level capacity");

// The scratch.  Host code must not take this name as a device address (in
// host code it names a host-side shadow); it uses the address returned by
// cudaGetSymbolAddress for the current device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_addr[64] = {nullptr};

// Device address of the scratch on the current device (looked up once per device).
sp_status scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= 64) return fail(SP_ERR_NO_DEVICE, "device index out of range");
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return SP_OK;
}

__global__ void noalloc_check_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int32_t n,
                                     int64_t nnz, const int32_t* __restrict__ src, int32_t nsrc,
                                     NoallocCheck* out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = t; v < n; v += stride) {
        int a = rp[v], b = rp[v + 1];
        if (a < 0 || b < a || (int64_t)b > nnz || (v == 0 && a != 0) || (v == n - 1 && (int64_t)b != nnz))
            atomicMin(&out->bad_rowptr, (int)v);
    }
    for (int64_t e = t; e < nnz; e += stride) {
        int c = ci[e];
        if (c < 0 || c >= n) atomicMin(&out->bad_col, (int)e);
    }
    for (int64_t i = t; i < nsrc; i += stride) {
        int s = src[i];
        if (s < 0 || s >= n) atomicMin(&out->bad_src, (int)i);
    }
}

// Device memory of device `dev` (or managed memory, which every device may
// access).  Memory of another GPU is refused: the kernels read and write the
// buffers directly, and without peer access that would be an illegal access.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace
}  // namespace sp

using namespace sp;

extern "C" sp_status sp_bc_noalloc(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int64_t nnz,
                                   const int32_t* sources, int32_t nsrc, double* bc_out, sp_stream stream) {
    set_last_error("");
    if (n <= 0 || nnz < 0 || nsrc < 0) return fail(SP_ERR_INVALID_ARG, "sp_bc_noalloc: n must be > 0, nnz and nsrc >= 0");
    if ((int64_t)n > kNoallocMaxN || nnz > kNoallocMaxNnz)
        return fail(SP_ERR_TOO_LARGE, "sp_bc_noalloc: the static scratch holds graphs of at most " +
                                          std::to_string(kNoallocMaxN) + " vertices and " +
                                          std::to_string(kNoallocMaxNnz) + " arcs (got n = " + std::to_string(n) +
                                          ", nnz = " + std::to_string(nnz) + "); use sp_bc");
    if (!row_ptr || !bc_out || (nnz > 0 && !col_idx) || (nsrc > 0 && !sources))
        return fail(SP_ERR_INVALID_ARG, "sp_bc_noalloc: NULL pointer");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(SP_ERR_NO_DEVICE, "no CUDA device");
    }
    if (!on_device(row_ptr, dev) || !on_device(bc_out, dev) || (nnz > 0 && !on_device(col_idx, dev)) ||
        (nsrc > 0 && !on_device(sources, dev)))
        return fail(SP_ERR_INVALID_ARG,
                    "sp_bc_noalloc: row_ptr, col_idx, sources and bc_out must be device memory of the current device");
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) return fail(SP_ERR_NO_DEVICE, "this build targets compute capability 10.3");
    unsigned char* ws = nullptr;
    sp_status rc = scratch_address(dev, &ws);
    if (rc != SP_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    // Clear what must start at zero; the rest of the scratch is written
    // before it is read by the kernel.
    NoallocCheck* d_check = reinterpret_cast<NoallocCheck*>(ws + kOffCheck);
    SP_CUDA(cudaMemsetAsync(d_check, 0x7F, sizeof(NoallocCheck), st));
    const int sms = device_sm_count(dev);
    noalloc_check_kernel<<<sms * 4, 256, 0, st>>>(row_ptr, col_idx, n, nnz, sources, nsrc, d_check);
    SP_CUDA(cudaGetLastError());
    NoallocCheck chk;
    SP_CUDA(cudaMemcpyAsync(&chk, d_check, sizeof(chk), cudaMemcpyDeviceToHost, st));
    SP_CUDA(cudaStreamSynchronize(st));
    if (chk.bad_rowptr != kNone)
        return fail(SP_ERR_BAD_GRAPH, "sp_bc_noalloc: row_ptr invalid at row " + std::to_string(chk.bad_rowptr));
    if (chk.bad_col != kNone)
        return fail(SP_ERR_BAD_GRAPH, "sp_bc_noalloc: col_idx out of [0, n) at arc " + std::to_string(chk.bad_col));
    if (chk.bad_src != kNone)
        return fail(SP_ERR_INVALID_ARG, "sp_bc_noalloc: source " + std::to_string(chk.bad_src) + " out of [0, n)");
    if (nsrc == 0) {
        SP_CUDA(cudaMemsetAsync(bc_out, 0, sizeof(double) * (size_t)n, st));
        SP_CUDA(cudaStreamSynchronize(st));
        return SP_OK;
    }

    PlainArgs a{};
    a.rp = row_ptr;
    a.ci = col_idx;
    a.n = n;
    a.sources = sources;
    a.nsrc = nsrc;
    a.bc = bc_out;
    a.bcpart = nullptr;
    a.ngroups = 1;
    a.lcap = (int32_t)kLevels;
    a.gctl = reinterpret_cast<GroupCtl*>(ws + kOffGctl);
    a.lvl = reinterpret_cast<int32_t*>(ws + kOffLvl);
    a.sig = ws + kOffSig;
    a.th = ws + kOffTh;
    a.q = reinterpret_cast<int32_t*>(ws + kOffQ);
    a.qrow = reinterpret_cast<int2*>(ws + kOffQrow);
    a.qoff = reinterpret_cast<int32_t*>(ws + kOffQoff);
    a.hubs = reinterpret_cast<HubRec*>(ws + kOffHubs);
    a.hcap = (int32_t)kHcap;
    a.hoff = reinterpret_cast<int32_t*>(ws + kOffHoff);
    a.hcnt = reinterpret_cast<unsigned long long*>(ws + kOffHcnt);
    a.hdone = reinterpret_cast<int32_t*>(ws + kOffHdone);
    a.part = reinterpret_cast<double*>(ws + kOffPart);
    a.segcap = (int32_t)kSegcap;
    a.emax = reinterpret_cast<int32_t*>(ws + kOffEmax);
    a.emin = reinterpret_cast<int32_t*>(ws + kOffEmin);
    a.fexp = reinterpret_cast<long long*>(ws + kOffFexp);
    a.ctl = reinterpret_cast<Ctl*>(ws + kOffCtl);
    a.pre_err = nullptr;
    a.gate = nullptr;
    a.mode = (int)PlainMode::BC;
    a.timeout_ns = 20000000000ull;
    a.t_thread = kTThread;
    a.t_hub = kTHub;
    a.seg = kSeg;
    a.bu_den = 0;
    a.centre_bound = sigma_centre_bound(true, false, PlainMode::BC);
    a.trace = nullptr;

    // Exact 64-bit path counts first; FP64 counts with per-level rescaling
    // when they overflow.
    for (int attempt = 0; attempt < 2; ++attempt) {
        const void* fn = attempt == 0
                             ? reinterpret_cast<const void*>(&plain_kernel<unsigned long long, double, false, false>)
                             : reinterpret_cast<const void*>(&plain_kernel<double, double, false, false>);
        int per_sm = 0;
        SP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPlainThreads, 0));
        if (per_sm < 1) return fail(SP_ERR_CUDA, "sp_bc_noalloc: kernel cannot be resident");
        SP_CUDA(cudaMemsetAsync(a.ctl, 0, sizeof(Ctl), st));
        SP_CUDA(cudaMemsetAsync(a.gctl, 0, sizeof(GroupCtl), st));
        a.gblocks = per_sm * sms;
        void* args[] = {&a};
        SP_CUDA(cudaLaunchCooperativeKernel(fn, dim3(per_sm * sms), dim3(kPlainThreads), args, 0, st));
        int err = 0;
        SP_CUDA(cudaMemcpyAsync(&err, &a.ctl->err, sizeof(int), cudaMemcpyDeviceToHost, st));
        SP_CUDA(cudaStreamSynchronize(st));
        if (err == 0) return SP_OK;
        if (err == kErrSigmaOverflow && attempt == 0) continue;
        if (err == SP_ERR_RANGE || err == kErrSigmaOverflow)
            return fail(SP_ERR_RANGE, "sp_bc_noalloc: a path count or dependency left the FP64 range");
        if (err == SP_ERR_TIMEOUT) return fail(SP_ERR_TIMEOUT, "sp_bc_noalloc: a grid barrier wait timed out");
        return fail(SP_ERR_CUDA, "sp_bc_noalloc: device error " + std::to_string(err));
    }
    return SP_OK;
}
