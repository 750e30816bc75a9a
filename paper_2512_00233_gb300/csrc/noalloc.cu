// kcore_run_noalloc: the decomposition without any device allocation.
//
// Some callers cannot allocate device memory while they run us: a serving
// process that reserved the whole device for its own pool up front, a
// real-time loop that must not stall on the allocator's implicit
// synchronisation, or code running inside another allocator's callback.  This
// entry point serves them.  Its working memory (control block, frontier
// bitmaps and lists) is one fixed array compiled into the library; the
// estimates live in the caller's output buffer.  The array holds
// KCORE_NOALLOC_MAX_N vertices and stays resident on every GPU where it has
// been loaded until the process exits.  With the CUDA runtime's lazy module
// loading (the default since CUDA 12.2) the array is reserved on a device the
// first time this file's device code is used there, i.e. on the first call,
// and the kernels are loaded on their first launch; a call with n = 0 does
// only that loading, so a caller can make it before it reserves the rest of
// the device.
//
// In host code `g_noalloc_scratch` names a host-side stand-in, not device
// memory: the device address is looked up on every call with
// cudaGetSymbolAddress (with the caller's device current; cheap once the
// module is loaded, and never stale after a context is re-created) and passed
// to the kernels.  Every call shares the array; each call clears what must
// start at zero, and calls that overlap on the GPU race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <string>

#include "kc_common.cuh"

namespace kc {

kcore_status fail(kcore_status s, const std::string& msg);
kcore_status cuda_status(cudaError_t e, const char* what);

namespace {

constexpr long long kMaxN = KCORE_NOALLOC_MAX_N;
constexpr long long kWords = (kMaxN + 31) / 32;
constexpr size_t round256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kCtlBytes = round256(sizeof(SweepCtl));
constexpr size_t kBitmapBytes = round256(sizeof(uint32_t) * kWords);
constexpr size_t kListBytes = round256(sizeof(int) * kTiers * kMaxN);  // one region per tier
constexpr size_t kScratchBytes = kCtlBytes + kParities * (kBitmapBytes + kListBytes);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the array on the current device.  Loads this file's
// module there if it is not loaded yet (which reserves the array).
cudaError_t scratch_address(unsigned char** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = (unsigned char*)p;
    return cudaSuccess;
}

// Estimates start at the degrees (tier in the top bits) and every vertex joins
// the first frontier in its tier's region.  Offsets are checked here (row
// bounds inside [0, nnz], rows in order); a bad row sets the status, which
// ends the sweep kernel before its first sweep, and counts as degree 0.
template <typename Off>
__global__ void k_noalloc_init(const Off* __restrict__ rp, int n, long long nnz, int t_lo, int t_hi,
                               uint32_t* __restrict__ est, int* __restrict__ list0, SweepCtl* ctl) {
    const int lane = threadIdx.x & 31;
    for (long long v0 = blockIdx.x * (long long)blockDim.x; v0 < n;
         v0 += (long long)gridDim.x * blockDim.x) {
        const long long v = v0 + threadIdx.x;
        const bool valid = v < n;
        int tier = -1;
        if (valid) {
            const long long b = (long long)rp[v];
            const long long e = (long long)rp[v + 1];
            const bool ok = e >= b && b >= 0 && e <= nnz && (v > 0 || b == 0);
            if (!ok) atomicCAS(&ctl->status, 0, (int)KCORE_ERR_INVALID);
            const long long d = ok ? e - b : 0;
            tier = d <= t_lo ? 0 : (d <= t_hi ? 1 : 2);
            est[v] = ((uint32_t)tier << kEstBits) | (uint32_t)d;
        }
#pragma unroll
        for (int q = 0; q < kTiers; q++) {
            const unsigned m = __ballot_sync(0xffffffffu, tier == q);
            if (m) {
                const int leader = __ffs(m) - 1;
                unsigned base = 0;
                if (lane == leader) base = atomicAdd(&ctl->fcnt[0][q], (unsigned)__popc(m));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (tier == q) list0[(long long)q * n + base + __popc(m & ((1u << lane) - 1u))] = (int)v;
            }
        }
    }
}

// The entries of a clean CSR, checked edge-parallel (a hub row is spread over
// many warps): every id in [0, n), no loop, each row strictly increasing.  A
// warp takes 32 consecutive entries; lane 0 finds the row of the first by
// bisection of row_ptr, and each lane walks forward to its own row.  Any
// failure sets the status.  Reads stay inside row_ptr[0, n] and col[0, nnz)
// even when the offsets are malformed (the init kernel reports those).
template <typename Off>
__global__ void k_noalloc_check(const Off* __restrict__ rp, const int* __restrict__ col, int n,
                                long long nnz, SweepCtl* ctl) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    bool ok = true;
    for (long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; w * 32 < nnz;
         w += warps) {
        const long long j0 = w * 32, j = j0 + lane;
        long long r = 0;
        if (lane == 0) {  // last row r in [0, n - 1] with rp[r] <= j0
            long long lo = 0, hi = n - 1;
            while (lo < hi) {
                const long long mid = (lo + hi + 1) >> 1;
                if ((long long)rp[mid] <= j0) lo = mid;
                else hi = mid - 1;
            }
            r = lo;
        }
        r = __shfl_sync(0xffffffffu, r, 0);
        if (j < nnz) {
            while (r < n - 1 && (long long)rp[r + 1] <= j) r++;
            const int x = col[j];
            const long long b = (long long)rp[r];
            ok = ok && (unsigned)x < (unsigned)n && x != (int)r;
            if (j > 0 && j > b) ok = ok && col[j - 1] < x;
        }
    }
    if (__any_sync(0xffffffffu, !ok) && lane == 0) atomicCAS(&ctl->status, 0, (int)KCORE_ERR_INVALID);
}

__global__ void k_noalloc_bitmap(uint32_t* bm0, long long words, int n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < words;
         i += (long long)gridDim.x * blockDim.x) {
        const long long hi = (i + 1) * 32;
        bm0[i] = hi <= n ? 0xffffffffu : ((1u << (n - i * 32)) - 1u);
    }
}

}  // namespace


}  // namespace kc

using namespace kc;

extern "C" kcore_status kcore_run_noalloc(int64_t n, const void* row_ptr, int32_t row_ptr_bytes,
                                          const int32_t* col_idx, int32_t* coreness_out,
                                          void* cuda_stream) {
    if (n < 0 || n > kMaxN)
        return fail(KCORE_ERR_INVALID, "kcore_run_noalloc: n must be in [0, " +
                                           std::to_string(kMaxN) + "] (KCORE_NOALLOC_MAX_N)");
    if (row_ptr_bytes != 4 && row_ptr_bytes != 8)
        return fail(KCORE_ERR_INVALID, "kcore_run_noalloc: row_ptr_bytes must be 4 or 8");
    unsigned char* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess)
        return cuda_status(e, "kcore_run_noalloc: cudaGetSymbolAddress (loading the module that "
                              "holds the fixed working array)");
    if (n == 0) {
        // preparation: load every kernel this entry point launches, so that
        // later calls load nothing (lazy loading would do it on first use)
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, k_noalloc_init<int>);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_noalloc_init<long long>);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_noalloc_check<int>);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_noalloc_check<long long>);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_noalloc_bitmap);
        kcore_options o;
        kcore_default_options(&o);
        int grid = 0;
        for (int off64 = 0; off64 < 2 && e == cudaSuccess; off64++)
            e = sweep_max_grid(o.block, o.t_lo, o.t_hi, off64, &grid);
        if (e != cudaSuccess) return cuda_status(e, "kcore_run_noalloc: loading its kernels");
        return KCORE_OK;
    }
    if (!row_ptr || !col_idx || !coreness_out)
        return fail(KCORE_ERR_INVALID, "kcore_run_noalloc: NULL pointer");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    SweepCtl* ctl = (SweepCtl*)base;
    uint32_t* bitmap[kParities];
    int* list[kParities];
    for (int p = 0; p < kParities; p++) {
        bitmap[p] = (uint32_t*)(base + kCtlBytes + p * kBitmapBytes);
        list[p] = (int*)(base + kCtlBytes + kParities * kBitmapBytes + p * kListBytes);
    }
    const long long words = (n + 31) / 32;
    long long nnz = 0;
    e = cudaMemcpyAsync(&nnz, (const char*)row_ptr + (size_t)row_ptr_bytes * n, row_ptr_bytes,
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e, "kcore_run_noalloc: read row_ptr[n]");
    if (row_ptr_bytes == 4) nnz = (long long)(int32_t)(nnz & 0xffffffffLL);
    if (nnz < 0) return fail(KCORE_ERR_INVALID, "kcore_run_noalloc: row_ptr[n] < 0");

    kcore_options o;
    kcore_default_options(&o);
    // what must start at zero: the control block and the bitmaps of sweeps 1, 2
    e = cudaMemsetAsync(ctl, 0, sizeof(SweepCtl), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bitmap[1], 0, sizeof(uint32_t) * words, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bitmap[2], 0, sizeof(uint32_t) * words, st);
    if (e != cudaSuccess) return cuda_status(e, "kcore_run_noalloc: clear");
    const int g = (int)std::min<long long>((n + 255) / 256, (long long)sm_count() * 8);
    k_noalloc_bitmap<<<g, 256, 0, st>>>(bitmap[0], words, (int)n);
    count_launch();
    uint32_t* est = (uint32_t*)coreness_out;
    const int gc = (int)std::max<long long>(1, std::min<long long>((nnz + 255) / 256,
                                                                   (long long)sm_count() * 8));
    if (row_ptr_bytes == 8) {
        k_noalloc_init<<<g, 256, 0, st>>>((const long long*)row_ptr, (int)n, nnz, o.t_lo, o.t_hi,
                                          est, list[0], ctl);
        if (nnz > 0)
            k_noalloc_check<<<gc, 256, 0, st>>>((const long long*)row_ptr, col_idx, (int)n, nnz, ctl);
    } else {
        k_noalloc_init<<<g, 256, 0, st>>>((const int*)row_ptr, (int)n, nnz, o.t_lo, o.t_hi, est,
                                          list[0], ctl);
        if (nnz > 0) k_noalloc_check<<<gc, 256, 0, st>>>((const int*)row_ptr, col_idx, (int)n, nnz, ctl);
    }
    count_launch();
    if (nnz > 0) count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, "kcore_run_noalloc: init");

    SweepArgs a;
    memset(&a, 0, sizeof(a));
    a.refined = 1;  // asynchronous sweeps: the refined activation rule
    a.row_ptr = row_ptr;
    a.col = col_idx;
    a.est = est;
    a.init_list = nullptr;
    for (int p = 0; p < kParities; p++) {
        a.list[p] = list[p];
        a.bitmap[p] = bitmap[p];
    }
    a.tier_off[0] = 0;
    a.tier_off[1] = n;
    a.tier_off[2] = 2 * n;
    a.ctl = ctl;
    a.trace = nullptr;
    a.max_trace = 0;
    a.first_sweep = 0;
    a.max_sweeps = 2 * nnz + n + 1;
    a.stop_sweep = LLONG_MAX;
    a.timeout_ns = (long long)(o.timeout_s * 1e9);
    a.words = words;
    a.n = (int)n;
    a.t_lo = o.t_lo;
    a.t_hi = o.t_hi;
    a.low_chunk = o.low_chunk;
    a.med_chunk = o.med_chunk;
    a.tail_max = o.tail_max;
    a.off64 = row_ptr_bytes == 8 ? 1 : 0;
    a.out = coreness_out;  // the estimates live there: the launch masks them to the coreness
    const long long want = std::max<long long>(1, (n + nnz + (long long)o.block * 32 - 1) /
                                                      ((long long)o.block * 32));
    int grid = 0;
    e = launch_sweep(a, o.block, (int)std::min<long long>(want, INT_MAX), 0, st, &grid);
    int h[2] = {0, 0};  // status, done
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, &ctl->status, sizeof(int) * 2, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e, "kcore_run_noalloc");
    if (h[0] == KCORE_ERR_INVALID)
        return fail(KCORE_ERR_INVALID, "kcore_run_noalloc: the CSR is not clean (KCORE_IN_CLEAN form)");
    if (h[0] != 0) return fail((kcore_status)h[0], "kcore_run_noalloc: sweep kernel reported an error");
    if (!h[1]) return fail(KCORE_ERR_CUDA, "kcore_run_noalloc: sweep kernel ended early");
    return KCORE_OK;
}
