// Device CSR cleaning (Sec. IV-A: graphs treated as undirected, self-loops
// removed; Sec. III-B: neighbour lists kept as sorted vectors).
//
// Pipeline, all on the device:
//   1. expand   every sample (u, v), u != v, becomes the two 64-bit keys
//               (u << 32 | v) and (v << 32 | u); loops become a sentinel that
//               sorts last.
//   2. sort     stable LSD radix sort, 8-bit digits, only over the bits that
//               vertex ids use (reduce-then-scan per digit; stable in-tile
//               ranking with __match_any_sync).
//   3. dedupe   keep a key when it differs from its predecessor; an exclusive
//               scan of the keep flags gives its position in col_idx.
//   4. rows     the first and last entry of every row give its degree; an
//               exclusive scan of the degrees gives row_ptr.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "kc_common.cuh"

namespace kc {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned long long kSentinel = ~0ull;

// ------------------------------------------------------------------ scan
constexpr int kScanT = 512, kScanI = 8, kScanTile = kScanT * kScanI;

__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v,
                                                              unsigned long long* total) {
    __shared__ unsigned long long wsum[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long s = lane < nw ? wsum[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        wsum[lane] = s;
    }
    __syncthreads();
    unsigned long long r = (wid ? wsum[wid - 1] : 0ull) + x - v;
    *total = wsum[nw - 1];
    __syncthreads();
    return r;
}

template <typename F>
__global__ void __launch_bounds__(kScanT) k_scan_reduce(F f, long long N, unsigned long long* bsum) {
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanI;
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanI; i++)
        if (base + i < N) s += f(base + i);
    unsigned long long tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

template <typename F, typename Out>
__global__ void __launch_bounds__(kScanT) k_scan_down(F f, long long N,
                                                      const unsigned long long* boff, Out* out,
                                                      int write_total) {
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanI;
    unsigned long long v[kScanI], s = 0;
#pragma unroll
    for (int i = 0; i < kScanI; i++) {
        v[i] = base + i < N ? f(base + i) : 0ull;
        s += v[i];
    }
    unsigned long long tot;
    unsigned long long run = block_excl_scan(s, &tot) + (boff ? boff[blockIdx.x] : 0ull);
#pragma unroll
    for (int i = 0; i < kScanI; i++) {
        if (base + i < N) out[base + i] = (Out)run;
        run += v[i];
    }
    if (write_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1)
        out[N] = (Out)((boff ? boff[blockIdx.x] : 0ull) + tot);
}

struct ReadU64 {
    const unsigned long long* p;
    __device__ unsigned long long operator()(long long i) const { return p[i]; }
};
struct ReadU32 {
    const uint32_t* p;
    __device__ unsigned long long operator()(long long i) const { return p[i]; }
};

// out[0..N) = exclusive prefix sums of f(0..N); out[N] = total if with_total.
template <typename F, typename Out>
cudaError_t exclusive_scan(F f, long long N, Out* out, bool with_total, cudaStream_t st) {
    if (N <= 0) {
        if (with_total) return cudaMemsetAsync(out, 0, sizeof(Out), st);
        return cudaSuccess;
    }
    const long long nb = (N + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        k_scan_down<<<1, kScanT, 0, st>>>(f, N, (const unsigned long long*)nullptr, out,
                                          with_total ? 1 : 0);
        return cudaGetLastError();
    }
    unsigned long long *bsum = nullptr, *boff = nullptr;
    cudaError_t e = cudaMallocAsync(&bsum, sizeof(unsigned long long) * nb, st);
    if (e != cudaSuccess) return e;
    e = cudaMallocAsync(&boff, sizeof(unsigned long long) * (nb + 1), st);
    if (e != cudaSuccess) { cudaFreeAsync(bsum, st); return e; }
    k_scan_reduce<<<(unsigned)nb, kScanT, 0, st>>>(f, N, bsum);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = exclusive_scan(ReadU64{bsum}, nb, boff, false, st);
    if (e == cudaSuccess) {
        k_scan_down<<<(unsigned)nb, kScanT, 0, st>>>(f, N, boff, out, with_total ? 1 : 0);
        e = cudaGetLastError();
    }
    cudaFreeAsync(bsum, st);
    cudaFreeAsync(boff, st);
    return e;
}

// ------------------------------------------------------------------ expand
__global__ void k_expand_coo(const int* __restrict__ src, const int* __restrict__ dst, long long S,
                             int n, unsigned long long* __restrict__ keys, int* bad) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S;
         i += (long long)gridDim.x * blockDim.x) {
        const int s = src[i], d = dst[i];
        unsigned long long a = kSentinel, b = kSentinel;
        if ((unsigned)s >= (unsigned)n || (unsigned)d >= (unsigned)n) {
            *bad = 1;
        } else if (s != d) {
            a = ((unsigned long long)(unsigned)s << 32) | (unsigned)d;
            b = ((unsigned long long)(unsigned)d << 32) | (unsigned)s;
        }
        keys[2 * i] = a;
        keys[2 * i + 1] = b;
    }
}

template <typename Off>
__global__ void k_check_rowptr(const Off* __restrict__ rp, int n, long long nnz, int* bad) {
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n;
         u += (long long)gridDim.x * blockDim.x) {
        if (rp[u + 1] < rp[u]) *bad = 1;
        if (u == 0 && rp[0] != 0) *bad = 1;
        if (u == n - 1 && (long long)rp[n] != nnz) *bad = 1;
    }
}

template <typename Off>
__global__ void k_expand_csr(const Off* __restrict__ rp, const int* __restrict__ col, int n,
                             unsigned long long* __restrict__ keys, int* bad) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long u = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        const long long b = rp[u], e = rp[u + 1];
        for (long long j = b + lane; j < e; j += 32) {
            const int v = col[j];
            unsigned long long x = kSentinel, y = kSentinel;
            if ((unsigned)v >= (unsigned)n) {
                *bad = 1;
            } else if (v != (int)u) {
                x = ((unsigned long long)u << 32) | (unsigned)v;
                y = ((unsigned long long)(unsigned)v << 32) | (unsigned long long)u;
            }
            keys[2 * j] = x;
            keys[2 * j + 1] = y;
        }
    }
}

// ------------------------------------------------------------------ radix sort
constexpr int kRsT = 512, kRsWarps = kRsT / 32, kRsKpt = 8, kRsTile = kRsT * kRsKpt;

__global__ void __launch_bounds__(kRsT) k_rs_hist(const unsigned long long* __restrict__ keys,
                                                  long long N, int shift, uint32_t* hist,
                                                  long long nt) {
    __shared__ uint32_t sh[256];
    for (int d = threadIdx.x; d < 256; d += kRsT) sh[d] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kRsTile;
#pragma unroll
    for (int i = 0; i < kRsKpt; i++) {
        const long long idx = base + (long long)i * kRsT + threadIdx.x;
        if (idx < N) atomicAdd(&sh[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += kRsT) hist[(long long)d * nt + blockIdx.x] = sh[d];
}

// Stable scatter: within a tile, warp w owns keys [w*256, w*256+256) and walks
// them in 8 rounds of 32; ranks follow (warp, round, lane) = input order.
__global__ void __launch_bounds__(kRsT) k_rs_scatter(const unsigned long long* __restrict__ in,
                                                     unsigned long long* __restrict__ out,
                                                     long long N, int shift,
                                                     const uint32_t* __restrict__ off,
                                                     long long nt) {
    __shared__ uint32_t wc[kRsWarps][256];
    __shared__ uint32_t soff[256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsT) (&wc[0][0])[i] = 0;
    for (int d = threadIdx.x; d < 256; d += kRsT) soff[d] = off[(long long)d * nt + blockIdx.x];
    __syncthreads();
    const unsigned lt_mask = (1u << lane) - 1u;
    const long long base = (long long)blockIdx.x * kRsTile + (long long)w * (32 * kRsKpt);
    unsigned long long key[kRsKpt];
    uint32_t rank[kRsKpt];
    int dig[kRsKpt];
#pragma unroll
    for (int r = 0; r < kRsKpt; r++) {
        const long long idx = base + r * 32 + lane;
        const bool valid = idx < N;
        const unsigned long long k = valid ? in[idx] : 0ull;
        const int d = valid ? (int)((k >> shift) & 255u) : 256 + lane;
        const unsigned peers = __match_any_sync(kFull, d);
        const unsigned lower = peers & lt_mask;
        uint32_t before = valid ? wc[w][d] : 0u;
        __syncwarp();
        if (valid && lower == 0) wc[w][d] = before + (uint32_t)__popc(peers);
        __syncwarp();
        key[r] = k;
        rank[r] = before + (uint32_t)__popc(lower);
        dig[r] = valid ? d : -1;
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += kRsT) {
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < kRsWarps; ww++) {
            const uint32_t c = wc[ww][d];
            wc[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRsKpt; r++)
        if (dig[r] >= 0) out[(long long)soff[dig[r]] + wc[w][dig[r]] + rank[r]] = key[r];
}

// Sorts keys[0..N) by the bits vertex ids use; returns the buffer holding the
// result (keys or alt).
cudaError_t radix_sort(unsigned long long* keys, unsigned long long* alt, long long N, int idbits,
                       cudaStream_t st, unsigned long long** result) {
    *result = keys;
    if (N <= 1 || idbits <= 0) return cudaSuccess;
    const long long nt = (N + kRsTile - 1) / kRsTile;
    uint32_t *hist = nullptr, *off = nullptr;
    cudaError_t e = cudaMallocAsync(&hist, sizeof(uint32_t) * 256 * nt, st);
    if (e != cudaSuccess) return e;
    e = cudaMallocAsync(&off, sizeof(uint32_t) * 256 * nt, st);
    if (e != cudaSuccess) { cudaFreeAsync(hist, st); return e; }
    std::vector<int> shifts;
    for (int s = 0; s < idbits; s += 8) shifts.push_back(s);
    for (int s = 0; s < idbits; s += 8) shifts.push_back(32 + s);
    unsigned long long *a = keys, *b = alt;
    for (int sh : shifts) {
        k_rs_hist<<<(unsigned)nt, kRsT, 0, st>>>(a, N, sh, hist, nt);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        e = exclusive_scan(ReadU32{hist}, 256 * nt, off, false, st);
        if (e != cudaSuccess) break;
        k_rs_scatter<<<(unsigned)nt, kRsT, 0, st>>>(a, b, N, sh, off, nt);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        std::swap(a, b);
    }
    cudaFreeAsync(hist, st);
    cudaFreeAsync(off, st);
    *result = a;
    return e;
}

// ------------------------------------------------------------------ dedupe, rows
struct KeepFlag {
    const unsigned long long* k;
    __device__ unsigned long long operator()(long long i) const {
        const unsigned long long x = k[i];
        return (x != kSentinel && (i == 0 || k[i - 1] != x)) ? 1ull : 0ull;
    }
};

__global__ void k_compact(const unsigned long long* __restrict__ k, long long N,
                          const uint32_t* __restrict__ pos, int* __restrict__ col,
                          uint32_t* __restrict__ rfirst, uint32_t* __restrict__ rlast) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long x = k[i];
        if (x == kSentinel) continue;
        const uint32_t u = (uint32_t)(x >> 32);
        const bool keep = (i == 0 || k[i - 1] != x);
        if (keep) col[pos[i]] = (int)(uint32_t)(x & 0xffffffffu);
        if (i == 0 || (uint32_t)(k[i - 1] >> 32) != u) rfirst[u] = pos[i];
        if (i + 1 == N || (uint32_t)(k[i + 1] >> 32) != u) rlast[u] = pos[i] + (keep ? 1u : 0u);
    }
}

struct RowDeg {
    const uint32_t* f;
    const uint32_t* l;
    __device__ unsigned long long operator()(long long u) const { return l[u] - f[u]; }
};

template <typename Off>
__global__ void k_check_clean(const Off* __restrict__ rp, const int* __restrict__ col, int n,
                              int* bad) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long u = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        const long long b = rp[u], e = rp[u + 1];
        for (long long j = b + lane; j < e; j += 32) {
            const int v = col[j];
            if ((unsigned)v >= (unsigned)n || v == (int)u) *bad = 1;
            if (j > b && col[j - 1] >= v) *bad = 1;
        }
    }
}

// ------------------------------------------------------------------ tier split
constexpr int kTsT = 1024;

template <typename Off>
__device__ __forceinline__ int tier_of(long long d, int t_lo, int t_hi) {
    return d <= t_lo ? 0 : (d <= t_hi ? 1 : 2);
}

template <typename Off>
__global__ void __launch_bounds__(kTsT) k_tier_count(const Off* __restrict__ rp, int n, int t_lo,
                                                     int t_hi, uint32_t* cnt, int nb) {
    __shared__ uint32_t c[kTiers];
    if (threadIdx.x < kTiers) c[threadIdx.x] = 0;
    __syncthreads();
    const long long v = (long long)blockIdx.x * kTsT + threadIdx.x;
    if (v < n) atomicAdd(&c[tier_of<Off>((long long)(rp[v + 1] - rp[v]), t_lo, t_hi)], 1u);
    __syncthreads();
    if (threadIdx.x < kTiers) cnt[threadIdx.x * nb + blockIdx.x] = c[threadIdx.x];
}

template <typename Off>
__global__ void __launch_bounds__(kTsT) k_tier_write(const Off* __restrict__ rp, int n, int t_lo,
                                                     int t_hi, const uint32_t* __restrict__ off,
                                                     int nb, uint32_t* __restrict__ est0,
                                                     int* __restrict__ list) {
    __shared__ uint32_t wcnt[kTiers][kTsT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long v = (long long)blockIdx.x * kTsT + threadIdx.x;
    const bool valid = v < n;
    const long long d = valid ? (long long)(rp[v + 1] - rp[v]) : 0;
    const int t = valid ? tier_of<Off>(d, t_lo, t_hi) : -1;
    unsigned mine = 0;
#pragma unroll
    for (int q = 0; q < kTiers; q++) {
        const unsigned m = __ballot_sync(kFull, t == q);
        if (lane == 0) wcnt[q][w] = __popc(m);
        if (t == q) mine = __popc(m & ((1u << lane) - 1u));
    }
    __syncthreads();
    if (valid) {
        uint32_t before = 0;
        for (int ww = 0; ww < w; ww++) before += wcnt[t][ww];
        est0[v] = ((uint32_t)t << kEstBits) | (uint32_t)d;
        list[off[t * nb + blockIdx.x] + before + mine] = (int)v;
    }
}

int id_bits(long long n) {
    int b = 0;
    while ((1ll << b) < n) b++;
    return b;
}

struct Temp {
    cudaStream_t st;
    std::vector<void*> ptrs;
    explicit Temp(cudaStream_t s) : st(s) {}
    ~Temp() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
    template <typename T>
    cudaError_t get(T** p, size_t count) {
        cudaError_t e = cudaMallocAsync((void**)p, std::max<size_t>(count, 1) * sizeof(T), st);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};

kcore_status cuda_fail(cudaError_t e, const char* what, std::string* err) {
    *err = std::string(what) + ": " + cudaGetErrorString(e);
    return (e == cudaErrorMemoryAllocation) ? KCORE_ERR_OOM : KCORE_ERR_CUDA;
}

#define KC_TRY(call, what)                                   \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, what, err); \
    } while (0)

// keys[0..N) -> clean CSR.
kcore_status finish_from_keys(Temp& tmp, int64_t n, unsigned long long* keys, long long N,
                              int off_bytes, cudaStream_t st, DevCsr* out, std::string* err) {
    unsigned long long* alt = nullptr;
    KC_TRY(tmp.get(&alt, (size_t)N), "sort buffer");
    unsigned long long* sorted = keys;
    KC_TRY(radix_sort(keys, alt, N, id_bits(n), st, &sorted), "radix sort");
    uint32_t *pos = nullptr, *rfirst = nullptr, *rlast = nullptr;
    KC_TRY(tmp.get(&pos, (size_t)N + 1), "positions");
    KC_TRY(exclusive_scan(KeepFlag{sorted}, N, pos, true, st), "dedupe scan");
    uint32_t total = 0;
    KC_TRY(cudaMemcpyAsync(&total, pos + N, sizeof(uint32_t), cudaMemcpyDeviceToHost, st), "read size");
    KC_TRY(cudaStreamSynchronize(st), "sync");
    if (off_bytes == 4 && total > 0x7fffffffu) {
        *err = "cleaned graph has 2m >= 2^31 entries; use 8-byte row_ptr";
        return KCORE_ERR_INVALID;
    }
    KC_TRY(tmp.get(&rfirst, (size_t)n), "row bounds");
    KC_TRY(tmp.get(&rlast, (size_t)n), "row bounds");
    KC_TRY(cudaMemsetAsync(rfirst, 0, sizeof(uint32_t) * std::max<int64_t>(n, 1), st), "memset");
    KC_TRY(cudaMemsetAsync(rlast, 0, sizeof(uint32_t) * std::max<int64_t>(n, 1), st), "memset");
    kcore_status s = dmalloc((void**)&out->col, sizeof(int) * std::max<size_t>(total, 1), err);
    if (s != KCORE_OK) return s;
    s = dmalloc(&out->row_ptr, (size_t)off_bytes * (n + 1), err);
    if (s != KCORE_OK) return s;
    if (N > 0) {
        const int g = (int)std::min<long long>((N + 255) / 256, 152LL * 64);
        k_compact<<<g, 256, 0, st>>>(sorted, N, pos, out->col, rfirst, rlast);
        KC_TRY(cudaGetLastError(), "compact");
    }
    if (off_bytes == 8)
        KC_TRY(exclusive_scan(RowDeg{rfirst, rlast}, n, (long long*)out->row_ptr, true, st), "row scan");
    else
        KC_TRY(exclusive_scan(RowDeg{rfirst, rlast}, n, (int*)out->row_ptr, true, st), "row scan");
    KC_TRY(cudaStreamSynchronize(st), "sync");
    out->n = n;
    out->nnz = total;
    out->off_bytes = off_bytes;
    return KCORE_OK;
}

}  // namespace

kcore_status dmalloc(void** p, size_t bytes, std::string* err) {
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        *err = std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? KCORE_ERR_OOM : KCORE_ERR_CUDA;
    }
    return KCORE_OK;
}

void dfree(void* p) {
    if (p) cudaFree(p);
}

cudaError_t scan_u32_to_u64(const uint32_t* in, unsigned long long* out, long long N,
                            cudaStream_t st) {
    return exclusive_scan(ReadU32{in}, N, out, true, st);
}

kcore_status clean_from_coo(int64_t n, int64_t samples, const int* src, const int* dst,
                            int off_bytes, cudaStream_t st, DevCsr* out, std::string* err) {
    if (samples > 0x7fffffffLL) {
        *err = "at most 2^31-1 samples per graph";
        return KCORE_ERR_INVALID;
    }
    Temp tmp(st);
    const long long N = 2 * (long long)samples;
    unsigned long long* keys = nullptr;
    int* bad = nullptr;
    KC_TRY(tmp.get(&keys, (size_t)N), "key buffer");
    KC_TRY(tmp.get(&bad, 1), "flag");
    KC_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st), "memset");
    if (samples > 0) {
        const int g = (int)std::min<long long>((samples + 255) / 256, 152LL * 64);
        k_expand_coo<<<g, 256, 0, st>>>(src, dst, samples, (int)n, keys, bad);
        KC_TRY(cudaGetLastError(), "expand");
    }
    int hbad = 0;
    KC_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st), "read flag");
    KC_TRY(cudaStreamSynchronize(st), "sync");
    if (hbad) {
        *err = "edge endpoint outside [0, n)";
        return KCORE_ERR_INVALID;
    }
    return finish_from_keys(tmp, n, keys, N, off_bytes, st, out, err);
}

kcore_status clean_from_csr(int64_t n, const void* row_ptr, int in_off_bytes, const int* col,
                            int64_t nnz, int off_bytes, cudaStream_t st, DevCsr* out,
                            std::string* err) {
    if (nnz > 0x7fffffffLL) {
        *err = "at most 2^31-1 input entries per graph";
        return KCORE_ERR_INVALID;
    }
    Temp tmp(st);
    int* bad = nullptr;
    KC_TRY(tmp.get(&bad, 1), "flag");
    KC_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st), "memset");
    const int g = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 64));
    if (n > 0) {
        if (in_off_bytes == 8)
            k_check_rowptr<<<g, 256, 0, st>>>((const long long*)row_ptr, (int)n, nnz, bad);
        else
            k_check_rowptr<<<g, 256, 0, st>>>((const int*)row_ptr, (int)n, nnz, bad);
        KC_TRY(cudaGetLastError(), "check row_ptr");
    }
    int hbad = 0;
    KC_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st), "read flag");
    KC_TRY(cudaStreamSynchronize(st), "sync");
    if (hbad) {
        *err = "row_ptr must start at 0, be non-decreasing and end at nnz";
        return KCORE_ERR_INVALID;
    }
    const long long N = 2 * (long long)nnz;
    unsigned long long* keys = nullptr;
    KC_TRY(tmp.get(&keys, (size_t)N), "key buffer");
    if (n > 0 && nnz > 0) {
        if (in_off_bytes == 8)
            k_expand_csr<<<g, 256, 0, st>>>((const long long*)row_ptr, col, (int)n, keys, bad);
        else
            k_expand_csr<<<g, 256, 0, st>>>((const int*)row_ptr, col, (int)n, keys, bad);
        KC_TRY(cudaGetLastError(), "expand");
    }
    KC_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st), "read flag");
    KC_TRY(cudaStreamSynchronize(st), "sync");
    if (hbad) {
        *err = "col_idx entry outside [0, n)";
        return KCORE_ERR_INVALID;
    }
    return finish_from_keys(tmp, n, keys, N, off_bytes, st, out, err);
}

kcore_status check_clean_csr(int64_t n, const void* row_ptr, int off_bytes, const int* col,
                             int64_t nnz, cudaStream_t st, std::string* err) {
    Temp tmp(st);
    int* bad = nullptr;
    KC_TRY(tmp.get(&bad, 1), "flag");
    KC_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st), "memset");
    const int g = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 64));
    if (n > 0) {
        if (off_bytes == 8) {
            k_check_rowptr<<<g, 256, 0, st>>>((const long long*)row_ptr, (int)n, nnz, bad);
            k_check_clean<<<g, 256, 0, st>>>((const long long*)row_ptr, col, (int)n, bad);
        } else {
            k_check_rowptr<<<g, 256, 0, st>>>((const int*)row_ptr, (int)n, nnz, bad);
            k_check_clean<<<g, 256, 0, st>>>((const int*)row_ptr, col, (int)n, bad);
        }
        KC_TRY(cudaGetLastError(), "check");
    }
    int hbad = 0;
    KC_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st), "read flag");
    KC_TRY(cudaStreamSynchronize(st), "sync");
    if (hbad) {
        *err = "KCORE_IN_CLEAN graph has an unsorted row, a repeat, a self-loop or a bad id";
        return KCORE_ERR_INVALID;
    }
    return KCORE_OK;
}

kcore_status tier_split(int64_t n, const void* row_ptr, int off_bytes, int t_lo, int t_hi,
                        uint32_t* est0, int* init_list, long long tier_cnt[kTiers],
                        cudaStream_t st, std::string* err) {
    for (int q = 0; q < kTiers; q++) tier_cnt[q] = 0;
    if (n == 0) return KCORE_OK;
    Temp tmp(st);
    const int nb = (int)((n + kTsT - 1) / kTsT);
    uint32_t *cnt = nullptr, *off = nullptr;
    KC_TRY(tmp.get(&cnt, (size_t)kTiers * nb), "tier counts");
    KC_TRY(tmp.get(&off, (size_t)kTiers * nb + 1), "tier offsets");
    if (off_bytes == 8)
        k_tier_count<<<nb, kTsT, 0, st>>>((const long long*)row_ptr, (int)n, t_lo, t_hi, cnt, nb);
    else
        k_tier_count<<<nb, kTsT, 0, st>>>((const int*)row_ptr, (int)n, t_lo, t_hi, cnt, nb);
    KC_TRY(cudaGetLastError(), "tier count");
    KC_TRY(exclusive_scan(ReadU32{cnt}, (long long)kTiers * nb, off, true, st), "tier scan");
    if (off_bytes == 8)
        k_tier_write<<<nb, kTsT, 0, st>>>((const long long*)row_ptr, (int)n, t_lo, t_hi, off, nb,
                                          est0, init_list);
    else
        k_tier_write<<<nb, kTsT, 0, st>>>((const int*)row_ptr, (int)n, t_lo, t_hi, off, nb, est0,
                                          init_list);
    KC_TRY(cudaGetLastError(), "tier write");
    std::vector<uint32_t> h(kTiers + 1);
    for (int q = 0; q <= kTiers; q++) {
        const long long idx = (q < kTiers) ? (long long)q * nb : (long long)kTiers * nb;
        KC_TRY(cudaMemcpyAsync(&h[q], off + idx, sizeof(uint32_t), cudaMemcpyDeviceToHost, st),
               "read tier offsets");
    }
    KC_TRY(cudaStreamSynchronize(st), "sync");
    for (int q = 0; q < kTiers; q++) tier_cnt[q] = (long long)h[q + 1] - h[q];
    return KCORE_OK;
}

}  // namespace kc
