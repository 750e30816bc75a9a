// Device CSR cleaning (Sec. IV-A: graphs treated as undirected, self-loops
// removed; Sec. III-B: neighbour lists kept as sorted vectors).
//
// Two pipelines give the same CSR, all on the device.
//
// Counted (raw CSR input, and edge samples whose rows are mostly short):
//   1. count    every sample (u, v) with u != v adds one to deg(u) and deg(v)
//               (atomics); ids outside [0, n) raise a flag and are skipped.
//   2. offsets  exclusive scan of the counts: the segment of each row; the
//               rows longer than 32 entries are listed by size class and the
//               classes copied to the host while steps 3-4 run.
//   3. scatter  each sample writes v into u's segment and u into v's, at a slot
//               taken with an atomic on the row's fill counter (unordered).
//   4. sort     each segment is sorted and its repeats dropped in place, by a
//               size class: one thread with a register sorting network (<= 32
//               entries), one warp with a register bitonic sort (<= 1024), one
//               CTA with shared-memory merges (<= 16384), and, for the few
//               larger hub rows, a stable LSD radix sort of 64-bit
//               (row rank, column) keys over the whole GPU.
//   5. rows     exclusive scan of the distinct counts gives row_ptr; the
//               sorted distinct prefixes are copied into col_idx.
//
// Sorted (edge samples where rows of more than 32 entries hold most entries):
// every sample becomes one canonical 64-bit key (min << 32 | max); an LSD
// radix sort over both ids orders them; a pass drops repeats and writes each
// distinct edge (a, b) twice, as is and transposed (b, a); a radix sort of
// the transposes over the row bits alone orders them by (b, a).  Row r is
// then its smaller neighbours (the transposes with row r) followed by its
// larger ones (the canonical keys with row r), both already ascending; two
// passes place them, and a scan of the row lengths gives row_ptr.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>
#include <string>
#include <vector>

#include "kc_common.cuh"

namespace kc {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kPad = 0xffffffffu;       // sorts after every vertex id
constexpr int kSmallMax = 32, kMidMax = 1024, kBigMax = 16384;
constexpr int kBigT = 512;
constexpr long long kSortAutoSamples = 1 << 18, kSortAutoDegree = 8;
constexpr int kSortProbe = 16;

// ------------------------------------------------------------------ temporaries
// The temporaries of one call, freed together (stream-ordered) when it ends.
// reserve() takes one block from the pool and get() carves 256-byte aligned
// arrays from it, so that a call makes a few allocations instead of one per
// array; a request that does not fit the block gets its own allocation.
struct Temp {
    cudaStream_t st;
    std::vector<void*> ptrs;
    char* base = nullptr;
    size_t cap = 0, used = 0;
    explicit Temp(cudaStream_t s) : st(s) {}
    ~Temp() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
    static size_t round(size_t bytes) { return (std::max<size_t>(bytes, 1) + 255) & ~size_t(255); }
    cudaError_t reserve(size_t bytes) {
        char* b = nullptr;
        cudaError_t e = pool_alloc((void**)&b, bytes, st);
        if (e != cudaSuccess) return e;
        ptrs.push_back(b);
        base = b;
        cap = bytes;
        used = 0;
        return cudaSuccess;
    }
    template <typename T>
    cudaError_t get(T** p, size_t count) {
        const size_t bytes = round(std::max<size_t>(count, 1) * sizeof(T));
        if (base && used + bytes <= cap) {
            *p = reinterpret_cast<T*>(base + used);
            used += bytes;
            return cudaSuccess;
        }
        cudaError_t e = pool_alloc((void**)p, bytes, st);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};

// Build state on the device: the error flag and the class lists of the rows
// that one thread does not sort.
struct BuildCtl {
    int bad;               // an id or offset out of range
    unsigned n_mid, n_big, n_huge;
    unsigned long long huge_entries;
    unsigned long long entries, heavy;  // all counted entries; those in rows above kSmallMax
};

// Rows longer than kSmallMax, listed by size class (row u of length len).
__device__ __forceinline__ void classify_row(long long u, uint32_t len, int* mid, int* big, int* huge,
                                             BuildCtl* bc) {
    if (len <= (uint32_t)kSmallMax) return;
    if (len <= (uint32_t)kMidMax) {
        mid[atomicAdd(&bc->n_mid, 1u)] = (int)u;
    } else if (len <= (uint32_t)kBigMax) {
        big[atomicAdd(&bc->n_big, 1u)] = (int)u;
    } else {
        huge[atomicAdd(&bc->n_huge, 1u)] = (int)u;
        atomicAdd(&bc->huge_entries, (unsigned long long)len);
    }
}

// Work a scan's down-sweep does on each input element: nothing, or (for the
// row offsets) listing the long rows, whose lengths are the scanned counts.
struct NoEpi {
    __device__ __forceinline__ void operator()(long long, uint32_t) const {}
};
struct ClassifyEpi {
    int *mid, *big, *huge;
    BuildCtl* bc;
    __device__ __forceinline__ void operator()(long long u, uint32_t len) const {
        classify_row(u, len, mid, big, huge, bc);
    }
};

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

template <typename Out, typename Epi = NoEpi>
cudaError_t exclusive_scan4(const uint32_t* in, long long N, Out* out, bool with_total, cudaStream_t st,
                            Temp* tmp, Epi epi = Epi());

// Block sums and their offsets of one scan level (from `tmp` when given).
inline cudaError_t scan_scratch(long long nb, unsigned long long** bsum, unsigned long long** boff,
                                cudaStream_t st, Temp* tmp) {
    if (tmp) {
        cudaError_t e = tmp->get(bsum, (size_t)nb);
        return e == cudaSuccess ? tmp->get(boff, (size_t)nb + 1) : e;
    }
    cudaError_t e = pool_alloc((void**)bsum, sizeof(unsigned long long) * nb, st);
    if (e != cudaSuccess) return e;
    e = pool_alloc((void**)boff, sizeof(unsigned long long) * (nb + 1), st);
    if (e != cudaSuccess) cudaFreeAsync(*bsum, st);
    return e;
}
inline void scan_scratch_free(unsigned long long* bsum, unsigned long long* boff, cudaStream_t st,
                              Temp* tmp) {
    if (tmp) return;
    cudaFreeAsync(bsum, st);
    cudaFreeAsync(boff, st);
}

// 32-bit inputs with 16-byte aligned arrays: each thread takes 4 consecutive
// elements in one 16-byte access, so a warp reads (and writes) contiguous
// bytes instead of every lane striding through its own chunk.
constexpr int kVecT = 512, kVecTile = kVecT * 4;

__device__ __forceinline__ uint4 load4(const uint32_t* p, long long i, long long N) {
    if (i + 4 <= N) return *reinterpret_cast<const uint4*>(p + i);
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (i < N) v.x = p[i];
    if (i + 1 < N) v.y = p[i + 1];
    if (i + 2 < N) v.z = p[i + 2];
    return v;
}

template <typename Out>
__device__ __forceinline__ void store4(Out* out, long long i, long long N, unsigned long long a,
                                      unsigned long long b, unsigned long long c,
                                      unsigned long long d) {
    if (i + 4 <= N) {
        if constexpr (sizeof(Out) == 4) {
            *reinterpret_cast<uint4*>(out + i) = make_uint4((uint32_t)a, (uint32_t)b, (uint32_t)c, (uint32_t)d);
        } else {
            *reinterpret_cast<ulonglong2*>(out + i) = make_ulonglong2(a, b);
            *reinterpret_cast<ulonglong2*>(out + i + 2) = make_ulonglong2(c, d);
        }
        return;
    }
    if (i < N) out[i] = (Out)a;
    if (i + 1 < N) out[i + 1] = (Out)b;
    if (i + 2 < N) out[i + 2] = (Out)c;
}

__global__ void __launch_bounds__(kVecT) k_scan_reduce4(const uint32_t* __restrict__ in, long long N,
                                                        unsigned long long* bsum) {
    const uint4 v = load4(in, (long long)blockIdx.x * kVecTile + threadIdx.x * 4, N);
    unsigned long long tot;
    block_excl_scan((unsigned long long)v.x + v.y + v.z + v.w, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

template <typename Out, typename Epi>
__global__ void __launch_bounds__(kVecT) k_scan_down4(const uint32_t* __restrict__ in, long long N,
                                                      const unsigned long long* boff, Out* out,
                                                      int write_total, Epi epi) {
    const long long i = (long long)blockIdx.x * kVecTile + threadIdx.x * 4;
    const uint4 v = load4(in, i, N);
    if (i < N) epi(i, v.x);
    if (i + 1 < N) epi(i + 1, v.y);
    if (i + 2 < N) epi(i + 2, v.z);
    if (i + 3 < N) epi(i + 3, v.w);
    unsigned long long tot;
    const unsigned long long b0 = boff ? boff[blockIdx.x] : 0ull;
    const unsigned long long r0 = block_excl_scan((unsigned long long)v.x + v.y + v.z + v.w, &tot) + b0;
    store4(out, i, N, r0, r0 + v.x, r0 + v.x + v.y, r0 + v.x + v.y + v.z);
    if (write_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1)
        out[N] = (Out)(b0 + tot);
}

// out[0..N) = exclusive prefix sums of f(0..N); out[N] = total if with_total.
// Scratch comes from `tmp` when given (no allocation of its own).
template <typename F, typename Out>
cudaError_t exclusive_scan(F f, long long N, Out* out, bool with_total, cudaStream_t st,
                           Temp* tmp = nullptr) {
    if (N <= 0) {
        if (with_total) return cudaMemsetAsync(out, 0, sizeof(Out), st);
        return cudaSuccess;
    }
    if constexpr (std::is_same<F, ReadU32>::value) {
        if ((reinterpret_cast<uintptr_t>(f.p) | reinterpret_cast<uintptr_t>(out)) % 16 == 0)
            return exclusive_scan4(f.p, N, out, with_total, st, tmp);
    }
    const long long nb = (N + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        k_scan_down<<<1, kScanT, 0, st>>>(f, N, (const unsigned long long*)nullptr, out,
                                          with_total ? 1 : 0);
        count_launch();
        return cudaGetLastError();
    }
    unsigned long long *bsum = nullptr, *boff = nullptr;
    cudaError_t e = scan_scratch(nb, &bsum, &boff, st, tmp);
    if (e != cudaSuccess) return e;
    k_scan_reduce<<<(unsigned)nb, kScanT, 0, st>>>(f, N, bsum);
    count_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess) e = exclusive_scan(ReadU64{bsum}, nb, boff, false, st, tmp);
    if (e == cudaSuccess) {
        k_scan_down<<<(unsigned)nb, kScanT, 0, st>>>(f, N, boff, out, with_total ? 1 : 0);
        count_launch();
        e = cudaGetLastError();
    }
    scan_scratch_free(bsum, boff, st, tmp);
    return e;
}

template <typename Out, typename Epi>
cudaError_t exclusive_scan4(const uint32_t* in, long long N, Out* out, bool with_total, cudaStream_t st,
                            Temp* tmp, Epi epi) {
    const long long nb = (N + kVecTile - 1) / kVecTile;
    if (nb == 1) {
        k_scan_down4<<<1, kVecT, 0, st>>>(in, N, (const unsigned long long*)nullptr, out,
                                          with_total ? 1 : 0, epi);
        count_launch();
        return cudaGetLastError();
    }
    unsigned long long *bsum = nullptr, *boff = nullptr;
    cudaError_t e = scan_scratch(nb, &bsum, &boff, st, tmp);
    if (e != cudaSuccess) return e;
    k_scan_reduce4<<<(unsigned)nb, kVecT, 0, st>>>(in, N, bsum);
    count_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess) e = exclusive_scan(ReadU64{bsum}, nb, boff, false, st, tmp);
    if (e == cudaSuccess) {
        k_scan_down4<<<(unsigned)nb, kVecT, 0, st>>>(in, N, boff, out, with_total ? 1 : 0, epi);
        count_launch();
        e = cudaGetLastError();
    }
    scan_scratch_free(bsum, boff, st, tmp);
    return e;
}

// Scratch bytes an exclusive scan of N 32-bit elements takes from a Temp.
size_t scan_scratch_bytes(long long N) {
    size_t b = 0;
    long long nb = (N + kVecTile - 1) / kVecTile;
    while (nb > 1) {
        b += Temp::round(sizeof(unsigned long long) * nb) + Temp::round(sizeof(unsigned long long) * (nb + 1));
        nb = (nb + kScanTile - 1) / kScanTile;
    }
    return b;
}

// ------------------------------------------------------------------ count / scatter
// The samples of every step-th run of 256 (step 1: all of them); runs keep
// the reads coalesced when only a share of the samples is counted.
__global__ void k_count_coo(const int* __restrict__ src, const int* __restrict__ dst, long long S,
                            int n, uint32_t* __restrict__ cnt, BuildCtl* bc, int step) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;; j += (long long)gridDim.x * blockDim.x) {
        const long long i = ((j >> 8) * step << 8) | (j & 255);
        if (i >= S) break;
        const int s = src[i], d = dst[i];
        if ((unsigned)s >= (unsigned)n || (unsigned)d >= (unsigned)n) {
            bc->bad = 1;
            continue;
        }
        if (s == d) continue;
        atomicAdd(&cnt[s], 1u);
        atomicAdd(&cnt[d], 1u);
    }
}

// Entries in rows of more than `limit` entries, and all entries (one pair of
// atomics per block).
__global__ void k_heavy(const uint32_t* __restrict__ cnt, long long n, uint32_t limit, BuildCtl* bc) {
    __shared__ unsigned long long ws[2][32];
    unsigned long long all = 0, heavy = 0;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n;
         u += (long long)gridDim.x * blockDim.x) {
        const uint32_t c = cnt[u];
        all += c;
        heavy += c > limit ? c : 0u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        all += __shfl_down_sync(kFull, all, o);
        heavy += __shfl_down_sync(kFull, heavy, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        ws[0][w] = all;
        ws[1][w] = heavy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); q++) {
            all += ws[0][q];
            heavy += ws[1][q];
        }
        if (all) {
            atomicAdd(&bc->entries, all);
            atomicAdd(&bc->heavy, heavy);
        }
    }
}

__global__ void k_scatter_coo(const int* __restrict__ src, const int* __restrict__ dst, long long S,
                              int n, const uint32_t* __restrict__ off, uint32_t* __restrict__ fill,
                              uint32_t* __restrict__ seg) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S;
         i += (long long)gridDim.x * blockDim.x) {
        const int s = src[i], d = dst[i];
        if ((unsigned)s >= (unsigned)n || (unsigned)d >= (unsigned)n || s == d) continue;
        seg[off[s] + atomicAdd(&fill[s], 1u)] = (uint32_t)d;
        seg[off[d] + atomicAdd(&fill[d], 1u)] = (uint32_t)s;
    }
}

// Raw CSR input: one warp per row; offsets are checked and clamped so that a
// malformed row_ptr cannot index outside col_idx.
template <typename Off>
__device__ __forceinline__ bool row_range(const Off* rp, int n, long long nnz, long long u,
                                          long long* b, long long* e) {
    const long long lo = (long long)rp[u], hi = (long long)rp[u + 1];
    bool ok = lo >= 0 && hi >= lo && hi <= nnz;
    if (u == 0 && lo != 0) ok = false;
    if (u == n - 1 && hi != nnz) ok = false;
    *b = ok ? lo : 0;
    *e = ok ? hi : 0;
    return ok;
}

template <typename Off>
__global__ void k_count_csr(const Off* __restrict__ rp, const int* __restrict__ col, int n,
                            long long nnz, uint32_t* __restrict__ cnt, BuildCtl* bc) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long u = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        long long b, e;
        if (!row_range(rp, n, nnz, u, &b, &e)) {
            if (lane == 0) bc->bad = 1;
            continue;
        }
        unsigned own = 0;
        for (long long j = b + lane; j < e; j += 32) {
            const int v = col[j];
            if ((unsigned)v >= (unsigned)n) {
                bc->bad = 1;
                continue;
            }
            if (v == (int)u) continue;
            own++;
            atomicAdd(&cnt[v], 1u);
        }
        own = __reduce_add_sync(kFull, own);
        if (lane == 0 && own) atomicAdd(&cnt[u], own);
    }
}

template <typename Off>
__global__ void k_scatter_csr(const Off* __restrict__ rp, const int* __restrict__ col, int n,
                              long long nnz, const uint32_t* __restrict__ off,
                              uint32_t* __restrict__ fill, uint32_t* __restrict__ seg) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long u = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        long long b, e;
        if (!row_range(rp, n, nnz, u, &b, &e)) continue;
        for (long long j0 = b; j0 < e; j0 += 32) {
            const long long j = j0 + lane;
            int v = -1;
            if (j < e) v = col[j];
            const bool ok = j < e && (unsigned)v < (unsigned)n && v != (int)u;
            const unsigned m = __ballot_sync(kFull, ok);
            unsigned base = 0;
            if (lane == 0 && m) base = atomicAdd(&fill[u], (unsigned)__popc(m));
            base = __shfl_sync(kFull, base, 0);
            if (ok) {
                seg[off[u] + base + __popc(m & ((1u << lane) - 1u))] = (uint32_t)v;
                seg[off[v] + atomicAdd(&fill[v], 1u)] = (uint32_t)u;
            }
        }
    }
}

// ------------------------------------------------------------------ segment sorts
// Bitonic network over P registers (every index is a compile-time constant).
template <int P>
__device__ __forceinline__ void sort_regs(uint32_t (&x)[P]) {
#pragma unroll
    for (int k = 2; k <= P; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int i = 0; i < P; i++) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const uint32_t a = x[i], b = x[l];
                    if ((a > b) == up) {
                        x[i] = b;
                        x[l] = a;
                    }
                }
            }
}

template <int P>
__device__ __forceinline__ uint32_t thread_sort_row(uint32_t* seg, int len) {
    uint32_t x[P];
#pragma unroll
    for (int i = 0; i < P; i++) x[i] = i < len ? seg[i] : kPad;
    sort_regs<P>(x);
    uint32_t c = 0;
#pragma unroll
    for (int i = 0; i < P; i++)
        if (i < len && (i == 0 || x[i] != x[i - 1])) seg[c++] = x[i];
    return c;
}

// Rows of at most 32 entries are sorted here; larger ones are listed by class.
__global__ void k_sort_small(int n, const uint32_t* __restrict__ off, uint32_t* __restrict__ seg,
                             uint32_t* __restrict__ ucnt) {
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n;
         u += (long long)gridDim.x * blockDim.x) {
        const uint32_t o = off[u];
        const int len = (int)(off[u + 1] - o);
        uint32_t* s = seg + o;
        if (len <= 1) {
            ucnt[u] = (uint32_t)len;
        } else if (len <= 4) {
            ucnt[u] = thread_sort_row<4>(s, len);
        } else if (len <= 8) {
            ucnt[u] = thread_sort_row<8>(s, len);
        } else if (len <= 16) {
            ucnt[u] = thread_sort_row<16>(s, len);
        } else if (len <= kSmallMax) {
            ucnt[u] = thread_sort_row<32>(s, len);
        }  // longer rows: listed by class after the offset scan, sorted by the class kernels
    }
}

// Lists the rows longer than kSmallMax by size class from the offsets alone,
// so that the host can read the classes while the scatter runs.  (Used when
// the offset scan cannot take its vector path, which lists them itself.)
__global__ void k_classify(int n, const uint32_t* __restrict__ off, int* __restrict__ mid,
                           int* __restrict__ big, int* __restrict__ huge, BuildCtl* bc) {
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n;
         u += (long long)gridDim.x * blockDim.x) {
        classify_row(u, off[u + 1] - off[u], mid, big, huge, bc);
    }
}

// Warp bitonic sort of 32*E values, blocked layout (lane holds positions
// lane*E .. lane*E+E-1); partners closer than E are in the same lane.
template <int E>
__device__ __forceinline__ void warp_sort(uint32_t (&x)[E]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32 * E; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= E) {
                const int lj = j / E;
                const bool lower = (lane & lj) == 0;
#pragma unroll
                for (int e = 0; e < E; e++) {
                    const int i = lane * E + e;
                    const bool up = (i & k) == 0;
                    const uint32_t y = __shfl_xor_sync(kFull, x[e], lj);
                    const uint32_t lo = min(x[e], y), hi = max(x[e], y);
                    x[e] = (lower == up) ? lo : hi;
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; e++) {
                    const int l = e ^ j;
                    if (l > e) {
                        const int i = lane * E + e;
                        const bool up = (i & k) == 0;
                        const uint32_t a = x[e], b = x[l];
                        if ((a > b) == up) {
                            x[e] = b;
                            x[l] = a;
                        }
                    }
                }
            }
        }
    }
}

template <int E>
__device__ __forceinline__ uint32_t warp_sort_row(uint32_t* seg, int len) {
    const int lane = threadIdx.x & 31;
    uint32_t x[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        const int i = lane * E + e;
        x[e] = i < len ? seg[i] : kPad;
    }
    warp_sort<E>(x);
    const uint32_t prev_last = __shfl_up_sync(kFull, x[E - 1], 1);
    unsigned keep = 0;
#pragma unroll
    for (int e = 0; e < E; e++) {
        const int i = lane * E + e;
        const uint32_t prev = e == 0 ? prev_last : x[e - 1];
        if (i < len && (i == 0 || x[e] != prev)) keep |= 1u << e;
    }
    const unsigned c = (unsigned)__popc(keep);
    unsigned incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    const unsigned total = __shfl_sync(kFull, incl, 31);
    __syncwarp();
    unsigned pos = incl - c;
#pragma unroll
    for (int e = 0; e < E; e++)
        if ((keep >> e) & 1u) seg[pos++] = x[e];
    return total;
}

// Rows of 33..1024 entries, one warp each.  Two instantiations split by row
// length (SHORT: up to 128), so that the many short rows do not run at the
// register count (and occupancy) of the 32-value sorts of the long ones.
constexpr int kMidShort = 128;

template <bool SHORT>
__global__ void k_sort_mid(const int* __restrict__ mid, const BuildCtl* bc,
                           const uint32_t* __restrict__ off, uint32_t* __restrict__ seg,
                           uint32_t* __restrict__ ucnt) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const unsigned nm = bc->n_mid;
    for (long long i = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; i < nm; i += warps) {
        const int u = mid[i];
        const uint32_t o = off[u];
        const int len = (int)(off[u + 1] - o);
        if ((len <= kMidShort) != SHORT) continue;
        uint32_t c;
        if (SHORT) {
            if (len <= 64) c = warp_sort_row<2>(seg + o, len);
            else c = warp_sort_row<4>(seg + o, len);
        } else {
            if (len <= 256) c = warp_sort_row<8>(seg + o, len);
            else if (len <= 512) c = warp_sort_row<16>(seg + o, len);
            else c = warp_sort_row<32>(seg + o, len);
        }
        if (lane == 0) ucnt[u] = c;
    }
}

// One CTA per row of 1025..16384 entries: every warp sorts 1024-entry blocks
// in registers (the warp bitonic sort), then log2(P / 1024) merge passes
// between two shared-memory buffers, each thread producing a contiguous
// stretch of the output after a merge-path search for its start; finally the
// repeats are dropped.  P = the row length rounded up to a power of two,
// padded with kPad.
__global__ void __launch_bounds__(kBigT) k_sort_big(const int* __restrict__ big, const BuildCtl* bc,
                                                    const uint32_t* __restrict__ off,
                                                    uint32_t* __restrict__ seg,
                                                    uint32_t* __restrict__ ucnt) {
    extern __shared__ uint32_t sm[];
    __shared__ unsigned long long wtot;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = kBigT >> 5;
    const unsigned nb = bc->n_big;
    for (unsigned r = blockIdx.x; r < nb; r += gridDim.x) {
        const int u = big[r];
        const uint32_t o = off[u];
        const int len = (int)(off[u + 1] - o);
        int P = 1024;
        while (P < len) P <<= 1;
        uint32_t* a = sm;
        uint32_t* b = sm + kBigMax;
        // 1024-entry blocks sorted by warps (blocked layout: lane holds 32 in a row)
        for (int blk = wid; blk * 1024 < P; blk += nw) {
            uint32_t x[32];
#pragma unroll
            for (int e = 0; e < 32; e++) {
                const int i = blk * 1024 + lane * 32 + e;
                x[e] = i < len ? seg[o + i] : kPad;
            }
            warp_sort<32>(x);
#pragma unroll
            for (int e = 0; e < 32; e++) a[blk * 1024 + lane * 32 + e] = x[e];
        }
        __syncthreads();
        // merge runs of width w into runs of 2w, a -> b, then swap
        for (int w = 1024; w < P; w <<= 1) {
            const int per = P / kBigT;
            const int i0 = tid * per;                // first output index of this thread
            const int base = i0 & ~(2 * w - 1);      // start of the pair of runs
            const int i = i0 - base;                 // position inside the merged pair
            const uint32_t* A = a + base;
            const uint32_t* B = a + base + w;
            int lo = max(0, i - w), hi = min(i, w);
            while (lo < hi) {  // number of entries taken from A before position i
                const int mid = (lo + hi) >> 1;
                if (A[mid] <= B[i - mid - 1]) lo = mid + 1;
                else hi = mid;
            }
            int ia = lo, ib = i - lo;
            for (int k = 0; k < per; k++) {
                const bool fromA = ib >= w || (ia < w && A[ia] <= B[ib]);
                b[i0 + k] = fromA ? A[ia++] : B[ib++];
            }
            __syncthreads();
            uint32_t* t = a;
            a = b;
            b = t;
        }
        // keep flags over each thread's contiguous chunk, then a block scan
        const int per = (len + kBigT - 1) / kBigT;
        const int j0 = min(len, tid * per), j1 = min(len, j0 + per);
        unsigned c = 0;
        for (int j = j0; j < j1; j++) c += (j == 0 || a[j] != a[j - 1]) ? 1u : 0u;
        unsigned long long tot;
        unsigned long long pos = block_excl_scan(c, &tot);
        for (int j = j0; j < j1; j++)
            if (j == 0 || a[j] != a[j - 1]) seg[o + pos++] = a[j];
        if (tid == 0) wtot = tot;
        __syncthreads();
        if (tid == 0) ucnt[u] = (uint32_t)wtot;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ LSD radix sort of 64-bit keys
// Tiles of kRsTile keys; one 8-bit digit per pass.  k_rs_hist counts each
// tile's digits; one exclusive scan of the digit-major count matrix gives the
// output start of every (digit, tile) run; k_rs_scatter ranks the tile's keys
// by digit (stable: in input order), stages them in shared memory in digit
// order and writes each digit's run contiguously.
constexpr int kRsT = 256, kRsWarps = kRsT / 32, kRsKpt = 16, kRsTile = kRsT * kRsKpt;
constexpr unsigned long long kNoKey = ~0ull;  // a dropped entry: sorts last

// The keys a pass reads: the previous pass's buffer.
struct KeyIn {
    const unsigned long long* k;
    __device__ __forceinline__ unsigned long long operator()(long long j) const { return k[j]; }
    __device__ __forceinline__ bool invalid(long long) const { return false; }
};

template <typename In>
__global__ void __launch_bounds__(kRsT) k_rs_hist(In keys, long long N, int shift, uint32_t* hist,
                                                  long long nt, int* bad) {
    __shared__ uint32_t sh[kRsWarps][256];  // one histogram per warp: fewer colliding adds
    const int w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kRsWarps; q++) sh[q][threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kRsTile;
    unsigned long long k[kRsKpt];
#pragma unroll
    for (int i = 0; i < kRsKpt; i++) {
        const long long idx = base + (long long)i * kRsT + threadIdx.x;
        k[i] = idx < N ? keys(idx) : 0ull;
        if (bad && idx < N && keys.invalid(idx)) *bad = 1;
    }
#pragma unroll
    for (int i = 0; i < kRsKpt; i++)
        if (base + (long long)i * kRsT + threadIdx.x < N) atomicAdd(&sh[w][(k[i] >> shift) & 255u], 1u);
    __syncthreads();
    uint32_t c = 0;
#pragma unroll
    for (int q = 0; q < kRsWarps; q++) c += sh[q][threadIdx.x];
    hist[(long long)threadIdx.x * nt + blockIdx.x] = c;
}

// Byte B of a 64-bit key (the digit of the pass at shift 8B).
template <int B>
__device__ __forceinline__ unsigned key_byte(unsigned long long k) {
    const uint32_t w = B < 4 ? (uint32_t)k : (uint32_t)(k >> 32);
    return __byte_perm(w, 0u, 0x4440u + (unsigned)(B & 3));
}

// One tile.  Warp w owns keys [w*512, w*512 + 512) of the tile and walks them
// in 16 rounds of 32; ranks follow (warp, round, lane), which is input order.
// The lanes holding the same digit in a round are found through a per-warp
// table of 256 words in shared memory: every lane writes its lane number into
// its digit's word and reads the word back; one writer per digit wins, so the
// number read is a label shared by exactly the lanes of that digit, and five
// ballots over its bits give the peers (eight would be needed over the digit
// itself; shared-memory atomics on the table cost more in bank conflicts).
// The tables live in the staging area, which is only written after the
// ranking.  FULL: the tile holds kRsTile keys (no bounds checks).
template <typename In, int B, bool FULL>
__device__ __forceinline__ void scatter_tile(const In& in, unsigned long long* __restrict__ out,
                                             long long N, long long tile0, uint32_t my_goff,
                                             unsigned long long* sk, uint32_t (*wc)[256],
                                             uint32_t* gd) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const long long base = tile0 + (long long)w * (32 * kRsKpt);
    unsigned long long key[kRsKpt];
    uint32_t rank[kRsKpt / 2];  // two 16-bit ranks (< kRsTile) per word
    // the tile's keys are fetched before any wait
#pragma unroll
    for (int r = 0; r < kRsKpt; r++) {
        const long long idx = base + r * 32 + lane;
        key[r] = (FULL || idx < N) ? in(idx) : 0ull;
    }
    uint32_t* label = reinterpret_cast<uint32_t*>(sk) + w * 256;
    for (int i = tid; i < kRsWarps * 256; i += kRsT) (&wc[0][0])[i] = 0;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRsKpt; r++) {
        const bool valid = FULL || base + r * 32 + lane < N;
        const unsigned d = key_byte<B>(key[r]);
        if (valid) label[d] = (uint32_t)lane;
        __syncwarp();
        const unsigned rep = valid ? label[d] : 0u;
        unsigned peers = FULL ? kFull : __ballot_sync(kFull, valid);
#pragma unroll
        for (int b = 0; b < 5; b++) {
            const bool bit = (rep >> b) & 1u;
            const unsigned m = __ballot_sync(kFull, bit);
            peers &= bit ? m : ~m;
        }
        if (!valid) peers = 0u;
        const unsigned lower = peers & lt_mask;
        const uint32_t before = valid ? wc[w][d] : 0u;
        __syncwarp();
        if (valid && lower == 0) wc[w][d] = before + (uint32_t)__popc(peers);
        const uint32_t rk = before + (uint32_t)__popc(lower);
        if (r & 1) rank[r >> 1] |= rk << 16;
        else rank[r >> 1] = rk;
    }
    __syncthreads();
    // thread tid = digit: exclusive prefix over the warps, then over the
    // digits; the warps' counts become their staging bases
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < kRsWarps; ww++) run += wc[ww][tid];
    unsigned long long tot;
    const uint32_t ds = (uint32_t)block_excl_scan(run, &tot);
    uint32_t acc = ds;
#pragma unroll
    for (int ww = 0; ww < kRsWarps; ww++) {
        const uint32_t c = wc[ww][tid];
        wc[ww][tid] = acc;
        acc += c;
    }
    gd[tid] = my_goff - ds;  // output index of staged position p: gd[digit] + p
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRsKpt; r++) {
        if (FULL || base + r * 32 + lane < N) {
            const unsigned d = key_byte<B>(key[r]);
            sk[wc[w][d] + ((rank[r >> 1] >> (16 * (r & 1))) & 0xffffu)] = key[r];
        }
    }
    __syncthreads();
    const int cnt = FULL ? kRsTile : (int)min((long long)kRsTile, N - tile0);
#pragma unroll
    for (int r = 0; r < kRsKpt; r++) {
        const int p = r * kRsT + tid;
        if (FULL || p < cnt) {
            const unsigned long long k = sk[p];
            out[(long long)(uint32_t)(gd[key_byte<B>(k)] + (uint32_t)p)] = k;
        }
    }
}

template <typename In, int B>
__global__ void __launch_bounds__(kRsT, 3) k_rs_scatter(In in, unsigned long long* __restrict__ out,
                                                        long long N, const uint32_t* __restrict__ off,
                                                        long long nt) {
    __shared__ __align__(16) unsigned long long sk[kRsTile];
    __shared__ uint32_t wc[kRsWarps][256];
    __shared__ uint32_t gd[256];
    const long long tile0 = (long long)blockIdx.x * kRsTile;
    const uint32_t my_goff = off[(long long)threadIdx.x * nt + blockIdx.x];
    if (tile0 + kRsTile <= N) scatter_tile<In, B, true>(in, out, N, tile0, my_goff, sk, wc, gd);
    else scatter_tile<In, B, false>(in, out, N, tile0, my_goff, sk, wc, gd);
}

template <typename In>
cudaError_t launch_scatter(int shift, unsigned grid, cudaStream_t st, In in,
                           unsigned long long* out, long long N, const uint32_t* off, long long nt) {
    switch (shift) {
        case 0: k_rs_scatter<In, 0><<<grid, kRsT, 0, st>>>(in, out, N, off, nt); break;
        case 8: k_rs_scatter<In, 1><<<grid, kRsT, 0, st>>>(in, out, N, off, nt); break;
        case 16: k_rs_scatter<In, 2><<<grid, kRsT, 0, st>>>(in, out, N, off, nt); break;
        case 24: k_rs_scatter<In, 3><<<grid, kRsT, 0, st>>>(in, out, N, off, nt); break;
        case 32: k_rs_scatter<In, 4><<<grid, kRsT, 0, st>>>(in, out, N, off, nt); break;
        case 40: k_rs_scatter<In, 5><<<grid, kRsT, 0, st>>>(in, out, N, off, nt); break;
        case 48: k_rs_scatter<In, 6><<<grid, kRsT, 0, st>>>(in, out, N, off, nt); break;
        case 56: k_rs_scatter<In, 7><<<grid, kRsT, 0, st>>>(in, out, N, off, nt); break;
        default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

// Sorts the N keys of `first` by bits [0, lowbits) then [32, 32 + highbits)
// (LSD).  Pass p writes buf[p % 2] and the next pass reads it; *result is the
// buffer holding the sorted keys.  `bad` (may be null) is raised when `first`
// reports an invalid key.  N >= 1.
template <typename In>
cudaError_t radix_sort(In first, long long N, unsigned long long* buf0, unsigned long long* buf1,
                       int lowbits, int highbits, cudaStream_t st, unsigned long long** result,
                       Temp* tmp, int* bad, const uint32_t* hist0 = nullptr) {
    const long long nt = (N + kRsTile - 1) / kRsTile;
    uint32_t *hist = nullptr, *off = nullptr;
    cudaError_t e = tmp->get(&hist, (size_t)256 * nt);
    if (e == cudaSuccess) e = tmp->get(&off, (size_t)256 * nt);
    if (e != cudaSuccess) return e;
    std::vector<int> shifts;
    for (int s = 0; s < lowbits; s += 8) shifts.push_back(s);
    for (int s = 0; s < highbits; s += 8) shifts.push_back(32 + s);
    if (shifts.empty()) shifts.push_back(0);  // the keys still pass through once
    unsigned long long* buf[2] = {buf0, buf1};
    for (size_t p = 0; p < shifts.size() && e == cudaSuccess; p++) {
        const int sh = shifts[p];
        unsigned long long* out = buf[p % 2];
        const uint32_t* h = hist;
        if (p == 0 && hist0) {
            h = hist0;  // counted by the caller while it wrote the keys
        } else {
            if (p == 0) {
                k_rs_hist<<<(unsigned)nt, kRsT, 0, st>>>(first, N, sh, hist, nt, bad);
            } else {
                k_rs_hist<<<(unsigned)nt, kRsT, 0, st>>>(KeyIn{buf[(p - 1) % 2]}, N, sh, hist, nt,
                                                         (int*)nullptr);
            }
            count_launch();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = exclusive_scan(ReadU32{h}, 256 * nt, off, false, st, tmp);
        if (e != cudaSuccess) break;
        if (p == 0)
            e = launch_scatter(sh, (unsigned)nt, st, first, out, N, off, nt);
        else
            e = launch_scatter(sh, (unsigned)nt, st, KeyIn{buf[(p - 1) % 2]}, out, N, off, nt);
        *result = out;
    }
    return e;
}

struct HubLen {
    const int* huge;
    const uint32_t* off;
    __device__ unsigned long long operator()(long long r) const {
        return off[huge[r] + 1] - off[huge[r]];
    }
};

// keys of the hub rows: (rank of the row among hub rows) << 32 | column
__global__ void k_huge_keys(const int* __restrict__ huge, unsigned nh,
                            const unsigned long long* __restrict__ hoff,
                            const uint32_t* __restrict__ off, const uint32_t* __restrict__ seg,
                            unsigned long long* __restrict__ keys) {
    for (unsigned r = blockIdx.x; r < nh; r += gridDim.x) {
        const int u = huge[r];
        const uint32_t o = off[u];
        const long long len = (long long)(off[u + 1] - o);
        for (long long i = threadIdx.x; i < len; i += blockDim.x)
            keys[hoff[r] + i] = ((unsigned long long)r << 32) | seg[o + i];
    }
}

__global__ void k_huge_back(const int* __restrict__ huge, unsigned nh,
                            const unsigned long long* __restrict__ hoff,
                            const uint32_t* __restrict__ off,
                            const unsigned long long* __restrict__ keys, uint32_t* __restrict__ seg,
                            uint32_t* __restrict__ ucnt) {
    __shared__ unsigned long long wtot;
    for (unsigned r = blockIdx.x; r < nh; r += gridDim.x) {
        const int u = huge[r];
        const uint32_t o = off[u];
        const long long len = (long long)(off[u + 1] - o);
        const unsigned long long* k = keys + hoff[r];
        const long long per = (len + blockDim.x - 1) / blockDim.x;
        const long long i0 = min(len, (long long)threadIdx.x * per), i1 = min(len, i0 + per);
        unsigned c = 0;
        for (long long i = i0; i < i1; i++) c += (i == 0 || k[i] != k[i - 1]) ? 1u : 0u;
        unsigned long long tot;
        unsigned long long pos = block_excl_scan(c, &tot);
        for (long long i = i0; i < i1; i++)
            if (i == 0 || k[i] != k[i - 1]) seg[o + pos++] = (uint32_t)(k[i] & 0xffffffffu);
        if (threadIdx.x == 0) wtot = tot;
        __syncthreads();
        if (threadIdx.x == 0) ucnt[u] = (uint32_t)wtot;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ compaction
// Rows of at most 32 entries: one thread each; the listed larger rows: one warp.
template <typename Off>
__global__ void k_compact_small(int n, const uint32_t* __restrict__ off,
                                const uint32_t* __restrict__ seg, const uint32_t* __restrict__ ucnt,
                                const Off* __restrict__ rp, int* __restrict__ col) {
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n;
         u += (long long)gridDim.x * blockDim.x) {
        if (off[u + 1] - off[u] > (uint32_t)kSmallMax) continue;
        const uint32_t c = ucnt[u];
        const uint32_t* s = seg + off[u];
        int* d = col + (long long)rp[u];
        for (uint32_t i = 0; i < c; i++) d[i] = (int)s[i];
    }
}

template <typename Off>
__global__ void k_compact_list(const int* __restrict__ list, const unsigned* count,
                               const uint32_t* __restrict__ off, const uint32_t* __restrict__ seg,
                               const uint32_t* __restrict__ ucnt, const Off* __restrict__ rp,
                               int* __restrict__ col) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const unsigned nl = *count;
    for (long long i = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; i < nl; i += warps) {
        const int u = list[i];
        const uint32_t c = ucnt[u];
        const uint32_t* s = seg + off[u];
        int* d = col + (long long)rp[u];
        for (uint32_t j = lane; j < c; j += 32) d[j] = (int)s[j];
    }
}

template <typename Off>
__global__ void k_check_clean(const Off* __restrict__ rp, const int* __restrict__ col, int n,
                              long long nnz, int* bad) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long u = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        long long b, e;
        if (!row_range(rp, n, nnz, u, &b, &e)) {
            if (lane == 0) *bad = 1;
            continue;
        }
        for (long long j = b + lane; j < e; j += 32) {
            const int v = col[j];
            if ((unsigned)v >= (unsigned)n || v == (int)u) *bad = 1;
            if (j > b && col[j - 1] >= v) *bad = 1;
        }
    }
}

// ------------------------------------------------------------------ tier split
constexpr int kTsT = 1024;

__device__ __forceinline__ int tier_of(long long d, int t_lo, int t_hi) {
    return d <= t_lo ? 0 : (d <= t_hi ? 1 : 2);
}

template <typename Off>
__global__ void __launch_bounds__(kTsT) k_tier_count(const Off* __restrict__ rp, int n, int t_lo,
                                                     int t_hi, uint32_t* cnt, int nb, TierOut* out) {
    __shared__ uint32_t c[kTiers];
    if (threadIdx.x < kTiers) c[threadIdx.x] = 0;
    __syncthreads();
    const long long v = (long long)blockIdx.x * kTsT + threadIdx.x;
    if (v < n) {
        const long long d = (long long)(rp[v + 1] - rp[v]);
        if (d > (long long)kEstMask) out->bad = 1;
        atomicAdd(&c[tier_of(d, t_lo, t_hi)], 1u);
    }
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
    const int t = valid ? tier_of(d, t_lo, t_hi) : -1;
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
        est0[v] = ((uint32_t)t << kEstBits) | (uint32_t)(d & kEstMask);
        list[off[t * nb + blockIdx.x] + before + mine] = (int)v;
    }
}

// Gathers the tier boundaries and row_ptr[n] into the block the host reads.
__global__ void k_tier_out(const uint32_t* off, int nb, const void* row_ptr, int off_bytes,
                           long long n, TierOut* out) {
    if (threadIdx.x <= kTiers) out->bound[threadIdx.x] = off[(long long)threadIdx.x * nb];
    if (threadIdx.x == 0)
        out->nnz = off_bytes == 8 ? ((const long long*)row_ptr)[n] : (long long)((const int*)row_ptr)[n];
}

// ------------------------------------------------------------------ sorted build
// For graphs whose hub rows hold most entries: one canonical key per sample,
// sorted over both ids; the distinct edges and their transposes written; the
// transposes sorted over the row bits only; then each row assembled from its
// two ascending halves.  Against sorting both directed entries of every
// sample over both ids, this sorts half the keys over both ids and the
// distinct half again over one: 4.5 instead of 6 full-size passes for 24-bit
// ids.  No per-row atomics on hot rows and no per-row sorts.  (Making the
// keys inside the first radix pass instead was slower.)
// Four samples per thread per round, their loads (and, when renumbering, the
// gathers of their new ids) issued before any is used.
constexpr int kSbU = 4;

// One key per sample: its canonical form (min << 32 | max) of the two
// (renumbered) ends; a loop or a bad id becomes kNoKey.  (Counting the first
// radix pass's digits here, a tile per CTA, made this kernel slower by more
// than the histogram pass it saved.)
__global__ void k_sb_keys(const int* __restrict__ src, const int* __restrict__ dst, long long S,
                          int n, unsigned long long* __restrict__ keys, BuildCtl* bc,
                          const int* __restrict__ remap) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; i0 < S; i0 += kSbU * stride) {
        int s[kSbU], d[kSbU];
        bool ok[kSbU];
#pragma unroll
        for (int r = 0; r < kSbU; r++) {
            const long long i = i0 + r * stride;
            s[r] = i < S ? src[i] : 0;
            d[r] = i < S ? dst[i] : 0;
        }
#pragma unroll
        for (int r = 0; r < kSbU; r++) {
            const long long i = i0 + r * stride;
            const bool in = (unsigned)s[r] < (unsigned)n && (unsigned)d[r] < (unsigned)n;
            if (i < S && !in) bc->bad = 1;
            ok[r] = i < S && in && s[r] != d[r];
        }
        if (remap) {
#pragma unroll
            for (int r = 0; r < kSbU; r++) {
                if (ok[r]) {
                    s[r] = __ldg(remap + s[r]);
                    d[r] = __ldg(remap + d[r]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kSbU; r++) {
            const long long i = i0 + r * stride;
            if (i >= S) continue;
            const unsigned lo = (unsigned)min(s[r], d[r]), hi = (unsigned)max(s[r], d[r]);
            keys[i] = ok[r] ? ((unsigned long long)lo << 32) | hi : kNoKey;
        }
    }
}

__device__ __forceinline__ bool sb_first(const unsigned long long* keys, long long i) {
    const unsigned long long k = keys[i];
    return k != kNoKey && (i == 0 || keys[i - 1] != k);
}

// Distinct keys per tile of kRsTile sorted keys.
__global__ void __launch_bounds__(kRsT) k_sb_count(const unsigned long long* __restrict__ keys,
                                                   long long N, uint32_t* __restrict__ tsum) {
    const long long base = (long long)blockIdx.x * kRsTile;
    unsigned c = 0;
#pragma unroll 4
    for (int i = 0; i < kRsKpt; i++) {
        const long long idx = base + (long long)i * kRsT + threadIdx.x;
        if (idx < N && sb_first(keys, idx)) c++;
    }
    unsigned long long tot;
    block_excl_scan(c, &tot);
    if (threadIdx.x == 0) tsum[blockIdx.x] = (uint32_t)tot;
}

// The distinct canonical keys (a, b), a < b, in order: up[p] = (a << 32 | b)
// and lo[p] = (b << 32 | a) at position p among the distinct keys, and
// ucnt[a] += the number of them (sorted keys: a warp's lanes share one or two
// rows, one add per row).
// All kRsKpt rounds' keys are loaded and judged first; one barrier then makes
// the per-round, per-warp counts visible, and each key's rank in the tile is
// the count of the rounds before it, of the warps before it in its round, and
// of the lanes before it in its warp.
__global__ void __launch_bounds__(kRsT) k_sb_emit(const unsigned long long* __restrict__ keys,
                                                  long long N, const uint32_t* __restrict__ toff,
                                                  unsigned long long* __restrict__ up,
                                                  unsigned long long* __restrict__ lo,
                                                  uint32_t* __restrict__ ucnt,
                                                  uint32_t* __restrict__ lhist, long long nt) {
    __shared__ uint32_t cnt[kRsKpt][kRsWarps];
    __shared__ uint32_t rbase[kRsKpt];
    __shared__ uint32_t th[2][256];  // first-pass digits of the transposes, by their tile
    th[0][threadIdx.x] = 0;
    th[1][threadIdx.x] = 0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const long long base = (long long)blockIdx.x * kRsTile;
    unsigned long long k[kRsKpt];
    uint32_t firsts = 0;
#pragma unroll
    for (int i = 0; i < kRsKpt; i++) {
        const long long idx = base + (long long)i * kRsT + threadIdx.x;
        k[i] = idx < N ? keys[idx] : kNoKey;
    }
#pragma unroll
    for (int i = 0; i < kRsKpt; i++) {
        const long long idx = base + (long long)i * kRsT + threadIdx.x;
        // the key before this one: the previous lane's, or the last of the
        // previous round / tile
        unsigned long long prev = __shfl_up_sync(kFull, k[i], 1);
        if (lane == 0) prev = idx > 0 ? keys[idx - 1] : ~k[i];
        const bool f = idx < N && k[i] != kNoKey && k[i] != prev;
        firsts |= (uint32_t)f << i;
        const unsigned m = __ballot_sync(kFull, f);
        if (lane == 0) cnt[i][w] = (uint32_t)__popc(m);
    }
    __syncthreads();
    if (threadIdx.x < kRsKpt) {
        uint32_t t = 0;
#pragma unroll
        for (int ww = 0; ww < kRsWarps; ww++) t += cnt[threadIdx.x][ww];
        rbase[threadIdx.x] = t;
    }
    __syncthreads();
    uint32_t run = toff[blockIdx.x];
    const uint32_t t0 = run / (uint32_t)kRsTile;  // this tile's keys land in transpose tiles t0, t0 + 1
#pragma unroll
    for (int i = 0; i < kRsKpt; i++) {
        const bool f = (firsts >> i) & 1u;
        const unsigned m = __ballot_sync(kFull, f);
        uint32_t before = 0;
#pragma unroll
        for (int ww = 0; ww < kRsWarps; ww++) before += ww < w ? cnt[i][ww] : 0u;
        const unsigned row = (unsigned)(k[i] >> 32);
        if (f) {
            const uint32_t p = run + before + (uint32_t)__popc(m & lt);
            up[p] = k[i];
            lo[p] = (k[i] << 32) | row;
            atomicAdd(&th[p / (uint32_t)kRsTile - t0][(unsigned)k[i] & 255u], 1u);
        }
        const unsigned peers = __match_any_sync(kFull, f ? row : 0xffffffffu);
        if (f && (peers & lt) == 0) atomicAdd(&ucnt[row], (uint32_t)__popc(peers));
        run += rbase[i];
    }
    __syncthreads();
    if (th[0][threadIdx.x]) atomicAdd(&lhist[(long long)threadIdx.x * nt + t0], th[0][threadIdx.x]);
    if (th[1][threadIdx.x]) atomicAdd(&lhist[(long long)threadIdx.x * nt + t0 + 1], th[1][threadIdx.x]);
}

// Positions [U, S) of up and lo (U = the distinct count, toff[nt]) get
// kNoKey, so the transposed keys sort after every real one and both emits
// skip them.
// They count as digit 255 in the transposes' first-pass histogram.
__global__ void k_sb_tail(const uint32_t* __restrict__ total, long long S,
                          unsigned long long* __restrict__ up, unsigned long long* __restrict__ lo,
                          uint32_t* __restrict__ lhist, long long nt) {
    const long long U = (long long)*total;
    const long long g0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long gs = (long long)gridDim.x * blockDim.x;
    for (long long p = U + g0; p < S; p += gs) {
        up[p] = kNoKey;
        lo[p] = kNoKey;
    }
    for (long long t = U / kRsTile + g0; t < nt; t += gs) {
        const long long a = U > t * kRsTile ? U : t * kRsTile;
        const long long b = S < (t + 1) * kRsTile ? S : (t + 1) * kRsTile;
        if (b > a) atomicAdd(&lhist[255LL * nt + t], (uint32_t)(b - a));
    }
}

// Lower halves: lo sorted by (b, a).  Row b lists its smaller neighbours
// first, and the j-th transposed key lands at col[j + su[b]] (su: exclusive
// scan of the upper counts), since row b starts at
// su[b] + #{transposed keys with row < b}.  Each run of one row adds its
// length to ucnt[b] (its first key subtracts its index, its last key adds
// the index after it), so that ucnt becomes the row lengths.
__global__ void k_sb_lower(const unsigned long long* __restrict__ lo, long long S,
                           const uint32_t* __restrict__ su, int* __restrict__ col,
                           uint32_t* __restrict__ ucnt) {
    const int lane = threadIdx.x & 31;
    const long long wstride = (long long)gridDim.x * blockDim.x;
    for (long long b0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) - lane; b0 < S; b0 += wstride) {
        const long long j = b0 + lane;
        const unsigned long long k = j < S ? lo[j] : kNoKey;
        unsigned long long prev = __shfl_up_sync(kFull, k, 1);
        unsigned long long next = __shfl_down_sync(kFull, k, 1);
        if (lane == 0) prev = j > 0 && j - 1 < S ? lo[j - 1] : kNoKey;
        if (lane == 31) next = j + 1 < S ? lo[j + 1] : kNoKey;
        if (k == kNoKey) continue;
        const unsigned r = (unsigned)(k >> 32);
        col[j + su[r]] = (int)(unsigned)k;
        if (prev == kNoKey || (unsigned)(prev >> 32) != r) atomicAdd(&ucnt[r], 0u - (uint32_t)j);
        if (next == kNoKey || (unsigned)(next >> 32) != r) atomicAdd(&ucnt[r], (uint32_t)(j + 1));
    }
}

// Upper halves: up sorted by (a, b).  Row a ends with its larger
// neighbours: the j-th key lands at col[row_ptr[a + 1] - (su[a + 1] - j)].
template <typename Off>
__global__ void k_sb_upper(const unsigned long long* __restrict__ up, long long S,
                           const uint32_t* __restrict__ su, const Off* __restrict__ row_ptr,
                           int* __restrict__ col) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < S;
         j += (long long)gridDim.x * blockDim.x) {
        const unsigned long long k = up[j];
        if (k == kNoKey) continue;
        const unsigned r = (unsigned)(k >> 32);
        col[(long long)row_ptr[r + 1] - ((long long)su[r + 1] - j)] = (int)(unsigned)k;
    }
}

int id_bits(long long n) {
    int b = 0;
    while ((1ll << b) < n) b++;
    return b;
}

kcore_status cuda_fail(cudaError_t e, const char* what, std::string* err) {
    cudaGetLastError();
    *err = std::string(what) + ": " + cudaGetErrorString(e);
    return (e == cudaErrorMemoryAllocation) ? KCORE_ERR_OOM : KCORE_ERR_CUDA;
}

#define KC_TRY(call, what)                                      \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, what, err); \
    } while (0)

int grid_for(long long items, int per_block) {
    return (int)std::max<long long>(1, std::min<long long>((items + per_block - 1) / per_block,
                                                           (long long)sm_count() * 64));
}

template <typename Off>
cudaError_t compact(int64_t n, const uint32_t* off, const uint32_t* seg, const uint32_t* ucnt,
                    const Off* rp, int* col, const int* const lists[3], const unsigned* const counts[3],
                    const unsigned hc[3], cudaStream_t st) {
    k_compact_small<<<grid_for(n, 256), 256, 0, st>>>((int)n, off, seg, ucnt, rp, col);
    count_launch();
    for (int q = 0; q < 3; q++)
        if (hc[q]) {
            k_compact_list<<<grid_for((long long)hc[q] * 32, 256), 256, 0, st>>>(
                lists[q], counts[q], off, seg, ucnt, rp, col);
            count_launch();
        }
    return cudaGetLastError();
}

// A pinned copy of the build state and the event that marks its arrival;
// released only once the copy has landed.
struct ClassRead {
    BuildCtl* h = nullptr;
    cudaEvent_t ev = nullptr;
    ~ClassRead() {
        if (ev) {
            cudaEventSynchronize(ev);
            cudaEventDestroy(ev);
        }
        if (h) pinned_put(h);
    }
};

// Steps 2-5, after the counts are in cnt.  `scatter` launches step 3.
template <typename ScatterFn>
kcore_status finish(Temp& tmp, int64_t n, long long N, uint32_t* cnt, BuildCtl* bc, int off_bytes,
                    cudaStream_t st, DevCsr* out, std::string* err, ScatterFn scatter) {
    // N: an upper bound of the entries (two per input sample or entry)
    const long long nn = std::max<int64_t>(n, 1);
    const size_t nbig = (size_t)std::min<long long>(nn, N / (kMidMax + 1) + 1);
    const size_t nhuge = (size_t)std::min<long long>(nn, N / (kBigMax + 1) + 1);
    uint32_t *off = nullptr, *seg = nullptr, *ucnt = nullptr;
    int *mid = nullptr, *big = nullptr, *huge = nullptr;
    KC_TRY(tmp.reserve(Temp::round(4 * (nn + 1)) + Temp::round(4 * (size_t)std::max<long long>(N, 1)) +
                       2 * Temp::round(4 * nn) + Temp::round(4 * nbig) + Temp::round(4 * nhuge) +
                       2 * scan_scratch_bytes(n)),
           "temporaries");
    KC_TRY(tmp.get(&off, (size_t)nn + 1), "row offsets");
    KC_TRY(tmp.get(&seg, (size_t)N), "segments");
    KC_TRY(tmp.get(&ucnt, (size_t)nn), "distinct counts");
    KC_TRY(tmp.get(&mid, (size_t)nn), "row lists");
    KC_TRY(tmp.get(&big, nbig), "row lists");
    KC_TRY(tmp.get(&huge, nhuge), "row lists");
    BuildCtl hbc;
    // offsets, and the size classes of the long rows (listed by the scan's
    // down-sweep when the arrays allow its vector path, else by k_classify),
    // copied to the host while the scatter and the small sorts run: the host
    // waits on the copy, not on the stream
    if (n > 0 && ((reinterpret_cast<uintptr_t>(cnt) | reinterpret_cast<uintptr_t>(off)) % 16 == 0)) {
        KC_TRY(exclusive_scan4(cnt, n, off, true, st, &tmp, ClassifyEpi{mid, big, huge, bc}),
               "offset scan");
    } else {
        KC_TRY(exclusive_scan(ReadU32{cnt}, n, off, true, st, &tmp), "offset scan");
        if (n > 0) {
            k_classify<<<grid_for(n, 256), 256, 0, st>>>((int)n, off, mid, big, huge, bc);
            count_launch();
            KC_TRY(cudaGetLastError(), "classify rows");
        }
    }
    ClassRead cr;
    KC_TRY(pinned_get((void**)&cr.h, sizeof(BuildCtl)), "pinned buffer");
    KC_TRY(cudaEventCreateWithFlags(&cr.ev, cudaEventDisableTiming), "event");
    KC_TRY(cudaMemcpyAsync(cr.h, bc, sizeof(BuildCtl), cudaMemcpyDeviceToHost, st), "read classes");
    KC_TRY(cudaEventRecord(cr.ev, st), "event");
    KC_TRY(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * nn, st), "memset");  // cnt becomes the fill counter
    KC_TRY(scatter(off, cnt, seg), "scatter");
    if (n > 0) {
        k_sort_small<<<grid_for(n, 256), 256, 0, st>>>((int)n, off, seg, ucnt);
        count_launch();
        KC_TRY(cudaGetLastError(), "sort small rows");
    }
    KC_TRY(cudaEventSynchronize(cr.ev), "sync");
    hbc = *cr.h;
    if (hbc.bad) {
        *err = "an edge endpoint or a row offset is out of range";
        return KCORE_ERR_INVALID;
    }
    if (hbc.n_mid) {
        k_sort_mid<true><<<grid_for((long long)hbc.n_mid * 32, 256), 256, 0, st>>>(mid, bc, off, seg, ucnt);
        count_launch();
        k_sort_mid<false><<<grid_for((long long)hbc.n_mid * 32, 256), 256, 0, st>>>(mid, bc, off, seg, ucnt);
        count_launch();
        KC_TRY(cudaGetLastError(), "sort mid rows");
    }
    if (hbc.n_big) {
        const size_t smem = sizeof(uint32_t) * 2 * kBigMax;  // two merge buffers
        KC_TRY(cudaFuncSetAttribute(k_sort_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem), "smem attribute");
        k_sort_big<<<(unsigned)std::min<unsigned>(hbc.n_big, (unsigned)sm_count() * 2u), kBigT, smem, st>>>(
            big, bc, off, seg, ucnt);
        count_launch();
        KC_TRY(cudaGetLastError(), "sort big rows");
    }
    if (hbc.n_huge) {
        const long long H = (long long)hbc.huge_entries;
        unsigned long long *keys = nullptr, *alt = nullptr, *hoff = nullptr, *sorted = nullptr;
        KC_TRY(tmp.get(&keys, (size_t)H), "hub keys");
        KC_TRY(tmp.get(&alt, (size_t)H), "hub keys");
        KC_TRY(tmp.get(&hoff, (size_t)hbc.n_huge + 1), "hub offsets");
        KC_TRY(exclusive_scan(HubLen{huge, off}, (long long)hbc.n_huge, hoff, true, st, &tmp), "hub offsets");
        const unsigned g = std::min<unsigned>(hbc.n_huge, (unsigned)sm_count() * 4u);
        k_huge_keys<<<g, 512, 0, st>>>(huge, hbc.n_huge, hoff, off, seg, keys);
        count_launch();
        KC_TRY(cudaGetLastError(), "hub keys");
        KC_TRY(radix_sort(KeyIn{keys}, H, alt, keys, id_bits(n), id_bits(hbc.n_huge), st, &sorted, &tmp,
                          (int*)nullptr),
               "hub sort");
        k_huge_back<<<g, 512, 0, st>>>(huge, hbc.n_huge, hoff, off, sorted, seg, ucnt);
        count_launch();
        KC_TRY(cudaGetLastError(), "hub write back");
    }
    // row_ptr and col_idx (col sized by the entries before repeats were dropped)
    kcore_status s = dmalloc(&out->row_ptr, (size_t)off_bytes * (n + 1), err, st);
    if (s != KCORE_OK) return s;
    s = dmalloc((void**)&out->col, sizeof(int) * std::max<size_t>(N, 1), err, st);
    if (s != KCORE_OK) return s;
    if (off_bytes == 8)
        KC_TRY(exclusive_scan(ReadU32{ucnt}, n, (long long*)out->row_ptr, true, st, &tmp), "row scan");
    else
        KC_TRY(exclusive_scan(ReadU32{ucnt}, n, (int*)out->row_ptr, true, st, &tmp), "row scan");
    if (n > 0) {
        const int* const lists[3] = {mid, big, huge};
        const unsigned* const counts[3] = {&bc->n_mid, &bc->n_big, &bc->n_huge};
        const unsigned hc[3] = {hbc.n_mid, hbc.n_big, hbc.n_huge};
        if (off_bytes == 8)
            KC_TRY(compact(n, off, seg, ucnt, (const long long*)out->row_ptr, out->col, lists, counts,
                           hc, st), "compact");
        else
            KC_TRY(compact(n, off, seg, ucnt, (const int*)out->row_ptr, out->col, lists, counts, hc,
                           st), "compact");
    }
    out->n = n;
    out->nnz = -1;  // row_ptr[n], read by the caller's next wait
    out->off_bytes = off_bytes;
    return KCORE_OK;
}

// The sorted build (kernels above); the host waits once, at the end, for the
// range flag.
kcore_status sorted_build(Temp& tmp, int64_t n, long long S, const int* src, const int* dst,
                          BuildCtl* bc, int off_bytes, cudaStream_t st, DevCsr* out,
                          std::string* err, const int* remap) {
    const long long N = std::max<long long>(S, 1), nn = std::max<int64_t>(n, 1);
    const long long nt = (N + kRsTile - 1) / kRsTile;
    unsigned long long *keys = nullptr, *alt = nullptr, *third = nullptr, *sorted = nullptr;
    uint32_t *ucnt = nullptr, *su = nullptr, *tsum = nullptr, *toff = nullptr;
    uint32_t* lhist = nullptr;  // first-pass digit counts of the transposes' sort
    KC_TRY(tmp.reserve(3 * Temp::round(8 * (size_t)N) + Temp::round(4 * nn) + Temp::round(4 * (nn + 1)) +
                       2 * Temp::round(4 * (nt + 1)) + 3 * Temp::round(4 * 256 * (size_t)nt) +
                       scan_scratch_bytes(256 * nt) + scan_scratch_bytes(nt) + 2 * scan_scratch_bytes(n)),
           "temporaries");
    KC_TRY(tmp.get(&lhist, (size_t)256 * nt), "digit counts");
    KC_TRY(tmp.get(&keys, (size_t)N), "keys");
    KC_TRY(tmp.get(&alt, (size_t)N), "keys");
    KC_TRY(tmp.get(&third, (size_t)N), "keys");
    KC_TRY(tmp.get(&ucnt, (size_t)nn), "row counts");
    KC_TRY(tmp.get(&su, (size_t)nn + 1), "upper offsets");
    KC_TRY(tmp.get(&tsum, (size_t)nt), "tile counts");
    KC_TRY(tmp.get(&toff, (size_t)nt + 1), "tile offsets");
    KC_TRY(cudaMemsetAsync(ucnt, 0, sizeof(uint32_t) * nn, st), "memset");
    if (S > 0) {
        k_sb_keys<<<grid_for(S, 256), 256, 0, st>>>(src, dst, S, (int)n, keys, bc, remap);
        count_launch();
        KC_TRY(cudaGetLastError(), "keys");
    } else {
        KC_TRY(cudaMemsetAsync(keys, 0xff, sizeof(unsigned long long), st), "keys");
    }
    const int bits = id_bits(n);
    // 1. the canonical keys by (a, b)
    KC_TRY(radix_sort(KeyIn{keys}, N, alt, keys, bits, bits, st, &sorted, &tmp, (int*)nullptr), "sort");
    unsigned long long* up = sorted == keys ? alt : keys;
    unsigned long long* lo = third;
    // 2. the distinct ones, with their transposes, and the upper counts
    k_sb_count<<<(unsigned)nt, kRsT, 0, st>>>(sorted, N, tsum);
    count_launch();
    KC_TRY(cudaGetLastError(), "distinct count");
    KC_TRY(exclusive_scan(ReadU32{tsum}, nt, toff, true, st, &tmp), "tile scan");
    KC_TRY(cudaMemsetAsync(lhist, 0, sizeof(uint32_t) * 256 * nt, st), "memset");
    k_sb_emit<<<(unsigned)nt, kRsT, 0, st>>>(sorted, N, toff, up, lo, ucnt, lhist, nt);
    count_launch();
    k_sb_tail<<<grid_for(N, 256), 256, 0, st>>>(toff + nt, N, up, lo, lhist, nt);
    count_launch();
    KC_TRY(cudaGetLastError(), "emit");
    KC_TRY(exclusive_scan(ReadU32{ucnt}, n, su, true, st, &tmp), "upper offsets");
    // 3. the transposes by b (stable: a stays ascending within a row)
    unsigned long long* lsorted = nullptr;
    unsigned long long* lalt = sorted;  // free once the emit has read it
    // (the first pass's digits, byte 4, were counted by the emit and the tail;
    // with no id bits the single pass would read byte 0 instead)
    KC_TRY(radix_sort(KeyIn{lo}, N, lalt, lo, 0, bits, st, &lsorted, &tmp, (int*)nullptr,
                      bits > 0 ? lhist : nullptr), "transpose sort");
    kcore_status s = dmalloc(&out->row_ptr, (size_t)off_bytes * (n + 1), err, st);
    if (s != KCORE_OK) return s;
    s = dmalloc((void**)&out->col, sizeof(int) * std::max<size_t>(2 * (size_t)N, 1), err, st);
    if (s != KCORE_OK) return s;
    // 4. lower halves, the row lengths, row_ptr, upper halves
    k_sb_lower<<<grid_for(N, 256), 256, 0, st>>>(lsorted, N, su, out->col, ucnt);
    count_launch();
    KC_TRY(cudaGetLastError(), "lower halves");
    if (off_bytes == 8) {
        KC_TRY(exclusive_scan(ReadU32{ucnt}, n, (long long*)out->row_ptr, true, st, &tmp), "row scan");
        k_sb_upper<long long><<<grid_for(N, 256), 256, 0, st>>>(up, N, su, (const long long*)out->row_ptr,
                                                                out->col);
    } else {
        KC_TRY(exclusive_scan(ReadU32{ucnt}, n, (int*)out->row_ptr, true, st, &tmp), "row scan");
        k_sb_upper<int><<<grid_for(N, 256), 256, 0, st>>>(up, N, su, (const int*)out->row_ptr, out->col);
    }
    count_launch();
    KC_TRY(cudaGetLastError(), "upper halves");
    int hbad = 0;
    KC_TRY(cudaMemcpyAsync(&hbad, &bc->bad, sizeof(int), cudaMemcpyDeviceToHost, st), "read flag");
    KC_TRY(cudaStreamSynchronize(st), "sync");
    if (hbad) {
        *err = "an edge endpoint or a row offset is out of range";
        return KCORE_ERR_INVALID;
    }
    out->n = n;
    out->nnz = -1;  // row_ptr[n], read by the caller's next wait
    out->off_bytes = off_bytes;
    return KCORE_OK;
}

}  // namespace

cudaError_t scan_u32_to_u64(const uint32_t* in, unsigned long long* out, long long N,
                            cudaStream_t st) {
    return exclusive_scan(ReadU32{in}, N, out, true, st);
}

namespace {

// ------------------------------------------------------------------ relabeling by degree
// Renumbering the vertices in order of degree packs the estimates of the
// high-degree vertices (the ones most adjacency entries point to) into few
// cache lines, and the cleaned rows, sorted by the new ids, then list the
// high-degree neighbours together: a warp's gathers of their estimates touch
// few sectors, and the no-change test of a hub meets its supporters early.
// The sorted build renumbers before it sorts, so the cleaned CSR comes out in
// the new ids with sorted rows at no extra sorting cost.  The order is that
// of the probe counts (every kSortProbe-th run of samples, an estimate of the
// degree), descending or ascending, ties by old id (a stable sort).
__global__ void k_rl_keys(const uint32_t* __restrict__ cnt, long long n, int descending,
                          unsigned long long* __restrict__ keys) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const unsigned long long c = cnt[v];
        const unsigned long long ck = descending ? 0xffffffffull - c : c;
        keys[v] = (ck << 32) | (unsigned long long)v;
    }
}

__global__ void k_rl_perm(const unsigned long long* __restrict__ sorted, long long n,
                          int* __restrict__ old_of_new, int* __restrict__ new_of_old) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int old = (int)(uint32_t)(sorted[i] & 0xffffffffull);
        old_of_new[i] = old;
        new_of_old[old] = (int)i;
    }
}

// The entries of a renumbered CSR as samples in the caller's ids (both
// directions are present already): row of entry p by bisection of row_ptr.
template <typename Off>
__global__ void k_rl_unmap(const Off* __restrict__ rp, const int* __restrict__ col, long long n,
                           long long nnz, const int* __restrict__ old_of_new, int* __restrict__ src,
                           int* __restrict__ dst) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nnz;
         p += (long long)gridDim.x * blockDim.x) {
        long long lo = 0, hi = n - 1;  // last row whose start is <= p
        while (lo < hi) {
            const long long mid = (lo + hi + 1) >> 1;
            if ((long long)rp[mid] <= p) lo = mid;
            else hi = mid - 1;
        }
        src[p] = old_of_new[lo];
        dst[p] = old_of_new[col[p]];
    }
}

__global__ void k_rl_start(const int* __restrict__ start, const int* __restrict__ frontier, long long nf,
                           long long n, const int* __restrict__ old_of_new,
                           const int* __restrict__ new_of_old, int* __restrict__ start2,
                           int* __restrict__ frontier2) {
    const long long total = n > nf ? n : nf;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        if (i < n) start2[i] = start[old_of_new[i]];
        if (frontier && i < nf) {
            const int f = frontier[i];
            frontier2[i] = (f >= 0 && f < n) ? new_of_old[f] : f;
        }
    }
}

// The renumbering of a build: new_of_old / old_of_new (n each, allocated
// here) from the probe counts in cnt.
kcore_status make_renumbering(Temp& tmp, int64_t n, const uint32_t* cnt, int descending, cudaStream_t st,
                              int** new_of_old, int** old_of_new, std::string* err) {
    const long long nn = std::max<int64_t>(n, 1);
    const long long nt = (nn + kRsTile - 1) / kRsTile;
    unsigned long long *keys = nullptr, *alt = nullptr, *sorted = nullptr;
    KC_TRY(tmp.get(&keys, (size_t)nn), "renumbering keys");
    KC_TRY(tmp.get(&alt, (size_t)nn), "renumbering keys");
    (void)nt;
    kcore_status s = dmalloc((void**)new_of_old, sizeof(int) * nn, err, st);
    if (s == KCORE_OK) s = dmalloc((void**)old_of_new, sizeof(int) * nn, err, st);
    if (s != KCORE_OK) return s;
    const int g = grid_for(n, 256);
    k_rl_keys<<<g, 256, 0, st>>>(cnt, n, descending, keys);
    count_launch();
    KC_TRY(cudaGetLastError(), "renumbering keys");
    KC_TRY(radix_sort(KeyIn{keys}, n, alt, keys, 0, 32, st, &sorted, &tmp, (int*)nullptr), "renumbering sort");
    k_rl_perm<<<g, 256, 0, st>>>(sorted, n, *old_of_new, *new_of_old);
    count_launch();
    KC_TRY(cudaGetLastError(), "renumbering");
    return KCORE_OK;
}

}  // namespace

cudaError_t launch_relabel_unmap(const void* row_ptr, int off_bytes, const int* col, long long n,
                                 long long nnz, const int* old_of_new, int* src, int* dst,
                                 cudaStream_t st) {
    if (nnz <= 0) return cudaSuccess;
    const int g = grid_for(nnz, 256);
    if (off_bytes == 8)
        k_rl_unmap<<<g, 256, 0, st>>>((const long long*)row_ptr, col, n, nnz, old_of_new, src, dst);
    else
        k_rl_unmap<<<g, 256, 0, st>>>((const int*)row_ptr, col, n, nnz, old_of_new, src, dst);
    count_launch();
    return cudaGetLastError();
}


kcore_status clean_from_coo(int64_t n, int64_t samples, const int* src, const int* dst,
                            int off_bytes, int sort_mode, int relabel, cudaStream_t st, DevCsr* out,
                            int** new_of_old, int** old_of_new, std::string* err) {
    if (new_of_old) *new_of_old = nullptr;
    if (old_of_new) *old_of_new = nullptr;
    if (samples > 0x7fffffffLL) {
        *err = "at most 2^31-1 samples per graph";
        return KCORE_ERR_INVALID;
    }
    if (!new_of_old || !old_of_new) relabel = -1;
    Temp tmp(st);
    uint32_t* cnt = nullptr;
    BuildCtl* bc = nullptr;
    const size_t cnt_bytes = sizeof(uint32_t) * std::max<int64_t>(n, 1);
    KC_TRY(tmp.reserve(Temp::round(sizeof(BuildCtl)) + Temp::round(cnt_bytes)), "temporaries");
    KC_TRY(tmp.get(&bc, 1), "build state");
    KC_TRY(tmp.get(&cnt, (size_t)std::max<int64_t>(n, 1)), "counts");
    KC_TRY(cudaMemsetAsync(tmp.base, 0, tmp.used, st), "memset");  // the state and the counts
    // The probe: every kSortProbe-th run of samples counted per row.  It
    // estimates the share of entries in rows longer than kSmallMax (the
    // automatic choice of the pipeline and of renumbering) and, for a
    // renumbered build, the degree order.
    bool probed = false, heavy = false;
    auto probe = [&]() -> kcore_status {
        k_count_coo<<<grid_for(samples / kSortProbe + 256, 256), 256, 0, st>>>(src, dst, samples, (int)n,
                                                                             cnt, bc, kSortProbe);
        count_launch();
        k_heavy<<<(unsigned)std::min<long long>(grid_for(n, 256), (long long)sm_count() * 4), 256, 0, st>>>(
            cnt, n, kSmallMax / kSortProbe, bc);
        count_launch();
        KC_TRY(cudaGetLastError(), "row classes");
        BuildCtl hbc;
        KC_TRY(cudaMemcpyAsync(&hbc, bc, sizeof(BuildCtl), cudaMemcpyDeviceToHost, st), "read");
        KC_TRY(cudaStreamSynchronize(st), "sync");
        if (hbc.bad) {
            *err = "an edge endpoint or a row offset is out of range";
            return KCORE_ERR_INVALID;
        }
        probed = true;
        heavy = hbc.entries > 0 && 2 * hbc.heavy >= hbc.entries;
        return KCORE_OK;
    };
    // Automatic choice, for large inputs of average degree >= kSortAutoDegree
    // only (the others skip the wait): the sorted build when rows of more than
    // kSmallMax entries hold at least half of the entries.  Per-row counting
    // and sorting is cheaper while rows are short; hub rows make its atomics
    // collide and need the larger sorts.  The same test picks renumbering by
    // descending degree (relabel 0).  Either way the cleaned graph is the same
    // up to the numbering.
    const bool auto_size = samples >= kSortAutoSamples && 2 * samples >= kSortAutoDegree * n;
    bool use_sorted = samples > 0 && sort_mode > 0;
    if (samples > 0 && ((sort_mode == 0 && auto_size) || (relabel == 0 && auto_size))) {
        kcore_status ps = probe();
        if (ps != KCORE_OK) return ps;
        if (sort_mode == 0) use_sorted = heavy;
    }
    int rmode = relabel > 0 ? relabel : (relabel == 0 && probed && heavy ? 1 : 0);
    if (samples == 0 || n < 2) rmode = 0;
    if (rmode) {
        use_sorted = true;  // renumbering is done by the sorted build
        if (!probed) {
            kcore_status ps = probe();
            if (ps != KCORE_OK) return ps;
        }
        kcore_status rs = make_renumbering(tmp, n, cnt, rmode == 1 ? 1 : 0, st, new_of_old, old_of_new, err);
        if (rs != KCORE_OK) return rs;
        return sorted_build(tmp, n, samples, src, dst, bc, off_bytes, st, out, err, *new_of_old);
    }
    if (use_sorted) return sorted_build(tmp, n, samples, src, dst, bc, off_bytes, st, out, err, nullptr);
    if (probed) KC_TRY(cudaMemsetAsync(cnt, 0, cnt_bytes, st), "memset");
    if (samples > 0) {
        k_count_coo<<<grid_for(samples, 256), 256, 0, st>>>(src, dst, samples, (int)n, cnt, bc, 1);
        count_launch();
        KC_TRY(cudaGetLastError(), "count");
    }
    kcore_status s = finish(tmp, n, 2 * (long long)samples, cnt, bc, off_bytes, st, out, err,
                            [&](const uint32_t* off, uint32_t* fill, uint32_t* seg) {
                                if (samples == 0) return cudaSuccess;
                                k_scatter_coo<<<grid_for(samples, 256), 256, 0, st>>>(
                                    src, dst, samples, (int)n, off, fill, seg);
                                count_launch();
                                return cudaGetLastError();
                            });
    return s;
}

kcore_status clean_from_csr(int64_t n, const void* row_ptr, int in_off_bytes, const int* col,
                            int64_t nnz, int off_bytes, cudaStream_t st, DevCsr* out,
                            std::string* err) {
    if (nnz > 0x7fffffffLL) {
        *err = "at most 2^31-1 input entries per graph";
        return KCORE_ERR_INVALID;
    }
    Temp tmp(st);
    uint32_t* cnt = nullptr;
    BuildCtl* bc = nullptr;
    const size_t cnt_bytes = sizeof(uint32_t) * std::max<int64_t>(n, 1);
    KC_TRY(tmp.reserve(Temp::round(sizeof(BuildCtl)) + Temp::round(cnt_bytes)), "temporaries");
    KC_TRY(tmp.get(&bc, 1), "build state");
    KC_TRY(tmp.get(&cnt, (size_t)std::max<int64_t>(n, 1)), "counts");
    KC_TRY(cudaMemsetAsync(tmp.base, 0, tmp.used, st), "memset");  // the state and the counts
    const int g = grid_for(n * 32, 256);
    if (n > 0) {
        if (in_off_bytes == 8)
            k_count_csr<<<g, 256, 0, st>>>((const long long*)row_ptr, col, (int)n, nnz, cnt, bc);
        else
            k_count_csr<<<g, 256, 0, st>>>((const int*)row_ptr, col, (int)n, nnz, cnt, bc);
        count_launch();
        KC_TRY(cudaGetLastError(), "count");
    }
    kcore_status s = finish(tmp, n, 2 * (long long)nnz, cnt, bc, off_bytes, st, out, err,
                            [&](const uint32_t* off, uint32_t* fill, uint32_t* seg) {
                                if (n == 0) return cudaSuccess;
                                if (in_off_bytes == 8)
                                    k_scatter_csr<<<g, 256, 0, st>>>((const long long*)row_ptr, col,
                                                                     (int)n, nnz, off, fill, seg);
                                else
                                    k_scatter_csr<<<g, 256, 0, st>>>((const int*)row_ptr, col, (int)n,
                                                                     nnz, off, fill, seg);
                                count_launch();
                                return cudaGetLastError();
                            });
    return s;
}

kcore_status check_clean_csr(int64_t n, const void* row_ptr, int off_bytes, const int* col,
                             int64_t nnz, cudaStream_t st, std::string* err) {
    Temp tmp(st);
    int* bad = nullptr;
    KC_TRY(tmp.get(&bad, 1), "flag");
    KC_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st), "memset");
    if (n > 0) {
        const int g = grid_for(n * 32, 256);
        if (off_bytes == 8)
            k_check_clean<<<g, 256, 0, st>>>((const long long*)row_ptr, col, (int)n, nnz, bad);
        else
            k_check_clean<<<g, 256, 0, st>>>((const int*)row_ptr, col, (int)n, nnz, bad);
        count_launch();
        KC_TRY(cudaGetLastError(), "check");
    }
    int hbad = 0;
    KC_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st), "read flag");
    KC_TRY(cudaStreamSynchronize(st), "sync");
    if (hbad) {
        *err = "KCORE_IN_CLEAN graph has a bad offset, an unsorted row, a repeat, a self-loop or a bad id";
        return KCORE_ERR_INVALID;
    }
    return KCORE_OK;
}

kcore_status tier_split(int64_t n, const void* row_ptr, int off_bytes, int t_lo, int t_hi,
                        uint32_t* est0, int* init_list, TierOut* dout, cudaStream_t st,
                        std::string* err) {
    KC_TRY(cudaMemsetAsync(dout, 0, sizeof(TierOut), st), "memset");
    if (n == 0) return KCORE_OK;
    Temp tmp(st);
    const int nb = (int)((n + kTsT - 1) / kTsT);
    uint32_t *cnt = nullptr, *off = nullptr;
    KC_TRY(tmp.reserve(Temp::round(4 * (size_t)kTiers * nb) + Temp::round(4 * ((size_t)kTiers * nb + 1)) +
                       scan_scratch_bytes((long long)kTiers * nb)),
           "temporaries");
    KC_TRY(tmp.get(&cnt, (size_t)kTiers * nb), "tier counts");
    KC_TRY(tmp.get(&off, (size_t)kTiers * nb + 1), "tier offsets");
    if (off_bytes == 8)
        k_tier_count<<<nb, kTsT, 0, st>>>((const long long*)row_ptr, (int)n, t_lo, t_hi, cnt, nb, dout);
    else
        k_tier_count<<<nb, kTsT, 0, st>>>((const int*)row_ptr, (int)n, t_lo, t_hi, cnt, nb, dout);
    count_launch();
    KC_TRY(cudaGetLastError(), "tier count");
    KC_TRY(exclusive_scan(ReadU32{cnt}, (long long)kTiers * nb, off, true, st, &tmp), "tier scan");
    if (off_bytes == 8)
        k_tier_write<<<nb, kTsT, 0, st>>>((const long long*)row_ptr, (int)n, t_lo, t_hi, off, nb,
                                          est0, init_list);
    else
        k_tier_write<<<nb, kTsT, 0, st>>>((const int*)row_ptr, (int)n, t_lo, t_hi, off, nb, est0,
                                          init_list);
    count_launch();
    KC_TRY(cudaGetLastError(), "tier write");
    k_tier_out<<<1, 32, 0, st>>>(off, nb, row_ptr, off_bytes, n, dout);
    count_launch();
    KC_TRY(cudaGetLastError(), "tier out");
    return KCORE_OK;
}
cudaError_t launch_relabel_start(const int* start, const int* frontier, long long nf, long long n,
                                 const int* old_of_new, const int* new_of_old, int* start2,
                                 int* frontier2, cudaStream_t st) {
    const long long items = std::max<long long>({n, nf, 1LL});
    k_rl_start<<<grid_for(items, 256), 256, 0, st>>>(start, frontier, nf, n, old_of_new, new_of_old, start2,
                                                     frontier2);
    count_launch();
    return cudaGetLastError();
}

}  // namespace kc
