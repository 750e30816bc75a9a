// Persistent sweep kernel: the local coreness iteration of Alg. 1 on the GPU.
//
// One cooperative launch runs every sweep.  Sweep s evaluates the vertices of
// frontier F_s: each computes the h-index of its neighbours' estimates capped
// at its own estimate (computeCoreness of Alg. 1, read as Montresor's
// computeIndex).  If that is lower, the estimate is lowered and neighbours are
// pushed into F_{s+1} by the activation rule (below).  Estimates only
// decrease, so they are updated in place while other vertices of the same
// sweep read them (asynchronous mode).  The run ends when a frontier is empty
// (the `changed` flag of Alg. 2/3 becomes the frontier count).
//
// Activation (u lowered from k to h, x = the value of est[v] that u reads):
//   simple  (selective sending, Sec. III-B):          push v iff h < x.
//   refined (Sec. IV, Further Optimizations):         push v iff h < x and
//           (x <= k  or  v may still be evaluating in this sweep).
// Only v writes est[v], and only while it is evaluated.  A vertex of F_s
// clears its own membership bit once its evaluation is over (a release, after
// its estimate store).  When u finds v's bit clear with an acquire read (v is
// done, or was never in F_s), it reads est[v] again and
// applies FastK's condition h < x <= k to that value: v's final value of the
// sweep.  If it exceeds k, v's h-index never counted u (u's value was at most
// k), so u's decrease cannot lower it.  When v's bit is still set, v may be
// reading u's old value right now, and the simple rule applies.  Either way
// every vertex whose support u withdraws is re-evaluated; a stale read can
// only over-activate.  (The plain refined condition, with no second read, is
// unsafe with in-place updates: v may lower concurrently using u's old value.)
// Membership bits are cleared only for the warp and CTA tiers, whose
// re-evaluation is expensive; a set bit is always safe.
//
// Degree tiers (est word bits 30-31): d <= t_lo one thread per vertex, its
// neighbour ids and estimates in registers and a byte-packed register
// histogram; d <= t_hi one warp per vertex, counts by warp reduction; larger
// degrees one CTA per vertex with a shared-memory histogram.  Work is handed
// out by atomic cursors (the dynamic chunking of Alg. 2), hubs first.
// Frontier membership is a bitmap per sweep (no vertex twice in a list);
// pushes are warp-aggregated.  Lists and bitmaps rotate over three sweeps so
// that F_s membership stays readable during sweep s and F_{s-1}'s bits are
// cleared during sweep s.
//
// Sweeps are separated by a grid barrier; once a frontier is at most tail_max
// vertices with no CTA-tier and few warp-tier vertices, CTA 0 continues alone
// with block barriers (the GPU analogue of FastK's switch to sequential
// processing, Sec. IV) and the other CTAs wait, to rejoin if the frontier
// grows again.  Every wait is bounded by timeout_ns
// (globaltimer) and reports KCORE_ERR_TIMEOUT instead of hanging.
//
// Synchronous mode (KCORE_SYNC_MODE) follows Alg. 3: phase A computes new
// values against the unchanged estimates and records them; after a barrier
// phase B writes them; with the refined rule a third phase decides
// activations against the written values: new_u < est(v) <= old_u.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "kc_common.cuh"

namespace kc {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxBlock = 512;
constexpr int kMinBlocks = 2;
constexpr int kTailMed = 16;        // warp-tier vertices a single-CTA tail sweep may hold
constexpr int kMedR = 4;             // warp tier: up to 32 * kMedR neighbours in registers

__device__ __forceinline__ unsigned long long gtime_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned vload(const unsigned* p) { return *(const volatile unsigned*)p; }
__device__ __forceinline__ int vload(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ long long vload(const long long* p) { return *(const volatile long long*)p; }

// Estimates, lists and bitmaps are read through L2 (ld.global.cg): another SM
// may have written them, and an L1 copy from an earlier sweep would be stale.
__device__ __forceinline__ uint32_t est_load(const uint32_t* p) { return __ldcg(p); }
__device__ __forceinline__ int list_load(const int* p) { return __ldcg(p); }


struct Acc {
    unsigned evaluated, updates, pushes;
    unsigned long long degsum;   // frontier degree sum
    unsigned long long skipped;  // adjacency entries an early exit did not read
    unsigned long long dec;      // sum of estimate decreases
    unsigned long long deg_w;    // of which warp tier
    unsigned long long deg_c;    // of which CTA tier
};

// Per-warp push buffers: each warp collects its pushes in its own slice of
// shared memory and appends them to the global frontier list itself, with one
// atomic per tier per flush (a single global counter per tier would otherwise
// serialise every push) and coalesced stores.  No CTA-wide synchronisation.
constexpr int kWCap0 = 64, kWCap1 = 32, kWCap2 = 32;
constexpr int kWCap = kWCap0 + kWCap1 + kWCap2;

__device__ __forceinline__ int wcap(int q) { return q == 0 ? kWCap0 : (q == 1 ? kWCap1 : kWCap2); }
__device__ __forceinline__ int woff(int q) { return q == 0 ? 0 : (q == 1 ? kWCap0 : kWCap0 + kWCap1); }

struct Sweep {
    const SweepArgs* a;
    int cur, nxt;          // counter slots
    const int* lcur;
    int* lnxt;
    const uint32_t* bmc;   // F_s membership
    uint32_t* bmc_w;       // the same bitmap, for clearing finished vertices
    bool mark;             // clear the bits of finished warp / CTA tier vertices
    uint32_t* bmn;         // F_{s+1} membership
    int* wbuf;             // shared: this warp's push buffer (kWCap entries)
};

// Warp-uniform fill counts of the warp's push buffer.
struct WarpQ {
    unsigned n[kTiers];
};

// Membership word read with acquire semantics: once v's bit is seen clear,
// v's estimate store made before its release is visible.
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// A thread-tier vertex never clears its own membership bit (done marks are
// made by the warp and CTA tiers only), so its bit in F_s does not change
// during sweep s: a plain read of it is exact, and a thread-tier neighbour
// whose bit is clear is not evaluated in this sweep, so the value already
// read is its final one.  Only warp- and CTA-tier neighbours need the
// acquire read and the second read of their estimate.
__device__ __forceinline__ uint32_t member_word(const Sweep& S, int v, uint32_t tier) {
    return tier == 0 ? __ldcg(S.bmc + (v >> 5)) : ld_acquire(S.bmc + (v >> 5));
}

// Refined rule (asynchronous) for a neighbour v read as x (tier bits in xw),
// h < x, while u goes from k to h: push if x <= k or v may still be
// evaluating (bit set); otherwise decide on v's final value: x itself for a
// thread-tier v, else read again after the bit.
__device__ __forceinline__ bool refined_push(const Sweep& S, int h, int k, int v, uint32_t xw) {
    const int x = (int)(xw & kEstMask);
    if (x <= k) return true;
    const uint32_t tier = xw >> kEstBits;
    if ((member_word(S, v, tier) >> (v & 31)) & 1u) return true;
    if (tier == 0) return false;  // x > k is its final value
    const int x2 = (int)(est_load(S.a->est + v) & kEstMask);
    return h < x2 && x2 <= k;
}

// Marks u's evaluation in sweep s as over (warp and CTA tiers, refined
// asynchronous mode): clears its F_s bit with release semantics, after its
// estimate store.
__device__ __forceinline__ void mark_done(const Sweep& S, int u) {
    const uint32_t m = ~(1u << (u & 31));
    asm volatile("red.release.gpu.global.and.b32 [%0], %1;" ::"l"(S.bmc_w + (u >> 5)), "r"(m) : "memory");
}

// Appends the warp's buffered pushes of tier q to the global list.  All 32
// lanes call (warp-uniform).
__device__ __forceinline__ void warp_flush(const Sweep& S, WarpQ& Q, int q) {
    const unsigned c = Q.n[q];
    if (c == 0) return;
    const int lane = threadIdx.x & 31;
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(&S.a->ctl->fcnt[S.nxt][q], c);
    base = __shfl_sync(kFull, base, 0);
    int* dst = S.lnxt + S.a->tier_off[q] + base;
    for (unsigned i = lane; i < c; i += 32) dst[i] = S.wbuf[woff(q) + i];
    __syncwarp();
    Q.n[q] = 0;
}

// End-of-sweep flush of every warp's push buffers with one global atomic per
// tier per CTA (instead of one per warp: thousands of warps adding to the same
// three counters serialise on them).  All threads of the CTA call.
// s_cnt: 3 * 32 words of shared memory.
__device__ __forceinline__ void cta_flush_all(const Sweep& S, WarpQ& Q, uint32_t* s_cnt) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
        for (int q = 0; q < kTiers; q++) s_cnt[q * 32 + wid] = Q.n[q];
    __syncthreads();
    if (wid == 0) {
        for (int q = 0; q < kTiers; q++) {
            const unsigned c = lane < nw ? s_cnt[q * 32 + lane] : 0u;
            unsigned incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            const unsigned total = __shfl_sync(kFull, incl, 31);
            unsigned base = 0;
            if (lane == 0 && total) base = atomicAdd(&S.a->ctl->fcnt[S.nxt][q], total);
            base = __shfl_sync(kFull, base, 0);
            if (lane < nw) s_cnt[q * 32 + lane] = base + incl - c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kTiers; q++) {
        const unsigned c = Q.n[q];
        if (c) {
            int* dst = S.lnxt + S.a->tier_off[q] + s_cnt[q * 32 + wid];
            for (unsigned i = lane; i < c; i += 32) dst[i] = S.wbuf[woff(q) + i];
        }
        Q.n[q] = 0;
    }
}

// All 32 lanes call this.  A lane with `fresh` appends v (tier `tier`) to
// the warp's push buffer; v's membership bit is already claimed.
__device__ __forceinline__ void warp_enqueue(const Sweep& S, WarpQ& Q, bool fresh, int v,
                                             uint32_t tier, Acc& acc) {
    const int lane = threadIdx.x & 31;
    const unsigned any = __ballot_sync(kFull, fresh);
    if (!any) return;
#pragma unroll
    for (int q = 0; q < kTiers; q++) {
        const unsigned m = __ballot_sync(kFull, fresh && tier == (uint32_t)q);
        if (m) {
            const unsigned cnt = (unsigned)__popc(m);
            if (Q.n[q] + cnt > (unsigned)wcap(q)) warp_flush(S, Q, q);
            if (fresh && tier == (uint32_t)q)
                S.wbuf[woff(q) + Q.n[q] + __popc(m & ((1u << lane) - 1u))] = v;
            Q.n[q] += cnt;
            __syncwarp();
        }
    }
    if (lane == 0) acc.pushes += (unsigned)__popc(any);
}

// Claims v's bit in the next frontier's bitmap; true if this call set it.
__device__ __forceinline__ bool claim(const Sweep& S, int v) {
    const uint32_t bit = 1u << (v & 31);
    uint32_t* word = S.bmn + (v >> 5);
    if (__ldcg(word) & bit) return false;
    return (atomicOr(word, bit) & bit) == 0;
}

// All 32 lanes call this: claim and enqueue one candidate per lane.
__device__ __forceinline__ void warp_push(const Sweep& S, WarpQ& Q, bool want, int v,
                                          uint32_t tier, Acc& acc) {
    const bool fresh = want && claim(S, v);
    warp_enqueue(S, Q, fresh, v, tier, acc);
}

// Pushes up to N candidates per lane (bit j of `cand` selects vs[j]).  The
// activation filter, the bitmap pre-tests and the atomics of all N slots are
// issued before any result is used, so they overlap in flight.  All lanes call.
template <int N>
__device__ __forceinline__ void warp_push_n(const Sweep& S, WarpQ& Q, uint32_t cand, int h, int k,
                                            const int (&vs)[N], const uint32_t (&xw)[N],
                                            Acc& acc) {
    if (!__any_sync(kFull, cand != 0)) return;
    uint32_t word[N];
    if (S.a->refined) {
        // refined rule: a candidate read above k is kept if it may still be
        // evaluating; otherwise its final value decides
        uint32_t chk = 0;
#pragma unroll
        for (int j = 0; j < N; j++)
            if (((cand >> j) & 1u) && (int)(xw[j] & kEstMask) > k) chk |= 1u << j;
#pragma unroll
        for (int j = 0; j < N; j++)
            word[j] = ((chk >> j) & 1u) ? member_word(S, vs[j], xw[j] >> kEstBits) : 0u;
        uint32_t again = 0;
#pragma unroll
        for (int j = 0; j < N; j++) {
            if (((chk >> j) & 1u) && !((word[j] >> (vs[j] & 31)) & 1u)) {
                if ((xw[j] >> kEstBits) == 0) cand &= ~(1u << j);  // thread tier: x > k is final
                else again |= 1u << j;
            }
        }
        if (again) {
#pragma unroll
            for (int j = 0; j < N; j++) word[j] = ((again >> j) & 1u) ? est_load(S.a->est + vs[j]) : 0u;
#pragma unroll
            for (int j = 0; j < N; j++) {
                const int x2 = (int)(word[j] & kEstMask);
                if (((again >> j) & 1u) && !(h < x2 && x2 <= k)) cand &= ~(1u << j);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < N; j++)
        word[j] = ((cand >> j) & 1u) ? __ldcg(S.bmn + (vs[j] >> 5)) : 0xffffffffu;
#pragma unroll
    for (int j = 0; j < N; j++) {
        const uint32_t bit = 1u << (vs[j] & 31);
        if (((cand >> j) & 1u) && !(word[j] & bit)) word[j] = atomicOr(S.bmn + (vs[j] >> 5), bit);
        else word[j] = 0xffffffffu;
    }
    uint32_t fresh = 0;
#pragma unroll
    for (int j = 0; j < N; j++)
        if (((cand >> j) & 1u) && !((word[j] >> (vs[j] & 31)) & 1u)) fresh |= 1u << j;
    if (!__any_sync(kFull, fresh != 0)) return;
#pragma unroll
    for (int j = 0; j < N; j++)
        if (__any_sync(kFull, (fresh >> j) & 1u))
            warp_enqueue(S, Q, (fresh >> j) & 1u, vs[j], xw[j] >> kEstBits, acc);
}

// Hands out items [0, count) of one tier: each warp takes `warp_items` at a
// time from the global cursor and calls fn(lo, hi).
template <class Fn>
__device__ __forceinline__ void run_tier(unsigned* cursor, unsigned count, unsigned warp_items,
                                         Fn fn) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned i = 0;
        if (lane == 0) i = atomicAdd(cursor, warp_items);
        i = __shfl_sync(kFull, i, 0);
        if (i >= count) return;
        fn(i, min(count, i + warp_items));
    }
}

// Record an update (u -> h).  Asynchronous: written in place.  Synchronous:
// appended to the update list, written after the barrier.  All lanes call.
__device__ __forceinline__ void warp_update(const Sweep& S, bool changed, int u, uint32_t w,
                                            int h) {
    const SweepArgs& a = *S.a;
    if (!a.sync_mode) {
        if (changed) a.est[u] = (w & ~kEstMask) | (uint32_t)h;
        return;
    }
    const int lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(kFull, changed);
    if (!m) return;
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(&a.ctl->ucnt[S.cur], (unsigned)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (changed) {
        const unsigned i = base + __popc(m & ((1u << lane) - 1u));
        a.upd_list[i] = u;
        a.upd_val[i] = h;
    }
}

// ---------------------------------------------------------------- thread tier
// Edge-parallel evaluation of 32 low-degree vertices, one per lane.  The warp
// takes an exclusive prefix sum of their degrees and walks their combined
// adjacency one entry per lane per step; the owner of entry g is the last lane
// whose prefix is <= g (a five-step shuffle bisection).  Each entry adds
// min(x, k_owner) to its owner's histogram of threshold counts, held in shared
// memory as bytes: word i of lane o counts #{x >= t} for t = 4i+1 .. 4i+4.
// The capped h-index of the owner is the number of thresholds t with
// count_t >= t, because that predicate holds exactly for t <= h.
// The first kLowCache steps keep their (entry, estimate) pairs in registers
// for the activation pass; longer walks read them again.
constexpr int kLowCache = 4;

__device__ __forceinline__ uint32_t byte_ramp(int q) {
    // bytes 0..q-1 set to 1 (q clamped to [0, 4])
    return q >= 4 ? 0x01010101u : (q <= 0 ? 0u : (0x01010101u & ((1u << (8 * q)) - 1u)));
}

__device__ __forceinline__ int owner_of(int g, int excl) {
    int o = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        const int e = __shfl_sync(kFull, excl, o + step);
        if (e <= g) o += step;
    }
    return o;
}

// `valid`: u is in range (DENSE: u is a vertex id, `member` its frontier bit;
// the row and estimate loads do not wait for the membership word).
template <typename Off, int TW, bool DENSE>
__device__ __forceinline__ void low_warp(const Sweep& S, WarpQ& Q, const Off* __restrict__ rp,
                                         bool valid, int u, const uint32_t* mword, uint32_t* hist,
                                         Acc& acc) {
    const SweepArgs& a = *S.a;
    const int lane = threadIdx.x & 31;
    long long b = 0;
    int d = 0, k = 0;
    uint32_t w = 0, mw = 0xffffffffu;
    if (DENSE) mw = __ldcg(mword);
    if (valid) {
        w = est_load(a.est + u);
        b = (long long)rp[u];
        d = (int)((long long)rp[u + 1] - b);
        k = (int)(w & kEstMask);
    }
    if (DENSE) valid = valid && ((mw >> lane) & 1u) && (w >> kEstBits) == 0;  // other tiers: lists
    if (valid) {
        acc.evaluated += 1;
        acc.degsum += (unsigned)d;
    }
    const bool work = valid && k > 0;
    const int dd = work ? d : 0;
    int incl = dd;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    const int excl = incl - dd;
    const int total = __shfl_sync(kFull, incl, 31);
    if (total == 0) return;
#pragma unroll
    for (int i = 0; i < TW; i++) hist[i * 32 + lane] = 0;
    __syncwarp();
    // pass 1: histograms.  The first kLowCache steps issue all their loads
    // before using any (two dependent round trips in all); longer walks loop.
    int cv[kLowCache], co[kLowCache];
    uint32_t cx[kLowCache];
#pragma unroll
    for (int c = 0; c < kLowCache; c++) {
        const int g = 32 * c + lane;
        co[c] = owner_of(g, excl);
        const long long bo = __shfl_sync(kFull, b, co[c]);
        const int eo = __shfl_sync(kFull, excl, co[c]);
        cv[c] = g < total ? __ldg(a.col + bo + (g - eo)) : -1;
    }
#pragma unroll
    for (int c = 0; c < kLowCache; c++) cx[c] = cv[c] >= 0 ? est_load(a.est + cv[c]) : 0u;
#pragma unroll
    for (int c = 0; c < kLowCache; c++) {
        const int ko = __shfl_sync(kFull, k, co[c]);
        if (cv[c] >= 0) {
            const int x = (int)(cx[c] & kEstMask);
            const int y = x < ko ? x : ko;
#pragma unroll
            for (int i = 0; i < TW; i++) {
                const uint32_t m = byte_ramp(y - 4 * i);
                if (m) atomicAdd(&hist[i * 32 + co[c]], m);
            }
        }
    }
    for (int g0 = 32 * kLowCache; g0 < total; g0 += 32) {
        const int g = g0 + lane;
        const int o = owner_of(g, excl);
        const long long bo = __shfl_sync(kFull, b, o);
        const int eo = __shfl_sync(kFull, excl, o);
        const int ko = __shfl_sync(kFull, k, o);
        if (g < total) {
            const int v = __ldg(a.col + bo + (g - eo));
            const int x = (int)(est_load(a.est + v) & kEstMask);
            const int y = x < ko ? x : ko;
#pragma unroll
            for (int i = 0; i < TW; i++) {
                const uint32_t m = byte_ramp(y - 4 * i);
                if (m) atomicAdd(&hist[i * 32 + o], m);
            }
        }
    }
    __syncwarp();
    int h = 0;
#pragma unroll
    for (int i = 0; i < TW; i++) {
        const uint32_t thr = (uint32_t)(4 * i + 1) | ((uint32_t)(4 * i + 2) << 8) |
                             ((uint32_t)(4 * i + 3) << 16) | ((uint32_t)(4 * i + 4) << 24);
        h += __popc(__vcmpgeu4(hist[i * 32 + lane], thr) & 0x01010101u);
    }
    __syncwarp();
    const bool changed = work && h < k;
    if (changed) {
        acc.updates += 1;
        acc.dec += (unsigned long long)(k - h);
    }
    warp_update(S, changed, u, w, h);
    if (a.sync_mode && a.refined) return;  // activation runs after the update phase
    if (!__any_sync(kFull, changed)) return;
    // pass 2: activation.  Cached steps are claimed together.
    {
        int pv[kLowCache];
        uint32_t word[kLowCache];
        uint32_t cand = 0;
#pragma unroll
        for (int c = 0; c < kLowCache; c++) {
            const int o = co[c];
            const int ho = __shfl_sync(kFull, h, o), ko = __shfl_sync(kFull, k, o);
            const bool ch = __shfl_sync(kFull, changed, o);
            const int x = (int)(cx[c] & kEstMask);
            pv[c] = cv[c];
            if (cv[c] >= 0 && ch && x > ho) {
                cand |= 1u << c;
                word[c] = (a.refined && x > ko) ? member_word(S, cv[c], cx[c] >> kEstBits) : 0xffffffffu;
            } else {
                word[c] = 0xffffffffu;
            }
        }
        uint32_t again = 0;
#pragma unroll
        for (int c = 0; c < kLowCache; c++) {
            if (((cand >> c) & 1u) && !((word[c] >> (pv[c] & 31)) & 1u)) {
                if ((cx[c] >> kEstBits) == 0) cand &= ~(1u << c);  // thread tier: x > k is final
                else again |= 1u << c;
            }
        }
        if (__any_sync(kFull, again != 0)) {  // refined rule, v done or never in F_s: its final value decides
#pragma unroll
            for (int c = 0; c < kLowCache; c++)
                word[c] = ((again >> c) & 1u) ? est_load(a.est + pv[c]) : 0u;
#pragma unroll
            for (int c = 0; c < kLowCache; c++) {
                const int o = co[c];
                const int ho = __shfl_sync(kFull, h, o), ko = __shfl_sync(kFull, k, o);
                const int x2 = (int)(word[c] & kEstMask);
                if (((again >> c) & 1u) && !(ho < x2 && x2 <= ko)) cand &= ~(1u << c);
            }
        }
#pragma unroll
        for (int c = 0; c < kLowCache; c++)
            word[c] = ((cand >> c) & 1u) ? atomicOr(S.bmn + (pv[c] >> 5), 1u << (pv[c] & 31))
                                          : 0xffffffffu;
#pragma unroll
        for (int c = 0; c < kLowCache; c++) {
            const bool fresh = ((cand >> c) & 1u) && !((word[c] >> (pv[c] & 31)) & 1u);
            if (__any_sync(kFull, fresh)) warp_enqueue(S, Q, fresh, pv[c], cx[c] >> kEstBits, acc);
        }
    }
    for (int g0 = 32 * kLowCache; g0 < total; g0 += 32) {
        const int g = g0 + lane;
        const int o = owner_of(g, excl);
        const long long bo = __shfl_sync(kFull, b, o);
        const int eo = __shfl_sync(kFull, excl, o);
        const int ho = __shfl_sync(kFull, h, o), ko = __shfl_sync(kFull, k, o);
        const bool ch = __shfl_sync(kFull, changed, o);
        bool want = false;
        int v = 0;
        uint32_t xw = 0;
        if (g < total && ch) {
            v = __ldg(a.col + bo + (g - eo));
            xw = est_load(a.est + v);
            const int x = (int)(xw & kEstMask);
            want = x > ho && (!a.refined || refined_push(S, ho, ko, v, xw));
        }
        warp_push(S, Q, want, v, xw >> kEstBits, acc);
    }
}

// ---------------------------------------------------------------- warp tier
// One warp per vertex, up to 32*R neighbour estimates held in registers; the
// count of neighbours >= t comes from a warp reduction, and h by bisection on
// t after the no-change test t = k.
template <int R>
__device__ __forceinline__ void med_vertex(const Sweep& S, WarpQ& Q, int u, long long b, int d,
                                           uint32_t w, Acc& acc) {
    const SweepArgs& a = *S.a;
    const int lane = threadIdx.x & 31;
    const int k = (int)(w & kEstMask);
    if (lane == 0) {
        acc.evaluated += 1;
        acc.degsum += (unsigned)d;
        acc.deg_w += (unsigned)d;
    }
    if (k == 0) {
        if (S.mark && lane == 0) mark_done(S, u);
        return;
    }
    int vs[R];
    uint32_t xw[R];
#pragma unroll
    for (int r = 0; r < R; r++) vs[r] = (r * 32 + lane < d) ? __ldg(a.col + b + r * 32 + lane) : -1;
#pragma unroll
    for (int r = 0; r < R; r++) xw[r] = vs[r] >= 0 ? est_load(a.est + vs[r]) : 0u;
    auto count_ge = [&](int t) {
        int c = 0;
#pragma unroll
        for (int r = 0; r < R; r++) c += (int)(xw[r] & kEstMask) >= t ? 1 : 0;
        return (int)__reduce_add_sync(kFull, (unsigned)c);
    };
    int h = k;
    if (count_ge(k) < k) {
        int lo = 0, hi = k - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (count_ge(mid) >= mid) lo = mid;
            else hi = mid - 1;
        }
        h = lo;
    }
    if (h >= k) {
        if (S.mark && lane == 0) mark_done(S, u);
        return;
    }
    if (lane == 0) {
        acc.updates += 1;
        acc.dec += (unsigned long long)(k - h);
    }
    warp_update(S, lane == 0, u, w, h);
    if (S.mark && lane == 0) mark_done(S, u);
    if (a.sync_mode && a.refined) return;
    uint32_t cand = 0;
#pragma unroll
    for (int r = 0; r < R; r++)
        if (vs[r] >= 0 && (int)(xw[r] & kEstMask) > h) cand |= 1u << r;
    warp_push_n<R>(S, Q, cand, h, k, vs, xw, acc);
}

// Warp tier, degrees above 32 * kMedR (up to kMedBig): one warp per vertex.
// The first pass gathers the estimates kMedU per lane at a time and keeps, as
// 16 bits in the warp's slice of shared memory, y = min(x, k + 1) (12 bits)
// and the neighbour's degree tier (bits 14-15), counting x >= k; once that
// count reaches k the estimate stands and the pass stops.  Otherwise h < k is
// found by bisection on t with counts of y >= t over the staged words (eight
// per 16-byte read; the slice is zero-padded to a whole number of reads), and
// a last pass pushes the neighbours with y > h.  A neighbour staged with
// y <= k is pushed on its staged value: the estimates only decrease, so the
// value read now would be at most y, the refined condition x <= k holds, and
// a value that dropped to h or below since only over-activates.  Only a
// neighbour staged above k is gathered again for the refined test.
constexpr int kMedU = 4;
constexpr int kMedSlice = kMedBig / 2;  // words per warp
constexpr int kMedWin = 32;             // exact counts kept for [k - kMedWin, k - 1]
constexpr uint32_t kStageVal = 0x0fffu;   // value bits of a staged word
constexpr int kStageTier = 14;            // tier bits of a staged word

__device__ __forceinline__ void med_big_vertex(const Sweep& S, WarpQ& Q, int u, long long b, int d,
                                               uint32_t w, uint32_t* slice, uint32_t* whist, Acc& acc) {
    const SweepArgs& a = *S.a;
    const int lane = threadIdx.x & 31;
    uint16_t* sx = (uint16_t*)slice;
    const int k = (int)(w & kEstMask);
    // values in the window [wl, k - 1] are also counted exactly in pass 1, so
    // that a vertex whose new estimate lands there (the usual case: the
    // estimates drop by a few per evaluation) needs no bisection
    const int wl = k > kMedWin ? k - kMedWin : 0;
    whist[lane] = 0;
    __syncwarp();
    if (lane == 0) {
        acc.evaluated += 1;
        acc.degsum += (unsigned)d;
        acc.deg_w += (unsigned)d;
    }
    if (k == 0) {
        if (S.mark && lane == 0) mark_done(S, u);
        return;
    }
    const int* colb = a.col + b;
    int ck = 0, read = d;
    bool stands = false;
    for (int j0 = 0; j0 < d; j0 += 32 * kMedU) {
        int vs[kMedU];
        uint32_t xw[kMedU];
#pragma unroll
        for (int r = 0; r < kMedU; r++) {
            const int j = j0 + r * 32 + lane;
            vs[r] = j < d ? __ldg(colb + j) : -1;
        }
#pragma unroll
        for (int r = 0; r < kMedU; r++) xw[r] = vs[r] >= 0 ? est_load(a.est + vs[r]) : 0u;
        int c = 0;
#pragma unroll
        for (int r = 0; r < kMedU; r++) {
            if (vs[r] >= 0) {
                const int x = (int)(xw[r] & kEstMask);
                c += x >= k ? 1 : 0;
                const uint32_t y = (uint32_t)(x <= k ? x : k + 1);
                sx[j0 + r * 32 + lane] = (uint16_t)(y | ((xw[r] >> kEstBits) << kStageTier));
                if (x >= wl && x < k) atomicAdd(&whist[x - wl], 1u);
            }
        }
        ck += (int)__reduce_add_sync(kFull, (unsigned)c);
        if (ck >= k) {
            stands = true;
            read = min(d, j0 + 32 * kMedU);
            break;
        }
    }
    if (lane == 0) acc.skipped += (unsigned long long)(d - read);
    if (stands) {
        if (S.mark && lane == 0) mark_done(S, u);
        __syncwarp();
        return;
    }
    // h from the window: lane l stands for t = wl + l, with
    // #{y >= t} = ck + the window counts of bins >= l (a suffix sum); the
    // predicate #{y >= t} >= t holds for a prefix of t, so h is the last lane
    // where it holds, if any
    __syncwarp();
    uint32_t sfx = whist[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_down_sync(kFull, sfx, o);
        if (lane + o < 32) sfx += t;
    }
    const int tw = wl + lane;
    const unsigned inwin = __ballot_sync(kFull, tw < k && (int)(sfx + (uint32_t)ck) >= tw);
    const int padded = (d + 255) & ~255;  // whole 16-byte reads for every lane
    for (int j = d + lane; j < padded; j += 32) sx[j] = 0;
    __syncwarp();
    const uint4* sv = (const uint4*)slice;
    const int nv = padded >> 8;  // 16-byte reads per lane
    int lo = 0, hi = k - 1;      // count(y >= 0) = d >= 0 holds; h < k
    if (inwin) {
        lo = hi = wl + (31 - __clz((int)inwin));
    } else {
        hi = wl - 1;             // below the window (wl > 0 here: t = 0 always holds)
    }
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const uint32_t mid2 = (uint32_t)mid * 0x00010001u;
        const uint32_t vm = kStageVal * 0x00010001u;
        int c = 0;
        for (int i = 0; i < nv; i++) {
            const uint4 q = sv[i * 32 + lane];
            c += __popc(__vcmpgeu2(q.x & vm, mid2)) + __popc(__vcmpgeu2(q.y & vm, mid2)) +
                 __popc(__vcmpgeu2(q.z & vm, mid2)) + __popc(__vcmpgeu2(q.w & vm, mid2));
        }
        c = (int)__reduce_add_sync(kFull, (unsigned)c) >> 4;  // 16 bits set per match
        if (c >= mid) lo = mid;
        else hi = mid - 1;
    }
    const int h = lo;
    if (lane == 0) {
        acc.updates += 1;
        acc.dec += (unsigned long long)(k - h);
    }
    warp_update(S, lane == 0, u, w, h);
    if (S.mark && lane == 0) mark_done(S, u);
    if (a.sync_mode && a.refined) {
        __syncwarp();
        return;
    }
    for (int j0 = 0; j0 < d; j0 += 32 * kMedU) {
        int vs[kMedU];
        uint32_t xw[kMedU];
        uint32_t cand = 0, again = 0;
#pragma unroll
        for (int r = 0; r < kMedU; r++) {
            const int j = j0 + r * 32 + lane;
            const uint32_t y = j < d ? (uint32_t)sx[j] : 0u;
            const int yv = (int)(y & kStageVal);
            const bool want = j < d && yv > h;
            vs[r] = want ? __ldg(colb + j) : -1;
            xw[r] = ((y >> kStageTier) << kEstBits) | (uint32_t)yv;
            if (want) {
                if (yv <= k) cand |= 1u << r;
                else again |= 1u << r;
            }
        }
        if (again) {
#pragma unroll
            for (int r = 0; r < kMedU; r++)
                if ((again >> r) & 1u) xw[r] = est_load(a.est + vs[r]);
#pragma unroll
            for (int r = 0; r < kMedU; r++)
                if (((again >> r) & 1u) && (int)(xw[r] & kEstMask) > h) cand |= 1u << r;
        }
        warp_push_n<kMedU>(S, Q, cand, h, k, vs, xw, acc);
    }
    __syncwarp();
}

// ---------------------------------------------------------------- CTA tier
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total,
                                                    uint32_t* wsum) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < nw ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        wsum[lane] = s;
    }
    __syncthreads();
    const uint32_t r = (wid ? wsum[wid - 1] : 0u) + x - v;
    *total = wsum[nw - 1];
    __syncthreads();
    return r;
}

// Over buckets i in [0, nb) of s_hist, with `above` values beyond the last
// bucket: counts how many i satisfy
//   above + #{values in buckets >= i} >= base + i * width.
// The predicate is monotone (true for a prefix of i), so the count minus one
// is the last i where it holds.  If want_after >= 0, *after gets
// above + #{values in buckets >= want_after}.
__device__ __forceinline__ int hub_count_true(const uint32_t* s_hist, int nb, uint32_t above,
                                              long long base, long long width, int want_after,
                                              uint32_t* after, uint32_t* wsum, int* s_int) {
    const int T = blockDim.x, tid = threadIdx.x;
    const int per = (nb + T - 1) / T;
    const int i0 = min(nb, tid * per), i1 = min(nb, i0 + per);
    uint32_t local = 0;
    for (int i = i0; i < i1; i++) local += s_hist[i];
    uint32_t total;
    uint32_t run = block_excl_scan(local, &total, wsum);
    int mine = 0;
    for (int i = i0; i < i1; i++) {
        const long long ge = (long long)above + (long long)(total - run);
        if (i == want_after) *after = (uint32_t)ge;
        if (ge >= base + (long long)i * width) mine++;
        run += s_hist[i];
    }
    if (want_after == nb && tid == 0) *after = above;
    const unsigned wm = __reduce_add_sync(kFull, (unsigned)mine);
    if ((tid & 31) == 0) atomicAdd(s_int, (int)wm);
    __syncthreads();
    const int r = *s_int;
    __syncthreads();
    if (tid == 0) *s_int = 0;
    __syncthreads();
    return r;
}

// Counts of min(x, k) by power-of-two class, private to each thread: word
// i * T + tid holds two 16-bit counters, classes 2i and 2i+1.  Conflict-free
// (a thread's words sit in its own bank) and free of atomics.
constexpr int kHubP = 4;                    // adjacency loads in flight per thread
constexpr int kLogClasses = 30;             // estimates are below 2^30
constexpr int kLogWords = kLogClasses / 2;
constexpr int kFoldChunks = 65535 / kHubP;  // a 16-bit counter cannot overflow sooner

// Streams colb[0, d) in rounds of T * kHubP entries, kHubP loads in flight
// per thread.  fn(vs, c) gets this thread's kHubP ids of round c (-1 past d)
// and returns true to stop (its result must be CTA-uniform).  Returns the
// entries covered.
template <class Fn>
__device__ __forceinline__ long long hub_stream(const int* colb, long long d, Fn fn) {
    const int T = blockDim.x, tid = threadIdx.x;
    const long long step = (long long)T * kHubP;
    const long long nch = (d + step - 1) / step;
    for (long long c = 0; c < nch; c++) {
        int vs[kHubP];
#pragma unroll
        for (int i = 0; i < kHubP; i++) {
            const long long j = c * step + (long long)i * T + tid;
            vs[i] = j < d ? __ldg(colb + j) : -1;
        }
        if (fn(vs, c)) return min(d, (c + 1) * step);
    }
    return d;
}

// Histogram of the values y in [lo, hi] in buckets (y - lo) >> shift;
// y = min(x, k).  nb <= kHubBins.
__device__ __forceinline__ void hub_hist_pass(const SweepArgs& a, const int* colb, long long d,
                                              int k, long long lo, long long hi, int shift,
                                              int nb, uint32_t* s_hist) {
    const int T = blockDim.x, tid = threadIdx.x;
    for (int i = tid; i < nb; i += T) s_hist[i] = 0;
    __syncthreads();
    hub_stream(colb, d, [&](const int (&vs)[kHubP], long long) {
        int xs[kHubP];
#pragma unroll
        for (int i = 0; i < kHubP; i++) xs[i] = vs[i] >= 0 ? (int)(est_load(a.est + vs[i]) & kEstMask) : -1;
#pragma unroll
        for (int i = 0; i < kHubP; i++) {
            const long long y = xs[i] < k ? xs[i] : k;
            if (xs[i] >= 0 && y >= lo && y <= hi) atomicAdd(&s_hist[(int)((y - lo) >> shift)], 1u);
        }
        return false;
    });
    __syncthreads();
}

// One CTA per hub u with estimate k.
//   Pass 1 streams the adjacency and counts c_k = #{x >= k}, the no-change
//   test of the capped h-index: as soon as the CTA's total reaches k the
//   estimate stands and the pass stops, so a hub whose estimate holds reads
//   only as much of its adjacency as it takes to find k supporters.
//   Alongside, each thread counts min(x, k) by power-of-two class.
//   Pass 1 also keeps an exact histogram of the values in the window
//   [wl, k - 1], wl = max(k / 2, k - kHubBins).
//   If c_k < k after the whole adjacency, h < k, and with N_m = #{min(x,k) >=
//   2^m} the largest m* with N_m* >= 2^m* brackets h in
//   [2^m*, min(2^(m*+1), k) - 1].  If the bracket starts inside the window, h
//   is the last t of the window with c_k + #{window values >= t} >= t.
//   Otherwise pass 2 takes the histogram of the values in the bracket
//   (buckets of one value, or coarse buckets and a further pass when the
//   bracket is wider than kHubBins) and h is the last t with #{x >= t} >= t.
//   A last pass pushes the neighbours.
template <typename Off>
__device__ __forceinline__ void hub_vertex(const Sweep& S, WarpQ& Q, const Off* __restrict__ rp,
                                           int u, uint32_t* s_pool, uint32_t* s_cls,
                                           uint32_t* s_hub, uint32_t* wsum, int* s_int,
                                           uint32_t* s_u32, Acc& acc) {
    const SweepArgs& a = *S.a;
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nw = T >> 5;
    uint32_t* s_lg = s_pool;
    uint32_t* s_hist = s_pool;
    uint32_t* s_win = s_pool + kLogWords * T;  // pass 1's histogram of [wl, k - 1]
    const long long b = (long long)rp[u];
    const long long d = (long long)rp[u + 1] - b;
    const uint32_t w = est_load(a.est + u);
    const int k = (int)(w & kEstMask);
    if (tid == 0) {
        acc.evaluated += 1;
        acc.degsum += (unsigned long long)d;
        acc.deg_c += (unsigned long long)d;
    }
    if (k == 0) {
        if (S.mark && tid == 0) mark_done(S, u);
        return;
    }
    const int* colb = a.col + b;
    // values in the window [wl, k - 1] are also counted exactly in pass 1: a
    // hub whose new estimate lands there (the usual case after the first
    // sweep) needs no second pass.  The window stays above k / 2, away from
    // the many small estimates of low-degree neighbours.
    const int wl = max((k + 1) / 2, k - kHubBins);
    const int nw_bins = k - wl;
#pragma unroll
    for (int i = 0; i < kLogWords; i++) s_lg[i * T + tid] = 0;
    for (int i = tid; i < nw_bins; i += T) s_win[i] = 0;
    if (tid < 32) s_cls[tid] = 0;
    if (tid == 0) s_hub[0] = 0;
    __syncthreads();

    // ---- pass 1
    const long long step = (long long)T * kHubP;
    unsigned ck = 0;  // this thread's supporters since the last check
    bool stands = false;
    const long long read = hub_stream(colb, d, [&](const int (&vs)[kHubP], long long c) {
        int xs[kHubP];
#pragma unroll
        for (int i = 0; i < kHubP; i++) xs[i] = vs[i] >= 0 ? (int)(est_load(a.est + vs[i]) & kEstMask) : -1;
#pragma unroll
        for (int i = 0; i < kHubP; i++) {
            const int x = xs[i];
            ck += x >= k ? 1u : 0u;
            const int y = x < k ? x : k;
            if (y > 0) {
                const int m = 31 - __clz(y);
                s_lg[(m >> 1) * T + tid] += 1u << ((m & 1) << 4);
            }
            if (y >= wl && y < k) atomicAdd(&s_win[y - wl], 1u);
        }
        if ((c + 1) % kFoldChunks == 0) {  // keep the 16-bit counters from overflowing
#pragma unroll
            for (int i = 0; i < kLogWords; i++) {
                const uint32_t v = s_lg[i * T + tid];
                s_lg[i * T + tid] = 0;
                if (v & 0xffffu) atomicAdd(&s_cls[2 * i], v & 0xffffu);
                if (v >> 16) atomicAdd(&s_cls[2 * i + 1], v >> 16);
            }
        }
        const unsigned cs = __reduce_add_sync(kFull, ck);
        ck = 0;
        if (lane == 0 && cs) atomicAdd(&s_hub[0], cs);
        __syncthreads();
        const unsigned tot = s_hub[0];
        __syncthreads();
        stands = tot >= (unsigned)k;
        return stands;
    });
    (void)step;
    if (tid == 0) acc.skipped += (unsigned long long)(d - read);
    if (stands) {
        if (S.mark && tid == 0) mark_done(S, u);
        return;
    }
    const unsigned c_k = s_hub[0];

    // ---- bracket from the power-of-two classes
    for (int i = wid; i < kLogWords; i += nw) {
        unsigned lo = 0, hi = 0;
        for (int t = lane; t < T; t += 32) {
            const uint32_t v = s_lg[i * T + t];
            lo += v & 0xffffu;
            hi += v >> 16;
        }
        lo = __reduce_add_sync(kFull, lo);
        hi = __reduce_add_sync(kFull, hi);
        if (lane == 0) {
            s_cls[2 * i] += lo;
            s_cls[2 * i + 1] += hi;
        }
    }
    __syncthreads();
    if (wid == 0) {
        unsigned c = lane < kLogClasses ? s_cls[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {  // suffix sums: N_m = sum over classes >= m
            const unsigned t = __shfl_down_sync(kFull, c, o);
            if (lane + o < 32) c += t;
        }
        const bool pred = lane < kLogClasses && (unsigned long long)c >= (1ull << lane);
        const unsigned bal = __ballot_sync(kFull, pred);
        const int ms = bal ? 31 - __clz(bal) : -1;
        const unsigned n_above = __shfl_sync(kFull, c, ms + 1 < 31 ? ms + 1 : 31);
        if (lane == 0) {
            s_hub[1] = (uint32_t)ms;
            s_hub[2] = n_above;
        }
    }
    __syncthreads();
    const int ms = (int)s_hub[1];
    int h = 0;
    if (ms >= 0 && (1LL << ms) >= (long long)wl) {
        // the bracket lies inside the window: pass 1's histogram decides
        const int nt = hub_count_true(s_win, nw_bins, c_k, wl, 1, -1, s_u32, wsum, s_int);
        h = wl + nt - 1;
    } else if (ms >= 0) {
        long long lo = 1LL << ms;
        long long hi = (2 * lo < (long long)k ? 2 * lo : (long long)k) - 1;
        uint32_t above = 2 * lo <= (long long)k ? s_hub[2] : c_k;  // #{x >= hi + 1}
        for (;;) {
            int shift = 0;
            while (((hi - lo) >> shift) >= kHubBins) shift++;
            const int nb = (int)((hi - lo) >> shift) + 1;
            hub_hist_pass(a, colb, d, k, lo, hi, shift, nb, s_hist);
            const int nt = hub_count_true(s_hist, nb, above, lo, 1LL << shift, -1, s_u32, wsum, s_int);
            if (shift == 0) {
                h = (int)(lo + nt - 1);
                break;
            }
            const int istar = nt - 1;
            if (tid == 0) *s_u32 = 0;
            __syncthreads();
            hub_count_true(s_hist, nb, above, lo, 1LL << shift, istar + 1, s_u32, wsum, s_int);
            above = *s_u32;
            __syncthreads();
            lo += (long long)istar << shift;
            hi = min(lo + (1LL << shift) - 1, hi);
        }
    }
    __syncthreads();
    if (tid == 0) {
        acc.updates += 1;
        acc.dec += (unsigned long long)(k - h);
    }
    if (wid == 0) warp_update(S, tid == 0, u, w, h);
    if (S.mark && tid == 0) mark_done(S, u);
    if (a.sync_mode && a.refined) return;

    // ---- activation
    hub_stream(colb, d, [&](const int (&vs)[kHubP], long long) {
        uint32_t xw[kHubP];
        uint32_t cand = 0;
#pragma unroll
        for (int i = 0; i < kHubP; i++) xw[i] = vs[i] >= 0 ? est_load(a.est + vs[i]) : 0u;
#pragma unroll
        for (int i = 0; i < kHubP; i++)
            if (vs[i] >= 0 && (int)(xw[i] & kEstMask) > h) cand |= 1u << i;
        warp_push_n<kHubP>(S, Q, cand, h, k, vs, xw, acc);
        return false;
    });
    __syncthreads();
}

// ---------------------------------------------------------------- barriers
// Grid barrier (all CTAs are co-resident: cooperative launch).  bar_count
// only grows during a launch (it is zeroed before each launch): the k-th
// barrier of the launch completes when it reaches k * gridDim.  Returns false
// if the wait ran past the budget; the status word then says TIMEOUT.
__device__ bool grid_barrier(SweepCtl* ctl, unsigned& nbar, long long timeout_ns, int* s_ok) {
    __syncthreads();
    nbar += 1;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = nbar * gridDim.x;
        __threadfence();
        atomicAdd(&ctl->bar_count, 1u);
        const unsigned long long t0 = gtime_ns();
        while ((int)(vload(&ctl->bar_count) - target) < 0) {
            if ((long long)(gtime_ns() - t0) > timeout_ns) {
                atomicCAS(&ctl->status, 0, (int)KCORE_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(20);
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// One CTA runs the sweep: its own barrier orders its global accesses.
__device__ __forceinline__ void block_barrier() { __syncthreads(); }

// ---------------------------------------------------------------- kernel
template <typename Off, int T>
__global__ void __launch_bounds__(kMaxBlock, kMinBlocks) k_sweep(const SweepArgs a) {
    // Dynamic shared memory: the warps' push buffers, then one pool that
    // serves, one after the other within a sweep, the CTA tier (power-of-two
    // counters, then the bracket histogram), the warp tier's staged estimates
    // and the thread tier's per-warp counts (sizes: sweep_smem_bytes).
    extern __shared__ __align__(16) uint32_t s_dyn[];
    int* s_wbuf = (int*)s_dyn;
    uint32_t* s_whist = s_dyn + (blockDim.x >> 5) * kWCap;  // warp tier: window counts
    uint32_t* s_pool = s_whist + (blockDim.x >> 5) * kMedWin;
    __shared__ uint32_t s_cls[32];
    __shared__ uint32_t s_cnt[3 * 32];
    __shared__ uint32_t s_hub[4];
    __shared__ uint32_t s_wsum[32];
    __shared__ unsigned long long s_acc[kAccN];
    __shared__ long long s_b[12];
    __shared__ int s_int[2];
    __shared__ uint32_t s_u32;

    const Off* rp = (const Off*)a.row_ptr;
    SweepCtl* ctl = a.ctl;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const bool multi = gridDim.x > 1;
    bool tail = !multi;
    bool prev_tail = tail;
    unsigned my_epoch = 0;
    unsigned nbar = 0;
    unsigned long long tot[kAccN] = {};  // block 0, thread 0: run totals
    long long tail_sweeps = 0;
    long long s = a.first_sweep;
    if (tid == 0) {
        s_int[0] = 0;
        s_int[1] = 1;
        my_epoch = vload(&ctl->tail_epoch);
    }
    if (tid < kAccN) s_acc[tid] = 0;
    __syncthreads();

    const long long gtid = (long long)blockIdx.x * blockDim.x + tid;
    const long long gstride = (long long)gridDim.x * blockDim.x;
    // a6 inside the launch: every CTA copies its share of the final estimates
    auto write_out = [&]() {
        if (a.out)
            for (long long v = gtid; v < a.n; v += gstride)
                a.out[v] = (int)(est_load(a.est + (a.perm ? __ldg(a.perm + v) : (int)v)) & kEstMask);
    };
    // a2 inside the launch: estimates from the degrees, F_0 = every vertex
    if (a.est0) {
        for (long long v = gtid; v < a.n; v += gstride) a.est[v] = __ldg(a.est0 + v);
        for (long long w = gtid; w < a.words; w += gstride) {
            a.bitmap[0][w] = 0xffffffffu;
            a.bitmap[1][w] = 0u;
            a.bitmap[2][w] = 0u;
        }
        if (blockIdx.x == 0 && tid < kTiers) ctl->fcnt[0][tid] = a.init_cnt[tid];
        if (multi) {
            if (!grid_barrier(ctl, nbar, a.timeout_ns, &s_int[1])) return;
        } else {
            __syncthreads();
        }
    }

    for (;;) {
        const int cur = (int)(s % kSlots), nxt = (int)((s + 1) % kSlots);
        const int prv = (int)((s + kSlots - 1) % kSlots);
        if (tid == 0) {
            // all loads first (one round trip), then the bookkeeping
            const unsigned f0 = __ldcg(&ctl->fcnt[cur][0]), f1 = __ldcg(&ctl->fcnt[cur][1]);
            const unsigned f2 = __ldcg(&ctl->fcnt[cur][2]);
            const int st = __ldcg(&ctl->status);
            unsigned pv[kTiers] = {0u, 0u, 0u};
            unsigned long long av[kAccN] = {};
            if (s > 0)
                for (int q = 0; q < kTiers; q++) pv[q] = __ldcg(&ctl->fcnt[prv][q]);
            const bool book = blockIdx.x == 0 && s > a.first_sweep;
            if (book)
                for (int i = 0; i < kAccN; i++) av[i] = __ldcg(&ctl->acc[prv][i]);
            s_b[0] = f0;
            s_b[1] = f1;
            s_b[2] = f2;
            s_b[3] = st;
            for (int q = 0; q < kTiers; q++) s_b[6 + q] = pv[q];
            if (book) {  // statistics of sweep s-1
                for (int i = 0; i < kAccN; i++) {
                    tot[i] += av[i];
                    ctl->acc[prv][i] = 0;
                }
                if (s - 1 < a.max_trace) {
                    long long* tr = a.trace + (s - 1) * kTraceCols;
                    tr[kTrFrontier] = (long long)av[kAccEvaluated];
                    tr[kTrDegsum] = (long long)av[kAccDegsum];
                    tr[kTrUpdates] = (long long)av[kAccUpdates];
                    tr[kTrRead] = (long long)(av[kAccDegsum] - av[kAccSkipped]);
                    tr[kTrDec] = (long long)av[kAccDec];
                    tr[kTrDegW] = (long long)av[kAccDegW];
                    tr[kTrDegC] = (long long)av[kAccDegC];
                }
                if (prev_tail) tail_sweeps += 1;
            }
            // start time of sweep s (globaltimer, ns)
            if (blockIdx.x == 0 && s < a.max_trace) {
                long long* tr = a.trace + s * kTraceCols;
                tr[kTrStart] = (long long)gtime_ns();
                tr[kTrF0] = f0;
                tr[kTrF1] = f1;
                tr[kTrF2] = f2;
            }
            // slot of sweep s-2: free now, push target of sweep s+1
            if (blockIdx.x == 0) {
                const int old = (int)((s + 2) % kSlots);
                for (int q = 0; q < 4; q++) {
                    ctl->fcnt[old][q] = 0;
                    ctl->cursor[old][q] = 0;
                }
                ctl->ucnt[old] = 0;
            }
        }
        __syncthreads();
        const unsigned c0 = (unsigned)s_b[0], c1 = (unsigned)s_b[1], c2 = (unsigned)s_b[2];
        const long long total = (long long)c0 + c1 + c2;
        const int status = (int)s_b[3];
        const long long p0 = s_b[6], p1 = s_b[7], p2 = s_b[8];
        __syncthreads();

        // ---- end of the launch?
        const bool finished = total == 0;
        const bool capped = !finished && s >= a.max_sweeps;
        if (status != 0 || finished || capped || s >= a.stop_sweep) {
            if (tid == 0 && blockIdx.x == 0) {
                ctl->sweep = s;
                for (int i = 0; i < kAccN; i++) ctl->tot[i] += tot[i];
                ctl->tail_sweeps += tail_sweeps;
                if (finished) ctl->done = 1;
                if (capped) atomicCAS(&ctl->status, 0, (int)KCORE_ERR_NOT_CONVERGED);
            }
            if (tid == 0 && multi && tail) {  // release the waiting CTAs
                ctl->tail_exit = 1;
                __threadfence();
                atomicAdd(&ctl->tail_epoch, 1u);
            }
            if (finished || capped || status != 0) write_out();
            return;
        }

        // ---- single-CTA tail transitions
        // The tail is for frontiers that are small in work, not only in
        // vertices: no CTA-tier vertex and at most kTailMed warp-tier ones
        // (one CTA alone on a frontier of high-degree vertices would take
        // milliseconds while the other CTAs wait).
        const bool small = total <= a.tail_max && c1 <= (unsigned)kTailMed && c2 == 0;
        if (multi && !tail && small) {
            // Every CTA has read this sweep's counts before CTA 0 goes on alone.
            if (!grid_barrier(ctl, nbar, a.timeout_ns, &s_int[1])) return;
            if (blockIdx.x != 0) {
                if (tid == 0) {
                    const unsigned long long t0 = gtime_ns();
                    int ok = 1;
                    while (vload(&ctl->tail_epoch) <= my_epoch) {
                        if ((long long)(gtime_ns() - t0) > a.timeout_ns) {
                            atomicCAS(&ctl->status, 0, (int)KCORE_ERR_TIMEOUT);
                            ok = 0;
                            break;
                        }
                        __nanosleep(1000);
                    }
                    my_epoch += 1;
                    __threadfence();
                    s_int[1] = ok && vload(&ctl->tail_exit) == 0;
                    s_b[4] = vload(&ctl->resume_sweep);
                }
                __syncthreads();
                const bool resume = s_int[1] != 0;
                const long long rs = s_b[4];
                __syncthreads();
                if (!resume) {  // the single-CTA tail ended the run
                    write_out();
                    return;
                }
                s = rs;
                prev_tail = false;
                continue;
            }
            tail = true;
        } else if (multi && tail && (total > 4LL * a.tail_max || c1 > (unsigned)(4 * kTailMed) || c2 > 0)) {
            if (tid == 0) {  // hand the sweeps back to every CTA
                ctl->resume_sweep = s;
                ctl->tail_exit = 0;
                __threadfence();
                atomicAdd(&ctl->tail_epoch, 1u);
                my_epoch += 1;
            }
            tail = false;
        }

        const int p_cur = (int)(s % kParities), p_nxt = (int)((s + 1) % kParities);
        const int p_old = (int)((s + 2) % kParities);
        Sweep S;
        S.a = &a;
        S.cur = cur;
        S.nxt = nxt;
        S.lcur = (s == 0 && a.init_list) ? a.init_list : a.list[p_cur];
        S.lnxt = a.list[p_nxt];
        S.bmc = a.bitmap[p_cur];
        S.bmc_w = a.bitmap[p_cur];
        S.mark = a.refined && !a.sync_mode;
        S.bmn = a.bitmap[p_nxt];
        S.wbuf = s_wbuf + wid * kWCap;
        WarpQ Q = {{0u, 0u, 0u}};
        Acc acc = {0u, 0u, 0u, 0ull, 0ull, 0ull, 0ull, 0ull};
        const unsigned warps_all = (tail ? 1u : gridDim.x) * (unsigned)nwarps;
        const long long gthreads = tail ? blockDim.x : (long long)gridDim.x * blockDim.x;
        const long long gt = tail ? tid : (long long)blockIdx.x * blockDim.x + tid;

        // ---- clear the membership bits of F_{s-1}: every set bit of bitmap
        // p_old belongs to it, so zeroing the word of each member is enough
        if (s > 0) {
            uint32_t* bmo = a.bitmap[p_old];
            const long long prev_total = p0 + p1 + p2;
            if (prev_total >= a.words) {
                for (long long i = gt; i < a.words; i += gthreads) bmo[i] = 0u;
            } else {
                const int* lold = a.list[p_old];
                for (long long i = gt; i < prev_total; i += gthreads) {
                    const long long at = i < p0 ? a.tier_off[0] + i
                                       : i < p0 + p1 ? a.tier_off[1] + (i - p0)
                                                     : a.tier_off[2] + (i - p0 - p1);
                    bmo[list_load(lold + at) >> 5] = 0u;
                }
            }
        }

        // ---- phase A: evaluate F_s.  CTA tier first (the longest items).
        if (c2 > 0) {
            for (;;) {
                if (tid == 0) s_b[5] = (long long)atomicAdd(&ctl->cursor[cur][2], 1u);
                __syncthreads();
                const long long i = s_b[5];
                __syncthreads();
                if (i >= c2) break;
                const int u = list_load(S.lcur + a.tier_off[2] + i);
                hub_vertex<Off>(S, Q, rp, u, s_pool, s_cls, s_hub, s_wsum, &s_int[0], &s_u32, acc);
                __syncthreads();
            }
        }
        // warp tier: one warp per vertex, med_chunk vertices per grab (fewer
        // when the tier is small, so that every warp gets some)
        if (c1 > 0) {
            const unsigned wi = max(1u, min((unsigned)a.med_chunk, c1 / warps_all));
            // the grab's vertex ids, row bounds and estimates are loaded together,
            // one vertex per lane, before the first evaluation (only u writes
            // est[u], so the early read is its value when u is evaluated)
            run_tier(&ctl->cursor[cur][1], c1, wi, [&](unsigned i0, unsigned i1) {
                for (unsigned base = i0; base < i1; base += 32u) {
                    const unsigned j = base + (unsigned)lane;
                    int u = 0;
                    long long rb = 0, re = 0;
                    uint32_t w = 0;
                    if (j < i1) {
                        u = list_load(S.lcur + a.tier_off[1] + j);
                        rb = (long long)rp[u];
                        re = (long long)rp[u + 1];
                        w = est_load(a.est + u);
                    }
                    const unsigned cnt = min(32u, i1 - base);
                    for (unsigned t = 0; t < cnt; t++) {
                        const int ut = __shfl_sync(kFull, u, (int)t);
                        const long long bt = __shfl_sync(kFull, rb, (int)t);
                        const int dt = (int)(__shfl_sync(kFull, re, (int)t) - bt);
                        const uint32_t wt = __shfl_sync(kFull, w, (int)t);
                        if (dt <= 32 * kMedR) med_vertex<kMedR>(S, Q, ut, bt, dt, wt, acc);
                        else med_big_vertex(S, Q, ut, bt, dt, wt, s_pool + wid * kMedSlice,
                                            s_whist + wid * kMedWin, acc);
                    }
                }
            });
        }
        // thread tier: one thread per vertex, 32 * low_chunk vertices per grab.
        // A large tier is walked by vertex id (dense): membership comes from the
        // bitmap word, and rows, estimates and adjacency are read coalesced.
        if (c0 > 0) {
            const bool dense = (long long)c0 * 2 >= a.n;
            const unsigned items = dense ? (unsigned)a.n : c0;
            const unsigned wi = 32u * max(1u, min((unsigned)a.low_chunk, items / (32u * warps_all)));
            uint32_t* hist = s_pool + wid * kMedSlice;
            if (dense) {
                run_tier(&ctl->cursor[cur][3], items, wi, [&](unsigned i0, unsigned i1) {
                    for (unsigned base = i0; base < i1; base += 32u) {
                        const unsigned i = base + (unsigned)lane;
                        low_warp<Off, T / 4, true>(S, Q, rp, i < i1, (int)i, S.bmc + (base >> 5), hist, acc);
                    }
                });
            } else {
                run_tier(&ctl->cursor[cur][0], items, wi, [&](unsigned i0, unsigned i1) {
                    for (unsigned base = i0; base < i1; base += 32u) {
                        const unsigned i = base + (unsigned)lane;
                        const bool valid = i < i1;
                        const int u = valid ? list_load(S.lcur + a.tier_off[0] + i) : 0;
                        low_warp<Off, T / 4, false>(S, Q, rp, valid, u, nullptr, hist, acc);
                    }
                });
            }
        }

        // ---- synchronous mode: write the recorded updates after a barrier
        if (a.sync_mode) {
            if (tail) block_barrier();
            else if (!grid_barrier(ctl, nbar, a.timeout_ns, &s_int[1])) return;
            const unsigned nu = vload(&ctl->ucnt[cur]);
            for (long long i = gt; i < nu; i += gthreads) {
                const int u = a.upd_list[i];
                const uint32_t old = est_load(a.est + u);
                a.est[u] = (old & ~kEstMask) | (uint32_t)a.upd_val[i];
                a.upd_val[i] = (int)(old & kEstMask);
            }
            if (a.refined) {
                if (tail) block_barrier();
                else if (!grid_barrier(ctl, nbar, a.timeout_ns, &s_int[1])) return;
                const long long gw = tail ? nwarps : (long long)gridDim.x * nwarps;
                const long long wi = tail ? wid : (long long)blockIdx.x * nwarps + wid;
                for (long long i = wi; i < nu; i += gw) {
                    const int u = a.upd_list[i];
                    const int old_u = a.upd_val[i];
                    const int new_u = (int)(est_load(a.est + u) & kEstMask);
                    const long long b = (long long)rp[u];
                    const long long d = (long long)rp[u + 1] - b;
                    for (long long j0 = 0; j0 < d; j0 += 32) {
                        const long long j = j0 + lane;
                        bool want = false;
                        int v = 0;
                        uint32_t tier = 0;
                        if (j < d) {
                            v = __ldg(a.col + b + j);
                            const uint32_t xw = est_load(a.est + v);
                            const int x = (int)(xw & kEstMask);
                            want = new_u < x && x <= old_u;
                            tier = xw >> kEstBits;
                        }
                        if (__any_sync(kFull, want)) warp_push(S, Q, want, v, tier, acc);
                    }
                }
            }
        }
        cta_flush_all(S, Q, s_cnt);

        // ---- per-sweep statistics
        {
            unsigned long long v4[kAccN] = {acc.evaluated, acc.degsum, acc.updates, acc.pushes,
                                            acc.skipped,   acc.dec,    acc.deg_w,   acc.deg_c};
#pragma unroll
            for (int i = 0; i < kAccN; i++) {
                unsigned long long x = v4[i];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFull, x, o);
                if (lane == 0 && x) atomicAdd(&s_acc[i], x);
            }
        }
        __syncthreads();
        if (tid < kAccN) {
            if (s_acc[tid]) atomicAdd(&ctl->acc[cur][tid], s_acc[tid]);
            s_acc[tid] = 0;
        }

        // ---- end of sweep
        prev_tail = tail;
        if (tail) block_barrier();
        else if (!grid_barrier(ctl, nbar, a.timeout_ns, &s_int[1])) return;
        s++;
    }
}

__global__ void k_ctl_init(SweepCtl* ctl, unsigned c0, unsigned c1, unsigned c2) {
    ctl->fcnt[0][0] = c0;
    ctl->fcnt[0][1] = c1;
    ctl->fcnt[0][2] = c2;
}

const void* pick_kernel(int t_lo, int off64) {
    (void)t_lo;
    return off64 ? (const void*)k_sweep<long long, 16> : (const void*)k_sweep<int, 16>;
}

// Dynamic shared memory of one CTA: push buffers, then the pool (the larger
// of the CTA tier's counters with its window histogram, and every warp's
// kMedBig 16-bit estimates).
size_t sweep_smem_bytes(int block) {
    const size_t nw = (size_t)block / 32;
    const size_t pool = std::max<size_t>({(size_t)kLogWords * block + kHubBins, nw * kMedSlice});
    static_assert((16 / 4) * 32 <= kMedSlice, "thread tier counts exceed a warp's slice");
    return sizeof(uint32_t) * (nw * (kWCap + kMedWin) + pool);
}

cudaError_t prepare(const void* fn, int block, int* per_sm) {
    const size_t smem = sweep_smem_bytes(block);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, block, smem);
}

}  // namespace

cudaError_t sweep_max_grid(int block, int t_lo, int t_hi, int off64, int* grid) {
    (void)t_hi;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = prepare(pick_kernel(t_lo, off64), block, &per_sm);
    if (e != cudaSuccess) return e;
    *grid = sms * per_sm;
    return cudaSuccess;
}

cudaError_t launch_sweep(const SweepArgs& a, int block, int grid_req, int ctas_per_sm,
                         cudaStream_t st, int* grid_used) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const void* fn = pick_kernel(a.t_lo, a.off64);
    e = prepare(fn, block, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    int grid = sms * per_sm;
    if (grid_req > 0 && grid_req < grid) grid = grid_req;
    if (grid < 1) grid = 1;
    *grid_used = grid;
    void* args[] = {(void*)&a};
    count_launch();
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, sweep_smem_bytes(block), st);
}

// Warm start (dynamic maintenance): est[v] = tier bits | min(start[v], deg v).
// With a frontier list, F_0 is that list plus every vertex the cap lowered
// and its neighbours (a lowered estimate is a change its neighbours must
// see), deduplicated by the F_0 bitmap and appended to list0 by tier; an id
// out of range sets the status to KCORE_ERR_INVALID.  Without a list every
// vertex is active and the caller sets up F_0.
__device__ __forceinline__ void warm_activate(int v, const uint32_t* est0, uint32_t* bm0, int* list0,
                                              const long long* tier_off, SweepCtl* ctl) {
    const uint32_t bit = 1u << (v & 31);
    if (atomicOr(bm0 + (v >> 5), bit) & bit) return;
    const int t = (int)(__ldg(est0 + v) >> kEstBits);
    const unsigned pos = atomicAdd(&ctl->fcnt[0][t], 1u);
    list0[tier_off[t] + pos] = v;
}

template <typename Off>
__global__ void k_warm_init(const Off* __restrict__ rp, const int* __restrict__ col, long long n,
                            const uint32_t* __restrict__ est0, const int* __restrict__ start,
                            uint32_t* __restrict__ est, const int* __restrict__ frontier, long long nf,
                            uint32_t* bm0, int* list0, long long off0, long long off1, long long off2,
                            SweepCtl* ctl) {
    const long long tier_off[kTiers] = {off0, off1, off2};
    const long long total = n > nf ? n : nf;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        if (frontier && i < nf) {
            const int v = frontier[i];
            if (v < 0 || v >= n) atomicCAS(&ctl->status, 0, (int)KCORE_ERR_INVALID);
            else warm_activate(v, est0, bm0, list0, tier_off, ctl);
        }
        if (i < n) {
            const uint32_t w0 = __ldg(est0 + i);
            const uint32_t d = w0 & kEstMask;
            const long long x = (long long)start[i];
            const uint32_t e = x < 0 ? 0u : (x < (long long)d ? (uint32_t)x : d);
            est[i] = (w0 & ~kEstMask) | e;
            if (frontier && x > (long long)d) {  // lowered by the cap: v and its neighbours
                warm_activate((int)i, est0, bm0, list0, tier_off, ctl);
                for (long long j = (long long)rp[i]; j < (long long)rp[i + 1]; j++)
                    warm_activate(__ldg(col + j), est0, bm0, list0, tier_off, ctl);
            }
        }
    }
}

cudaError_t launch_warm_init(const SweepArgs& a, const void* row_ptr, const uint32_t* est0,
                             const int* start, const int* frontier, long long nf, cudaStream_t st) {
    const long long items = std::max<long long>({(long long)a.n, nf, 1LL});
    const int g = (int)std::min<long long>((items + 255) / 256, (long long)sm_count() * 32);
    if (a.off64)
        k_warm_init<<<g, 256, 0, st>>>((const long long*)row_ptr, a.col, a.n, est0, start, a.est,
                                      frontier, nf, a.bitmap[0], a.list[0], a.tier_off[0],
                                      a.tier_off[1], a.tier_off[2], a.ctl);
    else
        k_warm_init<<<g, 256, 0, st>>>((const int*)row_ptr, a.col, a.n, est0, start, a.est, frontier,
                                      nf, a.bitmap[0], a.list[0], a.tier_off[0], a.tier_off[1],
                                      a.tier_off[2], a.ctl);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_ctl_init(SweepCtl* ctl, const long long tier_cnt[kTiers], cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(SweepCtl), st);
    if (e != cudaSuccess) return e;
    k_ctl_init<<<1, 1, 0, st>>>(ctl, (unsigned)tier_cnt[0], (unsigned)tier_cnt[1],
                                (unsigned)tier_cnt[2]);
    count_launch();
    return cudaGetLastError();
}


}  // namespace kc
