// Persistent sweep kernel: the local coreness iteration of Alg. 1 on the GPU.
//
// One cooperative launch runs every sweep.  Sweep s evaluates the vertices of
// frontier F_s: each computes the h-index of its neighbours' estimates capped
// at its own estimate (computeCoreness of Alg. 1, read as Montresor's
// computeIndex).  If that is lower, the estimate is lowered and every
// neighbour v whose estimate is above the new value is pushed into F_{s+1}
// (selective sending, Sec. III-B).  Estimates only decrease, so they are
// updated in place while other vertices of the same sweep read them
// (asynchronous mode); a stale read only over-activates, never misses a needed
// re-evaluation.  The run ends when a frontier is empty (the `changed` flag of
// Alg. 2/3 becomes the frontier count).
//
// Degree tiers (est word bits 30-31): d <= t_lo one thread per vertex with a
// register histogram; d <= t_hi one warp per vertex, counts by warp reduction;
// larger degrees one CTA per vertex with a shared-memory histogram.  Work is
// handed out by atomic cursors (the dynamic chunking of Alg. 2), hubs first.
// Frontier membership is a bitmap per sweep parity (no vertex twice in a
// list); pushes are warp-aggregated.
//
// Sweeps are separated by a grid barrier; once a frontier is at most tail_max
// vertices, CTA 0 continues alone with block barriers (the GPU analogue of
// FastK's switch to sequential processing, Sec. IV) and the other CTAs wait,
// to rejoin if the frontier grows again.  Every wait is bounded by timeout_ns
// (globaltimer) and reports KCORE_ERR_TIMEOUT instead of hanging.
//
// Synchronous mode (KCORE_SYNC_MODE) follows Alg. 3: phase A computes new
// values against the unchanged estimates and records them; after a barrier
// phase B writes them; with the refined rule (Sec. IV, Further
// Optimizations) a third phase decides activations against the written
// values: new_u < est(v) <= old_u.
#include <cuda_runtime.h>

#include <algorithm>

#include "kc_common.cuh"

namespace kc {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxBlock = 512;

__device__ __forceinline__ unsigned long long gtime_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned vload(const unsigned* p) { return *(const volatile unsigned*)p; }
__device__ __forceinline__ int vload(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ long long vload(const long long* p) { return *(const volatile long long*)p; }
__device__ __forceinline__ unsigned long long vload(const unsigned long long* p) {
    return *(const volatile unsigned long long*)p;
}

// Estimates are read through L2 (ld.global.cg): another SM may have lowered
// them, and an L1 copy from an earlier sweep would be stale.
__device__ __forceinline__ uint32_t est_load(const uint32_t* p) { return __ldcg(p); }
__device__ __forceinline__ int list_load(const int* p) { return __ldcg(p); }

struct Sweep {
    const SweepArgs* a;
    int cur, nxt;
    const int* lcur;
    int* lnxt;
    uint32_t* bmc;
    uint32_t* bmn;
};

// All 32 lanes call this.  A lane with `want` pushes v (tier `tier`) into the
// next frontier unless it is already there.
__device__ __forceinline__ void warp_push(const Sweep& S, bool want, int v, uint32_t tier,
                                          unsigned long long& pushes) {
    const int lane = threadIdx.x & 31;
    bool fresh = false;
    if (want) {
        const uint32_t bit = 1u << (v & 31);
        uint32_t* word = S.bmn + (v >> 5);
        if ((__ldcg(word) & bit) == 0) fresh = (atomicOr(word, bit) & bit) == 0;
    }
#pragma unroll
    for (int q = 0; q < kTiers; q++) {
        const unsigned m = __ballot_sync(kFull, fresh && tier == (uint32_t)q);
        if (m) {
            const int leader = __ffs(m) - 1;
            unsigned base = 0;
            if (lane == leader) base = atomicAdd(&S.a->ctl->fcnt[S.nxt][q], (unsigned)__popc(m));
            base = __shfl_sync(kFull, base, leader);
            if (fresh && tier == (uint32_t)q)
                S.lnxt[S.a->tier_off[q] + base + __popc(m & ((1u << lane) - 1u))] = v;
            if (lane == 0) pushes += (unsigned)__popc(m);
        }
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

__device__ __forceinline__ void clear_member(const Sweep& S, int u) {
    atomicAnd(S.bmc + (u >> 5), ~(1u << (u & 31)));
}

// ---------------------------------------------------------------- thread tier
// Register histogram: c[i] packs the counts #{x >= t} for the four thresholds
// t = 4i+1 .. 4i+4, one byte each (x = min(neighbour estimate, k)).  The
// capped h-index is the number of thresholds t with count_t >= t, because that
// predicate holds exactly for t <= h.
template <typename Off, int TW>
__device__ __forceinline__ void low_vertex(const Sweep& S, const Off* __restrict__ rp, bool valid,
                                           int u, unsigned long long acc[kAccN]) {
    const SweepArgs& a = *S.a;
    long long b = 0;
    int d = 0, k = 0;
    uint32_t w = 0;
    if (valid) {
        b = (long long)rp[u];
        d = (int)((long long)rp[u + 1] - b);
        w = est_load(a.est + u);
        k = (int)(w & kEstMask);
        clear_member(S, u);
        acc[kAccEvaluated] += 1;
        acc[kAccDegsum] += (unsigned)d;
    }
    const bool work = valid && k > 0;
    uint32_t c[TW];
#pragma unroll
    for (int i = 0; i < TW; i++) c[i] = 0;
    const int dmax = __reduce_max_sync(kFull, work ? d : 0);
    for (int j = 0; j < dmax; j++) {
        if (work && j < d) {
            const int v = __ldg(a.col + b + j);
            const int x = (int)(est_load(a.est + v) & kEstMask);
            const int y = x < k ? x : k;
#pragma unroll
            for (int i = 0; i < TW; i++) {
                const int q = y - 4 * i;
                c[i] += q >= 4 ? 0x01010101u : (q <= 0 ? 0u : (0x01010101u & ((1u << (8 * q)) - 1u)));
            }
        }
    }
    int h = 0;
#pragma unroll
    for (int i = 0; i < TW; i++) {
        const uint32_t thr = (uint32_t)(4 * i + 1) | ((uint32_t)(4 * i + 2) << 8) |
                             ((uint32_t)(4 * i + 3) << 16) | ((uint32_t)(4 * i + 4) << 24);
        h += __popc(__vcmpgeu4(c[i], thr) & 0x01010101u);
    }
    const bool changed = work && h < k;
    if (changed) acc[kAccUpdates] += 1;
    warp_update(S, changed, u, w, h);
    if (a.refined) return;  // refined activation runs after the update phase
    const int pmax = __reduce_max_sync(kFull, changed ? d : 0);
    for (int j = 0; j < pmax; j++) {
        bool want = false;
        int v = 0;
        uint32_t tier = 0;
        if (changed && j < d) {
            v = __ldg(a.col + b + j);
            const uint32_t xw = est_load(a.est + v);
            want = (uint32_t)h < (xw & kEstMask);
            tier = xw >> kEstBits;
        }
        warp_push(S, want, v, tier, acc[kAccPushes]);
    }
}

// ---------------------------------------------------------------- warp tier
// One warp per vertex, up to 32*R neighbours held in registers; the count of
// neighbours >= t comes from a warp reduction, and h by bisection on t after
// the no-change test t = k.
template <typename Off, int R>
__device__ __forceinline__ void med_vertex(const Sweep& S, const Off* __restrict__ rp, int u,
                                           unsigned long long acc[kAccN]) {
    const SweepArgs& a = *S.a;
    const int lane = threadIdx.x & 31;
    const long long b = (long long)rp[u];
    const int d = (int)((long long)rp[u + 1] - b);
    const uint32_t w = est_load(a.est + u);
    const int k = (int)(w & kEstMask);
    if (lane == 0) {
        clear_member(S, u);
        acc[kAccEvaluated] += 1;
        acc[kAccDegsum] += (unsigned)d;
    }
    if (k == 0) return;
    uint32_t xw[R];
    int vs[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int j = r * 32 + lane;
        vs[r] = 0;
        xw[r] = 0;
        if (j < d) {
            vs[r] = __ldg(a.col + b + j);
            xw[r] = est_load(a.est + vs[r]);
        }
    }
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
    if (h >= k) return;
    if (lane == 0) acc[kAccUpdates] += 1;
    warp_update(S, lane == 0, u, w, h);
    if (a.refined) return;
#pragma unroll
    for (int r = 0; r < R; r++) {
        if (r * 32 >= d) break;
        const bool want = (r * 32 + lane < d) && (uint32_t)h < (xw[r] & kEstMask);
        warp_push(S, want, vs[r], xw[r] >> kEstBits, acc[kAccPushes]);
    }
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

// Over buckets i in [0, nb) of s_hist, with above = number of values beyond
// the last bucket: counts how many i satisfy
// above + #{values in buckets >= i} >= base + i * width.  The predicate is
// monotone (true for a prefix of i), so the result minus one is the last i
// where it holds.  If want_after >= 0, *after gets #{values in buckets >=
// want_after} + above.
__device__ __forceinline__ int hub_count_true(const uint32_t* s_hist, int nb, uint32_t above, long long base,
                              long long width, int want_after, uint32_t* after, uint32_t* wsum,
                              int* s_int) {
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

template <typename Off>
__device__ __forceinline__ void hub_vertex(const Sweep& S, const Off* __restrict__ rp, int u, uint32_t* s_hist,
                           uint32_t* wsum, int* s_int, uint32_t* s_u32,
                           unsigned long long acc[kAccN]) {
    const SweepArgs& a = *S.a;
    const int T = blockDim.x, tid = threadIdx.x;
    const long long b = (long long)rp[u];
    const long long d = (long long)rp[u + 1] - b;
    const uint32_t w = est_load(a.est + u);
    const int k = (int)(w & kEstMask);
    if (tid == 0) {
        clear_member(S, u);
        acc[kAccEvaluated] += 1;
        acc[kAccDegsum] += (unsigned long long)d;
    }
    if (k == 0) return;
    // pass 1: histogram of min(x, k) >> shift, with 2^shift the smallest power
    // of two that brings the k+1 possible values into kHubBins buckets
    int shift = 0;
    while ((k >> shift) >= kHubBins) shift++;
    const long long width = 1LL << shift;
    const int nb = (k >> shift) + 1;
    for (int i = tid; i < nb; i += T) s_hist[i] = 0;
    __syncthreads();
    for (long long j = tid; j < d; j += T) {
        const int v = __ldg(a.col + b + j);
        int x = (int)(est_load(a.est + v) & kEstMask);
        x = x < k ? x : k;
        atomicAdd(&s_hist[x >> shift], 1u);
    }
    __syncthreads();
    const int ntrue = hub_count_true(s_hist, nb, 0u, 0, width, -1, s_u32, wsum, s_int);
    const int istar = ntrue - 1;
    int h;
    if (width == 1) {
        h = istar;
    } else {
        // above = #{x >= (istar+1) * width}
        if (tid == 0) *s_u32 = 0;
        __syncthreads();
        hub_count_true(s_hist, nb, 0u, 0, width, istar + 1, s_u32, wsum, s_int);
        const uint32_t above = *s_u32;
        __syncthreads();
        const long long lo = (long long)istar * width;
        const long long hi = min(lo + width - 1, (long long)k);
        const int wn = (int)(hi - lo + 1);
        for (int i = tid; i < wn; i += T) s_hist[i] = 0;
        __syncthreads();
        for (long long j = tid; j < d; j += T) {
            const int v = __ldg(a.col + b + j);
            int x = (int)(est_load(a.est + v) & kEstMask);
            x = x < k ? x : k;
            if (x >= lo && x <= hi) atomicAdd(&s_hist[x - lo], 1u);
        }
        __syncthreads();
        const int nt2 = hub_count_true(s_hist, wn, above, lo, 1, -1, s_u32, wsum, s_int);
        h = (int)(lo + nt2 - 1);
    }
    __syncthreads();
    if (h >= k) return;
    if (tid == 0) acc[kAccUpdates] += 1;
    if ((tid >> 5) == 0) warp_update(S, tid == 0, u, w, h);
    if (a.refined) return;
    for (long long j0 = 0; j0 < d; j0 += T) {
        const long long j = j0 + tid;
        bool want = false;
        int v = 0;
        uint32_t tier = 0;
        if (j < d) {
            v = __ldg(a.col + b + j);
            const uint32_t xw = est_load(a.est + v);
            want = (uint32_t)h < (xw & kEstMask);
            tier = xw >> kEstBits;
        }
        warp_push(S, want, v, tier, acc[kAccPushes]);
    }
}

// ---------------------------------------------------------------- barriers
// Grid barrier (all CTAs are co-resident: cooperative launch).  Returns false
// if the wait ran past the budget; the status word then says TIMEOUT.
__device__ bool grid_barrier(SweepCtl* ctl, long long timeout_ns, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned gen = vload(&ctl->bar_gen);
        __threadfence();
        const unsigned arrived = atomicAdd(&ctl->bar_count, 1u) + 1u;
        if (arrived == gridDim.x) {
            atomicExch(&ctl->bar_count, 0u);
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        } else {
            const unsigned long long t0 = gtime_ns();
            while (vload(&ctl->bar_gen) == gen) {
                if ((long long)(gtime_ns() - t0) > timeout_ns) {
                    atomicCAS(&ctl->status, 0, (int)KCORE_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

__device__ __forceinline__ void block_barrier() {
    __threadfence();
    __syncthreads();
}

// ---------------------------------------------------------------- kernel
template <typename Off, int TW, int R>
__global__ void __launch_bounds__(kMaxBlock, 1) k_sweep(const SweepArgs a) {
    __shared__ uint32_t s_hist[kHubBins];
    __shared__ uint32_t s_wsum[32];
    __shared__ unsigned long long s_acc[kAccN];
    __shared__ long long s_b[6];
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
    long long s = a.first_sweep;
    if (tid == 0) {
        s_int[0] = 0;
        s_int[1] = 1;
        my_epoch = vload(&ctl->tail_epoch);
    }
    if (tid < kAccN) s_acc[tid] = 0;
    __syncthreads();

    for (;;) {
        const int cur = (int)(s % kSlots), nxt = (int)((s + 1) % kSlots);
        if (tid == 0) {
            s_b[0] = vload(&ctl->fcnt[cur][0]);
            s_b[1] = vload(&ctl->fcnt[cur][1]);
            s_b[2] = vload(&ctl->fcnt[cur][2]);
            s_b[3] = vload(&ctl->status);
            // bookkeeping of sweep s-1 and clearing of its slot
            if (blockIdx.x == 0 && s > a.first_sweep) {
                const int ps = (int)((s - 1) % kSlots);
                unsigned long long v[kAccN];
                for (int i = 0; i < kAccN; i++) {
                    v[i] = vload(&ctl->acc[ps][i]);
                    ctl->tot[i] += v[i];
                    ctl->acc[ps][i] = 0;
                }
                if (s - 1 < a.max_trace) {
                    a.trace[(s - 1) * 3 + 0] = (long long)v[kAccEvaluated];
                    a.trace[(s - 1) * 3 + 1] = (long long)v[kAccDegsum];
                    a.trace[(s - 1) * 3 + 2] = (long long)v[kAccUpdates];
                }
                if (prev_tail) ctl->tail_sweeps += 1;
                for (int q = 0; q < 4; q++) {
                    ctl->fcnt[ps][q] = 0;
                    ctl->cursor[ps][q] = 0;
                }
                ctl->ucnt[ps] = 0;
            }
        }
        __syncthreads();
        const unsigned c0 = (unsigned)s_b[0], c1 = (unsigned)s_b[1], c2 = (unsigned)s_b[2];
        const long long total = (long long)c0 + c1 + c2;
        const int status = (int)s_b[3];
        __syncthreads();

        // ---- end of the launch?
        const bool finished = total == 0;
        const bool capped = !finished && s >= a.max_sweeps;
        if (status != 0 || finished || capped || s >= a.stop_sweep) {
            if (tid == 0 && blockIdx.x == 0) {
                ctl->sweep = s;
                if (finished) ctl->done = 1;
                if (capped) atomicCAS(&ctl->status, 0, (int)KCORE_ERR_NOT_CONVERGED);
            }
            if (tid == 0 && multi && tail) {  // release the waiting CTAs
                ctl->tail_exit = 1;
                __threadfence();
                atomicAdd(&ctl->tail_epoch, 1u);
            }
            return;
        }

        // ---- single-CTA tail transitions
        if (multi && !tail && total <= a.tail_max) {
            // Every CTA has read this sweep's counts before CTA 0 goes on alone
            // (it clears this slot at the start of the next sweep).
            if (!grid_barrier(ctl, a.timeout_ns, &s_int[1])) return;
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
                if (!resume) return;
                s = rs;
                prev_tail = false;
                continue;
            }
            tail = true;
        } else if (multi && tail && total > 4LL * a.tail_max) {
            if (tid == 0) {  // hand the sweeps back to every CTA
                ctl->resume_sweep = s;
                ctl->tail_exit = 0;
                __threadfence();
                atomicAdd(&ctl->tail_epoch, 1u);
                my_epoch += 1;
            }
            tail = false;
        }

        // ---- phase A: evaluate F_s
        Sweep S;
        S.a = &a;
        S.cur = cur;
        S.nxt = nxt;
        S.lcur = (s == 0 && a.init_list) ? a.init_list : a.list[s & 1];
        S.lnxt = a.list[(s + 1) & 1];
        S.bmc = a.bitmap[s & 1];
        S.bmn = a.bitmap[(s + 1) & 1];
        unsigned long long acc[kAccN] = {0, 0, 0, 0};

        // CTA tier (hubs first: the longest items)
        for (;;) {
            if (tid == 0) s_b[5] = (long long)atomicAdd(&ctl->cursor[cur][2], 1u);
            __syncthreads();
            const long long i = s_b[5];
            __syncthreads();
            if (i >= c2) break;
            const int u = list_load(S.lcur + a.tier_off[2] + i);
            hub_vertex<Off>(S, rp, u, s_hist, s_wsum, &s_int[0], &s_u32, acc);
            __syncthreads();
        }
        // warp tier
        for (;;) {
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(&ctl->cursor[cur][1], (unsigned)a.med_chunk);
            base = __shfl_sync(kFull, base, 0);
            if (base >= c1) break;
            const unsigned end = min(c1, base + (unsigned)a.med_chunk);
            for (unsigned i = base; i < end; i++) {
                const int u = list_load(S.lcur + a.tier_off[1] + i);
                med_vertex<Off, R>(S, rp, u, acc);
            }
        }
        // thread tier
        for (;;) {
            unsigned base = 0;
            const unsigned step = 32u * (unsigned)a.low_chunk;
            if (lane == 0) base = atomicAdd(&ctl->cursor[cur][0], step);
            base = __shfl_sync(kFull, base, 0);
            if (base >= c0) break;
            for (int r = 0; r < a.low_chunk; r++) {
                const unsigned i = base + (unsigned)r * 32u + (unsigned)lane;
                const bool valid = i < c0;
                const int u = valid ? list_load(S.lcur + a.tier_off[0] + i) : 0;
                low_vertex<Off, TW>(S, rp, valid, u, acc);
                if (base + (unsigned)(r + 1) * 32u >= c0) break;
            }
        }

        // ---- synchronous mode: write the recorded updates after a barrier
        if (a.sync_mode) {
            if (tail) block_barrier();
            else if (!grid_barrier(ctl, a.timeout_ns, &s_int[1])) return;
            const unsigned nu = vload(&ctl->ucnt[cur]);
            const long long gthreads = tail ? blockDim.x : (long long)gridDim.x * blockDim.x;
            const long long gt = tail ? tid : (long long)blockIdx.x * blockDim.x + tid;
            for (long long i = gt; i < nu; i += gthreads) {
                const int u = a.upd_list[i];
                const uint32_t old = est_load(a.est + u);
                a.est[u] = (old & ~kEstMask) | (uint32_t)a.upd_val[i];
                a.upd_val[i] = (int)(old & kEstMask);
            }
            if (a.refined) {
                if (tail) block_barrier();
                else if (!grid_barrier(ctl, a.timeout_ns, &s_int[1])) return;
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
                        warp_push(S, want, v, tier, acc[kAccPushes]);
                    }
                }
            }
        }

        // ---- per-sweep statistics
#pragma unroll
        for (int i = 0; i < kAccN; i++) {
            unsigned long long x = acc[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFull, x, o);
            if (lane == 0 && x) atomicAdd(&s_acc[i], x);
        }
        __syncthreads();
        if (tid < kAccN) {
            if (s_acc[tid]) atomicAdd(&ctl->acc[cur][tid], s_acc[tid]);
            s_acc[tid] = 0;
        }

        // ---- end of sweep
        prev_tail = tail;
        if (tail) block_barrier();
        else if (!grid_barrier(ctl, a.timeout_ns, &s_int[1])) return;
        s++;
    }
}

__global__ void k_ctl_init(SweepCtl* ctl, unsigned c0, unsigned c1, unsigned c2) {
    ctl->fcnt[0][0] = c0;
    ctl->fcnt[0][1] = c1;
    ctl->fcnt[0][2] = c2;
}

__global__ void k_output(const uint32_t* __restrict__ est, int* __restrict__ out, long long n) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x)
        out[v] = (int)(__ldcg(est + v) & kEstMask);
}

template <typename Off, int TW>
const void* pick_kernel_tw() {
    return (const void*)k_sweep<Off, TW, 16>;
}

const void* pick_kernel(int t_lo, int off64) {
    if (off64) {
        if (t_lo <= 8) return pick_kernel_tw<long long, 2>();
        if (t_lo <= 16) return pick_kernel_tw<long long, 4>();
        return pick_kernel_tw<long long, 8>();
    }
    if (t_lo <= 8) return pick_kernel_tw<int, 2>();
    if (t_lo <= 16) return pick_kernel_tw<int, 4>();
    return pick_kernel_tw<int, 8>();
}

}  // namespace

cudaError_t sweep_max_grid(int block, int t_lo, int t_hi, int off64, int* grid) {
    (void)t_hi;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pick_kernel(t_lo, off64), block, 0);
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
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    int grid = sms * per_sm;
    if (grid_req > 0 && grid_req < grid) grid = grid_req;
    if (grid < 1) grid = 1;
    *grid_used = grid;
    void* args[] = {(void*)&a};
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, 0, st);
}

cudaError_t launch_ctl_init(SweepCtl* ctl, const long long tier_cnt[kTiers], cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(SweepCtl), st);
    if (e != cudaSuccess) return e;
    k_ctl_init<<<1, 1, 0, st>>>(ctl, (unsigned)tier_cnt[0], (unsigned)tier_cnt[1],
                                (unsigned)tier_cnt[2]);
    return cudaGetLastError();
}

cudaError_t launch_output(const uint32_t* est, int* out, long long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int g = (int)std::min<long long>((n + 255) / 256, 152LL * 32);
    k_output<<<g, 256, 0, st>>>(est, out, n);
    return cudaGetLastError();
}

}  // namespace kc
