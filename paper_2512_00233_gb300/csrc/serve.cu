// Batch engine: continuous batching of many graphs in one device arena.
//
// The arena is one graph over NV vertex slots and NE entries (int64 row_ptr,
// int32 col_idx, estimates, the three frontier lists with a region per tier,
// the three membership bitmaps, and the slot of every vertex).  Each admitted
// graph owns a vertex range and an entry range; the persistent sweep kernel
// of the single-graph path runs over the whole arena, a chunk of sweeps per
// launch, so every resident graph advances in the same launch.
//
// Between chunks the engine thread
//   1. retires graphs with no vertex left in the frontier: their estimates are
//      the coreness (the iteration's fixed point), copied out, ranges freed;
//   2. admits queued graphs that fit: the whole admission batch is cleaned as
//      one disjoint union (one device CSR-cleaning call), placed into a
//      contiguous vertex range, its estimates set to the degrees and every
//      vertex pushed into the current frontier.  Each graph is followed by a
//      spare vertex of its own (isolated, never in a frontier), whose row_ptr
//      slot holds the end of the graph's last row: the graph owns that slot,
//      so placing another graph into a neighbouring freed range can never
//      move the end of a resident graph's last row.
// A graph admitted while others run joins at the next chunk.  The coreness is
// unique and the iteration reaches it from any schedule, so each result is
// the same alone or in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kc_common.cuh"
#include "ranges.h"

namespace kc {

kcore_status fail(kcore_status s, const std::string& msg);
kcore_status cuda_status(cudaError_t e, const char* what);
void set_error(const std::string& msg);
kcore_status normalize_options(const kcore_options* in, kcore_options* out);
cudaError_t launch_ctl_init(SweepCtl* ctl, const long long tier_cnt[kTiers], cudaStream_t st);

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    uint64_t ticket = 0;
    int64_t n = 0, nnz = 0;
    // raw samples (a CSR input is expanded at submit): sources at ps, targets
    // at pd; either the two halves of one 2*nnz-word range of the page-locked
    // staging pool (h_off >= 0) or the vectors
    int32_t *ps = nullptr, *pd = nullptr;
    long long h_off = -1;
    std::vector<int32_t> src, dst;
    // state
    enum { QUEUED, RESIDENT, DONE } state = QUEUED;
    bool cancelled = false;
    kcore_status status = KCORE_OK;
    // the result as raw estimates (flag bits cleared when read): n words of the
    // staging pool (r_off >= 0) or the vector
    const uint32_t* res = nullptr;
    long long r_off = -1;
    std::vector<uint32_t> result;
    double t_submit = 0, t_admit = 0, t_done = 0;
    long long admit_launch = -1, retire_launch = -1, resident_at_admit = 0;
    // placement
    int slot = -1;
    long long v0 = 0, vlen = 0, e0 = 0, elen = 0;
};

__device__ __forceinline__ int slot_index(const long long* starts, int count, long long v) {
    int lo = 0, hi = count - 1;  // last start <= v
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (starts[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Places the cleaned union (vertices [0, nu), its own row_ptr/col) at arena
// vertex V0 / entry E0, sets estimates and slots, and pushes every real vertex
// into the current frontier (list and bitmap parity pc, counter slot cs).
// Graph g holds union vertices [gstart[g], gstart[g+1] - 1) and its spare
// vertex gstart[g+1] - 1.  row_ptr is written for the block's own vertices
// only (a spare's row end is never read).
template <typename Off>
__global__ void k_place(const Off* __restrict__ urp, const int* __restrict__ ucol, long long nu,
                        long long V0, long long E0, const long long* __restrict__ gstart,
                        const int* __restrict__ gslot, int ng, int t_lo, int t_hi,
                        long long* __restrict__ rp, int* __restrict__ col, uint32_t* __restrict__ est,
                        int* __restrict__ slot_of, int* __restrict__ list, long long NV,
                        uint32_t* __restrict__ bm, SweepCtl* ctl, int cs) {
    const int lane = threadIdx.x & 31;
    for (long long i0 = blockIdx.x * (long long)blockDim.x; i0 < nu;
         i0 += (long long)gridDim.x * blockDim.x) {
        const long long i = i0 + threadIdx.x;
        int tier = -1;
        const long long v = V0 + i;
        if (i < nu) {
            const long long b = (long long)urp[i], e = (long long)urp[i + 1];
            rp[v] = E0 + b;
            const int g = slot_index(gstart, ng, i);
            if (i + 1 < gstart[g + 1]) {  // a real vertex of graph g
                for (long long j = b; j < e; j++) col[E0 + j] = (int)(V0 + ucol[j]);
                const long long d = e - b;
                tier = d <= t_lo ? 0 : (d <= t_hi ? 1 : 2);
                est[v] = ((uint32_t)tier << kEstBits) | (uint32_t)d;
                slot_of[v] = gslot[g];
            } else {                      // its spare vertex
                est[v] = 0;
                slot_of[v] = -1;
            }
        }
        if (tier >= 0) atomicOr(&bm[v >> 5], 1u << (v & 31));
#pragma unroll
        for (int q = 0; q < kTiers; q++) {
            const unsigned m = __ballot_sync(0xffffffffu, tier == q);
            if (m) {
                const int leader = __ffs(m) - 1;
                unsigned base = 0;
                if (lane == leader) base = atomicAdd(&ctl->fcnt[cs][q], (unsigned)__popc(m));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (tier == q) list[(long long)q * NV + base + __popc(m & ((1u << lane) - 1u))] = (int)v;
            }
        }
    }
}

// The admission batch as one disjoint union of edge samples.  Graph g's raw
// samples sit at raw[2 s_g, 2 s_g + c_g) (sources) and raw[2 s_g + c_g,
// 2 s_{g+1}) (targets), s = sstart, c_g = s_{g+1} - s_g; its vertex ids move up
// by vstart[g].
__global__ void k_union(const int* __restrict__ raw, const long long* __restrict__ sstart,
                        const long long* __restrict__ vstart, int ng, long long samples,
                        int* __restrict__ us, int* __restrict__ ud) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < samples;
         j += (long long)gridDim.x * blockDim.x) {
        const int g = slot_index(sstart, ng, j);  // empty graphs share their start
        const long long s0 = sstart[g], c = sstart[g + 1] - s0, k = j - s0;
        const int off = (int)vstart[g];
        us[j] = raw[2 * s0 + k] + off;
        ud[j] = raw[2 * s0 + c + k] + off;
    }
}

// starts[i] <- row_ptr[starts[i]] (in place: each thread reads and writes
// only its own boundaries).
__global__ void k_gather_rp(const long long* __restrict__ urp, long long* starts, int count) {
    for (int i = threadIdx.x; i < count; i += blockDim.x) starts[i] = urp[starts[i]];
}

// Per-slot count of the vertices in the current frontier.
__global__ void k_slot_count(const int* __restrict__ list, long long NV, const SweepCtl* ctl, int cs,
                             const int* __restrict__ slot_of, int* __restrict__ cnt) {
    for (int q = 0; q < kTiers; q++) {
        const unsigned c = ctl->fcnt[cs][q];
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < c;
             i += (long long)gridDim.x * blockDim.x) {
            const int s = slot_of[list[(long long)q * NV + i]];
            if (s >= 0) atomicAdd(&cnt[s], 1);
        }
    }
}

}  // namespace
}  // namespace kc

using namespace kc;

struct kcore_batch {
    kcore_serve_options opt{};
    int device = 0;
    cudaStream_t stream = nullptr;
    // arena
    long long NV = 0, NE = 0;
    long long* rp = nullptr;
    int* col = nullptr;
    uint32_t* est = nullptr;
    int* slot_of = nullptr;
    int* list[kParities] = {nullptr, nullptr, nullptr};
    uint32_t* bitmap[kParities] = {nullptr, nullptr, nullptr};
    SweepCtl* ctl = nullptr;
    long long* trace = nullptr;
    int* slot_cnt = nullptr;
    std::vector<int> h_slot_cnt;
    long long sweep = 0;  // next sweep index of the arena
    Ranges vr, er;
    // page-locked host staging pool (int32 words, ranges guarded by mu)
    int32_t* hpool = nullptr;
    Ranges hr;
    // requests
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::unordered_map<uint64_t, Request*> reqs;
    std::vector<Request*> slots;
    std::vector<int> free_slots;
    uint64_t next_ticket = 1;
    int resident = 0;
    // engine
    std::thread worker;
    bool stop = false;
    std::mutex step_mu;  // one engine step at a time
    // statistics
    long long submitted = 0, completed = 0, cancelled = 0, failed = 0, launches = 0, sweeps = 0,
              admissions = 0, admitted_while_busy = 0;
    double busy_s = 0, admit_s = 0, sweep_s = 0, retire_s = 0;
    std::vector<double> latencies;
};

namespace {

void batch_free(kcore_batch* b) {
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    dfree(b->rp, b->stream);
    dfree(b->col, b->stream);
    dfree(b->est, b->stream);
    dfree(b->slot_of, b->stream);
    for (int p = 0; p < kParities; p++) {
        dfree(b->list[p], b->stream);
        dfree(b->bitmap[p], b->stream);
    }
    dfree(b->ctl, b->stream);
    dfree(b->trace, b->stream);
    dfree(b->slot_cnt, b->stream);
    if (b->stream) {
        cudaStreamSynchronize(b->stream);
        cudaStreamDestroy(b->stream);
    }
    if (b->hpool) cudaFreeHost(b->hpool);
    for (auto& kv : b->reqs) delete kv.second;
    delete b;
}

// Storage for a request's samples: a range of the staging pool when one is
// free, else vectors.
void stage_samples(kcore_batch* b, Request* r) {
    long long at = -1;
    if (b->hpool && r->nnz > 0) {
        std::lock_guard<std::mutex> lk(b->mu);
        at = b->hr.take(2 * r->nnz);
    }
    if (at >= 0) {
        r->h_off = at;
        r->ps = b->hpool + at;
        r->pd = r->ps + r->nnz;
    } else {
        r->src.resize(r->nnz);
        r->dst.resize(r->nnz);
        r->ps = r->src.data();
        r->pd = r->dst.data();
    }
}

// Releases the samples' storage.  Called with b->mu held.
void drop_samples(kcore_batch* b, Request* r) {
    if (r->h_off >= 0) b->hr.give(r->h_off, 2 * r->nnz);
    r->h_off = -1;
    r->ps = r->pd = nullptr;
    std::vector<int32_t>().swap(r->src);
    std::vector<int32_t>().swap(r->dst);
}

// Releases the result's storage.  Called with b->mu held.
void drop_result(kcore_batch* b, Request* r) {
    if (r->r_off >= 0) b->hr.give(r->r_off, r->n);
    r->r_off = -1;
    r->res = nullptr;
    std::vector<uint32_t>().swap(r->result);
}

// A request refused at submission.
void discard(kcore_batch* b, Request* r) {
    std::lock_guard<std::mutex> lk(b->mu);
    drop_samples(b, r);
    delete r;
}

// to[i] = from[i]; returns the largest value read as unsigned, so a negative
// id shows up as >= 2^31 (one pass: copy and range check together).
uint32_t copy_max(int32_t* __restrict__ to, const int32_t* __restrict__ from, int64_t count) {
    uint32_t m = 0;
    for (int64_t i = 0; i < count; i++) {
        const uint32_t v = (uint32_t)from[i];
        to[i] = (int32_t)v;
        m = v > m ? v : m;
    }
    return m;
}

// Host-to-device or device-to-host copies merged while both sides stay
// contiguous.
struct CopyRun {
    cudaStream_t st;
    cudaMemcpyKind kind;
    char *dst = nullptr;
    const char* src = nullptr;
    size_t bytes = 0;
    cudaError_t e = cudaSuccess;
    void add(void* to, const void* from, size_t nb) {
        if (nb == 0) return;
        if (bytes && dst + bytes == (char*)to && src + bytes == (const char*)from) {
            bytes += nb;
            return;
        }
        flush();
        dst = (char*)to;
        src = (const char*)from;
        bytes = nb;
    }
    void flush() {
        if (bytes && e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, kind, st);
        bytes = 0;
    }
};

// Bytes of arena per vertex slot and per entry.
constexpr long long kBytesPerVertex = 8 + 4 + 4 + kParities * kTiers * 4 + 1;
constexpr long long kBytesPerEntry = 4;

// Retire converged graphs.  Called with step_mu held, GPU idle on b->stream.
kcore_status retire(kcore_batch* b) {
    const int cs = (int)(b->sweep % kSlots);
    cudaError_t e = cudaMemsetAsync(b->slot_cnt, 0, sizeof(int) * b->opt.max_slots, b->stream);
    if (e == cudaSuccess) {
        k_slot_count<<<sm_count() * 4, 256, 0, b->stream>>>(b->list[b->sweep % kParities], b->NV, b->ctl, cs,
                                                     b->slot_of, b->slot_cnt);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->h_slot_cnt.data(), b->slot_cnt, sizeof(int) * b->opt.max_slots,
                            cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_status(e, "batch retire");
    std::vector<Request*> done;
    {
        std::lock_guard<std::mutex> lk(b->mu);
        for (int s = 0; s < b->opt.max_slots; s++) {
            Request* r = b->slots[s];
            if (!r || b->h_slot_cnt[s] != 0) continue;
            done.push_back(r);
        }
    }
    // results as raw estimates, into the staging pool where it has room (the
    // copies then run asynchronously; graphs admitted together sit next to
    // each other in the arena and usually in the pool, so their copies merge)
    {
        std::lock_guard<std::mutex> lk(b->mu);
        for (Request* r : done)
            if (!r->cancelled && r->n > 0 && b->hpool) r->r_off = b->hr.take(r->n);
    }
    CopyRun cr{b->stream, cudaMemcpyDeviceToHost};
    for (Request* r : done) {
        if (r->cancelled || r->n == 0) continue;
        uint32_t* to;
        if (r->r_off >= 0) {
            to = (uint32_t*)(b->hpool + r->r_off);
        } else {
            r->result.resize(r->n);
            to = r->result.data();
        }
        r->res = to;
        cr.add(to, b->est + r->v0, sizeof(uint32_t) * r->n);
    }
    cr.flush();
    e = cr.e;
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    for (Request* r : done) {
        std::lock_guard<std::mutex> lk(b->mu);
        if (e != cudaSuccess && !r->cancelled) {
            r->status = cuda_status(e, "batch result copy");
            drop_result(b, r);
        }
        b->vr.give(r->v0, r->vlen);
        b->er.give(r->e0, r->elen);
        b->slots[r->slot] = nullptr;
        b->free_slots.push_back(r->slot);
        b->resident--;
        r->state = Request::DONE;
        r->t_done = now_s();
        r->retire_launch = b->launches;
        if (r->cancelled) {
            b->cancelled++;
        } else if (r->status == KCORE_OK) {
            b->completed++;
            b->latencies.push_back(r->t_done - r->t_submit);
        } else {
            b->failed++;
        }
    }
    if (!done.empty()) b->cv_done.notify_all();
    return KCORE_OK;
}

// Admit queued graphs that fit.  Called with step_mu held, GPU idle.
// A failure before placement (allocation, upload, cleaning) is confined to
// the admission batch: its graphs fail, its ranges and slots are given back
// and the resident graphs go on.  *fatal is set when the failure came during
// or after placement into the arena, whose state is then not trusted.
kcore_status admit(kcore_batch* b, bool* fatal) {
    *fatal = false;
    std::vector<Request*> batch;
    long long vtot = 0, etot = 0, samples = 0;
    {
        std::lock_guard<std::mutex> lk(b->mu);
        const long long vfree = b->vr.largest(), efree = b->er.largest();
        while (!b->queue.empty() && !b->free_slots.empty()) {
            Request* r = b->queue.front();
            if (r->cancelled) {
                b->queue.pop_front();
                drop_samples(b, r);
                r->state = Request::DONE;
                b->cancelled++;
                b->cv_done.notify_all();
                continue;
            }
            const long long v = r->n + 1, ee = 2LL * r->nnz;  // with its spare vertex
            if (vtot + v > vfree || etot + ee > efree) break;
            b->queue.pop_front();
            r->slot = b->free_slots.back();
            b->free_slots.pop_back();
            batch.push_back(r);
            vtot += v;
            etot += ee;
            samples += r->nnz;
        }
    }
    if (batch.empty()) return KCORE_OK;
    // the disjoint union of the batch, each graph followed by its spare vertex
    const long long nu = vtot;
    const int nb = (int)batch.size();
    std::vector<long long> gstart(nb + 1), sstart(nb + 1);
    std::vector<int> gslot(nb);
    long long vo = 0, so = 0;
    for (int i = 0; i < nb; i++) {
        gstart[i] = vo;
        sstart[i] = so;
        gslot[i] = batch[i]->slot;
        so += batch[i]->nnz;
        vo += batch[i]->n + 1;
    }
    gstart[nb] = vo;
    sstart[nb] = so;
    std::string err;
    kcore_status s = KCORE_OK;
    int *raw = nullptr, *dsrc = nullptr, *dst_ = nullptr;
    long long *dgs = nullptr, *dss = nullptr;
    int* dsl = nullptr;
    DevCsr csr;
    cudaStream_t st = b->stream;
    const long long sm1 = std::max<long long>(samples, 1);
    cudaError_t e = pool_alloc((void**)&raw, sizeof(int) * 2 * sm1, st);
    if (e == cudaSuccess) e = pool_alloc((void**)&dsrc, sizeof(int) * sm1, st);
    if (e == cudaSuccess) e = pool_alloc((void**)&dst_, sizeof(int) * sm1, st);
    if (e == cudaSuccess) e = pool_alloc((void**)&dgs, sizeof(long long) * (nb + 1), st);
    if (e == cudaSuccess) e = pool_alloc((void**)&dss, sizeof(long long) * (nb + 1), st);
    if (e == cudaSuccess) e = pool_alloc((void**)&dsl, sizeof(int) * nb, st);
    // each graph's samples as they were submitted (sources, then targets);
    // staged graphs are contiguous in the pool and usually with each other
    if (e == cudaSuccess) {
        CopyRun cr{st, cudaMemcpyHostToDevice};
        for (int i = 0; i < nb; i++) {
            Request* r = batch[i];
            int* at = raw + 2 * sstart[i];
            if (r->h_off >= 0) {
                cr.add(at, r->ps, sizeof(int) * 2 * r->nnz);
            } else {
                cr.add(at, r->ps, sizeof(int) * r->nnz);
                cr.add(at + r->nnz, r->pd, sizeof(int) * r->nnz);
            }
        }
        cr.flush();
        e = cr.e;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dgs, gstart.data(), sizeof(long long) * (nb + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dss, sstart.data(), sizeof(long long) * (nb + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dsl, gslot.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && samples) {
        const int g = (int)std::min<long long>((samples + 255) / 256, (long long)sm_count() * 8);
        k_union<<<g, 256, 0, st>>>(raw, dss, dgs, nb, samples, dsrc, dst_);
        count_launch();
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) s = cuda_status(e, "batch admission copy");
    if (s == KCORE_OK) {
        s = clean_from_coo(nu, samples, dsrc, dst_, 8, b->opt.sweep.build_sort, -1, st, &csr, nullptr,
                           nullptr, &err);
        if (s != KCORE_OK) set_error(err);
    }
    if (s == KCORE_OK) {  // the cleaned size
        e = cudaMemcpyAsync(&csr.nnz, (const long long*)csr.row_ptr + nu, sizeof(long long),
                            cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_status(e, "batch admission size");
    }
    long long V0 = -1, E0 = -1;
    std::vector<long long> bound(gstart.size(), 0);  // union row_ptr at graph starts
    if (s == KCORE_OK) {
        std::lock_guard<std::mutex> lk(b->mu);
        V0 = b->vr.take(nu);
        E0 = b->er.take(std::max<long long>(csr.nnz, 1));
        if (V0 < 0 || E0 < 0) s = fail(KCORE_ERR_OOM, "batch arena fragmented");
    }
    if (s == KCORE_OK) {
        *fatal = true;  // placement writes into the arena's frontier
        const int cs = (int)(b->sweep % kSlots), pc = (int)(b->sweep % kParities);
        const int g = (int)std::min<long long>((nu + 256) / 256, (long long)sm_count() * 16);
        k_place<long long><<<g, 256, 0, st>>>(
            (const long long*)csr.row_ptr, csr.col, nu, V0, E0, dgs, dsl, nb,
            b->opt.sweep.t_lo, b->opt.sweep.t_hi, b->rp, b->col, b->est, b->slot_of, b->list[pc],
            b->NV, b->bitmap[pc], b->ctl, cs);
        count_launch();
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            k_gather_rp<<<1, 256, 0, st>>>((const long long*)csr.row_ptr, dgs, (int)gstart.size());
            count_launch();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(bound.data(), dgs, sizeof(long long) * gstart.size(),
                                cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_status(e, "batch placement");
        else *fatal = false;
    }
    dfree(raw, st);
    dfree(dsrc, st);
    dfree(dst_, st);
    dfree(dgs, st);
    dfree(dss, st);
    dfree(dsl, st);
    dfree(csr.row_ptr, st);
    dfree(csr.col, st);
    cudaStreamSynchronize(st);  // no upload from the samples' storage in flight
    std::lock_guard<std::mutex> lk(b->mu);
    for (Request* r : batch) drop_samples(b, r);
    if (s != KCORE_OK) {
        if (V0 >= 0) b->vr.give(V0, nu);
        if (E0 >= 0) b->er.give(E0, std::max<long long>(csr.nnz, 1));
        for (Request* r : batch) {
            r->status = s;
            r->state = Request::DONE;
            r->t_done = now_s();
            b->free_slots.push_back(r->slot);
            b->failed++;
        }
        b->cv_done.notify_all();
        return s;
    }
    b->admissions++;
    // per-graph ranges inside the block: each graph with its spare vertex;
    // the block's unused entry slack goes with the last graph
    const double t_admit = now_s();
    const int before = b->resident;
    if (before > 0) b->admitted_while_busy += (long long)batch.size();
    for (size_t i = 0; i < batch.size(); i++) {
        Request* r = batch[i];
        r->t_admit = t_admit;
        r->admit_launch = b->launches;
        r->resident_at_admit = before;
        r->v0 = V0 + gstart[i];
        r->vlen = r->n + 1;
        r->e0 = E0 + bound[i];
        r->elen = (i + 1 == batch.size() ? std::max<long long>(csr.nnz, 1) : bound[i + 1]) - bound[i];
        r->state = Request::RESIDENT;
        b->slots[r->slot] = r;
        b->resident++;
    }
    return KCORE_OK;
}

// One chunk of sweeps over the whole arena.  GPU idle on entry and exit.
kcore_status run_chunk(kcore_batch* b) {
    SweepArgs a;
    memset(&a, 0, sizeof(a));
    a.refined = 1;  // asynchronous sweeps: the refined activation rule
    a.row_ptr = b->rp;
    a.col = b->col;
    a.est = b->est;
    a.init_list = nullptr;
    for (int p = 0; p < kParities; p++) {
        a.list[p] = b->list[p];
        a.bitmap[p] = b->bitmap[p];
    }
    a.tier_off[0] = 0;
    a.tier_off[1] = b->NV;
    a.tier_off[2] = 2 * b->NV;
    a.ctl = b->ctl;
    a.trace = nullptr;
    a.max_trace = 0;
    a.first_sweep = b->sweep;
    a.max_sweeps = LLONG_MAX;
    a.stop_sweep = b->sweep + b->opt.chunk_sweeps;
    a.timeout_ns = (long long)(b->opt.sweep.timeout_s * 1e9);
    a.words = (b->NV + 31) / 32;
    a.n = (int)b->NV;
    a.t_lo = b->opt.sweep.t_lo;
    a.t_hi = b->opt.sweep.t_hi;
    a.low_chunk = b->opt.sweep.low_chunk;
    a.med_chunk = b->opt.sweep.med_chunk;
    a.tail_max = b->opt.sweep.tail_max < 0 ? 0 : b->opt.sweep.tail_max;
    a.off64 = 1;
    // the grid barrier counter restarts at zero for every launch
    cudaError_t e = cudaMemsetAsync(&b->ctl->bar_count, 0, sizeof(unsigned), b->stream);
    int grid = 0;
    if (e == cudaSuccess)
        e = launch_sweep(a, b->opt.sweep.block, b->opt.sweep.max_ctas, b->opt.sweep.ctas_per_sm,
                         b->stream, &grid);
    long long hs[2] = {0, 0};  // sweep, status+done
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&hs[0], &b->ctl->sweep, sizeof(long long), cudaMemcpyDeviceToHost, b->stream);
    int st2[2] = {0, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(st2, &b->ctl->status, sizeof(int) * 2, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_status(e, "batch sweep launch");
    b->launches++;
    b->sweeps += hs[0] - b->sweep;
    b->sweep = hs[0];
    if (st2[0] != 0) return fail((kcore_status)st2[0], "batch sweep kernel reported an error");
    return KCORE_OK;
}

kcore_status step(kcore_batch* b, int64_t* active) {
    std::lock_guard<std::mutex> sl(b->step_mu);
    cudaSetDevice(b->device);
    const double t0 = now_s();
    bool fatal = false;
    const kcore_status sa = admit(b, &fatal);  // a confined failure is on its tickets
    kcore_status s = fatal ? sa : KCORE_OK;
    const double t1 = now_s();
    bool any;
    {
        std::lock_guard<std::mutex> lk(b->mu);
        any = b->resident > 0;
    }
    if (s == KCORE_OK && any) s = run_chunk(b);
    const double t2 = now_s();
    if (s == KCORE_OK && any) s = retire(b);
    if (any) {
        const double t3 = now_s();
        std::lock_guard<std::mutex> lk(b->mu);
        b->busy_s += t3 - t0;
        b->admit_s += t1 - t0;
        b->sweep_s += t2 - t1;
        b->retire_s += t3 - t2;
    }
    if (active) {
        std::lock_guard<std::mutex> lk(b->mu);
        *active = b->resident + (int64_t)b->queue.size();
    }
    if (s != KCORE_OK) {
        // fail everything resident: the arena state is no longer trusted
        std::lock_guard<std::mutex> lk(b->mu);
        for (int i = 0; i < b->opt.max_slots; i++) {
            Request* r = b->slots[i];
            if (!r) continue;
            r->status = s;
            r->state = Request::DONE;
            r->t_done = now_s();
            b->slots[i] = nullptr;
            b->free_slots.push_back(i);
            b->resident--;
            b->failed++;
        }
        b->vr.reset(b->NV);
        b->er.reset(b->NE);
        b->cv_done.notify_all();
    }
    return s;
}

void engine_loop(kcore_batch* b) {
    cudaSetDevice(b->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(b->mu);
            b->cv_work.wait(lk, [&] { return b->stop || !b->queue.empty() || b->resident > 0; });
            if (b->stop) return;
        }
        step(b, nullptr);
    }
}

kcore_status enqueue(kcore_batch* b, Request* r, uint64_t* ticket) {
    std::lock_guard<std::mutex> lk(b->mu);
    if ((long long)b->queue.size() >= b->opt.max_queue) {
        drop_samples(b, r);
        delete r;
        return fail(KCORE_ERR_AGAIN, "batch queue is full");
    }
    if (r->n + 1 > b->NV || 2LL * r->nnz > b->NE) {
        drop_samples(b, r);
        delete r;
        return fail(KCORE_ERR_AGAIN, "graph can never fit the batch arena");
    }
    r->ticket = b->next_ticket++;
    r->t_submit = now_s();
    b->reqs[r->ticket] = r;
    b->queue.push_back(r);
    b->submitted++;
    *ticket = r->ticket;
    b->cv_work.notify_one();
    return KCORE_OK;
}

}  // namespace

extern "C" {

void kcore_default_serve_options(kcore_serve_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->struct_size = sizeof(*o);
    o->mem_budget = 4LL << 30;
    o->max_slots = 4096;
    o->max_queue = 1 << 20;
    o->chunk_sweeps = 16;
    o->start_thread = 1;
    kcore_default_options(&o->sweep);
    o->host_staging = 1LL << 30;
}

kcore_status kcore_batch_create(const kcore_serve_options* opt, kcore_batch** out) {
    if (!out) return fail(KCORE_ERR_INVALID, "out is NULL");
    *out = nullptr;
    kcore_serve_options o;
    kcore_default_serve_options(&o);
    if (opt) {
        if (opt->struct_size != 0 && opt->struct_size < sizeof(kcore_serve_options))
            return fail(KCORE_ERR_INVALID, "kcore_serve_options.struct_size too small");
        if (opt->mem_budget) o.mem_budget = opt->mem_budget;
        if (opt->max_slots) o.max_slots = opt->max_slots;
        if (opt->max_queue) o.max_queue = opt->max_queue;
        if (opt->chunk_sweeps) o.chunk_sweeps = opt->chunk_sweeps;
        o.start_thread = opt->start_thread;
        if (opt->sweep.struct_size) o.sweep = opt->sweep;
        if (opt->host_staging) o.host_staging = opt->host_staging;
    }
    kcore_options norm;
    kcore_status ns = normalize_options(&o.sweep, &norm);
    if (ns != KCORE_OK) return ns;
    o.sweep = norm;
    if (o.mem_budget < (16LL << 20) || o.max_slots < 1 || o.max_queue < 1 || o.chunk_sweeps < 1)
        return fail(KCORE_ERR_INVALID, "bad serve options");
    kcore_batch* b = new kcore_batch();
    b->opt = o;
    cudaGetDevice(&b->device);
    // split the budget: a third for entries beyond 8 per vertex keeps typical
    // sparse graphs balanced
    const long long per_v = kBytesPerVertex + 8 * kBytesPerEntry;
    b->NV = std::min<long long>(o.mem_budget / per_v, (long long)INT_MAX - 1);
    b->NE = (o.mem_budget - b->NV * kBytesPerVertex) / kBytesPerEntry;
    b->NV = b->NV / 32 * 32;
    std::string err;
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete b;
        return cuda_status(e, "batch stream");
    }
    kcore_status s = KCORE_OK;
    auto al = [&](void** p, size_t bytes) {
        if (s == KCORE_OK) s = dmalloc(p, bytes, &err, b->stream);
    };
    al((void**)&b->rp, sizeof(long long) * (b->NV + 1));
    al((void**)&b->col, sizeof(int) * std::max<long long>(b->NE, 1));
    al((void**)&b->est, sizeof(uint32_t) * b->NV);
    al((void**)&b->slot_of, sizeof(int) * b->NV);
    for (int p = 0; p < kParities; p++) {
        al((void**)&b->list[p], sizeof(int) * kTiers * b->NV);
        al((void**)&b->bitmap[p], sizeof(uint32_t) * (b->NV / 32 + 1));
    }
    al((void**)&b->ctl, sizeof(SweepCtl));
    al((void**)&b->slot_cnt, sizeof(int) * o.max_slots);
    if (s != KCORE_OK) {
        set_error(err);
        batch_free(b);
        return s;
    }
    const long long zero[kTiers] = {0, 0, 0};
    e = launch_ctl_init(b->ctl, zero, b->stream);
    for (int p = 0; p < kParities && e == cudaSuccess; p++)
        e = cudaMemsetAsync(b->bitmap[p], 0, sizeof(uint32_t) * (b->NV / 32 + 1), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->slot_of, 0xff, sizeof(int) * b->NV, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_status(e, "batch init");
    }
    b->h_slot_cnt.assign(o.max_slots, 0);
    b->slots.assign(o.max_slots, nullptr);
    for (int i = o.max_slots - 1; i >= 0; i--) b->free_slots.push_back(i);
    b->vr.reset(b->NV);
    b->er.reset(b->NE);
    if (o.host_staging > 0) {
        // the pool is an optimisation: without it copies use pageable memory
        const long long words = o.host_staging / (long long)sizeof(int32_t);
        if (!alloc_fault() &&
            cudaHostAlloc((void**)&b->hpool, sizeof(int32_t) * words, cudaHostAllocDefault) == cudaSuccess) {
            b->hr.reset(words);
        } else {
            b->hpool = nullptr;
            cudaGetLastError();
        }
    }
    if (o.start_thread) b->worker = std::thread(engine_loop, b);
    *out = b;
    return KCORE_OK;
}

kcore_status kcore_submit_coo(kcore_batch* b, int64_t n, int64_t nnz, const int32_t* src,
                              const int32_t* dst, uint32_t flags, uint64_t* ticket) {
    if (!b || !ticket) return fail(KCORE_ERR_INVALID, "NULL argument");
    if (flags & KCORE_IN_DEVICE) return fail(KCORE_ERR_INVALID, "batch input must be host arrays");
    if (n < 0 || n >= INT_MAX || nnz < 0 || (nnz > 0 && (!src || !dst)))
        return fail(KCORE_ERR_INVALID, "bad graph arguments");
    Request* r = new Request();
    r->n = n;
    r->nnz = nnz;
    stage_samples(b, r);
    const uint32_t hi = std::max(copy_max(r->ps, src, nnz), copy_max(r->pd, dst, nnz));
    if (nnz > 0 && (uint64_t)hi >= (uint64_t)n) {
        discard(b, r);
        return fail(KCORE_ERR_INVALID, "edge endpoint outside [0, n)");
    }
    return enqueue(b, r, ticket);
}

kcore_status kcore_submit(kcore_batch* b, int64_t n, const void* row_ptr, int32_t row_ptr_bytes,
                          const int32_t* col_idx, uint32_t flags, uint64_t* ticket) {
    if (!b || !ticket || !row_ptr) return fail(KCORE_ERR_INVALID, "NULL argument");
    if (flags & KCORE_IN_DEVICE) return fail(KCORE_ERR_INVALID, "batch input must be host arrays");
    if (row_ptr_bytes != 4 && row_ptr_bytes != 8) return fail(KCORE_ERR_INVALID, "row_ptr_bytes");
    if (n < 0 || n >= INT_MAX) return fail(KCORE_ERR_INVALID, "bad n");
    auto at = [&](int64_t i) -> int64_t {
        return row_ptr_bytes == 8 ? ((const int64_t*)row_ptr)[i] : ((const int32_t*)row_ptr)[i];
    };
    const int64_t nnz = at(n);
    if (at(0) != 0 || nnz < 0 || (nnz > 0 && !col_idx))
        return fail(KCORE_ERR_INVALID, "row_ptr must start at 0 and end at nnz >= 0");
    Request* r = new Request();
    r->n = n;
    r->nnz = nnz;
    stage_samples(b, r);
    for (int64_t u = 0; u < n; u++) {
        const int64_t lo = at(u), hi = at(u + 1);
        if (hi < lo || hi > nnz) {
            discard(b, r);
            return fail(KCORE_ERR_INVALID, "row_ptr must be non-decreasing");
        }
        for (int64_t j = lo; j < hi; j++) r->ps[j] = (int32_t)u;
    }
    if (nnz > 0 && (uint64_t)copy_max(r->pd, col_idx, nnz) >= (uint64_t)n) {
        discard(b, r);
        return fail(KCORE_ERR_INVALID, "col_idx entry outside [0, n)");
    }
    return enqueue(b, r, ticket);
}

kcore_status kcore_poll(kcore_batch* b, uint64_t ticket, int32_t* coreness_out, int64_t timeout_us) {
    return kcore_poll_info(b, ticket, coreness_out, timeout_us, nullptr);
}

kcore_status kcore_poll_info(kcore_batch* b, uint64_t ticket, int32_t* coreness_out,
                             int64_t timeout_us, kcore_ticket_info* info) {
    if (!b) return fail(KCORE_ERR_INVALID, "NULL batch");
    std::unique_lock<std::mutex> lk(b->mu);
    auto it = b->reqs.find(ticket);
    if (it == b->reqs.end()) return fail(KCORE_ERR_INVALID, "unknown ticket");
    Request* r = it->second;
    auto ready = [&] { return r->state == Request::DONE; };
    if (!ready()) {
        if (timeout_us == 0) return KCORE_PENDING;
        if (!b->opt.start_thread) {
            // no engine thread: drive the engine from here
            lk.unlock();
            const double t_end = timeout_us < 0 ? 1e300 : now_s() + timeout_us * 1e-6;
            for (;;) {
                int64_t active = 0;
                kcore_status s = step(b, &active);
                (void)s;
                lk.lock();
                if (ready() || now_s() > t_end) break;
                lk.unlock();
            }
        } else if (timeout_us < 0) {
            b->cv_done.wait(lk, ready);
        } else {
            b->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
        }
        if (!ready()) return KCORE_PENDING;
    }
    kcore_status s = r->cancelled ? KCORE_ERR_CANCELLED : r->status;
    if (info) {
        info->submit_s = r->t_submit;
        info->admit_s = r->t_admit;
        info->done_s = r->t_done;
        info->admit_launch = r->admit_launch;
        info->retire_launch = r->retire_launch;
        info->resident_at_admit = r->resident_at_admit;
    }
    if (s == KCORE_OK && coreness_out && r->n) {
        const uint32_t* raw = r->res;
        for (int64_t i = 0; i < r->n; i++) coreness_out[i] = (int32_t)(raw[i] & kEstMask);
    }
    b->reqs.erase(it);
    drop_samples(b, r);
    drop_result(b, r);
    delete r;
    if (s < 0) set_error(s == KCORE_ERR_CANCELLED ? "request was cancelled" : "request failed");
    return s;
}

kcore_status kcore_cancel(kcore_batch* b, uint64_t ticket) {
    if (!b) return fail(KCORE_ERR_INVALID, "NULL batch");
    std::lock_guard<std::mutex> lk(b->mu);
    auto it = b->reqs.find(ticket);
    if (it == b->reqs.end()) return fail(KCORE_ERR_INVALID, "unknown ticket");
    it->second->cancelled = true;
    b->cv_work.notify_one();
    return KCORE_OK;
}

kcore_status kcore_batch_step(kcore_batch* b, int64_t* active) {
    if (!b) return fail(KCORE_ERR_INVALID, "NULL batch");
    if (b->opt.start_thread) return fail(KCORE_ERR_INVALID, "the engine runs its own thread");
    return step(b, active);
}

kcore_status kcore_batch_stats_get(kcore_batch* b, kcore_batch_stats* out) {
    if (!b || !out) return fail(KCORE_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(b->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = b->submitted;
    out->completed = b->completed;
    out->cancelled = b->cancelled;
    out->failed = b->failed;
    out->queued = (int64_t)b->queue.size();
    out->resident = b->resident;
    out->launches = b->launches;
    out->sweeps = b->sweeps;
    out->arena_bytes = b->NV * kBytesPerVertex + b->NE * kBytesPerEntry;
    out->arena_used_peak = b->vr.peak() * kBytesPerVertex + b->er.peak() * kBytesPerEntry;
    out->busy_s = b->busy_s;
    out->admit_s = b->admit_s;
    out->sweep_s = b->sweep_s;
    out->retire_s = b->retire_s;
    out->admissions = b->admissions;
    out->admitted_while_busy = b->admitted_while_busy;
    if (!b->latencies.empty()) {
        std::vector<double> l = b->latencies;
        std::sort(l.begin(), l.end());
        auto q = [&](double p) {
            const size_t i = (size_t)std::min<double>(l.size() - 1, std::max(0.0, p * (l.size() - 1)));
            return l[i] * 1e3;
        };
        out->latency_p50_ms = q(0.50);
        out->latency_p99_ms = q(0.99);
    }
    return KCORE_OK;
}

void kcore_batch_destroy(kcore_batch* b) {
    if (!b) return;
    {
        std::lock_guard<std::mutex> lk(b->mu);
        b->stop = true;
        b->cv_work.notify_all();
    }
    if (b->worker.joinable()) b->worker.join();
    batch_free(b);
}

}  // extern "C"
