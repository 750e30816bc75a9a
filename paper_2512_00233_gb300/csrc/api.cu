// C ABI of the single-graph path: kcore_create*, kcore_run, stats, destroy.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cstring>
#include <string>
#include <vector>

#include "kc_common.cuh"

namespace kc {

static thread_local std::string t_err;
static std::atomic<long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launches() { return g_launches.load(std::memory_order_relaxed); }

void set_error(const std::string& msg) { t_err = msg; }

kcore_status fail(kcore_status s, const std::string& msg) {
    t_err = msg;
    return s;
}

kcore_status cuda_status(cudaError_t e, const char* what) {
    cudaGetLastError();
    t_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? KCORE_ERR_OOM : KCORE_ERR_CUDA;
}

kcore_status normalize_options(const kcore_options* in, kcore_options* out) {
    kcore_default_options(out);
    if (!in) return KCORE_OK;
    if (in->struct_size != 0 && in->struct_size < sizeof(kcore_options))
        return fail(KCORE_ERR_INVALID, "kcore_options.struct_size too small");
    if (in->t_lo) out->t_lo = in->t_lo;
    if (in->t_hi) out->t_hi = in->t_hi;
    if (in->block) out->block = in->block;
    if (in->low_chunk) out->low_chunk = in->low_chunk;
    if (in->med_chunk) out->med_chunk = in->med_chunk;
    if (in->tail_max) out->tail_max = in->tail_max;
    if (in->ctas_per_sm) out->ctas_per_sm = in->ctas_per_sm;
    if (in->max_ctas) out->max_ctas = in->max_ctas;
    if (in->max_sweeps) out->max_sweeps = in->max_sweeps;
    if (in->timeout_s > 0) out->timeout_s = in->timeout_s;
    if (in->build_sort) out->build_sort = in->build_sort;
    if (in->relabel) out->relabel = in->relabel;
    if (out->t_lo < 1 || out->t_lo > 32) return fail(KCORE_ERR_INVALID, "t_lo must be in 1..32");
    if (out->t_hi < out->t_lo || out->t_hi > kMedBig)
        return fail(KCORE_ERR_INVALID, "t_hi must be in t_lo..2048");
    if (out->t_lo > 16) return fail(KCORE_ERR_INVALID, "t_lo must be in 1..16");
    if (out->block < 64 || out->block > 512 || out->block % 32)
        return fail(KCORE_ERR_INVALID, "block must be a multiple of 32 in 64..512");
    if (out->low_chunk < 1 || out->low_chunk > 8) return fail(KCORE_ERR_INVALID, "low_chunk 1..8");
    if (out->med_chunk < 1 || out->med_chunk > 64) return fail(KCORE_ERR_INVALID, "med_chunk 1..64");
    if (out->max_sweeps < 0 || out->ctas_per_sm < 0 || out->max_ctas < 0)
        return fail(KCORE_ERR_INVALID, "negative option");
    if (out->build_sort < -1 || out->build_sort > 1)
        return fail(KCORE_ERR_INVALID, "build_sort must be -1, 0 or 1");
    if (out->relabel < -1 || out->relabel > 2)
        return fail(KCORE_ERR_INVALID, "relabel must be -1, 0, 1 or 2");
    return KCORE_OK;
}

}  // namespace kc

using namespace kc;

struct kcore_graph {
    int device = 0;
    DevCsr csr;                // the cleaned CSR the sweeps read (renumbered when relabeled)
    bool relabeled = false;    // csr uses new ids: new_of_old[caller's id]
    int* new_of_old = nullptr; // the numbering (n each), when relabeled
    int* old_of_new = nullptr;
    int* hout = nullptr;       // coreness in the caller's ids before a copy to host memory
    kcore_options opt{};
    uint32_t* est0 = nullptr;
    uint32_t* est = nullptr;
    int* init_list = nullptr;
    int* list[kParities] = {nullptr, nullptr, nullptr};
    uint32_t* bitmap[kParities] = {nullptr, nullptr, nullptr};
    int* upd_list = nullptr;
    int* upd_val = nullptr;
    SweepCtl* ctl = nullptr;
    long long* trace = nullptr;
    long long max_trace = 0;
    long long tier_cnt[kTiers] = {0, 0, 0};
    SweepCtl* hctl = nullptr;  // pinned copy of the control block after a run
    TierOut* htier = nullptr;  // pinned copy of the tier split results (same block)
    TierOut* dtier = nullptr;  // device tier split results
    void* state = nullptr;     // one block holding est0 .. dtier above
    cudaEvent_t ev[6] = {};    // create0, create1, run0, sweep0, sweep1, run1
    bool pending = false;
    bool ran = false;
    kcore_status last_status = KCORE_OK;
    int last_grid = 0;
    float ms_create = 0.f;
    // KCORE_GRAPH: captured run
    cudaStream_t gstream = nullptr;
    cudaEvent_t join[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec = nullptr;
    int32_t* gout = nullptr;
    uint32_t gflags = 0;
    long long gopt_epoch = -1, opt_epoch = 0;
    long long gkernels = 0;   // kernels in the captured graph
};

namespace {

enum { EV_C0, EV_C1, EV_R0, EV_S0, EV_S1, EV_R1 };

void release(kcore_graph* g) {
    if (!g) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    dfree(g->csr.row_ptr);
    dfree(g->csr.col);
    dfree(g->new_of_old);
    dfree(g->old_of_new);
    dfree(g->hout);
    dfree(g->state);  // est0, est, lists, bitmaps, ctl, trace, dtier
    dfree(g->upd_list);
    dfree(g->upd_val);
    if (g->hctl) pinned_put(g->hctl);
    for (auto& e : g->ev)
        if (e) cudaEventDestroy(e);
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    for (auto& e : g->join)
        if (e) cudaEventDestroy(e);
    if (g->gstream) cudaStreamDestroy(g->gstream);
    cudaSetDevice(prev);
    delete g;
}

// The one wait of graph creation: tier sizes, row_ptr[n] and the degree check.
kcore_status read_tiers(kcore_graph* g, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(g->htier, g->dtier, sizeof(TierOut), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e, "tier split");
    const TierOut& t = *g->htier;
    if (t.bad) return fail(KCORE_ERR_INVALID, "a vertex degree is 2^30 or more");
    for (int q = 0; q < kTiers; q++) g->tier_cnt[q] = (long long)t.bound[q + 1] - t.bound[q];
    if (g->csr.n == 0) {
        g->csr.nnz = 0;
    } else {
        g->csr.nnz = t.nnz;
        if (g->csr.off_bytes == 4 && g->csr.nnz > 0x7fffffffLL)
            return fail(KCORE_ERR_INVALID, "cleaned graph has 2m >= 2^31 entries; use 8-byte row_ptr");
    }
    return KCORE_OK;
}

// Allocates the per-run state and splits the vertices into degree tiers.
kcore_status finish_graph(kcore_graph* g, cudaStream_t st) {
    std::string err;
    const int64_t n = g->csr.n;
    const size_t words = (size_t)((n + 31) / 32);
    g->max_trace = 1 << 16;
    // one allocation, carved into 256-byte aligned arrays
    auto rnd = [](size_t b) { return (std::max<size_t>(b, 1) + 255) & ~size_t(255); };
    const size_t vec = rnd(sizeof(uint32_t) * n), bm = rnd(sizeof(uint32_t) * words);
    const size_t total = (3 + kParities) * vec + kParities * bm + rnd(sizeof(SweepCtl)) +
                         rnd(sizeof(long long) * kTraceCols * g->max_trace) + rnd(sizeof(TierOut));
    kcore_status s = dmalloc(&g->state, total, &err, st);
    if (s != KCORE_OK) return fail(s, err);
    char* at = (char*)g->state;
    auto take = [&](size_t b) {
        char* p = at;
        at += b;
        return p;
    };
    g->est0 = (uint32_t*)take(vec);
    g->est = (uint32_t*)take(vec);
    g->init_list = (int*)take(vec);
    for (int p = 0; p < kParities; p++) {
        g->list[p] = (int*)take(vec);
        g->bitmap[p] = (uint32_t*)take(bm);
    }
    g->ctl = (SweepCtl*)take(rnd(sizeof(SweepCtl)));
    g->trace = (long long*)take(rnd(sizeof(long long) * kTraceCols * g->max_trace));
    g->dtier = (TierOut*)take(rnd(sizeof(TierOut)));
    static_assert(sizeof(SweepCtl) <= 2048 && sizeof(TierOut) <= kPinnedBlock - 2048,
                  "pinned block layout");
    cudaError_t e = pinned_get((void**)&g->hctl, kPinnedBlock);
    if (e != cudaSuccess) return cuda_status(e, "pinned host block");
    memset(g->hctl, 0, sizeof(SweepCtl));
    g->htier = (TierOut*)((char*)g->hctl + 2048);
    s = tier_split(n, g->csr.row_ptr, g->csr.off_bytes, g->opt.t_lo, g->opt.t_hi, g->est0,
                   g->init_list, g->dtier, st, &err);
    if (s != KCORE_OK) return fail(s, err);
    return read_tiers(g, st);
}

kcore_status begin_create(int64_t n, int32_t row_ptr_bytes, const kcore_options* opt,
                          kcore_graph** out, kcore_graph** g) {
    if (!out) return fail(KCORE_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (n < 0 || n > INT_MAX) return fail(KCORE_ERR_INVALID, "n must be in [0, 2^31)");
    if (row_ptr_bytes != 4 && row_ptr_bytes != 8)
        return fail(KCORE_ERR_INVALID, "row_ptr_bytes must be 4 or 8");
    kcore_options o;
    kcore_status s = normalize_options(opt, &o);
    if (s != KCORE_OK) return s;
    *g = new kcore_graph();
    (*g)->opt = o;
    cudaGetDevice(&(*g)->device);
    for (auto& e : (*g)->ev) {
        cudaError_t ce = cudaEventCreate(&e);
        if (ce != cudaSuccess) {
            release(*g);
            *g = nullptr;
            return cuda_status(ce, "cudaEventCreate");
        }
    }
    return KCORE_OK;
}

// Host input -> temporary device copy.
template <typename T>
kcore_status upload(const T* host, size_t count, cudaStream_t st, T** dev) {
    cudaError_t e = pool_alloc((void**)dev, std::max<size_t>(count, 1) * sizeof(T), st);
    if (e != cudaSuccess) return cuda_status(e, "cudaMallocAsync (input copy)");
    if (count) {
        e = cudaMemcpyAsync(*dev, host, count * sizeof(T), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_status(e, "cudaMemcpyAsync (input copy)");
    }
    return KCORE_OK;
}

// The update lists of synchronous mode, allocated on the first synchronous
// run: both or neither (a half-allocated pair is released again).
kcore_status ensure_sync_buffers(kcore_graph* g, cudaStream_t st) {
    if (g->upd_list && g->upd_val) return KCORE_OK;
    std::string err;
    const int64_t n = g->csr.n;
    kcore_status s = dmalloc((void**)&g->upd_list, sizeof(int) * n, &err, st);
    if (s == KCORE_OK) s = dmalloc((void**)&g->upd_val, sizeof(int) * n, &err, st);
    if (s == KCORE_OK && cudaStreamSynchronize(st) != cudaSuccess) {
        s = KCORE_ERR_CUDA;
        err = "synchronous-mode buffers";
    }
    if (s != KCORE_OK) {
        dfree(g->upd_list, st);
        dfree(g->upd_val, st);
        g->upd_list = nullptr;
        g->upd_val = nullptr;
        return fail(s, err);
    }
    return KCORE_OK;
}

kcore_status wait_run(kcore_graph* g) {
    if (!g->pending) return g->last_status;
    g->pending = false;
    cudaError_t e = cudaEventSynchronize(g->ev[EV_R1]);
    if (e != cudaSuccess) {
        g->last_status = cuda_status(e, "kcore_run");
        return g->last_status;
    }
    const int st = g->hctl->status;
    if (st != 0) {
        g->last_status = (kcore_status)st;
        if (st == KCORE_ERR_NOT_CONVERGED)
            set_error("sweep cap reached before the frontier emptied");
        else if (st == KCORE_ERR_TIMEOUT)
            set_error("a device wait exceeded timeout_s");
        else
            set_error("sweep kernel reported an error");
    } else if (!g->hctl->done) {
        g->last_status = KCORE_ERR_CUDA;
        set_error("sweep kernel ended without converging or reporting an error");
    } else {
        g->last_status = KCORE_OK;
    }
    return g->last_status;
}

}  // namespace

extern "C" {

void kcore_default_options(kcore_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->struct_size = sizeof(kcore_options);
    o->t_lo = 16;
    o->t_hi = 2048;
    o->block = 512;
    o->low_chunk = 8;
    o->med_chunk = 4;
    o->tail_max = 1024;
    o->ctas_per_sm = 0;
    o->max_ctas = 0;
    o->max_sweeps = 0;
    o->timeout_s = 20.0;
    o->build_sort = 0;
}

const char* kcore_last_error(void) { return t_err.c_str(); }

const char* kcore_version(void) { return "kcore-gb300 0.1 (sm_103a)"; }

int64_t kcore_kernel_launches(void) { return (int64_t)launches(); }

kcore_status kcore_create_coo(int64_t n, int64_t nnz, const int32_t* src, const int32_t* dst,
                              int32_t row_ptr_bytes, uint32_t flags, const kcore_options* opt,
                              void* cuda_stream, kcore_graph** out) {
    kcore_graph* g = nullptr;
    kcore_status s = begin_create(n, row_ptr_bytes, opt, out, &g);
    if (s != KCORE_OK) return s;
    if (nnz < 0 || (nnz > 0 && (!src || !dst))) {
        release(g);
        return fail(KCORE_ERR_INVALID, "bad edge arrays");
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaEventRecord(g->ev[EV_C0], st);
    const int *ds = src, *dd = dst;
    int *tmp_s = nullptr, *tmp_d = nullptr;
    if (!(flags & KCORE_IN_DEVICE)) {
        s = upload(src, (size_t)nnz, st, &tmp_s);
        if (s == KCORE_OK) s = upload(dst, (size_t)nnz, st, &tmp_d);
        ds = tmp_s;
        dd = tmp_d;
    }
    std::string err;
    if (s == KCORE_OK) {
        s = clean_from_coo(n, nnz, ds, dd, row_ptr_bytes, g->opt.build_sort, g->opt.relabel, st,
                           &g->csr, &g->new_of_old, &g->old_of_new, &err);
        if (s != KCORE_OK) set_error(err);
        g->relabeled = g->new_of_old != nullptr;
        if (s == KCORE_OK && g->relabeled) {
            s = dmalloc((void**)&g->hout, sizeof(int) * std::max<int64_t>(n, 1), &err, st);
            if (s != KCORE_OK) set_error(err);
        }
    }
    if (tmp_s) cudaFreeAsync(tmp_s, st);
    if (tmp_d) cudaFreeAsync(tmp_d, st);
    if (s == KCORE_OK) s = finish_graph(g, st);
    if (s == KCORE_OK) {
        cudaEventRecord(g->ev[EV_C1], st);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_status(e, "kcore_create_coo");
        else cudaEventElapsedTime(&g->ms_create, g->ev[EV_C0], g->ev[EV_C1]);
    }
    if (s != KCORE_OK) {
        release(g);
        return s;
    }
    *out = g;
    return KCORE_OK;
}

kcore_status kcore_create(int64_t n, const void* row_ptr, int32_t row_ptr_bytes,
                          const int32_t* col_idx, uint32_t flags, const kcore_options* opt,
                          void* cuda_stream, kcore_graph** out) {
    kcore_graph* g = nullptr;
    kcore_status s = begin_create(n, row_ptr_bytes, opt, out, &g);
    if (s != KCORE_OK) return s;
    if (!row_ptr) {
        release(g);
        return fail(KCORE_ERR_INVALID, "row_ptr is NULL");
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaEventRecord(g->ev[EV_C0], st);
    // nnz = row_ptr[n]
    int64_t nnz = 0;
    if (flags & KCORE_IN_DEVICE) {
        long long tmp = 0;
        cudaError_t e = cudaMemcpyAsync(&tmp, (const char*)row_ptr + (size_t)row_ptr_bytes * n,
                                        row_ptr_bytes, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            release(g);
            return cuda_status(e, "read row_ptr[n]");
        }
        nnz = row_ptr_bytes == 8 ? tmp : (int64_t)(int32_t)(tmp & 0xffffffffLL);
    } else {
        nnz = row_ptr_bytes == 8 ? ((const int64_t*)row_ptr)[n] : ((const int32_t*)row_ptr)[n];
    }
    if (nnz < 0 || (nnz > 0 && !col_idx)) {
        release(g);
        return fail(KCORE_ERR_INVALID, "row_ptr[n] must be >= 0 and col_idx non-NULL");
    }
    const void* drp = row_ptr;
    const int* dcol = col_idx;
    void* tmp_rp = nullptr;
    int* tmp_col = nullptr;
    if (!(flags & KCORE_IN_DEVICE)) {
        if (row_ptr_bytes == 8)
            s = upload((const long long*)row_ptr, (size_t)n + 1, st, (long long**)&tmp_rp);
        else
            s = upload((const int*)row_ptr, (size_t)n + 1, st, (int**)&tmp_rp);
        if (s == KCORE_OK) s = upload(col_idx, (size_t)nnz, st, &tmp_col);
        drp = tmp_rp;
        dcol = tmp_col;
    }
    std::string err;
    if (s == KCORE_OK) {
        if (flags & KCORE_IN_CLEAN) {
            s = check_clean_csr(n, drp, row_ptr_bytes, dcol, nnz, st, &err);
            if (s == KCORE_OK) s = dmalloc(&g->csr.row_ptr, (size_t)row_ptr_bytes * (n + 1), &err, st);
            if (s == KCORE_OK) s = dmalloc((void**)&g->csr.col, sizeof(int) * nnz, &err, st);
            if (s == KCORE_OK) {
                cudaError_t e = cudaMemcpyAsync(g->csr.row_ptr, drp, (size_t)row_ptr_bytes * (n + 1),
                                                cudaMemcpyDeviceToDevice, st);
                if (e == cudaSuccess && nnz)
                    e = cudaMemcpyAsync(g->csr.col, dcol, sizeof(int) * nnz,
                                        cudaMemcpyDeviceToDevice, st);
                if (e != cudaSuccess) s = cuda_status(e, "copy clean CSR");
                g->csr.n = n;
                g->csr.nnz = nnz;
                g->csr.off_bytes = row_ptr_bytes;
            }
        } else {
            s = clean_from_csr(n, drp, row_ptr_bytes, dcol, nnz, row_ptr_bytes, st, &g->csr, &err);
        }
        if (s != KCORE_OK && !err.empty()) set_error(err);
    }
    if (tmp_rp) cudaFreeAsync(tmp_rp, st);
    if (tmp_col) cudaFreeAsync(tmp_col, st);
    if (s == KCORE_OK) s = finish_graph(g, st);
    if (s == KCORE_OK) {
        cudaEventRecord(g->ev[EV_C1], st);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_status(e, "kcore_create");
        else cudaEventElapsedTime(&g->ms_create, g->ev[EV_C0], g->ev[EV_C1]);
    }
    if (s != KCORE_OK) {
        release(g);
        return s;
    }
    *out = g;
    return KCORE_OK;
}

kcore_status kcore_set_options(kcore_graph* g, const kcore_options* opt, void* cuda_stream) {
    if (!g) return fail(KCORE_ERR_INVALID, "graph is NULL");
    kcore_options o;
    kcore_status s = normalize_options(opt, &o);
    if (s != KCORE_OK) return s;
    s = wait_run(g);
    (void)s;
    const bool rebin = o.t_lo != g->opt.t_lo || o.t_hi != g->opt.t_hi;
    g->opt = o;
    g->opt_epoch++;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (!rebin) return KCORE_OK;
    std::string err;
    s = tier_split(g->csr.n, g->csr.row_ptr, g->csr.off_bytes, o.t_lo, o.t_hi, g->est0,
                   g->init_list, g->dtier, st, &err);
    if (s != KCORE_OK) return fail(s, err);
    return read_tiers(g, st);
}

// Enqueues one run on `st` (no wait).  The sequence is the same whether it
// runs directly or is captured into a CUDA graph.
// Under capture the events become event-record nodes of the graph, so the
// timings and the completion event work the same way on replay.
cudaError_t record(cudaEvent_t ev, cudaStream_t st, bool capture) {
    return cudaEventRecordWithFlags(ev, st, capture ? cudaEventRecordExternal : cudaEventRecordDefault);
}

// Warm start of a run (kcore_run_from): device arrays, null for a cold start.
struct WarmStart {
    const int* start = nullptr;
    const int* frontier = nullptr;
    long long nf = 0;
};

kcore_status enqueue_run(kcore_graph* g, int32_t* coreness_out, uint32_t flags, cudaStream_t st,
                         bool capture, const WarmStart& warm = WarmStart()) {
    const int64_t n = g->csr.n;
    const bool sync_mode = (flags & KCORE_SYNC_MODE) != 0;
    const size_t words = (size_t)((n + 31) / 32);
    // The launch itself initialises the estimates and the frontier (a2) and
    // writes the coreness out (a6); only the control block is cleared here.
    cudaError_t e = record(g->ev[EV_R0], st, capture);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->ctl, 0, sizeof(SweepCtl), st);
    if (e != cudaSuccess) return cuda_status(e, "kcore_run init");

    SweepArgs a;
    memset(&a, 0, sizeof(a));
    a.row_ptr = g->csr.row_ptr;
    a.col = g->csr.col;
    a.est = g->est;
    a.init_list = g->init_list;
    for (int p = 0; p < kParities; p++) {
        a.list[p] = g->list[p];
        a.bitmap[p] = g->bitmap[p];
    }
    a.words = (long long)words;
    a.upd_list = g->upd_list;
    a.upd_val = g->upd_val;
    a.tier_off[0] = 0;
    a.tier_off[1] = g->tier_cnt[0];
    a.tier_off[2] = g->tier_cnt[0] + g->tier_cnt[1];
    a.ctl = g->ctl;
    a.trace = g->trace;
    a.max_trace = g->max_trace;
    a.first_sweep = 0;
    a.max_sweeps = g->opt.max_sweeps ? g->opt.max_sweeps : 2 * g->csr.nnz + n + 1;
    a.stop_sweep = LLONG_MAX;
    a.timeout_ns = (long long)(g->opt.timeout_s * 1e9);
    a.n = (int)n;
    a.t_lo = g->opt.t_lo;
    a.t_hi = g->opt.t_hi;
    a.low_chunk = g->opt.low_chunk;
    a.med_chunk = g->opt.med_chunk;
    a.tail_max = g->opt.tail_max < 0 ? 0 : g->opt.tail_max;
    a.sync_mode = sync_mode ? 1 : 0;
    // synchronous: Alg. 3 as printed unless KCORE_REFINED; asynchronous: the
    // refined rule unless KCORE_SIMPLE
    a.refined = sync_mode ? ((flags & KCORE_REFINED) ? 1 : 0) : ((flags & KCORE_SIMPLE) ? 0 : 1);
    a.off64 = g->csr.off_bytes == 8 ? 1 : 0;
    a.est0 = g->est0;
    for (int q = 0; q < kTiers; q++) a.init_cnt[q] = (unsigned)g->tier_cnt[q];
    if (warm.start) {  // estimates and F_0 set up here instead of inside the launch
        a.est0 = nullptr;
        if (warm.frontier) a.init_list = nullptr;  // sweep 0 reads list[0]
        if (words) {
            e = cudaMemsetAsync(g->bitmap[0], warm.frontier ? 0 : 0xff, sizeof(uint32_t) * words, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(g->bitmap[1], 0, sizeof(uint32_t) * words, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(g->bitmap[2], 0, sizeof(uint32_t) * words, st);
        }
        if (e == cudaSuccess && !warm.frontier) e = launch_ctl_init(g->ctl, g->tier_cnt, st);
        if (e == cudaSuccess)
            e = launch_warm_init(a, g->csr.row_ptr, g->est0, warm.start, warm.frontier, warm.nf, st);
        if (e != cudaSuccess) return cuda_status(e, "warm start");
    }
    a.perm = g->relabeled ? g->new_of_old : nullptr;
    int* host_src = g->relabeled ? g->hout : (int*)g->est;  // coreness before the copy to the host
    a.out = (flags & KCORE_OUT_DEVICE) ? coreness_out : host_src;

    // Grid: enough CTAs for the first sweep's work, at most the co-resident maximum.
    const long long work = n + g->csr.nnz;
    long long want = (work + (long long)g->opt.block * 32 - 1) / ((long long)g->opt.block * 32);
    want = std::max<long long>(1, want);
    if (g->opt.max_ctas > 0) want = std::min<long long>(want, g->opt.max_ctas);
    e = record(g->ev[EV_S0], st, capture);
    if (e == cudaSuccess)
        e = launch_sweep(a, g->opt.block, (int)std::min<long long>(want, INT_MAX), g->opt.ctas_per_sm,
                         st, &g->last_grid);
    if (e == cudaSuccess) e = record(g->ev[EV_S1], st, capture);
    if (e != cudaSuccess) return cuda_status(e, "sweep launch");
    if (!(flags & KCORE_OUT_DEVICE) && n)
        e = cudaMemcpyAsync(coreness_out, host_src, sizeof(int) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->hctl, g->ctl, sizeof(SweepCtl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = record(g->ev[EV_R1], st, capture);
    if (e != cudaSuccess) return cuda_status(e, "kcore_run output");
    return KCORE_OK;
}

// KCORE_GRAPH: the run's sequence is captured once on the graph's own stream
// and replayed; the caller's stream and that stream are joined by events.
kcore_status graph_run(kcore_graph* g, int32_t* coreness_out, uint32_t flags, cudaStream_t st) {
    const uint32_t key_flags = flags & (KCORE_SYNC_MODE | KCORE_REFINED | KCORE_SIMPLE);
    cudaError_t e = cudaSuccess;
    if (!g->gstream) {
        e = cudaStreamCreateWithFlags(&g->gstream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->join[0], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->join[1], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_status(e, "graph stream");
    }
    if (!g->gexec || g->gout != coreness_out || g->gflags != key_flags || g->gopt_epoch != g->opt_epoch) {
        if (g->gexec) cudaGraphExecDestroy(g->gexec);
        g->gexec = nullptr;
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(g->gstream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_status(e, "begin capture");
        const long long before = g_launches.load();
        kcore_status s = enqueue_run(g, coreness_out, key_flags | KCORE_OUT_DEVICE, g->gstream, true);
        e = cudaStreamEndCapture(g->gstream, &graph);
        g->gkernels = g_launches.load() - before;
        g_launches.fetch_sub(g->gkernels);   // counted again at each replay
        if (s != KCORE_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess) return cuda_status(e, "end capture");
        e = cudaGraphInstantiate(&g->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_status(e, "graph instantiate");
        g->gout = coreness_out;
        g->gflags = key_flags;
        g->gopt_epoch = g->opt_epoch;
    }
    e = cudaEventRecord(g->join[0], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g->gstream, g->join[0], 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(g->gexec, g->gstream);
    if (e == cudaSuccess) g_launches.fetch_add(g->gkernels);
    if (e == cudaSuccess) e = cudaEventRecord(g->join[1], g->gstream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, g->join[1], 0);
    if (e != cudaSuccess) return cuda_status(e, "graph launch");
    return KCORE_OK;
}

kcore_status kcore_run(kcore_graph* g, int32_t* coreness_out, uint32_t flags, void* cuda_stream) {
    if (!g) return fail(KCORE_ERR_INVALID, "graph is NULL");
    const int64_t n = g->csr.n;
    if (n > 0 && !coreness_out) return fail(KCORE_ERR_INVALID, "coreness_out is NULL");
    if ((flags & KCORE_GRAPH) && !(flags & KCORE_OUT_DEVICE))
        return fail(KCORE_ERR_INVALID, "KCORE_GRAPH needs a device output (KCORE_OUT_DEVICE)");
    if (g->pending) wait_run(g);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (flags & KCORE_SYNC_MODE) {
        kcore_status s = ensure_sync_buffers(g, st);
        if (s != KCORE_OK) return s;
    }
    kcore_status s = (flags & KCORE_GRAPH) ? graph_run(g, coreness_out, flags, st)
                                          : enqueue_run(g, coreness_out, flags, st, false);
    if (s != KCORE_OK) return s;
    g->pending = true;
    g->ran = true;
    if (flags & KCORE_ASYNC) return KCORE_OK;
    return wait_run(g);
}

kcore_status kcore_run_from(kcore_graph* g, const int32_t* start, const int32_t* frontier,
                            int64_t nfrontier, int32_t* coreness_out, uint32_t flags,
                            void* cuda_stream) {
    if (!g) return fail(KCORE_ERR_INVALID, "graph is NULL");
    const int64_t n = g->csr.n;
    if (n > 0 && (!coreness_out || !start)) return fail(KCORE_ERR_INVALID, "start or coreness_out is NULL");
    if (nfrontier < 0 || (nfrontier > 0 && !frontier))
        return fail(KCORE_ERR_INVALID, "frontier is NULL or nfrontier < 0");
    if (flags & KCORE_GRAPH) return fail(KCORE_ERR_INVALID, "KCORE_GRAPH is not available with a warm start");
    if (g->pending) wait_run(g);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (flags & KCORE_SYNC_MODE) {
        kcore_status s = ensure_sync_buffers(g, st);
        if (s != KCORE_OK) return s;
    }
    WarmStart w;
    int *tmp_start = nullptr, *tmp_front = nullptr;
    kcore_status s = KCORE_OK;
    if (flags & KCORE_IN_DEVICE) {
        w.start = start;
        w.frontier = frontier;
    } else {
        s = upload(start, (size_t)n, st, &tmp_start);
        if (s == KCORE_OK && frontier) s = upload(frontier, (size_t)nfrontier, st, &tmp_front);
        w.start = tmp_start;
        w.frontier = frontier ? tmp_front : nullptr;
    }
    w.nf = frontier ? nfrontier : 0;
    int *map_start = nullptr, *map_front = nullptr;
    if (s == KCORE_OK && g->relabeled && n > 0) {  // the caller's ids -> the renumbered ones
        cudaError_t e = pool_alloc((void**)&map_start, sizeof(int) * n, st);
        if (e == cudaSuccess && w.frontier)
            e = pool_alloc((void**)&map_front, sizeof(int) * std::max<long long>(w.nf, 1), st);
        if (e == cudaSuccess)
            e = launch_relabel_start(w.start, w.frontier, w.nf, n, g->old_of_new, g->new_of_old,
                                     map_start, map_front, st);
        if (e != cudaSuccess) s = cuda_status(e, "warm start renumbering");
        w.start = map_start;
        if (w.frontier) w.frontier = map_front;
    }
    if (s == KCORE_OK && n > 0) s = enqueue_run(g, coreness_out, flags, st, false, w);
    if (tmp_start) cudaFreeAsync(tmp_start, st);
    if (tmp_front) cudaFreeAsync(tmp_front, st);
    if (map_start) cudaFreeAsync(map_start, st);
    if (map_front) cudaFreeAsync(map_front, st);
    if (s != KCORE_OK) return s;
    if (n == 0) return KCORE_OK;
    g->pending = true;
    g->ran = true;
    if (flags & KCORE_ASYNC) return KCORE_OK;
    return wait_run(g);
}

kcore_status kcore_wait(kcore_graph* g) {
    if (!g) return fail(KCORE_ERR_INVALID, "graph is NULL");
    return wait_run(g);
}

kcore_status kcore_graph_info(const kcore_graph* g, int64_t* n, int64_t* nnz,
                              int32_t* row_ptr_bytes) {
    if (!g) return fail(KCORE_ERR_INVALID, "graph is NULL");
    if (n) *n = g->csr.n;
    if (nnz) *nnz = g->csr.nnz;
    if (row_ptr_bytes) *row_ptr_bytes = g->csr.off_bytes;
    return KCORE_OK;
}

kcore_status kcore_copy_csr(const kcore_graph* g, void* row_ptr_out, int32_t* col_idx_out,
                            uint32_t flags) {
    if (!g) return fail(KCORE_ERR_INVALID, "graph is NULL");
    const cudaMemcpyKind kind =
        (flags & KCORE_OUT_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    DevCsr c = g->csr;
    if (g->relabeled) {
        // the caller's ids: the renumbered entries mapped back and cleaned
        // again (sorted build, no renumbering); rare, so not kept
        std::string err;
        int *src = nullptr, *dst = nullptr;
        cudaError_t ce = pool_alloc((void**)&src, sizeof(int) * std::max<int64_t>(g->csr.nnz, 1), 0);
        if (ce == cudaSuccess) ce = pool_alloc((void**)&dst, sizeof(int) * std::max<int64_t>(g->csr.nnz, 1), 0);
        if (ce == cudaSuccess)
            ce = launch_relabel_unmap(g->csr.row_ptr, g->csr.off_bytes, g->csr.col, g->csr.n, g->csr.nnz,
                                      g->old_of_new, src, dst, 0);
        kcore_status s = ce == cudaSuccess ? KCORE_OK : cuda_status(ce, "kcore_copy_csr");
        c = DevCsr();
        if (s == KCORE_OK) {
            s = clean_from_coo(g->csr.n, g->csr.nnz, src, dst, g->csr.off_bytes, 1, -1, 0, &c, nullptr,
                               nullptr, &err);
            if (s != KCORE_OK) set_error(err);
        }
        if (src) cudaFreeAsync(src, 0);
        if (dst) cudaFreeAsync(dst, 0);
        if (s == KCORE_OK && cudaStreamSynchronize(0) != cudaSuccess) s = cuda_status(cudaGetLastError(), "sync");
        if (s != KCORE_OK) {
            dfree(c.row_ptr, 0);
            dfree(c.col, 0);
            return s;
        }
        c.nnz = g->csr.nnz;
    }
    cudaError_t e = cudaSuccess;
    if (row_ptr_out) e = cudaMemcpy(row_ptr_out, c.row_ptr, (size_t)c.off_bytes * (c.n + 1), kind);
    if (e == cudaSuccess && col_idx_out && c.nnz)
        e = cudaMemcpy(col_idx_out, c.col, sizeof(int) * c.nnz, kind);
    if (g->relabeled) {
        dfree(c.row_ptr, 0);
        dfree(c.col, 0);
        cudaStreamSynchronize(0);
    }
    if (e != cudaSuccess) return cuda_status(e, "kcore_copy_csr");
    return KCORE_OK;
}

kcore_status kcore_stats(kcore_graph* g, kcore_run_stats* out) {
    if (!g || !out) return fail(KCORE_ERR_INVALID, "NULL argument");
    memset(out, 0, sizeof(*out));
    out->n = g->csr.n;
    out->nnz = g->csr.nnz;
    out->row_ptr_bytes = g->csr.off_bytes;
    out->ms_create = g->ms_create;
    out->block = g->opt.block;
    if (!g->ran) return KCORE_OK;
    kcore_status rs = wait_run(g);
    const SweepCtl& c = *g->hctl;
    out->status = rs;
    out->sweeps = c.sweep;
    out->tail_sweeps = c.tail_sweeps;
    out->evaluated = (int64_t)c.tot[kAccEvaluated];
    out->edges_scanned = (int64_t)c.tot[kAccDegsum];
    out->updates = (int64_t)c.tot[kAccUpdates];
    out->pushes = (int64_t)c.tot[kAccPushes];
    out->entries_read = (int64_t)(c.tot[kAccDegsum] - c.tot[kAccSkipped]);
    out->decrease = (int64_t)c.tot[kAccDec];
    out->bytes_algorithmic = out->evaluated * (2LL * g->csr.off_bytes + 4) +
                             8LL * out->entries_read + 4LL * out->updates +
                             16LL * out->n + 3LL * ((out->n + 31) / 32) * 4;  // a2 + a6
    out->grid = g->last_grid;
    cudaEventElapsedTime(&out->ms_sweep, g->ev[EV_S0], g->ev[EV_S1]);
    cudaEventElapsedTime(&out->ms_run, g->ev[EV_R0], g->ev[EV_R1]);
    return KCORE_OK;
}

// Copies the first min(cap, recorded) rows of the device trace to the host.
static kcore_status trace_rows(kcore_graph* g, int64_t cap, std::vector<long long>* rows,
                               long long* count) {
    *count = 0;
    if (!g->ran) return KCORE_OK;
    wait_run(g);
    const long long n = std::min<long long>({(long long)cap, g->hctl->sweep, g->max_trace});
    if (n <= 0) return KCORE_OK;
    rows->resize((size_t)(kTraceCols * n));
    cudaError_t e = cudaMemcpy(rows->data(), g->trace, sizeof(long long) * kTraceCols * n,
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e, "kcore_sweep_trace");
    *count = n;
    return KCORE_OK;
}

kcore_status kcore_sweep_trace(kcore_graph* g, int64_t* frontier, int64_t* degsum,
                               int64_t* updates, int64_t* start_ns, int64_t cap, int64_t* count) {
    if (!g) return fail(KCORE_ERR_INVALID, "graph is NULL");
    if (count) *count = 0;
    std::vector<long long> h;
    long long n = 0;
    kcore_status s = trace_rows(g, cap, &h, &n);
    if (s != KCORE_OK) return s;
    for (long long i = 0; i < n; i++) {
        const long long* r = h.data() + kTraceCols * i;
        if (frontier) frontier[i] = r[kTrFrontier];
        if (degsum) degsum[i] = r[kTrDegsum];
        if (updates) updates[i] = r[kTrUpdates];
        if (start_ns) start_ns[i] = r[kTrStart] - h[kTrStart];
    }
    if (count) *count = n;
    return KCORE_OK;
}

kcore_status kcore_sweep_detail(kcore_graph* g, int64_t* entries_read, int64_t* decrease,
                                int64_t cap, int64_t* count) {
    if (!g) return fail(KCORE_ERR_INVALID, "graph is NULL");
    if (count) *count = 0;
    std::vector<long long> h;
    long long n = 0;
    kcore_status s = trace_rows(g, cap, &h, &n);
    if (s != KCORE_OK) return s;
    for (long long i = 0; i < n; i++) {
        const long long* r = h.data() + kTraceCols * i;
        if (entries_read) entries_read[i] = r[kTrRead];
        if (decrease) decrease[i] = r[kTrDec];
    }
    if (count) *count = n;
    return KCORE_OK;
}

kcore_status kcore_sweep_tiers(kcore_graph* g, int64_t* frontier, int64_t* degsum, int64_t cap,
                               int64_t* count) {
    if (!g) return fail(KCORE_ERR_INVALID, "graph is NULL");
    if (count) *count = 0;
    std::vector<long long> h;
    long long n = 0;
    kcore_status s = trace_rows(g, cap, &h, &n);
    if (s != KCORE_OK) return s;
    for (long long i = 0; i < n; i++) {
        const long long* r = h.data() + kTraceCols * i;
        const long long w = r[kTrDegW], c = r[kTrDegC];
        if (frontier) {
            frontier[3 * i] = r[kTrF0];
            frontier[3 * i + 1] = r[kTrF1];
            frontier[3 * i + 2] = r[kTrF2];
        }
        if (degsum) {
            degsum[3 * i] = r[kTrDegsum] - w - c;
            degsum[3 * i + 1] = w;
            degsum[3 * i + 2] = c;
        }
    }
    if (count) *count = n;
    return KCORE_OK;
}

void kcore_destroy(kcore_graph* g) { release(g); }

}  // extern "C"
