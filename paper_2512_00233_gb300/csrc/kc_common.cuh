// Internal declarations shared by the library's CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "kcore.h"

namespace kc {

// ---------------------------------------------------------------- estimates
// Each estimate word holds the current coreness estimate in its low 30 bits
// and the vertex's degree tier (0 thread, 1 warp, 2 CTA) in the top 2 bits, so
// a push reads the tier of the neighbour from the same word it compares.
constexpr uint32_t kEstBits = 30;
constexpr uint32_t kEstMask = (1u << kEstBits) - 1u;
constexpr int kTiers = 3;
constexpr int kMedBig = 2048;      // largest degree of the warp tier (t_hi <= kMedBig)
constexpr int kHubBins = 4096;   // shared-memory histogram of the CTA tier

// Accumulator indices of per-sweep statistics.
enum {
    kAccEvaluated = 0,
    kAccDegsum = 1,   // frontier degree sum
    kAccUpdates = 2,
    kAccPushes = 3,
    kAccSkipped = 4,  // adjacency entries not read thanks to an early exit
    kAccDec = 5,      // sum of estimate decreases
    kAccDegW = 6,     // frontier degree sum of the warp tier
    kAccDegC = 7,     // frontier degree sum of the CTA tier
    kAccN = 8
};
// Columns of the per-sweep trace (kTrF0..2: frontier size per degree tier).
enum { kTrFrontier = 0, kTrDegsum, kTrUpdates, kTrStart, kTrRead, kTrDec, kTrF0, kTrF1, kTrF2,
       kTrDegW, kTrDegC, kTraceCols };

// Control block of the persistent sweep kernel (device memory).  Counter slot
// s % 4 holds the frontier counts of sweep s; sweep s pushes into slot
// (s+1) % 4, reads the size of F_{s-1} from slot (s-1) % 4 to clear its
// membership bits, and slot (s+2) % 4 is reset at the start of sweep s.
constexpr int kSlots = 4;
constexpr int kParities = 3;     // frontier lists / membership bitmaps
struct SweepCtl {
    unsigned int bar_count;          // grid barrier arrivals
    unsigned int bar_gen;            // grid barrier generation
    int status;                      // 0 or a negative kcore_status
    int done;                        // 1 once the frontier is empty
    long long sweep;                 // next sweep to run (resume point)
    long long tail_sweeps;           // sweeps run by one CTA
    unsigned int fcnt[kSlots][4];    // frontier size per tier
    unsigned int cursor[kSlots][4];  // work cursor per tier
    unsigned int ucnt[kSlots];       // synchronous mode: updates this sweep
    unsigned long long acc[kSlots][kAccN];
    unsigned long long tot[kAccN];
    unsigned int tail_epoch;         // bumped when the single-CTA tail hands over
    int tail_exit;                   // 1: launch over; 0: resume all CTAs
    long long resume_sweep;
};

// Arguments of one persistent sweep launch.  Sweep s reads frontier list and
// membership bitmap s % 3, pushes into (s+1) % 3 and clears (s+2) % 3.
struct SweepArgs {
    const void* row_ptr;             // int32 or int64 per off64
    const int* col;
    uint32_t* est;
    const int* init_list;            // frontier of sweep 0 (tiers contiguous), or null
    int* list[kParities];            // frontier lists
    uint32_t* bitmap[kParities];     // frontier membership
    int* upd_list;                   // synchronous mode: updated vertices
    int* upd_val;                    // synchronous mode: their new (then old) values
    long long tier_off[kTiers];      // start of each tier inside a list
    SweepCtl* ctl;
    long long* trace;                // [max_trace][kTraceCols]: see the kTr* columns
    long long max_trace;
    long long first_sweep;           // sweep index at which this launch starts
    long long max_sweeps;            // NOT_CONVERGED at this sweep index
    long long stop_sweep;            // this launch ends before this sweep index
    long long timeout_ns;            // budget of every bounded wait
    long long words;                 // 32-bit words per bitmap
    int n;
    int t_lo, t_hi;
    int low_chunk, med_chunk;
    int tail_max;
    int sync_mode, refined;
    int off64;
    // Optional steps folded into the launch (null: done by the caller).
    const uint32_t* est0;            // a2: est <- est0, F_0 = every vertex, with init_cnt per tier
    unsigned init_cnt[kTiers];
    int* out;                        // a6: out[v] = est[v] (coreness), at the end of the run
    const int* perm;                 // relabeled graph: out[v] = est[perm[v]], v in the caller's ids
};

// Launch the persistent sweep kernel (cooperative launch).  `grid` 0 picks the
// occupancy maximum; the grid used is returned.
// Warm start of a run: estimates from `start` (capped at the degree) and, with
// a frontier list, F_0 built in bitmap[0] / list[0] with counts in ctl.
cudaError_t launch_warm_init(const SweepArgs& a, const void* row_ptr, const uint32_t* est0,
                             const int* start, const int* frontier, long long nf, cudaStream_t st);
cudaError_t launch_ctl_init(SweepCtl* ctl, const long long tier_cnt[kTiers], cudaStream_t st);
cudaError_t launch_sweep(const SweepArgs& a, int block, int grid_req, int ctas_per_sm,
                         cudaStream_t st, int* grid_used);

// Largest cooperative grid for a block size.
cudaError_t sweep_max_grid(int block, int t_lo, int t_hi, int off64, int* grid);

// ---------------------------------------------------------------- CSR cleaning
struct DevCsr {
    int64_t n = 0, nnz = 0;  // nnz = -1 until row_ptr[n] has been read back
    int off_bytes = 4;
    void* row_ptr = nullptr;
    int* col = nullptr;
};

// Raw samples (device) -> clean CSR (device, allocated here).  sort_mode 1:
// the sorted build (one radix sort of all entries); -1: rows counted,
// scattered and sorted one by one; 0: chosen from the row sizes.  relabel
// (kcore_options.relabel; -1 when new_of_old / old_of_new are null): when the
// build renumbers the vertices by degree, the CSR is in the new ids (rows
// sorted by them) and *new_of_old / *old_of_new (n each, allocated here) give
// the numbering; otherwise both stay null.  Returns a kcore_status; on error
// *err names the problem.
kcore_status clean_from_coo(int64_t n, int64_t samples, const int* src, const int* dst,
                            int off_bytes, int sort_mode, int relabel, cudaStream_t st, DevCsr* out,
                            int** new_of_old, int** old_of_new, std::string* err);
kcore_status clean_from_csr(int64_t n, const void* row_ptr, int in_off_bytes, const int* col,
                            int64_t nnz, int off_bytes, cudaStream_t st, DevCsr* out,
                            std::string* err);
// Checks an already-clean device CSR (ids in range, rows strictly increasing,
// no loops, offsets monotone).  KCORE_OK or ERR_INVALID.
kcore_status check_clean_csr(int64_t n, const void* row_ptr, int off_bytes, const int* col,
                             int64_t nnz, cudaStream_t st, std::string* err);

// Tier split: est0 = (tier << 30) | degree, and the list of all vertices with
// tiers contiguous and ids ascending inside each tier.  Enqueued only: the
// tier boundaries, row_ptr[n] and a flag (a degree >= 2^30) land in *dout
// (device memory) for the caller's next wait.
struct TierOut {
    unsigned int bound[kTiers + 1];
    int bad;
    long long nnz;
};
kcore_status tier_split(int64_t n, const void* row_ptr, int off_bytes, int t_lo, int t_hi,
                        uint32_t* est0, int* init_list, TierOut* dout, cudaStream_t st,
                        std::string* err);

// The entries of a renumbered CSR as samples in the caller's ids: src[p] the
// old id of entry p's row, dst[p] the old id of its column (nnz each).
cudaError_t launch_relabel_unmap(const void* row_ptr, int off_bytes, const int* col, long long n,
                                 long long nnz, const int* old_of_new, int* src, int* dst,
                                 cudaStream_t st);

// start2[i] = start[old_of_new[i]] (i < n); frontier2[j] = new_of_old[frontier[j]]
// for ids in [0, n) (others copied as they are, so that they are still refused).
cudaError_t launch_relabel_start(const int* start, const int* frontier, long long nf, long long n,
                                 const int* old_of_new, const int* new_of_old, int* start2,
                                 int* frontier2, cudaStream_t st);

// Exclusive scan helper (device), out has N+1 entries when total_slot.
cudaError_t scan_u32_to_u64(const uint32_t* in, unsigned long long* out, long long N,
                            cudaStream_t st);

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount,
// cached per device ordinal); grid-stride kernels size their grids from it.
// 1 if the query fails (the launch that follows reports the error).
int sm_count();

// Number of kernels this library has launched in the process (all devices).
void count_launch();
long long launches();

// Device memory from the library's stream-ordered pool (OOM reported apart
// from other CUDA errors), and recycled small pinned host blocks.
kcore_status dmalloc(void** p, size_t bytes, std::string* err, cudaStream_t st = 0);
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st);  // free with cudaFreeAsync
void dfree(void* p, cudaStream_t st = 0);
constexpr size_t kPinnedBlock = 4096;
// Test hook (kcore_test.h): true when this allocation request is the one the
// injector was armed to fail.  Every allocation site asks once per request.
bool alloc_fault();
cudaError_t pinned_get(void** p, size_t bytes);
void pinned_put(void* p);

}  // namespace kc
