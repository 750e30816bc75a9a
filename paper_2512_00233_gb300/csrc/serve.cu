// Batch engine placeholder (replaced by the continuous-batching engine).
#include <cstring>
#include "kc_common.cuh"

namespace kc { kcore_status fail(kcore_status s, const std::string& msg); }

struct kcore_batch { int unused; };

extern "C" {
void kcore_default_serve_options(kcore_serve_options* o) { if (o) { memset(o, 0, sizeof(*o)); o->struct_size = sizeof(*o); } }
kcore_status kcore_batch_create(const kcore_serve_options*, kcore_batch** out) { if (out) *out = nullptr; return kc::fail(KCORE_ERR_INVALID, "batch engine not built"); }
kcore_status kcore_submit(kcore_batch*, int64_t, const void*, int32_t, const int32_t*, uint32_t, uint64_t*) { return kc::fail(KCORE_ERR_INVALID, "batch engine not built"); }
kcore_status kcore_submit_coo(kcore_batch*, int64_t, int64_t, const int32_t*, const int32_t*, uint32_t, uint64_t*) { return kc::fail(KCORE_ERR_INVALID, "batch engine not built"); }
kcore_status kcore_poll(kcore_batch*, uint64_t, int32_t*, int64_t) { return kc::fail(KCORE_ERR_INVALID, "batch engine not built"); }
kcore_status kcore_cancel(kcore_batch*, uint64_t) { return kc::fail(KCORE_ERR_INVALID, "batch engine not built"); }
kcore_status kcore_batch_step(kcore_batch*, int64_t*) { return kc::fail(KCORE_ERR_INVALID, "batch engine not built"); }
kcore_status kcore_batch_stats_get(kcore_batch*, kcore_batch_stats*) { return kc::fail(KCORE_ERR_INVALID, "batch engine not built"); }
void kcore_batch_destroy(kcore_batch*) {}
}
