// Host-side helpers shared by the translation units of libmsc (not part of the C ABI).
#pragma once
#include <atomic>
#include <string>

#include "../../include/msc.h"

namespace msc_rt {
// record msg as this thread's msc_last_error and return s
msc_status set_error(msc_status s, const std::string &msg);
// blocks of the persistent round kernel for a handle whose fixes share the device with
// `concurrent` other jobs: a fraction of the SMs each, so that the jobs' kernels fit at once
void share_device(msc_handle *h, int concurrent);
// device memory the library's pool keeps for reuse after handles free it (the server's budget)
void limit_cached_memory(uint64_t bytes);
// cancellation flag of the job this thread runs (nullptr: none); the fix loop checks it each
// time control returns to the host and then ends with MSC_ERR_CANCELLED
void set_cancel_flag(const std::atomic<int> *flag);
}  // namespace msc_rt
