// Shared declarations between the translation units of the library.
#pragma once
#include <string>

#include "../../include/rttda.h"

namespace rttda {
// Per-thread message returned by rttda_last_error().
extern thread_local std::string g_last_error;
// Record msg as the calling thread's last error and return s.
rttda_status set_error(rttda_status s, const std::string& msg);
}  // namespace rttda
