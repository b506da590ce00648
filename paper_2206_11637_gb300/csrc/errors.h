// Per-thread error message shared by the library's translation units
// (reported by pfl_last_error).
#pragma once
#include <string>

namespace pfl_internal {
void set_error(const std::string& msg);
}
