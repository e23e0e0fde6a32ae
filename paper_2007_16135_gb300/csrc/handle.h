// Handle state that translation units other than api.cu may use.
#pragma once

#include "../../include/twed.h"

namespace twed {
namespace detail {
// Records `msg` as the handle's last error and returns `st`.
twed_status_t set_error(twed_handle_t h, twed_status_t st, const char* msg);
int handle_sms(twed_handle_t h);
int handle_device(twed_handle_t h);
}  // namespace detail
}  // namespace twed
