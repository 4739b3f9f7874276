// No C++ exception crosses the C ABI: each extern "C" entry point runs its
// body inside abi_guard, which turns a failed host allocation into
// CCS_ERR_OOM and any other exception into CCS_ERR_INVALID_ARG, passing the
// code and a message to `on_error` (which records the message and returns
// the code).
#pragma once

#include <exception>
#include <new>

#include "ccs.h"

namespace ccs {

template <class OnError, class Body>
int abi_guard(OnError&& on_error, Body&& body) noexcept {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return on_error(CCS_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return on_error(CCS_ERR_INVALID_ARG, e.what());
  } catch (...) {
    return on_error(CCS_ERR_INVALID_ARG, "unexpected host error");
  }
}

}  // namespace ccs
