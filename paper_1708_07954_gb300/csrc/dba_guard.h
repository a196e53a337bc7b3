// Host-side helper shared by the C ABI translation units (dba_api.cu, dba_block.cu,
// dba_mlp.cu).  Not installed; not part of the public ABI.
#pragma once

#include <exception>
#include <new>
#include <string>

#include "../../include/dba.h"

namespace dba {

// Runs an entry point's body so that no C++ exception crosses the C ABI: a failed host
// allocation (or another exhausted host resource, such as a thread that cannot start)
// becomes DBA_ENOMEM with a message in *err (when err is not null).
template <typename F>
dba_status guarded(std::string* err, F&& body) {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    if (err) try { *err = "out of host memory"; } catch (...) {}
  } catch (const std::exception& e) {
    if (err) try { *err = std::string("host resources exhausted: ") + e.what(); } catch (...) {}
  }
  return DBA_ENOMEM;
}
}  // namespace dba
