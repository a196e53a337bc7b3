// Host-side helper shared by the C ABI translation units (dba_api.cu, dba_block.cu,
// dba_mlp.cu).  Not installed; not part of the public ABI.
#pragma once

#include <exception>
#include <new>
#include <string>

#include "../../include/dba.h"

namespace dba {

// Host allocation failures still to be injected on the calling thread (fault injection for
// tests, set by dba_inject_host_alloc_failure): while positive, each guarded entry point
// takes one and fails as if its first host allocation had thrown.
inline int& injected_host_alloc_failures() {
  static thread_local int n = 0;
  return n;
}

// Runs an entry point's whole body so that no C++ exception crosses the C ABI: a failed
// host allocation (or another exhausted host resource, such as a thread that cannot
// start) becomes DBA_ENOMEM with a message in *err (when err is not null).
template <typename F>
dba_status guarded(std::string* err, F&& body) {
  try {
    int& inject = injected_host_alloc_failures();
    if (inject > 0) {
      --inject;
      throw std::bad_alloc();
    }
    return body();
  } catch (const std::bad_alloc&) {
    if (err) try { *err = "out of host memory"; } catch (...) {}
  } catch (const std::exception& e) {
    if (err) try { *err = std::string("host resources exhausted: ") + e.what(); } catch (...) {}
  } catch (...) {
    if (err) try { *err = "unexpected host exception"; } catch (...) {}
  }
  return DBA_ENOMEM;
}
}  // namespace dba
