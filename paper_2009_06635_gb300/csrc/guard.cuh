// guard.cuh -- keeps C++ exceptions inside the library (host code only).
#pragma once
#include <exception>
#include <new>

#include "pdf_gb300.h"

namespace pdfgb {

int set_error(int code, const char *fmt, ...);

// Runs the body of a C entry point so that no C++ exception crosses the C
// ABI: a failed host allocation returns PDF_ERR_ALLOC, any other exception
// PDF_ERR_ARG, each with the message set.
template <typename F>
int guarded(const char *fn, F &&body) noexcept {
  try {
    return body();
  } catch (const std::bad_alloc &) {
    return set_error(PDF_ERR_ALLOC, "%s: host allocation failed", fn);
  } catch (const std::exception &e) {
    return set_error(PDF_ERR_ARG, "%s: %s", fn, e.what());
  } catch (...) {
    return set_error(PDF_ERR_ARG, "%s: unexpected exception", fn);
  }
}

}  // namespace pdfgb
