// host_util.h -- host-side helpers shared by the C-ABI files (errors, device
// buffers).  Not part of the public interface.
#pragma once

#include <cuda_runtime.h>

#include <new>
#include <stdexcept>
#include <string>

#include "mjp.h"

namespace mjp {

// Message of the last failure on the calling thread (defined in api.cu).
std::string& last_error();

inline int fail(int code, const std::string& msg) {
  last_error() = msg;
  return code;
}

// Status of the exception being handled: no C++ exception crosses the C ABI.
// Every entry point returning a status ends in a handler that calls this; a
// failed host allocation (std::bad_alloc, std::length_error) is MJP_ERR_ALLOC,
// anything else MJP_ERR_ARG.  Call only inside a catch block.
inline int exception_status() noexcept {
  int code = MJP_ERR_ARG;
  const char* msg = "unexpected host-side exception";
  try {
    throw;
  } catch (const std::bad_alloc&) {
    code = MJP_ERR_ALLOC;
    msg = "host allocation failed";
  } catch (const std::length_error&) {
    code = MJP_ERR_ALLOC;
    msg = "host allocation too large";
  } catch (...) {
  }
  try {
    last_error() = msg;
  } catch (...) {
  }
  return code;
}

#define MJP_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      cudaGetLastError();                                                                \
      return ::mjp::fail(MJP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                                    \
  } while (0)

// Grow-only device buffer.  Growing synchronises the device first so that no
// queued kernel still uses the old allocation.
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  int ensure(size_t bytes) {
    if (bytes <= cap) return MJP_OK;
    cudaDeviceSynchronize();
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    if (cudaMalloc(&p, bytes < 256 ? 256 : bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(MJP_ERR_ALLOC, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    cap = bytes < 256 ? 256 : bytes;
    return MJP_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  template <typename T>
  T* as() const {
    return reinterpret_cast<T*>(p);
  }
};

}  // namespace mjp
