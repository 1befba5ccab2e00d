// hooks.h -- what entry-point files other than capi.cu may do with a tet
// handle (capi.cu defines these).  Each call takes the handle's lock.
// Also the device guard every entry point declares first.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "../../include/ilu.h"

namespace ilu {
// n sweeps of Alg. 2 on device vectors, asynchronous on s
ilu_status tet_sweeps(ilu_tet t, void *x, const void *b, int n, cudaStream_t s);
// r = b - A x on the interior in the handle's vector type (r's boundary
// entries untouched); with d_norm (device) also ||r||_2
ilu_status tet_residual(ilu_tet t, const void *x, const void *b, void *r, double *d_norm, cudaStream_t s);
// synchronise s and report a bounded wait that ran out (ILU_ETIMEOUT)
ilu_status tet_check(ilu_tet t, cudaStream_t s);
void set_last_error(const std::string &msg);

// Entry points switch the calling thread to a handle's device; this guard,
// declared first in each of them, puts the caller's current device back on
// every return path.
struct DeviceRestore {
  int prev = -1;
  DeviceRestore() {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  }
  ~DeviceRestore() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
  DeviceRestore(const DeviceRestore &) = delete;
  DeviceRestore &operator=(const DeviceRestore &) = delete;
};
}  // namespace ilu
