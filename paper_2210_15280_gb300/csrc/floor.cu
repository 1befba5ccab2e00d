// floor.cu -- the dependency-depth floor of the substitutions (ilu_step_floor).
//
// A substitution is a chain of steps (hyperplanes of Alg. 2's dependency
// graph, or steps of a packed schedule): a point of step s needs values of
// steps s-1..s-3, so no step can start before the previous one's results are
// visible.  The floor kernel times the shortest body such a step can have on
// this GPU: each warp of one CTA reads three neighbour values of earlier
// steps from a shared-memory ring, applies a chain of seven dependent FMAs
// (the substitution's sum; the row polynomials can be evaluated ahead and are
// not part of it), writes its value back and meets the other warps at a block
// barrier.  Cycles per step times the number of steps is a depth bound no
// schedule of the substitution can beat with this synchronisation.
#include <cuda_runtime.h>

#include <string>

#include "../../include/ilu.h"
#include "hooks.h"

namespace {

constexpr int kRingSteps = 32;

__global__ void step_floor_kernel(int steps, long long *cycles, float *sink) {
  extern __shared__ float ring[];  // [kRingSteps][blockDim.x]
  const int n = blockDim.x, i = threadIdx.x;
  for (int k = i; k < kRingSteps * n; k += n) ring[k] = 1e-3f * (float)(k % 17);
  __syncthreads();
  float v = 0.5f;
  const float l = 0.25f;
  const int j1 = (i + 33) % n, j2 = (i + 97) % n;  // neighbours in other warps
  long long t0 = clock64();
  for (int s = 3; s < steps + 3; ++s) {
    const float a = ring[((s - 1) & (kRingSteps - 1)) * n + j1];
    const float b = ring[((s - 2) & (kRingSteps - 1)) * n + j2];
    const float c = ring[((s - 3) & (kRingSteps - 1)) * n + i];
    float acc = v;
    acc = fmaf(-l, a, acc);
    acc = fmaf(-l, b, acc);
    acc = fmaf(-l, c, acc);
    acc = fmaf(-l, a, acc);
    acc = fmaf(-l, b, acc);
    acc = fmaf(-l, c, acc);
    acc = fmaf(-l, v, acc);
    v = acc;
    ring[(s & (kRingSteps - 1)) * n + i] = acc;
    __syncthreads();
  }
  const long long t1 = clock64();
  if (i == 0) *cycles = t1 - t0;
  if (v == 1234.5f) sink[i] = v;  // keeps the chain alive
}

}  // namespace

extern "C" ilu_status ilu_step_floor(int device, int threads, int steps, double *cycles_per_step) {
  if (!cycles_per_step || threads < 32 || threads > 1024 || (threads & 31) || steps < 1) {
    ilu::set_last_error("ilu_step_floor: bad argument");
    return ILU_EINVAL;
  }
  ilu::DeviceRestore keep_device;
  if (cudaSetDevice(device) != cudaSuccess) {
    ilu::set_last_error("ilu_step_floor: no such device");
    return ILU_ENODEV;
  }
  long long *d_cyc = nullptr;
  float *d_sink = nullptr;
  cudaError_t e = cudaMalloc(&d_cyc, sizeof(long long));
  if (e == cudaSuccess) e = cudaMalloc(&d_sink, sizeof(float) * threads);
  const size_t smem = sizeof(float) * kRingSteps * threads;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(step_floor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  long long best = -1;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {  // the first run warms up
    step_floor_kernel<<<1, threads, smem>>>(steps, d_cyc, d_sink);
    e = cudaGetLastError();
    long long c = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&c, d_cyc, sizeof(c), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && rep > 0 && (best < 0 || c < best)) best = c;
  }
  cudaFree(d_cyc);
  cudaFree(d_sink);
  if (e != cudaSuccess) {
    ilu::set_last_error(std::string("ilu_step_floor: ") + cudaGetErrorString(e));
    return ILU_ECUDA;
  }
  *cycles_per_step = (double)best / steps;
  return ILU_OK;
}
