// noalloc.cu -- a residual entry point that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc: code that runs inside a
// device-memory budget owned by someone else (a framework's caching
// allocator, a serving process with a fixed pool), or latency-sensitive code
// where the implicit device synchronisation of cudaMalloc/cudaFree is not
// acceptable.  ilu_residual may allocate on first use (its norm buffer);
// ilu_residual_noalloc does the same computation with its only scratch, the
// per-block partial sums of ||r||^2, in the file-scope array below.
//
// The array is shared by every call on a device and keeps the last call's
// contents; every partial sum it uses is written before it is read, so no
// clearing is needed.  Calls whose kernels overlap on the GPU (different
// streams, or several host threads) race on it: serialise them.  Every GPU
// that loads the library holds the array (1 MiB) until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/ilu.h"
#include "hooks.h"
#include "kernels.cuh"

namespace ilu {
// direct view of a handle's device data (defined in capi.cu)
const DevTet *tet_dev_view(ilu_tet t, int *device, int *precision, size_t *nnodes);
// refuses null, host-only and failed handles; otherwise holds the handle's lock
ilu_status tet_acquire(ilu_tet t, std::unique_lock<std::mutex> *lk);
void tet_mark_failed(ilu_tet t);
void set_last_error(const std::string &msg);
}  // namespace ilu

namespace {

constexpr int kMaxPartials = 131072;  // residual blocks up to level 9 (about 87,000 at level 9)
static __device__ __align__(256) double g_partials[kMaxPartials];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_addr[kMaxDevices] = {};  // device address of g_partials, per device

ilu_status fail(ilu_status s, const std::string &msg) {
  ilu::set_last_error(msg);
  return s;
}

}  // namespace

extern "C" ilu_status ilu_residual_noalloc(ilu_tet t, const void *x, const void *b, void *r, double *norm_dev,
                                           void *stream) {
  if (!t || !x || !b || !r || !norm_dev) return fail(ILU_EINVAL, "null argument");
  ilu::DeviceRestore keep_device;
  // the same refusals as every other entry point (host-only or failed
  // handle), and the handle's lock for the launches
  std::unique_lock<std::mutex> lk;
  ilu_status st = ilu::tet_acquire(t, &lk);
  if (st != ILU_OK) return st;
  int device = -1, precision = 0;
  size_t nn = 0;
  const ilu::DevTet *d = ilu::tet_dev_view(t, &device, &precision, &nn);
  if (!d || device < 0) return fail(ILU_ENODEV, "host-only handle has no device part");
  if (device >= kMaxDevices) return fail(ILU_EINVAL, "device ordinal beyond the supported range");
  const int blocks = ilu::residual_blocks(d->N);
  if (blocks > kMaxPartials)
    return fail(ILU_EINVAL, "ilu_residual_noalloc supports levels up to 9: level " + std::to_string(d->L) +
                                " needs " + std::to_string(blocks) + " partial sums, the static scratch holds " +
                                std::to_string(kMaxPartials));
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return fail(ILU_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  double *partials = nullptr;
  {
    // first call on this device: look up the array's device address (with
    // the device current); later calls reuse it
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[device]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_partials);
      if (e != cudaSuccess) return fail(ILU_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_addr[device] = static_cast<double *>(p);
    }
    partials = g_addr[device];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t elem = precision == ILU_F32 ? sizeof(float) : sizeof(double);
  e = cudaMemsetAsync(r, 0, nn * elem, s);  // the kernel writes interior entries only
  if (e != cudaSuccess) {
    ilu::tet_mark_failed(t);
    return fail(ILU_ECUDA, std::string("clear r: ") + cudaGetErrorString(e));
  }
  int used = 0;
  e = ilu::launch_residual(*d, precision == ILU_F32 ? ilu::kSweepF32 : ilu::kSweepF64, x, b, r, partials,
                           kMaxPartials, &used, s);
  if (e == cudaSuccess) e = ilu::launch_norm_finish(partials, used, norm_dev, s);
  if (e != cudaSuccess) {
    ilu::tet_mark_failed(t);
    return fail(ILU_ECUDA, std::string("residual launch: ") + cudaGetErrorString(e));
  }
  return ILU_OK;
}
