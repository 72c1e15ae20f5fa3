// Allocation-free symmetric eigensolver entry point (see include/ricmrcc.h,
// ricmrcc_block_eigh_noalloc).
//
// Some callers cannot allocate device memory at the moment they need this
// step: code that runs while a CUDA stream is being captured into a graph,
// services that pin their whole device-memory budget up front, or hosts whose
// allocator is owned by another runtime.  This entry point therefore keeps its
// working memory in one fixed array that lives in the library image on every
// device that loads the library, instead of allocating it per call.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/ricmrcc.h"
#include "kernels.h"

namespace {

// Largest block this entry point accepts, and its working memory: a copy of
// the block that the Jacobi sweeps overwrite, the rotation accumulator, and
// one int for the sweep count (2 * 1024^2 doubles + 256 bytes = 16 MiB).
constexpr int kMaxN = RICMRCC_NOALLOC_MAX_N;
constexpr int64_t kScratchDoubles = 2LL * kMaxN * kMaxN + 32;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// Device address of the scratch array, looked up once per device.  In host
// code `g_noalloc_scratch` only names a host-side stand-in; kernels must be
// given the address returned by cudaGetSymbolAddress for the current device.
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_addr[kMaxDevices] = {nullptr};

int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RICMRCC_ECUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return RICMRCC_ECUDA;
    }
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return RICMRCC_OK;
}

// Eigenvalues in ascending order from the diagonal the sweeps converged to;
// all NaN when the sweeps stopped unconverged (*sweeps < 0), which is how an
// enqueue-only call reports that outcome to its caller.
__global__ void k_sorted_diagonal(const double* __restrict__ A, int n, const int* __restrict__ sweeps,
                                  double* __restrict__ w) {
  const bool failed = *sweeps < 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    if (failed) {
      w[j] = __longlong_as_double(0x7ff8000000000000ll);
      continue;
    }
    const double x = A[(int64_t)j * n + j];
    int rank = 0;
    for (int k = 0; k < n; ++k) {
      const double y = A[(int64_t)k * n + k];
      if (y < x || (y == x && k < j)) ++rank;
    }
    w[rank] = x;
  }
}

}  // namespace

extern "C" int ricmrcc_block_eigh_noalloc(const double* A, int n, double* eigenvalues,
                                          double* eigenvectors, void* stream) {
  if (!A || !eigenvalues || !eigenvectors || n < 1) return RICMRCC_EINVAL;
  if (n > kMaxN) return RICMRCC_EINVAL;  // larger than the fixed working memory
  double* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != RICMRCC_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* work = scratch;                          // n x n copy of A (overwritten)
  double* rot = scratch + (int64_t)kMaxN * kMaxN;  // n x n rotation accumulator
  int* sweeps = reinterpret_cast<int*>(scratch + 2LL * kMaxN * kMaxN);
  // The copy overwrites everything the sweeps read; the accumulator and the
  // sweep counter are (re)initialised by the kernels themselves.
  if (cudaMemcpyAsync(work, A, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToDevice, s) !=
      cudaSuccess)
    return RICMRCC_ECUDA;
  // every status below is the one of this call's own launch
  if (run_jacobi(work, rot, n, eigenvectors, n, 0, sweeps, s) != cudaSuccess) return RICMRCC_ECUDA;
  void* args[] = {(void*)&work, &n, (void*)&sweeps, &eigenvalues};
  if (cudaLaunchKernel((const void*)k_sorted_diagonal, dim3(1), dim3(256), args, 0, s) != cudaSuccess)
    return RICMRCC_ECUDA;
  return RICMRCC_OK;
}
