// noalloc.cu -- the brute-force sum for callers that cannot allocate device
// memory.
//
// Some callers must not allocate GPU memory while they run: code executed
// while a CUDA graph is being captured (an allocation there breaks the
// capture), hosts that hand the library a fixed memory budget or their own
// allocator and forbid driver allocations behind their back, and
// latency-critical loops where a cudaMalloc (which may synchronise the
// device) is not acceptable.  dfgt_sum_bruteforce_static serves them: it
// runs the split-reference brute force of bruteforce.cu, but its slice
// partials live in the file-scope array below instead of context-owned
// scratch, so the call itself allocates nothing.
#include <mutex>

#include "internal.hpp"

namespace {

// 16 MiB of float64 slice partials, reserved on every device that loads the
// library and held until the process exits.
constexpr size_t kStaticScratchDoubles = size_t(1) << 21;
static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// Device address of the array on the current device, looked up once per
// device (with that device current) and cached for the life of the process;
// a device reset (cudaDeviceReset or a primary-context reset) leaves the
// cached address stale, so the entry point must not be used after one.
cudaError_t static_scratch(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" dfgt_status dfgt_sum_bruteforce_static(const float* q_dev, int64_t nq, const float* r_dev,
                                                  int64_t nr, int d, const double* h_host, int nh,
                                                  double* G_dev, void* cuda_stream) {
  if (!q_dev || !r_dev || !G_dev || !h_host || nq < 1 || nr < 1 || nq > (1 << 30) ||
      nr > (1 << 30) || d < 1 || d > dfgt::kMaxD || nh < 1 || nh > 1024)
    return DFGT_EINVAL;
  for (int i = 0; i < nh; ++i)
    if (!(h_host[i] > 0.0) || !(h_host[i] < INFINITY)) return DFGT_EINVAL;
  long long launches = 0;
  const cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  int slices = dfgt::bruteforce_slices((int)nq, (int)nr);
  if (slices <= 1) {
    // enough queries to fill the GPU: one pass writes G_dev directly and
    // needs no scratch, so the array's limit does not apply
    const cudaError_t e = dfgt::launch_bruteforce_split(q_dev, (int)nq, r_dev, (int)nr, d, h_host, nh, G_dev,
                                                        1, nullptr, stream, &launches);
    return e == cudaSuccess ? DFGT_OK : DFGT_ECUDA;
  }
  // split references: the partials of at least two slices must fit the array
  const size_t per_slice = (size_t)nh * (size_t)nq;
  if (2 * per_slice > kStaticScratchDoubles) return DFGT_ECAPACITY;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return DFGT_ECUDA;
  double* scratch = nullptr;
  if (static_scratch(device, &scratch) != cudaSuccess) return DFGT_ECUDA;
  const size_t fit = kStaticScratchDoubles / per_slice;
  if ((size_t)slices > fit) slices = (int)fit;
  // every partial that the reduction reads is written by its slice in this
  // call, so nothing needs clearing between calls
  const cudaError_t e = dfgt::launch_bruteforce_split(q_dev, (int)nq, r_dev, (int)nr, d, h_host, nh, G_dev,
                                                      slices, scratch, stream, &launches);
  return e == cudaSuccess ? DFGT_OK : DFGT_ECUDA;
}
