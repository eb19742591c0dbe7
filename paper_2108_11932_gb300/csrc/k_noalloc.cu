// Allocation-free variant of the exact kernel-matrix product (tlr_kernel_matvec).
//
// tlr_kernel_matvec copies the caller's host points into device memory that
// the library allocates for the duration of the call.  Some callers cannot let
// a library allocate device memory: code that runs under a memory manager
// which owns the whole device heap, processes that must not trigger
// cudaMalloc's implicit synchronization, or callers without a tlr_ctx.  This
// variant stages the points in a fixed, file-scope device array instead, so a
// call allocates nothing and needs no context; the caller still owns X and Y.
//
// Cost of that choice: every GPU that loads the library keeps the array
// (kMaxPointDoubles doubles, 3 MiB) until the process exits, calls share it
// (the last call's points stay in it), and calls whose work overlaps on the
// GPU (different streams, or several host threads) race on it.
#include <mutex>

#include "common.h"

namespace {

// N * d doubles at most: 131072 points in three dimensions.
constexpr int64_t kMaxPointDoubles = 3 * 131072;
static __device__ __align__(256) double g_points[kMaxPointDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_points_addr[kMaxDevices] = {nullptr};

// Device address of g_points on the current device.  In host code the name
// g_points is only a host-side stand-in for the symbol, so the address must be
// asked for once per device, with that device current.
cudaError_t points_address(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_points_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_points);
    if (e != cudaSuccess) return e;
    g_points_addr[dev] = static_cast<double*>(p);
  }
  *out = g_points_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" tlr_status tlr_kernel_matvec_noalloc(void* cuda_stream, const double* points_host, int64_t N,
                                                int d, const tlr_kernel* kern, int nrhs, const double* X,
                                                int64_t ldx, double* Y, int64_t ldy) {
  if (!tlr::kernel_product_args_ok(points_host, kern, X, Y, N, d, nrhs, ldx, ldy)) return TLR_ERR_ARG;
  if (N * d > kMaxPointDoubles) return TLR_ERR_LIMIT;
  if (nrhs == 0) return TLR_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return TLR_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return TLR_ERR_LIMIT;
  double* pts = nullptr;
  if (points_address(dev, &pts) != cudaSuccess) {
    cudaGetLastError();
    return TLR_ERR_CUDA;
  }
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaMemcpyAsync(pts, points_host, sizeof(double) * N * d, cudaMemcpyHostToDevice, stream) != cudaSuccess) {
    cudaGetLastError();
    return TLR_ERR_CUDA;
  }
  // A context on the stack carries only the stream to the launcher; it owns no memory.
  tlr_ctx launch_ctx;
  launch_ctx.device = dev;
  launch_ctx.stream = stream;
  try {
    tlr::kernel_matvec(&launch_ctx, pts, N, d, kern->ell, kern->nugget, nrhs, X, ldx, Y, ldy);
  } catch (const tlr::Error& e) {
    cudaGetLastError();  // a failed launch leaves its error pending: do not hand it to the caller's next call
    return e.status;
  }
  return TLR_OK;
}
