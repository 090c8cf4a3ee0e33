// Allocation-free variant of the FP64 matrix-free operator apply.
//
// sfem_apply allocates, on every call, a masked copy of u and (on first use)
// the per-tet strain scratch through the context allocator.  This entry
// point allocates nothing: the strain scratch is a file-scope __device__
// array of fixed size, and the input mask is applied while gathering.
//
// Who needs it: callers that must not allocate device memory per call,
// e.g. an application whose memory pool (another framework's caching
// allocator) already holds the device memory, so that an extra allocation
// would fail, and latency-bound loops calling the operator thousands of
// times, where an allocation or a free may synchronise the device.
//
// The array is loaded with the library and every GPU that loads it keeps
// it (kNoAllocMaxTets * 8 doubles = 8 MiB) until the process exits.  All
// calls share it: calls that overlap on the GPU (two streams, two
// contexts) race on it.  Nothing in it needs clearing: the strain pass
// writes every entry the stress pass reads.

#include <cuda_runtime.h>

#include <mutex>

#include "sfem_internal.cuh"

namespace sfem {

constexpr int64_t kNoAllocMaxTets = 131072;
static __device__ __align__(256) double g_noalloc_w[kNoAllocMaxTets * 8];

constexpr int kNoAllocMaxDevices = 256;
static std::mutex g_noalloc_mu;
static double *g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on `dev` (the current device).  In
// host code g_noalloc_w names a host-side shadow, not device memory, so the
// address is looked up once per device and cached for the process's life.
// A cudaDeviceReset would make the cached address stale; it also ends every
// context of the library, so the entry point is not usable after one.
static double *noalloc_scratch(int dev) {
  SFEM_REQUIRE(dev >= 0 && dev < kNoAllocMaxDevices, SFEM_EINVAL, "device id out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_w);
    if (e != cudaSuccess || p == nullptr)
      throw Error{SFEM_ECUDA, std::string("cudaGetSymbolAddress of the scratch array failed: ") +
                                  cudaGetErrorString(e)};
    g_noalloc_addr[dev] = static_cast<double *>(p);
  }
  return g_noalloc_addr[dev];
}

// w_e = V_e eps_e of P u (prescribed DOFs read as zero), FP64
__global__ void k_noalloc_strain(int64_t n, const int4 *__restrict__ conn, const double *__restrict__ Gs,
                                 const double *__restrict__ u, const uint8_t *__restrict__ dmask,
                                 double *__restrict__ w) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int4 t = conn[e];
  const int v[4] = {t.x, t.y, t.z, t.w};
  double g[4][3];
  for (int k = 0; k < 9; ++k) g[1 + k / 3][k % 3] = Gs[k * n + e];
  for (int i = 0; i < 3; ++i) g[0][i] = -(g[1][i] + g[2][i] + g[3][i]);
  double H[3][3] = {};
  for (int a = 0; a < 4; ++a) {
    const int64_t d = 3 * (int64_t)v[a];
    const double u0 = dmask[d] ? u[d] : 0.0, u1 = dmask[d + 1] ? u[d + 1] : 0.0;
    const double u2 = dmask[d + 2] ? u[d + 2] : 0.0;
    for (int j = 0; j < 3; ++j) {
      H[0][j] += u0 * g[a][j];
      H[1][j] += u1 * g[a][j];
      H[2][j] += u2 * g[a][j];
    }
  }
  double *we = w + 8 * e;
  we[0] = H[0][0];
  we[1] = H[1][1];
  we[2] = H[2][2];
  we[3] = H[1][2] + H[2][1];
  we[4] = H[2][0] + H[0][2];
  we[5] = H[0][1] + H[1][0];
}

// rows of prescribed DOFs: y_i = u_i (the (I - P) u part of A u)
__global__ void k_noalloc_fix_rows(double *__restrict__ y, const double *__restrict__ u,
                                   const uint8_t *__restrict__ dmask, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !dmask[i]) y[i] = u[i];
}

}  // namespace sfem

using namespace sfem;

extern "C" int sfem_apply_noalloc(sfem_ctx *h, const double *u, double *y) {
  try {
    SFEM_REQUIRE(h && h->c.vol, SFEM_EINVAL, "context not set up");
    SFEM_REQUIRE(u && y, SFEM_EINVAL, "u and y must be device pointers");
    Ctx &c = h->c;
    SFEM_REQUIRE(c.n_tets <= kNoAllocMaxTets, SFEM_EINVAL,
                 "sfem_apply_noalloc handles at most " + std::to_string(kNoAllocMaxTets) + " tets (mesh has " +
                     std::to_string(c.n_tets) + "); use sfem_apply");
    int dev = -1;
    SFEM_CUDA(cudaGetDevice(&dev));
    SFEM_REQUIRE(dev == c.device, SFEM_EINVAL, "the context's device must be current");
    double *w = noalloc_scratch(dev);
    SFEM_CUDA(cudaMemsetAsync(y, 0, c.ndof * sizeof(double), c.stream));
    k_noalloc_strain<<<grid_for(c.n_tets, 256), 256, 0, c.stream>>>(
        c.n_tets, reinterpret_cast<const int4 *>(c.tets), c.Gs64, u, c.dmask, w);
    SFEM_CHECK_LAUNCH();
    launch_mf_stress<double, double>(c, c.stream, c.Gs64, c.kap64, w, y, 1, nullptr, nullptr);
    k_noalloc_fix_rows<<<grid_for(c.ndof, 256), 256, 0, c.stream>>>(y, u, c.dmask, c.ndof);
    SFEM_CHECK_LAUNCH();
  } catch (const Error &err) {
    set_last_error(err.msg);
    return err.status;
  }
  return SFEM_OK;
}
