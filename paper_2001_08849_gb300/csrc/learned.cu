// Learned coarse correction inside flexible PCG (the paper has no
// counterpart: it calls a direct solver and needs no preconditioner).
//
// The residual r is pooled over a regular grid of patches (mean of each
// patch's nodal 3-vectors).  Patch p gets 84 inputs: the pooled residuals
// of its 3x3x3 patch neighbourhood (zero outside the grid) divided by the
// RMS of all pooled values, and its centre normalised to [0,1]^3.  A
// 3-layer MLP (84 -> 128 -> GELU -> 128 -> GELU -> 3; BF16 weights, FP32
// biases, FP32 accumulation) maps them to one coarse 3-vector per patch;
// trilinear interpolation between patch centres carries those to the nodes
// (masked by P), giving c.  The preconditioned residual is
//     z = D^-1 r + alpha c,   alpha = c.r / c.A c,
// with c.A c from the FP32 tiled operator (one extra apply per iteration).
// Flexible CG (Polak-Ribiere beta) absorbs the iteration-dependent z.
//
// Safeguards, plain Jacobi-PCG being the fallback:
//   * an iteration whose c is unusable (c.A c <= 0 or a non-finite alpha or
//     z.r) takes z = D^-1 r and is counted;
//   * guards that switch the correction off for the rest of the solve: the
//     residual norm has not fallen 10% below its best value for `window`
//     iterations, or (with a reference count `pace`, e.g. the Jacobi-PCG
//     iterations measured on the training loads) it lies more than 30x
//     above the log-linear line from ||r_0|| to the tolerance over `pace`
//     iterations.  If a learned direction has been used since the last
//     restart, the direction restarts (beta = 0); either way CG goes on
//     from the current iterate with the Jacobi preconditioner;
//   * the FP64 true residual decides convergence, as for the other solvers.
//
// Training runs on the GPU with the kernels below: FP32 master weights,
// forward with cached activations, hand-written backward, Adam.  Training
// pairs (features of r, pooled and normalised u* - x) are taken from the
// library's own CG runs (sfem_learned_collect).

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>
#include <vector>

#include "mlp.cuh"
#include "reduce.cuh"
#include "sfem_internal.cuh"

namespace sfem {

constexpr int kIn = 84, kHid = 128, kOut = 3;
constexpr int kNbr = 81;  // 3x3x3 neighbourhood x 3 components
constexpr int oW1 = 0, oB1 = oW1 + kIn * kHid, oW2 = oB1 + kHid, oB2 = oW2 + kHid * kHid, oW3 = oB2 + kHid,
              oB3 = oW3 + kHid * kOut, kNParams = oB3 + kOut;
constexpr int kMaxPatches = 1 << 18;
constexpr int kPoolThreads = 128;
constexpr int kInferRows = 8;
constexpr uint32_t kBlobMagic = 0x4e4e4653u;  // "SFNN"
constexpr int kBlobVersion = 1;

struct Learned {
  int device = 0;
  cudaStream_t stream = nullptr;
  Allocator mem;
  PatchGrid g{};
  int P = 0;
  int64_t n_nodes = 0;
  int32_t *pnodes = nullptr;  // node ids grouped by patch, ascending within a patch
  int32_t *poff = nullptr;    // P + 1 offsets into pnodes
  float *theta = nullptr;     // FP32 master parameters
  float *mom = nullptr, *vel = nullptr, *grad = nullptr;
  __nv_bfloat16 *wbf = nullptr;  // BF16 copies of theta (the weights are used from here)
  int step = 0;
  double *pooled = nullptr;   // 3P + 3P (r and e)
  double *scale = nullptr;    // 2: 1/RMS of the pooled r, e
  double *partials = nullptr; // max(P, 4096)
  unsigned int *tickets = nullptr;  // 8, zero between kernels
  double *loss = nullptr;     // 2: loss of the last batch, accumulated loss
  // training scratch for `cap` rows
  int64_t cap = 0;
  float *Xb = nullptr, *Tb = nullptr, *a1 = nullptr, *h1 = nullptr, *a2 = nullptr, *h2 = nullptr, *y = nullptr,
        *dy = nullptr, *d2 = nullptr, *d1 = nullptr;
  float *split = nullptr;     // split-K partial products
  size_t split_floats = 0;
  int *gemm_err = nullptr;    // set by a tensor-core GEMM whose wait ran out
};

// ---- patches, pooling, features, prolongation ------------------------------

// pooled[3p+c] = mean over the nodes of patch p of v[3n+c] (0 for an empty
// patch); the last block writes scale = 1/RMS of all pooled values (0 if
// they are all zero).  One block per patch, fixed summation order.
__global__ void __launch_bounds__(kPoolThreads) k_pool(const double *__restrict__ v, const int32_t *__restrict__ pnodes,
                                                       const int32_t *__restrict__ poff, double *__restrict__ pooled,
                                                       double *scale, double *partials, unsigned int *ticket,
                                                       const int *off) {
  if (off && *off) return;
  const int p = blockIdx.x;
  const int b = poff[p], e = poff[p + 1];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int i = b + threadIdx.x; i < e; i += kPoolThreads) {
    const int64_t nd = pnodes[i];
    s0 += v[3 * nd];
    s1 += v[3 * nd + 1];
    s2 += v[3 * nd + 2];
  }
  s0 = block_sum<kPoolThreads>(s0);
  s1 = block_sum<kPoolThreads>(s1);
  s2 = block_sum<kPoolThreads>(s2);
  double sq = 0.0;
  if (threadIdx.x == 0) {
    const double cnt = (double)max(e - b, 1);
    const double m0 = s0 / cnt, m1 = s1 / cnt, m2 = s2 / cnt;
    pooled[3 * p] = m0;
    pooled[3 * p + 1] = m1;
    pooled[3 * p + 2] = m2;
    sq = m0 * m0 + m1 * m1 + m2 * m2;
  }
  double vv[1] = {sq};
  if (grid_sum<kPoolThreads, 1>(vv, partials, ticket, nullptr) && threadIdx.x == 0) {
    const double rms = sqrt(vv[0] / (3.0 * gridDim.x));
    *scale = rms > 0.0 ? 1.0 / rms : 0.0;
  }
}

// input f of patch p: 3x3x3 neighbourhood of pooled values x scale (k-major
// over the offsets (-1,0,1)^3, then the component), then the centre
__device__ __forceinline__ float feature(const double *__restrict__ pooled, double scale, const PatchGrid &g, int p,
                                         int f) {
  const int pz = p % g.d[2], py = (p / g.d[2]) % g.d[1], px = p / (g.d[1] * g.d[2]);
  if (f < kNbr) {
    const int k = f / 3, c = f % 3;
    const int qx = px + k / 9 - 1, qy = py + (k / 3) % 3 - 1, qz = pz + k % 3 - 1;
    if (qx < 0 || qy < 0 || qz < 0 || qx >= g.d[0] || qy >= g.d[1] || qz >= g.d[2]) return 0.f;
    return (float)(pooled[3 * ((qx * g.d[1] + qy) * g.d[2] + qz) + c] * scale);
  }
  const int a = f - kNbr;
  const int pa = a == 0 ? px : a == 1 ? py : pz;
  return (float)((pa + 0.5) / g.d[a]);
}

__global__ void k_features(const double *__restrict__ pooled, const double *__restrict__ scale, PatchGrid g, int P,
                           float *__restrict__ X) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)P * kIn) return;
  X[i] = feature(pooled, *scale, g, (int)(i / kIn), (int)(i % kIn));
}

__global__ void k_target(const double *__restrict__ pooled, const double *__restrict__ scale, int P,
                         float *__restrict__ T) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 3 * P) T[i] = (float)(pooled[i] * *scale);
}

// MLP inference: BF16 weights, FP32 biases and accumulation, 8 rows per
// 128-thread block (thread j owns hidden unit j).  Inputs come from X (rows
// x 84) or, with kFromPooled, are formed from the pooled residual.
template <bool kFromPooled>
__global__ void __launch_bounds__(kHid) k_mlp_infer(const float *__restrict__ X, const double *__restrict__ pooled,
                                                    const double *__restrict__ scale, PatchGrid g, int rows,
                                                    const __nv_bfloat16 *__restrict__ w,
                                                    const float *__restrict__ th, float *__restrict__ Y,
                                                    const int *off) {
  if (off && *off) return;
  __shared__ float xs[kInferRows][kIn];
  __shared__ float hs[kInferRows][kHid];
  __shared__ float gs[kInferRows][kHid];
  const int r0 = blockIdx.x * kInferRows;
  const int j = threadIdx.x;
  double sc = 0.0;
  if (kFromPooled) sc = *scale;
  for (int i = j; i < kInferRows * kIn; i += kHid) {
    const int r = r0 + i / kIn, f = i % kIn;
    float v = 0.f;
    if (r < rows) v = kFromPooled ? feature(pooled, sc, g, r, f) : X[(int64_t)r * kIn + f];
    xs[i / kIn][f] = v;
  }
  __syncthreads();
  float acc[kInferRows];
#pragma unroll
  for (int q = 0; q < kInferRows; ++q) acc[q] = th[oB1 + j];
  for (int i = 0; i < kIn; ++i) {
    const float wij = __bfloat162float(w[oW1 + i * kHid + j]);
#pragma unroll
    for (int q = 0; q < kInferRows; ++q) acc[q] = fmaf(xs[q][i], wij, acc[q]);
  }
#pragma unroll
  for (int q = 0; q < kInferRows; ++q) hs[q][j] = 0.5f * acc[q] * (1.f + erff(acc[q] * 0.70710678118654752f));
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kInferRows; ++q) acc[q] = th[oB2 + j];
  for (int i = 0; i < kHid; ++i) {
    const float wij = __bfloat162float(w[oW2 + i * kHid + j]);
#pragma unroll
    for (int q = 0; q < kInferRows; ++q) acc[q] = fmaf(hs[q][i], wij, acc[q]);
  }
#pragma unroll
  for (int q = 0; q < kInferRows; ++q) gs[q][j] = 0.5f * acc[q] * (1.f + erff(acc[q] * 0.70710678118654752f));
  __syncthreads();
  if (j < kInferRows * kOut) {
    const int q = j / kOut, o = j % kOut;
    float a = th[oB3 + o];
    for (int i = 0; i < kHid; ++i) a = fmaf(gs[q][i], __bfloat162float(w[oW3 + i * kOut + o]), a);
    if (r0 + q < rows) Y[(int64_t)(r0 + q) * kOut + o] = a;
  }
}

// c = P * trilinear(patch outputs) at the nodes (patch centres as the
// interpolation points, clamped to the outermost ones); Ac = 0
__global__ void k_prolong(const float *__restrict__ Y, PatchGrid g, const double *__restrict__ xyz, int64_t n,
                          const uint8_t *__restrict__ dmask, double *__restrict__ cvec, double *__restrict__ Ac,
                          const int *off) {
  if (off && *off) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int i0[3];
  double f[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double t = (xyz[3 * i + a] - g.lo[a]) / g.ext[a] * g.d[a] - 0.5;
    t = fmin(fmax(t, 0.0), (double)max(g.d[a] - 1, 0));
    const int k = min(max((int)floor(t), 0), max(g.d[a] - 2, 0));
    i0[a] = k;
    f[a] = g.d[a] > 1 ? t - k : 0.0;
  }
  double out[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int ia = min(i0[0] + a, g.d[0] - 1), ib = min(i0[1] + b, g.d[1] - 1), ic = min(i0[2] + cc, g.d[2] - 1);
        const double wgt = (a ? f[0] : 1 - f[0]) * (b ? f[1] : 1 - f[1]) * (cc ? f[2] : 1 - f[2]);
        const int q = (ia * g.d[1] + ib) * g.d[2] + ic;
#pragma unroll
        for (int c = 0; c < 3; ++c) out[c] += wgt * (double)Y[3 * q + c];
      }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cvec[3 * i + c] = dmask[3 * i + c] ? out[c] : 0.0;
    Ac[3 * i + c] = 0.0;
  }
}

// ---- dense training kernels (FP32) -------------------------------------------

// He-normal weights (std sqrt(2/fan_in); sqrt(1/fan_in) for the linear
// output layer) by Box-Muller on counter-based uniforms; zero biases
__global__ void k_init(float *theta, __nv_bfloat16 *wbf, int n, uint64_t seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float sd = 0.f;
  if (i < oB1)
    sd = sqrtf(2.f / kIn);
  else if (i >= oW2 && i < oB2)
    sd = sqrtf(2.f / kHid);
  else if (i >= oW3 && i < oB3)
    sd = sqrtf(1.f / kHid);
  float v = 0.f;
  if (sd > 0.f) {
    const uint64_t h = splitmix64(seed * 0x100000001b3ull + (uint64_t)i);
    const double u1 = (double)((h >> 11) + 1) * (1.0 / 9007199254740992.0);  // (0, 1]
    const double u2 = (double)(splitmix64(h) >> 11) * (1.0 / 9007199254740992.0);
    v = (float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2)) * sd;
  }
  theta[i] = v;
  wbf[i] = __float2bfloat16_rn(v);
}

// rows of (X, T) in the order r -> (a r + b) mod rows
__global__ void k_gather_rows(const float *__restrict__ X, const float *__restrict__ T, int64_t rows, int64_t first,
                              int64_t nb, uint64_t a, uint64_t b, float *__restrict__ Xb, float *__restrict__ Tb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb * (kIn + kOut)) return;
  const int64_t r = i / (kIn + kOut);
  const int f = (int)(i % (kIn + kOut));
  const uint64_t R = (uint64_t)rows;
  const int64_t src = (int64_t)(((a % R) * ((uint64_t)(first + r) % R) % R + b) % R);
  if (f < kIn)
    Xb[r * kIn + f] = X[src * kIn + f];
  else
    Tb[r * kOut + f - kIn] = T[src * kOut + f - kIn];
}

__global__ void k_sub(const double *a, const double *b, int64_t n, double *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] - b[i];
}

// ---- host helpers --------------------------------------------------------------

static void gemm(Learned &L, int M, int N, int K, const float *A, int lda, bool tA, const float *B, int ldb, bool tB,
                 float *C, int ldc) {
  mlp_gemm(L.mem, L.split, L.split_floats, L.stream, M, N, K, A, lda, tA, B, ldb, tB, C, ldc, L.gemm_err);
}

static void ensure_cap(Learned &L, int64_t rows) {
  if (rows <= L.cap) return;
  for (float *p : {L.Xb, L.Tb, L.a1, L.h1, L.a2, L.h2, L.y, L.dy, L.d2, L.d1})
    if (p) L.mem.drop(p);
  L.Xb = L.mem.get<float>(rows * kIn);
  L.Tb = L.mem.get<float>(rows * kOut);
  L.a1 = L.mem.get<float>(rows * kHid);
  L.h1 = L.mem.get<float>(rows * kHid);
  L.a2 = L.mem.get<float>(rows * kHid);
  L.h2 = L.mem.get<float>(rows * kHid);
  L.y = L.mem.get<float>(rows * kOut);
  L.dy = L.mem.get<float>(rows * kOut);
  L.d2 = L.mem.get<float>(rows * kHid);
  L.d1 = L.mem.get<float>(rows * kHid);
  L.cap = rows;
}

// Forward with cached activations (FP32 master weights), the loss
// sum((y - T)^2) / rows (L.loss[0], and L.loss[1] += sum) and its gradient
// by the chain rule through the three layers (L.grad).
static void loss_grad(Learned &L, const float *X, const float *T, int64_t rows) {
  ensure_cap(L, rows);
  cudaStream_t st = L.stream;
  const float *W1 = L.theta + oW1, *W2 = L.theta + oW2, *W3 = L.theta + oW3;
  const int r = (int)rows;
  const int gh = grid_for(rows * kHid, 256);
  gemm(L, r, kHid, kIn, X, kIn, false, W1, kHid, false, L.a1, kHid);
  k_bias_gelu<<<gh, 256, 0, st>>>(L.a1, L.h1, L.theta + oB1, rows, kHid);
  SFEM_CHECK_LAUNCH();
  gemm(L, r, kHid, kHid, L.h1, kHid, false, W2, kHid, false, L.a2, kHid);
  k_bias_gelu<<<gh, 256, 0, st>>>(L.a2, L.h2, L.theta + oB2, rows, kHid);
  SFEM_CHECK_LAUNCH();
  gemm(L, r, kOut, kHid, L.h2, kHid, false, W3, kOut, false, L.y, kOut);
  k_bias_gelu<<<grid_for(rows * kOut, 256), 256, 0, st>>>(L.y, nullptr, L.theta + oB3, rows, kOut);
  SFEM_CHECK_LAUNCH();
  k_mse<<<(unsigned)std::min<int64_t>(grid_for(rows * kOut, 256), 512), 256, 0, st>>>(
      L.y, T, rows * kOut, rows, L.dy, L.partials, L.tickets + 1, L.loss);
  SFEM_CHECK_LAUNCH();
  float *g = L.grad;
  gemm(L, kHid, kOut, r, L.h2, kHid, true, L.dy, kOut, false, g + oW3, kOut);
  k_colsum<<<kOut, 256, 0, st>>>(L.dy, rows, kOut, g + oB3);
  SFEM_CHECK_LAUNCH();
  gemm(L, r, kHid, kOut, L.dy, kOut, false, W3, kOut, true, L.d2, kHid);
  k_gelu_back<<<gh, 256, 0, st>>>(L.d2, L.a2, rows * kHid);
  SFEM_CHECK_LAUNCH();
  gemm(L, kHid, kHid, r, L.h1, kHid, true, L.d2, kHid, false, g + oW2, kHid);
  k_colsum<<<kHid, 256, 0, st>>>(L.d2, rows, kHid, g + oB2);
  SFEM_CHECK_LAUNCH();
  gemm(L, r, kHid, kHid, L.d2, kHid, false, W2, kHid, true, L.d1, kHid);
  k_gelu_back<<<gh, 256, 0, st>>>(L.d1, L.a1, rows * kHid);
  SFEM_CHECK_LAUNCH();
  gemm(L, kIn, kHid, r, X, kIn, true, L.d1, kHid, false, g + oW1, kHid);
  k_colsum<<<kHid, 256, 0, st>>>(L.d1, rows, kHid, g + oB1);
  SFEM_CHECK_LAUNCH();
}

static void adam_step(Learned &L, const float *g, float lr, float b1, float b2, float eps) {
  L.step += 1;
  const float c1 = (float)(1.0 - std::pow((double)b1, L.step));
  const float c2 = (float)(1.0 - std::pow((double)b2, L.step));
  k_adam<<<grid_for(kNParams, 256), 256, 0, L.stream>>>(L.theta, g, L.mom, L.vel, kNParams, lr, b1, b2, eps, c1, c2,
                                                       L.wbf);
  SFEM_CHECK_LAUNCH();
}

// pooled r (and e) features / targets of one snapshot into X, T
static void sample_into(Learned &L, const double *r, const double *e, float *X, float *T, cudaStream_t st) {
  k_pool<<<L.P, kPoolThreads, 0, st>>>(r, L.pnodes, L.poff, L.pooled, L.scale, L.partials, L.tickets + 2, nullptr);
  SFEM_CHECK_LAUNCH();
  k_features<<<grid_for((int64_t)L.P * kIn, 256), 256, 0, st>>>(L.pooled, L.scale, L.g, L.P, X);
  SFEM_CHECK_LAUNCH();
  if (e && T) {
    double *pe = L.pooled + 3 * L.P;
    k_pool<<<L.P, kPoolThreads, 0, st>>>(e, L.pnodes, L.poff, pe, L.scale + 1, L.partials, L.tickets + 2, nullptr);
    SFEM_CHECK_LAUNCH();
    k_target<<<grid_for(3 * L.P, 256), 256, 0, st>>>(pe, L.scale + 1, L.P, T);
    SFEM_CHECK_LAUNCH();
  }
}

}  // namespace sfem

// ============================================================================
// ABI: model object, sampling, training, inference
// ============================================================================
using namespace sfem;

struct sfem_learned {
  Learned L;
};

#define LRN_BEGIN try {
#define LRN_END              \
  }                          \
  catch (const Error &err) { \
    set_last_error(err.msg); \
    return err.status;       \
  }                          \
  return SFEM_OK;

static void check_model_ctx(const sfem_learned *m, const sfem_ctx *h) {
  SFEM_REQUIRE(m && h && h->c.vol, SFEM_EINVAL, "a model and a set-up context are required");
  SFEM_REQUIRE(h->c.n_nodes == m->L.n_nodes, SFEM_EINVAL, "the model was created on a mesh of another size");
  SFEM_REQUIRE(h->c.device == m->L.device, SFEM_EINVAL, "the model lives on another device");
  SFEM_REQUIRE(h->c.stream == m->L.stream, SFEM_EINVAL, "model and context must share a stream");
}

extern "C" int sfem_learned_create(sfem_learned **out, sfem_ctx *h, const sfem_learned_opts *opts) {
  sfem_learned *m = nullptr;
  try {
    SFEM_REQUIRE(out && h && h->c.vol, SFEM_EINVAL, "out and a set-up context are required");
    *out = nullptr;
    if (opts)
      for (int r : opts->reserved) SFEM_REQUIRE(r == 0, SFEM_EINVAL, "reserved options must be zero");
    Ctx &c = h->c;
    m = new sfem_learned();
    Learned &L = m->L;
    L.device = c.device;
    L.stream = c.stream;
    L.mem.alloc = c.mem.alloc;
    L.mem.free = c.mem.free;
    L.mem.user = c.mem.user;
    L.mem.stream = c.stream;
    L.n_nodes = c.n_nodes;
    // Patch grid over the bounding box.  This one-time grouping of nodes by
    // patch runs on the host: it orders node ids within each patch so that
    // the device pooling sums in a fixed order.
    std::vector<double> xyz(3 * c.n_nodes);
    SFEM_CUDA(cudaMemcpyAsync(xyz.data(), c.xyz, xyz.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    SFEM_CUDA(cudaStreamSynchronize(c.stream));
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < c.n_nodes; ++i)
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::min(lo[a], xyz[3 * i + a]);
        hi[a] = std::max(hi[a], xyz[3 * i + a]);
      }
    const int pn = (opts && opts->patch_nodes > 0) ? opts->patch_nodes : 8;
    // default: patches of about pn nodes per axis at the mesh's mean node density
    const double box = std::max((hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]), 1e-300);
    const double h_mean = std::cbrt(box / (double)c.n_nodes);
    int64_t P = 1;
    for (int a = 0; a < 3; ++a) {
      L.g.lo[a] = lo[a];
      L.g.ext[a] = std::max(hi[a] - lo[a], 1e-300);
      const int req = opts ? opts->patch_dims[a] : 0;
      SFEM_REQUIRE(req >= 0 && req <= kMaxPatches, SFEM_EINVAL, "patch_dims out of range");
      L.g.d[a] = req > 0 ? req : std::max(1, (int)std::ceil((hi[a] - lo[a]) / (pn * h_mean) - 1e-9));
      P *= L.g.d[a];
      SFEM_REQUIRE(P <= kMaxPatches, SFEM_EINVAL, "patch grid larger than 262144 patches");
    }
    L.P = (int)P;
    std::vector<int32_t> pid(c.n_nodes), off(L.P + 1, 0), nodes(c.n_nodes);
    for (int64_t i = 0; i < c.n_nodes; ++i) {
      int q[3];
      for (int a = 0; a < 3; ++a) {
        const double t = std::floor((xyz[3 * i + a] - L.g.lo[a]) / L.g.ext[a] * L.g.d[a]);
        q[a] = (int)std::min<double>(std::max<double>(t, 0.0), L.g.d[a] - 1);
      }
      pid[i] = (q[0] * L.g.d[1] + q[1]) * L.g.d[2] + q[2];
      off[pid[i] + 1] += 1;
    }
    for (int p = 0; p < L.P; ++p) off[p + 1] += off[p];
    {
      std::vector<int32_t> cur(off.begin(), off.end() - 1);
      for (int64_t i = 0; i < c.n_nodes; ++i) nodes[cur[pid[i]]++] = (int32_t)i;
    }
    L.pnodes = L.mem.get<int32_t>(c.n_nodes);
    L.poff = L.mem.get<int32_t>(L.P + 1);
    SFEM_CUDA(cudaMemcpyAsync(L.pnodes, nodes.data(), nodes.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                              L.stream));
    SFEM_CUDA(cudaMemcpyAsync(L.poff, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice, L.stream));
    L.theta = L.mem.get<float>(kNParams);
    L.mom = L.mem.get<float>(kNParams);
    L.vel = L.mem.get<float>(kNParams);
    L.grad = L.mem.get<float>(kNParams);
    L.wbf = L.mem.get<__nv_bfloat16>(kNParams);
    L.pooled = L.mem.get<double>(6 * (size_t)L.P);
    L.scale = L.mem.get<double>(2);
    L.partials = L.mem.get<double>(std::max(L.P, 4096));
    L.tickets = L.mem.get<unsigned int>(8);
    L.loss = L.mem.get<double>(2);
    L.gemm_err = L.mem.get<int>(1);
    SFEM_CUDA(cudaMemsetAsync(L.gemm_err, 0, sizeof(int), L.stream));
    SFEM_CUDA(cudaMemsetAsync(L.tickets, 0, 8 * sizeof(unsigned int), L.stream));
    SFEM_CUDA(cudaMemsetAsync(L.mom, 0, kNParams * sizeof(float), L.stream));
    SFEM_CUDA(cudaMemsetAsync(L.vel, 0, kNParams * sizeof(float), L.stream));
    SFEM_CUDA(cudaMemsetAsync(L.loss, 0, 2 * sizeof(double), L.stream));
    const uint64_t seed = opts ? (uint64_t)opts->seed : 0;
    k_init<<<grid_for(kNParams, 256), 256, 0, L.stream>>>(L.theta, L.wbf, kNParams, seed);
    SFEM_CHECK_LAUNCH();
    SFEM_CUDA(cudaStreamSynchronize(L.stream));
    *out = m;
    m = nullptr;
  } catch (const Error &err) {
    if (m) {
      cudaStreamSynchronize(m->L.stream);
      m->L.mem.release_all();
      delete m;
    }
    set_last_error(err.msg);
    return err.status;
  }
  return SFEM_OK;
}

extern "C" void sfem_learned_destroy(sfem_learned *m) {
  if (!m) return;
  cudaStreamSynchronize(m->L.stream);
  m->L.mem.release_all();
  delete m;
}

extern "C" int sfem_learned_info(const sfem_learned *m, int *patch_dims, int *n_patches, int *n_params) {
  if (!m) {
    set_last_error("model is NULL");
    return SFEM_EINVAL;
  }
  if (patch_dims)
    for (int a = 0; a < 3; ++a) patch_dims[a] = m->L.g.d[a];
  if (n_patches) *n_patches = m->L.P;
  if (n_params) *n_params = kNParams;
  return SFEM_OK;
}

extern "C" int sfem_learned_set_params(sfem_learned *m, const float *theta, int64_t n) {
  LRN_BEGIN
  SFEM_REQUIRE(m && theta && n == kNParams, SFEM_EINVAL, "parameter vector of the wrong size");
  Learned &L = m->L;
  SFEM_CUDA(cudaMemcpyAsync(L.theta, theta, n * sizeof(float), cudaMemcpyHostToDevice, L.stream));
  SFEM_CUDA(cudaMemsetAsync(L.mom, 0, kNParams * sizeof(float), L.stream));
  SFEM_CUDA(cudaMemsetAsync(L.vel, 0, kNParams * sizeof(float), L.stream));
  L.step = 0;
  k_to_bf16<<<grid_for(kNParams, 256), 256, 0, L.stream>>>(L.theta, L.wbf, kNParams);
  SFEM_CHECK_LAUNCH();
  SFEM_CUDA(cudaStreamSynchronize(L.stream));
  LRN_END
}

extern "C" int sfem_learned_get_params(sfem_learned *m, float *theta, int64_t n) {
  LRN_BEGIN
  SFEM_REQUIRE(m && theta && n == kNParams, SFEM_EINVAL, "parameter vector of the wrong size");
  SFEM_CUDA(cudaMemcpyAsync(theta, m->L.theta, n * sizeof(float), cudaMemcpyDeviceToHost, m->L.stream));
  SFEM_CUDA(cudaStreamSynchronize(m->L.stream));
  LRN_END
}

extern "C" int sfem_learned_export(sfem_learned *m, void *buf, size_t cap, size_t *size) {
  LRN_BEGIN
  SFEM_REQUIRE(m && size, SFEM_EINVAL, "model and size are required");
  const size_t need = 8 * sizeof(int32_t) + kNParams * sizeof(float);
  *size = need;
  if (!buf) return SFEM_OK;
  SFEM_REQUIRE(cap >= need, SFEM_EINVAL, "buffer too small");
  int32_t hdr[8] = {(int32_t)kBlobMagic, kBlobVersion, kIn, kHid, kOut, m->L.g.d[0], m->L.g.d[1], m->L.g.d[2]};
  std::memcpy(buf, hdr, sizeof hdr);
  SFEM_CUDA(cudaMemcpyAsync(static_cast<char *>(buf) + sizeof hdr, m->L.theta, kNParams * sizeof(float),
                            cudaMemcpyDeviceToHost, m->L.stream));
  SFEM_CUDA(cudaStreamSynchronize(m->L.stream));
  LRN_END
}

extern "C" int sfem_learned_import(sfem_learned *m, const void *buf, size_t size) {
  LRN_BEGIN
  SFEM_REQUIRE(m && buf, SFEM_EINVAL, "model and buffer are required");
  const size_t need = 8 * sizeof(int32_t) + kNParams * sizeof(float);
  SFEM_REQUIRE(size == need, SFEM_EINVAL, "blob of the wrong size");
  int32_t hdr[8];
  std::memcpy(hdr, buf, sizeof hdr);
  SFEM_REQUIRE(hdr[0] == (int32_t)kBlobMagic && hdr[1] == kBlobVersion, SFEM_EINVAL, "not a model blob of version 1");
  SFEM_REQUIRE(hdr[2] == kIn && hdr[3] == kHid && hdr[4] == kOut, SFEM_EINVAL, "blob of another network shape");
  SFEM_REQUIRE(hdr[5] == m->L.g.d[0] && hdr[6] == m->L.g.d[1] && hdr[7] == m->L.g.d[2], SFEM_EINVAL,
               "blob trained on another patch grid");
  std::vector<float> th(kNParams);
  std::memcpy(th.data(), static_cast<const char *>(buf) + sizeof hdr, kNParams * sizeof(float));
  Learned &L = m->L;
  SFEM_CUDA(cudaMemcpyAsync(L.theta, th.data(), kNParams * sizeof(float), cudaMemcpyHostToDevice, L.stream));
  SFEM_CUDA(cudaMemsetAsync(L.mom, 0, kNParams * sizeof(float), L.stream));
  SFEM_CUDA(cudaMemsetAsync(L.vel, 0, kNParams * sizeof(float), L.stream));
  L.step = 0;
  k_to_bf16<<<grid_for(kNParams, 256), 256, 0, L.stream>>>(L.theta, L.wbf, kNParams);
  SFEM_CHECK_LAUNCH();
  SFEM_CUDA(cudaStreamSynchronize(L.stream));
  LRN_END
}

extern "C" int sfem_learned_forward(sfem_learned *m, const float *X, float *Y, int64_t rows) {
  LRN_BEGIN
  SFEM_REQUIRE(m && X && Y && rows >= 1 && rows <= (int64_t)1 << 30, SFEM_EINVAL, "bad arguments");
  Learned &L = m->L;
  k_mlp_infer<false><<<(unsigned)((rows + kInferRows - 1) / kInferRows), kHid, 0, L.stream>>>(
      X, nullptr, nullptr, L.g, (int)rows, L.wbf, L.theta, Y, nullptr);
  SFEM_CHECK_LAUNCH();
  SFEM_CUDA(cudaStreamSynchronize(L.stream));
  LRN_END
}

extern "C" int sfem_learned_loss_grad(sfem_learned *m, const float *X, const float *T, int64_t rows, float *grad,
                                      double *loss) {
  LRN_BEGIN
  SFEM_REQUIRE(m && X && T && rows >= 1 && rows <= (int64_t)1 << 24, SFEM_EINVAL, "bad arguments");
  Learned &L = m->L;
  loss_grad(L, X, T, rows);
  if (grad)
    SFEM_CUDA(cudaMemcpyAsync(grad, L.grad, kNParams * sizeof(float), cudaMemcpyDeviceToDevice, L.stream));
  if (loss) SFEM_CUDA(cudaMemcpyAsync(loss, L.loss, sizeof(double), cudaMemcpyDeviceToHost, L.stream));
  check_gemm_err(L.gemm_err, L.stream);
  LRN_END
}

extern "C" int sfem_learned_adam(sfem_learned *m, const float *grad, float lr, float b1, float b2, float eps) {
  LRN_BEGIN
  SFEM_REQUIRE(m && lr > 0.f && b1 >= 0.f && b1 < 1.f && b2 >= 0.f && b2 < 1.f && eps > 0.f, SFEM_EINVAL,
               "bad arguments");
  adam_step(m->L, grad ? grad : m->L.grad, lr, b1, b2, eps);
  SFEM_CUDA(cudaStreamSynchronize(m->L.stream));
  LRN_END
}

extern "C" int sfem_learned_train(sfem_learned *m, const float *X, const float *T, int64_t rows, int64_t batch_rows,
                                  int epochs, float lr, uint64_t seed, double *loss) {
  LRN_BEGIN
  SFEM_REQUIRE(m && X && T && rows >= 1 && rows <= (int64_t)1 << 31 && batch_rows >= 1 &&
                   batch_rows <= (int64_t)1 << 20 && epochs >= 0 && lr > 0.f,
               SFEM_EINVAL, "bad arguments");
  Learned &L = m->L;
  const int64_t nbmax = std::min(batch_rows, rows);
  ensure_cap(L, nbmax);
  uint64_t s = seed;
  for (int ep = 0; ep < epochs; ++ep) {
    // rows visited in the order r -> (a r + b) mod rows, a coprime to rows
    s = splitmix64(s);
    uint64_t a = 1 + s % (uint64_t)rows;
    s = splitmix64(s);
    const uint64_t b = s % (uint64_t)rows;
    while (std::gcd(a, (uint64_t)rows) != 1) a = a % (uint64_t)rows + 1;
    for (int64_t b0 = 0; b0 < rows; b0 += nbmax) {
      const int64_t nb = std::min(nbmax, rows - b0);
      k_gather_rows<<<grid_for(nb * (kIn + kOut), 256), 256, 0, L.stream>>>(X, T, rows, b0, nb, a, b, L.Xb, L.Tb);
      SFEM_CHECK_LAUNCH();
      loss_grad(L, L.Xb, L.Tb, nb);
      adam_step(L, L.grad, lr, 0.9f, 0.999f, 1e-8f);
    }
  }
  if (loss) {
    // mean loss over all rows with the final parameters, in batches
    SFEM_CUDA(cudaMemsetAsync(L.loss + 1, 0, sizeof(double), L.stream));
    for (int64_t b0 = 0; b0 < rows; b0 += nbmax) {
      const int64_t nb = std::min(nbmax, rows - b0);
      loss_grad(L, X + b0 * kIn, T + b0 * kOut, nb);
    }
    double acc = 0.0;
    SFEM_CUDA(cudaMemcpyAsync(&acc, L.loss + 1, sizeof(double), cudaMemcpyDeviceToHost, L.stream));
    SFEM_CUDA(cudaStreamSynchronize(L.stream));
    *loss = acc / (double)rows;
  }
  check_gemm_err(L.gemm_err, L.stream);
  LRN_END
}

extern "C" int sfem_learned_sample(sfem_learned *m, sfem_ctx *h, const double *r, const double *e, float *X, float *T) {
  LRN_BEGIN
  check_model_ctx(m, h);
  SFEM_REQUIRE(r && X && (!e || T), SFEM_EINVAL, "r and X are required (and T with e)");
  sample_into(m->L, r, e, X, T, m->L.stream);
  SFEM_CUDA(cudaStreamSynchronize(m->L.stream));
  LRN_END
}

// ============================================================================
// flexible PCG with the learned correction
// ============================================================================
namespace sfem {

struct FpcgScalars {
  double rz;        // z_k . r_k of the current direction
  double pq;        // p . A p
  double a;         // step length of the last update
  double cAc;       // c . A c
  double alpha_c;   // scale of the correction (0: Jacobi z)
  double beta;
  double rr, best_rr, tol2, rr0;
  int iter, max_iter, done, status;
  int use_learned;  // the correction is active
  int corr_off;     // 1: skip the correction kernels (done, switched off or no model)
  int fallbacks;    // iterations that fell back to z = D^-1 r
  int learned_iters, best_it, window, pace, switched_at;
  int learned_dir;  // a direction since the last restart used the correction
  int restart;      // the next direction restarts (beta = 0)
  int pad;
};

__global__ void k_fp_init(FpcgScalars *S, double tol2, int max_iter, int use_learned, int window, int pace) {
  memset(S, 0, sizeof(FpcgScalars));
  S->tol2 = tol2;
  S->max_iter = max_iter;
  S->use_learned = use_learned;
  S->corr_off = use_learned ? 0 : 1;
  S->window = window;
  S->pace = pace;
  S->switched_at = -1;
}

// c.r -> alpha_c = c.r / c.A c (0 when c.A c <= 0 or not finite)
__global__ void __launch_bounds__(256) k_fp_cr(const double *__restrict__ c, const double *__restrict__ r, int64_t n,
                                               FpcgScalars *S, double *partials, unsigned int *ticket) {
  if (S->corr_off) return;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) s += c[i] * r[i];
  double vv[1] = {s};
  if (grid_sum<256, 1>(vv, partials, ticket, nullptr) && threadIdx.x == 0) {
    const double cAc = S->cAc;
    const double ac = cAc > 0.0 ? vv[0] / cAc : 0.0;
    S->alpha_c = isfinite(ac) ? ac : 0.0;
  }
}

// first direction: z.r of both candidates, the choice, rr
__global__ void __launch_bounds__(256) k_fp_first(const double *__restrict__ r, const double *__restrict__ c,
                                                  const double *__restrict__ dinv, int64_t n, FpcgScalars *S,
                                                  double *partials, unsigned int *ticket) {
  const double ac = S->corr_off ? 0.0 : S->alpha_c;
  double zr = 0.0, jr = 0.0, rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    const double ri = r[i], jz = dinv[i] * ri;
    zr += (ac != 0.0 ? jz + ac * c[i] : jz) * ri;
    jr += jz * ri;
    rr += ri * ri;
  }
  double vv[3] = {zr, jr, rr};
  if (grid_sum<256, 3>(vv, partials, ticket, nullptr) && threadIdx.x == 0) {
    if (S->use_learned) {
      const bool ok = ac != 0.0 && vv[0] > 0.0 && isfinite(vv[0]);
      if (!ok) {
        S->fallbacks += 1;
        S->alpha_c = 0.0;
        vv[0] = vv[1];
      }
    } else {
      S->alpha_c = 0.0;
    }
    S->rz = vv[0];
    S->rr = vv[2];
    S->rr0 = vv[2];
    S->best_rr = vv[2];
    S->beta = 0.0;
    S->learned_dir = S->alpha_c != 0.0 ? 1 : 0;
    if (vv[2] <= S->tol2 || !(vv[0] > 0.0) || !isfinite(vv[0])) {
      S->done = 1;
      S->corr_off = 1;
      if (vv[2] > S->tol2) S->status = 1;
    }
  }
}

__global__ void k_fp_p0(double *__restrict__ p, double *__restrict__ q, const double *__restrict__ r,
                        const double *__restrict__ c, const double *__restrict__ dinv, int64_t n,
                        const FpcgScalars *S) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double ac = S->alpha_c;
  p[i] = dinv[i] * r[i] + (ac != 0.0 ? ac * c[i] : 0.0);
  q[i] = 0.0;
}

// x += a p, r -= a P q, rr; convergence, iteration cap, stagnation guard
__global__ void __launch_bounds__(256) k_fp_update(double *__restrict__ x, double *__restrict__ r,
                                                   const double *__restrict__ p, const double *__restrict__ q,
                                                   const uint8_t *__restrict__ dmask, int64_t n, FpcgScalars *S,
                                                   double *partials, unsigned int *ticket) {
  if (S->done) return;
  const double pq = S->pq;
  const double a = S->rz / pq;
  if (!(pq > 0.0) || !isfinite(a)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      S->status = 1;
      S->done = 1;
      S->corr_off = 1;
    }
    return;
  }
  double rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    x[i] += a * p[i];
    const double rn = dmask[i] ? r[i] - a * q[i] : 0.0;
    r[i] = rn;
    rr += rn * rn;
  }
  double vv[1] = {rr};
  if (grid_sum<256, 1>(vv, partials, ticket, nullptr) && threadIdx.x == 0) {
    S->a = a;
    S->rr = vv[0];
    S->iter += 1;
    if (S->use_learned) {
      S->learned_iters += 1;
      bool off = false;
      if (vv[0] < 0.81 * S->best_rr) {  // ||r|| at least 10% below its best
        S->best_rr = vv[0];
        S->best_it = S->iter;
      } else if (S->iter - S->best_it >= S->window) {
        off = true;
      }
      if (S->pace > 0 && S->rr0 > S->tol2) {
        // keep pace with Jacobi-PCG: ||r|| within a factor 30 of the line
        // from ||r_0|| down to the tolerance over `pace` iterations (log scale)
        const double t = fmin((double)S->iter / S->pace, 1.0);
        const double target = S->rr0 * pow(S->tol2 / S->rr0, t);
        if (vv[0] > 900.0 * target) off = true;
      }
      if (off) {
        S->use_learned = 0;
        S->corr_off = 1;
        S->alpha_c = 0.0;
        S->restart = S->learned_dir;  // learned directions in the history: restart
        S->switched_at = S->iter;
      }
    }
    if (vv[0] <= S->tol2 || S->iter >= S->max_iter || !isfinite(vv[0])) {
      S->done = 1;
      S->corr_off = 1;
      if (!isfinite(vv[0])) S->status = 1;
    }
  }
}

// z.r and z.(P q) for the learned and the Jacobi z; the choice; flexible
// (Polak-Ribiere) beta = z_{k+1}.(r_{k+1} - r_k) / z_k.r_k with
// r_{k+1} - r_k = -a P q (z vanishes on prescribed DOFs)
__global__ void __launch_bounds__(256) k_fp_zsums(const double *__restrict__ r, const double *__restrict__ q,
                                                  const double *__restrict__ c, const double *__restrict__ dinv,
                                                  int64_t n, FpcgScalars *S, double *partials, unsigned int *ticket) {
  if (S->done) return;
  const double ac = S->corr_off ? 0.0 : S->alpha_c;
  double zr = 0.0, zq = 0.0, jr = 0.0, jq = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    const double ri = r[i], qi = q[i];
    const double jz = dinv[i] * ri;
    const double z = ac != 0.0 ? jz + ac * c[i] : jz;
    zr += z * ri;
    zq += z * qi;
    jr += jz * ri;
    jq += jz * qi;
  }
  double vv[4] = {zr, zq, jr, jq};
  if (grid_sum<256, 4>(vv, partials, ticket, nullptr) && threadIdx.x == 0) {
    if (S->use_learned) {
      const bool ok = ac != 0.0 && vv[0] > 0.0 && isfinite(vv[0]) && isfinite(vv[1]);
      if (!ok) {
        S->fallbacks += 1;
        S->alpha_c = 0.0;
        vv[0] = vv[2];
        vv[1] = vv[3];
      }
    } else {
      S->alpha_c = 0.0;
      vv[0] = vv[2];
      vv[1] = vv[3];
    }
    S->beta = S->restart ? 0.0 : -S->a * vv[1] / S->rz;
    if (S->restart) S->learned_dir = 0;
    S->restart = 0;
    if (S->alpha_c != 0.0) S->learned_dir = 1;
    S->rz = vv[0];
    if (!(vv[0] > 0.0) || !isfinite(vv[0])) {
      S->status = 1;
      S->done = 1;
      S->corr_off = 1;
    }
  }
}

// p = z + beta p with z = D^-1 r + alpha_c c; q = 0 when the operator accumulates
__global__ void __launch_bounds__(256) k_fp_dir(double *__restrict__ p, double *__restrict__ q,
                                                const double *__restrict__ r, const double *__restrict__ c,
                                                const double *__restrict__ dinv, int64_t n, const FpcgScalars *S,
                                                bool zero_q) {
  if (S->done) return;
  const double ac = S->alpha_c, b = S->beta;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    p[i] = dinv[i] * r[i] + (ac != 0.0 ? ac * c[i] : 0.0) + b * p[i];
    if (zero_q) q[i] = 0.0;
  }
}

struct FpcgRun {
  Ctx &c;
  Learned *L;
  int op;
  int chunk;
  double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *cv = nullptr, *Ac = nullptr;
  float *Y = nullptr;
  FpcgScalars *S = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  size_t nodes = 0;

  FpcgRun(Ctx &c_, Learned *L_, int op_, int chunk_) : c(c_), L(L_), op(op_), chunk(chunk_) {}
  ~FpcgRun() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }

  // c from the current r (pool, MLP, prolongation), c.A c by the FP32 tiled
  // operator, alpha_c; every kernel returns at once while S->corr_off
  void enqueue_correction(cudaStream_t st) {
    if (!L) return;
    const int *off = &S->corr_off;
    k_pool<<<L->P, kPoolThreads, 0, st>>>(r, L->pnodes, L->poff, L->pooled, L->scale, L->partials, L->tickets + 3,
                                         off);
    SFEM_CHECK_LAUNCH();
    k_mlp_infer<true><<<(unsigned)((L->P + kInferRows - 1) / kInferRows), kHid, 0, st>>>(
        nullptr, L->pooled, L->scale, L->g, L->P, L->wbf, L->theta, Y, off);
    SFEM_CHECK_LAUNCH();
    k_prolong<<<grid_for(c.n_nodes, 256), 256, 0, st>>>(Y, L->g, c.xyz, c.n_nodes, c.dmask, cv, Ac, off);
    SFEM_CHECK_LAUNCH();
    SFEM_CUDA(cudaMemsetAsync(&S->cAc, 0, sizeof(double), st));  // the apply accumulates c.A c
    launch_mf32_tiled<double, double>(c, st, cv, Ac, &S->cAc, off);
    k_fp_cr<<<c.red_blocks, 256, 0, st>>>(cv, r, c.ndof, S, c.red_partial, c.tickets + 7);
    SFEM_CHECK_LAUNCH();
  }

  void enqueue_iteration(cudaStream_t st) {
    const int *done = &S->done;
    const int64_t n = c.ndof;
    if (op == SFEM_OP_CSR64) {
      launch_csr64(c, st, p, q, p, &S->pq, done);
    } else {
      double *w = static_cast<double *>(c.w_scratch);
      launch_mf_strain<double, double>(c, st, c.Gs64, p, 1, w, done);
      launch_mf_stress<double, double>(c, st, c.Gs64, c.kap64, w, q, 1, &S->pq, done);
    }
    k_fp_update<<<c.red_blocks, 256, 0, st>>>(x, r, p, q, c.dmask, n, S, c.red_partial, c.tickets + 8);
    SFEM_CHECK_LAUNCH();
    enqueue_correction(st);
    k_fp_zsums<<<c.red_blocks, 256, 0, st>>>(r, q, cv, c.dinv64, n, S, c.red_partial, c.tickets + 9);
    SFEM_CHECK_LAUNCH();
    k_fp_dir<<<c.red_blocks, 256, 0, st>>>(p, q, r, cv, c.dinv64, n, S, op != SFEM_OP_CSR64);
    SFEM_CHECK_LAUNCH();
  }

  void build() {
    SFEM_CUDA(cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal));
    set_capturing(true);
    try {
      for (int i = 0; i < chunk; ++i) enqueue_iteration(c.cap_stream);
    } catch (...) {
      set_capturing(false);
      cudaGraph_t gr = nullptr;
      cudaStreamEndCapture(c.cap_stream, &gr);
      if (gr) cudaGraphDestroy(gr);
      throw;
    }
    set_capturing(false);
    SFEM_CUDA(cudaStreamEndCapture(c.cap_stream, &graph));
    SFEM_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    SFEM_CUDA(cudaGraphGetNodes(graph, nullptr, &nodes));
  }

  // r holds the masked true residual: start flexible CG from it.  Before
  // the first and after every further chunk of iterations, `snap` (if set)
  // sees x and r.
  FpcgScalars run(double tol2, int max_iter, bool learned, int window, int pace, const Snapshot *snap, int iter0) {
    k_fp_init<<<1, 1, 0, c.stream>>>(S, tol2, max_iter, learned ? 1 : 0, window, pace);
    SFEM_CHECK_LAUNCH();
    if (learned) enqueue_correction(c.stream);
    k_fp_first<<<c.red_blocks, 256, 0, c.stream>>>(r, cv, c.dinv64, c.ndof, S, c.red_partial, c.tickets + 9);
    SFEM_CHECK_LAUNCH();
    k_fp_p0<<<grid_for(c.ndof, 256), 256, 0, c.stream>>>(p, q, r, cv, c.dinv64, c.ndof, S);
    SFEM_CHECK_LAUNCH();
    if (snap && *snap) (*snap)(x, r, iter0);
    if (!exec) build();
    FpcgScalars h{};
    SFEM_CUDA(cudaMemcpyAsync(&h, S, sizeof h, cudaMemcpyDeviceToHost, c.stream));
    SFEM_CUDA(cudaStreamSynchronize(c.stream));
    const int64_t max_launch = (int64_t)max_iter / chunk + 2;
    for (int64_t launched = 0; !h.done && launched < max_launch; ++launched) {
      SFEM_CUDA(cudaGraphLaunch(exec, c.stream));
      count_launches((int64_t)nodes);
      SFEM_CUDA(cudaMemcpyAsync(&h, S, sizeof h, cudaMemcpyDeviceToHost, c.stream));
      SFEM_CUDA(cudaStreamSynchronize(c.stream));
      if (snap && *snap && !h.done) (*snap)(x, r, iter0 + h.iter);
    }
    return h;
  }
};

void solve_fpcg(Ctx &c, const void *learned, int op64, double *x, double *r, double bnorm, double tol, int max_iter,
                int chunk, int window, int pace, sfem_solve_info &info, const std::function<double()> &true_residual,
                const Snapshot *snap) {
  Learned *L = nullptr;
  if (learned) {
    L = &const_cast<sfem_learned *>(static_cast<const sfem_learned *>(learned))->L;
    SFEM_REQUIRE(L->n_nodes == c.n_nodes && L->device == c.device, SFEM_EINVAL,
                 "the learned model was created on another mesh or device");
    SFEM_REQUIRE(L->stream == c.stream, SFEM_EINVAL, "model and context must share a stream");
  }
  std::vector<void *> own;
  auto get = [&](size_t bytes) {
    void *p = c.mem.raw(bytes);
    own.push_back(p);
    return p;
  };
  int status = SFEM_OK, total = 0, restarts = 0, fallbacks = 0, learned_iters = 0;
  double rel = 0.0;
  try {
    const int64_t n = c.ndof;
    FpcgRun R(c, L, op64, chunk);
    R.x = x;
    R.r = r;
    R.p = (double *)get(n * sizeof(double));
    R.q = (double *)get(n * sizeof(double));
    R.cv = (double *)get(n * sizeof(double));
    R.Ac = (double *)get(n * sizeof(double));
    R.S = (FpcgScalars *)get(sizeof(FpcgScalars));
    if (L) R.Y = (float *)get((size_t)L->P * kOut * sizeof(float));
    SFEM_CUDA(cudaMemsetAsync(R.cv, 0, n * sizeof(double), c.stream));
    if (op64 == SFEM_OP_MF64) ensure_w_scratch(c, (size_t)c.n_tets * 8 * sizeof(double));
    rel = true_residual();
    bool learned_on = L != nullptr;
    while (rel > tol && total < max_iter && restarts <= 10) {
      FpcgScalars s = R.run(tol * tol * bnorm * bnorm, max_iter - total, learned_on, window, pace, snap, total);
      total += s.iter;
      fallbacks += s.fallbacks;
      learned_iters += s.learned_iters;
      if (!s.use_learned) learned_on = false;  // switched off by the guard: stays off
      ++restarts;
      rel = true_residual();
      if (s.status) {
        status = SFEM_EBREAKDOWN;
        break;
      }
    }
  } catch (...) {
    for (void *p : own) c.mem.drop(p);
    throw;
  }
  for (void *p : own) c.mem.drop(p);
  info.iterations = total;
  info.outer_iterations = restarts;
  info.fallbacks = fallbacks;
  info.learned_iterations = learned_iters;
  info.true_relres = rel;
  info.status = (status == SFEM_OK && rel > tol) ? SFEM_ENOCONV : status;
}

}  // namespace sfem

extern "C" int sfem_learned_correction(sfem_learned *m, sfem_ctx *h, const double *r, double *z, double *alpha) {
  LRN_BEGIN
  check_model_ctx(m, h);
  SFEM_REQUIRE(r && z, SFEM_EINVAL, "r and z are required");
  Ctx &c = h->c;
  Learned &L = m->L;
  const int64_t n = c.ndof;
  std::vector<void *> own;
  try {
    double *cv = c.mem.get<double>(n);
    own.push_back(cv);
    double *Ac = c.mem.get<double>(n);
    own.push_back(Ac);
    float *Y = c.mem.get<float>((size_t)L.P * kOut);
    own.push_back(Y);
    FpcgScalars *S = c.mem.get<FpcgScalars>(1);
    own.push_back(S);
    k_fp_init<<<1, 1, 0, c.stream>>>(S, 0.0, 1, 1, 1 << 30, 0);
    SFEM_CHECK_LAUNCH();
    FpcgRun R(c, &L, SFEM_OP_MF64, 1);
    R.r = const_cast<double *>(r);
    R.cv = cv;
    R.Ac = Ac;
    R.Y = Y;
    R.S = S;
    R.enqueue_correction(c.stream);
    k_fp_first<<<c.red_blocks, 256, 0, c.stream>>>(r, cv, c.dinv64, n, S, c.red_partial, c.tickets + 9);
    SFEM_CHECK_LAUNCH();
    k_fp_p0<<<grid_for(n, 256), 256, 0, c.stream>>>(z, Ac, r, cv, c.dinv64, n, S);
    SFEM_CHECK_LAUNCH();
    FpcgScalars hs{};
    SFEM_CUDA(cudaMemcpyAsync(&hs, S, sizeof hs, cudaMemcpyDeviceToHost, c.stream));
    SFEM_CUDA(cudaStreamSynchronize(c.stream));
    if (alpha) *alpha = hs.alpha_c;
  } catch (...) {
    for (void *p : own) c.mem.drop(p);
    throw;
  }
  for (void *p : own) c.mem.drop(p);
  LRN_END
}

extern "C" int sfem_learned_collect(sfem_learned *m, sfem_ctx *h, const sfem_solve_opts *opts, const double *u_star,
                                    float *X, float *T, int64_t cap_rows, int64_t *rows, sfem_solve_info *info) {
  LRN_BEGIN
  check_model_ctx(m, h);
  SFEM_REQUIRE(opts && u_star && X && T && rows && cap_rows >= 0, SFEM_EINVAL, "bad arguments");
  SFEM_REQUIRE(opts->kind == SFEM_SOLVE_FPCG_LEARNED, SFEM_EINVAL, "collect runs the flexible PCG kind");
  SFEM_REQUIRE(!opts->learned || opts->learned == (const void *)m, SFEM_EINVAL,
               "opts->learned must be NULL (Jacobi trajectory) or this model");
  Ctx &c = h->c;
  Learned &L = m->L;
  *rows = 0;
  std::vector<void *> own;
  int64_t written = 0;
  sfem_solve_info local{};
  try {
    double *e = c.mem.get<double>(c.ndof);
    own.push_back(e);
    double *u = c.mem.get<double>(c.ndof);
    own.push_back(u);
    Snapshot snap = [&](const double *x, const double *r, int) {
      if (written + L.P > cap_rows) return;
      k_sub<<<grid_for(c.ndof, 256), 256, 0, c.stream>>>(u_star, x, c.ndof, e);
      SFEM_CHECK_LAUNCH();
      sample_into(L, r, e, X + written * kIn, T + written * kOut, c.stream);
      written += L.P;
    };
    sfem_solve_opts o = *opts;
    o.u_on_device = 1;
    o.warm_start = 0;
    solve_impl(c, nullptr, u, o, local, &snap);
    SFEM_CUDA(cudaStreamSynchronize(c.stream));
  } catch (...) {
    for (void *p : own) c.mem.drop(p);
    throw;
  }
  for (void *p : own) c.mem.drop(p);
  *rows = written;
  if (info) *info = local;
  LRN_END
}
