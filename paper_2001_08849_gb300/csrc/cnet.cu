// Learned coarse solve inside truncated flexible CG (the paper has no
// counterpart: it calls a direct solver and needs no preconditioner).
//
// The network maps a pooled residual to a coarse displacement correction on
// the coarse space of the two-level preconditioner (coarse.cu: trilinear
// functions of a grid of patch centres, Pi masked by P):
//   r_c = Pi^T r (the restriction: a weighted pooling of r over the cells
//         around each centre), x = r_c / RMS(r_c);
//   y   = MLP(x): n_c -> H -> GELU -> H -> GELU -> n_c (n_c = 3 x centres,
//         H = 128 by default), BF16 weights, FP32 biases and accumulation;
//   z   = D^-1 r + alpha P Pi y,  alpha = y.r_c / y.A_c y
// (P Pi y . r = y.r_c and P Pi y . A P Pi y = y.A_c y: alpha is the A-optimal
// step along the correction, computed on the coarse level from the FP32
// packed A_c kept by the coarse setup; alpha = 0 when y.A_c y <= 0 or is not
// finite, counted as a fallback).  Training pairs are (x, t) with
// t = A_c^-1 r_c / RMS: the Galerkin coarse solution, whose prolongation is
// the A-orthogonal projection of the error onto the coarse space.  The pairs
// come from the library's own solves (sfem_cnet_solve with a row buffer),
// first of Jacobi-PCG, then of the learned solver itself (on-policy rounds).
//
// The solver is flexible CG with each new direction A-orthogonalised
// against the last m (1 <= m <= 8) directions: z = M_k r, p = z -
// sum_j (q_j.z / p_j.q_j) p_j, q = A p, x += a p, r -= a q with a = p.r / p.q.
// With the Jacobi preconditioner alone this is Jacobi-PCG.  A captured
// graph holds m iterations (direction slot j in graph position j) and is
// replayed until a device flag says stop; the FP64 true residual judges
// convergence, as for the other solvers.

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "coarse.cuh"
#include "mlp.cuh"
#include "reduce.cuh"
#include "sfem_internal.cuh"

namespace sfem {

constexpr int kCnMaxM = 8;        // longest direction window
constexpr int kCnMaxHid = 256;    // widest hidden layer
constexpr int kCnL1Blocks = 64;   // input chunks of the first layer's GEMV
constexpr int kCnOutThreads = 256;

struct CNet {
  int device = 0;
  cudaStream_t stream = nullptr;
  Allocator mem;
  int64_t n_nodes = 0;
  int nc = 0, npad = 0, hid = 0;
  int64_t np = 0, oW1 = 0, oB1 = 0, oW2 = 0, oB2 = 0, oW3 = 0, oB3 = 0;
  float *theta = nullptr, *mom = nullptr, *vel = nullptr, *grad = nullptr;
  __nv_bfloat16 *wbf = nullptr;  // BF16 copies of theta (the inference weights)
  int step = 0;
  // inference scratch
  float *part = nullptr;   // kCnL1Blocks x (hid + 1): first-layer partial sums and sum r_c^2
  float *h2 = nullptr;     // hid
  float *y = nullptr;      // npad (zero beyond nc)
  double *partials = nullptr;
  unsigned int *tickets = nullptr;  // 8, zero between kernels
  double *loss = nullptr;           // 2
  // training scratch for `cap` rows
  int64_t cap = 0;
  float *Xb = nullptr, *Tb = nullptr, *a1 = nullptr, *h1b = nullptr, *a2 = nullptr, *h2b = nullptr, *yb = nullptr,
        *dy = nullptr, *d2 = nullptr, *d1 = nullptr;
  float *split = nullptr;
  size_t split_floats = 0;
  int *gemm_err = nullptr;  // set by a tensor-core GEMM whose wait ran out
};

// device scalars of one solve (and of one correction)
struct CnScalars {
  double tol2, rr, pr, yr, yAy, alpha;
  double d[kCnMaxM];     // p_j . q_j of the directions in the window
  double beta[kCnMaxM];  // q_j . z / d_j for the current direction
  double s;              // RMS of r_c (0: no correction this iteration)
  int iter, max_iter, m, done, status, fallbacks;
  int snap_every, snap_skip, rows, cap;  // row collection (snap_every 0: none)
};

__device__ __forceinline__ float bf(__nv_bfloat16 v) { return __bfloat162float(v); }

// He-normal weights (std sqrt(2/fan_in) into a GELU, sqrt(1/fan_in) for the
// linear output layer) by Box-Muller on splitmix64 uniforms; zero biases
__global__ void k_cn_init(float *theta, __nv_bfloat16 *wbf, int64_t np, int64_t oB1, int64_t oW2, int64_t oB2,
                          int64_t oW3, int64_t oB3, int n_in, int hid, uint64_t seed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  float sd = 0.f;
  if (i < oB1)
    sd = sqrtf(2.f / n_in);
  else if (i >= oW2 && i < oB2)
    sd = sqrtf(2.f / hid);
  else if (i >= oW3 && i < oB3)
    sd = sqrtf(1.f / hid);
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

// ---- inference: one input vector (the solver's restricted residual) -------
// first layer, partial sums over input chunk g = blockIdx.x:
// part[g][j] = sum_i rc_i W1[i][j], part[g][hid] = sum_i rc_i^2 (rc raw;
// the 1/RMS scaling is applied after the sum)
__global__ void k_cn_l1(const float *__restrict__ rc, int nc, const __nv_bfloat16 *__restrict__ W1, int hid,
                        float *__restrict__ part, const int *skip) {
  if (skip && *skip) return;
  const int per = (nc + gridDim.x - 1) / gridDim.x;
  const int i0 = blockIdx.x * per, i1 = min(nc, i0 + per);
  const int j = threadIdx.x;  // blockDim.x == hid
  float s = 0.f, q = 0.f;
  for (int i = i0; i < i1; ++i) {
    const float x = rc[i];
    s = fmaf(x, bf(W1[(int64_t)i * hid + j]), s);
    if (j == 0) q = fmaf(x, x, q);
  }
  part[(int64_t)blockIdx.x * (hid + 1) + j] = s;
  if (j == 0) part[(int64_t)blockIdx.x * (hid + 1) + hid] = q;
}

// hidden layers (one block of hid threads): RMS s of rc, h1 = GELU(a1 / s +
// b1) with a1 the summed partials, h2 = GELU(W2^T h1 + b2); s -> *s_out
__global__ void k_cn_mid(const float *__restrict__ part, int nblk, int nc, const __nv_bfloat16 *__restrict__ W2,
                         const float *__restrict__ b1, const float *__restrict__ b2, int hid, float *__restrict__ h2,
                         double *s_out, const int *skip) {
  if (skip && *skip) return;
  __shared__ float h1[kCnMaxHid];
  __shared__ float ss;
  const int j = threadIdx.x;
  if (j == 0) {
    double q = 0.0;
    for (int g = 0; g < nblk; ++g) q += (double)part[(int64_t)g * (hid + 1) + hid];
    ss = (float)sqrt(q / nc);
    *s_out = (double)ss;
  }
  __syncthreads();
  const float s = ss;
  float a = 0.f;
  for (int g = 0; g < nblk; ++g) a += part[(int64_t)g * (hid + 1) + j];
  h1[j] = s > 0.f ? gelu_f(a / s + b1[j]) : 0.f;
  __syncthreads();
  float a2 = b2[j];
  for (int k = 0; k < hid; ++k) a2 = fmaf(h1[k], bf(W2[(int64_t)k * hid + j]), a2);
  h2[j] = s > 0.f ? gelu_f(a2) : 0.f;
}

// output layer y_k = sum_j h2_j W3[j][k] + b3_k (k < nc; 0 beyond, up to
// npad) and y.rc (deterministic grid sum into *yr)
__global__ void __launch_bounds__(kCnOutThreads) k_cn_out(const float *__restrict__ h2, const __nv_bfloat16 *__restrict__ W3,
                                                          const float *__restrict__ b3, const float *__restrict__ rc,
                                                          int nc, int npad, int hid, float *__restrict__ y,
                                                          const double *s, double *partials, unsigned int *ticket,
                                                          double *yr, const int *skip) {
  if (skip && *skip) return;
  __shared__ float hs[kCnMaxHid];
  for (int j = threadIdx.x; j < hid; j += blockDim.x) hs[j] = h2[j];
  __syncthreads();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  double part = 0.0;
  if (k < npad) {
    float v = 0.f;
    if (k < nc && *s > 0.0) {
      v = b3[k];
      for (int j = 0; j < hid; ++j) v = fmaf(hs[j], bf(W3[(int64_t)j * nc + k]), v);
      part = (double)v * (double)rc[k];
    }
    y[k] = v;
  }
  double vv[1] = {part};
  if (grid_sum<kCnOutThreads, 1>(vv, partials, ticket, nullptr) && threadIdx.x == 0) *yr = vv[0];
}

// q = y^T A_c y over the packed lower 64 x 64 blocks of A_c (one CTA per
// block, off-diagonal blocks counted twice; deterministic grid sum); the last
// block sets alpha = y.rc / q (0, and a fallback counted, when q <= 0 or the
// step is not finite)
__global__ void __launch_bounds__(256) k_cn_quad(const float *__restrict__ Ap, const float *__restrict__ y, int nb,
                                                 CnScalars *S, double *partials, unsigned int *ticket,
                                                 const int *skip) {
  if (skip && *skip) return;
  const int t = blockIdx.x;
  int a = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((a + 1) * (a + 2) / 2 <= t) ++a;
  while (a * (a + 1) / 2 > t) --a;
  const int b = t - a * (a + 1) / 2;
  constexpr int kB = 64;
  const float *blk = Ap + (int64_t)t * kB * kB;
  double s = 0.0;
  for (int e = threadIdx.x; e < kB * kB; e += 256) {
    const int i = e / kB, j = e - (e / kB) * kB;
    s += (double)y[a * kB + i] * (double)blk[e] * (double)y[b * kB + j];
  }
  if (a != b) s *= 2.0;
  double vv[1] = {s};
  if (grid_sum<256, 1>(vv, partials, ticket, nullptr) && threadIdx.x == 0) {
    S->yAy = vv[0];
    const double al = S->yr / vv[0];
    if (S->s > 0.0 && vv[0] > 0.0 && isfinite(al)) {
      S->alpha = al;
    } else {
      S->alpha = 0.0;
      if (S->s > 0.0) S->fallbacks += 1;
    }
  }
}

// (Pi y)_i for DOF i = 3 node + c (not masked), y on the coarse DOFs
__device__ __forceinline__ float cn_prolong(const CoarseDev &cs, const float *__restrict__ y, int64_t i) {
  const int64_t node = i / 3;
  const int c = (int)(i - 3 * node);
  const int ci = cs.cinfo[node];
  const int base = ci & 0xFFFFFF;
  const int ox = ((ci >> 24) & 1) ? 3 * cs.d[1] * cs.d[2] : 0;
  const int oy = ((ci >> 25) & 1) ? 3 * cs.d[2] : 0;
  const int oz = ((ci >> 26) & 1) ? 3 : 0;
  const float f[3] = {cs.frac[3 * node], cs.frac[3 * node + 1], cs.frac[3 * node + 2]};
  const float *yb = y + 3 * base + c;
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    s = fmaf(cs_weight(f, k), yb[((k & 4) ? ox : 0) + ((k & 2) ? oy : 0) + ((k & 1) ? oz : 0)], s);
  return s;
}

// z = D^-1 r + alpha P Pi y (alpha 0: Jacobi)
__global__ void k_cn_z(CoarseDev cs, const float *__restrict__ y, const double *__restrict__ r,
                       const double *__restrict__ dinv, const uint8_t *__restrict__ dmask, int64_t n,
                       const CnScalars *S, double *__restrict__ z) {
  if (S->done) return;
  const double al = S->alpha;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = dinv[i] * r[i];
    if (al != 0.0 && dmask[i]) v += al * (double)cn_prolong(cs, y, i);
    z[i] = v;
  }
}

// snapshot decision for this iteration: skip = (no collection, or not a
// snapshot iteration, or the row buffer is full, or done)
__global__ void k_cn_snap_flag(CnScalars *S) {
  S->snap_skip = (S->done || S->snap_every <= 0 || S->rows >= S->cap || S->iter % S->snap_every != 0) ? 1 : 0;
}

// one training row: X = rc / RMS(rc), T = yc / RMS(yc) (yc = A_c^-1 rc from
// the exact coarse product); single block
__global__ void k_cn_snap(const float *__restrict__ rc, const float *__restrict__ yc, int nc, CnScalars *S,
                          float *__restrict__ X, float *__restrict__ T) {
  if (S->snap_skip) return;
  __shared__ double red[2][32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    a += (double)rc[i] * rc[i];
    b += (double)yc[i] * yc[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  __shared__ float inv[2];
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      sa += red[0][w];
      sb += red[1][w];
    }
    sa = sqrt(sa / nc);
    sb = sqrt(sb / nc);
    inv[0] = sa > 0.0 ? (float)(1.0 / sa) : 0.f;
    inv[1] = sb > 0.0 ? (float)(1.0 / sb) : 0.f;
  }
  __syncthreads();
  const int64_t row = S->rows;
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    X[row * nc + i] = rc[i] * inv[0];
    T[row * nc + i] = yc[i] * inv[1];
  }
  __syncthreads();
  if (threadIdx.x == 0 && inv[0] > 0.f) S->rows = (int)row + 1;
}

// ---- truncated flexible CG ----------------------------------------------------
__global__ void k_fcg_init(CnScalars *S, double tol2, int max_iter, int m, int snap_every, int cap, int rows0) {
  S->tol2 = tol2;
  S->rr = 0.0;
  S->pr = 0.0;
  S->yr = 0.0;
  S->yAy = 0.0;
  S->alpha = 0.0;
  S->s = 0.0;
  for (int j = 0; j < kCnMaxM; ++j) S->d[j] = 0.0, S->beta[j] = 0.0;
  S->iter = 0;
  S->max_iter = max_iter;
  S->m = m;
  S->done = max_iter <= 0 ? 1 : 0;
  S->status = 0;
  S->fallbacks = 0;
  S->snap_every = snap_every;
  S->snap_skip = 1;
  S->rows = rows0;
  S->cap = cap;
}

// beta_j = q_j . z / d_j over the last min(iter, m) directions; the direction
// being formed goes into slot `slot`, so the previous ones are slot - 1,
// slot - 2, ... (mod m).  Q holds m pointers (slot order).
struct CnRing {
  double *P[kCnMaxM];
  double *Q[kCnMaxM];
};

__global__ void __launch_bounds__(256) k_fcg_beta(CnRing R, const double *__restrict__ z, int64_t n, int slot,
                                                  CnScalars *S, double *partials, unsigned int *ticket) {
  if (S->done) return;
  const int m = S->m, cnt = min(S->iter, m);
  double acc[kCnMaxM];
#pragma unroll
  for (int k = 0; k < kCnMaxM; ++k) acc[k] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    const double zi = z[i];
#pragma unroll
    for (int k = 0; k < kCnMaxM; ++k)
      if (k < cnt) acc[k] += R.Q[(slot - 1 - k + m) % m][i] * zi;
  }
  if (grid_sum<256, kCnMaxM>(acc, partials, ticket, nullptr) && threadIdx.x == 0)
    for (int k = 0; k < kCnMaxM; ++k) {
      double bk = 0.0;
      if (k < cnt) {
        const int j = (slot - 1 - k + m) % m;
        if (S->d[j] > 0.0) bk = acc[k] / S->d[j];
      }
      S->beta[k] = bk;
    }
}

// p_slot = z - sum_k beta_k p_(slot-1-k); p.r; q_slot = 0 when the operator
// accumulates into it
__global__ void __launch_bounds__(256) k_fcg_dir(CnRing R, const double *__restrict__ z,
                                                 const double *__restrict__ r, int64_t n, int slot, CnScalars *S,
                                                 bool zero_q, double *partials, unsigned int *ticket) {
  if (S->done) return;
  const int m = S->m, cnt = min(S->iter, m);
  double b[kCnMaxM];
  const double *Pk[kCnMaxM];
#pragma unroll
  for (int k = 0; k < kCnMaxM; ++k) {
    b[k] = k < cnt ? S->beta[k] : 0.0;
    Pk[k] = k < m ? R.P[(slot - 1 - k + m) % m] : nullptr;
  }
  double *p = R.P[slot];
  double *q = R.Q[slot];
  double pr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    double v = z[i];
#pragma unroll
    for (int k = 0; k < kCnMaxM; ++k)
      if (k < cnt) v -= b[k] * Pk[k][i];
    p[i] = v;  // (slot's old direction, if any, was read above as Pk[m-1][i])
    pr += v * r[i];
    if (zero_q) q[i] = 0.0;
  }
  double vv[1] = {pr};
  if (grid_sum<256, 1>(vv, partials, ticket, nullptr) && threadIdx.x == 0) S->pr = vv[0];
}

// x += a p, r -= a P q (a = p.r / p.q), rr; stop at rr <= tol2 or the cap;
// a direction with p.q <= 0 or a non-finite step is a breakdown
__global__ void __launch_bounds__(256) k_fcg_update(double *__restrict__ x, double *__restrict__ r, CnRing R,
                                                    const uint8_t *__restrict__ dmask, int64_t n, int slot,
                                                    CnScalars *S, double *partials, unsigned int *ticket) {
  if (S->done) return;
  const double d = S->d[slot];
  const double a = S->pr / d;
  if (!(d > 0.0) || !isfinite(a)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      S->status = 1;
      S->done = 1;
    }
    return;
  }
  const double *p = R.P[slot], *q = R.Q[slot];
  double rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    x[i] += a * p[i];
    const double rn = dmask[i] ? r[i] - a * q[i] : 0.0;
    r[i] = rn;
    rr += rn * rn;
  }
  double vv[1] = {rr};
  if (grid_sum<256, 1>(vv, partials, ticket, nullptr) && threadIdx.x == 0) {
    S->rr = vv[0];
    S->iter += 1;
    if (vv[0] <= S->tol2 || S->iter >= S->max_iter) S->done = 1;
  }
}

// ---- training (FP32 master weights) -------------------------------------------
// rows of (X, T) (n features each) in the order r -> (a r + b) mod rows
__global__ void k_cn_gather_rows(const float *__restrict__ X, const float *__restrict__ T, int64_t rows, int n,
                                 int64_t first, int64_t nb, uint64_t a, uint64_t b, float *__restrict__ Xb,
                                 float *__restrict__ Tb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb * 2 * n) return;
  const int64_t r = i / (2 * n);
  const int f = (int)(i % (2 * n));
  const uint64_t R = (uint64_t)rows;
  const int64_t src = (int64_t)(((a % R) * ((uint64_t)(first + r) % R) % R + b) % R);
  if (f < n)
    Xb[r * n + f] = X[src * n + f];
  else
    Tb[r * n + f - n] = T[src * n + f - n];
}

static void cn_gemm(CNet &L, int M, int N, int K, const float *A, int lda, bool tA, const float *B, int ldb, bool tB,
                    float *C, int ldc) {
  mlp_gemm(L.mem, L.split, L.split_floats, L.stream, M, N, K, A, lda, tA, B, ldb, tB, C, ldc, L.gemm_err);
}

static void cn_ensure_cap(CNet &L, int64_t rows) {
  if (rows <= L.cap) return;
  for (float *p : {L.Xb, L.Tb, L.a1, L.h1b, L.a2, L.h2b, L.yb, L.dy, L.d2, L.d1})
    if (p) L.mem.drop(p);
  const int64_t n = L.nc, h = L.hid;
  L.Xb = L.mem.get<float>(rows * n);
  L.Tb = L.mem.get<float>(rows * n);
  L.a1 = L.mem.get<float>(rows * h);
  L.h1b = L.mem.get<float>(rows * h);
  L.a2 = L.mem.get<float>(rows * h);
  L.h2b = L.mem.get<float>(rows * h);
  L.yb = L.mem.get<float>(rows * n);
  L.dy = L.mem.get<float>(rows * n);
  L.d2 = L.mem.get<float>(rows * h);
  L.d1 = L.mem.get<float>(rows * h);
  L.cap = rows;
}

// forward with cached activations, loss sum((y - T)^2) / rows (L.loss[0];
// L.loss[1] += sum) and its gradient into L.grad, by the chain rule
static void cn_loss_grad(CNet &L, const float *X, const float *T, int64_t rows) {
  cn_ensure_cap(L, rows);
  cudaStream_t st = L.stream;
  const int n = L.nc, h = L.hid, r = (int)rows;
  const float *W1 = L.theta + L.oW1, *W2 = L.theta + L.oW2, *W3 = L.theta + L.oW3;
  const int gh = grid_for(rows * h, 256);
  cn_gemm(L, r, h, n, X, n, false, W1, h, false, L.a1, h);
  k_bias_gelu<<<gh, 256, 0, st>>>(L.a1, L.h1b, L.theta + L.oB1, rows, h);
  SFEM_CHECK_LAUNCH();
  cn_gemm(L, r, h, h, L.h1b, h, false, W2, h, false, L.a2, h);
  k_bias_gelu<<<gh, 256, 0, st>>>(L.a2, L.h2b, L.theta + L.oB2, rows, h);
  SFEM_CHECK_LAUNCH();
  cn_gemm(L, r, n, h, L.h2b, h, false, W3, n, false, L.yb, n);
  k_bias_gelu<<<grid_for(rows * n, 256), 256, 0, st>>>(L.yb, nullptr, L.theta + L.oB3, rows, n);
  SFEM_CHECK_LAUNCH();
  k_mse<<<(unsigned)std::min<int64_t>(grid_for(rows * n, 256), 512), 256, 0, st>>>(L.yb, T, rows * n, rows, L.dy,
                                                                                   L.partials, L.tickets + 5, L.loss);
  SFEM_CHECK_LAUNCH();
  float *g = L.grad;
  cn_gemm(L, h, n, r, L.h2b, h, true, L.dy, n, false, g + L.oW3, n);
  k_colsum<<<n, 256, 0, st>>>(L.dy, rows, n, g + L.oB3);
  SFEM_CHECK_LAUNCH();
  cn_gemm(L, r, h, n, L.dy, n, false, W3, n, true, L.d2, h);
  k_gelu_back<<<gh, 256, 0, st>>>(L.d2, L.a2, rows * h);
  SFEM_CHECK_LAUNCH();
  cn_gemm(L, h, h, r, L.h1b, h, true, L.d2, h, false, g + L.oW2, h);
  k_colsum<<<h, 256, 0, st>>>(L.d2, rows, h, g + L.oB2);
  SFEM_CHECK_LAUNCH();
  cn_gemm(L, r, h, h, L.d2, h, false, W2, h, true, L.d1, h);
  k_gelu_back<<<gh, 256, 0, st>>>(L.d1, L.a1, rows * h);
  SFEM_CHECK_LAUNCH();
  cn_gemm(L, n, h, r, X, n, true, L.d1, h, false, g + L.oW1, h);
  k_colsum<<<h, 256, 0, st>>>(L.d1, rows, h, g + L.oB1);
  SFEM_CHECK_LAUNCH();
}

static void cn_adam(CNet &L, const float *g, float lr, float b1, float b2, float eps) {
  L.step += 1;
  const float c1 = (float)(1.0 - std::pow((double)b1, L.step));
  const float c2 = (float)(1.0 - std::pow((double)b2, L.step));
  k_adam<<<grid_for(L.np, 256), 256, 0, L.stream>>>(L.theta, g, L.mom, L.vel, (int)L.np, lr, b1, b2, eps, c1, c2,
                                                    L.wbf);
  SFEM_CHECK_LAUNCH();
}

// epochs of mini-batch Adam over rows (device X, T); returns the mean loss
// of the last epoch
static double cn_train(CNet &L, const float *X, const float *T, int64_t rows, int64_t batch, int epochs, float lr,
                       uint64_t seed) {
  batch = std::max<int64_t>(1, std::min(batch, rows));
  cn_ensure_cap(L, batch);
  double last = 0.0;
  for (int ep = 0; ep < epochs; ++ep) {
    // a -> odd multiplier coprime to rows (retry until gcd 1), b offset
    uint64_t h = splitmix64(seed * 0x9e3779b97f4a7c15ull + (uint64_t)ep);
    uint64_t a = (h | 1ull) % (uint64_t)rows;
    auto gcd = [](uint64_t x, uint64_t y) {
      while (y) {
        const uint64_t t = x % y;
        x = y;
        y = t;
      }
      return x;
    };
    while (a == 0 || gcd(a, (uint64_t)rows) != 1) a = (a + 1) % (uint64_t)rows, a = a ? a : 1;
    const uint64_t b = splitmix64(h) % (uint64_t)rows;
    SFEM_CUDA(cudaMemsetAsync(L.loss + 1, 0, sizeof(double), L.stream));
    for (int64_t f = 0; f < rows; f += batch) {
      const int64_t nb = std::min(batch, rows - f);
      k_cn_gather_rows<<<grid_for(nb * 2 * L.nc, 256), 256, 0, L.stream>>>(X, T, rows, L.nc, f, nb, a, b, L.Xb,
                                                                           L.Tb);
      SFEM_CHECK_LAUNCH();
      cn_loss_grad(L, L.Xb, L.Tb, nb);
      cn_adam(L, L.grad, lr, 0.9f, 0.999f, 1e-8f);
    }
    double s = 0.0;
    SFEM_CUDA(cudaMemcpyAsync(&s, L.loss + 1, sizeof(double), cudaMemcpyDeviceToHost, L.stream));
    SFEM_CUDA(cudaStreamSynchronize(L.stream));
    last = s / (double)rows;
  }
  check_gemm_err(L.gemm_err, L.stream);
  return last;
}

// ---- random training rows -------------------------------------------------------
// dense symmetric C (nc x nc) from its packed lower 64 x 64 blocks
__global__ void k_cn_unpack(const float *__restrict__ Cp, int nc, float *__restrict__ Cd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)nc * nc) return;
  int i = (int)(e / nc), j = (int)(e % nc);
  if (j > i) {
    const int t = i;
    i = j;
    j = t;
  }
  const int a = i / 64, b = j / 64;
  const int64_t t = (int64_t)a * (a + 1) / 2 + b;
  Cd[e] = Cp[t * 4096 + (i % 64) * 64 + (j % 64)];
}

// standard normal entries by Box-Muller on splitmix64 uniforms of (seed, index)
__global__ void k_cn_randn(float *__restrict__ X, int64_t n, uint64_t seed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t h = splitmix64(seed * 0x100000001b3ull + (uint64_t)i);
  const double u1 = (double)((h >> 11) + 1) * (1.0 / 9007199254740992.0);
  const double u2 = (double)(splitmix64(h) >> 11) * (1.0 / 9007199254740992.0);
  X[i] = (float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
}

// each row of A (rows x n) divided by its RMS (one block per row)
__global__ void k_cn_rownorm(float *__restrict__ A, int n) {
  float *row = A + (int64_t)blockIdx.x * n;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += (double)row[i] * row[i];
  s = block_sum<256>(s);
  __shared__ float inv;
  if (threadIdx.x == 0) inv = s > 0.0 ? (float)(1.0 / sqrt(s / n)) : 0.f;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) row[i] *= inv;
}

// rows [first, first + count) of (X, T): x Gaussian, t = C x, both
// normalised to unit RMS (C = A_c^-1 of the coarse setup, FP32)
static void cn_random_rows(CNet &L, const CoarseDev &cs, float *X, float *T, int64_t first, int64_t count,
                           uint64_t seed) {
  if (count <= 0) return;
  cudaStream_t st = L.stream;
  const int nc = L.nc;
  float *Cd = L.mem.get<float>((size_t)nc * nc);
  try {
    k_cn_unpack<<<grid_for((int64_t)nc * nc, 256), 256, 0, st>>>(cs.C, nc, Cd);
    SFEM_CHECK_LAUNCH();
    float *Xr = X + first * nc, *Tr = T + first * nc;
    k_cn_randn<<<grid_for(count * nc, 256), 256, 0, st>>>(Xr, count * nc, seed);
    SFEM_CHECK_LAUNCH();
    for (int64_t r0 = 0; r0 < count; r0 += 65536) {  // GEMM grids of at most 1024 row tiles
      const int nr = (int)std::min<int64_t>(65536, count - r0);
      cn_gemm(L, nr, nc, nc, Xr + r0 * nc, nc, false, Cd, nc, false, Tr + r0 * nc, nc);
    }
    k_cn_rownorm<<<(unsigned)count, 256, 0, st>>>(Xr, nc);
    SFEM_CHECK_LAUNCH();
    k_cn_rownorm<<<(unsigned)count, 256, 0, st>>>(Tr, nc);
    SFEM_CHECK_LAUNCH();
    check_gemm_err(L.gemm_err, st);
  } catch (...) {
    L.mem.drop(Cd);
    throw;
  }
  L.mem.drop(Cd);
}

// ---- inference and the solver ---------------------------------------------------
// y = MLP(rc / RMS(rc)) from the restricted residual in cs.rc, then alpha
// (S->s, S->yr, S->yAy, S->alpha); every kernel returns at once while *stop
static void cn_enqueue_net(CNet &L, const CoarseDev &cs, cudaStream_t st, CnScalars *S, const int *stop) {
  k_cn_l1<<<kCnL1Blocks, L.hid, 0, st>>>(cs.rc, L.nc, L.wbf + L.oW1, L.hid, L.part, stop);
  SFEM_CHECK_LAUNCH();
  k_cn_mid<<<1, L.hid, 0, st>>>(L.part, kCnL1Blocks, L.nc, L.wbf + L.oW2, L.theta + L.oB1, L.theta + L.oB2, L.hid,
                                L.h2, &S->s, stop);
  SFEM_CHECK_LAUNCH();
  k_cn_out<<<(unsigned)((L.npad + kCnOutThreads - 1) / kCnOutThreads), kCnOutThreads, 0, st>>>(
      L.h2, L.wbf + L.oW3, L.theta + L.oB3, cs.rc, L.nc, L.npad, L.hid, L.y, &S->s, L.partials, L.tickets + 0,
      &S->yr, stop);
  SFEM_CHECK_LAUNCH();
  const int nb = L.npad / 64;
  k_cn_quad<<<(unsigned)(nb * (nb + 1) / 2), 256, 0, st>>>(cs.Ap, L.y, nb, S, L.partials, L.tickets + 1, stop);
  SFEM_CHECK_LAUNCH();
}

struct CnRun {
  Ctx &c;
  CNet *L;
  int op, m;
  CnRunArgs *args;
  double *x = nullptr, *r = nullptr, *z = nullptr;
  CnRing ring{};
  CnScalars *S = nullptr;
  double *partials = nullptr;
  unsigned int *tickets = nullptr;  // 8
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  size_t nodes = 0;

  CnRun(Ctx &c_, CNet *L_, int op_, int m_, CnRunArgs *a_) : c(c_), L(L_), op(op_), m(m_), args(a_) {}
  ~CnRun() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }

  bool collecting() const { return args && args->snap_every > 0 && args->X && args->T; }

  // one iteration; its direction goes into ring slot `slot`
  void enqueue_iteration(cudaStream_t st, int slot) {
    const int *done = &S->done;
    const CoarseDev &cs = c.coarse->dev;
    const int64_t n = c.ndof;
    const bool coll = collecting();
    if (L || coll) coarse_restrict(c, st, r, done);
    if (coll) {
      k_cn_snap_flag<<<1, 1, 0, st>>>(S);
      SFEM_CHECK_LAUNCH();
      coarse_gemv(cs, st, &S->snap_skip);  // yc = C rc, the target
      k_cn_snap<<<1, 256, 0, st>>>(cs.rc, cs.yc, cs.nc, S, args->X, args->T);
      SFEM_CHECK_LAUNCH();
    }
    if (L) cn_enqueue_net(*L, cs, st, S, done);
    k_cn_z<<<c.red_blocks, 256, 0, st>>>(cs, L ? L->y : nullptr, r, c.dinv64, c.dmask, n, S, z);
    SFEM_CHECK_LAUNCH();
    k_fcg_beta<<<c.red_blocks, 256, 0, st>>>(ring, z, n, slot, S, partials, tickets + 2);
    SFEM_CHECK_LAUNCH();
    k_fcg_dir<<<c.red_blocks, 256, 0, st>>>(ring, z, r, n, slot, S, op != SFEM_OP_CSR64, partials, tickets + 3);
    SFEM_CHECK_LAUNCH();
    double *p = ring.P[slot], *q = ring.Q[slot];
    if (op == SFEM_OP_CSR64) {
      launch_csr64(c, st, p, q, p, &S->d[slot], done);
    } else {
      double *w = static_cast<double *>(c.w_scratch);
      launch_mf_strain<double, double>(c, st, c.Gs64, p, 1, w, done);
      launch_mf_stress<double, double>(c, st, c.Gs64, c.kap64, w, q, 1, &S->d[slot], done);
    }
    k_fcg_update<<<c.red_blocks, 256, 0, st>>>(x, r, ring, c.dmask, n, slot, S, partials, tickets + 4);
    SFEM_CHECK_LAUNCH();
  }

  void build() {
    SFEM_CUDA(cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal));
    set_capturing(true);
    try {
      for (int j = 0; j < m; ++j) enqueue_iteration(c.cap_stream, j);
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

  // flexible CG from the residual in r (x the iterate); returns the scalars
  CnScalars run(double tol2, int max_iter) {
    const int every = collecting() ? args->snap_every : 0;
    const int cap = collecting() ? (int)std::min<int64_t>(args->cap, INT32_MAX) : 0;
    const int rows0 = collecting() ? (int)args->rows : 0;
    k_fcg_init<<<1, 1, 0, c.stream>>>(S, tol2, max_iter, m, every, cap, rows0);
    SFEM_CHECK_LAUNCH();
    if (!exec) build();
    CnScalars h{};
    const int64_t max_launch = (int64_t)max_iter / m + 2;
    for (int64_t launched = 0; launched < max_launch; ++launched) {
      SFEM_CUDA(cudaGraphLaunch(exec, c.stream));
      count_launches((int64_t)nodes);
      SFEM_CUDA(cudaMemcpyAsync(&h, S, sizeof h, cudaMemcpyDeviceToHost, c.stream));
      SFEM_CUDA(cudaStreamSynchronize(c.stream));
      if (h.done) break;
    }
    if (collecting()) args->rows = h.rows;
    return h;
  }
};

static CNet &cn_model(const void *model);

void solve_cnet(Ctx &c, const void *model, CnRunArgs *args, int op64, double *x, double *r, double bnorm,
                double tol, int max_iter, sfem_solve_info &info, const std::function<double()> &true_residual) {
  CNet *L = model ? &cn_model(model) : nullptr;
  const bool coll = args && args->snap_every > 0 && args->X && args->T;
  if (L || coll) SFEM_REQUIRE(c.coarse != nullptr, SFEM_EINVAL, "FCG_CNET needs sfem_coarse_setup first");
  if (L) {
    SFEM_REQUIRE(L->device == c.device && L->stream == c.stream, SFEM_EINVAL,
                 "model and context must share a device and a stream");
    SFEM_REQUIRE(L->nc == c.coarse->dev.nc && L->npad == c.coarse->dev.npad && L->n_nodes == c.n_nodes, SFEM_EINVAL,
                 "the model was created on another mesh or coarse space");
  }
  if (coll) SFEM_REQUIRE(args->rows >= 0 && args->rows <= args->cap, SFEM_EINVAL, "rows out of range");
  const int m = args && args->window > 0 ? args->window : 5;
  SFEM_REQUIRE(m >= 1 && m <= kCnMaxM, SFEM_EINVAL, "window must be 1 .. 8");
  std::vector<void *> own;
  auto get = [&](size_t bytes) {
    void *p = c.mem.raw(bytes);
    own.push_back(p);
    return p;
  };
  int status = SFEM_OK, total = 0, restarts = 0, fallbacks = 0;
  double rel = 0.0;
  try {
    const int64_t n = c.ndof;
    CnRun R(c, L, op64, m, args);
    R.x = x;
    R.r = r;
    R.z = (double *)get(n * sizeof(double));
    for (int j = 0; j < m; ++j) {
      R.ring.P[j] = (double *)get(n * sizeof(double));
      R.ring.Q[j] = (double *)get(n * sizeof(double));
      SFEM_CUDA(cudaMemsetAsync(R.ring.P[j], 0, n * sizeof(double), c.stream));
      SFEM_CUDA(cudaMemsetAsync(R.ring.Q[j], 0, n * sizeof(double), c.stream));
    }
    for (int j = m; j < kCnMaxM; ++j) R.ring.P[j] = R.ring.Q[j] = nullptr;
    R.S = (CnScalars *)get(sizeof(CnScalars));
    const int64_t pblocks = std::max<int64_t>(c.red_blocks, 1);
    R.partials = (double *)get((size_t)kCnMaxM * pblocks * sizeof(double));
    R.tickets = (unsigned int *)get(8 * sizeof(unsigned int));
    SFEM_CUDA(cudaMemsetAsync(R.tickets, 0, 8 * sizeof(unsigned int), c.stream));
    if (op64 == SFEM_OP_MF64) ensure_w_scratch(c, (size_t)c.n_tets * 8 * sizeof(double));
    rel = true_residual();
    while (rel > tol && total < max_iter && restarts <= 10) {
      CnScalars s = R.run(tol * tol * bnorm * bnorm, max_iter - total);
      total += s.iter;
      fallbacks += s.fallbacks;
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
  info.learned_iterations = L ? total : 0;
  info.true_relres = rel;
  info.status = (status == SFEM_OK && rel > tol) ? SFEM_ENOCONV : status;
}

}  // namespace sfem

// ============================================================================
// ABI
// ============================================================================
using namespace sfem;

struct sfem_cnet {
  CNet L;
};

namespace sfem {
static CNet &cn_model(const void *model) {
  return const_cast<sfem_cnet *>(static_cast<const sfem_cnet *>(model))->L;
}
}  // namespace sfem

#define CN_BEGIN try {
#define CN_END                  \
  }                             \
  catch (const Error &err) {    \
    set_last_error(err.msg);    \
    return err.status;          \
  }                             \
  return SFEM_OK;

static void cn_check_ctx(const sfem_cnet *m, const sfem_ctx *h) {
  SFEM_REQUIRE(m && h && h->c.vol, SFEM_EINVAL, "model and context required");
  SFEM_REQUIRE(h->c.coarse != nullptr, SFEM_EINVAL, "the context has no coarse space (sfem_coarse_setup)");
  SFEM_REQUIRE(m->L.device == h->c.device && m->L.stream == h->c.stream && m->L.n_nodes == h->c.n_nodes &&
                   m->L.nc == h->c.coarse->dev.nc,
               SFEM_EINVAL, "the model was created on another context or coarse space");
}

extern "C" int sfem_cnet_create(sfem_cnet **out, sfem_ctx *h, const sfem_cnet_opts *opts) {
  CN_BEGIN
  SFEM_REQUIRE(out && h && h->c.vol, SFEM_EINVAL, "out and a set-up context are required");
  *out = nullptr;
  Ctx &c = h->c;
  SFEM_REQUIRE(c.coarse != nullptr, SFEM_EINVAL, "sfem_cnet_create needs sfem_coarse_setup first");
  const int hid = (opts && opts->hidden > 0) ? opts->hidden : 128;
  SFEM_REQUIRE(hid % 32 == 0 && hid <= kCnMaxHid, SFEM_EINVAL, "hidden must be a multiple of 32, at most 256");
  auto *m = new sfem_cnet();
  CNet &L = m->L;
  try {
    L.device = c.device;
    L.stream = c.stream;
    L.mem.alloc = c.mem.alloc;
    L.mem.free = c.mem.free;
    L.mem.user = c.mem.user;
    L.mem.stream = c.stream;
    L.n_nodes = c.n_nodes;
    L.nc = c.coarse->dev.nc;
    L.npad = c.coarse->dev.npad;
    L.hid = hid;
    const int64_t n = L.nc;
    L.oW1 = 0;
    L.oB1 = n * hid;
    L.oW2 = L.oB1 + hid;
    L.oB2 = L.oW2 + (int64_t)hid * hid;
    L.oW3 = L.oB2 + hid;
    L.oB3 = L.oW3 + (int64_t)hid * n;
    L.np = L.oB3 + n;
    SFEM_REQUIRE(L.np < (int64_t)1 << 31, SFEM_EINVAL, "network too large");
    L.theta = L.mem.get<float>(L.np);
    L.mom = L.mem.get<float>(L.np);
    L.vel = L.mem.get<float>(L.np);
    L.grad = L.mem.get<float>(L.np);
    L.wbf = L.mem.get<__nv_bfloat16>(L.np);
    SFEM_CUDA(cudaMemsetAsync(L.mom, 0, L.np * sizeof(float), L.stream));
    SFEM_CUDA(cudaMemsetAsync(L.vel, 0, L.np * sizeof(float), L.stream));
    L.part = L.mem.get<float>((size_t)kCnL1Blocks * (hid + 1));
    L.h2 = L.mem.get<float>(hid);
    L.y = L.mem.get<float>(L.npad);
    SFEM_CUDA(cudaMemsetAsync(L.y, 0, L.npad * sizeof(float), L.stream));
    const int nb = L.npad / 64;
    const int64_t pb = std::max<int64_t>({(int64_t)nb * (nb + 1) / 2, (L.npad + kCnOutThreads - 1) / kCnOutThreads, 512});
    L.partials = L.mem.get<double>(pb);
    L.tickets = L.mem.get<unsigned int>(8);
    SFEM_CUDA(cudaMemsetAsync(L.tickets, 0, 8 * sizeof(unsigned int), L.stream));
    L.loss = L.mem.get<double>(2);
    SFEM_CUDA(cudaMemsetAsync(L.loss, 0, 2 * sizeof(double), L.stream));
    L.gemm_err = L.mem.get<int>(1);
    SFEM_CUDA(cudaMemsetAsync(L.gemm_err, 0, sizeof(int), L.stream));
    k_cn_init<<<grid_for(L.np, 256), 256, 0, L.stream>>>(L.theta, L.wbf, L.np, L.oB1, L.oW2, L.oB2, L.oW3, L.oB3,
                                                         (int)n, hid, opts ? opts->seed : 0ull);
    SFEM_CHECK_LAUNCH();
    SFEM_CUDA(cudaStreamSynchronize(L.stream));
  } catch (...) {
    L.mem.release_all();
    delete m;
    throw;
  }
  *out = m;
  CN_END
}

extern "C" void sfem_cnet_destroy(sfem_cnet *m) {
  if (!m) return;
  cudaStreamSynchronize(m->L.stream);
  m->L.mem.release_all();
  delete m;
}

extern "C" int sfem_cnet_info(const sfem_cnet *m, int *n_coarse, int *hidden, int64_t *n_params) {
  CN_BEGIN
  SFEM_REQUIRE(m, SFEM_EINVAL, "model required");
  if (n_coarse) *n_coarse = m->L.nc;
  if (hidden) *hidden = m->L.hid;
  if (n_params) *n_params = m->L.np;
  CN_END
}

extern "C" int sfem_cnet_set_params(sfem_cnet *m, const float *theta, int64_t n) {
  CN_BEGIN
  SFEM_REQUIRE(m && theta && n == m->L.np, SFEM_EINVAL, "theta must hold n_params floats");
  CNet &L = m->L;
  SFEM_CUDA(cudaMemcpyAsync(L.theta, theta, n * sizeof(float), cudaMemcpyHostToDevice, L.stream));
  k_to_bf16<<<grid_for(n, 256), 256, 0, L.stream>>>(L.theta, L.wbf, (int)n);
  SFEM_CHECK_LAUNCH();
  SFEM_CUDA(cudaMemsetAsync(L.mom, 0, n * sizeof(float), L.stream));
  SFEM_CUDA(cudaMemsetAsync(L.vel, 0, n * sizeof(float), L.stream));
  L.step = 0;
  SFEM_CUDA(cudaStreamSynchronize(L.stream));
  CN_END
}

extern "C" int sfem_cnet_get_params(sfem_cnet *m, float *theta, int64_t n) {
  CN_BEGIN
  SFEM_REQUIRE(m && theta && n == m->L.np, SFEM_EINVAL, "theta must hold n_params floats");
  SFEM_CUDA(cudaMemcpyAsync(theta, m->L.theta, n * sizeof(float), cudaMemcpyDeviceToHost, m->L.stream));
  SFEM_CUDA(cudaStreamSynchronize(m->L.stream));
  CN_END
}

// Y[r] = MLP(X[r] / RMS(X[r])) by the inference path (BF16 weights); the
// rows are run one after the other through the solver's kernels
extern "C" int sfem_cnet_forward(sfem_cnet *m, sfem_ctx *h, const float *X, float *Y, int64_t rows) {
  CN_BEGIN
  cn_check_ctx(m, h);
  SFEM_REQUIRE(X && Y && rows >= 0, SFEM_EINVAL, "X, Y required");
  CNet &L = m->L;
  CoarseDev cs = h->c.coarse->dev;
  float *rc = L.mem.get<float>(L.npad);
  CnScalars *S = L.mem.get<CnScalars>(1);
  try {
    SFEM_CUDA(cudaMemsetAsync(rc, 0, L.npad * sizeof(float), L.stream));
    k_fcg_init<<<1, 1, 0, L.stream>>>(S, 0.0, 1, 1, 0, 0, 0);
    SFEM_CHECK_LAUNCH();
    cs.rc = rc;
    for (int64_t r = 0; r < rows; ++r) {
      SFEM_CUDA(cudaMemcpyAsync(rc, X + r * L.nc, L.nc * sizeof(float), cudaMemcpyDeviceToDevice, L.stream));
      cn_enqueue_net(L, cs, L.stream, S, &S->done);
      SFEM_CUDA(cudaMemcpyAsync(Y + r * L.nc, L.y, L.nc * sizeof(float), cudaMemcpyDeviceToDevice, L.stream));
    }
    SFEM_CUDA(cudaStreamSynchronize(L.stream));
  } catch (...) {
    L.mem.drop(rc);
    L.mem.drop(S);
    throw;
  }
  L.mem.drop(rc);
  L.mem.drop(S);
  CN_END
}

extern "C" int sfem_cnet_loss_grad(sfem_cnet *m, const float *X, const float *T, int64_t rows, float *grad,
                                   double *loss) {
  CN_BEGIN
  SFEM_REQUIRE(m && X && T && rows > 0, SFEM_EINVAL, "X, T and rows > 0 required");
  CNet &L = m->L;
  cn_loss_grad(L, X, T, rows);
  if (grad)
    SFEM_CUDA(cudaMemcpyAsync(grad, L.grad, L.np * sizeof(float), cudaMemcpyDeviceToDevice, L.stream));
  double lh[2];
  SFEM_CUDA(cudaMemcpyAsync(lh, L.loss, sizeof lh, cudaMemcpyDeviceToHost, L.stream));
  check_gemm_err(L.gemm_err, L.stream);
  if (loss) *loss = lh[0];
  CN_END
}

extern "C" int sfem_cnet_train(sfem_cnet *m, const float *X, const float *T, int64_t rows, int64_t batch_rows,
                               int epochs, float lr, uint64_t seed, double *loss) {
  CN_BEGIN
  SFEM_REQUIRE(m && X && T && rows > 0 && epochs >= 0 && lr > 0.f, SFEM_EINVAL, "bad training arguments");
  const double l = cn_train(m->L, X, T, rows, batch_rows > 0 ? batch_rows : 1024, epochs, lr, seed);
  if (loss) *loss = l;
  CN_END
}

// z = D^-1 r + alpha P Pi MLP(Pi^T r / RMS) for one residual; alpha to host
extern "C" int sfem_cnet_correction(sfem_cnet *m, sfem_ctx *h, const double *r, double *z, double *alpha) {
  CN_BEGIN
  cn_check_ctx(m, h);
  SFEM_REQUIRE(r && z, SFEM_EINVAL, "r and z are required");
  Ctx &c = h->c;
  CNet &L = m->L;
  CnScalars *S = L.mem.get<CnScalars>(1);
  try {
    k_fcg_init<<<1, 1, 0, c.stream>>>(S, 0.0, 1, 1, 0, 0, 0);
    SFEM_CHECK_LAUNCH();
    coarse_restrict(c, c.stream, r, &S->done);
    cn_enqueue_net(L, c.coarse->dev, c.stream, S, &S->done);
    k_cn_z<<<c.red_blocks, 256, 0, c.stream>>>(c.coarse->dev, L.y, r, c.dinv64, c.dmask, c.ndof, S, z);
    SFEM_CHECK_LAUNCH();
    CnScalars hs{};
    SFEM_CUDA(cudaMemcpyAsync(&hs, S, sizeof hs, cudaMemcpyDeviceToHost, c.stream));
    SFEM_CUDA(cudaStreamSynchronize(c.stream));
    if (alpha) *alpha = hs.alpha;
  } catch (...) {
    L.mem.drop(S);
    throw;
  }
  L.mem.drop(S);
  CN_END
}

extern "C" int sfem_cnet_random_rows(sfem_cnet *m, sfem_ctx *h, float *X, float *T, int64_t first, int64_t count,
                                     uint64_t seed) {
  CN_BEGIN
  cn_check_ctx(m, h);
  SFEM_REQUIRE(X && T && first >= 0 && count >= 0, SFEM_EINVAL, "X, T required, first and count >= 0");
  cn_random_rows(m->L, h->c.coarse->dev, X, T, first, count, seed);
  CN_END
}

// solve with truncated flexible CG (kind forced to SFEM_SOLVE_FCG_CNET),
// collecting training rows into run->X, run->T
extern "C" int sfem_cnet_solve(sfem_cnet *m, sfem_ctx *h, const sfem_solve_opts *opts, double *u, sfem_cnet_run *run,
                               sfem_solve_info *info) {
  sfem_solve_info local{};
  try {
    SFEM_REQUIRE(h && h->c.vol && h->c.dinv64 && opts && u, SFEM_EINVAL, "context, opts and u are required");
    if (m) cn_check_ctx(m, h);
    sfem_solve_opts o = *opts;
    o.kind = SFEM_SOLVE_FCG_CNET;
    o.learned = m;
    CnRunArgs a;
    if (run) {
      a.window = run->window;
      a.snap_every = run->snap_every;
      a.X = run->X;
      a.T = run->T;
      a.cap = run->cap_rows;
      a.rows = run->rows;
      SFEM_REQUIRE(a.snap_every == 0 || (a.X && a.T && a.cap >= 0), SFEM_EINVAL, "row buffers required");
      SFEM_REQUIRE(a.snap_every == 0 || h->c.coarse, SFEM_EINVAL, "collecting rows needs sfem_coarse_setup");
    }
    solve_impl(h->c, nullptr, u, o, local, nullptr, &a);
    if (run) run->rows = a.rows;
  } catch (const Error &err) {
    set_last_error(err.msg);
    local.status = err.status;
    if (info) *info = local;
    return err.status;
  }
  if (info) *info = local;
  if (local.status != SFEM_OK) set_last_error(sfem_strerror(local.status));
  return local.status;
}

// the training GEMM of both learned corrections, alone (device pointers,
// the legacy default stream of the current device)
extern "C" int sfem_gemm_f32(int M, int N, int K, const float *A, int lda, int ta, const float *B, int ldb, int tb,
                             float *C, int ldc, double *ms) {
  if (!(M >= 1 && N >= 1 && K >= 0 && C && (K == 0 || (A && B)))) {
    set_last_error("M, N >= 1, K >= 0, C and (for K > 0) A, B required");
    return SFEM_EINVAL;
  }
  if (!(lda >= (ta ? M : std::max(K, 1)) && ldb >= (tb ? std::max(K, 1) : N) && ldc >= N)) {
    set_last_error("leading dimensions too small");
    return SFEM_EINVAL;
  }
  Allocator mem;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int status = SFEM_OK;
  try {
    float *split = nullptr;
    size_t split_floats = 0;
    int *err = mem.get<int>(1);
    SFEM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), nullptr));
    SFEM_CUDA(cudaEventCreate(&e0));
    SFEM_CUDA(cudaEventCreate(&e1));
    SFEM_CUDA(cudaEventRecord(e0, nullptr));
    mlp_gemm(mem, split, split_floats, nullptr, M, N, K, A, lda, ta != 0, B, ldb, tb != 0, C, ldc, err);
    SFEM_CUDA(cudaEventRecord(e1, nullptr));
    check_gemm_err(err, nullptr);
    float t = 0.f;
    SFEM_CUDA(cudaEventElapsedTime(&t, e0, e1));
    if (ms) *ms = t;
  } catch (const Error &err) {
    set_last_error(err.msg);
    status = err.status;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(nullptr);
  mem.release_all();
  return status;
}
