// Iterative solves of K d = f (Eq. 8) with essential conditions imposed by
// elimination (STEP 5): A = P K P + (I - P), b = P (f - K g) + (I - P) g.
//
// The paper calls a direct solver (Section 3.3); the library runs
// Jacobi-preconditioned CG on the GPU instead (and, in learned.cu, flexible
// PCG with a learned coarse correction):
//   PCG64    all vectors, scalars and the operator in FP64;
//   IR32_64  mixed precision: Jacobi-PCG iterations on the FP32 matrix-free
//            operator with FP32 vectors (scalars and reductions in FP64)
//            accumulate a correction d; at reliable updates (FP32 residual
//            down by inner_tol, or at the tolerance) the FP64 solution takes
//            u += d, the FP64 true residual f - K u replaces the FP32 one and
//            CG goes on in the same Krylov space (search direction kept),
//            so the refinement costs no restart.
// The CG scalars live in device memory.  By default each CG (re)start is one
// graph launch: a conditional WHILE node whose body runs four iterations and
// then a kernel that clears the loop flag when the device-side state says
// stop (converged, reliable update due, breakdown, fallback, guard count);
// the host wakes only between restarts.  Where conditional nodes are not
// available, or with SFEM_GRAPH_LOOP=0 (kernels inside a conditional node
// are invisible to ncu), the solve replays captured graphs of `check_every`
// iterations instead: once converged, a device flag turns the remaining
// captured kernels into no-ops, and the host polls the scalars between
// graph launches (two launches kept in flight).  Both give the same
// iterates.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "reduce.cuh"
#include "sfem_internal.cuh"

namespace sfem {

constexpr int kVecBlock = 256;

template <class... P>
bool aligned16(const P *...ptrs) {
  return ((reinterpret_cast<uintptr_t>(ptrs) % 16 == 0) && ...);
}

// CG vectors: x (solution or correction) of type TX, residual r of type TR,
// search direction p and operator output q of type TP (the operator reads
// p and writes q), Jacobi scaling of type TP.  Scalars and reductions are
// FP64 throughout.
template <class TX, class TR, class TP>
struct PcgVecs {
  TX *x;
  TR *r;
  TP *p, *q;
  const TP *dinv;
  const uint8_t *dmask;
  int64_t n;
  bool coarse = false;  // two-level preconditioner: z = D^-1 r + P Pi yc
  CoarseDev cs{};
  const float *dinv32 = nullptr;
  float *xlo = nullptr;  // FP32 x: low words of a double-float correction (x + xlo), or none
  // penalty method: the operator is followed by q += alpha S p (S: the DOFs
  // with pen_mask == 0); null for the masked elimination
  const uint8_t *pen_mask = nullptr;
  double pen_alpha = 0.0;
};

// (hi, lo) += a p with a = ahi + alo split from an FP64 step length: the
// product's rounding error by FMA, then a compensated two-sum and
// renormalisation, all in FP32 arithmetic (about 48 significant bits; the
// FP64 pipe of this GPU is ~64x slower than FP32)
__device__ __forceinline__ void df_axpy(float &hi, float &lo, float ahi, float alo, float p) {
  const float yh = __fmul_rn(ahi, p);
  const float yl = __fadd_rn(__fmaf_rn(ahi, p, -yh), __fmul_rn(alo, p));
  const float s = __fadd_rn(hi, yh);
  const float bv = __fsub_rn(s, hi);
  float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(yh, bv));
  e = __fadd_rn(e, __fadd_rn(lo, yl));
  hi = __fadd_rn(s, e);
  lo = __fsub_rn(e, __fsub_rn(hi, s));
}
__device__ __forceinline__ void df_split(double a, float &hi, float &lo) {
  hi = (float)a;
  lo = (float)(a - (double)hi);
}

// preconditioned residual of DOF i (the coarse correction yc of the current
// r must have been computed before the kernel runs)
template <class TX, class TR, class TP>
__device__ __forceinline__ TP precond_z(const PcgVecs<TX, TR, TP> &v, int64_t i, TP ri) {
  TP z = v.dinv[i] * ri;
  if (v.coarse && v.dmask[i]) z += (TP)cs_prolong(v.cs, i);
  return z;
}

// r must already hold the masked residual.  p = D^-1 r, q = 0, and the
// scalars rz = r.D^-1 r, rr = r.r are set; done when rr <= tol2.
template <class TX, class TR, class TP>
__global__ void __launch_bounds__(kVecBlock) k_pcg_init(PcgVecs<TX, TR, TP> v, SolveScalars *S, double tol2, int max_iter,
                                                        double delta2, double *partials, unsigned int *ticket) {
  double rz = 0.0, rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kVecBlock + threadIdx.x; i < v.n; i += (int64_t)gridDim.x * kVecBlock) {
    const TP ri = (TP)v.r[i];
    const TP zi = precond_z(v, i, ri);
    v.p[i] = zi;
    v.q[i] = TP(0);
    rz += (double)(zi * ri);
    rr += (double)(ri * ri);
  }
  double vv[2] = {rz, rr};
  if (grid_sum<kVecBlock, 2>(vv, partials, ticket, nullptr) && threadIdx.x == 0) {
    S->rz = vv[0];
    S->rz_prev = vv[0];
    S->rr = vv[1];
    S->bb = vv[1];
    S->rmax2 = vv[1];
    S->tol2 = tol2;
    S->delta2 = delta2;
    S->iter = 0;
    S->max_iter = max_iter;
    S->status = 0;
    S->reason = 0;
    S->done = 0;
    if (vv[1] <= tol2) {
      S->done = 1;
      S->reason = 1;
    } else if (max_iter <= 0) {
      S->done = 1;
      S->reason = 3;
    }
    S->pq = 0.0;
  }
}

// Reliable update (mixed precision): r has been replaced by the true
// residual; keep the search direction, p = D^-1 r + beta p with
// beta = (r.D^-1 r) / rz_prev, and resume.  rmax2 restarts from ||r||^2.
template <class TX, class TR, class TP>
__global__ void __launch_bounds__(kVecBlock) k_pcg_replace(PcgVecs<TX, TR, TP> v, SolveScalars *S, int max_iter,
                                                           double *partials, unsigned int *ticket) {
  double rz = 0.0, rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kVecBlock + threadIdx.x; i < v.n; i += (int64_t)gridDim.x * kVecBlock) {
    const TP ri = (TP)v.r[i];
    const TP zi = precond_z(v, i, ri);
    rz += (double)(zi * ri);
    rr += (double)(ri * ri);
  }
  double vv[2] = {rz, rr};
  __shared__ double beta_s;
  const bool last = grid_sum<kVecBlock, 2>(vv, partials, ticket, nullptr);
  if (last && threadIdx.x == 0) {
    beta_s = vv[0] / S->rz_prev;
    S->beta = beta_s;
    S->rz = vv[0];
    S->rr = vv[1];
    S->rmax2 = vv[1];
    S->pq = 0.0;
    S->max_iter = max_iter;
    S->reason = 0;
    S->done = (vv[1] <= S->tol2) ? 1 : 0;
    if (S->done) S->reason = 1;
  }
}

// second half of the replacement: p = D^-1 r + beta p, q = 0
template <class TX, class TR, class TP>
__global__ void __launch_bounds__(kVecBlock) k_pcg_replace_dir(PcgVecs<TX, TR, TP> v, const SolveScalars *S) {
  const TP b = (TP)S->beta;
  for (int64_t i = (int64_t)blockIdx.x * kVecBlock + threadIdx.x; i < v.n; i += (int64_t)gridDim.x * kVecBlock) {
    v.p[i] = precond_z(v, i, (TP)v.r[i]) + b * v.p[i];
    v.q[i] = TP(0);
  }
}

// the last block of an update: iteration count, convergence, reliable-update
// trigger (||r||^2 = rr)
__device__ __forceinline__ void finish_update(SolveScalars *S, double alpha, double rz_old, double rr) {
  S->pq = 0.0;  // every block has read it; the next tiled apply accumulates into it
  S->alpha = alpha;
  S->rz_prev = rz_old;
  S->rr = rr;
  S->iter += 1;
  S->rmax2 = fmax(S->rmax2, rr);
  if (rr <= S->tol2) {
    S->done = 1;
    S->reason = 1;
  } else if (S->iter >= S->max_iter) {
    S->done = 1;
    S->reason = 3;
  } else if (rr < S->delta2 * S->rmax2) {
    S->done = 1;
    S->reason = 2;
  }
  if (!isfinite(rr)) {
    S->status = 1;
    S->done = 1;
  }
}

// alpha = rz / pq, or a breakdown flag (all blocks see the same scalars and
// return together)
__device__ __forceinline__ bool step_length(SolveScalars *S, double &alpha, double &rz_old) {
  const double pq = S->pq;
  rz_old = S->rz;
  alpha = rz_old / pq;
  if (!(pq > 0.0) || !isfinite(alpha)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      S->status = 1;
      S->done = 1;
    }
    return false;
  }
  return true;
}

// x += alpha p, r -= alpha P q, then rz_new, rr; the last block sets beta,
// the convergence flag and the reliable-update trigger.
template <class TX, class TR, class TP>
__global__ void __launch_bounds__(kVecBlock) k_pcg_update(PcgVecs<TX, TR, TP> v, SolveScalars *S,
                                                          double *partials, unsigned int *ticket) {
  if (S->done) return;
  double alpha, rz_old;
  if (!step_length(S, alpha, rz_old)) return;
  const TX ax = (TX)alpha;
  const TR ar = (TR)alpha;
  float ahi = 0.f, alo = 0.f;
  df_split(alpha, ahi, alo);
  double rz = 0.0, rr = 0.0;
#pragma unroll 4
  for (int64_t i = (int64_t)blockIdx.x * kVecBlock + threadIdx.x; i < v.n; i += (int64_t)gridDim.x * kVecBlock) {
    if constexpr (std::is_same_v<TX, float> && std::is_same_v<TP, float>) {
      if (v.xlo)
        df_axpy(v.x[i], v.xlo[i], ahi, alo, v.p[i]);
      else
        v.x[i] += ax * v.p[i];
    } else {
      v.x[i] += ax * (TX)v.p[i];
    }
    const TR ri = v.dmask[i] ? v.r[i] - ar * (TR)v.q[i] : TR(0);
    v.r[i] = ri;
    const TP rp = (TP)ri;
    rz += (double)(v.dinv[i] * rp * rp);
    rr += (double)(rp * rp);
  }
  double vv[2] = {rz, rr};
  if (grid_sum<kVecBlock, 2>(vv, partials, ticket, nullptr) && threadIdx.x == 0) {
    S->beta = vv[0] / rz_old;
    S->rz = vv[0];
    finish_update(S, alpha, rz_old, vv[1]);
    if (!isfinite(vv[0])) {
      S->status = 1;
      S->done = 1;
    }
  }
}

// p = D^-1 r + beta p; q = 0 (the matrix-free operator accumulates into q)
template <class TX, class TR, class TP>
__global__ void __launch_bounds__(kVecBlock) k_pcg_direction(PcgVecs<TX, TR, TP> v, const SolveScalars *S,
                                                             bool zero_q) {
  if (S->done) return;
  const TP b = (TP)S->beta;
#pragma unroll 4
  for (int64_t i = (int64_t)blockIdx.x * kVecBlock + threadIdx.x; i < v.n; i += (int64_t)gridDim.x * kVecBlock) {
    v.p[i] = precond_z(v, i, (TP)v.r[i]) + b * v.p[i];
    if (zero_q) v.q[i] = TP(0);
  }
}

// ---- two-level iteration ------------------------------------------------------
// With the coarse correction an iteration runs, after the operator:
//   k_tl_update    x += alpha p, r = P (r - alpha q), q = 0, ||r||^2 and
//                  r.D^-1 r: a streaming pass over the DOFs (4 per thread,
//                  vector loads when the vectors are FP32 and 16-byte
//                  aligned);
//   k_tl_restrict  rc += Pi^T r: one warp per run of 64 nodes of one
//                  interpolation cell (nodes grouped by cell), its 24
//                  sums (8 corners x 3 components, reduce-scattered over the
//                  warp) added to the cell's centres by FP32 atomics;
//   k_cs_symv      yc = C rc (packed symmetric C; yc cleared by the
//                  restriction) and rc.C rc;
//   k_tl_dir       z.r = r.D^-1 r + rc.C rc (since P Pi yc . r = yc . rc),
//                  beta, and p = D^-1 r + P Pi yc + beta p in one pass: z is
//                  never stored; rc = 0 for the next restriction.
// The restriction and the dot products' per-thread sums are FP32 (the
// preconditioner and the step lengths tolerate 1e-7 relative rounding).
// FP64 arithmetic runs at about one FMA per SM and clock on this GPU, so
// the per-DOF FP64 work is kept to x += alpha p.
template <class TX, class TR, class TP, bool kVec>
__global__ void __launch_bounds__(kVecBlock) k_tl_update(PcgVecs<TX, TR, TP> v, SolveScalars *S, bool zero_q,
                                                         double *partials, unsigned int *ticket) {
  static_assert(!kVec || (std::is_same_v<TX, float> && std::is_same_v<TR, float> && std::is_same_v<TP, float>),
                "vector path is FP32 with a double-float x");
  // x: FP64, or double-float (x, xlo) when TX is float
  constexpr bool df = std::is_same_v<TX, float>;
  if (S->done) return;
  double alpha, rz_old;
  if (!step_length(S, alpha, rz_old)) return;
  const TR ar = (TR)alpha;
  float ahi = 0.f, alo = 0.f;
  df_split(alpha, ahi, alo);
  TX *__restrict__ x = v.x;
  float *__restrict__ xl = v.xlo;
  TR *__restrict__ r = v.r;
  TP *__restrict__ q = v.q;
  const TP *__restrict__ p = v.p;
  const uint8_t *__restrict__ msk = v.dmask;
  const float *__restrict__ dinv = v.dinv32;
  float rr = 0.f, rzj = 0.f;
  const int64_t nq = v.n / 4, stride = (int64_t)gridDim.x * kVecBlock;
  for (int64_t t = (int64_t)blockIdx.x * kVecBlock + threadIdx.x; t < nq; t += stride) {
    const int64_t i = 4 * t;
    TX xv[4];
    float xlv[4] = {0.f, 0.f, 0.f, 0.f};
    TP pv[4], qv[4];
    TR rv[4];
    float dv[4];
    uint8_t mv[4];
    if constexpr (kVec) {
      const float4 x4 = *reinterpret_cast<const float4 *>(x + i), xl4 = *reinterpret_cast<const float4 *>(xl + i);
      const float4 p4 = *reinterpret_cast<const float4 *>(p + i), q4 = *reinterpret_cast<const float4 *>(q + i);
      const float4 r4 = *reinterpret_cast<const float4 *>(r + i);
      const uchar4 m4 = *reinterpret_cast<const uchar4 *>(msk + i);
      const float4 d4 = *reinterpret_cast<const float4 *>(dinv + i);
      dv[0] = d4.x, dv[1] = d4.y, dv[2] = d4.z, dv[3] = d4.w;
      xv[0] = x4.x, xv[1] = x4.y, xv[2] = x4.z, xv[3] = x4.w;
      xlv[0] = xl4.x, xlv[1] = xl4.y, xlv[2] = xl4.z, xlv[3] = xl4.w;
      pv[0] = p4.x, pv[1] = p4.y, pv[2] = p4.z, pv[3] = p4.w;
      qv[0] = q4.x, qv[1] = q4.y, qv[2] = q4.z, qv[3] = q4.w;
      rv[0] = r4.x, rv[1] = r4.y, rv[2] = r4.z, rv[3] = r4.w;
      mv[0] = m4.x, mv[1] = m4.y, mv[2] = m4.z, mv[3] = m4.w;
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        xv[c] = x[i + c];
        if constexpr (df) xlv[c] = xl[i + c];
        pv[c] = p[i + c];
        qv[c] = q[i + c];
        rv[c] = r[i + c];
        dv[c] = dinv[i + c];
        mv[c] = msk[i + c];
      }
    }
    TR rn[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if constexpr (df)
        df_axpy(xv[c], xlv[c], ahi, alo, (float)pv[c]);
      else
        xv[c] = fma(alpha, (double)pv[c], xv[c]);
      rn[c] = mv[c] ? fma(-ar, (TR)qv[c], rv[c]) : TR(0);
      const float rf = (float)rn[c];
      rr = fmaf(rf, rf, rr);
      rzj = fmaf(dv[c] * rf, rf, rzj);
    }
    if constexpr (kVec) {
      *reinterpret_cast<float4 *>(x + i) = make_float4(xv[0], xv[1], xv[2], xv[3]);
      *reinterpret_cast<float4 *>(xl + i) = make_float4(xlv[0], xlv[1], xlv[2], xlv[3]);
      *reinterpret_cast<float4 *>(r + i) = make_float4(rn[0], rn[1], rn[2], rn[3]);
      if (zero_q) *reinterpret_cast<float4 *>(q + i) = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        x[i + c] = xv[c];
        if constexpr (df) xl[i + c] = xlv[c];
        r[i + c] = rn[c];
        if (zero_q) q[i + c] = TP(0);
      }
    }
  }
  for (int64_t i = 4 * nq + (int64_t)blockIdx.x * kVecBlock + threadIdx.x; i < v.n; i += stride) {
    if constexpr (df)
      df_axpy(x[i], xl[i], ahi, alo, (float)p[i]);
    else
      x[i] = fma(alpha, (double)p[i], x[i]);
    const TR rn = msk[i] ? fma(-ar, (TR)q[i], r[i]) : TR(0);
    r[i] = rn;
    if (zero_q) q[i] = TP(0);
    const float rf = (float)rn;
    rr = fmaf(rf, rf, rr);
    rzj = fmaf(dinv[i] * rf, rf, rzj);
  }
  double vv[2] = {(double)rr, (double)rzj};
  if (grid_sum<kVecBlock, 2>(vv, partials, ticket, nullptr) && threadIdx.x == 0) {
    finish_update(S, alpha, rz_old, vv[0]);
    S->rzj = vv[1];
    S->rzc = 0.0;  // the coarse product adds rc.C rc
  }
}

// nodes per warp of the restriction (2 per lane) and per block
constexpr int kRestrictWarpNodes = kSubNodes / (kVecBlock / 32);
static_assert(kRestrictWarpNodes == 64, "two nodes per lane");

template <class TR>
__global__ void __launch_bounds__(kVecBlock) k_tl_restrict(const TR *__restrict__ r, CoarseDev cs, const int *done) {
  if (done && *done) return;
  if (blockIdx.x == 0)  // the coarse product accumulates into yc
    for (int i = threadIdx.x; i < cs.npad; i += kVecBlock) cs.yc[i] = 0.f;
  const int4 ch = cs.sub[blockIdx.x];
  const int lane = threadIdx.x & 31;
  const int b = ch.y + kRestrictWarpNodes * (threadIdx.x >> 5);
  if (b >= ch.z) return;  // whole warps; no block barrier follows
  const int e = min(b + kRestrictWarpNodes, ch.z);
  constexpr int U = kRestrictWarpNodes / 32;
  int64_t i0[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int k = b + lane + 32 * u;
    i0[u] = k < e ? 3 * (int64_t)cs.cnodes[k] : -1;
  }
  float f[U][3], rf[U][3];
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      f[u][c] = i0[u] >= 0 ? cs.frac[i0[u] + c] : 0.f;
      rf[u][c] = i0[u] >= 0 ? (float)r[i0[u] + c] : 0.f;
    }
  float acc[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) acc[j] = 0.f;
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const float w = cs_weight(f[u], kk);
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[3 * kk + c] = fmaf(w, rf[u][c], acc[3 * kk + c]);
    }
  const float t = warp_reduce_scatter32(acc);  // lane l: the warp total of value l
  if (lane < 24) atomicAdd(cs.rc + 3 * cs_corner(cs, ch.x, lane / 3) + lane % 3, t);
}

// z.r and beta from the two partial sums, then p = D^-1 r + P Pi yc + beta p
// (every block forms the same beta; block 0 stores it).  A non-positive or
// non-finite z.r is a breakdown: p is left as it is.
template <class TX, class TR, class TP>
__global__ void __launch_bounds__(kVecBlock) k_tl_dir(PcgVecs<TX, TR, TP> v, SolveScalars *S) {
  if (S->done) return;
  const double rz = S->rzj + S->rzc;
  const double beta = rz / S->rz_prev;
  const bool ok = isfinite(rz) && rz > 0.0 && isfinite(beta);
  const CoarseDev &cs = v.cs;
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < cs.npad; i += kVecBlock) cs.rc[i] = 0.f;  // k_cs_symv has consumed rc
    if (threadIdx.x == 0) {
      S->beta = beta;
      S->rz = rz;
      if (!ok) {
        S->status = 1;
        S->done = 1;
      }
    }
  }
  if (!ok) return;
  const TR *__restrict__ r = v.r;
  const float *__restrict__ dinv = v.dinv32;
  const uint8_t *__restrict__ msk = v.dmask;
  TP *__restrict__ p = v.p;
  const float *__restrict__ yc = cs.yc;
  const TP b = (TP)beta;
  const int64_t nn = v.n / 3;
  const int sx = 3 * cs.d[1] * cs.d[2], sy = 3 * cs.d[2];
#pragma unroll 2
  for (int64_t node = (int64_t)blockIdx.x * kVecBlock + threadIdx.x; node < nn;
       node += (int64_t)gridDim.x * kVecBlock) {
    const int64_t i0 = 3 * node;
    TR rv[3];
    TP pv[3];
    float dv[3];
    uint8_t mv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      rv[c] = r[i0 + c];
      pv[c] = p[i0 + c];
      dv[c] = dinv[i0 + c];
      mv[c] = msk[i0 + c];
    }
    const int ci = cs.cinfo[node];
    const float f[3] = {cs.frac[i0], cs.frac[i0 + 1], cs.frac[i0 + 2]};
    const float *yb = yc + 3 * (ci & 0xFFFFFF);
    const int ox = ((ci >> 24) & 1) ? sx : 0, oy = ((ci >> 25) & 1) ? sy : 0, oz = ((ci >> 26) & 1) ? 3 : 0;
    float y[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const float w = cs_weight(f, kk);
      const float *yk = yb + ((kk & 4) ? ox : 0) + ((kk & 2) ? oy : 0) + ((kk & 1) ? oz : 0);
#pragma unroll
      for (int c = 0; c < 3; ++c) y[c] = fmaf(w, yk[c], y[c]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float zc = fmaf(dv[c], (float)rv[c], mv[c] ? y[c] : 0.f);
      p[i0 + c] = fma(b, pv[c], (TP)zc);
    }
  }
}

// ---- FP64 residual and refinement helpers ----------------------------------
__global__ void k_residual(const double *__restrict__ f, const double *__restrict__ Kx,
                           const uint8_t *__restrict__ dmask, int64_t n, double *__restrict__ r) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = dmask[i] ? f[i] - Kx[i] : 0.0;
}
// ---- the penalty method of STEP 5 (Sec. 3.3) --------------------------------
// A = K + alpha S and b = f + alpha S g, S the prescribed DOFs (dmask == 0):
// no row or column is removed; a large alpha pins u to g on S.
__global__ void k_pen_rhs(const double *__restrict__ f, const double *__restrict__ g,
                          const uint8_t *__restrict__ dmask, double alpha, int64_t n, double *__restrict__ b) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = dmask[i] ? f[i] : f[i] + alpha * g[i];
}
__global__ void k_pen_dinv(const double *__restrict__ diag, const uint8_t *__restrict__ dmask, double alpha,
                           int64_t n, double *__restrict__ dinv) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double d = diag[i] + (dmask[i] ? 0.0 : alpha);
    dinv[i] = d > 0.0 ? 1.0 / d : 0.0;
  }
}
__global__ void k_pen_residual(const double *__restrict__ b, const double *__restrict__ Kx,
                               const double *__restrict__ x, const uint8_t *__restrict__ dmask, double alpha,
                               int64_t n, double *__restrict__ r) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = b[i] - Kx[i] - (dmask[i] ? 0.0 : alpha * x[i]);
}
// after the operator: q += alpha S p, and p.q += alpha |S p|^2 (one FP64 atomic
// per block into the scalar the operator has written)
__global__ void __launch_bounds__(256) k_pen_q(const double *__restrict__ p, double *__restrict__ q,
                                               const uint8_t *__restrict__ dmask, double alpha, int64_t n,
                                               double *pq, const int *done) {
  if (done && *done) return;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256)
    if (!dmask[i]) {
      const double ap = alpha * p[i];
      q[i] += ap;
      s = fma(ap, p[i], s);
    }
  s = block_sum<256>(s);
  if (threadIdx.x == 0 && s != 0.0) atomicAdd(pq, s);
}
// max of non-negative values: their bit patterns order like the values
__global__ void k_max_nonneg(const double *__restrict__ a, int64_t n, unsigned long long *out) {
  double m = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, a[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}
static double device_max_nonneg(Ctx &c, const double *a, int64_t n) {
  unsigned long long *d = c.mem.get<unsigned long long>(1);
  SFEM_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned long long), c.stream));
  k_max_nonneg<<<std::min(grid_for(n, 256), c.red_blocks), 256, 0, c.stream>>>(a, n, d);
  SFEM_CHECK_LAUNCH();
  unsigned long long h = 0;
  SFEM_CUDA(cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, c.stream));
  SFEM_CUDA(cudaStreamSynchronize(c.stream));
  c.mem.drop(d);
  double v;
  std::memcpy(&v, &h, sizeof v);
  return v;
}

__global__ void k_set_bc(double *__restrict__ x, const double *__restrict__ g, const uint8_t *__restrict__ dmask,
                         int64_t n, bool zero_free) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    if (!dmask[i])
      x[i] = g[i];
    else if (zero_free)
      x[i] = 0.0;
  }
}
__global__ void k_add(double *__restrict__ a, const double *__restrict__ b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] += b[i];
}
// u += hi + lo (the double-float correction), then hi = lo = 0
__global__ void k_add_df(double *__restrict__ u, float *__restrict__ hi, float *__restrict__ lo, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    u[i] += (double)hi[i] + (double)lo[i];
    hi[i] = 0.f;
    lo[i] = 0.f;
  }
}
__global__ void k_scale_to_f32(const double *__restrict__ r, double s, int64_t n, float *__restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)(r[i] * s);
}
__global__ void k_refine(double *__restrict__ x, float *__restrict__ d, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    x[i] += (double)d[i];
    d[i] = 0.f;
  }
}
__global__ void k_to_f32(const double *__restrict__ r, int64_t n, float *__restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)r[i];
}
__global__ void k_rhs_vec(const double *__restrict__ f, const double *__restrict__ Kg, const double *__restrict__ g,
                          const uint8_t *__restrict__ dmask, int64_t n, double *__restrict__ b) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = dmask[i] ? f[i] - Kg[i] : g[i];
}

// raw K x with the selected FP64 operator (stream c.stream)
static void apply_op64(Ctx &c, int op, const double *x, double *y) {
  if (op == SFEM_OP_CSR64)
    apply_csr64(c, x, y, 1, nullptr, nullptr);
  else if (op == SFEM_OP_NS64)
    apply_ns64(c, x, y);
  else if (op == SFEM_OP_ES64)
    apply_es64(c, x, y);
  else
    apply_mf64(c, x, y, 1, nullptr);
}

// WHILE-node condition of the iteration graph: another body execution while the
// solver is not done and the guard (body executions this launch) is below
// its limit, so the loop ends whatever state the scalars are in
__global__ void k_loop_cond(cudaGraphConditionalHandle h, const int *done, unsigned int *guard) {
  const unsigned int n = guard[0] + 1;
  guard[0] = n;
  cudaGraphSetConditional(h, (*done == 0 && n < guard[1]) ? 1u : 0u);
}

__global__ void k_guard_reset(unsigned int *guard, unsigned int limit) {
  guard[0] = 0;
  guard[1] = limit;
}

// Conditional graph nodes hide their kernels from kernel-level profilers;
// SFEM_GRAPH_LOOP=0 in the environment selects the captured chunks instead
// (same kernels and arithmetic, host polling between chunks).
// CG iterations per execution of the WHILE node's body (the kernels of an
// iteration after the one that set done return at once); SFEM_LOOP_UNROLL
static int loop_unroll() {
  static const int u = [] {
    const char *e = std::getenv("SFEM_LOOP_UNROLL");
    const int v = e ? std::atoi(e) : 0;
    return v >= 1 && v <= 16 ? v : 4;
  }();
  return u;
}

static bool loop_graphs_enabled() {
  static const bool on = [] {
    const char *e = std::getenv("SFEM_GRAPH_LOOP");
    return !(e && e[0] == '0');
  }();
  return on;
}

// ---- one CG run (PCG64 or the FP32 inner solve) ----------------------------
template <class TX, class TR, class TP>
struct CgRun {
  Ctx &c;
  PcgVecs<TX, TR, TP> v;
  int op;                 // SFEM_OP_CSR64 / SFEM_OP_MF64 (TP double) or SFEM_OP_MF32
  int chunk;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;

  // device-side loop: one graph launch runs iterations until done (a
  // conditional WHILE node); else captured chunks of `chunk` iterations
  bool looped = false;
  unsigned int *guard = nullptr;  // [0] body executions of a launch, [1] limit

  CgRun(Ctx &c_, PcgVecs<TX, TR, TP> v_, int op_, int chunk_) : c(c_), v(v_), op(op_), chunk(chunk_) {}
  ~CgRun() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (guard) c.mem.drop(guard);
  }

  // the iteration as the body of a WHILE node; false (and no graph) when
  // the runtime cannot build it
  bool build_loop_graph() {
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle hnd;
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    cp.type = cudaGraphNodeTypeConditional;
    if (cudaGraphConditionalHandleCreate(&hnd, g, 1, cudaGraphCondAssignDefault) != cudaSuccess ||
        (cp.conditional.handle = hnd, cp.conditional.type = cudaGraphCondTypeWhile, cp.conditional.size = 1,
         cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) != cudaSuccess) ||
        cudaStreamBeginCaptureToGraph(c.cap_stream, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphDestroy(g);
      return false;
    }
    if (!guard) guard = c.mem.get<unsigned int>(2);
    set_capturing(true);
    try {
      for (int u = 0; u < loop_unroll(); ++u) enqueue_iteration(c.cap_stream);
      k_loop_cond<<<1, 1, 0, c.cap_stream>>>(hnd, &c.scal->done, guard);
      SFEM_CUDA(cudaGetLastError());
    } catch (...) {
      set_capturing(false);
      cudaGraph_t tmp = nullptr;
      cudaStreamEndCapture(c.cap_stream, &tmp);
      cudaGraphDestroy(g);
      throw;
    }
    set_capturing(false);
    cudaGraph_t body = nullptr;
    if (cudaStreamEndCapture(c.cap_stream, &body) != cudaSuccess ||
        cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) {
      cudaGetLastError();
      if (exec) cudaGraphExecDestroy(exec);
      exec = nullptr;
      cudaGraphDestroy(g);
      return false;
    }
    graph = g;
    SFEM_CUDA(cudaGraphGetNodes(cp.conditional.phGraph_out[0], nullptr, &graph_nodes));
    looped = true;
    return true;
  }

  void enqueue_iteration(cudaStream_t st) {
    SolveScalars *S = c.scal;
    const int *done = &S->done;
    const bool mf = op != SFEM_OP_CSR64;
    if (op == SFEM_OP_CSR64) {
      launch_csr64(c, st, (const double *)v.p, (double *)v.q, (const double *)v.p, &S->pq, done);
    } else if (op == SFEM_OP_MF64) {
      double *w = static_cast<double *>(c.w_scratch);
      launch_mf_strain<double, double>(c, st, c.Gs64, (const double *)v.p, 1, w, done);
      launch_mf_stress<double, double>(c, st, c.Gs64, c.kap64, w, (double *)v.q, 1, &S->pq, done);
    } else if (op == SFEM_OP_NS64) {
      // q accumulated by atomics (zeroed by the direction pass); p.q added to
      // S->pq, which the update pass leaves at zero
      if constexpr (std::is_same_v<TP, double>) launch_ns64(c, st, v.p, v.q, &S->pq, done);
    } else if (op == SFEM_OP_ES64) {
      if constexpr (std::is_same_v<TP, double>) launch_es64(c, st, v.p, v.q, &S->pq, done);
    } else {
      // tiled FP32 operator reading p and accumulating q in type TP
      launch_mf32_tiled<TP, TP>(c, st, v.p, v.q, &S->pq, done);
    }
    if constexpr (std::is_same_v<TP, double>) {
      if (v.pen_mask) {
        k_pen_q<<<c.red_blocks, 256, 0, st>>>(v.p, v.q, v.pen_mask, v.pen_alpha, v.n, &S->pq, done);
        SFEM_CHECK_LAUNCH();
      }
    }
    {
      if (v.coarse) {  // FP64 x, or double-float x with FP32 r, p, q
        if constexpr (std::is_same_v<TX, float>)
          SFEM_REQUIRE(v.xlo != nullptr, SFEM_EINVAL, "the coarse correction needs an FP64 or double-float correction");
        const CoarseDev &cs = v.cs;
        // 4 blocks of 256 threads per SM (8 per SM measured 10 us slower per iteration)
        const int vb = c.red_blocks;
        constexpr bool f32 = std::is_same_v<TX, float> && std::is_same_v<TR, float> && std::is_same_v<TP, float>;
        bool vec = false;
        if constexpr (f32)
          vec = v.xlo && aligned16(v.x, v.xlo, v.r, v.p, v.q, v.dinv32) &&
                (reinterpret_cast<uintptr_t>(v.dmask) & 3) == 0;
        if constexpr (f32) {
          if (vec)
            k_tl_update<TX, TR, TP, true><<<vb, kVecBlock, 0, st>>>(v, S, mf, c.red_partial,
                                                                              c.tickets + 3);
        }
        if (!vec)
          k_tl_update<TX, TR, TP, false><<<vb, kVecBlock, 0, st>>>(v, S, mf, c.red_partial, c.tickets + 3);
        SFEM_CHECK_LAUNCH();
        k_tl_restrict<TR><<<cs.nsub, kVecBlock, 0, st>>>(v.r, cs, done);
        SFEM_CHECK_LAUNCH();
        coarse_gemv(cs, st, done, &S->rzc);
        k_tl_dir<TX, TR, TP><<<vb, kVecBlock, 0, st>>>(v, S);
        SFEM_CHECK_LAUNCH();
        return;
      }
    }
    k_pcg_update<TX, TR, TP><<<c.red_blocks, kVecBlock, 0, st>>>(v, S, c.red_partial, c.tickets + 3);
    SFEM_CHECK_LAUNCH();
    k_pcg_direction<TX, TR, TP><<<c.red_blocks, kVecBlock, 0, st>>>(v, S, mf);
    SFEM_CHECK_LAUNCH();
  }

  size_t graph_nodes = 0;

  void build_graph() {
    if (loop_graphs_enabled() && build_loop_graph()) return;
    SFEM_CUDA(cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal));
    set_capturing(true);
    try {
      for (int i = 0; i < chunk; ++i) enqueue_iteration(c.cap_stream);
    } catch (...) {
      set_capturing(false);
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(c.cap_stream, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    set_capturing(false);
    SFEM_CUDA(cudaStreamEndCapture(c.cap_stream, &graph));
    SFEM_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    SFEM_CUDA(cudaGraphGetNodes(graph, nullptr, &graph_nodes));
  }

  // r holds the masked residual on entry: (re)start CG from it.
  SolveScalars start(double tol2, int max_iter, double delta2) {
    if (v.coarse) coarse_correction(c, c.stream, v.r, nullptr);
    k_pcg_init<TX, TR, TP><<<c.red_blocks, kVecBlock, 0, c.stream>>>(v, c.scal, tol2, max_iter, delta2,
                                                                      c.red_partial, c.tickets + 4);
    SFEM_CHECK_LAUNCH();
    clear_restriction();
    return resume(max_iter);
  }

  // the iterations accumulate the restriction into rc by atomics
  void clear_restriction() {
    if (v.coarse) SFEM_CUDA(cudaMemsetAsync(v.cs.rc, 0, v.cs.npad * sizeof(float), c.stream));
  }

  // r has been replaced by the true residual: keep p, recompute beta, go on.
  SolveScalars replace(int max_iter) {
    if (v.coarse) coarse_correction(c, c.stream, v.r, nullptr);
    k_pcg_replace<TX, TR, TP><<<c.red_blocks, kVecBlock, 0, c.stream>>>(v, c.scal, max_iter, c.red_partial,
                                                                         c.tickets + 5);
    SFEM_CHECK_LAUNCH();
    k_pcg_replace_dir<TX, TR, TP><<<c.red_blocks, kVecBlock, 0, c.stream>>>(v, c.scal);
    SFEM_CHECK_LAUNCH();
    clear_restriction();
    return resume(max_iter);
  }

  // run captured chunks until the device sets done; returns the scalars
  SolveScalars resume(int max_iter) {
    if (!exec) build_graph();
    if (looped) {
      // one launch runs the iterations until the device flag says done
      SolveScalars out;
      unsigned int hg[2] = {0, 0};
      k_guard_reset<<<1, 1, 0, c.stream>>>(guard, (unsigned int)(max_iter / loop_unroll()) + 3u);
      SFEM_CHECK_LAUNCH();
      SFEM_CUDA(cudaGraphLaunch(exec, c.stream));
      SFEM_CUDA(cudaMemcpyAsync(&out, c.scal, sizeof out, cudaMemcpyDeviceToHost, c.stream));
      SFEM_CUDA(cudaMemcpyAsync(hg, guard, sizeof hg, cudaMemcpyDeviceToHost, c.stream));
      SFEM_CUDA(cudaStreamSynchronize(c.stream));
      count_launches((int64_t)graph_nodes * hg[0]);
      return out;
    }
    if (!c.h_scal) SFEM_CUDA(cudaMallocHost(&c.h_scal, 4 * sizeof(SolveScalars)));
    SolveScalars *h = c.h_scal;
    cudaEvent_t ev[2];
    SFEM_CUDA(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    SFEM_CUDA(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
    auto launch = [&](int slot) {
      SFEM_CUDA(cudaGraphLaunch(exec, c.stream));
      count_launches((int64_t)graph_nodes);
      SFEM_CUDA(cudaMemcpyAsync(&h[slot], c.scal, sizeof(SolveScalars), cudaMemcpyDeviceToHost, c.stream));
      SFEM_CUDA(cudaEventRecord(ev[slot], c.stream));
    };
    const int64_t max_launch = (int64_t)max_iter / chunk + 3;
    launch(0);
    launch(1);
    int64_t launched = 2;
    int slot = 0;
    while (true) {
      SFEM_CUDA(cudaEventSynchronize(ev[slot]));
      if (h[slot].done || launched >= max_launch) break;
      launch(slot);
      ++launched;
      slot ^= 1;
    }
    SFEM_CUDA(cudaStreamSynchronize(c.stream));
    SolveScalars out;
    SFEM_CUDA(cudaMemcpy(&out, c.scal, sizeof out, cudaMemcpyDeviceToHost));
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    return out;
  }
};

struct SolveBuffers {
  Ctx &c;
  std::vector<void *> owned;
  explicit SolveBuffers(Ctx &c_) : c(c_) {}
  template <class T>
  T *get(int64_t n) {
    T *p = c.mem.get<T>(n);
    owned.push_back(p);
    return p;
  }
  ~SolveBuffers() {
    for (void *p : owned) c.mem.drop(p);
  }
};

void solve_impl(Ctx &c, const double *f_extra, double *u, const sfem_solve_opts &o, sfem_solve_info &info,
                const Snapshot *snap, CnRunArgs *cn) {
  const int64_t n = c.ndof;
  const int g256 = grid_for(n, 256);
  cudaMemcpyKind in_kind = o.u_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaMemcpyKind out_kind = o.u_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const double tol = o.tol > 0 ? o.tol : 1e-8;
  const int max_iter = o.max_iter > 0 ? o.max_iter : 200000;
  const int chunk = o.check_every > 0 ? o.check_every : 32;
  const int op64 = o.op64;
  SFEM_REQUIRE(op64 == SFEM_OP_CSR64 || op64 == SFEM_OP_MF64 || op64 == SFEM_OP_NS64 || op64 == SFEM_OP_ES64,
               SFEM_EINVAL, "op64 must be CSR64, MF64, NS64 or ES64");
  const bool other_sfem = op64 == SFEM_OP_NS64 || op64 == SFEM_OP_ES64;
  if (other_sfem)
    SFEM_REQUIRE(o.kind == SFEM_SOLVE_PCG64 && o.precond == 0 && o.bc == 0 && !snap, SFEM_EINVAL,
                 "the NS-FEM and ES-FEM operators work with PCG64, the Jacobi preconditioner and eliminated BCs");
  if (op64 == SFEM_OP_ES64) prepare_es64(c);  // the edge table, before any capture
  if (op64 == SFEM_OP_CSR64) SFEM_REQUIRE(c.assembled, SFEM_EINVAL, "CSR64 needs sfem_assemble first");
  SFEM_REQUIRE(o.rhs >= 0 && o.rhs < c.nrhs, SFEM_EINVAL, "rhs out of range");
  SFEM_REQUIRE(o.precond == 0 || o.precond == 1, SFEM_EINVAL, "precond must be 0 or 1");
  const bool coarse = o.precond == 1;
  if (coarse) {
    SFEM_REQUIRE(c.coarse != nullptr, SFEM_EINVAL, "precond = 1 needs sfem_coarse_setup first");
    SFEM_REQUIRE(o.kind == SFEM_SOLVE_PCG64 ||
                     (o.kind == SFEM_SOLVE_IR32_64 && (o.fp32_vectors == 0 || o.fp32_vectors == 3)),
                 SFEM_EINVAL, "the coarse correction works with PCG64 and with IR32_64 on an FP64 correction");
  }
  SFEM_REQUIRE(o.fp32_vectors >= 0 && o.fp32_vectors <= 3, SFEM_EINVAL, "fp32_vectors must be 0, 1, 2 or 3");
  SFEM_REQUIRE(o.bc == 0 || o.bc == 1, SFEM_EINVAL, "bc must be 0 or 1");
  SFEM_REQUIRE(o.penalty_exp >= 0 && o.penalty_exp <= 15, SFEM_EINVAL, "penalty_exp must be 0 .. 15");
  const bool penalty = o.bc == 1;
  if (penalty)
    SFEM_REQUIRE(o.kind == SFEM_SOLVE_PCG64 && !coarse && !snap, SFEM_EINVAL,
                 "the penalty method works with PCG64 and the Jacobi preconditioner");

  cudaEvent_t e0, e1;
  SFEM_CUDA(cudaEventCreate(&e0));
  SFEM_CUDA(cudaEventCreate(&e1));
  SFEM_CUDA(cudaEventRecord(e0, c.stream));

  SolveBuffers B(c);
  auto with_coarse = [&](auto &vv) {
    if (coarse) {
      vv.coarse = true;
      vv.cs = c.coarse->dev;
      vv.dinv32 = c.dinv32;
    }
  };
  // total load f (+ f_extra) and ||b||
  double *ftot = B.get<double>(n);
  SFEM_CUDA(cudaMemcpyAsync(ftot, c.f + (int64_t)o.rhs * n, n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
  double *tmp = B.get<double>(n);
  double bnorm = c.bnorm[o.rhs];
  if (f_extra || other_sfem) {
    if (f_extra) {
      SFEM_CUDA(cudaMemcpyAsync(tmp, f_extra, n * sizeof(double), in_kind, c.stream));
      k_add<<<g256, 256, 0, c.stream>>>(ftot, tmp, n);
      SFEM_CHECK_LAUNCH();
    }
    // ||b|| of this load and operator: b = P (f - K g) + (I - P) g
    double *Kg = B.get<double>(n);
    if (other_sfem)
      apply_op64(c, op64, c.g, Kg);
    else
      apply_mf64(c, c.g, Kg, 1, nullptr);
    k_rhs_vec<<<g256, 256, 0, c.stream>>>(ftot, Kg, c.g, c.dmask, n, tmp);
    SFEM_CHECK_LAUNCH();
    bnorm = std::sqrt(device_norm2(c, tmp, n));
  }
  double pen_alpha = 0.0;
  double *bpen = nullptr, *dpen = nullptr;
  uint8_t *ones = nullptr;
  if (penalty) {
    // alpha = 10^penalty_exp times the largest diagonal entry of K
    pen_alpha = std::pow(10.0, o.penalty_exp > 0 ? o.penalty_exp : 8) * device_max_nonneg(c, c.diag, n);
    bpen = B.get<double>(n);
    k_pen_rhs<<<g256, 256, 0, c.stream>>>(ftot, c.g, c.dmask, pen_alpha, n, bpen);
    SFEM_CHECK_LAUNCH();
    bnorm = std::sqrt(device_norm2(c, bpen, n));
    dpen = B.get<double>(n);
    k_pen_dinv<<<g256, 256, 0, c.stream>>>(c.diag, c.dmask, pen_alpha, n, dpen);
    SFEM_CHECK_LAUNCH();
    ones = B.get<uint8_t>(n);
    SFEM_CUDA(cudaMemsetAsync(ones, 1, n, c.stream));
  }
  info.bnorm = bnorm;

  double *x = B.get<double>(n);
  if (o.warm_start) SFEM_CUDA(cudaMemcpyAsync(x, u, n * sizeof(double), in_kind, c.stream));
  k_set_bc<<<g256, 256, 0, c.stream>>>(x, c.g, c.dmask, n, !o.warm_start);
  SFEM_CHECK_LAUNCH();

  if (bnorm == 0.0) {
    info.true_relres = 0.0;
    info.status = SFEM_OK;
  } else {
    double *Kx = B.get<double>(n);
    double *r = B.get<double>(n);
    auto true_residual = [&]() {
      apply_op64(c, op64, x, Kx);
      if (penalty)
        k_pen_residual<<<g256, 256, 0, c.stream>>>(bpen, Kx, x, c.dmask, pen_alpha, n, r);
      else
        k_residual<<<g256, 256, 0, c.stream>>>(ftot, Kx, c.dmask, n, r);
      SFEM_CHECK_LAUNCH();
      return std::sqrt(device_norm2(c, r, n)) / bnorm;
    };
    int total_iter = 0, outer = 0, status = SFEM_OK;
    double rel = true_residual();
    if (o.kind == SFEM_SOLVE_PCG64) {
      if (op64 == SFEM_OP_MF64) ensure_w_scratch(c, (size_t)c.n_tets * 8 * sizeof(double));
      PcgVecs<double, double, double> v{x, r, B.get<double>(n), B.get<double>(n), penalty ? dpen : c.dinv64,
                                        penalty ? ones : c.dmask, n};
      with_coarse(v);
      if (penalty) {
        v.pen_mask = c.dmask;
        v.pen_alpha = pen_alpha;
      }
      CgRun<double, double, double> cg(c, v, op64, chunk);
      const int max_restarts = 10;
      while (rel > tol && total_iter < max_iter && outer <= max_restarts) {
        SolveScalars s = cg.start(tol * tol * bnorm * bnorm, max_iter - total_iter, 0.0);
        total_iter += s.iter;
        if (s.status) {
          status = SFEM_EBREAKDOWN;
          rel = true_residual();
          break;
        }
        rel = true_residual();  // also resets r for a restart
        ++outer;
      }
    } else if (o.kind == SFEM_SOLVE_IR32_64) {
      // Mixed precision with reliable updates: FP32 CG iterations on the
      // FP32 matrix-free operator accumulate a correction d; whenever the
      // FP32 recursive residual has fallen by `inner_tol` since the last
      // update (or reached the tolerance), u += d in FP64, the FP64 true
      // residual f - K u replaces the FP32 one, and CG continues in the
      // same Krylov space (the search direction is kept).
      const double delta = o.inner_tol > 0 ? o.inner_tol : 0.1;
      const int max_outer = o.max_outer > 0 ? o.max_outer : 200;
      ensure_w_scratch(c, (size_t)c.n_tets * 8 * sizeof(double));
      if (o.fp32_vectors == 1) {
        // all-FP32 inner iterations (vectors too): cheaper per iteration,
        // but finite-precision CG loses orthogonality much faster
        PcgVecs<float, float, float> v{B.get<float>(n), B.get<float>(n), B.get<float>(n), B.get<float>(n),
                                       c.dinv32, c.dmask, n};
        CgRun<float, float, float> cg(c, v, SFEM_OP_MF32, chunk);
        SFEM_CUDA(cudaMemsetAsync(v.x, 0, n * sizeof(float), c.stream));
        bool started = false;
        while (rel > tol && total_iter < max_iter && outer < max_outer) {
          k_to_f32<<<g256, 256, 0, c.stream>>>(r, n, v.r);
          SFEM_CHECK_LAUNCH();
          // S->iter counts across replacements, so the cap is the total one
          SolveScalars s = started ? cg.replace(max_iter)
                                   : cg.start(tol * tol * bnorm * bnorm, max_iter, delta * delta);
          started = true;
          total_iter = s.iter;
          ++outer;
          if (s.status) {
            status = SFEM_EBREAKDOWN;
            break;
          }
          k_refine<<<g256, 256, 0, c.stream>>>(x, v.x, n);
          SFEM_CHECK_LAUNCH();
          rel = true_residual();
        }
      } else if (o.fp32_vectors == 2) {
        // FP32 search direction p, operator output q and correction d; FP64
        // residual r
        PcgVecs<float, double, float> v{B.get<float>(n), r, B.get<float>(n), B.get<float>(n), c.dinv32, c.dmask,
                                        n};
        CgRun<float, double, float> cg(c, v, SFEM_OP_MF32, chunk);
        SFEM_CUDA(cudaMemsetAsync(v.x, 0, n * sizeof(float), c.stream));
        bool started = false;
        while (rel > tol && total_iter < max_iter && outer < max_outer) {
          SolveScalars s = started ? cg.replace(max_iter)
                                   : cg.start(tol * tol * bnorm * bnorm, max_iter, delta * delta);
          started = true;
          total_iter = s.iter;
          ++outer;
          if (s.status) {
            status = SFEM_EBREAKDOWN;
            break;
          }
          k_refine<<<g256, 256, 0, c.stream>>>(x, v.x, n);  // u += d, d = 0
          SFEM_CHECK_LAUNCH();
          rel = true_residual();  // writes the FP64 true residual into r = v.r
        }
      } else {
        // 0 (default): every CG vector in FP64 (correction d, residual r,
        // search direction p, operator output q); the FP32 operator reads p
        // in FP64 and accumulates q in FP64.  With Jacobi alone, an FP32 d
        // or p doubled the iteration count on the 2M-tet beam: their
        // rounding re-enters the FP64 true residual amplified by the
        // condition number at every update.
        // 3: double-float correction d (two FP32 words); FP32 r, p, q (and
        // z): with the two-level preconditioner the inner iterations converge
        // in as many steps as with FP64 vectors (emulated on a 123k-tet beam:
        // 428 vs 426), at half the vector traffic and without FP64
        // arithmetic in the per-DOF passes.
        auto reliable = [&](auto tag) {
          using TV = decltype(tag);
          constexpr bool f64 = std::is_same_v<TV, double>;
          TV *rv = nullptr;
          if constexpr (f64)
            rv = r;
          else
            rv = B.get<TV>(n);
          const TV *dinv = nullptr;
          if constexpr (f64)
            dinv = c.dinv64;
          else
            dinv = c.dinv32;
          // correction d: FP64, or double-float (two FP32 words) with FP32 vectors
          PcgVecs<TV, TV, TV> v{B.get<TV>(n), rv, B.get<TV>(n), B.get<TV>(n), dinv, c.dmask, n};
          if constexpr (!f64) {
            v.xlo = B.get<float>(n);
            SFEM_CUDA(cudaMemsetAsync(v.xlo, 0, n * sizeof(float), c.stream));
          }
          with_coarse(v);
          CgRun<TV, TV, TV> cg(c, v, SFEM_OP_MF32, chunk);
          SFEM_CUDA(cudaMemsetAsync(v.x, 0, n * sizeof(TV), c.stream));
          bool started = false;
          double best = rel;
          int stall = 0;
          while (rel > tol && total_iter < max_iter && outer < max_outer) {
            if constexpr (!f64) {
              k_to_f32<<<g256, 256, 0, c.stream>>>(r, n, v.r);
              SFEM_CHECK_LAUNCH();
            }
            SolveScalars s = started ? cg.replace(max_iter)
                                     : cg.start(tol * tol * bnorm * bnorm, max_iter, delta * delta);
            started = true;
            total_iter = s.iter;
            ++outer;
            if (s.status) {
              status = SFEM_EBREAKDOWN;
              break;
            }
            if constexpr (f64) {
              k_add<<<g256, 256, 0, c.stream>>>(x, v.x, n);  // u += d
              SFEM_CHECK_LAUNCH();
              SFEM_CUDA(cudaMemsetAsync(v.x, 0, n * sizeof(double), c.stream));  // d = 0
            } else {
              k_add_df<<<g256, 256, 0, c.stream>>>(x, v.x, v.xlo, n);  // u += d, d = 0
              SFEM_CHECK_LAUNCH();
            }
            rel = true_residual();  // the FP64 true residual into r
            // stagnation: the FP32 operator's error floor lies above tol
            if (rel < 0.9 * best) {
              best = rel;
              stall = 0;
            } else if (++stall >= 3) {
              break;
            }
          }
          if (rel > tol && status == SFEM_OK && stall >= 3 && total_iter < max_iter) {
            // finish with FP64 PCG from the current solution
            ensure_w_scratch(c, (size_t)c.n_tets * 8 * sizeof(double));
            double *p2 = nullptr, *q2 = nullptr;
            if constexpr (f64) {
              p2 = v.p;
              q2 = v.q;
            } else {
              p2 = B.get<double>(n);
              q2 = B.get<double>(n);
            }
            PcgVecs<double, double, double> v2{x, r, p2, q2, c.dinv64, c.dmask, n};
            with_coarse(v2);
            CgRun<double, double, double> cg2(c, v2, op64, chunk);
            info.fallbacks = 1;
            for (int restart = 0; rel > tol && total_iter < max_iter && restart <= 10; ++restart) {
              SolveScalars s2 = cg2.start(tol * tol * bnorm * bnorm, max_iter - total_iter, 0.0);
              total_iter += s2.iter;
              if (s2.status) {
                status = SFEM_EBREAKDOWN;
                break;
              }
              rel = true_residual();
            }
          }
        };
        if (o.fp32_vectors == 3)
          reliable(float{});
        else
          reliable(double{});
      }
    } else if (o.kind == SFEM_SOLVE_FPCG_LEARNED) {
      const int window = o.learned_window > 0 ? o.learned_window : 100;
      solve_fpcg(c, o.learned, op64, x, r, bnorm, tol, max_iter, chunk, window, std::max(o.learned_pace, 0), info,
                 true_residual, snap);
      total_iter = info.iterations;
      outer = info.outer_iterations;
      rel = info.true_relres;
      if (info.status != SFEM_OK && info.status != SFEM_ENOCONV) status = info.status;
    } else if (o.kind == SFEM_SOLVE_FCG_CNET) {
      SFEM_REQUIRE(!coarse && !penalty && !snap, SFEM_EINVAL,
                   "FCG_CNET takes its coarse space from the model, with eliminated BCs");
      solve_cnet(c, o.learned, cn, op64, x, r, bnorm, tol, max_iter, info, true_residual);
      total_iter = info.iterations;
      outer = info.outer_iterations;
      rel = info.true_relres;
      if (info.status != SFEM_OK && info.status != SFEM_ENOCONV) status = info.status;
    } else {
      throw Error{SFEM_EINVAL, "unknown solver kind"};
    }
    info.iterations = total_iter;
    info.outer_iterations = outer;
    info.true_relres = rel;
    if (status == SFEM_OK && rel > tol) status = SFEM_ENOCONV;
    info.status = status;
  }
  SFEM_CUDA(cudaMemcpyAsync(u, x, n * sizeof(double), out_kind, c.stream));
  SFEM_CUDA(cudaEventRecord(e1, c.stream));
  SFEM_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  SFEM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  info.solve_ms = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

}  // namespace sfem

using namespace sfem;

extern "C" int sfem_solve(sfem_ctx *h, const double *f_extra, double *u, const sfem_solve_opts *opts,
                          sfem_solve_info *info) {
  sfem_solve_info local{};
  try {
    SFEM_REQUIRE(h && h->c.vol && h->c.dinv64, SFEM_EINVAL, "context not set up");
    SFEM_REQUIRE(u && opts, SFEM_EINVAL, "u and opts must not be NULL");
    solve_impl(h->c, f_extra, u, *opts, local);
    check_tile_error(h->c);
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
