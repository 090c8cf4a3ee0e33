// Batched persistent solver: many beams (contexts) with several load cases
// each, solved together by the mixed-precision CG of solve.cu.
//
// One "system" is one (context, load case).  A round is
//   1. one persistent cooperative launch running FP32-operator CG
//      iterations (FP64 solution, residual and reductions; FP32 search
//      direction p and operator output q) for every active system:
//        P1  operator over the (active beam, tile) items; a tile's
//            geometry is loaded once for all active load cases of its beam
//        P2  x/r updates and the two dot products per system
//        P3  per-system decisions (converged / reliable update due /
//            iteration cap / breakdown) and new search directions
//      separated by grid barriers (bounded spins: a timed-out barrier sets
//      an error flag and the kernel returns);
//   2. the FP64 refresh of systems that stopped: u += d, the FP64 true
//      residual f - K u (two-pass FP64 operator, all load cases of a beam in
//      one pass), convergence test on it, and for systems that go on the
//      residual replacement with the search direction kept.
// Rounds repeat (as a captured CUDA graph) until no system is active.
// Per-system scalars are double-buffered by iteration parity so that no
// block reads a value another block is writing.  At the start of every
// iteration each block rebuilds, in shared memory, the lists of the active
// beams and systems (every block from the same flags, so the lists agree),
// and every phase walks those lists: inactive systems cost nothing, and the
// active work splits evenly over the grid (the P2 and P3 of the Jacobi mode
// split the active systems' DOFs; the decisions run one system per thread).
//
// precond = 2 runs the same rounds with the two-level preconditioner
// z = D^-1 r + P Pi C Pi^T r of each beam's coarse space (coarse.cu) inside
// the persistent launch:
//        P2  walks each beam's nodes grouped by interpolation cell (runs
//            of <= kSubNodes nodes of one cell, one item per run and load
//            case), one warp per 64 nodes: the x/r updates, D^-1 r.r and
//            r.r, and the restriction rc += Pi^T r (24 warp sums, FP32
//            atomics into the system's rc);
//        P2c yc = C rc over (beam, 64 x 64 block of the packed C) items, the
//            block read once for all load cases of the beam, and
//            rc.C rc added to z.r (z.r = D^-1 r.r + (Pi^T r).yc);
//        P3  p = D^-1 r + P Pi yc + beta p;
// one grid barrier more per iteration (four).  The refresh computes the
// same z for the recomputed residuals (restriction and coarse product
// kernels over the same items).  Beams without a coarse space fall back to
// Jacobi inside the same launch (their P2 items are plain node ranges).

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "reduce.cuh"
#include "sfem_internal.cuh"
#include "tile_apply.cuh"

namespace sfem {

// bounded wait of the grid barrier: 4 s of global time (%globaltimer), and
// 2^24 sleeps as a second bound (measured 4.3 s: __nanosleep's duration is
// only approximate, so the count alone does not bound the time)
constexpr long long kBarrierSpinLimit = 1ll << 24;
constexpr unsigned long long kBarrierWaitNs = 4000000000ull;

__device__ __forceinline__ unsigned long long barrier_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct BatchBeam {
  TileArgs A;
  int first_sys, nrhs;
  float lam, mu;
  int64_t n_nodes;
  int has_cs;   // precond 2: the beam has a coarse space (else Jacobi)
  CoarseDev cs; // its coarse space (rc / yc unused: every system has its own)
};

struct BatchSys {
  double *x, *r, *d, *Kx;  // FP64: solution, residual, correction since the last refresh, K x
  float *p, *q;             // FP32: search direction and its FP32-operator image
  const double *dinv;
  const uint8_t *dmask;
  const double *f;
  int64_t n;
  double bnorm;
  float *rc, *yc;  // precond 2: restricted residual and coarse correction (npad each)
  int beam;
};

struct SysState {
  double rz, rz_prev, rr, rmax2, beta, relres;
  int iter, active, reason, status;  // reason: 1 conv, 2 refresh due, 3 cap, 4 breakdown
                                     // status: 0 running, 1 converged, 2 no conv, 3 breakdown,
                                     //         4 stagnated (finished by FP64 PCG on the host side)
  int fresh;                         // 1: reactivated by the last refresh (direction not yet updated)
  int stall;                         // refreshes in a row improving the best true residual by < 10%
  double best;                       // best true relative residual so far
};

__host__ __device__ inline size_t wl_align(size_t x) { return (x + 15) / 16 * 16; }

// byte offsets of the lists from the start of the area
struct WlLayout {
  int bm, bm2, bt, bch, bcb, bfs, bnr, act_b, act_na, pt, pu, pc, act_s, scan_i, pd, scan_l, sn, beta, bytes;
};

__host__ __device__ inline WlLayout wl_layout(int n_sys, int nb) {
  WlLayout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = wl_align(o + bytes);
    return (int)at;
  };
  const size_t nw = (size_t)(n_sys + 31) / 32;
  L.bm = take(4 * nw);
  L.bm2 = take(4 * nw);
  L.bt = take(4 * (size_t)nb);
  L.bch = take(4 * (size_t)nb);
  L.bcb = take(4 * (size_t)nb);
  L.bfs = take(4 * (size_t)nb);
  L.bnr = take(4 * (size_t)nb);
  L.act_b = take(4 * (size_t)nb);
  L.act_na = take(4 * (size_t)nb);
  L.pt = take(4 * ((size_t)nb + 1));
  L.pu = take(4 * ((size_t)nb + 1));
  L.pc = take(4 * ((size_t)nb + 1));
  L.act_s = take(4 * (size_t)n_sys);
  L.scan_i = take(4 * 9 * 4);
  L.pd = take(8 * ((size_t)n_sys + 1));
  L.scan_l = take(8 * 9 * 2);
  L.sn = take(8 * (size_t)n_sys);
  L.beta = take(8 * (size_t)n_sys);
  L.bytes = (int)o;
  return L;
}

struct BatchDev {
  const BatchBeam *beams;
  int n_beams;
  const BatchSys *sys;
  int n_sys;
  const int *work_prefix;  // n_beams + 1: tiles x load cases per beam (P1 items, few systems active)
  int total_work;
  const int *tile_prefix;  // n_beams + 1: tiles per beam (P1 items, most systems active)
  int total_tiles;
  int act_off;             // byte offset of the work lists in dynamic shared memory
  WlLayout wl;             // their layout
  const int64_t *sys_off;  // n_sys + 1: the systems' DOFs concatenated (update phases split this range)
  int64_t total_dof;
  SysState *state;         // 2 * n_sys, slot *slot is current
  int *slot;
  double *sums;            // 2 * n_sys * 2 (rz, rr)
  double *pq;              // 2 * n_sys
  double tol2;             // relative tolerance squared
  double delta2;
  int max_iter;
  int max_iter_launch;
  unsigned int *bar_count, *bar_gen;
  int *err;
  int *beam_skip;          // per beam: 1 if no system of it needs the FP64 refresh
  int *any_active;
  long long *iters_run;    // total CG iterations (summed over systems) of the last launch
  long long *launch_iters; // iterations of the persistent launches, summed over launches
  // precond 2 (two-level inside the launch)
  int two_level;
  const int *uwork_prefix; // n_beams + 1: node runs x load cases per beam (P2 items)
  int total_uwork;
  const int *cwork_prefix; // n_beams + 1: packed C blocks per beam (P2c items)
  int total_cwork;
  float *cvec;             // every system's rc and yc, concatenated
  int64_t cvec_len;
};

// state written by another block during the same launch: read through L2
__device__ __forceinline__ SysState load_state(const SysState *p) {
  SysState s;
  s.rz = __ldcg(&p->rz);
  s.rz_prev = __ldcg(&p->rz_prev);
  s.rr = __ldcg(&p->rr);
  s.rmax2 = __ldcg(&p->rmax2);
  s.beta = __ldcg(&p->beta);
  s.relres = __ldcg(&p->relres);
  s.iter = __ldcg(&p->iter);
  s.active = __ldcg(&p->active);
  s.reason = __ldcg(&p->reason);
  s.status = __ldcg(&p->status);
  s.fresh = __ldcg(&p->fresh);
  s.stall = __ldcg(&p->stall);
  s.best = __ldcg(&p->best);
  return s;
}

__device__ __forceinline__ bool grid_barrier(const BatchDev &a) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int *gen = a.bar_gen;
    const unsigned int g = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(a.bar_count, 1u);
    int good = 1;
    if (arrived == gridDim.x - 1) {
      *a.bar_count = 0u;
      __threadfence();
      atomicAdd(a.bar_gen, 1u);
    } else {
      long long spins = 0;
      const unsigned long long t0 = barrier_ns();
      while (*gen == g) {
        if (++spins > kBarrierSpinLimit || ((spins & 255) == 0 && barrier_ns() - t0 > kBarrierWaitNs)) {
          atomicExch(a.err, 1);
          good = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*(volatile int *)a.err) good = 0;
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// this block's range [g0, g1) of the concatenated DOFs and the first system
// that overlaps it
struct DofChunk {
  int64_t g0, g1;
  int s0;
};
__device__ __forceinline__ DofChunk dof_chunk(const BatchDev &a) {
  DofChunk ch;
  const int64_t per = (a.total_dof + gridDim.x - 1) / gridDim.x;
  ch.g0 = min(a.total_dof, (int64_t)blockIdx.x * per);
  ch.g1 = min(a.total_dof, ch.g0 + per);
  int lo = 0, hi = a.n_sys - 1;  // largest s with sys_off[s] <= g0
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.sys_off[mid] <= ch.g0)
      lo = mid;
    else
      hi = mid - 1;
  }
  ch.s0 = lo;
  return ch;
}

// the per-system decision after an update (identical in every block)
__device__ __forceinline__ SysState decide(const BatchDev &a, const SysState *st, const double *pq,
                                           const double *sums, int s) {
  const SysState ss = load_state(st + s);
  SysState n2 = ss;
  n2.fresh = 0;
  if (!ss.active) return n2;
  const double pqs = __ldcg(&pq[s]);
  const double alpha = ss.rz / pqs;
  const BatchSys &S = a.sys[s];
  if (!(pqs > 0.0) || !isfinite(alpha)) {
    n2.active = 0;
    n2.reason = 4;
    return n2;
  }
  const double rz_new = __ldcg(&sums[2 * s]), rr = __ldcg(&sums[2 * s + 1]);
  n2.iter = ss.iter + 1;
  n2.rz_prev = ss.rz;
  n2.rz = rz_new;
  n2.rr = rr;
  n2.beta = rz_new / ss.rz;
  n2.rmax2 = fmax(ss.rmax2, rr);
  if (!isfinite(rz_new) || !isfinite(rr)) {
    n2.active = 0;
    n2.reason = 4;
  } else if (rr <= a.tol2 * S.bnorm * S.bnorm) {
    n2.active = 0;
    n2.reason = 1;
  } else if (n2.iter >= a.max_iter) {
    n2.active = 0;
    n2.reason = 3;
  } else if (rr < a.delta2 * n2.rmax2) {
    n2.active = 0;
    n2.reason = 2;
  }
  return n2;
}

// ---- two-level phases (precond 2) ------------------------------------------

constexpr int kBatchWarpNodes = kSubNodes / (kTileThreads / 32);  // nodes per warp of a P2 item (2 per lane)
static_assert(kTileThreads == 256, "the coarse product maps 64 rows x 4 column groups onto 256 threads");

// largest b with prefix[b] <= w
__device__ __forceinline__ int find_item(const int *prefix, int n, int w) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= w)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// a system the current iteration steps (P2 / P2c): active with a valid step
__device__ __forceinline__ bool stepping(const SysState *st, const double *pq, int s, double &alpha) {
  if (!__ldcg(&st[s].active)) return false;
  const double pqs = __ldcg(&pq[s]);
  alpha = __ldcg(&st[s].rz) / pqs;
  return pqs > 0.0 && isfinite(alpha);
}

// a system whose residual the refresh recomputes
__device__ __forceinline__ bool refreshing(const SysState &ss) {
  return ss.status == 0 && !ss.active && ss.reason != 0;
}

// butterfly sum over the warp (every lane gets the total)
__device__ __forceinline__ float warp_allsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- work lists in shared memory ---------------------------------------------
// Every block rebuilds, at the start of each phase that needs them, the same
// lists of the work of the active systems (in a fixed order, from the same
// flags), so that its loops visit active items only and the items split
// evenly over the grid: per active beam e (ascending) the beam act_b[e], its
// active load cases act_na[e] and the exclusive prefixes of its tiles (pt),
// node runs x active load cases (pu) and coarse blocks (pc); per active
// system i the system act_s[i] and the prefix of their DOFs (pd).

struct WorkLists {
  unsigned *bm, *bm2;
  int *bt, *bch, *bcb, *bfs, *bnr;
  int *act_b, *act_na, *pt, *pu, *pc, *act_s, *scan_i;
  long long *pd, *scan_l, *sn;  // sn: DOFs of each system
  double *beta;                 // each system's new beta (P3)
};

__device__ __forceinline__ WorkLists work_lists(const BatchDev &a, float4 *smem) {
  char *base = reinterpret_cast<char *>(smem) + a.act_off;
  const WlLayout &L = a.wl;
  WorkLists W;
  W.bm = reinterpret_cast<unsigned *>(base + L.bm);
  W.bm2 = reinterpret_cast<unsigned *>(base + L.bm2);
  W.bt = reinterpret_cast<int *>(base + L.bt);
  W.bch = reinterpret_cast<int *>(base + L.bch);
  W.bcb = reinterpret_cast<int *>(base + L.bcb);
  W.bfs = reinterpret_cast<int *>(base + L.bfs);
  W.bnr = reinterpret_cast<int *>(base + L.bnr);
  W.act_b = reinterpret_cast<int *>(base + L.act_b);
  W.act_na = reinterpret_cast<int *>(base + L.act_na);
  W.pt = reinterpret_cast<int *>(base + L.pt);
  W.pu = reinterpret_cast<int *>(base + L.pu);
  W.pc = reinterpret_cast<int *>(base + L.pc);
  W.act_s = reinterpret_cast<int *>(base + L.act_s);
  W.scan_i = reinterpret_cast<int *>(base + L.scan_i);
  W.pd = reinterpret_cast<long long *>(base + L.pd);
  W.scan_l = reinterpret_cast<long long *>(base + L.scan_l);
  W.sn = reinterpret_cast<long long *>(base + L.sn);
  W.beta = reinterpret_cast<double *>(base + L.beta);
  return W;
}

// exclusive scan of K values per thread over the block (kTileThreads); the
// totals in tot (every thread); scratch holds 9 K values
template <class T, int K>
__device__ __forceinline__ void block_scan(T (&v)[K], T (&tot)[K], T *scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T inc[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    inc[q] = v[q];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T t = __shfl_up_sync(0xffffffffu, inc[q], o);
      if (lane >= o) inc[q] += t;
    }
  }
  if (lane == 31)
#pragma unroll
    for (int q = 0; q < K; ++q) scratch[warp * K + q] = inc[q];
  __syncthreads();
  if (warp == 0) {
    constexpr int NW = kTileThreads / 32;
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const T x0 = lane < NW ? scratch[lane * K + q] : T(0);
      T x = x0;
#pragma unroll
      for (int o = 1; o < NW; o <<= 1) {
        const T t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
      }
      __syncwarp();
      if (lane < NW) scratch[lane * K + q] = x - x0;
      if (lane == NW - 1) scratch[NW * K + q] = x;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) {
    v[q] = inc[q] - v[q] + scratch[warp * K + q];
    tot[q] = scratch[(kTileThreads / 32) * K + q];
  }
  __syncthreads();  // scratch is reused
}

__device__ __forceinline__ bool is_active(const unsigned *bm, int s) { return (bm[s >> 5] >> (s & 31)) & 1u; }

// flags of all systems into a bitmap (one load per system and block);
// returns the number of active systems
__device__ __forceinline__ int load_active(const BatchDev &a, const SysState *st, unsigned *bm) {
  int count = 0;
  for (int base = 0; base < a.n_sys; base += kTileThreads) {
    const int s = base + threadIdx.x;
    const bool f = s < a.n_sys && __ldcg(&st[s].active);
    const unsigned m = __ballot_sync(0xffffffffu, f);
    const int word = (base >> 5) + (threadIdx.x >> 5);
    if ((threadIdx.x & 31) == 0 && 32 * word < a.n_sys) bm[word] = m;
    count += __syncthreads_count(f);
  }
  return count;
}

// the beams' static counts (tiles, node runs, coarse blocks, first
// system, load cases) and the systems' DOFs, once per launch
__device__ __forceinline__ void load_beam_info(const BatchDev &a, const WorkLists &W) {
  for (int b = threadIdx.x; b < a.n_beams; b += kTileThreads) {
    const int nr = a.beams[b].nrhs;
    W.bt[b] = a.tile_prefix[b + 1] - a.tile_prefix[b];
    W.bch[b] = (a.uwork_prefix[b + 1] - a.uwork_prefix[b]) / nr;
    W.bcb[b] = a.cwork_prefix[b + 1] - a.cwork_prefix[b];
    W.bfs[b] = a.beams[b].first_sys;
    W.bnr[b] = nr;
  }
  for (int s = threadIdx.x; s < a.n_sys; s += kTileThreads) W.sn[s] = a.sys[s].n;
  __syncthreads();
}

// lists of the active beams from the flags in W.bm; returns the number of
// active beams, the item counts in n_items (tiles, node-run items, coarse blocks)
__device__ __forceinline__ int build_beam_lists(const BatchDev &a, const WorkLists &W, int (&n_items)[3]) {
  int carry[4] = {0, 0, 0, 0};
  for (int base = 0; base < a.n_beams; base += kTileThreads) {
    const int b = base + threadIdx.x;
    int na = 0;
    if (b < a.n_beams)
      for (int j = 0; j < W.bnr[b]; ++j) na += is_active(W.bm, W.bfs[b] + j) ? 1 : 0;
    int v[4] = {na > 0 ? 1 : 0, na > 0 ? W.bt[b] : 0, na * (b < a.n_beams ? W.bch[b] : 0), na > 0 ? W.bcb[b] : 0};
    int tot[4];
    block_scan<int, 4>(v, tot, W.scan_i);
    if (na > 0) {
      const int e = carry[0] + v[0];
      W.act_b[e] = b;
      W.act_na[e] = na;
      W.pt[e] = carry[1] + v[1];
      W.pu[e] = carry[2] + v[2];
      W.pc[e] = carry[3] + v[3];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) carry[q] += tot[q];
  }
  if (threadIdx.x == 0) {
    W.pt[carry[0]] = carry[1];
    W.pu[carry[0]] = carry[2];
    W.pc[carry[0]] = carry[3];
  }
  __syncthreads();
  n_items[0] = carry[1];
  n_items[1] = carry[2];
  n_items[2] = carry[3];
  return carry[0];
}

// list of the systems flagged in `flags` and the prefix of their DOFs;
// returns the number of systems, their DOFs in n_dof
__device__ __forceinline__ int build_sys_list(const BatchDev &a, const WorkLists &W, const unsigned *flags,
                                              long long &n_dof) {
  long long carry[2] = {0, 0};
  for (int base = 0; base < a.n_sys; base += kTileThreads) {
    const int s = base + threadIdx.x;
    const bool f = s < a.n_sys && is_active(flags, s);
    long long v[2] = {f ? 1 : 0, f ? W.sn[s] : 0};
    long long tot[2];
    block_scan<long long, 2>(v, tot, W.scan_l);
    if (f) {
      W.act_s[carry[0] + v[0]] = s;
      W.pd[carry[0] + v[0]] = carry[1] + v[1];
    }
    carry[0] += tot[0];
    carry[1] += tot[1];
  }
  if (threadIdx.x == 0) W.pd[carry[0]] = carry[1];
  __syncthreads();
  n_dof = carry[1];
  return (int)carry[0];
}

// entry of item w in a prefix list p[0..n] (sentinel p[n]), walking forward
// from e (the items of a block ascend)
__device__ __forceinline__ int walk_list(const int *p, int n, int e, int w) {
  while (e + 1 < n && p[e + 1] <= w) ++e;
  return e;
}

// j-th active load case of beam b (jj counts the active ones)
__device__ __forceinline__ int active_rhs(const WorkLists &W, int b, int jj) {
  int j = 0;
  for (;; ++j)
    if (is_active(W.bm, W.bfs[b] + j) && jj-- == 0) break;
  return j;
}

// P2 item: node run k (<= kSubNodes nodes of one interpolation cell) of
// beam b, load case j; this warp's kBatchWarpNodes
// nodes of it.  kUpdate: the CG update of a stepping system (d += alpha p,
// r = P (r - alpha q)) with D^-1 r.r and r.r into sums, then rc += Pi^T r;
// else (refresh) rc += Pi^T r of a refreshing system's new residual.
// No block barrier: warps past the chunk's end return at once.
template <bool kUpdate>
__device__ __forceinline__ void tl_update_item(const BatchDev &a, const SysState *st, const double *pq,
                                               double *sums, int b, int k, int j) {
  const BatchBeam &B = a.beams[b];
  const bool cs_on = B.has_cs != 0;
  if (!kUpdate && !cs_on) return;  // nothing to restrict
  int cell = 0, first, end;
  if (cs_on) {
    const int4 ch = B.cs.sub[k];
    cell = ch.x;
    first = ch.y;
    end = ch.z;
  } else {
    first = k * kSubNodes;
    end = (int)min((int64_t)first + kSubNodes, B.n_nodes);
  }
  const int lane = threadIdx.x & 31;
  const int wb = first + kBatchWarpNodes * (threadIdx.x >> 5);
  if (wb >= end) return;
  const int we = min(wb + kBatchWarpNodes, end);
  {
    const int s = B.first_sys + j;
    double alpha = 0.0;
    if (kUpdate) {
      if (!stepping(st, pq, s, alpha)) return;
    } else {
      if (!refreshing(st[s])) return;
    }
    const BatchSys &S = a.sys[s];
    double *__restrict__ d = S.d;
    double *__restrict__ r = S.r;
    const float *__restrict__ p = S.p;
    const float *__restrict__ q = S.q;
    const double *__restrict__ dinv = S.dinv;
    const uint8_t *__restrict__ dmask = S.dmask;
    const int32_t *__restrict__ cnodes = B.cs.cnodes;
    const float *__restrict__ frac = B.cs.frac;
    double rz = 0.0, rr = 0.0;
    float acc[24];
#pragma unroll
    for (int v = 0; v < 24; ++v) acc[v] = 0.f;
    for (int i = wb + lane; i < we; i += 32) {
      const int64_t node = cs_on ? (int64_t)cnodes[i] : (int64_t)i;
      float rf[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int64_t dof = 3 * node + c;
        double ri;
        if (kUpdate) {
          d[dof] = __ldcg(&d[dof]) + alpha * __ldcg(&p[dof]);
          ri = dmask[dof] ? __ldcg(&r[dof]) - alpha * __ldcg(&q[dof]) : 0.0;
          r[dof] = ri;
          rz += dinv[dof] * ri * ri;
          rr += ri * ri;
        } else {
          ri = __ldcg(&r[dof]);
        }
        rf[c] = (float)ri;
      }
      if (cs_on) {
        const float f[3] = {frac[3 * node], frac[3 * node + 1], frac[3 * node + 2]};
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const float wk = cs_weight(f, kk);
#pragma unroll
          for (int c = 0; c < 3; ++c) acc[3 * kk + c] = fmaf(wk, rf[c], acc[3 * kk + c]);
        }
      }
    }
    if (kUpdate) {
      rz = warp_allsum(rz);
      rr = warp_allsum(rr);
      if (lane == 0) {
        atomicAdd(&sums[2 * s], rz);
        atomicAdd(&sums[2 * s + 1], rr);
      }
    }
    if (cs_on) {
      float v[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) v[q] = q < 24 ? acc[q] : 0.f;
      const float t = warp_reduce_scatter32(v);  // lane l: the warp total of value l
      if (lane < 24) atomicAdd(&S.rc[3 * cs_corner(B.cs, cell, lane / 3) + lane % 3], t);
    }
  }
}

// P2c item (beam b, block t of the packed C): yc += C rc for every selected
// system of the beam (kUpdate: stepping; else refreshing), the block read
// once, and rc.C rc added to sums[2 s] (z.r).  Block-uniform; uses
// 2 x 64 + 8 x 64 floats of sm.
template <bool kUpdate>
__device__ __forceinline__ void tl_coarse_item(const BatchDev &a, const SysState *st, const double *pq,
                                               double *sums, int b, int t, float *sm) {
  const BatchBeam &B = a.beams[b];
  int ab = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((ab + 1) * (ab + 2) / 2 <= t) ++ab;
  while (ab * (ab + 1) / 2 > t) --ab;
  const int bb = t - ab * (ab + 1) / 2;
  const int i = threadIdx.x >> 2, q = threadIdx.x & 3;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float4 *blk = reinterpret_cast<const float4 *>(B.cs.C + (int64_t)t * 4096) + i * 16 + q * 4;
  float4 v[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) v[u] = __ldg(blk + u);
  float *ra = sm, *rb = sm + 64, *part = sm + 128;  // part: 8 warps x 64
  for (int j = 0; j < B.nrhs; ++j) {
    const int s = B.first_sys + j;
    double alpha;
    const bool sel = kUpdate ? stepping(st, pq, s, alpha) : refreshing(st[s]);
    if (!sel) continue;  // uniform over the block
    const BatchSys &S = a.sys[s];
    __syncthreads();
    if (threadIdx.x < 64) {
      ra[threadIdx.x] = __ldcg(&S.rc[ab * 64 + threadIdx.x]);
      rb[threadIdx.x] = __ldcg(&S.rc[bb * 64 + threadIdx.x]);
    }
    __syncthreads();
    // row i of C_ab times rb
    const float *rbq = rb + 16 * q;
    float acc = 0.f;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      acc = fmaf(v[u].x, rbq[4 * u],
                 fmaf(v[u].y, rbq[4 * u + 1], fmaf(v[u].z, rbq[4 * u + 2], fmaf(v[u].w, rbq[4 * u + 3], acc))));
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (q == 0) atomicAdd(&S.yc[ab * 64 + i], acc);
    // rc.C rc: ra_i (C_ab rb)_i, twice for an off-diagonal block (C_ba = C_ab^T)
    float e = q == 0 ? ra[i] * acc * (ab == bb ? 1.f : 2.f) : 0.f;
    e = warp_allsum(e);
    if (lane == 0) atomicAdd(&sums[2 * s], (double)e);
    if (ab == bb) continue;  // uniform
    // C_ab^T ra: column 16 q + 4 u + w gets v[u].{x,y,z,w} ra_i, summed over i
    const float ri = ra[i];
    float cpart[16];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      cpart[4 * u] = v[u].x * ri;
      cpart[4 * u + 1] = v[u].y * ri;
      cpart[4 * u + 2] = v[u].z * ri;
      cpart[4 * u + 3] = v[u].w * ri;
    }
#pragma unroll
    for (int kk = 0; kk < 16; ++kk)
#pragma unroll
      for (int o = 4; o < 32; o <<= 1) cpart[kk] += __shfl_xor_sync(0xffffffffu, cpart[kk], o);
    if (lane < 4)
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) part[warp * 64 + 16 * lane + kk] = cpart[kk];
    __syncthreads();
    if (threadIdx.x < 64) {
      float x = 0.f;
#pragma unroll
      for (int w2 = 0; w2 < 8; ++w2) x += part[w2 * 64 + threadIdx.x];
      atomicAdd(&S.yc[bb * 64 + threadIdx.x], x);
    }
  }
}

// new search directions p = z + beta p, q = 0 over DOFs [lo, hi) of system
// S, z = D^-1 r (+ P Pi yc with the two-level preconditioner)
__device__ __forceinline__ void batch_directions(const BatchDev &a, const BatchSys &S, int64_t lo, int64_t hi,
                                                 int64_t step, double beta) {
  float *__restrict__ p = S.p;
  float *__restrict__ q = S.q;
  const double *__restrict__ r = S.r;
  const double *__restrict__ dinv = S.dinv;
  const uint8_t *__restrict__ dmask = S.dmask;
  if (a.two_level && a.beams[S.beam].has_cs) {
    const CoarseDev cs = a.beams[S.beam].cs;
    const float *yc = S.yc;
    for (int64_t i = lo; i < hi; i += step) {
      double z = dinv[i] * __ldcg(&r[i]);
      if (dmask[i]) z += (double)cs_prolong_y(cs, yc, i);
      p[i] = (float)(z + beta * (double)__ldcg(&p[i]));
      q[i] = 0.f;
    }
  } else {
    for (int64_t i = lo; i < hi; i += step) {
      p[i] = (float)(dinv[i] * __ldcg(&r[i]) + beta * (double)__ldcg(&p[i]));
      q[i] = 0.f;
    }
  }
}

// MINB: CTAs per SM the register budget is compiled for (1, 2 or 3); the
// autotuner times the variants
template <int MINB>
__global__ void __launch_bounds__(kTileThreads, MINB) k_batch_cg(BatchDev a) {
  extern __shared__ float4 smem[];
  const int start = *a.slot;
  const WorkLists W = work_lists(a, smem);
  load_beam_info(a, W);
  int k = 0;
  long long iters = 0;  // block 0: systems stepped, summed over iterations (per thread)
  for (; k < a.max_iter_launch; ++k) {
    const int par = (start + k) & 1;
    const SysState *st = a.state + par * a.n_sys;
    double *pq = a.pq + par * a.n_sys;
    double *sums = a.sums + 2 * par * a.n_sys;
    // work lists of the systems active in this iteration
    load_active(a, st, W.bm);
    int n_items[3];
    const int n_e = build_beam_lists(a, W, n_items);
    // P1: operator over (active beam, tile) items, the tile's records loaded
    // once for all its active load cases
    if (a.two_level)  // rc and yc of every system start from zero (P3 of the last iteration is done with yc)
      for (int64_t i = (int64_t)blockIdx.x * kTileThreads + threadIdx.x; i < a.cvec_len;
           i += (int64_t)gridDim.x * kTileThreads)
        a.cvec[i] = 0.f;
    for (int w = blockIdx.x, e = 0; w < n_items[0]; w += gridDim.x) {
      e = walk_list(W.pt, n_e, e, w);
      const int b = W.act_b[e], tile = w - W.pt[e];
      const BatchBeam &B = a.beams[b];
      TileRegs R;
      tile_load(B.A, tile, R);
      for (int j = 0; j < W.bnr[b]; ++j) {
        const int s = W.bfs[b] + j;
        if (!is_active(W.bm, s)) continue;
        const BatchSys &S = a.sys[s];
        tile_compute<float, float, true>(B.A, tile, R, S.p, S.q, B.lam, B.mu, smem, &pq[s]);
      }
    }
    if (!grid_barrier(a)) return;
    if (a.two_level) {
      // P2: updates and restriction over (active beam, node chunk, active
      // load case) items
      for (int w = blockIdx.x, e = 0; w < n_items[1]; w += gridDim.x) {
        e = walk_list(W.pu, n_e, e, w);
        const int b = W.act_b[e], local = w - W.pu[e], na = W.act_na[e];
        const int chunk = local / na;
        tl_update_item<true>(a, st, pq, sums, b, chunk, active_rhs(W, b, local - chunk * na));
      }
      if (!grid_barrier(a)) return;
      // P2c: coarse products over (active beam, C block) items
      float *sm = reinterpret_cast<float *>(smem);
      for (int w = blockIdx.x, e = 0; w < n_items[2]; w += gridDim.x) {
        e = walk_list(W.pc, n_e, e, w);
        tl_coarse_item<true>(a, st, pq, sums, W.act_b[e], w - W.pc[e], sm);
        __syncthreads();  // sm is reused by the next item
      }
    } else {
      // P2: updates of the active systems over this block's share of their
      // DOFs (a block meets one or two systems)
      long long n_dof = 0;
      const int n_s = build_sys_list(a, W, W.bm, n_dof);
      const long long per = (n_dof + gridDim.x - 1) / gridDim.x;
      const long long g0 = min(n_dof, (long long)blockIdx.x * per), g1 = min(n_dof, g0 + per);
      int i = 0;
      while (i + 1 < n_s && W.pd[i + 1] <= g0) ++i;
      for (; g0 < g1 && i < n_s && W.pd[i] < g1; ++i) {
        const int s = W.act_s[i];
        double alpha;
        if (!stepping(st, pq, s, alpha)) continue;
        const BatchSys &S = a.sys[s];
        const int64_t lo = max(g0, W.pd[i]) - W.pd[i], hi = min(g1, W.pd[i + 1]) - W.pd[i];
        double rz = 0.0, rr = 0.0;
        for (int64_t t = lo + threadIdx.x; t < hi; t += kTileThreads) {
          S.d[t] = __ldcg(&S.d[t]) + alpha * (double)__ldcg(&S.p[t]);
          const double ri = S.dmask[t] ? __ldcg(&S.r[t]) - alpha * (double)__ldcg(&S.q[t]) : 0.0;
          S.r[t] = ri;
          rz += S.dinv[t] * ri * ri;
          rr += ri * ri;
        }
        rz = block_sum<kTileThreads>(rz);
        rr = block_sum<kTileThreads>(rr);
        if (threadIdx.x == 0) {
          atomicAdd(&sums[2 * s], rz);
          atomicAdd(&sums[2 * s + 1], rr);
        }
      }
    }
    if (!grid_barrier(a)) return;
    // P3: decisions, one system per thread (identical in every block; block
    // 0 stores them), then new directions over this block's share of the
    // DOFs of the systems that go on
    SysState *nx = a.state + (par ^ 1) * a.n_sys;
    for (int base = 0; base < a.n_sys; base += kTileThreads) {
      const int s = base + threadIdx.x;
      bool act = false;
      if (s < a.n_sys) {
        const SysState n2 = decide(a, st, pq, sums, s);
        act = n2.active != 0;
        W.beta[s] = n2.beta;
        if (blockIdx.x == 0) {
          nx[s] = n2;
          double *nsums = a.sums + 2 * (par ^ 1) * a.n_sys;
          nsums[2 * s] = 0.0;
          nsums[2 * s + 1] = 0.0;
          a.pq[(par ^ 1) * a.n_sys + s] = 0.0;
          if (is_active(W.bm, s)) ++iters;
        }
      }
      const unsigned m = __ballot_sync(0xffffffffu, act);
      const int word = (base >> 5) + (threadIdx.x >> 5);
      if ((threadIdx.x & 31) == 0 && 32 * word < a.n_sys) W.bm2[word] = m;
    }
    __syncthreads();
    long long n_dof = 0;
    const int n_s = build_sys_list(a, W, W.bm2, n_dof);
    {
      const long long per = (n_dof + gridDim.x - 1) / gridDim.x;
      const long long g0 = min(n_dof, (long long)blockIdx.x * per), g1 = min(n_dof, g0 + per);
      int i = 0;
      while (i + 1 < n_s && W.pd[i + 1] <= g0) ++i;
      for (; g0 < g1 && i < n_s && W.pd[i] < g1; ++i) {
        const int s = W.act_s[i];
        const int64_t lo = max(g0, W.pd[i]) - W.pd[i], hi = min(g1, W.pd[i + 1]) - W.pd[i];
        batch_directions(a, a.sys[s], lo + threadIdx.x, hi, kTileThreads, W.beta[s]);
      }
    }
    if (n_s == 0) {
      ++k;
      break;
    }
    if (!grid_barrier(a)) return;
  }
  if (blockIdx.x == 0) {
    __shared__ unsigned long long s_it;
    if (threadIdx.x == 0) s_it = 0ull;
    __syncthreads();
    if (iters) atomicAdd(&s_it, (unsigned long long)iters);
    __syncthreads();
    if (threadIdx.x == 0) {
      *a.slot = (start + k) & 1;
      *a.iters_run = (long long)s_it;
      *a.launch_iters += k;
    }
  }
}

// ---- FP64 refresh kernels ---------------------------------------------------
// systems that stopped for a reason other than a final status: u += d, d = 0;
// beam_skip[b] = 1 when no system of beam b needs its residual recomputed
__global__ void k_refresh_x(BatchDev a) {
  const SysState *st = a.state + (*a.slot) * a.n_sys;
  const DofChunk ch = dof_chunk(a);
  for (int s = ch.s0; s < a.n_sys && a.sys_off[s] < ch.g1; ++s) {
    const SysState &ss = st[s];
    if (ss.status != 0 || ss.active || ss.reason == 0) continue;
    const BatchSys &S = a.sys[s];
    const int64_t lo = max(ch.g0, a.sys_off[s]) - a.sys_off[s], hi = min(ch.g1, a.sys_off[s + 1]) - a.sys_off[s];
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      S.x[i] += S.d[i];
      S.d[i] = 0.0;
    }
  }
  if (a.two_level)  // rc and yc start from zero for the refresh's restriction
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.cvec_len;
         i += (int64_t)gridDim.x * blockDim.x)
      a.cvec[i] = 0.f;
  if (blockIdx.x == 0) {
    for (int b = threadIdx.x; b < a.n_beams; b += blockDim.x) {
      const BatchBeam &B = a.beams[b];
      int need = 0;
      for (int j = 0; j < B.nrhs; ++j) {
        const SysState &ss = st[B.first_sys + j];
        need |= (ss.status == 0 && !ss.active && ss.reason != 0);
      }
      a.beam_skip[b] = need ? 0 : 1;
    }
  }
}

// r = P (f - K u) and its sums (rz~, |r|^2) for systems being refreshed
__global__ void __launch_bounds__(256) k_refresh_r(BatchDev a) {
  const SysState *st = a.state + (*a.slot) * a.n_sys;
  double *sums = a.sums + 2 * (*a.slot) * a.n_sys;
  const DofChunk ch = dof_chunk(a);
  for (int s = ch.s0; s < a.n_sys && a.sys_off[s] < ch.g1; ++s) {
    const SysState &ss = st[s];
    if (ss.status != 0 || ss.active || ss.reason == 0) continue;
    const BatchSys &S = a.sys[s];
    double rz = 0.0, rr = 0.0;
    const int64_t lo = max(ch.g0, a.sys_off[s]) - a.sys_off[s], hi = min(ch.g1, a.sys_off[s + 1]) - a.sys_off[s];
    for (int64_t i = lo + threadIdx.x; i < hi; i += 256) {
      const double ri = S.dmask[i] ? S.f[i] - S.Kx[i] : 0.0;
      S.r[i] = ri;
      rz += S.dinv[i] * ri * ri;
      rr += ri * ri;
    }
    rz = block_sum<256>(rz);
    rr = block_sum<256>(rr);
    if (threadIdx.x == 0) {
      atomicAdd(&sums[2 * s], rz);
      atomicAdd(&sums[2 * s + 1], rr);
    }
  }
}

// precond 2: rc = Pi^T r of the recomputed residuals (after k_refresh_r)
__global__ void __launch_bounds__(kTileThreads) k_refresh_restrict(BatchDev a) {
  const SysState *st = a.state + (*a.slot) * a.n_sys;
  for (int w = blockIdx.x; w < a.total_uwork; w += gridDim.x) {
    const int b = find_item(a.uwork_prefix, a.n_beams, w);
    const int nr = a.beams[b].nrhs, local = w - a.uwork_prefix[b];
    tl_update_item<false>(a, st, nullptr, nullptr, b, local / nr, local % nr);
  }
}

// precond 2: yc = C rc and rc.C rc into z.r of the refreshed systems
__global__ void __launch_bounds__(kTileThreads) k_refresh_coarse(BatchDev a) {
  __shared__ float sm[2 * 64 + 8 * 64];
  const SysState *st = a.state + (*a.slot) * a.n_sys;
  double *sums = a.sums + 2 * (*a.slot) * a.n_sys;
  for (int w = blockIdx.x; w < a.total_cwork; w += gridDim.x) {
    const int b = find_item(a.cwork_prefix, a.n_beams, w);
    tl_coarse_item<false>(a, st, nullptr, sums, b, w - a.cwork_prefix[b], sm);
    __syncthreads();
  }
}

// decisions on the FP64 true residual (one thread per system)
__global__ void k_refresh_state(BatchDev a) {
  SysState *st = a.state + (*a.slot) * a.n_sys;
  double *sums = a.sums + 2 * (*a.slot) * a.n_sys;
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < a.n_sys; s += blockDim.x) {
    SysState ss = st[s];
    if (ss.status == 0 && !ss.active && ss.reason != 0) {
      const BatchSys &S = a.sys[s];
      const double rz = sums[2 * s], rr = sums[2 * s + 1];
      const double rel = S.bnorm > 0.0 ? sqrt(rr) / S.bnorm : 0.0;
      ss.relres = rel;
      // stagnation: the FP32 operator's error floor is above the tolerance
      if (rel < 0.9 * ss.best) {
        ss.best = rel;
        ss.stall = 0;
      } else {
        ss.stall += 1;
      }
      if (ss.reason == 4) {
        ss.status = 3;
      } else if (rel * rel <= a.tol2) {
        ss.status = 1;
      } else if (ss.iter >= a.max_iter) {
        ss.status = 2;
      } else if (ss.stall >= 3) {
        ss.status = 4;
      } else {
        ss.active = 1;
        ss.beta = isfinite(ss.rz_prev) && ss.rz_prev > 0.0 ? rz / ss.rz_prev : 0.0;
        ss.rz = rz;
        ss.rr = rr;
        ss.rmax2 = rr;
        ss.reason = 0;
        ss.fresh = 1;
        atomicOr(&any, 1);
      }
      st[s] = ss;
    } else if (ss.active) {
      atomicOr(&any, 1);
    }
    sums[2 * s] = 0.0;
    sums[2 * s + 1] = 0.0;
    a.pq[(*a.slot) * a.n_sys + s] = 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) *a.any_active = any;
}

// new directions of the systems this refresh reactivated (systems still
// active because the launch hit its iteration cap already have theirs):
// p = z + beta p (z = D^-1 r, plus P Pi yc with precond 2), q = 0
__global__ void k_refresh_p(BatchDev a) {
  const SysState *st = a.state + (*a.slot) * a.n_sys;
  for (int s = 0; s < a.n_sys; ++s) {
    const SysState &ss = st[s];
    if (!ss.active || !ss.fresh) continue;
    batch_directions(a, a.sys[s], (int64_t)blockIdx.x * blockDim.x + threadIdx.x, a.sys[s].n,
                     (int64_t)gridDim.x * blockDim.x, ss.beta);
  }
}

__global__ void k_batch_init(BatchSys *sys, int n_sys, SysState *state) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_sys) return;
  SysState z;
  memset(&z, 0, sizeof z);
  z.rz_prev = INFINITY;
  z.best = INFINITY;
  z.reason = 2;  // needs its first residual
  state[s] = z;
  state[n_sys + s] = z;
}

__global__ void k_set_bc_all(double *x, const double *g, const uint8_t *dmask, int64_t n, int nrhs, bool zero_free) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * nrhs) return;
  const int64_t k = i % n;
  if (!dmask[k])
    x[i] = g[k];
  else if (zero_free)
    x[i] = 0.0;
}

// ---- autotuner: persistent-kernel CTAs per SM, cached per shape class -----
static std::mutex g_tune_mu;
static std::map<long long, int> g_tune_cache;  // key: (device, total tiles, mode) -> CTAs per SM

// Self-test of the bounded wait in grid_barrier: one CTA enters the barrier
// with the arrival counter offset by one, so it is never the last arrival
// and no block advances the generation.  Its wait runs out after
// kBarrierWaitNs (a few seconds), sets the error word and returns
// false; nothing else waits on it.
__global__ void k_barrier_selftest(BatchDev a, int *passed) {
  const bool ok = grid_barrier(a);
  if (threadIdx.x == 0) *passed = ok ? 1 : 0;
}

}  // namespace sfem

using namespace sfem;

// patch width (node spacings) of the coarse spaces the batched modes build:
// finer than the single-system default of 8, measured on the 64 x 4 batch
// of uneven cantilevers (6: 135k iterations and 1.10 s, against 181k and
// 1.40 s with 8, coarse setup 59 against 42 ms for the 64 beams; 5 leaves
// some coarse matrices not positive definite)
constexpr int kBatchPatchNodes = 6;

// precond = 1: every system by the two-level mixed-precision solve of its
// own context (IR32_64 with FP32 inner vectors and the Galerkin coarse
// correction, coarse space built with the default options where possible,
// else Jacobi), one after the other.  With the coarse correction a system
// needs about a sixth of the Jacobi iterations that the persistent kernel
// runs.  (Eight host threads driving different beams' contexts at once
// measured no faster: 6.95 vs 6.63 s on the 64-beam batch.)
static int batch_two_level(sfem_ctx *const *ctxs, int n, double *const *u, const sfem_batch_opts &o, double tol,
                           int max_iter, sfem_solve_info *infos, sfem_batch_stats *stats) {
  const auto t0 = std::chrono::steady_clock::now();
  int worst = SFEM_OK, k2 = 0, fallbacks = 0;
  long long total_it = 0;
  for (int b = 0; b < n; ++b) {
    Ctx &c = ctxs[b]->c;
    const bool coarse = o.patch_nodes < 0 ? c.coarse != nullptr
                                          : ensure_coarse(c, o.patch_nodes > 0 ? o.patch_nodes : kBatchPatchNodes);
    for (int j = 0; j < c.nrhs; ++j, ++k2) {
      sfem_solve_opts so{};
      so.kind = SFEM_SOLVE_IR32_64;
      so.op64 = SFEM_OP_MF64;
      so.rhs = j;
      so.u_on_device = o.u_on_device;
      so.warm_start = o.warm_start;
      so.tol = tol;
      so.max_iter = max_iter;
      so.inner_tol = o.inner_tol > 0 ? o.inner_tol : 0.03;
      so.precond = coarse ? 1 : 0;
      so.fp32_vectors = coarse ? 3 : 0;
      sfem_solve_info info{};
      const int rc = sfem_solve(ctxs[b], nullptr, u[b] + (int64_t)j * c.ndof, &so, &info);
      if (rc != SFEM_OK && worst == SFEM_OK) worst = rc;
      total_it += info.iterations;
      fallbacks += info.fallbacks;
      if (infos) infos[k2] = info;
    }
  }
  for (int b = 0; b < n; ++b) SFEM_CUDA(cudaStreamSynchronize(ctxs[b]->c.stream));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (stats) {
    *stats = sfem_batch_stats{};
    stats->n_systems = k2;
    stats->total_iterations = total_it;
    stats->ms = ms;
    stats->fallback_systems = fallbacks;
  }
  if (worst != SFEM_OK) set_last_error("some systems of the batch did not converge");
  return worst;
}

extern "C" int sfem_batch_solve(sfem_ctx *const *ctxs, int n, double *const *u, const sfem_batch_opts *opts,
                                sfem_solve_info *infos, sfem_batch_stats *stats) {
  std::vector<void *> owned;
  Ctx *c0 = nullptr;
  auto cleanup = [&]() {
    if (c0)
      for (void *p : owned) c0->mem.drop(p);
    owned.clear();
  };
  try {
    SFEM_REQUIRE(ctxs && n >= 1 && u && opts, SFEM_EINVAL, "ctxs, u and opts must not be NULL");
    for (int r : opts->reserved) SFEM_REQUIRE(r == 0, SFEM_EINVAL, "reserved options must be zero");
    c0 = &ctxs[0]->c;
    cudaStream_t st = c0->stream;
    int dev = -1;
    SFEM_CUDA(cudaGetDevice(&dev));
    int n_sys = 0, total_work = 0;
    size_t smem = 0;
    for (int b = 0; b < n; ++b) {
      SFEM_REQUIRE(ctxs[b] && ctxs[b]->c.vol && ctxs[b]->c.tl.ready, SFEM_EINVAL, "context not set up");
      SFEM_REQUIRE(ctxs[b]->c.device == dev, SFEM_EINVAL, "all contexts must live on the current device");
      n_sys += ctxs[b]->c.nrhs;
      total_work += (int)ctxs[b]->c.tl.n_tiles;
      smem = std::max(smem, ctxs[b]->c.tl.smem);
    }
    const double tol = opts->tol > 0 ? opts->tol : 1e-8;
    const bool two_level = opts->precond == 2;
    const double delta = opts->inner_tol > 0 ? opts->inner_tol : two_level ? 0.03 : 0.1;
    const int max_iter = opts->max_iter > 0 ? opts->max_iter : 200000;
    const int max_rounds = opts->max_rounds > 0 ? opts->max_rounds : 400;
    SFEM_REQUIRE(opts->precond >= 0 && opts->precond <= 2, SFEM_EINVAL, "precond must be 0, 1 or 2");
    SFEM_REQUIRE(opts->patch_nodes >= -1 && opts->patch_nodes <= 4096, SFEM_EINVAL, "patch_nodes out of range");
    if (opts->precond == 1) return batch_two_level(ctxs, n, u, *opts, tol, max_iter, infos, stats);
    auto get = [&](size_t bytes) {
      void *p = c0->mem.raw(bytes);
      owned.push_back(p);
      return p;
    };

    cudaEvent_t e0, e1;
    SFEM_CUDA(cudaEventCreate(&e0));
    SFEM_CUDA(cudaEventCreate(&e1));
    SFEM_CUDA(cudaEventRecord(e0, st));

    // per-beam vectors and host-side tables
    std::vector<BatchBeam> hb(n);
    std::vector<BatchSys> hs(n_sys);
    std::vector<int> prefix(n + 1, 0), tprefix(n + 1, 0), uprefix(n + 1, 0), cprefix(n + 1, 0);
    std::vector<double *> xbeam(n), kxbeam(n);
    // precond 2: coarse spaces (built with the default options on first use,
    // kept by the contexts) and every system's rc / yc
    int64_t cvec_len = 0;
    if (two_level)
      for (int b = 0; b < n; ++b) {
        Ctx &c = ctxs[b]->c;
        const bool cs_on = opts->patch_nodes < 0 ? c.coarse != nullptr
                                                  : ensure_coarse(c, opts->patch_nodes > 0 ? opts->patch_nodes
                                                                                           : kBatchPatchNodes);
        if (cs_on) cvec_len += 2 * (int64_t)c.coarse->dev.npad * c.nrhs;
      }
    float *cvec = cvec_len ? (float *)get(cvec_len * sizeof(float)) : nullptr;
    int64_t coff = 0;
    int s = 0;
    for (int b = 0; b < n; ++b) {
      Ctx &c = ctxs[b]->c;
      const int64_t nd = c.ndof;
      const int nr = c.nrhs;
      double *X = (double *)get(nd * nr * sizeof(double));
      double *R = (double *)get(nd * nr * sizeof(double));
      float *P = (float *)get(nd * nr * sizeof(float));
      float *Q = (float *)get(nd * nr * sizeof(float));
      double *D = (double *)get(nd * nr * sizeof(double));
      double *KX = (double *)get(nd * nr * sizeof(double));
      xbeam[b] = X;
      kxbeam[b] = KX;
      ensure_w_scratch(c, (size_t)c.n_tets * 8 * sizeof(double) * nr);
      if (opts->warm_start)
        SFEM_CUDA(cudaMemcpyAsync(X, u[b], nd * nr * sizeof(double),
                                  opts->u_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
      k_set_bc_all<<<grid_for(nd * nr, 256), 256, 0, st>>>(X, c.g, c.dmask, nd, nr, !opts->warm_start);
      SFEM_CHECK_LAUNCH();
      SFEM_CUDA(cudaMemsetAsync(D, 0, nd * nr * sizeof(double), st));
      for (float *v : {P, Q}) SFEM_CUDA(cudaMemsetAsync(v, 0, nd * nr * sizeof(float), st));
      hb[b].A = TileArgs{c.tl.tile_start, c.tl.hoff,     c.tl.noff, c.tl.halo_tet, c.tl.halo_lconn,
                         c.tl.tile_nodes, c.tl.node_inc, c.tl.rec,  c.n_tets,       c.tl.slot_stride};
      hb[b].first_sys = s;
      hb[b].nrhs = nr;
      hb[b].lam = (float)c.lam;
      hb[b].mu = (float)c.mu;
      hb[b].n_nodes = c.n_nodes;
      const bool cs_on = two_level && c.coarse;
      hb[b].has_cs = cs_on ? 1 : 0;
      if (cs_on) hb[b].cs = c.coarse->dev;
      prefix[b + 1] = prefix[b] + (int)c.tl.n_tiles * nr;
      tprefix[b + 1] = tprefix[b] + (int)c.tl.n_tiles;
      const int npad = cs_on ? c.coarse->dev.npad : 0;
      uprefix[b + 1] =
          uprefix[b] + nr * (cs_on ? c.coarse->dev.nsub : (int)((c.n_nodes + kSubNodes - 1) / kSubNodes));
      cprefix[b + 1] = cprefix[b] + (cs_on ? (npad / 64) * (npad / 64 + 1) / 2 : 0);
      for (int j = 0; j < nr; ++j, ++s) {
        BatchSys &S = hs[s];
        S.x = X + j * nd;
        S.r = R + j * nd;
        S.p = P + j * nd;
        S.q = Q + j * nd;
        S.d = D + j * nd;
        S.Kx = KX + j * nd;
        S.dinv = c.dinv64;
        S.dmask = c.dmask;
        S.f = c.f + j * nd;
        S.n = nd;
        S.bnorm = c.bnorm[j];
        S.beam = b;
        S.rc = cs_on ? cvec + coff : nullptr;
        S.yc = cs_on ? cvec + coff + npad : nullptr;
        coff += 2 * (int64_t)npad;
      }
    }
    std::vector<int64_t> soff(n_sys + 1, 0);
    for (int k2 = 0; k2 < n_sys; ++k2) soff[k2 + 1] = soff[k2] + hs[k2].n;
    BatchDev a{};
    a.sys_off = (const int64_t *)get((n_sys + 1) * sizeof(int64_t));
    SFEM_CUDA(cudaMemcpyAsync((void *)a.sys_off, soff.data(), (n_sys + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                              st));
    a.total_dof = soff[n_sys];
    a.beams = (BatchBeam *)get(n * sizeof(BatchBeam));
    a.sys = (BatchSys *)get(n_sys * sizeof(BatchSys));
    a.work_prefix = (int *)get((n + 1) * sizeof(int));
    a.tile_prefix = (int *)get((n + 1) * sizeof(int));
    SFEM_CUDA(cudaMemcpyAsync((void *)a.tile_prefix, tprefix.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice,
                              st));
    a.total_tiles = tprefix[n];
    a.uwork_prefix = (int *)get((n + 1) * sizeof(int));
    a.cwork_prefix = (int *)get((n + 1) * sizeof(int));
    SFEM_CUDA(cudaMemcpyAsync((void *)a.uwork_prefix, uprefix.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice,
                              st));
    SFEM_CUDA(cudaMemcpyAsync((void *)a.cwork_prefix, cprefix.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice,
                              st));
    a.total_uwork = uprefix[n];
    a.total_cwork = cprefix[n];
    a.two_level = two_level ? 1 : 0;
    a.cvec = cvec;
    a.cvec_len = cvec_len;
    SFEM_CUDA(cudaMemcpyAsync((void *)a.beams, hb.data(), n * sizeof(BatchBeam), cudaMemcpyHostToDevice, st));
    SFEM_CUDA(cudaMemcpyAsync((void *)a.sys, hs.data(), n_sys * sizeof(BatchSys), cudaMemcpyHostToDevice, st));
    SFEM_CUDA(cudaMemcpyAsync((void *)a.work_prefix, prefix.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice,
                              st));
    a.n_beams = n;
    a.n_sys = n_sys;
    a.total_work = prefix[n];
    // the work lists follow the tile view in dynamic shared memory
    a.act_off = (int)std::max<size_t>(wl_align(smem), 640 * sizeof(float));  // P2c uses 640 floats
    a.wl = wl_layout(n_sys, n);
    smem = (size_t)a.act_off + (size_t)a.wl.bytes;
    SFEM_REQUIRE(smem <= 227 * 1024, SFEM_EINVAL, "too many systems or beams for the batched kernel's shared memory");
    a.state = (SysState *)get(2 * n_sys * sizeof(SysState));
    a.slot = (int *)get(sizeof(int));
    a.sums = (double *)get(4 * n_sys * sizeof(double));
    a.pq = (double *)get(2 * n_sys * sizeof(double));
    a.bar_count = (unsigned int *)get(2 * sizeof(unsigned int));
    a.bar_gen = a.bar_count + 1;
    a.err = (int *)get(sizeof(int));
    a.beam_skip = (int *)get(n * sizeof(int));
    a.any_active = (int *)get(sizeof(int));
    a.iters_run = (long long *)get(sizeof(long long));
    a.launch_iters = (long long *)get(sizeof(long long));
    SFEM_CUDA(cudaMemsetAsync(a.launch_iters, 0, sizeof(long long), st));
    a.tol2 = tol * tol;
    a.delta2 = delta * delta;
    a.max_iter = max_iter;
    a.max_iter_launch = opts->iters_per_launch > 0 ? opts->iters_per_launch : 2000;
    SFEM_CUDA(cudaMemsetAsync(a.slot, 0, sizeof(int), st));
    SFEM_CUDA(cudaMemsetAsync(a.sums, 0, 4 * n_sys * sizeof(double), st));
    SFEM_CUDA(cudaMemsetAsync(a.pq, 0, 2 * n_sys * sizeof(double), st));
    SFEM_CUDA(cudaMemsetAsync(a.bar_count, 0, 2 * sizeof(unsigned int), st));
    SFEM_CUDA(cudaMemsetAsync(a.err, 0, sizeof(int), st));
    k_batch_init<<<grid_for(n_sys, 128), 128, 0, st>>>((BatchSys *)a.sys, n_sys, a.state);
    SFEM_CHECK_LAUNCH();

    // launch shapes of the persistent kernel: variant v compiled for v CTAs
    // per SM, usable when that many fit (registers and shared memory)
    int sms = 0;
    SFEM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    void (*variants[3])(BatchDev) = {k_batch_cg<1>, k_batch_cg<2>, k_batch_cg<3>};
    int occ = 0;  // largest v whose variant reaches v CTAs per SM
    for (int v = 1; v <= 3; ++v) {
      SFEM_CUDA(cudaFuncSetAttribute(variants[v - 1], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      int o = 0;
      SFEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, variants[v - 1], kTileThreads, smem));
      if (o >= v) occ = v;
    }
    SFEM_REQUIRE(occ >= 1, SFEM_EINVAL, "the batched kernel does not fit on an SM");
    const int red_grid = std::max(1, sms * 4);

    auto launch_persistent = [&](int bpsm, cudaStream_t s2) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(bpsm * sms));
      cfg.blockDim = dim3(kTileThreads);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = s2;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      SFEM_CUDA(cudaLaunchKernelEx(&cfg, variants[bpsm - 1], a));
      if (!capturing()) count_launches(1);
    };
    auto enqueue_refresh = [&](cudaStream_t s2) {
      k_refresh_x<<<red_grid, 256, 0, s2>>>(a);
      SFEM_CHECK_LAUNCH();
      for (int b = 0; b < n; ++b) {
        Ctx &c = ctxs[b]->c;
        SFEM_CUDA(cudaMemsetAsync(kxbeam[b], 0, c.ndof * c.nrhs * sizeof(double), s2));
        double *w = static_cast<double *>(c.w_scratch);
        launch_mf_strain<double, double>(c, s2, c.Gs64, xbeam[b], c.nrhs, w, a.beam_skip + b);
        launch_mf_stress<double, double>(c, s2, c.Gs64, c.kap64, w, kxbeam[b], c.nrhs, nullptr, a.beam_skip + b);
      }
      k_refresh_r<<<red_grid, 256, 0, s2>>>(a);
      SFEM_CHECK_LAUNCH();
      if (two_level) {
        k_refresh_restrict<<<red_grid, kTileThreads, 0, s2>>>(a);
        SFEM_CHECK_LAUNCH();
        k_refresh_coarse<<<red_grid, kTileThreads, 0, s2>>>(a);
        SFEM_CHECK_LAUNCH();
      }
      k_refresh_state<<<1, 256, 0, s2>>>(a);
      SFEM_CHECK_LAUNCH();
      k_refresh_p<<<red_grid, 256, 0, s2>>>(a);
      SFEM_CHECK_LAUNCH();
    };
    int err = 0, any = 0;
    auto check = [&]() {
      SFEM_CUDA(cudaMemcpyAsync(&err, a.err, sizeof(int), cudaMemcpyDeviceToHost, st));
      SFEM_CUDA(cudaMemcpyAsync(&any, a.any_active, sizeof(int), cudaMemcpyDeviceToHost, st));
      SFEM_CUDA(cudaStreamSynchronize(st));
      SFEM_REQUIRE(err == 0, SFEM_ETIMEOUT, "a grid barrier of the batched solver timed out");
    };

    // first residuals (all systems)
    enqueue_refresh(st);
    check();

    // autotune CTAs per SM on the first rounds (cached per shape class)
    const long long key = ((long long)dev << 40) | ((long long)total_work << 1) | (two_level ? 1 : 0);
    int bpsm = 0;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) bpsm = it->second;
    }
    int rounds = 0;
    if (bpsm == 0 && opts->autotune) {
      double best = 1e300;
      const int saved = a.max_iter_launch;
      for (int cand = 1; cand <= occ && any; ++cand) {
        a.max_iter_launch = 40;
        cudaEvent_t t0, t1;
        SFEM_CUDA(cudaEventCreate(&t0));
        SFEM_CUDA(cudaEventCreate(&t1));
        SFEM_CUDA(cudaEventRecord(t0, st));
        launch_persistent(cand, st);
        SFEM_CUDA(cudaEventRecord(t1, st));
        long long its = 0;
        SFEM_CUDA(cudaMemcpyAsync(&its, a.iters_run, sizeof its, cudaMemcpyDeviceToHost, st));
        enqueue_refresh(st);
        check();
        float ms = 0.f;
        SFEM_CUDA(cudaEventElapsedTime(&ms, t0, t1));
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        ++rounds;
        const double per = its > 0 ? ms / (double)its : 1e300;
        if (per < best) {
          best = per;
          bpsm = cand;
        }
      }
      a.max_iter_launch = saved;
      if (bpsm > 0) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = bpsm;
      }
    }
    if (bpsm == 0) bpsm = std::min(occ, 1);

    // rounds, captured once as a graph and replayed (direct launches if the
    // capture of the cooperative launch is refused)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (opts->use_graph && any) {
      bool ok = cudaStreamBeginCapture(c0->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        set_capturing(true);
        try {
          launch_persistent(bpsm, c0->cap_stream);
          enqueue_refresh(c0->cap_stream);
        } catch (...) {
          ok = false;
        }
        set_capturing(false);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(c0->cap_stream, &g);
        if (ok && ec == cudaSuccess && g && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess) {
          graph = g;
        } else {
          if (g) cudaGraphDestroy(g);
          exec = nullptr;
        }
      }
      cudaGetLastError();  // a refused capture leaves no sticky error
    }
    size_t nodes = 0;
    if (graph) SFEM_CUDA(cudaGraphGetNodes(graph, nullptr, &nodes));
    while (any && rounds < max_rounds) {
      if (exec) {
        SFEM_CUDA(cudaGraphLaunch(exec, st));
        count_launches((int64_t)nodes);
      } else {
        launch_persistent(bpsm, st);
        enqueue_refresh(st);
      }
      check();
      ++rounds;
    }
    const bool used_graph = exec != nullptr;
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;

    // results
    std::vector<SysState> hst(2 * n_sys);
    int slot = 0;
    SFEM_CUDA(cudaMemcpyAsync(&slot, a.slot, sizeof(int), cudaMemcpyDeviceToHost, st));
    SFEM_CUDA(cudaMemcpyAsync(hst.data(), a.state, 2 * n_sys * sizeof(SysState), cudaMemcpyDeviceToHost, st));
    SFEM_CUDA(cudaStreamSynchronize(st));
    // systems that stagnated on the FP32 operator: finish them with FP64
    // PCG (matrix-free FP64 operator), warm-started from the batch, with the
    // two-level preconditioner when a coarse space can be built for the
    // beam (default 8-node patches; about a tenth of Jacobi's iterations),
    // else Jacobi
    std::vector<sfem_solve_info> fb(n_sys);
    int n_fallback = 0;
    long long launch_iters = 0;
    SFEM_CUDA(cudaMemcpyAsync(&launch_iters, a.launch_iters, sizeof launch_iters, cudaMemcpyDeviceToHost, st));
    cudaEvent_t f0, f1;
    SFEM_CUDA(cudaEventCreate(&f0));
    SFEM_CUDA(cudaEventCreate(&f1));
    SFEM_CUDA(cudaEventRecord(f0, st));
    for (int b = 0, k2 = 0; b < n; ++b) {
      Ctx &c = ctxs[b]->c;
      for (int j = 0; j < c.nrhs; ++j, ++k2) {
        SysState &ss = hst[slot * n_sys + k2];
        if (ss.status != 4) continue;
        sfem_solve_opts so{};
        so.kind = SFEM_SOLVE_PCG64;
        so.op64 = SFEM_OP_MF64;
        so.precond = (opts->patch_nodes < 0 ? c.coarse != nullptr : ensure_coarse(c)) ? 1 : 0;
        so.rhs = j;
        so.u_on_device = 1;
        so.warm_start = 1;
        so.tol = tol;
        so.max_iter = std::max(1, max_iter - ss.iter);
        fb[k2] = sfem_solve_info{};
        const int rc = sfem_solve(ctxs[b], nullptr, xbeam[b] + j * c.ndof, &so, &fb[k2]);
        ss.iter += fb[k2].iterations;
        ss.relres = fb[k2].true_relres;
        ss.status = rc == SFEM_OK ? 1 : rc == SFEM_EBREAKDOWN ? 3 : 2;
        ++n_fallback;
      }
    }
    SFEM_CUDA(cudaEventRecord(f1, st));
    for (int b = 0; b < n; ++b) {
      Ctx &c = ctxs[b]->c;
      SFEM_CUDA(cudaMemcpyAsync(u[b], xbeam[b], c.ndof * c.nrhs * sizeof(double),
                                opts->u_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    }
    SFEM_CUDA(cudaEventRecord(e1, st));
    SFEM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f, fb_ms = 0.f;
    SFEM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    SFEM_CUDA(cudaEventElapsedTime(&fb_ms, f0, f1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(f0);
    cudaEventDestroy(f1);
    int worst = SFEM_OK;
    long long total_it = 0;
    for (int i = 0; i < n_sys; ++i) total_it += hst[slot * n_sys + i].iter;
    if (stats) {
      stats->fallback_systems = n_fallback;
      stats->rounds = rounds;
      stats->ctas_per_sm = bpsm;
      stats->graph = used_graph ? 1 : 0;
      stats->n_systems = n_sys;
      stats->total_iterations = total_it;
      stats->ms = ms;
      stats->launch_iterations = (int)std::min<long long>(launch_iters, INT32_MAX);
      stats->fallback_ms = fb_ms;
    }
    for (int i = 0; i < n_sys; ++i) {
      const SysState &ss = hst[slot * n_sys + i];
      int stt = ss.status == 1 ? SFEM_OK : ss.status == 3 ? SFEM_EBREAKDOWN : SFEM_ENOCONV;
      if (stt != SFEM_OK && worst == SFEM_OK) worst = stt;
      if (infos) {
        infos[i] = sfem_solve_info{};
        infos[i].status = stt;
        infos[i].iterations = ss.iter;
        infos[i].outer_iterations = rounds;
        infos[i].true_relres = ss.relres;
        infos[i].bnorm = hs[i].bnorm;
        infos[i].solve_ms = ms;
        infos[i].fallbacks = fb[i].iterations > 0 ? 1 : 0;
      }
    }
    cleanup();
    if (worst != SFEM_OK) set_last_error("some systems of the batch did not converge");
    return worst;
  } catch (const Error &err) {
    set_last_error(err.msg);
    cleanup();
    return err.status;
  }
}

extern "C" int sfem_selftest_barrier(sfem_ctx *h, int *status, double *wait_ms) {
  try {
    SFEM_REQUIRE(h && h->c.vol && status, SFEM_EINVAL, "context not set up or status NULL");
    Ctx &c = h->c;
    unsigned int *bar = c.mem.get<unsigned int>(2);
    int *words = c.mem.get<int>(2);  // error word, barrier result
    const unsigned int init[2] = {1u, 0u};  // arrival count offset by one, generation 0
    SFEM_CUDA(cudaMemcpyAsync(bar, init, sizeof init, cudaMemcpyHostToDevice, c.stream));
    SFEM_CUDA(cudaMemsetAsync(words, 0, 2 * sizeof(int), c.stream));
    BatchDev a{};
    a.bar_count = bar;
    a.bar_gen = bar + 1;
    a.err = words;
    cudaEvent_t e0, e1;
    SFEM_CUDA(cudaEventCreate(&e0));
    SFEM_CUDA(cudaEventCreate(&e1));
    SFEM_CUDA(cudaEventRecord(e0, c.stream));
    k_barrier_selftest<<<1, kTileThreads, 0, c.stream>>>(a, words + 1);
    SFEM_CHECK_LAUNCH();
    SFEM_CUDA(cudaEventRecord(e1, c.stream));
    int h_words[2] = {0, 0};
    SFEM_CUDA(cudaMemcpyAsync(h_words, words, sizeof h_words, cudaMemcpyDeviceToHost, c.stream));
    SFEM_CUDA(cudaStreamSynchronize(c.stream));
    float ms = 0.f;
    SFEM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c.mem.drop(words);
    c.mem.drop(bar);
    // the barrier must have given up: error word set, result false
    *status = (h_words[0] == 1 && h_words[1] == 0) ? SFEM_ETIMEOUT : SFEM_OK;
    if (wait_ms) *wait_ms = ms;
  } catch (const Error &err) {
    set_last_error(err.msg);
    return err.status;
  }
  return SFEM_OK;
}
