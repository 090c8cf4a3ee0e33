// Operators of the FS-FEM-T4 library: y = K u for the smoothed stiffness of
// Eq. 9, matrix-free (FP64 and FP32) and from the assembled CSR (FP64).
//
// Matrix-free form.  With the strain constant in each tet and each
// smoothing domain made of quarter-volume sub-tets (Fig. 1), the smoothed
// strain of face k between tets i and j is
//     eps_k = (V_i eps_i + V_j eps_j) / (V_i + V_j)     (Eq. 2-3),
// and V_k Bbar_k = sum_{e in k} (V_e/4) B_e on the stencil of face k, so
//     K u = sum_e B_e^T s_e,   s_e = (V_e/4) c sum_{faces k of e} eps_k.
// Pass 1 stores w_e = V_e eps_e per tet; pass 2 forms
//     t_e = c sum_a kap_ea (w_e + w_nbr(a)),  kap_ea = 1/(4 (V_e + V_nbr))
// (exterior faces: kap = 1/(4 V_e), no neighbour term), scatters
// (V_e B_e)^T t_e to the four nodes with atomics, and accumulates the
// energy u^T K u = sum_e w_e . t_e in FP64 for the CG step length.

#include <cuda_runtime.h>

#include "reduce.cuh"
#include "sfem_internal.cuh"

namespace sfem {

constexpr int kMfBlock = 256;
constexpr int kSpmvBlock = 256;

int reduction_blocks() {
  static int nb = 0;
  if (nb == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    nb = (sms > 0 ? sms : 152) * 4;
  }
  return nb;
}

// ---- vector helpers -------------------------------------------------------
template <class T>
struct Vec;
template <>
struct Vec<float> {
  static __device__ __forceinline__ void load4(const float *p, float (&v)[4]) {
    float4 a = *reinterpret_cast<const float4 *>(p);
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
  }
  static __device__ __forceinline__ void store8(float *p, const float (&v)[6]) {
    reinterpret_cast<float4 *>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float2 *>(p)[2] = make_float2(v[4], v[5]);
  }
  static __device__ __forceinline__ void load8(const float *p, float (&v)[6]) {
    float4 a = reinterpret_cast<const float4 *>(p)[0];
    float2 b = reinterpret_cast<const float2 *>(p)[2];
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y;
  }
};
template <>
struct Vec<double> {
  static __device__ __forceinline__ void load4(const double *p, double (&v)[4]) {
    double2 a = reinterpret_cast<const double2 *>(p)[0];
    double2 b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
  }
  static __device__ __forceinline__ void store8(double *p, const double (&v)[6]) {
    double2 *q = reinterpret_cast<double2 *>(p);
    q[0] = make_double2(v[0], v[1]);
    q[1] = make_double2(v[2], v[3]);
    q[2] = make_double2(v[4], v[5]);
  }
  static __device__ __forceinline__ void load8(const double *p, double (&v)[6]) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 a = q[0], b = q[1], d = q[2];
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y, v[4] = d.x, v[5] = d.y;
  }
};

template <class T>
__device__ __forceinline__ void load_grads(const T *__restrict__ Gs, int64_t n, int64_t e, T (&g)[4][3]) {
#pragma unroll
  for (int k = 0; k < 9; ++k) g[1 + k / 3][k % 3] = Gs[k * n + e];
#pragma unroll
  for (int i = 0; i < 3; ++i) g[0][i] = -(g[1][i] + g[2][i] + g[3][i]);
}

// ---- pass 1: w_e = V_e eps_e (Voigt, engineering shear; Eq. 4) -----------
template <class T, class TU>
__global__ void __launch_bounds__(kMfBlock) k_mf_strain(int64_t n, const int4 *__restrict__ conn,
                                                        const T *__restrict__ Gs, const TU *__restrict__ u,
                                                        int64_t ndof, int nrhs, T *__restrict__ w,
                                                        const int *done) {
  if (done && *done) return;
  int64_t e = (int64_t)blockIdx.x * kMfBlock + threadIdx.x;
  if (e >= n) return;
  int4 t = conn[e];
  const int v[4] = {t.x, t.y, t.z, t.w};
  T g[4][3];
  load_grads(Gs, n, e, g);
  for (int r = 0; r < nrhs; ++r) {
    const TU *ur = u + (int64_t)r * ndof;
    T H[3][3] = {};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const TU *ua = ur + 3 * (int64_t)v[a];
      T u0 = (T)__ldg(ua), u1 = (T)__ldg(ua + 1), u2 = (T)__ldg(ua + 2);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        H[0][j] += u0 * g[a][j];
        H[1][j] += u1 * g[a][j];
        H[2][j] += u2 * g[a][j];
      }
    }
    T s[6] = {H[0][0], H[1][1], H[2][2], H[1][2] + H[2][1], H[2][0] + H[0][2], H[0][1] + H[1][0]};
    Vec<T>::store8(w + ((int64_t)r * n + e) * 8, s);
  }
}

// ---- pass 2: face averages, stress, scatter (and energy) ------------------
template <class T, class TY>
__global__ void __launch_bounds__(kMfBlock)
    k_mf_stress(int64_t n, const int4 *__restrict__ conn, const T *__restrict__ Gs, const int4 *__restrict__ nbr,
                const T *__restrict__ kap, const T *__restrict__ w, int64_t ndof, int nrhs, T lam, T mu,
                TY *__restrict__ y, double *partials, unsigned int *ticket, double *energy_out,
                const int *done) {
  if (done && *done) return;
  int64_t e = (int64_t)blockIdx.x * kMfBlock + threadIdx.x;
  double en = 0.0;
  if (e < n) {
    int4 t = conn[e];
    int4 nb4 = nbr[e];
    const int v[4] = {t.x, t.y, t.z, t.w};
    const int nb[4] = {nb4.x, nb4.y, nb4.z, nb4.w};
    T k[4];
    Vec<T>::load4(kap + 4 * e, k);
    T g[4][3];
    load_grads(Gs, n, e, g);
    const T ksum = k[0] + k[1] + k[2] + k[3];
    for (int r = 0; r < nrhs; ++r) {
      const T *wr = w + (int64_t)r * n * 8;
      T W[6], S[6];
      Vec<T>::load8(wr + e * 8, W);
#pragma unroll
      for (int i = 0; i < 6; ++i) S[i] = ksum * W[i];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        if (nb[a] >= 0) {
          T Wn[6];
          Vec<T>::load8(wr + (int64_t)nb[a] * 8, Wn);
#pragma unroll
          for (int i = 0; i < 6; ++i) S[i] += k[a] * Wn[i];
        }
      }
      const T tr = S[0] + S[1] + S[2];
      T st[6] = {lam * tr + 2 * mu * S[0], lam * tr + 2 * mu * S[1], lam * tr + 2 * mu * S[2],
                 mu * S[3], mu * S[4], mu * S[5]};
      T el = 0;
#pragma unroll
      for (int i = 0; i < 6; ++i) el += W[i] * st[i];
      en += (double)el;
      TY *yr = y + (int64_t)r * ndof;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        T fx = g[a][0] * st[0] + g[a][1] * st[5] + g[a][2] * st[4];
        T fy = g[a][0] * st[5] + g[a][1] * st[1] + g[a][2] * st[3];
        T fz = g[a][0] * st[4] + g[a][1] * st[3] + g[a][2] * st[2];
        TY *ya = yr + 3 * (int64_t)v[a];
        atomicAdd(ya, (TY)fx);
        atomicAdd(ya + 1, (TY)fy);
        atomicAdd(ya + 2, (TY)fz);
      }
    }
  }
  if (energy_out) {
    double vv[1] = {en};
    grid_sum<kMfBlock, 1>(vv, partials, ticket, energy_out);
  }
}

void ensure_w_scratch(Ctx &c, size_t bytes) {
  if (c.w_bytes >= bytes) return;
  if (c.w_scratch) c.mem.drop(c.w_scratch);
  c.w_scratch = c.mem.raw(bytes);
  c.w_bytes = bytes;
}

template <class T, class TU>
void launch_mf_strain(Ctx &c, cudaStream_t st, const T *Gs, const TU *u, int nrhs, T *w, const int *done) {
  k_mf_strain<T, TU><<<grid_for(c.n_tets, kMfBlock), kMfBlock, 0, st>>>(
      c.n_tets, reinterpret_cast<const int4 *>(c.tets), Gs, u, c.ndof, nrhs, w, done);
  SFEM_CHECK_LAUNCH();
}

template <class T, class TY>
void launch_mf_stress(Ctx &c, cudaStream_t st, const T *Gs, const T *kap, const T *w, TY *y, int nrhs,
                      double *energy_out, const int *done) {
  k_mf_stress<T, TY><<<grid_for(c.n_tets, kMfBlock), kMfBlock, 0, st>>>(
      c.n_tets, reinterpret_cast<const int4 *>(c.tets), Gs, reinterpret_cast<const int4 *>(c.nbr), kap, w, c.ndof,
      nrhs, (T)c.lam, (T)c.mu, y, c.red_partial, c.tickets, energy_out, done);
  SFEM_CHECK_LAUNCH();
}

template void launch_mf_strain<float, float>(Ctx &, cudaStream_t, const float *, const float *, int, float *,
                                             const int *);
template void launch_mf_strain<float, double>(Ctx &, cudaStream_t, const float *, const double *, int, float *,
                                              const int *);
template void launch_mf_strain<double, double>(Ctx &, cudaStream_t, const double *, const double *, int, double *,
                                               const int *);
template void launch_mf_stress<float, float>(Ctx &, cudaStream_t, const float *, const float *, const float *,
                                             float *, int, double *, const int *);
template void launch_mf_stress<float, double>(Ctx &, cudaStream_t, const float *, const float *, const float *,
                                              double *, int, double *, const int *);
template void launch_mf_stress<double, double>(Ctx &, cudaStream_t, const double *, const double *,
                                               const double *, double *, int, double *, const int *);

template <class T>
static void apply_mf(Ctx &c, const T *Gs, const T *kap, const T *u, T *y, int nrhs, double *energy_out) {
  ensure_w_scratch(c, (size_t)c.n_tets * 8 * sizeof(T) * nrhs);
  T *w = static_cast<T *>(c.w_scratch);
  SFEM_CUDA(cudaMemsetAsync(y, 0, (size_t)nrhs * c.ndof * sizeof(T), c.stream));
  launch_mf_strain<T, T>(c, c.stream, Gs, u, nrhs, w, nullptr);
  launch_mf_stress<T, T>(c, c.stream, Gs, kap, w, y, nrhs, energy_out, nullptr);
}

void apply_mf64(Ctx &c, const double *u, double *y, int nrhs, double *energy_out) {
  apply_mf<double>(c, c.Gs64, c.kap64, u, y, nrhs, energy_out);
}
void apply_mf32(Ctx &c, const float *u, float *y, int nrhs, double *energy_out) {
  SFEM_CUDA(cudaMemsetAsync(y, 0, (size_t)nrhs * c.ndof * sizeof(float), c.stream));
  if (energy_out) SFEM_CUDA(cudaMemsetAsync(energy_out, 0, sizeof(double), c.stream));
  for (int r = 0; r < nrhs; ++r)
    launch_mf32_tiled<float, float>(c, c.stream, u + (int64_t)r * c.ndof, y + (int64_t)r * c.ndof,
                                    r == 0 ? energy_out : nullptr, nullptr);
}

// ---- CSR SpMV (FP64), kCsrLanes lanes per row, fixed grid -----------------
// A full-warp reduction per row would spend 5 x 32 FP64 lane-adds per row,
// more than the row's own FMAs on a GPU with a low FP64 rate; a group of 4
// lanes per row needs 2 shuffle steps and still reads 32-byte segments.
constexpr int kCsrLanes = 4;

__global__ void __launch_bounds__(kSpmvBlock)
    k_csr_spmv(int64_t nrows, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
               const double *__restrict__ val, const double *__restrict__ x, double *__restrict__ y,
               const double *__restrict__ dotv, double *partials, unsigned int *ticket, double *dot_out,
               const int *done) {
  if (done && *done) return;
  const int sub = threadIdx.x & (kCsrLanes - 1);
  const int64_t group = ((int64_t)blockIdx.x * kSpmvBlock + threadIdx.x) / kCsrLanes;
  const int64_t ngroups = ((int64_t)gridDim.x * kSpmvBlock) / kCsrLanes;
  // rows advance by a warp-uniform base so every lane runs the same trip
  // count (the shuffles below need the whole warp)
  const int64_t g0 = group - (int64_t)((threadIdx.x & 31) / kCsrLanes);
  double dot = 0.0;
  for (int64_t base = g0; base < nrows; base += ngroups) {
    const int64_t row = base + (group - g0);
    double s = 0.0;
    if (row < nrows) {
      const int64_t b = rp[row], e = rp[row + 1];
      for (int64_t j = b + sub; j < e; j += kCsrLanes) s += val[j] * __ldg(&x[col[j]]);
    }
#pragma unroll
    for (int o = kCsrLanes / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (sub == 0 && row < nrows) {
      y[row] = s;
      if (dotv) dot += s * dotv[row];
    }
  }
  if (dot_out) {
    double vv[1] = {dot};
    grid_sum<kSpmvBlock, 1>(vv, partials, ticket, dot_out);
  }
}

void launch_csr64(Ctx &c, cudaStream_t st, const double *u, double *y, const double *dotv, double *dot_out,
                  const int *done) {
  k_csr_spmv<<<c.red_blocks, kSpmvBlock, 0, st>>>(c.ndof, c.csr.row_ptr, c.csr.col, c.csr.val, u, y, dotv,
                                                  c.red_partial, c.tickets + 1, dot_out, done);
  SFEM_CHECK_LAUNCH();
}

void apply_csr64(Ctx &c, const double *u, double *y, int nrhs, const double *dotv, double *dot_out) {
  SFEM_REQUIRE(c.assembled, SFEM_EINVAL, "the CSR operator needs sfem_assemble first");
  for (int r = 0; r < nrhs; ++r)
    launch_csr64(c, c.stream, u + (int64_t)r * c.ndof, y + (int64_t)r * c.ndof, dotv, r == 0 ? dot_out : nullptr,
                 nullptr);
}

// ---- masking for the ABI apply: A u = P K P u + (I - P) u -----------------
template <class T>
__global__ void k_mask_copy(const T *__restrict__ u, T *__restrict__ out, const uint8_t *__restrict__ dmask,
                            int64_t ndof, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = dmask[i % ndof] ? u[i] : T(0);
}
template <class T>
__global__ void k_fix_rows(T *__restrict__ y, const T *__restrict__ u, const uint8_t *__restrict__ dmask,
                           int64_t ndof, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !dmask[i % ndof]) y[i] = u[i];
}

__global__ void k_norm2(const double *__restrict__ x, int64_t n, double *partials, unsigned int *ticket,
                        double *out) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) s += x[i] * x[i];
  double vv[1] = {s};
  grid_sum<256, 1>(vv, partials, ticket, out);
}

double device_norm2(Ctx &c, const double *x, int64_t n) {
  double *out = c.mem.get<double>(1);
  k_norm2<<<c.red_blocks, 256, 0, c.stream>>>(x, n, c.red_partial, c.tickets + 2, out);
  SFEM_CHECK_LAUNCH();
  double h = 0.0;
  SFEM_CUDA(cudaMemcpyAsync(&h, out, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  SFEM_CUDA(cudaStreamSynchronize(c.stream));
  c.mem.drop(out);
  return h;
}

}  // namespace sfem

using namespace sfem;

extern "C" int sfem_apply(sfem_ctx *h, const void *u, void *y, int op, int nrhs) {
  try {
    SFEM_REQUIRE(h && h->c.vol, SFEM_EINVAL, "context not set up");
    SFEM_REQUIRE(u && y, SFEM_EINVAL, "u and y must be device pointers");
    SFEM_REQUIRE(nrhs >= 1, SFEM_EINVAL, "nrhs must be >= 1");
    Ctx &c = h->c;
    const int64_t n = (int64_t)nrhs * c.ndof;
    const int grid = grid_for(n, 256);
    if (op == SFEM_OP_MF32) {
      float *tmp = c.mem.get<float>(n);
      k_mask_copy<float><<<grid, 256, 0, c.stream>>>((const float *)u, tmp, c.dmask, c.ndof, n);
      SFEM_CHECK_LAUNCH();
      apply_mf32(c, tmp, (float *)y, nrhs, nullptr);
      k_fix_rows<float><<<grid, 256, 0, c.stream>>>((float *)y, (const float *)u, c.dmask, c.ndof, n);
      SFEM_CHECK_LAUNCH();
      c.mem.drop(tmp);
      check_tile_error(c);
    } else if (op == SFEM_OP_MF32_F64) {
      // FP32 arithmetic on FP64 vectors (the operator of the mixed-precision solve)
      double *tmp = c.mem.get<double>(n);
      k_mask_copy<double><<<grid, 256, 0, c.stream>>>((const double *)u, tmp, c.dmask, c.ndof, n);
      SFEM_CHECK_LAUNCH();
      SFEM_CUDA(cudaMemsetAsync(y, 0, n * sizeof(double), c.stream));
      for (int k = 0; k < nrhs; ++k)
        launch_mf32_tiled<double, double>(c, c.stream, tmp + k * c.ndof, (double *)y + k * c.ndof, nullptr, nullptr);
      k_fix_rows<double><<<grid, 256, 0, c.stream>>>((double *)y, (const double *)u, c.dmask, c.ndof, n);
      SFEM_CHECK_LAUNCH();
      c.mem.drop(tmp);
      check_tile_error(c);
    } else if (op == SFEM_OP_MF64 || op == SFEM_OP_CSR64 || op == SFEM_OP_NS64 || op == SFEM_OP_ES64) {
      double *tmp = c.mem.get<double>(n);
      k_mask_copy<double><<<grid, 256, 0, c.stream>>>((const double *)u, tmp, c.dmask, c.ndof, n);
      SFEM_CHECK_LAUNCH();
      if (op == SFEM_OP_MF64)
        apply_mf64(c, tmp, (double *)y, nrhs, nullptr);
      else if (op == SFEM_OP_NS64)
        for (int k = 0; k < nrhs; ++k) apply_ns64(c, tmp + k * c.ndof, (double *)y + k * c.ndof);
      else if (op == SFEM_OP_ES64)
        for (int k = 0; k < nrhs; ++k) apply_es64(c, tmp + k * c.ndof, (double *)y + k * c.ndof);
      else
        apply_csr64(c, tmp, (double *)y, nrhs, nullptr, nullptr);
      k_fix_rows<double><<<grid, 256, 0, c.stream>>>((double *)y, (const double *)u, c.dmask, c.ndof, n);
      SFEM_CHECK_LAUNCH();
      c.mem.drop(tmp);
    } else {
      throw Error{SFEM_EINVAL, "unknown operator"};
    }
  } catch (const Error &err) {
    set_last_error(err.msg);
    return err.status;
  }
  return SFEM_OK;
}

// deterministic input for operator timing: values in [-1, 1) from a
// multiplicative hash of the index (a zero input would let the nodal force
// atomics add zeros and time an unrepresentative case)
template <class T>
__global__ void k_timing_input(T *u, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) u[i] = (T)((double)(((uint64_t)i * 2654435761ull) % 20011ull) / 10005.5 - 1.0);
}

extern "C" int sfem_time_operator(sfem_ctx *h, int op, int reps, double *ms_per_apply) {
  try {
    SFEM_REQUIRE(h && h->c.vol && ms_per_apply && reps >= 1, SFEM_EINVAL, "bad arguments");
    Ctx &c = h->c;
    const int64_t n = c.ndof;
    const size_t es = op == SFEM_OP_MF32 ? sizeof(float) : sizeof(double);
    void *u = c.mem.raw(n * es);
    void *y = c.mem.raw(n * es);
    if (op == SFEM_OP_MF32)
      k_timing_input<float><<<grid_for(n, 256), 256, 0, c.stream>>>((float *)u, n);
    else
      k_timing_input<double><<<grid_for(n, 256), 256, 0, c.stream>>>((double *)u, n);
    SFEM_CHECK_LAUNCH();
    SFEM_CUDA(cudaMemsetAsync(y, 0, n * es, c.stream));
    ensure_w_scratch(c, (size_t)c.n_tets * 8 * sizeof(double));
    cudaEvent_t e0, e1;
    SFEM_CUDA(cudaEventCreate(&e0));
    SFEM_CUDA(cudaEventCreate(&e1));
    // the CG launches the tiled operator with its energy sum (p.q) and the
    // stop flag; so does the timing
    double *energy = c.mem.get<double>(1);
    int *done = c.mem.get<int>(1);
    SFEM_CUDA(cudaMemsetAsync(done, 0, sizeof(int), c.stream));
    SFEM_CUDA(cudaMemsetAsync(energy, 0, sizeof(double), c.stream));
    auto once = [&]() {
      if (op == SFEM_OP_MF32) {
        launch_mf32_tiled<float, float>(c, c.stream, (const float *)u, (float *)y, energy, done);
      } else if (op == SFEM_OP_MF32_F64) {
        launch_mf32_tiled<double, double>(c, c.stream, (const double *)u, (double *)y, energy, done);
      } else if (op == SFEM_OP_MF64) {
        launch_mf_strain<double, double>(c, c.stream, c.Gs64, (const double *)u, 1, (double *)c.w_scratch,
                                         nullptr);
        launch_mf_stress<double, double>(c, c.stream, c.Gs64, c.kap64, (const double *)c.w_scratch, (double *)y, 1,
                                         nullptr, nullptr);
      } else if (op == SFEM_OP_CSR64) {
        SFEM_REQUIRE(c.assembled, SFEM_EINVAL, "CSR64 needs sfem_assemble first");
        launch_csr64(c, c.stream, (const double *)u, (double *)y, nullptr, nullptr, nullptr);
      } else if (op == SFEM_OP_NS64) {
        launch_ns64(c, c.stream, (const double *)u, (double *)y, nullptr, nullptr);
      } else if (op == SFEM_OP_ES64) {
        prepare_es64(c);
        launch_es64(c, c.stream, (const double *)u, (double *)y, nullptr, nullptr);
      } else {
        throw Error{SFEM_EINVAL, "unknown operator"};
      }
    };
    once();  // warm-up
    SFEM_CUDA(cudaEventRecord(e0, c.stream));
    for (int i = 0; i < reps; ++i) once();
    SFEM_CUDA(cudaEventRecord(e1, c.stream));
    SFEM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    SFEM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    *ms_per_apply = (double)ms / reps;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    check_tile_error(c);
    c.mem.drop(u);
    c.mem.drop(y);
    c.mem.drop(energy);
    c.mem.drop(done);
  } catch (const Error &err) {
    set_last_error(err.msg);
    return err.status;
  }
  return SFEM_OK;
}
