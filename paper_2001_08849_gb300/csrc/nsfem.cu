// NS-FEM-T4: the node-based smoothed FEM, one of the other S-FEM models the
// paper lists beside FS-FEM (Sec. 2.1).  The smoothing domain of node n is
// the union of a quarter of every tet that contains it, V_n = sum_e V_e / 4,
// and its smoothed strain is the volume average of those tets' strains,
// eps_n = sum_{e ni n} (V_e / 4) eps_e / V_n (the node-domain counterpart of
// Eq. 2-7).  K = sum_n V_n Bbar_n^T D Bbar_n; applied matrix-free in FP64:
//   1. per tet  w_e = (V_e / 4) B_e u_e            (scratch, 6 per tet)
//   2. per node eps_n = sum w_e / V_n over the node's tets (the node -> tet
//               lists of the setup, ascending: a fixed summation order),
//               sigma_n = D eps_n, and the energy V_n eps_n . sigma_n
//   3. per tet  t_e = (V_e / 4) sum_{n in e} sigma_n, f_I += B_I^T t_e for
//               its four nodes (FP64 atomics)
// since f_I = sum_n V_n Bbar_{n,I}^T sigma_n = sum_e sum_{n in e} (V_e/4) B_I^T sigma_n.
// The geometry (V_e, grad N) is the FS-FEM setup's; only the domain table
// differs (node -> tets instead of faces).

#include <cuda_runtime.h>

#include "reduce.cuh"
#include "sfem_internal.cuh"

namespace sfem {

namespace {

constexpr int kNsBlock = 256;

__global__ void __launch_bounds__(kNsBlock) k_ns_strain(int64_t n_tets, const int4 *__restrict__ tets,
                                                        const double *__restrict__ vol,
                                                        const double *__restrict__ grad,
                                                        const double *__restrict__ u, double *__restrict__ w,
                                                        const int *done) {
  if (done && *done) return;
  const int64_t e = (int64_t)blockIdx.x * kNsBlock + threadIdx.x;
  if (e >= n_tets) return;
  const int4 t = tets[e];
  const int nd[4] = {t.x, t.y, t.z, t.w};
  double H[3][3] = {};
  for (int a = 0; a < 4; ++a) {
    const double *ua = u + 3 * (int64_t)nd[a];
    const double *g = grad + 12 * e + 3 * a;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) H[i][j] = fma(ua[i], g[j], H[i][j]);
  }
  const double q = 0.25 * vol[e];
  double *we = w + 6 * e;
  we[0] = q * H[0][0];
  we[1] = q * H[1][1];
  we[2] = q * H[2][2];
  we[3] = q * (H[1][2] + H[2][1]);
  we[4] = q * (H[2][0] + H[0][2]);
  we[5] = q * (H[0][1] + H[1][0]);
}

__global__ void __launch_bounds__(kNsBlock) k_ns_node(int64_t n_nodes, const int64_t *__restrict__ ptr,
                                                      const int32_t *__restrict__ n2t,
                                                      const double *__restrict__ vol, const double *__restrict__ w,
                                                      double lam, double mu, double *__restrict__ sig,
                                                      double *energy, const int *done) {
  if (done && *done) return;
  const int64_t n = (int64_t)blockIdx.x * kNsBlock + threadIdx.x;
  double en = 0.0;
  if (n < n_nodes) {
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, Vn = 0.0;
    for (int64_t k = ptr[n]; k < ptr[n + 1]; ++k) {
      const int64_t e = n2t[k];
      Vn += 0.25 * vol[e];
      for (int j = 0; j < 6; ++j) acc[j] += w[6 * e + j];
    }
    const double inv = Vn > 0.0 ? 1.0 / Vn : 0.0;
    double ep[6];
    for (int j = 0; j < 6; ++j) ep[j] = acc[j] * inv;
    const double tr = ep[0] + ep[1] + ep[2];
    const double s[6] = {lam * tr + 2.0 * mu * ep[0], lam * tr + 2.0 * mu * ep[1], lam * tr + 2.0 * mu * ep[2],
                         mu * ep[3],                  mu * ep[4],                  mu * ep[5]};
    for (int j = 0; j < 6; ++j) {
      sig[6 * n + j] = s[j];
      en = fma(ep[j], s[j], en);
    }
    en *= Vn;
  }
  if (energy) {  // u^T K u = sum_n V_n eps_n . sigma_n, one FP64 atomic per block
    en = block_sum<kNsBlock>(en);
    if (threadIdx.x == 0) atomicAdd(energy, en);
  }
}

__global__ void __launch_bounds__(kNsBlock) k_ns_force(int64_t n_tets, const int4 *__restrict__ tets,
                                                       const double *__restrict__ vol,
                                                       const double *__restrict__ grad,
                                                       const double *__restrict__ sig, double *__restrict__ y,
                                                       const int *done) {
  if (done && *done) return;
  const int64_t e = (int64_t)blockIdx.x * kNsBlock + threadIdx.x;
  if (e >= n_tets) return;
  const int4 t = tets[e];
  const int nd[4] = {t.x, t.y, t.z, t.w};
  double s[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int a = 0; a < 4; ++a)
    for (int j = 0; j < 6; ++j) s[j] += sig[6 * (int64_t)nd[a] + j];
  const double q = 0.25 * vol[e];
  for (int j = 0; j < 6; ++j) s[j] *= q;
  for (int a = 0; a < 4; ++a) {
    const double *g = grad + 12 * e + 3 * a;
    double *ya = y + 3 * (int64_t)nd[a];
    atomicAdd(ya, g[0] * s[0] + g[1] * s[5] + g[2] * s[4]);
    atomicAdd(ya + 1, g[0] * s[5] + g[1] * s[1] + g[2] * s[3]);
    atomicAdd(ya + 2, g[0] * s[4] + g[1] * s[3] + g[2] * s[2]);
  }
}

}  // namespace

// y += K_NS u for one vector (y accumulated: zero it first); energy (may be
// null) += u^T K_NS u
void launch_ns64(Ctx &c, cudaStream_t st, const double *u, double *y, double *energy, const int *done) {
  ensure_w_scratch(c, (size_t)c.n_tets * 8 * sizeof(double));
  if (!c.ns_sig) c.ns_sig = c.mem.get<double>(6 * c.n_nodes);
  double *w = static_cast<double *>(c.w_scratch);
  const int4 *t4 = reinterpret_cast<const int4 *>(c.tets);
  k_ns_strain<<<grid_for(c.n_tets, kNsBlock), kNsBlock, 0, st>>>(c.n_tets, t4, c.vol, c.grad, u, w, done);
  SFEM_CHECK_LAUNCH();
  k_ns_node<<<grid_for(c.n_nodes, kNsBlock), kNsBlock, 0, st>>>(c.n_nodes, c.n2t_ptr, c.n2t, c.vol, w, c.lam, c.mu,
                                                               c.ns_sig, energy, done);
  SFEM_CHECK_LAUNCH();
  k_ns_force<<<grid_for(c.n_tets, kNsBlock), kNsBlock, 0, st>>>(c.n_tets, t4, c.vol, c.grad, c.ns_sig, y, done);
  SFEM_CHECK_LAUNCH();
}

void apply_ns64(Ctx &c, const double *u, double *y) {
  SFEM_CUDA(cudaMemsetAsync(y, 0, c.ndof * sizeof(double), c.stream));
  launch_ns64(c, c.stream, u, y, nullptr, nullptr);
}

}  // namespace sfem
