// ES-FEM-T4: the edge-based smoothed FEM, the third S-FEM model the paper
// lists beside FS-FEM and NS-FEM (Sec. 2.1).  The smoothing domain of an
// edge is a sixth of every tet that contains it (a tet has six edges),
// V_k = sum_e V_e / 6, and its smoothed strain is the volume average
// eps_k = sum_{e ni k} (V_e / 6) eps_e / V_k.  K = sum_k V_k Bbar_k^T D Bbar_k,
// applied matrix-free in FP64:
//   1. per tet  w_e = (V_e / 6) B_e u_e, added to the accumulators of its six
//               edges (FP64 atomics)
//   2. per edge sigma_k = D acc_k / V_k and the energy V_k eps_k . sigma_k
//   3. per tet  t_e = (V_e / 6) sum_{k in e} sigma_k, f_I += B_I^T t_e
// The edge table is built once on the GPU from the node -> tet lists of the
// setup: for every node a, the sorted distinct nodes b > a it shares a tet
// with (its edges), then every tet's six edge ids by binary search.

#include <cuda_runtime.h>

#include "reduce.cuh"
#include "sfem_internal.cuh"

namespace sfem {

namespace {

constexpr int kEsBlock = 256;
constexpr int kMaxNbr = 96;  // distinct higher neighbours of one node (3 per incident tet at most)

// the distinct nodes b > a of the tets around node a, ascending, into nb
// (returns their count; -1 if more than kMaxNbr)
__device__ int higher_neighbours(int64_t a, const int64_t *ptr, const int32_t *n2t, const int4 *tets, int *nb) {
  int cnt = 0;
  for (int64_t k = ptr[a]; k < ptr[a + 1]; ++k) {
    const int4 t = tets[n2t[k]];
    const int v[4] = {t.x, t.y, t.z, t.w};
    for (int i = 0; i < 4; ++i) {
      const int b = v[i];
      if (b <= a) continue;
      int j = cnt - 1;  // insertion into the sorted list, skipping duplicates
      while (j >= 0 && nb[j] > b) --j;
      if (j >= 0 && nb[j] == b) continue;
      if (cnt == kMaxNbr) return -1;
      for (int m = cnt; m > j + 1; --m) nb[m] = nb[m - 1];
      nb[j + 1] = b;
      ++cnt;
    }
  }
  return cnt;
}

__global__ void k_edge_count(int64_t n_nodes, const int64_t *__restrict__ ptr, const int32_t *__restrict__ n2t,
                             const int4 *__restrict__ tets, int64_t *__restrict__ cnt, int *overflow) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_nodes) return;
  int nb[kMaxNbr];
  const int c = higher_neighbours(a, ptr, n2t, tets, nb);
  if (c < 0) atomicExch(overflow, 1);
  cnt[a] = c < 0 ? 0 : c;
}

__global__ void k_edge_fill(int64_t n_nodes, const int64_t *__restrict__ ptr, const int32_t *__restrict__ n2t,
                            const int4 *__restrict__ tets, const int64_t *__restrict__ eoff,
                            int32_t *__restrict__ enb) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_nodes) return;
  int nb[kMaxNbr];
  const int c = higher_neighbours(a, ptr, n2t, tets, nb);
  for (int i = 0; i < c; ++i) enb[eoff[a] + i] = nb[i];
}

__global__ void k_tet_edges(int64_t n_tets, const int4 *__restrict__ tets, const double *__restrict__ vol,
                            const int64_t *__restrict__ eoff, const int32_t *__restrict__ enb,
                            int32_t *__restrict__ te, double *__restrict__ Vk) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_tets) return;
  const int4 t = tets[e];
  const int v[4] = {t.x, t.y, t.z, t.w};
  const int P[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  for (int k = 0; k < 6; ++k) {
    const int a = min(v[P[k][0]], v[P[k][1]]), b = max(v[P[k][0]], v[P[k][1]]);
    int64_t lo = eoff[a], hi = eoff[a + 1];
    while (lo < hi) {  // b is in a's list by construction
      const int64_t mid = (lo + hi) >> 1;
      if (enb[mid] < b)
        lo = mid + 1;
      else
        hi = mid;
    }
    te[6 * e + k] = (int32_t)lo;
    atomicAdd(Vk + lo, vol[e] / 6.0);
  }
}

__global__ void __launch_bounds__(kEsBlock) k_es_strain(int64_t n_tets, const int4 *__restrict__ tets,
                                                        const double *__restrict__ vol,
                                                        const double *__restrict__ grad,
                                                        const int32_t *__restrict__ te, const double *__restrict__ u,
                                                        double *__restrict__ acc, const int *done) {
  if (done && *done) return;
  const int64_t e = (int64_t)blockIdx.x * kEsBlock + threadIdx.x;
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
  const double q = vol[e] / 6.0;
  const double w[6] = {q * H[0][0], q * H[1][1], q * H[2][2], q * (H[1][2] + H[2][1]), q * (H[2][0] + H[0][2]),
                       q * (H[0][1] + H[1][0])};
  for (int k = 0; k < 6; ++k) {
    double *ak = acc + 6 * (int64_t)te[6 * e + k];
    for (int j = 0; j < 6; ++j) atomicAdd(ak + j, w[j]);
  }
}

__global__ void __launch_bounds__(kEsBlock) k_es_edge(int64_t n_edges, const double *__restrict__ Vk, double lam,
                                                      double mu, double *__restrict__ acc, double *energy,
                                                      const int *done) {
  if (done && *done) return;
  const int64_t k = (int64_t)blockIdx.x * kEsBlock + threadIdx.x;
  double en = 0.0;
  if (k < n_edges) {
    double *a = acc + 6 * k;
    const double inv = Vk[k] > 0.0 ? 1.0 / Vk[k] : 0.0;
    double ep[6];
    for (int j = 0; j < 6; ++j) ep[j] = a[j] * inv;
    const double tr = ep[0] + ep[1] + ep[2];
    const double s[6] = {lam * tr + 2.0 * mu * ep[0], lam * tr + 2.0 * mu * ep[1], lam * tr + 2.0 * mu * ep[2],
                         mu * ep[3],                  mu * ep[4],                  mu * ep[5]};
    for (int j = 0; j < 6; ++j) {
      a[j] = s[j];  // the accumulator now holds the edge's stress
      en = fma(ep[j], s[j], en);
    }
    en *= Vk[k];
  }
  if (energy) {
    en = block_sum<kEsBlock>(en);
    if (threadIdx.x == 0) atomicAdd(energy, en);
  }
}

__global__ void __launch_bounds__(kEsBlock) k_es_force(int64_t n_tets, const int4 *__restrict__ tets,
                                                       const double *__restrict__ vol,
                                                       const double *__restrict__ grad,
                                                       const int32_t *__restrict__ te,
                                                       const double *__restrict__ sig, double *__restrict__ y,
                                                       const int *done) {
  if (done && *done) return;
  const int64_t e = (int64_t)blockIdx.x * kEsBlock + threadIdx.x;
  if (e >= n_tets) return;
  double s[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int k = 0; k < 6; ++k) {
    const double *sk = sig + 6 * (int64_t)te[6 * e + k];
    for (int j = 0; j < 6; ++j) s[j] += sk[j];
  }
  const double q = vol[e] / 6.0;
  for (int j = 0; j < 6; ++j) s[j] *= q;
  const int4 t = tets[e];
  const int nd[4] = {t.x, t.y, t.z, t.w};
  for (int a = 0; a < 4; ++a) {
    const double *g = grad + 12 * e + 3 * a;
    double *ya = y + 3 * (int64_t)nd[a];
    atomicAdd(ya, g[0] * s[0] + g[1] * s[5] + g[2] * s[4]);
    atomicAdd(ya + 1, g[0] * s[5] + g[1] * s[1] + g[2] * s[3]);
    atomicAdd(ya + 2, g[0] * s[4] + g[1] * s[3] + g[2] * s[2]);
  }
}

void ensure_edges(Ctx &c) {
  if (c.es_te) return;
  const int4 *t4 = reinterpret_cast<const int4 *>(c.tets);
  int64_t *cnt = c.mem.get<int64_t>(c.n_nodes);
  int *ovf = c.mem.get<int>(1);
  SFEM_CUDA(cudaMemsetAsync(ovf, 0, sizeof(int), c.stream));
  k_edge_count<<<grid_for(c.n_nodes, 128), 128, 0, c.stream>>>(c.n_nodes, c.n2t_ptr, c.n2t, t4, cnt, ovf);
  SFEM_CHECK_LAUNCH();
  int h_ovf = 0;
  SFEM_CUDA(cudaMemcpyAsync(&h_ovf, ovf, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  SFEM_CUDA(cudaStreamSynchronize(c.stream));
  c.mem.drop(ovf);
  if (h_ovf) {
    c.mem.drop(cnt);
    throw Error{SFEM_EMESH, "a node has more than 96 higher-numbered edge neighbours"};
  }
  // exclusive scan of the counts on the host (one value per node, once per context)
  std::vector<int64_t> h(c.n_nodes), off(c.n_nodes + 1);
  SFEM_CUDA(cudaMemcpyAsync(h.data(), cnt, c.n_nodes * sizeof(int64_t), cudaMemcpyDeviceToHost, c.stream));
  SFEM_CUDA(cudaStreamSynchronize(c.stream));
  off[0] = 0;
  for (int64_t a = 0; a < c.n_nodes; ++a) off[a + 1] = off[a] + h[a];
  c.n_edges = off[c.n_nodes];
  SFEM_REQUIRE(c.n_edges < (int64_t(1) << 31), SFEM_EINVAL, "too many edges");
  int64_t *eoff = c.mem.get<int64_t>(c.n_nodes + 1);
  SFEM_CUDA(cudaMemcpyAsync(eoff, off.data(), (c.n_nodes + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c.stream));
  int32_t *enb = c.mem.get<int32_t>(std::max<int64_t>(c.n_edges, 1));
  k_edge_fill<<<grid_for(c.n_nodes, 128), 128, 0, c.stream>>>(c.n_nodes, c.n2t_ptr, c.n2t, t4, eoff, enb);
  SFEM_CHECK_LAUNCH();
  c.es_te = c.mem.get<int32_t>(6 * c.n_tets);
  c.es_Vk = c.mem.get<double>(std::max<int64_t>(c.n_edges, 1));
  c.es_acc = c.mem.get<double>(6 * std::max<int64_t>(c.n_edges, 1));
  SFEM_CUDA(cudaMemsetAsync(c.es_Vk, 0, c.n_edges * sizeof(double), c.stream));
  k_tet_edges<<<grid_for(c.n_tets, 128), 128, 0, c.stream>>>(c.n_tets, t4, c.vol, eoff, enb, c.es_te, c.es_Vk);
  SFEM_CHECK_LAUNCH();
  SFEM_CUDA(cudaStreamSynchronize(c.stream));
  c.mem.drop(enb);
  c.mem.drop(eoff);
  c.mem.drop(cnt);
}

}  // namespace

void prepare_es64(Ctx &c) { ensure_edges(c); }

void launch_es64(Ctx &c, cudaStream_t st, const double *u, double *y, double *energy, const int *done) {
  const int4 *t4 = reinterpret_cast<const int4 *>(c.tets);
  SFEM_CUDA(cudaMemsetAsync(c.es_acc, 0, 6 * c.n_edges * sizeof(double), st));
  k_es_strain<<<grid_for(c.n_tets, kEsBlock), kEsBlock, 0, st>>>(c.n_tets, t4, c.vol, c.grad, c.es_te, u, c.es_acc,
                                                                 done);
  SFEM_CHECK_LAUNCH();
  k_es_edge<<<grid_for(c.n_edges, kEsBlock), kEsBlock, 0, st>>>(c.n_edges, c.es_Vk, c.lam, c.mu, c.es_acc, energy,
                                                                done);
  SFEM_CHECK_LAUNCH();
  k_es_force<<<grid_for(c.n_tets, kEsBlock), kEsBlock, 0, st>>>(c.n_tets, t4, c.vol, c.grad, c.es_te, c.es_acc, y,
                                                                done);
  SFEM_CHECK_LAUNCH();
}

void apply_es64(Ctx &c, const double *u, double *y) {
  ensure_edges(c);
  SFEM_CUDA(cudaMemsetAsync(y, 0, c.ndof * sizeof(double), c.stream));
  launch_es64(c, c.stream, u, y, nullptr, nullptr);
}

}  // namespace sfem
