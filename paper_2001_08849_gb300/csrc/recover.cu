// Strain and stress recovery for output (the paper's post-processing,
// Sec. 3.4: strain and stress computed from the nodal displacements and
// written with the mesh for visualisation).
//
// Per face k, in the library's face order: the smoothed strain
// eps_k = sum_I B_I(b_I) u_I over the face's 4- or 5-node stencil (Eq. 5-7,
// b_I the smoothed gradients of the smoothing domain, formed by
// face_stencil from the tets' gradients), Voigt order (xx, yy, zz, yz, zx,
// xy) with engineering shear strains (Eq. 4), and the stress
// sigma_k = D eps_k of the isotropic material.  Per node: the V_k-weighted
// means of eps_k and sigma_k over the faces whose triangle contains the node
// (the smoothing domains whose closure holds it), and the von Mises
// equivalent of the mean stress.  FP64 throughout; the nodal sums use FP64
// atomics, so their rounding order is not fixed.

#include <cuda_runtime.h>

#include <cmath>

#include "face.cuh"
#include "sfem_internal.cuh"

namespace sfem {

namespace {

constexpr int kNodeAcc = 13;  // strain 6, stress 6, weight

__global__ void k_recover_faces(int64_t n_faces, const int32_t *__restrict__ tets,
                                const int32_t *__restrict__ face_tet, const int32_t *__restrict__ face_slot,
                                const double *__restrict__ vol, const double *__restrict__ grad,
                                const double *__restrict__ u, double lam, double mu, double *__restrict__ fstrain,
                                double *__restrict__ fstress, double *__restrict__ nacc) {
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_faces) return;
  FaceStencil s;
  face_stencil(f, tets, face_tet, face_slot, vol, grad, s);
  double e[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int i = 0; i < s.nn; ++i) {
    const double *ui = u + 3 * (int64_t)s.node[i];
    const double ux = ui[0], uy = ui[1], uz = ui[2];
    const double bx = s.b[i][0], by = s.b[i][1], bz = s.b[i][2];
    e[0] += bx * ux;
    e[1] += by * uy;
    e[2] += bz * uz;
    e[3] += bz * uy + by * uz;
    e[4] += bz * ux + bx * uz;
    e[5] += by * ux + bx * uy;
  }
  const double tr = e[0] + e[1] + e[2];
  const double sg[6] = {lam * tr + 2.0 * mu * e[0], lam * tr + 2.0 * mu * e[1], lam * tr + 2.0 * mu * e[2],
                        mu * e[3],                  mu * e[4],                  mu * e[5]};
  for (int j = 0; j < 6; ++j) {
    if (fstrain) fstrain[6 * f + j] = e[j];
    if (fstress) fstress[6 * f + j] = sg[j];
  }
  if (nacc) {
    for (int i = 0; i < 3; ++i) {  // the face's triangle
      double *a = nacc + kNodeAcc * (int64_t)s.node[i];
      for (int j = 0; j < 6; ++j) {
        atomicAdd(a + j, s.Vk * e[j]);
        atomicAdd(a + 6 + j, s.Vk * sg[j]);
      }
      atomicAdd(a + 12, s.Vk);
    }
  }
}

__device__ __forceinline__ double von_mises(const double *sg) {
  const double a = sg[0] - sg[1], b = sg[1] - sg[2], c = sg[2] - sg[0];
  return sqrt(0.5 * (a * a + b * b + c * c) + 3.0 * (sg[3] * sg[3] + sg[4] * sg[4] + sg[5] * sg[5]));
}

__global__ void k_recover_nodes(int64_t n_nodes, const double *__restrict__ nacc, double *__restrict__ nstrain,
                                double *__restrict__ nstress, double *__restrict__ nvm) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  const double *a = nacc + kNodeAcc * n;
  const double w = a[12] > 0.0 ? 1.0 / a[12] : 0.0;  // every node of a tet lies on a face
  double sg[6];
  for (int j = 0; j < 6; ++j) {
    sg[j] = a[6 + j] * w;
    if (nstrain) nstrain[6 * n + j] = a[j] * w;
    if (nstress) nstress[6 * n + j] = sg[j];
  }
  if (nvm) nvm[n] = von_mises(sg);
}

}  // namespace

}  // namespace sfem

using namespace sfem;

extern "C" int sfem_recover(sfem_ctx *h, const double *u, double *face_strain, double *face_stress,
                            double *node_strain, double *node_stress, double *node_vm) {
  try {
    SFEM_REQUIRE(h && h->c.vol && h->c.face_tet, SFEM_EINVAL, "context not set up");
    SFEM_REQUIRE(u, SFEM_EINVAL, "u must be a device pointer");
    Ctx &c = h->c;
    const bool nodal = node_strain || node_stress || node_vm;
    struct Scratch {  // the nodal sums, released on every exit
      Ctx &c;
      double *p = nullptr;
      ~Scratch() {
        if (p) c.mem.drop(p);
      }
    } acc{c};
    double *nacc = nullptr;
    if (nodal) {
      nacc = acc.p = c.mem.get<double>(kNodeAcc * c.n_nodes);
      SFEM_CUDA(cudaMemsetAsync(nacc, 0, kNodeAcc * c.n_nodes * sizeof(double), c.stream));
    }
    if (face_strain || face_stress || nodal) {
      k_recover_faces<<<grid_for(c.n_faces, 128), 128, 0, c.stream>>>(c.n_faces, c.tets, c.face_tet, c.face_slot,
                                                                     c.vol, c.grad, u, c.lam, c.mu, face_strain,
                                                                     face_stress, nacc);
      SFEM_CHECK_LAUNCH();
    }
    if (nodal) {
      k_recover_nodes<<<grid_for(c.n_nodes, 256), 256, 0, c.stream>>>(c.n_nodes, nacc, node_strain, node_stress,
                                                                      node_vm);
      SFEM_CHECK_LAUNCH();
    }
    SFEM_CUDA(cudaStreamSynchronize(c.stream));
  } catch (const Error &err) {
    set_last_error(err.msg);
    return err.status;
  }
  return SFEM_OK;
}
