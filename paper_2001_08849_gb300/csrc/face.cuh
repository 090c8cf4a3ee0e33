// Smoothed gradients of one face in FP64 (shared by setup and assembly).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sfem {

// ---------------------------------------------------------------------------
// smoothed gradients of one face (FP64): b_I = sum_e (V_e/4) grad N_I^e / V_k
// over the stencil (a, b, c, d0, d1)
// ---------------------------------------------------------------------------
struct FaceStencil {
  int node[5];
  double b[5][3];
  double Vk;
  int nn;
};

static __device__ __forceinline__ void face_stencil(int64_t f, const int32_t *__restrict__ tets,
                                             const int32_t *__restrict__ face_tet,
                                             const int32_t *__restrict__ face_slot, const double *__restrict__ vol,
                                             const double *__restrict__ grad, FaceStencil &s) {
  int e0 = face_tet[2 * f], e1 = face_tet[2 * f + 1];
  int a0 = face_slot[2 * f], a1 = face_slot[2 * f + 1];
  int4 t0 = reinterpret_cast<const int4 *>(tets)[e0];
  int v0[4] = {t0.x, t0.y, t0.z, t0.w};
  int loc0[5];
  int k = 0;
  for (int b = 0; b < 4; ++b)
    if (b != a0) {
      s.node[k] = v0[b];
      loc0[k] = b;
      ++k;
    }
  // order the face nodes ascending (a < b < c)
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (s.node[j] < s.node[i]) {
        int tn = s.node[i];
        s.node[i] = s.node[j];
        s.node[j] = tn;
        int tl = loc0[i];
        loc0[i] = loc0[j];
        loc0[j] = tl;
      }
  s.node[3] = v0[a0];
  loc0[3] = a0;
  double V0 = vol[e0], V1 = 0.0;
  s.nn = 4;
  s.node[4] = -1;
  int loc1[5] = {-1, -1, -1, -1, -1};
  if (e1 >= 0) {
    s.nn = 5;
    int4 t1 = reinterpret_cast<const int4 *>(tets)[e1];
    int v1[4] = {t1.x, t1.y, t1.z, t1.w};
    s.node[4] = v1[a1];
    loc1[4] = a1;
    for (int i = 0; i < 3; ++i)
      for (int b = 0; b < 4; ++b)
        if (v1[b] == s.node[i]) loc1[i] = b;
    V1 = vol[e1];
  }
  s.Vk = 0.25 * (V0 + V1);
  double w0 = 0.25 * V0 / s.Vk, w1 = 0.25 * V1 / s.Vk;
  for (int i = 0; i < 5; ++i)
    for (int c = 0; c < 3; ++c) s.b[i][c] = 0.0;
  for (int i = 0; i < 4; ++i)
    for (int c = 0; c < 3; ++c) s.b[i][c] += w0 * grad[12 * (int64_t)e0 + 3 * loc0[i] + c];
  if (e1 >= 0) {
    for (int i = 0; i < 5; ++i) {
      if (i == 3 || loc1[i] < 0) continue;  // loc1 >= 0 for a valid neighbour table
      for (int c = 0; c < 3; ++c) s.b[i][c] += w1 * grad[12 * (int64_t)e1 + 3 * loc1[i] + c];
    }
  }
}

}  // namespace sfem
