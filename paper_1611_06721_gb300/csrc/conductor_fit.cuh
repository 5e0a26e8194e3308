// Face fluxes and face reluctances of the conducting region (shared by the
// explicit-Euler update and its adjoint).  Faces are indexed by their lower
// corner and normal; the flux of a face is the circulation of a around it
// (right-handed), C a in the FIT notation of Sec. II.
#pragma once
#include "mqs_kernels.h"

namespace mqs {

__device__ __forceinline__ double lda(const double* ac, const double* w, double sw, int n, long long n3, int c,
                                      int i, int j, int k) {
  return fma(sw, ld(w, n, n3, c, i, j, k), ld(ac, n, n3, c, i, j, k));
}
// face fluxes of a = ac + sw w
__device__ __forceinline__ double fbx(const double* ac, const double* w, double sw, int n, long long n3, int i,
                                      int j, int k) {
  return (lda(ac, w, sw, n, n3, 1, i, j, k) - lda(ac, w, sw, n, n3, 2, i, j, k)) +
         (lda(ac, w, sw, n, n3, 2, i, j + 1, k) - lda(ac, w, sw, n, n3, 1, i, j, k + 1));
}
__device__ __forceinline__ double fby(const double* ac, const double* w, double sw, int n, long long n3, int i,
                                      int j, int k) {
  return (lda(ac, w, sw, n, n3, 2, i, j, k) - lda(ac, w, sw, n, n3, 0, i, j, k)) +
         (lda(ac, w, sw, n, n3, 0, i, j, k + 1) - lda(ac, w, sw, n, n3, 2, i + 1, j, k));
}
__device__ __forceinline__ double fbz(const double* ac, const double* w, double sw, int n, long long n3, int i,
                                      int j, int k) {
  return (lda(ac, w, sw, n, n3, 0, i, j, k) - lda(ac, w, sw, n, n3, 1, i, j, k)) +
         (lda(ac, w, sw, n, n3, 1, i + 1, j, k) - lda(ac, w, sw, n, n3, 0, i, j + 1, k));
}

__device__ __forceinline__ double cell_nu(const CondGeom& cg, int i, int j, int k) {
  if (i < cg.clo[0] || j < cg.clo[1] || k < cg.clo[2] || i >= cg.chi[0] || j >= cg.chi[1] || k >= cg.chi[2])
    return cg.nu0;
  const int wx = cg.chi[0] - cg.clo[0], wy = cg.chi[1] - cg.clo[1];
  return MQS_LDC(cg.nu, (i - cg.clo[0]) + wx * ((j - cg.clo[1]) + (long long)wy * (k - cg.clo[2])),
                 (long long)wx * wy * (cg.chi[2] - cg.clo[2]), 401);
}

}  // namespace mqs
