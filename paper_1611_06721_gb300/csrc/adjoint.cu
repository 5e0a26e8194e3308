// Discrete adjoint of the explicit-Euler / Schur-complement time loop
// (Sec. II, eqs. (ODE), (acm)): gradient of the time-integrated eddy-current
// loss J = sum_m dt F_m^T M_c^-1 F_m (the FIT edge form of sum over cells of
// sigma |E|^2 dV, E = -da/dt on conducting edges) with respect to the cell
// conductivities and the coil amplitude.
//
// With lambda_m = dJ/da^m (lambda_M = 0), every reverse step m = M .. 1 does
//   mu        = dt M_c^-1 (2 F_m - lambda_m)                 (dJ/dF_m)
//   K_n w'    = -K_cn^T mu                                    (one PCG solve)
//   lambda   += (C^T J_H^T C [mu; w'])_c,   J_H = d(M_nu(b) b)/db at b = C a^{m-1}
//   dJ/dM_c  += dt F_m (lambda_m - F_m) / M_c^2
//   dJ/dI0   += -g(t_m) X_s . w'                             (i(t) = I0 g(t))
// and dJ/dsigma_cell = (h/4) * sum of dJ/dM_c over the cell's conducting edges.
// J_H^T y at a face f = M_nu[f] y_f + sum over the Brauer cells c of f of
// t_c S_{c,d(f)}, with S_{c,d} the sum of the fluxes of c's two d-normal faces
// and t_c = nu'(B_c^2) / (2 h^4) * sum over c's faces g of b_g y_g / (2h)
// (nu' = d nu / d(B^2) = k1 k2 exp(k2 B^2) of the Brauer law).
#include <cmath>
#include "mqs_kernels.h"
#include "conductor_fit.cuh"

namespace mqs {

namespace {

__device__ __forceinline__ long long box_cell(const CondGeom& cg, int i, int j, int k) {
  if (i < cg.clo[0] || j < cg.clo[1] || k < cg.clo[2] || i >= cg.chi[0] || j >= cg.chi[1] || k >= cg.chi[2])
    return -1;
  const int wx = cg.chi[0] - cg.clo[0], wy = cg.chi[1] - cg.clo[1];
  return (i - cg.clo[0]) + (long long)wx * ((j - cg.clo[1]) + (long long)wy * (k - cg.clo[2]));
}

__device__ __forceinline__ long long box_cells(const CondGeom& cg) {
  return (long long)(cg.chi[0] - cg.clo[0]) * (cg.chi[1] - cg.clo[1]) * (cg.chi[2] - cg.clo[2]);
}

// t_c S_{c,d} of cell (i, j, k), zero outside the box and in linear cells
__device__ __forceinline__ double tsd(const CondGeom& cg, const double* tS, int d, int i, int j, int k) {
  const long long q = box_cell(cg, i, j, k);
  return q < 0 ? 0.0 : MQS_LDC(tS, d * box_cells(cg) + q, 3 * box_cells(cg), 501);
}

__device__ __forceinline__ double block_reduce(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  return sh[0];
}

}  // namespace

__global__ void adj_mu_kernel(CondGeom cg, const double* F, AdjBufs ab, double dt, long long n3) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < cg.n_c; q += gridDim.x * blockDim.x) {
    const double f = F[q], l = ab.lam[q], im = cg.inv_mc[q];
    MQS_STC(ab.mu_full, cg.c_idx[q], 3 * n3, 502, dt * im * fma(2.0, f, -l));
    ab.gmc[q] += dt * f * (l - f) * im * im;
  }
}

__global__ void adj_cell_kernel(Geom g, CondGeom cg, const double* x, AdjBufs ab) {
  const int n = g.n;
  const long long n3 = g.n3, nb = box_cells(cg);
  const int wx = cg.chi[0] - cg.clo[0], wy = cg.chi[1] - cg.clo[1];
  const double h = cg.h, h2 = h * h;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nb; q += (long long)gridDim.x * blockDim.x) {
    if (!cg.brauer[q]) {
      ab.tS[q] = 0.0; ab.tS[nb + q] = 0.0; ab.tS[2 * nb + q] = 0.0;
      continue;
    }
    const int i = cg.clo[0] + (int)(q % wx), j = cg.clo[1] + (int)((q / wx) % wy),
              k = cg.clo[2] + (int)(q / ((long long)wx * wy));
    const double* ap = ab.ap_full;
    const double* mu = ab.mu_full;
    // forward fluxes of a^{m-1} (the faces of a conducting cell carry c-edges only)
    const double bxm = fbx(ap, ap, 0.0, n, n3, i, j, k), bxp = fbx(ap, ap, 0.0, n, n3, i + 1, j, k);
    const double bym = fby(ap, ap, 0.0, n, n3, i, j, k), byp = fby(ap, ap, 0.0, n, n3, i, j + 1, k);
    const double bzm = fbz(ap, ap, 0.0, n, n3, i, j, k), bzp = fbz(ap, ap, 0.0, n, n3, i, j, k + 1);
    // adjoint fluxes of [mu; w']
    const double yxm = fbx(mu, x, 1.0, n, n3, i, j, k), yxp = fbx(mu, x, 1.0, n, n3, i + 1, j, k);
    const double yym = fby(mu, x, 1.0, n, n3, i, j, k), yyp = fby(mu, x, 1.0, n, n3, i, j + 1, k);
    const double yzm = fbz(mu, x, 1.0, n, n3, i, j, k), yzp = fbz(mu, x, 1.0, n, n3, i, j, k + 1);
    const double sx = bxm + bxp, sy = bym + byp, sz = bzm + bzp;
    const double s = 2.0 * h2;
    const double B2 = (sx * sx + sy * sy + sz * sz) / (s * s);
    const double ex = exp(cg.k2 * B2);
    cg.nu[q] = fma(cg.k1, ex, cg.k3);                // nu of the forward step (Brauer law)
    const double dnu = cg.k1 * cg.k2 * ex;           // d nu / d(B^2)
    const double by = bxm * yxm + bxp * yxp + bym * yym + byp * yyp + bzm * yzm + bzp * yzp;
    const double t = dnu / (2.0 * h2 * h2) * by / (2.0 * h);
    ab.tS[q] = t * sx;
    ab.tS[nb + q] = t * sy;
    ab.tS[2 * nb + q] = t * sz;
  }
}

// lam += (C^T J_H^T C [mu; w'])_c: the face structure of cond_update_kernel with
// the adjoint fluxes y and the Brauer term added per face
__global__ void adj_lambda_kernel(Geom g, CondGeom cg, const double* x, AdjBufs ab) {
  const int n = g.n;
  const long long n3 = g.n3;
  const double ih2 = 0.5 / cg.h;
  const double* mu = ab.mu_full;
  const double* tS = ab.tS;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < cg.n_c; q += gridDim.x * blockDim.x) {
    const long long e = cg.c_idx[q];
    const int c = (int)(e / n3);
    const long long pos = e - c * n3;
    const int i = (int)(pos % n), j = (int)((pos / n) % n), k = (int)(pos / ((long long)n * n));
    // Brauer terms of the x-, y- and z-normal faces at (a, b, c): both cells of the face
    auto Ex = [&](int a, int b, int cc) { return tsd(cg, tS, 0, a - 1, b, cc) + tsd(cg, tS, 0, a, b, cc); };
    auto Ey = [&](int a, int b, int cc) { return tsd(cg, tS, 1, a, b - 1, cc) + tsd(cg, tS, 1, a, b, cc); };
    auto Ez = [&](int a, int b, int cc) { return tsd(cg, tS, 2, a, b, cc - 1) + tsd(cg, tS, 2, a, b, cc); };
    double G;
    if (c == 0) {
      const double m1 = (cell_nu(cg, i, j, k - 1) + cell_nu(cg, i, j, k)) * ih2;
      const double m2 = (cell_nu(cg, i, j - 1, k - 1) + cell_nu(cg, i, j - 1, k)) * ih2;
      const double m3 = (cell_nu(cg, i, j - 1, k) + cell_nu(cg, i, j, k)) * ih2;
      const double m4 = (cell_nu(cg, i, j - 1, k - 1) + cell_nu(cg, i, j, k - 1)) * ih2;
      G = fma(m1, fbz(mu, x, 1.0, n, n3, i, j, k), Ez(i, j, k)) -
          fma(m2, fbz(mu, x, 1.0, n, n3, i, j - 1, k), Ez(i, j - 1, k)) -
          fma(m3, fby(mu, x, 1.0, n, n3, i, j, k), Ey(i, j, k)) +
          fma(m4, fby(mu, x, 1.0, n, n3, i, j, k - 1), Ey(i, j, k - 1));
    } else if (c == 1) {
      const double m1 = (cell_nu(cg, i - 1, j, k - 1) + cell_nu(cg, i - 1, j, k)) * ih2;
      const double m2 = (cell_nu(cg, i, j, k - 1) + cell_nu(cg, i, j, k)) * ih2;
      const double m3 = (cell_nu(cg, i - 1, j, k) + cell_nu(cg, i, j, k)) * ih2;
      const double m4 = (cell_nu(cg, i - 1, j, k - 1) + cell_nu(cg, i, j, k - 1)) * ih2;
      G = fma(m1, fbz(mu, x, 1.0, n, n3, i - 1, j, k), Ez(i - 1, j, k)) -
          fma(m2, fbz(mu, x, 1.0, n, n3, i, j, k), Ez(i, j, k)) +
          fma(m3, fbx(mu, x, 1.0, n, n3, i, j, k), Ex(i, j, k)) -
          fma(m4, fbx(mu, x, 1.0, n, n3, i, j, k - 1), Ex(i, j, k - 1));
    } else {
      const double m1 = (cell_nu(cg, i - 1, j - 1, k) + cell_nu(cg, i, j - 1, k)) * ih2;
      const double m2 = (cell_nu(cg, i - 1, j, k) + cell_nu(cg, i, j, k)) * ih2;
      const double m3 = (cell_nu(cg, i, j - 1, k) + cell_nu(cg, i, j, k)) * ih2;
      const double m4 = (cell_nu(cg, i - 1, j - 1, k) + cell_nu(cg, i - 1, j, k)) * ih2;
      G = fma(m1, fbx(mu, x, 1.0, n, n3, i, j - 1, k), Ex(i, j - 1, k)) -
          fma(m2, fbx(mu, x, 1.0, n, n3, i, j, k), Ex(i, j, k)) +
          fma(m3, fby(mu, x, 1.0, n, n3, i, j, k), Ey(i, j, k)) -
          fma(m4, fby(mu, x, 1.0, n, n3, i - 1, j, k), Ey(i - 1, j, k));
    }
    ab.lam[q] += G;
  }
}

// gI += -g(t) X_s . w' with g the unit-amplitude coil waveform (as in the right-hand side kernel)
__global__ void adj_coil_kernel(Geom g, CoilGeom coil, CoilDrive drv, const double* x, AdjBufs ab) {
  __shared__ double sh[256];
  const int n = g.n;
  const long long n3 = g.n3;
  const int L1 = coil.i1 - coil.i0, L2 = coil.j1 - coil.j0, tot = 2 * L1 + 2 * L2;
  double s = 0.0;
  for (int t = threadIdx.x; t < tot; t += blockDim.x) {
    if (t < L1) s += MQS_LDC(x, pidx(n, coil.i0 + t, coil.j0, coil.k), 3 * n3, 503);
    else if (t < 2 * L1) s -= MQS_LDC(x, pidx(n, coil.i0 + t - L1, coil.j1, coil.k), 3 * n3, 504);
    else if (t < 2 * L1 + L2) s += MQS_LDC(x, n3 + pidx(n, coil.i1, coil.j0 + t - 2 * L1, coil.k), 3 * n3, 505);
    else s -= MQS_LDC(x, n3 + pidx(n, coil.i0, coil.j0 + t - 2 * L1 - L2, coil.k), 3 * n3, 506);
  }
  const double tot_s = block_reduce(s, sh);
  if (threadIdx.x == 0) {
    const double gt = (drv.waveform == 0) ? sin(2.0 * 3.141592653589793 * drv.freq * drv.t)
                                          : 1.0 - exp(-drv.t / drv.tau);
    ab.gI[0] += -gt * tot_s;
  }
}

__global__ void adj_objective_kernel(CondGeom cg, const double* F, long long total, double* part) {
  __shared__ double sh[256];
  double s = 0.0;
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < total;
       u += (long long)gridDim.x * blockDim.x) {
    const double f = F[u];
    s = fma(f * f, cg.inv_mc[u % cg.n_c], s);
  }
  const double b = block_reduce(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

// out[0] += scale * sum(part[0..cnt))
__global__ void adj_sum_kernel(const double* part, int cnt, double scale, double* out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int q = threadIdx.x; q < cnt; q += blockDim.x) s += part[q];
  const double t = block_reduce(s, sh);
  if (threadIdx.x == 0) out[0] += scale * t;
}

__global__ void adj_qmap_kernel(Geom g, CondGeom cg, int* qmap) {
  const int ex = cg.chi[0] - cg.clo[0] + 1, ey = cg.chi[1] - cg.clo[1] + 1, ez = cg.chi[2] - cg.clo[2] + 1;
  const long long nn = (long long)ex * ey * ez;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < cg.n_c; q += gridDim.x * blockDim.x) {
    const long long e = cg.c_idx[q];
    const int c = (int)(e / g.n3);
    const long long pos = e - c * g.n3;
    const int i = (int)(pos % g.n) - cg.clo[0], j = (int)((pos / g.n) % g.n) - cg.clo[1],
              k = (int)(pos / ((long long)g.n * g.n)) - cg.clo[2];
    if (i >= 0 && j >= 0 && k >= 0 && i < ex && j < ey && k < ez)
      MQS_STC(qmap, c * nn + i + (long long)ex * (j + (long long)ey * k), 3 * nn, 507, q);
  }
}

__global__ void adj_sigma_kernel(CondGeom cg, const uint8_t* cond, AdjBufs ab, double* out) {
  const int wx = cg.chi[0] - cg.clo[0], wy = cg.chi[1] - cg.clo[1];
  const long long nb = box_cells(cg);
  const int ex = wx + 1, ey = wy + 1, ez = cg.chi[2] - cg.clo[2] + 1;
  const long long nn = (long long)ex * ey * ez;
  auto qm = [&](int c, int i, int j, int k) {
    return MQS_LDC(ab.qmap, c * nn + i + (long long)ex * (j + (long long)ey * k), 3 * nn, 508);
  };
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nb; q += (long long)gridDim.x * blockDim.x) {
    if (!cond[q]) { out[q] = 0.0; continue; }
    const int i = (int)(q % wx), j = (int)((q / wx) % wy), k = (int)(q / ((long long)wx * wy));   // box-relative
    double s = 0.0;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        const int qx = qm(0, i, j + a, k + b), qy = qm(1, i + a, j, k + b), qz = qm(2, i + a, j + b, k);
        if (qx >= 0) s += MQS_LDC(ab.gmc, qx, cg.n_c, 509);
        if (qy >= 0) s += MQS_LDC(ab.gmc, qy, cg.n_c, 510);
        if (qz >= 0) s += MQS_LDC(ab.gmc, qz, cg.n_c, 511);
      }
    out[q] = 0.25 * cg.h * s;          // M_kappa = h * mean sigma of the four cells of an edge
  }
}

static int blocks_for(long long work) {
  long long b = (work + 255) / 256;
  if (b > 1024) b = 1024;
  if (b < 1) b = 1;
  return (int)b;
}
static int ok() { return cudaGetLastError() == cudaSuccess ? MQS_OK : MQS_ERR_CUDA; }
static long long cell_count(const CondGeom& cg) {
  return (long long)(cg.chi[0] - cg.clo[0]) * (cg.chi[1] - cg.clo[1]) * (cg.chi[2] - cg.clo[2]);
}

int launch_adj_mu(const CondGeom& cg, const double* F, const AdjBufs& ab, double dt, long long n3, cudaStream_t st) {
  adj_mu_kernel<<<blocks_for(cg.n_c), 256, 0, st>>>(cg, F, ab, dt, n3);
  return ok();
}

int launch_adj_cell(const DevGeom& dg, const CondGeom& cg, const double* x, const AdjBufs& ab, cudaStream_t st) {
  adj_cell_kernel<<<blocks_for(cell_count(cg)), 256, 0, st>>>(dg.g, cg, x, ab);
  return ok();
}

int launch_adj_lambda(const DevGeom& dg, const CondGeom& cg, const double* x, const AdjBufs& ab, cudaStream_t st) {
  adj_lambda_kernel<<<blocks_for(cg.n_c), 256, 0, st>>>(dg.g, cg, x, ab);
  return ok();
}

int launch_adj_coil(const DevGeom& dg, const CoilGeom& coil, const CoilDrive& drv, const double* x,
                          const AdjBufs& ab, cudaStream_t st) {
  adj_coil_kernel<<<1, 256, 0, st>>>(dg.g, coil, drv, x, ab);
  return ok();
}

int launch_adj_objective(const CondGeom& cg, const double* F_traj, int nsteps, double dt, const AdjBufs& ab,
                         double* J_dev, cudaStream_t st) {
  const long long total = (long long)nsteps * cg.n_c;
  const int nb = blocks_for(total);
  adj_objective_kernel<<<nb, 256, 0, st>>>(cg, F_traj, total, ab.part);
  adj_sum_kernel<<<1, 256, 0, st>>>(ab.part, nb, dt, J_dev);
  return ok();
}

int launch_adj_qmap(const DevGeom& dg, const CondGeom& cg, const AdjBufs& ab, cudaStream_t st) {
  adj_qmap_kernel<<<blocks_for(cg.n_c), 256, 0, st>>>(dg.g, cg, ab.qmap);
  return ok();
}

int launch_adj_sigma(const DevGeom& dg, const CondGeom& cg, const uint8_t* cond, const AdjBufs& ab, double* out,
                     cudaStream_t st) {
  (void)dg;
  adj_sigma_kernel<<<blocks_for(cell_count(cg)), 256, 0, st>>>(cg, cond, ab, out);
  return ok();
}

MQS_DEBUG_TAKE(adjoint)

}  // namespace mqs
