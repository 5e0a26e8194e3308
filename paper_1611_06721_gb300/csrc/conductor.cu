// Right-hand side assembly, stand-alone stencil application and the
// conducting-region update of the explicit Euler step (Sec. II, eq. (acm)).
#include <cmath>
#include "mqs_kernels.h"
#include "conductor_fit.cuh"

namespace mqs {

struct EpiApply {  // y = scale * t on n-edges, zero elsewhere
  double* y; long long n3; double scale;
  __device__ void prefetch(long long) {}
  __device__ void operator()(long long e, unsigned m, double tx, double ty, double tz, double, double, double) {
    y[e] = (m & 1u) ? scale * tx : 0.0;
    y[e + n3] = (m & 2u) ? scale * ty : 0.0;
    y[e + 2 * n3] = (m & 4u) ? scale * tz : 0.0;
  }
};

__global__ void __launch_bounds__(kBlock) apply_L_kernel(Geom g, const double* s, double* y, double scale, Box box) {
  __shared__ SweepSmem sm;
  EpiApply ep{y, g.n3, scale};
  sweep_L(g, s, box, blockIdx.x, gridDim.x, sm, ep);
}

// coil distribution X_s of one edge (Sec. II, J_S = X_S i_S(t))
__device__ __forceinline__ double coil_xs(const CoilGeom& c, int comp, int i, int j, int k) {
  if (k != c.k) return 0.0;
  if (comp == 0 && i >= c.i0 && i < c.i1) return (j == c.j0) ? 1.0 : (j == c.j1) ? -1.0 : 0.0;
  if (comp == 1 && j >= c.j0 && j < c.j1) return (i == c.i1) ? 1.0 : (i == c.i0) ? -1.0 : 0.0;
  return 0.0;
}

// face fluxes of one layout vector (zero outside the grid), grouped as in sweep_L
__device__ __forceinline__ double flux_x(const double* a, int n, long long n3, int i, int j, int k) {
  return (ld(a, n, n3, 1, i, j, k) - ld(a, n, n3, 2, i, j, k)) + (ld(a, n, n3, 2, i, j + 1, k) - ld(a, n, n3, 1, i, j, k + 1));
}
__device__ __forceinline__ double flux_y(const double* a, int n, long long n3, int i, int j, int k) {
  return (ld(a, n, n3, 2, i, j, k) - ld(a, n, n3, 0, i, j, k)) + (ld(a, n, n3, 0, i, j, k + 1) - ld(a, n, n3, 2, i + 1, j, k));
}
__device__ __forceinline__ double flux_z(const double* a, int n, long long n3, int i, int j, int k) {
  return (ld(a, n, n3, 0, i, j, k) - ld(a, n, n3, 1, i, j, k)) + (ld(a, n, n3, 1, i + 1, j, k) - ld(a, n, n3, 0, i, j + 1, k));
}

// b = coil_scale X_s - (L ac) at the listed n-edges only (the right-hand side's
// support: edges sharing a face with a c-edge, and the coil); one edge per thread,
// the same arithmetic and grouping as the sweep's, so b is bitwise the sweep's
__global__ void __launch_bounds__(256) rhs_list_kernel(Geom g, const double* ac, double* b, CoilDrive drv,
                                                       CoilGeom coil, const int* sup, int nsup) {
  const double t = drv.m_dev ? (double)(*drv.m_dev + drv.level) * drv.dt : drv.t;
  const double i_t = (drv.waveform == 0) ? drv.amplitude * sin(2.0 * 3.141592653589793 * drv.freq * t)
                                         : drv.amplitude * (1.0 - exp(-t / drv.tau));
  const double cs = drv.scale * i_t;
  const int n = g.n;
  const long long n3 = g.n3;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nsup; q += gridDim.x * blockDim.x) {
    const int e = sup[q];
    const int c = (int)(e / n3);   // e < 3 n^3: checked at the store
    const int pos = (int)(e - c * n3);
    const int i = pos % n, j = (pos / n) % n, k = pos / (n * n);
    double t;
    if (c == 0) t = (flux_z(ac, n, n3, i, j, k) - flux_z(ac, n, n3, i, j - 1, k)) +
                    (flux_y(ac, n, n3, i, j, k - 1) - flux_y(ac, n, n3, i, j, k));
    else if (c == 1) t = (flux_z(ac, n, n3, i - 1, j, k) - flux_z(ac, n, n3, i, j, k)) +
                         (flux_x(ac, n, n3, i, j, k) - flux_x(ac, n, n3, i, j, k - 1));
    else t = (flux_x(ac, n, n3, i, j - 1, k) - flux_x(ac, n, n3, i, j, k)) +
             (flux_y(ac, n, n3, i, j, k) - flux_y(ac, n, n3, i - 1, j, k));
    MQS_STC(b, e, 3 * n3, 402, fma(cs, coil_xs(coil, c, i, j, k), -t));
  }
}

// Block size of the per-edge and per-cell kernels of the step (tens of thousands of
// edges or cells: 35-119 blocks of 256 threads).  64-thread blocks, spread over every SM,
// took the same time launch by launch but made graph-replayed steps 10% slower (2000 steps:
// 1891 against 2115 steps/s): beside them the side stream's push, one block per SM,
// started later.
constexpr int kSmallBlock = 256;

static int stencil_grid(const Box& box) {
  long long ntx = (box.hi[0] - box.lo[0] + 31) / 32, nty = (box.hi[1] - box.lo[1] + kTY - 1) / kTY;
  long long T = ntx * nty * (box.hi[2] - box.lo[2]);
  long long blocks = (T + 3) / 4;              // about four plane-tiles per block
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

int launch_apply_L(const DevGeom& dg, const double* s, double* y, double scale, Box box, cudaStream_t st) {
  apply_L_kernel<<<stencil_grid(box), kBlock, 0, st>>>(dg.g, s, y, scale, box);
  return cudaGetLastError() == cudaSuccess ? MQS_OK : MQS_ERR_CUDA;
}

int launch_rhs(const DevGeom& dg, const double* ac_full, double* b, CoilDrive drive, CoilGeom coil, const int* sup,
               int nsup, cudaStream_t st) {
  if (nsup <= 0) return MQS_OK;
  rhs_list_kernel<<<(nsup + kSmallBlock - 1) / kSmallBlock, kSmallBlock, 0, st>>>(dg.g, ac_full, b, drive, coil,
                                                                                   sup, nsup);
  return cudaGetLastError() == cudaSuccess ? MQS_OK : MQS_ERR_CUDA;
}

// ---- conducting region ------------------------------------------------------------
__global__ void cell_nu_kernel(Geom g, CondGeom cg, const double* ac, const double* w, int at_zero,
                               const int* halt) {
  if (halt && *halt) return;
  const int wx = cg.chi[0] - cg.clo[0], wy = cg.chi[1] - cg.clo[1], wz = cg.chi[2] - cg.clo[2];
  const long long ncell = (long long)wx * wy * wz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ncell;
       q += (long long)gridDim.x * blockDim.x) {
    if (!cg.brauer[q]) { cg.nu[q] = cg.nu0; continue; }
    double B2 = 0.0;
    if (!at_zero) {
      const int i = cg.clo[0] + (int)(q % wx), j = cg.clo[1] + (int)((q / wx) % wy),
                k = cg.clo[2] + (int)(q / ((long long)wx * wy));
      const int n = g.n;
      const long long n3 = g.n3;
      const double sx = fbx(ac, w, 1.0, n, n3, i, j, k) + fbx(ac, w, 1.0, n, n3, i + 1, j, k);
      const double sy = fby(ac, w, 1.0, n, n3, i, j, k) + fby(ac, w, 1.0, n, n3, i, j + 1, k);
      const double sz = fbz(ac, w, 1.0, n, n3, i, j, k) + fbz(ac, w, 1.0, n, n3, i, j, k + 1);
      const double s = 2.0 * cg.h * cg.h;
      B2 = (sx * sx + sy * sy + sz * sz) / (s * s);
    }
    cg.nu[q] = fma(cg.k1, exp(cg.k2 * B2), cg.k3);   // Brauer nu(B) = k1 exp(k2 B^2) + k3
  }
}

// The instability monitor's step (last block of a guarded conductor update): with
// e = M_c-energy of the increment d_m = a^m - a^{m-1} and s = d_m^T M_c d_{m-1}, a step
// whose increment grew (e > e_prev) while changing sign (s < 0), above 1e-20 of the
// largest increment energy seen, extends a run of such steps; `window` of them in a
// row, or a non-finite increment, is the explicit Euler instability of a mode with
// 1 - dt lambda < -1 (eq. (CFL) violated).  Each block's partials (e, s) are summed in a
// fixed order, so the verdict does not depend on scheduling.
__device__ void monitor_finish(const GuardView& gv, double e, double s) {
  __shared__ double red[2][32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  e = warp_sum(e);
  s = warp_sum(s);
  if (lane == 0) { red[0][w] = e; red[1][w] = s; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double be = 0.0, bs = 0.0;
    for (int q = 0; q < nw; ++q) { be += red[0][q]; bs += red[1][q]; }
    gv.part[2 * blockIdx.x] = be;
    gv.part[2 * blockIdx.x + 1] = bs;
    __threadfence();
    last = atomicAdd(&gv.gd->arrive, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || w != 0) return;
  __threadfence();
  // the partials from L2 (ld.global.cg: another SM wrote them), eight per lane issued
  // together before they are added (a loop that adds each load before issuing the next
  // waits one L2 round trip per 32 blocks)
  double E = 0.0, S = 0.0;
  const int nb = (int)gridDim.x;
  for (int b0 = 0; b0 < nb; b0 += 256) {
    double2 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int b = b0 + lane + 32 * q;
      v[q] = (b < nb) ? __ldcg(reinterpret_cast<const double2*>(gv.part) + b) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) { E += v[q].x; S += v[q].y; }
  }
  E = warp_sum(E);
  S = warp_sum(S);
  if (lane != 0) return;
  StepGuard* gd = gv.gd;
  int status = MQS_OK;
  if (!isfinite(E) || (gd->valid && !isfinite(S))) {
    status = MQS_ERR_UNSTABLE;
  } else {
    const bool grow = gd->valid && E > gd->e_prev && S < 0.0 && E > 1e-20 * gd->e_max;
    gd->count = grow ? gd->count + 1 : 0;
    if (gv.window > 0 && gd->count >= gv.window) status = MQS_ERR_UNSTABLE;
    gd->e_max = fmax(gd->e_max, E);
    gd->e_prev = E;
    gd->valid = 1;
  }
  gd->status = status;
  gd->arrive = 0u;
}

// F_e = sum over the four faces f of e of C_fe M_nu[f] (C a)_f with
// M_nu[f] = (nu of the two cells of f) / (2h); a_c update of eq. (acm).
__global__ void cond_update_kernel(Geom g, CondGeom cg, const double* ac, const double* w, double sw,
                                   const double* a_in, double* a_out, double dt, double* ac_out, double* F_out,
                                   double* a_prev_out, GuardView gv) {
  if (gv.gd) {
    // a halted call, a failed solve or a timed-out wait: this step writes nothing
    if (*(volatile const int*)&gv.gd->halt || (gv.pres && gv.pres->status != MQS_OK) || (gv.derr && *gv.derr != 0))
      return;
  }
  const bool mon = gv.gd != nullptr && dt != 0.0;
  const bool prev = mon && gv.gd->valid;     // a_out holds a^{m-2}: the previous increment is known
  double en = 0.0, sx = 0.0;
  const int n = g.n;
  const long long n3 = g.n3;
  const double ih2 = 0.5 / cg.h;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < cg.n_c; q += gridDim.x * blockDim.x) {
    const long long e = cg.c_idx[q];
    const int c = (int)(e / n3);
    const long long pos = e - c * n3;
    const int i = (int)(pos % n), j = (int)((pos / n) % n), k = (int)(pos / ((long long)n * n));
    double F;
    if (c == 0) {
      const double m1 = (cell_nu(cg, i, j, k - 1) + cell_nu(cg, i, j, k)) * ih2;        // z-face (i,j,k)
      const double m2 = (cell_nu(cg, i, j - 1, k - 1) + cell_nu(cg, i, j - 1, k)) * ih2; // z-face (i,j-1,k)
      const double m3 = (cell_nu(cg, i, j - 1, k) + cell_nu(cg, i, j, k)) * ih2;        // y-face (i,j,k)
      const double m4 = (cell_nu(cg, i, j - 1, k - 1) + cell_nu(cg, i, j, k - 1)) * ih2; // y-face (i,j,k-1)
      F = m1 * fbz(ac, w, sw, n, n3, i, j, k) - m2 * fbz(ac, w, sw, n, n3, i, j - 1, k) -
          m3 * fby(ac, w, sw, n, n3, i, j, k) + m4 * fby(ac, w, sw, n, n3, i, j, k - 1);
    } else if (c == 1) {
      const double m1 = (cell_nu(cg, i - 1, j, k - 1) + cell_nu(cg, i - 1, j, k)) * ih2; // z-face (i-1,j,k)
      const double m2 = (cell_nu(cg, i, j, k - 1) + cell_nu(cg, i, j, k)) * ih2;        // z-face (i,j,k)
      const double m3 = (cell_nu(cg, i - 1, j, k) + cell_nu(cg, i, j, k)) * ih2;        // x-face (i,j,k)
      const double m4 = (cell_nu(cg, i - 1, j, k - 1) + cell_nu(cg, i, j, k - 1)) * ih2; // x-face (i,j,k-1)
      F = m1 * fbz(ac, w, sw, n, n3, i - 1, j, k) - m2 * fbz(ac, w, sw, n, n3, i, j, k) +
          m3 * fbx(ac, w, sw, n, n3, i, j, k) - m4 * fbx(ac, w, sw, n, n3, i, j, k - 1);
    } else {
      const double m1 = (cell_nu(cg, i - 1, j - 1, k) + cell_nu(cg, i, j - 1, k)) * ih2; // x-face (i,j-1,k)
      const double m2 = (cell_nu(cg, i - 1, j, k) + cell_nu(cg, i, j, k)) * ih2;        // x-face (i,j,k)
      const double m3 = (cell_nu(cg, i, j - 1, k) + cell_nu(cg, i, j, k)) * ih2;        // y-face (i,j,k)
      const double m4 = (cell_nu(cg, i - 1, j - 1, k) + cell_nu(cg, i - 1, j, k)) * ih2; // y-face (i-1,j,k)
      F = m1 * fbx(ac, w, sw, n, n3, i, j - 1, k) - m2 * fbx(ac, w, sw, n, n3, i, j, k) +
          m3 * fby(ac, w, sw, n, n3, i, j, k) - m4 * fby(ac, w, sw, n, n3, i - 1, j, k);
    }
    const double a0 = a_in[q];
    const double v = (dt != 0.0) ? fma(-dt * cg.inv_mc[q], F, a0) : F;
    if (mon) {
      const double md = -dt * F;                  // M_c (a^m - a^{m-1})
      en = fma(md * md, cg.inv_mc[q], en);        // M_c |a^m - a^{m-1}|^2
      if (prev) sx = fma(md, a0 - a_out[q], sx);  // with a^{m-1} - a^{m-2} (a_out read before written)
    }
    if (F_out) F_out[q] = F;            // recorded trajectory (adjoint)
    if (a_prev_out) a_prev_out[q] = a0;
    a_out[q] = v;
    if (ac_out) MQS_STC(ac_out, e, 3 * n3, 403, v);   // the other layout buffer (read and written buffers differ)
  }
  if (mon) monitor_finish(gv, en, sx);
}

__global__ void scatter_c_kernel(int n_c, const int* c_idx, const double* a_c, double* ac_full, double scale,
                                 long long n3) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n_c; q += gridDim.x * blockDim.x)
    MQS_STC(ac_full, c_idx[q], 3 * n3, 404, scale * a_c[q]);
}

int launch_cell_nu(const DevGeom& dg, const CondGeom& cg, const double* ac_full, const double* w, bool at_zero,
                   cudaStream_t st, const int* halt) {
  const long long ncell = (long long)(cg.chi[0] - cg.clo[0]) * (cg.chi[1] - cg.clo[1]) * (cg.chi[2] - cg.clo[2]);
  int blocks = (int)((ncell + kSmallBlock - 1) / kSmallBlock);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  cell_nu_kernel<<<blocks, kSmallBlock, 0, st>>>(dg.g, cg, ac_full, w, at_zero ? 1 : 0, halt);
  return cudaGetLastError() == cudaSuccess ? MQS_OK : MQS_ERR_CUDA;
}

int launch_cond_update(const DevGeom& dg, const CondGeom& cg, const double* ac_full, const double* w,
                       double sign_w, const double* a_c_in, double* a_c_out, double dt, cudaStream_t st,
                       double* ac_full_out, double* F_out, double* a_prev_out, const GuardView* guard) {
  int blocks = (cg.n_c + kSmallBlock - 1) / kSmallBlock;
  if (blocks > kMonBlocks) blocks = kMonBlocks;
  if (blocks < 1) blocks = 1;
  const GuardView gv = guard ? *guard : GuardView{nullptr, nullptr, nullptr, nullptr, 0};
  cond_update_kernel<<<blocks, kSmallBlock, 0, st>>>(dg.g, cg, ac_full, w, sign_w, a_c_in, a_c_out, dt, ac_full_out, F_out,
                                             a_prev_out, gv);
  return cudaGetLastError() == cudaSuccess ? MQS_OK : MQS_ERR_CUDA;
}

int launch_scatter_c(const CondGeom& cg, const double* a_c, double* ac_full, double scale, long long n3,
                     cudaStream_t st) {
  int blocks = (cg.n_c + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  scatter_c_kernel<<<blocks, 256, 0, st>>>(cg.n_c, cg.c_idx, a_c, ac_full, scale, n3);
  return cudaGetLastError() == cudaSuccess ? MQS_OK : MQS_ERR_CUDA;
}

MQS_DEBUG_TAKE(conductor)

}  // namespace mqs
