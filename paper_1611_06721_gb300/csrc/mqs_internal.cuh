// Internal device-side building blocks of the mqs library (sm_103a).
//
// Edge layout: component c of the edge with lower node (i, j, k) lives at
// c*n^3 + i + n*(j + n*k), 0 <= i, j, k < n ("position" (i, j, k)).
// Dirichlet edges with a node index 0 normal to the edge are stored as zero;
// those with node index n are not stored and read as zero.
//
// The curl-curl operator on nonconducting edges is K_n = (nu0/h) L with the
// integer stencil L = C_n^T C_n (every face touching an n-edge has reluctivity
// nu0; Sec. II, "typically constant" K_n).  L is applied through face fluxes:
//   bx(i,j,k) = y(i,j,k) + z(i,j+1,k) - y(i,j,k+1) - z(i,j,k)
//   by(i,j,k) = z(i,j,k) + x(i,j,k+1) - z(i+1,j,k) - x(i,j,k)
//   bz(i,j,k) = x(i,j,k) + y(i+1,j,k) - x(i,j+1,k) - y(i,j,k)
// and their transposed sums
//   (Lv)_x = bz(i,j,k) - bz(i,j-1,k) - by(i,j,k) + by(i,j,k-1)
//   (Lv)_y = bz(i-1,j,k) - bz(i,j,k) + bx(i,j,k) - bx(i,j,k-1)
//   (Lv)_z = bx(i,j-1,k) - bx(i,j,k) + by(i,j,k) - by(i-1,j,k)
// i.e. 6 FP64 additions per edge when every face flux is formed once.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/mqs.h"

namespace mqs {

constexpr int kTY = 8;                  // row warps per stencil block
constexpr int kWarps = kTY + 1;         // + one warp for the j0-1 halo row
constexpr int kBlock = 32 * kWarps;     // 288 threads
constexpr int kMaxSeg = 32;             // planes per segment (x halo: one per lane)

struct Box { int lo[3]; int hi[3]; };

struct Geom {
  int n;
  long long n3;
  int cb_lo[3], cb_hi[3];               // positions where c-edges may exist
  const uint8_t* cflags;                // bit c set: edge (c; pos) is a c-edge
};

__device__ __forceinline__ long long pidx(int n, int i, int j, int k) {
  return (long long)i + (long long)n * ((long long)j + (long long)n * k);
}

// bit c set iff edge (c; i, j, k) is an n-edge (interior and not conducting)
__device__ __forceinline__ unsigned nmask(const Geom& g, int i, int j, int k) {
  unsigned m = 0u;
  if (j > 0 && k > 0) m |= 1u;
  if (i > 0 && k > 0) m |= 2u;
  if (i > 0 && j > 0) m |= 4u;
  if (i >= g.cb_lo[0] && i < g.cb_hi[0] && j >= g.cb_lo[1] && j < g.cb_hi[1] &&
      k >= g.cb_lo[2] && k < g.cb_hi[2]) {
    int w0 = g.cb_hi[0] - g.cb_lo[0], w1 = g.cb_hi[1] - g.cb_lo[1];
    unsigned cf = g.cflags[(i - g.cb_lo[0]) + w0 * ((j - g.cb_lo[1]) + w1 * (k - g.cb_lo[2]))];
    m &= ~cf;
  }
  return m;
}

// component load with zero outside [0, n)
__device__ __forceinline__ double ld(const double* __restrict__ v, int n, long long n3, int c,
                                     int i, int j, int k) {
  if (i < 0 || j < 0 || k < 0 || i >= n || j >= n || k >= n) return 0.0;
  return v[c * n3 + pidx(n, i, j, k)];
}

struct SweepSmem {
  double fz[2][kWarps][32];
  double fx[2][kWarps][32];
};

// Face fluxes bz, by at (i, j, k) (used for the x halo).
__device__ __forceinline__ void flux_zy(const double* __restrict__ s, int n, long long n3, int i, int j,
                                        int k, double& bz, double& by) {
  double x0 = ld(s, n, n3, 0, i, j, k), y0 = ld(s, n, n3, 1, i, j, k), z0 = ld(s, n, n3, 2, i, j, k);
  double yi = ld(s, n, n3, 1, i + 1, j, k), zi = ld(s, n, n3, 2, i + 1, j, k);
  double xj = ld(s, n, n3, 0, i, j + 1, k), xk = ld(s, n, n3, 0, i, j, k + 1);
  bz = (x0 - y0) + (yi - xj);
  by = (z0 - x0) + (xk - zi);
}

// Face fluxes bz, bx at (i, j, k) (used for the y halo row).
__device__ __forceinline__ void flux_zx(const double* __restrict__ s, int n, long long n3, int i, int j,
                                        int k, double& bz, double& bx) {
  double x0 = ld(s, n, n3, 0, i, j, k), y0 = ld(s, n, n3, 1, i, j, k), z0 = ld(s, n, n3, 2, i, j, k);
  double yi = ld(s, n, n3, 1, i + 1, j, k), xj = ld(s, n, n3, 0, i, j + 1, k);
  double zj = ld(s, n, n3, 2, i, j + 1, k), yk = ld(s, n, n3, 1, i, j, k + 1);
  bz = (x0 - y0) + (yi - xj);
  bx = (y0 - z0) + (zj - yk);
}

// Applies t = L s over the positions of `box`, calling
//   epi(e, mask, tx, ty, tz, sx, sy, sz)
// once per position (e = i + n(j + n k); mask from nmask; t unmasked; s the
// source values at the position).  Work is split into plane-tiles of 32 x kTY
// positions; part `part` of `nparts` takes a contiguous range of them and
// marches each tile column along z so every face flux is formed once (plus
// one halo row, one halo column and one warm-up plane per segment).
// Must be called by all kBlock threads of the block.
template <class Epi>
__device__ void sweep_L(const Geom& g, const double* __restrict__ s, const Box& box, int part, int nparts,
                        SweepSmem& sm, Epi& epi) {
  const int n = g.n;
  const long long n3 = g.n3;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int bx0 = box.hi[0] - box.lo[0], by0 = box.hi[1] - box.lo[1], nz = box.hi[2] - box.lo[2];
  if (bx0 <= 0 || by0 <= 0 || nz <= 0) return;
  const int ntx = (bx0 + 31) / 32, nty = (by0 + kTY - 1) / kTY;
  const long long T = (long long)ntx * nty * nz;
  long long u = T * part / nparts;
  const long long u1 = T * (part + 1) / nparts;
  while (u < u1) {
    const long long tc = u / nz;
    const int ka = (int)(u % nz);
    int len = nz - ka;
    if ((long long)len > u1 - u) len = (int)(u1 - u);
    if (len > kMaxSeg) len = kMaxSeg;
    u += len;
    const int i0 = box.lo[0] + (int)(tc % ntx) * 32;
    const int j0 = box.lo[1] + (int)(tc / ntx) * kTY;
    const int ks = box.lo[2] + ka, ke = ks + len;
    const int i = i0 + lane;
    __syncthreads();  // smem reuse across segments
    if (w < kTY) {
      const int j = j0 + w;
      const bool act = (i < box.hi[0]) && (j < box.hi[1]);
      const bool col = (i < n) && (j < n);
      // x halo (i0 - 1, j, ks + lane) for the whole segment, one plane per lane
      double hz = 0.0, hy = 0.0;
      if (i0 >= 1 && j < n && lane < len) flux_zy(s, n, n3, i0 - 1, j, ks + lane, hz, hy);
      // own column values at plane ks - 1 (warm-up) or ks
      double x0 = 0.0, y0 = 0.0, z0 = 0.0, bxm = 0.0, bym = 0.0;
      int k = ks - 1;
      if (k >= 0 && col) {
        x0 = ld(s, n, n3, 0, i, j, k); y0 = ld(s, n, n3, 1, i, j, k); z0 = ld(s, n, n3, 2, i, j, k);
        double zi = ld(s, n, n3, 2, i + 1, j, k), zj = ld(s, n, n3, 2, i, j + 1, k);
        double xk = ld(s, n, n3, 0, i, j, k + 1), yk = ld(s, n, n3, 1, i, j, k + 1);
        bxm = (y0 - z0) + (zj - yk);
        bym = (z0 - x0) + (xk - zi);
      }
      if (col) { x0 = ld(s, n, n3, 0, i, j, ks); y0 = ld(s, n, n3, 1, i, j, ks); z0 = ld(s, n, n3, 2, i, j, ks); }
      int buf = 0;
      for (k = ks; k < ke; ++k) {
        double bx = 0.0, by = 0.0, bz = 0.0, xk = 0.0, yk = 0.0, zk = 0.0;
        if (col) {
          const double yi = ld(s, n, n3, 1, i + 1, j, k), zi = ld(s, n, n3, 2, i + 1, j, k);
          const double xj = ld(s, n, n3, 0, i, j + 1, k), zj = ld(s, n, n3, 2, i, j + 1, k);
          xk = ld(s, n, n3, 0, i, j, k + 1); yk = ld(s, n, n3, 1, i, j, k + 1); zk = ld(s, n, n3, 2, i, j, k + 1);
          bx = (y0 - z0) + (zj - yk);
          by = (z0 - x0) + (xk - zi);
          bz = (x0 - y0) + (yi - xj);
        }
        sm.fz[buf][w + 1][lane] = bz;
        sm.fx[buf][w + 1][lane] = bx;
        __syncthreads();
        double bzi = __shfl_up_sync(0xffffffffu, bz, 1), byi = __shfl_up_sync(0xffffffffu, by, 1);
        const double hzk = __shfl_sync(0xffffffffu, hz, k - ks), hyk = __shfl_sync(0xffffffffu, hy, k - ks);
        if (lane == 0) { bzi = hzk; byi = hyk; }
        const double bzj = sm.fz[buf][w][lane], bxj = sm.fx[buf][w][lane];
        if (act) {
          const double tx = (bz - bzj) + (bym - by);
          const double ty = (bzi - bz) + (bx - bxm);
          const double tz = (bxj - bx) + (by - byi);
          epi(pidx(n, i, j, k), nmask(g, i, j, k), tx, ty, tz, x0, y0, z0);
        }
        bxm = bx; bym = by;
        x0 = xk; y0 = yk; z0 = zk;
        buf ^= 1;
      }
    } else {
      // halo row j0 - 1: bz and bx of every plane of the segment
      const int jh = j0 - 1;
      int buf = 0;
      for (int k = ks; k < ke; ++k) {
        double bz = 0.0, bx = 0.0;
        if (jh >= 0 && i < n) flux_zx(s, n, n3, i, jh, k, bz, bx);
        sm.fz[buf][0][lane] = bz;
        sm.fx[buf][0][lane] = bx;
        __syncthreads();
        buf ^= 1;
      }
    }
  }
}

// ---- reductions --------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum of NV values per thread; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red /* >= NV*32 doubles */) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int a = 0; a < NV; ++a) v[a] = warp_sum(v[a]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) red[a * 32 + w] = v[a];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      double s = 0.0;
      for (int q = 0; q < nw; ++q) s += red[a * 32 + q];
      v[a] = s;
    }
  }
  __syncthreads();
}

// Sum of part[0..cnt) computed identically by every caller (one warp).
__device__ __forceinline__ double fixed_sum(const double* part, int cnt) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int q = lane; q < cnt; q += 32) s += part[q];
  return warp_sum(s);
}

// ---- grid barrier with a bounded wait -------------------------------------------
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// All blocks of a co-resident grid meet here; `target` = gridDim.x * (number
// of barriers passed so far, this one included).  A wait longer than `spin`
// polls records MQS_ERR_TIMEOUT in *err and returns false.
__device__ __forceinline__ bool grid_barrier(unsigned* ctr, unsigned target, long long spin, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    red_release_add(ctr, 1u);
    long long polls = 0;
    while (ld_acquire(ctr) < target) {
      if (++polls > spin) { atomicExch(err, MQS_ERR_TIMEOUT); ok = 0; break; }
      __nanosleep(20);
    }
    __threadfence();
    if (ok && *((volatile int*)err) != 0) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace mqs
