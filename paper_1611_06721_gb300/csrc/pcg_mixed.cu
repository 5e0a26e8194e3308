// Mixed-precision solve of K_n x = b: FP64 iterative refinement around FP32
// conjugate-gradient inner solves, as one persistent cooperative kernel.
//
// Outer (FP64): r = b - L x by the FP64 stencil (which also yields L x for the
// start-vector history), ||r||, convergence test ||r|| <= tol ||b||, and the
// update x += ||r|| d.  Inner (FP32): CG on L d = r/||r|| with the stencil,
// vectors and products in FP32 (on this GPU FP32 arithmetic is 64x faster
// than FP64), each dot product's per-thread partial sums in FP32 and its
// cross-thread sum and the CG scalars in float-float; it stops once its residual has dropped by
// max(inner_tol, tol ||b|| / (2 ||r||)), i.e. as soon as the outer tolerance
// can be met, or when FP32 stagnates.  Jacobi is folded into the scaling as
// in the FP64 kernel (diag(K_n) is uniform).
#include <cmath>
#include "mqs_internal.cuh"
#include "mqs_kernels.h"
#include "pcg_fused.cuh"

namespace mqs {

struct MixedArgs {
  Geom g;
  Box full;
  const double* b;
  double* x;
  double* r;
  double* lx;
  float* r32;
  float* p32;
  float* q32;
  float* d32;
  float* r32b;          // variant 1: second r buffer, w = L r and s = L p (both double-buffered)
  float* w32a;
  float* w32b;
  float* s32a;
  float* s32b;
  int variant;          // inner CG: 0 two reductions per iteration, 1 one reduction (Chronopoulos-Gear)
  double* part;
  unsigned* bar;
  int* err;
  PcgResult* out;
  int* refinements;     // number of FP64 residual evaluations after the first
  double tol2;
  double inner_tol;
  int maxit;            // cap on the total inner iterations
  long long spin;
  int init;             // as in the FP64 kernel: 0 stencil, 2 zero start
  const int* halt;      // nullable: nonzero = an earlier step of the stepping call failed, skip the solve
  const int2* ptab;     // nullable: part ranges of the one-reduction pass (fused_partition)
};

// as in the FP64 kernel: a halted stepping call skips the solve (zero iterations)
__device__ __forceinline__ bool mixed_halted(const MixedArgs& a) {
  if (!a.halt || *(volatile const int*)a.halt == 0) return false;
  if (blockIdx.x == 0 && threadIdx.x == 0) { *a.out = PcgResult{0, MQS_OK, 0.0, 0.0}; *a.refinements = 0; }
  return true;
}

struct EpiResidualM {   // r = b - t, lx = t on n-edges; sums r.r and b.b (FP64)
  const double* b; double* r; double* lx; long long n3;
  double rr = 0.0, bb = 0.0;
  double bp[3];
  __device__ void prefetch(long long e) {
#pragma unroll
    for (int c = 0; c < 3; ++c) bp[c] = b[e + c * n3];
  }
  __device__ void operator()(long long e, unsigned m, double tx, double ty, double tz, double, double, double) {
    const double t[3] = {tx, ty, tz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long idx = e + c * n3;
      if (m >> c & 1u) {
        const double bv = bp[c];
        const double rv = bv - t[c];
        r[idx] = rv; lx[idx] = t[c];
        rr = fma(rv, rv, rr); bb = fma(bv, bv, bb);
      } else {
        r[idx] = 0.0; lx[idx] = 0.0;
      }
    }
  }
};

struct EpiDirection32 {  // q = t + beta q, p = r + beta p on n-edges (FP32); sums p.q
  float* p; float* q; long long n3; float beta; bool first;
  float pq = 0.f;
  float pp[3], qp[3];
  __device__ void prefetch(long long e) {
    if (first) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) { pp[c] = p[e + c * n3]; qp[c] = q[e + c * n3]; }
  }
  __device__ void operator()(long long e, unsigned m, float tx, float ty, float tz, float sx, float sy, float sz) {
    const float t[3] = {tx, ty, tz}, s[3] = {sx, sy, sz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long idx = e + c * n3;
      float qn = 0.f, pn = 0.f;
      if (m >> c & 1u) {
        qn = first ? t[c] : fmaf(beta, qp[c], t[c]);
        pn = first ? s[c] : fmaf(beta, pp[c], s[c]);
        pq = fmaf(pn, qn, pq);
      }
      q[idx] = qn; p[idx] = pn;
    }
  }
};

struct EpiApplyDot32 {  // w = t on n-edges (0 elsewhere, FP32); sums w.r with r the source values
  float* w; long long n3;
  float wr = 0.f;
  __device__ void prefetch(long long) {}
  __device__ void operator()(long long e, unsigned m, float tx, float ty, float tz, float sx, float sy, float sz) {
    const float t[3] = {tx, ty, tz}, s[3] = {sx, sy, sz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float wv = (m >> c & 1u) ? t[c] : 0.f;
      w[e + c * n3] = wv;
      wr = fmaf(wv, s[c], wr);
    }
  }
};

// ---- the FP32 inner pass that carries x, r and p only (pcg_variant 2) -------------
// Chronopoulos-Gear CG with s = L p and w = L r formed in the pass instead of stored:
//   p_i = r_i + beta p_{i-1},  s_i = L p_i,  x += alpha p_i,  r_{i+1} = r_i - alpha s_i,
//   w_{i+1} = L r_{i+1},  gamma = r_{i+1}.r_{i+1},  delta = r_{i+1}.w_{i+1}
// (s_i = w_i + beta s_{i-1} = L p_i by linearity: the same iterates in exact arithmetic as
// the fused pass).  A pass reads r_i and p_{i-1} (with a two-deep halo) and x, and writes
// p_i, r_{i+1} and x: 24 B per unknown in FP32, the three carried vectors once each way,
// against 40 B when s and w are stored.  A block (kWarps warps) owns a tile of kCgTX x
// kCgTY positions and covers the 32 x kWarps region around it: warp w is region row
// j0 - 2 + w, lane l region column i0 - 2 + l.  Marching along z, step k forms p(k+1)
// (whole region), the fluxes of p at plane k, s(k) and r_{i+1}(k) (one-deep region), the
// fluxes of r_{i+1} at plane k-1 and w(k-1) (owned tile), and writes the owned outputs of
// plane k-1.  Each thread stages its own column's r and p_{i-1} kCgAhead planes ahead with
// cp.async (zero-filled outside the grid; only the thread reads them back, so the ring
// needs no barrier); rows are exchanged through double-buffered shared memory with two
// block barriers per step.  A segment starts 2 planes early: the owned output of plane m
// needs r_{i+1} at m-1..m+1, hence s there, hence the fluxes of p from plane m-2 on.
constexpr int kCgTX = 28, kCgTY = kWarps - 4;
constexpr int kCgAhead = 6, kCgRing = kCgAhead + 1;
struct Cg24Smem {
  float stage[kCgRing][6][kBlock];          // per thread, per plane slot: r (3 comps), p_{i-1} (3)
  // row exchange, [parity][comp][row + 1][lane]: rows -1 and kWarps stay zero (pads)
  float p[2][2][kWarps + 2][32];            // p x, z comps by row (read by the row below)
  float pf[2][2][kWarps + 2][32];           // p fluxes bz, bx by row (read by the row above)
  float r1[2][2][kWarps + 2][32];           // r_{i+1} x, z comps
  float rf[2][2][kWarps + 2][32];           // r_{i+1} fluxes bz, bx
};
static_assert(sizeof(Cg24Smem) == sizeof(float) * (kCgRing * 6 * kBlock + 4 * 2 * 2 * (kWarps + 2) * 32),
              "the exchange buffers are contiguous (zeroed as one range)");
struct Cg24Vecs {
  const float* r_in;
  const float* p_in;
  float* r_out;
  float* p_out;
  float* x;
  float alpha, beta;
  bool first;
};

__device__ __forceinline__ void cp_async4(unsigned sdst, const float* gsrc, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sdst), "l"(gsrc), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ float shfl_dn1f(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_up1f(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }

__device__ void sweep_cg24(const Geom& g, const Cg24Vecs& v, const Box& box, int part, int nparts, Cg24Smem& sm,
                           float& gamma, float& delta) {
  const int n = g.n, n2 = n * n, n3 = (int)g.n3;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, t = threadIdx.x;
  const int bx0 = box.hi[0] - box.lo[0], by0 = box.hi[1] - box.lo[1], nz = box.hi[2] - box.lo[2];
  if (bx0 <= 0 || by0 <= 0 || nz <= 0) return;
  const int ntx = (bx0 + kCgTX - 1) / kCgTX, nty = (by0 + kCgTY - 1) / kCgTY;
  const long long ntiles = (long long)ntx * nty * nz;
  long long u = ntiles * part / nparts;
  const long long u1 = ntiles * (part + 1) / nparts;
  const int cw0 = g.cb_hi[0] - g.cb_lo[0], cw01 = cw0 * (g.cb_hi[1] - g.cb_lo[1]);
  const float al = v.alpha, be = v.beta;
  constexpr int kComp = (kWarps + 2) * 32;                // component stride of an exchange buffer
  constexpr int kPar = 2 * kComp;                         // parity stride
  // this thread's exchange addresses (parity 0; parity 1 at + kPar): own row, the row below
  // (j + 1) and the row above (j - 1)
  const int ow = (w + 1) * 32 + lane;
  float* const xp = &sm.p[0][0][0][0] + ow;
  float* const xpf = &sm.pf[0][0][0][0] + ow;
  float* const xr1 = &sm.r1[0][0][0][0] + ow;
  float* const xrf = &sm.rf[0][0][0][0] + ow;
  const unsigned stage0 = (unsigned)__cvta_generic_to_shared(&sm.stage[0][0][t]);
  constexpr unsigned kSlotBytes = 6u * kBlock * 4u, kCompBytes = kBlock * 4u;
  while (u < u1) {
    const long long tc = u / nz;
    const int ka = (int)(u % nz);
    int len = nz - ka;
    if ((long long)len > u1 - u) len = (int)(u1 - u);
    u += len;
    const int i0 = box.lo[0] + (int)(tc % ntx) * kCgTX;
    const int j0 = box.lo[1] + (int)(tc / ntx) * kCgTY;
    const int ks = box.lo[2] + ka, ke = ks + len;
    const int i = i0 - 2 + lane, j = j0 - 2 + w;        // this thread's region column
    const bool col = i >= 0 && i < n && j >= 0 && j < n;
    const int oc = col ? i + n * j : 0;                   // in-plane offset
    const bool own = lane >= 2 && lane < 2 + kCgTX && w >= 2 && w < 2 + kCgTY && i < box.hi[0] && j < box.hi[1];
    const unsigned mcol = (j > 0 ? 1u : 0u) | (i > 0 ? 2u : 0u) | ((i > 0 && j > 0) ? 4u : 0u);
    const bool incb = col && i >= g.cb_lo[0] && i < g.cb_hi[0] && j >= g.cb_lo[1] && j < g.cb_hi[1];
    const uint8_t* const cfcol = incb ? g.cflags + (i - g.cb_lo[0]) + cw0 * (j - g.cb_lo[1]) : g.cflags;
    // conductor flags of plane k (c-edges are not n-edges)
    auto cflag = [&](int k) -> unsigned {
      return (incb && k >= g.cb_lo[2] && k < g.cb_hi[2])
                 ? (unsigned)MQS_LDC(cfcol, cw01 * (k - g.cb_lo[2]),
                                     (long long)cw01 * (g.cb_hi[2] - g.cb_lo[2]) - (cfcol - g.cflags), 801)
                 : 0u;
    };
    const int kb = ks - 2;                               // first step (warm-up of the lag)
    // the staging ring: plane sm_ of slot ss_ is the next to issue
    int st_m = kb, st_slot = 0;
    auto stage_next = [&]() {
      const bool ok = col && st_m >= 0 && st_m < n && st_m <= ke + 1;
      const bool okp = ok && !v.first;
      const int off = ok ? oc + n2 * st_m : 0;
      const unsigned sa = stage0 + (unsigned)st_slot * kSlotBytes;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const bool okc = ok && MQS_IDX_OK(off + c * n3, 3 * n3, 802);   // zero-fill when out of range
        cp_async4(sa + c * kCompBytes, v.r_in + (okc ? off + c * n3 : 0), okc ? 4 : 0);
        cp_async4(sa + (3 + c) * kCompBytes, v.p_in + (okp && okc ? off + c * n3 : 0), okp && okc ? 4 : 0);
      }
      cp_async_commit();
      ++st_m;
      st_slot = (st_slot + 1 == kCgRing) ? 0 : st_slot + 1;
    };
    __syncthreads();                                     // shared memory reuse across segments
    {
      // the row exchange buffers (and their pad rows) start at zero
      float* ex = &sm.p[0][0][0][0];
      constexpr int kEx = 4 * 2 * 2 * (kWarps + 2) * 32;
      for (int q = t; q < kEx; q += kBlock) ex[q] = 0.f;
    }
    for (int q = 0; q <= kCgAhead; ++q) stage_next();   // planes kb .. kb + kCgAhead
    cp_async_wait<kCgAhead>();                           // plane kb
    __syncthreads();
    int rd_slot = 0;                                     // slot of the next plane to read
    float rk[3], pk[3];
    {
      const float* st = &sm.stage[rd_slot][0][t];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        rk[c] = st[c * kBlock];
        pk[c] = v.first ? rk[c] : fmaf(be, st[(3 + c) * kBlock], rk[c]);
      }
      rd_slot = (rd_slot + 1 == kCgRing) ? 0 : rd_slot + 1;
    }
    {
      const int par = kb & 1;
      xp[par * kPar] = pk[0];
      xp[par * kPar + kComp] = pk[2];
    }
    float pm1[3] = {0.f, 0.f, 0.f}, r1m1[3] = {0.f, 0.f, 0.f};
    float pbx_m1 = 0.f, pby_m1 = 0.f, rbx_m2 = 0.f, rby_m2 = 0.f;
    float xk[3] = {0.f, 0.f, 0.f};       // x of the plane the next output needs (loaded a step ahead)
    unsigned cf_k = cflag(kb);
    int ok_off = oc + n2 * kb;           // in-layout offset of plane k of this column
    __syncthreads();
    for (int k = kb; k <= ke; ++k, ok_off += n2) {
      const int par = k & 1, nq = par ^ 1;
      // plane k+1 staged; its slot is then free for plane k + 1 + kCgAhead
      cp_async_wait<kCgAhead - 1>();
      float rk1[3], pk1[3];
      {
        const float* st = &sm.stage[rd_slot][0][t];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          rk1[c] = st[c * kBlock];
          pk1[c] = v.first ? rk1[c] : fmaf(be, st[(3 + c) * kBlock], rk1[c]);
        }
        rd_slot = (rd_slot + 1 == kCgRing) ? 0 : rd_slot + 1;
      }
      stage_next();
      const unsigned cf_k1 = cflag(k + 1);               // for the next step
      float xn[3] = {0.f, 0.f, 0.f};                     // x of plane k (the next step's output)
      if (own && k >= ks && k < ke) {
#pragma unroll
        for (int c = 0; c < 3; ++c) xn[c] = MQS_LDC(v.x, ok_off + c * n3, 3 * n3, 803);
      }
      // p(k+1) rows for the next step; fluxes of p at plane k
      xp[nq * kPar] = pk1[0];
      xp[nq * kPar + kComp] = pk1[2];
      const float pxj = xp[par * kPar + 32], pzj = xp[par * kPar + kComp + 32];
      const float pyi = shfl_dn1f(pk[1]), pzi = shfl_dn1f(pk[2]);
      const float bx = (pk[1] - pk[2]) + (pzj - pk1[1]);
      const float by = (pk[2] - pk[0]) + (pk1[0] - pzi);
      const float bz = (pk[0] - pk[1]) + (pyi - pxj);
      xpf[par * kPar] = bz;
      xpf[par * kPar + kComp] = bx;
      __syncthreads();
      // s(k) = L p and r_{i+1}(k) = r(k) - alpha s(k) on n-edges
      float r1k[3];
      {
        const float bzj = xpf[par * kPar - 32], bxj = xpf[par * kPar + kComp - 32];
        const float bzi = shfl_up1f(bz), byi = shfl_up1f(by);
        const float sx = (bz - bzj) + (pby_m1 - by);
        const float sy = (bzi - bz) + (bx - pbx_m1);
        const float sz = (bxj - bx) + (by - byi);
        pbx_m1 = bx; pby_m1 = by;
        const unsigned m = (col && k >= 0 && k < n) ? (mcol & (k > 0 ? 7u : 4u) & ~cf_k) : 0u;
        r1k[0] = (m & 1u) ? fmaf(-al, sx, rk[0]) : 0.f;
        r1k[1] = (m & 2u) ? fmaf(-al, sy, rk[1]) : 0.f;
        r1k[2] = (m & 4u) ? fmaf(-al, sz, rk[2]) : 0.f;
      }
      xr1[par * kPar] = r1k[0];
      xr1[par * kPar + kComp] = r1k[2];
      // fluxes of r_{i+1} at plane k-1 (its rows of the row below were written last step)
      const float rxj = xr1[nq * kPar + 32], rzj = xr1[nq * kPar + kComp + 32];
      const float ryi = shfl_dn1f(r1m1[1]), rzi = shfl_dn1f(r1m1[2]);
      const float cx = (r1m1[1] - r1m1[2]) + (rzj - r1k[1]);
      const float cy = (r1m1[2] - r1m1[0]) + (r1k[0] - rzi);
      const float cz = (r1m1[0] - r1m1[1]) + (ryi - rxj);
      xrf[par * kPar] = cz;
      xrf[par * kPar + kComp] = cx;
      __syncthreads();
      // w(k-1) = L r_{i+1} and the owned outputs of plane k-1
      {
        const float czj = xrf[par * kPar - 32], cxj = xrf[par * kPar + kComp - 32];
        const float czi = shfl_up1f(cz), cyi = shfl_up1f(cy);
        const float wv[3] = {(cz - czj) + (rby_m2 - cy), (czi - cz) + (cx - rbx_m2), (cxj - cx) + (cy - cyi)};
        rbx_m2 = cx; rby_m2 = cy;
        if (own && k - 1 >= ks && k - 1 < ke) {
          const int o = ok_off - n2;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            MQS_STC(v.p_out, o + c * n3, 3 * n3, 804, pm1[c]);
            MQS_STC(v.r_out, o + c * n3, 3 * n3, 805, r1m1[c]);
            MQS_STC(v.x, o + c * n3, 3 * n3, 806, fmaf(al, pm1[c], xk[c]));
            gamma = fmaf(r1m1[c], r1m1[c], gamma);
            delta = fmaf(r1m1[c], wv[c], delta);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pm1[c] = pk[c]; pk[c] = pk1[c]; rk[c] = rk1[c]; r1m1[c] = r1k[c];
        xk[c] = xn[c];
      }
      cf_k = cf_k1;
    }
    cp_async_wait<0>();
  }
}

// shared memory of pcg_mixed_kernel, dynamic (the staging ring of sweep_cg24 exceeds the
// 48 KB of static shared memory)
union MixedSmem {
  SweepSmemT<double> d;
  SweepSmemT<float> f;
  FusedSmemBlockT<float> ff;
  Cg24Smem cg;
};

// BPS co-resident blocks per SM: 2 once the FP32 vectors are far beyond L2 (the inner
// sweep is then bound by memory latency and plane syncs, and 20 warps per SM hide more
// of both than 10; the register cap of 96 spills a little, in the FP64 passes), else 1.
// HW: halo warps per group of the one-reduction inner pass (2: kGroups more warps at the
// end of the block, which sit out every other sweep and the elementwise loops, so that
// the iterates are bitwise those of HW = 1; launched only with pcg_variant 1).
template <int BPS, int HW = 1>
__global__ void __launch_bounds__(32 * (kGroupWarps + HW - 1) * kGroups, BPS) pcg_mixed_kernel(MixedArgs a) {
  if (mixed_halted(a)) return;
  if (HW == 2 && a.variant != 1) return;   // not launched so (launch_pcg_mixed)
  extern __shared__ __align__(16) unsigned char mixed_dyn[];
  MixedSmem& sm = *reinterpret_cast<MixedSmem*>(mixed_dyn);
  __shared__ double red[32];
  __shared__ double gs[2];
  const int nb = gridDim.x, bid = blockIdx.x;
  unsigned nbar = 0;
  int slot = 0;
  const long long len = 3 * a.g.n3;
  const bool in_groups = HW == 1 || threadIdx.x < kBlock;
  const int gth = HW == 1 ? (int)blockDim.x : kBlock;
  const long long tid = in_groups ? (long long)bid * gth + threadIdx.x : len, nth = (long long)nb * gth;
  auto reduce2 = [&](double v0, double v1, double& s0, double& s1) -> bool {
    return grid_sum2<double>(v0, v1, s0, s1, a.part, slot, nbar, a.bar, a.spin, a.err, red, gs);
  };
  // float-float sums (the inner solves' products): the same partial slots and barrier sequence
  auto reduceF = [&](ffv v0, ffv v1, ffv& s0, ffv& s1) -> bool {
    return grid_sum2<ffv>(v0, v1, s0, s1, a.part, slot, nbar, a.bar, a.spin, a.err, reinterpret_cast<ffv*>(red),
                          reinterpret_cast<ffv*>(gs));
  };
  int status = MQS_OK, inner_total = 0, outer = 0;
  double bb = 0.0, start_rel = 0.0, relres = 0.0;
  if (a.init == 2) {
    for (long long e = tid; e < len; e += nth) a.x[e] = 0.0;
    double d0, d1;
    if (!reduce2(0.0, 0.0, d0, d1)) return;   // x visible before the first residual
  }
  for (;;) {
    // FP64 residual r = b - L x, its norm and L x
    double rr;
    {
      EpiResidualM ep{a.b, a.r, a.lx, a.g.n3};
      if (in_groups) sweep_L<double>(a.g, a.x, a.full, bid, nb, sm.d, ep);
      if (!reduce2(ep.rr, ep.bb, rr, bb)) return;
    }
    if (outer == 0) {
      if (bb == 0.0) {
        for (long long e = tid; e < len; e += nth) { a.x[e] = 0.0; a.r[e] = 0.0; a.lx[e] = 0.0; }
        if (bid == 0 && threadIdx.x == 0) { *a.out = PcgResult{0, MQS_OK, 0.0, 0.0}; *a.refinements = 0; }
        return;
      }
      start_rel = sqrt(rr / bb);
    }
    relres = sqrt(rr / bb);
    if (!isfinite(rr) || !isfinite(bb)) { status = MQS_ERR_NAN; break; }
    if (rr <= a.tol2 * bb) { status = MQS_OK; break; }
    if (inner_total >= a.maxit || outer >= 64) { status = MQS_ERR_NOT_CONVERGED; break; }
    // inner FP32 CG on L d = r / ||r||
    const double nr = sqrt(rr), inv = 1.0 / nr;
    ffv rho;
    {
      float acc = 0.f;
      for (long long e = tid; e < len; e += nth) {
        const float v = (float)(a.r[e] * inv);
        a.r32[e] = v;
        a.d32[e] = 0.f;
        acc = fmaf(v, v, acc);
      }
      ffv dummy;
      if (!reduceF(ffv(acc, 0.f), ffv(0), rho, dummy)) return;
    }
    // the inner scalars (products, alpha, beta) are float-float: FP64 division
    // and conversions are long dependent sequences on this GPU
    const double target = fmax(a.inner_tol, 0.5 * sqrt(a.tol2 * bb) / nr);
    const ffv stop2 = ff_from(target * target * ff_to(rho));
    float beta = 0.f;
    bool first = true;
    int it_in = 0;
    if (a.variant == 1) {
      // one reduction per inner iteration: w = L r once, then fused passes
      // (p, s, d, r updates + w = L r_new + gamma, delta) with r, w, s double-buffered
      auto rbuf = [&](int c) { return c ? a.r32b : a.r32; };
      auto wbuf = [&](int c) { return c ? a.w32b : a.w32a; };
      auto sbuf = [&](int c) { return c ? a.s32b : a.s32a; };
      int cur = 0;
      ffv delta, dummy;
      {
        EpiApplyDot32 ep{wbuf(0), a.g.n3};
        if (in_groups) sweep_L<float>(a.g, rbuf(0), a.full, bid, nb, sm.f, ep);
        if (!reduceF(ffv(ep.wr, 0.f), ffv(0), delta, dummy)) return;
      }
      ffv gamma = rho;
      bool ok = delta.hi > 0.f;
      ffv alpha = ok ? ff_div(gamma, delta) : ffv(0), bet = ffv(0);
      while (ok && inner_total < a.maxit) {
        FusedVecsT<float> v{a.d32, a.p32, rbuf(cur), wbuf(cur), sbuf(cur), rbuf(cur ^ 1), wbuf(cur ^ 1),
                            sbuf(cur ^ 1), alpha.hi, bet.hi, first};
        float g1 = 0.f, d1 = 0.f;
        sweep_fused<float, HW>(a.g, v, a.full, bid, nb, sm.ff, g1, d1, a.ptab);
        ffv gn, dn;
        if (!reduceF(ffv(g1, 0.f), ffv(d1, 0.f), gn, dn)) return;
        ++it_in; ++inner_total;
        cur ^= 1;
        if (!isfinite(gn.hi) || !isfinite(dn.hi)) break;
        if (ff_le(gn, stop2) || it_in >= 400) break;
        const ffv bnew = ff_div(gn, gamma);
        const ffv den = dn - ff_div(ff_mul(bnew, gn), alpha);
        if (!(den.hi > 0.f)) break;               // FP32 breakdown / stagnation: refine from here
        bet = bnew; alpha = ff_div(gn, den); gamma = gn;
        first = false;
      }
    }
    if (a.variant == 2) {
      // one reduction per inner iteration, x, r and p carried (r, p double-buffered);
      // delta = r.L r once for the first alpha (w into w32a, scratch)
      auto rbuf = [&](int c) { return c ? a.r32b : a.r32; };
      auto pbuf = [&](int c) { return c ? a.s32a : a.p32; };
      int cur = 0;
      ffv delta, dummy;
      {
        EpiApplyDot32 ep{a.w32a, a.g.n3};
        if (in_groups) sweep_L<float>(a.g, rbuf(0), a.full, bid, nb, sm.f, ep);
        if (!reduceF(ffv(ep.wr, 0.f), ffv(0), delta, dummy)) return;
      }
      ffv gamma = rho;
      bool ok = delta.hi > 0.f;
      ffv alpha = ok ? ff_div(gamma, delta) : ffv(0), bet = ffv(0);
      while (ok && inner_total < a.maxit) {
        const Cg24Vecs v{rbuf(cur), pbuf(cur), rbuf(cur ^ 1), pbuf(cur ^ 1), a.d32, alpha.hi, bet.hi, first};
        float g1 = 0.f, d1 = 0.f;
        sweep_cg24(a.g, v, a.full, bid, nb, sm.cg, g1, d1);
        ffv gn, dn;
        if (!reduceF(ffv(g1, 0.f), ffv(d1, 0.f), gn, dn)) return;
        ++it_in; ++inner_total;
        cur ^= 1;
        if (!isfinite(gn.hi) || !isfinite(dn.hi)) break;
        if (ff_le(gn, stop2) || it_in >= 400) break;
        const ffv bnew = ff_div(gn, gamma);
        const ffv den = dn - ff_div(ff_mul(bnew, gn), alpha);
        if (!(den.hi > 0.f)) break;               // FP32 breakdown / stagnation: refine from here
        bet = bnew; alpha = ff_div(gn, den); gamma = gn;
        first = false;
      }
    }
    while (a.variant == 0 && inner_total < a.maxit) {
      ffv pq, dummy;
      {
        EpiDirection32 ep{a.p32, a.q32, a.g.n3, beta, first};
        if (in_groups) sweep_L<float>(a.g, a.r32, a.full, bid, nb, sm.f, ep);
        if (!reduceF(ffv(ep.pq, 0.f), ffv(0), pq, dummy)) return;
      }
      ++it_in; ++inner_total;
      if (!(pq.hi > 0.f)) break;                  // FP32 breakdown / stagnation: refine from here
      const float alpha = ff_div(rho, pq).hi;
      ffv rn;
      {
        float acc = 0.f;
        const long long q4 = len >> 2;
        float4* d4 = reinterpret_cast<float4*>(a.d32);
        float4* r4 = reinterpret_cast<float4*>(a.r32);
        const float4* p4 = reinterpret_cast<const float4*>(a.p32);
        const float4* qq4 = reinterpret_cast<const float4*>(a.q32);
        for (long long e = tid; e < q4; e += nth) {
          const float4 pv = p4[e], qv = qq4[e];
          float4 dv = d4[e], rv = r4[e];
          dv.x = fmaf(alpha, pv.x, dv.x); dv.y = fmaf(alpha, pv.y, dv.y);
          dv.z = fmaf(alpha, pv.z, dv.z); dv.w = fmaf(alpha, pv.w, dv.w);
          rv.x = fmaf(-alpha, qv.x, rv.x); rv.y = fmaf(-alpha, qv.y, rv.y);
          rv.z = fmaf(-alpha, qv.z, rv.z); rv.w = fmaf(-alpha, qv.w, rv.w);
          d4[e] = dv; r4[e] = rv;
          acc = fmaf(rv.x, rv.x, acc); acc = fmaf(rv.y, rv.y, acc);
          acc = fmaf(rv.z, rv.z, acc); acc = fmaf(rv.w, rv.w, acc);
        }
        for (long long e = (q4 << 2) + tid; e < len; e += nth) {
          a.d32[e] = fmaf(alpha, a.p32[e], a.d32[e]);
          const float rv = fmaf(-alpha, a.q32[e], a.r32[e]);
          a.r32[e] = rv;
          acc = fmaf(rv, rv, acc);
        }
        if (!reduceF(ffv(acc, 0.f), ffv(0), rn, dummy)) return;
      }
      if (!isfinite(rn.hi)) break;
      if (ff_le(rn, stop2) || it_in >= 400) break;
      beta = ff_div(rn, rho).hi;
      rho = rn;
      first = false;
    }
    // x += ||r|| d (FP64); barrier so the next residual sees every update
    {
      for (long long e = tid; e < len; e += nth) a.x[e] = fma(nr, (double)a.d32[e], a.x[e]);
      double d0, d1;
      if (!reduce2(0.0, 0.0, d0, d1)) return;
    }
    ++outer;
  }
  if (bid == 0 && threadIdx.x == 0) {
    *a.out = PcgResult{inner_total, status, relres, start_rel};
    *a.refinements = outer;
  }
}

// ---- precision 2: float-float inner CG in FP64 refinement ----------------------------
// The outer loop is the one above (FP64 residual, norm, convergence test and update);
// the inner solves run the one-reduction CG in float-float arithmetic (about 48 bits,
// FP32 pipes), so they converge like FP64 CG and usually meet the outer tolerance in
// one refinement, at the FP32 cost of the arithmetic.

struct EpiApplyDotFF {  // w = t on n-edges (0 elsewhere); sums w.r with r the source values
  ffv* w; long long n3;
  ffv wr = ffv(0);
  __device__ void prefetch(long long) {}
  __device__ void operator()(long long e, unsigned m, ffv tx, ffv ty, ffv tz, ffv sx, ffv sy, ffv sz) {
    const ffv t[3] = {tx, ty, tz}, s[3] = {sx, sy, sz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const ffv wv = (m >> c & 1u) ? t[c] : ffv(0);
      w[e + c * n3] = wv;
      wr = fmaT(wv, s[c], wr);
    }
  }
};

__global__ void __launch_bounds__(kBlock, kPcgBlocksPerSM) pcg_ff_kernel(MixedArgs a) {
  if (mixed_halted(a)) return;
  __shared__ union { SweepSmemT<double> d; SweepSmemT<ffv> f; FusedSmemBlockT<ffv> ff; } sm;
  __shared__ double red[32];
  __shared__ double gs[2];
  const int nb = gridDim.x, bid = blockIdx.x;
  unsigned nbar = 0;
  int slot = 0;
  const long long len = 3 * a.g.n3;
  const long long tid = (long long)bid * blockDim.x + threadIdx.x, nth = (long long)nb * blockDim.x;
  auto reduce2 = [&](double v0, double v1, double& s0, double& s1) -> bool {
    return grid_sum2<double>(v0, v1, s0, s1, a.part, slot, nbar, a.bar, a.spin, a.err, red, gs);
  };
  // float-float sums (the inner solves' products): the same partial slots and barrier sequence
  auto reduceF = [&](ffv v0, ffv v1, ffv& s0, ffv& s1) -> bool {
    return grid_sum2<ffv>(v0, v1, s0, s1, a.part, slot, nbar, a.bar, a.spin, a.err, reinterpret_cast<ffv*>(red),
                          reinterpret_cast<ffv*>(gs));
  };
  ffv* const rb0 = reinterpret_cast<ffv*>(a.r32);
  ffv* const rb1 = reinterpret_cast<ffv*>(a.r32b);
  ffv* const wb0 = reinterpret_cast<ffv*>(a.w32a);
  ffv* const wb1 = reinterpret_cast<ffv*>(a.w32b);
  ffv* const sb0 = reinterpret_cast<ffv*>(a.s32a);
  ffv* const sb1 = reinterpret_cast<ffv*>(a.s32b);
  ffv* const pf = reinterpret_cast<ffv*>(a.p32);
  ffv* const df = reinterpret_cast<ffv*>(a.d32);
  auto rbuf = [&](int c) { return c ? rb1 : rb0; };
  auto wbuf = [&](int c) { return c ? wb1 : wb0; };
  auto sbuf = [&](int c) { return c ? sb1 : sb0; };
  int status = MQS_OK, inner_total = 0, outer = 0;
  double bb = 0.0, start_rel = 0.0, relres = 0.0;
  if (a.init == 2) {
    for (long long e = tid; e < len; e += nth) a.x[e] = 0.0;
    double d0, d1;
    if (!reduce2(0.0, 0.0, d0, d1)) return;
  }
  for (;;) {
    double rr;
    {
      EpiResidualM ep{a.b, a.r, a.lx, a.g.n3};
      sweep_L<double>(a.g, a.x, a.full, bid, nb, sm.d, ep);
      if (!reduce2(ep.rr, ep.bb, rr, bb)) return;
    }
    if (outer == 0) {
      if (bb == 0.0) {
        for (long long e = tid; e < len; e += nth) { a.x[e] = 0.0; a.r[e] = 0.0; a.lx[e] = 0.0; }
        if (bid == 0 && threadIdx.x == 0) { *a.out = PcgResult{0, MQS_OK, 0.0, 0.0}; *a.refinements = 0; }
        return;
      }
      start_rel = sqrt(rr / bb);
    }
    relres = sqrt(rr / bb);
    if (!isfinite(rr) || !isfinite(bb)) { status = MQS_ERR_NAN; break; }
    if (rr <= a.tol2 * bb) { status = MQS_OK; break; }
    if (inner_total >= a.maxit || outer >= 64) { status = MQS_ERR_NOT_CONVERGED; break; }
    // inner float-float CG on L d = r / ||r||
    const double nr = sqrt(rr), inv = 1.0 / nr;
    ffv rho;
    {
      ffv acc(0);
      for (long long e = tid; e < len; e += nth) {
        const ffv v = ff_from(a.r[e] * inv);
        rb0[e] = v;
        df[e] = ffv(0);
        acc = fmaT(v, v, acc);
      }
      ffv dummy;
      if (!reduceF(acc, ffv(0), rho, dummy)) return;
    }
    // products and scalars stay float-float (no FP64 division or conversion in the loop)
    const double target = fmax(a.inner_tol, 0.5 * sqrt(a.tol2 * bb) / nr);
    const ffv stop2 = ff_from(target * target * ff_to(rho));
    int it_in = 0, cur = 0;
    ffv delta, dummy;
    {
      EpiApplyDotFF ep{wbuf(0), a.g.n3};
      sweep_L<ffv>(a.g, rbuf(0), a.full, bid, nb, sm.f, ep);
      if (!reduceF(ep.wr, ffv(0), delta, dummy)) return;
    }
    ffv gamma = rho;
    bool ok = delta.hi > 0.f, first = true;
    ffv alpha = ok ? ff_div(gamma, delta) : ffv(0), bet = ffv(0);
    while (ok && inner_total < a.maxit) {
      FusedVecsT<ffv> v{df, pf, rbuf(cur), wbuf(cur), sbuf(cur), rbuf(cur ^ 1), wbuf(cur ^ 1), sbuf(cur ^ 1),
                        alpha, bet, first};
      ffv g1(0), d1(0);
      sweep_fused<ffv>(a.g, v, a.full, bid, nb, sm.ff, g1, d1, a.ptab);
      ffv gn, dn;
      if (!reduceF(g1, d1, gn, dn)) return;
      ++it_in; ++inner_total;
      cur ^= 1;
      if (!isfinite(gn.hi) || !isfinite(dn.hi)) break;
      if (ff_le(gn, stop2) || it_in >= 400) break;
      const ffv bnew = ff_div(gn, gamma);
      const ffv den = dn - ff_div(ff_mul(bnew, gn), alpha);
      if (!(den.hi > 0.f)) break;               // stagnation at the float-float floor: refine from here
      bet = bnew; alpha = ff_div(gn, den); gamma = gn;
      first = false;
    }
    // x += ||r|| d (FP64); barrier so the next residual sees every update
    {
      for (long long e = tid; e < len; e += nth) a.x[e] = fma(nr, ff_to(df[e]), a.x[e]);
      double d0, d1;
      if (!reduce2(0.0, 0.0, d0, d1)) return;
    }
    ++outer;
  }
  if (bid == 0 && threadIdx.x == 0) {
    *a.out = PcgResult{inner_total, status, relres, start_rel};
    *a.refinements = outer;
  }
}

int launch_pcg_ff(const DevGeom& dg, const double* b, double* x, double* r, double* lx, const MixedBufs& mb,
                  double* part, unsigned* bar, int* err, PcgResult* out, int* refinements, double tol,
                  double inner_tol, int maxit, int nblk, cudaStream_t st, int init, const int* halt,
                  const int2* ptab) {
  MixedArgs a;
  a.g = dg.g;
  a.full = Box{{0, 0, 0}, {dg.g.n, dg.g.n, dg.g.n}};
  a.b = b; a.x = x; a.r = r; a.lx = lx;
  a.r32 = mb.r32; a.p32 = mb.p32; a.q32 = mb.q32; a.d32 = mb.d32;
  a.r32b = mb.r32b; a.w32a = mb.w32a; a.w32b = mb.w32b; a.s32a = mb.s32a; a.s32b = mb.s32b;
  a.variant = 1;
  a.ptab = ptab;
  a.part = part; a.bar = bar; a.err = err; a.out = out; a.refinements = refinements;
  a.tol2 = tol * tol; a.inner_tol = inner_tol; a.maxit = maxit;
  a.spin = 1ll << 21;
  a.init = (init == 2) ? 2 : 0;
  a.halt = halt;
  if (!mb.r32b || !mb.w32a || !mb.w32b || !mb.s32a || !mb.s32b) return MQS_ERR_ARG;
  if (cudaMemsetAsync(bar, 0, sizeof(unsigned), st) != cudaSuccess) return MQS_ERR_CUDA;
  void* args[] = {&a};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)pcg_ff_kernel, dim3(nblk), dim3(kBlock), args, 0, st);
  return e == cudaSuccess ? MQS_OK : MQS_ERR_CUDA;
}

int launch_pcg_mixed(const DevGeom& dg, const double* b, double* x, double* r, double* lx, const MixedBufs& mb,
                     double* part, unsigned* bar, int* err, PcgResult* out, int* refinements, double tol,
                     double inner_tol, int maxit, int nblk, cudaStream_t st, int init, int variant,
                     const int* halt, const int2* ptab, int halo_warps) {
  MixedArgs a;
  a.g = dg.g;
  a.full = Box{{0, 0, 0}, {dg.g.n, dg.g.n, dg.g.n}};
  a.b = b; a.x = x; a.r = r; a.lx = lx;
  a.r32 = mb.r32; a.p32 = mb.p32; a.q32 = mb.q32; a.d32 = mb.d32;
  a.r32b = mb.r32b; a.w32a = mb.w32a; a.w32b = mb.w32b; a.s32a = mb.s32a; a.s32b = mb.s32b;
  const bool bufs = mb.r32b && mb.w32a && mb.w32b && mb.s32a && mb.s32b;
  a.variant = (variant >= 1 && bufs) ? variant : 0;
  a.part = part; a.bar = bar; a.err = err; a.out = out; a.refinements = refinements;
  a.tol2 = tol * tol; a.inner_tol = inner_tol; a.maxit = maxit;
  a.spin = 1ll << 21;
  a.init = (init == 2) ? 2 : 0;
  a.halt = halt;
  if (cudaMemsetAsync(bar, 0, sizeof(unsigned), st) != cudaSuccess) return MQS_ERR_CUDA;
  void* args[] = {&a};
  // 64^3 (FP32 vectors in L2): one block per SM; from 96^3 on, two (28% faster per
  // inner iteration at 128^3, 83.6 -> 62.8 us)
  const bool two = 3LL * dg.g.n3 >= kMixedTwoBlocksLen;
  a.ptab = two ? nullptr : ptab;                 // the table is for nblk blocks
  // two halo warps per group: the one-reduction inner pass at one block per SM only
  const bool hw2 = halo_warps == 2 && !two && a.variant == 1;
  const void* fn = two ? (const void*)pcg_mixed_kernel<2>
                       : hw2 ? (const void*)pcg_mixed_kernel<1, 2> : (const void*)pcg_mixed_kernel<1>;
  const int threads = hw2 ? 32 * (kGroupWarps + 1) * kGroups : kBlock;
  const int smem = (int)sizeof(MixedSmem);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return MQS_ERR_CUDA;
  if (hw2) {
    // the 384-thread block must fit once per SM (asked once per process)
    static const int occ = [smem] {
      int o = 0;
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, pcg_mixed_kernel<1, 2>, 32 * (kGroupWarps + 1) * kGroups,
                                                           (size_t)smem) == cudaSuccess
                 ? o
                 : -1;
    }();
    if (occ < 0) return MQS_ERR_CUDA;
    if (occ < 1) return MQS_ERR_ARG;
  }
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(two ? 2 * nblk : nblk), dim3(threads), args, (size_t)smem, st);
  return e == cudaSuccess ? MQS_OK : MQS_ERR_CUDA;
}

MQS_DEBUG_TAKE(mixed)

}  // namespace mqs
