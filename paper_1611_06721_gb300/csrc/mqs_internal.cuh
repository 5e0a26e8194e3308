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
#include <type_traits>
#include <cuda_runtime.h>
#include "../../include/mqs.h"
#include "ff.cuh"

namespace mqs {

// ---- debug build: checked global accesses ------------------------------------------
// The library's debug variant (compiled with -DMQS_DEBUG_CHECKS) tests every index that a
// hot kernel computes (stencil sweeps, fused passes, conductor, right-hand side and
// support-list kernels) against the length of the array it addresses.  An index outside
// records its site and value in the translation unit's debug word (the first one wins)
// and the access is skipped (a load gives 0): nothing traps.  mqs_debug_check reads the
// words.  Release builds compile the checks out.  Loops whose index is the loop bound
// itself (grid-stride element loops) need no check.
#ifdef MQS_DEBUG_CHECKS
static __device__ unsigned long long g_dbg_word;   // per translation unit
__device__ __forceinline__ bool dbg_ok(long long idx, long long len, int site) {
  if (idx >= 0 && idx < len) return true;
  atomicCAS(&g_dbg_word, 0ull,
            (1ull << 63) | ((unsigned long long)(site & 0x7FFF) << 48) | ((unsigned long long)idx & 0xFFFFFFFFFFFFull));
  return false;
}
#define MQS_LDC(arr, idx, len, site)                                          \
  (::mqs::dbg_ok((long long)(idx), (long long)(len), (site))                  \
       ? (arr)[(idx)]                                                         \
       : std::remove_cv_t<std::remove_reference_t<decltype((arr)[0])>>{})
#define MQS_STC(arr, idx, len, site, val)                                             \
  do {                                                                                \
    if (::mqs::dbg_ok((long long)(idx), (long long)(len), (site))) (arr)[(idx)] = (val); \
  } while (0)
// host: the word of this translation unit, cleared after reading
#define MQS_IDX_OK(idx, len, site) (::mqs::dbg_ok((long long)(idx), (long long)(len), (site)))
#define MQS_DEBUG_TAKE(name)                                                          \
  int dbg_take_##name(unsigned long long* out) {                                      \
    const unsigned long long zero = 0;                                                \
    if (cudaMemcpyFromSymbol(out, g_dbg_word, sizeof zero) != cudaSuccess) return -2; \
    return cudaMemcpyToSymbol(g_dbg_word, &zero, sizeof zero) == cudaSuccess ? 0 : -2; \
  }
#else
#define MQS_LDC(arr, idx, len, site) ((arr)[(idx)])
#define MQS_STC(arr, idx, len, site, val) ((arr)[(idx)] = (val))
#define MQS_IDX_OK(idx, len, site) true
#define MQS_DEBUG_TAKE(name)                       \
  int dbg_take_##name(unsigned long long* out) { \
    *out = 0;                                    \
    return 0;                                    \
  }
#endif

constexpr int kTY = 4;                  // row warps per stencil group (tile 32 x kTY)
constexpr int kGroupWarps = kTY + 1;    // + one warp for the j0-1 halo row
constexpr int kGroups = 2;              // independent groups per block (own named barrier)
constexpr int kWarps = kGroups * kGroupWarps;
constexpr int kBlock = 32 * kWarps;     // 320 threads
constexpr int kMaxSeg = 32;             // planes per segment (x halo: one per lane)
constexpr int kPcgBlocksPerSM = 1;      // co-resident PCG blocks per SM
// layout length (3 n^3) from which the FP64 PCG and the FP32-inner refinement run two
// blocks per SM (n >= 96: their vectors exceed the L2 several times)
constexpr long long kMixedTwoBlocksLen = 3LL * 96 * 96 * 96;

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
    unsigned cf = MQS_LDC(g.cflags, (i - g.cb_lo[0]) + w0 * ((j - g.cb_lo[1]) + w1 * (k - g.cb_lo[2])),
                          w0 * w1 * (g.cb_hi[2] - g.cb_lo[2]), 151);
    m &= ~cf;
  }
  return m;
}

// component load with zero outside [0, n)
__device__ __forceinline__ double ld(const double* __restrict__ v, int n, long long n3, int c,
                                     int i, int j, int k) {
  if (i < 0 || j < 0 || k < 0 || i >= n || j >= n || k >= n) return 0.0;
  return MQS_LDC(v, c * n3 + pidx(n, i, j, k), 3 * n3, 152);
}

// identity load conversion of sweep_L
struct LoadAs {
  template <class V>
  __device__ __forceinline__ V operator()(V v) const { return v; }
};

// ---- 64-bit fixed point for the integer stencil ----------------------------------
// On this GPU an FP64 addition issues at about 1.6 lanes per clock and SM, a 64-bit
// integer addition at about 32, and the hardware FP64 <-> int64 conversions at 2 (on
// the FP64 unit).  L has integer coefficients, so a sweep can convert its FP64 source
// v (all |v_i| < 2^(E-1)) to the integers V_i = round(v_i 2^(58-E)) (|V_i| < 2^58), form
// L V exactly in 64-bit integer arithmetic (every flux sums 4 values, every output 4
// fluxes: |L V| < 2^62), and convert back with one rounding, t = (L V) 2^(E-58).  Both
// conversions are bit manipulations on the integer pipes.

// round(v 2^sh) as a 64-bit integer (nearest, ties away from zero), for |v 2^sh| < 2^58;
// zero and subnormal v give 0 (they lie far below the resolution 2^-sh).
__host__ __device__ __forceinline__ long long fx_from_double(double v, int sh) {
#ifdef __CUDA_ARCH__
  const long long b = __double_as_longlong(v);
#else
  long long b;
  __builtin_memcpy(&b, &v, sizeof b);
#endif
  const int e = (int)((b >> 52) & 0x7FF);
  const int s = e - 1075 + sh;                                   // |v| 2^sh = m 2^s
  const long long m = (b & 0x000FFFFFFFFFFFFFLL) | 0x0010000000000000LL;
  const int rs = -s;
  long long r = 0;
  if (s >= 0) r = m << s;
  else if (rs < 54) r = (m + (1LL << (rs - 1))) >> rs;
  if (e == 0) r = 0;
  return b < 0 ? -r : r;
}

// t 2^sh as the nearest double (ties to even), for |t| < 2^63 and a normal result.
__host__ __device__ __forceinline__ double fx_to_double(long long t, int sh) {
  if (t == 0) return 0.0;
  const unsigned long long sgn = t < 0 ? 0x8000000000000000ull : 0ull;
  unsigned long long a = t < 0 ? 0ull - (unsigned long long)t : (unsigned long long)t;
#ifdef __CUDA_ARCH__
  const int lz = __clzll((long long)a);
#else
  const int lz = __builtin_clzll(a);
#endif
  a <<= lz;                                                      // leading one at bit 63
  unsigned long long mant = a >> 11;                             // 53 bits, leading one at bit 52
  const unsigned rem = (unsigned)(a & 0x7FFull);
  mant += (rem > 0x400u || (rem == 0x400u && (mant & 1ull))) ? 1ull : 0ull;
  const long long eb = 1023 + 63 - lz + sh;                      // biased exponent of the leading one
  // (eb - 1) 2^52 + mant: the implicit bit of mant completes the exponent, and a
  // rounding carry to 2^53 moves it up by one with a zero fraction
  const unsigned long long bits = ((unsigned long long)(eb - 1) << 52) + mant;
  const unsigned long long out = bits | sgn;
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)out);
#else
  double d;
  __builtin_memcpy(&d, &out, sizeof d);
  return d;
#endif
}

// E for a vector of squared norm ss (> 0, finite): every component lies below 2^(E-1)
// (|v_i| <= sqrt(ss) < 2^(floor(ilogb(ss) / 2) + 1)), with a factor 2 to spare
__host__ __device__ __forceinline__ int fx_exponent(double ss) {
#ifdef __CUDA_ARCH__
  const long long b = __double_as_longlong(ss);
#else
  long long b;
  __builtin_memcpy(&b, &ss, sizeof b);
#endif
  const int e2 = (int)((b >> 52) & 0x7FF) - 1023;
  return (e2 >> 1) + 2;
}

// load conversion of sweep_L: FP64 source to the fixed point of scale 2^sh (sh = 58 - E)
struct LoadFx {
  int sh;
  __device__ __forceinline__ long long operator()(double v) const { return fx_from_double(v, sh); }
};
__device__ __forceinline__ long long shfl_up1(long long v) { return __shfl_up_sync(0xffffffffu, v, 1); }

template <class T>
struct SweepGroupSmemT {
  T fz[2][kGroupWarps][32];
  T fx[2][kGroupWarps][32];
  T hz[2][kTY];                         // x halo: bz, by at (i0 - 1, j0 + row)
  T hy[2][kTY];
};
template <class T, int G = kGroups>
struct SweepSmemT {
  SweepGroupSmemT<T> g[G];
};
using SweepSmem = SweepSmemT<double>;

// barrier over the kGroupWarps warps of stencil group `grp` (ids 1.. ; 0 is __syncthreads)
__device__ __forceinline__ void group_sync(int grp) {
  asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(kGroupWarps * 32) : "memory");
}
// the same over NW warps (a group with more than one halo warp)
template <int NW>
__device__ __forceinline__ void group_sync_n(int grp) {
  asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(NW * 32) : "memory");
}

// Applies t = L s over the positions of `box`, calling
//   epi(e, mask, tx, ty, tz, sx, sy, sz)
// once per position (after epi.prefetch(e), which may start its loads early) (e = i + n(j + n k); mask from nmask; t unmasked; s the
// source values at the position).  Work is split into plane-tiles of 32 x kTY
// positions; each of the kGroups warp groups of the block is one part (of
// nparts * kGroups), takes a contiguous range of plane-tiles and marches each
// tile column along z so every face flux is formed once (plus one halo row,
// one halo column and one warm-up plane per segment).  Groups synchronise on
// their own named barrier, so one group's plane step never waits for the other.  Index
// arithmetic is 32-bit and incremental along the march (3 n^3 < 2^31 for
// n <= 800); bounds tests are hoisted out of the plane loop.
// Templated on the value type T (double for the FP64 path, float or the
// float-float ffv for the inner solves of the refined paths); arithmetic is in T.
// Values are loaded as M (= T by default) and turned into T by cv (the identity by
// default; the FP64 PCG's direction sweep loads FP64 and runs the stencil in 64-bit
// fixed point, exactly, on the integer pipes).
// Must be called by all G x kGroupWarps warps of the block (G groups; kGroups unless the
// caller's shared memory says otherwise), and by no other warp.
template <class T, class Epi, class M, class Cv = LoadAs, int G = kGroups>
__device__ void sweep_L(const Geom& g, const M* __restrict__ s, const Box& box, int part, int nparts,
                        SweepSmemT<T, G>& sm, Epi& epi, Cv cv = Cv()) {
  const int n = g.n;
  const int n2 = n * n;
  const int n3 = (int)g.n3;
  const int lane = threadIdx.x & 31, grp = (threadIdx.x >> 5) / kGroupWarps, w = (threadIdx.x >> 5) % kGroupWarps;
  SweepGroupSmemT<T>& sg = sm.g[grp];
  const int bx0 = box.hi[0] - box.lo[0], by0 = box.hi[1] - box.lo[1], nz = box.hi[2] - box.lo[2];
  if (bx0 <= 0 || by0 <= 0 || nz <= 0) return;
  const int ntx = (bx0 + 31) / 32, nty = (by0 + kTY - 1) / kTY;
  const long long ntiles = (long long)ntx * nty * nz;
  const long long gp = (long long)part * G + grp, gn = (long long)nparts * G;
  long long u = ntiles * gp / gn;
  const long long u1 = ntiles * (gp + 1) / gn;
  const int cw0 = g.cb_hi[0] - g.cb_lo[0], cw01 = cw0 * (g.cb_hi[1] - g.cb_lo[1]);
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
    group_sync(grp);  // smem reuse across segments
    if (w < kTY) {
      const int j = j0 + w;
      const bool act = (i < box.hi[0]) && (j < box.hi[1]);
      const bool col = (i < n) && (j < n);
      const bool vi1 = col && (i + 1 < n), vj1 = col && (j + 1 < n);
      // column part of the n-edge mask: x needs j,k > 0; y needs i,k > 0; z needs i,j > 0
      const unsigned mcol = (j > 0 ? 1u : 0u) | (i > 0 ? 2u : 0u) | ((i > 0 && j > 0) ? 4u : 0u);
      const bool incb = i >= g.cb_lo[0] && i < g.cb_hi[0] && j >= g.cb_lo[1] && j < g.cb_hi[1];
      const int cfc = incb ? (i - g.cb_lo[0]) + cw0 * (j - g.cb_lo[1]) : 0;
      const M* __restrict__ sx_ = s;
      const M* __restrict__ sy_ = s + n3;
      const M* __restrict__ sz_ = s + 2 * n3;
      int o = col ? i + n * (j + n * ks) : 0;     // position of plane ks
      // all loads of the segment start issued together: warm-up plane ks - 1,
      // plane ks (own, x+1 and y+1 neighbours) and own values of plane ks + 1
      const bool wu = (ks >= 1) && col;
      const int om = o - n2;
      const T xm = wu ? cv(MQS_LDC(sx_, om, n3, 101)) : T(0), ym = wu ? cv(MQS_LDC(sy_, om, n3, 102)) : T(0), zm = wu ? cv(MQS_LDC(sz_, om, n3, 103)) : T(0);
      const T zim = (wu && vi1) ? cv(MQS_LDC(sz_, om + 1, n3, 104)) : T(0), zjm = (wu && vj1) ? cv(MQS_LDC(sz_, om + n, n3, 105)) : T(0);
      T x0 = 0, y0 = 0, z0 = 0;
      T yi = 0, zi = 0, xj = 0, zj = 0, xk = 0, yk = 0, zk = 0;
      if (col) {
        x0 = cv(MQS_LDC(sx_, o, n3, 106)); y0 = cv(MQS_LDC(sy_, o, n3, 107)); z0 = cv(MQS_LDC(sz_, o, n3, 108));
        if (vi1) { yi = cv(MQS_LDC(sy_, o + 1, n3, 109)); zi = cv(MQS_LDC(sz_, o + 1, n3, 110)); }
        if (vj1) { xj = cv(MQS_LDC(sx_, o + n, n3, 111)); zj = cv(MQS_LDC(sz_, o + n, n3, 112)); }
        if (ks + 1 < n) { xk = cv(MQS_LDC(sx_, o + n2, n3, 113)); yk = cv(MQS_LDC(sy_, o + n2, n3, 114)); zk = cv(MQS_LDC(sz_, o + n2, n3, 115)); }
      }
      if (act) epi.prefetch(o);
      // warm-up fluxes bx, by at plane ks - 1 (zero when ks = 0: unused there)
      T bxm = 0, bym = 0;
      if (wu) {
        bxm = (ym - zm) + (zjm - y0);
        bym = (zm - xm) + (x0 - zim);
      }
      int buf = 0;
      for (int k = ks; k < ke; ++k, o += n2) {
        // issue the next plane's loads first; they are converted only when they become
        // the current plane's values, so the plane step never waits on them
        M nyi = M(0), nzi = M(0), nxj = M(0), nzj = M(0), nxk = M(0), nyk = M(0), nzk = M(0);
        const int o1 = o + n2;
        if (col && k + 1 < ke) {
          if (vi1) { nyi = MQS_LDC(sy_, o1 + 1, n3, 116); nzi = MQS_LDC(sz_, o1 + 1, n3, 117); }
          if (vj1) { nxj = MQS_LDC(sx_, o1 + n, n3, 118); nzj = MQS_LDC(sz_, o1 + n, n3, 119); }
          if (k + 2 < n) { nxk = MQS_LDC(sx_, o1 + n2, n3, 120); nyk = MQS_LDC(sy_, o1 + n2, n3, 121); nzk = MQS_LDC(sz_, o1 + n2, n3, 122); }
        }
        T bx = 0, by = 0, bz = 0;
        if (col) {
          bx = (y0 - z0) + (zj - yk);
          by = (z0 - x0) + (xk - zi);
          bz = (x0 - y0) + (yi - xj);
        }
        sg.fz[buf][w + 1][lane] = bz;
        sg.fx[buf][w + 1][lane] = bx;
        group_sync(grp);
        T bzi = shfl_up1(bz), byi = shfl_up1(by);
        if (lane == 0) { bzi = sg.hz[buf][w]; byi = sg.hy[buf][w]; }
        const T bzj = sg.fz[buf][w][lane], bxj = sg.fx[buf][w][lane];
        if (act) {
          const T tx = (bz - bzj) + (bym - by);
          const T ty = (bzi - bz) + (bx - bxm);
          const T tz = (bxj - bx) + (by - byi);
          unsigned m = mcol & (k > 0 ? 7u : 4u);
          if (incb && k >= g.cb_lo[2] && k < g.cb_hi[2]) m &= ~(unsigned)MQS_LDC(g.cflags, cfc + cw01 * (k - g.cb_lo[2]), cw01 * (g.cb_hi[2] - g.cb_lo[2]), 150);
          epi(o, m, tx, ty, tz, x0, y0, z0);
          if (k + 1 < ke) epi.prefetch(o1);
        }
        bxm = bx; bym = by;
        x0 = xk; y0 = yk; z0 = zk;
        yi = cv(nyi); zi = cv(nzi); xj = cv(nxj); zj = cv(nzj); xk = cv(nxk); yk = cv(nyk); zk = cv(nzk);
        buf ^= 1;
      }
    } else {
      // halo warp: per plane, bz and bx of row j0 - 1 (all lanes) and the x halo
      // bz, by at (i0 - 1, j0 + r) for rows r < kTY (lanes r); the next plane's
      // loads are issued before this plane's arithmetic.
      const int jh = j0 - 1;
      const bool hrow = (jh >= 0) && (i < n);
      const int jr = j0 + lane;
      const bool hcol = (i0 >= 1) && (lane < kTY) && (jr < n);
      const bool hi1 = hrow && (i + 1 < n), hj1 = hcol && (jr + 1 < n);
      const M* __restrict__ sx_ = s;
      const M* __restrict__ sy_ = s + n3;
      const M* __restrict__ sz_ = s + 2 * n3;
      int oh = hrow ? i + n * (jh + n * ks) : 0;          // halo row position, plane ks
      int oc = hcol ? (i0 - 1) + n * (jr + n * ks) : 0;   // halo column position, plane ks
      T a[7], c[8];
      // raw loads (converted when used, as in the row warps)
      auto load_row = [&](int k, int o, M* v) {
        v[0] = MQS_LDC(sx_, o, n3, 123); v[1] = MQS_LDC(sy_, o, n3, 124); v[2] = MQS_LDC(sz_, o, n3, 125);
        v[3] = hi1 ? MQS_LDC(sy_, o + 1, n3, 126) : M(0);
        v[4] = MQS_LDC(sx_, o + n, n3, 127); v[5] = MQS_LDC(sz_, o + n, n3, 128);
        v[6] = (k + 1 < n) ? MQS_LDC(sy_, o + n2, n3, 129) : M(0);
      };
      auto load_col = [&](int k, int o, M* v) {
        v[0] = MQS_LDC(sx_, o, n3, 130); v[1] = MQS_LDC(sy_, o + 1, n3, 131);
        v[2] = hj1 ? MQS_LDC(sx_, o + n, n3, 132) : M(0);
        v[3] = MQS_LDC(sy_, o, n3, 133); v[4] = MQS_LDC(sz_, o, n3, 134);
        v[5] = (k + 1 < n) ? MQS_LDC(sx_, o + n2, n3, 135) : M(0);
        v[6] = MQS_LDC(sz_, o + 1, n3, 136);
        v[7] = M(0);
      };
      {
        M ra[7], rc[8];
#pragma unroll
        for (int q = 0; q < 7; ++q) ra[q] = M(0);
#pragma unroll
        for (int q = 0; q < 8; ++q) rc[q] = M(0);
        if (hrow) load_row(ks, oh, ra);
        if (hcol) load_col(ks, oc, rc);
#pragma unroll
        for (int q = 0; q < 7; ++q) a[q] = cv(ra[q]);
#pragma unroll
        for (int q = 0; q < 8; ++q) c[q] = cv(rc[q]);
      }
      int buf = 0;
      for (int k = ks; k < ke; ++k) {
        M na[7], nc[8];
#pragma unroll
        for (int q = 0; q < 7; ++q) na[q] = M(0);
#pragma unroll
        for (int q = 0; q < 8; ++q) nc[q] = M(0);
        if (k + 1 < ke) {
          if (hrow) load_row(k + 1, oh + n2, na);
          if (hcol) load_col(k + 1, oc + n2, nc);
        }
        oh += n2;
        oc += n2;
        // bz = x + y(i+1) - x(j+1) - y ; bx = y + z(j+1) - y(k+1) - z
        sg.fz[buf][0][lane] = hrow ? (a[0] - a[1]) + (a[3] - a[4]) : T(0);
        sg.fx[buf][0][lane] = hrow ? (a[1] - a[2]) + (a[5] - a[6]) : T(0);
        if (lane < kTY) {
          // bz = x + y(i0) - x(j+1) - y ; by = z + x(k+1) - z(i0) - x
          sg.hz[buf][lane] = hcol ? (c[0] - c[3]) + (c[1] - c[2]) : T(0);
          sg.hy[buf][lane] = hcol ? (c[4] - c[0]) + (c[5] - c[6]) : T(0);
        }
        group_sync(grp);
#pragma unroll
        for (int q = 0; q < 7; ++q) a[q] = cv(na[q]);
#pragma unroll
        for (int q = 0; q < 8; ++q) c[q] = cv(nc[q]);
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

// Sums of two values over the block and the grid, deterministic (fixed order,
// the same in every block) in T = double or the float-float ffv.  One FP64
// warp instruction holds its sub-partition's FP64 unit for about 64 cycles on
// this GPU (not pipelined; a dependent FP64 add with a shuffle ~110 cycles),
// so the sums keep FP64 instructions and dependent steps few: a transposed
// butterfly (the first exchange leaves value 0 in lanes 0-15 and value 1 in
// lanes 16-31: five additions per warp for both values), the warp totals
// summed by one warp, and the grid's block partials loaded all at once and
// summed by two warps, one per value (two sub-partitions, two FP64 units).
__device__ __forceinline__ double shfl_x(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ ffv shfl_x(ffv v, int o) {
  return ffv(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}
__device__ __forceinline__ double shfl_from(double v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ ffv shfl_from(ffv v, int l) {
  return ffv(__shfl_sync(0xffffffffu, v.hi, l), __shfl_sync(0xffffffffu, v.lo, l));
}
__device__ __forceinline__ double ld_part(const double* p) { return *p; }
__device__ __forceinline__ ffv ld_part(const ffv* p) {
  const float2 f = *reinterpret_cast<const float2*>(p);
  return ffv(f.x, f.y);
}

// lanes 0-15: the warp's sum of v0 (exact total in lane 0); lanes 16-31: of v1 (lane 16)
template <class T>
__device__ __forceinline__ T warp_sum2(T v0, T v1) {
  const bool up = (threadIdx.x & 16) != 0;
  T s = (up ? v1 : v0) + shfl_x(up ? v0 : v1, 16);
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) s = s + shfl_x(s, o);
  return s;
}

// Block sums of (v0, v1); the totals land in thread 0 (t0 and t1).  red: 32 T
// of shared memory; at most 16 warps.  Ends without a block barrier: red may be
// reused only after the caller's next __syncthreads.
template <class T>
__device__ __forceinline__ void block_sum2(T v0, T v1, T* red, T& t0, T& t1) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const T s = warp_sum2(v0, v1);
  if ((lane & 15) == 0) red[(lane >> 4) * 16 + w] = s;   // red[w] = v0 sums, red[16 + w] = v1 sums
  __syncthreads();
  if (w == 0) {
    T t = ((lane & 15) < nw) ? red[lane] : T(0);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) t = t + shfl_x(t, o);
    t0 = t;
    t1 = shfl_from(t, 16);
  }
}

// Sum of p[0..cnt) by one warp (every lane returns the same value in FP64;
// lane 0's is the defined one).  Loads issue together, then a fixed chain.
template <class T>
__device__ __forceinline__ T warp_fixed_sum(const T* p, int cnt) {
  const int lane = threadIdx.x & 31;
  T v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = (lane + 32 * q < cnt) ? ld_part(p + lane + 32 * q) : T(0);
  const int nq = (cnt + 31) >> 5;
  T s = v[0];
#pragma unroll
  for (int q = 1; q < 8; ++q)
    if (q < nq) s = s + v[q];
  for (int q = lane + 256; q < cnt; q += 32) s = s + ld_part(p + q);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s = s + shfl_x(s, o);
  return s;
}

// Sum of part[0..cnt) computed identically by every caller (one warp).
__device__ __forceinline__ double fixed_sum(const double* part, int cnt) { return warp_fixed_sum(part, cnt); }

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
// of barriers passed so far, this one included).  Thread 0 publishes the
// block's prior writes with a release-add (ordered after the CTA barrier) and
// polls with acquire loads; a wait longer than `spin` polls records
// MQS_ERR_TIMEOUT in *err and returns false (the block then leaves the kernel;
// the other blocks time out at their next barrier).
__device__ __forceinline__ bool grid_barrier(unsigned* ctr, unsigned target, long long spin, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    red_release_add(ctr, 1u);
    long long polls = 0;
    while (ld_acquire(ctr) < target) {
      if (++polls > spin) { atomicExch(err, MQS_ERR_TIMEOUT); ok = 0; break; }
    }
  }
  __syncthreads();
  return ok != 0;
}

// Grid-wide sums of two values per thread, returned to every thread: block
// sums into this block's partial slots, a grid barrier, then every block sums
// the partials in the same fixed order.  part holds 2 slots x 4 x gridDim.x
// entries of 8 bytes (the slot alternates: a block already at the next sum
// cannot overwrite partials still being read); red: 32 T and gs: 2 T of shared
// memory.  Returns false when the barrier timed out.  All threads must call.
template <class T>
__device__ __forceinline__ bool grid_sum2(T v0, T v1, T& s0, T& s1, void* part, int& slot, unsigned& nbar,
                                          unsigned* bar, long long spin, int* err, T* red, T* gs) {
  const int nb = gridDim.x, w = threadIdx.x >> 5;
  T* p0 = reinterpret_cast<T*>(part) + (size_t)slot * 4 * nb;
  T* p1 = p0 + nb;
  T t0, t1;
  block_sum2(v0, v1, red, t0, t1);
  if (threadIdx.x == 0) { p0[blockIdx.x] = t0; p1[blockIdx.x] = t1; }
  if (!grid_barrier(bar, nb * (++nbar), spin, err)) return false;
  if (w < 2) {
    const T t = warp_fixed_sum(w ? p1 : p0, nb);
    if ((threadIdx.x & 31) == 0) gs[w] = t;
  }
  __syncthreads();
  s0 = gs[0]; s1 = gs[1];
  slot ^= 1;
  return true;
}

// grid_sum2 of (v0, v1) together with the grid-wide maxima of three ints m0..m2 in
// [0, 2^16) (biased exponents), packed into the third partial slot of each block:
// one grid barrier for all five.  The maxima take one warp instruction per warp
// (redux.sync) and one more warp after the barrier.  gm: 3 ints of shared memory.
__device__ __forceinline__ bool grid_sum2_max3(double v0, double v1, int m0, int m1, int m2, double& s0, double& s1,
                                               int& x0, int& x1, int& x2, void* part, int& slot, unsigned& nbar,
                                               unsigned* bar, long long spin, int* err, double* red, double* gs,
                                               int* gm) {
  __shared__ int wm[3][32];
  const int nb = gridDim.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double* p0 = reinterpret_cast<double*>(part) + (size_t)slot * 4 * nb;
  double* p1 = p0 + nb;
  long long* p2 = reinterpret_cast<long long*>(p0 + 2 * nb);
  const int a0 = __reduce_max_sync(0xffffffffu, m0), a1 = __reduce_max_sync(0xffffffffu, m1);
  const int a2 = __reduce_max_sync(0xffffffffu, m2);
  if (lane == 0) { wm[0][w] = a0; wm[1][w] = a1; wm[2][w] = a2; }
  double t0, t1;
  block_sum2(v0, v1, red, t0, t1);                    // its block barrier also publishes wm
  if (threadIdx.x == 0) {
    int b0 = 0, b1 = 0, b2 = 0;
    for (int q = 0; q < nw; ++q) { b0 = max(b0, wm[0][q]); b1 = max(b1, wm[1][q]); b2 = max(b2, wm[2][q]); }
    p0[blockIdx.x] = t0;
    p1[blockIdx.x] = t1;
    p2[blockIdx.x] = (long long)b0 | ((long long)b1 << 16) | ((long long)b2 << 32);
  }
  if (!grid_barrier(bar, nb * (++nbar), spin, err)) return false;
  if (w < 2) {
    const double t = warp_fixed_sum(w ? p1 : p0, nb);
    if (lane == 0) gs[w] = t;
  } else if (w == 2) {
    // the loads issued together (as in warp_fixed_sum), not one L2 round trip per 32 blocks
    int c0 = 0, c1 = 0, c2 = 0;
    long long pk[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) pk[q] = (lane + 32 * q < nb) ? p2[lane + 32 * q] : 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      c0 = max(c0, (int)(pk[q] & 0xFFFF));
      c1 = max(c1, (int)((pk[q] >> 16) & 0xFFFF));
      c2 = max(c2, (int)((pk[q] >> 32) & 0xFFFF));
    }
    for (int q = lane + 256; q < nb; q += 32) {
      const long long v = p2[q];
      c0 = max(c0, (int)(v & 0xFFFF));
      c1 = max(c1, (int)((v >> 16) & 0xFFFF));
      c2 = max(c2, (int)((v >> 32) & 0xFFFF));
    }
    c0 = __reduce_max_sync(0xffffffffu, c0);
    c1 = __reduce_max_sync(0xffffffffu, c1);
    c2 = __reduce_max_sync(0xffffffffu, c2);
    if (lane == 0) { gm[0] = c0; gm[1] = c1; gm[2] = c2; }
  }
  __syncthreads();
  s0 = gs[0]; s1 = gs[1];
  x0 = gm[0]; x1 = gm[1]; x2 = gm[2];
  slot ^= 1;
  return true;
}

}  // namespace mqs
