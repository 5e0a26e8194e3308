// One-reduction PCG iteration (Chronopoulos-Gear form of the CG recurrences)
// as a single stencil pass.  With w = L r and s = L p carried as vectors:
//   p_i = r_i + beta p_{i-1},  s_i = w_i + beta s_{i-1},
//   x_{i+1} = x_i + alpha p_i,  r_{i+1} = r_i - alpha s_i,
//   w_{i+1} = L r_{i+1},  gamma = r_{i+1}.r_{i+1},  delta = w_{i+1}.r_{i+1};
//   beta' = gamma'/gamma,  alpha' = gamma' / (delta' - beta' gamma' / alpha).
// The stencil source r_{i+1} is formed once per position by its owner from
// (r_i, w_i, s_{i-1}) - buffers nobody writes during the pass (r, s, w are
// double-buffered) - and shared with the x+1 neighbour by shuffle and the y+1
// neighbour through shared memory; the halo warp forms the tile halo.
#pragma once
#include "mqs_internal.cuh"

namespace mqs {

// fused multiply-add in the precision of the sweep
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }

template <class T>
struct FusedVecsT {
  T* x;
  T* p;
  const T* r_in;   // r_i
  const T* w_in;   // w_i = L r_i
  const T* s_in;   // s_{i-1}
  T* r_out;        // r_{i+1}
  T* w_out;        // w_{i+1}
  T* s_out;        // s_i
  T alpha, beta;
  bool first;           // beta = 0 and no previous p, s
};

template <class T>
struct FusedSmemT {
  // r_{i+1} of plane k (buffer k&1): rows j0-1 .. j0+kTY (index row+1),
  // columns i0-1 .. i0+32 (index lane+1), three components
  T src[2][3][kTY + 2][34];
  T fz[2][kTY + 1][32];      // bz, bx of rows j0-1 .. j0+kTY-1
  T fx[2][kTY + 1][32];
  T hz[2][kTY];              // x halo: bz, by at (i0 - 1, j0 + row)
  T hy[2][kTY];
};
template <class T>
struct FusedSmemBlockT { FusedSmemT<T> g[kGroups]; };
using FusedVecs = FusedVecsT<double>;
using FusedSmemBlock = FusedSmemBlockT<double>;

// r_{i+1} at one component position from the input buffers (no writes)
template <class T>
__device__ __forceinline__ T fused_src(const FusedVecsT<T>& v, int off, int n3) {
  const T w = MQS_LDC(v.w_in, off, 3 * n3, 331);
  const T sv = v.first ? w : fmaT(v.beta, MQS_LDC(v.s_in, off, 3 * n3, 332), w);
  return fmaT(-v.alpha, sv, MQS_LDC(v.r_in, off, 3 * n3, 333));
}

// Update of one owned position (3 components): writes p, x, s_out, r_out and
// returns r_{i+1} in src[3].
template <class T>
__device__ __forceinline__ void fused_update(const FusedVecsT<T>& v, int o, int n3, T* src) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int e = o + c * n3;
    const T r = MQS_LDC(v.r_in, e, 3 * n3, 301), w = MQS_LDC(v.w_in, e, 3 * n3, 302);
    const T s = v.first ? w : fmaT(v.beta, MQS_LDC(v.s_in, e, 3 * n3, 303), w);
    const T p = v.first ? r : fmaT(v.beta, MQS_LDC(v.p, e, 3 * n3, 304), r);
    const T x = MQS_LDC(v.x, e, 3 * n3, 305);
    MQS_STC(v.s_out, e, 3 * n3, 306, s);
    MQS_STC(v.p, e, 3 * n3, 307, p);
    MQS_STC(v.x, e, 3 * n3, 308, fmaT(v.alpha, p, x));
    const T rn = fmaT(-v.alpha, s, r);
    MQS_STC(v.r_out, e, 3 * n3, 309, rn);
    src[c] = rn;
  }
}

// Loaded inputs of one position (3 components): r_i, w_i, s_{i-1}, p_{i-1}, x_i.
template <class T>
struct FusedLoadT {
  T r[3], w[3], s[3], p[3], x[3];
};

template <class T>
__device__ __forceinline__ void fused_load(const FusedVecsT<T>& v, int o, int n3, bool owned, FusedLoadT<T>& L) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int e = o + c * n3;
    L.r[c] = MQS_LDC(v.r_in, e, 3 * n3, 310);
    L.w[c] = MQS_LDC(v.w_in, e, 3 * n3, 311);
    L.s[c] = v.first ? T(0) : MQS_LDC(v.s_in, e, 3 * n3, 312);
    L.p[c] = (owned && !v.first) ? MQS_LDC(v.p, e, 3 * n3, 313) : T(0);
    L.x[c] = owned ? MQS_LDC(v.x, e, 3 * n3, 314) : T(0);
  }
}

// r_{i+1} from loaded inputs; when owned also writes p, x, s_out, r_out
template <class T>
__device__ __forceinline__ void fused_apply(const FusedVecsT<T>& v, int o, int n3, bool owned, const FusedLoadT<T>& L,
                                            T* src) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T sv = v.first ? L.w[c] : fmaT(v.beta, L.s[c], L.w[c]);
    const T rn = fmaT(-v.alpha, sv, L.r[c]);
    src[c] = rn;
    if (owned) {
      const int e = o + c * n3;
      const T pv = v.first ? L.r[c] : fmaT(v.beta, L.p[c], L.r[c]);
      MQS_STC(v.s_out, e, 3 * n3, 315, sv);
      MQS_STC(v.p, e, 3 * n3, 316, pv);
      MQS_STC(v.x, e, 3 * n3, 317, fmaT(v.alpha, pv, L.x[c]));
      MQS_STC(v.r_out, e, 3 * n3, 318, rn);
    }
  }
}

// One fused pass over `box` for group-part `part` of `nparts` (block level,
// as in sweep_L).  Accumulates gamma and delta into the caller's registers.
// ptab (nullable): the part ranges of fused_partition (kGroups groups per block)
// HW: halo warps per group, as in sweep_fused_fx (2: kGroups more warps at the end of the
// block, each group's second halo warp forming row j0+kTY and column i0+32).
template <class T, int HW = 1>
__device__ void sweep_fused(const Geom& g, const FusedVecsT<T>& v, const Box& box, int part, int nparts,
                            FusedSmemBlockT<T>& smb, T& gamma, T& delta, const int2* ptab = nullptr) {
  static_assert(HW == 1 || HW == 2, "one or two halo warps per group");
  const int n = g.n;
  const int n2 = n * n;
  const int n3 = (int)g.n3;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool extra = HW == 2 && warp >= kGroups * kGroupWarps;     // a second halo warp
  const int grp = extra ? warp - kGroups * kGroupWarps : warp / kGroupWarps;
  const int w = extra ? kTY + 1 : warp % kGroupWarps;
  auto gsync = [&] {
    if (HW == 1) group_sync(grp);
    else group_sync_n<kGroupWarps + 1>(grp);
  };
  FusedSmemT<T>& sg = smb.g[grp];
  const int bx0 = box.hi[0] - box.lo[0], by0 = box.hi[1] - box.lo[1], nz = box.hi[2] - box.lo[2];
  if (bx0 <= 0 || by0 <= 0 || nz <= 0) return;
  const int ntx = (bx0 + 31) / 32, nty = (by0 + kTY - 1) / kTY;
  const long long ntiles = (long long)ntx * nty * nz;
  const long long gp = (long long)part * kGroups + grp, gn = (long long)nparts * kGroups;
  long long u = ptab ? (long long)ptab[gp].x : ntiles * gp / gn;
  const long long u1 = ptab ? (long long)ptab[gp].y : ntiles * (gp + 1) / gn;
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
    gsync();  // smem reuse across segments
    if (w < kTY) {
      const int j = j0 + w;
      const bool act = (i < box.hi[0]) && (j < box.hi[1]);   // owned position
      const bool col = (i < n) && (j < n);
      const unsigned mcol = (j > 0 ? 1u : 0u) | (i > 0 ? 2u : 0u) | ((i > 0 && j > 0) ? 4u : 0u);
      const bool incb = i >= g.cb_lo[0] && i < g.cb_hi[0] && j >= g.cb_lo[1] && j < g.cb_hi[1];
      const int cfc = incb ? (i - g.cb_lo[0]) + cw0 * (j - g.cb_lo[1]) : 0;
      int o = col ? i + n * (j + n * ks) : 0;
      // prologue: plane ks is owned -> update it; warm-up fluxes at ks - 1 from recomputed sources
      T sk[3] = {T(0), T(0), T(0)};
      if (act) fused_update(v, o, n3, sk);
      else if (col) { sk[0] = fused_src(v, o, n3); sk[1] = fused_src(v, o + n3, n3); sk[2] = fused_src(v, o + 2 * n3, n3); }
#pragma unroll
      for (int c = 0; c < 3; ++c) sg.src[ks & 1][c][w + 1][lane + 1] = sk[c];
      T bxm = T(0), bym = T(0);
      if (ks >= 1 && col) {
        const int om = o - n2;
        const T xm = fused_src(v, om, n3), ym = fused_src(v, om + n3, n3), zm = fused_src(v, om + 2 * n3, n3);
        const T zim = (i + 1 < n) ? fused_src(v, om + 1 + 2 * n3, n3) : T(0);
        const T zjm = (j + 1 < n) ? fused_src(v, om + n + 2 * n3, n3) : T(0);
        bxm = (ym - zm) + (zjm - sk[1]);
        bym = (zm - xm) + (sk[0] - zim);
      }
      gsync();
      // inputs of plane ks+1, loaded ahead of use
      FusedLoadT<T> ld1;
      if (col && ks + 1 < n) fused_load(v, o + n2, n3, act && ks + 1 < ke, ld1);
      int buf = ks & 1;
      for (int k = ks; k < ke; ++k, o += n2) {
        const int nb = buf ^ 1;
        // own r_{i+1} of plane k+1 from the inputs loaded during the previous step
        T sk1[3] = {T(0), T(0), T(0)};
        if (col && k + 1 < n) fused_apply(v, o + n2, n3, act && k + 1 < ke, ld1, sk1);
#pragma unroll
        for (int c = 0; c < 3; ++c) sg.src[nb][c][w + 1][lane + 1] = sk1[c];
        // then issue the loads of plane k+2
        if (col && k + 2 < n && k + 1 < ke) fused_load(v, o + 2 * n2, n3, act && k + 2 < ke, ld1);
        // fluxes at plane k: own (k, k+1), x+1 and y+1 neighbours of plane k from smem
        const T yi = sg.src[buf][1][w + 1][lane + 2], zi = sg.src[buf][2][w + 1][lane + 2];
        const T xj = sg.src[buf][0][w + 2][lane + 1], zj = sg.src[buf][2][w + 2][lane + 1];
        const T bx = (sk[1] - sk[2]) + (zj - sk1[1]);
        const T by = (sk[2] - sk[0]) + (sk1[0] - zi);
        const T bz = (sk[0] - sk[1]) + (yi - xj);
        sg.fz[buf][w + 1][lane] = bz;
        sg.fx[buf][w + 1][lane] = bx;
        gsync();
        T bzi = shfl_up1(bz), byi = shfl_up1(by);
        if (lane == 0) { bzi = sg.hz[buf][w]; byi = sg.hy[buf][w]; }
        const T bzj = sg.fz[buf][w][lane], bxj = sg.fx[buf][w][lane];
        if (act) {
          const T tx = (bz - bzj) + (bym - by);
          const T ty = (bzi - bz) + (bx - bxm);
          const T tz = (bxj - bx) + (by - byi);
          unsigned m = mcol & (k > 0 ? 7u : 4u);
          if (incb && k >= g.cb_lo[2] && k < g.cb_hi[2]) m &= ~(unsigned)g.cflags[cfc + cw01 * (k - g.cb_lo[2])];
          const T t[3] = {tx, ty, tz};
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const T wv = (m >> c & 1u) ? t[c] : T(0);
            MQS_STC(v.w_out, o + c * n3, 3 * n3, 319, wv);
            gamma = fmaT(sk[c], sk[c], gamma);
            delta = fmaT(wv, sk[c], delta);
          }
        }
        bxm = bx; bym = by;
#pragma unroll
        for (int c = 0; c < 3; ++c) sk[c] = sk1[c];
        buf = nb;
      }
    } else if (HW == 2) {
      // two halo warps, as in sweep_fused_fx: hw 0 forms row j0-1 and column i0-1 of plane
      // k+1 and the halo fluxes of plane k; hw 1 row j0+kTY and column i0+32
      const int hw = w - kTY;
      constexpr int kHSlots = 34 + kTY;
      constexpr int kHPairs = 3 * kHSlots;
      constexpr int kHR = (kHPairs + 31) / 32;
      auto pair_pos = [&](int p, int& c, int& hi, int& hj, int& row, int& cl) {
        c = p / kHSlots;
        const int sl = p - c * kHSlots;
        if (sl < 34) { hi = i0 - 1 + sl; hj = hw ? j0 + kTY : j0 - 1; row = hw ? kTY + 1 : 0; cl = sl; }
        else { hi = hw ? i0 + 32 : i0 - 1; hj = j0 + (sl - 34); row = sl - 34 + 1; cl = hw ? 33 : 0; }
      };
      struct HaloIn2 { T r, w, s; };
      auto halo_load = [&](int kk, HaloIn2* hin) {
#pragma unroll
        for (int q = 0; q < kHR; ++q) {
          const int p = lane + 32 * q;
          int c = 0, hi = -1, hj = -1, row = 0, cl = 0;
          if (p < kHPairs) pair_pos(p, c, hi, hj, row, cl);
          const bool ok = p < kHPairs && hi >= 0 && hj >= 0 && hi < n && hj < n && kk >= 0 && kk < n;
          const int oo = ok ? hi + n * (hj + n * kk) + c * n3 : 0;
          hin[q].r = ok ? MQS_LDC(v.r_in, oo, 3 * n3, 340) : T(0);
          hin[q].w = ok ? MQS_LDC(v.w_in, oo, 3 * n3, 341) : T(0);
          hin[q].s = (ok && !v.first) ? MQS_LDC(v.s_in, oo, 3 * n3, 342) : T(0);
        }
      };
      auto halo_store = [&](const HaloIn2* hin, int bufw) {
#pragma unroll
        for (int q = 0; q < kHR; ++q) {
          const int p = lane + 32 * q;
          if (p >= kHPairs) continue;
          int c, hi, hj, row, cl;
          pair_pos(p, c, hi, hj, row, cl);
          const T sv = v.first ? hin[q].w : fmaT(v.beta, hin[q].s, hin[q].w);
          sg.src[bufw][c][row][cl] = fmaT(-v.alpha, sv, hin[q].r);
        }
      };
      HaloIn2 h[kHR], h1[kHR];
      halo_load(ks, h);
      halo_load(ks + 1, h1);
      halo_store(h, ks & 1);
#pragma unroll
      for (int q = 0; q < kHR; ++q) h[q] = h1[q];
      gsync();
      int buf = ks & 1;
      for (int k = ks; k < ke; ++k) {
        const int nb = buf ^ 1;
        halo_store(h, nb);                     // plane k+1, loaded during the previous step
        if (k + 2 <= ke) halo_load(k + 2, h);  // in flight until the next step
        if (hw == 0) {
          __syncwarp();
          const T x0 = sg.src[buf][0][0][lane + 1], y0 = sg.src[buf][1][0][lane + 1];
          const T z0 = sg.src[buf][2][0][lane + 1], yi = sg.src[buf][1][0][lane + 2];
          const T xj = sg.src[buf][0][1][lane + 1], zj = sg.src[buf][2][1][lane + 1];
          const T yk = sg.src[nb][1][0][lane + 1];
          const bool hrow = (j0 >= 1) && (i < n);
          sg.fz[buf][0][lane] = hrow ? (x0 - y0) + (yi - xj) : T(0);
          sg.fx[buf][0][lane] = hrow ? (y0 - z0) + (zj - yk) : T(0);
          if (lane < kTY) {
            const int r = lane + 1;
            const T cx0 = sg.src[buf][0][r][0], cy0 = sg.src[buf][1][r][0], cz0 = sg.src[buf][2][r][0];
            const T cyi = sg.src[buf][1][r][1], czi = sg.src[buf][2][r][1];
            const T cxj = sg.src[buf][0][r + 1][0];
            const T cxk = sg.src[nb][0][r][0];
            const bool hcol = (i0 >= 1) && (j0 + lane < n);
            sg.hz[buf][lane] = hcol ? (cx0 - cy0) + (cyi - cxj) : T(0);
            sg.hy[buf][lane] = hcol ? (cz0 - cx0) + (cxk - czi) : T(0);
          }
        }
        gsync();
        buf = nb;
      }
    } else {
      // halo warp: r_{i+1} on the tile halo of plane k+1 (rows j0-1 and j0+kTY
      // over columns i0-1..i0+32, columns i0-1 and i0+32 over the tile rows),
      // then the halo fluxes of plane k: row j0-1 (bz, bx) and column i0-1 (bz, by)
      constexpr int kSlots = 2 * 34 + 2 * kTY;
      auto slot_pos = [&](int sl, int& hi, int& hj, int& row, int& cl) {
        if (sl < 34) { hi = i0 - 1 + sl; hj = j0 - 1; row = 0; cl = sl; }
        else if (sl < 68) { hi = i0 - 1 + (sl - 34); hj = j0 + kTY; row = kTY + 1; cl = sl - 34; }
        else if (sl < 68 + kTY) { hi = i0 - 1; hj = j0 + (sl - 68); row = sl - 68 + 1; cl = 0; }
        else { hi = i0 + 32; hj = j0 + (sl - 68 - kTY); row = sl - 68 - kTY + 1; cl = 33; }
      };
      // per lane up to three halo slots; their (r, w, s) inputs are loaded one
      // plane ahead of use
      constexpr int kHS = (kSlots + 31) / 32;
      struct HaloIn { T r[3], w[3], s[3]; };
      auto halo_load = [&](int kk, HaloIn* hin) {
#pragma unroll
        for (int q = 0; q < kHS; ++q) {
          const int sl = lane + 32 * q;
          int hi = -1, hj = -1, row = 0, cl = 0;
          if (sl < kSlots) slot_pos(sl, hi, hj, row, cl);
          const bool ok = sl < kSlots && hi >= 0 && hj >= 0 && hi < n && hj < n && kk >= 0 && kk < n;
          const int oo = ok ? hi + n * (hj + n * kk) : 0;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            hin[q].r[c] = ok ? MQS_LDC(v.r_in, oo + c * n3, 3 * n3, 325) : T(0);
            hin[q].w[c] = ok ? MQS_LDC(v.w_in, oo + c * n3, 3 * n3, 326) : T(0);
            hin[q].s[c] = (ok && !v.first) ? MQS_LDC(v.s_in, oo + c * n3, 3 * n3, 327) : T(0);
          }
        }
      };
      auto halo_store = [&](const HaloIn* hin, int bufw) {
#pragma unroll
        for (int q = 0; q < kHS; ++q) {
          const int sl = lane + 32 * q;
          if (sl >= kSlots) continue;
          int hi, hj, row, cl;
          slot_pos(sl, hi, hj, row, cl);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const T sv = v.first ? hin[q].w[c] : fmaT(v.beta, hin[q].s[c], hin[q].w[c]);
            sg.src[bufw][c][row][cl] = fmaT(-v.alpha, sv, hin[q].r[c]);
          }
        }
      };
      // consume a plane's inputs, then reuse the registers for the next loads
      HaloIn h[kHS];
      halo_load(ks, h);
      halo_store(h, ks & 1);
      halo_load(ks + 1, h);
      gsync();
      int buf = ks & 1;
      for (int k = ks; k < ke; ++k) {
        const int nb = buf ^ 1;
        halo_store(h, nb);                     // plane k+1, loaded during the previous step
        if (k + 2 <= ke) halo_load(k + 2, h);  // in flight until the next step
        __syncwarp();
        // row j0-1 at column i: bz = x + y(i+1) - x(j0) - y ; bx = y + z(j0) - y(k+1) - z
        {
          const T x0 = sg.src[buf][0][0][lane + 1], y0 = sg.src[buf][1][0][lane + 1];
          const T z0 = sg.src[buf][2][0][lane + 1], yi = sg.src[buf][1][0][lane + 2];
          const T xj = sg.src[buf][0][1][lane + 1], zj = sg.src[buf][2][1][lane + 1];
          const T yk = sg.src[nb][1][0][lane + 1];
          const bool hrow = (j0 >= 1) && (i < n);
          sg.fz[buf][0][lane] = hrow ? (x0 - y0) + (yi - xj) : T(0);
          sg.fx[buf][0][lane] = hrow ? (y0 - z0) + (zj - yk) : T(0);
        }
        // column i0-1 at row r: bz = x + y(i0) - x(j+1) - y ; by = z + x(k+1) - z(i0) - x
        if (lane < kTY) {
          const int r = lane + 1;
          const T x0 = sg.src[buf][0][r][0], y0 = sg.src[buf][1][r][0], z0 = sg.src[buf][2][r][0];
          const T yi = sg.src[buf][1][r][1], zi = sg.src[buf][2][r][1];
          const T xj = sg.src[buf][0][r + 1][0];
          const T xk = sg.src[nb][0][r][0];
          const bool hcol = (i0 >= 1) && (j0 + lane < n);
          sg.hz[buf][lane] = hcol ? (x0 - y0) + (yi - xj) : T(0);
          sg.hy[buf][lane] = hcol ? (z0 - x0) + (xk - zi) : T(0);
        }
        gsync();
        buf = nb;
      }
    }
  }
}

// ---- the FP64 one-reduction pass with the stencil in 64-bit fixed point ------------
// As sweep_fused for T = double, but the shared stencil sources are the integers
// R = round(r_{i+1} 2^sh_in) (fx_from_double; every |r_{i+1}| < 2^(58 - sh_in - 1) by the
// bound the kernel derives from the previous reduction), the face fluxes and L R are
// exact 64-bit integer sums, and w_{i+1} = (L R) 2^sh_out is rounded once (sh_out =
// -sh_in).  r_{i+1} is formed in FP64 (the FMAs of fused_apply / fused_src) by its owner,
// and by the halo warp for the tile halo, bitwise the same in both; gamma and delta
// are FP64 sums of the FP64 r_{i+1} and w_{i+1}.  Besides them the pass returns the
// largest biased FP64 exponents over the owned values of r_{i+1}, w_{i+1} and s_i, from
// which the next pass's scale is bounded.
struct FusedFxVecs {
  FusedVecs v;
  int sh_in, sh_out;
};
struct FusedFxSmem {
  long long src[2][3][kTY + 2][34];
  long long fz[2][kTY + 1][32];
  long long fx[2][kTY + 1][32];
  long long hz[2][kTY];
  long long hy[2][kTY];
};
template <int G = kGroups>
struct FusedFxSmemBlockG { FusedFxSmem g[G]; };
using FusedFxSmemBlock = FusedFxSmemBlockG<>;

// biased FP64 exponent field of v (|v| < 2^(e - 1022) for e > 0; 0 for zero and subnormals)
__device__ __forceinline__ int fx_expo(double v) { return (int)((__double_as_longlong(v) >> 52) & 0x7FF); }

// ptab (nullable): plane-tile range [x, y) of every group part (part * G + group), from
// fused_partition; else the even split of the formula below.
// HW: halo warps per group.  1: warp kTY of each group forms the whole tile halo.  2: the
// block has G more warps after the G x kGroupWarps (warp G kGroupWarps + grp is group grp's
// second halo warp); the first forms row j0-1 and column i0-1 of the halo and the halo
// fluxes, the second row j0+kTY and column i0+32, each over its (position, component)
// pairs packed 32 to a round.  With G = 2 that is 12 warps, three on each of the SM's four
// schedulers, each issuing about the same number of FP64 instructions per plane.
template <int G, int HW = 1>
__device__ inline void sweep_fused_fx(const Geom& g, const FusedFxVecs& fv, const Box& box, int part, int nparts,
                               FusedFxSmemBlockG<G>& smb, double& gamma, double& delta, int& mer, int& mew,
                               int& mes, const int2* ptab = nullptr) {
  static_assert(HW == 1 || HW == 2, "one or two halo warps per group");
  const FusedVecs& v = fv.v;
  const int shi = fv.sh_in, sho = fv.sh_out;
  const int n = g.n;
  const int n2 = n * n;
  const int n3 = (int)g.n3;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool extra = HW == 2 && warp >= G * kGroupWarps;     // a second halo warp
  const int grp = extra ? warp - G * kGroupWarps : warp / kGroupWarps;
  const int w = extra ? kTY + 1 : warp % kGroupWarps;
  auto gsync = [&] {
    if (HW == 1) group_sync(grp);
    else group_sync_n<kGroupWarps + 1>(grp);
  };
  FusedFxSmem& sg = smb.g[grp];
  const int bx0 = box.hi[0] - box.lo[0], by0 = box.hi[1] - box.lo[1], nz = box.hi[2] - box.lo[2];
  if (bx0 <= 0 || by0 <= 0 || nz <= 0) return;
  const int ntx = (bx0 + 31) / 32, nty = (by0 + kTY - 1) / kTY;
  const long long ntiles = (long long)ntx * nty * nz;
  const long long gp = (long long)part * G + grp, gn = (long long)nparts * G;
  long long u = ptab ? (long long)ptab[gp].x : ntiles * gp / gn;
  const long long u1 = ptab ? (long long)ptab[gp].y : ntiles * (gp + 1) / gn;
  const int cw0 = g.cb_hi[0] - g.cb_lo[0], cw01 = cw0 * (g.cb_hi[1] - g.cb_lo[1]);
  // owned position: the FP64 update of fused_apply, the exponents of r_{i+1} and s_i
  auto own_apply = [&](int o, const FusedLoadT<double>& L, double* rn) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double sv = v.first ? L.w[c] : fma(v.beta, L.s[c], L.w[c]);
      const double r1 = fma(-v.alpha, sv, L.r[c]);
      const int e = o + c * n3;
      const double pv = v.first ? L.r[c] : fma(v.beta, L.p[c], L.r[c]);
      MQS_STC(v.s_out, e, 3 * n3, 321, sv);
      MQS_STC(v.p, e, 3 * n3, 322, pv);
      MQS_STC(v.x, e, 3 * n3, 323, fma(v.alpha, pv, L.x[c]));
      MQS_STC(v.r_out, e, 3 * n3, 324, r1);
      rn[c] = r1;
      mes = max(mes, fx_expo(sv));
      mer = max(mer, fx_expo(r1));
    }
  };
  // r_{i+1} of a position this group does not own (no writes)
  auto other_apply = [&](const FusedLoadT<double>& L, double* rn) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double sv = v.first ? L.w[c] : fma(v.beta, L.s[c], L.w[c]);
      rn[c] = fma(-v.alpha, sv, L.r[c]);
    }
  };
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
    gsync();  // smem reuse across segments
    if (w < kTY) {
      const int j = j0 + w;
      const bool act = (i < box.hi[0]) && (j < box.hi[1]);   // owned position
      const bool col = (i < n) && (j < n);
      const unsigned mcol = (j > 0 ? 1u : 0u) | (i > 0 ? 2u : 0u) | ((i > 0 && j > 0) ? 4u : 0u);
      const bool incb = i >= g.cb_lo[0] && i < g.cb_hi[0] && j >= g.cb_lo[1] && j < g.cb_hi[1];
      const int cfc = incb ? (i - g.cb_lo[0]) + cw0 * (j - g.cb_lo[1]) : 0;
      int o = col ? i + n * (j + n * ks) : 0;
      // prologue: plane ks (owned: updated), warm-up fluxes at ks - 1 from recomputed sources;
      // the warm-up plane's inputs (x, y, z at the position, z at i+1 and at j+1) are loaded
      // together with plane ks, before the update's stores
      double skd[3] = {0.0, 0.0, 0.0};
      long long sk[3] = {0, 0, 0};
      const bool wu = ks >= 1 && col;
      long long wm[5] = {0, 0, 0, 0, 0};   // the warm-up plane's r_{i+1}, as fused_src forms it
      if (col) {
        FusedLoadT<double> L0;
        fused_load(v, o, n3, act, L0);
        if (wu) {
          const int om = o - n2;
          double wr[5] = {}, ww[5] = {}, ws[5] = {};
#pragma unroll
          for (int q = 0; q < 5; ++q) {
            const bool okq = q < 3 || (q == 3 ? i + 1 < n : j + 1 < n);
            const int oq = q < 3 ? om + q * n3 : (q == 3 ? om + 1 + 2 * n3 : om + n + 2 * n3);
            if (okq) {
              ww[q] = MQS_LDC(v.w_in, oq, 3 * n3, 337);
              ws[q] = v.first ? 0.0 : MQS_LDC(v.s_in, oq, 3 * n3, 338);
              wr[q] = MQS_LDC(v.r_in, oq, 3 * n3, 339);
            }
          }
#pragma unroll
          for (int q = 0; q < 5; ++q) {
            const bool okq = q < 3 || (q == 3 ? i + 1 < n : j + 1 < n);
            const double sv = v.first ? ww[q] : fma(v.beta, ws[q], ww[q]);
            wm[q] = okq ? fx_from_double(fma(-v.alpha, sv, wr[q]), shi) : 0;
          }
        }
        if (act) own_apply(o, L0, skd);
        else other_apply(L0, skd);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        sk[c] = fx_from_double(skd[c], shi);
        sg.src[ks & 1][c][w + 1][lane + 1] = sk[c];
      }
      long long bxm = 0, bym = 0;
      if (wu) {
        bxm = (wm[1] - wm[2]) + (wm[4] - sk[1]);
        bym = (wm[2] - wm[0]) + (sk[0] - wm[3]);
      }
      // inputs of plane ks+1 (nobody else writes them), in flight across the barrier
      FusedLoadT<double> ld1;
      if (col && ks + 1 < n) fused_load(v, o + n2, n3, act && ks + 1 < ke, ld1);
      gsync();
      int buf = ks & 1;
      for (int k = ks; k < ke; ++k, o += n2) {
        const int nb = buf ^ 1;
        // own r_{i+1} of plane k+1 from the inputs loaded during the previous step
        double sk1d[3] = {0.0, 0.0, 0.0};
        if (col && k + 1 < n) {
          if (act && k + 1 < ke) own_apply(o + n2, ld1, sk1d);
          else other_apply(ld1, sk1d);
        }
        long long sk1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          sk1[c] = fx_from_double(sk1d[c], shi);
          sg.src[nb][c][w + 1][lane + 1] = sk1[c];
        }
        // then issue the loads of plane k+2
        if (col && k + 2 < n && k + 1 < ke) fused_load(v, o + 2 * n2, n3, act && k + 2 < ke, ld1);
        // conductor flags of plane k (edges of K_c), loaded ahead of their use after the barrier
        const unsigned cfk = (act && incb && k >= g.cb_lo[2] && k < g.cb_hi[2])
                                 ? (unsigned)g.cflags[cfc + cw01 * (k - g.cb_lo[2])]
                                 : 0u;
        const long long yi = sg.src[buf][1][w + 1][lane + 2], zi = sg.src[buf][2][w + 1][lane + 2];
        const long long xj = sg.src[buf][0][w + 2][lane + 1], zj = sg.src[buf][2][w + 2][lane + 1];
        const long long bx = (sk[1] - sk[2]) + (zj - sk1[1]);
        const long long by = (sk[2] - sk[0]) + (sk1[0] - zi);
        const long long bz = (sk[0] - sk[1]) + (yi - xj);
        sg.fz[buf][w + 1][lane] = bz;
        sg.fx[buf][w + 1][lane] = bx;
        // gamma needs only this plane's r_{i+1}: summed before the barrier
        if (act) {
#pragma unroll
          for (int c = 0; c < 3; ++c) gamma = fma(skd[c], skd[c], gamma);
        }
        gsync();
        long long bzi = shfl_up1(bz), byi = shfl_up1(by);
        if (lane == 0) { bzi = sg.hz[buf][w]; byi = sg.hy[buf][w]; }
        const long long bzj = sg.fz[buf][w][lane], bxj = sg.fx[buf][w][lane];
        if (act) {
          const long long t[3] = {(bz - bzj) + (bym - by), (bzi - bz) + (bx - bxm), (bxj - bx) + (by - byi)};
          const unsigned m = mcol & (k > 0 ? 7u : 4u) & ~cfk;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const double wv = (m >> c & 1u) ? fx_to_double(t[c], sho) : 0.0;
            MQS_STC(v.w_out, o + c * n3, 3 * n3, 320, wv);
            delta = fma(wv, skd[c], delta);
            mew = max(mew, fx_expo(wv));
          }
        }
        bxm = bx; bym = by;
#pragma unroll
        for (int c = 0; c < 3; ++c) { sk[c] = sk1[c]; skd[c] = sk1d[c]; }
        buf = nb;
      }
    } else if (HW == 2) {
      // two halo warps: hw 0 forms rows j0-1 (columns i0-1 .. i0+32) and column i0-1 (rows
      // j0 .. j0+kTY-1) of plane k+1 and the halo fluxes of plane k, which need only its own
      // plane k+1 values; hw 1 forms row j0+kTY and column i0+32, read from plane k on
      const int hw = w - kTY;
      constexpr int kHSlots = 34 + kTY;
      constexpr int kHPairs = 3 * kHSlots;
      constexpr int kHR = (kHPairs + 31) / 32;
      // pair p: component p / kHSlots at the warp's slot p % kHSlots
      auto pair_pos = [&](int p, int& c, int& hi, int& hj, int& row, int& cl) {
        c = p / kHSlots;
        const int sl = p - c * kHSlots;
        if (sl < 34) { hi = i0 - 1 + sl; hj = hw ? j0 + kTY : j0 - 1; row = hw ? kTY + 1 : 0; cl = sl; }
        else { hi = hw ? i0 + 32 : i0 - 1; hj = j0 + (sl - 34); row = sl - 34 + 1; cl = hw ? 33 : 0; }
      };
      struct HaloIn2 { double r, w, s; };
      auto halo_load = [&](int kk, HaloIn2* hin) {
#pragma unroll
        for (int q = 0; q < kHR; ++q) {
          const int p = lane + 32 * q;
          int c = 0, hi = -1, hj = -1, row = 0, cl = 0;
          if (p < kHPairs) pair_pos(p, c, hi, hj, row, cl);
          const bool ok = p < kHPairs && hi >= 0 && hj >= 0 && hi < n && hj < n && kk >= 0 && kk < n;
          const int oo = ok ? hi + n * (hj + n * kk) + c * n3 : 0;
          hin[q].r = ok ? MQS_LDC(v.r_in, oo, 3 * n3, 334) : 0.0;
          hin[q].w = ok ? MQS_LDC(v.w_in, oo, 3 * n3, 335) : 0.0;
          hin[q].s = (ok && !v.first) ? MQS_LDC(v.s_in, oo, 3 * n3, 336) : 0.0;
        }
      };
      auto halo_store = [&](const HaloIn2* hin, int bufw) {
#pragma unroll
        for (int q = 0; q < kHR; ++q) {
          const int p = lane + 32 * q;
          if (p >= kHPairs) continue;
          int c, hi, hj, row, cl;
          pair_pos(p, c, hi, hj, row, cl);
          const double sv = v.first ? hin[q].w : fma(v.beta, hin[q].s, hin[q].w);
          sg.src[bufw][c][row][cl] = fx_from_double(fma(-v.alpha, sv, hin[q].r), shi);
        }
      };
      // planes ks and ks+1 loaded together
      HaloIn2 h[kHR], h1[kHR];
      halo_load(ks, h);
      halo_load(ks + 1, h1);
      halo_store(h, ks & 1);
#pragma unroll
      for (int q = 0; q < kHR; ++q) h[q] = h1[q];
      gsync();
      int buf = ks & 1;
      for (int k = ks; k < ke; ++k) {
        const int nb = buf ^ 1;
        halo_store(h, nb);                     // plane k+1, loaded during the previous step
        if (k + 2 <= ke) halo_load(k + 2, h);  // in flight until the next step
        if (hw == 0) {
          __syncwarp();
          // row j0-1 and column i0-1 fluxes of plane k, as for one halo warp
          const long long x0 = sg.src[buf][0][0][lane + 1], y0 = sg.src[buf][1][0][lane + 1];
          const long long z0 = sg.src[buf][2][0][lane + 1], yi = sg.src[buf][1][0][lane + 2];
          const long long xj = sg.src[buf][0][1][lane + 1], zj = sg.src[buf][2][1][lane + 1];
          const long long yk = sg.src[nb][1][0][lane + 1];
          const bool hrow = (j0 >= 1) && (i < n);
          sg.fz[buf][0][lane] = hrow ? (x0 - y0) + (yi - xj) : 0;
          sg.fx[buf][0][lane] = hrow ? (y0 - z0) + (zj - yk) : 0;
          if (lane < kTY) {
            const int r = lane + 1;
            const long long cx0 = sg.src[buf][0][r][0], cy0 = sg.src[buf][1][r][0], cz0 = sg.src[buf][2][r][0];
            const long long cyi = sg.src[buf][1][r][1], czi = sg.src[buf][2][r][1];
            const long long cxj = sg.src[buf][0][r + 1][0];
            const long long cxk = sg.src[nb][0][r][0];
            const bool hcol = (i0 >= 1) && (j0 + lane < n);
            sg.hz[buf][lane] = hcol ? (cx0 - cy0) + (cyi - cxj) : 0;
            sg.hy[buf][lane] = hcol ? (cz0 - cx0) + (cxk - czi) : 0;
          }
        }
        gsync();
        buf = nb;
      }
    } else {
      // halo warp, as in sweep_fused: r_{i+1} on the tile halo of plane k+1 (converted to
      // the fixed point), then the halo fluxes of plane k
      constexpr int kSlots = 2 * 34 + 2 * kTY;
      auto slot_pos = [&](int sl, int& hi, int& hj, int& row, int& cl) {
        if (sl < 34) { hi = i0 - 1 + sl; hj = j0 - 1; row = 0; cl = sl; }
        else if (sl < 68) { hi = i0 - 1 + (sl - 34); hj = j0 + kTY; row = kTY + 1; cl = sl - 34; }
        else if (sl < 68 + kTY) { hi = i0 - 1; hj = j0 + (sl - 68); row = sl - 68 + 1; cl = 0; }
        else { hi = i0 + 32; hj = j0 + (sl - 68 - kTY); row = sl - 68 - kTY + 1; cl = 33; }
      };
      constexpr int kHS = (kSlots + 31) / 32;
      struct HaloIn { double r[3], w[3], s[3]; };
      auto halo_load = [&](int kk, HaloIn* hin) {
#pragma unroll
        for (int q = 0; q < kHS; ++q) {
          const int sl = lane + 32 * q;
          int hi = -1, hj = -1, row = 0, cl = 0;
          if (sl < kSlots) slot_pos(sl, hi, hj, row, cl);
          const bool ok = sl < kSlots && hi >= 0 && hj >= 0 && hi < n && hj < n && kk >= 0 && kk < n;
          const int oo = ok ? hi + n * (hj + n * kk) : 0;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            hin[q].r[c] = ok ? MQS_LDC(v.r_in, oo + c * n3, 3 * n3, 328) : 0.0;
            hin[q].w[c] = ok ? MQS_LDC(v.w_in, oo + c * n3, 3 * n3, 329) : 0.0;
            hin[q].s[c] = (ok && !v.first) ? MQS_LDC(v.s_in, oo + c * n3, 3 * n3, 330) : 0.0;
          }
        }
      };
      auto halo_store = [&](const HaloIn* hin, int bufw) {
#pragma unroll
        for (int q = 0; q < kHS; ++q) {
          const int sl = lane + 32 * q;
          if (sl >= kSlots) continue;
          int hi, hj, row, cl;
          slot_pos(sl, hi, hj, row, cl);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const double sv = v.first ? hin[q].w[c] : fma(v.beta, hin[q].s[c], hin[q].w[c]);
            sg.src[bufw][c][row][cl] = fx_from_double(fma(-v.alpha, sv, hin[q].r[c]), shi);
          }
        }
      };
      HaloIn h[kHS];
      halo_load(ks, h);
      halo_store(h, ks & 1);
      halo_load(ks + 1, h);
      gsync();
      int buf = ks & 1;
      for (int k = ks; k < ke; ++k) {
        const int nb = buf ^ 1;
        halo_store(h, nb);                     // plane k+1, loaded during the previous step
        if (k + 2 <= ke) halo_load(k + 2, h);  // in flight until the next step
        __syncwarp();
        {
          const long long x0 = sg.src[buf][0][0][lane + 1], y0 = sg.src[buf][1][0][lane + 1];
          const long long z0 = sg.src[buf][2][0][lane + 1], yi = sg.src[buf][1][0][lane + 2];
          const long long xj = sg.src[buf][0][1][lane + 1], zj = sg.src[buf][2][1][lane + 1];
          const long long yk = sg.src[nb][1][0][lane + 1];
          const bool hrow = (j0 >= 1) && (i < n);
          sg.fz[buf][0][lane] = hrow ? (x0 - y0) + (yi - xj) : 0;
          sg.fx[buf][0][lane] = hrow ? (y0 - z0) + (zj - yk) : 0;
        }
        if (lane < kTY) {
          const int r = lane + 1;
          const long long x0 = sg.src[buf][0][r][0], y0 = sg.src[buf][1][r][0], z0 = sg.src[buf][2][r][0];
          const long long yi = sg.src[buf][1][r][1], zi = sg.src[buf][2][r][1];
          const long long xj = sg.src[buf][0][r + 1][0];
          const long long xk = sg.src[nb][0][r][0];
          const bool hcol = (i0 >= 1) && (j0 + lane < n);
          sg.hz[buf][lane] = hcol ? (x0 - y0) + (yi - xj) : 0;
          sg.hy[buf][lane] = hcol ? (z0 - x0) + (xk - zi) : 0;
        }
        gsync();
        buf = nb;
      }
    }
  }
}

}  // namespace mqs
