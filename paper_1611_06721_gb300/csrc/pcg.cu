// Jacobi-preconditioned CG for K_n x = b (Sec. III, eq. (mrhs)) as one
// persistent cooperative kernel per solve.
//
// K_n = (nu0/h) L with the integer stencil L and diag(K_n) = 4 nu0/h on every
// n-edge, so Jacobi-PCG on (K_n, b) produces the same iterates as CG on
// (L, b h/nu0); the kernel runs the latter (no preconditioner multiply, no
// stencil scaling).  Per iteration, with one grid barrier after each of the
// two reductions of the Hestenes-Stiefel recurrences:
//   phase A  t = L r;  q = t + beta q;  p = r + beta p;  pq = p.q
//            (q = L p by linearity, so the stencil reads r, which is final;
//            t is formed exactly in 64-bit fixed point on the integer pipes,
//            with r rounded once to 2^(E-58), |r_i| < 2^(E-1), and t rounded
//            once back to FP64: see fx_from_double in mqs_internal.cuh)
//   phase B  x += alpha p;  r -= alpha q;  rr = r.r
// Convergence ||r|| <= tol ||b|| is confirmed on the true residual b - L x,
// whose stencil output L x is kept for the start-vector history.
#include <cmath>
#include <vector>
#include "mqs_internal.cuh"
#include "mqs_kernels.h"
#include "pcg_fused.cuh"

namespace mqs {

struct PcgArgs {
  Geom g;
  Box full;
  const double* b;
  double* x;
  double* r;
  double* p;
  double* q;
  double* lx;
  double* part;       // 4 * 2 * nblk partial sums
  unsigned* bar;      // barrier counter (zero at launch)
  int* err;           // device error word (zero at launch)
  PcgResult* out;
  double tol2;
  int maxit;
  long long spin;
  int init;           // 0: r = b - L x (stencil); 1: r given (start vector's image known); 2: x = 0, r = b
  const int* halt;    // nullable: nonzero = an earlier step of the stepping call failed, skip the solve
};

// A solve inside a halted stepping call returns at once (every block reads the same
// word before any grid barrier) with a zero-iteration result the record kernel ignores.
__device__ __forceinline__ bool pcg_halted(const int* halt, PcgResult* out) {
  if (!halt || *(volatile const int*)halt == 0) return false;
  if (blockIdx.x == 0 && threadIdx.x == 0) *out = PcgResult{0, MQS_OK, 0.0, 0.0};
  return true;
}

struct EpiResidual {  // r = b - t, lx = t on n-edges; sums r.r and b.b
  const double* b; double* r; double* lx; long long n3;
  double rr = 0.0, bb = 0.0;
  double bp[3];
  __device__ void prefetch(long long e) {
#pragma unroll
    for (int c = 0; c < 3; ++c) bp[c] = MQS_LDC(b, e + c * n3, 3 * n3, 201);
  }
  __device__ void operator()(long long e, unsigned m, double tx, double ty, double tz, double, double, double) {
    const double t[3] = {tx, ty, tz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long idx = e + c * n3;
      if (m >> c & 1u) {
        const double bv = bp[c];
        const double rv = bv - t[c];
        MQS_STC(r, idx, 3 * n3, 202, rv); MQS_STC(lx, idx, 3 * n3, 203, t[c]);
        rr = fma(rv, rv, rr); bb = fma(bv, bv, bb);
      } else {
        MQS_STC(r, idx, 3 * n3, 204, 0.0); MQS_STC(lx, idx, 3 * n3, 205, 0.0);
      }
    }
  }
};

// The direction sweep of the FP64 kernel: t = L r formed exactly in 64-bit fixed point
// (sweep_L with LoadFx: r_i -> round(r_i 2^(58-E)), E from ||r||^2, see fx_exponent),
// converted back once (t 2^(E-58)); then q = t + beta q, p = r + beta p on n-edges and
// p.q, in FP64.  The FP64 r for p is loaded here (the sweep's source values are the
// fixed-point ones).
struct EpiDirectionFx {
  double* p; double* q; const double* r; long long n3; double beta; bool first; int sh;
  double pq = 0.0;
  double pp[3], qp[3], rp[3];
  __device__ void prefetch(long long e) {
#pragma unroll
    for (int c = 0; c < 3; ++c) rp[c] = MQS_LDC(r, e + c * n3, 3 * n3, 206);
    if (first) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      pp[c] = MQS_LDC(p, e + c * n3, 3 * n3, 207);
      qp[c] = MQS_LDC(q, e + c * n3, 3 * n3, 208);
    }
  }
  __device__ void operator()(long long e, unsigned m, long long tx, long long ty, long long tz, long long,
                             long long, long long) {
    const long long t[3] = {tx, ty, tz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long idx = e + c * n3;
      double qn = 0.0, pn = 0.0;
      if (m >> c & 1u) {
        const double tc = fx_to_double(t[c], sh);
        qn = first ? tc : fma(beta, qp[c], tc);
        pn = first ? rp[c] : fma(beta, pp[c], rp[c]);
        pq = fma(pn, qn, pq);
      }
      MQS_STC(q, idx, 3 * n3, 209, qn); MQS_STC(p, idx, 3 * n3, 210, pn);
    }
  }
};

// BPS co-resident blocks per SM: 2 once the vectors are far beyond L2 (there 20 warps
// per SM hide more of the plane-sync and memory latency than 10; measured 236 -> 191 us
// per iteration at 128^3), 1 while they stay in L2 (64^3: the extra blocks only add
// barrier arrivals and partials).
template <int BPS>
__global__ void __launch_bounds__(kBlock, BPS) pcg_kernel(PcgArgs a) {
  if (pcg_halted(a.halt, a.out)) return;
  __shared__ union {
    SweepSmem d;                      // FP64 sweeps (residuals)
    SweepSmemT<long long> fx;         // the fixed-point direction sweep
  } smu;
  SweepSmem& sm = smu.d;
  __shared__ double red[32];
  __shared__ double gs[2];
  const int nb = gridDim.x, bid = blockIdx.x;
  unsigned nbar = 0;
  int slot = 0;
  const long long len = 3 * a.g.n3;
  const long long tid = (long long)bid * blockDim.x + threadIdx.x, nth = (long long)nb * blockDim.x;

  // reduction helper: block sums -> partial slots -> barrier -> global sums
  auto reduce2 = [&](double v0, double v1, double& s0, double& s1) -> bool {
    return grid_sum2<double>(v0, v1, s0, s1, a.part, slot, nbar, a.bar, a.spin, a.err, red, gs);
  };

  int status = MQS_OK, it = 0;
  double rr = 0.0, bb = 0.0, start_rel = 0.0, relres = 0.0;
  // initial residual
  if (a.init == 0) {            // r = b - L x0 by the stencil
    EpiResidual ep{a.b, a.r, a.lx, a.g.n3};
    sweep_L(a.g, a.x, a.full, bid, nb, sm, ep);
    if (!reduce2(ep.rr, ep.bb, rr, bb)) return;
  } else {                      // r given (init 1) or x0 = 0 so r = b (init 2): sums only
    double s0 = 0.0, s1 = 0.0;
    for (long long e = tid; e < len; e += nth) {
      const double be = a.b[e];
      double re;
      if (a.init == 2) { re = be; a.r[e] = be; a.x[e] = 0.0; } else { re = a.r[e]; }
      s0 = fma(re, re, s0);
      s1 = fma(be, be, s1);
    }
    if (!reduce2(s0, s1, rr, bb)) return;
  }
  if (bb == 0.0) {  // zero right-hand side: x = 0 after 0 iterations
    for (long long e = tid; e < len; e += nth) { a.x[e] = 0.0; a.r[e] = 0.0; a.lx[e] = 0.0; }
    if (bid == 0 && threadIdx.x == 0) *a.out = PcgResult{0, MQS_OK, 0.0, 0.0};
    return;
  }
  start_rel = sqrt(rr / bb);
  bool need_true = false;
  if (a.init != 0 && isfinite(rr) && isfinite(bb) && rr <= a.tol2 * bb) {
    // the start vector's residual came from stored images: confirm it on the
    // true residual (which also yields L x for the history)
    EpiResidual ep{a.b, a.r, a.lx, a.g.n3};
    sweep_L(a.g, a.x, a.full, bid, nb, sm, ep);
    double rt, bt;
    if (!reduce2(ep.rr, ep.bb, rt, bt)) return;
    if (rt <= a.tol2 * bb) {
      if (bid == 0 && threadIdx.x == 0) *a.out = PcgResult{0, MQS_OK, sqrt(rt / bb), start_rel};
      return;
    }
    rr = rt;   // iterate from the true residual
  }
  if (!isfinite(rr) || !isfinite(bb)) {
    status = MQS_ERR_NAN;
  } else if (rr > a.tol2 * bb) {
    double beta = 0.0;
    bool first = true;
    int restarts = 0;
    for (;;) {
      double pq = 0.0, dummy;
      {
        // every |r_i| <= ||r||_2 < 2^(E-1): the stencil runs exactly in 64-bit integers
        const int E = fx_exponent(rr);
        EpiDirectionFx ep{a.p, a.q, a.r, a.g.n3, beta, first, E - 58};
        sweep_L(a.g, a.r, a.full, bid, nb, smu.fx, ep, LoadFx{58 - E});
        if (!reduce2(ep.pq, 0.0, pq, dummy)) return;
      }
      ++it;
      if (!(pq > 0.0)) { status = isnan(pq) ? MQS_ERR_NAN : MQS_ERR_BREAKDOWN; need_true = true; break; }
      const double alpha = rr / pq;
      double rn = 0.0;
      {
        // x += alpha p, r -= alpha q over the whole layout, two double2 per thread per pass
        double acc0 = 0.0, acc1 = 0.0;
        const long long half = len >> 1;
        double2* x2 = reinterpret_cast<double2*>(a.x);
        double2* r2 = reinterpret_cast<double2*>(a.r);
        const double2* p2 = reinterpret_cast<const double2*>(a.p);
        const double2* q2 = reinterpret_cast<const double2*>(a.q);
        long long e = tid;
        for (; e + nth < half; e += 2 * nth) {
          const double2 pa = p2[e], qa = q2[e], xa = x2[e], ra = r2[e];
          const double2 pb = p2[e + nth], qb = q2[e + nth], xb = x2[e + nth], rb = r2[e + nth];
          double2 xo, ro;
          xo.x = fma(alpha, pa.x, xa.x); xo.y = fma(alpha, pa.y, xa.y);
          ro.x = fma(-alpha, qa.x, ra.x); ro.y = fma(-alpha, qa.y, ra.y);
          x2[e] = xo; r2[e] = ro;
          acc0 = fma(ro.x, ro.x, acc0); acc1 = fma(ro.y, ro.y, acc1);
          xo.x = fma(alpha, pb.x, xb.x); xo.y = fma(alpha, pb.y, xb.y);
          ro.x = fma(-alpha, qb.x, rb.x); ro.y = fma(-alpha, qb.y, rb.y);
          x2[e + nth] = xo; r2[e + nth] = ro;
          acc0 = fma(ro.x, ro.x, acc0); acc1 = fma(ro.y, ro.y, acc1);
        }
        for (; e < half; e += nth) {
          const double2 pa = p2[e], qa = q2[e], xa = x2[e], ra = r2[e];
          double2 xo, ro;
          xo.x = fma(alpha, pa.x, xa.x); xo.y = fma(alpha, pa.y, xa.y);
          ro.x = fma(-alpha, qa.x, ra.x); ro.y = fma(-alpha, qa.y, ra.y);
          x2[e] = xo; r2[e] = ro;
          acc0 = fma(ro.x, ro.x, acc0); acc1 = fma(ro.y, ro.y, acc1);
        }
        if ((len & 1) && tid == 0) {
          const long long t = len - 1;
          a.x[t] = fma(alpha, a.p[t], a.x[t]);
          const double re = fma(-alpha, a.q[t], a.r[t]);
          a.r[t] = re;
          acc0 = fma(re, re, acc0);
        }
        if (!reduce2(acc0 + acc1, 0.0, rn, dummy)) return;
      }
      if (!isfinite(rn)) { status = MQS_ERR_NAN; need_true = true; break; }
      if (rn <= a.tol2 * bb) {
        EpiResidual ep{a.b, a.r, a.lx, a.g.n3};
        sweep_L(a.g, a.x, a.full, bid, nb, sm, ep);
        double rt, bt;
        if (!reduce2(ep.rr, ep.bb, rt, bt)) return;
        if (rt <= a.tol2 * bb || restarts >= 8) {
          relres = sqrt(rt / bb);
          status = (rt <= a.tol2 * bb) ? MQS_OK : MQS_ERR_NOT_CONVERGED;
          break;
        }
        rr = rt; first = true; beta = 0.0; ++restarts;   // restart from the true residual
      } else {
        beta = rn / rr; rr = rn; first = false;
      }
      if (it >= a.maxit) { status = MQS_ERR_NOT_CONVERGED; need_true = true; break; }
    }
  } else {
    relres = start_rel;  // the start vector already satisfies the tolerance (true residual)
  }
  if (need_true) {
    EpiResidual ep{a.b, a.r, a.lx, a.g.n3};
    sweep_L(a.g, a.x, a.full, bid, nb, sm, ep);
    double rt, bt;
    if (!reduce2(ep.rr, ep.bb, rt, bt)) return;
    relres = sqrt(rt / bb);
  }
  if (bid == 0 && threadIdx.x == 0) *a.out = PcgResult{it, status, relres, start_rel};
}

struct EpiApplyDot {  // w = t on n-edges (0 elsewhere); sums w.r with r the source values
  double* w; long long n3;
  double wr = 0.0;
  __device__ void prefetch(long long) {}
  __device__ void operator()(long long e, unsigned m, double tx, double ty, double tz, double sx, double sy,
                             double sz) {
    const double t[3] = {tx, ty, tz}, s[3] = {sx, sy, sz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double wv = (m >> c & 1u) ? t[c] : 0.0;
      MQS_STC(w, e + c * n3, 3 * n3, 211, wv);
      wr = fma(wv, s[c], wr);
    }
  }
};

struct FusedBufs { double* r1; double* w0; double* w1; double* s0; double* s1; const int2* ptab; };

// The one-reduction form: after the initial residual r and w = L r, every
// iteration is one fused pass (sweep_fused) and one grid reduction of
// (gamma, delta).  Same iterates as the two-reduction kernel in exact
// arithmetic; convergence is confirmed on the true residual as there.
// Scale of the fixed-point pass: E with bound < 2^(E-1) (bound >= every |r_{i+1}|); the
// pass converts with 2^(58-E) (|R| < 2^57, |L R| < 2^61).
__device__ __forceinline__ int fx_exponent_of_bound(double bound) {
  const int eb = (int)((__double_as_longlong(bound) >> 52) & 0x7FF);
  return (eb == 0 ? -1022 : eb - 1023) + 2;
}
// an upper bound of |v| for every v whose biased exponent is at most e (e > 0), 2^(e - 1022)
__device__ __forceinline__ double fx_below(int e) { return e == 0 ? 0x1.0p-1022 : ldexp(1.0, e - 1022); }

// The one-reduction form: after the initial residual r and w = L r, every
// iteration is one fused pass (sweep_fused_fx: the stencil in 64-bit fixed point) and
// one grid reduction of (gamma, delta) with the exponent maxima that bound the next
// pass's r_{i+2} = r_{i+1} - alpha' (w_{i+1} + beta' s_i):
//   max |r_{i+2}| <= max |r_{i+1}| + |alpha'| (max |w_{i+1}| + |beta'| max |s_i|).
// Same iterates as the two-reduction kernel in exact arithmetic; convergence is
// confirmed on the true residual as there.
// G: stencil groups per block (the tile shape of the sweeps: G tiles of 32 x kTY positions
// in flight per block, kGroupWarps warps each).  HW: halo warps per group in the fused
// pass (2: G more warps at the end of the block, which sit out the other sweeps).
template <int G, int HW = 1>
__global__ void __launch_bounds__(32 * (kGroupWarps + HW - 1) * G, kPcgBlocksPerSM)
    pcg_fused_kernel(PcgArgs a, FusedBufs fb) {
  if (pcg_halted(a.halt, a.out)) return;
  __shared__ union { SweepSmemT<double, G> s; FusedFxSmemBlockG<G> f; } sm;
  __shared__ double red[32];
  __shared__ double gs[2];
  __shared__ int gm[3];
  // the stencil sweeps other than the fused pass run on the G x kGroupWarps group warps
  const bool in_groups = HW == 1 || threadIdx.x < 32 * kGroupWarps * G;
  auto sweep_S = [&](const Geom& g, const double* src, const Box& box, int part, int nparts, auto& smem, auto& ep) {
    if (in_groups) sweep_L(g, src, box, part, nparts, smem, ep);
  };
  const int nb = gridDim.x, bid = blockIdx.x;
  unsigned nbar = 0;
  int slot = 0;
  const long long len = 3 * a.g.n3;
  // the elementwise loops run on the group warps only, so that every form with G groups
  // sums in the same order (the extra halo warps of HW = 2 add exact zeros)
  const int gth = HW == 1 ? (int)blockDim.x : 32 * kGroupWarps * G;
  const long long tid = in_groups ? (long long)bid * gth + threadIdx.x : len, nth = (long long)nb * gth;
  auto reduce2 = [&](double v0, double v1, double& s0, double& s1) -> bool {
    return grid_sum2<double>(v0, v1, s0, s1, a.part, slot, nbar, a.bar, a.spin, a.err, red, gs);
  };
  auto rb = [&](int c) { return c ? fb.r1 : a.r; };
  auto wb = [&](int c) { return c ? fb.w1 : fb.w0; };
  auto sb = [&](int c) { return c ? fb.s1 : fb.s0; };
  int status = MQS_OK, it = 0, cur = 0;
  double rr = 0.0, bb = 0.0, start_rel = 0.0, relres = 0.0;
  if (a.init == 0) {
    EpiResidual ep{a.b, a.r, a.lx, a.g.n3};
    sweep_S(a.g, a.x, a.full, bid, nb, sm.s, ep);
    if (!reduce2(ep.rr, ep.bb, rr, bb)) return;
  } else {
    double s0 = 0.0, s1 = 0.0;
    for (long long e = tid; e < len; e += nth) {
      const double be = a.b[e];
      double re;
      if (a.init == 2) { re = be; a.r[e] = be; a.x[e] = 0.0; } else { re = a.r[e]; }
      s0 = fma(re, re, s0);
      s1 = fma(be, be, s1);
    }
    if (!reduce2(s0, s1, rr, bb)) return;
  }
  if (bb == 0.0) {
    for (long long e = tid; e < len; e += nth) { a.x[e] = 0.0; a.r[e] = 0.0; a.lx[e] = 0.0; }
    if (bid == 0 && threadIdx.x == 0) *a.out = PcgResult{0, MQS_OK, 0.0, 0.0};
    return;
  }
  start_rel = sqrt(rr / bb);
  if (a.init != 0 && isfinite(rr) && isfinite(bb) && rr <= a.tol2 * bb) {
    EpiResidual ep{a.b, a.r, a.lx, a.g.n3};
    sweep_S(a.g, a.x, a.full, bid, nb, sm.s, ep);
    double rt, bt;
    if (!reduce2(ep.rr, ep.bb, rt, bt)) return;
    if (rt <= a.tol2 * bb) {
      if (bid == 0 && threadIdx.x == 0) *a.out = PcgResult{0, MQS_OK, sqrt(rt / bb), start_rel};
      return;
    }
    rr = rt;
  }
  bool need_true = false;
  if (!isfinite(rr) || !isfinite(bb)) {
    status = MQS_ERR_NAN;
  } else if (rr > a.tol2 * bb) {
    double gamma = rr, alpha = 0.0, beta = 0.0;
    double mr = 0.0, mw = 0.0, ms = 0.0;   // upper bounds of max |r|, max |w| of the current r, w; of max |s|
    bool first = true;
    int restarts = 0;
    bool restart_w = true;     // w = L r must be formed for the current r
    for (;;) {
      if (restart_w) {
        EpiApplyDot ep{wb(cur), a.g.n3};
        sweep_S(a.g, rb(cur), a.full, bid, nb, sm.s, ep);
        double delta, dummy;
        if (!reduce2(ep.wr, 0.0, delta, dummy)) return;
        if (!(delta > 0.0)) { status = isnan(delta) ? MQS_ERR_NAN : MQS_ERR_BREAKDOWN; need_true = true; break; }
        alpha = gamma / delta;
        beta = 0.0;
        first = true;
        restart_w = false;
        // max |r| <= ||r||_2 < 2^(E-1) and |(L r)_e| <= 16 max |r| (the absolute row sum of L)
        mr = ldexp(1.0, fx_exponent(gamma) - 1);
        mw = 16.0 * mr;
        ms = 0.0;
      }
      const double bound = mr + fabs(alpha) * (mw + (first ? 0.0 : fabs(beta) * ms));
      const int E = fx_exponent_of_bound(bound);
      FusedFxVecs v{FusedVecs{a.x, a.p, rb(cur), wb(cur), sb(cur), rb(cur ^ 1), wb(cur ^ 1), sb(cur ^ 1), alpha, beta,
                              first},
                    58 - E, E - 58};
      double g1 = 0.0, d1 = 0.0;
      int er = 0, ew = 0, es = 0;
      sweep_fused_fx<G, HW>(a.g, v, a.full, bid, nb, sm.f, g1, d1, er, ew, es, fb.ptab);
      double gn, dn;
      if (!grid_sum2_max3(g1, d1, er, ew, es, gn, dn, er, ew, es, a.part, slot, nbar, a.bar, a.spin, a.err, red, gs,
                          gm))
        return;
      mr = fx_below(er);
      mw = fx_below(ew);
      ms = fx_below(es);
      ++it;
      cur ^= 1;
      if (!isfinite(gn) || !isfinite(dn)) { status = MQS_ERR_NAN; need_true = true; break; }
      if (gn <= a.tol2 * bb) {
        EpiResidual ep{a.b, rb(cur), a.lx, a.g.n3};
        sweep_S(a.g, a.x, a.full, bid, nb, sm.s, ep);
        double rt, bt;
        if (!reduce2(ep.rr, ep.bb, rt, bt)) return;
        if (rt <= a.tol2 * bb || restarts >= 8) {
          relres = sqrt(rt / bb);
          status = (rt <= a.tol2 * bb) ? MQS_OK : MQS_ERR_NOT_CONVERGED;
          break;
        }
        gamma = rt; ++restarts; restart_w = true;   // restart from the true residual
      } else {
        const double bnew = gn / gamma;
        const double den = dn - bnew * gn / alpha;
        if (!(den > 0.0)) { status = isnan(den) ? MQS_ERR_NAN : MQS_ERR_BREAKDOWN; need_true = true; break; }
        beta = bnew;
        alpha = gn / den;
        gamma = gn;
        first = false;
      }
      if (it >= a.maxit) { status = MQS_ERR_NOT_CONVERGED; need_true = true; break; }
    }
  } else {
    relres = start_rel;
  }
  if (need_true) {
    EpiResidual ep{a.b, rb(cur), a.lx, a.g.n3};
    sweep_S(a.g, a.x, a.full, bid, nb, sm.s, ep);
    double rt, bt;
    if (!reduce2(ep.rr, ep.bb, rt, bt)) return;
    relres = sqrt(rt / bb);
  }
  if (bid == 0 && threadIdx.x == 0) *a.out = PcgResult{it, status, relres, start_rel};
}

// the block of a fused-pass form must fit once per SM beside nothing else (asked once per
// process and form; a function-local static is initialised once even with concurrent callers)
template <int G, int HW>
static int fused_form_fits() {
  static const int occ = [] {
    int o = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, pcg_fused_kernel<G, HW>, 32 * (kGroupWarps + HW - 1) * G,
                                                         0) == cudaSuccess
               ? o
               : -1;
  }();
  if (occ < 0) return MQS_ERR_CUDA;
  return occ >= kPcgBlocksPerSM ? MQS_OK : MQS_ERR_ARG;
}

int launch_pcg_fused(const DevGeom& dg, const double* b, double* x, double* r, double* p, double* lx,
                     const PcgExtra& ex, double* part, unsigned* bar, int* err, PcgResult* out, double tol, int maxit,
                     int nblk, cudaStream_t st, int init, const int* halt, int groups, const int2* ptab,
                     int halo_warps) {
  PcgArgs a;
  a.g = dg.g;
  a.full = Box{{0, 0, 0}, {dg.g.n, dg.g.n, dg.g.n}};
  a.b = b; a.x = x; a.r = r; a.p = p; a.q = nullptr; a.lx = lx;
  a.part = part; a.bar = bar; a.err = err; a.out = out;
  a.tol2 = tol * tol; a.maxit = maxit;
  a.spin = 1ll << 21;
  a.init = init;
  a.halt = halt;
  FusedBufs fb{ex.r1, ex.w0, ex.w1, ex.s0, ex.s1, ptab};
  if (groups == 0) groups = kGroups;
  if (halo_warps == 0) halo_warps = 1;
  // forms: (2 groups, 1 halo warp) 320 threads, (3, 1) 480, (2, 2) 384
  const void* fn = nullptr;
  int threads = 0, fits = MQS_ERR_ARG;
  if (groups == kGroups && halo_warps == 1) {
    fn = (const void*)pcg_fused_kernel<kGroups, 1>; threads = kBlock; fits = MQS_OK;
  } else if (groups == 3 && halo_warps == 1) {
    fn = (const void*)pcg_fused_kernel<3, 1>; threads = 32 * kGroupWarps * 3; fits = fused_form_fits<3, 1>();
  } else if (groups == kGroups && halo_warps == 2) {
    fn = (const void*)pcg_fused_kernel<kGroups, 2>; threads = 32 * (kGroupWarps + 1) * kGroups;
    fits = fused_form_fits<kGroups, 2>();
  }
  if (fits != MQS_OK) return fits;
  if (cudaMemsetAsync(bar, 0, sizeof(unsigned), st) != cudaSuccess) return MQS_ERR_CUDA;
  void* args[] = {&a, &fb};
  const cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(nblk), dim3(threads), args, 0, st);
  return e == cudaSuccess ? MQS_OK : MQS_ERR_CUDA;
}

int launch_pcg(const DevGeom& dg, const double* b, double* x, double* r, double* p, double* q, double* lx,
               double* part, unsigned* bar, int* err, PcgResult* out, double tol, int maxit, int nblk,
               cudaStream_t st, int init, const int* halt) {
  PcgArgs a;
  a.g = dg.g;
  a.full = Box{{0, 0, 0}, {dg.g.n, dg.g.n, dg.g.n}};
  a.b = b; a.x = x; a.r = r; a.p = p; a.q = q; a.lx = lx;
  a.part = part; a.bar = bar; a.err = err; a.out = out;
  a.tol2 = tol * tol; a.maxit = maxit;
  a.spin = 1ll << 21;   // about a second of polling before a barrier gives up
  a.init = init;
  a.halt = halt;
  if (cudaMemsetAsync(bar, 0, sizeof(unsigned), st) != cudaSuccess) return MQS_ERR_CUDA;
  void* args[] = {&a};
  const bool two = 3LL * dg.g.n3 >= kMixedTwoBlocksLen;
  cudaError_t e = two ? cudaLaunchCooperativeKernel((const void*)pcg_kernel<2>, dim3(2 * nblk), dim3(kBlock), args,
                                                    0, st)
                      : cudaLaunchCooperativeKernel((const void*)pcg_kernel<1>, dim3(nblk), dim3(kBlock), args, 0, st);
  return e == cudaSuccess ? MQS_OK : MQS_ERR_CUDA;
}

// every block waits at a barrier whose target exceeds the grid size
__global__ void __launch_bounds__(kBlock, kPcgBlocksPerSM) barrier_selftest_kernel(unsigned* ctr, int* err,
                                                                                    long long polls) {
  grid_barrier(ctr, gridDim.x + 1, polls, err);
}

int pcg_max_blocks(int* nblk) {
  int dev = 0, nsm = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MQS_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MQS_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pcg_kernel<1>, kBlock, 0) != cudaSuccess) return MQS_ERR_CUDA;
  if (occ < 1) return MQS_ERR_CUDA;
  *nblk = nsm * (occ < kPcgBlocksPerSM ? occ : kPcgBlocksPerSM);  // persistent, co-resident blocks
  return MQS_OK;
}

// The plane-tile ranges of the fused pass's group parts with the largest part as small as
// possible.  A part's cost is its plane-tiles plus one warm-up plane per segment (a
// segment starts at the part's first tile, at every tile column's first plane and after
// kMaxSeg planes).  The even split of the tile count can give one part two segments and
// the most tiles (64^3, 304 parts: 7 tiles + 2 warm-ups against 6.74 + 1.05 on average);
// a binary search on the largest cost with a greedy fill finds the smallest one (8 there).
// Parts past the last filled one get empty ranges.
static long long partition_fill(long long ntiles, int nz, long long cap, long long parts, int2* out) {
  long long u = 0, p = 0;
  while (u < ntiles) {
    if (p >= parts) return parts + 1;
    const long long u0 = u;
    long long cost = 0, seg = 0;
    while (u < ntiles) {
      const bool newseg = (u == u0) || (u % nz == 0) || (seg == kMaxSeg);
      const long long add = 1 + (newseg ? 1 : 0);
      if (cost + add > cap && u > u0) break;
      cost += add;
      seg = newseg ? 1 : seg + 1;
      ++u;
    }
    if (out) out[p] = make_int2((int)u0, (int)u);
    ++p;
  }
  if (out)
    for (long long q = p; q < parts; ++q) out[q] = make_int2((int)ntiles, (int)ntiles);
  return p;
}

int fused_partition_host(int n, int nblk, int groups, std::vector<int2>& tab) {
  if (groups == 0) groups = kGroups;
  if (n < 1 || nblk < 1 || groups < 1) return MQS_ERR_ARG;
  const long long ntx = (n + 31) / 32, nty = (n + kTY - 1) / kTY, ntiles = ntx * nty * n;
  const long long parts = (long long)nblk * groups;
  if (ntiles >= (1LL << 31) || parts >= (1LL << 31)) return MQS_ERR_ARG;
  long long lo = 1, hi = 2 * ntiles + 2;
  while (lo < hi) {
    const long long mid = (lo + hi) / 2;
    if (partition_fill(ntiles, n, mid, parts, nullptr) <= parts) hi = mid;
    else lo = mid + 1;
  }
  tab.assign((size_t)parts, make_int2(0, 0));
  partition_fill(ntiles, n, lo, parts, tab.data());
  return MQS_OK;
}

int fused_partition(int n, int nblk, int groups, int2* dev_table, cudaStream_t st) {
  std::vector<int2> tab;
  const int rc = fused_partition_host(n, nblk, groups, tab);
  if (rc != MQS_OK) return rc;
  if (cudaMemcpyAsync(dev_table, tab.data(), sizeof(int2) * tab.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return MQS_ERR_CUDA;
  return MQS_OK;
}

MQS_DEBUG_TAKE(pcg)

}  // namespace mqs

extern "C" int mqs_selftest_barrier_timeout(long long polls) {
  using namespace mqs;
  if (polls < 1) return MQS_ERR_ARG;
  int nblk = 0;
  if (pcg_max_blocks(&nblk) != MQS_OK) return MQS_ERR_CUDA;
  void* mem = nullptr;
  if (cudaMalloc(&mem, 64) != cudaSuccess) return MQS_ERR_OOM;
  unsigned* ctr = static_cast<unsigned*>(mem);
  int* err = reinterpret_cast<int*>(static_cast<char*>(mem) + 16);
  int rc = MQS_ERR_CUDA;
  if (cudaMemset(mem, 0, 64) == cudaSuccess) {
    void* args[] = {&ctr, &err, &polls};
    if (cudaLaunchCooperativeKernel((const void*)barrier_selftest_kernel, dim3(nblk), dim3(kBlock), args, 0, 0) ==
            cudaSuccess &&
        cudaDeviceSynchronize() == cudaSuccess) {
      int h = 0;
      if (cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess) rc = h;
    }
  }
  cudaFree(mem);
  return rc;
}
