// Start vectors for the multiple right-hand side problem (Sec. III).
//
// SPE (eq. (SPE_x0)): x0 is the Galerkin projection of K_n x = b onto the span
// of the last d solutions.  That span equals the span of the backward
// differences D_0 = w_m, D_p = D_{p-1}(m) - D_{p-1}(m-1), which the device keeps
// as a table updated in place once per step (one pass, d subtractions per
// entry) together with its K_n image (the PCG residual supplies K_n w for
// free).  The differences separate the scales of the nearly collinear
// solutions, so Gram-Schmidt in the K_n inner product can run on the small
// matrix H = D^T K_n D (a pivoted Cholesky factorisation, dropping columns
// whose K_n-remainder falls below eps_lin times the newest solution's K_n
// norm); x0 = D H^-1 D^T b.
//
// POD (eqs. (SVD), (relSV2), (keepInfo), (POD_x0)): method of snapshots.  The
// snapshot correlation G = X^T X and A = X^T K_n X gain one row per step; the
// small symmetric eigenproblem G = V Lambda V^T (parallel-order Jacobi) gives
// sigma_i = sqrt(lambda_i) and U = X V Sigma^-1, truncated at sigma_i/sigma_1
// >= eps_pod; then x0 = U_k (U_k^T K_n U_k)^-1 U_k^T b in the small space.
#include <algorithm>
#include <cmath>
#include "mrhs.h"

namespace mqs {

constexpr int kTS = 256;        // threads of the tall-skinny kernels

// ---- tiled dot products (FP64: POD snapshot rows, CSPE projections) -----------------
// part[blk * kTileSlots + p*8 + q] = sum_e A_p[e] B_q[e]   (p < ma <= 2, q < mb; kRow2)
// part[blk * kTileSlots + 64 + q]  = sum_e B_q[e] c[e]     (if c != nullptr)
// The c products are skipped where c vanishes (the right-hand side of eq. (mrhs) is
// zero away from the conductor and the coil).  The float-float product kernels of the
// SPE table use the tile modes kTri, kRect4, kTri4 (below).
enum DotsMode { kTri = 0, kRow2 = 2, kConly = 3, kRect4 = 4, kTri4 = 5 };

// 8x8 slot (p*8 + q) of the t-th upper-triangle product, in the order p, then q >= p
__constant__ int c_tri_slot[36] = {0,  1,  2,  3,  4,  5,  6,  7,  9,  10, 11, 12, 13, 14, 15, 18, 19, 20,
                                   21, 22, 23, 27, 28, 29, 30, 31, 36, 37, 38, 39, 45, 46, 47, 54, 55, 63};

template <int MODE>
__global__ void __launch_bounds__(kTS, 2) dots_kernel(VecSet A, VecSet B, const double* c, int ma, int mb,
                                                     long long len, double* part) {
  static_assert(MODE == kRow2 || MODE == kConly, "FP64 tiles: two rows, or the c products alone");
  constexpr int MA = (MODE == kRow2) ? 2 : 0;
  constexpr int NACC = MA * 8 > 0 ? MA * 8 : 1;
  double acc[NACC], accc[8];
#pragma unroll
  for (int t = 0; t < NACC; ++t) acc[t] = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) accc[q] = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x) {
    double a[MA > 0 ? MA : 1], b[8];
#pragma unroll
    for (int p = 0; p < MA; ++p) a[p] = (p < ma) ? A.v[p][e] : 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) b[q] = (q < mb) ? B.v[q][e] : 0.0;
    int t = 0;
#pragma unroll
    for (int p = 0; p < MA; ++p) {
#pragma unroll
      for (int q = 0; q < 8; ++q, ++t)
        if (p < ma && q < mb) acc[t] = fma(a[p], b[q], acc[t]);
    }
    if (c != nullptr) {
      const double ce = c[e];
      if (ce != 0.0) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q < mb) accc[q] = fma(b[q], ce, accc[q]);
      }
    }
  }
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  __shared__ double red[kTS / 32][kTileSlots];
  // Warp reduce-scatter over 48 slots (16 products, then the 8 c products): lane
  // pairs exchange the half they do not keep, four times, then one butterfly step;
  // 48 additions per lane instead of 5 per slot.
  double v[48];
#pragma unroll
  for (int t = 0; t < 48; ++t) v[t] = 0.0;
#pragma unroll
  for (int t = 0; t < MA * 8; ++t) v[t] = acc[t];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[36 + q] = accc[q];
#pragma unroll
  for (int half = 24, off = 16; off >= 2; half >>= 1, off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const double keep = up ? v[i + half] : v[i];
      const double send = up ? v[i] : v[i + half];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], 1);
  if ((lane & 1) == 0) {
    const int base = 24 * ((lane >> 4) & 1) + 12 * ((lane >> 3) & 1) + 6 * ((lane >> 2) & 1) + 3 * ((lane >> 1) & 1);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int sl = base + i;
      int dst = -1;
      if (sl >= 36) dst = (sl < 44) ? 64 + (sl - 36) : -1;
      else if (sl < MA * 8) dst = sl;
      if (dst >= 0) red[wp][dst] = v[i];
    }
  }
  // slots no lane writes (unused rows) are zero
  for (int t = lane; t < 64; t += 32)
    if (t / 8 >= MA) red[wp][t] = 0.0;
  __syncthreads();
  for (int s2 = threadIdx.x; s2 < kTileSlots; s2 += blockDim.x) {
    double t = 0.0;
    for (int q = 0; q < kTS / 32; ++q) t += red[q][s2];
    part[(size_t)blockIdx.x * kTileSlots + s2] = t;
  }
}

// ---- linear combination x = sum_p coef[p] V_p -------------------------------------
template <int MAXM>
__global__ void __launch_bounds__(kTS) lincomb_kernel(VecSet V, const double* coef, int m, long long len,
                                                      double* x) {
  __shared__ double cf[kMaxVec];
  for (int p = threadIdx.x; p < kMaxVec; p += blockDim.x) cf[p] = (p < m) ? coef[p] : 0.0;
  __syncthreads();
  const long long half = len >> 1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < half;
       e += (long long)gridDim.x * blockDim.x) {
    double2 v[MAXM];
#pragma unroll
    for (int p = 0; p < MAXM; ++p) v[p] = (p < m) ? reinterpret_cast<const double2*>(V.v[p])[e] : double2{0.0, 0.0};
    double sx = 0.0, sy = 0.0;
#pragma unroll
    for (int p = 0; p < MAXM; ++p) { sx = fma(cf[p], v[p].x, sx); sy = fma(cf[p], v[p].y, sy); }
    reinterpret_cast<double2*>(x)[e] = double2{sx, sy};
  }
  if ((len & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    double s = 0.0;
    for (int p = 0; p < m; ++p) s = fma(cf[p], V.v[p][len - 1], s);
    x[len - 1] = s;
  }
}

// x = sum_p coef[p] V_p and r = b - sum_p coef[p] W_p (W_p = L V_p): the start
// vector and its residual in one pass (no stencil needed)
template <int MAXM>
__global__ void __launch_bounds__(kTS) lincomb_res_kernel(VecSet V, VecSet W, const double* coef, int m,
                                                          const double* b, long long len, double* x, double* r) {
  __shared__ double cf[kMaxVec];
  for (int p = threadIdx.x; p < kMaxVec; p += blockDim.x) cf[p] = (p < m) ? coef[p] : 0.0;
  __syncthreads();
  const long long half = len >> 1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < half;
       e += (long long)gridDim.x * blockDim.x) {
    double sx = 0.0, sy = 0.0, tx = 0.0, ty = 0.0;
#pragma unroll
    for (int p = 0; p < MAXM; ++p) {
      if (p < m) {
        const double2 v = reinterpret_cast<const double2*>(V.v[p])[e];
        const double2 w = reinterpret_cast<const double2*>(W.v[p])[e];
        sx = fma(cf[p], v.x, sx); sy = fma(cf[p], v.y, sy);
        tx = fma(cf[p], w.x, tx); ty = fma(cf[p], w.y, ty);
      }
    }
    const double2 bb = reinterpret_cast<const double2*>(b)[e];
    reinterpret_cast<double2*>(x)[e] = double2{sx, sy};
    reinterpret_cast<double2*>(r)[e] = double2{bb.x - tx, bb.y - ty};
  }
  if ((len & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    double s = 0.0, t = 0.0;
    for (int p = 0; p < m; ++p) { s = fma(cf[p], V.v[p][len - 1], s); t = fma(cf[p], W.v[p][len - 1], t); }
    x[len - 1] = s;
    r[len - 1] = b[len - 1] - t;
  }
}

static void launch_lincomb_res(const VecSet& V, const VecSet& W, const double* coef, int m, const double* b,
                               long long len, double* x, double* r, int nb, cudaStream_t st) {
  nb *= 4;
  if (m <= 8) lincomb_res_kernel<8><<<nb, kTS, 0, st>>>(V, W, coef, m, b, len, x, r);
  else if (m <= 16) lincomb_res_kernel<16><<<nb, kTS, 0, st>>>(V, W, coef, m, b, len, x, r);
  else lincomb_res_kernel<40><<<nb, kTS, 0, st>>>(V, W, coef, m, b, len, x, r);
}

static void launch_lincomb(const VecSet& V, const double* coef, int m, long long len, double* x, int nb,
                           cudaStream_t st) {
  nb *= 4;   // memory-latency bound: more resident warps
  if (m <= 8) lincomb_kernel<8><<<nb, kTS, 0, st>>>(V, coef, m, len, x);
  else if (m <= 16) lincomb_kernel<16><<<nb, kTS, 0, st>>>(V, coef, m, len, x);
  else lincomb_kernel<40><<<nb, kTS, 0, st>>>(V, coef, m, len, x);
}

// ---- small dense kernels (one block) ----------------------------------------------------
// fixed-order sum over blocks of one partial slot (serial; small callers)
// Sum over the nblk block partials of one product slot by one warp (every lane calls
// it; the total comes back in every lane): each lane adds its blocks lane, lane + 32, ...
// with the loads issued ahead, then a fixed shuffle tree and lane 0's value broadcast,
// so the result does not depend on scheduling.  (A single thread walking the blocks in
// order waits one L2 round trip per block: ~47 us for 304 blocks.)
__device__ double sum_part(const double* part, int nblk, int slot) {
  const int lane = threadIdx.x & 31;
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  int q = lane;
  for (; q + 96 < nblk; q += 128) {
#pragma unroll
    for (int r = 0; r < 4; ++r) a[r] += __ldcg(part + (size_t)(q + 32 * r) * kTileSlots + slot);
  }
  // at most three blocks are left: q, q + 32, q + 64
  if (q < nblk) a[0] += __ldcg(part + (size_t)q * kTileSlots + slot);
  if (q + 32 < nblk) a[1] += __ldcg(part + (size_t)(q + 32) * kTileSlots + slot);
  if (q + 64 < nblk) a[2] += __ldcg(part + (size_t)(q + 64) * kTileSlots + slot);
  double s = (a[0] + a[1]) + (a[2] + a[3]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  return __shfl_sync(0xffffffffu, s, 0);
}

// Pivoted (in order) Cholesky of the symmetric m x m matrix H (row-major in
// smem, m <= 64), dropping column j when its pivot v satisfies
// v*H_jj <= drop2*H_00 (scaled-unit diagonal) or v <= rel_floor.  Solves
// H y = g on the kept columns; dropped entries of y are zero.  Returns the
// number kept.  Run by the first warp with one matrix row per lane (rows
// lane and lane + 32): right-looking factorisation and row-oriented
// substitutions, a broadcast shuffle per step instead of block barriers or
// per-row reductions.  One reciprocal square root per pivot and no divisions
// (FP64 divide and square root are long dependent sequences on this GPU).
// H and g in shared memory are overwritten; Ls is unused scratch.
__device__ int chol_drop_solve(double* H, double* g, double* y, int m, double drop2, double rel_floor,
                               double* /*Ls*/, int* keep) {
  __shared__ int nk_s;
  const int tid = threadIdx.x;
  if (tid < 32) {
    const int lane = tid;
    const int r0 = lane, r1 = lane + 32;
    const bool h0 = r0 < m, h1 = r1 < m;
    // scaling to unit diagonal
    const double d0 = h0 ? H[r0 * m + r0] : 0.0, d1 = h1 ? H[r1 * m + r1] : 0.0;
    const double s0 = (d0 > 0.0) ? rsqrt(d0) : 0.0, s1 = (d1 > 0.0) ? rsqrt(d1) : 0.0;
    const double hd00 = __shfl_sync(0xffffffffu, d0, 0);
    // scale row r (lane) : H_rc *= s_r s_c ; s_c from its owner lane
    for (int c = 0; c < m; ++c) {
      const double sc_c = (c < 32) ? __shfl_sync(0xffffffffu, s0, c) : __shfl_sync(0xffffffffu, s1, c - 32);
      if (h0) H[r0 * m + c] *= s0 * sc_c;
      if (h1) H[r1 * m + c] *= s1 * sc_c;
    }
    __syncwarp();
    int nk = 0;
    double inv0 = 0.0, inv1 = 0.0;
    for (int j = 0; j < m; ++j) {
      // owner of row j decides the pivot (its row holds the updated H_jj)
      const bool own0 = (j == r0), own1 = (j == r1);
      double v = 0.0, dj = 0.0;
      if (own0) { v = H[j * m + j]; dj = d0; }
      if (own1) { v = H[j * m + j]; dj = d1; }
      const int src = j & 31;
      v = __shfl_sync(0xffffffffu, v, src);
      dj = __shfl_sync(0xffffffffu, dj, src);
      const double sj = (dj > 0.0) ? 1.0 : 0.0;
      const bool kj = sj > 0.0 && v > rel_floor && v * dj > drop2 * hd00;
      const double r = kj ? rsqrt(v) : 0.0;
      if (own0) inv0 = r;
      if (own1) inv1 = r;
      if (lane == 0) keep[j] = kj ? 1 : 0;
      nk += kj ? 1 : 0;
      // column j of L: L_ij = H_ij r (i > j), L_jj = v r; rows below update their trailing part
      if (kj) {
        if (h0 && r0 > j) H[r0 * m + j] *= r;
        if (h1 && r1 > j) H[r1 * m + j] *= r;
        if (own0 || own1) H[j * m + j] = v * r;
        __syncwarp();
        if (h0 && r0 > j) {
          const double l = H[r0 * m + j];
          for (int k = j + 1; k <= r0; ++k) H[r0 * m + k] = fma(-l, H[k * m + j], H[r0 * m + k]);
        }
        if (h1 && r1 > j) {
          const double l = H[r1 * m + j];
          for (int k = j + 1; k <= r1; ++k) H[r1 * m + k] = fma(-l, H[k * m + j], H[r1 * m + k]);
        }
      } else {
        if (h0 && r0 > j) H[r0 * m + j] = 0.0;
        if (h1 && r1 > j) H[r1 * m + j] = 0.0;
      }
      __syncwarp();
    }
    // forward L z = S g: z_t finalised by its owner, then broadcast
    double a0 = h0 ? g[r0] * s0 : 0.0, a1 = h1 ? g[r1] * s1 : 0.0;
    double z0 = 0.0, z1 = 0.0;
    for (int t = 0; t < m; ++t) {
      double zt = 0.0;
      if (t == r0) { z0 = a0 * inv0; zt = z0; }
      if (t == r1) { z1 = a1 * inv1; zt = z1; }
      zt = __shfl_sync(0xffffffffu, zt, t & 31);
      if (h0 && r0 > t) a0 = fma(-H[r0 * m + t], zt, a0);
      if (h1 && r1 > t) a1 = fma(-H[r1 * m + t], zt, a1);
    }
    // backward L^T u = z
    double b0 = z0, b1 = z1, u0 = 0.0, u1 = 0.0;
    for (int t = m - 1; t >= 0; --t) {
      double ut = 0.0;
      if (t == r0) { u0 = b0 * inv0; ut = u0; }
      if (t == r1) { u1 = b1 * inv1; ut = u1; }
      ut = __shfl_sync(0xffffffffu, ut, t & 31);
      if (h0 && r0 < t) b0 = fma(-H[t * m + r0], ut, b0);
      if (h1 && r1 < t) b1 = fma(-H[t * m + r1], ut, b1);
    }
    if (h0) y[r0] = u0 * s0;
    if (h1) y[r1] = u1 * s1;
    if (lane == 0) nk_s = nk;
  }
  __syncthreads();
  return nk_s;
}

// chol_drop_solve for m <= M (8 or 16) held in registers, in two halves (the factor
// needs only H, the substitutions g): lane r keeps row r of the scaled matrix
// (compile-time indexed, every loop unrolled), column values travel by shuffles.
// Same pivot order, scaling, drop rule and substitutions as chol_drop_solve; on this
// GPU every dependent FP64 step costs the FP64 unit's issue time, so the register form
// keeps the serial chain short.  Called by warp 0.  Factor: h becomes row `lane` of
// the factor L (scaled units), inv its reciprocal pivot (0 where the column was
// dropped), sc the row's diagonal scaling; returns the number of kept columns.
template <int M>
__device__ int chol_drop_factor_reg(const double* H, int m, double drop2, double rel_floor, double (&h)[M],
                                    double& inv, double& sc) {
  static_assert(M <= 32, "one row per lane");
  const int lane = threadIdx.x & 31;
  const bool own = lane < m;
#pragma unroll
  for (int c = 0; c < M; ++c) h[c] = (own && c < m) ? H[lane * m + c] : 0.0;
  double d = 0.0;
#pragma unroll
  for (int c = 0; c < M; ++c) if (c == lane) d = h[c];
  sc = (own && d > 0.0) ? rsqrt(d) : 0.0;
  const double hd00 = __shfl_sync(0xffffffffu, d, 0);
#pragma unroll
  for (int c = 0; c < M; ++c) h[c] *= sc * __shfl_sync(0xffffffffu, sc, c);
  inv = 0.0;
  int nk = 0;
#pragma unroll
  for (int j = 0; j < M; ++j) {
    if (j >= m) break;
    const double v = __shfl_sync(0xffffffffu, h[j], j);      // updated pivot (row j)
    const double dj = __shfl_sync(0xffffffffu, d, j);
    const bool kj = dj > 0.0 && v > rel_floor && v * dj > drop2 * hd00;
    const double r = kj ? rsqrt(v) : 0.0;
    nk += kj ? 1 : 0;
    if (lane == j) { inv = r; h[j] = v * r; }
    const double lij = (lane > j) ? h[j] * r : 0.0;           // column j of L in rows below
    if (lane > j) h[j] = lij;
#pragma unroll
    for (int k = j + 1; k < M; ++k) {
      const double lkj = __shfl_sync(0xffffffffu, lij, k);
      if (lane >= k) h[k] = fma(-lij, lkj, h[k]);
    }
  }
  return nk;
}

// Substitutions with the factor of chol_drop_factor_reg: forward L z = S g, backward
// L^T u = z, y = S u (dropped entries zero).
template <int M>
__device__ void chol_solve_reg(const double (&h)[M], double inv, double sc, const double* g, double* y, int m) {
  const int lane = threadIdx.x & 31;
  const bool own = lane < m;
  double a = own ? g[lane] * sc : 0.0, z = 0.0;
#pragma unroll
  for (int t = 0; t < M; ++t) {
    if (t >= m) break;
    if (lane == t) z = a * inv;
    const double zt = __shfl_sync(0xffffffffu, z, t);
    if (lane > t) a = fma(-h[t], zt, a);
  }
  // backward: row t's entries go to the lanes of the columns
  double b = z, u = 0.0;
#pragma unroll
  for (int t = M - 1; t >= 0; --t) {
    if (t >= m) continue;
    if (lane == t) u = b * inv;
    const double ut = __shfl_sync(0xffffffffu, u, t);
    double lti = 0.0;
#pragma unroll
    for (int i = 0; i < M; ++i) {
      const double hv = __shfl_sync(0xffffffffu, h[i], t);
      if (i == lane) lti = hv;
    }
    if (lane < t) b = fma(-lti, ut, b);
  }
  if (own) y[lane] = u * sc;
}

// Gram row of a new snapshot: part tiles t = 0..ntile-1 hold (w, Lw) . X_q.
// (one warp per entry)
__global__ void pod_row_kernel(const double* part, int nblk, int m, int slot_new, double* G, double* A) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = wid; q < m; q += nw) {
    const int tile = q / 8, qq = q % 8;
    const double* pt = part + (size_t)tile * nblk * kTileSlots;
    const double gw = sum_part(pt, nblk, 0 * 8 + qq), aw = sum_part(pt, nblk, 1 * 8 + qq);
    if (lane == 0) {
      G[slot_new * kMaxPod + q] = gw; G[q * kMaxPod + slot_new] = gw;
      A[slot_new * kMaxPod + q] = aw; A[q * kMaxPod + slot_new] = aw;
    }
  }
}

// Jacobi rotation (c, s) annihilating a_pq of the symmetric block [[a_pp, a_pq], [a_pq, a_qq]]
// (the classical choice, Golub & Van Loan, "Matrix Computations", Sec. 8.5:
// tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = (1 + t^2)^(-1/2),
// s = t c).  t is formed in FP32: every t gives a rotation that is orthogonal to FP64 rounding
// once c and s are formed from it in FP64, and an FP32 t leaves |a_pq'| ~ 1e-7 |a_pq| for the
// next sweep to remove (the sweep and rotation counts of the FP64 form, emulated on the
// snapshot matrices of the stepping workloads).  c = (1 + t^2)^(-1/2) in FP64 from the FP32
// reciprocal square root by two Newton steps y <- y (3 - x y^2) / 2 (quadratic convergence:
// 1e-7 -> 1e-14 -> rounding).  Ratios outside FP32's range take the FP64 form (rare).
__device__ __forceinline__ void jacobi_rotation(double app, double aqq, double apq, double& c, double& s) {
  const double d = aqq - app;
  const float a32 = (float)(2.0 * apq), d32 = (float)d;
  const float th = d32 / a32;
  double t;
  if (!(fabsf(a32) >= 0x1p-120f && fabsf(a32) <= 0x1p120f && fabsf(th) <= 0x1p60f)) {
    const double th64 = d / (2.0 * apq);
    const double at = fabs(th64);
    t = (at > 1e150) ? 0.5 / th64 : copysign(1.0 / (at + sqrt(fma(th64, th64, 1.0))), th64);
  } else if (fabsf(th) > 0x1p20f) {
    t = (double)(0.5f / th);                       // 1/(2 tau): relative error tau^-2 < 2^-40
  } else {
    const float t32 = 1.0f / (fabsf(th) + sqrtf(fmaf(th, th, 1.0f)));
    t = (double)(th >= 0.f ? t32 : -t32);
  }
  const double x = fma(t, t, 1.0);
  double y = (double)rsqrtf((float)x);
  y = y * fma(-0.5 * x, y * y, 1.5);
  y = y * fma(-0.5 * x, y * y, 1.5);
  c = y;
  s = t * y;
}

// POD solve: Jacobi eigen-decomposition of G (m x m), truncation, reduced
// Galerkin system, coefficients z with x0 = X z.
constexpr int kPodThreads = 256;   // pod_solve_kernel's block (its fixed share of the rotation work)
__global__ void __launch_bounds__(kPodThreads) pod_solve_kernel(const double* Gg, const double* Ag, const double* part,
                                                               int nblk, int m,
                                 double eps_pod, double* coef, double* sigma_out, SmallOut* out) {
  __shared__ double Mt[kMaxPod * kMaxPod], V[kMaxPod * kMaxPod], Hs[kMaxPod * kMaxPod];
  double* W = Mt;   // Mt is free once the eigenvalues are read; W, then L, reuse it
  double* Ls = Mt;
  __shared__ double lam[kMaxPod], gv[kMaxPod], rhs[kMaxPod], y[kMaxPod];
  __shared__ int order[kMaxPod], keep[kMaxPod];
  __shared__ double cs[kMaxPod / 2 + 1], sn[kMaxPod / 2 + 1];
  __shared__ int pp[kMaxPod / 2 + 1], qq[kMaxPod / 2 + 1], rot[kMaxPod / 2 + 1];
  __shared__ int rotated;
  __shared__ double floor_abs;
  __shared__ int kk;
  const int tid = threadIdx.x;
  const int me = (m + 1) & ~1;  // even size for the round-robin ordering (padding index is inert)
  const int np = me / 2;
  for (int s = tid; s < me * me; s += blockDim.x) {
    const int p = s / me, q = s % me;
    Mt[s] = (p < m && q < m) ? Gg[p * kMaxPod + q] : 0.0;
    V[s] = (p == q) ? 1.0 : 0.0;
  }
  for (int p = tid >> 5; p < m; p += blockDim.x >> 5) {
    const int tile = p / 8;
    const double v = sum_part(part + (size_t)tile * nblk * kTileSlots, nblk, 64 + (p % 8));
    if ((tid & 31) == 0) gv[p] = v;
  }
  __syncthreads();
  if (tid == 0) {
    double tr = 0.0;
    for (int p = 0; p < m; ++p) tr += fabs(Mt[p * me + p]);
    floor_abs = 1e-15 * tr;
  }
  __syncthreads();
  // parallel-order cyclic Jacobi: me-1 rounds of me/2 disjoint rotations per sweep.
  // Threshold rule: a pair is rotated only while |a_pq| > 1e-15 sqrt(|a_pp a_qq|)
  // (relative to its own diagonal, so small eigenvalues keep their relative accuracy)
  // and |a_pq| > 1e-15 trace(G) (the FP64 rounding level of the matrix: eigenvalues
  // below it are noise, and far below the POD truncation at sigma_i/sigma_1 >= eps_POD);
  // the sweep that rotates no pair ends the iteration.  (An off-norm test against the
  // total norm cannot be met below the rounding level and ran every sweep.)
  // A round applies J^T M J (J: the round's rotations, block diagonal over its pairs) in one
  // pass over the 2 x 2 blocks of M on and above the block diagonal, from one buffer into the
  // other (Mt / Hs; Hs is free until the Galerkin system), and V <- V J on the rotated pairs'
  // columns: two barriers per round.  Pairs left alone cost no arithmetic.
  // the round-robin schedule of every round (pair t of round r at sched[r * np + t],
  // packed p | q << 8, p < q) and this thread's fixed share of the block and V updates,
  // formed once: the rounds then do no integer division
  __shared__ unsigned short sched[(kMaxPod - 1) * (kMaxPod / 2)];
  for (int w = tid; w < (me - 1) * np; w += blockDim.x) {
    const int round = w / np, t = w - round * np;
    // circle method: index me-1 meets `round`, the others pair symmetrically
    const int a = (t == 0) ? me - 1 : (round + t) % (me - 1);
    const int b = (t == 0) ? round : (round - t + me - 1) % (me - 1);
    sched[w] = (unsigned short)((a < b ? a : b) | ((a < b ? b : a) << 8));
  }
  constexpr int kMItems = (kMaxPod / 2) * (kMaxPod / 2) / kPodThreads + 1;   // blocks (i, j) per thread
  constexpr int kVItems = kMaxPod * (kMaxPod / 2) / kPodThreads + 1;         // (row, pair) V items per thread
  int mi[kMItems], mj[kMItems], vr[kVItems], vt[kVItems];
#pragma unroll
  for (int u = 0; u < kMItems; ++u) {
    const int w = tid + kPodThreads * u;
    const int i = w / np, j = w - (w / np) * np;
    const bool ok = w < np * np && i <= j;
    mi[u] = ok ? i : -1;
    mj[u] = j;
  }
#pragma unroll
  for (int u = 0; u < kVItems; ++u) {
    const int w = tid + kPodThreads * u;
    vr[u] = (w < me * np) ? w / np : -1;
    vt[u] = w - (w / np) * np;
  }
  __syncthreads();
  double* cur = Mt;
  double* nxt = Hs;
  for (int sweep = 0; sweep < 40 && me >= 2; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int round = 0; round < me - 1; ++round) {
      if (tid < np) {
        const int pq = sched[round * np + tid];
        const int p = pq & 0xFF, q = pq >> 8;
        pp[tid] = p; qq[tid] = q;
        const double apq = cur[p * me + q], app = cur[p * me + p], aqq = cur[q * me + q];
        double c = 1.0, s = 0.0;
        const int r = fabs(apq) > floor_abs && fabs(apq) > 1e-15 * sqrt(fabs(app * aqq));
        if (r) {
          jacobi_rotation(app, aqq, apq, c, s);
          rotated = 1;
        }
        cs[tid] = c; sn[tid] = s; rot[tid] = r;
      }
      __syncthreads();
      // M' = J^T M J by 2 x 2 blocks (pair i rows, pair j columns, i <= j), mirrored below
#pragma unroll
      for (int u = 0; u < kMItems; ++u) {
        const int i = mi[u], j = mj[u];
        if (i < 0) continue;
        const int pi = pp[i], qi = qq[i], pj = pp[j], qj = qq[j];
        double b00 = cur[pi * me + pj], b01 = cur[pi * me + qj], b10 = cur[qi * me + pj], b11 = cur[qi * me + qj];
        if (rot[j]) {
          const double c = cs[j], s = sn[j];
          const double n00 = fma(c, b00, -s * b01), n01 = fma(s, b00, c * b01);
          const double n10 = fma(c, b10, -s * b11), n11 = fma(s, b10, c * b11);
          b00 = n00; b01 = n01; b10 = n10; b11 = n11;
        }
        if (rot[i]) {
          const double c = cs[i], s = sn[i];
          const double n00 = fma(c, b00, -s * b10), n10 = fma(s, b00, c * b10);
          const double n01 = fma(c, b01, -s * b11), n11 = fma(s, b01, c * b11);
          b00 = n00; b01 = n01; b10 = n10; b11 = n11;
        }
        if (i == j) {
          const double o = 0.5 * (b01 + b10);
          b01 = o; b10 = o;
        }
        nxt[pi * me + pj] = b00; nxt[pi * me + qj] = b01; nxt[qi * me + pj] = b10; nxt[qi * me + qj] = b11;
        if (i != j) {
          nxt[pj * me + pi] = b00; nxt[qj * me + pi] = b01; nxt[pj * me + qi] = b10; nxt[qj * me + qi] = b11;
        }
      }
      // V <- V J on the rotated pairs
#pragma unroll
      for (int u = 0; u < kVItems; ++u) {
        const int row = vr[u], t = vt[u];
        if (row < 0 || !rot[t]) continue;
        const int p = pp[t], q = qq[t];
        const double c = cs[t], s = sn[t];
        const double vp = V[row * me + p], vq = V[row * me + q];
        V[row * me + p] = fma(c, vp, -s * vq);
        V[row * me + q] = fma(s, vp, c * vq);
      }
      __syncthreads();
      double* sw_ = cur; cur = nxt; nxt = sw_;
    }
    // every thread reads the flag before the barrier; thread 0 resets it only after,
    // so all threads take the same branch
    const int any = rotated;
    __syncthreads();
    if (!any) break;
  }
  // eigenvalues in descending order (ties by index): each thread places one by its rank
  for (int p = tid; p < m; p += blockDim.x) {
    const double lp = cur[p * me + p];
    const double kp = (lp == lp) ? lp : -INFINITY;       // a NaN ranks last: the ranks stay a permutation
    int rank = 0;
    for (int q = 0; q < m; ++q) {
      const double lq = cur[q * me + q];
      const double kq = (lq == lq) ? lq : -INFINITY;
      rank += (kq > kp || (kq == kp && q < p)) ? 1 : 0;
    }
    lam[p] = lp;
    order[rank] = p;
  }
  __syncthreads();
  for (int a = tid; a < m; a += blockDim.x) y[a] = sqrt(fmax(lam[order[a]], 0.0));   // sigma_a (y is free here)
  __syncthreads();
  if (tid == 0) {
    const double s1 = y[0];
    int k = 0;
    double sk = 0.0, sall = 0.0;
    for (int a = 0; a < m; ++a) {
      const double sa = y[a];
      sall += sa;
      if (s1 > 0.0 && sa / s1 >= eps_pod) { ++k; sk += sa; }
      if (sigma_out) sigma_out[a] = sa;
    }
    kk = k;
    out->rank = k;
    out->info = (sall > 0.0) ? sk / sall : 0.0;
  }
  __syncthreads();
  const int k = kk;
  if (k == 0) {
    for (int p = tid; p < m; p += blockDim.x) coef[p] = 0.0;
    return;
  }
  // W = X^T K X V_k Sigma_k^-1 (m x k) then H = Sigma_k^-1 V_k^T W (k x k)
  for (int s = tid; s < m * k; s += blockDim.x) {
    const int p = s / k, a = s % k, col = order[a];
    const double inv = 1.0 / sqrt(lam[col]);
    double v = 0.0;
    for (int q = 0; q < m; ++q) v = fma(Ag[p * kMaxPod + q], V[q * me + col], v);
    W[p * k + a] = v * inv;
  }
  __syncthreads();
  for (int s = tid; s < k * k; s += blockDim.x) {
    const int a = s / k, b = s % k, col = order[a];
    const double inv = 1.0 / sqrt(lam[col]);
    double v = 0.0;
    for (int p = 0; p < m; ++p) v = fma(V[p * me + col], W[p * k + b], v);
    Hs[s] = v * inv;
  }
  __syncthreads();   // W (aliasing Ls) fully consumed
  for (int a = tid; a < k; a += blockDim.x) {
    const int col = order[a];
    double v = 0.0;
    for (int p = 0; p < m; ++p) v = fma(V[p * me + col], gv[p], v);
    rhs[a] = v / sqrt(lam[col]);
  }
  __syncthreads();
  for (int s = tid; s < k * k; s += blockDim.x) {  // symmetrise
    const int a = s / k, b = s % k;
    if (a < b) { const double v = 0.5 * (Hs[a * k + b] + Hs[b * k + a]); Hs[a * k + b] = v; Hs[b * k + a] = v; }
  }
  __syncthreads();
  chol_drop_solve(Hs, rhs, y, k, 0.0, 1e-14, Ls, keep);
  // z = V_k Sigma_k^-1 y
  for (int p = tid; p < m; p += blockDim.x) {
    double v = 0.0;
    for (int a = 0; a < k; ++a) {
      const int col = order[a];
      v = fma(V[p * me + col], y[a] / sqrt(lam[col]), v);
    }
    coef[p] = v;
  }
}

// ---- cascaded SPE (K-orthonormal frozen columns + the newest solution) ----
__device__ __forceinline__ double tile_dot(const double* part, int nblk, int q) {
  return sum_part(part + (size_t)(q / 8) * nblk * kTileSlots, nblk, 64 + (q % 8));
}

// coef = [1, -h_1 .. -h_k] with h_i = product i; scal[0] = product k (x.Lx) when with_norm
// (one warp per value)
__global__ void cspe_proj_kernel(const double* part, int nblk, int k, int with_norm, double* coef, double* scal) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) coef[0] = 1.0;
  for (int q = wid; q < k + (with_norm ? 1 : 0); q += nw) {
    const double v = tile_dot(part, nblk, q);
    if (lane == 0) {
      if (q < k) coef[q + 1] = -v;
      else scal[0] = v;
    }
  }
}

// x0 coefficients [Q^T b, (z.b)/zeta] from partC (Q_i.b, then z.b) and partD (z.Lz)
// (one warp per product)
__global__ void cspe_coef_kernel(const double* partC, const double* partD, int nblk, int k, double drop2,
                                 double* coef, double* scal, SmallOut* out) {
  __shared__ double zz[2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = wid; q < k + 2; q += nw) {
    const double v = (q <= k) ? tile_dot(partC, nblk, q) : tile_dot(partD, nblk, 0);
    if (lane == 0) {
      if (q < k) coef[q] = v;
      else zz[q - k] = v;              // zz[0] = z.b, zz[1] = z.Lz
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double zeta = zz[1], zb = zz[0];
    const bool keep = zeta > 0.0 && zeta > drop2 * scal[0];
    coef[k] = keep ? zb / zeta : 0.0;
    scal[1] = keep ? rsqrt(zeta) : 0.0;
    out->rank = k + (keep ? 1 : 0);
    out->info = 0.0;
  }
}

__global__ void __launch_bounds__(kTS) cspe_freeze_kernel(const double* z, const double* lz, double* q, double* p,
                                                          long long len, const double* scal) {
  const double s = scal[1];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x) {
    q[e] = s * z[e];
    p[e] = s * lz[e];
  }
}

// ---- SPE table in float-float (hi + lo FP32 pair, about 48 significant bits) ----
// On this GPU FP64 arithmetic is about 68x slower than FP32, and the Galerkin
// products of the SPE table are an FP64 multiply-add per table pair and element.
// The table is therefore kept as float-float pairs (8 bytes per value, as FP64):
// the backward differences, the Galerkin products and the linear combination run on
// the FP32 pipes with error-free transformations (two-sum, FMA product error), and
// FP64 is used only to convert the newest solution, its image and b in and x0 out.
// __fadd_rn / __fmul_rn are never contracted into FMAs, which the error terms need.
__device__ __forceinline__ float2 ff_split(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - (double)hi));
}
__device__ __forceinline__ double ff_join(float s, float e) { return (double)s + (double)e; }
__device__ __forceinline__ float2 ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ float2 ff_fast_two_sum(float a, float b) {   // |a| >= |b| or a = 0
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// a - b, both parts summed error-free (the difference of two close values keeps its
// relative accuracy, as an FP64 subtraction does)
__device__ __forceinline__ float2 ff_sub(float2 a, float2 b) {
  float2 s = ff_two_sum(a.x, -b.x);
  const float2 t = ff_two_sum(a.y, -b.y);
  s.y = __fadd_rn(s.y, t.x);
  s = ff_fast_two_sum(s.x, s.y);
  s.y = __fadd_rn(s.y, t.y);
  return ff_fast_two_sum(s.x, s.y);
}
// (S, E) += a * b: S sums the rounded products, E their rounding errors (FMA), the
// cross terms and the rounding of the S sums (two-sum)
__device__ __forceinline__ void ff_mac(float2 a, float2 b, float& S, float& E) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float s = __fadd_rn(S, p), bb = __fsub_rn(s, S);
  const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  S = s;
  E = __fadd_rn(E, __fadd_rn(err, e));
}
// (S1, E1) += (S2, E2)
__device__ __forceinline__ void ff_acc(float& S1, float& E1, float S2, float E2) {
  const float2 t = ff_two_sum(S1, S2);
  S1 = t.x;
  E1 = __fadd_rn(__fadd_rn(E1, E2), t.y);
}

// new table D_0 = w, D_p = D_{p-1}^new - D_{p-1}^old (and likewise for the images)
template <int MAXD>
__global__ void __launch_bounds__(kTS) diff_push_ff_kernel(MutVecSet D, MutVecSet LD, const double* __restrict__ w,
                                                          const double* __restrict__ lw, int m_old, int m_new,
                                                          long long len) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x) {
    float2 od[MAXD], ol[MAXD];
#pragma unroll
    for (int p = 0; p < MAXD; ++p)
      if (p < m_old) {
        od[p] = reinterpret_cast<const float2*>(D.v[p])[e];
        ol[p] = reinterpret_cast<const float2*>(LD.v[p])[e];
      }
    float2 t = ff_split(w[e]), tl = ff_split(lw[e]);
#pragma unroll
    for (int p = 0; p < MAXD; ++p)
      if (p < m_new) {
        reinterpret_cast<float2*>(D.v[p])[e] = t;
        reinterpret_cast<float2*>(LD.v[p])[e] = tl;
        if (p < m_old) { t = ff_sub(t, od[p]); tl = ff_sub(tl, ol[p]); }
      }
  }
}

// ---- SPE products: float-float partial sums ---------------------------------------------
// Every product kernel below accumulates (S, E) pairs per thread (ff_mac), reduces
// them across the warp by a reduce-scatter (four halvings over lane offsets 16..2,
// then a butterfly over offset 1: the even lanes end with NS/16 slots each), sums
// the warps' pairs in shared memory and writes one normalised float-float partial
// per slot and block (float2 in the 8-byte slots of the partial buffers).  The
// small solve sums the partials of all blocks on the FP32 pipes as well.
template <int NS>
__device__ __forceinline__ void warp_scatter_ff(float (&vs)[NS], float (&ve)[NS]) {
  static_assert(NS % 16 == 0, "slots in multiples of 16");
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int half = NS / 2, off = 16; off >= 2; half >>= 1, off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float ks = up ? vs[i + half] : vs[i], ke = up ? ve[i + half] : ve[i];
      const float ss = up ? vs[i] : vs[i + half], se = up ? ve[i] : ve[i + half];
      vs[i] = ks;
      ve[i] = ke;
      ff_acc(vs[i], ve[i], __shfl_xor_sync(0xffffffffu, ss, off), __shfl_xor_sync(0xffffffffu, se, off));
    }
  }
#pragma unroll
  for (int i = 0; i < NS / 16; ++i)
    ff_acc(vs[i], ve[i], __shfl_xor_sync(0xffffffffu, vs[i], 1), __shfl_xor_sync(0xffffffffu, ve[i], 1));
}

// Block partials of NS slots: slot s goes to row[dst(s)] (dst < 0: not stored).
// red: shared (kTS / 32) x NS float2.  All threads of the block call.
template <int NS, class Dst>
__device__ __forceinline__ void block_partials_ff(float (&vs)[NS], float (&ve)[NS], float2 (*red)[NS], Dst dst,
                                                  float2* row) {
  warp_scatter_ff<NS>(vs, ve);
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  constexpr int FIN = NS / 16;
  if ((lane & 1) == 0) {
    const int base = FIN * (8 * ((lane >> 4) & 1) + 4 * ((lane >> 3) & 1) + 2 * ((lane >> 2) & 1) + ((lane >> 1) & 1));
#pragma unroll
    for (int i = 0; i < FIN; ++i) red[wp][base + i] = make_float2(vs[i], ve[i]);
  }
  __syncthreads();
  for (int s = threadIdx.x; s < NS; s += blockDim.x) {
    const int d = dst(s);
    if (d < 0) continue;
    float S = red[0][s].x, E = red[0][s].y;
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) ff_acc(S, E, red[q][s].x, red[q][s].y);
    row[d] = ff_fast_two_sum(S, E);
  }
}

// Galerkin products of float-float tables (slot layout of dots_kernel's tiles):
// kTri: A_p . B_q, q >= p < 8; kRect4: 8 columns of A x 4 rows of B; kTri4: the
// 4 x 4 triangle.  part: float2 partials, kTileSlots per block.
template <int MODE>
__global__ void __launch_bounds__(kTS, 1) dots_ff_kernel(VecSet A, VecSet B, int ma, int mb, long long len,
                                                        float2* part) {
  constexpr bool TRI4 = (MODE == kTri4);
  constexpr bool DIAG = (MODE == kTri) || TRI4;
  constexpr bool RECT = (MODE == kRect4);
  constexpr int NA = TRI4 ? 4 : 8;
  constexpr int NB = (RECT || TRI4) ? 4 : 8;
  constexpr int NP = (MODE == kTri) ? 36 : (TRI4 ? 10 : 32);
  constexpr int NS = (NP + 15) / 16 * 16;
  float S[NS], E[NS];
#pragma unroll
  for (int t = 0; t < NS; ++t) { S[t] = 0.f; E[t] = 0.f; }
  const long long stride = (long long)gridDim.x * blockDim.x;
  float2 a[NA], b[NB];
  auto load = [&](long long e, float2* aa, float2* bb) {
#pragma unroll
    for (int p = 0; p < NA; ++p) aa[p] = (p < ma) ? reinterpret_cast<const float2*>(A.v[p])[e] : make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < NB; ++q) bb[q] = (q < mb) ? reinterpret_cast<const float2*>(B.v[q])[e] : make_float2(0.f, 0.f);
  };
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e < len) load(e, a, b);
  for (; e < len; e += stride) {
    // the next element's inputs are in flight while this one is reduced
    float2 an[NA], bn[NB];
    if (e + stride < len) load(e + stride, an, bn);
    int t = 0;
#pragma unroll
    for (int p = 0; p < NA; ++p) {
#pragma unroll
      for (int q = (DIAG ? p : 0); q < NB; ++q, ++t)
        if (p < ma && q < mb) ff_mac(a[p], b[q], S[t], E[t]);
    }
#pragma unroll
    for (int p = 0; p < NA; ++p) a[p] = an[p];
#pragma unroll
    for (int q = 0; q < NB; ++q) b[q] = bn[q];
  }
  __shared__ float2 red[kTS / 32][NS];
  float2* row = part + (size_t)blockIdx.x * kTileSlots;
  if (MODE == kTri) {
    block_partials_ff<NS>(S, E, red, [](int s) { return s < 36 ? c_tri_slot[s] : -1; }, row);
  } else if (TRI4) {
    // product t of the 4 x 4 triangle (p, then q >= p) -> slot p * 8 + q
    block_partials_ff<NS>(S, E, red, [](int s) {
      const int p = s < 4 ? 0 : s < 7 ? 1 : s < 9 ? 2 : s < 10 ? 3 : -1;
      const int q = s < 4 ? s : s < 7 ? s - 3 : s < 9 ? s - 5 : s - 6;
      return p < 0 ? -1 : p * 8 + q;
    }, row);
  } else {
    // product p * 4 + q (column p of A, row q of B) -> slot p * 8 + q
    block_partials_ff<NS>(S, E, red, [](int s) { return (s >> 2) * 8 + (s & 3); }, row);
  }
}

// Push of the newest solution w (image lw) into the float-float table fused with the
// Galerkin products of the new table (tile 0: D_q . LD_p, p <= q < m_new <= 8):
// one pass over the table instead of a push and a second pass re-reading it.
// New table: D_0 = w, D_p = D_{p-1}^new - D_{p-1}^old (and likewise the images).
__device__ void spe_solve_body(const float2* gpart, int nbg, int m, const SpeFac* fac, double* coef, SmallOut* out);

// True in the block that arrives last at this call (every block calls it once, after its
// global writes); that block also returns the counter to zero for the next launch.  No
// block waits for another.
__device__ __forceinline__ bool last_block(unsigned* ctr) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    last = atomicAdd(ctr, 1u) == gridDim.x - 1;
    if (last) atomicExch(ctr, 0u);
  }
  __syncthreads();
  if (last) __threadfence();
  return last != 0;
}

__global__ void __launch_bounds__(kTS, 1) spe_push_dots_kernel(MutVecSet D, MutVecSet LD, const double* __restrict__ w,
                                                              const double* __restrict__ lw, int m_old, int m_new,
                                                              long long len, float2* part) {
  constexpr int M = 8;
  float S[48], E[48];
#pragma unroll
  for (int t = 0; t < 48; ++t) { S[t] = 0.f; E[t] = 0.f; }
  const long long stride = (long long)gridDim.x * blockDim.x;
  float2 od[M], ol[M];
  double we = 0.0, lwe = 0.0;
  auto load = [&](long long e, float2* a, float2* b, double& x, double& y) {
#pragma unroll
    for (int p = 0; p < M; ++p) {
      a[p] = (p < m_old) ? reinterpret_cast<const float2*>(D.v[p])[e] : make_float2(0.f, 0.f);
      b[p] = (p < m_old) ? reinterpret_cast<const float2*>(LD.v[p])[e] : make_float2(0.f, 0.f);
    }
    x = w[e];
    y = lw[e];
  };
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e < len) load(e, od, ol, we, lwe);
  for (; e < len; e += stride) {
    float2 nd[M], nl[M];
    double wn = 0.0, lwn = 0.0;
    if (e + stride < len) load(e + stride, nd, nl, wn, lwn);
    float2 cd[M], cl[M];
    float2 t = ff_split(we), tl = ff_split(lwe);
#pragma unroll
    for (int p = 0; p < M; ++p) {
      cd[p] = t;
      cl[p] = tl;
      if (p < m_new) {
        reinterpret_cast<float2*>(D.v[p])[e] = t;
        reinterpret_cast<float2*>(LD.v[p])[e] = tl;
      }
      if (p + 1 < M && p < m_old) { t = ff_sub(t, od[p]); tl = ff_sub(tl, ol[p]); }
    }
    int k = 0;
#pragma unroll
    for (int p = 0; p < M; ++p) {
#pragma unroll
      for (int q = p; q < M; ++q, ++k)
        if (q < m_new) ff_mac(cl[p], cd[q], S[k], E[k]);
    }
#pragma unroll
    for (int p = 0; p < M; ++p) { od[p] = nd[p]; ol[p] = nl[p]; }
    we = wn;
    lwe = lwn;
  }
  __shared__ float2 red[kTS / 32][48];
  block_partials_ff<48>(S, E, red, [](int s) { return s < 36 ? c_tri_slot[s] : -1; },
                        part + (size_t)blockIdx.x * kTileSlots);
}

// g_q = D_q . b (q < m <= MAXM) over the listed layout indices (idx != nullptr) or
// the edges of the positions in box (b is zero elsewhere); float-float partials,
// kSpeGSlots per block.  The last block to finish sums them and solves with the
// factor in fac (spe_solve_body): coef = y.
template <int MAXM>
__global__ void __launch_bounds__(kTS) spe_g_kernel(VecSet D, const double* __restrict__ b, int m, int n, Box box,
                                                    const int* __restrict__ idx, int nidx, float2* gpart,
                                                    SpeFac* fac, double* coef, SmallOut* out) {
  const int bx = box.hi[0] - box.lo[0], by = box.hi[1] - box.lo[1], bz = box.hi[2] - box.lo[2];
  const int npos = bx * by * bz;
  const long long n3 = (long long)n * n * n;
  const int cnt = idx ? nidx : 3 * npos;
  float S[16], E[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) { S[q] = 0.f; E[q] = 0.f; }
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < cnt; u += gridDim.x * blockDim.x) {
    long long e;
    if (idx) {
      e = idx[u];
    } else {
      const int c = u / npos, r = u - c * npos;
      const int i = box.lo[0] + r % bx, j = box.lo[1] + (r / bx) % by, k = box.lo[2] + r / (bx * by);
      e = c * n3 + i + (long long)n * (j + (long long)n * k);
    }
    const double be = MQS_LDC(b, e, 3 * n3, 601);
    if (be != 0.0) {
      const float2 bf = ff_split(be);
#pragma unroll
      for (int q = 0; q < MAXM; ++q)
        if (q < m) ff_mac(MQS_LDC(reinterpret_cast<const float2*>(D.v[q]), e, 3 * n3, 602), bf, S[q], E[q]);
    }
  }
  __shared__ float2 red[kTS / 32][16];
  block_partials_ff<16>(S, E, red, [](int s) { return s; }, gpart + (size_t)blockIdx.x * kSpeGSlots);
  if (last_block(&fac->g_done)) spe_solve_body(gpart, gridDim.x, m, fac, coef, out);
}

// x = sum_p coef_p V_p with float-float V and FP64 coefficients
template <int MAXM>
__global__ void __launch_bounds__(kTS) lincomb_ff_kernel(VecSet V, const double* coef, int m, long long len,
                                                        double* x) {
  __shared__ float2 cf[kMaxVec];
  for (int p = threadIdx.x; p < kMaxVec; p += blockDim.x) cf[p] = (p < m) ? ff_split(coef[p]) : make_float2(0.f, 0.f);
  __syncthreads();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x) {
    float2 v[MAXM];
#pragma unroll
    for (int p = 0; p < MAXM; ++p) v[p] = (p < m) ? reinterpret_cast<const float2*>(V.v[p])[e] : make_float2(0.f, 0.f);
    float s = 0.f, ee = 0.f;
#pragma unroll
    for (int p = 0; p < MAXM; ++p)
      if (p < m) ff_mac(cf[p], v[p], s, ee);
    x[e] = ff_join(s, ee);
  }
}

// Sum over cnt blocks of one float-float partial (base[q * stride], q < cnt) by one
// warp: loads issued together, a fixed pairwise tree, a shuffle butterfly; lane 0
// holds the defined value.
__device__ __forceinline__ ffv sum_parts_ff(const float2* base, int stride, int cnt) {
  const int lane = threadIdx.x & 31;
  ffv v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int q = lane + 32 * r;
    const float2 f = (q < cnt) ? __ldcg(base + (size_t)q * stride) : make_float2(0.f, 0.f);
    v[r] = ffv(f.x, f.y);
  }
#pragma unroll
  for (int w2 = 8; w2 >= 1; w2 >>= 1)
#pragma unroll
    for (int r = 0; r < w2; ++r) v[r] = v[r] + v[r + w2];
  ffv s = v[0];
  for (int q = lane + 512; q < cnt; q += 32) {
    const float2 f = __ldcg(base + (size_t)q * stride);
    s = s + ffv(f.x, f.y);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s = s + shfl_x(s, o);
  return s;
}

// SPE small system, first half (needs only the table): sums the product partials
// (entries (q, p), q >= p, of H = D^T K D in tiles of 8: tile 0 rows/columns 0-7,
// tiles 1 and 3 rows 8-11 and 12-15 against columns 0-7, tile 2 rows/columns 8-15)
// and factors H (pivoted Cholesky with the drop rule, register form, warp 0) into fac.
__device__ void spe_factor_body(const float2* hpart, int nbh, int m, double drop2, SpeFac* fac) {
  __shared__ double H[kMaxSpe * kMaxSpe];
  __shared__ double vals[kMaxSpe * (kMaxSpe + 1) / 2];
  const int npair = m * (m + 1) / 2;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = wid; t < npair; t += nw) {
    int qq = 0;
    while ((qq + 1) * (qq + 2) / 2 <= t) ++qq;
    const int pp = t - qq * (qq + 1) / 2;
    int tile, slot;
    if (qq < 8) { tile = 0; slot = pp * 8 + qq; }
    else if (pp < 8) { tile = qq < 12 ? 1 : 3; slot = pp * 8 + (qq < 12 ? qq - 8 : qq - 12); }
    else { tile = 2; slot = (pp - 8) * 8 + (qq - 8); }
    const ffv s = sum_parts_ff(hpart + (size_t)tile * nbh * kTileSlots + slot, kTileSlots, nbh);
    if (lane == 0) vals[t] = ff_to(s);
  }
  __syncthreads();
  for (int s = threadIdx.x; s < m * m; s += blockDim.x) {
    const int p = s / m, q = s % m;
    const int pp = p < q ? p : q, qq = p < q ? q : p;
    H[s] = vals[qq * (qq + 1) / 2 + pp];
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double inv, sc;
    int nk;
    if (m <= 8) {
      double h[8];
      nk = chol_drop_factor_reg<8>(H, m, drop2, 1e-13, h, inv, sc);
      if (lane < m)
        for (int c = 0; c < 8; ++c) fac->L[lane * kMaxSpe + c] = h[c];
    } else {
      double h[16];
      nk = chol_drop_factor_reg<16>(H, m, drop2, 1e-13, h, inv, sc);
      if (lane < m)
#pragma unroll
        for (int c = 0; c < 16; ++c) fac->L[lane * kMaxSpe + c] = h[c];
    }
    if (lane < m) { fac->inv[lane] = inv; fac->sc[lane] = sc; }
    if (lane == 0) { fac->nk = nk; fac->m = m; }
  }
}

__global__ void __launch_bounds__(512) spe_factor_kernel(const float2* hpart, int nbh, int m, double drop2,
                                                         SpeFac* fac) {
  spe_factor_body(hpart, nbh, m, drop2, fac);
}

// Second half (needs b): sums g = D^T b from its partials, the substitutions with
// fac, coef = y.  Any block size that is a multiple of 32.
__device__ void spe_solve_body(const float2* gpart, int nbg, int m, const SpeFac* fac, double* coef, SmallOut* out) {
  __shared__ double g[kMaxSpe], y[kMaxSpe];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = wid; t < m; t += nw) {
    const ffv s = sum_parts_ff(gpart + t, kSpeGSlots, nbg);
    if (lane == 0) g[t] = ff_to(s);
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool own = lane < m;
    const double inv = own ? fac->inv[lane] : 0.0, sc = own ? fac->sc[lane] : 0.0;
    if (m <= 8) {
      double h[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) h[c] = own ? fac->L[lane * kMaxSpe + c] : 0.0;
      chol_solve_reg<8>(h, inv, sc, g, y, m);
    } else {
      double h[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) h[c] = own ? fac->L[lane * kMaxSpe + c] : 0.0;
      chol_solve_reg<16>(h, inv, sc, g, y, m);
    }
    __syncwarp();
    if (own) coef[lane] = y[lane];
    if (lane == 0) { out->rank = fac->nk; out->info = 0.0; }
  }
}

// ---- host launchers --------------------------------------------------------------------
static int ts_max_blocks() {
  static int nb = 0;
  if (nb == 0) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    nb = (nsm > 0 ? nsm : 132) * 2;
  }
  return nb;
}

thread_local int t_launch_cap = 0;
void set_launch_cap(int cap) { t_launch_cap = cap > 0 ? cap : 0; }
int launch_cap() { return t_launch_cap; }
static int capped(int nb) { return (t_launch_cap > 0 && nb > t_launch_cap) ? t_launch_cap : nb; }

// blocks of a tall-skinny pass over len values: at least 8 values per thread, at
// most two blocks per SM (small problems do not flood the GPU with empty blocks), at
// most the launch cap
static int ts_blocks(long long len) {
  const long long want = (len + (long long)kTS * 8 - 1) / ((long long)kTS * 8);
  return capped((int)std::min<long long>(std::max<long long>(want, 8), ts_max_blocks()));
}
int ts_nblk() { return ts_max_blocks(); }

static int chk() { return cudaGetLastError() == cudaSuccess ? MQS_OK : MQS_ERR_CUDA; }

int spe_hblocks(long long len, int m) {
  // the fused push + product pass keeps one block per SM (its registers); the
  // separate product tiles (more than 8 columns) run ts_blocks blocks
  return m <= 8 ? std::min(ts_blocks(len), ts_max_blocks() / 2) : ts_blocks(len);
}
int spe_gblocks() { return ts_max_blocks(); }

int spe_factor(const double* hpart, int m, int nbh, double eps_lin, SpeFac* fac, cudaStream_t st) {
  if (m <= 0 || m > kMaxSpe || nbh <= 0) return MQS_ERR_ARG;
  spe_factor_kernel<<<1, 512, 0, st>>>(reinterpret_cast<const float2*>(hpart), nbh, m, eps_lin * eps_lin, fac);
  return chk();
}

int spe_push(const MutVecSet& D, const MutVecSet& LD, const double* w, const double* lw, int m_old, int m_new,
             long long len, double* hpart, double eps_lin, SpeFac* fac, cudaStream_t st) {
  float2* hp = reinterpret_cast<float2*>(hpart);
  if (m_new <= 8) {
    spe_push_dots_kernel<<<spe_hblocks(len, m_new), kTS, 0, st>>>(D, LD, w, lw, m_old, m_new, len, hp);
    return spe_factor(hpart, m_new, spe_hblocks(len, m_new), eps_lin, fac, st);
  }
  diff_push_ff_kernel<16><<<ts_blocks(len) * 2, kTS, 0, st>>>(D, LD, w, lw, m_old, m_new, len);
  // Entry (q, p), q >= p, of the Galerkin matrix is D_q . (K D_p): the
  // high-order differences are tested against the K-images of the low-order
  // ones, which the recursion carries accurately (the images of high orders
  // accumulate its rounding relative to their small size).
  const int nb = spe_hblocks(len, m_new), m = m_new;
  VecSet A0{}, B0{};
  for (int p = 0; p < 8; ++p) { A0.v[p] = LD.v[p]; B0.v[p] = D.v[p]; }
  dots_ff_kernel<kTri><<<nb, kTS, 0, st>>>(A0, B0, 8, 8, len, hp);
  // rows 8.. of D against the first 8 images, in 8 x 4 tiles (tile 1: rows 8-11, tile 3: rows 12-15)
  for (int h = 0; h < 2 && 8 + 4 * h < m; ++h) {
    VecSet A1{}, B1{};
    const int r0 = 8 + 4 * h, rows = (m - r0) < 4 ? (m - r0) : 4;
    for (int p = 0; p < 8; ++p) A1.v[p] = LD.v[p];
    for (int q = 0; q < 8; ++q) B1.v[q] = D.v[q < rows ? r0 + q : r0];
    dots_ff_kernel<kRect4><<<nb, kTS, 0, st>>>(A1, B1, 8, rows, len, hp + (size_t)(h == 0 ? 1 : 3) * nb * kTileSlots);
  }
  VecSet A2{}, B2{};
  for (int p = 0; p < 8; ++p) { A2.v[p] = LD.v[8 + p < m ? 8 + p : 8]; B2.v[p] = D.v[8 + p < m ? 8 + p : 8]; }
  if (m <= 12) dots_ff_kernel<kTri4><<<nb, kTS, 0, st>>>(A2, B2, m - 8, m - 8, len, hp + (size_t)2 * nb * kTileSlots);
  else dots_ff_kernel<kTri><<<nb, kTS, 0, st>>>(A2, B2, m - 8, m - 8, len, hp + (size_t)2 * nb * kTileSlots);
  return spe_factor(hpart, m, nb, eps_lin, fac, st);
}

int spe_x0(const VecSet& D, int m, const double* b, int n, const Box& bbox, const int* sup, int nsup, double* x0,
           long long len, SpeFac* fac, double* gpart, double* coef, SmallOut* out, cudaStream_t st) {
  if (m <= 0) {
    if (cudaMemsetAsync(x0, 0, sizeof(double) * len, st) != cudaSuccess) return MQS_ERR_CUDA;
    return MQS_OK;
  }
  if (m > kMaxSpe) return MQS_ERR_ARG;
  // g: about one edge per thread (most of the region's b vanishes: latency, not bandwidth)
  const long long edges =
      sup ? nsup : 3LL * (bbox.hi[0] - bbox.lo[0]) * (bbox.hi[1] - bbox.lo[1]) * (bbox.hi[2] - bbox.lo[2]);
  const int nbg = capped((int)std::min<long long>(std::max<long long>((edges + kTS - 1) / kTS, 1), spe_gblocks()));
  float2* gp = reinterpret_cast<float2*>(gpart);
  if (m <= 8) spe_g_kernel<8><<<nbg, kTS, 0, st>>>(D, b, m, n, bbox, sup, nsup, gp, fac, coef, out);
  else spe_g_kernel<16><<<nbg, kTS, 0, st>>>(D, b, m, n, bbox, sup, nsup, gp, fac, coef, out);
  const int nl = ts_blocks(len) * 4;
  if (m <= 8) lincomb_ff_kernel<8><<<nl, kTS, 0, st>>>(D, coef, m, len, x0);
  else if (m <= 12) lincomb_ff_kernel<12><<<nl, kTS, 0, st>>>(D, coef, m, len, x0);
  else lincomb_ff_kernel<16><<<nl, kTS, 0, st>>>(D, coef, m, len, x0);
  return chk();
}

int pod_push(const VecSet& X, const double* w, const double* lw, int m, int slot_new, long long len, double* part,
             double* G, double* A, cudaStream_t st) {
  const int nb = ts_blocks(len);
  const int ntile = (m + 7) / 8;
  for (int t = 0; t < ntile; ++t) {
    VecSet Aw, Bx;
    Aw.v[0] = w; Aw.v[1] = lw;
    const int mb = (m - 8 * t) < 8 ? (m - 8 * t) : 8;
    for (int q = 0; q < 8; ++q) Bx.v[q] = X.v[8 * t + (q < mb ? q : 0)];
    dots_kernel<kRow2><<<nb, kTS, 0, st>>>(Aw, Bx, nullptr, 2, mb, len, part + (size_t)t * nb * kTileSlots);
  }
  pod_row_kernel<<<1, 256, 0, st>>>(part, nb, m, slot_new, G, A);
  return chk();
}

int pod_x0(const VecSet& X, int m, const double* G, const double* A, const double* b, double* x0, long long len,
           double eps_pod, double* part, double* coef, double* sigma, SmallOut* out, cudaStream_t st,
           const VecSet* LX, double* r0) {
  const int nb = ts_blocks(len);
  if (m <= 0) {
    if (x0 && cudaMemsetAsync(x0, 0, sizeof(double) * len, st) != cudaSuccess) return MQS_ERR_CUDA;
    return MQS_OK;
  }
  const int ntile = (m + 7) / 8;
  for (int t = 0; t < ntile; ++t) {
    VecSet Ax;
    const int mb = (m - 8 * t) < 8 ? (m - 8 * t) : 8;
    for (int q = 0; q < 8; ++q) Ax.v[q] = X.v[8 * t + (q < mb ? q : 0)];
    dots_kernel<kConly><<<nb, kTS, 0, st>>>(Ax, Ax, b, 0, mb, len, part + (size_t)t * nb * kTileSlots);
  }
  pod_solve_kernel<<<1, kPodThreads, 0, st>>>(G, A, part, nb, m, eps_pod, coef, sigma, out);
  if (x0 && r0 && LX) launch_lincomb_res(X, *LX, coef, m, b, len, x0, r0, nb, st);
  else if (x0) launch_lincomb(X, coef, m, len, x0, nb, st);
  return chk();
}

// products X_q . v for q < m (tiles of eight, kConly) into part tiles 0 .. ceil(m/8)-1
static void dots_against(const VecSet& X, int m, const double* v, long long len, double* part, int nb,
                         cudaStream_t st) {
  for (int t = 0; t < (m + 7) / 8; ++t) {
    VecSet Ax;
    const int mb = (m - 8 * t) < 8 ? (m - 8 * t) : 8;
    for (int q = 0; q < 8; ++q) Ax.v[q] = X.v[8 * t + (q < mb ? q : 0)];
    dots_kernel<kConly><<<nb, kTS, 0, st>>>(Ax, Ax, v, 0, mb, len, part + (size_t)t * nb * kTileSlots);
  }
}

int cspe_x0(const CspeBufs& cb, int k, const double* x, const double* lx, const double* b, double* x0,
            long long len, double eps_lin, double* part, double* coef, SmallOut* out, cudaStream_t st) {
  if (k < 0 || k + 1 > kMaxCspe) return MQS_ERR_ARG;
  const int nb = ts_blocks(len);
  double* partC = part;                                   // tiles 0 .. 2
  double* partD = part + (size_t)3 * nb * kTileSlots;     // tile 3
  VecSet PX{}, V{}, W{};
  for (int i = 0; i < k; ++i) PX.v[i] = cb.P[i];
  PX.v[k] = lx;
  // pass 1: h = P^T x (= Q^T L x) and x.Lx; z = x - Q h, Lz = Lx - P h
  dots_against(PX, k + 1, x, len, part, nb, st);
  cspe_proj_kernel<<<1, 256, 0, st>>>(part, nb, k, 1, coef, cb.scal);
  V.v[0] = x;
  W.v[0] = lx;
  for (int i = 0; i < k; ++i) { V.v[1 + i] = cb.Q[i]; W.v[1 + i] = cb.P[i]; }
  launch_lincomb(V, coef, k + 1, len, cb.z, nb, st);
  launch_lincomb(W, coef, k + 1, len, cb.lz, nb, st);
  const double* zf = cb.z;
  const double* lzf = cb.lz;
  if (k > 0) {
    // pass 2 (re-orthogonalisation against the rounding of pass 1)
    dots_against(PX, k, cb.z, len, part, nb, st);
    cspe_proj_kernel<<<1, 256, 0, st>>>(part, nb, k, 0, coef, cb.scal);
    V.v[0] = cb.z;
    W.v[0] = cb.lz;
    launch_lincomb(V, coef, k + 1, len, cb.z2, nb, st);
    launch_lincomb(W, coef, k + 1, len, cb.lz2, nb, st);
    zf = cb.z2;
    lzf = cb.lz2;
  }
  // Galerkin system on the K-orthonormal basis: c = Q^T b, z.b, zeta = z.Lz
  VecSet QX{}, ZX{};
  for (int i = 0; i < k; ++i) QX.v[i] = cb.Q[i];
  QX.v[k] = zf;
  ZX.v[0] = zf;
  dots_against(QX, k + 1, b, len, partC, nb, st);
  dots_against(ZX, 1, lzf, len, partD, nb, st);
  cspe_coef_kernel<<<1, 256, 0, st>>>(partC, partD, nb, k, eps_lin * eps_lin, coef, cb.scal, out);
  launch_lincomb(QX, coef, k + 1, len, x0, nb, st);
  return chk();
}

int cspe_freeze(const CspeBufs& cb, int k, long long len, cudaStream_t st) {
  const double* z = k > 0 ? cb.z2 : cb.z;
  const double* lz = k > 0 ? cb.lz2 : cb.lz;
  cspe_freeze_kernel<<<ts_blocks(len) * 2, kTS, 0, st>>>(z, lz, cb.Q[k], cb.P[k], len, cb.scal);
  return chk();
}

MQS_DEBUG_TAKE(mrhs)

}  // namespace mqs
