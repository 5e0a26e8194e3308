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
#include <cmath>
#include "mrhs.h"

namespace mqs {

constexpr int kTS = 256;        // threads of the tall-skinny kernels

// ---- difference table push ---------------------------------------------------------
// All old entries of an element are loaded before any is overwritten (the
// table columns are distinct arrays, but the compiler cannot know it), two
// elements per thread per pass as double2.
template <int MAXD>
__global__ void __launch_bounds__(kTS) diff_push_kernel(MutVecSet D, MutVecSet LD, const double* __restrict__ w,
                                                       const double* __restrict__ lw, int m_old, int m_new,
                                                       long long len) {
  const long long half = len >> 1;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < half; e += stride) {
    double2 od[MAXD], ol[MAXD];
#pragma unroll
    for (int p = 0; p < MAXD; ++p)
      if (p < m_old) {
        od[p] = reinterpret_cast<const double2*>(D.v[p])[e];
        ol[p] = reinterpret_cast<const double2*>(LD.v[p])[e];
      }
    double2 t = reinterpret_cast<const double2*>(w)[e], tl = reinterpret_cast<const double2*>(lw)[e];
#pragma unroll
    for (int p = 0; p < MAXD; ++p)
      if (p < m_new) {
        reinterpret_cast<double2*>(D.v[p])[e] = t;
        reinterpret_cast<double2*>(LD.v[p])[e] = tl;
        if (p < m_old) {
          t.x -= od[p].x; t.y -= od[p].y;
          tl.x -= ol[p].x; tl.y -= ol[p].y;
        }
      }
  }
  if ((len & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const long long e = len - 1;
    double od[MAXD], ol[MAXD];
    for (int p = 0; p < m_old && p < MAXD; ++p) { od[p] = D.v[p][e]; ol[p] = LD.v[p][e]; }
    double t = w[e], tl = lw[e];
    for (int p = 0; p < m_new && p < MAXD; ++p) {
      D.v[p][e] = t; LD.v[p][e] = tl;
      if (p < m_old) { t -= od[p]; tl -= ol[p]; }
    }
  }
}

// ---- tiled dot products ------------------------------------------------------------
// part[blk * kTileSlots + p*8 + q] = sum_e A_p[e] B_q[e]   (p < ma, q < mb; q >= p if diag)
// part[blk * kTileSlots + 64 + q]  = sum_e B_q[e] c[e]     (if c != nullptr)
template <bool DIAG>
__global__ void __launch_bounds__(kTS) dots_kernel(VecSet A, VecSet B, const double* c, int ma, int mb,
                                                   long long len, double* part) {
  double acc[8][8], accc[8];
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    accc[p] = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[p][q] = 0.0;
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x) {
    double a[8], b[8];
#pragma unroll
    for (int p = 0; p < 8; ++p) a[p] = (p < ma) ? A.v[p][e] : 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) b[q] = (q < mb) ? B.v[q][e] : 0.0;
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      if (p < ma) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if ((!DIAG || q >= p) && q < mb) acc[p][q] = fma(a[p], b[q], acc[p][q]);
      }
    }
    if (c != nullptr) {
      const double ce = c[e];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (q < mb) accc[q] = fma(b[q], ce, accc[q]);
    }
  }
  __shared__ double red[kTS / 32][kTileSlots];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
  for (int p = 0; p < 8; ++p) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double v = warp_sum(acc[p][q]);
      if (lane == 0) red[wp][p * 8 + q] = v;
    }
    const double v = warp_sum(accc[p]);
    if (lane == 0) red[wp][64 + p] = v;
  }
  __syncthreads();
  for (int s = threadIdx.x; s < kTileSlots; s += blockDim.x) {
    double t = 0.0;
    for (int q = 0; q < kTS / 32; ++q) t += red[q][s];
    part[(size_t)blockIdx.x * kTileSlots + s] = t;
  }
}

// ---- linear combination x = sum_p coef[p] V_p -------------------------------------
__global__ void lincomb_kernel(VecSet V, const double* coef, int m, long long len, double* x) {
  __shared__ double cf[kMaxVec];
  for (int p = threadIdx.x; p < m; p += blockDim.x) cf[p] = coef[p];
  __syncthreads();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < m; ++p) s = fma(cf[p], V.v[p][e], s);
    x[e] = s;
  }
}

// ---- small dense kernels (one block) ----------------------------------------------------
// fixed-order sum over blocks of one partial slot (serial; small callers)
__device__ double sum_part(const double* part, int nblk, int slot) {
  double s = 0.0;
  for (int q = 0; q < nblk; ++q) s += part[(size_t)q * kTileSlots + slot];
  return s;
}

// out[t] = sum over blocks of partial slot slots[t], t < ns: one warp per
// slot, lanes strided over the blocks, then a fixed shuffle tree.
__device__ void sum_parts_warp(const double* part, int nblk, const int* tiles, const int* slots, int ns,
                               double* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = w; t < ns; t += nw) {
    const double* pt = part + (size_t)tiles[t] * nblk * kTileSlots;
    double s = 0.0;
    for (int q = lane; q < nblk; q += 32) s += pt[(size_t)q * kTileSlots + slots[t]];
    s = warp_sum(s);
    if (lane == 0) out[t] = s;
  }
}

// Pivoted (in order) Cholesky of the symmetric m x m matrix H (row-major in
// smem), dropping column j when its pivot v satisfies v*H_jj <= drop2*H_00
// (scaled-unit diagonal) or v <= rel_floor.  Solves H y = g on the kept
// columns; dropped entries of y are zero.  Returns the number kept.
// Executed by the whole block; H and g in shared memory are overwritten.
__device__ int chol_drop_solve(double* H, double* g, double* y, int m, double drop2, double rel_floor,
                               double* Ls, int* keep) {
  __shared__ double sc[kMaxVec];
  __shared__ int nk;
  __shared__ double piv;
  __shared__ int kj;
  const int tid = threadIdx.x;
  for (int p = tid; p < m; p += blockDim.x) sc[p] = (H[p * m + p] > 0.0) ? 1.0 / sqrt(H[p * m + p]) : 0.0;
  __syncthreads();
  for (int s = tid; s < m * m; s += blockDim.x) {
    const int p = s / m, q = s % m;
    Ls[s] = 0.0;
    H[s] *= sc[p] * sc[q];
  }
  if (tid == 0) nk = 0;
  __syncthreads();
  const double h00 = (sc[0] > 0.0) ? 1.0 / (sc[0] * sc[0]) : 0.0;
  for (int j = 0; j < m; ++j) {
    if (tid == 0) {
      double v = H[j * m + j];
      for (int t = 0; t < j; ++t) v -= Ls[j * m + t] * Ls[j * m + t];
      const double hjj = (sc[j] > 0.0) ? 1.0 / (sc[j] * sc[j]) : 0.0;
      kj = (sc[j] > 0.0 && v > rel_floor && v * hjj > drop2 * h00) ? 1 : 0;
      piv = kj ? sqrt(v) : 0.0;
      keep[j] = kj;
      if (kj) { Ls[j * m + j] = piv; ++nk; }
    }
    __syncthreads();
    if (kj) {
      for (int i = j + 1 + tid; i < m; i += blockDim.x) {
        double v = H[i * m + j];
        for (int t = 0; t < j; ++t) v -= Ls[i * m + t] * Ls[j * m + t];
        Ls[i * m + j] = v / piv;
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    // forward: L z = S g ; backward: L^T u = z ; y = S u   (dropped rows zero)
    double z[kMaxVec];
    for (int i = 0; i < m; ++i) {
      if (!keep[i]) { z[i] = 0.0; continue; }
      double v = g[i] * sc[i];
      for (int t = 0; t < i; ++t) v -= Ls[i * m + t] * z[t];
      z[i] = v / Ls[i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) {
      if (!keep[i]) { y[i] = 0.0; continue; }
      double v = z[i];
      for (int t = i + 1; t < m; ++t) v -= Ls[t * m + i] * y[t];
      y[i] = v / Ls[i * m + i];
    }
    for (int i = 0; i < m; ++i) y[i] *= sc[i];
  }
  __syncthreads();
  return nk;
}

__global__ void spe_solve_kernel(const double* part, int nblk, int m, double drop2, double* coef,
                                 SmallOut* out) {
  __shared__ double H[kMaxSpe * kMaxSpe], Ls[kMaxSpe * kMaxSpe], g[kMaxSpe], y[kMaxSpe];
  __shared__ double vals[kMaxSpe * (kMaxSpe + 1) / 2 + kMaxSpe];
  __shared__ int tiles[kMaxSpe * (kMaxSpe + 1) / 2 + kMaxSpe], slots[kMaxSpe * (kMaxSpe + 1) / 2 + kMaxSpe];
  __shared__ int keep[kMaxSpe];
  // entries (q, p), q >= p, live in tile 0 = rows/cols 0..7, tile 1 = (p < 8 <= q),
  // tile 2 = 8..15; g (D^T b) rows 0..7 in tile 0 and 8..15 in tile 2
  const int npair = m * (m + 1) / 2;
  if (threadIdx.x == 0) {
    int t = 0;
    for (int qq = 0; qq < m; ++qq)
      for (int pp = 0; pp <= qq; ++pp, ++t) {
        if (qq < 8) { tiles[t] = 0; slots[t] = pp * 8 + qq; }
        else if (pp < 8) { tiles[t] = 1; slots[t] = pp * 8 + (qq - 8); }
        else { tiles[t] = 2; slots[t] = (pp - 8) * 8 + (qq - 8); }
      }
    for (int p = 0; p < m; ++p, ++t) {
      tiles[t] = (p < 8) ? 0 : 2;
      slots[t] = 64 + (p % 8);
    }
  }
  __syncthreads();
  sum_parts_warp(part, nblk, tiles, slots, npair + m, vals);
  __syncthreads();
  for (int s = threadIdx.x; s < m * m; s += blockDim.x) {
    const int p = s / m, q = s % m;
    const int pp = p < q ? p : q, qq = p < q ? q : p;
    H[s] = vals[qq * (qq + 1) / 2 + pp];
  }
  for (int p = threadIdx.x; p < m; p += blockDim.x) g[p] = vals[npair + p];
  __syncthreads();
  const int nk = chol_drop_solve(H, g, y, m, drop2, 1e-13, Ls, keep);
  for (int p = threadIdx.x; p < m; p += blockDim.x) coef[p] = y[p];
  if (threadIdx.x == 0) { out->rank = nk; out->info = 0.0; }
}

// Gram row of a new snapshot: part tiles t = 0..ntile-1 hold (w, Lw) . X_q.
__global__ void pod_row_kernel(const double* part, int nblk, int m, int slot_new, double* G, double* A) {
  for (int q = threadIdx.x; q < m; q += blockDim.x) {
    const int tile = q / 8, qq = q % 8;
    const double* pt = part + (size_t)tile * nblk * kTileSlots;
    const double gw = sum_part(pt, nblk, 0 * 8 + qq), aw = sum_part(pt, nblk, 1 * 8 + qq);
    G[slot_new * kMaxPod + q] = gw; G[q * kMaxPod + slot_new] = gw;
    A[slot_new * kMaxPod + q] = aw; A[q * kMaxPod + slot_new] = aw;
  }
}

// POD solve: Jacobi eigen-decomposition of G (m x m), truncation, reduced
// Galerkin system, coefficients z with x0 = X z.
__global__ void pod_solve_kernel(const double* Gg, const double* Ag, const double* part, int nblk, int m,
                                 double eps_pod, double* coef, double* sigma_out, SmallOut* out) {
  __shared__ double Mt[kMaxPod * kMaxPod], V[kMaxPod * kMaxPod], Hs[kMaxPod * kMaxPod];
  double* W = Mt;   // Mt is free once the eigenvalues are read; W, then L, reuse it
  double* Ls = Mt;
  __shared__ double lam[kMaxPod], gv[kMaxPod], rhs[kMaxPod], y[kMaxPod];
  __shared__ int order[kMaxPod], keep[kMaxPod];
  __shared__ double cs[kMaxPod / 2 + 1], sn[kMaxPod / 2 + 1];
  __shared__ int pp[kMaxPod / 2 + 1], qq[kMaxPod / 2 + 1];
  __shared__ double offn, totn;
  __shared__ int kk;
  const int tid = threadIdx.x;
  const int me = (m + 1) & ~1;  // even size for the round-robin ordering (padding index is inert)
  for (int s = tid; s < me * me; s += blockDim.x) {
    const int p = s / me, q = s % me;
    Mt[s] = (p < m && q < m) ? Gg[p * kMaxPod + q] : 0.0;
    V[s] = (p == q) ? 1.0 : 0.0;
  }
  for (int p = tid; p < m; p += blockDim.x) {
    const int tile = p / 8;
    gv[p] = sum_part(part + (size_t)tile * nblk * kTileSlots, nblk, 64 + (p % 8));
  }
  __syncthreads();
  // parallel-order cyclic Jacobi: me-1 rounds of me/2 disjoint rotations per sweep
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (tid == 0) {
      double o = 0.0, t = 0.0;
      for (int p = 0; p < me; ++p)
        for (int q = 0; q < me; ++q) {
          const double v = Mt[p * me + q] * Mt[p * me + q];
          t += v;
          if (p != q) o += v;
        }
      offn = o; totn = t;
    }
    __syncthreads();
    if (!(offn > 1e-32 * totn) || me < 2) break;
    for (int round = 0; round < me - 1; ++round) {
      // pairs of the round-robin schedule: index me-1 fixed, others rotate
      for (int t = tid; t < me / 2; t += blockDim.x) {
        // circle method: index me-1 meets `round`, the others pair symmetrically
        const int a = (t == 0) ? me - 1 : (round + t) % (me - 1);
        const int b = (t == 0) ? round : (round - t + me - 1) % (me - 1);
        const int p = a < b ? a : b, q = a < b ? b : a;
        pp[t] = p; qq[t] = q;
        const double apq = Mt[p * me + q];
        double c = 1.0, s = 0.0;
        if (apq != 0.0) {
          const double theta = (Mt[q * me + q] - Mt[p * me + p]) / (2.0 * apq);
          const double tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
          c = 1.0 / sqrt(tt * tt + 1.0);
          s = tt * c;
        }
        cs[t] = c; sn[t] = s;
      }
      __syncthreads();
      // rows: M <- J^T M
      for (int w = tid; w < (me / 2) * me; w += blockDim.x) {
        const int t = w / me, col = w % me, p = pp[t], q = qq[t];
        const double c = cs[t], s = sn[t];
        const double mp = Mt[p * me + col], mq = Mt[q * me + col];
        Mt[p * me + col] = c * mp - s * mq;
        Mt[q * me + col] = s * mp + c * mq;
      }
      __syncthreads();
      // columns: M <- M J ; V <- V J
      for (int w = tid; w < (me / 2) * me; w += blockDim.x) {
        const int t = w / me, row = w % me, p = pp[t], q = qq[t];
        const double c = cs[t], s = sn[t];
        const double mp = Mt[row * me + p], mq = Mt[row * me + q];
        Mt[row * me + p] = c * mp - s * mq;
        Mt[row * me + q] = s * mp + c * mq;
        const double vp = V[row * me + p], vq = V[row * me + q];
        V[row * me + p] = c * vp - s * vq;
        V[row * me + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    for (int p = 0; p < m; ++p) { lam[p] = Mt[p * me + p]; order[p] = p; }
    for (int a = 0; a < m; ++a)            // selection sort, descending
      for (int b = a + 1; b < m; ++b)
        if (lam[order[b]] > lam[order[a]]) { const int t = order[a]; order[a] = order[b]; order[b] = t; }
    const double s1 = sqrt(fmax(lam[order[0]], 0.0));
    int k = 0;
    double sk = 0.0, sall = 0.0;
    for (int a = 0; a < m; ++a) {
      const double sa = sqrt(fmax(lam[order[a]], 0.0));
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

// ---- host launchers --------------------------------------------------------------------
static int ts_blocks() {
  static int nb = 0;
  if (nb == 0) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    nb = (nsm > 0 ? nsm : 132) * 2;
  }
  return nb;
}
int ts_nblk() { return ts_blocks(); }

static int chk() { return cudaGetLastError() == cudaSuccess ? MQS_OK : MQS_ERR_CUDA; }

int spe_push(const MutVecSet& D, const MutVecSet& LD, const double* w, const double* lw, int m_old, int m_new,
             long long len, cudaStream_t st) {
  if (m_new <= 4) diff_push_kernel<4><<<ts_blocks(), kTS, 0, st>>>(D, LD, w, lw, m_old, m_new, len);
  else if (m_new <= 8) diff_push_kernel<8><<<ts_blocks(), kTS, 0, st>>>(D, LD, w, lw, m_old, m_new, len);
  else diff_push_kernel<16><<<ts_blocks(), kTS, 0, st>>>(D, LD, w, lw, m_old, m_new, len);
  return chk();
}

int spe_x0(const VecSet& D, const VecSet& LD, int m, const double* b, double* x0, long long len, double eps_lin,
           double* part, double* coef, SmallOut* out, cudaStream_t st) {
  const int nb = ts_blocks();
  if (m <= 0) {
    if (cudaMemsetAsync(x0, 0, sizeof(double) * len, st) != cudaSuccess) return MQS_ERR_CUDA;
    return MQS_OK;
  }
  // Entry (q, p), q >= p, of the Galerkin matrix is D_q . (K D_p): the
  // high-order differences are tested against the K-images of the low-order
  // ones, which the recursion carries accurately (the images of high orders
  // accumulate its rounding relative to their small size).
  VecSet A0 = LD, B0 = D;
  dots_kernel<true><<<nb, kTS, 0, st>>>(A0, B0, b, m < 8 ? m : 8, m < 8 ? m : 8, len, part);
  if (m > 8) {
    VecSet A1, B1;
    for (int p = 0; p < 8; ++p) { A1.v[p] = LD.v[p]; B1.v[p] = D.v[8 + p < m ? 8 + p : 0]; }
    dots_kernel<false><<<nb, kTS, 0, st>>>(A1, B1, nullptr, 8, m - 8, len, part + (size_t)nb * kTileSlots);
    VecSet A2, B2;
    for (int p = 0; p < 8; ++p) { A2.v[p] = LD.v[8 + p < m ? 8 + p : 0]; B2.v[p] = D.v[8 + p < m ? 8 + p : 0]; }
    dots_kernel<true><<<nb, kTS, 0, st>>>(A2, B2, b, m - 8, m - 8, len, part + (size_t)2 * nb * kTileSlots);
  }
  spe_solve_kernel<<<1, 512, 0, st>>>(part, nb, m, eps_lin * eps_lin, coef, out);
  lincomb_kernel<<<nb, kTS, 0, st>>>(D, coef, m, len, x0);
  return chk();
}

int pod_push(const VecSet& X, const double* w, const double* lw, int m, int slot_new, long long len, double* part,
             double* G, double* A, cudaStream_t st) {
  const int nb = ts_blocks();
  const int ntile = (m + 7) / 8;
  for (int t = 0; t < ntile; ++t) {
    VecSet Aw, Bx;
    Aw.v[0] = w; Aw.v[1] = lw;
    const int mb = (m - 8 * t) < 8 ? (m - 8 * t) : 8;
    for (int q = 0; q < 8; ++q) Bx.v[q] = X.v[8 * t + (q < mb ? q : 0)];
    dots_kernel<false><<<nb, kTS, 0, st>>>(Aw, Bx, nullptr, 2, mb, len, part + (size_t)t * nb * kTileSlots);
  }
  pod_row_kernel<<<1, 64, 0, st>>>(part, nb, m, slot_new, G, A);
  return chk();
}

int pod_x0(const VecSet& X, int m, const double* G, const double* A, const double* b, double* x0, long long len,
           double eps_pod, double* part, double* coef, double* sigma, SmallOut* out, cudaStream_t st) {
  const int nb = ts_blocks();
  if (m <= 0) {
    if (x0 && cudaMemsetAsync(x0, 0, sizeof(double) * len, st) != cudaSuccess) return MQS_ERR_CUDA;
    return MQS_OK;
  }
  const int ntile = (m + 7) / 8;
  for (int t = 0; t < ntile; ++t) {
    VecSet Ax;
    const int mb = (m - 8 * t) < 8 ? (m - 8 * t) : 8;
    for (int q = 0; q < 8; ++q) Ax.v[q] = X.v[8 * t + (q < mb ? q : 0)];
    dots_kernel<false><<<nb, kTS, 0, st>>>(Ax, Ax, b, 0, mb, len, part + (size_t)t * nb * kTileSlots);
  }
  pod_solve_kernel<<<1, 256, 0, st>>>(G, A, part, nb, m, eps_pod, coef, sigma, out);
  if (x0) lincomb_kernel<<<nb, kTS, 0, st>>>(X, coef, m, len, x0);
  return chk();
}

}  // namespace mqs
