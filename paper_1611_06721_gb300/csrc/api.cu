// C ABI of the library: handle life cycle, the explicit Euler step driver and
// the stand-alone entry points declared in include/mqs.h.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <new>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <nvtx3/nvToolsExt.h>
#include "mqs_kernels.h"
#include "mrhs.h"

using namespace mqs;

namespace {
// The calling thread's tall-skinny launch cap for the duration of a scope
struct LaunchCap {
  int saved;
  explicit LaunchCap(int cap) : saved(launch_cap()) { set_launch_cap(cap); }
  ~LaunchCap() { set_launch_cap(saved); }
  LaunchCap(const LaunchCap&) = delete;
  LaunchCap& operator=(const LaunchCap&) = delete;
};
// NVTX range over the host's issue of one phase (a profiler shows the kernels each
// range launched); free when no tool is attached
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};
}  // namespace

namespace {
// what a captured step depends on besides its own launches: a replay is valid only
// while all of it is unchanged
struct GraphKey {
  cudaStream_t st, st2;
  int nblk, in_batch;
  mqs_options opt;
  double dt;
  const void *dstats, *ac, *spe0, *hpart, *fac;
};
struct StepGraph {
  cudaGraphExec_t exec = nullptr;
  GraphKey key{};
};
}  // namespace

struct mqs_handle {
  int n = 0;
  long long n3 = 0, len = 0;
  double h = 0, nu0 = 0, k1 = 0, k2 = 0, k3 = 0;
  mqs_coil coil{};
  mqs_options opt{};
  double dt = 0.0, t = 0.0;
  long m = 0;
  long n_c = 0, n_n = 0;
  int cb_lo[3], cb_hi[3], clo[3], chi[3];
  Box full{};
  int* sup = nullptr;     // right-hand side support: layout indices where b may be nonzero (sorted)
  int nsup = 0;
  bool any_brauer = false;
  cudaStream_t st = nullptr;
  int nblk = 0;
  int2* ptab = nullptr;               // part ranges of the fused pass for (ptab_nblk, ptab_groups)
  int ptab_nblk = -1, ptab_groups = -1;
  std::string err;
  std::vector<void*> allocs;
  std::vector<size_t> guard_at;   // debug builds: offset of each buffer's guard bytes
  // device buffers
  uint8_t* cflags = nullptr;
  int* cidx = nullptr;
  double *invmc = nullptr, *isqmc = nullptr;
  uint8_t* brauer = nullptr;
  double* nu = nullptr;
  double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *lx = nullptr, *b = nullptr;
  double *xu = nullptr, *bu = nullptr, *tmp = nullptr, *tmp2 = nullptr;
  double *ac_full = nullptr, *ac_full2 = nullptr, *ac = nullptr, *ac2 = nullptr, *cvec = nullptr, *cvec2 = nullptr;
  double* part = nullptr;
  unsigned* bar = nullptr;
  int* derr = nullptr;
  PcgResult* pres = nullptr;
  // halt flag and instability monitor of stepping calls; where the current call began
  StepGuard* guard = nullptr;
  double* mon_part = nullptr;
  long call_m0 = 0;
  double *call_ac0 = nullptr, *call_full0 = nullptr;
  double lambda = 0.0;       // lambda_max of eq. (CFL) found on this handle (0: none)
  double* spe_D[kMaxSpe] = {};
  double* spe_LD[kMaxSpe] = {};
  int spe_m = 0;
  double *spe_hpart = nullptr, *spe_gpart = nullptr;   // Galerkin product partials of the table, g partials
  SpeFac* spe_fac = nullptr;     // factor of the table's small system (drop rule at fac_eps)
  double fac_eps = -1.0;
  int spe_nbh = 0;               // block partials the last push wrote (the factor's layout)
  int ts_cap = 0;                // tall-skinny launch cap while in a batch (0: none)
  // side stream: the SPE table push (with its products) runs beside the conductor
  // update and the next right-hand side; the main stream joins before the table is read
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool side_pending = false;
  bool in_batch = false;     // in a batch: the instances overlap each other, no side stream
  int enqueued = 0;          // steps issued by mqs_step_enqueue and not yet finished
  // step counter on the device: [0] the time level of the last step issued, [1] the
  // statistics slot of the next one; the record kernel advances both and the right-hand
  // side reads [0], so the launches of one step do not depend on m
  long long* dctr = nullptr;
  long long ctr_m = -1, ctr_slot = -1;   // what dctr holds once the issued work ran (-1: unknown)
  // CUDA graphs of one steady-state SPE step (two: the conductor buffers alternate)
  StepGraph graphs[2];
  int graph_next = 0;        // the entry the next capture replaces
  bool graph_off = false;    // a capture failed: steps are issued launch by launch
  long graph_steps = 0;      // steps replayed from (or captured into) a graph
  // b is formed at the end of a step for the next one (beside the side stream's push);
  // it is reused only while its key still holds: the step it was formed for, the state
  // generation (bumped when a_c changes outside a step), dt and the source time level
  long b_for_m = -1, ac_gen = 0, b_ac_gen = -1;
  double b_dt = 0.0;
  int b_rhs_time = -1;
  double* pod_X[kMaxPod] = {};
  double* pod_LX[kMaxPod] = {};
  double *pod_G = nullptr, *pod_A = nullptr;
  int pod_m = 0, pod_next = 0;
  int cspe_k = 0;            // CSPE: K-orthonormal frozen columns (POD ring slots 0..k-1)
  bool cspe_live = false;    // a newest solution exists (H->x)
  bool cspe_projected = false;   // this step's start vector projected it (cspe_scal, work vectors valid)
  bool cspe_froze = false;
  double* cspe_scal = nullptr;
  long cspe_count = 0;       // solutions pushed since the history was cleared
  double *tspart = nullptr, *coef = nullptr, *sigma = nullptr, *scal = nullptr;
  SmallOut* small = nullptr;
  mqs_step_stats* dstats = nullptr;
  int dstats_cap = 0;
  bool lx_valid = false;   // lx holds L x for the step solution x
  double *r1 = nullptr, *w0 = nullptr, *w1 = nullptr, *s1 = nullptr;   // one-reduction PCG buffers
  float *r32 = nullptr, *p32 = nullptr, *q32 = nullptr, *d32 = nullptr;  // mixed precision
  float *r32b = nullptr, *w32a = nullptr, *w32b = nullptr, *s32a = nullptr, *s32b = nullptr;  // its one-reduction form
  int* refin = nullptr;
  cudaStream_t own_st = nullptr;
  // adjoint (discrete adjoint of the time loop)
  uint8_t* condbox = nullptr;              // conducting flag per cell of the cell box
  long ccells = 0;                         // cells of the cell box
  double *rec_a = nullptr, *rec_F = nullptr;   // recording targets of the next conductor update
  double* traj = nullptr;                  // [2 x steps x n_c]: a^{m-1}, then F_m
  long traj_cap = 0;
  AdjBufs adj{};
  double *adjJ = nullptr, *adj_sig = nullptr;
  double* ckpt = nullptr;                  // checkpointed adjoint: a_c at every segment start + end state
  long ckpt_cap = 0;
  // second SPE history: the adjoint solves' own, while forward segments are recomputed
  double* alt_D[kMaxSpe] = {};
  double* alt_LD[kMaxSpe] = {};
  int alt_m = 0, alt_cols = 0;
  // separate right-hand sides (rhs_split): coil-type b, conductor-type solution, zero vector
  double *bs = nullptr, *xc = nullptr, *zero_full = nullptr;
  double* alt_hpart = nullptr;
  SpeFac* alt_fac = nullptr;
  double alt_eps = -1.0;
  int alt_nbh = 0;
  // timing
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  long launches = 0, pcg_launches = 0, tsteps = 0;
  DevGeom dg{};
  CondGeom cg{};
};

namespace {

int fail(mqs_handle* H, int code, const char* msg) {
  if (H) H->err = msg;
  return code;
}

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      H->err = std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #call;      \
      return MQS_ERR_CUDA;                                                         \
    }                                                                              \
  } while (0)
#define RK(call)                                                                   \
  do {                                                                             \
    int r_ = (call);                                                               \
    if (r_ != MQS_OK) {                                                            \
      if (H->err.empty()) H->err = "kernel launch failed: " #call;                 \
      return r_;                                                                   \
    }                                                                              \
  } while (0)

// Debug builds follow every device buffer with kGuardBytes of kGuardByte (after the
// buffer's 64 bytes of slack, rounded up to kGuardBytes); mqs_debug_check compares them.
#ifdef MQS_DEBUG_CHECKS
constexpr bool kDebugBuild = true;
#else
constexpr bool kDebugBuild = false;
#endif
constexpr size_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xA5;

template <class T>
int dalloc(mqs_handle* H, T** ptr, size_t count) {
  void* v = nullptr;
  const size_t body = count * sizeof(T) + 64;
  const size_t guard = (body + kGuardBytes - 1) / kGuardBytes * kGuardBytes;
  if (cudaMalloc(&v, kDebugBuild ? guard + kGuardBytes : body) != cudaSuccess) {
    cudaGetLastError();
    H->err = "device allocation failed";
    return MQS_ERR_OOM;
  }
  if (kDebugBuild && cudaMemset(static_cast<char*>(v) + guard, kGuardByte, kGuardBytes) != cudaSuccess) {
    cudaFree(v);
    H->err = "guard bytes not written";
    return MQS_ERR_CUDA;
  }
  H->allocs.push_back(v);
  H->guard_at.push_back(kDebugBuild ? guard : 0);
  *ptr = static_cast<T*>(v);
  return MQS_OK;
}

// The fused pass's part table for the handle's block count and tile groups (a synchronous
// upload: called where those change, never inside a stream capture; pcg_launch uses the
// table only when it matches)
int ensure_ptab(mqs_handle* H) {
  // three tile groups only in the FP64 one-reduction pass; the refined paths use two
  const int g = (H->opt.tile_groups == 3 && H->opt.precision == 0) ? 3 : kGroups;
  if (H->ptab_nblk == H->nblk && H->ptab_groups == g) return MQS_OK;
  H->ptab_nblk = H->ptab_groups = -1;
  if (!H->ptab || H->nblk < 1) return MQS_OK;
  RK(fused_partition(H->n, H->nblk, g, H->ptab, H->st));
  H->ptab_nblk = H->nblk;
  H->ptab_groups = g;
  return MQS_OK;
}

// ---- small elementwise kernels -------------------------------------------------------
// y = mask_n * s * v  (layout vectors)
__global__ void mask_scale_kernel(Geom g, const double* v, double* y, double s) {
  const long long len = 3 * g.n3;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e / g.n3);
    const long long pos = e - c * g.n3;
    const int i = (int)(pos % g.n), j = (int)((pos / g.n) % g.n), k = (int)(pos / ((long long)g.n * g.n));
    y[e] = (nmask(g, i, j, k) >> c & 1u) ? s * v[e] : 0.0;
  }
}

// power method pieces over the n_c conducting unknowns (one block)
__global__ void power_prep_kernel(int n_c, const double* v, const double* isq, double* u) {
  for (int q = threadIdx.x + blockIdx.x * blockDim.x; q < n_c; q += blockDim.x * gridDim.x) u[q] = v[q] * isq[q];
}
__global__ void power_update_kernel(int n_c, const double* F, const double* isq, double* v, double* out) {
  __shared__ double red[2][32];
  double a = 0.0, zz = 0.0;
  for (int q = threadIdx.x; q < n_c; q += blockDim.x) {
    const double z = F[q] * isq[q];
    a = fma(v[q], z, a);
    zz = fma(z, z, zz);
  }
  a = warp_sum(a); zz = warp_sum(zz);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) { red[0][w] = a; red[1][w] = zz; }
  __syncthreads();
  __shared__ double nz;
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int t = 0; t < nw; ++t) { s0 += red[0][t]; s1 += red[1][t]; }
    nz = sqrt(s1);
    out[0] = s0;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < n_c; q += blockDim.x) v[q] = F[q] * isq[q] / nz;
}

// The step's statistics; a grid-barrier timeout recorded in *derr since the call
// began marks the step failed (the timed-out kernel did not write its result).  With
// the step counter ctr the record goes to dst[ctr[1]] and the counter advances one
// step; without it, to *dst.
// With the step guard gd: a step of a halted call is recorded as MQS_ERR_HALTED; a
// step whose solve succeeded takes the instability monitor's verdict; a failing step
// halts the call.
__global__ void record_kernel(const PcgResult* pr, const SmallOut* so, int use_small, const int* refin,
                              const int* derr, mqs_step_stats* dst, long long* ctr, StepGuard* gd, int cap) {
  if (ctr) {
    if (!MQS_IDX_OK(ctr[1], cap, 701)) return;
    dst += ctr[1];
    ctr[0] += 1;
    ctr[1] += 1;
  }
  mqs_step_stats s;
  if (gd && gd->halt) {
    *dst = mqs_step_stats{0, MQS_ERR_HALTED, 0, 0, 0.0, 0.0, 0.0};
    return;
  }
  s.iterations = pr->iterations;
  s.status = (*derr != 0) ? *derr : pr->status;
  if (gd) {
    if (s.status == MQS_OK) s.status = gd->status;
    if (s.status != MQS_OK) gd->halt = 1;
  }
  s.rank = use_small ? so->rank : 0;
  s.refinements = refin ? *refin : 0;
  s.relres = pr->relres;
  s.start_relres = pr->start_relres;
  s.pod_info = (use_small == 2) ? so->info : 0.0;
  *dst = s;
}

// Adds a second solve of the same step (separate right-hand sides) to its record
// (the one record_kernel wrote last: dst[ctr[1] - 1]).
__global__ void record_add_kernel(const PcgResult* pr, const SmallOut* so, int use_small, const int* refin,
                                  const int* derr, mqs_step_stats* dst, const long long* ctr, StepGuard* gd, int cap) {
  if (!MQS_IDX_OK(ctr[1] - 1, cap, 702)) return;
  dst += ctr[1] - 1;
  mqs_step_stats s = *dst;
  if (s.status == MQS_ERR_HALTED) return;
  s.iterations += pr->iterations;
  if (s.status == MQS_OK) s.status = (*derr != 0) ? *derr : pr->status;
  if (s.status != MQS_OK) gd->halt = 1;
  s.rank += use_small ? so->rank : 0;
  s.refinements += refin ? *refin : 0;
  s.relres = fmax(s.relres, pr->relres);
  s.start_relres = fmax(s.start_relres, pr->start_relres);
  *dst = s;
}

// Separate right-hand sides record their solves before the conductor update: its
// monitor verdict joins the step's record afterwards.
__global__ void record_mon_kernel(StepGuard* gd, mqs_step_stats* dst, const long long* ctr, int cap) {
  if (!MQS_IDX_OK(ctr[1] - 1, cap, 703)) return;
  dst += ctr[1] - 1;
  if (dst->status == MQS_OK && gd->status != MQS_OK) {
    dst->status = gd->status;
    gd->halt = 1;
  }
}

__global__ void set_ctr_kernel(long long* ctr, long long m, long long slot) {
  ctr[0] = m;
  ctr[1] = slot;
}

__global__ void add_kernel(double* x, const double* y, long long len) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x)
    x[e] += y[e];
}

int mask_scale(mqs_handle* H, const double* v, double* y, double s, cudaStream_t st) {
  mask_scale_kernel<<<H->nblk * 2, 256, 0, st>>>(H->dg.g, v, y, s);
  return cudaGetLastError() == cudaSuccess ? MQS_OK : MQS_ERR_CUDA;
}

int ensure_mixed(mqs_handle* H) {
  // 8 bytes per value: float-float inner vectors (precision 2); FP32 uses the first half
  if (!H->r32)
    for (float** v : {&H->r32, &H->p32, &H->q32, &H->d32}) RK(dalloc(H, v, 2 * H->len));
  if ((H->opt.pcg_variant >= 1 || H->opt.precision == 2) && !H->r32b)
    for (float** v : {&H->r32b, &H->w32a, &H->w32b, &H->s32a, &H->s32b}) RK(dalloc(H, v, 2 * H->len));
  return MQS_OK;
}

// the PCG kernel selected by opt.precision and opt.pcg_variant
int pcg_launch(mqs_handle* H, const double* b, double* x, double tol, int maxit, cudaStream_t st, int init,
               const int* halt = nullptr) {
  const Range range_("mqs pcg");
  if (H->opt.precision == 2) {
    RK(ensure_mixed(H));
    const MixedBufs mb{H->r32, H->p32, H->q32, H->d32, H->r32b, H->w32a, H->w32b, H->s32a, H->s32b};
    const double itol = H->opt.inner_tol > 0.0 ? H->opt.inner_tol : 1e-12;
    const bool tab = H->ptab_nblk == H->nblk && H->ptab_groups == kGroups;
    return launch_pcg_ff(H->dg, b, x, H->r, H->lx, mb, H->part, H->bar, H->derr, H->pres, H->refin, tol, itol,
                         maxit, H->nblk, st, init, halt, tab ? H->ptab : nullptr);
  }
  if (H->opt.precision == 1) {
    RK(ensure_mixed(H));
    const MixedBufs mb{H->r32, H->p32, H->q32, H->d32, H->r32b, H->w32a, H->w32b, H->s32a, H->s32b};
    const double itol = H->opt.inner_tol > 0.0 ? H->opt.inner_tol : 1e-5;
    const bool tab = H->ptab_nblk == H->nblk && H->ptab_groups == kGroups;
    return launch_pcg_mixed(H->dg, b, x, H->r, H->lx, mb, H->part, H->bar, H->derr, H->pres, H->refin, tol, itol,
                            maxit, H->nblk, st, init, H->opt.pcg_variant, halt, tab ? H->ptab : nullptr,
                            H->opt.halo_warps);
  }
  if (H->opt.pcg_variant >= 1) {
    const PcgExtra ex{H->r1, H->w0, H->w1, H->q, H->s1};
    const bool tab = H->ptab_nblk == H->nblk && H->ptab_groups == (H->opt.tile_groups == 3 ? 3 : kGroups);
    return launch_pcg_fused(H->dg, b, x, H->r, H->p, H->lx, ex, H->part, H->bar, H->derr, H->pres, tol, maxit,
                            H->nblk, st, init, halt, H->opt.tile_groups, tab ? H->ptab : nullptr,
                            H->opt.halo_warps);
  }
  return launch_pcg(H->dg, b, x, H->r, H->p, H->q, H->lx, H->part, H->bar, H->derr, H->pres, tol, maxit, H->nblk,
                    st, init, halt);
}

int run_pcg(mqs_handle* H, const double* b, double* x, double tol, int maxit, cudaStream_t st) {
  H->lx_valid = false;   // lx is reused as scratch
  CK(cudaMemsetAsync(H->derr, 0, sizeof(int), st));
  return pcg_launch(H, b, x, tol, maxit, st, 0);
}

int read_pcg(mqs_handle* H, mqs_pcg_info* info, cudaStream_t st) {
  PcgResult pr{};
  int derr = 0;
  CK(cudaMemcpyAsync(&pr, H->pres, sizeof(pr), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&derr, H->derr, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (info) { info->iterations = pr.iterations; info->status = pr.status; info->relres = pr.relres; info->start_relres = pr.start_relres; }
  if (derr != 0) return fail(H, derr, "a bounded grid barrier wait timed out");
  if (pr.status != MQS_OK) H->err = "PCG did not converge";
  return pr.status;
}

VecSet vs(double* const* a, int m) {
  VecSet s{};
  for (int p = 0; p < kMaxVec; ++p) s.v[p] = (p < m) ? a[p] : (m > 0 ? a[0] : nullptr);
  return s;
}
MutVecSet mvs(double* const* a, int m) {
  MutVecSet s{};
  for (int p = 0; p < kMaxVec; ++p) s.v[p] = (p < m) ? a[p] : (m > 0 ? a[0] : nullptr);
  return s;
}

// push solution w (layout, physical units) with L w into the active history
CspeBufs cspe_bufs(mqs_handle* H) {
  // frozen columns in POD ring slots 0..18, work vectors in the last two slots
  return CspeBufs{H->pod_X, H->pod_LX, H->pod_X[kMaxPod - 1], H->pod_LX[kMaxPod - 1], H->pod_X[kMaxPod - 2],
                  H->pod_LX[kMaxPod - 2], H->cspe_scal};
}
// the main stream waits for the side stream's work (no-op when none is pending)
int join_side(mqs_handle* H) {
  if (!H->side_pending) return MQS_OK;
  CK(cudaStreamWaitEvent(H->st, H->ev_join, 0));
  H->side_pending = false;
  return MQS_OK;
}

// the table's factor again when eps_lin changed since the push (the products stay valid)
int refactor_spe(mqs_handle* H, cudaStream_t st) {
  if (H->fac_eps == H->opt.eps_lin) return MQS_OK;
  RK(spe_factor(H->spe_hpart, H->spe_m, H->spe_nbh, H->opt.eps_lin, H->spe_fac, st));
  H->fac_eps = H->opt.eps_lin;
  return MQS_OK;
}

int history_push(mqs_handle* H, const double* w, const double* lw, cudaStream_t st) {
  const Range range_("mqs history push");
  const int mode = H->opt.start_mode;
  if (mode == MQS_START_SPE) {
    const int d = H->opt.spe_depth;
    const int mn = H->spe_m + 1 < d ? H->spe_m + 1 : d;
    if (st == H->st && !H->in_batch) {
      // fork: the push reads w and lw, which nothing on the main stream writes
      // before the next start vector (which joins first)
      CK(cudaEventRecord(H->ev_fork, st));
      CK(cudaStreamWaitEvent(H->st2, H->ev_fork, 0));
      RK(spe_push(mvs(H->spe_D, d), mvs(H->spe_LD, d), w, lw, H->spe_m, mn, H->len, H->spe_hpart, H->opt.eps_lin,
                  H->spe_fac, H->st2));
      CK(cudaEventRecord(H->ev_join, H->st2));
      H->side_pending = true;
    } else {
      RK(spe_push(mvs(H->spe_D, d), mvs(H->spe_LD, d), w, lw, H->spe_m, mn, H->len, H->spe_hpart, H->opt.eps_lin,
                  H->spe_fac, st));
    }
    H->spe_m = mn;
    H->spe_nbh = spe_hblocks(H->len, mn);      // under the same launch cap as the push
    H->fac_eps = H->opt.eps_lin;
  } else if (mode == MQS_START_POD) {
    const int np = H->opt.pod_snapshots;
    const int slot = H->pod_next;
    CK(cudaMemcpyAsync(H->pod_X[slot], w, sizeof(double) * H->len, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(H->pod_LX[slot], lw, sizeof(double) * H->len, cudaMemcpyDeviceToDevice, st));
    const int mn = H->pod_m + 1 < np ? H->pod_m + 1 : np;
    RK(pod_push(vs(H->pod_X, mn), H->pod_X[slot], H->pod_LX[slot], mn, slot, H->len, H->tspart, H->pod_G,
                H->pod_A, st));
    H->pod_m = mn;
    H->pod_next = (slot + 1) % np;
  } else if (mode == MQS_START_CSPE) {
    // push c (1-based): the newest solution of the previous step (projected by this step's
    // start vector) is frozen when c-1 is a multiple of the period, so the frozen columns
    // are the solutions of steps P, 2P, 3P, ...; the live column is always the newest
    // solution (H->x, L x in H->lx), so nothing is copied otherwise
    const int period = H->opt.cspe_period > 0 ? H->opt.cspe_period : 25;
    H->cspe_count += 1;
    H->cspe_froze = false;
    if (H->cspe_live && H->cspe_projected && (H->cspe_count - 1) % period == 0 &&
        H->cspe_k + 1 < H->opt.spe_depth) {
      RK(cspe_freeze(cspe_bufs(H), H->cspe_k, H->len, st));
      H->cspe_k += 1;
      H->cspe_froze = true;
    }
    H->cspe_live = true;
    H->cspe_projected = false;
  }
  (void)w; (void)lw;
  return MQS_OK;
}

// start vector into x for right-hand side b (scaled units); sets H->small.
// *init tells the PCG how to form the initial residual (see launch_pcg):
// with the images L x0 known from the history, r = b - L x0 is written here.
__global__ void sub_kernel(const double* b, const double* lx, double* r, long long len) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x)
    r[e] = b[e] - lx[e];
}

int start_vector(mqs_handle* H, const double* b, double* x, cudaStream_t st, int* used_small, int* init) {
  const Range range_("mqs start vector");
  *used_small = 0;
  *init = 0;
  RK(join_side(H));
  switch (H->opt.start_mode) {
    case MQS_START_ZERO:
      *init = 2;
      break;
    case MQS_START_PREV:
      if (H->lx_valid) {
        sub_kernel<<<H->nblk * 4, 256, 0, st>>>(b, H->lx, H->r, H->len);
        *init = 1;
      }
      break;
    case MQS_START_SPE:
      if (H->spe_m == 0) { *init = 2; break; }
      // r = b - L x0 by the PCG's own stencil pass: forming it from the recursion
      // images costs a second read of the table and, measured, more iterations
      // b vanishes off the right-hand side support, so g = D^T b is summed there
      RK(refactor_spe(H, st));
      RK(spe_x0(vs(H->spe_D, H->opt.spe_depth), H->spe_m, b, H->n, H->full, H->sup, H->nsup, x, H->len, H->spe_fac,
                H->spe_gpart, H->coef, H->small, st));
      *used_small = 1;
      *init = 0;
      break;
    case MQS_START_CSPE:
      if (!H->cspe_live) { *init = 2; break; }
      // the live column is the newest solution, which the start vector overwrites in place
      if (x != H->x) return fail(H, MQS_ERR_ARG, "CSPE start vector must be formed in the step's solution buffer");
      if (!H->lx_valid) RK(launch_apply_L(H->dg, H->x, H->lx, 1.0, H->full, st));
      RK(cspe_x0(cspe_bufs(H), H->cspe_k, H->x, H->lx, b, x, H->len, H->opt.eps_lin, H->tspart, H->coef, H->small,
                 st));
      H->cspe_projected = true;
      *used_small = 1;
      *init = 0;
      break;
    case MQS_START_POD: {
      if (H->pod_m == 0) { *init = 2; break; }
      RK(pod_x0(vs(H->pod_X, H->opt.pod_snapshots), H->pod_m, H->pod_G, H->pod_A, b, x, H->len, H->opt.eps_pod,
                H->tspart, H->coef, H->sigma, H->small, st));
      *used_small = 2;
      *init = 0;
      break;
    }
    default:
      return fail(H, MQS_ERR_ARG, "unknown start mode");
  }
  return MQS_OK;
}

// kernels launched by start_vector / history_push for the current state
long start_launches(const mqs_handle* H) {
  switch (H->opt.start_mode) {
    case MQS_START_SPE: {
      const int m = H->spe_m;  // value before this step's push: g with the substitutions, linear combination
      return m == 0 ? 0 : 2;
    }
    case MQS_START_POD:
      return H->pod_m == 0 ? 0 : (H->pod_m + 7) / 8 + 2;
    case MQS_START_PREV:
      return H->lx_valid ? 1 : 0;
    case MQS_START_CSPE: {
      if (!H->cspe_live) return 0;
      const int k = H->cspe_k;
      return (H->lx_valid ? 0 : 1) + (k + 8) / 8 + 3 + (k > 0 ? (k + 7) / 8 + 3 : 0) + (k + 8) / 8 + 3;
    }
    default:
      return 0;
  }
}
long history_launches(const mqs_handle* H) {
  switch (H->opt.start_mode) {
    case MQS_START_SPE: {    // after the push: fused push + products (or push and tiles), factor
      const int m = H->spe_m;
      return m <= 8 ? 2 : 4 + (m > 12 ? 2 : 1);
    }
    case MQS_START_POD: return (H->pod_m + 7) / 8 + 1;   // after the push
    case MQS_START_CSPE: return H->cspe_froze ? 1 : 0;
    default: return 0;
  }
}

int validate_options(const mqs_options* o, std::string& why) {
  if (!(o->tol > 0.0) || o->tol >= 1.0) { why = "tol must lie in (0, 1)"; return MQS_ERR_ARG; }
  if (o->maxit < 1) { why = "maxit must be positive"; return MQS_ERR_ARG; }
  if (o->start_mode < 0 || o->start_mode > 4) { why = "unknown start mode"; return MQS_ERR_ARG; }
  if (o->start_mode == MQS_START_CSPE) {
    if (o->spe_depth < 1 || o->spe_depth > kMaxCspe) { why = "CSPE spe_depth must be in [1, 19]"; return MQS_ERR_ARG; }
  } else if (o->spe_depth < 1 || o->spe_depth > kMaxSpe) {
    why = "spe_depth must be in [1, 16]";
    return MQS_ERR_ARG;
  }
  if (o->pod_snapshots < 1 || o->pod_snapshots > kMaxPod) { why = "pod_snapshots must be in [1, 40]"; return MQS_ERR_ARG; }
  if (!(o->eps_pod > 0.0) || !(o->eps_lin >= 0.0)) { why = "eps_pod must be positive, eps_lin non-negative"; return MQS_ERR_ARG; }
  if (o->rhs_time != 0 && o->rhs_time != 1) { why = "rhs_time must be 0 or 1"; return MQS_ERR_ARG; }
  if (o->pcg_variant < 0 || o->pcg_variant > 2) { why = "pcg_variant must be 0, 1 or 2"; return MQS_ERR_ARG; }
  if (o->tile_groups != 0 && o->tile_groups != 2 && o->tile_groups != 3) {
    why = "tile_groups must be 0, 2 or 3";
    return MQS_ERR_ARG;
  }
  if (o->halo_warps < 0 || o->halo_warps > 2 || (o->halo_warps == 2 && o->tile_groups == 3)) {
    why = "halo_warps must be 0, 1 or 2 (2 only with two tile groups)";
    return MQS_ERR_ARG;
  }
  if (o->precision < 0 || o->precision > 2) { why = "precision must be 0, 1 or 2"; return MQS_ERR_ARG; }
  if (!std::isfinite(o->inner_tol) || o->inner_tol >= 1.0) { why = "inner_tol must be < 1"; return MQS_ERR_ARG; }
  if (o->dt < 0.0 || !std::isfinite(o->dt)) { why = "dt must be >= 0"; return MQS_ERR_ARG; }
  if (o->rhs_split != 0 && o->rhs_split != 1) { why = "rhs_split must be 0 or 1"; return MQS_ERR_ARG; }
  if (!std::isfinite(o->cfl_factor) || o->cfl_factor < 0.0) { why = "cfl_factor must be >= 0"; return MQS_ERR_ARG; }
  if (o->rhs_split && o->start_mode != MQS_START_ZERO && o->start_mode != MQS_START_SPE) {
    why = "rhs_split needs the zero or the SPE start";
    return MQS_ERR_ARG;
  }
  return MQS_OK;
}

int do_setup(mqs_handle* H, const mqs_grid* grid, const mqs_materials* mat, const uint8_t* cmask,
             const mqs_coil* coil, const mqs_options* opts) {
  if (grid->nx != grid->ny || grid->nx != grid->nz)
    return fail(H, MQS_ERR_UNIMPLEMENTED, "only cubic grids (nx = ny = nz) are implemented");
  const int n = grid->nx;
  if (n < 2 || n > 800) return fail(H, MQS_ERR_ARG, "grid n must be in [2, 800]");
  if (!(grid->h > 0.0) || !std::isfinite(grid->h)) return fail(H, MQS_ERR_ARG, "grid spacing must be positive");
  if (!mat->sigma_cell) return fail(H, MQS_ERR_ARG, "sigma_cell is NULL");
  if (!(mat->nu0 > 0.0)) return fail(H, MQS_ERR_ARG, "nu0 must be positive");
  std::string why;
  if (validate_options(opts, why) != MQS_OK) return fail(H, MQS_ERR_ARG, why.c_str());
  H->n = n;
  H->n3 = (long long)n * n * n;
  H->len = 3 * H->n3;
  H->h = grid->h;
  H->nu0 = mat->nu0; H->k1 = mat->k1; H->k2 = mat->k2; H->k3 = mat->k3;
  H->coil = *coil;
  H->opt = *opts;
  H->dt = opts->dt;
  const long long n3 = H->n3;
  // conducting cells
  std::vector<double> sig(n3);
  std::vector<uint8_t> br(n3, 0);
  int lo[3] = {n, n, n}, hi[3] = {0, 0, 0};
  for (long long c = 0; c < n3; ++c) {
    const double s = mat->sigma_cell[c];
    if (!(s >= 0.0) || !std::isfinite(s)) return fail(H, MQS_ERR_ARG, "sigma must be finite and >= 0");
    bool cond = cmask ? (cmask[c] != 0) : (s > 0.0);
    if (cmask && cmask[c] && !(s > 0.0)) return fail(H, MQS_ERR_ARG, "a masked conducting cell has sigma <= 0");
    sig[c] = cond ? s : 0.0;
    if (mat->brauer_cell && mat->brauer_cell[c]) {
      if (!cond) return fail(H, MQS_ERR_ARG, "a Brauer (nonlinear) cell must conduct");
      br[c] = 1;
      H->any_brauer = true;
    }
    if (cond) {
      const int i = (int)(c % n), j = (int)((c / n) % n), k = (int)(c / ((long long)n * n));
      const int v[3] = {i, j, k};
      for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], v[a]); hi[a] = std::max(hi[a], v[a] + 1); }
    }
  }
  if (hi[0] == 0) return fail(H, MQS_ERR_ARG, "no conducting cell");
  for (int a = 0; a < 3; ++a) {
    H->clo[a] = lo[a]; H->chi[a] = hi[a];
    H->cb_lo[a] = lo[a]; H->cb_hi[a] = std::min(hi[a] + 1, n);
  }
  auto cellsig = [&](int i, int j, int k) -> double {
    if (i < 0 || j < 0 || k < 0 || i >= n || j >= n || k >= n) return 0.0;
    return sig[i + (long long)n * (j + (long long)n * k)];
  };
  // c-edges: interior edges with a conducting neighbour cell (M_kappa > 0)
  const int w0 = H->cb_hi[0] - H->cb_lo[0], w1 = H->cb_hi[1] - H->cb_lo[1], w2 = H->cb_hi[2] - H->cb_lo[2];
  std::vector<uint8_t> cf((size_t)w0 * w1 * w2, 0);
  std::vector<int> cidx;
  std::vector<double> invmc, isqmc;
  for (int c = 0; c < 3; ++c)
    for (int k = H->cb_lo[2]; k < H->cb_hi[2]; ++k)
      for (int j = H->cb_lo[1]; j < H->cb_hi[1]; ++j)
        for (int i = H->cb_lo[0]; i < H->cb_hi[0]; ++i) {
          bool interior = (c == 0) ? (j > 0 && k > 0) : (c == 1) ? (i > 0 && k > 0) : (i > 0 && j > 0);
          if (!interior) continue;
          double s = 0.0;
          for (int da = -1; da <= 0; ++da)
            for (int db = -1; db <= 0; ++db) {
              if (c == 0) s += cellsig(i, j + da, k + db);
              else if (c == 1) s += cellsig(i + da, j, k + db);
              else s += cellsig(i + da, j + db, k);
            }
          if (!(s > 0.0)) continue;
          const double mk = H->h * s * 0.25;        // M_kappa = h * mean sigma of 4 cells
          cf[(i - H->cb_lo[0]) + (size_t)w0 * ((j - H->cb_lo[1]) + (size_t)w1 * (k - H->cb_lo[2]))] |= (uint8_t)(1u << c);
          cidx.push_back((int)(c * n3 + i + (long long)n * (j + (long long)n * k)));
          invmc.push_back(1.0 / mk);
          isqmc.push_back(1.0 / std::sqrt(mk));
        }
  H->n_c = (long)cidx.size();
  H->n_n = 3L * n * (long)(n - 1) * (n - 1) - H->n_c;
  // coil on interior n-edges
  const mqs_coil& cl = *coil;
  if (cl.plane_k < 1 || cl.plane_k > n - 1 || cl.i0 < 1 || cl.j0 < 1 || cl.i1 > n - 1 || cl.j1 > n - 1 ||
      cl.i0 >= cl.i1 || cl.j0 >= cl.j1)
    return fail(H, MQS_ERR_ARG, "coil loop must lie strictly inside the grid");
  if (cl.waveform != 0 && cl.waveform != 1) return fail(H, MQS_ERR_ARG, "unknown waveform");
  if (cl.waveform == 1 && !(cl.tau > 0.0)) return fail(H, MQS_ERR_ARG, "tau must be positive");
  auto isc = [&](int c, int i, int j, int k) -> bool {
    if (i < H->cb_lo[0] || j < H->cb_lo[1] || k < H->cb_lo[2] || i >= H->cb_hi[0] || j >= H->cb_hi[1] || k >= H->cb_hi[2])
      return false;
    return (cf[(i - H->cb_lo[0]) + (size_t)w0 * ((j - H->cb_lo[1]) + (size_t)w1 * (k - H->cb_lo[2]))] >> c) & 1u;
  };
  for (int i = cl.i0; i < cl.i1; ++i)
    if (isc(0, i, cl.j0, cl.plane_k) || isc(0, i, cl.j1, cl.plane_k))
      return fail(H, MQS_ERR_ARG, "coil edges must not touch a conducting cell");
  for (int j = cl.j0; j < cl.j1; ++j)
    if (isc(1, cl.i0, j, cl.plane_k) || isc(1, cl.i1, j, cl.plane_k))
      return fail(H, MQS_ERR_ARG, "coil edges must not touch a conducting cell");
  H->full = Box{{0, 0, 0}, {n, n, n}};
  // right-hand side support: n-edges sharing a face with a c-edge (K_cn^T a_c can be
  // nonzero only there) and the coil loop's edges; b vanishes on every other edge
  std::vector<int> sup;
  {
    auto add = [&](int c, int i, int j, int k) {
      if (i < 0 || j < 0 || k < 0 || i >= n || j >= n || k >= n) return;
      const bool interior = (c == 0) ? (j > 0 && k > 0) : (c == 1) ? (i > 0 && k > 0) : (i > 0 && j > 0);
      if (interior && !isc(c, i, j, k)) sup.push_back((int)(c * n3 + i + (long long)n * (j + (long long)n * k)));
    };
    // the four edges of the face with lower corner (i, j, k) and normal d (the stencil's flux formulas)
    auto face = [&](int d, int i, int j, int k) {
      if (d == 2) { add(0, i, j, k); add(1, i + 1, j, k); add(0, i, j + 1, k); add(1, i, j, k); }
      else if (d == 0) { add(1, i, j, k); add(2, i, j + 1, k); add(1, i, j, k + 1); add(2, i, j, k); }
      else { add(2, i, j, k); add(0, i, j, k + 1); add(2, i + 1, j, k); add(0, i, j, k); }
    };
    for (const int e : cidx) {
      const int c = (int)(e / n3);
      const long long pos = e - c * n3;
      const int i = (int)(pos % n), j = (int)((pos / n) % n), k = (int)(pos / ((long long)n * n));
      if (c == 0) { face(2, i, j, k); face(2, i, j - 1, k); face(1, i, j, k); face(1, i, j, k - 1); }
      else if (c == 1) { face(2, i, j, k); face(2, i - 1, j, k); face(0, i, j, k); face(0, i, j, k - 1); }
      else { face(0, i, j, k); face(0, i, j - 1, k); face(1, i, j, k); face(1, i - 1, j, k); }
    }
    for (int i = cl.i0; i < cl.i1; ++i) { add(0, i, cl.j0, cl.plane_k); add(0, i, cl.j1, cl.plane_k); }
    for (int j = cl.j0; j < cl.j1; ++j) { add(1, cl.i1, j, cl.plane_k); add(1, cl.i0, j, cl.plane_k); }
    std::sort(sup.begin(), sup.end());
    sup.erase(std::unique(sup.begin(), sup.end()), sup.end());
  }
  // device
  CK(cudaStreamCreateWithFlags(&H->st, cudaStreamNonBlocking));
  H->own_st = H->st;
  CK(cudaStreamCreateWithFlags(&H->st2, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&H->ev_fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&H->ev_join, cudaEventDisableTiming));
  RK(pcg_max_blocks(&H->nblk));
  const size_t L = (size_t)H->len;
  const long ccells = (long)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
  RK(dalloc(H, &H->cflags, cf.size()));
  RK(dalloc(H, &H->cidx, std::max<long>(H->n_c, 1)));
  RK(dalloc(H, &H->invmc, std::max<long>(H->n_c, 1)));
  RK(dalloc(H, &H->isqmc, std::max<long>(H->n_c, 1)));
  RK(dalloc(H, &H->brauer, ccells));
  RK(dalloc(H, &H->nu, ccells));
  for (double** v : {&H->x, &H->r, &H->p, &H->q, &H->lx, &H->b, &H->xu, &H->bu, &H->tmp, &H->tmp2, &H->ac_full,
                     &H->ac_full2, &H->r1, &H->w0, &H->w1, &H->s1})
    RK(dalloc(H, v, L));
  for (double** v : {&H->ac, &H->ac2, &H->cvec, &H->cvec2}) RK(dalloc(H, v, std::max<long>(H->n_c, 1)));
  RK(dalloc(H, &H->part, (size_t)16 * H->nblk));    // 2 slots x 4 values x blocks (x2: two blocks per SM)
  RK(dalloc(H, &H->bar, 1));
  RK(dalloc(H, &H->derr, 1));
  RK(dalloc(H, &H->pres, 1));
  RK(dalloc(H, &H->guard, 1));
  RK(dalloc(H, &H->mon_part, 2 * kMonBlocks));
  RK(dalloc(H, &H->ptab, (size_t)3 * H->nblk));
  CK(cudaMemset(H->guard, 0, sizeof(StepGuard)));
  RK(dalloc(H, &H->tspart, (size_t)5 * ts_nblk() * kTileSlots));
  RK(dalloc(H, &H->spe_hpart, (size_t)4 * ts_nblk() * kTileSlots));
  RK(dalloc(H, &H->spe_gpart, (size_t)spe_gblocks() * kSpeGSlots));
  RK(dalloc(H, &H->spe_fac, 1));
  CK(cudaMemset(H->spe_fac, 0, sizeof(SpeFac)));     // arrival counters start at zero
  H->nsup = (int)sup.size();
  RK(dalloc(H, &H->sup, std::max<size_t>(sup.size(), 1)));
  if (!sup.empty()) CK(cudaMemcpy(H->sup, sup.data(), sizeof(int) * sup.size(), cudaMemcpyHostToDevice));
  RK(dalloc(H, &H->coef, kMaxVec));
  RK(dalloc(H, &H->sigma, kMaxVec));
  RK(dalloc(H, &H->scal, 4));
  RK(dalloc(H, &H->small, 1));
  RK(dalloc(H, &H->refin, 1));
  RK(dalloc(H, &H->cspe_scal, 2));
  RK(dalloc(H, &H->pod_G, kMaxPod * kMaxPod));
  RK(dalloc(H, &H->pod_A, kMaxPod * kMaxPod));
  for (int a = 0; a < kMaxSpe; ++a) { RK(dalloc(H, &H->spe_D[a], L)); RK(dalloc(H, &H->spe_LD[a], L)); }
  // POD ring allocated on first use of that mode
  std::vector<uint8_t> brbox(ccells);
  for (int k = lo[2]; k < hi[2]; ++k)
    for (int j = lo[1]; j < hi[1]; ++j)
      for (int i = lo[0]; i < hi[0]; ++i)
        brbox[(i - lo[0]) + (size_t)(hi[0] - lo[0]) * ((j - lo[1]) + (size_t)(hi[1] - lo[1]) * (k - lo[2]))] =
            br[i + (long long)n * (j + (long long)n * k)];
  CK(cudaMemcpy(H->cflags, cf.data(), cf.size(), cudaMemcpyHostToDevice));
  if (H->n_c) {
    CK(cudaMemcpy(H->cidx, cidx.data(), sizeof(int) * H->n_c, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(H->invmc, invmc.data(), sizeof(double) * H->n_c, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(H->isqmc, isqmc.data(), sizeof(double) * H->n_c, cudaMemcpyHostToDevice));
  }
  CK(cudaMemcpy(H->brauer, brbox.data(), ccells, cudaMemcpyHostToDevice));
  {
    std::vector<uint8_t> cbox(ccells);
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i)
          cbox[(i - lo[0]) + (size_t)(hi[0] - lo[0]) * ((j - lo[1]) + (size_t)(hi[1] - lo[1]) * (k - lo[2]))] =
              sig[i + (long long)n * (j + (long long)n * k)] > 0.0 ? 1 : 0;
    RK(dalloc(H, &H->condbox, ccells));
    CK(cudaMemcpy(H->condbox, cbox.data(), ccells, cudaMemcpyHostToDevice));
    H->ccells = (long)ccells;
  }
  {
    std::vector<double> nuinit(ccells, H->nu0);   // linear cells keep nu0 (cell_nu_kernel runs only with Brauer cells)
    CK(cudaMemcpy(H->nu, nuinit.data(), sizeof(double) * ccells, cudaMemcpyHostToDevice));
  }
  for (double* v : {H->x, H->r, H->p, H->q, H->lx, H->b, H->xu, H->bu, H->tmp, H->tmp2, H->ac_full, H->ac_full2})
    CK(cudaMemset(v, 0, sizeof(double) * L));
  CK(cudaMemset(H->ac, 0, sizeof(double) * std::max<long>(H->n_c, 1)));
  CK(cudaMemset(H->pod_G, 0, sizeof(double) * kMaxPod * kMaxPod));
  CK(cudaMemset(H->pod_A, 0, sizeof(double) * kMaxPod * kMaxPod));
  H->dg.g.n = n;
  H->dg.g.n3 = n3;
  for (int a = 0; a < 3; ++a) { H->dg.g.cb_lo[a] = H->cb_lo[a]; H->dg.g.cb_hi[a] = H->cb_hi[a]; }
  H->dg.g.cflags = H->cflags;
  for (int a = 0; a < 3; ++a) { H->cg.clo[a] = lo[a]; H->cg.chi[a] = hi[a]; }
  H->cg.n_c = (int)H->n_c;
  H->cg.c_idx = H->cidx;
  H->cg.inv_mc = H->invmc;
  H->cg.brauer = H->brauer;
  H->cg.nu = H->nu;
  H->cg.nu0 = H->nu0; H->cg.k1 = H->k1; H->cg.k2 = H->k2; H->cg.k3 = H->k3; H->cg.h = H->h;
  RK(ensure_ptab(H));
  CK(cudaDeviceSynchronize());
  return MQS_OK;
}

// events for the per-phase timing (pool reused across steps)
cudaEvent_t next_event(mqs_handle* H) {
  if (H->ev_used == H->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    H->ev_pool.push_back(e);
  }
  return H->ev_pool[H->ev_used++];
}
void mark(mqs_handle* H) {
  if (!H->timing) return;
  cudaEvent_t e = next_event(H);
  if (e) cudaEventRecord(e, H->st);
}

int ensure_pod(mqs_handle* H) {
  if (H->pod_X[0]) return MQS_OK;
  for (int a = 0; a < kMaxPod; ++a) {
    RK(dalloc(H, &H->pod_X[a], H->len));
    RK(dalloc(H, &H->pod_LX[a], H->len));
  }
  return MQS_OK;
}

void clear_history(mqs_handle* H) {
  if (H->opt.rhs_split) H->alt_m = 0;    // the coil type's table
  H->spe_m = 0;
  H->pod_m = 0;
  H->pod_next = 0;
  H->cspe_k = 0;
  H->cspe_live = false;
  H->cspe_projected = false;
  H->cspe_count = 0;
}

// room for nsteps records; the first `keep` records (steps enqueued and not yet
// finished) move to a grown buffer in stream order
int ensure_stats(mqs_handle* H, int nsteps, int keep = 0) {
  if (H->dstats_cap >= nsteps) return MQS_OK;
  const int cap = std::max(nsteps, std::max(2 * H->dstats_cap, 256));
  mqs_step_stats* old = H->dstats;
  RK(dalloc(H, &H->dstats, cap));
  if (keep > 0 && old)
    CK(cudaMemcpyAsync(H->dstats, old, sizeof(mqs_step_stats) * keep, cudaMemcpyDeviceToDevice, H->st));
  H->dstats_cap = cap;
  return MQS_OK;
}

// conductor update for the state currently in H->ac / H->ac_full with w = x;
// the new state goes to the other compact and layout buffers, then they swap
// device address of the guard's halt flag (no host dereference of the device pointer)
const int* halt_flag(const mqs_handle* H) {
  return reinterpret_cast<const int*>(reinterpret_cast<const char*>(H->guard) + offsetof(StepGuard, halt));
}

// The instability monitor forgets its history (the other conductor buffer no longer
// holds the state before the current one).
int reset_monitor(mqs_handle* H) {
  const size_t off = offsetof(StepGuard, count);
  CK(cudaMemsetAsync(reinterpret_cast<char*>(H->guard) + off, 0, sizeof(StepGuard) - off, H->st));
  return MQS_OK;
}

// a_c changed outside a step: b must be formed again and the monitor starts afresh
int state_changed(mqs_handle* H) {
  H->ac_gen += 1;
  return reset_monitor(H);
}

int conductor_step(mqs_handle* H, const double* w, double dt, cudaStream_t st) {
  const Range range_("mqs conductor update");
  const int window = H->opt.monitor_steps == 0 ? 8 : H->opt.monitor_steps;
  const GuardView gv{H->guard, H->mon_part, H->pres, H->derr, window};
  if (H->any_brauer) RK(launch_cell_nu(H->dg, H->cg, H->ac_full, w, false, st, halt_flag(H)));
  RK(launch_cond_update(H->dg, H->cg, H->ac_full, w, 1.0, H->ac, H->ac2, dt, st, H->ac_full2, H->rec_F, H->rec_a,
                        &gv));
  std::swap(H->ac, H->ac2);
  std::swap(H->ac_full, H->ac_full2);
  return MQS_OK;
}

// eq. (CFL): power method on M_c^-1/2 K_S(0) M_c^-1/2 from v0 (n_c values, host),
// Rayleigh quotient; every application of K_S takes one PCG solve of K_n.
int power_method(mqs_handle* H, const double* v0, double pcg_tol, double rtol, int maxit, double* lambda_max,
                 int* iters) {
  if (!(pcg_tol > 0.0) || !(rtol > 0.0) || maxit < 1) return fail(H, MQS_ERR_ARG, "bad power-method settings");
  cudaStream_t st = H->st;
  double nv = 0.0;
  for (long q = 0; q < H->n_c; ++q) nv += v0[q] * v0[q];
  if (!(nv > 0.0)) return fail(H, MQS_ERR_ARG, "v0 must be nonzero");
  std::vector<double> vn(v0, v0 + H->n_c);
  for (double& v : vn) v /= std::sqrt(nv);
  CK(cudaMemcpyAsync(H->cvec, vn.data(), sizeof(double) * H->n_c, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(H->xu, 0, sizeof(double) * H->len, st));
  CK(cudaMemsetAsync(H->tmp, 0, sizeof(double) * H->len, st));
  CK(cudaMemsetAsync(H->bu, 0, sizeof(double) * H->len, st));
  const CoilDrive nodrv{H->h / H->nu0, 0.0, 0.0, 1.0, 0.0, 0};
  const CoilGeom coil{H->coil.plane_k, H->coil.i0, H->coil.j0, H->coil.i1, H->coil.j1};
  double lam = 0.0, lam_old = 0.0;
  int it = 0;
  for (it = 1; it <= maxit; ++it) {
    // u = M_c^-1/2 v scattered to the layout; b = -(L u)|_n, so w = -K_n^+ K_cn^T u
    power_prep_kernel<<<8, 256, 0, st>>>((int)H->n_c, H->cvec, H->isqmc, H->cvec2);
    RK(launch_scatter_c(H->cg, H->cvec2, H->tmp, 1.0, H->dg.g.n3, st));
    RK(launch_rhs(H->dg, H->tmp, H->bu, nodrv, coil, H->sup, H->nsup, st));
    RK(run_pcg(H, H->bu, H->xu, pcg_tol, 100000, st));
    // K_S u = (K(0) [u; w])_c ; z = M_c^-1/2 K_S u ; lambda = v.z ; v = z/|z|
    RK(launch_cell_nu(H->dg, H->cg, H->tmp, H->xu, true, st));
    RK(launch_cond_update(H->dg, H->cg, H->tmp, H->xu, 1.0, H->cvec2, H->ac2, 0.0, st));
    power_update_kernel<<<1, 1024, 0, st>>>((int)H->n_c, H->ac2, H->isqmc, H->cvec, H->scal + 1);
    PcgResult pr{};
    CK(cudaMemcpyAsync(&lam, H->scal + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&pr, H->pres, sizeof(pr), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (pr.status != MQS_OK) return fail(H, pr.status, "PCG failed inside the power method");
    if (it > 1 && std::fabs(lam - lam_old) < rtol * std::fabs(lam)) break;
    lam_old = lam;
  }
  // the scratch a_c buffer ac2 was used (ac holds the state): the monitor's history is gone
  RK(reset_monitor(H));
  H->lambda = lam;
  *lambda_max = lam;
  if (iters) *iters = it > maxit ? maxit : it;
  return MQS_OK;
}


// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
// OOPSLA 2014): the state advances by the golden-ratio increment and each output is a
// mix of it by two xor-shift-multiply rounds.  Used for the library's own start vector
// of the power method (uniform in [-1, 1)).
uint64_t splitmix64(uint64_t& state) {
  uint64_t z = (state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// dt = cfl_factor * 2 / lambda_max (eq. (CFL)) by the power method from the library's
// own start vector, at the settings of the oracle's power method
int setup_dt(mqs_handle* H, double cfl) {
  const Range range_("mqs setup dt");
  std::vector<double> v0(H->n_c);
  uint64_t state = 1611;
  for (double& v : v0) v = 2.0 * ((double)(splitmix64(state) >> 11) * 0x1.0p-53) - 1.0;
  double lam = 0.0;
  int it = 0;
  RK(power_method(H, v0.data(), 1e-12, 1e-8, 2000, &lam, &it));
  if (!(lam > 0.0) || !std::isfinite(lam)) return fail(H, MQS_ERR_NAN, "the power method gave no positive lambda_max");
  H->dt = cfl * 2.0 / lam;
  CK(cudaStreamSynchronize(H->st));
  return MQS_OK;
}

}  // namespace

// =====================================================================================
extern "C" {

int mqs_setup(const mqs_grid* grid, const mqs_materials* mat, const uint8_t* conductor_mask, const mqs_coil* coil,
              const mqs_options* opts, mqs_handle** out) {
  const Range range_("mqs_setup");
  if (!out) return MQS_ERR_ARG;
  *out = nullptr;
  if (!grid || !mat || !coil || !opts) return MQS_ERR_ARG;
  mqs_handle* H = new (std::nothrow) mqs_handle();
  if (!H) return MQS_ERR_OOM;
  int rc = do_setup(H, grid, mat, conductor_mask, coil, opts);
  if (rc == MQS_OK && !(opts->dt > 0.0) && opts->cfl_factor > 0.0) rc = setup_dt(H, opts->cfl_factor);
  if (rc != MQS_OK) {
    fprintf(stderr, "mqs_setup: %s\n", H->err.c_str());
    mqs_destroy(H);
    return rc;
  }
  *out = H;
  return MQS_OK;
}

int mqs_destroy(mqs_handle* H) {
  if (!H) return MQS_OK;
  if (H->st) cudaStreamSynchronize(H->st);
  if (H->st2) cudaStreamSynchronize(H->st2);
  for (void* v : H->allocs) cudaFree(v);
  for (cudaEvent_t e : H->ev_pool) cudaEventDestroy(e);
  if (H->own_st) cudaStreamDestroy(H->own_st);
  if (H->st2) cudaStreamDestroy(H->st2);
  if (H->ev_fork) cudaEventDestroy(H->ev_fork);
  if (H->ev_join) cudaEventDestroy(H->ev_join);
  for (StepGraph& g : H->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  delete H;
  return MQS_OK;
}

int mqs_last_error(const mqs_handle* H, char* buf, size_t len) {
  if (!H || !buf || len == 0) return MQS_ERR_ARG;
  snprintf(buf, len, "%s", H->err.c_str());
  return MQS_OK;
}

int mqs_layout(const mqs_handle* H, mqs_layout_info* info) {
  if (!H || !info) return MQS_ERR_ARG;
  info->n = H->n;
  info->n_layout = (long)H->len;
  info->n_c = H->n_c;
  info->n_n = H->n_n;
  for (int a = 0; a < 3; ++a) { info->box_lo[a] = H->cb_lo[a]; info->box_hi[a] = H->cb_hi[a]; }
  return MQS_OK;
}

int mqs_set_dt(mqs_handle* H, double dt) {
  if (!H) return MQS_ERR_ARG;
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(H, MQS_ERR_ARG, "dt must be positive");
  H->dt = dt;
  return MQS_OK;
}

int mqs_get_dt(const mqs_handle* H, double* dt, double* lambda_max) {
  if (!H) return MQS_ERR_ARG;
  if (dt) *dt = H->dt;
  if (lambda_max) *lambda_max = H->lambda;
  return MQS_OK;
}

int mqs_set_options(mqs_handle* H, const mqs_options* o) {
  if (!H || !o) return MQS_ERR_ARG;
  std::string why;
  if (validate_options(o, why) != MQS_OK) return fail(H, MQS_ERR_ARG, why.c_str());
  const bool reset = o->start_mode != H->opt.start_mode || o->spe_depth != H->opt.spe_depth ||
                     o->pod_snapshots != H->opt.pod_snapshots || o->cspe_period != H->opt.cspe_period ||
                     o->rhs_split != H->opt.rhs_split;
  const double dt = H->dt;
  H->opt = *o;
  H->dt = (o->dt > 0.0) ? o->dt : dt;
  if (reset) clear_history(H);
  return ensure_ptab(H);
}

int mqs_get_options(const mqs_handle* H, mqs_options* o) {
  if (!H || !o) return MQS_ERR_ARG;
  *o = H->opt;
  o->dt = H->dt;
  return MQS_OK;
}

int mqs_reset_history(mqs_handle* H) {
  if (!H) return MQS_ERR_ARG;
  clear_history(H);
  return MQS_OK;
}

namespace {

// swap the active SPE history with the second one (pointers only; the side stream joins
// first, so no pending push writes a table after it changed role)
int swap_spe(mqs_handle* H) {
  RK(join_side(H));
  for (int a = 0; a < kMaxSpe; ++a) { std::swap(H->spe_D[a], H->alt_D[a]); std::swap(H->spe_LD[a], H->alt_LD[a]); }
  std::swap(H->spe_m, H->alt_m);
  std::swap(H->spe_hpart, H->alt_hpart);
  std::swap(H->spe_fac, H->alt_fac);
  std::swap(H->fac_eps, H->alt_eps);
  std::swap(H->spe_nbh, H->alt_nbh);
  return MQS_OK;
}

int ensure_spe_alt(mqs_handle* H) {
  const int d = H->opt.spe_depth;
  if (!H->alt_hpart) {
    RK(dalloc(H, &H->alt_hpart, (size_t)4 * ts_nblk() * kTileSlots));
    RK(dalloc(H, &H->alt_fac, 1));
    CK(cudaMemsetAsync(H->alt_fac, 0, sizeof(SpeFac), H->st));
  }
  for (int a = H->alt_cols; a < d; ++a) { RK(dalloc(H, &H->alt_D[a], H->len)); RK(dalloc(H, &H->alt_LD[a], H->len)); }
  H->alt_cols = std::max(H->alt_cols, d);
  return MQS_OK;
}

bool rhs_ready(const mqs_handle* H, long m) {
  return H->b_for_m == m && H->b_ac_gen == H->ac_gen && H->b_dt == H->dt && H->b_rhs_time == H->opt.rhs_time;
}

// the host's copy of the device step counter follows a record_kernel launch
void advance_ctr(mqs_handle* H) {
  if (H->ctr_m >= 0) H->ctr_m += 1;
  if (H->ctr_slot >= 0) H->ctr_slot += 1;
}

// the source of the step after the last one issued, at t_m (rhs_time 0) or t_{m-1},
// with m taken from the device step counter
CoilDrive step_drive(const mqs_handle* H, double amplitude) {
  CoilDrive d{H->h / H->nu0, amplitude, H->coil.freq_hz, H->coil.tau, 0.0, H->coil.waveform};
  d.m_dev = H->dctr;
  d.level = H->opt.rhs_time == 0 ? 1 : 0;
  d.dt = H->dt;
  return d;
}

// b of eq. (mrhs) for step m = (last step issued) + 1 (scaled by h / nu0) from the
// current conductor state
int form_rhs(mqs_handle* H, long m, cudaStream_t st) {
  const CoilGeom coil{H->coil.plane_k, H->coil.i0, H->coil.j0, H->coil.i1, H->coil.j1};
  RK(launch_rhs(H->dg, H->ac_full, H->b, step_drive(H, H->coil.amplitude), coil, H->sup, H->nsup, st));
  H->b_for_m = m;
  H->b_ac_gen = H->ac_gen;
  H->b_dt = H->dt;
  H->b_rhs_time = H->opt.rhs_time;
  return MQS_OK;
}

// One step with the separate right-hand sides listed after eq. (mrhs): K_n w_c =
// -(h/nu0) K_cn^T a_c^{m-1} and K_n w_s = (h/nu0) i(t) X_s, each started from the
// SPE projection on past solutions of its own type (the handle's table holds the
// conductor type, the second table the coil type), then w = w_c + w_s and the conductor
// update.  Phase marks: rhs (both), start (conductor type), PCG (conductor type, then
// the coil type's start vector and solve), history, conductor.
int enqueue_split_step(mqs_handle* H) {
  const Range range_("mqs step");
  const LaunchCap cap_(H->ts_cap);
  cudaStream_t st = H->st;
  const CoilGeom coil{H->coil.plane_k, H->coil.i0, H->coil.j0, H->coil.i1, H->coil.j1};
  const long m = H->m + 1;
  const int refin = H->opt.precision != 0;
  mark(H);
  const CoilDrive none = step_drive(H, 0.0);
  const CoilDrive drv = step_drive(H, H->coil.amplitude);
  RK(launch_rhs(H->dg, H->ac_full, H->b, none, coil, H->sup, H->nsup, st));     // conductor type
  H->b_for_m = -1;
  RK(launch_rhs(H->dg, H->zero_full, H->bs, drv, coil, H->sup, H->nsup, st));   // coil type
  mark(H);
  int used_c = 0, init_c = 0, used_s = 0, init_s = 0;
  const long nl_start = start_launches(H);
  RK(start_vector(H, H->b, H->x, st, &used_c, &init_c));
  mark(H);
  RK(pcg_launch(H, H->b, H->x, H->opt.tol, H->opt.maxit, st, init_c, halt_flag(H)));
  record_kernel<<<1, 1, 0, st>>>(H->pres, H->small, used_c, refin ? H->refin : nullptr, H->derr, H->dstats,
                                 H->dctr, H->guard, H->dstats_cap);
  advance_ctr(H);
  RK(history_push(H, H->x, H->lx, st));
  CK(cudaMemcpyAsync(H->xc, H->x, sizeof(double) * H->len, cudaMemcpyDeviceToDevice, st));
  RK(swap_spe(H));                                    // the coil type's table (joins the push)
  const long nl_start_s = start_launches(H);
  RK(start_vector(H, H->bs, H->x, st, &used_s, &init_s));
  RK(pcg_launch(H, H->bs, H->x, H->opt.tol, H->opt.maxit, st, init_s, halt_flag(H)));
  record_add_kernel<<<1, 1, 0, st>>>(H->pres, H->small, used_s, refin ? H->refin : nullptr, H->derr,
                                     H->dstats, H->dctr, H->guard, H->dstats_cap);
  mark(H);
  RK(history_push(H, H->x, H->lx, st));
  const long nl_hist = 2 * history_launches(H);
  RK(swap_spe(H));                                    // back to the conductor type (joins the push)
  add_kernel<<<H->nblk * 2, 256, 0, st>>>(H->x, H->xc, H->len);   // w = w_s + w_c
  H->lx_valid = false;                                // lx holds L w_s only
  mark(H);
  RK(conductor_step(H, H->x, H->dt, st));
  record_mon_kernel<<<1, 1, 0, st>>>(H->guard, H->dstats, H->dctr, H->dstats_cap);
  mark(H);
  if (H->timing) {
    H->launches += 2 + nl_start + nl_start_s + 2 + 2 + nl_hist + 1 + (H->any_brauer ? 2 : 1) + 1;
    H->pcg_launches += 2;
    H->tsteps += 1;
  }
  H->m = m;
  H->t = m * H->dt;
  return MQS_OK;
}

// Issues the launches of one explicit-Euler step of H on H->st (no host wait); the
// step's statistics go to the slot the device step counter names.
int enqueue_step(mqs_handle* H) {
  const Range range_("mqs step");
  const LaunchCap cap_(H->ts_cap);
  if (H->opt.rhs_split) return enqueue_split_step(H);
  cudaStream_t st = H->st;
  const long m = H->m + 1;
  long nl = 0;
  mark(H);
  // (a2) right-hand side of eq. (mrhs), scaled by h / nu0 (usually formed by the
  // previous step already)
  if (!rhs_ready(H, m)) {
    RK(form_rhs(H, m, st));
    nl += 1;
  }
  mark(H);
  // (a3) start vector
  int used_small = 0, init = 0;
  nl += start_launches(H);
  RK(start_vector(H, H->b, H->x, st, &used_small, &init));
  mark(H);
  // (a4) PCG (the error word was cleared when the call began: a timeout stays visible)
  RK(pcg_launch(H, H->b, H->x, H->opt.tol, H->opt.maxit, st, init, halt_flag(H)));
  H->lx_valid = true;
  nl += 1;
  mark(H);
  // (a6) history first: the SPE push forks to the side stream here and runs beside
  // the conductor update (both only read w and L w)
  RK(history_push(H, H->x, H->lx, st));
  nl += history_launches(H);
  mark(H);
  // (a5) conducting update, eq. (acm)
  RK(conductor_step(H, H->x, H->dt, st));
  nl += H->any_brauer ? 2 : 1;
  record_kernel<<<1, 1, 0, st>>>(H->pres, H->small, used_small, H->opt.precision != 0 ? H->refin : nullptr,
                                 H->derr, H->dstats, H->dctr, H->guard, H->dstats_cap);
  advance_ctr(H);
  nl += 1;
  // the next step's right-hand side from the new state, beside the side stream's push
  H->m = m;
  RK(form_rhs(H, m + 1, st));
  nl += 1;
  mark(H);
  if (H->timing) { H->launches += nl; H->pcg_launches += 1; H->tsteps += 1; }
  H->m = m;
  H->t = m * H->dt;
  return MQS_OK;
}

// ---- CUDA graphs of the steady-state SPE step ----------------------------------------
// Once the SPE table is full (and b was formed by the step before), a step issues the
// same launches with the same arguments every time, except that the conductor buffers
// alternate: one graph per buffer parity replays them.  The host-side effect of such a
// step is fixed (after_step), so a replay updates the host state without issuing it.

GraphKey graph_key(const mqs_handle* H) {
  GraphKey k;
  memset(&k, 0, sizeof k);
  k.st = H->st;
  k.st2 = H->st2;
  k.nblk = H->nblk;
  k.in_batch = H->in_batch ? 1 : 0;
  memcpy(&k.opt, &H->opt, sizeof k.opt);
  k.dt = H->dt;
  k.dstats = H->dstats;
  k.ac = H->ac;
  k.spe0 = H->spe_D[0];
  k.hpart = H->spe_hpart;
  k.fac = H->spe_fac;
  return k;
}

bool graph_eligible(const mqs_handle* H) {
  return H->opt.graph && !H->graph_off && !H->timing && !H->opt.rhs_split && H->opt.start_mode == MQS_START_SPE &&
         H->spe_m == H->opt.spe_depth && H->fac_eps == H->opt.eps_lin && !H->rec_F && !H->rec_a &&
         rhs_ready(H, H->m + 1);
}

// the host fields a step changes
struct StepHost {
  long long ctr_m, ctr_slot;
  long m, b_for_m, b_ac_gen;
  double t, b_dt, fac_eps;
  int b_rhs_time, spe_m;
  bool lx_valid, side_pending;
  double *ac, *ac2, *ac_full, *ac_full2;
};
StepHost save_host(const mqs_handle* H) {
  return StepHost{H->ctr_m, H->ctr_slot,   H->m,     H->b_for_m, H->b_ac_gen, H->t,   H->b_dt,
                  H->fac_eps, H->b_rhs_time, H->spe_m, H->lx_valid, H->side_pending, H->ac, H->ac2, H->ac_full,
                  H->ac_full2};
}
void load_host(mqs_handle* H, const StepHost& s) {
  H->ctr_m = s.ctr_m; H->ctr_slot = s.ctr_slot;
  H->m = s.m; H->b_for_m = s.b_for_m; H->b_ac_gen = s.b_ac_gen; H->t = s.t; H->b_dt = s.b_dt;
  H->fac_eps = s.fac_eps; H->b_rhs_time = s.b_rhs_time; H->spe_m = s.spe_m; H->lx_valid = s.lx_valid;
  H->side_pending = s.side_pending; H->ac = s.ac; H->ac2 = s.ac2; H->ac_full = s.ac_full;
  H->ac_full2 = s.ac_full2;
}
bool same_host(const StepHost& a, const StepHost& b) {
  return a.ctr_m == b.ctr_m && a.ctr_slot == b.ctr_slot && a.m == b.m && a.b_for_m == b.b_for_m && a.b_ac_gen == b.b_ac_gen && a.t == b.t && a.b_dt == b.b_dt &&
         a.fac_eps == b.fac_eps && a.b_rhs_time == b.b_rhs_time && a.spe_m == b.spe_m &&
         a.lx_valid == b.lx_valid && a.side_pending == b.side_pending && a.ac == b.ac && a.ac2 == b.ac2 &&
         a.ac_full == b.ac_full && a.ac_full2 == b.ac_full2;
}
// what a steady-state SPE step (its side stream joined) leaves on the host
StepHost after_step(const mqs_handle* H, const StepHost& s) {
  StepHost r = s;
  if (r.ctr_m >= 0) r.ctr_m += 1;
  if (r.ctr_slot >= 0) r.ctr_slot += 1;
  r.m = s.m + 1;
  r.t = r.m * H->dt;
  r.b_for_m = r.m + 1;
  r.b_ac_gen = H->ac_gen;
  r.b_dt = H->dt;
  r.b_rhs_time = H->opt.rhs_time;
  r.fac_eps = H->opt.eps_lin;
  r.lx_valid = true;
  r.side_pending = false;
  std::swap(r.ac, r.ac2);
  std::swap(r.ac_full, r.ac_full2);
  return r;
}

void drop_graph(StepGraph& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g.exec = nullptr;
}

// Captures the launches `issue` makes on `origin` into an executable graph; false (and
// nothing left captured) when the capture or the instantiation fails.
extern "C++" template <class F>
bool capture(cudaStream_t origin, F issue, cudaGraphExec_t* exec) {
  *exec = nullptr;
  if (cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const bool issued = issue();
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(origin, &graph);
  bool ok = issued && ec == cudaSuccess && graph && cudaGraphInstantiate(exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  if (!ok) {
    if (*exec) cudaGraphExecDestroy(*exec);
    *exec = nullptr;
    cudaGetLastError();
  }
  return ok;
}

// One step of H from a graph when the step is eligible: replayed when a graph with this
// step's key exists, else captured (launch by launch as enqueue_step issues them, the
// side stream joined at the end) and launched.  *done is false when the step is to be
// issued without a graph (not eligible, or the capture failed: graphs then stay off).
int graph_step(mqs_handle* H, bool* done) {
  const Range range_("mqs step graph");
  *done = false;
  if (!graph_eligible(H)) return MQS_OK;
  RK(join_side(H));
  const GraphKey k = graph_key(H);
  const StepHost s0 = save_host(H);
  for (StepGraph& g : H->graphs)
    if (g.exec && memcmp(&g.key, &k, sizeof k) == 0) {
      CK(cudaGraphLaunch(g.exec, H->st));
      load_host(H, after_step(H, s0));
      H->graph_steps += 1;
      *done = true;
      return MQS_OK;
    }
  StepGraph& g = H->graphs[H->graph_next];
  H->graph_next ^= 1;
  drop_graph(g);
  cudaGraphExec_t exec = nullptr;
  const bool ok = capture(
      H->st,
      [&] {
        const bool issued = enqueue_step(H) == MQS_OK;
        const bool joined = join_side(H) == MQS_OK;     // also after a failure: no fork left open
        return issued && joined && same_host(save_host(H), after_step(H, s0));
      },
      &exec);
  if (!ok) {
    load_host(H, s0);
    H->graph_off = true;
    H->err.clear();
    return MQS_OK;
  }
  g.exec = exec;
  g.key = k;
  CK(cudaGraphLaunch(exec, H->st));
  H->graph_steps += 1;
  *done = true;
  return MQS_OK;
}

void dfree(mqs_handle* H, void* p) {
  for (size_t i = 0; i < H->allocs.size(); ++i)
    if (H->allocs[i] == p) {
      cudaFree(p);
      H->allocs.erase(H->allocs.begin() + (long)i);
      H->guard_at.erase(H->guard_at.begin() + (long)i);
      return;
    }
}

// trajectory storage for nsteps steps and the adjoint work buffers (first use)
int ensure_adjoint(mqs_handle* H, int nsteps) {
  if (H->traj_cap < nsteps) {
    if (H->traj) { CK(cudaStreamSynchronize(H->st)); dfree(H, H->traj); H->traj = nullptr; H->traj_cap = 0; }
    RK(dalloc(H, &H->traj, (size_t)2 * nsteps * H->n_c));
    H->traj_cap = nsteps;
  }
  if (H->adj.lam) return MQS_OK;
  const size_t L = (size_t)H->len;
  const int ex = H->cg.chi[0] - H->cg.clo[0] + 1, ey = H->cg.chi[1] - H->cg.clo[1] + 1,
            ez = H->cg.chi[2] - H->cg.clo[2] + 1;
  const size_t nq = (size_t)3 * ex * ey * ez;
  RK(dalloc(H, &H->adj.lam, H->n_c));
  RK(dalloc(H, &H->adj.gmc, H->n_c));
  RK(dalloc(H, &H->adj.mu_full, L));
  RK(dalloc(H, &H->adj.ap_full, L));
  RK(dalloc(H, &H->adj.tS, (size_t)3 * H->ccells));
  RK(dalloc(H, &H->adj.gI, 1));
  RK(dalloc(H, &H->adj.part, 1024));
  RK(dalloc(H, &H->adj.qmap, nq));
  RK(dalloc(H, &H->adjJ, 1));
  RK(dalloc(H, &H->adj_sig, H->ccells));
  CK(cudaMemsetAsync(H->adj.mu_full, 0, sizeof(double) * L, H->st));
  CK(cudaMemsetAsync(H->adj.ap_full, 0, sizeof(double) * L, H->st));
  CK(cudaMemsetAsync(H->adj.qmap, 0xff, sizeof(int) * nq, H->st));     // -1: not a c-edge
  RK(launch_adj_qmap(H->dg, H->cg, H->adj, H->st));
  return MQS_OK;
}

// buffers of the separate right-hand sides (rhs_split) and the coil type's table
int ensure_split(mqs_handle* H) {
  if (!H->bs) {
    for (double** v : {&H->bs, &H->xc, &H->zero_full}) RK(dalloc(H, v, H->len));
    for (double* v : {H->bs, H->zero_full}) CK(cudaMemsetAsync(v, 0, sizeof(double) * H->len, H->st));
  }
  return ensure_spe_alt(H);
}

// the device step counter at (H->m, slot); unless forced, launched only when it would hold
// other values once the issued work ran (steps enqueued behind each other need none)
int set_ctr(mqs_handle* H, long long slot, bool force) {
  if (!force && H->ctr_m == H->m && H->ctr_slot == slot) return MQS_OK;
  set_ctr_kernel<<<1, 1, 0, H->st>>>(H->dctr, H->m, slot);
  CK(cudaGetLastError());
  H->ctr_m = H->m;
  H->ctr_slot = slot;
  return MQS_OK;
}

// Before the steps of a call: buffers, and (unless steps are already queued) a cleared
// device error word, so a barrier timeout of any step of the call stays recorded.
int prepare_steps(mqs_handle* H, int nsteps, int keep = 0) {
  if (!(H->dt > 0.0)) return fail(H, MQS_ERR_ARG, "dt is not set");
  if (H->opt.start_mode == MQS_START_POD || H->opt.start_mode == MQS_START_CSPE) RK(ensure_pod(H));
  if (H->opt.rhs_split) RK(ensure_split(H));
  if (H->opt.precision != 0) RK(ensure_mixed(H));
  if (!H->dctr) RK(dalloc(H, &H->dctr, 2));
  if (keep == 0) {
    CK(cudaMemsetAsync(H->derr, 0, sizeof(int), H->st));
    CK(cudaMemsetAsync(const_cast<int*>(halt_flag(H)), 0, sizeof(int), H->st));   // a new call runs
    H->call_m0 = H->m;
    H->call_ac0 = H->ac;
    H->call_full0 = H->ac_full;
  }
  RK(ensure_stats(H, nsteps, keep));
  return set_ctr(H, keep, keep == 0);
}

// After the first failing step of a call (index f among its steps, which the device
// halted after it): the handle goes back to the state after the call's first f steps.
// The conductor buffer pair alternates once per issued step, and the failing step and
// the halted ones wrote nothing but the failing step's discarded update into the
// other buffer, so the state after f steps is the buffer of parity f.  Its start-vector
// history and b are dropped (halted steps pushed start vectors, not solutions).
int roll_back(mqs_handle* H, int f) {
  double* a0 = H->call_ac0;
  double* a1 = (H->ac == a0) ? H->ac2 : H->ac;
  double* f0 = H->call_full0;
  double* f1 = (H->ac_full == f0) ? H->ac_full2 : H->ac_full;
  H->ac = (f % 2 == 0) ? a0 : a1;
  H->ac2 = (f % 2 == 0) ? a1 : a0;
  H->ac_full = (f % 2 == 0) ? f0 : f1;
  H->ac_full2 = (f % 2 == 0) ? f1 : f0;
  H->m = H->call_m0 + f;
  H->t = H->m * H->dt;
  H->ctr_m = H->ctr_slot = -1;       // the device counter ran on through the halted steps
  H->b_for_m = -1;
  H->lx_valid = false;
  clear_history(H);
  return state_changed(H);
}

// The statistics of a finished stepping call: OK, or the first failing step's status
// with the handle rolled back to the step before it.
int finish_call(mqs_handle* H, int nsteps, const mqs_step_stats* hs, int derr) {
  for (int s = 0; s < nsteps; ++s)
    if (hs[s].status != MQS_OK) {
      const int code = hs[s].status;
      RK(roll_back(H, s));
      char buf[160];
      snprintf(buf, sizeof buf, "step %d of the call failed (status %d); the handle is at the step before it",
               s + 1, code);
      H->err = buf;
      return code;
    }
  if (derr != 0) return fail(H, derr, "a bounded grid barrier wait timed out");
  return MQS_OK;
}

// Copies the step statistics of the last nsteps steps into hs (async on H->st).
int fetch_stats(mqs_handle* H, int nsteps, mqs_step_stats* hs, int* derr) {
  RK(join_side(H));
  CK(cudaMemcpyAsync(hs, H->dstats, sizeof(mqs_step_stats) * nsteps, cudaMemcpyDeviceToHost, H->st));
  CK(cudaMemcpyAsync(derr, H->derr, sizeof(int), cudaMemcpyDeviceToHost, H->st));
  return MQS_OK;
}

int check_stats(mqs_handle* H, int nsteps, const mqs_step_stats* hs, int derr) {
  if (derr != 0) return fail(H, derr, "a bounded grid barrier wait timed out");
  for (int s = 0; s < nsteps; ++s)
    if (hs[s].status != MQS_OK) {
      H->err = "PCG failed in a time step";
      return hs[s].status;
    }
  return MQS_OK;
}

}  // namespace

int mqs_step(mqs_handle* H, int nsteps, mqs_step_stats* per_step) {
  const Range range_("mqs_step");
  if (!H || nsteps < 0) return MQS_ERR_ARG;
  if (H->enqueued) return fail(H, MQS_ERR_ARG, "steps are enqueued: call mqs_step_finish first");
  if (nsteps == 0) return (H->dt > 0.0) ? MQS_OK : fail(H, MQS_ERR_ARG, "dt is not set");
  RK(mqs_step_enqueue(H, nsteps));
  return mqs_step_finish(H, nsteps, per_step);
}

int mqs_step_enqueue(mqs_handle* H, int nsteps) {
  const Range range_("mqs_step_enqueue");
  if (!H || nsteps < 1) return MQS_ERR_ARG;
  if (!(H->dt > 0.0)) return fail(H, MQS_ERR_ARG, "dt is not set");
  if (nsteps > (1 << 30) - H->enqueued) return fail(H, MQS_ERR_ARG, "too many steps enqueued");
  const int base = H->enqueued;
  int rc = prepare_steps(H, base + nsteps, base);
  for (int s = 0; s < nsteps && rc == MQS_OK; ++s) {
    bool done = false;
    rc = graph_step(H, &done);
    if (rc == MQS_OK && !done) rc = enqueue_step(H);
  }
  const int rj = join_side(H);          // also after a failed launch: nothing left running beside
  if (rc != MQS_OK) { H->enqueued = 0; return rc; }
  if (rj != MQS_OK) { H->enqueued = 0; return rj; }
  H->enqueued = base + nsteps;
  return MQS_OK;
}

int mqs_step_finish(mqs_handle* H, int nsteps, mqs_step_stats* per_step) {
  if (!H || nsteps < 1 || nsteps != H->enqueued) return MQS_ERR_ARG;
  H->enqueued = 0;
  std::vector<mqs_step_stats> hs(nsteps);
  int derr = 0;
  RK(fetch_stats(H, nsteps, hs.data(), &derr));
  CK(cudaStreamSynchronize(H->st));
  if (per_step) memcpy(per_step, hs.data(), sizeof(mqs_step_stats) * nsteps);
  return finish_call(H, nsteps, hs.data(), derr);
}

namespace {

// forward steps recording a^{m-1} and F_m of every step, then J on the device
int adjoint_forward(mqs_handle* H, int nsteps, int stats_steps) {
  if (!H || nsteps < 1) return MQS_ERR_ARG;
  if (H->n_c < 1) return fail(H, MQS_ERR_ARG, "no conducting edges");
  RK(prepare_steps(H, stats_steps));
  RK(ensure_adjoint(H, nsteps));
  const long nc = H->n_c;
  double* trajA = H->traj;
  double* trajF = H->traj + (size_t)nsteps * nc;
  for (int s = 0; s < nsteps; ++s) {
    H->rec_a = trajA + (size_t)s * nc;
    H->rec_F = trajF + (size_t)s * nc;
    const int rc = enqueue_step(H);
    if (rc != MQS_OK) { H->rec_a = H->rec_F = nullptr; return rc; }
  }
  H->rec_a = H->rec_F = nullptr;
  CK(cudaMemsetAsync(H->adjJ, 0, sizeof(double), H->st));
  return launch_adj_objective(H->cg, trajF, nsteps, H->dt, H->adj, H->adjJ, H->st);
}

}  // namespace

int mqs_loss(mqs_handle* H, int nsteps, double* objective) {
  if (!H) return MQS_ERR_ARG;
  RK(adjoint_forward(H, nsteps, nsteps));
  std::vector<mqs_step_stats> hs(nsteps);
  int derr = 0;
  double J = 0.0;
  RK(fetch_stats(H, nsteps, hs.data(), &derr));
  CK(cudaMemcpyAsync(&J, H->adjJ, sizeof(double), cudaMemcpyDeviceToHost, H->st));
  CK(cudaStreamSynchronize(H->st));
  RK(check_stats(H, nsteps, hs.data(), derr));
  if (objective) *objective = J;
  return MQS_OK;
}

namespace {

int ensure_ckpt(mqs_handle* H, long count) {
  if (H->ckpt_cap >= count) return MQS_OK;
  if (H->ckpt) { CK(cudaStreamSynchronize(H->st)); dfree(H, H->ckpt); H->ckpt = nullptr; H->ckpt_cap = 0; }
  RK(dalloc(H, &H->ckpt, (size_t)count * H->n_c));
  H->ckpt_cap = count;
  return MQS_OK;
}

// One step of the reverse sweep: the adjoint of step mabs (absolute) from the forward
// record a^{m-1} (A) and F_m (F); statistics into slot.
int adjoint_reverse_step(mqs_handle* H, long mabs, const double* A, const double* F, int slot) {
  cudaStream_t st = H->st;
  const CoilGeom coil{H->coil.plane_k, H->coil.i0, H->coil.j0, H->coil.i1, H->coil.j1};
  RK(launch_adj_mu(H->cg, F, H->adj, H->dt, H->dg.g.n3, st));
  RK(launch_scatter_c(H->cg, A, H->adj.ap_full, 1.0, H->dg.g.n3, st));
  const double t_src = (H->opt.rhs_time == 0 ? (double)mabs : (double)(mabs - 1)) * H->dt;
  // b' = -(h/nu0) K_cn^T mu: the right-hand side with the coil switched off
  const CoilDrive none{H->h / H->nu0, 0.0, H->coil.freq_hz, H->coil.tau, t_src, H->coil.waveform};
  RK(launch_rhs(H->dg, H->adj.mu_full, H->b, none, coil, H->sup, H->nsup, st));
  H->b_for_m = -1;                                      // b now holds an adjoint right-hand side
  int used_small = 0, init = 0;
  RK(start_vector(H, H->b, H->x, st, &used_small, &init));
  RK(pcg_launch(H, H->b, H->x, H->opt.tol, H->opt.maxit, st, init));
  H->lx_valid = true;
  record_kernel<<<1, 1, 0, st>>>(H->pres, H->small, used_small, H->opt.precision != 0 ? H->refin : nullptr,
                                 H->derr, H->dstats + slot, nullptr, nullptr, 1);
  RK(history_push(H, H->x, H->lx, st));
  RK(launch_adj_cell(H->dg, H->cg, H->x, H->adj, st));
  RK(launch_adj_lambda(H->dg, H->cg, H->x, H->adj, st));
  const CoilDrive unit{1.0, 1.0, H->coil.freq_hz, H->coil.tau, t_src, H->coil.waveform};
  RK(launch_adj_coil(H->dg, coil, unit, H->x, H->adj, st));
  return MQS_OK;
}

// The discrete adjoint over nsteps steps.  k <= 0 (or k >= nsteps) records the whole
// trajectory in the forward sweep.  k > 0 keeps a_c every k steps (checkpoints) and
// one segment's record: the reverse sweep recomputes each segment's forward steps from
// its checkpoint (on a start-vector history of their own, cold at each segment) before
// its adjoint steps (whose history runs on across segments).
int adjoint_run(mqs_handle* H, int nsteps, int k, double* grad_sigma_cell, mqs_adjoint_info* info) {
  const Range range_("mqs_adjoint");
  if (!H || nsteps < 1) return MQS_ERR_ARG;
  if (H->opt.rhs_split) return fail(H, MQS_ERR_ARG, "the adjoint runs the fused solve (rhs_split = 0)");
  if (H->n_c < 1) return fail(H, MQS_ERR_ARG, "no conducting edges");
  const bool ck = k > 0 && k < nsteps;
  const long m0 = H->m;
  const long nc = H->n_c;
  const int seglen = ck ? k : nsteps, nseg = ck ? (nsteps + k - 1) / k : 1;
  const int nstat = ck ? 3 * nsteps : 2 * nsteps;
  cudaStream_t st = H->st;
  RK(prepare_steps(H, nstat));
  RK(ensure_adjoint(H, seglen));
  if (ck) RK(ensure_ckpt(H, nseg + 1));
  double* trajA = H->traj;
  double* trajF = H->traj + (size_t)seglen * nc;
  // forward sweep: J accumulated per recorded segment
  CK(cudaMemsetAsync(H->adjJ, 0, sizeof(double), st));
  for (int s = 0; s < nsteps; ++s) {
    const int j = s % seglen;
    if (ck && j == 0) CK(cudaMemcpyAsync(H->ckpt + (size_t)(s / k) * nc, H->ac, sizeof(double) * nc,
                                         cudaMemcpyDeviceToDevice, st));
    H->rec_a = trajA + (size_t)j * nc;
    H->rec_F = trajF + (size_t)j * nc;
    const int rc = enqueue_step(H);
    if (rc != MQS_OK) { H->rec_a = H->rec_F = nullptr; return rc; }
    if (j == seglen - 1 || s == nsteps - 1) RK(launch_adj_objective(H->cg, trajF, j + 1, H->dt, H->adj, H->adjJ, st));
  }
  H->rec_a = H->rec_F = nullptr;
  const long m_end = H->m;
  if (ck) CK(cudaMemcpyAsync(H->ckpt + (size_t)nseg * nc, H->ac, sizeof(double) * nc, cudaMemcpyDeviceToDevice, st));
  // reverse sweep; the start-vector history now follows the adjoint solves
  const bool spe2 = ck && H->opt.start_mode == MQS_START_SPE;
  if (spe2) { RK(ensure_spe_alt(H)); H->alt_m = 0; RK(swap_spe(H)); }
  clear_history(H);
  H->lx_valid = false;
  CK(cudaMemsetAsync(H->adj.lam, 0, sizeof(double) * nc, st));
  CK(cudaMemsetAsync(H->adj.gmc, 0, sizeof(double) * nc, st));
  CK(cudaMemsetAsync(H->adj.gI, 0, sizeof(double), st));
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int lo = seg * seglen, hi = std::min(lo + seglen, nsteps);
    if (ck) {
      // recompute steps lo+1 .. hi from the checkpoint, recording them
      if (spe2) RK(swap_spe(H));
      clear_history(H);
      H->lx_valid = false;
      CK(cudaMemcpyAsync(H->ac, H->ckpt + (size_t)seg * nc, sizeof(double) * nc, cudaMemcpyDeviceToDevice, st));
      RK(launch_scatter_c(H->cg, H->ac, H->ac_full, 1.0, H->dg.g.n3, st));
      RK(state_changed(H));
      H->m = m0 + lo;
      H->t = H->m * H->dt;
      RK(set_ctr(H, 2 * nsteps + lo, true));
      for (int s = lo; s < hi; ++s) {
        H->rec_a = trajA + (size_t)(s - lo) * nc;
        H->rec_F = trajF + (size_t)(s - lo) * nc;
        const int rc = enqueue_step(H);
        if (rc != MQS_OK) { H->rec_a = H->rec_F = nullptr; return rc; }
      }
      H->rec_a = H->rec_F = nullptr;
      if (spe2) RK(swap_spe(H));
      else clear_history(H);
      H->lx_valid = false;
    }
    for (int m = hi; m > lo; --m)
      RK(adjoint_reverse_step(H, m0 + m, trajA + (size_t)(m - 1 - lo) * nc, trajF + (size_t)(m - 1 - lo) * nc,
                              nsteps + (nsteps - m)));
  }
  if (ck) {
    // back to the forward end state
    CK(cudaMemcpyAsync(H->ac, H->ckpt + (size_t)nseg * nc, sizeof(double) * nc, cudaMemcpyDeviceToDevice, st));
    RK(launch_scatter_c(H->cg, H->ac, H->ac_full, 1.0, H->dg.g.n3, st));
    RK(state_changed(H));
    H->m = m_end;
    H->t = H->m * H->dt;
  }
  if (spe2) { RK(swap_spe(H)); H->alt_m = 0; }
  clear_history(H);            // holds adjoint solutions, not solutions of the time loop
  H->lx_valid = false;
  RK(launch_adj_sigma(H->dg, H->cg, H->condbox, H->adj, H->adj_sig, st));
  std::vector<mqs_step_stats> hs((size_t)nstat);
  std::vector<double> sg(H->ccells);
  double J = 0.0, gI = 0.0;
  int derr = 0;
  RK(fetch_stats(H, nstat, hs.data(), &derr));
  CK(cudaMemcpyAsync(&J, H->adjJ, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&gI, H->adj.gI, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(sg.data(), H->adj_sig, sizeof(double) * H->ccells, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  RK(check_stats(H, nstat, hs.data(), derr));
  if (grad_sigma_cell) {
    const int n = H->n;
    std::fill(grad_sigma_cell, grad_sigma_cell + (size_t)n * n * n, 0.0);
    const int* lo = H->cg.clo;
    const int* hi = H->cg.chi;
    for (int kk = lo[2]; kk < hi[2]; ++kk)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i)
          grad_sigma_cell[i + (size_t)n * (j + (size_t)n * kk)] =
              sg[(i - lo[0]) + (size_t)(hi[0] - lo[0]) * ((j - lo[1]) + (size_t)(hi[1] - lo[1]) * (kk - lo[2]))];
  }
  if (info) {
    info->objective = J;
    info->grad_amplitude = gI;
    info->forward_iterations = 0;
    info->adjoint_iterations = 0;
    info->recompute_iterations = 0;
    for (int s = 0; s < nsteps; ++s) {
      info->forward_iterations += hs[s].iterations;
      info->adjoint_iterations += hs[nsteps + s].iterations;
      if (ck) info->recompute_iterations += hs[2 * nsteps + s].iterations;
    }
  }
  return MQS_OK;
}

}  // namespace

int mqs_adjoint(mqs_handle* H, int nsteps, double* grad_sigma_cell, mqs_adjoint_info* info) {
  return adjoint_run(H, nsteps, 0, grad_sigma_cell, info);
}

int mqs_adjoint_ckpt(mqs_handle* H, int nsteps, int checkpoint_every, double* grad_sigma_cell,
                     mqs_adjoint_info* info) {
  if (!H || checkpoint_every < 0) return MQS_ERR_ARG;
  return adjoint_run(H, nsteps, checkpoint_every, grad_sigma_cell, info);
}

int mqs_get_state(mqs_handle* H, double* a_c, size_t n_c, double* t, long* m) {
  if (!H) return MQS_ERR_ARG;
  if (a_c) {
    if (n_c != (size_t)H->n_c) return fail(H, MQS_ERR_ARG, "n_c mismatch");
    CK(cudaMemcpyAsync(a_c, H->ac, sizeof(double) * n_c, cudaMemcpyDeviceToHost, H->st));
  }
  CK(cudaStreamSynchronize(H->st));
  if (t) *t = H->t;
  if (m) *m = H->m;
  return MQS_OK;
}

int mqs_set_state(mqs_handle* H, const double* a_c, size_t n_c, double t, long m) {
  if (!H || !a_c) return MQS_ERR_ARG;
  if (n_c != (size_t)H->n_c) return fail(H, MQS_ERR_ARG, "n_c mismatch");
  CK(cudaMemcpyAsync(H->ac, a_c, sizeof(double) * n_c, cudaMemcpyHostToDevice, H->st));
  RK(launch_scatter_c(H->cg, H->ac, H->ac_full, 1.0, H->dg.g.n3, H->st));
  RK(state_changed(H));
  CK(cudaStreamSynchronize(H->st));
  H->t = t;
  H->m = m;
  return MQS_OK;
}

int mqs_get_state_dev(mqs_handle* H, double* a_c_dev, size_t n_c, void* stream) {
  if (!H || !a_c_dev) return MQS_ERR_ARG;
  if (n_c != (size_t)H->n_c) return fail(H, MQS_ERR_ARG, "n_c mismatch");
  cudaStream_t st = stream ? (cudaStream_t)stream : H->st;
  if (st != H->st) CK(cudaStreamSynchronize(H->st));
  CK(cudaMemcpyAsync(a_c_dev, H->ac, sizeof(double) * n_c, cudaMemcpyDeviceToDevice, st));
  return MQS_OK;
}

int mqs_set_state_dev(mqs_handle* H, const double* a_c_dev, size_t n_c, void* stream) {
  if (!H || !a_c_dev) return MQS_ERR_ARG;
  if (n_c != (size_t)H->n_c) return fail(H, MQS_ERR_ARG, "n_c mismatch");
  cudaStream_t st = stream ? (cudaStream_t)stream : H->st;
  if (st != H->st) CK(cudaStreamSynchronize(st));
  CK(cudaMemcpyAsync(H->ac, a_c_dev, sizeof(double) * n_c, cudaMemcpyDeviceToDevice, H->st));
  RK(launch_scatter_c(H->cg, H->ac, H->ac_full, 1.0, H->dg.g.n3, H->st));
  RK(state_changed(H));
  if (st != H->st) CK(cudaStreamSynchronize(H->st));
  return MQS_OK;
}

int mqs_get_solution(mqs_handle* H, double* w) {
  if (!H || !w) return MQS_ERR_ARG;
  CK(cudaMemcpyAsync(w, H->x, sizeof(double) * H->len, cudaMemcpyDeviceToHost, H->st));
  CK(cudaStreamSynchronize(H->st));
  return MQS_OK;
}

int mqs_solve_an(mqs_handle* H, double* a_n, mqs_pcg_info* info) {
  if (!H) return MQS_ERR_ARG;
  cudaStream_t st = H->st;
  const CoilGeom coil{H->coil.plane_k, H->coil.i0, H->coil.j0, H->coil.i1, H->coil.j1};
  const long m = H->m;
  const double t_src = (H->opt.rhs_time == 0 ? (double)m : (double)(m - 1)) * H->dt;
  // right-hand side j^m_{s,n} - K_cn^T a_c^m (eq. (anm)), scaled by h / nu0 as in a step
  const CoilDrive drv{H->h / H->nu0, H->coil.amplitude, H->coil.freq_hz, H->coil.tau, t_src, H->coil.waveform};
  CK(cudaMemsetAsync(H->bu, 0, sizeof(double) * H->len, st));
  RK(launch_rhs(H->dg, H->ac_full, H->bu, drv, coil, H->sup, H->nsup, st));
  CK(cudaMemcpyAsync(H->xu, H->x, sizeof(double) * H->len, cudaMemcpyDeviceToDevice, st));
  RK(run_pcg(H, H->bu, H->xu, H->opt.tol, H->opt.maxit, st));
  if (a_n) CK(cudaMemcpyAsync(a_n, H->xu, sizeof(double) * H->len, cudaMemcpyDeviceToHost, st));
  return read_pcg(H, info, st);
}

int pcg_solve_dev(mqs_handle* H, const double* b_dev, double* x_dev, double tol, int maxit, mqs_pcg_info* info,
                  void* stream) {
  if (!H || !b_dev || !x_dev) return MQS_ERR_ARG;
  if (!(tol > 0.0) || maxit < 1) return fail(H, MQS_ERR_ARG, "tol must be positive and maxit >= 1");
  cudaStream_t st = stream ? (cudaStream_t)stream : H->st;
  if (st != H->st) CK(cudaStreamSynchronize(H->st));
  RK(mask_scale(H, b_dev, H->bu, H->h / H->nu0, st));
  RK(mask_scale(H, x_dev, H->xu, 1.0, st));
  RK(run_pcg(H, H->bu, H->xu, tol, maxit, st));
  CK(cudaMemcpyAsync(x_dev, H->xu, sizeof(double) * H->len, cudaMemcpyDeviceToDevice, st));
  return read_pcg(H, info, st);
}

int pcg_solve(mqs_handle* H, const double* b, double* x, double tol, int maxit, mqs_pcg_info* info) {
  if (!H || !b || !x) return MQS_ERR_ARG;
  if (!(tol > 0.0) || maxit < 1) return fail(H, MQS_ERR_ARG, "tol must be positive and maxit >= 1");
  cudaStream_t st = H->st;
  CK(cudaMemcpyAsync(H->tmp, b, sizeof(double) * H->len, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(H->tmp2, x, sizeof(double) * H->len, cudaMemcpyHostToDevice, st));
  RK(mask_scale(H, H->tmp, H->bu, H->h / H->nu0, st));
  RK(mask_scale(H, H->tmp2, H->xu, 1.0, st));
  RK(run_pcg(H, H->bu, H->xu, tol, maxit, st));
  CK(cudaMemcpyAsync(x, H->xu, sizeof(double) * H->len, cudaMemcpyDeviceToHost, st));
  return read_pcg(H, info, st);
}

int mqs_apply_kn_dev(mqs_handle* H, const double* x_dev, double* y_dev, void* stream) {
  if (!H || !x_dev || !y_dev) return MQS_ERR_ARG;
  cudaStream_t st = stream ? (cudaStream_t)stream : H->st;
  if (st != H->st) CK(cudaStreamSynchronize(H->st));
  RK(mask_scale(H, x_dev, H->tmp2, 1.0, st));
  RK(launch_apply_L(H->dg, H->tmp2, y_dev, H->nu0 / H->h, H->full, st));
  return MQS_OK;
}

int mqs_apply_kn(mqs_handle* H, const double* x, double* y) {
  if (!H || !x || !y) return MQS_ERR_ARG;
  cudaStream_t st = H->st;
  CK(cudaMemcpyAsync(H->tmp, x, sizeof(double) * H->len, cudaMemcpyHostToDevice, st));
  RK(mask_scale(H, H->tmp, H->tmp2, 1.0, st));
  RK(launch_apply_L(H->dg, H->tmp2, H->tmp, H->nu0 / H->h, H->full, st));
  CK(cudaMemcpyAsync(y, H->tmp, sizeof(double) * H->len, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return MQS_OK;
}

int mqs_conductor_rate(mqs_handle* H, const double* a_c, const double* w, double* F) {
  if (!H || !a_c || !w || !F) return MQS_ERR_ARG;
  cudaStream_t st = H->st;
  CK(cudaMemcpyAsync(H->cvec, a_c, sizeof(double) * H->n_c, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(H->tmp, w, sizeof(double) * H->len, cudaMemcpyHostToDevice, st));
  RK(mask_scale(H, H->tmp, H->tmp2, 1.0, st));
  CK(cudaMemsetAsync(H->xu, 0, sizeof(double) * H->len, st));
  RK(launch_scatter_c(H->cg, H->cvec, H->xu, 1.0, H->dg.g.n3, st));
  RK(launch_cell_nu(H->dg, H->cg, H->xu, H->tmp2, !H->any_brauer, st));
  RK(launch_cond_update(H->dg, H->cg, H->xu, H->tmp2, 1.0, H->cvec, H->cvec2, 0.0, st));
  CK(cudaMemcpyAsync(F, H->cvec2, sizeof(double) * H->n_c, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return MQS_OK;
}

int mqs_lambda_max(mqs_handle* H, const double* v0, double pcg_tol, double rtol, int maxit, double* lambda_max,
                   int* iters) {
  if (!H || !v0 || !lambda_max) return MQS_ERR_ARG;
  return power_method(H, v0, pcg_tol, rtol, maxit, lambda_max, iters);
}

int mqs_set_stream(mqs_handle* H, void* stream) {
  if (!H) return MQS_ERR_ARG;
  cudaStream_t ns = stream ? (cudaStream_t)stream : H->own_st;
  if (ns != H->st) {
    CK(cudaStreamSynchronize(H->st));
    H->st = ns;
  }
  return MQS_OK;
}

int mqs_timing_enable(mqs_handle* H, int on) {
  if (!H) return MQS_ERR_ARG;
  CK(cudaStreamSynchronize(H->st));
  H->timing = on != 0;
  if (on) { H->ev_used = 0; H->launches = 0; H->pcg_launches = 0; H->tsteps = 0; }
  return MQS_OK;
}

int mqs_graph_steps(const mqs_handle* H, long* steps) {
  if (!H || !steps) return MQS_ERR_ARG;
  *steps = H->graph_steps;
  return MQS_OK;
}

int mqs_timing_get(mqs_handle* H, mqs_timing* out) {
  if (!H || !out) return MQS_ERR_ARG;
  CK(cudaStreamSynchronize(H->st));
  double acc[5] = {0, 0, 0, 0, 0};
  // six marks per step: phases between consecutive marks, in issue order rhs, start,
  // PCG, history (the fork of the SPE push), conductor (with the statistics record)
  for (size_t s = 0; s + 6 <= H->ev_used; s += 6)
    for (int ph = 0; ph < 5; ++ph) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, H->ev_pool[s + ph], H->ev_pool[s + ph + 1]));
      acc[ph] += ms;
    }
  out->ms_rhs = acc[0]; out->ms_start = acc[1]; out->ms_pcg = acc[2]; out->ms_history = acc[3];
  out->ms_conductor = acc[4];
  out->launches = H->launches;
  out->pcg_launches = H->pcg_launches;
  out->steps = H->tsteps;
  return MQS_OK;
}

int mqs_push_history(mqs_handle* H, const double* w) {
  if (!H || !w) return MQS_ERR_ARG;
  cudaStream_t st = H->st;
  if (H->opt.start_mode == MQS_START_POD || H->opt.start_mode == MQS_START_CSPE) RK(ensure_pod(H));
  CK(cudaMemcpyAsync(H->tmp, w, sizeof(double) * H->len, cudaMemcpyHostToDevice, st));
  RK(mask_scale(H, H->tmp, H->tmp2, 1.0, st));
  RK(launch_apply_L(H->dg, H->tmp2, H->tmp, 1.0, H->full, st));
  if (H->opt.start_mode == MQS_START_PREV) {
    CK(cudaMemcpyAsync(H->x, H->tmp2, sizeof(double) * H->len, cudaMemcpyDeviceToDevice, st));
    H->lx_valid = false;
  } else if (H->opt.start_mode == MQS_START_CSPE) {
    // the pushed solution becomes the newest (live) column, with its image
    CK(cudaMemcpyAsync(H->x, H->tmp2, sizeof(double) * H->len, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(H->lx, H->tmp, sizeof(double) * H->len, cudaMemcpyDeviceToDevice, st));
    H->lx_valid = true;
  }
  RK(history_push(H, H->tmp2, H->tmp, st));
  RK(join_side(H));
  CK(cudaStreamSynchronize(st));
  return MQS_OK;
}

int spe_start(mqs_handle* H, const double* b, double* x0, int* rank_used) {
  if (!H || !b || !x0) return MQS_ERR_ARG;
  cudaStream_t st = H->st;
  CK(cudaMemcpyAsync(H->tmp, b, sizeof(double) * H->len, cudaMemcpyHostToDevice, st));
  RK(mask_scale(H, H->tmp, H->bu, H->h / H->nu0, st));
  const int d = H->opt.spe_depth;
  RK(join_side(H));
  if (H->spe_m > 0) RK(refactor_spe(H, st));
  RK(spe_x0(vs(H->spe_D, d), H->spe_m, H->bu, H->n, H->full, nullptr, 0, H->xu, H->len, H->spe_fac, H->spe_gpart,
            H->coef, H->small, st));
  SmallOut so{};
  CK(cudaMemcpyAsync(x0, H->xu, sizeof(double) * H->len, cudaMemcpyDeviceToHost, st));
  if (H->spe_m > 0) CK(cudaMemcpyAsync(&so, H->small, sizeof(so), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (rank_used) *rank_used = so.rank;
  return MQS_OK;
}

int pod_basis(mqs_handle* H, int* k, double* sigma, double* info_ratio) {
  if (!H) return MQS_ERR_ARG;
  cudaStream_t st = H->st;
  SmallOut so{};
  const int np = H->opt.pod_snapshots;
  std::vector<double> sg(kMaxVec, 0.0);
  if (H->pod_m > 0) {
    CK(cudaMemsetAsync(H->sigma, 0, sizeof(double) * kMaxVec, st));
    CK(cudaMemsetAsync(H->bu, 0, sizeof(double) * H->len, st));
    RK(pod_x0(vs(H->pod_X, np), H->pod_m, H->pod_G, H->pod_A, H->bu, nullptr, H->len, H->opt.eps_pod, H->tspart,
              H->coef, H->sigma, H->small, st));
    CK(cudaMemcpyAsync(&so, H->small, sizeof(so), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(sg.data(), H->sigma, sizeof(double) * kMaxVec, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  if (k) *k = so.rank;
  if (info_ratio) *info_ratio = so.info;
  if (sigma) for (int a = 0; a < np; ++a) sigma[a] = (a < H->pod_m) ? sg[a] : 0.0;
  return MQS_OK;
}

int pod_start(mqs_handle* H, const double* b, double* x0, int* k) {
  if (!H || !b || !x0) return MQS_ERR_ARG;
  cudaStream_t st = H->st;
  if (H->pod_m == 0) {
    memset(x0, 0, sizeof(double) * H->len);
    if (k) *k = 0;
    return MQS_OK;
  }
  CK(cudaMemcpyAsync(H->tmp, b, sizeof(double) * H->len, cudaMemcpyHostToDevice, st));
  RK(mask_scale(H, H->tmp, H->bu, H->h / H->nu0, st));
  RK(pod_x0(vs(H->pod_X, H->opt.pod_snapshots), H->pod_m, H->pod_G, H->pod_A, H->bu, H->xu, H->len,
            H->opt.eps_pod, H->tspart, H->coef, H->sigma, H->small, st));
  SmallOut so{};
  CK(cudaMemcpyAsync(x0, H->xu, sizeof(double) * H->len, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&so, H->small, sizeof(so), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (k) *k = so.rank;
  return MQS_OK;
}

int mqs_debug_check(mqs_handle* H, mqs_debug_report* rep) {
  if (!rep) return MQS_ERR_ARG;
  *rep = mqs_debug_report{};
  if (!kDebugBuild) return MQS_OK;
  rep->enabled = 1;
  if (cudaDeviceSynchronize() != cudaSuccess) {
    if (H) H->err = "mqs_debug_check: device synchronization failed";
    return MQS_ERR_CUDA;
  }
  int (*const take[])(unsigned long long*) = {dbg_take_pcg,  dbg_take_mixed, dbg_take_conductor, dbg_take_mrhs,
                                              dbg_take_adjoint, dbg_take_api, dbg_take_noalloc};
  for (auto f : take) {
    unsigned long long w = 0;
    if (f(&w) != 0) return MQS_ERR_CUDA;
    if (!(w >> 63)) continue;
    if (rep->faults++ == 0) {
      rep->site = (int)((w >> 48) & 0x7FFF);
      rep->index = (long long)((w & 0xFFFFFFFFFFFFull) << 16) >> 16;   // 48-bit two's complement
    }
  }
  if (H) {
    unsigned char buf[kGuardBytes];
    for (size_t i = 0; i < H->allocs.size(); ++i) {
      if (cudaMemcpy(buf, static_cast<char*>(H->allocs[i]) + H->guard_at[i], kGuardBytes, cudaMemcpyDeviceToHost) !=
          cudaSuccess)
        return MQS_ERR_CUDA;
      ++rep->buffers;
      for (size_t q = 0; q < kGuardBytes; ++q)
        if (buf[q] != kGuardByte) { ++rep->canaries_bad; break; }
    }
  }
  return MQS_OK;
}

int mqs_part_ranges(int n, int nblk, int groups, int* ranges) {
  if (!ranges) return MQS_ERR_ARG;
  std::vector<int2> tab;
  const int rc = fused_partition_host(n, nblk, groups, tab);
  if (rc != MQS_OK) return rc;
  for (size_t q = 0; q < tab.size(); ++q) {
    ranges[2 * q] = tab[q].x;
    ranges[2 * q + 1] = tab[q].y;
  }
  return MQS_OK;
}

}  // extern "C"

namespace mqs {
MQS_DEBUG_TAKE(api)
}  // namespace mqs

// ---- batched multi-query ---------------------------------------------------------------

int mqs_set_blocks(mqs_handle* H, int nblk) {
  if (!H || nblk < 0) return MQS_ERR_ARG;
  int mx = 0;
  RK(pcg_max_blocks(&mx));
  if (nblk > mx) return fail(H, MQS_ERR_ARG, "more persistent blocks than can be co-resident");
  CK(cudaStreamSynchronize(H->st));     // no solve with the old block count in flight
  H->nblk = nblk == 0 ? mx : nblk;
  return ensure_ptab(H);
}

// Kernel-form tuner: the PCG forms that compute the same iterates (precision 0: the
// two-reduction kernel and the one-reduction fused pass on two tile groups with one or two
// halo warps each and on three; precision 1: the FP32 inner CG with two reductions, with
// one reduction carrying five vectors (one or two halo warps per group), and with one
// reduction carrying three vectors over a two-deep halo) differ in their tiles' halo depth, staging
// and traffic, and which is fastest depends on the grid size and the block count.  Each
// candidate solves K_n x = b_coil (the coil's pattern, unit current, the conductors at
// rest) from zero, trials + 1 times on the handle's stream and block count (the first
// untimed); the fastest median keeps its pcg_variant.  The state, the start-vector
// history and the step's right-hand side are untouched.
int mqs_tune_pcg(mqs_handle* H, int trials, int* chosen) {
  if (!H || trials < 1) return MQS_ERR_ARG;
  const Range range_("mqs_tune_pcg");
  // candidates (pcg_variant, tile_groups, halo_warps)
  int cand[4][3] = {}, nc = 0;
  if (H->opt.precision == 0) {
    const int f[4][3] = {{0, 0, 0}, {1, 2, 1}, {1, 3, 1}, {1, 2, 2}};
    for (nc = 0; nc < 4; ++nc)
      for (int q = 0; q < 3; ++q) cand[nc][q] = f[nc][q];
  } else if (H->opt.precision == 1) {
    const int f[4][3] = {{0, 0, 0}, {1, 0, 0}, {1, 0, 2}, {2, 0, 0}};
    for (nc = 0; nc < 4; ++nc)
      for (int q = 0; q < 3; ++q) cand[nc][q] = f[nc][q];
  } else {
    cand[0][0] = H->opt.pcg_variant;    // one float-float inner form
    nc = 1;
  }
  cudaStream_t st = H->st;
  RK(join_side(H));
  const CoilGeom coil{H->coil.plane_k, H->coil.i0, H->coil.j0, H->coil.i1, H->coil.j1};
  const CoilDrive unit{H->h / H->nu0, 1.0, 0.0, 1.0, 50.0, 1};   // ramp waveform at t = 50 tau: i = 1
  CK(cudaMemsetAsync(H->tmp, 0, sizeof(double) * H->len, st));
  CK(cudaMemsetAsync(H->bu, 0, sizeof(double) * H->len, st));
  RK(launch_rhs(H->dg, H->tmp, H->bu, unit, coil, H->sup, H->nsup, st));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(H, MQS_ERR_CUDA, "mqs_tune_pcg: event creation failed");
  }
  const int saved = H->opt.pcg_variant, saved_groups = H->opt.tile_groups, saved_halo = H->opt.halo_warps;
  int best = saved, best_groups = saved_groups, best_halo = saved_halo, rc = MQS_OK;
  float best_ms = 0.f;
  for (int c = 0; c < nc && rc == MQS_OK; ++c) {
    H->opt.pcg_variant = cand[c][0];
    H->opt.tile_groups = cand[c][1];
    H->opt.halo_warps = cand[c][2];
    rc = ensure_ptab(H);
    if (rc != MQS_OK) break;
    std::vector<float> ms;
    for (int r = 0; r <= trials && rc == MQS_OK; ++r) {
      if (cudaMemsetAsync(H->derr, 0, sizeof(int), st) != cudaSuccess ||
          cudaMemsetAsync(H->xu, 0, sizeof(double) * H->len, st) != cudaSuccess ||
          cudaEventRecord(e0, st) != cudaSuccess) {
        rc = fail(H, MQS_ERR_CUDA, "mqs_tune_pcg: enqueue failed");
        break;
      }
      rc = pcg_launch(H, H->bu, H->xu, H->opt.tol, H->opt.maxit, st, 2);
      if (rc != MQS_OK) break;
      PcgResult pr{};
      int derr = 0;
      if (cudaEventRecord(e1, st) != cudaSuccess ||
          cudaMemcpyAsync(&pr, H->pres, sizeof pr, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaMemcpyAsync(&derr, H->derr, sizeof derr, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        rc = fail(H, MQS_ERR_CUDA, "mqs_tune_pcg: trial solve failed");
        break;
      }
      if (derr != 0 || pr.status != MQS_OK) {
        rc = fail(H, derr ? derr : pr.status, "mqs_tune_pcg: trial solve did not converge");
        break;
      }
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (r > 0) ms.push_back(t);
    }
    if (rc != MQS_OK) break;
    std::sort(ms.begin(), ms.end());
    const float med = ms[ms.size() / 2];
    if (c == 0 || med < best_ms) { best = cand[c][0]; best_groups = cand[c][1]; best_halo = cand[c][2]; best_ms = med; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  H->opt.pcg_variant = (rc == MQS_OK) ? best : saved;
  H->opt.tile_groups = (rc == MQS_OK) ? best_groups : saved_groups;
  H->opt.halo_warps = (rc == MQS_OK) ? best_halo : saved_halo;
  if (ensure_ptab(H) != MQS_OK && rc == MQS_OK) rc = MQS_ERR_CUDA;
  H->lx_valid = false;                   // lx held the trial solves' images
  if (chosen) *chosen = H->opt.pcg_variant;
  return rc;
}

// status-only variants of CK / RK for calls that belong to no single handle
#define BCK(call)                                         \
  do {                                                    \
    if ((call) != cudaSuccess) return MQS_ERR_CUDA;       \
  } while (0)
#define BRK(call)                                         \
  do {                                                    \
    int r_ = (call);                                      \
    if (r_ != MQS_OK) return r_;                          \
  } while (0)

// streams of a batch: CUDA maps streams onto at most 32 hardware queues
// (CUDA_DEVICE_MAX_CONNECTIONS), so more streams would only alias
constexpr int kBatchStreams = 32;

// a graph of kBatchGraphSteps steps of every handle of a batch, issued step-major as
// the launch-by-launch path does (each handle's launches on its own batch stream, so
// the handles drift apart inside the graph and meet only at its end)
constexpr int kBatchGraphSteps = 8;
struct BatchGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<GraphKey> keys;
};

struct mqs_batch {
  std::vector<mqs_handle*> hs;
  std::vector<cudaStream_t> streams, saved_st;
  std::vector<int> saved_nblk;
  std::vector<cudaEvent_t> done;
  cudaStream_t master = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evf = nullptr;
  double scale = 2.0;
  float last_ms = 0.f;
  BatchGraph graphs[2];
  int graph_next = 0;
  bool graph_off = false;
  long graph_steps = 0;     // batch steps replayed from (or captured into) a graph
  // block shares by unknowns (false) or by unknowns x PCG iterations per step (true)
  bool by_work = false;
  std::vector<double> its_avg;   // per handle: mean PCG iterations per step of the last call
  double last_work = 0.0;        // sum over handles and steps of the last call: unknowns x iterations
};

namespace {

// block counts proportional to each problem's share of the work, scaled so that they add
// up to about `scale` blocks per SM.  The share is its unknowns, or (by_work) its unknowns
// times its PCG iterations per step in the last call: the problems' solves then take
// about the same time on their blocks, and the batch step is not paced by the problems
// whose iteration counts are highest.
int batch_assign(mqs_batch* B) {
  int mx = 0;
  BRK(pcg_max_blocks(&mx));
  const size_t cnt = B->hs.size();
  std::vector<double> w(cnt);
  double wsum = 0.0;
  for (size_t i = 0; i < cnt; ++i) {
    const double its = (B->by_work && i < B->its_avg.size() && B->its_avg[i] > 0.0) ? B->its_avg[i] : 1.0;
    w[i] = (double)B->hs[i]->n_n * its;
    wsum += w[i];
  }
  for (size_t i = 0; i < cnt; ++i) {
    mqs_handle* H = B->hs[i];
    long nb = std::lround(B->scale * mx * w[i] / std::max(wsum, 1.0));
    H->nblk = (int)std::min<long>(std::max<long>(nb, 1), mx);
    H->ts_cap = std::max(2 * H->nblk, 4);    // its tall-skinny kernels: about its share of the SMs
    BRK(ensure_ptab(H));
  }
  return MQS_OK;
}

void batch_release(mqs_batch* B) {
  for (cudaStream_t s : B->streams)
    if (s) cudaStreamSynchronize(s);
  for (size_t i = 0; i < B->hs.size(); ++i) {
    B->hs[i]->st = B->saved_st[i];
    B->hs[i]->nblk = B->saved_nblk[i];
    B->hs[i]->ts_cap = 0;
    ensure_ptab(B->hs[i]);
    B->hs[i]->in_batch = false;
  }
  if (B->master) cudaStreamSynchronize(B->master);
  for (BatchGraph& g : B->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (cudaStream_t s : B->streams) if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : B->done) if (e) cudaEventDestroy(e);
  if (B->ev0) cudaEventDestroy(B->ev0);
  if (B->ev1) cudaEventDestroy(B->ev1);
  if (B->evf) cudaEventDestroy(B->evf);
  if (B->master) cudaStreamDestroy(B->master);
  delete B;
}

// the batch streams' work so far joins the master stream / the master's joins the streams
int batch_to_master(mqs_batch* B) {
  for (size_t i = 0; i < B->streams.size(); ++i) {
    if (cudaEventRecord(B->done[i], B->streams[i]) != cudaSuccess) return MQS_ERR_CUDA;
    if (cudaStreamWaitEvent(B->master, B->done[i], 0) != cudaSuccess) return MQS_ERR_CUDA;
  }
  return MQS_OK;
}
int master_to_batch(mqs_batch* B) {
  if (cudaEventRecord(B->evf, B->master) != cudaSuccess) return MQS_ERR_CUDA;
  for (cudaStream_t s : B->streams)
    if (cudaStreamWaitEvent(s, B->evf, 0) != cudaSuccess) return MQS_ERR_CUDA;
  return MQS_OK;
}

// kBatchGraphSteps steps of every handle from a graph on the master stream, when every
// handle is eligible (see graph_step); *done false otherwise.  *on_master tracks where
// the batch's latest work is.
int batch_graph_steps(mqs_batch* B, bool* on_master, bool* done) {
  *done = false;
  if (B->graph_off) return MQS_OK;
  for (mqs_handle* H : B->hs)
    if (!graph_eligible(H)) return MQS_OK;
  const size_t cnt = B->hs.size();
  std::vector<GraphKey> keys(cnt);
  std::vector<StepHost> s0(cnt), s1(cnt);
  for (size_t i = 0; i < cnt; ++i) {
    keys[i] = graph_key(B->hs[i]);
    s0[i] = save_host(B->hs[i]);
    s1[i] = s0[i];
    for (int k = 0; k < kBatchGraphSteps; ++k) s1[i] = after_step(B->hs[i], s1[i]);
  }
  if (!*on_master) {
    const int r = batch_to_master(B);
    if (r != MQS_OK) return r;
    *on_master = true;
  }
  for (BatchGraph& g : B->graphs)
    if (g.exec && g.keys.size() == cnt && memcmp(g.keys.data(), keys.data(), sizeof(GraphKey) * cnt) == 0) {
      if (cudaGraphLaunch(g.exec, B->master) != cudaSuccess) return MQS_ERR_CUDA;
      for (size_t i = 0; i < cnt; ++i) load_host(B->hs[i], s1[i]);
      B->graph_steps += kBatchGraphSteps;
      *done = true;
      return MQS_OK;
    }
  BatchGraph& g = B->graphs[B->graph_next];
  B->graph_next ^= 1;
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g.exec = nullptr;
  cudaGraphExec_t exec = nullptr;
  const bool ok = capture(
      B->master,
      [&] {
        if (master_to_batch(B) != MQS_OK) return false;
        bool good = true;
        for (int k = 0; k < kBatchGraphSteps && good; ++k)
          for (size_t i = 0; i < cnt && good; ++i) good = enqueue_step(B->hs[i]) == MQS_OK;
        for (size_t i = 0; i < cnt; ++i) good = good && same_host(save_host(B->hs[i]), s1[i]);
        return batch_to_master(B) == MQS_OK && good;   // joined also after a failure
      },
      &exec);
  if (!ok) {
    for (size_t i = 0; i < cnt; ++i) {
      load_host(B->hs[i], s0[i]);
      B->hs[i]->err.clear();
    }
    B->graph_off = true;
    return MQS_OK;
  }
  g.exec = exec;
  g.keys = keys;
  if (cudaGraphLaunch(exec, B->master) != cudaSuccess) return MQS_ERR_CUDA;
  B->graph_steps += kBatchGraphSteps;
  *done = true;
  return MQS_OK;
}

}  // namespace

int mqs_batch_create(mqs_handle* const* handles, int count, double blocks_scale, mqs_batch** out) {
  if (!out) return MQS_ERR_ARG;
  *out = nullptr;
  if (!handles || count < 1) return MQS_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    if (!handles[i]) return MQS_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) return MQS_ERR_ARG;
  }
  mqs_batch* B = new (std::nothrow) mqs_batch;
  if (!B) return MQS_ERR_OOM;
  B->scale = blocks_scale > 0.0 ? blocks_scale : 2.0;
  bool ok = cudaStreamCreateWithFlags(&B->master, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreate(&B->ev0) == cudaSuccess && cudaEventCreate(&B->ev1) == cudaSuccess &&
            cudaEventCreateWithFlags(&B->evf, cudaEventDisableTiming) == cudaSuccess;
  const int ns = std::min(count, kBatchStreams);
  for (int i = 0; ok && i < ns; ++i) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (s) B->streams.push_back(s);
    if (e) B->done.push_back(e);
  }
  for (int i = 0; ok && i < count; ++i) {
    mqs_handle* H = handles[i];
    ok = cudaStreamSynchronize(H->st) == cudaSuccess;
    if (!ok) break;
    B->hs.push_back(H);
    B->saved_st.push_back(H->st);
    B->saved_nblk.push_back(H->nblk);
    H->st = B->streams[i % ns];
    H->in_batch = true;
  }
  if (!ok) { batch_release(B); return MQS_ERR_CUDA; }
  const int rc = batch_assign(B);
  if (rc != MQS_OK) { batch_release(B); return rc; }
  *out = B;
  return MQS_OK;
}

int mqs_batch_set_scale(mqs_batch* B, double blocks_scale) {
  if (!B || !(blocks_scale > 0.0)) return MQS_ERR_ARG;
  for (cudaStream_t s : B->streams) BCK(cudaStreamSynchronize(s));
  B->scale = blocks_scale;
  return batch_assign(B);
}

int mqs_batch_step(mqs_batch* B, int nsteps, mqs_step_stats* per_step) {
  const Range range_("mqs_batch_step");
  if (!B || nsteps < 0) return MQS_ERR_ARG;
  const int cnt = (int)B->hs.size();
  for (mqs_handle* H : B->hs)
    if (!(H->dt > 0.0)) return fail(H, MQS_ERR_ARG, "dt is not set");
  if (nsteps == 0) return MQS_OK;
  for (mqs_handle* H : B->hs) RK(prepare_steps(H, nsteps));
  BCK(cudaEventRecord(B->ev0, B->master));
  for (cudaStream_t s : B->streams) BCK(cudaStreamWaitEvent(s, B->ev0, 0));
  int rc = MQS_OK;
  // step-major issue order: every problem's step s is queued before any step s+1,
  // so the streams advance side by side; whole chunks of steady-state steps come
  // from a graph
  bool on_master = false;
  for (int s = 0; s < nsteps && rc == MQS_OK;) {
    bool done = false;
    if (nsteps - s >= kBatchGraphSteps) rc = batch_graph_steps(B, &on_master, &done);
    if (rc != MQS_OK) break;
    if (done) {
      s += kBatchGraphSteps;
      continue;
    }
    if (on_master) {
      rc = master_to_batch(B);
      on_master = false;
    }
    for (int i = 0; i < cnt && rc == MQS_OK; ++i) rc = enqueue_step(B->hs[i]);
    ++s;
  }
  for (mqs_handle* H : B->hs)
    if (join_side(H) != MQS_OK && rc == MQS_OK) rc = MQS_ERR_CUDA;   // side streams inside the timed span
  if (!on_master) BRK(batch_to_master(B));
  BCK(cudaEventRecord(B->ev1, B->master));
  BRK(master_to_batch(B));     // the statistics copies below follow every step
  if (rc != MQS_OK) {
    for (cudaStream_t s : B->streams) cudaStreamSynchronize(s);
    return rc;
  }
  std::vector<mqs_step_stats> hs((size_t)nsteps * cnt);
  std::vector<int> derr(cnt, 0);
  for (int i = 0; i < cnt; ++i) BRK(fetch_stats(B->hs[i], nsteps, hs.data() + (size_t)i * nsteps, &derr[i]));
  for (cudaStream_t s : B->streams) BCK(cudaStreamSynchronize(s));
  BCK(cudaEventSynchronize(B->ev1));
  BCK(cudaEventElapsedTime(&B->last_ms, B->ev0, B->ev1));
  B->its_avg.assign(cnt, 0.0);
  B->last_work = 0.0;
  for (int i = 0; i < cnt; ++i) {
    double its = 0.0;
    for (int s = 0; s < nsteps; ++s) its += hs[(size_t)i * nsteps + s].iterations;
    B->its_avg[i] = its / nsteps;
    B->last_work += its * (double)B->hs[i]->n_n;
  }
  if (per_step)
    for (int s = 0; s < nsteps; ++s)
      for (int i = 0; i < cnt; ++i) per_step[(size_t)s * cnt + i] = hs[(size_t)i * nsteps + s];
  for (int i = 0; i < cnt; ++i) {
    const int r = finish_call(B->hs[i], nsteps, hs.data() + (size_t)i * nsteps, derr[i]);
    if (r != MQS_OK && rc == MQS_OK) rc = r;
  }
  return rc;
}

int mqs_batch_last_ms(mqs_batch* B, double* ms) {
  if (!B || !ms) return MQS_ERR_ARG;
  *ms = B->last_ms;
  return MQS_OK;
}

int mqs_batch_tune(mqs_batch* B, int trial_steps, double* best_scale) {
  if (!B || trial_steps < 1) return MQS_ERR_ARG;
  // candidates: the scales, with the current block shares (by unknowns unless
  // mqs_batch_set_weighting chose the work weighting: in the tuner it measured slower,
  // 2862-2903 against 3177-3238 instance-steps/s on the 64-problem FP64 set, and won
  // trials by noise).  Each is scored by device time per unit of PCG work (unknowns x
  // iterations) of its trial, so that the falling iteration counts of a starting
  // transient do not favour the candidates tried last, and the candidates run in the
  // order c_0 .. c_3, then c_3 .. c_0 with both scores added.
  struct Cand { double scale; bool by_work; };
  const Cand cand[] = {{1.0, B->by_work}, {2.0, B->by_work}, {4.0, B->by_work}, {8.0, B->by_work}};
  constexpr int kc = 4;
  double score[kc] = {};
  for (int r = 0; r < 2 * kc; ++r) {
    const Cand& c = cand[r < kc ? r : 2 * kc - 1 - r];
    B->by_work = c.by_work;
    BRK(mqs_batch_set_scale(B, c.scale));
    BRK(mqs_batch_step(B, trial_steps, nullptr));
    score[r < kc ? r : 2 * kc - 1 - r] += B->last_ms / std::max(B->last_work, 1.0);
  }
  int best = 0;
  for (int c = 1; c < kc; ++c)
    if (score[c] < score[best]) best = c;
  B->by_work = cand[best].by_work;
  BRK(mqs_batch_set_scale(B, cand[best].scale));
  if (best_scale) *best_scale = cand[best].scale;
  return MQS_OK;
}

int mqs_batch_tune_pcg(mqs_batch* B, int trials, int* chosen) {
  if (!B || trials < 1) return MQS_ERR_ARG;
  for (cudaStream_t s : B->streams) BCK(cudaStreamSynchronize(s));
  const size_t cnt = B->hs.size();
  std::vector<int> done(cnt, 0);
  for (size_t i = 0; i < cnt; ++i) {
    if (done[i]) continue;
    mqs_handle* H = B->hs[i];
    int v = 0;
    RK(mqs_tune_pcg(H, trials, &v));      // on its batch stream and its share of the blocks
    for (size_t j = i + 1; j < cnt; ++j) {
      mqs_handle* G = B->hs[j];
      if (!done[j] && G->n == H->n && G->opt.precision == H->opt.precision) {
        G->opt.pcg_variant = v;
        G->opt.tile_groups = H->opt.tile_groups;
        G->opt.halo_warps = H->opt.halo_warps;
        RK(ensure_ptab(G));
        done[j] = 1;
      }
    }
    done[i] = 1;
  }
  if (chosen)
    for (size_t i = 0; i < cnt; ++i) chosen[i] = B->hs[i]->opt.pcg_variant;
  return MQS_OK;
}

int mqs_batch_set_weighting(mqs_batch* B, int by_work) {
  if (!B || by_work < 0 || by_work > 1) return MQS_ERR_ARG;
  for (cudaStream_t s : B->streams) BCK(cudaStreamSynchronize(s));
  B->by_work = by_work != 0;
  return batch_assign(B);
}

int mqs_batch_get_weighting(const mqs_batch* B, int* by_work) {
  if (!B || !by_work) return MQS_ERR_ARG;
  *by_work = B->by_work ? 1 : 0;
  return MQS_OK;
}

int mqs_batch_tune_depth(mqs_batch* B, int trial_steps, const int* depths, int ndepths, int* chosen) {
  if (!B || trial_steps < 1 || !depths || ndepths < 1) return MQS_ERR_ARG;
  int dmax = 0;
  for (int c = 0; c < ndepths; ++c) {
    if (depths[c] < 1 || depths[c] > kMaxSpe) return MQS_ERR_ARG;
    dmax = std::max(dmax, depths[c]);
  }
  const size_t cnt = B->hs.size();
  // the SPE handles grouped by grid size, each group's depth searched in turn with the
  // others held (coordinate search on the batch's device time)
  std::vector<int> sizes;
  for (mqs_handle* H : B->hs)
    if (H->opt.start_mode == MQS_START_SPE && std::find(sizes.begin(), sizes.end(), H->n) == sizes.end())
      sizes.push_back(H->n);
  std::sort(sizes.begin(), sizes.end());
  auto set_group = [&](int n, int d) -> int {
    for (mqs_handle* H : B->hs)
      if (H->opt.start_mode == MQS_START_SPE && H->n == n && H->opt.spe_depth != d) {
        mqs_options o = H->opt;
        o.spe_depth = d;
        RK(mqs_set_options(H, &o));   // a new depth starts a new history
      }
    return MQS_OK;
  };
  // candidates in the order c_0 .. c_{k-1}, c_{k-1} .. c_0 with the two trial times of a
  // candidate added: the iteration counts of a transient drift from trial to trial, and
  // the mirrored order cancels a linear drift (one pass in one order favours the last)
  for (int n : sizes) {
    std::vector<double> ms(ndepths, 0.0);
    for (int r = 0; r < 2 * ndepths; ++r) {
      const int c = r < ndepths ? r : 2 * ndepths - 1 - r;
      BRK(set_group(n, depths[c]));
      BRK(mqs_batch_step(B, dmax + 1, nullptr));       // every table full again
      BRK(mqs_batch_step(B, trial_steps, nullptr));
      ms[c] += B->last_ms;
    }
    int best = 0;
    for (int c = 1; c < ndepths; ++c)
      if (ms[c] < ms[best]) best = c;
    BRK(set_group(n, depths[best]));
  }
  if (chosen)
    for (size_t i = 0; i < cnt; ++i) chosen[i] = B->hs[i]->opt.spe_depth;
  return MQS_OK;
}

int mqs_batch_graph_steps(const mqs_batch* B, long* steps) {
  if (!B || !steps) return MQS_ERR_ARG;
  *steps = B->graph_steps;
  return MQS_OK;
}

int mqs_batch_destroy(mqs_batch* B) {
  if (!B) return MQS_ERR_ARG;
  batch_release(B);
  return MQS_OK;
}
