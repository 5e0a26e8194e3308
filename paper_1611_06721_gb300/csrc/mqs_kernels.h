// Host-side declarations shared by the translation units of the library.
#pragma once
#include <vector>
#include <cuda_runtime.h>
#include "mqs_internal.cuh"

namespace mqs {

struct PcgResult {
  int iterations;
  int status;
  double relres;
  double start_relres;
};

struct DevGeom {
  Geom g;                 // device view (cflags points to device memory)
};

// Device state of a stepping call (one per handle): the halt flag that makes every
// step after a failing one skip its solve and its conductor update, and the
// instability monitor of the explicit Euler update (mqs_options.monitor_steps).
struct StepGuard {
  int halt;               // 1 once a step of the current call failed (set by the record kernels)
  int status;             // the monitor's verdict on the last conductor update it checked
  unsigned arrive;        // blocks of the running conductor update that wrote their partials
  int pad;
  // from here on: the monitor's history, cleared whenever the state changes outside a step
  int count;              // consecutive steps with growing, sign-alternating increments
  int valid;              // the other conductor buffer holds the state before the current one
  double e_prev;          // M_c-energy of the last increment
  double e_max;           // largest increment energy since the last clear
};
constexpr int kMonBlocks = 1024;          // most blocks of a conductor update (2 partials each)
// what a guarded conductor update reads besides its operands: the guard and its partials,
// the solve it follows (its result and the call's error word) and the monitor window
struct GuardView {
  StepGuard* gd;
  double* part;
  const PcgResult* pres;
  const int* derr;
  int window;             // > 0: consecutive steps that flag an instability; <= 0: finiteness only
};

// init: 0 = the kernel forms r = b - L x; 1 = r holds b - L x already;
// 2 = zero start (the kernel sets x = 0, r = b).
// halt (nullable): a solve issued inside a stepping call returns at once, writing a
// zero-iteration MQS_OK result, when *halt != 0 (an earlier step of the call failed).
int launch_pcg(const DevGeom& dg, const double* b, double* x, double* r, double* p, double* q, double* lx,
               double* part, unsigned* bar, int* err, PcgResult* out, double tol, int maxit, int nblk,
               cudaStream_t st, int init = 0, const int* halt = nullptr);
int pcg_max_blocks(int* nblk);

// mixed precision: FP64 iterative refinement around FP32 CG inner solves
struct MixedBufs {
  float* r32; float* p32; float* q32; float* d32;
  float* r32b; float* w32a; float* w32b; float* s32a; float* s32b;   // one-reduction inner CG only
};
// halo_warps 2: the one-reduction inner pass (variant 1) with two halo warps per group in
// 384-thread blocks, at one block per SM (below 96^3); other forms ignore it
int launch_pcg_mixed(const DevGeom& dg, const double* b, double* x, double* r, double* lx, const MixedBufs& mb,
                     double* part, unsigned* bar, int* err, PcgResult* out, int* refinements, double tol,
                     double inner_tol, int maxit, int nblk, cudaStream_t st, int init = 0, int variant = 0,
                     const int* halt = nullptr, const int2* ptab = nullptr, int halo_warps = 0);
// precision 2: the same refinement with float-float one-reduction inner solves
// (MixedBufs sized for 8 bytes per value, all nine buffers)
int launch_pcg_ff(const DevGeom& dg, const double* b, double* x, double* r, double* lx, const MixedBufs& mb,
                  double* part, unsigned* bar, int* err, PcgResult* out, int* refinements, double tol,
                  double inner_tol, int maxit, int nblk, cudaStream_t st, int init = 0,
                  const int* halt = nullptr, const int2* ptab = nullptr);

// one-reduction PCG (one fused stencil pass and one grid reduction per
// iteration); needs five more layout vectors
struct PcgExtra { double* r1; double* w0; double* w1; double* s0; double* s1; };
// groups: stencil groups per block (0 or 2: the default 320-thread block; 3: 480 threads,
// 128 registers a thread).  halo_warps: halo warps per group of the fused pass (0 or 1; 2
// with two groups: 384 threads).  MQS_ERR_ARG for other forms or a block that does not fit.
// ptab (nullable): the fused pass's part ranges from fused_partition for this n, nblk and
// groups; nullptr splits the plane-tiles evenly.
int launch_pcg_fused(const DevGeom& dg, const double* b, double* x, double* r, double* p, double* lx,
                     const PcgExtra& ex, double* part, unsigned* bar, int* err, PcgResult* out, double tol, int maxit,
                     int nblk, cudaStream_t st, int init = 0, const int* halt = nullptr, int groups = 0,
                     const int2* ptab = nullptr, int halo_warps = 0);
// the cost-balanced part ranges of the fused pass (nblk x groups int2 entries) into
// dev_table; blocks the host (a synchronous upload on st: not for use during stream capture)
int fused_partition(int n, int nblk, int groups, int2* dev_table, cudaStream_t st);
// the same table on the host (no CUDA call): nblk x groups ranges into tab
int fused_partition_host(int n, int nblk, int groups, std::vector<int2>& tab);

// y = scale * (L s) on n-edges of `box` (zero on other edges of the box).
int launch_apply_L(const DevGeom& dg, const double* s, double* y, double scale, Box box, cudaStream_t st);

// the coil loop (plane_k, i0, j0, i1, j1) and its current: i_S(t) = amplitude sin(2 pi
// freq t) (waveform 0) or amplitude (1 - exp(-t / tau)) (waveform 1), times scale
struct CoilGeom { int k, i0, j0, i1, j1; };
// i_S at time t, or (m_dev != nullptr) at t = (*m_dev + level) * dt: the step counter on
// the device, so a captured step's launches do not change from step to step
struct CoilDrive {
  double scale, amplitude, freq, tau, t;
  int waveform;
  const long long* m_dev = nullptr;
  long long level = 0;
  double dt = 0.0;
};
// b = scale i_S(t) X_s - L ac_full (eq. (mrhs) in scaled units, scale = h/nu0;
// amplitude 0 gives b = -L ac) at the listed layout indices only: the right-hand side's support (n-edges
// sharing a face with a c-edge, and the coil); b keeps its values elsewhere (zero for
// the step's b)
int launch_rhs(const DevGeom& dg, const double* ac_full, double* b, CoilDrive drive, CoilGeom coil, const int* sup,
               int nsup, cudaStream_t st);

// Conductor region kernels (eq. (acm)).
struct CondGeom {
  int clo[3], chi[3];     // cell box of the conducting cells
  int n_c;
  const int* c_idx;       // layout index of every c-edge (compact order)
  const double* inv_mc;   // 1 / M_c per c-edge
  const uint8_t* brauer;  // flags over the cell box (1 = Brauer)
  double* nu;             // reluctivity over the cell box
  double nu0, k1, k2, k3, h;
  // No further fields: with one more (n^3, for the debug checks) the compiler gave
  // cond_update_kernel 48 registers instead of 56, and the step's conductor phase took
  // 90 instead of 60 us.  Launchers that need n^3 take it as a parameter.
};
// nu per cell of the cell box from a = ac_full + w (nonlinear cells); if
// `at_zero` the Brauer law is evaluated at B = 0.  halt (nullable): nothing is done
// when *halt != 0.
int launch_cell_nu(const DevGeom& dg, const CondGeom& cg, const double* ac_full, const double* w, bool at_zero,
                   cudaStream_t st, const int* halt = nullptr);
// F = (K(a) a)_c at every c-edge (a = ac_full + sign_w * w).  If dt != 0:
// a_c_out = a_c_in - dt F / M_c, else F is written to a_c_out.  If
// ac_full_out is given (a layout buffer other than ac_full), the result is
// also written there at the c-edges.  F_out / a_prev_out (nullable) receive
// F and a_c_in per c-edge (the recorded trajectory of the adjoint).
// guard (nullable; steps only): the update writes nothing when the call is halted, the
// solve it follows failed or a device wait timed out; otherwise (dt != 0) it also runs
// the instability monitor, whose verdict goes to guard->gd->status.  a_c_out must then
// hold the state before a_c_in (the buffer pair alternates), read before it is written.
int launch_cond_update(const DevGeom& dg, const CondGeom& cg, const double* ac_full, const double* w,
                       double sign_w, const double* a_c_in, double* a_c_out, double dt, cudaStream_t st,
                       double* ac_full_out = nullptr, double* F_out = nullptr, double* a_prev_out = nullptr,
                       const GuardView* guard = nullptr);
// scatter compact a_c into the layout vector ac_full (c-edges only)
// (n3: n^3 of the grid, for the debug build's index checks)
int launch_scatter_c(const CondGeom& cg, const double* a_c, double* ac_full, double scale, long long n3,
                     cudaStream_t st);


// ---- discrete adjoint of the time loop (adjoint.cu) ----
struct AdjBufs {
  double* lam;            // [n_c] dJ/da^m
  double* gmc;            // [n_c] dJ/dM_c accumulated
  double* mu_full;        // layout: mu on c-edges, zero elsewhere
  double* ap_full;        // layout: a^{m-1} on c-edges, zero elsewhere
  double* tS;             // 3 x cell-box: t_c S_{c,d} per Brauer cell (0 elsewhere)
  double* gI;             // [1] dJ/d(coil amplitude) accumulated
  double* part;           // >= 1024 doubles of reduction scratch
  int* qmap;              // 3 x (node box + 1)^3: compact c-index of an edge or -1
};
// mu = dt M_c^-1 (2F - lam) scattered to mu_full; gmc += dt F (lam - F) / M_c^2
int launch_adj_mu(const CondGeom& cg, const double* F, const AdjBufs& ab, double dt, long long n3, cudaStream_t st);
// per Brauer cell: nu from a^{m-1} (into cg.nu) and t_c S_c from the forward fluxes of
// ap_full and the adjoint fluxes of mu_full + x
int launch_adj_cell(const DevGeom& dg, const CondGeom& cg, const double* x, const AdjBufs& ab, cudaStream_t st);
// lam += (C^T J_H^T C [mu; x])_c
int launch_adj_lambda(const DevGeom& dg, const CondGeom& cg, const double* x, const AdjBufs& ab, cudaStream_t st);
// gI += -g(t) X_s . x over the coil loop (g: the unit-amplitude waveform of drv at drv.t)
int launch_adj_coil(const DevGeom& dg, const CoilGeom& coil, const CoilDrive& drv, const double* x,
                    const AdjBufs& ab, cudaStream_t st);
// *J_dev += dt sum over the nsteps recorded steps and c-edges of F^2 / M_c
int launch_adj_objective(const CondGeom& cg, const double* F_traj, int nsteps, double dt, const AdjBufs& ab,
                         double* J_dev, cudaStream_t st);
// qmap from the compact c-edge list (node box lo = cg.clo, extent cg.chi - cg.clo + 1 per axis)
int launch_adj_qmap(const DevGeom& dg, const CondGeom& cg, const AdjBufs& ab, cudaStream_t st);
// dJ/dsigma per cell of the cell box: (h/4) * sum of gmc over the cell's c-edges where
// cond[cell] != 0, else 0
int launch_adj_sigma(const DevGeom& dg, const CondGeom& cg, const uint8_t* cond, const AdjBufs& ab, double* out,
                     cudaStream_t st);

// debug builds (MQS_DEBUG_CHECKS): the first out-of-range index a translation unit's
// kernels met, as (1 << 63) | site << 48 | index (0: none), cleared by the read.
// Release builds report 0.  Returns 0 or -2 (CUDA error).
int dbg_take_pcg(unsigned long long* out);
int dbg_take_mixed(unsigned long long* out);
int dbg_take_conductor(unsigned long long* out);
int dbg_take_mrhs(unsigned long long* out);
int dbg_take_adjoint(unsigned long long* out);
int dbg_take_api(unsigned long long* out);
int dbg_take_noalloc(unsigned long long* out);

}  // namespace mqs
