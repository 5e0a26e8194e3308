// Start-vector kernels (Sec. III): SPE difference table and POD snapshots.
#pragma once
#include "mqs_internal.cuh"

namespace mqs {

constexpr int kMaxSpe = 16;
constexpr int kMaxPod = 40;
constexpr int kMaxCspe = 19;        // CSPE basis: frozen columns + the live one (below 20, Sec. IV)
constexpr int kMaxVec = 40;
constexpr int kTileSlots = 72;      // 8 x 8 products + 8 right-hand side products

struct VecSet { const double* v[kMaxVec]; };
struct MutVecSet { double* v[kMaxVec]; };
struct SmallOut { int rank; int pad; double info; };

int ts_nblk();
// Most blocks a tall-skinny launch of the calling host thread may use (0: no limit, up
// to two per SM): a batch sets each problem's share around its launches so that the
// problems' start-vector and history kernels run side by side, as their PCG kernels do.
void set_launch_cap(int cap);
int launch_cap();
// partial-sum buffer needed: 5 tiles * ts_nblk() * kTileSlots doubles
constexpr int kSpeGSlots = 16;      // g = D^T b partials per block
// Factor of the SPE small system (device memory): rows of the scaled Cholesky factor
// with the drop rule applied, reciprocal pivots (0 = dropped), diagonal scaling
struct SpeFac {
  double L[kMaxSpe * kMaxSpe];
  double inv[kMaxSpe];
  double sc[kMaxSpe];
  int nk, m;
  // arrival counter of the g kernel (zero between launches): its last block solves the
  // small system from the partials of all blocks
  unsigned g_done;
};
// SPE difference table D_p and images L D_p, stored as float-float pairs (8 bytes per
// value, the buffers are FP64-sized): push the new solution w (FP64) and its image lw,
// form the block partials of the Galerkin products D_q . L D_p (q >= p) of the new
// table in hpart (4 tiles * ts_nblk() * kTileSlots 8-byte slots, float-float pairs) and
// factor H = D^T K D into fac (drop rule at eps_lin)
int spe_push(const MutVecSet& D, const MutVecSet& LD, const double* w, const double* lw, int m_old, int m_new,
             long long len, double* hpart, double eps_lin, SpeFac* fac, cudaStream_t st);
// the factor again from the partials in hpart (another eps_lin); nbh: the block count
// of the push that wrote them (spe_hblocks at that time)
int spe_factor(const double* hpart, int m, int nbh, double eps_lin, SpeFac* fac, cudaStream_t st);
// blocks of the product partials of a table of m columns (their layout in hpart), under
// the calling thread's launch cap
int spe_hblocks(long long len, int m);
// gpart needed: spe_gblocks() * kSpeGSlots 8-byte slots
int spe_gblocks();
// x0 (FP64) = Galerkin start from the table of m columns factored in fac: g = D^T b
// over the nsup layout indices sup, or (sup == nullptr) over the edges of the
// positions in bbox (b must vanish elsewhere; n is the grid size), the
// substitutions, x0 = D y
int spe_x0(const VecSet& D, int m, const double* b, int n, const Box& bbox, const int* sup, int nsup, double* x0,
           long long len, SpeFac* fac, double* gpart, double* coef, SmallOut* out, cudaStream_t st);
int pod_push(const VecSet& X, const double* w, const double* lw, int m, int slot_new, long long len, double* part,
             double* G, double* A, cudaStream_t st);
int pod_x0(const VecSet& X, int m, const double* G, const double* A, const double* b, double* x0, long long len,
           double eps_pod, double* part, double* coef, double* sigma, SmallOut* out, cudaStream_t st,
           const VecSet* LX = nullptr, double* r0 = nullptr);

// CSPE start vector (Sec. III, "cascaded SPE"): Galerkin projection of K_n x = b onto
// span(Q_1 .. Q_k, x) with Q K-orthonormal frozen past solutions (images P = L Q) and x
// the newest solution (lx = L x).  x is projected out against Q twice (vector-level
// Gram-Schmidt in the K inner product, with the stored images: no stencil), giving z and
// zeta = z.Lz; the new direction is dropped when zeta <= eps_lin^2 x.Lx.  Then
// x0 = Q (Q^T b) + z (z^T b) / zeta.  x0 may be the buffer x.
struct CspeBufs {
  double* const* Q;       // k frozen columns
  double* const* P;       // their images
  double *z, *lz, *z2, *lz2;
  double* scal;           // [2]: x.Lx, then 1/sqrt(zeta) (0 when the new direction is dropped)
};
int cspe_x0(const CspeBufs& cb, int k, const double* x, const double* lx, const double* b, double* x0,
            long long len, double eps_lin, double* part, double* coef, SmallOut* out, cudaStream_t st);
// freeze the projected newest solution of the last cspe_x0 as column k: Q_k = z / sqrt(zeta)
int cspe_freeze(const CspeBufs& cb, int k, long long len, cudaStream_t st);

}  // namespace mqs
