// Start-vector kernels (Sec. III): SPE difference table and POD snapshots.
#pragma once
#include "mqs_internal.cuh"

namespace mqs {

constexpr int kMaxSpe = 16;
constexpr int kMaxPod = 40;
constexpr int kMaxVec = 40;
constexpr int kTileSlots = 72;      // 8 x 8 products + 8 right-hand side products

struct VecSet { const double* v[kMaxVec]; };
struct MutVecSet { double* v[kMaxVec]; };
struct SmallOut { int rank; int pad; double info; };

int ts_nblk();
// partial-sum buffer needed: 5 tiles * ts_nblk() * kTileSlots doubles
int spe_push(const MutVecSet& D, const MutVecSet& LD, const double* w, const double* lw, int m_old, int m_new,
             long long len, cudaStream_t st);
// x0 = Galerkin start; if r0 is given also r0 = b - L x0 from the stored images
int spe_x0(const VecSet& D, const VecSet& LD, int m, const double* b, double* x0, long long len, double eps_lin,
           double* part, double* coef, SmallOut* out, cudaStream_t st, double* r0 = nullptr);
int pod_push(const VecSet& X, const double* w, const double* lw, int m, int slot_new, long long len, double* part,
             double* G, double* A, cudaStream_t st);
int pod_x0(const VecSet& X, int m, const double* G, const double* A, const double* b, double* x0, long long len,
           double eps_pod, double* part, double* coef, double* sigma, SmallOut* out, cudaStream_t st,
           const VecSet* LX = nullptr, double* r0 = nullptr);

}  // namespace mqs
