// Jacobi-PCG solve of K_n x = b that allocates no device memory.
//
// Some callers cannot call cudaMalloc: a host application whose device memory
// is owned entirely by its own pool allocator, or a real-time loop in which an
// allocation (which may synchronise the device) is not allowed.  This entry
// point serves them: the caller passes inputs and outputs, and every scratch
// vector lives in one file-scope device array of fixed size, reserved by every
// GPU that loads the library until the process exits.
#include <cuda.h>   // driver types only: the two driver calls below are looked up at run time
#include <cstdint>
#include <cstdio>
#include <mutex>
#include "mqs_kernels.h"

using namespace mqs;

namespace {

constexpr int kMaxN = MQS_NOALLOC_MAX_N;
constexpr long long kMaxLen = 3LL * kMaxN * kMaxN * kMaxN;          // doubles per layout vector
constexpr long long kFlagDoubles = ((long long)kMaxN * kMaxN * kMaxN + 7) / 8;
constexpr int kMaxBlocks = 512;
// r, p, q, L x, scaled b | 8 x kMaxBlocks partial sums | conductor flags | barrier, error, result
constexpr long long kOffR = 0, kOffP = kMaxLen, kOffQ = 2 * kMaxLen, kOffLx = 3 * kMaxLen, kOffB = 4 * kMaxLen;
constexpr long long kOffPart = 5 * kMaxLen;
constexpr long long kOffFlags = kOffPart + 8LL * kMaxBlocks;
constexpr long long kOffTail = kOffFlags + kFlagDoubles;
constexpr long long kScratchDoubles = kOffTail + 8;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

// The scratch array's device address, looked up once per CUDA context (the set-up of
// this entry point) with that context's device current.  Keyed by the driver's
// context ID, which is unique for the life of the process: after a device reset
// the primary context is a new one, so the address is looked up again instead of
// reusing one that may have moved.  The table is guarded by a mutex (host threads
// may make their first calls at the same time).
struct ScratchSlot {
  unsigned long long ctx_id;
  double* addr;
};
constexpr int kMaxContexts = 64;
std::mutex s_mu;
ScratchSlot s_slots[kMaxContexts];
int s_used = 0, s_next = 0;
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn s_get_current = nullptr;
CtxGetIdFn s_get_id = nullptr;

// bit c of flags[pos] set iff edge (c; pos) touches a conducting cell
__global__ void cell_flags_kernel(int n, const uint8_t* cell, uint8_t* flags) {
  const long long n3 = (long long)n * n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n3; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)((e / n) % n), k = (int)(e / ((long long)n * n));
    auto c = [&](int a, int b, int d) -> unsigned {
      if (a < 0 || b < 0 || d < 0 || a >= n || b >= n || d >= n) return 0u;
      return MQS_LDC(cell, a + (long long)n * (b + (long long)n * d), n3, 901) ? 1u : 0u;
    };
    unsigned f = 0u;
    if (c(i, j - 1, k - 1) | c(i, j, k - 1) | c(i, j - 1, k) | c(i, j, k)) f |= 1u;
    if (c(i - 1, j, k - 1) | c(i, j, k - 1) | c(i - 1, j, k) | c(i, j, k)) f |= 2u;
    if (c(i - 1, j - 1, k) | c(i, j - 1, k) | c(i - 1, j, k) | c(i, j, k)) f |= 4u;
    flags[e] = (uint8_t)f;
  }
}

// bs = (h/nu0) b on n-edges, 0 elsewhere; x zeroed off the n-edges
__global__ void prepare_kernel(Geom g, const double* b, double* bs, double* x, double s) {
  const long long len = 3 * g.n3;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e / g.n3);
    const long long pos = e - c * g.n3;
    const int i = (int)(pos % g.n), j = (int)((pos / g.n) % g.n), k = (int)(pos / ((long long)g.n * g.n));
    const bool on = (nmask(g, i, j, k) >> c) & 1u;
    bs[e] = on ? s * b[e] : 0.0;
    if (!on) x[e] = 0.0;
  }
}

// ID of the calling thread's current context; the runtime creates the device's
// primary context first if there is none yet.
int current_context(unsigned long long* id) {
  if (!s_get_current || !s_get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1{}, q2{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
      fprintf(stderr, "mqs_pcg_solve_noalloc: the driver does not provide cuCtxGetCurrent / cuCtxGetId\n");
      return MQS_ERR_CUDA;
    }
    s_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    s_get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext ctx = nullptr;
  if (s_get_current(&ctx) != CUDA_SUCCESS) return MQS_ERR_CUDA;
  if (!ctx) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess) return MQS_ERR_CUDA;
    if (s_get_current(&ctx) != CUDA_SUCCESS || !ctx) return MQS_ERR_CUDA;
  }
  return s_get_id(ctx, id) == CUDA_SUCCESS ? MQS_OK : MQS_ERR_CUDA;
}

// The scratch address in the current context (set-up on the first call in it).
int scratch_address(double** out) {
  std::lock_guard<std::mutex> lock(s_mu);
  unsigned long long id = 0;
  const int rc = current_context(&id);
  if (rc != MQS_OK) return rc;
  for (int q = 0; q < s_used; ++q)
    if (s_slots[q].ctx_id == id) {
      *out = s_slots[q].addr;
      return MQS_OK;
    }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess || p == nullptr) {
    fprintf(stderr, "mqs_pcg_solve_noalloc: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
    return MQS_ERR_CUDA;
  }
  ScratchSlot& slot = s_used < kMaxContexts ? s_slots[s_used++] : s_slots[s_next++ % kMaxContexts];
  slot.ctx_id = id;
  slot.addr = static_cast<double*>(p);
  *out = slot.addr;
  return MQS_OK;
}

}  // namespace

extern "C" int mqs_pcg_solve_noalloc(int n, double h, double nu0, const uint8_t* cell_mask_dev, const double* b_dev,
                                     double* x_dev, double tol, int maxit, mqs_pcg_info* info, void* stream) {
  if (n < 2 || n > kMaxN) {
    fprintf(stderr, "mqs_pcg_solve_noalloc: n = %d outside [2, %d] (the static scratch size)\n", n, kMaxN);
    return MQS_ERR_ARG;
  }
  if (!(h > 0.0) || !(nu0 > 0.0) || !(tol > 0.0) || maxit < 1 || !cell_mask_dev || !b_dev || !x_dev)
    return MQS_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(x_dev) % 16 != 0 || reinterpret_cast<uintptr_t>(b_dev) % 8 != 0) {
    fprintf(stderr, "mqs_pcg_solve_noalloc: x_dev must be 16-byte and b_dev 8-byte aligned\n");
    return MQS_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != MQS_OK) return rc;
  int nblk = 0;
  rc = pcg_max_blocks(&nblk);
  if (rc != MQS_OK) return rc;
  if (nblk > kMaxBlocks / 2) nblk = kMaxBlocks / 2;   // large grids launch two blocks per SM
  uint8_t* flags = reinterpret_cast<uint8_t*>(base + kOffFlags);
  unsigned* bar = reinterpret_cast<unsigned*>(base + kOffTail);
  int* err = reinterpret_cast<int*>(base + kOffTail + 1);
  PcgResult* res = reinterpret_cast<PcgResult*>(base + kOffTail + 2);
  DevGeom dg{};
  dg.g.n = n;
  dg.g.n3 = (long long)n * n * n;
  for (int a = 0; a < 3; ++a) { dg.g.cb_lo[a] = 0; dg.g.cb_hi[a] = n; }
  dg.g.cflags = flags;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MQS_ERR_CUDA;
  const int eb = 2 * nsm;   // element-wise helpers: two blocks per SM
  cell_flags_kernel<<<eb, 256, 0, st>>>(n, cell_mask_dev, flags);
  prepare_kernel<<<eb, 256, 0, st>>>(dg.g, b_dev, base + kOffB, x_dev, h / nu0);
  if (cudaGetLastError() != cudaSuccess) return MQS_ERR_CUDA;
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return MQS_ERR_CUDA;
  rc = launch_pcg(dg, base + kOffB, x_dev, base + kOffR, base + kOffP, base + kOffQ, base + kOffLx,
                  base + kOffPart, bar, err, res, tol, maxit, nblk, st);
  if (rc != MQS_OK) return rc;
  PcgResult pr{};
  int derr = 0;
  if (cudaMemcpyAsync(&pr, res, sizeof(pr), cudaMemcpyDeviceToHost, st) != cudaSuccess) return MQS_ERR_CUDA;
  if (cudaMemcpyAsync(&derr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return MQS_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MQS_ERR_CUDA;
  if (info) {
    info->iterations = pr.iterations;
    info->status = pr.status;
    info->relres = pr.relres;
    info->start_relres = pr.start_relres;
  }
  if (derr != 0) return derr;
  return pr.status;
}

namespace mqs {
MQS_DEBUG_TAKE(noalloc)
}  // namespace mqs
