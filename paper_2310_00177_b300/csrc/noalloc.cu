// An allocation-free variant of the FP64 true-residual check
// (npsolve_true_residual_noalloc, declared in include/npsolve.h).
//
// npsolve_true_residual obtains its reduction scratch (one pair of FP64
// partial sums per thread block) with cudaMallocAsync.  Some callers cannot
// allocate device memory at the point where they check a solution: a
// simulation loop that reserves all of its GPU memory up front and forbids
// allocation inside a frame, or a plug-in whose host application owns the
// device memory.  This variant keeps the partial sums in a fixed device
// array of this file instead, so it calls no allocator at all.
//
// Limits and sharing: the array holds the partials of at most
// kNoAllocMaxBlocks blocks of kNAThreads threads that each cover
// kNACellsPerThread cells, i.e. grids of at most 16,777,216 cells (one
// 256^3 grid); larger grids are rejected with NPSOLVE_BAD_DIMS.  Every call
// on a device uses the same array and overwrites every entry it reads, so
// nothing has to be cleared between calls, but two calls whose work overlaps
// on the GPU (different streams, no ordering) race on it.  The first call on
// a device looks up the array's device address (cudaGetSymbolAddress) with
// that device current; make that first call before any stream capture.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>

#include <mutex>
#include <string>

#include "../../include/npsolve.h"
#include "nps_common.cuh"
#include "nps_kernels.h"

namespace {

constexpr int kNAThreads = 256;
constexpr int kNACellsPerThread = 8;
constexpr int kNoAllocMaxBlocks = 8192;
constexpr long long kNoAllocMaxCells = (long long)kNoAllocMaxBlocks * kNAThreads * kNACellsPerThread;  // 2^24
constexpr int kNoAllocMaxDevices = 64;

// Errors are reported through npsolve_last_error(NULL), like the other
// handle-less entry points.
int na_fail(int code, const char *fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  nps::set_thread_error(buf);
  return code;
}

}  // namespace

// Partial sums of ||b - A x||^2 and ||b||^2 per block, then the two reduced
// values at the end.
static __device__ __align__(256) double g_relres_scratch[2 * kNoAllocMaxBlocks + 2];

namespace {

std::mutex g_na_mutex;
double *g_na_ptr[kNoAllocMaxDevices] = {};

// Device address of g_relres_scratch on the current device (looked up once).
int scratch_for_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(NPSOLVE_CUDA_ERROR, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return na_fail(NPSOLVE_CUDA_ERROR, "device index %d unsupported", dev);
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    double *p = nullptr;
    e = cudaGetSymbolAddress((void **)&p, g_relres_scratch);
    if (e != cudaSuccess || !p)
      return na_fail(NPSOLVE_CUDA_ERROR, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_na_ptr[dev] = p;
  }
  *out = g_na_ptr[dev];
  return NPSOLVE_OK;
}

}  // namespace

// block_sum_store sizes its shared array for nps::kRedThreads threads.
static_assert(kNAThreads == nps::kRedThreads, "the partial-sum kernel runs kRedThreads threads per block");

// Per fluid cell the same FP64 operations, in the same order, as the
// library's true-residual kernel: (A x)_p = diag_p x_p - sum of the fluid
// neighbours' x (Sec. 3.2), res = b_p - fma(diag_p, x_p, -sum), and the
// squares accumulated with FMAs.  Only the order of the cross-thread
// reduction differs (this grid has its own block count), so the two results
// agree to FP64 rounding of the final sums.
__global__ void __launch_bounds__(kNAThreads) k_relres_partials_na(const uint8_t *__restrict__ lab, nps::Dims dm,
                                                                   const float *__restrict__ b,
                                                                   const double *__restrict__ x,
                                                                   double *__restrict__ part) {
  const long long n = dm.n();
  const long long sxy = (long long)dm.nx * dm.ny;
  double v[2] = {0.0, 0.0};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    int xx, yy, zz;
    nps::cell_xyz(p, dm, xx, yy, zz);
    if (lab[p] != nps::kFluid) continue;
    const long long nb[6] = {p - 1, p + 1, p - dm.nx, p + dm.nx, p - sxy, p + sxy};
    const bool ok[6] = {xx > 0, xx < dm.nx - 1, yy > 0, yy < dm.ny - 1, zz > 0, zz < dm.nz - 1};
    double sum = 0.0;
    int diag = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      if (!ok[k]) continue;
      const uint8_t ln = lab[nb[k]];
      if (ln == nps::kFluid) {
        sum += x[nb[k]];
        diag += 1;
      } else if (ln == nps::kAir) {
        diag += 1;
      }
    }
    const double bp = (double)b[p];
    const double res = bp - fma((double)diag, x[p], -sum);
    v[0] = fma(res, res, v[0]);
    v[1] = fma(bp, bp, v[1]);
  }
  nps::block_sum_store<2>(v, part + (size_t)blockIdx.x * 2);
}

__global__ void k_relres_final_na(const double *part, int nblocks, double *out) {
  double t[2];
  nps::reduce_partials<2>(part, nblocks, t);
  if (threadIdx.x != 0) return;
  out[0] = t[1] > 0.0 ? sqrt(t[0] / t[1]) : 0.0;
  out[1] = sqrt(t[1]);
}

extern "C" int npsolve_true_residual_noalloc(const uint8_t *labels, int nx, int ny, int nz, const float *b,
                                             const double *x, double *rel_residual, void *stream) {
  if (!labels || !b || !x || !rel_residual) return na_fail(NPSOLVE_BAD_ARG, "null pointer argument");
  if ((((uintptr_t)labels | (uintptr_t)b | (uintptr_t)x) & 15u) != 0)
    return na_fail(NPSOLVE_BAD_ARG, "device pointers must be 16-byte aligned");
  if (nx < 1 || ny < 1 || nz < 1) return na_fail(NPSOLVE_BAD_DIMS, "bad dims %dx%dx%d", nx, ny, nz);
  const long long n = (long long)nx * ny * nz;
  if (n > kNoAllocMaxCells)
    return na_fail(NPSOLVE_BAD_DIMS,
                   "grid of %lld cells exceeds the %lld-cell maximum of npsolve_true_residual_noalloc "
                   "(use npsolve_true_residual)",
                   n, kNoAllocMaxCells);
  double *scratch = nullptr;
  int st = scratch_for_current_device(&scratch);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const long long per_block = (long long)kNAThreads * kNACellsPerThread;
  const int nblocks = (int)((n + per_block - 1) / per_block);  // <= kNoAllocMaxBlocks by the check above
  // An error already pending on this thread belongs to earlier work: peek
  // (never clear) so that it stays with its owner, and take a launch error
  // as this call's only when nothing was pending before.
  const cudaError_t prior = cudaPeekAtLastError();
  k_relres_partials_na<<<nblocks, kNAThreads, 0, s>>>(labels, nps::Dims{nx, ny, nz}, b, x, scratch);
  k_relres_final_na<<<1, nps::kRedThreads, 0, s>>>(scratch, nblocks, scratch + 2 * kNoAllocMaxBlocks);
  double res[2] = {0.0, 0.0};
  cudaError_t e = cudaSuccess;
  if (prior == cudaSuccess) {
    e = cudaPeekAtLastError();
    if (e != cudaSuccess) (void)cudaGetLastError();  // this call's launch error: report it here
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(res, scratch + 2 * kNoAllocMaxBlocks, sizeof(res), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return na_fail(NPSOLVE_CUDA_ERROR, "true residual (no-alloc): %s", cudaGetErrorString(e));
  *rel_residual = res[0];
  return NPSOLVE_OK;
}
