// Shared device-side definitions of the npsolve CUDA library (sm_103a).
//
// Layout conventions (all vectors full-grid, x fastest):
//   p = (z*ny + y)*nx + x; labels uint8 0 solid, 1 fluid, 2 air; the region
//   outside the grid is solid (Sec. 3.1) and vectors are zero there (Sec. 4.2.1).
//   Level l of the network has dims (nx, ny, nz) >> (l-1); at l >= 2 the image
//   is stored as exact integer counts of fluid and air fine cells (ushort2),
//   the solid count being 8^(l-1) - fluid - air.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace nps {

// Division of 32-bit unsigned integers by a divisor fixed for a launch, by a
// multiply-high and shifts (Granlund and Montgomery, "Division by invariant
// integers using multiplication", 1994, Fig. 4.1): l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (t + ((n - t) >> 1)) >> (l - 1)
// with t = mulhi(m, n); d = 1 returns n.  Exact for every 32-bit n.
struct FastDiv {
  uint32_t d, m, s;
};
inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  f.s = l;
  f.m = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
  return f;
}
__device__ __forceinline__ uint32_t fdiv(const FastDiv &f, uint32_t n) {
  if (f.d == 1) return n;
  const uint32_t t = __umulhi(f.m, n);
  return (t + ((n - t) >> 1)) >> (f.s - 1);
}

constexpr int kSolid = 0, kFluid = 1, kAir = 2;
constexpr int kMaxLevels = 7;
constexpr int kMaxOrtho = 4;
constexpr int kMaxLanczos = 2048;  // Lanczos steps of the training right-hand-side generator
constexpr int kRing = kMaxOrtho + 1;
constexpr int kRedThreads = 256;   // threads of every reduction kernel
constexpr int kRedMaxBlocks = 1184; // 148 SMs x 8
constexpr int kMaxPartials = 8;    // quantities reduced per kernel

// Prepared weights of one CConv block (Sec. 4.2.1), folded with the fact that
// the image channels sum to one (Sec. 3.2): I_solid = 1 - I_fluid - I_air, so
//   K_a(p) = Bp[a] + sum_l ( Wf[a][l] nF(p+l) + Wa[a][l] nA(p+l) )
// with Wf = (W[a][fluid][l] - W[a][solid][l]) / 8^(lvl-1),
//      Wa = (W[a][air][l]   - W[a][solid][l]) / 8^(lvl-1),
//      Bp = B[a] + sum_l W[a][solid][l],
// and nF, nA the integer fluid/air counts (0/1 at level 1, 0 outside the grid).
struct CConvW {
  float wf[27][27];
  float wa[27][27];
  float bp[27];
};

// Per-level device copy of the Aff weights in the same folded form:
//   Aff = bconst + (1/(27 n)) sum_p sum_l ( wf[l] nF(p+l) + wa[l] nA(p+l) ).
struct AffW {
  float wf[27];
  float wa[27];
  double bconst;  // Bbar + (1/27) sum_l Wbar[solid][l]
};

// Device-resident state of one NPSDO solve (Alg. 1).  Written only by the
// single-block scalar kernels; read by every iteration kernel.
struct SolveState {
  double bnorm2;        // ||b||^2
  double eps2;          // (tol ||b||)^2: converged when ||r||^2 < eps2
  double rnorm2;        // ||r_k||^2
  double alpha;         // line-search step of the current iteration
  double coef[kMaxOrtho];  // orthogonalisation coefficients of the current iteration
  double dAd[kRing];    // d_i^T A d_i per ring slot
  float rscale;         // 1/||r_k||, the network input normalisation
  int k;                // completed iterations
  int done;             // 0 running, 1 converged, 2 breakdown, 3 non-finite input
  int max_iter;
  int n_ortho;
  int x_upto;           // steps 1..x_upto are in x (the recurrence mode adds several steps to x at once)
  int upd_pending;      // alpha of step k + 1 is known and r_{k+1} = r_k - alpha q not yet formed
  double alpha_slot[kRing];  // alpha of the step whose direction is in each ring slot
  // PCG / flexible PCG with the network as preconditioner (method != 0): the
  // ring holds two directions (n_ortho = 1) and the step uses sigma
  int method;           // kMethodNpsdo, kMethodPcg or kMethodFpcg
  int fresh;            // the next direction starts a new conjugate sequence (beta = 0)
  double sigma;         // r_k^T zhat_k of the current direction (zhat = P_net(r_k / ||r_k||))
};

enum { kDoneRunning = 0, kDoneConverged = 1, kDoneBreakdown = 2, kDoneBadInput = 3 };
enum { kMethodNpsdo = 0, kMethodPcg = 1, kMethodFpcg = 2 };

__host__ __device__ inline int ring_slot(int iter1, int n_ortho) { return (iter1 - 1) % (n_ortho + 1); }

// Vectors whose dot products with the network output z are taken before the
// direction is formed, for the iteration k1 = k + 1 being formed:
//   NPSDO: q_i = A d_i, i = k1-1, k1-2, ... (at most n_ortho, i >= 1) (Alg. 1);
//   PCG:   the current residual r_k (sigma = r_k^T z);
//   FPCG:  r_k and, from the second direction on, q_k = A d_k.
// Returns the count; entry j is the residual when dot_is_residual(st, j).
__host__ __device__ inline int direction_dot_count(int method, int k1, int n_ortho, int cap) {
  int c;
  if (method == kMethodNpsdo) c = n_ortho < k1 - 1 ? n_ortho : k1 - 1;
  else c = (method == kMethodFpcg && k1 > 1) ? 2 : 1;
  return c < cap ? c : cap;
}

// The coefficients of d_{k1} = z - sum_j coef[j] d_{k1-1-j} from the reduced
// dots t[] (the vectors above), on the single thread of a finishing block.
//   NPSDO (Alg. 1, classical Gram-Schmidt form): coef[j] = z^T A d_i / d_i^T A d_i.
//   PCG (preconditioned CG with z = ||r|| P_net(r / ||r||), the network being
//   linear in r, Sec. 4.2): beta = rho_k / rho_{k-1} with rho = r^T z.  With
//   zhat = P_net(r / ||r||) and the directions kept scaled by 1 / ||r_k||,
//   beta becomes sigma_k / sigma_{k-1} (sigma = r^T zhat), the step
//   alpha = sigma_k / dhat^T A dhat and x, r are unchanged.
//   FPCG (flexible PCG): beta = z_k^T (r_k - r_{k-1}) / rho_{k-1}; with
//   r_k - r_{k-1} = -alpha_k A d_k it is -alpha_k zhat^T q_k / sigma_{k-1}
//   in the scaled form.
// sigma = 0 or non-finite ends the solve as a breakdown (beta divides by it).
__device__ __forceinline__ void set_direction_coefs(SolveState *st, const double *t, int cnt) {
  const int k1 = st->k + 1, no = st->n_ortho;
  for (int j = 0; j < kMaxOrtho; ++j) st->coef[j] = 0.0;
  if (st->method == kMethodNpsdo) {
    for (int j = 0; j < cnt; ++j) st->coef[j] = t[j] / st->dAd[ring_slot(k1 - 1 - j, no)];
    return;
  }
  const double sig = t[0];
  if (!(sig != 0.0) || !isfinite(sig)) {
    st->done = kDoneBreakdown;
    return;
  }
  if (!st->fresh && k1 > 1) {
    const double beta = st->method == kMethodPcg ? sig / st->sigma : -st->alpha * t[1] / st->sigma;
    st->coef[0] = -beta;
  }
  st->fresh = 0;
  st->sigma = sig;
}

// ---------------------------------------------------------------------------
// Deterministic reductions: fixed grid, fixed tree, FP64 above the thread.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum NV per-thread values over the block (1-D block of kRedThreads) and
// store them at out[0..NV) (thread 0).
template <int NV>
__device__ __forceinline__ void block_sum_store(double (&v)[NV], double *out) {
  __shared__ double sm[NV][kRedThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) sm[i][warp] = v[i];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double t = lane < kRedThreads / 32 ? sm[i][lane] : 0.0;
      t = warp_sum(t);
      if (lane == 0) out[i] = t;
    }
  }
}

// Reduce `nblocks` rows of NV partials (row-major) inside one block of
// kRedThreads threads; every thread gets the totals in tot[].
template <int NV>
__device__ __forceinline__ void reduce_partials(const double *part, int nblocks, double (&tot)[NV]) {
  double v[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = 0.0;
  for (int j = threadIdx.x; j < nblocks; j += kRedThreads) {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] += part[(size_t)j * NV + i];
  }
  __shared__ double res[NV];
  block_sum_store<NV>(v, res);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) tot[i] = res[i];
}

inline int red_blocks(long long n) {
  long long b = (n + kRedThreads - 1) / kRedThreads;
  if (b > kRedMaxBlocks) b = kRedMaxBlocks;
  if (b < 1) b = 1;
  return (int)b;
}

struct Dims {
  int nx, ny, nz;
  __host__ __device__ long long n() const { return (long long)nx * ny * nz; }
};

// The x2 linear upsampling of Alg. 2 per axis (half-pixel centres, edge
// clamp): fine 2j = 0.25 c[j-1] + 0.75 c[j] (c[0] itself at j = 0), fine
// 2j+1 = 0.75 c[j] + 0.25 c[j+1] (c[n-1] for c[n]).  Written as explicit FMAs
// so that every kernel that interpolates rounds identically.
__device__ __forceinline__ float lerp_lo(float a, float b) { return fmaf(0.25f, a, 0.75f * b); }  // c[j-1], c[j]
__device__ __forceinline__ float lerp_hi(float b, float c) { return fmaf(0.75f, b, 0.25f * c); }  // c[j], c[j+1]

// Grids hold fewer than 2^31 cells, so the index arithmetic is 32-bit.
__device__ __forceinline__ void cell_xyz(long long p, const Dims &d, int &x, int &y, int &z) {
  const unsigned q = (unsigned)p, nx = (unsigned)d.nx, ny = (unsigned)d.ny;
  const unsigned t = q / nx;
  x = (int)(q - t * nx);
  y = (int)(t % ny);
  z = (int)(t / ny);
}

}  // namespace nps
