// Stencil, vector and scalar kernels of the NPSDO iteration (Alg. 1) and of
// Jacobi-PCG: masked 7-point Laplacian (Sec. 3.2), A-orthogonalisation
// (Alg. 1 inner loop), exact line search and updates, FP64 reductions.
//
// Every iteration kernel first reads SolveState::done and returns when the
// solve has finished, so a fixed sequence of launches (or a CUDA graph) can
// run past convergence without changing the result.
#include "nps_common.cuh"
#include "nps_kernels.h"

namespace nps {

// ---------------------------------------------------------------------------
// Masked 7-point Laplacian, q = A d.  For a fluid cell
//   q_p = sum_{fluid n} (d_p - d_n) + (#air neighbours) d_p,
// which equals (#fluid-or-air neighbours) d_p - sum_{fluid n} d_n; the
// difference form keeps FP32 rounding proportional to the local variation of
// d rather than to |d|.  Non-fluid rows are zero.  Optional FP64 partial dot
// products d.q and r.d per block.
// ---------------------------------------------------------------------------
template <bool DOTS>
__global__ void __launch_bounds__(kRedThreads) k_lap(const uint8_t *__restrict__ lab, Dims dm,
                                                       const float *__restrict__ d, float *__restrict__ q,
                                                       const float *__restrict__ r, double *__restrict__ part,
                                                       const SolveState *st) {
  if (st && st->done) return;
  const long long n = dm.n();
  const long long sxy = (long long)dm.nx * dm.ny;
  double v[2] = {0.0, 0.0};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(p, dm, x, y, z);
    float out = 0.f;
    if (lab[p] == kFluid) {
      const float dp = d[p];
      float acc = 0.f;
      int nair = 0;
      const long long nb[6] = {p - 1, p + 1, p - dm.nx, p + dm.nx, p - sxy, p + sxy};
      const bool ok[6] = {x > 0, x < dm.nx - 1, y > 0, y < dm.ny - 1, z > 0, z < dm.nz - 1};
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        if (!ok[k]) continue;
        const uint8_t ln = lab[nb[k]];
        if (ln == kFluid) acc += dp - d[nb[k]];
        else if (ln == kAir) nair += 1;
      }
      out = acc + (float)nair * dp;
      if (DOTS) {
        v[0] += (double)dp * (double)out;
        v[1] += (double)r[p] * (double)dp;
      }
    }
    q[p] = out;
  }
  if (DOTS) block_sum_store<2>(v, part + (size_t)blockIdx.x * 2);
}

// r = mask(b) (FP32), x = 0, partial ||b||^2.
__global__ void __launch_bounds__(kRedThreads) k_init(const uint8_t *__restrict__ lab, long long n,
                                                        const float *__restrict__ b, float *__restrict__ r,
                                                        double *__restrict__ x, double *__restrict__ part) {
  double v[1] = {0.0};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    const float bv = lab[p] == kFluid ? b[p] : 0.f;
    r[p] = bv;
    x[p] = 0.0;
    v[0] += (double)bv * (double)bv;
  }
  block_sum_store<1>(v, part + blockIdx.x);
}

// Initial scalars: ||b||, the stopping threshold, the first input scale.
__global__ void k_init_final(const double *part, int nblocks, double tol, int max_iter, int n_ortho, int method,
                             SolveState *st, double *hist) {
  double t[1];
  reduce_partials<1>(part, nblocks, t);
  if (threadIdx.x != 0) return;
  SolveState s;
  s.bnorm2 = t[0];
  s.eps2 = tol * tol * t[0];
  s.rnorm2 = t[0];
  s.alpha = 0.0;
  for (int i = 0; i < kMaxOrtho; ++i) s.coef[i] = 0.0;
  for (int i = 0; i < kRing; ++i) s.dAd[i] = 1.0;
  s.k = 0;
  s.max_iter = max_iter;
  s.n_ortho = n_ortho;
  s.upd_pending = 0;
  s.x_upto = 0;
  for (int i = 0; i < kRing; ++i) s.alpha_slot[i] = 0.0;
  s.method = method;
  s.fresh = 1;
  s.sigma = 0.0;
  s.rscale = t[0] > 0.0 ? (float)(1.0 / sqrt(t[0])) : 0.f;
  if (!isfinite(t[0])) s.done = kDoneBadInput;
  else if (!(t[0] >= s.eps2) || t[0] == 0.0) s.done = kDoneConverged;  // ||r_0|| < tol ||b|| or b = 0
  else s.done = kDoneRunning;
  *st = s;
  hist[0] = sqrt(t[0]);
}

// Alg. 1 inner loop, classical Gram-Schmidt form: c_i = z^T (A d_i) / d_i^T A d_i
// for the previous directions i = max(1, k - n_ortho) .. k-1 (or the PCG /
// FPCG conjugation coefficient).  The partials hold the dots of z with the
// vectors of direction_dot_count (written by the level-1 combine kernel).
__global__ void k_ortho_final(const double *part, int nblocks, SolveState *st) {
  if (st->done) return;
  double t[kMaxOrtho];
  reduce_partials<kMaxOrtho>(part, nblocks, t);
  if (threadIdx.x != 0) return;
  set_direction_coefs(st, t, direction_dot_count(st->method, st->k + 1, st->n_ortho, kMaxOrtho));
}

// d_k = z - sum_j c_j d_{k-1-j}  (into ring slot of iteration k).
__global__ void __launch_bounds__(kRedThreads) k_direction(long long n, const float *__restrict__ zv,
                                                             float *__restrict__ dring, const SolveState *st) {
  if (st->done) return;
  const int k1 = st->k + 1, no = st->n_ortho;
  float c[kMaxOrtho];
  const float *src[kMaxOrtho];
  int cnt = 0;
  for (int i = k1 - 1; i >= k1 - no && i >= 1; --i) {
    c[cnt] = (float)st->coef[k1 - 1 - i];
    src[cnt] = dring + (size_t)ring_slot(i, no) * n;
    ++cnt;
  }
  float *dst = dring + (size_t)ring_slot(k1, no) * n;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    float v = zv[p];
    for (int j = 0; j < cnt; ++j) v -= c[j] * src[j][p];
    dst[p] = v;
  }
}

// q_k = A d_k with partials d.q and r.d, on the ring slot of iteration k.
__global__ void __launch_bounds__(kRedThreads) k_lap_ring(const uint8_t *__restrict__ lab, Dims dm,
                                                            const float *__restrict__ dring, float *__restrict__ qring,
                                                            const float *__restrict__ r, double *__restrict__ part,
                                                            const SolveState *st);

// alpha_k = r^T d_k / d_k^T A d_k (PCG / FPCG: sigma_k / d_k^T A d_k); breakdown
// when d^T A d <= 0 or non-finite.
__global__ void k_alpha_final(const double *part, int nblocks, SolveState *st) {
  if (st->done) return;
  double t[2];
  reduce_partials<2>(part, nblocks, t);
  if (threadIdx.x != 0) return;
  const double dq = t[0], rd = t[1];
  const int k1 = st->k + 1;
  if (!(dq > 0.0) || !isfinite(dq) || !isfinite(rd)) {
    st->done = kDoneBreakdown;
    return;
  }
  st->alpha = (st->method == kMethodNpsdo ? rd : st->sigma) / dq;
  st->dAd[ring_slot(k1, st->n_ortho)] = dq;
}

// x_k = x_{k-1} + alpha d_k (FP64); recurrence mode also r -= alpha q and the
// partial ||r||^2.
template <bool RECUR>
__global__ void __launch_bounds__(kRedThreads) k_update(long long n, double *__restrict__ x, float *__restrict__ r,
                                                          const float *__restrict__ dring,
                                                          const float *__restrict__ qring, double *__restrict__ part,
                                                          const SolveState *st) {
  if (st->done) return;
  const int k1 = st->k + 1;
  const int slot = ring_slot(k1, st->n_ortho);
  const float *d = dring + (size_t)slot * n;
  const float *q = qring + (size_t)slot * n;
  const double a = st->alpha;
  const float af = (float)a;
  double v[1] = {0.0};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    x[p] = fma(a, (double)d[p], x[p]);
    if (RECUR) {
      const float rn = fmaf(-af, q[p], r[p]);
      r[p] = rn;
      v[0] += (double)rn * (double)rn;
    }
  }
  if (RECUR) block_sum_store<1>(v, part + blockIdx.x);
}

// r = b - A x evaluated in FP64 (x FP64, b FP32), stored as FP32; partials of
// ||b - A x||^2 (FP64 values) and ||mask(b)||^2.  Used by the explicit
// residual mode, residual replacement and the final true-residual check.
// r (optional) receives b - A x; with r_alt, r_k's buffer by the parity of
// sel->k (the residual alternates between two buffers on the fused path).
__global__ void __launch_bounds__(kRedThreads) k_true_residual(const uint8_t *__restrict__ lab, Dims dm,
                                                                 const float *__restrict__ b,
                                                                 const double *__restrict__ x, float *r,
                                                                 float *r_alt, const SolveState *sel,
                                                                 double *__restrict__ part, const SolveState *st) {
  if (st && st->done) return;
  if (r_alt && sel && (sel->k & 1)) r = r_alt;
  const long long n = dm.n();
  const long long sxy = (long long)dm.nx * dm.ny;
  double v[2] = {0.0, 0.0};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    int xx, yy, zz;
    cell_xyz(p, dm, xx, yy, zz);
    double res = 0.0;
    if (lab[p] == kFluid) {
      // (A x)_p = (fluid + air neighbours) x_p - sum of the fluid neighbours' x
      // (Sec. 3.2): one FP64 add per fluid neighbour and one FMA, since B300's
      // FP64 rate bounds this kernel
      const long long nb[6] = {p - 1, p + 1, p - dm.nx, p + dm.nx, p - sxy, p + sxy};
      const bool ok[6] = {xx > 0, xx < dm.nx - 1, yy > 0, yy < dm.ny - 1, zz > 0, zz < dm.nz - 1};
      double sum = 0.0;
      int diag = 0;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        if (!ok[k]) continue;
        const uint8_t ln = lab[nb[k]];
        if (ln == kFluid) {
          sum += x[nb[k]];
          diag += 1;
        } else if (ln == kAir) {
          diag += 1;
        }
      }
      const double bp = (double)b[p];
      res = bp - fma((double)diag, x[p], -sum);
      v[0] = fma(res, res, v[0]);
      v[1] = fma(bp, bp, v[1]);
    }
    if (r) r[p] = (float)res;
  }
  block_sum_store<2>(v, part + (size_t)blockIdx.x * 2);
}

// End of an iteration: ||r_k||, history, stop test ||r_k|| < tol ||b||
// (Alg. 1 continues while ||r_k|| >= eps), next input scale.
// part_stride = 1 for the recurrence partials, 2 for k_true_residual's.
__global__ void k_converge_final(const double *part, int nblocks, int part_stride, SolveState *st, double *hist) {
  if (st->done) return;
  double t[2] = {0.0, 0.0};
  if (part_stride == 1) {
    double u[1];
    reduce_partials<1>(part, nblocks, u);
    t[0] = u[0];
  } else {
    reduce_partials<2>(part, nblocks, t);
  }
  if (threadIdx.x != 0) return;
  const double rr = t[0];
  st->k += 1;
  st->rnorm2 = rr;
  hist[st->k] = sqrt(rr);
  if (!isfinite(rr)) st->done = kDoneBreakdown;
  else if (rr < st->eps2 || rr == 0.0) st->done = kDoneConverged;
  else st->rscale = (float)(1.0 / sqrt(rr));
}

// After a residual replacement: take ||r||^2 from k_true_residual partials,
// re-open the iteration if it is still above tolerance.
__global__ void k_restart_final(const double *part, int nblocks, SolveState *st, int *reopened, double *relres) {
  double t[2];
  reduce_partials<2>(part, nblocks, t);
  if (threadIdx.x != 0) return;
  const double rr = t[0];
  // the same figures as k_relres_final: the final check when nothing re-opens
  relres[0] = t[1] > 0.0 ? sqrt(t[0] / t[1]) : 0.0;
  relres[1] = sqrt(t[1]);
  *reopened = 0;
  if (st->done != kDoneConverged) return;
  if (rr >= st->eps2 && rr > 0.0 && isfinite(rr)) {
    st->rnorm2 = rr;
    st->rscale = (float)(1.0 / sqrt(rr));
    st->done = kDoneRunning;
    st->fresh = 1;  // PCG / FPCG restart their conjugate sequence from the replaced residual
    *reopened = 1;
  }
}

// Final: relative true residual into out[0], ||b|| into out[1].
__global__ void k_relres_final(const double *part, int nblocks, double *out) {
  double t[2];
  reduce_partials<2>(part, nblocks, t);
  if (threadIdx.x != 0) return;
  out[0] = t[1] > 0.0 ? sqrt(t[0] / t[1]) : 0.0;
  out[1] = sqrt(t[1]);
}

__global__ void __launch_bounds__(kRedThreads) k_lap_ring(const uint8_t *__restrict__ lab, Dims dm,
                                                            const float *__restrict__ dring, float *__restrict__ qring,
                                                            const float *__restrict__ r, double *__restrict__ part,
                                                            const SolveState *st) {
  if (st->done) return;
  const int slot = ring_slot(st->k + 1, st->n_ortho);
  const long long n = dm.n();
  const float *d = dring + (size_t)slot * n;
  float *q = qring + (size_t)slot * n;
  const long long sxy = (long long)dm.nx * dm.ny;
  double v[2] = {0.0, 0.0};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(p, dm, x, y, z);
    float out = 0.f;
    if (lab[p] == kFluid) {
      const float dp = d[p];
      float acc = 0.f;
      int nair = 0;
      const long long nb[6] = {p - 1, p + 1, p - dm.nx, p + dm.nx, p - sxy, p + sxy};
      const bool ok[6] = {x > 0, x < dm.nx - 1, y > 0, y < dm.ny - 1, z > 0, z < dm.nz - 1};
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        if (!ok[k]) continue;
        const uint8_t ln = lab[nb[k]];
        if (ln == kFluid) acc += dp - d[nb[k]];
        else if (ln == kAir) nair += 1;
      }
      out = acc + (float)nair * dp;
      v[0] += (double)dp * (double)out;
      v[1] += (double)r[p] * (double)dp;
    }
    q[p] = out;
  }
  block_sum_store<2>(v, part + (size_t)blockIdx.x * 2);
}

// Label validation: counts codes > 2 into *bad.
__global__ void k_check_labels(const uint8_t *__restrict__ lab, long long n, unsigned int *bad) {
  unsigned int local = 0;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
    local |= lab[p] > 2 ? 1u : 0u;
  if (local) atomicOr(bad, 1u);
}

// ---------------------------------------------------------------------------
// Jacobi-PCG (textbook, M = diag(A) on fluid cells).
// ---------------------------------------------------------------------------
struct PcgState {
  double bnorm2, eps2, rz, alpha, beta, rnorm2;
  int k, done;
};

__device__ __forceinline__ float lap_diag_at(const uint8_t *lab, Dims dm, long long p, int x, int y, int z) {
  const long long sxy = (long long)dm.nx * dm.ny;
  int c = 0;
  if (x > 0) c += lab[p - 1] != kSolid;
  if (x < dm.nx - 1) c += lab[p + 1] != kSolid;
  if (y > 0) c += lab[p - dm.nx] != kSolid;
  if (y < dm.ny - 1) c += lab[p + dm.nx] != kSolid;
  if (z > 0) c += lab[p - sxy] != kSolid;
  if (z < dm.nz - 1) c += lab[p + sxy] != kSolid;
  return (float)c;
}

// r = mask(b), z = M^-1 r, p = z, x = 0; partials ||b||^2, r.z
__global__ void __launch_bounds__(kRedThreads) k_pcg_init(const uint8_t *__restrict__ lab, Dims dm,
                                                            const float *__restrict__ b, float *__restrict__ r,
                                                            float *__restrict__ pv, double *__restrict__ x,
                                                            double *__restrict__ part) {
  const long long n = dm.n();
  double v[2] = {0.0, 0.0};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    int xx, yy, zz;
    cell_xyz(p, dm, xx, yy, zz);
    float rv = 0.f, zv = 0.f;
    if (lab[p] == kFluid) {
      rv = b[p];
      const float dg = lap_diag_at(lab, dm, p, xx, yy, zz);
      zv = dg > 0.f ? rv / dg : 0.f;
    }
    r[p] = rv;
    pv[p] = zv;
    x[p] = 0.0;
    v[0] += (double)rv * rv;
    v[1] += (double)rv * zv;
  }
  block_sum_store<2>(v, part + (size_t)blockIdx.x * 2);
}

__global__ void k_pcg_init_final(const double *part, int nblocks, double tol, PcgState *st, double *hist) {
  double t[2];
  reduce_partials<2>(part, nblocks, t);
  if (threadIdx.x != 0) return;
  st->bnorm2 = t[0];
  st->eps2 = tol * tol * t[0];
  st->rz = t[1];
  st->rnorm2 = t[0];
  st->k = 0;
  st->done = (!isfinite(t[0])) ? kDoneBadInput : ((t[0] < st->eps2 || t[0] == 0.0) ? kDoneConverged : kDoneRunning);
  hist[0] = sqrt(t[0]);
}

// q = A p with partial p.q
__global__ void __launch_bounds__(kRedThreads) k_pcg_lap(const uint8_t *__restrict__ lab, Dims dm,
                                                           const float *__restrict__ pv, float *__restrict__ q,
                                                           double *__restrict__ part, const PcgState *st) {
  if (st->done) return;
  const long long n = dm.n();
  const long long sxy = (long long)dm.nx * dm.ny;
  double v[1] = {0.0};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(p, dm, x, y, z);
    float out = 0.f;
    if (lab[p] == kFluid) {
      const float dp = pv[p];
      float acc = 0.f;
      int nair = 0;
      const long long nb[6] = {p - 1, p + 1, p - dm.nx, p + dm.nx, p - sxy, p + sxy};
      const bool ok[6] = {x > 0, x < dm.nx - 1, y > 0, y < dm.ny - 1, z > 0, z < dm.nz - 1};
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        if (!ok[k]) continue;
        const uint8_t ln = lab[nb[k]];
        if (ln == kFluid) acc += dp - pv[nb[k]];
        else if (ln == kAir) nair += 1;
      }
      out = acc + (float)nair * dp;
      v[0] += (double)dp * out;
    }
    q[p] = out;
  }
  block_sum_store<1>(v, part + blockIdx.x);
}

__global__ void k_pcg_alpha(const double *part, int nblocks, PcgState *st) {
  if (st->done) return;
  double t[1];
  reduce_partials<1>(part, nblocks, t);
  if (threadIdx.x != 0) return;
  if (!(t[0] > 0.0) || !isfinite(t[0])) {
    st->done = kDoneBreakdown;
    return;
  }
  st->alpha = st->rz / t[0];
}

// x += alpha p; r -= alpha q; z = M^-1 r (kept in q's buffer); partials r.z, r.r
__global__ void __launch_bounds__(kRedThreads) k_pcg_update(const uint8_t *__restrict__ lab, Dims dm,
                                                              double *__restrict__ x, float *__restrict__ r,
                                                              const float *__restrict__ pv, float *__restrict__ q,
                                                              double *__restrict__ part, const PcgState *st) {
  if (st->done) return;
  const long long n = dm.n();
  const double a = st->alpha;
  const float af = (float)a;
  double v[2] = {0.0, 0.0};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    int xx, yy, zz;
    cell_xyz(p, dm, xx, yy, zz);
    x[p] = fma(a, (double)pv[p], x[p]);
    const float rn = fmaf(-af, q[p], r[p]);
    r[p] = rn;
    float zv = 0.f;
    if (lab[p] == kFluid) {
      const float dg = lap_diag_at(lab, dm, p, xx, yy, zz);
      zv = dg > 0.f ? rn / dg : 0.f;
    }
    q[p] = zv;
    v[0] += (double)rn * zv;
    v[1] += (double)rn * rn;
  }
  block_sum_store<2>(v, part + (size_t)blockIdx.x * 2);
}

__global__ void k_pcg_beta(const double *part, int nblocks, PcgState *st, double *hist) {
  if (st->done) return;
  double t[2];
  reduce_partials<2>(part, nblocks, t);
  if (threadIdx.x != 0) return;
  st->beta = t[0] / st->rz;
  st->rz = t[0];
  st->rnorm2 = t[1];
  st->k += 1;
  hist[st->k] = sqrt(t[1]);
  if (!isfinite(t[1])) st->done = kDoneBreakdown;
  else if (t[1] < st->eps2 || t[1] == 0.0) st->done = kDoneConverged;
}

// p = z + beta p
__global__ void __launch_bounds__(kRedThreads) k_pcg_dir(long long n, const float *__restrict__ zv,
                                                           float *__restrict__ pv, const PcgState *st) {
  if (st->done) return;
  const float bt = (float)st->beta;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
    pv[p] = fmaf(bt, pv[p], zv[p]);
}

// ---------------------------------------------------------------------------
// Host-side launchers.
// ---------------------------------------------------------------------------
void launch_lap(const uint8_t *lab, Dims dm, const float *d, float *q, cudaStream_t s) {
  k_lap<false><<<red_blocks(dm.n()), kRedThreads, 0, s>>>(lab, dm, d, q, nullptr, nullptr, nullptr);
}
void launch_check_labels(const uint8_t *lab, long long n, unsigned int *bad, cudaStream_t s) {
  k_check_labels<<<red_blocks(n), kRedThreads, 0, s>>>(lab, n, bad);
}
void launch_init(const uint8_t *lab, long long n, const float *b, float *r, double *x, double *part, double tol,
                 int max_iter, int n_ortho, int method, SolveState *st, double *hist, cudaStream_t s) {
  const int nb = red_blocks(n);
  k_init<<<nb, kRedThreads, 0, s>>>(lab, n, b, r, x, part);
  k_init_final<<<1, kRedThreads, 0, s>>>(part, nb, tol, max_iter, n_ortho, method, st, hist);
}
void launch_ortho_final(const double *part, long long n, SolveState *st, cudaStream_t s) {
  k_ortho_final<<<1, kRedThreads, 0, s>>>(part, red_blocks(n), st);
}
void launch_direction(long long n, const float *z, float *dring, const SolveState *st, cudaStream_t s) {
  k_direction<<<red_blocks(n), kRedThreads, 0, s>>>(n, z, dring, st);
}
void launch_lap_ring(const uint8_t *lab, Dims dm, const float *dring, float *qring, const float *r, double *part,
                     SolveState *st, cudaStream_t s) {
  const int nb = red_blocks(dm.n());
  k_lap_ring<<<nb, kRedThreads, 0, s>>>(lab, dm, dring, qring, r, part, st);
  k_alpha_final<<<1, kRedThreads, 0, s>>>(part, nb, st);
}
void launch_update(bool recurrence, long long n, double *x, float *r, const float *dring, const float *qring,
                   double *part, SolveState *st, double *hist, cudaStream_t s) {
  const int nb = red_blocks(n);
  if (recurrence) {
    k_update<true><<<nb, kRedThreads, 0, s>>>(n, x, r, dring, qring, part, st);
    k_converge_final<<<1, kRedThreads, 0, s>>>(part, nb, 1, st, hist);
  } else {
    k_update<false><<<nb, kRedThreads, 0, s>>>(n, x, r, dring, qring, part, st);
  }
}
void launch_explicit_residual(const uint8_t *lab, Dims dm, const float *b, const double *x, float *r, double *part,
                              SolveState *st, double *hist, cudaStream_t s) {
  const int nb = red_blocks(dm.n());
  k_true_residual<<<nb, kRedThreads, 0, s>>>(lab, dm, b, x, r, nullptr, nullptr, part, st);
  k_converge_final<<<1, kRedThreads, 0, s>>>(part, nb, 2, st, hist);
}
void launch_replace_residual(const uint8_t *lab, Dims dm, const float *b, const double *x, float *r, float *r_alt,
                             double *part, SolveState *st, int *reopened, double *relres, cudaStream_t s) {
  const int nb = red_blocks(dm.n());
  k_true_residual<<<nb, kRedThreads, 0, s>>>(lab, dm, b, x, r, r_alt, st, part, nullptr);
  k_restart_final<<<1, kRedThreads, 0, s>>>(part, nb, st, reopened, relres);
}
void launch_restart_final(const double *part, int nblocks, SolveState *st, int *reopened, double *relres,
                          cudaStream_t s) {
  k_restart_final<<<1, kRedThreads, 0, s>>>(part, nblocks, st, reopened, relres);
}
void launch_relres_final(const double *part, int nblocks, double *relres, cudaStream_t s) {
  k_relres_final<<<1, kRedThreads, 0, s>>>(part, nblocks, relres);
}
void launch_relres(const uint8_t *lab, Dims dm, const float *b, const double *x, double *part, double *out,
                   cudaStream_t s) {
  const int nb = red_blocks(dm.n());
  k_true_residual<<<nb, kRedThreads, 0, s>>>(lab, dm, b, x, nullptr, nullptr, nullptr, part, nullptr);
  k_relres_final<<<1, kRedThreads, 0, s>>>(part, nb, out);
}

size_t pcg_state_bytes() { return sizeof(PcgState); }
void launch_pcg_init(const uint8_t *lab, Dims dm, const float *b, float *r, float *p, double *x, double *part,
                     double tol, void *st, double *hist, cudaStream_t s) {
  const int nb = red_blocks(dm.n());
  k_pcg_init<<<nb, kRedThreads, 0, s>>>(lab, dm, b, r, p, x, part);
  k_pcg_init_final<<<1, kRedThreads, 0, s>>>(part, nb, tol, (PcgState *)st, hist);
}
void launch_pcg_iter(const uint8_t *lab, Dims dm, double *x, float *r, float *p, float *q, double *part, void *stv,
                     double *hist, cudaStream_t s) {
  PcgState *st = (PcgState *)stv;
  const int nb = red_blocks(dm.n());
  k_pcg_lap<<<nb, kRedThreads, 0, s>>>(lab, dm, p, q, part, st);
  k_pcg_alpha<<<1, kRedThreads, 0, s>>>(part, nb, st);
  k_pcg_update<<<nb, kRedThreads, 0, s>>>(lab, dm, x, r, p, q, part, st);
  k_pcg_beta<<<1, kRedThreads, 0, s>>>(part, nb, st, hist);
  k_pcg_dir<<<nb, kRedThreads, 0, s>>>(dm.n(), q, p, st);
}
int pcg_done_offset() { return (int)offsetof(PcgState, done); }
int pcg_k_offset() { return (int)offsetof(PcgState, k); }

}  // namespace nps
