// Bandwidth-oriented versions of the per-iteration vector / stencil kernels
// of Alg. 1 for grids with nx % 4 == 0 (every grid the network accepts for
// L >= 3): each thread handles groups of 4 consecutive cells along x with
// 16-byte loads and stores, 32-bit indexing, and no division per cell.
//
// Dot products: each thread sums the 4 products of a group in FP32 and adds
// the group sum into a double-float (hi + lo FP32 pair, error-free TwoSum)
// accumulator; the block reduction is FP64.  This keeps FP64 instructions
// (slow on B300) out of the per-cell path while giving FP64-quality sums.
//
// Each reduction kernel ends with a last-block-done step: the block that
// finishes last (atomic ticket after a memory fence) reduces the per-block
// partials in a fixed order and updates the solver scalars itself, so no
// separate single-block kernel is launched and the result is deterministic.
#include "nps_common.cuh"
#include "nps_kernels.h"

namespace nps {

namespace {

struct DF {
  float hi = 0.f, lo = 0.f;
};
__device__ __forceinline__ void df_add(DF &a, float b) {
  const float s = a.hi + b;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b - bb);
  a.hi = s;
  a.lo += e;
}
__device__ __forceinline__ double df_val(const DF &a) { return (double)a.hi + (double)a.lo; }

// Partials of the grid are reduced by the last block (fixed order, FP64).
template <int NV>
__device__ __forceinline__ void reduce_partials_cg(const double *part, int nblocks, double (&tot)[NV]) {
  double v[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = 0.0;
  for (int j = threadIdx.x; j < nblocks; j += kRedThreads) {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] += __ldcg(part + (size_t)j * NV + i);
  }
  __shared__ double res[NV];
  block_sum_store<NV>(v, res);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) tot[i] = res[i];
}

// Store this block's partials; the last block to arrive reduces all of them
// and calls finish(tot) on thread 0, then re-arms the ticket counter.
template <int NV, class F>
__device__ __forceinline__ void reduce_and_finish(double (&v)[NV], double *part, unsigned *ticket, F finish) {
  block_sum_store<NV>(v, part + (size_t)blockIdx.x * NV);
  __shared__ unsigned s_last;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    s_last = (t == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    double tot[NV];
    reduce_partials_cg<NV>(part, gridDim.x, tot);
    if (threadIdx.x == 0) {
      finish(tot);
      *ticket = 0u;
    }
  }
}

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ uchar4 ldl4(const uint8_t *p) { return *reinterpret_cast<const uchar4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float f4(const float4 &v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }

constexpr int kThreads = 256;
inline int grid4(long long n4, int num_sms, int per_sm = 8) {
  long long b = (n4 + kThreads - 1) / kThreads;
  long long cap = (long long)num_sms * per_sm;  // one wave: the loops are grid-strided
  if (cap > kRedMaxBlocks) cap = kRedMaxBlocks;  // the partials buffer holds kRedMaxBlocks rows
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

// Resident blocks per SM of a kernel (looked up once per kernel).
template <auto F>
int resident_blocks() {
  static int per_sm = 0;
  if (!per_sm) {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, F, kThreads, 0);
    per_sm = b < 1 ? 1 : b;
  }
  return per_sm;
}

}  // namespace

// ---------------------------------------------------------------------------
// r = mask(b), x = 0, ||b||^2 -> initial solver scalars.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_init4(const uint8_t *__restrict__ lab, int n, const float *__restrict__ b,
                                                    float *__restrict__ r, double *__restrict__ x,
                                                    float *__restrict__ xhi, float *__restrict__ xlo,
                                                    double *__restrict__ part, unsigned *ticket, double tol,
                                                    int max_iter, int n_ortho, int method, SolveState *st,
                                                    double *hist) {
  DF acc;
  const int n4 = n >> 2;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n4; g += gridDim.x * blockDim.x) {
    const int p = g << 2;
    const uchar4 l = ldl4(lab + p);
    const float4 bv = ld4(b + p);
    const float4 rv = make_float4(l.x == kFluid ? bv.x : 0.f, l.y == kFluid ? bv.y : 0.f, l.z == kFluid ? bv.z : 0.f,
                                  l.w == kFluid ? bv.w : 0.f);
    st4(r + p, rv);
    if (xhi) {
      st4(xhi + p, make_float4(0.f, 0.f, 0.f, 0.f));
      st4(xlo + p, make_float4(0.f, 0.f, 0.f, 0.f));
    } else {
      reinterpret_cast<double2 *>(x + p)[0] = make_double2(0.0, 0.0);
      reinterpret_cast<double2 *>(x + p)[1] = make_double2(0.0, 0.0);
    }
    df_add(acc, rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w);
  }
  double v[1] = {df_val(acc)};
  reduce_and_finish<1>(v, part, ticket, [&](const double *t) {
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
    else if (!(t[0] >= s.eps2) || t[0] == 0.0) s.done = kDoneConverged;
    else s.done = kDoneRunning;
    *st = s;
    hist[0] = sqrt(t[0]);
  });
}

// ---------------------------------------------------------------------------
// Level-1 combination z = mask_fluid(c1 x1 + c2 x2) with the dot products
// z . (A d_i) of the previous directions; the last block turns them into the
// orthogonalisation coefficients c_i = z^T A d_i / d_i^T A d_i (Alg. 1).  For
// PCG / FPCG the dots are r_k . z and q_k . z (r_k in r0, or in r0 / r1 by
// the parity of k when the residual alternates between two buffers).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_combine1_4(const uint8_t *__restrict__ lab, int n,
                                                         const float *__restrict__ x1, const float *__restrict__ x2,
                                                         const double *__restrict__ c12, float *__restrict__ z,
                                                         const float *__restrict__ qring, const float *r0,
                                                         const float *r1, double *__restrict__ part,
                                                         unsigned *ticket, SolveState *st) {
  if (st->done) return;
  const float c1 = (float)c12[0], c2 = (float)c12[1];
  const int k1 = st->k + 1, no = st->n_ortho;
  // q of the previous directions i = k1-1-j (j < no, i >= 1), each without dynamic indexing
  const int cnt = direction_dot_count(st->method, k1, no, kMaxOrtho);
  const bool pcg = st->method != kMethodNpsdo;
  const float *q0 = pcg ? ((r1 && (st->k & 1)) ? r1 : r0) : qring + (size_t)ring_slot(max(k1 - 1, 1), no) * n;
  const float *q1 = qring + (size_t)ring_slot(max(k1 - (pcg ? 1 : 2), 1), no) * n;
  const float *q2 = qring + (size_t)ring_slot(max(k1 - 3, 1), no) * n;
  const float *q3 = qring + (size_t)ring_slot(max(k1 - 4, 1), no) * n;
  DF acc[kMaxOrtho];
  const int n4 = n >> 2;
  const int stride = gridDim.x * blockDim.x;
  auto group = [&](int g) {
    const int p = g << 2;
    const uchar4 l = ldl4(lab + p);
    const float4 a = ld4(x1 + p), b = ld4(x2 + p);
    float4 qv[kMaxOrtho];
    qv[0] = cnt > 0 ? ld4(q0 + p) : make_float4(0.f, 0.f, 0.f, 0.f);
    qv[1] = cnt > 1 ? ld4(q1 + p) : make_float4(0.f, 0.f, 0.f, 0.f);
    qv[2] = cnt > 2 ? ld4(q2 + p) : make_float4(0.f, 0.f, 0.f, 0.f);
    qv[3] = cnt > 3 ? ld4(q3 + p) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 zv = make_float4(l.x == kFluid ? fmaf(c1, a.x, c2 * b.x) : 0.f,
                                  l.y == kFluid ? fmaf(c1, a.y, c2 * b.y) : 0.f,
                                  l.z == kFluid ? fmaf(c1, a.z, c2 * b.z) : 0.f,
                                  l.w == kFluid ? fmaf(c1, a.w, c2 * b.w) : 0.f);
    st4(z + p, zv);
#pragma unroll
    for (int j = 0; j < kMaxOrtho; ++j)
      if (j < cnt) df_add(acc[j], zv.x * qv[j].x + zv.y * qv[j].y + zv.z * qv[j].z + zv.w * qv[j].w);
  };
  // two groups per iteration: twice the loads in flight per thread
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  for (; g + stride < n4; g += 2 * stride) {
    group(g);
    group(g + stride);
  }
  if (g < n4) group(g);
  double v[kMaxOrtho];
#pragma unroll
  for (int j = 0; j < kMaxOrtho; ++j) v[j] = df_val(acc[j]);
  reduce_and_finish<kMaxOrtho>(v, part, ticket, [&](const double *t) { set_direction_coefs(st, t, cnt); });
}

// x += a d for x held as a double-float pair (hi, lo) (|lo| <= ulp(hi) / 2,
// about 48 significant bits) and a = ah + al split into two floats: the
// product by the exact FMA product error, the sum by TwoSum, then one
// renormalisation (Dekker / Knuth).  B300 runs FP32 at 64 times its FP64
// rate, so this keeps the per-cell FP64 arithmetic off the iteration.
// (The _rn intrinsics keep the compiler from contracting a product into the
// error-free sums, which would break them.)
__device__ __forceinline__ void df_axpy(float &hi, float &lo, float ah, float al, float d) {
  const float ph = __fmul_rn(ah, d);
  const float pl = fmaf(al, d, fmaf(ah, d, -ph));
  const float s = __fadd_rn(hi, ph);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(ph, bb)), __fadd_rn(lo, pl));
  hi = __fadd_rn(s, e);
  lo = __fsub_rn(e, __fsub_rn(hi, s));
}

__device__ __forceinline__ void df_axpy4(float4 &hi, float4 &lo, float ah, float al, const float4 &d) {
  df_axpy(hi.x, lo.x, ah, al, d.x);
  df_axpy(hi.y, lo.y, ah, al, d.y);
  df_axpy(hi.z, lo.z, ah, al, d.z);
  df_axpy(hi.w, lo.w, ah, al, d.w);
}

__device__ __forceinline__ void split_alpha(double a, float &ah, float &al) {
  ah = (float)a;
  al = (float)(a - (double)ah);
}

// d_k = z - sum_j c_j d_{k-1-j} (Alg. 1's A-orthogonalisation against the last
// n_ortho directions).  DEFER (recurrence mode): x is not read during the
// iterations, so the steps alpha_i d_i are added to x (a double-float pair)
// here, R = n_ortho + 1 of them at once, when the ring slot that d_k
// overwrites still holds a pending step: x += alpha_{k-R} d_{k-R} + ... +
// alpha_{k-1} d_{k-1}, oldest first.  The directions d_{k-1} .. d_{k-n_ortho}
// are read for the orthogonalisation anyway and d_{k-R} is the old content
// of the slot being written, so the steps cost x's read and write once every
// R iterations.  The lap kernel's last block records the flush (x_upto)
// after every block here has read the state.
template <bool DEFER, int NO>
__global__ void __launch_bounds__(kThreads) k_direction4(int n, const float *__restrict__ zv, float *__restrict__ dring,
                                                         float *__restrict__ xhi, float *__restrict__ xlo,
                                                         const uint32_t *__restrict__ gmask, const SolveState *st) {
  if (st->done) return;
  constexpr int NA = NO > 0 ? NO : 1;  // array extents (n_ortho is a template argument)
  const int k1 = st->k + 1, no = NO;
  const int cnt = min(no, k1 - 1);
  const bool flush = DEFER && (k1 - 1) - st->x_upto == no + 1;  // then cnt == no
  float c[NA];
  const float *src[NA];
#pragma unroll
  for (int j = 0; j < NA; ++j) {
    c[j] = j < cnt ? (float)st->coef[j] : 0.f;
    src[j] = dring + (size_t)ring_slot(max(k1 - 1 - j, 1), no) * n;
  }
  float *dst = dring + (size_t)ring_slot(k1, no) * n;
  const int n4 = n >> 2;
  const int stride = gridDim.x * blockDim.x;
  auto ortho = [&](int p, float4 (&sv)[NA]) {
    float4 v = ld4(zv + p);
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      if (j < cnt) {
        sv[j] = ld4(src[j] + p);
        v.x -= c[j] * sv[j].x;
        v.y -= c[j] * sv[j].y;
        v.z -= c[j] * sv[j].z;
        v.w -= c[j] * sv[j].w;
      }
    }
    return v;
  };
  if (DEFER && flush) {
    // one group at a time, so that the flush path does not raise the
    // kernel's register count (the common path keeps two groups in flight)
    float ah[NA], al[NA], oh, ol;  // oh, ol: step k - R, whose direction is in d_k's slot
#pragma unroll
    for (int j = 0; j < NA; ++j) split_alpha(j < cnt ? st->alpha_slot[ring_slot(k1 - 1 - j, no)] : 0.0, ah[j], al[j]);
    split_alpha(st->alpha_slot[ring_slot(k1, no)], oh, ol);
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n4; g += stride) {
      const int p = g << 2;
      if (!((__ldg(gmask + (g >> 5)) >> (g & 31)) & 1u)) {  // no fluid: z, d and x are zero there
        st4(dst + p, make_float4(0.f, 0.f, 0.f, 0.f));
        continue;
      }
      float4 sv[NA];
      const float4 v = ortho(p, sv);
      const float4 dold = ld4(dst + p);
      float4 h = ld4(xhi + p), l = ld4(xlo + p);
      df_axpy4(h, l, oh, ol, dold);
#pragma unroll
      for (int j = NA - 1; j >= 0; --j)
        if (j < cnt) df_axpy4(h, l, ah[j], al[j], sv[j]);
      st4(xhi + p, h);
      st4(xlo + p, l);
      st4(dst + p, v);
    }
    return;
  }
  auto group = [&](int g) {
    const int p = g << 2;
    if (!((__ldg(gmask + (g >> 5)) >> (g & 31)) & 1u)) {  // no fluid: z and the d_i are zero there
      st4(dst + p, make_float4(0.f, 0.f, 0.f, 0.f));
      return;
    }
    float4 sv[NA];
    st4(dst + p, ortho(p, sv));
  };
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  for (; g + stride < n4; g += 2 * stride) {
    group(g);
    group(g + stride);
  }
  if (g < n4) group(g);
}


// Per-cell stencil code of the masked 7-point Laplacian (Sec. 3.2), built once
// per solve from the labels: bits 0-5 = the neighbour -x, +x, -y, +y, -z, +z
// is fluid (inside the grid), bits 8-10 = number of air neighbours, bit 15 =
// the cell itself is fluid.  With it, one bit per 4-cell group (bit g & 31 of
// word g >> 5 of gmask): the group holds a fluid cell; vectors are zero on
// the other groups, so the direction kernel skips their loads (occupancy-aware
// sparsity).  A thread codes a 4-cell group (nx % 4 == 0) from one 4-byte
// label load per row (the group, y +- 1, z +- 1) and the two x-neighbours; the
// mask word comes from a warp ballot.  Outside the grid is solid.
__global__ void __launch_bounds__(kThreads) k_lap_codes4(const uint8_t *__restrict__ lab, Dims dm,
                                                         uint16_t *__restrict__ code, uint32_t *__restrict__ gmask) {
  const int nx = dm.nx, ny = dm.ny, nz = dm.nz;
  const int nxy = nx * ny, n4 = (nx * ny * nz) >> 2, words = (n4 + 31) >> 5;
  const uchar4 solid4 = make_uchar4(0, 0, 0, 0);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < words * 32; g += gridDim.x * blockDim.x) {
    bool f = false;
    if (g < n4) {
      const int p = g << 2;
      const int yz = p / nx, x0 = p - yz * nx, z = yz / ny, y = yz - z * ny;
      const uchar4 lc = ldl4(lab + p);
      const uchar4 ym = y > 0 ? ldl4(lab + p - nx) : solid4, yp = y < ny - 1 ? ldl4(lab + p + nx) : solid4;
      const uchar4 zm = z > 0 ? ldl4(lab + p - nxy) : solid4, zp = z < nz - 1 ? ldl4(lab + p + nxy) : solid4;
      const uint8_t xl = x0 > 0 ? lab[p - 1] : (uint8_t)0, xr = x0 + 4 < nx ? lab[p + 4] : (uint8_t)0;
      const uint8_t c4[4] = {lc.x, lc.y, lc.z, lc.w};
      const uint8_t m4[4] = {ym.x, ym.y, ym.z, ym.w}, p4[4] = {yp.x, yp.y, yp.z, yp.w};
      const uint8_t zm4[4] = {zm.x, zm.y, zm.z, zm.w}, zp4[4] = {zp.x, zp.y, zp.z, zp.w};
      uint16_t out[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        uint32_t c = 0;
        if (c4[e] == kFluid) {
          const uint8_t nb[6] = {e == 0 ? xl : c4[e - 1], e == 3 ? xr : c4[e + 1], m4[e], p4[e], zm4[e], zp4[e]};
          uint32_t nair = 0;
          c = 0x8000u;
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            if (nb[k] == kFluid) c |= 1u << k;
            else if (nb[k] == kAir) nair += 1;
          }
          c |= nair << 8;
          f = true;
        }
        out[e] = (uint16_t)c;
      }
      *reinterpret_cast<ushort4 *>(code + p) = make_ushort4(out[0], out[1], out[2], out[3]);
    }
    const uint32_t bm = __ballot_sync(0xffffffffu, f);
    if ((threadIdx.x & 31) == 0) gmask[g >> 5] = bm;
  }
}

// q_k = A d_k (masked 7-point Laplacian, difference form: sum over the fluid
// neighbours n of (d_p - d_n), plus d_p per air neighbour, 0 off fluid) with
// the dot products d.q and r.d; the last block computes the line search
// alpha = r^T d / d^T A d and flags breakdown (d^T A d <= 0 or non-finite).
__global__ void __launch_bounds__(kThreads) k_lap4(const uint16_t *__restrict__ code, Dims dm, FastDiv dnx,
                                                   FastDiv dny, const float *__restrict__ dring,
                                                   float *__restrict__ qring, const float *__restrict__ r0,
                                                   const float *__restrict__ r1, double *__restrict__ part,
                                                   unsigned *ticket, SolveState *st) {
  if (st->done) return;
  const float *__restrict__ r = (r1 && (st->k & 1)) ? r1 : r0;  // r_k (two buffers: r_k in buffer k mod 2)
  const int nx = dm.nx, ny = dm.ny, nz = dm.nz;
  const int n = nx * ny * nz, nxy = nx * ny;
  const int slot = ring_slot(st->k + 1, st->n_ortho);
  const float *d = dring + (size_t)slot * n;
  float *q = qring + (size_t)slot * n;
  DF a0, a1;
  const int n4 = n >> 2;
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  auto group = [&](int g) {
    const int p = g << 2;
    const ushort4 cc = *reinterpret_cast<const ushort4 *>(code + p);
    if (((cc.x | cc.y | cc.z | cc.w) & 0x8000u) == 0u) {
      st4(q + p, zero4);
      return;
    }
    const int yz = (int)fdiv(dnx, (uint32_t)p);  // p / nx, (p / nx) / ny without the divide sequence
    const int x0 = p - yz * nx;
    const int z = (int)fdiv(dny, (uint32_t)yz);
    const int y = yz - z * ny;
    const float4 dc = ld4(d + p);
    const float dxl = x0 > 0 ? d[p - 1] : 0.f;
    const float dxr = x0 + 4 < nx ? d[p + 4] : 0.f;
    const float4 dym = y > 0 ? ld4(d + p - nx) : zero4, dyp = y < ny - 1 ? ld4(d + p + nx) : zero4;
    const float4 dzm = z > 0 ? ld4(d + p - nxy) : zero4, dzp = z < nz - 1 ? ld4(d + p + nxy) : zero4;
    const float4 rv = ld4(r + p);
    const uint16_t cs[4] = {cc.x, cc.y, cc.z, cc.w};
    float qo[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const uint32_t c = cs[e];
      const float dp = f4(dc, e);
      const float nv[6] = {e == 0 ? dxl : f4(dc, e - 1), e == 3 ? dxr : f4(dc, e + 1), f4(dym, e), f4(dyp, e),
                           f4(dzm, e), f4(dzp, e)};
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if (c & (1u << k)) acc += dp - nv[k];
      qo[e] = (c & 0x8000u) ? acc + (float)((c >> 8) & 7u) * dp : 0.f;
    }
    const float4 qv = make_float4(qo[0], qo[1], qo[2], qo[3]);
    st4(q + p, qv);
    df_add(a0, dc.x * qv.x + dc.y * qv.y + dc.z * qv.z + dc.w * qv.w);
    df_add(a1, rv.x * dc.x + rv.y * dc.y + rv.z * dc.z + rv.w * dc.w);
  };
  const int stride = gridDim.x * blockDim.x;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  for (; g + stride < n4; g += 2 * stride) {
    group(g);
    group(g + stride);
  }
  if (g < n4) group(g);
  double v[2] = {df_val(a0), df_val(a1)};
  reduce_and_finish<2>(v, part, ticket, [&](const double *t) {
    const double dq = t[0], rd = t[1];
    const int k1 = st->k + 1;
    if ((k1 - 1) - st->x_upto == st->n_ortho + 1) st->x_upto = k1 - 1;  // k_direction4 added those steps
    if (!(dq > 0.0) || !isfinite(dq) || !isfinite(rd)) {
      st->done = kDoneBreakdown;
      return;
    }
    st->alpha = (st->method == kMethodNpsdo ? rd : st->sigma) / dq;  // PCG / FPCG: sigma_k / d^T A d
    st->alpha_slot[slot] = st->alpha;
    st->dAd[slot] = dq;
    st->upd_pending = 1;
  });
}

// Recurrence mode: r -= alpha q with ||r||^2; the last block advances the
// iteration and applies the stop test ||r_k|| < tol ||b|| (the step's
// alpha d goes into x later, in k_direction4 or k_flush_x).  Explicit mode:
// x += alpha d in FP64 (the residual is then recomputed from x).
// With two residual buffers (r_alt non-null) it forms r_{k+1} = r_k - alpha q
// from buffer k mod 2 into the other one, and only while the step is
// pending (the level-1 CConv1 usually forms it, see k_cconv_stream).
template <bool RECUR>
__global__ void __launch_bounds__(kThreads) k_update4(int n, double *__restrict__ x, float *__restrict__ r_buf,
                                                      float *__restrict__ r_alt, const float *__restrict__ dring,
                                                      const float *__restrict__ qring, double *__restrict__ part,
                                                      unsigned *ticket, SolveState *st, double *hist) {
  if (st->done) return;
  if (RECUR && r_alt && !st->upd_pending) return;
  const bool odd = r_alt && (st->k & 1);
  const float *__restrict__ r_in = odd ? r_alt : r_buf;
  float *__restrict__ r_out = r_alt ? (odd ? r_buf : r_alt) : r_buf;
  const int slot = ring_slot(st->k + 1, st->n_ortho);
  const double a = st->alpha;
  const int n4 = n >> 2;
  const int stride = gridDim.x * blockDim.x;
  if (!RECUR) {
    const float *d = dring + (size_t)slot * n;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n4; g += stride) {
      const int p = g << 2;
      const float4 dv = ld4(d + p);
      double2 *xp = reinterpret_cast<double2 *>(x + p);
      double2 x01 = xp[0], x23 = xp[1];
      x01.x = fma(a, (double)dv.x, x01.x);
      x01.y = fma(a, (double)dv.y, x01.y);
      x23.x = fma(a, (double)dv.z, x23.x);
      x23.y = fma(a, (double)dv.w, x23.y);
      xp[0] = x01;
      xp[1] = x23;
    }
    return;
  }
  const float *q = qring + (size_t)slot * n;
  const float af = (float)a;
  DF acc;
  auto group = [&](int g) {
    const int p = g << 2;
    const float4 qv = ld4(q + p);
    float4 rv = ld4(r_in + p);
    rv.x = fmaf(-af, qv.x, rv.x);
    rv.y = fmaf(-af, qv.y, rv.y);
    rv.z = fmaf(-af, qv.z, rv.z);
    rv.w = fmaf(-af, qv.w, rv.w);
    st4(r_out + p, rv);
    df_add(acc, rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w);
  };
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  for (; g + stride < n4; g += 2 * stride) {
    group(g);
    group(g + stride);
  }
  if (g < n4) group(g);
  double v[1] = {df_val(acc)};
  reduce_and_finish<1>(v, part, ticket, [&](const double *t) {
    const double rr = t[0];
    st->k += 1;
    st->upd_pending = 0;
    st->rnorm2 = rr;
    hist[st->k] = sqrt(rr);
    if (!isfinite(rr)) st->done = kDoneBreakdown;
    else if (rr < st->eps2 || rr == 0.0) st->done = kDoneConverged;
    else st->rscale = (float)(1.0 / sqrt(rr));
  });
}

// Exact FP32 -> FP64 widening by re-biasing the exponent field (binary32:
// 8-bit exponent, bias 127, 23-bit fraction; binary64: 11-bit exponent, bias
// 1023, 52-bit fraction) on the integer units; zeros keep their sign,
// subnormal, infinite and NaN inputs take the conversion instruction.  B300's
// FP64 pipe is 1/64 of its FP32 rate, so x = hi + lo then costs one FP64 add.
__device__ __forceinline__ double widen(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if (e == 0u || e == 0xFFu) return (u & 0x7FFFFFFFu) == 0u ? __longlong_as_double((long long)sign) : (double)f;
  return __longlong_as_double(
      (long long)(sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

// Adds the steps not yet in x (x_upto < i <= k, at most n_ortho + 1 of them,
// their directions still in the ring) to the double-float pair, oldest
// first, and writes x = xhi + xlo in FP64; k_clear_pend then marks them
// added.
__global__ void __launch_bounds__(kThreads) k_flush_x(int n, float *__restrict__ xhi, float *__restrict__ xlo,
                                                      double *__restrict__ x, const float *__restrict__ dring,
                                                      const SolveState *st) {
  const int k = st->k, from = st->x_upto + 1, no = st->n_ortho;
  const int n4 = n >> 2;
  // the pending steps' alphas split once per thread (FP64, off the per-cell path)
  const int npend = k - from + 1;
  float pah[kRing], pal[kRing];
  int psl[kRing];
#pragma unroll
  for (int i = 0; i < kRing; ++i) {
    psl[i] = ring_slot(from + i, no);
    pah[i] = pal[i] = 0.f;
    if (i < npend) split_alpha(st->alpha_slot[psl[i]], pah[i], pal[i]);
  }
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n4; g += gridDim.x * blockDim.x) {
    const int p = g << 2;
    float4 h = ld4(xhi + p), l = ld4(xlo + p);
    if (npend > 0) {
#pragma unroll
      for (int i = 0; i < kRing; ++i)
        if (i < npend) df_axpy4(h, l, pah[i], pal[i], ld4(dring + (size_t)psl[i] * n + p));
      for (int it = from + kRing; it <= k; ++it) {  // more pending steps than ring slots: never on this path
        const int sl = ring_slot(it, no);
        float ah, al;
        split_alpha(st->alpha_slot[sl], ah, al);
        df_axpy4(h, l, ah, al, ld4(dring + (size_t)sl * n + p));
      }
      st4(xhi + p, h);
      st4(xlo + p, l);
    }
    double2 *xp = reinterpret_cast<double2 *>(x + p);
    xp[0] = make_double2(widen(h.x) + widen(l.x), widen(h.y) + widen(l.y));
    xp[1] = make_double2(widen(h.z) + widen(l.z), widen(h.w) + widen(l.w));
  }
}
__global__ void k_clear_pend(SolveState *st) { st->x_upto = st->k; }

// ---------------------------------------------------------------------------
// The true residual b - A x of the recurrence mode's x, held as a double-float
// pair (xhi, xlo) after the last flush (the returned FP64 x is the same value,
// widened).  Double-float arithmetic on FP32 (Knuth's TwoSum, the FMA exact
// product, Dekker's renormalisation; about 48 significant bits) instead of
// FP64, which B300 runs at 1/64 of its FP32 rate:
//   (A x)_p = sum over fluid neighbours (x_p - x_n) + (air neighbours) x_p
// (Sec. 3.2, from the stencil codes of k_lap4), r_p = b_p - (A x)_p, and the
// per-thread sums of r^2 and b^2 in double-float, FP64 only above the thread.
// Writes r (FP32, 0 off fluid) into r_k's buffer when r is given; the partials
// are those of k_true_residual (two per block of kRedThreads).
// ---------------------------------------------------------------------------
struct DD {
  float h, l;
};
__device__ __forceinline__ DD dd_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DD dd_norm(float s, float e) {  // |e| small against s
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ DD dd_add(DD a, DD b) {
  const DD s = dd_two_sum(a.h, b.h);
  return dd_norm(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ DD dd_sub(DD a, DD b) { return dd_add(a, DD{-b.h, -b.l}); }
__device__ __forceinline__ DD dd_mul(DD a, float m) {
  const float p = __fmul_rn(a.h, m);
  return dd_norm(p, fmaf(a.l, m, fmaf(a.h, m, -p)));
}
__device__ __forceinline__ DD dd_sqr(DD a) {
  const float p = __fmul_rn(a.h, a.h);
  return dd_norm(p, fmaf(__fmul_rn(2.f, a.h), a.l, fmaf(a.h, a.h, -p)));
}

__global__ void __launch_bounds__(kRedThreads) k_true_residual4(const uint16_t *__restrict__ code, Dims dm,
                                                                  const float *__restrict__ b,
                                                                  const float *__restrict__ xhi,
                                                                  const float *__restrict__ xlo, float *r,
                                                                  float *r_alt, const SolveState *sel,
                                                                  double *__restrict__ part) {
  if (r_alt && sel && (sel->k & 1)) r = r_alt;
  const int nx = dm.nx, ny = dm.ny, nz = dm.nz;
  const int n = nx * ny * nz, nxy = nx * ny, n4 = n >> 2;
  DD sr{0.f, 0.f}, sb{0.f, 0.f};
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n4; g += gridDim.x * blockDim.x) {
    const int p = g << 2;
    const ushort4 cc = *reinterpret_cast<const ushort4 *>(code + p);
    if (((cc.x | cc.y | cc.z | cc.w) & 0x8000u) == 0u) {
      if (r) st4(r + p, make_float4(0.f, 0.f, 0.f, 0.f));
      continue;
    }
    const int yz = p / nx, x0 = p - yz * nx, z = yz / ny, y = yz - z * ny;
    const float4 bv = ld4(b + p);
    const float4 hc = ld4(xhi + p), lc = ld4(xlo + p);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float hxl = x0 > 0 ? xhi[p - 1] : 0.f, lxl = x0 > 0 ? xlo[p - 1] : 0.f;
    const float hxr = x0 + 4 < nx ? xhi[p + 4] : 0.f, lxr = x0 + 4 < nx ? xlo[p + 4] : 0.f;
    const float4 hym = y > 0 ? ld4(xhi + p - nx) : zero4, lym = y > 0 ? ld4(xlo + p - nx) : zero4;
    const float4 hyp = y < ny - 1 ? ld4(xhi + p + nx) : zero4, lyp = y < ny - 1 ? ld4(xlo + p + nx) : zero4;
    const float4 hzm = z > 0 ? ld4(xhi + p - nxy) : zero4, lzm = z > 0 ? ld4(xlo + p - nxy) : zero4;
    const float4 hzp = z < nz - 1 ? ld4(xhi + p + nxy) : zero4, lzp = z < nz - 1 ? ld4(xlo + p + nxy) : zero4;
    const uint16_t cs[4] = {cc.x, cc.y, cc.z, cc.w};
    float ro[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const uint32_t c = cs[e];
      if (!(c & 0x8000u)) {
        ro[e] = 0.f;
        continue;
      }
      const DD xp{f4(hc, e), f4(lc, e)};
      const DD nb[6] = {DD{e == 0 ? hxl : f4(hc, e - 1), e == 0 ? lxl : f4(lc, e - 1)},
                        DD{e == 3 ? hxr : f4(hc, e + 1), e == 3 ? lxr : f4(lc, e + 1)},
                        DD{f4(hym, e), f4(lym, e)}, DD{f4(hyp, e), f4(lyp, e)},
                        DD{f4(hzm, e), f4(lzm, e)}, DD{f4(hzp, e), f4(lzp, e)}};
      DD ax{0.f, 0.f};
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if (c & (1u << k)) ax = dd_add(ax, dd_sub(xp, nb[k]));
      ax = dd_add(ax, dd_mul(xp, (float)((c >> 8) & 7u)));
      const float bp = f4(bv, e);
      const DD res = dd_sub(DD{bp, 0.f}, ax);
      ro[e] = res.h;
      sr = dd_add(sr, dd_sqr(res));
      sb = dd_add(sb, dd_sqr(DD{bp, 0.f}));
    }
    if (r) st4(r + p, make_float4(ro[0], ro[1], ro[2], ro[3]));
  }
  double v[2] = {(double)sr.h + (double)sr.l, (double)sb.h + (double)sb.l};
  block_sum_store<2>(v, part + (size_t)blockIdx.x * 2);
}



// ---------------------------------------------------------------------------
// Host-side launchers.
// ---------------------------------------------------------------------------
void launch_init4(const uint8_t *lab, int n, const float *b, float *r, double *x, float *xhi, float *xlo, double *part,
                  unsigned *ticket, double tol, int max_iter, int n_ortho, int method, SolveState *st, double *hist,
                  int num_sms, cudaStream_t s) {
  k_init4<<<grid4(n / 4, num_sms, resident_blocks<k_init4>()), kThreads, 0, s>>>(
      lab, n, b, r, x, xhi, xlo, part, ticket, tol, max_iter, n_ortho, method, st, hist);
}
void launch_combine1_4(const uint8_t *lab, int n, const float *x1, const float *x2, const double *c12, float *z,
                       const float *qring, const float *r0, const float *r1, double *part, unsigned *ticket,
                       SolveState *st, int num_sms, cudaStream_t s) {
  k_combine1_4<<<grid4(n / 4, num_sms, resident_blocks<k_combine1_4>()), kThreads, 0, s>>>(lab, n, x1, x2, c12, z,
                                                                                          qring, r0, r1, part, ticket,
                                                                                          st);
}
void launch_direction4(bool defer_x, int n, const float *z, float *dring, float *xhi, float *xlo, const uint32_t *gmask,
                       const SolveState *st, int n_ortho, int num_sms, cudaStream_t s) {
  switch ((defer_x ? 8 : 0) + n_ortho) {
#define NPS_DIR_CASE(D, NO)                                                                                        \
  case (D ? 8 : 0) + NO:                                                                                           \
    k_direction4<D, NO><<<grid4(n / 4, num_sms, resident_blocks<k_direction4<D, NO>>()), kThreads, 0, s>>>(       \
        n, z, dring, xhi, xlo, gmask, st);                                                                         \
    break;
    NPS_DIR_CASE(false, 0)
    NPS_DIR_CASE(false, 1)
    NPS_DIR_CASE(false, 2)
    NPS_DIR_CASE(false, 3)
    NPS_DIR_CASE(false, 4)
    NPS_DIR_CASE(true, 0)
    NPS_DIR_CASE(true, 1)
    NPS_DIR_CASE(true, 2)
    NPS_DIR_CASE(true, 3)
    NPS_DIR_CASE(true, 4)
#undef NPS_DIR_CASE
    default:
      break;
  }
}
void launch_lap_codes(const uint8_t *lab, Dims dm, uint16_t *code, uint32_t *gmask, cudaStream_t s) {
  const int n4 = (int)(dm.n() / 4);
  long long g = ((long long)((n4 + 31) / 32) * 32 + kThreads - 1) / kThreads;
  if (g > 148LL * 16) g = 148LL * 16;
  k_lap_codes4<<<(int)(g < 1 ? 1 : g), kThreads, 0, s>>>(lab, dm, code, gmask);
}
void launch_lap4(const uint16_t *code, Dims dm, const float *dring, float *qring, const float *r, const float *r_alt,
                 double *part, unsigned *ticket, SolveState *st, int num_sms, cudaStream_t s) {
  k_lap4<<<grid4(dm.n() / 4, num_sms, resident_blocks<k_lap4>()), kThreads, 0, s>>>(
      code, dm, make_fastdiv((uint32_t)dm.nx), make_fastdiv((uint32_t)dm.ny), dring, qring, r, r_alt, part, ticket, st);
}
// The true residual from the double-float x: the figures only (r null), or
// the residual replacement of the recurrence (r_k's buffer by parity) with the
// re-opening decision; the final kernels are those of the FP64 form.
void launch_true_residual4(const uint16_t *code, Dims dm, const float *b, const float *xhi, const float *xlo, float *r,
                           float *r_alt, double *part, SolveState *st, int *reopened, double *relres,
                           cudaStream_t s) {
  const int nb = red_blocks(dm.n());
  k_true_residual4<<<nb, kRedThreads, 0, s>>>(code, dm, b, xhi, xlo, r, r_alt, st, part);
  if (reopened) launch_restart_final(part, nb, st, reopened, relres, s);
  else launch_relres_final(part, nb, relres, s);
}
void launch_flush_x(int n, float *xhi, float *xlo, double *x, const float *dring, SolveState *st, int num_sms,
                    cudaStream_t s) {
  k_flush_x<<<grid4(n / 4, num_sms, resident_blocks<k_flush_x>()), kThreads, 0, s>>>(n, xhi, xlo, x, dring, st);
  k_clear_pend<<<1, 1, 0, s>>>(st);
}
void launch_update4(bool recurrence, int n, double *x, float *r, float *r_alt, const float *dring, const float *qring,
                    double *part, unsigned *ticket, SolveState *st, double *hist, int num_sms, cudaStream_t s) {
  if (recurrence)
    k_update4<true><<<grid4(n / 4, num_sms, resident_blocks<k_update4<true>>()), kThreads, 0, s>>>(n, x, r, r_alt, dring, qring, part, ticket, st, hist);
  else
    k_update4<false><<<grid4(n / 4, num_sms, resident_blocks<k_update4<false>>()), kThreads, 0, s>>>(n, x, r, nullptr, dring, qring, part, ticket, st, hist);
}

}  // namespace nps
