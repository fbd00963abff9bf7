// Backward kernels of the network (reverse of Alg. 2) and of the training
// loss of Sec. 4.2.3, Loss = || b - A P_net(I, b) ||_2.
//
// CConv backward for an output cotangent g (per level):
//   input gradient   gv(q) = sum_a K_a(q - a) g(q - a)          (gather form)
//   kernel gradient  gK_a(p) = g(p) v(p + a)
//   weight gradient  gW'[a][j] = sum_p gK_a(p) F_j(p),  F = (nF window, nA window, 1)
// with K stored per cell by the training forward (k_cconv_store_K) so the
// input gradient is a deterministic gather, and the 27 x 55 weight gradient a
// [27 x P] . [P x 55] contraction over the cells: on the tcgen05 tensor cores
// where the level's image counts are exact in BF16 (k_cconv_wgrad_tc), on
// CUDA cores in FP32 32-cell batches beyond (k_cconv_wgrad); block partials
// reduced in FP64 in a fixed order.
#include <cuda_bf16.h>
#include <string.h>

#include "nps_common.cuh"
#include "nps_kernels.h"
#include "umma.cuh"

namespace nps {

namespace {

__device__ __forceinline__ float2 feat_at(const uint8_t *lab, const ushort2 *counts, const Dims &d, int x, int y,
                                          int z) {
  if (x < 0 || y < 0 || z < 0 || x >= d.nx || y >= d.ny || z >= d.nz) return make_float2(0.f, 0.f);
  const long long p = ((long long)z * d.ny + y) * d.nx + x;
  if (lab) {
    const uint8_t l = lab[p];
    return make_float2(l == kFluid ? 1.f : 0.f, l == kAir ? 1.f : 0.f);
  }
  const ushort2 c = counts[p];
  return make_float2((float)c.x, (float)c.y);
}

__device__ __forceinline__ float vec_at(const float *v, const Dims &d, int x, int y, int z) {
  if (x < 0 || y < 0 || z < 0 || x >= d.nx || y >= d.ny || z >= d.nz) return 0.f;
  return v[((long long)z * d.ny + y) * d.nx + x];
}

inline int gridn(long long n, int t) {
  long long b = (n + t - 1) / t;
  if (b > 148LL * 16) b = 148LL * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

// K[p][a] for every cell of a level (27 floats per cell, FP32 generation).
__global__ void __launch_bounds__(128) k_materialize_K(const uint8_t *__restrict__ lab, const ushort2 *__restrict__ counts,
                                                       Dims d, const CConvW *__restrict__ w, float *__restrict__ K) {
  __shared__ CConvW sw;
  {
    const float *src = (const float *)w;
    float *dst = (float *)&sw;
    for (int i = threadIdx.x; i < (int)(sizeof(CConvW) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const long long n = d.n();
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(p, d, x, y, z);
    float nf[27], na[27];
#pragma unroll
    for (int l = 0; l < 27; ++l) {
      const float2 f = feat_at(lab, counts, d, x + l % 3 - 1, y + (l / 3) % 3 - 1, z + l / 9 - 1);
      nf[l] = f.x;
      na[l] = f.y;
    }
#pragma unroll 1
    for (int a = 0; a < 27; ++a) {
      float k = sw.bp[a];
#pragma unroll
      for (int l = 0; l < 27; ++l) k = fmaf(sw.wf[a][l], nf[l], fmaf(sw.wa[a][l], na[l], k));
      K[p * 27 + a] = k;
    }
  }
}

// Training forward of one CConv block: out(p) = sum_a K_a(p) v(p + a), the
// per-cell kernels stored to K[p][a] for the backward.  A window that is all
// one pure class (all solid, all fluid or all air, the grid's outside solid)
// takes that class's constant kernel (computed once on the host, as the
// solve's cached path does); any other window computes K_a(p) as the solve's
// CUDA-core CConv does (the same FMA order; rounded to BF16 when RK).  The
// folded weights are a kernel parameter (uniform constant operands of the
// FMAs, no shared-memory load per FMA), and a warp whose 32 windows are all
// pure skips the FMA chain.  A warp owns 32 consecutive cells; with ROWS (nx a
// multiple of 32) they are 32 cells of one grid row and the warp loads each of
// the nine window rows once, coalesced, taking the x-1 and x+1 taps from the
// neighbouring lanes.  Each warp's 32 x 27 kernels go out through shared
// memory as contiguous stores.
struct PureK {
  float k[3][27];  // the constant kernels of pure solid, fluid and air windows
};
constexpr int kSKWarps = 4;

// One window cell's features and input value (0 outside the grid; the input
// zeroed off fluid when mask_input).  SRC: where the features come from,
// kSrcLabels (level 1), kSrcCounts (coarser levels) or kSrcEither (lab if set).
enum { kSrcEither = 0, kSrcLabels = 1, kSrcCounts = 2 };
template <int SRC = kSrcEither>
__device__ __forceinline__ void window_cell(const uint8_t *lab, const ushort2 *counts, const float *v, long long q,
                                            int mask_input, float &f, float &a, float &val) {
  if (SRC == kSrcLabels || (SRC == kSrcEither && lab)) {
    const uint8_t l = lab[q];
    f = l == kFluid ? 1.f : 0.f;
    a = l == kAir ? 1.f : 0.f;
  } else {
    const ushort2 c = counts[q];
    f = (float)c.x;
    a = (float)c.y;
  }
  val = v[q];
  if (mask_input && f == 0.f) val = 0.f;  // level 1: f == 1 exactly on fluid
}

// The window (features and input) of the 32 cells x0 .. x0+31 of one grid row,
// lane i holding cell x0+i's: each of the nine window rows is loaded once,
// coalesced, the x-1 and x+1 taps taken from the neighbouring lanes (lanes 0
// and 31 load the halo columns).
template <int SRC = kSrcEither>
__device__ __forceinline__ void window_rows(const uint8_t *lab, const ushort2 *counts, const float *v, const Dims &d,
                                            int mask_input, long long p0, int lane, float (&nf)[27], float (&na)[27],
                                            float (&vv)[27]) {
  int x0, y, z;
  cell_xyz(p0, d, x0, y, z);
#pragma unroll
  for (int r = 0; r < 9; ++r) {  // window row dy = r % 3 - 1, dz = r / 3 - 1
    const int yy = y + r % 3 - 1, zz = z + r / 3 - 1;
    float cf = 0.f, ca = 0.f, cv = 0.f, hf = 0.f, ha = 0.f, hv = 0.f;
    if (yy >= 0 && yy < d.ny && zz >= 0 && zz < d.nz) {  // the same for the whole warp
      const long long rb = ((long long)zz * d.ny + yy) * d.nx;
      window_cell<SRC>(lab, counts, v, rb + x0 + lane, mask_input, cf, ca, cv);
      const int hx = lane == 0 ? x0 - 1 : x0 + 32;  // the halo columns, read by lanes 0 and 31
      if ((lane == 0 || lane == 31) && hx >= 0 && hx < d.nx)
        window_cell<SRC>(lab, counts, v, rb + hx, mask_input, hf, ha, hv);
    }
    float lf = __shfl_up_sync(0xffffffffu, cf, 1), la = __shfl_up_sync(0xffffffffu, ca, 1);
    float lv = __shfl_up_sync(0xffffffffu, cv, 1);
    float rf = __shfl_down_sync(0xffffffffu, cf, 1), ra = __shfl_down_sync(0xffffffffu, ca, 1);
    float rv = __shfl_down_sync(0xffffffffu, cv, 1);
    if (lane == 0) {
      lf = hf;
      la = ha;
      lv = hv;
    }
    if (lane == 31) {
      rf = hf;
      ra = ha;
      rv = hv;
    }
    nf[3 * r] = lf;
    na[3 * r] = la;
    vv[3 * r] = lv;
    nf[3 * r + 1] = cf;
    na[3 * r + 1] = ca;
    vv[3 * r + 1] = cv;
    nf[3 * r + 2] = rf;
    na[3 * r + 2] = ra;
    vv[3 * r + 2] = rv;
  }
}

// 0 pure solid, 1 pure fluid, 2 pure air, -1 anything else (a cell of a pure
// class has count `full` of it: 1 at level 1, 8^(l-1) at level l).
__device__ __forceinline__ int window_class(const float (&nf)[27], const float (&na)[27], float full) {
  bool all_s = true, all_f = true, all_a = true;
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    all_s &= nf[t] == 0.f && na[t] == 0.f;
    all_f &= nf[t] == full;
    all_a &= na[t] == full;
  }
  return all_f ? 1 : (all_a ? 2 : (all_s ? 0 : -1));
}

__device__ __forceinline__ float pure_k(const PureK &pk, int c, int a) {
  return c == 1 ? pk.k[1][a] : (c == 2 ? pk.k[2][a] : pk.k[0][a]);
}

// A warp's 32 x 27 kernels (staged in shared memory at stride 27, odd: no bank
// conflicts) out to K as contiguous stores.
__device__ __forceinline__ void store_tile_K(const float *sk, long long wt, long long n, int lane, float *K) {
  __syncwarp();
  const long long lim = (n - wt * 32) * 27;  // floats of this tile inside the grid
  float *dst = K + wt * 32 * 27;
  for (int i = lane; i < 32 * 27; i += 32)
    if (i < lim) dst[i] = sk[i];
  __syncwarp();
}

template <bool RK, bool ROWS>
__global__ void __launch_bounds__(kSKWarps * 32) k_cconv_store_K(const uint8_t *__restrict__ lab,
                                                                 const ushort2 *__restrict__ counts, Dims d,
                                                                 const __grid_constant__ CConvW w,
                                                                 const __grid_constant__ PureK pk, float full,
                                                                 const float *__restrict__ v, int mask_input,
                                                                 float *__restrict__ K, float *__restrict__ out) {
  __shared__ float sk[kSKWarps][32 * 27];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long n = d.n();
  const long long ntiles = (n + 31) / 32;
  for (long long wt = (long long)blockIdx.x * kSKWarps + warp; wt < ntiles; wt += (long long)gridDim.x * kSKWarps) {
    const long long p = wt * 32 + lane;
    const bool act = p < n;
    float nf[27], na[27], vv[27];
    if (ROWS) {  // n is a multiple of 32: every lane is active
      window_rows(lab, counts, v, d, mask_input, wt * 32, lane, nf, na, vv);
    } else if (act) {
      int x, y, z;
      cell_xyz(p, d, x, y, z);
#pragma unroll
      for (int t = 0; t < 27; ++t) {
        const int xx = x + t % 3 - 1, yy = y + (t / 3) % 3 - 1, zz = z + t / 9 - 1;
        nf[t] = na[t] = vv[t] = 0.f;
        if (xx >= 0 && yy >= 0 && zz >= 0 && xx < d.nx && yy < d.ny && zz < d.nz)
          window_cell(lab, counts, v, ((long long)zz * d.ny + yy) * d.nx + xx, mask_input, nf[t], na[t], vv[t]);
      }
    } else {
#pragma unroll
      for (int t = 0; t < 27; ++t) nf[t] = na[t] = vv[t] = 0.f;  // lanes past the end: solid
    }
    const int cls = window_class(nf, na, full);
    const int c = cls < 0 ? 0 : cls;
    float acc = 0.f;
    if (__all_sync(0xffffffffu, cls >= 0)) {
#pragma unroll
      for (int a = 0; a < 27; ++a) {
        const float k = pure_k(pk, c, a);
        acc = fmaf(k, vv[a], acc);
        sk[warp][lane * 27 + a] = k;
      }
    } else {
#pragma unroll
      for (int a = 0; a < 27; ++a) {
        float k = w.bp[a];
#pragma unroll
        for (int l = 0; l < 27; ++l) k = fmaf(w.wf[a][l], nf[l], fmaf(w.wa[a][l], na[l], k));
        if (RK) k = __bfloat162float(__float2bfloat16_rn(k));
        if (cls >= 0) k = pure_k(pk, c, a);
        acc = fmaf(k, vv[a], acc);
        sk[warp][lane * 27 + a] = k;
      }
    }
    if (act) out[p] = acc;
    store_tile_K(sk[warp], wt, n, lane, K);
  }
}

// The same block on the tcgen05 tensor cores, for levels whose image counts
// are exact in BF16 (at most 256 fine cells per cell) and rows of a multiple
// of 32 cells.  A CTA takes 128 cells (four 32-cell row runs, one per warp,
// loaded as in window_rows); each thread writes its cell's 64 BF16 features
// (the exact counts, the bias 1) into TMEM as the MMA's A rows, one thread
// issues the contraction with the folded weights split into `nsplit` BF16
// terms (K-major in shared memory, the solve's kernel-generation layout), and
// the FP32 result comes back per cell from TMEM: the kernels of windows that
// are not pure, the same values as the solve's tensor-core generation.  Pure
// windows take their class kernel; BF16 rounding (RK), the output sum and the
// stores are those of k_cconv_store_K.  A timed-out MMA wait sets *err.
constexpr int kSTCells = 128;
template <bool RK, int SRC>
__global__ void __launch_bounds__(kSTCells) k_cconv_store_K_tc(const uint8_t *__restrict__ lab,
                                                               const ushort2 *__restrict__ counts, Dims d,
                                                               const uint8_t *__restrict__ wsplit, int nsplit,
                                                               const __grid_constant__ PureK pk, float full,
                                                               const float *__restrict__ v, int mask_input,
                                                               float *__restrict__ K, float *__restrict__ out,
                                                               int *err) {
  using namespace umma;
  __shared__ __align__(1024) uint8_t sW[3 * kBBytes];
  __shared__ float sk[kSTCells / 32][32 * 27];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < nsplit * kBBytes / 16; i += kSTCells) ((uint4 *)sW)[i] = ((const uint4 *)wsplit)[i];
  if (warp == 0) {
    tmem_alloc(&s_tmem, kTmemCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&mbar, 1);
    fence_mbar_init();
  }
  fence_proxy_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = s_tmem;
  const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
  const uint32_t idesc = idesc_bf16(kTileM, kN);
  const long long n = d.n();  // a multiple of 32
  const long long nch = (n + kSTCells - 1) / kSTCells;
  uint32_t phase = 0u;
  bool aborted = false, issued = false;
  for (long long ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const long long wt = ch * (kSTCells / 32) + warp;  // this warp's 32-cell run
    const long long p = wt * 32 + lane;
    const bool act = wt * 32 < n;
    float nf[27], na[27], vv[27];
    uint32_t fw[32];
    int cls = 0;
    if (act) {
      window_rows<SRC>(lab, counts, v, d, mask_input, wt * 32, lane, nf, na, vv);
      cls = window_class(nf, na, full);
      uint32_t wc[27];  // (fluid, air) of each window cell as a BF16 pair: exact, the counts are at most 256
#pragma unroll
      for (int l = 0; l < 27; ++l) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(nf[l], na[l]);
        wc[l] = *reinterpret_cast<const uint32_t *>(&h);
      }
      build_feature_words(wc, fw);
    } else {
#pragma unroll
      for (int t = 0; t < 27; ++t) nf[t] = na[t] = vv[t] = 0.f;
#pragma unroll
      for (int q = 0; q < 32; ++q) fw[q] = 0u;
    }
    tmem_st32(tmem + lane_off, fw);
    tmem_wait_st();
    fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      for (int sp = 0; sp < nsplit; ++sp)
#pragma unroll
        for (int kk = 0; kk < kK / 16; ++kk) {
          const uint64_t bd = smem_desc_kmajor(smem_u32(sW + sp * kBBytes + kk * 2 * kLBO), kLBO, kSBO);
          mma_bf16_ts(tmem + 32, tmem + kk * 8, bd, idesc, (sp | kk) != 0);
        }
      umma_commit(&mbar);
    }
    issued = true;
    const bool ok = mbar_wait_bounded(&mbar, phase, kWaitNs);
    if (__syncthreads_or(!ok)) {
      aborted = true;
      break;
    }
    phase ^= 1u;
    issued = false;
    fence_after_sync();
    uint32_t kr[32];
    tmem_ld32(tmem + 32 + lane_off, kr);
    tmem_wait_ld();
    const int c = cls < 0 ? 0 : cls;
    float acc = 0.f;
#pragma unroll
    for (int a = 0; a < 27; ++a) {
      float k = __uint_as_float(kr[a]);
      if (RK) k = __bfloat162float(__float2bfloat16_rn(k));
      if (cls >= 0) k = pure_k(pk, c, a);
      acc = fmaf(k, vv[a], acc);
      sk[warp][lane * 27 + a] = k;
    }
    if (act) {
      out[p] = acc;
      store_tile_K(sk[warp], wt, n, lane, K);
    }
    // the next chunk's MMAs are issued after its barrier, which every thread
    // reaches only after its TMEM load above has completed
  }
  if (aborted) {
    if (tid == 0 && err) atomicExch(err, 1);
    if (issued) (void)mbar_wait_bounded(&mbar, phase, kWaitNs);  // the MMAs possibly still in flight
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// gv(q) = sum_a K_a(q - a) g(q - a) over neighbours p = q - a inside the grid.
__global__ void k_cconv_transpose(const float *__restrict__ K, const float *__restrict__ g, Dims d,
                                  float *__restrict__ gv) {
  const long long n = d.n();
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(q, d, x, y, z);
    float acc = 0.f;
#pragma unroll
    for (int a = 0; a < 27; ++a) {
      const int px = x - (a % 3 - 1), py = y - ((a / 3) % 3 - 1), pz = z - (a / 9 - 1);
      if (px < 0 || py < 0 || pz < 0 || px >= d.nx || py >= d.ny || pz >= d.nz) continue;
      const long long p = ((long long)pz * d.ny + py) * d.nx + px;
      acc = fmaf(K[p * 27 + a], g[p], acc);
    }
    gv[q] = acc;
  }
}

// Weight gradient of one CConv block: block partials of
//   G[a][j] = sum_p g(p) v(p + a) F_j(p),  j < 27: nF(p + l_j), j < 54: nA(p + l_{j-27}), j = 54: 1.
constexpr int kWG = 27 * 55;  // 1485 outputs
constexpr int kWGBatch = 32;
__global__ void __launch_bounds__(256) k_cconv_wgrad(const uint8_t *__restrict__ lab, const ushort2 *__restrict__ counts,
                                                     Dims d, const float *__restrict__ v, const float *__restrict__ g,
                                                     double *__restrict__ part) {
  __shared__ float sGK[kWGBatch][27];
  __shared__ float sF[kWGBatch][56];
  const int tid = threadIdx.x;
  float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // outputs tid, tid+256, ... (< kWG)
  const long long n = d.n();
  const long long nb = (n + kWGBatch - 1) / kWGBatch;
  for (long long bt = blockIdx.x; bt < nb; bt += gridDim.x) {
    const long long p0 = bt * kWGBatch;
    // stage gK (27 per cell) and F (55 per cell) of the batch
    for (int i = tid; i < kWGBatch * 27; i += blockDim.x) {
      const int c = i / 27, a = i % 27;
      const long long p = p0 + c;
      float val = 0.f;
      if (p < n) {
        int x, y, z;
        cell_xyz(p, d, x, y, z);
        const float gp = g[p];
        if (gp != 0.f) val = gp * vec_at(v, d, x + a % 3 - 1, y + (a / 3) % 3 - 1, z + a / 9 - 1);
      }
      sGK[c][a] = val;
    }
    for (int i = tid; i < kWGBatch * 28; i += blockDim.x) {
      const int c = i / 28, l = i % 28;
      const long long p = p0 + c;
      float ff = 0.f, fa = 0.f;
      if (p < n && l < 27) {
        int x, y, z;
        cell_xyz(p, d, x, y, z);
        const float2 f = feat_at(lab, counts, d, x + l % 3 - 1, y + (l / 3) % 3 - 1, z + l / 9 - 1);
        ff = f.x;
        fa = f.y;
      }
      if (l < 27) {
        sF[c][l] = ff;
        sF[c][27 + l] = fa;
      } else {
        sF[c][54] = p < n ? 1.f : 0.f;
        sF[c][55] = 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int o = tid + k * 256;
      if (o < kWG) {
        const int a = o / 55, j = o % 55;
        float s = acc[k];
#pragma unroll 8
        for (int c = 0; c < kWGBatch; ++c) s = fmaf(sGK[c][a], sF[c][j], s);
        acc[k] = s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int o = tid + k * 256;
    if (o < kWG) part[(size_t)blockIdx.x * kWG + o] = (double)acc[k];
  }
}

// The same weight gradient on the tcgen05 tensor cores, for levels whose
// image counts are exact in BF16 (at most 256 fine cells per cell: levels
// 1-3 here).  The contraction over cells is the MMA's K dimension:
//   D[j][s * 32 + a] = sum_p F_j(p) gK_a^(s)(p)   (FP32 in TMEM)
// with A = F (the 54 window counts and the bias 1 per cell, rows 55..127 zero)
// and B = the kernel gradient gK_a(p) = g(p) v(p + a) split into three BF16
// terms s (hi, mid, lo; their sum is the FP32 value to 2^-24 relative), both
// K-major in shared memory in 128-cell chunks.  The threads stage a chunk in
// runs of 8 cells (rows of a multiple of 8 cells: wg_load_run / wg_store_run)
// or one cell each (any grid: wg_stage_cells, the window counts and 27
// products of its 3 x 3 x 3 window); one thread issues the chunk's eight MMAs
// (K = 16 each) and commits them to the buffer's mbarrier, while the CTA stages
// the next chunk into the other buffer.  D accumulates over all of the CTA's chunks; at the end lane
// j holds G[a][j] = D[j][a] + D[j][32 + a] + D[j][64 + a], written as the
// CTA's partial in the layout of k_cconv_wgrad (reduced by k_wgrad_final).
constexpr int kWgCells = 128;                      // cells per chunk (MMA K = 8 x 16)
// threads: the 144 staging tasks of a chunk of runs (16 runs x 9 window rows)
// one each; the per-cell staging uses the first 128, the epilogue warps 0-1
// (TMEM lanes 0-63 hold the 55 feature rows)
constexpr int kWgThreads = 160;
constexpr int kWgRowsA = 128;                      // MMA M: 55 feature rows, padded
constexpr int kWgRowsB = 96;                       // MMA N: 3 BF16 terms x 32 taps
constexpr int kWgSBO = (kWgCells / 8) * 128;       // bytes between 8-row groups (K-major, no swizzle)
constexpr int kWgABytes = kWgRowsA * kWgCells * 2;  // 32 KB
constexpr int kWgBBytes = kWgRowsB * kWgCells * 2;  // 24 KB
constexpr int kWgBufBytes = kWgABytes + kWgBBytes;
constexpr int kWgSmem = 2 * kWgBufBytes + 1024;     // two buffers + barriers (and 1 KB alignment slack)
constexpr int kWgTmemCols = 128;

// Byte offset of element (row, k) in a K-major, non-swizzled operand tile.
__device__ __forceinline__ uint32_t wg_off(int row, int k) {
  return (uint32_t)((row >> 3) * kWgSBO + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// The three BF16 terms hi + mid + lo of two FP32 values (hi = bf16(x),
// mid = bf16(x - hi), lo = bf16(x - hi - mid)), packed in pairs.
__device__ __forceinline__ void split3_pair(float a, float b, uint32_t &hi, uint32_t &mid, uint32_t &lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float ra = a - __low2float(h), rb = b - __high2float(h);
  const __nv_bfloat162 m = __floats2bfloat162_rn(ra, rb);
  const __nv_bfloat162 l = __floats2bfloat162_rn(ra - __low2float(m), rb - __high2float(m));
  hi = *(const uint32_t *)&h;
  mid = *(const uint32_t *)&m;
  lo = *(const uint32_t *)&l;
}

__device__ __forceinline__ uint32_t bf16_bits_of_count(uint32_t c) {  // exact: c <= 256
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn((float)c));
}

// Operand staging of one 128-cell chunk when nx % 8 == 0 (and the sources are
// aligned for vector loads): the chunk is 16 runs of 8 consecutive cells of
// one grid row.  A task is one run and one (dy, dz) row of the 3 x 3 x 3
// window, one per thread (144 tasks, kWgThreads >= 144): wg_load_run issues its
// loads -- the ten labels / counts and input values x0-1 .. x0+8 of that row and
// the run's eight cotangents -- and wg_store_run writes the taps dx = -1, 0, 1
// of both feature channels and of the three BF16 terms of gK, each one 16-byte
// row of the K-major operands.  (Issuing the next chunk's loads before this
// chunk's stores was measured: no faster, 128 registers instead of 104.)  The
// values are those of the per-cell staging, bit for bit.
struct WgRaw {
  uint4 i0, i1;         // labels (i0.x, i0.y: 8 bytes) or counts (8 ushort2) of x0 .. x0+7
  uint32_t el, er;      // the same at x0-1 and x0+8 (0 outside the grid)
  float4 a0, a1, g0, g1;  // input at x0 .. x0+7; cotangents of the run
  float vl, vr;         // input at x0-1 and x0+8
  int run, r;           // r < 0: no task
  bool valid;
};
static_assert(kWgThreads >= (kWgCells / 8) * 9, "one staging task per thread");

template <bool LABELS>
__device__ __forceinline__ WgRaw wg_load_run(const uint8_t *__restrict__ lab, const ushort2 *__restrict__ counts,
                                             const Dims &d, const float *__restrict__ v,
                                             const float *__restrict__ g, long long ch, int tid) {
  WgRaw w;
  w.i0 = w.i1 = make_uint4(0u, 0u, 0u, 0u);
  w.el = w.er = 0u;
  w.a0 = w.a1 = w.g0 = w.g1 = make_float4(0.f, 0.f, 0.f, 0.f);
  w.vl = w.vr = 0.f;
  w.run = tid / 9;
  w.r = tid < (kWgCells / 8) * 9 ? tid - w.run * 9 : -1;
  w.valid = false;
  if (w.r < 0) return w;
  const long long n = d.n();
  const long long p0 = ch * kWgCells + w.run * 8;
  w.valid = p0 < n;  // n is a multiple of 8
  int x0 = 0, y = 0, z = 0;
  if (w.valid) cell_xyz(p0, d, x0, y, z);
  const int yy = y + w.r % 3 - 1, zz = z + w.r / 3 - 1;
  const bool rowin = w.valid && yy >= 0 && yy < d.ny && zz >= 0 && zz < d.nz;
  const long long rb = rowin ? ((long long)zz * d.ny + yy) * d.nx + x0 : 0;  // cell x0 of the row
  const bool has_l = rowin && x0 > 0, has_r = rowin && x0 + 8 < d.nx;
  if (LABELS) {
    if (rowin) {
      const uint2 m = *(const uint2 *)(lab + rb);
      w.i0.x = m.x;
      w.i0.y = m.y;
    }
    if (has_l) w.el = lab[rb - 1];
    if (has_r) w.er = lab[rb + 8];
  } else {
    if (rowin) {
      w.i0 = *(const uint4 *)(counts + rb);
      w.i1 = *(const uint4 *)(counts + rb + 4);
    }
    if (has_l) w.el = *(const uint32_t *)(counts + rb - 1);
    if (has_r) w.er = *(const uint32_t *)(counts + rb + 8);
  }
  if (rowin) {
    w.a0 = *(const float4 *)(v + rb);
    w.a1 = *(const float4 *)(v + rb + 4);
  }
  if (w.valid) {
    w.g0 = *(const float4 *)(g + p0);
    w.g1 = *(const float4 *)(g + p0 + 4);
  }
  if (has_l) w.vl = v[rb - 1];
  if (has_r) w.vr = v[rb + 8];
  return w;
}

template <bool LABELS>
__device__ __forceinline__ void wg_store_run(const WgRaw &w, uint8_t *A, uint8_t *B) {
  if (w.r < 0) return;
  // the fluid and air features at x0-1 .. x0+8 as BF16 bits (0 outside the grid)
  uint32_t hf[10], ha[10];
  if (LABELS) {
    hf[0] = w.el == kFluid ? 0x3F80u : 0u;
    ha[0] = w.el == kAir ? 0x3F80u : 0u;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint32_t c = ((i < 4 ? w.i0.x : w.i0.y) >> (8 * (i & 3))) & 0xFFu;
      hf[1 + i] = c == kFluid ? 0x3F80u : 0u;
      ha[1 + i] = c == kAir ? 0x3F80u : 0u;
    }
    hf[9] = w.er == kFluid ? 0x3F80u : 0u;
    ha[9] = w.er == kAir ? 0x3F80u : 0u;
  } else {
    const uint32_t wv[10] = {w.el, w.i0.x, w.i0.y, w.i0.z, w.i0.w, w.i1.x, w.i1.y, w.i1.z, w.i1.w, w.er};
#pragma unroll
    for (int i = 0; i < 10; ++i) {
      hf[i] = bf16_bits_of_count(wv[i] & 0xFFFFu);
      ha[i] = bf16_bits_of_count(wv[i] >> 16);
    }
  }
  const float vr[10] = {w.vl, w.a0.x, w.a0.y, w.a0.z, w.a0.w, w.a1.x, w.a1.y, w.a1.z, w.a1.w, w.vr};
  const float gp[8] = {w.g0.x, w.g0.y, w.g0.z, w.g0.w, w.g1.x, w.g1.y, w.g1.z, w.g1.w};
  const uint32_t col = (uint32_t)w.run * 8;
#pragma unroll
  for (int k = 0; k < 3; ++k) {  // dx = k - 1: tap a = 3 r + k
    const int a = 3 * w.r + k;
    uint4 f, q, hi, md, lo;
    f.x = hf[k] | (hf[k + 1] << 16);
    f.y = hf[k + 2] | (hf[k + 3] << 16);
    f.z = hf[k + 4] | (hf[k + 5] << 16);
    f.w = hf[k + 6] | (hf[k + 7] << 16);
    q.x = ha[k] | (ha[k + 1] << 16);
    q.y = ha[k + 2] | (ha[k + 3] << 16);
    q.z = ha[k + 4] | (ha[k + 5] << 16);
    q.w = ha[k + 6] | (ha[k + 7] << 16);
    *(uint4 *)(A + wg_off(a, col)) = f;
    *(uint4 *)(A + wg_off(27 + a, col)) = q;
    float gk[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) gk[i] = gp[i] != 0.f ? gp[i] * vr[i + k] : 0.f;
    split3_pair(gk[0], gk[1], hi.x, md.x, lo.x);
    split3_pair(gk[2], gk[3], hi.y, md.y, lo.y);
    split3_pair(gk[4], gk[5], hi.z, md.z, lo.z);
    split3_pair(gk[6], gk[7], hi.w, md.w, lo.w);
    *(uint4 *)(B + wg_off(a, col)) = hi;
    *(uint4 *)(B + wg_off(32 + a, col)) = md;
    *(uint4 *)(B + wg_off(64 + a, col)) = lo;
  }
  if (w.r == 0) {  // the constant feature of the bias
    const uint32_t one = w.valid ? 0x3F803F80u : 0u;
    *(uint4 *)(A + wg_off(54, col)) = make_uint4(one, one, one, one);
  }
}

// Operand staging of one 128-cell chunk, one cell per thread (any grid).
__device__ __forceinline__ void wg_stage_cells(const uint8_t *__restrict__ lab, const ushort2 *__restrict__ counts,
                                               const Dims &d, const float *__restrict__ v,
                                               const float *__restrict__ g, long long ch, uint8_t *A, uint8_t *B,
                                               int tid) {
  if (tid >= kWgCells) return;
  const long long n = d.n();
  const long long p = ch * kWgCells + tid;
  float gp = 0.f;
  int x = 0, y = 0, z = 0;
  if (p < n) {
    cell_xyz(p, d, x, y, z);
    gp = g[p];
  }
#pragma unroll
  for (int l = 0; l < 27; ++l) {
    const float2 f = p < n ? feat_at(lab, counts, d, x + l % 3 - 1, y + (l / 3) % 3 - 1, z + l / 9 - 1)
                           : make_float2(0.f, 0.f);
    *(__nv_bfloat16 *)(A + wg_off(l, tid)) = __float2bfloat16_rn(f.x);  // exact: counts <= 256
    *(__nv_bfloat16 *)(A + wg_off(27 + l, tid)) = __float2bfloat16_rn(f.y);
  }
  *(__nv_bfloat16 *)(A + wg_off(54, tid)) = __float2bfloat16_rn(p < n ? 1.f : 0.f);
#pragma unroll
  for (int a = 0; a < 27; ++a) {
    const float gk = gp != 0.f ? gp * vec_at(v, d, x + a % 3 - 1, y + (a / 3) % 3 - 1, z + a / 9 - 1) : 0.f;
    const __nv_bfloat16 hi = __float2bfloat16_rn(gk);
    const float r1 = gk - __bfloat162float(hi);
    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
    const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
    *(__nv_bfloat16 *)(B + wg_off(a, tid)) = hi;
    *(__nv_bfloat16 *)(B + wg_off(32 + a, tid)) = mid;
    *(__nv_bfloat16 *)(B + wg_off(64 + a, tid)) = lo;
  }
}

// STAGE: kStageCells (any grid), kStageRunsLabels / kStageRunsCounts (8-cell runs of level 1 / coarser levels)
enum { kStageCells = 0, kStageRunsLabels = 1, kStageRunsCounts = 2 };
template <int STAGE>
__global__ void __launch_bounds__(kWgThreads) k_cconv_wgrad_tc(const uint8_t *__restrict__ lab,
                                                             const ushort2 *__restrict__ counts, Dims d,
                                                             const float *__restrict__ v, const float *__restrict__ g,
                                                             double *__restrict__ part, int *err) {
  using namespace umma;
  extern __shared__ uint8_t wg_raw[];
  uint8_t *sm = (uint8_t *)(((uintptr_t)wg_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *mbar = (uint64_t *)(sm + 2 * kWgBufBytes);
  uint32_t *s_tmem = (uint32_t *)(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  // zero both buffers once: the padding rows are never written again
  for (int i = tid; i < 2 * kWgBufBytes / 16; i += kWgThreads) ((uint4 *)sm)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) {
    tmem_alloc(s_tmem, kWgTmemCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_mbar_init();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *s_tmem;
  const uint32_t idesc = idesc_bf16(kWgRowsA, kWgRowsB);
  const long long n = d.n();
  const long long nch = (n + kWgCells - 1) / kWgCells;
  uint32_t phase[2] = {0u, 0u};
  int issued[2] = {0, 0};  // commits not yet waited for, per buffer
  bool aborted = false;
  int i = 0;
  for (long long ch = blockIdx.x; ch < nch && !aborted; ch += gridDim.x, ++i) {
    const int b = i & 1;
    if (issued[b]) {  // the MMAs of two chunks ago read this buffer
      const bool ok = mbar_wait_bounded(&mbar[b], phase[b], umma::kWaitNs);
      if (__syncthreads_or(!ok)) {  // still outstanding: waited for once more below
        aborted = true;
        break;
      }
      phase[b] ^= 1u;
      issued[b] = 0;
    }
    uint8_t *A = sm + b * kWgBufBytes, *B = A + kWgABytes;
    if (STAGE == kStageRunsLabels) wg_store_run<true>(wg_load_run<true>(lab, counts, d, v, g, ch, tid), A, B);
    else if (STAGE == kStageRunsCounts) wg_store_run<false>(wg_load_run<false>(lab, counts, d, v, g, ch, tid), A, B);
    else wg_stage_cells(lab, counts, d, v, g, ch, A, B, tid);
    fence_proxy_async_smem();  // the generic stores, before the tensor core reads them
    fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < kWgCells / 16; ++kk) {
        const uint64_t ad = smem_desc_kmajor(smem_u32(A + kk * 256), 128, kWgSBO);
        const uint64_t bd = smem_desc_kmajor(smem_u32(B + kk * 256), 128, kWgSBO);
        mma_bf16_ss(tmem, ad, bd, idesc, (i > 0 || kk > 0) ? 1u : 0u);
      }
      umma_commit(&mbar[b]);
    }
    issued[b] = 1;
  }
  // the last commits of both buffers
  for (int b = 0; b < 2; ++b)
    if (issued[b]) {
      const bool ok = mbar_wait_bounded(&mbar[b], phase[b], umma::kWaitNs);
      if (!ok) aborted = true;
    }
  aborted = __syncthreads_or(aborted);
  fence_after_sync();
  if (aborted) {
    if (tid == 0 && err) atomicExch(err, 1);
  } else if (i == 0) {
    for (int o = tid; o < kWG; o += kWgThreads) part[(size_t)blockIdx.x * kWG + o] = 0.0;
  } else if (warp < 2) {
    uint32_t c[3][32];
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
#pragma unroll
    for (int sgrp = 0; sgrp < 3; ++sgrp) tmem_ld32(tmem + lane_off + 32 * sgrp, c[sgrp]);
    tmem_wait_ld();
    if (tid < 55) {
#pragma unroll
      for (int a = 0; a < 27; ++a) {
        const float s = (__uint_as_float(c[0][a]) + __uint_as_float(c[1][a])) + __uint_as_float(c[2][a]);
        part[(size_t)blockIdx.x * kWG + a * 55 + tid] = (double)s;
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kWgTmemCols);
}

// Sum the block partials of the weight gradient into out[1485] in a fixed
// order: a CTA takes 32 consecutive outputs, its warp i the blocks i, i + 8,
// ..., and the eight warp sums are added in order.
constexpr int kWFSlices = 8;
__global__ void __launch_bounds__(kWFSlices * 32) k_wgrad_final(const double *__restrict__ part, int nblocks,
                                                                double *__restrict__ out) {
  __shared__ double sm[kWFSlices][32];
  const int lane = threadIdx.x & 31, sl = threadIdx.x >> 5;
  const int o = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (o < kWG)
    for (int b = sl; b < nblocks; b += kWFSlices) s += part[(size_t)b * kWG + o];
  sm[sl][lane] = s;
  __syncthreads();
  if (sl == 0 && o < kWG) {
    double t = 0.0;
#pragma unroll
    for (int i = 0; i < kWFSlices; ++i) t += sm[i][lane];
    out[o] = t;
  }
}

// Adjoint of 2x2x2 average pooling: fine(p) = coarse(parent(p)) / 8, added into gf.
__global__ void k_pool_adjoint_add(const float *__restrict__ gc, Dims fine, float *__restrict__ gf) {
  const long long n = fine.n();
  const int cx = fine.nx / 2, cy = fine.ny / 2;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(p, fine, x, y, z);
    gf[p] += 0.125f * gc[((long long)(z >> 1) * cy + (y >> 1)) * cx + (x >> 1)];
  }
}

// Weight of coarse index X in the x2 linear upsampling of fine index f (half-
// pixel centres, edge clamp): the sum of the tap weights of f that hit X.
__device__ __forceinline__ float up_weight(int f, int X, int nc) {
  const int j = f >> 1;
  int i0, i1;
  float w1;
  if (f & 1) {
    i0 = j;
    i1 = j + 1 < nc ? j + 1 : nc - 1;
    w1 = 0.25f;
  } else if (j > 0) {
    i0 = j - 1;
    i1 = j;
    w1 = 0.75f;
  } else {
    i0 = 0;
    i1 = 0;
    w1 = 0.f;
  }
  return (i0 == X ? 1.f - w1 : 0.f) + (i1 == X ? w1 : 0.f);
}

// Adjoint of the x2 trilinear interpolation (gather over the fine cells whose
// taps reach each coarse cell), added into gc.
__global__ void k_interp_adjoint_add(const float *__restrict__ gfine, Dims coarse, float *__restrict__ gc) {
  const long long n = coarse.n();
  const int fx = coarse.nx * 2, fy = coarse.ny * 2, fz = coarse.nz * 2;
  for (long long P = (long long)blockIdx.x * blockDim.x + threadIdx.x; P < n; P += (long long)gridDim.x * blockDim.x) {
    int X, Y, Z;
    cell_xyz(P, coarse, X, Y, Z);
    float acc = 0.f;
    for (int z = 2 * Z - 1; z <= 2 * Z + 2; ++z) {
      if (z < 0 || z >= fz) continue;
      const float wz = up_weight(z, Z, coarse.nz);
      if (wz == 0.f) continue;
      for (int y = 2 * Y - 1; y <= 2 * Y + 2; ++y) {
        if (y < 0 || y >= fy) continue;
        const float wy = up_weight(y, Y, coarse.ny);
        if (wy == 0.f) continue;
        for (int x = 2 * X - 1; x <= 2 * X + 2; ++x) {
          if (x < 0 || x >= fx) continue;
          const float wx = up_weight(x, X, coarse.nx);
          if (wx == 0.f) continue;
          acc += wz * wy * wx * gfine[((long long)z * fy + y) * fx + x];
        }
      }
    }
    gc[P] += acc;
  }
}

// Plain dot product partials (deterministic, FP64 above the thread).
__global__ void __launch_bounds__(kRedThreads) k_dot2(const float *__restrict__ a, const float *__restrict__ b,
                                                      const float *__restrict__ c, long long n,
                                                      double *__restrict__ part) {
  double v[2] = {0.0, 0.0};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    v[0] += (double)a[p] * b[p];
    if (c) v[1] += (double)a[p] * c[p];
  }
  block_sum_store<2>(v, part + (size_t)blockIdx.x * 2);
}

// The pairs of dots of several levels in two launches (blockIdx.y = the level's
// index; each level with the block count, grid stride and fixed-order partial
// sum of k_dot2 / k_dot2_final, so the results are those of a launch per level).
__global__ void __launch_bounds__(kRedThreads) k_dot2_levels(const __grid_constant__ Dot2Levels D,
                                                             double *__restrict__ part) {
  const int l = D.l0 + blockIdx.y;
  const int nb = D.nb[l];
  if ((int)blockIdx.x >= nb) return;  // the whole block
  const float *__restrict__ a = D.a[l], *__restrict__ b = D.b[l], *__restrict__ c = D.c[l];
  const long long n = D.n[l];
  double v[2] = {0.0, 0.0};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)nb * blockDim.x) {
    v[0] += (double)a[p] * b[p];
    if (c) v[1] += (double)a[p] * c[p];
  }
  block_sum_store<2>(v, part + ((size_t)blockIdx.y * kRedMaxBlocks + blockIdx.x) * 2);
}
__global__ void k_dot2_levels_final(const __grid_constant__ Dot2Levels D, const double *part) {
  const int l = D.l0 + blockIdx.x;
  double t[2];
  reduce_partials<2>(part + (size_t)blockIdx.x * kRedMaxBlocks * 2, D.nb[l], t);
  if (threadIdx.x == 0) {
    D.out[l][0] = t[0];
    D.out[l][1] = t[1];
  }
  if (D.stats_src[l] && threadIdx.x < 54) D.stats_dst[l][threadIdx.x] = D.stats_src[l][threadIdx.x];
}

__global__ void k_dot2_final(const double *part, int nblocks, double *out) {
  double t[2];
  reduce_partials<2>(part, nblocks, t);
  if (threadIdx.x == 0) {
    out[0] = t[0];
    out[1] = t[1];
  }
}

// out = alpha * a + beta * b (masked to fluid when lab != null).
__global__ void k_axpby(const uint8_t *__restrict__ lab, long long n, float alpha, const float *__restrict__ a,
                        float beta, const float *__restrict__ b, float *__restrict__ out) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    float v = alpha * a[p] + (b ? beta * b[p] : 0.f);
    if (lab && lab[p] != kFluid) v = 0.f;
    out[p] = v;
  }
}

// out = alpha[0] * a + beta * b (b optional; zero off fluid when lab is given)
// with alpha a device scalar (an Aff coefficient of the current image).
__global__ void k_axpby_dev(const uint8_t *__restrict__ lab, long long n, const double *__restrict__ alpha,
                            const float *__restrict__ a, float beta, const float *__restrict__ b,
                            float *__restrict__ out) {
  const float al = (float)alpha[0];
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    float v = al * a[p] + (b ? beta * b[p] : 0.f);
    if (lab && lab[p] != kFluid) v = 0.f;
    out[p] = v;
  }
}

// out = alpha * a (masked) with a device scalar alpha = scale / sqrt(*norm2) (loss gradient).
__global__ void k_scale_by_inv_norm(const uint8_t *__restrict__ lab, long long n, float scale,
                                    const double *__restrict__ norm2, const float *__restrict__ a,
                                    float *__restrict__ out) {
  const double nn = *norm2;
  const float alpha = nn > 0.0 ? (float)(scale / sqrt(nn)) : 0.f;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
    out[p] = (lab && lab[p] != kFluid) ? 0.f : alpha * a[p];
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
void launch_materialize_K(const uint8_t *lab, const ushort2 *counts, Dims d, const CConvW *w, float *K,
                          cudaStream_t s) {
  k_materialize_K<<<gridn(d.n(), 128), 128, 0, s>>>(lab, counts, d, w, K);
}
void launch_cconv_store_K(const uint8_t *lab, const ushort2 *counts, Dims d, const CConvW &w, const float *kpure,
                          float full, const float *v, int mask_input, int round_k, float *K, float *out,
                          cudaStream_t s) {
  const long long tiles = (d.n() + 31) / 32;
  long long g = (tiles + kSKWarps - 1) / kSKWarps;
  if (g > 148LL * 16) g = 148LL * 16;
  if (g < 1) g = 1;
  PureK pk;
  memcpy(&pk, kpure, sizeof(pk));
  auto go = [&](auto kern) {
    kern<<<(int)g, kSKWarps * 32, 0, s>>>(lab, counts, d, w, pk, full, v, mask_input, K, out);
  };
  const bool rows = d.nx % 32 == 0;  // a warp's 32 cells in one grid row
  if (round_k) rows ? go(k_cconv_store_K<true, true>) : go(k_cconv_store_K<true, false>);
  else rows ? go(k_cconv_store_K<false, true>) : go(k_cconv_store_K<false, false>);
}
void launch_cconv_store_K_tc(const uint8_t *lab, const ushort2 *counts, Dims d, const uint8_t *wsplit, int nsplit,
                             const float *kpure, float full, const float *v, int mask_input, int round_k, float *K,
                             float *out, int *err, int num_sms, cudaStream_t s) {
  const long long nch = (d.n() + kSTCells - 1) / kSTCells;
  long long g = (long long)num_sms * 4;  // up to four CTAs per SM by registers; 64 TMEM columns each
  if (g > nch) g = nch;
  if (g < 1) g = 1;
  PureK pk;
  memcpy(&pk, kpure, sizeof(pk));
  auto go = [&](auto kern) {
    kern<<<(int)g, kSTCells, 0, s>>>(lab, counts, d, wsplit, nsplit, pk, full, v, mask_input, K, out, err);
  };
  if (lab) round_k ? go(k_cconv_store_K_tc<true, kSrcLabels>) : go(k_cconv_store_K_tc<false, kSrcLabels>);
  else round_k ? go(k_cconv_store_K_tc<true, kSrcCounts>) : go(k_cconv_store_K_tc<false, kSrcCounts>);
}
void launch_cconv_transpose(const float *K, const float *g, Dims d, float *gv, cudaStream_t s) {
  k_cconv_transpose<<<gridn(d.n(), 256), 256, 0, s>>>(K, g, d, gv);
}
int wgrad_blocks(Dims d) {
  long long nb = (d.n() + kWGBatch - 1) / kWGBatch;
  if (nb > 148 * 4) nb = 148 * 4;
  return (int)(nb < 1 ? 1 : nb);
}
void launch_cconv_wgrad(const uint8_t *lab, const ushort2 *counts, Dims d, const float *v, const float *g,
                        double *part, double *out, cudaStream_t s) {
  const int nb = wgrad_blocks(d);
  k_cconv_wgrad<<<nb, 256, 0, s>>>(lab, counts, d, v, g, part);
  k_wgrad_final<<<(kWG + 31) / 32, kWFSlices * 32, 0, s>>>(part, nb, out);
}
// The tensor-core weight gradient (levels with counts <= 256 per cell); `err`
// is set if an MMA wait timed out.  Two CTAs per SM (112 KB of shared memory
// and 128 TMEM columns each).
void launch_cconv_wgrad_tc(const uint8_t *lab, const ushort2 *counts, Dims d, const float *v, const float *g,
                           double *part, double *out, int *err, int num_sms, cudaStream_t s) {
  static int configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !configured[dev]) {
    cudaFuncSetAttribute(k_cconv_wgrad_tc<kStageCells>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmem);
    cudaFuncSetAttribute(k_cconv_wgrad_tc<kStageRunsLabels>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmem);
    cudaFuncSetAttribute(k_cconv_wgrad_tc<kStageRunsCounts>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmem);
    configured[dev] = 1;
  }
  const long long nch = (d.n() + kWgCells - 1) / kWgCells;
  long long nb = (long long)num_sms * 2;
  if (nb > nch) nb = nch;
  if (nb < 1) nb = 1;
  // runs of 8 cells: rows of a multiple of 8 cells, and sources aligned for
  // the 8- and 16-byte loads (the level buffers are; user labels may not be)
  const bool runs = d.nx % 8 == 0 && ((uintptr_t)lab % 8) == 0 && ((uintptr_t)counts % 16) == 0 &&
                    ((uintptr_t)v % 16) == 0 && ((uintptr_t)g % 16) == 0;
  auto go = [&](auto kern) { kern<<<(int)nb, kWgThreads, kWgSmem, s>>>(lab, counts, d, v, g, part, err); };
  if (!runs) go(k_cconv_wgrad_tc<kStageCells>);
  else if (lab) go(k_cconv_wgrad_tc<kStageRunsLabels>);
  else go(k_cconv_wgrad_tc<kStageRunsCounts>);
  k_wgrad_final<<<(kWG + 31) / 32, kWFSlices * 32, 0, s>>>(part, (int)nb, out);
}
void launch_pool_adjoint_add(const float *gc, Dims fine, float *gf, cudaStream_t s) {
  k_pool_adjoint_add<<<gridn(fine.n(), 256), 256, 0, s>>>(gc, fine, gf);
}
void launch_interp_adjoint_add(const float *gfine, Dims coarse, float *gc, cudaStream_t s) {
  k_interp_adjoint_add<<<gridn(coarse.n(), 256), 256, 0, s>>>(gfine, coarse, gc);
}
void launch_dot2_levels(const Dot2Levels &D, double *part, cudaStream_t s) {
  if (D.count < 1) return;
  Dot2Levels P = D;
  int nbmax = 1;
  for (int i = 0; i < D.count; ++i) {
    P.nb[D.l0 + i] = red_blocks(D.n[D.l0 + i]);
    if (P.nb[D.l0 + i] > nbmax) nbmax = P.nb[D.l0 + i];
  }
  k_dot2_levels<<<dim3((unsigned)nbmax, (unsigned)D.count), kRedThreads, 0, s>>>(P, part);
  k_dot2_levels_final<<<D.count, kRedThreads, 0, s>>>(P, part);
}
void launch_dot2(const float *a, const float *b, const float *c, long long n, double *part, double *out,
                 cudaStream_t s) {
  const int nb = red_blocks(n);
  k_dot2<<<nb, kRedThreads, 0, s>>>(a, b, c, n, part);
  k_dot2_final<<<1, kRedThreads, 0, s>>>(part, nb, out);
}
void launch_axpby(const uint8_t *lab, long long n, float alpha, const float *a, float beta, const float *b, float *out,
                  cudaStream_t s) {
  k_axpby<<<gridn(n, 256), 256, 0, s>>>(lab, n, alpha, a, beta, b, out);
}
void launch_axpby_dev(const uint8_t *lab, long long n, const double *alpha, const float *a, float beta,
                      const float *b, float *out, cudaStream_t s) {
  k_axpby_dev<<<gridn(n, 256), 256, 0, s>>>(lab, n, alpha, a, beta, b, out);
}
void launch_scale_by_inv_norm(const uint8_t *lab, long long n, float scale, const double *norm2, const float *a,
                              float *out, cudaStream_t s) {
  k_scale_by_inv_norm<<<gridn(n, 256), 256, 0, s>>>(lab, n, scale, norm2, a, out);
}
int wgrad_outputs() { return kWG; }

// *acc |= *flag (the label check of one training example into the batch's flag).
__global__ void k_or_flag(const unsigned int *__restrict__ flag, unsigned int *__restrict__ acc) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && *flag) *acc = 1u;
}
void launch_or_flag(const unsigned int *flag, unsigned int *acc, cudaStream_t s) { k_or_flag<<<1, 32, 0, s>>>(flag, acc); }

}  // namespace nps

namespace nps {

// ---------------------------------------------------------------------------
// Lanczos helpers (training right-hand sides): dot products of a vector with
// the m columns of a basis, and linear combinations of basis columns.
// ---------------------------------------------------------------------------
// Block partials of the dots sum_p Q[j][p] w[p], j < m: basis columns in
// groups of 8 (w read once per group), FP32 products summed in runs of 32
// elements per thread, runs and threads summed in FP64, one partial per
// (block, column) in a fixed order.
__global__ void __launch_bounds__(256) k_multidot(const float *__restrict__ Q, long long n, int m,
                                                  const float *__restrict__ w, double *__restrict__ part) {
  __shared__ double sred[8][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j0 = 0; j0 < m; j0 += 8) {
    const int jn = m - j0 < 8 ? m - j0 : 8;
    double acc[8];
    float run[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      acc[t] = 0.0;
      run[t] = 0.f;
    }
    int cnt = 0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
      const float wp = w[p];
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (t < jn) run[t] = fmaf(Q[(size_t)(j0 + t) * n + p], wp, run[t]);
      if (++cnt == 32) {
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          acc[t] += (double)run[t];
          run[t] = 0.f;
        }
        cnt = 0;
      }
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      acc[t] = warp_sum(acc[t] + (double)run[t]);
      if (lane == 0) sred[warp][t] = acc[t];
    }
    __syncthreads();
    if (threadIdx.x < jn) {
      double t = 0.0;
      for (int w8 = 0; w8 < 8; ++w8) t += sred[w8][threadIdx.x];
      part[(size_t)blockIdx.x * m + j0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

__global__ void k_multidot_final(const double *__restrict__ part, int nblocks, int m, double *__restrict__ out) {
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += part[(size_t)b * m + j];
    out[j] = t;
  }
}

// out[p] = beta * out[p] + sum_j c[j] Q[j][p]  (c in device memory, FP64):
// FP32 products in four interleaved FP32 sums, combined in FP64.
__global__ void k_combine_basis(const float *__restrict__ Q, long long n, int m, const double *__restrict__ c,
                                float beta, float *__restrict__ out) {
  extern __shared__ float cs[];
  for (int j = threadIdx.x; j < m; j += blockDim.x) cs[j] = (float)c[j];
  __syncthreads();
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    int j = 0;
    for (; j + 4 <= m; j += 4) {
#pragma unroll
      for (int t = 0; t < 4; ++t) a[t] = fmaf(cs[j + t], Q[(size_t)(j + t) * n + p], a[t]);
    }
    for (; j < m; ++j) a[0] = fmaf(cs[j], Q[(size_t)j * n + p], a[0]);
    double acc = (double)(a[0] + a[1]) + (double)(a[2] + a[3]);
    if (beta != 0.f) acc += (double)beta * out[p];
    out[p] = (float)acc;
  }
}

void launch_multidot(const float *Q, long long n, int m, const float *w, double *part, double *out, cudaStream_t s) {
  long long nb = (n + 255) / 256;
  if (nb > 148 * 4) nb = 148 * 4;
  k_multidot<<<(int)nb, 256, 0, s>>>(Q, n, m, w, part);
  k_multidot_final<<<1, 128, 0, s>>>(part, (int)nb, m, out);
}

void launch_combine_basis(const float *Q, long long n, int m, const double *c, float beta, float *out,
                          cudaStream_t s) {
  long long nb = (n + 255) / 256;
  if (nb > 148 * 16) nb = 148 * 16;
  k_combine_basis<<<(int)nb, 256, sizeof(float) * (size_t)m, s>>>(Q, n, m, c, beta, out);
}

}  // namespace nps
