// The coarse tail of the network (Alg. 2 below a size threshold) in one
// launch of one thread-block cluster.
//
// At the coarse levels of a large grid (32^3 cells and fewer: levels 4-6 of a
// 256^3 grid) a CConv or an interpolation is a few microseconds of latency and
// almost no work, and each level costs two or three dependent launches.  Here
// the levels T..L run as the phases of one kernel on one cluster of kTailCtas
// CTAs, separated by the cluster's hardware barrier (release / acquire at
// cluster scope, so every phase sees the previous phase's global stores):
//   down:  x1^l = CConv1^l(r1^l) and r1^(l+1) = Pool(x1^l)   (l = T .. L-1)
//          x^L  = CConv1^L(r1^L)
//   up:    x^l = c1^l x1^l + c2^l CConv2^l(Interp(x^(l+1)))   (l = L-1 .. T)
//   out:   r2^(T-1) = Interp(x^T), the input of the finer level's CConv2.
// The per-cell kernels of these levels are materialised once per solve
// (k_tail_kernels: 27 FP32 words per cell, tap-major, rounded to BF16 in the
// BF16 form), so a phase is a plain 27-point gather per cell.  Every phase
// first stages its input field in each CTA's shared memory (at most 32,768
// cells, 128 KB), so the gathers hit shared memory; the CConv2 input is
// interpolated by each CTA for the whole level into its own shared memory (a
// little redundant arithmetic instead of a barrier and a global round trip).
// The interpolation applies the per-axis rule of the finer levels'
// interpolation kernel (x, then y, then z, with the same FMAs), so its output
// is identical.  Inside a solve the launch returns at once when the state
// says converged.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "nps_common.cuh"
#include "nps_kernels.h"

namespace cg = cooperative_groups;

namespace nps {

namespace {

constexpr int kTailThreads = 1024;

__device__ __forceinline__ float2 tail_img(const uint8_t *lab, const ushort2 *counts, const Dims &d, int x, int y,
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

// One axis of the x2 upsampling for fine index f of a coarse axis of n cells:
// the two coarse indices and how they combine (0: the first alone, 1:
// lerp_lo, 2: lerp_hi), as in the finer levels' interpolation kernel.
__device__ __forceinline__ void up_axis(int f, int n, int &i0, int &i1, int &mode) {
  const int j = f >> 1;
  if (f & 1) {
    i0 = j;
    i1 = min(j + 1, n - 1);
    mode = 2;
  } else if (j > 0) {
    i0 = j - 1;
    i1 = j;
    mode = 1;
  } else {
    i0 = i1 = 0;
    mode = 0;
  }
}
__device__ __forceinline__ float up_mix(int mode, float a, float b) {
  return mode == 0 ? a : (mode == 1 ? lerp_lo(a, b) : lerp_hi(a, b));
}

// Stage a level's field (n floats, written by an earlier phase or launch) in
// shared memory; the caller synchronises the CTA before reading it.
__device__ __forceinline__ void stage(float *dst, const float *src, int n) {
  if ((n & 3) == 0) {
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    for (int i = threadIdx.x; i < (n >> 2); i += blockDim.x) d4[i] = __ldcg(s4 + i);
  } else {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = __ldcg(src + i);
  }
}

// sum_a K_a(p) v(p + a) with v staged in shared memory (zero outside the
// grid) and the kernels tap-major in global memory (K[a n + p]).
__device__ __forceinline__ float smem_cconv(const float *__restrict__ K, const float *v, const Dims &d, int x, int y,
                                            int z) {
  const int n = (int)d.n();
  const int p = (z * d.ny + y) * d.nx + x;
  float k[27];
#pragma unroll
  for (int a = 0; a < 27; ++a) k[a] = __ldg(K + (size_t)a * n + p);
  float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int a = 0; a < 27; ++a) {
    const int xx = x + a % 3 - 1, yy = y + (a / 3) % 3 - 1, zz = z + a / 9 - 1;
    const bool in = xx >= 0 && yy >= 0 && zz >= 0 && xx < d.nx && yy < d.ny && zz < d.nz;
    s[a / 9] = fmaf(k[a], in ? v[(zz * d.ny + yy) * d.nx + xx] : 0.f, s[a / 9]);
  }
  return (s[0] + s[1]) + s[2];
}

// Fine cell (x, y, z) of the x2 upsampling of the coarse field c staged in
// shared memory (dims dc): along x on each coarse row, then y, then z.
__device__ __forceinline__ float smem_interp(const float *c, const Dims &dc, int x, int y, int z) {
  int x0, x1, mx, y0, y1, my, z0, z1, mz;
  up_axis(x, dc.nx, x0, x1, mx);
  up_axis(y, dc.ny, y0, y1, my);
  up_axis(z, dc.nz, z0, z1, mz);
  float yz[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int zc = k ? z1 : z0;
    float xr[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const float *row = c + (zc * dc.ny + (j ? y1 : y0)) * dc.nx;
      xr[j] = up_mix(mx, row[x0], row[x1]);
    }
    yz[k] = up_mix(my, xr[0], xr[1]);
  }
  return up_mix(mz, yz[0], yz[1]);
}

}  // namespace

// Per-cell kernels K_a(p) = Bp[a] + sum_l (Wf[a][l] nF(p+l) + Wa[a][l] nA(p+l))
// of one CConv block at a tail level, tap-major (K[a n + p]); the BF16 form
// rounds each value to BF16 (nearest even).
__global__ void __launch_bounds__(128) k_tail_kernels(const uint8_t *__restrict__ lab, const ushort2 *__restrict__ counts,
                                                      Dims d, const CConvW *__restrict__ w, int round_k,
                                                      float *__restrict__ K) {
  __shared__ CConvW sw;
  {
    const float *src = (const float *)w;
    float *dst = (float *)&sw;
    for (int i = threadIdx.x; i < (int)(sizeof(CConvW) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int n = (int)d.n();
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(p, d, x, y, z);
    float nf[27], na[27];
#pragma unroll
    for (int l = 0; l < 27; ++l) {
      const float2 f = tail_img(lab, counts, d, x + l % 3 - 1, y + (l / 3) % 3 - 1, z + l / 9 - 1);
      nf[l] = f.x;
      na[l] = f.y;
    }
#pragma unroll 1
    for (int a = 0; a < 27; ++a) {
      float k = sw.bp[a];
#pragma unroll
      for (int l = 0; l < 27; ++l) k = fmaf(sw.wf[a][l], nf[l], fmaf(sw.wa[a][l], na[l], k));
      if (round_k) k = __bfloat162float(__float2bfloat16_rn(k));
      K[(size_t)a * n + p] = k;
    }
  }
}

__global__ void __launch_bounds__(kTailThreads, 1) k_tail(const __grid_constant__ TailParams P) {
  if (P.st && P.st->done) return;  // the same for every CTA of the cluster
  extern __shared__ __align__(16) float tsm[];
  cg::cluster_group cluster = cg::this_cluster();
  const int T = P.T, L = P.L;
  const int rank = (int)cluster.block_rank(), nct = (int)cluster.num_blocks();
  const int tid = rank * kTailThreads + (int)threadIdx.x;
  const int nthr = nct * kTailThreads;
  // down: x1^l = CConv1^l(r1^l) and r1^(l+1) = Pool(x1^l).  Thread t takes
  // child t & 7 of pooling block t >> 3, so a block's eight children are
  // eight neighbouring lanes and the mean is a three-step lane reduction.
  for (int l = T; l < L; ++l) {
    const Dims d = P.dims[l], dc = P.dims[l + 1];
    stage(tsm, P.r1[l], (int)d.n());
    __syncthreads();
    const int n = (int)d.n();
    for (int q0 = tid & ~31; q0 < n; q0 += nthr) {  // warp-uniform trip count (the shuffles)
      const int q = q0 + (tid & 31);
      const bool act = q < n;
      const int blk = q >> 3, c = q & 7;
      int bx = 0, by = 0, bz = 0;
      if (act) cell_xyz(blk, dc, bx, by, bz);
      const int x = 2 * bx + (c & 1), y = 2 * by + ((c >> 1) & 1), z = 2 * bz + (c >> 2);
      float o = act ? smem_cconv(P.k1[l], tsm, d, x, y, z) : 0.f;
      if (act) P.x1[l][(z * d.ny + y) * d.nx + x] = o;
      o += __shfl_xor_sync(0xffffffffu, o, 1);
      o += __shfl_xor_sync(0xffffffffu, o, 2);
      o += __shfl_xor_sync(0xffffffffu, o, 4);
      if (act && c == 0) P.r1[l + 1][blk] = 0.125f * o;
    }
    cluster.sync();
  }
  // coarsest: x^L = CConv1^L(r1^L)
  {
    const Dims d = P.dims[L];
    const int n = (int)d.n();
    stage(tsm, P.r1[L], n);
    __syncthreads();
    for (int p = tid; p < n; p += nthr) {
      int x, y, z;
      cell_xyz(p, d, x, y, z);
      P.x1[L][p] = smem_cconv(P.k1[L], tsm, d, x, y, z);
    }
    cluster.sync();
  }
  // up: x^l = c1 x1^l + c2 CConv2^l(Interp(x^(l+1))).  Every CTA interpolates
  // the whole level into its own shared memory (the levels here are small),
  // so the interpolated field needs no barrier of its own.
  for (int l = L - 1; l >= T; --l) {
    const Dims d = P.dims[l], dc = P.dims[l + 1];
    const int n = (int)d.n(), nc = (int)dc.n();
    float *sc = tsm, *sf = tsm + ((nc + 3) & ~3);
    stage(sc, l + 1 == L ? P.x1[L] : P.xc[l + 1], nc);
    __syncthreads();
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
      int x, y, z;
      cell_xyz(p, d, x, y, z);
      sf[p] = smem_interp(sc, dc, x, y, z);
    }
    __syncthreads();
    const float c1 = (float)P.affc[2 * l], c2 = (float)P.affc[2 * l + 1];
    for (int p = tid; p < n; p += nthr) {
      int x, y, z;
      cell_xyz(p, d, x, y, z);
      P.xc[l][p] = fmaf(c1, __ldcg(P.x1[l] + p), c2 * smem_cconv(P.k2[l], sf, d, x, y, z));
    }
    cluster.sync();
  }
  // out: r2^(T-1) = Interp(x^T), the finer level's CConv2 input
  {
    const Dims d = P.dims[T - 1], dc = P.dims[T];
    const int nc = (int)dc.n();
    stage(tsm, T == L ? P.x1[L] : P.xc[T], nc);
    __syncthreads();
    const int n = (int)d.n();
    for (int p = tid; p < n; p += nthr) {
      int x, y, z;
      cell_xyz(p, d, x, y, z);
      P.r2[T - 1][p] = smem_interp(tsm, dc, x, y, z);
    }
  }
}

void launch_tail_kernels(const uint8_t *lab, const ushort2 *counts, Dims d, const CConvW *w, int round_k, float *K,
                         cudaStream_t s) {
  long long b = (d.n() + 127) / 128;
  if (b > 148 * 8) b = 148 * 8;
  k_tail_kernels<<<(int)(b < 1 ? 1 : b), 128, 0, s>>>(lab, counts, d, w, round_k, K);
}

// Shared memory of the tail: the largest field a phase stages (the level-T
// input, or a coarse field beside its interpolated level).
size_t tail_smem_bytes(const TailParams &P) {
  size_t m = 0;
  for (int l = P.T; l <= P.L; ++l) {
    const size_t n = (size_t)P.dims[l].n();
    const size_t nc = l < P.L ? (size_t)P.dims[l + 1].n() : 0;
    m = std::max(m, n);
    if (l < P.L) m = std::max(m, ((nc + 3) & ~(size_t)3) + n);
  }
  return m * sizeof(float);
}

int launch_tail(const TailParams &P, cudaStream_t s) {
  const size_t smem = tail_smem_bytes(P);
  static int configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !configured[dev]) {
    if (cudaFuncSetAttribute(k_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, kTailMaxSmem) != cudaSuccess)
      return 1;
    configured[dev] = 1;
  }
  if (smem > (size_t)kTailMaxSmem) return 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kTailCtas, 1, 1);
  cfg.blockDim = dim3(kTailThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kTailCtas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_tail, P) == cudaSuccess ? 0 : 1;
}

}  // namespace nps
