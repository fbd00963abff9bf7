// CConv (Sec. 4.2.1) with per-solve kernel caching of the non-uniform cells.
//
// The per-cell kernel K_a(p) = Bp[a] + sum_l (Wf[a][l] nF(p+l) + Wa[a][l] nA(p+l))
// depends only on the image, which is fixed during a solve.  When the whole
// 3x3x3 window of a cell carries the same (nF, nA) pair (with the solid
// padding outside the grid), the sum collapses exactly to
//   K_a = Bp[a] + nF * SWf[a] + nA * SWa[a],   SWf[a] = sum_l Wf[a][l],
// so the kernel is a function of the cell's own class.  Only the cells with a
// mixed window (about 7% of the cells at level 1, 16% at level 2 and 32% at
// level 3 of a 256^3 scene) need the full generation.  Per solve:
//   classify  - per 32-plane column chunk (x, y, zc): a bit mask of the mixed
//               cells and an offset into the kernel cache (atomic allocation);
//   generate  - K of every mixed cell (FP32 CUDA-core contraction of the 54
//               image features, the same arithmetic as the FP32 CConv),
//               stored as 28 FP32 (FP32 form) or 32 BF16 (BF16 form) values.
// Per iteration, the apply kernel marches along z through a 16 x 8 column
// tile: the vector window of planes z-1, z in registers, plane z+1 from a
// shared-memory ring (prefetched one step ahead), K held in registers while
// the class does not change and loaded from the cache for mixed cells.
// Fusions: zero-masking and scaling of the level-1 input, 2x2x2 average
// pooling of the output (CConv1), trilinear interpolation of the input from
// the coarser level (CConv2) and the combination x = c1 x1 + c2 x2 (CConv2 of
// levels >= 2).
#include <cuda_bf16.h>

#include "nps_common.cuh"
#include "nps_kernels.h"

namespace nps {

namespace {

constexpr int TX = 16, TY = 8;           // column tile (pooling pairs: lanes ^1 in x, ^16 in y)
constexpr int PX = TX + 2, PY = TY + 2;  // plane with a one-cell halo
constexpr int PLANE = PX * PY;           // 180
constexpr int RING = 4;
constexpr int ZC = 32;                   // planes per column chunk (one mask word)

// Image key of a cell: fluid count | air count << 16 (0/1 at level 1); zero
// outside the grid (solid padding).
__device__ __forceinline__ uint32_t image_key(const uint8_t *lab, const ushort2 *counts, const Dims &d, int x, int y,
                                              int z) {
  if (x < 0 || y < 0 || z < 0 || x >= d.nx || y >= d.ny || z >= d.nz) return 0u;
  const long long p = ((long long)z * d.ny + y) * d.nx + x;
  if (lab) {
    const uint8_t l = lab[p];
    return l == kFluid ? 1u : (l == kAir ? 0x10000u : 0u);
  }
  const ushort2 c = counts[p];
  return (uint32_t)c.x | ((uint32_t)c.y << 16);
}

}  // namespace

// ---------------------------------------------------------------------------
// Setup 1: classification.  One thread per column chunk (x, y, zc).
// ---------------------------------------------------------------------------
__global__ void k_classify(const uint8_t *__restrict__ lab, const ushort2 *__restrict__ counts, Dims d,
                           uint32_t *__restrict__ mask, uint32_t *__restrict__ offset, unsigned *total) {
  const int nzc = (d.nz + ZC - 1) / ZC;
  const long long ncol = (long long)d.nx * d.ny * nzc;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncol; c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % d.nx);
    const int y = (int)((c / d.nx) % d.ny);
    const int zc = (int)(c / ((long long)d.nx * d.ny));
    const int zs = zc * ZC, ze = min(zs + ZC, d.nz);
    uint32_t m = 0;
    for (int z = zs; z < ze; ++z) {
      const uint32_t k0 = image_key(lab, counts, d, x, y, z);
      bool uni = true;
      for (int l = 0; l < 27 && uni; ++l)
        uni = image_key(lab, counts, d, x + l % 3 - 1, y + (l / 3) % 3 - 1, z + l / 9 - 1) == k0;
      if (!uni) m |= 1u << (z - zs);
    }
    mask[c] = m;
    offset[c] = m ? atomicAdd(total, (unsigned)__popc(m)) : 0u;
  }
}

// ---------------------------------------------------------------------------
// Setup 2: kernel generation for the mixed cells of one CConv block.
// FP32 form: 28 floats per cell (K_0..K_26, 0); BF16 form: 32 BF16 values.
// ---------------------------------------------------------------------------
template <bool BF16>
__global__ void __launch_bounds__(128) k_generate(const uint8_t *__restrict__ lab, const ushort2 *__restrict__ counts,
                                                  Dims d, const CConvW *__restrict__ w,
                                                  const uint32_t *__restrict__ mask,
                                                  const uint32_t *__restrict__ offset, void *__restrict__ cache) {
  __shared__ CConvW sw;
  {
    const float *src = (const float *)w;
    float *dst = (float *)&sw;
    for (int i = threadIdx.x; i < (int)(sizeof(CConvW) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int nzc = (d.nz + ZC - 1) / ZC;
  const long long ncol = (long long)d.nx * d.ny * nzc;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncol; c += (long long)gridDim.x * blockDim.x) {
    uint32_t m = mask[c];
    if (!m) continue;
    const int x = (int)(c % d.nx);
    const int y = (int)((c / d.nx) % d.ny);
    const int zs = (int)(c / ((long long)d.nx * d.ny)) * ZC;
    uint32_t idx = offset[c];
    while (m) {
      const int bit = __ffs(m) - 1;
      m &= m - 1;
      const int z = zs + bit;
      float nf[27], na[27];
#pragma unroll
      for (int l = 0; l < 27; ++l) {
        const uint32_t k = image_key(lab, counts, d, x + l % 3 - 1, y + (l / 3) % 3 - 1, z + l / 9 - 1);
        nf[l] = (float)(k & 0xFFFFu);
        na[l] = (float)(k >> 16);
      }
      float K[28];
#pragma unroll 1
      for (int a = 0; a < 27; ++a) {
        float kk = sw.bp[a];
#pragma unroll
        for (int l = 0; l < 27; ++l) kk = fmaf(sw.wf[a][l], nf[l], fmaf(sw.wa[a][l], na[l], kk));
        K[a] = kk;
      }
      K[27] = 0.f;
      if (BF16) {
        uint4 *dst = (uint4 *)((__nv_bfloat16 *)cache + (size_t)idx * 32);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          uint32_t wv[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int a0 = q * 8 + 2 * e, a1 = a0 + 1;
            const float f0 = a0 < 27 ? K[a0] : 0.f, f1 = a1 < 27 ? K[a1] : 0.f;
            wv[e] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(f0)) |
                    ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(f1)) << 16);
          }
          dst[q] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
      } else {
        float4 *dst = (float4 *)((float *)cache + (size_t)idx * 28);
#pragma unroll
        for (int q = 0; q < 7; ++q) dst[q] = make_float4(K[4 * q], K[4 * q + 1], K[4 * q + 2], K[4 * q + 3]);
      }
      ++idx;
    }
  }
}

// ---------------------------------------------------------------------------
// Per-iteration apply: a z-marching 27-point stencil.
//   uniform-window cell: out = conv(Bp, v) + nF conv(SWf, v) + nA conv(SWa, v)
//                        (constant coefficients, read from the kernel
//                        parameters by the FMAs themselves)
//   mixed-window cell:   out = sum_a K_a(p) v(p+a) with K from the cache
// The vector planes (18 x 10 with halo) go through a register queue DQ planes
// deep into a 4-plane shared-memory ring, so every global load has DQ steps
// to arrive; the cell's own image key is queued the same way.
// ---------------------------------------------------------------------------
constexpr int DQ = 4;  // prefetch distance in planes

struct StencilParams {
  Dims dm;
  const uint8_t *lab;      // level 1
  const ushort2 *counts;   // levels >= 2
  const uint32_t *mask, *offset;
  const void *cache;       // mixed-cell kernels (FP32 x 28 or BF16 x 32)
  const float *v;          // input of this level (zero off fluid at level 1)
  const float *vscale;     // optional scale of the output (the input normalisation)
  float *out;              // output (x1, x2 or the combination)
  float *pooled;           // optional 2x2x2 mean of the output
  const float *x1;         // optional: out = c1 * x1 + c2 * CConv(...)
  const double *c12;
  const SolveState *st;
  float cb[27], cf[27], ca[27];  // uniform-window kernel = cb + nF cf + nA ca
};

template <bool BF16C>
__global__ void __launch_bounds__(128, 5) k_cconv_stencil(const __grid_constant__ StencilParams P) {
  if (P.st && P.st->done) return;
  __shared__ float sV[RING][PLANE];
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const float sc = P.vscale ? *P.vscale : 1.f;
  const float c1 = P.x1 ? (float)P.c12[0] : 0.f, c2 = P.x1 ? (float)P.c12[1] : 1.f;
  const Dims dm = P.dm;
  const long long nxy = (long long)dm.nx * dm.ny;
  const int ntx = (dm.nx + TX - 1) / TX, nty = (dm.ny + TY - 1) / TY, nzc = (dm.nz + ZC - 1) / ZC;
  const int units = ntx * nty * nzc;
  const bool has1 = tid + 128 < PLANE;

  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    const int utx = u % ntx, uty = (u / ntx) % nty, uz = u / (ntx * nty);
    const int x0 = utx * TX, y0 = uty * TY;
    const int zs = uz * ZC, ze = min(zs + ZC, dm.nz);
    // the two plane entries this thread moves: x-y position and validity
    const int ex0 = x0 - 1 + tid % PX, ey0 = y0 - 1 + tid / PX;
    const int ex1 = x0 - 1 + (tid + 128) % PX, ey1 = y0 - 1 + (tid + 128) / PX;
    const bool ok0 = ex0 >= 0 && ey0 >= 0 && ex0 < dm.nx && ey0 < dm.ny;
    const bool ok1 = has1 && ex1 >= 0 && ey1 >= 0 && ex1 < dm.nx && ey1 < dm.ny;
    const float *b0 = P.v + ((long long)ey0 * dm.nx + ex0);
    const float *b1 = P.v + ((long long)ey1 * dm.nx + ex1);
    auto ld0 = [&](int z) { return (ok0 && z >= 0 && z < dm.nz) ? __ldg(b0 + z * nxy) : 0.f; };
    auto ld1 = [&](int z) { return (ok1 && z >= 0 && z < dm.nz) ? __ldg(b1 + z * nxy) : 0.f; };
    const int gx = x0 + tx, gy = y0 + ty;
    const bool inside = gx < dm.nx && gy < dm.ny;
    auto key = [&](int z) -> uint32_t {
      if (!inside || z >= ze) return 0u;
      const long long p = (long long)z * nxy + (long long)gy * dm.nx + gx;
      if (P.lab) {
        const uint8_t l = __ldg(P.lab + p);
        return l == kFluid ? 1u : (l == kAir ? 0x10000u : 0u);
      }
      const ushort2 c = P.counts[p];
      return (uint32_t)c.x | ((uint32_t)c.y << 16);
    };
    // prologue: ring planes zs-1 .. zs+1, queues for planes zs+2 .. zs+1+DQ (vector), zs .. zs+DQ-1 (keys)
    for (int pz = zs - 1; pz <= zs + 1; ++pz) {
      sV[(pz + RING) % RING][tid] = ld0(pz);
      if (has1) sV[(pz + RING) % RING][tid + 128] = ld1(pz);
    }
    float q0[DQ], q1[DQ];
    uint32_t kq[DQ];
#pragma unroll
    for (int i = 0; i < DQ; ++i) {
      q0[i] = ld0(zs + 2 + i);
      q1[i] = has1 ? ld1(zs + 2 + i) : 0.f;
      kq[i] = key(zs + i);
    }
    uint32_t cmask = 0, coff = 0;
    if (inside) {
      const long long col = ((long long)uz * dm.ny + gy) * dm.nx + gx;
      cmask = P.mask[col];
      coff = P.offset[col];
    }
    __syncthreads();
    float vA[9], vB[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const int e = (ty + j / 3) * PX + (tx + j % 3);
      vA[j] = sV[(zs - 1 + RING) % RING][e];
      vB[j] = sV[zs % RING][e];
    }
    float psum = 0.f;
    for (int z = zs; z < ze; ++z) {
      float vC[9];
#pragma unroll
      for (int j = 0; j < 9; ++j) vC[j] = sV[(z + 1) % RING][(ty + j / 3) * PX + (tx + j % 3)];
      const uint32_t k0 = kq[0];
      const int bit = z - zs;
      float acc;
      if (cmask >> bit & 1u) {
        // mixed window: cached kernel
        const uint32_t idx = coff + __popc(cmask & ((1u << bit) - 1u));
        float K[28];
        if (BF16C) {
          const uint4 *src = (const uint4 *)((const __nv_bfloat16 *)P.cache + (size_t)idx * 32);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint4 wv = __ldg(src + q);
            const uint32_t ww[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int a0 = q * 8 + 2 * e;
              if (a0 < 28) K[a0] = __uint_as_float(ww[e] << 16);
              if (a0 + 1 < 28) K[a0 + 1] = __uint_as_float(ww[e] & 0xFFFF0000u);
            }
          }
        } else {
          const float4 *src = (const float4 *)((const float *)P.cache + (size_t)idx * 28);
#pragma unroll
          for (int q = 0; q < 7; ++q) {
            const float4 f = __ldg(src + q);
            K[4 * q] = f.x;
            K[4 * q + 1] = f.y;
            K[4 * q + 2] = f.z;
            K[4 * q + 3] = f.w;
          }
        }
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
          s0 = fmaf(K[j], vA[j], s0);
          s1 = fmaf(K[9 + j], vB[j], s1);
          s2 = fmaf(K[18 + j], vC[j], s2);
        }
        acc = (s0 + s1) + s2;
      } else {
        // uniform window: K = cb + nF cf + nA ca
        float sb = 0.f, sf = 0.f, sa = 0.f;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
          sb = fmaf(P.cb[j], vA[j], fmaf(P.cb[9 + j], vB[j], fmaf(P.cb[18 + j], vC[j], sb)));
          sf = fmaf(P.cf[j], vA[j], fmaf(P.cf[9 + j], vB[j], fmaf(P.cf[18 + j], vC[j], sf)));
          sa = fmaf(P.ca[j], vA[j], fmaf(P.ca[9 + j], vB[j], fmaf(P.ca[18 + j], vC[j], sa)));
        }
        acc = fmaf((float)(k0 & 0xFFFFu), sf, fmaf((float)(k0 >> 16), sa, sb));
      }
      acc *= sc;
      if (inside) {
        const long long p = (long long)z * nxy + (long long)gy * dm.nx + gx;
        if (P.x1) acc = fmaf(c1, __ldg(P.x1 + p), c2 * acc);
        P.out[p] = acc;
      }
      if (P.pooled) {
        if ((bit & 1) == 0) {
          psum = acc;
        } else {
          float t = psum + acc;
          t += __shfl_xor_sync(0xffffffffu, t, 1);
          t += __shfl_xor_sync(0xffffffffu, t, 16);
          if (inside && !(tx & 1) && !(ty & 1)) {
            const int cx = dm.nx >> 1, cy = dm.ny >> 1;
            P.pooled[((long long)(z >> 1) * cy + (gy >> 1)) * cx + (gx >> 1)] = 0.125f * t;
          }
        }
      }
      // queues: plane z+2 -> ring; advance; issue plane z+2+DQ (vector) and z+DQ (key)
      sV[(z + 2) % RING][tid] = q0[0];
      if (has1) sV[(z + 2) % RING][tid + 128] = q1[0];
#pragma unroll
      for (int i = 0; i < DQ - 1; ++i) {
        q0[i] = q0[i + 1];
        q1[i] = q1[i + 1];
        kq[i] = kq[i + 1];
      }
      q0[DQ - 1] = ld0(z + 2 + DQ);
      q1[DQ - 1] = has1 ? ld1(z + 2 + DQ) : 0.f;
      kq[DQ - 1] = key(z + DQ);
      __syncthreads();
#pragma unroll
      for (int j = 0; j < 9; ++j) {
        vA[j] = vB[j];
        vB[j] = vC[j];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
long long cached_columns(Dims d) { return (long long)d.nx * d.ny * ((d.nz + ZC - 1) / ZC); }

void launch_classify(const uint8_t *lab, const ushort2 *counts, Dims d, uint32_t *mask, uint32_t *offset,
                     unsigned *total, cudaStream_t s) {
  const long long nc = cached_columns(d);
  long long g = (nc + 127) / 128;
  if (g > 148LL * 16) g = 148LL * 16;
  k_classify<<<(int)(g < 1 ? 1 : g), 128, 0, s>>>(lab, counts, d, mask, offset, total);
}

void launch_generate(bool bf16, const uint8_t *lab, const ushort2 *counts, Dims d, const CConvW *w,
                     const uint32_t *mask, const uint32_t *offset, void *cache, cudaStream_t s) {
  const long long nc = cached_columns(d);
  long long g = (nc + 127) / 128;
  if (g > 148LL * 16) g = 148LL * 16;
  if (bf16) k_generate<true><<<(int)(g < 1 ? 1 : g), 128, 0, s>>>(lab, counts, d, w, mask, offset, cache);
  else k_generate<false><<<(int)(g < 1 ? 1 : g), 128, 0, s>>>(lab, counts, d, w, mask, offset, cache);
}

int cached_entry_bytes(bool bf16) { return bf16 ? 64 : 112; }

void launch_cconv_cached(bool bf16, const uint8_t *lab, const ushort2 *counts, Dims dm, const float *uni_host,
                         const uint32_t *mask, const uint32_t *offset, const void *cache, const float *v,
                         const float *vscale, float *out, float *pooled, const float *x1, const double *c12,
                         const SolveState *st, int num_sms, cudaStream_t s) {
  StencilParams P;
  P.dm = dm;
  P.lab = lab;
  P.counts = counts;
  P.mask = mask;
  P.offset = offset;
  P.cache = cache;
  P.v = v;
  P.vscale = vscale;
  P.out = out;
  P.pooled = pooled;
  P.x1 = x1;
  P.c12 = c12;
  P.st = st;
  for (int a = 0; a < 27; ++a) {
    P.cb[a] = uni_host[a];
    P.cf[a] = uni_host[27 + a];
    P.ca[a] = uni_host[54 + a];
  }
  const int units = ((dm.nx + TX - 1) / TX) * ((dm.ny + TY - 1) / TY) * ((dm.nz + ZC - 1) / ZC);
  int grid = num_sms * 5;
  if (grid > units) grid = units;
  if (bf16) k_cconv_stencil<true><<<grid, 128, 0, s>>>(P);
  else k_cconv_stencil<false><<<grid, 128, 0, s>>>(P);
}

}  // namespace nps
