// CConv (Sec. 4.2.1) on the tensor cores, z-marching form.
//
// A CTA owns a 16 x 8 column of cells (one MMA tile of M = 128 per z-plane)
// and marches along z through a chunk of planes.  Per plane z:
//   * features: each thread builds its cell's 64 BF16 features from the
//     3x3x3 window of packed image codes (fluid / air BF16 bits per cell,
//     exact integers) -- planes z-1 and z are kept in registers, only plane
//     z+1 is read from the shared-memory plane ring -- and writes them into
//     its TMEM lane (A operand, double-buffered);
//   * one thread issues the kernel-generation MMAs D = F . W^T (W in shared
//     memory, BF16; three BF16 terms in the FP32 form) into a TMEM
//     accumulator (double-buffered), completion tracked by an mbarrier;
//   * meanwhile the threads apply the taps of plane z-1 (whose MMA finished
//     during the previous step): out = sum_a K_a v(p+a), with the vector
//     window of planes z-2..z in registers (plane z read from the ring);
//   * the next planes' image codes and vector values are prefetched from
//     global memory into registers at the start of the step and written to
//     the ring at its end, so global latency overlaps the step's work.
// Optional fusions: a 2x2x2 average-pooling epilogue (CConv1 of levels
// < L writes the next level's input), and an interpolation prologue (CConv2
// reads the coarse level and interpolates x2 trilinearly while loading).
//
// Every wait on an mbarrier is bounded (1 s); on time-out the kernel records
// an error, waits (bounded) for its MMAs in flight, frees its TMEM and exits.
#include <cuda_bf16.h>

#include "nps_common.cuh"
#include "nps_kernels.h"
#include "umma.cuh"

namespace nps {

using namespace umma;

namespace {

constexpr int TX = 16, TY = 8;           // x-y tile: 128 cells = MMA M
constexpr int PX = TX + 2, PY = TY + 2;  // plane with a one-cell halo: 18 x 10
constexpr int PLANE = PX * PY;           // 180 entries
constexpr int RING = 4;                  // planes kept in shared memory
constexpr int ZCHUNK = 32;               // planes per work unit (even: pooling pairs)
constexpr int MARCH_TMEM_COLS = 128;     // A0 [0,32) A1 [32,64) D0 [64,96) D1 [96,128)
constexpr int MARCH_CTAS_PER_SM = 4;     // 4 x 128 TMEM columns = 512
constexpr int MARCH_SMEM_TARGET = 46 * 1024;  // per-CTA shared memory incl. padding: 5 x 47 KB > 228 KB

struct MarchParams {
  Dims dm;                 // dims of this level
  const uint8_t *lab;      // level-1 labels (nullptr at coarser levels)
  const ushort2 *counts;   // fluid / air counts at levels >= 2
  const uint8_t *wsplit;   // NSPLIT x 4 KB of W in the canonical K-major layout
  const float *v;          // input vector of this level (when not interpolating)
  const float *coarse;     // coarse vector (dims / 2) interpolated on load
  const float *vscale;     // optional device scalar multiplying the input
  int mask_input;          // zero the input off fluid (level-1 CConv1)
  float *out;              // output of this level
  float *pooled;           // optional 2x2x2 mean of the output (dims / 2)
  const SolveState *st;
  int *err;
};

// Packed image code of one cell: BF16 bits of the air count in the high half,
// of the fluid count in the low half; zero outside the grid (solid padding).
__device__ __forceinline__ uint32_t image_code(const MarchParams &P, int x, int y, int z) {
  const Dims &d = P.dm;
  if (x < 0 || y < 0 || z < 0 || x >= d.nx || y >= d.ny || z >= d.nz) return 0u;
  const long long p = ((long long)z * d.ny + y) * d.nx + x;
  if (P.lab) {
    const uint8_t l = P.lab[p];
    return l == kFluid ? 0x00003F80u : (l == kAir ? 0x3F800000u : 0u);
  }
  const ushort2 c = P.counts[p];
  return bf16_bits_small(c.x) | (bf16_bits_small(c.y) << 16);
}

// x2 linear upsampling taps (half-pixel centres, edge clamp) along one axis.
__device__ __forceinline__ void up_taps_m(int f, int nc, int &i0, int &i1, float &w1) {
  const int j = f >> 1;
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
}

// Input vector value at a cell of this level (zero outside the grid).
template <bool INTERP>
__device__ __forceinline__ float input_value(const MarchParams &P, int x, int y, int z, float sc) {
  const Dims &d = P.dm;
  if (x < 0 || y < 0 || z < 0 || x >= d.nx || y >= d.ny || z >= d.nz) return 0.f;
  if (INTERP) {
    const int cx = d.nx >> 1, cy = d.ny >> 1, cz = d.nz >> 1;
    int x0, x1, y0, y1, z0, z1;
    float wx, wy, wz;
    up_taps_m(x, cx, x0, x1, wx);
    up_taps_m(y, cy, y0, y1, wy);
    up_taps_m(z, cz, z0, z1, wz);
    const float *c = P.coarse;
    auto C = [&](int zz, int yy, int xx) { return __ldg(c + ((long long)zz * cy + yy) * cx + xx); };
    const float c00 = (1.f - wx) * C(z0, y0, x0) + wx * C(z0, y0, x1);
    const float c01 = (1.f - wx) * C(z0, y1, x0) + wx * C(z0, y1, x1);
    const float c10 = (1.f - wx) * C(z1, y0, x0) + wx * C(z1, y0, x1);
    const float c11 = (1.f - wx) * C(z1, y1, x0) + wx * C(z1, y1, x1);
    const float c0 = (1.f - wy) * c00 + wy * c01;
    const float c1 = (1.f - wy) * c10 + wy * c11;
    return (1.f - wz) * c0 + wz * c1;
  }
  const long long p = ((long long)z * d.ny + y) * d.nx + x;
  float val = P.v[p] * sc;
  if (P.mask_input && P.lab[p] != kFluid) val = 0.f;
  return val;
}

}  // namespace

template <int NSPLIT, bool INTERP>
__global__ void __launch_bounds__(128, 4) k_cconv_march(MarchParams P) {
  if (P.st && P.st->done) return;
  __shared__ __align__(1024) uint8_t sW[NSPLIT * kBBytes];
  __shared__ uint32_t sCode[RING][PLANE];
  __shared__ float sV[RING][PLANE];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5;
  const int tx = tid % TX, ty = tid / TX;
  {
    const uint4 *src = (const uint4 *)P.wsplit;
    uint4 *dst = (uint4 *)sW;
    for (int i = tid; i < NSPLIT * kBBytes / 16; i += blockDim.x) dst[i] = src[i];
  }
  if (warp == 0) {
    tmem_alloc(&s_tmem, MARCH_TMEM_COLS);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_mbar_init();
    s_abort = 0;
  }
  fence_proxy_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = s_tmem;
  const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
  const uint32_t idesc = idesc_bf16(kTileM, kN);
  const float sc = P.vscale ? *P.vscale : 1.f;
  uint32_t phase[2] = {0u, 0u};

  const Dims dm = P.dm;
  const int ntx = (dm.nx + TX - 1) / TX, nty = (dm.ny + TY - 1) / TY, nzc = (dm.nz + ZCHUNK - 1) / ZCHUNK;
  const int units = ntx * nty * nzc;
  // the two ring entries this thread loads / stores per plane
  const int e0 = tid, e1 = tid + 128;  // e1 valid when < PLANE
  bool aborted = false;

  for (int u = blockIdx.x; u < units && !aborted; u += gridDim.x) {
    const int utx = u % ntx, uty = (u / ntx) % nty, uz = u / (ntx * nty);
    const int x0 = utx * TX, y0 = uty * TY;
    const int zs = uz * ZCHUNK, ze = min(zs + ZCHUNK, dm.nz);
    auto ex = [&](int e) { return x0 - 1 + e % PX; };
    auto ey = [&](int e) { return y0 - 1 + e / PX; };
    // prologue: image planes zs-1, zs, zs+1 and vector planes zs-1, zs
    for (int pz = zs - 1; pz <= zs + 1; ++pz) {
      uint32_t *row = sCode[(pz + RING) % RING];
      row[e0] = image_code(P, ex(e0), ey(e0), pz);
      if (e1 < PLANE) row[e1] = image_code(P, ex(e1), ey(e1), pz);
    }
    for (int pz = zs - 1; pz <= zs; ++pz) {
      float *row = sV[(pz + RING) % RING];
      row[e0] = input_value<INTERP>(P, ex(e0), ey(e0), pz, sc);
      if (e1 < PLANE) row[e1] = input_value<INTERP>(P, ex(e1), ey(e1), pz, sc);
    }
    __syncthreads();
    uint32_t fA[9], fB[9];  // image codes of planes z-1, z (3x3 neighbourhood)
    float vA[9], vB[9];     // vector values of planes z-2, z-1
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const int e = (ty + j / 3) * PX + (tx + j % 3);
      fA[j] = sCode[(zs - 1 + RING) % RING][e];
      fB[j] = sCode[zs % RING][e];
      vA[j] = 0.f;
      vB[j] = sV[(zs - 1 + RING) % RING][e];
    }
    float psum = 0.f;

    for (int z = zs; z <= ze; ++z) {
      const bool do_feat = z < ze, do_apply = z > zs;
      const int b = z & 1;
      // (a) prefetch image plane z+2 and vector plane z+1 into registers
      uint32_t pc0 = 0, pc1 = 0;
      float pv0 = 0.f, pv1 = 0.f;
      if (do_feat) {
        pc0 = image_code(P, ex(e0), ey(e0), z + 2);
        if (e1 < PLANE) pc1 = image_code(P, ex(e1), ey(e1), z + 2);
        pv0 = input_value<INTERP>(P, ex(e0), ey(e0), z + 1, sc);
        if (e1 < PLANE) pv1 = input_value<INTERP>(P, ex(e1), ey(e1), z + 1, sc);
      }
      // (b) features of plane z -> TMEM A[b]
      uint32_t fC[9];
#pragma unroll
      for (int j = 0; j < 9; ++j) fC[j] = sCode[(z + 1) % RING][(ty + j / 3) * PX + (tx + j % 3)];
      if (do_feat) {
        uint32_t win[27];
#pragma unroll
        for (int j = 0; j < 9; ++j) {
          win[j] = fA[j];
          win[9 + j] = fB[j];
          win[18 + j] = fC[j];
        }
        uint32_t fw[32];
        build_feature_words(win, fw);
        tmem_st32(tmem + 32 * b + lane_off, fw);
        tmem_wait_st();
      }
      // (c) vector plane z
      float vC[9];
#pragma unroll
      for (int j = 0; j < 9; ++j) vC[j] = sV[z % RING][(ty + j / 3) * PX + (tx + j % 3)];
      fence_before_sync();
      __syncthreads();
      // (d) kernel-generation MMAs of plane z
      if (do_feat && tid == 0) {
        fence_after_sync();
#pragma unroll
        for (int s = 0; s < NSPLIT; ++s)
#pragma unroll
          for (int kk = 0; kk < kK / 16; ++kk) {
            const uint64_t bd = smem_desc_kmajor(smem_u32(sW + s * kBBytes + kk * 2 * kLBO), kLBO, kSBO);
            mma_bf16_ts(tmem + 64 + 32 * b, tmem + 32 * b + kk * 8, bd, idesc, (s | kk) != 0);
          }
        umma_commit(&mbar[b]);
      }
      // (e) apply the taps of plane z-1
      if (do_apply) {
        const int pb = b ^ 1;
        // warp-uniform success flag (the pooling shuffles below need all lanes)
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&mbar[pb], phase[pb], kWaitNs));
        if (ok) phase[pb] ^= 1u;
        else s_abort = 1;
        fence_after_sync();
        if (ok) {
          uint32_t kr[32];
          tmem_ld32(tmem + 64 + 32 * pb + lane_off, kr);
          tmem_wait_ld();
          if (NSPLIT == 1) {  // BF16 form: every kernel value rounded to BF16
#pragma unroll
            for (int j = 0; j < 27; ++j)
              kr[j] = __float_as_uint(__bfloat162float(__float2bfloat16_rn(__uint_as_float(kr[j]))));
          }
          float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
          for (int j = 0; j < 9; ++j) {
            s0 = fmaf(__uint_as_float(kr[j]), vA[j], s0);
            s1 = fmaf(__uint_as_float(kr[9 + j]), vB[j], s1);
            s2 = fmaf(__uint_as_float(kr[18 + j]), vC[j], s2);
          }
          const float acc = (s0 + s1) + s2;
          const int gx = x0 + tx, gy = y0 + ty, gz = z - 1;
          const bool inside = gx < dm.nx && gy < dm.ny;
          if (inside) P.out[((long long)gz * dm.ny + gy) * dm.nx + gx] = acc;
          if (P.pooled) {
            if (((gz - zs) & 1) == 0) {
              psum = acc;
            } else {
              float s2 = psum + acc;
              s2 += __shfl_xor_sync(0xffffffffu, s2, 1);   // x pair
              s2 += __shfl_xor_sync(0xffffffffu, s2, 16);  // y pair (rows 2w, 2w+1 of warp w)
              if (inside && !(tx & 1) && !(ty & 1)) {
                const int cx = dm.nx >> 1, cy = dm.ny >> 1;
                P.pooled[((long long)(gz >> 1) * cy + (gy >> 1)) * cx + (gx >> 1)] = 0.125f * s2;
              }
            }
          }
        }
      }
      // (f) prefetched planes -> ring
      if (do_feat) {
        sCode[(z + 2) % RING][e0] = pc0;
        if (e1 < PLANE) sCode[(z + 2) % RING][e1] = pc1;
        sV[(z + 1) % RING][e0] = pv0;
        if (e1 < PLANE) sV[(z + 1) % RING][e1] = pv1;
      }
      fence_before_sync();
      __syncthreads();
      if (s_abort) {
        aborted = true;
        break;
      }
#pragma unroll
      for (int j = 0; j < 9; ++j) {
        fA[j] = fB[j];
        fB[j] = fC[j];
        vA[j] = vB[j];
        vB[j] = vC[j];
      }
    }
  }
  if (aborted) {
    if (tid == 0) atomicExch(P.err, 1);
    // MMAs possibly in flight complete the phases not yet consumed
    (void)mbar_wait_bounded(&mbar[0], phase[0], kWaitNs);
    (void)mbar_wait_bounded(&mbar[1], phase[1], kWaitNs);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, MARCH_TMEM_COLS);
}

// ---------------------------------------------------------------------------
template <int NSPLIT, bool INTERP>
static void launch_march_t(const MarchParams &P, int num_sms, cudaStream_t s) {
  static int pad = -1;
  if (pad < 0) {
    cudaFuncAttributes a;
    cudaFuncGetAttributes(&a, k_cconv_march<NSPLIT, INTERP>);
    pad = MARCH_SMEM_TARGET - (int)a.sharedSizeBytes;
    if (pad < 0) pad = 0;
  }
  const int units = ((P.dm.nx + TX - 1) / TX) * ((P.dm.ny + TY - 1) / TY) * ((P.dm.nz + ZCHUNK - 1) / ZCHUNK);
  int grid = num_sms * MARCH_CTAS_PER_SM;
  if (grid > units) grid = units;
  k_cconv_march<NSPLIT, INTERP><<<grid, 128, pad, s>>>(P);
}

void launch_cconv_march(int nsplit, const uint8_t *lab, const ushort2 *counts, Dims dm, const uint8_t *wsplit,
                        const float *v, const float *coarse, const float *vscale, int mask_input, float *out,
                        float *pooled, const SolveState *st, int *err, int num_sms, cudaStream_t s) {
  MarchParams P;
  P.dm = dm;
  P.lab = lab;
  P.counts = counts;
  P.wsplit = wsplit;
  P.v = v;
  P.coarse = coarse;
  P.vscale = vscale;
  P.mask_input = mask_input;
  P.out = out;
  P.pooled = pooled;
  P.st = st;
  P.err = err;
  const bool interp = coarse != nullptr;
  if (nsplit == 1) {
    if (interp) launch_march_t<1, true>(P, num_sms, s);
    else launch_march_t<1, false>(P, num_sms, s);
  } else {
    if (interp) launch_march_t<3, true>(P, num_sms, s);
    else launch_march_t<3, false>(P, num_sms, s);
  }
}

}  // namespace nps
