// CConv (Sec. 4.2.1) with the per-cell kernel generation on the 5th-generation
// tensor cores (tcgen05, sm_103a).
//
// For a brick of 128 cells (8 x 4 x 4), the kernel-generation step
//   K_a(p) = Bp[a] + sum_l ( Wf[a][l] nF(p+l) + Wa[a][l] nA(p+l) ),
// is the dense contraction D[128 x 32] = F[128 x 64] . W^T[64 x 32] with
//   F[p][j] = nF(p + l_j) (j < 27), nA(p + l_{j-27}) (27 <= j < 54), 1 (j = 54), 0 else
//   W[a][j] = Wf / Wa / Bp accordingly (a < 27; rows 27..31 zero).
// The image features are small integers (0/1 at level 1, counts <= 64 at
// levels 2-3) and therefore exact in BF16; only W is rounded.  The BF16 form
// uses W rounded to BF16; the FP32 form splits W = W_hi + W_mid + W_lo into
// three BF16 terms and accumulates the three products in the same FP32
// accumulator, which recovers FP32 accuracy.
//
// Data path per brick: every thread builds its cell's 64 BF16 features and
// writes them into its own TMEM lane (the A operand lives in tensor memory);
// one elected thread issues the MMAs against W held in shared memory (B
// operand, K-major, no swizzle) into a 128 x 32 FP32 accumulator in TMEM; the
// threads read their 27 taps back with tcgen05.ld and apply them to the
// zero-padded vector halo held in shared memory:
//   out_p = sum_a K_a(p) v(p + a).
// Every wait on the MMA-completion mbarrier is bounded (1 s of %globaltimer);
// on time-out the kernel records an error code, waits once more (bounded),
// releases its TMEM and returns.
#include <cuda_bf16.h>

#include "nps_common.cuh"
#include "nps_kernels.h"
#include "umma.cuh"

namespace nps {



using namespace umma;

template <int NSPLIT>
__global__ void __launch_bounds__(128) k_cconv_umma(const uint8_t *__restrict__ lab, const ushort2 *__restrict__ counts,
                                                      Dims dm, const uint8_t *__restrict__ wsplit,
                                                      const float *__restrict__ v, const float *__restrict__ vscale,
                                                      int mask_input, float *__restrict__ out, const SolveState *st,
                                                      int *err) {
  if (st && st->done) return;
  __shared__ __align__(1024) uint8_t sB[NSPLIT * kBBytes];
  __shared__ float sv[kHalo];
  __shared__ uchar2 simg[kHalo];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  // W splits -> shared memory (already in the canonical layout)
  {
    const uint4 *src = (const uint4 *)wsplit;
    uint4 *dst = (uint4 *)sB;
    for (int i = tid; i < NSPLIT * kBBytes / 16; i += blockDim.x) dst[i] = src[i];
  }
  if (warp == 0) {
    tmem_alloc(&s_tmem, kTmemCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&mbar, 1);
    fence_mbar_init();
    s_abort = 0;
  }
  fence_proxy_async_smem();  // make the generic-proxy writes of sB visible to the tensor core
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = s_tmem;
  const uint32_t a_tmem = tmem;       // columns [0, 32)
  const uint32_t d_tmem = tmem + 32;  // columns [32, 64)
  const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
  const uint32_t idesc = idesc_bf16(kTileM, kN);
  const float sc = vscale ? *vscale : 1.f;

  const int ntx = (dm.nx + BX - 1) / BX, nty = (dm.ny + BY - 1) / BY, ntz = (dm.nz + BZ - 1) / BZ;
  const long long ntiles = (long long)ntx * nty * ntz;
  const int cx = tid % BX, cy = (tid / BX) % BY, cz = tid / (BX * BY);
  uint32_t phase = 0;

  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int tx = (int)(tile % ntx);
    const int ty = (int)((tile / ntx) % nty);
    const int tz = (int)(tile / ((long long)ntx * nty));
    const int x0 = tx * BX, y0 = ty * BY, z0 = tz * BZ;
    // halo of image features and (scaled, zero-padded) vector values
    for (int i = tid; i < kHalo; i += blockDim.x) {
      const int hx = i % HX, hy = (i / HX) % HY, hz = i / (HX * HY);
      const int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = z0 - 1 + hz;
      uchar2 f = make_uchar2(0, 0);
      float val = 0.f;
      if (gx >= 0 && gy >= 0 && gz >= 0 && gx < dm.nx && gy < dm.ny && gz < dm.nz) {
        const long long p = ((long long)gz * dm.ny + gy) * dm.nx + gx;
        if (lab) {
          const uint8_t l = lab[p];
          f = make_uchar2(l == kFluid, l == kAir);
        } else {
          const ushort2 c = counts[p];
          f = make_uchar2((unsigned char)c.x, (unsigned char)c.y);
        }
        val = v[p] * sc;
        if (mask_input && f.x == 0) val = 0.f;
      }
      sv[i] = val;
      simg[i] = f;
    }
    __syncthreads();
    // features of this thread's cell -> its TMEM lane (A operand)
    {
      uint32_t fw[32];
      unsigned nf[27], na[27];
#pragma unroll
      for (int l = 0; l < 27; ++l) {
        const int hx = cx + l % 3, hy = cy + (l / 3) % 3, hz = cz + l / 9;
        const uchar2 f = simg[(hz * HY + hy) * HX + hx];
        nf[l] = f.x;
        na[l] = f.y;
      }
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        uint32_t lo = 0, hi = 0;
        const int j0 = 2 * c, j1 = 2 * c + 1;
        lo = j0 < 27 ? bf16_bits_small(nf[j0]) : (j0 < 54 ? bf16_bits_small(na[j0 - 27]) : (j0 == 54 ? 0x3F80u : 0u));
        hi = j1 < 27 ? bf16_bits_small(nf[j1]) : (j1 < 54 ? bf16_bits_small(na[j1 - 27]) : (j1 == 54 ? 0x3F80u : 0u));
        fw[c] = lo | (hi << 16);
      }
      tmem_st32(a_tmem + lane_off, fw);
      tmem_wait_st();
    }
    fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
#pragma unroll
      for (int s = 0; s < NSPLIT; ++s)
#pragma unroll
        for (int kk = 0; kk < kK / 16; ++kk) {
          const uint64_t bd = smem_desc_kmajor(smem_u32(sB + s * kBBytes + kk * 2 * kLBO), kLBO, kSBO);
          mma_bf16_ts(d_tmem, a_tmem + kk * 8, bd, idesc, (s | kk) != 0);
        }
      umma_commit(&mbar);
    }
    const bool ok = mbar_wait_bounded(&mbar, phase, kWaitNs);
    phase ^= 1u;
    if (!ok) s_abort = 1;
    fence_after_sync();
    __syncthreads();
    if (s_abort) break;
    // taps of this cell from TMEM, then the 27-tap apply
    uint32_t kr[32];
    tmem_ld32(d_tmem + lane_off, kr);
    tmem_wait_ld();
    float acc = 0.f;
#pragma unroll
    for (int a = 0; a < 27; ++a) {
      const int hx = cx + a % 3, hy = cy + (a / 3) % 3, hz = cz + a / 9;
      acc = fmaf(__uint_as_float(kr[a]), sv[(hz * HY + hy) * HX + hx], acc);
    }
    const int gx = x0 + cx, gy = y0 + cy, gz = z0 + cz;
    if (gx < dm.nx && gy < dm.ny && gz < dm.nz) out[((long long)gz * dm.ny + gy) * dm.nx + gx] = acc;
    fence_before_sync();
    __syncthreads();  // halo and TMEM are reused by the next brick
  }
  if (s_abort) {
    if (tid == 0) atomicExch(err, 1);
    (void)mbar_wait_bounded(&mbar, phase ^ 1u, kWaitNs);  // the MMAs still in flight, if any
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// Self-test of the tensor-core data path used above: one brick-sized MMA
// D[128 x 32] = A[128 x 64] . B[32 x 64]^T with A in TMEM (as built by the
// CConv kernel) and B in shared memory (canonical K-major layout), compared
// with a CUDA-core FP32 evaluation of the same products.  A and B hold small
// integers / exact BF16 values, so both results are exact.
__global__ void __launch_bounds__(128) k_umma_selftest(float *__restrict__ d_out, float *__restrict__ d_ref,
                                                         int *err) {
  __shared__ __align__(1024) uint8_t sB[kBBytes];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5;
  auto aval = [](int m, int k) { return (float)(((m * 7 + k * 3) % 5) - 2); };  // -2..2
  auto bval = [](int n, int k) { return (float)(((n * 5 + k * 11) % 9) - 4) * 0.125f; };
  for (int i = tid; i < kN * kK; i += blockDim.x) {
    const int n = i / kK, k = i % kK;
    const int off = (n / 8) * kSBO + (k / 8) * kLBO + (n % 8) * 16 + (k % 8) * 2;
    *(uint16_t *)(sB + off) = __bfloat16_as_ushort(__float2bfloat16_rn(bval(n, k)));
  }
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
  const uint32_t tmem = s_tmem, lane_off = (uint32_t)(warp * 32) << 16;
  uint32_t fw[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(aval(tid, 2 * c)));
    const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(aval(tid, 2 * c + 1)));
    fw[c] = lo | (hi << 16);
  }
  tmem_st32(tmem + lane_off, fw);
  tmem_wait_st();
  fence_before_sync();
  __syncthreads();
  if (tid == 0) {
    fence_after_sync();
    for (int kk = 0; kk < kK / 16; ++kk)
      mma_bf16_ts(tmem + 32, tmem + kk * 8, smem_desc_kmajor(smem_u32(sB + kk * 2 * kLBO), kLBO, kSBO),
                  idesc_bf16(kTileM, kN), kk != 0);
    umma_commit(&mbar);
  }
  const bool ok = mbar_wait_bounded(&mbar, 0, kWaitNs);
  fence_after_sync();
  if (ok) {
    uint32_t kr[32];
    tmem_ld32(tmem + 32 + lane_off, kr);
    tmem_wait_ld();
    for (int n = 0; n < kN; ++n) {
      float ref = 0.f;
      for (int k = 0; k < kK; ++k) ref += aval(tid, k) * bval(n, k);
      d_out[tid * kN + n] = __uint_as_float(kr[n]);
      d_ref[tid * kN + n] = ref;
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
    (void)mbar_wait_bounded(&mbar, 0, kWaitNs);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
static uint16_t f32_to_bf16_rne(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)(u >> 16);  // inf / nan
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7FFFu + lsb;
  return (uint16_t)(u >> 16);
}
static float bf16_to_f32(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

// Lay out W of one CConv block as NSPLIT BF16 terms in the canonical K-major
// shared-memory layout (4 KB each): row n = output tap a, column k = feature j.
void prepare_umma_weights(const CConvW &w, int nsplit, uint8_t *out) {
  memset(out, 0, (size_t)nsplit * kBBytes);
  for (int n = 0; n < 27; ++n)
    for (int k = 0; k < 55; ++k) {
      float val = k < 27 ? w.wf[n][k] : (k < 54 ? w.wa[n][k - 27] : w.bp[n]);
      const int off = (n / 8) * kSBO + (k / 8) * kLBO + (n % 8) * 16 + (k % 8) * 2;
      for (int s = 0; s < nsplit; ++s) {
        const uint16_t h = f32_to_bf16_rne(val);
        memcpy(out + (size_t)s * kBBytes + off, &h, 2);
        val = val - bf16_to_f32(h);
      }
    }
}

int umma_weight_bytes(int nsplit) { return nsplit * kBBytes; }

void launch_cconv_umma(int nsplit, const uint8_t *lab, const ushort2 *counts, Dims dm, const uint8_t *wsplit,
                       const float *v, const float *vscale, int mask_input, float *out, const SolveState *st,
                       int *err, int num_sms, cudaStream_t s) {
  const long long ntiles = (long long)((dm.nx + BX - 1) / BX) * ((dm.ny + BY - 1) / BY) * ((dm.nz + BZ - 1) / BZ);
  // At most kCtasPerSm resident CTAs per SM (so their TMEM allocations,
  // kTmemCols each, always fit in the 512 columns): the launch reserves
  // unused dynamic shared memory to cap the residency.
  long long grid = (long long)num_sms * kCtasPerSm;
  if (grid > ntiles) grid = ntiles;
  if (nsplit == 1)
    k_cconv_umma<1><<<(int)grid, 128, kResidencyPad, s>>>(lab, counts, dm, wsplit, v, vscale, mask_input, out, st,
                                                            err);
  else
    k_cconv_umma<3><<<(int)grid, 128, kResidencyPad, s>>>(lab, counts, dm, wsplit, v, vscale, mask_input, out, st,
                                                            err);
}

void launch_umma_selftest(float *d_out, float *d_ref, int *err, cudaStream_t s) {
  k_umma_selftest<<<1, 128, 0, s>>>(d_out, d_ref, err);
}

}  // namespace nps
