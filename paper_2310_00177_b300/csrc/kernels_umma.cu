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

namespace nps {

namespace umma {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on an mbarrier phase: gives up after `limit_ns` of wall time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && globaltimer() - t0 > limit_ns) return false;
  }
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// D[tmem] (+)= A[tmem] . B[smem desc]^T, kind::f16 (BF16 inputs, FP32 accumulate).
__device__ __forceinline__ void mma_bf16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

#define NPS_R32(a)                                                                                          \
  "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]), "=r"(a[8]), \
      "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15]), "=r"(a[16]),   \
      "=r"(a[17]), "=r"(a[18]), "=r"(a[19]), "=r"(a[20]), "=r"(a[21]), "=r"(a[22]), "=r"(a[23]), "=r"(a[24]),  \
      "=r"(a[25]), "=r"(a[26]), "=r"(a[27]), "=r"(a[28]), "=r"(a[29]), "=r"(a[30]), "=r"(a[31])
#define NPS_W32(a)                                                                                            \
  "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[8]), "r"(a[9]), \
      "r"(a[10]), "r"(a[11]), "r"(a[12]), "r"(a[13]), "r"(a[14]), "r"(a[15]), "r"(a[16]), "r"(a[17]),           \
      "r"(a[18]), "r"(a[19]), "r"(a[20]), "r"(a[21]), "r"(a[22]), "r"(a[23]), "r"(a[24]), "r"(a[25]),           \
      "r"(a[26]), "r"(a[27]), "r"(a[28]), "r"(a[29]), "r"(a[30]), "r"(a[31])

// Thread i of warp w writes lane 32w+i, columns [col, col+32) (32-bit each).
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      NPS_W32(v)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : NPS_R32(v)
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major, no swizzle (canonical
// interleaved layout of 8-row x 16-byte core matrices): start address,
// leading-dimension byte offset (between core matrices along K), stride
// byte offset (between 8-row groups along N), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc_kmajor(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // version
  return d;                // base offset 0, lbo mode 0, layout SWIZZLE_NONE (0)
}

// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major,
// N = n, M = m.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

constexpr int kTileM = 128;       // cells per brick (MMA M)
constexpr int kN = 32;            // taps padded to 32 (MMA N)
constexpr int kK = 64;            // features padded to 64 (4 MMAs of K = 16)
constexpr int kBBytes = kN * kK * 2;  // one split of W, 4 KB
constexpr int kLBO = 128, kSBO = 1024;  // canonical K-major offsets of the W tile
constexpr int kTmemCols = 64;     // A: columns [0,32), D: columns [32,64)
constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s
constexpr int kCtasPerSm = 6;                 // 6 x 64 TMEM columns <= 512
constexpr int kResidencyPad = 24 * 1024;      // 228 KB / (24 KB + static) -> <= 7 CTAs per SM

// Brick of 8 (x) x 4 (y) x 4 (z) cells; thread t <-> cell (t%8, (t/8)%4, t/32),
// so warp w holds the z-plane w of the brick and TMEM lanes 32w..32w+31.
constexpr int BX = 8, BY = 4, BZ = 4;
constexpr int HX = BX + 2, HY = BY + 2, HZ = BZ + 2;
constexpr int kHalo = HX * HY * HZ;  // 360

__device__ __forceinline__ uint32_t bf16_bits_small(unsigned n) {
  // exact BF16 of a small non-negative integer (n <= 256)
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn((float)n));
}

}  // namespace umma

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
