// CConv (Sec. 4.2.1) with per-solve kernel caching of the mixed-window cells,
// streamed through shared memory by the tensor memory accelerator (TMA).
//
// The per-cell kernel K_a(p) = Bp[a] + sum_l (Wf[a][l] nF(p+l) + Wa[a][l] nA(p+l))
// depends only on the image, which is fixed during a solve.  When the whole
// 3x3x3 window of a cell (solid padding outside the grid) is pure fluid, pure
// air or pure solid, the sum collapses to one of three constant kernels
//   K^S = Bp,  K^F = Bp + F sum_l Wf[a][l],  K^A = Bp + F sum_l Wa[a][l]
// with F = 8^(lvl-1) fine cells per cell of level lvl.  Every other cell (a
// "mixed window": 7% of the level-1 cells of a 256^3 sloshing scene) gets its
// own kernel, generated once per solve and cached in HBM.
//
// Layout of one level:
//   tiles of 32 (x) x 8 (y) cells;
//   one plane descriptor per (tile, z): for each row of the tile the bit masks
//   "mixed window", "pure-fluid window", "pure-air window" and "the cell is
//   fluid" (bit = x within the tile), and the place of the plane's kernel
//   block in the cache;
//   a kernel block holds the kernels of the plane's mixed cells in the order of
//   their bit index (row-major), tap-major: word (j, i) of a block with stride
//   cpad is tap pair j of mixed cell i (BF16 form: taps 2j and 2j+1 as a BF16
//   pair, 14 words per cell) or tap j of mixed cell i (FP32 form: 27 words per
//   cell); cpad is the mixed count rounded up to 4, so that every block starts
//   and ends on a 16-byte boundary.
//
// Per solve: k_classify (masks, block sizes, block offsets by one atomic per
// unit of 32 planes) and k_generate_tc / k_generate (the contraction of the 54
// image features and the bias of each mixed cell with the folded weights, on
// the tensor cores where the counts are exact in BF16, else on CUDA cores).
// The BF16 form rounds every kernel value to BF16, the three constant ones
// included.
//
// Per iteration: k_cconv_stream.  Each CTA marches units (a tile and a chunk
// of planes) along z, two planes per step.  One producer warp (one thread)
// loads per unit the plane descriptors (bulk copy, three buffers), and per
// step, into one of RV slots completing on one mbarrier: the 44 x 10 x 2 TMA
// box of the input planes z+1, z+2 (one-cell halo), the 36 x 8 x 2 box of x1
// (combination only) and, with a bulk copy into a circular buffer, the two
// planes' kernel blocks (contiguous in the cache).  Four consumer warps each
// own two rows of the tile: a thread keeps the 4-row x 3-column window
// columns of planes z-1, z in registers and computes the 2 x 2 cells (rows y,
// y+1; planes z, z+1) of its column, so a 2x2x2 pooling block is a pair of
// adjacent lanes.  A row whose 32 windows are all pure takes a constant
// kernel from the kernel parameters; any other row reads each lane's kernel
// from shared memory (the class tables of the three constant kernels or the
// cell's cached block), one code path for all lanes.  Slots and descriptor
// buffers are released with mbarrier arrivals; there is no CTA-wide barrier
// in the march.  Fusions: scaling by the input normalisation (level-1
// CConv1), the 2x2x2 mean pooling of the output (CConv1), the combination
// x = c1 x1 + c2 x2 (CConv2 at levels >= 2).
//
// Every wait on an mbarrier is bounded (1 s of %globaltimer, with the thread
// suspended in hardware meanwhile); a timeout sets *err, and every warp then
// leaves; the producer waits (bounded) for its copies in flight first.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "nps_common.cuh"
#include "nps_kernels.h"
#include "umma.cuh"

namespace nps {

namespace {

using umma::globaltimer;
using umma::mbar_init;
using umma::mbar_wait_bounded;
using umma::smem_u32;

constexpr int TX = 32, TY = 8, NT = TX * TY;  // tile (x, y)
constexpr int ZCG = 32;                       // planes per unit of the setup kernels
constexpr int BXW = TX + 12;                  // vector box: x0-4 .. x0+39 (start on a 16-byte boundary; the
                                              // width 44 keeps the 8x8-patch reads free of bank conflicts)
constexpr int BYH = TY + 2;                   // rows y0-1 .. y0+4
constexpr int VPLANE = BXW * BYH * 4;         // 1760 bytes per plane of the vector box
constexpr int XBW = TX + 4;                   // x1 / q box width: rows 36 words apart, so that the four
                                              // rows a warp reads of an 8x8 patch fall in distinct banks
constexpr int XBOX = XBW * TY * 2 * 4;        // 2304 bytes per x1 / q box (36 x 8 x 2)
constexpr int X1OFF = 3584;                   // x1 box in a slot (128-byte aligned, after 3520)
constexpr int SLOT = X1OFF + XBOX;            // 5888 bytes, 46 x 128
static_assert(X1OFF >= 2 * VPLANE && X1OFF % 128 == 0 && SLOT % 128 == 0 && XBOX % 128 == 0, "slot layout");
constexpr int PW = 8;                         // patch width: consumer warp w covers x in [8w, 8w+8) x 8 rows
constexpr int RV = 4;                         // step slots
constexpr int ND = 3;                         // descriptor buffers (units)
constexpr int kMetaBytes = 640;               // mbarriers, block positions, class tables, abort flag
constexpr uint64_t kWaitNs = 1000000000ull;   // 1 s

// Plane descriptor: per row w of the tile the masks {mixed window, pure-fluid
// window, pure-air window, fluid cell} (bit = x within the tile), then the
// kernel block.
struct PlaneDesc {
  uint4 row[TY];     // x: mixed, y: pure fluid, z: pure air, w: the cell is fluid
  uint32_t off;      // first cache entry of the plane's kernel block (a multiple of 4)
  uint32_t count;    // mixed cells of the plane
  uint32_t cpad;     // entries of the block: the mixed count rounded up to 4
  uint32_t patch;    // bits 2p, 2p+1: class of the 8x8 patch p (x in [8p, 8p+8)): 0 all pure solid,
                     // 1 all pure fluid, 2 all pure air, 3 anything else
  uint32_t rowbase[2];  // byte w: mixed cells in rows 0..w-1 (the rank of row w's first one)
  uint32_t pad1[2];
};
static_assert(sizeof(PlaneDesc) == 160, "plane descriptor is 160 bytes");
constexpr int DWORDS = (int)sizeof(PlaneDesc) / 4;  // 40
constexpr int DBUF = ZCG * (int)sizeof(PlaneDesc);  // one unit's descriptors

// Slots of the fused level-1 CConv2 (+ combination and orthogonalisation dots):
// the vector box, x1 and up to two q boxes of the previous directions.
// Slots of the level-1 CConv1 that also forms r_{k+1} = r_k - alpha q_k: the
// residual box and the q box of the same geometry.
constexpr int QUOFF = 3584;                   // q box (44 x 10 x 2) after the residual box
constexpr int SLOT_U = 7168;                  // 3584 + 3520 bytes rounded up to 56 x 128
static_assert(QUOFF >= 2 * VPLANE && QUOFF + 2 * VPLANE <= SLOT_U && SLOT_U % 128 == 0, "update slot layout");
constexpr int QOFF = SLOT;                    // q box j (36 x 8 x 2) at QOFF + XBOX j
constexpr int SLOT_F = SLOT + 2 * XBOX;       // 10496 bytes, 82 x 128
constexpr int kMaxFusedOrtho = 2;

template <bool BF16C, bool FUSE = false, bool UPD = false>
struct KCfg {
  static constexpr int EB = BF16C ? 56 : 108;        // bytes per cached kernel
  static constexpr int CB = BF16C ? 28672 : 55296;   // circular kernel-block buffer (>= two full planes)
  static constexpr int NRV = FUSE ? 3 : RV;          // step slots
  static constexpr int SL = FUSE ? SLOT_F : (UPD ? SLOT_U : SLOT);  // bytes per slot
  static constexpr int SMEM = NRV * SL + ND * DBUF + CB + kMetaBytes;
};
// three CTAs per SM (1 KB of shared memory reserved per CTA, 228 KB per SM) for the BF16 form
static_assert(3 * (KCfg<true, true>::SMEM + 1024) <= 228 * 1024, "three fused BF16 CTAs per SM");
static_assert(3 * (KCfg<true, false, true>::SMEM + 1024) <= 228 * 1024, "three update-fused BF16 CTAs per SM");

// Image key of a cell: fluid count | air count << 16 (0/1 at level 1); zero
// outside the grid (solid padding).
__device__ __forceinline__ uint32_t image_key(const uint8_t *lab, const ushort2 *counts, const Dims &d, int x, int y,
                                              int z) {
  if (x < 0 || y < 0 || z < 0 || x >= d.nx || y >= d.ny || z >= d.nz) return 0u;
  const long long p = ((long long)z * d.ny + y) * d.nx + x;
  if (lab) {
    const uint8_t l = __ldg(lab + p);
    return l == kFluid ? 1u : (l == kAir ? 0x10000u : 0u);
  }
  const ushort2 c = counts[p];
  return (uint32_t)c.x | ((uint32_t)c.y << 16);
}

// Rank of row w's first mixed cell within the plane's block.
__device__ __forceinline__ uint32_t row_base(const PlaneDesc &d, int w) {
  return (d.rowbase[w >> 2] >> (8 * (w & 3))) & 0xFFu;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Wait for an mbarrier phase with the thread suspended in hardware (up to
// 100 us per try) instead of spinning; gives up after limit_ns of wall time.
__device__ __forceinline__ bool mbar_sleep_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
  constexpr uint32_t kHintNs = 100000u;
  uint32_t ok;
  uint64_t t0 = 0;
  for (int it = 0;; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kHintNs)
        : "memory");
    if (ok) return true;
    if (it == 0) t0 = globaltimer();
    else if (globaltimer() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// 3-D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
// 4-D tiled TMA load (the fourth coordinate picks a vector of a ring).
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int x, int y, int z, int w,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
      : "memory");
}
// Bulk (untiled) copy global -> shared; both addresses and the size multiples of 16 bytes.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

}  // namespace

// ---------------------------------------------------------------------------
// Setup 1: classification.  One CTA (the 32 x 8 tile) per unit of planes.
// A cell's window is pure when its 27 cells are all pure solid, all pure
// fluid or all pure air (solid outside the grid): with one class bit per cell
// (1 pure solid, 2 pure fluid, 4 pure air, 8 anything else) that is a window
// OR of 1, 2 or 4.  The OR is separable: along x by lane shuffles (the two
// halo columns loaded by the edge lanes), along y through shared memory, along
// z by keeping the last two planes' 3x3 ORs in registers, so each cell's class
// is loaded about 1.3 times instead of 27 times.  Ten warps, one per row
// y0-1 .. y0+8 (the two halo rows included, so that every warp loads one row
// per plane), and each thread's loads for the next plane are issued before
// the current plane's barrier.
// ---------------------------------------------------------------------------
// The class bit of a cell, and bit 4 set if it holds fluid (level 1: its
// label; coarser levels: a non-zero fluid count).
__device__ __forceinline__ uint32_t class_bit(const uint8_t *lab, const ushort2 *counts, const Dims &d, int x, int y,
                                              int z, uint32_t kF, uint32_t kA) {
  if ((unsigned)x >= (unsigned)d.nx || (unsigned)y >= (unsigned)d.ny || (unsigned)z >= (unsigned)d.nz) return 1u;
  const uint32_t p = ((uint32_t)z * (uint32_t)d.ny + (uint32_t)y) * (uint32_t)d.nx + (uint32_t)x;  // n < 2^31
  if (lab) {
    const uint8_t l = __ldg(lab + p);
    return l == kFluid ? 2u | 16u : (l == kAir ? 4u : 1u);  // level 1: every cell is pure
  }
  const ushort2 c = counts[p];
  const uint32_t k = (uint32_t)c.x | ((uint32_t)c.y << 16);
  const uint32_t b = k == 0u ? 1u : (k == kF ? 2u : (k == kA ? 4u : 8u));
  return b | (c.x > 0 ? 16u : 0u);
}

constexpr int CLW = TY + 2;    // classification warps: rows y0-1 .. y0+8
constexpr int CLT = CLW * 32;  // classification threads

__global__ void __launch_bounds__(CLT) k_classify(const uint8_t *__restrict__ lab, const ushort2 *__restrict__ counts,
                                                  Dims d, uint32_t full, int zcc, PlaneDesc *__restrict__ desc,
                                                  unsigned *__restrict__ totals, uint8_t *__restrict__ skip,
                                                  uint16_t *__restrict__ mcount) {
  __shared__ uint32_t sd[ZCG][DWORDS];
  __shared__ uint8_t rows[2][CLW][TX];  // x-ORed class bits of rows y0-1 .. y0+8 of one plane, two buffers
  __shared__ uint32_t sbase;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ntx = (d.nx + TX - 1) / TX, nty = (d.ny + TY - 1) / TY, nch = (d.nz + zcc - 1) / zcc;
  const int ntiles = ntx * nty;
  const long long units = (long long)ntiles * nch;
  const uint32_t kF = full, kA = full << 16;
  const bool interior = warp >= 1 && warp <= TY;  // rows y0 .. y0+7: the tile's cells
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    const int t = (int)(u % ntiles), c = (int)(u / ntiles);
    const int x0 = (t % ntx) * TX, y0 = (t / ntx) * TY;
    const int x = x0 + lane, y = y0 + warp - 1;  // this warp's row
    const int zs = c * zcc, nzu = min(zcc, d.nz - zs);
    const bool inside = interior && x < d.nx && y < d.ny;
    // the raw bits of this thread's column and (lanes 0 and 31) of its halo column in plane z
    auto load_row = [&](int z, uint32_t &b, uint32_t &e) {
      b = class_bit(lab, counts, d, x, y, z, kF, kA);
      e = 1u;
      if (lane == 0) e = class_bit(lab, counts, d, x - 1, y, z, kF, kA);
      else if (lane == 31) e = class_bit(lab, counts, d, x + 1, y, z, kF, kA);
    };
    uint32_t bn, en;
    load_row(zs - 1, bn, en);
    uint32_t pm = 0u, p0 = 0u, own = 0u;  // 3x3 ORs of planes z-2, z-1; class bits of this cell in plane z-1
    for (int st = 0; st < nzu + 2; ++st) {  // plane zs - 1 + st
      const uint32_t b = bn, e = en;
      if (st + 1 < nzu + 2) load_row(zs + st, bn, en);  // the next plane, in flight across the barrier
      uint32_t left = __shfl_up_sync(0xffffffffu, b, 1), right = __shfl_down_sync(0xffffffffu, b, 1);
      if (lane == 0) left = e;
      if (lane == 31) right = e;
      const int buf = st & 1;
      rows[buf][warp][lane] = (uint8_t)((b | left | right) & 15u);
      __syncthreads();
      if (interior) {
        const uint32_t pp = (uint32_t)(rows[buf][warp - 1][lane] | rows[buf][warp][lane] | rows[buf][warp + 1][lane]);
        if (st >= 2) {
          const int j = st - 2;  // plane zs + j: window OR over planes zs+j-1 .. zs+j+1
          const uint32_t wor = pm | p0 | pp;
          const bool pure = wor == 1u || wor == 2u || wor == 4u;
          const bool mixed = inside && !pure, fl = inside && wor == 2u, ai = inside && wor == 4u;
          const bool self = inside && (own & 16u) != 0u;  // the cell holds fluid
          const uint32_t bm = __ballot_sync(0xffffffffu, mixed), bf = __ballot_sync(0xffffffffu, fl);
          const uint32_t ba = __ballot_sync(0xffffffffu, ai), bs = __ballot_sync(0xffffffffu, self);
          if (lane == 0) {
            const int w = warp - 1;
            sd[j][4 * w] = bm;
            sd[j][4 * w + 1] = bf;
            sd[j][4 * w + 2] = ba;
            sd[j][4 * w + 3] = bs;
          }
        }
        pm = p0;
        p0 = pp;
      }
      own = b;
    }
    __syncthreads();
    // per plane (one thread each): mixed count, block size, row ranks, patch classes
    for (int j = threadIdx.x; j < nzu; j += CLT) {
      uint32_t m = 0, rb[2] = {0u, 0u};
      for (int w = 0; w < TY; ++w) {
        rb[w >> 2] |= m << (8 * (w & 3));
        m += __popc(sd[j][4 * w]);
      }
      uint32_t pc = 0u;
      for (int q = 0; q < TX / PW; ++q) {
        const uint32_t pmk = ((1u << PW) - 1u) << (PW * q);
        bool allf = true, alla = true, alls = true;
        for (int w = 0; w < TY; ++w) {
          const uint32_t mx = sd[j][4 * w] & pmk, f = sd[j][4 * w + 1] & pmk, a = sd[j][4 * w + 2] & pmk;
          allf &= f == pmk;
          alla &= a == pmk;
          alls &= (mx | f | a) == 0u;
        }
        pc |= (allf ? 1u : alla ? 2u : alls ? 0u : 3u) << (2 * q);
      }
      sd[j][4 * TY + 1] = m;
      sd[j][4 * TY + 2] = (m + 3u) & ~3u;
      sd[j][4 * TY + 3] = pc;
      if (skip) {  // bit 0: every window pure solid or pure air (a zero level-1 CConv1 output); bit 1: no fluid cell
        uint32_t anyf = 0u;
        for (int w = 0; w < TY; ++w) anyf |= sd[j][4 * w + 3];
        skip[(size_t)t * d.nz + zs + j] = (uint8_t)(((pc & 0x55u) == 0u ? 1u : 0u) | (anyf == 0u ? 2u : 0u));
      }
      if (mcount) mcount[(size_t)t * d.nz + zs + j] = (uint16_t)m;  // mixed cells of the (tile, plane)
      sd[j][4 * TY + 4] = rb[0];
      sd[j][4 * TY + 5] = rb[1];
      sd[j][4 * TY + 6] = 0u;
      sd[j][4 * TY + 7] = 0u;
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // block offsets within the unit, then one atomic for the unit
      uint32_t tot = 0, cnt = 0;
      for (int j = 0; j < nzu; ++j) {
        sd[j][4 * TY] = tot;
        tot += sd[j][4 * TY + 2];
        cnt += sd[j][4 * TY + 1];
      }
      sbase = tot ? atomicAdd(&totals[0], tot) : 0u;
      if (cnt) atomicAdd(&totals[1], cnt);
    }
    __syncthreads();
    uint32_t *dst = (uint32_t *)(desc + (size_t)t * d.nz + zs);
    for (int i = threadIdx.x; i < nzu * DWORDS; i += CLT) {
      uint32_t v = sd[i / DWORDS][i % DWORDS];
      if (i % DWORDS == 4 * TY) v += sbase;
      dst[i] = v;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Setup 2: kernels of the mixed cells, for nblk CConv blocks of one level
// (CConv1 and CConv2 share the classification).
// ---------------------------------------------------------------------------
template <bool BF16>
__global__ void __launch_bounds__(NT) k_generate(const uint8_t *__restrict__ lab, const ushort2 *__restrict__ counts,
                                                 Dims d, const CConvW *__restrict__ w, int nblk,
                                                 const PlaneDesc *__restrict__ desc, uint32_t *__restrict__ cache0,
                                                 uint32_t *__restrict__ cache1) {
  constexpr int KW = BF16 ? 14 : 27;
  __shared__ CConvW sw[2];
  __shared__ PlaneDesc sd[ZCG];
  {
    const float *src = (const float *)w;
    float *dstw = (float *)sw;
    for (int i = threadIdx.x; i < nblk * (int)(sizeof(CConvW) / 4); i += NT) dstw[i] = src[i];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ntx = (d.nx + TX - 1) / TX, nty = (d.ny + TY - 1) / TY;
  const int ntiles = ntx * nty;
  // one work item per (tile, plane): the coarse levels that run here are small
  const long long items = (long long)ntiles * d.nz;
  for (long long u = blockIdx.x; u < items; u += gridDim.x) {
    const int t = (int)(u % ntiles), zs = (int)(u / ntiles), nzu = 1;
    const int x = (t % ntx) * TX + lane, y = (t / ntx) * TY + warp;
    __syncthreads();  // previous item done with sd (and the weights are in place)
    {
      const uint32_t *src = (const uint32_t *)(desc + (size_t)t * d.nz + zs);
      uint32_t *dsd = (uint32_t *)sd;
      for (int i = threadIdx.x; i < nzu * DWORDS; i += NT) dsd[i] = src[i];
    }
    __syncthreads();
    for (int j = 0; j < nzu; ++j) {
      const PlaneDesc &pd = sd[j];
      const uint32_t mw = pd.row[warp].x;
      if (!((mw >> lane) & 1u)) continue;
      const uint32_t rank = __popc(mw & lanemask_lt()) + row_base(pd, warp);
      const int z = zs + j;
      float nf[27], na[27];
#pragma unroll
      for (int l = 0; l < 27; ++l) {
        const uint32_t k = image_key(lab, counts, d, x + l % 3 - 1, y + (l / 3) % 3 - 1, z + l / 9 - 1);
        nf[l] = (float)(k & 0xFFFFu);
        na[l] = (float)(k >> 16);
      }
      const size_t base = (size_t)pd.off * KW + rank;
      const uint32_t cp = pd.cpad;
      for (int b = 0; b < nblk; ++b) {
        const CConvW &cw = sw[b];
        uint32_t *cache = b == 0 ? cache0 : cache1;
        if (BF16) {
#pragma unroll 1
          for (int jj = 0; jj < 14; ++jj) {
            const int a0 = 2 * jj, a1 = 2 * jj + 1;
            float k0 = cw.bp[a0];
#pragma unroll
            for (int l = 0; l < 27; ++l) k0 = fmaf(cw.wf[a0][l], nf[l], fmaf(cw.wa[a0][l], na[l], k0));
            float k1 = 0.f;
            if (a1 < 27) {
              k1 = cw.bp[a1];
#pragma unroll
              for (int l = 0; l < 27; ++l) k1 = fmaf(cw.wf[a1][l], nf[l], fmaf(cw.wa[a1][l], na[l], k1));
            }
            cache[base + (size_t)jj * cp] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(k0)) |
                                            ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(k1)) << 16);
          }
        } else {
#pragma unroll 1
          for (int a = 0; a < 27; ++a) {
            float k0 = cw.bp[a];
#pragma unroll
            for (int l = 0; l < 27; ++l) k0 = fmaf(cw.wf[a][l], nf[l], fmaf(cw.wa[a][l], na[l], k0));
            cache[base + (size_t)a * cp] = __float_as_uint(k0);
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Setup 2 on the tensor cores (levels whose image counts are exact in BF16):
// the kernels of the mixed cells of a unit, 128 cells per tcgen05 MMA
//   D[128 cells x 32 taps] = F[128 x 64 features] . W^T[64 x 32]  (FP32 in TMEM),
// the feature rows F = (fluid counts of the 27 window cells, air counts, 1)
// written into TMEM by the threads, W (folded CConv weights and bias, K-major
// in shared memory, NSPLIT BF16 terms: 1 in the BF16 form, 3 in the FP32
// form) from the host.  Thread i owns TMEM lane i and mixed cell i of the
// chunk; it reads its 32 results back and writes them tap-major into the
// plane's block, rounded to BF16 in the BF16 form.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t image_code_bf16(const uint8_t *lab, const ushort2 *counts, const Dims &d, int x,
                                                    int y, int z) {
  if ((unsigned)x >= (unsigned)d.nx || (unsigned)y >= (unsigned)d.ny || (unsigned)z >= (unsigned)d.nz) return 0u;
  const uint32_t p = ((uint32_t)z * (uint32_t)d.ny + (uint32_t)y) * (uint32_t)d.nx + (uint32_t)x;  // n < 2^31
  if (lab) {
    const uint8_t l = __ldg(lab + p);
    return l == kFluid ? 0x00003F80u : (l == kAir ? 0x3F800000u : 0u);
  }
  const ushort2 c = counts[p];
  return umma::bf16_bits_small(c.x) | (umma::bf16_bits_small(c.y) << 16);
}

constexpr int kGenTmemCols = 64;  // A: columns [0, 32), D: [32, 64)
constexpr int GT = 128;           // threads of the tensor-core generator: one per TMEM lane / MMA row
constexpr int kWinRow = TX + 2, kWinPlane = (TY + 2) * kWinRow;  // the label window of a unit (level 1)
constexpr int kWinBytes = ((ZCG + 2) * kWinPlane + 15) & ~15;
// dynamic shared memory of the generator: W splits of both blocks, the unit's
// plane descriptors, its cache-entry map and (level 1) label window, + alignment slack
constexpr int gen_smem_bytes(int nsplit, bool window) {
  return 2 * nsplit * umma::kBBytes + ZCG * (int)sizeof(PlaneDesc) + ZCG * NT * 2 + (window ? kWinBytes : 0) + 1024;
}

template <int NSPLIT, bool BF16>
__global__ void __launch_bounds__(GT) k_generate_tc(const uint8_t *__restrict__ lab, const ushort2 *__restrict__ counts,
                                                    Dims d, const uint8_t *__restrict__ w0,
                                                    const uint8_t *__restrict__ w1, int nblk,
                                                    const PlaneDesc *__restrict__ desc, uint32_t *__restrict__ cache0,
                                                    uint32_t *__restrict__ cache1, int zcc, int *err) {
  using namespace umma;
  constexpr int KW = BF16 ? 14 : 27;
  extern __shared__ uint8_t gen_raw[];
  uint8_t *gsm = (uint8_t *)(((uintptr_t)gen_raw + 1023) & ~(uintptr_t)1023);
  uint8_t(*sW)[NSPLIT * kBBytes] = reinterpret_cast<uint8_t(*)[NSPLIT * kBBytes]>(gsm);
  PlaneDesc *sd = (PlaneDesc *)(gsm + 2 * NSPLIT * kBBytes);
  uint16_t *cell_of = (uint16_t *)(sd + ZCG);  // unit-local cache entry -> plane << 8 | cell (0xFFFF: padding)
  uint8_t *win = (uint8_t *)(cell_of + ZCG * NT);  // level 1: labels of planes zs-1 .., rows y0-1 .., x0-1 ..
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  {
    const uint4 *src0 = (const uint4 *)w0;
    const uint4 *src1 = (const uint4 *)w1;
    uint4 *dst0 = (uint4 *)sW[0];
    uint4 *dst1 = (uint4 *)sW[1];
    for (int i = tid; i < NSPLIT * kBBytes / 16; i += GT) {
      dst0[i] = src0[i];
      if (nblk > 1) dst1[i] = src1[i];
    }
  }
  if (warp == 0) {
    tmem_alloc(&s_tmem, kGenTmemCols);
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
  uint32_t phase = 0u;
  bool aborted = false;
  const int ntx = (d.nx + TX - 1) / TX, nty = (d.ny + TY - 1) / TY, nch = (d.nz + zcc - 1) / zcc;
  const int ntiles = ntx * nty;
  const long long units = (long long)ntiles * nch;
  for (long long u = blockIdx.x; u < units && !aborted; u += gridDim.x) {
    const int t = (int)(u % ntiles), c = (int)(u / ntiles);
    const int x0 = (t % ntx) * TX, y0 = (t / ntx) * TY;
    const int zs = c * zcc, nzu = min(zcc, d.nz - zs);
    {
      const uint32_t *src = (const uint32_t *)(desc + (size_t)t * d.nz + zs);
      uint32_t *dsd = (uint32_t *)sd;
      for (int i = tid; i < nzu * DWORDS; i += GT) dsd[i] = src[i];
    }
    __syncthreads();
    const uint32_t base = sd[0].off;
    const int total = (int)(sd[nzu - 1].off + sd[nzu - 1].cpad - base);  // entries of the unit, padding included
    if (total > 0) {
      if (lab) {
        // the unit's label window (solid outside the grid): a warp takes rows warp, warp + 4, ...; lane c loads
        // column c and lanes 0, 1 also columns 32, 33; eight rows' loads are in flight before their stores
        constexpr int kNW = GT / 32, kBatch = 8;
        const int nrows = (nzu + 2) * (TY + 2);
        for (int r0 = warp; r0 < nrows; r0 += kBatch * kNW) {
          uint32_t v0[kBatch], v1[kBatch];
#pragma unroll
          for (int k = 0; k < kBatch; ++k) {
            const int rr = r0 + k * kNW;
            v0[k] = v1[k] = (uint32_t)kSolid;
            const int gz = zs - 1 + rr / (TY + 2), gy = y0 - 1 + rr % (TY + 2);
            if (rr < nrows && gz >= 0 && gz < d.nz && gy >= 0 && gy < d.ny) {
              const long long rb = ((long long)gz * d.ny + gy) * d.nx;
              const int gx = x0 - 1 + lane, gx2 = x0 + 31 + lane;
              if (gx >= 0 && gx < d.nx) v0[k] = __ldg(lab + rb + gx);
              if (lane < 2 && gx2 < d.nx) v1[k] = __ldg(lab + rb + gx2);
            }
          }
#pragma unroll
          for (int k = 0; k < kBatch; ++k) {
            const int rr = r0 + k * kNW;
            if (rr < nrows) {
              win[rr * kWinRow + lane] = (uint8_t)v0[k];
              if (lane < 2) win[rr * kWinRow + 32 + lane] = (uint8_t)v1[k];
            }
          }
        }
      }
      for (int i = tid; i < total; i += GT) cell_of[i] = 0xFFFFu;
      __syncthreads();
      for (int j = 0; j < nzu; ++j) {
        for (int cc = tid; cc < NT; cc += GT) {  // cell cc = row * 32 + x of the tile
          const int row = cc >> 5, xb = cc & 31;
          const uint32_t m = sd[j].row[row].x;
          if ((m >> xb) & 1u) {
            const uint32_t rank = __popc(m & ((1u << xb) - 1u)) + row_base(sd[j], row);
            cell_of[sd[j].off - base + rank] = (uint16_t)((j << 8) | cc);
          }
        }
      }
      __syncthreads();
      for (int c0 = 0; c0 < total && !aborted; c0 += GT) {
        const int li = c0 + tid;
        const uint32_t e = li < total ? cell_of[li] : 0xFFFFu;
        const bool valid = e != 0xFFFFu;
        uint32_t fw[32];
        int j = 0;
        if (valid) {
          j = (int)(e >> 8);
          const int cell = (int)(e & 255u);
          const int x = x0 + (cell & 31), y = y0 + (cell >> 5), z = zs + j;
          uint32_t wc[27];
          if (lab) {
            const uint8_t *w0p = win + (j + 1) * kWinPlane + ((cell >> 5) + 1) * kWinRow + (cell & 31) + 1;
#pragma unroll
            for (int l = 0; l < 27; ++l) {
              const uint8_t lb = w0p[(l / 9 - 1) * kWinPlane + ((l / 3) % 3 - 1) * kWinRow + (l % 3 - 1)];
              wc[l] = lb == kFluid ? 0x00003F80u : (lb == kAir ? 0x3F800000u : 0u);
            }
          } else {
#pragma unroll
            for (int l = 0; l < 27; ++l)
              wc[l] = image_code_bf16(lab, counts, d, x + l % 3 - 1, y + (l / 3) % 3 - 1, z + l / 9 - 1);
          }
          build_feature_words(wc, fw);
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) fw[q] = 0u;
        }
        tmem_st32(tmem + lane_off, fw);
        tmem_wait_st();
        for (int b = 0; b < nblk; ++b) {
          fence_before_sync();
          __syncthreads();
          if (tid == 0) {
            fence_after_sync();
#pragma unroll
            for (int sp = 0; sp < NSPLIT; ++sp)
#pragma unroll
              for (int kk = 0; kk < kK / 16; ++kk) {
                const uint64_t bd = smem_desc_kmajor(smem_u32(sW[b] + sp * kBBytes + kk * 2 * kLBO), kLBO, kSBO);
                mma_bf16_ts(tmem + 32, tmem + kk * 8, bd, idesc, (sp | kk) != 0);
              }
            umma_commit(&mbar);
          }
          const bool ok = mbar_wait_bounded(&mbar, phase, umma::kWaitNs);
          phase ^= 1u;
          if (__syncthreads_or(!ok)) {
            aborted = true;
            break;
          }
          fence_after_sync();
          uint32_t kr[32];
          tmem_ld32(tmem + 32 + lane_off, kr);
          tmem_wait_ld();
          if (valid) {
            const PlaneDesc &pd = sd[j];
            const uint32_t rank = (uint32_t)li - (pd.off - base);
            uint32_t *dst = (b == 0 ? cache0 : cache1) + (size_t)pd.off * KW + rank;
            if (BF16) {
#pragma unroll
              for (int jj = 0; jj < 14; ++jj) {
                const float k0 = __uint_as_float(kr[2 * jj]);
                const float k1 = 2 * jj + 1 < 27 ? __uint_as_float(kr[2 * jj + 1]) : 0.f;
                dst[(size_t)jj * pd.cpad] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(k0)) |
                                            ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(k1)) << 16);
              }
            } else {
#pragma unroll
              for (int a = 0; a < 27; ++a) dst[(size_t)a * pd.cpad] = kr[a];
            }
          }
        }
        fence_before_sync();
        __syncthreads();  // the next chunk overwrites A and D
      }
    }
    __syncthreads();  // sd and cell_of are reloaded for the next unit
  }
  if (aborted) {
    if (tid == 0 && err) atomicExch(err, 1);
    (void)mbar_wait_bounded(&mbar, phase, umma::kWaitNs);  // an MMA batch possibly still in flight
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kGenTmemCols);
}

// ---------------------------------------------------------------------------
// Per iteration: the streamed z-marching CConv.
// ---------------------------------------------------------------------------
// The constant kernel of one pure class laid out for packed FP32 FMAs
// (fma.rn.f32x2: two independent, correctly rounded FP32 FMAs).  A thread
// holds a window column of 4 rows x 3 columns per plane as six register
// pairs c(0,1) .. c(10,11) (row-major) and computes the cell of row y (window
// rows 0..2, tap j of a plane is c_j) and of row y+1 (rows 1..3, tap j is
// c_{j+3}).  Per plane dz: the upper cell pairs taps (0,1) (2,3) (4,5) (6,7)
// with c(0,1) .. c(6,7) and takes tap 8 alone; the lower cell pairs taps
// (1,2) (3,4) (5,6) (7,8) with c(4,5) .. c(10,11) and takes tap 0 alone.
struct PairKernel {
  float2 up[3][4];  // per plane: (k0,k1) (k2,k3) (k4,k5) (k6,k7)
  float2 lo[3][4];  // per plane: (k1,k2) (k3,k4) (k5,k6) (k7,k8)
  float up8[3], lo0[3];
};

struct StreamParams {
  CUtensorMap tv;   // input vector of the level: box 44 x 10 x 2 (FP32)
  CUtensorMap tx1;  // x1 of the level (combination only): box 36 x 8 x 2
  Dims dm;
  int ntx, ntiles, zc, units;
  const int *ulist;     // optional: the units to process (indices c * ntiles + t), `units` of them
  const PlaneDesc *desc;
  const uint8_t *cache;
  const float *vscale;  // optional scale of the output (the input normalisation)
  float *out;
  float *pooled;        // optional 2x2x2 mean of the output
  const double *c12;    // non-null: out = c1 x1 + c2 CConv(v)
  const SolveState *st;
  int *err;
  int mode;             // which outputs are computed (STREAM_MODE_*)
  int method;           // fused CConv2: the solver's method (kMethod*), fixed for a solve
  // fused level-1 combination: z = mask_fluid(c1 x1 + c2 CConv2) and the dots z . q_i
  CUtensorMap tq;       // q ring: dims (nx, ny, nz, ring), box 36 x 8 x 2 x 1
  double *part;         // partial dots, one row per CTA
  unsigned *ticket;     // last-CTA-done counter
  SolveState *stw;      // the solve state (orthogonalisation coefficients are written)
  // level-1 CConv1 that first forms r_{k+1} = r_k - alpha q_{k+1} (Alg. 1's
  // recurrence) while a step is pending: r_k in buffer k mod 2
  // (one pair of maps serves both fusions, which never share a launch:)
  //   residual update: aux[0] the second residual buffer, as tv; aux[1] the q
  //                    ring, dims (nx, ny, nz, ring), box 44 x 10 x 2 x 1;
  //   fused CConv2 of PCG / FPCG: the residual buffers (r_k in aux[k & 1]),
  //                    one-slot 4-D maps with tq's 36 x 8 x 2 x 1 box.
  CUtensorMap aux[2];
  float *rb[2];         // the residual buffers (r_{k+1} is written to rb[(k + 1) & 1])
  double *upart;        // ||r_{k+1}||^2 partials, one per CTA
  unsigned *uticket;
  double *hist;
  PairKernel kp[3];              // kernels of the pure-solid, pure-fluid, pure-air windows, paired
  uint32_t ktab[3][27];          // the same as stored in the class tables (BF16 pairs or FP32 words)
};

struct Unit {
  int t, x0, y0, zs, nzu;
};

__device__ __forceinline__ Unit unit_at(const StreamParams &P, int i) {
  const int u = P.ulist ? __ldg(P.ulist + i) : i;
  Unit U;
  U.t = u % P.ntiles;
  const int c = u / P.ntiles;
  U.x0 = (U.t % P.ntx) * TX;
  U.y0 = (U.t / P.ntx) * TY;
  U.zs = c * P.zc;
  U.nzu = min(P.zc, P.dm.nz - U.zs);
  return U;
}

// A thread's window column of one plane: rows y-1 .. y+2 x columns x-1 .. x+1
// (row-major, 12 values) in six register pairs, so that rows 0..2 are the 3x3
// window of cell y and rows 1..3 that of cell y+1.
struct Col {
  float2 v[6];
  __device__ __forceinline__ float at(int i) const { return (i & 1) ? v[i >> 1].y : v[i >> 1].x; }
  __device__ __forceinline__ void set(int i, float f) {
    if (i & 1) v[i >> 1].y = f;
    else v[i >> 1].x = f;
  }
};

// sum_a k[a] v[a] of the two cells of a thread's column pair (rows y, y+1) of
// one pure class, over the planes p0, p1, p2 (Alg. 2's CConv with a constant
// kernel): 24 packed FMAs and 6 scalar ones for the two cells.
__device__ __forceinline__ void dot27_pair(const PairKernel &K, const Col &p0, const Col &p1, const Col &p2,
                                           float &oa, float &ob) {
  float2 a02 = make_float2(0.f, 0.f), a1 = a02, b02 = a02, b1 = a02;
  float sa = 0.f, sb = 0.f;
#pragma unroll
  for (int dz = 0; dz < 3; ++dz) {
    const Col &c = dz == 0 ? p0 : (dz == 1 ? p1 : p2);
    float2 &A = dz == 1 ? a1 : a02;
    float2 &B = dz == 1 ? b1 : b02;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      A = __ffma2_rn(c.v[i], K.up[dz][i], A);
      B = __ffma2_rn(c.v[i + 2], K.lo[dz][i], B);
    }
    sa = fmaf(c.v[4].x, K.up8[dz], sa);
    sb = fmaf(c.v[1].y, K.lo0[dz], sb);
  }
  oa = ((a02.x + a02.y) + (a1.x + a1.y)) + sa;
  ob = ((b02.x + b02.y) + (b1.x + b1.y)) + sb;
}

// A cell of a patch that is not all one pure class: its kernel is read from
// shared memory, the class table of its pure class (stride 1) or the cell's
// mixed block (stride cpad), one code path for all lanes.  Cells whose output
// is not needed get 0: with a zero input off fluid (level-1 CConv1) a
// pure-air or pure-solid window sums to exactly 0, and the level-1 CConv2
// output is used on fluid cells only.
template <bool BF16C, int MODE, int R>
__device__ __forceinline__ float cconv_generic(uint4 rw, uint32_t rank, uint32_t cp, const uint32_t *kblk,
                                               const uint32_t *ktab, uint32_t bit, const Col &pA, const Col &pB,
                                               const Col &pC) {
  const bool mixed = (rw.x & bit) != 0u, fl = (rw.y & bit) != 0u, ai = (rw.z & bit) != 0u;
  bool need = true;
  if (MODE == STREAM_MODE_ZERO_PURE) need = mixed || fl;
  else if (MODE == STREAM_MODE_FLUID_ONLY) need = (rw.w & bit) != 0u;
  const uint32_t *src = ktab + (fl ? 27 : (ai ? 54 : 0));
  uint32_t stride = 1;
  if (mixed) {
    src = kblk + rank;
    stride = cp;
  }
  float K[28];
  if (BF16C) {
#pragma unroll
    for (int q = 0; q < 14; ++q) {
      const uint32_t wv = src[q * stride];
      K[2 * q] = __uint_as_float(wv << 16);
      K[2 * q + 1] = __uint_as_float(wv & 0xFFFF0000u);
    }
  } else {
#pragma unroll
    for (int a = 0; a < 27; ++a) K[a] = __uint_as_float(src[a * stride]);
  }
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    s0 = fmaf(K[q], pA.at(3 * R + q), s0);
    s1 = fmaf(K[9 + q], pB.at(3 * R + q), s1);
    s2 = fmaf(K[18 + q], pC.at(3 * R + q), s2);
  }
  const float acc = (s0 + s1) + s2;
  return need ? acc : 0.f;
}

// The two cells (rows y, y+1) of one plane for a patch of one pure class cls
// (0 solid, 1 fluid, 2 air): the class's constant kernel from the kernel
// parameters, or 0 where the mode says the output is exactly 0 or unused.
template <int MODE>
__device__ __forceinline__ void cconv_pure_pair(const StreamParams &P, int cls, const Col &p0, const Col &p1,
                                                const Col &p2, float &oa, float &ob) {
  if (MODE != STREAM_MODE_ALL && cls != 1) {
    oa = 0.f;
    ob = 0.f;
  } else if (cls == 1) {
    dot27_pair(P.kp[1], p0, p1, p2, oa, ob);
  } else if (cls == 2) {
    dot27_pair(P.kp[2], p0, p1, p2, oa, ob);
  } else {
    dot27_pair(P.kp[0], p0, p1, p2, oa, ob);
  }
}

// The two cells of one plane (rows ra, ra+1, bit b of the row masks) of a
// patch that is not all one pure class.
template <bool BF16C, int MODE>
__device__ __forceinline__ void cconv_generic_pair(const PlaneDesc &d, int ra, int b,
                                                   const uint32_t *kblk, const uint32_t *ktab, const Col &p0,
                                                   const Col &p1, const Col &p2, float &oa, float &ob) {
  const uint4 wa = d.row[ra], wb = d.row[ra + 1];
  const uint32_t rb = d.rowbase[ra >> 2] >> (8 * (ra & 3));
  const uint32_t cp = min(d.cpad, (uint32_t)NT);
  const uint32_t bit = 1u << b, below = bit - 1u;
  oa = cconv_generic<BF16C, MODE, 0>(wa, __popc(wa.x & below) + (rb & 0xFFu), cp, kblk, ktab, bit, p0, p1, p2);
  ob = cconv_generic<BF16C, MODE, 1>(wb, __popc(wb.x & below) + ((rb >> 8) & 0xFFu), cp, kblk, ktab, bit, p0, p1,
                                     p2);
}

// Shared memory after the slots, descriptor buffers and the kernel-block
// buffer (16-byte aligned): mbarriers, block positions, class tables.
struct StreamMeta {
  uint64_t full[RV], empty[RV], dfull[ND], dempty[ND];
  double fsum[4][kMaxFusedOrtho];  // fused dots: per consumer warp (final reduction)
  int unit[ND];                       // the unit of each descriptor buffer (-1: no more units)
  uint32_t kstart[RV], kend[RV];
  uint32_t ktab[3 * 27];
  int abort_;
  int last_;
};
static_assert(sizeof(StreamMeta) <= kMetaBytes, "stream metadata fits");

namespace {

// Double-float accumulator (error-free TwoSum into a (hi, lo) FP32 pair).
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

// Consumer-only barrier (named barrier 1): the producer warp has left.
__device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// End of the fused level-1 CConv2: each consumer warp's dots z . q_i (its
// patch in all of the CTA's units; the units of a CTA are fixed by the grid,
// blockIdx.x + m gridDim.x) go to the CTA's row of partials in a fixed order;
// the last CTA to arrive reduces the rows in a fixed order and sets the
// orthogonalisation coefficients c_i = z^T A d_i / d_i^T A d_i (Alg. 1; for
// PCG / FPCG the conjugation coefficient from r_k . z and q_k . z), then
// re-arms the counter.  Deterministic for a given grid.
__device__ __noinline__ void fused_finish(const StreamParams &P, StreamMeta &M, DF (&fdot)[kMaxFusedOrtho], int cnt) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int j = 0; j < kMaxFusedOrtho; ++j) {
    double v = (double)fdot[j].hi + (double)fdot[j].lo;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) M.fsum[warp][j] = v;
  }
  consumers_sync();
  if (tid == 0) {
    for (int j = 0; j < kMaxFusedOrtho; ++j)
      P.part[(size_t)blockIdx.x * kMaxFusedOrtho + j] = ((M.fsum[0][j] + M.fsum[1][j]) + M.fsum[2][j]) + M.fsum[3][j];
    __threadfence();
    const unsigned t = atomicAdd(P.ticket, 1u);
    M.last_ = t == gridDim.x - 1 ? 1 : 0;
  }
  consumers_sync();
  if (!M.last_) return;
  __threadfence();
#pragma unroll
  for (int j = 0; j < kMaxFusedOrtho; ++j) {
    double a = 0.0;
    for (int i = tid; i < (int)gridDim.x; i += 128) a += __ldcg(P.part + (size_t)i * kMaxFusedOrtho + j);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) M.fsum[warp][j] = a;
  }
  consumers_sync();
  if (tid == 0) {
    double t[kMaxFusedOrtho];
    for (int j = 0; j < kMaxFusedOrtho; ++j) t[j] = ((M.fsum[0][j] + M.fsum[1][j]) + M.fsum[2][j]) + M.fsum[3][j];
    set_direction_coefs(P.stw, t, cnt);
    *P.ticket = 0u;
  }
}

// End of the residual update fused into the level-1 CConv1: the CTA's
// ||r_{k+1}||^2 partial (consumer warps in a fixed order) goes to its slot;
// the last CTA sums the slots in a fixed order and, as k_update4's last
// block does, advances the iteration, records ||r_{k+1}||, applies the stop
// test ||r_{k+1}|| < tol ||b|| and the next input normalisation, then
// re-arms the counter.
__device__ __noinline__ void update_finish(const StreamParams &P, StreamMeta &M, DF unorm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double v = (double)unorm.hi + (double)unorm.lo;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) M.fsum[warp][0] = v;
  consumers_sync();
  if (tid == 0) {
    P.upart[blockIdx.x] = ((M.fsum[0][0] + M.fsum[1][0]) + M.fsum[2][0]) + M.fsum[3][0];
    __threadfence();
    const unsigned t = atomicAdd(P.uticket, 1u);
    M.last_ = t == gridDim.x - 1 ? 1 : 0;
  }
  consumers_sync();
  if (!M.last_) return;
  __threadfence();
  double a = 0.0;
  for (int i = tid; i < (int)gridDim.x; i += 128) a += __ldcg(P.upart + i);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  if (lane == 0) M.fsum[warp][0] = a;
  consumers_sync();
  if (tid == 0) {
    SolveState *st = P.stw;
    const double rr = ((M.fsum[0][0] + M.fsum[1][0]) + M.fsum[2][0]) + M.fsum[3][0];
    st->k += 1;
    st->upd_pending = 0;
    st->rnorm2 = rr;
    P.hist[st->k] = sqrt(rr);
    if (!isfinite(rr)) st->done = kDoneBreakdown;
    else if (rr < st->eps2 || rr == 0.0) st->done = kDoneConverged;
    else st->rscale = (float)(1.0 / sqrt(rr));
    *P.uticket = 0u;
  }
}

}  // namespace

constexpr int NCW = 4;                    // consumer warps: two tile rows each
constexpr int NTHREADS = NCW * 32 + 32;   // and one producer warp

template <bool BF16C, bool FUSE, int MODE, bool UPD = false>
__global__ void __launch_bounds__(NTHREADS, 3) k_cconv_stream(const __grid_constant__ StreamParams P) {
  static_assert(!FUSE || MODE == STREAM_MODE_FLUID_ONLY, "the fused CConv2 computes fluid outputs only");
  static_assert(!UPD || (!FUSE && MODE == STREAM_MODE_ZERO_PURE), "the residual update goes with the level-1 CConv1");
  using C = KCfg<BF16C, FUSE, UPD>;
  constexpr int NRV = C::NRV;
  if (P.st && P.st->done) return;
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t *vs = smem;
  uint8_t *ds = smem + NRV * C::SL;
  uint8_t *kb = ds + ND * DBUF;
  StreamMeta &M = *(StreamMeta *)(kb + C::CB);
  volatile int *sabort = &M.abort_;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x;
  const int nz = P.dm.nz;
  const bool has_x1 = P.c12 != nullptr;

  if (tid == 0) {
    for (int i = 0; i < NRV; ++i) {
      mbar_init(&M.full[i], 1);
      mbar_init(&M.empty[i], NCW);
      M.kstart[i] = 0u;
      M.kend[i] = 0u;
    }
    for (int i = 0; i < ND; ++i) {
      mbar_init(&M.dfull[i], 1);
      mbar_init(&M.dempty[i], NCW);
    }
    *sabort = 0;
    M.last_ = 0;
    umma::fence_mbar_init();
    umma::fence_proxy_async_smem();
  }
  for (int i = tid; i < 3 * 27; i += NTHREADS) M.ktab[i] = (&P.ktab[0][0])[i];
  __syncthreads();  // the only CTA-wide barrier

  if (warp == NCW) {
    // ------------------------------------------------------------------ producer
    if (lane != 0) return;
    bool fail = false;
    uint32_t vi = 0, vrel = 0;  // loads issued / slots known released
    uint32_t khead = 0, ktail = 0, kpos = 0;
    uint32_t di = 0;            // descriptor loads issued (= units)
    // fused: q of the previous directions i = k1-1-j (j < qcnt, i >= 1) of Alg. 1; for PCG / FPCG the
    // current residual r_k and (FPCG) q_k
    int qcnt = 0, qslot[kMaxFusedOrtho] = {0, 0};
    const CUtensorMap *qmap0 = &P.tq;  // the map of box 0 (box 1 is always from the q ring)
    if (FUSE) {
      const int k1 = P.st->k + 1, no = P.st->n_ortho;
      qcnt = direction_dot_count(P.method, k1, no, kMaxFusedOrtho);
      if (P.method == kMethodNpsdo) {
        for (int j = 0; j < kMaxFusedOrtho; ++j) qslot[j] = ring_slot(max(k1 - 1 - j, 1), no);
      } else {
        qmap0 = &P.aux[P.st->k & 1];
        qslot[1] = ring_slot(max(k1 - 1, 1), no);
      }
    }
    // the residual update: r_k from buffer k mod 2 and q of the pending step
    const bool upd = UPD && P.st->upd_pending;
    const CUtensorMap *tvm = (UPD && (P.st->k & 1)) ? &P.aux[0] : &P.tv;
    const int uslot = UPD ? ring_slot(P.st->k + 1, P.st->n_ortho) : 0;
    auto release_next = [&]() {
      const int sl = (int)(vrel % NRV);
      if (!mbar_sleep_wait(&M.empty[sl], (vrel / NRV) & 1u, kWaitNs)) {
        fail = true;
        return;
      }
      ktail = M.kend[sl];
      ++vrel;
    };
    // units blockIdx.x + m G: the CTAs sweep the units in order together, so
    // neighbouring tiles are streamed at about the same time and their halo
    // rows are read from HBM once (L2); handing units out dynamically was
    // measured 10-20% slower for that reason.
    // descriptors of this CTA's m-th unit u (u < 0: tell the consumers there is none)
    auto issue_desc = [&](int m, int u) {
      if (fail) return;
      const int b = m % ND;
      if (m >= ND && !mbar_sleep_wait(&M.dempty[b], ((m / ND) - 1) & 1, kWaitNs)) {
        fail = true;
        return;
      }
      M.unit[b] = u;
      if (u < 0) {
        mbar_arrive(&M.dfull[b]);
      } else {
        const Unit U = unit_at(P, u);
        mbar_expect_tx(&M.dfull[b], (uint32_t)(U.nzu * (int)sizeof(PlaneDesc)));
        bulk_load(ds + b * DBUF, P.desc + (size_t)U.t * nz + U.zs, (uint32_t)(U.nzu * (int)sizeof(PlaneDesc)),
                  &M.dfull[b]);
      }
      ++di;
    };
    int u = (int)blockIdx.x < P.units ? (int)blockIdx.x : -1;
    issue_desc(0, u);
    for (int m = 0; u >= 0 && !fail && !*sabort; ++m) {
      const Unit U = unit_at(P, u);
      const int un = u + G < P.units ? u + G : -1;
      const PlaneDesc *D = (const PlaneDesc *)(ds + (m % ND) * DBUF);
      bool dready = false;
      const int T = (U.nzu + 1) >> 1;
      for (int t = -1; t < T && !fail; ++t) {
        // slot: planes z0+1, z0+2 (prologue: zs-1, zs), x1 of z0, z0+1 and the kernel blocks of z0, z0+1
        while (!fail && vrel + NRV <= vi) release_next();
        uint32_t kbytes = 0, koff = 0;
        if (t >= 0) {
          if (!dready) {
            if (!mbar_sleep_wait(&M.dfull[m % ND], (m / ND) & 1, kWaitNs)) {
              fail = true;
              break;
            }
            dready = true;
          }
          const int j0 = 2 * t;
          const uint32_t cp0 = min(D[j0].cpad, (uint32_t)NT);
          const uint32_t cp1 = j0 + 1 < U.nzu ? min(D[j0 + 1].cpad, (uint32_t)NT) : 0u;
          koff = D[j0].off;
          kbytes = (cp0 + cp1) * (uint32_t)C::EB;
        }
        // the block must not cross the end of the buffer: if it would, it starts at 0
        // and the bytes left at the end count as used until this slot is released
        const bool wrap = kpos + kbytes > (uint32_t)C::CB;
        const uint32_t waste = wrap ? (uint32_t)C::CB - kpos : 0u;
        while (!fail && vrel < vi && (khead - ktail) + waste + kbytes > (uint32_t)C::CB) release_next();
        if (fail) break;
        const int sl = (int)(vi % NRV);
        if (wrap) {
          khead += waste;
          kpos = 0;
        }
        M.kstart[sl] = kpos;
        khead += kbytes;
        M.kend[sl] = khead;
        uint8_t *dst = vs + sl * C::SL;
        uint64_t *bar = &M.full[sl];
        const int zv = t < 0 ? U.zs - 1 : U.zs + 2 * t + 1;
        const bool x1 = has_x1 && t >= 0;
        const int nq = (FUSE && t >= 0) ? qcnt : 0;
        mbar_expect_tx(bar, 2u * VPLANE + (upd ? 2u * VPLANE : 0u) + (x1 ? (uint32_t)XBOX : 0u) +
                                (uint32_t)nq * (uint32_t)XBOX + kbytes);
        tma_load_3d(dst, tvm, U.x0 - 4, U.y0 - 1, zv, bar);
        if (upd) tma_load_4d(dst + QUOFF, &P.aux[1], U.x0 - 4, U.y0 - 1, zv, uslot, bar);
        if (x1) tma_load_3d(dst + X1OFF, &P.tx1, U.x0, U.y0, U.zs + 2 * t, bar);
        if (FUSE)
          for (int j = 0; j < nq; ++j)
            tma_load_4d(dst + QOFF + XBOX * j, j ? &P.tq : qmap0, U.x0, U.y0, U.zs + 2 * t, qslot[j], bar);
        if (kbytes) bulk_load(kb + kpos, P.cache + (size_t)koff * C::EB, kbytes, bar);
        kpos += kbytes;
        ++vi;
        if (t == 0) issue_desc(m + 1, un);  // one unit ahead
      }
      if (fail) break;
      u = un;
    }
    if (fail) {
      *sabort = 1;
      if (P.err) atomicExch(P.err, 1);
    }
    // every copy must have landed before the CTA may exit
    for (uint32_t i = vi > (uint32_t)NRV ? vi - NRV : 0u; i < vi; ++i)
      (void)mbar_sleep_wait(&M.full[i % NRV], (i / NRV) & 1u, kWaitNs);
    for (uint32_t m = di > (uint32_t)ND ? di - ND : 0u; m < di; ++m)
      (void)mbar_sleep_wait(&M.dfull[m % ND], (m / ND) & 1u, kWaitNs);
    return;
  }

  // -------------------------------------------------------------------- consumers
  // warp w owns the 8x8 patch x in [8w, 8w+8) of the tile; a thread owns
  // column xi = lane % 8 and rows ra = 2 (lane / 8), ra + 1
  bool ok = true;
  auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
    if (ok && !mbar_sleep_wait(bar, parity, kWaitNs)) {
      ok = false;
      *sabort = 1;
      if (P.err) atomicExch(P.err, 1);
    }
    return ok;
  };
  const float sc = P.vscale ? *P.vscale : 1.f;
  const float c1 = has_x1 ? (float)P.c12[0] : 0.f, c2 = has_x1 ? (float)P.c12[1] : 1.f;
  const int cxn = P.dm.nx >> 1, cyn = P.dm.ny >> 1;
  const long long nxy = (long long)P.dm.nx * P.dm.ny;
  const int xi = lane & 7, ra = 2 * (lane >> 3);
  const int xb = PW * warp + xi;  // x within the tile = bit of the row masks
  // box index of the cell (x-1, y-1) of row ra in a plane (the box starts at x0-4, y0-1)
  const int vbase = ra * BXW + xb + 3;
  uint32_t sl = 0, sph = 0;  // next slot and the parity of its phase
  DF fdot[kMaxFusedOrtho];   // fused: per-thread double-float dots z . q_i
  int fqcnt = 0;
  if (FUSE) fqcnt = direction_dot_count(P.method, P.st->k + 1, P.st->n_ortho, kMaxFusedOrtho);
  // residual update: every window value is r_k - alpha q (the same FP32 FMA as
  // k_update4), the thread's own cells are written to the other buffer and
  // summed into ||r_{k+1}||^2
  const bool upd = UPD && P.st->upd_pending;
  const float uaf = upd ? (float)P.st->alpha : 0.f;
  float *const rnext = upd ? P.rb[(P.st->k + 1) & 1] : nullptr;
  DF unorm;
  auto load_col = [&](const float *pl, int e) -> float {
    return upd ? fmaf(-uaf, pl[(QUOFF / 4) + e], pl[e]) : pl[e];
  };

  for (int m = 0; ok; ++m) {
    if (!wait(&M.dfull[m % ND], (m / ND) & 1)) break;
    const int u = M.unit[m % ND];
    if (u < 0) break;
    const Unit U = unit_at(P, u);
    const int gx = U.x0 + xb, gy = U.y0 + ra;
    const bool in_x = gx < P.dm.nx;
    const bool in_a = in_x && gy < P.dm.ny, in_b = in_x && gy + 1 < P.dm.ny;
    const PlaneDesc *D = (const PlaneDesc *)(ds + (m % ND) * DBUF);
    Col pA, pB;  // planes zs-1, zs
    {
      if (!wait(&M.full[sl], sph)) break;
      const float *pl = (const float *)(vs + sl * C::SL);
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        const int e = vbase + (q / 3) * BXW + q % 3;
        pA.set(q, load_col(pl, e));
        pB.set(q, load_col(pl, BXW * BYH + e));
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&M.empty[sl]);
      if (++sl == NRV) {
        sl = 0;
        sph ^= 1u;
      }
    }
    float *op = P.out + (long long)U.zs * nxy + (long long)gy * P.dm.nx + gx;
    float *rp = upd ? rnext + (long long)U.zs * nxy + (long long)gy * P.dm.nx + gx : nullptr;
    float *pp = P.pooled ? P.pooled + ((long long)(U.zs >> 1) * cyn + (gy >> 1)) * cxn + (gx >> 1) : nullptr;
    const long long pstep = (long long)cxn * cyn;
    const bool pown = in_a && !(xi & 1);  // even column writes the 2x2x2 block's mean
    const int T = (U.nzu + 1) >> 1;
    for (int t = 0; t < T; ++t) {
      const int j0 = 2 * t;
      const bool two = j0 + 1 < U.nzu;
      if (!wait(&M.full[sl], sph)) break;
      const uint8_t *slot = vs + sl * C::SL;
      const float *pl = (const float *)slot;
      Col pC, pD;  // planes z0+1, z0+2
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        const int e = vbase + (q / 3) * BXW + q % 3;
        pC.set(q, load_col(pl, e));
        pD.set(q, load_col(pl, BXW * BYH + e));
      }
      if (UPD && upd) {  // r_{k+1} of the thread's cells: the window centres of planes z0 (pB) and z0+1 (pC)
        const float ra0 = in_a ? pB.at(4) : 0.f, rb0 = in_b ? pB.at(7) : 0.f;
        const float ra1 = in_a && two ? pC.at(4) : 0.f, rb1 = in_b && two ? pC.at(7) : 0.f;
        if (in_a) rp[0] = ra0;
        if (in_b) rp[P.dm.nx] = rb0;
        if (two) {
          if (in_a) rp[nxy] = ra1;
          if (in_b) rp[nxy + P.dm.nx] = rb1;
        }
        rp += 2 * nxy;
        df_add(unorm, (ra0 * ra0 + rb0 * rb0) + (ra1 * ra1 + rb1 * rb1));
      }
      float x1v[4] = {0.f, 0.f, 0.f, 0.f};  // (row a, z0), (row b, z0), (row a, z1), (row b, z1)
      if (has_x1) {
        const float *xs = (const float *)(slot + X1OFF) + ra * XBW + xb;
        x1v[0] = xs[0];
        x1v[1] = xs[XBW];
        x1v[2] = xs[XBW * TY];
        x1v[3] = xs[XBW * TY + XBW];
      }
      const uint32_t *kblk = (const uint32_t *)(kb + M.kstart[sl]);
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      {
        const PlaneDesc &d0 = D[j0];
        const int cl0 = (int)((d0.patch >> (2 * warp)) & 3u);
        if (cl0 != 3) cconv_pure_pair<MODE>(P, cl0, pA, pB, pC, acc[0], acc[1]);
        else cconv_generic_pair<BF16C, MODE>(d0, ra, xb, kblk, M.ktab, pA, pB, pC, acc[0], acc[1]);
        if (two) {
          const PlaneDesc &d1 = D[j0 + 1];
          const int cl1 = (int)((d1.patch >> (2 * warp)) & 3u);
          if (cl1 != 3) {
            cconv_pure_pair<MODE>(P, cl1, pB, pC, pD, acc[2], acc[3]);
          } else {
            const uint32_t *kblk1 = kblk + (size_t)min(d0.cpad, (uint32_t)NT) * (C::EB / 4);
            cconv_generic_pair<BF16C, MODE>(d1, ra, xb, kblk1, M.ktab, pB, pC, pD, acc[2], acc[3]);
          }
        }
      }
      if (FUSE) {
        // z = mask_fluid(c1 x1 + c2 x2) (Sec. 4.2 output restriction) and the dots z . q_i
        const uint32_t bit = 1u << xb;
        const PlaneDesc &d0 = D[j0];
        bool fl[4];
        fl[0] = (d0.row[ra].w & bit) != 0u;
        fl[1] = (d0.row[ra + 1].w & bit) != 0u;
        fl[2] = two && (D[j0 + 1].row[ra].w & bit) != 0u;
        fl[3] = two && (D[j0 + 1].row[ra + 1].w & bit) != 0u;
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] = fl[i] ? fmaf(c1, x1v[i], c2 * acc[i]) : 0.f;
#pragma unroll
        for (int j = 0; j < kMaxFusedOrtho; ++j) {
          if (j < fqcnt) {
            const float *qs = (const float *)(slot + QOFF + XBOX * j) + ra * XBW + xb;
            df_add(fdot[j], (acc[0] * qs[0] + acc[1] * qs[XBW]) + (acc[2] * qs[XBW * TY] + acc[3] * qs[XBW * TY + XBW]));
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&M.empty[sl]);
      if (++sl == NRV) {
        sl = 0;
        sph ^= 1u;
      }
      if (!FUSE) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          acc[i] *= sc;
          if (has_x1) acc[i] = fmaf(c1, x1v[i], c2 * acc[i]);
        }
      }
      if (in_a) op[0] = acc[0];
      if (in_b) op[P.dm.nx] = acc[1];
      if (two) {
        if (in_a) op[nxy] = acc[2];
        if (in_b) op[nxy + P.dm.nx] = acc[3];
      }
      op += 2 * nxy;
      if (pp) {  // z0 even, rows ra, ra+1: the thread holds half of a 2x2x2 block, its neighbour lane the rest
        float tp = (acc[0] + acc[1]) + (acc[2] + acc[3]);
        tp += __shfl_xor_sync(0xffffffffu, tp, 1);
        if (pown) *pp = 0.125f * tp;
        pp += pstep;
      }
      pA = pC;
      pB = pD;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&M.dempty[m % ND]);
  }
  if (FUSE) fused_finish(P, M, fdot, fqcnt);
  if (UPD && upd) update_finish(P, M, unorm);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
namespace {

int grid_for_units(long long units, int cap) {
  long long g = units < cap ? units : cap;
  return (int)(g < 1 ? 1 : g);
}

template <bool BF16C, bool FUSE, int MODE, bool UPD = false>
int stream_occupancy() {
  // per device: the dynamic shared-memory opt-in is a per-device function attribute
  static int occ[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!occ[dev]) {
    int o = 0;
    using C = KCfg<BF16C, FUSE, UPD>;
    cudaFuncSetAttribute(k_cconv_stream<BF16C, FUSE, MODE, UPD>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_cconv_stream<BF16C, FUSE, MODE, UPD>, NTHREADS, C::SMEM);
    occ[dev] = o < 1 ? 1 : o;
  }
  return occ[dev];
}

// The instantiation for a (fused, mode) pair: the mode is a template argument
// so that the level-1 launches carry only the fluid kernel's code.
template <bool BF16C>
int stream_occupancy_of(bool fused, int mode, bool upd) {
  if (fused) return stream_occupancy<BF16C, true, STREAM_MODE_FLUID_ONLY>();
  if (upd) return stream_occupancy<BF16C, false, STREAM_MODE_ZERO_PURE, true>();
  if (mode == STREAM_MODE_ZERO_PURE) return stream_occupancy<BF16C, false, STREAM_MODE_ZERO_PURE>();
  if (mode == STREAM_MODE_FLUID_ONLY) return stream_occupancy<BF16C, false, STREAM_MODE_FLUID_ONLY>();
  return stream_occupancy<BF16C, false, STREAM_MODE_ALL>();
}

template <bool BF16C>
void launch_stream_of(bool fused, bool upd, const StreamParams &P, int grid, cudaStream_t s) {
  if (fused)
    k_cconv_stream<BF16C, true, STREAM_MODE_FLUID_ONLY><<<grid, NTHREADS, KCfg<BF16C, true>::SMEM, s>>>(P);
  else if (upd)
    k_cconv_stream<BF16C, false, STREAM_MODE_ZERO_PURE, true><<<grid, NTHREADS, KCfg<BF16C, false, true>::SMEM, s>>>(P);
  else if (P.mode == STREAM_MODE_ZERO_PURE)
    k_cconv_stream<BF16C, false, STREAM_MODE_ZERO_PURE><<<grid, NTHREADS, KCfg<BF16C, false>::SMEM, s>>>(P);
  else if (P.mode == STREAM_MODE_FLUID_ONLY)
    k_cconv_stream<BF16C, false, STREAM_MODE_FLUID_ONLY><<<grid, NTHREADS, KCfg<BF16C, false>::SMEM, s>>>(P);
  else
    k_cconv_stream<BF16C, false, STREAM_MODE_ALL><<<grid, NTHREADS, KCfg<BF16C, false>::SMEM, s>>>(P);
}

// cuTensorMapEncodeTiled, looked up through the runtime so that the library
// has no link-time dependency on the driver library.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

bool encode_map(CUtensorMap *m, const float *base, Dims d, int bw, int bh, int bd) {
  const EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz};
  cuuint64_t strides[2] = {(cuuint64_t)d.nx * 4u, (cuuint64_t)d.nx * (cuuint64_t)d.ny * 4u};
  cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, (cuuint32_t)bd};
  cuuint32_t es[3] = {1u, 1u, 1u};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)base, dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

CUresult encode_map_4d(CUtensorMap *m, const float *base, Dims d, int nring, int bw = XBW, int bh = TY) {
  const EncodeTiledFn fn = encode_fn();
  if (!fn) return CUDA_ERROR_NOT_SUPPORTED;
  cuuint64_t dims[4] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz, (cuuint64_t)nring};
  const cuuint64_t rowb = (cuuint64_t)d.nx * 4u;
  cuuint64_t strides[3] = {rowb, rowb * (cuuint64_t)d.ny, rowb * (cuuint64_t)d.ny * (cuuint64_t)d.nz};
  cuuint32_t box[4] = {(cuuint32_t)bw, (cuuint32_t)bh, 2u, 1u};
  cuuint32_t es[4] = {1u, 1u, 1u, 1u};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void *)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

}  // namespace

bool stream_shape_ok(Dims d) { return d.nx % 4 == 0 && d.nx >= 4; }

long long stream_desc_count(Dims d) {
  const long long ntiles = (long long)((d.nx + TX - 1) / TX) * ((d.ny + TY - 1) / TY);
  return ntiles * d.nz;
}

size_t stream_desc_bytes() { return sizeof(PlaneDesc); }

int cached_entry_bytes(bool bf16) { return bf16 ? KCfg<true>::EB : KCfg<false>::EB; }

bool stream_fusion_ok(int n_ortho) { return n_ortho <= kMaxFusedOrtho; }

int stream_cap(bool bf16, bool fused, int mode, bool upd, int num_sms) {
  const int occ = bf16 ? stream_occupancy_of<true>(fused, mode, upd) : stream_occupancy_of<false>(fused, mode, upd);
  int cap = num_sms * occ;
  if ((fused || upd) && cap > kRedMaxBlocks) cap = kRedMaxBlocks;
  return cap;
}

int choose_stream_units(Dims d, const uint8_t *skip, int bit, int cap, int *list, int *n) {
  // the even chunk with the fewest slots per CTA over the units that have a
  // plane without the skip bit (per-tile prefix counts of those planes), and
  // those units in ascending order
  const int ntiles = ((d.nx + TX - 1) / TX) * ((d.ny + TY - 1) / TY);
  std::vector<int> pre((size_t)ntiles * (d.nz + 1));
  for (int t = 0; t < ntiles; ++t) {
    const uint8_t *f = skip + (size_t)t * d.nz;
    int *pt = pre.data() + (size_t)t * (d.nz + 1);
    pt[0] = 0;
    for (int z = 0; z < d.nz; ++z) pt[z + 1] = pt[z] + ((f[z] & bit) ? 0 : 1);
  }
  auto active = [&](int t, int z0, int z1) {
    const int *pt = pre.data() + (size_t)t * (d.nz + 1);
    return pt[std::min(z1, d.nz)] > pt[z0];
  };
  int zc = 32;
  long long best = -1;
  for (int c = 32; c >= 2; c -= 2) {
    const int nch = (d.nz + c - 1) / c;
    long long act = 0;
    for (int ch = 0; ch < nch; ++ch)
      for (int t = 0; t < ntiles; ++t) act += active(t, ch * c, (ch + 1) * c) ? 1 : 0;
    const long long cost = ((act + cap - 1) / cap) * ((c + 1) / 2 + 1);
    if (best < 0 || cost < best) {
      best = cost;
      zc = c;
    }
  }
  const int nch = (d.nz + zc - 1) / zc;
  int m = 0;
  for (int ch = 0; ch < nch; ++ch)
    for (int t = 0; t < ntiles; ++t)
      if (active(t, ch * zc, (ch + 1) * zc)) list[m++] = ch * ntiles + t;
  *n = m;
  return zc;
}

void stream_units_work(Dims d, const int *list, int n, int zc, const uint16_t *mcount, long long *cells,
                       long long *mixed) {
  const int ntx = (d.nx + TX - 1) / TX, nty = (d.ny + TY - 1) / TY, ntiles = ntx * nty;
  long long c = 0, m = 0;
  for (int i = 0; i < n; ++i) {
    const int t = list[i] % ntiles, ch = list[i] / ntiles;
    const int w = std::min(TX, d.nx - (t % ntx) * TX), hgt = std::min(TY, d.ny - (t / ntx) * TY);
    const int z0 = ch * zc, z1 = std::min(d.nz, z0 + zc);
    c += (long long)w * hgt * (z1 - z0);
    if (mcount)
      for (int z = z0; z < z1; ++z) m += mcount[(size_t)t * d.nz + z];
  }
  *cells = c;
  *mixed = m;
}

namespace {
// out[t][z] = any (tile, plane) within (+-rx, +-ry, +-rz) tiles and planes of
// (t, z) lacks `bit` in skip; stored inverted (1 = none does) when `invert`.
__global__ void k_dilate_flags(const uint8_t *__restrict__ skip, int ntx, int nty, int nz, int bit, int rx, int ry,
                               int rz, int invert, uint8_t *__restrict__ out) {
  const int total = ntx * nty * nz;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int z = i % nz, t = i / nz, tx = t % ntx, ty = t / ntx;
    bool any = false;
    for (int dy = -ry; dy <= ry && !any; ++dy)
      for (int dx = -rx; dx <= rx && !any; ++dx) {
        const int ux = tx + dx, uy = ty + dy;
        if (ux < 0 || uy < 0 || ux >= ntx || uy >= nty) continue;
        const uint8_t *f = skip + (size_t)(uy * ntx + ux) * nz;
        for (int dz = -rz; dz <= rz; ++dz) {
          const int uz = z + dz;
          if (uz >= 0 && uz < nz && !(f[uz] & bit)) {
            any = true;
            break;
          }
        }
      }
    out[i] = (uint8_t)(invert ? !any : any);
  }
}
}  // namespace

void launch_dilate_flags(const uint8_t *skip, Dims d, int bit, int rx, int ry, int rz, bool invert, uint8_t *out,
                         cudaStream_t s) {
  const int ntx = (d.nx + TX - 1) / TX, nty = (d.ny + TY - 1) / TY;
  const long long total = (long long)ntx * nty * d.nz;
  const int g = (int)std::min<long long>((total + 255) / 256, 148LL * 8);
  k_dilate_flags<<<g < 1 ? 1 : g, 256, 0, s>>>(skip, ntx, nty, d.nz, bit, rx, ry, rz, invert ? 1 : 0, out);
}

// Planes per unit of the setup kernels at a level: up to 32 (a unit's kernel
// blocks are contiguous in the cache, so the chunks must be even), fewer when
// the level is too small to give every SM a few units.
static int setup_chunk(Dims d, int num_sms) {
  const long long ntiles = (long long)((d.nx + TX - 1) / TX) * ((d.ny + TY - 1) / TY);
  int zc = ZCG;
  while (zc > 2 && ntiles * ((d.nz + zc - 1) / zc) < 4LL * num_sms) zc >>= 1;
  return zc;
}

void launch_classify(const uint8_t *lab, const ushort2 *counts, Dims d, uint32_t full, void *desc, unsigned *totals,
                     uint8_t *skip, uint16_t *mcount, int num_sms, cudaStream_t s) {
  const int zc = setup_chunk(d, num_sms);
  const long long units = (long long)((d.nx + TX - 1) / TX) * ((d.ny + TY - 1) / TY) * ((d.nz + zc - 1) / zc);
  k_classify<<<grid_for_units(units, num_sms * 8), CLT, 0, s>>>(lab, counts, d, full, zc, (PlaneDesc *)desc, totals,
                                                                  skip, mcount);
}

void launch_generate(bool bf16, const uint8_t *lab, const ushort2 *counts, Dims d, const CConvW *w, int nblk,
                     const void *desc, void *cache0, void *cache1, const uint8_t *wsplit0, const uint8_t *wsplit1,
                     int nsplit, int *err, int num_sms, cudaStream_t s) {
  const PlaneDesc *pd = (const PlaneDesc *)desc;
  if (wsplit0) {  // tensor cores: image counts exact in BF16 (levels <= 3); units within the classification's
    const int zc = setup_chunk(d, num_sms);
    const long long units = (long long)((d.nx + TX - 1) / TX) * ((d.ny + TY - 1) / TY) * ((d.nz + zc - 1) / zc);
    // CTAs per SM by shared memory (at most 7 by TMEM: 64 columns each): the level-1
    // label window takes 11.3 KB more
    const bool window = lab != nullptr;
    const int smem = gen_smem_bytes(nsplit, window);
    const int per_sm = std::min(7, (227 * 1024) / (smem + 1024));
    const int g = grid_for_units(units, num_sms * per_sm);
    static int configured[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !configured[dev]) {
      cudaFuncSetAttribute(k_generate_tc<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, gen_smem_bytes(1, true));
      cudaFuncSetAttribute(k_generate_tc<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, gen_smem_bytes(3, true));
      cudaFuncSetAttribute(k_generate_tc<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           gen_smem_bytes(3, true));
      configured[dev] = 1;
    }
    if (nsplit == 1)
      k_generate_tc<1, true><<<g, GT, smem, s>>>(lab, counts, d, wsplit0, wsplit1, nblk, pd, (uint32_t *)cache0,
                                                 (uint32_t *)cache1, zc, err);
    else if (bf16)
      k_generate_tc<3, true><<<g, GT, smem, s>>>(lab, counts, d, wsplit0, wsplit1, nblk, pd, (uint32_t *)cache0,
                                                 (uint32_t *)cache1, zc, err);
    else
      k_generate_tc<3, false><<<g, GT, smem, s>>>(lab, counts, d, wsplit0, wsplit1, nblk, pd, (uint32_t *)cache0,
                                                  (uint32_t *)cache1, zc, err);
    return;
  }
  const int g = grid_for_units((long long)((d.nx + TX - 1) / TX) * ((d.ny + TY - 1) / TY) * d.nz, num_sms * 8);
  if (bf16)
    k_generate<true><<<g, NT, 0, s>>>(lab, counts, d, w, nblk, pd, (uint32_t *)cache0, (uint32_t *)cache1);
  else
    k_generate<false><<<g, NT, 0, s>>>(lab, counts, d, w, nblk, pd, (uint32_t *)cache0, (uint32_t *)cache1);
}

int launch_cconv_stream(bool bf16, Dims dm, const float *kfix, const void *desc, const void *cache, const float *v,
                        const float *vscale, float *out, float *pooled, const float *x1, const double *c12, int mode,
                        const SolveState *st, int *err, int num_sms, cudaStream_t s,
                        const StreamFusion *fuse, const StreamUpdate *upd, const StreamUnits *units) {
  StreamParams P;
  memset(&P, 0, sizeof(P));
  if (upd && (fuse || mode != STREAM_MODE_ZERO_PURE || c12)) return -1;
  P.mode = fuse ? STREAM_MODE_FLUID_ONLY : mode;
  if (upd) {
    // r_k is read from buffer k mod 2 (tv over rb[0], aux[0] over rb[1]); q of the pending step from the ring
    if (v != upd->rb[0] || !encode_map(&P.aux[0], upd->rb[1], dm, BXW, BYH, 2)) return -1;
    if (encode_map_4d(&P.aux[1], upd->qring, dm, upd->nring, BXW, BYH) != CUDA_SUCCESS) return -1;
    P.rb[0] = upd->rb[0];
    P.rb[1] = upd->rb[1];
    P.upart = upd->part;
    P.uticket = upd->ticket;
    P.hist = upd->hist;
    P.stw = upd->st;
  }
  if (fuse) {
    // the q ring as a 4-D tensor (nx, ny, nz, slot); slot stride = one grid
    const CUresult r = encode_map_4d(&P.tq, fuse->qring, dm, fuse->nring);
    if (r != CUDA_SUCCESS) return -1;
    // the residual buffers as one-slot tensors of the same shape (read by PCG / FPCG)
    for (int i = 0; i < 2; ++i)
      if (encode_map_4d(&P.aux[i], fuse->rb[i] ? fuse->rb[i] : fuse->rb[0], dm, 1) != CUDA_SUCCESS) return -1;
    P.part = fuse->part;
    P.ticket = fuse->ticket;
    P.method = fuse->method;
    P.stw = fuse->st;
  }
  if (!encode_map(&P.tv, v, dm, BXW, BYH, 2)) return -1;
  if (c12 && !encode_map(&P.tx1, x1, dm, XBW, TY, 2)) return -1;
  // class tables in the stored format: BF16 pairs (the constants are BF16 values in that form) or FP32 words
  for (int c = 0; c < 3; ++c) {
    const float *k = kfix + 27 * c;
    for (int a = 0; a < 27; ++a) {
      uint32_t u;
      memcpy(&u, &k[a], 4);
      P.ktab[c][a] = u;
    }
    if (bf16)
      for (int j = 0; j < 14; ++j) {
        uint32_t lo, hi = 0u;
        memcpy(&lo, &k[2 * j], 4);
        if (2 * j + 1 < 27) memcpy(&hi, &k[2 * j + 1], 4);
        P.ktab[c][j] = (lo >> 16) | (hi & 0xFFFF0000u);
      }
  }
  P.dm = dm;
  P.ntx = (dm.nx + TX - 1) / TX;
  P.ntiles = P.ntx * ((dm.ny + TY - 1) / TY);
  P.desc = (const PlaneDesc *)desc;
  P.cache = (const uint8_t *)cache;
  P.vscale = vscale;
  P.out = out;
  P.pooled = pooled;
  P.c12 = c12;
  P.st = st;
  P.err = err;
  for (int c = 0; c < 3; ++c) {
    const float *k = kfix + 27 * c;
    PairKernel &K = P.kp[c];
    for (int dz = 0; dz < 3; ++dz) {
      const float *kz = k + 9 * dz;
      for (int i = 0; i < 4; ++i) {
        K.up[dz][i] = make_float2(kz[2 * i], kz[2 * i + 1]);
        K.lo[dz][i] = make_float2(kz[2 * i + 1], kz[2 * i + 2]);
      }
      K.up8[dz] = kz[8];
      K.lo0[dz] = kz[0];
    }
  }
  const int occ = bf16 ? stream_occupancy_of<true>(fuse != nullptr, P.mode, upd != nullptr)
                       : stream_occupancy_of<false>(fuse != nullptr, P.mode, upd != nullptr);
  int cap = num_sms * occ;
  if ((fuse || upd) && cap > kRedMaxBlocks) cap = kRedMaxBlocks;  // one row of partials per CTA
  // the chunk of planes (even, so that a step's two planes never straddle a
  // classification unit) that minimises the slots on the critical path:
  // units per CTA (rounded up) x (steps per unit + the prologue slot)
  if (units) {  // a list of the units that have work, with its chunk
    P.zc = units->zc;
    P.units = units->n;
    P.ulist = units->list;
  } else {
    int zc = 32;
    long long best = -1;
    for (int c = 32; c >= 2; c -= 2) {
      const long long nu = (long long)P.ntiles * ((dm.nz + c - 1) / c);
      const long long per_cta = (nu + cap - 1) / cap;
      const long long cost = per_cta * ((c + 1) / 2 + 1);
      if (best < 0 || cost < best) {
        best = cost;
        zc = c;
      }
    }
    P.zc = zc;
    P.units = P.ntiles * ((dm.nz + zc - 1) / zc);
  }
  if (fuse && (size_t)cap * kMaxFusedOrtho > fuse->part_cap) return -1;  // partials do not fit
  if (upd && (size_t)cap > upd->part_cap) return -1;
  const int grid = grid_for_units(P.units, cap);
  if (bf16) launch_stream_of<true>(fuse != nullptr, upd != nullptr, P, grid, s);
  else launch_stream_of<false>(fuse != nullptr, upd != nullptr, P, grid, s);
  return 0;
}

}  // namespace nps
