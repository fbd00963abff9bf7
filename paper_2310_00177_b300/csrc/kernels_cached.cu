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
//   tiles of 32 (x) x 4 (y) cells; warp w of a CTA holds row w of a tile;
//   one plane descriptor per (tile, z): one word per row of each of the bit
//   masks "mixed window", "pure-fluid window", "pure-air window" and "the cell
//   is fluid", and the place of the plane's kernel block in the cache;
//   a kernel block holds the kernels of the plane's mixed cells in the order of
//   their bit index, tap-major: word (j, i) of a block with stride cpad is
//   tap pair j of mixed cell i (BF16 form: taps 2j and 2j+1 as a BF16 pair,
//   14 words per cell) or tap j of mixed cell i (FP32 form: 27 words per cell);
//   cpad is the mixed count rounded up to 4, so that every block starts and
//   ends on a 16-byte boundary.
//
// Per solve: k_classify (masks, block sizes, block offsets by one atomic per
// unit of 32 planes) and k_generate (the FP32 contraction of the 54 image
// features of a mixed cell, the arithmetic of the CUDA-core CConv, rounded to
// BF16 in the BF16 form).
//
// Per iteration: k_cconv_stream.  Each CTA marches units (a tile and a chunk
// of planes) along z.  Thread 0 is the producer: it keeps RV vector planes in
// flight (a 40 x 6 TMA tensor box with the one-cell halo, the plane's
// descriptor and, when the output is combined, the 32 x 4 box of x1), and as
// soon as a plane's descriptor has arrived it issues the bulk copy of the
// plane's kernel block into a circular buffer of shared memory, up to NK
// blocks ahead.  All threads consume: planes z-1 and z of the vector window
// live in registers, plane z+1 comes from its slot, the kernel of a uniform
// window is one of the three constants (kernel parameters), that of a mixed
// window is read from its block.  One CTA barrier per plane frees the slots.
// Fusions: scaling by the input normalisation (level-1 CConv1), the 2x2x2
// mean pooling of the output (CConv1), the combination x = c1 x1 + c2 x2
// (CConv2 at levels >= 2).
//
// Every wait on an mbarrier is bounded (1 s of %globaltimer); a timeout sets
// *err, ends the kernel uniformly at the next CTA barrier and waits (bounded)
// for the copies still in flight before returning.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "nps_common.cuh"
#include "nps_kernels.h"
#include "umma.cuh"

namespace nps {

namespace {

using umma::globaltimer;
using umma::mbar_init;
using umma::mbar_try_wait;
using umma::mbar_wait_bounded;
using umma::smem_u32;

constexpr int TX = 32, TY = 4, NT = TX * TY;  // tile; warp w holds row w
constexpr int ZCG = 32;                       // planes per unit of the setup kernels
constexpr int BXW = TX + 8;                   // vector box: x0-4 .. x0+35 (start on a 16-byte boundary)
constexpr int BYH = TY + 2;                   // rows y0-1 .. y0+4
constexpr int VBYTES = BXW * BYH * 4;         // 960
constexpr int X1OFF = 1024;                   // x1 box (32 x 4) in a slot
constexpr int DOFF = X1OFF + NT * 4;          // plane descriptor in a slot
constexpr int VSLOT = DOFF + 128;             // 1664 bytes = 13 x 128
constexpr int RV = 10;                        // vector-plane slots
constexpr int NK = 8;                         // kernel blocks in flight
constexpr int kMetaBytes = 768;               // mbarriers, block positions, pooling exchange, abort flag
constexpr uint64_t kWaitNs = 1000000000ull;   // 1 s

struct PlaneDesc {
  uint32_t mixed[TY], fluid[TY], air[TY], self[TY];
  uint32_t off;    // first cache entry of the plane's kernel block (a multiple of 4)
  uint32_t cpad;   // entries of the block: the mixed count rounded up to 4
  uint32_t count;  // mixed cells of the plane
  uint32_t pad_;
};
static_assert(sizeof(PlaneDesc) == 80, "plane descriptor is 80 bytes");

template <bool BF16C>
struct KCfg {
  static constexpr int EB = BF16C ? 56 : 108;        // bytes per cached kernel
  static constexpr int CB = BF16C ? 16384 : 28672;   // circular kernel-block buffer
  static constexpr int SMEM = RV * VSLOT + CB + kMetaBytes;
};

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

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
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
// Bulk (untiled) copy global -> shared; both addresses and the size multiples of 16 bytes.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

}  // namespace

// ---------------------------------------------------------------------------
// Setup 1: classification.  One CTA (a 32 x 4 tile) per unit of ZCG planes.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_classify(const uint8_t *__restrict__ lab, const ushort2 *__restrict__ counts,
                                                 Dims d, uint32_t full, PlaneDesc *__restrict__ desc,
                                                 unsigned *__restrict__ totals) {
  __shared__ uint32_t sd[ZCG][20];
  __shared__ uint32_t sbase;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ntx = (d.nx + TX - 1) / TX, nty = (d.ny + TY - 1) / TY, nch = (d.nz + ZCG - 1) / ZCG;
  const int ntiles = ntx * nty;
  const long long units = (long long)ntiles * nch;
  const uint32_t kF = full, kA = full << 16;
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    const int t = (int)(u % ntiles), c = (int)(u / ntiles);
    const int x = (t % ntx) * TX + lane, y = (t / ntx) * TY + warp;
    const int zs = c * ZCG, nzu = min(ZCG, d.nz - zs);
    const bool inside = x < d.nx && y < d.ny;
    for (int j = 0; j < nzu; ++j) {
      const int z = zs + j;
      bool mixed = false, fl = false, ai = false, self = false;
      if (inside) {
        uint32_t k[27];
#pragma unroll
        for (int l = 0; l < 27; ++l)
          k[l] = image_key(lab, counts, d, x + l % 3 - 1, y + (l / 3) % 3 - 1, z + l / 9 - 1);
        bool uni = true;
#pragma unroll
        for (int l = 0; l < 27; ++l) uni &= k[l] == k[13];
        const bool pure = k[13] == 0u || k[13] == kF || k[13] == kA;
        mixed = !(uni && pure);
        fl = !mixed && k[13] == kF;
        ai = !mixed && k[13] == kA;
        self = lab != nullptr && k[13] == 1u;
      }
      const uint32_t bm = __ballot_sync(0xffffffffu, mixed), bf = __ballot_sync(0xffffffffu, fl);
      const uint32_t ba = __ballot_sync(0xffffffffu, ai), bs = __ballot_sync(0xffffffffu, self);
      if (lane == 0) {
        sd[j][warp] = bm;
        sd[j][TY + warp] = bf;
        sd[j][2 * TY + warp] = ba;
        sd[j][3 * TY + warp] = bs;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t tot = 0, cnt = 0;
      for (int j = 0; j < nzu; ++j) {
        uint32_t m = 0;
        for (int w = 0; w < TY; ++w) m += __popc(sd[j][w]);
        const uint32_t cp = (m + 3u) & ~3u;
        sd[j][16] = tot;
        sd[j][17] = cp;
        sd[j][18] = m;
        sd[j][19] = 0u;
        tot += cp;
        cnt += m;
      }
      sbase = tot ? atomicAdd(&totals[0], tot) : 0u;
      if (cnt) atomicAdd(&totals[1], cnt);
    }
    __syncthreads();
    uint32_t *dst = (uint32_t *)(desc + (size_t)t * d.nz + zs);
    for (int i = threadIdx.x; i < nzu * 20; i += NT) {
      uint32_t v = sd[i / 20][i % 20];
      if (i % 20 == 16) v += sbase;
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
  const int ntx = (d.nx + TX - 1) / TX, nty = (d.ny + TY - 1) / TY, nch = (d.nz + ZCG - 1) / ZCG;
  const int ntiles = ntx * nty;
  const long long units = (long long)ntiles * nch;
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    const int t = (int)(u % ntiles), c = (int)(u / ntiles);
    const int x = (t % ntx) * TX + lane, y = (t / ntx) * TY + warp;
    const int zs = c * ZCG, nzu = min(ZCG, d.nz - zs);
    __syncthreads();  // previous unit done with sd (and the weights are in place)
    {
      const uint32_t *src = (const uint32_t *)(desc + (size_t)t * d.nz + zs);
      uint32_t *dsd = (uint32_t *)sd;
      for (int i = threadIdx.x; i < nzu * 20; i += NT) dsd[i] = src[i];
    }
    __syncthreads();
    for (int j = 0; j < nzu; ++j) {
      const PlaneDesc &pd = sd[j];
      const uint32_t mw = pd.mixed[warp];
      if (!((mw >> lane) & 1u)) continue;
      uint32_t rank = __popc(mw & lanemask_lt());
      for (int q = 0; q < warp; ++q) rank += __popc(pd.mixed[q]);
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
// Per iteration: the streamed z-marching CConv.
// ---------------------------------------------------------------------------
struct StreamParams {
  CUtensorMap tv;   // input vector of the level: box 40 x 6 x 1 (FP32)
  CUtensorMap tx1;  // x1 of the level (combination only): box 32 x 4 x 1
  Dims dm;
  int ntx, ntiles, zc, units;
  const PlaneDesc *desc;
  const uint8_t *cache;
  const float *vscale;  // optional scale of the output (the input normalisation)
  float *out;
  float *pooled;        // optional 2x2x2 mean of the output
  const double *c12;    // non-null: out = c1 x1 + c2 CConv(v)
  const SolveState *st;
  int *err;
  float kS[27], kF[27], kA[27];  // kernels of the pure-solid, pure-fluid, pure-air windows
};

struct Unit {
  int t, x0, y0, zs, nzu;
};

__device__ __forceinline__ Unit unit_at(const StreamParams &P, int u) {
  Unit U;
  U.t = u % P.ntiles;
  const int c = u / P.ntiles;
  U.x0 = (U.t % P.ntx) * TX;
  U.y0 = (U.t / P.ntx) * TY;
  U.zs = c * P.zc;
  U.nzu = min(P.zc, P.dm.nz - U.zs);
  return U;
}

// sum_a k[a] v[a] over the window held as three 3x3 planes.
__device__ __forceinline__ float dot27(const float (&k)[27], const float (&vA)[9], const float (&vB)[9],
                                       const float (&vC)[9]) {
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    s0 = fmaf(k[j], vA[j], s0);
    s1 = fmaf(k[9 + j], vB[j], s1);
    s2 = fmaf(k[18 + j], vC[j], s2);
  }
  return (s0 + s1) + s2;
}

// Shared memory after the slots and the kernel-block buffer (8-byte aligned):
// vfull / vempty [RV], kfull / kempty [NK], pfull / pempty [2 pairs][2 buffers]
// (mbarriers), kstart / kend [NK] (positions of the blocks), poolx [2][2][16]
// (pooling exchange between the two warps of a row pair), abort flag.
struct StreamMeta {
  uint64_t vfull[RV], vempty[RV], kfull[NK], kempty[NK], pfull[4], pempty[4];
  uint32_t kstart[NK], kend[NK];
  float poolx[4][16];
  int abort_;
};
static_assert(sizeof(StreamMeta) <= kMetaBytes, "stream metadata fits");

constexpr int NTHREADS = NT + 32;  // four consumer warps (tile rows) and one producer warp

template <bool BF16C>
__global__ void __launch_bounds__(NTHREADS, 4) k_cconv_stream(const __grid_constant__ StreamParams P) {
  using C = KCfg<BF16C>;
  if (P.st && P.st->done) return;
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t *vs = smem;
  uint8_t *kb = smem + RV * VSLOT;
  StreamMeta &M = *(StreamMeta *)(kb + C::CB);
  volatile int *sabort = &M.abort_;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x;
  const int nz = P.dm.nz;
  const bool has_x1 = P.c12 != nullptr;

  if (tid == 0) {
    for (int i = 0; i < RV; ++i) {
      mbar_init(&M.vfull[i], 1);
      mbar_init(&M.vempty[i], TY);
    }
    for (int i = 0; i < NK; ++i) {
      mbar_init(&M.kfull[i], 1);
      mbar_init(&M.kempty[i], TY);
      M.kstart[i] = 0u;
      M.kend[i] = 0u;
    }
    for (int i = 0; i < 4; ++i) {
      mbar_init(&M.pfull[i], 1);
      mbar_init(&M.pempty[i], 1);
    }
    *sabort = 0;
    umma::fence_mbar_init();
    umma::fence_proxy_async_smem();
  }
  __syncthreads();  // the only CTA-wide barrier

  if (warp == TY) {
    // ------------------------------------------------------------------ producer
    if (lane != 0) return;
    bool fail = false;
    // V cursor: load vi = plane vu.zs - 1 + vj of the vm-th unit of this CTA
    int vm = 0, vj = 0;
    uint32_t vi = 0;
    Unit vu{};
    bool vvalid = (int)blockIdx.x < P.units;
    if (vvalid) vu = unit_at(P, blockIdx.x);
    // K cursor: block ki = plane ku.zs + kj; its descriptor travels with V load kvbase + kj + 1
    int km = 0, kj = 0;
    uint32_t ki = 0, kvbase = 0, kdone = 0;
    Unit ku = vu;
    bool kvalid = vvalid;
    uint32_t khead = 0, ktail = 0, kpos = 0;

    auto issue_k = [&](bool block) -> bool {
      if (!kvalid || fail) return false;
      const uint32_t dv = kvbase + (uint32_t)kj + 1u;
      if (dv >= vi) return false;
      const int vslot = (int)(dv % RV);
      if (block) {
        if (!mbar_wait_bounded(&M.vfull[vslot], (dv / RV) & 1u, kWaitNs)) {
          fail = true;
          return false;
        }
      } else if (!mbar_try_wait(&M.vfull[vslot], (dv / RV) & 1u)) {
        return false;
      }
      const PlaneDesc *d = (const PlaneDesc *)(vs + vslot * VSLOT + DOFF);
      const uint32_t cp = min(d->cpad, (uint32_t)NT);
      const uint32_t bytes = cp * (uint32_t)C::EB;
      const uint32_t waste = (kpos + bytes > (uint32_t)C::CB) ? (uint32_t)C::CB - kpos : 0u;
      // retire released blocks until a slot and the space are free
      while (kdone < ki && (ki - kdone >= (uint32_t)NK || (khead - ktail) + waste + bytes > (uint32_t)C::CB)) {
        const int ds = (int)(kdone % NK);
        if (block) {
          if (!mbar_wait_bounded(&M.kempty[ds], (kdone / NK) & 1u, kWaitNs)) {
            fail = true;
            return false;
          }
        } else if (!mbar_try_wait(&M.kempty[ds], (kdone / NK) & 1u)) {
          return false;
        }
        ktail = M.kend[ds];
        ++kdone;
      }
      const int ks = (int)(ki % NK);
      if (waste) {
        khead += waste;
        kpos = 0;
      }
      M.kstart[ks] = kpos;
      khead += bytes;
      M.kend[ks] = khead;
      if (bytes) {
        mbar_expect_tx(&M.kfull[ks], bytes);
        bulk_load(kb + kpos, P.cache + (size_t)d->off * C::EB, bytes, &M.kfull[ks]);
      } else {
        mbar_arrive(&M.kfull[ks]);
      }
      kpos += bytes;
      ++ki;
      if (++kj == ku.nzu) {
        kj = 0;
        kvbase += (uint32_t)ku.nzu + 2u;
        ++km;
        const int u = blockIdx.x + km * G;
        kvalid = u < P.units;
        if (kvalid) ku = unit_at(P, u);
      }
      return true;
    };

    auto issue_v = [&](bool block) -> bool {
      if (!vvalid || fail) return false;
      const int slot = (int)(vi % RV);
      if (vi >= (uint32_t)RV) {
        // the descriptor in the load being replaced must have served its block
        while (kvalid && kvbase + (uint32_t)kj + 1u <= vi - (uint32_t)RV) {
          if (!issue_k(block)) return false;
        }
        if (block) {
          if (!mbar_wait_bounded(&M.vempty[slot], ((vi / RV) - 1u) & 1u, kWaitNs)) {
            fail = true;
            return false;
          }
        } else if (!mbar_try_wait(&M.vempty[slot], ((vi / RV) - 1u) & 1u)) {
          return false;
        }
      }
      const int z = vu.zs - 1 + vj;
      const bool hasd = vj >= 1 && vj <= vu.nzu;
      uint8_t *dst = vs + slot * VSLOT;
      uint64_t *bar = &M.vfull[slot];
      mbar_expect_tx(bar, (uint32_t)VBYTES +
                              (hasd ? (uint32_t)sizeof(PlaneDesc) + (has_x1 ? (uint32_t)(NT * 4) : 0u) : 0u));
      tma_load_3d(dst, &P.tv, vu.x0 - 4, vu.y0 - 1, z, bar);
      if (hasd) {
        bulk_load(dst + DOFF, P.desc + (size_t)vu.t * nz + z, (uint32_t)sizeof(PlaneDesc), bar);
        if (has_x1) tma_load_3d(dst + X1OFF, &P.tx1, vu.x0, vu.y0, z, bar);
      }
      ++vi;
      if (++vj == vu.nzu + 2) {
        vj = 0;
        ++vm;
        const int u = blockIdx.x + vm * G;
        vvalid = u < P.units;
        if (vvalid) vu = unit_at(P, u);
      }
      return true;
    };

    while (!fail && !*sabort && (vvalid || kvalid)) {
      bool prog = false;
      while (issue_v(false)) prog = true;
      while (issue_k(false)) prog = true;
      if (!prog) {
        if (vvalid) (void)issue_v(true);
        else (void)issue_k(true);
      }
    }
    if (fail && P.err) {
      *sabort = 1;
      atomicExch(P.err, 1);
    }
    // every copy must have landed before the CTA may exit
    for (uint32_t i = vi > (uint32_t)RV ? vi - RV : 0u; i < vi; ++i)
      (void)mbar_wait_bounded(&M.vfull[i % RV], (i / RV) & 1u, kWaitNs);
    for (uint32_t i = ki > (uint32_t)NK ? ki - NK : 0u; i < ki; ++i)
      (void)mbar_wait_bounded(&M.kfull[i % NK], (i / NK) & 1u, kWaitNs);
    return;
  }

  // -------------------------------------------------------------------- consumers
  bool ok = true;
  auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
    if (ok && !mbar_wait_bounded(bar, parity, kWaitNs)) {
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
  const uint32_t below = lanemask_lt();
  const int pair = warp >> 1;
  uint32_t vc = 0, kc = 0;  // V loads / K blocks consumed
  uint32_t pround = 0;      // pooling rounds (odd planes) so far
  // pooling of the even row of a pair: the value of round pend_r waits for the odd row's sum
  float psum = 0.f, pend_t = 0.f;
  long long pend_idx = -1;
  bool pend = false;
  uint32_t pend_r = 0;
  auto flush_pool = [&]() {
    if (!pend) return;
    pend = false;
    const int buf = (int)(pend_r & 1u);
    if (!wait(&M.pfull[pair * 2 + buf], (pend_r >> 1) & 1u)) return;
    const float o = M.poolx[pair * 2 + buf][lane >> 1];
    __syncwarp();
    if (lane == 0) mbar_arrive(&M.pempty[pair * 2 + buf]);
    if (pend_idx >= 0) P.pooled[pend_idx] = 0.125f * (pend_t + o);
  };

  for (int m = 0; ok; ++m) {
    const int u = blockIdx.x + m * G;
    if (u >= P.units) break;
    const Unit U = unit_at(P, u);
    const int gx = U.x0 + lane, gy = U.y0 + warp;
    const bool inside = gx < P.dm.nx && gy < P.dm.ny;
    float vA[9], vB[9];
    uint32_t cm = 0u, cf = 0u, ca = 0u, crank = 0u, ccp = 0u;
    float cx1 = 0.f;
    // unit prologue: planes zs-1 and zs, descriptor (and x1) of plane zs
    flush_pool();
    {
      const uint32_t i0 = vc, i1 = vc + 1u;
      if (!wait(&M.vfull[i0 % RV], (i0 / RV) & 1u) || !wait(&M.vfull[i1 % RV], (i1 / RV) & 1u)) break;
      const float *s0 = (const float *)(vs + (i0 % RV) * VSLOT);
      const uint8_t *slot1 = vs + (i1 % RV) * VSLOT;
      const float *s1 = (const float *)slot1;
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const int e = (warp + q / 3) * BXW + lane + 3 + q % 3;
        vA[q] = s0[e];
        vB[q] = s1[e];
      }
      const PlaneDesc *d = (const PlaneDesc *)(slot1 + DOFF);
      cm = d->mixed[warp];
      cf = d->fluid[warp];
      ca = d->air[warp];
      crank = __popc(cm & below);
      for (int q = 0; q < warp; ++q) crank += __popc(d->mixed[q]);
      ccp = min(d->cpad, (uint32_t)NT);
      if (has_x1) cx1 = ((const float *)(slot1 + X1OFF))[warp * TX + lane];
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&M.vempty[i0 % RV]);
        mbar_arrive(&M.vempty[i1 % RV]);
      }
      vc += 2u;
    }

    for (int j = 0; j < U.nzu; ++j) {
      const int z = U.zs + j;
      flush_pool();
      const uint32_t iv = vc, ik = kc;
      if (!wait(&M.vfull[iv % RV], (iv / RV) & 1u)) break;
      const uint8_t *slot = vs + (iv % RV) * VSLOT;
      float vC[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) vC[q] = ((const float *)slot)[(warp + q / 3) * BXW + lane + 3 + q % 3];
      // descriptor and x1 of the next centre plane
      uint32_t nm = 0u, nf = 0u, na = 0u, nrank = 0u, ncp = 0u;
      float nx1 = 0.f;
      if (j + 1 < U.nzu) {
        const PlaneDesc *d = (const PlaneDesc *)(slot + DOFF);
        nm = d->mixed[warp];
        nf = d->fluid[warp];
        na = d->air[warp];
        nrank = __popc(nm & below);
        for (int q = 0; q < warp; ++q) nrank += __popc(d->mixed[q]);
        ncp = min(d->cpad, (uint32_t)NT);
        if (has_x1) nx1 = ((const float *)(slot + X1OFF))[warp * TX + lane];
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&M.vempty[iv % RV]);
      vc += 1u;
      if (!wait(&M.kfull[ik % NK], (ik / NK) & 1u)) break;
      float acc;
      if (cm == 0u && cf == 0xFFFFFFFFu) {
        acc = dot27(P.kF, vA, vB, vC);
      } else if (cm == 0u && ca == 0xFFFFFFFFu) {
        acc = dot27(P.kA, vA, vB, vC);
      } else if ((cm | cf | ca) == 0u) {
        acc = dot27(P.kS, vA, vB, vC);
      } else {
        const float sS = dot27(P.kS, vA, vB, vC), sF = dot27(P.kF, vA, vB, vC), sA = dot27(P.kA, vA, vB, vC);
        acc = ((cf >> lane) & 1u) ? sF : (((ca >> lane) & 1u) ? sA : sS);
        if ((cm >> lane) & 1u) {
          const uint32_t *kw = (const uint32_t *)(kb + M.kstart[ik % NK]) + crank;
          float K[28];
          if (BF16C) {
#pragma unroll
            for (int q = 0; q < 14; ++q) {
              const uint32_t wv = kw[q * ccp];
              K[2 * q] = __uint_as_float(wv << 16);
              K[2 * q + 1] = __uint_as_float(wv & 0xFFFF0000u);
            }
          } else {
#pragma unroll
            for (int a = 0; a < 27; ++a) K[a] = __uint_as_float(kw[a * ccp]);
          }
          float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
          for (int q = 0; q < 9; ++q) {
            s0 = fmaf(K[q], vA[q], s0);
            s1 = fmaf(K[9 + q], vB[q], s1);
            s2 = fmaf(K[18 + q], vC[q], s2);
          }
          acc = (s0 + s1) + s2;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&M.kempty[ik % NK]);
      kc += 1u;
      acc *= sc;
      if (has_x1) acc = fmaf(c1, cx1, c2 * acc);
      if (inside) P.out[(long long)z * nxy + (long long)gy * P.dm.nx + gx] = acc;
      if (P.pooled) {
        if ((z & 1) == 0) {
          psum = acc;
        } else {
          float t = psum + acc;
          t += __shfl_xor_sync(0xffffffffu, t, 1);
          const int buf = (int)(pround & 1u);
          if (warp & 1) {
            // odd row: hand the x/z-pooled sums to the even row of the pair
            if (pround >= 2u && !wait(&M.pempty[pair * 2 + buf], ((pround >> 1) - 1u) & 1u)) break;
            if (!(lane & 1)) M.poolx[pair * 2 + buf][lane >> 1] = t;
            __syncwarp();
            if (lane == 0) mbar_arrive(&M.pfull[pair * 2 + buf]);
          } else {
            pend = true;
            pend_r = pround;
            pend_t = t;
            pend_idx = (inside && !(lane & 1)) ? ((long long)(z >> 1) * cyn + (gy >> 1)) * cxn + (gx >> 1) : -1;
          }
          ++pround;
        }
      }
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        vA[q] = vB[q];
        vB[q] = vC[q];
      }
      cm = nm;
      cf = nf;
      ca = na;
      crank = nrank;
      ccp = ncp;
      cx1 = nx1;
    }
  }
  if (ok) flush_pool();
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
namespace {

int grid_for_units(long long units, int cap) {
  long long g = units < cap ? units : cap;
  return (int)(g < 1 ? 1 : g);
}

template <bool BF16C>
int stream_occupancy() {
  static int occ = 0;
  if (!occ) {
    int o = 0;
    cudaFuncSetAttribute(k_cconv_stream<BF16C>, cudaFuncAttributeMaxDynamicSharedMemorySize, KCfg<BF16C>::SMEM);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_cconv_stream<BF16C>, NTHREADS, KCfg<BF16C>::SMEM);
    occ = o < 1 ? 1 : o;
  }
  return occ;
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

bool encode_map(CUtensorMap *m, const float *base, Dims d, int bw, int bh) {
  const EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz};
  cuuint64_t strides[2] = {(cuuint64_t)d.nx * 4u, (cuuint64_t)d.nx * (cuuint64_t)d.ny * 4u};
  cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1u};
  cuuint32_t es[3] = {1u, 1u, 1u};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)base, dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

bool stream_shape_ok(Dims d) { return d.nx % 4 == 0 && d.nx >= 4; }

long long stream_desc_count(Dims d) {
  const long long ntiles = (long long)((d.nx + TX - 1) / TX) * ((d.ny + TY - 1) / TY);
  return ntiles * d.nz;
}

size_t stream_desc_bytes() { return sizeof(PlaneDesc); }

int cached_entry_bytes(bool bf16) { return bf16 ? KCfg<true>::EB : KCfg<false>::EB; }

void launch_classify(const uint8_t *lab, const ushort2 *counts, Dims d, uint32_t full, void *desc, unsigned *totals,
                     int num_sms, cudaStream_t s) {
  const long long units = (long long)((d.nx + TX - 1) / TX) * ((d.ny + TY - 1) / TY) * ((d.nz + ZCG - 1) / ZCG);
  k_classify<<<grid_for_units(units, num_sms * 8), NT, 0, s>>>(lab, counts, d, full, (PlaneDesc *)desc, totals);
}

void launch_generate(bool bf16, const uint8_t *lab, const ushort2 *counts, Dims d, const CConvW *w, int nblk,
                     const void *desc, void *cache0, void *cache1, int num_sms, cudaStream_t s) {
  const long long units = (long long)((d.nx + TX - 1) / TX) * ((d.ny + TY - 1) / TY) * ((d.nz + ZCG - 1) / ZCG);
  const int g = grid_for_units(units, num_sms * 8);
  if (bf16)
    k_generate<true><<<g, NT, 0, s>>>(lab, counts, d, w, nblk, (const PlaneDesc *)desc, (uint32_t *)cache0,
                                      (uint32_t *)cache1);
  else
    k_generate<false><<<g, NT, 0, s>>>(lab, counts, d, w, nblk, (const PlaneDesc *)desc, (uint32_t *)cache0,
                                       (uint32_t *)cache1);
}

int launch_cconv_stream(bool bf16, Dims dm, const float *kfix, const void *desc, const void *cache, const float *v,
                        const float *vscale, float *out, float *pooled, const float *x1, const double *c12,
                        const SolveState *st, int *err, int num_sms, cudaStream_t s) {
  StreamParams P;
  memset(&P, 0, sizeof(P));
  if (!encode_map(&P.tv, v, dm, BXW, BYH)) return -1;
  if (c12 && !encode_map(&P.tx1, x1, dm, TX, TY)) return -1;
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
  for (int a = 0; a < 27; ++a) {
    P.kS[a] = kfix[a];
    P.kF[a] = kfix[27 + a];
    P.kA[a] = kfix[54 + a];
  }
  const int cap = num_sms * (bf16 ? stream_occupancy<true>() : stream_occupancy<false>());
  // the longest even chunk of planes that still gives every resident CTA a unit
  int zc = 32;
  while (zc > 2 && (long long)P.ntiles * ((dm.nz + zc - 1) / zc) < cap) zc >>= 1;
  P.zc = zc;
  P.units = P.ntiles * ((dm.nz + zc - 1) / zc);
  const int grid = grid_for_units(P.units, cap);
  if (bf16) k_cconv_stream<true><<<grid, NTHREADS, KCfg<true>::SMEM, s>>>(P);
  else k_cconv_stream<false><<<grid, NTHREADS, KCfg<false>::SMEM, s>>>(P);
  return 0;
}

}  // namespace nps
