// Network kernels of Alg. 2 on CUDA cores (FP32): image pyramid, Aff
// reductions, the spatially varying convolution CConv (Sec. 4.2.1), 2x2x2
// average pooling, x2 trilinear interpolation and the per-level combination
// x^l = c1 x1^l + c2 x2^l.  These are the FP32 reference kernels of the
// library; the tensor-core CConv lives in kernels_umma.cu.
#include <cuda_bf16.h>

#include "nps_common.cuh"
#include "nps_kernels.h"

namespace nps {

// ---------------------------------------------------------------------------
// Image pyramid (Alg. 2 "Pooling" of I): exact integer counts of fluid and
// air fine cells per coarse cell.  Level 2 from the labels, level l+1 from
// level l.
// ---------------------------------------------------------------------------
__global__ void k_pyramid_from_labels(const uint8_t *__restrict__ lab, Dims fine, ushort2 *__restrict__ out) {
  const Dims c{fine.nx / 2, fine.ny / 2, fine.nz / 2};
  const long long n = c.n();
  for (long long P = (long long)blockIdx.x * blockDim.x + threadIdx.x; P < n; P += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(P, c, x, y, z);
    unsigned nf = 0, na = 0;
    for (int k = 0; k < 2; ++k)
      for (int j = 0; j < 2; ++j)
        for (int i = 0; i < 2; ++i) {
          const uint8_t l = lab[((long long)(2 * z + k) * fine.ny + (2 * y + j)) * fine.nx + (2 * x + i)];
          nf += l == kFluid;
          na += l == kAir;
        }
    out[P] = make_ushort2((unsigned short)nf, (unsigned short)na);
  }
}

__global__ void k_pyramid_next(const ushort2 *__restrict__ in, Dims fine, ushort2 *__restrict__ out) {
  const Dims c{fine.nx / 2, fine.ny / 2, fine.nz / 2};
  const long long n = c.n();
  for (long long P = (long long)blockIdx.x * blockDim.x + threadIdx.x; P < n; P += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(P, c, x, y, z);
    unsigned nf = 0, na = 0;
    for (int k = 0; k < 2; ++k)
      for (int j = 0; j < 2; ++j)
        for (int i = 0; i < 2; ++i) {
          const ushort2 v = in[((long long)(2 * z + k) * fine.ny + (2 * y + j)) * fine.nx + (2 * x + i)];
          nf += v.x;
          na += v.y;
        }
    out[P] = make_ushort2((unsigned short)nf, (unsigned short)na);
  }
}

// Image feature pair (fluid count, air count) at (x,y,z) of a level; zero
// outside the grid (solid padding).  Level 1 reads labels, levels >= 2 counts.
struct ImgSrc {
  const uint8_t *lab;     // level 1
  const ushort2 *counts;  // level >= 2
};

__device__ __forceinline__ float2 img_at(const ImgSrc &im, const Dims &dm, int x, int y, int z) {
  if (x < 0 || y < 0 || z < 0 || x >= dm.nx || y >= dm.ny || z >= dm.nz) return make_float2(0.f, 0.f);
  const long long p = ((long long)z * dm.ny + y) * dm.nx + x;
  if (im.lab) {
    const uint8_t l = im.lab[p];
    return make_float2(l == kFluid ? 1.f : 0.f, l == kAir ? 1.f : 0.f);
  }
  const ushort2 c = im.counts[p];
  return make_float2((float)c.x, (float)c.y);
}

// ---------------------------------------------------------------------------
// Aff (Sec. 4.2.1) through exact window sums.  The image outside the grid is
// solid, I = (0, 0, 1), so for the fluid and air channels
//   sum_p I_c(p + l) = sum of I_c(q) over the cells q of the grid with q - l
//                      also inside, i.e. all cells except the face plane that
//                      the offset l pushes out of the grid.
// The whole reduction therefore needs, per channel, the counts over the 4x4x4
// boundary classes of a cell (per axis: interior, first plane, last plane,
// both when the axis has one plane); the 27 window sums follow by inclusion.
// The counts are exact integers, so their summation order does not matter;
// the final 27-term sums are FP64.  The solid channel is folded into the
// weights (AffW).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int edge_class(int q, int n) { return (q == 0 ? 1 : 0) | (q == n - 1 ? 2 : 0); }

// A cell of boundary class c (bit 0: first plane, bit 1: last plane) along an
// axis stays inside the window sum of offset o unless o pushes it out.
__device__ __forceinline__ bool keeps(int c, int o) { return !((o == 1 && (c & 1)) || (o == -1 && (c & 2))); }

// The Aff blocks of every level (1..L-1) in two launches.  k_aff_counts_all:
// the boundary-class counts of all levels (blockIdx.y = level - 1; a warp per
// grid row, level 1 reading four labels per lane), interior cells summed per
// thread, the other 63 classes in shared memory, one global atomic per class.
// k_aff_from_counts_all: one block of 128 threads per level loads the 128
// counters, 27 threads form the window sums of their offsets (exact: integer
// counts below 2^53) and the weighted FP64 terms, thread 0 sums them in a fixed
// order into c1, c2; optionally the 54 window sums scaled by 1 / (8^(l-1) 27 n)
// (fluid [0, 27), air [27, 54)) for the training backward's Aff gradient.
__device__ __forceinline__ void aff_count_cell(uint32_t f, uint32_t a, int cls, unsigned long long &inf,
                                               unsigned long long &ina, unsigned long long *sc) {
  if (cls == 0) {
    inf += f;
    ina += a;
  } else {
    if (f) atomicAdd(&sc[2 * cls], (unsigned long long)f);
    if (a) atomicAdd(&sc[2 * cls + 1], (unsigned long long)a);
  }
}

__global__ void __launch_bounds__(256) k_aff_counts_all(const __grid_constant__ AffAll A) {
  __shared__ unsigned long long sc[128];
  const int lvl = blockIdx.y + 1;
  const Dims dm = A.dims[lvl];
  for (int i = threadIdx.x; i < 128; i += blockDim.x) sc[i] = 0ull;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long long rows = (long long)dm.ny * dm.nz;
  unsigned long long inf = 0ull, ina = 0ull;
  const bool vec = lvl == 1 && (dm.nx & 3) == 0;
  for (long long r = (long long)blockIdx.x * nw + warp; r < rows; r += (long long)gridDim.x * nw) {
    const int y = (int)(r % dm.ny), z = (int)(r / dm.ny);
    const int cyz = 4 * edge_class(y, dm.ny) + 16 * edge_class(z, dm.nz);
    const long long base = r * dm.nx;
    if (vec) {
      for (int x4 = lane; x4 < (dm.nx >> 2); x4 += 32) {
        const uchar4 l4 = *reinterpret_cast<const uchar4 *>(A.lab + base + 4 * x4);
        const uint8_t ls[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
          aff_count_cell(ls[e] == kFluid, ls[e] == kAir, cyz + edge_class(4 * x4 + e, dm.nx), inf, ina, sc);
      }
    } else {
      for (int x = lane; x < dm.nx; x += 32) {
        uint32_t f, a;
        if (lvl == 1) {
          const uint8_t l = A.lab[base + x];
          f = l == kFluid;
          a = l == kAir;
        } else {
          const ushort2 c = A.counts[lvl][base + x];
          f = c.x;
          a = c.y;
        }
        aff_count_cell(f, a, cyz + edge_class(x, dm.nx), inf, ina, sc);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    inf += __shfl_down_sync(0xffffffffu, inf, o);
    ina += __shfl_down_sync(0xffffffffu, ina, o);
  }
  if (lane == 0) {
    atomicAdd(&sc[0], inf);
    atomicAdd(&sc[1], ina);
  }
  __syncthreads();
  unsigned long long *cnt = A.cnt + 128 * lvl;
  for (int i = threadIdx.x; i < 128; i += blockDim.x)
    if (sc[i]) atomicAdd(&cnt[i], sc[i]);
}

__global__ void k_aff_from_counts_all(const __grid_constant__ AffAll A) {
  const int lvl = blockIdx.x + 1;
  __shared__ unsigned long long cnt[128];
  __shared__ double t1[27], t2[27];
  const AffW *a1 = A.aw + 2 * lvl, *a2 = A.aw + 2 * lvl + 1;
  const long long n = A.dims[lvl].n();
  double *stats = A.stats ? A.stats + 54 * lvl : nullptr;
  const double stat_scale = ldexp(1.0, -3 * (lvl - 1)) / (27.0 * (double)n);  // 1 / (8^(lvl-1) 27 n)
  const int l = threadIdx.x;
  cnt[l] = A.cnt[128 * lvl + l];
  __syncthreads();
  if (l < 27) {
    const int ox = l % 3 - 1, oy = (l / 3) % 3 - 1, oz = l / 9 - 1;
    double sf = 0.0, sa = 0.0;  // exact: integer counts below 2^53
    for (int c = 0; c < 64; ++c) {
      if (!(keeps(c & 3, ox) && keeps((c >> 2) & 3, oy) && keeps(c >> 4, oz))) continue;
      sf += (double)cnt[2 * c];
      sa += (double)cnt[2 * c + 1];
    }
    t1[l] = (double)a1->wf[l] * sf + (double)a1->wa[l] * sa;
    t2[l] = (double)a2->wf[l] * sf + (double)a2->wa[l] * sa;
    if (stats) {
      stats[l] = sf * stat_scale;
      stats[27 + l] = sa * stat_scale;
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double s1 = 0.0, s2 = 0.0;
  for (int i = 0; i < 27; ++i) {
    s1 += t1[i];
    s2 += t2[i];
  }
  A.out[2 * lvl] = a1->bconst + s1 / (27.0 * (double)n);
  A.out[2 * lvl + 1] = a2->bconst + s2 / (27.0 * (double)n);
}

void launch_aff_all(const AffAll &A, cudaStream_t s) {
  if (A.L < 2) return;
  cudaMemsetAsync(A.cnt, 0, sizeof(unsigned long long) * 128 * A.L, s);
  const long long rows = (long long)A.dims[1].ny * A.dims[1].nz;
  long long g = (rows + 7) / 8;
  if (g > 148LL * 8) g = 148LL * 8;
  k_aff_counts_all<<<dim3((unsigned)(g < 1 ? 1 : g), (unsigned)(A.L - 1)), 256, 0, s>>>(A);
  k_aff_from_counts_all<<<A.L - 1, 128, 0, s>>>(A);
}

// ---------------------------------------------------------------------------
// CConv on CUDA cores (FP32):
//   K_a(p) = bp[a] + sum_l (wf[a][l] nF(p+l) + wa[a][l] nA(p+l))
//   out_p  = sum_a K_a(p) v(p+a) * vscale,  v zero outside the grid.
// When mask_input is set (level-1 CConv1), v is also zeroed off fluid (the
// reduced input vector padded with zeros, Sec. 4.2).  round_k = 0: FP32
// kernels; nonzero: the BF16 form (kernel values rounded to BF16).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_cconv_f32(ImgSrc im, Dims dm, const CConvW *__restrict__ w,
                                                     const float *__restrict__ v, const float *__restrict__ vscale,
                                                     int mask_input, int round_k, float *__restrict__ out,
                                                     const SolveState *st) {
  if (st && st->done) return;
  __shared__ CConvW sw;
  {
    const float *src = (const float *)w;
    float *dst = (float *)&sw;
    for (int i = threadIdx.x; i < (int)(sizeof(CConvW) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const float sc = vscale ? *vscale : 1.f;
  const long long n = dm.n();
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(p, dm, x, y, z);
    float nf[27], na[27], vv[27];
#pragma unroll
    for (int t = 0; t < 27; ++t) {
      const int xx = x + t % 3 - 1, yy = y + (t / 3) % 3 - 1, zz = z + t / 9 - 1;
      const float2 f = img_at(im, dm, xx, yy, zz);
      nf[t] = f.x;
      na[t] = f.y;
      float val = 0.f;
      if (xx >= 0 && yy >= 0 && zz >= 0 && xx < dm.nx && yy < dm.ny && zz < dm.nz) {
        val = v[((long long)zz * dm.ny + yy) * dm.nx + xx];
        if (mask_input && f.x == 0.f) val = 0.f;  // level 1: f.x == 1 exactly on fluid
      }
      vv[t] = val * sc;
    }
    // BF16 form: every per-cell kernel value is rounded to BF16 (nearest even)
    const bool rk = round_k != 0;
    float acc = 0.f;
#pragma unroll 1
    for (int a = 0; a < 27; ++a) {
      float k = sw.bp[a];
#pragma unroll
      for (int l = 0; l < 27; ++l) k = fmaf(sw.wf[a][l], nf[l], fmaf(sw.wa[a][l], na[l], k));
      if (rk) k = __bfloat162float(__float2bfloat16_rn(k));
      acc = fmaf(k, vv[a], acc);
    }
    out[p] = acc;
  }
}

// out = in on fluid cells, 0 elsewhere (the reduced vector padded with zeros).
__global__ void k_mask_copy(const uint8_t *__restrict__ lab, long long n, const float *__restrict__ in,
                            float *__restrict__ out) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
    out[p] = lab[p] == kFluid ? in[p] : 0.f;
}

// 2x2x2 average pooling of a vector: out[P] = mean of its 8 children.
__global__ void k_pool(const float *__restrict__ in, Dims fine, float *__restrict__ out, const SolveState *st) {
  if (st && st->done) return;
  const Dims c{fine.nx / 2, fine.ny / 2, fine.nz / 2};
  const long long n = c.n();
  for (long long P = (long long)blockIdx.x * blockDim.x + threadIdx.x; P < n; P += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(P, c, x, y, z);
    float s = 0.f;
    for (int k = 0; k < 2; ++k)
      for (int j = 0; j < 2; ++j)
        for (int i = 0; i < 2; ++i) s += in[((long long)(2 * z + k) * fine.ny + (2 * y + j)) * fine.nx + (2 * x + i)];
    out[P] = 0.125f * s;
  }
}

// One axis of x2 linear upsampling with half-pixel centres and edge clamp:
// even f = 2j: 0.25 c[j-1] + 0.75 c[j] (c[0] at j = 0);
// odd  f = 2j+1: 0.75 c[j] + 0.25 c[j+1] (c[n-1] at j = n-1).
__device__ __forceinline__ void up_taps(int f, int nc, int &i0, int &i1, float &w1) {
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

__global__ void k_interp(const float *__restrict__ in, Dims coarse, float *__restrict__ out, const SolveState *st) {
  if (st && st->done) return;
  const Dims f{coarse.nx * 2, coarse.ny * 2, coarse.nz * 2};
  const long long n = f.n();
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(p, f, x, y, z);
    int x0, x1, y0, y1, z0, z1;
    float wx, wy, wz;
    up_taps(x, coarse.nx, x0, x1, wx);
    up_taps(y, coarse.ny, y0, y1, wy);
    up_taps(z, coarse.nz, z0, z1, wz);
    auto C = [&](int zz, int yy, int xx) { return in[((long long)zz * coarse.ny + yy) * coarse.nx + xx]; };
    const float c00 = (1.f - wx) * C(z0, y0, x0) + wx * C(z0, y0, x1);
    const float c01 = (1.f - wx) * C(z0, y1, x0) + wx * C(z0, y1, x1);
    const float c10 = (1.f - wx) * C(z1, y0, x0) + wx * C(z1, y0, x1);
    const float c11 = (1.f - wx) * C(z1, y1, x0) + wx * C(z1, y1, x1);
    const float c0 = (1.f - wy) * c00 + wy * c01;
    const float c1 = (1.f - wy) * c10 + wy * c11;
    out[p] = (1.f - wz) * c0 + wz * c1;
  }
}

// The same interpolation for grids whose coarse dims are all even... and any
// nz: each thread produces a 4 (x) x 2 (y) x 2 (z) block of fine cells from
// the 3 x 3 coarse rows around it, sharing the x- and then y-interpolated
// values between the fine rows and planes of the block (about 12 operations
// per fine cell), and writes four 16-byte rows.  Per axis, fine 2j uses
// 0.25 c[j-1] + 0.75 c[j] (c[0] at j = 0) and fine 2j+1 uses
// 0.75 c[j] + 0.25 c[j+1] (c[n-1] at the end), as in k_interp.

// skip (optional): one byte per (32 x 8 fine tile, fine plane), tile-major;
// blocks whose two planes are both marked non-zero are not written (no later read).
//
// Each thread marches along z over zc coarse planes: it keeps the x- and
// y-interpolated values of the coarse planes kz-1, kz, kz+1 (4 fine columns x
// 2 fine rows each) and loads one new plane's three coarse rows per step, so
// the loads and the x/y interpolation are shared by the two fine planes of a
// coarse plane and by the neighbouring coarse planes.  The arithmetic per
// output does not depend on zc (same operands, same order).  zc = 4 on grids
// with threads to spare (at least 2^19 of one block each), else 1.
constexpr int kInterpZC = 4;

__device__ __forceinline__ void interp_xy(const float *__restrict__ in, int cx, int cy, int q, int jy, int zc,
                                          float (&yl)[2][4]) {
  const int xm = max(2 * q - 1, 0), x0 = 2 * q, xp = min(2 * q + 2, cx - 1);  // x0, x0 + 1 by one 8-byte load
  const int ys[3] = {max(jy - 1, 0), jy, min(jy + 1, cy - 1)};
  float xl[3][4];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const float *row = in + ((long long)zc * cy + ys[b]) * cx;
    const float2 v01 = __ldg(reinterpret_cast<const float2 *>(row + x0));
    const float vm = __ldg(row + xm), vp = __ldg(row + xp);
    xl[b][0] = q > 0 ? lerp_lo(vm, v01.x) : v01.x;
    xl[b][1] = lerp_hi(v01.x, v01.y);
    xl[b][2] = lerp_lo(v01.x, v01.y);
    xl[b][3] = lerp_hi(v01.y, vp);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    yl[0][i] = jy > 0 ? lerp_lo(xl[0][i], xl[1][i]) : xl[1][i];
    yl[1][i] = lerp_hi(xl[1][i], xl[2][i]);
  }
}

__global__ void __launch_bounds__(256) k_interp_blk(const float *__restrict__ in, Dims coarse, float *__restrict__ out,
                                                    const uint8_t *__restrict__ skip, int zc, const SolveState *st) {
  if (st && st->done) return;
  const int cx = coarse.nx, cy = coarse.ny, cz = coarse.nz;
  const int fx = 2 * cx, fy = 2 * cy, fz = 2 * cz;
  const int nq = fx >> 2;  // x groups of 4 fine cells (cx / 2)
  const int nzc = (cz + zc - 1) / zc;
  const long long nthr = (long long)nq * cy * nzc;
  const long long fxy = (long long)fx * fy;
  // 32-bit index arithmetic (a fine grid below 2^31 cells has nthr < 2^27)
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < (unsigned)nthr; t += gridDim.x * blockDim.x) {
    const int q = (int)(t % (unsigned)nq);
    const unsigned r = t / (unsigned)nq;
    const int jy = (int)(r % (unsigned)cy), kc = (int)(r / (unsigned)cy);  // fine rows 2jy, 2jy+1
    const int k0 = kc * zc, k1 = min(k0 + zc, cz);
    const uint8_t *sk = nullptr;
    if (skip) {
      sk = skip + ((size_t)((4 * q) / 32) + (size_t)((2 * jy) / 8) * (size_t)((fx + 31) / 32)) * fz;
      bool all = true;
      for (int kz = k0; kz < k1; ++kz) all = all && sk[2 * kz] && sk[2 * kz + 1];
      if (all) continue;
    }
    float ym[2][4], yc[2][4], yp[2][4];  // coarse planes kz-1, kz, kz+1 (clamped)
    interp_xy(in, cx, cy, q, jy, max(k0 - 1, 0), ym);
    interp_xy(in, cx, cy, q, jy, k0, yc);
    for (int kz = k0; kz < k1; ++kz) {
      interp_xy(in, cx, cy, q, jy, min(kz + 1, cz - 1), yp);
      if (!sk || !(sk[2 * kz] && sk[2 * kz + 1])) {
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
          for (int dy = 0; dy < 2; ++dy) {
            float o[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
              o[i] = dz == 0 ? (kz > 0 ? lerp_lo(ym[dy][i], yc[dy][i]) : yc[dy][i]) : lerp_hi(yc[dy][i], yp[dy][i]);
            const long long p = (long long)(2 * kz + dz) * fxy + (long long)(2 * jy + dy) * fx + 4 * q;
            *reinterpret_cast<float4 *>(out + p) = make_float4(o[0], o[1], o[2], o[3]);
          }
      }
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          ym[dy][i] = yc[dy][i];
          yc[dy][i] = yp[dy][i];
        }
    }
  }
}

// x^l = c1 x1 + c2 x2 (levels >= 2, no masking).
__global__ void k_combine(long long n, const float *__restrict__ x1, const float *__restrict__ x2,
                          const double *__restrict__ c12, float *__restrict__ out, const SolveState *st) {
  if (st && st->done) return;
  const float c1 = (float)c12[0], c2 = (float)c12[1];
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
    out[p] = fmaf(c1, x1[p], c2 * x2[p]);
}

// Level 1: z = mask_fluid(c1 x1 + c2 x2) (the output restriction of Sec.
// 4.2) and, inside a solve, the partial dot products z.(A d_i) for the
// previous directions i = k-1, k-2, ... (Alg. 1 orthogonalisation), or for
// PCG / FPCG z.r_k and z.(A d_k).
__global__ void __launch_bounds__(kRedThreads) k_combine1(const uint8_t *__restrict__ lab, long long n,
                                                            const float *__restrict__ x1, const float *__restrict__ x2,
                                                            const double *__restrict__ c12, float *__restrict__ z,
                                                            const float *__restrict__ qring, const float *rk,
                                                            double *__restrict__ part, const SolveState *st) {
  if (st && st->done) return;
  const float c1 = (float)c12[0], c2 = (float)c12[1];
  const float *qs[kMaxOrtho];
  int cnt = 0;
  if (st) {
    const int k1 = st->k + 1, no = st->n_ortho;
    if (st->method == kMethodNpsdo) {
      for (int i = k1 - 1; i >= k1 - no && i >= 1; --i) qs[cnt++] = qring + (size_t)ring_slot(i, no) * n;
    } else {
      cnt = direction_dot_count(st->method, k1, no, kMaxOrtho);
      qs[0] = rk;
      qs[1] = qring + (size_t)ring_slot(k1 > 1 ? k1 - 1 : 1, no) * n;
    }
  }
  double v[kMaxOrtho] = {0.0, 0.0, 0.0, 0.0};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    const float val = lab[p] == kFluid ? fmaf(c1, x1[p], c2 * x2[p]) : 0.f;
    z[p] = val;
    for (int j = 0; j < cnt; ++j) v[j] += (double)val * (double)qs[j][p];
  }
  if (st) block_sum_store<kMaxOrtho>(v, part + (size_t)blockIdx.x * kMaxOrtho);
}

// ---------------------------------------------------------------------------
// Host-side launchers.
// ---------------------------------------------------------------------------
static inline int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 148LL * 16) b = 148LL * 16;
  return (int)(b < 1 ? 1 : b);
}

void launch_pyramid(const uint8_t *lab, Dims d1, ushort2 *const *counts, int L, cudaStream_t s) {
  Dims d = d1;
  for (int l = 2; l <= L; ++l) {
    const long long nc = (long long)(d.nx / 2) * (d.ny / 2) * (d.nz / 2);
    if (l == 2) k_pyramid_from_labels<<<grid_for(nc, 256), 256, 0, s>>>(lab, d, counts[2]);
    else k_pyramid_next<<<grid_for(nc, 256), 256, 0, s>>>(counts[l - 1], d, counts[l]);
    d = Dims{d.nx / 2, d.ny / 2, d.nz / 2};
  }
}

void launch_cconv_f32(const uint8_t *lab, const ushort2 *counts, Dims dm, const CConvW *w, const float *v,
                      const float *vscale, int mask_input, int round_k, float *out, const SolveState *st,
                      cudaStream_t s) {
  ImgSrc im{lab, counts};
  if (counts) im.lab = nullptr;
  k_cconv_f32<<<grid_for(dm.n(), 128), 128, 0, s>>>(im, dm, w, v, vscale, mask_input, round_k, out, st);
}

void launch_mask_copy(const uint8_t *lab, long long n, const float *in, float *out, cudaStream_t s) {
  k_mask_copy<<<grid_for(n, 256), 256, 0, s>>>(lab, n, in, out);
}

void launch_pool(const float *in, Dims fine, float *out, const SolveState *st, cudaStream_t s) {
  const long long nc = (long long)(fine.nx / 2) * (fine.ny / 2) * (fine.nz / 2);
  k_pool<<<grid_for(nc, 256), 256, 0, s>>>(in, fine, out, st);
}

void launch_interp(const float *in, Dims coarse, float *out, const SolveState *st, cudaStream_t s,
                   const uint8_t *skip) {
  if (coarse.nx % 2 == 0) {  // fine rows of a multiple of 4 cells: 16-byte stores
    const long long blocks = (long long)(coarse.nx / 2) * coarse.ny * coarse.nz;
    const int zc = blocks >= (1LL << 19) ? kInterpZC : 1;
    const long long nthr = (long long)(coarse.nx / 2) * coarse.ny * ((coarse.nz + zc - 1) / zc);
    k_interp_blk<<<grid_for(nthr, 256), 256, 0, s>>>(in, coarse, out, skip, zc, st);
    return;
  }
  k_interp<<<grid_for(coarse.n() * 8, 256), 256, 0, s>>>(in, coarse, out, st);
}

void launch_combine(long long n, const float *x1, const float *x2, const double *c12, float *out,
                    const SolveState *st, cudaStream_t s) {
  k_combine<<<grid_for(n, 256), 256, 0, s>>>(n, x1, x2, c12, out, st);
}

void launch_combine1(const uint8_t *lab, long long n, const float *x1, const float *x2, const double *c12, float *z,
                     const float *qring, const float *rk, double *part, const SolveState *st, cudaStream_t s) {
  k_combine1<<<red_blocks(n), kRedThreads, 0, s>>>(lab, n, x1, x2, c12, z, qring, rk, part, st);
}

}  // namespace nps
