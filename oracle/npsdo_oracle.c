/*
 * npsdo_oracle.c -- plain FP64 CPU oracle for the neural-preconditioned
 * Poisson solve of arXiv 2310.00177 ("A Neural-Preconditioned Poisson Solver
 * for Mixed Dirichlet and Neumann Boundary Conditions").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, literal reference that the
 * CUDA path is compared against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or helper with the CUDA library.
 *
 * Everything is double precision and follows the paper's formulas in the
 * paper's order, without blocking, fusion or algebraic rewriting:
 *   - masked 7-point Laplacian              (Sec. 3.1-3.2)
 *   - image pyramid, CConv, Aff, pooling,
 *     interpolation, network forward        (Sec. 4.2, Algorithm 2)
 *   - network backward (reverse of Alg. 2)  (Sec. 4.2.3, training loss)
 *   - NPSDO solver                          (Sec. 4.1, Algorithm 1)
 *   - PCG / flexible PCG with the network   (Sec. 4.1, appendix: solver
 *     as preconditioner                      variant comparison)
 *   - Jacobi-preconditioned CG              (textbook PCG, Sec. 4.1)
 *
 * Conventions (the readings where the paper is silent):
 *   grid index       p = (z*ny + y)*nx + x, x fastest
 *   label codes      0 = solid, 1 = fluid, 2 = air   (cells outside the grid
 *                    are solid, Sec. 3.1)
 *   image channels   c = 0 fluid, 1 air, 2 solid     (Sec. 3.2 three-channel
 *                    indicator image; channels sum to one)
 *   3x3x3 offsets    t = 9*(dz+1) + 3*(dy+1) + (dx+1), dz,dy,dx in {-1,0,1}
 *                    (the 3D extension of the "3a+b" tap index of Sec. 4.2.1)
 *   CConv weights    W[t_a][c][t_l] (27 x 3 x 27), bias B[t_a] (27)
 *   Aff weights      Wbar[c][t_l] (3 x 27), bias Bbar (1)
 *   weight blob      for level l = 1..L-1: CConv1 (W,B), CConv2 (W,B),
 *                    Aff1 (Wbar,Bbar), Aff2 (Wbar,Bbar); then level L: CConv1.
 *
 * Parity pins for every function here live in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define LAB_SOLID 0
#define LAB_FLUID 1
#define LAB_AIR 2

#define CCONV_PARAMS (27 * 3 * 27 + 27) /* 2214 */
#define AFF_PARAMS (3 * 27 + 1)         /* 82 */

/* Status codes shared in meaning (not in code) with the CUDA library. */
#define OR_OK 0
#define OR_BAD_ARG 1
#define OR_BAD_DIMS 2
#define OR_BAD_LABELS 3
#define OR_NO_CONVERGENCE 4
#define OR_BREAKDOWN 5

static size_t cells(int nx, int ny, int nz) { return (size_t)nx * ny * nz; }

static int inside(int nx, int ny, int nz, int x, int y, int z) {
  return x >= 0 && y >= 0 && z >= 0 && x < nx && y < ny && z < nz;
}

/* Label lookup; the region outside the grid is solid (Sec. 3.1). */
static int label_at(const uint8_t *lab, int nx, int ny, int nz, int x, int y, int z) {
  if (!inside(nx, ny, nz, x, y, z)) return LAB_SOLID;
  return lab[((size_t)z * ny + y) * nx + x];
}

/* Validate labels; returns OR_BAD_LABELS on a code outside {0,1,2}. */
int or_check_labels(const uint8_t *lab, int nx, int ny, int nz) {
  size_t n = cells(nx, ny, nz);
  for (size_t p = 0; p < n; ++p)
    if (lab[p] > 2) return OR_BAD_LABELS;
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2: the masked 7-point Laplacian A.  For a fluid cell, stencil points
 * outside the fluid are dropped and the diagonal is the number of neighbours
 * that are fluid or air; rows and columns of non-fluid cells are empty.       */
/* ------------------------------------------------------------------------ */
void or_lap_apply(const uint8_t *lab, int nx, int ny, int nz, const double *d, double *q) {
  static const int off[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        size_t p = ((size_t)z * ny + y) * nx + x;
        if (lab[p] != LAB_FLUID) {
          q[p] = 0.0;
          continue;
        }
        double diag = 0.0, offsum = 0.0;
        for (int k = 0; k < 6; ++k) {
          int xx = x + off[k][0], yy = y + off[k][1], zz = z + off[k][2];
          int ln = label_at(lab, nx, ny, nz, xx, yy, zz);
          if (ln == LAB_FLUID) {
            diag += 1.0;
            offsum += d[((size_t)zz * ny + yy) * nx + xx];
          } else if (ln == LAB_AIR) {
            diag += 1.0;
          }
        }
        q[p] = diag * d[p] - offsum;
      }
}

/* Diagonal of A (number of fluid-or-air neighbours on fluid cells, 0 else). */
void or_lap_diag(const uint8_t *lab, int nx, int ny, int nz, double *diag) {
  static const int off[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        size_t p = ((size_t)z * ny + y) * nx + x;
        double dg = 0.0;
        if (lab[p] == LAB_FLUID)
          for (int k = 0; k < 6; ++k) {
            int ln = label_at(lab, nx, ny, nz, x + off[k][0], y + off[k][1], z + off[k][2]);
            if (ln == LAB_FLUID || ln == LAB_AIR) dg += 1.0;
          }
        diag[p] = dg;
      }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2 / Alg. 2: the three-channel image and its pyramid.                */
/* ------------------------------------------------------------------------ */

/* Level-1 image: one-hot of the label, channel-major I[c*n + p]. */
void or_image_from_labels(const uint8_t *lab, int nx, int ny, int nz, double *img) {
  size_t n = cells(nx, ny, nz);
  for (size_t p = 0; p < n; ++p) {
    img[0 * n + p] = lab[p] == LAB_FLUID ? 1.0 : 0.0;
    img[1 * n + p] = lab[p] == LAB_AIR ? 1.0 : 0.0;
    img[2 * n + p] = lab[p] == LAB_SOLID ? 1.0 : 0.0;
  }
}

/* Alg. 2 "Pooling": 2x2x2 average pooling of a multi-channel field of fine
 * dims (nx,ny,nz) (all even) into coarse dims (nx/2,ny/2,nz/2). */
void or_avgpool2(const double *in, int nch, int nx, int ny, int nz, double *out) {
  int cx = nx / 2, cy = ny / 2, cz = nz / 2;
  size_t nf = cells(nx, ny, nz), ncc = cells(cx, cy, cz);
  for (int c = 0; c < nch; ++c)
    for (int z = 0; z < cz; ++z)
      for (int y = 0; y < cy; ++y)
        for (int x = 0; x < cx; ++x) {
          double s = 0.0;
          for (int k = 0; k < 2; ++k)
            for (int j = 0; j < 2; ++j)
              for (int i = 0; i < 2; ++i)
                s += in[c * nf + ((size_t)(2 * z + k) * ny + (2 * y + j)) * nx + (2 * x + i)];
          out[c * ncc + ((size_t)z * cy + y) * cx + x] = s / 8.0;
        }
}

/* Adjoint of or_avgpool2 for one channel: each fine cell receives 1/8 of its
 * parent's value. */
void or_avgpool2_adjoint(const double *gc, int nx, int ny, int nz, double *gf) {
  int cx = nx / 2, cy = ny / 2;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x)
        gf[((size_t)z * ny + y) * nx + x] = gc[((size_t)(z / 2) * cy + y / 2) * cx + x / 2] / 8.0;
}

/* One axis of the x2 linear upsampling with half-pixel centres and edge clamp:
 * source coordinate s = (f + 0.5)/2 - 0.5 clamped below at 0, taps i0 = floor(s),
 * i1 = min(i0 + 1, n - 1), weights (1 - lam, lam).  This is the 3D reading of
 * the "bilinear interpolation" of Alg. 2. */
static void interp_taps(int f, int n, int *i0, int *i1, double *lam) {
  double s = (f + 0.5) / 2.0 - 0.5;
  if (s < 0.0) s = 0.0;
  int a = (int)floor(s);
  if (a > n - 1) a = n - 1;
  *i0 = a;
  *i1 = a + 1 < n ? a + 1 : n - 1;
  *lam = s - a;
}

/* Alg. 2 "Interpolation": trilinear x2 upsampling of a coarse field of dims
 * (cx,cy,cz) to the fine field (2cx,2cy,2cz). */
void or_interp_up2(const double *coarse, int cx, int cy, int cz, double *fine) {
  int fx = 2 * cx, fy = 2 * cy, fz = 2 * cz;
  for (int z = 0; z < fz; ++z) {
    int z0, z1;
    double lz;
    interp_taps(z, cz, &z0, &z1, &lz);
    for (int y = 0; y < fy; ++y) {
      int y0, y1;
      double ly;
      interp_taps(y, cy, &y0, &y1, &ly);
      for (int x = 0; x < fx; ++x) {
        int x0, x1;
        double lx;
        interp_taps(x, cx, &x0, &x1, &lx);
        int zs[2] = {z0, z1}, ys[2] = {y0, y1}, xs[2] = {x0, x1};
        double wz[2] = {1.0 - lz, lz}, wy[2] = {1.0 - ly, ly}, wx[2] = {1.0 - lx, lx};
        double s = 0.0;
        for (int k = 0; k < 2; ++k)
          for (int j = 0; j < 2; ++j)
            for (int i = 0; i < 2; ++i)
              s += wz[k] * wy[j] * wx[i] * coarse[((size_t)zs[k] * cy + ys[j]) * cx + xs[i]];
        fine[((size_t)z * fy + y) * fx + x] = s;
      }
    }
  }
}

/* Adjoint of or_interp_up2: scatter each fine value back with the same
 * weights. */
void or_interp_up2_adjoint(const double *gfine, int cx, int cy, int cz, double *gcoarse) {
  int fx = 2 * cx, fy = 2 * cy, fz = 2 * cz;
  memset(gcoarse, 0, sizeof(double) * cells(cx, cy, cz));
  for (int z = 0; z < fz; ++z) {
    int z0, z1;
    double lz;
    interp_taps(z, cz, &z0, &z1, &lz);
    for (int y = 0; y < fy; ++y) {
      int y0, y1;
      double ly;
      interp_taps(y, cy, &y0, &y1, &ly);
      for (int x = 0; x < fx; ++x) {
        int x0, x1;
        double lx;
        interp_taps(x, cx, &x0, &x1, &lx);
        int zs[2] = {z0, z1}, ys[2] = {y0, y1}, xs[2] = {x0, x1};
        double wz[2] = {1.0 - lz, lz}, wy[2] = {1.0 - ly, ly}, wx[2] = {1.0 - lx, lx};
        double g = gfine[((size_t)z * fy + y) * fx + x];
        for (int k = 0; k < 2; ++k)
          for (int j = 0; j < 2; ++j)
            for (int i = 0; i < 2; ++i)
              gcoarse[((size_t)zs[k] * cy + ys[j]) * cx + xs[i]] += wz[k] * wy[j] * wx[i] * g;
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.2.1: the custom convolution block CConv.                           */
/* ------------------------------------------------------------------------ */

/* Image value with the paper's padding rule: outside the grid the image is a
 * solid pixel, i.e. channel values (fluid, air, solid) = (0, 0, 1). */
static double image_at(const double *img, int c, int nx, int ny, int nz, int x, int y, int z) {
  if (!inside(nx, ny, nz, x, y, z)) return c == 2 ? 1.0 : 0.0;
  return img[(size_t)c * cells(nx, ny, nz) + ((size_t)z * ny + y) * nx + x];
}

/* Vector value with zero padding outside the grid. */
static double vec_at(const double *v, int nx, int ny, int nz, int x, int y, int z) {
  if (!inside(nx, ny, nz, x, y, z)) return 0.0;
  return v[((size_t)z * ny + y) * nx + x];
}

/* The per-cell kernel of CConv at cell (x,y,z):
 *   K_a = B_a + sum_c sum_l W[a][c][l] * I_c(p + l). */
static void cconv_kernel_at(const double *img, int nx, int ny, int nz, const double *W, const double *B, int x,
                            int y, int z, double K[27]) {
  double feat[3][27];
  for (int c = 0; c < 3; ++c)
    for (int l = 0; l < 27; ++l)
      feat[c][l] = image_at(img, c, nx, ny, nz, x + (l % 3) - 1, y + (l / 3) % 3 - 1, z + l / 9 - 1);
  for (int a = 0; a < 27; ++a) {
    double k = B[a];
    for (int c = 0; c < 3; ++c)
      for (int l = 0; l < 27; ++l) k += W[(a * 3 + c) * 27 + l] * feat[c][l];
    K[a] = k;
  }
}

/* CConv output at every cell of the level (no interior masking):
 *   out_p = sum_a K_a(p) * v(p + a),  v zero-padded. */
void or_cconv(const double *img, int nx, int ny, int nz, const double *W, const double *B, const double *v,
              double *out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        double K[27];
        cconv_kernel_at(img, nx, ny, nz, W, B, x, y, z, K);
        double acc = 0.0;
        for (int a = 0; a < 27; ++a)
          acc += K[a] * vec_at(v, nx, ny, nz, x + (a % 3) - 1, y + (a / 3) % 3 - 1, z + a / 9 - 1);
        out[((size_t)z * ny + y) * nx + x] = acc;
      }
}

/* Per-cell kernels of a CConv block for every cell, K[p*27 + a] (used by the
 * tests to inspect the kernel generator on its own). */
void or_cconv_kernels(const double *img, int nx, int ny, int nz, const double *W, const double *B, double *K) {
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x)
        cconv_kernel_at(img, nx, ny, nz, W, B, x, y, z, K + 27 * (((size_t)z * ny + y) * nx + x));
}

/* Reverse of or_cconv for a given output cotangent g:
 *   gv(q)      += K_a(p) g(p)             for q = p + a inside the grid
 *   gK_a(p)     = g(p) v(p + a)
 *   gW[a][c][l]+= gK_a(p) I_c(p + l)      (padding included, as in forward)
 *   gB[a]      += gK_a(p)
 * gv, gW, gB are accumulated into (callers zero them). */
void or_cconv_backward(const double *img, int nx, int ny, int nz, const double *W, const double *B, const double *v,
                       const double *g, double *gv, double *gW, double *gB) {
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        size_t p = ((size_t)z * ny + y) * nx + x;
        double K[27];
        cconv_kernel_at(img, nx, ny, nz, W, B, x, y, z, K);
        for (int a = 0; a < 27; ++a) {
          int xx = x + (a % 3) - 1, yy = y + (a / 3) % 3 - 1, zz = z + a / 9 - 1;
          if (gv && inside(nx, ny, nz, xx, yy, zz)) gv[((size_t)zz * ny + yy) * nx + xx] += K[a] * g[p];
          double gk = g[p] * vec_at(v, nx, ny, nz, xx, yy, zz);
          if (gB) gB[a] += gk;
          if (gW)
            for (int c = 0; c < 3; ++c)
              for (int l = 0; l < 27; ++l)
                gW[(a * 3 + c) * 27 + l] +=
                    gk * image_at(img, c, nx, ny, nz, x + (l % 3) - 1, y + (l / 3) % 3 - 1, z + l / 9 - 1);
        }
      }
}

/* ------------------------------------------------------------------------ */
/* The BF16 precision form.  This is a numerical form of the CUDA library    */
/* (its NPSOLVE_BF16 setting), not something the paper defines; it is        */
/* modelled here so that the library's BF16 solves can be compared with a    */
/* definition of what they compute.  The form is the network of Alg. 2 with */
/* every CConv kernel value rounded to BF16:                                  */
/*  1. The three image channels sum to one (Sec. 3.2), also at the solid     */
/*     padding, so I_solid = 1 - I_fluid - I_air and the kernel of Sec. 4.2.1 */
/*     K_a(p) = B_a + sum_c sum_l W[a][c][l] I_c(p+l) equals                 */
/*       B'_a + sum_l ( Wf'[a][l] nF(p+l) + Wa'[a][l] nA(p+l) )              */
/*     with B'_a = B_a + sum_l W[a][solid][l],                               */
/*          Wf'[a][l] = (W[a][fluid][l] - W[a][solid][l]) / F,               */
/*          Wa'[a][l] = (W[a][air][l] - W[a][solid][l]) / F,                 */
/*     F = 8^(lvl-1) fine cells per cell of level lvl, and the integer       */
/*     counts nF = F I_fluid, nA = F I_air (0 at the padding).               */
/*  2. B', Wf', Wa' are rounded to FP32 and then to BF16.                    */
/*  3. Each K_a(p), summed exactly from the rounded terms, is rounded to     */
/*     FP32 and then to BF16.                                                */
/*  4. Everything else (applying the kernels, pooling, interpolation, Aff,   */
/*     the solver) is unchanged, in FP64.                                    */
/* ------------------------------------------------------------------------ */

/* Round to BF16 (8 significant bits, FP32's exponent range), ties to even,
 * after rounding to FP32.  Written from the definition of the format: a
 * normal value m 2^e (0.5 <= |m| < 1) keeps round(m 2^8) 2^(e-8); below the
 * smallest normal 2^-126 the spacing is fixed at 2^-133. */
double or_round_bf16(double v) {
  float f = (float)v;
  if (f == 0.0f || isnan(f) || isinf(f)) return f;
  double a = (double)f, r;
  if (fabs(a) < ldexp(1.0, -126)) {
    r = ldexp(nearbyint(ldexp(a, 133)), -133);
  } else {
    int e;
    double m = frexp(a, &e);
    r = ldexp(nearbyint(ldexp(m, 8)), e - 8);
  }
  if (fabs(r) > 3.4028234663852886e38) r = r > 0 ? INFINITY : -INFINITY;
  return r;
}

/* Step 1-2: the rounded folded parameters of one CConv block at level lvl. */
static void bf16_fold(const double *W, const double *B, int lvl, double Wf[27][27], double Wa[27][27], double Bp[27]) {
  double F = pow(8.0, lvl - 1);
  for (int a = 0; a < 27; ++a) {
    double bsum = B[a];
    for (int l = 0; l < 27; ++l) bsum += W[(a * 3 + 2) * 27 + l];
    Bp[a] = or_round_bf16(bsum);
    for (int l = 0; l < 27; ++l) {
      Wf[a][l] = or_round_bf16((W[(a * 3 + 0) * 27 + l] - W[(a * 3 + 2) * 27 + l]) / F);
      Wa[a][l] = or_round_bf16((W[(a * 3 + 1) * 27 + l] - W[(a * 3 + 2) * 27 + l]) / F);
    }
  }
}

/* Step 3: the BF16-form kernel of the cell (x,y,z) of level lvl. */
static void bf16_kernel_at(const double *img, int nx, int ny, int nz, double Wf[27][27], double Wa[27][27],
                           const double Bp[27], int lvl, int x, int y, int z, double K[27]) {
  double F = pow(8.0, lvl - 1), nF[27], nA[27];
  for (int l = 0; l < 27; ++l) {
    int xx = x + (l % 3) - 1, yy = y + (l / 3) % 3 - 1, zz = z + l / 9 - 1;
    nF[l] = F * image_at(img, 0, nx, ny, nz, xx, yy, zz);
    nA[l] = F * image_at(img, 1, nx, ny, nz, xx, yy, zz);
  }
  for (int a = 0; a < 27; ++a) {
    double k = Bp[a];
    for (int l = 0; l < 27; ++l) k += Wf[a][l] * nF[l] + Wa[a][l] * nA[l];
    K[a] = or_round_bf16(k);
  }
}

/* CConv of level lvl in the BF16 form (step 4: the kernels applied in FP64). */
void or_cconv_bf16(const double *img, int nx, int ny, int nz, const double *W, const double *B, int lvl,
                   const double *v, double *out) {
  double Wf[27][27], Wa[27][27], Bp[27];
  bf16_fold(W, B, lvl, Wf, Wa, Bp);
#pragma omp parallel for schedule(dynamic, 1)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        double K[27];
        bf16_kernel_at(img, nx, ny, nz, Wf, Wa, Bp, lvl, x, y, z, K);
        double acc = 0.0;
        for (int a = 0; a < 27; ++a)
          acc += K[a] * vec_at(v, nx, ny, nz, x + (a % 3) - 1, y + (a / 3) % 3 - 1, z + a / 9 - 1);
        out[((size_t)z * ny + y) * nx + x] = acc;
      }
}

/* BF16-form kernels of every cell of level lvl, K[p*27 + a] (for the tests). */
void or_cconv_kernels_bf16(const double *img, int nx, int ny, int nz, const double *W, const double *B, int lvl,
                           double *K) {
  double Wf[27][27], Wa[27][27], Bp[27];
  bf16_fold(W, B, lvl, Wf, Wa, Bp);
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x)
        bf16_kernel_at(img, nx, ny, nz, Wf, Wa, Bp, lvl, x, y, z, K + 27 * (((size_t)z * ny + y) * nx + x));
}

/* A CConv of level lvl in the exact form (form 0) or the BF16 form (form 1). */
static void cconv_form(const double *img, int nx, int ny, int nz, const double *W, int lvl, int form, const double *v,
                       double *out) {
  if (form == 1) or_cconv_bf16(img, nx, ny, nz, W, W + 27 * 3 * 27, lvl, v, out);
  else or_cconv(img, nx, ny, nz, W, W + 27 * 3 * 27, v, out);
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.2.1: the affine block Aff, read in 3D with normaliser 1/(27 n_l):    */
/*   Aff(I) = Bbar + 1/(27 n) sum_p sum_c sum_l Wbar[c][l] I_c(p + l).        */
/* ------------------------------------------------------------------------ */
double or_aff(const double *img, int nx, int ny, int nz, const double *Wbar, double Bbar) {
  double s = 0.0;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x)
        for (int c = 0; c < 3; ++c)
          for (int l = 0; l < 27; ++l)
            s += Wbar[c * 27 + l] *
                 image_at(img, c, nx, ny, nz, x + (l % 3) - 1, y + (l / 3) % 3 - 1, z + l / 9 - 1);
  return Bbar + s / (27.0 * (double)cells(nx, ny, nz));
}

/* d Aff / d Wbar[c][l] = 1/(27 n) sum_p I_c(p + l)  (d Aff / d Bbar = 1). */
void or_aff_grad(const double *img, int nx, int ny, int nz, double *dWbar) {
  for (int i = 0; i < 81; ++i) dWbar[i] = 0.0;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x)
        for (int c = 0; c < 3; ++c)
          for (int l = 0; l < 27; ++l)
            dWbar[c * 27 + l] += image_at(img, c, nx, ny, nz, x + (l % 3) - 1, y + (l / 3) % 3 - 1, z + l / 9 - 1);
  for (int i = 0; i < 81; ++i) dWbar[i] /= 27.0 * (double)cells(nx, ny, nz);
}

/* ------------------------------------------------------------------------ */
/* Alg. 2: the L-level network P_net(I, r).                                   */
/* ------------------------------------------------------------------------ */

size_t or_weight_count(int L) {
  if (L < 1) return 0;
  return (size_t)(L - 1) * (2 * CCONV_PARAMS + 2 * AFF_PARAMS) + CCONV_PARAMS;
}

/* Offsets of each block inside the flat weight blob. */
static const double *w_cconv1(const double *w, int L, int lvl) {
  if (lvl < L) return w + (size_t)(lvl - 1) * (2 * CCONV_PARAMS + 2 * AFF_PARAMS);
  return w + (size_t)(L - 1) * (2 * CCONV_PARAMS + 2 * AFF_PARAMS);
}
static const double *w_cconv2(const double *w, int lvl) {
  return w + (size_t)(lvl - 1) * (2 * CCONV_PARAMS + 2 * AFF_PARAMS) + CCONV_PARAMS;
}
static const double *w_aff(const double *w, int lvl, int which) {
  return w + (size_t)(lvl - 1) * (2 * CCONV_PARAMS + 2 * AFF_PARAMS) + 2 * CCONV_PARAMS + (size_t)which * AFF_PARAMS;
}

/* Everything a forward pass produces, kept for the backward pass. */
typedef struct {
  int L;
  int dims[8][3];
  double *img[8]; /* I^l, 3 channels */
  double *r1[8];  /* input of CConv1^l */
  double *x1[8];  /* CConv1^l output (x^L at l = L) */
  double *r2[8];  /* interpolated input of CConv2^l */
  double *x2[8];  /* CConv2^l output */
  double *x[8];   /* combined output of level l (x^L = x1^L) */
  double c1[8], c2[8];
} or_fwd;

static void fwd_free(or_fwd *f) {
  for (int l = 1; l <= f->L; ++l) {
    free(f->img[l]);
    free(f->r1[l]);
    free(f->x1[l]);
    free(f->r2[l]);
    free(f->x2[l]);
    if (l < f->L) free(f->x[l]);
  }
}

static int check_dims(int nx, int ny, int nz, int L) {
  if (L < 1 || L > 7 || nx < 1 || ny < 1 || nz < 1) return OR_BAD_DIMS;
  int m = 1 << (L - 1);
  if (nx % m || ny % m || nz % m) return OR_BAD_DIMS; /* Sec. 4.2.1: sizes divisible by 2^(L-1) */
  return OR_OK;
}

/* Forward pass of Alg. 2, keeping all intermediates.  The input r is first
 * zeroed outside the fluid (the reduced vector padded with zeros, Sec. 4.2). */
static int network_forward(const uint8_t *lab, int nx, int ny, int nz, int L, const double *w, int form,
                           const double *r, or_fwd *f) {
  int st = check_dims(nx, ny, nz, L);
  if (st) return st;
  memset(f, 0, sizeof(*f));
  f->L = L;
  for (int l = 1; l <= L; ++l) {
    f->dims[l][0] = nx >> (l - 1);
    f->dims[l][1] = ny >> (l - 1);
    f->dims[l][2] = nz >> (l - 1);
    size_t n = cells(f->dims[l][0], f->dims[l][1], f->dims[l][2]);
    f->img[l] = malloc(sizeof(double) * 3 * n);
    f->r1[l] = malloc(sizeof(double) * n);
    f->x1[l] = malloc(sizeof(double) * n);
    f->r2[l] = calloc(n, sizeof(double));
    f->x2[l] = calloc(n, sizeof(double));
    if (l < L) f->x[l] = malloc(sizeof(double) * n);
  }
  size_t n1 = cells(nx, ny, nz);
  or_image_from_labels(lab, nx, ny, nz, f->img[1]);
  for (size_t p = 0; p < n1; ++p) f->r1[1][p] = lab[p] == LAB_FLUID ? r[p] : 0.0;
  /* Down pass: I^{l+1} = Pool(I^l); x1^l = CConv1^l(r1^l, I^l); r1^{l+1} = Pool(x1^l). */
  for (int l = 1; l < L; ++l) {
    int *d = f->dims[l];
    or_avgpool2(f->img[l], 3, d[0], d[1], d[2], f->img[l + 1]);
    const double *W = w_cconv1(w, L, l);
    cconv_form(f->img[l], d[0], d[1], d[2], W, l, form, f->r1[l], f->x1[l]);
    or_avgpool2(f->x1[l], 1, d[0], d[1], d[2], f->r1[l + 1]);
  }
  /* Coarsest level: a single convolution. */
  {
    int *d = f->dims[L];
    const double *W = w_cconv1(w, L, L);
    cconv_form(f->img[L], d[0], d[1], d[2], W, L, form, f->r1[L], f->x1[L]);
    f->x[L] = f->x1[L];
  }
  /* Up pass: r2^l = Interp(x^{l+1}); x2^l = CConv2^l(r2^l, I^l);
   * x^l = Aff1^l(I^l) x1^l + Aff2^l(I^l) x2^l. */
  for (int l = L - 1; l >= 1; --l) {
    int *d = f->dims[l];
    int *dc = f->dims[l + 1];
    or_interp_up2(f->x[l + 1], dc[0], dc[1], dc[2], f->r2[l]);
    const double *W = w_cconv2(w, l);
    cconv_form(f->img[l], d[0], d[1], d[2], W, l, form, f->r2[l], f->x2[l]);
    const double *A1 = w_aff(w, l, 0), *A2 = w_aff(w, l, 1);
    f->c1[l] = or_aff(f->img[l], d[0], d[1], d[2], A1, A1[81]);
    f->c2[l] = or_aff(f->img[l], d[0], d[1], d[2], A2, A2[81]);
    size_t n = cells(d[0], d[1], d[2]);
    for (size_t p = 0; p < n; ++p) f->x[l][p] = f->c1[l] * f->x1[l][p] + f->c2[l] * f->x2[l][p];
  }
  return OR_OK;
}

/* z = P_net(I, r): Alg. 2, with the output restricted to the fluid cells
 * (Sec. 4.2: the non-fluid entries of the output are removed). */
int or_network(const uint8_t *lab, int nx, int ny, int nz, int L, const double *w, const double *r, double *z) {
  or_fwd f;
  int st = network_forward(lab, nx, ny, nz, L, w, 0, r, &f);
  if (st) return st;
  size_t n = cells(nx, ny, nz);
  for (size_t p = 0; p < n; ++p) z[p] = lab[p] == LAB_FLUID ? f.x[1][p] : 0.0;
  fwd_free(&f);
  return OR_OK;
}

/* z = P_net(I, r) in the exact form (form 0, as or_network) or the BF16
 * form (form 1). */
int or_network_form(const uint8_t *lab, int nx, int ny, int nz, int L, const double *w, int form, const double *r,
                    double *z) {
  or_fwd f;
  int st = network_forward(lab, nx, ny, nz, L, w, form, r, &f);
  if (st) return st;
  size_t n = cells(nx, ny, nz);
  for (size_t p = 0; p < n; ++p) z[p] = lab[p] == LAB_FLUID ? f.x[1][p] : 0.0;
  fwd_free(&f);
  return OR_OK;
}

/* Intermediates of one forward pass, for inspecting a single level:
 * which = 0 x1^l, 1 r2^l, 2 x2^l, 3 x^l, 4 r1^l; also returns c1^l, c2^l. */
int or_network_level(const uint8_t *lab, int nx, int ny, int nz, int L, const double *w, const double *r, int lvl,
                     int which, double *out, double *c12) {
  or_fwd f;
  int st = network_forward(lab, nx, ny, nz, L, w, 0, r, &f);
  if (st) return st;
  if (lvl < 1 || lvl > L) {
    fwd_free(&f);
    return OR_BAD_ARG;
  }
  size_t n = cells(f.dims[lvl][0], f.dims[lvl][1], f.dims[lvl][2]);
  const double *src = which == 0 ? f.x1[lvl] : which == 1 ? f.r2[lvl] : which == 2 ? f.x2[lvl]
                    : which == 3 ? f.x[lvl] : f.r1[lvl];
  memcpy(out, src, sizeof(double) * n);
  if (c12) {
    c12[0] = f.c1[lvl];
    c12[1] = f.c2[lvl];
  }
  fwd_free(&f);
  return OR_OK;
}

/* Reverse-mode derivative of z = P_net(I, r) for an output cotangent gz:
 * accumulates d<gz, z>/dw into gw (zeroed here) and d<gz,z>/dr into gr
 * (optional).  All forward intermediates are stored, not recomputed. */
int or_network_backward(const uint8_t *lab, int nx, int ny, int nz, int L, const double *w, const double *r,
                        const double *gz, double *gw, double *gr) {
  or_fwd f;
  int st = network_forward(lab, nx, ny, nz, L, w, 0, r, &f);
  if (st) return st;
  size_t nw = or_weight_count(L);
  memset(gw, 0, sizeof(double) * nw);
  double *gx[8] = {0}, *gx1[8] = {0};
  for (int l = 1; l <= L; ++l) {
    size_t n = cells(f.dims[l][0], f.dims[l][1], f.dims[l][2]);
    gx[l] = calloc(n, sizeof(double));
    gx1[l] = calloc(n, sizeof(double));
  }
  size_t n1 = cells(nx, ny, nz);
  for (size_t p = 0; p < n1; ++p) gx[1][p] = lab[p] == LAB_FLUID ? gz[p] : 0.0; /* output restriction */
  if (L == 1) memcpy(gx1[1], gx[1], sizeof(double) * n1);                       /* x^1 = x1^1 */
  /* Up pass in reverse (l = 1 .. L-1): combine, CConv2, interpolation. */
  for (int l = 1; l < L; ++l) {
    int *d = f.dims[l], *dc = f.dims[l + 1];
    size_t n = cells(d[0], d[1], d[2]);
    double gc1 = 0.0, gc2 = 0.0;
    for (size_t p = 0; p < n; ++p) {
      gc1 += gx[l][p] * f.x1[l][p];
      gc2 += gx[l][p] * f.x2[l][p];
    }
    double *gA1 = gw + (w_aff(w, l, 0) - w), *gA2 = gw + (w_aff(w, l, 1) - w);
    double dW[81];
    or_aff_grad(f.img[l], d[0], d[1], d[2], dW);
    for (int i = 0; i < 81; ++i) {
      gA1[i] += gc1 * dW[i];
      gA2[i] += gc2 * dW[i];
    }
    gA1[81] += gc1;
    gA2[81] += gc2;
    double *gx2 = malloc(sizeof(double) * n), *gr2 = calloc(n, sizeof(double));
    for (size_t p = 0; p < n; ++p) {
      gx1[l][p] += f.c1[l] * gx[l][p];
      gx2[p] = f.c2[l] * gx[l][p];
    }
    const double *W = w_cconv2(w, l);
    double *gW = gw + (W - w);
    or_cconv_backward(f.img[l], d[0], d[1], d[2], W, W + 2187, f.r2[l], gx2, gr2, gW, gW + 2187);
    double *gxc = malloc(sizeof(double) * cells(dc[0], dc[1], dc[2]));
    or_interp_up2_adjoint(gr2, dc[0], dc[1], dc[2], gxc);
    size_t nc = cells(dc[0], dc[1], dc[2]);
    if (l + 1 == L)
      for (size_t p = 0; p < nc; ++p) gx1[L][p] += gxc[p]; /* x^L = x1^L */
    else
      for (size_t p = 0; p < nc; ++p) gx[l + 1][p] += gxc[p];
    free(gx2);
    free(gr2);
    free(gxc);
  }
  /* Down pass in reverse (l = L .. 1): CConv1 and pooling. */
  double *gr1_next = NULL;
  for (int l = L; l >= 1; --l) {
    int *d = f.dims[l];
    size_t n = cells(d[0], d[1], d[2]);
    if (gr1_next) {
      double *tmp = malloc(sizeof(double) * n);
      or_avgpool2_adjoint(gr1_next, d[0], d[1], d[2], tmp);
      for (size_t p = 0; p < n; ++p) gx1[l][p] += tmp[p];
      free(tmp);
      free(gr1_next);
    }
    const double *W = w_cconv1(w, L, l);
    double *gW = gw + (W - w);
    double *gr1 = calloc(n, sizeof(double));
    or_cconv_backward(f.img[l], d[0], d[1], d[2], W, W + 2187, f.r1[l], gx1[l], gr1, gW, gW + 2187);
    gr1_next = gr1;
  }
  if (gr)
    for (size_t p = 0; p < n1; ++p) gr[p] = lab[p] == LAB_FLUID ? gr1_next[p] : 0.0; /* input padding */
  free(gr1_next);
  for (int l = 1; l <= L; ++l) {
    free(gx[l]);
    free(gx1[l]);
  }
  fwd_free(&f);
  return OR_OK;
}

/* Training loss of Sec. 4.2.3 for one example, Loss = || b - A P_net(I, b) ||_2,
 * and (if gw != NULL) its gradient with respect to the weights:
 *   dLoss/dz = -A res / ||res||, res = b - A z (A symmetric). */
int or_loss(const uint8_t *lab, int nx, int ny, int nz, int L, const double *w, const double *b, double *loss,
            double *gw) {
  size_t n = cells(nx, ny, nz);
  double *bm = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n), *az = malloc(sizeof(double) * n);
  for (size_t p = 0; p < n; ++p) bm[p] = lab[p] == LAB_FLUID ? b[p] : 0.0;
  int st = or_network(lab, nx, ny, nz, L, w, bm, z);
  if (st) {
    free(bm);
    free(z);
    free(az);
    return st;
  }
  or_lap_apply(lab, nx, ny, nz, z, az);
  double s = 0.0;
  for (size_t p = 0; p < n; ++p) {
    az[p] = bm[p] - az[p]; /* res, zero off fluid */
    s += az[p] * az[p];
  }
  double nres = sqrt(s);
  *loss = nres;
  if (gw) {
    double *gz = malloc(sizeof(double) * n);
    or_lap_apply(lab, nx, ny, nz, az, gz);
    for (size_t p = 0; p < n; ++p) gz[p] = nres > 0.0 ? -gz[p] / nres : 0.0;
    st = or_network_backward(lab, nx, ny, nz, L, w, bm, gz, gw, NULL);
    free(gz);
  }
  free(bm);
  free(z);
  free(az);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.1, Algorithm 1: NPSDO.                                              */
/* ------------------------------------------------------------------------ */

static double dot(const double *a, const double *b, size_t n) {
  double s = 0.0;
  for (size_t p = 0; p < n; ++p) s += a[p] * b[p];
  return s;
}

/* Preconditioner choices for the solver, so that the reductions stated in
 * Sec. 4.1 can be checked: 0 = the network of Alg. 2, 1 = identity (masked),
 * 2 = a dense n x n matrix applied to the masked vector, 3 = the symmetric
 * variant P_sym,1 = P_net^T P_net of the appendix's symmetry analysis, 4 =
 * the network in the BF16 form (or_cconv_bf16). */
#define PREC_NETWORK 0
#define PREC_IDENTITY 1
#define PREC_DENSE 2
#define PREC_NETWORK_SYM 3
#define PREC_NETWORK_BF16 4

/* out = P(v) for the preconditioner choices above, restricted to fluid cells
 * (the network's output restriction, Sec. 4.2).  P_net^T is the input
 * gradient of <g, P_net(v)> (the network is linear in v), taken from the
 * reverse of Alg. 2; its weight gradient is discarded. */
static void apply_prec(const uint8_t *lab, int nx, int ny, int nz, int L, const double *w, int prec,
                       const double *pdense, const double *v, double *out) {
  size_t n = cells(nx, ny, nz);
  if (prec == PREC_NETWORK) {
    or_network(lab, nx, ny, nz, L, w, v, out);
  } else if (prec == PREC_NETWORK_BF16) {
    or_network_form(lab, nx, ny, nz, L, w, 1, v, out);
  } else if (prec == PREC_NETWORK_SYM) {
    double *t = malloc(sizeof(double) * n), *gw = malloc(sizeof(double) * or_weight_count(L));
    or_network(lab, nx, ny, nz, L, w, v, t);
    or_network_backward(lab, nx, ny, nz, L, w, v, t, gw, out);
    free(t);
    free(gw);
  } else if (prec == PREC_IDENTITY) {
    for (size_t p = 0; p < n; ++p) out[p] = lab[p] == LAB_FLUID ? v[p] : 0.0;
  } else {
    for (size_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (size_t j = 0; j < n; ++j) s += pdense[i * n + j] * v[j];
      out[i] = lab[i] == LAB_FLUID ? s : 0.0;
    }
  }
}

/* Residual modes: 0 = recurrence r_k = r_{k-1} - alpha A d_k, with a true-
 * residual check on exit that restarts from r = b - A x if it fails (at most
 * 4 times); 1 = explicit r_k = b - A x_k, as printed in Alg. 1. */
int or_npsdo(const uint8_t *lab, int nx, int ny, int nz, int L, const double *w, int prec, const double *pdense,
             const double *b, double tol, int max_iter, int n_ortho, int residual_mode, double *x, int *iters,
             double *res_hist, double *final_relres) {
  size_t n = cells(nx, ny, nz);
  if (prec == PREC_NETWORK || prec == PREC_NETWORK_SYM || prec == PREC_NETWORK_BF16) {
    int st = check_dims(nx, ny, nz, L);
    if (st) return st;
  }
  if (or_check_labels(lab, nx, ny, nz)) return OR_BAD_LABELS;
  if (n_ortho < 0 || n_ortho > 16 || max_iter < 0) return OR_BAD_ARG;
  double *bm = malloc(sizeof(double) * n), *r = malloc(sizeof(double) * n), *rn = malloc(sizeof(double) * n);
  double *d = malloc(sizeof(double) * n), *ad = malloc(sizeof(double) * n), *tmp = malloc(sizeof(double) * n);
  int ring = n_ortho > 0 ? n_ortho : 1;
  double *D = malloc(sizeof(double) * n * ring), *AD = malloc(sizeof(double) * n * ring);
  double *dAd_hist = malloc(sizeof(double) * ring);
  for (size_t p = 0; p < n; ++p) {
    bm[p] = lab[p] == LAB_FLUID ? b[p] : 0.0;
    x[p] = 0.0;
    r[p] = bm[p]; /* r_0 = b - A x_0 with x_0 = 0 */
  }
  double nb = sqrt(dot(bm, bm, n));
  if (!isfinite(nb) || !(tol >= 0.0)) {
    free(bm);
    free(r);
    free(rn);
    free(d);
    free(ad);
    free(tmp);
    free(D);
    free(AD);
    free(dAd_hist);
    return OR_BAD_ARG;
  }
  double eps = tol * nb; /* convergence when ||r_k|| < tol ||b|| */
  int k = 0, status = OR_OK, restarts = 0;
  double nr = nb;
  if (res_hist) res_hist[0] = nb;
  for (;;) {
    while (nr >= eps && nr > 0.0) {
      if (k >= max_iter) {
        status = OR_NO_CONVERGENCE;
        break;
      }
      k += 1;
      /* d_k = P_net(I, r_{k-1} / ||r_{k-1}||) */
      for (size_t p = 0; p < n; ++p) rn[p] = r[p] / nr;
      apply_prec(lab, nx, ny, nz, L, w, prec, pdense, rn, d);
      /* for k - n_ortho <= i < k (and i >= 1): d_k -= (d_k^T A d_i)/(d_i^T A d_i) d_i,
       * in ascending i, each coefficient using the already-updated d_k. */
      int i0 = k - n_ortho;
      if (i0 < 1) i0 = 1;
      for (int i = i0; i < k; ++i) {
        int slot = (i - 1) % ring;
        double cij = dot(d, AD + (size_t)slot * n, n) / dAd_hist[slot];
        const double *Di = D + (size_t)slot * n;
        for (size_t p = 0; p < n; ++p) d[p] -= cij * Di[p];
      }
      or_lap_apply(lab, nx, ny, nz, d, ad);
      double dAd = dot(d, ad, n);
      if (!(dAd > 0.0) || !isfinite(dAd)) {
        status = OR_BREAKDOWN;
        break;
      }
      double alpha = dot(r, d, n) / dAd;
      for (size_t p = 0; p < n; ++p) x[p] += alpha * d[p];
      if (residual_mode == 1) {
        or_lap_apply(lab, nx, ny, nz, x, tmp);
        for (size_t p = 0; p < n; ++p) r[p] = bm[p] - tmp[p];
      } else {
        for (size_t p = 0; p < n; ++p) r[p] -= alpha * ad[p];
      }
      if (n_ortho > 0) {
        int slot = (k - 1) % ring;
        memcpy(D + (size_t)slot * n, d, sizeof(double) * n);
        memcpy(AD + (size_t)slot * n, ad, sizeof(double) * n);
        dAd_hist[slot] = dAd;
      }
      nr = sqrt(dot(r, r, n));
      if (res_hist) res_hist[k] = nr;
    }
    if (status != OR_OK || residual_mode == 1 || restarts >= 4) break;
    /* Recurrence mode: confirm with the true residual before returning. */
    or_lap_apply(lab, nx, ny, nz, x, tmp);
    for (size_t p = 0; p < n; ++p) tmp[p] = bm[p] - tmp[p];
    double ntrue = sqrt(dot(tmp, tmp, n));
    if (ntrue < eps || ntrue == 0.0) break;
    memcpy(r, tmp, sizeof(double) * n);
    nr = ntrue;
    restarts += 1;
  }
  or_lap_apply(lab, nx, ny, nz, x, tmp);
  for (size_t p = 0; p < n; ++p) tmp[p] = bm[p] - tmp[p];
  *final_relres = nb > 0.0 ? sqrt(dot(tmp, tmp, n)) / nb : 0.0;
  *iters = k;
  free(bm);
  free(r);
  free(rn);
  free(d);
  free(ad);
  free(tmp);
  free(D);
  free(AD);
  free(dAd_hist);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Textbook PCG with the Jacobi preconditioner M = diag(A) on fluid cells.   */
/* ------------------------------------------------------------------------ */
int or_jacobi_pcg(const uint8_t *lab, int nx, int ny, int nz, const double *b, double tol, int max_iter, double *x,
                  int *iters, double *res_hist, double *final_relres) {
  size_t n = cells(nx, ny, nz);
  if (or_check_labels(lab, nx, ny, nz)) return OR_BAD_LABELS;
  double *r = malloc(sizeof(double) * n), *zz = malloc(sizeof(double) * n), *pp = malloc(sizeof(double) * n);
  double *q = malloc(sizeof(double) * n), *dg = malloc(sizeof(double) * n);
  or_lap_diag(lab, nx, ny, nz, dg);
  for (size_t p = 0; p < n; ++p) {
    x[p] = 0.0;
    r[p] = lab[p] == LAB_FLUID ? b[p] : 0.0;
    zz[p] = dg[p] > 0.0 ? r[p] / dg[p] : 0.0;
    pp[p] = zz[p];
  }
  double nb = sqrt(dot(r, r, n)), nr = nb, rz = dot(r, zz, n);
  int k = 0, status = OR_OK;
  if (res_hist) res_hist[0] = nb; /* ||r_k|| for k = 0 .. iters (res_hist may be NULL) */
  while (nr >= tol * nb && nr > 0.0) {
    if (k >= max_iter) {
      status = OR_NO_CONVERGENCE;
      break;
    }
    k += 1;
    or_lap_apply(lab, nx, ny, nz, pp, q);
    double pq = dot(pp, q, n);
    if (!(pq > 0.0)) {
      status = OR_BREAKDOWN;
      break;
    }
    double alpha = rz / pq;
    for (size_t p = 0; p < n; ++p) {
      x[p] += alpha * pp[p];
      r[p] -= alpha * q[p];
      zz[p] = dg[p] > 0.0 ? r[p] / dg[p] : 0.0;
    }
    double rz_new = dot(r, zz, n);
    double beta = rz_new / rz;
    rz = rz_new;
    for (size_t p = 0; p < n; ++p) pp[p] = zz[p] + beta * pp[p];
    nr = sqrt(dot(r, r, n));
    if (res_hist) res_hist[k] = nr;
  }
  double *ax = q;
  or_lap_apply(lab, nx, ny, nz, x, ax);
  double s = 0.0;
  for (size_t p = 0; p < n; ++p) {
    double e = (lab[p] == LAB_FLUID ? b[p] : 0.0) - ax[p];
    s += e * e;
  }
  *final_relres = nb > 0.0 ? sqrt(s) / nb : 0.0;
  *iters = k;
  free(r);
  free(zz);
  free(pp);
  free(q);
  free(dg);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.1 and the solver-variant comparison of the appendix: PCG and      */
/* flexible PCG with the network (or another preconditioner of or_npsdo) as */
/* the preconditioner.                                                      */
/* ------------------------------------------------------------------------ */

/* PCG in the textbook arrangement (Shewchuk 1994, the preconditioned CG
 * algorithm): z_k = P(r_k), rho_k = r_k^T z_k, d_1 = z_0, later
 * d = z_k + beta_k d, alpha = rho_k / d^T A d, x += alpha d, r -= alpha A d.
 *   flexible = 0: beta_k = rho_k / rho_{k-1} (Fletcher-Reeves form);
 *   flexible = 1: beta_k = z_k^T (r_k - r_{k-1}) / rho_{k-1} (the Polak-Ribiere
 *                 form of flexible PCG for non-symmetric preconditioners).
 * The network is linear in r (Sec. 4.2), and it is given the unit residual as
 * in Alg. 1: z_k = ||r_k|| P(r_k / ||r_k||).  Stop test, residual modes and
 * the replacement of the recurrence residual on exit are those of or_npsdo;
 * after a replacement the conjugate sequence restarts (beta = 0).  rho_k = 0
 * or non-finite (beta would divide by it) and d^T A d <= 0 are breakdowns. */
int or_npcg(const uint8_t *lab, int nx, int ny, int nz, int L, const double *w, int prec, const double *pdense,
            const double *b, double tol, int max_iter, int flexible, int residual_mode, double *x, int *iters,
            double *res_hist, double *final_relres) {
  size_t n = cells(nx, ny, nz);
  if (prec == PREC_NETWORK || prec == PREC_NETWORK_SYM || prec == PREC_NETWORK_BF16) {
    int st = check_dims(nx, ny, nz, L);
    if (st) return st;
  }
  if (or_check_labels(lab, nx, ny, nz)) return OR_BAD_LABELS;
  if (max_iter < 0 || !(tol >= 0.0)) return OR_BAD_ARG;
  double *bm = malloc(sizeof(double) * n), *r = malloc(sizeof(double) * n), *rprev = malloc(sizeof(double) * n);
  double *rn = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n), *d = malloc(sizeof(double) * n);
  double *ad = malloc(sizeof(double) * n), *tmp = malloc(sizeof(double) * n);
  for (size_t p = 0; p < n; ++p) {
    bm[p] = lab[p] == LAB_FLUID ? b[p] : 0.0;
    x[p] = 0.0;
    r[p] = bm[p];
    d[p] = 0.0;
  }
  double nb = sqrt(dot(bm, bm, n));
  int status = OR_OK;
  if (!isfinite(nb)) status = OR_BAD_ARG;
  double eps = tol * nb, nr = nb, rho_prev = 0.0;
  int k = 0, restarts = 0, fresh = 1;
  if (res_hist) res_hist[0] = nb;
  while (status == OR_OK) {
    while (nr >= eps && nr > 0.0) {
      if (k >= max_iter) {
        status = OR_NO_CONVERGENCE;
        break;
      }
      k += 1;
      for (size_t p = 0; p < n; ++p) rn[p] = r[p] / nr;
      apply_prec(lab, nx, ny, nz, L, w, prec, pdense, rn, z);
      for (size_t p = 0; p < n; ++p) z[p] *= nr;
      double rho = dot(r, z, n);
      if (!(rho != 0.0) || !isfinite(rho)) {
        status = OR_BREAKDOWN;
        break;
      }
      if (fresh) {
        memcpy(d, z, sizeof(double) * n);
      } else {
        double beta;
        if (flexible) {
          for (size_t p = 0; p < n; ++p) tmp[p] = r[p] - rprev[p];
          beta = dot(z, tmp, n) / rho_prev;
        } else {
          beta = rho / rho_prev;
        }
        for (size_t p = 0; p < n; ++p) d[p] = z[p] + beta * d[p];
      }
      fresh = 0;
      or_lap_apply(lab, nx, ny, nz, d, ad);
      double dAd = dot(d, ad, n);
      if (!(dAd > 0.0) || !isfinite(dAd)) {
        status = OR_BREAKDOWN;
        break;
      }
      double alpha = rho / dAd;
      for (size_t p = 0; p < n; ++p) x[p] += alpha * d[p];
      memcpy(rprev, r, sizeof(double) * n);
      if (residual_mode == 1) {
        or_lap_apply(lab, nx, ny, nz, x, tmp);
        for (size_t p = 0; p < n; ++p) r[p] = bm[p] - tmp[p];
      } else {
        for (size_t p = 0; p < n; ++p) r[p] -= alpha * ad[p];
      }
      rho_prev = rho;
      nr = sqrt(dot(r, r, n));
      if (res_hist) res_hist[k] = nr;
    }
    if (status != OR_OK || residual_mode == 1 || restarts >= 4) break;
    or_lap_apply(lab, nx, ny, nz, x, tmp);
    for (size_t p = 0; p < n; ++p) tmp[p] = bm[p] - tmp[p];
    double ntrue = sqrt(dot(tmp, tmp, n));
    if (ntrue < eps || ntrue == 0.0) break;
    memcpy(r, tmp, sizeof(double) * n);
    nr = ntrue;
    fresh = 1;
    restarts += 1;
  }
  or_lap_apply(lab, nx, ny, nz, x, tmp);
  for (size_t p = 0; p < n; ++p) tmp[p] = bm[p] - tmp[p];
  *final_relres = nb > 0.0 ? sqrt(dot(tmp, tmp, n)) / nb : 0.0;
  *iters = k;
  free(bm);
  free(r);
  free(rprev);
  free(rn);
  free(z);
  free(d);
  free(ad);
  free(tmp);
  return status;
}
