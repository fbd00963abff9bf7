// Host-side launchers of the npsolve kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nps_common.cuh"

namespace nps {

// npsolve.cu: the per-thread message returned by npsolve_last_error(NULL).
void set_thread_error(const char *msg);

// kernels_vec.cu
void launch_lap(const uint8_t *lab, Dims dm, const float *d, float *q, cudaStream_t s);
void launch_check_labels(const uint8_t *lab, long long n, unsigned int *bad, cudaStream_t s);
void launch_init(const uint8_t *lab, long long n, const float *b, float *r, double *x, double *part, double tol,
                 int max_iter, int n_ortho, int method, SolveState *st, double *hist, cudaStream_t s);
void launch_ortho_final(const double *part, long long n, SolveState *st, cudaStream_t s);
void launch_direction(long long n, const float *z, float *dring, const SolveState *st, cudaStream_t s);
void launch_lap_ring(const uint8_t *lab, Dims dm, const float *dring, float *qring, const float *r, double *part,
                     SolveState *st, cudaStream_t s);
void launch_update(bool recurrence, long long n, double *x, float *r, const float *dring, const float *qring,
                   double *part, SolveState *st, double *hist, cudaStream_t s);
void launch_explicit_residual(const uint8_t *lab, Dims dm, const float *b, const double *x, float *r, double *part,
                              SolveState *st, double *hist, cudaStream_t s);
// r = b - A x (FP64 arithmetic); re-opens a converged solve whose true
// residual is above tolerance; relres[0..1] = ||b - A x|| / ||b||, ||b||.
// The final kernels of the true residual (partials of two per block).
void launch_restart_final(const double *part, int nblocks, SolveState *st, int *reopened, double *relres,
                          cudaStream_t s);
void launch_relres_final(const double *part, int nblocks, double *relres, cudaStream_t s);
// The true residual of the double-float x (xhi, xlo) in double-float FP32 arithmetic, with the stencil codes;
// reopened null: the figures only; else the residual replacement (r_k's buffer by parity) and re-opening.
void launch_true_residual4(const uint16_t *code, Dims dm, const float *b, const float *xhi, const float *xlo, float *r,
                           float *r_alt, double *part, SolveState *st, int *reopened, double *relres,
                           cudaStream_t s);
void launch_replace_residual(const uint8_t *lab, Dims dm, const float *b, const double *x, float *r, float *r_alt,
                             double *part, SolveState *st, int *reopened, double *relres, cudaStream_t s);
void launch_relres(const uint8_t *lab, Dims dm, const float *b, const double *x, double *part, double *out,
                   cudaStream_t s);
size_t pcg_state_bytes();
void launch_pcg_init(const uint8_t *lab, Dims dm, const float *b, float *r, float *p, double *x, double *part,
                     double tol, void *st, double *hist, cudaStream_t s);
void launch_pcg_iter(const uint8_t *lab, Dims dm, double *x, float *r, float *p, float *q, double *part, void *st,
                     double *hist, cudaStream_t s);
int pcg_done_offset();
int pcg_k_offset();

// kernels_net.cu
void launch_pyramid(const uint8_t *lab, Dims d1, ushort2 *const *counts, int L, cudaStream_t s);
// The Aff coefficients (and training statistics) of levels 1..L-1 in two
// launches: out[2 l], out[2 l + 1] = c1, c2 of level l; stats (may be null)
// + 54 l the 54 window sums scaled by 1 / (8^(l-1) 27 n_l); cnt: 128 L
// counters of scratch.
struct AffAll {
  const uint8_t *lab;
  const ushort2 *counts[kMaxLevels + 1];
  Dims dims[kMaxLevels + 1];
  const AffW *aw;
  double *out, *stats;
  unsigned long long *cnt;
  int L;
};
void launch_aff_all(const AffAll &A, cudaStream_t s);
void launch_cconv_f32(const uint8_t *lab, const ushort2 *counts, Dims dm, const CConvW *w, const float *v,
                      const float *vscale, int mask_input, int round_k, float *out, const SolveState *st,
                      cudaStream_t s);
void launch_pool(const float *in, Dims fine, float *out, const SolveState *st, cudaStream_t s);
// skip (optional, even coarse nx only): per (32 x 8 fine tile, fine plane) byte, tile-major;
// the fine cells of planes marked non-zero are left unwritten
void launch_interp(const float *in, Dims coarse, float *out, const SolveState *st, cudaStream_t s,
                   const uint8_t *skip = nullptr);
void launch_combine(long long n, const float *x1, const float *x2, const double *c12, float *out,
                    const SolveState *st, cudaStream_t s);
void launch_combine1(const uint8_t *lab, long long n, const float *x1, const float *x2, const double *c12, float *z,
                     const float *qring, const float *rk, double *part, const SolveState *st, cudaStream_t s);

// kernels_vec4.cu (nx % 4 == 0, n < 2^31)
// r = mask(b), ||b||^2 -> the solver state; x = 0, or (xhi, xlo) = 0 when
// xhi is non-null (x is then written by launch_flush_x at the end).
void launch_init4(const uint8_t *lab, int n, const float *b, float *r, double *x, float *xhi, float *xlo, double *part,
                  unsigned *ticket, double tol, int max_iter, int n_ortho, int method, SolveState *st, double *hist,
                  int num_sms, cudaStream_t s);
void launch_combine1_4(const uint8_t *lab, int n, const float *x1, const float *x2, const double *c12, float *z,
                       const float *qring, const float *r0, const float *r1, double *part, unsigned *ticket,
                       SolveState *st, int num_sms, cudaStream_t s);
void launch_direction4(bool defer_x, int n, const float *z, float *dring, float *xhi, float *xlo, const uint32_t *gmask,
                       const SolveState *st, int n_ortho, int num_sms, cudaStream_t s);
// per-cell stencil codes of the masked Laplacian (once per solve) and q = A d with them
// per-cell stencil codes and the 1-bit-per-4-cell-group fluid mask ((n / 4 + 31) / 32 words)
void launch_lap_codes(const uint8_t *lab, Dims dm, uint16_t *code, uint32_t *gmask, cudaStream_t s);
void launch_lap4(const uint16_t *code, Dims dm, const float *dring, float *qring, const float *r, const float *r_alt,
                 double *part, unsigned *ticket, SolveState *st, int num_sms, cudaStream_t s);
// Adds the pending steps to (xhi, xlo) and writes x = xhi + xlo in FP64.
void launch_flush_x(int n, float *xhi, float *xlo, double *x, const float *dring, SolveState *st, int num_sms,
                    cudaStream_t s);
// r_alt non-null: two residual buffers (r_k in buffer k mod 2), applied only while a step is pending
void launch_update4(bool recurrence, int n, double *x, float *r, float *r_alt, const float *dring, const float *qring,
                    double *part, unsigned *ticket, SolveState *st, double *hist, int num_sms, cudaStream_t s);

// kernels_umma.cu
void prepare_umma_weights(const CConvW &w, int nsplit, uint8_t *out);
int umma_weight_bytes(int nsplit);
void launch_cconv_umma(int nsplit, const uint8_t *lab, const ushort2 *counts, Dims dm, const uint8_t *wsplit,
                       const float *v, const float *vscale, int mask_input, float *out, const SolveState *st,
                       int *err, int num_sms, cudaStream_t s);
void launch_umma_selftest(float *d_out, float *d_ref, int *err, cudaStream_t s);

// kernels_cached.cu: per-solve classification and kernel cache, streamed CConv
bool stream_shape_ok(Dims d);          // the TMA boxes need rows of a multiple of 16 bytes

// kernels_tail.cu: the coarse levels T..L of the network in one cluster launch.
constexpr int kTailCtas = 8;                 // CTAs of the cluster
constexpr long long kTailMaxCells = 4096;    // levels of at most this many cells run in the tail
constexpr int kTailMaxSmem = 160 * 1024;     // shared memory a tail CTA may stage (bytes)
struct TailParams {
  int T, L;                                  // levels T..L (T >= 2); r2 of level T-1 is written too
  Dims dims[kMaxLevels + 1];
  const float *k1[kMaxLevels + 1], *k2[kMaxLevels + 1];  // per-cell kernels, 27 x n floats, tap-major
  float *x1[kMaxLevels + 1], *r1[kMaxLevels + 1], *r2[kMaxLevels + 1], *xc[kMaxLevels + 1];
  const double *affc;                        // c1, c2 of each level (2 l, 2 l + 1)
  const SolveState *st;                      // may be null
};
void launch_tail_kernels(const uint8_t *lab, const ushort2 *counts, Dims d, const CConvW *w, int round_k, float *K,
                         cudaStream_t s);
int launch_tail(const TailParams &P, cudaStream_t s);  // 0 on success
long long stream_desc_count(Dims d);   // plane descriptors of a level (tiles x nz)
size_t stream_desc_bytes();            // bytes of one plane descriptor
int cached_entry_bytes(bool bf16);     // bytes of one cached kernel
// totals[0] += cache entries (blocks padded to 4), totals[1] += mixed cells
// skip (optional, ntiles x nz bytes, tile-major): bit 0 = every window of the
// tile's plane is pure solid or pure air, bit 1 = the plane has no fluid cell.
// mcount (optional, same layout): the mixed-window cells of each (tile, plane).
void launch_classify(const uint8_t *lab, const ushort2 *counts, Dims d, uint32_t full, void *desc, unsigned *totals,
                     uint8_t *skip, uint16_t *mcount, int num_sms, cudaStream_t s);
// Cells and mixed-window cells (from mcount, host) of the units of a list (host).
void stream_units_work(Dims d, const int *list, int n, int zc, const uint16_t *mcount, long long *cells,
                       long long *mixed);
// wsplit0/1: the tensor-core weight splits of the two blocks (nsplit BF16
// terms each) to generate on the tensor cores, or null for CUDA cores
void launch_generate(bool bf16, const uint8_t *lab, const ushort2 *counts, Dims d, const CConvW *w, int nblk,
                     const void *desc, void *cache0, void *cache1, const uint8_t *wsplit0, const uint8_t *wsplit1,
                     int nsplit, int *err, int num_sms, cudaStream_t s);
// kfix: the 81 constants K^S, K^F, K^A of the pure windows.  mode: which
// outputs are computed, the others written as 0: STREAM_MODE_ALL; _ZERO_PURE
// (the input is zero off fluid, so pure-air and pure-solid windows give
// exactly 0: level-1 CConv1); _FLUID_ONLY (only fluid cells are used: the
// level-1 CConv2 inside the network).  Returns -1 if a tensor map cannot be
// encoded.
enum { STREAM_MODE_ALL = 0, STREAM_MODE_ZERO_PURE = 1, STREAM_MODE_FLUID_ONLY = 2 };
// Fusion of the level-1 combination into the level-1 CConv2 inside a solve:
// out = z = mask_fluid(c1 x1 + c2 CConv2(v)) and the orthogonalisation dots
// z . q_i of the previous directions (ring of nring vectors of one grid each),
// finished by the last CTA into st->coef (as launch_combine1_4).
struct StreamFusion {
  const float *qring;
  int nring;
  const float *rb[2];  // the residual buffers: r_k in rb[k & 1] (rb[1] null: one buffer)
  int method;          // the solver's method (kMethod*; the state holds the same)
  double *part;     // partial dots: one row of 2 per (unit, consumer warp)
  size_t part_cap;  // doubles part can hold
  unsigned *ticket;
  SolveState *st;
};
bool stream_fusion_ok(int n_ortho);  // the fused kernel loads up to two previous directions
// The units (tile x chunk of zc planes, index chunk * ntiles + tile) a launch
// processes when the others have nothing to compute (occupancy-aware
// sparsity: a level-1 CConv1 over windows that are all pure solid or air
// outputs zeros, a level-1 CConv2 is needed on fluid cells only).
struct StreamUnits {
  const int *list;  // device
  int n;
  int zc;
};
int stream_cap(bool bf16, bool fused, int mode, bool upd, int num_sms);  // CTAs of one wave
// Picks the chunk for the units with a plane whose skip byte lacks `bit`,
// writes their indices to list (ntiles x nz / 2 entries at most), returns the chunk.
int choose_stream_units(Dims d, const uint8_t *skip, int bit, int cap, int *list, int *n);
// out[t][z] (ntiles x nz, tile-major) = some (tile, plane) within +-rx, +-ry tiles and +-rz
// planes of (t, z) lacks `bit` in skip; inverted (1 = none) when `invert`.
void launch_dilate_flags(const uint8_t *skip, Dims d, int bit, int rx, int ry, int rz, bool invert, uint8_t *out,
                         cudaStream_t s);
// The level-1 CConv1 that first forms the pending residual step: r_{k+1} =
// r_k - alpha q_{k+1} with r_k in rb[k mod 2] (the launch's v must be rb[0]),
// written to rb[(k + 1) mod 2], with ||r_{k+1}||^2 and the end-of-step state
// update of the recurrence (k_update4's), when SolveState.upd_pending is set.
struct StreamUpdate {
  float *rb[2];
  const float *qring;
  int nring;
  double *part;     // one partial per CTA
  size_t part_cap;  // doubles part can hold
  unsigned *ticket;
  double *hist;
  SolveState *st;
};
int launch_cconv_stream(bool bf16, Dims dm, const float *kfix, const void *desc, const void *cache, const float *v,
                        const float *vscale, float *out, float *pooled, const float *x1, const double *c12, int mode,
                        const SolveState *st, int *err, int num_sms, cudaStream_t s,
                        const StreamFusion *fuse = nullptr, const StreamUpdate *upd = nullptr,
                        const StreamUnits *units = nullptr);
void launch_mask_copy(const uint8_t *lab, long long n, const float *in, float *out, cudaStream_t s);

// kernels_train.cu
void launch_materialize_K(const uint8_t *lab, const ushort2 *counts, Dims d, const CConvW *w, float *K,
                          cudaStream_t s);
// Training forward of one CConv block with the weights as kernel parameters;
// the per-cell kernels go to K[p][27] for the backward.  kpure (host, 81
// floats): the kernels of pure solid, fluid and air windows; full: the count
// of a pure cell of the level (8^(l-1)).
void launch_cconv_store_K(const uint8_t *lab, const ushort2 *counts, Dims d, const CConvW &w, const float *kpure,
                          float full, const float *v, int mask_input, int round_k, float *K, float *out,
                          cudaStream_t s);
// The same on the tensor cores (levels with counts <= 256 per cell, nx a
// multiple of 32): wsplit (device) the block's folded weights in `nsplit` BF16
// terms, the solve's kernel-generation layout; *err set if an MMA wait timed out.
void launch_cconv_store_K_tc(const uint8_t *lab, const ushort2 *counts, Dims d, const uint8_t *wsplit, int nsplit,
                             const float *kpure, float full, const float *v, int mask_input, int round_k, float *K,
                             float *out, int *err, int num_sms, cudaStream_t s);
void launch_cconv_transpose(const float *K, const float *g, Dims d, float *gv, cudaStream_t s);
int wgrad_blocks(Dims d);
int wgrad_outputs();
void launch_cconv_wgrad(const uint8_t *lab, const ushort2 *counts, Dims d, const float *v, const float *g,
                        double *part, double *out, cudaStream_t s);
void launch_cconv_wgrad_tc(const uint8_t *lab, const ushort2 *counts, Dims d, const float *v, const float *g,
                           double *part, double *out, int *err, int num_sms, cudaStream_t s);
void launch_pool_adjoint_add(const float *gc, Dims fine, float *gf, cudaStream_t s);
void launch_interp_adjoint_add(const float *gfine, Dims coarse, float *gc, cudaStream_t s);
// Dots a.b and a.c (c optional) of the levels l0 .. l0+count-1 in two launches;
// part holds count x kRedMaxBlocks x 2 doubles; out[l] receives the pair; when
// stats_src[l] is set, its 54 doubles are copied to stats_dst[l] as well.
struct Dot2Levels {
  const float *a[kMaxLevels + 1], *b[kMaxLevels + 1], *c[kMaxLevels + 1];
  long long n[kMaxLevels + 1];
  double *out[kMaxLevels + 1];
  const double *stats_src[kMaxLevels + 1];
  double *stats_dst[kMaxLevels + 1];
  int nb[kMaxLevels + 1];  // set by the launcher
  int l0, count;
};
void launch_dot2_levels(const Dot2Levels &D, double *part, cudaStream_t s);
void launch_dot2(const float *a, const float *b, const float *c, long long n, double *part, double *out,
                 cudaStream_t s);
void launch_axpby_dev(const uint8_t *lab, long long n, const double *alpha, const float *a, float beta,
                      const float *b, float *out, cudaStream_t s);
void launch_axpby(const uint8_t *lab, long long n, float alpha, const float *a, float beta, const float *b, float *out,
                  cudaStream_t s);
void launch_scale_by_inv_norm(const uint8_t *lab, long long n, float scale, const double *norm2, const float *a,
                              float *out, cudaStream_t s);

void launch_or_flag(const unsigned int *flag, unsigned int *acc, cudaStream_t s);
void launch_multidot(const float *Q, long long n, int m, const float *w, double *part, double *out, cudaStream_t s);
void launch_combine_basis(const float *Q, long long n, int m, const double *c, float beta, float *out,
                          cudaStream_t s);

// kernels_march.cu
void launch_cconv_march(int nsplit, const uint8_t *lab, const ushort2 *counts, Dims dm, const uint8_t *wsplit,
                        const float *v, const float *coarse, const float *vscale, int mask_input, float *out,
                        float *pooled, const SolveState *st, int *err, int num_sms, cudaStream_t s);

}  // namespace nps
