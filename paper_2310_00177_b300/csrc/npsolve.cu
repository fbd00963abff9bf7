// Host runtime and C ABI of the npsolve library (declared in include/npsolve.h).
//
// One handle = one network (weights in device memory, prepared once) plus a
// workspace grown on demand for the largest grid seen.  A solve is:
//   setup (once per solve, depends only on the labels): label check, image
//     pyramid, Aff coefficients c1^l, c2^l of every level (Sec. 4.2.1);
//   the NPSDO iteration (Alg. 1), device-resident: the network (Alg. 2), the
//     orthogonalisation coefficients, the direction and q = A d with fused dot
//     products, the line search, the x/r update and the stop test.  One
//     iteration is captured once as a CUDA graph and replayed; the kernels
//     turn into no-ops after the device-side stop flag is set, and the host
//     polls that flag asynchronously every few iterations;
//   a final FP64 true-residual check (with residual replacement in the
//     recurrence mode).
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <random>
#include <algorithm>
#include <string>
#include <initializer_list>
#include <vector>

#include "../../include/npsolve.h"
#include "nps_common.cuh"
#include "nps_kernels.h"

using namespace nps;

namespace {

thread_local std::string g_thread_error;

constexpr int kCConvParams = 27 * 3 * 27 + 27;
constexpr int kAffParams = 3 * 27 + 1;
constexpr int kPollEvery = 4;      // iterations per captured graph / poll
constexpr int kMaxRestarts = 4;    // residual replacements in the recurrence mode

size_t weight_count(int L) {
  if (L < 1 || L > kMaxLevels) return 0;
  return (size_t)(L - 1) * (2 * kCConvParams + 2 * kAffParams) + kCConvParams;
}

struct Workspace {
  Dims dims{0, 0, 0};
  long long cap = 0;  // cells of level 1 the buffers were sized for
  size_t bytes = 0;   // device bytes held by this workspace
  float *r = nullptr, *z = nullptr, *dring = nullptr, *qring = nullptr;
  float *xhi = nullptr, *xlo = nullptr;  // x as a double-float pair during recurrence-mode iterations
  float *r_alt = nullptr;  // second residual buffer when the update is fused into the level-1 CConv1
  uint16_t *lapcode = nullptr;  // per-cell stencil codes of the masked Laplacian (vec4 path)
  uint32_t *gmask = nullptr;    // one bit per 4-cell group: the group holds a fluid cell (vec4 path)
  float *x1[kMaxLevels + 1] = {}, *r1[kMaxLevels + 1] = {}, *r2[kMaxLevels + 1] = {}, *x2[kMaxLevels + 1] = {},
        *xc[kMaxLevels + 1] = {};
  ushort2 *counts[kMaxLevels + 1] = {};
  // the coarse tail (kernels_tail.cu): its first level (0: none) for the
  // current grid and the materialised per-cell kernels of its levels
  int tail_T = 0;
  float *tailk = nullptr;
  size_t tailk_cap = 0;  // floats
  float *tk1[kMaxLevels + 1] = {}, *tk2[kMaxLevels + 1] = {};
  // per-solve kernel cache of the mixed-window cells (cached path)
  uint8_t *kdesc[kMaxLevels + 1] = {};    // plane descriptors per level
  long long kdesc_cap[kMaxLevels + 1] = {};  // descriptors kdesc can hold
  void *kcache[(kMaxLevels + 1) * 2] = {};
  size_t kcap[(kMaxLevels + 1) * 2] = {};    // cache entries kcache can hold
  // per level: [2 l] cache entries (blocks padded to 4), [2 l + 1] mixed cells
  unsigned *ktotal = nullptr, *h_ktotal = nullptr;
  // level-1 occupancy-aware sparsity: per (tile, plane) skip bytes (host copy: the dilated flags, then the
  // classification's) and the units of the level-1 CConv1 ([0, kskip_cap)) and CConv2 ([kskip_cap, 2 kskip_cap))
  uint8_t *kskip = nullptr, *h_kskip = nullptr;
  uint16_t *kmcount = nullptr, *h_kmcount = nullptr;  // mixed cells per level-1 (tile, plane)
  long long uwork[2][2] = {{0, 0}, {0, 0}};           // cells and mixed cells of the two level-1 lists
  int *ulist = nullptr, *h_ulist = nullptr;
  long long kskip_cap = 0;
  int un[2] = {0, 0}, uzc[2] = {0, 0};
  bool ulist_ok = false;
  // level 1: per (tile, plane) 1 = no fluid within one tile or plane (the CConv1 output is zero and the
  // level-2 -> 1 interpolation output is not read there)
  uint8_t *ineed = nullptr;
  // level 2 (not the coarsest): per (tile, plane) skip bytes, the units within
  // two coarse cells of fluid (both level-2 CConvs), and their count and chunk
  uint8_t *kskip2 = nullptr, *h_kskip2 = nullptr;
  int *ulist2 = nullptr, *h_ulist2 = nullptr;
  long long kskip2_cap = 0;
  int un2 = 0, uzc2 = 0;
  bool ulist2_ok = false;
  size_t part_cap = 0;        // doubles of part
  double *part = nullptr, *affc = nullptr, *relres = nullptr, *hist = nullptr;
  double *affs = nullptr;     // per level: the 54 scaled image window sums of the Aff blocks
  int hist_cap = 0;
  SolveState *st = nullptr;
  unsigned *tickets = nullptr;  // last-block-done counters of the fused reduction kernels
  void *pcg_st = nullptr;
  unsigned int *bad = nullptr;
  int *reopened = nullptr;
  // pinned host mirrors for polling, and the events that guard them
  SolveState *h_st = nullptr;
  int *h_flag = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  // device staging buffers of npsolve_solve_host
  uint8_t *stage_lab = nullptr;
  float *stage_b = nullptr;
  double *stage_x = nullptr;
  // captured iteration graph
  cudaGraphExec_t graph = nullptr;
  Dims graph_dims{0, 0, 0};
  const uint8_t *graph_lab = nullptr;
  const float *graph_b = nullptr;
  double *graph_x = nullptr;
  int graph_pcg = 0;
  int graph_units[6] = {0, 0, 0, 0, 0, 0};  // the unit counts and chunks baked into the captured launches
  long long graph_kernels = 0;  // kernels per replay of the graph
};

// Kernel classes timed by the optional per-class profiling (CUDA events on
// the solve's stream around each launch of the class).
enum ProfClass {
  P_SETUP,          // label check, image pyramid, Aff coefficients, r = b
  P_CCONV_L1,       // CConv1 / CConv2 of level 1 (one launch each)
  P_CCONV_COARSE,   // CConv of levels >= 2
  P_POOL,
  P_INTERP,
  P_COMBINE,        // c1 x1 + c2 x2 (level 1: with mask and orthogonalisation dots)
  P_ORTHO_DIR,      // orthogonalisation coefficients + direction
  P_LAP,            // q = A d with dots + line search
  P_UPDATE,         // x, r update + stop test
  P_FINAL,          // residual replacement check and final true residual
  P_COUNT
};
const char *const kProfNames[P_COUNT] = {"setup",   "cconv_l1",  "cconv_coarse", "pool",   "interp",
                                         "combine", "ortho_dir", "lap_alpha",    "update", "final"};

struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<int> cls;  // class of event pair i (events 2i, 2i+1)
  double ms[P_COUNT] = {};
  long long launches[P_COUNT] = {};
};

}  // namespace

struct npsolve {
  npsolve_config cfg;
  int device = 0;
  std::vector<float> weights;      // host copy of the flat blob
  CConvW *cw = nullptr;            // [(kMaxLevels+1)*2], index lvl*2 + (type-1)
  std::vector<CConvW> cw_host;     // the same on the host (kernel parameters of the training forward)
  uint8_t *uw = nullptr;           // tensor-core W splits, [(kMaxLevels+1)*2][umma_weight_bytes(3)]
  float *uni = nullptr;            // uniform-window kernel terms Bp, SWf, SWa: [(kMaxLevels+1)*2][81]
  std::vector<float> uni_host;     // the same on the host
  std::vector<float> kfix_host;    // [(kMaxLevels+1)*2][81]: K^S, K^F, K^A of the pure windows (kernel parameters)
  int nsplit = 3;                  // BF16 terms of W on the tensor cores (3: FP32 form, 1: BF16 form)
  int num_sms = 148;
  int *umma_err = nullptr;         // set by a kernel whose bounded wait (MMA or TMA completion) timed out
  bool stream_err = false;         // a tensor map of the streamed CConv could not be encoded
  AffW *aw = nullptr;              // [(kMaxLevels+1)*2]
  double *unit_c12 = nullptr;      // {1, 0} for L = 1
  Workspace ws;
  cudaStream_t cap_stream = nullptr;
  // npsolve_solve_host: the right-hand side is uploaded on copy_stream while the
  // solve's stream runs the setup from the labels; b_ready orders init after it
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t b_ready = nullptr;
  cudaEvent_t x_ready = nullptr;  // the final x is written: its download may start
  std::string err;
  std::vector<double> last_hist;
  Profiler prof;
  long long launches = 0;  // kernels enqueued by this handle since creation
  // training: backward buffers (grown on demand) and Adam state
  struct {
    long long cap = 0;
    float *gx[kMaxLevels + 1] = {}, *gx1[kMaxLevels + 1] = {};
    float *rm = nullptr, *tmp = nullptr, *tmp2 = nullptr, *res = nullptr, *gz = nullptr, *K = nullptr;
    // the per-cell kernels of every CConv of the last training forward, K[p][a]
    // per block (slot lvl*2 + type-1), kept for the backward
    float *kall = nullptr;
    long long kall_cap = 0;  // floats
    float *kslot[(kMaxLevels + 1) * 2] = {};
    bool kstore = false;     // cconv() computes and stores the kernels (training forward)
    double *part = nullptr, *out = nullptr;  // partials, and the reduced results (see train_backward)
    double *outb = nullptr;                  // one reduced-results block per example of a batch
    int outb_cap = 0;                        // examples outb holds
    unsigned int *badb = nullptr;            // label-check flag accumulated over a batch
    std::vector<double> m, v;
    long long t = 0;
  } tr;
};

namespace {

// The kernels read and write device arrays with 8- and 16-byte vector
// accesses, so every device pointer argument must be 16-byte aligned (cudaMalloc
// and framework allocators return blocks aligned far beyond that; an offset
// view into one may not be).  True if one of `ps` is not.
bool misaligned16(std::initializer_list<const void *> ps) {
  for (const void *p : ps)
    if (((uintptr_t)p & 15u) != 0) return true;
  return false;
}
constexpr const char *kAlignMsg = "device pointers must be 16-byte aligned";

int fail(npsolve *h, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  g_thread_error = buf;
  return code;
}

#define CK(h, call)                                                                                 \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return fail((h), e_ == cudaErrorMemoryAllocation ? NPSOLVE_OOM : NPSOLVE_CUDA_ERROR,          \
                  "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);      \
  } while (0)

// Records an event pair around the launches issued in its lifetime when
// profiling is on.
struct ProfScope {
  npsolve *h;
  int c;
  cudaStream_t s;
  ProfScope(npsolve *h_, int c_, cudaStream_t s_) : h(h_), c(c_), s(s_) {
    if (!h->prof.on) return;
    const size_t i = h->prof.cls.size();
    while (h->prof.pool.size() < 2 * i + 2) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      h->prof.pool.push_back(e);
    }
    h->prof.cls.push_back(c);
    cudaEventRecord(h->prof.pool[2 * i], s);
  }
  ~ProfScope() {
    if (!h->prof.on) return;
    cudaEventRecord(h->prof.pool[2 * (h->prof.cls.size() - 1) + 1], s);
  }
};

// Add the recorded pairs into the per-class totals (the stream must be idle).
void prof_collect(npsolve *h) {
  if (!h->prof.on) return;
  for (size_t i = 0; i < h->prof.cls.size(); ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->prof.pool[2 * i], h->prof.pool[2 * i + 1]) == cudaSuccess) {
      h->prof.ms[h->prof.cls[i]] += ms;
      h->prof.launches[h->prof.cls[i]] += 1;
    }
  }
  h->prof.cls.clear();
}

// cudaMalloc of `count` elements (+256 bytes of slack), adding the bytes to
// *counter (the workspace's footprint, used for HBM-budget admission).
template <class T>
cudaError_t dalloc(size_t *counter, T **p, size_t count) {
  const size_t bytes = count * sizeof(T) + 256;
  const cudaError_t e = cudaMalloc((void **)p, bytes);
  if (e == cudaSuccess && counter) *counter += bytes;
  return e;
}

void free_ws(Workspace &w) {
  if (w.graph) cudaGraphExecDestroy(w.graph);
  w.graph = nullptr;
  cudaFree(w.r);
  cudaFree(w.z);
  cudaFree(w.xhi);
  cudaFree(w.xlo);
  cudaFree(w.r_alt);
  cudaFree(w.lapcode);
  cudaFree(w.gmask);
  cudaFree(w.dring);
  cudaFree(w.qring);
  for (int l = 0; l <= kMaxLevels; ++l) {
    cudaFree(w.x1[l]);
    cudaFree(w.r1[l]);
    cudaFree(w.r2[l]);
    cudaFree(w.x2[l]);
    cudaFree(w.xc[l]);
    cudaFree(w.counts[l]);
    cudaFree(w.kdesc[l]);
  }
  for (int i = 0; i < (kMaxLevels + 1) * 2; ++i) cudaFree(w.kcache[i]);
  cudaFree(w.tailk);
  cudaFree(w.ktotal);
  cudaFreeHost(w.h_ktotal);
  cudaFree(w.kskip);
  cudaFreeHost(w.h_kskip);
  cudaFree(w.kmcount);
  cudaFreeHost(w.h_kmcount);
  cudaFree(w.ulist);
  cudaFreeHost(w.h_ulist);
  cudaFree(w.ineed);
  cudaFree(w.kskip2);
  cudaFreeHost(w.h_kskip2);
  cudaFree(w.ulist2);
  cudaFreeHost(w.h_ulist2);
  cudaFree(w.part);
  cudaFree(w.affc);
  cudaFree(w.affs);
  cudaFree(w.relres);
  cudaFree(w.hist);
  cudaFree(w.st);
  cudaFree(w.tickets);
  cudaFree(w.pcg_st);
  cudaFree(w.bad);
  cudaFree(w.reopened);
  cudaFreeHost(w.h_st);
  cudaFreeHost(w.h_flag);
  for (int i = 0; i < 2; ++i)
    if (w.ev[i]) cudaEventDestroy(w.ev[i]);
  cudaFree(w.stage_lab);
  cudaFree(w.stage_b);
  cudaFree(w.stage_x);
  w = Workspace{};
}

Dims level_dims(Dims d, int lvl) { return Dims{d.nx >> (lvl - 1), d.ny >> (lvl - 1), d.nz >> (lvl - 1)}; }

// Make sure the workspace holds buffers for a grid of dims (L levels).
int ensure_ws(npsolve *h, Dims d, int hist_cap) {
  Workspace &w = h->ws;
  const int L = h->cfg.levels;
  const long long n = d.n();
  bool fits = w.r && n <= w.cap;
  if (fits) {
    // per-level sizes must fit too (they do when n <= cap only for the same shape family;
    // re-allocate when any level would overflow)
    long long cap_l = w.cap;
    for (int l = 1; l <= L; ++l, cap_l /= 8) {
      const long long nl = (long long)(d.nx >> (l - 1)) * (d.ny >> (l - 1)) * (d.nz >> (l - 1));
      if (nl > cap_l) fits = false;
    }
  }
  if (!fits) {
    free_ws(w);
    const long long cap = n;
    const int R = kRing;
    CK(h, dalloc(&w.bytes, &w.r, cap));
    CK(h, dalloc(&w.bytes, &w.z, cap));
    CK(h, dalloc(&w.bytes, &w.xhi, cap));
    CK(h, dalloc(&w.bytes, &w.xlo, cap));
    CK(h, dalloc(&w.bytes, &w.r_alt, cap));
    CK(h, dalloc(&w.bytes, &w.lapcode, cap));
    CK(h, dalloc(&w.bytes, &w.gmask, cap / 128 + 64));
    CK(h, dalloc(&w.bytes, &w.dring, cap * R));
    CK(h, dalloc(&w.bytes, &w.qring, cap * R));
    long long cl = cap;
    for (int l = 1; l <= L; ++l, cl = (cl + 7) / 8) {
      CK(h, dalloc(&w.bytes, &w.x1[l], cl));
      if (l >= 2) {
        CK(h, dalloc(&w.bytes, &w.r1[l], cl));
        CK(h, dalloc(&w.bytes, &w.counts[l], cl));
      }
      if (l < L) {
        CK(h, dalloc(&w.bytes, &w.r2[l], cl));
        CK(h, dalloc(&w.bytes, &w.x2[l], cl));
        if (l >= 2) CK(h, dalloc(&w.bytes, &w.xc[l], cl));
      }
    }
    // reduction partials: per block of the reduction kernels, or per (unit, warp) of the fused CConv
    w.part_cap = (size_t)kRedMaxBlocks * kMaxPartials + (size_t)(cap / 64) + 64;
    CK(h, dalloc(&w.bytes, &w.part, w.part_cap));
    CK(h, dalloc(&w.bytes, &w.affc, (size_t)(kMaxLevels + 1) * 2));
  CK(h, dalloc(&w.bytes, &w.affs, (size_t)(kMaxLevels + 1) * 54));
    CK(h, dalloc(&w.bytes, &w.relres, 2));
    CK(h, dalloc(&w.bytes, &w.st, 1));
    CK(h, dalloc(&w.bytes, &w.tickets, 8));
    CK(h, dalloc(&w.bytes, &w.ktotal, 2 * (kMaxLevels + 1)));
    CK(h, cudaHostAlloc((void **)&w.h_ktotal, sizeof(unsigned) * 2 * (kMaxLevels + 1), cudaHostAllocDefault));
    CK(h, cudaMemset(w.tickets, 0, 8 * sizeof(unsigned)));
    CK(h, cudaMalloc(&w.pcg_st, pcg_state_bytes()));
    CK(h, dalloc(&w.bytes, &w.bad, 1));
    CK(h, dalloc(&w.bytes, &w.reopened, 1));
    CK(h, cudaHostAlloc((void **)&w.h_st, sizeof(SolveState) * 2, cudaHostAllocDefault));
    CK(h, cudaHostAlloc((void **)&w.h_flag, sizeof(int) * 8, cudaHostAllocDefault));
    for (int i = 0; i < 2; ++i) CK(h, cudaEventCreateWithFlags(&w.ev[i], cudaEventDisableTiming));
    w.cap = cap;
  }
  if (hist_cap > w.hist_cap) {
    if (w.graph) cudaGraphExecDestroy(w.graph);  // the graph refers to the old history buffer
    w.graph = nullptr;
    if (w.hist) w.bytes -= (size_t)w.hist_cap * sizeof(double) + 256;
    cudaFree(w.hist);
    w.hist = nullptr;
    CK(h, dalloc(&w.bytes, &w.hist, (size_t)hist_cap));
    w.hist_cap = hist_cap;
  }
  w.dims = d;
  return NPSOLVE_OK;
}

// Round to the nearest BF16 value (ties to even), kept as FP32.
float bf16_round_host(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) != 0x7F800000u) u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
  memcpy(&f, &u, 4);
  return f;
}

// Fold the blob into the device form of every CConv / Aff block (Sec. 4.2.1
// with the channel-sum-to-one identity; see CConvW / AffW).
int upload_weights(npsolve *h) {
  const int L = h->cfg.levels;
  const float *w = h->weights.data();
  std::vector<CConvW> cw((kMaxLevels + 1) * 2);
  std::vector<AffW> aw((kMaxLevels + 1) * 2);
  memset(cw.data(), 0, cw.size() * sizeof(CConvW));
  memset(aw.data(), 0, aw.size() * sizeof(AffW));
  const size_t per = 2 * kCConvParams + 2 * kAffParams;
  auto fold_conv = [&](const float *blk, int lvl, CConvW &o) {
    const double scale = 1.0 / pow(8.0, lvl - 1);
    for (int a = 0; a < 27; ++a) {
      double bp = blk[2187 + a];
      for (int l = 0; l < 27; ++l) {
        const double wf = blk[(a * 3 + 0) * 27 + l], wa = blk[(a * 3 + 1) * 27 + l], ws = blk[(a * 3 + 2) * 27 + l];
        o.wf[a][l] = (float)((wf - ws) * scale);
        o.wa[a][l] = (float)((wa - ws) * scale);
        bp += ws;
      }
      o.bp[a] = (float)bp;
    }
  };
  auto fold_aff = [&](const float *blk, int lvl, AffW &o) {
    const double scale = 1.0 / pow(8.0, lvl - 1);
    double bc = blk[81];
    for (int l = 0; l < 27; ++l) {
      const double wf = blk[l], wa = blk[27 + l], ws = blk[54 + l];
      o.wf[l] = (float)((wf - ws) * scale);
      o.wa[l] = (float)((wa - ws) * scale);
      bc += ws / 27.0;
    }
    o.bconst = bc;
  };
  for (int lvl = 1; lvl <= L; ++lvl) {
    const float *base = w + (size_t)(lvl - 1) * per;
    fold_conv(base, lvl, cw[lvl * 2 + 0]);
    if (lvl < L) {
      fold_conv(base + kCConvParams, lvl, cw[lvl * 2 + 1]);
      fold_aff(base + 2 * kCConvParams, lvl, aw[lvl * 2 + 0]);
      fold_aff(base + 2 * kCConvParams + kAffParams, lvl, aw[lvl * 2 + 1]);
    }
  }
  if (h->cfg.precision == NPSOLVE_BF16) {
    // the BF16 form: every folded CConv weight rounded to BF16 (nearest even)
    auto rnd = bf16_round_host;
    for (auto &c : cw) {
      for (int a = 0; a < 27; ++a) {
        for (int l = 0; l < 27; ++l) {
          c.wf[a][l] = rnd(c.wf[a][l]);
          c.wa[a][l] = rnd(c.wa[a][l]);
        }
        c.bp[a] = rnd(c.bp[a]);
      }
    }
  }
  {
    const int wb = umma_weight_bytes(3);
    std::vector<uint8_t> uw((size_t)(kMaxLevels + 1) * 2 * wb, 0);
    for (int i = 0; i < (kMaxLevels + 1) * 2; ++i) prepare_umma_weights(cw[i], h->nsplit, uw.data() + (size_t)i * wb);
    CK(h, cudaMemcpy(h->uw, uw.data(), uw.size(), cudaMemcpyHostToDevice));
  }
  {
    // uniform-window kernels K_a = Bp[a] + nF SWf[a] + nA SWa[a] (row sums in FP64)
    std::vector<float> uni((size_t)(kMaxLevels + 1) * 2 * 81, 0.f);
    for (int i = 0; i < (kMaxLevels + 1) * 2; ++i)
      for (int a = 0; a < 27; ++a) {
        double sf = 0.0, sa = 0.0;
        for (int l = 0; l < 27; ++l) {
          sf += cw[i].wf[a][l];
          sa += cw[i].wa[a][l];
        }
        uni[(size_t)i * 81 + a] = cw[i].bp[a];
        uni[(size_t)i * 81 + 27 + a] = (float)sf;
        uni[(size_t)i * 81 + 54 + a] = (float)sa;
      }
    CK(h, cudaMemcpy(h->uni, uni.data(), uni.size() * sizeof(float), cudaMemcpyHostToDevice));
    h->uni_host = uni;
    // kernels of the pure windows of level lvl (F = 8^(lvl-1) fine cells per cell):
    // K^S = Bp, K^F = Bp + F SWf, K^A = Bp + F SWa
    std::vector<float> kfix((size_t)(kMaxLevels + 1) * 2 * 81, 0.f);
    for (int i = 2; i < (kMaxLevels + 1) * 2; ++i) {
      const double F = pow(8.0, i / 2 - 1);
      for (int a = 0; a < 27; ++a) {
        double sf = 0.0, sa = 0.0;
        for (int l = 0; l < 27; ++l) {
          sf += cw[i].wf[a][l];
          sa += cw[i].wa[a][l];
        }
        kfix[(size_t)i * 81 + a] = cw[i].bp[a];
        kfix[(size_t)i * 81 + 27 + a] = (float)((double)cw[i].bp[a] + F * sf);
        kfix[(size_t)i * 81 + 54 + a] = (float)((double)cw[i].bp[a] + F * sa);
      }
    }
    if (h->cfg.precision == NPSOLVE_BF16)  // the BF16 form rounds every kernel value, these included
      for (float &f : kfix) f = bf16_round_host(f);
    h->kfix_host = kfix;
  }
  CK(h, cudaMemcpy(h->cw, cw.data(), cw.size() * sizeof(CConvW), cudaMemcpyHostToDevice));
  h->cw_host = cw;
  CK(h, cudaMemcpy(h->aw, aw.data(), aw.size() * sizeof(AffW), cudaMemcpyHostToDevice));
  return NPSOLVE_OK;
}


int check_dims(npsolve *h, int nx, int ny, int nz) {
  if (nx < 1 || ny < 1 || nz < 1 || nx > 4096 || ny > 4096 || nz > 4096)
    return fail(h, NPSOLVE_BAD_DIMS, "dims %dx%dx%d out of range", nx, ny, nz);
  if ((long long)nx * ny * nz > (1LL << 31) - 1) return fail(h, NPSOLVE_BAD_DIMS, "grid too large");
  const int m = 1 << (h->cfg.levels - 1);
  if (nx % m || ny % m || nz % m)
    return fail(h, NPSOLVE_BAD_DIMS, "dims %dx%dx%d not divisible by 2^(L-1) = %d", nx, ny, nz, m);
  return NPSOLVE_OK;
}

// Levels whose CConv runs on the tensor cores in the per-iteration
// recompute path (image counts <= 64 are exact in BF16 up to level 3).
bool tensor_level(const npsolve *h, int lvl) { return h->cfg.kernel_path == NPSOLVE_PATH_TENSOR && lvl <= 3; }
// The cached path streams vector planes with TMA boxes, whose rows must be a
// multiple of 16 bytes.  The decision is per level: a level whose rows are not
// (a coarse level of a small or odd-sized grid, e.g. the 2^3 or 6^3 level of a
// 6-level network on 64^3 or 192^3) runs on the CUDA-core kernels with a
// separate pooling / combination, the other levels stay on the cached path.
bool stream_shape_level(const npsolve *h, Dims d1, int l) {
  return h->cfg.kernel_path == NPSOLVE_PATH_CACHED && l <= h->cfg.levels && stream_shape_ok(level_dims(d1, l));
}
// Level 1 on the cached path (the level-1 fusions, unit lists and setup).
bool cached_path(const npsolve *h, Dims d1) { return stream_shape_level(h, d1, 1); }
// The first level of the coarse tail (kernels_tail.cu) for this grid, 0 for
// none: on the cached path, the first level from 2 on with at most
// kTailMaxCells cells.  The levels from there on run in one cluster launch
// inside solves and network evaluations, on their own materialised kernels.
int tail_level(const npsolve *h, Dims d1) {
  if (!cached_path(h, d1) || h->cfg.symmetric) return 0;
  for (int l = 2; l <= h->cfg.levels; ++l)
    if (level_dims(d1, l).n() <= kTailMaxCells) return l;
  return 0;
}
// A level on the streamed cached kernels (not in the tail).
bool stream_level(const npsolve *h, Dims d1, int l) {
  const int T = tail_level(h, d1);
  return stream_shape_level(h, d1, l) && !(T && l >= T);
}

// The recurrence step r_{k+1} = r_k - alpha q of an iteration is formed by the
// next iteration's level-1 CConv1 (two residual buffers, r_k in buffer k mod
// 2) on the multilevel, 16-byte-vector, cached path.
bool fused_update(const npsolve *h, Dims d1) {
  return h->cfg.levels > 1 && !h->cfg.symmetric && d1.nx % 4 == 0 && d1.n() <= (long long)INT32_MAX &&
         h->cfg.residual_mode == NPSOLVE_RESIDUAL_RECURRENCE && cached_path(h, d1);
}

// One CConv block of level lvl (type 1 or 2), CUDA-core kernel.
void cconv(npsolve *h, const uint8_t *lab, Dims d1, int lvl, int type, const float *in, const float *vscale,
           int mask_input, float *out, const SolveState *st, cudaStream_t s) {
  Workspace &w = h->ws;
  const Dims dl = level_dims(d1, lvl);
  const int idx = lvl * 2 + (type - 1);
  ProfScope ps(h, lvl == 1 ? P_CCONV_L1 : P_CCONV_COARSE, s);
  h->launches += 1;
  if (h->tr.kstore) {  // training forward: no input scale, no solve state
    const uint8_t *ll = lvl == 1 ? lab : nullptr;
    const ushort2 *lc = lvl == 1 ? nullptr : w.counts[lvl];
    const float *kpure = h->kfix_host.data() + (size_t)idx * 81;
    const float full = (float)ldexp(1.0, 3 * (lvl - 1));
    const int rk = h->cfg.precision == NPSOLVE_BF16 ? 1 : 0;
    if (lvl <= 3 && dl.nx % 32 == 0)  // counts exact in BF16, rows of whole warps: the tensor cores
      launch_cconv_store_K_tc(ll, lc, dl, h->uw + (size_t)idx * umma_weight_bytes(3), h->nsplit, kpure, full, in,
                              mask_input, rk, h->tr.kslot[idx], out, h->umma_err, h->num_sms, s);
    else
      launch_cconv_store_K(ll, lc, dl, h->cw_host[idx], kpure, full, in, mask_input, rk, h->tr.kslot[idx], out, s);
    return;
  }
  launch_cconv_f32(lvl == 1 ? lab : nullptr, lvl == 1 ? nullptr : w.counts[lvl], dl, h->cw + idx, in, vscale,
                   mask_input, h->cfg.precision == NPSOLVE_BF16 ? 1 : 0, out, st, s);
}

// One CConv block on the tensor cores (z-marching kernel), with the input
// either read (in) or interpolated from the coarser level (coarse), and an
// optional fused 2x2x2 pooling of the output into `pooled`.
void cconv_tc(npsolve *h, const uint8_t *lab, Dims d1, int lvl, int type, const float *in, const float *coarse,
              const float *vscale, int mask_input, float *out, float *pooled, const SolveState *st,
              cudaStream_t s) {
  Workspace &w = h->ws;
  const int idx = lvl * 2 + (type - 1);
  ProfScope ps(h, lvl == 1 ? P_CCONV_L1 : P_CCONV_COARSE, s);
  h->launches += 1;
  launch_cconv_march(h->nsplit, lvl == 1 ? lab : nullptr, lvl == 1 ? nullptr : w.counts[lvl], level_dims(d1, lvl),
                     h->uw + (size_t)idx * umma_weight_bytes(3), in, coarse, vscale, mask_input, out, pooled, st,
                     h->umma_err, h->num_sms, s);
}

// One CConv block with the per-solve kernel cache (kernels_cached.cu): input
// read (in) or interpolated (coarse), optional fused pooling, optional fused
// combination out = c1 x1 + c2 CConv(...).
void cconv_cached(npsolve *h, Dims d1, int lvl, int type, const float *in, const float *vscale, float *out,
                  float *pooled, const float *x1, const double *c12, const SolveState *st, cudaStream_t s,
                  int mode = STREAM_MODE_ALL, const StreamFusion *fuse = nullptr, const StreamUpdate *upd = nullptr,
                  const StreamUnits *units = nullptr) {
  Workspace &w = h->ws;
  const int idx = lvl * 2 + (type - 1);
  ProfScope ps(h, lvl == 1 ? P_CCONV_L1 : P_CCONV_COARSE, s);
  h->launches += 1;
  if (launch_cconv_stream(h->cfg.precision == NPSOLVE_BF16, level_dims(d1, lvl), h->kfix_host.data() + (size_t)idx * 81,
                          w.kdesc[lvl], w.kcache[idx], in, vscale, out, pooled, x1, c12, mode, st, h->umma_err,
                          h->num_sms, s, fuse, upd, units))
    h->stream_err = true;
}

// Grids with nx % 4 == 0 use the 16-byte vector kernels with fused
// last-block reductions (kernels_vec4.cu).
bool vec4_path(Dims d) { return d.nx % 4 == 0 && d.n() <= (long long)INT32_MAX; }
enum { kTicketInit = 0, kTicketCombine = 1, kTicketLap = 2, kTicketUpdate = 3 };

// The network z = P_net(I, r) of Alg. 2 on the prepared pyramid and Aff
// coefficients.  Inside a solve (st != null) the level-1 input is scaled by
// 1/||r|| from the state and the orthogonalisation dots are fused into the
// last combination.  `unfused` materialises every intermediate (r2, x2) for
// the per-level inspection entry point.
void run_network(npsolve *h, const uint8_t *lab, Dims d1, const float *r, const float *vscale, float *z,
                 SolveState *st, cudaStream_t s, bool unfused = false, bool dots = true) {
  // dots = false inside a solve: z is not the preconditioned vector itself (the
  // symmetric variant applies the transpose to it), so no dots are taken here
  Workspace &w = h->ws;
  const int L = h->cfg.levels;
  const bool cached = cached_path(h, d1);  // level 1
  if (cached && !st) {
    // the cached stencil expects an input that is zero off fluid: inside a solve
    // r is, for a user-supplied vector zero it here
    h->launches += 1;
    launch_mask_copy(lab, d1.n(), r, w.r, s);
    r = w.r;
  }
  // inside a solve the level-1 CConvs process only the units with work (the
  // rest of z, the pooled input of level 2 and the second residual buffer
  // were zeroed once for the solve)
  const bool lists = st && cached && w.ulist_ok;
  const StreamUnits u1{w.ulist, w.un[0], w.uzc[0]}, u2{w.ulist + w.kskip_cap, w.un[1], w.uzc[1]};
  const StreamUnits *pu1 = lists ? &u1 : nullptr, *pu2 = lists ? &u2 : nullptr;
  const StreamUnits ul2{w.ulist2, w.un2, w.uzc2};
  const StreamUnits *pl2 = lists && w.ulist2_ok ? &ul2 : nullptr;  // level 2 (L >= 3)
  const uint8_t *skip1 = lists ? w.ineed : nullptr;                // what the level-1 CConv2 does not read of r2
  // levels T..L in one cluster launch (kernels_tail.cu), which also writes the
  // interpolated input r2^(T-1) of the finer level's CConv2; not for the
  // per-level inspection (it keeps no x2)
  const int T = (!unfused && w.tail_T && w.tail_T == tail_level(h, d1)) ? w.tail_T : 0;
  // down pass: x1^l = CConv1^l(r1^l), r1^{l+1} = Pool(x1^l)
  for (int l = 1; l < (T ? T : L); ++l) {
    const float *in = l == 1 ? r : w.r1[l];
    const float *vs = l == 1 ? vscale : nullptr;
    if (cached && l == 1 && st && fused_update(h, d1)) {
      // the pending residual step first (r_k from buffer k mod 2, in = w.r is buffer 0)
      const StreamUpdate up{{w.r, w.r_alt}, w.qring, kRing, w.part, w.part_cap, w.tickets + kTicketUpdate, w.hist, st};
      cconv_cached(h, d1, l, 1, w.r, vs, w.x1[l], w.r1[l + 1], nullptr, nullptr, st, s, STREAM_MODE_ZERO_PURE,
                   nullptr, &up, pu1);
    } else if (stream_level(h, d1, l)) {
      cconv_cached(h, d1, l, 1, in, vs, w.x1[l], w.r1[l + 1], nullptr, nullptr, st, s,
                   l == 1 ? STREAM_MODE_ZERO_PURE : STREAM_MODE_ALL, nullptr, nullptr,
                   l == 1 ? pu1 : (l == 2 ? pl2 : nullptr));
    } else if (tensor_level(h, l)) {
      cconv_tc(h, lab, d1, l, 1, in, nullptr, vs, l == 1, w.x1[l], w.r1[l + 1], st, s);
    } else {
      cconv(h, lab, d1, l, 1, in, vs, l == 1, w.x1[l], st, s);
      ProfScope ps(h, P_POOL, s);
      h->launches += 1;
      launch_pool(w.x1[l], level_dims(d1, l), w.r1[l + 1], st, s);
    }
  }
  if (T) {
    TailParams tp{};
    tp.T = T;
    tp.L = L;
    for (int l = 1; l <= L; ++l) {
      tp.dims[l] = level_dims(d1, l);
      tp.k1[l] = w.tk1[l];
      tp.k2[l] = w.tk2[l];
      tp.x1[l] = w.x1[l];
      tp.r1[l] = w.r1[l];
      tp.r2[l] = w.r2[l];
      tp.xc[l] = w.xc[l];
    }
    tp.affc = w.affc;
    tp.st = st;
    ProfScope ps(h, P_CCONV_COARSE, s);
    h->launches += 1;
    if (launch_tail(tp, s)) h->stream_err = true;
  }
  // coarsest level: x^L = CConv1^L(r1^L)
  if (!T) {
    const float *in = L == 1 ? r : w.r1[L];
    const float *vs = L == 1 ? vscale : nullptr;
    if (stream_level(h, d1, L))
      cconv_cached(h, d1, L, 1, in, vs, w.x1[L], nullptr, nullptr, nullptr, st, s,
                   L == 1 ? STREAM_MODE_ZERO_PURE : STREAM_MODE_ALL);
    else if (tensor_level(h, L)) cconv_tc(h, lab, d1, L, 1, in, nullptr, vs, L == 1, w.x1[L], nullptr, st, s);
    else cconv(h, lab, d1, L, 1, in, vs, L == 1, w.x1[L], st, s);
  }
  if (L == 1) {
    ProfScope ps(h, P_COMBINE, s);
    h->launches += 1;
    launch_combine1(lab, d1.n(), w.x1[1], w.x1[1], h->unit_c12, z, w.qring, w.r, w.part, dots ? st : nullptr, s);
    return;
  }
  // up pass: r2^l = Interp(x^{l+1}); x2^l = CConv2^l(r2^l); x^l = c1 x1^l + c2 x2^l
  for (int l = (T ? T - 1 : L - 1); l >= 1; --l) {
    const float *coarse = (l + 1 == L) ? w.x1[L] : w.xc[l + 1];
    const double *c12 = w.affc + 2 * l;
    const bool cached_l = stream_level(h, d1, l);
    const bool interp_done = T && l == T - 1;  // the tail wrote r2^(T-1)
    if (cached_l && !unfused) {
      if (!interp_done) {
        ProfScope ps(h, P_INTERP, s);
        h->launches += 1;
        launch_interp(coarse, level_dims(d1, l + 1), w.r2[l], st, s, l == 1 ? skip1 : nullptr);
      }
      if (l > 1) {  // CConv2 and the combination in one pass
        cconv_cached(h, d1, l, 2, w.r2[l], nullptr, w.xc[l], nullptr, w.x1[l], c12, st, s, STREAM_MODE_ALL, nullptr,
                     nullptr, l == 2 ? pl2 : nullptr);
        continue;
      }
      if (st && dots && vec4_path(d1) && stream_fusion_ok(h->cfg.n_ortho)) {
        // level-1 CConv2, z = mask_fluid(c1 x1 + c2 x2) and the orthogonalisation dots in one pass
        const StreamFusion fu{w.qring,   kRing,     {w.r, fused_update(h, d1) ? w.r_alt : nullptr},
                              h->cfg.method, w.part,  w.part_cap, w.tickets + kTicketCombine,
                              st};
        cconv_cached(h, d1, 1, 2, w.r2[1], nullptr, z, nullptr, w.x1[1], c12, st, s, STREAM_MODE_FLUID_ONLY, &fu,
                     nullptr, pu2);
        continue;
      }
      // level 1: only the fluid cells of x2 enter z (the output restriction)
      cconv_cached(h, d1, l, 2, w.r2[l], nullptr, w.x2[l], nullptr, nullptr, nullptr, st, s,
                   STREAM_MODE_FLUID_ONLY, nullptr, nullptr, pu2);
    } else if (tensor_level(h, l) && !unfused) {
      cconv_tc(h, lab, d1, l, 2, nullptr, coarse, nullptr, 0, w.x2[l], nullptr, st, s);
    } else {
      if (!interp_done) {
        ProfScope ps(h, P_INTERP, s);
        h->launches += 1;
        launch_interp(coarse, level_dims(d1, l + 1), w.r2[l], st, s);
      }
      if (cached_l) cconv_cached(h, d1, l, 2, w.r2[l], nullptr, w.x2[l], nullptr, nullptr, nullptr, st, s);
      else if (tensor_level(h, l))
        cconv_tc(h, lab, d1, l, 2, w.r2[l], nullptr, nullptr, 0, w.x2[l], nullptr, st, s);
      else cconv(h, lab, d1, l, 2, w.r2[l], nullptr, 0, w.x2[l], st, s);
    }
    ProfScope ps(h, P_COMBINE, s);
    h->launches += 1;
    if (l > 1) launch_combine(level_dims(d1, l).n(), w.x1[l], w.x2[l], c12, w.xc[l], st, s);
    else if (st && dots && vec4_path(d1))  // fused: dots and orthogonalisation coefficients in one launch
      launch_combine1_4(lab, (int)d1.n(), w.x1[1], w.x2[1], c12, z, w.qring, w.r,
                        fused_update(h, d1) ? w.r_alt : nullptr, w.part, w.tickets + kTicketCombine, st, h->num_sms,
                        s);
    else launch_combine1(lab, d1.n(), w.x1[1], w.x2[1], c12, z, w.qring, w.r, w.part, dots ? st : nullptr, s);
  }
}

// Label check, pyramid and Aff coefficients for this grid; for the cached
// path also the classification of every level and the kernel generation of
// the mixed-window cells (one host synchronisation to size the cache).
int setup_image(npsolve *h, const uint8_t *lab, Dims d1, cudaStream_t s, bool check) {
  Workspace &w = h->ws;
  const int L = h->cfg.levels;
  if (check) {
    CK(h, cudaMemsetAsync(w.bad, 0, sizeof(unsigned int), s));
    launch_check_labels(lab, d1.n(), w.bad, s);
  }
  launch_pyramid(lab, d1, w.counts, L, s);
  if (vec4_path(d1)) {
    launch_lap_codes(lab, d1, w.lapcode, w.gmask, s);
    h->launches += 2;
  }
  {
    AffAll aa{};
    aa.lab = lab;
    for (int l = 1; l <= L; ++l) {
      aa.counts[l] = l == 1 ? nullptr : w.counts[l];
      aa.dims[l] = level_dims(d1, l);
    }
    aa.aw = h->aw;
    aa.out = w.affc;
    aa.stats = w.affs;
    aa.cnt = (unsigned long long *)w.part;  // 128 L counters of the reduction scratch
    aa.L = L;
    launch_aff_all(aa, s);
  }
  h->launches += 1 + (L - 1) + (L > 1 ? 2 : 0);
  w.tail_T = tail_level(h, d1);
  if (w.tail_T) {
    // the coarse tail's per-cell kernels: CConv1 of levels T..L, CConv2 of T..L-1
    size_t need = 0;
    for (int l = w.tail_T; l <= L; ++l) need += (size_t)27 * level_dims(d1, l).n() * (l < L ? 2 : 1);
    if (need > w.tailk_cap) {
      if (w.graph) cudaGraphExecDestroy(w.graph);  // the graph refers to the old buffer
      w.graph = nullptr;
      CK(h, cudaStreamSynchronize(s));
      if (w.tailk) w.bytes -= w.tailk_cap * sizeof(float) + 256;
      cudaFree(w.tailk);
      w.tailk = nullptr;
      w.tailk_cap = 0;
      CK(h, dalloc(&w.bytes, &w.tailk, need));
      w.tailk_cap = need;
    }
    float *kp = w.tailk;
    const int rk = h->cfg.precision == NPSOLVE_BF16 ? 1 : 0;
    for (int l = w.tail_T; l <= L; ++l) {
      const Dims dl = level_dims(d1, l);
      for (int t = 0; t < (l < L ? 2 : 1); ++t) {
        (t ? w.tk2 : w.tk1)[l] = kp;
        launch_tail_kernels(nullptr, w.counts[l], dl, h->cw + l * 2 + t, rk, kp, s);
        h->launches += 1;
        kp += (size_t)27 * dl.n();
      }
    }
  }
  if (cached_path(h, d1)) {
    const bool bf16 = h->cfg.precision == NPSOLVE_BF16;
    for (int l = 1; l <= L; ++l) {  // plane descriptors sized for this grid's shape
      if (!stream_level(h, d1, l)) continue;
      const long long nd = stream_desc_count(level_dims(d1, l));
      if (nd > w.kdesc_cap[l]) {
        if (w.graph) cudaGraphExecDestroy(w.graph);  // the graph refers to the old buffers
        w.graph = nullptr;
        CK(h, cudaStreamSynchronize(s));
        if (w.kdesc[l]) w.bytes -= (size_t)w.kdesc_cap[l] * stream_desc_bytes() + 256;
        cudaFree(w.kdesc[l]);
        w.kdesc[l] = nullptr;
        CK(h, dalloc(&w.bytes, &w.kdesc[l], (size_t)nd * stream_desc_bytes()));
        w.kdesc_cap[l] = nd;
      }
    }
    const long long nsk = stream_desc_count(d1);  // level-1 (tile, plane) pairs
    if (nsk > w.kskip_cap) {
      if (w.graph) cudaGraphExecDestroy(w.graph);  // the graph refers to the old lists
      w.graph = nullptr;
      CK(h, cudaStreamSynchronize(s));
      cudaFree(w.kskip);
      cudaFreeHost(w.h_kskip);
      cudaFree(w.ulist);
      cudaFreeHost(w.h_ulist);
      w.kskip = nullptr;
      w.h_kskip = nullptr;
      w.ulist = nullptr;
      w.h_ulist = nullptr;
      w.kskip_cap = 0;
      cudaFree(w.ineed);
      w.ineed = nullptr;
      cudaFree(w.kmcount);
      cudaFreeHost(w.h_kmcount);
      w.kmcount = nullptr;
      w.h_kmcount = nullptr;
      CK(h, cudaMalloc(&w.kmcount, sizeof(uint16_t) * (size_t)nsk));
      CK(h, cudaHostAlloc((void **)&w.h_kmcount, sizeof(uint16_t) * (size_t)nsk, cudaHostAllocDefault));
      CK(h, cudaMalloc(&w.kskip, (size_t)nsk));
      CK(h, cudaHostAlloc((void **)&w.h_kskip, 2 * (size_t)nsk, cudaHostAllocDefault));
      CK(h, cudaMalloc(&w.ulist, sizeof(int) * 2 * (size_t)nsk));
      CK(h, cudaHostAlloc((void **)&w.h_ulist, sizeof(int) * 2 * (size_t)nsk, cudaHostAllocDefault));
      CK(h, cudaMalloc(&w.ineed, (size_t)nsk));
      w.kskip_cap = nsk;
    }
    const bool lv2 = L >= 3 && stream_level(h, d1, 2);  // level 2 has a CConv1 and a CConv2
    const long long nsk2 = lv2 ? stream_desc_count(level_dims(d1, 2)) : 0;
    if (nsk2 > w.kskip2_cap) {
      if (w.graph) cudaGraphExecDestroy(w.graph);
      w.graph = nullptr;
      CK(h, cudaStreamSynchronize(s));
      cudaFree(w.kskip2);
      cudaFreeHost(w.h_kskip2);
      cudaFree(w.ulist2);
      cudaFreeHost(w.h_ulist2);
      w.kskip2 = nullptr;
      w.h_kskip2 = nullptr;
      w.ulist2 = nullptr;
      w.h_ulist2 = nullptr;
      w.kskip2_cap = 0;
      CK(h, cudaMalloc(&w.kskip2, 2 * (size_t)nsk2));
      CK(h, cudaHostAlloc((void **)&w.h_kskip2, (size_t)nsk2, cudaHostAllocDefault));
      CK(h, cudaMalloc(&w.ulist2, sizeof(int) * (size_t)nsk2));
      CK(h, cudaHostAlloc((void **)&w.h_ulist2, sizeof(int) * (size_t)nsk2, cudaHostAllocDefault));
      w.kskip2_cap = nsk2;
    }
    CK(h, cudaMemsetAsync(w.ktotal, 0, sizeof(unsigned) * 2 * (kMaxLevels + 1), s));
    for (int l = 1; l <= L; ++l) {
      if (!stream_level(h, d1, l)) continue;
      launch_classify(l == 1 ? lab : nullptr, l == 1 ? nullptr : w.counts[l], level_dims(d1, l),
                      1u << (3 * (l - 1)), w.kdesc[l], w.ktotal + 2 * l,
                      l == 1 ? w.kskip : (l == 2 && lv2 ? w.kskip2 : nullptr), l == 1 ? w.kmcount : nullptr,
                      h->num_sms, s);
      h->launches += 1;
    }
    CK(h, cudaMemcpyAsync(w.h_ktotal, w.ktotal, sizeof(unsigned) * 2 * (kMaxLevels + 1), cudaMemcpyDeviceToHost, s));
    CK(h, cudaMemcpyAsync(w.h_kskip + nsk, w.kskip, (size_t)nsk, cudaMemcpyDeviceToHost, s));
    CK(h, cudaMemcpyAsync(w.h_kmcount, w.kmcount, sizeof(uint16_t) * (size_t)nsk, cudaMemcpyDeviceToHost, s));
    // level-1 (tile, plane) pairs with no fluid within one tile or plane (1 = skip): the level-1 CConv1
    // output is exactly zero there (a window without fluid sees a zero input), and the level-1 CConv2 reads
    // nothing of the level-2 -> 1 interpolation there (its units hold fluid; their halo is one cell)
    launch_dilate_flags(w.kskip, d1, 2, 1, 1, 1, true, w.ineed, s);
    h->launches += 1;
    CK(h, cudaMemcpyAsync(w.h_kskip, w.ineed, (size_t)nsk, cudaMemcpyDeviceToHost, s));
    if (lv2) {
      // level 2: the units within two coarse cells (one tile across, two planes along z) of a cell with
      // fluid; elsewhere both level-2 CConv outputs are zero or never read (1 = may be skipped)
      launch_dilate_flags(w.kskip2, level_dims(d1, 2), 2, 1, 1, 2, true, w.kskip2 + nsk2, s);
      h->launches += 1;
      CK(h, cudaMemcpyAsync(w.h_kskip2, w.kskip2 + nsk2, (size_t)nsk2, cudaMemcpyDeviceToHost, s));
    }
    CK(h, cudaStreamSynchronize(s));
    for (int l = 1; l <= L; ++l) {
      if (!stream_level(h, d1, l)) continue;
      const int nblk = l < L ? 2 : 1;
      for (int t = 0; t < nblk; ++t) {
        const int idx = l * 2 + t;
        const size_t need = (size_t)w.h_ktotal[2 * l] + 4;
        if (need > w.kcap[idx]) {
          if (w.graph) cudaGraphExecDestroy(w.graph);  // the graph refers to the old cache buffer
          w.graph = nullptr;
          CK(h, cudaStreamSynchronize(s));
          if (w.kcache[idx]) w.bytes -= w.kcap[idx] * (size_t)cached_entry_bytes(bf16) + 256;
          cudaFree(w.kcache[idx]);
          w.kcache[idx] = nullptr;
          const size_t cap = (need + need / 4 + 3) & ~(size_t)3;
          CK(h, dalloc(&w.bytes, (uint8_t **)&w.kcache[idx], cap * cached_entry_bytes(bf16)));
          w.kcap[idx] = cap;
        }
      }
      // kernel generation on the tensor cores where the image counts are exact in BF16 (<= 64 fine cells)
      const bool tc = l <= 3;
      const size_t wb = (size_t)umma_weight_bytes(3);
      launch_generate(bf16, l == 1 ? lab : nullptr, l == 1 ? nullptr : w.counts[l], level_dims(d1, l), h->cw + l * 2,
                      nblk, w.kdesc[l], w.kcache[l * 2], nblk > 1 ? w.kcache[l * 2 + 1] : nullptr,
                      tc ? h->uw + (size_t)(l * 2) * wb : nullptr, tc ? h->uw + (size_t)(l * 2 + 1) * wb : nullptr,
                      h->nsplit, h->umma_err, h->num_sms, s);
      h->launches += 1;
    }
    // the unit lists are built on the host while the GPU generates the kernels
    {
      // the level-1 units with work: CConv1 (a window that is not pure solid or
      // air) and CConv2 (a fluid cell), each with its plane chunk
      const bool fusedc2 = vec4_path(d1) && stream_fusion_ok(h->cfg.n_ortho);
      const int cap1 = stream_cap(bf16, false, STREAM_MODE_ZERO_PURE, fused_update(h, d1), h->num_sms);
      const int cap2 = stream_cap(bf16, fusedc2, STREAM_MODE_FLUID_ONLY, false, h->num_sms);
      const long long off2 = w.kskip_cap;  // the second list's place (run_network reads it there)
      w.uzc[0] = choose_stream_units(d1, w.h_kskip, 1, cap1, w.h_ulist, &w.un[0]);
      w.uzc[1] = choose_stream_units(d1, w.h_kskip + nsk, 2, cap2, w.h_ulist + off2, &w.un[1]);
      if (w.un[0])
        CK(h, cudaMemcpyAsync(w.ulist, w.h_ulist, sizeof(int) * (size_t)w.un[0], cudaMemcpyHostToDevice, s));
      if (w.un[1])
        CK(h, cudaMemcpyAsync(w.ulist + off2, w.h_ulist + off2, sizeof(int) * (size_t)w.un[1], cudaMemcpyHostToDevice,
                              s));
      w.ulist_ok = true;
      for (int i = 0; i < 2; ++i)
        stream_units_work(d1, w.h_ulist + (i ? off2 : 0), w.un[i], w.uzc[i], w.h_kmcount, &w.uwork[i][0],
                          &w.uwork[i][1]);
      w.ulist2_ok = false;
      if (lv2) {
        const Dims d2 = level_dims(d1, 2);
        const int cap2l = stream_cap(bf16, false, STREAM_MODE_ALL, false, h->num_sms);
        w.uzc2 = choose_stream_units(d2, w.h_kskip2, 1, cap2l, w.h_ulist2, &w.un2);
        if (w.un2) CK(h, cudaMemcpyAsync(w.ulist2, w.h_ulist2, sizeof(int) * (size_t)w.un2, cudaMemcpyHostToDevice, s));
        w.ulist2_ok = true;
      }
    }
  }
  CK(h, cudaGetLastError());
  return NPSOLVE_OK;
}



// ---------------------------------------------------------------------------
// Training: forward with stored intermediates, hand-written backward of
// Alg. 2 (kernels_train.cu) and the loss of Sec. 4.2.3.
// ---------------------------------------------------------------------------
constexpr int kWGOut = 27 * 55;
// layout of tr.out (doubles): per level l: [G1 (1485)][G2 (1485)][dots (2)][stats (54)][norm2 (1)]
constexpr int kTrOutPerLevel = 2 * kWGOut + 2 + 54 + 1;

void free_train(npsolve *h) {
  auto &t = h->tr;
  for (int l = 0; l <= kMaxLevels; ++l) {
    cudaFree(t.gx[l]);
    cudaFree(t.gx1[l]);
    t.gx[l] = t.gx1[l] = nullptr;
  }
  cudaFree(t.rm);
  cudaFree(t.tmp);
  cudaFree(t.tmp2);
  cudaFree(t.res);
  cudaFree(t.gz);
  cudaFree(t.K);
  cudaFree(t.kall);
  t.kall = nullptr;
  t.kall_cap = 0;
  cudaFree(t.part);
  cudaFree(t.out);
  t.rm = t.tmp = t.tmp2 = t.res = t.gz = t.K = nullptr;
  t.part = t.out = nullptr;
  t.cap = 0;
}

// The per-cell kernels of one block for the network transpose (t.cap x 27
// floats), allocated only by the paths that run it, before any graph capture.
int ensure_transpose_K(npsolve *h) {
  auto &t = h->tr;
  if (!t.K) CK(h, dalloc(nullptr, &t.K, (size_t)t.cap * 27));
  return NPSOLVE_OK;
}

int ensure_train(npsolve *h, Dims d1) {
  auto &t = h->tr;
  const long long n = d1.n();
  if (t.cap >= n) return NPSOLVE_OK;
  if (h->ws.graph) {  // a symmetric-variant iteration graph refers to these buffers
    cudaGraphExecDestroy(h->ws.graph);
    h->ws.graph = nullptr;
  }
  free_train(h);
  const int L = h->cfg.levels;
  long long cl = n;
  for (int l = 1; l <= L; ++l, cl = (cl + 7) / 8) {
    CK(h, dalloc(nullptr, &t.gx[l], (size_t)cl));
    CK(h, dalloc(nullptr, &t.gx1[l], (size_t)cl));
  }
  CK(h, dalloc(nullptr, &t.rm, (size_t)n));
  CK(h, dalloc(nullptr, &t.tmp, (size_t)n));
  CK(h, dalloc(nullptr, &t.tmp2, (size_t)n));
  CK(h, dalloc(nullptr, &t.res, (size_t)n));
  CK(h, dalloc(nullptr, &t.gz, (size_t)n));
  CK(h, dalloc(nullptr, &t.part, (size_t)148 * 4 * kWGOut + (size_t)kRedMaxBlocks * 64));
  CK(h, dalloc(nullptr, &t.out, (size_t)(kMaxLevels + 1) * kTrOutPerLevel));
  t.cap = n;
  return NPSOLVE_OK;
}

// Forward of Alg. 2 on r (zeroed off fluid into tr.rm) with every
// intermediate kept in the workspace; returns z in ws.z.  On the CUDA-core
// kernels: training evaluates each image once, so the per-solve kernel cache
// (classification, generation and its host synchronisation) does not pay.
// The label check's flag is OR-ed into tr.badb, which the caller reads once
// for the whole batch.  Enqueues only: no host synchronisation.
int train_forward(npsolve *h, const uint8_t *lab, Dims d1, const float *r, cudaStream_t s) {
  int st = check_dims(h, d1.nx, d1.ny, d1.nz);
  if (st) return st;
  st = ensure_ws(h, d1, 1);
  if (st) return st;
  st = ensure_train(h, d1);
  if (st) return st;
  if (!h->tr.badb) {
    CK(h, cudaMalloc(&h->tr.badb, sizeof(unsigned int)));
    CK(h, cudaMemsetAsync(h->tr.badb, 0, sizeof(unsigned int), s));
  }
  {
    // room for the per-cell kernels of every CConv block
    auto &t = h->tr;
    const int L = h->cfg.levels;
    long long need = 0;
    for (int l = 1; l <= L; ++l) need += (l < L ? 2 : 1) * level_dims(d1, l).n() * 27;
    if (need > t.kall_cap) {
      cudaFree(t.kall);
      t.kall = nullptr;
      t.kall_cap = 0;
      CK(h, dalloc(nullptr, &t.kall, (size_t)need));
      t.kall_cap = need;
    }
    long long off = 0;
    for (int l = 1; l <= L; ++l)
      for (int ty = 0; ty < (l < L ? 2 : 1); ++ty) {
        t.kslot[l * 2 + ty] = t.kall + off;
        off += level_dims(d1, l).n() * 27;
      }
  }
  const int path = h->cfg.kernel_path;
  h->cfg.kernel_path = NPSOLVE_PATH_CUDA_CORE;
  st = setup_image(h, lab, d1, s, true);
  if (!st) {
    launch_or_flag(h->ws.bad, h->tr.badb, s);
    launch_mask_copy(lab, d1.n(), r, h->tr.rm, s);
    h->tr.kstore = true;
    run_network(h, lab, d1, h->tr.rm, nullptr, h->ws.z, nullptr, s, true);
    h->tr.kstore = false;
  }
  h->cfg.kernel_path = path;
  if (st) return st;
  CK(h, cudaGetLastError());
  return NPSOLVE_OK;
}

// Room for `count` examples' reduced results (tr.outb).
int ensure_outb(npsolve *h, int count) {
  auto &t = h->tr;
  if (t.outb_cap >= count) return NPSOLVE_OK;
  cudaFree(t.outb);
  t.outb = nullptr;
  t.outb_cap = 0;
  CK(h, dalloc(nullptr, &t.outb, (size_t)count * (kMaxLevels + 1) * kTrOutPerLevel));
  t.outb_cap = count;
  return NPSOLVE_OK;
}

int check_umma_err(npsolve *h);

// Reads the batch's label-check flag (one host synchronisation, after the
// batch's results were copied) and clears it.
int check_batch_labels(npsolve *h, cudaStream_t s) {
  if (!h->tr.badb) return NPSOLVE_OK;
  unsigned int bad = 0;
  CK(h, cudaMemcpyAsync(&bad, h->tr.badb, sizeof(bad), cudaMemcpyDeviceToHost, s));
  CK(h, cudaMemsetAsync(h->tr.badb, 0, sizeof(unsigned int), s));
  CK(h, cudaStreamSynchronize(s));
  if (bad) return fail(h, NPSOLVE_BAD_LABELS, "labels must be 0 (solid), 1 (fluid) or 2 (air)");
  return check_umma_err(h);  // a tensor-core wait of the weight gradient that timed out
}

// Reverse of Alg. 2 for the output cotangent gz (device), after train_forward:
// the folded weight gradients, the Aff dots and image statistics of every
// level into `out` (device, (kMaxLevels + 1) x kTrOutPerLevel doubles, zeroed
// here; fold_gradients turns them into the raw blob layout) and, when gr !=
// null, d<gz, z>/dr into gr.  Enqueues only: no host synchronisation.
int train_backward(npsolve *h, const uint8_t *lab, Dims d1, const float *gz, double *out, float *gr,
                   cudaStream_t s) {
  Workspace &w = h->ws;
  auto &t = h->tr;
  const int L = h->cfg.levels;
  const long long n1 = d1.n();
  auto lc = [&](int l) { return l == 1 ? nullptr : w.counts[l]; };
  auto ll = [&](int l) { return l == 1 ? lab : nullptr; };
  auto O = [&](int l) { return out + (size_t)l * kTrOutPerLevel; };
  // the weight-gradient contraction on the tensor cores where the level's image
  // counts are exact in BF16 (at most 256 fine cells per cell: levels 1-3), on
  // CUDA cores beyond
  auto wgrad = [&](int l, Dims dl, const float *v, const float *g, double *dst) {
    if (l <= 3) launch_cconv_wgrad_tc(ll(l), lc(l), dl, v, g, t.part, dst, h->umma_err, h->num_sms, s);
    else launch_cconv_wgrad(ll(l), lc(l), dl, v, g, t.part, dst, s);
  };
  CK(h, cudaMemsetAsync(out, 0, sizeof(double) * (kMaxLevels + 1) * kTrOutPerLevel, s));
  for (int l = 1; l <= L; ++l) {
    const long long nl = level_dims(d1, l).n();
    CK(h, cudaMemsetAsync(t.gx[l], 0, sizeof(float) * nl, s));
    CK(h, cudaMemsetAsync(t.gx1[l], 0, sizeof(float) * nl, s));
  }
  launch_axpby(lab, n1, 1.f, gz, 0.f, nullptr, t.gx[1], s);  // output restriction
  if (L == 1) launch_axpby(nullptr, n1, 1.f, t.gx[1], 0.f, nullptr, t.gx1[1], s);
  // up pass in reverse: combination, CConv2, interpolation
  for (int l = 1; l < L; ++l) {
    const Dims dl = level_dims(d1, l);
    const long long nl = dl.n();
    launch_axpby_dev(nullptr, nl, w.affc + 2 * l, t.gx[l], 1.f, t.gx1[l], t.gx1[l], s);   // gx1 += c1 gx
    launch_axpby_dev(nullptr, nl, w.affc + 2 * l + 1, t.gx[l], 0.f, nullptr, t.tmp, s);     // g x2 = c2 gx
    wgrad(l, dl, w.r2[l], t.tmp, O(l) + kWGOut);
    launch_cconv_transpose(t.kslot[l * 2 + 1], t.tmp, dl, t.tmp2, s);  // g r2 (the forward's kernels)
    launch_interp_adjoint_add(t.tmp2, level_dims(d1, l + 1), (l + 1 == L) ? t.gx1[L] : t.gx[l + 1], s);
    h->launches += 6;
  }
  if (L > 1) {
    // Aff's weight gradient of every level, now that every gx[l] is final: the dots gx.x1, gx.x2 and the
    // image statistics (the exact window sums of the setup), in two launches
    Dot2Levels D{};
    D.l0 = 1;
    D.count = L - 1;
    for (int l = 1; l < L; ++l) {
      D.a[l] = t.gx[l];
      D.b[l] = w.x1[l];
      D.c[l] = w.x2[l];
      D.n[l] = level_dims(d1, l).n();
      D.out[l] = O(l) + 2 * kWGOut;
      D.stats_src[l] = w.affs + 54 * l;
      D.stats_dst[l] = O(l) + 2 * kWGOut + 2;
    }
    launch_dot2_levels(D, t.part, s);
    h->launches += 2;
  }
  // down pass in reverse: CConv1 and pooling
  for (int l = L; l >= 1; --l) {
    const Dims dl = level_dims(d1, l);
    const float *v = l == 1 ? t.rm : w.r1[l];
    wgrad(l, dl, v, t.gx1[l], O(l));
    h->launches += 2;
    if (l > 1 || gr) {
      launch_cconv_transpose(t.kslot[l * 2], t.gx1[l], dl, t.tmp, s);  // g r1^l
      h->launches += 1;
      if (l > 1) {
        launch_pool_adjoint_add(t.tmp, level_dims(d1, l - 1), t.gx1[l - 1], s);
        h->launches += 1;
      } else {
        launch_axpby(lab, n1, 1.f, t.tmp, 0.f, nullptr, gr, s);  // input padding
        h->launches += 1;
      }
    }
  }
  CK(h, cudaGetLastError());
  return NPSOLVE_OK;
}

// The folded gradients of one example's reduced results `ho` (host copy of a
// train_backward output block) added into gw in the raw blob layout.
void fold_gradients(const npsolve *h, const double *ho, std::vector<double> &gw) {
  const int L = h->cfg.levels;
  const size_t per = 2 * kCConvParams + 2 * kAffParams;
  for (int l = 1; l <= L; ++l) {
    const double sc = 1.0 / pow(8.0, l - 1);
    const double *Ol = ho + (size_t)l * kTrOutPerLevel;
    for (int type = 1; type <= (l < L ? 2 : 1); ++type) {
      const double *G = Ol + (type - 1) * kWGOut;
      const size_t base = (size_t)(l - 1) * per + (type == 2 ? kCConvParams : 0);
      for (int a = 0; a < 27; ++a) {
        for (int lp = 0; lp < 27; ++lp) {
          const double gf = G[a * 55 + lp], ga = G[a * 55 + 27 + lp];
          gw[base + (a * 3 + 0) * 27 + lp] += sc * gf;
          gw[base + (a * 3 + 1) * 27 + lp] += sc * ga;
          gw[base + (a * 3 + 2) * 27 + lp] += -sc * (gf + ga) + G[a * 55 + 54];
        }
        gw[base + 2187 + a] += G[a * 55 + 54];
      }
    }
    if (l < L) {
      const double *dots = Ol + 2 * kWGOut;
      const double *S = dots + 2;
      for (int k = 0; k < 2; ++k) {
        const size_t base = (size_t)(l - 1) * per + 2 * kCConvParams + (size_t)k * kAffParams;
        const double gc = dots[k];
        for (int lp = 0; lp < 27; ++lp) {
          gw[base + lp] += gc * S[lp];
          gw[base + 27 + lp] += gc * S[27 + lp];
          gw[base + 54 + lp] += gc * (1.0 / 27.0 - S[lp] - S[27 + lp]);
        }
        gw[base + 81] += gc;
      }
    }
  }
}

// out = P_net^T g: the adjoint of the network z = mask_fluid(N(mask_fluid(r)))
// (Alg. 2 is linear in r, Sec. 4.2), needed for the symmetric variant
// P_sym,1 = P_net^T P_net of the paper's symmetry analysis (appendix).  The
// reverse of Alg. 2 without the weight gradients: combinations (c1, c2 read
// on the device), CConv^T by gathering K_a(q - a) g(q - a) from the
// materialised kernels, trilinear interpolation^T and pooling^T.  No host
// synchronisation, so it can be captured in the iteration graph; the train
// workspace must be sized for d1 (ensure_train).
void run_network_transpose(npsolve *h, const uint8_t *lab, Dims d1, const float *g, float *out, cudaStream_t s) {
  Workspace &w = h->ws;
  auto &t = h->tr;
  const int L = h->cfg.levels;
  const long long n1 = d1.n();
  auto lc = [&](int l) { return l == 1 ? nullptr : w.counts[l]; };
  auto ll = [&](int l) { return l == 1 ? lab : nullptr; };
  for (int l = 1; l <= L; ++l) {
    const size_t nl = (size_t)level_dims(d1, l).n();
    cudaMemsetAsync(t.gx[l], 0, sizeof(float) * nl, s);  // errors surface at the caller's launch check
    cudaMemsetAsync(t.gx1[l], 0, sizeof(float) * nl, s);
  }
  launch_axpby(lab, n1, 1.f, g, 0.f, nullptr, t.gx[1], s);  // output restriction
  h->launches += 1;
  if (L == 1) {
    launch_axpby(nullptr, n1, 1.f, t.gx[1], 0.f, nullptr, t.gx1[1], s);
    h->launches += 1;
  }
  for (int l = 1; l < L; ++l) {  // up pass in reverse: combination, CConv2, interpolation
    const Dims dl = level_dims(d1, l);
    const long long nl = dl.n();
    launch_axpby_dev(nullptr, nl, w.affc + 2 * l, t.gx[l], 1.f, t.gx1[l], t.gx1[l], s);       // gx1 += c1 gx
    launch_axpby_dev(nullptr, nl, w.affc + 2 * l + 1, t.gx[l], 0.f, nullptr, t.tmp, s);         // g x2 = c2 gx
    launch_materialize_K(ll(l), lc(l), dl, h->cw + l * 2 + 1, t.K, s);
    launch_cconv_transpose(t.K, t.tmp, dl, t.tmp2, s);                                          // g r2
    launch_interp_adjoint_add(t.tmp2, level_dims(d1, l + 1), (l + 1 == L) ? t.gx1[L] : t.gx[l + 1], s);
    h->launches += 5;
  }
  for (int l = L; l >= 1; --l) {  // down pass in reverse: CConv1 and pooling
    const Dims dl = level_dims(d1, l);
    launch_materialize_K(ll(l), lc(l), dl, h->cw + l * 2, t.K, s);
    launch_cconv_transpose(t.K, t.gx1[l], dl, t.tmp, s);  // g r1^l
    if (l > 1) launch_pool_adjoint_add(t.tmp, level_dims(d1, l - 1), t.gx1[l - 1], s);
    else launch_axpby(lab, n1, 1.f, t.tmp, 0.f, nullptr, out, s);  // input restriction
    h->launches += 3;
  }
}

// Loss = || b - A P_net(I, b) || (Sec. 4.2.3) of one example and the
// reduced results of its weight gradient, scaled by `weight`, into `out`
// (device block of kTrOutPerLevel (kMaxLevels + 1) doubles; its last entry
// receives ||b - A P_net(I, b)||^2).  Enqueues only.
int loss_grad_enqueue(npsolve *h, const uint8_t *lab, Dims d1, const float *b, double weight, double *out,
                      cudaStream_t s) {
  int st = train_forward(h, lab, d1, b, s);
  if (st) return st;
  auto &t = h->tr;
  const long long n = d1.n();
  launch_lap(lab, d1, h->ws.z, t.res, s);                      // A z
  launch_axpby(lab, n, 1.f, t.rm, -1.f, t.res, t.res, s);      // res = b - A z
  double *nrm = t.out + (size_t)(kMaxLevels + 1) * kTrOutPerLevel - 1;
  launch_dot2(t.res, t.res, nullptr, n, t.part, nrm - 1, s);   // ||res||^2 (two-slot output)
  launch_lap(lab, d1, t.res, t.tmp2, s);                       // A res
  launch_scale_by_inv_norm(lab, n, (float)(-weight), nrm - 1, t.tmp2, t.gz, s);  // gz = -w A res / ||res||
  h->launches += 7;
  st = train_backward(h, lab, d1, t.gz, out, nullptr, s);
  if (st) return st;
  // the squared loss into the block's last entry (train_backward zeroed the block)
  CK(h, cudaMemcpyAsync(out + (size_t)(kMaxLevels + 1) * kTrOutPerLevel - 1, nrm - 1, sizeof(double),
                        cudaMemcpyDeviceToDevice, s));
  return NPSOLVE_OK;
}

// Enqueue one NPSDO iteration (Alg. 1 loop body) on stream s.
void enqueue_iteration(npsolve *h, const uint8_t *lab, Dims d1, const float *b, double *x, cudaStream_t s) {
  Workspace &w = h->ws;
  const long long n = d1.n();
  const bool fast = vec4_path(d1) && h->cfg.levels > 1;
  const bool sym = h->cfg.symmetric != 0;
  run_network(h, lab, d1, w.r, &w.st->rscale, w.z, w.st, s, false, !sym);
  if (sym) {
    // P_sym,1 = P_net^T P_net (appendix, symmetry analysis): the transpose of the
    // network applied to its output, then the dots of the combination kernel
    // (unit coefficients) on the symmetric preconditioned vector
    ProfScope ps(h, P_COMBINE, s);
    run_network_transpose(h, lab, d1, w.z, h->tr.res, s);
    h->launches += 1;
    if (vec4_path(d1) && h->cfg.levels > 1)
      launch_combine1_4(lab, (int)n, h->tr.res, h->tr.res, h->unit_c12, w.z, w.qring, w.r, nullptr, w.part,
                        w.tickets + kTicketCombine, w.st, h->num_sms, s);
    else launch_combine1(lab, n, h->tr.res, h->tr.res, h->unit_c12, w.z, w.qring, w.r, w.part, w.st, s);
  }
  const bool recur = h->cfg.residual_mode == NPSOLVE_RESIDUAL_RECURRENCE;
  const bool fused = fused_update(h, d1);  // the step's r update happens in the next level-1 CConv1
  h->launches += fast ? (recur ? (fused ? 2 : 3) : 5) : (recur ? 6 : 7);
  if (fast) {
    {
      ProfScope ps(h, P_ORTHO_DIR, s);
      launch_direction4(recur, (int)n, w.z, w.dring, w.xhi, w.xlo, w.gmask, w.st, h->cfg.n_ortho, h->num_sms, s);
    }
    {
      ProfScope ps(h, P_LAP, s);
      launch_lap4(w.lapcode, d1, w.dring, w.qring, w.r, fused ? w.r_alt : nullptr, w.part, w.tickets + kTicketLap,
                  w.st, h->num_sms, s);
    }
    if (fused) return;
    ProfScope ps(h, P_UPDATE, s);
    launch_update4(recur, (int)n, x, w.r, nullptr, w.dring, w.qring, w.part, w.tickets + kTicketUpdate, w.st, w.hist,
                   h->num_sms, s);
    if (!recur) launch_explicit_residual(lab, d1, b, x, w.r, w.part, w.st, w.hist, s);
    return;
  }
  {
    ProfScope ps(h, P_ORTHO_DIR, s);
    launch_ortho_final(w.part, n, w.st, s);
    launch_direction(n, w.z, w.dring, w.st, s);
  }
  {
    ProfScope ps(h, P_LAP, s);
    launch_lap_ring(lab, d1, w.dring, w.qring, w.r, w.part, w.st, s);
  }
  ProfScope ps(h, P_UPDATE, s);
  launch_update(recur, n, x, w.r, w.dring, w.qring, w.part, w.st, w.hist, s);
  if (!recur) launch_explicit_residual(lab, d1, b, x, w.r, w.part, w.st, w.hist, s);
}

// A kernel whose bounded wait (tensor-core MMA or TMA copy completion) timed
// out leaves a flag; a tensor map that could not be encoded leaves another.
int check_umma_err(npsolve *h) {
  if (h->stream_err) {
    h->stream_err = false;
    return fail(h, NPSOLVE_CUDA_ERROR, "streamed CConv: a TMA tensor map could not be encoded");
  }
  int e = 0;
  CK(h, cudaMemcpy(&e, h->umma_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    cudaMemset(h->umma_err, 0, sizeof(int));
    return fail(h, NPSOLVE_CUDA_ERROR, "a bounded device wait (MMA or TMA completion) timed out");
  }
  return NPSOLVE_OK;
}

int get_graph(npsolve *h, const uint8_t *lab, Dims d1, const float *b, double *x) {
  Workspace &w = h->ws;
  if (w.graph && w.graph_dims.nx == d1.nx && w.graph_dims.ny == d1.ny && w.graph_dims.nz == d1.nz &&
      w.graph_lab == lab && w.graph_b == b && w.graph_x == x && !w.graph_pcg && w.graph_units[0] == w.un[0] &&
      w.graph_units[1] == w.uzc[0] && w.graph_units[2] == w.un[1] && w.graph_units[3] == w.uzc[1] &&
      w.graph_units[4] == w.un2 && w.graph_units[5] == w.uzc2)
    return NPSOLVE_OK;
  if (w.graph) cudaGraphExecDestroy(w.graph);
  w.graph = nullptr;
  cudaGraph_t g;
  const long long before = h->launches;
  CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < kPollEvery; ++i) enqueue_iteration(h, lab, d1, b, x, h->cap_stream);
  CK(h, cudaStreamEndCapture(h->cap_stream, &g));
  w.graph_kernels = h->launches - before;  // captured, not launched
  h->launches = before;
  cudaError_t e = cudaGraphInstantiate(&w.graph, g, 0);
  cudaGraphDestroy(g);
  CK(h, e);
  w.graph_dims = d1;
  w.graph_lab = lab;
  w.graph_b = b;
  w.graph_x = x;
  w.graph_pcg = 0;
  w.graph_units[0] = w.un[0];
  w.graph_units[1] = w.uzc[0];
  w.graph_units[2] = w.un[1];
  w.graph_units[3] = w.uzc[1];
  w.graph_units[4] = w.un2;
  w.graph_units[5] = w.uzc2;
  return NPSOLVE_OK;
}

int solve_impl(npsolve *h, const uint8_t *lab, int nx, int ny, int nz, const float *b, double tol, int max_iter,
               cudaStream_t s, double *x, int *iters, double *rel_residual, cudaEvent_t b_ready = nullptr,
               double *x_host = nullptr) {
  if (!h) return fail(nullptr, NPSOLVE_BAD_ARG, "null handle");
  if (!lab || !b || !x || !iters || !rel_residual) return fail(h, NPSOLVE_BAD_ARG, "null pointer argument");
  if (misaligned16({lab, b, x})) return fail(h, NPSOLVE_BAD_ARG, kAlignMsg);
  if (!(tol > 0.0) || !isfinite(tol)) return fail(h, NPSOLVE_BAD_ARG, "tolerance must be finite and > 0");
  if (max_iter < 0) return fail(h, NPSOLVE_BAD_ARG, "max_iter must be >= 0");
  int st = check_dims(h, nx, ny, nz);
  if (st) return st;
  CK(h, cudaSetDevice(h->device));
  const Dims d1{nx, ny, nz};
  st = ensure_ws(h, d1, max_iter + 1);
  if (st) return st;
  if (h->cfg.symmetric) {  // the transpose pass of P_sym uses the train workspace
    st = ensure_train(h, d1);
    if (st) return st;
    st = ensure_transpose_K(h);
    if (st) return st;
  }
  Workspace &w = h->ws;
  {
    ProfScope ps(h, P_SETUP, s);
    st = setup_image(h, lab, d1, s, true);
    if (st) return st;
    if (cached_path(h, d1) && w.ulist_ok) {
      // the level-1 CConvs skip the units without work: what they would write there is zero
      CK(h, cudaMemsetAsync(w.z, 0, sizeof(float) * (size_t)d1.n(), s));
      if (h->cfg.levels > 1) CK(h, cudaMemsetAsync(w.r1[2], 0, sizeof(float) * (size_t)level_dims(d1, 2).n(), s));
      if (fused_update(h, d1)) CK(h, cudaMemsetAsync(w.r_alt, 0, sizeof(float) * (size_t)d1.n(), s));
      if (w.ulist2_ok) {  // the level-2 units without work: their outputs and pooled inputs of level 3 are zero
        const size_t n2 = (size_t)level_dims(d1, 2).n();
        CK(h, cudaMemsetAsync(w.x1[2], 0, sizeof(float) * n2, s));
        CK(h, cudaMemsetAsync(w.xc[2], 0, sizeof(float) * n2, s));
        CK(h, cudaMemsetAsync(w.r1[3], 0, sizeof(float) * (size_t)level_dims(d1, 3).n(), s));
      }
    }
    if (b_ready) CK(h, cudaStreamWaitEvent(s, b_ready, 0));  // b arrives on another stream during the setup
    if (vec4_path(d1)) {
      // the recurrence mode of the multilevel path keeps x as a double-float pair until the end
      const bool xdf = h->cfg.levels > 1 && h->cfg.residual_mode == NPSOLVE_RESIDUAL_RECURRENCE;
      launch_init4(lab, (int)d1.n(), b, w.r, x, xdf ? w.xhi : nullptr, xdf ? w.xlo : nullptr, w.part,
                   w.tickets + kTicketInit, tol, max_iter, h->cfg.n_ortho, h->cfg.method, w.st, w.hist, h->num_sms, s);
      h->launches += 1;
    } else {
      launch_init(lab, d1.n(), b, w.r, x, w.part, tol, max_iter, h->cfg.n_ortho, h->cfg.method, w.st, w.hist, s);
      h->launches += 2;
    }
  }
  CK(h, cudaGetLastError());
  CK(h, cudaMemcpyAsync(w.h_flag, w.bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
  CK(h, cudaMemcpyAsync(w.h_st, w.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
  CK(h, cudaStreamSynchronize(s));
  if (w.h_flag[0]) return fail(h, NPSOLVE_BAD_LABELS, "labels must be 0 (solid), 1 (fluid) or 2 (air)");
  if (w.h_st[0].done == kDoneBadInput) return fail(h, NPSOLVE_BAD_ARG, "b has non-finite entries on fluid cells");
  if (!h->prof.on) {  // profiling runs the iterations one at a time, without the graph
    st = get_graph(h, lab, d1, b, x);
    if (st) return st;
  }
  int launched = 0, restarts = 0;
  double rr[2] = {0.0, 0.0};  // final relative true residual, ||b||
  SolveState hs = w.h_st[0];
  for (;;) {
    // Replay the captured iterations until the device flags completion or the
    // cap is reached.  The state copy of batch i is read only after batch i+1
    // has been queued, so the GPU does not wait for the host between batches.
    // Once the residual's rate of decrease says that the batch just queued is
    // likely to converge, its state is read before anything more is queued:
    // that costs one short host wait, where a batch queued past convergence
    // replays kPollEvery iterations whose kernels return at once.
    int nb = 0;
    int rate_k = -1;       // the iteration count and ||r||^2 of an earlier state read
    double rate_r2 = 0.0;
    bool near = false;     // from the first prediction on, every batch's state is read before the next is queued
    auto near_convergence = [&](const SolveState &c) {
      bool close = false;
      if (rate_k >= 0 && c.k > rate_k && rate_r2 > 0.0 && c.rnorm2 > 0.0) {
        const double per_iter = pow(c.rnorm2 / rate_r2, 1.0 / (double)(c.k - rate_k));  // of ||r||^2
        // within a factor 10 of the tolerance after the queued batch: stop looking ahead
        close = per_iter < 1.0 && c.rnorm2 * pow(per_iter, (double)kPollEvery) < 100.0 * c.eps2;
      }
      if (c.k > rate_k) {
        rate_k = c.k;
        rate_r2 = c.rnorm2;
      }
      return close;
    };
    while (hs.done == kDoneRunning && launched < max_iter) {
      if (h->prof.on) {  // one iteration at a time, so that no no-op iteration is timed
        enqueue_iteration(h, lab, d1, b, x, s);
        CK(h, cudaGetLastError());
        launched += 1;
        CK(h, cudaMemcpyAsync(&w.h_st[0], w.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        CK(h, cudaStreamSynchronize(s));
        hs = w.h_st[0];
        continue;
      }
      if (max_iter - launched >= kPollEvery) {
        CK(h, cudaGraphLaunch(w.graph, s));
        h->launches += w.graph_kernels;
        launched += kPollEvery;
      } else {
        enqueue_iteration(h, lab, d1, b, x, s);
        CK(h, cudaGetLastError());
        launched += 1;
      }
      CK(h, cudaMemcpyAsync(&w.h_st[nb & 1], w.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
      CK(h, cudaEventRecord(w.ev[nb & 1], s));
      if (nb >= 1) {
        CK(h, cudaEventSynchronize(w.ev[(nb - 1) & 1]));
        hs = w.h_st[(nb - 1) & 1];
      }
      nb += 1;
      if (hs.done == kDoneRunning && (near || (near = near_convergence(hs)))) {
        CK(h, cudaEventSynchronize(w.ev[(nb - 1) & 1]));  // the batch just queued, before any more
        hs = w.h_st[(nb - 1) & 1];
      }
    }
    // The end of a pass, decided on the device and read back with one host
    // synchronisation: the last pending residual step (a no-op when none is
    // pending), the pending steps of x, and in the recurrence mode the FP64
    // true residual that replaces r and re-opens the iteration when a converged
    // solve's true residual is still above tolerance (k_restart_final);
    // otherwise the final figures only.
    const bool fused = fused_update(h, d1);
    if (fused) {
      ProfScope ps(h, P_UPDATE, s);
      launch_update4(true, (int)d1.n(), x, w.r, w.r_alt, w.dring, w.qring, w.part, w.tickets + kTicketUpdate, w.st,
                     w.hist, h->num_sms, s);
      h->launches += 1;
    }
    if (vec4_path(d1) && h->cfg.levels > 1 &&
        h->cfg.residual_mode == NPSOLVE_RESIDUAL_RECURRENCE) {  // the last steps may still be pending
      launch_flush_x((int)d1.n(), w.xhi, w.xlo, x, w.dring, w.st, h->num_sms, s);
      h->launches += 2;
    }
    if (x_host) {
      // x is final unless the check below re-opens the iteration: its download runs beside
      // the check on the copy stream (a re-opened pass copies it again, in order on that stream)
      CK(h, cudaEventRecord(h->x_ready, s));
      CK(h, cudaStreamWaitEvent(h->copy_stream, h->x_ready, 0));
      CK(h, cudaMemcpyAsync(x_host, x, sizeof(double) * (size_t)d1.n(), cudaMemcpyDeviceToHost, h->copy_stream));
    }
    const bool check = h->cfg.residual_mode == NPSOLVE_RESIDUAL_RECURRENCE && restarts < kMaxRestarts;
    // x as the double-float pair (the recurrence mode of the multilevel vector path): the
    // check in double-float FP32 arithmetic; otherwise in FP64 from x
    const bool xdf = vec4_path(d1) && h->cfg.levels > 1 && h->cfg.residual_mode == NPSOLVE_RESIDUAL_RECURRENCE;
    {
      ProfScope ps(h, P_FINAL, s);
      // r_k lives in buffer k mod 2 when the update is fused into the level-1 CConv1
      float *r_alt = fused ? w.r_alt : nullptr;
      if (xdf)
        launch_true_residual4(w.lapcode, d1, b, w.xhi, w.xlo, check ? w.r : nullptr, check ? r_alt : nullptr, w.part,
                              w.st, check ? w.reopened : nullptr, w.relres, s);
      else if (check)
        launch_replace_residual(lab, d1, b, x, w.r, r_alt, w.part, w.st, w.reopened, w.relres, s);
      else launch_relres(lab, d1, b, x, w.part, w.relres, s);
      h->launches += 2;
    }
    if (check) CK(h, cudaMemcpyAsync(w.h_flag, w.reopened, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(h, cudaMemcpyAsync(rr, w.relres, sizeof(rr), cudaMemcpyDeviceToHost, s));
    CK(h, cudaMemcpyAsync(&w.h_st[0], w.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    // the residual history up to the iterations launched so far (an upper bound of k + 1 entries)
    h->last_hist.resize((size_t)std::min(launched, max_iter) + 1);
    CK(h, cudaMemcpyAsync(h->last_hist.data(), w.hist, sizeof(double) * h->last_hist.size(), cudaMemcpyDeviceToHost,
                          s));
    CK(h, cudaStreamSynchronize(s));
    if (x_host) CK(h, cudaStreamSynchronize(h->copy_stream));
    hs = w.h_st[0];
    if (check && w.h_flag[0]) {
      restarts += 1;
      launched = hs.k;
      continue;
    }
    break;
  }
  *iters = hs.k;
  *rel_residual = rr[0];
  prof_collect(h);
  st = check_umma_err(h);
  if (st) return st;
  h->last_hist.resize(hs.k + 1);
  if (hs.done == kDoneBreakdown) return fail(h, NPSOLVE_BREAKDOWN, "breakdown: d^T A d <= 0 or non-finite at iteration %d", hs.k + 1);
  if (hs.done != kDoneConverged) return fail(h, NPSOLVE_NO_CONVERGENCE, "no convergence in %d iterations", hs.k);
  h->err.clear();
  return NPSOLVE_OK;
}

}  // namespace

namespace nps {
void set_thread_error(const char *msg) { g_thread_error = msg; }
}  // namespace nps

extern "C" {

size_t npsolve_weight_count(int levels) { return weight_count(levels); }

int npsolve_create(const npsolve_config *cfg, const float *weights_host, size_t n_weights, npsolve_t *out) {
  if (!cfg || !out) return fail(nullptr, NPSOLVE_BAD_ARG, "null argument");
  *out = nullptr;
  if (cfg->levels < 1 || cfg->levels > kMaxLevels) return fail(nullptr, NPSOLVE_BAD_ARG, "levels must be 1..%d", kMaxLevels);
  if (cfg->n_ortho < 0 || cfg->n_ortho > kMaxOrtho) return fail(nullptr, NPSOLVE_BAD_ARG, "n_ortho must be 0..%d", kMaxOrtho);
  if (cfg->precision != NPSOLVE_FP32 && cfg->precision != NPSOLVE_BF16)
    return fail(nullptr, NPSOLVE_BAD_ARG, "precision must be NPSOLVE_FP32 or NPSOLVE_BF16");
  if (cfg->residual_mode != NPSOLVE_RESIDUAL_RECURRENCE && cfg->residual_mode != NPSOLVE_RESIDUAL_EXPLICIT)
    return fail(nullptr, NPSOLVE_BAD_ARG, "bad residual_mode");
  if (!weights_host || n_weights != weight_count(cfg->levels))
    return fail(nullptr, NPSOLVE_BAD_ARG, "expected %zu weights for %d levels", weight_count(cfg->levels), cfg->levels);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, NPSOLVE_CUDA_ERROR, "no CUDA device: %s", cudaGetErrorString(e));
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return fail(nullptr, NPSOLVE_CUDA_ERROR, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
  if (prop.major * 10 + prop.minor != 103)
    return fail(nullptr, NPSOLVE_CUDA_ERROR, "device %s is sm_%d%d; this library is built for sm_103a", prop.name,
                prop.major, prop.minor);
  if (cfg->kernel_path != NPSOLVE_PATH_CACHED && cfg->kernel_path != NPSOLVE_PATH_CUDA_CORE &&
      cfg->kernel_path != NPSOLVE_PATH_TENSOR)
    return fail(nullptr, NPSOLVE_BAD_ARG, "bad kernel_path");
  if (cfg->method != NPSOLVE_METHOD_NPSDO && cfg->method != NPSOLVE_METHOD_PCG && cfg->method != NPSOLVE_METHOD_FPCG)
    return fail(nullptr, NPSOLVE_BAD_ARG, "bad method");
  if (cfg->symmetric != 0 && cfg->symmetric != 1) return fail(nullptr, NPSOLVE_BAD_ARG, "symmetric must be 0 or 1");
  npsolve *h = new npsolve();
  h->cfg = *cfg;
  // PCG and FPCG keep one previous direction: the ring of two slots of n_ortho = 1
  if (cfg->method != NPSOLVE_METHOD_NPSDO) h->cfg.n_ortho = 1;
  h->device = dev;
  h->nsplit = cfg->precision == NPSOLVE_BF16 ? 1 : 3;
  h->num_sms = prop.multiProcessorCount;
  h->weights.assign(weights_host, weights_host + n_weights);
  int st = NPSOLVE_OK;
  {
    cudaError_t e1 = cudaMalloc(&h->cw, sizeof(CConvW) * (kMaxLevels + 1) * 2);
    cudaError_t e2 = cudaMalloc(&h->aw, sizeof(AffW) * (kMaxLevels + 1) * 2);
    cudaError_t e3 = cudaMalloc(&h->unit_c12, 2 * sizeof(double));
    cudaError_t e4 = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e4 == cudaSuccess) e4 = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
    if (e4 == cudaSuccess) e4 = cudaEventCreateWithFlags(&h->b_ready, cudaEventDisableTiming);
    if (e4 == cudaSuccess) e4 = cudaEventCreateWithFlags(&h->x_ready, cudaEventDisableTiming);
    cudaError_t e5 = cudaMalloc(&h->uw, (size_t)(kMaxLevels + 1) * 2 * umma_weight_bytes(3));
    cudaError_t e6 = cudaMalloc(&h->umma_err, sizeof(int));
    cudaError_t e7 = cudaMalloc(&h->uni, sizeof(float) * (kMaxLevels + 1) * 2 * 81);
    if (e1 || e2 || e3 || e4 || e5 || e6 || e7) st = fail(nullptr, NPSOLVE_OOM, "device allocation failed");
    if (!st && cudaMemset(h->umma_err, 0, sizeof(int)) != cudaSuccess)
      st = fail(nullptr, NPSOLVE_CUDA_ERROR, "cudaMemset failed");
  }
  if (!st) {
    const double one_zero[2] = {1.0, 0.0};
    if (cudaMemcpy(h->unit_c12, one_zero, sizeof(one_zero), cudaMemcpyHostToDevice) != cudaSuccess)
      st = fail(nullptr, NPSOLVE_CUDA_ERROR, "cudaMemcpy failed");
  }
  if (!st) st = upload_weights(h);
  if (st) {
    g_thread_error = h->err.empty() ? g_thread_error : h->err;
    npsolve_destroy(h);
    return st;
  }
  *out = h;
  return NPSOLVE_OK;
}

int npsolve_set_weights(npsolve_t h, const float *weights_host, size_t n) {
  if (!h || !weights_host) return fail(h, NPSOLVE_BAD_ARG, "null argument");
  if (n != h->weights.size()) return fail(h, NPSOLVE_BAD_ARG, "expected %zu weights", h->weights.size());
  CK(h, cudaSetDevice(h->device));
  h->weights.assign(weights_host, weights_host + n);
  return upload_weights(h);
}

int npsolve_get_weights(npsolve_t h, float *weights_host, size_t n) {
  if (!h || !weights_host) return fail(h, NPSOLVE_BAD_ARG, "null argument");
  if (n != h->weights.size()) return fail(h, NPSOLVE_BAD_ARG, "expected %zu weights", h->weights.size());
  memcpy(weights_host, h->weights.data(), n * sizeof(float));
  return NPSOLVE_OK;
}

void npsolve_destroy(npsolve_t h) {
  if (!h) return;
  cudaSetDevice(h->device);
  free_ws(h->ws);
  free_train(h);
  cudaFree(h->tr.outb);
  cudaFree(h->tr.badb);
  for (cudaEvent_t e : h->prof.pool) cudaEventDestroy(e);
  cudaFree(h->cw);
  cudaFree(h->aw);
  cudaFree(h->unit_c12);
  cudaFree(h->uw);
  cudaFree(h->uni);
  cudaFree(h->umma_err);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  if (h->b_ready) cudaEventDestroy(h->b_ready);
  if (h->x_ready) cudaEventDestroy(h->x_ready);
  delete h;
}

const char *npsolve_last_error(npsolve_t h) { return h ? h->err.c_str() : g_thread_error.c_str(); }

int npsolve_solve(npsolve_t h, const uint8_t *labels, int nx, int ny, int nz, const float *b, double tol,
                  int max_iter, void *stream, double *x, int *iters, double *rel_residual) {
  return solve_impl(h, labels, nx, ny, nz, b, tol, max_iter, (cudaStream_t)stream, x, iters, rel_residual);
}

int npsolve_solve_host(npsolve_t h, const uint8_t *labels_host, int nx, int ny, int nz, const float *b_host,
                       double tol, int max_iter, void *stream, double *x_host, int *iters, double *rel_residual) {
  if (!h) return fail(nullptr, NPSOLVE_BAD_ARG, "null handle");
  if (!labels_host || !b_host || !x_host) return fail(h, NPSOLVE_BAD_ARG, "null pointer argument");
  int st = check_dims(h, nx, ny, nz);
  if (st) return st;
  CK(h, cudaSetDevice(h->device));
  cudaStream_t s = (cudaStream_t)stream;
  st = ensure_ws(h, Dims{nx, ny, nz}, max_iter + 1);
  if (st) return st;
  Workspace &w = h->ws;
  const size_t n = (size_t)nx * ny * nz;
  if (!w.stage_lab) {  // staging buffers live as long as the workspace
    CK(h, dalloc(&w.bytes, &w.stage_lab, (size_t)w.cap));
    CK(h, dalloc(&w.bytes, &w.stage_b, (size_t)w.cap));
    CK(h, dalloc(&w.bytes, &w.stage_x, (size_t)w.cap));
  }
  // the labels first on the solve's stream (the setup needs them), b beside the setup on the copy stream
  CK(h, cudaMemcpyAsync(w.stage_lab, labels_host, n, cudaMemcpyHostToDevice, s));
  CK(h, cudaEventRecord(h->b_ready, s));  // after the previous user of the staging buffers on s
  CK(h, cudaStreamWaitEvent(h->copy_stream, h->b_ready, 0));
  CK(h, cudaMemcpyAsync(w.stage_b, b_host, n * sizeof(float), cudaMemcpyHostToDevice, h->copy_stream));
  CK(h, cudaEventRecord(h->b_ready, h->copy_stream));
  // x comes back inside solve_impl, beside the final residual check
  return solve_impl(h, w.stage_lab, nx, ny, nz, w.stage_b, tol, max_iter, s, w.stage_x, iters, rel_residual,
                    h->b_ready, x_host);
}

int npsolve_residual_history(npsolve_t h, double *hist_host, int cap, int *count) {
  if (!h || !hist_host || !count) return fail(h, NPSOLVE_BAD_ARG, "null argument");
  const int m = (int)h->last_hist.size() < cap ? (int)h->last_hist.size() : cap;
  memcpy(hist_host, h->last_hist.data(), sizeof(double) * (m > 0 ? m : 0));
  *count = m;
  return NPSOLVE_OK;
}

int npsolve_network_intermediate(npsolve_t h, const uint8_t *labels, int nx, int ny, int nz, const float *r,
                                 int level, int which, float *out, double *c12_host, void *stream) {
  if (!h) return fail(nullptr, NPSOLVE_BAD_ARG, "null handle");
  if (!labels || !r || !out) return fail(h, NPSOLVE_BAD_ARG, "null pointer argument");
  if (misaligned16({labels, r, out})) return fail(h, NPSOLVE_BAD_ARG, kAlignMsg);
  const int L = h->cfg.levels;
  if (level < 0 || level > L || which < 0 || which > 4) return fail(h, NPSOLVE_BAD_ARG, "bad level/which");
  int st = check_dims(h, nx, ny, nz);
  if (st) return st;
  CK(h, cudaSetDevice(h->device));
  cudaStream_t s = (cudaStream_t)stream;
  const Dims d1{nx, ny, nz};
  st = ensure_ws(h, d1, 1);
  if (st) return st;
  Workspace &w = h->ws;
  st = setup_image(h, labels, d1, s, true);
  if (st) return st;
  CK(h, cudaMemcpyAsync(w.h_flag, w.bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
  CK(h, cudaStreamSynchronize(s));
  if (w.h_flag[0]) return fail(h, NPSOLVE_BAD_LABELS, "labels must be 0 (solid), 1 (fluid) or 2 (air)");
  run_network(h, labels, d1, r, nullptr, w.z, nullptr, s, level > 0);
  CK(h, cudaGetLastError());
  if (level == 0) {  // the network output z
    CK(h, cudaMemcpyAsync(out, w.z, sizeof(float) * d1.n(), cudaMemcpyDeviceToDevice, s));
  } else {
    const long long nl = level_dims(d1, level).n();
    const float *src = nullptr;
    if (which == 0) src = w.x1[level];
    else if (which == 1) src = level < L ? w.r2[level] : nullptr;
    else if (which == 2) src = level < L ? w.x2[level] : nullptr;
    else if (which == 3) src = level == L ? w.x1[L] : (level == 1 ? w.z : w.xc[level]);
    else src = level == 1 ? r : w.r1[level];
    if (!src) return fail(h, NPSOLVE_BAD_ARG, "level %d has no such intermediate", level);
    CK(h, cudaMemcpyAsync(out, src, sizeof(float) * nl, cudaMemcpyDeviceToDevice, s));
    if (c12_host) {
      if (level < L) CK(h, cudaMemcpyAsync(c12_host, w.affc + 2 * level, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      else c12_host[0] = c12_host[1] = 0.0;
    }
  }
  CK(h, cudaStreamSynchronize(s));
  return check_umma_err(h);
}

int npsolve_apply_network(npsolve_t h, const uint8_t *labels, int nx, int ny, int nz, const float *r, float *z,
                          void *stream) {
  return npsolve_network_intermediate(h, labels, nx, ny, nz, r, 0, 0, z, nullptr, stream);
}

// Shared prologue of the symmetry entry points: dims, workspaces (the train
// workspace holds the transpose's buffers), image setup and the label check.
static int symmetry_setup(npsolve *h, const uint8_t *labels, Dims d1, cudaStream_t s) {
  int st = check_dims(h, d1.nx, d1.ny, d1.nz);
  if (st) return st;
  CK(h, cudaSetDevice(h->device));
  st = ensure_ws(h, d1, 1);
  if (st) return st;
  st = ensure_train(h, d1);
  if (st) return st;
  st = ensure_transpose_K(h);
  if (st) return st;
  st = setup_image(h, labels, d1, s, true);
  if (st) return st;
  CK(h, cudaMemcpyAsync(h->ws.h_flag, h->ws.bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
  CK(h, cudaStreamSynchronize(s));
  if (h->ws.h_flag[0]) return fail(h, NPSOLVE_BAD_LABELS, "labels must be 0 (solid), 1 (fluid) or 2 (air)");
  return NPSOLVE_OK;
}

int npsolve_network_transpose(npsolve_t h, const uint8_t *labels, int nx, int ny, int nz, const float *g, float *out,
                              void *stream) {
  if (!h) return fail(nullptr, NPSOLVE_BAD_ARG, "null handle");
  if (!labels || !g || !out) return fail(h, NPSOLVE_BAD_ARG, "null pointer argument");
  if (misaligned16({labels, g, out})) return fail(h, NPSOLVE_BAD_ARG, kAlignMsg);
  cudaStream_t s = (cudaStream_t)stream;
  const Dims d1{nx, ny, nz};
  int st = symmetry_setup(h, labels, d1, s);
  if (st) return st;
  run_network_transpose(h, labels, d1, g, out, s);
  CK(h, cudaGetLastError());
  CK(h, cudaStreamSynchronize(s));
  return NPSOLVE_OK;
}

int npsolve_asymmetry(npsolve_t h, const uint8_t *labels, int nx, int ny, int nz, const float *x, const float *y,
                      void *stream, double *S, double *dots_host) {
  if (!h) return fail(nullptr, NPSOLVE_BAD_ARG, "null handle");
  if (!labels || !x || !y || !S) return fail(h, NPSOLVE_BAD_ARG, "null pointer argument");
  if (misaligned16({labels, x, y})) return fail(h, NPSOLVE_BAD_ARG, kAlignMsg);
  cudaStream_t s = (cudaStream_t)stream;
  const Dims d1{nx, ny, nz};
  int st = symmetry_setup(h, labels, d1, s);
  if (st) return st;
  Workspace &w = h->ws;
  auto &t = h->tr;
  const long long n = d1.n();
  run_network(h, labels, d1, x, nullptr, w.z, nullptr, s);  // P(x)
  CK(h, cudaMemcpyAsync(t.res, w.z, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, s));
  run_network(h, labels, d1, y, nullptr, w.z, nullptr, s);  // P(y)
  launch_dot2(x, w.z, t.res, n, t.part, t.out, s);          // x.P(y), x.P(x)
  launch_dot2(y, t.res, w.z, n, t.part, t.out + 2, s);      // y.P(x), y.P(y)
  h->launches += 4;
  double d[4] = {0, 0, 0, 0};
  CK(h, cudaGetLastError());
  CK(h, cudaMemcpyAsync(d, t.out, sizeof(d), cudaMemcpyDeviceToHost, s));
  CK(h, cudaStreamSynchronize(s));
  const double den = sqrt(fabs(d[1]) * fabs(d[3]));
  *S = den > 0.0 ? fabs(d[0] - d[2]) / den : 0.0;
  if (dots_host)
    for (int i = 0; i < 4; ++i) dots_host[i] = d[i];
  return check_umma_err(h);
}

int npsolve_apply_laplacian(const uint8_t *labels, int nx, int ny, int nz, const float *d, float *q, void *stream) {
  if (!labels || !d || !q) return fail(nullptr, NPSOLVE_BAD_ARG, "null pointer argument");
  if (misaligned16({labels, d, q})) return fail(nullptr, NPSOLVE_BAD_ARG, kAlignMsg);
  if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz > (1LL << 31) - 1)
    return fail(nullptr, NPSOLVE_BAD_DIMS, "bad dims");
  launch_lap(labels, Dims{nx, ny, nz}, d, q, (cudaStream_t)stream);
  CK(nullptr, cudaGetLastError());
  CK(nullptr, cudaStreamSynchronize((cudaStream_t)stream));
  return NPSOLVE_OK;
}

int npsolve_true_residual(const uint8_t *labels, int nx, int ny, int nz, const float *b, const double *x,
                          double *rel_residual, void *stream) {
  if (!labels || !b || !x || !rel_residual) return fail(nullptr, NPSOLVE_BAD_ARG, "null pointer argument");
  if (misaligned16({labels, b, x})) return fail(nullptr, NPSOLVE_BAD_ARG, kAlignMsg);
  if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz > (1LL << 31) - 1)
    return fail(nullptr, NPSOLVE_BAD_DIMS, "bad dims");
  cudaStream_t s = (cudaStream_t)stream;
  double *part = nullptr;
  CK(nullptr, cudaMallocAsync((void **)&part, sizeof(double) * (kRedMaxBlocks * 2 + 2), s));
  launch_relres(labels, Dims{nx, ny, nz}, b, x, part, part + kRedMaxBlocks * 2, s);
  double rr[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(rr, part + kRedMaxBlocks * 2, sizeof(rr), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(part, s);
  CK(nullptr, e);
  CK(nullptr, cudaStreamSynchronize(s));
  *rel_residual = rr[0];
  return NPSOLVE_OK;
}

int npsolve_jacobi_pcg(const uint8_t *labels, int nx, int ny, int nz, const float *b, double tol, int max_iter,
                       void *stream, double *x, int *iters, double *rel_residual) {
  if (!labels || !b || !x || !iters || !rel_residual) return fail(nullptr, NPSOLVE_BAD_ARG, "null pointer argument");
  if (misaligned16({labels, b, x})) return fail(nullptr, NPSOLVE_BAD_ARG, kAlignMsg);
  if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz > (1LL << 31) - 1)
    return fail(nullptr, NPSOLVE_BAD_DIMS, "bad dims");
  if (!(tol > 0.0) || max_iter < 0) return fail(nullptr, NPSOLVE_BAD_ARG, "bad tol/max_iter");
  cudaStream_t s = (cudaStream_t)stream;
  const Dims dm{nx, ny, nz};
  const size_t n = dm.n();
  float *r = nullptr, *p = nullptr, *q = nullptr;
  double *part = nullptr, *hist = nullptr;
  void *st = nullptr;
  int *hst = nullptr;
  CK(nullptr, cudaMalloc(&r, n * 4));
  CK(nullptr, cudaMalloc(&p, n * 4));
  CK(nullptr, cudaMalloc(&q, n * 4));
  CK(nullptr, cudaMalloc(&part, sizeof(double) * (kRedMaxBlocks * 2 + 2)));
  CK(nullptr, cudaMalloc(&hist, sizeof(double) * (max_iter + 1)));
  CK(nullptr, cudaMalloc(&st, pcg_state_bytes()));
  CK(nullptr, cudaHostAlloc((void **)&hst, 64, cudaHostAllocDefault));
  launch_pcg_init(labels, dm, b, r, p, x, part, tol, st, hist, s);
  int launched = 0, done = 0, k = 0;
  while (launched < max_iter) {
    const int batch = (max_iter - launched) < 16 ? (max_iter - launched) : 16;
    for (int i = 0; i < batch; ++i) launch_pcg_iter(labels, dm, x, r, p, q, part, st, hist, s);
    launched += batch;
    cudaMemcpyAsync(hst, st, pcg_state_bytes() < 64 ? pcg_state_bytes() : 64, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    done = *(int *)((char *)hst + pcg_done_offset());
    if (done) break;
  }
  cudaMemcpyAsync(hst, st, pcg_state_bytes() < 64 ? pcg_state_bytes() : 64, cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  done = *(int *)((char *)hst + pcg_done_offset());
  k = *(int *)((char *)hst + pcg_k_offset());
  launch_relres(labels, dm, b, x, part, part + kRedMaxBlocks * 2, s);
  double rr[2] = {0, 0};
  cudaMemcpyAsync(rr, part + kRedMaxBlocks * 2, sizeof(rr), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(r);
  cudaFree(p);
  cudaFree(q);
  cudaFree(part);
  cudaFree(hist);
  cudaFree(st);
  cudaFreeHost(hst);
  CK(nullptr, e);
  *iters = k;
  *rel_residual = rr[0];
  if (done == kDoneBadInput) return fail(nullptr, NPSOLVE_BAD_ARG, "non-finite b");
  if (done == kDoneBreakdown) return fail(nullptr, NPSOLVE_BREAKDOWN, "PCG breakdown");
  if (done != kDoneConverged) return fail(nullptr, NPSOLVE_NO_CONVERGENCE, "no convergence in %d iterations", k);
  return NPSOLVE_OK;
}

long long npsolve_launch_count(npsolve_t h) { return h ? h->launches : 0; }

size_t npsolve_workspace_bytes(npsolve_t h) { return h ? h->ws.bytes : 0; }

long long npsolve_mixed_cells(npsolve_t h, int level) {
  if (!h || level < 1 || level > h->cfg.levels || !h->ws.h_ktotal || !stream_level(h, h->ws.dims, level)) return -1;
  return (long long)h->ws.h_ktotal[2 * level + 1];
}

int npsolve_level1_work(npsolve_t h, int which, long long *cells, long long *mixed) {
  if (!h || !cells || !mixed || which < 0 || which > 1) return fail(h, NPSOLVE_BAD_ARG, "bad argument");
  if (!h->ws.ulist_ok) return fail(h, NPSOLVE_BAD_ARG, "no level-1 unit lists (no cached-path solve yet)");
  *cells = h->ws.uwork[which][0];
  *mixed = h->ws.uwork[which][1];
  return NPSOLVE_OK;
}

int npsolve_profile_count(void) { return P_COUNT; }

const char *npsolve_profile_name(int cls) { return (cls >= 0 && cls < P_COUNT) ? kProfNames[cls] : ""; }

int npsolve_set_profiling(npsolve_t h, int on) {
  if (!h) return fail(nullptr, NPSOLVE_BAD_ARG, "null handle");
  h->prof.on = on != 0;
  for (int i = 0; i < P_COUNT; ++i) {
    h->prof.ms[i] = 0.0;
    h->prof.launches[i] = 0;
  }
  h->prof.cls.clear();
  return NPSOLVE_OK;
}

int npsolve_get_profile(npsolve_t h, double *ms_host, long long *launches_host) {
  if (!h || !ms_host || !launches_host) return fail(h, NPSOLVE_BAD_ARG, "null argument");
  for (int i = 0; i < P_COUNT; ++i) {
    ms_host[i] = h->prof.ms[i];
    launches_host[i] = h->prof.launches[i];
  }
  return NPSOLVE_OK;
}

int npsolve_network_vjp(npsolve_t h, const uint8_t *labels, int nx, int ny, int nz, const float *r, const float *gz,
                        float *grad_w_host, float *grad_r, void *stream) {
  if (!h) return fail(nullptr, NPSOLVE_BAD_ARG, "null handle");
  if (!labels || !r || !gz || !grad_w_host) return fail(h, NPSOLVE_BAD_ARG, "null pointer argument");
  if (misaligned16({labels, r, gz, grad_r})) return fail(h, NPSOLVE_BAD_ARG, kAlignMsg);
  CK(h, cudaSetDevice(h->device));
  cudaStream_t s = (cudaStream_t)stream;
  const Dims d1{nx, ny, nz};
  int st = train_forward(h, labels, d1, r, s);
  if (st) return st;
  st = ensure_outb(h, 1);
  if (st) return st;
  st = train_backward(h, labels, d1, gz, h->tr.outb, grad_r, s);
  if (st) return st;
  std::vector<double> ho((size_t)(kMaxLevels + 1) * kTrOutPerLevel);
  CK(h, cudaMemcpyAsync(ho.data(), h->tr.outb, sizeof(double) * ho.size(), cudaMemcpyDeviceToHost, s));
  st = check_batch_labels(h, s);  // synchronises
  if (st) return st;
  std::vector<double> gw(h->weights.size(), 0.0);
  fold_gradients(h, ho.data(), gw);
  for (size_t i = 0; i < gw.size(); ++i) grad_w_host[i] = (float)gw[i];
  return NPSOLVE_OK;
}

// The mean loss and weight gradient of a batch: every example enqueued into
// its own results block, one copy and one host synchronisation at the end.
int batch_loss_grad(npsolve *h, int batch, const uint8_t *const *labels, const int *dims, const float *const *b,
                    double weight, cudaStream_t s, double *mean_loss, std::vector<double> &gw) {
  int st = ensure_outb(h, batch);
  if (st) return st;
  const size_t blk = (size_t)(kMaxLevels + 1) * kTrOutPerLevel;
  for (int i = 0; i < batch; ++i) {
    if (!labels[i] || !b[i]) return fail(h, NPSOLVE_BAD_ARG, "null example pointer");
    if (misaligned16({labels[i], b[i]})) return fail(h, NPSOLVE_BAD_ARG, kAlignMsg);
    st = loss_grad_enqueue(h, labels[i], Dims{dims[3 * i], dims[3 * i + 1], dims[3 * i + 2]}, b[i], weight,
                           h->tr.outb + (size_t)i * blk, s);
    if (st) return st;
  }
  std::vector<double> ho((size_t)batch * blk);
  CK(h, cudaMemcpyAsync(ho.data(), h->tr.outb, sizeof(double) * ho.size(), cudaMemcpyDeviceToHost, s));
  st = check_batch_labels(h, s);  // synchronises
  if (st) return st;
  double total = 0.0;
  for (int i = 0; i < batch; ++i) {
    fold_gradients(h, ho.data() + (size_t)i * blk, gw);
    total += sqrt(ho[(size_t)i * blk + blk - 1]);
  }
  *mean_loss = total / batch;
  return NPSOLVE_OK;
}

int npsolve_loss_grad(npsolve_t h, const uint8_t *labels, int nx, int ny, int nz, const float *b, void *stream,
                      double *loss, float *grad_w_host) {
  if (!h) return fail(nullptr, NPSOLVE_BAD_ARG, "null handle");
  if (!labels || !b || !loss) return fail(h, NPSOLVE_BAD_ARG, "null pointer argument");
  CK(h, cudaSetDevice(h->device));
  std::vector<double> gw(h->weights.size(), 0.0);
  const int dims[3] = {nx, ny, nz};
  int st = batch_loss_grad(h, 1, &labels, dims, &b, 1.0, (cudaStream_t)stream, loss, gw);
  if (st) return st;
  if (grad_w_host)
    for (size_t i = 0; i < gw.size(); ++i) grad_w_host[i] = (float)gw[i];
  return NPSOLVE_OK;
}

int npsolve_train_step(npsolve_t h, int batch, const uint8_t *const *labels, const int *dims, const float *const *b,
                       float lr, void *stream, double *loss) {
  if (!h) return fail(nullptr, NPSOLVE_BAD_ARG, "null handle");
  if (batch < 1 || !labels || !dims || !b || !loss || !(lr > 0.f)) return fail(h, NPSOLVE_BAD_ARG, "bad argument");
  CK(h, cudaSetDevice(h->device));
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nw = h->weights.size();
  std::vector<double> gw(nw, 0.0);
  double mean_loss = 0.0;
  int st = batch_loss_grad(h, batch, labels, dims, b, 1.0 / batch, s, &mean_loss, gw);
  if (st) return st;
  // Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the raw weights, FP64 moments
  auto &t = h->tr;
  if (t.m.size() != nw) {
    t.m.assign(nw, 0.0);
    t.v.assign(nw, 0.0);
    t.t = 0;
  }
  t.t += 1;
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  const double c1 = 1.0 - pow(b1, (double)t.t), c2 = 1.0 - pow(b2, (double)t.t);
  for (size_t k = 0; k < nw; ++k) {
    const double g = gw[k];
    if (!std::isfinite(g)) return fail(h, NPSOLVE_BREAKDOWN, "non-finite gradient");
    t.m[k] = b1 * t.m[k] + (1.0 - b1) * g;
    t.v[k] = b2 * t.v[k] + (1.0 - b2) * g * g;
    h->weights[k] = (float)(h->weights[k] - lr * (t.m[k] / c1) / (sqrt(t.v[k] / c2) + eps));
  }
  *loss = mean_loss;
  return upload_weights(h);
}

// Eigenpairs of the symmetric tridiagonal matrix with diagonal d[0..m-1] and
// off-diagonal e[0..m-2] by implicit QR steps with the Wilkinson shift
// (Golub and Van Loan, Matrix Computations, Sec. 8.3: bulge chasing with
// Givens rotations, deflation of negligible off-diagonal entries).  On return
// d holds the eigenvalues and, if `vectors`, column j of Z (row-major m x m)
// the eigenvector of d[j].  Returns false if a block fails to converge in
// 30 m steps.
static bool tridiag_eigen(std::vector<double> &d, std::vector<double> e, int m, std::vector<double> &Z,
                          bool vectors = true) {
  Z.assign(vectors ? (size_t)m * m : 0, 0.0);
  if (vectors)
    for (int i = 0; i < m; ++i) Z[(size_t)i * m + i] = 1.0;
  const double eps = 2.220446049250313e-16;
  auto negligible = [&](int i) { return fabs(e[i]) <= eps * (fabs(d[i]) + fabs(d[i + 1])); };
  long long steps = 0;
  int hi = m - 1;
  while (hi > 0) {
    if (negligible(hi - 1)) {  // d[hi] has converged
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    if (++steps > 30LL * m) return false;
    int lo = hi - 1;  // the unreduced block lo..hi
    while (lo > 0 && !negligible(lo - 1)) --lo;
    // Wilkinson shift: the eigenvalue of the trailing 2x2 block nearer d[hi]
    const double h = 0.5 * (d[hi - 1] - d[hi]), eh = e[hi - 1];
    const double mu = d[hi] - eh * eh / (h + (h >= 0.0 ? 1.0 : -1.0) * hypot(h, eh));
    // the first rotation acts on (d[lo] - mu, e[lo]); each later one removes the bulge
    double a = d[lo] - mu, b = e[lo], bulge = 0.0;
    for (int k = lo; k < hi; ++k) {
      const double r = hypot(a, b);
      const double c = r > 0.0 ? a / r : 1.0, sn = r > 0.0 ? -b / r : 0.0;
      if (k > lo) e[k - 1] = r;  // the bulge is rotated into the off-diagonal entry
      const double p = d[k], q = e[k], t = d[k + 1];
      d[k] = c * c * p - 2.0 * c * sn * q + sn * sn * t;
      d[k + 1] = sn * sn * p + 2.0 * c * sn * q + c * c * t;
      e[k] = c * sn * (p - t) + (c * c - sn * sn) * q;
      if (k + 1 < hi) {  // the next bulge at (k+2, k)
        bulge = -sn * e[k + 1];
        e[k + 1] = c * e[k + 1];
        a = e[k];
        b = bulge;
      }
      for (int i = 0; i < (vectors ? m : 0); ++i) {  // Z <- Z G on columns k, k+1
        double *zr = &Z[(size_t)i * m];
        const double zk = zr[k], zk1 = zr[k + 1];
        zr[k] = c * zk - sn * zk1;
        zr[k + 1] = sn * zk + c * zk1;
      }
    }
  }
  return true;
}

int npsolve_lanczos_rhs(const uint8_t *labels, int nx, int ny, int nz, const float *start, int m, int k, int count,
                        unsigned long long seed, float *out, double *ritz_values_host, void *stream) {
  if (!labels || !start || !out || m < 2 || m > kMaxLanczos || k < 1 || k > m || count < 0)
    return fail(nullptr, NPSOLVE_BAD_ARG, "bad argument");
  if (misaligned16({labels, start, out})) return fail(nullptr, NPSOLVE_BAD_ARG, kAlignMsg);
  if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz > (1LL << 31) - 1)
    return fail(nullptr, NPSOLVE_BAD_DIMS, "bad dims");
  cudaStream_t s = (cudaStream_t)stream;
  const Dims d{nx, ny, nz};
  const long long n = d.n();
  float *Q = nullptr, *wv = nullptr;
  double *part = nullptr, *dres = nullptr, *coef = nullptr;
  CK(nullptr, cudaMalloc(&Q, sizeof(float) * (size_t)n * (m + 1)));
  CK(nullptr, cudaMalloc(&wv, sizeof(float) * (size_t)n));
  CK(nullptr, cudaMalloc(&part, sizeof(double) * 148 * 4 * (m + 2)));
  CK(nullptr, cudaMalloc(&dres, sizeof(double) * (m + 2)));
  CK(nullptr, cudaMalloc(&coef, sizeof(double) * (m + 2)));
  std::vector<double> alpha(m, 0.0), beta(m, 0.0), hc(m + 2, 0.0);
  int ret = NPSOLVE_OK;
  // q_1 = start / ||start|| (zero off fluid)
  launch_mask_copy(labels, n, start, wv, s);
  launch_multidot(wv, n, 1, wv, part, dres, s);
  cudaMemcpyAsync(hc.data(), dres, sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if (!(hc[0] > 0.0)) ret = fail(nullptr, NPSOLVE_BAD_ARG, "start vector is zero on the fluid cells");
  int steps = 0;
  if (!ret) {
    hc[0] = 1.0 / sqrt(hc[0]);
    cudaMemcpyAsync(coef, hc.data(), sizeof(double), cudaMemcpyHostToDevice, s);
    launch_combine_basis(wv, n, 1, coef, 0.f, Q, s);
    for (int j = 0; j < m; ++j) {
      float *qj = Q + (size_t)j * n;
      launch_lap(labels, d, qj, wv, s);  // w = A q_j
      // full reorthogonalisation, twice: w -= Q (Q^T w)
      for (int pass = 0; pass < 2; ++pass) {
        launch_multidot(Q, n, j + 1, wv, part, dres, s);
        cudaMemcpyAsync(hc.data(), dres, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        if (pass == 0) alpha[j] = hc[j];
        else alpha[j] += hc[j];
        for (int i = 0; i <= j; ++i) hc[i] = -hc[i];
        cudaMemcpyAsync(coef, hc.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, s);
        launch_combine_basis(Q, n, j + 1, coef, 1.f, wv, s);
      }
      launch_multidot(wv, n, 1, wv, part, dres, s);
      cudaMemcpyAsync(hc.data(), dres, sizeof(double), cudaMemcpyDeviceToHost, s);
      cudaStreamSynchronize(s);
      steps = j + 1;
      beta[j] = sqrt(fmax(hc[0], 0.0));
      if (j + 1 == m || beta[j] < 1e-10) break;
      hc[0] = 1.0 / beta[j];
      cudaMemcpyAsync(coef, hc.data(), sizeof(double), cudaMemcpyHostToDevice, s);
      launch_combine_basis(wv, n, 1, coef, 0.f, Q + (size_t)(j + 1) * n, s);
    }
  }
  double *coefs = nullptr;  // all combinations' basis coefficients (count x steps)
  if (!ret) {
    // Ritz pairs of T = tridiag(beta, alpha, beta)
    const int mm = steps;
    // With every Ritz vector in the combinations (k >= steps) the eigenvectors
    // are not needed: Y is orthogonal, so Y c with c ~ N(0, I) is again
    // N(0, I), and b = Q g / ||g|| with g ~ N(0, I) in the Lanczos basis has
    // the same distribution as the normalised Q Y c.
    const int kk = k < mm ? k : mm;
    const bool all_ritz = kk == mm;
    std::vector<double> ev(alpha.begin(), alpha.begin() + mm), off(mm > 1 ? mm - 1 : 1, 0.0), V;
    for (int i = 0; i + 1 < mm; ++i) off[i] = beta[i];
    if (!tridiag_eigen(ev, off, mm, V, !all_ritz))
      ret = fail(nullptr, NPSOLVE_CUDA_ERROR, "lanczos: tridiagonal eigensolver did not converge");
    std::vector<int> order(mm);
    for (int i = 0; i < mm; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return ev[a] < ev[b]; });
    if (!ret && ritz_values_host)
      for (int i = 0; i < kk; ++i) ritz_values_host[i] = ev[order[i]];
    // count random normalised combinations b = Q Y c, c ~ N(0, 1)
    std::mt19937_64 rng(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    std::vector<double> qcs((size_t)(count > 0 ? count : 1) * mm, 0.0);
    for (int c = 0; c < count && !ret; ++c) {
      std::vector<double> cc(kk);
      double nrm = 0.0;
      for (int i = 0; i < kk; ++i) {
        cc[i] = nd(rng);
        nrm += cc[i] * cc[i];
      }
      nrm = sqrt(nrm);  // Ritz vectors are orthonormal: ||Q Y c|| = ||c||
      double *qc = qcs.data() + (size_t)c * mm;
      if (all_ritz) {
        for (int r = 0; r < mm; ++r) qc[r] = cc[r] / nrm;
        continue;
      }
      for (int r = 0; r < mm; ++r) {
        const double *vr = V.data() + (size_t)r * mm;
        double t = 0.0;
        for (int i = 0; i < kk; ++i) t += vr[order[i]] * cc[i];
        qc[r] = t / nrm;
      }
    }
    if (!ret && count > 0) {
      if (cudaMalloc(&coefs, sizeof(double) * qcs.size()) != cudaSuccess) {
        ret = fail(nullptr, NPSOLVE_OOM, "lanczos: coefficient buffer");
      } else {
        cudaMemcpyAsync(coefs, qcs.data(), sizeof(double) * qcs.size(), cudaMemcpyHostToDevice, s);
        for (int c = 0; c < count; ++c)
          launch_combine_basis(Q, n, mm, coefs + (size_t)c * mm, 0.f, out + (size_t)c * n, s);
      }
    }
  }
  cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(coefs);
  cudaFree(Q);
  cudaFree(wv);
  cudaFree(part);
  cudaFree(dres);
  cudaFree(coef);
  if (!ret && e != cudaSuccess) ret = fail(nullptr, NPSOLVE_CUDA_ERROR, "lanczos: %s", cudaGetErrorString(e));
  return ret;
}

int npsolve_selftest_tensor_core(double *max_abs_err) {
  if (!max_abs_err) return fail(nullptr, NPSOLVE_BAD_ARG, "null argument");
  int dev = 0;
  cudaDeviceProp prop;
  CK(nullptr, cudaGetDevice(&dev));
  CK(nullptr, cudaGetDeviceProperties(&prop, dev));
  if (prop.major * 10 + prop.minor != 103)
    return fail(nullptr, NPSOLVE_CUDA_ERROR, "device is sm_%d%d, not sm_103a", prop.major, prop.minor);
  float *buf = nullptr;
  int *err = nullptr;
  CK(nullptr, cudaMalloc(&buf, 2 * 128 * 32 * sizeof(float)));
  CK(nullptr, cudaMalloc(&err, sizeof(int)));
  CK(nullptr, cudaMemset(err, 0, sizeof(int)));
  launch_umma_selftest(buf, buf + 128 * 32, err, 0);
  std::vector<float> hb(2 * 128 * 32);
  int herr = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(hb.data(), buf, hb.size() * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(buf);
  cudaFree(err);
  CK(nullptr, e);
  if (herr) return fail(nullptr, NPSOLVE_CUDA_ERROR, "tensor-core self-test: MMA wait timed out");
  double m = 0.0;
  for (int i = 0; i < 128 * 32; ++i) m = fmax(m, fabs((double)hb[i] - (double)hb[128 * 32 + i]));
  *max_abs_err = m;
  return NPSOLVE_OK;
}

}  // extern "C"
