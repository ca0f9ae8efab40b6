// Internal declarations of the sm_103a SDMM-SARA library (not part of the C ABI).
#pragma once

#include <cuda.h>  // CUtensorMap (the map is encoded through the runtime's driver entry point)
#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstddef>
#include <utility>
#include <vector>

#include "purify.h"
#include "gather_plan.h"

namespace purify {

// ---------------------------------------------------------------------------
// Small complex helpers (float2 = complex64).
// ---------------------------------------------------------------------------
// The (re, im) pair is one 64-bit register pair: the packed FP32x2
// instructions of sm_100+ (one FADD2 / FMUL2 / FFMA2 per complex add, scale
// or real-by-complex FMA) round each component exactly as the scalar
// instruction would, so these are bit-identical to the scalar forms.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
// y + s x (s real)
__device__ __forceinline__ float2 caxpy(float s, float2 x, float2 y) { return __ffma2_rn(make_float2(s, s), x, y); }
// a b = a.x (b.x, b.y) + a.y (-b.y, b.x)
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return __ffma2_rn(make_float2(a.y, a.y), make_float2(-b.y, b.x), __fmul2_rn(make_float2(a.x, a.x), b));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// ---------------------------------------------------------------------------
// Kaiser-Bessel kernel as per-tap polynomials.
//
// For a visibility with fractional offset x = kappa - floor(kappa) in [0, 1),
// tap a (cell floor(kappa) - J/2 + 1 + a) has weight g(x + J/2 - 1 - a).  On
// x in [0, 1) that is a smooth function; the host fits it, per tap, by a
// polynomial in z = 2x - 1 (Chebyshev interpolation in double, converted to
// monomials) so the device evaluates J weights by Horner.
// ---------------------------------------------------------------------------
constexpr int kMaxJ = 8;
constexpr int kKbDeg = 8;  // degree of every tap polynomial (fit error <= 1.5e-7 for J <= 8)
struct KbPoly {
  int J;
  float c[kMaxJ][kKbDeg + 1];   // c[a][k]: coefficient of z^k for tap a
  float max_err;                // max abs fit error measured on the host
};

// Error-free splitting of kappa = u * (2n / (2 pi)) into floor and fraction
// with float arithmetic: scale = s_hi + s_lo (double-float), the product
// error is recovered exactly with an FMA.
struct KappaScale {
  float hi, lo;
};

__device__ __forceinline__ void split_kappa(float u, KappaScale s, int& k, float& frac) {
  float p = u * s.hi;
  float e = fmaf(u, s.hi, -p) + u * s.lo;  // exact product error + low part
  float fl = floorf(p);
  float f = (p - fl) + e;                  // p - fl is exact
  if (f < 0.0f) { f += 1.0f; fl -= 1.0f; }
  else if (f >= 1.0f) { f -= 1.0f; fl += 1.0f; }
  k = (int)fl;
  frac = f;
}

// Weights w[a], a = 0..J-1, for fractional offset x in [0, 1).
template <int J>
__device__ __forceinline__ void kb_weights(const KbPoly& kb, float x, float* w) {
  const float z = fmaf(2.0f, x, -1.0f);
#pragma unroll
  for (int a = 0; a < J; ++a) {
    float acc = kb.c[a][kKbDeg];
#pragma unroll
    for (int k = kKbDeg - 1; k >= 0; --k) acc = fmaf(acc, z, kb.c[a][k]);
    w[a] = acc;
  }
}

// floor(k / d) for 0 <= k < 2^16 and 1 <= d <= 128 from the rounded
// reciprocal r = 1/d: (k + 1/2) r lies at least 1/(2d) from an integer and
// its rounding error is below 2^-22 (k + 1/2)/d, so truncation is exact
// (checked exhaustively over that range by a host test).
__device__ __forceinline__ int quot_small(int k, float r) {
  return __float2int_rz(__fmul_rn(__fadd_rn((float)k, 0.5f), r));
}

__device__ __forceinline__ int wrap(int k, int L) {
  k %= L;
  return k < 0 ? k + L : k;
}

// ---------------------------------------------------------------------------
// Division by a divisor of the form 2^sh or 3 * 2^sh without an integer
// divide: q = x >> sh, then q / 3 as the high half of q * ceil(2^33 / 3).
// Every index split in the FFT passes (by L, n, the signal count, L/R and
// the Stockham span Ns) has this form.
// ---------------------------------------------------------------------------
struct Div {
  int d;
  int sh;
  int three;
};

__host__ __device__ inline Div make_div(int d) {
  Div v{d, 0, 0};
  int r = d;
  if (r % 3 == 0) {
    v.three = 1;
    r /= 3;
  }
  while (r > 1) {
    r >>= 1;
    ++v.sh;
  }
  return v;
}

__device__ __forceinline__ int udiv(int x, const Div& v) {
  const unsigned q = (unsigned)x >> v.sh;
  return v.three ? (int)(__umulhi(q, 0xAAAAAAABu) >> 1) : (int)q;
}

// ---------------------------------------------------------------------------
// FFT plan: Stockham stages with radices in {2, 3, 4, 8}.
// ---------------------------------------------------------------------------
struct FftPlan {
  int L;
  int nst;
  int radix[24];
  Div ns[24];   // Ns of each stage (product of the earlier radices)
  Div lr[24];   // L / R of each stage
  Div divL;
};

// Fill the per-stage divisors of a plan whose radix list is set.
inline void finish_plan(FftPlan& p) {
  int ns = 1;
  for (int st = 0; st < p.nst; ++st) {
    p.ns[st] = make_div(ns);
    p.lr[st] = make_div(p.L / p.radix[st]);
    ns *= p.radix[st];
  }
  p.divL = make_div(p.L);
}

// ---------------------------------------------------------------------------
// Daubechies filters (db1..db8), generated on the host at library load.
// h of db_p starts at off[p] and has 2p taps; the high-pass is derived.
// ---------------------------------------------------------------------------
struct WaveletFilters {
  float h[72];
  int off[9];
};

// ---------------------------------------------------------------------------
// Device scalars of the reductions (FP64) and the SDMM bookkeeping.
// ---------------------------------------------------------------------------
enum CounterSlot {
  kCntDot = 0,     // <p, Qp>
  kCntRho,         // ||r||^2
  kCntL2,          // ||s2 + z2 - y||^2 and ||s2 - y||^2
  kCntF1,          // sum w |alpha|
  kCntMax,         // max |.|
  kCntNorm,        // generic ||a - b||^2
  kCntRho0,        // ||r0||^2 after an SDMM step
  kCntBlk,         // per-block ||s2 + z2 - y||^2, ||s2 - y||^2 (distributed form)
  kNumCounters
};

struct DevScalars {
  double rho;        // current <r, r>
  double alpha;      // CG step
  double beta;       // CG direction update
  double pqp;        // <p, Qp>
  double l2_dn2;     // ||s2 + z2 - y||^2
  double l2_res2;    // ||s2 - y||^2
  double l2_scale;   // min(1, eps / ||s2 + z2 - y||)
  double f1;         // sum w |Psi^H x|
  double f1_prev;
  double amax;       // max |.| reductions
  double norm2;      // generic squared norm
  double gamma;      // penalty
  double eps;        // l2 bound
  double zeta, nu;   // halting quantities (nu: the largest block's in the distributed form)
  double nu_min;     // smallest block's nu (= nu for one ball)
  double iters;
  double cg_res;
  double cg_rho[2];   // gamma and alpha of CG steps j - 1 and j, by parity of j
  double cg_alpha[2];
  int cg_step_first;  // the step sizes in alpha, beta are those of a first step
  int dev_error;      // nonzero when a bounded device wait gave up (reported as PURIFY_E_TIMEOUT)
  unsigned int counter[kNumCounters];
};



// Static plus dynamic shared memory above 48 KB needs a per-kernel opt-in
// (the kernels' static shared memory is well under 8 KB).
template <class K>
inline void allow_smem(K kernel, size_t bytes) {
  if (bytes > 40 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

constexpr int kMaxPartials = 32768;  // blocks per reduction (NV <= 2 values each)
constexpr int kMaxBlocks = 4096;     // data blocks of the distributed form

// ---------------------------------------------------------------------------
// Kernel timing: when enabled on a context, every launch is bracketed by two
// CUDA events on its stream; collect() aggregates the durations per kernel.
// A process-wide counter counts every kernel launch of the library.
// ---------------------------------------------------------------------------
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<std::pair<const char*, size_t>> recs;  // kernel name, index of its start event
};

extern std::atomic<unsigned long long> g_launches;

}  // namespace purify

// ---------------------------------------------------------------------------
// The context (opaque to callers).
// ---------------------------------------------------------------------------
// Shared-memory layout of one gridding chunk (k_grid): per entry the value
// and the zero-padded row and column kernel weights (stride kept odd against
// bank conflicts); per CTA the prefix of the cell blocks' work and two
// partial-sum slots per thread.
namespace purify {
__host__ __device__ constexpr int grid_wstride(int J) { return 2 * (J + 2) + 1; }
__host__ __device__ constexpr size_t grid_entry_bytes(int J) { return 8 + 4 * (size_t)grid_wstride(J); }
// The partial-sum slots share their space with the grid halo that the Gram
// form (G^T G in one pass) stages before the entries.
// Halo of the Gram form: T + 2(J - 1) rows of T + 2(J - 1) + 2 cells (the TMA
// box starts one column early so that its first column is even, i.e. its
// start 16-byte aligned, and its width stays even).
__host__ __device__ constexpr int grid_halo_w(int T, int J) { return T + 2 * (J - 1); }
__host__ __device__ constexpr int grid_halo_ws(int T, int J) { return T + 2 * (J - 1) + 2; }
__host__ __device__ constexpr size_t grid_halo_bytes(int T, int J) {
  return (size_t)grid_halo_w(T, J) * grid_halo_ws(T, J) * 8;
}
__host__ __device__ constexpr size_t grid_slot_bytes(int T, int J) {
  return grid_halo_bytes(T, J) > (size_t)2 * kGridThreads * 32 ? (grid_halo_bytes(T, J) + 15) / 16 * 16
                                                                : (size_t)2 * kGridThreads * 32;
}
__host__ __device__ constexpr size_t grid_fixed_bytes(int T, int J) {
  return grid_slot_bytes(T, J) + (size_t)((T / 2) * (T / 2) + 1) * 4;
}
// Shared-memory budget of one gridding CTA: the chunks of a tile's list are
// sized so that the kernel fits 56 KB (four CTAs per SM, a 64-register
// build).  Measured at 1024^2 (Gram / gridding launch): 72 KB, three CTAs per
// SM: 139 / 154 us; 44 KB, five: 131 / 154 us; 56 KB, four: 129.5 / 146 us.
// The gather is latency-bound, so resident warps matter, but smaller chunks
// split more tiles into several chunks (partial tiles and their merge).
// offsets d = (dr, dc) >= 0 (lexicographic) of a half G^T G stencil
__host__ __device__ constexpr int dense_gram_slices(int J) { return J + (J - 1) * (2 * J - 1); }
#ifndef PURIFY_GRID_SMEM_BUDGET_KB
#define PURIFY_GRID_SMEM_BUDGET_KB 56
#endif
constexpr size_t kGridSmemBudget = PURIFY_GRID_SMEM_BUDGET_KB * 1024;
// 16-bit per-chunk table of the gather: the NO + 1 owner-work prefix values
// (stride rounded to 8 entries = 16 bytes)
__host__ __device__ constexpr int grid_tab_stride(int T) { return ((T / 2) * (T / 2) + 1 + 7) / 8 * 8; }
}  // namespace purify

struct purify_ctx {
  int device;
  int sms;               // streaming multiprocessors of the device
  int n, L, J, levels, q;
  int kernel;           // PURIFY_KERNEL_KB or PURIFY_KERNEL_GAUSS
  float2* d_tv;         // 7 N scratch of the TV prox (input, two dual pairs ping-ponged, last dual pair)
  float2* d_diff;       // scratch of the differentiation calls (3 M + 4 N + D), allocated on first use
  float* d_beam;        // primary beam B (N floats), allocated by the first purify_set_beam
  bool beam_on;         // B applied (otherwise B = I)
  int beam_version;     // bumped by every purify_set_beam (graphs re-capture)
  int64_t M;
  uint32_t mask;
  int bases[9];  // basis index (0 = Dirac, p = db_p) of each plane

  purify::KbPoly kb;
  purify::KappaScale ks;
  purify::FftPlan plan;
  purify::WaveletFilters wf;

  float* d_deapod;      // n: 1 / g_hat((r - n/2) / 2n)
  float2* d_tw;         // L: exp(-2 pi i m / L)
  int fft_engine;       // 1: compile-time power-of-two engine (L = 256 .. 4096), 0: generic Stockham
  float2* d_twp[2];     // per-stage twiddle tables of the power-of-two engine (8 and 16 per thread)

  // visibility table (sorted by grid tile of the first footprint cell)
  float2* d_uv;         // M sorted frequencies
  int* d_perm;          // sorted position -> caller position
  int tileT;            // tile side (cells)
  int tiles_1d;         // L / tileT
  int ntiles;
  int4* d_list;         // per tile, the visibilities whose footprint meets it, by start cell:
                        // (sorted index, start-cell key, kappa fractions of row and column as float bits)
  int64_t nlist;
  // gridding work units: each tile's list cut into chunks of at most chunk_max entries;
  // a tile with several chunks sums their partial tiles (slots) in chunk order
  int nchunks;
  int chunk_max;
  int4* d_chunks;       // (tile, begin, end, slot or -1)
  uint16_t* d_chunk_tab; // per chunk: owner-work prefix (grid_tab_stride entries)
  int chunk_tab_stride;
  uint32_t* d_items;    // per chunk, the gather steps of its threads (grid_item), step-major:
                        // step s of thread j at d_items[(item_row[chunk] + s) * kGridThreads + j]
  int* d_item_row;      // per chunk, its first row of d_items
  int64_t nitem_rows;
  int* d_tile_slot0;    // first slot of a multi-chunk tile
  int* d_tile_nchunk;   // chunks per tile
  unsigned* d_tile_cnt; // arrival counters (zero between launches)
  int nslots;
  float2* d_slots;      // nslots x tileT^2 partial tiles
  // dense tiles of the Gram pass: G^T G stored per cell as a (2J - 1)^2
  // stencil (§5 proposes precomputing G^H G for the CG solve), applied in the
  // Gram launch's first n_dense CTAs; the other CTAs run the gather over the
  // chunks of the remaining tiles (gram_chunks)
  int n_dense;
  int* d_dense_tiles;   // tile of each dense CTA
  int dense_half;       // 1: d_H holds half stencils (build_dense_gram_half), 0: full ones
  float* d_H;           // full: n_dense x (2J - 1)^2 x T^2: H[t][d][cell], d = (dr + J - 1)(2J - 1) + dc + J - 1;
                        // half: n_dense x dense_gram_slices(J) x (T + J - 1)(T + 2J - 2)
  int n_gram_chunks;
  int* d_gram_chunks;   // chunks of the tiles that are not dense
  // degridding work units: (tile, begin, end, -) runs of home visibilities
  int ndchunks;
  int4* d_dchunks;

  // scratch
  CUtensorMap halo_map; // TMA map of d_grid: one box = the halo of one interior tile of the Gram pass
  int halo_map_ok;      // the map was encoded (the Gram pass stages interior halos with TMA)
  float2* d_grid;       // L x L
  float2* d_grid2;      // L x L: output of the Gram pass (G^T G reads d_grid)
  float2* d_half;       // n x L (rows of the image after the row pass)
  float2* d_vis;        // M (sorted order)
  float2* d_vis2;       // M
  float2* d_ll[2];      // q x (n/2)^2 each: low-low ping-pong of the DWT
  float2* d_img[4];     // N each: CG work vectors of purify_cg_solve
  double* d_partials;   // kNumCounters x kMaxPartials
  purify::DevScalars* d_sc;
  purify::DevScalars* h_sc;  // pinned host mirror

  purify::Profiler prof;
};

namespace purify {

// Bracket one kernel launch (see Profiler).
inline size_t prof_start(purify_ctx* c, cudaStream_t s) {
  if (!c || !c->prof.on) return (size_t)-1;
  while (c->prof.pool.size() < c->prof.used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return (size_t)-1;
    c->prof.pool.push_back(e);
  }
  const size_t i = c->prof.used;
  cudaEventRecord(c->prof.pool[i], s);
  c->prof.used += 2;
  return i;
}

inline void prof_stop(purify_ctx* c, const char* name, cudaStream_t s, size_t i) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (i == (size_t)-1) return;
  cudaEventRecord(c->prof.pool[i + 1], s);
  c->prof.recs.emplace_back(name, i);
}

}  // namespace purify

// Launch statement `stmt` (a kernel launch) under the profiler.
#define PURIFY_LAUNCH(ctx, name, stream, stmt)                \
  do {                                                        \
    const size_t _pi = purify::prof_start((ctx), (stream));   \
    stmt;                                                     \
    purify::prof_stop((ctx), (name), (stream), _pi);          \
  } while (0)

namespace purify {
// What a captured SDMM step depends on besides the state's fixed buffers: a
// graph whose key differs from the state's current key must be re-captured.
struct GraphKey {
  int cg_iters = -1;
  int y_bf16 = 0;
  int shape = -1;  // purify_sdmm_state::shape_version
  int beam = -1;   // purify_ctx::beam_version
  bool operator==(const GraphKey& o) const {
    return cg_iters == o.cg_iters && y_bf16 == o.y_bf16 && shape == o.shape && beam == o.beam;
  }
  bool operator!=(const GraphKey& o) const { return !(*this == o); }
};
}  // namespace purify

struct purify_sdmm_state {
  purify_ctx* ctx;
  // image-size vectors
  float2* xhat;   // N
  float2* r;      // N  CG residual
  float2* p;      // N  CG direction
  float2* qp;     // N  w = Q r
  float2* sv;     // N  s = Q p (single-reduction CG)
  float2* x1;     // N  Psi u1
  float2* z3;     // N
  // coefficient-size vectors
  float2* z1;     // D
  float2* u1;     // D
  float* w;       // D weights
  // visibility-size vectors (sorted order)
  float2* y;      // M data
  uint16_t* yb;   // 2M bf16 data (when bf16)
  float* yscale;  // ceil(M/4096)
  int y_bf16;
  float2* z2;     // M
  float2* s2;     // M   Phi x_hat
  float2* v;      // M   u2 - Phi x_hat
  double eps;
  int64_t iters;
  purify_sdmm_params params;
  // CUDA graph of one SDMM step (captured on a private stream, replayed on the caller's)
  cudaStream_t cap_stream;
  cudaStream_t side;        // the SDMM prior branch (i = 1), concurrent with the data branch
  cudaEvent_t ev_fork, ev_join;
  cudaGraphExec_t step_exec;
  // distributed form (§4.5 eq. dbp1): R balls over consecutive caller-order
  // blocks of the visibilities; nblocks = 0 is the single ball of eq. delta
  int nblocks;
  int* d_block_of;          // M, sorted order: block of each visibility
  int* d_pos;               // M, caller order: sorted position
  int4* d_bchunks;          // (block, caller begin, caller end, first chunk of the block)
  int nbchunks;
  double* d_beps;           // R bounds eps_i
  float* d_bscale;          // R projection factors min(1, eps_i / ||a_i - y_i||)
  int prior;                // PURIFY_PRIOR_SARA or PURIFY_PRIOR_TV
  int fgp_iters;            // TV prox inner iterations
  int shape_version;        // bumped by every call that changes what one step launches or the
                            // buffers its kernels read (prior, blocks, data format, import)
  purify::GraphKey graph_key;  // key of the captured per-state graph
  int launches_per_step;    // kernels in one captured step
};

namespace purify {

// Launchers (implemented in the .cu files).
int check_cuda(cudaError_t e);
int enqueue_sdmm_step(purify_ctx* c, purify_sdmm_state* st, cudaStream_t s);  // capi.cu
GraphKey step_graph_key(const purify_sdmm_state* st);                          // capi.cu

// nufft.cu
// kRowInCgUpd: apply the pending CG vector update, then transform r;
// kRowInCgFinish: apply it, then transform x.
enum RowInMode { kRowInPlain = 0, kRowInCgUpd = 1, kRowInCgFinish = 2 };
enum DegridOut { kDegridPerm = 0, kDegridSorted = 1, kDegridSdmm = 2 };
enum GridIn { kGridPerm = 0, kGridSorted = 1, kGridGram = 2 };
enum RowOutMode { kRowOutPlain = 0, kRowOutCgQ = 1, kRowOutSdmm = 2 };

struct RowInArgs {
  const float2* in;     // plain: the image to transform
  // CG (single-reduction form): the pending update of step i-1 is
  //   p = r + beta p; s = w + beta s; x += alpha p; r -= alpha s
  float2* x;
  float2* r;
  float2* p;
  float2* s;
  const float2* w;
};
struct DegridArgs {
  float2* out;              // y (perm) or sorted output
  const float2* z2;         // sdmm
  const float2* y;          // sdmm data (sorted) or NULL when bf16
  const uint16_t* yb;       // sdmm bf16 data
  const float* yscale;
};
struct RowOutArgs {
  float2* out;          // plain: image; cg: w = Q r; sdmm: r0
  const float2* p;      // cg: r (the vector Q is applied to); sdmm: x_hat
  const float2* x1;     // sdmm: Psi u1
  float2* z3;           // sdmm
};

int fft_prepare(purify_ctx* c);  // tables of the power-of-two FFT engine (at context creation)
// cg_j: in the CG modes, the CG step whose update this pass applies (its
// inner-product partials are in the kCntDot slot).
int phi_forward_grid(purify_ctx* c, RowInMode mode, const RowInArgs& a, cudaStream_t s, int cg_j = 0);
int cg_partial_blocks(const purify_ctx* c);
// CG step sizes formed by the consuming kernels (few partials) or by a
// one-block kernel after the inverse row pass (many partials: at 256
// partials, e.g. 1024^2, every block of the 1024-block forward row pass
// summing them cost 9 us per CG step against ~2 us for the extra launch).
constexpr int kCgConsumeMaxBlocks = 128;
int cg_consumer_blocks(const purify_ctx* c);  // nblk for the consumers: the partial count, or 0
int launch_cg_scalars(purify_ctx* c, int cg_j, cudaStream_t s);
int degrid(purify_ctx* c, DegridOut mode, const DegridArgs& a, cudaStream_t s);
int grid_adjoint(purify_ctx* c, GridIn mode, const float2* vis, cudaStream_t s);
int gram_grid(purify_ctx* c, cudaStream_t s);
int phi_adjoint_image(purify_ctx* c, RowOutMode mode, const RowOutArgs& a, cudaStream_t s,
                      const float2* grid = nullptr, cudaEvent_t before_rows = nullptr);

// sara.cu
enum SaraMode { kSaraPlain = 0, kSaraProx = 1 };
struct SaraProxArgs {
  float2* z1;
  float2* u1;
  const float* w;       // NULL = 1
};
// Prox mode: the analysis leaves per-block partials of f1 (in the kCntF1
// slot) and returns their count in *f1_parts; the synthesis launched next
// with that count forms f1 and zeta in an extra block (no ticket, no fence in
// the analysis).  *f1_parts = 0: the analysis formed them itself.
int sara_analysis(purify_ctx* c, const float2* x, float2* alpha, SaraMode mode,
                  const SaraProxArgs& pa, cudaStream_t s, int* f1_parts = nullptr);
int sara_synthesis(purify_ctx* c, const float2* alpha, float2* x, cudaStream_t s, int f1_parts = 0);
void make_daubechies(WaveletFilters& wf);

// vecops.cu
int launch_soft_threshold(int64_t count, const float2* in, const float* w, const double* gamma_dev,
                          float gamma, float2* out, cudaStream_t s);
int launch_l2_norm_diff(purify_ctx* c, int64_t count, const float2* a, const float2* b, cudaStream_t s);
int launch_l2_project(int64_t count, const float2* in, const float2* y, double eps,
                      const double* norm2_dev, float2* out, cudaStream_t s);
int launch_positive(int64_t count, const float2* in, float2* out, cudaStream_t s);
int launch_cg_apply(purify_ctx* c, float2* x, float2* r, float2* p, float2* sv, const float2* w, int cg_j,
                    cudaStream_t s);
int launch_cg_residual_init(purify_ctx* c, const float2* b, const float2* qx, float2* r, cudaStream_t s);
int launch_max_abs(purify_ctx* c, int64_t count, const float2* a, cudaStream_t s);
int launch_sdmm_l2_update(purify_sdmm_state* st, cudaStream_t s);
int launch_block_norms(purify_sdmm_state* st, cudaStream_t s);
int tv_sdmm_branch(purify_ctx* c, purify_sdmm_state* st, cudaStream_t s);
int tv_scratch_ready(purify_ctx* c, float2** out);
int tv_gradmag(purify_ctx* c, const float2* x, float2** g, cudaStream_t s);
int tv_prox(purify_ctx* c, const float2* in, const float* w, float lam, int iters, float2* out, cudaStream_t s);
int launch_reweight(purify_ctx* c, int64_t count, const float2* alpha, float* w, int round,
                    cudaStream_t s);
int launch_quantize_bf16(int64_t M, const float2* y, uint16_t* yb, float* yscale, cudaStream_t s);
int launch_gather_perm(int64_t M, const float2* src, const int* perm, float2* dst, cudaStream_t s);
int launch_set_gamma(purify_ctx* c, double beta, cudaStream_t s);

}  // namespace purify
