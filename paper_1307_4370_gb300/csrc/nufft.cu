// The FFT side of Phi = G F D Z B (§5 eq. opmodel) and its adjoint; the
// interpolation G and G^T are in gridding.cu.
//
// Forward:  k_row_fwd   B, D, Z and the row DFTs of the n non-zero grid rows
//                       (the zero padding is never written);
//           k_col_fwd   column DFTs, reading only the n non-zero rows.
// Adjoint:  k_col_inv   inverse column DFTs, keeping the n rows of the image;
//           k_row_inv   inverse row DFTs, crop Z^T, D and B, with fused
//                       epilogues for the CG operator Q = Phi^H Phi + 2I and
//                       the SDMM step.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "fft_p2.cuh"
#include "reduce.cuh"

namespace purify {

// ---------------------------------------------------------------------------
// Launch shapes
// ---------------------------------------------------------------------------
struct FftShape {
  int ept;      // elements per thread (8, 12 or 16)
  int nsig;     // signals per CTA
  int threads;  // nsig * L / ept
};

static int pick_ept(int L) { return (L % 3 == 0) ? 12 : 8; }

// Row passes: nsig rows per CTA, at most 256 threads (16 elements per thread
// for L = 4096), nsig divides n.
static FftShape row_shape(const purify_ctx* c) {
  FftShape f;
  f.ept = pick_ept(c->L);
  if (f.ept == 8 && c->L / 8 > 256) f.ept = 16;
  int nsig = 1;
  while (nsig * 2 * c->L / f.ept <= 128 && c->n % (nsig * 2) == 0) nsig *= 2;
  f.nsig = nsig;
  f.threads = nsig * c->L / f.ept;
  return f;
}

// Column passes: nsig adjacent columns per CTA (>= 4 for 32-byte segments).
static FftShape col_shape(const purify_ctx* c) {
  FftShape f;
  f.ept = pick_ept(c->L);
  int nsig = 4;
  while (nsig * 2 * c->L / f.ept <= 256 && c->L % (nsig * 2) == 0 && nsig < 16) nsig *= 2;
  while (nsig > 1 && nsig * c->L / f.ept > 1024) nsig /= 2;  // at most 1024 threads
  f.nsig = nsig;
  f.threads = nsig * c->L / f.ept;
  return f;
}

// ---------------------------------------------------------------------------
// Forward row pass: g[r][e] = v[r][c] / (ghat_r ghat_c) / L at e = (c - n/2) mod L,
// then the row DFT; rows stored in `half` (n x L).  In the CG modes the pixel
// first receives the pending vector update of the previous CG step
// (single-reduction CG: p = r + beta p, s = w + beta s, x += alpha p,
// r -= alpha s), and v is the new r (kRowInCgUpd) or x (kRowInCgFinish).
// ---------------------------------------------------------------------------
struct EmptyAux {};

struct RawPlain {
  float2 v;
  float f;
  int off;  // pixel index, or -1 in the zero padding
};
struct RawCg {
  float2 r, w, p, s, x;
  float f;
  int off;
};

template <int MODE>
struct RowFwdSrc {
  using Raw = typename std::conditional<MODE == kRowInPlain, RawPlain, RawCg>::type;
  RowInArgs a;
  const float* dz;
  const float* beam;  // primary beam B (N), or null
  int n, L, r0;
  float invL, alpha, beta;
  bool first;
  // CG modes: inner-product partials of the previous CG step j
  const double* cgpart;
  int cg_nblk, cg_j;
  DevScalars* sc;
  __device__ __forceinline__ void between() {}
  __device__ __forceinline__ Raw fetch(int s, int e) const {
    Raw o;
    const int row = r0 + s;
    int cc = e + (n >> 1);
    if (cc >= L) cc -= L;
    o.off = -1;
    if (cc < n) {
      o.off = row * n + cc;
      o.f = __ldg(&dz[row]) * __ldg(&dz[cc]) * invL;
      if (beam) o.f *= __ldg(&beam[o.off]);
      if constexpr (MODE == kRowInPlain) {
        o.v = a.in[o.off];
      } else {
        o.r = a.r[o.off];
        o.w = a.w[o.off];
        if (!first) {
          o.p = a.p[o.off];
          o.s = a.s[o.off];
        }
        o.x = a.x[o.off];
      }
    }
    return o;
  }
  __device__ __forceinline__ float2 prep(const Raw& o, int, int) const {
    if (o.off < 0) return make_float2(0.f, 0.f);
    if constexpr (MODE == kRowInPlain) {
      return cscale(o.v, o.f);
    } else {
      float2 pp = o.r, ss = o.w;
      if (!first) {
        pp = caxpy(beta, o.p, o.r);
        ss = caxpy(beta, o.s, o.w);
      }
      const float2 xx = caxpy(alpha, pp, o.x);
      const float2 rn = caxpy(-alpha, ss, o.r);
      a.p[o.off] = pp;
      a.s[o.off] = ss;
      a.x[o.off] = xx;
      a.r[o.off] = rn;
      return cscale(MODE == kRowInCgUpd ? rn : xx, o.f);
    }
  }
};

struct RowStoreDst {  // row-major rows of length L
  using Aux = EmptyAux;
  float2* out;
  int L;
  __device__ __forceinline__ Aux fetch(int, int) const { return Aux{}; }
  __device__ __forceinline__ void put(int s, int e, float2 v, const Aux&) { out[(size_t)s * L + e] = v; }
};

template <int EPT, int MODE>
__global__ void __launch_bounds__(256) k_row_fwd(RowInArgs a, float2* __restrict__ half, const float* __restrict__ dz,
                                                 const float* __restrict__ beam, const float2* __restrict__ tw,
                                                 FftPlan plan, int n, int nsig, DevScalars* sc,
                                                 const double* __restrict__ cgpart, int cg_nblk, int cg_j) {
  extern __shared__ float2 sm[];
  const int L = plan.L;
  RowFwdSrc<MODE> src;
  src.a = a;
  src.dz = dz;
  src.beam = beam;
  src.n = n;
  src.L = L;
  src.r0 = blockIdx.x * nsig;
  src.invL = 1.0f / (float)L;
  src.alpha = src.beta = 0.f;
  src.first = false;
  src.cgpart = cgpart;
  src.cg_nblk = cg_nblk;
  src.cg_j = cg_j;
  src.sc = sc;
  if constexpr (MODE != kRowInPlain) {
    // step sizes of the pending update, before any data load is in flight
    // (overlapping them costs registers, hence occupancy, in this pass)
    const CgStep st = cg_consume(cgpart, cg_nblk, cg_j, sc);
    src.alpha = st.alpha;
    src.beta = st.beta;
    src.first = st.first;
  }
  RowStoreDst dst{half + (size_t)src.r0 * L, L};
  fft_fused<EPT, false>(sm, SigLayout{L, 1}, plan, nsig, sm + nsig * L, tw, src, dst);
}

// ---------------------------------------------------------------------------
// Forward column pass: column c of the grid holds half[r][c] at row
// (r - n/2) mod L and zeros elsewhere; DFT along the column into X.
// ---------------------------------------------------------------------------
struct ColFwdSrc {
  using Raw = float2;
  __device__ __forceinline__ void between() {}
  const float2* half;
  int n, L, c0;
  __device__ __forceinline__ Raw fetch(int s, int e) const {
    int r = e + (n >> 1);
    if (r >= L) r -= L;
    return r < n ? half[(size_t)r * L + c0 + s] : make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ float2 prep(const Raw& v, int, int) const { return v; }
};

struct ColStoreDst {  // column c0 + s of an L x L grid
  using Aux = EmptyAux;
  float2* X;
  int L, c0;
  __device__ __forceinline__ Aux fetch(int, int) const { return Aux{}; }
  __device__ __forceinline__ void put(int s, int e, float2 v, const Aux&) { X[(size_t)e * L + c0 + s] = v; }
};

template <int EPT>
__global__ void __launch_bounds__(1024) k_col_fwd(const float2* __restrict__ half, float2* __restrict__ X,
                                                  const float2* __restrict__ tw, FftPlan plan, int n, int nsig) {
  extern __shared__ float2 sm[];
  const int L = plan.L;
  const int c0 = blockIdx.x * nsig;
  ColFwdSrc src{half, n, L, c0};
  ColStoreDst dst{X, L, c0};
  fft_fused<EPT, true>(sm, SigLayout{1, nsig}, plan, nsig, sm + nsig * L, tw, src, dst);
}

// ---------------------------------------------------------------------------
// Inverse column pass: inverse DFT of columns of X (by conjugation), keep rows
// (r - n/2) mod L.
// ---------------------------------------------------------------------------
struct ColInvSrc {
  using Raw = float2;
  __device__ __forceinline__ void between() {}
  const float2* X;
  int L, c0;
  __device__ __forceinline__ Raw fetch(int s, int e) const { return X[(size_t)e * L + c0 + s]; }
  __device__ __forceinline__ float2 prep(const Raw& v, int, int) const { return cconj(v); }
};

struct ColCropDst {
  using Aux = EmptyAux;
  float2* half;
  int n, L, c0;
  __device__ __forceinline__ Aux fetch(int, int) const { return Aux{}; }
  __device__ __forceinline__ void put(int s, int e, float2 v, const Aux&) {
    int r = e + (n >> 1);
    if (r >= L) r -= L;
    if (r < n) half[(size_t)r * L + c0 + s] = cconj(v);
  }
};

template <int EPT>
__global__ void __launch_bounds__(1024) k_col_inv(const float2* __restrict__ X, float2* __restrict__ half,
                                                  const float2* __restrict__ tw, FftPlan plan, int n, int nsig) {
  extern __shared__ float2 sm[];
  const int L = plan.L;
  const int c0 = blockIdx.x * nsig;
  ColInvSrc src{X, L, c0};
  ColCropDst dst{half, n, L, c0};
  fft_fused<EPT, true>(sm, SigLayout{1, nsig}, plan, nsig, sm + nsig * L, tw, src, dst);
}

// ---------------------------------------------------------------------------
// Inverse row pass, crop and deapodise, with epilogues:
//   plain: out = Phi^H (.)
//   CG:    w = Q r = Phi^H Phi r + 2r with gamma = <r, r> and delta = <w, r>
//          (FP64, one reduction); the last block forms the step sizes of
//          single-reduction CG (Chronopoulos & Gear 1989):
//          beta = gamma / gamma_prev, alpha = gamma / (delta - beta gamma / alpha_prev)
//   SDMM:  positivity branch (z3, u3) and the warm-start CG residual
//          r0 = x1 + u3 - 2 x_hat + Phi^H v
// ---------------------------------------------------------------------------
struct RowInvSrc {
  using Raw = float2;
  __device__ __forceinline__ void between() {}
  const float2* half;
  int L, r0;
  __device__ __forceinline__ Raw fetch(int s, int e) const { return half[(size_t)(r0 + s) * L + e]; }
  __device__ __forceinline__ float2 prep(const Raw& v, int, int) const { return cconj(v); }
};

struct AuxPix {
  float2 p, z3, x1;
  float f;
  int off;  // pixel index, or -1 outside the crop
};

template <int MODE>
struct RowInvDst {
  using Aux = AuxPix;
  RowOutArgs a;
  const float* dz;
  const float* beam;  // primary beam B (N), or null
  int n, L, r0;
  float invL;
  FPair part[2];  // per-thread exact sums of a few terms; FP64 across threads
  __device__ __forceinline__ Aux fetch(int s, int e) const {
    Aux o;
    const int row = r0 + s;
    int c = e + (n >> 1);
    if (c >= L) c -= L;
    o.off = -1;
    if (c < n) {
      o.off = row * n + c;
      o.f = __ldg(&dz[row]) * __ldg(&dz[c]) * invL;
      if (beam) o.f *= __ldg(&beam[o.off]);
      if (MODE != kRowOutPlain) o.p = a.p[o.off];
      if (MODE == kRowOutSdmm) {
        o.z3 = a.z3[o.off];
        o.x1 = a.x1[o.off];
      }
    }
    return o;
  }
  __device__ __forceinline__ void put(int, int, float2 w, const Aux& o) {
    if (o.off < 0) return;
    const float2 v = cscale(cconj(w), o.f);
    if (MODE == kRowOutPlain) {
      a.out[o.off] = v;
    } else if (MODE == kRowOutCgQ) {
      const float2 p = o.p;
      const float2 q = caxpy(2.f, p, v);
      a.out[o.off] = q;
      part[0].add_prod(p.x, p.x);  // <r, r>
      part[0].add_prod(p.y, p.y);
      part[1].add_prod(p.x, q.x);  // Re <w, r>
      part[1].add_prod(p.y, q.y);
    } else {
      const float2 xh = o.p;
      const float2 a3 = cadd(xh, o.z3);
      const float r3 = fmaxf(a3.x, 0.f);
      const float2 z3n = make_float2(a3.x - r3, a3.y);  // a3 - r3
      const float2 u3 = make_float2(r3 - z3n.x, -z3n.y);
      float2 r0v;
      r0v.x = o.x1.x + u3.x - 2.f * xh.x + v.x;
      r0v.y = o.x1.y + u3.y - 2.f * xh.y + v.y;
      a.z3[o.off] = z3n;
      a.out[o.off] = r0v;
    }
  }
};

template <int EPT, int MODE>
__global__ void __launch_bounds__(256) k_row_inv(const float2* __restrict__ half, RowOutArgs a,
                                                 const float* __restrict__ dz, const float* __restrict__ beam,
                                                 const float2* __restrict__ tw, FftPlan plan, int n, int nsig,
                                                 double* partials, DevScalars* sc) {
  extern __shared__ float2 sm[];
  const int L = plan.L;
  const int r0 = blockIdx.x * nsig;
  RowInvSrc src{half, L, r0};
  RowInvDst<MODE> dst;
  dst.a = a;
  dst.dz = dz;
  dst.beam = beam;
  dst.n = n;
  dst.L = L;
  dst.r0 = r0;
  dst.invL = 1.0f / (float)L;
  fft_fused<EPT, false>(sm, SigLayout{L, 1}, plan, nsig, sm + nsig * L, tw, src, dst);
  if (MODE == kRowOutCgQ) {
    // per-block partials of gamma = <r, r> and delta = <Qr, r>; the kernel
    // that applies this step's update adds them and forms the step sizes
    double acc[2] = {dst.part[0].value(), dst.part[1].value()};
    block_reduce<2>(acc);
    if (threadIdx.x == 0) {
      partials[kCntDot * 2 * kMaxPartials + blockIdx.x] = acc[0];
      partials[kCntDot * 2 * kMaxPartials + kMaxPartials + blockIdx.x] = acc[1];
    }
  }
}

// ---------------------------------------------------------------------------
// The same four passes on power-of-two grids (L = 256 .. 4096) with the
// compile-time engine of fft_p2.cuh: the zero padding of the forward passes
// and the crop of the adjoint ones prune the first / last stage.
// ---------------------------------------------------------------------------
#ifndef P2_E_LARGE
#define P2_E_LARGE 16
#endif
#ifndef P2_E_CG
#define P2_E_CG 8
#endif
#ifndef P2_NS_COL
#define P2_NS_COL (L == 2048 ? 8 : 4)  // at most 1024 threads: NS L / E
#endif
#ifndef P2_ROWCG_THREADS
#define P2_ROWCG_THREADS 256
#endif
#ifndef P2_RINV_THREADS
#define P2_RINV_THREADS 512
#endif
template <int L>
struct P2Cfg {
  static constexpr int E = L >= 1024 ? P2_E_LARGE : 8;             // plain row, column and inverse row passes
  static constexpr int E_CG = P2_E_CG;                             // forward row pass with the CG update
  static constexpr int NS_ROW = 256 / (L / E) > 0 ? 256 / (L / E) : 1;
  static constexpr int NS_ROWCG = P2_ROWCG_THREADS / (L / E_CG) > 0 ? P2_ROWCG_THREADS / (L / E_CG) : 1;
  static constexpr int NS_RINV =
      P2_RINV_THREADS / (L / E) > 0 ? (P2_RINV_THREADS / (L / E) > 8 ? 8 : P2_RINV_THREADS / (L / E)) : 1;
  static constexpr int NS_COL = P2_NS_COL;
};

template <int L, int E, int NSIG, int MODE>
__global__ void __launch_bounds__(NSIG * L / E) k_row_fwd_p2(RowInArgs a, float2* __restrict__ half,
                                                             const float* __restrict__ dz,
                                                             const float* __restrict__ beam,
                                                             const float2* __restrict__ twt, int n, DevScalars* sc,
                                                             const double* __restrict__ cgpart, int cg_nblk,
                                                             int cg_j) {
  extern __shared__ float2 sm[];
  RowFwdSrc<MODE> src;
  src.a = a;
  src.dz = dz;
  src.beam = beam;
  src.n = n;
  src.L = L;
  src.r0 = blockIdx.x * NSIG;
  src.invL = 1.0f / (float)L;
  src.alpha = src.beta = 0.f;
  src.first = false;
  src.cgpart = cgpart;
  src.cg_nblk = cg_nblk;
  src.cg_j = cg_j;
  src.sc = sc;
  if constexpr (MODE != kRowInPlain) {
    const CgStep st = cg_consume(cgpart, cg_nblk, cg_j, sc);
    src.alpha = st.alpha;
    src.beta = st.beta;
    src.first = st.first;
  }
  RowStoreDst dst{half + (size_t)src.r0 * L, L};
  fft_p2<L, E, NSIG, false, true, false>(sm, twt, src, dst);
}

template <int L, int E, int NSIG>
__global__ void __launch_bounds__(NSIG * L / E) k_col_fwd_p2(const float2* __restrict__ half, float2* __restrict__ X,
                                                             const float2* __restrict__ twt, int n) {
  extern __shared__ float2 sm[];
  const int c0 = blockIdx.x * NSIG;
  ColFwdSrc src{half, n, L, c0};
  ColStoreDst dst{X, L, c0};
  fft_p2<L, E, NSIG, true, true, false>(sm, twt, src, dst);
}

template <int L, int E, int NSIG>
__global__ void __launch_bounds__(NSIG * L / E) k_col_inv_p2(const float2* __restrict__ X, float2* __restrict__ half,
                                                             const float2* __restrict__ twt, int n) {
  extern __shared__ float2 sm[];
  const int c0 = blockIdx.x * NSIG;
  ColInvSrc src{X, L, c0};
  ColCropDst dst{half, n, L, c0};
  fft_p2<L, E, NSIG, true, false, true>(sm, twt, src, dst);
}

// Register cap: two CTAs per SM for the CG and plain epilogues; the SDMM
// epilogue (five operands per pixel) keeps its registers.
constexpr int p2_rinv_minb(int T, int MODE) { return MODE == kRowOutSdmm ? 1 : (1024 / T > 1 ? 1024 / T : 1); }

template <int L, int E, int NSIG, int MODE>
__global__ void __launch_bounds__(NSIG * L / E, p2_rinv_minb(NSIG * L / E, MODE)) k_row_inv_p2(const float2* __restrict__ half, RowOutArgs a,
                                                             const float* __restrict__ dz,
                                                             const float* __restrict__ beam,
                                                             const float2* __restrict__ twt, int n,
                                                             double* partials) {
  extern __shared__ float2 sm[];
  const int r0 = blockIdx.x * NSIG;
  RowInvSrc src{half, L, r0};
  RowInvDst<MODE> dst;
  dst.a = a;
  dst.dz = dz;
  dst.beam = beam;
  dst.n = n;
  dst.L = L;
  dst.r0 = r0;
  dst.invL = 1.0f / (float)L;
  fft_p2<L, E, NSIG, false, false, true>(sm, twt, src, dst);
  if (MODE == kRowOutCgQ) {
    double acc[2] = {dst.part[0].value(), dst.part[1].value()};
    block_reduce<2>(acc);
    if (threadIdx.x == 0) {
      partials[kCntDot * 2 * kMaxPartials + blockIdx.x] = acc[0];
      partials[kCntDot * 2 * kMaxPartials + kMaxPartials + blockIdx.x] = acc[1];
    }
  }
}

// Whether the grid side has the compile-time engine.
static bool p2_side(int L) { return L == 256 || L == 512 || L == 1024 || L == 2048 || L == 4096; }

// Concatenated twiddle tables of the engine for (L, E) (device, owned by the context).
template <int L, int E>
static int p2_table(purify_ctx* c, const float2** out) {
  const int idx = (E == 16) ? 1 : 0;
  if (!c->d_twp[idx]) {
    std::vector<float2> t(std::max(1, p2_twsize(L, E)));
    p2_twiddles<L, E>(t.data());
    float2* d = nullptr;
    if (cudaMalloc((void**)&d, t.size() * sizeof(float2)) != cudaSuccess) return PURIFY_E_ALLOC;
    if (cudaMemcpy(d, t.data(), t.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(d);
      return PURIFY_E_CUDA;
    }
    c->d_twp[idx] = d;
  }
  *out = c->d_twp[idx];
  return PURIFY_OK;
}

template <int L>
static int p2_prepare_L(purify_ctx* c) {
  const float2* t;
  if (int rc = p2_table<L, P2Cfg<L>::E>(c, &t)) return rc;
  return p2_table<L, P2Cfg<L>::E_CG>(c, &t);
}

// Twiddle tables of the power-of-two engine, built when the context is
// created (never inside a stream capture).
int fft_prepare(purify_ctx* c) {
  if (c->fft_engine != 1) return PURIFY_OK;
  switch (c->L) {
    case 256: return p2_prepare_L<256>(c);
    case 512: return p2_prepare_L<512>(c);
    case 1024: return p2_prepare_L<1024>(c);
    case 2048: return p2_prepare_L<2048>(c);
    case 4096: return p2_prepare_L<4096>(c);
    default: c->fft_engine = 0; return PURIFY_OK;
  }
}

template <int L>
static int p2_forward(purify_ctx* c, RowInMode mode, const RowInArgs& a, cudaStream_t s, int cg_j,
                      const float* beam) {
  using C = P2Cfg<L>;
  const float2 *tw, *twcg;
  if (int rc = p2_table<L, C::E>(c, &tw)) return rc;
  if (int rc = p2_table<L, C::E_CG>(c, &twcg)) return rc;
  const double* cgpart = c->d_partials + kCntDot * 2 * kMaxPartials;
  const int cg_nblk = cg_consumer_blocks(c);
  const int n = c->n;
  if (mode == kRowInPlain) {
    constexpr int NS = C::NS_ROW;
    constexpr size_t sm = p2_smem_bytes<L, NS>();
    allow_smem(k_row_fwd_p2<L, C::E, NS, kRowInPlain>, sm);
    PURIFY_LAUNCH(c, "row_fwd", s,
                  (k_row_fwd_p2<L, C::E, NS, kRowInPlain><<<n / NS, NS * L / C::E, sm, s>>>(
                      a, c->d_half, c->d_deapod, beam, tw, n, c->d_sc, cgpart, cg_nblk, cg_j)));
  } else {
    constexpr int NS = C::NS_ROWCG;
    constexpr size_t sm = p2_smem_bytes<L, NS>();
#define ROWCG(MD)                                                                                         \
  do {                                                                                                    \
    allow_smem(k_row_fwd_p2<L, C::E_CG, NS, MD>, sm);                                                     \
    PURIFY_LAUNCH(c, "row_fwd", s,                                                                        \
                  (k_row_fwd_p2<L, C::E_CG, NS, MD><<<n / NS, NS * L / C::E_CG, sm, s>>>(                  \
                      a, c->d_half, c->d_deapod, beam, twcg, n, c->d_sc, cgpart, cg_nblk, cg_j)));          \
  } while (0)
    if (mode == kRowInCgUpd) ROWCG(kRowInCgUpd);
    else ROWCG(kRowInCgFinish);
#undef ROWCG
  }
  {
    constexpr int NS = C::NS_COL;
    constexpr size_t sm = p2_smem_bytes<L, NS>();
    allow_smem(k_col_fwd_p2<L, C::E, NS>, sm);
    PURIFY_LAUNCH(c, "col_fwd", s,
                  (k_col_fwd_p2<L, C::E, NS><<<L / NS, NS * L / C::E, sm, s>>>(c->d_half, c->d_grid, tw, n)));
  }
  return check_cuda(cudaGetLastError());
}

template <int L>
static int p2_adjoint(purify_ctx* c, RowOutMode mode, const RowOutArgs& a, cudaStream_t s, const float2* Xg,
                      cudaEvent_t before_rows, const float* beam) {
  using C = P2Cfg<L>;
  const float2* tw;
  if (int rc = p2_table<L, C::E>(c, &tw)) return rc;
  const int n = c->n;
  {
    constexpr int NS = C::NS_COL;
    constexpr size_t sm = p2_smem_bytes<L, NS>();
    allow_smem(k_col_inv_p2<L, C::E, NS>, sm);
    PURIFY_LAUNCH(c, "col_inv", s, (k_col_inv_p2<L, C::E, NS><<<L / NS, NS * L / C::E, sm, s>>>(Xg, c->d_half, tw, n)));
  }
  if (before_rows) {
    const int rc = check_cuda(cudaStreamWaitEvent(s, before_rows, 0));
    if (rc != PURIFY_OK) return rc;
  }
  constexpr int NS = C::NS_RINV;
  constexpr size_t sm = p2_smem_bytes<L, NS>();
#define ROWI2(MD)                                                                                          \
  do {                                                                                                     \
    allow_smem(k_row_inv_p2<L, C::E, NS, MD>, sm);                                                         \
    PURIFY_LAUNCH(c, "row_inv", s,                                                                         \
                  (k_row_inv_p2<L, C::E, NS, MD><<<n / NS, NS * L / C::E, sm, s>>>(c->d_half, a, c->d_deapod, \
                                                                                     beam, tw, n,            \
                                                                                     c->d_partials)));       \
  } while (0)
  if (mode == kRowOutPlain) ROWI2(kRowOutPlain);
  else if (mode == kRowOutCgQ) ROWI2(kRowOutCgQ);
  else ROWI2(kRowOutSdmm);
#undef ROWI2
  return check_cuda(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
// Blocks of the inverse row pass, i.e. the CG inner-product partials it leaves.
int cg_partial_blocks(const purify_ctx* c) {
  switch (p2_side(c->L) ? c->L : 0) {
    case 256: return c->n / P2Cfg<256>::NS_RINV;
    case 512: return c->n / P2Cfg<512>::NS_RINV;
    case 1024: return c->n / P2Cfg<1024>::NS_RINV;
    case 2048: return c->n / P2Cfg<2048>::NS_RINV;
    case 4096: return c->n / P2Cfg<4096>::NS_RINV;
    default: return c->n / row_shape(c).nsig;
  }
}

int cg_consumer_blocks(const purify_ctx* c) {
  const int nb = cg_partial_blocks(c);
  return nb <= kCgConsumeMaxBlocks ? nb : 0;
}

// One block: the step sizes of CG step j from the partials, for consumers
// that read them (cg_consumer_blocks == 0).
__global__ void __launch_bounds__(256) k_cg_scalars(const double* __restrict__ part, int nblk, int j, DevScalars* sc) {
  cg_consume(part, nblk, j, sc);
}

int launch_cg_scalars(purify_ctx* c, int cg_j, cudaStream_t s) {
  PURIFY_LAUNCH(c, "cg_scalars", s,
                (k_cg_scalars<<<1, 256, 0, s>>>(c->d_partials + kCntDot * 2 * kMaxPartials, cg_partial_blocks(c), cg_j,
                                               c->d_sc)));
  return check_cuda(cudaGetLastError());
}

int phi_forward_grid(purify_ctx* c, RowInMode mode, const RowInArgs& a, cudaStream_t s, int cg_j) {
  const float* beam = c->beam_on ? c->d_beam : nullptr;
  if (c->fft_engine == 1) {
    switch (c->L) {
      case 256: return p2_forward<256>(c, mode, a, s, cg_j, beam);
      case 512: return p2_forward<512>(c, mode, a, s, cg_j, beam);
      case 1024: return p2_forward<1024>(c, mode, a, s, cg_j, beam);
      case 2048: return p2_forward<2048>(c, mode, a, s, cg_j, beam);
      case 4096: return p2_forward<4096>(c, mode, a, s, cg_j, beam);
      default: break;
    }
  }
  const FftShape rs = row_shape(c), cs = col_shape(c);
  const double* cgpart = c->d_partials + kCntDot * 2 * kMaxPartials;
  const int cg_nblk = cg_consumer_blocks(c);
  const size_t smr = (size_t)(rs.nsig + 1) * c->L * sizeof(float2);
  const size_t smc = (size_t)(cs.nsig + 1) * c->L * sizeof(float2);
  const int gr = c->n / rs.nsig, gc = c->L / cs.nsig;
#define ROWF(E, MD)                                                                                        \
  do {                                                                                                     \
    allow_smem(k_row_fwd<E, MD>, smr);                                                                     \
    PURIFY_LAUNCH(c, "row_fwd", s,                                                                         \
                  (k_row_fwd<E, MD><<<gr, rs.threads, smr, s>>>(a, c->d_half, c->d_deapod, beam, c->d_tw, c->plan, \
                                                                c->n, rs.nsig, c->d_sc, cgpart, cg_nblk, cg_j)));   \
  } while (0)
  if (rs.ept == 8) {
    if (mode == kRowInPlain) ROWF(8, kRowInPlain);
    else if (mode == kRowInCgUpd) ROWF(8, kRowInCgUpd);
    else ROWF(8, kRowInCgFinish);
  } else if (rs.ept == 16) {
    if (mode == kRowInPlain) ROWF(16, kRowInPlain);
    else if (mode == kRowInCgUpd) ROWF(16, kRowInCgUpd);
    else ROWF(16, kRowInCgFinish);
  } else {
    if (mode == kRowInPlain) ROWF(12, kRowInPlain);
    else if (mode == kRowInCgUpd) ROWF(12, kRowInCgUpd);
    else ROWF(12, kRowInCgFinish);
  }
#undef ROWF
  if (cs.ept == 8) {
    allow_smem(k_col_fwd<8>, smc);
    PURIFY_LAUNCH(c, "col_fwd", s,
                  (k_col_fwd<8><<<gc, cs.threads, smc, s>>>(c->d_half, c->d_grid, c->d_tw, c->plan, c->n, cs.nsig)));
  } else {
    allow_smem(k_col_fwd<12>, smc);
    PURIFY_LAUNCH(c, "col_fwd", s,
                  (k_col_fwd<12><<<gc, cs.threads, smc, s>>>(c->d_half, c->d_grid, c->d_tw, c->plan, c->n, cs.nsig)));
  }
  return check_cuda(cudaGetLastError());
}


int phi_adjoint_image(purify_ctx* c, RowOutMode mode, const RowOutArgs& a, cudaStream_t s, const float2* grid,
                      cudaEvent_t before_rows) {
  const float* beam = c->beam_on ? c->d_beam : nullptr;
  const float2* Xg = grid ? grid : c->d_grid;
  if (c->fft_engine == 1) {
    switch (c->L) {
      case 256: return p2_adjoint<256>(c, mode, a, s, Xg, before_rows, beam);
      case 512: return p2_adjoint<512>(c, mode, a, s, Xg, before_rows, beam);
      case 1024: return p2_adjoint<1024>(c, mode, a, s, Xg, before_rows, beam);
      case 2048: return p2_adjoint<2048>(c, mode, a, s, Xg, before_rows, beam);
      case 4096: return p2_adjoint<4096>(c, mode, a, s, Xg, before_rows, beam);
      default: break;
    }
  }
  const FftShape rs = row_shape(c), cs = col_shape(c);
  const size_t smr = (size_t)(rs.nsig + 1) * c->L * sizeof(float2);
  const size_t smc = (size_t)(cs.nsig + 1) * c->L * sizeof(float2);
  const int gr = c->n / rs.nsig, gc = c->L / cs.nsig;
  if (cs.ept == 8) {
    allow_smem(k_col_inv<8>, smc);
    PURIFY_LAUNCH(c, "col_inv", s,
                  (k_col_inv<8><<<gc, cs.threads, smc, s>>>(Xg, c->d_half, c->d_tw, c->plan, c->n, cs.nsig)));
  } else {
    allow_smem(k_col_inv<12>, smc);
    PURIFY_LAUNCH(c, "col_inv", s,
                  (k_col_inv<12><<<gc, cs.threads, smc, s>>>(Xg, c->d_half, c->d_tw, c->plan, c->n, cs.nsig)));
  }
  // the row pass may read operands of another stream (the SDMM prior branch)
  if (before_rows) {
    const int rc = check_cuda(cudaStreamWaitEvent(s, before_rows, 0));
    if (rc != PURIFY_OK) return rc;
  }
#define ROWI(E, MD)                                                                                          \
  do {                                                                                                       \
    allow_smem(k_row_inv<E, MD>, smr);                                                                       \
    PURIFY_LAUNCH(c, "row_inv", s,                                                                           \
                  (k_row_inv<E, MD><<<gr, rs.threads, smr, s>>>(c->d_half, a, c->d_deapod, beam, c->d_tw, c->plan, \
                                                                c->n, rs.nsig, c->d_partials, c->d_sc)));     \
  } while (0)
  if (rs.ept == 8) {
    if (mode == kRowOutPlain) ROWI(8, kRowOutPlain);
    else if (mode == kRowOutCgQ) ROWI(8, kRowOutCgQ);
    else ROWI(8, kRowOutSdmm);
  } else if (rs.ept == 16) {
    if (mode == kRowOutPlain) ROWI(16, kRowOutPlain);
    else if (mode == kRowOutCgQ) ROWI(16, kRowOutCgQ);
    else ROWI(16, kRowOutSdmm);
  } else {
    if (mode == kRowOutPlain) ROWI(12, kRowOutPlain);
    else if (mode == kRowOutCgQ) ROWI(12, kRowOutCgQ);
    else ROWI(12, kRowOutSdmm);
  }
#undef ROWI
  return check_cuda(cudaGetLastError());
}

}  // namespace purify
