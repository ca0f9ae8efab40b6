// Power-of-two FFT engine with the radices, strides and thread mapping fixed
// at compile time (L = 2^p, 256 <= L <= 4096): the unitary DFT F of §5 eq.
// opmodel, applied as 1-D transforms of the rows and of the columns of the
// oversampled grid.
//
// Same Stockham autosort formulation as fft.cuh (stage with radix R after
// stages whose radices multiply to Ns: read R values L/R apart, twiddle by
// exp(-2 pi i r k / (Ns R)), k = j mod Ns, R-point DFT, write Ns apart from
// (j / Ns) Ns R + k; natural-order output), specialised so that
//  * every index split is a shift or a mask, every loop is unrolled;
//  * each thread runs E / R butterflies of a stage, E = elements per thread;
//  * shared memory is padded by one complex value per 16, so the strided
//    writes of the first stages and the strided reads of the column layout
//    fall in distinct banks;
//  * twiddles come from per-stage tables (entry (r - 1) Ns + k of the stage)
//    read through the L1 cache, consecutive across the lanes of a warp;
//  * with HALF_IN the inputs are known to vanish outside e in [0, L/4) and
//    [3L/4, L) (the zero padding Z of an n-point signal centred on a 2n grid),
//    so the first stage loads and transforms only half of its inputs; with
//    HALF_OUT only the outputs in those two ranges are produced (the crop Z^T
//    of the adjoint).
#pragma once

#include "common.cuh"
#include "fft.cuh"

namespace purify {

// -i^k style constants of the 16-point DFT: exp(-2 pi i m / 16), m = 0..9.
__device__ __forceinline__ float2 w16(int m) {
  constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, r2 = 0.70710678118654752f;
  switch (m) {
    case 0: return make_float2(1.f, 0.f);
    case 1: return make_float2(c1, -s1);
    case 2: return make_float2(r2, -r2);
    case 3: return make_float2(s1, -c1);
    case 4: return make_float2(0.f, -1.f);
    case 5: return make_float2(-s1, -c1);
    case 6: return make_float2(-r2, -r2);
    case 7: return make_float2(-c1, -s1);
    case 8: return make_float2(-1.f, 0.f);
    default: return make_float2(-c1, s1);  // m = 9
  }
}

// 16-point DFT in natural order: j = 4 j1 + j2, k = k1 + 4 k2;
// X[k] = sum_j2 w4^(j2 k2) w16^(j2 k1) sum_j1 w4^(j1 k1) x[4 j1 + j2].
template <>
__device__ __forceinline__ void dft_small<16>(float2* v) {
  float2 a[4][4];
#pragma unroll
  for (int j2 = 0; j2 < 4; ++j2) {
    float2 t[4] = {v[j2], v[4 + j2], v[8 + j2], v[12 + j2]};
    dft_small<4>(t);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) a[j2][k1] = (j2 * k1 == 0) ? t[k1] : cmul(t[k1], w16(j2 * k1));
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 t[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
    dft_small<4>(t);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
  }
}

constexpr int p2_log2(int x) { return x <= 1 ? 0 : 1 + p2_log2(x >> 1); }
constexpr int p2_min(int a, int b) { return a < b ? a : b; }
// Radix of stage st: E until fewer than E remain.
constexpr int p2_radix(int L, int E, int st) {
  int rem = L;
  for (int i = 0; i < st; ++i) rem /= p2_min(E, rem);
  return p2_min(E, rem);
}
constexpr int p2_nstages(int L, int E) {
  int n = 0;
  for (int rem = L; rem > 1; rem /= p2_min(E, rem)) ++n;
  return n;
}
constexpr int p2_ns(int L, int E, int st) {
  int ns = 1;
  for (int i = 0; i < st; ++i) ns *= p2_radix(L, E, i);
  return ns;
}
// Offset of stage st's twiddle table in the concatenated tables (stages >= 1).
constexpr int p2_twoff(int L, int E, int st) {
  int off = 0;
  for (int i = 1; i < st; ++i) off += (p2_radix(L, E, i) - 1) * p2_ns(L, E, i);
  return off;
}
constexpr int p2_twsize(int L, int E) { return p2_twoff(L, E, p2_nstages(L, E)); }

// Padded shared-memory index: one complex value of padding per 16.
__device__ __forceinline__ int p2_pad(int i) { return i + (i >> 4); }

// Layout of NSIG signals of length L: signal-major rows, or element-major
// with the signals adjacent (columns of the grid).
template <int L, int NSIG, bool SIG_FAST>
__device__ __forceinline__ int p2_at(int s, int e) {
  if constexpr (SIG_FAST) return p2_pad(e * NSIG + s);
  else return s * (L + L / 16) + p2_pad(e);
}
template <int L, int NSIG>
constexpr size_t p2_smem_bytes() { return (size_t)NSIG * (L + L / 16) * sizeof(float2); }

// Butterfly q of this thread in a stage with L/R butterflies per signal.
template <int L, int R, int NSIG, bool SIG_FAST, int T>
__device__ __forceinline__ void p2_map(int q, int& s, int& j) {
  const int b = threadIdx.x + q * T;
  constexpr int LR = L / R;
  if constexpr (SIG_FAST) {
    s = b & (NSIG - 1);
    j = b >> p2_log2(NSIG);
  } else {
    s = b >> p2_log2(LR);
    j = b & (LR - 1);
  }
}

// Middle stage st (1 <= st < nstages - 1): shared memory to shared memory.
template <int L, int E, int NSIG, bool SIG_FAST, int ST>
__device__ __forceinline__ void p2_stage_mid(float2* buf, const float2* __restrict__ twt) {
  constexpr int R = p2_radix(L, E, ST), NS = p2_ns(L, E, ST), NB = E / R, T = NSIG * L / E;
  constexpr int LR = L / R;
  const float2* tw = twt + p2_twoff(L, E, ST);
  float2 v[NB][R];
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    int s, j;
    p2_map<L, R, NSIG, SIG_FAST, T>(q, s, j);
    const int k = j & (NS - 1);
#pragma unroll
    for (int r = 0; r < R; ++r) v[q][r] = buf[p2_at<L, NSIG, SIG_FAST>(s, j + r * LR)];
#pragma unroll
    for (int r = 1; r < R; ++r) v[q][r] = cmul(v[q][r], __ldg(&tw[(r - 1) * NS + k]));
    dft_small<R>(v[q]);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    int s, j;
    p2_map<L, R, NSIG, SIG_FAST, T>(q, s, j);
    const int k = j & (NS - 1);
    const int base = (j >> p2_log2(NS)) * NS * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) buf[p2_at<L, NSIG, SIG_FAST>(s, base + r * NS)] = v[q][r];
  }
  __syncthreads();
}

template <int L, int E, int NSIG, bool SIG_FAST, int ST>
__device__ __forceinline__ void p2_mid_stages(float2* buf, const float2* __restrict__ twt) {
  if constexpr (ST < p2_nstages(L, E) - 1) {
    p2_stage_mid<L, E, NSIG, SIG_FAST, ST>(buf, twt);
    p2_mid_stages<L, E, NSIG, SIG_FAST, ST + 1>(buf, twt);
  }
}

// The whole transform: inputs from src (first stage, Ns = 1), outputs to dst
// (last stage, Ns = L / R, output index j + r L / R), shared memory between.
// Interfaces as fft_fused (fft.cuh):
//   Src: typename Raw; Raw fetch(s, e) const; void between(); float2 prep(const Raw&, s, e) const
//   Dst: typename Aux; Aux fetch(s, e) const; void put(s, e, float2, const Aux&)
// blockDim.x must be NSIG * L / E.
template <int L, int E, int NSIG, bool SIG_FAST, bool HALF_IN, bool HALF_OUT, class Src, class Dst>
__device__ __forceinline__ void fft_p2(float2* buf, const float2* __restrict__ twt, Src& src, Dst& dst) {
  constexpr int T = NSIG * L / E;
  constexpr int NST = p2_nstages(L, E);
  static_assert(NST >= 2, "at least two stages");
  static_assert((L & (L - 1)) == 0 && (NSIG & (NSIG - 1)) == 0, "powers of two");
  // ---- first stage: radix R0 = E, one butterfly per thread per signal set
  {
    constexpr int R = p2_radix(L, E, 0), NB = E / R, LR = L / R;
    static_assert(!HALF_IN || R >= 4, "pruned inputs need a radix of at least 4");
    typename Src::Raw raw[NB][R];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      int s, j;
      p2_map<L, R, NSIG, SIG_FAST, T>(q, s, j);
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (!HALF_IN || r < R / 4 || r >= 3 * R / 4) raw[q][r] = src.fetch(s, j + r * LR);
    }
    src.between();
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      int s, j;
      p2_map<L, R, NSIG, SIG_FAST, T>(q, s, j);
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r)
        v[r] = (!HALF_IN || r < R / 4 || r >= 3 * R / 4) ? src.prep(raw[q][r], s, j + r * LR) : make_float2(0.f, 0.f);
      dft_small<R>(v);
      // Ns = 1: outputs to j R + r
#pragma unroll
      for (int r = 0; r < R; ++r) buf[p2_at<L, NSIG, SIG_FAST>(s, j * R + r)] = v[r];
    }
  }
  __syncthreads();
  p2_mid_stages<L, E, NSIG, SIG_FAST, 1>(buf, twt);
  // ---- last stage: Ns = L / R, k = j, outputs at j + r L / R
  {
    constexpr int ST = NST - 1;
    constexpr int R = p2_radix(L, E, ST), NS = p2_ns(L, E, ST), NB = E / R, LR = L / R;
    static_assert(NS == LR, "last stage");
    static_assert(!HALF_OUT || R >= 4, "pruned outputs need a radix of at least 4");
    const float2* tw = twt + p2_twoff(L, E, ST);
    typename Dst::Aux aux[NB][R];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      int s, j;
      p2_map<L, R, NSIG, SIG_FAST, T>(q, s, j);
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (!HALF_OUT || r < R / 4 || r >= 3 * R / 4) aux[q][r] = dst.fetch(s, j + r * LR);
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      int s, j;
      p2_map<L, R, NSIG, SIG_FAST, T>(q, s, j);
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = buf[p2_at<L, NSIG, SIG_FAST>(s, j + r * LR)];
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], __ldg(&tw[(r - 1) * NS + j]));
      dft_small<R>(v);
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (!HALF_OUT || r < R / 4 || r >= 3 * R / 4) dst.put(s, j + r * LR, v[r], aux[q][r]);
    }
  }
}

// Host: the concatenated per-stage twiddle tables of (L, E), entry
// (r - 1) Ns + k of stage st = exp(-2 pi i r k / (Ns R)), in double.
template <int L, int E>
inline void p2_twiddles(float2* out) {
  constexpr int NST = p2_nstages(L, E);
  for (int st = 1; st < NST; ++st) {
    const int R = p2_radix(L, E, st), NS = p2_ns(L, E, st);
    float2* t = out + p2_twoff(L, E, st);
    for (int r = 1; r < R; ++r)
      for (int k = 0; k < NS; ++k) {
        const double a = -2.0 * 3.14159265358979323846 * (double)(r * k) / (double)(NS * R);
        t[(r - 1) * NS + k] = make_float2((float)std::cos(a), (float)std::sin(a));
      }
  }
}

}  // namespace purify
