// Shared-memory Stockham FFT building blocks (forward sign; inverse by conjugation).
//
// The unitary DFT F of §5 eq. opmodel, X[k] = (1/L) sum_j g[j] exp(-2 pi i k.j / L)
// per axis pair, is computed as 1-D transforms of rows and of columns.  One CTA
// holds `nsig` signals of length L in shared memory and runs the Stockham
// autosort stages on them: stage (radix R, Ns = product of earlier radices)
// reads R values spaced L/R apart, twiddles them by exp(-2 pi i r k / (Ns R)),
// k = j mod Ns, does a radix-R DFT and writes them Ns apart from
// (j / Ns) Ns R + k.  The output is in natural order.
#pragma once

#include "common.cuh"

namespace purify {

template <int R>
__device__ __forceinline__ void dft_small(float2* v);

template <>
__device__ __forceinline__ void dft_small<2>(float2* v) {
  float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

// -i * a
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }

template <>
__device__ __forceinline__ void dft_small<4>(float2* v) {
  float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
  float2 a2 = cadd(v[1], v[3]), a3 = mul_mi(csub(v[1], v[3]));
  v[0] = cadd(a0, a2);
  v[2] = csub(a0, a2);
  v[1] = cadd(a1, a3);
  v[3] = csub(a1, a3);
}

template <>
__device__ __forceinline__ void dft_small<3>(float2* v) {
  const float h = 0.8660254037844386f;  // sqrt(3)/2
  float2 s = cadd(v[1], v[2]);
  float2 d = csub(v[1], v[2]);
  float2 t = make_float2(fmaf(-0.5f, s.x, v[0].x), fmaf(-0.5f, s.y, v[0].y));
  float2 m = make_float2(h * d.y, -h * d.x);  // -i sqrt(3)/2 d
  v[0] = cadd(v[0], s);
  v[1] = cadd(t, m);
  v[2] = csub(t, m);
}

template <>
__device__ __forceinline__ void dft_small<8>(float2* v) {
  const float r = 0.70710678118654752f;
  // radix-4 on evens and odds, then combine with exp(-2 pi i k / 8)
  float2 e[4] = {v[0], v[2], v[4], v[6]};
  float2 o[4] = {v[1], v[3], v[5], v[7]};
  dft_small<4>(e);
  dft_small<4>(o);
  float2 o1 = make_float2(r * (o[1].x + o[1].y), r * (o[1].y - o[1].x));   // * (1 - i)/sqrt2
  float2 o2 = mul_mi(o[2]);                                               // * -i
  float2 o3 = make_float2(r * (o[3].y - o[3].x), -r * (o[3].x + o[3].y));  // * (-1 - i)/sqrt2
  v[0] = cadd(e[0], o[0]);
  v[4] = csub(e[0], o[0]);
  v[1] = cadd(e[1], o1);
  v[5] = csub(e[1], o1);
  v[2] = cadd(e[2], o2);
  v[6] = csub(e[2], o2);
  v[3] = cadd(e[3], o3);
  v[7] = csub(e[3], o3);
}

// Shared-memory address of element e of signal s.
struct SigLayout {
  int sstride;  // between signals
  int estride;  // between elements of one signal
  __device__ __forceinline__ int at(int s, int e) const { return s * sstride + e * estride; }
};

// One Stockham stage over all signals held by the CTA.  Each thread owns
// EPT / R butterflies; butterfly b maps to (signal, j) either signal-fastest
// (SIG_FAST, for column transforms where signals are adjacent in memory) or
// element-fastest.  Butterflies beyond nsig * L / R (when the CTA has more
// threads than the signals need) are skipped.
template <int R, int EPT, bool SIG_FAST>
__device__ __forceinline__ void stockham_stage(float2* buf, SigLayout lay, int L, const Div& ns, const Div& lr,
                                               const Div& dsig, int nsig, const float2* tw) {
  static_assert(EPT % R == 0, "radix must divide elements per thread");
  constexpr int NB = EPT / R;
  const int nthr = blockDim.x;
  const int LR = lr.d;
  const int Ns = ns.d;
  const int nbfly = nsig * LR;
  const int twstep = L / (Ns * R);
  float2 v[EPT];
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    const int b = threadIdx.x + k * nthr;
    if (b < nbfly) {
      int s, j;
      if (SIG_FAST) { j = udiv(b, dsig); s = b - j * nsig; }
      else { s = udiv(b, lr); j = b - s * LR; }
      const int kk = j - udiv(j, ns) * Ns;
#pragma unroll
      for (int r = 0; r < R; ++r) v[k * R + r] = buf[lay.at(s, j + r * LR)];
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[k * R + r] = cmul(v[k * R + r], tw[r * kk * twstep]);
      }
      dft_small<R>(&v[k * R]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    const int b = threadIdx.x + k * nthr;
    if (b < nbfly) {
      int s, j;
      if (SIG_FAST) { j = udiv(b, dsig); s = b - j * nsig; }
      else { s = udiv(b, lr); j = b - s * LR; }
      const int jq = udiv(j, ns);
      const int kk = j - jq * Ns;
      const int base = jq * Ns * R + kk;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[lay.at(s, base + r * Ns)] = v[k * R + r];
    }
  }
  __syncthreads();
}

// Forward FFT of all signals in shared memory (in place, natural order).
template <int EPT, bool SIG_FAST>
__device__ __forceinline__ void fft_smem(float2* buf, SigLayout lay, const FftPlan& plan, int nsig,
                                         const float2* __restrict__ tw) {
  const Div dsig = make_div(nsig);
  for (int st = 0; st < plan.nst; ++st) {
    const int R = plan.radix[st];
    const Div& ns = plan.ns[st];
    const Div& lr = plan.lr[st];
    if constexpr (EPT % 8 == 0) {
      if (R == 8) { stockham_stage<8, EPT, SIG_FAST>(buf, lay, plan.L, ns, lr, dsig, nsig, tw); continue; }
    }
    if constexpr (EPT % 4 == 0) {
      if (R == 4) { stockham_stage<4, EPT, SIG_FAST>(buf, lay, plan.L, ns, lr, dsig, nsig, tw); continue; }
    }
    if constexpr (EPT % 3 == 0) {
      if (R == 3) { stockham_stage<3, EPT, SIG_FAST>(buf, lay, plan.L, ns, lr, dsig, nsig, tw); continue; }
    }
    if constexpr (EPT % 2 == 0) {
      if (R == 2) { stockham_stage<2, EPT, SIG_FAST>(buf, lay, plan.L, ns, lr, dsig, nsig, tw); continue; }
    }
  }
}

// ---------------------------------------------------------------------------
// Fused driver: the first stage (Ns = 1) reads its inputs from global memory
// and the last stage (Ns = L / R) hands its outputs to global memory, so a
// transform costs one shared-memory pass less on each side.  Every thread
// issues all of its global loads (inputs and twiddles) before it uses any of
// them.
//
//   Src: typename Raw; Raw fetch(s, e) const;  void between();  float2 prep(const Raw&, s, e) const
//   Dst: typename Aux; Aux fetch(s, e) const;  void put(s, e, float2, const Aux&)
// (s = signal, e = element; Src::between runs in every thread after the first
// stage's loads are issued, for block-wide work they can overlap; Dst::fetch
// runs before the last stage's arithmetic so the epilogue operands are in
// flight meanwhile.)
// ---------------------------------------------------------------------------
template <int R, int EPT, bool SIG_FAST, class Src>
__device__ __forceinline__ void stage_first(float2* buf, SigLayout lay, const Div& lr, const Div& dsig, int nsig,
                                            Src& src, float2* tws, const float2 (&twr)[EPT], int L) {
  constexpr int NB = EPT / R;
  const int LR = lr.d;
  const int nbfly = nsig * LR;
  typename Src::Raw raw[EPT];
  int ss[NB], jj[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    const int b = threadIdx.x + k * blockDim.x;
    int s = 0, j = 0;
    if (b < nbfly) {
      if (SIG_FAST) { j = udiv(b, dsig); s = b - j * nsig; }
      else { s = udiv(b, lr); j = b - s * LR; }
#pragma unroll
      for (int r = 0; r < R; ++r) raw[k * R + r] = src.fetch(s, j + r * LR);
    }
    ss[k] = s;
    jj[k] = j;
  }
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int i = threadIdx.x + k * blockDim.x;
    if (i < L) tws[i] = twr[k];
  }
  src.between();  // block-wide work that overlaps the loads in flight (all threads)
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    const int b = threadIdx.x + k * blockDim.x;
    if (b < nbfly) {
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = src.prep(raw[k * R + r], ss[k], jj[k] + r * LR);
      dft_small<R>(v);
#pragma unroll
      for (int r = 0; r < R; ++r) buf[lay.at(ss[k], jj[k] * R + r)] = v[r];
    }
  }
}

template <int R, int EPT, bool SIG_FAST, class Dst>
__device__ __forceinline__ void stage_last(const float2* buf, SigLayout lay, const Div& lr, const Div& dsig, int nsig,
                                           const float2* tw, Dst& dst) {
  constexpr int NB = EPT / R;
  const int LR = lr.d;
  const int nbfly = nsig * LR;
  typename Dst::Aux aux[EPT];
  int ss[NB], jj[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    const int b = threadIdx.x + k * blockDim.x;
    int s = 0, j = 0;
    if (b < nbfly) {
      if (SIG_FAST) { j = udiv(b, dsig); s = b - j * nsig; }
      else { s = udiv(b, lr); j = b - s * LR; }
#pragma unroll
      for (int r = 0; r < R; ++r) aux[k * R + r] = dst.fetch(s, j + r * LR);
    }
    ss[k] = s;
    jj[k] = j;
  }
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    const int b = threadIdx.x + k * blockDim.x;
    if (b < nbfly) {
      const int j = jj[k];
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = buf[lay.at(ss[k], j + r * LR)];
      // last stage: Ns = L / R, so k = j and the twiddle step is 1
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[r * j]);
      dft_small<R>(v);
#pragma unroll
      for (int r = 0; r < R; ++r) dst.put(ss[k], j + r * LR, v[r], aux[k * R + r]);
    }
  }
}

// Forward FFT of nsig signals of length L (at least two stages): inputs from
// `src`, outputs to `dst`, `buf` holds the signals in between and `tws` gets
// the L twiddles exp(-2 pi i t / L) copied from `tw`.
template <int EPT, bool SIG_FAST, class Src, class Dst>
__device__ __forceinline__ void fft_fused(float2* buf, SigLayout lay, const FftPlan& plan, int nsig, float2* tws,
                                          const float2* __restrict__ tw, Src& src, Dst& dst) {
  const Div dsig = make_div(nsig);
  const int L = plan.L;
  float2 twr[EPT];
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int i = threadIdx.x + k * blockDim.x;
    if (i < L) twr[k] = __ldg(&tw[i]);
  }
  {
    const int R = plan.radix[0];
    const Div& lr = plan.lr[0];
    if constexpr (EPT % 8 == 0) { if (R == 8) stage_first<8, EPT, SIG_FAST>(buf, lay, lr, dsig, nsig, src, tws, twr, L); }
    if constexpr (EPT % 4 == 0) { if (R == 4) stage_first<4, EPT, SIG_FAST>(buf, lay, lr, dsig, nsig, src, tws, twr, L); }
    if constexpr (EPT % 3 == 0) { if (R == 3) stage_first<3, EPT, SIG_FAST>(buf, lay, lr, dsig, nsig, src, tws, twr, L); }
    if constexpr (EPT % 2 == 0) { if (R == 2) stage_first<2, EPT, SIG_FAST>(buf, lay, lr, dsig, nsig, src, tws, twr, L); }
  }
  __syncthreads();
  for (int st = 1; st < plan.nst - 1; ++st) {
    const int R = plan.radix[st];
    const Div& ns = plan.ns[st];
    const Div& lr = plan.lr[st];
    if constexpr (EPT % 8 == 0) {
      if (R == 8) { stockham_stage<8, EPT, SIG_FAST>(buf, lay, L, ns, lr, dsig, nsig, tws); continue; }
    }
    if constexpr (EPT % 4 == 0) {
      if (R == 4) { stockham_stage<4, EPT, SIG_FAST>(buf, lay, L, ns, lr, dsig, nsig, tws); continue; }
    }
    if constexpr (EPT % 3 == 0) {
      if (R == 3) { stockham_stage<3, EPT, SIG_FAST>(buf, lay, L, ns, lr, dsig, nsig, tws); continue; }
    }
    if constexpr (EPT % 2 == 0) {
      if (R == 2) { stockham_stage<2, EPT, SIG_FAST>(buf, lay, L, ns, lr, dsig, nsig, tws); continue; }
    }
  }
  {
    const int R = plan.radix[plan.nst - 1];
    const Div& lr = plan.lr[plan.nst - 1];
    if constexpr (EPT % 8 == 0) { if (R == 8) stage_last<8, EPT, SIG_FAST>(buf, lay, lr, dsig, nsig, tws, dst); }
    if constexpr (EPT % 4 == 0) { if (R == 4) stage_last<4, EPT, SIG_FAST>(buf, lay, lr, dsig, nsig, tws, dst); }
    if constexpr (EPT % 3 == 0) { if (R == 3) stage_last<3, EPT, SIG_FAST>(buf, lay, lr, dsig, nsig, tws, dst); }
    if constexpr (EPT % 2 == 0) { if (R == 2) stage_last<2, EPT, SIG_FAST>(buf, lay, lr, dsig, nsig, tws, dst); }
  }
}

}  // namespace purify
