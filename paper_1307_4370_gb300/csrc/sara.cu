// SARA dictionary (§3.3): Psi = (1/sqrt q) [Dirac, db1, ..., db8], Psi^H its adjoint.
//
// Each Daubechies plane is a periodic, separable, orthonormal 2-D DWT in
// Mallat layout.  One launch per level processes every wavelet basis at once
// (grid.z = basis): a CTA loads the input region its coefficient tile needs
// (with periodic wrap, also when the filter is longer than the signal),
// filters rows then columns in shared memory, and writes the four sub-bands.
// The synthesis runs the transpose level by level; its finest level sums all
// bases and the Dirac plane in the same CTA, so x is written once.  In prox
// mode the analysis epilogue applies the weighted soft threshold of §4.4
// eq. prox1 and the dual update of Algorithm 1 steps 7-9 to each final
// coefficient as it is produced, so alpha itself is never stored; each
// block leaves one FP64 partial of f1, and the first synthesis launch that
// follows sums them into f1 and the halting quantity zeta (§4.4).
#include <cmath>
#include <complex>
#include <vector>

#include "common.cuh"
#include "reduce.cuh"

namespace purify {

constexpr int kTile = 16;     // coefficient tile (analysis) / half output tile (synthesis)

struct LevelGeom {
  int tile;     // coefficient tile side (analysis) / half output tile (synthesis); divides L/2
  int n;        // image side (plane row stride)
  int L;        // input side of this analysis level / output side of this synthesis level
  int nb;       // wavelet planes in the launch
  int plane0;   // index of the first wavelet plane in the coefficient array
  int last;     // analysis: last level (LL goes to the plane); synthesis: finest level
  float scale;  // 1 / sqrt(q)
  int first;    // analysis: first level
  int dirac;    // analysis, first level: plane of the Dirac basis handled by the CTAs with z = nb, or -1
  int f1_off;   // analysis, prox mode: index of this launch's first f1 partial
};

struct BasisList {
  int p[8];     // Daubechies order of wavelet plane k
};

// Soft threshold + dual update for one final coefficient alpha at index j;
// returns w |alpha| (its term of f1), summed per thread in FP32 (a few terms)
// and across threads in FP64.
// The same with z1_j and w_j already loaded.
__device__ __forceinline__ float sara_prox_v(float2 al, float2 z, float w, size_t j, const SaraProxArgs& pa,
                                             float gamma) {
  const float2 a = cadd(al, z);
  // shrink factor (|a| - lam)^+ / |a| = max(1 - lam / |a|, 0), with 1 / |a|
  // from the hardware reciprocal square root (0 where a = 0)
  const float m2 = fmaf(a.x, a.x, a.y * a.y);
  const float s = m2 > 0.0f ? fmaxf(fmaf(-gamma * w, rsqrtf(m2), 1.0f), 0.0f) : 0.0f;
  const float2 r1 = cscale(a, s);
  const float2 z1n = csub(a, r1);
  pa.z1[j] = z1n;
  pa.u1[j] = csub(r1, z1n);
  const float al2 = fmaf(al.x, al.x, al.y * al.y);
  return w * (al2 > 0.0f ? al2 * rsqrtf(al2) : 0.0f);
}

__device__ __forceinline__ float sara_prox(float2 al, size_t j, const SaraProxArgs& pa, float gamma) {
  const float w = pa.w ? pa.w[j] : 1.0f;
  return sara_prox_v(al, pa.z1[j], w, j, pa, gamma);
}

// ---------------------------------------------------------------------------
// Dirac plane: alpha_0 = x / sqrt(q) (plain), or its prox update.
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void k_dirac(const float2* __restrict__ x, float2* __restrict__ alpha, int64_t N, float scale,
                        SaraProxArgs pa, double* partials, DevScalars* sc) {
  float f1 = 0.f;
  const float gamma = (MODE == kSaraProx) ? (float)sc->gamma : 0.f;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
    const float2 al = cscale(x[j], scale);
    if (MODE == kSaraPlain) alpha[j] = al;
    else f1 += sara_prox(al, (size_t)j, pa, gamma);
  }
  if (MODE == kSaraProx) {
    double f1d = (double)f1, tot;
    if (reduce_last_block<1>(&f1d, partials + kCntF1 * 2 * kMaxPartials, &sc->counter[kCntF1], &tot))
      sc->f1 = tot;  // first contribution of this analysis
  }
}

// One wavelet plane of one analysis level, for the Daubechies order P fixed at
// compile time (filters in registers, tap loops unrolled).  Returns this
// thread's terms of f1 (prox mode).
template <int P, int MODE>
__device__ __forceinline__ float dwt_plane(const float2* __restrict__ in, int in_shared, float2* __restrict__ ll_out,
                                           float2* __restrict__ coef, const LevelGeom& G, const WaveletFilters& wf,
                                           const SaraProxArgs& pa, int k, float gamma) {
  extern __shared__ float2 sm[];
  constexpr int taps = 2 * P;
  constexpr int hoff = P * (P - 1);  // db_p starts after db_1 .. db_(p-1): sum of 2q, q < p
  float2 h[taps], g[taps];  // each tap as a (w, w) pair for the FFMA2s
#pragma unroll
  for (int m = 0; m < taps; ++m) {
    const float hm = wf.h[hoff + m];
    const float hr = wf.h[hoff + taps - 1 - m];
    h[m] = make_float2(hm, hm);
    g[m] = (m & 1) ? make_float2(-hr, -hr) : make_float2(hr, hr);
  }
  float f1 = 0.f;
  const int L = G.L, H = L / 2;
  const int TI = G.tile;
  const int I1 = blockIdx.y * TI, I2 = blockIdx.x * TI;
  const int RH = 2 * TI + taps - 2;  // input rows/cols the tile needs
  float2* inb = sm;                  // RH x RH
  float2* rowp = sm + RH * RH;       // RH x 2TI  ([a | d] per input row)
  const float2* src = in_shared ? in : in + (size_t)k * (G.n / 2) * (G.n / 2);
  const Div dTI = make_div(TI), d2TI = make_div(2 * TI);
  // input tile with its halo (periodic): warps take rows, lanes columns (RH <=
  // 2 * 16 + 14 = 46, two column rounds); the halo wraps past L at most once
  // when L >= RH, and index by index (a remainder) otherwise
  {
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int rr0 = (threadIdx.x >> 5); rr0 < RH; rr0 += 4 * nw) {
      float2 v[4][2];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int rr = rr0 + q * nw;
        if (rr < RH) {
          int r = 2 * I1 + rr;
          r = (L >= RH) ? (r >= L ? r - L : r) : r % L;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int cc = lane + 32 * h;
            if (cc < RH) {
              int c = 2 * I2 + cc;
              c = (L >= RH) ? (c >= L ? c - L : c) : c % L;
              v[q][h] = src[(size_t)r * L + c];
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int rr = rr0 + q * nw;
        if (rr < RH) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int cc = lane + 32 * h;
            if (cc < RH) inb[rr * RH + cc] = v[q][h];
          }
        }
      }
    }
  }
  __syncthreads();
  // rows: a[i2] = sum_m h[m] s[2 i2 + m], d[i2] = sum_m g[m] s[2 i2 + m]
  for (int idx = threadIdx.x; idx < RH * TI; idx += blockDim.x) {
    const int rr = udiv(idx, dTI), i2 = idx - rr * TI;
    const float2* sp = inb + rr * RH + 2 * i2;
    float2 a = make_float2(0.f, 0.f), d = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < taps; ++m) {
      const float2 v = sp[m];
      a = __ffma2_rn(h[m], v, a);
      d = __ffma2_rn(g[m], v, d);
    }
    rowp[rr * (2 * TI) + i2] = a;
    rowp[rr * (2 * TI) + TI + i2] = d;
  }
  __syncthreads();
  // columns, and the write-out of the four sub-bands
  float2* plane = coef + (size_t)(G.plane0 + k) * G.n * G.n;
  float2* llk = ll_out + (size_t)k * (G.n / 2) * (G.n / 2);
  // columns of this thread's (at most two, TI <= 16) outputs, then every
  // output with its prox operands loaded together
  constexpr int kMaxIdx = 2;  // TI * 2TI / 256
  float2 lov[kMaxIdx], hiv[kMaxIdx];
  int idxv[kMaxIdx];
#pragma unroll
  for (int t = 0; t < kMaxIdx; ++t) {
    const int idx = threadIdx.x + t * blockDim.x;
    idxv[t] = idx < TI * 2 * TI ? idx : -1;
    float2 lo = make_float2(0.f, 0.f), hi = make_float2(0.f, 0.f);
    if (idxv[t] >= 0) {
      const int i1 = udiv(idx, d2TI), kc = idx - i1 * (2 * TI);
      const float2* cp = rowp + (2 * i1) * (2 * TI) + kc;
#pragma unroll
      for (int m = 0; m < taps; ++m) {
        const float2 v = cp[m * (2 * TI)];
        lo = __ffma2_rn(h[m], v, lo);
        hi = __ffma2_rn(g[m], v, hi);
      }
    }
    lov[t] = lo;
    hiv[t] = hi;
  }
  // destinations: LL = lo of a (top-left), LH = lo of d (top-right),
  // HL = hi of a (bottom-left), HH = hi of d; on coarser levels LL goes to llk
  size_t jo[2 * kMaxIdx];
  float2 ao[2 * kMaxIdx];
  bool to_plane[2 * kMaxIdx];
#pragma unroll
  for (int t = 0; t < kMaxIdx; ++t) {
    jo[2 * t] = jo[2 * t + 1] = 0;
    to_plane[2 * t] = to_plane[2 * t + 1] = false;
    ao[2 * t] = ao[2 * t + 1] = make_float2(0.f, 0.f);
    if (idxv[t] < 0) continue;
    const int i1 = udiv(idxv[t], d2TI), kc = idxv[t] - i1 * (2 * TI);
    const int gi1 = I1 + i1;
    const bool rowlow = kc < TI;
    const int gi2 = I2 + (rowlow ? kc : kc - TI);
    if (rowlow) {
      if (G.last) {
        jo[2 * t] = (size_t)gi1 * G.n + gi2;
        ao[2 * t] = cscale(lov[t], G.scale);
        to_plane[2 * t] = true;
      } else {
        llk[(size_t)gi1 * H + gi2] = lov[t];
      }
      jo[2 * t + 1] = (size_t)(H + gi1) * G.n + gi2;  // HL
      ao[2 * t + 1] = cscale(hiv[t], G.scale);
    } else {
      jo[2 * t] = (size_t)gi1 * G.n + H + gi2;                // LH
      jo[2 * t + 1] = (size_t)(H + gi1) * G.n + H + gi2;      // HH
      ao[2 * t] = cscale(lov[t], G.scale);
      ao[2 * t + 1] = cscale(hiv[t], G.scale);
      to_plane[2 * t] = true;
    }
    to_plane[2 * t + 1] = true;
  }
  const size_t pbase = (size_t)(G.plane0 + k) * G.n * G.n;
  if (MODE == kSaraPlain) {
#pragma unroll
    for (int o = 0; o < 2 * kMaxIdx; ++o)
      if (to_plane[o]) plane[jo[o]] = ao[o];
  } else {
    float2 zv[2 * kMaxIdx];
    float wv[2 * kMaxIdx];
#pragma unroll
    for (int o = 0; o < 2 * kMaxIdx; ++o) {
      if (to_plane[o]) {
        zv[o] = pa.z1[pbase + jo[o]];
        wv[o] = pa.w ? pa.w[pbase + jo[o]] : 1.0f;
      }
    }
#pragma unroll
    for (int o = 0; o < 2 * kMaxIdx; ++o)
      if (to_plane[o]) f1 += sara_prox_v(ao[o], zv[o], wv[o], pbase + jo[o], pa, gamma);
  }
    return f1;
}

// ---------------------------------------------------------------------------
// One analysis level for every wavelet plane.
//   input  : level 0: x (shared by all planes); else ll_in + k * (n/2)^2, L x L
//   output : LH, HL, HH at their Mallat positions of plane k; LL to
//            ll_out + k * (n/2)^2, or to the plane on the last level.
// CTA: coefficient tile [I1, I1 + TI) x [I2, I2 + TI) of the L/2 x L/2 sub-bands.
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256) k_dwt_level(const float2* __restrict__ in, int in_shared,
                                                   float2* __restrict__ ll_out, float2* __restrict__ coef,
                                                   LevelGeom G, BasisList bl, WaveletFilters wf,
                                                   SaraProxArgs pa, double* partials, DevScalars* sc) {
  extern __shared__ float2 sm[];
  const int k = blockIdx.z;
  const float gamma = (MODE == kSaraProx) ? (float)sc->gamma : 0.f;
  float f1 = 0.f;
  if (k == G.nb) {
    // the Dirac plane (first level only): alpha_0 = x / sqrt(q) on this CTA's
    // 2TI x 2TI block of pixels, with its prox update
    const int TI = G.tile, r0 = 2 * blockIdx.y * TI, c0 = 2 * blockIdx.x * TI;
    const size_t base = (size_t)G.dirac * G.n * G.n;
    for (int e = threadIdx.x; e < 4 * TI * TI; e += blockDim.x) {
      const int rr = e / (2 * TI), cc = e - rr * (2 * TI);
      const size_t j = (size_t)(r0 + rr) * G.n + c0 + cc;
      const float2 al = cscale(in[j], G.scale);
      if (MODE == kSaraPlain) coef[base + j] = al;
      else f1 += sara_prox(al, base + j, pa, gamma);
    }
  } else {
    switch (bl.p[k]) {
      case 1: f1 += dwt_plane<1, MODE>(in, in_shared, ll_out, coef, G, wf, pa, k, gamma); break;
      case 2: f1 += dwt_plane<2, MODE>(in, in_shared, ll_out, coef, G, wf, pa, k, gamma); break;
      case 3: f1 += dwt_plane<3, MODE>(in, in_shared, ll_out, coef, G, wf, pa, k, gamma); break;
      case 4: f1 += dwt_plane<4, MODE>(in, in_shared, ll_out, coef, G, wf, pa, k, gamma); break;
      case 5: f1 += dwt_plane<5, MODE>(in, in_shared, ll_out, coef, G, wf, pa, k, gamma); break;
      case 6: f1 += dwt_plane<6, MODE>(in, in_shared, ll_out, coef, G, wf, pa, k, gamma); break;
      case 7: f1 += dwt_plane<7, MODE>(in, in_shared, ll_out, coef, G, wf, pa, k, gamma); break;
      default: f1 += dwt_plane<8, MODE>(in, in_shared, ll_out, coef, G, wf, pa, k, gamma); break;
    }
  }
  if (MODE == kSaraProx) {
    // this block's f1 partial; the first synthesis launch adds them all up
    double f1d = (double)f1;
    block_reduce<1>(&f1d);
    if (threadIdx.x == 0)
      partials[kCntF1 * 2 * kMaxPartials + G.f1_off + blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] =
          f1d;
  }
}

// f1 of §4.4 as the sum of the analysis levels' block partials (in index
// order), and the halting quantity zeta = |f1 - f1_prev| / f1_prev.
__device__ __forceinline__ void sara_f1_finish(const double* __restrict__ part, int n, DevScalars* sc) {
  // eight independent sums per thread (loads in flight together), in a fixed order
  constexpr int U = 8;
  const int nt = blockDim.x;
  double a[U];
#pragma unroll
  for (int u = 0; u < U; ++u) a[u] = 0.0;
  int i = threadIdx.x;
  for (; i + (U - 1) * nt < n; i += U * nt) {
    double t[U];
#pragma unroll
    for (int u = 0; u < U; ++u) t[u] = __ldcg(&part[i + u * nt]);
#pragma unroll
    for (int u = 0; u < U; ++u) a[u] += t[u];
  }
  for (; i < n; i += nt) a[0] += __ldcg(&part[i]);
  double v = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
  block_reduce<1>(&v);
  if (threadIdx.x == 0) {
    sc->f1 = v;
    const double prev = sc->f1_prev;
    sc->zeta = (prev != 0.0) ? fabs(v - prev) / fabs(prev) : INFINITY;
    sc->f1_prev = v;
  }
}

// Column then row synthesis of one plane's coefficient windows (in shared
// memory) for the Daubechies order P fixed at compile time; the finest level
// accumulates into accum, coarser levels write their low-low output.
constexpr int kIdwtMaxOut = 4;  // (2TO)^2 / blockDim outputs per thread: 1024 / 256
template <int P>
__device__ __forceinline__ void idwt_filter(const float2* LLs, const float2* HLs, const float2* LHs,
                                            const float2* HHs, float2* As, float2* Ds, const LevelGeom& G,
                                            const WaveletFilters& wf, int k, int K1, int K2,
                                            float2* __restrict__ ll_out, float2 (&accum)[kIdwtMaxOut]) {
  constexpr int taps = 2 * P;
  constexpr int hoff = P * (P - 1);
  float2 h[taps], g[taps];  // (w, w) pairs
#pragma unroll
  for (int m = 0; m < taps; ++m) {
    const float hm = wf.h[hoff + m];
    const float hr = wf.h[hoff + taps - 1 - m];
    h[m] = make_float2(hm, hm);
    g[m] = (m & 1) ? make_float2(-hr, -hr) : make_float2(hr, hr);
  }
  const int L = G.L;
  const int TO = G.tile;
  const int CW = TO + P - 1;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int nout = (2 * TO) * (2 * TO);
  const Div d2TO = make_div(2 * TO);
  // column synthesis: output row kappa1 in [0, 2TO), window column t2;
  // taps of one parity: m = par + 2u, t1 = (k1 - par) / 2 - u + P - 1
  for (int t2 = threadIdx.x >> 5; t2 < CW; t2 += nw)
    for (int k1 = lane; k1 < 2 * TO; k1 += 32) {
      const int idx = k1 * CW + t2;
      const int par = k1 & 1;
      const int tb = (k1 - par) / 2 + P - 1;
      float2 av = make_float2(0.f, 0.f), dv = make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < P; ++u) {
        const int t1 = tb - u;
        const float2 hm = par ? h[2 * u + 1] : h[2 * u], gm = par ? g[2 * u + 1] : g[2 * u];
        const float2 ll = LLs[t1 * CW + t2], hl = HLs[t1 * CW + t2];
        const float2 lh = LHs[t1 * CW + t2], hh = HHs[t1 * CW + t2];
        av = __ffma2_rn(hm, ll, __ffma2_rn(gm, hl, av));
        dv = __ffma2_rn(hm, lh, __ffma2_rn(gm, hh, dv));
      }
      As[idx] = av;
      Ds[idx] = dv;
    }
  __syncthreads();
  // row synthesis
#pragma unroll
  for (int t = 0; t < kIdwtMaxOut; ++t) {
    const int idx = threadIdx.x + t * blockDim.x;
    if (idx >= nout) continue;
    const int k1 = udiv(idx, d2TO), k2 = idx - k1 * (2 * TO);
    const int par = k2 & 1;
    const int tb = (k2 - par) / 2 + P - 1;
    float2 sacc = make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < P; ++u) {
      const int t2 = tb - u;
      const float2 hm = par ? h[2 * u + 1] : h[2 * u], gm = par ? g[2 * u + 1] : g[2 * u];
      const float2 av = As[k1 * CW + t2], dv = Ds[k1 * CW + t2];
      sacc = __ffma2_rn(hm, av, __ffma2_rn(gm, dv, sacc));
    }
    if (G.last) {
      accum[t] = cadd(accum[t], sacc);
    } else {
      const int gk1 = K1 + k1, gk2 = K2 + k2;
      if (gk1 < L && gk2 < L) ll_out[(size_t)k * (G.n / 2) * (G.n / 2) + (size_t)gk1 * L + gk2] = sacc;
    }
  }
}

// ---------------------------------------------------------------------------
// One synthesis level for every wavelet plane (transpose of k_dwt_level):
//   A  = colsyn(LL, HL), Dr = colsyn(LH, HH), s = rowsyn(A, Dr),
//   s[k] = sum_{m = k mod 2} h[m] a[((k - m)/2) mod H] + g[m] d[((k - m)/2) mod H].
// Output: L x L; to ll_out + k (n/2)^2, or, on the finest level, summed over
// planes (plus the Dirac plane) into x, scaled by 1/sqrt(q).
// CTA: output tile [K1, K1 + 2TO) x [K2, K2 + 2TO).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_idwt_level(const float2* __restrict__ ll_in, int ll_from_plane,
                                                    float2* __restrict__ ll_out, const float2* __restrict__ coef,
                                                    float2* __restrict__ x, int dirac_plane, LevelGeom G,
                                                    BasisList bl, WaveletFilters wf, const double* f1_part, int f1_n,
                                                    DevScalars* sc) {
  extern __shared__ float2 sm[];
  // with f1 partials to sum, the first z slice is extra (dispatched first, so
  // that its block (0, 0), which forms f1 and zeta, overlaps the tiles)
  if (f1_n > 0 && blockIdx.z == 0) {
    if (blockIdx.x == 0 && blockIdx.y == 0) sara_f1_finish(f1_part, f1_n, sc);
    return;
  }
  const int bz = (int)blockIdx.z - (f1_n > 0 ? 1 : 0);  // the plane slice of this block
  const int L = G.L, H = L / 2;
  const int TO = G.tile;
  const int K1 = blockIdx.y * 2 * TO, K2 = blockIdx.x * 2 * TO;
  // the finest level loops over all planes in one CTA; otherwise one plane per z
  const int kbeg = G.last ? 0 : bz;
  const int kend = G.last ? G.nb : bz + 1;
  constexpr int kMaxOut = kIdwtMaxOut;
  float2 accum[kMaxOut];
  const int nout = (2 * TO) * (2 * TO);
  const Div dH = make_div(H), d2TO = make_div(2 * TO);
#pragma unroll
  for (int t = 0; t < kMaxOut; ++t) accum[t] = make_float2(0.f, 0.f);
  // the four coefficient windows of plane kk, loaded into registers (CW^2 <=
  // 4 blockDim for TO <= 16, p <= 8): plane k + 1's loads are in flight while
  // plane k is synthesised
  float2 v[4][4];
  auto issue = [&](int kk) {
    const int pk = bl.p[kk];
    const int CWk = TO + pk - 1;
    const float2* plk = coef + (size_t)(G.plane0 + kk) * G.n * G.n;
    const float2* llk = ll_from_plane ? plk : ll_in + (size_t)kk * (G.n / 2) * (G.n / 2);
    const int lls = ll_from_plane ? G.n : H;
    // window origin: coefficient K/2 - p + 1 (mod H), shifted to stay >= 0
    const int o1 = K1 / 2 - pk + 1 + 8 * H, o2 = K2 / 2 - pk + 1 + 8 * H;
    const float rcw = 1.0f / (float)CWk;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      if (e < CWk * CWk) {
        const int t1 = quot_small(e, rcw), t2 = e - t1 * CWk;
        int c1 = o1 + t1, c2 = o2 + t2;
        c1 -= udiv(c1, dH) * H;
        c2 -= udiv(c2, dH) * H;
        v[q][0] = llk[(size_t)c1 * lls + c2];
        v[q][1] = plk[(size_t)(H + c1) * G.n + c2];
        v[q][2] = plk[(size_t)c1 * G.n + H + c2];
        v[q][3] = plk[(size_t)(H + c1) * G.n + H + c2];
      }
    }
  };
  issue(kbeg);
  for (int k = kbeg; k < kend; ++k) {
    const int p = bl.p[k];
    const int CW = TO + p - 1;                 // coefficient window per axis
    float2* LLs = sm;                          // CW x CW each
    float2* HLs = LLs + CW * CW;
    float2* LHs = HLs + CW * CW;
    float2* HHs = LHs + CW * CW;
    float2* As = HHs + CW * CW;                // 2TO x CW
    float2* Ds = As + 2 * TO * CW;             // 2TO x CW
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      if (e < CW * CW) {
        LLs[e] = v[q][0];
        HLs[e] = v[q][1];
        LHs[e] = v[q][2];
        HHs[e] = v[q][3];
      }
    }
    __syncthreads();
    if (k + 1 < kend) issue(k + 1);
    switch (p) {
      case 1: idwt_filter<1>(LLs, HLs, LHs, HHs, As, Ds, G, wf, k, K1, K2, ll_out, accum); break;
      case 2: idwt_filter<2>(LLs, HLs, LHs, HHs, As, Ds, G, wf, k, K1, K2, ll_out, accum); break;
      case 3: idwt_filter<3>(LLs, HLs, LHs, HHs, As, Ds, G, wf, k, K1, K2, ll_out, accum); break;
      case 4: idwt_filter<4>(LLs, HLs, LHs, HHs, As, Ds, G, wf, k, K1, K2, ll_out, accum); break;
      case 5: idwt_filter<5>(LLs, HLs, LHs, HHs, As, Ds, G, wf, k, K1, K2, ll_out, accum); break;
      case 6: idwt_filter<6>(LLs, HLs, LHs, HHs, As, Ds, G, wf, k, K1, K2, ll_out, accum); break;
      case 7: idwt_filter<7>(LLs, HLs, LHs, HHs, As, Ds, G, wf, k, K1, K2, ll_out, accum); break;
      default: idwt_filter<8>(LLs, HLs, LHs, HHs, As, Ds, G, wf, k, K1, K2, ll_out, accum); break;
    }
  }
  if (G.last) {
#pragma unroll
    for (int t = 0; t < kMaxOut; ++t) {
      const int idx = threadIdx.x + t * blockDim.x;
      if (idx >= nout) continue;
      const int k1 = udiv(idx, d2TO), k2 = idx - k1 * (2 * TO);
      const int gk1 = K1 + k1, gk2 = K2 + k2;
      if (gk1 < L && gk2 < L) {
        float2 s = accum[t];
        const size_t j = (size_t)gk1 * G.n + gk2;
        if (dirac_plane >= 0) s = cadd(s, coef[(size_t)dirac_plane * G.n * G.n + j]);
        x[j] = cscale(s, G.scale);
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_f1_finish(const double* __restrict__ part, int n, DevScalars* sc) {
  sara_f1_finish(part, n, sc);
}

// Dirac-only synthesis: x = alpha_0 / sqrt(q).
__global__ void k_dirac_syn(const float2* __restrict__ a, float2* __restrict__ x, int64_t N, float scale) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x)
    x[j] = cscale(a[j], scale);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static void basis_layout(const purify_ctx* c, int& dirac_plane, int& plane0, BasisList& bl, int& nb) {
  dirac_plane = -1;
  nb = 0;
  plane0 = 0;
  for (int k = 0; k < c->q; ++k) {
    if (c->bases[k] == 0) dirac_plane = k;
    else {
      if (nb == 0) plane0 = k;
      bl.p[nb++] = c->bases[k];
    }
  }
}

// Tile of one level: the largest divisor t <= kTile of H whose grid of
// (H / t)^2 tiles per plane times `planes` gives every SM a CTA; failing
// that, the largest divisor <= kMinTile (deep levels are small, and a CTA per
// tile of a few coefficients only wastes its halo).  Every divisor of
// H = 2^a or 3 * 2^a has the same form, as the index splits need.
constexpr int kMinTile = 4;
static int tile_for(int H, int64_t planes, int sms) {
  int fallback = 1;
  for (int t = std::min(kTile, H); t >= 1; --t) {
    if (H % t != 0) continue;
    if ((int64_t)(H / t) * (H / t) * planes >= (int64_t)sms) return t;
    if (t <= kMinTile) {
      fallback = t;
      break;
    }
  }
  return fallback;
}

// Finish zeta when the dictionary has no wavelet plane (Dirac only).
__global__ void k_finish_zeta(DevScalars* sc) {
  const double prev = sc->f1_prev;
  sc->zeta = (prev != 0.0) ? fabs(sc->f1 - prev) / fabs(prev) : INFINITY;
  sc->f1_prev = sc->f1;
}

static size_t dwt_smem(int TI, int taps) {
  const int RH = 2 * TI + taps - 2;
  return (size_t)(RH * RH + RH * 2 * TI) * sizeof(float2);
}

static size_t idwt_smem(int TO, int p) {
  const int CW = TO + p - 1;
  return (size_t)(4 * CW * CW + 2 * 2 * TO * CW) * sizeof(float2);
}

int sara_analysis(purify_ctx* c, const float2* x, float2* alpha, SaraMode mode, const SaraProxArgs& pa,
                  cudaStream_t s, int* f1_parts) {
  if (f1_parts) *f1_parts = 0;
  int dirac_plane, plane0, nb;
  BasisList bl{};
  basis_layout(c, dirac_plane, plane0, bl, nb);
  const int64_t N = (int64_t)c->n * c->n;
  const float scale = 1.0f / sqrtf((float)c->q);
  if (dirac_plane >= 0 && nb == 0) {
    int blocks = (int)std::min<int64_t>((N + 255) / 256, 1024);
    if (mode == kSaraPlain)
      PURIFY_LAUNCH(c, "dirac", s,
                    (k_dirac<kSaraPlain><<<blocks, 256, 0, s>>>(x, alpha + (size_t)dirac_plane * N, N, scale, pa,
                                                                c->d_partials, c->d_sc)));
    else
      PURIFY_LAUNCH(c, "dirac", s,
                    (k_dirac<kSaraProx><<<blocks, 256, 0, s>>>(x, nullptr, N, scale, pa, c->d_partials, c->d_sc)));
  }
  if (nb == 0) {
    if (mode == kSaraProx) PURIFY_LAUNCH(c, "finish_zeta", s, (k_finish_zeta<<<1, 1, 0, s>>>(c->d_sc)));
    return check_cuda(cudaGetLastError());
  }
  int maxp = 1;
  for (int k = 0; k < nb; ++k) maxp = std::max(maxp, bl.p[k]);
  int f1_off = 0;
  for (int lev = 0; lev < c->levels; ++lev) {
    const int L = c->n >> lev;
    const int H = L / 2;
    const int TI = tile_for(H, nb + (lev == 0 && dirac_plane >= 0 ? 1 : 0), c->sms);
    LevelGeom G{TI, c->n, L, nb, plane0, lev == c->levels - 1, scale, lev == 0, lev == 0 ? dirac_plane : -1, f1_off};
    const float2* in = (lev == 0) ? x : c->d_ll[(lev - 1) & 1];
    float2* llo = c->d_ll[lev & 1];
    dim3 grid(H / TI, H / TI, nb + (G.dirac >= 0 ? 1 : 0));
    f1_off += (int)(grid.x * grid.y * grid.z);
    if (mode == kSaraProx && f1_off > 2 * kMaxPartials) return PURIFY_E_SIZE;  // the kCntF1 slot holds 2 kMaxPartials
    const size_t sm = dwt_smem(TI, 2 * maxp);
    if (mode == kSaraPlain)
      PURIFY_LAUNCH(c, "dwt_level", s,
                    (k_dwt_level<kSaraPlain><<<grid, 256, sm, s>>>(in, lev == 0, llo, alpha, G, bl, c->wf, pa,
                                                                   c->d_partials, c->d_sc)));
    else
      PURIFY_LAUNCH(c, "dwt_level", s,
                    (k_dwt_level<kSaraProx><<<grid, 256, sm, s>>>(in, lev == 0, llo, pa.z1, G, bl, c->wf, pa,
                                                                  c->d_partials, c->d_sc)));
  }
  if (mode == kSaraProx) {
    if (f1_parts) {
      *f1_parts = f1_off;
    } else {  // no synthesis follows to finish f1: one block does
      PURIFY_LAUNCH(c, "f1_finish", s,
                    (k_f1_finish<<<1, 256, 0, s>>>(c->d_partials + kCntF1 * 2 * kMaxPartials, f1_off, c->d_sc)));
    }
  }
  return check_cuda(cudaGetLastError());
}

int sara_synthesis(purify_ctx* c, const float2* alpha, float2* x, cudaStream_t s, int f1_parts) {
  int dirac_plane, plane0, nb;
  BasisList bl{};
  basis_layout(c, dirac_plane, plane0, bl, nb);
  const int64_t N = (int64_t)c->n * c->n;
  const float scale = 1.0f / sqrtf((float)c->q);
  if (nb == 0) {
    int blocks = (int)std::min<int64_t>((N + 255) / 256, 1024);
    PURIFY_LAUNCH(c, "dirac", s, (k_dirac_syn<<<blocks, 256, 0, s>>>(alpha + (size_t)dirac_plane * N, x, N, scale)));
    return check_cuda(cudaGetLastError());
  }
  int maxp = 1;
  for (int k = 0; k < nb; ++k) maxp = std::max(maxp, bl.p[k]);
  for (int lev = c->levels - 1; lev >= 0; --lev) {
    const int L = c->n >> lev;  // output side
    const int H = L / 2;
    const int TO = tile_for(H, lev == 0 ? 1 : nb, c->sms);
    LevelGeom G{TO, c->n, L, nb, plane0, lev == 0, scale, 0, -1};
    const bool from_plane = (lev == c->levels - 1);
    const float2* llin = from_plane ? nullptr : c->d_ll[(lev + 1) & 1];
    float2* llo = c->d_ll[lev & 1];
    // the first launch (coarsest level) carries one more z slice (the first)
    // whose first block forms f1 and zeta from the analysis partials
    const int f1n = (lev == c->levels - 1) ? f1_parts : 0;
    dim3 grid(L / (2 * TO), L / (2 * TO), (lev == 0 ? 1 : nb) + (f1n > 0 ? 1 : 0));
    const size_t sm = idwt_smem(TO, maxp);
    PURIFY_LAUNCH(c, "idwt_level", s,
                  (k_idwt_level<<<grid, 256, sm, s>>>(llin, from_plane, llo, alpha, x, dirac_plane, G, bl, c->wf,
                                                      c->d_partials + kCntF1 * 2 * kMaxPartials, f1n, c->d_sc)));
  }
  return check_cuda(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Daubechies filters by spectral factorisation (Daubechies 1988): the roots y_k
// of P(y) = sum_{k<p} C(p-1+k, k) y^k (Durand-Kerner iteration), each mapped to
// the zero inside the unit circle of z^2 - (2 - 4y) z + 1; h is the coefficient
// list of (z + 1)^p prod (z - z_k) in descending powers, scaled to sum sqrt(2).
// ---------------------------------------------------------------------------
static std::vector<double> daubechies(int p) {
  using cd = std::complex<double>;
  const int d = p - 1;
  std::vector<double> P(p);
  double binom = 1.0;  // C(p-1+k, k)
  for (int k = 0; k < p; ++k) {
    if (k > 0) binom = binom * (double)(p - 1 + k) / (double)k;
    P[k] = binom;
  }
  std::vector<cd> roots(d);
  if (d > 0) {
    // monic in y: divide by the leading coefficient P[d]
    std::vector<cd> r(d);
    const cd seed(0.4, 0.9);
    cd pw(1.0, 0.0);
    for (int k = 0; k < d; ++k) { r[k] = pw; pw *= seed; }
    auto evalP = [&](cd y) {
      cd acc = P[d];
      for (int k = d - 1; k >= 0; --k) acc = acc * y + P[k];
      return acc / P[d];
    };
    for (int it = 0; it < 2000; ++it) {
      double delta = 0.0;
      for (int k = 0; k < d; ++k) {
        cd den(1.0, 0.0);
        for (int j = 0; j < d; ++j)
          if (j != k) den *= (r[k] - r[j]);
        const cd step = evalP(r[k]) / den;
        r[k] -= step;
        delta = std::max(delta, std::abs(step));
      }
      if (delta < 1e-17) break;
    }
    roots = r;
  }
  // polynomial coefficients in ascending powers of z
  std::vector<cd> poly(1, cd(1.0, 0.0));
  auto mul_root = [&](cd z0) {  // poly *= (z - z0)
    std::vector<cd> out(poly.size() + 1, cd(0.0, 0.0));
    for (size_t i = 0; i < poly.size(); ++i) {
      out[i + 1] += poly[i];
      out[i] -= z0 * poly[i];
    }
    poly.swap(out);
  };
  for (int k = 0; k < p; ++k) mul_root(cd(-1.0, 0.0));
  for (int k = 0; k < d; ++k) {
    const cd c = 2.0 - 4.0 * roots[k];
    const cd disc = std::sqrt(c * c - 4.0);
    cd z1 = (c + disc) / 2.0, z2 = (c - disc) / 2.0;
    mul_root(std::abs(z1) < 1.0 ? z1 : z2);
  }
  // descending powers: h[m] = coefficient of z^(2p-1-m)
  std::vector<double> h(2 * p);
  double sum = 0.0;
  for (int m = 0; m < 2 * p; ++m) {
    h[m] = poly[2 * p - 1 - m].real();
    sum += h[m];
  }
  for (auto& v : h) v *= std::sqrt(2.0) / sum;
  return h;
}

void make_daubechies(WaveletFilters& wf) {
  int off = 0;
  wf.off[0] = 0;
  for (int p = 1; p <= 8; ++p) {
    wf.off[p] = off;
    std::vector<double> h = daubechies(p);
    for (int m = 0; m < 2 * p; ++m) wf.h[off + m] = (float)h[m];
    off += 2 * p;
  }
}

}  // namespace purify
