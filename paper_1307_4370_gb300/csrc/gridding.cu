// Interpolation operator G of Phi = G F D Z B (§5 eq. opmodel) and its
// adjoint on the 2n x 2n grid, with the Kaiser-Bessel (or Gaussian) taps
// evaluated from their fitted polynomials:
//   k_degrid   G: per grid tile, a shared-memory halo and one visibility per
//              thread (SDMM mode: the FP64 norms of the l2 branch);
//   k_grid     G^T as an atomic-free gather (and, in the Gram form, G^T G in
//              one pass for the CG steps).
#include "common.cuh"
#include "reduce.cuh"

namespace purify {

// ---------------------------------------------------------------------------
// Degridding G.  The visibilities are sorted by the grid tile (T x T) holding
// the first cell of their footprint; one CTA takes a run of one tile's
// visibilities, stages the (T + J - 1)^2 cells their footprints can reach in
// shared memory, and gathers J x J cells per visibility from there.
// ---------------------------------------------------------------------------
template <int J, int MODE>
__global__ void __launch_bounds__(256) k_degrid(const float2* __restrict__ X, const float2* __restrict__ uv,
                                                const int* __restrict__ perm, DegridArgs a,
                                                const int4* __restrict__ dchunks, KbPoly kb, KappaScale ks, int L,
                                                int T, int tiles_1d, double* partials, DevScalars* sc) {
  extern __shared__ float2 halo[];
  constexpr int NT = 256;
  const int W = T + J - 1, NW = W * W;
  const int4 ch = dchunks[blockIdx.x];
  const int tr = ch.x / tiles_1d, tc = ch.x - tr * tiles_1d;
  const int R0 = tr * T, C0 = tc * T;
  // the first frequencies of this thread, in flight with the halo loads
  constexpr int QV = 4;
  float2 uq[QV];
#pragma unroll
  for (int q = 0; q < QV; ++q) {
    const int i = ch.y + threadIdx.x + q * NT;
    if (i < ch.z) uq[q] = __ldg(&uv[i]);
  }
  // halo of the tile: eight cells per thread per round, all loads issued first
  const float inv_w = 1.0f / (float)W;
  for (int k0 = 0; k0 < NW; k0 += 8 * NT) {
    float2 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = k0 + threadIdx.x + q * NT;
      if (k < NW) {
        const int rr = quot_small(k, inv_w), cc = k - rr * W;  // W = T + J - 1 <= 71, k < 2^13
        int r = R0 + rr, c = C0 + cc;
        if (r >= L) r -= L;
        if (c >= L) c -= L;
        v[q] = __ldg(&X[(size_t)r * L + c]);
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = k0 + threadIdx.x + q * NT;
      if (k < NW) halo[k] = v[q];
    }
  }
  __syncthreads();
  FPair part[2];  // per-thread exact sums of a few terms; FP64 across threads
  auto visit = [&](int i, float2 u) {
    int k0r, k0c;
    float fr, fc;
    split_kappa(u.x, ks, k0r, fr);
    split_kappa(u.y, ks, k0c, fc);
    k0r -= J / 2 - 1;
    k0c -= J / 2 - 1;
    float wr[J], wc[J];
    kb_weights<J>(kb, fr, wr);
    kb_weights<J>(kb, fc, wc);
    const int dr = wrap(k0r - R0, L), dc = wrap(k0c - C0, L);
    float2 acc = make_float2(0.f, 0.f);
    if (dr < T && dc < T) {
      const float2* base = halo + dr * W + dc;
      float2 wcc[J];  // the column weights as (w, w) pairs for the FFMA2s
#pragma unroll
      for (int b = 0; b < J; ++b) wcc[b] = make_float2(wc[b], wc[b]);
#pragma unroll
      for (int aa = 0; aa < J; ++aa) {
        float2 t = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < J; ++b) t = __ffma2_rn(wcc[b], base[aa * W + b], t);
        acc = caxpy(wr[aa], t, acc);
      }
    } else {
      // not in this tile (never for a consistent table): read the grid directly
#pragma unroll
      for (int aa = 0; aa < J; ++aa) {
        const float2* row = X + (size_t)wrap(k0r + aa, L) * L;
        float2 t = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < J; ++b) {
          const float2 g = __ldg(&row[wrap(k0c + b, L)]);
          t.x = fmaf(wc[b], g.x, t.x);
          t.y = fmaf(wc[b], g.y, t.y);
        }
        acc.x = fmaf(wr[aa], t.x, acc.x);
        acc.y = fmaf(wr[aa], t.y, acc.y);
      }
    }
    if (MODE == kDegridPerm) {
      a.out[perm[i]] = acc;
    } else if (MODE == kDegridSorted) {
      a.out[i] = acc;
    } else {
      // SDMM: s2 = Phi x_hat, and the two FP64 norms of the l2 branch
      a.out[i] = acc;
      float2 y;
      if (a.y) {
        y = a.y[i];
      } else {
        const float sc4 = a.yscale[i >> 12];
        const uint32_t bits = reinterpret_cast<const uint32_t*>(a.yb)[i];
        y = make_float2(__uint_as_float(bits << 16) * sc4, __uint_as_float(bits & 0xffff0000u) * sc4);
      }
      const float2 z = a.z2[i];
      const float2 av = cadd(acc, z);
      part[0].add_sq_diff(av.x, y.x);
      part[0].add_sq_diff(av.y, y.y);
      part[1].add_sq_diff(acc.x, y.x);
      part[1].add_sq_diff(acc.y, y.y);
    }
  };
#pragma unroll
  for (int q = 0; q < QV; ++q) {
    const int i = ch.y + threadIdx.x + q * NT;
    if (i < ch.z) visit(i, uq[q]);
  }
  for (int i = ch.y + threadIdx.x + QV * NT; i < ch.z; i += NT) visit(i, __ldg(&uv[i]));
  if (MODE == kDegridSdmm) {
    double acc2[2] = {part[0].value(), part[1].value()};
    double tot[2];
    if (reduce_last_block<2>(acc2, partials + kCntL2 * 2 * kMaxPartials, &sc->counter[kCntL2], tot)) {
      sc->l2_dn2 = tot[0];
      sc->l2_res2 = tot[1];
      sc->nu = sqrt(tot[1]) / sc->eps;
      sc->nu_min = sc->nu;
      const double nd = sqrt(tot[0]);
      sc->l2_scale = (nd > sc->eps) ? sc->eps / nd : 1.0;  // projection factor of the l2 ball
    }
  }
}

// ---------------------------------------------------------------------------
// Gridding G^T, as a gather (no atomics).  The grid is cut into T x T tiles;
// set-up listed, per tile, the visibilities whose footprint meets it, sorted
// by the footprint's first cell relative to the tile (one run per start
// cell), and cut each list into chunks.  One CTA per chunk stages its
// entries (value, J + J kernel weights) in shared memory.  A 2 x 2 block of
// cells ("owner") sums, in a fixed order, the entries of the (J + 1)^2 start
// cells whose footprint reaches it: J + 1 runs of the sorted list, one per
// start row.  The owners' work is uneven (dense start cells where tracks
// cross), so the concatenation of all owners' runs is split into equal
// slices, one per thread (merge-path style): a thread writes the owners that
// lie inside its slice and leaves two partial sums for the owners cut by its
// slice ends, which are added afterwards in slice order.  The walk depends
// on the frequencies only, so set-up stores it: one 32-bit item per step
// (entry, owner, row and column tap), laid out step-major so that the loads
// of one step by a warp are contiguous.
// A tile with one chunk is written to X directly; otherwise each chunk
// stores a partial tile and the last chunk to finish adds the partials in
// chunk order.  Every cell is written once and the result does not depend
// on scheduling.
// The Gram form (G^T G applied to a grid, one per CG step) runs the same
// gather after degridding each entry from a staged halo of the input grid;
// its dense tiles instead apply a stored stencil of G^T G per cell (the full
// (2J - 1)^2 offsets, or the offsets d >= 0 of the symmetric operator on the
// tile extended by J - 1 cells; built at set-up, build_dense_gram*).
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// TMA (cp.async.bulk.tensor) with an mbarrier, in inline PTX
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make the initialised barrier visible to the asynchronous (TMA) proxy
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// 2-D tiled copy of one box of the map at element coordinates (x, y) into
// shared memory; completion is counted on the barrier in bytes.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Wait for phase `parity` of the barrier, giving up after a bounded number of
// polls (each poll may itself suspend the thread for a while); true when the
// phase completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  for (int it = 0; it < (1 << 22); ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

struct Acc4 {  // a 2 x 2 block of complex sums
  float2 a00, a01, a10, a11;
};

template <int J, int MODE, int MINB>
__global__ void __launch_bounds__(kGridThreads, MINB) k_grid(float2* __restrict__ X, const float2* __restrict__ Xin,
                                                       const int* __restrict__ perm, const float2* __restrict__ vis,
                                                       const int4* __restrict__ list,
                                                       const int4* __restrict__ chunks,
                                                       const uint16_t* __restrict__ tab, int tab_stride,
                                                       const uint32_t* __restrict__ items,
                                                       const int* __restrict__ item_row,
                                                       const int* __restrict__ tile_slot0,
                                                       const int* __restrict__ tile_nchunk,
                                                       unsigned* __restrict__ tile_cnt, float2* __restrict__ slots,
                                                       KbPoly kb, KappaScale ks, int L, int T, int tiles_1d,
                                                       int chunk_max, const __grid_constant__ CUtensorMap halo_map,
                                                       int use_tma, DevScalars* sc, int n_dense,
                                                       const int* __restrict__ dense_tiles,
                                                       const float* __restrict__ H,
                                                       const int* __restrict__ gram_chunks, int dense_half) {
  constexpr int NT = kGridThreads;
  constexpr int S = grid_wstride(J);  // [0 wr_0 .. wr_{J-1} 0 | 0 wc_0 .. wc_{J-1} 0 | pad]
  extern __shared__ __align__(128) float4 sm4[];
  __shared__ bool s_last;
  __shared__ __align__(8) uint64_t s_bar;  // completion of the halo's TMA copy
  const int W = T + J - 1, HB = T / 2, NO = HB * HB;
  const int lhb = __ffs(HB) - 1;  // T is a power of two
  float4* part = sm4;  // slot j: first[j] at 4j, last[j] at 4j + 2 (Gram form: the halo first)
  float2* yv = reinterpret_cast<float2*>(reinterpret_cast<char*>(sm4) + grid_slot_bytes(T, J));
  float* wt = reinterpret_cast<float*>(yv + chunk_max);
  int* P = reinterpret_cast<int*>(wt + (size_t)chunk_max * S);  // NO + 1 work prefix of the owners
  // Gram form: the first n_dense CTAs apply the stored G^T G of one dense tile
  // each; the others gather over the chunks of the remaining tiles
  int q = blockIdx.x;  // this CTA's chunk
  bool dense = false;
  int dtile = 0;
  if constexpr (MODE == kGridGram) {
    if ((int)blockIdx.x < n_dense) {
      dense = true;
      dtile = dense_tiles[blockIdx.x];
    } else {
      q = gram_chunks[blockIdx.x - n_dense];
    }
  }
  const int4 ch = dense ? make_int4(dtile, 0, 0, -1) : chunks[q];
  const int tile = ch.x;
  const int tr = tile / tiles_1d, tc = tile - tr * tiles_1d;
  const int R0 = tr * T, C0 = tc * T;
  const int ne = ch.z - ch.y;
  // ---- Gram form (G^T G): stage the (T + 2J - 2)^2 grid cells that the
  // footprints of the tile's entries cover; each entry's value is then its
  // degridded sample, in the same order of operations as k_degrid.  The halo
  // holds rows R0 - (J - 1) .. and columns from C0 - J (even, so that a copy
  // starts 16-byte aligned), HWS = HW + 2 per row.  For a tile whose halo
  // lies inside the grid one thread issues it as a TMA copy
  // (cp.async.bulk.tensor) at kernel start, and it lands while the entries
  // are being read; the halos of the outer ring of tiles wrap around the
  // grid's edges and are loaded cell by cell.
  const int HW = grid_halo_w(T, J), HWS = grid_halo_ws(T, J);
  const float inv_hws = 1.0f / (float)HWS, inv_w = 1.0f / (float)W;
  float2* halo = reinterpret_cast<float2*>(sm4);
  const bool tma = (MODE == kGridGram) && use_tma && R0 - (J - 1) >= 0 && R0 - (J - 1) + HW <= L &&
                   C0 - J >= 0 && C0 - J + HWS <= L;
  if (tma) {
    if (threadIdx.x == 0) {
      mbar_init(&s_bar, 1);
      fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      mbar_expect_tx(&s_bar, (unsigned)(HW * HWS * sizeof(float2)));
      tma_load_2d(halo, &halo_map, 2 * (C0 - J), R0 - (J - 1), &s_bar);
    }
  }
  // this chunk's owner-work prefix (16-bit, set up with the lists; one
  // 16-byte group per thread for T <= 64), the first four list entries of
  // each thread, and the halo: all in flight together
  uint4 tv;
  const uint4* tab4 = reinterpret_cast<const uint4*>(tab + (size_t)q * tab_stride);
  if (!dense && threadIdx.x < tab_stride / 8) tv = __ldg(&tab4[threadIdx.x]);
  int4 le[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = threadIdx.x + q * NT;
    le[q] = e < ne ? __ldg(&list[ch.y + e]) : make_int4(-1, 0, 0, 0);
  }
  if constexpr (MODE == kGridGram) {
    if (tma) {
      // every thread waits for the copy (bounded: a copy that never lands
      // sets the device error flag and the CTA leaves after a second wait)
      if (!mbar_wait_bounded(&s_bar, 0)) {
        if (threadIdx.x == 0) atomicOr(&sc->dev_error, 1);
        mbar_wait_bounded(&s_bar, 0);
        return;
      }
    } else {
      for (int k0 = 0; k0 < HW * HWS; k0 += 8 * NT) {
        float2 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int k = k0 + threadIdx.x + q * NT;
          if (k < HW * HWS) {
            const int rr = quot_small(k, inv_hws), cc = k - rr * HWS;
            int r = R0 - (J - 1) + rr, c = C0 - J + cc;
            if (r < 0) r += L;
            if (r >= L) r -= L;
            if (c < 0) c += L;
            if (c >= L) c -= L;
            v[q] = __ldg(&Xin[(size_t)r * L + c]);
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int k = k0 + threadIdx.x + q * NT;
          if (k < HW * HWS) halo[k] = v[q];
        }
      }
    }
    __syncthreads();
    if (dense && dense_half) {
      // (G^T G X)(k) = sum_{d >= 0} H[d][k] X(k + d) + sum_{d > 0} H[d][k - d] X(k - d)
      // over the lexicographically non-negative offsets d (the half stencil,
      // on the tile extended by J - 1 rows above and J - 1 columns each side);
      // the slice of one offset serves both terms.  X from the halo.
      constexpr int NDW = 2 * J - 1, NH = dense_gram_slices(J);
      const int TT = T * T, lt = lhb + 1;
      const int EW = T + 2 * (J - 1), ES = EW * (T + J - 1);
      const float* Ht = H + (size_t)blockIdx.x * NH * ES;
      for (int k = threadIdx.x; k < TT; k += NT) {
        const int r = k >> lt, cc = k & (T - 1);
        const int e0 = (r + J - 1) * EW + cc + J - 1;          // k in the extended region
        const float2* xk = halo + (r + J - 1) * HWS + cc + J;  // X(k)
        float2 acc = make_float2(0.f, 0.f);
        {  // dr = 0, dc = 0 .. J - 1
          float hf[J], hb[J];
#pragma unroll
          for (int dc = 0; dc < J; ++dc) {
            hf[dc] = __ldg(&Ht[(size_t)dc * ES + e0]);
            hb[dc] = dc > 0 ? __ldg(&Ht[(size_t)dc * ES + e0 - dc]) : 0.f;
          }
#pragma unroll
          for (int dc = 0; dc < J; ++dc) {
            acc = caxpy(hf[dc], xk[dc], acc);
            if (dc > 0) acc = caxpy(hb[dc], xk[-dc], acc);
          }
        }
#pragma unroll 1
        for (int dr = 1; dr < J; ++dr) {  // dc = -(J - 1) .. J - 1
          const float* hs = Ht + (size_t)(J + (dr - 1) * NDW) * ES;
          const float2* xf = xk + dr * HWS - (J - 1);
          const float2* xb = xk - dr * HWS + (J - 1);
          float hf[NDW], hb[NDW];
#pragma unroll
          for (int u = 0; u < NDW; ++u) {  // u = dc + J - 1
            hf[u] = __ldg(&hs[(size_t)u * ES + e0]);
            hb[u] = __ldg(&hs[(size_t)u * ES + e0 - dr * EW - (u - (J - 1))]);
          }
#pragma unroll
          for (int u = 0; u < NDW; ++u) {
            acc = caxpy(hf[u], xf[u], acc);
            acc = caxpy(hb[u], xb[-u], acc);
          }
        }
        X[(size_t)(R0 + r) * L + C0 + cc] = acc;
      }
      return;
    }
    if (dense) {
      // (G^T G X)(k) = sum_d H[d][k] X(k + d) over the (2J - 1)^2 offsets, H
      // streamed once per launch (coalesced over the cells), X from the halo
      constexpr int NDW = 2 * J - 1;
      const int TT = T * T, lt = lhb + 1;
      const float* Ht = H + (size_t)blockIdx.x * NDW * NDW * TT;
      for (int k = threadIdx.x; k < TT; k += NT) {
        const int r = k >> lt, cc = k & (T - 1);
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll 1
        for (int dr = 0; dr < NDW; ++dr) {
          const float2* hrow = halo + (r + dr) * HWS + cc + 1;
          const float* hh = Ht + (size_t)dr * NDW * TT + k;
          float hv[NDW];
#pragma unroll
          for (int dc = 0; dc < NDW; ++dc) hv[dc] = __ldcs(&hh[(size_t)dc * TT]);
#pragma unroll
          for (int dc = 0; dc < NDW; ++dc) acc = caxpy(hv[dc], hrow[dc], acc);
        }
        X[(size_t)(R0 + r) * L + C0 + cc] = acc;
      }
      return;
    }
  }
  // ---- stage the chunk's entries (loads of four entries per thread in flight)
  for (int e0 = 0; e0 < ne; e0 += 4 * NT) {
    float2 val[4];
    if (e0 > 0) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = e0 + threadIdx.x + q * NT;
        le[q] = e < ne ? __ldg(&list[ch.y + e]) : make_int4(-1, 0, 0, 0);
      }
    }
    if constexpr (MODE != kGridGram) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (le[q].x >= 0) val[q] = (MODE == kGridPerm) ? __ldg(&vis[__ldg(&perm[le[q].x])]) : __ldg(&vis[le[q].x]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (le[q].x < 0) continue;
      const int e = e0 + threadIdx.x + q * NT;
      float wr[J], wc[J];
      kb_weights<J>(kb, __int_as_float(le[q].z), wr);
      kb_weights<J>(kb, __int_as_float(le[q].w), wc);
      if constexpr (MODE == kGridGram) {
        const int kr = quot_small(le[q].y, inv_w), kc = le[q].y - kr * W;  // footprint start in the halo
        const float2* base = halo + kr * HWS + kc + 1;  // the halo's first column is C0 - J
        float2 acc = make_float2(0.f, 0.f);
        float2 wcc[J];
#pragma unroll
        for (int b = 0; b < J; ++b) wcc[b] = make_float2(wc[b], wc[b]);
#pragma unroll
        for (int aa = 0; aa < J; ++aa) {
          float2 t = make_float2(0.f, 0.f);
#pragma unroll
          for (int b = 0; b < J; ++b) t = __ffma2_rn(wcc[b], base[aa * HWS + b], t);
          acc = caxpy(wr[aa], t, acc);
        }
        val[q] = acc;
      }
      yv[e] = val[q];
      float* w = wt + (size_t)e * S;
      w[0] = 0.f;
      w[J + 1] = 0.f;
      w[J + 2] = 0.f;
      w[2 * J + 3] = 0.f;
#pragma unroll
      for (int k = 0; k < J; ++k) {
        w[1 + k] = wr[k];
        w[J + 3 + k] = wc[k];
      }
    }
  }
  __syncthreads();
  // ---- the owner-work prefix into shared memory
  if (threadIdx.x < tab_stride / 8) {
    const uint32_t w[4] = {tv.x, tv.y, tv.z, tv.w};
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const int idx = 8 * threadIdx.x + h;
      if (idx <= NO) P[idx] = (int)((w[h >> 1] >> (16 * (h & 1))) & 0xffffu);
    }
  }
  __syncthreads();
  const int Wt = P[NO];
  const bool multi = ch.w >= 0;
  float2* dst = multi ? slots + (size_t)ch.w * T * T : nullptr;
  auto write_owner = [&](int o, const Acc4& a) {
    const int R = 2 * (o >> lhb), C = 2 * (o & (HB - 1));
    if (!multi) {
      float2* row0 = X + (size_t)(R0 + R) * L + C0 + C;
      reinterpret_cast<float4*>(row0)[0] = make_float4(a.a00.x, a.a00.y, a.a01.x, a.a01.y);
      reinterpret_cast<float4*>(row0 + L)[0] = make_float4(a.a10.x, a.a10.y, a.a11.x, a.a11.y);
    } else {
      reinterpret_cast<float4*>(dst + R * T + C)[0] = make_float4(a.a00.x, a.a00.y, a.a01.x, a.a01.y);
      reinterpret_cast<float4*>(dst + (R + 1) * T + C)[0] = make_float4(a.a10.x, a.a10.y, a.a11.x, a.a11.y);
    }
  };
  // ---- this thread's slice [t0, t1) of the concatenated runs, one stored
  // item per step (the lanes of a warp stay in step)
  const int j = threadIdx.x;
  const int t0 = (j * Wt + NT - 1) / NT, t1 = ((j + 1) * Wt + NT - 1) / NT;
  const int nmy = t1 - t0;
  if (nmy > 0) {
    const uint32_t* its = items + (size_t)item_row[q] * NT + j;
    constexpr int PF = MINB >= 5 ? 4 : 8;  // items in flight per thread
    uint32_t pf[PF];
#pragma unroll
    for (int q = 0; q < PF; ++q) pf[q] = q < nmy ? __ldcs(&its[(size_t)q * NT]) : 0u;
    int o = (int)(pf[0] >> 20);
    Acc4 a;
    a.a00 = a.a01 = a.a10 = a.a11 = make_float2(0.f, 0.f);
    auto flush = [&]() {
      const int Po = P[o], Pe = P[o + 1];
      if (Po >= t0 && Pe <= t1) {
        write_owner(o, a);
      } else {
        float4* sl = part + 4 * j + (Po < t0 ? 0 : 2);  // first / last owner of the slice
        sl[0] = make_float4(a.a00.x, a.a00.y, a.a01.x, a.a01.y);
        sl[1] = make_float4(a.a10.x, a.a10.y, a.a11.x, a.a11.y);
      }
    };
    for (int s0 = 0; s0 < nmy; s0 += PF) {
#pragma unroll
      for (int q = 0; q < PF; ++q) {
        const int st = s0 + q;
        if (st < nmy) {
          const uint32_t it = pf[q];
          if (st + PF < nmy) pf[q] = __ldcs(&its[(size_t)(st + PF) * NT]);
          const int oi = (int)(it >> 20);
          if (oi != o) {
            flush();
            a.a00 = a.a01 = a.a10 = a.a11 = make_float2(0.f, 0.f);
            o = oi;
          }
          const int ee = (int)(it & ((1u << kItemEntryBits) - 1));
          const int ar = (int)((it >> 12) & 15u), bc = (int)((it >> 16) & 15u);
          const float2 v = yv[ee];
          const float* w = wt + ee * S;
          const float wr0 = w[ar], wr1 = w[ar + 1];
          const float wc0 = w[J + 2 + bc], wc1 = w[J + 3 + bc];
          const float2 v0 = cscale(v, wr0), v1 = cscale(v, wr1);
          const float2 c0 = make_float2(wc0, wc0), c1 = make_float2(wc1, wc1);
          a.a00 = __ffma2_rn(c0, v0, a.a00);
          a.a01 = __ffma2_rn(c1, v0, a.a01);
          a.a10 = __ffma2_rn(c0, v1, a.a10);
          a.a11 = __ffma2_rn(c1, v1, a.a11);
        }
      }
    }
    flush();
  }
  __syncthreads();
  // ---- owners cut by slice ends (sum in slice order) and owners with no work
  const float inv_wt = Wt > 0 ? 1.0f / (float)Wt : 0.f;
  for (int o = threadIdx.x; o < NO; o += NT) {
    const int Po = P[o], Pe = P[o + 1];
    Acc4 a;
    a.a00 = a.a01 = a.a10 = a.a11 = make_float2(0.f, 0.f);
    if (Pe > Po) {
      // slices holding the owner's first and last step: floor(P NT / Wt),
      // through a float reciprocal (the quotient is at most NT, so the
      // product is within one of it) and one integer correction
      auto slice_of = [&](int x) {
        int qq = __float2int_rz((float)x * inv_wt);
        if (qq * Wt > x) --qq;
        else if ((qq + 1) * Wt <= x) ++qq;
        return qq;
      };
      const int ja = slice_of(Po * NT), jb = slice_of((Pe - 1) * NT);
      if (ja == jb) continue;  // written by its slice
      float4 p0 = part[4 * ja + 2], p1 = part[4 * ja + 3];
      for (int jj = ja + 1; jj <= jb; ++jj) {
        if ((jj * Wt + NT - 1) / NT == ((jj + 1) * Wt + NT - 1) / NT) continue;  // empty slice
        const float4 q0 = part[4 * jj], q1 = part[4 * jj + 1];
        p0 = make_float4(p0.x + q0.x, p0.y + q0.y, p0.z + q0.z, p0.w + q0.w);
        p1 = make_float4(p1.x + q1.x, p1.y + q1.y, p1.z + q1.z, p1.w + q1.w);
      }
      a.a00 = make_float2(p0.x, p0.y);
      a.a01 = make_float2(p0.z, p0.w);
      a.a10 = make_float2(p1.x, p1.y);
      a.a11 = make_float2(p1.z, p1.w);
    }
    write_owner(o, a);
  }
  if (!multi) return;
  __threadfence();
  __syncthreads();
  const int nc = tile_nchunk[tile];
  if (threadIdx.x == 0) s_last = (atomicAdd(&tile_cnt[tile], 1u) == (unsigned)(nc - 1));
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int TT = T * T;
  const float2* first = slots + (size_t)tile_slot0[tile] * TT;
  for (int k = threadIdx.x; k < TT; k += NT) {
    float2 sum = make_float2(0.f, 0.f);
    for (int c = 0; c < nc; ++c) sum = cadd(sum, __ldcg(&first[(size_t)c * TT + k]));
    const int rr = k / T, cc = k - rr * T;
    X[(size_t)(R0 + rr) * L + C0 + cc] = sum;
  }
  if (threadIdx.x == 0) tile_cnt[tile] = 0u;
}

template <int J>
static void degrid_J(purify_ctx* c, DegridOut mode, const DegridArgs& a, cudaStream_t s) {
  const int threads = 256;
  const int W = c->tileT + J - 1;
  const size_t sm = (size_t)W * W * sizeof(float2);
#define DEG(MD)                                                                                               \
  do {                                                                                                        \
    allow_smem(k_degrid<J, MD>, sm);                                                                          \
    PURIFY_LAUNCH(c, "degrid", s,                                                                             \
                  (k_degrid<J, MD><<<c->ndchunks, threads, sm, s>>>(c->d_grid, c->d_uv, c->d_perm, a, c->d_dchunks, \
                                                                    c->kb, c->ks, c->L, c->tileT, c->tiles_1d,     \
                                                                    c->d_partials, c->d_sc)));                     \
  } while (0)
  if (mode == kDegridPerm) DEG(kDegridPerm);
  else if (mode == kDegridSorted) DEG(kDegridSorted);
  else DEG(kDegridSdmm);
#undef DEG
}

int degrid(purify_ctx* c, DegridOut mode, const DegridArgs& a, cudaStream_t s) {
  switch (c->J) {
    case 2: degrid_J<2>(c, mode, a, s); break;
    case 4: degrid_J<4>(c, mode, a, s); break;
    case 6: degrid_J<6>(c, mode, a, s); break;
    default: degrid_J<8>(c, mode, a, s); break;
  }
  return check_cuda(cudaGetLastError());
}

template <int J>
static size_t grid_smem(const purify_ctx* c) {
  return grid_fixed_bytes(c->tileT, J) + (size_t)c->chunk_max * grid_entry_bytes(J);
}

// Chunks small enough for five (four) resident CTAs per SM take the build
// with a register cap that allows five (four); larger ones (three per SM by
// shared memory) keep more registers.
template <int J, int MINB>
static void grid_JB(purify_ctx* c, GridIn mode, const float2* vis, size_t sm, cudaStream_t s) {
#define GRD(MD, NAME, OUT, IN)                                                                                 \
  do {                                                                                                         \
    allow_smem(k_grid<J, MD, MINB>, sm);                                                                       \
    PURIFY_LAUNCH(c, NAME, s,                                                                                  \
                  (k_grid<J, MD, MINB><<<MD == kGridGram ? c->n_dense + c->n_gram_chunks : c->nchunks,       \
                                         kGridThreads, sm, s>>>(                                               \
                      OUT, IN, c->d_perm, vis, c->d_list, c->d_chunks, c->d_chunk_tab, c->chunk_tab_stride,     \
                      c->d_items, c->d_item_row,                                                                \
                      c->d_tile_slot0, c->d_tile_nchunk,                                                        \
                      c->d_tile_cnt, c->d_slots, c->kb, c->ks, c->L, c->tileT, c->tiles_1d, c->chunk_max,      \
                      c->halo_map, c->halo_map_ok, c->d_sc, c->n_dense, c->d_dense_tiles, c->d_H,             \
                      c->d_gram_chunks, c->dense_half)));                                                       \
  } while (0)
  if (mode == kGridPerm) GRD(kGridPerm, "grid", c->d_grid, nullptr);
  else if (mode == kGridSorted) GRD(kGridSorted, "grid", c->d_grid, nullptr);
  else GRD(kGridGram, "gram", c->d_grid2, c->d_grid);
#undef GRD
}

template <int J>
static void grid_J(purify_ctx* c, GridIn mode, const float2* vis, cudaStream_t s) {
  const size_t sm = grid_smem<J>(c);
  if (sm <= 44 * 1024) grid_JB<J, 5>(c, mode, vis, sm, s);
  else if (sm <= 56 * 1024) grid_JB<J, 4>(c, mode, vis, sm, s);
  else grid_JB<J, 3>(c, mode, vis, sm, s);
}

// G^T G of the grid in d_grid into d_grid2 (one pass; the M samples are not stored).
int gram_grid(purify_ctx* c, cudaStream_t s) { return grid_adjoint(c, kGridGram, nullptr, s); }

int grid_adjoint(purify_ctx* c, GridIn mode, const float2* vis, cudaStream_t s) {
  switch (c->J) {
    case 2: grid_J<2>(c, mode, vis, s); break;
    case 4: grid_J<4>(c, mode, vis, s); break;
    case 6: grid_J<6>(c, mode, vis, s); break;
    default: grid_J<8>(c, mode, vis, s); break;
  }
  return check_cuda(cudaGetLastError());
}

}  // namespace purify
