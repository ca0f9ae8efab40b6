// Entrywise proximity operators, projections, CG vector updates and reductions.
//
// §4.5 notes that the proximity operators are entrywise and parallel; each
// kernel here is one pass over its vectors with the FP64 reduction it needs
// finished by the last block (reduce.cuh), so a scalar such as a CG step size
// is ready on the device for the next kernel without a host round trip.
#include <cuda_bf16.h>

#include "common.cuh"
#include "reduce.cuh"

namespace purify {

static unsigned blocks_for(int64_t n, int threads = 256, int cap = 2048) {
  int64_t b = (n + threads - 1) / threads;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

#define GRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// §4.4 eq. prox1: a/|a| (|a| - gamma w)^+, with gamma from the host or the device.
__global__ void k_soft(int64_t n, const float2* __restrict__ in, const float* __restrict__ w,
                       const double* gamma_dev, float gamma, float2* __restrict__ out) {
  const float gm = gamma_dev ? (float)*gamma_dev : gamma;
  GRID_STRIDE(j, n) {
    const float2 a = in[j];
    const float lam = gm * (w ? w[j] : 1.0f);
    const float mag = sqrtf(a.x * a.x + a.y * a.y);
    const float s = mag > 0.0f ? fmaxf(mag - lam, 0.0f) / mag : 0.0f;
    out[j] = cscale(a, s);
  }
}

// ||a - b||^2 in FP64 -> sc->norm2
__global__ void k_norm_diff(int64_t n, const float2* __restrict__ a, const float2* __restrict__ b,
                            double* partials, DevScalars* sc) {
  FPair part;  // per-thread exact sum of a few terms; FP64 across threads
  GRID_STRIDE(j, n) {
    part.add_sq_diff(a[j].x, b[j].x);
    part.add_sq_diff(a[j].y, b[j].y);
  }
  double acc = part.value(), tot;
  if (reduce_last_block<1>(&acc, partials + kCntNorm * 2 * kMaxPartials, &sc->counter[kCntNorm], &tot))
    sc->norm2 = tot;
}

// Projection onto {r : ||r - y|| <= eps} given ||in - y||^2 on the device.
__global__ void k_l2_project(int64_t n, const float2* __restrict__ in, const float2* __restrict__ y, double eps,
                             const double* norm2, float2* __restrict__ out) {
  __shared__ float s_scale;  // one FP64 square root per block
  if (threadIdx.x == 0) {
    const double nd = sqrt(*norm2);
    s_scale = (nd > eps) ? (float)(eps / nd) : 1.0f;
  }
  __syncthreads();
  const float scale = s_scale;
  GRID_STRIDE(j, n) {
    const float2 yy = y[j], r = in[j];
    out[j] = make_float2(fmaf(scale, r.x - yy.x, yy.x), fmaf(scale, r.y - yy.y, yy.y));
  }
}

// §4.4 eq. prox3 with complex entries as real pairs: max(Re a, 0).
__global__ void k_positive(int64_t n, const float2* __restrict__ in, float2* __restrict__ out) {
  GRID_STRIDE(j, n) out[j] = make_float2(fmaxf(in[j].x, 0.f), 0.f);
}

// The last pending update of a single-reduction CG solve (the earlier ones are
// applied by the forward row pass of the next step):
// p = r + beta p; s = w + beta s; x += alpha p; r -= alpha s.
__global__ void k_cg_apply(int64_t n, float2* __restrict__ x, float2* __restrict__ r, float2* __restrict__ p,
                           float2* __restrict__ sv, const float2* __restrict__ w, double* partials, DevScalars* sc,
                           int cg_nblk, int cg_j) {
  const CgStep cs = cg_consume(partials + kCntDot * 2 * kMaxPartials, cg_nblk, cg_j, sc);
  const float al = cs.alpha, be = cs.beta;
  const bool first = cs.first;
  FPair part;
  GRID_STRIDE(j, n) {
    const float2 rr = r[j], ww = w[j];
    float2 pp, ss;
    if (first) {
      pp = rr;
      ss = ww;
    } else {
      pp = make_float2(fmaf(be, p[j].x, rr.x), fmaf(be, p[j].y, rr.y));
      ss = make_float2(fmaf(be, sv[j].x, ww.x), fmaf(be, sv[j].y, ww.y));
    }
    p[j] = pp;
    sv[j] = ss;
    x[j] = make_float2(fmaf(al, pp.x, x[j].x), fmaf(al, pp.y, x[j].y));
    const float2 rn = make_float2(fmaf(-al, ss.x, rr.x), fmaf(-al, ss.y, rr.y));
    r[j] = rn;
    part.add_prod(rn.x, rn.x);
    part.add_prod(rn.y, rn.y);
  }
  double acc = part.value(), tot;
  if (reduce_last_block<1>(&acc, partials + kCntRho * 2 * kMaxPartials, &sc->counter[kCntRho], &tot))
    sc->cg_res = sqrt(tot);  // recurrence residual after the last update
}

// r = b - Qx (the start of purify_cg_solve).
__global__ void k_cg_residual_init(int64_t n, const float2* __restrict__ b, const float2* __restrict__ qx,
                                   float2* __restrict__ r, DevScalars* sc) {
  GRID_STRIDE(j, n) r[j] = csub(b[j], qx[j]);
}

// max |a_j| -> sc->amax
__global__ void k_max_abs(int64_t n, const float2* __restrict__ a, double* partials, DevScalars* sc) {
  float mf = 0.f;
  GRID_STRIDE(j, n) mf = fmaxf(mf, sqrtf(fmaf(a[j].x, a[j].x, a[j].y * a[j].y)));
  double m = (double)mf, tot;
  if (reduce_last_block<1, true>(&m, partials + kCntMax * 2 * kMaxPartials, &sc->counter[kCntMax], &tot))
    sc->amax = tot;
}

// SDMM l2 branch (Algorithm 1 steps 7-9, i = 2) after the degridding kernel
// left s2 = Phi x_hat and ||s2 + z2 - y||^2 on the device:
//   a = s2 + z2; r2 = y + min(1, eps/||a - y||)(a - y); z2 <- a - r2;
//   u2 = r2 - z2; v = u2 - s2 (gridded next: Phi^H v = x2 - Phi^H Phi x_hat).
// In the distributed form (§4.5 eq. dbp1) each visibility takes the factor
// of its block (block_of non-null).
__global__ void k_sdmm_l2(int64_t M, const float2* __restrict__ s2, float2* __restrict__ z2,
                          const float2* __restrict__ y, const uint16_t* __restrict__ yb,
                          const float* __restrict__ yscale, float2* __restrict__ v, const DevScalars* sc,
                          const int* __restrict__ block_of, const float* __restrict__ bscale) {
  const float scale1 = (float)sc->l2_scale;
  GRID_STRIDE(i, M) {
    const float scale = block_of ? bscale[block_of[i]] : scale1;
    float2 yy;
    if (y) {
      yy = y[i];
    } else {
      const float s4 = yscale[i >> 12];
      const uint32_t bits = reinterpret_cast<const uint32_t*>(yb)[i];
      yy = make_float2(__uint_as_float(bits << 16) * s4, __uint_as_float(bits & 0xffff0000u) * s4);
    }
    const float2 s = s2[i];
    const float2 a = cadd(s, z2[i]);
    const float2 r2 = make_float2(fmaf(scale, a.x - yy.x, yy.x), fmaf(scale, a.y - yy.y, yy.y));
    const float2 zn = csub(a, r2);
    z2[i] = zn;
    v[i] = csub(csub(r2, zn), s);
  }
}

// Distributed form (§4.5 eqs. blocks, dbp1): per block i of consecutive
// caller-order visibilities, ||s2_i + z2_i - y_i||^2 and ||s2_i - y_i||^2
// (gathered through the sorted positions; exact FP32 terms, FP64 sums).  One
// CTA per chunk of a block; the last CTA to finish adds each block's chunk
// partials in chunk order and forms its ball factor min(1, eps_i / ||.||) and
// nu_i = ||y_i - Phi_i x_hat|| / eps_i (nu = the largest, nu_min the smallest).
__global__ void __launch_bounds__(256) k_block_norms(const int4* __restrict__ bchunks, int nbchunks,
                                                     const int* __restrict__ pos, const float2* __restrict__ s2,
                                                     const float2* __restrict__ z2, const float2* __restrict__ y,
                                                     const uint16_t* __restrict__ yb,
                                                     const float* __restrict__ yscale, int R,
                                                     const double* __restrict__ beps, float* __restrict__ bscale,
                                                     double* partials, DevScalars* sc) {
  __shared__ bool am_last;
  const int4 ch = bchunks[blockIdx.x];
  FPair part[2];
  for (int m = ch.y + threadIdx.x; m < ch.z; m += blockDim.x) {
    const int j = pos[m];
    float2 yy;
    if (y) {
      yy = y[j];
    } else {
      const float s4 = yscale[j >> 12];
      const uint32_t bits = reinterpret_cast<const uint32_t*>(yb)[j];
      yy = make_float2(__uint_as_float(bits << 16) * s4, __uint_as_float(bits & 0xffff0000u) * s4);
    }
    const float2 s = s2[j];
    const float2 a = cadd(s, z2[j]);
    part[0].add_sq_diff(a.x, yy.x);
    part[0].add_sq_diff(a.y, yy.y);
    part[1].add_sq_diff(s.x, yy.x);
    part[1].add_sq_diff(s.y, yy.y);
  }
  double v[2] = {part[0].value(), part[1].value()};
  block_reduce<2>(v);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = v[0];
    partials[kMaxPartials + blockIdx.x] = v[1];
    __threadfence();
    am_last = atomicAdd(&sc->counter[kCntBlk], 1u) == (unsigned)(gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  double numax = 0.0, numin = INFINITY;
  for (int b = threadIdx.x; b < R; b += blockDim.x) {
    // chunks of block b: from its first chunk up to the next block's first
    int k0 = 0;
    {
      int lo = 0, hi = nbchunks;  // first chunk whose block is >= b
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (bchunks[mid].x < b) lo = mid + 1;
        else hi = mid;
      }
      k0 = lo;
    }
    double dn2 = 0.0, res2 = 0.0;
    for (int k = k0; k < nbchunks && bchunks[k].x == b; ++k) {
      dn2 += __ldcg(&partials[k]);
      res2 += __ldcg(&partials[kMaxPartials + k]);
    }
    const double e = beps[b];
    const double nd = sqrt(dn2);
    bscale[b] = (float)(nd > e ? e / nd : 1.0);
    const double nu = sqrt(res2) / e;
    numax = fmax(numax, nu);
    numin = fmin(numin, nu);
  }
  double mx[1] = {numax}, mn[1] = {-numin};
  block_reduce<1, true>(mx);
  block_reduce<1, true>(mn);
  if (threadIdx.x == 0) {
    sc->nu = mx[0];
    sc->nu_min = -mn[0];
    sc->counter[kCntBlk] = 0u;
  }
}

// Reweighting (§3.3): w = delta / (delta + |alpha|).
__global__ void k_reweight(int64_t n, const float2* __restrict__ alpha, float* __restrict__ w, int round,
                           const DevScalars* sc) {
  const double amax = sc->amax;
  const float delta = (float)fmax(pow(10.0, -(double)round) * amax, 1e-6 * amax);
  GRID_STRIDE(j, n) {
    if (delta == 0.f) {
      w[j] = 1.0f;
    } else {
      const float a = sqrtf(fmaf(alpha[j].x, alpha[j].x, alpha[j].y * alpha[j].y));
      w[j] = delta / (delta + a);
    }
  }
}

__global__ void k_gather(int64_t n, const float2* __restrict__ src, const int* __restrict__ perm,
                         float2* __restrict__ dst) {
  GRID_STRIDE(i, n) dst[i] = src[perm[i]];
}

// bf16 storage of y: one CTA per block of 4096 visibilities, scale = max |component|.
__global__ void __launch_bounds__(256) k_quantize_bf16(int64_t M, const float2* __restrict__ y,
                                                       uint32_t* __restrict__ yb, float* __restrict__ yscale) {
  __shared__ float wmax[8];
  const int64_t b0 = (int64_t)blockIdx.x * 4096;
  const int64_t b1 = min(b0 + 4096, M);
  float m = 0.f;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) m = fmaxf(m, fmaxf(fabsf(y[i].x), fabsf(y[i].y)));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  m = 0.f;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = fmaxf(m, wmax[k]);
  const float sc = m > 0.f ? m : 1.f;
  if (threadIdx.x == 0) yscale[blockIdx.x] = sc;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    const __nv_bfloat16 re = __float2bfloat16_rn(y[i].x / sc);
    const __nv_bfloat16 im = __float2bfloat16_rn(y[i].y / sc);
    yb[i] = (uint32_t)__bfloat16_as_ushort(re) | ((uint32_t)__bfloat16_as_ushort(im) << 16);
  }
}

__global__ void k_set_gamma(DevScalars* sc, double beta) { sc->gamma = beta * sc->amax; }

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int launch_soft_threshold(int64_t count, const float2* in, const float* w, const double* gamma_dev, float gamma,
                          float2* out, cudaStream_t s) {
  PURIFY_LAUNCH(nullptr, "soft", s, (k_soft<<<blocks_for(count), 256, 0, s>>>(count, in, w, gamma_dev, gamma, out)));
  return check_cuda(cudaGetLastError());
}

int launch_l2_norm_diff(purify_ctx* c, int64_t count, const float2* a, const float2* b, cudaStream_t s) {
  PURIFY_LAUNCH(c, "norm_diff", s, (k_norm_diff<<<blocks_for(count), 256, 0, s>>>(count, a, b, c->d_partials, c->d_sc)));
  return check_cuda(cudaGetLastError());
}

int launch_l2_project(int64_t count, const float2* in, const float2* y, double eps, const double* norm2_dev,
                      float2* out, cudaStream_t s) {
  PURIFY_LAUNCH(nullptr, "l2_project", s, (k_l2_project<<<blocks_for(count), 256, 0, s>>>(count, in, y, eps, norm2_dev, out)));
  return check_cuda(cudaGetLastError());
}

int launch_positive(int64_t count, const float2* in, float2* out, cudaStream_t s) {
  PURIFY_LAUNCH(nullptr, "positive", s, (k_positive<<<blocks_for(count), 256, 0, s>>>(count, in, out)));
  return check_cuda(cudaGetLastError());
}

int launch_cg_apply(purify_ctx* c, float2* x, float2* r, float2* p, float2* sv, const float2* w, int cg_j,
                    cudaStream_t s) {
  const int64_t N = (int64_t)c->n * c->n;
  PURIFY_LAUNCH(c, "cg_apply", s, (k_cg_apply<<<blocks_for(N), 256, 0, s>>>(N, x, r, p, sv, w, c->d_partials, c->d_sc,
                                                                           cg_consumer_blocks(c), cg_j)));
  return check_cuda(cudaGetLastError());
}

int launch_cg_residual_init(purify_ctx* c, const float2* b, const float2* qx, float2* r, cudaStream_t s) {
  const int64_t N = (int64_t)c->n * c->n;
  PURIFY_LAUNCH(c, "cg_residual_init", s, (k_cg_residual_init<<<blocks_for(N), 256, 0, s>>>(N, b, qx, r, c->d_sc)));
  return check_cuda(cudaGetLastError());
}

int launch_max_abs(purify_ctx* c, int64_t count, const float2* a, cudaStream_t s) {
  PURIFY_LAUNCH(c, "max_abs", s, (k_max_abs<<<blocks_for(count), 256, 0, s>>>(count, a, c->d_partials, c->d_sc)));
  return check_cuda(cudaGetLastError());
}

int launch_sdmm_l2_update(purify_sdmm_state* st, cudaStream_t s) {
  purify_ctx* c = st->ctx;
  const bool blk = st->nblocks > 0;
  PURIFY_LAUNCH(st->ctx, "sdmm_l2", s, (k_sdmm_l2<<<blocks_for(c->M), 256, 0, s>>>(c->M, st->s2, st->z2, st->y_bf16 ? nullptr : st->y, st->yb,
                                             st->yscale, st->v, c->d_sc, blk ? st->d_block_of : nullptr,
                                             blk ? st->d_bscale : nullptr)));
  return check_cuda(cudaGetLastError());
}

int launch_block_norms(purify_sdmm_state* st, cudaStream_t s) {
  purify_ctx* c = st->ctx;
  PURIFY_LAUNCH(c, "block_norms", s,
                (k_block_norms<<<st->nbchunks, 256, 0, s>>>(st->d_bchunks, st->nbchunks, st->d_pos, st->s2, st->z2,
                                                            st->y_bf16 ? nullptr : st->y, st->yb, st->yscale,
                                                            st->nblocks, st->d_beps, st->d_bscale,
                                                            c->d_partials + kCntBlk * 2 * kMaxPartials, c->d_sc)));
  return check_cuda(cudaGetLastError());
}

int launch_reweight(purify_ctx* c, int64_t count, const float2* alpha, float* w, int round, cudaStream_t s) {
  PURIFY_LAUNCH(c, "reweight", s, (k_reweight<<<blocks_for(count), 256, 0, s>>>(count, alpha, w, round, c->d_sc)));
  return check_cuda(cudaGetLastError());
}

int launch_gather_perm(int64_t M, const float2* src, const int* perm, float2* dst, cudaStream_t s) {
  PURIFY_LAUNCH(nullptr, "gather", s, (k_gather<<<blocks_for(M), 256, 0, s>>>(M, src, perm, dst)));
  return check_cuda(cudaGetLastError());
}

int launch_quantize_bf16(int64_t M, const float2* y, uint16_t* yb, float* yscale, cudaStream_t s) {
  const int64_t blocks = (M + 4095) / 4096;
  PURIFY_LAUNCH(nullptr, "quantize_bf16", s, (k_quantize_bf16<<<(unsigned)blocks, 256, 0, s>>>(M, y, reinterpret_cast<uint32_t*>(yb), yscale)));
  return check_cuda(cudaGetLastError());
}

int launch_set_gamma(purify_ctx* c, double beta, cudaStream_t s) {
  PURIFY_LAUNCH(c, "set_gamma", s, (k_set_gamma<<<1, 1, 0, s>>>(c->d_sc, beta)));
  return check_cuda(cudaGetLastError());
}

}  // namespace purify
