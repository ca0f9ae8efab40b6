// Deterministic FP64 block reductions with a "last block finishes" epilogue.
//
// Every block writes its partial sums to a slot of a partial buffer, then
// takes a ticket on a counter; the block that takes the last ticket sums the
// partials in a fixed order and runs the finishing code.  The result does not
// depend on block scheduling, and no extra kernel launch is needed.
#pragma once

#include "common.cuh"

namespace purify {

// ---------------------------------------------------------------------------
// Per-thread accumulation without FP64 arithmetic (GB300 has little FP64
// throughput): terms are formed exactly with error-free transformations
// (TwoSum for a difference, an FMA for a product's rounding error) and summed
// into a float pair (hi, lo); the pair goes to FP64 once per thread, and the
// sums across threads and blocks are FP64.  With the few terms each thread
// holds, the per-thread error is far below FP64 rounding of the total.
// ---------------------------------------------------------------------------
struct FPair {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float p, float pe) {  // += p + pe
    const float s = hi + p;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo += e + pe;
  }
  // += x * y (exact product)
  __device__ __forceinline__ void add_prod(float x, float y) {
    const float p = x * y;
    add(p, fmaf(x, y, -p));
  }
  // += (a - b)^2 with a - b formed exactly
  __device__ __forceinline__ void add_sq_diff(float a, float b) {
    const float d = a - b;
    const float bb = d - a;
    const float de = (a - (d - bb)) + (-b - bb);
    const float p = d * d;
    add(p, fmaf(d, d, -p) + 2.f * d * de);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Tree over the first `valid` lanes of a warp whose first `present` lanes
// exist (any block size, including a partial last warp); every present lane
// calls it, and the result is valid in lane 0.
template <bool MAX>
__device__ __forceinline__ double warp_tree(double v, int lane, int present, int valid) {
  const unsigned mask = present >= 32 ? 0xffffffffu : ((1u << present) - 1u);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_down_sync(mask, v, o);
    if (lane + o < valid) v = MAX ? fmax(v, t) : v + t;
  }
  return v;
}

// Sum (or max) of NV values over the block; the result is valid in thread 0.
template <int NV, bool MAX = false>
__device__ __forceinline__ void block_reduce(double* v) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  const int mylanes = min(32, (int)blockDim.x - wid * 32);
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_tree<MAX>(v[k], lane, mylanes, mylanes);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][wid] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double t = lane < nw ? sh[k][lane] : 0.0;
      v[k] = warp_tree<MAX>(t, lane, mylanes, nw);
    }
  }
}

// Writes the block's NV partials, and in the last block to finish sums all
// partials (fixed order) into total[0..NV).  Returns true in thread 0 of that
// last block only.  partials holds NV x kMaxPartials doubles; the grid must
// have at most kMaxPartials blocks.  The counter is reset for the next use.
template <int NV, bool MAX = false>
__device__ __forceinline__ bool reduce_last_block(double* v, double* partials, unsigned int* counter,
                                                  double* total) {
  __shared__ bool am_last;
  const unsigned int nblk = gridDim.x * gridDim.y * gridDim.z;
  const unsigned int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  block_reduce<NV, MAX>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[k * kMaxPartials + bid] = v[k];
    __threadfence();
    const unsigned int ticket = atomicAdd(counter, 1u);
    am_last = (ticket == nblk - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = 0.0;
    for (unsigned int i = threadIdx.x; i < nblk; i += blockDim.x) {
      const double t = __ldcg(&partials[k * kMaxPartials + i]);
      s = MAX ? fmax(s, t) : s + t;
    }
    acc[k] = s;
  }
  block_reduce<NV, MAX>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) total[k] = acc[k];
    *counter = 0u;
  }
  return threadIdx.x == 0;
}

// ---------------------------------------------------------------------------
// Step sizes of single-reduction CG (Chronopoulos & Gear 1989), formed by the
// kernel that applies the update rather than by a last block of the kernel
// that produced the inner products.  CG step j's Q-epilogue left per-block
// partials of gamma_j = <r, r> and delta_j = <Qr, r>; every block of the
// consumer adds them in the same fixed order (so all blocks agree bit for
// bit) and forms
//   beta_j  = gamma_j / gamma_{j-1}         (0 for the first step)
//   alpha_j = gamma_j / (delta_j - beta_j gamma_j / alpha_{j-1}),
// reading step j-1's (gamma, alpha) from slot (j-1) & 1; block 0 stores step
// j's in slot j & 1, which no block of this kernel reads.  Every thread of
// the block calls it; the results are returned to all of them.  With many
// partials (large images) a one-block kernel forms them once instead
// (k_cg_scalars) and the consumers pass nblk = 0 to read its result.
// ---------------------------------------------------------------------------
struct CgStep {
  float alpha, beta;
  bool first;
};

__device__ __forceinline__ CgStep cg_consume(const double* __restrict__ part, int nblk, int j, DevScalars* sc) {
  __shared__ float s_al, s_be;
  __shared__ int s_first;
  if (nblk == 0) {  // formed by k_cg_scalars for this step (many partials)
    return CgStep{(float)sc->alpha, (float)sc->beta, sc->cg_step_first != 0};
  }
  double v[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
    v[0] += __ldcg(&part[i]);
    v[1] += __ldcg(&part[kMaxPartials + i]);
  }
  block_reduce<2>(v);
  if (threadIdx.x == 0) {
    const double gamma = v[0], delta = v[1];
    const int prev = (j - 1) & 1;
    const double rho_p = j > 0 ? sc->cg_rho[prev] : 0.0, al_p = j > 0 ? sc->cg_alpha[prev] : 0.0;
    const bool first = j == 0 || al_p == 0.0 || rho_p == 0.0;
    const double beta = first ? 0.0 : gamma / rho_p;
    const double den = first ? delta : delta - beta * gamma / al_p;
    const double alpha = den > 0.0 ? gamma / den : 0.0;
    s_al = (float)alpha;
    s_be = (float)beta;
    s_first = first ? 1 : 0;
    if (blockIdx.x == 0) {
      sc->cg_rho[j & 1] = gamma;
      sc->cg_alpha[j & 1] = alpha;
      sc->alpha = alpha;
      sc->beta = beta;
      sc->rho = gamma;
      sc->pqp = den;
      sc->cg_res = sqrt(gamma);
      sc->cg_step_first = first ? 1 : 0;
    }
  }
  __syncthreads();
  return CgStep{s_al, s_be, s_first != 0};
}

}  // namespace purify
