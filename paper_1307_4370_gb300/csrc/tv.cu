// Weighted total variation prior (§3.3 eq. tvproblem, §5 weighted TV).
//
// f1(x) = ||W grad x||_1 with the isotropic gradient magnitude of forward
// differences (zero on the last row and column), complex pixels counted by
// modulus.  Its prox, prox_{lam f1}(b) = argmin 1/2||x - b||^2 + lam f1(x),
// is computed as §5 states SOPT does, with the fast gradient projection of
// Beck & Teboulle (2009) on the dual pair (p, q):
//   L(p, q)_{i,j} = p_{i,j} + q_{i,j} - p_{i-1,j} - q_{i,j-1}      (-div)
//   L^T(z)        = (z_{i,j} - z_{i+1,j}, z_{i,j} - z_{i,j+1})      (-grad)
//   (p, q)_k = Proj_{|.| <= w}[(r, s) + L^T(b - lam L(r, s)) / (8 lam)]
//   (r, s)   = (p, q)_k + c_k ((p, q)_k - (p, q)_{k-1}),  c_k = (t_k - 1) / t_{k+1}
//   x        = b - lam L(p_K, q_K)
// One launch per FGP iteration (the iterations are coupled through the
// neighbours); each thread owns one pixel and reads the dual values of its
// few neighbours (L1-cached).  The momentum coefficients are host constants.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "reduce.cuh"

#define TV_TRY(expr)                  \
  do {                                \
    const int _st = (expr);           \
    if (_st != PURIFY_OK) return _st; \
  } while (0)

namespace purify {

namespace {

// L(r, s) at (i, j) of an m x n image (row-major, m = n here).
__device__ __forceinline__ float2 op_L(const float2* __restrict__ r, const float2* __restrict__ s, int i, int j,
                                       int n) {
  float2 v = make_float2(0.f, 0.f);
  const int k = i * n + j;
  if (i < n - 1) v = cadd(v, r[k]);
  if (j < n - 1) v = cadd(v, s[k]);
  if (i > 0) v = csub(v, r[k - n]);
  if (j > 0) v = csub(v, s[k - 1]);
  return v;
}

__device__ __forceinline__ float tv_lambda(const DevScalars* sc, float lam) {
  return sc ? (float)sc->gamma : lam;
}

// b = x_hat + z1 (SDMM) or the prox input; dual variables and momentum to zero.
__global__ void k_tv_init(int64_t N, const float2* __restrict__ xa, const float2* __restrict__ xb,
                          float2* __restrict__ b, float2* __restrict__ r, float2* __restrict__ s,
                          float2* __restrict__ p, float2* __restrict__ q) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    b[k] = xb ? cadd(xa[k], xb[k]) : xa[k];
    const float2 z = make_float2(0.f, 0.f);
    r[k] = z;
    s[k] = z;
    p[k] = z;
    q[k] = z;
  }
}

// One FGP iteration: (r, s) -> (r2, s2), (p, q) updated in place.
__global__ void k_tv_fgp_step(int n, const float2* __restrict__ b, const float2* __restrict__ r,
                              const float2* __restrict__ s, float2* __restrict__ p, float2* __restrict__ q,
                              float2* __restrict__ r2, float2* __restrict__ s2, const float* __restrict__ w,
                              float cmom, const DevScalars* __restrict__ sc, float lam_host) {
  const float lam = tv_lambda(sc, lam_host);
  const int64_t N = (int64_t)n * n;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    if (!(lam > 0.f)) {
      r2[k] = make_float2(0.f, 0.f);
      s2[k] = make_float2(0.f, 0.f);
      continue;
    }
    const int i = (int)k / n, j = (int)k - i * n;
    // z = b - lam L(r, s) at (i, j), (i + 1, j), (i, j + 1); g = L^T z at (i, j)
    const float2 z0 = csub(b[k], cscale(op_L(r, s, i, j, n), lam));
    float2 g1 = make_float2(0.f, 0.f), g2 = g1;
    if (i < n - 1) g1 = csub(z0, csub(b[k + n], cscale(op_L(r, s, i + 1, j, n), lam)));
    if (j < n - 1) g2 = csub(z0, csub(b[k + 1], cscale(op_L(r, s, i, j + 1, n), lam)));
    const float step = 1.0f / (8.0f * lam);
    float2 pn = make_float2(fmaf(step, g1.x, r[k].x), fmaf(step, g1.y, r[k].y));
    float2 qn = make_float2(fmaf(step, g2.x, s[k].x), fmaf(step, g2.y, s[k].y));
    if (i == n - 1) pn = make_float2(0.f, 0.f);
    if (j == n - 1) qn = make_float2(0.f, 0.f);
    // projection of the pair onto the disc of radius w
    const float rad = w ? w[k] : 1.0f;
    const float mag = sqrtf(pn.x * pn.x + pn.y * pn.y + qn.x * qn.x + qn.y * qn.y);
    if (mag > rad) {
      const float f = rad / mag;
      pn = cscale(pn, f);
      qn = cscale(qn, f);
    }
    const float2 po = p[k], qo = q[k];
    p[k] = pn;
    q[k] = qn;
    r2[k] = make_float2(fmaf(cmom, pn.x - po.x, pn.x), fmaf(cmom, pn.y - po.y, pn.y));
    s2[k] = make_float2(fmaf(cmom, qn.x - qo.x, qn.x), fmaf(cmom, qn.y - qo.y, qn.y));
  }
}

// x = b - lam L(p, q).  SDMM mode (z1 non-null): r1 = x, z1 <- b - r1 (= z1 +
// x_hat - r1), x1 = r1 - z1, and f1 = ||W grad x_hat||_1 with zeta (FP64
// across threads, exact FP32 products per thread).  Plain mode: out = x.
__global__ void k_tv_finish(int n, const float2* __restrict__ b, const float2* __restrict__ p,
                            const float2* __restrict__ q, float2* __restrict__ out, float2* __restrict__ z1,
                            const float2* __restrict__ xhat, const float* __restrict__ w, double* partials,
                            DevScalars* sc, float lam_host) {
  const float lam = tv_lambda(z1 ? sc : nullptr, lam_host);
  const int64_t N = (int64_t)n * n;
  FPair f1;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)k / n, j = (int)k - i * n;
    const float2 bk = b[k];
    const float2 x = (lam > 0.f) ? csub(bk, cscale(op_L(p, q, i, j, n), lam)) : bk;
    if (!z1) {
      out[k] = x;
      continue;
    }
    const float2 zn = csub(bk, x);  // z1 + x_hat - r1
    z1[k] = zn;
    out[k] = csub(x, zn);           // x1 = r1 - z1
    // f1 term of this pixel: w |grad x_hat|
    const float2 xc = xhat[k];
    float2 d1 = make_float2(0.f, 0.f), d2 = d1;
    if (i < n - 1) d1 = csub(xhat[k + n], xc);
    if (j < n - 1) d2 = csub(xhat[k + 1], xc);
    const float mag = sqrtf(d1.x * d1.x + d1.y * d1.y + d2.x * d2.x + d2.y * d2.y);
    f1.add_prod(w ? w[k] : 1.0f, mag);
  }
  if (!z1) return;
  double v = f1.value(), tot;
  if (reduce_last_block<1>(&v, partials + kCntF1 * 2 * kMaxPartials, &sc->counter[kCntF1], &tot)) {
    sc->f1 = tot;
    const double prev = sc->f1_prev;
    sc->zeta = (prev != 0.0) ? fabs(tot - prev) / fabs(prev) : INFINITY;
    sc->f1_prev = tot;
  }
}

// |grad x| per pixel, as complex (|grad x|, 0) so the complex max and
// reweighting kernels apply.
__global__ void k_tv_gradmag(int n, const float2* __restrict__ x, float2* __restrict__ g) {
  const int64_t N = (int64_t)n * n;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)k / n, j = (int)k - i * n;
    const float2 xc = x[k];
    float2 d1 = make_float2(0.f, 0.f), d2 = d1;
    if (i < n - 1) d1 = csub(x[k + n], xc);
    if (j < n - 1) d2 = csub(x[k + 1], xc);
    g[k] = make_float2(sqrtf(d1.x * d1.x + d1.y * d1.y + d2.x * d2.x + d2.y * d2.y), 0.f);
  }
}

unsigned tv_blocks(int64_t N) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 4096)); }

}  // namespace

// The FGP iterations on b into scratch; `sc` non-null takes lam = gamma from
// the device scalars (SDMM), otherwise lam_host.  Scratch: 6 N complex after b.
static int tv_fgp(purify_ctx* c, float2* scratch, const float* w, int iters, const DevScalars* sc, float lam_host,
                  cudaStream_t s) {
  const int64_t N = ((int64_t)c->n * c->n);
  float2* b = scratch;
  float2* r[2] = {scratch + N, scratch + 3 * N};
  float2* sv[2] = {scratch + 2 * N, scratch + 4 * N};
  float2* p = scratch + 5 * N;
  float2* q = scratch + 6 * N;
  double t = 1.0;
  for (int k = 0; k < iters; ++k) {
    const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
    const float cm = (float)((t - 1.0) / tn);
    t = tn;
    const int a = k & 1;
    PURIFY_LAUNCH(c, "tv_fgp", s,
                  (k_tv_fgp_step<<<tv_blocks(N), 256, 0, s>>>(c->n, b, r[a], sv[a], p, q, r[a ^ 1], sv[a ^ 1], w, cm,
                                                              sc, lam_host)));
  }
  return check_cuda(cudaGetLastError());
}

int tv_scratch_ready(purify_ctx* c, float2** out) {
  if (!c->d_tv) {
    const int64_t N = ((int64_t)c->n * c->n);
    if (cudaMalloc(&c->d_tv, 7 * N * sizeof(float2)) != cudaSuccess) {
      c->d_tv = nullptr;
      cudaGetLastError();
      return PURIFY_E_ALLOC;
    }
  }
  *out = c->d_tv;
  return PURIFY_OK;
}

// SDMM branch i = 1 for the TV prior: r1 = prox_{gamma f1}(x_hat + z1),
// z1 <- z1 + x_hat - r1, x1 = r1 - z1, and f1, zeta.
int tv_sdmm_branch(purify_ctx* c, purify_sdmm_state* st, cudaStream_t s) {
  const int64_t N = ((int64_t)c->n * c->n);
  float2* sc_buf = nullptr;
  TV_TRY(tv_scratch_ready(c, &sc_buf));
  PURIFY_LAUNCH(c, "tv_init", s,
                (k_tv_init<<<tv_blocks(N), 256, 0, s>>>(N, st->xhat, st->z1, sc_buf, sc_buf + N, sc_buf + 2 * N,
                                                        sc_buf + 5 * N, sc_buf + 6 * N)));
  TV_TRY(tv_fgp(c, sc_buf, st->w, st->fgp_iters, c->d_sc, 0.f, s));
  PURIFY_LAUNCH(c, "tv_finish", s,
                (k_tv_finish<<<tv_blocks(N), 256, 0, s>>>(c->n, sc_buf, sc_buf + 5 * N, sc_buf + 6 * N, st->x1, st->z1,
                                                          st->xhat, st->w, c->d_partials, c->d_sc, 0.f)));
  return check_cuda(cudaGetLastError());
}

// |grad x| into the TV scratch (complex), for gamma and reweighting.
int tv_gradmag(purify_ctx* c, const float2* x, float2** g, cudaStream_t s) {
  float2* sc_buf = nullptr;
  TV_TRY(tv_scratch_ready(c, &sc_buf));
  PURIFY_LAUNCH(c, "tv_gradmag", s, (k_tv_gradmag<<<tv_blocks(((int64_t)c->n * c->n)), 256, 0, s>>>(c->n, x, sc_buf)));
  *g = sc_buf;
  return check_cuda(cudaGetLastError());
}

// Standalone prox of lam ||W grad .||_1.
int tv_prox(purify_ctx* c, const float2* in, const float* w, float lam, int iters, float2* out, cudaStream_t s) {
  const int64_t N = ((int64_t)c->n * c->n);
  float2* sc_buf = nullptr;
  TV_TRY(tv_scratch_ready(c, &sc_buf));
  PURIFY_LAUNCH(c, "tv_init", s,
                (k_tv_init<<<tv_blocks(N), 256, 0, s>>>(N, in, nullptr, sc_buf, sc_buf + N, sc_buf + 2 * N,
                                                        sc_buf + 5 * N, sc_buf + 6 * N)));
  TV_TRY(tv_fgp(c, sc_buf, w, iters, nullptr, lam, s));
  PURIFY_LAUNCH(c, "tv_finish", s,
                (k_tv_finish<<<tv_blocks(N), 256, 0, s>>>(c->n, sc_buf, sc_buf + 5 * N, sc_buf + 6 * N, out, nullptr,
                                                          nullptr, nullptr, nullptr, nullptr, lam)));
  return check_cuda(cudaGetLastError());
}

}  // namespace purify
