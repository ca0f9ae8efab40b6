// Differentiation of the SDMM iteration (the unrolled-solver graft): one
// iteration of Algorithm 1 (§4.3-§4.4) for the weighted problem
//   min ||W Psi^H x||_1  s.t.  ||y_w - Phi_w x|| <= eps,  x >= 0,
// Phi_w = diag(w) Phi, y_w = w o y (§5: weighting matrices fold into Phi),
// run forward with a tape, and its vector-Jacobian product (reverse mode)
// from that tape.  Every vector operation is a kernel of this file or one of
// the library's operators (Phi, Phi^H, Psi, Psi^H); the scalar recurrences
// of CG (a few doubles per step) run on the host.
//
// Forward, from the input state S = (x_hat, z1, z2, z3, x1, x2, x3), as the
// oracle's Algorithm 1 steps 5-9 with S = 3:
//   step 5   x_hat' = CG_k(Q_w, b = x1 + x2 + x3, x0 = x_hat),  Q_w = Phi_w^H Phi_w + 2I,
//            standard CG with k steps (stops early when <r, r> = 0);
//   i = 1    a1 = Psi^H x_hat' + z1,  r1 = S(a1, gamma omega),  z1' = a1 - r1,  x1' = Psi (2 r1 - a1);
//   i = 2    a2 = w o Phi x_hat' + z2,  r2 = P_B(a2) (ball of radius eps around y_w),
//            z2' = a2 - r2,  x2' = Phi_w^H (2 r2 - a2);
//   i = 3    a3 = x_hat' + z3,  r3 = max(Re a3, 0),  z3' = a3 - r3,  x3' = 2 r3 - a3.
// Complex vectors are treated as real pairs (§4.1): the adjoint of a complex
// entry is dL/dRe + i dL/dIm, and <a, b> = Re sum conj(a) b.
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "reduce.cuh"

namespace purify {

namespace {

#define DGRID(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

unsigned dblocks(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 2048)); }

// ---------------------------------------------------------------------------
// Elementwise and reduction kernels
// ---------------------------------------------------------------------------
// out = w^pw o in (complex by real), pw = 1 or 2
__global__ void k_wmul(int64_t n, const float2* __restrict__ in, const float* __restrict__ w, int pw,
                       float2* __restrict__ out) {
  DGRID(i, n) {
    const float s = pw == 2 ? w[i] * w[i] : w[i];
    out[i] = cscale(in[i], s);
  }
}

// Re <a, b> in FP64 -> *out
__global__ void k_dot(int64_t n, const float2* __restrict__ a, const float2* __restrict__ b, double* partials,
                      unsigned* counter, double* out) {
  FPair part;
  DGRID(i, n) {
    part.add_prod(a[i].x, b[i].x);
    part.add_prod(a[i].y, b[i].y);
  }
  double v = part.value(), tot;
  if (reduce_last_block<1>(&v, partials, counter, &tot)) *out = tot;
}

// ||a - w o y||^2 in FP64 -> *out
__global__ void k_norm_wdiff(int64_t n, const float2* __restrict__ a, const float* __restrict__ w,
                             const float2* __restrict__ y, double* partials, unsigned* counter, double* out) {
  FPair part;
  DGRID(i, n) {
    const float2 d = csub(a[i], cscale(y[i], w[i]));
    part.add_prod(d.x, d.x);
    part.add_prod(d.y, d.y);
  }
  double v = part.value(), tot;
  if (reduce_last_block<1>(&v, partials, counter, &tot)) *out = tot;
}

// Re <a - w o y, r> in FP64 -> *out
__global__ void k_dot_wdiff(int64_t n, const float2* __restrict__ a, const float* __restrict__ w,
                            const float2* __restrict__ y, const float2* __restrict__ r, double* partials,
                            unsigned* counter, double* out) {
  FPair part;
  DGRID(i, n) {
    const float2 d = csub(a[i], cscale(y[i], w[i]));
    part.add_prod(d.x, r[i].x);
    part.add_prod(d.y, r[i].y);
  }
  double v = part.value(), tot;
  if (reduce_last_block<1>(&v, partials, counter, &tot)) *out = tot;
}

// out = a + b + c
__global__ void k_sum3(int64_t n, const float2* __restrict__ a, const float2* __restrict__ b,
                       const float2* __restrict__ c, float2* __restrict__ out) {
  DGRID(i, n) out[i] = cadd(cadd(a[i], b[i]), c[i]);
}

// out = u - (v + 2 p): the residual b - Q x0 with v = Phi_w^H Phi_w x0
__global__ void k_resid0(int64_t n, const float2* __restrict__ u, const float2* __restrict__ v,
                         const float2* __restrict__ p, float2* __restrict__ out, float2* __restrict__ out2) {
  DGRID(i, n) {
    const float2 r = make_float2(u[i].x - v[i].x - 2.f * p[i].x, u[i].y - v[i].y - 2.f * p[i].y);
    out[i] = r;
    if (out2) out2[i] = r;
  }
}

// q = v + 2 p (Q_w p from v = Phi_w^H Phi_w p)
__global__ void k_plus2(int64_t n, const float2* __restrict__ v, const float2* __restrict__ p, float2* __restrict__ q) {
  DGRID(i, n) q[i] = make_float2(fmaf(2.f, p[i].x, v[i].x), fmaf(2.f, p[i].y, v[i].y));
}

// x += alpha p; r_next = r - alpha q
__global__ void k_cg_upd(int64_t n, float alpha, float2* __restrict__ x, const float2* __restrict__ p,
                         const float2* __restrict__ r, const float2* __restrict__ q, float2* __restrict__ rn) {
  DGRID(i, n) {
    x[i] = make_float2(fmaf(alpha, p[i].x, x[i].x), fmaf(alpha, p[i].y, x[i].y));
    rn[i] = make_float2(fmaf(-alpha, q[i].x, r[i].x), fmaf(-alpha, q[i].y, r[i].y));
  }
}

// p_next = r + beta p
__global__ void k_cg_dir(int64_t n, float beta, const float2* __restrict__ r, const float2* __restrict__ p,
                         float2* __restrict__ pn) {
  DGRID(i, n) pn[i] = make_float2(fmaf(beta, p[i].x, r[i].x), fmaf(beta, p[i].y, r[i].y));
}

// i = 1 forward: a1 = s1 + z1 (kept in place of s1), r1 = S(a1, gamma omega),
// z1' = a1 - r1, u1 = 2 r1 - a1
__global__ void k_b1_fwd(int64_t n, float2* __restrict__ a1, const float2* __restrict__ z1,
                         const float* __restrict__ om, float gamma, float2* __restrict__ z1o,
                         float2* __restrict__ u1) {
  DGRID(i, n) {
    const float2 a = cadd(a1[i], z1[i]);
    a1[i] = a;
    const float lam = gamma * om[i];
    const float mag = sqrtf(a.x * a.x + a.y * a.y);
    const float sc = mag > lam ? (mag - lam) / mag : 0.f;
    const float2 r = cscale(a, sc);
    z1o[i] = csub(a, r);
    u1[i] = make_float2(2.f * r.x - a.x, 2.f * r.y - a.y);
  }
}

// i = 2 forward, first half: a2 = w o s + z2 (s = Phi x_hat')
__global__ void k_b2_a(int64_t n, const float2* __restrict__ s, const float* __restrict__ w,
                       const float2* __restrict__ z2, float2* __restrict__ a2) {
  DGRID(i, n) a2[i] = cadd(cscale(s[i], w[i]), z2[i]);
}

// i = 2 forward, second half: r2 = y_w + c (a2 - y_w), z2' = a2 - r2,
// u2 = 2 r2 - a2, and t = w o u2 (gridded next)
__global__ void k_b2_b(int64_t n, const float2* __restrict__ a2, const float* __restrict__ w,
                       const float2* __restrict__ y, float c, float2* __restrict__ z2o, float2* __restrict__ u2,
                       float2* __restrict__ t) {
  DGRID(i, n) {
    const float2 yw = cscale(y[i], w[i]);
    const float2 d = csub(a2[i], yw);
    const float2 r = make_float2(fmaf(c, d.x, yw.x), fmaf(c, d.y, yw.y));
    z2o[i] = csub(a2[i], r);
    const float2 u = make_float2(2.f * r.x - a2[i].x, 2.f * r.y - a2[i].y);
    u2[i] = u;
    t[i] = cscale(u, w[i]);
  }
}

// i = 3 forward: a3 = x_hat' + z3, r3 = max(Re a3, 0), z3' = a3 - r3, x3' = 2 r3 - a3
__global__ void k_b3_fwd(int64_t n, const float2* __restrict__ xh, const float2* __restrict__ z3,
                         float2* __restrict__ a3o, float2* __restrict__ z3o, float2* __restrict__ x3o) {
  DGRID(i, n) {
    const float2 a = cadd(xh[i], z3[i]);
    a3o[i] = a;
    const float r = fmaxf(a.x, 0.f);
    z3o[i] = make_float2(a.x - r, a.y);
    x3o[i] = make_float2(2.f * r - a.x, -a.y);
  }
}

// ---------------------------------------------------------------------------
// Vector-Jacobian products of the proximity operators (§4.4 eqs. prox1-prox3)
// ---------------------------------------------------------------------------
// Soft threshold r = S(a, lam), lam = gamma omega (eq. prox1): for |a| > lam,
// r = a (1 - lam/|a|), so abar = (1 - lam/|a|) rbar + (lam/|a|^3) a <a, rbar>
// and dL/dlam = -<a, rbar>/|a|; zero where |a| <= lam.  omega_bar += gamma
// dL/dlam (when omega_bar is not NULL).
__device__ __forceinline__ float2 vjp_soft(float2 a, float lam, float2 rb, float& dlam) {
  const float m2 = a.x * a.x + a.y * a.y;
  const float mag = sqrtf(m2);
  if (!(mag > lam)) {
    dlam = 0.f;
    return make_float2(0.f, 0.f);
  }
  const float ar = a.x * rb.x + a.y * rb.y;
  const float k1 = 1.f - lam / mag, k2 = lam / (mag * m2) * ar;
  dlam = -ar / mag;
  return make_float2(fmaf(k1, rb.x, k2 * a.x), fmaf(k1, rb.y, k2 * a.y));
}

__global__ void k_vjp_soft(int64_t n, const float2* __restrict__ a, const float* __restrict__ om, float gamma,
                           const float2* __restrict__ rb, float2* __restrict__ ab, float* __restrict__ omb) {
  DGRID(i, n) {
    const float w = om ? om[i] : 1.f;
    float dlam;
    ab[i] = vjp_soft(a[i], gamma * w, rb[i], dlam);
    if (omb) omb[i] += gamma * dlam;
  }
}

// Positivity r = max(Re a, 0) + 0i (eq. prox3): abar = (Re rbar [Re a > 0], 0).
__global__ void k_vjp_pos(int64_t n, const float2* __restrict__ a, const float2* __restrict__ rb,
                          float2* __restrict__ ab) {
  DGRID(i, n) ab[i] = make_float2(a[i].x > 0.f ? rb[i].x : 0.f, 0.f);
}

// l2-ball projection r = c_ + c (a - c_), c = min(1, eps/||a - c_||) around
// the centre c_ (eq. prox2 read as the projection onto B): inside the ball
// abar = rbar; outside, with d = a - c_, dbar = c (rbar - d <d, rbar>/||d||^2),
// abar = dbar and the centre's adjoint is rbar - dbar.  dr = <d, rbar> and
// nd = ||d|| come from FP64 reductions.
__global__ void k_vjp_ball(int64_t n, const float2* __restrict__ a, const float2* __restrict__ ctr, int outside,
                           float c, float k2, const float2* __restrict__ rb, float2* __restrict__ ab,
                           float2* __restrict__ cb) {
  DGRID(i, n) {
    if (!outside) {
      ab[i] = rb[i];
      if (cb) cb[i] = make_float2(0.f, 0.f);
    } else {
      const float2 d = csub(a[i], ctr[i]);
      // dbar = c rbar - (c dr / nd^2) d, k2 = c dr / nd^2
      const float2 db = make_float2(fmaf(c, rb[i].x, -k2 * d.x), fmaf(c, rb[i].y, -k2 * d.y));
      ab[i] = db;
      if (cb) cb[i] = csub(rb[i], db);
    }
  }
}

// i = 3 reverse: rbar3 = 2 x3bar' - z3bar', abar3 = z3bar' - x3bar' + J_P^T rbar3;
// z3bar = abar3 and xbar += abar3 (x_hat' feeds a3)
__global__ void k_b3_bwd(int64_t n, const float2* __restrict__ a3, const float2* __restrict__ z3b_o,
                         const float2* __restrict__ x3b_o, float2* __restrict__ z3b_i, float2* __restrict__ xacc) {
  DGRID(i, n) {
    const float2 zb = z3b_o[i], xb = x3b_o[i];
    const float rbx = 2.f * xb.x - zb.x;
    float2 ab = make_float2(zb.x - xb.x, zb.y - xb.y);
    if (a3[i].x > 0.f) ab.x += rbx;
    z3b_i[i] = ab;
    xacc[i] = cadd(xacc[i], ab);
  }
}

// i = 1 reverse: ubar = Psi^H x1bar' (in ub), rbar1 = 2 ubar - z1bar',
// abar1 = z1bar' - ubar + J_S^T rbar1; z1bar = abar1 (written over z1b, which
// holds z1bar' on entry), omega_bar += gamma dL/dlam
__global__ void k_b1_bwd(int64_t n, const float2* __restrict__ a1, const float* __restrict__ om, float gamma,
                         const float2* __restrict__ ub, float2* __restrict__ z1b, float* __restrict__ omb) {
  DGRID(i, n) {
    const float2 zb = z1b[i], u = ub[i];
    const float2 rb = make_float2(2.f * u.x - zb.x, 2.f * u.y - zb.y);
    float dlam;
    const float2 js = vjp_soft(a1[i], gamma * om[i], rb, dlam);
    z1b[i] = make_float2(zb.x - u.x + js.x, zb.y - u.y + js.y);
    omb[i] += gamma * dlam;
  }
}

// i = 2 reverse, first half: g = Phi x2bar' (M), ubar2 = w o g,
// w_bar += Re(conj(g) u2); rbar2 = 2 ubar2 - z2bar' (into rb),
// partial abar2 = z2bar' - ubar2 (into ab)
__global__ void k_b2_bwd1(int64_t n, const float2* __restrict__ g, const float* __restrict__ w,
                          const float2* __restrict__ u2, const float2* __restrict__ z2b_o, float2* __restrict__ rb,
                          float2* __restrict__ ab, float* __restrict__ wb) {
  DGRID(i, n) {
    const float2 ub = cscale(g[i], w[i]);
    wb[i] += g[i].x * u2[i].x + g[i].y * u2[i].y;
    rb[i] = make_float2(2.f * ub.x - z2b_o[i].x, 2.f * ub.y - z2b_o[i].y);
    ab[i] = csub(z2b_o[i], ub);
  }
}

// i = 2 reverse, second half: through r2 = P_B(a2) around y_w: abar2 += dbar
// (or rbar2 inside the ball), w_bar += Re(conj(y) (rbar2 - dbar)); then
// s2 = w o Phi x_hat': sbar2 = abar2, w_bar += Re(conj(Phi x_hat') abar2),
// z2bar = abar2, t = w o abar2 (gridded into x_bar next)
__global__ void k_b2_bwd2(int64_t n, const float2* __restrict__ a2, const float* __restrict__ w,
                          const float2* __restrict__ y, int outside, float c, float k2, const float2* __restrict__ rb,
                          float2* __restrict__ ab, const float2* __restrict__ phx, float* __restrict__ wb,
                          float2* __restrict__ z2b_i, float2* __restrict__ t) {
  DGRID(i, n) {
    const float2 yw = cscale(y[i], w[i]);
    float2 db, cbar;
    if (!outside) {
      db = rb[i];
      cbar = make_float2(0.f, 0.f);
    } else {
      const float2 d = csub(a2[i], yw);
      db = make_float2(fmaf(c, rb[i].x, -k2 * d.x), fmaf(c, rb[i].y, -k2 * d.y));
      cbar = csub(rb[i], db);
    }
    const float2 a = cadd(ab[i], db);
    wb[i] += y[i].x * cbar.x + y[i].y * cbar.y + phx[i].x * a.x + phx[i].y * a.y;
    z2b_i[i] = a;
    t[i] = cscale(a, w[i]);
  }
}

// w_bar += f w o Re(conj(g) h) (the weights' term of <qbar, Q_w p>)
__global__ void k_wbar_q(int64_t n, float f, const float* __restrict__ w, const float2* __restrict__ g,
                         const float2* __restrict__ h, float* __restrict__ wb) {
  DGRID(i, n) wb[i] += f * w[i] * (g[i].x * h[i].x + g[i].y * h[i].y);
}

// r_bar += p_bar + 2 rho_bar r
__global__ void k_cgb_r(int64_t n, float2* __restrict__ rb, const float2* __restrict__ pb, float tr,
                        const float2* __restrict__ r) {
  DGRID(i, n) rb[i] = make_float2(rb[i].x + pb[i].x + tr * r[i].x, rb[i].y + pb[i].y + tr * r[i].y);
}

// q_bar = -alpha r_bar + pi_bar p
__global__ void k_cgb_q(int64_t n, float alpha, const float2* __restrict__ rb, float pib, const float2* __restrict__ p,
                        float2* __restrict__ qb) {
  DGRID(i, n) qb[i] = make_float2(fmaf(-alpha, rb[i].x, pib * p[i].x), fmaf(-alpha, rb[i].y, pib * p[i].y));
}

// p_bar = beta p_bar + alpha x_bar + pi_bar q + (v + 2 q_bar), v = Phi_w^H Phi_w q_bar
__global__ void k_cgb_p(int64_t n, float beta, float2* __restrict__ pb, float alpha, const float2* __restrict__ xb,
                        float pib, const float2* __restrict__ q, const float2* __restrict__ v,
                        const float2* __restrict__ qb) {
  DGRID(i, n) {
    pb[i] = make_float2(beta * pb[i].x + alpha * xb[i].x + pib * q[i].x + v[i].x + 2.f * qb[i].x,
                        beta * pb[i].y + alpha * xb[i].y + pib * q[i].y + v[i].y + 2.f * qb[i].y);
  }
}

// x_bar0 = x_bar - (v + 2 r_bar); b_bar = r_bar into x1bar, x2bar, x3bar
__global__ void k_cgb_end(int64_t n, const float2* __restrict__ xb, const float2* __restrict__ v,
                          const float2* __restrict__ rb, float2* __restrict__ xb0, float2* __restrict__ b1,
                          float2* __restrict__ b2, float2* __restrict__ b3) {
  DGRID(i, n) {
    const float2 r = rb[i];
    xb0[i] = make_float2(xb[i].x - v[i].x - 2.f * r.x, xb[i].y - v[i].y - 2.f * r.y);
    b1[i] = r;
    b2[i] = r;
    b3[i] = r;
  }
}

// out = a + b
__global__ void k_add(int64_t n, const float2* __restrict__ a, const float2* __restrict__ b, float2* __restrict__ out) {
  DGRID(i, n) out[i] = cadd(a[i], b[i]);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
int64_t nN(const purify_ctx* c) { return (int64_t)c->n * c->n; }
int64_t nD(const purify_ctx* c) { return (int64_t)c->q * c->n * c->n; }

// Tape layout (device): a header of doubles, then complex vectors.
struct TapeHeader {
  double alpha[64], beta[64], rho[65], pi[64];
  double nd;      // ||a2 - y_w||
  double cball;   // min(1, eps / nd)
  int32_t steps;  // CG steps run
  int32_t k;
};
constexpr size_t kHdr = (sizeof(TapeHeader) + 255) / 256 * 256;

struct Tape {
  float2 *R, *P, *Qp, *PhiP, *PhiX0;  // R: k + 1 vectors of N; P, Qp: k of N; PhiP: k of M
  float2 *A1, *U1, *PhiXh, *A2, *U2, *A3;
};

Tape tape_views(const purify_ctx* c, int k, void* base) {
  const int64_t N = nN(c), M = c->M, D = nD(c);
  float2* p = reinterpret_cast<float2*>(static_cast<char*>(base) + kHdr);
  Tape t;
  t.R = p; p += (k + 1) * N;
  t.P = p; p += (int64_t)k * N;
  t.Qp = p; p += (int64_t)k * N;
  t.PhiP = p; p += (int64_t)k * M;
  t.PhiX0 = p; p += M;
  t.A1 = p; p += D;
  t.U1 = p; p += D;
  t.PhiXh = p; p += M;
  t.A2 = p; p += M;
  t.U2 = p; p += M;
  t.A3 = p; p += N;
  return t;
}

size_t tape_bytes(const purify_ctx* c, int k) {
  const int64_t N = nN(c), M = c->M, D = nD(c);
  return kHdr + (size_t)((3 * k + 2) * N + (k + 4) * M + 2 * D) * sizeof(float2);
}

// Scratch of the differentiation calls (allocated on first use): three
// visibility-size and four image-size complex vectors, one coefficient-size.
int diff_scratch(purify_ctx* c, float2** m, float2** im, float2** dv) {
  const int64_t N = nN(c), M = c->M, D = nD(c);
  if (!c->d_diff) {
    if (cudaMalloc((void**)&c->d_diff, (size_t)(3 * M + 4 * N + D) * sizeof(float2)) != cudaSuccess) {
      cudaGetLastError();
      c->d_diff = nullptr;
      return PURIFY_E_ALLOC;
    }
  }
  for (int i = 0; i < 3; ++i) m[i] = c->d_diff + i * M;
  for (int i = 0; i < 4; ++i) im[i] = c->d_diff + 3 * M + i * N;
  *dv = c->d_diff + 3 * M + 4 * N;
  return PURIFY_OK;
}

// Phi v (caller order) into out (M)
int phi_into(purify_ctx* c, const float2* v, float2* out, cudaStream_t s) {
  RowInArgs ia{};
  ia.in = v;
  if (int rc = phi_forward_grid(c, kRowInPlain, ia, s)) return rc;
  DegridArgs da{};
  da.out = out;
  return degrid(c, kDegridPerm, da, s);
}

// Phi^H u (u in caller order) into out (N)
int phi_adj_into(purify_ctx* c, const float2* u, float2* out, cudaStream_t s) {
  if (int rc = grid_adjoint(c, kGridPerm, u, s)) return rc;
  RowOutArgs ra{};
  ra.out = out;
  return phi_adjoint_image(c, kRowOutPlain, ra, s);
}

int host_dot(purify_ctx* c, int64_t n, const float2* a, const float2* b, double* out, cudaStream_t s) {
  double* slot = &c->d_sc->norm2;
  k_dot<<<dblocks(n), 256, 0, s>>>(n, a, b, c->d_partials + kCntNorm * 2 * kMaxPartials, &c->d_sc->counter[kCntNorm],
                                  slot);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (int rc = check_cuda(cudaGetLastError())) return rc;
  if (int rc = check_cuda(cudaMemcpyAsync(out, slot, sizeof(double), cudaMemcpyDeviceToHost, s))) return rc;
  return check_cuda(cudaStreamSynchronize(s));
}

#define LAUNCH(stmt)                                         \
  do {                                                       \
    stmt;                                                    \
    g_launches.fetch_add(1, std::memory_order_relaxed);      \
    if (int _rc = check_cuda(cudaGetLastError())) return _rc; \
  } while (0)

// v = Phi_w^H Phi_w p (without the 2p); g (M) receives Phi p, t (M) is scratch
int apply_ww(purify_ctx* c, const float2* p, const float* w, float2* g, float2* t, float2* v, cudaStream_t s) {
  const int64_t M = c->M;
  if (int rc = phi_into(c, p, g, s)) return rc;
  LAUNCH((k_wmul<<<dblocks(M), 256, 0, s>>>(M, g, w, 2, t)));
  return phi_adj_into(c, t, v, s);
}

struct DiffArgs {
  const float2* y;
  const float* w;
  const float* om;
  double gamma, eps;
  int k;
};

bool ok_dev(const void* p) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  int cur = -1;
  cudaGetDevice(&cur);
  return a.type == cudaMemoryTypeDevice && a.device == cur;
}

int diff_forward(purify_ctx* c, const DiffArgs& A, float2* const* in, float2* const* out, void* tape_mem,
                 cudaStream_t s) {
  const int64_t N = nN(c), M = c->M, D = nD(c);
  const int k = A.k;
  float2 *m[3], *im[4], *dv;
  if (int rc = diff_scratch(c, m, im, &dv)) return rc;
  if (!tape_mem) return PURIFY_E_INVALID_ARG;  // the forward keeps its vectors on the tape
  Tape T = tape_views(c, k, tape_mem);
  TapeHeader H;
  std::memset(&H, 0, sizeof(H));
  H.k = k;
  // ---- step 5: b = x1 + x2 + x3; r0 = b - Q_w x0; CG from x0 = x_hat
  float2* b = im[0];
  float2* x = out[0];
  LAUNCH((k_sum3<<<dblocks(N), 256, 0, s>>>(N, in[4], in[5], in[6], b)));
  if (int rc = check_cuda(cudaMemcpyAsync(x, in[0], N * sizeof(float2), cudaMemcpyDeviceToDevice, s))) return rc;
  if (int rc = apply_ww(c, x, A.w, T.PhiX0, m[0], im[1], s)) return rc;
  LAUNCH((k_resid0<<<dblocks(N), 256, 0, s>>>(N, b, im[1], x, T.R, T.P)));
  double rho;
  if (int rc = host_dot(c, N, T.R, T.R, &rho, s)) return rc;
  H.rho[0] = rho;
  int steps = 0;
  for (int j = 0; j < k; ++j) {
    if (rho == 0.0) break;  // as the oracle: nothing left to do
    float2* pj = T.P + (int64_t)j * N;
    float2* qj = T.Qp + (int64_t)j * N;
    if (int rc = apply_ww(c, pj, A.w, T.PhiP + (int64_t)j * M, m[0], im[1], s)) return rc;
    LAUNCH((k_plus2<<<dblocks(N), 256, 0, s>>>(N, im[1], pj, qj)));
    double pq;
    if (int rc = host_dot(c, N, pj, qj, &pq, s)) return rc;
    const double alpha = pq > 0.0 ? rho / pq : 0.0;
    LAUNCH((k_cg_upd<<<dblocks(N), 256, 0, s>>>(N, (float)alpha, x, pj, T.R + (int64_t)j * N, qj,
                                                 T.R + (int64_t)(j + 1) * N)));
    double rho_n;
    if (int rc = host_dot(c, N, T.R + (int64_t)(j + 1) * N, T.R + (int64_t)(j + 1) * N, &rho_n, s)) return rc;
    const double beta = rho_n / rho;
    if (j + 1 < k)
      LAUNCH((k_cg_dir<<<dblocks(N), 256, 0, s>>>(N, (float)beta, T.R + (int64_t)(j + 1) * N, pj,
                                                  T.P + (int64_t)(j + 1) * N)));
    H.alpha[j] = alpha;
    H.beta[j] = beta;
    H.pi[j] = pq;
    H.rho[j + 1] = rho_n;
    rho = rho_n;
    steps = j + 1;
  }
  H.steps = steps;
  // ---- i = 1: a1 = Psi^H x_hat' + z1; z1', x1' = Psi (2 r1 - a1)
  SaraProxArgs pa{};
  if (int rc = sara_analysis(c, x, T.A1, kSaraPlain, pa, s)) return rc;
  LAUNCH((k_b1_fwd<<<dblocks(D), 256, 0, s>>>(D, T.A1, in[1], A.om, (float)A.gamma, out[1], T.U1)));
  if (int rc = sara_synthesis(c, T.U1, out[4], s)) return rc;
  // ---- i = 2: a2 = w o Phi x_hat' + z2; projection onto the ball around y_w
  if (int rc = phi_into(c, x, T.PhiXh, s)) return rc;
  LAUNCH((k_b2_a<<<dblocks(M), 256, 0, s>>>(M, T.PhiXh, A.w, in[2], T.A2)));
  double nd2;
  {
    double* slot = &c->d_sc->norm2;
    LAUNCH((k_norm_wdiff<<<dblocks(M), 256, 0, s>>>(M, T.A2, A.w, A.y, c->d_partials + kCntNorm * 2 * kMaxPartials,
                                                    &c->d_sc->counter[kCntNorm], slot)));
    if (int rc = check_cuda(cudaMemcpyAsync(&nd2, slot, sizeof(double), cudaMemcpyDeviceToHost, s))) return rc;
    if (int rc = check_cuda(cudaStreamSynchronize(s))) return rc;
  }
  const double nd = std::sqrt(nd2);
  const double cb = nd > A.eps ? A.eps / nd : 1.0;
  H.nd = nd;
  H.cball = cb;
  LAUNCH((k_b2_b<<<dblocks(M), 256, 0, s>>>(M, T.A2, A.w, A.y, (float)cb, out[2], T.U2, m[1])));
  if (int rc = phi_adj_into(c, m[1], out[5], s)) return rc;
  // ---- i = 3
  LAUNCH((k_b3_fwd<<<dblocks(N), 256, 0, s>>>(N, x, in[3], T.A3, out[3], out[6])));
  // header last (host staging copy, then synchronise so H may go out of scope)
  if (int rc = check_cuda(cudaMemcpyAsync(tape_mem, &H, sizeof(H), cudaMemcpyHostToDevice, s))) return rc;
  return check_cuda(cudaStreamSynchronize(s));
}

int diff_backward(purify_ctx* c, const DiffArgs& A, float2* const* in, const void* tape_mem, float2* const* ob,
                  float2* const* ib, float* wb, float* omb, cudaStream_t s) {
  const int64_t N = nN(c), M = c->M, D = nD(c);
  const int k = A.k;
  float2 *m[3], *im[4], *dv;
  if (int rc = diff_scratch(c, m, im, &dv)) return rc;
  Tape T = tape_views(c, k, const_cast<void*>(tape_mem));
  TapeHeader H;
  if (int rc = check_cuda(cudaMemcpyAsync(&H, tape_mem, sizeof(H), cudaMemcpyDeviceToHost, s))) return rc;
  if (int rc = check_cuda(cudaStreamSynchronize(s))) return rc;
  if (H.k != k) return PURIFY_E_INVALID_ARG;
  float2* xacc = im[0];  // adjoint of x_hat' (the CG output)
  if (int rc = check_cuda(cudaMemcpyAsync(xacc, ob[0], N * sizeof(float2), cudaMemcpyDeviceToDevice, s))) return rc;
  // ---- i = 3
  LAUNCH((k_b3_bwd<<<dblocks(N), 256, 0, s>>>(N, T.A3, ob[3], ob[6], ib[3], xacc)));
  // ---- i = 1: ubar = Psi^H x1bar'; z1bar; x_bar += Psi abar1
  if (int rc = check_cuda(cudaMemcpyAsync(ib[1], ob[1], D * sizeof(float2), cudaMemcpyDeviceToDevice, s))) return rc;
  SaraProxArgs pa{};
  if (int rc = sara_analysis(c, ob[4], dv, kSaraPlain, pa, s)) return rc;
  LAUNCH((k_b1_bwd<<<dblocks(D), 256, 0, s>>>(D, T.A1, A.om, (float)A.gamma, dv, ib[1], omb)));
  if (int rc = sara_synthesis(c, ib[1], im[1], s)) return rc;
  LAUNCH((k_add<<<dblocks(N), 256, 0, s>>>(N, xacc, im[1], xacc)));
  // ---- i = 2: g = Phi x2bar'; through the ball; x_bar += Phi^H (w o abar2)
  if (int rc = phi_into(c, ob[5], m[0], s)) return rc;
  LAUNCH((k_b2_bwd1<<<dblocks(M), 256, 0, s>>>(M, m[0], A.w, T.U2, ob[2], m[1], m[2], wb)));
  const int outside = H.nd > A.eps ? 1 : 0;
  float k2 = 0.f;
  if (outside) {
    // <d, rbar2>, d = a2 - y_w (FP64): the ball's Jacobian needs it
    double* slot = &c->d_sc->norm2;
    double dr;
    LAUNCH((k_dot_wdiff<<<dblocks(M), 256, 0, s>>>(M, T.A2, A.w, A.y, m[1], c->d_partials + kCntNorm * 2 * kMaxPartials,
                                                   &c->d_sc->counter[kCntNorm], slot)));
    if (int rc = check_cuda(cudaMemcpyAsync(&dr, slot, sizeof(double), cudaMemcpyDeviceToHost, s))) return rc;
    if (int rc = check_cuda(cudaStreamSynchronize(s))) return rc;
    k2 = (float)(H.cball * dr / (H.nd * H.nd));
  }
  LAUNCH((k_b2_bwd2<<<dblocks(M), 256, 0, s>>>(M, T.A2, A.w, A.y, outside, (float)H.cball, k2, m[1], m[2], T.PhiXh,
                                               wb, ib[2], m[0])));
  if (int rc = phi_adj_into(c, m[0], im[1], s)) return rc;
  LAUNCH((k_add<<<dblocks(N), 256, 0, s>>>(N, xacc, im[1], xacc)));
  // ---- step 5: CG reversed (x_bar stays xacc through every step)
  float2* rb = im[1];
  float2* pb = im[2];
  float2* qb = im[3];
  float2* vN = dv;  // the coefficient-size scratch, used as one more image vector
  if (int rc = check_cuda(cudaMemsetAsync(rb, 0, N * sizeof(float2), s))) return rc;
  if (int rc = check_cuda(cudaMemsetAsync(pb, 0, N * sizeof(float2), s))) return rc;
  double rhob = 0.0;  // adjoint of rho_{j+1}, carried down
  for (int j = H.steps - 1; j >= 0; --j) {
    const float2* pj = T.P + (int64_t)j * N;
    const float2* qj = T.Qp + (int64_t)j * N;
    const float2* rj1 = T.R + (int64_t)(j + 1) * N;
    double betab = 0.0;  // p_bar_{j+1} is zero for the last step run
    if (j < H.steps - 1) {
      if (int rc = host_dot(c, N, pb, pj, &betab, s)) return rc;
    }
    const double rho_j = H.rho[j], rho_j1 = H.rho[j + 1], al = H.alpha[j], be = H.beta[j], pq = H.pi[j];
    rhob += betab / rho_j;
    LAUNCH((k_cgb_r<<<dblocks(N), 256, 0, s>>>(N, rb, pb, (float)(2.0 * rhob), rj1)));
    double rq, xp;
    if (int rc = host_dot(c, N, rb, qj, &rq, s)) return rc;
    if (int rc = host_dot(c, N, xacc, pj, &xp, s)) return rc;
    const double alb = pq > 0.0 ? -rq + xp : 0.0;
    const double rhob_j = -betab * rho_j1 / (rho_j * rho_j) + (pq > 0.0 ? alb / pq : 0.0);
    const double pib = pq > 0.0 ? -alb * rho_j / (pq * pq) : 0.0;
    LAUNCH((k_cgb_q<<<dblocks(N), 256, 0, s>>>(N, (float)al, rb, (float)pib, pj, qb)));
    // v = Phi_w^H Phi_w qbar (m0 = Phi qbar); w_bar += 2 w Re(conj(Phi qbar) Phi p_j)
    if (int rc = apply_ww(c, qb, A.w, m[0], m[1], vN, s)) return rc;
    LAUNCH((k_wbar_q<<<dblocks(M), 256, 0, s>>>(M, 2.f, A.w, m[0], T.PhiP + (int64_t)j * M, wb)));
    LAUNCH((k_cgb_p<<<dblocks(N), 256, 0, s>>>(N, (float)be, pb, (float)al, xacc, (float)pib, qj, vN, qb)));
    rhob = rhob_j;
  }
  // p_0 = r_0 and rho_0 = <r_0, r_0>
  LAUNCH((k_cgb_r<<<dblocks(N), 256, 0, s>>>(N, rb, pb, (float)(2.0 * rhob), T.R)));
  // r_0 = b - Q_w x_0: b_bar = r_bar; x0_bar = x_bar - Q_w r_bar; w term
  if (int rc = apply_ww(c, rb, A.w, m[0], m[1], vN, s)) return rc;
  LAUNCH((k_wbar_q<<<dblocks(M), 256, 0, s>>>(M, -2.f, A.w, m[0], T.PhiX0, wb)));
  LAUNCH((k_cgb_end<<<dblocks(N), 256, 0, s>>>(N, xacc, vN, rb, ib[0], ib[4], ib[5], ib[6])));
  return check_cuda(cudaStreamSynchronize(s));
}

}  // namespace

}  // namespace purify

using namespace purify;

extern "C" {

int purify_diff_tape_bytes(purify_ctx* c, int32_t cg_iters, size_t* bytes) {
  if (!c || !bytes || cg_iters < 0 || cg_iters > 64) return PURIFY_E_INVALID_ARG;
  *bytes = tape_bytes(c, cg_iters);
  return PURIFY_OK;
}

int purify_diff_iteration(purify_ctx* c, const float* y, const float* wvis, const float* omega, double gamma,
                          double eps, int32_t cg_iters, const float* const* state_in, float* const* state_out,
                          void* tape, purify_stream_t stream) {
  if (!c || !y || !wvis || !omega || !state_in || !state_out || !tape || cg_iters < 0 || cg_iters > 64 ||
      !(gamma >= 0.0) || !(eps > 0.0))
    return PURIFY_E_INVALID_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  int rc = PURIFY_OK;
  for (int i = 0; i < 7 && rc == PURIFY_OK; ++i)
    if (!ok_dev(state_in[i]) || !ok_dev(state_out[i])) rc = PURIFY_E_NOT_DEVICE_PTR;
  if (rc == PURIFY_OK && (!ok_dev(y) || !ok_dev(wvis) || !ok_dev(omega) || !ok_dev(tape))) rc = PURIFY_E_NOT_DEVICE_PTR;
  if (rc == PURIFY_OK) {
    DiffArgs A{(const float2*)y, wvis, omega, gamma, eps, cg_iters};
    float2* in[7];
    float2* out[7];
    for (int i = 0; i < 7; ++i) {
      in[i] = (float2*)state_in[i];
      out[i] = (float2*)state_out[i];
    }
    rc = diff_forward(c, A, in, out, tape, (cudaStream_t)stream);
  }
  if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
  return rc;
}

int purify_diff_iteration_vjp(purify_ctx* c, const float* y, const float* wvis, const float* omega, double gamma,
                              double eps, int32_t cg_iters, const float* const* state_in, const void* tape,
                              float* const* bar_out, float* const* bar_in, float* wvis_bar, float* omega_bar,
                              purify_stream_t stream) {
  if (!c || !y || !wvis || !omega || !state_in || !tape || !bar_out || !bar_in || !wvis_bar || !omega_bar ||
      cg_iters < 0 || cg_iters > 64 || !(gamma >= 0.0) || !(eps > 0.0))
    return PURIFY_E_INVALID_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  int rc = PURIFY_OK;
  for (int i = 0; i < 7 && rc == PURIFY_OK; ++i)
    if (!ok_dev(state_in[i]) || !ok_dev(bar_out[i]) || !ok_dev(bar_in[i])) rc = PURIFY_E_NOT_DEVICE_PTR;
  if (rc == PURIFY_OK && (!ok_dev(y) || !ok_dev(wvis) || !ok_dev(omega) || !ok_dev(tape) || !ok_dev(wvis_bar) ||
                          !ok_dev(omega_bar)))
    rc = PURIFY_E_NOT_DEVICE_PTR;
  if (rc == PURIFY_OK) {
    DiffArgs A{(const float2*)y, wvis, omega, gamma, eps, cg_iters};
    float2 *in[7], *ob[7], *ib[7];
    for (int i = 0; i < 7; ++i) {
      in[i] = (float2*)state_in[i];
      ob[i] = (float2*)bar_out[i];
      ib[i] = (float2*)bar_in[i];
    }
    rc = diff_backward(c, A, in, tape, ob, ib, wvis_bar, omega_bar, (cudaStream_t)stream);
  }
  if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
  return rc;
}

int purify_diff_penalty(purify_ctx* c, const float* y, const float* wvis, double beta, double* gamma,
                        purify_stream_t stream) {
  if (!c || !y || !wvis || !gamma || !(beta >= 0.0)) return PURIFY_E_INVALID_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  int rc = (ok_dev(y) && ok_dev(wvis)) ? PURIFY_OK : PURIFY_E_NOT_DEVICE_PTR;
  cudaStream_t s = (cudaStream_t)stream;
  float2 *m[3], *im[4], *dv;
  if (rc == PURIFY_OK) rc = diff_scratch(c, m, im, &dv);
  if (rc == PURIFY_OK) {
    // Phi_w^H y_w = Phi^H (w^2 o y), then Psi^H, then the largest modulus
    const int64_t M = c->M;
    k_wmul<<<dblocks(M), 256, 0, s>>>(M, (const float2*)y, wvis, 2, m[0]);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    rc = check_cuda(cudaGetLastError());
    if (rc == PURIFY_OK) rc = phi_adj_into(c, m[0], im[0], s);
    SaraProxArgs pa{};
    if (rc == PURIFY_OK) rc = sara_analysis(c, im[0], dv, kSaraPlain, pa, s);
    if (rc == PURIFY_OK) rc = launch_max_abs(c, nD(c), dv, s);
    double amax = 0.0;
    if (rc == PURIFY_OK) rc = check_cuda(cudaMemcpyAsync(&amax, &c->d_sc->amax, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (rc == PURIFY_OK) rc = check_cuda(cudaStreamSynchronize(s));
    if (rc == PURIFY_OK) *gamma = beta * amax;
  }
  if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
  return rc;
}

int purify_vjp_soft_threshold(int64_t count, const float* a, const float* w, float gamma, const float* rbar,
                              float* abar, float* wbar, purify_stream_t stream) {
  if (count < 0 || !a || !rbar || !abar || !(gamma >= 0.0f)) return PURIFY_E_INVALID_ARG;
  if (count == 0) return PURIFY_OK;
  if (!ok_dev(a) || !ok_dev(rbar) || !ok_dev(abar) || (w && !ok_dev(w)) || (wbar && !ok_dev(wbar)))
    return PURIFY_E_NOT_DEVICE_PTR;
  cudaStream_t s = (cudaStream_t)stream;
  k_vjp_soft<<<dblocks(count), 256, 0, s>>>(count, (const float2*)a, w, gamma, (const float2*)rbar, (float2*)abar,
                                            wbar);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return check_cuda(cudaGetLastError());
}

int purify_vjp_positive(int64_t count, const float* a, const float* rbar, float* abar, purify_stream_t stream) {
  if (count < 0 || !a || !rbar || !abar) return PURIFY_E_INVALID_ARG;
  if (count == 0) return PURIFY_OK;
  if (!ok_dev(a) || !ok_dev(rbar) || !ok_dev(abar)) return PURIFY_E_NOT_DEVICE_PTR;
  cudaStream_t s = (cudaStream_t)stream;
  k_vjp_pos<<<dblocks(count), 256, 0, s>>>(count, (const float2*)a, (const float2*)rbar, (float2*)abar);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return check_cuda(cudaGetLastError());
}

int purify_vjp_l2ball(purify_ctx* c, int64_t count, const float* a, const float* y, double eps, const float* rbar,
                      float* abar, float* ybar, purify_stream_t stream) {
  if (!c || count < 0 || !a || !y || !rbar || !abar || !(eps >= 0.0)) return PURIFY_E_INVALID_ARG;
  if (count == 0) return PURIFY_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  int rc = PURIFY_OK;
  if (!ok_dev(a) || !ok_dev(y) || !ok_dev(rbar) || !ok_dev(abar) || (ybar && !ok_dev(ybar))) rc = PURIFY_E_NOT_DEVICE_PTR;
  cudaStream_t s = (cudaStream_t)stream;
  if (rc == PURIFY_OK) {
    // ||a - y||^2 and <a - y, rbar> = <a, rbar> - <y, rbar> in FP64
    double nd2 = 0.0, ar = 0.0, yr = 0.0, ay = 0.0, aa = 0.0, yy = 0.0;
    const float2 *A = (const float2*)a, *Y = (const float2*)y, *RB = (const float2*)rbar;
    rc = host_dot(c, count, A, A, &aa, s);
    if (rc == PURIFY_OK) rc = host_dot(c, count, Y, Y, &yy, s);
    if (rc == PURIFY_OK) rc = host_dot(c, count, A, Y, &ay, s);
    if (rc == PURIFY_OK) rc = host_dot(c, count, A, RB, &ar, s);
    if (rc == PURIFY_OK) rc = host_dot(c, count, Y, RB, &yr, s);
    if (rc == PURIFY_OK) {
      nd2 = std::max(0.0, aa - 2.0 * ay + yy);
      const double nd = std::sqrt(nd2);
      const int outside = nd > eps ? 1 : 0;
      const double cb = outside ? eps / nd : 1.0;
      const float k2 = outside ? (float)(cb * (ar - yr) / nd2) : 0.f;
      k_vjp_ball<<<dblocks(count), 256, 0, s>>>(count, A, Y, outside, (float)cb, k2, RB, (float2*)abar,
                                                 (float2*)ybar);
      g_launches.fetch_add(1, std::memory_order_relaxed);
      rc = check_cuda(cudaGetLastError());
    }
  }
  if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
  return rc;
}

}  // extern "C"
