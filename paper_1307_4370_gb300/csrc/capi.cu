// C ABI of the library (include/purify.h): context set-up, the operator
// calls, the conjugate-gradient solve and the SDMM driver of Algorithm 1.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <new>
#include <thread>
#include <vector>

#include <cudaTypedefs.h>

#include "common.cuh"

using namespace purify;

namespace purify {

// The last CUDA error a library call of this thread turned into
// PURIFY_E_CUDA (reported by purify_last_error).
thread_local cudaError_t t_last_cuda_error = cudaSuccess;

int check_cuda(cudaError_t e) {
  if (e == cudaSuccess) return PURIFY_OK;
  t_last_cuda_error = e;
  return PURIFY_E_CUDA;
}

std::atomic<unsigned long long> g_launches{0};

}  // namespace purify

namespace {

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

#define TRY(expr)                  \
  do {                             \
    int _st = (expr);              \
    if (_st != PURIFY_OK) return _st; \
  } while (0)

#define TRY_CUDA(expr) TRY(check_cuda(expr))

// Device (or managed) memory that the current device may dereference: device
// memory must belong to the current device (every call makes the context's
// device current first), so a buffer of another GPU is rejected instead of
// being read through peer access or faulting.
bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  if (a.type != cudaMemoryTypeDevice) return false;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.device == cur;
}

template <class T>
int dev_alloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc((void**)p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return PURIFY_E_ALLOC;
  }
  return PURIFY_OK;
}

// ---------------------------------------------------------------------------
// Kaiser-Bessel: beta of Beatty et al. (2005) for oversampling 2, the kernel
// g(t) = I0(beta sqrt(1 - (2t/J)^2)) / I0(beta) and its closed-form transform.
// ---------------------------------------------------------------------------
double kb_beta(int J) {
  const double a = 2.0;
  return M_PI * std::sqrt((J / a) * (J / a) * (a - 0.5) * (a - 0.5) - 0.8);
}

double kb_g(double t, int J, double beta, double i0b) {
  const double s = 2.0 * t / J;
  if (std::fabs(s) > 1.0) return 0.0;
  return std::cyl_bessel_i(0.0, beta * std::sqrt(std::max(0.0, 1.0 - s * s))) / i0b;
}

double kb_ghat(double f, int J, double beta, double i0b) {
  const double a = std::sqrt(beta * beta - (M_PI * J * f) * (M_PI * J * f));
  return J * std::sinh(a) / (i0b * a);
}

// Solve V c = f (Gaussian elimination with partial pivoting, long double).
void solve_dense(std::vector<long double>& A, std::vector<long double>& b, int n) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs((double)A[i * n + k]) > std::fabs((double)A[piv * n + k])) piv = i;
    if (piv != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[piv * n + j]);
      std::swap(b[k], b[piv]);
    }
    for (int i = k + 1; i < n; ++i) {
      const long double f = A[i * n + k] / A[k * n + k];
      for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    long double s = b[k];
    for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * b[j];
    b[k] = s / A[k * n + k];
  }
}

// The paper's Gaussian kernel (§5): g(t) = exp(-b t^2) on |t| <= J/2 with
// b = pi (alpha - 1/2) / (alpha J / 2), alpha = 2 (the width of Greengard &
// Lee 2004 in grid cells); g_hat is the transform of the untruncated Gaussian.
double gauss_b(int J) { return M_PI * 1.5 / (2.0 * (J / 2.0)); }
double gauss_g(double t, int J) { return std::fabs(t) <= J / 2.0 ? std::exp(-gauss_b(J) * t * t) : 0.0; }
double gauss_ghat(double f, int J) {
  const double b = gauss_b(J);
  return std::sqrt(M_PI / b) * std::exp(-M_PI * M_PI * f * f / b);
}

// g and g_hat of the context's kernel.
double interp_g(double t, int J, int kernel, double beta, double i0b) {
  return kernel == PURIFY_KERNEL_GAUSS ? gauss_g(t, J) : kb_g(t, J, beta, i0b);
}
double interp_ghat(double f, int J, int kernel, double beta, double i0b) {
  return kernel == PURIFY_KERNEL_GAUSS ? gauss_ghat(f, J) : kb_ghat(f, J, beta, i0b);
}

// Fit each tap's weight, as a function of z = 2x - 1 on [-1, 1], by the
// degree-kKbDeg polynomial interpolating it at Chebyshev nodes (long double),
// and record the largest error of its float Horner evaluation.
KbPoly fit_kb(int J, int kernel) {
  const double beta = kb_beta(J);
  const double i0b = std::cyl_bessel_i(0.0, beta);
  KbPoly kb{};
  kb.J = J;
  const int np = kKbDeg + 1;
  float err = 0.f;
  for (int a = 0; a < J; ++a) {
    std::vector<long double> A(np * np), f(np);
    for (int i = 0; i < np; ++i) {
      const long double z = std::cos(M_PI * (i + 0.5) / np);
      const double x = 0.5 * ((double)z + 1.0);
      long double zp = 1.0L;
      for (int j = 0; j < np; ++j) {
        A[i * np + j] = zp;
        zp *= z;
      }
      f[i] = interp_g(x + J / 2 - 1 - a, J, kernel, beta, i0b);
    }
    solve_dense(A, f, np);
    for (int j = 0; j < np; ++j) kb.c[a][j] = (float)f[j];
    for (int t = 0; t <= 4000; ++t) {
      const double x = t / 4000.0 * (1.0 - 1e-12);
      const float z = std::fma(2.0f, (float)x, -1.0f);
      float acc = kb.c[a][kKbDeg];
      for (int k = kKbDeg - 1; k >= 0; --k) acc = std::fma(acc, z, kb.c[a][k]);
      err = std::max(err, (float)std::fabs(acc - interp_g(x + J / 2 - 1 - a, J, kernel, beta, i0b)));
    }
  }
  kb.max_err = err;
  return kb;
}

FftPlan make_plan(int L) {
  FftPlan p{};
  p.L = L;
  int rest = L;
  if (rest % 3 == 0) {
    p.radix[p.nst++] = 3;
    rest /= 3;
    while (rest % 4 == 0) { p.radix[p.nst++] = 4; rest /= 4; }
    if (rest % 2 == 0) { p.radix[p.nst++] = 2; rest /= 2; }
  } else {
    while (rest % 8 == 0) { p.radix[p.nst++] = 8; rest /= 8; }
    if (rest % 4 == 0) { p.radix[p.nst++] = 4; rest /= 4; }
    if (rest % 2 == 0) { p.radix[p.nst++] = 2; rest /= 2; }
  }
  if (rest != 1) p.nst = -1;
  else finish_plan(p);
  return p;
}

bool good_side(int L) {
  int r = L;
  int threes = 0;
  while (r % 3 == 0) { r /= 3; ++threes; }
  while (r % 2 == 0) r /= 2;
  return r == 1 && threes <= 1;
}

// First footprint cell of every visibility (same arithmetic as the kernels).
__global__ void k_footprint(const float2* __restrict__ uv, int64_t M, KappaScale ks, int J, int L,
                            int2* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
    int kr, kc;
    float fr, fc;
    split_kappa(uv[i].x, ks, kr, fr);
    split_kappa(uv[i].y, ks, kc, fc);
    out[i] = make_int2(wrap(kr - (J / 2 - 1), L), wrap(kc - (J / 2 - 1), L));
  }
}

// Per tile-list entry: the sorted index, the start-cell key and the kappa
// fractions (same arithmetic as the kernels), so the gridding needs no
// frequency gather and no integer wrap per call.
__global__ void k_list_setup(const int2* __restrict__ lk, const float2* __restrict__ uv, KappaScale ks, int64_t n,
                             int4* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int2 v = lk[e];
    const float2 u = uv[v.x];
    int kr, kc;
    float fr, fc;
    split_kappa(u.x, ks, kr, fr);
    split_kappa(u.y, ks, kc, fc);
    out[e] = make_int4(v.x, v.y, __float_as_int(fr), __float_as_int(fc));
  }
}

// Distributed form: the block of each sorted visibility (offsets in caller
// order, R + 1 entries) and the sorted position of each caller index.
__global__ void k_block_of(const int* __restrict__ perm, int64_t M, const int64_t* __restrict__ offsets, int R,
                           int* __restrict__ block_of, int* __restrict__ pos) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = perm[j];
    int lo = 0, hi = R;  // last b with offsets[b] <= m
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (offsets[mid] <= m) lo = mid;
      else hi = mid - 1;
    }
    block_of[j] = lo;
    pos[m] = (int)j;
  }
}

__global__ void k_fill_f32(int64_t n, float* p, float v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

__global__ void k_sqrt_to(const double* src, double* dst) { *dst = sqrt(*src); }

unsigned nblk(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 2048)); }

// TMA map of the forward grid whose box is one Gram-pass tile halo: float32
// view, inner dimension 2 L floats, rows L; box of 2 grid_halo_ws(T, J)
// floats by grid_halo_w(T, J) rows.  Encoded through the runtime's driver
// entry point (no link against the driver library).  When the driver cannot
// encode it, the Gram pass stages every halo with loads.
void encode_halo_map(purify_ctx* c) {
  c->halo_map_ok = 0;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return;
  }
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  const cuuint64_t dims[2] = {(cuuint64_t)2 * c->L, (cuuint64_t)c->L};
  const cuuint64_t strides[1] = {(cuuint64_t)c->L * sizeof(float2)};
  const cuuint32_t box[2] = {(cuuint32_t)(2 * grid_halo_ws(c->tileT, c->J)), (cuuint32_t)grid_halo_w(c->tileT, c->J)};
  const cuuint32_t estr[2] = {1, 1};
  if (box[0] > 256 || box[1] > 256) return;
  const CUresult r = encode(&c->halo_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->d_grid, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  c->halo_map_ok = (r == CUDA_SUCCESS) ? 1 : 0;
}

void free_ctx(purify_ctx* c) {
  if (!c) return;
  void* ptrs[] = {c->d_dense_tiles, c->d_H, c->d_gram_chunks, c->d_diff, c->d_twp[0], c->d_twp[1], c->d_deapod, c->d_beam, c->d_tv, c->d_tw, c->d_uv, c->d_perm, c->d_list, c->d_chunks, c->d_chunk_tab, c->d_items, c->d_item_row, c->d_dchunks, c->d_tile_slot0,
                  c->d_tile_nchunk, c->d_tile_cnt, c->d_slots,
                  c->d_grid, c->d_grid2, c->d_half, c->d_vis, c->d_vis2, c->d_ll[0], c->d_ll[1], c->d_img[0],
                  c->d_img[1], c->d_img[2], c->d_img[3], c->d_partials, c->d_sc};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->h_sc) cudaFreeHost(c->h_sc);
  for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
  delete c;
}

// Tiles whose gridding lists hold more than this many entries per cell keep
// G^T G as a stored stencil instead of gathering (measured on this GPU: the
// stencil streams (2J - 1)^2 floats per cell from memory, the gather issues
// ~1500 instructions per entry, and the two overlap in one launch).
#ifndef PURIFY_DENSE_ENTRIES_PER_CELL
#define PURIFY_DENSE_ENTRIES_PER_CELL 2.0
#endif
constexpr double kDenseEntriesPerCell = PURIFY_DENSE_ENTRIES_PER_CELL;
// ... and one per cell, stored by half, when those stencils fit a quarter of L2
#ifndef PURIFY_DENSE_ENTRIES_PER_CELL_L2
#define PURIFY_DENSE_ENTRIES_PER_CELL_L2 1.0
#endif
constexpr double kDenseEntriesPerCellL2 = PURIFY_DENSE_ENTRIES_PER_CELL_L2;
constexpr size_t kDenseL2Bytes = (size_t)32 << 20;

// G^T G restricted to the cells of the dense tiles (§5: G^H G, precomputed
// and stored, to speed up the CG solve): for cell k of tile t and offset d in
// [-(J-1), J-1]^2, H[t][d][k] = sum over the tile's list entries m of
// w_m(k) w_m(k + d), w_m the J x J interpolation weights of visibility m
// (exact kernel values in double, at the fractions the device uses).  Every
// visibility whose footprint covers a cell of the tile is on the tile's list,
// so (G^T G X)(k) = sum_d H[t][d][k] X(k + d) exactly.  Built in double on
// the host, one tile per thread of a small pool, and stored as float.
int build_dense_gram(const purify_ctx* c, const purify::GatherPlan& plan, const std::vector<int4>& entries,
                      const std::vector<int>& dense, std::vector<float>& H) {
  const int T = c->tileT, J = c->J, W = T + J - 1, ND = (2 * J - 1) * (2 * J - 1), TT = T * T;
  const double beta = kb_beta(J), i0b = std::cyl_bessel_i(0.0, beta);
  H.assign((size_t)dense.size() * ND * TT, 0.0f);
  std::atomic<size_t> next{0};
  std::atomic<bool> failed{false};
  auto work = [&]() {
    try {
      std::vector<double> acc((size_t)ND * TT);
      for (size_t q = next.fetch_add(1); q < dense.size(); q = next.fetch_add(1)) {
        const int t = dense[q];
        std::fill(acc.begin(), acc.end(), 0.0);
        for (int e = plan.list_off[t]; e < plan.list_off[t + 1]; ++e) {
          const int4 le = entries[e];
          const int kr = le.y / W, kc = le.y - kr * W;  // footprint start + (J - 1), relative to the tile
          float frf, fcf;
          std::memcpy(&frf, &le.z, 4);
          std::memcpy(&fcf, &le.w, 4);
          double wr[kMaxJ], wc[kMaxJ];
          for (int a = 0; a < J; ++a) {
            wr[a] = interp_g((double)frf + J / 2 - 1 - a, J, c->kernel, beta, i0b);
            wc[a] = interp_g((double)fcf + J / 2 - 1 - a, J, c->kernel, beta, i0b);
          }
          for (int a = 0; a < J; ++a) {
            const int r = kr - (J - 1) + a;
            if (r < 0 || r >= T) continue;
            for (int b = 0; b < J; ++b) {
              const int cc = kc - (J - 1) + b;
              if (cc < 0 || cc >= T) continue;
              const double wk = wr[a] * wc[b];
              double* hk = acc.data() + r * T + cc;
              for (int a2 = 0; a2 < J; ++a2) {
                const int drow = (a2 - a + J - 1) * (2 * J - 1) - b + J - 1;
                for (int b2 = 0; b2 < J; ++b2) hk[(size_t)(drow + b2) * TT] += wk * wr[a2] * wc[b2];
              }
            }
          }
        }
        float* out = H.data() + q * (size_t)ND * TT;
        for (size_t i = 0; i < acc.size(); ++i) out[i] = (float)acc[i];
      }
    } catch (...) {  // no exception leaves a worker thread (nor the C ABI)
      failed = true;
    }
  };
  const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  try {
    for (unsigned i = 1; i < hw; ++i) pool.emplace_back(work);
  } catch (...) {
    // fewer threads: the queue of tiles is shared, the started ones and this one finish it
  }
  work();
  for (auto& th : pool) th.join();
  return failed ? PURIFY_E_ALLOC : PURIFY_OK;
}

// The same operator stored by half (for small problems, whose stencils stay
// in L2): G^T G is symmetric, (G^T G)[k][k + d] = (G^T G)[k + d][k], so only
// the offsets d >= 0 in lexicographic order are kept, NH = J + (J - 1)(2J - 1)
// of the (2J - 1)^2:
//   H[t][s(d)][e] = sum over visibilities m of w_m(e) w_m(e + d)
// for the cells e of the tile extended by J - 1 rows above and J - 1 columns
// on each side (the cells k - d of the tile's cells k), and
//   (G^T G X)(k) = sum_{d >= 0} H[s(d)][k] X(k + d) + sum_{d > 0} H[s(d)][k - d] X(k - d).
// Every visibility whose footprint covers a tile cell is on the tile's list,
// so every value that equation reads is complete.  Slice order: s = dc for
// dr = 0, dc = 0 .. J - 1; then s = J + (dr - 1)(2J - 1) + dc + J - 1 for
// dr = 1 .. J - 1, dc = -(J - 1) .. J - 1.
int build_dense_gram_half(const purify_ctx* c, const purify::GatherPlan& plan, const std::vector<int4>& entries,
                           const std::vector<int>& dense, std::vector<float>& H) {
  const int T = c->tileT, J = c->J, W = T + J - 1, NDW = 2 * J - 1;
  const int NH = dense_gram_slices(J), EW = T + 2 * (J - 1), EH = T + J - 1, ES = EW * EH;
  const double beta = kb_beta(J), i0b = std::cyl_bessel_i(0.0, beta);
  H.assign((size_t)dense.size() * NH * ES, 0.0f);
  std::atomic<size_t> next{0};
  std::atomic<bool> failed{false};
  auto work = [&]() {
    try {
      std::vector<double> acc((size_t)NH * ES);
      for (size_t q = next.fetch_add(1); q < dense.size(); q = next.fetch_add(1)) {
        const int t = dense[q];
        std::fill(acc.begin(), acc.end(), 0.0);
        for (int e = plan.list_off[t]; e < plan.list_off[t + 1]; ++e) {
          const int4 le = entries[e];
          const int kr = le.y / W, kc = le.y - kr * W;  // footprint start + (J - 1), relative to the tile
          float frf, fcf;
          std::memcpy(&frf, &le.z, 4);
          std::memcpy(&fcf, &le.w, 4);
          double wr[kMaxJ], wc[kMaxJ];
          for (int a = 0; a < J; ++a) {
            wr[a] = interp_g((double)frf + J / 2 - 1 - a, J, c->kernel, beta, i0b);
            wc[a] = interp_g((double)fcf + J / 2 - 1 - a, J, c->kernel, beta, i0b);
          }
          // every ordered pair of footprint cells (a, b) -> (a2, b2) with a
          // lexicographically non-negative offset, accumulated at the first cell
          for (int a = 0; a < J; ++a) {
            const int er = kr + a;  // extended-region row of the first cell: tile row + J - 1
            if (er >= EH) continue;
            for (int b = 0; b < J; ++b) {
              const int ec = kc + b;  // extended-region column: tile column + J - 1
              if (ec >= EW) continue;
              const double wk = wr[a] * wc[b];
              double* he = acc.data() + (size_t)er * EW + ec;
              for (int a2 = a; a2 < J; ++a2) {
                const int dr = a2 - a;
                for (int b2 = (dr == 0 ? b : 0); b2 < J; ++b2) {
                  const int dc = b2 - b;
                  const int sl = dr == 0 ? dc : J + (dr - 1) * NDW + dc + J - 1;
                  he[(size_t)sl * ES] += wk * wr[a2] * wc[b2];
                }
              }
            }
          }
        }
        float* out = H.data() + q * (size_t)NH * ES;
        for (size_t i = 0; i < acc.size(); ++i) out[i] = (float)acc[i];
      }
    } catch (...) {  // no exception leaves a worker thread (nor the C ABI)
      failed = true;
    }
  };
  const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  try {
    for (unsigned i = 1; i < hw; ++i) pool.emplace_back(work);
  } catch (...) {
    // fewer threads: the queue of tiles is shared, the started ones and this one finish it
  }
  work();
  for (auto& th : pool) th.join();
  return failed ? PURIFY_E_ALLOC : PURIFY_OK;
}

// Visibility table: sort by the grid tile of the first footprint cell and
// list, per tile, every visibility whose J x J footprint meets it.
int setup_visibilities(purify_ctx* c, const float* uv_in, cudaStream_t s) {
  const int64_t M = c->M;
  float2* d_uv_user = nullptr;
  int2* d_k0 = nullptr;
  int2* d_lk = nullptr;
  int st = PURIFY_OK;
  TRY(dev_alloc(&d_uv_user, M));
  if ((st = dev_alloc(&d_k0, M)) != PURIFY_OK) { cudaFree(d_uv_user); return st; }
  cudaMemcpyAsync(d_uv_user, uv_in, M * sizeof(float2), cudaMemcpyDefault, s);
  PURIFY_LAUNCH(c, "footprint", s, (k_footprint<<<nblk(M), 256, 0, s>>>(d_uv_user, M, c->ks, c->J, c->L, d_k0)));
  std::vector<int2> k0(M);
  cudaMemcpyAsync(k0.data(), d_k0, M * sizeof(int2), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaFree(d_uv_user);
    cudaFree(d_k0);
    return PURIFY_E_CUDA;
  }
  const int T = c->tileT, NT = purify::kGridThreads;
  // sort, tile lists, work units and the gather walk (host; gather_plan.cpp)
  purify::GatherPlanParams prm{};
  prm.M = M;
  prm.L = c->L;
  prm.J = c->J;
  prm.T = T;
  prm.fixed_bytes = purify::grid_fixed_bytes(T, c->J);
  prm.entry_bytes = purify::grid_entry_bytes(c->J);
  prm.smem_budget = purify::kGridSmemBudget;
  prm.tab_stride = purify::grid_tab_stride(T);
  prm.max_partials = kMaxPartials;
  purify::GatherPlan plan;
  const int prc = purify::build_gather_plan(reinterpret_cast<const int*>(k0.data()), prm, plan);
  if (prc != 0) {
    cudaFree(d_uv_user);
    cudaFree(d_k0);
    return prc == -1 ? PURIFY_E_INVALID_ARG : PURIFY_E_SIZE;
  }
  c->nlist = (int64_t)plan.list.size();
  c->chunk_max = plan.chunk_max;
  c->nchunks = (int)plan.chunks.size();
  c->nslots = plan.nslots;
  c->chunk_tab_stride = prm.tab_stride;
  c->nitem_rows = plan.nitem_rows;
  c->ndchunks = (int)plan.dchunks.size();
  const int nslots = plan.nslots;
  if ((st = dev_alloc(&c->d_uv, M)) == PURIFY_OK && (st = dev_alloc(&c->d_perm, M)) == PURIFY_OK &&
      (st = dev_alloc(&c->d_list, c->nlist)) == PURIFY_OK && (st = dev_alloc(&d_lk, c->nlist)) == PURIFY_OK &&
      (st = dev_alloc(&c->d_chunks, c->nchunks)) == PURIFY_OK &&
      (st = dev_alloc(&c->d_chunk_tab, (size_t)c->nchunks * c->chunk_tab_stride)) == PURIFY_OK &&
      (st = dev_alloc(&c->d_items, (size_t)std::max<int64_t>(1, c->nitem_rows) * NT)) == PURIFY_OK &&
      (st = dev_alloc(&c->d_item_row, c->nchunks)) == PURIFY_OK &&
      (st = dev_alloc(&c->d_dchunks, std::max(1, c->ndchunks))) == PURIFY_OK &&
      (st = dev_alloc(&c->d_tile_slot0, c->ntiles)) == PURIFY_OK &&
      (st = dev_alloc(&c->d_tile_nchunk, c->ntiles)) == PURIFY_OK &&
      (st = dev_alloc(&c->d_tile_cnt, c->ntiles)) == PURIFY_OK &&
      (st = dev_alloc(&c->d_slots, (size_t)std::max(1, nslots) * T * T)) == PURIFY_OK) {
    cudaMemcpyAsync(c->d_perm, plan.perm.data(), M * sizeof(int), cudaMemcpyHostToDevice, s);
    {
      std::vector<int2> lk(c->nlist);
      for (int64_t e = 0; e < c->nlist; ++e) lk[e] = make_int2(plan.list[e], plan.lkey[e]);
      cudaMemcpyAsync(d_lk, lk.data(), c->nlist * sizeof(int2), cudaMemcpyHostToDevice, s);
      launch_gather_perm(M, d_uv_user, c->d_perm, c->d_uv, s);
      PURIFY_LAUNCH(c, "list_setup", s,
                    (k_list_setup<<<nblk(c->nlist), 256, 0, s>>>(d_lk, c->d_uv, c->ks, c->nlist, c->d_list)));
      if (cudaStreamSynchronize(s) != cudaSuccess) st = PURIFY_E_CUDA;
    }
    static_assert(sizeof(purify::PlanI4) == sizeof(int4), "plan work units have the layout of int4");
    cudaMemcpyAsync(c->d_chunks, plan.chunks.data(), c->nchunks * sizeof(int4), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(c->d_chunk_tab, plan.tab.data(), plan.tab.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, s);
    if (!plan.items.empty())
      cudaMemcpyAsync(c->d_items, plan.items.data(), plan.items.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(c->d_item_row, plan.item_row.data(), c->nchunks * sizeof(int), cudaMemcpyHostToDevice, s);
    if (c->ndchunks > 0)
      cudaMemcpyAsync(c->d_dchunks, plan.dchunks.data(), c->ndchunks * sizeof(int4), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(c->d_tile_slot0, plan.slot0.data(), c->ntiles * sizeof(int), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(c->d_tile_nchunk, plan.nchunk.data(), c->ntiles * sizeof(int), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(c->d_tile_cnt, 0, c->ntiles * sizeof(unsigned), s);
    if (cudaStreamSynchronize(s) != cudaSuccess) st = PURIFY_E_CUDA;
  }
  // dense tiles of the Gram pass and their stored G^T G (see build_dense_gram)
  if (st == PURIFY_OK) {
    // layout: the half stencil, with one entry per cell as the threshold,
    // when those stencils fit a quarter of L2 (they stay resident across the
    // CG steps; 256^2 workload: Gram 15.4 -> 12.8 us); the full stencil, two
    // entries per cell, otherwise (HBM-streamed: 1024^2 half 136.8 us, full
    // 130.9 us)
    const size_t half_bytes = (size_t)dense_gram_slices(c->J) * (T + c->J - 1) * (T + 2 * (c->J - 1)) * 4;
    int n_low = 0;
    for (int t = 0; t < c->ntiles; ++t)
      if ((double)(plan.list_off[t + 1] - plan.list_off[t]) > kDenseEntriesPerCellL2 * T * T) ++n_low;
    c->dense_half = (size_t)n_low * half_bytes <= kDenseL2Bytes ? 1 : 0;
    const double per_cell = c->dense_half ? kDenseEntriesPerCellL2 : kDenseEntriesPerCell;
    std::vector<int> dense;
    std::vector<char> is_dense(c->ntiles, 0);
    for (int t = 0; t < c->ntiles; ++t)
      if ((double)(plan.list_off[t + 1] - plan.list_off[t]) > per_cell * T * T) {
        dense.push_back(t);
        is_dense[t] = 1;
      }
    std::vector<int> gram_chunks;
    for (int q = 0; q < c->nchunks; ++q)
      if (!is_dense[plan.chunks[q].x]) gram_chunks.push_back(q);
    c->n_dense = (int)dense.size();
    c->n_gram_chunks = (int)gram_chunks.size();
    std::vector<float> H;
    if (c->n_dense > 0) {
      std::vector<int4> entries(c->nlist);
      if (cudaMemcpy(entries.data(), c->d_list, c->nlist * sizeof(int4), cudaMemcpyDeviceToHost) != cudaSuccess)
        st = PURIFY_E_CUDA;
      if (st == PURIFY_OK)
        st = c->dense_half ? build_dense_gram_half(c, plan, entries, dense, H)
                           : build_dense_gram(c, plan, entries, dense, H);
    }
    if (st == PURIFY_OK && ((st = dev_alloc(&c->d_dense_tiles, std::max(1, c->n_dense))) ||
                            (st = dev_alloc(&c->d_gram_chunks, std::max(1, c->n_gram_chunks))) ||
                            (st = dev_alloc(&c->d_H, std::max<size_t>(1, H.size())))))
      ;
    if (st == PURIFY_OK) {
      if ((c->n_dense > 0 &&
           (cudaMemcpy(c->d_dense_tiles, dense.data(), dense.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(c->d_H, H.data(), H.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)) ||
          (c->n_gram_chunks > 0 && cudaMemcpy(c->d_gram_chunks, gram_chunks.data(), gram_chunks.size() * sizeof(int),
                                              cudaMemcpyHostToDevice) != cudaSuccess))
        st = PURIFY_E_CUDA;
    }
  }
  cudaFree(d_lk);
  cudaFree(d_uv_user);
  cudaFree(d_k0);
  return st;
}

// One step of single-reduction CG on Q = Phi^H Phi + 2I: apply the pending
// update of the previous step (not before the first step), w = Q r, and the
// step sizes from <r, r> and <w, r> (Chronopoulos & Gear 1989; in exact
// arithmetic the iterates are those of the standard CG of the x-update).
int cg_step(purify_ctx* c, float2* x, float2* r, float2* p, float2* sv, float2* w, int i, cudaStream_t s) {
  RowInArgs ia{};
  ia.in = r;
  ia.x = x;
  ia.r = r;
  ia.p = p;
  ia.s = sv;
  ia.w = w;
  TRY(phi_forward_grid(c, i == 0 ? kRowInPlain : kRowInCgUpd, ia, s, i - 1));  // applies step i - 1's update
  TRY(gram_grid(c, s));  // G^T G in one pass (the M samples are not stored)
  RowOutArgs ra{};
  ra.out = w;
  ra.p = r;
  TRY(phi_adjoint_image(c, kRowOutCgQ, ra, s, c->d_grid2));
  return cg_consumer_blocks(c) > 0 ? PURIFY_OK : launch_cg_scalars(c, i, s);
}

int64_t ctx_N(const purify_ctx* c) { return (int64_t)c->n * c->n; }
int64_t ctx_D(const purify_ctx* c) { return (int64_t)c->q * c->n * c->n; }

int load_data(purify_ctx* c, purify_sdmm_state* st, const float* y, cudaStream_t s) {
  const int64_t M = c->M;
  // caller order -> sorted order through the context's spare visibility buffer
  TRY_CUDA(cudaMemcpyAsync(c->d_vis2, y, M * sizeof(float2), cudaMemcpyDefault, s));
  TRY(launch_gather_perm(M, c->d_vis2, c->d_perm, st->y, s));
  st->y_bf16 = 0;
  return PURIFY_OK;
}

}  // namespace

namespace purify {

// Algorithm 1 steps 5-9 for one iteration, enqueued on s.
int enqueue_sdmm_step(purify_ctx* c, purify_sdmm_state* st, cudaStream_t s) {
  const unsigned long long l0 = g_launches.load(std::memory_order_relaxed);
  // step 5: x_hat = Q^{-1} sum_i x_i by warm-started CG (r holds r0 = b - Q x_hat(t-1))
  const int k = st->params.cg_iters;
  for (int i = 0; i < k; ++i) TRY(cg_step(c, st->xhat, st->r, st->p, st->sv, st->qp, i, s));
  // i = 2, first half: s2 = Phi x_hat (after the last CG update) and the l2 norms (FP64)
  RowInArgs ia{};
  ia.in = st->xhat;
  ia.x = st->xhat;
  ia.r = st->r;
  ia.p = st->p;
  ia.s = st->sv;
  ia.w = st->qp;
  TRY(phi_forward_grid(c, k > 0 ? kRowInCgFinish : kRowInPlain, ia, s, k - 1));
  // steps 7-9: the branches are independent until the next residual (§4.5:
  // the proximity operators can run in parallel).  i = 1 (the prior) on the
  // side stream, i = 2 (the data) on s; i = 3 is fused into the final pass.
  TRY_CUDA(cudaEventRecord(st->ev_fork, s));
  TRY_CUDA(cudaStreamWaitEvent(st->side, st->ev_fork, 0));
  if (st->prior == PURIFY_PRIOR_TV) {
    // TV prior (L1 = I): r1 = prox of gamma ||W grad .||_1 at x_hat + z1, z1, x1 = r1 - z1
    TRY(tv_sdmm_branch(c, st, st->side));
  } else {
    // Psi^H x_hat with the soft threshold and dual update fused (u1 = r1 - z1), then x1 = Psi u1
    SaraProxArgs pa{st->z1, st->u1, st->w};
    int f1_parts = 0;
    TRY(sara_analysis(c, st->xhat, nullptr, kSaraProx, pa, st->side, &f1_parts));
    TRY(sara_synthesis(c, st->u1, st->x1, st->side, f1_parts));
  }
  TRY_CUDA(cudaEventRecord(st->ev_join, st->side));
  // i = 2: s2 = Phi x_hat and the l2 norms (FP64), the ball projection, z2 and v = u2 - s2
  DegridArgs da{};
  da.out = st->s2;
  da.z2 = st->z2;
  da.y = st->y_bf16 ? nullptr : st->y;
  da.yb = st->yb;
  da.yscale = st->yscale;
  TRY(degrid(c, kDegridSdmm, da, s));
  if (st->nblocks > 0) TRY(launch_block_norms(st, s));  // distributed form: one ball per block
  TRY(launch_sdmm_l2_update(st, s));
  // x2 - Phi^H Phi x_hat = Phi^H v; i = 3 (positivity) and the next CG residual, after x1
  TRY(grid_adjoint(c, kGridSorted, st->v, s));
  RowOutArgs ra{};
  ra.out = st->r;
  ra.p = st->xhat;
  ra.x1 = st->x1;
  ra.z3 = st->z3;
  TRY(phi_adjoint_image(c, kRowOutSdmm, ra, s, nullptr, st->ev_join));
  st->launches_per_step = (int)(g_launches.load(std::memory_order_relaxed) - l0);
  return PURIFY_OK;
}

GraphKey step_graph_key(const purify_sdmm_state* st) {
  GraphKey k;
  k.cg_iters = st->params.cg_iters;
  k.y_bf16 = st->y_bf16;
  k.shape = st->shape_version;
  k.beam = st->ctx->beam_version;
  return k;
}

}  // namespace purify

namespace {

int drop_graph(purify_sdmm_state* st) {
  if (st->step_exec) {
    cudaGraphExecDestroy(st->step_exec);
    st->step_exec = nullptr;
  }
  return PURIFY_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* purify_status_string(int status) {
  switch (status) {
    case PURIFY_OK: return "ok";
    case PURIFY_E_INVALID_ARG: return "invalid argument";
    case PURIFY_E_SIZE: return "size out of the supported range";
    case PURIFY_E_NOT_DEVICE_PTR: return "argument is not device memory";
    case PURIFY_E_ALLOC: return "allocation failed";
    case PURIFY_E_CUDA: return "CUDA runtime error";
    case PURIFY_E_TIMEOUT: return "bounded device wait gave up";
    case PURIFY_E_UNSUPPORTED: return "unsupported grid size";
    default: return "unknown status";
  }
}

const char* purify_last_error(void) {
  return t_last_cuda_error == cudaSuccess ? "no CUDA error" : cudaGetErrorString(t_last_cuda_error);
}

static int purify_create_impl(purify_ctx** out, const purify_desc* d, const float* uv, purify_stream_t stream) {
  if (!out) return PURIFY_E_INVALID_ARG;
  *out = nullptr;
  if (!d || !uv) return PURIFY_E_INVALID_ARG;
  if (d->oversample != 2) return PURIFY_E_SIZE;
  if (d->J != 2 && d->J != 4 && d->J != 6 && d->J != 8) return PURIFY_E_SIZE;
  if (d->levels < 1 || d->levels > 6) return PURIFY_E_SIZE;
  if (d->n < 8 || d->n > 2048 || d->n % (1 << d->levels) != 0 || d->n % 2 != 0) return PURIFY_E_SIZE;
  if (d->M < 1 || d->M > 2147483647LL) return PURIFY_E_SIZE;
  if (d->bases_mask == 0 || (d->bases_mask & ~0x1FFu)) return PURIFY_E_INVALID_ARG;
  if (d->kernel != PURIFY_KERNEL_KB && d->kernel != PURIFY_KERNEL_GAUSS) return PURIFY_E_INVALID_ARG;
  if (!good_side(2 * d->n)) return PURIFY_E_UNSUPPORTED;
  if (d->tile != 0 && ((d->tile != 8 && d->tile != 16 && d->tile != 32 && d->tile != 64) || d->tile < d->J ||
                       (2 * d->n) % d->tile != 0))
    return PURIFY_E_SIZE;
  cudaStream_t s = (cudaStream_t)stream;
  purify_ctx* c = new (std::nothrow) purify_ctx();
  if (!c) return PURIFY_E_ALLOC;
  if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return PURIFY_E_CUDA; }
  if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || c->sms < 1)
    c->sms = 1;
  c->n = d->n;
  c->L = 2 * d->n;
  c->J = d->J;
  c->kernel = d->kernel;
  c->levels = d->levels;
  c->M = d->M;
  c->mask = d->bases_mask;
  c->q = 0;
  for (int b = 0; b < 9; ++b)
    if (c->mask & (1u << b)) c->bases[c->q++] = b;
  c->kb = fit_kb(c->J, c->kernel);
  const double sc = (double)c->L / (2.0 * M_PI);
  c->ks.hi = (float)sc;
  c->ks.lo = (float)(sc - (double)c->ks.hi);
  c->plan = make_plan(c->L);
  if (c->plan.nst < 0) { delete c; return PURIFY_E_UNSUPPORTED; }
  c->fft_engine = (c->L >= 256 && c->L <= 4096 && (c->L & (c->L - 1)) == 0) ? 1 : 0;
  make_daubechies(c->wf);
  if (d->tile != 0) {
    c->tileT = d->tile;
  } else {
    c->tileT = c->L >= 512 ? 32 : (c->L >= 64 ? 16 : 8);
    while (c->tileT < c->J || c->L % c->tileT) c->tileT *= 2;
  }
  c->tiles_1d = c->L / c->tileT;
  c->ntiles = c->tiles_1d * c->tiles_1d;
  const int64_t N = ctx_N(c), n2 = (int64_t)(c->n / 2) * (c->n / 2);
  int st = PURIFY_OK;
  auto fail = [&](int code) { free_ctx(c); return code; };
  if ((st = dev_alloc(&c->d_deapod, c->n)) || (st = dev_alloc(&c->d_tw, c->L)) ||
      (st = dev_alloc(&c->d_grid, (size_t)c->L * c->L)) || (st = dev_alloc(&c->d_grid2, (size_t)c->L * c->L)) || (st = dev_alloc(&c->d_half, (size_t)c->n * c->L)) ||
      (st = dev_alloc(&c->d_vis, c->M)) || (st = dev_alloc(&c->d_vis2, c->M)) ||
      (st = dev_alloc(&c->d_ll[0], c->q * n2)) || (st = dev_alloc(&c->d_ll[1], c->q * n2)) ||
      (st = dev_alloc(&c->d_img[0], N)) || (st = dev_alloc(&c->d_img[1], N)) || (st = dev_alloc(&c->d_img[2], N)) ||
      (st = dev_alloc(&c->d_img[3], N)) ||
      (st = dev_alloc(&c->d_partials, (size_t)kNumCounters * 2 * kMaxPartials)) ||
      (st = dev_alloc(&c->d_sc, 1)))
    return fail(st);
  if (cudaMallocHost((void**)&c->h_sc, sizeof(DevScalars)) != cudaSuccess) { cudaGetLastError(); return fail(PURIFY_E_ALLOC); }
  // deapodisation 1 / g_hat((r - n/2) / 2n) and twiddles exp(-2 pi i m / L), in double
  {
    const double beta = kb_beta(c->J), i0b = std::cyl_bessel_i(0.0, beta);
    std::vector<float> dz(c->n);
    for (int r = 0; r < c->n; ++r) dz[r] = (float)(1.0 / interp_ghat((double)(r - c->n / 2) / c->L, c->J, c->kernel, beta, i0b));
    std::vector<float2> tw(c->L);
    for (int m = 0; m < c->L; ++m) {
      const double a = -2.0 * M_PI * (double)m / c->L;
      tw[m] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    if (cudaMemcpyAsync(c->d_deapod, dz.data(), c->n * sizeof(float), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(c->d_tw, tw.data(), c->L * sizeof(float2), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(c->d_sc, 0, sizeof(DevScalars), s) != cudaSuccess ||
        cudaMemsetAsync(c->d_ll[0], 0, c->q * n2 * sizeof(float2), s) != cudaSuccess ||
        cudaMemsetAsync(c->d_ll[1], 0, c->q * n2 * sizeof(float2), s) != cudaSuccess)
      return fail(PURIFY_E_CUDA);
    // dz and tw are pageable host vectors: finish the copies before they go out of scope
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(PURIFY_E_CUDA);
  }
  if ((st = fft_prepare(c)) != PURIFY_OK) return fail(st);
  encode_halo_map(c);
  try {
    st = setup_visibilities(c, uv, s);
  } catch (const std::bad_alloc&) {  // host vectors of the plan and the stencils
    st = PURIFY_E_ALLOC;
  }
  if (st != PURIFY_OK) return fail(st);
  // shared memory above 48 KB needs an opt-in per kernel; sizes here stay below it
  *out = c;
  return PURIFY_OK;
}

int purify_create(purify_ctx** out, const purify_desc* d, const float* uv, purify_stream_t stream) {
  // host containers may throw; no exception crosses the C ABI
  try {
    return purify_create_impl(out, d, uv, stream);
  } catch (const std::bad_alloc&) {
    return PURIFY_E_ALLOC;
  }
}

void purify_destroy(purify_ctx* c) {
  if (!c) return;
  DeviceGuard g(c->device);
  cudaDeviceSynchronize();
  free_ctx(c);
}

int purify_set_beam(purify_ctx* c, const float* beam, purify_stream_t stream) {
  if (!c) return PURIFY_E_INVALID_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (!beam) {
    c->beam_on = false;  // the buffer stays until purify_destroy
  } else {
    if (!c->d_beam) TRY(dev_alloc(&c->d_beam, ctx_N(c)));
    TRY_CUDA(cudaMemcpyAsync(c->d_beam, beam, ctx_N(c) * sizeof(float), cudaMemcpyDefault, s));
    TRY_CUDA(cudaStreamSynchronize(s));
    c->beam_on = true;
  }
  c->beam_version++;
  return PURIFY_OK;
}

int purify_l2_bound(int64_t M, double sigma_n, double* eps) {
  if (!eps || M < 1 || !(sigma_n >= 0.0)) return PURIFY_E_INVALID_ARG;
  const double m = (double)M;
  *eps = std::sqrt((2.0 * m + 4.0 * std::sqrt(m)) * sigma_n * sigma_n / 2.0);
  return PURIFY_OK;
}

int purify_sizes(const purify_ctx* c, int64_t* N, int64_t* M, int32_t* q, int64_t* D) {
  if (!c) return PURIFY_E_INVALID_ARG;
  if (N) *N = ctx_N(c);
  if (M) *M = c->M;
  if (q) *q = c->q;
  if (D) *D = ctx_D(c);
  return PURIFY_OK;
}

int purify_phi(purify_ctx* c, const float* x, float* y, purify_stream_t stream) {
  if (!c || !x || !y) return PURIFY_E_INVALID_ARG;
  DeviceGuard g(c->device);
  if (!is_device_ptr(x) || !is_device_ptr(y)) return PURIFY_E_NOT_DEVICE_PTR;
  cudaStream_t s = (cudaStream_t)stream;
  RowInArgs ia{};
  ia.in = (const float2*)x;
  TRY(phi_forward_grid(c, kRowInPlain, ia, s));
  DegridArgs da{};
  da.out = (float2*)y;
  return degrid(c, kDegridPerm, da, s);
}

int purify_phi_adj(purify_ctx* c, const float* y, float* x, purify_stream_t stream) {
  if (!c || !x || !y) return PURIFY_E_INVALID_ARG;
  DeviceGuard g(c->device);
  if (!is_device_ptr(x) || !is_device_ptr(y)) return PURIFY_E_NOT_DEVICE_PTR;
  cudaStream_t s = (cudaStream_t)stream;
  TRY(grid_adjoint(c, kGridPerm, (const float2*)y, s));
  RowOutArgs ra{};
  ra.out = (float2*)x;
  return phi_adjoint_image(c, kRowOutPlain, ra, s);
}

int purify_sara_analysis(purify_ctx* c, const float* x, float* alpha, purify_stream_t stream) {
  if (!c || !x || !alpha) return PURIFY_E_INVALID_ARG;
  DeviceGuard g(c->device);
  if (!is_device_ptr(x) || !is_device_ptr(alpha)) return PURIFY_E_NOT_DEVICE_PTR;
  SaraProxArgs pa{};
  return sara_analysis(c, (const float2*)x, (float2*)alpha, kSaraPlain, pa, (cudaStream_t)stream);
}

int purify_sara_synthesis(purify_ctx* c, const float* alpha, float* x, purify_stream_t stream) {
  if (!c || !x || !alpha) return PURIFY_E_INVALID_ARG;
  DeviceGuard g(c->device);
  if (!is_device_ptr(x) || !is_device_ptr(alpha)) return PURIFY_E_NOT_DEVICE_PTR;
  return sara_synthesis(c, (const float2*)alpha, (float2*)x, (cudaStream_t)stream);
}

int purify_prox_l1_reweighted(purify_ctx* c, int64_t count, const float* in, const float* w, float gamma,
                              float* out, purify_stream_t stream) {
  if (!c || !in || !out || count < 0 || !(gamma >= 0.0f)) return PURIFY_E_INVALID_ARG;
  if (count == 0) return PURIFY_OK;
  DeviceGuard g(c->device);
  if (!is_device_ptr(in) || !is_device_ptr(out) || (w && !is_device_ptr(w))) return PURIFY_E_NOT_DEVICE_PTR;
  return launch_soft_threshold(count, (const float2*)in, w, nullptr, gamma, (float2*)out, (cudaStream_t)stream);
}

int purify_proj_l2ball(purify_ctx* c, int64_t count, const float* in, const float* y, double eps, float* out,
                       double* norm_out, purify_stream_t stream) {
  if (!c || !in || !y || !out || count < 0 || !(eps >= 0.0)) return PURIFY_E_INVALID_ARG;
  if (count == 0) return PURIFY_OK;
  DeviceGuard g(c->device);
  if (!is_device_ptr(in) || !is_device_ptr(out) || !is_device_ptr(y) || (norm_out && !is_device_ptr(norm_out)))
    return PURIFY_E_NOT_DEVICE_PTR;
  cudaStream_t s = (cudaStream_t)stream;
  TRY(launch_l2_norm_diff(c, count, (const float2*)in, (const float2*)y, s));
  TRY(launch_l2_project(count, (const float2*)in, (const float2*)y, eps, &c->d_sc->norm2, (float2*)out, s));
  if (norm_out) {
    PURIFY_LAUNCH(c, "sqrt", s, (k_sqrt_to<<<1, 1, 0, s>>>(&c->d_sc->norm2, norm_out)));
    TRY_CUDA(cudaGetLastError());
  }
  return PURIFY_OK;
}

int purify_proj_positive(purify_ctx* c, int64_t count, const float* in, float* out, purify_stream_t stream) {
  if (!c || !in || !out || count < 0) return PURIFY_E_INVALID_ARG;
  if (count == 0) return PURIFY_OK;
  DeviceGuard g(c->device);
  if (!is_device_ptr(in) || !is_device_ptr(out)) return PURIFY_E_NOT_DEVICE_PTR;
  return launch_positive(count, (const float2*)in, (float2*)out, (cudaStream_t)stream);
}

int purify_cg_solve(purify_ctx* c, const float* b, float* x, int32_t iters, double* resid_out,
                    purify_stream_t stream) {
  if (!c || !b || !x || iters < 0) return PURIFY_E_INVALID_ARG;
  DeviceGuard g(c->device);
  if (!is_device_ptr(b) || !is_device_ptr(x) || (resid_out && !is_device_ptr(resid_out)))
    return PURIFY_E_NOT_DEVICE_PTR;
  cudaStream_t s = (cudaStream_t)stream;
  float2* X = (float2*)x;
  float2 *r = c->d_img[0], *p = c->d_img[1], *sv = c->d_img[2], *w = c->d_img[3];
  // Q x0 (into w), then r = b - Q x0
  RowInArgs ia{};
  ia.in = X;
  TRY(phi_forward_grid(c, kRowInPlain, ia, s));
  DegridArgs da{};
  da.out = c->d_vis;
  TRY(degrid(c, kDegridSorted, da, s));
  TRY(grid_adjoint(c, kGridSorted, c->d_vis, s));
  RowOutArgs ra{};
  ra.out = w;
  ra.p = X;
  TRY(phi_adjoint_image(c, kRowOutCgQ, ra, s));
  TRY(launch_cg_residual_init(c, (const float2*)b, w, r, s));
  for (int k = 0; k < iters; ++k) TRY(cg_step(c, X, r, p, sv, w, k, s));
  if (iters > 0) TRY(launch_cg_apply(c, X, r, p, sv, w, iters - 1, s));
  if (resid_out) TRY_CUDA(cudaMemcpyAsync(resid_out, &c->d_sc->cg_res, sizeof(double), cudaMemcpyDeviceToDevice, s));
  return PURIFY_OK;
}

// ---------------------------------------------------------------------------
// SDMM
// ---------------------------------------------------------------------------
void purify_sdmm_default_params(purify_sdmm_params* p) {
  if (!p) return;
  p->max_iters = 300;
  p->cg_iters = 10;
  p->rounds = 1;
  p->check_every = 0;
  p->beta = 1e-3;
  p->xi = 1e-3;
  p->tau = 0.1;
  p->use_graph = 1;
}

void purify_sdmm_state_destroy(purify_sdmm_state* st) {
  if (!st) return;
  DeviceGuard g(st->ctx->device);
  cudaDeviceSynchronize();
  drop_graph(st);
  if (st->cap_stream) cudaStreamDestroy(st->cap_stream);
  if (st->side) cudaStreamDestroy(st->side);
  if (st->ev_fork) cudaEventDestroy(st->ev_fork);
  if (st->ev_join) cudaEventDestroy(st->ev_join);
  void* ptrs[] = {st->xhat, st->r, st->p, st->qp, st->sv, st->x1, st->z3, st->z1, st->u1,
                  st->w, st->y, st->yb, st->yscale, st->z2, st->s2, st->v,
                  st->d_block_of, st->d_pos, st->d_bchunks, st->d_beps, st->d_bscale};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete st;
}

int purify_sdmm_state_create(purify_ctx* c, purify_sdmm_state** out) {
  if (!c || !out) return PURIFY_E_INVALID_ARG;
  *out = nullptr;
  DeviceGuard g(c->device);
  purify_sdmm_state* st = new (std::nothrow) purify_sdmm_state();
  if (!st) return PURIFY_E_ALLOC;
  st->ctx = c;
  const int64_t N = ctx_N(c), D = ctx_D(c), M = c->M;
  int e;
  if ((e = dev_alloc(&st->xhat, N)) || (e = dev_alloc(&st->r, N)) || (e = dev_alloc(&st->p, N)) ||
      (e = dev_alloc(&st->qp, N)) || (e = dev_alloc(&st->sv, N)) || (e = dev_alloc(&st->x1, N)) ||
      (e = dev_alloc(&st->z3, N)) ||
      (e = dev_alloc(&st->z1, D)) || (e = dev_alloc(&st->u1, D)) || (e = dev_alloc(&st->w, D)) ||
      (e = dev_alloc(&st->y, M)) || (e = dev_alloc(&st->yb, 2 * M)) || (e = dev_alloc(&st->yscale, (M + 4095) / 4096)) ||
      (e = dev_alloc(&st->z2, M)) || (e = dev_alloc(&st->s2, M)) || (e = dev_alloc(&st->v, M))) {
    purify_sdmm_state_destroy(st);
    return e;
  }
  if (cudaStreamCreateWithFlags(&st->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&st->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&st->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    purify_sdmm_state_destroy(st);
    return PURIFY_E_CUDA;
  }
  purify_sdmm_default_params(&st->params);
  *out = st;
  return PURIFY_OK;
}

int purify_sdmm_set_data(purify_ctx* c, purify_sdmm_state* st, const float* y, purify_stream_t stream) {
  if (!c || !st || !y || st->ctx != c) return PURIFY_E_INVALID_ARG;
  DeviceGuard g(c->device);
  return load_data(c, st, y, (cudaStream_t)stream);
}

int purify_sdmm_set_data_bf16(purify_ctx* c, purify_sdmm_state* st, const float* y, purify_stream_t stream) {
  if (!c || !st || !y || st->ctx != c) return PURIFY_E_INVALID_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  TRY(load_data(c, st, y, s));
  TRY(launch_quantize_bf16(c->M, st->y, st->yb, st->yscale, s));
  st->y_bf16 = 1;
  return PURIFY_OK;
}

int purify_sdmm_init(purify_ctx* c, purify_sdmm_state* st, const float* y, double eps,
                     const purify_sdmm_params* params, purify_stream_t stream) {
  if (!c || !st || !y || st->ctx != c || !(eps > 0.0)) return PURIFY_E_INVALID_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (params) st->params = *params;
  if (st->params.cg_iters < 0 || st->params.max_iters < 0 || st->params.rounds < 1) return PURIFY_E_INVALID_ARG;
  const int64_t N = ctx_N(c), D = ctx_D(c), M = c->M;
  TRY(load_data(c, st, y, s));
  st->eps = eps;
  st->iters = 0;
  TRY_CUDA(cudaMemsetAsync(st->xhat, 0, N * sizeof(float2), s));
  TRY_CUDA(cudaMemsetAsync(st->r, 0, N * sizeof(float2), s));
  TRY_CUDA(cudaMemsetAsync(st->p, 0, N * sizeof(float2), s));
  TRY_CUDA(cudaMemsetAsync(st->qp, 0, N * sizeof(float2), s));
  TRY_CUDA(cudaMemsetAsync(st->sv, 0, N * sizeof(float2), s));
  TRY_CUDA(cudaMemsetAsync(st->x1, 0, N * sizeof(float2), s));
  TRY_CUDA(cudaMemsetAsync(st->z3, 0, N * sizeof(float2), s));
  TRY_CUDA(cudaMemsetAsync(st->z1, 0, D * sizeof(float2), s));
  TRY_CUDA(cudaMemsetAsync(st->u1, 0, D * sizeof(float2), s));
  TRY_CUDA(cudaMemsetAsync(st->z2, 0, M * sizeof(float2), s));
  TRY_CUDA(cudaMemsetAsync(st->s2, 0, M * sizeof(float2), s));
  TRY_CUDA(cudaMemsetAsync(st->v, 0, M * sizeof(float2), s));
  PURIFY_LAUNCH(c, "fill", s, (k_fill_f32<<<nblk(D), 256, 0, s>>>(D, st->w, 1.0f)));
  TRY_CUDA(cudaGetLastError());
  // scalars: everything zero but eps
  DevScalars z{};
  z.eps = eps;
  std::memcpy(c->h_sc, &z, sizeof(z));
  TRY_CUDA(cudaMemcpyAsync(c->d_sc, c->h_sc, sizeof(DevScalars), cudaMemcpyHostToDevice, s));
  // gamma = beta ||Psi^H Phi^H y||_inf (§4.4), via Phi^H y (sorted) into x1 and Psi^H into u1
  TRY(grid_adjoint(c, kGridSorted, st->y, s));
  RowOutArgs ra{};
  ra.out = st->x1;
  TRY(phi_adjoint_image(c, kRowOutPlain, ra, s));
  if (st->prior == PURIFY_PRIOR_TV) {
    // TV: gamma = beta max |grad Phi^H y|
    float2* g = nullptr;
    TRY(tv_gradmag(c, st->x1, &g, s));
    TRY(launch_max_abs(c, N, g, s));
  } else {
    SaraProxArgs pa{};
    TRY(sara_analysis(c, st->x1, st->u1, kSaraPlain, pa, s));
    TRY(launch_max_abs(c, D, st->u1, s));
  }
  TRY(launch_set_gamma(c, st->params.beta, s));
  TRY_CUDA(cudaMemsetAsync(st->x1, 0, N * sizeof(float2), s));
  TRY_CUDA(cudaMemsetAsync(st->u1, 0, D * sizeof(float2), s));
  // the host staging copy of the scalars must land before h_sc is reused
  TRY_CUDA(cudaStreamSynchronize(s));
  return PURIFY_OK;
}

int purify_sdmm_set_prior(purify_ctx* c, purify_sdmm_state* st, int32_t prior, int32_t fgp_iters) {
  if (!c || !st || st->ctx != c) return PURIFY_E_INVALID_ARG;
  if (prior != PURIFY_PRIOR_SARA && prior != PURIFY_PRIOR_TV) return PURIFY_E_INVALID_ARG;
  if (prior == PURIFY_PRIOR_TV && (fgp_iters < 1 || fgp_iters > 1000)) return PURIFY_E_INVALID_ARG;
  DeviceGuard g(c->device);
  if (prior == PURIFY_PRIOR_TV) {
    float2* scr = nullptr;
    TRY(tv_scratch_ready(c, &scr));
  }
  drop_graph(st);
  st->shape_version++;  // batches that captured this state re-capture
  st->prior = prior;
  st->fgp_iters = prior == PURIFY_PRIOR_TV ? fgp_iters : 0;
  return PURIFY_OK;
}

int purify_prox_tv(purify_ctx* c, const float* in, const float* w, float lambda, int32_t iters, float* out,
                   purify_stream_t stream) {
  if (!c || !in || !out || !(lambda >= 0.0f) || iters < 0 || iters > 100000) return PURIFY_E_INVALID_ARG;
  DeviceGuard g(c->device);
  if (!is_device_ptr(in) || !is_device_ptr(out) || (w && !is_device_ptr(w))) return PURIFY_E_NOT_DEVICE_PTR;
  return tv_prox(c, (const float2*)in, w, lambda, iters, (float2*)out, (cudaStream_t)stream);
}

static int purify_sdmm_set_blocks_impl(purify_ctx* c, purify_sdmm_state* st, int32_t R, const int64_t* offsets,
                           const double* eps, purify_stream_t stream) {
  if (!c || !st || st->ctx != c || R < 0 || R > kMaxBlocks) return PURIFY_E_INVALID_ARG;
  const int64_t M = c->M;
  if (R > 0) {
    if (!offsets || !eps || offsets[0] != 0 || offsets[R] != M) return PURIFY_E_INVALID_ARG;
    for (int b = 0; b < R; ++b)
      if (offsets[b + 1] <= offsets[b] || !(eps[b] > 0.0)) return PURIFY_E_INVALID_ARG;
  }
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  TRY_CUDA(cudaStreamSynchronize(s));
  drop_graph(st);  // the iteration changes shape: re-capture on the next step
  st->shape_version++;  // (and so do batches that captured this state)
  void* old[] = {st->d_block_of, st->d_pos, st->d_bchunks, st->d_beps, st->d_bscale};
  for (void* p : old)
    if (p) cudaFree(p);
  st->d_block_of = st->d_pos = nullptr;
  st->d_bchunks = nullptr;
  st->d_beps = nullptr;
  st->d_bscale = nullptr;
  st->nblocks = 0;
  st->nbchunks = 0;
  if (R == 0) return PURIFY_OK;
  // chunks of at most ch visibilities per block, at most kMaxPartials in all
  const int64_t ch = std::max<int64_t>(1024, (M + (kMaxPartials - R) - 1) / (kMaxPartials - R));
  std::vector<int4> chunks;
  for (int b = 0; b < R; ++b) {
    const int64_t nb = offsets[b + 1] - offsets[b];
    const int64_t nc = (nb + ch - 1) / ch;
    for (int64_t k = 0; k < nc; ++k)
      chunks.push_back(make_int4(b, (int)(offsets[b] + nb * k / nc), (int)(offsets[b] + nb * (k + 1) / nc), 0));
  }
  int64_t* d_off = nullptr;
  int e;
  if ((e = dev_alloc(&st->d_block_of, M)) || (e = dev_alloc(&st->d_pos, M)) ||
      (e = dev_alloc(&st->d_bchunks, (int64_t)chunks.size())) || (e = dev_alloc(&st->d_beps, (int64_t)R)) ||
      (e = dev_alloc(&st->d_bscale, (int64_t)R)) || (e = dev_alloc(&d_off, (int64_t)R + 1)))
    return e;
  int rc = PURIFY_OK;
  if (cudaMemcpyAsync(d_off, offsets, (R + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(st->d_beps, eps, R * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(st->d_bchunks, chunks.data(), chunks.size() * sizeof(int4), cudaMemcpyHostToDevice, s) !=
          cudaSuccess)
    rc = PURIFY_E_CUDA;
  if (rc == PURIFY_OK) {
    k_block_of<<<nblk(M), 256, 0, s>>>(c->d_perm, M, d_off, R, st->d_block_of, st->d_pos);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = PURIFY_E_CUDA;
  }
  cudaFree(d_off);
  if (rc != PURIFY_OK) return rc;
  st->nblocks = R;
  st->nbchunks = (int)chunks.size();
  return PURIFY_OK;
}

int purify_sdmm_set_blocks(purify_ctx* c, purify_sdmm_state* st, int32_t R, const int64_t* offsets,
                           const double* eps, purify_stream_t stream) {
  // host containers may throw; no exception crosses the C ABI
  try {
    return purify_sdmm_set_blocks_impl(c, st, R, offsets, eps, stream);
  } catch (const std::bad_alloc&) {
    return PURIFY_E_ALLOC;
  }
}

int purify_sdmm_step(purify_ctx* c, purify_sdmm_state* st, purify_stream_t stream) {
  if (!c || !st || st->ctx != c) return PURIFY_E_INVALID_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (!st->params.use_graph || c->prof.on) {
    TRY(enqueue_sdmm_step(c, st, s));
  } else {
    const GraphKey key = step_graph_key(st);
    if (!st->step_exec || st->graph_key != key) {
      TRY(drop_graph(st));
      if (!st->cap_stream) TRY_CUDA(cudaStreamCreateWithFlags(&st->cap_stream, cudaStreamNonBlocking));
      TRY_CUDA(cudaStreamBeginCapture(st->cap_stream, cudaStreamCaptureModeRelaxed));
      const int rc = enqueue_sdmm_step(c, st, st->cap_stream);
      cudaGraph_t graph = nullptr;
      const cudaError_t e = cudaStreamEndCapture(st->cap_stream, &graph);
      if (rc != PURIFY_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc != PURIFY_OK ? rc : PURIFY_E_CUDA;
      }
      const cudaError_t ie = cudaGraphInstantiate(&st->step_exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) {
        st->step_exec = nullptr;
        return PURIFY_E_CUDA;
      }
      st->graph_key = key;
      g_launches.fetch_sub((unsigned long long)st->launches_per_step, std::memory_order_relaxed);  // capture only
    }
    TRY_CUDA(cudaGraphLaunch(st->step_exec, s));
    g_launches.fetch_add(st->launches_per_step, std::memory_order_relaxed);
  }
  st->iters++;
  return PURIFY_OK;
}

int purify_sdmm_reweight(purify_ctx* c, purify_sdmm_state* st, int32_t round, purify_stream_t stream) {
  if (!c || !st || st->ctx != c || round < 1) return PURIFY_E_INVALID_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t D = ctx_D(c);
  if (st->prior == PURIFY_PRIOR_TV) {
    // TV weights delta / (delta + |grad x_hat|) (same rule as SARA's)
    float2* g = nullptr;
    TRY(tv_gradmag(c, st->xhat, &g, s));
    TRY(launch_max_abs(c, ctx_N(c), g, s));
    return launch_reweight(c, ctx_N(c), g, st->w, round, s);
  }
  SaraProxArgs pa{};
  TRY(sara_analysis(c, st->xhat, st->u1, kSaraPlain, pa, s));
  TRY(launch_max_abs(c, D, st->u1, s));
  return launch_reweight(c, D, st->u1, st->w, round, s);
}

int purify_sdmm_set_weights(purify_ctx* c, purify_sdmm_state* st, const float* w, purify_stream_t stream) {
  if (!c || !st || !w || st->ctx != c) return PURIFY_E_INVALID_ARG;
  DeviceGuard g(c->device);
  if (!is_device_ptr(w)) return PURIFY_E_NOT_DEVICE_PTR;
  return check_cuda(cudaMemcpyAsync(st->w, w, ctx_D(c) * sizeof(float), cudaMemcpyDeviceToDevice,
                                    (cudaStream_t)stream));
}

int purify_sdmm_get_image(purify_ctx* c, purify_sdmm_state* st, float* x_out, purify_stream_t stream) {
  if (!c || !st || !x_out || st->ctx != c) return PURIFY_E_INVALID_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  TRY_CUDA(cudaMemcpyAsync(x_out, st->xhat, ctx_N(c) * sizeof(float2), cudaMemcpyDefault, s));
  if (!is_device_ptr(x_out)) TRY_CUDA(cudaStreamSynchronize(s));
  return PURIFY_OK;
}

int purify_sdmm_get_report(purify_ctx* c, purify_sdmm_state* st, purify_report* rep, purify_stream_t stream) {
  if (!c || !st || !rep || st->ctx != c) return PURIFY_E_INVALID_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  TRY_CUDA(cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
  TRY_CUDA(cudaStreamSynchronize(s));
  if (c->h_sc->dev_error) return PURIFY_E_TIMEOUT;
  rep->iters = st->iters;
  rep->f1 = c->h_sc->f1;
  rep->zeta = c->h_sc->zeta;
  rep->nu = c->h_sc->nu;
  rep->nu_min = c->h_sc->nu_min;
  rep->gamma = c->h_sc->gamma;
  rep->cg_residual = c->h_sc->cg_res;
  return PURIFY_OK;
}

int purify_sdmm_solve(purify_ctx* c, const float* y, double eps, const purify_sdmm_params* params, float* x_out,
                      purify_report* report, purify_stream_t stream) {
  if (!c || !y || !x_out || !(eps > 0.0)) return PURIFY_E_INVALID_ARG;
  DeviceGuard g(c->device);
  purify_sdmm_state* st = nullptr;
  TRY(purify_sdmm_state_create(c, &st));
  int rc = purify_sdmm_init(c, st, y, eps, params, stream);
  purify_report rep{};
  for (int round = 0; rc == PURIFY_OK && round < st->params.rounds; ++round) {
    if (round > 0) rc = purify_sdmm_reweight(c, st, round, stream);
    for (int it = 0; rc == PURIFY_OK && it < st->params.max_iters; ++it) {
      rc = purify_sdmm_step(c, st, stream);
      if (rc == PURIFY_OK && st->params.check_every > 0 && (it + 1) % st->params.check_every == 0) {
        rc = purify_sdmm_get_report(c, st, &rep, stream);
        if (rc == PURIFY_OK && rep.zeta < st->params.xi && rep.nu_min >= 1.0 - st->params.tau &&
            rep.nu <= 1.0 + st->params.tau)
          break;
      }
    }
  }
  if (rc == PURIFY_OK) rc = purify_sdmm_get_image(c, st, x_out, stream);
  if (rc == PURIFY_OK && report) rc = purify_sdmm_get_report(c, st, report, stream);
  if (rc == PURIFY_OK) rc = check_cuda(cudaStreamSynchronize((cudaStream_t)stream));
  purify_sdmm_state_destroy(st);
  return rc;
}

// ---------------------------------------------------------------------------
// Checkpoint blob: header, then xhat r p x1 z3 (N each), z1 (D), w (D float),
// z2 (M), y (M), then the device scalars.
// ---------------------------------------------------------------------------
struct BlobHeader {
  uint64_t magic;
  int64_t n, M, q, iters;
  double eps;
};
static const uint64_t kBlobMagic = 0x5055524946594331ull;  // "PURIFYC1"

static size_t blob_bytes(const purify_ctx* c) {
  const int64_t N = ctx_N(c), D = ctx_D(c), M = c->M;
  return sizeof(BlobHeader) + (5 * N + D + 2 * M) * sizeof(float2) + D * sizeof(float) + sizeof(DevScalars);
}

int purify_sdmm_state_bytes(purify_ctx* c, size_t* bytes) {
  if (!c || !bytes) return PURIFY_E_INVALID_ARG;
  *bytes = blob_bytes(c);
  return PURIFY_OK;
}

int purify_sdmm_export(purify_ctx* c, purify_sdmm_state* st, void* host_buf, size_t bytes, purify_stream_t stream) {
  if (!c || !st || !host_buf || st->ctx != c) return PURIFY_E_INVALID_ARG;
  if (bytes < blob_bytes(c)) return PURIFY_E_SIZE;
  if (st->y_bf16) return PURIFY_E_UNSUPPORTED;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = ctx_N(c), D = ctx_D(c), M = c->M;
  char* p = (char*)host_buf;
  BlobHeader h{kBlobMagic, c->n, c->M, c->q, st->iters, st->eps};
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  float2* vecs[] = {st->xhat, st->r, st->p, st->x1, st->z3};
  for (float2* v : vecs) {
    TRY_CUDA(cudaMemcpyAsync(p, v, N * sizeof(float2), cudaMemcpyDeviceToHost, s));
    p += N * sizeof(float2);
  }
  TRY_CUDA(cudaMemcpyAsync(p, st->z1, D * sizeof(float2), cudaMemcpyDeviceToHost, s));
  p += D * sizeof(float2);
  TRY_CUDA(cudaMemcpyAsync(p, st->w, D * sizeof(float), cudaMemcpyDeviceToHost, s));
  p += D * sizeof(float);
  TRY_CUDA(cudaMemcpyAsync(p, st->z2, M * sizeof(float2), cudaMemcpyDeviceToHost, s));
  p += M * sizeof(float2);
  TRY_CUDA(cudaMemcpyAsync(p, st->y, M * sizeof(float2), cudaMemcpyDeviceToHost, s));
  p += M * sizeof(float2);
  TRY_CUDA(cudaMemcpyAsync(p, c->d_sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
  return check_cuda(cudaStreamSynchronize(s));
}

int purify_sdmm_import(purify_ctx* c, purify_sdmm_state* st, const void* host_buf, size_t bytes,
                       purify_stream_t stream) {
  if (!c || !st || !host_buf || st->ctx != c) return PURIFY_E_INVALID_ARG;
  if (bytes < blob_bytes(c)) return PURIFY_E_SIZE;
  const char* p = (const char*)host_buf;
  BlobHeader h;
  std::memcpy(&h, p, sizeof(h));
  if (h.magic != kBlobMagic || h.n != c->n || h.M != c->M || h.q != c->q) return PURIFY_E_INVALID_ARG;
  p += sizeof(h);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = ctx_N(c), D = ctx_D(c), M = c->M;
  float2* vecs[] = {st->xhat, st->r, st->p, st->x1, st->z3};
  for (float2* v : vecs) {
    TRY_CUDA(cudaMemcpyAsync(v, p, N * sizeof(float2), cudaMemcpyHostToDevice, s));
    p += N * sizeof(float2);
  }
  TRY_CUDA(cudaMemcpyAsync(st->z1, p, D * sizeof(float2), cudaMemcpyHostToDevice, s));
  p += D * sizeof(float2);
  TRY_CUDA(cudaMemcpyAsync(st->w, p, D * sizeof(float), cudaMemcpyHostToDevice, s));
  p += D * sizeof(float);
  TRY_CUDA(cudaMemcpyAsync(st->z2, p, M * sizeof(float2), cudaMemcpyHostToDevice, s));
  p += M * sizeof(float2);
  TRY_CUDA(cudaMemcpyAsync(st->y, p, M * sizeof(float2), cudaMemcpyHostToDevice, s));
  p += M * sizeof(float2);
  TRY_CUDA(cudaMemcpyAsync(c->d_sc, p, sizeof(DevScalars), cudaMemcpyHostToDevice, s));
  st->iters = h.iters;
  st->eps = h.eps;
  st->y_bf16 = 0;
  st->shape_version++;
  return check_cuda(cudaStreamSynchronize(s));
}

int purify_profile_enable(purify_ctx* c, int on) {
  if (!c) return PURIFY_E_INVALID_ARG;
  c->prof.on = on != 0;
  return PURIFY_OK;
}

static int purify_profile_collect_impl(purify_ctx* c, int32_t max_entries, char* names, int64_t* launches, double* ms,
                           int32_t* n_entries) {
  if (!c || max_entries < 0 || !n_entries || (max_entries > 0 && (!names || !launches || !ms)))
    return PURIFY_E_INVALID_ARG;
  DeviceGuard g(c->device);
  TRY_CUDA(cudaDeviceSynchronize());
  std::vector<std::string> keys;
  std::vector<int64_t> cnt;
  std::vector<double> tot;
  for (const auto& r : c->prof.recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, c->prof.pool[r.second], c->prof.pool[r.second + 1]) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    size_t k = 0;
    while (k < keys.size() && keys[k] != r.first) ++k;
    if (k == keys.size()) {
      keys.emplace_back(r.first);
      cnt.push_back(0);
      tot.push_back(0.0);
    }
    cnt[k] += 1;
    tot[k] += t;
  }
  const int ne = (int)std::min<size_t>(keys.size(), (size_t)max_entries);
  for (int k = 0; k < ne; ++k) {
    std::memset(names + 32 * k, 0, 32);
    std::strncpy(names + 32 * k, keys[k].c_str(), 31);
    launches[k] = cnt[k];
    ms[k] = tot[k];
  }
  *n_entries = ne;
  c->prof.recs.clear();
  c->prof.used = 0;
  return PURIFY_OK;
}

int purify_profile_collect(purify_ctx* c, int32_t max_entries, char* names, int64_t* launches, double* ms,
                           int32_t* n_entries) {
  // host containers may throw; no exception crosses the C ABI
  try {
    return purify_profile_collect_impl(c, max_entries, names, launches, ms, n_entries);
  } catch (const std::bad_alloc&) {
    return PURIFY_E_ALLOC;
  }
}

uint64_t purify_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
