// purify_phi_static: the measurement operator y = Phi x with no allocation.
//
// Some callers cannot allocate device memory when they need Phi: a process
// whose GPU memory is already reserved in full by another allocator (a
// framework's caching pool, an inference server that pins its arena at
// start-up), or a latency-critical loop where a cudaMalloc, with its implicit
// device synchronisation, is not acceptable.  purify_create allocates tables
// and scratch, so it cannot serve them.  This entry point needs no context:
// its scratch (the oversampled grid, the row-transformed half grid, twiddles
// and deapodisation factors) lives in one file-scope __device__ array of
// fixed size, which every GPU that loads the library holds until the process
// exits.  The caller passes the frequencies, the image and the output.
//
// Limits: image side n <= kStaticMaxN (256), so the array is
// 2n*2n + n*2n complex64 + tables, about 3 MiB.  All calls share the array:
// two calls that overlap on the GPU (different streams, or different host
// threads) race on it and give wrong results; order them on one stream.
// The first call on a device looks up the array's device address with that
// device current; make that first call before any stream capture.  The
// array keeps the twiddles and deapodisation factors of the last (n, J) used
// on the device: a call of another size rewrites them (on its stream) before
// its transforms read them, a call of the same size reuses them.
//
// The arithmetic is that of purify_phi (§5 eq. opmodel with B = I): the same
// deapodisation, zero padding, unitary DFT and Kaiser-Bessel interpolation;
// the visibilities are gathered in the caller's order (no sorting, which
// would need a table).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <utility>

#include "common.cuh"
#include "fft.cuh"

namespace {

using namespace purify;

constexpr int kStaticMaxN = 256;
constexpr int kStaticMaxL = 2 * kStaticMaxN;
constexpr size_t kGridBytes = (size_t)kStaticMaxL * kStaticMaxL * sizeof(float2);
constexpr size_t kHalfBytes = (size_t)kStaticMaxN * kStaticMaxL * sizeof(float2);
constexpr size_t kTwBytes = (size_t)kStaticMaxL * sizeof(float2);
constexpr size_t kDzBytes = (size_t)kStaticMaxN * sizeof(float);
constexpr size_t kStaticBytes = kGridBytes + kHalfBytes + kTwBytes + kDzBytes;

// The scratch array (its host-side name is not a device address).
__device__ __align__(256) unsigned char g_phi_scratch[kStaticBytes];

// Device address of g_phi_scratch per device, looked up once per device,
// and the (n, J) whose twiddles and deapodisation factors that device's
// array holds (0 = none yet), so repeated calls of one size skip the tables.
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices];
int g_table_key[kMaxDevices];
std::mutex g_scratch_mu;

// Fitted tap polynomials per kernel support J (they do not depend on n).
KbPoly g_kb[kMaxJ + 1];
bool g_kb_ready[kMaxJ + 1];

int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return PURIFY_E_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_phi_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return PURIFY_E_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return PURIFY_OK;
}

double st_beta(int J) { return M_PI * std::sqrt((J / 2.0) * (J / 2.0) * 2.25 - 0.8); }

double st_kernel(double t, int J, double beta, double i0b) {
  const double s = 2.0 * t / J;
  if (std::fabs(s) > 1.0) return 0.0;
  return std::cyl_bessel_i(0.0, beta * std::sqrt(std::max(0.0, 1.0 - s * s))) / i0b;
}

// Per-tap polynomials of degree kKbDeg in z = 2x - 1, interpolating the
// kernel at Chebyshev nodes (fixed-size arrays: nothing is allocated).
void st_fit(int J, KbPoly& kb) {
  constexpr int np = kKbDeg + 1;
  const double beta = st_beta(J), i0b = std::cyl_bessel_i(0.0, beta);
  kb = KbPoly{};
  kb.J = J;
  for (int a = 0; a < J; ++a) {
    long double A[np][np], f[np];
    for (int i = 0; i < np; ++i) {
      const long double z = std::cos(M_PI * (i + 0.5) / np);
      long double zp = 1.0L;
      for (int j = 0; j < np; ++j) { A[i][j] = zp; zp *= z; }
      f[i] = st_kernel(0.5 * ((double)z + 1.0) + J / 2 - 1 - a, J, beta, i0b);
    }
    for (int k = 0; k < np; ++k) {  // Gaussian elimination, partial pivoting
      int piv = k;
      for (int i = k + 1; i < np; ++i)
        if (std::fabs((double)A[i][k]) > std::fabs((double)A[piv][k])) piv = i;
      for (int j = 0; j < np; ++j) std::swap(A[k][j], A[piv][j]);
      std::swap(f[k], f[piv]);
      for (int i = k + 1; i < np; ++i) {
        const long double m = A[i][k] / A[k][k];
        for (int j = k; j < np; ++j) A[i][j] -= m * A[k][j];
        f[i] -= m * f[k];
      }
    }
    for (int k = np - 1; k >= 0; --k) {
      long double s = f[k];
      for (int j = k + 1; j < np; ++j) s -= A[k][j] * f[j];
      f[k] = s / A[k][k];
    }
    for (int j = 0; j < np; ++j) kb.c[a][j] = (float)f[j];
  }
}

bool st_plan(int L, FftPlan& p) {
  p = FftPlan{};
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
  if (rest != 1) return false;
  finish_plan(p);
  return true;
}

// Twiddles exp(-2 pi i m / L) and 1 / g_hat((r - n/2) / L), in double.
__global__ void k_static_tables(int n, int L, int J, double beta, double i0b, float2* tw, float* dz) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < L; m += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)m / (double)L, &s, &c);
    tw[m] = make_float2((float)c, (float)s);
  }
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const double f = (double)(r - n / 2) / (double)L;
    const double a = sqrt(beta * beta - (M_PI * J * f) * (M_PI * J * f));
    dz[r] = (float)(i0b * a / (J * sinh(a)));
  }
}

template <int EPT>
__global__ void __launch_bounds__(1024) k_static_rows(const float2* __restrict__ x, float2* __restrict__ half,
                                                      const float* __restrict__ dz, const float2* __restrict__ tw,
                                                      FftPlan plan, int n, int nsig) {
  extern __shared__ float2 sm[];
  const int L = plan.L;
  const int r0 = blockIdx.x * nsig;
  const float invL = 1.0f / (float)L;
  for (int idx = threadIdx.x; idx < nsig * L; idx += blockDim.x) {
    const int s = idx / L, e = idx - s * L;
    int cc = e + (n >> 1);
    if (cc >= L) cc -= L;
    float2 v = make_float2(0.f, 0.f);
    if (cc < n) v = cscale(x[(size_t)(r0 + s) * n + cc], dz[r0 + s] * dz[cc] * invL);
    sm[idx] = v;
  }
  __syncthreads();
  fft_smem<EPT, false>(sm, SigLayout{L, 1}, plan, nsig, tw);
  for (int idx = threadIdx.x; idx < nsig * L; idx += blockDim.x) half[(size_t)r0 * L + idx] = sm[idx];
}

template <int EPT>
__global__ void __launch_bounds__(1024) k_static_cols(const float2* __restrict__ half, float2* __restrict__ X,
                                                      const float2* __restrict__ tw, FftPlan plan, int n, int nsig) {
  extern __shared__ float2 sm[];
  const int L = plan.L;
  const int c0 = blockIdx.x * nsig;
  for (int idx = threadIdx.x; idx < nsig * L; idx += blockDim.x) {
    const int e = idx / nsig, s = idx - e * nsig;
    int r = e + (n >> 1);
    if (r >= L) r -= L;
    sm[idx] = (r < n) ? half[(size_t)r * L + c0 + s] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_smem<EPT, true>(sm, SigLayout{1, nsig}, plan, nsig, tw);
  for (int idx = threadIdx.x; idx < nsig * L; idx += blockDim.x) {
    const int e = idx / nsig, s = idx - e * nsig;
    X[(size_t)e * L + c0 + s] = sm[idx];
  }
}

template <int J>
__global__ void k_static_degrid(const float2* __restrict__ X, const float2* __restrict__ uv, float2* __restrict__ y,
                                KbPoly kb, KappaScale ks, int L, int64_t M) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 u = uv[i];
    int k0r, k0c;
    float fr, fc;
    split_kappa(u.x, ks, k0r, fr);
    split_kappa(u.y, ks, k0c, fc);
    k0r -= J / 2 - 1;
    k0c -= J / 2 - 1;
    float wr[J], wc[J];
    kb_weights<J>(kb, fr, wr);
    kb_weights<J>(kb, fc, wc);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < J; ++a) {
      const float2* row = X + (size_t)wrap(k0r + a, L) * L;
      float2 t = make_float2(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < J; ++b) {
        const float2 g = row[wrap(k0c + b, L)];
        t.x = fmaf(wc[b], g.x, t.x);
        t.y = fmaf(wc[b], g.y, t.y);
      }
      acc.x = fmaf(wr[a], t.x, acc.x);
      acc.y = fmaf(wr[a], t.y, acc.y);
    }
    y[i] = acc;
  }
}

// Managed memory, or device memory of the current device (the one whose copy
// of the scratch array the call uses); another GPU's buffer is rejected.
bool is_dev(const void* p, int dev) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

template <int EPT>
int st_fft(const float2* x, float2* half, float2* X, const float* dz, const float2* tw, const FftPlan& plan, int n,
           cudaStream_t s) {
  const int L = plan.L;
  int rs = 1;
  while (rs * 2 * L / EPT <= 128 && n % (rs * 2) == 0) rs *= 2;
  int cs = 4;
  while (cs * 2 * L / EPT <= 256 && L % (cs * 2) == 0 && cs < 16) cs *= 2;
  k_static_rows<EPT><<<n / rs, rs * L / EPT, rs * L * sizeof(float2), s>>>(x, half, dz, tw, plan, n, rs);
  k_static_cols<EPT><<<L / cs, cs * L / EPT, cs * L * sizeof(float2), s>>>(half, X, tw, plan, n, cs);
  return cudaGetLastError() == cudaSuccess ? PURIFY_OK : PURIFY_E_CUDA;
}

}  // namespace

extern "C" int purify_phi_static(int32_t n, int32_t J, int64_t M, const float* uv, const float* x, float* y,
                                 purify_stream_t stream) {
  if (!uv || !x || !y) return PURIFY_E_INVALID_ARG;
  if (J != 2 && J != 4 && J != 6 && J != 8) return PURIFY_E_SIZE;
  if (n < 8 || n > kStaticMaxN || n % 2 != 0 || M < 1 || M > 2147483647LL) return PURIFY_E_SIZE;
  const int L = 2 * n;
  FftPlan plan;
  if (!st_plan(L, plan) || (L % 3 == 0 && L % 12 != 0)) return PURIFY_E_UNSUPPORTED;
  {
    int r = L, threes = 0;
    while (r % 3 == 0) { r /= 3; ++threes; }
    if (threes > 1) return PURIFY_E_UNSUPPORTED;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return PURIFY_E_CUDA;
  }
  if (!is_dev(uv, dev) || !is_dev(x, dev) || !is_dev(y, dev)) return PURIFY_E_NOT_DEVICE_PTR;
  void* base = nullptr;
  const int rc = scratch_address(dev, &base);
  if (rc != PURIFY_OK) return rc;
  unsigned char* b = static_cast<unsigned char*>(base);
  float2* X = reinterpret_cast<float2*>(b);
  float2* half = reinterpret_cast<float2*>(b + kGridBytes);
  float2* tw = reinterpret_cast<float2*>(b + kGridBytes + kHalfBytes);
  float* dz = reinterpret_cast<float*>(b + kGridBytes + kHalfBytes + kTwBytes);
  cudaStream_t s = (cudaStream_t)stream;
  const double beta = st_beta(J), i0b = std::cyl_bessel_i(0.0, beta);
  KbPoly kb;
  {
    // the tables in the array are rewritten only when (n, J) changes on this
    // device; the polynomials are fitted once per J in the process
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    const int key = n * 16 + J;
    if (g_table_key[dev] != key) {
      k_static_tables<<<(L + 255) / 256, 256, 0, s>>>(n, L, J, beta, i0b, tw, dz);
      if (cudaGetLastError() != cudaSuccess) return PURIFY_E_CUDA;
      g_table_key[dev] = key;
    }
    if (!g_kb_ready[J]) {
      st_fit(J, g_kb[J]);
      g_kb_ready[J] = true;
    }
    kb = g_kb[J];
  }
  const int frc = (L % 3 == 0) ? st_fft<12>((const float2*)x, half, X, dz, tw, plan, n, s)
                               : st_fft<8>((const float2*)x, half, X, dz, tw, plan, n, s);
  if (frc != PURIFY_OK) return frc;
  const double sc = (double)L / (2.0 * M_PI);
  KappaScale ks{(float)sc, (float)(sc - (double)(float)sc)};
  const unsigned blocks = (unsigned)std::min<int64_t>((M + 255) / 256, 4096);
  switch (J) {
    case 2: k_static_degrid<2><<<blocks, 256, 0, s>>>(X, (const float2*)uv, (float2*)y, kb, ks, L, M); break;
    case 4: k_static_degrid<4><<<blocks, 256, 0, s>>>(X, (const float2*)uv, (float2*)y, kb, ks, L, M); break;
    case 6: k_static_degrid<6><<<blocks, 256, 0, s>>>(X, (const float2*)uv, (float2*)y, kb, ks, L, M); break;
    default: k_static_degrid<8><<<blocks, 256, 0, s>>>(X, (const float2*)uv, (float2*)y, kb, ks, L, M); break;
  }
  return cudaGetLastError() == cudaSuccess ? PURIFY_OK : PURIFY_E_CUDA;
}
