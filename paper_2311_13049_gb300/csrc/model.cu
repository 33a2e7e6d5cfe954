// model.cu -- once-per-model precompute, all in double on the GPU:
//   gamma = arctan(1/Q)/pi and c, eta, tau (Sec. 1, coefficients of Eq. (1.1));
//   gamma0 = grid mean of gamma (the expansion centre s0 of Eq. (2.13) is the
//   domain average of s; s = 1 + gamma and s = 1/2 + gamma share gamma0);
//   delta = gamma - gamma0, A = c^2 eta, B = c^2 tau (rounded to the working
//   precision);
//   spectral tables |mu_k|^{2 s0} / N and ln|mu_k|^2 of Eq. (2.13) (k = 0 -> 0);
//   FFT twiddles exp(-2 pi i r k / N).
#include <cuda_runtime.h>

#include <cstdlib>
#include <mutex>
#include <unordered_map>
#include <vector>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace vofl {

namespace {

constexpr int RED_BLOCKS = 512;
constexpr int RED_THREADS = 256;

// may run in place (q == g): each element is read before it is written
__global__ void k_gamma_from_q(const double* q, double* g, long long n, int* bad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double Q = q[i];
    if (!(Q > 0.0) || !isfinite(Q)) atomicExch(bad, 1);
    g[i] = atan(1.0 / Q) / M_PI;
  }
}

__global__ void k_check_gamma(const double* __restrict__ g, long long n, int* bad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = g[i];
    if (!(v >= 0.0 && v < 0.5)) atomicExch(bad, 1);
  }
}

__global__ void k_check_order(const double* __restrict__ s, long long n, int* bad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = s[i];
    if (!(v > 0.0 && v <= 2.0)) atomicExch(bad, 1);
  }
}

// General model: delta = s - s0, A = -kappa, B = 0 (the seismic update with
// these coefficients is the leap-frog scheme of the general model).
template <typename T>
__global__ void k_coeffs_general(const double* __restrict__ sfield, double s0, double kappa, long long n,
                                 T* __restrict__ delta, T* __restrict__ A, T* __restrict__ B) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    delta[i] = T(sfield[i] - s0);
    A[i] = T(-kappa);
    B[i] = T(0);
  }
}

// Deterministic two-pass sum: fixed grid, fixed tree order.
__global__ void k_sum_pass1(const double* __restrict__ x, long long n, double* __restrict__ part) {
  __shared__ double s[RED_THREADS];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)RED_THREADS + threadIdx.x; i < n; i += (long long)RED_BLOCKS * RED_THREADS)
    acc += x[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void k_sum_pass2(const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double s[RED_BLOCKS];
  for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) s[i] = part[i];
  __syncthreads();
  for (int w = RED_BLOCKS / 2; w > 0; w >>= 1) {
    for (int i = threadIdx.x; i < w; i += blockDim.x) s[i] += s[i + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = s[0];
}

// rel-L2 diagnostics: per block, in double, over a grid-stride slice:
// sum (x - y)^2, sum y^2, max |x - y|, max |y|; then one block combines the
// partials in a fixed order (deterministic for a given launch shape).
constexpr int DIAG_BLOCKS = 240;  // 4 partials each: 960 doubles of the context scratch
// max that keeps a NaN (fmax drops it): a field with a NaN reports NaN
__device__ __forceinline__ double nan_max(double a, double b) { return (a != a || b != b) ? NAN : fmax(a, b); }
template <typename TX, typename TY>
__global__ void k_diff_pass1(const TX* __restrict__ x, const TY* __restrict__ y, long long n,
                             double* __restrict__ part) {
  __shared__ double s[4][RED_THREADS];
  double d2 = 0.0, y2 = 0.0, dm = 0.0, ym = 0.0;
  for (long long i = blockIdx.x * (long long)RED_THREADS + threadIdx.x; i < n;
       i += (long long)DIAG_BLOCKS * RED_THREADS) {
    const double yi = (double)y[i];
    const double di = (double)x[i] - yi;
    d2 = fma(di, di, d2);
    y2 = fma(yi, yi, y2);
    dm = nan_max(dm, fabs(di));
    ym = nan_max(ym, fabs(yi));
  }
  s[0][threadIdx.x] = d2;
  s[1][threadIdx.x] = y2;
  s[2][threadIdx.x] = dm;
  s[3][threadIdx.x] = ym;
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s[0][threadIdx.x] += s[0][threadIdx.x + w];
      s[1][threadIdx.x] += s[1][threadIdx.x + w];
      s[2][threadIdx.x] = nan_max(s[2][threadIdx.x], s[2][threadIdx.x + w]);
      s[3][threadIdx.x] = nan_max(s[3][threadIdx.x], s[3][threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x < 4) part[threadIdx.x * DIAG_BLOCKS + blockIdx.x] = s[threadIdx.x][0];
}

// out: ||x - y|| / ||y||, max|x - y| / max|y|, ||y||, max|y| (ratios 0 when
// y is all zero and x equals it, +inf when only y is zero, NaN when either
// field holds a NaN)
__global__ void k_diff_pass2(const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double s[4][256];
  for (int k = 0; k < 4; ++k) s[k][threadIdx.x] = threadIdx.x < DIAG_BLOCKS ? part[k * DIAG_BLOCKS + threadIdx.x] : 0.0;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s[0][threadIdx.x] += s[0][threadIdx.x + w];
      s[1][threadIdx.x] += s[1][threadIdx.x + w];
      s[2][threadIdx.x] = nan_max(s[2][threadIdx.x], s[2][threadIdx.x + w]);
      s[3][threadIdx.x] = nan_max(s[3][threadIdx.x], s[3][threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double dn = sqrt(s[0][0]), yn = sqrt(s[1][0]);
    auto ratio = [](double a, double b) { return b > 0 ? a / b : (a > 0 ? INFINITY : (a == 0 ? 0.0 : NAN)); };
    out[0] = (dn != dn || yn != yn) ? NAN : ratio(dn, yn);
    out[1] = (s[2][0] != s[2][0] || s[3][0] != s[3][0]) ? NAN : ratio(s[2][0], s[3][0]);
    out[2] = yn;
    out[3] = s[3][0];
  }
}

template <typename T>
__global__ void k_coeffs(const double* __restrict__ g, const double* __restrict__ c0f, double c0s, double w0,
                         double g0, long long n, T* __restrict__ delta, T* __restrict__ A, T* __restrict__ B) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double gm = g[i];
    const double c0 = c0f ? c0f[i] : c0s;
    const double c = c0 * cos(M_PI * gm / 2.0);
    const double sc = pow(c0, 2.0 * gm) * pow(w0, -2.0 * gm);  // c0^{2g} w0^{-2g}
    const double eta = -sc * cos(M_PI * gm);
    const double tau = -(sc / c0) * sin(M_PI * gm);
    delta[i] = T(gm - g0);
    A[i] = T(c * c * eta);
    B[i] = T(c * c * tau);
  }
}

// Tables in the fused 2D layout: column-major over the half spectrum,
// index [c][k2] for c = k1 in [0, nx/2], k2 in [0, ny).
// P[0] = |mu|^{2 s01}/(N lambda), P[1] = scale2 |mu|^{2 s02}/(N lambda),
// Lg = ln|mu|^2, lambda = the symbol of the transformed discrete Laplacian.
__global__ void k_tables_fused2d(int nx, int ny, double lx, double ly, double s01, double s02, double scale2,
                                 double ryy, float* __restrict__ P, float* __restrict__ Lg) {
  const int H = nx / 2;
  const long long total = (long long)(H + 1) * ny;
  const double invN = 1.0 / ((double)nx * (double)ny);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / ny);
    const int k2 = (int)(i % ny);
    const int k2s = (k2 < ny / 2) ? k2 : k2 - ny;
    const double m1 = 2.0 * M_PI * (double)c / lx;
    const double m2 = 2.0 * M_PI * (double)k2s / ly;
    const double mu2 = m1 * m1 + m2 * m2;
    if (mu2 == 0.0) {
      P[i] = 0.f;
      P[total + i] = 0.f;
      Lg[i] = 0.f;
    } else {
      // the forward transform is of the discrete Laplacian w (symbol lambda)
      const double s1 = sinpi((double)c / nx), s2 = sinpi((double)k2 / ny);
      const double lam = -4.0 * s1 * s1 - 4.0 * ryy * s2 * s2;
      const double L = log(mu2);
      P[i] = (float)(exp(s01 * L) * invN / lam);
      P[total + i] = (float)(exp(s02 * L) * invN * scale2 / lam);
      Lg[i] = (float)L;
    }
  }
}

// omega(x) = sqrt|c^2 eta| |mu_max|^{1 + gamma}: the largest angular
// frequency of the undamped part of Eq. (1.1) at x (the highest Fourier mode
// |mu_max| of the grid); for the general model sqrt(kappa) |mu_max|^{s}
// (A = -kappa, g = s, off = 0).  Max over the grid as an atomic max of the bit
// pattern (non-negative doubles order like their bits): order-independent.
template <typename T>
__global__ void k_omega_max(const T* __restrict__ A, const double* __restrict__ g, long long n, double lmu,
                            double off, unsigned long long* out) {
  double m = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, sqrt(fabs((double)A[i])) * exp((off + g[i]) * lmu));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// max_x |g(x) - centre| (non-negative doubles order like their bits)
__global__ void k_abs_dev_max(const double* __restrict__ g, double centre, long long n, unsigned long long* out) {
  double m = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(g[i] - centre));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// Tables in the cuFFT R2C layout [..][nz][ny][nx/2+1] (row-major, x halved),
// for a forward transform of the discrete Laplacian (symbol lambda, see
// fused2d.cu): P = |mu|^{2 s0} / (N lambda).
template <typename T>
__global__ void k_tables_plain(int nx, int ny, int nz, double lx, double ly, double lz, double s01, double s02,
                               double invN, double ry, double rz, T* __restrict__ P1, T* __restrict__ P2,
                               T* __restrict__ Lg) {
  const int hx = nx / 2 + 1;
  const long long total = (long long)hx * ny * nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(i % hx);
    const int ky = (int)((i / hx) % ny);
    const int kz = (int)(i / ((long long)hx * ny));
    const int kys = (ky < ny / 2) ? ky : ky - ny;
    const int kzs = (kz < nz / 2) ? kz : kz - nz;
    const double mx = 2.0 * M_PI * kx / lx;
    const double my = (ny > 1) ? 2.0 * M_PI * kys / ly : 0.0;
    const double mz = (nz > 1) ? 2.0 * M_PI * kzs / lz : 0.0;
    const double mu2 = mx * mx + my * my + mz * mz;
    if (mu2 == 0.0) {
      P1[i] = T(0);
      P2[i] = T(0);
      Lg[i] = T(0);
    } else {
      const double sx = sinpi((double)kx / nx), sy = sinpi((double)ky / ny), sz = sinpi((double)kz / nz);
      const double lam = -4.0 * (sx * sx + ry * sy * sy + rz * sz * sz);
      const double L = log(mu2);
      P1[i] = T(exp(s01 * L) * invN / lam);
      P2[i] = T(exp(s02 * L) * invN / lam);
      Lg[i] = T(L);
    }
  }
}

// tw[r*NB + k] = exp(-2 pi i r k / N), r < R, k < NB; then, for N with a
// middle stage, tw[N + t] = exp(-2 pi i t / NM), t < NM
__global__ void k_twiddles(int N, int NB, int R, int NM, float2* tw) {
  const int total = NB * R + NM;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    long long t;
    int n;
    if (i < NB * R) {
      const int r = i / NB, k = i % NB;
      t = ((long long)r * k) % N;
      n = N;
    } else {
      t = i - NB * R;
      n = NM;
    }
    double s, c;
    sincospi(-2.0 * (double)t / (double)n, &s, &c);
    tw[i] = make_float2((float)c, (float)s);
  }
}

// Twiddles of the wide line transform (fft_wide.cuh) of length N:
// tw[r (N/4) + j] = w_N^{r j} (r < 4, j < N/4), then
// tw[N + r 16 + k] = w_{N/4}^{r k} (r < N/64, k < 16).
__global__ void k_twiddles_wide(int N, float2* tw) {
  const int total = N + (N / 64) * 16;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    long long t;
    int n;
    if (i < N) {
      const int r = i / (N / 4), j = i % (N / 4);
      t = (long long)r * j;
      n = N;
    } else {
      const int r = (i - N) / 16, k = (i - N) % 16;
      t = (long long)r * k;
      n = N / 4;
    }
    double s, c;
    sincospi(-2.0 * (double)(t % n) / (double)n, &s, &c);
    tw[i] = make_float2((float)c, (float)s);
  }
}

inline int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 4096) b = 4096;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

std::atomic<uint64_t> g_kernel_launches{0};

// > 0: device allocations left until the injected failure (the last one
// fails); 0: none pending
std::atomic<long long> g_fail_alloc{0};

long long debug_fail_alloc(long long k) { return g_fail_alloc.exchange(k < 0 ? 0 : k); }

// Canary mode, a stand-in for a memory checker: every buffer gets 64 KB
// pads of a known byte on both sides; a kernel that writes past either end
// of a buffer (by up to 64 KB) changes a pad, found when the buffer is freed
// or by debug_canaries.
namespace {
constexpr size_t kCanaryPad = size_t(64) << 10;  // a multiple of 256: the buffer keeps its alignment
constexpr unsigned char kCanaryByte = 0xA5;
struct CanaryAlloc {
  unsigned char* base;
  size_t bytes;
  unsigned long long serial;
};
std::mutex g_canary_mu;
std::unordered_map<void*, CanaryAlloc>& canary_live() {
  static auto* live = new std::unordered_map<void*, CanaryAlloc>();  // outlives static destruction
  return *live;
}
std::atomic<long long> g_canary_bad{0};
std::atomic<unsigned long long> g_canary_serial{0};

bool canary_mode() {
  static const bool on = [] {
    const char* e = std::getenv("VOFL_DEBUG_CANARY");
    return e && e[0] == '1';
  }();
  return on;
}

bool pads_intact(const CanaryAlloc& a) {
  std::vector<unsigned char> h(2 * kCanaryPad);
  if (cudaMemcpy(h.data(), a.base, kCanaryPad, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(h.data() + kCanaryPad, a.base + kCanaryPad + a.bytes, kCanaryPad, cudaMemcpyDeviceToHost) !=
          cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  for (unsigned char c : h)
    if (c != kCanaryByte) return false;
  return true;
}
}  // namespace

cudaError_t dev_malloc_bytes(void** p, size_t bytes) {
  long long k = g_fail_alloc.load();
  while (k > 0) {
    if (g_fail_alloc.compare_exchange_weak(k, k - 1)) {
      if (k == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  if (!canary_mode()) return cudaMalloc(p, bytes);
  unsigned char* base = nullptr;
  cudaError_t e = cudaMalloc((void**)&base, bytes + 2 * kCanaryPad);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  if ((e = cudaMemset(base, kCanaryByte, kCanaryPad)) != cudaSuccess ||
      (e = cudaMemset(base + kCanaryPad + bytes, kCanaryByte, kCanaryPad)) != cudaSuccess ||
      (e = cudaDeviceSynchronize()) != cudaSuccess) {
    cudaFree(base);
    *p = nullptr;
    return e;
  }
  {
    std::lock_guard<std::mutex> lock(g_canary_mu);
    canary_live()[base + kCanaryPad] = {base, bytes, g_canary_serial.fetch_add(1)};
  }
  *p = base + kCanaryPad;
  return cudaSuccess;
}

cudaError_t dev_free(void* p) {
  if (!p) return cudaSuccess;
  if (canary_mode()) {
    CanaryAlloc a{};
    bool found = false;
    {
      std::lock_guard<std::mutex> lock(g_canary_mu);
      auto it = canary_live().find(p);
      if (it != canary_live().end()) {
        a = it->second;
        canary_live().erase(it);
        found = true;
      }
    }
    if (found) {
      cudaDeviceSynchronize();  // kernels still writing the buffer finish first
      if (!pads_intact(a)) g_canary_bad.fetch_add(1);
      return cudaFree(a.base);
    }
  }
  return cudaFree(p);
}

long long debug_canaries(long long* live, int poke) {
  if (live) *live = 0;
  if (!canary_mode()) return -1;
  cudaDeviceSynchronize();
  std::lock_guard<std::mutex> lock(g_canary_mu);
  if (poke) {  // change one pad byte of the newest live buffer (a check that the check sees it)
    const CanaryAlloc* newest = nullptr;
    for (auto& kv : canary_live())
      if (!newest || kv.second.serial > newest->serial) newest = &kv.second;
    if (newest) {
      cudaMemset(newest->base + kCanaryPad + newest->bytes, 0, 1);
      cudaDeviceSynchronize();
    }
  }
  long long bad = g_canary_bad.load();
  for (auto& kv : canary_live()) {
    if (!pads_intact(kv.second)) ++bad;
    if (live) ++*live;
  }
  return bad;
}

int cuda_err(vofl_ctx* c, cudaError_t e, const char* where) {
  if (c) {
    c->err = std::string(where) + ": " + cudaGetErrorString(e);
  }
  return e == cudaErrorMemoryAllocation ? VOFL_ENOMEM : VOFL_ECUDA;
}

// dt = courant * 2 / omega_max (the explicit leap-frog bound 2/omega of the
// undamped part, scaled by a safety factor).
int model_suggest_dt(vofl_ctx* c, double courant, double* dt) {
  double mu2 = 0.0;
  for (int i = 0; i < c->ndim; ++i) {
    const double m = M_PI * (double)c->n[i] / (c->hi[i] - c->lo[i]);  // Nyquist |mu| along axis i
    mu2 += m * m;
  }
  unsigned long long* d_out = reinterpret_cast<unsigned long long*>(c->d_scratch + RED_BLOCKS + 2);
  VOFL_CUDA(c, cudaMemsetAsync(d_out, 0, sizeof(unsigned long long), c->stream));
  const double lmu = 0.5 * std::log(mu2);
  const double off = c->general ? 0.0 : 1.0;
  if (c->prec == VOFL_F32)
    k_omega_max<float><<<grid_for(c->N, 256), 256, 0, c->stream>>>((const float*)c->A, c->d_gamma, c->N, lmu, off,
                                                                    d_out);
  else
    k_omega_max<double><<<grid_for(c->N, 256), 256, 0, c->stream>>>((const double*)c->A, c->d_gamma, c->N, lmu,
                                                                     off, d_out);
  count_launch();
  VOFL_CUDA(c, cudaGetLastError());
  unsigned long long bits = 0;
  VOFL_CUDA(c, cudaMemcpyAsync(&bits, d_out, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
  VOFL_CUDA(c, cudaStreamSynchronize(c->stream));
  double wmax;
  std::memcpy(&wmax, &bits, sizeof(wmax));
  if (!(wmax > 0.0)) return set_err(c, VOFL_EINVAL, "the model has no positive frequency");
  *dt = courant * 2.0 / wmax;
  return VOFL_OK;
}

// Smallest M <= M_max whose Taylor remainder bound a^{M+1}/(M+1)! e^{2a}
// (a = max|delta| max_k |ln|mu_k|^2|, k != 0) is at most tol: the relative
// truncation error of every mode's weight |mu_k|^{2 s0} exp(delta ln|mu_k|^2)
// in Eq. (2.13).
int model_suggest_M(vofl_ctx* c, double tol, int M_max, int* M) {
  double lmu_min = 1e300, mu2 = 0.0;
  for (int i = 0; i < c->ndim; ++i) {
    const double L = c->hi[i] - c->lo[i];
    lmu_min = std::min(lmu_min, 2.0 * M_PI / L);
    const double m = M_PI * (double)c->n[i] / L;
    mu2 += m * m;
  }
  const double lmax = std::max(std::fabs(std::log(lmu_min * lmu_min)), std::fabs(std::log(mu2)));
  unsigned long long* d_out = reinterpret_cast<unsigned long long*>(c->d_scratch + RED_BLOCKS + 3);
  VOFL_CUDA(c, cudaMemsetAsync(d_out, 0, sizeof(unsigned long long), c->stream));
  const double centre = c->general ? c->s01 : c->gamma0;  // the field in d_gamma is s or gamma
  k_abs_dev_max<<<grid_for(c->N, 256), 256, 0, c->stream>>>(c->d_gamma, centre, c->N, d_out);
  count_launch();
  VOFL_CUDA(c, cudaGetLastError());
  unsigned long long bits = 0;
  VOFL_CUDA(c, cudaMemcpyAsync(&bits, d_out, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
  VOFL_CUDA(c, cudaStreamSynchronize(c->stream));
  double dmax;
  std::memcpy(&dmax, &bits, sizeof(dmax));
  const double a = dmax * lmax;
  double term = a * std::exp(2.0 * a);  // the bound for M = 0
  for (int m = 0; m <= M_max; ++m) {
    if (term <= tol) {
      *M = m;
      return VOFL_OK;
    }
    term *= a / (m + 2);
  }
  *M = M_max;
  return VOFL_OK;
}

int model_gamma_from_q(vofl_ctx* c, const double* d_q, double* d_gamma) {
  int* d_bad = reinterpret_cast<int*>(c->d_scratch + RED_BLOCKS + 1);
  VOFL_CUDA(c, cudaMemsetAsync(d_bad, 0, sizeof(int), c->stream));
  k_gamma_from_q<<<grid_for(c->N, 256), 256, 0, c->stream>>>(d_q, d_gamma, c->N, d_bad);
  count_launch();
  VOFL_CUDA(c, cudaGetLastError());
  int bad = 0;
  VOFL_CUDA(c, cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  VOFL_CUDA(c, cudaStreamSynchronize(c->stream));
  if (bad) return set_err(c, VOFL_EINVAL, "Q must be positive and finite at every grid point");
  return VOFL_OK;
}

int model_from_gamma(vofl_ctx* c, const double* d_gamma, const double* d_c0field, double c0, double omega0) {
  int* d_bad = reinterpret_cast<int*>(c->d_scratch + RED_BLOCKS + 1);
  VOFL_CUDA(c, cudaMemsetAsync(d_bad, 0, sizeof(int), c->stream));
  k_check_gamma<<<grid_for(c->N, 256), 256, 0, c->stream>>>(d_gamma, c->N, d_bad);
  k_sum_pass1<<<RED_BLOCKS, RED_THREADS, 0, c->stream>>>(d_gamma, c->N, c->d_scratch);
  k_sum_pass2<<<1, 256, 0, c->stream>>>(c->d_scratch, c->d_scratch + RED_BLOCKS);
  count_launch(3);
  VOFL_CUDA(c, cudaGetLastError());
  double sum = 0;
  int bad = 0;
  VOFL_CUDA(c, cudaMemcpyAsync(&sum, c->d_scratch + RED_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  VOFL_CUDA(c, cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  VOFL_CUDA(c, cudaStreamSynchronize(c->stream));
  if (bad) return set_err(c, VOFL_EINVAL, "gamma must lie in [0, 1/2) at every grid point");
  const double g0 = sum / (double)c->N;
  c->gamma0 = g0;
  c->general = false;
  c->s01 = 1.0 + g0;  // (-Delta)^{1+gamma}
  c->s02 = 0.5 + g0;  // (-Delta)^{1/2+gamma}
  if (c->prec == VOFL_F32) {
    k_coeffs<float><<<grid_for(c->N, 256), 256, 0, c->stream>>>(d_gamma, d_c0field, c0, omega0, g0, c->N,
                                                                 (float*)c->delta, (float*)c->A, (float*)c->B);
  } else {
    k_coeffs<double><<<grid_for(c->N, 256), 256, 0, c->stream>>>(d_gamma, d_c0field, c0, omega0, g0, c->N,
                                                                  (double*)c->delta, (double*)c->A, (double*)c->B);
  }
  count_launch();
  VOFL_CUDA(c, cudaGetLastError());
  return VOFL_OK;
}

// General model: order field s(x) in (0, 2] (kept in c->d_gamma), s0 =
// grid mean; operator 1 is (-Delta)^{s(x)} (centre s0), operator 2 (centre
// s0 - 1/2, same delta) is computed alongside and unused by the update.
int model_from_order(vofl_ctx* c, const double* d_s, double kappa) {
  int* d_bad = reinterpret_cast<int*>(c->d_scratch + RED_BLOCKS + 1);
  VOFL_CUDA(c, cudaMemsetAsync(d_bad, 0, sizeof(int), c->stream));
  k_check_order<<<grid_for(c->N, 256), 256, 0, c->stream>>>(d_s, c->N, d_bad);
  k_sum_pass1<<<RED_BLOCKS, RED_THREADS, 0, c->stream>>>(d_s, c->N, c->d_scratch);
  k_sum_pass2<<<1, 256, 0, c->stream>>>(c->d_scratch, c->d_scratch + RED_BLOCKS);
  count_launch(3);
  VOFL_CUDA(c, cudaGetLastError());
  double sum = 0;
  int bad = 0;
  VOFL_CUDA(c, cudaMemcpyAsync(&sum, c->d_scratch + RED_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  VOFL_CUDA(c, cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  VOFL_CUDA(c, cudaStreamSynchronize(c->stream));
  if (bad) return set_err(c, VOFL_EINVAL, "the order s must lie in (0, 2] at every grid point");
  const double s0 = sum / (double)c->N;
  c->general = true;
  c->gamma0 = s0 - 1.0;
  c->s01 = s0;
  c->s02 = s0 - 0.5;
  c->kappa = kappa;
  if (c->prec == VOFL_F32)
    k_coeffs_general<float><<<grid_for(c->N, 256), 256, 0, c->stream>>>(d_s, s0, kappa, c->N, (float*)c->delta,
                                                                        (float*)c->A, (float*)c->B);
  else
    k_coeffs_general<double><<<grid_for(c->N, 256), 256, 0, c->stream>>>(d_s, s0, kappa, c->N, (double*)c->delta,
                                                                         (double*)c->A, (double*)c->B);
  count_launch();
  VOFL_CUDA(c, cudaGetLastError());
  return VOFL_OK;
}

int make_line_twiddles(int N, float2* d_tw, cudaStream_t s) {
  int nb, r, nm;
  line_twiddle_layout(N, &nb, &r, &nm);
  k_twiddles<<<grid_for((long long)nb * r + nm, 256), 256, 0, s>>>(N, nb, r, nm, d_tw);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? VOFL_OK : VOFL_ECUDA;
}

int model_rel_l2(vofl_ctx* c, const void* x, int x_prec, const void* y, int y_prec, double* out) {
  static_assert(4 * DIAG_BLOCKS + 4 <= 1024, "diagnostics fit the context scratch");
  double* part = c->d_scratch;
  double* d_out = c->d_scratch + 4 * DIAG_BLOCKS;
  const long long n = c->N;
  if (x_prec == VOFL_F32 && y_prec == VOFL_F32)
    k_diff_pass1<float, float><<<DIAG_BLOCKS, RED_THREADS, 0, c->stream>>>((const float*)x, (const float*)y, n, part);
  else if (x_prec == VOFL_F32)
    k_diff_pass1<float, double><<<DIAG_BLOCKS, RED_THREADS, 0, c->stream>>>((const float*)x, (const double*)y, n, part);
  else if (y_prec == VOFL_F32)
    k_diff_pass1<double, float><<<DIAG_BLOCKS, RED_THREADS, 0, c->stream>>>((const double*)x, (const float*)y, n, part);
  else
    k_diff_pass1<double, double><<<DIAG_BLOCKS, RED_THREADS, 0, c->stream>>>((const double*)x, (const double*)y, n, part);
  k_diff_pass2<<<1, 256, 0, c->stream>>>(part, d_out);
  count_launch(2);
  VOFL_CUDA(c, cudaGetLastError());
  VOFL_CUDA(c, cudaMemcpyAsync(out, d_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  VOFL_CUDA(c, cudaStreamSynchronize(c->stream));
  return VOFL_OK;
}

int make_wide_twiddles(int N, float2* d_tw, cudaStream_t s) {
  if (N != 512 && N != 1024) return VOFL_EINVAL;
  k_twiddles_wide<<<grid_for(wide_twiddle_entries(N), 256), 256, 0, s>>>(N, d_tw);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? VOFL_OK : VOFL_ECUDA;
}

int make_tile_map(CUtensorMap* map, const void* base, int ncols, long long rows, int pitch, int box_cols,
                  int box_rows) {
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return VOFL_ECUDA;
    encode = reinterpret_cast<Encode>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)ncols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch * 8};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(base), dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? VOFL_OK : VOFL_ECUDA;
}

int make_fused2d_tables(int nx, int ny, double lx, double ly, double s01, double s02, double scale2, double ryy,
                        float* P, float* Lg, cudaStream_t s) {
  const long long total = (long long)(nx / 2 + 1) * ny;
  k_tables_fused2d<<<grid_for(total, 256), 256, 0, s>>>(nx, ny, lx, ly, s01, s02, scale2, ryy, P, Lg);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? VOFL_OK : VOFL_ECUDA;
}

__global__ void k_omega_fused2d(int nx, int ny, double lx, double ly, double s0, double kappa, float* __restrict__ W) {
  const long long total = (long long)(nx / 2 + 1) * ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / ny), k2 = (int)(i % ny);
    const int k2s = (k2 < ny / 2) ? k2 : k2 - ny;
    const double m1 = 2.0 * M_PI * (double)c / lx, m2 = 2.0 * M_PI * (double)k2s / ly;
    const double mu2 = m1 * m1 + m2 * m2;
    W[i] = (float)(mu2 > 0.0 ? sqrt(kappa) * pow(mu2, 0.5 * s0) : 0.0);
  }
}

int make_fused2d_omega(int nx, int ny, double lx, double ly, double s0, double kappa, float* W, cudaStream_t s) {
  const long long total = (long long)(nx / 2 + 1) * ny;
  k_omega_fused2d<<<grid_for(total, 256), 256, 0, s>>>(nx, ny, lx, ly, s0, kappa, W);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? VOFL_OK : VOFL_ECUDA;
}

template <typename T>
int make_plain_tables(int ndim, const int64_t* n, const double* lo, const double* hi, double s01, double s02, T* P1,
                      T* P2, T* Lg, cudaStream_t s) {
  const int nx = (int)n[0];
  const int ny = ndim > 1 ? (int)n[1] : 1;
  const int nz = ndim > 2 ? (int)n[2] : 1;
  const double lx = hi[0] - lo[0];
  const double ly = ndim > 1 ? hi[1] - lo[1] : 1.0;
  const double lz = ndim > 2 ? hi[2] - lo[2] : 1.0;
  const double invN = 1.0 / ((double)nx * ny * nz);
  const long long total = (long long)(nx / 2 + 1) * ny * nz;
  const double hx = lx / nx, hy = ly / ny, hz = lz / nz;
  const double ry = ndim > 1 ? (hx * hx) / (hy * hy) : 0.0;
  const double rz = ndim > 2 ? (hx * hx) / (hz * hz) : 0.0;
  k_tables_plain<T><<<grid_for(total, 256), 256, 0, s>>>(nx, ny, nz, lx, ly, lz, s01, s02, invN, ry, rz, P1, P2, Lg);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? VOFL_OK : VOFL_ECUDA;
}

template int make_plain_tables<float>(int, const int64_t*, const double*, const double*, double, double, float*,
                                      float*, float*, cudaStream_t);
template int make_plain_tables<double>(int, const int64_t*, const double*, const double*, double, double, double*,
                                       double*, double*, cudaStream_t);

}  // namespace vofl
