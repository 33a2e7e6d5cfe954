// plain.cu -- the plain baseline: the same arithmetic as the fused path
// (Eq. (2.13) of arXiv 2311.13049 for both operators of Eq. (1.1), then the
// leap-frog update of Eq. (3.4)) with library transforms (cuFFT R2C / C2R)
// and separate elementwise kernels, every intermediate field in memory:
//   stencil: w = discrete Laplacian of u                         (kernel)
//   forward R2C of w                                             (cuFFT)
//   multiply: X[op][m] = w_hat * P_op(k) (ln|mu_k|^2)^m / m!,
//             all terms of both operators                        (kernel)
//   inverse C2R of all 2(M+1) spectra in one batched call        (cuFFT)
//   accumulate: acc_op = sum_m (s(x) - s0)^m Y[op][m], Horner     (kernel)
//   pointwise update                                             (kernel)
// Works for 1D, 2D, 3D and for float or double.  It keeps all 2(M+1)
// transformed fields in memory (O(MN) storage and traffic); that is what
// the fused path removes.
// For the general model it also runs the second-order time splitting of
// Sec. 3.3 (step_split): exact half-step rotations of (u_hat, v_hat) in
// Fourier space, the variable-order kick (terms m >= 1), the rotations
// again; and the Crank-Nicolson scheme of Sec. 3.1 (step_cn, below).
#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>
#include <string>

#include "internal.h"

namespace vofl {

namespace {

template <typename T>
struct CT;
template <>
struct CT<float> {
  using C = cufftComplex;
};
template <>
struct CT<double> {
  using C = cufftDoubleComplex;
};

inline int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 8192) b = 8192;
  return (int)(b < 1 ? 1 : b);
}
// 64-thread blocks: short lines (a 1D spectrum of 2049 bins) still spread
// over many SMs, which matters for FP64 arithmetic (~8 GFLOP/s per SM)
constexpr int kSmallBlock = 64;
inline int grid_small(long long n) {
  long long b = (n + kSmallBlock - 1) / kSmallBlock;
  if (b > 32768) b = 32768;
  return (int)(b < 1 ? 1 : b);
}

// 1/k for k = 0..41 (entry 0 unused): the Taylor recurrences multiply by
// these instead of dividing (a division costs tens of FP64 operations)
#define VOFL_R4(k) 1.0 / (k), 1.0 / ((k) + 1), 1.0 / ((k) + 2), 1.0 / ((k) + 3)
__constant__ double c_rcp[44] = {0.0, 1.0, 0.5, 1.0 / 3, VOFL_R4(4), VOFL_R4(8), VOFL_R4(12), VOFL_R4(16),
                                 VOFL_R4(20), VOFL_R4(24), VOFL_R4(28), VOFL_R4(32), VOFL_R4(36), VOFL_R4(40)};
#undef VOFL_R4

// Time splitting (Sec. 3.3): the exact flow of u_t = v, v_t = -kappa
// (-Delta)^{s0} u over time t, mode by mode on the R2C half spectra of u
// and v (unnormalised transforms: the 1/N goes in here); w_k = sqrt(kappa)
// |mu_k|^{s0}, and the k = 0 mode drifts (u += t v).
template <typename T, typename C>
__global__ void k_rotate(C* __restrict__ uh, C* __restrict__ vh, const T* __restrict__ W, T t, T invN,
                         long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const T w = W[i];
    const C a = uh[i], b = vh[i];
    C a2, b2;
    if (w > T(0)) {
      T sn, cs;
      if constexpr (sizeof(T) == 8)
        sincos(w * t, &sn, &cs);
      else
        sincosf(w * t, &sn, &cs);
      const T q = sn / w;
      a2.x = a.x * cs + b.x * q;
      a2.y = a.y * cs + b.y * q;
      b2.x = b.x * cs - a.x * w * sn;
      b2.y = b.y * cs - a.y * w * sn;
    } else {
      a2.x = a.x + t * b.x;
      a2.y = a.y + t * b.y;
      b2 = b;
    }
    a2.x *= invN;
    a2.y *= invN;
    b2.x *= invN;
    b2.y *= invN;
    uh[i] = a2;
    vh[i] = b2;
  }
}

// w_k = sqrt(kappa) |mu_k|^{s0} on the R2C layout [nz][ny][nx/2+1] (double, rounded once)
template <typename T>
__global__ void k_omega_table(int nx, int ny, int nz, double lx, double ly, double lz, double s0, double kappa,
                              T* __restrict__ W) {
  const int H = nx / 2 + 1;
  const long long n = (long long)H * ny * nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(i % H);
    const int ky0 = (int)((i / H) % ny), kz0 = (int)(i / ((long long)H * ny));
    const int ky = ky0 < ny / 2 ? ky0 : ky0 - ny, kz = kz0 < nz / 2 ? kz0 : kz0 - nz;
    const double m1 = 2.0 * M_PI * kx / lx, m2 = 2.0 * M_PI * ky / ly, m3 = 2.0 * M_PI * kz / lz;
    const double mu2 = m1 * m1 + (ny > 1 ? m2 * m2 : 0.0) + (nz > 1 ? m3 * m3 : 0.0);
    W[i] = T(mu2 > 0.0 ? sqrt(kappa) * pow(mu2, 0.5 * s0) : 0.0);
  }
}

// the kick of the splitting: v += dt (-kappa D u + f1 u + f3 u^3), D u the
// variable-order remainder sum_{m >= 1} delta^m Y_m
template <typename T>
__global__ void k_kick(T* __restrict__ v, const T* __restrict__ Du, const T* __restrict__ u, T dt, T kappa, T f1,
                       T f3, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const T x = u[i];
    v[i] += dt * (-kappa * Du[i] + f1 * x + f3 * x * x * x);
  }
}

__global__ void k_inc(int* p) { *p += 1; }

// w = D_xx u + ry D_yy u + rz D_zz u (periodic second differences without
// 1/h^2, ry = (h_x/h_y)^2, rz = (h_x/h_z)^2).  The forward transform is taken
// of w; the multiplier tables carry 1/lambda_k (see model.cu).
template <typename T>
__global__ void k_laplacian(const T* __restrict__ u, T* __restrict__ w, int nx, int ny, int nz, T ry, T rz) {
  const long long n = (long long)nx * ny * nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx);
    const int y = (int)((i / nx) % ny);
    const int z = (int)(i / ((long long)nx * ny));
    const T c = u[i];
    const long long row = i - x;
    T acc = (u[row + (x + 1 == nx ? 0 : x + 1)] - c) - (c - u[row + (x == 0 ? nx - 1 : x - 1)]);
    if (ny > 1) {
      const long long pl = (long long)nx * ny * z + x;
      const T d = (u[pl + (long long)nx * (y + 1 == ny ? 0 : y + 1)] - c) - (c - u[pl + (long long)nx * (y == 0 ? ny - 1 : y - 1)]);
      acc = acc + ry * d;
    }
    if (nz > 1) {
      const long long col = (long long)nx * y + x;
      const long long pln = (long long)nx * ny;
      const T d = (u[col + pln * (z + 1 == nz ? 0 : z + 1)] - c) - (c - u[col + pln * (z == 0 ? nz - 1 : z - 1)]);
      acc = acc + rz * d;
    }
    w[i] = acc;
  }
}

template <typename T>
__global__ void k_update(const T* __restrict__ L1, const T* __restrict__ L2, EpiArgs<T> e, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    epilogue_point<T>(e, i, L1[i], L2[i]);
}

// ---------------------------------------------------------------------------
// Crank-Nicolson scheme (CNFP, Sec. 3.1, Eq. (3.2)) of the general model.
// With c = kappa dt^2/2 and h2 = dt^2/2 each step solves
//     A v - h2 f(v) = b,  A = I + c L,
//     b = 2 u^n - u^{n-1} - c L u^{n-1} + h2 f(u^{n-1}),
// for v = u^{n+1}, L the matrix-free operator of Eq. (2.13).  L is not
// symmetric when s varies in x, so the conjugate gradients run on the normal
// equations (CGNR): A^T A d = A^T r.  The cubic term is handled by a
// fixed-point (Picard) outer loop: r = b + h2 f(v) - A v is the residual of
// the nonlinear system, and each outer pass solves A d = r by CGNR and sets
// v += d, until |r| <= tol |b + h2 f(v)|.
//   L v   = sum_m delta^m IFFT[P l^m/m! FFT(Lap v)]         (M+1 inverse
//           transforms in one batched cuFFT call; l = ln|mu|^2)
//   L^T r = IFFT[P sum_m l^m/m! FFT(Lap(delta^m r))]       (M+1 forward
//           transforms in one batched call; the circulant factors are
//           symmetric, so the transpose only moves delta^m to the front)
// Dot products are two-pass (fixed block partials, then one block in fixed
// order) so that runs are bitwise reproducible; CG scalars stay on the
// device and the host reads them once per chunk of iterations.
constexpr int CN_THREADS = 256;
constexpr int CN_MAXG = 304;  // partial blocks of a dot product (two per SM)
enum CnSlot { S_ZZ = 0, S_WW, S_RR, S_GG, S_ALPHA, S_BETA, S_STOP, S_ITERS, S_THR2, S_COUNT };
enum CnFin { FIN_RRGG = 0, FIN_ZZ0, FIN_WW, FIN_RR, FIN_ZZ };

inline int cn_grid(long long n) {
  long long b = (n + CN_THREADS - 1) / CN_THREADS;
  if (b > CN_MAXG) b = CN_MAXG;
  return (int)(b < 1 ? 1 : b);
}

// sum over the block (blockDim.x == CN_THREADS) of a and b; valid in thread 0
__device__ __forceinline__ void cn_block_sum2(double& a, double& b) {
  __shared__ double wa[CN_THREADS / 32], wb[CN_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    wa[wid] = a;
    wb[wid] = b;
  }
  __syncthreads();
  if (wid == 0) {
    a = lane < CN_THREADS / 32 ? wa[lane] : 0.0;
    b = lane < CN_THREADS / 32 ? wb[lane] : 0.0;
    for (int o = (CN_THREADS / 32) / 2; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
  }
}

// the multiplied spectra of both operators: X[op][m] = u_hat P_op L^m / m!
template <typename T, typename C>
__global__ void k_mult_ops(const C* __restrict__ uh, const T* __restrict__ P1, const T* __restrict__ P2,
                           const T* __restrict__ Lg, int M, int nops, C* __restrict__ X, long long nh) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nh; i += (long long)gridDim.x * blockDim.x) {
    const T l = Lg[i];
    const C v = uh[i];
    for (int op = 0; op < nops; ++op) {
      T t = op == 0 ? P1[i] : P2[i];
      C* out = X + (long long)op * (M + 1) * nh + i;
      for (int m = 0; m <= M; ++m) {
        C o;
        o.x = v.x * t;
        o.y = v.y * t;
        out[m * nh] = o;
        t = t * l * T(c_rcp[m + 1]);
      }
    }
  }
}

// acc_op = sum_{m = m0..M} delta^m Y[op][m] for op < nops (Horner, then
// delta^m0); zero when m0 > M
template <typename T>
__global__ void k_acc_ops(const T* __restrict__ Y, const T* __restrict__ delta, int M, int m0, int nops,
                          T* __restrict__ acc1, T* __restrict__ acc2, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const T d = delta[i];
    for (int op = 0; op < nops; ++op) {
      const T* y = Y + (long long)op * (M + 1) * n + i;
      T acc = T(0);
      if (m0 <= M) {
        acc = y[M * n];
        for (int m = M - 1; m >= m0; --m) acc = y[m * n] + d * acc;
        for (int m = 0; m < m0; ++m) acc *= d;
      }
      (op == 0 ? acc1 : acc2)[i] = acc;
    }
  }
}

// out = cv v + cA sum_m delta^m Ym[m] (Horner); optional partials of |out|^2
template <typename T>
__global__ void __launch_bounds__(CN_THREADS)
    k_cn_horner(const T* __restrict__ Ym, const T* __restrict__ delta, int M, const T* __restrict__ v, T cv, T cA,
                T* __restrict__ out, double* __restrict__ part, long long n) {
  double s = 0.0, dummy = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const T d = delta[i];
    T acc = Ym[M * n + i];
    for (int m = M - 1; m >= 0; --m) acc = Ym[m * n + i] + d * acc;
    const T o = (v ? cv * v[i] : T(0)) + cA * acc;
    out[i] = o;
    s += (double)o * (double)o;
  }
  if (part) {
    cn_block_sum2(s, dummy);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

// Ym[m] = Lap(delta^m r), m = 0..M (the stencil of k_laplacian)
template <typename T>
__global__ void k_cn_pow_lap(const T* __restrict__ r, const T* __restrict__ delta, int M, T* __restrict__ Ym, int nx,
                             int ny, int nz, T ry, T rz) {
  const long long n = (long long)nx * ny * nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx);
    const int y = (int)((i / nx) % ny);
    const int z = (int)(i / ((long long)nx * ny));
    const long long row = i - x;
    const long long ixp = row + (x + 1 == nx ? 0 : x + 1), ixm = row + (x == 0 ? nx - 1 : x - 1);
    const long long pl = (long long)nx * ny * z + x;
    const long long iyp = pl + (long long)nx * (y + 1 == ny ? 0 : y + 1), iym = pl + (long long)nx * (y == 0 ? ny - 1 : y - 1);
    const long long col = (long long)nx * y + x, pln = (long long)nx * ny;
    const long long izp = col + pln * (z + 1 == nz ? 0 : z + 1), izm = col + pln * (z == 0 ? nz - 1 : z - 1);
    T qc = r[i], qxp = r[ixp], qxm = r[ixm];
    const T dc = delta[i], dxp = delta[ixp], dxm = delta[ixm];
    T qyp = T(0), qym = T(0), qzp = T(0), qzm = T(0), dyp = T(0), dym = T(0), dzp = T(0), dzm = T(0);
    if (ny > 1) {
      qyp = r[iyp];
      qym = r[iym];
      dyp = delta[iyp];
      dym = delta[iym];
    }
    if (nz > 1) {
      qzp = r[izp];
      qzm = r[izm];
      dzp = delta[izp];
      dzm = delta[izm];
    }
    for (int m = 0; m <= M; ++m) {
      T acc = (qxp - qc) - (qc - qxm);
      if (ny > 1) acc = acc + ry * ((qyp - qc) - (qc - qym));
      if (nz > 1) acc = acc + rz * ((qzp - qc) - (qc - qzm));
      Ym[m * n + i] = acc;
      qc *= dc;
      qxp *= dxp;
      qxm *= dxm;
      qyp *= dyp;
      qym *= dym;
      qzp *= dzp;
      qzm *= dzm;
    }
  }
}

// X = P sum_m L^m/m! Xm[m] (Horner in L)
template <typename T, typename C>
__global__ void k_cn_tsum(const C* __restrict__ Xm, const T* __restrict__ P, const T* __restrict__ Lg, int M,
                          C* __restrict__ X, long long nh) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nh; i += (long long)gridDim.x * blockDim.x) {
    const T l = Lg[i];
    C acc = Xm[M * nh + i];
    for (int m = M - 1; m >= 0; --m) {
      const T q = l * T(c_rcp[m + 1]);
      const C w = Xm[m * nh + i];
      acc.x = w.x + q * acc.x;
      acc.y = w.y + q * acc.y;
    }
    const T p = P[i];
    acc.x *= p;
    acc.y *= p;
    X[i] = acc;
  }
}

// b = 2 u^n - u^{n-1} - c L u^{n-1} + h2 f(u^{n-1}), and the first iterate
// x = 2 u^n - u^{n-1}
template <typename T>
__global__ void k_cn_rhs(const T* __restrict__ un, const T* __restrict__ uo, const T* __restrict__ Lp, T c, T h2, T f1,
                         T f3, T* __restrict__ b, T* __restrict__ x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const T p = uo[i], u = un[i];
    const T ext = T(2) * u - p;
    b[i] = ext - c * Lp[i] + h2 * (f1 * p + f3 * p * p * p);
    x[i] = ext;
  }
}

// r = b + h2 f(x) - A x (w = A x); partials of |r|^2 and |b + h2 f(x)|^2
template <typename T>
__global__ void __launch_bounds__(CN_THREADS)
    k_cn_resid(const T* __restrict__ b, const T* __restrict__ x, const T* __restrict__ w, T h2, T f1, T f3,
               T* __restrict__ r, double* __restrict__ pa, double* __restrict__ pb, long long n) {
  double sr = 0.0, sg = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const T xx = x[i];
    const T g = b[i] + h2 * (f1 * xx + f3 * xx * xx * xx);
    const T rr = g - w[i];
    r[i] = rr;
    sr += (double)rr * (double)rr;
    sg += (double)g * (double)g;
  }
  cn_block_sum2(sr, sg);
  if (threadIdx.x == 0) {
    pa[blockIdx.x] = sr;
    pb[blockIdx.x] = sg;
  }
}

// z = r + c LT r (= A^T r); with `p` set also p = z; partials of |z|^2
template <typename T>
__global__ void __launch_bounds__(CN_THREADS)
    k_cn_z(const T* __restrict__ r, const T* __restrict__ LTr, T c, T* __restrict__ z, T* __restrict__ p,
           double* __restrict__ pa, long long n) {
  double s = 0.0, dummy = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const T v = r[i] + c * LTr[i];
    z[i] = v;
    if (p) p[i] = v;
    s += (double)v * (double)v;
  }
  cn_block_sum2(s, dummy);
  if (threadIdx.x == 0) pa[blockIdx.x] = s;
}

// x += alpha p, r -= alpha w (unless stopped); partials of |r|^2
template <typename T>
__global__ void __launch_bounds__(CN_THREADS)
    k_cn_xr(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p, const T* __restrict__ w,
            const double* __restrict__ s, double* __restrict__ pa, long long n) {
  const bool go = s[S_STOP] == 0.0;
  const T a = T(s[S_ALPHA]);
  double acc = 0.0, dummy = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    T rr = r[i];
    if (go) {
      x[i] += a * p[i];
      rr -= a * w[i];
      r[i] = rr;
    }
    acc += (double)rr * (double)rr;
  }
  cn_block_sum2(acc, dummy);
  if (threadIdx.x == 0) pa[blockIdx.x] = acc;
}

// p = z + beta p (unless stopped)
template <typename T>
__global__ void k_cn_p(const T* __restrict__ z, T* __restrict__ p, const double* __restrict__ s, long long n) {
  if (s[S_STOP] != 0.0) return;
  const T be = T(s[S_BETA]);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = z[i] + be * p[i];
}

// finish a dot product (partials summed in a fixed order) and update the
// CG scalars; tol2 = (inner tolerance)^2 for FIN_RRGG
__global__ void __launch_bounds__(CN_THREADS)
    k_cn_fin(int op, const double* __restrict__ pa, const double* __restrict__ pb, int G, double tol2,
             double* __restrict__ s) {
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < G; i += CN_THREADS) {
    a += pa[i];
    if (pb) b += pb[i];
  }
  cn_block_sum2(a, b);
  if (threadIdx.x != 0) return;
  switch (op) {
    case FIN_RRGG:
      s[S_RR] = a;
      s[S_GG] = b;
      s[S_THR2] = tol2 * b;
      break;
    case FIN_ZZ0:
      s[S_ZZ] = a;
      s[S_STOP] = (a == 0.0 || s[S_RR] <= s[S_THR2]) ? 1.0 : 0.0;
      break;
    case FIN_WW:
      s[S_WW] = a;
      if (s[S_STOP] == 0.0) {
        if (a > 0.0) {
          s[S_ALPHA] = s[S_ZZ] / a;
          s[S_ITERS] += 1.0;
        } else {
          s[S_STOP] = 1.0;
        }
      }
      break;
    case FIN_RR:
      s[S_RR] = a;
      if (s[S_STOP] == 0.0 && a <= s[S_THR2]) s[S_STOP] = 1.0;
      break;
    case FIN_ZZ:
      if (s[S_STOP] == 0.0) {
        if (s[S_ZZ] > 0.0) {
          s[S_BETA] = a / s[S_ZZ];
          s[S_ZZ] = a;
        } else {
          s[S_STOP] = 1.0;
        }
      }
      break;
  }
}

template <typename T>
struct Plain : Engine {
  using C = typename CT<T>::C;
  int ndim = 0;
  long long N = 0, Nh = 0;  // real points, half-spectrum points
  cufftHandle fwd = 0, inv = 0;
  bool have_fwd = false, have_inv = false;
  C* uh = nullptr;
  C* X = nullptr;
  T* Y = nullptr;
  T* acc1 = nullptr;
  T* acc2 = nullptr;
  T* P1 = nullptr;
  T* P2 = nullptr;
  T* Lg = nullptr;
  T* W = nullptr;  // splitting: sqrt(kappa) |mu|^{s0} (general model)
  C* vh = nullptr;
  size_t nbytes = 0;

  // all Taylor terms of both operators (sized by M in prepare(), before any
  // graph capture: plans and allocations are not stream operations)
  struct Terms {
    int M = -1;
    int gen = 0;                              // bumped on every re-allocation
    cufftHandle fwd1 = 0, inv1 = 0, inv2 = 0;  // M+1 R2C, M+1 C2R, 2(M+1) C2R
    bool have = false;
    C* X = nullptr;  // [2][M+1][Nh]
    T* Y = nullptr;  // [2][M+1][N]
    size_t bytes = 0;
  } tb;

  // Crank-Nicolson solver state (allocated on first use)
  struct Cn {
    int gen = -1;  // term-batch generation the graphs were captured with
    T *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *w = nullptr;
    double *pa = nullptr, *pb = nullptr, *s = nullptr;
    double* hs = nullptr;  // pinned copy of s
    size_t bytes = 0;
    cudaGraphExec_t g_rhs[2] = {nullptr, nullptr}, g_resid = nullptr, g_init = nullptr, g_chunk = nullptr;
    uint64_t n_rhs = 0, n_resid = 0, n_init = 0, n_chunk = 0;
    bool graphs_ok = true;
    // what the graphs bake in
    double key_dt = -1, key_kappa = 0, key_f1 = 0, key_f3 = 0, key_tol = -1;
  } cn;
  static constexpr int kCnChunk = 4;   // CG iterations per host check
  static constexpr int kCnOuter = 50;  // fixed-point passes per step

  void cn_drop_graphs() {
    for (cudaGraphExec_t* g : {&cn.g_rhs[0], &cn.g_rhs[1], &cn.g_resid, &cn.g_init, &cn.g_chunk}) {
      if (*g) cudaGraphExecDestroy(*g);
      *g = nullptr;
    }
  }
  void cn_free() {
    cn_drop_graphs();
    for (void* q : {(void*)cn.b, (void*)cn.x, (void*)cn.r, (void*)cn.z, (void*)cn.p, (void*)cn.w, (void*)cn.pa,
                    (void*)cn.pb, (void*)cn.s})
      dev_free(q);
    if (cn.hs) cudaFreeHost(cn.hs);
    nbytes -= cn.bytes;
    cn = Cn{};
  }
  void tb_free() {
    if (tb.have) {
      cufftDestroy(tb.fwd1);
      cufftDestroy(tb.inv1);
      cufftDestroy(tb.inv2);
    }
    dev_free(tb.X);
    dev_free(tb.Y);
    nbytes -= tb.bytes;
    const int gen = tb.gen;
    tb = Terms{};
    tb.gen = gen + 1;
  }

  ~Plain() override {
    cn_free();
    tb_free();
    if (have_fwd) cufftDestroy(fwd);
    if (have_inv) cufftDestroy(inv);
    dev_free(uh);
    dev_free(X);
    dev_free(Y);
    dev_free(acc1);
    dev_free(acc2);
    dev_free(P1);
    dev_free(P2);
    dev_free(Lg);
    dev_free(W);
    dev_free(vh);
  }
  size_t bytes() const override { return nbytes; }

  int alloc(vofl_ctx* c, void** p, size_t b) {
    cudaError_t e = dev_malloc(p, b);
    if (e != cudaSuccess) return cuda_err(c, e, "cudaMalloc (plain scratch)");
    nbytes += b;
    return VOFL_OK;
  }

  int init(vofl_ctx* c) {
    ndim = c->ndim;
    N = c->N;
    Nh = (c->n[0] / 2 + 1) * (N / c->n[0]);
    int dims[3];
    for (int i = 0; i < ndim; ++i) dims[i] = (int)c->n[ndim - 1 - i];  // slowest first
    const bool dbl = sizeof(T) == 8;
    if (cufftPlanMany(&fwd, ndim, dims, nullptr, 1, 0, nullptr, 1, 0, dbl ? CUFFT_D2Z : CUFFT_R2C, 1) !=
        CUFFT_SUCCESS)
      return set_err(c, VOFL_ECUDA, "cufftPlanMany (forward)");
    have_fwd = true;
    if (cufftPlanMany(&inv, ndim, dims, nullptr, 1, 0, nullptr, 1, 0, dbl ? CUFFT_Z2D : CUFFT_C2R, 1) !=
        CUFFT_SUCCESS)
      return set_err(c, VOFL_ECUDA, "cufftPlanMany (inverse)");
    have_inv = true;
    cufftSetStream(fwd, c->stream);
    cufftSetStream(inv, c->stream);
    int st;
    if ((st = alloc(c, (void**)&uh, sizeof(C) * Nh))) return st;
    if ((st = alloc(c, (void**)&X, sizeof(C) * Nh))) return st;
    if ((st = alloc(c, (void**)&Y, sizeof(T) * N))) return st;
    if ((st = alloc(c, (void**)&acc1, sizeof(T) * N))) return st;
    if ((st = alloc(c, (void**)&acc2, sizeof(T) * N))) return st;
    if ((st = alloc(c, (void**)&P1, sizeof(T) * Nh))) return st;
    if ((st = alloc(c, (void**)&P2, sizeof(T) * Nh))) return st;
    if ((st = alloc(c, (void**)&Lg, sizeof(T) * Nh))) return st;
    if ((st = alloc(c, (void**)&W, sizeof(T) * Nh))) return st;
    if ((st = alloc(c, (void**)&vh, sizeof(C) * Nh))) return st;
    return VOFL_OK;
  }

  int set_model(vofl_ctx* c) override {
    if (make_plain_tables<T>(c->ndim, c->n, c->lo, c->hi, c->s01, c->s02, P1, P2, Lg, c->stream))
      return cuda_err(c, cudaGetLastError(), "plain tables");
    if (c->general) {
      const int nx = (int)c->n[0], ny = c->ndim > 1 ? (int)c->n[1] : 1, nz = c->ndim > 2 ? (int)c->n[2] : 1;
      const double lx = c->hi[0] - c->lo[0], ly = c->ndim > 1 ? c->hi[1] - c->lo[1] : 1.0;
      const double lz = c->ndim > 2 ? c->hi[2] - c->lo[2] : 1.0;
      k_omega_table<T><<<grid_for(Nh), 256, 0, c->stream>>>(nx, ny, nz, lx, ly, lz, c->s01, c->kappa, W);
      count_launch();
      if (cudaGetLastError() != cudaSuccess) return set_err(c, VOFL_ECUDA, "splitting frequency table");
    }
    return VOFL_OK;
  }

  uint64_t kernels_per_step(const vofl_ctx* c) const override {
    (void)c;
    // our own kernels only (cuFFT's are library launches): step counter,
    // stencil, multiply, accumulate, update
    return 5;
  }

  // size the term batch for the context's M
  int prepare(vofl_ctx* c) override {
    if (tb.M == c->M) return VOFL_OK;
    VOFL_CUDA(c, cudaStreamSynchronize(c->stream));  // queued work may still use the old buffers
    tb_free();
    const int B = c->M + 1;
    int dims[3];
    for (int i = 0; i < ndim; ++i) dims[i] = (int)c->n[ndim - 1 - i];
    const bool dbl = sizeof(T) == 8;
    if (cufftPlanMany(&tb.fwd1, ndim, dims, nullptr, 1, 0, nullptr, 1, 0, dbl ? CUFFT_D2Z : CUFFT_R2C, B) !=
        CUFFT_SUCCESS)
      return set_err(c, VOFL_ECUDA, "cufftPlanMany (batched forward)");
    if (cufftPlanMany(&tb.inv1, ndim, dims, nullptr, 1, 0, nullptr, 1, 0, dbl ? CUFFT_Z2D : CUFFT_C2R, B) !=
        CUFFT_SUCCESS) {
      cufftDestroy(tb.fwd1);
      return set_err(c, VOFL_ECUDA, "cufftPlanMany (batched inverse)");
    }
    if (cufftPlanMany(&tb.inv2, ndim, dims, nullptr, 1, 0, nullptr, 1, 0, dbl ? CUFFT_Z2D : CUFFT_C2R, 2 * B) !=
        CUFFT_SUCCESS) {
      cufftDestroy(tb.fwd1);
      cufftDestroy(tb.inv1);
      return set_err(c, VOFL_ECUDA, "cufftPlanMany (batched inverse, two operators)");
    }
    tb.have = true;
    cufftSetStream(tb.fwd1, c->stream);
    cufftSetStream(tb.inv1, c->stream);
    cufftSetStream(tb.inv2, c->stream);
    cudaError_t e = dev_malloc(&tb.X, sizeof(C) * Nh * 2 * B);
    if (e == cudaSuccess) e = dev_malloc(&tb.Y, sizeof(T) * N * 2 * B);
    if (e != cudaSuccess) {
      tb_free();  // plans and whatever was allocated; the next call starts afresh
      return cuda_err(c, e, "cudaMalloc (plain term batch)");
    }
    tb.bytes = (sizeof(C) * Nh + sizeof(T) * N) * 2 * B;
    nbytes += tb.bytes;
    tb.M = c->M;
    return VOFL_OK;
  }

  int exec_fwd(vofl_ctx* c, const T* u) {
    cufftResult r;
    if constexpr (sizeof(T) == 8)
      r = cufftExecD2Z(fwd, (cufftDoubleReal*)const_cast<T*>(u), (cufftDoubleComplex*)uh);
    else
      r = cufftExecR2C(fwd, (cufftReal*)const_cast<T*>(u), (cufftComplex*)uh);
    if (r != CUFFT_SUCCESS) return set_err(c, VOFL_ECUDA, "cuFFT forward");
    return VOFL_OK;
  }
  int exec_inv(vofl_ctx* c, C* in = nullptr, T* out = nullptr) {
    cufftResult r;
    if (!in) in = X;
    if (!out) out = Y;
    if constexpr (sizeof(T) == 8)
      r = cufftExecZ2D(inv, (cufftDoubleComplex*)in, (cufftDoubleReal*)out);
    else
      r = cufftExecC2R(inv, (cufftComplex*)in, (cufftReal*)out);
    if (r != CUFFT_SUCCESS) return set_err(c, VOFL_ECUDA, "cuFFT inverse");
    return VOFL_OK;
  }
  int exec_fwd_to(vofl_ctx* c, const T* u, C* out) {
    cufftResult r;
    if constexpr (sizeof(T) == 8)
      r = cufftExecD2Z(fwd, (cufftDoubleReal*)const_cast<T*>(u), (cufftDoubleComplex*)out);
    else
      r = cufftExecR2C(fwd, (cufftReal*)const_cast<T*>(u), (cufftComplex*)out);
    if (r != CUFFT_SUCCESS) return set_err(c, VOFL_ECUDA, "cuFFT forward");
    return VOFL_OK;
  }

  // sums of Eq. (2.13) for terms m0..M of the first nops operators into
  // acc1 (, acc2): one forward transform, every term's inverse transform in
  // one batched call
  int operators(vofl_ctx* c, const T* u, int m0 = 0, int nops = 2) {
    if (tb.M != c->M) return set_err(c, VOFL_ESTATE, "plain path: term batch not prepared for this M");
    int st;
    // forward transform of the discrete Laplacian of u (into Y, free here)
    const int nx = (int)c->n[0], ny = c->ndim > 1 ? (int)c->n[1] : 1, nz = c->ndim > 2 ? (int)c->n[2] : 1;
    k_laplacian<T><<<grid_for(N), 256, 0, c->stream>>>(u, Y, nx, ny, nz, ryy(c), rzz(c));
    count_launch();
    if ((st = exec_fwd(c, Y))) return st;
    k_mult_ops<T, C><<<grid_small(Nh), kSmallBlock, 0, c->stream>>>(uh, P1, P2, Lg, c->M, nops, tb.X, Nh);
    count_launch();
    cufftResult r;
    const cufftHandle plan = nops == 2 ? tb.inv2 : tb.inv1;
    if constexpr (sizeof(T) == 8)
      r = cufftExecZ2D(plan, (cufftDoubleComplex*)tb.X, (cufftDoubleReal*)tb.Y);
    else
      r = cufftExecC2R(plan, (cufftComplex*)tb.X, (cufftReal*)tb.Y);
    if (r != CUFFT_SUCCESS) return set_err(c, VOFL_ECUDA, "cuFFT batched inverse");
    k_acc_ops<T><<<grid_small(N), kSmallBlock, 0, c->stream>>>(tb.Y, (const T*)c->delta, c->M, m0, nops, acc1, acc2, N);
    count_launch();
    return VOFL_OK;
  }

  bool can_split() const override { return true; }

  // one step of the second-order time splitting (Sec. 3.3) of the general
  // model: u = u[cur], v = u[1 - cur], both updated in place
  int step_split(vofl_ctx* c) override {
    T* u = (T*)c->u[c->cur];
    T* v = (T*)c->u[1 - c->cur];
    const T half = T(0.5 * c->dt), invN = T(1.0 / (double)N);
    auto rotate = [&]() -> int {
      int st;
      if ((st = exec_fwd_to(c, u, uh))) return st;
      if ((st = exec_fwd_to(c, v, vh))) return st;
      k_rotate<T, C><<<grid_for(Nh), 256, 0, c->stream>>>(uh, vh, W, half, invN, Nh);
      count_launch();
      if ((st = exec_inv(c, uh, u))) return st;
      return exec_inv(c, vh, v);
    };
    int st;
    if ((st = rotate())) return st;
    if ((st = operators(c, u, 1, 1))) return st;
    k_kick<T><<<grid_for(N), 256, 0, c->stream>>>(v, acc1, u, T(c->dt), T(c->kappa), T(c->f1), T(c->f3), N);
    count_launch();
    if ((st = rotate())) return st;
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_err(c, err, "plain splitting step");
    return VOFL_OK;
  }

  // ---- Crank-Nicolson (see the kernels above) ----
  bool can_cn() const override { return true; }

  int cn_alloc(vofl_ctx* c) {
    if (tb.M != c->M) return set_err(c, VOFL_ESTATE, "plain path: term batch not prepared for this M");
    if (cn.gen != tb.gen) {  // the graphs hold term-batch pointers
      cn_drop_graphs();
      cn.gen = tb.gen;
    }
    if (cn.b) return VOFL_OK;
    auto get = [&](void** q, size_t b) -> int {
      cudaError_t e = dev_malloc(q, b);
      if (e != cudaSuccess) return cuda_err(c, e, "cudaMalloc (Crank-Nicolson scratch)");
      cn.bytes += b;
      return VOFL_OK;
    };
    // all or nothing: a failure frees what this call allocated, so that
    // the next call does not find a half-allocated solver (cn.b set)
    auto fail = [&](int st) {
      nbytes += cn.bytes;  // cn_free takes off what was counted
      cn_free();
      return st;
    };
    int st;
    for (T** v : {&cn.b, &cn.x, &cn.r, &cn.z, &cn.p, &cn.w})
      if ((st = get((void**)v, sizeof(T) * N))) return fail(st);
    if ((st = get((void**)&cn.pa, sizeof(double) * CN_MAXG))) return fail(st);
    if ((st = get((void**)&cn.pb, sizeof(double) * CN_MAXG))) return fail(st);
    if ((st = get((void**)&cn.s, sizeof(double) * S_COUNT))) return fail(st);
    if (cudaMallocHost(&cn.hs, sizeof(double) * S_COUNT) != cudaSuccess) {
      cudaGetLastError();
      cn.hs = nullptr;
      return fail(set_err(c, VOFL_ENOMEM, "cudaMallocHost (solver scalars)"));
    }
    VOFL_CUDA(c, cudaMemsetAsync(cn.s, 0, sizeof(double) * S_COUNT, c->stream));
    nbytes += cn.bytes;
    return VOFL_OK;
  }

  // v -> Ym[m] = IFFT[P1 L^m/m! FFT(Lap v)], m = 0..M
  int cn_terms(vofl_ctx* c, const T* v) {
    const int nx = (int)c->n[0], ny = c->ndim > 1 ? (int)c->n[1] : 1, nz = c->ndim > 2 ? (int)c->n[2] : 1;
    k_laplacian<T><<<grid_for(N), 256, 0, c->stream>>>(v, Y, nx, ny, nz, ryy(c), rzz(c));
    count_launch();
    int st;
    if ((st = exec_fwd(c, Y))) return st;
    k_mult_ops<T, C><<<grid_small(Nh), kSmallBlock, 0, c->stream>>>(uh, P1, P2, Lg, c->M, 1, tb.X, Nh);
    count_launch();
    cufftResult r;
    if constexpr (sizeof(T) == 8)
      r = cufftExecZ2D(tb.inv1, (cufftDoubleComplex*)tb.X, (cufftDoubleReal*)tb.Y);
    else
      r = cufftExecC2R(tb.inv1, (cufftComplex*)tb.X, (cufftReal*)tb.Y);
    if (r != CUFFT_SUCCESS) return set_err(c, VOFL_ECUDA, "cuFFT batched inverse");
    return VOFL_OK;
  }

  // r -> Y = L^T r
  int cn_transpose(vofl_ctx* c, const T* r) {
    const int nx = (int)c->n[0], ny = c->ndim > 1 ? (int)c->n[1] : 1, nz = c->ndim > 2 ? (int)c->n[2] : 1;
    k_cn_pow_lap<T><<<grid_small(N), kSmallBlock, 0, c->stream>>>(r, (const T*)c->delta, c->M, tb.Y, nx, ny, nz, ryy(c),
                                                         rzz(c));
    count_launch();
    cufftResult res;
    if constexpr (sizeof(T) == 8)
      res = cufftExecD2Z(tb.fwd1, (cufftDoubleReal*)tb.Y, (cufftDoubleComplex*)tb.X);
    else
      res = cufftExecR2C(tb.fwd1, (cufftReal*)tb.Y, (cufftComplex*)tb.X);
    if (res != CUFFT_SUCCESS) return set_err(c, VOFL_ECUDA, "cuFFT batched forward");
    k_cn_tsum<T, C><<<grid_small(Nh), kSmallBlock, 0, c->stream>>>(tb.X, P1, Lg, c->M, X, Nh);
    count_launch();
    return exec_inv(c, X, Y);
  }

  static T ryy(const vofl_ctx* c) {
    if (c->ndim < 2) return T(1);
    const double hx = (c->hi[0] - c->lo[0]) / c->n[0], hy = (c->hi[1] - c->lo[1]) / c->n[1];
    return T((hx * hx) / (hy * hy));
  }
  static T rzz(const vofl_ctx* c) {
    if (c->ndim < 3) return T(1);
    const double hx = (c->hi[0] - c->lo[0]) / c->n[0], hz = (c->hi[2] - c->lo[2]) / c->n[2];
    return T((hx * hx) / (hz * hz));
  }

  // b and the first iterate from u^n = u[cur], u^{n-1} = u[1-cur]
  int cn_body_rhs(vofl_ctx* c, int cur) {
    k_inc<<<1, 1, 0, c->stream>>>(c->d_step);
    count_launch();
    int st;
    if ((st = cn_terms(c, (const T*)c->u[1 - cur]))) return st;
    const int G = cn_grid(N);
    k_cn_horner<T><<<G, CN_THREADS, 0, c->stream>>>(tb.Y, (const T*)c->delta, c->M, nullptr, T(0), T(1), acc1,
                                                     nullptr, N);
    count_launch();
    const double c2 = 0.5 * c->kappa * c->dt * c->dt, h2 = 0.5 * c->dt * c->dt;
    k_cn_rhs<T><<<grid_for(N), 256, 0, c->stream>>>((const T*)c->u[cur], (const T*)c->u[1 - cur], acc1, T(c2), T(h2),
                                                     T(c->f1), T(c->f3), cn.b, cn.x, N);
    count_launch();
    return VOFL_OK;
  }

  // r = b + h2 f(x) - A x and its norms
  int cn_body_resid(vofl_ctx* c) {
    int st;
    if ((st = cn_terms(c, cn.x))) return st;
    const int G = cn_grid(N);
    const double c2 = 0.5 * c->kappa * c->dt * c->dt, h2 = 0.5 * c->dt * c->dt;
    k_cn_horner<T><<<G, CN_THREADS, 0, c->stream>>>(tb.Y, (const T*)c->delta, c->M, cn.x, T(1), T(c2), cn.w,
                                                     nullptr, N);
    count_launch();
    k_cn_resid<T><<<G, CN_THREADS, 0, c->stream>>>(cn.b, cn.x, cn.w, T(h2), T(c->f1), T(c->f3), cn.r, cn.pa, cn.pb,
                                                    N);
    count_launch();
    k_cn_fin<<<1, CN_THREADS, 0, c->stream>>>(FIN_RRGG, cn.pa, cn.pb, G, 0.25 * c->cn_tol * c->cn_tol, cn.s);
    count_launch();
    return VOFL_OK;
  }

  // CGNR start: z = A^T r, p = z
  int cn_body_init(vofl_ctx* c) {
    int st;
    if ((st = cn_transpose(c, cn.r))) return st;
    const int G = cn_grid(N);
    const double c2 = 0.5 * c->kappa * c->dt * c->dt;
    k_cn_z<T><<<G, CN_THREADS, 0, c->stream>>>(cn.r, Y, T(c2), cn.z, cn.p, cn.pa, N);
    count_launch();
    k_cn_fin<<<1, CN_THREADS, 0, c->stream>>>(FIN_ZZ0, cn.pa, nullptr, G, 0.0, cn.s);
    count_launch();
    return VOFL_OK;
  }

  // kCnChunk CGNR iterations
  int cn_body_chunk(vofl_ctx* c) {
    const int G = cn_grid(N);
    const double c2 = 0.5 * c->kappa * c->dt * c->dt;
    for (int it = 0; it < kCnChunk; ++it) {
      int st;
      if ((st = cn_terms(c, cn.p))) return st;  // w = A p
      k_cn_horner<T><<<G, CN_THREADS, 0, c->stream>>>(tb.Y, (const T*)c->delta, c->M, cn.p, T(1), T(c2), cn.w,
                                                       cn.pa, N);
      count_launch();
      k_cn_fin<<<1, CN_THREADS, 0, c->stream>>>(FIN_WW, cn.pa, nullptr, G, 0.0, cn.s);
      count_launch();
      k_cn_xr<T><<<G, CN_THREADS, 0, c->stream>>>(cn.x, cn.r, cn.p, cn.w, cn.s, cn.pa, N);
      count_launch();
      k_cn_fin<<<1, CN_THREADS, 0, c->stream>>>(FIN_RR, cn.pa, nullptr, G, 0.0, cn.s);
      count_launch();
      if ((st = cn_transpose(c, cn.r))) return st;  // z = A^T r
      k_cn_z<T><<<G, CN_THREADS, 0, c->stream>>>(cn.r, Y, T(c2), cn.z, nullptr, cn.pa, N);
      count_launch();
      k_cn_fin<<<1, CN_THREADS, 0, c->stream>>>(FIN_ZZ, cn.pa, nullptr, G, 0.0, cn.s);
      count_launch();
      k_cn_p<T><<<grid_for(N), 256, 0, c->stream>>>(cn.z, cn.p, cn.s, N);
      count_launch();
    }
    return VOFL_OK;
  }

  // run `body` through its captured graph (capturing it on first use)
  template <typename F>
  int cn_run(vofl_ctx* c, cudaGraphExec_t* g, uint64_t* nk, F&& body) {
    if (!*g && cn.graphs_ok) {
      const uint64_t before = g_kernel_launches.load();
      cudaGraph_t gr = nullptr;
      if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const int st = body();
        const cudaError_t e = cudaStreamEndCapture(c->stream, &gr);
        *nk = g_kernel_launches.load() - before;
        g_kernel_launches.store(before);
        if (st == VOFL_OK && e == cudaSuccess && cudaGraphInstantiate(g, gr, 0) == cudaSuccess) {
          cudaGraphDestroy(gr);
        } else {
          if (gr) cudaGraphDestroy(gr);
          *g = nullptr;
          cn.graphs_ok = false;
          cudaGetLastError();
          c->err.clear();
        }
      } else {
        cudaGetLastError();
        cn.graphs_ok = false;
      }
    }
    if (*g) {
      VOFL_CUDA(c, cudaGraphLaunch(*g, c->stream));
      count_launch(*nk);
      return VOFL_OK;
    }
    return body();
  }

  int cn_read(vofl_ctx* c) {
    VOFL_CUDA(c, cudaMemcpyAsync(cn.hs, cn.s, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, c->stream));
    VOFL_CUDA(c, cudaStreamSynchronize(c->stream));
    return VOFL_OK;
  }

  // one Crank-Nicolson step n >= 1: u^{n+1} into u[1 - cur] (the caller
  // flips cur)
  int step_cn(vofl_ctx* c) override {
    NvtxRange nvtx_range("cnfp_step");
    int st;
    if ((st = cn_alloc(c))) return st;
    if (cn.key_dt != c->dt || cn.key_kappa != c->kappa || cn.key_f1 != c->f1 || cn.key_f3 != c->f3 ||
        cn.key_tol != c->cn_tol) {
      cn_drop_graphs();
      cn.key_dt = c->dt;
      cn.key_kappa = c->kappa;
      cn.key_f1 = c->f1;
      cn.key_f3 = c->f3;
      cn.key_tol = c->cn_tol;
    }
    if (c->steps == 1) VOFL_CUDA(c, cudaMemsetAsync(cn.s + S_ITERS, 0, sizeof(double), c->stream));
    const int cur = c->cur;
    if ((st = cn_run(c, &cn.g_rhs[cur], &cn.n_rhs, [&] { return cn_body_rhs(c, cur); }))) return st;
    const double tol2 = c->cn_tol * c->cn_tol;
    double rr_prev = 0.0;
    for (int outer = 0;; ++outer) {
      if ((st = cn_run(c, &cn.g_resid, &cn.n_resid, [&] { return cn_body_resid(c); }))) return st;
      if ((st = cn_read(c))) return st;
      const double rr = cn.hs[S_RR], gg = cn.hs[S_GG];
      if (!std::isfinite(rr) || !std::isfinite(gg))
        return set_err(c, VOFL_ENOCONV, "Crank-Nicolson step: the solution is not finite");
      if (rr <= tol2 * gg) break;
      if (outer >= kCnOuter) return set_err(c, VOFL_ENOCONV, "Crank-Nicolson step: fixed-point passes exhausted");
      if (outer >= 2 && rr > 0.81 * rr_prev) {
        if (rr <= 100.0 * tol2 * gg) break;  // at the rounding floor, within 10 tol
        return set_err(c, VOFL_ENOCONV,
                       ("Crank-Nicolson step: the residual stagnated at " + std::to_string(std::sqrt(rr / gg)) +
                        " relative; raise the tolerance (vofl_set_solver)")
                           .c_str());
      }
      rr_prev = rr;
      c->cn_solves += 1;
      if ((st = cn_run(c, &cn.g_init, &cn.n_init, [&] { return cn_body_init(c); }))) return st;
      for (int it = 0;;) {
        if ((st = cn_run(c, &cn.g_chunk, &cn.n_chunk, [&] { return cn_body_chunk(c); }))) return st;
        it += kCnChunk;
        if ((st = cn_read(c))) return st;
        if (cn.hs[S_STOP] != 0.0) break;
        if (!std::isfinite(cn.hs[S_RR]))
          return set_err(c, VOFL_ENOCONV, "Crank-Nicolson step: CG diverged");
        if (it >= c->cn_maxit) return set_err(c, VOFL_ENOCONV, "Crank-Nicolson step: CG iterations exhausted");
      }
      c->cn_iters = (int64_t)cn.hs[S_ITERS];
    }
    VOFL_CUDA(c, cudaMemcpyAsync(c->u[1 - cur], cn.x, sizeof(T) * N, cudaMemcpyDeviceToDevice, c->stream));
    return VOFL_OK;
  }

  int apply_pair(vofl_ctx* c, const void* u, void* o1, void* o2) override {
    int st = operators(c, (const T*)u);
    if (st) return st;
    if (o1) VOFL_CUDA(c, cudaMemcpyAsync(o1, acc1, sizeof(T) * N, cudaMemcpyDeviceToDevice, c->stream));
    if (o2) VOFL_CUDA(c, cudaMemcpyAsync(o2, acc2, sizeof(T) * N, cudaMemcpyDeviceToDevice, c->stream));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(c, e, "plain apply");
    return VOFL_OK;
  }

  int step(vofl_ctx* c, int mode, bool count_step) override {
    if (count_step) {
      k_inc<<<1, 1, 0, c->stream>>>(c->d_step);
      count_launch();
    }
    int st = operators(c, (const T*)c->u[c->cur]);
    if (st) return st;
    EpiArgs<T> e{};
    e.mode = mode;
    e.u_cur = (const T*)c->u[c->cur];
    e.u_other = (T*)c->u[1 - c->cur];
    e.l2p = (T*)c->l2p;
    e.A = (const T*)c->A;
    e.B = (const T*)c->B;
    e.dt1 = (T)c->dt;
    e.dt2 = (T)(c->dt * c->dt);
    e.src_flat = c->nsrc > 0 ? c->src_flat : -1;
    e.src = c->d_src;
    e.nsrc = c->nsrc;
    e.step = c->d_step;
    double hd = 1.0;
    for (int i = 0; i < c->ndim; ++i) hd *= (c->hi[i] - c->lo[i]) / (double)c->n[i];
    e.src_scale = c->dt * c->dt / hd;
    epi_model(c, &e);
    k_update<T><<<grid_for(N), 256, 0, c->stream>>>(acc1, acc2, e, N);
    count_launch();
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_err(c, err, "plain step");
    return VOFL_OK;
  }

};

}  // namespace

size_t plain_footprint(int ndim, const int64_t* n, int prec, int M) {
  long long N = 1;
  for (int i = 0; i < ndim; ++i) N *= n[i];
  const long long Nh = (n[0] / 2 + 1) * (N / n[0]);
  const size_t r = prec == VOFL_F64 ? 8 : 4;
  const size_t B = 2 * (size_t)(M + 1);  // the term batch: spectra and fields of both operators
  // + cuFFT work areas (about one real field per transform of the batch)
  return r * (2 * Nh * 2 + 3 * N + 3 * Nh) + 2 * r * N + B * r * (2 * Nh + N) + B * r * N;
}

Engine* make_plain(vofl_ctx* c, int* status) {
  Engine* e = nullptr;
  if (c->prec == VOFL_F64) {
    auto* p = new Plain<double>();
    *status = p->init(c);
    e = p;
  } else {
    auto* p = new Plain<float>();
    *status = p->init(c);
    e = p;
  }
  if (*status != VOFL_OK) {
    delete e;
    return nullptr;
  }
  return e;
}

}  // namespace vofl
