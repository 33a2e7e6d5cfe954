// plain.cu -- the plain baseline: the same arithmetic as the fused path
// (Eq. (2.13) of arXiv 2311.13049 for both operators of Eq. (1.1), then the
// leap-frog update of Eq. (3.4)) with library transforms (cuFFT R2C / C2R)
// and one separate elementwise kernel per step of the formula:
//   forward R2C of u;
//   for m = 0..M, op in {1, 2}:
//     multiply: X = u_hat * P_op(k) (ln|mu_k|^2)^m / m!      (kernel)
//     inverse C2R of X                                        (cuFFT)
//     accumulate: acc_op += (s(x) - s0)^m * Y                 (kernel)
//   pointwise update                                          (kernel)
// Works for 1D, 2D, 3D and for float or double.  It keeps every field in
// memory between kernels; that traffic is what the fused path removes.
// For the general model it also runs the second-order time splitting of
// Sec. 3.3 (step_split): exact half-step rotations of (u_hat, v_hat) in
// Fourier space, the variable-order kick (terms m >= 1), the rotations again.
#include <cuda_runtime.h>
#include <cufft.h>

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

template <typename T, typename C>
__global__ void k_mult(const C* __restrict__ uh, const T* __restrict__ P, const T* __restrict__ Lg, int m, T inv_fact,
                       C* __restrict__ X, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    T c = P[i] * inv_fact;
    const T l = Lg[i];
    for (int j = 0; j < m; ++j) c *= l;
    C v = uh[i];
    v.x *= c;
    v.y *= c;
    X[i] = v;
  }
}

template <typename T>
__global__ void k_acc(const T* __restrict__ Y, const T* __restrict__ delta, int m, int first, T* __restrict__ acc,
                      long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    T w = T(1);
    const T d = delta[i];
    for (int j = 0; j < m; ++j) w *= d;
    acc[i] = (first ? T(0) : acc[i]) + w * Y[i];
  }
}

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

  ~Plain() override {
    if (have_fwd) cufftDestroy(fwd);
    if (have_inv) cufftDestroy(inv);
    cudaFree(uh);
    cudaFree(X);
    cudaFree(Y);
    cudaFree(acc1);
    cudaFree(acc2);
    cudaFree(P1);
    cudaFree(P2);
    cudaFree(Lg);
    cudaFree(W);
    cudaFree(vh);
  }
  size_t bytes() const override { return nbytes; }

  int alloc(vofl_ctx* c, void** p, size_t b) {
    cudaError_t e = cudaMalloc(p, b);
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
    // our own kernels only (cuFFT's are library launches)
    return 2ull * 2 * (c->M + 1) + 3;  // multiply + accumulate per term, stencil, update, step counter
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
  // acc1 (, acc2)
  int operators(vofl_ctx* c, const T* u, int m0 = 0, int nops = 2) {
    int st;
    // forward transform of the discrete Laplacian of u (into Y, free here)
    const int nx = (int)c->n[0], ny = c->ndim > 1 ? (int)c->n[1] : 1, nz = c->ndim > 2 ? (int)c->n[2] : 1;
    const double hx = (c->hi[0] - c->lo[0]) / nx;
    const double hy = c->ndim > 1 ? (c->hi[1] - c->lo[1]) / ny : 1.0;
    const double hz = c->ndim > 2 ? (c->hi[2] - c->lo[2]) / nz : 1.0;
    k_laplacian<T><<<grid_for(N), 256, 0, c->stream>>>(u, Y, nx, ny, nz, T((hx * hx) / (hy * hy)),
                                                        T((hx * hx) / (hz * hz)));
    count_launch();
    if ((st = exec_fwd(c, Y))) return st;
    double fact = 1.0;
    for (int m = 0; m <= c->M; ++m) {
      if (m > 0) fact *= m;
      if (m < m0) continue;
      for (int op = 0; op < nops; ++op) {
        k_mult<T, C><<<grid_for(Nh), 256, 0, c->stream>>>(uh, op == 0 ? P1 : P2, Lg, m, T(1.0 / fact), X, Nh);
        count_launch();
        if ((st = exec_inv(c))) return st;
        k_acc<T><<<grid_for(N), 256, 0, c->stream>>>(Y, (const T*)c->delta, m, m == m0 ? 1 : 0,
                                                      op == 0 ? acc1 : acc2, N);
        count_launch();
      }
    }
    if (m0 > c->M) {
      for (int op = 0; op < nops; ++op)
        VOFL_CUDA(c, cudaMemsetAsync(op == 0 ? acc1 : acc2, 0, sizeof(T) * N, c->stream));
    }
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

size_t plain_footprint(int ndim, const int64_t* n, int prec) {
  long long N = 1;
  for (int i = 0; i < ndim; ++i) N *= n[i];
  const long long Nh = (n[0] / 2 + 1) * (N / n[0]);
  const size_t r = prec == VOFL_F64 ? 8 : 4;
  return r * (2 * Nh * 2 + 3 * N + 3 * Nh) + 2 * r * N;  // + cuFFT work area (about one real field)
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
