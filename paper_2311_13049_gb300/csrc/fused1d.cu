// fused1d.cu -- fused 1D path (float or double): the whole leap-frog run of
// Eq. (1.1) with both operators by the matrix-free scheme of Eq. (2.10) of
// arXiv 2311.13049, every transform in shared memory, every requested step
// inside one kernel launch.
//
// Per step (N points, M+1 Taylor terms):
//   w = D_xx u (periodic second difference) -> complex FFT -> S = DFT(w),
//       S_k = lambda_k * N * u_hat_k with lambda_k = -4 sin^2(pi k/N);
//   per slot index m: W_k = S_k (c1_m(k) + i c2_m(k)), c_op,m = P_op L^m/m!
//       (P_op = |mu|^{2 s0_op}/(N lambda_k), op 2 scaled by an exact power of
//       two lambda2), one complex inverse FFT gives L1-term + i L2-term
//       (both multiplied spectra are Hermitian); for the general model (one
//       operator) the two slots carry terms m and m + K instead;
//   the delta^m weights by Horner's rule, then the pointwise leap-frog update
//   (Eq. (3.4) extended to Eq. (1.1)).
// Two kernels: k1d_cluster_run spreads the slot indices of one line over a
// thread-block cluster of up to 8 CTAs (distributed shared memory, per-term
// multiplier tables); k1d_run keeps the whole line in one CTA (a single
// slot index, or when no cluster can be resident).
// The FFT is a radix-2 Stockham autosort over the CTA (Govindaraju et al.,
// SC 2008), ping-ponging between two shared buffers.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.h"

namespace vofl {

namespace {

constexpr int T1D = 256;  // threads per CTA
constexpr int MAX_PTS_PER_THREAD = 16;

template <typename R>
struct C2;
template <>
struct C2<float> {
  using T = float2;
};
template <>
struct C2<double> {
  using T = double2;
};

template <typename C>
__device__ __forceinline__ C cm(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

// radix-2 Stockham over the CTA; `a` holds the input, the returned pointer
// (a or b) holds the output; tw[t] = exp(-2 pi i t / N), t < N/2
template <typename C>
__device__ C* block_fft(C* a, C* b, const C* tw, int N, bool inv) {
  const int H = N / 2;
  for (int Ns = 1; Ns < N; Ns <<= 1) {
    const int step = H / Ns;  // N / (2 Ns)
    for (int j = threadIdx.x; j < H; j += blockDim.x) {
      const int k = j & (Ns - 1);
      C w = tw[k * step];
      if (inv) w.y = -w.y;
      const C x0 = a[j];
      const C x1 = cm(a[j + H], w);
      const int o = ((j - k) << 1) + k;
      C s, d;
      s.x = x0.x + x1.x;
      s.y = x0.y + x1.y;
      d.x = x0.x - x1.x;
      d.y = x0.y - x1.y;
      b[o] = s;
      b[o + Ns] = d;
    }
    __syncthreads();
    C* t = a;
    a = b;
    b = t;
  }
  return a;
}

// the term layout of the two packed slots (as term_split in kernels.cuh)
struct TermSplit1 {
  int split_k, k2;
};
inline TermSplit1 term_split1(int M, bool one_operator) {
  if (!one_operator) return {0, M + 1};
  const int K = (M + 2) / 2;
  return {K, M + 1 - K};
}

template <typename R>
struct Sim1D {
  int N, M;
  int mode_first;         // EPI_START for the first step of a run, EPI_STEP otherwise, EPI_APPLY for apply
  int nsteps;             // steps to run in this launch
  int step0;              // index n of the first step (source sample index)
  R* u[2];                // u buffers
  int cur;                // buffer holding u^n at launch start
  R* l2p;                 // L2 u^{n-1} (or L2 psi before the start step)
  const R* delta;
  const R* A;
  const R* B;
  const R* P1;            // [N] |mu|^{2 s01} / (N lambda)
  const R* P2;            // [N] lambda2 |mu|^{2 s02} / (N lambda)
  const R* Lg;            // [N] ln |mu|^2 (0 at k = 0)
  const typename C2<R>::T* tw;  // [N/2]
  R inv_lambda2;
  R dt1, dt2;
  long long src_flat;
  const double* src;
  long long nsrc;
  double src_scale;
  int nonlin;             // general model: f(u) = f1 u + f3 u^3
  R f1, f3;
  int split_k;            // > 0: one operator, terms K.. in the imaginary slot (K = split_k)
  int k2;                 // ... of which the first k2 exist (terms K..M)
  const R* T;             // [2][M+1][N] multipliers P_op ln|mu|^{2m}/m! (cluster kernel)
  const R* apply_in;      // EPI_APPLY: input field
  R* out1;
  R* out2;
};

template <typename R>
__global__ void __launch_bounds__(T1D) k1d_run(const Sim1D<R>* sims) {
  using C = typename C2<R>::T;
  const Sim1D<R> sp = sims[blockIdx.x];
  const int N = sp.N, H = N / 2;
  const int PPT = N / T1D > 0 ? N / T1D : 1;  // points per thread (N >= T1D) or 1
  extern __shared__ unsigned char smem_raw[];
  C* S = reinterpret_cast<C*>(smem_raw);
  C* B0 = S + N;
  C* B1 = B0 + N;
  C* tws = B1 + N;
  for (int i = threadIdx.x; i < H; i += blockDim.x) tws[i] = sp.tw[i];
  // per-thread owned points j = t + T1D*i (i < PPT), only if j < N
  R dl[MAX_PTS_PER_THREAD], a1[MAX_PTS_PER_THREAD], a2[MAX_PTS_PER_THREAD];
  for (int i = 0; i < PPT; ++i) {
    const int j = threadIdx.x + T1D * i;
    dl[i] = j < N ? sp.delta[j] : R(0);
  }
  __syncthreads();
  R* ucur = sp.u[sp.cur];
  R* uoth = sp.u[1 - sp.cur];
  for (int s = 0; s < sp.nsteps; ++s) {
    const int mode = (s == 0) ? sp.mode_first : EPI_STEP;
    const R* uin = (mode == EPI_APPLY) ? sp.apply_in : ucur;
    // w = D_xx u into B0 (complex, zero imaginary part)
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      const R c = uin[j];
      const R d = (uin[j + 1 == N ? 0 : j + 1] - c) - (c - uin[j == 0 ? N - 1 : j - 1]);
      C v;
      v.x = d;
      v.y = R(0);
      B0[j] = v;
    }
    __syncthreads();
    C* f = block_fft<C>(B0, B1, tws, N, false);
    for (int k = threadIdx.x; k < N; k += blockDim.x) S[k] = f[k];
    __syncthreads();
    for (int i = 0; i < PPT; ++i) a1[i] = a2[i] = R(0);
    // two operators: slot indices m = M..0, operator 1 real, operator 2
    // imaginary; one operator (split_k = K): m = K-1..0, term m real and
    // term m + K imaginary (when it exists)
    const int K = sp.split_k;
    const int top = K > 0 ? K - 1 : sp.M;
    double fact = 1.0, fact2 = 1.0;  // m! and (m + K)! in double (40! overflows float)
    for (int m = 1; m <= top; ++m) fact *= m;
    for (int m = 1; m <= top + K; ++m) fact2 *= m;
    for (int m = top; m >= 0; --m) {
      const R invf = R(1.0 / fact);
      const R invf2 = K > 0 ? (m < sp.k2 ? R(1.0 / fact2) : R(0)) : invf;
      for (int k = threadIdx.x; k < N; k += blockDim.x) {
        // L^m (and L^{m+K}) by squaring
        const R l0 = sp.Lg[k];
        R l = l0, p = R(1), q = R(1);
        int e = m;
        while (e) {
          if (e & 1) p *= l;
          l *= l;
          e >>= 1;
        }
        const R t = p * invf;
        R c1 = sp.P1[k] * t, c2;
        if (K > 0) {
          l = l0;
          e = m + K;
          while (e) {
            if (e & 1) q *= l;
            l *= l;
            e >>= 1;
          }
          c2 = sp.P1[k] * q * invf2;
        } else {
          c2 = sp.P2[k] * t;
        }
        const C sk = S[k];
        C w;  // (c1 + i c2) * S_k
        w.x = c1 * sk.x - c2 * sk.y;
        w.y = c1 * sk.y + c2 * sk.x;
        B0[k] = w;
      }
      __syncthreads();
      C* y = block_fft<C>(B0, B1, tws, N, true);
      for (int i = 0; i < PPT; ++i) {
        const int j = threadIdx.x + T1D * i;
        if (j < N) {
          const C v = y[j];
          a1[i] = v.x + dl[i] * a1[i];
          a2[i] = v.y + dl[i] * a2[i];
        }
      }
      __syncthreads();
      if (m > 0) fact /= m;
      if (m + K > 0) fact2 /= m + K;
    }
    // epilogue
    EpiArgs<R> e{};
    e.mode = mode;
    e.out1 = sp.out1;
    e.out2 = sp.out2;
    e.u_cur = ucur;
    e.u_other = uoth;
    e.l2p = sp.l2p;
    e.A = sp.A;
    e.B = sp.B;
    e.dt1 = sp.dt1;
    e.dt2 = sp.dt2;
    e.src_flat = sp.src_flat;
    e.src = sp.src;
    e.nsrc = sp.nsrc;
    const int n_step = sp.step0 + s;
    e.step = &n_step;
    e.src_scale = sp.src_scale;
    e.nonlin = sp.nonlin;
    e.f1 = sp.f1;
    e.f3 = sp.f3;
    for (int i = 0; i < PPT; ++i) {
      const int j = threadIdx.x + T1D * i;
      if (j >= N) continue;
      if (K > 0) {  // sum_{m<K} + delta^K sum_{m>=K}
        R dk = R(1);
        for (int r = 0; r < K; ++r) dk *= dl[i];
        epilogue_point<R>(e, j, a1[i] + dk * a2[i], R(0));
      } else {
        epilogue_point<R>(e, j, a1[i], a2[i] * sp.inv_lambda2);
      }
    }
    __syncthreads();  // the next step reads the new u everywhere
    if (mode == EPI_APPLY) break;
    R* t = ucur;
    ucur = uoth;
    uoth = t;
  }
}

// The same run on a thread-block cluster of CL CTAs (distributed shared
// memory).  GB300's FP64 rate is ~8 GFLOP/s per SM, so one CTA per line is
// FP64-bound on a single SM; the cluster spreads the M+1 (or K) inverse
// transforms over CL SMs.  Per step:
//   1. every CTA transforms the whole u^n (held in its shared memory U);
//   2. CTA r takes the slot indices m = r, r+CL, ... (descending), sums
//      Y_m delta^(m-r) by Horner in delta^CL and scales by delta^r;
//   3. it stores its partial sums for the points of slice q (N/CL points)
//      into CTA q's receive buffer (DSMEM);          -- cluster barrier
//   4. CTA q adds the CL partials of its slice in rank order, runs the
//      epilogue for its slice and stores u^{n+1} of the slice into every
//      CTA's U (DSMEM);                               -- cluster barrier
// Every CTA runs the same steps, so every CTA reaches every barrier.
template <typename R>
size_t smem_1dc(int N) {
  using C = typename C2<R>::T;
  return sizeof(C) * (3 * (size_t)N + N / 2) + sizeof(R) * 3 * (size_t)N;
}

template <typename R>
__global__ void __launch_bounds__(T1D) k1d_cluster_run(const Sim1D<R>* sims, int CL) {
  namespace cg = cooperative_groups;
  using C = typename C2<R>::T;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const Sim1D<R> sp = sims[blockIdx.x / CL];
  const int N = sp.N, H = N / 2, SL = N / CL;
  const int PPT = N / T1D > 0 ? N / T1D : 1;
  extern __shared__ unsigned char smem_raw[];
  C* S = reinterpret_cast<C*>(smem_raw);
  C* B0 = S + N;
  C* B1 = B0 + N;
  C* tws = B1 + N;
  R* U = reinterpret_cast<R*>(tws + H);  // u^n, whole line
  R* RX = U + N;                         // [CL][SL][2] partial sums of this CTA's slice
  const int K = sp.split_k;
  const int slots = K > 0 ? K : sp.M + 1;
  for (int i = threadIdx.x; i < H; i += blockDim.x) tws[i] = sp.tw[i];
  R dl[MAX_PTS_PER_THREAD], dcl[MAX_PTS_PER_THREAD], a1[MAX_PTS_PER_THREAD], a2[MAX_PTS_PER_THREAD];
  for (int i = 0; i < PPT; ++i) {
    const int j = threadIdx.x + T1D * i;
    dl[i] = j < N ? sp.delta[j] : R(0);
    R p = R(1);
    for (int r = 0; r < CL; ++r) p *= dl[i];
    dcl[i] = p;
  }
  R* ucur = sp.u[sp.cur];
  R* uoth = sp.u[1 - sp.cur];
  {
    const R* u0 = sp.mode_first == EPI_APPLY ? sp.apply_in : ucur;
    for (int j = threadIdx.x; j < N; j += blockDim.x) U[j] = u0[j];
  }
  cluster.sync();  // every CTA of the cluster runs before any remote access
  // this CTA's highest slot index m = rank + CL t
  const int mtop = rank < slots ? rank + CL * ((slots - 1 - rank) / CL) : -1;
  for (int s = 0; s < sp.nsteps; ++s) {
    const int mode = (s == 0) ? sp.mode_first : EPI_STEP;
    // 1. spectrum of D_xx u^n
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      const R c = U[j];
      C v;
      v.x = (U[j + 1 == N ? 0 : j + 1] - c) - (c - U[j == 0 ? N - 1 : j - 1]);
      v.y = R(0);
      B0[j] = v;
    }
    __syncthreads();
    C* f = block_fft<C>(B0, B1, tws, N, false);
    for (int k = threadIdx.x; k < N; k += blockDim.x) S[k] = f[k];
    __syncthreads();
    // 2. this CTA's slot indices, Horner in delta^CL
    for (int i = 0; i < PPT; ++i) a1[i] = a2[i] = R(0);
    for (int m = mtop; m >= 0; m -= CL) {
      const R* t1 = sp.T + (size_t)m * N;
      const R* t2 = K > 0 ? (m < sp.k2 ? sp.T + (size_t)(m + K) * N : nullptr) : sp.T + (size_t)(sp.M + 1 + m) * N;
      for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const R c1 = t1[k], c2 = t2 ? t2[k] : R(0);
        const C sk = S[k];
        C w;
        w.x = c1 * sk.x - c2 * sk.y;
        w.y = c1 * sk.y + c2 * sk.x;
        B0[k] = w;
      }
      __syncthreads();
      C* y = block_fft<C>(B0, B1, tws, N, true);
      for (int i = 0; i < PPT; ++i) {
        const int j = threadIdx.x + T1D * i;
        if (j < N) {
          const C v = y[j];
          a1[i] = v.x + dcl[i] * a1[i];
          a2[i] = v.y + dcl[i] * a2[i];
        }
      }
      __syncthreads();
    }
    // 3. scale by delta^rank and send each slice's partials to its owner
    for (int i = 0; i < PPT; ++i) {
      const int j = threadIdx.x + T1D * i;
      if (j >= N) continue;
      R dr = R(1);
      for (int r = 0; r < rank; ++r) dr *= dl[i];
      const int q = j / SL, jj = j - q * SL;
      R* dst = cluster.map_shared_rank(RX, q) + 2 * ((size_t)rank * SL + jj);
      dst[0] = a1[i] * dr;
      dst[1] = a2[i] * dr;
    }
    cluster.sync();
    // 4. the owner of slice `rank` sums, updates and broadcasts
    EpiArgs<R> e{};
    e.mode = mode;
    e.out1 = sp.out1;
    e.out2 = sp.out2;
    e.u_cur = ucur;
    e.u_other = uoth;
    e.l2p = sp.l2p;
    e.A = sp.A;
    e.B = sp.B;
    e.dt1 = sp.dt1;
    e.dt2 = sp.dt2;
    e.src_flat = sp.src_flat;
    e.src = sp.src;
    e.nsrc = sp.nsrc;
    const int n_step = sp.step0 + s;
    e.step = &n_step;
    e.src_scale = sp.src_scale;
    e.nonlin = sp.nonlin;
    e.f1 = sp.f1;
    e.f3 = sp.f3;
    for (int jj = threadIdx.x; jj < SL; jj += blockDim.x) {
      const int j = rank * SL + jj;
      R L1 = R(0), L2 = R(0);
      for (int r = 0; r < CL; ++r) {
        L1 += RX[2 * ((size_t)r * SL + jj)];
        L2 += RX[2 * ((size_t)r * SL + jj) + 1];
      }
      if (K > 0) {  // sum_{m<K} + delta^K sum_{m>=K}
        const R d = sp.delta[j];
        R dk = R(1);
        for (int r = 0; r < K; ++r) dk *= d;
        epilogue_point<R>(e, j, L1 + dk * L2, R(0));
      } else {
        epilogue_point<R>(e, j, L1, L2 * sp.inv_lambda2);
      }
      if (mode != EPI_APPLY) {
        const R un = uoth[j];
        for (int q = 0; q < CL; ++q) cluster.map_shared_rank(U, q)[j] = un;
      }
    }
    cluster.sync();  // U holds u^{n+1} everywhere; RX may be rewritten
    if (mode == EPI_APPLY) break;
    R* t = ucur;
    ucur = uoth;
    uoth = t;
  }
}

// T[op][m][k] = P_op[k] ln|mu_k|^{2m} / m!, m = 0..M (the multipliers of
// Eq. (2.13) per term; the cluster kernel reads them instead of forming
// the powers every step)
template <typename R>
__global__ void k1d_term_tables(int N, int M, const R* __restrict__ P1, const R* __restrict__ P2,
                                const R* __restrict__ Lg, R* __restrict__ T) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    // in double, rounded once to R (set-up work)
    const double l = (double)Lg[k], p1 = (double)P1[k], p2 = (double)P2[k];
    double t = 1.0;  // ln|mu|^{2m} / m!
    for (int m = 0; m <= M; ++m) {
      if (m > 0) t = t * l / m;
      T[(size_t)m * N + k] = R(p1 * t);
      T[(size_t)(M + 1 + m) * N + k] = R(p2 * t);
    }
  }
}

template <typename R>
__global__ void k1d_tables(int N, double L, double s01, double s02, double lambda2, R* P1, R* P2, R* Lg) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    const int ks = k < N / 2 ? k : k - N;
    const double mu = 2.0 * M_PI * ks / L;
    const double m2 = mu * mu;
    if (m2 == 0.0) {
      P1[k] = R(0);
      P2[k] = R(0);
      Lg[k] = R(0);
    } else {
      const double s = sinpi((double)k / N);
      const double lam = -4.0 * s * s;
      const double lg = log(m2);
      P1[k] = R(exp(s01 * lg) / (N * lam));
      P2[k] = R(lambda2 * exp(s02 * lg) / (N * lam));
      Lg[k] = R(lg);
    }
  }
}

template <typename C>
__global__ void k1d_twiddles(int N, C* tw) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N / 2; t += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)t / (double)N, &s, &c);
    C v;
    v.x = (decltype(v.x))c;
    v.y = (decltype(v.y))s;
    tw[t] = v;
  }
}

template <typename R>
size_t smem_1d(int N) {
  using C = typename C2<R>::T;
  return sizeof(C) * (3 * (size_t)N + N / 2);
}

template <typename R>
struct Fused1D : Engine {
  using C = typename C2<R>::T;
  int N = 0;
  R *P1 = nullptr, *P2 = nullptr, *Lg = nullptr;
  C* tw = nullptr;
  Sim1D<R>* d_sim = nullptr;
  double lambda2 = 1.0;
  size_t nbytes = 0;
  bool cluster_ok = false;
  R* T = nullptr;  // per-term multipliers [2][M+1][N] (cluster kernel)
  int tab_M = -1, model_gen = 0, tab_gen = -1;
  size_t tab_bytes = 0;
  int cluster_fits[4] = {-1, -1, -1, -1};  // CL = 2, 4, 8: can one cluster be resident (-1 unknown)
  static constexpr size_t kMaxSmem = 227 * 1024;

  cudaLaunchConfig_t cluster_cfg(int CL, cudaLaunchAttribute* at, cudaStream_t st) const {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(T1D);
    cfg.dynamicSmemBytes = smem_1dc<R>(N);
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
  }
  // whether a cluster of CL CTAs with this line's shared memory can run
  bool fits(int CL, cudaStream_t st) {
    int& f = cluster_fits[CL == 2 ? 0 : CL == 4 ? 1 : 2];
    if (f < 0) {
      cudaLaunchAttribute at[1];
      cudaLaunchConfig_t cfg = cluster_cfg(CL, at, st);
      int n = 0;
      f = cudaOccupancyMaxActiveClusters(&n, k1d_cluster_run<R>, &cfg) == cudaSuccess && n >= 1 ? 1 : 0;
      cudaGetLastError();
    }
    return f == 1;
  }

  ~Fused1D() override {
    dev_free(P1);
    dev_free(P2);
    dev_free(Lg);
    dev_free(tw);
    dev_free(d_sim);
    dev_free(T);
  }
  size_t bytes() const override { return nbytes; }

  int init(vofl_ctx* c) {
    N = (int)c->n[0];
    const size_t b = sizeof(R) * N;
    bool ok = dev_malloc(&P1, b) == cudaSuccess && dev_malloc(&P2, b) == cudaSuccess &&
              dev_malloc(&Lg, b) == cudaSuccess && dev_malloc(&tw, sizeof(C) * (N / 2)) == cudaSuccess &&
              dev_malloc(&d_sim, sizeof(Sim1D<R>)) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      return set_err(c, VOFL_ENOMEM, "cudaMalloc (fused 1D tables)");
    }
    nbytes = 3 * b + sizeof(C) * (N / 2) + sizeof(Sim1D<R>);
    if (cudaFuncSetAttribute(k1d_run<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_1d<R>(N)) !=
        cudaSuccess) {
      cudaGetLastError();
      return set_err(c, VOFL_EUNSUPPORTED, "fused 1D path: line too long for shared memory");
    }
    // the cluster form where its buffers fit one CTA's shared memory
    cluster_ok = smem_1dc<R>(N) <= kMaxSmem &&
                 cudaFuncSetAttribute(k1d_cluster_run<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem_1dc<R>(N)) == cudaSuccess;
    cudaGetLastError();
    k1d_twiddles<C><<<std::max(1, N / 512), 256, 0, c->stream>>>(N, tw);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return set_err(c, VOFL_ECUDA, "fused 1D twiddles");
    return VOFL_OK;
  }

  int set_model(vofl_ctx* c) override {
    const double L = c->hi[0] - c->lo[0];
    const double mu_max = M_PI * N / L;
    lambda2 = std::ldexp(1.0, (int)std::lround(0.5 * std::log2(std::max(mu_max, 1.0))));
    k1d_tables<R><<<std::max(1, N / 256), 256, 0, c->stream>>>(N, L, c->s01, c->s02, lambda2, P1,
                                                               P2, Lg);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return set_err(c, VOFL_ECUDA, "fused 1D tables");
    ++model_gen;  // the term tables follow in prepare()
    return VOFL_OK;
  }

  // per-term multiplier tables for the context's M and model
  int prepare(vofl_ctx* c) override {
    if (T && tab_M == c->M && tab_gen == model_gen) return VOFL_OK;
    if (tab_M != c->M) {
      VOFL_CUDA(c, cudaStreamSynchronize(c->stream));  // queued work may still read the old table
      dev_free(T);
      T = nullptr;
      nbytes -= tab_bytes;
      tab_bytes = sizeof(R) * 2 * (size_t)(c->M + 1) * N;
      const cudaError_t e = dev_malloc(&T, tab_bytes);
      if (e != cudaSuccess) {
        T = nullptr;
        tab_bytes = 0;
        tab_M = -1;
        return cuda_err(c, e, "cudaMalloc (fused 1D term tables)");
      }
      nbytes += tab_bytes;
      tab_M = c->M;
    }
    k1d_term_tables<R><<<std::max(1, N / 256), 256, 0, c->stream>>>(N, c->M, P1, P2, Lg, T);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return set_err(c, VOFL_ECUDA, "fused 1D term tables");
    tab_gen = model_gen;
    return VOFL_OK;
  }

  Sim1D<R> base(vofl_ctx* c) const {
    Sim1D<R> s{};
    s.N = N;
    s.M = c->M;
    s.u[0] = (R*)c->u[0];
    s.u[1] = (R*)c->u[1];
    s.cur = c->cur;
    s.l2p = (R*)c->l2p;
    s.delta = (const R*)c->delta;
    s.A = (const R*)c->A;
    s.B = (const R*)c->B;
    s.P1 = P1;
    s.P2 = P2;
    s.Lg = Lg;
    s.tw = tw;
    s.inv_lambda2 = R(1.0 / lambda2);
    s.dt1 = R(c->dt);
    s.dt2 = R(c->dt * c->dt);
    s.src_flat = c->nsrc > 0 ? c->src_flat : -1;
    s.src = c->d_src;
    s.nsrc = c->nsrc;
    s.src_scale = c->dt * c->dt / ((c->hi[0] - c->lo[0]) / N);
    {
      EpiArgs<R> em{};
      epi_model(c, &em);
      s.nonlin = em.nonlin;
      s.f1 = em.f1;
      s.f3 = em.f3;
    }
    const TermSplit1 ts = term_split1(c->M, c->general);
    s.split_k = ts.split_k;
    s.k2 = ts.k2;
    s.T = (T && tab_M == c->M && tab_gen == model_gen) ? T : nullptr;
    return s;
  }

  int launch(vofl_ctx* c, const Sim1D<R>& s) {
    // the parameter block goes to the device on the context stream; a copy
    // from pageable host memory is staged before the call returns, so `s`
    // may go out of scope, and the stream orders it after earlier launches
    if (cudaMemcpyAsync(d_sim, &s, sizeof(s), cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
      cudaGetLastError();
      return set_err(c, VOFL_ECUDA, "fused 1D parameters");
    }
    // CTAs per line: a power of two up to 8 (the portable cluster size), at
    // most one per slot index
    const int slots = s.split_k > 0 ? s.split_k : s.M + 1;
    int CL = 1;
    while (CL * 2 <= std::min(8, slots) && N % (CL * 2) == 0) CL *= 2;
    while (CL > 1 && !(cluster_ok && s.T && fits(CL, c->stream))) CL /= 2;
    if (CL > 1) {
      cudaLaunchAttribute at[1];
      cudaLaunchConfig_t cfg = cluster_cfg(CL, at, c->stream);
      const cudaError_t e = cudaLaunchKernelEx(&cfg, k1d_cluster_run<R>, (const Sim1D<R>*)d_sim, CL);
      count_launch();
      if (e != cudaSuccess) return cuda_err(c, e, "fused 1D cluster launch");
      return VOFL_OK;
    }
    k1d_run<R><<<1, T1D, smem_1d<R>(N), c->stream>>>(d_sim);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return set_err(c, VOFL_ECUDA, "fused 1D launch");
    return VOFL_OK;
  }

  uint64_t kernels_per_step(const vofl_ctx*) const override { return 1; }

  int apply_pair(vofl_ctx* c, const void* u, void* o1, void* o2) override {
    Sim1D<R> s = base(c);
    s.mode_first = EPI_APPLY;
    s.nsteps = 1;
    s.step0 = 0;
    s.apply_in = (const R*)u;
    s.out1 = (R*)o1;
    s.out2 = (R*)o2;
    return launch(c, s);
  }

  int step(vofl_ctx* c, int mode, bool count_step) override {
    (void)count_step;
    Sim1D<R> s = base(c);
    s.mode_first = mode;
    s.nsteps = 1;
    s.step0 = (int)c->steps;
    return launch(c, s);
  }

  bool can_run() const override { return true; }

  int run(vofl_ctx* c, int64_t nsteps, int first_mode) override {
    Sim1D<R> s = base(c);
    s.mode_first = first_mode;
    s.nsteps = (int)nsteps;
    s.step0 = (int)c->steps;
    return launch(c, s);
  }
};

}  // namespace

bool fused1d_supported(int ndim, const int64_t* n, int prec) {
  if (ndim != 1) return false;
  const int64_t N = n[0];
  if (N < 16 || N > T1D * MAX_PTS_PER_THREAD || (N & (N - 1))) return false;
  const size_t sm = prec == VOFL_F64 ? smem_1d<double>((int)N) : smem_1d<float>((int)N);
  return sm <= 200 * 1024;
}

Engine* make_fused1d(vofl_ctx* c, int* status) {
  Engine* e = nullptr;
  if (c->prec == VOFL_F64) {
    auto* p = new Fused1D<double>();
    *status = p->init(c);
    e = p;
  } else {
    auto* p = new Fused1D<float>();
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
