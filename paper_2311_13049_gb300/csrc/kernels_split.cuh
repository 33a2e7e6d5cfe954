// kernels_split.cuh -- the exact flow of the second-order time splitting
// (Sec. 3.3 of arXiv 2311.13049) on the fused FP32 2D path: over a time t,
//   u_t = v,  v_t = -kappa (-Delta)^{s0} u
// is solved mode by mode in Fourier space,
//   (u_k, v_k) <- (c u_k + (s / w) v_k,  c v_k - w s u_k),
//   w = sqrt(kappa) |mu_k|^{s0},  c = cos(w t),  s = sin(w t)
// (u_k <- u_k + t v_k where w = 0).  The variable-order remainder (terms
// m >= 1 of Eq. (2.13)) and the kick v += dt (-kappa D u + f(u)) run on the
// fused operator kernels (fused2d.cu).
//
// Three passes on the line transforms of fft_warp.cuh (one warp per line
// or several lines per warp, as in kernels.cuh):
//   S1 k2d_rot_fwd_rows   u, v -> row half spectra Su, Sv ([ny][pT] c64):
//        one complex FFT along x of u[y] + i v[y] per row, split into the
//        two half spectra;
//   S2 k2d_rot_cols       per column k_x: the forward FFT along y of Su
//        and Sv, the flow above (c, s / w, w s per mode from a table that
//        k_flow_table builds in double for a run's dt and dt/2), the
//        1/(nx ny) of the unnormalised
//        transforms, the inverse FFT along y of both, back to Su, Sv (loads
//        and stores are row segments of the CTA's columns: the first and
//        last stages are done cooperatively as in k2d_inv_cols);
//   S3 k2d_rot_inv_rows   per row: one complex inverse FFT along x of the
//        Hermitian extensions A + iB of (Su[y], Sv[y]) gives u[y] + i v[y].
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace vofl {
namespace {

constexpr int W_ROT = 4;  // warps per CTA of the splitting kernels

template <int N>
constexpr size_t rot_rows_smem() {
  return exch_smem<N, W_ROT>();
}
template <int N>
constexpr size_t rot_cols_smem() {
  return 2 * exch_smem<N, W_ROT>();  // one exchange set per field
}

// S1: row y of u and v -> Su[y][0..H], Sv[y][0..H]
template <int NX>
__global__ void __launch_bounds__(W_ROT * 32) k2d_rot_fwd_rows(const float* __restrict__ u, const float* __restrict__ v,
                                                               float2* __restrict__ Su, float2* __restrict__ Sv, int ny,
                                                               int pT, const float2* __restrict__ twx) {
  using F = LineFFT<NX>;
  constexpr int E = F::E, LANES = F::LANES, LPW = F::LPW, H = NX / 2;
  __shared__ float2 s_tw[F::TW];
  extern __shared__ __align__(128) float2 s_buf[];
  for (int i = threadIdx.x; i < F::TW; i += W_ROT * 32) s_tw[i] = twx[i];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int li = lane % LANES, line = lane / LANES;
  const int y = (blockIdx.x * W_ROT + warp) * LPW + line;
  const bool active = y < ny;
  const size_t row = (size_t)(active ? y : 0) * NX;
  __syncthreads();
  pdl_wait();  // u, v are written by the previous kernel
  pdl_trigger();
  float2 x[E];
#pragma unroll
  for (int m = 0; m < E; ++m) x[m] = make_float2(u[row + li + LANES * m], v[row + li + LANES * m]);
  float2* wbuf = s_buf + warp * warp_stride<NX>();
  fft_line<NX, false>(x, wbuf, s_tw, li, line);
  float2* lb = wbuf + line * F::PAD_LINE;
#pragma unroll
  for (int m = 0; m < E; ++m) lb[F::pad(li + LANES * m)] = x[m];
  __syncwarp();
  if (!active) return;
  float2* tu = Su + (size_t)y * pT;
  float2* tv = Sv + (size_t)y * pT;
  for (int k = li; k <= H; k += LANES) {
    const float2 a = lb[F::pad(k)];
    const float2 b = lb[F::pad(k == 0 ? 0 : NX - k)];
    // U = (X_k + conj X_{-k}) / 2, V = (X_k - conj X_{-k}) / (2i)
    tu[k] = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
    tv[k] = make_float2(0.5f * (a.y + b.y), -0.5f * (a.x - b.x));
  }
}

// S2: columns c0 .. c0 + CW of the row spectra Su, Sv ([NY][pT]): forward
// FFT along y of both (stage 0 cooperatively: thread q takes column q % CW,
// butterfly q / CW, so loads are row segments of CW adjacent columns; the
// other stages by the column's own lanes, leaving the column's spectrum in
// natural order in registers), the flow over time t (omega table W,
// [ncols][NY]), the 1/(nx ny) of the unnormalised transforms, then the
// inverse FFT along y of both back into Su, Sv (last stage cooperatively:
// stores are row segments too).  Each CTA reads and writes only its own
// columns, so the pass runs in place.
// The flow over t comes from a table of (c, r, q) = (cos wt, sin(wt)/w,
// w sin wt) per mode (k_flow_table; t for w = 0 in r), [3][ncols][NY];
// sign = -1 runs it backwards (the flow over -t: r and q change sign).
template <int NY>
__global__ void __launch_bounds__(W_ROT * 32) k2d_rot_cols(float2* __restrict__ Su, float2* __restrict__ Sv,
                                                           const float* __restrict__ tab, float sign, float invN,
                                                           int pT, int ncols, const float2* __restrict__ twy) {
  using F = LineFFT<NY>;
  constexpr int E = F::E, LANES = F::LANES, LPW = F::LPW, BPL = F::BPL, RL = F::RL, NBL = F::NBL;
  constexpr int THREADS = W_ROT * 32, CW = W_ROT * LPW;  // columns per CTA
  constexpr int SET = W_ROT * warp_stride<NY>();
  static_assert(CW * LANES == THREADS, "one stage-0 butterfly per thread");
  __shared__ float2 s_tw[F::TW];
  extern __shared__ __align__(128) float2 s_buf[];  // [field][warp] exchange buffers
  for (int i = threadIdx.x; i < F::TW; i += THREADS) s_tw[i] = twy[i];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int li = lane % LANES, line = lane / LANES;
  const int c0 = blockIdx.x * CW;
  const int cc = min(c0 + warp * LPW + line, ncols - 1);
  const long long tsz = (long long)ncols * NY;
  pdl_wait();  // Su, Sv are written by k2d_rot_fwd_rows
  pdl_trigger();
  float2* lbu = s_buf + warp * warp_stride<NY>() + line * F::PAD_LINE;
  float2* lbv = lbu + SET;
  {
    const int fc = threadIdx.x % CW, j = threadIdx.x / CW;
    const int col = min(c0 + fc, ncols - 1);
    float2* lb = s_buf + (fc / LPW) * warp_stride<NY>() + (fc % LPW) * F::PAD_LINE;
    float2 x[E];
#pragma unroll
    for (int r = 0; r < E; ++r) x[r] = Su[(size_t)(j + LANES * r) * pT + col];
    stage0_to_smem<NY, false>(x, lb, j);
#pragma unroll
    for (int r = 0; r < E; ++r) x[r] = Sv[(size_t)(j + LANES * r) * pT + col];
    stage0_to_smem<NY, false>(x, lb + SET, j);
  }
  __syncthreads();  // twiddles; every column's stage 0 in place
  mid_stage<NY, false>(lbu, s_tw, li);
  mid_stage<NY, false>(lbv, s_tw, li);
  __syncwarp();
  float2 a[E], b[E];
#pragma unroll
  for (int q = 0; q < BPL; ++q) {
    float2 w[RL];
    stage1_from_smem<NY, false>(w, lbu, s_tw, li + LANES * q);
#pragma unroll
    for (int r = 0; r < RL; ++r) a[q + BPL * r] = w[r];
    stage1_from_smem<NY, false>(w, lbv, s_tw, li + LANES * q);
#pragma unroll
    for (int r = 0; r < RL; ++r) b[q + BPL * r] = w[r];
  }
  // the flow, element y = li + LANES m of the column (natural order)
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const size_t i = (size_t)cc * NY + li + LANES * m;
    const float cs = tab[i], r = sign * tab[tsz + i], ws = sign * tab[2 * tsz + i];
    const float2 p = a[m], q = b[m];
    const float2 p2 = make_float2(fmaf(p.x, cs, q.x * r), fmaf(p.y, cs, q.y * r));
    const float2 q2 = make_float2(fmaf(q.x, cs, -p.x * ws), fmaf(q.y, cs, -p.y * ws));
    a[m] = cscale(p2, invN);
    b[m] = cscale(q2, invN);
  }
  __syncwarp();  // the line's stage-1 reads are done before its buffers are rewritten
  stage0_to_smem<NY, true>(a, lbu, li);
  mid_stage<NY, true>(lbu, s_tw, li);
  stage0_to_smem<NY, true>(b, lbv, li);
  mid_stage<NY, true>(lbv, s_tw, li);
  __syncthreads();
  // last stage cooperatively: thread q takes column q % CW, butterfly q / CW
#pragma unroll
  for (int q = 0; q < BPL; ++q) {
    const int bb = threadIdx.x + THREADS * q;
    const int sc = bb % CW, sj = bb / CW;
    const float2* lb = s_buf + (sc / LPW) * warp_stride<NY>() + (sc % LPW) * F::PAD_LINE;
    float2 w[RL];
    const bool store = c0 + sc < ncols;
    stage1_from_smem<NY, true>(w, lb, s_tw, sj);
    if (store) {
#pragma unroll
      for (int r = 0; r < RL; ++r) Su[(size_t)(sj + r * NBL) * pT + c0 + sc] = w[r];
    }
    stage1_from_smem<NY, true>(w, lb + SET, s_tw, sj);
    if (store) {
#pragma unroll
      for (int r = 0; r < RL; ++r) Sv[(size_t)(sj + r * NBL) * pT + c0 + sc] = w[r];
    }
  }
}

// S3: rows of Su, Sv -> u, v (in place of the state)
template <int NX>
__global__ void __launch_bounds__(W_ROT * 32) k2d_rot_inv_rows(const float2* __restrict__ Su,
                                                               const float2* __restrict__ Sv, float* __restrict__ u,
                                                               float* __restrict__ v, int ny, int pT,
                                                               const float2* __restrict__ twx) {
  using F = LineFFT<NX>;
  constexpr int E = F::E, LANES = F::LANES, LPW = F::LPW, H = NX / 2;
  __shared__ float2 s_tw[F::TW];
  extern __shared__ __align__(128) float2 s_buf[];
  for (int i = threadIdx.x; i < F::TW; i += W_ROT * 32) s_tw[i] = twx[i];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int li = lane % LANES, line = lane / LANES;
  const int y = (blockIdx.x * W_ROT + warp) * LPW + line;
  const bool active = y < ny;
  const float2* su = Su + (size_t)(active ? y : 0) * pT;
  const float2* sv = Sv + (size_t)(active ? y : 0) * pT;
  __syncthreads();
  pdl_wait();  // Su, Sv are written by k2d_rot_cols
  pdl_trigger();
  // Hermitian extensions: X[n] = A[n] + i B[n], A[NX - n] = conj A[n]
  float2 x[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int n = li + LANES * m;
    if (n <= H) {
      const float2 p = su[n], q = sv[n];
      x[m] = (n == 0 || n == H) ? make_float2(p.x, q.x) : make_float2(p.x - q.y, p.y + q.x);
    } else {
      const float2 p = su[NX - n], q = sv[NX - n];
      x[m] = make_float2(p.x + q.y, q.x - p.y);
    }
  }
  fft_line<NX, true>(x, s_buf + warp * warp_stride<NX>(), s_tw, li, line);
  if (!active) return;
  const size_t row = (size_t)y * NX;
#pragma unroll
  for (int m = 0; m < E; ++m) {
    u[row + li + LANES * m] = x[m].x;
    v[row + li + LANES * m] = x[m].y;
  }
}

// The flow table over time t from the frequencies W (float, [ncols][ny]),
// in double: (cos wt, sin(wt)/w, w sin wt), and (1, t, 0) where w = 0.
__global__ void k_flow_table(const float* __restrict__ W, double t, float* __restrict__ tab, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double w = (double)W[i];
    if (w > 0.0) {
      double sn, cs;
      sincos(w * t, &sn, &cs);
      tab[i] = (float)cs;
      tab[n + i] = (float)(sn / w);
      tab[2 * n + i] = (float)(w * sn);
    } else {
      tab[i] = 1.f;
      tab[n + i] = (float)t;
      tab[2 * n + i] = 0.f;
    }
  }
}

// The kick alone (M = 0: no variable-order remainder), pointwise:
// v += dt f(u), f(u) = f1 u + f3 u^3
__global__ void k2d_kick_f(const float* __restrict__ u, float* __restrict__ v, long long n, float dt, float f1, float f3) {
  pdl_wait();
  pdl_trigger();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float x = u[i];
    v[i] = v[i] + dt * (f1 * x + f3 * x * x * x);
  }
}

}  // namespace
}  // namespace vofl
