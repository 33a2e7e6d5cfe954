// fft_warp.cuh -- register-resident complex FFT of one line by a group of
// lanes of a warp, for the spectral transforms of the matrix-free scheme
// (Eq. (2.13) of arXiv 2311.13049: one forward transform of u, then one
// inverse transform per Taylor term).
//
// Algorithm: Stockham autosort (Govindaraju et al., "High performance
// discrete Fourier transforms on graphics processors", SC 2008, restated
// here for a register/warp mapping).  A stage of radix R at span Ns takes
// butterfly j (0 <= j < N/R) from x[j + r N/R], r < R, multiplies input r by
// w_{Ns R}^{r (j mod Ns)}, does a DFT-R and writes output r to
// (j / Ns) Ns R + (j mod Ns) + r Ns.
//
// Power-of-two N (64..1024), two stages N = E * LANES:
//   stage 0 (Ns = 1, radix E): every lane holds E elements in registers and
//     does one DFT-E; no twiddles;
//   exchange through shared memory (one write, one read per element);
//   last stage (Ns = E, radix RL = LANES): NBL = E butterflies per line,
//     E/LANES per lane, twiddles w_N^{r j}.
// N = 768 = 24 * 8 * 4 (for grids with a factor 3), three stages, E = 24,
// LANES = 32:
//   stage 0 (Ns = 1, radix 24 = 3 * 8 in registers);
//   middle stage (Ns = 24, radix 8) in place in the warp's shared line
//     buffer, 3 butterflies per lane, twiddles w_192^{r (j mod 24)};
//   last stage (Ns = 192, radix RL = 4): NBL = 192 butterflies per line,
//     6 per lane, twiddles w_768^{r j}.
// In both cases the last stage's butterfly j returns X[j + NBL r], r < RL.
// A line of N complex values is owned by LANES = N/E consecutive lanes; lane
// li of the line holds element m at line index li + LANES*m, on input AND on
// output (natural order, no bit reversal).  Global loads/stores of that
// pattern are coalesced (LANES consecutive elements per instruction).
//
// Shared-memory layout of the exchange: element a of a line sits at
// a + a/E (one pad slot per E elements), which makes the stage-0 writes
// (stride E between lanes) and the later reads (consecutive) conflict-free
// for E in {8, 16, 32} and nearly so for E = 24.
//
// Twiddles come from a per-size table: tw[r NBL + j] = exp(-2 pi i r j / N)
// (r < RL, j < NBL), followed for N = 768 by exp(-2 pi i t / 192), t < 192;
// generated in double and rounded to float; the inverse uses the conjugate.
// The in-register DFT-R is a compile-time decimation-in-time recursion
// (radix 2, and one radix-3 split for R = 3 * 2^k) whose constant twiddles
// are evaluated at compile time; the trivial ones (1, -i, -1, i) are folded
// away.
#pragma once
#include <cuda_runtime.h>

namespace vofl {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// a * b
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// cos and sin of 2 pi a / R at compile time: Taylor series about the
// nearest multiple of pi/2 (|x| <= pi/4 there; 20 terms are far below double
// round-off), then rounded once to float by the caller.
constexpr double kHalfPi = 1.5707963267948966192313216916398;
constexpr double taylor_cos(double x) {
  double t = 1.0, s = 1.0;
  for (int i = 1; i < 20; ++i) {
    t *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
    s += t;
  }
  return s;
}
constexpr double taylor_sin(double x) {
  double t = x, s = x;
  for (int i = 1; i < 20; ++i) {
    t *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
    s += t;
  }
  return s;
}
// 2 pi a / R = q pi/2 + x, q the nearest integer to 4a/R (0 <= a < R)
constexpr int turn_quarter(int a, int R) { return (8 * a + R) / (2 * R); }
constexpr double turn_rest(int a, int R) { return kHalfPi * (double)(4 * a - turn_quarter(a, R) * R) / (double)R; }
constexpr double cos_turn(int a, int R) {
  const int q = turn_quarter(a, R) & 3;
  const double x = turn_rest(a, R);
  return q == 0 ? taylor_cos(x) : q == 1 ? -taylor_sin(x) : q == 2 ? -taylor_cos(x) : taylor_sin(x);
}
constexpr double sin_turn(int a, int R) {
  const int q = turn_quarter(a, R) & 3;
  const double x = turn_rest(a, R);
  return q == 0 ? taylor_sin(x) : q == 1 ? taylor_cos(x) : q == 2 ? -taylor_sin(x) : -taylor_cos(x);
}

// v * exp(-/+ 2 pi i K / R) (forward: minus, INV: plus), K, R compile-time.
template <int R, int K, bool INV>
__device__ __forceinline__ float2 twiddle_const(float2 v) {
  constexpr int a = ((K % R) + R) % R;
  if constexpr (a == 0) {
    return v;
  } else if constexpr (2 * a == R) {
    return make_float2(-v.x, -v.y);
  } else if constexpr (4 * a == R) {
    // forward: * (-i); inverse: * (+i)
    return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
  } else if constexpr (4 * a == 3 * R) {
    return INV ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
  } else {
    constexpr float c = (float)cos_turn(a, R);
    constexpr float s = (float)sin_turn(a, R);
    // forward: (c - i s); inverse: (c + i s)
    if constexpr (INV) {
      return make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.y, c, v.x * s));
    } else {
      return make_float2(fmaf(v.x, c, v.y * s), fmaf(v.y, c, -v.x * s));
    }
  }
}

// Radix-2 butterflies of a DFT-R level: v[K] = e[K] + w^K o[K],
// v[K + R/2] = e[K] - w^K o[K], w = exp(-/+ 2 pi i / R).  Trivial twiddles
// (1, -i, -1, i) cost additions only; the others are fused into FMAs:
// x = e + w o in four FMAs, then e - w o = 2e - x in two (six instructions
// instead of a complex multiply and two complex additions).
template <int R, int K, bool INV>
__device__ __forceinline__ void butterflies(float2* v, const float2* e, const float2* o) {
  if constexpr (K < R / 2) {
    constexpr int a = ((K % R) + R) % R;
    if constexpr (a == 0 || 2 * a == R || 4 * a == R || 4 * a == 3 * R) {
      const float2 t = twiddle_const<R, K, INV>(o[K]);
      v[K] = cadd(e[K], t);
      v[K + R / 2] = csub(e[K], t);
    } else {
      constexpr float wr = (float)cos_turn(a, R);
      constexpr float wi = INV ? (float)sin_turn(a, R) : -(float)sin_turn(a, R);
      const float2 ek = e[K], ok = o[K];
      const float2 x = make_float2(fmaf(wr, ok.x, fmaf(-wi, ok.y, ek.x)), fmaf(wr, ok.y, fmaf(wi, ok.x, ek.y)));
      v[K] = x;
      v[K + R / 2] = make_float2(fmaf(2.0f, ek.x, -x.x), fmaf(2.0f, ek.y, -x.y));
    }
    butterflies<R, K + 1, INV>(v, e, o);
  }
}

// DFT-3 of (a, b, c): x0 = a + b + c, x1 = a + w b + w^2 c,
// x2 = a + w^2 b + w c, w = exp(-/+ 2 pi i / 3).
template <bool INV>
__device__ __forceinline__ void bfly3(float2 a, float2 b, float2 c, float2& x0, float2& x1, float2& x2) {
  constexpr float h = 0.86602540378443864676f;  // sqrt(3) / 2
  const float2 s = cadd(b, c);
  const float2 t = make_float2(fmaf(-0.5f, s.x, a.x), fmaf(-0.5f, s.y, a.y));
  const float2 d = make_float2(h * (b.x - c.x), h * (b.y - c.y));
  x0 = cadd(a, s);
  // forward: x1 = t - i d, x2 = t + i d; inverse: the other way round
  const float2 m = make_float2(t.x + d.y, t.y - d.x), p = make_float2(t.x - d.y, t.y + d.x);
  x1 = INV ? p : m;
  x2 = INV ? m : p;
}

template <int R, int K, bool INV>
__device__ __forceinline__ void radix3_combine(float2* v, const float2* s0, const float2* s1, const float2* s2) {
  if constexpr (K < R / 3) {
    bfly3<INV>(s0[K], twiddle_const<R, K, INV>(s1[K]), twiddle_const<R, 2 * K, INV>(s2[K]), v[K], v[K + R / 3],
               v[K + 2 * R / 3]);
    radix3_combine<R, K + 1, INV>(v, s0, s1, s2);
  }
}

// In-register DFT of length R (2^k <= 32 or 3 * 2^k), natural order in and out.
template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v) {
  if constexpr (R == 1) {
    return;
  } else if constexpr (R == 2) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if constexpr (R == 3) {
    bfly3<INV>(v[0], v[1], v[2], v[0], v[1], v[2]);
  } else if constexpr (R % 3 == 0) {
    float2 s0[R / 3], s1[R / 3], s2[R / 3];
#pragma unroll
    for (int i = 0; i < R / 3; ++i) {
      s0[i] = v[3 * i];
      s1[i] = v[3 * i + 1];
      s2[i] = v[3 * i + 2];
    }
    dft<R / 3, INV>(s0);
    dft<R / 3, INV>(s1);
    dft<R / 3, INV>(s2);
    radix3_combine<R, 0, INV>(v, s0, s1, s2);
  } else {
    float2 e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    dft<R / 2, INV>(e);
    dft<R / 2, INV>(o);
    butterflies<R, 0, INV>(v, e, o);
  }
}

// Static description of the line FFT of length N.
template <int N>
struct LineFFT {
  static constexpr bool MIXED = (N == 768);
  static_assert(MIXED || (N >= 64 && N <= 1024 && (N & (N - 1)) == 0),
                "line length must be a power of two in [64, 1024] or 768");
  static constexpr int E = MIXED ? 24 : (N >= 512) ? 32 : (N >= 128 ? 16 : 8);  // elements per lane (stage-0 radix)
  static constexpr int LANES = N / E;                                            // lanes per line
  static constexpr int LPW = 32 / LANES;                                         // lines per warp
  static constexpr int RL = MIXED ? 4 : LANES;                                   // radix of the last stage
  static constexpr int NBL = N / RL;                                             // last-stage butterflies per line
  static constexpr int BPL = NBL / LANES;                                        // ... per lane
  static constexpr int RM = MIXED ? 8 : 1;                                       // radix of the middle stage
  static constexpr int BPM = MIXED ? N / (RM * LANES) : 0;                       // middle butterflies per lane
  static constexpr int TW_MID = MIXED ? E * RM : 0;                              // middle twiddle entries
  static constexpr int TW = N + TW_MID;                                          // twiddle table entries
  static constexpr int PAD_LINE = N + N / E;                                     // padded shared slots per line
  static constexpr int WARP_SLOTS = LPW * PAD_LINE;                              // shared float2 per warp
  static_assert(LANES * LPW == 32 && NBL % LANES == 0 && E * RM * RL == N, "line layout");
  __device__ __forceinline__ static int pad(int a) { return a + a / E; }
};

// Stockham write of stage 0's output (butterfly j) to the line buffer `lb`
// at pad(j E + r).
template <int N>
__device__ __forceinline__ void stage0_write(const float2 (&v)[LineFFT<N>::E], float2* lb, int j) {
  constexpr int E = LineFFT<N>::E;
  float2* o = lb + j * (E + 1);  // pad(j E + r) = j (E + 1) + r
#pragma unroll
  for (int r = 0; r < E; ++r) o[r] = v[r];
}

// Stage 0 of the line transform for one lane: DFT-E over the lane's E
// elements v[r] = x[j + LANES r] (butterfly j), then its Stockham write.
template <int N, bool INV>
__device__ __forceinline__ void stage0_to_smem(float2 (&v)[LineFFT<N>::E], float2* lb, int j) {
  dft<LineFFT<N>::E, INV>(v);
  stage0_write<N>(v, lb, j);
}

// Middle stage (N = 768 only; no-op otherwise), in place in the line buffer
// `lb` of the calling lanes' line, li the lane index inside the line; the
// middle twiddles start at tw + N.  Contains __syncwarp(); all 32 lanes must
// call it together, after stage 0 of their line is in `lb`.
template <int N, bool INV>
__device__ __forceinline__ void mid_stage(float2* lb, const float2* __restrict__ tw, int li) {
  using F = LineFFT<N>;
  if constexpr (F::MIXED) {
    constexpr int E = F::E, RM = F::RM, BPM = F::BPM, LANES = F::LANES, S = N / RM;
    static_assert(S % E == 0, "middle-stage stride");
    constexpr int SP = S + S / E;  // pad(a + r S) = pad(a) + r SP
    const float2* twm = tw + N;
    __syncwarp();
    float2 x[BPM][RM];
#pragma unroll
    for (int q = 0; q < BPM; ++q) {
      const int j = li + LANES * q, k = j % E;
      const float2* in = lb + F::pad(j);
#pragma unroll
      for (int r = 0; r < RM; ++r) x[q][r] = in[r * SP];
#pragma unroll
      for (int r = 1; r < RM; ++r) {
        const float2 t = twm[r * k];
        x[q][r] = INV ? cmulc(x[q][r], t) : cmul(x[q][r], t);
      }
      dft<RM, INV>(x[q]);
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < BPM; ++q) {
      const int j = li + LANES * q, k = j % E;
      float2* out = lb + (j / E) * (E + 1) * RM + k;  // pad((j/E) E RM + k + r E)
#pragma unroll
      for (int r = 0; r < RM; ++r) out[r * (E + 1)] = x[q][r];
    }
  }
}

// Last-stage butterfly j (0 <= j < NBL) of a line whose previous stages are
// in `lb`: inputs lb[pad(j + r NBL)], twiddles w_N^{r j}, DFT-RL; on return
// w[r] = X[j + r NBL], r < RL.
template <int N, bool INV>
__device__ __forceinline__ void stage1_from_smem(float2 (&w)[LineFFT<N>::RL], const float2* lb,
                                                 const float2* __restrict__ tw, int j) {
  using F = LineFFT<N>;
  constexpr int NBL = F::NBL, RL = F::RL;
  static_assert(NBL % F::E == 0, "last-stage stride");
  constexpr int SP = NBL + NBL / F::E;  // pad(j + r NBL) = pad(j) + r SP
  const float2* in = lb + F::pad(j);
#pragma unroll
  for (int r = 0; r < RL; ++r) w[r] = in[r * SP];
#pragma unroll
  for (int r = 1; r < RL; ++r) {
    const float2 t = tw[r * NBL + j];
    w[r] = INV ? cmulc(w[r], t) : cmul(w[r], t);
  }
  dft<RL, INV>(w);
}

// Transform one line in place.  v[m] = x[li + LANES*m] on entry and
// X[li + LANES*m] on exit.  `buf` is the warp's exchange buffer
// (LineFFT<N>::WARP_SLOTS float2), `tw` the twiddle table (shared or global),
// li the lane index inside its line, line the line index inside the warp.
// Contains __syncwarp(); all 32 lanes must call it together.
template <int N, bool INV>
__device__ __forceinline__ void fft_line(float2 (&v)[LineFFT<N>::E], float2* buf, const float2* __restrict__ tw,
                                         int li, int line) {
  using F = LineFFT<N>;
  constexpr int LANES = F::LANES, BPL = F::BPL, RL = F::RL;
  float2* lb = buf + line * F::PAD_LINE;
  stage0_to_smem<N, INV>(v, lb, li);
  mid_stage<N, INV>(lb, tw, li);
  __syncwarp();
#pragma unroll
  for (int q = 0; q < BPL; ++q) {
    float2 w[RL];
    stage1_from_smem<N, INV>(w, lb, tw, li + LANES * q);
    // outputs X[j + r NBL] = X[li + LANES (q + BPL r)]
#pragma unroll
    for (int r = 0; r < RL; ++r) v[q + BPL * r] = w[r];
  }
  __syncwarp();
}

// Integer power by squaring (n >= 0).
__device__ __forceinline__ float powi(float x, int n) {
  float r = 1.f;
  while (n) {
    if (n & 1) r *= x;
    x *= x;
    n >>= 1;
  }
  return r;
}

}  // namespace vofl
