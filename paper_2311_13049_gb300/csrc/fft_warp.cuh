// fft_warp.cuh -- register-resident complex FFT of one line by a group of
// lanes of a warp, for the spectral transforms of the matrix-free scheme
// (Eq. (2.13) of arXiv 2311.13049: one forward transform of u, then one
// inverse transform per Taylor term).
//
// Algorithm: Stockham autosort, two radix stages N = R0 * R1 (Govindaraju et
// al., "High performance discrete Fourier transforms on graphics processors",
// SC 2008, restated here for a register/warp mapping):
//   stage 0 (Ns = 1, radix R0 = E): every lane holds E elements in registers
//     and does one DFT-E; no twiddles;
//   exchange through shared memory (one write, one read per element);
//   stage 1 (Ns = E, radix R1 = LANES): E/LANES butterflies per lane, each
//     with twiddles w_N^{r k}, k = j mod E, then a DFT-R1.
// A line of N complex values is owned by LANES = N/E consecutive lanes; lane
// li of the line holds element m at line index li + LANES*m, on input AND on
// output (natural order, no bit reversal).  Global loads/stores of that
// pattern are coalesced (LANES consecutive elements per instruction).
//
// Shared-memory layout of the exchange: element a of a line sits at
// a + a/E (one pad slot per E elements), which makes both the stage-0 writes
// (stride E between lanes) and the stage-1 reads (consecutive) conflict-free
// for E in {8, 16, 32}.
//
// Twiddles come from a per-size table tw[r][k] = exp(-2 pi i r k / N),
// r < R1, k < E, generated in double and rounded to float; the inverse uses
// the conjugate.  The in-register DFT-R is a compile-time radix-2
// decimation-in-time recursion whose trivial twiddles (1, -i, -1, i) are
// folded away.
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

// cos(2 pi a / 32), a = 0..31 (double literals rounded to float at compile time)
struct Cos32 {
  static constexpr double v[32] = {
      1.0, 0.98078528040323044913, 0.92387953251128675613, 0.83146961230254523708,
      0.70710678118654752440, 0.55557023301960222474, 0.38268343236508977173, 0.19509032201612826785,
      0.0, -0.19509032201612826785, -0.38268343236508977173, -0.55557023301960222474,
      -0.70710678118654752440, -0.83146961230254523708, -0.92387953251128675613, -0.98078528040323044913,
      -1.0, -0.98078528040323044913, -0.92387953251128675613, -0.83146961230254523708,
      -0.70710678118654752440, -0.55557023301960222474, -0.38268343236508977173, -0.19509032201612826785,
      0.0, 0.19509032201612826785, 0.38268343236508977173, 0.55557023301960222474,
      0.70710678118654752440, 0.83146961230254523708, 0.92387953251128675613, 0.98078528040323044913};
};

// v * exp(-/+ 2 pi i K / R) (forward: minus, INV: plus), K, R compile-time.
template <int R, int K, bool INV>
__device__ __forceinline__ float2 twiddle_const(float2 v) {
  constexpr int a = ((K * (32 / R)) % 32 + 32) % 32;  // angle in units of 2 pi / 32
  if constexpr (a == 0) {
    return v;
  } else if constexpr (a == 16) {
    return make_float2(-v.x, -v.y);
  } else if constexpr (a == 8) {
    // forward: * (-i); inverse: * (+i)
    return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
  } else if constexpr (a == 24) {
    return INV ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
  } else {
    constexpr float c = (float)Cos32::v[a];
    constexpr float s = (float)Cos32::v[(a + 24) % 32];  // sin(2 pi a/32) = cos(2 pi (a-8)/32)
    // forward: (c - i s); inverse: (c + i s)
    if constexpr (INV) {
      return make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.y, c, v.x * s));
    } else {
      return make_float2(fmaf(v.x, c, v.y * s), fmaf(v.y, c, -v.x * s));
    }
  }
}

template <int R, int K, bool INV>
__device__ __forceinline__ void butterflies(float2* v, const float2* e, const float2* o) {
  if constexpr (K < R / 2) {
    const float2 t = twiddle_const<R, K, INV>(o[K]);
    v[K] = cadd(e[K], t);
    v[K + R / 2] = csub(e[K], t);
    butterflies<R, K + 1, INV>(v, e, o);
  }
}

// In-register DFT of length R (power of two <= 32), natural order in and out.
template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v) {
  if constexpr (R == 1) {
    return;
  } else if constexpr (R == 2) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
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

// Static description of the two-stage line FFT of length N.
template <int N>
struct LineFFT {
  static_assert(N >= 64 && N <= 1024 && (N & (N - 1)) == 0, "line length must be a power of two in [64, 1024]");
  static constexpr int E = (N >= 512) ? 32 : (N >= 128 ? 16 : 8);  // elements per lane (radix of stage 0)
  static constexpr int LANES = N / E;                               // lanes per line (radix of stage 1)
  static constexpr int LPW = 32 / LANES;                            // lines per warp
  static constexpr int BPL = E / LANES;                             // stage-1 butterflies per lane
  static constexpr int PAD_LINE = N + N / E;                        // padded shared slots per line
  static constexpr int WARP_SLOTS = LPW * PAD_LINE;                 // shared float2 per warp
  static constexpr int TW = LANES * E;                              // twiddle table entries (= N)
  __device__ __forceinline__ static int pad(int a) { return a + a / E; }
};

// Stage 0 of the line transform for one lane: DFT-E over the lane's E
// elements v[r] = x[j + LANES r] (butterfly j), Stockham write of the result
// to the line buffer `lb` at pad(j E + r).
template <int N, bool INV>
__device__ __forceinline__ void stage0_to_smem(float2 (&v)[LineFFT<N>::E], float2* lb, int j) {
  using F = LineFFT<N>;
  constexpr int E = F::E;
  dft<E, INV>(v);
#pragma unroll
  for (int r = 0; r < E; ++r) lb[F::pad(j * E + r)] = v[r];
}

// Stage 1 butterfly j (0 <= j < E) of a line whose stage-0 output is in
// `lb`: inputs lb[pad(j + r E)], twiddles w_N^{r j}, DFT-LANES; on return
// w[r] = X[j + r E], r < LANES.
template <int N, bool INV>
__device__ __forceinline__ void stage1_from_smem(float2 (&w)[LineFFT<N>::LANES], const float2* lb,
                                                 const float2* __restrict__ tw, int j) {
  using F = LineFFT<N>;
  constexpr int E = F::E, LANES = F::LANES;
#pragma unroll
  for (int r = 0; r < LANES; ++r) w[r] = lb[F::pad(j + r * E)];
#pragma unroll
  for (int r = 1; r < LANES; ++r) {
    const float2 t = tw[r * E + j];
    w[r] = INV ? cmulc(w[r], t) : cmul(w[r], t);
  }
  dft<LANES, INV>(w);
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
  constexpr int LANES = F::LANES, BPL = F::BPL;
  float2* lb = buf + line * F::PAD_LINE;
  stage0_to_smem<N, INV>(v, lb, li);
  __syncwarp();
#pragma unroll
  for (int q = 0; q < BPL; ++q) {
    float2 w[LANES];
    stage1_from_smem<N, INV>(w, lb, tw, li + LANES * q);
    // outputs X[j + r E] = X[li + LANES (q + BPL r)]
#pragma unroll
    for (int r = 0; r < LANES; ++r) v[q + BPL * r] = w[r];
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
