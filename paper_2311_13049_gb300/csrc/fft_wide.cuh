// fft_wide.cuh -- the "wide" line FFT: a line of N = 512 or 1024 complex
// values spread over N/16 lanes (one warp at 512, two warps at 1024) with
// 16 elements per lane, for the spectral transforms of the matrix-free
// scheme (Eq. (2.13) of arXiv 2311.13049).
//
// The narrow form of fft_warp.cuh keeps 32 elements per lane (64 registers
// of data) and one warp per 1024-point line; this one halves the data
// registers and doubles the number of warps per line, so that the
// multiplier recurrence (column pass) or the Horner accumulators (row pass)
// fit beside the transform at four warps per SM sub-partition.
//
// Algorithm: Stockham autosort (Govindaraju et al., SC 2008) as in
// fft_warp.cuh, three stages N = 16 * R1 * 4 (R1 = N / 64):
//   stage 0 (Ns = 1, radix 16): lane j (0 <= j < LANES = N/16) does one
//     DFT-16 of its elements x[j + LANES r] in registers, no twiddles, and
//     writes output r to 16 j + r of buffer A;
//   stage 1 (Ns = 16, radix R1): 64 butterflies j (64 / LANES per lane)
//     read A[j + 64 r], r < R1, twiddle w_{16 R1}^{r (j mod 16)}, DFT-R1,
//     write output r to (j / 16) 16 R1 + (j mod 16) + 16 r of buffer B;
//   stage 2 (Ns = 16 R1 = N/4, radix 4): N/4 butterflies j read B[j + (N/4) r],
//     twiddle w_N^{r j}, DFT-4, and return X[j + (N/4) r] (natural order).
// Lane li of a line holds element li + LANES m (m < 16) on input and on
// output.  With butterfly j = li + LANES q in stage 2, output r of it is
// X[li + LANES (q + 4 r)], i.e. register m = q + 4 r.
//
// Buffers: two per line (A, B), element a at a + a/16 (one pad slot per 16
// elements: stage-0 writes at stride 17 between lanes and every other
// access at consecutive addresses are conflict-free).  Two buffers make two
// barriers per transform enough: the barrier after stage 1 also orders
// every lane's stage-1 reads of A before the next transform's stage-0
// writes, and the barrier after the next stage 0 orders every stage-2 read
// of B before the next stage-1 writes.
//
// Twiddles (generated in double, rounded to float; the inverse uses the
// conjugate): tw[r (N/4) + j] = w_N^{r j} (r < 4, j < N/4), then
// tw[N + r 16 + k] = w_{16 R1}^{r k} (r < R1, k < 16).
#pragma once
#include <cuda_runtime.h>

#include "fft_warp.cuh"

namespace vofl {

template <int N>
struct WideFFT {
  static_assert(N == 512 || N == 1024, "wide line transform: N = 512 or 1024");
  static constexpr int E = 16;               // elements per lane (stage-0 radix)
  static constexpr int LANES = N / E;        // lanes per line: 32 or 64
  static constexpr int WPL = LANES / 32;     // warps per line: 1 or 2
  static constexpr int R1 = N / 64;          // stage-1 radix: 8 or 16
  static constexpr int NB1 = 64;             // stage-1 butterflies per line
  static constexpr int BPL1 = NB1 / LANES;   // ... per lane: 2 or 1
  static constexpr int R2 = 4;               // stage-2 radix
  static constexpr int NB2 = N / R2;         // stage-2 butterflies per line
  static constexpr int BPL2 = NB2 / LANES;   // ... per lane: 4
  static constexpr int PAD_LINE = N + N / 16;  // padded float2 slots of one buffer
  static constexpr int TW = N + R1 * 16;       // twiddle table entries
  static_assert(E * R1 * R2 == N && BPL2 == 4, "wide line layout");
  __device__ __forceinline__ static int pad(int a) { return a + (a >> 4); }
};

// Barrier over the lanes of one line: the warp itself (N = 512), or the two
// warps of the line (named barrier `id`, 64 threads).
template <int N>
__device__ __forceinline__ void line_sync(int id) {
  if constexpr (WideFFT<N>::WPL == 1) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory");
  }
}

// line_sync that also returns whether any lane of the line passed `flag`
// set (a barrier reduction): every lane of the line takes the same branch
// afterwards, so a line never splits across a later barrier.
template <int N>
__device__ __forceinline__ bool line_sync_any(int id, bool flag) {
  if constexpr (WideFFT<N>::WPL == 1) {
    __syncwarp();
    return __any_sync(0xffffffffu, flag);
  } else {
    uint32_t any;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, 64, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(any)
        : "r"((uint32_t)flag), "r"(id)
        : "memory");
    return any != 0;
  }
}

// Stage 0: DFT-16 of the lane's elements, written to buffer A.
template <int N, bool INV>
__device__ __forceinline__ void wide_stage0(float2 (&v)[16], float2* A, int li) {
  dft<16, INV>(v);
  float2* o = A + li * 17;  // pad(16 li + r) = 17 li + r
#pragma unroll
  for (int r = 0; r < 16; ++r) o[r] = v[r];
}

// Stage 1 of the lanes' butterflies, A -> B.
template <int N, bool INV>
__device__ __forceinline__ void wide_stage1(const float2* A, float2* B, const float2* __restrict__ tw, int li) {
  using F = WideFFT<N>;
  constexpr int R1 = F::R1, LANES = F::LANES;
  const float2* tw1 = tw + N;
#pragma unroll
  for (int q = 0; q < F::BPL1; ++q) {
    const int j = li + LANES * q, k = j & 15;
    float2 x[R1];
#pragma unroll
    for (int r = 0; r < R1; ++r) x[r] = A[F::pad(j + 64 * r)];
#pragma unroll
    for (int r = 1; r < R1; ++r) {
      const float2 t = tw1[r * 16 + k];
      x[r] = INV ? cmulc(x[r], t) : cmul(x[r], t);
    }
    dft<R1, INV>(x);
    float2* o = B + F::pad((j >> 4) * 16 * R1 + k);  // + pad step of 16 r = 17 r
#pragma unroll
    for (int r = 0; r < R1; ++r) o[17 * r] = x[r];
  }
}

// Stage-2 butterfly j (0 <= j < N/4) from buffer B: on return
// w[r] = X[j + (N/4) r], r < 4.
template <int N, bool INV>
__device__ __forceinline__ void wide_stage2_bfly(float2 (&w)[4], const float2* B, const float2* __restrict__ tw,
                                                 int j) {
  using F = WideFFT<N>;
  constexpr int NB2 = F::NB2;
  constexpr int SP = NB2 + NB2 / 16;  // pad(j + NB2 r) = pad(j) + SP r
  const float2* in = B + F::pad(j);
#pragma unroll
  for (int r = 0; r < 4; ++r) w[r] = in[r * SP];
#pragma unroll
  for (int r = 1; r < 4; ++r) {
    const float2 t = tw[r * NB2 + j];
    w[r] = INV ? cmulc(w[r], t) : cmul(w[r], t);
  }
  dft<4, INV>(w);
}

// Transform one line: v[m] = x[li + LANES m] on entry, X[li + LANES m] on
// exit.  A, B: the line's two buffers; bar: the line's named barrier id
// (N = 1024).  Every lane of the line must call it together.
template <int N, bool INV>
__device__ __forceinline__ void wide_fft(float2 (&v)[16], float2* A, float2* B, const float2* __restrict__ tw, int li,
                                         int bar) {
  using F = WideFFT<N>;
  wide_stage0<N, INV>(v, A, li);
  line_sync<N>(bar);
  wide_stage1<N, INV>(A, B, tw, li);
  line_sync<N>(bar);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float2 w[4];
    wide_stage2_bfly<N, INV>(w, B, tw, li + F::LANES * q);
#pragma unroll
    for (int r = 0; r < 4; ++r) v[q + 4 * r] = w[r];
  }
}

}  // namespace vofl
