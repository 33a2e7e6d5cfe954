// kernels.cuh -- the fused transform kernels shared by the 2D and 3D paths
// (see fused2d.cu for the data path).  Included by fused2d.cu and
// fused3d.cu; everything has internal linkage.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "fft_warp.cuh"
#include "internal.h"
#include "tma.cuh"

namespace vofl {

namespace {

// CTA sizes (warps) per kernel
constexpr int W_FROWS = 1;  // forward rows: one-warp CTAs, 512 of them at 1024^2
constexpr int W_FCOLS = 4;  // forward columns: 4 columns -> 32-byte row segments
constexpr int W_YCOLS = 4;  // 3D y-inverse kernel
constexpr int W_IROWS = 4;  // inverse row kernel

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

template <int N>
constexpr int warp_stride() {
  // consecutive warp buffers start 2 (mod 16) float2 slots apart, so a
  // half-warp reading one element from each of 8 warp buffers for 2
  // consecutive rows touches 16 distinct bank pairs
  return (LineFFT<N>::WARP_SLOTS + 15) / 16 * 16 + 2;
}
template <int N, int W>
constexpr size_t exch_smem() {
  return (size_t)W * warp_stride<N>() * sizeof(float2);
}

// The multiplier/inverse column kernel: long lines (E >= 24 elements per
// lane: one CTA per SM whatever its size) transform two Taylor terms at a
// time in CTAs of 8 warps; short lines one term at a time in CTAs of 4
// warps, so that several CTAs share an SM.
template <int N>
constexpr bool icols_pair() {
  return LineFFT<N>::E >= 24;
}
// Warps (columns) per CTA of the narrow column kernel: 8 at 1024 points
// (65 column blocks x 2 operators = 130 CTAs of one per SM; 4-warp CTAs two
// per SM measured 10% slower), 4 elsewhere (768: 194 CTAs instead of 98).
template <int N>
constexpr int icols_warps() {
  return N == 1024 ? 8 : 4;
}
// float2 slots of one exchange set of the column kernel: its warps'
// buffers, rounded to 128 bytes (the second set of the paired form is a
// tensor-copy source)
template <int N>
constexpr int icols_set() {
  return (icols_warps<N>() * warp_stride<N>() + 15) / 16 * 16;
}

// -------------------------------------------------------------------------
// F1: forward FFT along x of two rows at once, split into half spectra.
// The rows the stencil needs (the pair, its y neighbours and, in 3D, the
// pair in the z-neighbour planes) are copied into shared memory by TMA bulk
// copies (one mbarrier per line, bounded wait) right after the
// programmatic wait: one round trip instead of dependent global loads.
// -------------------------------------------------------------------------
template <bool Z3>
constexpr int frows_nrows() {
  return Z3 ? 8 : 4;
}
template <int NX, bool Z3, int W = W_FROWS>
constexpr size_t frows_smem() {
  return exch_smem<NX, W>() + (size_t)W * LineFFT<NX>::LPW * frows_nrows<Z3>() * NX * sizeof(float);
}

// W: warps per CTA (bx counts blocks of W warps)
template <int NX, bool Z3, int W = W_FROWS>
__device__ __forceinline__ void fwd_rows_body(int bx, const float* __restrict__ u, float2* __restrict__ T, int ny,
                                              int nz, int pT, float ryy, float rzz, const float2* __restrict__ twx,
                                              int* step_ctr, int inc_step, int* err) {
  using F = LineFFT<NX>;
  constexpr int E = F::E, LANES = F::LANES, LPW = F::LPW, H = NX / 2, THREADS = W * 32;
  constexpr int NR = frows_nrows<Z3>();
  constexpr uint32_t ROWB = NX * sizeof(float);
  __shared__ float2 s_tw[F::TW];
  __shared__ uint64_t s_rbar[W * LPW];
  extern __shared__ __align__(128) float2 s_buf[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int li = lane % LANES, line = lane / LANES;
  const int lid = warp * LPW + line;
  uint64_t* bar = &s_rbar[lid];
  // rows of this line: 0 y-1, 1 y0, 2 y0+1, 3 y0+2 [, 4-5 the pair at z-1, 6-7 at z+1]
  float* srow = reinterpret_cast<float*>(s_buf + W * warp_stride<NX>()) + (size_t)lid * NR * NX;
  if (li == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < F::TW; i += THREADS) s_tw[i] = twx[i];
  __syncthreads();
  pdl_wait();  // u is written by the previous step's last kernel
  pdl_trigger();
  if (inc_step && bx == 0 && threadIdx.x == 0) *step_ctr += 1;
  float2* wbuf = s_buf + warp * warp_stride<NX>();
  // rows are flattened over planes: row = z * ny + y (nz = 1 in 2D); a
  // pair of rows never straddles two planes (ny is even)
  const int pair = (bx * W + warp) * LPW + line;
  const bool active = pair < (ny / 2) * nz;
  const int r0i = 2 * (active ? pair : 0);
  const int yy = r0i % ny, zz = r0i / ny;
  if (li == 0 && active) {
    const float* plane = u + (size_t)zz * ny * NX;
    const float* r0 = plane + (size_t)yy * NX;
    mbar_arrive_expect_tx(bar, NR * ROWB);
    bulk_copy_g2s(srow + 0 * NX, plane + (size_t)(yy == 0 ? ny - 1 : yy - 1) * NX, ROWB, bar);
    bulk_copy_g2s(srow + 1 * NX, r0, ROWB, bar);
    bulk_copy_g2s(srow + 2 * NX, r0 + NX, ROWB, bar);
    bulk_copy_g2s(srow + 3 * NX, plane + (size_t)(yy + 2 == ny ? 0 : yy + 2) * NX, ROWB, bar);
    if constexpr (Z3) {
      const size_t pl = (size_t)ny * NX;  // plane stride
      const float* zm = r0 - (size_t)zz * pl + (size_t)(zz == 0 ? nz - 1 : zz - 1) * pl;
      const float* zp = r0 - (size_t)zz * pl + (size_t)(zz + 1 == nz ? 0 : zz + 1) * pl;
      bulk_copy_g2s(srow + 4 * NX, zm, ROWB, bar);
      bulk_copy_g2s(srow + 5 * NX, zm + NX, ROWB, bar);
      bulk_copy_g2s(srow + 6 * NX, zp, ROWB, bar);
      bulk_copy_g2s(srow + 7 * NX, zp + NX, ROWB, bar);
    }
  }
  const bool got = active ? mbar_wait_bounded(bar, 0, err) : true;
  if (!__all_sync(0xffffffffu, got)) {
    // give up (error word set): drain this line's copies (bounded), leave
    if (active && !got) mbar_wait_bounded(bar, 0, err);
    return;
  }
  // w = D_xx u + (h_x/h_y)^2 D_yy u [+ (h_x/h_z)^2 D_zz u] (second
  // differences, no 1/h^2): its DFT is lambda_k u_hat_k exactly, with
  // lambda_k = -4 sin^2(pi k1/nx) - 4 (h_x/h_y)^2 sin^2(pi k2/ny) [- ...];
  // 1/lambda_k is folded into the multiplier table.  On FP32 data the
  // neighbour differences are exact or carry a rounding relative to
  // themselves, so w's transform keeps the high-wavenumber content that an
  // FP32 transform of u would bury under round-off of size eps*|u|.
  const float* rm = srow;
  const float* r0 = srow + NX;
  const float* r1 = srow + 2 * NX;
  const float* rp = srow + 3 * NX;
  float2 v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int x = li + LANES * m;
    const int xm = x == 0 ? NX - 1 : x - 1, xp = x + 1 == NX ? 0 : x + 1;
    const float a = r0[x], b = r1[x];
    const float dxa = (r0[xp] - a) - (a - r0[xm]);
    const float dxb = (r1[xp] - b) - (b - r1[xm]);
    const float dya = (b - a) - (a - rm[x]);
    const float dyb = (rp[x] - b) - (b - a);
    float wa = dxa + ryy * dya, wb = dxb + ryy * dyb;
    if constexpr (Z3) {
      const float dza = (srow[6 * NX + x] - a) - (a - srow[4 * NX + x]);
      const float dzb = (srow[7 * NX + x] - b) - (b - srow[5 * NX + x]);
      wa = wa + rzz * dza;
      wb = wb + rzz * dzb;
    }
    v[m] = make_float2(wa, wb);
  }
  fft_line<NX, false>(v, wbuf, s_tw, li, line);
  float2* lb = wbuf + line * F::PAD_LINE;
#pragma unroll
  for (int m = 0; m < E; ++m) lb[F::pad(li + LANES * m)] = v[m];
  __syncwarp();
  float2* t0 = T + (size_t)r0i * pT;
  float2* t1 = t0 + pT;
  for (int k = li; k <= H; k += LANES) {
    const float2 a = lb[F::pad(k)];
    const float2 b = lb[F::pad(k == 0 ? 0 : NX - k)];
    // A = (X_k + conj X_{-k})/2 (row y0), B = (X_k - conj X_{-k})/(2i) (row y0+1)
    if (active) {
      t0[k] = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
      t1[k] = make_float2(0.5f * (a.y + b.y), -0.5f * (a.x - b.x));
    }
  }
}

template <int NX, bool Z3>
__global__ void __launch_bounds__(W_FROWS * 32) k2d_fwd_rows(const float* __restrict__ u, float2* __restrict__ T,
                                                             int ny, int nz, int pT, float ryy, float rzz,
                                                             const float2* __restrict__ twx, int* step_ctr,
                                                             int inc_step, int* err) {
  fwd_rows_body<NX, Z3>(blockIdx.x, u, T, ny, nz, pT, ryy, rzz, twx, step_ctr, inc_step, err);
}

// -------------------------------------------------------------------------
// F2: forward FFT along y of each half-spectrum column.  Stage 0 is done
// cooperatively by the CTA: thread b takes column b % CW, butterfly b / CW,
// so each load instruction reads row segments of CW adjacent columns of T
// (coalesced, no transposition pass); stage 1 is done by the warp owning
// the column, whose output is a contiguous column of Uh.  blockIdx.y runs
// over independent planes (strides in_plane, out_plane).
// -------------------------------------------------------------------------
// COHERENT: T was written earlier in the same launch by other CTAs (the
// two-pass forward kernel): its loads bypass L1 (ld.global.cg).
template <int NY, int W = W_FCOLS, bool COHERENT = false>
__device__ __forceinline__ void fwd_cols_body(int bx, const float2* __restrict__ T, int pT, float2* __restrict__ Uh,
                                              int ncols, const float2* __restrict__ twy) {
  using F = LineFFT<NY>;
  constexpr int E = F::E, LANES = F::LANES, LPW = F::LPW, BPL = F::BPL;
  constexpr int THREADS = W * 32, CW = W * LPW;  // columns per CTA
  __shared__ float2 s_tw[F::TW];
  extern __shared__ __align__(128) float2 s_buf[];
  for (int i = threadIdx.x; i < F::TW; i += THREADS) s_tw[i] = twy[i];
  pdl_wait();  // T is written by k2d_fwd_rows
  pdl_trigger();
  const int c0 = bx * CW;
  {
    // cooperative stage 0: one radix-E butterfly per thread
    const int cc = threadIdx.x % CW, j = threadIdx.x / CW;
    const int col = min(c0 + cc, ncols - 1);
    float2 v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const float2* src = T + (size_t)(j + LANES * r) * pT + col;
      v[r] = COHERENT ? __ldcg(src) : *src;
    }
    float2* lb = s_buf + (cc / LPW) * warp_stride<NY>() + (cc % LPW) * F::PAD_LINE;
    stage0_to_smem<NY, false>(v, lb, j);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int li = lane % LANES, line = lane / LANES;
  float2* lb = s_buf + warp * warp_stride<NY>() + line * F::PAD_LINE;
  mid_stage<NY, false>(lb, s_tw, li);
  __syncwarp();
  const int c = c0 + warp * LPW + line;
  if (c < ncols) {
    float2* dst = Uh + (size_t)c * NY;
#pragma unroll
    for (int q = 0; q < BPL; ++q) {
      float2 w[F::RL];
      stage1_from_smem<NY, false>(w, lb, s_tw, li + LANES * q);
#pragma unroll
      for (int r = 0; r < F::RL; ++r) dst[li + LANES * (q + BPL * r)] = w[r];
    }
  }
}

template <int NY>
__global__ void __launch_bounds__(W_FCOLS * 32) k2d_fwd_cols(const float2* __restrict__ T, int pT,
                                                             float2* __restrict__ Uh, int ncols,
                                                             const float2* __restrict__ twy, long long in_plane,
                                                             long long out_plane) {
  // blockIdx.y: independent planes (3D: one per z)
  fwd_cols_body<NY>(blockIdx.x, T + blockIdx.y * in_plane, pT, Uh + blockIdx.y * out_plane, ncols, twy);
}

// -------------------------------------------------------------------------
// F1 + F2 in one cooperative launch (every CTA resident at once): the
// forward row pass over blocks of W_FBOTH warps, a grid-wide barrier
// (bounded), then the forward column pass over blocks of W_FBOTH columns.
// The arithmetic of k2d_fwd_rows and k2d_fwd_cols, so the same bits, with
// one kernel boundary (launch ramp and drain) fewer per step.
// -------------------------------------------------------------------------
constexpr int W_FBOTH = 4;
template <int NX, int NY>
constexpr size_t fboth_smem() {
  return std::max(frows_smem<NX, false, W_FBOTH>(), exch_smem<NY, W_FBOTH>());
}
template <int NX, int NY>
__global__ void __launch_bounds__(W_FBOTH * 32) k2d_fwd_both(const float* __restrict__ u, float2* __restrict__ T,
                                                             float2* __restrict__ Uh, int ny, int pT, int ncols,
                                                             float ryy, const float2* __restrict__ twx,
                                                             const float2* __restrict__ twy, int* step_ctr,
                                                             int inc_step, int* err, unsigned long long* gbar) {
  constexpr int RB = W_FBOTH * LineFFT<NX>::LPW, CB = W_FBOTH * LineFFT<NY>::LPW;
  const int nrb = (ny / 2 + RB - 1) / RB, ncb = (ncols + CB - 1) / CB;
  for (int b = blockIdx.x; b < nrb; b += gridDim.x) {
    fwd_rows_body<NX, false, W_FBOTH>(b, u, T, ny, 1, pT, ryy, 0.f, twx, step_ctr, inc_step, err);
    __syncthreads();  // shared buffers free for the next block
  }
  grid_barrier_bounded(gbar, err);
  for (int b = blockIdx.x; b < ncb; b += gridDim.x) {
    fwd_cols_body<NY, W_FBOTH, true>(b, T, pT, Uh, ncols, twy);
    __syncthreads();
  }
}

// -------------------------------------------------------------------------
// I1: multiplier + inverse FFT along y, for terms [m_lo, m_hi) of one
// operator (blockIdx.y).  Output Z[s][op][y][c], s = m - m_lo.
// Each warp keeps its column's multiplied spectrum
// v_m = u_hat P ln|mu|^{2m}/m! in registers, advanced term to term by
// v_{m+1} = v_m ln|mu|^2/(m+1), and does
// stage 0 (long lines: of two terms at a time, two independent register
// transforms into two exchange-buffer sets).  The last stage is done
// cooperatively by the CTA (thread b: column b % CW, butterfly b / CW); its
// results are written back into the exchange set as the CTA's output tile
// [NY rows][CW columns], which one thread stores to Z with 2D tensor copies
// (TMA, asynchronous: the next term's register transforms run while the
// copy unit reads the tile).
// -------------------------------------------------------------------------
template <int NY>
constexpr size_t inv_cols_smem() {
  // long lines: two exchange-buffer sets (two terms in flight) and
  // ln|mu|^2 per column; short lines: one set (ln|mu|^2 in registers)
  constexpr int W = icols_warps<NY>();
  return icols_pair<NY>() ? 2 * (size_t)icols_set<NY>() * sizeof(float2) + (size_t)W * LineFFT<NY>::LPW * NY * sizeof(float)
                          : (size_t)icols_set<NY>() * sizeof(float2);
}

template <int NY>
constexpr int icols_box_rows() {
  return NY < 256 ? NY : 256;
}

// The runs of Taylor terms one CTA of an inverse column pass transforms.  A
// unit is (column block cb, operator slot op), numbered u = 2 cb + op; a
// unit's group terms [m_lo, m_hi) are cut into slots of `step` terms (the
// paired kernel transforms two terms per iteration: step 2).
//   pack = 0: CTA (bx, yidx) owns unit (bx, yidx & 1) and run yidx >> 1 of
//     `parts` equal runs (one run: i = 0 only; it is empty when the runs
//     outnumber the terms);
//   pack = K > 0: a grid of K CTAs; the slots of all 2 ncb units, in
//     unit-major order, are dealt out evenly: CTA bx takes slots
//     [bx U S / K, (bx + 1) U S / K), i.e. the tail of one unit's terms,
//     whole units and the head of the next.  Every CTA then has the same
//     number of slots to within one, where whole units per CTA leave SMs
//     idle (a 1024-point column pass has 130 units of eight columns for
//     152 SMs).  Run i is the CTA's i-th unit from the last: a CTA ends on
//     the top terms of a unit where it can, as the CTAs of pack = 0 all
//     do, and the row pass, which reads the group's terms from the top
//     down, finds those most recently written ones in L2.
// Every run restarts the multiplier recurrence at its first term, so the
// bits depend on the cut (deterministic for given parts, pack and grid).
struct ColRun {
  int cb, op, lo, hi;
};
__device__ __forceinline__ bool col_run(int i, int bx, int yidx, int parts, int pack, int ncb, int m_lo, int m_hi,
                                        int step, ColRun& r) {
  if (pack <= 0) {
    if (i > 0) return false;
    const int part = yidx >> 1, per = (m_hi - m_lo + parts - 1) / parts;
    r.cb = bx;
    r.op = yidx & 1;
    r.lo = m_lo + part * per;
    r.hi = min(m_hi, r.lo + per);
    return true;
  }
  const long long S = (m_hi - m_lo + step - 1) / step, US = 2LL * ncb * S;
  const long long s0 = US * bx / pack, s1 = US * (bx + 1) / pack;
  const long long u = (s1 - 1) / S - i;
  if (s0 >= s1 || (u + 1) * S <= s0) return false;
  const long long a = max(s0, u * S) - u * S, b = min(s1, (u + 1) * S) - u * S;
  r.cb = (int)(u >> 1);
  r.op = (int)(u & 1);
  r.lo = m_lo + (int)a * step;
  r.hi = min(m_hi, m_lo + (int)b * step);
  return true;
}

template <int NY>
// (bx, yidx, parts, pack): the CTA's runs of terms (col_run).
// base > 0: slot index m stands for the term m + base (the splitting's
// remainder of terms 1..M, Sec. 3.3: base = 1).
// fwd = 1: the column spectra are not in Uh yet; every run computes them
// from the row half spectra T (pitch pT) itself, by the arithmetic of
// k2d_fwd_cols (so bit for bit the same), and the run of operator slot 0
// that starts at m_lo stores them to Uh for later groups.
__device__ __forceinline__ void inv_cols_body(int bx, int yidx, int parts, int pack, float2* __restrict__ Uh,
                                              const float* __restrict__ P, const float* __restrict__ Lg,
                                              const void* zmap, int ncols, int m_lo, int m_hi, float inv_fact_lo,
                                              float inv_fact_lo1, int split_k, const float2* __restrict__ twy,
                                              const float2* __restrict__ T = nullptr, int pT = 0, int fwd = 0,
                                              int base = 0) {
  using F = LineFFT<NY>;
  constexpr int E = F::E, LANES = F::LANES, LPW = F::LPW, BPL = F::BPL, RL = F::RL;
  constexpr int W = icols_warps<NY>(), THREADS = W * 32, CW = W * LPW;  // columns per CTA
  constexpr bool PAIR = icols_pair<NY>();
  constexpr int SET = icols_set<NY>();  // float2 slots of one exchange set
  constexpr int BOXR = icols_box_rows<NY>();
  // the output tile fits an exchange set; the second set (paired terms)
  // starts 128-byte aligned like the first, as the tensor copies require
  static_assert(NY * CW <= SET, "output tile fits an exchange set");
  static_assert(!PAIR || (SET * sizeof(float2)) % 128 == 0, "second exchange set alignment");
  __shared__ float2 s_tw[F::TW];
  extern __shared__ __align__(128) float2 s_buf[];
  for (int i = threadIdx.x; i < F::TW; i += THREADS) s_tw[i] = twy[i];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int li = lane % LANES, line = lane / LANES;
  float2* lb_own = s_buf + warp * warp_stride<NY>() + line * F::PAD_LINE;  // set 0; set 1 at + SET
  // ln|mu|^2 of the column: shared memory for long lines (registers are
  // short there), registers for short lines
  float* s_lg = reinterpret_cast<float*>(s_buf + 2 * SET) + (size_t)(warp * LPW + line) * NY;
  const long long tot = (long long)ncols * NY;
  const int ncb = (ncols + CW - 1) / CW;
  ColRun run;
  // every condition below is uniform over the CTA (barriers inside)
  for (int ri = 0; col_run(ri, bx, yidx, parts, pack, ncb, m_lo, m_hi, PAIR ? 2 : 1, run); ++ri) {
    if (run.lo >= run.hi) continue;
    const int lo = run.lo, hi = run.hi;
    const int c0 = run.cb * CW;
    const int c = c0 + warp * LPW + line;
    const int cc = min(c, ncols - 1);
    const float2* uh_col = Uh + (size_t)cc * NY;
    // split_k > 0 (one operator): slot op = 1 carries the terms m + split_k of
    // operator 1 (multiplier P[0] ln|mu|^{2(m + split_k)} / (m + split_k)!)
    const int op = run.op;
    const int off = base + ((split_k > 0 && op) ? split_k : 0);
    const float* p_col = P + (split_k > 0 ? 0 : op) * tot + (size_t)cc * NY;
    const float* l_col = Lg + (size_t)cc * NY;
    float tm[E], lg[PAIR ? 1 : E];
    // 1 / (lo + off)!: the group's factor advanced to this run's first term
    float fstart = op ? inv_fact_lo1 : inv_fact_lo;
    for (int j = m_lo + 1; j <= lo; ++j) fstart *= 1.0f / (float)(j + off);
    // tables first (they do not depend on the previous kernel)
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int y = li + LANES * m;
      const float l = l_col[y];
      if constexpr (PAIR)
        s_lg[y] = l;
      else
        lg[m] = l;
      tm[m] = p_col[y] * powi(l, lo + off) * fstart;
    }
    if (threadIdx.x == 0) bulk_wait_read_all();  // a previous run's last tiles have left shared memory
    __syncthreads();
    pdl_wait();  // Uh (k2d_fwd_cols) or T (k2d_fwd_rows) ready; the previous group's readers of Z are done
    pdl_trigger();
    // v = the multiplied spectrum of the current term: u_hat P ln|mu|^{2m}/m!
    float2 v[E];
    if (fwd) {
      {
        // forward stage 0 cooperatively: thread b takes column b % CW,
        // butterfly b / CW (row segments of CW adjacent columns of T)
        const int fc = threadIdx.x % CW, j = threadIdx.x / CW;
        const int col = min(c0 + fc, ncols - 1);
        float2 x[E];
#pragma unroll
        for (int r = 0; r < E; ++r) x[r] = T[(size_t)(j + LANES * r) * pT + col];
        float2* lb = s_buf + (fc / LPW) * warp_stride<NY>() + (fc % LPW) * F::PAD_LINE;
        stage0_to_smem<NY, false>(x, lb, j);
      }
      __syncthreads();
      mid_stage<NY, false>(lb_own, s_tw, li);
      __syncwarp();
#pragma unroll
      for (int q = 0; q < BPL; ++q) {
        float2 w[RL];
        stage1_from_smem<NY, false>(w, lb_own, s_tw, li + LANES * q);
#pragma unroll
        for (int r = 0; r < RL; ++r) v[q + BPL * r] = w[r];
      }
      if (op == 0 && lo == m_lo && c < ncols) {
#pragma unroll
        for (int m = 0; m < E; ++m) Uh[(size_t)c * NY + li + LANES * m] = v[m];
      }
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = cscale(v[m], tm[m]);
    } else {
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = cscale(uh_col[li + LANES * m], tm[m]);
    }
    // v <- v ln|mu|^2 / (m + 1): the next term
    auto advance = [&](int mt) {
      const float rinv = 1.0f / (float)(mt + 1 + off);
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = cscale(v[m], (PAIR ? s_lg[li + LANES * m] : lg[m]) * rinv);
    };
    // last stage of exchange set `set`, cooperatively: thread b takes column
    // b % CW, butterfly b / CW; results in registers
    auto last_read = [&](int set, float2 (&w)[BPL][RL]) {
#pragma unroll
      for (int q = 0; q < BPL; ++q) {
        const int b = threadIdx.x + THREADS * q;
        const int sc = b % CW, sj = b / CW;
        const float2* lb = s_buf + set * SET + (sc / LPW) * warp_stride<NY>() + (sc % LPW) * F::PAD_LINE;
        stage1_from_smem<NY, true>(w[q], lb, s_tw, sj);
      }
    };
    // ... written back into the (fully read) set as the output tile
    // [NY rows][CW columns], made visible to the tensor-copy unit
    auto tile_write = [&](int set, const float2 (&w)[BPL][RL]) {
      float2* tile = s_buf + set * SET;
#pragma unroll
      for (int q = 0; q < BPL; ++q) {
        const int b = threadIdx.x + THREADS * q;
        const int sc = b % CW, sj = b / CW;
#pragma unroll
        for (int r = 0; r < RL; ++r) tile[(sj + F::NBL * r) * CW + sc] = w[q][r];
      }
      fence_proxy_async_smem();
    };
    // one thread stores the tile of `set` to Z slot (mt - m_lo) of operator op
    // (rows (slot * 2 + op) * NY .. + NY, columns c0 .. c0 + CW; columns past
    // ncols are clipped by the copy unit)
    auto tile_store = [&](int set, int mt) {
      const int y0 = ((mt - m_lo) * 2 + op) * NY;
#pragma unroll
      for (int k = 0; k < NY / BOXR; ++k) tma_store_2d(zmap, c0, y0 + k * BOXR, s_buf + set * SET + k * BOXR * CW);
    };
    int mt = lo;
    // two terms per iteration: two independent register transforms in flight;
    // an odd last term runs through the same code with its partner computed
    // and not stored (one copy of the unrolled term code: the kernel's
    // instruction footprint, not its arithmetic, limited it)
    for (; PAIR && mt < hi; mt += 2) {
      const bool two = mt + 1 < hi;
      float2 xa[E], xb[E];
#pragma unroll
      for (int m = 0; m < E; ++m) xa[m] = v[m];
      advance(mt);
#pragma unroll
      for (int m = 0; m < E; ++m) xb[m] = v[m];
      dft<E, true>(xa);
      dft<E, true>(xb);
      if (threadIdx.x == 0) bulk_wait_read_all();  // the previous tiles have left shared memory
      __syncthreads();
      stage0_write<NY>(xa, lb_own, li);
      stage0_write<NY>(xb, lb_own + SET, li);
      mid_stage<NY, true>(lb_own, s_tw, li);
      mid_stage<NY, true>(lb_own + SET, s_tw, li);
      __syncthreads();
      {
        float2 w[BPL][RL];
        last_read(0, w);
        __syncthreads();
        tile_write(0, w);
      }
      {
        float2 w[BPL][RL];
        last_read(1, w);
        __syncthreads();
        tile_write(1, w);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        tile_store(0, mt);
        if (two) tile_store(1, mt + 1);
        bulk_commit();
      }
      if (mt + 2 < hi) advance(mt + 1);
    }
    if (!PAIR) {
      // short lines: one term per iteration (a separate loop: sharing it with
      // the odd last term above made the paired form markedly slower)
      for (; mt < hi; ++mt) {
        float2 x[E];
#pragma unroll
        for (int m = 0; m < E; ++m) x[m] = v[m];
        dft<E, true>(x);
        if (threadIdx.x == 0) bulk_wait_read_all();
        __syncthreads();
        stage0_write<NY>(x, lb_own, li);
        mid_stage<NY, true>(lb_own, s_tw, li);
        __syncthreads();
        float2 w[BPL][RL];
        last_read(0, w);
        __syncthreads();
        tile_write(0, w);
        __syncthreads();
        if (threadIdx.x == 0) {
          tile_store(0, mt);
          bulk_commit();
        }
        if (mt + 1 < hi) advance(mt);
      }
    }
  }  // runs
  if (threadIdx.x == 0) bulk_wait_all();  // stores complete before the CTA's shared memory goes
}

template <int NY>
__global__ void __launch_bounds__(icols_warps<NY>() * 32) k2d_inv_cols(float2* __restrict__ Uh, const float* __restrict__ P,
                                                           const float* __restrict__ Lg,
                                                           const __grid_constant__ CUtensorMap zmap, int ncols,
                                                           int m_lo, int m_hi, float inv_fact_lo,
                                                           float inv_fact_lo1, int split_k, int parts,
                                                           int pack, const float2* __restrict__ twy,
                                                           const float2* __restrict__ T, int pT, int fwd, int base) {
  inv_cols_body<NY>(blockIdx.x, blockIdx.y, parts, pack, Uh, P, Lg, &zmap, ncols, m_lo, m_hi, inv_fact_lo, inv_fact_lo1,
                    split_k, twy, T, pT, fwd, base);
}

// -------------------------------------------------------------------------
// I2: inverse FFT along x of both operators (A + iB), Horner accumulation
// over the group's terms, then partial store or epilogue.
// The two Z rows (operator 1 and 2) of the next term are copied into shared
// memory by TMA bulk copies while the current term is transformed (double
// buffer per line, mbarrier completion, bounded waits).
// -------------------------------------------------------------------------
template <int NX>
constexpr int rows_rb() {
  return (NX / 2 + 2) & ~1;  // Z row copy length in float2: >= H+1, 16-byte multiple
}
template <int NX, int W = W_IROWS>
constexpr size_t inv_rows_smem() {
  return exch_smem<NX, W>() + (size_t)W * LineFFT<NX>::LPW * 2 * 2 * rows_rb<NX>() * sizeof(float2);
}

// SPLIT: one operator whose terms fill both slots (TermSplit); k2 and
// split_k are read only then.  W: warps per CTA.
// rsplit (dividing W): the group's terms of each row are split into rsplit
// runs of per = ceil(G / rsplit) terms, one warp each; every warp sums its
// run by Horner's rule, and the row's sum is the Horner sum of the runs,
// T = S_0 + delta^per (S_1 + delta^per (S_2 + ...)), formed through shared
// memory (short rows have few lines: this shortens each warp's chain of
// terms).  rsplit = 1: one warp per row takes every term.
template <int NX, bool SPLIT, int W = W_IROWS>
__device__ __forceinline__ void inv_rows_body(int bx, const float2* __restrict__ Z, long long zslot, int pZ, int ny,
                                              int m_lo, int m_hi, int top, int k2, int split_k,
                                              const float* __restrict__ delta,
                                              float* __restrict__ part1, float* __restrict__ part2,
                                              const EpiArgs<float>& epi, float inv_lambda,
                                              const float2* __restrict__ twx, int* err, int rsplit = 1) {
  using F = LineFFT<NX>;
  constexpr int E = F::E, LANES = F::LANES, H = NX / 2, LPW = F::LPW, THREADS = W * 32;
  constexpr int RB = rows_rb<NX>();
  constexpr uint32_t RB_BYTES = RB * sizeof(float2);
  __shared__ float2 s_tw[F::TW];
  __shared__ uint64_t s_bar[W * LPW * 2];
  extern __shared__ __align__(128) float2 s_buf[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int li = lane % LANES, line = lane / LANES;
  const int lid = warp * LPW + line;  // line id inside the CTA
  uint64_t* bar = s_bar + 2 * lid;
  float2* zbuf = s_buf + W * warp_stride<NX>() + (size_t)lid * 4 * RB;  // [buf][op][RB]
  if (li == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < F::TW; i += THREADS) s_tw[i] = twx[i];
  float2* wbuf = s_buf + warp * warp_stride<NX>();
  // this warp's rows and run of terms
  const int rs = rsplit, sub = warp % rs;
  const int yr = (bx * (W / rs) + warp / rs) * LPW + line;
  const bool active = yr < ny;
  const int per = (m_hi - m_lo + rs - 1) / rs;
  const int r_lo = min(m_hi, m_lo + sub * per), r_hi = min(m_hi, r_lo + per);
  const bool from_part = !top && r_hi == m_hi && r_lo < r_hi;  // the run that continues the previous group's sum
  const int y = active ? yr : 0;
  const size_t row = (size_t)y * NX;
  // rows this line reads later, produced two or more kernels ago: into L2
  // now (the last group's epilogue reads five fields that the step's
  // spectrum traffic has usually evicted)
  if (li == 0 && active) {
    constexpr uint32_t RowB = NX * sizeof(float);
    if (from_part) {
      prefetch_l2(part1 + row, RowB);
      prefetch_l2(part2 + row, RowB);
    }
    if (m_lo == 0 && (epi.mode == EPI_STEP || epi.mode == EPI_START)) {
      prefetch_l2(epi.u_cur + row, RowB);
      prefetch_l2(epi.u_other + row, RowB);
      prefetch_l2(epi.l2p + row, RowB);
      prefetch_l2(epi.A + row, RowB);
      prefetch_l2(epi.B + row, RowB);
    }
  }
  // delta = gamma - gamma0 does not depend on earlier kernels: into
  // registers before the programmatic wait
  float dl[E];
#pragma unroll
  for (int m = 0; m < E; ++m) dl[m] = delta[row + li + LANES * m];
  __syncthreads();
  pdl_wait();  // Z of this group and the previous group's partial sums are ready
  pdl_trigger();
  auto issue = [&](int buf, int mt) {
    const float2* z1 = Z + (long long)((mt - m_lo) * 2 + 0) * zslot + (size_t)y * pZ;
    const float2* z2 = Z + (long long)((mt - m_lo) * 2 + 1) * zslot + (size_t)y * pZ;
    mbar_arrive_expect_tx(&bar[buf], 2 * RB_BYTES);
    bulk_copy_g2s(zbuf + buf * 2 * RB, z1, RB_BYTES, &bar[buf]);
    bulk_copy_g2s(zbuf + buf * 2 * RB + RB, z2, RB_BYTES, &bar[buf]);
  };
  if (li == 0 && r_lo < r_hi) issue(0, r_hi - 1);
  float a1[E], a2[E];
  if (!from_part) {
#pragma unroll
    for (int m = 0; m < E; ++m) a1[m] = a2[m] = 0.f;
  } else {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      a1[m] = part1[row + li + LANES * m];
      a2[m] = part2[row + li + LANES * m];
    }
  }
  uint32_t phase = 0;  // bit b: parity to wait for on buffer b
  int it = 0;
  bool ok = true;
  for (int mt = r_hi - 1; mt >= r_lo; --mt, ++it) {
    const int b = it & 1;
    if (mt > r_lo) {
      __syncwarp();  // every lane finished reading buffer b^1 (two terms ago)
      if (li == 0) {
        fence_proxy_async_smem();
        issue(b ^ 1, mt - 1);
      }
    }
    const bool got = mbar_wait_bounded(&bar[b], (phase >> b) & 1u, err);
    phase ^= 1u << b;
    if (!__all_sync(0xffffffffu, got)) {
      // give up: drain the prefetch still in flight (bounded) and leave
      if (mt > r_lo) mbar_wait_bounded(&bar[b ^ 1], (phase >> (b ^ 1)) & 1u, err);
      ok = false;
      break;
    }
    const float2* z1 = zbuf + b * 2 * RB;
    const float2* z2 = z1 + RB;
    float2 w[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int n = li + LANES * m;
      if (n <= H) {
        const float2 p = z1[n], q = z2[n];
        w[m] = (n == 0 || n == H) ? make_float2(p.x, q.x) : make_float2(p.x - q.y, p.y + q.x);
      } else {
        const float2 p = z1[NX - n], q = z2[NX - n];
        w[m] = make_float2(p.x + q.y, q.x - p.y);
      }
    }
    fft_line<NX, true>(w, wbuf, s_tw, li, line);
    const bool use2 = !SPLIT || mt < k2;  // slot 2 holds a term of the expansion
#pragma unroll
    for (int m = 0; m < E; ++m) {
      a1[m] = fmaf(dl[m], a1[m], w[m].x);
      if (use2) a2[m] = fmaf(dl[m], a2[m], w[m].y);
    }
  }
  if (rs > 1) {
    // the runs' sums meet in the row's warps' staging buffers (no copies in
    // flight any more): run s publishes, run 0 combines, highest first
    float* pub = reinterpret_cast<float*>(zbuf);  // 2 NX floats fit in 4 RB float2
    if (sub > 0) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        pub[li + LANES * m] = a1[m];
        pub[NX + li + LANES * m] = a2[m];
      }
    }
    __syncthreads();
    if (sub > 0) return;
    float dp[E];  // delta^per
#pragma unroll
    for (int m = 0; m < E; ++m) dp[m] = powi(dl[m], per);
    float t1[E], t2[E];
#pragma unroll
    for (int m = 0; m < E; ++m) t1[m] = t2[m] = 0.f;
    for (int q = rs - 1; q >= 1; --q) {
      const float* src = reinterpret_cast<const float*>(zbuf + (size_t)q * LPW * 4 * RB);  // warp + q, same line
#pragma unroll
      for (int m = 0; m < E; ++m) {
        t1[m] = fmaf(dp[m], t1[m], src[li + LANES * m]);
        t2[m] = fmaf(dp[m], t2[m], src[NX + li + LANES * m]);
      }
    }
#pragma unroll
    for (int m = 0; m < E; ++m) {
      a1[m] = fmaf(dp[m], t1[m], a1[m]);
      a2[m] = fmaf(dp[m], t2[m], a2[m]);
    }
  }
  if (!active || !ok) return;
  if (m_lo > 0) {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      part1[row + li + LANES * m] = a1[m];
      part2[row + li + LANES * m] = a2[m];
    }
  } else if constexpr (SPLIT) {  // one operator: sum_{m<K} + delta^K sum_{m>=K}
#pragma unroll
    for (int m = 0; m < E; ++m) {
      float dk = 1.f;
      for (int j = 0; j < split_k; ++j) dk *= dl[m];
      float L = fmaf(dk, a2[m], a1[m]);
      for (int j = 0; j < epi.dpow; ++j) L *= dl[m];  // terms from dpow on
      epilogue_point<float>(epi, (long long)(row + li + LANES * m), L, 0.f);
    }
  } else {
#pragma unroll
    for (int m = 0; m < E; ++m)
      epilogue_point<float>(epi, (long long)(row + li + LANES * m), a1[m], a2[m] * inv_lambda);
  }
}

template <int NX, bool SPLIT, int W = W_IROWS>
__global__ void __launch_bounds__(W * 32) k2d_inv_rows(const float2* __restrict__ Z, long long zslot, int pZ,
                                                           int ny, int m_lo, int m_hi, int top, int k2, int split_k,
                                                           const float* __restrict__ delta, float* __restrict__ part1,
                                                           float* __restrict__ part2, EpiArgs<float> epi,
                                                           float inv_lambda, const float2* __restrict__ twx,
                                                           int* err, int rsplit) {
  inv_rows_body<NX, SPLIT, W>(blockIdx.x, Z, zslot, pZ, ny, m_lo, m_hi, top, k2, split_k, delta, part1, part2, epi,
                              inv_lambda, twx, err, rsplit);
}

// -------------------------------------------------------------------------
// 3D y pass: inverse FFT along y of the columns of independent planes
// (blockIdx.y = plane), no multiplier.  Input plane [H+1][ny] (column-major,
// stride in_plane), output rows [ny][pZ] (stride out_plane); stage 1 is
// cooperative as in k2d_inv_cols, so stores are row segments.
// -------------------------------------------------------------------------
template <int NY>
__global__ void __launch_bounds__(W_YCOLS * 32) k3d_inv_ycols(const float2* __restrict__ in, long long in_plane,
                                                            float2* __restrict__ out, long long out_plane, int pZ,
                                                            int ncols, const float2* __restrict__ twy) {
  using F = LineFFT<NY>;
  constexpr int E = F::E, LANES = F::LANES, LPW = F::LPW, BPL = F::BPL;
  constexpr int THREADS = W_YCOLS * 32, CW = W_YCOLS * LPW;
  __shared__ float2 s_tw[F::TW];
  extern __shared__ __align__(128) float2 s_buf[];
  for (int i = threadIdx.x; i < F::TW; i += THREADS) s_tw[i] = twy[i];
  __syncthreads();
  pdl_wait();
  pdl_trigger();
  in += blockIdx.y * in_plane;
  out += blockIdx.y * out_plane;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int li = lane % LANES, line = lane / LANES;
  float2* lb_own = s_buf + warp * warp_stride<NY>() + line * F::PAD_LINE;
  const int c0 = blockIdx.x * CW;
  const int cc = min(c0 + warp * LPW + line, ncols - 1);
  float2 x[E];
#pragma unroll
  for (int m = 0; m < E; ++m) x[m] = in[(size_t)cc * NY + li + LANES * m];
  stage0_to_smem<NY, true>(x, lb_own, li);
  mid_stage<NY, true>(lb_own, s_tw, li);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < BPL; ++q) {
    const int b = threadIdx.x + THREADS * q;
    const int sc = b % CW, sj = b / CW;
    const float2* lb = s_buf + (sc / LPW) * warp_stride<NY>() + (sc % LPW) * F::PAD_LINE;
    float2 w[F::RL];
    stage1_from_smem<NY, true>(w, lb, s_tw, sj);
    if (c0 + sc < ncols) {
#pragma unroll
      for (int r = 0; r < F::RL; ++r) out[(size_t)(sj + F::NBL * r) * pZ + c0 + sc] = w[r];
    }
  }
}

// Dynamic shared memory of a fused kernel, and the whole shared-memory
// carveout for all of them: consecutive kernels of a step (overlapped by
// programmatic dependent launch) then never need the SM's L1/shared split
// changed between them.
template <typename... KArgs>
cudaError_t set_kernel_smem(void (*kern)(KArgs...), size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  return e;
}

inline int round_up(int a, int b) { return (a + b - 1) / b * b; }


// How the Taylor terms m = 0..M fill the two operator slots of the inverse
// kernels: one term of each operator per slot index (two operators), or,
// for a model with one operator, terms 0..K-1 in slot 0 and K..M in slot 1
// (K = ceil((M+1)/2)), combined as sum_0 + delta^K sum_1 in the epilogue.
struct TermSplit {
  int slots;    // slot indices 0..slots-1
  int k2;       // slot-1 indices below k2 hold a term
  int split_k;  // slot-1 term offset (0: two operators)
};
inline TermSplit term_split(int M, bool one_operator) {
  if (!one_operator) return {M + 1, M + 1, 0};
  const int K = (M + 2) / 2;
  return {K, M + 1 - K, K};
}

inline float inv_factorial(int m) {
  double f = 1.0;
  for (int i = 2; i <= m; ++i) f *= i;
  return (float)(1.0 / f);
}

// Cooperative launch (every CTA resident at once, for kernels with a
// grid-wide barrier); the grid must not exceed the resident capacity.
template <typename... KArgs, typename... Args>
cudaError_t launch_coop(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Launch with programmatic stream serialisation: the kernel may start while
// its predecessor finishes and synchronises itself with griddepcontrol.wait.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}


}  // namespace
}  // namespace vofl
