// kernels_wide.cuh -- the inverse column and row passes of the fused 2D step
// (Eq. (2.13) of arXiv 2311.13049, see fused2d.cu) on the wide line
// transform of fft_wide.cuh, for lines of 512 and 1024 points.
//
// Same data path and arithmetic order as the narrow kernels of kernels.cuh
// (multiplier recurrence t_{m+1} = t_m ln|mu|^2/(m+1) in registers, Horner
// over the group's terms in registers), with 16 elements per lane: a 1024
// point line is owned by two warps, so a pass has twice the warps of the
// narrow form and each holds half the registers.
//
// Lines per CTA (L) is a template parameter.  At 1024 points seven lines
// per CTA and one CTA per SM (128 registers a thread) make one step's
// 6156 column or 6144 row line transforms of a six-term group 5.8 waves of
// seven per SM, against 5.06 waves (rounded up to 6) of eight.
#pragma once
#include <cuda_runtime.h>

#include "fft_wide.cuh"
#include "kernels.cuh"

namespace vofl {
namespace {

// Default transform schedule of a 2D grid (the single-context and the
// batched launches both follow it, so a batch member gives the bits of the
// same grid stepped alone): wide inverse column pass at 512 points, wide
// inverse row pass at 512 and 1024 (measured per size; vofl_set_schedule
// changes it per context).
inline bool wide_cols_default(int ny) { return ny == 512; }
// wide forward row pass: an option only (at 1024 it made the two-kernel
// forward 1% shorter, but both forward passes in one launch, which use
// 32-element lines, are 2% shorter still)
inline bool wide_fwd_default(int nx) {
  (void)nx;
  return false;
}
inline bool wide_rows_default(int nx) { return nx == 512 || nx == 1024; }
// Taylor terms per group: 17, so that M <= 16 runs in one group (one column
// and one row launch per step).  Every launch boundary costs a few
// microseconds; at 1024^2 one group of 17 (145 MB of per-term column
// transforms, beyond L2) measured 7% faster than two groups of 9 (77 MB,
// in L2) and 12% faster than three of 6.
inline int group_default(int nx, int ny) {
  (void)nx;
  (void)ny;
  return 17;
}
// Runs of terms per row in the 32-element row kernel (dividing its warps
// per CTA): grids of up to 256^2 points have few row lines (256 rows in
// 128 warps), so each row's group of 17 terms goes to four warps.
inline int row_split_default(int nx, int ny, int warps) {
  const int want = (long long)nx * ny <= 256LL * 256 ? 4 : 1;
  return warps % want == 0 ? want : 1;
}
// Forward passes.  1: the forward column transform inside the top group's
// inverse column kernel (one launch fewer per step; every CTA of the group
// transforms its own columns, the same arithmetic as k2d_fwd_cols): on
// grids of up to 256 rows, where a launch boundary is a large part of the
// step (256^2: 6% shorter); at 768 and 1024 the duplicated column
// transforms (two operators, every run) cost more than the launch (2%
// longer).  2: both forward passes in one cooperative launch
// (k2d_fwd_both): per leap-frog step, M = 16, 512^2 0.0486 -> 0.0471 ms,
// 768^2 0.1008 -> 0.0985, 1024^2 0.1166 -> 0.1142; at 256^2 and 128^2 it
// loses to 1 (0.0266 vs 0.0246, 0.0233 vs 0.0205).
inline int fuse_forward_default(int nx, int ny) {
  if (ny <= 256) return 1;
  return (nx == ny && (nx == 512 || nx == 768 || nx == 1024)) ? 2 : 0;
}
// Runs of terms per group in the column pass (each on its own CTAs): small
// grids have fewer column blocks than SMs.
inline int col_parts_default(int ny) { return ny <= 256 ? 3 : (ny <= 512 ? 6 : 1); }
// The group's terms of all column blocks dealt out evenly over `waves`
// times the SM count CTAs (col_run, pack > 0) instead of whole column
// blocks (and col_parts runs) per CTA; 0 = not.  Measured per leap-frog
// step, M = 16: 128^2 one CTA per SM, 0.0225 -> 0.0195 ms; 512^2 (wide
// columns, eight warps a CTA) one per SM, 0.0594 -> 0.0483 ms, where two
// per SM measured 0.0635 (one column CTA per SM leaves room for the row
// kernel's CTAs to start early); 768^2 (four-warp CTAs) two per SM, 0.1095
// -> 0.1006 ms; no gain at 256^2 (0.0246 either way) nor at 1024^2
// (0.1164 vs 0.1158: the 17-term launch's 145 MB of column transforms,
// not idle SMs, set its time).
inline int col_pack_waves(int nx, int ny) {
  if (nx != ny) return 0;
  return (nx == 128 || nx == 512) ? 1 : nx == 768 ? 2 : 0;
}

// Lines per CTA: eight columns (the cooperative last stage stores 64-byte
// row segments, whole L2 sectors: seven columns' 56-byte segments left
// partial sectors and measured far slower); rows: seven two-warp lines at
// 1024 points, two one-warp lines at 512 (a 512-row pass has only 512
// lines: 256 CTAs).
template <int N>
constexpr int wide_lines_per_cta() {
  return 8;  // 64-byte row segments: whole 32-byte sectors
}
template <int N>
constexpr int wide_rows_per_cta() {
  return N == 1024 ? 7 : 2;
}
template <int N>
constexpr int wide_threads() {
  return wide_lines_per_cta<N>() * WideFFT<N>::LANES;
}
template <int N>
constexpr int wide_rows_threads() {
  return wide_rows_per_cta<N>() * WideFFT<N>::LANES;
}
// CTAs per SM the register budget is set for: one 14-warp CTA at 1024
// points, two 8-warp CTAs at 512
template <int N>
constexpr int wide_min_blocks() {
  return N == 1024 ? 1 : 2;
}
// Offset between consecutive lines' buffer pairs: the two buffers plus a
// stagger that puts the lines of the cooperative last stage (thread b:
// line b % L, butterfly b / L) on distinct shared-memory banks (checked
// exhaustively for L = 4, 7, 8).
template <int N, int L>
constexpr int wide_line_stride() {
  return 2 * WideFFT<N>::PAD_LINE + (L == 7 ? 7 : L == 8 ? 2 : L == 4 ? 4 : 1);
}
template <int N>
constexpr int wide_rows_rb() {
  return (N / 2 + 2) & ~1;  // Z row copy length in float2: >= N/2+1, 16-byte multiple
}
template <int N>
constexpr size_t wide_cols_smem() {
  constexpr int L = wide_lines_per_cta<N>();
  return (size_t)L * wide_line_stride<N, L>() * sizeof(float2);
}
// rows: the line buffers, then (from a 128-byte boundary, as bulk copies
// need 16-byte aligned destinations) one staged pair of Z rows per line
template <int N>
constexpr int wide_rows_zs_off() {
  constexpr int L = wide_rows_per_cta<N>();
  return (L * wide_line_stride<N, L>() + 15) / 16 * 16;
}
template <int N>
constexpr size_t wide_rows_smem() {
  constexpr int L = wide_rows_per_cta<N>();
  return ((size_t)wide_rows_zs_off<N>() + (size_t)L * 2 * wide_rows_rb<N>()) * sizeof(float2);
}

// -------------------------------------------------------------------------
// I1 (wide): multiplier + inverse FFT along y of L columns of one operator
// for the CTA's runs of terms of the group [m_lo, m_hi) (col_run: runs of
// `parts` per unit, or the units' terms dealt out over `pack` CTAs).
// Stages 0 and 1 by the column's own lanes; stage 2 cooperatively (thread
// b: column b % L, butterfly b / L), whose outputs are row segments of L
// adjacent columns stored straight to Z[slot][op][y][c].
// -------------------------------------------------------------------------
template <int NY>
__device__ __forceinline__ void inv_cols_wide_body(int bx, int yidx, int parts, int pack, const float2* __restrict__ Uh,
                                                   const float* __restrict__ P, const float* __restrict__ Lg,
                                                   float2* __restrict__ Z, int pZ, int ncols, int m_lo, int m_hi,
                                                   float inv_fact_lo, float inv_fact_lo1, int split_k,
                                                   const float2* __restrict__ twy, int base = 0) {
  using F = WideFFT<NY>;
  constexpr int LANES = F::LANES, CW = wide_lines_per_cta<NY>(), THREADS = CW * LANES, NB2 = F::NB2;
  constexpr int LS = wide_line_stride<NY, CW>();
  __shared__ float2 s_tw[F::TW];
  extern __shared__ __align__(128) float2 s_buf[];  // [CW][A, B, stagger]
  for (int i = threadIdx.x; i < F::TW; i += THREADS) s_tw[i] = twy[i];
  const int line = threadIdx.x / LANES, li = threadIdx.x % LANES;
  float2* A = s_buf + (size_t)line * LS;
  float2* B = A + F::PAD_LINE;
  const long long tot = (long long)ncols * NY;
  const int ncb = (ncols + CW - 1) / CW;
  // this thread's cooperative stage-2 butterflies: line sc, butterflies
  // sj0 + LANES q (q < 4); rows sj0 + LANES q + NB2 r of column c0 + sc
  const int sc = threadIdx.x % CW, sj0 = threadIdx.x / CW;
  const float2* Bc = s_buf + (size_t)sc * LS + F::PAD_LINE;
  const size_t zslot2 = (size_t)2 * NY * pZ;  // one term: both operators' slots
  ColRun run;
  // every condition below is uniform over the CTA (barriers inside)
  for (int ri = 0; col_run(ri, bx, yidx, parts, pack, ncb, m_lo, m_hi, 1, run); ++ri) {
    if (run.lo >= run.hi) continue;
    const int lo = run.lo, hi = run.hi, op = run.op;
    const int c0 = run.cb * CW;
    const int cc = min(c0 + line, ncols - 1);
    const int off = base + ((split_k > 0 && op) ? split_k : 0);  // base: as in inv_cols_body
    const float* p_col = P + (split_k > 0 ? 0 : op) * tot + (size_t)cc * NY;
    const float* l_col = Lg + (size_t)cc * NY;
    const float2* uh_col = Uh + (size_t)cc * NY;
    float fstart = op ? inv_fact_lo1 : inv_fact_lo;
    for (int j = m_lo + 1; j <= lo; ++j) fstart *= 1.0f / (float)(j + off);
    // tables first (they do not depend on the previous kernel)
    float lg[16], tm[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int y = li + LANES * m;
      lg[m] = l_col[y];
      tm[m] = p_col[y] * powi(lg[m], lo + off) * fstart;
    }
    const bool store = c0 + sc < ncols;
    __syncthreads();  // twiddles; every thread's stage-2 reads of a previous run done
    pdl_wait();       // Uh ready; the previous group's readers of Z are done
    pdl_trigger();
    float2 v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = cscale(uh_col[li + LANES * m], tm[m]);
    float2* zcol = Z + (size_t)op * NY * pZ + (size_t)sj0 * pZ + c0 + sc;
    for (int mt = lo; mt < hi; ++mt) {
      float2 x[16];
#pragma unroll
      for (int m = 0; m < 16; ++m) x[m] = v[m];
      wide_stage0<NY, true>(x, A, li);
      __syncthreads();  // A complete; every thread's previous stage-2 reads of B done
      wide_stage1<NY, true>(A, B, s_tw, li);
      __syncthreads();  // every column's B complete
      float2* zt = zcol + (size_t)(mt - m_lo) * zslot2;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float2 w[4];
        wide_stage2_bfly<NY, true>(w, Bc, s_tw, sj0 + LANES * q);
        if (store) {
#pragma unroll
          for (int r = 0; r < 4; ++r) zt[(size_t)(LANES * q + NB2 * r) * pZ] = w[r];
        }
      }
      if (mt + 1 < hi) {
        const float rinv = 1.0f / (float)(mt + 1 + off);
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = cscale(v[m], lg[m] * rinv);
      }
    }
  }
}

template <int NY>
__global__ void __launch_bounds__(wide_threads<NY>(), wide_min_blocks<NY>())
    k2d_inv_cols_w(const float2* __restrict__ Uh, const float* __restrict__ P, const float* __restrict__ Lg,
                   float2* __restrict__ Z, int pZ, int ncols, int m_lo, int m_hi, float inv_fact_lo,
                   float inv_fact_lo1, int split_k, int parts, int pack, const float2* __restrict__ twy,
                   int base) {
  inv_cols_wide_body<NY>(blockIdx.x, blockIdx.y, parts, pack, Uh, P, Lg, Z, pZ, ncols, m_lo, m_hi, inv_fact_lo,
                         inv_fact_lo1, split_k, twy, base);
}

// -------------------------------------------------------------------------
// I2 (wide): inverse FFT along x of both operators (A + iB) for L rows,
// Horner accumulation over the group's terms, then partial store or the
// epilogue.  The two Z rows (operator 1 and 2) of the next term are copied
// into the row's staging buffer by TMA bulk copies as soon as every lane
// of the row has read the current term from it (right after the first
// barrier of the transform), so the copy overlaps the rest of the term.
// Waits are bounded; the row's lanes decide together (barrier reduction)
// whether a wait gave up, drain the copy in flight (bounded) and leave.
// -------------------------------------------------------------------------
template <int NX, bool SPLIT>
__device__ __forceinline__ void inv_rows_wide_body(int bx, const float2* __restrict__ Z, long long zslot, int pZ,
                                                   int ny, int m_lo, int m_hi, int top, int k2, int split_k,
                                                   const float* __restrict__ delta, float* __restrict__ part1,
                                                   float* __restrict__ part2, const EpiArgs<float>& epi,
                                                   float inv_lambda, const float2* __restrict__ twx, int* err) {
  using F = WideFFT<NX>;
  constexpr int LANES = F::LANES, RPC = wide_rows_per_cta<NX>(), THREADS = RPC * LANES, H = NX / 2;
  constexpr int LS = wide_line_stride<NX, RPC>(), RB = wide_rows_rb<NX>();
  constexpr uint32_t RB_BYTES = RB * sizeof(float2);
  static_assert(RPC <= 15, "named barriers 1..15");
  __shared__ float2 s_tw[F::TW];
  __shared__ uint64_t s_bar[RPC];
  extern __shared__ __align__(128) float2 s_buf[];  // [RPC][A, B, stagger], then [RPC][op][RB]
  const int line = threadIdx.x / LANES, li = threadIdx.x % LANES;
  const int bar_id = 1 + line;
  float2* A = s_buf + (size_t)line * LS;
  float2* B = A + F::PAD_LINE;
  float2* zs = s_buf + wide_rows_zs_off<NX>() + (size_t)line * 2 * RB;  // 128-byte base, RB even
  static_assert(RB % 2 == 0 && wide_rows_zs_off<NX>() % 16 == 0, "bulk-copy destinations 16-byte aligned");
  uint64_t* bar = &s_bar[line];
  if (li == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < F::TW; i += THREADS) s_tw[i] = twx[i];
  const int yr = bx * RPC + line;
  const bool active = yr < ny;
  const int y = active ? yr : 0;
  const size_t row = (size_t)y * NX;
  if (li == 0 && active) {
    constexpr uint32_t RowB = NX * sizeof(float);
    if (!top) {
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
  float dl[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) dl[m] = delta[row + li + LANES * m];
  __syncthreads();
  pdl_wait();  // Z of this group and the previous group's partial sums are ready
  pdl_trigger();
  auto issue = [&](int mt) {
    const float2* z1 = Z + (long long)((mt - m_lo) * 2) * zslot + (size_t)y * pZ;
    mbar_arrive_expect_tx(bar, 2 * RB_BYTES);
    bulk_copy_g2s(zs, z1, RB_BYTES, bar);
    bulk_copy_g2s(zs + RB, z1 + zslot, RB_BYTES, bar);
  };
  if (li == 0) {
    issue(m_hi - 1);
    if (m_hi - 2 >= m_lo) {
      const float2* z3 = Z + (long long)((m_hi - 2 - m_lo) * 2) * zslot + (size_t)y * pZ;
      prefetch_l2(z3, RB_BYTES);
      prefetch_l2(z3 + zslot, RB_BYTES);
    }
  }
  float a1[16], a2[16];
  if (top) {
#pragma unroll
    for (int m = 0; m < 16; ++m) a1[m] = a2[m] = 0.f;
  } else {
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      a1[m] = part1[row + li + LANES * m];
      a2[m] = part2[row + li + LANES * m];
    }
  }
  uint32_t phase = 0;
  for (int mt = m_hi - 1; mt >= m_lo; --mt) {
    const bool got = mbar_wait_bounded(bar, phase, err);
    phase ^= 1u;
    const float2* z1 = zs;
    const float2* z2 = zs + RB;
    float2 w[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int n = li + LANES * m;
      if (n <= H) {
        const float2 p = z1[n], q = z2[n];
        w[m] = (n == 0 || n == H) ? make_float2(p.x, q.x) : make_float2(p.x - q.y, p.y + q.x);
      } else {
        const float2 p = z1[NX - n], q = z2[NX - n];
        w[m] = make_float2(p.x + q.y, q.x - p.y);
      }
    }
    wide_stage0<NX, true>(w, A, li);
    // every lane has read the staged rows (and written A): the staging
    // buffer is free for the next term's copy
    if (line_sync_any<NX>(bar_id, !got)) {
      // a wait gave up (error word set): no copy is in flight unless this
      // lane's own wait was the one that failed; drain it (bounded), leave
      if (li == 0 && !got) mbar_wait_bounded(bar, phase ^ 1u, err);
      return;
    }
    if (li == 0 && mt > m_lo) {
      fence_proxy_async_smem();
      issue(mt - 1);
      // the term after that into L2 already: a group larger than L2
      // streams its rows from DRAM, and one term of lookahead in shared
      // memory does not cover that latency
      if (mt - 1 > m_lo) {
        const float2* z3 = Z + (long long)((mt - 2 - m_lo) * 2) * zslot + (size_t)y * pZ;
        prefetch_l2(z3, RB_BYTES);
        prefetch_l2(z3 + zslot, RB_BYTES);
      }
    }
    wide_stage1<NX, true>(A, B, s_tw, li);
    line_sync<NX>(bar_id);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float2 t[4];
      wide_stage2_bfly<NX, true>(t, B, s_tw, li + LANES * q);
#pragma unroll
      for (int r = 0; r < 4; ++r) w[q + 4 * r] = t[r];
    }
    const bool use2 = !SPLIT || mt < k2;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      a1[m] = fmaf(dl[m], a1[m], w[m].x);
      if (use2) a2[m] = fmaf(dl[m], a2[m], w[m].y);
    }
  }
  if (!active) return;
  if (m_lo > 0) {
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      part1[row + li + LANES * m] = a1[m];
      part2[row + li + LANES * m] = a2[m];
    }
  } else if constexpr (SPLIT) {
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      float dk = 1.f;
      for (int j = 0; j < split_k; ++j) dk *= dl[m];
      float L = fmaf(dk, a2[m], a1[m]);
      for (int j = 0; j < epi.dpow; ++j) L *= dl[m];  // terms from dpow on
      epilogue_point<float>(epi, (long long)(row + li + LANES * m), L, 0.f);
    }
  } else {
#pragma unroll
    for (int m = 0; m < 16; ++m)
      epilogue_point<float>(epi, (long long)(row + li + LANES * m), a1[m], a2[m] * inv_lambda);
  }
}

// -------------------------------------------------------------------------
// F1 (wide): forward FFT along x of a pair of rows (the complex line
// w[y0] + i w[y0+1] of the discrete Laplacian w, as k2d_fwd_rows), split
// into the two half spectra, on the wide line transform: two lines (row
// pairs) per CTA.  The four rows each line's stencil reads come by TMA bulk
// copies (bounded wait; the line's lanes decide together whether it gave
// up).
// -------------------------------------------------------------------------
template <int NX>
constexpr int wide_frows_lines() {
  return 2;
}
template <int NX>
constexpr int wide_frows_threads() {
  return wide_frows_lines<NX>() * WideFFT<NX>::LANES;
}
template <int NX>
constexpr size_t wide_frows_smem() {
  // per line: buffers A, B, then four staged rows of NX floats
  return (size_t)wide_frows_lines<NX>() * (2 * WideFFT<NX>::PAD_LINE * sizeof(float2) + 4 * NX * sizeof(float));
}

template <int NX>
__device__ __forceinline__ void fwd_rows_wide_body(int bx, const float* __restrict__ u, float2* __restrict__ T,
                                                   int ny, int pT, float ryy, const float2* __restrict__ twx,
                                                   int* step_ctr, int inc_step, int* err) {
  using F = WideFFT<NX>;
  constexpr int LANES = F::LANES, L = wide_frows_lines<NX>(), THREADS = L * LANES, H = NX / 2;
  constexpr uint32_t ROWB = NX * sizeof(float);
  constexpr size_t LINE_BYTES = 2 * F::PAD_LINE * sizeof(float2) + 4 * NX * sizeof(float);
  static_assert(LINE_BYTES % 16 == 0 && (2 * F::PAD_LINE * sizeof(float2)) % 16 == 0, "bulk-copy alignment");
  __shared__ float2 s_tw[F::TW];
  __shared__ uint64_t s_bar[L];
  extern __shared__ __align__(128) unsigned char s_raw[];
  const int line = threadIdx.x / LANES, li = threadIdx.x % LANES;
  const int bar_id = 1 + line;
  float2* A = reinterpret_cast<float2*>(s_raw + (size_t)line * LINE_BYTES);
  float2* B = A + F::PAD_LINE;
  float* srow = reinterpret_cast<float*>(B + F::PAD_LINE);  // rows y0-1, y0, y0+1, y0+2
  uint64_t* bar = &s_bar[line];
  if (li == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < F::TW; i += THREADS) s_tw[i] = twx[i];
  __syncthreads();
  pdl_wait();  // u is written by the previous step's last kernel
  pdl_trigger();
  if (inc_step && bx == 0 && threadIdx.x == 0) *step_ctr += 1;
  const int pair = bx * L + line;
  const bool active = pair < ny / 2;
  const int yy = 2 * (active ? pair : 0);
  if (li == 0) {
    const float* r0 = u + (size_t)yy * NX;
    mbar_arrive_expect_tx(bar, 4 * ROWB);
    bulk_copy_g2s(srow + 0 * NX, u + (size_t)(yy == 0 ? ny - 1 : yy - 1) * NX, ROWB, bar);
    bulk_copy_g2s(srow + 1 * NX, r0, ROWB, bar);
    bulk_copy_g2s(srow + 2 * NX, r0 + NX, ROWB, bar);
    bulk_copy_g2s(srow + 3 * NX, u + (size_t)(yy + 2 == ny ? 0 : yy + 2) * NX, ROWB, bar);
  }
  const bool got = mbar_wait_bounded(bar, 0, err);
  if (line_sync_any<NX>(bar_id, !got)) {
    if (li == 0 && !got) mbar_wait_bounded(bar, 0, err);  // drain (bounded), leave
    return;
  }
  // w = D_xx u + (h_x/h_y)^2 D_yy u of rows y0 (real part) and y0+1 (imag)
  const float* rm = srow;
  const float* ra = srow + NX;
  const float* rb = srow + 2 * NX;
  const float* rp = srow + 3 * NX;
  float2 v[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const int x = li + LANES * m;
    const int xm = x == 0 ? NX - 1 : x - 1, xp = x + 1 == NX ? 0 : x + 1;
    const float a = ra[x], b = rb[x];
    const float dxa = (ra[xp] - a) - (a - ra[xm]);
    const float dxb = (rb[xp] - b) - (b - rb[xm]);
    const float dya = (b - a) - (a - rm[x]);
    const float dyb = (rp[x] - b) - (b - a);
    v[m] = make_float2(dxa + ryy * dya, dxb + ryy * dyb);
  }
  wide_fft<NX, false>(v, A, B, s_tw, li, bar_id);
  // every lane's stage-1 reads of A are done (second barrier of the
  // transform): A takes the spectrum for the split
#pragma unroll
  for (int m = 0; m < 16; ++m) A[F::pad(li + LANES * m)] = v[m];
  line_sync<NX>(bar_id);
  float2* t0 = T + (size_t)yy * pT;
  float2* t1 = t0 + pT;
  for (int k = li; k <= H; k += LANES) {
    const float2 a = A[F::pad(k)];
    const float2 b = A[F::pad(k == 0 ? 0 : NX - k)];
    // A = (X_k + conj X_{-k})/2 (row y0), B = (X_k - conj X_{-k})/(2i) (row y0+1)
    if (active) {
      t0[k] = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
      t1[k] = make_float2(0.5f * (a.y + b.y), -0.5f * (a.x - b.x));
    }
  }
}

template <int NX>
__global__ void __launch_bounds__(wide_frows_threads<NX>())
    k2d_fwd_rows_w(const float* __restrict__ u, float2* __restrict__ T, int ny, int nz, int pT, float ryy,
                   float rzz, const float2* __restrict__ twx, int* step_ctr, int inc_step, int* err) {
  (void)nz;  // 2D only
  (void)rzz;
  fwd_rows_wide_body<NX>(blockIdx.x, u, T, ny, pT, ryy, twx, step_ctr, inc_step, err);
}

template <int NX, bool SPLIT>
__global__ void __launch_bounds__(wide_rows_threads<NX>(), NX == 1024 ? 1 : 6)
    k2d_inv_rows_w(const float2* __restrict__ Z, long long zslot, int pZ, int ny, int m_lo, int m_hi, int top, int k2,
                   int split_k, const float* __restrict__ delta, float* __restrict__ part1,
                   float* __restrict__ part2, EpiArgs<float> epi, float inv_lambda, const float2* __restrict__ twx,
                   int* err, int rsplit) {
  (void)rsplit;  // every row on its own lanes (the wide form has warps enough)
  inv_rows_wide_body<NX, SPLIT>(blockIdx.x, Z, zslot, pZ, ny, m_lo, m_hi, top, k2, split_k, delta, part1, part2, epi,
                                inv_lambda, twx, err);
}

}  // namespace
}  // namespace vofl
