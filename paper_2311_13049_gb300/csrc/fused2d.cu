// fused2d.cu -- fused FP32 kernels for the 2D matrix-free operator pair
// (-Delta)^{1+gamma(x)} u, (-Delta)^{1/2+gamma(x)} u (Eq. (2.13) of
// arXiv 2311.13049) and the leap-frog step of Eq. (1.1) (Eq. (3.4)).
//
// Data path of one step on an nx * ny grid (x fastest), H = nx/2:
//   F1 k2d_fwd_rows   u (ny x nx f32) -> T (ny x (H+1) c64)
//        one line per PAIR of rows: the complex FFT of w[y0] + i w[y0+1],
//        w = the discrete Laplacian of u, split into the two half spectra;
//   F2 k2d_fwd_cols   T -> Uh ((H+1) x ny c64, column-major)
//        complex FFT along y of each of the H+1 columns;
//   then for Taylor groups g = K-1 .. 0 (terms [m_lo, m_hi)):
//   I1 k2d_inv_cols   Uh -> Z[g] (per term and operator, ny x (H+1) c64)
//        multiplier P_op(k) ln|mu_k|^{2m}/m! applied in registers by the
//        recurrence t_m = t_{m-1} ln|mu|^2 / m, then the inverse FFT along y;
//        the M+1 multiplied spectra never exist in memory;
//   I2 k2d_inv_rows   Z[g] -> accumulators / epilogue
//        inverse FFT along x of BOTH operators at once: the row spectra A
//        (operator 1) and B (operator 2) are Hermitian, so one complex
//        inverse FFT of A + iB returns L1-term + i L2-term; the delta^m
//        weights of Eq. (2.13) are applied by Horner's rule in registers
//        (acc = Y_m + delta * acc, m descending), and the last group runs the
//        pointwise leap-frog update (or writes the operator values).
// Only the between-group partial sums (2 fields) and one group of spectra
// (G terms) are stored: storage O(N) in M, against O(MN) for storing every
// term.
// A model with one operator (the general model) puts its terms 0..K-1 in
// the operator-1 slot and K..M in the operator-2 slot (K = ceil((M+1)/2)),
// summed as sum_0 + delta^K sum_1 in the epilogue: half the line
// transforms.  The schedule (kernels_wide.cuh: group_default,
// col_parts_default, col_pack_waves, wide_cols_default, wide_rows_default,
// fuse_forward_default) sets per grid size the terms per group, how the
// column pass deals a group's terms to CTAs, whether the 512/1024-point
// inverse passes use the wide line transform (fft_wide.cuh), and whether
// F2 runs inside the top group's I1 or F1 and F2 share one cooperative
// launch (k2d_fwd_both); vofl_set_schedule overrides it.
// The second-order time splitting of the general model (Sec. 3.3) runs the
// exact flow of its constant-order part on the kernels of kernels_split.cuh
// and the kick with the remainder (terms 1..M) on F1, F2, I1, I2.
//
// Launches use programmatic dependent launch: each kernel does the work
// that does not read its predecessor's output (twiddle and table loads,
// barrier set-up) before griddepcontrol.wait, so it overlaps the tail of
// the previous kernel.  The cooperative launch does not (it is launched
// after its predecessor ends); its successor still overlaps it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "kernels_split.cuh"
#include "kernels_wide.cuh"

namespace vofl {

namespace {

// -------------------------------------------------------------------------
// size dispatch
// -------------------------------------------------------------------------
struct Kernels {
  void (*fwd_rows)(const float*, float2*, int, int, int, float, float, const float2*, int*, int, int*);
  void (*fwd_cols)(const float2*, int, float2*, int, const float2*, long long, long long);
  // both forward passes in one cooperative launch
  void (*fwd_both)(const float*, float2*, float2*, int, int, int, float, const float2*, const float2*, int*, int, int*,
                   unsigned long long*);
  size_t smem_fboth;
  void (*inv_cols)(float2*, const float*, const float*, CUtensorMap, int, int, int, float, float, int, int, int,
                   const float2*, const float2*, int, int, int);
  using InvRows = void (*)(const float2*, long long, int, int, int, int, int, int, int, const float*, float*, float*,
                           EpiArgs<float>, float, const float2*, int*, int);
  using InvColsW = void (*)(const float2*, const float*, const float*, float2*, int, int, int, int, float, float, int,
                            int, int, const float2*, int);
  InvRows inv_rows;        // two operators
  InvRows inv_rows_split;  // one operator, terms split over the slots
  // wide line transforms (fft_wide.cuh) of the inverse passes, for lines of
  // 512 and 1024 points (null elsewhere)
  InvColsW inv_cols_w = nullptr;
  InvRows inv_rows_w = nullptr, inv_rows_w_split = nullptr;
  void (*fwd_rows_w)(const float*, float2*, int, int, int, float, float, const float2*, int*, int, int*) = nullptr;
  size_t smem_frows_w = 0;
  int rpc_fw = 0, thr_fw = 0;  // row pairs per CTA / threads of the wide forward row kernel
  size_t smem_frows, smem_fcols, smem_icols, smem_irows, smem_icols_w = 0, smem_irows_w = 0;
  int lpw_x, lpw_y;
  int wic;  // warps per CTA of inv_cols
  int wir;  // warps (rows) per CTA of inv_rows
  int cpc_w = 0, rpc_w = 0, thr_w_c = 0, thr_w_r = 0;  // lines per CTA / threads of the wide kernels
  // the exact flow of the time splitting (kernels_split.cuh)
  void (*rot_rows)(const float*, const float*, float2*, float2*, int, int, const float2*);
  void (*rot_cols)(float2*, float2*, const float*, float, float, int, int, const float2*);
  void (*rot_irows)(const float2*, const float2*, float*, float*, int, int, const float2*);
  size_t smem_rot_rows, smem_rot_cols;
};

// warps per CTA of the inverse row kernel: 7 at 1024^2 (147 CTAs, one per
// SM, instead of 256 four-row CTAs in 1.7 waves: a 1.4% shorter step), one
// (two 16-lane rows) at 512^2 (256 CTAs instead of 64), 4 elsewhere
template <int NX, int NY>
constexpr int irows_warps() {
  return (NX == 1024 && NY == 1024) ? 7 : (NX == 512 && NY == 512) ? 1 : W_IROWS;
}

template <int NX, int NY>
Kernels kernels_for() {
  Kernels k;
  constexpr int WR = irows_warps<NX, NY>();
  k.wir = WR;
  k.fwd_rows = k2d_fwd_rows<NX, false>;
  k.fwd_cols = k2d_fwd_cols<NY>;
  k.fwd_both = k2d_fwd_both<NX, NY>;
  k.smem_fboth = fboth_smem<NX, NY>();
  k.inv_cols = k2d_inv_cols<NY>;
  k.inv_rows = k2d_inv_rows<NX, false, WR>;
  k.inv_rows_split = k2d_inv_rows<NX, true, WR>;
  k.smem_frows = frows_smem<NX, false>();
  k.smem_fcols = exch_smem<NY, W_FCOLS>();
  k.smem_icols = inv_cols_smem<NY>();
  k.smem_irows = inv_rows_smem<NX, WR>();
  k.lpw_x = LineFFT<NX>::LPW;
  k.lpw_y = LineFFT<NY>::LPW;
  k.wic = icols_warps<NY>();
  k.rot_rows = k2d_rot_fwd_rows<NX>;
  k.rot_cols = k2d_rot_cols<NY>;
  k.rot_irows = k2d_rot_inv_rows<NX>;
  k.smem_rot_rows = rot_rows_smem<NX>();
  k.smem_rot_cols = rot_cols_smem<NY>();
  if constexpr (NY == 512 || NY == 1024) {
    k.inv_cols_w = k2d_inv_cols_w<NY>;
    k.smem_icols_w = wide_cols_smem<NY>();
    k.cpc_w = wide_lines_per_cta<NY>();
    k.thr_w_c = wide_threads<NY>();
  }
  if constexpr (NX == 512 || NX == 1024) {
    k.inv_rows_w = k2d_inv_rows_w<NX, false>;
    k.inv_rows_w_split = k2d_inv_rows_w<NX, true>;
    k.fwd_rows_w = k2d_fwd_rows_w<NX>;
    k.smem_frows_w = wide_frows_smem<NX>();
    k.rpc_fw = wide_frows_lines<NX>();
    k.thr_fw = wide_frows_threads<NX>();
    k.smem_irows_w = wide_rows_smem<NX>();
    k.rpc_w = wide_rows_per_cta<NX>();
    k.thr_w_r = wide_rows_threads<NX>();
  }
  return k;
}

bool pick_kernels(int nx, int ny, Kernels* k) {
#define VOFL_CASE(X, Y)            \
  if (nx == X && ny == Y) {        \
    *k = kernels_for<X, Y>();      \
    return true;                   \
  }
  VOFL_CASE(64, 64)
  VOFL_CASE(128, 128)
  VOFL_CASE(256, 256)
  VOFL_CASE(512, 512)
  VOFL_CASE(768, 768)
  VOFL_CASE(1024, 1024)
  VOFL_CASE(256, 128)
  VOFL_CASE(128, 256)
  VOFL_CASE(512, 64)
  VOFL_CASE(64, 512)
  VOFL_CASE(1024, 256)
#undef VOFL_CASE
  return false;
}

int set_smem_attributes(const Kernels& k) {
  if (set_kernel_smem(k.fwd_rows, k.smem_frows) ||
      set_kernel_smem(k.fwd_cols, k.smem_fcols) || set_kernel_smem(k.fwd_both, k.smem_fboth) ||
      set_kernel_smem(k.inv_cols, k.smem_icols) ||
      set_kernel_smem(k.inv_rows, k.smem_irows) || set_kernel_smem(k.inv_rows_split, k.smem_irows) ||
      (k.inv_cols_w && set_kernel_smem(k.inv_cols_w, k.smem_icols_w)) ||
      (k.inv_rows_w && (set_kernel_smem(k.inv_rows_w, k.smem_irows_w) ||
                        set_kernel_smem(k.inv_rows_w_split, k.smem_irows_w))) ||
      (k.fwd_rows_w && set_kernel_smem(k.fwd_rows_w, k.smem_frows_w)) ||
      set_kernel_smem(k.rot_rows, k.smem_rot_rows) || set_kernel_smem(k.rot_irows, k.smem_rot_rows) ||
      set_kernel_smem(k.rot_cols, k.smem_rot_cols)) {
    cudaGetLastError();
    return VOFL_ECUDA;
  }
  return VOFL_OK;
}

// Every buffer and constant one fused 2D apply / step needs.
struct Plan2D {
  Kernels k{};
  int nx = 0, ny = 0, ncols = 0, pT = 0, pZ = 0, G = 6;
  long long zslot = 0;
  float2 *T = nullptr, *Uh = nullptr, *Z = nullptr;
  float* part = nullptr;  // 2 fields
  float* P = nullptr;     // [2][ncols][ny]
  float* Lg = nullptr;    // [ncols][ny]
  float2 *twx = nullptr, *twy = nullptr;
  float2 *twxw = nullptr, *twyw = nullptr;  // wide line twiddles (512, 1024 points)
  float* Wrot = nullptr;  // time splitting: sqrt(kappa) |mu|^{s0}, [ncols][ny] (general model)
  // flow tables over dt and over dt/2 ([2][3][ncols][ny], k_flow_table) and
  // the dt they were built for (NaN: none)
  float* flow = nullptr;
  double flow_dt = std::nan("");
  const float* delta = nullptr;
  int* step_ctr = nullptr;
  int* err = nullptr;
  float ryy = 1.f, inv_lambda = 1.f;
  CUtensorMap zmap{};  // Z as [2 G ny rows][pZ] for the column kernel's tile stores
  // schedule: wide line transforms in the inverse column / row passes
  // (where built), the column-pass term split (0: col_parts_default), and
  // the forward column transform done inside the top group's inverse
  // column kernel (32-element column kernel only)
  bool wide_c = false, wide_r = false, wide_f = false;
  // forward passes: 0 two kernels, 1 the column transform inside the top
  // group's column kernel, 2 both passes in one cooperative launch
  int fuse_fwd = 0;
  int both_grid = 0;                   // CTAs of that launch (0: not resident-safe here)
  unsigned long long* gbar = nullptr;  // its grid barrier's count and generation
  int cparts = 0;
  int cpack = 0;   // > 0: the column pass's terms dealt out over cpack CTAs (col_run)
  int rsplit = 1;  // runs of terms per row in the (32-element) row kernel

  bool fused_forward() const { return fuse_fwd == 1 && !(wide_c && k.inv_cols_w); }
  bool forward_both() const { return fuse_fwd == 2 && both_grid > 0 && !(wide_f && k.fwd_rows_w); }
  bool one_forward_launch() const { return fused_forward() || forward_both(); }

  // one_op: a model with one operator (its terms fill both slots)
  int groups(int M, bool one_op = false) const { return (term_split(M, one_op).slots + G - 1) / G; }

  int make_zmap() {
    return make_tile_map(&zmap, Z, ncols, 2LL * G * ny, pZ, k.wic * k.lpw_y, std::min(ny, 256));
  }

  // optional events: ev[1] after F1, ev[2] after F2 (ev[0] recorded by the
  // caller).  coop = false: the two forward kernels even where the schedule
  // has the cooperative launch (same bits), for eagerly launched applies:
  // there the cooperative launch cost more than the boundary it saves (the
  // generic 512^2 apply, M = 20: 0.0395 ms with it, 0.0365 without), while
  // steps replay it from a graph
  cudaError_t forward(cudaStream_t s, const float* u, bool inc_step, cudaEvent_t* ev = nullptr,
                      bool coop = true) const {
    cudaError_t e;
    if (coop && forward_both()) {
      e = launch_coop(k.fwd_both, dim3(both_grid), dim3(W_FBOTH * 32), k.smem_fboth, s, u, T, Uh, ny, pT, ncols, ryy,
                      (const float2*)twx, (const float2*)twy, step_ctr, inc_step ? 1 : 0, err, gbar);
      if (!e && ev) cudaEventRecord(ev[1], s);
      return e;
    }
    if (wide_f && k.fwd_rows_w) {
      e = launch_pdl(k.fwd_rows_w, dim3((ny / 2 + k.rpc_fw - 1) / k.rpc_fw), dim3(k.thr_fw), k.smem_frows_w, s, u, T,
                     ny, 1, pT, ryy, 0.0f, (const float2*)twxw, step_ctr, inc_step ? 1 : 0, err);
    } else {
      const int rpc = W_FROWS * k.lpw_x;  // row pairs per CTA
      e = launch_pdl(k.fwd_rows, dim3((ny / 2 + rpc - 1) / rpc), dim3(W_FROWS * 32), k.smem_frows, s, u, T, ny, 1,
                     pT, ryy, 0.0f, (const float2*)twx, step_ctr, inc_step ? 1 : 0, err);
    }
    if (e) return e;
    if (ev) cudaEventRecord(ev[1], s);
    if (fused_forward()) return cudaSuccess;  // the top group's column kernel does F2
    const int cpc = W_FCOLS * k.lpw_y;
    e = launch_pdl(k.fwd_cols, dim3((ncols + cpc - 1) / cpc), dim3(W_FCOLS * 32), k.smem_fcols, s, (const float2*)T,
                   pT, Uh, ncols, (const float2*)twy, 0LL, 0LL);
    if (ev) cudaEventRecord(ev[2], s);
    return e;
  }

  // optional events: one after every inverse kernel, from ev[3] on (ev[2]
  // when the forward column transform is fused)
  // base > 0 (one operator only): the terms base..M of the expansion (the
  // splitting's remainder, Sec. 3.3: base = 1), the epilogue's L1 carrying
  // the factor delta^base (epi.dpow = base)
  cudaError_t inverse(cudaStream_t s, int M, const EpiArgs<float>& epi, cudaEvent_t* ev = nullptr,
                      bool one_op = false, int base = 0, bool coop = true) const {
    const TermSplit ts = term_split(M - base, one_op);
    const int K = groups(M - base, one_op);
    const bool wc = wide_c && k.inv_cols_w, wr = wide_r && k.inv_rows_w;
    const int cpc = wc ? k.cpc_w : k.wic * k.lpw_y;
    const int parts = cparts > 0 ? cparts : col_parts_default(ny);
    const dim3 gic = cpack > 0 ? dim3(cpack) : dim3((ncols + cpc - 1) / cpc, 2 * parts);
    const int rsp = wr ? 1 : rsplit;
    const int rpc = wr ? k.rpc_w : (k.wir / rsp) * k.lpw_x;
    const dim3 gir((ny + rpc - 1) / rpc);
    const bool ff = fused_forward();
    int e_i = (fused_forward() || (coop && forward_both())) ? 2 : 3;
    for (int gi = K - 1; gi >= 0; --gi) {
      const int m_lo = gi * G, m_hi = std::min(ts.slots, m_lo + G);
      const float f0 = inv_factorial(m_lo + base), f1 = ts.split_k ? inv_factorial(m_lo + base + ts.split_k) : f0;
      cudaError_t e;
      if (wc)
        e = launch_pdl(k.inv_cols_w, gic, dim3(k.thr_w_c), k.smem_icols_w, s, (const float2*)Uh, (const float*)P,
                       (const float*)Lg, Z, pZ, ncols, m_lo, m_hi, f0, f1, ts.split_k, parts, cpack,
                       (const float2*)twyw, base);
      else
        e = launch_pdl(k.inv_cols, gic, dim3(k.wic * 32), k.smem_icols, s, Uh, (const float*)P,
                       (const float*)Lg, zmap, ncols, m_lo, m_hi, f0, f1, ts.split_k, parts, cpack, (const float2*)twy,
                       (const float2*)T, pT, (ff && gi == K - 1) ? 1 : 0, base);
      if (e) return e;
      if (ev) cudaEventRecord(ev[e_i++], s);
      EpiArgs<float> ep = epi;
      if (gi > 0) ep.mode = EPI_PARTIAL;
      Kernels::InvRows kr = wr ? (one_op ? k.inv_rows_w_split : k.inv_rows_w) : (one_op ? k.inv_rows_split : k.inv_rows);
      e = launch_pdl(kr, gir, dim3(wr ? k.thr_w_r : k.wir * 32), wr ? k.smem_irows_w : k.smem_irows, s,
                     (const float2*)Z, zslot, pZ, ny, m_lo, m_hi,
                     gi == K - 1 ? 1 : 0, ts.k2, ts.split_k, delta, part, part + (size_t)nx * ny, ep, inv_lambda,
                     (const float2*)(wr ? twxw : twx), err, rsp);
      if (e) return e;
      if (ev) cudaEventRecord(ev[e_i++], s);
    }
    return cudaSuccess;
  }

  // The exact flow of the splitting over time t (Sec. 3.3) on u, v in place
  // (kernels_split.cuh), three launches.  Scratch: the row spectra in the Z
  // buffer (two [ny][pT] planes; Z holds at least that).
  // half: the flow over dt/2 (else over dt); sign -1: backwards
  cudaError_t rotate(cudaStream_t s, float* u, float* v, bool half, float sign) const {
    float2* Su = Z;
    float2* Sv = Z + (size_t)ny * pT;
    const float invN = (float)(1.0 / ((double)nx * (double)ny));
    const int rpc = W_ROT * k.lpw_x, cpc = W_ROT * k.lpw_y;
    const float* tab = flow + (half ? (size_t)3 * ncols * ny : 0);
    cudaError_t e = launch_pdl(k.rot_rows, dim3((ny + rpc - 1) / rpc), dim3(W_ROT * 32), k.smem_rot_rows, s,
                               (const float*)u, (const float*)v, Su, Sv, ny, pT, (const float2*)twx);
    if (!e)
      e = launch_pdl(k.rot_cols, dim3((ncols + cpc - 1) / cpc), dim3(W_ROT * 32), k.smem_rot_cols, s, Su, Sv, tab,
                     sign, invN, pT, ncols, (const float2*)twy);
    if (!e)
      e = launch_pdl(k.rot_irows, dim3((ny + rpc - 1) / rpc), dim3(W_ROT * 32), k.smem_rot_rows, s,
                     (const float2*)Su, (const float2*)Sv, u, v, ny, pT, (const float2*)twx);
    return e;
  }

};

// constants of a model on an nx * ny box of size lx * ly
void plan_constants(int nx, int ny, double lx, double ly, int* e2, float* ryy) {
  const double mx = M_PI * nx / lx, my = M_PI * ny / ly;
  *e2 = (int)std::lround(0.5 * std::log2(std::max(std::sqrt(mx * mx + my * my), 1.0)));
  const double hx = lx / nx, hy = ly / ny;
  *ryy = (float)((hx * hx) / (hy * hy));
}

struct Fused2D : Engine {
  Plan2D p;
  size_t nbytes = 0;
  // Operator 2's multiplier carries an exact power-of-two factor lambda so
  // that the two operators packed into one complex row transform (A + iB)
  // have comparable magnitude (|P1/P2| = |mu|); the row transform's
  // round-off is relative to |A + iB|, so without it operator 2 would see
  // round-off up to |mu|_max times its own size.  lambda ~ sqrt(|mu|_max)
  // balances the two; it is divided out exactly in the epilogue.
  double lambda = 1.0;
  int zcap = 0;  // Taylor terms the group buffer holds (>= p.G)

  ~Fused2D() override {
    dev_free(p.T);
    dev_free(p.Uh);
    dev_free(p.Z);
    dev_free(p.part);
    dev_free(p.P);
    dev_free(p.Lg);
    dev_free(p.twx);
    dev_free(p.twy);
    dev_free(p.twxw);
    dev_free(p.twyw);
    dev_free(p.Wrot);
    dev_free(p.flow);
    dev_free(p.gbar);
  }

  size_t bytes() const override { return nbytes; }

  bool batch_desc(const vofl_ctx* c, BatchSim* d) const override {
    (void)c;
    // the batched launches follow the size class's transform schedule,
    // which the batch takes from (and checks against) its members'
    // (vofl_batch_add)
    d->T = p.T;
    d->Uh = p.Uh;
    d->Z = p.Z;
    d->part = p.part;
    d->P = p.P;
    d->Lg = p.Lg;
    d->twx = p.twx;
    d->twy = p.twy;
    d->twxw = p.twxw;
    d->twyw = p.twyw;
    d->ryy = p.ryy;
    d->inv_lambda = p.inv_lambda;
    d->zslot = p.zslot;
    d->zmap = p.zmap;
    d->pT = p.pT;
    d->pZ = p.pZ;
    return true;
  }

  int alloc(vofl_ctx* c, void** ptr, size_t b) {
    cudaError_t e = dev_malloc(ptr, b);
    if (e != cudaSuccess) return cuda_err(c, e, "cudaMalloc (fused 2D scratch)");
    nbytes += b;
    return VOFL_OK;
  }

  int init(vofl_ctx* c) {
    p.nx = (int)c->n[0];
    p.ny = (int)c->n[1];
    p.ncols = p.nx / 2 + 1;
    if (!pick_kernels(p.nx, p.ny, &p.k)) return set_err(c, VOFL_EUNSUPPORTED, "fused 2D path: grid size not built");
    p.pT = round_up(p.ncols, 8);
    p.pZ = p.pT;
    p.zslot = (long long)p.ny * p.pZ;
    p.G = group_default(p.nx, p.ny);
    int st;
    const size_t nx = p.nx, ny = p.ny, nc = p.ncols;
    if ((st = alloc(c, (void**)&p.T, sizeof(float2) * ny * p.pT))) return st;
    if ((st = alloc(c, (void**)&p.Uh, sizeof(float2) * nc * ny))) return st;
    if ((st = alloc(c, (void**)&p.Z, sizeof(float2) * (size_t)p.zslot * 2 * p.G))) return st;
    zcap = p.G;
    if ((st = alloc(c, (void**)&p.part, sizeof(float) * 2 * nx * ny))) return st;
    if ((st = alloc(c, (void**)&p.P, sizeof(float) * 2 * nc * ny))) return st;
    if ((st = alloc(c, (void**)&p.Lg, sizeof(float) * nc * ny))) return st;
    if ((st = alloc(c, (void**)&p.twx, sizeof(float2) * line_twiddle_entries(p.nx)))) return st;
    if ((st = alloc(c, (void**)&p.twy, sizeof(float2) * line_twiddle_entries(p.ny)))) return st;
    if (p.k.inv_rows_w && (st = alloc(c, (void**)&p.twxw, sizeof(float2) * wide_twiddle_entries(p.nx)))) return st;
    if (p.k.inv_cols_w && (st = alloc(c, (void**)&p.twyw, sizeof(float2) * wide_twiddle_entries(p.ny)))) return st;
    p.wide_c = p.k.inv_cols_w != nullptr && wide_cols_default(p.ny);
    p.wide_r = p.k.inv_rows_w != nullptr && wide_rows_default(p.nx);
    p.fuse_fwd = fuse_forward_default(p.nx, p.ny);
    p.wide_f = p.k.fwd_rows_w != nullptr && wide_fwd_default(p.nx);
    p.rsplit = row_split_default(p.nx, p.ny, p.k.wir);
    if (set_smem_attributes(p.k)) return set_err(c, VOFL_ECUDA, "shared-memory attributes of the fused kernels");
    p.cpack = col_pack_waves(p.nx, p.ny) * device_sm_count();
    // the two-pass forward launch: one block of rows and one of columns per
    // CTA where one wave holds them all, never more CTAs than fit at once
    if ((st = alloc(c, (void**)&p.gbar, 2 * sizeof(unsigned long long)))) return st;
    if (cudaMemsetAsync(p.gbar, 0, 2 * sizeof(unsigned long long), c->stream) != cudaSuccess)
      return cuda_err(c, cudaGetLastError(), "grid-barrier counter");
    {
      int dev = 0, coop = 0, per = 0;
      const int sms = device_sm_count();
      if (cudaGetDevice(&dev) == cudaSuccess &&
          cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, p.k.fwd_both, W_FBOTH * 32, p.k.smem_fboth) ==
              cudaSuccess) {
        const int rb = W_FBOTH * p.k.lpw_x, cb = W_FBOTH * p.k.lpw_y;
        const int want = std::max((p.ny / 2 + rb - 1) / rb, (p.ncols + cb - 1) / cb);
        p.both_grid = std::min(want, sms * per);
      }
      cudaGetLastError();
    }
    if (make_line_twiddles(p.nx, p.twx, c->stream) ||
        make_line_twiddles(p.ny, p.twy, c->stream) ||
        (p.twxw && make_wide_twiddles(p.nx, p.twxw, c->stream)) ||
        (p.twyw && make_wide_twiddles(p.ny, p.twyw, c->stream)))
      return cuda_err(c, cudaGetLastError(), "twiddles");
    p.delta = (const float*)c->delta;
    p.step_ctr = c->d_step;
    p.err = c->d_step + 1;
    if (p.make_zmap()) return set_err(c, VOFL_ECUDA, "tensor map of the Z buffer");
    return VOFL_OK;
  }

  int set_model(vofl_ctx* c) override {
    const double lx = c->hi[0] - c->lo[0], ly = c->hi[1] - c->lo[1];
    int e2;
    plan_constants(p.nx, p.ny, lx, ly, &e2, &p.ryy);
    lambda = std::ldexp(1.0, e2);
    p.inv_lambda = std::ldexp(1.0f, -e2);
    if (make_fused2d_tables(p.nx, p.ny, lx, ly, c->s01, c->s02, lambda, (double)p.ryy, p.P, p.Lg,
                            c->stream))
      return cuda_err(c, cudaGetLastError(), "fused 2D tables");
    if (c->general) {  // the time splitting's frequencies (Sec. 3.3)
      if (!p.Wrot) {
        const size_t b = sizeof(float) * (size_t)p.ncols * p.ny;
        if (int st = alloc(c, (void**)&p.Wrot, b)) return st;
      }
      if (!p.flow) {
        const size_t b = sizeof(float) * 6 * (size_t)p.ncols * p.ny;
        if (int st = alloc(c, (void**)&p.flow, b)) return st;
      }
      if (make_fused2d_omega(p.nx, p.ny, lx, ly, c->s01, c->kappa, p.Wrot, c->stream))
        return cuda_err(c, cudaGetLastError(), "splitting frequency table");
      p.flow_dt = std::nan("");  // the flow tables follow the frequencies
    }
    return VOFL_OK;
  }

  // Second-order time splitting (Sec. 3.3) of the general model: the exact
  // flow of the constant-order part, the kick with the variable-order
  // remainder (terms 1..M of Eq. (2.13), on the operator kernels) and f(u).
  // Consecutive half-step flows are merged: a step is the kick followed by
  // the flow over dt, and a run is bracketed by the flows over +dt/2 and
  // -dt/2 (vofl_step), one flow per step instead of two.
  bool can_split() const override { return true; }
  bool split_merged() const override { return true; }
  int split_flow(vofl_ctx* c, double t) override {
    if (!p.Wrot || !p.flow) return set_err(c, VOFL_ESTATE, "set the general model first");
    if (!(p.flow_dt == c->dt)) {  // flow tables for this dt (outside any capture: a run starts here)
      const long long n = (long long)p.ncols * p.ny;
      const unsigned g = (unsigned)std::min<long long>((n + 255) / 256, 4096);
      k_flow_table<<<g, 256, 0, c->stream>>>(p.Wrot, c->dt, p.flow, n);
      k_flow_table<<<g, 256, 0, c->stream>>>(p.Wrot, 0.5 * c->dt, p.flow + 3 * n, n);
      count_launch(2);
      if (cudaGetLastError() != cudaSuccess) return set_err(c, VOFL_ECUDA, "splitting flow tables");
      p.flow_dt = c->dt;
    }
    // the bracketing flows of a run: over +dt/2 and -dt/2
    cudaError_t err = p.rotate(c->stream, (float*)c->u[c->cur], (float*)c->u[1 - c->cur], true, t < 0 ? -1.f : 1.f);
    if (err) return cuda_err(c, err, "fused 2D splitting flow");
    return VOFL_OK;
  }
  int step_split(vofl_ctx* c) override {
    // the flow tables of c->dt were built by split_flow, which every run
    // starts with
    if (!p.Wrot || !p.flow || !(p.flow_dt == c->dt)) return set_err(c, VOFL_ESTATE, "set the general model first");
    float* u = (float*)c->u[c->cur];
    float* v = (float*)c->u[1 - c->cur];
    cudaError_t err = cudaSuccess;
    if (c->M >= 1) {
      EpiArgs<float> e{};
      e.mode = EPI_KICK;
      e.u_cur = u;
      e.u_other = v;
      e.A = (const float*)c->A;
      e.dt1 = (float)c->dt;
      e.src_flat = -1;
      e.dpow = 1;
      epi_model(c, &e);
      err = p.forward(c->stream, u, false);
      if (!err) err = p.inverse(c->stream, c->M, e, nullptr, true, 1);
    } else {
      const long long n = (long long)p.nx * p.ny;
      err = launch_pdl(k2d_kick_f, dim3((unsigned)std::min<long long>((n + 255) / 256, 4096)), dim3(256), 0,
                       c->stream, (const float*)u, v, n, (float)c->dt, (float)c->f1, (float)c->f3);
    }
    if (!err) err = p.rotate(c->stream, u, v, false, 1.f);
    if (err) return cuda_err(c, err, "fused 2D splitting step");
    return VOFL_OK;
  }

  // a grid barrier that timed out leaves its count short of a full round
  void reset_waits(vofl_ctx* c) override {
    (void)c;
    if (p.gbar && cudaMemset(p.gbar, 0, 2 * sizeof(unsigned long long)) != cudaSuccess) cudaGetLastError();
  }

  uint64_t kernels_per_step(const vofl_ctx* c) const override {
    return (p.one_forward_launch() ? 1 : 2) + 2 * (uint64_t)p.groups(c->M, c->general);
  }

  int set_schedule(vofl_ctx* c, const vofl_schedule* s) override {
    if (s->row_split != 0 && p.k.wir % s->row_split != 0)
      return set_err(c, VOFL_EINVAL, "row_split must divide the row kernel's warps per CTA");
    const bool wc = p.k.inv_cols_w && (s->wide_cols < 0 ? wide_cols_default(p.ny) : s->wide_cols == 1);
    const bool wr = p.k.inv_rows_w && (s->wide_rows < 0 ? wide_rows_default(p.nx) : s->wide_rows == 1);
    const int G = s->group == 0 ? group_default(p.nx, p.ny) : s->group;
    if (G > zcap) {  // a larger group buffer; a smaller group uses the one there is
      const size_t b_old = sizeof(float2) * (size_t)p.zslot * 2 * zcap;
      const size_t b_new = sizeof(float2) * (size_t)p.zslot * 2 * G;
      float2* z = nullptr;
      cudaError_t e = dev_malloc((void**)&z, b_new);
      if (e != cudaSuccess) return cuda_err(c, e, "cudaMalloc (Taylor group buffer)");
      dev_free(p.Z);
      p.Z = z;
      zcap = G;
      nbytes = nbytes - b_old + b_new;
    }
    if (G != p.G) {
      p.G = G;
      if (p.make_zmap()) return set_err(c, VOFL_ECUDA, "tensor map of the Z buffer");
    }
    p.wide_c = wc;
    p.wide_r = wr;
    p.cparts = s->col_parts;
    p.cpack = s->col_pack < 0 ? col_pack_waves(p.nx, p.ny) * device_sm_count() : s->col_pack;
    p.fuse_fwd = s->fuse_forward < 0 ? fuse_forward_default(p.nx, p.ny) : s->fuse_forward;
    p.wide_f = p.k.fwd_rows_w && (s->wide_fwd < 0 ? wide_fwd_default(p.nx) : s->wide_fwd == 1);
    p.rsplit = s->row_split == 0 ? row_split_default(p.nx, p.ny, p.k.wir) : s->row_split;
    return VOFL_OK;
  }

  int get_schedule(const vofl_ctx* c, vofl_schedule* s) const override {
    (void)c;
    s->wide_cols = p.wide_c && p.k.inv_cols_w ? 1 : 0;
    s->wide_rows = p.wide_r && p.k.inv_rows_w ? 1 : 0;
    s->col_parts = p.cparts > 0 ? p.cparts : col_parts_default(p.ny);
    s->col_pack = p.cpack;
    s->group = p.G;
    s->fuse_forward = p.forward_both() ? 2 : p.fused_forward() ? 1 : 0;
    s->wide_fwd = p.wide_f && p.k.fwd_rows_w ? 1 : 0;
    s->row_split = (p.wide_r && p.k.inv_rows_w) ? 1 : p.rsplit;
    return VOFL_OK;
  }

  int apply_pair(vofl_ctx* c, const void* u, void* o1, void* o2) override {
    EpiArgs<float> e{};
    e.mode = EPI_APPLY;
    e.out1 = (float*)o1;
    e.out2 = (float*)o2;
    e.src_flat = -1;
    cudaError_t err = p.forward(c->stream, (const float*)u, false, nullptr, false);
    if (!err) err = p.inverse(c->stream, c->M, e, nullptr, c->general, 0, false);
    if (err) return cuda_err(c, err, "fused 2D launch");
    return VOFL_OK;
  }

  int step(vofl_ctx* c, int mode, bool count_step) override {
    EpiArgs<float> e{};
    e.mode = mode;
    e.u_cur = (const float*)c->u[c->cur];
    e.u_other = (float*)c->u[1 - c->cur];
    e.l2p = (float*)c->l2p;
    e.A = (const float*)c->A;
    e.B = (const float*)c->B;
    e.dt1 = (float)c->dt;
    e.dt2 = (float)(c->dt * c->dt);
    e.src_flat = c->nsrc > 0 ? c->src_flat : -1;
    e.src = c->d_src;
    e.nsrc = c->nsrc;
    e.step = c->d_step;
    double hd = 1.0;
    for (int i = 0; i < c->ndim; ++i) hd *= (c->hi[i] - c->lo[i]) / (double)c->n[i];
    e.src_scale = c->dt * c->dt / hd;
    epi_model(c, &e);
    cudaError_t err = p.forward(c->stream, (const float*)c->u[c->cur], count_step);
    if (!err) err = p.inverse(c->stream, c->M, e, nullptr, c->general);
    if (err) return cuda_err(c, err, "fused 2D launch");
    return VOFL_OK;
  }

  // Time every kernel of one operator-pair application in its real order
  // (events recorded between consecutive kernels on the context stream),
  // averaged over `reps` repetitions; each interval is the kernel's
  // duration plus its launch gap.  The epilogue writes nothing (apply mode
  // with null outputs), so the context state is unchanged.
  int profile(vofl_ctx* c, int reps, std::string& names, double* ms, double* units, int cap) override {
    if (cap < 4) return 0;
    const int K = p.groups(c->M, c->general);
    const int slots = term_split(c->M, c->general).slots;
    const bool ff = p.fused_forward(), one = p.one_forward_launch();
    const int base = one ? 1 : 2;  // event after which the first inverse kernel starts
    const int nk = base + 2 * K;
    // one event set per repetition; all repetitions are queued back to back
    // (one warm-up first) and read after a single synchronisation, so the
    // host launch latency never shows up in the intervals
    const int R = reps + 1;
    std::vector<cudaEvent_t> ev((size_t)R * (nk + 1));
    for (auto& e : ev) cudaEventCreate(&e);
    EpiArgs<float> ep{};
    ep.mode = EPI_APPLY;
    ep.src_flat = -1;
    const float* u = (const float*)c->u[c->cur];
    double acc[4] = {0, 0, 0, 0};
    double terms = 0;
    for (int g = 0; g < K; ++g) terms += std::min(slots, (g + 1) * p.G) - g * p.G;
    for (int r = 0; r < R; ++r) {
      cudaEvent_t* er = ev.data() + (size_t)r * (nk + 1);
      cudaEventRecord(er[0], c->stream);
      cudaError_t err = p.forward(c->stream, u, false, er);
      if (!err) err = p.inverse(c->stream, c->M, ep, er, c->general);
      if (err) {
        for (auto& e : ev) cudaEventDestroy(e);
        return cuda_err(c, err, "profile");
      }
    }
    cudaEventSynchronize(ev.back());
    for (int r = 1; r < R; ++r) {
      const cudaEvent_t* er = ev.data() + (size_t)r * (nk + 1);
      float t;
      cudaEventElapsedTime(&t, er[0], er[1]);
      acc[0] += t;
      if (!one) {
        cudaEventElapsedTime(&t, er[1], er[2]);
        acc[1] += t;
      }
      for (int i = 0; i < K; ++i) {
        cudaEventElapsedTime(&t, er[base + 2 * i], er[base + 2 * i + 1]);
        acc[2] += t;
        cudaEventElapsedTime(&t, er[base + 2 * i + 1], er[base + 2 * i + 2]);
        acc[3] += t;
      }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    const bool wc = p.wide_c && p.k.inv_cols_w, wr = p.wide_r && p.k.inv_rows_w;
    const std::string ic = wc ? "k2d_inv_cols_w" : "k2d_inv_cols", ir = wr ? "k2d_inv_rows_w" : "k2d_inv_rows";
    // ms = average per launch; units = complex line transforms per launch
    // (algorithmic: a fused forward column transform counts once per step)
    int n = 0;
    std::string nm = p.forward_both() ? "k2d_fwd_both" : p.wide_f && p.k.fwd_rows_w ? "k2d_fwd_rows_w" : "k2d_fwd_rows";
    ms[n] = acc[0] / reps;
    units[n++] = p.ny / 2.0 + (p.forward_both() ? p.ncols : 0);
    if (!one) {
      nm += ";k2d_fwd_cols";
      ms[n] = acc[1] / reps;
      units[n++] = p.ncols;
    }
    nm += ";" + ic + ";" + ir;
    ms[n] = acc[2] / reps / K;
    units[n++] = (2.0 * p.ncols * terms + (ff ? p.ncols : 0)) / K;
    ms[n] = acc[3] / reps / K;
    units[n++] = (double)p.ny * terms / K;
    names = nm;
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_err(c, err, "profile");
    return n;
  }
};

}  // namespace

bool fused2d_supported(int ndim, const int64_t* n, int prec) {
  Kernels k;
  return ndim == 2 && prec == VOFL_F32 && pick_kernels((int)n[0], (int)n[1], &k);
}

size_t fused2d_footprint(const int64_t* n, int M) {
  const size_t nx = n[0], ny = n[1], nc = nx / 2 + 1, p = (nc + 7) / 8 * 8;
  (void)M;  // the group buffer is sized for the grid's default group, whatever M
  const size_t G = group_default((int)nx, (int)ny);
  const size_t tww = (wide_line((int)nx) ? wide_twiddle_entries((int)nx) : 0) +
                     (wide_line((int)ny) ? wide_twiddle_entries((int)ny) : 0);
  // float tables: P (two), ln|mu|^2 and, for the general model, the time
  // splitting's frequencies (counted always: an upper bound); then the
  // grid barrier's two words
  return sizeof(float2) * (ny * p + nc * ny + ny * p * 2 * G + line_twiddle_entries((int)nx) +
                           line_twiddle_entries((int)ny) + tww) +
         sizeof(float) * (2 * nx * ny + 4 * nc * ny) + 2 * sizeof(unsigned long long);
}

Engine* make_fused2d(vofl_ctx* c, int* status) {
  Fused2D* e = new Fused2D();
  *status = e->init(c);
  if (*status != VOFL_OK) {
    delete e;
    return nullptr;
  }
  return e;
}

}  // namespace vofl

// ---------------------------------------------------------------------------
// Allocation-free operator pair for small 2D grids.
//
// Some callers cannot allocate device memory at the moment they need the
// operator: code that runs while an outside allocator owns the whole GPU
// memory budget, latency-critical loops where cudaMalloc / cudaFree would
// synchronise the device and stall other streams, or host callbacks and
// plug-ins that are not allowed to call the CUDA allocator at all.  For
// them vofl_apply_pair_2d_noalloc runs the same fused kernels with every
// intermediate (the per-model tables, twiddles, spectra, partial sums) in
// one file-scope device array of fixed size, g_noalloc_scratch: 6 MiB,
// enough for grids up to 256 x 256.  Every GPU that loads the library keeps
// that array until the process exits.
// ---------------------------------------------------------------------------
namespace vofl {
namespace {

constexpr int NOALLOC_MAX_AXIS = 256;
constexpr size_t NOALLOC_BYTES = size_t(6) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

struct NoAllocLayout {
  size_t delta, A, B, red, T, Uh, Z, part, P, Lg, twx, twy, step, total;
};

NoAllocLayout noalloc_layout(int nx, int ny, int G) {
  const size_t N = (size_t)nx * ny, ncols = nx / 2 + 1, p = (size_t)round_up((int)ncols, 8);
  NoAllocLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  L.delta = take(sizeof(float) * N);
  L.A = take(sizeof(float) * N);
  L.B = take(sizeof(float) * N);
  L.red = take(sizeof(double) * 1024);
  L.T = take(sizeof(float2) * ny * p);
  L.Uh = take(sizeof(float2) * ncols * ny);
  L.Z = take(sizeof(float2) * ny * p * 2 * G);
  L.part = take(sizeof(float) * 2 * N);
  L.P = take(sizeof(float) * 2 * ncols * ny);
  L.Lg = take(sizeof(float) * ncols * ny);
  L.twx = take(sizeof(float2) * line_twiddle_entries(nx));
  L.twy = take(sizeof(float2) * line_twiddle_entries(ny));
  L.step = take(sizeof(int) * 4);
  L.total = off;
  return L;
}

std::mutex g_noalloc_mu;
constexpr int NOALLOC_MAX_DEVICES = 64;
void* g_noalloc_dev_ptr[NOALLOC_MAX_DEVICES] = {};
bool g_noalloc_attr_set[NOALLOC_MAX_DEVICES] = {};

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (together with the kernels' shared-memory attributes).  In
// host code the array's name is only a host-side stand-in, so kernels are
// always given this looked-up address.
int noalloc_base(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    cudaGetLastError();
    return VOFL_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_dev_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return VOFL_ECUDA;
    }
    g_noalloc_dev_ptr[dev] = p;
  }
  if (!g_noalloc_attr_set[dev]) {
    const int shapes[5][2] = {{64, 64}, {128, 128}, {256, 256}, {256, 128}, {128, 256}};
    for (const auto& sh : shapes) {
      Kernels kk;
      if (pick_kernels(sh[0], sh[1], &kk) && set_smem_attributes(kk)) return VOFL_ECUDA;
    }
    g_noalloc_attr_set[dev] = true;
  }
  *out = static_cast<unsigned char*>(g_noalloc_dev_ptr[dev]);
  return VOFL_OK;
}

}  // namespace
}  // namespace vofl

extern "C" int vofl_apply_pair_2d_noalloc(int nx, int ny, double lx, double ly, int M, const double* gamma_dev,
                                          const float* u_dev, float* out1_dev, float* out2_dev, void* stream) {
  using namespace vofl;
  if (!gamma_dev || !u_dev || (!out1_dev && !out2_dev)) return VOFL_EINVAL;
  if (!(lx > 0) || !(ly > 0) || M < 0 || M > 40) return VOFL_EINVAL;
  if (nx < 2 || ny < 2 || (nx % 2) || (ny % 2)) return VOFL_EINVAL;
  Plan2D p;
  if (nx > NOALLOC_MAX_AXIS || ny > NOALLOC_MAX_AXIS || !pick_kernels(nx, ny, &p.k)) return VOFL_EUNSUPPORTED;
  p.G = std::min(6, M + 1);
  const NoAllocLayout L = noalloc_layout(nx, ny, p.G);
  if (L.total > NOALLOC_BYTES) return VOFL_EUNSUPPORTED;
  unsigned char* base = nullptr;
  int st = noalloc_base(&base);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;

  // per-model part: gamma0 = grid mean of gamma and delta = gamma - gamma0
  // (the A, B fields of the seismic model are written but not used here)
  vofl_ctx m;
  m.ndim = 2;
  m.n[0] = nx;
  m.n[1] = ny;
  m.N = (int64_t)nx * ny;
  m.prec = VOFL_F32;
  m.stream = s;
  m.d_scratch = reinterpret_cast<double*>(base + L.red);
  m.delta = base + L.delta;
  m.A = base + L.A;
  m.B = base + L.B;
  st = model_from_gamma(&m, gamma_dev, nullptr, 1.0, 1.0);
  if (st) return st;
  int e2;
  plan_constants(nx, ny, lx, ly, &e2, &p.ryy);
  p.inv_lambda = std::ldexp(1.0f, -e2);
  p.nx = nx;
  p.ny = ny;
  p.ncols = nx / 2 + 1;
  p.pT = round_up(p.ncols, 8);
  p.pZ = p.pT;
  p.zslot = (long long)ny * p.pZ;
  p.T = reinterpret_cast<float2*>(base + L.T);
  p.Uh = reinterpret_cast<float2*>(base + L.Uh);
  p.Z = reinterpret_cast<float2*>(base + L.Z);
  p.part = reinterpret_cast<float*>(base + L.part);
  p.P = reinterpret_cast<float*>(base + L.P);
  p.Lg = reinterpret_cast<float*>(base + L.Lg);
  p.twx = reinterpret_cast<float2*>(base + L.twx);
  p.twy = reinterpret_cast<float2*>(base + L.twy);
  p.delta = reinterpret_cast<const float*>(m.delta);
  p.step_ctr = reinterpret_cast<int*>(base + L.step);
  p.err = p.step_ctr + 1;
  if (p.make_zmap()) return VOFL_ECUDA;
  if (make_fused2d_tables(nx, ny, lx, ly, m.s01, m.s02, std::ldexp(1.0, e2), (double)p.ryy, p.P,
                          p.Lg, s))
    return VOFL_ECUDA;
  if (make_line_twiddles(nx, p.twx, s) ||
      make_line_twiddles(ny, p.twy, s))
    return VOFL_ECUDA;
  EpiArgs<float> epi{};
  epi.mode = EPI_APPLY;
  epi.out1 = out1_dev;
  epi.out2 = out2_dev;
  epi.src_flat = -1;
  // the step counter and the kernels' error word start at zero on every
  // call: a word left set by an earlier call must not be read as this one's
  if (cudaMemsetAsync(p.step_ctr, 0, 2 * sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return VOFL_ECUDA;
  }
  if (p.forward(s, u_dev, false) || p.inverse(s, M, epi)) {
    cudaGetLastError();
    return VOFL_ECUDA;
  }
  // a bounded device wait that gave up leaves the outputs incomplete and
  // sets the error word: read it back once the call's work is done
  int word = 0;
  if (cudaMemcpyAsync(&word, p.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return VOFL_ECUDA;
  }
  return word ? VOFL_ETIMEDOUT : VOFL_OK;
}
