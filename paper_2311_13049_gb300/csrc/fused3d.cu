// fused3d.cu -- fused FP32 path on a 3D periodic grid nx * ny * nz (x
// fastest) for the operator pair of Eq. (1.1) by the matrix-free scheme of
// Eq. (2.13) of arXiv 2311.13049, and the leap-frog step.
//
// The transform passes reuse the 2D kernels of kernels.cuh:
//   forward  F1 x rows (pairs of rows, two-for-one; 3D Laplacian stencil)
//            F2 y columns of every z plane            (k2d_fwd_cols, batched)
//            F3 z lines of every (k1, k2) column pair  (k2d_fwd_cols on the
//               [z][(k1,k2)] view)
//   per Taylor group g = K-1 .. 0:
//            Iz z lines with the spectral multiplier (k2d_inv_cols on the
//               [(k1,k2)][z] spectrum)
//            Iy y columns of every (term, operator, z) plane (k3d_inv_ycols)
//            Ix x rows of both operators, Horner over the group, epilogue
//               (k2d_inv_rows with rows flattened over (z, y))
// Between passes the data lives in HBM (a 256^3 spectrum is 68 MB per
// operator); the multiplier and the delta^m accumulation are still fused
// into the first and last inverse passes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "kernels.cuh"

namespace vofl {

// Taylor terms per inverse group.  Each group re-reads the z spectrum and
// reads and rewrites both partial sums in HBM, so the fewer groups the
// better; 9 terms make M = 8 one group (Zz + Zy hold 18 transformed planes
// per z: 2.5 GB at 256^3) and M = 16 two.
constexpr int kTerms3D = 9;

namespace {

struct Kernels3 {
  void (*fwd_rows)(const float*, float2*, int, int, int, float, float, const float2*, int*, int, int*);
  void (*fwd_ycols)(const float2*, int, float2*, int, const float2*, long long, long long);
  void (*fwd_zcols)(const float2*, int, float2*, int, const float2*, long long, long long);
  void (*inv_z)(float2*, const float*, const float*, CUtensorMap, int, int, int, float, float, int, int, int,
                const float2*, const float2*, int, int, int);
  void (*inv_y)(const float2*, long long, float2*, long long, int, int, const float2*);
  using InvRows = void (*)(const float2*, long long, int, int, int, int, int, int, int, const float*, float*, float*,
                           EpiArgs<float>, float, const float2*, int*, int);
  InvRows inv_x;        // two operators
  InvRows inv_x_split;  // one operator, terms split over the slots
  size_t sm_frows, sm_fy, sm_fz, sm_iz, sm_iy, sm_ix;
  int lpw_x, lpw_y, lpw_z;
  int wiz;  // warps per CTA of inv_z
};

template <int NX, int NY, int NZ>
Kernels3 kernels3_for() {
  Kernels3 k;
  k.fwd_rows = k2d_fwd_rows<NX, true>;
  k.fwd_ycols = k2d_fwd_cols<NY>;
  k.fwd_zcols = k2d_fwd_cols<NZ>;
  k.inv_z = k2d_inv_cols<NZ>;
  k.inv_y = k3d_inv_ycols<NY>;
  k.inv_x = k2d_inv_rows<NX, false>;
  k.inv_x_split = k2d_inv_rows<NX, true>;
  k.sm_frows = frows_smem<NX, true>();
  k.sm_fy = exch_smem<NY, W_FCOLS>();
  k.sm_fz = exch_smem<NZ, W_FCOLS>();
  k.sm_iz = inv_cols_smem<NZ>();
  k.sm_iy = exch_smem<NY, W_YCOLS>();
  k.sm_ix = inv_rows_smem<NX>();
  k.lpw_x = LineFFT<NX>::LPW;
  k.lpw_y = LineFFT<NY>::LPW;
  k.lpw_z = LineFFT<NZ>::LPW;
  k.wiz = icols_warps<NZ>();
  return k;
}

bool pick_kernels3(int nx, int ny, int nz, Kernels3* k) {
#define VOFL_CASE3(X, Y, Z)          \
  if (nx == X && ny == Y && nz == Z) { \
    *k = kernels3_for<X, Y, Z>();    \
    return true;                     \
  }
  VOFL_CASE3(64, 64, 64)
  VOFL_CASE3(128, 128, 128)
  VOFL_CASE3(256, 256, 256)
  VOFL_CASE3(128, 64, 256)
#undef VOFL_CASE3
  return false;
}

int set_smem3(const Kernels3& k) {
  if (set_kernel_smem(k.fwd_rows, k.sm_frows) ||
      set_kernel_smem(k.fwd_ycols, k.sm_fy) ||
      set_kernel_smem(k.fwd_zcols, k.sm_fz) ||
      set_kernel_smem(k.inv_z, k.sm_iz) ||
      set_kernel_smem(k.inv_y, k.sm_iy) ||
      set_kernel_smem(k.inv_x, k.sm_ix) || set_kernel_smem(k.inv_x_split, k.sm_ix)) {
    cudaGetLastError();
    return VOFL_ECUDA;
  }
  return VOFL_OK;
}

// |mu|^{2 s0}/(N lambda), scale2 * |mu|^{2 s02}/(N lambda) and ln|mu|^2 on
// the [(k1, k2)][k3] layout (k3 fastest), lambda = the symbol of the
// transformed discrete Laplacian.  Double precision.
__global__ void k_tables_fused3d(int nx, int ny, int nz, double lx, double ly, double lz, double s01, double s02,
                                 double scale2, double ryy, double rzz, float* __restrict__ P,
                                 float* __restrict__ Lg) {
  const long long total = (long long)(nx / 2 + 1) * ny * nz;
  const double invN = 1.0 / ((double)nx * ny * nz);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int k3 = (int)(i % nz);
    const int k2 = (int)((i / nz) % ny);
    const int k1 = (int)(i / ((long long)nz * ny));
    const int k2s = k2 < ny / 2 ? k2 : k2 - ny;
    const int k3s = k3 < nz / 2 ? k3 : k3 - nz;
    const double m1 = 2.0 * M_PI * k1 / lx, m2 = 2.0 * M_PI * k2s / ly, m3 = 2.0 * M_PI * k3s / lz;
    const double mu2 = m1 * m1 + m2 * m2 + m3 * m3;
    if (mu2 == 0.0) {
      P[i] = 0.f;
      P[total + i] = 0.f;
      Lg[i] = 0.f;
    } else {
      const double s1 = sinpi((double)k1 / nx), s2 = sinpi((double)k2 / ny), s3 = sinpi((double)k3 / nz);
      const double lam = -4.0 * (s1 * s1 + ryy * s2 * s2 + rzz * s3 * s3);
      const double L = log(mu2);
      P[i] = (float)(exp(s01 * L) * invN / lam);
      P[total + i] = (float)(exp(s02 * L) * invN * scale2 / lam);
      Lg[i] = (float)L;
    }
  }
}

struct Fused3D : Engine {
  Kernels3 k{};
  int nx = 0, ny = 0, nz = 0, H = 0, c2 = 0, c3 = 0;  // c2 = H+1 columns per plane, c3 = (H+1)*ny z-columns
  int pT = 0, pZ = 0, p3 = 0, G = kTerms3D;
  float2 *T = nullptr, *U2 = nullptr, *U3 = nullptr, *Zz = nullptr, *Zy = nullptr;
  float *part = nullptr, *P = nullptr, *Lg = nullptr;
  float2 *twx = nullptr, *twy = nullptr, *twz = nullptr;
  float ryy = 1.f, rzz = 1.f, inv_lambda = 1.f;
  double lambda = 1.0;
  size_t nbytes = 0;
  CUtensorMap zmap{};  // Zz as [2 G nz rows][p3] for the z-inverse kernel's tile stores

  ~Fused3D() override {
    for (void* q : {(void*)T, (void*)U2, (void*)U3, (void*)Zz, (void*)Zy, (void*)part, (void*)P, (void*)Lg,
                    (void*)twx, (void*)twy, (void*)twz})
      dev_free(q);
  }
  size_t bytes() const override { return nbytes; }

  int alloc(vofl_ctx* c, void** ptr, size_t b) {
    cudaError_t e = dev_malloc(ptr, b);
    if (e != cudaSuccess) return cuda_err(c, e, "cudaMalloc (fused 3D scratch)");
    nbytes += b;
    return VOFL_OK;
  }

  int init(vofl_ctx* c) {
    nx = (int)c->n[0];
    ny = (int)c->n[1];
    nz = (int)c->n[2];
    if (!pick_kernels3(nx, ny, nz, &k)) return set_err(c, VOFL_EUNSUPPORTED, "fused 3D path: grid size not built");
    H = nx / 2;
    c2 = H + 1;
    c3 = c2 * ny;
    pT = round_up(c2, 8);
    pZ = pT;
    p3 = round_up(c3, 8);
    G = kTerms3D;
    const size_t N = (size_t)nx * ny * nz;
    int st;
    if ((st = alloc(c, (void**)&T, sizeof(float2) * (size_t)nz * ny * pT))) return st;
    if ((st = alloc(c, (void**)&U2, sizeof(float2) * (size_t)nz * c3))) return st;
    if ((st = alloc(c, (void**)&U3, sizeof(float2) * (size_t)c3 * nz))) return st;
    if ((st = alloc(c, (void**)&Zz, sizeof(float2) * (size_t)2 * G * nz * p3))) return st;
    if ((st = alloc(c, (void**)&Zy, sizeof(float2) * (size_t)2 * G * nz * ny * pZ))) return st;
    if ((st = alloc(c, (void**)&part, sizeof(float) * 2 * N))) return st;
    if ((st = alloc(c, (void**)&P, sizeof(float) * 2 * (size_t)c3 * nz))) return st;
    if ((st = alloc(c, (void**)&Lg, sizeof(float) * (size_t)c3 * nz))) return st;
    if ((st = alloc(c, (void**)&twx, sizeof(float2) * line_twiddle_entries(nx)))) return st;
    if ((st = alloc(c, (void**)&twy, sizeof(float2) * line_twiddle_entries(ny)))) return st;
    if ((st = alloc(c, (void**)&twz, sizeof(float2) * line_twiddle_entries(nz)))) return st;
    if (set_smem3(k)) return set_err(c, VOFL_ECUDA, "shared-memory attributes of the fused 3D kernels");
    if (make_line_twiddles(nx, twx, c->stream) ||
        make_line_twiddles(ny, twy, c->stream) ||
        make_line_twiddles(nz, twz, c->stream))
      return cuda_err(c, cudaGetLastError(), "twiddles");
    if (make_tile_map(&zmap, Zz, c3, 2LL * G * nz, p3, k.wiz * k.lpw_z, std::min(nz, 256)))
      return set_err(c, VOFL_ECUDA, "tensor map of the Zz buffer");
    return VOFL_OK;
  }

  int set_model(vofl_ctx* c) override {
    const double lx = c->hi[0] - c->lo[0], ly = c->hi[1] - c->lo[1], lz = c->hi[2] - c->lo[2];
    const double mx = M_PI * nx / lx, my = M_PI * ny / ly, mz = M_PI * nz / lz;
    const int e2 = (int)std::lround(0.5 * std::log2(std::max(std::sqrt(mx * mx + my * my + mz * mz), 1.0)));
    lambda = std::ldexp(1.0, e2);
    inv_lambda = std::ldexp(1.0f, -e2);
    const double hx = lx / nx, hy = ly / ny, hz = lz / nz;
    ryy = (float)((hx * hx) / (hy * hy));
    rzz = (float)((hx * hx) / (hz * hz));
    const long long total = (long long)c3 * nz;
    k_tables_fused3d<<<(int)std::min<long long>(4096, (total + 255) / 256), 256, 0, c->stream>>>(
        nx, ny, nz, lx, ly, lz, c->s01, c->s02, lambda, (double)ryy, (double)rzz, P, Lg);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return set_err(c, VOFL_ECUDA, "fused 3D tables");
    return VOFL_OK;
  }

  // one_op: a model with one operator (its terms fill both slots)
  int groups(int M, bool one_op) const { return (term_split(M, one_op).slots + G - 1) / G; }
  uint64_t kernels_per_step(const vofl_ctx* c) const override {
    return 3 + 3 * (uint64_t)groups(c->M, c->general);
  }

  cudaError_t forward(vofl_ctx* c, const float* u, bool inc_step) {
    cudaStream_t s = c->stream;
    const int rpc = W_FROWS * k.lpw_x;
    const int pairs = (ny / 2) * nz;
    cudaError_t e = launch_pdl(k.fwd_rows, dim3((pairs + rpc - 1) / rpc), dim3(W_FROWS * 32), k.sm_frows, s, u, T,
                               ny, nz, pT, ryy, rzz, (const float2*)twx, c->d_step, inc_step ? 1 : 0,
                               c->d_step + 1);
    if (e) return e;
    const int cy = W_FCOLS * k.lpw_y;
    e = launch_pdl(k.fwd_ycols, dim3((c2 + cy - 1) / cy, nz), dim3(W_FCOLS * 32), k.sm_fy, s, (const float2*)T, pT, U2,
                   c2, (const float2*)twy, (long long)ny * pT, (long long)c3);
    if (e) return e;
    const int cz = W_FCOLS * k.lpw_z;
    return launch_pdl(k.fwd_zcols, dim3((c3 + cz - 1) / cz, 1), dim3(W_FCOLS * 32), k.sm_fz, s, (const float2*)U2, c3,
                      U3, c3, (const float2*)twz, 0LL, 0LL);
  }

  cudaError_t inverse(vofl_ctx* c, const EpiArgs<float>& epi) {
    cudaStream_t s = c->stream;
    const TermSplit ts = term_split(c->M, c->general);
    const int K = groups(c->M, c->general);
    const long long zslot_y = (long long)nz * ny * pZ;
    const int rows = ny * nz;
    for (int gi = K - 1; gi >= 0; --gi) {
      const int m_lo = gi * G, m_hi = std::min(ts.slots, m_lo + G);
      const float f0 = inv_factorial(m_lo), f1 = ts.split_k ? inv_factorial(m_lo + ts.split_k) : f0;
      const int cz = k.wiz * k.lpw_z;
      cudaError_t e = launch_pdl(k.inv_z, dim3((c3 + cz - 1) / cz, 2), dim3(k.wiz * 32), k.sm_iz, s, U3,
                                 (const float*)P, (const float*)Lg, zmap, c3, m_lo, m_hi, f0, f1, ts.split_k, 1, 0,
                                 (const float2*)twz, (const float2*)nullptr, 0, 0, 0);
      if (e) return e;
      const int cy = W_YCOLS * k.lpw_y;
      e = launch_pdl(k.inv_y, dim3((c2 + cy - 1) / cy, 2 * (m_hi - m_lo) * nz), dim3(W_YCOLS * 32), k.sm_iy, s,
                     (const float2*)Zz, (long long)p3, Zy, (long long)ny * pZ, pZ, c2, (const float2*)twy);
      if (e) return e;
      EpiArgs<float> ep = epi;
      if (gi > 0) ep.mode = EPI_PARTIAL;
      const int rpc = W_IROWS * k.lpw_x;
      e = launch_pdl(ts.split_k ? k.inv_x_split : k.inv_x, dim3((rows + rpc - 1) / rpc), dim3(W_IROWS * 32), k.sm_ix,
                     s, (const float2*)Zy, zslot_y,
                     pZ, rows, m_lo, m_hi, gi == K - 1 ? 1 : 0, ts.k2, ts.split_k, (const float*)c->delta, part,
                     part + (size_t)nx * ny * nz, ep, inv_lambda, (const float2*)twx, c->d_step + 1, 1);
      if (e) return e;
    }
    return cudaSuccess;
  }

  int apply_pair(vofl_ctx* c, const void* u, void* o1, void* o2) override {
    EpiArgs<float> e{};
    e.mode = EPI_APPLY;
    e.out1 = (float*)o1;
    e.out2 = (float*)o2;
    e.src_flat = -1;
    cudaError_t err = forward(c, (const float*)u, false);
    if (!err) err = inverse(c, e);
    if (err) return cuda_err(c, err, "fused 3D launch");
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
    for (int i = 0; i < 3; ++i) hd *= (c->hi[i] - c->lo[i]) / (double)c->n[i];
    e.src_scale = c->dt * c->dt / hd;
    epi_model(c, &e);
    cudaError_t err = forward(c, (const float*)c->u[c->cur], count_step);
    if (!err) err = inverse(c, e);
    if (err) return cuda_err(c, err, "fused 3D launch");
    return VOFL_OK;
  }
};

}  // namespace

bool fused3d_supported(int ndim, const int64_t* n, int prec) {
  Kernels3 k;
  return ndim == 3 && prec == VOFL_F32 && pick_kernels3((int)n[0], (int)n[1], (int)n[2], &k);
}

size_t fused3d_footprint(const int64_t* n, int M) {
  const size_t nx = n[0], ny = n[1], nz = n[2], c2 = nx / 2 + 1, c3 = c2 * ny;
  const size_t pT = (c2 + 7) / 8 * 8, p3 = (c3 + 7) / 8 * 8, G = kTerms3D;
  return sizeof(float2) * (nz * ny * pT + 2 * nz * c3 + 2 * G * nz * p3 + 2 * G * nz * ny * pT + nx + ny + nz) +
         sizeof(float) * (2 * nx * ny * nz + 3 * c3 * nz);
}

Engine* make_fused3d(vofl_ctx* c, int* status) {
  Fused3D* e = new Fused3D();
  *status = e->init(c);
  if (*status != VOFL_OK) {
    delete e;
    return nullptr;
  }
  return e;
}

}  // namespace vofl
