// internal.h -- context state and engine interface of the vofl library.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "vofl.h"

namespace vofl {

// NVTX range over one C-ABI call (nsys, ncu --nvtx); without an attached
// tool a push/pop pair costs a function-pointer test
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

extern std::atomic<uint64_t> g_kernel_launches;

// Every device allocation of the library goes through dev_malloc, so that
// a test can make the k-th one fail as if the device were out of memory
// (vofl_debug_fail_alloc) and check that each caller frees what it holds
// and reports VOFL_ENOMEM.
cudaError_t dev_malloc_bytes(void** p, size_t bytes);
long long debug_fail_alloc(long long k);  // set the countdown, return the old one
// Frees what dev_malloc gave (cudaFree, or, in the canary mode, the padded
// allocation after checking its pads).
cudaError_t dev_free(void* p);
// Canary mode (VOFL_DEBUG_CANARY=1 in the environment at the first
// allocation): buffers found with changed pads, -1 when the mode is off.
long long debug_canaries(long long* live, int poke);
template <typename T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc_bytes(reinterpret_cast<void**>(p), bytes);
}
inline void count_launch(uint64_t n = 1) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }

struct Engine;


// Epilogue of the last inverse pass: what to do with L1 u, L2 u at a point.
// EPI_KICK: the kick of the time splitting (Sec. 3.3), v += dt (A L1 + f(u))
// with v = u_other, u = u_cur (L2 unused, l2p untouched).
enum EpiMode { EPI_PARTIAL = 0, EPI_APPLY = 1, EPI_STEP = 2, EPI_START = 3, EPI_KICK = 4 };

template <typename T>
struct EpiArgs {
  int mode;
  T* out1;            // EPI_APPLY: L1 u (may be null)
  T* out2;            // EPI_APPLY: L2 u (may be null)
  const T* u_cur;     // u^n
  T* u_other;         // in: u^{n-1} (STEP) or psi (START); out: u^{n+1}
  T* l2p;             // in: L2 u^{n-1} (STEP) or L2 psi (START); out: L2 u^n
  const T* A;         // c^2 eta
  const T* B;         // c^2 tau
  T dt1, dt2;         // dt, dt^2
  long long src_flat; // flat index of the source node, -1 = none
  const double* src;  // samples r_n
  long long nsrc;
  const int* step;    // device step counter n
  double src_scale;   // dt^2 / h^d
  int nonlin;         // general model with a source term f(u) = f1 u + f3 u^3
  T f1, f3;
  int dpow;           // one-operator sums of terms dpow..M: L1 = delta^dpow (slot sums)
};

// Pointwise update of Eq. (3.4) extended to Eq. (1.1) (see vofl.h).
template <typename T>
__device__ __forceinline__ void epilogue_point(const EpiArgs<T>& e, long long idx, T L1, T L2) {
  if (e.mode == EPI_APPLY) {
    if (e.out1) e.out1[idx] = L1;
    if (e.out2) e.out2[idx] = L2;
    return;
  }
  const T un = e.u_cur[idx];
  const T other = e.u_other[idx];
  if (e.mode == EPI_KICK) {
    T f = e.A[idx] * L1;
    if (e.nonlin) f += e.f1 * un + e.f3 * un * un * un;
    e.u_other[idx] = other + e.dt1 * f;
    return;
  }
  const T l2o = e.l2p[idx];
  T unew;
  if (e.mode == EPI_STEP) {
    // 2u^n - u^{n-1} + dt^2 A L1 u^n + dt B (L2 u^n - L2 u^{n-1})
    unew = (T(2) * un - other) + e.dt2 * e.A[idx] * L1 + e.dt1 * e.B[idx] * (L2 - l2o);
    if (e.nonlin) unew += e.dt2 * (e.f1 * un + e.f3 * un * un * un);
    if (idx == e.src_flat) {
      const int n = *e.step;
      if (n < e.nsrc) unew += T(e.src_scale * e.src[n]);
    }
  } else {  // EPI_START: u^0 + dt psi + dt^2/2 (A L1 u^0 + B L2 psi + f_0)
    unew = un + e.dt1 * other + T(0.5) * e.dt2 * (e.A[idx] * L1 + e.B[idx] * l2o);
    if (e.nonlin) unew += T(0.5) * e.dt2 * (e.f1 * un + e.f3 * un * un * un);
    if (idx == e.src_flat && e.nsrc > 0) unew += T(0.5 * e.src_scale * e.src[0]);
  }
  e.u_other[idx] = unew;
  e.l2p[idx] = L2;
}

// One simulation of a batch, as the batched 2D kernels see it (device copy):
// every buffer belongs to the simulation's own context.
struct BatchSim {
  CUtensorMap zmap;     // Z as [2 G ny rows][pZ] for the column kernel's tile stores
  EpiArgs<float> epi;   // state buffers, coefficients, dt, source, step counter, mode
  const float* delta;   // gamma - gamma0
  float2* T;            // row half spectra
  float2* Uh;           // column spectra
  float2* Z;            // one group of per-term transforms
  float* part;          // two partial-sum fields
  const float* P;       // multipliers of both operators
  const float* Lg;      // ln |mu|^2
  const float2* twx;    // line twiddles along x
  const float2* twy;    // ... along y
  const float2* twxw;   // wide line twiddles along x (512 or 1024 points, else null)
  const float2* twyw;   // ... along y
  int* err;             // device error word
  float ryy;            // (h_x / h_y)^2
  float inv_lambda;     // 1 / (operator-2 balance factor)
  long long zslot;      // Z slot stride (float2)
  int pT, pZ;           // row pitches of T and Z (float2)
  int M;                // top Taylor power
  int inc_step;         // 1: advance the step counter in this step
};

}  // namespace vofl

struct vofl_ctx {
  int ndim = 0;
  int64_t n[3] = {1, 1, 1};  // x, y, z
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  int64_t N = 0;             // total points
  int prec = VOFL_F32;
  int impl = VOFL_IMPL_FUSED;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  int M = 8;

  // model (after set_q / set_gamma / set_order)
  bool model_set = false;
  bool general = false;   // general model u_tt = -kappa (-Delta)^{s(x)} u + f(u)
  double gamma0 = 0;      // seismic: grid mean of gamma
  double s01 = 1, s02 = 0.5;  // expansion orders of the two operators (Eq. (2.13))
  double kappa = 1, f1 = 0, f3 = 0;
  int scheme = VOFL_SCHEME_LFFP;  // time stepping of vofl_step
  double cn_tol = 0;              // Crank-Nicolson: relative residual of each step's system (set by precision at creation)
  int cn_maxit = 5000;            // ... CG iterations per linear solve
  int64_t cn_iters = 0, cn_solves = 0;  // ... totals since the state was set
  void* delta = nullptr;  // gamma - gamma0        (prec)
  void* A = nullptr;      // c^2 eta               (prec)
  void* B = nullptr;      // c^2 tau               (prec)
  double* d_gamma = nullptr;  // gamma (double), kept for re-derivation
  double* d_scratch = nullptr;  // reduction partials

  // time stepping
  void* u[2] = {nullptr, nullptr};
  int cur = 0;
  void* l2p = nullptr;
  bool state_set = false;
  bool psi_nonzero = false;
  int64_t steps = 0;
  double dt = 0;
  int* d_step = nullptr;

  // source
  long long src_flat = -1;
  double* d_src = nullptr;
  int64_t nsrc = 0;
  int64_t src_cap = 0;

  vofl::Engine* eng = nullptr;
  struct vofl_batch* batch = nullptr;  // set while a batch steps this context

  // captured one-step graphs (index = cur buffer at the start of the step)
  cudaGraphExec_t step_graph[2] = {nullptr, nullptr};
  uint64_t step_graph_kernels = 0;
  bool graphs_ok = true;
  // what the captured graphs bake in besides the context's fixed buffers
  struct GraphKey {
    double dt = -1;
    int M = -1;
    long long src_flat = -2;
    const double* d_src = nullptr;
    int64_t nsrc = -1;
    double f1 = 0, f3 = 0, kappa = 0;
    int scheme = 0;
    bool operator==(const GraphKey& o) const {
      return dt == o.dt && M == o.M && src_flat == o.src_flat && d_src == o.d_src && nsrc == o.nsrc && f1 == o.f1 &&
             f3 == o.f3 && kappa == o.kappa && scheme == o.scheme;
    }
  } graph_key;

  std::string err;
};

namespace vofl {

struct Engine {
  virtual ~Engine() {}
  // (re)build spectral tables after the model changed (gamma0 known)
  virtual int set_model(vofl_ctx* c) = 0;
  // L1 u -> o1, L2 u -> o2 (either may be null)
  virtual int apply_pair(vofl_ctx* c, const void* u, void* o1, void* o2) = 0;
  // one step with the given epilogue (mode EPI_STEP or EPI_START); state
  // buffers are taken from the context (cur / other / l2p)
  virtual int step(vofl_ctx* c, int mode, bool count_step) = 0;
  // number of kernels launched by one step(mode = EPI_STEP)
  virtual uint64_t kernels_per_step(const vofl_ctx* c) const = 0;
  virtual int profile(vofl_ctx* c, int reps, std::string& names, double* ms, double* units, int cap) {
    (void)c; (void)reps; (void)names; (void)ms; (void)units; (void)cap;
    return 0;
  }
  virtual size_t bytes() const = 0;
  // transform schedule (fused 2D only)
  virtual int set_schedule(vofl_ctx* c, const vofl_schedule* s) {
    (void)c;
    (void)s;
    return VOFL_EUNSUPPORTED;
  }
  virtual int get_schedule(const vofl_ctx* c, vofl_schedule* s) const {
    (void)c;
    (void)s;
    return VOFL_EUNSUPPORTED;
  }
  // Fill the engine-owned part of a batch descriptor (buffers, tables,
  // pitches); false if this engine cannot take part in a 2D batch.
  virtual bool batch_desc(const vofl_ctx* c, BatchSim* d) const {
    (void)c;
    (void)d;
    return false;
  }
  // engines that advance many steps in one launch (the first step with
  // first_mode: EPI_START or EPI_STEP); the context's cur/steps are updated
  // by the caller
  virtual bool can_run() const { return false; }
  // engines with the second-order time splitting (Sec. 3.3) of the general
  // model: one step, u = u[cur] and v = u[1 - cur] updated in place
  virtual bool can_split() const { return false; }
  virtual int step_split(vofl_ctx* c) {
    (void)c;
    return VOFL_EUNSUPPORTED;
  }
  // engines whose step_split is the kick followed by the flow over the whole
  // step (consecutive half-step flows merged): a run of n steps is then
  // split_flow(+dt/2), n x step_split, split_flow(-dt/2)
  virtual bool split_merged() const { return false; }
  virtual int split_flow(vofl_ctx* c, double t) {
    (void)c;
    (void)t;
    return VOFL_EUNSUPPORTED;
  }
  // after a device wait gave up (the error word was set): put back the
  // device-side state of the engine's waits (grid-barrier counters), so
  // later launches start from a clean barrier; called with the stream idle
  virtual void reset_waits(vofl_ctx* c) { (void)c; }
  // size M-dependent scratch before stepping or applying (outside any graph
  // capture: allocations and plans are not stream operations)
  virtual int prepare(vofl_ctx* c) {
    (void)c;
    return VOFL_OK;
  }
  // engines with the Crank-Nicolson scheme (Sec. 3.1) of the general model:
  // one step n >= 1, u^{n+1} written to u[1 - cur]
  virtual bool can_cn() const { return false; }
  virtual int step_cn(vofl_ctx* c) {
    (void)c;
    return VOFL_EUNSUPPORTED;
  }
  virtual int run(vofl_ctx* c, int64_t nsteps, int first_mode) {
    (void)c;
    (void)nsteps;
    (void)first_mode;
    return VOFL_EUNSUPPORTED;
  }
};

Engine* make_fused2d(vofl_ctx* c, int* status);
Engine* make_fused1d(vofl_ctx* c, int* status);
bool fused1d_supported(int ndim, const int64_t* n, int prec);
Engine* make_fused3d(vofl_ctx* c, int* status);
bool fused3d_supported(int ndim, const int64_t* n, int prec);
size_t fused3d_footprint(const int64_t* n, int M);
Engine* make_plain(vofl_ctx* c, int* status);
size_t fused2d_footprint(const int64_t* n, int M);
size_t plain_footprint(int ndim, const int64_t* n, int prec, int M);
bool fused2d_supported(int ndim, const int64_t* n, int prec);

// run set-up shared by vofl_step and batches (capi.cu)
int prepare_run(vofl_ctx* c, double dt);
// take a context out of the batch that steps it (waits for the batch's
// queued work); used when the context is destroyed (batch2d.cu)
void batch_detach(vofl_ctx* c);

// model precompute (model.cu)
int model_from_gamma(vofl_ctx* c, const double* d_gamma, const double* d_c0field, double c0, double omega0);
int model_gamma_from_q(vofl_ctx* c, const double* d_q, double* d_gamma);
int model_from_order(vofl_ctx* c, const double* d_s, double kappa);
// the general-model part of the epilogue arguments of a context
template <typename T>
void epi_model(const vofl_ctx* c, EpiArgs<T>* e) {
  e->nonlin = c->general && (c->f1 != 0.0 || c->f3 != 0.0);
  e->f1 = T(c->f1);
  e->f3 = T(c->f3);
}
int model_suggest_dt(vofl_ctx* c, double courant, double* dt);
// rel-L2 / pointwise diagnostics of two fields of the context's grid (model.cu)
int model_rel_l2(vofl_ctx* c, const void* x, int x_prec, const void* y, int y_prec, double* out);
int model_suggest_M(vofl_ctx* c, double tol, int M_max, int* M);

// twiddles / tables (model.cu)
// Twiddle layout of the warp line FFT of length N (fft_warp.cuh): the last
// stage has radix R over NB butterflies (table of NB * R = N entries), and
// N = 768 adds a middle stage whose NM = 192 twiddles follow.
inline void line_twiddle_layout(int N, int* NB, int* R, int* NM) {
  if (N == 768) {
    *NB = 192;
    *R = 4;
    *NM = 192;
  } else {
    const int e = N >= 512 ? 32 : (N >= 128 ? 16 : 8);
    *NB = e;
    *R = N / e;
    *NM = 0;
  }
}
inline int line_twiddle_entries(int N) {
  int nb, r, nm;
  line_twiddle_layout(N, &nb, &r, &nm);
  return nb * r + nm;
}
int make_line_twiddles(int N, float2* d_tw, cudaStream_t s);
// The wide line transform of N = 512 or 1024 points (fft_wide.cuh): its
// last stage's N twiddles w_N^{r j}, then the 16 (N/64) of the middle stage.
inline bool wide_line(int N) { return N == 512 || N == 1024; }
// SMs of the current device (0 if it cannot be read)
inline int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return sms;
}
inline int wide_twiddle_entries(int N) { return N + (N / 64) * 16; }
int make_wide_twiddles(int N, float2* d_tw, cudaStream_t s);
// Tensor map of a [rows][pitch] array of 8-byte elements (ncols valid per
// row) for 2D tiled TMA copies of boxes of box_cols x box_rows (model.cu).
int make_tile_map(CUtensorMap* map, const void* base, int ncols, long long rows, int pitch, int box_cols,
                  int box_rows);
int make_fused2d_tables(int nx, int ny, double lx, double ly, double s01, double s02, double scale2, double ryy,
                        float* P, float* Lg, cudaStream_t s);
// sqrt(kappa) |mu_k|^{s0} on the fused 2D column-spectrum layout [H+1][ny]
// (the time splitting's exact flow, Sec. 3.3)
int make_fused2d_omega(int nx, int ny, double lx, double ly, double s0, double kappa, float* W, cudaStream_t s);
template <typename T>
int make_plain_tables(int ndim, const int64_t* n, const double* lo, const double* hi, double s01, double s02,
                      T* P1, T* P2, T* Lg, cudaStream_t s);

inline int set_err(vofl_ctx* c, int code, const char* msg) {
  if (c) c->err = msg;
  return code;
}
int cuda_err(vofl_ctx* c, cudaError_t e, const char* where);

}  // namespace vofl

#define VOFL_CUDA(ctx, call)                                    \
  do {                                                          \
    cudaError_t _e = (call);                                    \
    if (_e != cudaSuccess) return ::vofl::cuda_err(ctx, _e, #call); \
  } while (0)
