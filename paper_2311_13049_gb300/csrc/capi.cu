// capi.cu -- the C ABI declared in include/vofl.h: context lifecycle,
// argument checks, host/device copies, the leap-frog run state machine and
// CUDA-graph replay of steps.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>

#include "internal.h"

using namespace vofl;

namespace {

const char* kVersion = "vofl 0.1.0 (sm_103a)";

size_t elem_size(const vofl_ctx* c) { return c->prec == VOFL_F64 ? 8 : 4; }

void drop_graphs(vofl_ctx* c) {
  for (auto& g : c->step_graph) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

void reset_run(vofl_ctx* c) {
  c->steps = 0;
  c->cur = 0;
  c->cn_iters = 0;
  c->cn_solves = 0;
}

vofl_ctx::GraphKey current_key(const vofl_ctx* c) {
  vofl_ctx::GraphKey k;
  k.dt = c->dt;
  k.M = c->M;
  k.src_flat = c->nsrc > 0 ? c->src_flat : -1;
  k.d_src = c->d_src;
  k.nsrc = c->nsrc;
  k.f1 = c->general ? c->f1 : 0.0;
  k.f3 = c->general ? c->f3 : 0.0;
  k.kappa = c->general ? c->kappa : 0.0;
  k.scheme = c->scheme;
  return k;
}

int check_ctx(vofl_ctx* c) {
  if (!c) return VOFL_EINVAL;
  if (c->batch) return set_err(c, VOFL_ESTATE, "the context is stepped by a batch; remove it from the batch first");
  return VOFL_OK;
}

}  // namespace

// Checks before stepping and, before the first step, the run set-up: the
// step counter starts at 0 and L2 psi (Taylor start) goes into l2p.
int vofl::prepare_run(vofl_ctx* c, double dt) {
  if (!c->model_set || !c->state_set) return set_err(c, VOFL_ESTATE, "set the model and the state first");
  if (!(dt > 0) || !std::isfinite(dt)) return set_err(c, VOFL_EINVAL, "bad dt");
  if (c->steps > 0 && dt != c->dt) return set_err(c, VOFL_EINVAL, "dt must stay fixed during a run");
  if (int st = c->eng->prepare(c)) return st;
  if (c->steps == 0) {
    c->dt = dt;
    VOFL_CUDA(c, cudaMemsetAsync(c->d_step, 0, sizeof(int), c->stream));
    if (c->psi_nonzero) {
      int st = c->eng->apply_pair(c, c->u[1], nullptr, c->l2p);
      if (st) return st;
    }
  }
  return VOFL_OK;
}

namespace {

int upload(vofl_ctx* c, void* dst, const void* src, size_t bytes, int on_device) {
  VOFL_CUDA(c, cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                               c->stream));
  if (!on_device) VOFL_CUDA(c, cudaStreamSynchronize(c->stream));  // host buffer may be pageable/transient
  return VOFL_OK;
}

// Capture one STEP of the engine into a graph for the current `cur`.
int capture_step(vofl_ctx* c) {
  const uint64_t before = g_kernel_launches.load();
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return VOFL_EUNSUPPORTED;
  }
  int st = c->eng->step(c, EPI_STEP, true);
  e = cudaStreamEndCapture(c->stream, &g);
  g_kernel_launches.store(before);  // captured launches are counted when replayed
  if (st != VOFL_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return VOFL_EUNSUPPORTED;
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return VOFL_EUNSUPPORTED;
  }
  c->step_graph[c->cur] = ex;
  c->step_graph_kernels = c->eng->kernels_per_step(c);
  return VOFL_OK;
}

// Capture one step of the time splitting into the graph slot of `cur`.
int capture_split(vofl_ctx* c) {
  const uint64_t before = g_kernel_launches.load();
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return VOFL_EUNSUPPORTED;
  }
  int st = c->eng->step_split(c);
  e = cudaStreamEndCapture(c->stream, &g);
  const uint64_t n = g_kernel_launches.load() - before;
  g_kernel_launches.store(before);
  if (st != VOFL_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return VOFL_EUNSUPPORTED;
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return VOFL_EUNSUPPORTED;
  }
  c->step_graph[c->cur] = ex;
  c->step_graph_kernels = n;
  return VOFL_OK;
}

// one step of the time splitting (u, v in place; `cur` does not change)
int split_step(vofl_ctx* c) {
  const vofl_ctx::GraphKey key = current_key(c);
  if (!(key == c->graph_key)) {
    drop_graphs(c);
    c->graph_key = key;
  }
  if (c->graphs_ok && !c->step_graph[c->cur]) {
    if (capture_split(c) != VOFL_OK) c->graphs_ok = false;
  }
  if (c->graphs_ok && c->step_graph[c->cur]) {
    VOFL_CUDA(c, cudaGraphLaunch(c->step_graph[c->cur], c->stream));
    count_launch(c->step_graph_kernels);
  } else {
    int st = c->eng->step_split(c);
    if (st) return st;
  }
  c->steps += 1;
  return VOFL_OK;
}

int one_step(vofl_ctx* c) {
  const vofl_ctx::GraphKey key = current_key(c);
  if (!(key == c->graph_key)) {
    drop_graphs(c);
    c->graph_key = key;
  }
  if (c->graphs_ok && !c->step_graph[c->cur]) {
    if (capture_step(c) != VOFL_OK) c->graphs_ok = false;
  }
  if (c->graphs_ok && c->step_graph[c->cur]) {
    VOFL_CUDA(c, cudaGraphLaunch(c->step_graph[c->cur], c->stream));
    count_launch(c->step_graph_kernels);
  } else {
    int st = c->eng->step(c, EPI_STEP, true);
    if (st) return st;
  }
  c->cur ^= 1;
  c->steps += 1;
  return VOFL_OK;
}

}  // namespace

extern "C" {

const char* vofl_version(void) { return kVersion; }

uint64_t vofl_kernel_launches(void) { return g_kernel_launches.load(); }

size_t vofl_footprint_bytes(int ndim, const int64_t* n, int prec, int impl, int M) {
  if (ndim < 1 || ndim > 3 || !n) return 0;
  long long N = 1;
  for (int i = 0; i < ndim; ++i) N *= n[i];
  const size_t r = prec == VOFL_F64 ? 8 : 4;
  size_t b = r * (size_t)N * 6 + sizeof(double) * (size_t)N + 8192;  // delta A B u0 u1 l2p, gamma
  if (impl == VOFL_IMPL_FUSED && fused2d_supported(ndim, n, prec))
    b += fused2d_footprint(n, M);
  else if (impl == VOFL_IMPL_FUSED && fused3d_supported(ndim, n, prec))
    b += fused3d_footprint(n, M);
  else if (impl == VOFL_IMPL_FUSED && fused1d_supported(ndim, n, prec))
    b += (size_t)N * (prec == VOFL_F64 ? 8 : 4) * (4 + 2 * (size_t)(M + 1));  // tables, twiddles, term tables
  else
    b += plain_footprint(ndim, n, prec, M);
  return b;
}

int vofl_create(vofl_ctx** out, int ndim, const int64_t* n, const double* lo, const double* hi, int prec, int impl,
                void* stream) {
  if (!out) return VOFL_EINVAL;
  *out = nullptr;
  if (ndim < 1 || ndim > 3 || !n || !lo || !hi) return VOFL_EINVAL;
  if (prec != VOFL_F32 && prec != VOFL_F64) return VOFL_EINVAL;
  if (impl != VOFL_IMPL_FUSED && impl != VOFL_IMPL_PLAIN) return VOFL_EINVAL;
  long long N = 1;
  for (int i = 0; i < ndim; ++i) {
    if (n[i] < 2 || (n[i] % 2) != 0 || n[i] > (1 << 20)) return VOFL_EINVAL;
    if (!(hi[i] > lo[i]) || !std::isfinite(lo[i]) || !std::isfinite(hi[i])) return VOFL_EINVAL;
    N *= n[i];
  }
  if (N > (1LL << 34)) return VOFL_EINVAL;
  if (impl == VOFL_IMPL_FUSED && !fused2d_supported(ndim, n, prec) && !fused1d_supported(ndim, n, prec) &&
      !fused3d_supported(ndim, n, prec))
    return VOFL_EUNSUPPORTED;

  vofl_ctx* c = new vofl_ctx();
  c->ndim = ndim;
  c->N = N;
  c->prec = prec;
  c->impl = impl;
  c->cn_tol = prec == VOFL_F64 ? 1e-15 : 1e-6;
  for (int i = 0; i < ndim; ++i) {
    c->n[i] = n[i];
    c->lo[i] = lo[i];
    c->hi[i] = hi[i];
  }
  cudaGetDevice(&c->device);
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else if (cudaStreamCreate(&c->stream) != cudaSuccess) {  // blocking: ordered with the legacy stream
    delete c;
    return VOFL_ECUDA;
  } else {
    c->own_stream = true;
  }
  const size_t r = elem_size(c);
  bool ok = true;
  ok &= dev_malloc(&c->delta, r * N) == cudaSuccess;
  ok &= dev_malloc(&c->A, r * N) == cudaSuccess;
  ok &= dev_malloc(&c->B, r * N) == cudaSuccess;
  ok &= dev_malloc(&c->u[0], r * N) == cudaSuccess;
  ok &= dev_malloc(&c->u[1], r * N) == cudaSuccess;
  ok &= dev_malloc(&c->l2p, r * N) == cudaSuccess;
  ok &= dev_malloc(&c->d_gamma, sizeof(double) * N) == cudaSuccess;
  ok &= dev_malloc(&c->d_scratch, sizeof(double) * 1024) == cudaSuccess;
  ok &= dev_malloc(&c->d_step, sizeof(int) * 4) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    vofl_destroy(c);
    return VOFL_ENOMEM;
  }
  cudaMemsetAsync(c->u[0], 0, r * N, c->stream);
  cudaMemsetAsync(c->u[1], 0, r * N, c->stream);
  cudaMemsetAsync(c->l2p, 0, r * N, c->stream);
  cudaMemsetAsync(c->d_step, 0, sizeof(int) * 4, c->stream);
  int st = VOFL_OK;
  if (impl == VOFL_IMPL_FUSED)
    c->eng = ndim == 1 ? make_fused1d(c, &st) : (ndim == 2 ? make_fused2d(c, &st) : make_fused3d(c, &st));
  else
    c->eng = make_plain(c, &st);
  if (!c->eng) {
    vofl_destroy(c);
    return st ? st : VOFL_ECUDA;
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    vofl_destroy(c);
    return VOFL_ECUDA;
  }
  *out = c;
  return VOFL_OK;
}

void vofl_destroy(vofl_ctx* c) {
  if (!c) return;
  if (c->batch) batch_detach(c);
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  delete c->eng;
  dev_free(c->delta);
  dev_free(c->A);
  dev_free(c->B);
  dev_free(c->u[0]);
  dev_free(c->u[1]);
  dev_free(c->l2p);
  dev_free(c->d_gamma);
  dev_free(c->d_scratch);
  dev_free(c->d_step);
  dev_free(c->d_src);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* vofl_last_error(const vofl_ctx* c) { return c ? c->err.c_str() : "null context"; }

static int finish_model(vofl_ctx* c, const double* d_c0field, double c0, double omega0) {
  int st = model_from_gamma(c, c->d_gamma, d_c0field, c0, omega0);
  if (st) return st;
  c->f1 = c->f3 = 0.0;
  st = c->eng->set_model(c);
  if (st) return st;
  c->model_set = true;
  reset_run(c);
  return VOFL_OK;
}

int vofl_set_q(vofl_ctx* c, const double* Q, int on_device, double c0, double omega0) {
  NvtxRange nvtx_range("vofl_set_q");
  if (int st = check_ctx(c)) return st;
  if (!Q) return set_err(c, VOFL_EINVAL, "Q is null");
  if (!(c0 > 0) || !(omega0 > 0)) return set_err(c, VOFL_EINVAL, "c0 and omega0 must be positive");
  int st = upload(c, c->d_gamma, Q, sizeof(double) * c->N, on_device);
  if (st) return st;
  st = model_gamma_from_q(c, c->d_gamma, c->d_gamma);
  if (st) return st;
  return finish_model(c, nullptr, c0, omega0);
}

int vofl_set_order(vofl_ctx* c, const double* s, int on_device, double kappa, double f1, double f3) {
  NvtxRange nvtx_range("vofl_set_order");
  if (int st = check_ctx(c)) return st;
  if (!s) return set_err(c, VOFL_EINVAL, "s is null");
  if (!(kappa > 0) || !std::isfinite(kappa) || !std::isfinite(f1) || !std::isfinite(f3))
    return set_err(c, VOFL_EINVAL, "kappa must be positive, f1 and f3 finite");
  int st = upload(c, c->d_gamma, s, sizeof(double) * c->N, on_device);
  if (st) return st;
  st = model_from_order(c, c->d_gamma, kappa);
  if (st) return st;
  c->f1 = f1;
  c->f3 = f3;
  st = c->eng->set_model(c);
  if (st) return st;
  c->model_set = true;
  reset_run(c);
  return VOFL_OK;
}

int vofl_set_gamma(vofl_ctx* c, const double* gamma, const double* c0_field, int on_device, double c0,
                   double omega0) {
  if (int st = check_ctx(c)) return st;
  if (!gamma) return set_err(c, VOFL_EINVAL, "gamma is null");
  if (!(omega0 > 0) || (!c0_field && !(c0 > 0))) return set_err(c, VOFL_EINVAL, "c0 and omega0 must be positive");
  int st = upload(c, c->d_gamma, gamma, sizeof(double) * c->N, on_device);
  if (st) return st;
  double* d_c0 = nullptr;
  if (c0_field) {
    VOFL_CUDA(c, dev_malloc(&d_c0, sizeof(double) * c->N));
    st = upload(c, d_c0, c0_field, sizeof(double) * c->N, on_device);
    if (st) {
      dev_free(d_c0);
      return st;
    }
  }
  st = finish_model(c, d_c0, c0, omega0);
  if (d_c0) {
    cudaStreamSynchronize(c->stream);
    dev_free(d_c0);
  }
  return st;
}

int vofl_set_M(vofl_ctx* c, int M) {
  if (int st = check_ctx(c)) return st;
  if (M < 0 || M > 40) return set_err(c, VOFL_EINVAL, "M must be in [0, 40]");
  c->M = M;  // captured graphs are re-keyed on the next step
  return VOFL_OK;
}

namespace {
int apply_checked(vofl_ctx* c, const void* u, void* o1, void* o2) {
  if (!c->model_set) return set_err(c, VOFL_ESTATE, "set the model first");
  if (!u || (!o1 && !o2)) return set_err(c, VOFL_EINVAL, "null array");
  if (int st = c->eng->prepare(c)) return st;
  return c->eng->apply_pair(c, u, o1, o2);
}
}  // namespace

int vofl_apply_pair(vofl_ctx* c, const void* u, void* o1, void* o2) {
  NvtxRange nvtx_range("vofl_apply_pair");
  if (int st = check_ctx(c)) return st;
  if (c->general) return set_err(c, VOFL_EINVAL, "the general model has one operator: vofl_apply(VOFL_OP_S)");
  return apply_checked(c, u, o1, o2);
}

int vofl_apply(vofl_ctx* c, int op, const void* u, void* out) {
  NvtxRange nvtx_range("vofl_apply");
  if (int st = check_ctx(c)) return st;
  if (op != VOFL_OP_1PG && op != VOFL_OP_HPG && op != VOFL_OP_S) return set_err(c, VOFL_EINVAL, "unknown operator");
  if (c->model_set && (op == VOFL_OP_S) != c->general)
    return set_err(c, VOFL_EINVAL, "VOFL_OP_S goes with vofl_set_order, the two seismic operators with set_q/gamma");
  return apply_checked(c, u, op != VOFL_OP_HPG ? out : nullptr, op == VOFL_OP_HPG ? out : nullptr);
}

int vofl_set_state(vofl_ctx* c, const void* u0, const void* v0, int on_device) {
  if (int st = check_ctx(c)) return st;
  if (!u0) return set_err(c, VOFL_EINVAL, "u0 is null");
  const size_t b = elem_size(c) * c->N;
  reset_run(c);
  int st = upload(c, c->u[0], u0, b, on_device);
  if (st) return st;
  if (v0) {
    st = upload(c, c->u[1], v0, b, on_device);
    if (st) return st;
    c->psi_nonzero = true;
  } else {
    VOFL_CUDA(c, cudaMemsetAsync(c->u[1], 0, b, c->stream));
    c->psi_nonzero = false;
  }
  VOFL_CUDA(c, cudaMemsetAsync(c->l2p, 0, b, c->stream));
  c->state_set = true;
  return VOFL_OK;
}

int vofl_set_source(vofl_ctx* c, const int64_t* idx, const double* samples, int64_t nsamples, int on_device) {
  if (int st = check_ctx(c)) return st;
  if (nsamples <= 0) {
    c->nsrc = 0;
    c->src_flat = -1;
    return VOFL_OK;
  }
  if (!idx || !samples) return set_err(c, VOFL_EINVAL, "null source argument");
  long long flat = 0, stride = 1;
  for (int i = 0; i < c->ndim; ++i) {
    if (idx[i] < 0 || idx[i] >= c->n[i]) return set_err(c, VOFL_EINVAL, "source index outside the grid");
    flat += idx[i] * stride;
    stride *= c->n[i];
  }
  if (nsamples > c->src_cap) {
    // a new buffer first: a failed allocation leaves the old source in place
    double* d_new = nullptr;
    VOFL_CUDA(c, dev_malloc(&d_new, sizeof(double) * nsamples));
    drop_graphs(c);  // graphs hold the old pointer
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {  // queued steps may still read the old samples
      dev_free(d_new);
      return cuda_err(c, cudaGetLastError(), "cudaStreamSynchronize");
    }
    dev_free(c->d_src);
    c->d_src = d_new;
    c->src_cap = nsamples;
  }
  int st = upload(c, c->d_src, samples, sizeof(double) * nsamples, on_device);
  if (st) return st;
  c->nsrc = nsamples;
  c->src_flat = flat;
  return VOFL_OK;
}

int vofl_set_scheme(vofl_ctx* c, int scheme) {
  if (int st = check_ctx(c)) return st;
  if (scheme != VOFL_SCHEME_LFFP && scheme != VOFL_SCHEME_TSFP2 && scheme != VOFL_SCHEME_CNFP)
    return set_err(c, VOFL_EINVAL, "unknown scheme");
  if (c->steps > 0 && scheme != c->scheme) return set_err(c, VOFL_ESTATE, "a run is in progress; set the state first");
  c->scheme = scheme;
  return VOFL_OK;
}

int vofl_step(vofl_ctx* c, int64_t nsteps, double dt) {
  NvtxRange nvtx_range("vofl_step");
  if (int st = check_ctx(c)) return st;
  if (nsteps < 0) return set_err(c, VOFL_EINVAL, "bad nsteps");
  if (c->scheme == VOFL_SCHEME_TSFP2) {
    if (!c->general || !c->eng->can_split())
      return set_err(c, VOFL_EUNSUPPORTED,
                     "the time splitting needs the general model and the plain path or the fused 2D path");
    if (!c->model_set || !c->state_set) return set_err(c, VOFL_ESTATE, "set the model and the state first");
    if (!(dt > 0) || !std::isfinite(dt)) return set_err(c, VOFL_EINVAL, "bad dt");
    if (c->steps > 0 && dt != c->dt) return set_err(c, VOFL_EINVAL, "dt must stay fixed during a run");
    if (int st = c->eng->prepare(c)) return st;
    c->dt = dt;
    // merged flows: S(dt/2) [K S(dt)]^n S(-dt/2) = [S(dt/2) K S(dt/2)]^n
    const bool merged = c->eng->split_merged() && nsteps > 0;
    if (merged)
      if (int st = c->eng->split_flow(c, 0.5 * dt)) return st;
    for (int64_t i = 0; i < nsteps; ++i)
      if (int st = split_step(c)) return st;
    if (merged)
      if (int st = c->eng->split_flow(c, -0.5 * dt)) return st;
    return VOFL_OK;
  }
  if (c->scheme == VOFL_SCHEME_CNFP) {
    if (!c->general || !c->eng->can_cn())
      return set_err(c, VOFL_EUNSUPPORTED, "the Crank-Nicolson scheme needs the general model and the plain path");
    if (c->nsrc > 0) return set_err(c, VOFL_EUNSUPPORTED, "the Crank-Nicolson scheme takes no point source");
    if (int st = prepare_run(c, dt)) return st;
    if (nsteps == 0) return VOFL_OK;
    if (c->steps == 0) {  // explicit start (Eq. (3.3)), as in the leap-frog scheme
      int st = c->eng->step(c, EPI_START, false);
      if (st) return st;
      c->cur ^= 1;
      c->steps = 1;
      --nsteps;
    }
    for (int64_t i = 0; i < nsteps; ++i) {
      int st = c->eng->step_cn(c);
      if (st) return st;
      c->cur ^= 1;
      c->steps += 1;
    }
    return VOFL_OK;
  }
  if (int st = prepare_run(c, dt)) return st;
  if (nsteps == 0) return VOFL_OK;
  if (c->eng->can_run()) {
    // the whole request in one launch
    const int st = c->eng->run(c, nsteps, c->steps == 0 ? EPI_START : EPI_STEP);
    if (st) return st;
    c->cur = (int)((c->cur + nsteps) & 1);
    c->steps += nsteps;
    return VOFL_OK;
  }
  if (c->steps == 0) {
    int st = c->eng->step(c, EPI_START, false);
    if (st) return st;
    c->cur ^= 1;
    c->steps = 1;
    --nsteps;
  }
  for (int64_t i = 0; i < nsteps; ++i) {
    int st = one_step(c);
    if (st) return st;
  }
  return VOFL_OK;
}

// ---- checkpoint / resume ----
namespace {
// the fixed part of a checkpoint; the arrays follow it in this order:
// u[0], u[1], l2p, delta, A, B (N elements of the context precision each),
// the order field s or gamma (N doubles), the source samples (nsrc doubles)
struct Checkpoint {
  char magic[8];
  int64_t ndim, n[3], prec, M, scheme, general, cur, psi_nonzero, steps, cn_maxit, nsrc, src_flat;
  double lo[3], hi[3], dt, gamma0, s01, s02, kappa, f1, f3, cn_tol;
  int32_t d_step[2];  // step counter and error word
};
const char kCkptMagic[8] = {'V', 'O', 'F', 'L', 'C', 'K', 'P', '1'};

size_t ckpt_bytes(const vofl_ctx* c, int64_t nsrc) {
  return sizeof(Checkpoint) + 6 * elem_size(c) * (size_t)c->N + sizeof(double) * ((size_t)c->N + (size_t)nsrc);
}
}  // namespace

int vofl_save_state(vofl_ctx* c, void* blob, size_t* nbytes) {
  NvtxRange nvtx_range("vofl_save_state");
  if (int st = check_ctx(c)) return st;
  if (!nbytes) return set_err(c, VOFL_EINVAL, "nbytes is null");
  if (!c->model_set || !c->state_set) return set_err(c, VOFL_ESTATE, "set the model and the state first");
  const size_t need = ckpt_bytes(c, c->nsrc);
  if (!blob) {
    *nbytes = need;
    return VOFL_OK;
  }
  if (*nbytes < need) {
    *nbytes = need;
    return set_err(c, VOFL_EINVAL, "checkpoint buffer too small");
  }
  VOFL_CUDA(c, cudaStreamSynchronize(c->stream));  // the queued steps first
  Checkpoint h{};
  std::memcpy(h.magic, kCkptMagic, 8);
  h.ndim = c->ndim;
  h.prec = c->prec;
  for (int i = 0; i < 3; ++i) {
    h.n[i] = c->n[i];
    h.lo[i] = c->lo[i];
    h.hi[i] = c->hi[i];
  }
  h.M = c->M;
  h.scheme = c->scheme;
  h.general = c->general ? 1 : 0;
  h.cur = c->cur;
  h.psi_nonzero = c->psi_nonzero ? 1 : 0;
  h.steps = c->steps;
  h.cn_maxit = c->cn_maxit;
  h.nsrc = c->nsrc;
  h.src_flat = c->src_flat;
  h.dt = c->dt;
  h.gamma0 = c->gamma0;
  h.s01 = c->s01;
  h.s02 = c->s02;
  h.kappa = c->kappa;
  h.f1 = c->f1;
  h.f3 = c->f3;
  h.cn_tol = c->cn_tol;
  VOFL_CUDA(c, cudaMemcpy(h.d_step, c->d_step, 2 * sizeof(int), cudaMemcpyDeviceToHost));
  unsigned char* p = static_cast<unsigned char*>(blob);
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  const size_t b = elem_size(c) * (size_t)c->N;
  for (const void* src : {(const void*)c->u[0], (const void*)c->u[1], (const void*)c->l2p, (const void*)c->delta,
                          (const void*)c->A, (const void*)c->B}) {
    VOFL_CUDA(c, cudaMemcpy(p, src, b, cudaMemcpyDeviceToHost));
    p += b;
  }
  VOFL_CUDA(c, cudaMemcpy(p, c->d_gamma, sizeof(double) * c->N, cudaMemcpyDeviceToHost));
  p += sizeof(double) * c->N;
  if (c->nsrc > 0) VOFL_CUDA(c, cudaMemcpy(p, c->d_src, sizeof(double) * c->nsrc, cudaMemcpyDeviceToHost));
  *nbytes = need;
  return VOFL_OK;
}

int vofl_load_state(vofl_ctx* c, const void* blob, size_t nbytes) {
  NvtxRange nvtx_range("vofl_load_state");
  if (int st = check_ctx(c)) return st;
  if (!blob || nbytes < sizeof(Checkpoint)) return set_err(c, VOFL_EINVAL, "not a checkpoint");
  Checkpoint h;
  std::memcpy(&h, blob, sizeof(h));
  if (std::memcmp(h.magic, kCkptMagic, 8) != 0) return set_err(c, VOFL_EINVAL, "not a checkpoint");
  bool same = h.ndim == c->ndim && h.prec == c->prec;
  for (int i = 0; i < 3; ++i) same = same && h.n[i] == c->n[i] && h.lo[i] == c->lo[i] && h.hi[i] == c->hi[i];
  if (!same) return set_err(c, VOFL_EINVAL, "the checkpoint belongs to another grid or precision");
  if (h.nsrc < 0 || h.M < 0 || h.M > 40 || nbytes != ckpt_bytes(c, h.nsrc))
    return set_err(c, VOFL_EINVAL, "checkpoint size does not match its header");
  // every header field that indexes memory or selects a code path is
  // checked before anything is copied: a damaged or foreign header must
  // not index past the state buffers or move the source node off the grid
  if (h.cur != 0 && h.cur != 1) return set_err(c, VOFL_EINVAL, "checkpoint: bad state buffer index");
  if (h.nsrc > 0 && (h.src_flat < 0 || h.src_flat >= c->N))
    return set_err(c, VOFL_EINVAL, "checkpoint: source node outside the grid");
  if (h.scheme != VOFL_SCHEME_LFFP && h.scheme != VOFL_SCHEME_TSFP2 && h.scheme != VOFL_SCHEME_CNFP)
    return set_err(c, VOFL_EINVAL, "checkpoint: unknown scheme");
  if ((h.general != 0 && h.general != 1) || (h.psi_nonzero != 0 && h.psi_nonzero != 1))
    return set_err(c, VOFL_EINVAL, "checkpoint: bad flag");
  if (!h.general && h.scheme != VOFL_SCHEME_LFFP)
    return set_err(c, VOFL_EINVAL, "checkpoint: the seismic model has only the leap-frog scheme");
  if (h.cn_maxit < 1 || h.cn_maxit > INT32_MAX || !(h.cn_tol > 0) || !(h.cn_tol < 1))
    return set_err(c, VOFL_EINVAL, "checkpoint: bad solver settings");
  if (h.steps < 0 || !std::isfinite(h.dt) || h.dt < 0 || h.d_step[0] < 0)
    return set_err(c, VOFL_EINVAL, "checkpoint: bad step count or time step");
  if (!std::isfinite(h.gamma0) || !std::isfinite(h.s01) || !std::isfinite(h.s02) || !std::isfinite(h.kappa) ||
      !std::isfinite(h.f1) || !std::isfinite(h.f3))
    return set_err(c, VOFL_EINVAL, "checkpoint: non-finite model constant");
  VOFL_CUDA(c, cudaStreamSynchronize(c->stream));
  // the one allocation first, into a new buffer: if it fails the context
  // is left exactly as it was
  if (h.nsrc > c->src_cap) {
    double* d_new = nullptr;
    VOFL_CUDA(c, dev_malloc(&d_new, sizeof(double) * h.nsrc));
    drop_graphs(c);  // they hold the old source pointer
    dev_free(c->d_src);
    c->d_src = d_new;
    c->src_cap = h.nsrc;
  }
  const unsigned char* p = static_cast<const unsigned char*>(blob) + sizeof(h);
  const size_t b = elem_size(c) * (size_t)c->N;
  for (void* dst : {c->u[0], c->u[1], c->l2p, c->delta, c->A, c->B}) {
    VOFL_CUDA(c, cudaMemcpy(dst, p, b, cudaMemcpyHostToDevice));
    p += b;
  }
  VOFL_CUDA(c, cudaMemcpy(c->d_gamma, p, sizeof(double) * c->N, cudaMemcpyHostToDevice));
  p += sizeof(double) * c->N;
  if (h.nsrc > 0) VOFL_CUDA(c, cudaMemcpy(c->d_src, p, sizeof(double) * h.nsrc, cudaMemcpyHostToDevice));
  VOFL_CUDA(c, cudaMemcpy(c->d_step, h.d_step, 2 * sizeof(int), cudaMemcpyHostToDevice));
  drop_graphs(c);  // they may hold the old source pointer
  c->M = (int)h.M;
  c->scheme = (int)h.scheme;
  c->general = h.general != 0;
  c->gamma0 = h.gamma0;
  c->s01 = h.s01;
  c->s02 = h.s02;
  c->kappa = h.kappa;
  c->f1 = h.f1;
  c->f3 = h.f3;
  c->cn_tol = h.cn_tol;
  c->cn_maxit = (int)h.cn_maxit;
  c->nsrc = h.nsrc;
  c->src_flat = h.nsrc > 0 ? h.src_flat : -1;
  // the engine's spectral tables follow from s01, s02 (and kappa)
  if (int st = c->eng->set_model(c)) return st;
  c->model_set = true;
  c->state_set = true;
  c->cur = (int)h.cur;
  c->psi_nonzero = h.psi_nonzero != 0;
  c->steps = h.steps;
  c->dt = h.dt;
  c->cn_iters = 0;
  c->cn_solves = 0;
  return VOFL_OK;
}

int vofl_set_solver(vofl_ctx* c, double tol, int max_iter) {
  if (int st = check_ctx(c)) return st;
  if (!(tol > 0) || !(tol < 1) || max_iter < 1) return set_err(c, VOFL_EINVAL, "bad solver tolerance or iteration cap");
  c->cn_tol = tol;
  c->cn_maxit = max_iter;
  return VOFL_OK;
}

int vofl_solver_stats(vofl_ctx* c, int64_t* iterations, int64_t* solves) {
  if (!c) return VOFL_EINVAL;
  if (iterations) *iterations = c->cn_iters;
  if (solves) *solves = c->cn_solves;
  return VOFL_OK;
}

int vofl_suggest_M(vofl_ctx* c, double tol, int* M) {
  if (int st = check_ctx(c)) return st;
  if (!M || !(tol > 0) || !std::isfinite(tol)) return set_err(c, VOFL_EINVAL, "bad tol or M pointer");
  if (!c->model_set) return set_err(c, VOFL_ESTATE, "set the model first");
  return model_suggest_M(c, tol, 40, M);
}

int vofl_query(vofl_ctx* c) {
  if (!c) return VOFL_EINVAL;
  const cudaError_t e = cudaStreamQuery(c->stream);
  if (e == cudaSuccess) return 1;
  if (e == cudaErrorNotReady) {
    cudaGetLastError();
    return 0;
  }
  return cuda_err(c, e, "cudaStreamQuery");
}

int vofl_suggest_dt(vofl_ctx* c, double courant, double* dt) {
  if (int st = check_ctx(c)) return st;
  if (!dt || !(courant > 0) || !std::isfinite(courant)) return set_err(c, VOFL_EINVAL, "bad courant or dt pointer");
  if (!c->model_set) return set_err(c, VOFL_ESTATE, "set the model first");
  return model_suggest_dt(c, courant, dt);
}

int64_t vofl_steps_taken(const vofl_ctx* c) { return c ? c->steps : -1; }

int vofl_get_state(vofl_ctx* c, void* u_out, int on_device) {
  if (int st = check_ctx(c)) return st;
  if (!u_out) return set_err(c, VOFL_EINVAL, "null output");
  const size_t b = elem_size(c) * c->N;
  VOFL_CUDA(c, cudaMemcpyAsync(u_out, c->u[c->cur], b, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                               c->stream));
  if (!on_device) VOFL_CUDA(c, cudaStreamSynchronize(c->stream));
  return VOFL_OK;
}

int vofl_sync(vofl_ctx* c) {
  if (int st = check_ctx(c)) return st;
  VOFL_CUDA(c, cudaStreamSynchronize(c->stream));
  VOFL_CUDA(c, cudaGetLastError());
  // device error word (d_step[1]): set by a bounded wait that gave up
  int werr = 0;
  VOFL_CUDA(c, cudaMemcpy(&werr, c->d_step + 1, sizeof(int), cudaMemcpyDeviceToHost));
  if (werr) {
    VOFL_CUDA(c, cudaMemset(c->d_step + 1, 0, sizeof(int)));
    c->eng->reset_waits(c);
    return set_err(c, VOFL_ETIMEDOUT, "a device wait gave up (asynchronous copy never completed)");
  }
  return VOFL_OK;
}

int64_t vofl_debug_fail_alloc(int64_t k) { return (int64_t)debug_fail_alloc((long long)k); }

int64_t vofl_debug_canaries(int64_t* live_buffers, int poke) {
  long long live = 0;
  const long long bad = debug_canaries(&live, poke);
  if (live_buffers) *live_buffers = (int64_t)live;
  return (int64_t)bad;
}

int vofl_rel_l2(vofl_ctx* c, const void* x_dev, int x_prec, const void* y_dev, int y_prec, double* out) {
  NvtxRange nvtx_range("vofl_rel_l2");
  if (int st = check_ctx(c)) return st;
  if (!x_dev || !y_dev || !out) return set_err(c, VOFL_EINVAL, "null diagnostic argument");
  if ((x_prec != VOFL_F32 && x_prec != VOFL_F64) || (y_prec != VOFL_F32 && y_prec != VOFL_F64))
    return set_err(c, VOFL_EINVAL, "bad precision");
  return model_rel_l2(c, x_dev, x_prec, y_dev, y_prec, out);
}

int vofl_set_schedule(vofl_ctx* c, const vofl_schedule* sched) {
  NvtxRange nvtx_range("vofl_set_schedule");
  if (int st = check_ctx(c)) return st;
  if (!sched) return set_err(c, VOFL_EINVAL, "null schedule");
  if (sched->wide_cols < -1 || sched->wide_cols > 1 || sched->wide_rows < -1 || sched->wide_rows > 1 ||
      sched->col_parts < 0 || sched->col_parts > 41 || sched->group < 0 || sched->group > 41 ||
      sched->fuse_forward < -1 || sched->fuse_forward > 2 || sched->wide_fwd < -1 || sched->wide_fwd > 1 ||
      sched->row_split < 0 || sched->row_split > 16 || sched->col_pack < -1 || sched->col_pack > 65535)
    return set_err(c, VOFL_EINVAL, "schedule field out of range");
  VOFL_CUDA(c, cudaStreamSynchronize(c->stream));  // queued work may use the buffers being re-sized
  drop_graphs(c);
  return c->eng->set_schedule(c, sched);
}

int vofl_get_schedule(vofl_ctx* c, vofl_schedule* sched) {
  // a host-side query: allowed while a batch steps the context
  if (!c || !c->eng) return VOFL_EINVAL;
  if (!sched) return set_err(c, VOFL_EINVAL, "null schedule");
  return c->eng->get_schedule(c, sched);
}

int vofl_profile_kernels(vofl_ctx* c, int reps, char* names_out, size_t names_cap, double* ms_out, double* units_out,
                         int cap) {
  if (int st = check_ctx(c)) return st;
  if (!c->model_set || !c->state_set) return set_err(c, VOFL_ESTATE, "set the model and the state first");
  if (reps < 1 || !names_out || !ms_out || !units_out) return set_err(c, VOFL_EINVAL, "bad profile arguments");
  std::string names;
  int k = c->eng->profile(c, reps, names, ms_out, units_out, cap);
  if (k < 0) return k;
  if (names.size() + 1 > names_cap) return set_err(c, VOFL_EINVAL, "names buffer too small");
  std::memcpy(names_out, names.c_str(), names.size() + 1);
  return k;
}

}  // extern "C"
