// batch2d.cu -- many independent 2D simulations stepped together.
//
// A batch borrows fused FP32 2D contexts (each keeps its own fields, tables
// and scratch) and advances all of them by the same number of leap-frog
// steps of Eq. (1.1) (the step of fused2d.cu: F1, F2, then per Taylor group
// I1, I2).  Simulations of one grid size form a class; each kernel of a step
// is launched once per class (or per chunk of a class), with blockIdx.z
// selecting the simulation and every pointer and scalar read from that
// simulation's descriptor (BatchSim).  Small grids that leave the GPU idle
// alone fill it together; classes may run on parallel branches of the step
// graph.  Simulations may differ in size, model, M, dt, source and start
// time: a simulation whose M has fewer Taylor groups skips the groups above
// its own, and one that joins before its first step takes the Taylor start.
//
// The arithmetic per simulation is the same code as the single-context
// path (the kernel bodies of kernels.cuh), so a simulation gives the same
// bits alone and in a batch.
//
// Steps are replayed from CUDA graphs: a two-step graph (descriptor sets
// for the two buffer parities) and a one-step graph.  The descriptors are
// rewritten (one host-to-device copy) at each call, so the graphs survive
// everything except a change of membership or schedule.
//
// Autotuning: the schedule is how many simulations of a class share one
// launch (the whole class gives the most parallelism; smaller chunks keep a
// chunk's intermediates in L2) and whether classes run on parallel graph
// branches.  vofl_batch_tune times candidates by coordinate search on the
// live batch, from a saved copy of the state that is put back afterwards.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "kernels_wide.cuh"

namespace vofl {
namespace {


constexpr double inv_fact_d(int m) {
  double f = 1.0;
  for (int i = 2; i <= m; ++i) f *= i;
  return 1.0 / f;
}
#define VOFL_IF(m) inv_fact_d(m)
// 1/m! in double; rounded once to float where used (as the single-context
// launcher rounds it), which keeps the float subnormals of large m
__constant__ double c_inv_fact[41] = {
    VOFL_IF(0),  VOFL_IF(1),  VOFL_IF(2),  VOFL_IF(3),  VOFL_IF(4),  VOFL_IF(5),  VOFL_IF(6),  VOFL_IF(7),  VOFL_IF(8),
    VOFL_IF(9),  VOFL_IF(10), VOFL_IF(11), VOFL_IF(12), VOFL_IF(13), VOFL_IF(14), VOFL_IF(15), VOFL_IF(16), VOFL_IF(17),
    VOFL_IF(18), VOFL_IF(19), VOFL_IF(20), VOFL_IF(21), VOFL_IF(22), VOFL_IF(23), VOFL_IF(24), VOFL_IF(25), VOFL_IF(26),
    VOFL_IF(27), VOFL_IF(28), VOFL_IF(29), VOFL_IF(30), VOFL_IF(31), VOFL_IF(32), VOFL_IF(33), VOFL_IF(34), VOFL_IF(35),
    VOFL_IF(36), VOFL_IF(37), VOFL_IF(38), VOFL_IF(39), VOFL_IF(40)};
#undef VOFL_IF

// -------------------------------------------------------------------------
// batched entry points (blockIdx.z = simulation of the chunk)
// -------------------------------------------------------------------------
template <int NX, int NY>
__global__ void __launch_bounds__(W_FROWS * 32) kb_fwd_rows(const BatchSim* __restrict__ sims) {
  const BatchSim* s = sims + blockIdx.z;
  fwd_rows_body<NX, false>(blockIdx.x, s->epi.u_cur, s->T, NY, 1, s->pT, s->ryy, 0.0f, s->twx,
                           const_cast<int*>(s->epi.step), s->inc_step, s->err);
}

template <int NX, int NY>
__global__ void __launch_bounds__(wide_frows_threads<NX>()) kb_fwd_rows_w(const BatchSim* __restrict__ sims) {
  const BatchSim* s = sims + blockIdx.z;
  fwd_rows_wide_body<NX>(blockIdx.x, s->epi.u_cur, s->T, NY, s->pT, s->ryy, s->twxw, const_cast<int*>(s->epi.step),
                         s->inc_step, s->err);
}

template <int NX, int NY>
__global__ void __launch_bounds__(W_FCOLS * 32) kb_fwd_cols(const BatchSim* __restrict__ sims) {
  const BatchSim* s = sims + blockIdx.z;
  fwd_cols_body<NY>(blockIdx.x, s->T, s->pT, s->Uh, NX / 2 + 1, s->twy);
}

template <int NX, int NY>
__global__ void __launch_bounds__(icols_warps<NY>() * 32) kb_inv_cols(const BatchSim* __restrict__ sims, int g,
                                                                      int parts, int pack, int BG) {
  const BatchSim* s = sims + blockIdx.z;
  const int m_lo = g * BG;
  if (m_lo > s->M) return;  // this simulation has fewer groups
  const int m_hi = min(s->M + 1, m_lo + BG);
  // the descriptor (with its tensor map) was written by a host copy
  if (threadIdx.x == 0) tmap_acquire(&s->zmap);
  inv_cols_body<NY>(blockIdx.x, blockIdx.y, parts, pack, s->Uh, s->P, s->Lg, &s->zmap, NX / 2 + 1, m_lo, m_hi,
                    (float)c_inv_fact[m_lo], (float)c_inv_fact[m_lo], 0, s->twy);
}

template <int NX, int NY>
__global__ void __launch_bounds__(W_IROWS * 32) kb_inv_rows(const BatchSim* __restrict__ sims, int g, int BG, int rsplit) {
  const BatchSim* s = sims + blockIdx.z;
  const int m_lo = g * BG;
  if (m_lo > s->M) return;
  const int m_hi = min(s->M + 1, m_lo + BG);
  // groups above 0 store partial sums (the body tests m_lo), so the
  // epilogue arguments are read from the descriptor only by group 0
  inv_rows_body<NX, false>(blockIdx.x, s->Z, s->zslot, s->pZ, NY, m_lo, m_hi, m_hi == s->M + 1 ? 1 : 0, s->M + 1, 0, s->delta,
                    s->part,
                    s->part + (size_t)NX * NY, s->epi, s->inv_lambda, s->twx, s->err, rsplit);
}

// wide inverse passes (fft_wide.cuh) for 512 and 1024 points, as the
// single-context launches of those sizes use them
template <int NX, int NY>
__global__ void __launch_bounds__(wide_threads<NY>(), wide_min_blocks<NY>()) kb_inv_cols_w(const BatchSim* __restrict__ sims, int g,
                                                                       int parts, int pack, int BG) {
  const BatchSim* s = sims + blockIdx.z;
  const int m_lo = g * BG;
  if (m_lo > s->M) return;
  const int m_hi = min(s->M + 1, m_lo + BG);
  inv_cols_wide_body<NY>(blockIdx.x, blockIdx.y, parts, pack, s->Uh, s->P, s->Lg, s->Z, s->pZ, NX / 2 + 1, m_lo, m_hi,
                         (float)c_inv_fact[m_lo], (float)c_inv_fact[m_lo], 0, s->twyw);
}

template <int NX, int NY>
__global__ void __launch_bounds__(wide_rows_threads<NX>(), NX == 1024 ? 1 : 6) kb_inv_rows_w(const BatchSim* __restrict__ sims, int g, int BG, int rsplit) {
  (void)rsplit;
  const BatchSim* s = sims + blockIdx.z;
  const int m_lo = g * BG;
  if (m_lo > s->M) return;
  const int m_hi = min(s->M + 1, m_lo + BG);
  inv_rows_wide_body<NX, false>(blockIdx.x, s->Z, s->zslot, s->pZ, NY, m_lo, m_hi, m_hi == s->M + 1 ? 1 : 0,
                                s->M + 1, 0, s->delta, s->part, s->part + (size_t)NX * NY, s->epi, s->inv_lambda,
                                s->twxw, s->err);
}

struct BKernels {
  // 32-element (narrow) kernels, and the wide-line ones where built
  // (512 and 1024 points; null elsewhere)
  void (*fr)(const BatchSim*);
  void (*fr_w)(const BatchSim*) = nullptr;
  void (*fc)(const BatchSim*);
  void (*ic)(const BatchSim*, int, int, int, int);
  void (*ic_w)(const BatchSim*, int, int, int, int) = nullptr;
  void (*ir)(const BatchSim*, int, int, int);
  void (*ir_w)(const BatchSim*, int, int, int) = nullptr;
  size_t smem_fr, smem_fr_w = 0, smem_fc, smem_ic, smem_ic_w = 0, smem_ir, smem_ir_w = 0;
  int lpw_x, lpw_y;
  int wic;               // warps per CTA of kb_inv_cols
  int rpf, thr_fr;       // row pairs per CTA and threads: forward rows
  int rpf_w = 0, thr_fr_w = 0;
  int cpc, thr_ic;       // columns per CTA and threads: inverse columns
  int cpc_w = 0, thr_ic_w = 0;
  int wir, thr_ir;       // warps (rows x runs) per CTA and threads: inverse rows
  int rpc_w = 0, thr_ir_w = 0;
};

template <int NX, int NY>
BKernels bkernels_for() {
  BKernels k;
  k.fr = kb_fwd_rows<NX, NY>;
  k.fc = kb_fwd_cols<NX, NY>;
  k.smem_fr = frows_smem<NX, false>();
  k.smem_fc = exch_smem<NY, W_FCOLS>();
  k.lpw_x = LineFFT<NX>::LPW;
  k.lpw_y = LineFFT<NY>::LPW;
  k.wic = icols_warps<NY>();
  k.rpf = W_FROWS * k.lpw_x;
  k.thr_fr = W_FROWS * 32;
  k.ic = kb_inv_cols<NX, NY>;
  k.smem_ic = inv_cols_smem<NY>();
  k.cpc = k.wic * k.lpw_y;
  k.thr_ic = k.wic * 32;
  k.ir = kb_inv_rows<NX, NY>;
  k.smem_ir = inv_rows_smem<NX>();
  k.wir = W_IROWS;
  k.thr_ir = W_IROWS * 32;
  if constexpr (NY == 512 || NY == 1024) {
    k.ic_w = kb_inv_cols_w<NX, NY>;
    k.smem_ic_w = wide_cols_smem<NY>();
    k.cpc_w = wide_lines_per_cta<NY>();
    k.thr_ic_w = wide_threads<NY>();
  }
  if constexpr (NX == 512 || NX == 1024) {
    k.fr_w = kb_fwd_rows_w<NX, NY>;
    k.smem_fr_w = wide_frows_smem<NX>();
    k.rpf_w = wide_frows_lines<NX>();
    k.thr_fr_w = wide_frows_threads<NX>();
    k.ir_w = kb_inv_rows_w<NX, NY>;
    k.smem_ir_w = wide_rows_smem<NX>();
    k.rpc_w = wide_rows_per_cta<NX>();
    k.thr_ir_w = wide_rows_threads<NX>();
  }
  return k;
}

bool pick_bkernels(int nx, int ny, BKernels* k) {
  if (nx != ny) return false;
  switch (nx) {
    case 64: *k = bkernels_for<64, 64>(); return true;
    case 128: *k = bkernels_for<128, 128>(); return true;
    case 256: *k = bkernels_for<256, 256>(); return true;
    case 512: *k = bkernels_for<512, 512>(); return true;
    case 768: *k = bkernels_for<768, 768>(); return true;
    case 1024: *k = bkernels_for<1024, 1024>(); return true;
    default: return false;
  }
}

bool set_bsmem(const BKernels& k) {
  return set_kernel_smem(k.fr, k.smem_fr) == cudaSuccess &&
         set_kernel_smem(k.fc, k.smem_fc) == cudaSuccess &&
         set_kernel_smem(k.ic, k.smem_ic) == cudaSuccess &&
         set_kernel_smem(k.ir, k.smem_ir) == cudaSuccess &&
         (!k.fr_w || set_kernel_smem(k.fr_w, k.smem_fr_w) == cudaSuccess) &&
         (!k.ic_w || set_kernel_smem(k.ic_w, k.smem_ic_w) == cudaSuccess) &&
         (!k.ir_w || set_kernel_smem(k.ir_w, k.smem_ir_w) == cudaSuccess);
}

// The transform schedule of one size class: the fields of vofl_schedule
// that decide the arithmetic of the batched launches (its members' own
// schedule, so a member gives the bits of the same context stepped alone).
struct TSched {
  bool wc = false, wr = false, wf = false;
  int parts = 1, G = 17, rs = 1, pack = 0;
  bool operator==(const TSched& o) const {
    return wc == o.wc && wr == o.wr && wf == o.wf && parts == o.parts && G == o.G && rs == o.rs && pack == o.pack;
  }
};
TSched tsched_of(const vofl_schedule& v) {
  TSched t;
  t.wc = v.wide_cols == 1;
  t.wr = v.wide_rows == 1;
  t.wf = v.wide_fwd == 1;
  t.parts = v.col_parts;
  t.G = v.group;
  t.rs = v.row_split;
  t.pack = v.col_pack;
  return t;
}
vofl_schedule schedule_of(const TSched& t) {
  vofl_schedule v{};
  v.wide_cols = t.wc ? 1 : 0;
  v.wide_rows = t.wr ? 1 : 0;
  v.col_parts = t.parts;
  v.group = t.G;
  v.fuse_forward = -1;  // the same bits either way
  v.wide_fwd = t.wf ? 1 : 0;
  v.row_split = t.rs;
  v.col_pack = t.pack;
  return v;
}

// plain (non-programmatic) launch, for the first kernel of a graph branch
template <typename... KArgs, typename... Args>
cudaError_t launch_plain(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  count_launch();
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

}  // namespace
}  // namespace vofl

using namespace vofl;

struct vofl_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;

  struct Member {
    vofl_ctx* c;
    double dt;
    int slot;
  };
  std::vector<Member> mem;
  int next_slot = 0;

  // schedule: per grid size, simulations per launch (0 = the whole class),
  // and whether classes run on parallel branches
  std::map<int, int> chunk;
  bool parallel = true;
  // per grid size, the transform schedule of the batched launches (set by
  // the first member of the size, or by vofl_batch_tune_transform)
  std::map<int, TSched> tsched;

  struct Class {
    int n = 0;  // grid edge
    BKernels k{};
    TSched ts{};
    int off = 0, count = 0;  // descriptor range
  };
  std::vector<Class> classes;
  std::vector<int> order;  // member index per descriptor position

  BatchSim* d_desc = nullptr;  // [2][cap]
  int cap = 0;
  std::vector<BatchSim> h_desc;  // [2][n]

  cudaGraphExec_t g1 = nullptr, g2 = nullptr;
  bool dirty = true;
  uint64_t kernels_per_step = 0;
  std::vector<cudaStream_t> aux;
  std::vector<cudaEvent_t> ev;  // [0] fork, [1 + i] join of class i

  std::string err;
};

namespace {

int berr(vofl_batch* b, int code, const std::string& m) {
  if (b) b->err = m;
  return code;
}
int bcuda(vofl_batch* b, cudaError_t e, const char* where) {
  return berr(b, e == cudaErrorMemoryAllocation ? VOFL_ENOMEM : VOFL_ECUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

// a size whose last member left takes the schedule of its next first member
void forget_empty_sizes(vofl_batch* b) {
  for (auto it = b->tsched.begin(); it != b->tsched.end();) {
    bool used = false;
    for (auto& m : b->mem) used |= m.c->n[0] == it->first;
    it = used ? std::next(it) : b->tsched.erase(it);
  }
}

void drop_bgraphs(vofl_batch* b) {
  if (b->g1) cudaGraphExecDestroy(b->g1);
  if (b->g2) cudaGraphExecDestroy(b->g2);
  b->g1 = b->g2 = nullptr;
  b->dirty = true;
}

// Group members into classes (descriptor order = class order).
int plan(vofl_batch* b) {
  std::map<int, std::vector<int>> by;
  for (size_t i = 0; i < b->mem.size(); ++i) by[(int)b->mem[i].c->n[0]].push_back((int)i);
  b->classes.clear();
  b->order.clear();
  for (auto& kv : by) {
    vofl_batch::Class cl;
    cl.n = kv.first;
    cl.ts = b->tsched[cl.n];
    if (!pick_bkernels(cl.n, cl.n, &cl.k)) return berr(b, VOFL_EUNSUPPORTED, "batched kernels: grid size not built");
    if (!set_bsmem(cl.k)) return berr(b, VOFL_ECUDA, "shared-memory attributes of the batched kernels");
    cl.off = (int)b->order.size();
    cl.count = (int)kv.second.size();
    for (int i : kv.second) b->order.push_back(i);
    b->classes.push_back(cl);
  }
  const int n = (int)b->order.size();
  if (n > b->cap) {
    dev_free(b->d_desc);
    b->d_desc = nullptr;
    b->cap = 0;
    const int cap = std::max(16, n + n / 2);
    cudaError_t e = dev_malloc(&b->d_desc, sizeof(BatchSim) * 2 * cap);
    if (e != cudaSuccess) return bcuda(b, e, "cudaMalloc (batch descriptors)");
    b->cap = cap;
  }
  while (b->aux.size() < b->classes.size()) {
    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bcuda(b, e, "cudaStreamCreate (batch branch)");
    b->aux.push_back(s);
  }
  while (b->ev.size() < b->classes.size() + 1) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (r != cudaSuccess) return bcuda(b, r, "cudaEventCreate (batch)");
    b->ev.push_back(e);
  }
  return VOFL_OK;
}

// Descriptor of member i for a step at parity p (0: the call's first step
// of a pair, 1: the second) -- the context's current buffers swapped p times.
void describe(const vofl_batch::Member& m, int p, bool tune, BatchSim* d) {
  vofl_ctx* c = m.c;
  *d = BatchSim{};
  c->eng->batch_desc(c, d);
  const int cur = c->cur ^ p;
  EpiArgs<float>& e = d->epi;
  const bool start = !tune && c->steps + p == 0;
  e.mode = start ? EPI_START : EPI_STEP;
  e.u_cur = (const float*)c->u[cur];
  e.u_other = (float*)c->u[1 - cur];
  e.l2p = (float*)c->l2p;
  e.A = (const float*)c->A;
  e.B = (const float*)c->B;
  e.step = c->d_step;
  e.src = c->d_src;
  e.nsrc = c->nsrc;
  e.src_flat = c->nsrc > 0 ? c->src_flat : -1;
  double hd = 1.0;
  for (int i = 0; i < c->ndim; ++i) hd *= (c->hi[i] - c->lo[i]) / (double)c->n[i];
  e.src_scale = m.dt * m.dt / hd;
  epi_model(c, &e);
  e.dt1 = (float)m.dt;
  e.dt2 = (float)(m.dt * m.dt);
  d->delta = (const float*)c->delta;
  d->err = c->d_step + 1;
  d->M = c->M;
  d->inc_step = start ? 0 : 1;
}

int write_desc(vofl_batch* b, bool tune) {
  const int n = (int)b->order.size();
  b->h_desc.assign((size_t)2 * b->cap, BatchSim{});
  for (int p = 0; p < 2; ++p)
    for (int j = 0; j < n; ++j) describe(b->mem[b->order[j]], p, tune, &b->h_desc[(size_t)p * b->cap + j]);
  // pageable source: staged before return, copied in stream order
  cudaError_t e = cudaMemcpyAsync(b->d_desc, b->h_desc.data(), sizeof(BatchSim) * 2 * b->cap,
                                  cudaMemcpyHostToDevice, b->stream);
  return e == cudaSuccess ? VOFL_OK : bcuda(b, e, "descriptor upload");
}

int chunk_of(const vofl_batch* b, const vofl_batch::Class& cl) {
  auto it = b->chunk.find(cl.n);
  const int w = it == b->chunk.end() ? 0 : it->second;
  return (w <= 0 || w > cl.count) ? cl.count : w;
}

// Queue one step of every member (descriptor parity p).
cudaError_t enqueue_step(vofl_batch* b, int p) {
  const BatchSim* d = b->d_desc + (size_t)p * b->cap;
  const bool par = b->parallel && b->classes.size() > 1;
  cudaError_t e = cudaSuccess;
  if (par) {
    e = cudaEventRecord(b->ev[0], b->stream);
    if (e) return e;
  }
  for (size_t ci = 0; ci < b->classes.size(); ++ci) {
    const vofl_batch::Class& cl = b->classes[ci];
    cudaStream_t s = par ? b->aux[ci] : b->stream;
    if (par) {
      e = cudaStreamWaitEvent(s, b->ev[0], 0);
      if (e) return e;
    }
    const int w = chunk_of(b, cl);
    const int nx = cl.n, ny = cl.n, ncols = nx / 2 + 1;
    bool first = par;  // first kernel of a branch: plain launch
    for (int c0 = 0; c0 < cl.count; c0 += w) {
      const int nz = std::min(w, cl.count - c0);
      const BatchSim* dc = d + cl.off + c0;
      int Mmax = 0;
      for (int j = 0; j < nz; ++j) Mmax = std::max(Mmax, b->mem[b->order[cl.off + c0 + j]].c->M);
      const TSched& t = cl.ts;
      const bool wf = t.wf && cl.k.fr_w, wc = t.wc && cl.k.ic_w, wr = t.wr && cl.k.ir_w;
      const int rpc = wf ? cl.k.rpf_w : cl.k.rpf;
      const dim3 gfr((ny / 2 + rpc - 1) / rpc, 1, nz);
      auto* fr = wf ? cl.k.fr_w : cl.k.fr;
      const int thr_fr = wf ? cl.k.thr_fr_w : cl.k.thr_fr;
      const size_t sm_fr = wf ? cl.k.smem_fr_w : cl.k.smem_fr;
      e = first ? launch_plain(fr, gfr, dim3(thr_fr), sm_fr, s, dc) : launch_pdl(fr, gfr, dim3(thr_fr), sm_fr, s, dc);
      if (e) return e;
      first = false;
      const int cpf = W_FCOLS * cl.k.lpw_y;
      e = launch_pdl(cl.k.fc, dim3((ncols + cpf - 1) / cpf, 1, nz), dim3(W_FCOLS * 32), cl.k.smem_fc, s, dc);
      if (e) return e;
      const int cpc = wc ? cl.k.cpc_w : cl.k.cpc;
      const int rs = wr ? 1 : t.rs;
      const int rpi = wr ? cl.k.rpc_w : (cl.k.wir / rs) * cl.k.lpw_x;
      auto* ic = wc ? cl.k.ic_w : cl.k.ic;
      auto* ir = wr ? cl.k.ir_w : cl.k.ir;
      const int BG = t.G, parts = t.parts, pack = t.pack;
      const dim3 gic = pack > 0 ? dim3(pack, 1, nz) : dim3((ncols + cpc - 1) / cpc, 2 * parts, nz);
      for (int g = Mmax / BG; g >= 0; --g) {
        e = launch_pdl(ic, gic, dim3(wc ? cl.k.thr_ic_w : cl.k.thr_ic), wc ? cl.k.smem_ic_w : cl.k.smem_ic, s, dc, g,
                       parts, pack, BG);
        if (e) return e;
        e = launch_pdl(ir, dim3((ny + rpi - 1) / rpi, 1, nz), dim3(wr ? cl.k.thr_ir_w : cl.k.thr_ir),
                       wr ? cl.k.smem_ir_w : cl.k.smem_ir, s, dc, g, BG, rs);
        if (e) return e;
      }
    }
    if (par) {
      e = cudaEventRecord(b->ev[1 + ci], s);
      if (e) return e;
      e = cudaStreamWaitEvent(b->stream, b->ev[1 + ci], 0);
      if (e) return e;
    }
  }
  return cudaSuccess;
}

int capture(vofl_batch* b, int nsteps, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e) return bcuda(b, e, "batch graph capture");
  const uint64_t before = g_kernel_launches.load();
  cudaError_t le = cudaSuccess;
  for (int p = 0; p < nsteps && !le; ++p) le = enqueue_step(b, p);
  e = cudaStreamEndCapture(b->stream, &g);
  if (le || e) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return bcuda(b, le ? le : e, "batch step launch");
  }
  b->kernels_per_step = (g_kernel_launches.load() - before) / nsteps;
  g_kernel_launches.fetch_sub(b->kernels_per_step * nsteps);  // counted again at each replay
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return e == cudaSuccess ? VOFL_OK : bcuda(b, e, "batch graph instantiate");
}

int ensure_graphs(vofl_batch* b) {
  if (!b->dirty && b->g1 && b->g2) return VOFL_OK;
  drop_bgraphs(b);
  if (int st = plan(b)) return st;
  if (int st = capture(b, 1, &b->g1)) return st;
  if (int st = capture(b, 2, &b->g2)) return st;
  b->dirty = false;
  return VOFL_OK;
}

int replay(vofl_batch* b, cudaGraphExec_t g, int steps) {
  cudaError_t e = cudaGraphLaunch(g, b->stream);
  if (e) return bcuda(b, e, "batch graph launch");
  count_launch(b->kernels_per_step * steps);
  return VOFL_OK;
}

// Advance every member n >= 1 steps from the contexts' current state.
int run_steps(vofl_batch* b, int64_t n, bool tune) {
  if (int st = ensure_graphs(b)) return st;
  bool any_start = false;
  for (auto& m : b->mem) any_start |= m.c->steps == 0;
  auto advance = [&](int64_t k) {
    if (tune) return;
    for (auto& m : b->mem) {
      m.c->cur = (int)((m.c->cur + k) & 1);
      m.c->steps += k;
    }
  };
  if (any_start && !tune) {
    // the Taylor start of new members: one step, then all members step on
    if (int st = write_desc(b, false)) return st;
    if (int st = replay(b, b->g1, 1)) return st;
    advance(1);
    --n;
  }
  if (n <= 0) return VOFL_OK;
  if (int st = write_desc(b, tune)) return st;
  for (int64_t i = 0; i + 1 < n; i += 2)
    if (int st = replay(b, b->g2, 2)) return st;
  if (n & 1)
    if (int st = replay(b, b->g1, 1)) return st;
  advance(n);
  return VOFL_OK;
}

// ms per batch step of the current schedule, over `reps` two-step replays
int time_schedule(vofl_batch* b, int reps, double* ms) {
  if (int st = ensure_graphs(b)) return st;
  if (int st = write_desc(b, true)) return st;
  if (int st = replay(b, b->g2, 2)) return st;  // warm-up
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, b->stream);
  for (int r = 0; r < reps; ++r)
    if (int st = replay(b, b->g2, 2)) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return st;
    }
  cudaEventRecord(e1, b->stream);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e) return bcuda(b, e, "batch timing");
  *ms = t / (2.0 * reps);
  return VOFL_OK;
}

// hand the context back: its own stream waits for the batch's queued work
int release(vofl_batch* b, vofl_ctx* c) {
  cudaEvent_t e;
  cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  if (r == cudaSuccess) r = cudaEventRecord(e, b->stream);
  if (r == cudaSuccess) r = cudaStreamWaitEvent(c->stream, e, 0);
  cudaEventDestroy(e);
  c->batch = nullptr;
  return r == cudaSuccess ? VOFL_OK : bcuda(b, r, "batch release");
}

// What timing steps overwrite, saved and put back: both state buffers,
// L2 u^{n-1} and the step counter of every member.
struct Snapshot {
  std::vector<void*> buf;  // 4 per member
  int take(vofl_batch* b) {
    for (auto& m : b->mem) {
      const size_t bytes = sizeof(float) * (size_t)m.c->N;
      const void* src[4] = {m.c->u[0], m.c->u[1], m.c->l2p, m.c->d_step};
      for (int j = 0; j < 4; ++j) {
        const size_t nb = j < 3 ? bytes : sizeof(int);
        void* p = nullptr;
        cudaError_t e = dev_malloc(&p, nb);
        if (e == cudaSuccess) e = cudaMemcpyAsync(p, src[j], nb, cudaMemcpyDeviceToDevice, b->stream);
        buf.push_back(p);
        if (e != cudaSuccess) {
          release_all();
          return bcuda(b, e, "state snapshot");
        }
      }
    }
    return VOFL_OK;
  }
  void restore(vofl_batch* b) {
    size_t k = 0;
    for (auto& m : b->mem) {
      const size_t bytes = sizeof(float) * (size_t)m.c->N;
      void* dst[4] = {m.c->u[0], m.c->u[1], m.c->l2p, m.c->d_step};
      for (int j = 0; j < 4; ++j, ++k)
        cudaMemcpyAsync(dst[j], buf[k], j < 3 ? bytes : sizeof(int), cudaMemcpyDeviceToDevice, b->stream);
    }
    cudaStreamSynchronize(b->stream);
    release_all();
  }
  void release_all() {
    for (void* p : buf) dev_free(p);
    buf.clear();
  }
  ~Snapshot() { release_all(); }
};

}  // namespace

void vofl::batch_detach(vofl_ctx* c) {
  vofl_batch* b = c->batch;
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (size_t i = 0; i < b->mem.size(); ++i)
    if (b->mem[i].c == c) {
      b->mem.erase(b->mem.begin() + (long)i);
      break;
    }
  c->batch = nullptr;
  forget_empty_sizes(b);
  drop_bgraphs(b);
}

extern "C" {

int vofl_batch_create(vofl_batch** out, void* cuda_stream) {
  if (!out) return VOFL_EINVAL;
  *out = nullptr;
  vofl_batch* b = new vofl_batch();
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) {
    if (cuda_stream) {
      b->stream = (cudaStream_t)cuda_stream;
    } else {
      e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
      b->own_stream = e == cudaSuccess;
    }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return VOFL_ECUDA;
  }
  *out = b;
  return VOFL_OK;
}

void vofl_batch_destroy(vofl_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (auto& m : b->mem) release(b, m.c);
  drop_bgraphs(b);
  for (auto s : b->aux) cudaStreamDestroy(s);
  for (auto e : b->ev) cudaEventDestroy(e);
  dev_free(b->d_desc);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

const char* vofl_batch_last_error(const vofl_batch* b) { return b ? b->err.c_str() : "null batch"; }

int vofl_batch_add(vofl_batch* b, vofl_ctx* c, double dt, int* slot) {
  if (!b || !c) return VOFL_EINVAL;
  if (c->batch) return berr(b, VOFL_ESTATE, "the context is already in a batch");
  if (c->ndim != 2 || c->prec != VOFL_F32 || c->impl != VOFL_IMPL_FUSED || c->n[0] != c->n[1])
    return berr(b, VOFL_EUNSUPPORTED, "batches take fused FP32 contexts of square 2D grids");
  if (c->general)  // its solo steps split one operator's terms over both slots; batched steps do not
    return berr(b, VOFL_EUNSUPPORTED, "batches take contexts of the seismic model");
  BatchSim probe{};
  BKernels k;
  if (!c->eng || !c->eng->batch_desc(c, &probe) || !pick_bkernels((int)c->n[0], (int)c->n[1], &k))
    return berr(b, VOFL_EUNSUPPORTED, "this grid size has no batched kernels");
  if (c->device != b->device) return berr(b, VOFL_EINVAL, "the context lives on another GPU");
  if (c->M > 40) return berr(b, VOFL_EINVAL, "M above 40");
  // the size's transform schedule: the first member's, which every later
  // member of the size must share (the batched launches give each member
  // the bits of its context stepped alone)
  vofl_schedule vs{};
  if (c->eng->get_schedule(c, &vs) != VOFL_OK) return berr(b, VOFL_EUNSUPPORTED, "no transform schedule");
  const TSched ts = tsched_of(vs);
  if (!ts.wr && W_IROWS % ts.rs != 0)
    return berr(b, VOFL_EUNSUPPORTED, "row split not available in batched launches");
  if ((ts.wc && !k.ic_w) || (ts.wr && !k.ir_w) || (ts.wf && !k.fr_w))
    return berr(b, VOFL_EUNSUPPORTED, "wide line transform not built for batched launches of this size");
  forget_empty_sizes(b);
  auto known = b->tsched.find((int)c->n[0]);
  if (known != b->tsched.end() && !(known->second == ts))
    return berr(b, VOFL_EUNSUPPORTED,
                "the context's transform schedule differs from the batch's for this grid size");
  if (int st = prepare_run(c, dt)) return berr(b, st, std::string("context: ") + c->err);
  // the batch stream waits for the context's queued work (set-up, start)
  cudaEvent_t e;
  cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  if (r == cudaSuccess) r = cudaEventRecord(e, c->stream);
  if (r == cudaSuccess) r = cudaStreamWaitEvent(b->stream, e, 0);
  cudaEventDestroy(e);
  if (r != cudaSuccess) return bcuda(b, r, "batch join");
  c->batch = b;
  b->tsched[(int)c->n[0]] = ts;
  b->mem.push_back({c, dt, b->next_slot});
  if (slot) *slot = b->next_slot;
  ++b->next_slot;
  drop_bgraphs(b);
  return VOFL_OK;
}

int vofl_batch_remove(vofl_batch* b, int slot) {
  if (!b) return VOFL_EINVAL;
  for (size_t i = 0; i < b->mem.size(); ++i)
    if (b->mem[i].slot == slot) {
      vofl_ctx* c = b->mem[i].c;
      b->mem.erase(b->mem.begin() + (long)i);
      forget_empty_sizes(b);
      drop_bgraphs(b);
      return release(b, c);
    }
  return berr(b, VOFL_EINVAL, "no such slot");
}

int vofl_batch_size(const vofl_batch* b) { return b ? (int)b->mem.size() : VOFL_EINVAL; }

int vofl_batch_step(vofl_batch* b, int64_t nsteps) {
  NvtxRange nvtx_range("vofl_batch_step");
  if (!b || nsteps < 0) return berr(b, VOFL_EINVAL, "bad batch or nsteps");
  if (nsteps == 0 || b->mem.empty()) return VOFL_OK;
  return run_steps(b, nsteps, false);
}

int vofl_batch_query(vofl_batch* b) {
  if (!b) return VOFL_EINVAL;
  const cudaError_t e = cudaStreamQuery(b->stream);
  if (e == cudaSuccess) return 1;
  if (e == cudaErrorNotReady) {
    cudaGetLastError();
    return 0;
  }
  return bcuda(b, e, "cudaStreamQuery");
}

int64_t vofl_batch_kernels_per_step(vofl_batch* b) {
  if (!b) return VOFL_EINVAL;
  if (b->mem.empty()) return 0;
  if (int st = ensure_graphs(b)) return st;
  return (int64_t)b->kernels_per_step;
}

int vofl_batch_sync(vofl_batch* b) {
  if (!b) return VOFL_EINVAL;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "batch stream");
  for (auto& m : b->mem) {
    int werr = 0;
    e = cudaMemcpy(&werr, m.c->d_step + 1, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, e, "batch error word");
    if (werr) {
      cudaMemset(m.c->d_step + 1, 0, sizeof(int));
      return berr(b, VOFL_ETIMEDOUT, "a device wait gave up (asynchronous copy never completed)");
    }
  }
  return VOFL_OK;
}

int vofl_batch_time(vofl_batch* b, int reps, double* ms_per_step) {
  if (!b || reps < 1 || !ms_per_step) return berr(b, VOFL_EINVAL, "bad batch, reps or output");
  *ms_per_step = 0;
  if (b->mem.empty()) return VOFL_OK;
  Snapshot snap;
  if (int st = snap.take(b)) return st;
  drop_bgraphs(b);
  int st = time_schedule(b, reps, ms_per_step);
  drop_bgraphs(b);
  snap.restore(b);
  return st;
}

int vofl_batch_tune(vofl_batch* b, int reps, double* ms_per_step) {
  if (!b || reps < 1) return berr(b, VOFL_EINVAL, "bad batch or reps");
  if (b->mem.empty()) return VOFL_OK;
  Snapshot snap;
  if (int st = snap.take(b)) return st;
  int st = plan(b);
  double best = 1e300;
  auto trial = [&](double* ms) -> int {
    drop_bgraphs(b);
    return time_schedule(b, reps, ms);
  };
  if (!st) st = trial(&best);
  // coordinate search: each class's chunk, then the branch layout
  for (size_t ci = 0; !st && ci < b->classes.size(); ++ci) {
    const int n = b->classes[ci].n, count = b->classes[ci].count;
    int keep = b->chunk.count(n) ? b->chunk[n] : 0;
    for (int w : {1, 2, 4, 8, 16}) {
      if (w >= count) break;
      b->chunk[n] = w;
      double ms;
      if ((st = trial(&ms))) break;
      if (ms < best) {
        best = ms;
        keep = w;
      }
    }
    b->chunk[n] = keep;
  }
  if (!st && b->classes.size() > 1) {
    b->parallel = !b->parallel;
    double ms;
    st = trial(&ms);
    if (!st && ms < best)
      best = ms;
    else
      b->parallel = !b->parallel;
  }
  drop_bgraphs(b);
  snap.restore(b);
  if (st) return st;
  if (ms_per_step) *ms_per_step = best;
  return VOFL_OK;
}

int vofl_batch_tune_transform(vofl_batch* b, int reps, double* ms_per_step) {
  if (!b || reps < 1) return berr(b, VOFL_EINVAL, "bad batch or reps");
  if (b->mem.empty()) return VOFL_OK;
  Snapshot snap;
  if (int st = snap.take(b)) return st;
  int st = plan(b);
  double best = 1e300;
  auto trial = [&](double* ms) -> int {
    drop_bgraphs(b);
    return time_schedule(b, reps, ms);
  };
  if (!st) st = trial(&best);
  // coordinate search, size by size: line transforms of each pass, column
  // runs, terms per group (never above the members' own: their buffers
  // hold that many), runs per row
  for (size_t ci = 0; !st && ci < b->classes.size(); ++ci) {
    const int n = b->classes[ci].n;
    const BKernels k = b->classes[ci].k;  // a copy: every trial re-plans the classes
    TSched cur = b->tsched[n];
    const int gmax = cur.G;
    auto attempt = [&](TSched t) {
      if (st || t == cur) return;
      b->tsched[n] = t;
      for (auto& cl : b->classes) cl.ts = b->tsched[cl.n];
      double ms;
      if ((st = trial(&ms))) return;
      if (ms < best) {
        best = ms;
        cur = t;
      }
      b->tsched[n] = cur;
      for (auto& cl : b->classes) cl.ts = b->tsched[cl.n];
    };
    if (k.ic_w) { TSched t = cur; t.wc = !t.wc; attempt(t); }
    if (k.ir_w) { TSched t = cur; t.wr = !t.wr; if (!t.wr && W_IROWS % t.rs) t.rs = 1; attempt(t); }
    if (k.fr_w) { TSched t = cur; t.wf = !t.wf; attempt(t); }
    for (int parts : {1, 2, 3, 6}) { TSched t = cur; t.parts = parts; t.pack = 0; attempt(t); }
    const int sms = device_sm_count();
    for (int pk : {0, sms, 2 * sms}) { TSched t = cur; t.pack = pk; attempt(t); }
    for (int G : {17, 9, 6}) if (G <= gmax) { TSched t = cur; t.G = G; attempt(t); }
    if (!cur.wr)
      for (int rs : {1, 2, 4}) { TSched t = cur; t.rs = rs; attempt(t); }
  }
  // then the launch layout, as vofl_batch_tune
  for (size_t ci = 0; !st && ci < b->classes.size(); ++ci) {
    const int n = b->classes[ci].n, count = b->classes[ci].count;
    int keep = b->chunk.count(n) ? b->chunk[n] : 0;
    for (int w : {1, 2, 4, 8, 16}) {
      if (w >= count) break;
      b->chunk[n] = w;
      double ms;
      if ((st = trial(&ms))) break;
      if (ms < best) {
        best = ms;
        keep = w;
      }
    }
    b->chunk[n] = keep;
  }
  drop_bgraphs(b);
  snap.restore(b);
  if (st) return st;
  // the members take their size's schedule (a member stepped alone later
  // keeps the arithmetic it had in the batch)
  for (auto& m : b->mem) {
    const vofl_schedule v = schedule_of(b->tsched[(int)m.c->n[0]]);
    if (int e = m.c->eng->set_schedule(m.c, &v)) return berr(b, e, "member schedule");
    for (auto& g : m.c->step_graph) {  // captured with the old schedule
      if (g) cudaGraphExecDestroy(g);
      g = nullptr;
    }
  }
  if (ms_per_step) *ms_per_step = best;
  return VOFL_OK;
}

int vofl_batch_get_transform(const vofl_batch* b, int n, vofl_schedule* out) {
  if (!b || !out) return VOFL_EINVAL;
  auto it = b->tsched.find(n);
  if (it == b->tsched.end()) return VOFL_EINVAL;
  *out = schedule_of(it->second);
  return VOFL_OK;
}

int vofl_batch_get_schedule(const vofl_batch* b, int* parallel, int* sizes, int* chunks, int cap) {
  if (!b || !parallel) return VOFL_EINVAL;
  *parallel = b->parallel ? 1 : 0;
  int k = 0;
  for (auto& kv : b->chunk) {
    if (k < cap && sizes && chunks) {
      sizes[k] = kv.first;
      chunks[k] = kv.second;
    }
    ++k;
  }
  return k;
}

int vofl_batch_set_schedule(vofl_batch* b, int parallel, const int* sizes, const int* chunks, int n) {
  if (!b || n < 0 || (n > 0 && (!sizes || !chunks))) return VOFL_EINVAL;
  b->parallel = parallel != 0;
  b->chunk.clear();
  for (int i = 0; i < n; ++i) b->chunk[sizes[i]] = chunks[i];
  drop_bgraphs(b);
  return VOFL_OK;
}

}  // extern "C"
