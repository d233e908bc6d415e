// C ABI of the FE-P3M library: argument checking, memory ownership, host/device
// staging and the order of the stages of Algorithm 1.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

using namespace fep3m;

namespace fep3m {
std::atomic<unsigned long long> g_kernel_launches{0};
thread_local bool t_uncounted = false;
}

namespace {

constexpr int PT = 256;

int from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return FEP3M_OK;
  if (e == cudaErrorMemoryAllocation) return FEP3M_ENOMEM;
  return FEP3M_ECUDA;
}

#define CK(x)                          \
  do {                                 \
    cudaError_t e_ = (x);              \
    if (e_ != cudaSuccess) {           \
      (void)cudaGetLastError();        \
      return from_cuda(e_);            \
    }                                  \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, count * sizeof(T));
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

template <class A>
__global__ void k_to_double(int64_t n, const A* in, double* out, double a) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (double)in[i] * a;
}
// the mixed periodic solver's float pairs (h, l) to FP64: out = (h + l) a
__global__ void k_pairs_to_double(int64_t n, const float2* __restrict__ in, double* __restrict__ out, double a) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = ((double)in[i].x + (double)in[i].y) * a;
}
// FP64 to float pairs: h = fl32(v), l = fl32(v - h)
__global__ void k_double_to_pairs(int64_t n, const double* __restrict__ in, float2* __restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = in[i];
  const float h = (float)v;
  out[i] = make_float2(h, (float)(v - (double)h));
}
// flag (1) when any of the n values is not finite
__global__ void k_check_finite(int64_t n, const double* __restrict__ v, int* __restrict__ flag) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && !isfinite(v[i])) atomicOr(flag, 1);
}
// sum Q and sum |Q| (the neutrality check): per-block partials, the last
// block to finish adds them in block order (deterministic)
__global__ void k_charge_sums(int64_t N, const double* __restrict__ Q, double* __restrict__ partials,
                              unsigned int* __restrict__ counter, double* __restrict__ out) {
  __shared__ double s1[PT], s2[PT];
  __shared__ bool last;
  double a = 0, b = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    a += Q[i];
    b += fabs(Q[i]);
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int o = PT / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s1[0];
    partials[2 * blockIdx.x + 1] = s2[0];
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double t1 = 0, t2 = 0;
    for (unsigned k = 0; k < gridDim.x; ++k) {
      t1 += ((volatile double*)partials)[2 * k];
      t2 += ((volatile double*)partials)[2 * k + 1];
    }
    out[0] = t1;
    out[1] = t2;
    *counter = 0u;
  }
}

inline int gsz(int64_t n) { return (int)((n + PT - 1) / PT); }

void free_particles(fep3m_ctx* c) {
  void* p[] = {c->pos_in, c->Q_in, c->cell, c->delta, c->perm, c->ecoord, c->part, c->phi_s, c->E_s, c->w_s,
               c->psi_s, c->gpsi_s, c->out_tmp, c->Q_s, c->gphi_dev, c->w_s32};
  for (void* q : p) dfree(q);
  c->pos_in = c->Q_in = c->delta = c->phi_s = c->E_s = c->w_s = c->psi_s = c->gpsi_s = c->out_tmp = c->Q_s =
      c->gphi_dev = nullptr;
  c->cell = c->perm = c->ecoord = nullptr;
  c->part = nullptr;
  c->w_s32 = nullptr;
  c->cap = 0;
}

int grow_particles(fep3m_ctx* c, int64_t N) {
  if (N <= c->cap) return FEP3M_OK;
  free_particles(c);
  const size_t es = c->precision == FEP3M_MIXED ? sizeof(float4) : sizeof(vec4<double>::type);
  CK(dalloc(&c->pos_in, 3 * N));
  CK(dalloc(&c->Q_in, N));
  CK(dalloc(&c->cell, N));
  CK(dalloc(&c->delta, 3 * N));
  CK(dalloc(&c->perm, N));
  CK(dalloc(&c->ecoord, N));
  CK(cudaMalloc(&c->part, N * es));
  CK(dalloc(&c->phi_s, N));
  CK(dalloc(&c->E_s, 3 * N));
  CK(dalloc(&c->w_s, N));
  if (c->precision == FEP3M_MIXED) CK(dalloc(&c->w_s32, N));
  CK(dalloc(&c->psi_s, N));
  CK(dalloc(&c->gpsi_s, 3 * N));
  CK(dalloc(&c->out_tmp, 5 * N));
  CK(dalloc(&c->Q_s, N));
  CK(dalloc(&c->gphi_dev, N));
  c->cap = N;
  return FEP3M_OK;
}

// copy n elements of device data to a caller pointer (host or device)
int deliver(fep3m_ctx* c, void* dst, const void* src, size_t bytes) {
  if (!dst) return FEP3M_OK;
  if (is_device_ptr(dst)) {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream));
  } else {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return FEP3M_OK;
}

void ev_record(fep3m_ctx* c, int k, cudaStream_t s = nullptr) {
  if (c->timing) cudaEventRecord(c->ev[k], s ? s : c->stream);
}
double ev_ms(fep3m_ctx* c, int a, int b) {
  float ms = 0;
  if (cudaEventElapsedTime(&ms, c->ev[a], c->ev[b]) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return ms;
}

// the pair statistics of the last set_particles, once their copy has landed
void take_counts(fep3m_ctx* c) {
  const unsigned long long* n = c->host_cnt;
  c->stats.singular_pairs = (int64_t)n[0];
  c->stats.nonempty_elements = (int64_t)n[1];
  c->stats.max_per_element = (int)n[2];
  c->stats.screen_element_pairs = (int64_t)n[3];
  c->stats.screen_charge_pairs = (int64_t)n[4];
  c->counts_stale = false;
}

void solve_stats(fep3m_ctx* c) {
  const fep3m::Solver& F = c->solv[0];
  c->stats.solve_rhs = 1;
  c->stats.mg_iterations = F.iters;
  c->stats.mg_rel_residual = F.relres;
  c->stats.refine_steps = F.refine_steps;
}

// The forward chain (assembly, mesh solve, pair kernels) on the context's
// highest-priority stream, forked from the caller's stream and joined back to
// it.  The screen contraction and the singular sums need no mesh solution and
// run on the pair stream, concurrently with the solve.  With force_dev, the
// adjoint chain for forces (weights Q/2 need nothing from the forward solve)
// runs concurrently on the auxiliary stream: deposit, adjoint mesh solve,
// vertex adjoint, with the screen and singular adjoint sweeps on a third
// stream; the per-charge assembly joins all chains.  The critical path
// (assembly, then the forward solve) is enqueued first.  Nothing here waits
// for the device once the solvers are calibrated: the replayed solves'
// residuals are checked by solves_missed after the caller's final
// synchronisation.
int run_forward(fep3m_ctx* c, double* phi_dev, int want_grad, double* force_dev, double* U_dev = nullptr) {
  struct Restore {
    fep3m_ctx* c;
    cudaStream_t s;
    ~Restore() { c->stream = s; }
  } restore{c, c->stream};
  const cudaStream_t caller = c->stream;
  CK(cudaEventRecord(c->ev_ffork, caller));
  CK(cudaStreamWaitEvent(c->fwd_stream, c->ev_ffork, 0));
  c->stream = c->fwd_stream;
  fep3m::Solver* F = &c->solv[0];
  fep3m::Solver* A = &c->solv[1];
  F->stream = c->stream;
  CK(cudaMemsetAsync(c->iflags + 2, 0, sizeof(int), c->stream));   // bounded-wait flag of the pair kernels
  // with forces and the paired solve, the adjoint right-hand side is deposited
  // on the auxiliary stream while this one assembles, and one chain of kernels
  // solves both (the adjoint's right-hand side and solution sit one mesh after
  // the forward ones)
  const bool paired = force_dev && fep3m::mesh_solve_paired(F);
  c->paired_last = paired;
  if (force_dev) CK(cudaEventRecord(c->ev_fork, c->stream));
  ev_record(c, 0);
  CK(assemble_forward(c));
  ev_record(c, 1);
  CK(cudaEventRecord(c->ev_pfork, c->stream));
  if (force_dev) {
    CK(cudaStreamWaitEvent(c->aux_stream, c->ev_fork, 0));
    CK(adjoint_pre(c, 1.0, nullptr, c->aux_stream));
    CK(cudaEventRecord(c->ev_fork2, c->aux_stream));
  }
  if (paired) {
    CK(cudaStreamWaitEvent(c->stream, c->ev_fork2, 0));
    CK(mesh_solve_begin2(F, c->b64, c->phi64));
    CK(cudaEventRecord(c->ev_solved, c->stream));
  } else {
    CK(mesh_solve_begin(F, c->b64, c->phi64));
  }
  CK(cudaStreamWaitEvent(c->pair_stream, c->ev_pfork, 0));
  ev_record(c, 8, c->pair_stream);
  CK(pair_screen(c, want_grad, c->pair_stream, force_dev != nullptr));
  ev_record(c, 9, c->pair_stream);
  CK(cudaEventRecord(c->ev_pjoin, c->pair_stream));
  if (force_dev) {
    CK(cudaStreamWaitEvent(c->sweep_stream, c->ev_fork2, 0));
    CK(adjoint_sweeps(c, c->sweep_stream, false));   // singular part: from the screen kernel
    CK(cudaEventRecord(c->ev_join2, c->sweep_stream));
    if (paired) CK(cudaStreamWaitEvent(c->aux_stream, c->ev_solved, 0));
    else CK(mesh_solve_begin(A, c->g64, c->lam64));
  }
  CK(pair_prepare(c));
  ev_record(c, 2);
  CK(cudaStreamWaitEvent(c->stream, c->ev_pjoin, 0));
  ev_record(c, 10);
  CK(pair_eval(c, phi_dev, want_grad));
  ev_record(c, 3);
  if (U_dev) {   // the energy on the pair stream (idle since the screen kernel), beside the force assembly
    CK(cudaEventRecord(c->ev_pfork, c->stream));
    CK(cudaStreamWaitEvent(c->pair_stream, c->ev_pfork, 0));
    CK(energy(c, U_dev, c->pair_stream));
    CK(cudaEventRecord(c->ev_pjoin, c->pair_stream));
  }
  c->have_forward = true;
  c->have_grad = want_grad != 0;
  if (force_dev) {
    CK(adjoint_vertex(c, c->aux_stream));
    CK(cudaEventRecord(c->ev_join, c->aux_stream));
    CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    CK(cudaStreamWaitEvent(c->stream, c->ev_join2, 0));
    CK(adjoint_final(c, 1.0, force_dev, nullptr, -1.0, c->stream));
    ev_record(c, 4);
  }
  if (U_dev) CK(cudaStreamWaitEvent(c->stream, c->ev_pjoin, 0));
  CK(cudaEventRecord(c->ev_fjoin, c->stream));
  CK(cudaStreamWaitEvent(caller, c->ev_fjoin, 0));
  return FEP3M_OK;
}

// after the stream has completed a run_forward: residual checks of its
// replayed solves; true when one missed its tolerance (run_forward again: the
// missed solve re-calibrates with one more refinement sweep)
bool solves_missed(fep3m_ctx* c, bool adjoint) {
  if (adjoint && c->paired_last) return !mesh_solve_check2(&c->solv[0]);
  bool miss = !mesh_solve_check(&c->solv[0]);
  if (adjoint && !mesh_solve_check(&c->solv[1])) miss = true;
  return miss;
}

// status of the last run_forward's solves (after solves_missed)
int solve_status(fep3m_ctx* c, bool adjoint) {
  const fep3m::Solver* F = &c->solv[0];
  const fep3m::Solver* A = &c->solv[1];
  solve_stats(c);
  const bool paired = adjoint && c->paired_last;
  if (paired) c->stats.solve_rhs = 2;
  const double arel = paired ? F->relres2 : A->relres;
  if (adjoint) {
    c->stats.adj_iterations = paired ? F->iters2 : A->iters;
    c->stats.adj_rel_residual = arel;
  }
  const double rtol = c->cfg.mg_rtol > 0 ? c->cfg.mg_rtol : (c->precision == FEP3M_FP64 ? 1e-13 : 1e-10);
  const bool ok = F->relres <= 10 * rtol && (!adjoint || arel <= 10 * rtol);
  return ok ? FEP3M_OK : FEP3M_ENOCONV;
}

// order q >= 2: potentials and energy (no forces in this build)
int compute_orderq(fep3m_ctx* c, double* phi, double* U) {
  const int64_t N = c->N;
  const bool phi_dev = is_device_ptr(phi);
  double* pd = phi_dev ? phi : (phi ? c->out_tmp : nullptr);
  ev_record(c, 0);
  const int st = orderq_compute(c, pd, U ? c->scal + 40 : nullptr);
  ev_record(c, 3);
  if (st != FEP3M_OK && st != FEP3M_ENOCONV) return st;
  if (U) CK(cudaMemcpyAsync(U, c->scal + 40, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->have_forward = true;
  c->have_grad = false;
  c->stats.refine_steps = c->oq->sweeps;
  c->stats.mg_rel_residual = c->oq->relres;
  if (phi && !phi_dev) {
    int s2 = deliver(c, phi, c->out_tmp, N * sizeof(double));
    if (s2 != FEP3M_OK) return s2;
  }
  if (c->timing) c->stats.ms_solve = ev_ms(c, 0, 3);
  return st;
}

// A non-blocking stream `below` priority levels under the device's highest
// (clamped to the device's range).  The forward chain (assembly, mesh solve,
// evaluation: the step's critical path) and the auxiliary chain (the adjoint
// deposit the paired mesh solve waits for, then the vertex adjoint) run at the
// highest level, the short-range kernels one below, the adjoint sweeps (which
// have the whole mesh solve to finish in) at the lowest: the block scheduler
// then starts the critical path's CTAs first as SMs free up, and the other
// chains fill the SMs around its short latency-bound kernels.
cudaError_t create_stream_at(cudaStream_t* s, int below) {
  int least = 0, greatest = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
  if (e != cudaSuccess) return e;
  return cudaStreamCreateWithPriority(s, cudaStreamNonBlocking, std::min(greatest + below, least));
}
constexpr int kPrioForward = 0, kPrioPair = 1, kPrioSweep = 1 << 20;

// the Dirichlet box: potentials and energy
int compute_box(fep3m_ctx* c, double* phi, double* U) {
  const int64_t N = c->N;
  const bool phi_dev = is_device_ptr(phi);
  double* pd = phi_dev ? phi : (phi ? c->out_tmp : nullptr);
  ev_record(c, 0);
  const int st = box_compute(c, pd, U ? c->scal + 40 : nullptr);
  ev_record(c, 3);
  if (st != FEP3M_OK && st != FEP3M_ENOCONV) return st;
  if (U) CK(cudaMemcpyAsync(U, c->scal + 40, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(c->host_err, c->iflags + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (*c->host_err) return FEP3M_ETIMEOUT;
  c->have_forward = true;
  c->have_grad = false;
  c->stats.refine_steps = c->box->sweeps;
  c->stats.mg_rel_residual = c->box->relres;
  if (phi && !phi_dev) {
    int s2 = deliver(c, phi, c->out_tmp, N * sizeof(double));
    if (s2 != FEP3M_OK) return s2;
  }
  if (c->timing) c->stats.ms_solve = ev_ms(c, 0, 3);
  return st;
}

constexpr int kMaxReruns = 3;

}  // namespace

extern "C" {

const char* fep3m_strerror(int s) {
  switch (s) {
    case FEP3M_OK: return "ok";
    case FEP3M_EINVAL: return "invalid argument";
    case FEP3M_ENOTNEUTRAL: return "charges are not neutral (set FEP3M_NEUTRALIZE to add a background)";
    case FEP3M_ENOMEM: return "device allocation failed";
    case FEP3M_ECUDA: return "CUDA runtime error";
    case FEP3M_ENOCONV: return "mesh solve did not reach its tolerance";
    case FEP3M_ESTATE: return "call out of order";
    case FEP3M_ETIMEOUT: return "bounded device wait gave up";
    default: return "unknown status";
  }
}

void fep3m_destroy(fep3m_ctx* c) {
  if (!c) return;
  free_particles(c);
  void* p[] = {c->Hw64, c->count, c->start, c->fill, c->scan_tmp, c->C, c->rv, c->Cv, c->b64, c->phi64,
               c->res64, c->scal, c->iflags, c->phi_hl, c->W_el, c->A_el, c->mu_v, c->Gscr, c->Hb, c->HbA,
               c->Hdf, c->red_tmp, c->red_counter, c->D_adj, c->Ha64, c->H0df, c->Wsum};
  for (void* q : p) dfree(q);
  fep3m::solver_destroy(&c->solv[0]);
  fep3m::solver_destroy(&c->solv[1]);
  fep3m::orderq_destroy(c);
  fep3m::box_destroy(c);
  if (c->host_err) cudaFreeHost(c->host_err);
  if (c->aux_stream) cudaStreamDestroy(c->aux_stream);
  if (c->sweep_stream) cudaStreamDestroy(c->sweep_stream);
  if (c->pair_stream) cudaStreamDestroy(c->pair_stream);
  if (c->fwd_stream) cudaStreamDestroy(c->fwd_stream);
  if (c->ev_ffork) cudaEventDestroy(c->ev_ffork);
  if (c->ev_fjoin) cudaEventDestroy(c->ev_fjoin);
  if (c->ev_solved) cudaEventDestroy(c->ev_solved);
  if (c->ev_pfork) cudaEventDestroy(c->ev_pfork);
  if (c->ev_pjoin) cudaEventDestroy(c->ev_pjoin);
  if (c->ev_pcount) cudaEventDestroy(c->ev_pcount);
  if (c->host_cnt) cudaFreeHost(c->host_cnt);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_fork2) cudaEventDestroy(c->ev_fork2);
  if (c->ev_join2) cudaEventDestroy(c->ev_join2);
  if (c->ev_init)
    for (int k = 0; k < 11; ++k) cudaEventDestroy(c->ev[k]);
  delete c;
}

int fep3m_create(const fep3m_config* cfg, void* stream, fep3m_ctx** out) {
  if (!cfg || !out) return FEP3M_EINVAL;
  *out = nullptr;
  if (!(cfg->L > 0) || !std::isfinite(cfg->L) || cfg->q < 1 || cfg->q > 4 || cfg->n_sr < 1 || cfg->n_sr > 4 ||
      cfg->n_el < 2 * cfg->n_sr + 1 || cfg->n_el > 400 ||
      (cfg->precision != FEP3M_FP64 && cfg->precision != FEP3M_MIXED) || cfg->mg_rtol < 0 || cfg->table_pad < 0 ||
      cfg->table_pad > 8 || ((cfg->flags & FEP3M_ONE_ELEMENT) && cfg->q < 2) ||
      ((cfg->flags & FEP3M_MULTIGRID) && cfg->q > 1) || (long long)(cfg->q + 2) * cfg->n_el > 1024 ||
      ((cfg->flags & (FEP3M_DIRICHLET | FEP3M_NEUMANN)) &&
       (cfg->q != 1 || (cfg->flags & (FEP3M_MULTIGRID | FEP3M_NEUTRALIZE)) != 0)) ||
      ((cfg->flags & FEP3M_DIRICHLET) && (cfg->flags & FEP3M_NEUMANN)))
    return FEP3M_EINVAL;
  fep3m_ctx* c = new (std::nothrow) fep3m_ctx();
  if (!c) return FEP3M_ENOMEM;
  c->cfg = *cfg;
  c->stream = (cudaStream_t)stream;
  cudaGetDevice(&c->device);
  c->n = cfg->n_el;
  c->n_sr = cfg->n_sr;
  c->keep = cfg->n_sr + 1;
  c->noff = 2 * cfg->n_sr + 2;
  c->L = cfg->L;
  c->h = cfg->L / cfg->n_el;
  c->inv_h = cfg->n_el / cfg->L;
  c->precision = cfg->precision;
  std::memset(&c->stats, 0, sizeof(c->stats));
  int st = FEP3M_OK;
  auto fail = [&](int s) {
    fep3m_destroy(c);
    return s;
  };
  make_stencils(c->st);
  if (cfg->q >= 2) {
    // screens of order q >= 2: the binning and bookkeeping buffers here, the
    // rest in orderq_create
    const int64_t ne = (int64_t)c->n * c->n * c->n;
    cudaError_t e = cudaSuccess;
    if ((e = dalloc(&c->count, ne)) != cudaSuccess || (e = dalloc(&c->start, ne + 1)) != cudaSuccess ||
        (e = dalloc(&c->fill, ne)) != cudaSuccess || (e = cudaMalloc(&c->scan_tmp, scan_tmp_bytes(ne))) != cudaSuccess ||
        (e = dalloc(&c->scal, 64)) != cudaSuccess || (e = dalloc(&c->iflags, 16)) != cudaSuccess ||
        (e = dalloc(&c->red_tmp, 1024)) != cudaSuccess || (e = dalloc(&c->red_counter, 1)) != cudaSuccess ||
        (e = cudaMallocHost(&c->host_err, sizeof(int))) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&c->pair_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->ev_pfork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->ev_pjoin, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->ev_pcount, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaMallocHost(&c->host_cnt, 5 * sizeof(unsigned long long))) != cudaSuccess)
      return fail(from_cuda(e));
    cudaMemset(c->red_counter, 0, sizeof(unsigned int));
    cudaMemset(c->iflags, 0, 16 * sizeof(int));
    *c->host_err = 0;
    if ((st = orderq_create(c)) != FEP3M_OK) return fail(st);
    for (int k = 0; k < 11; ++k) cudaEventCreate(&c->ev[k]);
    c->ev_init = true;
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(from_cuda(e));
    *out = c;
    return FEP3M_OK;
  }
  // box (Dirichlet or Neumann data): the order-1 kernels run on a periodic grid
  // of n_el + n_sr elements per axis (period L (n_el + n_sr) / n_el), the box
  // in its first n_el
  const bool box = (cfg->flags & (FEP3M_DIRICHLET | FEP3M_NEUMANN)) != 0;
  if (box) {
    c->n = cfg->n_el + cfg->n_sr;
    c->L = c->n * c->h;
  }
  // FE basis-screen table and its [vertex offset][node] layout for the kernels
  build_table(c->n_sr, cfg->table_pad > 0 ? cfg->table_pad : 4, c->table_host);
  const int keep = c->keep, noff = c->noff, sk = 6 * keep + 1;
  std::vector<double> Hw((size_t)noff * noff * noff * 64);
  for (int oz = 0; oz < noff; ++oz)
    for (int oy = 0; oy < noff; ++oy)
      for (int ox = 0; ox < noff; ++ox)
        for (int m = 0; m < 64; ++m) {
          const int mx = m & 3, my = (m >> 2) & 3, mz = m >> 4;
          const size_t o = ox + (size_t)noff * (oy + (size_t)noff * oz);
          Hw[o * 64 + m] = c->table_host[(3 * ox + mx) + (size_t)sk * ((3 * oy + my) + (size_t)sk * (3 * oz + mz))];
        }
  // MIXED: the FP32 contractions take the tables in relative form (the screen
  // field's relative to each element's corners, the adjoint's to node 0), so
  // their FP32 sums carry no large smooth part (pair_relative_table)
  std::vector<double> Hrel(Hw.size()), Hd(Hw.size());
  std::vector<float> H0((size_t)noff * noff * noff * 2);
  if (c->precision == FEP3M_MIXED) {
    pair_relative_table(c->n_sr, Hw.data(), Hrel.data());
    pair_adjoint_table(c->n_sr, Hw.data(), Hd.data(), H0.data());
  } else {
    Hrel = Hw;
  }
  if ((st = from_cuda(dalloc(&c->Hw64, Hw.size()))) != FEP3M_OK) return fail(st);
  cudaMemcpy(c->Hw64, Hw.data(), Hw.size() * 8, cudaMemcpyHostToDevice);
  if (c->precision == FEP3M_FP64 || (cfg->flags & FEP3M_CUDA_CORES)) {
    // hi = fl32(H), lo = fl32(H - hi): the operand pairs of the double-float
    // screen contraction on the CUDA cores (MIXED: of the relative table)
    std::vector<float> hdf(2 * Hrel.size());
    for (size_t i = 0; i < Hrel.size(); ++i) {
      hdf[2 * i] = (float)Hrel[i];
      hdf[2 * i + 1] = (float)(Hrel[i] - (double)hdf[2 * i]);
    }
    if ((st = from_cuda(cudaMalloc(&c->Hdf, hdf.size() * 4))) != FEP3M_OK) return fail(st);
    cudaMemcpy(c->Hdf, hdf.data(), hdf.size() * 4, cudaMemcpyHostToDevice);
  }
  if (c->precision == FEP3M_MIXED) {
    if ((st = from_cuda(dalloc(&c->Ha64, Hd.size()))) != FEP3M_OK) return fail(st);
    cudaMemcpy(c->Ha64, Hd.data(), Hd.size() * 8, cudaMemcpyHostToDevice);
    if ((st = from_cuda(cudaMalloc(&c->H0df, H0.size() * 4))) != FEP3M_OK) return fail(st);
    cudaMemcpy(c->H0df, H0.data(), H0.size() * 4, cudaMemcpyHostToDevice);
  }
  if (c->precision == FEP3M_MIXED && !(cfg->flags & FEP3M_CUDA_CORES)) {
    // bf16 pieces of the table for the tensor-core screen contraction
    std::vector<uint16_t> hb(pair_tc_table_bytes(c->n_sr) / 2);
    pair_tc_table(c->n_sr, Hrel.data(), hb.data());
    if ((st = from_cuda(cudaMalloc(&c->Hb, hb.size() * 2))) != FEP3M_OK) return fail(st);
    cudaMemcpy(c->Hb, hb.data(), hb.size() * 2, cudaMemcpyHostToDevice);
    std::vector<uint16_t> ha(pair_adj_table_bytes(c->n_sr) / 2);
    pair_adj_table(c->n_sr, Hd.data(), ha.data());
    if ((st = from_cuda(cudaMalloc(&c->HbA, ha.size() * 2))) != FEP3M_OK) return fail(st);
    cudaMemcpy(c->HbA, ha.data(), ha.size() * 2, cudaMemcpyHostToDevice);
    if ((st = from_cuda(tc_rows_prepare(128))) != FEP3M_OK) return fail(st);
  }
  if ((st = from_cuda(cudaMallocHost(&c->host_err, sizeof(int)))) != FEP3M_OK) return fail(st);
  *c->host_err = 0;
  const int64_t ne = (int64_t)c->n * c->n * c->n, nodes = 27 * ne;
  const size_t es = c->precision == FEP3M_MIXED ? 4 : 8;
  cudaError_t e = cudaSuccess;
  if ((e = dalloc(&c->count, ne)) != cudaSuccess || (e = dalloc(&c->start, ne + 1)) != cudaSuccess ||
      (e = dalloc(&c->fill, ne)) != cudaSuccess ||
      (e = cudaMalloc(&c->scan_tmp, scan_tmp_bytes(ne))) != cudaSuccess ||
      (e = cudaMalloc(&c->C, ne * 8 * es)) != cudaSuccess || (e = cudaMalloc(&c->rv, ne * es)) != cudaSuccess ||
      (e = cudaMalloc(&c->Cv, ne * 8 * es)) != cudaSuccess ||
      (e = dalloc(&c->b64, 2 * nodes)) != cudaSuccess || (e = dalloc(&c->phi64, 2 * nodes)) != cudaSuccess ||
      (e = dalloc(&c->res64, nodes)) != cudaSuccess || (e = dalloc(&c->scal, 64)) != cudaSuccess ||
      (e = dalloc(&c->iflags, 16)) != cudaSuccess || (e = cudaMalloc(&c->W_el, ne * 64 * es)) != cudaSuccess ||
      (e = cudaMalloc(&c->A_el, ne * 8 * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&c->mu_v, ne * sizeof(double))) != cudaSuccess ||
      (e = dalloc(&c->red_tmp, 1024)) != cudaSuccess || (e = dalloc(&c->red_counter, 1)) != cudaSuccess ||
      (e = cudaMalloc(&c->Gscr, pair_screen_bytes(c))) != cudaSuccess)
    return fail(from_cuda(e));
  // the adjoint's right-hand side and solution follow the forward ones: the
  // paired mesh solve takes both at one stride
  c->g64 = c->b64 + nodes;
  c->lam64 = c->phi64 + nodes;
  // MIXED: the element weight sums; a box's hi + lo copy of its FP64 mesh potential (the periodic
  // solver's output is float pairs already)
  if (c->precision == FEP3M_MIXED &&
      ((box && (e = cudaMalloc(&c->phi_hl, nodes * 2 * sizeof(float))) != cudaSuccess) ||
       (e = cudaMalloc(&c->Wsum, ne * sizeof(float2))) != cudaSuccess))
    return fail(from_cuda(e));
  cudaMemset(c->red_counter, 0, sizeof(unsigned int));
  cudaMemset(c->iflags, 0, 16 * sizeof(int));
  if ((e = create_stream_at(&c->aux_stream, kPrioForward)) != cudaSuccess ||
      (e = create_stream_at(&c->sweep_stream, kPrioSweep)) != cudaSuccess ||
      (e = create_stream_at(&c->pair_stream, kPrioPair)) != cudaSuccess ||
      (e = create_stream_at(&c->fwd_stream, kPrioForward)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_ffork, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_fjoin, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_solved, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_pfork, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_pjoin, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_pcount, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaMallocHost(&c->host_cnt, 5 * sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_fork2, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming)) != cudaSuccess)
    return fail(from_cuda(e));
  if (box) {
    if ((st = box_create(c, cfg->n_el, (cfg->flags & FEP3M_NEUMANN) != 0)) != FEP3M_OK) return fail(st);
  } else {
    // the forward solver also pairs the forward and adjoint right-hand sides (tensor-core
    // fast diagonalisation); the second solver serves the multigrid path and fep3m_vjp
    const bool pairable = !(cfg->flags & (FEP3M_MULTIGRID | FEP3M_CUDA_CORES));
    if ((e = solver_init(&c->solv[0], c, c->stream, pairable ? 2 : 1)) != cudaSuccess) return fail(from_cuda(e));
    if ((e = solver_init(&c->solv[1], c, c->aux_stream)) != cudaSuccess) return fail(from_cuda(e));
    c->stats.mg_levels = (int)c->solv[0].mg.lv.size();
  }
  for (int k = 0; k < 11; ++k) cudaEventCreate(&c->ev[k]);
  c->ev_init = true;
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(from_cuda(e));
  *out = c;
  return FEP3M_OK;
}

int fep3m_set_particles(fep3m_ctx* c, int64_t N, const double* pos, const double* Q) {
  if (!c || !pos || !Q || N < 1 || N > ((int64_t)1 << 31) - 1) return FEP3M_EINVAL;
  int st = grow_particles(c, N);
  if (st != FEP3M_OK) return st;
  c->N = N;
  c->stats.n_particles = N;
  const double* dpos = pos;
  const double* dQ = Q;
  if (!is_device_ptr(pos)) {
    CK(cudaMemcpyAsync(c->pos_in, pos, 3 * N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    dpos = c->pos_in;
  }
  if (!is_device_ptr(Q)) {
    CK(cudaMemcpyAsync(c->Q_in, Q, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    dQ = c->Q_in;
  }
  ev_record(c, 6);
  // the previous call's pair counts read the element counts this call rewrites
  CK(cudaStreamWaitEvent(c->stream, c->ev_pcount, 0));
  CK(cudaMemsetAsync(c->iflags, 0, sizeof(int), c->stream));
  // the charge sums of the neutrality check on the pair stream, beside the binning (the sorted
  // charges come from the binning's gather)
  CK(cudaEventRecord(c->ev_pfork, c->stream));
  CK(cudaStreamWaitEvent(c->pair_stream, c->ev_pfork, 0));
  FEP3M_CL k_charge_sums<<<(unsigned)std::min<int64_t>(std::max<int64_t>(gsz(N) / 4, 1), 256), PT, 0,
                           c->pair_stream>>>(N, dQ, (double*)c->red_tmp, c->red_counter, c->scal + 32);
  CK(cudaEventRecord(c->ev_pjoin, c->pair_stream));
  CK(bin_particles(c, dpos, dQ, c->precision == FEP3M_MIXED));
  CK(cudaStreamWaitEvent(c->stream, c->ev_pjoin, 0));
  ev_record(c, 7);
  c->counts_stale = true;   // pair statistics: counted when fep3m_get_stats asks for them
  double sums[2];
  int flag = 0;
  CK(cudaMemcpyAsync(sums, c->scal + 32, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&flag, c->iflags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->have_particles = false;
  c->have_forward = false;
  if (flag) return FEP3M_EINVAL;
  if (!c->box && !(c->cfg.flags & FEP3M_NEUTRALIZE) && std::fabs(sums[0]) > 1e-12 * sums[1])
    return FEP3M_ENOTNEUTRAL;
  c->have_particles = true;
  if (c->timing) c->stats.ms_bin = ev_ms(c, 6, 7);
  return FEP3M_OK;
}


int fep3m_compute(fep3m_ctx* c, double* phi, double* U, double* force) {
  if (!c) return FEP3M_EINVAL;
  if (!c->have_particles) return FEP3M_ESTATE;
  if (c->oq) return force ? FEP3M_EINVAL : compute_orderq(c, phi, U);
  if (c->box) return force ? FEP3M_EINVAL : compute_box(c, phi, U);
  const int64_t N = c->N;
  const bool phi_dev = is_device_ptr(phi);
  const bool fdev = force && is_device_ptr(force);
  double* fdst = force ? (fdev ? force : c->out_tmp + N) : nullptr;
  for (int attempt = 0;; ++attempt) {
    int st = run_forward(c, phi_dev ? phi : (phi ? c->out_tmp : nullptr), force != nullptr, fdst,
                         U ? c->scal + 40 : nullptr);
    if (st != FEP3M_OK) return st;
    if (U) CK(cudaMemcpyAsync(U, c->scal + 40, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(c->host_err, c->iflags + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (*c->host_err) return FEP3M_ETIMEOUT;
    if (!solves_missed(c, force != nullptr) || attempt == kMaxReruns) break;
  }
  const int st = solve_status(c, force != nullptr);
  if (phi && !phi_dev) {
    int s2 = deliver(c, phi, c->out_tmp, N * sizeof(double));
    if (s2 != FEP3M_OK) return s2;
  }
  if (force && !fdev) {
    int s2 = deliver(c, force, fdst, 3 * N * sizeof(double));
    if (s2 != FEP3M_OK) return s2;
  }
  CK(cudaStreamSynchronize(c->stream));
  if (c->timing) {
    c->stats.ms_assemble = ev_ms(c, 0, 1);
    c->stats.ms_solve = ev_ms(c, 1, 2);
    c->stats.ms_pair_screen = ev_ms(c, 8, 9);
    c->stats.ms_pair_eval = ev_ms(c, 10, 3);
    c->stats.ms_pair = c->stats.ms_pair_screen + c->stats.ms_pair_eval;
    c->stats.ms_adjoint = force ? ev_ms(c, 3, 4) : 0.0;
    float ms = 0;
    const fep3m::Solver& F = c->solv[0];
    c->stats.ms_inner_solve = ((F.solve_exec || F.solve2_exec) && cudaEventElapsedTime(&ms, F.ev_in0, F.ev_in1) == cudaSuccess)
                                  ? (double)ms
                                  : 0.0;
    (void)cudaGetLastError();
  }
  return st;
}

int fep3m_vjp(fep3m_ctx* c, double gU, const double* gphi, double* dpos, double* dQ) {
  if (!c || !std::isfinite(gU) || c->oq || c->box) return FEP3M_EINVAL;
  if (!c->have_particles) return FEP3M_ESTATE;
  const int64_t N = c->N;
  if (!c->have_forward || !c->have_grad) {
    for (int attempt = 0;; ++attempt) {
      int st = run_forward(c, nullptr, 1, nullptr);
      if (st != FEP3M_OK) return st;
      CK(cudaMemcpyAsync(c->host_err, c->iflags + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      if (*c->host_err) return FEP3M_ETIMEOUT;
      if (!solves_missed(c, false) || attempt == kMaxReruns) break;
    }
    solve_status(c, false);
  }
  const double* g = gphi;
  if (gphi && !is_device_ptr(gphi)) {
    CK(cudaMemcpyAsync(c->gphi_dev, gphi, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    g = c->gphi_dev;
  }
  const bool pdev = is_device_ptr(dpos), qdev = is_device_ptr(dQ);
  double* dp = dpos ? (pdev ? dpos : c->out_tmp + N) : nullptr;
  double* dq = dQ ? (qdev ? dQ : c->out_tmp + 4 * N) : nullptr;
  CK(cudaEventRecord(c->ev_fork, c->stream));
  CK(cudaStreamWaitEvent(c->aux_stream, c->ev_fork, 0));
  CK(adjoint_pre(c, gU, g, c->aux_stream));
  CK(cudaEventRecord(c->ev_fork2, c->aux_stream));
  CK(cudaStreamWaitEvent(c->sweep_stream, c->ev_fork2, 0));
  CK(adjoint_sweeps(c, c->sweep_stream, true));
  CK(cudaEventRecord(c->ev_join2, c->sweep_stream));
  CK(mesh_solve(&c->solv[1], c->g64, c->lam64));
  c->stats.adj_iterations = c->solv[1].iters;
  c->stats.adj_rel_residual = c->solv[1].relres;
  CK(adjoint_vertex(c, c->aux_stream));
  CK(cudaEventRecord(c->ev_join, c->aux_stream));
  CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
  CK(cudaStreamWaitEvent(c->stream, c->ev_join2, 0));
  CK(adjoint_final(c, gU, dp, dq, 1.0, c->stream));
  if (dpos && !pdev) {
    int s = deliver(c, dpos, c->out_tmp + N, 3 * N * sizeof(double));
    if (s != FEP3M_OK) return s;
  }
  if (dQ && !qdev) {
    int s = deliver(c, dQ, c->out_tmp + 4 * N, N * sizeof(double));
    if (s != FEP3M_OK) return s;
  }
  CK(cudaStreamSynchronize(c->stream));
  return FEP3M_OK;
}

int fep3m_get_stats(const fep3m_ctx* c, fep3m_stats* out) {
  if (!c || !out) return FEP3M_EINVAL;
  // the pair statistics of the particles last set, counted on first request (on the pair stream, ordered
  // after the binning); filling them in is not a visible change of the context
  fep3m_ctx* m = const_cast<fep3m_ctx*>(c);
  if (m->counts_stale && m->have_particles) {
    t_uncounted = true;   // bookkeeping, not a launch of the method
    if (cudaEventRecord(m->ev_pfork, m->stream) == cudaSuccess &&
        cudaStreamWaitEvent(m->pair_stream, m->ev_pfork, 0) == cudaSuccess &&
        pair_counts(m, (unsigned long long*)(m->scal + 48), m->pair_stream) == cudaSuccess &&
        cudaMemcpyAsync(m->host_cnt, m->scal + 48, 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                        m->pair_stream) == cudaSuccess &&
        cudaEventRecord(m->ev_pcount, m->pair_stream) == cudaSuccess &&
        cudaEventSynchronize(m->ev_pcount) == cudaSuccess)
      take_counts(m);
    else
      (void)cudaGetLastError();
    t_uncounted = false;
  }
  *out = c->stats;
  out->kernel_launches = (int64_t)g_kernel_launches.load(std::memory_order_relaxed);
  return FEP3M_OK;
}

int fep3m_set_timing(fep3m_ctx* c, int enable) {
  if (!c) return FEP3M_EINVAL;
  c->timing = enable != 0;
  return FEP3M_OK;
}

int fep3m_get_binning(const fep3m_ctx* cc, int32_t* perm, int32_t* count, int32_t* cell, double* delta) {
  fep3m_ctx* c = const_cast<fep3m_ctx*>(cc);
  if (!c) return FEP3M_EINVAL;
  if (!c->have_particles) return FEP3M_ESTATE;
  const int64_t N = c->N, ne = (int64_t)c->n * c->n * c->n;
  int s;
  if ((s = deliver(c, perm, c->perm, N * 4)) != FEP3M_OK) return s;
  if (c->box) {
    // the box's elements out of the padded grid: counts via the box scratch, ids via out_tmp
    const int64_t nb3 = (int64_t)c->box->nb * c->box->nb * c->box->nb;
    int* cnt = (int*)c->box->t[0];
    int* cel = (int*)c->out_tmp;
    CK(box_binning(c, count ? cnt : nullptr, cell ? cel : nullptr));
    if ((s = deliver(c, count, cnt, nb3 * 4)) != FEP3M_OK) return s;
    if ((s = deliver(c, cell, cel, N * 4)) != FEP3M_OK) return s;
  } else {
    if ((s = deliver(c, count, c->count, ne * 4)) != FEP3M_OK) return s;
    if ((s = deliver(c, cell, c->cell, N * 4)) != FEP3M_OK) return s;
  }
  if ((s = deliver(c, delta, c->delta, 3 * N * 8)) != FEP3M_OK) return s;
  CK(cudaStreamSynchronize(c->stream));
  return FEP3M_OK;
}

int fep3m_get_mesh(const fep3m_ctx* cc, double* C, double* b, double* phi_mesh) {
  fep3m_ctx* c = const_cast<fep3m_ctx*>(cc);
  if (!c) return FEP3M_EINVAL;
  if (!c->have_forward) return FEP3M_ESTATE;
  if (c->oq) {
    const fep3m::OrderQ* o = c->oq;
    const int64_t ne = (int64_t)c->n * c->n * c->n, np3 = (int64_t)o->Np * o->Np * o->Np;
    const int Q1 = o->q + 1;
    int s;
    if ((s = deliver(c, C, o->C, ne * Q1 * Q1 * Q1 * 8)) != FEP3M_OK) return s;
    if ((s = deliver(c, b, o->b, np3 * 8)) != FEP3M_OK) return s;
    if (phi_mesh) {
      FEP3M_CL k_to_double<double><<<gsz(np3), PT, 0, c->stream>>>(np3, o->phi, o->t[0], c->inv_h);
      if ((s = deliver(c, phi_mesh, o->t[0], np3 * 8)) != FEP3M_OK) return s;
    }
    CK(cudaStreamSynchronize(c->stream));
    return FEP3M_OK;
  }
  if (c->box) {
    const fep3m::Box* B = c->box;
    const int64_t nn3 = (int64_t)B->Nn * B->Nn * B->Nn, nb3 = (int64_t)B->nb * B->nb * B->nb;
    int s;
    if (C) {
      CK(box_coeffs(c, B->t[0]));   // 8 nb^3 <= Nn^3
      if ((s = deliver(c, C, B->t[0], 8 * nb3 * 8)) != FEP3M_OK) return s;
    }
    if ((s = deliver(c, b, B->b, nn3 * 8)) != FEP3M_OK) return s;
    if (phi_mesh) {
      FEP3M_CL k_to_double<double><<<gsz(nn3), PT, 0, c->stream>>>(nn3, c->phi64, B->t[1], c->inv_h);
      if ((s = deliver(c, phi_mesh, B->t[1], nn3 * 8)) != FEP3M_OK) return s;
    }
    CK(cudaStreamSynchronize(c->stream));
    return FEP3M_OK;
  }
  const int64_t ne = (int64_t)c->n * c->n * c->n, nodes = 27 * ne;
  // staging through res64 (FP64, nodes >= 8 ne since 27 > 8)
  if (C) {
    if (c->precision == FEP3M_MIXED)
      FEP3M_CL k_to_double<float><<<gsz(8 * ne), PT, 0, c->stream>>>(8 * ne, (const float*)c->C, c->res64, 1.0);
    else
      FEP3M_CL k_to_double<double><<<gsz(8 * ne), PT, 0, c->stream>>>(8 * ne, (const double*)c->C, c->res64, 1.0);
    int s = deliver(c, C, c->res64, 8 * ne * 8);
    if (s != FEP3M_OK) return s;
  }
  // MIXED: the mesh vectors are float pairs (the mixed solver's format)
  const bool pairs = c->precision == FEP3M_MIXED;
  if (b) {
    if (pairs) FEP3M_CL k_pairs_to_double<<<gsz(nodes), PT, 0, c->stream>>>(nodes, (const float2*)c->b64, c->res64, 1.0);
    int s = deliver(c, b, pairs ? c->res64 : c->b64, nodes * 8);
    if (s != FEP3M_OK) return s;
  }
  if (phi_mesh) {
    if (pairs)
      FEP3M_CL k_pairs_to_double<<<gsz(nodes), PT, 0, c->stream>>>(nodes, (const float2*)c->phi64, c->res64, c->inv_h);
    else
      FEP3M_CL k_to_double<double><<<gsz(nodes), PT, 0, c->stream>>>(nodes, c->phi64, c->res64, c->inv_h);
    int s = deliver(c, phi_mesh, c->res64, nodes * 8);
    if (s != FEP3M_OK) return s;
  }
  CK(cudaStreamSynchronize(c->stream));
  return FEP3M_OK;
}

int fep3m_solve_mesh(fep3m_ctx* c, const double* b, double* phi) {
  if (!c || !b || !phi) return FEP3M_EINVAL;
  if (c->oq) {
    fep3m::OrderQ* o = c->oq;
    const int64_t np3 = (int64_t)o->Np * o->Np * o->Np;
    CK(cudaMemcpyAsync(o->t[2], b, np3 * 8, is_device_ptr(b) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       c->stream));
    const int st = orderq_solve(c, o->t[2], o->t[3]);
    if (st != FEP3M_OK && st != FEP3M_ENOCONV) return st;
    c->stats.refine_steps = o->sweeps;
    c->stats.mg_rel_residual = o->relres;
    FEP3M_CL k_to_double<double><<<gsz(np3), PT, 0, c->stream>>>(np3, o->t[3], o->t[0], c->inv_h);
    int s = deliver(c, phi, o->t[0], np3 * 8);
    if (s != FEP3M_OK) return s;
    CK(cudaStreamSynchronize(c->stream));
    return st;
  }
  if (c->box) {
    // right-hand side in g64, solution in lam64 (both (3n)^3 >= (3 nb + 1)^3 of the padded grid)
    const fep3m::Box* B = c->box;
    const int64_t nn3 = (int64_t)B->Nn * B->Nn * B->Nn;
    CK(cudaMemcpyAsync(c->g64, b, nn3 * 8, is_device_ptr(b) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       c->stream));
    const int st = box_solve(c, c->g64, c->lam64);
    if (st != FEP3M_OK && st != FEP3M_ENOCONV) return st;
    c->stats.refine_steps = B->sweeps;
    c->stats.mg_rel_residual = B->relres;
    FEP3M_CL k_to_double<double><<<gsz(nn3), PT, 0, c->stream>>>(nn3, c->lam64, c->res64, c->inv_h);
    int s = deliver(c, phi, c->res64, nn3 * 8);
    if (s != FEP3M_OK) return s;
    CK(cudaStreamSynchronize(c->stream));
    return st;
  }
  const int64_t nodes = (int64_t)27 * c->n * c->n * c->n;
  // MIXED: the solver takes and returns float pairs (staged through res64)
  const bool pairs = c->precision == FEP3M_MIXED;
  CK(cudaMemcpyAsync(pairs ? c->res64 : c->g64, b, nodes * 8,
                     is_device_ptr(b) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  if (pairs) FEP3M_CL k_double_to_pairs<<<gsz(nodes), PT, 0, c->stream>>>(nodes, c->res64, (float2*)c->g64);
  c->solv[0].stream = c->stream;
  CK(mesh_solve(&c->solv[0], c->g64, c->lam64));
  solve_stats(c);
  const double rel = c->solv[0].relres;
  if (pairs)
    FEP3M_CL k_pairs_to_double<<<gsz(nodes), PT, 0, c->stream>>>(nodes, (const float2*)c->lam64, c->res64, c->inv_h);
  else
    FEP3M_CL k_to_double<double><<<gsz(nodes), PT, 0, c->stream>>>(nodes, c->lam64, c->res64, c->inv_h);
  int s = deliver(c, phi, c->res64, nodes * 8);
  if (s != FEP3M_OK) return s;
  CK(cudaStreamSynchronize(c->stream));
  if (c->timing) {
    // the first inner solve of the replayed solve, alone on the GPU
    float ms = 0;
    const fep3m::Solver& F = c->solv[0];
    c->stats.ms_inner_solve = ((F.solve_exec || F.solve2_exec) && cudaEventElapsedTime(&ms, F.ev_in0, F.ev_in1) == cudaSuccess)
                                  ? (double)ms
                                  : 0.0;
    (void)cudaGetLastError();
  }
  const double rtol = c->cfg.mg_rtol > 0 ? c->cfg.mg_rtol : (c->precision == FEP3M_FP64 ? 1e-13 : 1e-10);
  return rel <= 10 * rtol ? FEP3M_OK : FEP3M_ENOCONV;
}

int fep3m_mesh_eigenbasis(int n_el, double* lam, double* V) {
  if (n_el < 1 || n_el > 4096 || !lam || !V) return FEP3M_EINVAL;
  fep3m::Stencils st;
  fep3m::make_stencils(st);
  std::vector<double> l, v;
  fep3m::periodic_eigen(n_el, st, l, v);
  std::memcpy(lam, l.data(), l.size() * sizeof(double));
  std::memcpy(V, v.data(), v.size() * sizeof(double));
  return FEP3M_OK;
}

int fep3m_set_boundary(fep3m_ctx* c, const double* g) {
  if (!c || !g || !c->box) return FEP3M_EINVAL;
  const int64_t len = box_data_size(c);
  // staged and checked for finite values before it replaces the data
  double* stage = c->box->gstage;
  CK(cudaMemcpyAsync(stage, g, len * 8, is_device_ptr(g) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     c->stream));
  CK(cudaMemsetAsync(c->iflags + 3, 0, sizeof(int), c->stream));
  FEP3M_CL k_check_finite<<<gsz(len), PT, 0, c->stream>>>(len, stage, c->iflags + 3);
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, c->iflags + 3, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (flag) return FEP3M_EINVAL;
  const int st = box_set_boundary(c, stage);
  c->have_forward = false;
  return st;
}

int fep3m_get_table(const fep3m_ctx* c, double* table) {
  if (!c || !table || c->oq) return FEP3M_EINVAL;
  if (is_device_ptr(table)) {
    CK(cudaMemcpy(table, c->table_host.data(), c->table_host.size() * 8, cudaMemcpyHostToDevice));
  } else {
    std::memcpy(table, c->table_host.data(), c->table_host.size() * 8);
  }
  return FEP3M_OK;
}

}  // extern "C"
