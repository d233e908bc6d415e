// Internal declarations of the FE-P3M library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstddef>
#include <vector>

#include "fep3m.h"

namespace fep3m {

// every kernel launch of the library is prefixed with FEP3M_CL, which counts it
// (relaxed atomic: the allocation-free entry point may run on other host
// threads).  Launches a host thread issues while capturing a graph, or for
// bookkeeping, are not counted (t_uncounted); a replayed graph adds its kernels.
extern std::atomic<unsigned long long> g_kernel_launches;
extern thread_local bool t_uncounted;
inline void count_launches(unsigned long long k = 1) {
  if (!t_uncounted) g_kernel_launches.fetch_add(k, std::memory_order_relaxed);
}
#define FEP3M_CL ::fep3m::count_launches(),

// Programmatic dependent launch (the mesh solve: chains of short
// dependent kernels).  A kernel launched by launch_pdl may be set up while the
// kernel before it on the stream finishes; its first statement must be
// pdl_wait(), which returns once the preceding grid has completed and its
// writes are visible (so the ordering stays transitive along the chain).  No
// kernel triggers its dependents early: measured on the solve, an early
// trigger let waiting CTAs take SM slots from the running grid (slower than
// no programmatic launch at all), while waiting alone was 10 % faster.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
#define PDL_PROLOGUE ::fep3m::pdl_wait();

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  count_launches();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------------------
// Order-3 equispaced Lagrange basis on [0, 1] (nodes 0, 1/3, 2/3, 1): the 1-D
// factors of the order-p = 3 hexahedral FE basis u_m (Sec. 2.2, Eq. evalsmooth).
// ---------------------------------------------------------------------------
template <class T>
__host__ __device__ __forceinline__ void q3_values(T t, T v[4]) {
  const T a = t, b = t - T(1) / T(3), c = t - T(2) / T(3), d = t - T(1);
  v[0] = T(-4.5) * b * c * d;
  v[1] = T(13.5) * a * c * d;
  v[2] = T(-13.5) * a * b * d;
  v[3] = T(4.5) * a * b * c;
}
template <class T>
__host__ __device__ __forceinline__ void q3_derivs(T t, T v[4]) {
  const T a = t, b = t - T(1) / T(3), c = t - T(2) / T(3), d = t - T(1);
  v[0] = T(-4.5) * (c * d + b * d + b * c);
  v[1] = T(13.5) * (c * d + a * d + a * c);
  v[2] = T(-13.5) * (b * d + a * d + a * b);
  v[3] = T(4.5) * (b * c + a * c + a * b);
}

template <class T> struct vec4;
template <> struct vec4<double> { typedef double4_32a type; };
template <> struct vec4<float> { typedef float4 type; };

// 1-D periodic 7-tap stencils of the reference (h = 1) order-3 mass and
// stiffness matrices: row of global node g with type tau = g mod 3 has
// coefficients S[tau][j + 3] on node g + j, j = -3..3.
struct Stencils {
  double M[3][7];
  double K[3][7];
  double diagM[3], diagK[3];
  // prolongation coarse (element 2h) -> fine (element h), 1-D: fine node at
  // position s/6 (s = 0..5) of a coarse element takes sum_j P[s][j] x_c[3E + j]
  double P[6][4];
  // mixed mass order-3 rows x order-1 columns, element level: Mpq[k][j]
  double Mpq[4][2];
};

// multigrid level: n elements per axis, N = 3n nodes per axis
struct Level {
  int n = 0, N = 0;
  size_t size = 0;            // N^3
  void* x = nullptr;          // correction (levels >= 1)
  void* b = nullptr;          // right-hand side (levels >= 1)
  void* r = nullptr;          // residual (all but the coarsest)
  void* d = nullptr;          // Chebyshev direction (all but the coarsest)
  void* t1 = nullptr;         // grid-transfer and coarsest-solve scratch
  void* t2 = nullptr;
  void* a = nullptr;          // second Chebyshev iterate (all but the coarsest)
};

struct CoarseSolver {
  int N = 0;                  // nodes per axis on the coarsest level
  float* V32 = nullptr;       // N x N, V[i][k] (row i node, column k mode), M-orthonormal
  float* Dinv32 = nullptr;    // N^3 inverse eigenvalue sums (0 for the constant mode)
  float* VT32 = nullptr;      // V^T (row k mode): the forward transform
};

// Exact FP32 solve of the fine-level system by fast diagonalisation: the
// periodic Q3 operator is K1 (x) M1 (x) M1 + M1 (x) K1 (x) M1 + M1 (x) M1 (x) K1,
// so with V^T K1 V = Lambda, V^T M1 V = I its pseudo-inverse is
// (V (x) V (x) V) (Lambda_i + Lambda_j + Lambda_k)^+ (V (x) V (x) V)^T.
struct FineFDM {
  int N = 0;                  // nodes per axis (3 n)
  float* V32 = nullptr;       // N x N, V[node][mode]
  float* VT32 = nullptr;      // V^T
  float* lam32 = nullptr;     // N generalized eigenvalues
  int null_mode = -1;         // the constant mode (eigenvalue 0)
  // tensor-core transforms: bf16 pieces of V^T (analysis) and V (synthesis)
  // per column tile of nt modes and chunk of 64 nodes (unset: CUDA cores)
  void* BpF = nullptr;
  void* BpI = nullptr;
  int nt = 0, ntile = 0;
  int* err = nullptr;         // device flag: a bounded wait gave up
};

struct Hierarchy {
  int elem_size = 0;          // 4: the multigrid runs in FP32
  std::vector<Level> lv;
  CoarseSolver coarse;
  FineFDM fdm;                // set when the fine level is solved by fast diagonalisation
  double lmax = 0;            // estimate of lambda_max(D^-1 K)
  int cheb_degree = 4;
};

// One mesh solver instance (the context holds two, so that the forward
// and adjoint mesh solves can run concurrently on different streams).
struct Solver {
  fep3m_config cfg;
  int n = 0, precision = 0;
  Stencils st;
  cudaStream_t stream = nullptr;   // stream the solver's work is issued on
  Hierarchy mg;
  int nv = 1;                      // right-hand sides the refinement buffers hold (2: the paired solve)
  int V = 1;                       // right-hand sides of the solve being issued, at a stride of
  int64_t vs = 0;                  //   vs nodes (0 for one); scalars and partials per vector
  void* sb[6] = {};                // CG vectors r, z, p, q, x, rhs (working precision, fine level)
  size_t sb_bytes = 0;
  double* scal = nullptr;          // device scalars (64)
  double* red_tmp = nullptr;       // reduction partials (1024)
  unsigned int* red_counter = nullptr;
  double* res64 = nullptr;         // refinement: projected b as float pairs (MIXED)
  double* phidf = nullptr;         // refinement: the iterate as float pairs (MIXED)
  // replayed solve: iteration counts calibrated on the first solve, captured as a graph
  int plan_kin = 0, plan_kout = 0;
  cudaGraphExec_t solve_exec = nullptr;
  int solve_graph_kernels = 0;
  cudaStream_t cap_stream = nullptr;
  double* in64 = nullptr;          // solver input / output (fixed addresses for the graph)
  double* out64 = nullptr;
  double* host_res = nullptr;      // pinned: |Pi b|^2 and |r|^2 of a replayed solve
  bool pending = false;            // a replayed solve whose residual is not yet checked
  const double* pend_b = nullptr;
  double* pend_phi = nullptr;
  int iters = 0, refine_steps = 0;
  double relres = 0;
  // recorded around the first inner solve of a replayed solve (events in the graph)
  cudaEvent_t ev_in0 = nullptr, ev_in1 = nullptr;
  // the paired solve: two right-hand sides at b and b + nodes into phi and phi + nodes in one
  // chain of kernels (tensor-core fast diagonalisation only), captured for its fixed pointers
  int plan2_kout = 0;
  cudaGraphExec_t solve2_exec = nullptr;
  int solve2_graph_kernels = 0;
  const double* plan2_b = nullptr;
  double* plan2_phi = nullptr;
  bool pending2 = false;
  int iters2 = 0, refine_steps2 = 0;   // the second right-hand side's counts and residual
  double relres2 = 0;
};

// Screens of order q >= 2 on the order p = q + 2 mesh (orderq.cu).  Per-order
// constants passed to the kernels by value (q <= 4, p <= 6).
struct OQParams {
  int q, p;
  double W[25];         // screen weight polynomials: w_i = sum_l W[i (q+1) + l] (delta / h)^l (times h)
  double Mpq[35];       // element mixed mass int l^p_i l^q_j, (p+1) x (q+1), h = 1
  double bM[6][13];     // 1-D periodic order-p mass row of node type t = g mod p: tap o -> node g + o - p
  double bK[6][13];     // the same for the stiffness
  double wn[6];         // node integrals by type
};

// host-side data of the order-q path (highorder.cpp)
struct OrderQHost {
  int q = 0, p = 0;
  std::vector<double> Me, Ke, Mpq, W, H, lam, V;
};
bool orderq_host(int q, int n, int n_sr, int pad, bool one_element, OrderQHost& h);

struct OrderQ {
  int q = 0, p = 0, Nq = 0, Np = 0, U = 0;
  bool one_element = false;
  OQParams prm;
  double* C = nullptr;        // n^3 (q+1)^3 element-to-point lists (dimensionless)
  double* r = nullptr;        // (q n)^3 nodal screen density
  double* b = nullptr;        // (p n)^3 load vector (element units)
  double* pb = nullptr;       // the load vector less its neutralising background
  double* phi = nullptr;      // (p n)^3 mesh potential (element units)
  double* res = nullptr;      // refinement residual
  double* t[4] = {};          // scratch of the stiffness apply
  float* r32 = nullptr;       // FP32 inner solve: right-hand side, solution, scratch
  float* x32 = nullptr;
  float* w1 = nullptr;
  float* w2 = nullptr;
  double* S = nullptr;        // n^3 (p+1)^3 screen field at each element's order-p nodes
  double* H = nullptr;        // U^3 (p+1)^3 node-regrouped tables
  double* red = nullptr;      // reduction partials
  double* host_red = nullptr; // pinned: one reduction result
  FineFDM fdm;
  int sweeps = 0;
  double relres = 0;
};

// The box [0, L]^3 with Dirichlet data (box.cu): order-3 mesh of nb elements
// per axis, Nn = 3 nb + 1 nodes, the NI = 3 nb - 1 interior ones solved for.
struct BoxBand {
  double bM[3][7];      // 1-D order-3 mass row of node type t = g mod 3: tap o -> node g + o - 3
  double bK[3][7];      // the same for the stiffness (interior rows of the open matrices)
  double dM[2], dK[2];  // diagonals of the open matrices' first and last rows (one element each)
  double Mpq[4][2];     // element mixed mass int l^3_i l^1_j (h = 1)
  double wn[3];         // node integrals by node type t (t = 0: a vertex shared by two elements)
  double wend;          // the node integral of the first and last node
};
// Gauss-Legendre rule on [0, 1] of the Neumann face integrals
constexpr int BOX_NGL = 8;
struct BoxQuad {
  double t[BOX_NGL], w[BOX_NGL];
};
struct Box {
  int nb = 0, Nn = 0, NI = 0;
  bool neumann = false;       // Neumann data (flux) instead of Dirichlet data
  int Ns = 0, off = 0;        // solved nodes per axis and their first index: NI, 1 (Dirichlet) or Nn, 0
  BoxBand band;
  BoxQuad quad;
  double* sface = nullptr;    // Neumann: per face element its 16 face-node loads (6 nb^2 x 16)
  double* g = nullptr;        // Dirichlet: Nn^3 data at the nodes (physical units; boundary nodes read);
                              // Neumann: 6 nb^2 BOX_NGL^2 fluxes at the face quadrature points
  double* gstage = nullptr;   // the same size: new data, checked before they replace g
  double* b = nullptr;        // Nn^3 load vector (element units)
  double* rhs = nullptr;      // Nn^3 Neumann right-hand side: b + s, made compatible
  double* phi = nullptr;      // Nn^3 mesh potential (element units: h Phi^sm)
  double* res = nullptr;      // Nn^3 residual b - K phi (interior rows)
  double* t[4] = {};          // Nn^3 scratch of the stiffness apply and the load passes
  float* r32 = nullptr;       // Ns^3 FP32 inner solve: right-hand side, correction, scratch
  float* x32 = nullptr;
  float* w1 = nullptr;
  float* w2 = nullptr;
  int* bel = nullptr;         // boundary elements (ids in the padded grid)
  int nbel = 0;
  double* red = nullptr;      // reduction partials
  double* host_red = nullptr; // pinned: one reduction result
  FineFDM fdm;                // box eigenbasis of the solved nodes (Dirichlet: no null mode)
  int sweeps = 0;
  double relres = 0;
};

}  // namespace fep3m

struct fep3m_ctx {
  fep3m_config cfg;
  cudaStream_t stream = nullptr;
  int device = 0;
  int n = 0, n_sr = 3, keep = 4, noff = 8;   // noff = 2 n_sr + 2 vertex offsets per axis
  double L = 1, h = 1, inv_h = 1;
  int precision = FEP3M_FP64;
  fep3m::Stencils st;
  // kept FE table (host copy) and its device copy in [offset][node] layout
  std::vector<double> table_host;
  double* Hw64 = nullptr;
  // particles
  int64_t N = 0, cap = 0;
  bool have_particles = false, have_forward = false, have_grad = false;
  double* pos_in = nullptr;      // N*3 (staging for host inputs)
  double* Q_in = nullptr;        // N
  int* cell = nullptr;           // N
  double* delta = nullptr;       // N*3 original order
  int* perm = nullptr;           // N
  int* ecoord = nullptr;         // N sorted: element coords ex | ey << 10 | ez << 20
  int* count = nullptr;          // n^3
  int* start = nullptr;          // n^3 + 1
  int* fill = nullptr;           // n^3
  void* part = nullptr;          // sorted (t, Q): double4 or float4, N
  void* scan_tmp = nullptr;
  size_t scan_tmp_bytes = 0;
  // element / vertex fields
  void* C = nullptr;             // n^3 * 8 (T)
  void* rv = nullptr;            // n^3 vertex density (T)
  void* Cv = nullptr;            // n^3 * 8 (T): C regrouped by vertex, Cv[v][k] = C[v - k][k]
  // fine-level FP64 vectors
  // the periodic mesh vectors hold FP64 values, or in MIXED float pairs h + l
  // (the mixed solver's format, 8 bytes a node as well); a box's are FP64
  double* b64 = nullptr;         // (3n)^3 load vector
  double* phi64 = nullptr;       // (3n)^3 mesh potential, reference units
  double* res64 = nullptr;       // refinement residual
  double* g64 = nullptr;         // adjoint right-hand side (b64 + nodes: one allocation)
  double* lam64 = nullptr;       // adjoint mesh solution (phi64 + nodes)
  double* scal = nullptr;        // device scalars (dots, norms, flags), 64 doubles
  void* phi_hl = nullptr;        // MIXED box: the FP64 mesh potential as hi + lo floats, (3n)^3 float2
  int* iflags = nullptr;         // device int flags: [0] input error, [1] converged, ...
  void* lam_T = nullptr;
  // per-particle outputs, sorted order
  double* phi_s = nullptr;       // N
  double* E_s = nullptr;         // N*3 target-side gradient
  double* w_s = nullptr;         // N adjoint weights
  float* w_s32 = nullptr;        // MIXED: the same in FP32 (the element deposit's input)
  double* psi_s = nullptr;       // N singular adjoint potential
  double* gpsi_s = nullptr;      // N*3
  double* Q_s = nullptr;         // N sorted charges (FP64)
  double* gphi_dev = nullptr;    // N staging for a host gphi
  void* W_el = nullptr;          // n^3 * 64 element deposits (T)
  void* A_el = nullptr;          // n^3 * 8 screen adjoint (FP64)
  void* D_adj = nullptr;         // adjoint table-field GEMM output, chunk of offsets x n^3 (T)
  size_t D_bytes = 0;
  void* mu_v = nullptr;          // n^3 vertex adjoint (FP64)
  void* Gscr = nullptr;          // screen field at each brick element's 64 nodes, bricks * 4096 (T)
  void* Hb = nullptr;            // bf16 pieces of the table for the tensor-core contraction (MIXED)
  void* HbA = nullptr;           // the same for the screen adjoint's contraction (MIXED)
  void* Hdf = nullptr;           // hi + lo float pairs of the table (MIXED: of Hrel), the double-float
                                 // screen contraction on the CUDA cores
  double* Ha64 = nullptr;        // MIXED: the screen adjoint's table relative to node 0 (pair_adjoint_table)
  void* H0df = nullptr;          // MIXED: H(o, 0) per vertex offset as hi + lo floats
  void* Wsum = nullptr;          // MIXED: per element, the sum of the adjoint weights as hi + lo floats
  int* host_err = nullptr;       // pinned: device-side error flags read after a step
  double* red_tmp = nullptr;     // reduction partials (1024)
  unsigned int* red_counter = nullptr;
  double* out_tmp = nullptr;     // N*3 staging for host outputs
  fep3m::Solver solv[2];          // [0] forward mesh solve, [1] adjoint mesh solve
  cudaStream_t aux_stream = nullptr;   // adjoint chain, concurrent with the forward one
  cudaStream_t sweep_stream = nullptr; // adjoint screen and singular sweeps (need no mesh solution)
  cudaStream_t pair_stream = nullptr;  // screen contraction and singular sums (need no mesh solution)
  cudaStream_t fwd_stream = nullptr;   // the forward chain (the step's critical path), highest priority
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_fork2 = nullptr, ev_join2 = nullptr;
  cudaEvent_t ev_ffork = nullptr, ev_fjoin = nullptr;   // the forward chain's fork from and join to stream
  cudaEvent_t ev_solved = nullptr;     // the paired mesh solve has finished
  bool paired_last = false;            // the last forward step paired its two mesh solves
  int adj_planes = 0;                  // offset planes of the screen adjoint's product D per piece (0: unset)
  cudaEvent_t ev_pfork = nullptr, ev_pjoin = nullptr;
  cudaEvent_t ev_pcount = nullptr;          // the pair statistics' copy to host_cnt
  unsigned long long* host_cnt = nullptr;   // pinned: 5 pair statistics of the last set_particles
  bool counts_stale = false;               // the pair statistics predate the particles last set
  fep3m::OrderQ* oq = nullptr;   // screens of order q >= 2 (orderq.cu)
  fep3m::Box* box = nullptr;     // FEP3M_DIRICHLET / FEP3M_NEUMANN (box.cu): n is then nb + n_sr,
                                 // the box elements first on a periodic grid padded with empty ones
  // stats
  fep3m_stats stats;
  bool timing = false;
  cudaEvent_t ev[11];
  bool ev_init = false;
};

namespace fep3m {
// host setup (setup.cpp)
// Raises a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device, calling the runtime only when the limit has to grow (the
// call costs host time on every launch otherwise).  Safe from several threads.
cudaError_t smem_limit(const void* kern, size_t bytes);
void element_matrices_q3(double Me[4][4], double Ke[4][4], double Mpq[4][2]);
void make_stencils(Stencils& st);
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w);
void generalized_eigen(int n, const std::vector<double>& A, const std::vector<double>& B,
                       std::vector<double>& lam, std::vector<double>& V);
void periodic_eigen(int n, const Stencils& st, std::vector<double>& lam, std::vector<double>& V);
void build_table(int n_sr, int pad, std::vector<double>& kept);
double estimate_lmax(const Stencils& st, int n);

// device launches (return cudaGetLastError-style codes)
cudaError_t bin_particles(fep3m_ctx* c, const double* pos, const double* Q, int use_fp32);
// screen lists C and the vertex density (and its by-vertex copy Cv) of the binned charges
cudaError_t element_lists(fep3m_ctx* c);
cudaError_t assemble_forward(fep3m_ctx* c);
// nv: right-hand sides the refinement buffers hold (2 for the paired solve, which
// needs the tensor-core fast diagonalisation; otherwise 1)
cudaError_t solver_init(Solver* s, const fep3m_ctx* c, cudaStream_t stream, int nv = 1);
// fast-diagonalisation solve of a periodic N^3 mesh from its 1-D eigenpairs
// (mesh.cu): device data, x = K^+ b in FP32 (six transform passes; w1, w2 N^3
// scratch), release
// (rhs: right-hand sides per pass the solve will usually take, for the tile shape)
cudaError_t fdm_setup(FineFDM& f, int N, const std::vector<double>& lam, const std::vector<double>& V, int rhs,
                      bool tensor_cores, bool null_mode = true);
// V vectors at a stride of vs values (V = 2 with the tensor-core passes only)
cudaError_t fdm_apply(const FineFDM& f, const float* b, float* x, float* w1, float* w2, cudaStream_t s, int V = 1,
                      int64_t vs = 0);
void fdm_free(FineFDM& f);
void solver_destroy(Solver* s);
size_t scan_tmp_bytes(int64_t n);
// mu = 4 pi (Mpq^T)^(x)3 lam on the vertex grid (FP64; lam in the solver's
// format); work1/2 sized n*(3n)^2
cudaError_t vertex_adjoint(fep3m_ctx* c, const double* lam, void* mu, void* work1, void* work2, cudaStream_t s);
// solve K phi = b (reference units; FP64 in and out, in MIXED float pairs h + l
// in the same 8-byte slots) on the solver's stream; begin
// may return before the solve has finished (a replayed graph), end waits for
// it, checks the residual and re-solves if needed.  Results in s->iters etc.
cudaError_t mesh_solve_begin(Solver* s, const double* b, double* phi);
cudaError_t mesh_solve_end(Solver* s);
// after the caller has synchronised with the replayed solve (and its residual
// copy): true if it met its tolerance; false drops the plan, so that the next
// mesh_solve_begin re-calibrates with one more refinement sweep
bool mesh_solve_check(Solver* s);
cudaError_t mesh_solve(Solver* s, const double* b, double* phi);
// the paired solve (s->nv == 2): K phi = b and K phi' = b' with b' = b + nodes and
// phi' = phi + nodes, one chain of kernels for both.  Calibrates (synchronously,
// one right-hand side at a time) on its first call for a pair of pointers, then
// replays; the second result's counts and residual in s->iters2 etc.
cudaError_t mesh_solve_begin2(Solver* s, const double* b, double* phi);
// as mesh_solve_check, for both right-hand sides of the paired solve
bool mesh_solve_check2(Solver* s);
bool mesh_solve_paired(const Solver* s);   // the solver can pair right-hand sides
cudaError_t pair_counts(fep3m_ctx* c, unsigned long long* dev5, cudaStream_t s);
// short-range part in two launches: the screen contraction and the singular
// sums need only the binned charges and the vertex density, so they run on
// their own stream while the mesh is solved; the evaluation of the mesh
// potential minus the screen field at the targets follows the solve.
size_t pair_screen_bytes(const fep3m_ctx* c);
size_t pair_tc_table_bytes(int n_sr);
void pair_tc_table(int n_sr, const double* Hw, uint16_t* out);
size_t pair_adj_table_bytes(int n_sr);
void pair_adj_table(int n_sr, const double* Hw, uint16_t* out);
// the FP32 path's tables: the screen field's relative to each element's
// corners, the screen adjoint's relative to node 0 (with H(o, 0) as hi + lo
// floats, 2 per offset)
void pair_relative_table(int n_sr, const double* Hw, double* Hrel);
void pair_adjoint_table(int n_sr, const double* Hw, double* Hd, float* H0);
// energy_adjoint: also leave half the singular sums in psi_s / gpsi_s (the
// singular adjoint of the energy's weights Q / 2)
cudaError_t pair_screen(fep3m_ctx* c, int want_grad, cudaStream_t s, bool energy_adjoint);
cudaError_t pair_prepare(fep3m_ctx* c);
// tensor-core row GEMM with transposed output (mesh.cu): out[(i - cb) R + r]
// = sum_{a < K} in[r K + a] B[i][a] for the columns cb <= i < ce; B in split
// bf16 pieces per column tile of nt
cudaError_t tc_rows_prepare(int nt);
cudaError_t tc_rows_gemm(int64_t R, int K, int cb, int ce, int nt, const float* in, const void* Bp, float* out,
                         int* err, cudaStream_t s);
cudaError_t pair_eval(fep3m_ctx* c, double* phi_out, int want_grad);
// adjoint in three parts: weights and deposit (-> g64), the parts that need
// lam (vertex adjoint, screen sweep, singular adjoint), and the per-charge assembly
cudaError_t adjoint_pre(fep3m_ctx* c, double gU, const double* gphi, cudaStream_t s);
cudaError_t adjoint_sweeps(fep3m_ctx* c, cudaStream_t s, bool singular);
cudaError_t adjoint_vertex(fep3m_ctx* c, cudaStream_t s);
cudaError_t adjoint_final(fep3m_ctx* c, double gU, double* dpos, double* dQ, double sign, cudaStream_t s);
// U = 1/2 sum Q phi on stream s (the context's stream when null)
cudaError_t energy(fep3m_ctx* c, double* U_dev, cudaStream_t s = nullptr);
// sum_j w_j / r and sum_j w_j (x_j - x_t) / r^3 over each target's block, j != t
// (sorted order; physical units)
cudaError_t singular_sums(fep3m_ctx* c, const double* w, double* psi, double* gpsi, cudaStream_t s);
// the order-q path (orderq.cu)
int orderq_create(fep3m_ctx* c);
void orderq_destroy(fep3m_ctx* c);
int orderq_compute(fep3m_ctx* c, double* phi_dev, double* U_dev);
int orderq_solve(fep3m_ctx* c, const double* b_dev, double* phi_dev);
// the box (box.cu); n is the padded grid's, nb the box's elements per axis
int box_create(fep3m_ctx* c, int nb, bool neumann);
int64_t box_data_size(const fep3m_ctx* c);
void box_destroy(fep3m_ctx* c);
int box_set_boundary(fep3m_ctx* c, const double* g_dev);
int box_compute(fep3m_ctx* c, double* phi_dev, double* U_dev);
int box_solve(fep3m_ctx* c, double* rhs_dev, double* phi_dev);   // rhs_dev may be overwritten
cudaError_t box_binning(fep3m_ctx* c, int* count_out, int* cell_out);
cudaError_t box_coeffs(fep3m_ctx* c, double* out);
}  // namespace fep3m
