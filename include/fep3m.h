/*
 * fep3m.h -- C ABI of the GB300 (sm_103a) finite-element P3M library.
 *
 * The method (Beams, Olson, Freund, "A Finite Element Based P3M Method for
 * N-body Problems") computes, for N point charges Q_i at x_i in the periodic
 * cube [0, L)^3, the potentials
 *     Phi_i = sum_n sum_{j != i or n != 0} Q_j / |x_i - x_j + n L|       (Eq. potential)
 * and the energy U = 1/2 sum_i Q_i Phi_i (Eq. potentialenergy), split as
 * Phi = Phi^sr + Phi^sm (Eq. phisplit): a polynomial screen of order q = 1
 * (Sec. 2.1, Eq. moment1d) turns the long-range part into a periodic order
 * p = 3 finite-element Poisson problem (Sec. 2.2) solved here by iterative
 * refinement around an exact FP32 fast-diagonalisation solve (or multigrid),
 * evaluated at the charges by Eq. evalsmooth (Sec. 2.3); the short-range
 * part (Sec. 2.4, Eq. sc, self term Sec. 2.5) is a sum over the
 * (2 n_sr + 1)^3 elements around each charge's element using FE basis-screen
 * tables (Remark of Sec. 4).  Forces are -dU/dx of the discrete U, from a
 * hand-written adjoint.
 *
 * Conventions shared by every entry point
 *   - Units: Gaussian, Coulomb constant 1 (Phi = Q / R).
 *   - Return value: FEP3M_OK (0) or a negative FEP3M_E* status; a failing
 *     call leaves caller buffers unspecified but the context usable unless
 *     it returns FEP3M_ECUDA.  fep3m_strerror() names the status.
 *   - Pointers: "host or device" arguments may be either; the library asks
 *     the CUDA runtime which one it is and copies host data through the
 *     context's stream.  Device pointers must be on the context's device.
 *   - Layouts: positions and gradients are N x 3 row-major (x, y, z of
 *     charge i at 3i..3i+2), float64; per-charge arrays are length N, float64,
 *     in the caller's original charge order.
 *   - Ownership: the caller owns every buffer it passes; the library owns all
 *     of its scratch (allocated in fep3m_create / grown in
 *     fep3m_set_particles) and frees it in fep3m_destroy.
 *   - Streams: all device work is ordered on the stream given to
 *     fep3m_create: a call's work starts after the work queued there before
 *     it, and work queued there after the call starts after the call's work.
 *     Inside fep3m_set_particles and fep3m_compute (periodic, q = 1) the
 *     library forks its work onto streams of its own (the forward chain at
 *     the device's highest priority, the short-range kernels one level below,
 *     the adjoint chain and its sweeps) and joins them back to that stream.
 *     Calls returning host values synchronise it.
 *   - A context is not thread-safe; use one per host thread.
 *   - Reproducibility: fep3m_compute and fep3m_vjp are bitwise reproducible
 *     for the same inputs, configuration and GPU model: their only atomics
 *     are on integers (bin counts, pair counts, last-block counters), and
 *     every floating-point sum has a fixed order (the sorted charge order of
 *     fep3m_set_particles is stable by index).  fep3m_load_vector_static
 *     accumulates the vertex density with FP64 atomics and is reproducible
 *     to rounding only.
 */
#ifndef FEP3M_H
#define FEP3M_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  FEP3M_OK = 0,
  FEP3M_EINVAL = -1,       /* bad argument: sizes, q, n_sr, non-finite input  */
  FEP3M_ENOTNEUTRAL = -2,  /* |sum Q| > 1e-12 sum |Q| without FEP3M_NEUTRALIZE */
  FEP3M_ENOMEM = -3,       /* device allocation failed                        */
  FEP3M_ECUDA = -4,        /* CUDA runtime error (context may be unusable)    */
  FEP3M_ENOCONV = -5,      /* mesh solve hit its cycle cap; outputs written   */
  FEP3M_ESTATE = -6,       /* call out of order (e.g. compute before set)     */
  FEP3M_ETIMEOUT = -7      /* a bounded device wait gave up                   */
};

enum { FEP3M_FP64 = 0, FEP3M_MIXED = 1 };

/* flags */
#define FEP3M_NEUTRALIZE 1u    /* accept non-neutral input: uniform background */
#define FEP3M_CUDA_CORES 2u    /* the split-precision contractions (screen field
                                  of the MIXED pair kernel, transforms of the
                                  fast-diagonalisation solve) on the FP32 CUDA
                                  cores instead of the tensor cores             */
#define FEP3M_MULTIGRID 4u     /* inner mesh solver: multigrid-preconditioned CG
                                  instead of the exact fast-diagonalisation
                                  solve (both inside the same refinement; q = 1) */
#define FEP3M_ONE_ELEMENT 8u   /* one-element screens (Sec. 5.3): weights on the
                                  interior nodes of the charge's element only,
                                  the moments l < q - 1; needs q >= 2           */
#define FEP3M_DIRICHLET 16u    /* the box [0, L]^3 with Dirichlet data Phi = g on
                                  its boundary (Sec. "Alternate boundary
                                  conditions", Eq. bcadjust) instead of the
                                  periodic cube: charges must lie in the box,
                                  need not be neutral, and each short-range
                                  block is cut off at the box faces (no
                                  images).  g is set by fep3m_set_boundary
                                  (default 0, a grounded box).  q = 1 only, no
                                  FEP3M_MULTIGRID; potentials and energy
                                  (fep3m_compute with force = NULL; fep3m_vjp
                                  returns FEP3M_EINVAL)                        */
#define FEP3M_NEUMANN 32u      /* the box [0, L]^3 with Neumann data dPhi/dn = g
                                  (outward normal) on its boundary: as
                                  FEP3M_DIRICHLET, with the adjusted flux
                                  g - dPhi^sr/dn entering the mesh problem as a
                                  boundary load (Eq. bcadjust for Neumann
                                  data).  The data fix Phi up to a constant:
                                  the load is made compatible by removing its
                                  component along the node integrals and the
                                  mesh solution has int phi = 0, so Phi and U
                                  carry that convention                         */
#define FEP3M_NEUMANN_NGL 8    /* Gauss-Legendre points per axis of a face
                                  element in the Neumann face integrals        */

typedef struct fep3m_ctx fep3m_ctx;

typedef struct {
  double L;            /* periodic cube edge, > 0                              */
  int n_el;            /* elements per axis; >= 2 n_sr + 1; h = L / n_el        */
  int q;               /* screen order 1..4 (Sec. 2.1), mesh order p = q + 2.
                          q = 1: potentials, energy, forces and the VJP, in
                          both precisions as described below.  q >= 2: the
                          screen basis on Gauss-Lobatto nodes, potentials and
                          energy only (fep3m_compute with force = NULL;
                          fep3m_vjp returns FEP3M_EINVAL), the screen
                          contraction in FP64 in both precisions; p n_el <=
                          1024                                                  */
  int n_sr;            /* short-range block half-width in elements, 1..4 (3 in
                          the paper's tests, Sec. 4: a 7 x 7 x 7 block)         */
  int precision;       /* FEP3M_FP64 or FEP3M_MIXED.  Both solve the mesh
                          system by iterative refinement around an FP32 inner
                          solve (fast diagonalisation on the tensor cores, or
                          with FEP3M_MULTIGRID a multigrid-preconditioned CG);
                          the iterate and residual are FP64 (FP64) or
                          double-float pairs (MIXED: a departure from an FP64
                          refinement residual, for speed -- FP64 issues at
                          1/64 of the FP32 rate on this GPU -- accurate to
                          about 2e-14 relative, far inside the 1e-10 the
                          refinement reaches).  Pair sums run in FP64
                          (FP64) or FP32 (MIXED); the screen contractions in
                          double-float arithmetic on the FP32 pipes (FP64, and
                          MIXED with FEP3M_CUDA_CORES) or as split-precision
                          bf16 tensor-core MMAs against tables relative to
                          each element's corners (MIXED), with the parts that
                          carry an element's potential level in double-float
                          or FP64; projections and the energy reduction in
                          FP64.  Both paths hold charges and
                          screen weights in FP32 ranges somewhere (the FP64
                          path's double-float contractions, whose low words
                          sit 2^-24 below the charges): keep |Q| within
                          about 1e-30 .. 1e30 for full accuracy.               */
  double mg_rtol;      /* relative FE residual target; 0 -> 1e-13 (FP64) or
                          1e-10 (MIXED)                                          */
  int mg_max_cycles;   /* cap on refinement sweeps; 0 -> 10                      */
  int table_pad;       /* Dirichlet box margin, elements, beyond the kept table;
                          0 -> 4 (q = 1) or 2 (q >= 2); at most 8               */
  unsigned flags;      /* FEP3M_NEUTRALIZE, FEP3M_CUDA_CORES, FEP3M_MULTIGRID,
                          FEP3M_ONE_ELEMENT, FEP3M_DIRICHLET or FEP3M_NEUMANN   */
} fep3m_config;

typedef struct {
  int64_t n_particles;
  int mg_levels;
  int mg_iterations;        /* last forward solve: total inner CG iterations     */
  int refine_steps;         /* last forward solve: refinement sweeps              */
  double mg_rel_residual;   /* last forward solve, FP64 residual / |b|            */
  int adj_iterations;       /* last adjoint solve                                 */
  double adj_rel_residual;
  int64_t singular_pairs;   /* ordered (target, source) pairs in the blocks       */
  int64_t nonempty_elements;
  int max_per_element;
  double ms_bin, ms_assemble, ms_solve, ms_pair, ms_adjoint;  /* last call, if
                               timing was enabled with fep3m_set_timing; ms_pair
                               = ms_pair_screen + ms_pair_eval (below)           */
  int64_t kernel_launches;  /* CUDA kernels launched by this library in this
                               process so far (all contexts)                     */
  int64_t screen_element_pairs;  /* (non-empty element, non-empty element of its
                               block) pairs: the units of the element-to-point
                               screen sums of Sec. 3.1.2 per target element      */
  int64_t screen_charge_pairs;   /* (charge, non-empty element of its block) pairs:
                               the same per target charge                        */
  double ms_pair_screen;    /* the screen-contraction and singular-sum launch,
                               which runs on its own stream concurrently with
                               the forward mesh solve                            */
  double ms_pair_eval;      /* the evaluation of the mesh potential minus the
                               screen field at the targets, after the solve      */
  double ms_inner_solve;    /* the first FP32 inner solve of the last replayed
                               forward mesh solve (six transform passes of the
                               fast diagonalisation, or the multigrid-
                               preconditioned CG): inside fep3m_compute, where it
                               shares the GPU with the concurrent streams; after
                               fep3m_solve_mesh, alone                            */
  int solve_rhs;            /* right-hand sides that went through each kernel of
                               the last mesh solve: 2 when fep3m_compute with
                               forces paired the forward and adjoint solves
                               (tensor-core fast diagonalisation), else 1; each
                               transform pass then moves twice the data         */
} fep3m_stats;

/* Create a context: validates cfg, builds the FE basis-screen table (a
 * Dirichlet order-3 FE solve around one vertex hat, Remark of Sec. 4), the
 * mesh solver (the 1-D eigenbasis of the fast-diagonalisation solve and the
 * multigrid hierarchy) and the screen constants (Eq. moment1d).  cuda_stream is a cudaStream_t (NULL = legacy default).
 * On success *out owns everything and must be released by fep3m_destroy.  */
int fep3m_create(const fep3m_config* cfg, void* cuda_stream, fep3m_ctx** out);

/* Charge positions (N x 3, host or device, any real values: they are wrapped
 * into [0, L); in a box (FEP3M_DIRICHLET, FEP3M_NEUMANN) they must lie in [0, L]^3, a charge
 * on the faces x = L belonging to the last element) and charges (N, host or
 * device).  Bins the charges into
 * elements (stable counting sort) and stores the sorted SoA copy; grows the
 * context's scratch when N exceeds earlier calls.  N >= 1.  Returns
 * FEP3M_EINVAL for non-finite input (or, in a box, a charge outside it) and
 * FEP3M_ENOTNEUTRAL for a net charge (periodic cube, unless
 * FEP3M_NEUTRALIZE); either leaves no particles set.  Synchronises
 * the stream.                                                                */
int fep3m_set_particles(fep3m_ctx* ctx, int64_t N, const double* pos, const double* Q);

/* Phi_i (N, host or device; may be NULL) and U (host scalar; may be NULL) for
 * the charges last set.  force (N x 3, host or device, or NULL) receives
 * -dU/dx_i; computing it runs the adjoint (a second mesh right-hand side,
 * which the tensor-core fast-diagonalisation solve takes in the same chain of
 * kernels as the forward one; q = 1 only, FEP3M_EINVAL for q >= 2).
 * Synchronises the stream when U, force-on-host or phi-on-host is asked.   */
int fep3m_compute(fep3m_ctx* ctx, double* phi, double* U, double* force);

/* Vector-Jacobian product of the last fep3m_compute: for the scalar
 *   Lf = gU * U + sum_i gphi_i Phi_i
 * writes dLf/dx (N x 3) into dpos and dLf/dQ (N) into dQ (host or device;
 * either may be NULL).  gphi may be NULL (zero).  The derivative is that of
 * the discrete method (element and block membership held fixed); the mesh
 * part uses the same mesh solver on the adjoint right-hand side.           */
int fep3m_vjp(fep3m_ctx* ctx, double gU, const double* gphi, double* dpos, double* dQ);

/* Counters of the last calls (see fep3m_stats).  The pair statistics
 * (singular_pairs ... screen_charge_pairs) are counted on the first request
 * after fep3m_set_particles, which then synchronises with the device.       */
int fep3m_get_stats(const fep3m_ctx* ctx, fep3m_stats* out);

/* Enable (1) / disable (0) per-stage CUDA-event timing in fep3m_stats.      */
int fep3m_set_timing(fep3m_ctx* ctx, int enable);

/* Inspection of intermediate results of the last set/compute, for testing
 * each stage against a reference.  All outputs host or device, float64
 * unless stated; NULL skips an output.
 *   perm       int32[N]    charge index at each sorted slot (stable by index)
 *   count      int32[n^3]  charges per element, element id ex + n ey + n^2 ez
 *   cell       int32[N]    element id of each charge (original order)
 *   delta      [N x 3]     offset of each charge from its element centre     */
int fep3m_get_binning(const fep3m_ctx* ctx, int32_t* perm, int32_t* count,
                      int32_t* cell, double* delta);

/*   C      [n^3 x 8]  element-to-point screen list sum_{j in e} Q_j c_k(delta_j)
 *                     with c_k the dimensionless (h^3-scaled) weights of
 *                     Eq. oned, k = i + 2 j + 4 k' the corner
 *   b      [(3n)^3]   FE load vector 4 pi int rho u_m (index ix + 3n iy + 9n^2 iz)
 *   phi_mesh [(3n)^3] mesh potential nodal values (physical units, mean zero)
 *   Phi^sm / Phi^sing / Phi^scr parts are not kept separately.
 * For q >= 2: C [n^3 x (q+1)^3] (screen node i + (q+1)(j + (q+1) k)), b and
 * phi_mesh [(p n)^3] on the order-p mesh (index ix + pn iy + (pn)^2 iz).
 * Box (FEP3M_DIRICHLET, FEP3M_NEUMANN): b and phi_mesh on the (3n + 1)^3
 * nodes of the box, index ix + (3n+1) iy + (3n+1)^2 iz, node (ix, iy, iz) at
 * (ix, iy, iz) h / 3; b is the box integral of the screens (the part of a
 * screen outside the box is not a load; the Neumann face load is not
 * included); with Dirichlet data phi_mesh holds the adjusted boundary values
 * g - Phi^sr on the boundary nodes (Eq. bcadjust) and is not shifted, with
 * Neumann data it has int phi = 0.                                           */
int fep3m_get_mesh(const fep3m_ctx* ctx, double* C, double* b, double* phi_mesh);

/* Solve the periodic FE system K phi = b - (sum b) w / sum w, int phi = 0,
 * for a caller right-hand side b ((p n)^3, host or device) with the context's
 * mesh solver (precision as configured); writes phi (physical units).  Used
 * to test the solver alone.  Box: b and phi on the (3n+1)^3 box nodes (as
 * fep3m_get_mesh); FEP3M_DIRICHLET solves K phi = b at the interior nodes
 * with phi = g (fep3m_set_boundary, no adjustment: no charges enter) on the
 * boundary nodes, FEP3M_NEUMANN solves K phi = b - (sum b) w / sum w on all
 * nodes with int phi = 0 (the data of fep3m_set_boundary do not enter).      */
int fep3m_solve_mesh(fep3m_ctx* ctx, const double* b, double* phi);

/* Boundary data of a box (host or device, float64; copied, kept until the
 * next call; initially 0).
 * FEP3M_DIRICHLET: g at the (3n + 1)^3 nodes of the order-3 box mesh (index
 * ix + (3n+1) iy + (3n+1)^2 iz, node (ix, iy, iz) at (ix, iy, iz) h / 3);
 * only the boundary nodes (an index 0 or 3n) are read, and the FE solution
 * takes their values interpolated by the order-3 basis on each face (Sec.
 * "Alternate boundary conditions": the mesh problem's boundary values are g
 * less the short-range potential there, Eq. bcadjust, so that Phi = g at the
 * boundary nodes).
 * FEP3M_NEUMANN: the outward normal derivative g at the face quadrature
 * points, 6 n^2 NGL^2 values (NGL = FEP3M_NEUMANN_NGL) in the order [face]
 * [e1][e2][i][j]: face = 2 a + s for the face x_a = s L (s = 0, 1; outward
 * normal (2 s - 1) along a), e1 and e2 the face element's indices along the
 * axes a + 1 and a + 2 (mod 3), (i, j) the Gauss-Legendre points t_i, t_j of
 * [0, 1] along those axes: point x_a = s L, x_{a+1} = (e1 + t_i) h,
 * x_{a+2} = (e2 + t_j) h.
 * FEP3M_EINVAL for a periodic context or non-finite data (the previous data
 * are then kept).                                                           */
int fep3m_set_boundary(fep3m_ctx* ctx, const double* g);

/* The kept FE basis-screen table (h = 1): nodal values on [-(n_sr+1), n_sr+1]^3
 * in steps of 1/3, (6 n_sr + 7)^3 values, index ix + s iy + s^2 iz with
 * s = 6 n_sr + 7.  q = 1 only (FEP3M_EINVAL otherwise; the order-q tables
 * come from fep3m_screen_type_table).                                        */
int fep3m_get_table(const fep3m_ctx* ctx, double* table);

/* The 1-D eigenbasis of the fast-diagonalisation mesh solve (host only, no
 * context or GPU): the generalized eigenpairs K1 v = lam M1 v of the periodic
 * order-3 stiffness and mass matrices on n_el elements of unit length
 * (N = 3 n_el nodes), M1-orthonormal.  lam: N values; V: N x N host array,
 * V[node * N + mode].  Returns FEP3M_EINVAL for n_el < 1 or n_el > 4096.    */
int fep3m_mesh_eigenbasis(int n_el, double* lam, double* V);

/* Host-only building blocks for screens of order q >= 2 and the order
 * p = q + 2 mesh (Sec. 2: p = q + 2); no context or GPU is involved.
 *
 * fep3m_mesh_eigenbasis_order: as fep3m_mesh_eigenbasis for the periodic
 * order-p matrices (equispaced Lagrange nodes, N = p n_el nodes): lam: N
 * values, V: N x N host array, V[node * N + mode], M1-orthonormal.
 * FEP3M_EINVAL unless 1 <= p <= 8, n_el >= 1 and p n_el <= 8192.
 *
 * fep3m_screen_type_table: the FE table (Remark of Sec. 4) of one basis
 * screen of order q (1 <= q <= 4).  The order-q nodal functions of the screen
 * mesh (Lagrange functions on Gauss-Lobatto-Legendre nodes, which are the
 * equispaced ones for q <= 2) come in q types per axis: type 0, the function
 * of a vertex (support the two elements next to it), and type t = 1 .. q-1,
 * the interior function of an element with its t-th interior node.
 * (tx, ty, tz) picks the product
 * screen; the table is the order-(q+2) Galerkin solution of
 * -Lap H = 4 pi psi (h = 1) on a box reaching n_sr + 1 + pad elements
 * beyond the screen's anchor vertex (the left vertex of the element holding
 * its node) on each side, one element more on the right along interior-type
 * axes, with the continuum potential of psi as Dirichlet data.  kept: host
 * array of K^3 values, K = 2 (n_sr + 1)(q + 2) + 1, the nodal values on
 * [-(n_sr+1), n_sr+1]^3 about the anchor in steps of 1/(q+2), index
 * ix + K iy + K^2 iz.  For q = 1 this is the table of fep3m_get_table.
 * FEP3M_EINVAL for q, n_sr (1..4), pad (1..8) or a type out of range.       */
int fep3m_mesh_eigenbasis_order(int p, int n_el, double* lam, double* V);
int fep3m_screen_type_table(int q, int tx, int ty, int tz, int n_sr, int pad, double* kept);

/* Host only: the table operand of the node-regrouped screen contraction of
 * order q (Sec. 2.4, Eq. sc with the tables of the Remark of Sec. 4), p = q + 2.
 * The screens of a target element's block are the sum over the order-q screen
 * nodes u of the block (U = (2 n_sr + 1) q + 1 per axis, u = -q n_sr ..
 * q (n_sr + 1) in steps of 1/q element from the target element's origin) of
 * the node's weight times the table of its type (u mod q) anchored at
 * floor(u / q).  H: host array of U^3 (q + 3)^3 values, H[o (q+3)^3 + m],
 * o = ox + U (oy + U oz) with o_a = q (n_sr + 1) - u_a, m = mx + (q+3) (my +
 * (q+3) mz) the target element's order-p nodes; the values are those of the
 * type tables (h = 1).  For q = 1 this is the vertex-offset table of the
 * order-1 screen contraction.  FEP3M_EINVAL as fep3m_screen_type_table.     */
int fep3m_screen_node_table(int q, int n_sr, int pad, double* H);

/* Host only: the screen weights of Eq. moment1d as polynomials.  Per axis the
 * weight of local node i (0..q) of the charge's element, offset delta from
 * the element's centre, is w_i = sum_l W[i (q+1) + l] (delta / h)^l / h, with
 * W the inverse of the centred moment matrix of the order-q nodal functions
 * (Gauss-Lobatto nodes; the vertex functions reach into the neighbouring
 * elements).  one_element != 0: the one-element screens (Sec. 5.3), interior
 * nodes only and moments l < q - 1 (needs q >= 2); other entries are zero.
 * W: host array of (q+1)^2 values.  FEP3M_EINVAL for q outside 1..4.        */
int fep3m_screen_weight_poly(int q, int one_element, double* W);

/* Host only: the 1-D eigenbasis of the order-p mesh on a box of n_el
 * elements of unit length (Sec. "Alternate boundary conditions"), for the
 * fast-diagonalisation solve of a box.  dirichlet != 0: the interior nodes,
 * N = p n_el - 1; else (Neumann data) all nodes, N = p n_el + 1, with one
 * zero eigenvalue (the constant).  lam: N values (ascending); V: N x N host
 * array, V[node * N + mode], M1-orthonormal.  FEP3M_EINVAL unless
 * 1 <= p <= 8, n_el >= 1 and p n_el <= 1024.                                */
int fep3m_box_eigenbasis(int p, int n_el, int dirichlet, double* lam, double* V);

/* Load vector without any allocation (the paper has no counterpart; this is a
 * service for callers that cannot allocate device memory: work issued while a
 * stream is being captured into a CUDA graph, applications whose memory
 * manager owns the whole device, loops that cannot afford cudaMalloc's
 * implicit synchronisation).  Computes the same b as fep3m_get_mesh after a
 * compute: b = 4 pi (Mpq (x) Mpq (x) Mpq) r, r the order-1 vertex density of
 * the charges' screens, index ix + 3n iy + 9n^2 iz, without the neutrality
 * projection.  pos (N x 3), Q (N) and b ((3 n_el)^3) must be device (or
 * managed) pointers of the current device, else FEP3M_EINVAL; cuda_stream is a
 * cudaStream_t (NULL = default).  Unlike fep3m_set_particles this call does
 * not check its inputs for finiteness: a non-finite coordinate is taken as 0
 * and a non-finite charge carries into b (the call returns before the device
 * has looked at the data).
 * Scratch is a file-scope device array of FEP3M_STATIC_MAX_NEL^3 doubles
 * (2 MiB) held by every GPU that loads the library until the process exits;
 * n_el > FEP3M_STATIC_MAX_NEL returns FEP3M_EINVAL.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress), so make
 * the first call on each device before any stream capture.  Every call
 * clears and reuses the same array: calls that overlap on the GPU (other
 * streams, other host threads) race and give wrong results.  Accumulation
 * uses atomics, so b may differ from the context path in the last bits.     */
#define FEP3M_STATIC_MAX_NEL 64
int fep3m_load_vector_static(double L, int n_el, int64_t N, const double* pos, const double* Q, double* b,
                             void* cuda_stream);

const char* fep3m_strerror(int status);

/* Release the context and all of its device memory.  NULL is a no-op.      */
void fep3m_destroy(fep3m_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* FEP3M_H */
