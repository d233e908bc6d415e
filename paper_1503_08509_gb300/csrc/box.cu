// The box [0, L]^3 with Dirichlet data Phi = g or Neumann data dPhi/dn = g on
// its boundary (Sec. "Alternate boundary conditions"), screens of order q = 1
// on the order-3 mesh.
//
// The paper carries the periodic method over to a box by one change: the mesh
// problem's boundary data are the given data less what the short-range
// potential already carries there (Eq. bcadjust), Phi^sm = g - Phi^sr, so that
// Phi = Phi^sm + Phi^sr = g on the boundary (Algorithm 1 marks the step for
// the surface elements); for Neumann data the same holds for the normal
// derivatives, and in the Galerkin form the adjusted flux is a boundary load
// s_m = int (g - dPhi^sr/dn) v_m dS.  Here:
//   binning, screens, short-range sums, evaluation: the periodic path's
//     kernels, on a periodic grid of nb + n_sr elements per axis whose first
//     nb hold the box (the context's n).  The n_sr empty layers make the
//     block around every box element reach box elements and empty ones only,
//     and no image of a charge: the block cut off at the box faces;
//   load vector: b = 4 pi (Mpq (x) Mpq (x) Mpq) r with the open (box-only)
//     mixed mass on the (3 nb + 1)^3 box nodes: the parts of boundary
//     charges' screens outside the box are not loads of the box problem;
//   boundary values: h (g - Phi^sr) at each boundary node, from the singular
//     sum over the node's block and the screen field at the node (the
//     vertex-regrouped contraction of the pair kernel for the node's element,
//     in FP64), one CTA per boundary element;
//   Neumann load: s at the face nodes, per face element by a tensor
//     Gauss-Legendre rule (BOX_NGL points per axis) of g less the normal
//     derivative of Phi^sr (singular sum over the point's block and the
//     screen field's gradient through the order-3 basis), one CTA per face
//     element, gathered per node in a fixed order;
//   mesh solve: K phi = b at the (3 nb - 1)^3 interior nodes with the
//     boundary values fixed (Dirichlet), or K phi = b + s less its component
//     along the node integrals (the constant null space) on all (3 nb + 1)^3
//     nodes with int phi = 0 (Neumann), by iterative refinement: the residual
//     in FP64 (separable banded passes over the whole node grid), the
//     correction by the FP32 fast-diagonalisation solve of the solved nodes
//     with the box eigenbasis (Dirichlet: no null mode; the periodic solve's
//     transform passes, on the tensor cores unless FEP3M_CUDA_CORES);
//   evaluation: Phi_i = Phi^sm(x_i) + Phi^sr_i by the periodic evaluation
//     kernel on the box's node grid, and U = 1/2 sum_i Q_i Phi_i (FP64).
// Mesh values are in element units (h Phi), as on the periodic path.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace fep3m {

void box_eigen(int p, int n, bool dirichlet, std::vector<double>& lam, std::vector<double>& V);

namespace {

constexpr int BT = 256;
static_assert(BOX_NGL == FEP3M_NEUMANN_NGL, "the face rule of the ABI");

inline unsigned gsz(int64_t n, int t = BT) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ int wrapb(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// the vertices (and weights) that order-3 node g of an axis takes on the
// open box mesh: the box elements containing g (node 0: element 0 only;
// node 3 nb: element nb - 1 only), each with its two vertices.  FP32: the
// weights times 120, exact integers (as the periodic path's load vector; the
// caller's scale divides by 120^3)
template <class T>
__device__ __forceinline__ int box_mpq_row(int g, int nb, const BoxBand& bd, int vtx[4], T wgt[4]) {
  const double s = sizeof(T) == 4 ? 120.0 : 1.0;
  const int e = g / 3, t = g - 3 * e;
  int k = 0;
  auto add = [&](int el, int local) {
    vtx[k] = el;
    wgt[k++] = sizeof(T) == 4 ? (T)rint(s * bd.Mpq[local][0]) : (T)bd.Mpq[local][0];
    vtx[k] = el + 1;
    wgt[k++] = sizeof(T) == 4 ? (T)rint(s * bd.Mpq[local][1]) : (T)bd.Mpq[local][1];
  };
  if (t != 0) {
    add(e, t);
  } else {
    if (e > 0) add(e - 1, 3);
    if (e < nb) add(e, 0);
  }
  return k;
}

// One axis of b = 4 pi (Mpq (x) Mpq (x) Mpq) r on the box: out (extents d[3])
// at order-3 node idx[axis] sums the input's vertices along the axis; the
// input is read with strides si[3] (the first pass reads the vertex density
// of the padded periodic grid, whose first nb + 1 vertices per axis are the
// box's)
template <class Tin, class Tout>
__global__ void k_box_load_axis(int nb, int axis, int d0, int d1, int d2, int64_t si0, int64_t si1, int64_t si2,
                                BoxBand bd, const Tin* __restrict__ in, Tout* __restrict__ out, double scale) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= (int64_t)d0 * d1 * d2) return;
  int idx[3] = {(int)(g % d0), (int)((g / d0) % d1), (int)(g / ((int64_t)d0 * d1))};
  const int64_t si[3] = {si0, si1, si2};
  int vtx[4];
  Tin w[4];
  const int k = box_mpq_row<Tin>(idx[axis], nb, bd, vtx, w);
  idx[axis] = 0;
  const int64_t base = idx[0] * si[0] + idx[1] * si[1] + idx[2] * si[2];
  Tin acc = Tin(0);
  for (int j = 0; j < k; ++j) acc += w[j] * in[base + vtx[j] * si[axis]];
  out[g] = (Tout)(scale * (double)acc);
}

// Boundary values of the mesh problem (Eq. bcadjust), element units:
//   phi[node] = h g[node] - sum_{j in block} Q_j / |x_node - x_j| (element
//   units) + sum_o A_e(o) H(o, m),
// the last term the screen field of the block's charges at node m of the
// node's element e (H the absolute FP64 vertex table [offset][node], A_e(o)
// the vertex amplitudes: the corner terms C[v - k][k] at vertex v = e - o of
// the block's elements).  One CTA (128 threads) per boundary element; the
// element writes the boundary nodes it owns (per axis local nodes 0 .. 2, and
// 3 on the last element: the binning rule min(i / 3, nb - 1)), one warp per
// node.  A charge at a boundary node makes that node's value infinite.
//
// The screen field of element E's block at E's 64 nodes, sum_o A_E(o) H(o, m),
// into G[0 .. 63] (element units), by a CTA of 128 threads; A: noff^3 + 128
// doubles of shared scratch.  Ends with a barrier.
template <class T>
__device__ void element_screen_field(int n, int n_sr, const int E[3], const T* __restrict__ Cv,
                                     const double* __restrict__ Hw, double* A, double* G) {
  const int keep = n_sr + 1, noff = 2 * n_sr + 2, no3 = noff * noff * noff;
  const int tid = threadIdx.x;
  for (int o = tid; o < no3; o += blockDim.x) {
    const int oa[3] = {o % noff - keep, (o / noff) % noff - keep, o / (noff * noff) - keep};
    const int64_t v = wrapb(E[0] - oa[0], n) + (int64_t)n * (wrapb(E[1] - oa[1], n) + (int64_t)n * wrapb(E[2] - oa[2], n));
    double a = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      // the corner's element v - k is in the block: |e - (v - k)| = |o + k| <= n_sr per axis
      if (abs(oa[0] + (k & 1)) <= n_sr && abs(oa[1] + ((k >> 1) & 1)) <= n_sr && abs(oa[2] + (k >> 2)) <= n_sr)
        a += (double)Cv[8 * v + k];
    }
    A[o] = a;
  }
  __syncthreads();
  double* Gp = A + no3;
  {
    const int m = tid & 63, half = tid >> 6;
    double s = 0.0;
    for (int o = half; o < no3; o += 2) s = fma(A[o], Hw[(int64_t)o * 64 + m], s);
    Gp[half * 64 + m] = s;
  }
  __syncthreads();
  if (tid < 64) G[tid] = Gp[tid] + Gp[64 + tid];
  __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(128) k_box_boundary(int n, int nb, int n_sr, double h, const int* __restrict__ bel,
                                                      const int* __restrict__ start, const int* __restrict__ count,
                                                      const typename vec4<T>::type* __restrict__ part,
                                                      const T* __restrict__ Cv, const double* __restrict__ Hw,
                                                      const double* __restrict__ g, double* __restrict__ phi) {
  extern __shared__ double A[];   // noff^3 vertex amplitudes and 128 partial sums, then G (64)
  const int noff = 2 * n_sr + 2, no3 = noff * noff * noff, nbk = 2 * n_sr + 1;
  const int e = bel[blockIdx.x];
  const int E[3] = {e % n, (e / n) % n, e / (n * n)};
  const int tid = threadIdx.x;
  double* G = A + no3 + 128;
  element_screen_field<T>(n, n_sr, E, Cv, Hw, A, G);
  const int lane = tid & 31, warp = tid >> 5, Nn = 3 * nb + 1, nb3 = nbk * nbk * nbk;
  for (int m = warp; m < 64; m += 4) {
    const int mm[3] = {m & 3, (m >> 2) & 3, m >> 4};
    bool own = true, bnd = false;
    int gi[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      own = own && (mm[d] < 3 || E[d] == nb - 1);
      gi[d] = 3 * E[d] + mm[d];
      bnd = bnd || gi[d] == 0 || gi[d] == 3 * nb;
    }
    if (!own || !bnd) continue;   // uniform across the warp
    const double tn[3] = {mm[0] / 3.0, mm[1] / 3.0, mm[2] / 3.0};
    double s = 0.0;
    for (int b = lane; b < nb3; b += 32) {
      const int d[3] = {b % nbk - n_sr, (b / nbk) % nbk - n_sr, b / (nbk * nbk) - n_sr};
      const int sx = E[0] + d[0], sy = E[1] + d[1], sz = E[2] + d[2];
      if (sx < 0 || sy < 0 || sz < 0 || sx >= nb || sy >= nb || sz >= nb) continue;
      const int64_t se = sx + (int64_t)n * (sy + (int64_t)n * sz);
      const int j0 = start[se], j1 = j0 + count[se];
      for (int j = j0; j < j1; ++j) {
        const typename vec4<T>::type pj = part[j];
        const double rx = (d[0] + (double)pj.x) - tn[0], ry = (d[1] + (double)pj.y) - tn[1],
                     rz = (d[2] + (double)pj.z) - tn[2];
        s += (double)pj.w / sqrt(rx * rx + ry * ry + rz * rz);
      }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const int64_t node = gi[0] + (int64_t)Nn * (gi[1] + (int64_t)Nn * gi[2]);
      phi[node] = h * g[node] - s + G[m];
    }
  }
}

// Neumann face loads, element units (the mesh problem K phi = b + s):
//   s_m = int_face (g - dPhi^sr/dn) v_m dS
//       = sum_p w_p (h^2 g_p - D_p) l_i(t1_p) l_j(t2_p)
// over the BOX_NGL^2 Gauss-Legendre points p of a face element (weights w_p on
// the unit square), D_p the normal derivative of Phi^sr in element units:
// -sum_{j in block} Q_j (r . n) / |r|^3 (r the point less x_j) less the
// screen field's derivative sum_m G_m du_m/dn at the point.  One CTA (128
// threads) per face element fe = (face, e1, e2), face = 2 axis + side (side 1:
// the face at L, outward normal +axis), e1 and e2 along the next two axes
// (e2 fastest); the point data g in the same order, points (i, j) with i along
// the first of those axes.  Writes the 16 face-node sums (node i1 + 4 i2).
template <class T>
__global__ void __launch_bounds__(128) k_box_flux(int n, int nb, int n_sr, double h, BoxQuad qd,
                                                  const int* __restrict__ start, const int* __restrict__ count,
                                                  const typename vec4<T>::type* __restrict__ part,
                                                  const T* __restrict__ Cv, const double* __restrict__ Hw,
                                                  const double* __restrict__ g, double* __restrict__ sface) {
  extern __shared__ double A[];   // noff^3 + 128 scratch, G (64), point values (BOX_NGL^2)
  const int noff = 2 * n_sr + 2, no3 = noff * noff * noff, nbk = 2 * n_sr + 1, nb3 = nbk * nbk * nbk;
  constexpr int NP = BOX_NGL * BOX_NGL;
  const int fe = blockIdx.x, face = fe / (nb * nb), e1 = (fe / nb) % nb, e2 = fe % nb;
  const int ax = face >> 1, side = face & 1, a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
  int E[3];
  E[ax] = side ? nb - 1 : 0;
  E[a1] = e1;
  E[a2] = e2;
  double* G = A + no3 + 128;
  double* fp = G + 64;
  element_screen_field<T>(n, n_sr, E, Cv, Hw, A, G);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double sgn = side ? 1.0 : -1.0;   // outward normal along ax
  for (int p = warp; p < NP; p += 4) {
    double tau[3];
    tau[ax] = side;
    tau[a1] = qd.t[p / BOX_NGL];
    tau[a2] = qd.t[p % BOX_NGL];
    double sg = 0.0;   // sum_j Q_j (r . n) / |r|^3, element units
    for (int b = lane; b < nb3; b += 32) {
      const int d[3] = {b % nbk - n_sr, (b / nbk) % nbk - n_sr, b / (nbk * nbk) - n_sr};
      const int sx = E[0] + d[0], sy = E[1] + d[1], sz = E[2] + d[2];
      if (sx < 0 || sy < 0 || sz < 0 || sx >= nb || sy >= nb || sz >= nb) continue;
      const int64_t se = sx + (int64_t)n * (sy + (int64_t)n * sz);
      const int j0 = start[se], j1 = j0 + count[se];
      for (int j = j0; j < j1; ++j) {
        const typename vec4<T>::type pj = part[j];
        const double r[3] = {tau[0] - (d[0] + (double)pj.x), tau[1] - (d[1] + (double)pj.y),
                             tau[2] - (d[2] + (double)pj.z)};
        const double ir = 1.0 / sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        sg += (double)pj.w * (sgn * r[ax]) * ir * ir * ir;
      }
    }
    for (int o = 16; o > 0; o >>= 1) sg += __shfl_xor_sync(0xffffffffu, sg, o);
    if (lane == 0) {
      // screen field's normal derivative: only the ax factor is differentiated
      double v[3][4], dv[4];
      for (int a = 0; a < 3; ++a) q3_values<double>(tau[a], v[a]);
      q3_derivs<double>(tau[ax], dv);
      double sd = 0.0;
      for (int m = 0; m < 64; ++m) {
        const int mm[3] = {m & 3, (m >> 2) & 3, m >> 4};
        double u = 1.0;
        for (int a = 0; a < 3; ++a) u *= a == ax ? dv[mm[a]] : v[a][mm[a]];
        sd = fma(G[m], u, sd);
      }
      const double D = -sg - sgn * sd;
      const double w = qd.w[p / BOX_NGL] * qd.w[p % BOX_NGL];
      fp[p] = w * (h * h * g[(int64_t)fe * NP + p] - D);
    }
  }
  __syncthreads();
  if (tid < 16) {
    const int i1 = tid & 3, i2 = tid >> 2;
    double s = 0.0;
    for (int p = 0; p < NP; ++p) {
      double l1[4], l2[4];
      q3_values<double>(qd.t[p / BOX_NGL], l1);
      q3_values<double>(qd.t[p % BOX_NGL], l2);
      s = fma(fp[p], l1[i1] * l2[i2], s);
    }
    sface[(int64_t)fe * 16 + tid] = s;
  }
}

// rhs = b + s: every boundary node collects the loads of the face elements
// (of each face it lies on) that contain it, in a fixed order
__global__ void k_box_sgather(int nb, const double* __restrict__ b, const double* __restrict__ sface,
                              double* __restrict__ rhs) {
  const int Nn = 3 * nb + 1;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)Nn * Nn * Nn) return;
  const int c[3] = {(int)(i % Nn), (int)((i / Nn) % Nn), (int)(i / ((int64_t)Nn * Nn))};
  double s = 0.0;
  for (int ax = 0; ax < 3; ++ax)
    for (int side = 0; side < 2; ++side) {
      if (c[ax] != (side ? 3 * nb : 0)) continue;
      const int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3, face = 2 * ax + side;
      for (int k1 = 0; k1 < 2; ++k1) {
        const int f1 = c[a1] / 3 - 1 + k1, i1 = c[a1] - 3 * f1;
        if (f1 < 0 || f1 >= nb || i1 > 3) continue;
        for (int k2 = 0; k2 < 2; ++k2) {
          const int f2 = c[a2] / 3 - 1 + k2, i2 = c[a2] - 3 * f2;
          if (f2 < 0 || f2 >= nb || i2 > 3) continue;
          s += sface[((int64_t)(face * nb + f1) * nb + f2) * 16 + i1 + 4 * i2];
        }
      }
    }
  rhs[i] = b[i] + s;
}

// phi = h g on the boundary nodes (no adjustment), 0 inside
__global__ void k_box_plain_bvals(int Nn, double h, const double* __restrict__ g, double* __restrict__ phi) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)Nn * Nn * Nn) return;
  const int x = (int)(i % Nn), y = (int)((i / Nn) % Nn), z = (int)(i / ((int64_t)Nn * Nn));
  const bool bnd = x == 0 || y == 0 || z == 0 || x == Nn - 1 || y == Nn - 1 || z == Nn - 1;
  phi[i] = bnd ? h * g[i] : 0.0;
}

// One axis of a separable banded apply on the box's node grid:
//   out = A_axis(in) [+ B_axis(in2) + C_axis(in3)], then out = base - out with
// base; rows by node type (tap o couples node g to g + o - 3), taps past the
// grid's ends dropped and the end rows' diagonals those of one element: the
// rows of the open matrices.
__global__ void k_box_band(int Nn, int axis, BoxBand bd, int ma, const double* __restrict__ in, int mb,
                           const double* __restrict__ in2, int mc, const double* __restrict__ in3,
                           const double* __restrict__ base, double* __restrict__ out) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= (int64_t)Nn * Nn * Nn) return;
  const int idx[3] = {(int)(g % Nn), (int)((g / Nn) % Nn), (int)(g / ((int64_t)Nn * Nn))};
  const int64_t st[3] = {1, Nn, (int64_t)Nn * Nn};
  const int ga = idx[axis], t = ga % 3;
  const int64_t b0 = g - (int64_t)ga * st[axis];
  const double* rows[3] = {ma ? bd.bK[t] : bd.bM[t], mb ? bd.bK[t] : bd.bM[t], mc ? bd.bK[t] : bd.bM[t]};
  const int end = ga == 0 ? 0 : (ga == Nn - 1 ? 1 : -1);   // the first and last rows: one element's diagonal
  double acc = 0.0;
#pragma unroll
  for (int o = 0; o < 7; ++o) {
    const int ja = ga + o - 3;
    if (ja < 0 || ja >= Nn) continue;
    const int64_t j = b0 + (int64_t)ja * st[axis];
    double w0 = rows[0][o], w1 = rows[1][o], w2 = rows[2][o];
    if (o == 3 && end >= 0) {
      w0 = ma ? bd.dK[end] : bd.dM[end];
      w1 = mb ? bd.dK[end] : bd.dM[end];
      w2 = mc ? bd.dK[end] : bd.dM[end];
    }
    double v = w0 * in[j];
    if (in2) v += w1 * in2[j];
    if (in3) v += w2 * in3[j];
    acc += v;
  }
  out[g] = base ? base[g] - acc : acc;
}

// node of solved index i: the Ns^3 solved nodes start at index off per axis
// (Dirichlet: the interior, off = 1; Neumann: all nodes, off = 0)
__device__ __forceinline__ int64_t solved_node(int64_t i, int Ns, int Nn, int off) {
  const int x = (int)(i % Ns) + off, y = (int)((i / Ns) % Ns) + off, z = (int)(i / ((int64_t)Ns * Ns)) + off;
  return x + (int64_t)Nn * (y + (int64_t)Nn * z);
}

// node integral (h = 1) of node g of an axis of the open mesh
__device__ __forceinline__ double box_w1(int g, int Nn, const BoxBand& bd) {
  return (g == 0 || g == Nn - 1) ? bd.wend : bd.wn[g % 3];
}

// deterministic FP64 sums: mode 0, sum of squares of v at the solved nodes;
// mode 1, sum of v over all nodes; mode 2, sum of w3 v over all nodes (w3
// the 3-D node integrals).  Per-block partials, then one block adds them in order
__global__ void k_box_partial(int mode, int Ns, int Nn, int off, BoxBand bd, const double* __restrict__ v,
                              double* __restrict__ partial) {
  __shared__ double sh[BT / 32];
  const int64_t len = mode == 0 ? (int64_t)Ns * Ns * Ns : (int64_t)Nn * Nn * Nn;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    if (mode == 0) {
      const double x = v[solved_node(i, Ns, Nn, off)];
      acc = fma(x, x, acc);
    } else if (mode == 1) {
      acc += v[i];
    } else {
      const int x = (int)(i % Nn), y = (int)((i / Nn) % Nn), z = (int)(i / ((int64_t)Nn * Nn));
      acc = fma(box_w1(x, Nn, bd) * box_w1(y, Nn, bd) * box_w1(z, Nn, bd), v[i], acc);
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < BT / 32; ++k) s += sh[k];
    partial[blockIdx.x] = s;
  }
}
__global__ void k_box_final(int nb, const double* __restrict__ partial, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < nb; ++k) s += partial[k];
    *out = s;
  }
}

// the residual at the solved nodes, scaled into FP32; the FP32 correction added back
__global__ void k_box_round(int Ns, int Nn, int off, const double* __restrict__ res, double scale,
                            float* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < (int64_t)Ns * Ns * Ns) out[i] = (float)(res[solved_node(i, Ns, Nn, off)] * scale);
}
__global__ void k_box_add(int Ns, int Nn, int off, const float* __restrict__ x, double scale,
                          double* __restrict__ phi) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < (int64_t)Ns * Ns * Ns) {
    const int64_t j = solved_node(i, Ns, Nn, off);
    phi[j] += (double)x[i] * scale;
  }
}

// out = in - s w3 (w3 the node integrals: the load of a constant density, the
// compatibility projection of a Neumann load) or, with constant, out = in - s;
// s = *sum * scale
__global__ void k_box_sub(int Nn, BoxBand bd, const double* __restrict__ sum, double scale, int constant,
                          const double* __restrict__ in, double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)Nn * Nn * Nn) return;
  const int x = (int)(i % Nn), y = (int)((i / Nn) % Nn), z = (int)(i / ((int64_t)Nn * Nn));
  const double w = constant ? 1.0 : box_w1(x, Nn, bd) * box_w1(y, Nn, bd) * box_w1(z, Nn, bd);
  out[i] = in[i] - (*sum) * scale * w;
}

// box views of the padded grid: element counts and element ids of the charges
__global__ void k_box_counts(int n, int nb, const int* __restrict__ count, int* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)nb * nb * nb) return;
  const int x = (int)(i % nb), y = (int)((i / nb) % nb), z = (int)(i / ((int64_t)nb * nb));
  out[i] = count[x + (int64_t)n * (y + (int64_t)n * z)];
}
__global__ void k_box_cells(int64_t N, int n, int nb, const int* __restrict__ cell, int* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int e = cell[i];
  out[i] = e % n + nb * ((e / n) % n + nb * (e / (n * n)));
}
template <class T>
__global__ void k_box_coeffs(int n, int nb, const T* __restrict__ C, double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)8 * nb * nb * nb) return;
  const int64_t e = i >> 3;
  const int x = (int)(e % nb), y = (int)((e / nb) % nb), z = (int)(e / ((int64_t)nb * nb));
  out[i] = (double)C[8 * (x + (int64_t)n * (y + (int64_t)n * z)) + (i & 7)];
}

double box_rtol(const fep3m_ctx* c) {
  return c->cfg.mg_rtol > 0 ? c->cfg.mg_rtol : (c->precision == FEP3M_FP64 ? 1e-13 : 1e-10);
}

struct BoxReducer {
  Box* B;
  int nblk;
  // the sum of the given mode into dst (device); no sync
  void run(int mode, const double* v, double* dst, cudaStream_t s) {
    FEP3M_CL k_box_partial<<<nblk, BT, 0, s>>>(mode, B->Ns, B->Nn, B->off, B->band, v, B->red);
    FEP3M_CL k_box_final<<<1, 32, 0, s>>>(nblk, B->red, dst);
  }
  double host_norm2(const double* v, cudaStream_t s) {
    run(0, v, B->red + 1024, s);
    cudaMemcpyAsync(B->host_red, B->red + 1024, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    return *B->host_red;
  }
};

BoxReducer box_reducer(Box* B) {
  const int64_t len = (int64_t)B->Nn * B->Nn * B->Nn;
  return BoxReducer{B, (int)std::min<int64_t>(1024, std::max<int64_t>(1, len / (BT * 8)))};
}

// r = rhs - K phi with K = K1 (x) M1 (x) M1 + M1 (x) K1 (x) M1 + M1 (x) M1 (x) K1
// (interior rows): a = M_z phi, b = K_z phi; c = M_y a, d = K_y a, f = M_y b;
// r = rhs - (K_x c + M_x d + M_x f)
void box_residual(Box* B, const double* rhs, const double* phi, double* r, cudaStream_t s) {
  const int Nn = B->Nn;
  const int64_t len = (int64_t)Nn * Nn * Nn;
  double *a = B->t[0], *b = B->t[1], *c = B->t[2], *d = B->t[3];
  FEP3M_CL k_box_band<<<gsz(len), BT, 0, s>>>(Nn, 2, B->band, 0, phi, 0, nullptr, 0, nullptr, nullptr, a);
  FEP3M_CL k_box_band<<<gsz(len), BT, 0, s>>>(Nn, 2, B->band, 1, phi, 0, nullptr, 0, nullptr, nullptr, b);
  FEP3M_CL k_box_band<<<gsz(len), BT, 0, s>>>(Nn, 1, B->band, 0, a, 0, nullptr, 0, nullptr, nullptr, c);
  FEP3M_CL k_box_band<<<gsz(len), BT, 0, s>>>(Nn, 1, B->band, 1, a, 0, nullptr, 0, nullptr, nullptr, d);
  FEP3M_CL k_box_band<<<gsz(len), BT, 0, s>>>(Nn, 1, B->band, 0, b, 0, nullptr, 0, nullptr, nullptr, a);
  FEP3M_CL k_box_band<<<gsz(len), BT, 0, s>>>(Nn, 0, B->band, 1, c, 0, d, 0, a, rhs, r);
}

// K phi = rhs at the solved nodes (Dirichlet: the interior, phi's boundary
// values held; Neumann: all, rhs compatible): iterative refinement around the
// FP32 fast-diagonalisation solve; sets B->sweeps and B->relres (the residual
// relative to that of phi's starting values)
cudaError_t box_refine(fep3m_ctx* c, Box* B, const double* rhs, double* phi) {
  const int Ns = B->Ns;
  const int64_t len = (int64_t)Ns * Ns * Ns;
  cudaStream_t s = c->stream;
  BoxReducer red = box_reducer(B);
  const double rtol = box_rtol(c);
  const int max_sweeps = c->cfg.mg_max_cycles > 0 ? c->cfg.mg_max_cycles : 10;
  box_residual(B, rhs, phi, B->res, s);
  const double n0 = std::sqrt(red.host_norm2(B->res, s));
  B->sweeps = 0;
  B->relres = 0.0;
  if (!(n0 > 0.0)) return cudaGetLastError();   // zero (or, for non-finite data, NaN) residual: nothing to solve
  double nr = n0;
  for (int k = 0; k < max_sweeps; ++k) {
    // scale the residual by a power of two near 1 / RMS into FP32
    const double sc = std::ldexp(1.0, -std::ilogb(nr / std::sqrt((double)len)));
    FEP3M_CL k_box_round<<<gsz(len), BT, 0, s>>>(Ns, B->Nn, B->off, B->res, sc, B->r32);
    cudaError_t e = fdm_apply(B->fdm, B->r32, B->x32, B->w1, B->w2, s);
    if (e != cudaSuccess) return e;
    FEP3M_CL k_box_add<<<gsz(len), BT, 0, s>>>(Ns, B->Nn, B->off, B->x32, 1.0 / sc, phi);
    box_residual(B, rhs, phi, B->res, s);
    nr = std::sqrt(red.host_norm2(B->res, s));
    B->sweeps = k + 1;
    B->relres = nr / n0;
    if (!(B->relres > rtol)) break;
  }
  return cudaGetLastError();
}

}  // namespace

int box_create(fep3m_ctx* c, int nb, bool neumann) {
  Box* B = new (std::nothrow) Box();
  if (!B) return FEP3M_ENOMEM;
  c->box = B;
  B->nb = nb;
  B->Nn = 3 * nb + 1;
  B->NI = 3 * nb - 1;
  B->neumann = neumann;
  B->Ns = neumann ? B->Nn : B->NI;
  B->off = neumann ? 0 : 1;
  // rows of the open order-3 matrices (h = 1): the periodic stencils inside,
  // one element's diagonal at the two ends; node integrals
  double Me[4][4], Ke[4][4], Mpq[4][2];
  element_matrices_q3(Me, Ke, Mpq);
  for (int t = 0; t < 3; ++t)
    for (int j = 0; j < 7; ++j) {
      B->band.bM[t][j] = c->st.M[t][j];
      B->band.bK[t][j] = c->st.K[t][j];
    }
  B->band.dM[0] = Me[0][0];
  B->band.dK[0] = Ke[0][0];
  B->band.dM[1] = Me[3][3];
  B->band.dK[1] = Ke[3][3];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 2; ++j) B->band.Mpq[i][j] = Mpq[i][j];
  double rs[4] = {0, 0, 0, 0};   // element row sums: the integrals of the shape functions
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) rs[i] += Me[i][j];
  B->band.wn[0] = rs[0] + rs[3];
  B->band.wn[1] = rs[1];
  B->band.wn[2] = rs[2];
  B->band.wend = rs[0];
  {
    std::vector<double> x, w;
    gauss_legendre01(BOX_NGL, x, w);
    for (int k = 0; k < BOX_NGL; ++k) {
      B->quad.t[k] = x[k];
      B->quad.w[k] = w[k];
    }
  }
  // boundary elements (padded-grid ids)
  std::vector<int> bel;
  const int n = c->n;
  for (int z = 0; z < nb; ++z)
    for (int y = 0; y < nb; ++y)
      for (int x = 0; x < nb; ++x)
        if (x == 0 || y == 0 || z == 0 || x == nb - 1 || y == nb - 1 || z == nb - 1)
          bel.push_back(x + n * (y + n * z));
  B->nbel = (int)bel.size();
  const int64_t nn3 = (int64_t)B->Nn * B->Nn * B->Nn, ns3 = (int64_t)B->Ns * B->Ns * B->Ns;
  cudaError_t e = cudaSuccess;
  auto al = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
  };
  al((void**)&B->g, box_data_size(c) * sizeof(double));
  al((void**)&B->gstage, box_data_size(c) * sizeof(double));
  al((void**)&B->b, nn3 * sizeof(double));
  al((void**)&B->rhs, nn3 * sizeof(double));
  al((void**)&B->res, nn3 * sizeof(double));
  for (double*& t : B->t) al((void**)&t, nn3 * sizeof(double));
  al((void**)&B->r32, ns3 * sizeof(float));
  al((void**)&B->x32, ns3 * sizeof(float));
  al((void**)&B->w1, ns3 * sizeof(float));
  al((void**)&B->w2, ns3 * sizeof(float));
  al((void**)&B->bel, bel.size() * sizeof(int));
  al((void**)&B->red, 1040 * sizeof(double));
  if (neumann) al((void**)&B->sface, (size_t)6 * nb * nb * 16 * sizeof(double));
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? FEP3M_ENOMEM : FEP3M_ECUDA;
  if (cudaMallocHost(&B->host_red, sizeof(double)) != cudaSuccess) return FEP3M_ENOMEM;
  cudaMemset(B->g, 0, box_data_size(c) * sizeof(double));
  cudaMemcpy(B->bel, bel.data(), bel.size() * sizeof(int), cudaMemcpyHostToDevice);
  std::vector<double> lam, V;
  box_eigen(3, nb, !neumann, lam, V);
  e = fdm_setup(B->fdm, B->Ns, lam, V, 1, !(c->cfg.flags & FEP3M_CUDA_CORES), neumann);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? FEP3M_ENOMEM : FEP3M_ECUDA;
  const int noff = c->noff;
  const size_t smem = ((size_t)noff * noff * noff + 128 + 64 + BOX_NGL * BOX_NGL) * sizeof(double);
  if (cudaFuncSetAttribute(k_box_boundary<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(k_box_boundary<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(k_box_flux<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(k_box_flux<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return FEP3M_ECUDA;
  return FEP3M_OK;
}

void box_destroy(fep3m_ctx* c) {
  Box* B = c->box;
  if (!B) return;
  void* p[] = {B->g, B->gstage, B->b, B->rhs, B->res, B->r32, B->x32, B->w1, B->w2, B->bel, B->red, B->sface};
  for (void* x : p)
    if (x) cudaFree(x);
  for (double* t : B->t)
    if (t) cudaFree(t);
  if (B->host_red) cudaFreeHost(B->host_red);
  fdm_free(B->fdm);
  delete B;
  c->box = nullptr;
}

// values of the boundary data: the (3 nb + 1)^3 nodes (Dirichlet) or the
// 6 nb^2 BOX_NGL^2 face quadrature points (Neumann)
int64_t box_data_size(const fep3m_ctx* c) {
  const Box* B = c->box;
  if (B->neumann) return (int64_t)6 * B->nb * B->nb * BOX_NGL * BOX_NGL;
  return (int64_t)B->Nn * B->Nn * B->Nn;
}

int box_set_boundary(fep3m_ctx* c, const double* g_dev) {
  Box* B = c->box;
  return cudaMemcpyAsync(B->g, g_dev, box_data_size(c) * sizeof(double), cudaMemcpyDeviceToDevice, c->stream) ==
                 cudaSuccess
             ? FEP3M_OK
             : FEP3M_ECUDA;
}

// the load vector of the box (three separable passes; the first reads the
// padded grid's vertex density)
static void box_load(fep3m_ctx* c, Box* B, cudaStream_t s) {
  const int nb = B->nb, n = c->n, Nn = B->Nn, V1 = nb + 1;
  const int64_t n1 = (int64_t)Nn * V1 * V1, n2 = (int64_t)Nn * Nn * V1, n3 = (int64_t)Nn * Nn * Nn;
  if (c->precision == FEP3M_MIXED) {
    float *t1 = (float*)B->t[0], *t2 = (float*)B->t[1];
    FEP3M_CL k_box_load_axis<float, float><<<gsz(n1), BT, 0, s>>>(nb, 0, Nn, V1, V1, 1, n, (int64_t)n * n, B->band,
                                                                 (const float*)c->rv, t1, 1.0);
    FEP3M_CL k_box_load_axis<float, float><<<gsz(n2), BT, 0, s>>>(nb, 1, Nn, Nn, V1, 1, Nn, (int64_t)Nn * V1, B->band,
                                                                 t1, t2, 1.0);
    FEP3M_CL k_box_load_axis<float, double><<<gsz(n3), BT, 0, s>>>(nb, 2, Nn, Nn, Nn, 1, Nn, (int64_t)Nn * Nn, B->band,
                                                                  t2, B->b, 4.0 * M_PI / (120.0 * 120.0 * 120.0));
  } else {
    double *t1 = B->t[0], *t2 = B->t[1];
    FEP3M_CL k_box_load_axis<double, double><<<gsz(n1), BT, 0, s>>>(nb, 0, Nn, V1, V1, 1, n, (int64_t)n * n, B->band,
                                                                   (const double*)c->rv, t1, 1.0);
    FEP3M_CL k_box_load_axis<double, double><<<gsz(n2), BT, 0, s>>>(nb, 1, Nn, Nn, V1, 1, Nn, (int64_t)Nn * V1,
                                                                   B->band, t1, t2, 1.0);
    FEP3M_CL k_box_load_axis<double, double><<<gsz(n3), BT, 0, s>>>(nb, 2, Nn, Nn, Nn, 1, Nn, (int64_t)Nn * Nn,
                                                                   B->band, t2, B->b, 4.0 * M_PI);
  }
}

// Neumann: rhs less its component along the node integrals (compatible with
// the constant null space); after the solve, phi less its mean (int phi = 0)
static void box_project(Box* B, double* rhs, cudaStream_t s) {
  const int64_t nn3 = (int64_t)B->Nn * B->Nn * B->Nn;
  const double w3 = (double)B->nb * B->nb * B->nb;   // the box's volume, h = 1
  BoxReducer red = box_reducer(B);
  red.run(1, rhs, B->red + 1025, s);
  FEP3M_CL k_box_sub<<<gsz(nn3), BT, 0, s>>>(B->Nn, B->band, B->red + 1025, 1.0 / w3, 0, rhs, rhs);
}
static void box_zero_mean(Box* B, double* phi, cudaStream_t s) {
  const int64_t nn3 = (int64_t)B->Nn * B->Nn * B->Nn;
  const double w3 = (double)B->nb * B->nb * B->nb;
  BoxReducer red = box_reducer(B);
  red.run(2, phi, B->red + 1026, s);
  FEP3M_CL k_box_sub<<<gsz(nn3), BT, 0, s>>>(B->Nn, B->band, B->red + 1026, 1.0 / w3, 1, phi, phi);
}

int box_compute(fep3m_ctx* c, double* phi_dev, double* U_dev) {
  Box* B = c->box;
  cudaStream_t s = c->stream;
  const int64_t nn3 = (int64_t)B->Nn * B->Nn * B->Nn;
  cudaError_t e;
  if (cudaMemsetAsync(c->iflags + 2, 0, sizeof(int), s) != cudaSuccess) return FEP3M_ECUDA;
  if ((e = element_lists(c)) != cudaSuccess) return FEP3M_ECUDA;
  box_load(c, B, s);
  // singular sums and screen field of the targets (need no mesh solution)
  if ((e = pair_screen(c, 0, s, false)) != cudaSuccess) return FEP3M_ECUDA;
  if (cudaMemsetAsync(c->phi64, 0, nn3 * sizeof(double), s) != cudaSuccess) return FEP3M_ECUDA;
  const size_t smem = ((size_t)c->noff * c->noff * c->noff + 128 + 64 + BOX_NGL * BOX_NGL) * sizeof(double);
  const bool f32 = c->precision == FEP3M_MIXED;
  const double* rhs = B->b;
  if (!B->neumann) {
    // boundary values (Eq. bcadjust), then the interior solve
    if (f32)
      FEP3M_CL k_box_boundary<float><<<B->nbel, 128, smem, s>>>(c->n, B->nb, c->n_sr, c->h, B->bel, c->start,
                                                               c->count, (const float4*)c->part, (const float*)c->Cv,
                                                               c->Hw64, B->g, c->phi64);
    else
      FEP3M_CL k_box_boundary<double><<<B->nbel, 128, smem, s>>>(c->n, B->nb, c->n_sr, c->h, B->bel, c->start,
                                                                c->count, (const vec4<double>::type*)c->part,
                                                                (const double*)c->Cv, c->Hw64, B->g, c->phi64);
  } else {
    // the adjusted flux as a boundary load, made compatible
    const unsigned nfe = (unsigned)(6 * B->nb * B->nb);
    if (f32)
      FEP3M_CL k_box_flux<float><<<nfe, 128, smem, s>>>(c->n, B->nb, c->n_sr, c->h, B->quad, c->start, c->count,
                                                       (const float4*)c->part, (const float*)c->Cv, c->Hw64, B->g,
                                                       B->sface);
    else
      FEP3M_CL k_box_flux<double><<<nfe, 128, smem, s>>>(c->n, B->nb, c->n_sr, c->h, B->quad, c->start, c->count,
                                                        (const vec4<double>::type*)c->part, (const double*)c->Cv,
                                                        c->Hw64, B->g, B->sface);
    FEP3M_CL k_box_sgather<<<gsz(nn3), BT, 0, s>>>(B->nb, B->b, B->sface, B->rhs);
    box_project(B, B->rhs, s);
    rhs = B->rhs;
  }
  if ((e = box_refine(c, B, rhs, c->phi64)) != cudaSuccess) return FEP3M_ECUDA;
  if (B->neumann) box_zero_mean(B, c->phi64, s);
  if ((e = pair_prepare(c)) != cudaSuccess) return FEP3M_ECUDA;
  if ((e = pair_eval(c, phi_dev, 0)) != cudaSuccess) return FEP3M_ECUDA;
  if (U_dev && (e = energy(c, U_dev)) != cudaSuccess) return FEP3M_ECUDA;
  if (cudaGetLastError() != cudaSuccess) return FEP3M_ECUDA;
  return B->relres <= 10 * box_rtol(c) ? FEP3M_OK : FEP3M_ENOCONV;
}

int box_solve(fep3m_ctx* c, double* rhs_dev, double* phi_dev) {
  Box* B = c->box;
  const int Nn = B->Nn;
  const int64_t nn3 = (int64_t)Nn * Nn * Nn;
  if (B->neumann) {
    box_project(B, rhs_dev, c->stream);
    cudaMemsetAsync(phi_dev, 0, nn3 * sizeof(double), c->stream);
  } else {
    FEP3M_CL k_box_plain_bvals<<<gsz(nn3), BT, 0, c->stream>>>(Nn, c->h, B->g, phi_dev);
  }
  if (box_refine(c, B, rhs_dev, phi_dev) != cudaSuccess) return FEP3M_ECUDA;
  if (B->neumann) box_zero_mean(B, phi_dev, c->stream);
  if (cudaGetLastError() != cudaSuccess) return FEP3M_ECUDA;
  return B->relres <= 10 * box_rtol(c) ? FEP3M_OK : FEP3M_ENOCONV;
}

// box views for the inspection entry points: counts (nb^3) and element ids
// (N) into device buffers, and the element lists as FP64 (8 nb^3)
cudaError_t box_binning(fep3m_ctx* c, int* count_out, int* cell_out) {
  const int nb = c->box->nb;
  if (count_out)
    FEP3M_CL k_box_counts<<<gsz((int64_t)nb * nb * nb), BT, 0, c->stream>>>(c->n, nb, c->count, count_out);
  if (cell_out) FEP3M_CL k_box_cells<<<gsz(c->N), BT, 0, c->stream>>>(c->N, c->n, nb, c->cell, cell_out);
  return cudaGetLastError();
}
cudaError_t box_coeffs(fep3m_ctx* c, double* out) {
  const int nb = c->box->nb;
  const int64_t len = (int64_t)8 * nb * nb * nb;
  if (c->precision == FEP3M_MIXED)
    FEP3M_CL k_box_coeffs<float><<<gsz(len), BT, 0, c->stream>>>(c->n, nb, (const float*)c->C, out);
  else
    FEP3M_CL k_box_coeffs<double><<<gsz(len), BT, 0, c->stream>>>(c->n, nb, (const double*)c->C, out);
  return cudaGetLastError();
}

}  // namespace fep3m
