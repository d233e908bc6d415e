// Charge assignment and the periodic FE mesh solve (Sec. 2.1-2.2).
//
//   element-to-point list  C[e][k] = sum_{j in e} Q_j c_k(t_j)      (Eq. oned, q = 1)
//   vertex density         r_v     = sum over (element, corner) at v (Eq. assign)
//   load vector            b       = 4 pi (Mpq (x) Mpq (x) Mpq) r    (Eq. poisson, 4 pi units)
//   mesh solve             K phi   = b - (sum b) w / sum w, int phi = 0
//
// Everything on the mesh is in reference units (element size 1): the
// physical mesh potential is phi / h.  K is the Kronecker sum of 1-D periodic
// order-3 stiffness and mass matrices, applied matrix-free by sum
// factorisation (three 7-tap passes).  Both precisions solve by iterative
// refinement (residual and iterate in FP64, or in double-float pairs for
// FEP3M_MIXED) around an FP32 inner solve:
//   - by default the exact one by fast diagonalisation: with the 1-D
//     generalized eigenpairs K1 V = M1 V Lambda, V^T M1 V = I, the
//     pseudo-inverse of K is (V x V x V) diag(1 / (l_i + l_j + l_k)) (V x V x V)^T,
//     six dense transform passes on the tensor cores;
//   - or (FEP3M_MULTIGRID) a conjugate gradient preconditioned by one
//     multigrid V-cycle: h-coarsening with the same order-3 operator on every
//     level (the coarse spaces are nested, so the Galerkin coarse operator is
//     the coarse-mesh operator), Chebyshev-Jacobi smoothing and an exact
//     coarsest solve by fast diagonalisation.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "tc.cuh"

namespace fep3m {

__constant__ double cM64[3][7], cK64[3][7], cP64[6][4], cMpq64[4][2], cDM64[3], cDK64[3];
// the mixed mass times 120 (exact integers: the element entries are 13/120,
// 1/60, 3/10 and 3/40), for the FP32 and double-float passes
__constant__ float cMpq120[4][2];
__constant__ float cM32[3][7], cK32[3][7], cP32[6][4], cDM32[3], cDK32[3];
// inverse diagonal of K by node types, index x + 3 y + 9 z
__constant__ double cDinv64[27];
__constant__ float cDinv32[27];

// Double-float value h + l (two FP32 numbers, about 48 significant bits),
// for the refinement residual: FP64 arithmetic is a small fraction of the
// FP32 rate on this GPU.  A product keeps its exact rounding error (FMA
// two-product) plus the cross terms; a sum keeps its exact rounding error
// (two-sum, Knuth) in l.  Values stay unnormalised (|l| may exceed half an
// ulp of h); the represented number is always h + l.
struct dfv {
  float h, l;
};
__device__ __forceinline__ dfv operator*(dfv c, dfv x) {
  const float p = c.h * x.h;
  float e = fmaf(c.h, x.h, -p);
  e = fmaf(c.h, x.l, e);
  e = fmaf(c.l, x.h, e);
  return {p, e};
}
__device__ __forceinline__ dfv& operator+=(dfv& s, dfv t) {
  const float a = s.h, b = t.h;
  const float sum = a + b;
  const float bv = sum - a;
  const float err = (a - (sum - bv)) + (b - bv);
  s.h = sum;
  s.l = (s.l + t.l) + err;
  return s;
}
__device__ __forceinline__ dfv& operator*=(dfv& s, dfv t) {
  s = s * t;
  return s;
}

__constant__ float cMh[3][7], cMl[3][7], cKh[3][7], cKl[3][7];

template <class T> struct Cst;
template <> struct Cst<double> {
  static __device__ __forceinline__ double M(int t, int j) { return cM64[t][j]; }
  static __device__ __forceinline__ double K(int t, int j) { return cK64[t][j]; }
  static __device__ __forceinline__ double P(int s, int j) { return cP64[s][j]; }
  static __device__ __forceinline__ double DM(int t) { return cDM64[t]; }
  static __device__ __forceinline__ double DK(int t) { return cDK64[t]; }
  static __device__ __forceinline__ double Dinv(int k) { return cDinv64[k]; }
};
template <> struct Cst<dfv> {
  static __device__ __forceinline__ dfv M(int t, int j) { return {cMh[t][j], cMl[t][j]}; }
  static __device__ __forceinline__ dfv K(int t, int j) { return {cKh[t][j], cKl[t][j]}; }
  static __device__ __forceinline__ dfv Dinv(int k) { return {cDinv32[k], 0.0f}; }
};
template <> struct Cst<float> {
  static __device__ __forceinline__ float M(int t, int j) { return cM32[t][j]; }
  static __device__ __forceinline__ float K(int t, int j) { return cK32[t][j]; }
  static __device__ __forceinline__ float P(int s, int j) { return cP32[s][j]; }
  static __device__ __forceinline__ float DM(int t) { return cDM32[t]; }
  static __device__ __forceinline__ float DK(int t) { return cDK32[t]; }
  static __device__ __forceinline__ float Dinv(int k) { return cDinv32[k]; }
};

namespace {

constexpr int TPB = 256;

inline int grid_for(size_t n) { return (int)std::min<size_t>((n + TPB - 1) / TPB, (size_t)1 << 30); }

__device__ __forceinline__ int wrapi(int i, int N) { return i < 0 ? i + N : (i >= N ? i - N : i); }

// ---------------------------------------------------------------- assembly
template <class T>
__global__ void k_elem_coeff(int64_t ne, const int* __restrict__ start, const int* __restrict__ count,
                             const typename vec4<T>::type* __restrict__ part, T* __restrict__ C) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= ne) return;
  T acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = T(0);
  const int s = start[e], cnt = count[e];
  for (int j = s; j < s + cnt; ++j) {
    typename vec4<T>::type p = part[j];
    const T wx[2] = {T(1) - p.x, p.x}, wy[2] = {T(1) - p.y, p.y}, wz[2] = {T(1) - p.z, p.z};
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] += p.w * (wx[k & 1] * wy[(k >> 1) & 1] * wz[k >> 2]);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) C[e * 8 + k] = acc[k];
}

// vertex density r_v = sum_k C[v - k][k], and the same eight terms stored by
// vertex (Cv[v][k]) for the short-range kernel's partial (block-boundary) sums
template <class T>
__global__ void k_vertex_density(int n, const T* __restrict__ C, T* __restrict__ rv, T* __restrict__ Cv) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ne = (int64_t)n * n * n;
  if (v >= ne) return;
  const int vx = (int)(v % n), vy = (int)((v / n) % n), vz = (int)(v / ((int64_t)n * n));
  T acc = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    int ex = wrapi(vx - (k & 1), n), ey = wrapi(vy - ((k >> 1) & 1), n), ez = wrapi(vz - (k >> 2), n);
    const T ck = C[(ex + (int64_t)n * (ey + (int64_t)n * ez)) * 8 + k];
    Cv[v * 8 + k] = ck;
    acc += ck;
  }
  rv[v] = acc;
}

// one axis of the order-3 x order-1 mixed mass: global order-3 node g -> up to
// three vertices with weights.  FP32: the weights times 120, which are exact
// integers (the element entries are 13/120, 1/60, 3/10 and 3/40), so that the
// load vector carries no systematic rounding of the weights (it would scale
// each charge's own smooth potential against its screen and bias U); the
// last pass divides by 120^3 in FP64.
template <class T>
__device__ __forceinline__ T mpq_w(int t, int j) {
  if constexpr (sizeof(T) == 4) return cMpq120[t][j];
  else return cMpq64[t][j];
}
template <class T>
__device__ __forceinline__ int mpq_row(int g, int n, int vtx[3], T wgt[3]) {
  const int e = g / 3, t = g - 3 * e;
  if (t == 0) {
    vtx[0] = wrapi(e - 1, n); wgt[0] = mpq_w<T>(3, 0);
    vtx[1] = e;               wgt[1] = mpq_w<T>(0, 0) + mpq_w<T>(3, 1);
    vtx[2] = wrapi(e + 1, n); wgt[2] = mpq_w<T>(0, 1);
    return 3;
  }
  vtx[0] = e;               wgt[0] = mpq_w<T>(t, 0);
  vtx[1] = wrapi(e + 1, n); wgt[1] = mpq_w<T>(t, 1);
  return 2;
}

// One axis of b = 4 pi (Mpq (x) Mpq (x) Mpq) r, three separable passes (x, y,
// then z): out[.., g, ..] = scale sum_k w_k in[.., v_k, ..], vertices v_k of
// order-3 node g along `axis` (mpq_row; FP32: integer weights, the caller's
// scale divides by 120^3 at the last pass).  d[3]: the output's extents (3n
// along the axes done, n along the others; their product < 2^32).  The scale:
// s64 for an FP64 output, s32 for FP32, the pair s32 + s32lo for float pairs
// (dfv: the FP32 sum times the scale as a two-product).
template <class Tin, class Tout>
__global__ void k_load_axis(int n, int axis, int d0, int d1, int d2, const Tin* __restrict__ in,
                            Tout* __restrict__ out, double s64, float s32, float s32lo) {
  const unsigned g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (unsigned)d0 * (unsigned)d1 * (unsigned)d2) return;
  const unsigned q = g / (unsigned)d0;
  int idx[3] = {(int)(g - q * (unsigned)d0), (int)(q % (unsigned)d1), (int)(q / (unsigned)d1)};
  int din[3] = {d0, d1, d2};
  din[axis] = n;
  const int64_t st[3] = {1, din[0], (int64_t)din[0] * din[1]};
  int vtx[3];
  Tin w[3];
  const int k = mpq_row<Tin>(idx[axis], n, vtx, w);
  idx[axis] = 0;
  const int64_t base = idx[0] * st[0] + idx[1] * st[1] + idx[2] * st[2];
  Tin acc = Tin(0);
  for (int j = 0; j < k; ++j) acc += w[j] * in[base + vtx[j] * st[axis]];
  if constexpr (std::is_same<Tout, dfv>::value) {
    const float p = acc * s32;
    out[g] = {p, fmaf(acc, s32lo, fmaf(acc, s32, -p))};
  } else if constexpr (std::is_same<Tout, float>::value) {
    out[g] = acc * s32;
  } else {
    out[g] = (Tout)(s64 * (double)acc);
  }
}

// Coarsest-level exact solve x = V (Dinv o (V^T b)) (V the 1-D generalized
// eigenvectors, applied along every axis), in three launches for N <= CP_MAX:
//   k_coarse_plane   one CTA per z plane: the x and y transforms in shared memory
//   k_coarse_pencil  CP_PEN z pencils per CTA: z transform, Dinv, inverse z transform
//   k_coarse_plane   the inverse x and y transforms
// Each thread computes 3 x 3 outputs of a transform (six shared loads per nine
// multiply-adds); the CTA's 256 threads cover a 48 x 48 tile per round.
constexpr int CP_MAX = 64, CP_PEN = 48;

// out[r][c] = sum_k L[r][k] R[k][c] for r < nr, c < nc, k < K (shared
// memory, row strides ls, rs); 3 x 3 register tiles, rounds of 48 x 48
template <class T, class Store>
__device__ __forceinline__ void cp_matmul(int nr, int nc, int K, const T* L, int ls, const T* R, int rs, Store st) {
  const int t3r = threadIdx.x >> 4, t3c = threadIdx.x & 15;
  for (int r0 = 0; r0 < nr; r0 += 48)
    for (int c0 = 0; c0 < nc; c0 += 48) {
      const int r = r0 + 3 * t3r, c = c0 + 3 * t3c;
      T acc[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) acc[i][j] = T(0);
      // rows / columns past the edge read row or column 0 and are not stored
      const int ri[3] = {r < nr ? r : 0, r + 1 < nr ? r + 1 : 0, r + 2 < nr ? r + 2 : 0};
      const int ci[3] = {c < nc ? c : 0, c + 1 < nc ? c + 1 : 0, c + 2 < nc ? c + 2 : 0};
      for (int k = 0; k < K; ++k) {
        T l[3], rr[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          l[i] = L[ri[i] * ls + k];
          rr[i] = R[k * rs + ci[i]];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) acc[i][j] += l[i] * rr[j];
      }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          if (r + i < nr && c + j < nc) st(r + i, c + j, acc[i][j]);
    }
}

// out[z][r'][r] = sum_{j,k} A[r'][j] A[r][k] in[z][j][k] (A row r = output r);
// dynamic shared memory 3 N (N + 1) elements; grid N, 256 threads
template <class T>
__global__ void __launch_bounds__(256) k_coarse_plane(int N, const T* __restrict__ A, const T* __restrict__ in,
                                                      T* __restrict__ out) {
  PDL_PROLOGUE
  extern __shared__ __align__(16) unsigned char cpsm[];
  const int P = N + 1;   // padded row
  T* As = (T*)cpsm;      // A[r][k] at r P + k
  T* X = As + N * P;     // plane [y][x]
  T* Y = X + N * P;      // after the x transform [y][r]
  const int64_t base = (int64_t)blockIdx.x * N * N;
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
    const int r = i / N, k = i - r * N;
    As[r * P + k] = A[i];
    X[r * P + k] = in[base + i];
  }
  __syncthreads();
  // x transform: Y[y][r] = sum_k X[y][k] A[r][k]  (L = X, R = A^T: R[k][r] = As[r P + k])
  {
    const int t3r = threadIdx.x >> 4, t3c = threadIdx.x & 15;
    for (int r0 = 0; r0 < N; r0 += 48)
      for (int c0 = 0; c0 < N; c0 += 48) {
        const int y = r0 + 3 * t3r, rr0 = c0 + 3 * t3c;
        T acc[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) acc[i][j] = T(0);
        const int yi[3] = {y < N ? y : 0, y + 1 < N ? y + 1 : 0, y + 2 < N ? y + 2 : 0};
        const int ri[3] = {rr0 < N ? rr0 : 0, rr0 + 1 < N ? rr0 + 1 : 0, rr0 + 2 < N ? rr0 + 2 : 0};
        for (int k = 0; k < N; ++k) {
          T xv[3], av[3];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            xv[i] = X[yi[i] * P + k];
            av[i] = As[ri[i] * P + k];
          }
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) acc[i][j] += xv[i] * av[j];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j)
            if (y + i < N && rr0 + j < N) Y[(y + i) * P + rr0 + j] = acc[i][j];
      }
  }
  __syncthreads();
  // y transform: out[r'][x] = sum_k A[r'][k] Y[k][x]
  cp_matmul<T>(N, N, N, As, P, Y, P,
               [&](int rp, int x, T v) { out[base + (int64_t)rp * N + x] = v; });
}

// for the CP_PEN pencils q = x + N y starting at blockIdx.x CP_PEN:
//   u[z'] = sum_z VT[z'][z] in[z][q];  u[z'] *= Dinv[z'][q];  out[z][q] = sum_z' V[z][z'] u[z']
// dynamic shared memory (2 N (N + 1) + 2 N (CP_PEN + 1)) elements; grid ceil(N^2 / CP_PEN)
template <class T>
__global__ void __launch_bounds__(256) k_coarse_pencil(int N, const T* __restrict__ VT, const T* __restrict__ V,
                                                       const T* __restrict__ Dinv, const T* __restrict__ in,
                                                       T* __restrict__ out) {
  PDL_PROLOGUE
  extern __shared__ __align__(16) unsigned char cpsm[];
  const int P = N + 1, Q = CP_PEN + 1;
  T* VTs = (T*)cpsm;
  T* Vs = VTs + N * P;
  T* U = Vs + N * P;          // [z][pencil]
  T* W = U + N * Q;           // [z'][pencil]
  const int64_t NN = (int64_t)N * N;
  const int64_t q0 = (int64_t)blockIdx.x * CP_PEN;
  const int np = (int)min((int64_t)CP_PEN, NN - q0);
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
    const int r = i / N, k = i - r * N;
    VTs[r * P + k] = VT[i];
    Vs[r * P + k] = V[i];
  }
  for (int i = threadIdx.x; i < CP_PEN * N; i += blockDim.x) {
    const int z = i / CP_PEN, p = i - z * CP_PEN;
    U[z * Q + p] = p < np ? in[z * NN + q0 + p] : T(0);
  }
  __syncthreads();
  // W[z'][p] = Dinv[z'][q0 + p] sum_z VT[z'][z] U[z][p]
  cp_matmul<T>(N, np, N, VTs, P, U, Q, [&](int zp, int p, T v) { W[zp * Q + p] = v * Dinv[zp * NN + q0 + p]; });
  __syncthreads();
  // out[z][q0 + p] = sum_z' V[z][z'] W[z'][p]
  cp_matmul<T>(N, np, N, Vs, P, W, Q, [&](int z, int p, T v) { out[z * NN + q0 + p] = v; });
}

// ------------------------------------------------------------ operator apply
enum { EPI_Y = 0, EPI_RESID = 1, EPI_CHEB = 2, EPI_CHEB0 = 3 };

// scalars derived on the device by the reductions: doubles at
// scal[SC_DERIVED + k], floats at ((float*)(scal + SC_DERIVED_F))[k]
constexpr int SC_DERIVED = 16, SC_DERIVED_F = 32;
enum { SD_ALPHA = 0, SD_BETA = 1, SD_MEAN = 2, SD_SCALE = 3, SD_INVSCALE = 4, SD_MEANLO = 5 };
// what the last block derives from the total t (written next to it, so that
// the consumers read one ready scalar instead of recomputing it per node)
enum { POST_NONE = 0, POST_ALPHA = 1, POST_BETA = 2, POST_MEAN = 3, POST_SCALE = 4 };

// Deterministic block-then-grid sum (blockDim.x == 256): the block's total
// (in thread 0) goes to partials[bid]; the last block to finish adds the
// partials in index order, writes the total to *out and derives the post
// scalar from it.  Called by every thread of the block.
__device__ void block_total_finish(double total, unsigned bid, unsigned nblocks, double* __restrict__ partials,
                                   unsigned int* __restrict__ counter, double* __restrict__ out, int post,
                                   double arg, double* __restrict__ scal) {
  __shared__ double sh[8];
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[bid] = total;
    __threadfence();
    unsigned int done = atomicAdd(counter, 1u);
    last = (done == nblocks - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0;
  for (unsigned int k = threadIdx.x; k < nblocks; k += blockDim.x) s += ((volatile double*)partials)[k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x != 0) return;
  double t = 0;
  for (int k = 0; k < 8; ++k) t += sh[k];
  *out = t;
  *counter = 0u;
  double* dd = scal + SC_DERIVED;
  float* df = (float*)(scal + SC_DERIVED_F);
  if (post == POST_ALPHA) {          // alpha = (r.z) / (p.q), t = p.q
    const double a = t != 0.0 ? scal[0] / t : 0.0;
    dd[SD_ALPHA] = a;
    df[SD_ALPHA] = (float)a;
  } else if (post == POST_BETA) {    // beta = (r.z)_new / (r.z), t = (r.z)_new
    const double bta = scal[0] != 0.0 ? t / scal[0] : 0.0;
    dd[SD_BETA] = bta;
    df[SD_BETA] = (float)bta;
    scal[0] = t;
  } else if (post == POST_MEAN) {    // t * arg (arg = 1 / W); the float value also as a pair
    const double m = t * arg;
    dd[SD_MEAN] = m;
    df[SD_MEAN] = (float)m;
    df[SD_MEANLO] = (float)(m - (double)(float)m);
  } else if (post == POST_SCALE) {   // 2^-k with 2^k near the RMS sqrt(t arg)
    const double rms = sqrt(t * arg);
    int k = rms > 0.0 && isfinite(rms) ? ilogb(rms) : 0;
    k = max(-100, min(100, k));
    dd[SD_SCALE] = ldexp(1.0, -k);
    dd[SD_INVSCALE] = ldexp(1.0, k);
    df[SD_SCALE] = (float)ldexp(1.0, -k);
    df[SD_INVSCALE] = (float)ldexp(1.0, k);
  }
}

__device__ void block_sum_finish(double acc, unsigned bid, unsigned nblocks, double* __restrict__ partials,
                                 unsigned int* __restrict__ counter, double* __restrict__ out, int post,
                                 double arg, double* __restrict__ scal) {
  __shared__ double shw[8];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) shw[threadIdx.x >> 5] = acc;
  __syncthreads();
  double t = 0;
  if (threadIdx.x == 0)
    for (int k = 0; k < 8; ++k) t += shw[k];
  block_total_finish(t, bid, nblocks, partials, counter, out, post, arg, scal);
}

// the warp's sum of float pairs (two-sums), in lane 0
__device__ __forceinline__ dfv warp_sum_df(dfv a) {
  for (int o = 16; o > 0; o >>= 1) {
    const dfv b = {__shfl_down_sync(0xffffffffu, a.h, o), __shfl_down_sync(0xffffffffu, a.l, o)};
    a += b;
  }
  return a;
}

// the block's sum of float pairs (two-sums), in thread 0
__device__ __forceinline__ dfv block_sum_df(dfv acc) {
  __shared__ dfv shd[8];
  acc = warp_sum_df(acc);
  if ((threadIdx.x & 31) == 0) shd[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 1; k < 8; ++k) acc += shd[k];
  return acc;
}

// block_sum_finish with a float-pair value per thread: the block sums as float
// pairs (an FP64 instruction costs a whole warp's slot on the FP64 pipe, a
// small fraction of the FP32 rate here, even with one lane active), FP64 from
// the block total on
__device__ void block_sum_finish_df(dfv acc, unsigned bid, unsigned nblocks, double* __restrict__ partials,
                                    unsigned int* __restrict__ counter, double* __restrict__ out, int post,
                                    double arg, double* __restrict__ scal) {
  acc = block_sum_df(acc);
  block_total_finish(threadIdx.x == 0 ? (double)acc.h + (double)acc.l : 0.0, bid, nblocks, partials, counter, out,
                     post, arg, scal);
}

// Two block-then-grid sums at once (blockDim.x == 256) of float-pair values:
// the block sums as float pairs, its totals (FP64) go to partials[2 bid],
// partials[2 bid + 1]; the last block adds the partials in index order and
// returns true on its thread 0 with the totals in ta, tb.
__device__ bool block_sum2_finish(dfv a2, dfv b2, unsigned bid, unsigned nblocks, double* __restrict__ partials,
                                  unsigned int* __restrict__ counter, double& ta, double& tb) {
  __shared__ double sh[2][8];
  __shared__ bool last;
  a2 = block_sum_df(a2);
  __syncthreads();   // block_sum_df's shared slots are reused by the second sum
  b2 = block_sum_df(b2);
  if (threadIdx.x == 0) {
    partials[2 * bid] = (double)a2.h + (double)a2.l;
    partials[2 * bid + 1] = (double)b2.h + (double)b2.l;
    __threadfence();
    const unsigned int done = atomicAdd(counter, 1u);
    last = (done == nblocks - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double s0 = 0, s1 = 0;
  for (unsigned int k = threadIdx.x; k < nblocks; k += blockDim.x) {
    s0 += ((volatile double*)partials)[2 * k];
    s1 += ((volatile double*)partials)[2 * k + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o);
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = s0;
    sh[1][threadIdx.x >> 5] = s1;
  }
  __syncthreads();
  if (threadIdx.x != 0) return false;
  ta = tb = 0;
  for (int k = 0; k < 8; ++k) {
    ta += sh[0][k];
    tb += sh[1][k];
  }
  *counter = 0u;
  return true;
}

// a dot product accumulated by an apply: block partials, counter, total, post;
// wout (the double-float residual's last apply): also the iterate's integral
// sum w3 phi into *wout, with its mean (times invW) derived as POST_MEAN does
struct ApplyDot {
  double* partials;
  unsigned int* counter;
  double* out;
  int post;
  double* wout = nullptr;
  double invW = 0.0;
};


// Fused apply y = K x, tiled by elements (2.5-D).  A CTA owns an AFX x AFY
// column of output nodes (AEX x AEY elements, origin on a vertex) and marches
// in z one element (three planes) at a time.  Since tiles and z steps start on
// vertices, the node type (vertex, or the first or second interior node of an
// element) is a compile-time constant in all three passes, and the interior
// nodes' 1-D stencils run with their 4 nonzero taps (7 for a vertex):
//   z pass (registers)  t1 = Mz x, t2 = Kz x            on (AFX+6) x (AFY+6)
//   y pass (shared)     a = My t1, c = Ky t1 + My t2     on (AFX+6) x AFY
//   x pass (shared)     y = Kx a + Mx c                  on AFX x AFY
// Each thread keeps, for each of its halo columns, the 7 input planes of the
// current element's three output planes in registers and prefetches the next
// element's three new planes while it computes.  The epilogue:
//   EPI_Y      out = y
//   EPI_RESID  out = b - y
//   EPI_CHEB   d = c1 d + c2 D^-1 (b - y); xo = x + d   (one Chebyshev step;
//              not in place: neighbouring tiles still read x as their halo)
//   EPI_CHEB0  the second Chebyshev step from a zero start, whose first step
//              is d = x = c0 D^-1 b: the input is formed from b on the fly
//              (x must point at b), then as EPI_CHEB with that d and x
constexpr int AEX = 16, AEY = 4;                  // elements per tile in x, y
constexpr int AFX = 3 * AEX, AFY = 3 * AEY;       // output nodes per tile
constexpr int AHX = AFX + 6, AHY = AFY + 6;       // halo column extents
constexpr int ANC = AHX * AHY;                    // halo columns per tile
constexpr int AT = 256;                           // threads per CTA
constexpr int APL = (ANC + AT - 1) / AT;          // halo columns per thread
static_assert(AHX * AEY <= AT && AEX * AFY <= AT, "one y item and one x item per thread");

template <class T>
struct Pair2 {
  T a, b;
};

// operands of the epilogue staged in shared memory (cp.async): b for the
// residual and the zero-start step; b, d and (single precision) x for a
// Chebyshev step
// (with DOT, EPI_Y stages x for the dot x.Kx)
template <class T, int EPI, bool DOT = false>
__host__ __device__ constexpr int apply_nst() {
  return EPI == EPI_CHEB ? (sizeof(T) == 4 ? 3 : 2) : (EPI == EPI_Y ? (DOT ? 1 : 0) : 1);
}

template <class T, int EPI, bool DOT = false>
struct ApplySmem {
  Pair2<T> tz[3][AHY][AHX];        // z pass: (Mz x, Kz x)
  Pair2<T> ac[3][AFY][AHX];        // y pass: (a, c)
  T dinv[27];                      // D^-1 by node types: x + 3 y + 9 z
  T stg[apply_nst<T, EPI, DOT>() > 0 ? apply_nst<T, EPI, DOT>() : 1][3][AFY][AFX];
};

// asynchronous global -> shared copy of one element (4, 8 or 16 bytes)
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// nonzero taps j (offset j - 3) of the 1-D stencil of a node of type t
template <int t> struct Taps {
  static constexpr int lo = t == 0 ? 0 : (t == 1 ? 2 : 1);
  static constexpr int hi = t == 0 ? 6 : (t == 1 ? 5 : 4);
};

// sum_j M(t, j) v[j] and sum_j K(t, j) v[j]; v[j] is the value at offset j - 3
template <class T, int t>
__device__ __forceinline__ void st_MK(const T* v, T& sm, T& sk) {
  constexpr int lo = Taps<t>::lo, hi = Taps<t>::hi;
  sm = Cst<T>::M(t, lo) * v[lo];
  sk = Cst<T>::K(t, lo) * v[lo];
#pragma unroll
  for (int j = lo + 1; j <= hi; ++j) {
    sm += Cst<T>::M(t, j) * v[j];
    sk += Cst<T>::K(t, j) * v[j];
  }
}

// sum_j M(t, j) u[j]
template <class T, int t>
__device__ __forceinline__ T st_M(const T* u) {
  constexpr int lo = Taps<t>::lo, hi = Taps<t>::hi;
  T s = Cst<T>::M(t, lo) * u[lo];
#pragma unroll
  for (int j = lo + 1; j <= hi; ++j) s += Cst<T>::M(t, j) * u[j];
  return s;
}

// sum_j K(t, j) u[j] + M(t, j) w[j]
template <class T, int t>
__device__ __forceinline__ T st_KM(const T* u, const T* w) {
  constexpr int lo = Taps<t>::lo, hi = Taps<t>::hi;
  T s = Cst<T>::K(t, lo) * u[lo];
  s += Cst<T>::M(t, lo) * w[lo];
#pragma unroll
  for (int j = lo + 1; j <= hi; ++j) {
    s += Cst<T>::K(t, j) * u[j];
    s += Cst<T>::M(t, j) * w[j];
  }
  return s;
}

// the epilogue at node g with y = (K x)_g and the staged b_g, d_g, x_g
// returns y (EPI_Y) or the new iterate (EPI_CHEB), the factor of the fused dots
template <class T, int EPI>
__device__ __forceinline__ T apply_epilogue(int64_t g, T y, T bg, T dg, T xg, T* __restrict__ out,
                                               T* __restrict__ d, T* __restrict__ xo, T c0, T c1, T c2, T dv,
                                               float rs, float& rsd) {
  if constexpr (std::is_same<T, dfv>::value) {
    static_assert(EPI == EPI_RESID, "the double-float apply computes residuals only");
    // FP32 output rs (b - y): the double-float difference (two-sum), rounded
    const float sm = bg.h - y.h;
    const float bv = sm - bg.h;
    const float err = (bg.h - (sm - bv)) + (-y.h - bv);
    rsd = (sm + ((bg.l - y.l) + err)) * rs;
    reinterpret_cast<float*>(out)[g] = rsd;
    return y;
  } else if constexpr (EPI == EPI_Y) {
    out[g] = y;
    return y;
  } else if constexpr (EPI == EPI_RESID) {
    if constexpr (std::is_same<T, float>::value) out[g] = bg - y;
    else reinterpret_cast<float*>(out)[g] = (float)((bg - y) * (double)rs);   // FP64 refinement residual
    return y;
  } else if constexpr (EPI == EPI_CHEB) {
    const T dn = c1 * dg + c2 * dv * (bg - y);
    const T xn = xg + dn;
    d[g] = dn;
    xo[g] = xn;
    return xn;
  } else {
    const T d0 = c0 * dv * bg;
    const T dn = c1 * d0 + c2 * dv * (bg - y);
    d[g] = dn;
    xo[g] = d0 + dn;
    return d0 + dn;
  }
}

// grid: (ceil(N / AFX), ceil(N / AFY), V ceil(n / steps)) for V vectors at a
// stride of vs nodes (scalars at scal + 64 v; DOT with V = 1), AT threads, dynamic
// shared memory sizeof(ApplySmem<T, EPI>); N = 3 n with n >= 3.  T = double or
// dfv (EPI_RESID only, the refinement residual): out is FP32 and receives the
// residual times the power of two the scaling reduction derived (scal)
//
// DOT (EPI_Y: x.(Kx); EPI_CHEB: b.(new iterate); EPI_RESID with dfv: |r|^2 of
// the FP32 residual written): each thread accumulates its nodes' products,
// then block_sum_finish with dt (partials indexed by the block's linear id
// within its vector; vector v's partials, counter and total at
// dt.partials + v nblocks, dt.counter + v, dt.out + 64 v).
//
// F32IN (dfv, EPI_RESID: the first refinement sweep, whose iterate is the
// FP32 correction e over the power-of-two scale s): x points at e (floats),
// the apply reads the pairs (e / s, 0) and writes them to xo as the iterate.
template <class T, int EPI, bool DOT = false, bool F32IN = false>
__global__ void __launch_bounds__(AT, sizeof(T) == 4 ? 3 : 2)
    k_apply_el(int N, int steps, const T* __restrict__ x, T* __restrict__ out, const T* __restrict__ b,
               T* __restrict__ d, T* __restrict__ xo, T c0, T c1, T c2, double* __restrict__ scal, ApplyDot dt,
               int64_t vs) {
  PDL_PROLOGUE
  static_assert(!DOT || EPI == EPI_Y || EPI == EPI_CHEB || (EPI == EPI_RESID && std::is_same<T, dfv>::value),
                "fused dots: EPI_Y, EPI_CHEB and the double-float residual");
  static_assert(!F32IN || (EPI == EPI_RESID && std::is_same<T, dfv>::value), "FP32 input: the double-float residual");
  extern __shared__ __align__(16) unsigned char apply_smem_raw[];
  ApplySmem<T, EPI, DOT>& S = *reinterpret_cast<ApplySmem<T, EPI, DOT>*>(apply_smem_raw);
  constexpr int NST = apply_nst<T, EPI, DOT>();
  double dacc = 0.0;
  float facc = 0.f;          // EPI_RESID dot: |r|^2 in FP32
  dfv wacc = {0.f, 0.f};     // EPI_RESID dot with dt.wout: the iterate's integral
  const int n = N / 3;
  const int64_t NN = (int64_t)N * N;
  const int x0 = blockIdx.x * AFX, y0 = blockIdx.y * AFY;
  // several vectors (vs: their stride in nodes; scalars in blocks of 64): the z blocks of vector v follow those of v - 1
  const int zsb = (n + steps - 1) / steps, vi = (int)blockIdx.z / zsb;
  const int e0 = ((int)blockIdx.z - vi * zsb) * steps, e1 = min(n, e0 + steps);
  if (vi > 0) {
    const int64_t o = vi * vs;
    if constexpr (F32IN) x = reinterpret_cast<const T*>(reinterpret_cast<const float*>(x) + o);
    else x += o;
    if constexpr (EPI == EPI_RESID && !std::is_same<T, float>::value)
      out = reinterpret_cast<T*>(reinterpret_cast<float*>(out) + o);   // the FP32 residual
    else
      out += o;
    if (b) b += o;
    if (d) d += o;
    if (xo) xo += o;
    scal += 64 * vi;
  }
  const int tid = threadIdx.x;
  float rs = 0.0f;   // power-of-two scale of the refinement residual (FP64, double-float)
  if constexpr (!std::is_same<T, float>::value) rs = reinterpret_cast<const float*>(scal + SC_DERIVED_F)[SD_SCALE];
  float ris = 0.0f;  // F32IN: 1 / s
  if constexpr (F32IN) ris = reinterpret_cast<const float*>(scal + SC_DERIVED_F)[SD_INVSCALE];
  const float* xf = reinterpret_cast<const float*>(x);   // F32IN: the correction e
  auto ldx = [&](int64_t off) -> T {
    if constexpr (F32IN) return T{xf[off] * ris, 0.f};
    else return x[off];
  };
  if constexpr (!std::is_same<T, dfv>::value) {
    if (tid < 27) S.dinv[tid] = Cst<T>::Dinv(tid);
  }
  // this thread's halo columns (periodic in x and y); columns past the halo
  // read column 0 and store nothing
  int coff[APL];
#pragma unroll
  for (int k = 0; k < APL; ++k) {
    const int i = tid + k * AT;
    const int hy = i / AHX, hx = i - hy * AHX;
    const int gx = ((x0 + hx - 3) % N + N) % N, gy = ((y0 + hy - 3) % N + N) % N;
    coff[k] = i < ANC ? gy * N + gx : 0;
  }
  // window slot s holds plane 3e - 3 + s (wrapped); N >= 9, so one wrap suffices
  int zs = 3 * e0 - 3;
  if (zs < 0) zs += N;
  // EPI_CHEB0: input c0 D^-1 b, scaled per column and plane type (a halo
  // column's x and y types are hx % 3 and hy % 3: the tile starts on a vertex)
  T fs[EPI == EPI_CHEB0 ? APL : 1][3];
  if (EPI == EPI_CHEB0) {
#pragma unroll
    for (int k = 0; k < APL; ++k) {
      const int i = tid + k * AT;
      const int hy = i / AHX, hx = i - hy * AHX;
#pragma unroll
      for (int t = 0; t < 3; ++t) fs[k][t] = c0 * Cst<T>::Dinv(hx % 3 + 3 * (hy % 3) + 9 * t);
    }
  }
  T w[APL][7], nx[APL][3];
#pragma unroll
  for (int s = 0; s < 7; ++s) {
    int zz = zs + s;
    if (zz >= N) zz -= N;
#pragma unroll
    for (int k = 0; k < APL; ++k) {
      w[k][s] = ldx(zz * NN + coff[k]);
      if (EPI == EPI_CHEB0) w[k][s] *= fs[k][s % 3];
    }
  }
  // y item: halo column hx, element row ey; x item: row yy, element column ex
  const int y_ey = tid / AHX, y_hx = tid - y_ey * AHX;
  const bool y_on = tid < AHX * AEY;
  const int x_yy = tid / AEX, x_ex = tid - x_yy * AEX;
  const bool x_on = tid < AEX * AFY && x0 + 3 * x_ex < N && y0 + x_yy < N;
  const int gx0 = x0 + 3 * x_ex, gy = y0 + x_yy, ty3 = x_yy % 3;

#pragma unroll 1
  for (int e = e0; e < e1; ++e) {
    // prefetch planes 3e + 4 .. 3e + 6 for the next element
    if (e + 1 < e1) {
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        int zz = zs + 7 + s;
        if (zz >= N) zz -= N;
#pragma unroll
        for (int k = 0; k < APL; ++k) nx[k][s] = ldx(zz * NN + coff[k]);
      }
    }
    if (EPI == EPI_CHEB0 && e > e0) {   // planes 3e + 1 .. 3e + 3 arrived in the previous round
#pragma unroll
      for (int k = 0; k < APL; ++k) {
#pragma unroll
        for (int s = 4; s < 7; ++s) w[k][s] *= fs[k][s % 3];
      }
    }
    // stage this thread's epilogue operands for the step (its own nodes only,
    // so its own wait makes them visible: no barrier needed)
    if (NST > 0 && x_on) {
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const int64_t g = (int64_t)(3 * e + p) * NN + (int64_t)gy * N + gx0;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          cp_async<sizeof(T)>(&S.stg[0][p][x_yy][3 * x_ex + r], (EPI == EPI_Y ? x : b) + g + r);
          if constexpr (NST > 1) cp_async<sizeof(T)>(&S.stg[NST > 1 ? 1 : 0][p][x_yy][3 * x_ex + r], d + g + r);
          if constexpr (NST > 2) cp_async<sizeof(T)>(&S.stg[NST > 2 ? 2 : 0][p][x_yy][3 * x_ex + r], x + g + r);
        }
      }
    }
    if (NST > 0) cp_async_commit();
    // z pass: planes 3e, 3e + 1, 3e + 2 are a vertex and the two interior nodes
#pragma unroll
    for (int k = 0; k < APL; ++k) {
      const int i = tid + k * AT;
      if (i < ANC) {
        T m0, k0, m1, k1, m2, k2;
        st_MK<T, 0>(w[k], m0, k0);
        st_MK<T, 1>(w[k] + 1, m1, k1);
        st_MK<T, 2>(w[k] + 2, m2, k2);
        (&S.tz[0][0][0])[i] = {m0, k0};
        (&S.tz[1][0][0])[i] = {m1, k1};
        (&S.tz[2][0][0])[i] = {m2, k2};
      }
    }
    __syncthreads();
    // y pass: rows 3 ey .. 3 ey + 2 of column hx, for the three planes
    if (y_on) {
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        T u[7], v[7];
#pragma unroll
        for (int j = 0; j < 7; ++j) {
          const Pair2<T> q = S.tz[p][3 * y_ey + j][y_hx];
          u[j] = q.a;
          v[j] = q.b;
        }
        S.ac[p][3 * y_ey + 0][y_hx] = {st_M<T, 0>(u), st_KM<T, 0>(u, v)};
        S.ac[p][3 * y_ey + 1][y_hx] = {st_M<T, 1>(u + 1), st_KM<T, 1>(u + 1, v + 1)};
        S.ac[p][3 * y_ey + 2][y_hx] = {st_M<T, 2>(u + 2), st_KM<T, 2>(u + 2, v + 2)};
      }
    }
    __syncthreads();
    // x pass and epilogue: nodes 3 ex .. 3 ex + 2 of row yy, for the three planes
    if (NST > 0) cp_async_wait_all();
    if (x_on) {
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        T u[7], v[7];
#pragma unroll
        for (int j = 0; j < 7; ++j) {
          const Pair2<T> q = S.ac[p][x_yy][3 * x_ex + j];
          u[j] = q.a;
          v[j] = q.b;
        }
        const int64_t g = (int64_t)(3 * e + p) * NN + (int64_t)gy * N + gx0;
        const T* dv = S.dinv + 3 * ty3 + 9 * p;
        T y[3];
        y[0] = st_KM<T, 0>(u, v);
        y[1] = st_KM<T, 1>(u + 1, v + 1);
        y[2] = st_KM<T, 2>(u + 2, v + 2);
        T dsum{};
        float dres = 0.f;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          T bg{}, dg{}, xg{};
          if constexpr (NST > 0) bg = S.stg[0][p][x_yy][3 * x_ex + r];
          if constexpr (NST > 1) dg = S.stg[NST > 1 ? 1 : 0][p][x_yy][3 * x_ex + r];
          if constexpr (NST > 2) xg = S.stg[NST > 2 ? 2 : 0][p][x_yy][3 * x_ex + r];
          if constexpr (EPI == EPI_CHEB && NST == 2) xg = x[g + r];
          float rsd = 0.f;
          const T f = apply_epilogue<T, EPI>(g + r, y[r], bg, dg, xg, out, d, xo, c0, c1, c2, dv[r], rs, rsd);
          if constexpr (F32IN) xo[g + r] = T{xf[g + r] * ris, 0.f};   // the iterate after the first sweep
          if constexpr (DOT && EPI == EPI_RESID) {
            if (dt.wout) {   // the node weight (1/4 or 3/8 per axis) times the iterate, as a two-product
              const float wn = (r ? 0.375f : 0.25f) * (ty3 ? 0.375f : 0.25f) * (p ? 0.375f : 0.25f);
              const T xv = ldx(g + r);
              const float pr = wn * xv.h;
              wacc += dfv{pr, fmaf(wn, xv.l, fmaf(wn, xv.h, -pr))};
            }
          }
          if constexpr (DOT && EPI == EPI_RESID) dres = fmaf(rsd, rsd, dres);
          else if constexpr (DOT) dsum = r == 0 ? bg * f : dsum + bg * f;   // EPI_Y stages x in the b slot
        }
        if constexpr (DOT && EPI != EPI_RESID) dacc += (double)dsum;
        if constexpr (DOT && EPI == EPI_RESID) facc += dres;
      }
    }
    // next element: slots 0..3 <- 3..6, slots 4..6 <- the prefetched planes
#pragma unroll
    for (int k = 0; k < APL; ++k) {
#pragma unroll
      for (int s = 0; s < 4; ++s) w[k][s] = w[k][s + 3];
#pragma unroll
      for (int s = 0; s < 3; ++s) w[k][4 + s] = nx[k][s];
    }
    zs += 3;
    if (zs >= N) zs -= N;
  }
  if constexpr (DOT) {
    const unsigned nbv = gridDim.x * gridDim.y * zsb;   // blocks per vector
    const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * (blockIdx.z - vi * zsb));
    if constexpr (EPI == EPI_RESID) {
      if (dt.wout) {   // two totals: |r|^2 and the integral (partials two per block)
        double tr, tw;
        if (block_sum2_finish(dfv{facc, 0.f}, wacc, bid, nbv, dt.partials + (size_t)vi * 2 * nbv, dt.counter + vi,
                              tr, tw)) {
          dt.out[64 * vi] = tr;
          dt.wout[64 * vi] = tw;
          double* dd = scal + SC_DERIVED;
          float* dfs = (float*)(scal + SC_DERIVED_F);
          const double m = tw * dt.invW;
          dd[SD_MEAN] = m;
          dfs[SD_MEAN] = (float)m;
          dfs[SD_MEANLO] = (float)(m - (double)(float)m);
        }
      } else {
        block_sum_finish_df(dfv{facc, 0.f}, bid, nbv, dt.partials + (size_t)vi * nbv, dt.counter + vi,
                            dt.out + 64 * vi, dt.post, 0.0, scal);
      }
    } else
      block_sum_finish(dacc, bid, nbv, dt.partials + (size_t)vi * nbv, dt.counter + vi, dt.out + 64 * vi, dt.post,
                       0.0, scal);
  }
}

template <class T, int EPI, bool DOT = false, bool F32IN = false>
static cudaError_t apply_set_smem_one() {
  return cudaFuncSetAttribute(k_apply_el<T, EPI, DOT, F32IN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(ApplySmem<T, EPI, DOT>));
}

// the tiles need more than the default 48 KB of dynamic shared memory
static cudaError_t apply_set_smem() {
  cudaError_t e = apply_set_smem_one<float, EPI_Y>();
  if (e == cudaSuccess) e = apply_set_smem_one<float, EPI_RESID>();
  if (e == cudaSuccess) e = apply_set_smem_one<float, EPI_CHEB>();
  if (e == cudaSuccess) e = apply_set_smem_one<float, EPI_CHEB0>();
  if (e == cudaSuccess) e = apply_set_smem_one<float, EPI_Y, true>();
  if (e == cudaSuccess) e = apply_set_smem_one<float, EPI_CHEB, true>();
  if (e == cudaSuccess) e = apply_set_smem_one<double, EPI_RESID>();
  if (e == cudaSuccess) e = apply_set_smem_one<dfv, EPI_RESID>();
  if (e == cudaSuccess) e = apply_set_smem_one<dfv, EPI_RESID, true>();
  if (e == cudaSuccess) e = apply_set_smem_one<dfv, EPI_RESID, false, true>();
  if (e == cudaSuccess) e = apply_set_smem_one<dfv, EPI_RESID, true, true>();
  // coarsest-level kernels at N = CP_MAX
  const int smp = 3 * CP_MAX * (CP_MAX + 1) * (int)sizeof(float);
  const int smq = (2 * CP_MAX * (CP_MAX + 1) + 2 * CP_MAX * (CP_PEN + 1)) * (int)sizeof(float);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_coarse_plane<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smp);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_coarse_pencil<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smq);
  return e;
}

// elements per CTA in z: enough CTAs to fill the GPU a few times over
static inline int apply_steps(int N) {
  const int n = N / 3;
  const int64_t cols = (int64_t)((N + AFX - 1) / AFX) * ((N + AFY - 1) / AFY);
  const int64_t s = cols * n / (152 * 6);
  return (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(16, n), s));
}

static inline dim3 apply_grid(int N, int steps) {
  return dim3((N + AFX - 1) / AFX, (N + AFY - 1) / AFY, (N / 3 + steps - 1) / steps);
}

// first Chebyshev step from x = 0: d = D^-1 b / theta, x = d (used alone
// when the smoothing degree is 1); grid (ceil(N / 128), N, N)
template <class T>
__global__ void k_cheb0(int N, const T* __restrict__ b, T* __restrict__ d, T* __restrict__ x, T inv_theta) {
  PDL_PROLOGUE
  const int ix = blockIdx.x * blockDim.x + threadIdx.x;
  if (ix >= N) return;
  const int iy = blockIdx.y, iz = blockIdx.z;
  const int64_t g = ix + (int64_t)N * (iy + (int64_t)N * iz);
  const T v = inv_theta * Cst<T>::Dinv(ix % 3 + 3 * (iy % 3) + 9 * (iz % 3)) * b[g];
  d[g] = v;
  x[g] = v;
}

// ---------------------------------------------- fused grid transfers (3-D)
// Restriction (transpose of the prolongation, scaled) and prolongation in one
// launch each.  A CTA owns RX x RY coarse elements in x and y and marches one
// coarse element (three coarse planes, six fine planes) at a time in z; the x
// and y passes of each plane run in shared memory, the z weights in registers.
// 1-D rules, coarse node 3E + j, fine node 6E + s (P the 1-D prolongation):
//   restrict:  c[3E + j] = sum_{s=1..5} P[s][j] f[6E + s]  (j = 1, 2)
//              c[3E]     = f[6E] + sum_{s=1..5} (P[s][0] f[6E + s] + P[s][3] f[6E - 6 + s])
//   prolong:   f[6E + s] = sum_{j=0..3} P[s][j] c[3E + j]   (3E + 3 wraps)
constexpr int RX = 4, RY = 4;                       // coarse elements per tile
constexpr int RCX = 3 * RX, RCY = 3 * RY;           // coarse nodes per tile
constexpr int RFX = 6 * RX + 5, RFY = 6 * RY + 5;   // fine halo tile of a restriction plane
constexpr int RT = 256;                             // threads (>= RCX * RCY)
constexpr int RNF = RFX * RFY, RPL = (RNF + RT - 1) / RT;
static_assert(RCX * RCY <= RT, "one coarse column per thread");

__device__ __forceinline__ int wrap_mod(int v, int n) { return ((v % n) + n) % n; }

// grid (ceil(nc / RX), ceil(nc / RY), ceil(nc / steps)), RT threads; Nf = 2 Nc, Nc = 3 nc
template <class T>
__global__ void __launch_bounds__(RT) k_restrict3(int Nf, int steps, const T* __restrict__ in, T* __restrict__ out,
                                                  T scale) {
  PDL_PROLOGUE
  __shared__ T F[RFY][RFX];      // one fine plane of the tile (halo 5 below)
  __shared__ T Xt[RCX][RFY];     // after the x pass, coarse x major
  __shared__ T Ps[6][4];
  const int Nc = Nf / 2, nc = Nc / 3;
  const int64_t NNf = (int64_t)Nf * Nf, NNc = (int64_t)Nc * Nc;
  const int X0 = blockIdx.x * RX, Y0 = blockIdx.y * RY;
  const int E0 = blockIdx.z * steps, E1 = min(nc, E0 + steps);
  const int tid = threadIdx.x;
  if (tid < 24) Ps[tid / 4][tid % 4] = Cst<T>::P(tid / 4, tid % 4);
  int foff[RPL];
#pragma unroll
  for (int k = 0; k < RPL; ++k) {
    const int i = tid + k * RT;
    const int row = i / RFX, col = i - row * RFX;
    foff[k] = i < RNF ? wrap_mod(6 * Y0 - 5 + row, Nf) * Nf + wrap_mod(6 * X0 - 5 + col, Nf) : 0;
  }
  // this thread's coarse column
  const int cy = tid / RCX, cx = tid - cy * RCX;
  const bool col_on = tid < RCX * RCY && X0 + cx / 3 < nc && Y0 + cy / 3 < nc;
  const int64_t gcol = (int64_t)(3 * Y0 + cy) * Nc + 3 * X0 + cx;
  T acc_v = T(0), acc_1 = T(0), acc_2 = T(0), acc_n = T(0);
  // the next fine plane is fetched into registers while the current one is reduced
  T pf[RPL];
  auto fetch = [&](int f) {
    const int fz = f < 0 ? f + Nf : (f >= Nf ? f - Nf : f);
    const T* src = in + fz * NNf;
#pragma unroll
    for (int k = 0; k < RPL; ++k) pf[k] = src[foff[k]];
  };
  fetch(6 * E0 - 5);
  for (int f = 6 * E0 - 5; f < 6 * E1; ++f) {
    __syncthreads();   // the previous plane's x pass is done with F
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      const int i = tid + k * RT;
      if (i < RNF) (&F[0][0])[i] = pf[k];
    }
    if (f + 1 < 6 * E1) fetch(f + 1);
    __syncthreads();
    // x pass: item w = (coarse x, fine row), rows fastest (conflict-free reads of F)
    for (int w = tid; w < RCX * RFY; w += RT) {
      const int c = w / RFY, row = w - c * RFY;
      const int Ex = c / 3, j = c - 3 * Ex;
      const T* fr = &F[row][6 * Ex + 5];
      T a = T(0);
#pragma unroll
      for (int s = 1; s < 6; ++s) a += Ps[s][j] * fr[s];
      if (j == 0) {
        a += fr[0];
#pragma unroll
        for (int s = 1; s < 6; ++s) a += Ps[s][3] * fr[s - 6];
      }
      Xt[c][row] = a;
    }
    __syncthreads();
    // y pass of this thread's column, then the z weights of fine plane f = 6 Ez + sz
    if (tid < RCX * RCY) {
      const int Ey = cy / 3, jy = cy - 3 * Ey;
      const T* xr = &Xt[cx][6 * Ey + 5];
      T v = T(0);
#pragma unroll
      for (int s = 1; s < 6; ++s) v += Ps[s][jy] * xr[s];
      if (jy == 0) {
        v += xr[0];
#pragma unroll
        for (int s = 1; s < 6; ++s) v += Ps[s][3] * xr[s - 6];
      }
      const int Ez = (f + 6) / 6 - 1, sz = f - 6 * Ez;   // f >= -5
      if (Ez < E0) {
        acc_v += Ps[sz][3] * v;                           // element E0 - 1: vertex of E0
      } else if (sz == 0) {
        acc_v += v;
      } else {
        acc_v += Ps[sz][0] * v;
        acc_1 += Ps[sz][1] * v;
        acc_2 += Ps[sz][2] * v;
        acc_n += Ps[sz][3] * v;
      }
      if (sz == 5 && Ez >= E0) {                          // element Ez complete
        if (col_on) {
          out[(3 * Ez) * NNc + gcol] = scale * acc_v;
          out[(3 * Ez + 1) * NNc + gcol] = scale * acc_1;
          out[(3 * Ez + 2) * NNc + gcol] = scale * acc_2;
        }
        acc_v = acc_n;
        acc_1 = acc_2 = acc_n = T(0);
      }
    }
  }
}

// fine = add + P c.  grid (ceil(nc / RX), ceil(nc / RY), ceil(nc / steps)), PTH threads
constexpr int PFX = 6 * RX, PFY = 6 * RY;           // fine nodes per tile
constexpr int PCX = 3 * RX + 1, PCY = 3 * RY + 1;   // coarse nodes of a tile plane (with the next vertex)
constexpr int PTH = 192;
constexpr int PPT = (PFX * PFY + PTH - 1) / PTH;    // fine columns per thread
template <class T>
__global__ void __launch_bounds__(PTH) k_prolong3(int Nf, int steps, const T* __restrict__ in,
                                                  T* __restrict__ out, const T* __restrict__ add) {
  PDL_PROLOGUE
  __shared__ T Cc[PCY][PCX];          // one coarse plane of the tile
  __shared__ T Xp[PCY][PFX];          // after the x pass
  __shared__ T Yp[4][PFY][PFX];       // prolonged coarse planes 3E .. 3E + 3 (ring)
  __shared__ T Ps[6][4];
  const int Nc = Nf / 2, nc = Nc / 3;
  const int64_t NNf = (int64_t)Nf * Nf, NNc = (int64_t)Nc * Nc;
  const int X0 = blockIdx.x * RX, Y0 = blockIdx.y * RY;
  const int E0 = blockIdx.z * steps, E1 = min(nc, E0 + steps);
  const int tid = threadIdx.x;
  if (tid < 24) Ps[tid / 4][tid % 4] = Cst<T>::P(tid / 4, tid % 4);
  // coarse tile offsets (x, y wrapped), one per thread
  const int ci_r = tid / PCX, ci_c = tid - ci_r * PCX;
  const bool ci_on = tid < PCX * PCY;
  const int64_t coff = ci_on ? (int64_t)((3 * Y0 + ci_r) % Nc) * Nc + (3 * X0 + ci_c) % Nc : 0;
  // this thread's fine columns
  int64_t fo[PPT];
  bool fon[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int i = tid + k * PTH;
    const int fy = i / PFX, fx = i - fy * PFX;
    fon[k] = i < PFX * PFY && X0 + fx / 6 < nc && Y0 + fy / 6 < nc;
    fo[k] = fon[k] ? (int64_t)(6 * Y0 + fy) * Nf + 6 * X0 + fx : 0;
  }
  // the x and y passes of coarse plane cz into ring slot r
  auto plane2d = [&](int cz, int r) {
    __syncthreads();   // Cc and Xp are free
    if (ci_on) Cc[ci_r][ci_c] = in[(int64_t)cz * NNc + coff];
    __syncthreads();
    for (int w = tid; w < PCY * PFX; w += PTH) {
      const int row = w / PFX, fx = w - row * PFX;
      const int Ex = fx / 6, sx = fx - 6 * Ex;
      T a = T(0);
#pragma unroll
      for (int j = 0; j < 4; ++j) a += Ps[sx][j] * Cc[row][3 * Ex + j];
      Xp[row][fx] = a;
    }
    __syncthreads();
    for (int w = tid; w < PFY * PFX; w += PTH) {
      const int fy = w / PFX, fx = w - fy * PFX;
      const int Ey = fy / 6, sy = fy - 6 * Ey;
      T a = T(0);
#pragma unroll
      for (int j = 0; j < 4; ++j) a += Ps[sy][j] * Xp[3 * Ey + j][fx];
      Yp[r][fy][fx] = a;
    }
  };
  plane2d(3 * E0, 0);
  for (int E = E0; E < E1; ++E) {
    const int r0 = (3 * (E - E0)) & 3;   // ring slot of plane 3E
    for (int j = 1; j < 4; ++j) {
      int cz = 3 * E + j;
      if (cz >= Nc) cz -= Nc;
      plane2d(cz, (r0 + j) & 3);
    }
    __syncthreads();
    for (int s = 0; s < 6; ++s) {
      const int64_t zb = (int64_t)(6 * E + s) * NNf;
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        const int i = tid + k * PTH;
        if (!fon[k]) continue;
        const int fy = i / PFX, fx = i - fy * PFX;
        T a = T(0);
#pragma unroll
        for (int j = 0; j < 4; ++j) a += Ps[s][j] * Yp[(r0 + j) & 3][fy][fx];
        out[zb + fo[k]] = add[zb + fo[k]] + a;
      }
    }
  }
}

// coarse elements per CTA in z for the fused transfers (nc coarse elements per axis)
static inline int transfer_steps(int nc) {
  const int64_t cols = (int64_t)((nc + RX - 1) / RX) * ((nc + RY - 1) / RY);
  return (int)std::max<int64_t>(1, std::min<int64_t>(8, cols * nc / (152 * 4)));
}

// One pass of the fine-level fast-diagonalisation solve: a dense 1-D transform
// along the fastest axis of an N^3 array with the axes rotated on output,
//   out[i R + r] = s(r, i) sum_a in[r N + a] W[a N + i],   R = N^2 rows r,
// so that three passes contract x, y and z in turn and return to the input's
// axis order.  SCALE (the third analysis pass): s = 1 / (lam_i + lam_{r mod N}
// + lam_{r / N}), 0 for the constant mode.  Tiled GEMM: FM rows x FN columns
// per CTA, FK-deep chunks of the contraction in shared memory, 8 x 4 outputs
// per thread (rows tr + 16 m, columns 4 tc + c: the stores of a half-warp are
// 16 consecutive rows of one output column).
constexpr int FM = 128, FN = 64, FK = 32;

template <bool SCALE>
__global__ void __launch_bounds__(256) k_fdm_axis(int N, const float* __restrict__ in, const float* __restrict__ W,
                                                  const float* __restrict__ lam, int null_mode, float* __restrict__ out) {
  PDL_PROLOGUE
  __shared__ float As[FK][FM + 1];                  // [k][row]
  __shared__ __align__(16) float Ws[FK][FN];        // [k][column]
  const int64_t R = (int64_t)N * N;
  const int64_t r0 = (int64_t)blockIdx.x * FM;
  const int i0 = blockIdx.y * FN;
  const int tid = threadIdx.x, tr = tid & 15, tc = tid >> 4;
  float acc[8][4];
#pragma unroll
  for (int m = 0; m < 8; ++m)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[m][c] = 0.f;
  for (int k0 = 0; k0 < N; k0 += FK) {
    for (int e = tid; e < FM * FK; e += 256) {   // lanes along the contraction: coalesced rows
      const int rr = e / FK, kk = e % FK;
      const int64_t r = r0 + rr;
      const int a = k0 + kk;
      As[kk][rr] = (r < R && a < N) ? in[r * N + a] : 0.f;
    }
    for (int e = tid; e < FK * FN; e += 256) {
      const int kk = e / FN, cc = e % FN;
      const int a = k0 + kk, i = i0 + cc;
      Ws[kk][cc] = (a < N && i < N) ? W[(int64_t)a * N + i] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < FK; ++kk) {
      const float4 w = *reinterpret_cast<const float4*>(&Ws[kk][4 * tc]);
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const float a = As[kk][tr + 16 * m];
        acc[m][0] = fmaf(a, w.x, acc[m][0]);
        acc[m][1] = fmaf(a, w.y, acc[m][1]);
        acc[m][2] = fmaf(a, w.z, acc[m][2]);
        acc[m][3] = fmaf(a, w.w, acc[m][3]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int64_t r = r0 + tr + 16 * m;
    if (r >= R) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = i0 + 4 * tc + c;
      if (i >= N) continue;
      float v = acc[m][c];
      if (SCALE) {
        const int j = (int)(r % N), k = (int)(r / N);
        v = (i == null_mode && j == null_mode && k == null_mode) ? 0.f : v / (lam[i] + lam[j] + lam[k]);
      }
      out[(int64_t)i * R + r] = v;
    }
  }
}

// The same pass on the tensor cores, as a general row GEMM with the output
// transposed: out[(i - cb) R + r] = s(r, i) sum_{a < K} in[r K + a] B[i][a]
// for R rows r and columns cb <= i < ce (the column tiles of nt from the one
// holding cb).  Per CTA 128 rows and the nt columns of one column tile; the
// contraction in chunks of 64 as tcgen05 bf16 MMAs (M = 128, N = nt) on
// three-piece splits of both operands (six piece products, two TMEM
// accumulators: the leading product, the other five).  A (the input rows) is
// split in the kernel into 128-byte-swizzled K-major tiles; B comes split and
// laid out in advance (Bp: [column tile][chunk][piece][nt rows][64], zero
// outside NC x K).  nt <= 256: the two accumulators take up to all 512 TMEM
// columns.  The epilogue reads one row per thread from TMEM, so a
// warp's stores of one column are 32 consecutive rows.  Used for the
// fast-diagonalisation passes (R = N^2, K = NC = N, B = W^T; SCALE: the
// inverse eigenvalue sums, rows r = j + N k) and for the screen adjoint's
// contraction (R elements, K = 64 nodes, NC offsets).  err: a bounded wait
// that gave up.  gridDim.y vectors at a stride of vs values (in and out).
// one hardware reciprocal (within an ulp or two): the scaling pass divides each
// mode by its eigenvalue sum, and the inner solve's accuracy is set by the
// conditioning of the correction it returns (relative 1e-7 ... 1e-4 per
// refinement sweep), far above that rounding
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

constexpr int FT_THREADS = 256;

template <bool SCALE>
__global__ void __launch_bounds__(FT_THREADS) k_tc_rows(int64_t R, int K, int cb, int ce, int nt,
                                                         const float* __restrict__ in, const uint4* __restrict__ Bp,
                                                         const float* __restrict__ lam, int null_mode, int N,
                                                         float* __restrict__ out, int* __restrict__ err, int64_t vs) {
  PDL_PROLOGUE
  using namespace tc;
  in += (int64_t)blockIdx.y * vs;   // vector blockIdx.y of several at a stride of vs values
  out += (int64_t)blockIdx.y * vs;
  extern __shared__ __align__(16) unsigned char fsm[];
  unsigned char* tiles = fsm + ((1024u - (smem_u32(fsm) & 1023u)) & 1023u);
  const uint32_t tl = smem_u32(tiles), tb = tl + 3 * 16384;   // A pieces (128 x 64 each), then B pieces (nt x 64)
  const uint32_t bpiece = (uint32_t)nt * 128;
  uint64_t* mbar = (uint64_t*)(tiles + 3 * 16384 + 3 * bpiece);
  uint32_t* tslot = (uint32_t*)(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  // one-dimensional grid, column tile fastest: the CTAs that read the same 128
  // rows run together, so each row tile comes from DRAM once and from L2 after
  const int ntl = (ce + nt - 1) / nt - cb / nt;
  const int64_t r0 = (int64_t)(blockIdx.x / ntl) * 128;
  const int tile = cb / nt + (int)(blockIdx.x % ntl), n0 = tile * nt;
  const int kc = (K + 63) / 64;
  uint32_t ncols = 32;
  while (ncols < 2u * (uint32_t)nt) ncols <<= 1;
  const uint32_t lo_off = ncols / 2, idesc = umma_idesc((uint32_t)nt);
  if (warp == 0) tmem_alloc(smem_u32(tslot), ncols);
  if (tid == 0) mbar_init(smem_u32(mbar));
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint4* bsrc = Bp + (size_t)tile * kc * 3 * (bpiece / 16);
  // this thread's input units: 128 rows x 8 groups of 8, four per thread, eight threads per row;
  // the next chunk's values are loaded while the current chunk's MMAs run
  const bool vec = (K & 7) == 0;   // whole units, 32-byte aligned: two vector loads each
  float x[4][8];
  auto load_units = [&](int c) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int u = tid + FT_THREADS * j, row = u >> 3, g = u & 7;
      const int64_t r = r0 + row;
      const int a0 = 64 * c + 8 * g;
      if (vec) {
        float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
        if (r < R && a0 < K) {
          const float4* src = reinterpret_cast<const float4*>(in + r * K + a0);
          v0 = src[0];
          v1 = src[1];
        }
        x[j][0] = v0.x; x[j][1] = v0.y; x[j][2] = v0.z; x[j][3] = v0.w;
        x[j][4] = v1.x; x[j][5] = v1.y; x[j][6] = v1.z; x[j][7] = v1.w;
      } else {
#pragma unroll
        for (int t = 0; t < 8; ++t) x[j][t] = (r < R && a0 + t < K) ? in[r * K + a0 + t] : 0.f;
      }
    }
  };
  load_units(0);
  bool failed = false;
  for (int c = 0; c < kc; ++c) {
    for (int i = tid; i < 3 * (int)(bpiece / 16); i += FT_THREADS) cp_async16(tb + 16 * i, bsrc + (size_t)c * 3 * (bpiece / 16) + i);
    cp_async_commit();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int u = tid + FT_THREADS * j, row = u >> 3, g = u & 7;
      uint32_t p0[4], p1[4], p2[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) bf16_split2(x[j][2 * t], x[j][2 * t + 1], p0[t], p1[t], p2[t]);
      const uint32_t off = sw128_off(row, 8 * g);
      sts128(tl + off, p0);
      sts128(tl + 16384 + off, p1);
      sts128(tl + 32768 + off, p2);
    }
    cp_async_wait_all();
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t a = tl + 32 * kk, b = tb + 32 * kk;
        const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
        umma_bf16(tmem, umma_desc(a), umma_desc(b), idesc, acc);                                 // a0 b0
        umma_bf16(tmem + lo_off, umma_desc(a), umma_desc(b + bpiece), idesc, acc);               // a0 b1
        umma_bf16(tmem + lo_off, umma_desc(a + 16384), umma_desc(b), idesc, 1u);                 // a1 b0
        umma_bf16(tmem + lo_off, umma_desc(a), umma_desc(b + 2 * bpiece), idesc, 1u);            // a0 b2
        umma_bf16(tmem + lo_off, umma_desc(a + 16384), umma_desc(b + bpiece), idesc, 1u);        // a1 b1
        umma_bf16(tmem + lo_off, umma_desc(a + 32768), umma_desc(b), idesc, 1u);                 // a2 b0
      }
      umma_commit(smem_u32(mbar));
    }
    if (c + 1 < kc) load_units(c + 1);
    // one warp polls the barrier; the others wait at the CTA barrier
    const bool done = tid < 32 ? mbar_wait(smem_u32(mbar), (uint32_t)(c & 1)) : true;
    if (__syncthreads_or(!done)) {
      failed = true;
      break;
    }
  }
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
    (void)mbar_wait(smem_u32(mbar), 0u);
    (void)mbar_wait(smem_u32(mbar), 1u);
  }
  tc_fence_after();
  if (!failed) {
    const int q4 = warp & 3;
    const int64_t r = r0 + 32 * q4 + (tid & 31);
    float djk = 0.f;
    bool jk_null = false;
    if (SCALE && r < R) {
      const int j = (int)(r % N), k = (int)(r / N);
      djk = lam[j] + lam[k];
      jk_null = j == null_mode && k == null_mode;
    }
    for (int grp = warp >> 2; 16 * grp < nt; grp += 2) {
      uint32_t vh[16], vl[16];
      const uint32_t ta = tmem + ((uint32_t)(32 * q4) << 16) + 16 * grp;
      tmem_ld16(ta, vh);
      tmem_ld16(ta + lo_off, vl);
      tmem_wait_ld();
      if (r < R) {
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          const int i = n0 + 16 * grp + t;
          if (i < cb || i >= ce || 16 * grp + t >= nt) continue;
          float v = __uint_as_float(vh[t]) + __uint_as_float(vl[t]);
          if (SCALE) v = (jk_null && i == null_mode) ? 0.f : v * rcp_approx(lam[i] + djk);
          out[(int64_t)(i - cb) * R + r] = v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

static size_t tc_rows_smem(int nt) { return 1024 + 3 * 16384 + (size_t)3 * nt * 128 + 16; }


// dense 1-D transform along an axis: out[.. i ..] = sum_k A[i][k] in[.. k ..]
// (A = V^T when transpose), optionally scaled elementwise by s after.
template <class T>
__global__ void k_dense_axis(int N, int axis, const T* __restrict__ V, bool transpose, const T* __restrict__ in,
                             T* __restrict__ out, const T* __restrict__ scale) {
  PDL_PROLOGUE
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t NN = (int64_t)N * N;
  if (g >= NN * N) return;
  int i[3] = {(int)(g % N), (int)((g / N) % N), (int)(g / NN)};
  const int64_t st[3] = {1, N, NN};
  const int r = i[axis];
  i[axis] = 0;
  const int64_t base = i[0] + i[1] * st[1] + i[2] * st[2];
  T acc = T(0);
  for (int k = 0; k < N; ++k) {
    const T a = transpose ? V[(int64_t)k * N + r] : V[(int64_t)r * N + k];
    acc += a * in[base + k * st[axis]];
  }
  if (scale) acc *= scale[g];
  out[g] = acc;
}


// ---------------------------------------------------------- reductions
enum { RD_DOT = 0, RD_SUM = 1, RD_WSUM = 2, RD_NORM2 = 3 };

template <class T, int MODE>
__device__ __forceinline__ T reduce_term(const T* __restrict__ x, const T* __restrict__ y, int64_t g) {
  const T v = x[g];
  if (MODE == RD_DOT) return v * y[g];
  if (MODE == RD_NORM2) return v * v;
  return v;
}

// each thread adds its nodes (four per round, in the working precision) into
// an FP64 accumulator; then block_sum_finish.  MODE: x.y, sum x, sum w3 x
// (node integrals), x.x.  gridDim.y vectors: vector v at x + v vs, its total
// at out + 64 v (out lies in the vector's block of 64 scalars)
template <class T, int MODE>
__global__ void k_reduce(int N, const T* __restrict__ x, const T* __restrict__ y, double* __restrict__ partials,
                         unsigned int* __restrict__ counter, double* __restrict__ out, int post, double arg,
                         double* __restrict__ scal, int64_t vs) {
  PDL_PROLOGUE
  if (blockIdx.y > 0) {   // vector blockIdx.y: x, y at a stride of vs; out, scal in its block of 64 scalars
    const int v = blockIdx.y;
    x += v * vs;
    if (y) y += v * vs;
    partials += (size_t)v * gridDim.x;
    counter += v;
    out += 64 * v;
    scal += 64 * v;
  }
  const int64_t NN = (int64_t)N * N, tot = NN * N;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  if (MODE == RD_WSUM) {
    // whole rows per warp: the node types come from the row and the lane
    const int64_t rows = NN;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5, nwarps = stride >> 5;
    for (int64_t row = warp; row < rows; row += nwarps) {
      const int iz = (int)(row / N), iy = (int)(row - (int64_t)iz * N);
      const double wyz = (iy % 3 ? 0.375 : 0.25) * (iz % 3 ? 0.375 : 0.25);
      const T* xr = x + row * N;
      double s0 = 0.0, s1 = 0.0;   // vertex / interior columns
      for (int ix = lane; ix < N; ix += 32) {
        const double v = (double)xr[ix];
        if (ix % 3 == 0) s0 += v;
        else s1 += v;
      }
      acc += wyz * (0.25 * s0 + 0.375 * s1);
    }
  } else {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < tot; g += 4 * stride) {
      T v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t h = g + u * stride;
        v[u] = h < tot ? reduce_term<T, MODE>(x, y, h) : T(0);
      }
      acc += (double)((v[0] + v[1]) + (v[2] + v[3]));
    }
  }
  block_sum_finish(acc, blockIdx.x, gridDim.x, partials, counter, out, post, arg, scal);
}

template <class T>
__device__ __forceinline__ T derived(const double* scal, int k) {
  if (sizeof(T) == 8) return (T)scal[SC_DERIVED + k];
  return (T)((const float*)(scal + SC_DERIVED_F))[k];
}

// v -= m w3 (removes the load of a uniform background, m = sum v / W), or
// v -= m (mean zero, m = sum w3 v / W); grid (ceil(N / bx), V N, N) for V
// vectors at a stride of vs (the same for k_project_copy64)
template <class T>
__global__ void k_project(int N, T* __restrict__ v, const double* __restrict__ scal, int mean_zero, int64_t vs) {
  PDL_PROLOGUE
  const int ix = blockIdx.x * blockDim.x + threadIdx.x;
  if (ix >= N) return;
  const int vi = (int)blockIdx.y / N, iy = (int)blockIdx.y - vi * N, iz = blockIdx.z;
  v += vi * vs;
  scal += 64 * vi;
  const int64_t g = ix + (int64_t)N * (iy + (int64_t)N * iz);
  const T m = derived<T>(scal, SD_MEAN);
  if (mean_zero) {
    v[g] -= m;
  } else {
    const T wx = ix % 3 ? T(0.375) : T(0.25), wy = iy % 3 ? T(0.375) : T(0.25), wz = iz % 3 ? T(0.375) : T(0.25);
    v[g] -= m * (wx * wy * wz);
  }
}

// CG updates with scalars derived on the device (no host round trip):
//   x += alpha p;  r -= alpha q
template <class T>
__global__ void k_cg_update(int64_t n, const double* __restrict__ scal, T* __restrict__ x, T* __restrict__ r,
                            const T* __restrict__ p, const T* __restrict__ q) {
  PDL_PROLOGUE
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n) return;
  const T alpha = derived<T>(scal, SD_ALPHA);
  x[g] += alpha * p[g];
  r[g] -= alpha * q[g];
}
//   p = z + beta p
template <class T>
__global__ void k_cg_dir(int64_t n, const double* __restrict__ scal, T* __restrict__ p, const T* __restrict__ z) {
  PDL_PROLOGUE
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n) return;
  const T beta = derived<T>(scal, SD_BETA);
  p[g] = z[g] + beta * p[g];
}

// ------------------------------------------------------ refinement helpers
// FP64: r = s v rounded to FP32 (v the projected right-hand side, s the
// power-of-two scale) and |r|^2 into *out (grid of the reductions)
__global__ void k_round_scaled_norm(int64_t n, const double* __restrict__ v, float* __restrict__ r,
                                    double* __restrict__ partials, unsigned int* __restrict__ counter,
                                    double* __restrict__ out, double* __restrict__ scal, int64_t vs) {
  PDL_PROLOGUE
  if (blockIdx.y > 0) {
    const int vi = blockIdx.y;
    v += vi * vs;
    r += vi * vs;
    partials += (size_t)vi * gridDim.x;
    counter += vi;
    out += 64 * vi;
    scal += 64 * vi;
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += stride) {
    const float x = (float)(v[g] * scal[SC_DERIVED + SD_SCALE]);
    r[g] = x;
    acc += (double)x * (double)x;
  }
  block_sum_finish(acc, blockIdx.x, gridDim.x, partials, counter, out, POST_NONE, 0.0, scal);
}

// phi += e / s (exact: s is a power of two), two-sum then renormalised
__global__ void k_df_update(int64_t n, dfv* __restrict__ phi, const float* __restrict__ e,
                            const double* __restrict__ scal, int64_t vs) {
  PDL_PROLOGUE
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n) return;
  phi += blockIdx.y * vs;   // vector blockIdx.y
  e += blockIdx.y * vs;
  scal += 64 * blockIdx.y;
  const float is = reinterpret_cast<const float*>(scal + SC_DERIVED_F)[SD_INVSCALE];
  const float t = e[g] * is;
  dfv p = phi[g];
  const float sum = p.h + t;
  const float bv = sum - p.h;
  const float err = (p.h - (sum - bv)) + (t - bv);
  const float lo = p.l + err;
  const float h = sum + lo;
  phi[g] = {h, lo - (h - sum)};
}

// ---- double-float refinement bookkeeping (MIXED).  FP64 arithmetic runs at a
// small fraction of the FP32 rate on this GPU, so in MIXED the solver takes its
// right-hand sides and returns its solutions as float pairs (h + l, 8 bytes a
// node like FP64), and the sums, the projection and the scaling work on float
// pairs.  Several right-hand sides: vector blockIdx.y at a stride of vs values,
// scalars in its block of 64, partials and counter per vector.

// a normalised pair: |l| <= half an ulp of h
__device__ __forceinline__ dfv df_norm(dfv a) {
  const float h = a.h + a.l;
  return {h, a.l - (h - a.h)};
}

// m w as a pair (w a node weight, exact in FP32; m as the pair mh + ml)
__device__ __forceinline__ dfv df_scaled(float mh, float ml, float w) {
  const float p = mh * w;
  return {p, fmaf(ml, w, fmaf(mh, w, -p))};
}

// setup, first pass: sum b into scal[5] with the mean m = sum b / W derived,
// sum b^2 into scal[7] with the scale s = 2^-k, 2^k near the RMS
// sqrt(sum b^2 / n), derived (the POST_MEAN and POST_SCALE forms)
__global__ void k_ref_sums(int64_t n, const dfv* __restrict__ b, double* __restrict__ partials,
                           unsigned int* __restrict__ counter, double* __restrict__ scal, double invW, int64_t vs) {
  PDL_PROLOGUE
  const int vi = blockIdx.y;
  b += vi * vs;
  partials += 2 * (size_t)vi * gridDim.x;
  counter += vi;
  scal += 64 * vi;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  dfv sum = {0.f, 0.f};
  float sq = 0.f;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += stride) {
    const dfv x = b[g];
    sum += x;
    sq = fmaf(x.h, x.h, sq);
  }
  double ta, tb;
  if (block_sum2_finish(sum, dfv{sq, 0.f}, blockIdx.x, gridDim.x, partials, counter, ta, tb)) {
    double* dd = scal + SC_DERIVED;
    float* df = (float*)(scal + SC_DERIVED_F);
    scal[5] = ta;
    scal[7] = tb;
    const double m = ta * invW;
    dd[SD_MEAN] = m;
    df[SD_MEAN] = (float)m;
    df[SD_MEANLO] = (float)(m - (double)(float)m);
    const double rms = sqrt(tb / (double)n);
    int k = rms > 0.0 && isfinite(rms) ? ilogb(rms) : 0;
    k = max(-100, min(100, k));
    dd[SD_SCALE] = ldexp(1.0, -k);
    dd[SD_INVSCALE] = ldexp(1.0, k);
    df[SD_SCALE] = (float)ldexp(1.0, -k);
    df[SD_INVSCALE] = (float)ldexp(1.0, k);
  }
}

// setup, second pass: bdf = Pi b = b - m w3 (float pairs), r = s Pi b in FP32
// and |r|^2 into scal[10]; whole rows per warp (the node weights from the row
// and the column)
__global__ void k_ref_project_scale(int N, const dfv* __restrict__ b, dfv* __restrict__ bdf, float* __restrict__ r,
                                    double* __restrict__ partials, unsigned int* __restrict__ counter,
                                    double* __restrict__ scal, int64_t vs) {
  PDL_PROLOGUE
  const int vi = blockIdx.y;
  b += vi * vs;
  bdf += vi * vs;
  r += vi * vs;
  partials += (size_t)vi * gridDim.x;
  counter += vi;
  scal += 64 * vi;
  const float* dfs = reinterpret_cast<const float*>(scal + SC_DERIVED_F);
  const float mh = dfs[SD_MEAN], ml = dfs[SD_MEANLO], sc = dfs[SD_SCALE];
  const int64_t rows = (int64_t)N * N, stride = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5, nwarps = stride >> 5;
  float acc = 0.f;
  for (int64_t row = warp; row < rows; row += nwarps) {
    const int iz = (int)(row / N), iy = (int)(row - (int64_t)iz * N);
    const float wyz = (iy % 3 ? 0.375f : 0.25f) * (iz % 3 ? 0.375f : 0.25f);
    const dfv* bi = b + row * N;
    dfv* br = bdf + row * N;
    float* rr = r + row * N;
    for (int ix = lane; ix < N; ix += 32) {
      const dfv mw = df_scaled(mh, ml, wyz * (ix % 3 ? 0.375f : 0.25f));
      dfv v = bi[ix];
      v += dfv{-mw.h, -mw.l};
      v = df_norm(v);
      br[ix] = v;
      const float x = (v.h + v.l) * sc;
      rr[ix] = x;
      acc = fmaf(x, x, acc);
    }
  }
  block_sum_finish_df(dfv{acc, 0.f}, blockIdx.x, gridDim.x, partials, counter, scal + 10, POST_NONE, 0.0, scal);
}

// finish, first pass: the integral sum w3 phi of the iterate (float pairs) into
// scal[6] with the mean derived (POST_MEAN, arg = 1 / W); rows per warp, the
// weighted values summed as float pairs
__global__ void k_ref_wsum(int N, const dfv* __restrict__ v, double* __restrict__ partials,
                           unsigned int* __restrict__ counter, double* __restrict__ scal, double invW, int64_t vs) {
  PDL_PROLOGUE
  const int vi = blockIdx.y;
  v += vi * vs;
  partials += (size_t)vi * gridDim.x;
  counter += vi;
  scal += 64 * vi;
  const int64_t rows = (int64_t)N * N, stride = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5, nwarps = stride >> 5;
  dfv acc = {0.f, 0.f};
  for (int64_t row = warp; row < rows; row += nwarps) {
    const int iz = (int)(row / N), iy = (int)(row - (int64_t)iz * N);
    const dfv* vr = v + row * N;
    for (int ix = lane; ix < N; ix += 32) {
      // the node weight (1/4 or 3/8 per axis) times the value as a two-product
      const float w = (ix % 3 ? 0.375f : 0.25f) * (iy % 3 ? 0.375f : 0.25f) * (iz % 3 ? 0.375f : 0.25f);
      const dfv x = vr[ix];
      const float p = w * x.h;
      acc += dfv{p, fmaf(w, x.l, fmaf(w, x.h, -p))};
    }
  }
  block_sum_finish_df(acc, blockIdx.x, gridDim.x, partials, counter, scal + 6, POST_MEAN, invW, scal);
}

// finish, second pass: phi = v - m as normalised float pairs (m the mean just
// derived)
__global__ void k_ref_out(int64_t n, const dfv* __restrict__ v, dfv* __restrict__ phi, const double* __restrict__ scal,
                          int64_t vs) {
  PDL_PROLOGUE
  const int vi = blockIdx.y;
  v += vi * vs;
  phi += vi * vs;
  scal += 64 * vi;
  const float* dfs = reinterpret_cast<const float*>(scal + SC_DERIVED_F);
  const float mh = dfs[SD_MEAN], ml = dfs[SD_MEANLO];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += stride) {
    dfv y = v[g];
    y += dfv{-mh, -ml};
    phi[g] = df_norm(y);
  }
}

// FP64 refinement: bp = b - m w3 (m = sum b / W); grid (ceil(N / bx), N, N)
__global__ void k_project_copy64(int N, const double* __restrict__ b, const double* __restrict__ scal,
                                 double* __restrict__ bp, int64_t vs) {
  PDL_PROLOGUE
  const int ix = blockIdx.x * blockDim.x + threadIdx.x;
  if (ix >= N) return;
  const int vi = (int)blockIdx.y / N, iy = (int)blockIdx.y - vi * N, iz = blockIdx.z;
  b += vi * vs;
  bp += vi * vs;
  scal += 64 * vi;
  const int64_t g = ix + (int64_t)N * (iy + (int64_t)N * iz);
  const double w = (ix % 3 ? 0.375 : 0.25) * (iy % 3 ? 0.375 : 0.25) * (iz % 3 ? 0.375 : 0.25);
  bp[g] = b[g] - scal[SC_DERIVED + SD_MEAN] * w;
}

// phi += e / s (FP64 accumulation of an FP32 correction)
__global__ void k_add_scaled(int64_t n, double* __restrict__ phi, const float* __restrict__ e,
                             const double* __restrict__ scal, int64_t vs) {
  PDL_PROLOGUE
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n) return;
  phi += blockIdx.y * vs;   // vector blockIdx.y
  e += blockIdx.y * vs;
  scal += 64 * blockIdx.y;
  phi[g] += scal[SC_DERIVED + SD_INVSCALE] * (double)e[g];
}

}  // namespace

// allow the row GEMM the dynamic shared memory of its largest column tile
// (nt <= 256), whatever nt a caller uses
cudaError_t tc_rows_prepare(int nt) {
  if (nt > 256 || nt % 16 != 0) return cudaErrorInvalidValue;
  const int sm = (int)tc_rows_smem(256);
  cudaError_t e = cudaFuncSetAttribute(k_tc_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tc_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  return e;
}

// out[(i - cb) R + r] = sum_{a < K} in[r K + a] B[i][a] for the columns cb <= i < ce
cudaError_t tc_rows_gemm(int64_t R, int K, int cb, int ce, int nt, const float* in, const void* Bp, float* out,
                         int* err, cudaStream_t s) {
  const dim3 g((unsigned)((R + 127) / 128 * ((ce + nt - 1) / nt - cb / nt)));
  FEP3M_CL k_tc_rows<false><<<g, FT_THREADS, tc_rows_smem(nt), s>>>(R, K, cb, ce, nt, in, (const uint4*)Bp,
                                                                    nullptr, -1, 0, out, err, (int64_t)0);
  return cudaGetLastError();
}

// ======================================================================
// host side
// ======================================================================

static size_t reduce_blocks(size_t n) { return std::min<size_t>(std::max<size_t>((n + 4 * TPB - 1) / (4 * TPB), 1), 608); }

template <class T>
static void reduce(Solver* c, int N, int mode, const T* x, const T* y, double* out, int post = POST_NONE,
                   double arg = 0.0) {
  const size_t tot = (size_t)N * N * N;
  const dim3 nb((unsigned)reduce_blocks(tot), (unsigned)c->V);   // the issued right-hand sides
  double* tmp = (double*)c->red_tmp;
  cudaStream_t s = c->stream;
  const int64_t vs = c->vs;
  if (mode == RD_DOT)
    launch_pdl(k_reduce<T, RD_DOT>, nb, TPB, 0, s, N, x, y, tmp, c->red_counter, out, post, arg, c->scal, vs);
  else if (mode == RD_SUM)
    launch_pdl(k_reduce<T, RD_SUM>, nb, TPB, 0, s, N, x, y, tmp, c->red_counter, out, post, arg, c->scal, vs);
  else if (mode == RD_WSUM)
    launch_pdl(k_reduce<T, RD_WSUM>, nb, TPB, 0, s, N, x, y, tmp, c->red_counter, out, post, arg, c->scal, vs);
  else
    launch_pdl(k_reduce<T, RD_NORM2>, nb, TPB, 0, s, N, x, y, tmp, c->red_counter, out, post, arg, c->scal, vs);
}

// remove the background load (mean_zero 0) or the mean (1) with the scalar
// that the preceding POST_MEAN reduction derived
template <class T>
static void project(Solver* c, int N, T* v, int mean_zero) {
  const int bx = std::min(N, 256);
  const dim3 grid((N + bx - 1) / bx, N * c->V, N);
  launch_pdl(k_project<T>, grid, bx, 0, c->stream, N, v, c->scal, mean_zero, c->vs);
}

template <class T>
struct MG {
  Solver* c;
  Hierarchy& H;
  explicit MG(Solver* cc) : c(cc), H(cc->mg) {}

  // one fused apply; EPI_CHEB reads x and writes the new iterate to xo (xo != x);
  // dot (EPI_Y, EPI_CHEB): also accumulate x.(Kx) or b.(new iterate)
  void apply(const Level& L, const T* x, int epi, T* out, const T* b, T* d, T* xo, T c1, T c2, T c0 = T(0),
             const ApplyDot* dot = nullptr) {
    cudaStream_t s = c->stream;
    const int steps = apply_steps(L.N);
    const dim3 grid = apply_grid(L.N, steps);
    double* sc = c->scal;
    const ApplyDot nd = {nullptr, nullptr, nullptr, 0};
    if (epi == EPI_Y && dot)
      launch_pdl(k_apply_el<T, EPI_Y, true>, grid, AT, sizeof(ApplySmem<T, EPI_Y, true>), s, 
          L.N, steps, x, out, b, d, xo, c0, c1, c2, sc, *dot, (int64_t)0);
    else if (epi == EPI_Y)
      launch_pdl(k_apply_el<T, EPI_Y>, grid, AT, sizeof(ApplySmem<T, EPI_Y>), s, L.N, steps, x, out, b, d, xo,
                                                                                  c0, c1, c2, sc, nd, (int64_t)0);
    else if (epi == EPI_RESID)
      launch_pdl(k_apply_el<T, EPI_RESID>, grid, AT, sizeof(ApplySmem<T, EPI_RESID>), s, 
          L.N, steps, x, out, b, d, xo, c0, c1, c2, sc, nd, (int64_t)0);
    else if (epi == EPI_CHEB && dot)
      launch_pdl(k_apply_el<T, EPI_CHEB, true>, grid, AT, sizeof(ApplySmem<T, EPI_CHEB, true>), s, 
          L.N, steps, x, out, b, d, xo, c0, c1, c2, sc, *dot, (int64_t)0);
    else if (epi == EPI_CHEB)
      launch_pdl(k_apply_el<T, EPI_CHEB>, grid, AT, sizeof(ApplySmem<T, EPI_CHEB>), s, 
          L.N, steps, x, out, b, d, xo, c0, c1, c2, sc, nd, (int64_t)0);
    else
      launch_pdl(k_apply_el<T, EPI_CHEB0>, grid, AT, sizeof(ApplySmem<T, EPI_CHEB0>), s, 
          L.N, steps, x, out, b, d, xo, c0, c1, c2, sc, nd, (int64_t)0);
  }

  ApplyDot dot_into(int slot, int post) const {
    return {(double*)c->red_tmp, c->red_counter, c->scal + slot, post};
  }

  // Chebyshev smoothing of A x = b (D-preconditioned) on [lmax/ratio, lmax].
  // from_zero: start from x = 0 (the first step, x = D^-1 b / theta, is folded
  // into the second); otherwise the start iterate is in the level's spare
  // buffer L.a.  Iterates alternate between L.a and x; the result is in x.
  // dot: accumulate b.x (x the final iterate) in the last step (degree >= 2)
  void smooth(const Level& L, T* x, const T* b, bool from_zero, int degree, const ApplyDot* dot = nullptr) {
    const double up = 1.1 * H.lmax, lo = up / 15.0;
    const double theta = 0.5 * (up + lo), delta = 0.5 * (up - lo), sigma = theta / delta;
    double rho = 1.0 / sigma;
    T* cur = (T*)L.a;
    T* oth = x;
    if (from_zero) {
      if (degree <= 1) {
        launch_pdl(k_cheb0<T>, dim3((L.N + 127) / 128, L.N, L.N), 128, 0, c->stream, L.N, b, (T*)L.d, x,
                                                                                      (T)(1.0 / theta));
        return;
      }
      const double rn = 1.0 / (2.0 * sigma - rho);
      apply(L, b, EPI_CHEB0, nullptr, b, (T*)L.d, (T*)L.a, (T)(rn * rho), (T)(2.0 * rn / delta), (T)(1.0 / theta));
      rho = rn;
      cur = (T*)L.a;
      oth = x;
    }
    for (int k = from_zero ? 2 : 0; k < degree; ++k) {
      const ApplyDot* dk = k == degree - 1 ? dot : nullptr;
      if (k == 0) {
        apply(L, cur, EPI_CHEB, nullptr, b, (T*)L.d, oth, T(0), (T)(1.0 / theta), T(0), dk);
      } else {
        const double rn = 1.0 / (2.0 * sigma - rho);
        apply(L, cur, EPI_CHEB, nullptr, b, (T*)L.d, oth, (T)(rn * rho), (T)(2.0 * rn / delta), T(0), dk);
        rho = rn;
      }
      T* t = cur;
      cur = oth;
      oth = t;
    }
    if (cur != x) cudaMemcpyAsync(x, cur, L.size * sizeof(T), cudaMemcpyDeviceToDevice, c->stream);
  }

  void coarse_solve(const Level& L, const T* b, T* x) {
    const CoarseSolver& cs = H.coarse;
    static_assert(std::is_same<T, float>::value, "the multigrid runs in FP32");
    const T* V = cs.V32;
    const T* VT = cs.VT32;
    const T* Dinv = cs.Dinv32;
    const int N = L.N;
    cudaStream_t s = c->stream;
    T* w1 = (T*)L.t1;
    T* w2 = (T*)L.t2;
    if (N <= CP_MAX) {
      const size_t smp = (size_t)3 * N * (N + 1) * sizeof(T);
      const size_t smq = ((size_t)2 * N * (N + 1) + (size_t)2 * N * (CP_PEN + 1)) * sizeof(T);
      const unsigned gq = (unsigned)(((int64_t)N * N + CP_PEN - 1) / CP_PEN);
      launch_pdl(k_coarse_plane<T>, N, 256, smp, s, N, VT, b, w1);
      launch_pdl(k_coarse_pencil<T>, gq, 256, smq, s, N, VT, V, Dinv, w1, w2);
      launch_pdl(k_coarse_plane<T>, N, 256, smp, s, N, V, w2, x);
      return;
    }
    const int gsz = grid_for(L.size);
    launch_pdl(k_dense_axis<T>, gsz, TPB, 0, s, N, 0, V, true, b, w1, nullptr);
    launch_pdl(k_dense_axis<T>, gsz, TPB, 0, s, N, 1, V, true, w1, w2, nullptr);
    launch_pdl(k_dense_axis<T>, gsz, TPB, 0, s, N, 2, V, true, w2, w1, Dinv);
    launch_pdl(k_dense_axis<T>, gsz, TPB, 0, s, N, 0, V, false, w1, w2, nullptr);
    launch_pdl(k_dense_axis<T>, gsz, TPB, 0, s, N, 1, V, false, w2, w1, nullptr);
    launch_pdl(k_dense_axis<T>, gsz, TPB, 0, s, N, 2, V, false, w1, x, nullptr);
  }

  // exact FP32 solve of the fine level, x = K^+ b, by fast diagonalisation:
  // three analysis passes (the third scaled by the inverse eigenvalue sums)
  // and three synthesis passes; w1, w2 are N^3 scratch
  void fdm_solve(const T* b, T* x, T* w1, T* w2) {
    static_assert(std::is_same<T, float>::value, "the inner solve runs in FP32");
    const FineFDM& f = H.fdm;
    const int N = f.N;
    cudaStream_t s = c->stream;
    if (f.BpF) {
      fdm_apply(f, b, x, w1, w2, s, c->V, c->vs);
      return;
    }
    const dim3 g((unsigned)(((int64_t)N * N + FM - 1) / FM), (unsigned)((N + FN - 1) / FN));
    launch_pdl(k_fdm_axis<false>, g, 256, 0, s, N, b, f.V32, f.lam32, f.null_mode, w1);
    launch_pdl(k_fdm_axis<false>, g, 256, 0, s, N, (const T*)w1, f.V32, f.lam32, f.null_mode, w2);
    launch_pdl(k_fdm_axis<true>, g, 256, 0, s, N, (const T*)w2, f.V32, f.lam32, f.null_mode, w1);
    launch_pdl(k_fdm_axis<false>, g, 256, 0, s, N, (const T*)w1, f.VT32, f.lam32, f.null_mode, w2);
    launch_pdl(k_fdm_axis<false>, g, 256, 0, s, N, (const T*)w2, f.VT32, f.lam32, f.null_mode, w1);
    launch_pdl(k_fdm_axis<false>, g, 256, 0, s, N, (const T*)w1, f.VT32, f.lam32, f.null_mode, x);
  }

  // approximately solve A_l x = b on level l (x overwritten)
  // dot: accumulate b.x of the result (fused into the last smoothing step)
  void vcycle(int l, const T* b, T* x, const ApplyDot* dot = nullptr) {
    Level& L = H.lv[l];
    if (l == (int)H.lv.size() - 1) {
      coarse_solve(L, b, x);
      if (dot) reduce<T>(c, L.N, RD_DOT, b, x, dot->out, dot->post);
      return;
    }
    Level& Cl = H.lv[l + 1];
    cudaStream_t s = c->stream;
    smooth(L, x, b, true, H.cheb_degree);
    apply(L, x, EPI_RESID, (T*)L.r, b, nullptr, nullptr, T(0), T(0));
    // restrict r (scaled by 1/2: reference-unit Galerkin), coarse cycle, prolong and add
    const int Nf = L.N, nc = Cl.n;
    const int ts = transfer_steps(nc);
    const dim3 gt((nc + RX - 1) / RX, (nc + RY - 1) / RY, (nc + ts - 1) / ts);
    launch_pdl(k_restrict3<T>, gt, RT, 0, s, Nf, ts, (const T*)L.r, (T*)Cl.b, T(0.5));
    vcycle(l + 1, (T*)Cl.b, (T*)Cl.x);
    launch_pdl(k_prolong3<T>, gt, PTH, 0, s, Nf, ts, (const T*)Cl.x, (T*)L.a, (const T*)x);
    smooth(L, x, b, false, H.cheb_degree, dot);   // starts from L.a = x + P e
  }

  // preconditioned CG on level 0: x = A^+ Pi b, returns iterations; the
  // relative residual (FP64 dot products) goes to *relres.  The dot products
  // p.q and r.z are accumulated by the apply and the last smoothing step.
  int pcg(const T* b, T* x, T* r, T* z, T* p, T* q, double rtol, int maxit, double* relres) {
    Level& L = H.lv[0];
    const int N = L.N;
    const size_t n = L.size;
    cudaStream_t s = c->stream;
    double* sc = c->scal;   // [0] rz, [1] pq, [2] rz_new, [3] rr, [4] bb, [5] sum
    const double W = (double)L.n * L.n * L.n;
    cudaMemcpyAsync(r, b, n * sizeof(T), cudaMemcpyDeviceToDevice, s);
    reduce<T>(c, N, RD_SUM, r, nullptr, sc + 5, POST_MEAN, 1.0 / W);
    project<T>(c, N, r, 0);
    cudaMemsetAsync(x, 0, n * sizeof(T), s);
    reduce<T>(c, N, RD_NORM2, r, nullptr, sc + 4);
    double bb = 0;
    cudaMemcpyAsync(&bb, sc + 4, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (bb == 0.0) {
      *relres = 0.0;
      return 0;
    }
    const ApplyDot d_rz0 = dot_into(0, POST_NONE), d_pq = dot_into(1, POST_ALPHA), d_rz = dot_into(2, POST_BETA);
    vcycle(0, r, z, &d_rz0);
    cudaMemcpyAsync(p, z, n * sizeof(T), cudaMemcpyDeviceToDevice, s);
    int it = 0;
    double rr = bb;
    for (it = 1; it <= maxit; ++it) {
      apply(L, p, EPI_Y, q, nullptr, nullptr, nullptr, T(0), T(0), T(0), &d_pq);
      launch_pdl(k_cg_update<T>, grid_for(n), TPB, 0, s, (int64_t)n, sc, x, r, p, q);
      reduce<T>(c, N, RD_NORM2, r, nullptr, sc + 3);
      cudaMemcpyAsync(&rr, sc + 3, sizeof(double), cudaMemcpyDeviceToHost, s);
      cudaStreamSynchronize(s);
      if (rr <= rtol * rtol * bb) break;
      vcycle(0, r, z, &d_rz);
      launch_pdl(k_cg_dir<T>, grid_for(n), TPB, 0, s, (int64_t)n, sc, p, z);
    }
    *relres = std::sqrt(rr / bb);
    return std::min(it, maxit);
  }

  // the same iteration with a fixed count and no host round trip (graph-capturable);
  // leaves |Pi b|^2 in scal[4] and the final |r|^2 in scal[3]
  void pcg_fixed(const T* b, T* x, T* r, T* z, T* p, T* q, int k) {
    Level& L = H.lv[0];
    const int N = L.N;
    const size_t n = L.size;
    cudaStream_t s = c->stream;
    double* sc = c->scal;
    const double W = (double)L.n * L.n * L.n;
    cudaMemcpyAsync(r, b, n * sizeof(T), cudaMemcpyDeviceToDevice, s);
    reduce<T>(c, N, RD_SUM, r, nullptr, sc + 5, POST_MEAN, 1.0 / W);
    project<T>(c, N, r, 0);
    cudaMemsetAsync(x, 0, n * sizeof(T), s);
    reduce<T>(c, N, RD_NORM2, r, nullptr, sc + 4);
    const ApplyDot d_rz0 = dot_into(0, POST_NONE), d_pq = dot_into(1, POST_ALPHA), d_rz = dot_into(2, POST_BETA);
    vcycle(0, r, z, &d_rz0);
    cudaMemcpyAsync(p, z, n * sizeof(T), cudaMemcpyDeviceToDevice, s);
    for (int it = 1; it <= k; ++it) {
      apply(L, p, EPI_Y, q, nullptr, nullptr, nullptr, T(0), T(0), T(0), &d_pq);
      launch_pdl(k_cg_update<T>, grid_for(n), TPB, 0, s, (int64_t)n, sc, x, r, p, q);
      if (it == k) {
        reduce<T>(c, N, RD_NORM2, r, nullptr, sc + 3);
        break;
      }
      vcycle(0, r, z, &d_rz);
      launch_pdl(k_cg_dir<T>, grid_for(n), TPB, 0, s, (int64_t)n, sc, p, z);
    }
    if (k <= 0) reduce<T>(c, N, RD_NORM2, r, nullptr, sc + 3);
  }
};

static void upload_constants(const Stencils& st) {
  static bool done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && done[dev]) return;
  float M32[3][7], K32[3][7], P32[6][4], DM32[3], DK32[3];
  for (int t = 0; t < 3; ++t) {
    for (int j = 0; j < 7; ++j) {
      M32[t][j] = (float)st.M[t][j];
      K32[t][j] = (float)st.K[t][j];
    }
    DM32[t] = (float)st.diagM[t];
    DK32[t] = (float)st.diagK[t];
  }
  for (int s = 0; s < 6; ++s)
    for (int j = 0; j < 4; ++j) P32[s][j] = (float)st.P[s][j];
  cudaMemcpyToSymbol(cM64, st.M, sizeof(st.M));
  cudaMemcpyToSymbol(cK64, st.K, sizeof(st.K));
  cudaMemcpyToSymbol(cP64, st.P, sizeof(st.P));
  cudaMemcpyToSymbol(cMpq64, st.Mpq, sizeof(st.Mpq));
  float Mpq120[4][2];
  for (int t = 0; t < 4; ++t)
    for (int j = 0; j < 2; ++j) Mpq120[t][j] = (float)std::rint(120.0 * st.Mpq[t][j]);
  cudaMemcpyToSymbol(cMpq120, Mpq120, sizeof(Mpq120));
  cudaMemcpyToSymbol(cDM64, st.diagM, sizeof(st.diagM));
  cudaMemcpyToSymbol(cDK64, st.diagK, sizeof(st.diagK));
  cudaMemcpyToSymbol(cM32, M32, sizeof(M32));
  cudaMemcpyToSymbol(cK32, K32, sizeof(K32));
  cudaMemcpyToSymbol(cP32, P32, sizeof(P32));
  cudaMemcpyToSymbol(cDM32, DM32, sizeof(DM32));
  cudaMemcpyToSymbol(cDK32, DK32, sizeof(DK32));
  double Di64[27];
  float Di32[27];
  for (int k = 0; k < 27; ++k) {
    const int a = k % 3, b = (k / 3) % 3, cz = k / 9;
    Di64[k] = 1.0 / (st.diagK[a] * st.diagM[b] * st.diagM[cz] + st.diagM[a] * st.diagK[b] * st.diagM[cz] +
                     st.diagM[a] * st.diagM[b] * st.diagK[cz]);
    Di32[k] = 1.0f / (DK32[a] * DM32[b] * DM32[cz] + DM32[a] * DK32[b] * DM32[cz] + DM32[a] * DM32[b] * DK32[cz]);
  }
  cudaMemcpyToSymbol(cDinv64, Di64, sizeof(Di64));
  // double-float stencils: h = fl32(c), l = fl32(c - h)
  float Mh[3][7], Ml[3][7], Kh[3][7], Kl[3][7];
  for (int t = 0; t < 3; ++t)
    for (int j = 0; j < 7; ++j) {
      Mh[t][j] = (float)st.M[t][j];
      Ml[t][j] = (float)(st.M[t][j] - (double)Mh[t][j]);
      Kh[t][j] = (float)st.K[t][j];
      Kl[t][j] = (float)(st.K[t][j] - (double)Kh[t][j]);
    }
  cudaMemcpyToSymbol(cMh, Mh, sizeof(Mh));
  cudaMemcpyToSymbol(cMl, Ml, sizeof(Ml));
  cudaMemcpyToSymbol(cKh, Kh, sizeof(Kh));
  cudaMemcpyToSymbol(cKl, Kl, sizeof(Kl));
  cudaMemcpyToSymbol(cDinv32, Di32, sizeof(Di32));
  if (dev < 64) done[dev] = true;
}

static cudaError_t mg_setup(Solver* c) {
  upload_constants(c->st);
  Hierarchy& H = c->mg;
  H.elem_size = 4;   // the multigrid runs in FP32 in both precisions (refinement supplies the rest)
  H.lv.clear();
  int n = c->n;
  while (true) {
    Level L;
    L.n = n;
    L.N = 3 * n;
    L.size = (size_t)L.N * L.N * L.N;
    H.lv.push_back(L);
    if (n % 2 != 0 || n <= 16) break;   // the coarsest level (<= 48^3 nodes) is solved exactly
    n /= 2;
  }
  const size_t es = H.elem_size;
  for (size_t l = 0; l < H.lv.size(); ++l) {
    Level& L = H.lv[l];
    const bool coarsest = l + 1 == H.lv.size();
    // level 0 solves for the CG vectors (no x, b of its own); the coarsest
    // level neither smooths nor restricts (no r, d, a)
    void** bufs[] = {l > 0 ? &L.x : nullptr, l > 0 ? &L.b : nullptr, coarsest ? nullptr : &L.r,
                     coarsest ? nullptr : &L.d, &L.t1, &L.t2, coarsest ? nullptr : &L.a};
    for (void** p : bufs) {
      if (!p) continue;
      cudaError_t e = cudaMalloc(p, L.size * es);
      if (e != cudaSuccess) return e;
    }
  }
  // coarsest level: exact inverse by fast diagonalisation of the 1-D pencil
  const Level& Lc = H.lv.back();
  const int N = Lc.N;
  std::vector<double> K1((size_t)N * N, 0.0), M1((size_t)N * N, 0.0);
  for (int g = 0; g < N; ++g)
    for (int j = -3; j <= 3; ++j) {
      int h = ((g + j) % N + N) % N;
      K1[(size_t)g * N + h] += c->st.K[g % 3][j + 3];
      M1[(size_t)g * N + h] += c->st.M[g % 3][j + 3];
    }
  std::vector<double> lam, V;
  generalized_eigen(N, K1, M1, lam, V);
  int null = 0;
  for (int i = 1; i < N; ++i)
    if (std::fabs(lam[i]) < std::fabs(lam[null])) null = i;
  std::vector<float> D32((size_t)N * N * N);
  for (int k = 0; k < N; ++k)
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) {
        double D = lam[i] + lam[j] + lam[k];
        D32[i + (size_t)N * (j + (size_t)N * k)] = (i == null && j == null && k == null) ? 0.0f : (float)(1.0 / D);
      }
  CoarseSolver& cs = H.coarse;
  cs.N = N;
  cudaError_t e;
  std::vector<float> V32(V.begin(), V.end()), VT32((size_t)N * N);
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < N; ++k) VT32[(size_t)i * N + k] = (float)V[(size_t)k * N + i];
  if ((e = cudaMalloc(&cs.V32, V32.size() * 4)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&cs.VT32, VT32.size() * 4)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&cs.Dinv32, D32.size() * 4)) != cudaSuccess) return e;
  cudaMemcpy(cs.V32, V32.data(), V32.size() * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(cs.VT32, VT32.data(), VT32.size() * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(cs.Dinv32, D32.data(), D32.size() * 4, cudaMemcpyHostToDevice);
  H.lmax = estimate_lmax(c->st, 6);
  if (!(c->cfg.flags & FEP3M_MULTIGRID)) {
    // fine level by fast diagonalisation (block-Fourier eigenbasis, O(N^2) on the host)
    const int Nf = 3 * c->n;
    std::vector<double> lamf, Vf;
    periodic_eigen(c->n, c->st, lamf, Vf);
    if ((e = fdm_setup(H.fdm, Nf, lamf, Vf, c->nv, !(c->cfg.flags & FEP3M_CUDA_CORES))) != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

static void mg_free(Solver* c) {
  for (Level& L : c->mg.lv) {
    void* bufs[] = {L.x, L.b, L.r, L.d, L.t1, L.t2, L.a};
    for (void* p : bufs)
      if (p) cudaFree(p);
  }
  c->mg.lv.clear();
  fdm_free(c->mg.fdm);
  CoarseSolver& cs = c->mg.coarse;
  if (cs.VT32) cudaFree(cs.VT32);
  if (cs.V32) cudaFree(cs.V32);
  if (cs.Dinv32) cudaFree(cs.Dinv32);
  cs = CoarseSolver();
}

static void free_list(void** p, int k) {
  for (int i = 0; i < k; ++i)
    if (p[i]) {
      cudaFree(p[i]);
      p[i] = nullptr;
    }
}

static void solver_free(Solver* c) {
  free_list(c->sb, 6);
  c->sb_bytes = 0;
}

// PCG work vectors r, z, p, q, x, rhs in the working precision (level-0 size);
// the four the fast-diagonalisation refinement uses (r, z, x, rhs) once per
// right-hand side of the paired solve
static cudaError_t ensure_solver_buffers(Solver* c) {
  const size_t bytes = c->mg.lv[0].size * c->mg.elem_size;
  if (c->sb_bytes == bytes) return cudaSuccess;
  free_list(c->sb, 6);
  for (int i = 0; i < 6; ++i) {
    const size_t m = (i == 0 || i == 1 || i == 4 || i == 5) ? (size_t)c->nv : 1;
    cudaError_t e = cudaMalloc(&c->sb[i], bytes * m);
    if (e != cudaSuccess) return e;
  }
  c->sb_bytes = bytes;
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Iterative refinement.  Both precisions solve K e = r for corrections with the
// FP32 multigrid-preconditioned CG; the iterate, Pi b and the residual
// r = Pi b - K phi are kept in a wider format: double-float (MIXED) or FP64
// (FP64).  Every residual handed to the FP32 solve is scaled by one power of
// two s (2^-k with 2^k near the RMS of b), so its range suits FP32 whatever
// the units of b.
//   MIXED: Pi b in res64 and the iterate in phidf, as float pairs
//   FP64:  Pi b in res64 and the iterate in the output buffer, FP64

// 1 / W (W = n^3 elements): the mean's factor of the integral
static double apply_invW(const Solver* c) {
  const Level& L0 = c->mg.lv[0];
  return 1.0 / ((double)L0.n * L0.n * L0.n);
}

// r = s (Pi b - K phi) in FP32; norm_out (MIXED): |r|^2 accumulated by the
// apply into norm_out (per right-hand side at norm_out + 64 v); e_first
// (MIXED, the first sweep): phi is e_first / s, read from the FP32
// correction and written to the iterate by the apply (no update launch)
static cudaError_t refine_resid(Solver* c, const double* phi64, float* r, double* norm_out = nullptr,
                                const float* e_first = nullptr, double* wsum_out = nullptr) {
  const Level& L0 = c->mg.lv[0];
  const int N = L0.N;
  const int steps = apply_steps(N);
  const ApplyDot nd = {nullptr, nullptr, nullptr, 0};
  dim3 grid = apply_grid(N, steps);
  grid.z *= c->V;
  if (c->precision == FEP3M_FP64) {
    launch_pdl(k_apply_el<double, EPI_RESID>, grid, AT, sizeof(ApplySmem<double, EPI_RESID>), c->stream, N, steps,
               phi64, reinterpret_cast<double*>(r), c->res64, nullptr, nullptr, 0.0, 0.0, 0.0, c->scal, nd, c->vs);
  } else if (e_first) {
    const dfv z = {0.0f, 0.0f};
    const dfv* xin = reinterpret_cast<const dfv*>(e_first);   // read as floats (F32IN)
    dfv* it = reinterpret_cast<dfv*>(c->phidf);
    if (norm_out) {
      const ApplyDot dt = {(double*)c->red_tmp, c->red_counter, norm_out, POST_NONE, wsum_out, apply_invW(c)};
      launch_pdl(k_apply_el<dfv, EPI_RESID, true, true>, grid, AT, sizeof(ApplySmem<dfv, EPI_RESID, true>),
                 c->stream, N, steps, xin, reinterpret_cast<dfv*>(r), reinterpret_cast<const dfv*>(c->res64),
                 (dfv*)nullptr, it, z, z, z, c->scal, dt, c->vs);
    } else {
      launch_pdl(k_apply_el<dfv, EPI_RESID, false, true>, grid, AT, sizeof(ApplySmem<dfv, EPI_RESID>), c->stream,
                 N, steps, xin, reinterpret_cast<dfv*>(r), reinterpret_cast<const dfv*>(c->res64), (dfv*)nullptr,
                 it, z, z, z, c->scal, nd, c->vs);
    }
  } else if (norm_out) {
    const dfv z = {0.0f, 0.0f};
    const ApplyDot dt = {(double*)c->red_tmp, c->red_counter, norm_out, POST_NONE, wsum_out, apply_invW(c)};
    launch_pdl(k_apply_el<dfv, EPI_RESID, true>, grid, AT, sizeof(ApplySmem<dfv, EPI_RESID, true>), c->stream, N,
               steps, reinterpret_cast<const dfv*>(c->phidf), reinterpret_cast<dfv*>(r),
               reinterpret_cast<const dfv*>(c->res64), nullptr, nullptr, z, z, z, c->scal, dt, c->vs);
  } else {
    const dfv z = {0.0f, 0.0f};
    launch_pdl(k_apply_el<dfv, EPI_RESID>, grid, AT, sizeof(ApplySmem<dfv, EPI_RESID>), c->stream, N, steps,
               reinterpret_cast<const dfv*>(c->phidf), reinterpret_cast<dfv*>(r),
               reinterpret_cast<const dfv*>(c->res64), nullptr, nullptr, z, z, z, c->scal, nd, c->vs);
  }
  return cudaGetLastError();
}

// start: Pi b, the scale s, phi = 0 (FP64; MIXED: the first update assigns),
// r = s Pi b in FP32 and |r|^2 into scal[10]
static void refine_setup(Solver* c, const double* b, double* phi64, float* r) {
  const Level& L0 = c->mg.lv[0];
  const int N = L0.N;
  const size_t n = L0.size;
  const double W = (double)L0.n * L0.n * L0.n;
  cudaStream_t s = c->stream;
  double* sc = c->scal;
  if (c->precision != FEP3M_FP64) {
    // b as float pairs
    const dim3 gr((unsigned)reduce_blocks(n), (unsigned)c->V);
    const dfv* bd = reinterpret_cast<const dfv*>(b);
    launch_pdl(k_ref_sums, gr, TPB, 0, s, (int64_t)n, bd, (double*)c->red_tmp, c->red_counter, sc, 1.0 / W, c->vs);
    launch_pdl(k_ref_project_scale, gr, TPB, 0, s, N, bd, reinterpret_cast<dfv*>(c->res64), r, (double*)c->red_tmp,
               c->red_counter, sc, c->vs);
    return;
  }
  reduce<double>(c, N, RD_SUM, b, nullptr, sc + 5, POST_MEAN, 1.0 / W);
  reduce<double>(c, N, RD_NORM2, b, nullptr, sc + 7, POST_SCALE, 1.0 / (double)n);
  const int bx = std::min(N, 256);
  const int V = c->V;
  const int64_t vs = c->vs;
  const dim3 g3((N + bx - 1) / bx, N * V, N);
  const dim3 gr((unsigned)reduce_blocks(n), (unsigned)V);
  launch_pdl(k_project_copy64, g3, bx, 0, s, N, b, sc, c->res64, vs);
  for (int v = 0; v < V; ++v) cudaMemsetAsync(phi64 + v * vs, 0, n * sizeof(double), s);
  launch_pdl(k_round_scaled_norm, gr, TPB, 0, s, (int64_t)n, (const double*)c->res64, r, (double*)c->red_tmp,
             c->red_counter, sc + 10, sc, vs);
}

// phi += e / s (MIXED: after the first sweep, whose apply formed phi)
static void refine_update(Solver* c, double* phi64, const float* e) {
  const size_t n = c->mg.lv[0].size;
  const dim3 g((unsigned)grid_for(n), (unsigned)c->V);
  if (c->precision == FEP3M_FP64)
    launch_pdl(k_add_scaled, g, TPB, 0, c->stream, (int64_t)n, phi64, e, c->scal, c->vs);
  else
    launch_pdl(k_df_update, g, TPB, 0, c->stream, (int64_t)n, reinterpret_cast<dfv*>(c->phidf), e, c->scal, c->vs);
}

// end: phi with mean zero (FP64; MIXED: float pairs); have_mean: the last
// residual apply already summed the integral and derived the mean
static void refine_finish(Solver* c, double* phi, bool have_mean = false) {
  const Level& L0 = c->mg.lv[0];
  const int N = L0.N;
  const size_t n = L0.size;
  const double W = (double)L0.n * L0.n * L0.n;
  if (c->precision != FEP3M_FP64) {
    const dfv* v = reinterpret_cast<const dfv*>(c->phidf);
    if (!have_mean)
      launch_pdl(k_ref_wsum, dim3((unsigned)reduce_blocks(n), (unsigned)c->V), TPB, 0, c->stream, N, v,
               (double*)c->red_tmp, c->red_counter, c->scal, 1.0 / W, c->vs);
    launch_pdl(k_ref_out, dim3((unsigned)grid_for(n), (unsigned)c->V), TPB, 0, c->stream, (int64_t)n, v,
               reinterpret_cast<dfv*>(phi), (const double*)c->scal, c->vs);
    return;
  }
  reduce<double>(c, N, RD_WSUM, phi, nullptr, c->scal + 6, POST_MEAN, 1.0 / W);
  project<double>(c, N, phi, 1);
}

static double solver_rtol(const Solver* c) {
  return c->cfg.mg_rtol > 0 ? c->cfg.mg_rtol : (c->precision == FEP3M_FP64 ? 1e-13 : 1e-10);
}

// host-checked solve (used once to calibrate the iteration counts, and as the
// fallback when a replayed solve misses its tolerance)
static cudaError_t solve_checked(Solver* c, const double* b, double* phi, int* iters, double* relres,
                                 int* refine_steps, int* k_inner_max) {
  void** sb = c->sb;   // r, z, p, q, x, rhs
  const Level& L0 = c->mg.lv[0];
  const int N = L0.N;
  cudaStream_t s = c->stream;
  double* sc = c->scal;
  *refine_steps = 0;
  *k_inner_max = 0;
  *iters = 0;
  *relres = 0;
  MG<float> mg(c);
  const double rtol = solver_rtol(c);
  const int maxout = c->cfg.mg_max_cycles > 0 ? c->cfg.mg_max_cycles : 10;
  float* r32 = (float*)sb[5];
  float* e32 = (float*)sb[4];
  refine_setup(c, b, phi, r32);   // |r|^2 into sc[10]
  double bb = 0;
  cudaMemcpyAsync(&bb, sc + 10, sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if (bb == 0.0) {
    if (c->phidf) cudaMemsetAsync(c->phidf, 0, L0.size * sizeof(dfv), s);
    refine_finish(c, phi);
    return cudaGetLastError();
  }
  double rr = bb;
  int step = 0;
  const bool fdm = c->mg.fdm.N > 0;
  for (step = 0; step < maxout; ++step) {
    double inner_res = 0;
    int it = 1;
    if (fdm) mg.fdm_solve(r32, e32, (float*)sb[0], (float*)sb[1]);
    else it = mg.pcg(r32, e32, (float*)sb[0], (float*)sb[1], (float*)sb[2], (float*)sb[3], 1e-5, 30, &inner_res);
    *iters += it;
    *k_inner_max = std::max(*k_inner_max, it);
    // MIXED, first sweep: the residual's apply forms the iterate e / s itself
    const bool first_df = c->precision != FEP3M_FP64 && step == 0;
    if (!first_df) refine_update(c, phi, e32);
    // the residual's sum is rounding noise (K has zero column sums), and the
    // inner solve projects its right-hand side: no projection here
    cudaError_t e = refine_resid(c, phi, r32, nullptr, first_df ? e32 : nullptr);
    if (e != cudaSuccess) return e;
    reduce<float>(c, N, RD_NORM2, r32, nullptr, sc + 9);
    cudaMemcpyAsync(&rr, sc + 9, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (rr <= rtol * rtol * bb) {
      ++step;
      break;
    }
  }
  *refine_steps = step;
  *relres = std::sqrt(rr / bb);
  refine_finish(c, phi);
  return cudaGetLastError();
}

// fixed-count solve of the c->V right-hand sides at b (stride c->vs) into phi
// with kout refinement sweeps, no host round trip; leaves |s Pi b|^2 in
// scal[10] and the final scaled residual |r|^2 in scal[11] (scal[64 v + ...]
// for right-hand side v)
static cudaError_t solve_fixed(Solver* c, const double* b, double* phi, int kout) {
  void** sb = c->sb;
  const Level& L0 = c->mg.lv[0];
  const int N = L0.N;
  double* sc = c->scal;
  MG<float> mg(c);
  float* r32 = (float*)sb[5];
  float* e32 = (float*)sb[4];
  refine_setup(c, b, phi, r32);   // |r|^2 into sc[10]
  const bool mixed = c->precision != FEP3M_FP64;
  for (int step = 0; step < kout; ++step) {
    if (step == 0 && c->ev_in0) cudaEventRecordWithFlags(c->ev_in0, c->stream, cudaEventRecordExternal);
    if (c->mg.fdm.N > 0) mg.fdm_solve(r32, e32, (float*)sb[0], (float*)sb[1]);
    else mg.pcg_fixed(r32, e32, (float*)sb[0], (float*)sb[1], (float*)sb[2], (float*)sb[3], c->plan_kin);
    if (step == 0 && c->ev_in1) cudaEventRecordWithFlags(c->ev_in1, c->stream, cudaEventRecordExternal);
    // MIXED: the first sweep's apply forms the iterate e / s itself, and the
    // last residual's |r|^2 is accumulated by its apply
    const bool first_df = mixed && step == 0;
    if (!first_df) refine_update(c, phi, e32);
    const bool last = mixed && step == kout - 1;   // also the iterate's integral, for the finish
    cudaError_t e = refine_resid(c, phi, r32, last ? sc + 11 : nullptr, first_df ? e32 : nullptr, last ? sc + 6 : nullptr);
    if (e != cudaSuccess) return e;
  }
  if (mixed && kout == 0)
    cudaMemsetAsync(c->phidf, 0, (c->V > 1 ? c->V * c->vs : (int64_t)L0.size) * sizeof(dfv), c->stream);
  if (!mixed || kout == 0) reduce<float>(c, N, RD_NORM2, r32, nullptr, sc + 11);
  refine_finish(c, phi, mixed && kout > 0);
  return cudaGetLastError();
}

static void destroy_plan(Solver* c) {
  if (c->solve_exec) cudaGraphExecDestroy(c->solve_exec);
  c->solve_exec = nullptr;
  c->solve_graph_kernels = 0;
}

static void destroy_plan2(Solver* c) {
  if (c->solve2_exec) cudaGraphExecDestroy(c->solve2_exec);
  c->solve2_exec = nullptr;
  c->solve2_graph_kernels = 0;
}

// capture solve_fixed into a graph on the library's private stream: one
// right-hand side from c->in64 into c->out64, or (paired) the two at
// c->plan2_b into c->plan2_phi
static cudaError_t build_plan(Solver* c, bool paired = false) {
  if (paired) destroy_plan2(c);
  else destroy_plan(c);
  cudaGraphExec_t* exec = paired ? &c->solve2_exec : &c->solve_exec;
  int* kernels = paired ? &c->solve2_graph_kernels : &c->solve_graph_kernels;
  cudaStream_t user = c->stream;
  const bool unc = t_uncounted;
  t_uncounted = true;   // captured launches run (and count) when the graph is replayed
  c->stream = c->cap_stream;
  if (paired) {
    c->V = 2;
    c->vs = (int64_t)c->mg.lv[0].size;
  }
  cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e1 = paired ? solve_fixed(c, c->plan2_b, c->plan2_phi, c->plan2_kout)
                            : solve_fixed(c, c->in64, c->out64, c->plan_kout);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->cap_stream, &g);
    if (e == cudaSuccess) e = e1;
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
    if (g) {
      size_t nn = 0;
      cudaGraphGetNodes(g, nullptr, &nn);
      std::vector<cudaGraphNode_t> nodes(nn);
      if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
      int kn = 0;
      for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kn;
      }
      *kernels = kn;
      cudaGraphDestroy(g);
    }
  }
  c->V = 1;
  c->vs = 0;
  c->stream = user;
  t_uncounted = unc;
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    if (paired) destroy_plan2(c);
    else destroy_plan(c);
  }
  return e;
}

// synchronous calibrated solve; records the counts and captures the replay graph
static cudaError_t solve_calibrate(Solver* c, const double* b, double* phi) {
  int kin = 0;
  cudaError_t e = solve_checked(c, b, phi, &c->iters, &c->relres, &c->refine_steps, &kin);
  if (e != cudaSuccess || c->relres > solver_rtol(c)) return e;
  c->plan_kin = std::max(c->plan_kin, kin);
  c->plan_kout = std::max(c->plan_kout, c->refine_steps);
  const size_t n = c->mg.lv[0].size;
  if (!c->in64 && (e = cudaMalloc(&c->in64, n * sizeof(double))) != cudaSuccess) return e;
  if (!c->out64 && (e = cudaMalloc(&c->out64, n * sizeof(double))) != cudaSuccess) return e;
  if (!c->cap_stream && (e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return e;
  if (build_plan(c) != cudaSuccess) (void)cudaGetLastError();   // keep the checked path if capture fails
  return cudaSuccess;
}

cudaError_t mesh_solve_begin(Solver* c, const double* b, double* phi) {
  cudaError_t e = ensure_solver_buffers(c);
  if (e != cudaSuccess) return e;
  c->pending = false;
  if (!c->solve_exec) return solve_calibrate(c, b, phi);
  const size_t n = c->mg.lv[0].size;
  cudaStream_t s = c->stream;
  cudaMemcpyAsync(c->in64, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if ((e = cudaGraphLaunch(c->solve_exec, s)) != cudaSuccess) return e;
  count_launches((unsigned long long)c->solve_graph_kernels);
  cudaMemcpyAsync(phi, c->out64, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(c->host_res, c->scal + 10, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  c->pending = true;
  c->pend_b = b;
  c->pend_phi = phi;
  return cudaGetLastError();
}

bool mesh_solve_check(Solver* c) {
  if (!c->pending) return true;
  c->pending = false;
  const double bb = c->host_res[0], rr = c->host_res[1];
  const double rel = bb > 0 ? std::sqrt(rr / bb) : 0.0;
  if (rel <= solver_rtol(c)) {
    c->relres = rel;
    c->iters = c->plan_kin * c->plan_kout;
    c->refine_steps = c->plan_kout;
    return true;
  }
  // this right-hand side needs more iterations: one more sweep from now on,
  // and the next solve re-calibrates
  ++c->plan_kout;
  destroy_plan(c);
  return false;
}

cudaError_t mesh_solve_end(Solver* c) {
  if (!c->pending) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return e;
  if (mesh_solve_check(c)) return cudaSuccess;
  return solve_calibrate(c, c->pend_b, c->pend_phi);
}

cudaError_t mesh_solve(Solver* c, const double* b, double* phi) {
  cudaError_t e = mesh_solve_begin(c, b, phi);
  if (e != cudaSuccess) return e;
  return mesh_solve_end(c);
}

bool mesh_solve_paired(const Solver* c) { return c->nv == 2 && c->mg.fdm.BpF != nullptr; }

cudaError_t mesh_solve_begin2(Solver* c, const double* b, double* phi) {
  if (!mesh_solve_paired(c)) return cudaErrorInvalidValue;
  cudaError_t e = ensure_solver_buffers(c);
  if (e != cudaSuccess) return e;
  c->pending2 = false;
  const size_t n = c->mg.lv[0].size;
  if (!c->solve2_exec || c->plan2_b != b || c->plan2_phi != phi) {
    // calibrate: each right-hand side by the host-checked solve, then capture the pair
    int kin0 = 0, kin1 = 0;
    e = solve_checked(c, b, phi, &c->iters, &c->relres, &c->refine_steps, &kin0);
    if (e != cudaSuccess) return e;
    e = solve_checked(c, b + n, phi + n, &c->iters2, &c->relres2, &c->refine_steps2, &kin1);
    if (e != cudaSuccess) return e;
    if (c->relres > solver_rtol(c) || c->relres2 > solver_rtol(c)) return cudaSuccess;
    c->plan_kin = std::max(c->plan_kin, std::max(kin0, kin1));
    c->plan2_kout = std::max(c->plan2_kout, std::max(c->refine_steps, c->refine_steps2));
    c->plan2_b = b;
    c->plan2_phi = phi;
    if (!c->cap_stream && (e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
      return e;
    if (build_plan(c, true) != cudaSuccess) (void)cudaGetLastError();   // calibrate again next time
    return cudaSuccess;
  }
  cudaStream_t s = c->stream;
  if ((e = cudaGraphLaunch(c->solve2_exec, s)) != cudaSuccess) return e;
  count_launches((unsigned long long)c->solve2_graph_kernels);
  cudaMemcpyAsync(c->host_res, c->scal + 10, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(c->host_res + 2, c->scal + 64 + 10, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  c->pending2 = true;
  return cudaGetLastError();
}

bool mesh_solve_check2(Solver* c) {
  if (!c->pending2) return true;
  c->pending2 = false;
  double rel[2];
  for (int v = 0; v < 2; ++v) {
    const double bb = c->host_res[2 * v], rr = c->host_res[2 * v + 1];
    rel[v] = bb > 0 ? std::sqrt(rr / bb) : 0.0;
  }
  if (rel[0] <= solver_rtol(c) && rel[1] <= solver_rtol(c)) {
    c->relres = rel[0];
    c->relres2 = rel[1];
    c->iters = c->iters2 = std::max(1, c->plan_kin) * c->plan2_kout;
    c->refine_steps = c->refine_steps2 = c->plan2_kout;
    return true;
  }
  // a right-hand side needs more sweeps: one more from now on, calibrated on the next call
  ++c->plan2_kout;
  destroy_plan2(c);
  return false;
}

static void solver_plan_free(Solver* c) {
  destroy_plan(c);
  destroy_plan2(c);
  if (c->in64) cudaFree(c->in64);
  if (c->out64) cudaFree(c->out64);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  c->in64 = c->out64 = nullptr;
  c->cap_stream = nullptr;
}

// Device data of a fast-diagonalisation solve on an N^3 periodic mesh from the
// 1-D generalized eigenpairs (lamf, Vf[node * N + mode], M-orthonormal): the
// FP32 eigenbasis for the CUDA-core passes and, with tensor_cores, its bf16
// pieces in the layout of the tensor-core row GEMM (column tiles of nt modes,
// chunks of 64 nodes).  Used by the order-3 fine level and the order-p mesh.
cudaError_t fdm_setup(FineFDM& f, int Nf, const std::vector<double>& lamf, const std::vector<double>& Vf,
                      int rhs,
                      bool tensor_cores, bool null_mode) {
  cudaError_t e;
  {
    // the constant mode of a periodic (or fully Neumann) mesh: the eigenvalue
    // nearest 0, dropped from the solve; none for Dirichlet data
    f.null_mode = null_mode ? 0 : -1;
    if (null_mode)
      for (int i = 1; i < Nf; ++i)
        if (std::fabs(lamf[i]) < std::fabs(lamf[f.null_mode])) f.null_mode = i;
    std::vector<float> Vf32(Vf.begin(), Vf.end()), VTf32((size_t)Nf * Nf), lf32(lamf.begin(), lamf.end());
    for (int i = 0; i < Nf; ++i)
      for (int k = 0; k < Nf; ++k) VTf32[(size_t)k * Nf + i] = (float)Vf[(size_t)i * Nf + k];
    if ((e = cudaMalloc(&f.V32, Vf32.size() * 4)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&f.VT32, VTf32.size() * 4)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&f.lam32, lf32.size() * 4)) != cudaSuccess) return e;
    cudaMemcpy(f.V32, Vf32.data(), Vf32.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(f.VT32, VTf32.data(), VTf32.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(f.lam32, lf32.data(), lf32.size() * 4, cudaMemcpyHostToDevice);
    f.N = Nf;
    if (tensor_cores) {
      // column tiles of nt modes (a multiple of 16, <= 128: two CTAs per SM); where the rows are few, the
      // tile count that brings a pass (rows x tiles x right-hand sides CTAs) nearest one CTA per SM
      // (measured on the paired 32^3 solve: one tile of 96 modes, 144 CTAs, 0.629 ms a step against 0.656
      // with three; tiles of 192 or 256 modes, one CTA per SM, read the input fewer times but were no
      // faster at 128^3, nor one tile at 64^3)
      const int64_t rt = ((int64_t)Nf * Nf + 127) / 128;
      const int64_t rows = rt * std::max(1, rhs);
      int ntile = std::max<int>((Nf + 127) / 128, (int)std::max<int64_t>(1, (152 + rows / 2) / rows));
      const int nt = ((Nf + ntile - 1) / ntile + 15) / 16 * 16;
      ntile = (Nf + nt - 1) / nt;
      const int kc = (Nf + 63) / 64;
      const size_t per = (size_t)3 * nt * 64;   // bf16 values per (tile, chunk)
      std::vector<uint16_t> bf((size_t)ntile * kc * per), bi((size_t)ntile * kc * per);
      for (int t = 0; t < ntile; ++t)
        for (int ch = 0; ch < kc; ++ch)
          for (int ii = 0; ii < nt; ++ii)
            for (int k = 0; k < 64; ++k) {
              const int i = t * nt + ii, a = 64 * ch + k;
              const bool in = i < Nf && a < Nf;
              uint16_t pf[3] = {0, 0, 0}, pi[3] = {0, 0, 0};
              if (in) {
                tc::bf16_pieces(Vf[(size_t)a * Nf + i], pf);   // analysis: B[i][a] = V[a][i]
                tc::bf16_pieces(Vf[(size_t)i * Nf + a], pi);   // synthesis: B[i][a] = V[i][a]
              }
              for (int p = 0; p < 3; ++p) {
                const size_t o = ((size_t)(t * kc + ch) * 3 + p) * nt * 64 + tc::sw128_off(ii, k) / 2;
                bf[o] = pf[p];
                bi[o] = pi[p];
              }
            }
      if ((e = cudaMalloc(&f.BpF, bf.size() * 2)) != cudaSuccess) return e;
      if ((e = cudaMalloc(&f.BpI, bi.size() * 2)) != cudaSuccess) return e;
      cudaMemcpy(f.BpF, bf.data(), bf.size() * 2, cudaMemcpyHostToDevice);
      cudaMemcpy(f.BpI, bi.data(), bi.size() * 2, cudaMemcpyHostToDevice);
      f.nt = nt;
      f.ntile = ntile;
      if ((e = tc_rows_prepare(nt)) != cudaSuccess) return e;
      if ((e = cudaMalloc(&f.err, sizeof(int))) != cudaSuccess) return e;
      cudaMemset(f.err, 0, sizeof(int));
    }
  }
  return cudaGetLastError();
}

void fdm_free(FineFDM& f) {
  void* p[] = {f.BpF, f.BpI, f.err, f.V32, f.VT32, f.lam32};
  for (void* q : p)
    if (q) cudaFree(q);
  f = FineFDM();
}

// x = K^+ b by the six transform passes (tensor cores when the pieces are
// set, else the CUDA-core passes); w1, w2: N^3 scratch
cudaError_t fdm_apply(const FineFDM& f, const float* b, float* x, float* w1, float* w2, cudaStream_t s, int V,
                      int64_t vs) {
  const int N = f.N;
  if (f.BpF) {
    const dim3 g((unsigned)(((int64_t)N * N + 127) / 128 * f.ntile), (unsigned)V);
    const size_t sm = tc_rows_smem(f.nt);
    const uint4* F = (const uint4*)f.BpF;
    const uint4* I = (const uint4*)f.BpI;
    const int64_t R = (int64_t)N * N;
    const float* lm = f.lam32;
    const int nm = f.null_mode, nt = f.nt;
    auto k0 = k_tc_rows<false>;
    auto k1 = k_tc_rows<true>;
    launch_pdl(k0, g, FT_THREADS, sm, s, R, N, 0, N, nt, b, F, lm, nm, N, w1, f.err, vs);
    launch_pdl(k0, g, FT_THREADS, sm, s, R, N, 0, N, nt, (const float*)w1, F, lm, nm, N, w2, f.err, vs);
    launch_pdl(k1, g, FT_THREADS, sm, s, R, N, 0, N, nt, (const float*)w2, F, lm, nm, N, w1, f.err, vs);
    launch_pdl(k0, g, FT_THREADS, sm, s, R, N, 0, N, nt, (const float*)w1, I, lm, nm, N, w2, f.err, vs);
    launch_pdl(k0, g, FT_THREADS, sm, s, R, N, 0, N, nt, (const float*)w2, I, lm, nm, N, w1, f.err, vs);
    launch_pdl(k0, g, FT_THREADS, sm, s, R, N, 0, N, nt, (const float*)w1, I, lm, nm, N, x, f.err, vs);
    return cudaGetLastError();
  }
  if (V != 1) return cudaErrorInvalidValue;   // one vector on the CUDA-core passes
  const dim3 g((unsigned)(((int64_t)N * N + FM - 1) / FM), (unsigned)((N + FN - 1) / FN));
  launch_pdl(k_fdm_axis<false>, g, 256, 0, s, N, b, f.V32, f.lam32, f.null_mode, w1);
  launch_pdl(k_fdm_axis<false>, g, 256, 0, s, N, (const float*)w1, f.V32, f.lam32, f.null_mode, w2);
  launch_pdl(k_fdm_axis<true>, g, 256, 0, s, N, (const float*)w2, f.V32, f.lam32, f.null_mode, w1);
  launch_pdl(k_fdm_axis<false>, g, 256, 0, s, N, (const float*)w1, f.VT32, f.lam32, f.null_mode, w2);
  launch_pdl(k_fdm_axis<false>, g, 256, 0, s, N, (const float*)w2, f.VT32, f.lam32, f.null_mode, w1);
  launch_pdl(k_fdm_axis<false>, g, 256, 0, s, N, (const float*)w1, f.VT32, f.lam32, f.null_mode, x);
  return cudaGetLastError();
}

cudaError_t solver_init(Solver* s, const fep3m_ctx* c, cudaStream_t stream, int nv) {
  s->cfg = c->cfg;
  s->n = c->n;
  s->precision = c->precision;
  s->st = c->st;
  s->stream = stream;
  s->nv = nv = std::max(1, std::min(2, nv));
  const size_t nodes = (size_t)27 * c->n * c->n * c->n;
  cudaError_t e;
  // per right-hand side: a block of 64 scalars, the reduction partials (one per block of
  // k_reduce (<= 608), two per block of k_ref_sums, up to two per block of a fine-level apply
  // with a fused dot), a counter, res64 and phidf
  if ((e = cudaMalloc(&s->scal, nv * 64 * sizeof(double))) != cudaSuccess) return e;
  {
    const int N0 = 3 * c->n;
    const dim3 g = apply_grid(N0, apply_steps(N0));
    const size_t nb = std::max<size_t>(2 * 608, 2 * (size_t)g.x * g.y * g.z);
    if ((e = cudaMalloc(&s->red_tmp, nv * nb * sizeof(double))) != cudaSuccess) return e;
  }
  if ((e = cudaMalloc(&s->red_counter, nv * sizeof(unsigned int))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&s->res64, nv * nodes * sizeof(double))) != cudaSuccess) return e;
  if (s->precision == FEP3M_MIXED && (e = cudaMalloc(&s->phidf, nv * nodes * sizeof(dfv))) != cudaSuccess) return e;
  if ((e = cudaMallocHost(&s->host_res, 4 * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&s->ev_in0)) != cudaSuccess || (e = cudaEventCreate(&s->ev_in1)) != cudaSuccess) return e;
  cudaMemset(s->red_counter, 0, nv * sizeof(unsigned int));
  cudaMemset(s->scal, 0, nv * 64 * sizeof(double));
  if ((e = apply_set_smem()) != cudaSuccess) return e;
  return mg_setup(s);
}

void solver_destroy(Solver* s) {
  if (s->ev_in0) cudaEventDestroy(s->ev_in0);
  if (s->ev_in1) cudaEventDestroy(s->ev_in1);
  s->ev_in0 = s->ev_in1 = nullptr;
  solver_plan_free(s);
  mg_free(s);
  solver_free(s);
  if (s->scal) cudaFree(s->scal);
  if (s->red_tmp) cudaFree(s->red_tmp);
  if (s->red_counter) cudaFree(s->red_counter);
  if (s->res64) cudaFree(s->res64);
  if (s->phidf) cudaFree(s->phidf);
  s->phidf = nullptr;
  if (s->host_res) cudaFreeHost(s->host_res);
  s->scal = s->red_tmp = s->res64 = s->host_res = nullptr;
  s->red_counter = nullptr;
}

cudaError_t element_lists(fep3m_ctx* c) {
  const int n = c->n;
  const int64_t ne = (int64_t)n * n * n;
  cudaStream_t s = c->stream;
  if (c->precision == FEP3M_MIXED) {
    FEP3M_CL k_elem_coeff<float><<<grid_for(ne), TPB, 0, s>>>(ne, c->start, c->count, (const float4*)c->part, (float*)c->C);
    FEP3M_CL k_vertex_density<float><<<grid_for(ne), TPB, 0, s>>>(n, (const float*)c->C, (float*)c->rv,
                                                                   (float*)c->Cv);
  } else {
    FEP3M_CL k_elem_coeff<double><<<grid_for(ne), TPB, 0, s>>>(ne, c->start, c->count, (const vec4<double>::type*)c->part, (double*)c->C);
    FEP3M_CL k_vertex_density<double><<<grid_for(ne), TPB, 0, s>>>(n, (const double*)c->C, (double*)c->rv,
                                                                    (double*)c->Cv);
  }
  return cudaGetLastError();
}

cudaError_t assemble_forward(fep3m_ctx* c) {
  const int n = c->n;
  cudaStream_t s = c->stream;
  cudaError_t e = element_lists(c);
  if (e != cudaSuccess) return e;
  // the load vector in three separable passes through the forward solver's
  // fine-level scratch (free until its solve, which follows on this stream)
  const Level& L0 = c->solv[0].mg.lv[0];
  const int N3 = 3 * n;
  if (c->precision == FEP3M_MIXED) {
    // b as float pairs (the mixed solver's right-hand side): the FP32 sums of the
    // integer-weighted passes times 4 pi / 120^3 as a two-product
    const double sc = 4.0 * M_PI / (120.0 * 120.0 * 120.0);
    const float sh = (float)sc, sl = (float)(sc - (double)sh);
    float *t1 = (float*)L0.t1, *t2 = (float*)L0.t2;
    FEP3M_CL k_load_axis<float, float><<<grid_for((int64_t)N3 * n * n), TPB, 0, s>>>(n, 0, N3, n, n, (const float*)c->rv,
                                                                                    t1, 1.0, 1.0f, 0.0f);
    FEP3M_CL k_load_axis<float, float><<<grid_for((int64_t)N3 * N3 * n), TPB, 0, s>>>(n, 1, N3, N3, n, t1, t2, 1.0,
                                                                                     1.0f, 0.0f);
    FEP3M_CL k_load_axis<float, dfv><<<grid_for((int64_t)N3 * N3 * N3), TPB, 0, s>>>(n, 2, N3, N3, N3, t2,
                                                                                    reinterpret_cast<dfv*>(c->b64), sc,
                                                                                    sh, sl);
  } else {
    double *t1 = (double*)L0.t1, *t2 = (double*)L0.t2;
    FEP3M_CL k_load_axis<double, double><<<grid_for((int64_t)N3 * n * n), TPB, 0, s>>>(n, 0, N3, n, n,
                                                                                      (const double*)c->rv, t1, 1.0,
                                                                                      1.0f, 0.0f);
    FEP3M_CL k_load_axis<double, double><<<grid_for((int64_t)N3 * N3 * n), TPB, 0, s>>>(n, 1, N3, N3, n, t1, t2, 1.0,
                                                                                       1.0f, 0.0f);
    FEP3M_CL k_load_axis<double, double><<<grid_for((int64_t)N3 * N3 * N3), TPB, 0, s>>>(n, 2, N3, N3, N3, t2, c->b64,
                                                                                        4.0 * M_PI, 1.0f, 0.0f);
  }
  return cudaGetLastError();
}

// mu = 4 pi (Mpq^T (x) Mpq^T (x) Mpq^T) lam (order-3 nodes -> vertices), three separable passes.
// One axis: vertex v collects order-3 nodes 3v-3 .. 3v+3.
template <class T>
__global__ void k_mpqT_axis(int axis, int n, int e0, int e1, int e2, const double* __restrict__ in64,
                            const T* __restrict__ inT, T* __restrict__ out, double scale) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t tot = (int64_t)e0 * e1 * e2;
  if (g >= tot) return;
  int i[3] = {(int)(g % e0), (int)((g / e0) % e1), (int)(g / ((int64_t)e0 * e1))};
  int ein[3] = {e0, e1, e2};
  const int N = 3 * n;
  ein[axis] = N;
  const int64_t st[3] = {1, ein[0], (int64_t)ein[0] * ein[1]};
  const int v = i[axis];
  i[axis] = 0;
  const int64_t base = i[0] * st[0] + i[1] * st[1] + i[2] * st[2];
  const double w[7] = {cMpq64[0][1], cMpq64[1][1], cMpq64[2][1], cMpq64[3][1] + cMpq64[0][0],
                       cMpq64[1][0], cMpq64[2][0], cMpq64[3][0]};
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    int gg = 3 * v - 3 + k;
    gg = gg < 0 ? gg + N : (gg >= N ? gg - N : gg);
    const double val = in64 ? in64[base + gg * st[axis]] : (double)inT[base + gg * st[axis]];
    acc += w[k] * val;
  }
  out[g] = (T)(scale * acc);
}

// MIXED: the same passes on float pairs (lam as float pairs, the mixed solver's
// output) with the integer weights (times 120; w v as a two-product, the sums
// as two-sums); the last pass (Tout = double) forms mu = scale (h + l) in FP64
template <class Tout>
__global__ void k_mpqT_axis_df(int axis, int n, int e0, int e1, int e2, const dfv* __restrict__ in,
                               Tout* __restrict__ out, double scale) {
  const unsigned g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (unsigned)e0 * (unsigned)e1 * (unsigned)e2) return;
  const unsigned q = g / (unsigned)e0;
  int i[3] = {(int)(g - q * (unsigned)e0), (int)(q % (unsigned)e1), (int)(q / (unsigned)e1)};
  int ein[3] = {e0, e1, e2};
  const int N = 3 * n;
  ein[axis] = N;
  const int64_t st[3] = {1, ein[0], (int64_t)ein[0] * ein[1]};
  const int v = i[axis];
  i[axis] = 0;
  const int64_t base = i[0] * st[0] + i[1] * st[1] + i[2] * st[2];
  const float w[7] = {cMpq120[0][1], cMpq120[1][1], cMpq120[2][1], cMpq120[3][1] + cMpq120[0][0],
                      cMpq120[1][0], cMpq120[2][0], cMpq120[3][0]};
  dfv acc = {0.f, 0.f};
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    int gg = 3 * v - 3 + k;
    gg = gg < 0 ? gg + N : (gg >= N ? gg - N : gg);
    const dfv x = in[base + gg * st[axis]];
    const float p = w[k] * x.h;
    acc += dfv{p, fmaf(w[k], x.l, fmaf(w[k], x.h, -p))};
  }
  if constexpr (std::is_same<Tout, dfv>::value) out[g] = df_norm(acc);
  else out[g] = scale * ((double)acc.h + (double)acc.l);
}

cudaError_t vertex_adjoint(fep3m_ctx* c, const double* lam, void* mu, void* work1, void* work2, cudaStream_t s) {
  // mu in FP64 in both precisions: it meets the screen adjoint in a difference
  // that cancels; the two partial passes (9 n^3 and 3 n^3 values) fit as
  // doubles (or float pairs) in work buffers of (3n)^3 floats
  const int n = c->n, N = 3 * n;
  if (c->precision == FEP3M_MIXED) {   // lam as float pairs
    const dfv* l = reinterpret_cast<const dfv*>(lam);
    dfv *w1 = (dfv*)work1, *w2 = (dfv*)work2;
    FEP3M_CL k_mpqT_axis_df<dfv><<<grid_for((size_t)n * N * N), TPB, 0, s>>>(0, n, n, N, N, l, w1, 1.0);
    FEP3M_CL k_mpqT_axis_df<dfv><<<grid_for((size_t)n * n * N), TPB, 0, s>>>(1, n, n, n, N, w1, w2, 1.0);
    FEP3M_CL k_mpqT_axis_df<double><<<grid_for((size_t)n * n * n), TPB, 0, s>>>(2, n, n, n, n, w2, (double*)mu,
                                                                              4.0 * M_PI / (120.0 * 120.0 * 120.0));
    return cudaGetLastError();
  }
  FEP3M_CL k_mpqT_axis<double><<<grid_for((size_t)n * N * N), TPB, 0, s>>>(0, n, n, N, N, lam, nullptr, (double*)work1, 1.0);
  FEP3M_CL k_mpqT_axis<double><<<grid_for((size_t)n * n * N), TPB, 0, s>>>(1, n, n, n, N, nullptr, (double*)work1, (double*)work2, 1.0);
  FEP3M_CL k_mpqT_axis<double><<<grid_for((size_t)n * n * n), TPB, 0, s>>>(2, n, n, n, n, nullptr, (double*)work2, (double*)mu, 4.0 * M_PI);
  return cudaGetLastError();
}

}  // namespace fep3m
