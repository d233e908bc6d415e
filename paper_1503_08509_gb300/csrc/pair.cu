// Short-range evaluation (Sec. 2.4-2.5) and the smooth-potential evaluation
// (Sec. 2.3, Eq. evalsmooth), and the reverse sweeps of the adjoint.
//
// For a target charge t in element e (local coordinate tau_t in [0,1]^3):
//   Phi_t = (1/h) sum_m G_e[m] u_m(tau_t) + sum_{j in block(e), j != t} Q_j / |x_j - x_t|
//   G_e[m] = phi[node(e, m)] - sum_{o} A_e(o) H(o, m)
// where the second term of G_e is the screen potential of every charge of the
// (2 n_sr + 1)^3 block around e (own charge included: the self term of
// Sec. 2.5), written at the 64 order-3 nodes of e.  It is the element-to-point
// evaluation of Sec. 3.1.2 (Eq. sc with per-element combined coefficients),
// regrouped by vertex: all screens are sums of vertex hats, every vertex hat
// has the same FE table H (Remark of Sec. 4), so the block's screens act
// through the vertex amplitudes
//   A_e(o) = sum over the corners k of block elements at vertex v = e - o of C[v - k][k]
// which equal the full vertex density r_v inside the block and partial sums on
// its boundary.  H(o, m) is the table value at node m of an element at offset
// o (element units) from the vertex.
//
// Two launches per evaluation: k_pair_screen (the screen field sum_o A_e(o)
// H(o, m) and the singular sums; it needs no mesh solution and runs while the
// mesh is solved) and k_pair_eval (G_e and the contraction with u_m(tau_t)
// after the solve).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "tc.cuh"

namespace fep3m {

namespace {

using namespace tc;
constexpr uint32_t UMMA_IDESC = umma_idesc(64, 64);   // the screen contraction: M = 64 elements, N = 64 nodes

constexpr int PT = 256;
constexpr int PTC = 512;   // threads of the tensor-core screen kernel

__device__ __forceinline__ int wrapn(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

template <class T> __device__ __forceinline__ T rsq(T x);
// the hardware estimate of 1 / sqrt(x) (PTX rsqrt.approx, relative error
// about 2^-23; subnormal input and output flushed to zero, which the
// squared distances of distinct charges never are)
__device__ __forceinline__ float rsqrt_est(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// 1 / sqrt(x) in FP64 from the FP32 hardware estimate y, refined by one
// third-order (Householder) step: with e = 1 - x y^2, 1 / sqrt(x) =
// y (1 - e)^(-1/2) = y (1 + e/2 + 3 e^2 / 8 + O(e^3)), and the dropped term is
// below 2^-64 (emulated worst case 0.9 ulp).  Outside [2^-100, 2^100), where
// the FP32 estimate could under- or overflow (including x = 0, coincident
// charges, and negative or NaN x), the FP64 division is used; the range test
// reads the exponent bits on the integer pipe.
template <> __device__ __forceinline__ double rsq<double>(double x) {
  const int bexp = __double2hiint(x) >> 20;   // sign and biased exponent
  if ((unsigned)(bexp - 923) >= 200u) return 1.0 / sqrt(x);
  const double y = (double)rsqrt_est((float)x);
  const double e = fma(-x * y, y, 1.0);
  return fma(y * e, fma(0.375, e, 0.5), y);
}
// the hardware estimate refined by one Newton step, y (3 - x y^2) / 2 (for x
// = 0 the estimate is +inf and the step gives NaN: coincident charges)
template <> __device__ __forceinline__ float rsq<float>(float x) {
  const float y = rsqrt_est(x);
  return y * fmaf(-0.5f * x, y * y, 1.5f);
}

// fused multiply-add in the working precision
__device__ __forceinline__ float fmaw(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaw(double a, double b, double c) { return fma(a, b, c); }

// compensated (Kahan) accumulator; FP64 uses plain sums
template <class T> struct Acc {
  T s = T(0), c = T(0);
  __device__ __forceinline__ void add(T v) {
    if (sizeof(T) == 4) {
      T y = v - c;
      T t = s + y;
      c = (t - s) - y;
      s = t;
    } else {
      s += v;
    }
  }
  __device__ __forceinline__ T get() const { return s - c; }
};

// ----------------------------------------------------------- brick kernels
// k_pair_screen: one CTA per brick of BX x BY x BZ target elements:
//  (1) the brick's "extended vertex field" R in shared memory (below);
//  (2) the screen field of all brick elements at their 64 nodes,
//      sum_o A(e, o) H(o, m): on the tensor cores (split bf16 MMAs) or as 512
//      rank-1 updates of a 64 x 64 tile on the CUDA cores (4 x 4 register
//      tile per thread, A and H staged in chunks of OCH offsets);
//  (3) the charges of the brick's short-range halo, staged in shared memory
//      in element order (when they fit) with each charge's halo x index;
//  (4) a few threads per target, each summing some of the 49 element rows of
//      the target's block (one contiguous run of staged charges per row).
// k_pair_eval: one CTA per brick after the solve: G = phi - screen field at
// the nodes, contracted with the shape functions at each target.
constexpr int BX = 4, BY = 4, BZ = 4, BE = BX * BY * BZ;   // 64 elements per brick
constexpr int OCH = 32;                                      // offsets per chunk
constexpr int MAXRUN = 2 * 81;                               // rows of the block (n_sr <= 4), 2 runs each

// source weights of the singular sum: the charge itself, or an adjoint weight array
template <class T> struct WeightQ {
  __device__ __forceinline__ T operator()(int, const typename vec4<T>::type& pj) const { return pj.w; }
};
template <class T> struct WeightArr {
  const double* w;
  __device__ __forceinline__ T operator()(int j, const typename vec4<T>::type&) const { return (T)w[j]; }
};

template <class T>
__device__ __forceinline__ void warp_sum(T& v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
}

// singular sum for one target over its block, lanes of one warp in parallel.
// W(j) = source weight (Q_j, or the adjoint weight); returns sum W/r and
// sum W (x_j - x_t)/r^3 in every lane.
template <class T, bool GRAD, class WeightF>
__device__ __forceinline__ void warp_singular(int n, int n_sr, T h, int ex, int ey, int ez, int slot,
                                              typename vec4<T>::type pt, const int* __restrict__ start,
                                              const typename vec4<T>::type* __restrict__ part,
                                              const int* __restrict__ ecoord, int* runs /* 2*MAXRUN */,
                                              int* pre /* MAXRUN+1 */, WeightF W, T out[4]) {
  const int lane = threadIdx.x & 31;
  const int nb = 2 * n_sr + 1, rows = nb * nb;
  // runs of consecutive element ids (split where the row wraps)
  for (int r = lane; r < rows; r += 32) {
    const int dy = r % nb - n_sr, dz = r / nb - n_sr;
    const int yy = wrapn(ey + dy, n), zz = wrapn(ez + dz, n);
    const int64_t rowbase = (int64_t)n * (yy + (int64_t)n * zz);
    int x0 = ex - n_sr, x1 = ex + n_sr;
    int a0, a1, b0 = 0, b1 = 0;
    if (x0 < 0) {
      a0 = start[rowbase + x0 + n]; a1 = start[rowbase + n];        // x0+n .. n-1
      b0 = start[rowbase];          b1 = start[rowbase + x1 + 1];   // 0 .. x1
    } else if (x1 >= n) {
      a0 = start[rowbase + x0];     a1 = start[rowbase + n];        // x0 .. n-1
      b0 = start[rowbase];          b1 = start[rowbase + x1 - n + 1];
    } else {
      a0 = start[rowbase + x0];     a1 = start[rowbase + x1 + 1];
    }
    runs[4 * r + 0] = a0; runs[4 * r + 1] = a1 - a0;
    runs[4 * r + 2] = b0; runs[4 * r + 3] = b1 - b0;
  }
  __syncwarp();
  if (lane == 0) {
    int acc = 0;
    for (int k = 0; k < 2 * rows; ++k) {
      pre[k] = acc;
      acc += runs[2 * k + 1];
    }
    pre[2 * rows] = acc;
  }
  __syncwarp();
  const int total = pre[2 * rows];
  Acc<T> ps, fx, fy, fz;
  int k = 0;
  for (int f = lane; f < total; f += 32) {
    while (pre[k + 1] <= f) ++k;
    const int j = runs[2 * k] + (f - pre[k]);
    if (j == slot) continue;
    const typename vec4<T>::type pj = part[j];
    const int ec = ecoord[j];
    int dx = (ec & 1023) - ex, dy = ((ec >> 10) & 1023) - ey, dz = (ec >> 20) - ez;
    dx = dx > n_sr ? dx - n : (dx < -n_sr ? dx + n : dx);
    dy = dy > n_sr ? dy - n : (dy < -n_sr ? dy + n : dy);
    dz = dz > n_sr ? dz - n : (dz < -n_sr ? dz + n : dz);
    const T rx = (T(dx) + (pj.x - pt.x)) * h, ry = (T(dy) + (pj.y - pt.y)) * h, rz = (T(dz) + (pj.z - pt.z)) * h;
    const T ir = rsq<T>(rx * rx + ry * ry + rz * rz);
    const T wj = W(j, pj);
    ps.add(wj * ir);
    if (GRAD) {
      const T f3 = wj * ir * ir * ir;
      fx.add(f3 * rx);
      fy.add(f3 * ry);
      fz.add(f3 * rz);
    }
  }
  out[0] = ps.get();
  out[1] = fx.get();
  out[2] = fy.get();
  out[3] = fz.get();
  for (int i = 0; i < 4; ++i) warp_sum(out[i]);
  __syncwarp();
}

// Extended vertex field: per axis SW = 3 BX + 2 n_sr - 1 slots, the first
// SF = BX + 2 n_sr - 1 the full vertex densities of the vertices interior
// offsets reach, then BX slots of corner-1-only sums (offset -(n_sr+1),
// vertex e + n_sr + 1) and BX of corner-0-only sums (offset n_sr, vertex
// e - n_sr).  A(e, o) is then the single value R[beta(o) + lambda(e)].
constexpr int STAGE_CAP = 1536;   // halo charges staged in shared memory (T = float)

// CUDA-core layout (TC = false): region 1 holds R first, then the staged
// charges; A and H chunks follow.  Tensor-core layout (TC = true): 48 KB of
// operand tiles (1 KB aligned; the staged charges reuse them after the
// contraction), then R.  Both end with the index tables.
template <class T, bool TC = false>
struct Pair3Smem {
  static constexpr int NT = TC ? PTC : PT;
  // bytes per R and chunk-operand entry: one float (tensor cores) or a hi + lo
  // float pair (the double-float CUDA-core contraction, both precisions)
  static constexpr int ES = TC ? 4 : 8;
  __host__ __device__ static int SW(int n_sr) { return 3 * BX + 2 * n_sr - 1; }
  __host__ __device__ static int HW(int n_sr) { return BX + 2 * n_sr; }
  // charges that can be staged: STAGE_CAP floats-worth of float4 (half as many double4)
  __host__ __device__ static int cap() { return STAGE_CAP * 4 / (int)sizeof(T); }
  __host__ __device__ static size_t rbytes(int n_sr) {
    const int sw = SW(n_sr);
    return (((size_t)sw * sw * sw * ES) + 31) / 32 * 32;
  }
  __host__ __device__ static size_t region1(int n_sr) {
    const size_t r = rbytes(n_sr);
    const size_t stg = (size_t)cap() * sizeof(typename vec4<T>::type);
    return r > stg ? r : stg;
  }
  __host__ __device__ static size_t ints(int n_sr) {
    const int hw = HW(n_sr);
    const int noff = 2 * n_sr + 2, nb = 2 * n_sr + 1, sw = SW(n_sr);
    return (size_t)hw * hw * hw + 1 + BE + 1 + 1 + NT / 32 + 1 + (size_t)noff * noff * noff + (size_t)nb * nb +
           3 * sw + 3 * hw + 32;
  }
  static constexpr size_t TILES = 6 * 8192;   // three bf16 pieces of A (64 x 64) and of B (64 x 64)
  // tensor cores: the staged charges in a region of their own (staged while the contraction runs)
  __host__ __device__ static size_t stgbytes() {
    return (size_t)cap() * sizeof(typename vec4<T>::type) + ((size_t)cap() + 15) / 16 * 16;
  }
  static size_t bytes(int n_sr) {
    if (TC) return 1024 + TILES + rbytes(n_sr) + stgbytes() + ints(n_sr) * sizeof(int) + 16;
    return region1(n_sr) + 2 * (size_t)OCH * 64 * ES + ints(n_sr) * sizeof(int) + (size_t)cap();
  }
};

// exclusive scan of one int per thread over the block (NT threads); returns the
// thread's prefix and writes the total to *total
template <int NT>
__device__ __forceinline__ int block_scan_excl(int v, int* wsum /* NT/32 + 1 */, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0;
    for (int w = 0; w < NT / 32; ++w) {
      const int t = wsum[w];
      wsum[w] = a;
      a += t;
    }
    wsum[NT / 32] = a;
  }
  __syncthreads();
  const int res = wsum[wid] + x - v;
  *total = wsum[NT / 32];
  __syncthreads();
  return res;
}

// Named CTA barriers (bar.sync id, n): groups of whole warps synchronise
// among themselves (id 0 with the CTA's thread count is __syncthreads).
__device__ __forceinline__ void group_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
// group_sync that also returns whether v was true in any thread of the group
__device__ __forceinline__ bool group_sync_or(int id, int n, bool v) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, %2, %3, p;\nselp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

// exclusive scan of one int per thread over a group of GN threads (gt its
// index in the group, whole warps; barrier id); returns the prefix, writes
// the total to *total
template <int GN>
__device__ __forceinline__ int group_scan_excl(int gt, int id, int v, int* wsum /* GN/32 + 1 */, int* total) {
  const int lane = gt & 31, wid = gt >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  group_sync(id, GN);
  if (gt == 0) {
    int a = 0;
    for (int w = 0; w < GN / 32; ++w) {
      const int t = wsum[w];
      wsum[w] = a;
      a += t;
    }
    wsum[GN / 32] = a;
  }
  group_sync(id, GN);
  const int res = wsum[wid] + x - v;
  *total = wsum[GN / 32];
  group_sync(id, GN);
  return res;
}

constexpr int SG = 256;   // threads of the short-range sums (the whole CTA on the CUDA cores, half of it
                          // beside the tensor-core contraction)

// How the halo's charges reach the singular sums: all staged in shared memory
// at once; staged tile by tile (consecutive runs of halo elements whose charges
// fit); or, when a single element holds more charges than fit, read from
// global memory.
enum HaloMode { HALO_STAGED = 0, HALO_TILED = 1, HALO_GLOBAL = 2 };

// the halo element id of halo index i (HW^3 elements, x fastest)
__device__ __forceinline__ int halo_gid(int i, int n, int HW, const int* __restrict__ we) {
  const int hx = i % HW, hy = (i / HW) % HW, hz = i / (HW * HW);
  return we[hx] + n * (we[HW + hy] + n * we[2 * HW + hz]);
}

// Prefix of the charges of the brick's short-range halo (HW^3 elements):
// hs[i] = the first slot of halo element i in halo order, hs[HW^3] = the total;
// the charges are staged in shared memory in that order (with each charge's
// halo x index) when they all fit (cap).  By SG threads (gt, barrier id).
// Returns the HaloMode.
template <class T>
__device__ int stage_halo(int gt, int id, int n, int HW, const int* __restrict__ we, const int* __restrict__ start,
                          const int* __restrict__ count, const typename vec4<T>::type* __restrict__ part, int cap,
                          typename vec4<T>::type* stg, unsigned char* sxb, int* hs, int* flag, int* wsum) {
  const int nh = HW * HW * HW;
  const int per = (nh + SG - 1) / SG, i0 = gt * per;
  int cnt[8], gid[8];   // per <= 7 for n_sr <= 4 (nh <= 1728)
  int sum = 0, big = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int i = i0 + k;
    cnt[k] = 0;
    gid[k] = 0;
    if (k < per && i < nh) {
      gid[k] = halo_gid(i, n, HW, we);
      cnt[k] = count[gid[k]];
    }
    sum += cnt[k];
    big |= cnt[k] > cap;
  }
  int total;
  int run = group_scan_excl<SG>(gt, id, sum, wsum, &total);
  const bool fits = total <= cap;
  const bool single = group_sync_or(id, SG, big != 0);   // an element over the cap: no tiling
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int i = i0 + k;
    if (k < per && i < nh) {
      hs[i] = run;
      if (fits) {
        const int j0 = start[gid[k]];
        const unsigned char hx = (unsigned char)(i % HW);
        for (int q = 0; q < cnt[k]; ++q) {
          stg[run + q] = part[j0 + q];
          sxb[run + q] = hx;
        }
      }
    }
    run += cnt[k];
  }
  if (gt == 0) {
    hs[nh] = total;
    flag[0] = fits ? HALO_STAGED : (single ? HALO_GLOBAL : HALO_TILED);
  }
  group_sync(id, SG);
  return flag[0];
}

// Singular sums of every target charge in the brick, by SG threads (gt), four
// per target: each walks the rows r = q, q + 4, ... of its target's block (a
// row (dy, dz) is 2 n_sr + 1 consecutive halo elements, so its staged charges
// are one run), two charges per step, each row's terms summed in order in
// FP32 and the row sums added with compensation; a shuffle tree combines the
// four.  Staged tile by tile (a dense halo): the tiles are consecutive runs of
// halo elements whose charges fit; each target takes the part of each row
// inside the tile, and its tile sums are added in FP64 in tile order (into
// phi_s / E_s, element units, scaled at the last tile).  Global (an element
// over the staging area): the same rows read from global memory, element by
// element.  Writes phi_s and E_s (and half of them to psi, gpsi).
template <class T, bool GRAD>
__device__ void singular_targets(int gt, int id, int mode, int n, int n_sr, T h, int E0x, int E0y, int E0z, int HW,
                                 int ntarget, const int* __restrict__ epre, const int* __restrict__ hs,
                                 const int* __restrict__ rtab, const int* __restrict__ we,
                                 typename vec4<T>::type* stg, unsigned char* sxb, int cap,
                                 const int* __restrict__ start, const int* __restrict__ count,
                                 const typename vec4<T>::type* __restrict__ part, double* __restrict__ phi_s,
                                 double* __restrict__ E_s, double* __restrict__ psi, double* __restrict__ gpsi) {
  typedef typename vec4<T>::type V4;
  constexpr int TPT = 4;
  const int nb = 2 * n_sr + 1, nrow = nb * nb, nh = HW * HW * HW;
  const int q = gt & (TPT - 1);
  const double ih = 1.0 / (double)h;   // the sums are in element units
  int ta = 0, tz = nh;                 // the tile: halo elements [ta, tz)
  for (int tile = 0;; ++tile) {
    int c0 = 0;                        // the tile's first charge slot
    if (mode == HALO_TILED) {
      // the longest run of elements from ta whose charges fit (every element does)
      int lo = ta + 1, hi = nh;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (hs[mid] - hs[ta] <= cap) lo = mid;
        else hi = mid - 1;
      }
      tz = lo;
      c0 = hs[ta];
      for (int i = ta + gt; i < tz; i += SG) {
        const int j0 = start[halo_gid(i, n, HW, we)], k0 = hs[i] - c0, cnt = hs[i + 1] - hs[i];
        const unsigned char hx = (unsigned char)(i % HW);
        for (int k = 0; k < cnt; ++k) {
          stg[k0 + k] = part[j0 + k];
          sxb[k0 + k] = hx;
        }
      }
      group_sync(id, SG);
    }
    const bool last = tz >= nh;
    for (int tb = 0; tb < ntarget; tb += SG / TPT) {
      const int k = tb + gt / TPT;
      const bool valid = k < ntarget;
      T v4[4] = {T(0), T(0), T(0), T(0)};
      int slot = 0;
      if (valid) {
        int lo = 0, hi2 = BE;                 // element of target k: epre[l] <= k < epre[l + 1]
        while (hi2 - lo > 1) {
          const int mid = (lo + hi2) >> 1;
          if (epre[mid] <= k) lo = mid;
          else hi2 = mid;
        }
        const int l = lo;
        const int lx = l % BX, ly = (l / BX) % BY, lz = l / (BX * BY);
        const int ex = E0x + lx, ey = E0y + ly, ez = E0z + lz;
        const int kk = k - epre[l];
        slot = start[ex + (int64_t)n * (ey + (int64_t)n * ez)] + kk;
        const int base = lx + HW * (ly + HW * lz);          // halo index of block offset (-n_sr, -n_sr, -n_sr)
        const int cx = lx + n_sr;                           // the target's halo x index
        Acc<T> ps, fx, fy, fz;
        if (mode != HALO_GLOBAL) {
          const int selfh = base + n_sr * (1 + HW + HW * HW);   // the target's own halo element
          const int self = hs[selfh] + kk - c0;
          const V4 pt = mode == HALO_STAGED ? stg[self] : part[slot];
          const T cxf = T(cx);
          T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0), ddy = T(0), ddz = T(0);
          int r = q, j = 0, je = 0;
          for (;;) {
            if (j >= je) {
              ps.add(s0);
              if (GRAD) {
                fx.add(s1);
                fy.add(s2);
                fz.add(s3);
              }
              s0 = s1 = s2 = s3 = T(0);
              if (r >= nrow) break;
              const int rt = rtab[r];
              const int h0 = base + (rt & 0xFFFF);
              const int ha = h0 > ta ? h0 : ta, hb = h0 + nb < tz ? h0 + nb : tz;   // the row's part in the tile
              j = ha < hb ? hs[ha] - c0 : 0;
              je = ha < hb ? hs[hb] - c0 : 0;
              ddy = T(((rt >> 16) & 0xFF) - n_sr);
              ddz = T((rt >> 24) - n_sr);
              r += TPT;
              continue;
            }
            const bool two = j + 1 < je;
            const int jb = two ? j + 1 : j;
            const V4 pa = stg[j], pb = stg[jb];
            // element units (1/h applied once per target, in FP64), fused r^2 and sums
            const T rxa = (T(sxb[j]) - cxf) + (pa.x - pt.x), rya = ddy + (pa.y - pt.y), rza = ddz + (pa.z - pt.z);
            const T rxb = (T(sxb[jb]) - cxf) + (pb.x - pt.x), ryb = ddy + (pb.y - pt.y), rzb = ddz + (pb.z - pt.z);
            const T ira = j == self ? T(0) : rsq<T>(fmaw(rxa, rxa, fmaw(rya, rya, rza * rza)));
            const T irb = (!two || jb == self) ? T(0) : rsq<T>(fmaw(rxb, rxb, fmaw(ryb, ryb, rzb * rzb)));
            const T qa = pa.w * ira, qb = pb.w * irb;
            s0 += qa;
            s0 += qb;
            if (GRAD) {
              const T f3a = qa * (ira * ira), f3b = qb * (irb * irb);
              s1 = fmaw(f3a, rxa, s1);
              s2 = fmaw(f3a, rya, s2);
              s3 = fmaw(f3a, rza, s3);
              s1 = fmaw(f3b, rxb, s1);
              s2 = fmaw(f3b, ryb, s2);
              s3 = fmaw(f3b, rzb, s3);
            }
            j += 2;
          }
        } else {
          // a row may wrap around the periodic box
          const V4 pt = part[slot];
          for (int r = q; r < nrow; r += TPT) {
            const int ay = r % nb, az = r / nb;
            const int64_t rowg = (int64_t)n * (we[HW + ly + ay] + (int64_t)n * we[2 * HW + lz + az]);
            const T ddy = T(ay - n_sr), ddz = T(az - n_sr);
            T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
            for (int ax = 0; ax < nb; ++ax) {
              const int64_t g = rowg + we[lx + ax];
              const T ddx = T(ax - n_sr);
              const int j0 = start[g], j1 = j0 + count[g];
              for (int j = j0; j < j1; ++j) {
                const V4 pj = part[j];
                const T rx = ddx + (pj.x - pt.x), ry = ddy + (pj.y - pt.y), rz = ddz + (pj.z - pt.z);
                const T ir = j == slot ? T(0) : rsq<T>(fmaw(rx, rx, fmaw(ry, ry, rz * rz)));
                const T qi = pj.w * ir;
                s0 += qi;
                if (GRAD) {
                  const T f3 = qi * (ir * ir);
                  s1 = fmaw(f3, rx, s1);
                  s2 = fmaw(f3, ry, s2);
                  s3 = fmaw(f3, rz, s3);
                }
              }
            }
            ps.add(s0);
            if (GRAD) {
              fx.add(s1);
              fy.add(s2);
              fz.add(s3);
            }
          }
        }
        v4[0] = ps.get();
        v4[1] = fx.get();
        v4[2] = fy.get();
        v4[3] = fz.get();
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int o = 1; o < TPT; o <<= 1) v4[i] += __shfl_xor_sync(0xffffffffu, v4[i], o);
      if (valid && q == 0) {
        // element units; tile sums added in FP64 in tile order, scaled at the last tile
        double sum[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) sum[a] = (double)v4[a];
        if (tile > 0) {
          sum[0] += phi_s[slot];
          if (GRAD)
#pragma unroll
            for (int a = 0; a < 3; ++a) sum[1 + a] += E_s[3 * slot + a];
        }
        if (last) {
          const double ps0 = sum[0] * ih;
          phi_s[slot] = ps0;
          if (psi) psi[slot] = 0.5 * ps0;
          if (GRAD) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              const double e = sum[1 + a] * (ih * ih);
              E_s[3 * slot + a] = e;
              if (gpsi) gpsi[3 * slot + a] = 0.5 * e;
            }
          }
        } else {
          phi_s[slot] = sum[0];
          if (GRAD)
#pragma unroll
            for (int a = 0; a < 3; ++a) E_s[3 * slot + a] = sum[1 + a];
        }
      }
    }
    if (last) break;
    group_sync(id, SG);   // the next tile overwrites the staging area
    ta = tz;
  }
}

// One CTA per brick of BX x BY x BZ elements: the screen field of every brick
// element at its 64 nodes (written to Gscr, brick-major) and the singular sums
// of every target charge in the brick (written to phi_s and E_s; with psi,
// half of them to psi and gpsi as well: the singular adjoint for the weights
// Q / 2 of the energy, whose kernel 1/r is symmetric).  TC: the
// contraction on the tensor cores (FP32 only; Hb holds the table's bf16
// pieces in the tiles' layout, err receives a bounded wait that gave up),
// 512 threads and eight per target; otherwise CUDA cores, 256 threads and
// four per target.
template <class T, bool GRAD, bool TC>
__global__ void __launch_bounds__(TC ? PTC : PT, 2) k_pair_screen(int n, int n_sr, T h, const int* __restrict__ start,
                                                             const int* __restrict__ count,
                                                             const typename vec4<T>::type* __restrict__ part,
                                                             const T* __restrict__ Cv, const T* __restrict__ rv,
                                                             const uint4* __restrict__ Hb, const float2* __restrict__ H0,
                                                             const float2* __restrict__ Hdf, T* __restrict__ Gscr, double* __restrict__ phi_s,
                                                             double* __restrict__ E_s, double* __restrict__ psi,
                                                             double* __restrict__ gpsi, int* __restrict__ err) {
  static_assert(!TC || sizeof(T) == 4, "the tensor-core contraction is the FP32 path's");
  static_assert(PT == SG && PTC == 2 * SG, "the short-range sums take the whole CUDA-core CTA, half the tensor-core one");
  constexpr int NT = TC ? PTC : PT;
  typedef typename vec4<T>::type V4;
  typedef Pair3Smem<T, TC> SM;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nbx = (n + BX - 1) / BX, nby = (n + BY - 1) / BY;
  const int E0x = (blockIdx.x % nbx) * BX, E0y = ((blockIdx.x / nbx) % nby) * BY, E0z = (blockIdx.x / (nbx * nby)) * BZ;
  const int keep = n_sr + 1, noff = 2 * n_sr + 2, no3 = noff * noff * noff;
  const int SW = 3 * BX + 2 * n_sr - 1, SF = BX + 2 * n_sr - 1, HW = BX + 2 * n_sr;
  const int nb = 2 * n_sr + 1, nrow = nb * nb;
  T *R, *A_c = nullptr, *H_c = nullptr;
  V4* stg;
  unsigned char* tiles = nullptr;
  int* hs;                                                // halo element prefix, HW^3 + 1
  unsigned char* sxb;                                     // cap(): halo x index of each staged charge
  if (TC) {
    tiles = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);   // swizzle atoms on 1 KB
    R = (T*)(tiles + SM::TILES);
    stg = (V4*)((unsigned char*)R + SM::rbytes(n_sr));
    sxb = (unsigned char*)(stg + SM::cap());
    hs = (int*)((unsigned char*)stg + SM::stgbytes());
  } else {
    const size_t r1 = SM::region1(n_sr);
    R = (T*)smem_raw;                                     // region 1: R, later the staged charges
    stg = (V4*)smem_raw;
    A_c = (T*)(smem_raw + r1);                            // [OCH][64] chunks of A and H (float pairs)
    H_c = (T*)((unsigned char*)A_c + OCH * 64 * SM::ES);
    hs = (int*)((unsigned char*)H_c + OCH * 64 * SM::ES);
  }
  int* epre = hs + HW * HW * HW + 1;                      // BE + 1
  int* flag = epre + BE + 1;
  int* wsum = flag + 1;                                   // NT/32 + 1 scan scratch
  int* otab = wsum + NT / 32 + 1;                         // no3: R base index of each offset
  int* rtab = otab + no3;                                 // nb^2 rows (dy, dz): halo offset | ay << 16 | az << 24
  int* wv = rtab + nrow;                                  // 3 x SW wrapped vertex coords times 1, n, n^2
  int* we = wv + 3 * SW;                                  // 3 x HW wrapped halo element coords
  if (!TC) sxb = (unsigned char*)(we + 3 * HW + 32);
  uint64_t* mbar = (uint64_t*)(((uintptr_t)(we + 3 * HW) + 7) & ~(uintptr_t)7);   // TC only
  uint32_t* tslot = (uint32_t*)(mbar + 1);
  const int tid = threadIdx.x;
  int ntarget;
  {
    int c0 = 0;
    if (tid < BE) {
      const int lx = E0x + (tid % BX), ly = E0y + (tid / BX) % BY, lz = E0z + tid / (BX * BY);
      if (lx < n && ly < n && lz < n) c0 = count[lx + (int64_t)n * (ly + (int64_t)n * lz)];
    }
    const int pre = block_scan_excl<NT>(c0, wsum, &ntarget);
    if (tid < BE) epre[tid] = pre;
    if (tid == 0) epre[BE] = ntarget;
  }
  if (ntarget == 0) return;
  // index tables (no divisions in the hot loops below)
  for (int o = tid; o < no3; o += NT) {
    const int ox = o % noff - keep, oy = (o / noff) % noff - keep, oz = o / (noff * noff) - keep;
    const int bx = ox == -keep ? SF : (ox == n_sr ? SF + BX : n_sr - 1 - ox);
    const int by = oy == -keep ? SF : (oy == n_sr ? SF + BX : n_sr - 1 - oy);
    const int bz = oz == -keep ? SF : (oz == n_sr ? SF + BX : n_sr - 1 - oz);
    otab[o] = bx + SW * (by + SW * bz);
  }
  for (int r = tid; r < nrow; r += NT) rtab[r] = HW * ((r % nb) + HW * (r / nb)) | (r % nb) << 16 | (r / nb) << 24;
  {
    const int E0[3] = {E0x, E0y, E0z};
    for (int i = tid; i < 3 * SW; i += NT) {
      const int a = i / SW, sa = i % SW;
      int v;
      if (sa < SF) v = E0[a] + sa - (n_sr - 1);
      else if (sa < SF + BX) v = E0[a] + (sa - SF) + keep;
      else v = E0[a] + (sa - SF - BX) - n_sr;
      wv[i] = wrapn(v, n) * (a == 0 ? 1 : (a == 1 ? n : n * n));   // the vertex id's term of axis a
    }
    for (int i = tid; i < 3 * HW; i += NT) {
      const int a = i / HW, ha = i % HW;
      we[i] = wrapn(E0[a] - n_sr + ha, n);
    }
  }
  __syncthreads();
  // (1) extended vertex field (unrolled: the gathers of several entries in flight); the
  // coordinates of entries i = tid + k NT advanced without divisions
  const int dsx = NT % SW, dsy = (NT / SW) % SW, dsz = NT / (SW * SW);
  int sx = tid % SW, sy = (tid / SW) % SW, sz = tid / (SW * SW);
#pragma unroll 4
  for (int i = tid; i < SW * SW * SW; i += NT) {
    // allowed corners k = kx + 2 ky + 4 kz as a bit mask: per axis both
    // corners, corner 1 only (k with kx = 1: 0xAA) or corner 0 only (0x55)
    const unsigned mx = sx < SF ? 0xFFu : (sx < SF + BX ? 0xAAu : 0x55u);
    const unsigned my = sy < SF ? 0xFFu : (sy < SF + BX ? 0xCCu : 0x33u);
    const unsigned mz = sz < SF ? 0xFFu : (sz < SF + BX ? 0xF0u : 0x0Fu);
    const unsigned mask = mx & my & mz;
    const int v = wv[sx] + wv[SW + sy] + wv[2 * SW + sz];   // < n^3 <= 2^30
    T val = T(0);
    if (mask == 0xFFu) {
      val = rv[v];
    } else {
      // the vertex's eight corner terms are contiguous: two vector loads
      const V4 c03 = reinterpret_cast<const V4*>(Cv + 8 * v)[0], c47 = reinterpret_cast<const V4*>(Cv + 8 * v)[1];
      const T c8[8] = {c03.x, c03.y, c03.z, c03.w, c47.x, c47.y, c47.z, c47.w};
#pragma unroll
      for (int k = 0; k < 8; ++k) val += ((mask >> k) & 1u) ? c8[k] : T(0);
    }
    if constexpr (!TC) {
      // split once here into the hi + lo floats of the double-float
      // contraction (each R value is read by several offsets; an FP32 value
      // has lo = 0)
      const float vh = (float)val;
      reinterpret_cast<float2*>(R)[i] = make_float2(vh, (float)((double)val - (double)vh));
    } else {
      R[i] = val;
    }
    sx += dsx;
    sy += dsy;
    sz += dsz;
    if (sx >= SW) {
      sx -= SW;
      ++sy;
    }
    if (sy >= SW) {
      sy -= SW;
      ++sz;
    }
  }
  // (2) screen field and (3) singular sums
  if constexpr (TC) {
    // Tensor cores: two groups of eight warps run side by side.  Group A
    // (warps 0 .. 7: two of each TMEM lane quarter) computes the screen field:
    // for each chunk of 64 offsets, the three bf16 pieces of A (64 brick
    // elements x 64 offsets, built from R) and of H (64 nodes x 64 offsets,
    // precomputed) in shared memory; one thread issues the six piece products
    // per K step of 16 (M = 64, N = 64) into two TMEM accumulators (hi: the
    // product of the leading pieces, lo: the other five).  The hi accumulator
    // holds one chunk at a time and is added into registers after each chunk,
    // so that no accumulation inside the tensor core spans more than 64 terms
    // of the leading product; the chunk sums are added with compensation.  In
    // the FP32 path the table is relative to each element's corners (see
    // pair_relative_table), so these sums carry no large smooth part.  Group
    // B (warps 8 .. 15) stages the halo charges in a region of their own and
    // computes the singular sums meanwhile.
    const uint32_t tl = smem_u32(tiles);
    if (tid < 32) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(tslot)));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) mbar_init(smem_u32(mbar));
    tc_fence_before();
    __syncthreads();   // R complete; TMEM address and barrier visible
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const int warp = tid >> 5;
    bool failed = false;
    if (tid < SG) {
      const int gt = tid;
      // The field at node 0 (the one absolute column of the relative table,
      // the element's potential level) is summed on the CUDA cores from the A
      // values each thread splits anyway, with the table's hi + lo floats (H0)
      // in two FP32 sums rounded to nearest (the tensor cores' accumulation
      // would round it alike in every element, and U adds that up); four
      // partial sums per element, combined in the epilogue.
      __shared__ float2 s0p[(SG / 64) * BE];
      float s0h = 0.f, s0l = 0.f;
      const int l = gt & 63, g = gt >> 6;   // this thread's A units: row l, chunk offsets 8 g .. and 8 (g + 4) ..
      const int lam = (l % BX) + SW * (((l / BX) % BY) + SW * (l / (BX * BY)));
      const uint32_t aoff[2] = {sw128_off(l, 8 * g), sw128_off(l, 8 * (g + 4))};
      const int nch = (no3 + 63) / 64;
      // this thread's accumulator entries (tmem_ld16x64b): register jj holds element row
      // 16 qq + (lane / 4) + 8 (lane mod 2), node column 32 hh + 2 jj + (lane / 2) mod 2
      const int qq = warp & 3, hh = warp >> 2, lane = tid & 31;
      const int arow = 16 * qq + (lane >> 2) + 8 * (lane & 1), acol = 32 * hh + ((lane >> 1) & 1);
      const uint32_t ta = tmem + ((uint32_t)(32 * qq) << 16) + 32 * hh;
      float hsum[16], hcmp[16];   // compensated chunk sums of the hi accumulator
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) hsum[jj] = hcmp[jj] = 0.f;
      for (int c = 0; c < nch; ++c) {
        for (int i = gt; i < 1536; i += SG) cp_async16(tl + 24576 + 16 * i, Hb + (size_t)c * 1536 + i);
        asm volatile("cp.async.commit_group;" ::: "memory");
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          uint32_t p0[4], p1[4], p2[4];
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int o = 64 * c + 8 * (g + 4 * hf) + 2 * jj;
            const float xa = o < no3 ? (float)R[otab[o] + lam] : 0.f;
            const float xb = o + 1 < no3 ? (float)R[otab[o + 1] + lam] : 0.f;
            bf16_split2(xa, xb, p0[jj], p1[jj], p2[jj]);
            if (o + 1 < no3) {
              const float4 h2 = *reinterpret_cast<const float4*>(H0 + o);   // H0[o], H0[o + 1]
              s0h = fmaf(xa, h2.x, fmaf(xb, h2.z, s0h));
              s0l = fmaf(xa, h2.y, fmaf(xb, h2.w, s0l));
            }
          }
          sts128(tl + aoff[hf], p0);
          sts128(tl + 8192 + aoff[hf], p1);
          sts128(tl + 16384 + aoff[hf], p2);
        }
        cp_async_wait_all();
        fence_async_smem();
        group_sync(1, SG);
        if (gt == 0) {
          tc_fence_after();
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t a = tl + 32 * kk, b = tl + 24576 + 32 * kk;
            const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
            umma_bf16(tmem, umma_desc(a), umma_desc(b), UMMA_IDESC, kk > 0 ? 1u : 0u);         // a0 b0
            umma_bf16(tmem + 64, umma_desc(a), umma_desc(b + 8192), UMMA_IDESC, acc);          // a0 b1
            umma_bf16(tmem + 64, umma_desc(a + 8192), umma_desc(b), UMMA_IDESC, 1u);           // a1 b0
            umma_bf16(tmem + 64, umma_desc(a), umma_desc(b + 16384), UMMA_IDESC, 1u);          // a0 b2
            umma_bf16(tmem + 64, umma_desc(a + 8192), umma_desc(b + 8192), UMMA_IDESC, 1u);   // a1 b1
            umma_bf16(tmem + 64, umma_desc(a + 16384), umma_desc(b), UMMA_IDESC, 1u);          // a2 b0
          }
          umma_commit(smem_u32(mbar));
        }
        // one warp polls the barrier; the group waits at its named barrier
        const bool done = warp == 0 ? mbar_wait(smem_u32(mbar), (uint32_t)(c & 1)) : true;
        if (group_sync_or(1, SG, !done)) {
          failed = true;
          break;
        }
        tc_fence_after();
        uint32_t vh[16];
        tmem_ld16x64b(ta, vh);
        tmem_wait_ld();
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const float y = __uint_as_float(vh[jj]) - hcmp[jj], t = hsum[jj] + y;
          hcmp[jj] = (t - hsum[jj]) - y;
          hsum[jj] = t;
        }
        tc_fence_before();   // the next chunk's MMAs overwrite hi after the next barrier
      }
      if (failed) {
        if (gt == 0) atomicExch(err, 1);
        // a last bounded wait on both phases for MMAs still in flight, and for the table copy
        (void)mbar_wait(smem_u32(mbar), 0u);
        (void)mbar_wait(smem_u32(mbar), 1u);
        cp_async_wait_all();
      }
      s0p[g * BE + l] = make_float2(s0h, s0l);
      group_sync(1, SG);
      tc_fence_after();
      if (!failed) {
        uint32_t vl[16];
        tmem_ld16x64b(ta + 64, vl);
        tmem_wait_ld();
        float* drow = (float*)Gscr + (int64_t)blockIdx.x * (BE * 64) + arow * 64 + acol;
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) drow[2 * jj] = (hsum[jj] - hcmp[jj]) + __uint_as_float(vl[jj]);
        if (acol == 0) {   // column 0 from the CUDA-core sums
          double sum = 0.0;
#pragma unroll
          for (int q = 0; q < SG / 64; ++q) {
            const float2 v = s0p[q * BE + arow];
            sum += (double)v.x + (double)v.y;
          }
          drow[0] = (float)sum;
        }
      }
      tc_fence_before();
    } else {
      const int gt = tid - SG;
      const int mode = stage_halo<T>(gt, 2, n, HW, we, start, count, part, SM::cap(), stg, sxb, hs, flag, wsum);
      singular_targets<T, GRAD>(gt, 2, mode, n, n_sr, h, E0x, E0y, E0z, HW, ntarget, epre, hs, rtab, we, stg, sxb,
                                SM::cap(), start, count, part, phi_s, E_s, psi, gpsi);
    }
    __syncthreads();   // every TMEM read done
    if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
  } else {
    // CUDA cores: 4 x 4 register tile, per-chunk partial sums added into a
    // total, in double-float arithmetic on the FP32 pipes in both precisions
    // (FP64 issues at a small fraction of the FP32 rate here): A and H are
    // staged as hi + lo float pairs (the table's from FP64; an FP32 A has lo =
    // 0), each product keeps its exact leading part (fused two-product) and the
    // two cross terms, and the products are summed by two-sum into a hi + lo
    // accumulator; each chunk's sum goes into an FP64 total, which keeps the
    // relative error near 2^-48 of the chunk's sum of |A H| instead of growing
    // over all offsets.  The FP32 path's result is then rounded to FP32.
    const int eb = tid >> 4, mb = tid & 15;
    // this thread stages entries i = tid + k PT: element l = i & 63 is fixed per thread
    const int lst = tid & 63;
    const int lam = (lst % BX) + SW * (((lst / BX) % BY) + SW * (lst / (BX * BY)));
    constexpr int SPT = OCH * 64 / PT;   // staged entries per thread per chunk
    T* gb = Gscr + (int64_t)blockIdx.x * (BE * 64);
    {
      // the table's hi + lo floats come precomputed (Hdf); R was split in (1)
      float2 hpf[SPT];                   // next chunk's table values, fetched during this chunk
#pragma unroll
      for (int k = 0; k < SPT; ++k) {
        const int i = tid + k * PT, o = i >> 6;
        hpf[k] = o < no3 ? Hdf[(int64_t)o * 64 + (i & 63)] : make_float2(0.f, 0.f);
      }
      const float2* R2 = reinterpret_cast<const float2*>(R);
      float sh[4][4], sl[4][4];
      double tot[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) tot[i][j] = 0.0;
      float2* A2 = reinterpret_cast<float2*>(A_c);
      float2* H2 = reinterpret_cast<float2*>(H_c);
      for (int o0 = 0; o0 < no3; o0 += OCH) {
        __syncthreads();
#pragma unroll
        for (int k = 0; k < SPT; ++k) {
          const int i = tid + k * PT;
          const int o = o0 + (i >> 6);
          H2[i] = hpf[k];
          A2[i] = o < no3 ? R2[otab[o] + lam] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (o0 + OCH < no3) {
#pragma unroll
          for (int k = 0; k < SPT; ++k) {
            const int i = tid + k * PT, o = o0 + OCH + (i >> 6);
            hpf[k] = o < no3 ? Hdf[(int64_t)o * 64 + (i & 63)] : make_float2(0.f, 0.f);
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) sh[i][j] = sl[i][j] = 0.f;
#pragma unroll 2
        for (int oi = 0; oi < OCH; ++oi) {
          const float4* ap = reinterpret_cast<const float4*>(A2 + oi * 64 + 4 * eb);
          const float4* hp = reinterpret_cast<const float4*>(H2 + oi * 64 + 4 * mb);
          const float4 a01 = ap[0], a23 = ap[1], h01 = hp[0], h23 = hp[1];
          const float ah[4] = {a01.x, a01.z, a23.x, a23.z}, al[4] = {a01.y, a01.w, a23.y, a23.w};
          const float hh[4] = {h01.x, h01.z, h23.x, h23.z}, hl[4] = {h01.y, h01.w, h23.y, h23.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const float p = ah[i] * hh[j];
              float e = fmaf(ah[i], hh[j], -p);
              e = fmaf(ah[i], hl[j], e);
              e = fmaf(al[i], hh[j], e);
              const float t = sh[i][j] + p, z = t - sh[i][j];
              sl[i][j] += ((sh[i][j] - (t - z)) + (p - z)) + e;
              sh[i][j] = t;
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) tot[i][j] += (double)sh[i][j] + (double)sl[i][j];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        V4 v;
        v.x = (T)tot[i][0];
        v.y = (T)tot[i][1];
        v.z = (T)tot[i][2];
        v.w = (T)tot[i][3];
        *reinterpret_cast<V4*>(gb + (4 * eb + i) * 64 + 4 * mb) = v;
      }
    }
    // Region 1 (R) was last read before the chunk loop's final barrier, so the
    // staging may overwrite it without another one.
    const int mode = stage_halo<T>(tid, 0, n, HW, we, start, count, part, SM::cap(), stg, sxb, hs, flag, wsum);
    singular_targets<T, GRAD>(tid, 0, mode, n, n_sr, h, E0x, E0y, E0z, HW, ntarget, epre, hs, rtab, we, stg, sxb,
                              SM::cap(), start, count, part, phi_s, E_s, psi, gpsi);
  }
}

// One CTA per brick, after the mesh solve: G = mesh potential - screen field
// at the 64 nodes of each non-empty brick element, then four threads per
// target charge each contract 16 of the nodes with the order-3 shape
// functions (and their derivatives) at the charge; the mesh part is added to
// the singular part the screen kernel left in phi_s / E_s.
//
// FP64 path: G is held in shared memory relative to its value G0 at the
// element's first node (kept in FP64): the shape functions sum to one and
// their gradients to zero, so G0 enters the potential alone and the rounding
// acts on the variation of G only.
//
// FP32 path: the screen field arrives relative to the element's corners (the
// field at node 0, corner fields relative to it, elsewhere the field less its
// trilinear interpolant; pair_relative_table), and G is split the same way:
// G0 and the corner values of G - G0 in FP64 (the mesh potential's hi + lo
// float pair added in FP64), and the remainder G - G0 - trilinear(corners) in
// FP32 (from the same pairs).  The trilinear part and its gradient at the
// charge are evaluated in FP64; only the small remainder goes through the FP32
// contraction.
template <class T, bool GRAD>
__global__ void __launch_bounds__(PT) k_pair_eval(int n, int Nm, T inv_h, const int* __restrict__ start,
                                                  const int* __restrict__ count,
                                                  const typename vec4<T>::type* __restrict__ part,
                                                  const double* __restrict__ phi64, const float2* __restrict__ phi_hl,
                                                  const T* __restrict__ Gscr,
                                                  const int* __restrict__ perm, double* __restrict__ phi_s,
                                                  double* __restrict__ E_s, double* __restrict__ phi_out) {
  typedef typename vec4<T>::type V4;
  constexpr bool F32 = sizeof(T) == 4;
  __shared__ __align__(32) T G[BE * 64];
  __shared__ double G0[BE];
  __shared__ double Gc[F32 ? BE * 8 : 1];   // FP32 path: corner values of G - G0
  __shared__ int epre[BE + 1];
  __shared__ int wsum[PT / 32 + 1];
  const int nbx = (n + BX - 1) / BX, nby = (n + BY - 1) / BY;
  const int E0x = (blockIdx.x % nbx) * BX, E0y = ((blockIdx.x / nbx) % nby) * BY, E0z = (blockIdx.x / (nbx * nby)) * BZ;
  const int tid = threadIdx.x;
  int ntarget;
  {
    int c0 = 0;
    if (tid < BE) {
      const int lx = E0x + (tid % BX), ly = E0y + (tid / BX) % BY, lz = E0z + tid / (BX * BY);
      if (lx < n && ly < n && lz < n) c0 = count[lx + (int64_t)n * (ly + (int64_t)n * lz)];
    }
    const int pre = block_scan_excl<PT>(c0, wsum, &ntarget);
    if (tid < BE) epre[tid] = pre;
    if (tid == 0) epre[BE] = ntarget;
  }
  if (ntarget == 0) return;
  __syncthreads();
  const T* gb = Gscr + (int64_t)blockIdx.x * (BE * 64);
  const int N = Nm;
  // mesh node of node m of brick element l: on the periodic mesh (Nm = 3n
  // nodes per axis) wrapped, on a box's (Nm = 3 nb + 1, targets in the first
  // nb elements) never past the last node
  auto node = [&](int l, int m) -> int64_t {
    const int ex = E0x + l % BX, ey = E0y + (l / BX) % BY, ez = E0z + l / (BX * BY);
    const int gx = 3 * ex + (m & 3), gy = 3 * ey + ((m >> 2) & 3), gz = 3 * ez + (m >> 4);   // < 3n + 3
    return (gx >= N ? gx - N : gx) + (int64_t)N * ((gy >= N ? gy - N : gy) + (int64_t)N * (gz >= N ? gz - N : gz));
  };
  if constexpr (F32) {
    auto phd = [&](int64_t k) -> double {
      const float2 p = phi_hl[k];
      return (double)p.x + (double)p.y;
    };
    if (tid < BE && epre[tid + 1] != epre[tid]) {
      const double p00 = phd(node(tid, 0));
      G0[tid] = p00 - (double)gb[tid * 64];
      Gc[tid * 8] = 0.0;
#pragma unroll
      for (int c = 1; c < 8; ++c) {
        const int mc = 3 * (c & 1) + 12 * ((c >> 1) & 1) + 48 * (c >> 2);
        Gc[tid * 8 + c] = (phd(node(tid, mc)) - p00) - (double)gb[tid * 64 + mc];
      }
    }
    // node differences of the mesh potential from its hi + lo floats
    for (int i = tid; i < BE * 64; i += PT) {
      const int l = i >> 6, m = i & 63;
      if (epre[l + 1] == epre[l]) continue;   // empty (or outside the mesh): never read
      const float2 p = phi_hl[node(l, m)], p0 = phi_hl[node(l, 0)];
      G[i] = (p.x - p0.x) + (p.y - p0.y);
    }
    __syncthreads();
    // remainder: the difference less its trilinear interpolant, less the screen
    // remainder; zero at the corners
    constexpr int PER = BE * 64 / PT;
    float rem[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = tid + k * PT, l = i >> 6, m = i & 63;
      const int mx = m & 3, my = (m >> 2) & 3, mz = m >> 4;
      rem[k] = 0.f;
      if (epre[l + 1] == epre[l]) continue;
      if ((mx == 0 || mx == 3) && (my == 0 || my == 3) && (mz == 0 || mz == 3)) continue;
      const float* g = G + l * 64;
      const float tx = mx * (1.f / 3.f), ty = my * (1.f / 3.f), tz = mz * (1.f / 3.f);
      // corners (0,0,0) 0, (3,0,0) 3, (0,3,0) 12, (3,3,0) 15, z + 48
      const float x00 = fmaf(tx, g[3] - g[0], g[0]), x10 = fmaf(tx, g[15] - g[12], g[12]);
      const float x01 = fmaf(tx, g[51] - g[48], g[48]), x11 = fmaf(tx, g[63] - g[60], g[60]);
      const float y0 = fmaf(ty, x10 - x00, x00), y1 = fmaf(ty, x11 - x01, x01);
      rem[k] = (g[m] - fmaf(tz, y1 - y0, y0)) - gb[i];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) G[tid + k * PT] = rem[k];
  } else {
    if (tid < BE && epre[tid + 1] != epre[tid]) G0[tid] = phi64[node(tid, 0)] - gb[tid * 64];
    __syncthreads();
    for (int i = tid; i < BE * 64; i += PT) {
      const int l = i >> 6, m = i & 63;
      if (epre[l + 1] == epre[l]) continue;   // empty (or outside the mesh): never read
      G[i] = (phi64[node(l, m)] - gb[i]) - G0[l];
    }
  }
  __syncthreads();
  const int q = tid & 3;   // nodes 16 q .. 16 q + 15: mz = q, (mx, my) over 4 x 4
  for (int tb = 0; tb < ntarget; tb += PT / 4) {
    const int k = tb + (tid >> 2);
    const bool valid = k < ntarget;
    T v4[4] = {T(0), T(0), T(0), T(0)};
    int slot = 0, l = 0;
    V4 pt;
    pt.x = pt.y = pt.z = pt.w = T(0);
    if (valid) {
      int lo = 0, hi2 = BE;
      while (hi2 - lo > 1) {
        const int mid = (lo + hi2) >> 1;
        if (epre[mid] <= k) lo = mid;
        else hi2 = mid;
      }
      l = lo;
      const int ex = E0x + l % BX, ey = E0y + (l / BX) % BY, ez = E0z + l / (BX * BY);
      slot = start[ex + (int64_t)n * (ey + (int64_t)n * ez)] + (k - epre[l]);
      pt = part[slot];
      T ux[4], uy[4], uz[4], dx4[4], dy4[4], dz4[4];
      q3_values<T>(pt.x, ux);
      q3_values<T>(pt.y, uy);
      q3_values<T>(pt.z, uz);
      if (GRAD) {
        q3_derivs<T>(pt.x, dx4);
        q3_derivs<T>(pt.y, dy4);
        q3_derivs<T>(pt.z, dz4);
      }
#pragma unroll
      for (int my = 0; my < 4; ++my) {
        const V4 gv = *reinterpret_cast<const V4*>(G + l * 64 + 16 * q + 4 * my);
        const T g4[4] = {gv.x, gv.y, gv.z, gv.w};
#pragma unroll
        for (int mx = 0; mx < 4; ++mx) {
          const T g = g4[mx];
          const T wyz = uy[my] * uz[q];
          v4[0] += g * ux[mx] * wyz;
          if (GRAD) {
            v4[1] += g * dx4[mx] * wyz;
            v4[2] += g * ux[mx] * dy4[my] * uz[q];
            v4[3] += g * ux[mx] * uy[my] * dz4[q];
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      v4[i] += __shfl_xor_sync(0xffffffffu, v4[i], 1);
      v4[i] += __shfl_xor_sync(0xffffffffu, v4[i], 2);
    }
    if (valid && q == 0) {
      // FP32 path: the trilinear part of G - G0 and its gradient at the charge, in FP64
      double tv = 0.0, tg[3] = {0.0, 0.0, 0.0};
      if constexpr (F32) {
        const double* g = Gc + l * 8;
        const double x = pt.x, y = pt.y, z = pt.z;
        double a[4], b[4];   // x-lerps and x-differences of the corner pairs j = cy + 2 cz
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          b[j] = g[2 * j + 1] - g[2 * j];
          a[j] = fma(x, b[j], g[2 * j]);
        }
        const double ay0 = a[1] - a[0], ay1 = a[3] - a[2];
        const double a0 = fma(y, ay0, a[0]), a1 = fma(y, ay1, a[2]);
        const double bx0 = fma(y, b[1] - b[0], b[0]), bx1 = fma(y, b[3] - b[2], b[2]);
        tv = fma(z, a1 - a0, a0);
        tg[0] = fma(z, bx1 - bx0, bx0);
        tg[1] = fma(z, ay1 - ay0, ay0);
        tg[2] = a1 - a0;
      }
      const double phi = (((double)v4[0] + tv) + G0[l]) * (double)inv_h + phi_s[slot];
      phi_s[slot] = phi;
      if (phi_out) phi_out[perm[slot]] = phi;
      if (GRAD) {
        const double ih2 = (double)inv_h * (double)inv_h;
        E_s[3 * slot + 0] = ((double)v4[1] + tg[0]) * ih2 + E_s[3 * slot + 0];
        E_s[3 * slot + 1] = ((double)v4[2] + tg[1]) * ih2 + E_s[3 * slot + 1];
        E_s[3 * slot + 2] = ((double)v4[3] + tg[2]) * ih2 + E_s[3 * slot + 2];
      }
    }
  }
}

// ----------------------------------------------------------------- adjoint
__global__ void k_weights(int64_t N, double gU, const double* __restrict__ gphi, const int* __restrict__ perm,
                          const double* __restrict__ Qs, double* __restrict__ w, float* __restrict__ w32) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= N) return;
  const double v = 0.5 * gU * Qs[k] + (gphi ? gphi[perm[k]] : 0.0);
  w[k] = v;
  if (w32) w32[k] = (float)v;
}


// W[e][m] = sum_{t in e} w_t u_m(tau_t): the adjoint's point deposit, per
// element.  wsum (FP32 path): sum_{t in e} w_t in FP64 as hi + lo floats, the
// exact sum over m of W[e][m] (the shape functions sum to one).  wT: the
// weights in the working precision (FP32: a copy, so that the 64 threads of
// an element do not each convert them).
template <class T>
__global__ void k_elem_deposit(int64_t ne, const int* __restrict__ start, const int* __restrict__ count,
                               const typename vec4<T>::type* __restrict__ part, const double* __restrict__ w,
                               const T* __restrict__ wT, T* __restrict__ W, float2* __restrict__ wsum) {
  // wsum: the block's elements by the lanes of its first warp (an FP64
  // instruction takes the FP64 pipe for a whole warp, however few lanes are on)
  const int per = blockDim.x / 64;
  if (wsum && threadIdx.x < per) {
    const int64_t e = blockIdx.x * (int64_t)per + threadIdx.x;
    if (e < ne) {
      double ws = 0.0;
      for (int j = start[e], j1 = start[e] + count[e]; j < j1; ++j) ws += w[j];
      const float hi = (float)ws;
      wsum[e] = make_float2(hi, (float)(ws - (double)hi));
    }
  }
  const int64_t e = blockIdx.x * (int64_t)per + threadIdx.x / 64;
  if (e >= ne) return;
  const int m = threadIdx.x & 63, mx = m & 3, my = (m >> 2) & 3, mz = m >> 4;
  const int s = start[e], cnt = count[e];
  T acc = T(0);
  for (int j = s; j < s + cnt; ++j) {
    const typename vec4<T>::type p = part[j];
    T ux[4], uy[4], uz[4];
    q3_values<T>(p.x, ux);
    q3_values<T>(p.y, uy);
    q3_values<T>(p.z, uz);
    acc += wT[j] * ux[mx] * uy[my] * uz[mz];
  }
  W[e * 64 + m] = acc;
}

// g[node] = sum over (element, local node) pairs at the node of W: in FP64,
// or (T = float, the mixed solver's right-hand side) as a float pair h + l
// summed by two-sums; (3n)^3 < 2^32
template <class T>
__global__ void k_node_assemble(int n, const T* __restrict__ W, double* __restrict__ g) {
  const int N = 3 * n;
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (unsigned)N * (unsigned)N * (unsigned)N) return;
  const unsigned q = i / (unsigned)N;
  const int ix = (int)(i - q * (unsigned)N), iy = (int)(q % (unsigned)N), iz = (int)(q / (unsigned)N);
  int el[3][2], lo[3][2], cnt[3];
  const int id[3] = {ix, iy, iz};
  for (int a = 0; a < 3; ++a) {
    const int e = id[a] / 3, t = id[a] - 3 * e;
    el[a][0] = e;
    lo[a][0] = t;
    cnt[a] = 1;
    if (t == 0) {
      el[a][1] = wrapn(e - 1, n);
      lo[a][1] = 3;
      cnt[a] = 2;
    }
  }
  if constexpr (sizeof(T) == 4) {
    float sh = 0.f, sl = 0.f;
    for (int c = 0; c < cnt[2]; ++c)
      for (int b = 0; b < cnt[1]; ++b)
        for (int a = 0; a < cnt[0]; ++a) {
          const int64_t e = el[0][a] + (int64_t)n * (el[1][b] + (int64_t)n * el[2][c]);
          const float v = W[e * 64 + lo[0][a] + 4 * lo[1][b] + 16 * lo[2][c]];
          const float t = sh + v, bv = t - sh;
          sl += (sh - (t - bv)) + (v - bv);
          sh = t;
        }
    const float h = sh + sl;
    reinterpret_cast<float2*>(g)[i] = make_float2(h, sl - (h - sh));
  } else {
    double acc = 0.0;
    for (int c = 0; c < cnt[2]; ++c)
      for (int b = 0; b < cnt[1]; ++b)
        for (int a = 0; a < cnt[0]; ++a) {
          const int64_t e = el[0][a] + (int64_t)n * (el[1][b] + (int64_t)n * el[2][c]);
          acc += (double)W[e * 64 + lo[0][a] + 4 * lo[1][b] + 16 * lo[2][c]];
        }
    g[i] = acc;
  }
}

// Screen part of the adjoint, as a GEMM and a gather (deterministic, no atomics):
//   D[o][e] = sum_m W[e][m] H(o, m)               (every element e, every vertex offset o)
//   A[s][k] = sum_{o : o + k in block} D[o][s + k + o]
// D[o][e] is the table field of element e's deposit seen from the vertex e - o
// (k_adj_gemm on the CUDA cores, the tensor-core row GEMM in the FP32 path;
// the gather is k_adj_vertex).
constexpr int GT = 64;   // GEMM tile: 64 elements x 64 offsets, K = 64 nodes
constexpr int ADJ_NT = 128;   // tensor-core column tile: offsets per tile

// The products are summed in double-float arithmetic on the FP32 pipes in both
// precisions, as in the screen contraction (hi + lo float pairs in shared
// memory: the table's from FP64, an FP32 deposit has lo = 0; fused two-product
// with the cross terms, two-sum accumulation), in two halves of 32 nodes whose
// sums are added in FP64; D is stored in T.
template <class T>
__global__ void __launch_bounds__(PT) k_adj_gemm(int64_t ne, int o0, int no, const T* __restrict__ W,
                                                 const double* __restrict__ Hw, T* __restrict__ D) {
  __shared__ float2 Ws2[64][GT + 1];   // [m][element]
  __shared__ float2 Hs2[64][GT + 1];   // [m][offset]
  const int64_t e0 = (int64_t)blockIdx.x * GT;
  const int oo0 = o0 + blockIdx.y * GT;
  for (int i = threadIdx.x; i < GT * 64; i += PT) {
    const int r = i >> 6, m = i & 63;
    const int64_t e = e0 + r;
    const int o = oo0 + r;
    const double w = e < ne ? (double)W[e * 64 + m] : 0.0;
    const double hv = (o < o0 + no) ? Hw[(int64_t)o * 64 + m] : 0.0;
    const float wh = (float)w, hh = (float)hv;
    Ws2[m][r] = make_float2(wh, (float)(w - (double)wh));
    Hs2[m][r] = make_float2(hh, (float)(hv - (double)hh));
  }
  __syncthreads();
  const int te = threadIdx.x & 15, to = threadIdx.x >> 4;   // 4 elements x 4 offsets per thread
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
#pragma unroll 1
  for (int half = 0; half < 2; ++half) {
    float sh[4][4], sl[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) sh[i][j] = sl[i][j] = 0.f;
#pragma unroll 4
    for (int m = 32 * half; m < 32 * half + 32; ++m) {
      float2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = Ws2[m][te + 16 * i];
        b[i] = Hs2[m][to + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float p = a[i].x * b[j].x;
          float e = fmaf(a[i].x, b[j].x, -p);
          e = fmaf(a[i].x, b[j].y, e);
          e = fmaf(a[i].y, b[j].x, e);
          const float t = sh[i][j] + p, z = t - sh[i][j];
          sl[i][j] += ((sh[i][j] - (t - z)) + (p - z)) + e;
          sh[i][j] = t;
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += (double)sh[i][j] + (double)sl[i][j];
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int o = oo0 + to + 16 * j;
    if (o >= o0 + no) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t e = e0 + te + 16 * i;
      if (e < ne) D[(int64_t)(o - o0) * ne + e] = (T)acc[i][j];
    }
  }
}

// Double-float accumulator (hi + lo floats, summed by two-sum): the FP32
// path's screen adjoint sums, whose terms cancel to a small remainder.
struct dfacc {
  float h = 0.f, l = 0.f;
};
__device__ __forceinline__ void acc_add(dfacc& a, float b) {
  const float s = a.h + b, bb = s - a.h;
  a.l += (a.h - (s - bb)) + (b - bb);
  a.h = s;
}
__device__ __forceinline__ void acc_merge(dfacc& a, const dfacc& b) {
  const float s = a.h + b.h, bb = s - a.h;
  a.l += ((a.h - (s - bb)) + (b.h - bb)) + b.l;
  a.h = s;
}
__device__ __forceinline__ void acc_merge(double& a, double b) { a += b; }
__device__ __forceinline__ double acc_value(const dfacc& a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ double acc_value(double a) { return a; }

// Screen adjoint, gathered by vertex:
//   A[s][k] = sum over the offsets o with o + k inside the block of D(o, s + k + o).
// For the vertex v = s + k the terms are D(o, v + o) over the offsets that
// corner k's block holds: along each axis, o_a = -(n_sr + 1) only for k_a = 1,
// o_a = n_sr only for k_a = 0, the others for both.  The terms of a vertex are
// summed into 27 classes (the three cases per axis); A(v - k, k) is the sum of
// the eight classes that corner k admits.  A CTA of eight warps takes 32
// consecutive vertices (one per lane: consecutive lanes read consecutive
// elements of D) and a chunk of whole offset planes (oz in [z0, z1)); the
// chunk's rows of offsets (oz, oy) are dealt to the warps in turn, each warp
// sums its rows' terms into its own 27 classes, and the warps' classes are
// combined in shared memory in warp order, one thread per (vertex, corner):
// deterministic.  FP32 path (H0 set): D holds the contraction with the
// node-0-relative table, and each term gains H(o, 0) Wsum(v + o)
// (pair_adjoint_table); terms and sums in double-float arithmetic.  FP64
// path: D is the whole contraction, summed in FP64.
constexpr int AV_WARPS = 8;
template <class T, int NSR>
__global__ void __launch_bounds__(32 * AV_WARPS) k_adj_vertex(int n, int z0, int z1, int first,
                                                              const int* __restrict__ count, const T* __restrict__ D,
                                                              const float2* __restrict__ H0,
                                                              const float2* __restrict__ wsum, double* __restrict__ A) {
  constexpr int KEEP = NSR + 1, NOFF = 2 * NSR + 2, PLANE = NOFF * NOFF;
  constexpr bool DF = sizeof(T) == 4;
  typedef typename std::conditional<DF, dfacc, double>::type Acc;
  extern __shared__ __align__(16) unsigned char av_smem[];
  Acc(*part)[27][32] = reinterpret_cast<Acc(*)[27][32]>(av_smem);   // [AV_WARPS][27][32]: each warp's classes
  __shared__ int live[32];
  const int64_t ne = (int64_t)n * n * n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t v = blockIdx.x * (int64_t)32 + lane;
  const bool in = v < ne;
  const int vx = in ? (int)(v % n) : 0, vy = in ? (int)((v / n) % n) : 0, vz = in ? (int)(v / ((int64_t)n * n)) : 0;
  if (warp == 0) {
    bool any = false;   // the eight elements v - k; A is read only for non-empty ones
    if (in)
#pragma unroll
      for (int k = 0; k < 8; ++k)
        any |= count[wrapn(vx - (k & 1), n) + (int64_t)n * (wrapn(vy - ((k >> 1) & 1), n) +
                                                            (int64_t)n * wrapn(vz - (k >> 2), n))] != 0;
    live[lane] = any;
  }
  __syncthreads();
  const bool act = live[lane] != 0;
#pragma unroll
  for (int c = 0; c < 27; ++c) part[warp][c][lane] = Acc{};
  if (__any_sync(0xffffffffu, act)) {
    int wx[NOFF];
#pragma unroll
    for (int i = 0; i < NOFF; ++i) wx[i] = wrapn(vx + i - KEEP, n);
    const int rows = (z1 - z0) * NOFF;
    for (int rho = warp; rho < rows; rho += AV_WARPS) {
      const int oz = z0 + rho / NOFF, oy = rho % NOFF;
      const int cz = oz == 0 ? 0 : (oz == NOFF - 1 ? 2 : 1), cy = oy == 0 ? 0 : (oy == NOFF - 1 ? 2 : 1);
      const int64_t erow = (int64_t)n * (wrapn(vy + oy - KEEP, n) + (int64_t)n * wrapn(vz + oz - KEEP, n));
      const T* Dp = D + ((int64_t)(oz - z0) * PLANE + oy * NOFF) * ne;
      Acc P[3] = {};
#pragma unroll
      for (int ox = 0; ox < NOFF; ++ox) {
        const int cx = ox == 0 ? 0 : (ox == NOFF - 1 ? 2 : 1);
        if (!act) continue;
        const int64_t e = erow + wx[ox];
        const T d = Dp[(int64_t)ox * ne + e];
        if constexpr (DF) {
          const float2 h = H0[oz * PLANE + oy * NOFF + ox], w = wsum[e];
          const float p = h.x * w.x;
          float r = fmaf(h.x, w.x, -p);
          r = fmaf(h.x, w.y, r);
          r = fmaf(h.y, w.x, r);
          acc_add(P[cx], p);
          acc_add(P[cx], d + r);
        } else {
          P[cx] += d;
        }
      }
      Acc* row = &part[warp][cz * 9 + cy * 3][lane];
#pragma unroll
      for (int c = 0; c < 3; ++c) acc_merge(row[32 * c], P[c]);
    }
  }
  __syncthreads();
  // one thread per (vertex, corner): the admitted classes, warps in order
  const int vl = threadIdx.x & 31, k = threadIdx.x >> 5;   // 256 threads = 32 vertices x 8 corners
  const int64_t vv = blockIdx.x * (int64_t)32 + vl;
  if (vv >= ne || !live[vl]) return;
  const int kx = k & 1, ky = (k >> 1) & 1, kz = k >> 2;
  Acc s = {};
#pragma unroll
  for (int cz = kz ? 0 : 1; cz <= (kz ? 1 : 2); ++cz)
#pragma unroll
    for (int cy = ky ? 0 : 1; cy <= (ky ? 1 : 2); ++cy)
#pragma unroll
      for (int cx = kx ? 0 : 1; cx <= (kx ? 1 : 2); ++cx)
#pragma unroll
        for (int w = 0; w < AV_WARPS; ++w) acc_merge(s, part[w][cz * 9 + cy * 3 + cx][vl]);
  const int ux = (int)(vv % n), uy = (int)((vv / n) % n), uz = (int)(vv / ((int64_t)n * n));
  const int64_t se = wrapn(ux - kx, n) + (int64_t)n * (wrapn(uy - ky, n) + (int64_t)n * wrapn(uz - kz, n));
  double* dst = A + se * 8 + k;
  *dst = first ? acc_value(s) : *dst + acc_value(s);
}

template <class T>
__global__ void __launch_bounds__(PT) k_pair_adj_warp(int64_t N, int n, int n_sr, T h, const int* __restrict__ start,
                                                      const typename vec4<T>::type* __restrict__ part,
                                                      const int* __restrict__ ecoord, const double* __restrict__ w,
                                                      double* __restrict__ psi, double* __restrict__ gpsi) {
  __shared__ int runs_all[8 * 2 * MAXRUN];
  __shared__ int pre_all[8 * (MAXRUN + 1)];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t = blockIdx.x * (int64_t)(PT / 32) + warp;
  if (t >= N) return;
  const typename vec4<T>::type pt = part[t];
  const int ec = ecoord[t];
  T sg[4];
  WeightArr<T> wf{w};
  warp_singular<T, true>(n, n_sr, h, ec & 1023, (ec >> 10) & 1023, ec >> 20, (int)t, pt, start, part, ecoord,
                         runs_all + warp * 2 * MAXRUN, pre_all + warp * (MAXRUN + 1), wf, sg);
  if (lane == 0) {
    psi[t] = (double)sg[0];
    gpsi[3 * t + 0] = (double)sg[1];
    gpsi[3 * t + 1] = (double)sg[2];
    gpsi[3 * t + 2] = (double)sg[3];
  }
}

// per charge: dLf/dQ and dLf/dx from the pieces (see fep3m_vjp)
template <class T>
__global__ void k_final(int64_t N, int n, double inv_h, double gU, double sign,
                        const typename vec4<T>::type* __restrict__ part,
                        const int* __restrict__ perm, const int* __restrict__ cell, const double* __restrict__ w,
                        const double* __restrict__ phi_s, const double* __restrict__ E_s,
                        const double* __restrict__ psi, const double* __restrict__ gpsi, const double* __restrict__ mu,
                        const double* __restrict__ A, double* __restrict__ dpos, double* __restrict__ dQ) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= N) return;
  const int i = perm[t];
  const int e = cell[i];
  const int ex = e % n, ey = (e / n) % n, ez = e / (n * n);
  const typename vec4<T>::type p = part[t];
  const double tx = p.x, ty = p.y, tz = p.z, Q = p.w;
  const double wx[2] = {1.0 - tx, tx}, wy[2] = {1.0 - ty, ty}, wz[2] = {1.0 - tz, tz};
  const double sg[2] = {-1.0, 1.0};
  double sQ = 0, gx = 0, gy = 0, gz = 0;
  for (int k = 0; k < 8; ++k) {
    const int kx = k & 1, ky = (k >> 1) & 1, kz = k >> 2;
    const int64_t v = wrapn(ex + kx, n) + (int64_t)n * (wrapn(ey + ky, n) + (int64_t)n * wrapn(ez + kz, n));
    const double coef = (mu[v] - A[(int64_t)e * 8 + k]) * inv_h;
    sQ += wx[kx] * wy[ky] * wz[kz] * coef;
    gx += sg[kx] * wy[ky] * wz[kz] * coef;
    gy += wx[kx] * sg[ky] * wz[kz] * coef;
    gz += wx[kx] * wy[ky] * sg[kz] * coef;
  }
  const double wt = w[t];
  if (dQ) dQ[i] = 0.5 * gU * phi_s[t] + psi[t] + sQ;
  if (dpos) {
    dpos[3 * i + 0] = sign * (wt * E_s[3 * t + 0] + Q * (gpsi[3 * t + 0] + gx * inv_h));
    dpos[3 * i + 1] = sign * (wt * E_s[3 * t + 1] + Q * (gpsi[3 * t + 1] + gy * inv_h));
    dpos[3 * i + 2] = sign * (wt * E_s[3 * t + 2] + Q * (gpsi[3 * t + 2] + gz * inv_h));
  }
}

// deterministic sum of a per-charge product (FP64): out = 1/2 sum Q phi
__global__ void k_energy(int64_t N, const double* __restrict__ Qs, const double* __restrict__ phi,
                         double* __restrict__ partials, unsigned int* __restrict__ counter, double* __restrict__ out) {
  __shared__ double sh[PT / 32];
  __shared__ bool last;
  double acc = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x)
    acc += Qs[k] * phi[k];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int k = 0; k < PT / 32; ++k) s += sh[k];
    partials[blockIdx.x] = s;
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double s = 0;
    for (unsigned int k = 0; k < gridDim.x; ++k) s += ((volatile double*)partials)[k];
    *out = 0.5 * s;
    *counter = 0u;
  }
}

template <class A, class B>
__global__ void k_cast(int64_t n, const A* __restrict__ in, B* __restrict__ out, double scale) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n) return;
  out[g] = (B)((double)in[g] * scale);
}

inline int gsz(int64_t n, int t = PT) { return (int)((n + t - 1) / t); }

}  // namespace

// ordered singular pairs, non-empty elements and the largest element population
// per non-empty element e with c0 charges and s charges in its block (nb
// non-empty block elements): singular pairs c0 s - c0, one non-empty element,
// the largest c0, nb (element pairs of the screen contraction) and c0 nb
// (charge-element pairs)
__device__ __forceinline__ void pair_count_one(int n, int n_sr, const int* __restrict__ count, int64_t e,
                                               unsigned long long v[5]) {
  const int c0 = count[e];
  if (c0 == 0) return;
  const int ex = (int)(e % n), ey = (int)((e / n) % n), ez = (int)(e / ((int64_t)n * n));
  long long s = 0, nb = 0;
  for (int dz = -n_sr; dz <= n_sr; ++dz)
    for (int dy = -n_sr; dy <= n_sr; ++dy)
      for (int dx = -n_sr; dx <= n_sr; ++dx) {
        const int cj = count[wrapn(ex + dx, n) + (int64_t)n * (wrapn(ey + dy, n) + (int64_t)n * wrapn(ez + dz, n))];
        s += cj;
        nb += cj > 0;
      }
  v[0] = (unsigned long long)((long long)c0 * s - c0);
  v[1] = 1ull;
  v[2] = (unsigned long long)c0;
  v[3] = (unsigned long long)nb;
  v[4] = (unsigned long long)((long long)c0 * nb);
}

// warp sums (and max) first: one atomic per warp and counter
__global__ void k_pair_count(int n, int n_sr, const int* __restrict__ count, unsigned long long* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  unsigned long long v[5] = {0ull, 0ull, 0ull, 0ull, 0ull};
  if (e < (int64_t)n * n * n) pair_count_one(n, n_sr, count, e, v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v[0] += __shfl_down_sync(0xffffffffu, v[0], o);
    v[1] += __shfl_down_sync(0xffffffffu, v[1], o);
    const unsigned long long m = __shfl_down_sync(0xffffffffu, v[2], o);
    v[2] = m > v[2] ? m : v[2];
    v[3] += __shfl_down_sync(0xffffffffu, v[3], o);
    v[4] += __shfl_down_sync(0xffffffffu, v[4], o);
  }
  if ((threadIdx.x & 31) == 0 && v[1] != 0ull) {
    atomicAdd(&out[0], v[0]);
    atomicAdd(&out[1], v[1]);
    atomicMax(&out[2], v[2]);
    atomicAdd(&out[3], v[3]);
    atomicAdd(&out[4], v[4]);
  }
}

cudaError_t pair_counts(fep3m_ctx* c, unsigned long long* dev5, cudaStream_t s) {
  const int64_t ne = (int64_t)c->n * c->n * c->n;
  cudaMemsetAsync(dev5, 0, 5 * sizeof(unsigned long long), s);
  FEP3M_CL k_pair_count<<<gsz(ne), PT, 0, s>>>(c->n, c->n_sr, c->count, dev5);
  return cudaGetLastError();
}

static int pair_bricks(const fep3m_ctx* c) {
  const int n = c->n;
  return ((n + BX - 1) / BX) * ((n + BY - 1) / BY) * ((n + BZ - 1) / BZ);
}

size_t pair_screen_bytes(const fep3m_ctx* c) {
  return (size_t)pair_bricks(c) * BE * 64 * (c->precision == FEP3M_MIXED ? sizeof(float) : sizeof(double));
}

template <class T, bool GRAD, bool TC>
static cudaError_t launch_pair_screen(fep3m_ctx* c, cudaStream_t s, bool half) {
  const size_t smem = Pair3Smem<T, TC>::bytes(c->n_sr);
  auto kern = k_pair_screen<T, GRAD, TC>;
  cudaError_t e = smem_limit((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  FEP3M_CL kern<<<(unsigned)pair_bricks(c), TC ? PTC : PT, smem, s>>>(
      c->n, c->n_sr, (T)c->h, c->start, c->count, (const typename vec4<T>::type*)c->part, (const T*)c->Cv,
      (const T*)c->rv, (const uint4*)c->Hb, (const float2*)c->H0df, (const float2*)c->Hdf, (T*)c->Gscr, c->phi_s, c->E_s,
      half ? c->psi_s : nullptr,
      half ? c->gpsi_s : nullptr, c->iflags + 2);
  return cudaGetLastError();
}

// nodes per axis of the mesh the evaluation reads: the periodic order-3 mesh,
// or a box's
static int mesh_nodes_per_axis(const fep3m_ctx* c) { return c->box ? c->box->Nn : 3 * c->n; }

// MIXED: the mesh potential as hi + lo floats: the periodic solver's output
// itself, a box's split by pair_prepare
static const float2* mesh_potential_pairs(const fep3m_ctx* c) {
  if (c->precision != FEP3M_MIXED) return nullptr;
  return c->box ? (const float2*)c->phi_hl : (const float2*)c->phi64;
}

template <class T, bool GRAD>
static cudaError_t launch_pair_eval(fep3m_ctx* c, double* phi_out) {
  FEP3M_CL k_pair_eval<T, GRAD><<<(unsigned)pair_bricks(c), PT, 0, c->stream>>>(
      c->n, mesh_nodes_per_axis(c), (T)c->inv_h, c->start, c->count, (const typename vec4<T>::type*)c->part, c->phi64,
      mesh_potential_pairs(c), (const T*)c->Gscr, c->perm, c->phi_s, c->E_s, phi_out);
  return cudaGetLastError();
}

cudaError_t pair_screen(fep3m_ctx* c, int want_grad, cudaStream_t s, bool energy_adjoint) {
  const bool half = energy_adjoint && want_grad;
  if (c->precision == FEP3M_MIXED) {
    if (c->Hb)
      return want_grad ? launch_pair_screen<float, true, true>(c, s, half)
                       : launch_pair_screen<float, false, true>(c, s, half);
    return want_grad ? launch_pair_screen<float, true, false>(c, s, half)
                     : launch_pair_screen<float, false, false>(c, s, half);
  }
  return want_grad ? launch_pair_screen<double, true, false>(c, s, half)
                   : launch_pair_screen<double, false, false>(c, s, half);
}

// Corner structure of an element's 64 order-3 nodes (m = mx + 4 my + 16 mz):
// corner c = cx + 2 cy + 4 cz sits at node 3 cx + 12 cy + 48 cz, and the
// trilinear interpolant of the eight corner values has weight
// prod_a (c_a ? m_a / 3 : 1 - m_a / 3) at node m.
static int corner_node(int c) { return 3 * (c & 1) + 12 * ((c >> 1) & 1) + 48 * (c >> 2); }
static bool is_corner_node(int m) {
  const int mx = m & 3, my = (m >> 2) & 3, mz = m >> 4;
  return (mx == 0 || mx == 3) && (my == 0 || my == 3) && (mz == 0 || mz == 3);
}
static double corner_weight(int c, int m) {
  const int mm[3] = {m & 3, (m >> 2) & 3, m >> 4};
  double w = 1.0;
  for (int a = 0; a < 3; ++a) w *= ((c >> a) & 1) ? mm[a] / 3.0 : 1.0 - mm[a] / 3.0;
  return w;
}

// The FP32 path's screen-field table, relative to each element's corners:
// column 0 is H(o, 0); the other corner columns H(o, c) - H(o, 0); every
// other column H(o, m) minus the trilinear interpolant of H(o, corners) at m.
// The contraction sum_o A(o) Hrel(o, m) then returns the field at node 0, the
// corner fields relative to it and, elsewhere, the field less its trilinear
// interpolant: the same field with its large smooth part taken out of the
// FP32 sums (its corner values enter the evaluation in FP64).
void pair_relative_table(int n_sr, const double* Hw, double* Hrel) {
  const int noff = 2 * n_sr + 2, no3 = noff * noff * noff;
  for (int o = 0; o < no3; ++o) {
    const double* h = Hw + (size_t)o * 64;
    double* r = Hrel + (size_t)o * 64;
    for (int m = 0; m < 64; ++m) {
      if (m == 0) {
        r[m] = h[0];
      } else if (is_corner_node(m)) {
        r[m] = h[m] - h[0];
      } else {
        double t = 0.0;
        for (int c = 0; c < 8; ++c) t += corner_weight(c, m) * h[corner_node(c)];
        r[m] = h[m] - t;
      }
    }
  }
}

// The FP32 path's screen-adjoint table: Hd(o, m) = H(o, m) - H(o, 0), column 0
// zero.  With Wsum(e) = sum_m W[e][m] the contraction splits as
//   D(o, e) = H(o, 0) Wsum(e) + sum_m W[e][m] Hd(o, m):
// the tensor cores form the second part (small terms), the gather adds the
// first in double-float arithmetic (H0: hi + lo floats of H(o, 0)).
void pair_adjoint_table(int n_sr, const double* Hw, double* Hd, float* H0) {
  const int noff = 2 * n_sr + 2, no3 = noff * noff * noff;
  for (int o = 0; o < no3; ++o) {
    const double h0 = Hw[(size_t)o * 64];
    for (int m = 0; m < 64; ++m) Hd[(size_t)o * 64 + m] = m == 0 ? 0.0 : Hw[(size_t)o * 64 + m] - h0;
    const float hi = (float)h0;
    H0[2 * o] = hi;
    H0[2 * o + 1] = (float)(h0 - (double)hi);
  }
}

// the table's three bf16 pieces for the screen adjoint's contraction
// D[o][e] = sum_m W[e][m] H(o, m) on the tensor cores: B[o][m] = H(o, m) in
// column tiles of ADJ_NT offsets, one chunk of the 64 nodes
size_t pair_adj_table_bytes(int n_sr) {
  const int noff = 2 * n_sr + 2, no3 = noff * noff * noff;
  return (size_t)((no3 + ADJ_NT - 1) / ADJ_NT) * 3 * ADJ_NT * 64 * 2;
}
void pair_adj_table(int n_sr, const double* Hw, uint16_t* out) {
  const int noff = 2 * n_sr + 2, no3 = noff * noff * noff, ntile = (no3 + ADJ_NT - 1) / ADJ_NT;
  std::memset(out, 0, pair_adj_table_bytes(n_sr));
  for (int t = 0; t < ntile; ++t)
    for (int ii = 0; ii < ADJ_NT; ++ii) {
      const int o = t * ADJ_NT + ii;
      if (o >= no3) continue;
      for (int m = 0; m < 64; ++m) {
        uint16_t pc[3];
        bf16_pieces(Hw[(size_t)o * 64 + m], pc);
        for (int p = 0; p < 3; ++p) out[((size_t)t * 3 + p) * ADJ_NT * 64 + sw128_off(ii, m) / 2] = pc[p];
      }
    }
}

// the table's three bf16 pieces per chunk of 64 offsets, in the swizzled
// K-major layout of the tensor-core tiles: [chunk][piece][node row][offset]
size_t pair_tc_table_bytes(int n_sr) {
  const int noff = 2 * n_sr + 2, no3 = noff * noff * noff;
  return (size_t)((no3 + 63) / 64) * 3 * 8192;
}
void pair_tc_table(int n_sr, const double* Hw, uint16_t* out) {
  const int noff = 2 * n_sr + 2, no3 = noff * noff * noff, nch = (no3 + 63) / 64;
  auto bits = [](double v) -> uint16_t {   // round to nearest even bf16 (finite v)
    const float f = (float)v;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
  };
  auto val = [](uint16_t b) -> double {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return (double)f;
  };
  std::memset(out, 0, pair_tc_table_bytes(n_sr));
  for (int ch = 0; ch < nch; ++ch)
    for (int m = 0; m < 64; ++m)
      for (int k = 0; k < 64; ++k) {
        const int o = 64 * ch + k;
        double r = o < no3 ? Hw[(size_t)o * 64 + m] : 0.0;
        for (int p = 0; p < 3; ++p) {
          const uint16_t b = bits(r);
          r -= val(b);
          out[((size_t)(ch * 3 + p) * 8192 + sw128_off(m, k)) / 2] = b;
        }
      }
}

// a box's FP64 mesh potential as hi + lo floats for the FP32 pair kernels
__global__ void k_phi_hilo(int64_t n, const double* __restrict__ phi, float2* __restrict__ out) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n) return;
  const double v = phi[g];
  const float hi = (float)v;
  out[g] = make_float2(hi, (float)(v - (double)hi));
}

cudaError_t pair_prepare(fep3m_ctx* c) {
  if (c->precision == FEP3M_MIXED && c->box) {   // the periodic solver writes float pairs itself
    const int64_t na = mesh_nodes_per_axis(c), nodes = na * na * na;
    FEP3M_CL k_phi_hilo<<<gsz(nodes), PT, 0, c->stream>>>(nodes, c->phi64, (float2*)c->phi_hl);
  }
  return cudaGetLastError();
}

cudaError_t pair_eval(fep3m_ctx* c, double* phi_out, int want_grad) {
  if (c->precision == FEP3M_MIXED)
    return want_grad ? launch_pair_eval<float, true>(c, phi_out) : launch_pair_eval<float, false>(c, phi_out);
  return want_grad ? launch_pair_eval<double, true>(c, phi_out) : launch_pair_eval<double, false>(c, phi_out);
}

cudaError_t energy(fep3m_ctx* c, double* U_dev, cudaStream_t s) {
  const int64_t N = c->N;
  const int nb = (int)std::min<int64_t>(std::max<int64_t>(gsz(N), 1), 1024);
  FEP3M_CL k_energy<<<nb, PT, 0, s ? s : c->stream>>>(N, c->Q_s, c->phi_s, (double*)c->red_tmp, c->red_counter, U_dev);
  return cudaGetLastError();
}

template <class T, int NSR>
static void launch_adj_vertex(fep3m_ctx* c, int z0, int z1, const T* D, double* A, cudaStream_t s) {
  const int64_t ne = (int64_t)c->n * c->n * c->n;
  const bool df = sizeof(T) == 4;
  const size_t smem = (size_t)AV_WARPS * 27 * 32 * 8;   // dfacc and double: 8 bytes
  (void)smem_limit((const void*)k_adj_vertex<T, NSR>, smem);   // a failure shows as the launch's error
  FEP3M_CL k_adj_vertex<T, NSR><<<(unsigned)((ne + 31) / 32), 32 * AV_WARPS, smem, s>>>(
      c->n, z0, z1, z0 == 0, c->count, D, df ? (const float2*)c->H0df : nullptr, df ? (const float2*)c->Wsum : nullptr,
      A);
}

// D-GEMM + gather over chunks of whole offset planes (all offsets with one
// oz), sized so D stays within a memory budget
template <class T>
static cudaError_t screen_adjoint(fep3m_ctx* c, const T* W, const double* Hw, double* A) {
  const int n = c->n;
  const int64_t ne = (int64_t)n * n * n;
  const int noff = c->noff, plane = noff * noff;
  // bytes of D held at once: a quarter of the device's memory (at least 2 GiB), so that on a
  // large GPU even the 256^3 mesh takes D in one piece (each further piece re-reads and
  // re-writes A and launches the gather again); sized at the context's first sweep
  if (c->adj_planes == 0) {
    size_t budget = (size_t)1 << 31;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) budget = std::max(budget, std::min(total_b / 4, free_b / 2));
    else (void)cudaGetLastError();
    c->adj_planes = (int)std::min<int64_t>(noff, std::max<int64_t>(1, (int64_t)(budget / ((size_t)ne * sizeof(T) * plane))));
  }
  // tensor cores (FP32 path, table pieces prepared): column tiles of ADJ_NT offsets
  const bool tcore = sizeof(T) == 4 && c->HbA != nullptr;
  const int planes = c->adj_planes;
  const size_t need = (size_t)planes * plane * ne * sizeof(T);
  if (c->D_bytes < need) {
    if (c->D_adj) cudaFree(c->D_adj);
    c->D_adj = nullptr;
    c->D_bytes = 0;
    cudaError_t e = cudaMalloc(&c->D_adj, need);
    if (e != cudaSuccess) return e;
    c->D_bytes = need;
  }
  cudaStream_t s = c->stream;
  for (int z0 = 0; z0 < noff; z0 += planes) {
    const int z1 = std::min(noff, z0 + planes), o0 = z0 * plane, no = (z1 - z0) * plane;
    if (tcore) {
      cudaError_t e = tc_rows_gemm(ne, 64, o0, o0 + no, ADJ_NT, (const float*)W, c->HbA, (float*)c->D_adj,
                                   c->iflags + 2, s);
      if (e != cudaSuccess) return e;
    } else {
      dim3 grid((unsigned)((ne + GT - 1) / GT), (unsigned)((no + GT - 1) / GT));
      FEP3M_CL k_adj_gemm<T><<<grid, PT, 0, s>>>(ne, o0, no, W, Hw, (T*)c->D_adj);
    }
    const T* D = (const T*)c->D_adj;
    switch (c->n_sr) {
      case 1: launch_adj_vertex<T, 1>(c, z0, z1, D, A, s); break;
      case 2: launch_adj_vertex<T, 2>(c, z0, z1, D, A, s); break;
      case 3: launch_adj_vertex<T, 3>(c, z0, z1, D, A, s); break;
      default: launch_adj_vertex<T, 4>(c, z0, z1, D, A, s); break;
    }
  }
  return cudaGetLastError();
}

// weights w = gU Q / 2 + gphi (sorted order), element deposits, adjoint right-hand side g64
cudaError_t adjoint_pre(fep3m_ctx* c, double gU, const double* gphi, cudaStream_t s) {
  const int n = c->n;
  const int64_t ne = (int64_t)n * n * n, nodes = 27 * ne, N = c->N;
  FEP3M_CL k_weights<<<gsz(N), PT, 0, s>>>(N, gU, gphi, c->perm, c->Q_s, c->w_s, c->w_s32);
  const int per = PT / 64;
  if (c->precision == FEP3M_MIXED) {
    FEP3M_CL k_elem_deposit<float><<<gsz(ne, per), PT, 0, s>>>(ne, c->start, c->count, (const float4*)c->part, c->w_s,
                                                               c->w_s32, (float*)c->W_el, (float2*)c->Wsum);
    FEP3M_CL k_node_assemble<float><<<gsz(nodes), PT, 0, s>>>(n, (const float*)c->W_el, c->g64);
  } else {
    FEP3M_CL k_elem_deposit<double><<<gsz(ne, per), PT, 0, s>>>(ne, c->start, c->count, (const vec4<double>::type*)c->part,
                                                                c->w_s, c->w_s, (double*)c->W_el, nullptr);
    FEP3M_CL k_node_assemble<double><<<gsz(nodes), PT, 0, s>>>(n, (const double*)c->W_el, c->g64);
  }
  return cudaGetLastError();
}

// the screen sweep A and (with singular) the singular adjoint potential: they
// need the deposit of the weights (adjoint_pre) but not the adjoint mesh
// solution, so they run concurrently with the mesh solves
cudaError_t adjoint_sweeps(fep3m_ctx* c, cudaStream_t s, bool singular) {
  const int n = c->n;
  const int64_t N = c->N;
  cudaStream_t keep = c->stream;
  c->stream = s;   // screen_adjoint issues on c->stream
  cudaError_t e;
  if (c->precision == FEP3M_MIXED) {
    e = screen_adjoint<float>(c, (const float*)c->W_el, c->Ha64, (double*)c->A_el);
    if (e == cudaSuccess && singular)
      FEP3M_CL k_pair_adj_warp<float><<<(unsigned)((N + 7) / 8), PT, 0, s>>>(N, n, c->n_sr, (float)c->h, c->start,
                                                         (const float4*)c->part, c->ecoord, c->w_s, c->psi_s, c->gpsi_s);
  } else {
    e = screen_adjoint<double>(c, (const double*)c->W_el, c->Hw64, (double*)c->A_el);
    if (e == cudaSuccess && singular)
      FEP3M_CL k_pair_adj_warp<double><<<(unsigned)((N + 7) / 8), PT, 0, s>>>(N, n, c->n_sr, c->h, c->start,
                                                          (const vec4<double>::type*)c->part, c->ecoord, c->w_s,
                                                          c->psi_s, c->gpsi_s);
  }
  c->stream = keep;
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// the part that needs lam: the vertex adjoint mu = 4 pi (Mpq^T)^3 lam
cudaError_t adjoint_vertex(fep3m_ctx* c, cudaStream_t s) {
  const fep3m::Level& L0 = c->solv[1].mg.lv[0];
  return vertex_adjoint(c, c->lam64, c->mu_v, L0.t1, L0.t2, s);
}

cudaError_t singular_sums(fep3m_ctx* c, const double* w, double* psi, double* gpsi, cudaStream_t s) {
  const int64_t N = c->N;
  if (c->precision == FEP3M_MIXED)
    FEP3M_CL k_pair_adj_warp<float><<<(unsigned)((N + 7) / 8), PT, 0, s>>>(N, c->n, c->n_sr, (float)c->h, c->start,
                                                                           (const float4*)c->part, c->ecoord, w, psi,
                                                                           gpsi);
  else
    FEP3M_CL k_pair_adj_warp<double><<<(unsigned)((N + 7) / 8), PT, 0, s>>>(N, c->n, c->n_sr, c->h, c->start,
                                                                            (const vec4<double>::type*)c->part,
                                                                            c->ecoord, w, psi, gpsi);
  return cudaGetLastError();
}

// per-charge dLf/dx (times sign) and dLf/dQ
cudaError_t adjoint_final(fep3m_ctx* c, double gU, double* dpos, double* dQ, double sign, cudaStream_t s) {
  const int64_t N = c->N;
  if (c->precision == FEP3M_MIXED)
    FEP3M_CL k_final<float><<<gsz(N), PT, 0, s>>>(N, c->n, c->inv_h, gU, sign, (const float4*)c->part, c->perm, c->cell,
                                         c->w_s, c->phi_s, c->E_s, c->psi_s, c->gpsi_s, (const double*)c->mu_v,
                                         (const double*)c->A_el, dpos, dQ);
  else
    FEP3M_CL k_final<double><<<gsz(N), PT, 0, s>>>(N, c->n, c->inv_h, gU, sign, (const vec4<double>::type*)c->part, c->perm,
                                          c->cell, c->w_s, c->phi_s, c->E_s, c->psi_s, c->gpsi_s,
                                          (const double*)c->mu_v, (const double*)c->A_el, dpos, dQ);
  return cudaGetLastError();
}

}  // namespace fep3m
