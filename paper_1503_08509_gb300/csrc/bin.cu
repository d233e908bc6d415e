// Binning of charges into FE elements (Sec. 3.1.1: "the element containing
// each charge is identified, and the offsets from the center of these
// elements determined"): wrap, element id, FP64 offset, and a stable counting
// sort (count -> exclusive scan -> scatter -> per-element index sort) so the
// sorted order is unique: by element, then by original index.
#include <cmath>

#include "common.cuh"

namespace fep3m {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;

// x -> element and offset, written with explicit round-to-nearest intrinsics
// so that no multiply-add is fused: the result is bit-identical to the same
// expression evaluated one IEEE operation at a time.  Periodic cube (box_L =
// 0): x wrapped into [0, L), element index at most n - 1.  Box [0, box_L]^3
// (box_L > 0, L the longer padded period, which wraps nothing in the box): a
// coordinate outside the box is an input error, the element index at most
// cmax (a charge on the far face belongs to the last box element).
__global__ void k_bin(const double* __restrict__ pos, const double* __restrict__ Q, int64_t N, double L,
                      int n, double h, double inv_h, double box_L, int cmax, int* __restrict__ cell,
                      double* __restrict__ delta, int* __restrict__ count, int* __restrict__ err) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  int c3[3];
  bool bad = !isfinite(Q[i]);
  for (int a = 0; a < 3; ++a) {
    double x = pos[3 * i + a];
    if (!isfinite(x) || (box_L > 0.0 && !(x >= 0.0 && x <= box_L))) {
      bad = true;
      x = 0.0;
    }
    double fl = floor(x / L);
    double xw = __dsub_rn(x, __dmul_rn(L, fl));
    if (xw >= L) xw = 0.0;
    double cf = floor(__dmul_rn(xw, inv_h));
    int c = (int)fmax(0.0, fmin(cf, (double)cmax));
    c3[a] = c;
    delta[3 * i + a] = __dsub_rn(xw, __dmul_rn((double)c + 0.5, h));
  }
  if (bad) atomicOr(err, 1);
  int e = c3[0] + n * (c3[1] + n * c3[2]);
  cell[i] = e;
  atomicAdd(&count[e], 1);
}

__device__ __forceinline__ int block_exclusive_scan(int v, int* sh, int& total) {
  // warp-level inclusive scan, then across warps
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sh[lane] = w;
  }
  __syncthreads();
  int warp_off = wid ? sh[wid - 1] : 0;
  total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return warp_off + x - v;
}

__global__ void k_scan_sums(const int* __restrict__ in, int64_t n, int* __restrict__ bsum) {
  __shared__ int sh[32];
  int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanPer;
  int s = 0;
  for (int k = 0; k < kScanPer; ++k)
    if (base + k < n) s += in[base + k];
  int total;
  block_exclusive_scan(s, sh, total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// exclusive scan of the block sums by one block (looping over chunks)
__global__ void k_scan_block_sums(int* __restrict__ bsum, int nb) {
  __shared__ int sh[32];
  int carry = 0;
  for (int base = 0; base < nb; base += blockDim.x * kScanPer) {
    int v[kScanPer];
    int s = 0;
    for (int k = 0; k < kScanPer; ++k) {
      int idx = base + threadIdx.x * kScanPer + k;
      v[k] = idx < nb ? bsum[idx] : 0;
      s += v[k];
    }
    int total;
    int off = block_exclusive_scan(s, sh, total);
    int run = carry + off;
    for (int k = 0; k < kScanPer; ++k) {
      int idx = base + threadIdx.x * kScanPer + k;
      if (idx < nb) bsum[idx] = run;
      run += v[k];
    }
    carry += total;
    __syncthreads();
  }
}

__global__ void k_scan_final(const int* __restrict__ in, int64_t n, const int* __restrict__ boff, int* __restrict__ out) {
  __shared__ int sh[32];
  int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanPer;
  int v[kScanPer];
  int s = 0;
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  int total;
  int run = boff[blockIdx.x] + block_exclusive_scan(s, sh, total);
  for (int k = 0; k < kScanPer; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (base <= n - 1 && n - 1 < base + kScanPer) out[n] = run;   // total after the last element
}

__global__ void k_scatter(const int* __restrict__ cell, int64_t N, const int* __restrict__ start,
                          int* __restrict__ fill, int* __restrict__ perm) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  int e = cell[i];
  int slot = start[e] + atomicAdd(&fill[e], 1);
  perm[slot] = (int)i;
}

// the atomics above leave each element's segment in arbitrary order; sort it by index
__global__ void k_sort_segments(int64_t ne, const int* __restrict__ start, const int* __restrict__ count,
                                int* __restrict__ perm) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= ne) return;
  int s = start[e], c = count[e];
  for (int a = s + 1; a < s + c; ++a) {
    int v = perm[a];
    int b = a - 1;
    while (b >= s && perm[b] > v) {
      perm[b + 1] = perm[b];
      --b;
    }
    perm[b + 1] = v;
  }
}

// sorted structure of arrays: local coordinates t = delta / h + 1/2 in [0, 1] and Q, and the sorted
// charges in FP64 as the working precision holds them (Qs)
template <class T>
__global__ void k_gather(int64_t N, int n, const int* __restrict__ perm, const int* __restrict__ cell,
                         const double* __restrict__ delta, const double* __restrict__ Q, double inv_h,
                         typename vec4<T>::type* __restrict__ part, int* __restrict__ ecoord, double* __restrict__ Qs) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= N) return;
  int i = perm[k];
  const int e = cell[i];
  ecoord[k] = (e % n) | (((e / n) % n) << 10) | ((e / (n * n)) << 20);
  typename vec4<T>::type p;
  p.x = (T)(delta[3 * i] * inv_h + 0.5);
  p.y = (T)(delta[3 * i + 1] * inv_h + 0.5);
  p.z = (T)(delta[3 * i + 2] * inv_h + 0.5);
  p.w = (T)Q[i];
  part[k] = p;
  Qs[k] = (double)p.w;
}

}  // namespace

static cudaError_t exclusive_scan(const int* in, int64_t n, int* out, int* tmp, cudaStream_t s) {
  int nb = (int)((n + kScanTile - 1) / kScanTile);
  FEP3M_CL k_scan_sums<<<nb, kScanThreads, 0, s>>>(in, n, tmp);
  FEP3M_CL k_scan_block_sums<<<1, kScanThreads, 0, s>>>(tmp, nb);
  FEP3M_CL k_scan_final<<<nb, kScanThreads, 0, s>>>(in, n, tmp, out);
  return cudaGetLastError();
}

size_t scan_tmp_bytes(int64_t n) { return sizeof(int) * (size_t)((n + kScanTile - 1) / kScanTile + 1); }

cudaError_t bin_particles(fep3m_ctx* c, const double* pos, const double* Q, int use_fp32) {
  const int64_t ne = (int64_t)c->n * c->n * c->n;
  cudaStream_t s = c->stream;
  cudaMemsetAsync(c->count, 0, sizeof(int) * ne, s);
  cudaMemsetAsync(c->fill, 0, sizeof(int) * ne, s);
  const int T = 256;
  const int gN = (int)((c->N + T - 1) / T), gE = (int)((ne + T - 1) / T);
  const double box_L = c->box ? c->cfg.L : 0.0;
  const int cmax = c->box ? c->box->nb - 1 : c->n - 1;
  FEP3M_CL k_bin<<<gN, T, 0, s>>>(pos, Q, c->N, c->L, c->n, c->h, c->inv_h, box_L, cmax, c->cell, c->delta, c->count,
                                  c->iflags);
  cudaError_t e = exclusive_scan(c->count, ne, c->start, (int*)c->scan_tmp, s);
  if (e != cudaSuccess) return e;
  FEP3M_CL k_scatter<<<gN, T, 0, s>>>(c->cell, c->N, c->start, c->fill, c->perm);
  FEP3M_CL k_sort_segments<<<gE, T, 0, s>>>(ne, c->start, c->count, c->perm);
  if (use_fp32)
    FEP3M_CL k_gather<float><<<gN, T, 0, s>>>(c->N, c->n, c->perm, c->cell, c->delta, Q, c->inv_h, (float4*)c->part,
                                              c->ecoord, c->Q_s);
  else
    FEP3M_CL k_gather<double><<<gN, T, 0, s>>>(c->N, c->n, c->perm, c->cell, c->delta, Q, c->inv_h,
                                               (vec4<double>::type*)c->part, c->ecoord, c->Q_s);
  return cudaGetLastError();
}

}  // namespace fep3m
