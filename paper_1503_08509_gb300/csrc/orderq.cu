// Screens of order q >= 2 (Sec. 2.1, Eq. moment1d) on the order p = q + 2 mesh
// (Sec. 2: p = q + 2): potentials and energy.
//
// The stages of Algorithm 1 for a general order:
//   coefficients  C[e][kappa] = sum_{j in e} Q_j c_kappa(delta_j) on the element's
//                 (q+1)^3 screen nodes (Eq. oned, Eq. moment1d; the weights are
//                 polynomials in delta / h made on the host);
//   density       r on the periodic order-q mesh (Eq. assign): the element lists
//                 added at the shared nodes;
//   load vector   b = 4 pi (Mpq (x) Mpq (x) Mpq) r, less its neutralising
//                 background (Sec. 2.2);
//   mesh solve    K phi = b, int phi = 0, by iterative refinement: the residual
//                 in FP64 (separable banded passes of the order-p matrices),
//                 the correction by the FP32 fast-diagonalisation solve of the
//                 order-p mesh (the tensor-core transform passes of the order-3
//                 mesh with the order-p eigenbasis);
//   screen field  S[e][m] = sum over the block elements e + d and their screen
//                 nodes kappa of C[e + d][kappa] times the FE table of kappa's
//                 type at node m of e (Eq. sc with the tables of the Remark of
//                 Sec. 4, in the node-regrouped layout, FP64);
//   evaluation    Phi_t = sum_m (phi - S)[e_t][m] u_m(tau_t) + the singular sum
//                 over the block (Eq. evalsmooth, Sec. 2.4), and U (FP64).
// One-element screens (Sec. 5.3) are the same stages with weights on the
// element's interior nodes only.  Both precisions take this path in FP64
// arithmetic, except the FP32 inner solve of the refinement and, in the mixed
// precision, the FP32 singular sums.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace fep3m {

namespace {

constexpr int OT = 256;

__device__ __forceinline__ int wrapq(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

inline unsigned gsz(int64_t n, int t = OT) { return (unsigned)((n + t - 1) / t); }

// C[e][kappa], one thread per (element, screen node); kappa = i + (q+1)(j + (q+1) k)
template <class V4>
__global__ void k_oq_coeff(int64_t ne, OQParams prm, const int* __restrict__ start, const int* __restrict__ count,
                           const V4* __restrict__ part, double* __restrict__ C) {
  const int q = prm.q, Q1 = q + 1, nk = Q1 * Q1 * Q1;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= ne * nk) return;
  const int64_t e = g / nk;
  const int kap = (int)(g - e * nk);
  const int ki[3] = {kap % Q1, (kap / Q1) % Q1, kap / (Q1 * Q1)};
  double acc = 0.0;
  const int s0 = start[e], cnt = count[e];
  for (int j = s0; j < s0 + cnt; ++j) {
    const V4 pj = part[j];
    const double t[3] = {(double)pj.x - 0.5, (double)pj.y - 0.5, (double)pj.z - 0.5};   // delta / h
    double w = (double)pj.w;
    for (int a = 0; a < 3; ++a) {
      const double* Wr = prm.W + ki[a] * Q1;
      double v = Wr[q];
      for (int l = q - 1; l >= 0; --l) v = fma(v, t[a], Wr[l]);   // Horner
      w *= v;
    }
    acc += w;
  }
  C[g] = acc;
}

// r on the order-q mesh: node g of an axis is local node g mod q of element
// g / q, and for g mod q = 0 also local node q of the element before
__global__ void k_oq_density(int n, int q, const double* __restrict__ C, double* __restrict__ r) {
  const int Nq = q * n, Q1 = q + 1, nk = Q1 * Q1 * Q1;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= (int64_t)Nq * Nq * Nq) return;
  const int gg[3] = {(int)(g % Nq), (int)((g / Nq) % Nq), (int)(g / ((int64_t)Nq * Nq))};
  int el[3][2], lo[3][2], cnt[3];
  for (int a = 0; a < 3; ++a) {
    el[a][0] = gg[a] / q;
    lo[a][0] = gg[a] - q * el[a][0];
    cnt[a] = 1;
    if (lo[a][0] == 0) {
      el[a][1] = wrapq(el[a][0] - 1, n);
      lo[a][1] = q;
      cnt[a] = 2;
    }
  }
  double acc = 0.0;
  for (int c = 0; c < cnt[2]; ++c)
    for (int b = 0; b < cnt[1]; ++b)
      for (int a = 0; a < cnt[0]; ++a) {
        const int64_t e = el[0][a] + (int64_t)n * (el[1][b] + (int64_t)n * el[2][c]);
        acc += C[e * nk + lo[0][a] + Q1 * (lo[1][b] + Q1 * lo[2][c])];
      }
  r[g] = acc;
}

// the screen nodes that order-p node g of an axis couples to, with the mixed
// mass weights: element g / p with local index g mod p, and for g mod p = 0
// also the element before with local index p
__device__ __forceinline__ int oq_mpq_row(int g, int n, const OQParams& prm, int node[10], double wgt[10]) {
  const int p = prm.p, q = prm.q, Q1 = q + 1, Nq = q * n;
  const int e = g / p, t = g - p * e;
  int k = 0;
  for (int j = 0; j <= q; ++j, ++k) {
    node[k] = wrapq(q * e + j, Nq);
    wgt[k] = prm.Mpq[t * Q1 + j];
  }
  if (t == 0)
    for (int j = 0; j <= q; ++j, ++k) {
      node[k] = wrapq(q * (e - 1) + j, Nq);
      wgt[k] = prm.Mpq[p * Q1 + j];
    }
  return k;
}

// b = 4 pi (Mpq (x) Mpq (x) Mpq) r
__global__ void k_oq_load(int n, OQParams prm, const double* __restrict__ r, double* __restrict__ b) {
  const int Np = prm.p * n, Nq = prm.q * n;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= (int64_t)Np * Np * Np) return;
  int nx[10], ny[10], nz[10];
  double wx[10], wy[10], wz[10];
  const int cx = oq_mpq_row((int)(g % Np), n, prm, nx, wx);
  const int cy = oq_mpq_row((int)((g / Np) % Np), n, prm, ny, wy);
  const int cz = oq_mpq_row((int)(g / ((int64_t)Np * Np)), n, prm, nz, wz);
  double acc = 0.0;
  for (int c = 0; c < cz; ++c)
    for (int bb = 0; bb < cy; ++bb) {
      const double wyz = wy[bb] * wz[c];
      const int64_t row = (int64_t)Nq * (ny[bb] + (int64_t)Nq * nz[c]);
      for (int a = 0; a < cx; ++a) acc += wx[a] * wyz * r[nx[a] + row];
    }
  b[g] = 4.0 * M_PI * acc;
}

// deterministic FP64 sum of v (or of w3 v, the node-integral weighted sum, with
// weighted): per-block partials, then one block adds them in order
__global__ void k_oq_partial(int64_t len, int Np, OQParams prm, int weighted, const double* __restrict__ v,
                             const double* __restrict__ v2, double* __restrict__ partial) {
  __shared__ double sh[OT / 32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    double x = v[i];
    if (v2) x *= v2[i];   // squares: v2 = v
    if (weighted) {
      const int p = prm.p;
      x *= prm.wn[(int)(i % Np) % p] * prm.wn[(int)((i / Np) % Np) % p] * prm.wn[(int)(i / ((int64_t)Np * Np)) % p];
    }
    acc += x;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < OT / 32; ++k) s += sh[k];
    partial[blockIdx.x] = s;
  }
}
__global__ void k_oq_final(int nb, const double* __restrict__ partial, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < nb; ++k) s += partial[k];
    *out = s;
  }
}

// out = in - s w3 (the load of a uniform background; w3 the node integrals) or,
// with constant, out = in - s (the mean); s = *sum * scale
__global__ void k_oq_subtract_w3(int Np, OQParams prm, const double* __restrict__ sum, double scale, int constant,
                                 const double* __restrict__ in, double* __restrict__ out) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= (int64_t)Np * Np * Np) return;
  const int p = prm.p;
  const double w = constant ? 1.0
                            : prm.wn[(int)(g % Np) % p] * prm.wn[(int)((g / Np) % Np) % p] *
                                  prm.wn[(int)(g / ((int64_t)Np * Np)) % p];
  out[g] = in[g] - (*sum) * scale * w;
}

// One axis of a separable banded apply on the periodic order-p mesh:
//   out = A_axis(in) [+ B_axis(in2) + C_axis(in3)], then out = base - out with base,
// the rows by node type (tap o couples node g to node g + o - p).
__global__ void k_oq_band(int Np, int axis, OQParams prm, int ma, const double* __restrict__ in, int mb,
                          const double* __restrict__ in2, int mc, const double* __restrict__ in3,
                          const double* __restrict__ base, double* __restrict__ out) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= (int64_t)Np * Np * Np) return;
  const int p = prm.p;
  int idx[3] = {(int)(g % Np), (int)((g / Np) % Np), (int)(g / ((int64_t)Np * Np))};
  const int64_t st[3] = {1, Np, (int64_t)Np * Np};
  const int ga = idx[axis], t = ga % p;
  const int64_t b0 = g - (int64_t)ga * st[axis];
  const double* rows[3] = {ma ? prm.bK[t] : prm.bM[t], mb ? prm.bK[t] : prm.bM[t], mc ? prm.bK[t] : prm.bM[t]};
  double acc = 0.0;
  for (int o = 0; o <= 2 * p; ++o) {
    const int64_t j = b0 + (int64_t)wrapq(ga + o - p, Np) * st[axis];
    double v = rows[0][o] * in[j];
    if (in2) v += rows[1][o] * in2[j];
    if (in3) v += rows[2][o] * in3[j];
    acc += v;
  }
  out[g] = base ? base[g] - acc : acc;
}

__global__ void k_oq_round(int64_t n, const double* __restrict__ in, double scale, float* __restrict__ out) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g < n) out[g] = (float)(in[g] * scale);
}
__global__ void k_oq_add(int64_t n, const float* __restrict__ x, double scale, double* __restrict__ phi, int first) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g < n) phi[g] = (first ? 0.0 : phi[g]) + (double)x[g] * scale;
}

// S[e][m] = sum_{d, kappa} C[e + d][kappa] H[o(d, kappa)][m], one CTA per
// non-empty element, one z plane of the block's source elements at a time in
// shared memory; o_a = q (n_sr + 1) - (q d_a + kappa_a)
__global__ void __launch_bounds__(128) k_oq_screen(int n, int n_sr, OQParams prm, const int* __restrict__ count,
                                                   const double* __restrict__ C, const double* __restrict__ H,
                                                   double* __restrict__ S) {
  extern __shared__ double cs[];   // (2 n_sr + 1)^2 (q+1)^3
  const int q = prm.q, p = prm.p, Q1 = q + 1, nk = Q1 * Q1 * Q1, P1 = p + 1, P3 = P1 * P1 * P1;
  const int nb = 2 * n_sr + 1, U = nb * q + 1, qk = q * (n_sr + 1);
  const int64_t e = blockIdx.x;
  if (count[e] == 0) return;
  const int ex = (int)(e % n), ey = (int)((e / n) % n), ez = (int)(e / ((int64_t)n * n));
  double acc[3] = {0.0, 0.0, 0.0};   // nodes m = tid + 128 k, P3 <= 384
  for (int dz = -n_sr; dz <= n_sr; ++dz) {
    __syncthreads();
    for (int i = threadIdx.x; i < nb * nb * nk; i += blockDim.x) {
      const int kap = i % nk, r2 = i / nk, dx = r2 % nb - n_sr, dy = r2 / nb - n_sr;
      const int64_t s = wrapq(ex + dx, n) + (int64_t)n * (wrapq(ey + dy, n) + (int64_t)n * wrapq(ez + dz, n));
      cs[i] = C[s * nk + kap];
    }
    __syncthreads();
    for (int r2 = 0; r2 < nb * nb; ++r2) {
      const int dx = r2 % nb - n_sr, dy = r2 / nb - n_sr;
      for (int kap = 0; kap < nk; ++kap) {
        const double c = cs[r2 * nk + kap];
        if (c == 0.0) continue;
        const int kx = kap % Q1, ky = (kap / Q1) % Q1, kz = kap / (Q1 * Q1);
        const int64_t o = (qk - (q * dx + kx)) + (int64_t)U * ((qk - (q * dy + ky)) + (int64_t)U * (qk - (q * dz + kz)));
        const double* h = H + o * P3;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int m = threadIdx.x + 128 * k;
          if (m < P3) acc[k] = fma(c, h[m], acc[k]);
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int m = threadIdx.x + 128 * k;
    if (m < P3) S[e * P3 + m] = acc[k];
  }
}

// Phi at each charge: (phi - S) contracted with the order-p shape functions
// at the charge (element units, FP64), plus the singular part already in phi_s
template <class V4>
__global__ void k_oq_eval(int64_t N, int n, OQParams prm, double inv_h, const int* __restrict__ perm,
                          const int* __restrict__ ecoord, const V4* __restrict__ part, const double* __restrict__ phi,
                          const double* __restrict__ S, double* __restrict__ phi_s, double* __restrict__ phi_out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= N) return;
  const int p = prm.p, P1 = p + 1, Np = p * n;
  const int ec = ecoord[t];
  const int ex = ec & 1023, ey = (ec >> 10) & 1023, ez = ec >> 20;
  const int64_t e = ex + (int64_t)n * (ey + (int64_t)n * ez);
  const V4 pt = part[t];
  const double tau[3] = {(double)pt.x, (double)pt.y, (double)pt.z};
  double l[3][7];   // equispaced order-p Lagrange values per axis
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k <= p; ++k) {
      double v = 1.0;
      for (int j = 0; j <= p; ++j)
        if (j != k) v *= (tau[a] * p - j) / (double)(k - j);
      l[a][k] = v;
    }
  const double* Se = S + e * (int64_t)(P1 * P1 * P1);
  double acc = 0.0;
  for (int mz = 0; mz <= p; ++mz) {
    const int64_t gz = (int64_t)Np * Np * wrapq(p * ez + mz, Np);
    for (int my = 0; my <= p; ++my) {
      const int64_t gy = gz + (int64_t)Np * wrapq(p * ey + my, Np);
      double row = 0.0;
      for (int mx = 0; mx <= p; ++mx)
        row += (phi[gy + wrapq(p * ex + mx, Np)] - Se[mx + P1 * (my + P1 * mz)]) * l[0][mx];
      acc += row * l[1][my] * l[2][mz];
    }
  }
  const double val = acc * inv_h + phi_s[t];
  phi_s[t] = val;
  if (phi_out) phi_out[perm[t]] = val;
}

// ---------------------------------------------------------------- host side
struct Reducer {
  OrderQ* o;
  int nb;
  // sum of v (v2: of v * v2; weighted: of w3 v) into dst (device); no sync
  void run(int64_t len, int Np, int weighted, const double* v, const double* v2, double* dst, cudaStream_t s) {
    FEP3M_CL k_oq_partial<<<nb, OT, 0, s>>>(len, Np, o->prm, weighted, v, v2, o->red);
    FEP3M_CL k_oq_final<<<1, 32, 0, s>>>(nb, o->red, dst);
  }
  double host(int64_t len, int Np, int weighted, const double* v, const double* v2, cudaStream_t s) {
    run(len, Np, weighted, v, v2, o->red + 1024, s);
    cudaMemcpyAsync(o->host_red, o->red + 1024, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    return *o->host_red;
  }
};

// r = pb - K phi with K = K1 (x) M1 (x) M1 + M1 (x) K1 (x) M1 + M1 (x) M1 (x) K1:
// a = M_z phi, b = K_z phi; c = M_y a, d = K_y a, f = M_y b; r = pb - (K_x c + M_x d + M_x f)
void oq_residual(OrderQ* o, int n, const double* phi, double* r, cudaStream_t s) {
  const int Np = o->p * n;
  const int64_t len = (int64_t)Np * Np * Np;
  double *a = o->t[0], *b = o->t[1], *c = o->t[2], *d = o->t[3];
  FEP3M_CL k_oq_band<<<gsz(len), OT, 0, s>>>(Np, 2, o->prm, 0, phi, 0, nullptr, 0, nullptr, nullptr, a);
  FEP3M_CL k_oq_band<<<gsz(len), OT, 0, s>>>(Np, 2, o->prm, 1, phi, 0, nullptr, 0, nullptr, nullptr, b);
  FEP3M_CL k_oq_band<<<gsz(len), OT, 0, s>>>(Np, 1, o->prm, 0, a, 0, nullptr, 0, nullptr, nullptr, c);
  FEP3M_CL k_oq_band<<<gsz(len), OT, 0, s>>>(Np, 1, o->prm, 1, a, 0, nullptr, 0, nullptr, nullptr, d);
  FEP3M_CL k_oq_band<<<gsz(len), OT, 0, s>>>(Np, 1, o->prm, 0, b, 0, nullptr, 0, nullptr, nullptr, a);
  FEP3M_CL k_oq_band<<<gsz(len), OT, 0, s>>>(Np, 0, o->prm, 1, c, 0, d, 0, a, o->pb, r);
}

// K phi = pb (pb neutral), int phi = 0: iterative refinement around the FP32
// fast-diagonalisation solve; returns the FP64 relative residual reached
cudaError_t oq_solve(fep3m_ctx* ctx, OrderQ* o, double rtol, int max_sweeps) {
  const int n = ctx->n, Np = o->p * n;
  const int64_t len = (int64_t)Np * Np * Np;
  cudaStream_t s = ctx->stream;
  Reducer red{o, (int)std::min<int64_t>(1024, std::max<int64_t>(1, len / (OT * 8)))};
  const double nb = std::sqrt(red.host(len, Np, 0, o->pb, o->pb, s));
  o->sweeps = 0;
  o->relres = 0.0;
  if (!(nb > 0.0)) {
    cudaMemsetAsync(o->phi, 0, len * sizeof(double), s);
    return cudaGetLastError();
  }
  cudaMemcpyAsync(o->res, o->pb, len * sizeof(double), cudaMemcpyDeviceToDevice, s);
  double nr = nb;
  for (int k = 0; k < max_sweeps; ++k) {
    // scale the residual by a power of two near 1 / RMS into FP32
    const double rms = nr / std::sqrt((double)len);
    const double sc = std::ldexp(1.0, -std::ilogb(rms));
    FEP3M_CL k_oq_round<<<gsz(len), OT, 0, s>>>(len, o->res, sc, o->r32);
    cudaError_t e = fdm_apply(o->fdm, o->r32, o->x32, o->w1, o->w2, s);
    if (e != cudaSuccess) return e;
    FEP3M_CL k_oq_add<<<gsz(len), OT, 0, s>>>(len, o->x32, 1.0 / sc, o->phi, k == 0);
    oq_residual(o, n, o->phi, o->res, s);
    nr = std::sqrt(red.host(len, Np, 0, o->res, o->res, s));
    o->sweeps = k + 1;
    o->relres = nr / nb;
    if (o->relres <= rtol) break;
  }
  // int phi = 0: remove the node-integral weighted mean the FP32 corrections leave
  red.run(len, Np, 1, o->phi, nullptr, o->red + 1025, s);
  FEP3M_CL k_oq_subtract_w3<<<gsz(len), OT, 0, s>>>(Np, o->prm, o->red + 1025, 1.0 / ((double)n * n * n), 1,
                                                    o->phi, o->phi);
  return cudaGetLastError();
}

void oq_params(const OrderQHost& h, OQParams& prm) {
  std::memset(&prm, 0, sizeof(prm));
  const int p = h.p, q = h.q, P1 = p + 1;
  prm.q = q;
  prm.p = p;
  for (size_t i = 0; i < h.W.size(); ++i) prm.W[i] = h.W[i];
  for (size_t i = 0; i < h.Mpq.size(); ++i) prm.Mpq[i] = h.Mpq[i];
  // global periodic rows: node type t = 0 (a vertex: local p of the element
  // before, local 0 of its own) or t (local t of its element)
  for (int t = 0; t < p; ++t) {
    auto add = [&](int local, int shift) {   // element whose local 0 sits at node g - shift
      for (int j = 0; j <= p; ++j) {
        const int o = j - shift + p;
        prm.bM[t][o] += h.Me[local * P1 + j];
        prm.bK[t][o] += h.Ke[local * P1 + j];
      }
    };
    if (t == 0) {
      add(p, p);
      add(0, 0);
    } else {
      add(t, t);
    }
    double wi = 0.0;
    const int li = t == 0 ? 0 : t;
    for (int j = 0; j <= p; ++j) wi += h.Me[li * P1 + j];   // int of the shape function (they sum to one)
    prm.wn[t] = t == 0 ? 2.0 * wi : wi;
  }
}

}  // namespace

int orderq_create(fep3m_ctx* c) {
  const int q = c->cfg.q, n = c->n;
  OrderQ* o = new (std::nothrow) OrderQ();
  if (!o) return FEP3M_ENOMEM;
  c->oq = o;
  const int pad = c->cfg.table_pad > 0 ? c->cfg.table_pad : 2;
  OrderQHost h;
  o->one_element = (c->cfg.flags & FEP3M_ONE_ELEMENT) != 0;
  if (!orderq_host(q, n, c->n_sr, pad, o->one_element, h)) return FEP3M_EINVAL;
  oq_params(h, o->prm);
  o->q = q;
  o->p = q + 2;
  o->Nq = q * n;
  o->Np = o->p * n;
  o->U = (2 * c->n_sr + 1) * q + 1;
  const int64_t ne = (int64_t)n * n * n, nq3 = (int64_t)o->Nq * o->Nq * o->Nq, np3 = (int64_t)o->Np * o->Np * o->Np;
  const int Q1 = q + 1, P1 = o->p + 1;
  cudaError_t e = cudaSuccess;
  auto al = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
  };
  al((void**)&o->C, ne * Q1 * Q1 * Q1 * sizeof(double));
  al((void**)&o->r, nq3 * sizeof(double));
  al((void**)&o->b, np3 * sizeof(double));
  al((void**)&o->pb, np3 * sizeof(double));
  al((void**)&o->phi, np3 * sizeof(double));
  al((void**)&o->res, np3 * sizeof(double));
  for (int k = 0; k < 4; ++k) al((void**)&o->t[k], np3 * sizeof(double));
  al((void**)&o->r32, np3 * sizeof(float));
  al((void**)&o->x32, np3 * sizeof(float));
  al((void**)&o->w1, np3 * sizeof(float));
  al((void**)&o->w2, np3 * sizeof(float));
  al((void**)&o->S, ne * P1 * P1 * P1 * sizeof(double));
  al((void**)&o->H, h.H.size() * sizeof(double));
  al((void**)&o->red, 1040 * sizeof(double));
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? FEP3M_ENOMEM : FEP3M_ECUDA;
  if (cudaMallocHost(&o->host_red, sizeof(double)) != cudaSuccess) return FEP3M_ENOMEM;
  cudaMemcpy(o->H, h.H.data(), h.H.size() * sizeof(double), cudaMemcpyHostToDevice);
  e = fdm_setup(o->fdm, o->Np, h.lam, h.V, 1, !(c->cfg.flags & FEP3M_CUDA_CORES));
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? FEP3M_ENOMEM : FEP3M_ECUDA;
  const size_t smem = (size_t)(2 * c->n_sr + 1) * (2 * c->n_sr + 1) * Q1 * Q1 * Q1 * sizeof(double);
  if (cudaFuncSetAttribute(k_oq_screen, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return FEP3M_ECUDA;
  return FEP3M_OK;
}

void orderq_destroy(fep3m_ctx* c) {
  OrderQ* o = c->oq;
  if (!o) return;
  void* p[] = {o->C, o->r, o->b, o->pb, o->phi, o->res, o->t[0], o->t[1], o->t[2], o->t[3], o->r32, o->x32,
               o->w1, o->w2, o->S, o->H, o->red};
  for (void* x : p)
    if (x) cudaFree(x);
  if (o->host_red) cudaFreeHost(o->host_red);
  fdm_free(o->fdm);
  delete o;
  c->oq = nullptr;
}

// the load vector less its background, from b (device)
static void oq_project(fep3m_ctx* c, OrderQ* o, cudaStream_t s) {
  const int n = c->n, Np = o->Np;
  const int64_t len = (int64_t)Np * Np * Np;
  Reducer red{o, (int)std::min<int64_t>(1024, std::max<int64_t>(1, len / (OT * 8)))};
  red.run(len, Np, 0, o->b, nullptr, o->red + 1026, s);
  FEP3M_CL k_oq_subtract_w3<<<gsz(len), OT, 0, s>>>(Np, o->prm, o->red + 1026, 1.0 / ((double)n * n * n), 0, o->b,
                                                    o->pb);
}

static double oq_rtol(const fep3m_ctx* c) {
  return c->cfg.mg_rtol > 0 ? c->cfg.mg_rtol : (c->precision == FEP3M_FP64 ? 1e-13 : 1e-10);
}

int orderq_compute(fep3m_ctx* c, double* phi_dev, double* U_dev) {
  OrderQ* o = c->oq;
  const int n = c->n, q = o->q, Q1 = q + 1, P1 = o->p + 1;
  const int64_t ne = (int64_t)n * n * n, N = c->N;
  const int64_t nq3 = (int64_t)o->Nq * o->Nq * o->Nq, np3 = (int64_t)o->Np * o->Np * o->Np;
  cudaStream_t s = c->stream;
  const int64_t nc = ne * Q1 * Q1 * Q1;
  if (c->precision == FEP3M_MIXED)
    FEP3M_CL k_oq_coeff<float4><<<gsz(nc), OT, 0, s>>>(ne, o->prm, c->start, c->count, (const float4*)c->part, o->C);
  else
    FEP3M_CL k_oq_coeff<vec4<double>::type><<<gsz(nc), OT, 0, s>>>(ne, o->prm, c->start, c->count,
                                                                     (const vec4<double>::type*)c->part, o->C);
  FEP3M_CL k_oq_density<<<gsz(nq3), OT, 0, s>>>(n, q, o->C, o->r);
  FEP3M_CL k_oq_load<<<gsz(np3), OT, 0, s>>>(n, o->prm, o->r, o->b);
  oq_project(c, o, s);
  cudaError_t e = oq_solve(c, o, oq_rtol(c), c->cfg.mg_max_cycles > 0 ? c->cfg.mg_max_cycles : 10);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? FEP3M_ENOMEM : FEP3M_ECUDA;
  const size_t smem = (size_t)(2 * c->n_sr + 1) * (2 * c->n_sr + 1) * Q1 * Q1 * Q1 * sizeof(double);
  FEP3M_CL k_oq_screen<<<(unsigned)ne, 128, smem, s>>>(n, c->n_sr, o->prm, c->count, o->C, o->H, o->S);
  if ((e = singular_sums(c, c->Q_s, c->phi_s, c->E_s, s)) != cudaSuccess) return FEP3M_ECUDA;
  if (c->precision == FEP3M_MIXED)
    FEP3M_CL k_oq_eval<float4><<<gsz(N), OT, 0, s>>>(N, n, o->prm, c->inv_h, c->perm, c->ecoord,
                                                      (const float4*)c->part, o->phi, o->S, c->phi_s, phi_dev);
  else
    FEP3M_CL k_oq_eval<vec4<double>::type><<<gsz(N), OT, 0, s>>>(N, n, o->prm, c->inv_h, c->perm, c->ecoord,
                                                                  (const vec4<double>::type*)c->part, o->phi, o->S,
                                                                  c->phi_s, phi_dev);
  if (U_dev && (e = energy(c, U_dev)) != cudaSuccess) return FEP3M_ECUDA;
  (void)P1;
  e = cudaGetLastError();
  if (e != cudaSuccess) return FEP3M_ECUDA;
  return o->relres <= 10 * oq_rtol(c) ? FEP3M_OK : FEP3M_ENOCONV;
}

int orderq_solve(fep3m_ctx* c, const double* b_dev, double* phi_dev) {
  OrderQ* o = c->oq;
  const int64_t np3 = (int64_t)o->Np * o->Np * o->Np;
  cudaStream_t s = c->stream;
  cudaMemcpyAsync(o->b, b_dev, np3 * sizeof(double), cudaMemcpyDeviceToDevice, s);
  oq_project(c, o, s);
  cudaError_t e = oq_solve(c, o, oq_rtol(c), c->cfg.mg_max_cycles > 0 ? c->cfg.mg_max_cycles : 10);
  if (e != cudaSuccess) return FEP3M_ECUDA;
  cudaMemcpyAsync(phi_dev, o->phi, np3 * sizeof(double), cudaMemcpyDeviceToDevice, s);
  return o->relres <= 10 * oq_rtol(c) ? FEP3M_OK : FEP3M_ENOCONV;
}

}  // namespace fep3m
