// Create-time host computations for screens of any order q and the order
// p = q + 2 mesh: Lagrange element matrices (equispaced order-p mesh basis,
// Gauss-Lobatto order-q screen basis), the 1-D eigenbasis of
// the periodic order-p mesh (block-Fourier reduction), and the FE tables of the
// q^3 basis-screen types (Remark of Sec. 4).  Host code only; nothing here runs
// per evaluation.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#include "common.cuh"

namespace fep3m {

namespace {

// Nodes on [0, 1] of the order-p Lagrange basis: equispaced (the order-p mesh
// space, which does not depend on them) or Gauss-Lobatto-Legendre (the order-q
// screen basis: the ends and the roots of P_q', closed forms for q <= 4; the two
// sets coincide for q <= 2).
void node_set(int p, bool gll, double* x) {
  for (int k = 0; k <= p; ++k) x[k] = (double)k / p;
  if (!gll || p <= 2) return;
  if (p == 3) {
    const double r = 1.0 / std::sqrt(5.0);
    x[1] = 0.5 * (1.0 - r);
    x[2] = 0.5 * (1.0 + r);
  } else if (p == 4) {
    const double r = std::sqrt(3.0 / 7.0);
    x[1] = 0.5 * (1.0 - r);
    x[2] = 0.5;
    x[3] = 0.5 * (1.0 + r);
  }
}

// Order-p Lagrange basis on the nodes x at t, and its derivative (product
// rule, one factor at a time).
void lagrange(int p, const double* x, double t, double* v, double* d) {
  for (int k = 0; k <= p; ++k) {
    const double xk = x[k];
    double val = 1.0, der = 0.0;
    for (int j = 0; j <= p; ++j) {
      if (j == k) continue;
      const double xj = x[j], den = xk - xj;
      der = der * (t - xj) / den + val / den;
      val *= (t - xj) / den;
    }
    v[k] = val;
    if (d) d[k] = der;
  }
}

// Element matrices on [0, 1] (h = 1): mass Me and stiffness Ke of the order-p
// basis ((p+1) x (p+1), equispaced nodes), mixed mass Mpq = int l^p_i l^q_j
// ((p+1) x (q+1), the order-q screen basis on Gauss-Lobatto nodes).
struct ElementPQ {
  int p, q;
  std::vector<double> Me, Ke, Mpq;
  ElementPQ(int p_, int q_) : p(p_), q(q_), Me((p_ + 1) * (p_ + 1)), Ke((p_ + 1) * (p_ + 1)), Mpq((p_ + 1) * (q_ + 1)) {
    std::vector<double> x, w;
    gauss_legendre01(p + 2, x, w);   // exact for degree 2 p + 3
    std::vector<double> v(p + 1), d(p + 1), vq(q + 1), np_(p + 1), nq(q + 1);
    node_set(p, false, np_.data());
    node_set(q, true, nq.data());
    for (size_t g = 0; g < x.size(); ++g) {
      lagrange(p, np_.data(), x[g], v.data(), d.data());
      lagrange(q, nq.data(), x[g], vq.data(), nullptr);
      for (int i = 0; i <= p; ++i) {
        for (int j = 0; j <= p; ++j) {
          Me[i * (p + 1) + j] += w[g] * v[i] * v[j];
          Ke[i * (p + 1) + j] += w[g] * d[i] * d[j];
        }
        for (int j = 0; j <= q; ++j) Mpq[i * (q + 1) + j] += w[g] * v[i] * vq[j];
      }
    }
  }
};

// y = A x along one axis of an n0 x n1 x n2 array (index i0 + n0 (i1 + n1 i2)),
// A dense na x na (row major), na = the axis length.
void axis_apply(const int dims[3], const std::vector<double>& A, const std::vector<double>& x, std::vector<double>& y,
                int axis, bool transpose) {
  y.assign(x.size(), 0.0);
  const size_t s[3] = {1, (size_t)dims[0], (size_t)dims[0] * dims[1]};
  const int na = dims[axis], o1 = (axis + 1) % 3, o2 = (axis + 2) % 3;
  for (int j1 = 0; j1 < dims[o1]; ++j1)
    for (int j2 = 0; j2 < dims[o2]; ++j2) {
      const size_t base = j1 * s[o1] + j2 * s[o2];
      for (int i = 0; i < na; ++i) {
        double acc = 0;
        for (int k = 0; k < na; ++k)
          acc += (transpose ? A[(size_t)k * na + i] : A[(size_t)i * na + k]) * x[base + k * s[axis]];
        y[base + i * s[axis]] = acc;
      }
    }
}

// Quadrature of the 1-D type-t order-q nodal function (Gauss-Lobatto nodes; anchor at 0, element
// units): points and weights times the function, ngl Gauss points per
// polynomial piece.  Type 0: the vertex function on [-1, 0] (local node q of
// the left element) and [0, 1] (local node 0 of the right one); type t >= 1:
// local node t of the element [0, 1].
void type_quadrature(int q, int t, int ngl, std::vector<double>& px, std::vector<double>& pw) {
  std::vector<double> x, w, vq(q + 1), nq(q + 1);
  gauss_legendre01(ngl, x, w);
  node_set(q, true, nq.data());
  px.clear();
  pw.clear();
  auto piece = [&](double lo, int node) {
    for (int g = 0; g < ngl; ++g) {
      lagrange(q, nq.data(), x[g], vq.data(), nullptr);
      px.push_back(lo + x[g]);
      pw.push_back(w[g] * vq[node]);
    }
  };
  if (t == 0) {
    piece(-1.0, q);
    piece(0.0, 0);
  } else {
    piece(0.0, t);
  }
}

}  // namespace

// Generalized eigenpairs K1 v = lam M1 v of the periodic 1-D order-p matrices on
// n elements (N = p n nodes), V M1-orthonormal, V[node * N + mode].  The
// matrices are block circulant with p x p blocks B_d (d = -1, 0, 1): element
// e's local node l is node l mod p of element e + [l = p].  Per wavenumber
// k (theta = 2 pi k / n) the span of {cos(theta e) w, sin(theta e) w} is
// invariant, so each k is a 2p x 2p problem (p x p for k = 0 and k = n / 2)
// with the matrices (n/2) [[Sc, Ss], [-Ss, Sc]], Sc = sum_d B_d cos(theta d),
// Ss = sum_d B_d sin(theta d), and n Sc for the real modes.
void periodic_eigen_order(int p, int n, std::vector<double>& lam, std::vector<double>& V) {
  const ElementPQ E(p, 1);
  const int N = p * n, pp = p * p;
  std::vector<double> BK(3 * pp, 0.0), BM(3 * pp, 0.0);   // [d + 1][tau][tau']
  for (int l = 0; l <= p; ++l)
    for (int l2 = 0; l2 <= p; ++l2) {
      const int d = (l2 == p) - (l == p);
      const size_t at = (size_t)(d + 1) * pp + (l % p) * p + (l2 % p);
      BK[at] += E.Ke[l * (p + 1) + l2];
      BM[at] += E.Me[l * (p + 1) + l2];
    }
  lam.clear();
  V.assign((size_t)N * N, 0.0);
  int mode = 0;
  for (int k = 0; 2 * k <= n; ++k) {
    const double th = 2.0 * M_PI * k / n;
    const bool real = k == 0 || 2 * k == n;
    const int m = real ? p : 2 * p;
    std::vector<double> Kc(pp, 0.0), Ks(pp, 0.0), Mc(pp, 0.0), Ms(pp, 0.0);
    for (int d = -1; d <= 1; ++d)
      for (int i = 0; i < pp; ++i) {
        Kc[i] += BK[(d + 1) * pp + i] * std::cos(th * d);
        Ks[i] += BK[(d + 1) * pp + i] * std::sin(th * d);
        Mc[i] += BM[(d + 1) * pp + i] * std::cos(th * d);
        Ms[i] += BM[(d + 1) * pp + i] * std::sin(th * d);
      }
    const double w = real ? (double)n : 0.5 * n;
    std::vector<double> A((size_t)m * m, 0.0), B((size_t)m * m, 0.0);
    for (int a = 0; a < p; ++a)
      for (int b = 0; b < p; ++b) {
        A[(size_t)a * m + b] = w * Kc[a * p + b];
        B[(size_t)a * m + b] = w * Mc[a * p + b];
        if (!real) {
          A[(size_t)a * m + p + b] = w * Ks[a * p + b];
          A[(size_t)(p + a) * m + b] = -w * Ks[a * p + b];
          A[(size_t)(p + a) * m + p + b] = w * Kc[a * p + b];
          B[(size_t)a * m + p + b] = w * Ms[a * p + b];
          B[(size_t)(p + a) * m + b] = -w * Ms[a * p + b];
          B[(size_t)(p + a) * m + p + b] = w * Mc[a * p + b];
        }
      }
    std::vector<double> lk, vk;
    generalized_eigen(m, A, B, lk, vk);
    for (int j = 0; j < m; ++j, ++mode) {
      lam.push_back(lk[j]);
      for (int e = 0; e < n; ++e) {
        const double ce = std::cos(th * e), se = std::sin(th * e);
        for (int tau = 0; tau < p; ++tau) {
          double v = vk[(size_t)tau * m + j] * ce;
          if (!real) v += vk[(size_t)(p + tau) * m + j] * se;
          V[(size_t)(p * e + tau) * N + mode] = v;
        }
      }
    }
  }
}

// FE table of the basis screen of type (t0, t1, t2) (order q, order-p mesh,
// h = 1; Remark of Sec. 4): the Galerkin solution H of -Lap H = 4 pi psi on a
// box extending B = keep + pad elements beyond the screen's anchor vertex on
// each side, and one element more on the right along interior-type axes (so
// the box is symmetric about the screen's support), with the continuum
// potential of psi (Eq. screenintegral, tensor Gauss-Legendre, ngl points per
// piece) as Dirichlet data, solved exactly by fast diagonalisation of the 1-D
// Dirichlet pencils.  Returns the nodal values on [-keep, keep]^3 about the
// anchor, K = 2 keep p + 1 per axis, index ix + K (iy + K iz).
void screen_type_table(int p, int q, const int t3[3], int keep, int pad, int ngl, std::vector<double>& kept) {
  const ElementPQ E(p, q);
  const int B = keep + pad;
  int nel[3], dims[3], dI[3];
  std::vector<double> M1[3], K1[3], m1[3], qx[3], qw[3];
  for (int a = 0; a < 3; ++a) {
    nel[a] = 2 * B + (t3[a] ? 1 : 0);
    const int N = p * nel[a] + 1;
    dims[a] = N;
    dI[a] = N - 2;
    M1[a].assign((size_t)N * N, 0.0);
    K1[a].assign((size_t)N * N, 0.0);
    for (int e = 0; e < nel[a]; ++e)
      for (int i = 0; i <= p; ++i)
        for (int j = 0; j <= p; ++j) {
          M1[a][(size_t)(p * e + i) * N + p * e + j] += E.Me[i * (p + 1) + j];
          K1[a][(size_t)(p * e + i) * N + p * e + j] += E.Ke[i * (p + 1) + j];
        }
    // int phi^p_k psi_t: the anchor is the left end of element B
    m1[a].assign(N, 0.0);
    for (int k = 0; k <= p; ++k) {
      if (t3[a] == 0) {
        m1[a][p * (B - 1) + k] += E.Mpq[k * (q + 1) + q];
        m1[a][p * B + k] += E.Mpq[k * (q + 1) + 0];
      } else {
        m1[a][p * B + k] += E.Mpq[k * (q + 1) + t3[a]];
      }
    }
    type_quadrature(q, t3[a], ngl, qx[a], qw[a]);
  }
  const size_t NN = (size_t)dims[0] * dims[1] * dims[2];
  std::vector<double> H(NN, 0.0);
  auto idx = [&](int i, int j, int k) { return i + (size_t)dims[0] * (j + (size_t)dims[1] * k); };
  auto pos = [&](int k) { return -B + (double)k / p; };
  for (int k = 0; k < dims[2]; ++k)
    for (int j = 0; j < dims[1]; ++j)
      for (int i = 0; i < dims[0]; ++i) {
        if (!(i == 0 || j == 0 || k == 0 || i == dims[0] - 1 || j == dims[1] - 1 || k == dims[2] - 1)) continue;
        const double x = pos(i), y = pos(j), z = pos(k);
        double acc = 0;
        for (size_t c = 0; c < qx[2].size(); ++c) {
          const double dz = z - qx[2][c];
          for (size_t b = 0; b < qx[1].size(); ++b) {
            const double dy = y - qx[1][b], wyz = qw[1][b] * qw[2][c];
            for (size_t g = 0; g < qx[0].size(); ++g) {
              const double dx = x - qx[0][g];
              acc += qw[0][g] * wyz / std::sqrt(dx * dx + dy * dy + dz * dz);
            }
          }
        }
        H[idx(i, j, k)] = acc;
      }
  // interior residual rhs - K Hb, K = K1 (x) M1 (x) M1 + M1 (x) K1 (x) M1 + M1 (x) M1 (x) K1
  std::vector<double> tA, tB, tC, acc(NN, 0.0);
  for (int term = 0; term < 3; ++term) {
    axis_apply(dims, term == 0 ? K1[0] : M1[0], H, tA, 0, false);
    axis_apply(dims, term == 1 ? K1[1] : M1[1], tA, tB, 1, false);
    axis_apply(dims, term == 2 ? K1[2] : M1[2], tB, tC, 2, false);
    for (size_t i = 0; i < NN; ++i) acc[i] += tC[i];
  }
  const size_t NI = (size_t)dI[0] * dI[1] * dI[2];
  std::vector<double> r(NI);
  for (int k = 0; k < dI[2]; ++k)
    for (int j = 0; j < dI[1]; ++j)
      for (int i = 0; i < dI[0]; ++i)
        r[i + (size_t)dI[0] * (j + (size_t)dI[1] * k)] =
            4.0 * M_PI * m1[0][i + 1] * m1[1][j + 1] * m1[2][k + 1] - acc[idx(i + 1, j + 1, k + 1)];
  std::vector<double> lam[3], Vv[3];
  for (int a = 0; a < 3; ++a) {
    const int n = dI[a], N = dims[a];
    std::vector<double> KI((size_t)n * n), MI((size_t)n * n);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        KI[(size_t)i * n + j] = K1[a][(size_t)(i + 1) * N + j + 1];
        MI[(size_t)i * n + j] = M1[a][(size_t)(i + 1) * N + j + 1];
      }
    generalized_eigen(n, KI, MI, lam[a], Vv[a]);
  }
  std::vector<double> s1, s2;
  axis_apply(dI, Vv[0], r, s1, 0, true);
  axis_apply(dI, Vv[1], s1, s2, 1, true);
  axis_apply(dI, Vv[2], s2, s1, 2, true);
  for (int k = 0; k < dI[2]; ++k)
    for (int j = 0; j < dI[1]; ++j)
      for (int i = 0; i < dI[0]; ++i) s1[i + (size_t)dI[0] * (j + (size_t)dI[1] * k)] /= lam[0][i] + lam[1][j] + lam[2][k];
  axis_apply(dI, Vv[0], s1, s2, 0, false);
  axis_apply(dI, Vv[1], s2, s1, 1, false);
  axis_apply(dI, Vv[2], s1, s2, 2, false);
  for (int k = 0; k < dI[2]; ++k)
    for (int j = 0; j < dI[1]; ++j)
      for (int i = 0; i < dI[0]; ++i) H[idx(i + 1, j + 1, k + 1)] = s2[i + (size_t)dI[0] * (j + (size_t)dI[1] * k)];
  const int K = 2 * keep * p + 1, o = p * (B - keep);
  kept.assign((size_t)K * K * K, 0.0);
  for (int k = 0; k < K; ++k)
    for (int j = 0; j < K; ++j)
      for (int i = 0; i < K; ++i) kept[i + (size_t)K * (j + (size_t)K * k)] = H[idx(i + o, j + o, k + o)];
}

// The table operand of the node-regrouped screen contraction for order q
// (Sec. 2.4, Eq. sc with the Remark's tables): the screens of a target
// element's block are sums over the order-q screen nodes u of the block
// (U = (2 n_sr + 1) q + 1 per axis, u = -q n_sr .. q (n_sr + 1) in steps of
// 1 / q element from the target element's origin), each node's weight times
// the table of its type (u mod q) anchored at floor(u / q).  Row o (per axis
// o = q (n_sr + 1) - u, so that q = 1 gives the vertex-offset order of the
// order-1 contraction) holds that table at the (p+1)^3 nodes m of the target
// element: table index p ceil(o / q) + m along each axis.  H[o * (p+1)^3 + m],
// o = ox + U (oy + U oz), m = mx + (p+1) (my + (p+1) mz).
void screen_node_table(int q, int n_sr, int pad, int ngl, std::vector<double>& H) {
  const int p = q + 2, keep = n_sr + 1, U = (2 * n_sr + 1) * q + 1, P1 = p + 1, K = 2 * keep * p + 1;
  std::vector<std::vector<double>> T((size_t)q * q * q);
  for (int tz = 0; tz < q; ++tz)
    for (int ty = 0; ty < q; ++ty)
      for (int tx = 0; tx < q; ++tx) {
        const int t3[3] = {tx, ty, tz};
        screen_type_table(p, q, t3, keep, pad, ngl, T[tx + q * (ty + q * tz)]);
      }
  const int M = P1 * P1 * P1;
  H.assign((size_t)U * U * U * M, 0.0);
  for (int oz = 0; oz < U; ++oz)
    for (int oy = 0; oy < U; ++oy)
      for (int ox = 0; ox < U; ++ox) {
        const int o[3] = {ox, oy, oz};
        int type[3], base[3];
        for (int a = 0; a < 3; ++a) {
          type[a] = (q - o[a] % q) % q;            // (u mod q) with u = q keep - o
          base[a] = p * ((o[a] + q - 1) / q);      // p ceil(o / q)
        }
        const std::vector<double>& Tt = T[type[0] + q * (type[1] + q * type[2])];
        double* row = H.data() + ((size_t)ox + (size_t)U * (oy + (size_t)U * oz)) * M;
        for (int mz = 0; mz < P1; ++mz)
          for (int my = 0; my < P1; ++my)
            for (int mx = 0; mx < P1; ++mx)
              row[mx + P1 * (my + P1 * mz)] =
                  Tt[(base[0] + mx) + (size_t)K * ((base[1] + my) + (size_t)K * (base[2] + mz))];
      }
}

// Screen weights as polynomials in delta / h (Eq. moment1d): per axis the
// weights w_i(delta) of the order-q nodal functions of the charge's element
// solve sum_i Omega[l][i] w_i = delta^l, Omega[l][i] = int x^l omega_i(x) dx
// (centred element [-1/2, 1/2], h = 1; the vertex functions reach into the
// neighbouring elements), so w = Omega^-1 (1, delta, delta^2, ...) and
// W = Omega^-1 holds the coefficients: w_i = sum_l W[i][l] (delta / h)^l / h.
// One-element screens (Sec. 5.3) use the interior functions only, with the
// moments l < q - 1; their rows and columns sit at i = 1 .. q-1, l = 0 .. q-2,
// the rest zero.  Gauss-Lobatto nodes, as the type tables.  Returns false if
// the moment matrix is singular.
bool screen_weight_poly(int q, bool one_element, std::vector<double>& W) {
  std::vector<double> x, w, vq(q + 1), nq(q + 1);
  gauss_legendre01(q + 2, x, w);
  node_set(q, true, nq.data());
  std::vector<double> Om((size_t)(q + 1) * (q + 1), 0.0);   // [l][i]
  auto add_piece = [&](double lo, int local, int node) {   // piece [lo, lo + 1], local basis index
    for (size_t g = 0; g < x.size(); ++g) {
      lagrange(q, nq.data(), x[g], vq.data(), nullptr);
      const double xs = lo + x[g];
      double xl = 1.0;
      for (int l = 0; l <= q; ++l, xl *= xs) Om[(size_t)l * (q + 1) + node] += w[g] * xl * vq[local];
    }
  };
  for (int i = 0; i <= q; ++i) add_piece(-0.5, i, i);
  add_piece(-1.5, q, 0);    // node 0 is the right vertex of the left neighbour
  add_piece(0.5, 0, q);     // node q is the left vertex of the right neighbour
  const int i0 = one_element ? 1 : 0, m = one_element ? q - 1 : q + 1;
  if (m < 1) return false;
  // Gauss-Jordan inverse of the m x m block Om[l][i0 + i], l < m, partial pivoting
  std::vector<double> A((size_t)m * 2 * m, 0.0);
  for (int l = 0; l < m; ++l) {
    for (int i = 0; i < m; ++i) A[(size_t)l * 2 * m + i] = Om[(size_t)l * (q + 1) + i0 + i];
    A[(size_t)l * 2 * m + m + l] = 1.0;
  }
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (std::fabs(A[(size_t)r * 2 * m + c]) > std::fabs(A[(size_t)piv * 2 * m + c])) piv = r;
    if (std::fabs(A[(size_t)piv * 2 * m + c]) < 1e-300) return false;
    if (piv != c)
      for (int k = 0; k < 2 * m; ++k) std::swap(A[(size_t)c * 2 * m + k], A[(size_t)piv * 2 * m + k]);
    const double d = A[(size_t)c * 2 * m + c];
    for (int k = 0; k < 2 * m; ++k) A[(size_t)c * 2 * m + k] /= d;
    for (int r = 0; r < m; ++r) {
      if (r == c) continue;
      const double f = A[(size_t)r * 2 * m + c];
      if (f != 0.0)
        for (int k = 0; k < 2 * m; ++k) A[(size_t)r * 2 * m + k] -= f * A[(size_t)c * 2 * m + k];
    }
  }
  // A's right half is Om_block^-1: rows = nodes i, columns = moments l
  W.assign((size_t)(q + 1) * (q + 1), 0.0);
  for (int i = 0; i < m; ++i)
    for (int l = 0; l < m; ++l) W[(size_t)(i0 + i) * (q + 1) + l] = A[(size_t)i * 2 * m + m + l];
  return true;
}

// Generalized eigenpairs K1 v = lam M1 v of the order-p mesh on a box of n
// elements (open mesh, p n + 1 nodes, h = 1): Dirichlet data fixes the two end
// nodes, so the pencil is the interior block (p n - 1 nodes); Neumann data
// leaves every node free (p n + 1 nodes; one eigenvalue is 0, the constant).
// The boxes' fast-diagonalisation solves (Sec. "Alternate boundary
// conditions") transform with V, V^T M1 V = I, V[node * N + mode].
void box_eigen(int p, int n, bool dirichlet, std::vector<double>& lam, std::vector<double>& V) {
  const ElementPQ E(p, 1);
  const int Nall = p * n + 1, o = dirichlet ? 1 : 0, N = dirichlet ? Nall - 2 : Nall;
  std::vector<double> M((size_t)N * N, 0.0), K((size_t)N * N, 0.0);
  for (int e = 0; e < n; ++e)
    for (int i = 0; i <= p; ++i)
      for (int j = 0; j <= p; ++j) {
        const int r = p * e + i - o, c = p * e + j - o;
        if (r < 0 || c < 0 || r >= N || c >= N) continue;
        M[(size_t)r * N + c] += E.Me[i * (p + 1) + j];
        K[(size_t)r * N + c] += E.Ke[i * (p + 1) + j];
      }
  std::vector<double> l0, V0;
  generalized_eigen(N, K, M, l0, V0);
  std::vector<int> ord(N);
  for (int i = 0; i < N; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return l0[a] < l0[b]; });
  lam.resize(N);
  V.assign((size_t)N * N, 0.0);
  for (int k = 0; k < N; ++k) {
    lam[k] = l0[ord[k]];
    for (int i = 0; i < N; ++i) V[(size_t)i * N + k] = V0[(size_t)i * N + ord[k]];
  }
}

// Create-time data of the order-q path: the order-p element matrices (h = 1),
// the mixed mass against the order-q screen basis, the screen weight
// polynomials (patch or one-element screens), the node-regrouped table of the
// screen contraction and the periodic order-p eigenbasis.  False if the weight
// system is singular.
bool orderq_host(int q, int n, int n_sr, int pad, bool one_element, OrderQHost& h) {
  const int p = q + 2;
  const ElementPQ E(p, q);
  h.q = q;
  h.p = p;
  h.Me = E.Me;
  h.Ke = E.Ke;
  h.Mpq = E.Mpq;
  if (!screen_weight_poly(q, one_element, h.W)) return false;
  screen_node_table(q, n_sr, pad, 8, h.H);
  periodic_eigen_order(p, n, h.lam, h.V);
  return true;
}

}  // namespace fep3m

extern "C" {

int fep3m_box_eigenbasis(int p, int n_el, int dirichlet, double* lam, double* V) {
  if (p < 1 || p > 8 || n_el < 1 || (long long)p * n_el > 1024 || !lam || !V) return FEP3M_EINVAL;
  if (dirichlet && p * n_el < 2) return FEP3M_EINVAL;
  std::vector<double> l, v;
  fep3m::box_eigen(p, n_el, dirichlet != 0, l, v);
  std::memcpy(lam, l.data(), l.size() * sizeof(double));
  std::memcpy(V, v.data(), v.size() * sizeof(double));
  return FEP3M_OK;
}

int fep3m_screen_weight_poly(int q, int one_element, double* W) {
  if (q < 1 || q > 4 || !W || (one_element && q < 2)) return FEP3M_EINVAL;
  std::vector<double> out;
  if (!fep3m::screen_weight_poly(q, one_element != 0, out)) return FEP3M_EINVAL;
  std::memcpy(W, out.data(), out.size() * sizeof(double));
  return FEP3M_OK;
}

int fep3m_mesh_eigenbasis_order(int p, int n_el, double* lam, double* V) {
  if (p < 1 || p > 8 || n_el < 1 || (long long)p * n_el > 8192 || !lam || !V) return FEP3M_EINVAL;
  std::vector<double> l, v;
  fep3m::periodic_eigen_order(p, n_el, l, v);
  std::memcpy(lam, l.data(), l.size() * sizeof(double));
  std::memcpy(V, v.data(), v.size() * sizeof(double));
  return FEP3M_OK;
}

int fep3m_screen_node_table(int q, int n_sr, int pad, double* H) {
  if (q < 1 || q > 4 || n_sr < 1 || n_sr > 4 || pad < 1 || pad > 8 || !H) return FEP3M_EINVAL;
  std::vector<double> out;
  fep3m::screen_node_table(q, n_sr, pad, 8, out);
  std::memcpy(H, out.data(), out.size() * sizeof(double));
  return FEP3M_OK;
}

int fep3m_screen_type_table(int q, int tx, int ty, int tz, int n_sr, int pad, double* kept) {
  if (q < 1 || q > 4 || n_sr < 1 || n_sr > 4 || pad < 1 || pad > 8 || !kept) return FEP3M_EINVAL;
  const int t3[3] = {tx, ty, tz};
  for (int a = 0; a < 3; ++a)
    if (t3[a] < 0 || t3[a] >= q) return FEP3M_EINVAL;
  std::vector<double> out;
  fep3m::screen_type_table(q + 2, q, t3, n_sr + 1, pad, 8, out);
  std::memcpy(kept, out.data(), out.size() * sizeof(double));
  return FEP3M_OK;
}

}  // extern "C"
