// Create-time host computations: 1-D order-3 element matrices, a symmetric
// generalised eigensolver (Cholesky + cyclic Jacobi), the FE basis-screen
// table (Remark of Sec. 4) and the multigrid smoother bound.  Nothing here
// runs per evaluation.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <map>
#include <mutex>
#include <utility>
#include <random>
#include <vector>

#include "common.cuh"

namespace fep3m {

cudaError_t smem_limit(const void* kern, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> set;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = set[{dev, kern}];
  if (have >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) have = bytes;
  return e;
}

// n-point Gauss-Legendre rule on [0, 1] by Newton iteration on P_n.
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      // p1 = P_n(z), p0 = P_{n-1}(z) (n >= 2)
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);   // 2/((1-z^2) P'^2) mapped by 1/2
  }
}

void element_matrices_q3(double Me[4][4], double Ke[4][4], double Mpq[4][2]) {
  std::vector<double> x, w;
  gauss_legendre01(6, x, w);
  for (int i = 0; i < 4; ++i) {
    for (int j = 0; j < 4; ++j) Me[i][j] = Ke[i][j] = 0.0;
    Mpq[i][0] = Mpq[i][1] = 0.0;
  }
  for (size_t g = 0; g < x.size(); ++g) {
    double v[4], d[4];
    q3_values<double>(x[g], v);
    q3_derivs<double>(x[g], d);
    double lin[2] = {1.0 - x[g], x[g]};
    for (int i = 0; i < 4; ++i) {
      for (int j = 0; j < 4; ++j) {
        Me[i][j] += w[g] * v[i] * v[j];
        Ke[i][j] += w[g] * d[i] * d[j];
      }
      Mpq[i][0] += w[g] * v[i] * lin[0];
      Mpq[i][1] += w[g] * v[i] * lin[1];
    }
  }
}

void make_stencils(Stencils& st) {
  double Me[4][4], Ke[4][4], Mpq[4][2];
  element_matrices_q3(Me, Ke, Mpq);
  const double (*E[2])[4] = {Me, Ke};
  for (int which = 0; which < 2; ++which) {
    double (*S)[7] = which == 0 ? st.M : st.K;
    const double (*A)[4] = E[which];
    for (int t = 0; t < 3; ++t)
      for (int j = 0; j < 7; ++j) S[t][j] = 0.0;
    // vertex node: local 3 of the left element, local 0 of the right element
    S[0][0] = A[3][0];
    S[0][1] = A[3][1];
    S[0][2] = A[3][2];
    S[0][3] = A[3][3] + A[0][0];
    S[0][4] = A[0][1];
    S[0][5] = A[0][2];
    S[0][6] = A[0][3];
    for (int t = 1; t <= 2; ++t)
      for (int k = 0; k < 4; ++k) S[t][3 - t + k] = A[t][k];
  }
  for (int t = 0; t < 3; ++t) {
    st.diagM[t] = st.M[t][3];
    st.diagK[t] = st.K[t][3];
  }
  for (int s = 0; s < 6; ++s) q3_values<double>(s / 6.0, st.P[s]);
  for (int k = 0; k < 4; ++k) {
    st.Mpq[k][0] = Mpq[k][0];
    st.Mpq[k][1] = Mpq[k][1];
  }
}

// Symmetric eigen-decomposition by cyclic Jacobi rotations: A (n x n, row
// major, destroyed) -> eigenvalues d, eigenvectors V (column k = vector k).
static void jacobi_sym(int n, std::vector<double>& A, std::vector<double>& d, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
  double scale = 0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) scale += a(i, j) * a(i, j);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += a(p, q) * a(p, q);
    if (off <= 1e-34 * scale) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double apq = a(p, q);
        if (std::fabs(apq) < 1e-300) continue;
        double theta = (a(q, q) - a(p, p)) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          double akp = a(k, p), akq = a(k, q);
          a(k, p) = c * akp - s * akq;
          a(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = a(p, k), aqk = a(q, k);
          a(p, k) = c * apk - s * aqk;
          a(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  d.resize(n);
  for (int i = 0; i < n; ++i) d[i] = a(i, i);
}

// A v = lam B v with B SPD: returns lam and V (row i, column k) with
// V^T B V = I and V^T A V = diag(lam).
void generalized_eigen(int n, const std::vector<double>& A, const std::vector<double>& B,
                       std::vector<double>& lam, std::vector<double>& V) {
  std::vector<double> Lc((size_t)n * n, 0.0);   // Cholesky factor, lower
  for (int j = 0; j < n; ++j) {
    double s = B[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= Lc[(size_t)j * n + k] * Lc[(size_t)j * n + k];
    Lc[(size_t)j * n + j] = std::sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      double t = B[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= Lc[(size_t)i * n + k] * Lc[(size_t)j * n + k];
      Lc[(size_t)i * n + j] = t / Lc[(size_t)j * n + j];
    }
  }
  // Cm = L^-1 A L^-T: first Y = L^-1 A (forward substitution on columns), then Cm = L^-1 Y^T
  std::vector<double> Y((size_t)n * n), Cm((size_t)n * n);
  auto fwd = [&](const std::vector<double>& R, std::vector<double>& out) {
    for (int col = 0; col < n; ++col)
      for (int i = 0; i < n; ++i) {
        double t = R[(size_t)i * n + col];
        for (int k = 0; k < i; ++k) t -= Lc[(size_t)i * n + k] * out[(size_t)k * n + col];
        out[(size_t)i * n + col] = t / Lc[(size_t)i * n + i];
      }
  };
  fwd(A, Y);
  std::vector<double> Yt((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Yt[(size_t)i * n + j] = Y[(size_t)j * n + i];
  fwd(Yt, Cm);
  for (int i = 0; i < n; ++i)   // symmetrise rounding
    for (int j = i + 1; j < n; ++j) {
      double m = 0.5 * (Cm[(size_t)i * n + j] + Cm[(size_t)j * n + i]);
      Cm[(size_t)i * n + j] = Cm[(size_t)j * n + i] = m;
    }
  std::vector<double> Qv;
  jacobi_sym(n, Cm, lam, Qv);
  // V = L^-T Q (back substitution)
  V.assign((size_t)n * n, 0.0);
  for (int col = 0; col < n; ++col)
    for (int i = n - 1; i >= 0; --i) {
      double t = Qv[(size_t)i * n + col];
      for (int k = i + 1; k < n; ++k) t -= Lc[(size_t)k * n + i] * V[(size_t)k * n + col];
      V[(size_t)i * n + col] = t / Lc[(size_t)i * n + i];
    }
}

// Generalized eigenpairs K1 v = lam M1 v of the periodic 1-D order-3 matrices
// on n elements (N = 3 n nodes), V M1-orthonormal (V^T M1 V = I), V[g][mode].
// Both matrices are block circulant (3 x 3 blocks B_d, d = -1, 0, 1, one per
// element), so the span of {cos(theta e) w, sin(theta e) w : w in R^3},
// theta = 2 pi k / n, is invariant under both: per wavenumber k the problem
// reduces to a 6 x 6 one (3 x 3 for k = 0 and k = n / 2) in the coefficients
// (c, s) of u_e = c cos(theta e) + s sin(theta e), with the matrices
//   (n / 2) [[Sc, Ss], [-Ss, Sc]],  Sc = sum_d B_d cos(theta d),
//   Ss = sum_d B_d sin(theta d)  (Sc symmetric, Ss antisymmetric),
// and (n) Sc for the real modes.  O(N^2) work in all, against O(N^3) for a
// dense eigensolver of the N x N pencil.
void periodic_eigen(int n, const Stencils& st, std::vector<double>& lam, std::vector<double>& V) {
  const int N = 3 * n;
  double BK[3][3][3] = {}, BM[3][3][3] = {};   // [d + 1][tau][tau']
  for (int tau = 0; tau < 3; ++tau)
    for (int j = -3; j <= 3; ++j) {
      const int t = tau + j;
      const int d = t < 0 ? -1 : (t >= 3 ? 1 : 0);
      const int tp = t - 3 * d;
      BK[d + 1][tau][tp] += st.K[tau][j + 3];
      BM[d + 1][tau][tp] += st.M[tau][j + 3];
    }
  lam.clear();
  V.assign((size_t)N * N, 0.0);
  int mode = 0;
  for (int k = 0; 2 * k <= n; ++k) {
    const double th = 2.0 * M_PI * k / n;
    const bool real = k == 0 || 2 * k == n;
    const int m = real ? 3 : 6;
    std::vector<double> A((size_t)m * m, 0.0), B((size_t)m * m, 0.0);
    double Kc[3][3] = {}, Ks[3][3] = {}, Mc[3][3] = {}, Ms[3][3] = {};
    for (int d = -1; d <= 1; ++d)
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          Kc[a][b] += BK[d + 1][a][b] * std::cos(th * d);
          Ks[a][b] += BK[d + 1][a][b] * std::sin(th * d);
          Mc[a][b] += BM[d + 1][a][b] * std::cos(th * d);
          Ms[a][b] += BM[d + 1][a][b] * std::sin(th * d);
        }
    const double w = real ? (double)n : 0.5 * n;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        A[(size_t)a * m + b] = w * Kc[a][b];
        B[(size_t)a * m + b] = w * Mc[a][b];
        if (!real) {
          A[(size_t)a * m + 3 + b] = w * Ks[a][b];
          A[(size_t)(3 + a) * m + b] = -w * Ks[a][b];
          A[(size_t)(3 + a) * m + 3 + b] = w * Kc[a][b];
          B[(size_t)a * m + 3 + b] = w * Ms[a][b];
          B[(size_t)(3 + a) * m + b] = -w * Ms[a][b];
          B[(size_t)(3 + a) * m + 3 + b] = w * Mc[a][b];
        }
      }
    std::vector<double> l6, v6;
    generalized_eigen(m, A, B, l6, v6);
    for (int q = 0; q < m; ++q, ++mode) {
      lam.push_back(l6[q]);
      for (int e = 0; e < n; ++e) {
        const double ce = std::cos(th * e), se = std::sin(th * e);
        for (int tau = 0; tau < 3; ++tau) {
          double v = v6[(size_t)tau * m + q] * ce;
          if (!real) v += v6[(size_t)(3 + tau) * m + q] * se;
          V[(size_t)(3 * e + tau) * N + mode] = v;
        }
      }
    }
  }
}

namespace {

// y = A x along one axis of an N^3 array (index ix + N iy + N^2 iz), A dense N x N.
void dense_axis(int N, const std::vector<double>& A, const std::vector<double>& x, std::vector<double>& y,
                int axis, bool transpose) {
  y.assign(x.size(), 0.0);
  const size_t s[3] = {1, (size_t)N, (size_t)N * N};
  const size_t sa = s[axis], so1 = s[(axis + 1) % 3], so2 = s[(axis + 2) % 3];
  for (int j1 = 0; j1 < N; ++j1)
    for (int j2 = 0; j2 < N; ++j2) {
      const size_t base = j1 * so1 + j2 * so2;
      for (int i = 0; i < N; ++i) {
        double acc = 0;
        for (int k = 0; k < N; ++k) {
          double aik = transpose ? A[(size_t)k * N + i] : A[(size_t)i * N + k];
          acc += aik * x[base + k * sa];
        }
        y[base + i * sa] = acc;
      }
    }
}

// continuum potential of the unit vertex hat psi(xi) = prod(1 - |xi_a|) at x:
// tensor Gauss-Legendre on its 8 polynomial pieces (Eq. screenintegral)
struct HatQuad {
  std::vector<double> px, py, pz, pw;
  explicit HatQuad(int ngl) {
    std::vector<double> t, w;
    gauss_legendre01(ngl, t, w);
    std::vector<double> x1, w1;
    for (double lo : {-1.0, 0.0})
      for (int g = 0; g < ngl; ++g) {
        double x = lo + t[g];
        x1.push_back(x);
        w1.push_back(w[g] * (1.0 - std::fabs(x)));
      }
    for (size_t i = 0; i < x1.size(); ++i)
      for (size_t j = 0; j < x1.size(); ++j)
        for (size_t k = 0; k < x1.size(); ++k) {
          px.push_back(x1[i]);
          py.push_back(x1[j]);
          pz.push_back(x1[k]);
          pw.push_back(w1[i] * w1[j] * w1[k]);
        }
  }
  double operator()(double x, double y, double z) const {
    double acc = 0;
    for (size_t g = 0; g < pw.size(); ++g) {
      double dx = x - px[g], dy = y - py[g], dz = z - pz[g];
      acc += pw[g] / std::sqrt(dx * dx + dy * dy + dz * dz);
    }
    return acc;
  }
};

}  // namespace

// FE basis-screen table for q = 1 (Remark of Sec. 4): the order-3 Galerkin
// solution H of -Lap H = 4 pi psi on the cube [-B, B]^3 (h = 1, B = n_sr + 1 + pad
// elements, centred on the hat's vertex, node-aligned with the global mesh),
// with the continuum potential of psi as Dirichlet data, solved exactly by
// fast diagonalisation of the 1-D Dirichlet pencils.  Returns the nodal
// values on [-(n_sr+1), n_sr+1]^3.
void build_table(int n_sr, int pad, std::vector<double>& kept) {
  const int keep = n_sr + 1, B = keep + pad, nb = 2 * B, N = 3 * nb + 1, Ni = N - 2;
  double Me[4][4], Ke[4][4], Mpq[4][2];
  element_matrices_q3(Me, Ke, Mpq);
  std::vector<double> M1((size_t)N * N, 0.0), K1((size_t)N * N, 0.0);
  for (int e = 0; e < nb; ++e)
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        M1[(size_t)(3 * e + i) * N + 3 * e + j] += Me[i][j];
        K1[(size_t)(3 * e + i) * N + 3 * e + j] += Ke[i][j];
      }
  // load: 4 pi int psi u_m = 4 pi m1_i m1_j m1_k; the hat's vertex is node 3B
  std::vector<double> m1(N, 0.0);
  for (int k = 0; k < 4; ++k) {
    m1[3 * (B - 1) + k] += Mpq[k][1];   // element left of the vertex, hat = t
    m1[3 * B + k] += Mpq[k][0];         // element right of the vertex, hat = 1 - t
  }
  const size_t NN = (size_t)N * N * N;
  std::vector<double> Hb(NN, 0.0);
  HatQuad hat(8);
  auto pos = [&](int k) { return -B + k / 3.0; };
  for (int iz = 0; iz < N; ++iz)
    for (int iy = 0; iy < N; ++iy)
      for (int ix = 0; ix < N; ++ix) {
        bool onb = ix == 0 || iy == 0 || iz == 0 || ix == N - 1 || iy == N - 1 || iz == N - 1;
        if (onb) Hb[ix + (size_t)N * (iy + (size_t)N * iz)] = hat(pos(ix), pos(iy), pos(iz));
      }
  // r = rhs - K Hb with K = K1 (x) M1 (x) M1 + M1 (x) K1 (x) M1 + M1 (x) M1 (x) K1
  std::vector<double> tA, tB, tC, acc(NN, 0.0);
  const std::vector<double>* mats[3][3] = {{&K1, &M1, &M1}, {&M1, &K1, &M1}, {&M1, &M1, &K1}};
  for (int term = 0; term < 3; ++term) {
    dense_axis(N, *mats[term][0], Hb, tA, 0, false);
    dense_axis(N, *mats[term][1], tA, tB, 1, false);
    dense_axis(N, *mats[term][2], tB, tC, 2, false);
    for (size_t i = 0; i < NN; ++i) acc[i] += tC[i];
  }
  std::vector<double> rI((size_t)Ni * Ni * Ni);
  for (int iz = 0; iz < Ni; ++iz)
    for (int iy = 0; iy < Ni; ++iy)
      for (int ix = 0; ix < Ni; ++ix) {
        size_t g = (ix + 1) + (size_t)N * ((iy + 1) + (size_t)N * (iz + 1));
        rI[ix + (size_t)Ni * (iy + (size_t)Ni * iz)] =
            4.0 * M_PI * m1[ix + 1] * m1[iy + 1] * m1[iz + 1] - acc[g];
      }
  std::vector<double> KI((size_t)Ni * Ni), MI((size_t)Ni * Ni);
  for (int i = 0; i < Ni; ++i)
    for (int j = 0; j < Ni; ++j) {
      KI[(size_t)i * Ni + j] = K1[(size_t)(i + 1) * N + j + 1];
      MI[(size_t)i * Ni + j] = M1[(size_t)(i + 1) * N + j + 1];
    }
  std::vector<double> lam, V;
  generalized_eigen(Ni, KI, MI, lam, V);
  std::vector<double> s1, s2;
  dense_axis(Ni, V, rI, s1, 0, true);
  dense_axis(Ni, V, s1, s2, 1, true);
  dense_axis(Ni, V, s2, s1, 2, true);
  for (int iz = 0; iz < Ni; ++iz)
    for (int iy = 0; iy < Ni; ++iy)
      for (int ix = 0; ix < Ni; ++ix) s1[ix + (size_t)Ni * (iy + (size_t)Ni * iz)] /= lam[ix] + lam[iy] + lam[iz];
  dense_axis(Ni, V, s1, s2, 0, false);
  dense_axis(Ni, V, s2, s1, 1, false);
  dense_axis(Ni, V, s1, s2, 2, false);
  for (int iz = 0; iz < Ni; ++iz)
    for (int iy = 0; iy < Ni; ++iy)
      for (int ix = 0; ix < Ni; ++ix)
        Hb[(ix + 1) + (size_t)N * ((iy + 1) + (size_t)N * (iz + 1))] = s2[ix + (size_t)Ni * (iy + (size_t)Ni * iz)];
  const int K = 6 * keep + 1, o = 3 * (B - keep);
  kept.assign((size_t)K * K * K, 0.0);
  for (int iz = 0; iz < K; ++iz)
    for (int iy = 0; iy < K; ++iy)
      for (int ix = 0; ix < K; ++ix)
        kept[ix + (size_t)K * (iy + (size_t)K * iz)] = Hb[(ix + o) + (size_t)N * ((iy + o) + (size_t)N * (iz + o))];
}

// Largest eigenvalue of D^-1 K (D = diag K) for the periodic reference
// order-3 operator on n^3 elements, by power iteration on D^-1/2 K D^-1/2.
double estimate_lmax(const Stencils& st, int n) {
  const int N = 3 * n;
  const size_t NN = (size_t)N * N * N;
  std::vector<double> x(NN), y(NN), t1(NN), t2(NN), a(NN), c(NN), dis(NN);
  std::mt19937_64 rng(12345);
  std::normal_distribution<double> nd;
  for (auto& v : x) v = nd(rng);
  auto idx = [&](int i, int j, int k) { return (size_t)((i + N) % N) + (size_t)N * (((j + N) % N) + (size_t)N * ((k + N) % N)); };
  for (int k = 0; k < N; ++k)
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) {
        int a0 = i % 3, a1 = j % 3, a2 = k % 3;
        double dg = st.diagK[a0] * st.diagM[a1] * st.diagM[a2] + st.diagM[a0] * st.diagK[a1] * st.diagM[a2] +
                    st.diagM[a0] * st.diagM[a1] * st.diagK[a2];
        dis[idx(i, j, k)] = 1.0 / std::sqrt(dg);
      }
  double lam = 0;
  for (int it = 0; it < 300; ++it) {
    double nrm = 0;
    for (double v : x) nrm += v * v;
    nrm = std::sqrt(nrm);
    for (size_t i = 0; i < NN; ++i) x[i] /= nrm;
    for (size_t i = 0; i < NN; ++i) y[i] = x[i] * dis[i];
    // z pass
    for (int k = 0; k < N; ++k)
      for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
          double s1 = 0, s2 = 0;
          for (int q = -3; q <= 3; ++q) {
            s1 += st.M[k % 3][q + 3] * y[idx(i, j, k + q)];
            s2 += st.K[k % 3][q + 3] * y[idx(i, j, k + q)];
          }
          t1[idx(i, j, k)] = s1;
          t2[idx(i, j, k)] = s2;
        }
    for (int k = 0; k < N; ++k)
      for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
          double s1 = 0, s2 = 0;
          for (int q = -3; q <= 3; ++q) {
            s1 += st.M[j % 3][q + 3] * t1[idx(i, j + q, k)];
            s2 += st.K[j % 3][q + 3] * t1[idx(i, j + q, k)] + st.M[j % 3][q + 3] * t2[idx(i, j + q, k)];
          }
          a[idx(i, j, k)] = s1;
          c[idx(i, j, k)] = s2;
        }
    double ray = 0;
    for (int k = 0; k < N; ++k)
      for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
          double s = 0;
          for (int q = -3; q <= 3; ++q)
            s += st.K[i % 3][q + 3] * a[idx(i + q, j, k)] + st.M[i % 3][q + 3] * c[idx(i + q, j, k)];
          size_t g = idx(i, j, k);
          y[g] = s * dis[g];
          ray += y[g] * x[g];
        }
    lam = ray;
    x.swap(y);
  }
  return lam;
}

}  // namespace fep3m
