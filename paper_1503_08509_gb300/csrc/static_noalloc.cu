// Allocation-free variant of the load-vector assembly.
//
// Some callers cannot call cudaMalloc: code issuing work while a stream is
// being captured into a CUDA graph (allocation calls are not allowed there),
// applications whose memory manager owns the whole device and forbids
// allocations from libraries, and loops where cudaMalloc's implicit
// synchronisation is unacceptable.  fep3m_load_vector_static serves them: its
// only scratch, the order-1 vertex density, lives in the file-scope device
// array below, which every GPU that loads this library holds until the
// process exits (FEP3M_STATIC_MAX_NEL^3 doubles = 2 MiB).
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace {

constexpr int kMaxNel = 64;   // FEP3M_STATIC_MAX_NEL
constexpr int kMaxDevices = 64;
constexpr int PT = 256;

static __device__ __align__(256) double g_static_vertex_density[kMaxNel * kMaxNel * kMaxNel];

std::mutex g_static_mutex;
double* g_static_ptr[kMaxDevices] = {};

struct MpqWeights {
  double w[4][2];
};

__device__ __forceinline__ int wrapv(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// bin each charge (the same wrap/element/offset rule as fep3m_set_particles) and
// scatter Q times its order-1 screen weights onto the 8 vertices of its element.
// Inputs are not checked for finiteness (that would need a flag read back on
// the host): a non-finite coordinate is taken as 0 and a non-finite charge
// carries into b.
__global__ void k_static_deposit(int64_t N, const double* __restrict__ pos, const double* __restrict__ Q, double L,
                                 int n, double h, double inv_h, double* __restrict__ r) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  int c3[3];
  double t[3];
  for (int a = 0; a < 3; ++a) {
    double x = pos[3 * i + a];
    if (!isfinite(x)) x = 0.0;
    const double xw0 = __dsub_rn(x, __dmul_rn(L, floor(x / L)));
    const double xw = xw0 >= L ? 0.0 : xw0;
    const int c = (int)fmax(0.0, fmin(floor(__dmul_rn(xw, inv_h)), (double)(n - 1)));
    c3[a] = c;
    t[a] = __dsub_rn(xw, __dmul_rn((double)c + 0.5, h)) * inv_h + 0.5;
  }
  const double q = Q[i];
  for (int k = 0; k < 8; ++k) {
    const int kx = k & 1, ky = (k >> 1) & 1, kz = k >> 2;
    const double w = (kx ? t[0] : 1.0 - t[0]) * (ky ? t[1] : 1.0 - t[1]) * (kz ? t[2] : 1.0 - t[2]);
    const int vx = wrapv(c3[0] + kx, n), vy = wrapv(c3[1] + ky, n), vz = wrapv(c3[2] + kz, n);
    atomicAdd(&r[vx + (int64_t)n * (vy + (int64_t)n * vz)], q * w);
  }
}

__device__ __forceinline__ int static_mpq_row(int g, int n, const MpqWeights& m, int vtx[3], double wgt[3]) {
  const int e = g / 3, t = g - 3 * e;
  if (t == 0) {
    vtx[0] = wrapv(e - 1, n); wgt[0] = m.w[3][0];
    vtx[1] = e;               wgt[1] = m.w[0][0] + m.w[3][1];
    vtx[2] = wrapv(e + 1, n); wgt[2] = m.w[0][1];
    return 3;
  }
  vtx[0] = e;               wgt[0] = m.w[t][0];
  vtx[1] = wrapv(e + 1, n); wgt[1] = m.w[t][1];
  return 2;
}

// b = 4 pi (Mpq (x) Mpq (x) Mpq) r on the order-3 nodes
__global__ void k_static_load(int n, MpqWeights m, const double* __restrict__ r, double* __restrict__ b) {
  const int N = 3 * n;
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= (int64_t)N * N * N) return;
  const int ix = (int)(g % N), iy = (int)((g / N) % N), iz = (int)(g / ((int64_t)N * N));
  int vx[3], vy[3], vz[3];
  double wx[3], wy[3], wz[3];
  const int nx = static_mpq_row(ix, n, m, vx, wx), ny = static_mpq_row(iy, n, m, vy, wy),
            nz = static_mpq_row(iz, n, m, vz, wz);
  double acc = 0.0;
  for (int c = 0; c < nz; ++c)
    for (int bb = 0; bb < ny; ++bb)
      for (int a = 0; a < nx; ++a) acc += wx[a] * wy[bb] * wz[c] * r[vx[a] + (int64_t)n * (vy[bb] + (int64_t)n * vz[c])];
  b[g] = 4.0 * M_PI * acc;
}

// device memory of the current device, or managed memory
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int fep3m_load_vector_static(double L, int n_el, int64_t N, const double* pos, const double* Q, double* b,
                                        void* cuda_stream) {
  if (!(L > 0) || !std::isfinite(L) || n_el < 1 || n_el > kMaxNel || N < 1 || N > ((int64_t)1 << 31) - 1)
    return FEP3M_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return FEP3M_ECUDA;
  }
  if (!on_device(pos, dev) || !on_device(Q, dev) || !on_device(b, dev)) return FEP3M_EINVAL;
  double* r = nullptr;
  {
    // first call on this device: look up the device address of the static array
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_static_vertex_density);
      if (e != cudaSuccess || !p) {
        (void)cudaGetLastError();
        return FEP3M_ECUDA;
      }
      g_static_ptr[dev] = (double*)p;
    }
    r = g_static_ptr[dev];
  }
  // element mixed mass int l3_k (1 - t), int l3_k t by 3-point Gauss-Legendre
  // (exact: the integrands have degree 4); no host allocation either
  MpqWeights m = {};
  {
    const double gx[3] = {0.5 - 0.5 * std::sqrt(0.6), 0.5, 0.5 + 0.5 * std::sqrt(0.6)};
    const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    for (int g = 0; g < 3; ++g) {
      double v[4];
      fep3m::q3_values<double>(gx[g], v);
      for (int k = 0; k < 4; ++k) {
        m.w[k][0] += gw[g] * v[k] * (1.0 - gx[g]);
        m.w[k][1] += gw[g] * v[k] * gx[g];
      }
    }
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int64_t nv = (int64_t)n_el * n_el * n_el, nodes = 27 * nv;
  if (cudaMemsetAsync(r, 0, nv * sizeof(double), s) != cudaSuccess) {
    (void)cudaGetLastError();
    return FEP3M_ECUDA;
  }
  const double h = L / n_el, inv_h = n_el / L;
  FEP3M_CL k_static_deposit<<<(unsigned)((N + PT - 1) / PT), PT, 0, s>>>(N, pos, Q, L, n_el, h, inv_h, r);
  FEP3M_CL k_static_load<<<(unsigned)((nodes + PT - 1) / PT), PT, 0, s>>>(n_el, m, r, b);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FEP3M_OK : FEP3M_ECUDA;
}
