// rt_gradients_noalloc: limited least-squares gradients for callers that
// cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not available or not
// allowed -- inside a host framework that owns all device memory through its
// own pool, in a real-time loop that must not allocate, or in a plug-in that
// only receives device pointers.  Such a caller cannot create an rt_ctx
// (rt_init_mesh allocates), so this entry point takes the whole mesh and state
// as caller-owned device arrays and keeps its only scratch -- the inverse
// least-squares matrix of every cell -- in a fixed static device array
// compiled into the library.
//
// The scratch array lives on every GPU that loads the library, until the
// process exits, and is shared by all calls on that device: each call
// overwrites the entries of its cells before reading them, so nothing needs
// clearing, but calls that overlap on the GPU (different streams, or host
// threads without ordering) race on it.
//
// The array's device address is looked up once per device context and
// cached; when the device's current context changes (a cudaDeviceReset tears
// the primary context down and the next runtime call creates a new one), the
// next call looks it up again.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/rt.h"

namespace {

constexpr int64_t kNoallocMaxCells = 262144;   // 6 doubles each: 12.6 MB of device memory
constexpr int kMaxDevices = 64;

// Host code must not take the address of this array directly: on the host the
// name is only a stand-in.  The device address comes from cudaGetSymbolAddress.
__device__ __align__(256) double g_noalloc_minv[6 * kNoallocMaxCells];

std::mutex g_mu;
double* g_minv_ptr[kMaxDevices] = {};
void* g_minv_ctx[kMaxDevices] = {};   // the context each cached address belongs to

// cuCtxGetCurrent through the runtime's driver entry point (the library does
// not link the driver library itself).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return (CtxGetCurrentFn)p;
  }();
  return fn;
}

// Kernel launch that returns this launch's own status (a triple-chevron
// launch only leaves it in the thread's last-error slot, where an error the
// caller left pending is indistinguishable from it).
template <class T> struct ident { using type = T; };
template <class... KA>
cudaError_t launch(void (*k)(KA...), dim3 grid, dim3 block, cudaStream_t s, typename ident<KA>::type... args) {
  void* p[] = {(void*)&args...};
  return cudaLaunchKernel((const void*)k, grid, block, p, 0, s);
}

thread_local char g_err[256];

rt_status set_err(rt_status st, const char* msg) {
  snprintf(g_err, sizeof g_err, "%s", msg);
  return st;
}

__device__ __forceinline__ double mimg(double d, double L) {
  return L > 0.0 ? __dsub_rn(d, __dmul_rn(L, round(__ddiv_rn(d, L)))) : d;
}

// Inverse of M_i = sum over the cell's faces of A n n^T (n: unit vector to the
// neighbour's centroid), into the static scratch.
__global__ void k_noalloc_minv(int C, double box, const int32_t* __restrict__ off, const int32_t* __restrict__ csr,
                               const int32_t* __restrict__ left, const int32_t* __restrict__ right,
                               const double* __restrict__ cx, const double* __restrict__ cy,
                               const double* __restrict__ cz, const double* __restrict__ area, double* minv,
                               int* bad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C) return;
  double m00 = 0, m01 = 0, m02 = 0, m11 = 0, m12 = 0, m22 = 0;
  for (int k = off[i]; k < off[i + 1]; ++k) {
    int e = csr[k], f = e >> 1;
    int j = (e & 1) ? left[f] : right[f];
    double d0 = mimg(cx[j] - cx[i], box), d1 = mimg(cy[j] - cy[i], box), d2 = mimg(cz[j] - cz[i], box);
    double dl = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    double n0 = d0 / dl, n1 = d1 / dl, n2 = d2 / dl;
    double A = area[f];
    m00 += A * n0 * n0; m01 += A * n0 * n1; m02 += A * n0 * n2;
    m11 += A * n1 * n1; m12 += A * n1 * n2; m22 += A * n2 * n2;
  }
  double c00 = m11 * m22 - m12 * m12, c01 = m12 * m02 - m01 * m22, c02 = m01 * m12 - m11 * m02;
  double det = m00 * c00 + m01 * c01 + m02 * c02;
  double* o = minv + 6 * (size_t)i;
  if (!(det != 0.0) || !isfinite(det)) {
    atomicExch(bad, 1);
    for (int q = 0; q < 6; ++q) o[q] = 0.0;
    return;
  }
  o[0] = c00 / det;
  o[1] = c01 / det;
  o[2] = c02 / det;
  o[3] = (m00 * m22 - m02 * m02) / det;
  o[4] = (m02 * m01 - m00 * m12) / det;
  o[5] = (m00 * m11 - m01 * m01) / det;
}

__device__ __forceinline__ double comp_of(const double* N, const double* Fr, int C, int b, int q, int i) {
  return q == 0 ? N[(size_t)b * C + i] : Fr[(size_t)(3 * b + q - 1) * C + i];
}

// Variant of the gradient kernel: the same least-squares sum and slope
// limiter, with the face weights and face-centre offsets formed on the fly
// from the caller's geometry and M^-1 read from the static scratch.
__global__ void k_noalloc_grad(int C, int B, double box, int limiter, double lim_eps2,
                               const int32_t* __restrict__ off, const int32_t* __restrict__ csr,
                               const int32_t* __restrict__ left, const int32_t* __restrict__ right,
                               const double* __restrict__ cx, const double* __restrict__ cy,
                               const double* __restrict__ cz, const double* __restrict__ area,
                               const double* __restrict__ fx, const double* __restrict__ fy,
                               const double* __restrict__ fz, const double* __restrict__ minv,
                               const double* __restrict__ N, const double* __restrict__ Fr, double* __restrict__ G) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= C * B) return;
  const int i = t / B, b = t % B;
  double pi[4], r[4][3], mx[4], mn[4];
  for (int q = 0; q < 4; ++q) {
    pi[q] = comp_of(N, Fr, C, b, q, i);
    r[q][0] = r[q][1] = r[q][2] = 0.0;
    mx[q] = mn[q] = pi[q];
  }
  for (int k = off[i]; k < off[i + 1]; ++k) {
    const int e = csr[k], f = e >> 1;
    const int L = left[f], R = right[f];
    const int j = (e & 1) ? L : R;
    double d0 = mimg(cx[R] - cx[L], box), d1 = mimg(cy[R] - cy[L], box), d2 = mimg(cz[R] - cz[L], box);
    double s = area[f] / (d0 * d0 + d1 * d1 + d2 * d2);
    double w0 = s * d0, w1 = s * d1, w2 = s * d2;
    for (int q = 0; q < 4; ++q) {
      double vj = comp_of(N, Fr, C, b, q, j);
      double dphi = (e & 1) ? (pi[q] - vj) : (vj - pi[q]);
      r[q][0] += w0 * dphi;
      r[q][1] += w1 * dphi;
      r[q][2] += w2 * dphi;
      mx[q] = vj > mx[q] ? vj : mx[q];
      mn[q] = vj < mn[q] ? vj : mn[q];
    }
  }
  const double* m = minv + 6 * (size_t)i;
  double g[4][3], gg[4], psi[4];
  for (int q = 0; q < 4; ++q) {
    g[q][0] = m[0] * r[q][0] + m[1] * r[q][1] + m[2] * r[q][2];
    g[q][1] = m[1] * r[q][0] + m[3] * r[q][1] + m[4] * r[q][2];
    g[q][2] = m[2] * r[q][0] + m[4] * r[q][1] + m[5] * r[q][2];
    gg[q] = g[q][0] * g[q][0] + g[q][1] * g[q][1] + g[q][2] * g[q][2];
    psi[q] = 1.0;
  }
  if (limiter) {
    for (int k = off[i]; k < off[i + 1]; ++k) {
      const int f = csr[k] >> 1;
      double x0 = mimg(fx[f] - cx[i], box), x1 = mimg(fy[f] - cy[i], box), x2 = mimg(fz[f] - cz[i], box);
      double xx = x0 * x0 + x1 * x1 + x2 * x2;
      for (int q = 0; q < 4; ++q) {
        double dphi = g[q][0] * x0 + g[q][1] * x1 + g[q][2] * x2;
        double lim = 1.0;
        if (dphi * dphi > lim_eps2 * gg[q] * xx) lim = dphi > 0 ? (mx[q] - pi[q]) / dphi : (mn[q] - pi[q]) / dphi;
        psi[q] = lim < psi[q] ? lim : psi[q];
      }
    }
  }
  double* Go = G + (size_t)t * 12;
  for (int q = 0; q < 4; ++q) {
    Go[3 * q + 0] = g[q][0] * psi[q];
    Go[3 * q + 1] = g[q][1] * psi[q];
    Go[3 * q + 2] = g[q][2] * psi[q];
  }
}

// Device memory of the current device `dev`, or managed memory.  Device memory
// of another GPU is refused: the kernels run on `dev` and would otherwise read
// another GPU's memory (a fault, or peer traffic where peer access is on).
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" {

rt_status rt_gradients_noalloc(const rt_cells* cells, const rt_faces* faces, const int32_t* cell_off,
                               const int32_t* cell_faces, int n_bins, int order, int limiter, double lim_eps,
                               double box, const double* N, const double* F_red, double* G, int* bad_cell,
                               void* stream) {
  if (!cells || !faces || !cell_off || !cell_faces || !N || !F_red || !G || !bad_cell)
    return set_err(RT_INVALID_ARG, "rt_gradients_noalloc: NULL argument");
  if (n_bins < 1 || n_bins > 3 || order < 1 || order > 2 || lim_eps < 0 || box < 0)
    return set_err(RT_INVALID_ARG, "rt_gradients_noalloc: bad n_bins, order, lim_eps or box");
  const int64_t C = cells->n, F = faces->n;
  if (C <= 0 || F <= 0) return set_err(RT_INVALID_ARG, "rt_gradients_noalloc: empty mesh");
  if (C > kNoallocMaxCells)
    return set_err(RT_INVALID_ARG, "rt_gradients_noalloc: more than 262144 cells (size of its static scratch)");
  if (F > (1LL << 29)) return set_err(RT_INVALID_ARG, "rt_gradients_noalloc: too many faces");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return set_err(RT_CUDA, "rt_gradients_noalloc: no current device");
  }
  const void* dev_ptrs[] = {cells->cx, cells->cy, cells->cz, faces->left, faces->right, faces->area, faces->fx,
                            faces->fy, faces->fz, cell_off, cell_faces, N, F_red, G, bad_cell};
  for (const void* p : dev_ptrs)
    if (!p || !on_device(p, dev))
      return set_err(RT_INVALID_ARG, "rt_gradients_noalloc: every array must be device memory of the current device");
  double* minv = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    CUcontext cur = nullptr;
    CtxGetCurrentFn get = ctx_get_current();
    if (get && get(&cur) != CUDA_SUCCESS) cur = nullptr;
    if (!g_minv_ptr[dev] || (cur && cur != (CUcontext)g_minv_ctx[dev])) {
      // first call on this device, or its context was replaced: look the
      // address up with this device current
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_minv);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return set_err(RT_CUDA, "rt_gradients_noalloc: cudaGetSymbolAddress failed");
      }
      g_minv_ptr[dev] = (double*)p;
      g_minv_ctx[dev] = (void*)cur;
    }
    minv = g_minv_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int Ci = (int)C;
  if (order < 2) {
    if (cudaMemsetAsync(G, 0, (size_t)C * n_bins * 12 * sizeof(double), s) != cudaSuccess ||
        cudaMemsetAsync(bad_cell, 0, sizeof(int), s) != cudaSuccess) {
      cudaGetLastError();
      return set_err(RT_CUDA, "rt_gradients_noalloc: memset failed");
    }
    return RT_OK;
  }
  if (cudaMemsetAsync(bad_cell, 0, sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return set_err(RT_CUDA, "rt_gradients_noalloc: memset failed");
  }
  const int t = 256;
  cudaError_t e = launch(k_noalloc_minv, dim3((Ci + t - 1) / t), dim3(t), s, Ci, box, cell_off, cell_faces,
                         faces->left, faces->right, cells->cx, cells->cy, cells->cz, faces->area, minv, bad_cell);
  if (e == cudaSuccess) {
    const long long n = (long long)C * n_bins;
    e = launch(k_noalloc_grad, dim3((unsigned)((n + t - 1) / t)), dim3(t), s, Ci, n_bins, box, limiter,
               lim_eps * lim_eps, cell_off, cell_faces, faces->left, faces->right, cells->cx, cells->cy, cells->cz,
               faces->area, faces->fx, faces->fy, faces->fz, (const double*)minv, N, F_red, G);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();   // the failed launch's own error
    return set_err(RT_CUDA, cudaGetErrorString(e));
  }
  return RT_OK;
}

const char* rt_noalloc_last_error(void) { return g_err; }

}  // extern "C"
