// dg_apply_affine_static: the FP64 scalar apply on the affine unit-cube mesh for callers
// that cannot allocate device memory. The apply's scratch (reference tables, Gauss-point
// volume residual, face traces, face residuals) lives in one file-scope device array of
// fixed size instead of operator-owned cudaMalloc buffers; the kernels are the same ones
// dg_apply launches.
//
// Layout of the array: five table slots (degrees 1..5, k+1 Gauss points), filled once
// per device by the first call on that device, then the scratch of the current call:
// rvol [ncell][M^3], traces [ncell][12][M^2], face residuals [ncell][12][M^2] (doubles).
#include <mutex>
#include <string.h>

#include "dg_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB, held by every GPU that loads libdg
constexpr size_t kTableSlot = 4096;                  // one DevTables<double> per degree
constexpr int kMaxDegree = 5;
constexpr size_t kTableBytes = kTableSlot * kMaxDegree;
static_assert(sizeof(DevTables<double>) <= kTableSlot, "tables must fit their slot");

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

// Per device: the device address of g_static_scratch (looked up with that device current;
// the host-side name of the array is not a device address) and whether the table slots
// have been uploaded.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Host copy of the reference tables of degree k (k+1 Gauss points), in the device layout.
bool host_tables(int k, DevTables<double> *tab) {
  HostTables ht;
  if (dg_build_tables(k, k + 1, false, &ht)) return false;
  const int P = k + 1, M = P;
  memset(tab, 0, sizeof(*tab));
  for (int i = 0; i < M * P; ++i) tab->interp[i] = ht.interp[i];
  for (int i = 0; i < M * M; ++i) tab->dcol[i] = ht.dcol[i];
  for (int i = 0; i < M; ++i) {
    tab->e0[i] = ht.e0[i]; tab->e1[i] = ht.e1[i];
    tab->d0[i] = ht.d0[i]; tab->d1[i] = ht.d1[i];
    tab->w[i] = ht.gauss_w[i]; tab->s[i] = ht.gauss_s[i];
  }
  return true;
}

// Set-up of the current device on its first use: address lookup, then one synchronous
// upload of the five table slots. Later calls on the device only launch kernels.
dg_status scratch_address(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DG_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return DG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess) return DG_ERR_CUDA;
    static unsigned char host[kTableBytes];
    for (int k = 1; k <= kMaxDegree; ++k)
      if (!host_tables(k, reinterpret_cast<DevTables<double> *>(host + (k - 1) * kTableSlot))) return DG_ERR_UNSUPPORTED;
    if (cudaMemcpy(p, host, kTableBytes, cudaMemcpyHostToDevice) != cudaSuccess) return DG_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return DG_OK;
}

}  // namespace

extern "C" dg_status dg_apply_affine_static(int nx, int ny, int nz, int degree, double c, double theta,
                                            double penalty_alpha, int dirichlet_mask, const double *x, double *y,
                                            void *stream) {
  if (nx < 1 || ny < 1 || nz < 1 || degree < 1 || !x || !y) return DG_ERR_INVALID_ARG;
  if (dirichlet_mask < 0 || dirichlet_mask > 63) return DG_ERR_INVALID_ARG;
  if (((uintptr_t)x & 15u) || ((uintptr_t)y & 15u)) return DG_ERR_INVALID_ARG;
  if (degree > kMaxDegree) return DG_ERR_UNSUPPORTED;
  const int P = degree + 1, M = P, M2 = M * M, M3 = M * M * M;
  const int64_t ncell = (int64_t)nx * ny * nz;
  // x and y must not overlap anywhere (each spans ncell P^3 doubles)
  const uintptr_t vbytes = (uintptr_t)ncell * P * P * P * sizeof(double);
  const uintptr_t xa = (uintptr_t)x, ya = (uintptr_t)y;
  if (xa < ya + vbytes && ya < xa + vbytes) return DG_ERR_INVALID_ARG;
  const double per_cell = (double)(M3 + 24 * M2) * sizeof(double);
  if ((double)ncell * per_cell > (double)(kScratchBytes - kTableBytes)) return DG_ERR_UNSUPPORTED;

  void *base = nullptr;
  const dg_status st = scratch_address(&base);
  if (st != DG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;

  ScalarArgs<double> a;
  memset(&a, 0, sizeof(a));
  a.nx = nx; a.ny = ny; a.nz = nz;
  a.ncell = ncell;
  const int n[3] = {nx, ny, nz};
  a.face_off[0] = 0;
  for (int ax = 0; ax < 3; ++ax) {
    const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
    a.face_off[ax + 1] = a.face_off[ax] + (int64_t)(n[ax] + 1) * n[t1] * n[t2];
  }
  a.nface = a.face_off[3];
  a.tab = (const DevTables<double> *)((unsigned char *)base + (degree - 1) * kTableSlot);
  const double h[3] = {1.0 / nx, 1.0 / ny, 1.0 / nz};
  const double V = h[0] * h[1] * h[2];
  for (int d = 0; d < 3; ++d) {
    a.vol_g[d] = V / (h[d] * h[d]);
    a.face_b[d] = V / (h[d] * h[d]);
    a.face_pw[d] = penalty_alpha * degree * (degree + 1) * n[d] * V / h[d];
  }
  a.vol_m = c * V;
  a.vol = 1.0 / ((double)nx * ny * nz);
  a.c = c;
  a.dmask = (unsigned)dirichlet_mask;
  a.sc = -1.0;
  a.ss = theta;
  // every scratch entry below is written before it is read within one call, so nothing
  // carried over from an earlier call needs clearing
  double *rvol = (double *)((unsigned char *)base + kTableBytes);
  double *tr = rvol + ncell * M3;
  double *fres = tr + ncell * 12 * M2;
  const int cpb = 256 / M3 > 0 ? 256 / M3 : 1;
  const int fpb = 256 / M2 > 0 ? 256 / M2 : 1;
  cudaError_t e = launch_scalar_apply<double>(P, M, GEO_AFFINE, false, a, x, y, rvol, tr, fres, 1, ncell * P * P * P,
                                              ncell * M3, ncell * 12 * M2, cpb, fpb, s, nullptr);
  return e == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}
