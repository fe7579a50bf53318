// Single-pass persistent apply for affine (axis-parallel) meshes, used for FP32.
//
// One launch of one wave of blocks (blocks per SM x SMs) that loop over work items
// (right-hand side, row of `tile` consecutive cells along x). Each cell does Algorithm 1
// for its volume term as in k_cell, and handles each of its six faces from its own side
// only: its own trace comes from its Gauss-point values, the neighbour's trace is
// gathered from the neighbour's GLL coefficients (the face layer of nodes for u, the
// end row of the GLL derivative matrix along the normal lines for the normal
// derivative) and interpolated tangentially to the face Gauss points (facet sum
// factorisation, Sec. 2.2). Each face's flux is thus evaluated twice, once per side,
// in exchange for no scratch memory at all: the apply reads x (neighbours through L2)
// and writes y once, which is what FP32, with its ~60x higher ALU throughput than FP64,
// needs. The whole tile stays in shared memory between the steps.
#include "dg_scalar_kernels.cuh"

namespace dgf {

using dgk::align16;

template <int P, typename T>
struct FTab {
  T interp[P * P];  // M = P: [q][j]
  T dcol[P * P];
  T e0[P], e1[P], d0[P], d1[P], w[P];
  T gd0[P], gd1[P];
};

template <int P, typename T>
constexpr size_t fused_smem(int tile) {
  constexpr int P2 = P * P, P3 = P * P * P;
  return align16<T>(sizeof(FTab<P, T>)) + size_t(tile) * (P3 + 7 * P3 + 36 * P2 + 12 * P2 + 12 * P2) * sizeof(T);
}

template <int P, typename T>
__global__ void __launch_bounds__(256) k_fused(const ScalarArgs<T> a, const T *__restrict__ x, T *__restrict__ y,
                                               int64_t sdof, int tile, int tiles_x, int64_t nitems) {
  constexpr int M = P, P2 = P * P, P3 = P * P * P, M2 = M * M, M3 = M * M * M;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto &tb = *reinterpret_cast<FTab<P, T> *>(smem_raw);
  T *X = reinterpret_cast<T *>(smem_raw + align16<T>(sizeof(FTab<P, T>)));
  T *T1 = X + tile * P3, *T2 = T1 + tile * M3, *U = T2 + tile * M3;
  T *F0 = U + tile * M3, *F1 = F0 + tile * M3, *F2 = F1 + tile * M3, *R = F2 + tile * M3;
  T *TRo = R + tile * M3;       // own traces [c][lf][qty][M2]
  T *FR = TRo + tile * 12 * M2;  // own face residuals [c][lf][qty][M2]
  T *NBq = FR + tile * 12 * M2;  // neighbour traces at the face Gauss points
  T *NBg = NBq + tile * 12 * M2; // neighbour face data at the GLL nodes [c][lq][P2]
  T *NB1 = NBg + tile * 12 * P2; // after the first tangential sweep [c][lq][n2][q1]
  const int tid = threadIdx.x, nt = blockDim.x;
  {
    const DevTables<T> *g = a.tab;
    for (int i = tid; i < P * P; i += nt) { tb.interp[i] = g->interp[i]; tb.dcol[i] = g->dcol[i]; }
    for (int i = tid; i < P; i += nt) {
      tb.e0[i] = g->e0[i]; tb.e1[i] = g->e1[i]; tb.d0[i] = g->d0[i]; tb.d1[i] = g->d1[i];
      tb.w[i] = g->w[i]; tb.gd0[i] = g->gd0[i]; tb.gd1[i] = g->gd1[i];
    }
  }
  __syncthreads();
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int64_t ntiles = (int64_t)tiles_x * ny * nz;
  const T sc = a.sc, ss = a.ss, half = T(0.5);
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int rhs = (int)(item / ntiles);
    const int64_t t = item - (int64_t)rhs * ntiles;
    const int tx = (int)(t % tiles_x);
    const int64_t yz = t / tiles_x;
    const int cy = (int)(yz % ny), cz = (int)(yz / ny);
    const int cx0 = tx * tile;
    const int nc = min(tile, nx - cx0);
    const int64_t c0 = cx0 + (int64_t)nx * (cy + (int64_t)ny * cz);
    const T *xr = x + rhs * sdof;
    T *yr = y + rhs * sdof;
    // ---- gather: own coefficients and the neighbours' face data at the GLL nodes
    for (int i = tid; i < nc * P3; i += nt) X[i] = xr[c0 * P3 + i];
    for (int i = tid; i < nc * 12 * P2; i += nt) {
      const int c = i / (12 * P2), r = i - c * (12 * P2);
      const int lq = r / P2, nd = r - lq * P2;
      const int lf = lq >> 1, qty = lq & 1, ax = lf >> 1, side = lf & 1;
      int cc[3] = {cx0 + c, cy, cz};
      const int nlim = ax == 0 ? nx : (ax == 1 ? ny : nz);
      cc[ax] += side ? 1 : -1;
      T v = T(0);
      if (cc[ax] >= 0 && cc[ax] < nlim) {
        const int64_t nb = cc[0] + (int64_t)nx * (cc[1] + (int64_t)ny * cc[2]);
        const int n1 = nd % P, n2 = nd / P;
        // DOF of the neighbour at layer j along ax and tangential node (n1, n2)
        int base, stride;
        if (ax == 0) { base = P * (n1 + P * n2); stride = 1; }
        else if (ax == 1) { base = n1 + P2 * n2; stride = P; }
        else { base = n1 + P * n2; stride = P2; }
        const T *src = xr + nb * P3 + base;
        if (qty == 0) {
          v = src[(side ? 0 : P - 1) * stride];  // the neighbour's face layer (GLL node at the face)
        } else {
          const T *row = side ? tb.gd0 : tb.gd1;
          v = row[0] * src[0];
#pragma unroll
          for (int j = 1; j < P; ++j) v = fma(row[j], src[j * stride], v);
        }
      }
      NBg[i] = v;
    }
    __syncthreads();
    // ---- own axis 0 / neighbour tangential sweep along t1
    for (int i = tid; i < nc * P2 * M; i += nt) {
      const int c = i / (P2 * M), r = i - c * (P2 * M);
      const int q0 = r % M, j12 = r / M;
      const T *src = X + c * P3 + j12 * P;
      T acc = tb.interp[q0 * P] * src[0];
#pragma unroll
      for (int j = 1; j < P; ++j) acc = fma(tb.interp[q0 * P + j], src[j], acc);
      T1[c * M3 + r] = acc;
    }
    for (int i = tid; i < nc * 12 * P * M; i += nt) {
      const int c = i / (12 * P * M), r = i - c * (12 * P * M);
      const int lq = r / (P * M), rr = r - lq * (P * M);
      const int q1 = rr % M, n2 = rr / M;
      const T *src = NBg + (c * 12 + lq) * P2 + n2 * P;
      T acc = tb.interp[q1 * P] * src[0];
#pragma unroll
      for (int j = 1; j < P; ++j) acc = fma(tb.interp[q1 * P + j], src[j], acc);
      NB1[(c * 12 + lq) * P * M + rr] = acc;
    }
    __syncthreads();
    // ---- own axis 1 / neighbour tangential sweep along t2
    for (int i = tid; i < nc * P * M2; i += nt) {
      const int c = i / (P * M2), r = i - c * (P * M2);
      const int q0 = r % M, q1 = (r / M) % M, j2 = r / M2;
      const T *src = T1 + c * M3 + j2 * (P * M) + q0;
      T acc = tb.interp[q1 * P] * src[0];
#pragma unroll
      for (int j = 1; j < P; ++j) acc = fma(tb.interp[q1 * P + j], src[j * M], acc);
      T2[c * M3 + r] = acc;
    }
    for (int i = tid; i < nc * 12 * M2; i += nt) {
      const int c = i / (12 * M2), r = i - c * (12 * M2);
      const int lq = r / M2, qf = r - lq * M2;
      const int q1 = qf % M, q2 = qf / M;
      const T *src = NB1 + (c * 12 + lq) * P * M + q1;
      T acc = tb.interp[q2 * P] * src[0];
#pragma unroll
      for (int j = 1; j < P; ++j) acc = fma(tb.interp[q2 * P + j], src[j * M], acc);
      NBq[i] = acc;
    }
    __syncthreads();
    // ---- own axis 2 -> U
    for (int i = tid; i < nc * M3; i += nt) {
      const int c = i / M3, r = i - c * M3;
      const int q01 = r % M2, q2 = r / M2;
      const T *src = T2 + c * M3 + q01;
      T acc = tb.interp[q2 * P] * src[0];
#pragma unroll
      for (int j = 1; j < P; ++j) acc = fma(tb.interp[q2 * P + j], src[j * M2], acc);
      U[i] = acc;
    }
    __syncthreads();
    // ---- own traces; gradient and pointwise volume flux
    for (int i = tid; i < nc * 12 * M2; i += nt) {
      const int c = i / (12 * M2), r = i - c * (12 * M2);
      const int lq = r / M2, qf = r - lq * M2;
      const int lf = lq >> 1, qty = lq & 1, ax = lf >> 1, side = lf & 1;
      const int qs = qf % M, qt = qf / M;
      int base, stride;
      if (ax == 0) { base = M * (qs + M * qt); stride = 1; }
      else if (ax == 1) { base = qs + M2 * qt; stride = M; }
      else { base = qs + M * qt; stride = M2; }
      const T *row = side ? (qty ? tb.d1 : tb.e1) : (qty ? tb.d0 : tb.e0);
      const T *src = U + c * M3 + base;
      T acc = row[0] * src[0];
#pragma unroll
      for (int j = 1; j < M; ++j) acc = fma(row[j], src[j * stride], acc);
      TRo[i] = acc;
    }
    for (int i = tid; i < nc * M3; i += nt) {
      const int c = i / M3, q = i - c * M3;
      const int q0 = q % M, q1 = (q / M) % M, q2 = q / M2;
      const T *u = U + c * M3;
      T g0 = tb.dcol[q0 * M] * u[q1 * M + q2 * M2];
      T g1 = tb.dcol[q1 * M] * u[q0 + q2 * M2];
      T g2 = tb.dcol[q2 * M] * u[q0 + q1 * M];
#pragma unroll
      for (int k = 1; k < M; ++k) {
        g0 = fma(tb.dcol[q0 * M + k], u[k + q1 * M + q2 * M2], g0);
        g1 = fma(tb.dcol[q1 * M + k], u[q0 + k * M + q2 * M2], g1);
        g2 = fma(tb.dcol[q2 * M + k], u[q0 + q1 * M + k * M2], g2);
      }
      const T W = tb.w[q0] * tb.w[q1] * tb.w[q2];
      F0[i] = (W * a.vol_g[0]) * g0;
      F1[i] = (W * a.vol_g[1]) * g1;
      F2[i] = (W * a.vol_g[2]) * g2;
    }
    __syncthreads();
    // ---- volume residual at the Gauss points; face terms of each own face
    for (int i = tid; i < nc * M3; i += nt) {
      const int c = i / M3, q = i - c * M3;
      const int q0 = q % M, q1 = (q / M) % M, q2 = q / M2;
      T acc = ((tb.w[q0] * tb.w[q1] * tb.w[q2]) * a.vol_m) * U[i];
      const T *f0 = F0 + c * M3, *f1 = F1 + c * M3, *f2 = F2 + c * M3;
#pragma unroll
      for (int k = 0; k < M; ++k) {
        acc = fma(tb.dcol[k * M + q0], f0[k + q1 * M + q2 * M2], acc);
        acc = fma(tb.dcol[k * M + q1], f1[q0 + k * M + q2 * M2], acc);
        acc = fma(tb.dcol[k * M + q2], f2[q0 + q1 * M + k * M2], acc);
      }
      R[i] = acc;
    }
    for (int i = tid; i < nc * 6 * M2; i += nt) {
      const int c = i / (6 * M2), r = i - c * (6 * M2);
      const int lf = r / M2, qf = r - lf * M2;
      const int ax = lf >> 1, side = lf & 1;
      const int qs = qf % M, qt = qf / M;
      const T W = tb.w[qs] * tb.w[qt];
      const T bW = W * a.face_b[ax], pw = W * a.face_pw[ax];
      const int cc = ax == 0 ? cx0 + c : (ax == 1 ? cy : cz);
      const int nlim = ax == 0 ? nx : (ax == 1 ? ny : nz);
      const bool bnd = side ? (cc + 1 >= nlim) : (cc == 0);
      const T uo = TRo[(c * 12 + 2 * lf) * M2 + qf], dno = TRo[(c * 12 + 2 * lf + 1) * M2 + qf];
      T Rv = T(0), Rn = T(0);
      if (bnd) {
        if ((a.dmask >> lf) & 1u) {
          const T b = side ? bW : -bW;
          Rv = fma(sc, b * dno, pw * uo);
          Rn = ss * uo * b;
        }
      } else {
        const T un = NBq[(c * 12 + 2 * lf) * M2 + qf], dnn = NBq[(c * 12 + 2 * lf + 1) * M2 + qf];
        const T J = side ? uo - un : un - uo;  // u- - u+ with T- the lower cell along ax
        const T flux = half * bW * (dno + dnn);
        const T v = fma(sc, flux, pw * J);
        Rv = side ? v : -v;
        Rn = ss * half * J * bW;
      }
      FR[(c * 12 + 2 * lf) * M2 + qf] = Rv;
      FR[(c * 12 + 2 * lf + 1) * M2 + qf] = Rn;
    }
    __syncthreads();
    // ---- lift the face residuals onto the Gauss points
    for (int i = tid; i < nc * M3; i += nt) {
      const int c = i / M3, q = i - c * M3;
      const int qv[3] = {q % M, (q / M) % M, q / M2};
      const T *sf = FR + c * 12 * M2;
      T acc = R[i];
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        const int qa = qv[ax];
        const int qf = (ax == 0) ? qv[1] + M * qv[2] : (ax == 1 ? qv[0] + M * qv[2] : qv[0] + M * qv[1]);
        const T *lo = sf + (2 * ax) * 2 * M2, *hi = sf + (2 * ax + 1) * 2 * M2;
        acc = fma(tb.e0[qa], lo[qf], acc);
        acc = fma(tb.d0[qa], lo[M2 + qf], acc);
        acc = fma(tb.e1[qa], hi[qf], acc);
        acc = fma(tb.d1[qa], hi[M2 + qf], acc);
      }
      T1[i] = acc;
    }
    __syncthreads();
    // ---- transposed interpolation back to the GLL coefficients
    for (int i = tid; i < nc * M2 * P; i += nt) {
      const int c = i / (M2 * P), r = i - c * (M2 * P);
      const int j0 = r % P, q12 = r / P;
      const T *src = T1 + c * M3 + q12 * M;
      T acc = tb.interp[j0] * src[0];
#pragma unroll
      for (int q = 1; q < M; ++q) acc = fma(tb.interp[q * P + j0], src[q], acc);
      T2[c * M3 + r] = acc;
    }
    __syncthreads();
    for (int i = tid; i < nc * M * P2; i += nt) {
      const int c = i / (M * P2), r = i - c * (M * P2);
      const int j0 = r % P, j1 = (r / P) % P, q2 = r / P2;
      const T *src = T2 + c * M3 + q2 * (M * P) + j0;
      T acc = tb.interp[j1] * src[0];
#pragma unroll
      for (int q = 1; q < M; ++q) acc = fma(tb.interp[q * P + j1], src[q * P], acc);
      T1[c * M3 + r] = acc;
    }
    __syncthreads();
    for (int i = tid; i < nc * P3; i += nt) {
      const int c = i / P3, r = i - c * P3;
      const int j01 = r % P2, j2 = r / P2;
      const T *src = T1 + c * M3 + j01;
      T acc = tb.interp[j2] * src[0];
#pragma unroll
      for (int q = 1; q < M; ++q) acc = fma(tb.interp[q * P + j2], src[q * P2], acc);
      yr[c0 * P3 + i] = acc;
    }
    __syncthreads();
  }
}

template <int P, typename T>
cudaError_t run(const ScalarArgs<T> &a, const T *x, T *y, int nrhs, int64_t sdof, int tile, cudaStream_t s,
                const cudaEvent_t *ev, int *grid_out) {
  const size_t sm = fused_smem<P, T>(tile);
  auto k = k_fused<P, T>;
  cudaError_t e;
  if (sm > 48 * 1024 && (e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
    return e;
  const int threads = 256;
  int per_sm = 0, dev = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, sm)) != cudaSuccess) return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int tiles_x = (a.nx + tile - 1) / tile;
  const int64_t nitems = (int64_t)nrhs * tiles_x * a.ny * a.nz;
  int64_t grid = (int64_t)(per_sm > 0 ? per_sm : 1) * sms;
  if (grid > nitems) grid = nitems;
  if (grid_out) *grid_out = (int)grid;
  if (ev) cudaEventRecord(ev[0], s);
  k<<<(unsigned)grid, threads, sm, s>>>(a, x, y, sdof, tile, tiles_x, nitems);
  if (ev) {
    cudaEventRecord(ev[1], s);
    cudaEventRecord(ev[2], s);
    cudaEventRecord(ev[3], s);
  }
  return cudaGetLastError();
}

}  // namespace dgf

template <typename T>
cudaError_t launch_fused_apply(int p, const ScalarArgs<T> &a, const T *x, T *y, int nrhs, int64_t sdof, int tile,
                               cudaStream_t s, const cudaEvent_t *ev, int *grid_out) {
  switch (p) {
    case 2: return dgf::run<2, T>(a, x, y, nrhs, sdof, tile, s, ev, grid_out);
    case 3: return dgf::run<3, T>(a, x, y, nrhs, sdof, tile, s, ev, grid_out);
    case 4: return dgf::run<4, T>(a, x, y, nrhs, sdof, tile, s, ev, grid_out);
    case 5: return dgf::run<5, T>(a, x, y, nrhs, sdof, tile, s, ev, grid_out);
    case 6: return dgf::run<6, T>(a, x, y, nrhs, sdof, tile, s, ev, grid_out);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_fused_apply<float>(int, const ScalarArgs<float> &, const float *, float *, int, int64_t,
                                               int, cudaStream_t, const cudaEvent_t *, int *);
template cudaError_t launch_fused_apply<double>(int, const ScalarArgs<double> &, const double *, double *, int,
                                                int64_t, int, cudaStream_t, const cudaEvent_t *, int *);
