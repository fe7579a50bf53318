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

// Per-cell shared memory: T1, T2, U (values along the interpolation), then one region
// used first for the neighbours' face data (NBg, NB1) and later for R, TRo and FR, then
// NBq. Each array's per-cell stride is padded to an odd number of words so that the
// stride-(k+1) line accesses of neighbouring cells fall into different banks.
template <int P>
struct FLayout {
  static constexpr int P2 = P * P, P3 = P * P * P;
  static constexpr int pad(int n) { return n | 1; }
  static constexpr int sV = pad(P3);                              // T1, T2, U, R
  static constexpr int sTR = pad(12 * P2);                        // TRo, FR, NBq
  static constexpr int sNBg = pad(12 * P2), sNB1 = pad(12 * P2);  // M = P
  static constexpr int late = 3 * sV + 2 * sTR, early = sNBg + sNB1;  // R per direction
  static constexpr int region = late > early ? late : early;
  static constexpr int per_cell = 3 * sV + region + sTR;
};

template <int P, typename T>
constexpr size_t fused_smem(int tile) {
  return size_t(tile) * FLayout<P>::per_cell * sizeof(T);
}

// Thread layout: (k+1)^2 threads per cell; in every pass a thread owns one tensor line
// of its cell (index l = l1 + P l2 over the two directions the line does not run along),
// so the contraction along the line runs in registers and the index arithmetic is done
// once per work item. Affine cells have a diagonal G, so each direction's gradient,
// pointwise flux and transposed derivative run on lines of that direction alone.
// The reference tables are a by-value kernel parameter: in the line passes every thread
// of a warp reads the same entry, so they are served from the constant bank as FFMA
// operands instead of shared-memory loads. Entries indexed by the thread's own line
// coordinates are copied to registers once.
template <int P, typename T>
__global__ void __launch_bounds__(1024) k_fused(const ScalarArgs<T> a, const FTab<P, T> tb, const T *__restrict__ x,
                                                T *__restrict__ y, int64_t sdof, int tile, int tiles_x,
                                                int64_t nitems) {
  constexpr int M = P, L = P * P, P2 = P * P, P3 = P * P * P, M2 = M * M, M3 = M * M * M;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using LY = FLayout<P>;
  T *base = reinterpret_cast<T *>(smem_raw);
  const int tid = threadIdx.x;
  const int c = tid / L, l = tid - (tid / L) * L;
  const int l1 = l % P, l2 = l / P;
  // thread-dependent table entries
  T w1 = tb.w[0], w2 = tb.w[0], e0_1 = tb.e0[0], d0_1 = tb.d0[0], e1_1 = tb.e1[0], d1_1 = tb.d1[0];
  T e0_2 = tb.e0[0], d0_2 = tb.d0[0], e1_2 = tb.e1[0], d1_2 = tb.d1[0];
#pragma unroll
  for (int i = 1; i < P; ++i) {
    if (l1 == i) { w1 = tb.w[i]; e0_1 = tb.e0[i]; d0_1 = tb.d0[i]; e1_1 = tb.e1[i]; d1_1 = tb.d1[i]; }
    if (l2 == i) { w2 = tb.w[i]; e0_2 = tb.e0[i]; d0_2 = tb.d0[i]; e1_2 = tb.e1[i]; d1_2 = tb.d1[i]; }
  }
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int64_t ntiles = (int64_t)tiles_x * ny * nz;
  const T sc = a.sc, ss = a.ss, half = T(0.5);
  T *cellmem = base + c * LY::per_cell;
  T *t1 = cellmem, *t2 = t1 + LY::sV, *u = t2 + LY::sV;
  T *region = u + LY::sV;
  T *rr = region, *ry = rr + LY::sV, *rz = ry + LY::sV;     // after the neighbour sweeps
  T *tro = rz + LY::sV, *fr = tro + LY::sTR;
  T *nbg = region, *nb1 = region + LY::sNBg;                  // before (same memory)
  T *nbq = region + LY::region;
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int rhs = (int)(item / ntiles);
    const int64_t t = item - (int64_t)rhs * ntiles;
    const int tx = (int)(t % tiles_x);
    const int64_t yz = t / tiles_x;
    const int cy = (int)(yz % ny), cz = (int)(yz / ny);
    const int cx0 = tx * tile;
    const int nc = min(tile, nx - cx0);
    const bool act = c < nc;
    const int64_t cell = cx0 + c + (int64_t)nx * (cy + (int64_t)ny * cz);
    const T *xr = x + rhs * sdof;
    T *yr = y + rhs * sdof;
    const int cc0 = cx0 + c;
    T uz[M];  // this thread's z-line of Gauss-point values (kept from the axis-2 pass)
    if (act) {
      // own x-line (j1, j2) = (l1, l2), interpolated along x in registers
      T xl[P];
#pragma unroll
      for (int j = 0; j < P; ++j) xl[j] = xr[cell * P3 + l * P + j];
#pragma unroll
      for (int q = 0; q < M; ++q) {
        T acc = tb.interp[q * P] * xl[0];
#pragma unroll
        for (int j = 1; j < P; ++j) acc = fma(tb.interp[q * P + j], xl[j], acc);
        t1[l * M + q] = acc;
      }
      // neighbours' face data at GLL node (n1, n2) = (l1, l2) of each face
#pragma unroll
      for (int lf = 0; lf < 6; ++lf) {
        const int ax = lf >> 1, side = lf & 1;
        const int coord = ax == 0 ? cc0 : (ax == 1 ? cy : cz);
        const int nlim = ax == 0 ? nx : (ax == 1 ? ny : nz);
        const int nbc = coord + (side ? 1 : -1);
        // x-neighbours inside this row tile hand over their own traces later (no gather)
        const bool in_tile = ax == 0 && (side ? c + 1 < nc : c > 0);
        T vu = T(0), vd = T(0);
        if (!in_tile && nbc >= 0 && nbc < nlim) {
          const int64_t step = ax == 0 ? 1 : (ax == 1 ? (int64_t)nx : (int64_t)nx * ny);
          const int64_t nb = side ? cell + step : cell - step;
          int base, stride;
          if (ax == 0) { base = P * (l1 + P * l2); stride = 1; }
          else if (ax == 1) { base = l1 + P2 * l2; stride = P; }
          else { base = l1 + P * l2; stride = P2; }
          const T *src = xr + nb * P3 + base;
          const T *row = side ? tb.gd0 : tb.gd1;
          T line[P];
#pragma unroll
          for (int j = 0; j < P; ++j) line[j] = src[j * stride];
          vu = line[side ? 0 : P - 1];
          vd = row[0] * line[0];
#pragma unroll
          for (int j = 1; j < P; ++j) vd = fma(row[j], line[j], vd);
        }
        nbg[(2 * lf) * P2 + l] = vu;
        nbg[(2 * lf + 1) * P2 + l] = vd;
      }
    }
    __syncthreads();
    if (act) {
      // own axis-1 line (q0, j2) = (l1, l2)
      T in[P];
#pragma unroll
      for (int j = 0; j < P; ++j) in[j] = t1[l2 * P * M + j * M + l1];
#pragma unroll
      for (int q = 0; q < M; ++q) {
        T acc = tb.interp[q * P] * in[0];
#pragma unroll
        for (int j = 1; j < P; ++j) acc = fma(tb.interp[q * P + j], in[j], acc);
        t2[l2 * M2 + q * M + l1] = acc;
      }
      // neighbour tangential sweep along t1: lines (lq, n2); x faces with an in-tile
      // neighbour (lq 0,1: lower; 2,3: upper) are skipped
      for (int ln = l; ln < 12 * P; ln += L) {
        const int lq = ln / P, n2 = ln - (ln / P) * P;
        if ((lq < 2 && c > 0) || (lq >= 2 && lq < 4 && c + 1 < nc)) continue;
        const T *src = nbg + lq * P2 + n2 * P;
#pragma unroll
        for (int q = 0; q < M; ++q) {
          T acc = tb.interp[q * P] * src[0];
#pragma unroll
          for (int j = 1; j < P; ++j) acc = fma(tb.interp[q * P + j], src[j], acc);
          nb1[lq * P * M + n2 * M + q] = acc;
        }
      }
    }
    __syncthreads();
    if (act) {
      // own axis-2 line (q0, q1) = (l1, l2) -> U, kept in registers
      T in[P];
#pragma unroll
      for (int j = 0; j < P; ++j) in[j] = t2[j * M2 + l2 * M + l1];
#pragma unroll
      for (int q = 0; q < M; ++q) {
        T acc = tb.interp[q * P] * in[0];
#pragma unroll
        for (int j = 1; j < P; ++j) acc = fma(tb.interp[q * P + j], in[j], acc);
        uz[q] = acc;
        u[q * M2 + l2 * M + l1] = acc;
      }
      // neighbour tangential sweep along t2: lines (lq, q1)
      for (int ln = l; ln < 12 * M; ln += L) {
        const int lq = ln / M, q1 = ln - (ln / M) * M;
        if ((lq < 2 && c > 0) || (lq >= 2 && lq < 4 && c + 1 < nc)) continue;
        const T *src = nb1 + lq * P * M + q1;
#pragma unroll
        for (int q = 0; q < M; ++q) {
          T acc = tb.interp[q * P] * src[0];
#pragma unroll
          for (int j = 1; j < P; ++j) acc = fma(tb.interp[q * P + j], src[j * M], acc);
          nbq[lq * M2 + q1 + M * q] = acc;
        }
      }
    }
    __syncthreads();
    // direction passes: line values v, gradient g, flux f, transposed derivative, traces
    // of the two faces normal to the direction (face point = the line's (l1, l2))
    auto pass = [&](const T *v, T coefd, T massc, T *acc_out, int lf0, bool first, bool mass) {
      T g[M];
#pragma unroll
      for (int q = 0; q < M; ++q) {
        T s = tb.dcol[q * M] * v[0];
#pragma unroll
        for (int r = 1; r < M; ++r) s = fma(tb.dcol[q * M + r], v[r], s);
        g[q] = s;
      }
      T f[M];
#pragma unroll
      for (int q = 0; q < M; ++q) f[q] = (coefd * tb.w[q]) * g[q];
#pragma unroll
      for (int q = 0; q < M; ++q) {
        T s = first ? T(0) : acc_out[q];
        if (mass) s = fma(massc * tb.w[q], v[q], s);
#pragma unroll
        for (int r = 0; r < M; ++r) s = fma(tb.dcol[r * M + q], f[r], s);
        acc_out[q] = s;
      }
      T u0 = tb.e0[0] * v[0], d0 = tb.d0[0] * v[0], u1 = tb.e1[0] * v[0], d1 = tb.d1[0] * v[0];
#pragma unroll
      for (int r = 1; r < M; ++r) {
        u0 = fma(tb.e0[r], v[r], u0); d0 = fma(tb.d0[r], v[r], d0);
        u1 = fma(tb.e1[r], v[r], u1); d1 = fma(tb.d1[r], v[r], d1);
      }
      tro[(2 * lf0) * M2 + l] = u0;
      tro[(2 * lf0 + 1) * M2 + l] = d0;
      tro[(2 * lf0 + 2) * M2 + l] = u1;
      tro[(2 * lf0 + 3) * M2 + l] = d1;
    };
    // the three passes are independent: each writes its own residual array
    if (act) {  // x-lines (q1, q2) = (l1, l2)
      T v[M], o[M];
#pragma unroll
      for (int r = 0; r < M; ++r) v[r] = u[l2 * M2 + l1 * M + r];
      pass(v, (w1 * w2) * a.vol_g[0], T(0), o, 0, true, false);
#pragma unroll
      for (int q = 0; q < M; ++q) rr[l2 * M2 + l1 * M + q] = o[q];
      // y-lines (q0, q2) = (l1, l2)
#pragma unroll
      for (int r = 0; r < M; ++r) v[r] = u[l2 * M2 + r * M + l1];
      pass(v, (w1 * w2) * a.vol_g[1], T(0), o, 2, true, false);
#pragma unroll
      for (int q = 0; q < M; ++q) ry[l2 * M2 + q * M + l1] = o[q];
      // z-lines (q0, q1) = (l1, l2), with the mass term
      pass(uz, (w1 * w2) * a.vol_g[2], (w1 * w2) * a.vol_m, o, 4, true, true);
#pragma unroll
      for (int q = 0; q < M; ++q) rz[q * M2 + l2 * M + l1] = o[q];
    }
    __syncthreads();
    if (act) {  // own-side face terms at face point qf = l of each face
      const T W = w1 * w2;
#pragma unroll
      for (int lf = 0; lf < 6; ++lf) {
        const int ax = lf >> 1, side = lf & 1;
        const T bW = W * a.face_b[ax], pw = W * a.face_pw[ax];
        const int coord = ax == 0 ? cc0 : (ax == 1 ? cy : cz);
        const int nlim = ax == 0 ? nx : (ax == 1 ? ny : nz);
        const bool bnd = side ? (coord + 1 >= nlim) : (coord == 0);
        const T uo = tro[(2 * lf) * M2 + l], dno = tro[(2 * lf + 1) * M2 + l];
        T Rv = T(0), Rn = T(0);
        if (bnd) {
          if ((a.dmask >> lf) & 1u) {
            const T b = side ? bW : -bW;
            Rv = fma(sc, b * dno, pw * uo);
            Rn = ss * uo * b;
          }
        } else {
          T un, dnn;
          if (ax == 0 && (side ? c + 1 < nc : c > 0)) {
            // the neighbour's own trace of the shared face (its face lf ^ 1)
            const T *ntro = base + (c + (side ? 1 : -1)) * LY::per_cell + 3 * LY::sV + 3 * LY::sV;
            un = ntro[(2 * (lf ^ 1)) * M2 + l];
            dnn = ntro[(2 * (lf ^ 1) + 1) * M2 + l];
          } else {
            un = nbq[(2 * lf) * M2 + l];
            dnn = nbq[(2 * lf + 1) * M2 + l];
          }
          const T J = side ? uo - un : un - uo;
          const T flux = half * bW * (dno + dnn);
          const T v = fma(sc, flux, pw * J);
          Rv = side ? v : -v;
          Rn = ss * half * J * bW;
        }
        fr[(2 * lf) * M2 + l] = Rv;
        fr[(2 * lf + 1) * M2 + l] = Rn;
      }
    }
    __syncthreads();
    if (act) {  // lifting and transposed interpolation along x: line (q1, q2) = (l1, l2)
      const int q1 = l1, q2 = l2;
      T v[M];
#pragma unroll
      for (int q0 = 0; q0 < M; ++q0) {
        const int qq = q2 * M2 + q1 * M + q0;
        T s = rr[qq] + ry[qq] + rz[qq];
        s = fma(tb.e0[q0], fr[0 * M2 + q1 + M * q2], s);
        s = fma(tb.d0[q0], fr[1 * M2 + q1 + M * q2], s);
        s = fma(tb.e1[q0], fr[2 * M2 + q1 + M * q2], s);
        s = fma(tb.d1[q0], fr[3 * M2 + q1 + M * q2], s);
        s = fma(e0_1, fr[4 * M2 + q0 + M * q2], s);
        s = fma(d0_1, fr[5 * M2 + q0 + M * q2], s);
        s = fma(e1_1, fr[6 * M2 + q0 + M * q2], s);
        s = fma(d1_1, fr[7 * M2 + q0 + M * q2], s);
        s = fma(e0_2, fr[8 * M2 + q0 + M * q1], s);
        s = fma(d0_2, fr[9 * M2 + q0 + M * q1], s);
        s = fma(e1_2, fr[10 * M2 + q0 + M * q1], s);
        s = fma(d1_2, fr[11 * M2 + q0 + M * q1], s);
        v[q0] = s;
      }
#pragma unroll
      for (int j = 0; j < P; ++j) {
        T acc = tb.interp[j] * v[0];
#pragma unroll
        for (int q = 1; q < M; ++q) acc = fma(tb.interp[q * P + j], v[q], acc);
        t1[q2 * M * P + q1 * P + j] = acc;
      }
    }
    __syncthreads();
    if (act) {  // along y: line (j0, q2) = (l1, l2)
      T in[M];
#pragma unroll
      for (int q = 0; q < M; ++q) in[q] = t1[l2 * M * P + q * P + l1];
#pragma unroll
      for (int j = 0; j < P; ++j) {
        T acc = tb.interp[j] * in[0];
#pragma unroll
        for (int q = 1; q < M; ++q) acc = fma(tb.interp[q * P + j], in[q], acc);
        t2[l2 * P2 + j * P + l1] = acc;
      }
    }
    __syncthreads();
    if (act) {  // along z: line (j0, j1) = (l1, l2) -> y
      T in[M];
#pragma unroll
      for (int q = 0; q < M; ++q) in[q] = t2[q * P2 + l2 * P + l1];
#pragma unroll
      for (int j = 0; j < P; ++j) {
        T acc = tb.interp[j] * in[0];
#pragma unroll
        for (int q = 1; q < M; ++q) acc = fma(tb.interp[q * P + j], in[q], acc);
        yr[cell * P3 + j * P2 + l2 * P + l1] = acc;
      }
    }
    __syncthreads();
  }
}

template <int P, typename T>
cudaError_t run(const ScalarArgs<T> &a, const HostTables &ht, const T *x, T *y, int nrhs, int64_t sdof, int tile,
                cudaStream_t s, const cudaEvent_t *ev, int *grid_out, LaunchInfo *q) {
  FTab<P, T> tb;
  for (int i = 0; i < P * P; ++i) { tb.interp[i] = (T)ht.interp[i]; tb.dcol[i] = (T)ht.dcol[i]; }
  for (int i = 0; i < P; ++i) {
    tb.e0[i] = (T)ht.e0[i]; tb.e1[i] = (T)ht.e1[i]; tb.d0[i] = (T)ht.d0[i]; tb.d1[i] = (T)ht.d1[i];
    tb.w[i] = (T)ht.gauss_w[i]; tb.gd0[i] = (T)ht.gd0[i]; tb.gd1[i] = (T)ht.gd1[i];
  }
  const size_t sm = fused_smem<P, T>(tile);
  auto k = k_fused<P, T>;
  cudaError_t e;
  if (sm > 48 * 1024 && (e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
    return e;
  constexpr int L = P * P;
  if (tile < 1 || tile * L > 1024) return cudaErrorInvalidValue;
  const int threads = tile * L;
  int per_sm = 0, dev = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, sm)) != cudaSuccess) return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int tiles_x = (a.nx + tile - 1) / tile;
  const int64_t nitems = (int64_t)nrhs * tiles_x * a.ny * a.nz;
  int64_t grid = (int64_t)(per_sm > 0 ? per_sm : 1) * sms;
  if (grid > nitems) grid = nitems;
  if (grid_out) *grid_out = (int)grid;
  if (q) {
    q->blocks = grid;
    q->threads = threads;
    q->blocks_per_sm = per_sm;
    q->items = nitems;
    return cudaSuccess;
  }
  if (ev) cudaEventRecord(ev[0], s);
  k<<<(unsigned)grid, threads, sm, s>>>(a, tb, x, y, sdof, tile, tiles_x, nitems);
  if (ev) {
    cudaEventRecord(ev[1], s);
    cudaEventRecord(ev[2], s);
    cudaEventRecord(ev[3], s);
  }
  return cudaGetLastError();
}

}  // namespace dgf

template <typename T>
cudaError_t launch_fused_apply(int p, const ScalarArgs<T> &a, const HostTables &ht, const T *x, T *y, int nrhs,
                               int64_t sdof, int tile, cudaStream_t s, const cudaEvent_t *ev, int *grid_out,
                               LaunchInfo *q) {
  if (ht.m != p || ht.p != p) return cudaErrorInvalidValue;
  switch (p) {
    case 2: return dgf::run<2, T>(a, ht, x, y, nrhs, sdof, tile, s, ev, grid_out, q);
    case 3: return dgf::run<3, T>(a, ht, x, y, nrhs, sdof, tile, s, ev, grid_out, q);
    case 4: return dgf::run<4, T>(a, ht, x, y, nrhs, sdof, tile, s, ev, grid_out, q);
    case 5: return dgf::run<5, T>(a, ht, x, y, nrhs, sdof, tile, s, ev, grid_out, q);
    case 6: return dgf::run<6, T>(a, ht, x, y, nrhs, sdof, tile, s, ev, grid_out, q);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_fused_apply<float>(int, const ScalarArgs<float> &, const HostTables &, const float *,
                                               float *, int, int64_t, int, cudaStream_t, const cudaEvent_t *, int *,
                                               LaunchInfo *);
template cudaError_t launch_fused_apply<double>(int, const ScalarArgs<double> &, const HostTables &, const double *,
                                                double *, int, int64_t, int, cudaStream_t, const cudaEvent_t *, int *,
                                                LaunchInfo *);
