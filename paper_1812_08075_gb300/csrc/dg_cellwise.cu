// One-thread-per-cell persistent apply for affine (axis-parallel) meshes and low degree
// (k <= 3), used for FP32.
//
// A block owns a brick of bx x by x bz cells, one thread per cell, and loops over work
// items (right-hand side, brick) in one wave of blocks. Each thread runs the whole of
// Algorithm 1 for its cell in registers: interpolation to the Gauss points, the three
// derivative contractions with the (diagonal) affine metric, the transposed contractions
// and the transposed interpolation, every contraction fully unrolled so that the
// reference-table entries, identical across the block, are read as constant-bank operands
// of the FMAs. The face terms (Sec. 2.2) are evaluated per axis from each side: a cell
// publishes the trace (u and the reference normal derivative at the face Gauss points) of
// its two faces normal to the axis in shared memory, and reads its neighbours' traces
// there; neighbours across the brick boundary were turned into traces at the start of the
// item from their GLL coefficients (the face layer of nodes and the end row of the GLL
// derivative along the normal, then facet sum factorisation to the face Gauss points), one
// brick-boundary face per thread. The apply reads x and writes y once, both staged through
// shared memory so that the global accesses are coalesced rows of the brick.
#include <type_traits>

#include "dg_internal.h"

namespace dgc {

// Reference tables and the affine per-point weights, passed by value (constant bank).
template <int P, typename T>
struct CTab {
  T interp[P * P];        // [q][j] GLL basis j at Gauss point q
  T dcol[P * P];          // [q][r] derivative of Gauss-Lagrange basis r at Gauss point q
  T e0[P], e1[P], d0[P], d1[P];  // Gauss-Lagrange basis and derivative at xi = 0, 1
  T gd0[P], gd1[P];       // GLL basis derivative at xi = 0, 1
  T mw[P * P * P];        // c detJ w_q0 w_q1 w_q2
  T gw[3][P * P * P];     // G_dd w_q0 w_q1 w_q2 (G diagonal on axis-parallel cells)
  T hbw[3][P * P];        // half the normal-derivative weight of an axis-d face point
  T pw[3][P * P];         // penalty weight of an axis-d face point
};

// Index of the value at position r along axis D of the line (t1, t2) of a cell's
// Gauss-point array [q2][q1][q0]; t1 < t2 are the other two axes in increasing order.
template <int M, int D>
__device__ __forceinline__ constexpr int lidx(int r, int t1, int t2) {
  return D == 0 ? r + M * (t1 + M * t2) : (D == 1 ? t1 + M * (r + M * t2) : t1 + M * (t2 + M * r));
}

template <int P>
struct CLayout {
  static constexpr int P3 = P * P * P, M2 = P * P;
  static constexpr int sX = P3 | 1;            // per-cell stride of the x / y staging (odd)
  static constexpr int NT = 4 * M2;            // trace words per cell and axis
  static constexpr int buf = NT > sX ? NT : sX;
};

// Shared memory words: two trace buffers (the second one doubles as x/y staging) and the
// brick-boundary traces of the three axes.
template <int P>
inline size_t cellwise_words(int bx, int by, int bz) {
  using LY = CLayout<P>;
  const size_t nb = (size_t)bx * by * bz;
  return 2 * LY::buf * nb + (size_t)LY::NT * (by * bz + bx * bz + bx * by);
}

// Trace of a neighbour cell's face normal to axis D from its GLL coefficients `src`:
// SIDE 1 is the neighbour's lower face (xi_D = 0), SIDE 0 its upper face. Values go to
// dst[pt * nd], normal derivatives to dst[(M2 + pt) * nd].
template <int P, typename T, int D, int SIDE>
__device__ __forceinline__ void halo_trace(const T *__restrict__ src, const CTab<P, T> &tb, T *dst, int nd) {
  constexpr int M = P, P2 = P * P, M2 = M * M;
  constexpr int stn = D == 0 ? 1 : (D == 1 ? P : P2);
  constexpr int st1 = D == 0 ? P : 1;
  constexpr int st2 = D == 2 ? P : P2;
  T v[P2], dv[P2];
#pragma unroll
  for (int n2 = 0; n2 < P; ++n2)
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) {
      T line[P];
#pragma unroll
      for (int j = 0; j < P; ++j) line[j] = __ldg(src + n1 * st1 + n2 * st2 + j * stn);
      v[n1 + P * n2] = SIDE ? line[0] : line[P - 1];
      T s = (SIDE ? tb.gd0[0] : tb.gd1[0]) * line[0];
#pragma unroll
      for (int j = 1; j < P; ++j) s = fma(SIDE ? tb.gd0[j] : tb.gd1[j], line[j], s);
      dv[n1 + P * n2] = s;
    }
  T tv[M * P], tdv[M * P];  // after the sweep along t1: [n2][q1]
#pragma unroll
  for (int n2 = 0; n2 < P; ++n2)
#pragma unroll
    for (int q1 = 0; q1 < M; ++q1) {
      T a = tb.interp[q1 * P] * v[P * n2], b = tb.interp[q1 * P] * dv[P * n2];
#pragma unroll
      for (int n1 = 1; n1 < P; ++n1) {
        a = fma(tb.interp[q1 * P + n1], v[n1 + P * n2], a);
        b = fma(tb.interp[q1 * P + n1], dv[n1 + P * n2], b);
      }
      tv[q1 + M * n2] = a;
      tdv[q1 + M * n2] = b;
    }
#pragma unroll
  for (int q2 = 0; q2 < M; ++q2)
#pragma unroll
    for (int q1 = 0; q1 < M; ++q1) {
      T a = tb.interp[q2 * P] * tv[q1], b = tb.interp[q2 * P] * tdv[q1];
#pragma unroll
      for (int n2 = 1; n2 < P; ++n2) {
        a = fma(tb.interp[q2 * P + n2], tv[q1 + M * n2], a);
        b = fma(tb.interp[q2 * P + n2], tdv[q1 + M * n2], b);
      }
      dst[(q1 + M * q2) * nd] = a;
      dst[(M2 + q1 + M * q2) * nd] = b;
    }
}

// The brick is 8 x 4 x BZ cells (a warp spans 8 x 4 cells); its shape is a template
// parameter so that every shared-memory slot is an immediate offset from one address.
// Resident blocks the compiler must allow for (measured at 128^3 x 16 right-hand sides):
// FP32 Q1 and FP32 Q2 with bricks of 256 cells are held to 128 registers (16 warps per SM;
// Q1 needs no more, Q2 spills a little and is still fastest), Q2 with bricks of 128 cells to
// 168 (12 warps); the others take what they need.
template <int P, typename T, int BZ>
constexpr int cellwise_min_blocks() {
  if (sizeof(T) == 4 && P == 2) return 512 / (32 * BZ);
  if (sizeof(T) == 4 && P == 3) return BZ == 8 ? 2 : (BZ == 4 ? 3 : 1);  // 128 / 168 / any registers
  return 1;
}

template <int P, typename T, int BZ>
__global__ void __launch_bounds__(32 * BZ, cellwise_min_blocks<P, T, BZ>()) k_cellwise(const ScalarArgs<T> a, const CTab<P, T> tb, const T *__restrict__ x,
                                                  T *__restrict__ y, int64_t sdof, int nbx, int nby, int64_t nbricks,
                                                  int64_t nitems) {
  constexpr int M = P, P2 = P * P, P3 = P2 * P, M2 = M * M, M3 = M2 * M;
  using LY = CLayout<P>;
  constexpr int sX = LY::sX;
  constexpr int bx = 8, by = 4, bz = BZ, nb = bx * by * bz;
  constexpr int n0 = by * bz, n1 = bx * bz, n2 = bx * by;  // brick-boundary planes per axis
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *buf0 = reinterpret_cast<T *>(smem_raw);
  T *buf1 = buf0 + LY::buf * nb;
  T *xs = buf1;                 // x / y staging: [cell of the brick][sX]
  T *hl = buf1 + LY::buf * nb;  // [axis][side][qty][pt][plane]
  auto hoff = [](int d) { return d == 0 ? 0 : (d == 1 ? LY::NT * n0 : LY::NT * (n0 + n1)); };
  const int tid = threadIdx.x;
  const int lx = tid % bx, ly = (tid / bx) % by, lz = tid / (bx * by);
  const int warp = tid >> 5, lane = tid & 31;
  constexpr int nwarps = nb >> 5;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const T sc = a.sc, ss = a.ss;
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int rhs = (int)(item / nbricks);
    const int64_t bi = item - (int64_t)rhs * nbricks;
    const int ibx = (int)(bi % nbx);
    const int64_t bq = bi / nbx;
    const int iby = (int)(bq % nby), ibz = (int)(bq / nby);
    const int ox = ibx * bx, oy = iby * by, oz = ibz * bz;
    const int nax = min(bx, nx - ox), nay = min(by, ny - oy), naz = min(bz, nz - oz);
    const T *xr = x + rhs * sdof;
    T *yr = y + rhs * sdof;
    const int gx = ox + lx, gy = oy + ly, gz = oz + lz;
    const bool act = lx < nax && ly < nay && lz < naz;
    // stage x: each warp copies whole rows of the brick (coalesced)
    for (int row = warp; row < by * bz; row += nwarps) {
      const int ry = row % by, rz = row / by;
      if (ry >= nay || rz >= naz) continue;
      const T *src = xr + (ox + (int64_t)nx * (oy + ry + (int64_t)ny * (oz + rz))) * P3;
      T *dst = xs + row * bx * sX;
      if constexpr (sX == P3 && sizeof(T) == 4) {
        if ((nax * P3) % 4 == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
          // the staged row is laid out as in memory: copy it as 16-byte vectors
          const float4 *s4 = reinterpret_cast<const float4 *>(src);
          float4 *d4 = reinterpret_cast<float4 *>(dst);
          for (int j = lane; j < nax * P3 / 4; j += 32) d4[j] = __ldg(s4 + j);
          continue;
        }
      }
      for (int j = lane; j < nax * P3; j += 32) {
        const int cl = j / P3;
        dst[cl * sX + (j - cl * P3)] = __ldg(src + j);
      }
    }
    // traces of the neighbours across the brick boundary, one face per thread
    const int nh = 2 * (n0 + n1 + n2);
    for (int h = tid; h < nh; h += nb) {
      int d = 0, rem = h;
      if (rem >= 2 * n0) {
        rem -= 2 * n0;
        d = 1;
        if (rem >= 2 * n1) { rem -= 2 * n1; d = 2; }
      }
      const int nd = d == 0 ? n0 : (d == 1 ? n1 : n2);
      const int side = rem >= nd ? 1 : 0;
      const int p = rem - side * nd;
      int cx, cy, cz;  // neighbour cell
      bool ok;
      if (d == 0) {
        const int py = p % by, pz = p / by;
        cy = oy + py; cz = oz + pz; cx = side ? ox + bx : ox - 1;
        ok = py < nay && pz < naz && (side ? ox + bx < nx : ox > 0);
      } else if (d == 1) {
        const int px = p % bx, pz = p / bx;
        cx = ox + px; cz = oz + pz; cy = side ? oy + by : oy - 1;
        ok = px < nax && pz < naz && (side ? oy + by < ny : oy > 0);
      } else {
        const int px = p % bx, py = p / bx;
        cx = ox + px; cy = oy + py; cz = side ? oz + bz : oz - 1;
        ok = px < nax && py < nay && (side ? oz + bz < nz : oz > 0);
      }
      if (!ok) continue;
      const T *src = xr + (cx + (int64_t)nx * (cy + (int64_t)ny * cz)) * P3;
      T *dst = hl + hoff(d) + side * 2 * M2 * nd + p;
      if (d == 0) {
        if (side) halo_trace<P, T, 0, 1>(src, tb, dst, nd); else halo_trace<P, T, 0, 0>(src, tb, dst, nd);
      } else if (d == 1) {
        if (side) halo_trace<P, T, 1, 1>(src, tb, dst, nd); else halo_trace<P, T, 1, 0>(src, tb, dst, nd);
      } else {
        if (side) halo_trace<P, T, 2, 1>(src, tb, dst, nd); else halo_trace<P, T, 2, 0>(src, tb, dst, nd);
      }
    }
    __syncthreads();
    // own cell: Gauss-point values u and the mass term of the residual R
    T u[M3], R[M3];
    if (act) {
      T xl[P3];
#pragma unroll
      for (int i = 0; i < P3; ++i) xl[i] = xs[tid * sX + i];
      T t1[P2 * M];  // [j2][j1][q0]
#pragma unroll
      for (int jj = 0; jj < P2; ++jj)
#pragma unroll
        for (int q = 0; q < M; ++q) {
          T s = tb.interp[q * P] * xl[jj * P];
#pragma unroll
          for (int j = 1; j < P; ++j) s = fma(tb.interp[q * P + j], xl[jj * P + j], s);
          t1[jj * M + q] = s;
        }
      T t2[P * M2];  // [j2][q1][q0]
#pragma unroll
      for (int j2 = 0; j2 < P; ++j2)
#pragma unroll
        for (int q1 = 0; q1 < M; ++q1)
#pragma unroll
          for (int q0 = 0; q0 < M; ++q0) {
            T s = tb.interp[q1 * P] * t1[(j2 * P) * M + q0];
#pragma unroll
            for (int j = 1; j < P; ++j) s = fma(tb.interp[q1 * P + j], t1[(j2 * P + j) * M + q0], s);
            t2[(j2 * M + q1) * M + q0] = s;
          }
#pragma unroll
      for (int q2 = 0; q2 < M; ++q2)
#pragma unroll
        for (int qq = 0; qq < M2; ++qq) {
          T s = tb.interp[q2 * P] * t2[qq];
#pragma unroll
          for (int j = 1; j < P; ++j) s = fma(tb.interp[q2 * P + j], t2[j * M2 + qq], s);
          u[q2 * M2 + qq] = s;
        }
#pragma unroll
      for (int q = 0; q < M3; ++q) R[q] = tb.mw[q] * u[q];
    }
    // per axis: volume contraction, own traces, then the face terms of the two faces
    auto axis = [&](auto Dc, T *trb) {
      constexpr int D = decltype(Dc)::value;
      if (act) {
#pragma unroll
        for (int t2 = 0; t2 < M; ++t2)
#pragma unroll
          for (int t1 = 0; t1 < M; ++t1) {
            const int pt = t1 + M * t2;
            T v[M];
#pragma unroll
            for (int r = 0; r < M; ++r) v[r] = u[lidx<M, D>(r, t1, t2)];
            T f[M];
#pragma unroll
            for (int q = 0; q < M; ++q) {
              T s = tb.dcol[q * M] * v[0];
#pragma unroll
              for (int r = 1; r < M; ++r) s = fma(tb.dcol[q * M + r], v[r], s);
              f[q] = tb.gw[D][lidx<M, D>(q, t1, t2)] * s;
            }
#pragma unroll
            for (int q = 0; q < M; ++q) {
              T s = R[lidx<M, D>(q, t1, t2)];
#pragma unroll
              for (int r = 0; r < M; ++r) s = fma(tb.dcol[r * M + q], f[r], s);
              R[lidx<M, D>(q, t1, t2)] = s;
            }
            T u0 = tb.e0[0] * v[0], g0 = tb.d0[0] * v[0], u1 = tb.e1[0] * v[0], g1 = tb.d1[0] * v[0];
#pragma unroll
            for (int r = 1; r < M; ++r) {
              u0 = fma(tb.e0[r], v[r], u0); g0 = fma(tb.d0[r], v[r], g0);
              u1 = fma(tb.e1[r], v[r], u1); g1 = fma(tb.d1[r], v[r], g1);
            }
            trb[(0 * M2 + pt) * nb + tid] = u0;
            trb[(1 * M2 + pt) * nb + tid] = g0;
            trb[(2 * M2 + pt) * nb + tid] = u1;
            trb[(3 * M2 + pt) * nb + tid] = g1;
          }
        // A face on the brick boundary is read by no cell of the brick, so its slots take
        // the neighbour's trace from the halo instead: every neighbour trace is then at a
        // fixed offset from one address per side.
        const int lc = D == 0 ? lx : (D == 1 ? ly : lz);
        constexpr int bd = D == 0 ? bx : (D == 1 ? by : bz);
        constexpr int nd = D == 0 ? n0 : (D == 1 ? n1 : n2);
        const int p = D == 0 ? ly + by * lz : (D == 1 ? lx + bx * lz : lx + bx * ly);
        if (lc == 0) {
          const T *h = hl + hoff(D) + p;
#pragma unroll
          for (int i = 0; i < 2 * M2; ++i) trb[i * nb + tid] = h[i * nd];
        }
        if (lc == bd - 1) {
          const T *h = hl + hoff(D) + 2 * M2 * nd + p;
#pragma unroll
          for (int i = 0; i < 2 * M2; ++i) trb[(2 * M2 + i) * nb + tid] = h[i * nd];
        }
      }
      __syncthreads();
      if (act) {
        const int gc = D == 0 ? gx : (D == 1 ? gy : gz);
        const int nlim = D == 0 ? nx : (D == 1 ? ny : nz);
        const int lc = D == 0 ? lx : (D == 1 ? ly : lz);
        constexpr int bd = D == 0 ? bx : (D == 1 ? by : bz);
        constexpr int nstep = D == 0 ? 1 : (D == 1 ? bx : bx * by);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const bool bnd = s ? gc + 1 >= nlim : gc == 0;
          const bool dir = ((a.dmask >> (2 * D + s)) & 1u) != 0;
          // neighbour trace: values at nsrc[pt * nb], derivatives at nsrc[(M2 + pt) * nb]
          const bool inb = s ? lc + 1 < bd : lc > 0;
          const T *nsrc = trb + tid +
                          (s ? (inb ? nstep : 2 * M2 * nb) : (inb ? 2 * M2 * nb - nstep : 0));
#pragma unroll
          for (int t2 = 0; t2 < M; ++t2)
#pragma unroll
            for (int t1 = 0; t1 < M; ++t1) {
              const int pt = t1 + M * t2;
              // this cell's own trace, recomputed from its Gauss-point values (cheaper than
              // keeping it live in registers across the barrier)
              T uo, dno;
              {
                T v0 = u[lidx<M, D>(0, t1, t2)];
                uo = (s ? tb.e1[0] : tb.e0[0]) * v0;
                dno = (s ? tb.d1[0] : tb.d0[0]) * v0;
#pragma unroll
                for (int r = 1; r < M; ++r) {
                  const T vr = u[lidx<M, D>(r, t1, t2)];
                  uo = fma(s ? tb.e1[r] : tb.e0[r], vr, uo);
                  dno = fma(s ? tb.d1[r] : tb.d0[r], vr, dno);
                }
              }
              const T hb = tb.hbw[D][pt], pwv = tb.pw[D][pt];
              T Rv, Rn;
              if (bnd) {
                const T b = s ? hb + hb : -(hb + hb);
                Rv = dir ? fma(sc, b * dno, pwv * uo) : T(0);
                Rn = dir ? ss * uo * b : T(0);
              } else {
                const T un = nsrc[pt * nb], dnn = nsrc[(M2 + pt) * nb];
                const T J = s ? uo - un : un - uo;
                const T v = fma(sc, hb * (dno + dnn), pwv * J);
                Rv = s ? v : -v;
                Rn = ss * hb * J;
              }
#pragma unroll
              for (int r = 0; r < M; ++r) {
                T acc = R[lidx<M, D>(r, t1, t2)];
                acc = fma(s ? tb.e1[r] : tb.e0[r], Rv, acc);
                acc = fma(s ? tb.d1[r] : tb.d0[r], Rn, acc);
                R[lidx<M, D>(r, t1, t2)] = acc;
              }
            }
        }
      }
    };
    // x staging (buf1) was read above; axis 1 reuses buf1, axis 2 reuses buf0 (whose
    // axis-0 readers all passed the axis-1 barrier)
    axis(std::integral_constant<int, 0>{}, buf0);
    axis(std::integral_constant<int, 1>{}, buf1);
    axis(std::integral_constant<int, 2>{}, buf0);
    // transposed interpolation to the GLL coefficients, staged for a coalesced store
    // (buf1's last readers, the axis-1 face terms, all passed the axis-2 barrier)
    if (act) {
      T t2[P * M2];  // [j2][q1][q0]
#pragma unroll
      for (int j = 0; j < P; ++j)
#pragma unroll
        for (int qq = 0; qq < M2; ++qq) {
          T s = tb.interp[j] * R[qq];
#pragma unroll
          for (int q = 1; q < M; ++q) s = fma(tb.interp[q * P + j], R[q * M2 + qq], s);
          t2[j * M2 + qq] = s;
        }
      T t1[P2 * M];  // [j2][j1][q0]
#pragma unroll
      for (int j2 = 0; j2 < P; ++j2)
#pragma unroll
        for (int j1 = 0; j1 < P; ++j1)
#pragma unroll
          for (int q0 = 0; q0 < M; ++q0) {
            T s = tb.interp[j1] * t2[(j2 * M) * M + q0];
#pragma unroll
            for (int q = 1; q < M; ++q) s = fma(tb.interp[q * P + j1], t2[(j2 * M + q) * M + q0], s);
            t1[(j2 * P + j1) * M + q0] = s;
          }
#pragma unroll
      for (int jj = 0; jj < P2; ++jj)
#pragma unroll
        for (int j = 0; j < P; ++j) {
          T s = tb.interp[j] * t1[jj * M];
#pragma unroll
          for (int q = 1; q < M; ++q) s = fma(tb.interp[q * P + j], t1[jj * M + q], s);
          xs[tid * sX + jj * P + j] = s;
        }
    }
    __syncthreads();
    for (int row = warp; row < by * bz; row += nwarps) {
      const int ry = row % by, rz = row / by;
      if (ry >= nay || rz >= naz) continue;
      T *dst = yr + (ox + (int64_t)nx * (oy + ry + (int64_t)ny * (oz + rz))) * P3;
      const T *src = xs + row * bx * sX;
      if constexpr (sX == P3 && sizeof(T) == 4) {
        if ((nax * P3) % 4 == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
          const float4 *s4 = reinterpret_cast<const float4 *>(src);
          float4 *d4 = reinterpret_cast<float4 *>(dst);
          for (int j = lane; j < nax * P3 / 4; j += 32) d4[j] = s4[j];
          continue;
        }
      }
      for (int j = lane; j < nax * P3; j += 32) {
        const int cl = j / P3;
        dst[j] = src[cl * sX + (j - cl * P3)];
      }
    }
    __syncthreads();
  }
}

template <int P, typename T, int BZ>
cudaError_t run(const ScalarArgs<T> &a, const HostTables &ht, const T *x, T *y, int nrhs, int64_t sdof,
                cudaStream_t s, const cudaEvent_t *ev, int *grid_out, LaunchInfo *q) {
  constexpr int M = P, M2 = M * M, M3 = M2 * M;
  constexpr int bx = 8, by = 4, bz = BZ, nb = bx * by * bz;
  CTab<P, T> tb;
  for (int i = 0; i < P * P; ++i) { tb.interp[i] = (T)ht.interp[i]; tb.dcol[i] = (T)ht.dcol[i]; }
  for (int i = 0; i < P; ++i) {
    tb.e0[i] = (T)ht.e0[i]; tb.e1[i] = (T)ht.e1[i]; tb.d0[i] = (T)ht.d0[i]; tb.d1[i] = (T)ht.d1[i];
    tb.gd0[i] = (T)ht.gd0[i]; tb.gd1[i] = (T)ht.gd1[i];
  }
  const double *w = ht.gauss_w;
  for (int q = 0; q < M3; ++q) {
    const double W = w[q % M] * w[(q / M) % M] * w[q / M2];
    tb.mw[q] = (T)((double)a.vol_m * W);
    for (int d = 0; d < 3; ++d) tb.gw[d][q] = (T)((double)a.vol_g[d] * W);
  }
  for (int pt = 0; pt < M2; ++pt) {
    const double W = w[pt % M] * w[pt / M];
    for (int d = 0; d < 3; ++d) {
      tb.hbw[d][pt] = (T)(0.5 * W * (double)a.face_b[d]);
      tb.pw[d][pt] = (T)(W * (double)a.face_pw[d]);
    }
  }
  const size_t sm = cellwise_words<P>(bx, by, bz) * sizeof(T);
  auto k = k_cellwise<P, T, BZ>;
  cudaError_t e;
  if (sm > 48 * 1024 && (e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
    return e;
  int per_sm = 0, dev = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, nb, sm)) != cudaSuccess) return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int nbx = (a.nx + bx - 1) / bx, nby = (a.ny + by - 1) / by, nbz = (a.nz + bz - 1) / bz;
  const int64_t nbricks = (int64_t)nbx * nby * nbz;
  const int64_t nitems = (int64_t)nrhs * nbricks;
  int64_t grid = (int64_t)(per_sm > 0 ? per_sm : 1) * sms;
  if (grid > nitems) grid = nitems;
  if (grid_out) *grid_out = (int)grid;
  if (q) {
    q->blocks = grid;
    q->threads = nb;
    q->blocks_per_sm = per_sm;
    q->items = nitems;
    return cudaSuccess;
  }
  if (ev) cudaEventRecord(ev[0], s);
  k<<<(unsigned)grid, nb, sm, s>>>(a, tb, x, y, sdof, nbx, nby, nbricks, nitems);
  if (ev) {
    cudaEventRecord(ev[1], s);
    cudaEventRecord(ev[2], s);
    cudaEventRecord(ev[3], s);
  }
  return cudaGetLastError();
}

}  // namespace dgc

// Bricks of 8 x 4 x bz cells: `cells` = 64, 128 or 256 threads per block.
static int cellwise_bz(int cells) { return cells == 64 ? 2 : (cells == 128 ? 4 : (cells == 256 ? 8 : 0)); }

size_t cellwise_smem_bytes(int p, int cells, int es) {
  const int bz = cellwise_bz(cells);
  if (!bz) return 0;
  switch (p) {
    case 2: return dgc::cellwise_words<2>(8, 4, bz) * es;
    case 3: return dgc::cellwise_words<3>(8, 4, bz) * es;
    default: return 0;
  }
}

template <int P, typename T>
static cudaError_t run_bz(int bz, const ScalarArgs<T> &a, const HostTables &ht, const T *x, T *y, int nrhs,
                          int64_t sdof, cudaStream_t s, const cudaEvent_t *ev, int *grid_out, LaunchInfo *q) {
  switch (bz) {
    case 2: return dgc::run<P, T, 2>(a, ht, x, y, nrhs, sdof, s, ev, grid_out, q);
    case 4: return dgc::run<P, T, 4>(a, ht, x, y, nrhs, sdof, s, ev, grid_out, q);
    case 8: return dgc::run<P, T, 8>(a, ht, x, y, nrhs, sdof, s, ev, grid_out, q);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_cellwise_apply(int p, const ScalarArgs<T> &a, const HostTables &ht, const T *x, T *y, int nrhs,
                                  int64_t sdof, int cells, cudaStream_t s, const cudaEvent_t *ev, int *grid_out,
                                  LaunchInfo *q) {
  if (ht.m != p || ht.p != p) return cudaErrorInvalidValue;
  const int bz = cellwise_bz(cells);
  switch (p) {
    case 2: return run_bz<2, T>(bz, a, ht, x, y, nrhs, sdof, s, ev, grid_out, q);
    case 3: return run_bz<3, T>(bz, a, ht, x, y, nrhs, sdof, s, ev, grid_out, q);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_cellwise_apply<float>(int, const ScalarArgs<float> &, const HostTables &, const float *,
                                                  float *, int, int64_t, int, cudaStream_t, const cudaEvent_t *, int *,
                                                  LaunchInfo *);
template cudaError_t launch_cellwise_apply<double>(int, const ScalarArgs<double> &, const HostTables &,
                                                   const double *, double *, int, int64_t, int, cudaStream_t,
                                                   const cudaEvent_t *, int *, LaunchInfo *);
