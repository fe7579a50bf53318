// Line-per-thread forms of the scalar cell and back-projection kernels, for the number
// types whose pipes run far faster than FP64 (FP32 and double-float). The thread-per-point
// kernels decompose a flat index into cell and tensor indices for every element and read
// the table entry of every product from shared memory; with the FP64 pipe as the bound
// that work is hidden, on the FP32 pipes it is the bound. Here a thread contracts a whole
// tensor line (P inputs to M outputs or back), so the index arithmetic is paid once per
// line, and the tables arrive by value as a kernel parameter: after unrolling, every table
// entry is a constant-bank operand of the FMA. The arithmetic, its order within each sum
// and the scratch layouts are those of k_cell / k_back (Algorithm 1 Parts 1-3; facet
// traces of Sec. 2.2), except that the volume residual is accumulated axis by axis.
#pragma once
#include "dg_scalar_kernels.cuh"

namespace dgk {

template <int P, int M, typename T>
struct LineTab {
  T interp[M * P];  // [q][j]
  T dcol[M * M];    // [q][r]
  T e0[M], e1[M], d0[M], d1[M];
};

template <int P, int M, typename T>
LineTab<P, M, T> line_tables(const HostTables &h) {
  LineTab<P, M, T> t;
  for (int i = 0; i < M * P; ++i) t.interp[i] = T(h.interp[i]);
  for (int i = 0; i < M * M; ++i) t.dcol[i] = T(h.dcol[i]);
  for (int i = 0; i < M; ++i) {
    t.e0[i] = T(h.e0[i]); t.e1[i] = T(h.e1[i]);
    t.d0[i] = T(h.d0[i]); t.d1[i] = T(h.d1[i]);
  }
  return t;
}

// The loops over the three axes are unrolled (compile-time line strides and bases: less
// index arithmetic) for FP32 up to M = 4; for double-float and larger M the unrolled code
// measured slower (instruction cache), so they stay loops.
template <int M, typename T>
__host__ __device__ constexpr int axis_unroll() {
  return (std::is_same<T, float>::value && M <= 4) ? 3 : 1;
}

// out[o * os] = sum_n mat[o][n] in[n * is] for o < NO (mat row-major NO x NI, or its
// transpose when TR), one line
template <int NI, int NO, bool TR, typename T, typename TI, typename TO>
__device__ __forceinline__ void line_contract(const T (&mat)[NI * NO], const TI *in, int is, TO *out, int os) {
  T v[NI];
#pragma unroll
  for (int n = 0; n < NI; ++n) v[n] = in[n * is];
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    Acc<T> acc;
    acc.init(TR ? mat[o] : mat[o * NI], v[0]);
#pragma unroll
    for (int n = 1; n < NI; ++n) acc.add(TR ? mat[n * NO + o] : mat[o * NI + n], v[n]);
    store_to(out + o * os, acc.get());
  }
}

// base and stride of the line along axis d through the face point qf = s + M t (s, t the
// other two axes in increasing order), in a [M][M][M] block with axis 0 fastest
template <int M>
__device__ __forceinline__ void line_of(int d, int qf, int &base, int &stride) {
  const int s = qf % M, t = qf / M;
  base = d == 0 ? M * qf : (d == 1 ? s + M * M * t : qf);
  stride = d == 0 ? 1 : (d == 1 ? M : M * M);
}

template <int P, int M, typename T, int GEO, bool KAPPA>
__global__ void __launch_bounds__(256) k_cell_lines(const ScalarArgs<T> a, const LineTab<P, M, T> tb,
                                                    const io_t<T> *__restrict__ x, T *__restrict__ rvol,
                                                    T *__restrict__ traces, int cpb, int64_t sx, int64_t sr,
                                                    int64_t st) {
  constexpr int P3 = P * P * P, M2 = M * M, M3 = M * M * M;
  constexpr int kAxisUnroll = axis_unroll<M, T>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *S0 = reinterpret_cast<T *>(smem_raw);
  T *S1 = S0 + cpb * M3, *S2 = S1 + cpb * M3, *S3 = S2 + cpb * M3;
  const int tid = threadIdx.x, nt = blockDim.x;
  x += blockIdx.y * sx;
  rvol += blockIdx.y * sr;
  traces += blockIdx.y * st;
  const int64_t c0 = (int64_t)blockIdx.x * cpb;
  const int nc = (int)min((int64_t)cpb, a.ncell - c0);
  {
    const io_t<T> *xb = x + c0 * P3;
    if constexpr (std::is_same<io_t<T>, T>::value) {
      stage_async<T>(S0, xb, nc * P3, tid, nt);
      dg_cp_async_wait_all();
    } else {
      for (int i = tid; i < nc * P3; i += nt) S0[i] = io_in<T>(xb[i]);
    }
  }
  __syncthreads();
  // interpolation: [c][j2][j1][j0] -> [c][j2][j1][q0] -> [c][j2][q1][q0] -> U [c][q2][q1][q0]
  for (int l = tid; l < nc * P * P; l += nt) line_contract<P, M, false>(tb.interp, S0 + l * P, 1, S1 + l * M, 1);
  __syncthreads();
  for (int l = tid; l < nc * P * M; l += nt) {
    const int q0 = l % M, cj = l / M;
    line_contract<P, M, false>(tb.interp, S1 + cj * (P * M) + q0, M, S0 + cj * M2 + q0, M);
  }
  __syncthreads();
  for (int l = tid; l < nc * M2; l += nt) {
    const int q01 = l % M2, c = l / M2;
    line_contract<P, M, false>(tb.interp, S0 + c * (P * M2) + q01, M2, S2 + c * M3 + q01, M2);
  }
  __syncthreads();
  const T *U = S2;
  // along each axis d: the four face values (u and d_n u on both faces normal to d) and the
  // reference derivative d/dxi_d at every point of the line, into G_d (S0, S1, S3)
  {
    T *tr = traces + c0 * (12 * M2);
    auto trace_line = [&](int c, int d, int qf) {
      int base, stride;
      line_of<M>(d, qf, base, stride);
      const T *u = U + c * M3 + base;
      T v[M];
#pragma unroll
      for (int j = 0; j < M; ++j) v[j] = u[j * stride];
      Acc<T> a0, a1, a2, a3;
      a0.init(tb.e0[0], v[0]); a1.init(tb.d0[0], v[0]); a2.init(tb.e1[0], v[0]); a3.init(tb.d1[0], v[0]);
#pragma unroll
      for (int j = 1; j < M; ++j) {
        a0.add(tb.e0[j], v[j]); a1.add(tb.d0[j], v[j]); a2.add(tb.e1[j], v[j]); a3.add(tb.d1[j], v[j]);
      }
      T *tc = tr + c * (12 * M2) + qf;
      tc[(4 * d + 0) * M2] = a0.get();
      tc[(4 * d + 1) * M2] = a1.get();
      tc[(4 * d + 2) * M2] = a2.get();
      tc[(4 * d + 3) * M2] = a3.get();
      T *g = (d == 0 ? S0 : (d == 1 ? S1 : S3)) + c * M3 + base;
#pragma unroll
      for (int q = 0; q < M; ++q) {
        Acc<T> acc;
        acc.init(tb.dcol[q * M], v[0]);
#pragma unroll
        for (int j = 1; j < M; ++j) acc.add(tb.dcol[q * M + j], v[j]);
        g[q * stride] = acc.get();
      }
    };
    if constexpr (kAxisUnroll == 3) {
      // one pass per axis, unrolled: each pass's line stride and base are compile-time
#pragma unroll
      for (int d = 0; d < 3; ++d)
        for (int l = tid; l < nc * M2; l += nt) trace_line(l / M2, d, l % M2);
    } else {
      for (int l = tid; l < nc * 3 * M2; l += nt) {
        const int c = l / (3 * M2), r = l - c * (3 * M2), d = r / M2;
        trace_line(c, d, r - d * M2);
      }
    }
  }
  __syncthreads();
  // pointwise volume flux (in place in G_d) and the mass term, which starts R in S2
  for (int i = tid; i < nc * M3; i += nt) {
    const int c = i / M3, q = i - c * M3;
    const int q0 = q % M, q1 = (q / M) % M, q2 = q / M2;
    T g0 = S0[i], g1 = S1[i], g2 = S3[i], f0, f1, f2, mw;
    if (GEO == GEO_AFFINE) {
      // the weights' indices differ between threads: read them from the device table (L1)
      // rather than the constant bank, which would serialise the distinct addresses
      const T W = a.tab->w[q0] * a.tab->w[q1] * a.tab->w[q2];
      T Wk = W;
      if (KAPPA) Wk *= io_in<T>(a.kappa_vol[(c0 + c) * M3 + q]);
      f0 = (Wk * a.vol_g[0]) * g0;
      f1 = (Wk * a.vol_g[1]) * g1;
      f2 = (Wk * a.vol_g[2]) * g2;
      mw = W * a.vol_m;
    } else {
      const T *G = a.gvol + (c0 + c) * (7 * M3) + q;
      if (KAPPA) {
        const T kq = io_in<T>(a.kappa_vol[(c0 + c) * M3 + q]);
        g0 *= kq; g1 *= kq; g2 *= kq;
      }
      const T G00 = G[0], G01 = G[M3], G02 = G[2 * M3], G11 = G[3 * M3], G12 = G[4 * M3], G22 = G[5 * M3];
      Acc<T> b0, b1, b2;
      b0.init(G02, g2); b0.add(G01, g1); b0.add(G00, g0);
      b1.init(G12, g2); b1.add(G11, g1); b1.add(G01, g0);
      b2.init(G22, g2); b2.add(G12, g1); b2.add(G02, g0);
      f0 = b0.get(); f1 = b1.get(); f2 = b2.get();
      mw = G[6 * M3];
    }
    S0[i] = f0;
    S1[i] = f1;
    S3[i] = f2;
    S2[i] = mw * U[i];
  }
  __syncthreads();
  // R += D_d^T f_d, one axis at a time; the last axis writes R_vol
#pragma unroll kAxisUnroll
  for (int d = 0; d < 3; ++d) {
    const T *F = d == 0 ? S0 : (d == 1 ? S1 : S3);
    for (int l = tid; l < nc * M2; l += nt) {
      const int c = l / M2, qf = l - c * M2;
      int base, stride;
      line_of<M>(d, qf, base, stride);
      const T *f = F + c * M3 + base;
      T *R = S2 + c * M3 + base;
      T v[M];
#pragma unroll
      for (int j = 0; j < M; ++j) v[j] = f[j * stride];
#pragma unroll
      for (int q = 0; q < M; ++q) {
        Acc<T> acc;
        acc.set(R[q * stride]);
#pragma unroll
        for (int j = 0; j < M; ++j) acc.add(tb.dcol[j * M + q], v[j]);
        if (d < 2) R[q * stride] = acc.get();
        else rvol[(c0 + c) * M3 + base + q * stride] = acc.get();
      }
    }
    if (d < 2) __syncthreads();
  }
}

template <int P, int M, typename T>
__global__ void __launch_bounds__(256) k_back_lines(const ScalarArgs<T> a, const LineTab<P, M, T> tb,
                                                    const T *__restrict__ rvol, const T *__restrict__ fres,
                                                    io_t<T> *__restrict__ y, int cpb, int64_t sy, int64_t sr,
                                                    int64_t st) {
  constexpr int P3 = P * P * P, M2 = M * M, M3 = M * M * M;
  constexpr int kAxisUnroll = axis_unroll<M, T>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *S0 = reinterpret_cast<T *>(smem_raw);
  T *S1 = S0 + cpb * M3, *SF = S1 + cpb * M3;
  const int tid = threadIdx.x, nt = blockDim.x;
  y += blockIdx.y * sy;
  rvol += blockIdx.y * sr;
  fres += blockIdx.y * st;
  const int64_t c0 = (int64_t)blockIdx.x * cpb;
  const int nc = (int)min((int64_t)cpb, a.ncell - c0);
  stage_async<T>(S0, rvol + c0 * M3, nc * M3, tid, nt);
  stage_async<T>(SF, fres + c0 * 12 * M2, nc * 12 * M2, tid, nt);
  dg_cp_async_wait_all();
  __syncthreads();
  // face residuals lifted along the normal axis of each face pair, one axis at a time
#pragma unroll kAxisUnroll
  for (int d = 0; d < 3; ++d) {
    for (int l = tid; l < nc * M2; l += nt) {
      const int c = l / M2, qf = l - c * M2;
      int base, stride;
      line_of<M>(d, qf, base, stride);
      const T *sf = SF + c * (12 * M2) + qf;
      const T lu = sf[(4 * d + 0) * M2], ld = sf[(4 * d + 1) * M2];
      const T hu = sf[(4 * d + 2) * M2], hd = sf[(4 * d + 3) * M2];
      T *R = S0 + c * M3 + base;
#pragma unroll
      for (int q = 0; q < M; ++q) {
        Acc<T> acc;
        acc.set(R[q * stride]);
        acc.add(tb.e0[q], lu);
        acc.add(tb.d0[q], ld);
        acc.add(tb.e1[q], hu);
        acc.add(tb.d1[q], hd);
        R[q * stride] = acc.get();
      }
    }
    __syncthreads();
  }
  // transposed interpolation: [c][q2][q1][q0] -> [c][q2][q1][j0] -> [c][q2][j1][j0] -> y
  for (int l = tid; l < nc * M2; l += nt) line_contract<M, P, true>(tb.interp, S0 + l * M, 1, S1 + l * P, 1);
  __syncthreads();
  for (int l = tid; l < nc * M * P; l += nt) {
    const int j0 = l % P, cq = l / P;
    line_contract<M, P, true>(tb.interp, S1 + cq * (M * P) + j0, P, S0 + cq * (P * P) + j0, P);
  }
  __syncthreads();
  {
    io_t<T> *yb = y + c0 * P3;
    for (int l = tid; l < nc * P * P; l += nt) {
      const int j01 = l % (P * P), c = l / (P * P);
      line_contract<M, P, true>(tb.interp, S0 + c * (M * P * P) + j01, P * P, yb + c * P3 + j01, P * P);
    }
  }
}

}  // namespace dgk
