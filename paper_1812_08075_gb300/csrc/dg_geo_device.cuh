// Device helpers for trilinear cell geometry (each cell is the image of the reference
// cube under the trilinear map through its eight vertices, Sec. 2.1).
#pragma once
#include <stdint.h>

#include "dg_internal.h"

namespace dgg {

__device__ __forceinline__ void cell_corners(const double *verts, int nx, int ny, int64_t cell, double V[8][3]) {
  const int cx = (int)(cell % nx);
  const int cy = (int)((cell / nx) % ny);
  const int cz = (int)(cell / ((int64_t)nx * ny));
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int64_t v = (cx + (a & 1)) + (int64_t)(nx + 1) * ((cy + ((a >> 1) & 1)) + (int64_t)(ny + 1) * (cz + (a >> 2)));
#pragma unroll
    for (int d = 0; d < 3; ++d) V[a][d] = verts[3 * v + d];
  }
}

// J[i][d] = d x_i / d xi_d of the trilinear map at (x0, x1, x2).
__device__ __forceinline__ void trilinear_jacobian(const double V[8][3], double x0, double x1, double x2, double J[3][3]) {
  const double f[3][2] = {{1.0 - x0, x0}, {1.0 - x1, x1}, {1.0 - x2, x2}};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int d = 0; d < 3; ++d) J[i][d] = 0.0;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int b0 = a & 1, b1 = (a >> 1) & 1, b2 = a >> 2;
    const double s0 = b0 ? 1.0 : -1.0, s1 = b1 ? 1.0 : -1.0, s2 = b2 ? 1.0 : -1.0;
    const double dN0 = s0 * f[1][b1] * f[2][b2];
    const double dN1 = f[0][b0] * s1 * f[2][b2];
    const double dN2 = f[0][b0] * f[1][b1] * s2;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      J[i][0] += dN0 * V[a][i];
      J[i][1] += dN1 * V[a][i];
      J[i][2] += dN2 * V[a][i];
    }
  }
}

// Adjugate (transpose of the cofactor matrix) and determinant: J^-1 = adj / det.
template <typename T>
__device__ __forceinline__ T adjugate(const T J[3][3], T A[3][3]) {
  A[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  A[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  A[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  A[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  A[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  A[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  A[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  A[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  A[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  return J[0][0] * A[0][0] + J[0][1] * A[1][0] + J[0][2] * A[2][0];
}

// Area vector of the face xi_a = const of a cell at its point with Jacobian J: the cross
// product of the tangential columns (t1 < t2), oriented along +xi_a (dir = +1) or -xi_a.
template <typename T>
__device__ __forceinline__ void area_vector(const T J[3][3], int a, int dir, T n[3]) {
  const int t1 = (a == 0) ? 1 : 0, t2 = (a == 2) ? 1 : 2;
  const T u0 = dg_pick3(J[0][0], J[0][1], J[0][2], t1), u1 = dg_pick3(J[1][0], J[1][1], J[1][2], t1);
  const T u2 = dg_pick3(J[2][0], J[2][1], J[2][2], t1);
  const T v0 = dg_pick3(J[0][0], J[0][1], J[0][2], t2), v1 = dg_pick3(J[1][0], J[1][1], J[1][2], t2);
  const T v2 = dg_pick3(J[2][0], J[2][1], J[2][2], t2);
  // (a, t1, t2) is an even permutation of (0,1,2) for a = 0, 2 and odd for a = 1; dir = +-1
  const T sg = ((a == 1) != (dir < 0)) ? T(-1) : T(1);
  n[0] = sg * (u1 * v2 - u2 * v1);
  n[1] = sg * (u2 * v0 - u0 * v2);
  n[2] = sg * (u0 * v1 - u1 * v0);
}


// Coefficients of the Jacobian columns of a trilinear map: column d of J at xi equals
// C[d][0] + xi_a C[d][1] + xi_b C[d][2] + xi_a xi_b C[d][3] with (a, b) the other two
// axes in increasing order; C[d][k][i] for coordinate i.
__device__ __forceinline__ void jacobian_coeffs(const double V[8][3], double C[3][4][3]) {
  for (int d = 0; d < 3; ++d) {
    const int a = d == 0 ? 1 : 0, b = d == 2 ? 1 : 2;
    double D[2][2][3];
    for (int ba = 0; ba < 2; ++ba)
      for (int bb = 0; bb < 2; ++bb) {
        int lo = (ba << a) | (bb << b), hi = lo | (1 << d);
        for (int i = 0; i < 3; ++i) D[ba][bb][i] = V[hi][i] - V[lo][i];
      }
    for (int i = 0; i < 3; ++i) {
      C[d][0][i] = D[0][0][i];
      C[d][1][i] = D[1][0][i] - D[0][0][i];
      C[d][2][i] = D[0][1][i] - D[0][0][i];
      C[d][3][i] = D[1][1][i] - D[1][0][i] - D[0][1][i] + D[0][0][i];
    }
  }
}

// J from those coefficients (C laid out as 36 consecutive values, [d][k][i]).
template <typename T>
__device__ __forceinline__ void jacobian_from_coeffs(const T *C, T x0, T x1, T x2, T J[3][3]) {
  const T xi[3] = {x0, x1, x2};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const T xa = xi[d == 0 ? 1 : 0], xb = xi[d == 2 ? 1 : 2], xab = xa * xb;
    const T *c = C + d * 12;
#pragma unroll
    for (int i = 0; i < 3; ++i) J[i][d] = fma(xab, c[9 + i], fma(xb, c[6 + i], fma(xa, c[3 + i], c[i])));
  }
}

}  // namespace dgg
