// One-thread-per-cell persistent apply for affine (axis-parallel) meshes and low degree
// (k <= 2), used for FP32.
//
// A block owns a brick of bx x by x bz cells, one thread per cell, and loops over work
// items (right-hand side, brick) in one wave of blocks. Each thread runs Algorithm 1 for
// its cell in registers, every contraction fully unrolled so that the table entries,
// identical across the block, are constant-bank operands of the FMAs.
//
// The cell works on weighted Gauss-point values u~ = W u (W_q = w_q0 w_q1 w_q2, folded
// into the interpolation tables). On an axis-parallel cell with constant coefficients
// everything that couples a cell to itself acts along one tensor line at a time, so per
// axis d it is one M x M matrix applied to each line of u~ (Sec. 2.2's tensor structure):
//   - the stiffness g_d D^T diag(w) D (the metric G is diagonal and constant);
//   - the cell's own side of its two faces normal to d (Eq. diffreac_weak: the flux,
//     symmetry and penalty terms with the neighbour's trace set to zero, or the Dirichlet
//     terms on a boundary face; face weights W_t = w_t1 w_t2 are those of u~'s line);
//   - on axis 0, the mass term c detJ.
// These matrices are formed on the host in FP64. What is left per face point is the
// coupling to the neighbour: its weighted trace (u~ and the reference normal derivative)
// times two coefficient vectors of length M. Cells exchange traces through shared memory,
// one axis at a time; neighbours across the brick boundary are turned into traces at the
// start of the item from their GLL coefficients (face layer of nodes, end row of the GLL
// derivative along the normal, facet sum factorisation to the face Gauss points with the
// weights folded in), one brick-boundary face per thread. x and y are staged through
// shared memory so that the global accesses are coalesced rows of the brick. In FP32 the
// sweeps along y and z and four of the six interpolation sweeps run two tensor lines at a
// time on the packed FP32 FMA (f32x2), with the same operations per line as the scalar code.
#include <limits.h>

#include <type_traits>

#include "dg_internal.h"

namespace dgc {

// Set by a cellwise launch whose wait for its bulk copies gave up (bit 0); read and cleared
// by dg_device_faults.
__device__ unsigned g_cellwise_fault = 0;

// Bulk copies global -> shared completed on an mbarrier (Blackwell TMA engine, untiled form)
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect(unsigned long long *bar, unsigned bytes) {
  asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
  asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(smem_addr(bar)) : "memory");
}

// 16-byte aligned source and destination, size a multiple of 16
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Generic-proxy accesses of this thread ordered before later async-proxy (bulk copy) ones
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Wait for the phase of the given parity, at most about one second (clock cycles); false
// when it gave up (the fault word is then set and the caller carries on).
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
  const long long t0 = clock64();
  for (;;) {
    unsigned done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > 2000000000LL) {
      atomicOr(&g_cellwise_fault, 1u);
      return false;
    }
  }
}

// Tables and per-axis operators, passed by value (constant bank).
template <int P, typename T>
struct CTab {
  T iw[P * P];             // [q][j] w_q * (GLL basis j at Gauss point q): interpolation to u~
  T it[P * P];             // [q][j] GLL basis j at Gauss point q: transposed interpolation
  T gd0[P], gd1[P];        // GLL basis derivative at xi = 0, 1
  T te[4][P];              // e0 / w, d0 / w, e1 / w, d1 / w: weighted traces from u~
  T K[3][P * P];           // [d][q][r] line operator of axis d (interior faces on both sides)
  T corr[3][2][P * P];     // [d][side] correction of a cell on the domain boundary
  T na[3][2][P], nbv[3][2][P];  // neighbour coupling: R[r] += na[r] u~n + nbv[r] dn~n
};

// Index of the value at position r along axis D of the line (t1, t2) of a cell's
// Gauss-point array [q2][q1][q0]; t1 < t2 are the other two axes in increasing order.
template <int M, int D>
__device__ __forceinline__ constexpr int lidx(int r, int t1, int t2) {
  return D == 0 ? r + M * (t1 + M * t2) : (D == 1 ? t1 + M * (r + M * t2) : t1 + M * (t2 + M * r));
}

// Packed FP32 (f32x2: one instruction does the FMA of two lanes) on pairs of tensor lines
// that share every coefficient. Each lane does the same operations in the same order as the
// scalar code, so results are unchanged.
__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 bc(float c) { return make_float2(c, c); }

// One sum-factorisation sweep over NO outputs, contracting NJ inputs:
// out[o os + b] = sum_j c[o co + j cj] in[j is + b], for b over NR rows of M unit-stride
// values. With PK, pairs of neighbouring values in a row (lines sharing the coefficients)
// go through packed FMAs.
template <int NO, int NJ, int NR, int M, bool PK, typename T>
__device__ __forceinline__ void sweep(T *out, const int os, const T *in, const int is, const T *c, const int co,
                                      const int cj) {
#pragma unroll
  for (int o = 0; o < NO; ++o)
#pragma unroll
    for (int row = 0; row < NR; ++row) {
#pragma unroll
      for (int q = 0; q < M; ++q) {
        const int b = row * M + q;
        if constexpr (PK) {
          if (q & 1) continue;  // the second value of a pair
          if (q + 1 < M) {
            float2 s = __fmul2_rn(bc(c[o * co]), pk(in[b], in[b + 1]));
#pragma unroll
            for (int j = 1; j < NJ; ++j) s = __ffma2_rn(bc(c[o * co + j * cj]), pk(in[j * is + b], in[j * is + b + 1]), s);
            out[o * os + b] = s.x;
            out[o * os + b + 1] = s.y;
            continue;
          }
        }
        T s = c[o * co] * in[b];
#pragma unroll
        for (int j = 1; j < NJ; ++j) s = fma(c[o * co + j * cj], in[j * is + b], s);
        out[o * os + b] = s;
      }
    }
}

// Two running sums of FP32 products in double-float (lanes x and y): each product's
// rounding error is kept exactly (FMA), and the high parts add by TwoSum (Knuth), as in the
// solver's dot products.
struct DotPair {
  float2 hi = make_float2(0.f, 0.f), lo = make_float2(0.f, 0.f);
  static __device__ __forceinline__ float2 neg(float2 v) { return make_float2(-v.x, -v.y); }
  __device__ __forceinline__ void add(float2 a, float2 b) {
    const float2 p = __fmul2_rn(a, b);
    const float2 e = __ffma2_rn(a, b, neg(p));  // a b - p exactly
    // TwoSum(hi, p): sm + t = hi + p exactly
    const float2 sm = __fadd2_rn(hi, p);
    const float2 bb = __fadd2_rn(sm, neg(hi));
    const float2 t = __fadd2_rn(__fadd2_rn(hi, neg(__fadd2_rn(sm, neg(bb)))), __fadd2_rn(p, neg(bb)));
    hi = sm;
    lo = __fadd2_rn(lo, __fadd2_rn(t, e));
  }
  __device__ __forceinline__ double value() const {
    return ((double)hi.x + (double)lo.x) + ((double)hi.y + (double)lo.y);
  }
};

// Vector access to shared memory: four values (16-byte aligned) and pairs (8-byte
// aligned for float, 16-byte for double).
__device__ __forceinline__ void store4(float *p, float a, float b, float c, float d) {
  *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void store4(double *p, double a, double b, double c, double d) {
  reinterpret_cast<double2 *>(p)[0] = make_double2(a, b);
  reinterpret_cast<double2 *>(p)[1] = make_double2(c, d);
}
__device__ __forceinline__ void store2(float *p, float a, float b) { *reinterpret_cast<float2 *>(p) = make_float2(a, b); }
__device__ __forceinline__ void store2(double *p, double a, double b) {
  *reinterpret_cast<double2 *>(p) = make_double2(a, b);
}
__device__ __forceinline__ void load2(const float *p, float &a, float &b) {
  const float2 v = *reinterpret_cast<const float2 *>(p);
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ void load2(const double *p, double &a, double &b) {
  const double2 v = *reinterpret_cast<const double2 *>(p);
  a = v.x;
  b = v.y;
}

// Trace buffer of one axis: [cell][face point][u0, g0, u1, g1] (value and reference normal
// derivative on the lower and upper face), NT = 4 M^2 words per cell; halo traces of the
// brick-boundary neighbours: [axis][side][plane][face point][u, g].
template <int P>
struct CLayout {
  static constexpr int P3 = P * P * P, M2 = P * P;
  static constexpr int sX = P3 | 1;            // per-cell stride of the x / y staging (odd)
  static constexpr int NT = 4 * M2;            // trace words per cell and axis
  static constexpr int buf = NT > sX ? NT : sX;
};

// FP32 with x rows staged as laid out in memory (k = 2) copies each item's x rows and the
// GLL coefficients of its brick-boundary neighbours into shared memory with bulk copies
// (cp.async.bulk, completed on mbarriers) one item ahead. Neighbour staging: the 2 bz rows
// across y and the 2 by rows across z (bx cells each, as in memory) and the 2 by bz single
// cells across x, each in a slot holding the 16-byte-aligned span around the cell. The slot
// stride (36 words, 4 mod 32) keeps the lanes reading consecutive slots on 8 banks.
template <int P, typename T>
__host__ __device__ constexpr bool cellwise_stage() {
  return sizeof(T) == 4 && (P * P * P) % 2 == 1;
}
constexpr int kHaloSlot = 36;
template <int P>
inline constexpr size_t halo_stage_words(int bx, int by, int bz) {
  return (size_t)(2 * bz + 2 * by) * bx * P * P * P + (size_t)2 * by * bz * kHaloSlot;
}

// Shared memory words: the x / y staging rows, one trace buffer (the z exchange; x and y
// neighbours are lanes of the same warp and exchange by shuffles) and the brick-boundary
// traces of the three axes.
template <int P>
inline size_t cellwise_words(int bx, int by, int bz, bool stage) {
  using LY = CLayout<P>;
  const size_t nb = (size_t)bx * by * bz;
  return (size_t)(LY::sX + LY::NT) * nb + (size_t)LY::NT * (by * bz + bx * bz + bx * by) +
         (stage ? halo_stage_words<P>(bx, by, bz) : 0);
}

// Host construction of CTab from the reference tables (FP64) and the affine constants.
template <int P, typename T>
CTab<P, T> make_tab(const ScalarArgs<T> &a, const HostTables &ht) {
  constexpr int M = P;
  CTab<P, T> tb;
  const double *w = ht.gauss_w;
  for (int q = 0; q < M; ++q)
    for (int j = 0; j < P; ++j) {
      tb.iw[q * P + j] = (T)(w[q] * ht.interp[q * P + j]);
      tb.it[q * P + j] = (T)ht.interp[q * P + j];
    }
  for (int j = 0; j < P; ++j) { tb.gd0[j] = (T)ht.gd0[j]; tb.gd1[j] = (T)ht.gd1[j]; }
  const double *ev[2] = {ht.e0, ht.e1}, *dv[2] = {ht.d0, ht.d1};
  for (int r = 0; r < M; ++r) {
    tb.te[0][r] = (T)(ht.e0[r] / w[r]); tb.te[1][r] = (T)(ht.d0[r] / w[r]);
    tb.te[2][r] = (T)(ht.e1[r] / w[r]); tb.te[3][r] = (T)(ht.d1[r] / w[r]);
  }
  const double sc = (double)a.sc, ss = (double)a.ss;
  for (int d = 0; d < 3; ++d) {
    const double g = (double)a.vol_g[d], hb = 0.5 * (double)a.face_b[d], pw = (double)a.face_pw[d];
    double K[M][M], F[2][2][M][M];  // F[side][0: interior, 1: Dirichlet][row r][col k]
    for (int q = 0; q < M; ++q)
      for (int r = 0; r < M; ++r) {
        double s = 0.0;
        for (int p = 0; p < M; ++p) s += ht.dcol[p * M + q] * w[p] * ht.dcol[p * M + r];
        K[q][r] = g * s / w[r];
      }
    if (d == 0)
      for (int q = 0; q < M; ++q) K[q][q] += (double)a.vol_m;
    for (int s = 0; s < 2; ++s) {
      const double sg = s ? 1.0 : -1.0;
      for (int r = 0; r < M; ++r)
        for (int k = 0; k < M; ++k) {
          const double et = ev[s][k] / w[k], dt = dv[s][k] / w[k];
          // own side of an interior face: neighbour trace zero in the jump and average
          F[s][0][r][k] = ev[s][r] * (sg * sc * hb * dt + pw * et) + dv[s][r] * sg * ss * hb * et;
          // Dirichlet face: jump = average = trace, outward normal, no factor 1/2
          F[s][1][r][k] = ev[s][r] * (2.0 * sg * sc * hb * dt + pw * et) + dv[s][r] * 2.0 * sg * ss * hb * et;
        }
      for (int r = 0; r < M; ++r) {
        tb.na[d][s][r] = (T)(-pw * ev[s][r] - sg * ss * hb * dv[s][r]);
        tb.nbv[d][s][r] = (T)(sg * sc * hb * ev[s][r]);
      }
    }
    const bool dir[2] = {((a.dmask >> (2 * d)) & 1u) != 0, ((a.dmask >> (2 * d + 1)) & 1u) != 0};
    for (int r = 0; r < M; ++r)
      for (int k = 0; k < M; ++k) {
        tb.K[d][r * M + k] = (T)(K[r][k] + F[0][0][r][k] + F[1][0][r][k]);
        for (int s = 0; s < 2; ++s)
          tb.corr[d][s][r * M + k] = (T)((dir[s] ? F[s][1][r][k] : 0.0) - F[s][0][r][k]);
      }
  }
  return tb;
}

// Weighted trace of a neighbour cell's face normal to axis D from its GLL coefficients
// `src`: SIDE 1 is the neighbour's lower face (xi_D = 0), SIDE 0 its upper face. The pair
// (W_t u, W_t du/dxi_D) of face point pt goes to dst[2 pt], dst[2 pt + 1].
// One code path for every axis and side (strides and side at run time, a single call
// site): six specialisations made the kernel's code outgrow the instruction cache.
template <int P, typename T, bool SHARED>
__device__ __forceinline__ void halo_trace(const T *__restrict__ src, const CTab<P, T> &tb, T *dst, int stn, int st1,
                                            int st2, int side) {
  constexpr int M = P, P2 = P * P, M2 = M * M;
  T gd[P];
#pragma unroll
  for (int j = 0; j < P; ++j) gd[j] = side ? tb.gd0[j] : tb.gd1[j];
  T v[P2], dv[P2];
#pragma unroll
  for (int n2 = 0; n2 < P; ++n2)
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) {
      T line[P];
#pragma unroll
      for (int j = 0; j < P; ++j) line[j] = SHARED ? src[n1 * st1 + n2 * st2 + j * stn] : __ldg(src + n1 * st1 + n2 * st2 + j * stn);
      v[n1 + P * n2] = side ? line[0] : line[P - 1];
      T s = gd[0] * line[0];
#pragma unroll
      for (int j = 1; j < P; ++j) s = fma(gd[j], line[j], s);
      dv[n1 + P * n2] = s;
    }
  T tv[M * P], tdv[M * P];  // after the sweep along t1: [n2][q1]
#pragma unroll
  for (int n2 = 0; n2 < P; ++n2)
#pragma unroll
    for (int q1 = 0; q1 < M; ++q1) {
      T a = tb.iw[q1 * P] * v[P * n2], b = tb.iw[q1 * P] * dv[P * n2];
#pragma unroll
      for (int n1 = 1; n1 < P; ++n1) {
        a = fma(tb.iw[q1 * P + n1], v[n1 + P * n2], a);
        b = fma(tb.iw[q1 * P + n1], dv[n1 + P * n2], b);
      }
      tv[q1 + M * n2] = a;
      tdv[q1 + M * n2] = b;
    }
#pragma unroll
  for (int q2 = 0; q2 < M; ++q2)
#pragma unroll
    for (int q1 = 0; q1 < M; ++q1) {
      T a = tb.iw[q2 * P] * tv[q1], b = tb.iw[q2 * P] * tdv[q1];
#pragma unroll
      for (int n2 = 1; n2 < P; ++n2) {
        a = fma(tb.iw[q2 * P + n2], tv[q1 + M * n2], a);
        b = fma(tb.iw[q2 * P + n2], tdv[q1 + M * n2], b);
      }
      store2(dst + 2 * (q1 + M * q2), a, b);
    }
}

// The brick is 8 x 4 x BZ cells (a warp spans 8 x 4 cells); its shape is a template
// parameter so that every shared-memory slot is an immediate offset from one address.
// Resident blocks the compiler must allow for: FP32 with bricks of 256 cells, 2 (128
// registers, 16 warps per SM); with 128 cells, 3; the others take what they need.
template <int P, typename T, int BZ>
constexpr int cellwise_min_blocks() {
  if (sizeof(T) == 4 && P == 2) return 512 / (32 * BZ);
  if (sizeof(T) == 4 && P == 3) return BZ == 8 ? 2 : (BZ == 4 ? 3 : 1);
  return 1;
}

// DOT (FP32): also the per-block partial sums of x . y per right-hand side, written to
// dotp[rhs * dot_stride + block] (every right-hand side, 0 where the block had no item).
template <int P, typename T, int BZ, bool DOT>
__global__ void __launch_bounds__(32 * BZ, cellwise_min_blocks<P, T, BZ>())
    k_cellwise(const ScalarArgs<T> a, const CTab<P, T> tb, const T *__restrict__ x, T *__restrict__ y, int64_t sdof,
               int nbx, int nby, int nbricks, int nitems, int nrhs, int bulk_ok, double *__restrict__ dotp,
               int dot_stride) {
  constexpr int M = P, P2 = P * P, P3 = P2 * P, M2 = M * M, M3 = M2 * M;
  using LY = CLayout<P>;
  constexpr int sX = LY::sX;
  constexpr int bx = 8, by = 4, bz = BZ, nb = bx * by * bz;
  constexpr int n0 = by * bz, n1 = bx * bz, n2 = bx * by;  // brick-boundary planes per axis
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *trz = reinterpret_cast<T *>(smem_raw);  // z traces: [cell][pt][u0, g0, u1, g1]
  T *xs = trz + LY::NT * nb;                   // x / y staging: [cell of the brick][sX]
  T *hl = xs + LY::sX * nb;                    // halo traces: [axis][side][plane][pt][u, g]
  constexpr bool STAGE = cellwise_stage<P, T>();
  constexpr bool PK = std::is_same<T, float>::value;  // packed FP32 FMAs on pairs of lines
  T *const hsy = hl + LY::NT * (n0 + n1 + n2);  // neighbour rows across y: [side][z][bx cells]
  T *const hsz = hsy + 2 * bz * bx * P3;        // neighbour rows across z: [side][y][bx cells]
  T *const hsx = hsz + 2 * by * bx * P3;        // neighbour cells across x: [side][y + by z][slot]
  // mbar[w]: x rows of warp w; mbar[nwarps]: the neighbours (one arrival per thread)
  __shared__ __align__(8) unsigned long long mbar[(32 * BZ) / 32 + 1];
  __shared__ unsigned blk_fault;  // a wait of this block gave up (read by all after a barrier)
  // DOT: x . y of the block's cells per warp and right-hand side (written by the warp's lane 0)
  __shared__ double dacc[DOT ? (32 * BZ) / 32 * 16 : 1];
  static_assert(!DOT || std::is_same<T, float>::value, "the fused dot is an FP32 form");
  auto hoff = [](int d) { return d == 0 ? 0 : (d == 1 ? LY::NT * n0 : LY::NT * (n0 + n1)); };
  const int tid = threadIdx.x;
  const int lx = tid % bx, ly = (tid / bx) % by, lz = tid / (bx * by);
  const int warp = tid >> 5, lane = tid & 31;
  if constexpr (DOT) {
    if (lane == 0)
      for (int r = 0; r < 16; ++r) dacc[warp * 16 + r] = 0.0;
  }
  constexpr int nwarps = nb >> 5;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const T *const xend = x + nrhs * sdof;
  // item -> (right-hand side, brick origin)
  auto decode = [&](int it, int &r, int &ox, int &oy, int &oz) {
    r = it / nbricks;
    const int bi = it - r * nbricks;
    const int bq = bi / nbx;
    const int ibz = bq / nby;
    ox = (bi - bq * nbx) * bx;
    oy = (bq - ibz * nby) * by;
    oz = ibz * bz;
  };
  // The next item's x rows and the neighbour cells it evaluates brick-boundary traces from
  // go to L2 one item ahead, so that its staging and halo loads hit L2 instead of DRAM:
  // by*bz rows, 2*bz rows across y, 2*by rows across z, 2*by*bz single cells across x,
  // one bulk prefetch each, spread over the even lanes of every warp. With bulk staging of
  // the next item only its rows are prefetched (its neighbours are copied one item ahead).
  auto prefetch_item = [&](int r, int px, int py, int pz, bool rows_only) {
    const T *xb = x + r * sdof;
    const int qx = min(bx, nx - px);
    const int nranges = rows_only ? by * bz : by * bz + 2 * bz + 2 * by + 2 * by * bz;
    if (tid & 1) return;
    for (int t0 = tid >> 1; t0 < nranges; t0 += nb / 2) {
      int t = t0, cy, cz, cx = px, ncx = qx;
      if (t < by * bz) {
        cy = py + t % by; cz = pz + t / by;
      } else if ((t -= by * bz) < 2 * bz) {
        cz = pz + t % bz; cy = t < bz ? py - 1 : py + by;
      } else if ((t -= 2 * bz) < 2 * by) {
        cy = py + t % by; cz = t < by ? pz - 1 : pz + bz;
      } else {
        t -= 2 * by;
        const int pl = t % (by * bz);
        cy = py + pl % by; cz = pz + pl / by; cx = t < by * bz ? px - 1 : px + bx; ncx = 1;
      }
      if (cx < 0 || cx >= nx || cy < 0 || cy >= ny || cz < 0 || cz >= nz) continue;
      dg_prefetch_l2(x, xend, xb + (cx + (int64_t)nx * (cy + (int64_t)ny * cz)) * P3, (size_t)ncx * P3 * sizeof(T));
    }
  };
  // Bulk staging applies to a whole brick inside the mesh (its rows and neighbour cells
  // then start on 16-byte boundaries: bulk_ok says x, the right-hand-side stride and nx
  // allow it).
  auto full_brick = [&](int px, int py, int pz) {
    return STAGE && bulk_ok && px + bx <= nx && py + by <= ny && pz + bz <= nz;
  };
  // words from the 16-byte boundary below cell c's first coefficient to it
  auto cell_off = [](int64_t c) { return (int)((c * P3) & 3); };
  // neighbours of brick (px, py, pz): copy unit tid (rows across y, rows across z, cells
  // across x); every thread arrives once on mbar[nwarps], announcing its copy's bytes
  auto issue_halo = [&](int r, int px, int py, int pz) {
    const T *xb = x + r * sdof;
    constexpr unsigned rb = bx * P3 * sizeof(T);
    unsigned bytes = 0;
    const T *src = x;
    T *dst = hsy;
    int t = tid;
    if (t < 2 * bz) {
      const int side = t / bz, cz = pz + t - side * bz, cy = side ? py + by : py - 1;
      if (side ? cy < ny : cy >= 0) {
        src = xb + (px + (int64_t)nx * (cy + (int64_t)ny * cz)) * P3;
        dst = hsy + t * bx * P3;
        bytes = rb;
      }
    } else if ((t -= 2 * bz) < 2 * by) {
      const int side = t / by, cy = py + t - side * by, cz = side ? pz + bz : pz - 1;
      if (side ? cz < nz : cz >= 0) {
        src = xb + (px + (int64_t)nx * (cy + (int64_t)ny * cz)) * P3;
        dst = hsz + t * bx * P3;
        bytes = rb;
      }
    } else if ((t -= 2 * by) < 2 * n0) {
      const int side = t / n0, pl = t - side * n0, cx = side ? px + bx : px - 1;
      if (side ? cx < nx : cx >= 0) {
        const int64_t c = cx + (int64_t)nx * (py + pl % by + (int64_t)ny * (pz + pl / by));
        const int o = cell_off(c);
        src = xb + c * P3 - o;
        dst = hsx + t * kHaloSlot;
        bytes = (unsigned)(((o + P3 + 3) & ~3) * sizeof(T));
      }
    }
    if (bytes) {
      mbar_arrive_expect(&mbar[nwarps], bytes);
      bulk_g2s(dst, src, bytes, &mbar[nwarps]);
    } else {
      mbar_arrive(&mbar[nwarps]);
    }
  };
  // x rows of this warp's z layer of brick (px, py, pz), issued by lane 0
  auto issue_rows = [&](int r, int px, int py, int pz) {
    const T *xb = x + r * sdof;
    constexpr unsigned rb = bx * P3 * sizeof(T);
    mbar_arrive_expect(&mbar[warp], by * rb);
    for (int ry = 0; ry < by; ++ry)
      bulk_g2s(xs + (ry + by * warp) * bx * sX, xb + (px + (int64_t)nx * (py + ry + (int64_t)ny * (pz + warp))) * P3,
               rb, &mbar[warp]);
  };
  // the same neighbour layout filled by plain loads (cells across x at offset 0), for an
  // item that is not bulk-staged
  auto fill_halo = [&](const T *xb, int px, int py, int pz) {
    constexpr int wy = 2 * bz * bx * P3, wz = 2 * by * bx * P3, wx = 2 * n0 * P3;
    for (int j = tid; j < wy + wz + wx; j += nb) {
      int t = j;
      int cx, cy, cz, e;
      T *dst;
      if (t < wy) {
        const int row = t / (bx * P3), side = row / bz;
        e = t - row * bx * P3;
        cx = px + e / P3; e -= (e / P3) * P3;
        cz = pz + row - side * bz; cy = side ? py + by : py - 1;
        dst = hsy + t;
      } else if ((t -= wy) < wz) {
        const int row = t / (bx * P3), side = row / by;
        e = t - row * bx * P3;
        cx = px + e / P3; e -= (e / P3) * P3;
        cy = py + row - side * by; cz = side ? pz + bz : pz - 1;
        dst = hsz + t;
      } else {
        t -= wz;
        const int slot = t / P3, side = slot / n0, pl = slot - side * n0;
        e = t - slot * P3;
        cy = py + pl % by; cz = pz + pl / by; cx = side ? px + bx : px - 1;
        dst = hsx + slot * kHaloSlot + e;
      }
      if (cx < 0 || cx >= nx || cy < 0 || cy >= ny || cz < 0 || cz >= nz) continue;
      *dst = __ldg(xb + (cx + (int64_t)nx * (cy + (int64_t)ny * cz)) * P3 + e);
    }
  };
  int rhs = 0, ox = 0, oy = 0, oz = 0;
  if (blockIdx.x < (unsigned)nitems) decode(blockIdx.x, rhs, ox, oy, oz);
  bool cur_bulk = false;  // this item's rows and neighbours are bulk copies in flight
  unsigned ph = 0;        // parity of the mbarrier phase the bulk items wait for
  if constexpr (STAGE) {
    if (tid == 0) {
      for (int w = 0; w <= nwarps; ++w) mbar_init(&mbar[w], w < nwarps ? 1u : (unsigned)nb);
      blk_fault = 0;
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (blockIdx.x < (unsigned)nitems && full_brick(ox, oy, oz)) {
      cur_bulk = true;
      issue_halo(rhs, ox, oy, oz);
      if (lane == 0) issue_rows(rhs, ox, oy, oz);
    }
  }
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    int nr = 0, nox = 0, noy = 0, noz = 0;
    const bool more = item + (int)gridDim.x < nitems;
    bool nxt_bulk = false;
    if (more) {
      decode(item + gridDim.x, nr, nox, noy, noz);
      nxt_bulk = full_brick(nox, noy, noz);
      prefetch_item(nr, nox, noy, noz, nxt_bulk);
    }
    const int nax = min(bx, nx - ox), nay = min(by, ny - oy), naz = min(bz, nz - oz);
    const T *xr = x + rhs * sdof;
    T *yr = y + rhs * sdof;
    const int gx = ox + lx, gy = oy + ly, gz = oz + lz;
    const bool act = lx < nax && ly < nay && lz < naz;
    static_assert(nwarps == bz, "one z layer of the brick per warp");
    bool waited = true;  // false when a bulk-copy wait gave up
    if constexpr (STAGE) {
      if (cur_bulk) {
        waited = mbar_wait(&mbar[nwarps], ph);
      } else {
        fill_halo(xr, ox, oy, oz);
        __syncthreads();
      }
    }
    // weighted traces of the neighbours across the brick boundary, one face per thread
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
      int sp;          // its row (across y or z) or slot (across x) in the neighbour staging
      bool ok;
      if (d == 0) {
        const int py = p % by, pz = p / by;
        cy = oy + py; cz = oz + pz; cx = side ? ox + bx : ox - 1;
        ok = py < nay && pz < naz && (side ? ox + bx < nx : ox > 0);
        sp = side * n0 + p;
      } else if (d == 1) {
        const int px = p % bx, pz = p / bx;
        cx = ox + px; cz = oz + pz; cy = side ? oy + by : oy - 1;
        ok = px < nax && pz < naz && (side ? oy + by < ny : oy > 0);
        sp = side * bz + pz;
      } else {
        const int px = p % bx, py = p / bx;
        cx = ox + px; cy = oy + py; cz = side ? oz + bz : oz - 1;
        ok = px < nax && py < nay && (side ? oz + bz < nz : oz > 0);
        sp = side * by + py;
      }
      if (!ok) continue;
      const int64_t c = cx + (int64_t)nx * (cy + (int64_t)ny * cz);
      const T *src;
      if constexpr (STAGE)
        src = d == 0 ? hsx + sp * kHaloSlot + (cur_bulk ? cell_off(c) : 0)
                     : (d == 1 ? hsy : hsz) + sp * bx * P3 + (cx - ox) * P3;
      else
        src = xr + c * P3;
      T *dst = hl + hoff(d) + (side * nd + p) * 2 * M2;
      // strides of the normal direction and of the two tangential directions in the
      // neighbour's GLL coefficients (j0 + p (j1 + p j2))
      const int stn = d == 0 ? 1 : (d == 1 ? P : P2);
      const int st1 = d == 0 ? P : 1;
      const int st2 = d == 2 ? P : P2;
      halo_trace<P, T, STAGE>(src, tb, dst, stn, st1, st2, side);
    }
    // x: warp w's rows are those of its own cells (z layer w of the brick): bulk-copied,
    // or loaded here coalesced
    if (STAGE && cur_bulk) {
      waited &= mbar_wait(&mbar[warp], ph);
    } else {
      for (int ry = 0; ry < by; ++ry) {
        const int rz = warp, row = ry + by * rz;
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
      __syncwarp();
    }
    // own cell: weighted Gauss-point values u~ (interpolation tables carry the weights)
    T u[M3], R[M3];
#pragma unroll
    for (int q = 0; q < M3; ++q) u[q] = T(0);  // lanes outside the mesh take part in the shuffles
    if (act) {
      T xl[P3];
#pragma unroll
      for (int i = 0; i < P3; ++i) xl[i] = xs[tid * sX + i];
      T t1[P2 * M];  // [j2][j1][q0]
#pragma unroll
      for (int jj = 0; jj < P2; ++jj)
#pragma unroll
        for (int q = 0; q < M; ++q) {
          T s = tb.iw[q * P] * xl[jj * P];
#pragma unroll
          for (int j = 1; j < P; ++j) s = fma(tb.iw[q * P + j], xl[jj * P + j], s);
          t1[jj * M + q] = s;
        }
      T t2[P * M2];  // [j2][q1][q0]
#pragma unroll
      for (int j2 = 0; j2 < P; ++j2)
        sweep<M, P, 1, M, PK>(t2 + j2 * M2, M, t1 + j2 * P * M, M, tb.iw, P, 1);
      sweep<M, P, M, M, PK>(u, M2, t2, M2, tb.iw, P, 1);
    }
    if constexpr (STAGE) {
      // the neighbour staging was read through the generic proxy: order that before the
      // next item's bulk copies into it, which are issued after this barrier
      fence_proxy_async();
      if (!waited) blk_fault = 1u;
      __syncthreads();
      if (blk_fault) {
        // a bulk copy did not complete within the time limit (the fault word records it):
        // wait once more, bounded, for the copies in flight, then leave
        mbar_wait(&mbar[nwarps], ph);
        mbar_wait(&mbar[warp], ph);
        return;
      }
      if (cur_bulk) ph ^= 1u;
      if (nxt_bulk) issue_halo(nr, nox, noy, noz);
    } else {
      __syncthreads();
    }
    // x and y axes: a warp spans 8 x 4 cells of one z layer, so the x and y neighbours are
    // lanes +-1 and +-8. Per tensor line: the four weighted traces, the neighbours' pairs by
    // shuffles (the halo trace at the brick boundary), the axis's line operator (stiffness,
    // own face sides, on axis 0 the mass) and the neighbour coupling; all lanes take part.
    auto axis_xy = [&](auto Dc) {
      constexpr int D = decltype(Dc)::value;
      constexpr unsigned full = 0xffffffffu;
      constexpr int dl = D == 0 ? 1 : bx;
      constexpr int bd = D == 0 ? bx : by;
      constexpr int nd = D == 0 ? n0 : n1;
      const int gc = D == 0 ? gx : gy;
      const int nlim = D == 0 ? nx : ny;
      const int lc = D == 0 ? lx : ly;
      const int p = D == 0 ? ly + by * lz : lx + bx * lz;
      const bool lo_bnd = gc == 0, hi_bnd = gc + 1 >= nlim;
      const T *hlo = hl + hoff(D) + p * 2 * M2, *hhi = hl + hoff(D) + (nd + p) * 2 * M2;
#pragma unroll
      for (int t2 = 0; t2 < M; ++t2)
#pragma unroll
        for (int t1 = 0; t1 < M; ++t1) {
          const int pt = t1 + M * t2;
          if constexpr (PK && D == 1) {
            // lines (t1, t2) and (t1 + 1, t2), neighbours in x, as one packed pair
            if (t1 & 1) continue;
            if (t1 + 1 < M) {
              float2 v2[M];
#pragma unroll
              for (int r = 0; r < M; ++r) v2[r] = pk(u[lidx<M, D>(r, t1, t2)], u[lidx<M, D>(r, t1 + 1, t2)]);
              float2 tr2[4];
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                float2 s = __fmul2_rn(bc(tb.te[k][0]), v2[0]);
#pragma unroll
                for (int r = 1; r < M; ++r) s = __ffma2_rn(bc(tb.te[k][r]), v2[r], s);
                tr2[k] = s;
              }
              T huA = __shfl_down_sync(full, tr2[0].x, dl), huB = __shfl_down_sync(full, tr2[0].y, dl);
              T hgA = __shfl_down_sync(full, tr2[1].x, dl), hgB = __shfl_down_sync(full, tr2[1].y, dl);
              T luA = __shfl_up_sync(full, tr2[2].x, dl), luB = __shfl_up_sync(full, tr2[2].y, dl);
              T lgA = __shfl_up_sync(full, tr2[3].x, dl), lgB = __shfl_up_sync(full, tr2[3].y, dl);
              if (lc == bd - 1) {
                load2(hhi + 2 * pt, huA, hgA);
                load2(hhi + 2 * (pt + 1), huB, hgB);
              }
              if (lc == 0) {
                load2(hlo + 2 * pt, luA, lgA);
                load2(hlo + 2 * (pt + 1), luB, lgB);
              }
              const float2 hu = pk(huA, huB), hg = pk(hgA, hgB), lu = pk(luA, luB), lg = pk(lgA, lgB);
#pragma unroll
              for (int q = 0; q < M; ++q) {
                float2 s = __ffma2_rn(bc(tb.K[D][q * M]), v2[0],
                                      pk(R[lidx<M, D>(q, t1, t2)], R[lidx<M, D>(q, t1 + 1, t2)]));
#pragma unroll
                for (int r = 1; r < M; ++r) s = __ffma2_rn(bc(tb.K[D][q * M + r]), v2[r], s);
                if (!hi_bnd) s = __ffma2_rn(bc(tb.na[D][1][q]), hu, __ffma2_rn(bc(tb.nbv[D][1][q]), hg, s));
                if (!lo_bnd) s = __ffma2_rn(bc(tb.na[D][0][q]), lu, __ffma2_rn(bc(tb.nbv[D][0][q]), lg, s));
                R[lidx<M, D>(q, t1, t2)] = s.x;
                R[lidx<M, D>(q, t1 + 1, t2)] = s.y;
              }
              continue;
            }
          }
          T v[M];
#pragma unroll
          for (int r = 0; r < M; ++r) v[r] = u[lidx<M, D>(r, t1, t2)];
          T tr[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            T s = tb.te[k][0] * v[0];
#pragma unroll
            for (int r = 1; r < M; ++r) s = fma(tb.te[k][r], v[r], s);
            tr[k] = s;
          }
          // upper neighbour's lower-face pair, lower neighbour's upper-face pair
          T hu = __shfl_down_sync(full, tr[0], dl), hg = __shfl_down_sync(full, tr[1], dl);
          T lu = __shfl_up_sync(full, tr[2], dl), lg = __shfl_up_sync(full, tr[3], dl);
          if (lc == bd - 1) load2(hhi + 2 * pt, hu, hg);
          if (lc == 0) load2(hlo + 2 * pt, lu, lg);
#pragma unroll
          for (int q = 0; q < M; ++q) {
            T s = D == 0 ? tb.K[D][q * M] * v[0] : fma(tb.K[D][q * M], v[0], R[lidx<M, D>(q, t1, t2)]);
#pragma unroll
            for (int r = 1; r < M; ++r) s = fma(tb.K[D][q * M + r], v[r], s);
            if (!hi_bnd) s = fma(tb.na[D][1][q], hu, fma(tb.nbv[D][1][q], hg, s));
            if (!lo_bnd) s = fma(tb.na[D][0][q], lu, fma(tb.nbv[D][0][q], lg, s));
            R[lidx<M, D>(q, t1, t2)] = s;
          }
        }
      // own side of a domain-boundary face
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        if (s ? hi_bnd : lo_bnd) {
#pragma unroll
          for (int t2 = 0; t2 < M; ++t2)
#pragma unroll
            for (int t1 = 0; t1 < M; ++t1)
#pragma unroll
              for (int q = 0; q < M; ++q) {
                T acc = R[lidx<M, D>(q, t1, t2)];
#pragma unroll
                for (int r = 0; r < M; ++r) acc = fma(tb.corr[D][s][q * M + r], u[lidx<M, D>(r, t1, t2)], acc);
                R[lidx<M, D>(q, t1, t2)] = acc;
              }
        }
      }
    };
    // z axis: neighbours in the warps of the adjacent z layers, exchanged through shared
    // memory: publish the weighted traces, line operator and boundary correction, barrier,
    // then the neighbours' coupling. A face on the brick boundary is read by no cell of the
    // brick, so its slots take the neighbour's trace from the halo instead.
    auto axis_z = [&]() {
      constexpr int D = 2;
      constexpr int bd = bz, nd = n2, nstep = bx * by;
      const int gc = gz, nlim = nz, lc = lz;
      if (act) {
#pragma unroll
        for (int t2 = 0; t2 < M; ++t2)
#pragma unroll
          for (int t1 = 0; t1 < M; ++t1) {
            const int pt = t1 + M * t2;
            if constexpr (PK) {
              // lines (t1, t2) and (t1 + 1, t2), neighbours in x, as one packed pair
              if (t1 & 1) continue;
              if (t1 + 1 < M) {
                float2 v2[M];
#pragma unroll
                for (int r = 0; r < M; ++r) v2[r] = pk(u[lidx<M, D>(r, t1, t2)], u[lidx<M, D>(r, t1 + 1, t2)]);
                float2 tr2[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                  float2 s = __fmul2_rn(bc(tb.te[k][0]), v2[0]);
#pragma unroll
                  for (int r = 1; r < M; ++r) s = __ffma2_rn(bc(tb.te[k][r]), v2[r], s);
                  tr2[k] = s;
                }
                store4(trz + tid * LY::NT + 4 * pt, tr2[0].x, tr2[1].x, tr2[2].x, tr2[3].x);
                store4(trz + tid * LY::NT + 4 * (pt + 1), tr2[0].y, tr2[1].y, tr2[2].y, tr2[3].y);
#pragma unroll
                for (int q = 0; q < M; ++q) {
                  float2 s = __ffma2_rn(bc(tb.K[D][q * M]), v2[0],
                                        pk(R[lidx<M, D>(q, t1, t2)], R[lidx<M, D>(q, t1 + 1, t2)]));
#pragma unroll
                  for (int r = 1; r < M; ++r) s = __ffma2_rn(bc(tb.K[D][q * M + r]), v2[r], s);
                  R[lidx<M, D>(q, t1, t2)] = s.x;
                  R[lidx<M, D>(q, t1 + 1, t2)] = s.y;
                }
                continue;
              }
            }
            T v[M];
#pragma unroll
            for (int r = 0; r < M; ++r) v[r] = u[lidx<M, D>(r, t1, t2)];
            T tr[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              T s = tb.te[k][0] * v[0];
#pragma unroll
              for (int r = 1; r < M; ++r) s = fma(tb.te[k][r], v[r], s);
              tr[k] = s;
            }
            store4(trz + tid * LY::NT + 4 * pt, tr[0], tr[1], tr[2], tr[3]);
#pragma unroll
            for (int q = 0; q < M; ++q) {
              T s = fma(tb.K[D][q * M], v[0], R[lidx<M, D>(q, t1, t2)]);
#pragma unroll
              for (int r = 1; r < M; ++r) s = fma(tb.K[D][q * M + r], v[r], s);
              R[lidx<M, D>(q, t1, t2)] = s;
            }
          }
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          if (s ? gc + 1 >= nlim : gc == 0) {
#pragma unroll
            for (int t2 = 0; t2 < M; ++t2)
#pragma unroll
              for (int t1 = 0; t1 < M; ++t1)
#pragma unroll
                for (int q = 0; q < M; ++q) {
                  T acc = R[lidx<M, D>(q, t1, t2)];
#pragma unroll
                  for (int r = 0; r < M; ++r) acc = fma(tb.corr[D][s][q * M + r], u[lidx<M, D>(r, t1, t2)], acc);
                  R[lidx<M, D>(q, t1, t2)] = acc;
                }
          }
        }
        const int p = lx + bx * ly;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          if (side ? lc == bd - 1 : lc == 0) {
            const T *h = hl + hoff(D) + (side * nd + p) * 2 * M2;
#pragma unroll
            for (int pt = 0; pt < M2; ++pt) {
              T hu, hg;
              load2(h + 2 * pt, hu, hg);
              store2(trz + tid * LY::NT + 4 * pt + 2 * side, hu, hg);
            }
          }
        }
      }
      __syncthreads();
      if (act) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          if (s ? gc + 1 >= nlim : gc == 0) continue;  // domain boundary: no neighbour
          const bool inb = s ? lc + 1 < bd : lc > 0;
          // neighbour trace pair of face point pt at nsrc[4 pt]: the neighbour's lower (s = 1) or
          // upper (s = 0) face, or this cell's outward slots holding the halo trace
          const T *nsrc = trz + (inb ? (s ? tid + nstep : tid - nstep) : tid) * LY::NT + (s == inb ? 0 : 2);
#pragma unroll
          for (int t2 = 0; t2 < M; ++t2)
#pragma unroll
            for (int t1 = 0; t1 < M; ++t1) {
              const int pt = t1 + M * t2;
              if constexpr (PK) {
                if (t1 & 1) continue;
                if (t1 + 1 < M) {
                  T unA, dnA, unB, dnB;
                  load2(nsrc + 4 * pt, unA, dnA);
                  load2(nsrc + 4 * (pt + 1), unB, dnB);
                  const float2 un2 = pk(unA, unB), dn2 = pk(dnA, dnB);
#pragma unroll
                  for (int r = 0; r < M; ++r) {
                    const float2 a2 = __ffma2_rn(bc(tb.na[D][s][r]), un2,
                                                 __ffma2_rn(bc(tb.nbv[D][s][r]), dn2,
                                                            pk(R[lidx<M, D>(r, t1, t2)], R[lidx<M, D>(r, t1 + 1, t2)])));
                    R[lidx<M, D>(r, t1, t2)] = a2.x;
                    R[lidx<M, D>(r, t1 + 1, t2)] = a2.y;
                  }
                  continue;
                }
              }
              T un, dn;
              load2(nsrc + 4 * pt, un, dn);
#pragma unroll
              for (int r = 0; r < M; ++r)
                R[lidx<M, D>(r, t1, t2)] =
                    fma(tb.na[D][s][r], un, fma(tb.nbv[D][s][r], dn, R[lidx<M, D>(r, t1, t2)]));
            }
        }
      }
    };
    axis_xy(std::integral_constant<int, 0>{});
    axis_xy(std::integral_constant<int, 1>{});
    axis_z();
    double cell_dot = 0.0;  // DOT: x . y of this thread's cell
    // transposed interpolation to the GLL coefficients, staged in this warp's own rows of xs
    // for a coalesced store
    if (act) {
      T t2[P * M2];  // [j2][q1][q0]
      sweep<P, M, M, M, PK>(t2, M2, R, M2, tb.it, 1, P);
      T t1[P2 * M];  // [j2][j1][q0]
#pragma unroll
      for (int j2 = 0; j2 < P; ++j2)
        sweep<P, M, 1, M, PK>(t1 + j2 * P * M, M, t2 + j2 * M2, M, tb.it, 1, P);
      T yv[P3];
#pragma unroll
      for (int jj = 0; jj < P2; ++jj)
#pragma unroll
        for (int j = 0; j < P; ++j) {
          T s = tb.it[j] * t1[jj * M];
#pragma unroll
          for (int q = 1; q < M; ++q) s = fma(tb.it[q * P + j], t1[jj * M + q], s);
          yv[jj * P + j] = s;
        }
      if constexpr (DOT) {
        // this cell's x . y, x still in the staging slots that y is about to take
        DotPair dp;
#pragma unroll
        for (int i = 0; i + 1 < P3; i += 2)
          dp.add(pk(xs[tid * sX + i], xs[tid * sX + i + 1]), pk(yv[i], yv[i + 1]));
        if constexpr (P3 & 1) dp.add(pk(xs[tid * sX + P3 - 1], 0.f), pk(yv[P3 - 1], 0.f));
        cell_dot = dp.value();
      }
#pragma unroll
      for (int i = 0; i < P3; ++i) xs[tid * sX + i] = yv[i];
    }
    if constexpr (DOT) {
      // the warp's sum of its cells' x . y, added to its slot of this item's right-hand side
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cell_dot += __shfl_down_sync(0xffffffffu, cell_dot, o);
      if (lane == 0) dacc[warp * 16 + rhs] += cell_dot;
    }
    // each warp stores the rows it staged itself: a warp barrier suffices, and the next
    // item's staging by the same warp reuses the same rows
    __syncwarp();
    for (int ry = 0; ry < by; ++ry) {
      const int rz = warp, row = ry + by * rz;
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
    // this warp's rows of the next item as a bulk copy, once the warp's reads of them are
    // ordered before the copy's writes
    if constexpr (STAGE) {
      if (nxt_bulk) {
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) issue_rows(nr, nox, noy, noz);
      }
    }
    if (more) {
      rhs = nr;
      ox = nox;
      oy = noy;
      oz = noz;
      cur_bulk = nxt_bulk;
    }
    // no block barrier here: the next item's first shared-memory writes are this warp's own
    // staging rows, the halo traces, whose last readers all passed the axis-2 barrier, and
    // the neighbour staging, whose last readers passed the first barrier
  }
  if constexpr (DOT) {
    // the block's partial sums, over its warps in a fixed order
    __syncthreads();
    for (int r = tid; r < nrhs; r += nb) {
      double v = 0.0;
      for (int w = 0; w < nwarps; ++w) v += dacc[w * 16 + r];
      dotp[(int64_t)r * dot_stride + blockIdx.x] = v;
    }
  }
}

template <int P, typename T, int BZ, bool DOT>
cudaError_t run_k(const ScalarArgs<T> &a, const HostTables &ht, const T *x, T *y, int nrhs, int64_t sdof,
                  cudaStream_t s, const cudaEvent_t *ev, int *grid_out, LaunchInfo *q, double *dotp, int dot_stride) {
  constexpr int bx = 8, by = 4, bz = BZ, nb = bx * by * bz;
  const CTab<P, T> tb = make_tab<P, T>(a, ht);
  const size_t sm = cellwise_words<P>(bx, by, bz, cellwise_stage<P, T>()) * sizeof(T);
  auto k = k_cellwise<P, T, BZ, DOT>;
  cudaError_t e;
  if (sm > 48 * 1024 && (e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
    return e;
  int per_sm = 0, dev = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, nb, sm)) != cudaSuccess) return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int64_t nbx = (a.nx + bx - 1) / bx, nby = (a.ny + by - 1) / by, nbz = (a.nz + bz - 1) / bz;
  const int64_t nbricks = nbx * nby * nbz;
  const int64_t nitems = (int64_t)nrhs * nbricks;
  if (nitems > INT_MAX) return cudaErrorInvalidValue;  // work items are decoded in 32 bits
  int64_t grid = (int64_t)(per_sm > 0 ? per_sm : 1) * sms;
  if (grid > nitems) grid = nitems;
  if (DOT && grid > dot_stride) return cudaErrorInvalidValue;  // one partial per block and rhs
  if (grid_out) *grid_out = (int)grid;
  if (q) {
    q->blocks = grid;
    q->threads = nb;
    q->blocks_per_sm = per_sm;
    q->items = nitems;
    return cudaSuccess;
  }
  if (ev) cudaEventRecord(ev[0], s);
  // bulk staging needs every brick row and neighbour span on a 16-byte boundary
  const int bulk_ok = cellwise_stage<P, T>() && (reinterpret_cast<uintptr_t>(x) & 15) == 0 && sdof % 4 == 0 &&
                      a.nx % 4 == 0;
  k<<<(unsigned)grid, nb, sm, s>>>(a, tb, x, y, sdof, (int)nbx, (int)nby, (int)nbricks, (int)nitems, nrhs, bulk_ok,
                                   dotp, dot_stride);
  if (ev) {
    cudaEventRecord(ev[1], s);
    cudaEventRecord(ev[2], s);
    cudaEventRecord(ev[3], s);
  }
  return cudaGetLastError();
}

template <int P, typename T, int BZ>
cudaError_t run(const ScalarArgs<T> &a, const HostTables &ht, const T *x, T *y, int nrhs, int64_t sdof,
                cudaStream_t s, const cudaEvent_t *ev, int *grid_out, LaunchInfo *q, double *dotp, int dot_stride) {
  if constexpr (std::is_same<T, float>::value) {
    if (dotp) return run_k<P, T, BZ, true>(a, ht, x, y, nrhs, sdof, s, ev, grid_out, q, dotp, dot_stride);
  } else {
    if (dotp) return cudaErrorInvalidValue;  // the fused dot is an FP32 form
  }
  return run_k<P, T, BZ, false>(a, ht, x, y, nrhs, sdof, s, ev, grid_out, q, nullptr, 0);
}

}  // namespace dgc

// Bricks of 8 x 4 x bz cells: `cells` = 64, 128 or 256 threads per block.
static int cellwise_bz(int cells) { return cells == 64 ? 2 : (cells == 128 ? 4 : (cells == 256 ? 8 : 0)); }

size_t cellwise_smem_bytes(int p, int cells, int es) {
  const int bz = cellwise_bz(cells);
  if (!bz) return 0;
  switch (p) {
    case 2: return dgc::cellwise_words<2>(8, 4, bz, false) * es;
    case 3: return dgc::cellwise_words<3>(8, 4, bz, es == 4) * es;
    default: return 0;
  }
}

template <int P, typename T>
static cudaError_t run_bz(int bz, const ScalarArgs<T> &a, const HostTables &ht, const T *x, T *y, int nrhs,
                          int64_t sdof, cudaStream_t s, const cudaEvent_t *ev, int *grid_out, LaunchInfo *q,
                          double *dotp, int dot_stride) {
  switch (bz) {
    case 2: return dgc::run<P, T, 2>(a, ht, x, y, nrhs, sdof, s, ev, grid_out, q, dotp, dot_stride);
    case 4: return dgc::run<P, T, 4>(a, ht, x, y, nrhs, sdof, s, ev, grid_out, q, dotp, dot_stride);
    case 8: return dgc::run<P, T, 8>(a, ht, x, y, nrhs, sdof, s, ev, grid_out, q, dotp, dot_stride);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_cellwise_apply(int p, const ScalarArgs<T> &a, const HostTables &ht, const T *x, T *y, int nrhs,
                                  int64_t sdof, int cells, cudaStream_t s, const cudaEvent_t *ev, int *grid_out,
                                  LaunchInfo *q, double *dotp, int dot_stride) {
  if (ht.m != p || ht.p != p) return cudaErrorInvalidValue;
  const int bz = cellwise_bz(cells);
  switch (p) {
    case 2: return run_bz<2, T>(bz, a, ht, x, y, nrhs, sdof, s, ev, grid_out, q, dotp, dot_stride);
    case 3: return run_bz<3, T>(bz, a, ht, x, y, nrhs, sdof, s, ev, grid_out, q, dotp, dot_stride);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_cellwise_apply<float>(int, const ScalarArgs<float> &, const HostTables &, const float *,
                                                  float *, int, int64_t, int, cudaStream_t, const cudaEvent_t *, int *,
                                                  LaunchInfo *, double *, int);
template cudaError_t launch_cellwise_apply<double>(int, const ScalarArgs<double> &, const HostTables &,
                                                   const double *, double *, int, int64_t, int, cudaStream_t,
                                                   const cudaEvent_t *, int *, LaunchInfo *, double *, int);

extern "C" dg_status dg_device_faults(int clear, unsigned *faults) {
  if (!faults) return dg_record_error(DG_ERR_INVALID_ARG);
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, dgc::g_cellwise_fault, sizeof v) != cudaSuccess) return dg_record_error(DG_ERR_CUDA);
  if (clear && v) {
    const unsigned zero = 0;
    if (cudaMemcpyToSymbol(dgc::g_cellwise_fault, &zero, sizeof zero) != cudaSuccess)
      return dg_record_error(DG_ERR_CUDA);
  }
  *faults = v;
  return DG_OK;
}
