// C ABI of libdg: object lifetimes, validation, table upload, geometry precompute and
// kernel dispatch. All arithmetic of an apply runs in the CUDA kernels.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <type_traits>
#include <vector>

#include "dg_internal.h"

namespace {

thread_local dg_status g_last = DG_OK;

dg_status fail(dg_status s) {
  g_last = s;
  return s;
}

#define CK(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return fail(DG_ERR_CUDA); \
  } while (0)

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

int dg_device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1) {
    cudaGetLastError();
    return 1;
  }
  return sms;
}

extern "C" {

const char *dg_status_string(dg_status s) {
  switch (s) {
    case DG_OK: return "DG_OK";
    case DG_ERR_INVALID_ARG: return "DG_ERR_INVALID_ARG";
    case DG_ERR_UNSUPPORTED: return "DG_ERR_UNSUPPORTED";
    case DG_ERR_OOM: return "DG_ERR_OOM";
    case DG_ERR_CUDA: return "DG_ERR_CUDA";
    case DG_ERR_NOT_CONVERGED: return "DG_ERR_NOT_CONVERGED";
    case DG_ERR_TIMEOUT: return "DG_ERR_TIMEOUT";
  }
  return "DG_ERR_UNKNOWN";
}

dg_status dg_get_last_error(void) {
  dg_status s = g_last;
  g_last = DG_OK;
  return s;
}

dg_status dg_mesh_create(int nx, int ny, int nz, const double *vertices, dg_mesh **out) {
  if (!out || nx < 1 || ny < 1 || nz < 1) return fail(DG_ERR_INVALID_ARG);
  if ((int64_t)nx * ny * nz > (int64_t)1 << 31) return fail(DG_ERR_UNSUPPORTED);
  dg_mesh *m = new (std::nothrow) dg_mesh;
  if (!m) return fail(DG_ERR_OOM);
  m->nx = nx; m->ny = ny; m->nz = nz;
  m->affine = (vertices == nullptr);
  if (vertices) {
    size_t n = (size_t)(nx + 1) * (ny + 1) * (nz + 1) * 3;
    try {
      m->verts.assign(vertices, vertices + n);
    } catch (...) {
      delete m;
      return fail(DG_ERR_OOM);
    }
  }
  *out = m;
  return DG_OK;
}

dg_status dg_mesh_destroy(dg_mesh *mesh) {
  delete mesh;
  return DG_OK;
}

}  // extern "C"

static void free_op(dg_operator *o) {
  if (o && o->d_antab) cudaFree(o->d_antab);
  if (!o) return;
  void *ptrs[] = {o->d_tab, o->d_verts, o->d_gamma, o->d_cellvol, o->d_gvol, o->d_gface,
                  o->d_rvol, o->d_tr, o->d_fres, o->d_xh, o->d_yh, o->d_tr2,
                  o->d_tab_df, o->d_gvol_df, o->d_gface_df};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (cudaEvent_t e : o->prof_ev) cudaEventDestroy(e);
  for (cudaEvent_t e : o->hs_ev) cudaEventDestroy(e);
  if (o->hs_copy) cudaStreamDestroy(o->hs_copy);
  dg_solver_release(o);
  delete o;
}

template <typename T>
static void fill_devtables(const HostTables &h, DevTables<T> &d) {
  memset(&d, 0, sizeof(d));
  for (int q = 0; q < h.m; ++q)
    for (int j = 0; j < h.p; ++j) d.interp[q * h.p + j] = (T)h.interp[q * h.p + j];
  for (int i = 0; i < h.m * h.m; ++i) d.dcol[i] = (T)h.dcol[i];
  for (int i = 0; i < h.m; ++i) {
    d.e0[i] = (T)h.e0[i]; d.e1[i] = (T)h.e1[i];
    d.d0[i] = (T)h.d0[i]; d.d1[i] = (T)h.d1[i];
    d.w[i] = (T)h.gauss_w[i];
    d.s[i] = (T)h.gauss_s[i];
  }
  for (int j = 0; j < h.p; ++j) {
    d.gd0[j] = (T)h.gd0[j];
    d.gd1[j] = (T)h.gd1[j];
  }
  for (int q = 0; q < h.m; ++q)
    for (int j = 0; j < h.pp; ++j) d.interp_p[q * h.pp + j] = (T)h.interp_p[q * h.pp + j];
}

template <typename T>
static ScalarArgs<T> scalar_args(const dg_operator *o, bool transpose) {
  ScalarArgs<T> a;
  memset(&a, 0, sizeof(a));
  a.nx = o->nx; a.ny = o->ny; a.nz = o->nz;
  a.ncell = o->ncell;
  a.nface = o->nface;
  for (int i = 0; i < 4; ++i) a.face_off[i] = o->face_off[i];
  a.tab = (const DevTables<T> *)o->d_tab;
  const double h[3] = {1.0 / o->nx, 1.0 / o->ny, 1.0 / o->nz};
  const double V = h[0] * h[1] * h[2];
  for (int d = 0; d < 3; ++d) {
    a.vol_g[d] = (T)(V / (h[d] * h[d]));
    a.face_b[d] = (T)(V / (h[d] * h[d]));
    a.face_pw[d] = (T)(o->gamma_axis[d] * V / h[d]);
    a.face_area[d] = (T)(V / h[d]);
  }
  a.vol_m = (T)(o->c * V);
  if constexpr (std::is_same<T, df64>::value) a.vol = df64(1.0 / ((double)o->nx * o->ny * o->nz));
  else a.vol = T(1) / (T(o->nx) * T(o->ny) * T(o->nz));  // as the kernels computed it
  a.gvol = (const T *)o->d_gvol;
  a.gface = (const T *)o->d_gface;
  a.verts = o->d_verts;
  a.gamma_face = o->d_gamma;
  a.c = o->c;
  a.kappa_vol = (const io_t<T> *)o->kappa_vol;
  a.kappa_face = (const io_t<T> *)o->kappa_face;
  a.dmask = o->dmask;
  a.sc = (T)(transpose ? o->theta : -1.0);
  a.ss = (T)(transpose ? -1.0 : o->theta);
  return a;
}

static void default_blocking(dg_operator *o) {
  const int M3 = o->m * o->m * o->m, M2 = o->m * o->m;
  o->cpb = 256 / M3 > 0 ? 256 / M3 : 1;
  o->fpb = 256 / M2 > 0 ? 256 / M2 : 1;
  const int lines = o->p * o->p;  // threads per cell of the fused kernel
  o->tile = 256 / lines > 0 ? 256 / lines : 1;
  // cellwise bricks, the measured best: 8 x 4 x 8 cells for FP32 Q2, 8 x 4 x 4 otherwise
  o->brick = (o->precision == DG_FP32 && o->p == 3) ? 256 : 128;
}

static bool fused_ok(const dg_operator *o) {
  return o->problem == DG_SCALAR && o->geo == GEO_AFFINE && o->kappa_vol == nullptr && o->m == o->p;
}

static bool cellwise_ok(const dg_operator *o) { return fused_ok(o) && o->p <= 3; }

// double-float kernels: FP64 scalar operators (any geometry, kappa; recomputed geometry
// and the adjoint run through the double-float adjoint kernels) and FP64 Stokes operators
static bool df64_ok(const dg_operator *o) {
  return o->precision == DG_FP64 && !o->aniso && (o->problem == DG_SCALAR || o->geo == GEO_AFFINE);
}

// Kernel arguments of the double-float variant: its tables and stored geometry.
static ScalarArgs<df64> df64_args(const dg_operator *op, bool transpose) {
  ScalarArgs<df64> a = scalar_args<df64>(op, transpose);
  a.tab = (const DevTables<df64> *)op->d_tab_df;
  a.gvol = (const df64 *)op->d_gvol_df;
  a.gface = (const df64 *)op->d_gface_df;
  return a;
}

// Tables and stored geometry of the operator as double-float (DG_VARIANT_DF64), converted
// once from the FP64 ones.
static dg_status ensure_df64(dg_operator *o) {
  if (o->d_tab_df) return DG_OK;
  DevTables<df64> t;
  fill_devtables(o->ht, t);
  const int M = o->m, M2 = M * M, M3 = M2 * M;
  void *tab = nullptr, *gv = nullptr, *gf = nullptr;
  auto undo = [&](dg_status st) {
    cudaGetLastError();
    for (void *q : {tab, gv, gf})
      if (q) cudaFree(q);
    return fail(st);
  };
  if (cudaMalloc(&tab, sizeof(t)) != cudaSuccess) return undo(DG_ERR_OOM);
  if (cudaMemcpy(tab, &t, sizeof(t), cudaMemcpyHostToDevice) != cudaSuccess) return undo(DG_ERR_CUDA);
  if (o->geo == GEO_STORED) {
    const int64_t nv = o->ncell * 7 * M3, nf = o->nface * 7 * M2;
    if (cudaMalloc(&gv, nv * sizeof(df64)) != cudaSuccess || cudaMalloc(&gf, nf * sizeof(df64)) != cudaSuccess)
      return undo(DG_ERR_OOM);
    if (convert_to_df64((const double *)o->d_gvol, (df64 *)gv, nv, 0) != cudaSuccess ||
        convert_to_df64((const double *)o->d_gface, (df64 *)gf, nf, 0) != cudaSuccess ||
        cudaStreamSynchronize(0) != cudaSuccess)
      return undo(DG_ERR_CUDA);
  }
  o->d_tab_df = tab;
  o->d_gvol_df = gv;
  o->d_gface_df = gf;
  return DG_OK;
}

static const size_t kMaxSmemBlock = 227 * 1024;  // opt-in shared memory per block

static bool variant_ok(const dg_operator *o, int v) {
  return v == DG_VARIANT_THREE_KERNEL || (v == DG_VARIANT_FUSED && fused_ok(o)) ||
         (v == DG_VARIANT_CELLWISE && cellwise_ok(o)) || (v == DG_VARIANT_DF64 && df64_ok(o));
}

static int resolve_variant(const dg_operator *o, int v) {
  if (v == DG_VARIANT_AUTO) {
    if (o->precision == DG_FP32 && cellwise_ok(o)) return DG_VARIANT_CELLWISE;
    return (o->precision == DG_FP32 && fused_ok(o)) ? DG_VARIANT_FUSED : DG_VARIANT_THREE_KERNEL;
  }
  return v;
}

extern "C" {

// any_recompute: also FP32 with recomputed trilinear geometry (the anisotropic operator,
// whose kernels recompute it themselves, uses the isotropic one only for its bookkeeping).
static dg_status create_impl(const dg_mesh *mesh, int degree, int quad_points_1d, const dg_penalty *pen,
                             const dg_coefficients *co, dg_operator **out, bool any_recompute);

dg_status dg_operator_create(const dg_mesh *mesh, int degree, int quad_points_1d, const dg_penalty *pen,
                             const dg_coefficients *co, dg_operator **out) {
  return create_impl(mesh, degree, quad_points_1d, pen, co, out, false);
}

static dg_status create_impl(const dg_mesh *mesh, int degree, int quad_points_1d, const dg_penalty *pen,
                             const dg_coefficients *co, dg_operator **out, bool any_recompute) {
  if (!mesh || !pen || !co || !out) return fail(DG_ERR_INVALID_ARG);
  *out = nullptr;
  if (degree < 1) return fail(DG_ERR_INVALID_ARG);
  if (degree > 5) return fail(DG_ERR_UNSUPPORTED);
  const int m = quad_points_1d == 0 ? degree + 1 : quad_points_1d;
  if (m < degree + 1) return fail(DG_ERR_INVALID_ARG);
  if (m > degree + 2 || (m != degree + 1 && co->problem == DG_STOKES)) return fail(DG_ERR_UNSUPPORTED);
  if (co->problem != DG_SCALAR && co->problem != DG_STOKES) return fail(DG_ERR_INVALID_ARG);
  if (co->problem == DG_STOKES && (degree < 2 || !mesh->affine)) return fail(DG_ERR_UNSUPPORTED);
  if (co->precision != DG_FP64 && co->precision != DG_FP32) return fail(DG_ERR_INVALID_ARG);
  if (co->max_rhs < 1 || co->max_rhs > 16) return fail(DG_ERR_INVALID_ARG);
  if (pen->mode != DG_PEN_CONFIG && pen->mode != DG_PEN_PAPER) return fail(DG_ERR_INVALID_ARG);
  if (co->dirichlet_mask < 0 || co->dirichlet_mask > 63) return fail(DG_ERR_INVALID_ARG);
  if (co->geometry < DG_GEOM_AUTO || co->geometry > DG_GEOM_RECOMPUTE) return fail(DG_ERR_INVALID_ARG);
  if (co->geometry == DG_GEOM_RECOMPUTE && !mesh->affine && !any_recompute &&
      (co->problem != DG_SCALAR || m != degree + 1))
    return fail(DG_ERR_UNSUPPORTED);

  dg_operator *o = new (std::nothrow) dg_operator;
  if (!o) return fail(DG_ERR_OOM);
  o->nx = mesh->nx; o->ny = mesh->ny; o->nz = mesh->nz;
  o->k = degree; o->p = degree + 1; o->m = m;
  o->problem = co->problem;
  o->precision = co->precision;
  o->max_rhs = co->max_rhs;
  o->dmask = (unsigned)co->dirichlet_mask;
  o->c = co->c; o->mu = co->mu; o->theta = co->theta;
  o->pen = *pen;
  o->geo = mesh->affine ? GEO_AFFINE : (co->geometry == DG_GEOM_RECOMPUTE ? GEO_RECOMPUTE : GEO_STORED);
  o->ncell = (int64_t)o->nx * o->ny * o->nz;
  const int n[3] = {o->nx, o->ny, o->nz};
  o->face_off[0] = 0;
  o->nbface = 0;
  for (int a = 0; a < 3; ++a) {
    const int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
    o->face_off[a + 1] = o->face_off[a] + (int64_t)(n[a] + 1) * n[t1] * n[t2];
    o->nbface += 2 * (int64_t)n[t1] * n[t2];
  }
  o->nface = o->face_off[3];
  const int P3 = o->p * o->p * o->p, M2 = m * m, M3 = m * m * m;
  const bool stokes = o->problem == DG_STOKES;
  o->ndofs = stokes ? o->ncell * (3 * P3 + degree * degree * degree) : o->ncell * P3;
  for (int a = 0; a < 3; ++a)
    o->gamma_axis[a] = pen->mode == DG_PEN_CONFIG ? pen->alpha * degree * (degree + 1) * n[a]
                                                  : pen->alpha * degree * (degree + 2) * n[a];
  if (dg_build_tables(degree, m, stokes, &o->ht)) { free_op(o); return fail(DG_ERR_UNSUPPORTED); }
  default_blocking(o);
  o->variant = resolve_variant(o, DG_VARIANT_AUTO);
  const size_t es = o->precision == DG_FP64 ? sizeof(double) : sizeof(float);

#define ALLOC(ptr, bytes)                                       \
  do {                                                          \
    if (cudaMalloc((void **)&(ptr), (bytes)) != cudaSuccess) {  \
      cudaGetLastError();                                       \
      free_op(o);                                               \
      return fail(DG_ERR_OOM);                                  \
    }                                                           \
  } while (0)

  if (o->precision == DG_FP64) {
    DevTables<double> t;
    fill_devtables(o->ht, t);
    ALLOC(o->d_tab, sizeof(t));
    if (cudaMemcpy(o->d_tab, &t, sizeof(t), cudaMemcpyHostToDevice) != cudaSuccess) { free_op(o); return fail(DG_ERR_CUDA); }
  } else {
    DevTables<float> t;
    fill_devtables(o->ht, t);
    ALLOC(o->d_tab, sizeof(t));
    if (cudaMemcpy(o->d_tab, &t, sizeof(t), cudaMemcpyHostToDevice) != cudaSuccess) { free_op(o); return fail(DG_ERR_CUDA); }
  }
  if (!mesh->affine) {
    const size_t vb = mesh->verts.size() * sizeof(double);
    ALLOC(o->d_verts, vb);
    ALLOC(o->d_gamma, (size_t)o->nface * sizeof(double));
    ALLOC(o->d_cellvol, (size_t)o->ncell * sizeof(double));
    if (cudaMemcpy(o->d_verts, mesh->verts.data(), vb, cudaMemcpyHostToDevice) != cudaSuccess) { free_op(o); return fail(DG_ERR_CUDA); }
    if (launch_penalty(m, degree, pen->mode, pen->alpha, o->nx, o->ny, o->nz, o->nface, o->face_off, o->d_verts,
                       o->ht.gauss_s, o->ht.gauss_w, o->d_gamma, o->d_cellvol, 0) != cudaSuccess) {
      free_op(o);
      return fail(DG_ERR_CUDA);
    }
    if (o->geo == GEO_RECOMPUTE) {
      if (cudaDeviceSynchronize() != cudaSuccess) { free_op(o); return fail(DG_ERR_CUDA); }
      goto geometry_done;
    }
    ALLOC(o->d_gvol, (size_t)o->ncell * 7 * M3 * es);
    ALLOC(o->d_gface, (size_t)o->nface * 7 * M2 * es);
    cudaError_t e;
    if (o->precision == DG_FP64)
      e = launch_geometry<double>(m, scalar_args<double>(o, false), o->d_verts, o->c, o->d_gamma, o->ht.gauss_s,
                                  o->ht.gauss_w, (double *)o->d_gvol, (double *)o->d_gface, 0);
    else
      e = launch_geometry<float>(m, scalar_args<float>(o, false), o->d_verts, o->c, o->d_gamma, o->ht.gauss_s,
                                 o->ht.gauss_w, (float *)o->d_gvol, (float *)o->d_gface, 0);
    if (e != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) { free_op(o); return fail(DG_ERR_CUDA); }
  }
geometry_done:
  const size_t R = (size_t)o->max_rhs;
  const size_t nrv = stokes ? 4 : 1, ntr = stokes ? 42 : 12;
  ALLOC(o->d_rvol, R * o->ncell * nrv * M3 * es);
  ALLOC(o->d_tr, R * o->ncell * ntr * M2 * es);
  ALLOC(o->d_fres, R * o->ncell * ntr * M2 * es);
#undef ALLOC
  *out = o;
  return DG_OK;
}

dg_status dg_operator_destroy(dg_operator *op) {
  free_op(op);
  return DG_OK;
}

dg_status dg_operator_create_aniso(const dg_mesh *mesh, const int32_t degrees[3], const int32_t quad_points[3],
                                   const dg_penalty *pen, const dg_coefficients *co, dg_operator **out) {
  if (!mesh || !degrees || !pen || !co || !out) return fail(DG_ERR_INVALID_ARG);
  int kmax = 0, mq[3];
  for (int a = 0; a < 3; ++a) {
    if (degrees[a] < 1 || degrees[a] + 1 > DG_MAXP) return fail(DG_ERR_INVALID_ARG);
    kmax = degrees[a] > kmax ? degrees[a] : kmax;
    mq[a] = (quad_points && quad_points[a]) ? quad_points[a] : degrees[a] + 1;
    if (mq[a] < degrees[a] + 1) return fail(DG_ERR_INVALID_ARG);
    if (mq[a] > DG_MAXM) return fail(DG_ERR_UNSUPPORTED);
  }
  if (co->problem != DG_SCALAR) return fail(DG_ERR_UNSUPPORTED);
  // the paper's penalty needs face and cell measures by the anisotropic rule: affine only
  if (!mesh->affine && pen->mode != DG_PEN_CONFIG) return fail(DG_ERR_UNSUPPORTED);
  // an isotropic operator of the largest degree supplies the mesh bookkeeping (vertices,
  // face numbering); trilinear geometry is recomputed by the anisotropic kernels, so none
  // is stored, and the scratch is reallocated below for the per-direction sizes
  dg_coefficients co2 = *co;
  co2.geometry = DG_GEOM_RECOMPUTE;
  dg_status st = create_impl(mesh, kmax, 0, pen, &co2, out, true);
  if (st != DG_OK) return st;
  dg_operator *o = *out;
  HostTables ht[3];
  const int n[3] = {o->nx, o->ny, o->nz};
  int npts = 1, nq = 1;
  for (int a = 0; a < 3; ++a) {
    const int k = degrees[a];
    if (dg_build_tables(k, mq[a], false, &ht[a])) { free_op(o); *out = nullptr; return fail(DG_ERR_UNSUPPORTED); }
    o->kax[a] = k;
    o->max_q[a] = mq[a];
    // the penalty of a face takes the degree along its normal
    o->gamma_axis[a] = pen->mode == DG_PEN_CONFIG ? pen->alpha * k * (k + 1) * n[a] : pen->alpha * k * (k + 2) * n[a];
    npts *= k + 1;
    nq *= mq[a];
  }
  const bool f64 = o->precision == DG_FP64;
  const size_t es = f64 ? sizeof(double) : sizeof(float);
  std::vector<unsigned char> host(f64 ? aniso_tab_bytes<double>() : aniso_tab_bytes<float>());
  int ts = 0;
  bool ok = (f64 ? aniso_tables<double>(ht, host.data(), &ts) : aniso_tables<float>(ht, host.data(), &ts)) == 0;
  if (ok) {
    cudaFree(o->d_rvol);
    cudaFree(o->d_tr);
    cudaFree(o->d_fres);
    o->d_rvol = o->d_tr = o->d_fres = nullptr;
    const size_t R = (size_t)o->max_rhs;
    ok = cudaMalloc(&o->d_antab, host.size()) == cudaSuccess &&
         cudaMemcpy(o->d_antab, host.data(), host.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMalloc(&o->d_rvol, R * o->ncell * nq * es) == cudaSuccess &&
         cudaMalloc(&o->d_tr, R * o->ncell * ts * es) == cudaSuccess &&
         cudaMalloc(&o->d_fres, R * o->ncell * ts * es) == cudaSuccess;
  }
  if (ok && !mesh->affine) {  // per-face penalty alpha k_a (k_a + 1) n_a for the recomputed-geometry kernels
    std::vector<double> g((size_t)o->nface);
    for (int a = 0; a < 3; ++a)
      for (int64_t f = o->face_off[a]; f < o->face_off[a + 1]; ++f) g[(size_t)f] = o->gamma_axis[a];
    ok = cudaMemcpy(o->d_gamma, g.data(), g.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    free_op(o);
    *out = nullptr;
    return fail(DG_ERR_OOM);
  }
  o->aniso = 1;
  o->an_npts = npts;
  o->an_nq = nq;
  o->an_ts = ts;
  o->ndofs = o->ncell * npts;
  o->variant = DG_VARIANT_THREE_KERNEL;
  o->cpb = 256 / nq > 0 ? 256 / nq : 1;
  o->fpb = 256 / (DG_MAXM * DG_MAXM) > 0 ? 256 / (DG_MAXM * DG_MAXM) : 1;
  return DG_OK;
}

dg_status dg_operator_ndofs(const dg_operator *op, int64_t *n) {
  if (!op || !n) return fail(DG_ERR_INVALID_ARG);
  *n = op->ndofs;
  return DG_OK;
}

dg_status dg_operator_set_kappa(dg_operator *op, const void *kappa_vol, const void *kappa_face) {
  if (!op) return fail(DG_ERR_INVALID_ARG);
  if ((kappa_vol && !aligned16(kappa_vol)) || (kappa_face && !aligned16(kappa_face))) return fail(DG_ERR_INVALID_ARG);
  if ((kappa_vol == nullptr) != (kappa_face == nullptr)) return fail(DG_ERR_INVALID_ARG);
  if (op->problem != DG_SCALAR) return fail(DG_ERR_UNSUPPORTED);
  if (op->kappa_vol != kappa_vol || op->kappa_face != kappa_face) {
    if (op->sv_dinv) cudaFree(op->sv_dinv);  // the Jacobi diagonal depends on kappa
    op->sv_dinv = nullptr;
  }
  op->kappa_vol = kappa_vol;
  op->kappa_face = kappa_face;
  if (!variant_ok(op, op->variant)) op->variant = DG_VARIANT_THREE_KERNEL;
  return DG_OK;
}

dg_status dg_operator_stats(const dg_operator *op, dg_stats *out) {
  if (!op || !out) return fail(DG_ERR_INVALID_ARG);
  memset(out, 0, sizeof(*out));
  out->ndofs = op->ndofs;
  out->ncell = op->ncell;
  out->nface = op->nface;
  const int es = op->precision == DG_FP64 ? 8 : 4;
  if (op->aniso)
    aniso_work_model(op->kax, op->max_q, op->geo, op->kappa_vol != nullptr, op->ncell, op->nface, op->nbface,
                     out->flops, out->bytes, es);
  else if (op->problem == DG_STOKES)
    stokes_work_model(op->p, op->ncell, op->nface, op->nbface, out->flops, out->bytes, es);
  else if (op->variant == DG_VARIANT_FUSED)
    fused_work_model(op->p, op->ncell, op->nbface, out->flops, out->bytes, es);
  else if (op->variant == DG_VARIANT_CELLWISE)
    cellwise_work_model(op->p, op->nx, op->ny, op->nz, op->brick, op->nbface, out->flops, out->bytes, es);
  else
    scalar_work_model(op->p, op->m, op->geo, op->kappa_vol != nullptr, op->ncell, op->nface, op->nbface, out->flops,
                      out->bytes, es);
  out->dofs_bytes = 2.0 * es * (double)op->ndofs;
  out->cells_per_block = op->cpb;
  out->faces_per_block = op->fpb;
  const int M3 = op->m * op->m * op->m, M2 = op->m * op->m;
  auto thr = [](int w) { int t = ((w + 31) / 32) * 32; return t < 64 ? 64 : (t > 256 ? 256 : t); };
  out->threads_cell = thr(op->cpb * M3);
  out->threads_face = thr(op->fpb * M2);
  out->geometry = op->geo == GEO_AFFINE ? 0 : (op->geo == GEO_STORED ? DG_GEOM_STORED : DG_GEOM_RECOMPUTE);
  out->variant = op->variant;
  out->persistent_grid = op->fused_grid;
  if (op->variant == DG_VARIANT_FUSED || op->variant == DG_VARIANT_CELLWISE) {
    const bool fz = op->variant == DG_VARIANT_FUSED;
    out->cells_per_block = fz ? op->tile : op->brick;
    out->threads_cell = fz ? op->tile * op->p * op->p : op->brick;
    out->faces_per_block = 0;
    out->threads_face = 0;
  }
  return DG_OK;
}

}  // extern "C"

static const cudaEvent_t *next_events(dg_operator *op) {
  if (!op->prof) return nullptr;
  const size_t need = 4 * (op->prof_used + 1);
  while (op->prof_ev.size() < need) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    op->prof_ev.push_back(e);
  }
  return op->prof_ev.data() + 4 * op->prof_used++;
}

dg_status dg_record_error(dg_status s) { return fail(s); }

dg_status dg_apply_internal(const dg_operator *op, const void *x, void *y, int nrhs, cudaStream_t s, bool transpose);

static dg_status apply_impl(const dg_operator *op_c, const void *x, void *y, int nrhs, cudaStream_t s, bool transpose) {
  dg_operator *op = const_cast<dg_operator *>(op_c);
  const cudaEvent_t *ev = next_events(op);
  const int M2 = op->m * op->m, M3 = op->m * op->m * op->m;
  cudaError_t e;
  if (op->problem == DG_STOKES) {
    const int64_t sdof = op->ndofs, srv = op->ncell * 4 * M3, str = op->ncell * 42 * M2;
    if (op->variant == DG_VARIANT_DF64 && df64_ok(op)) {
      e = launch_stokes_apply<df64>(op->p, df64_args(op, transpose), df64(op->mu), (const double *)x, (double *)y, (df64 *)op->d_rvol,
                                    (df64 *)op->d_tr, (df64 *)op->d_fres, nrhs, sdof, srv, str, op->cpb, op->fpb, s,
                                    ev);
      if (e != cudaSuccess) return fail(DG_ERR_CUDA);
      return DG_OK;
    }
    if (op->precision == DG_FP64)
      e = launch_stokes_apply<double>(op->p, scalar_args<double>(op, transpose), op->mu, (const double *)x,
                                      (double *)y, (double *)op->d_rvol, (double *)op->d_tr, (double *)op->d_fres,
                                      nrhs, sdof, srv, str, op->cpb, op->fpb, s, ev);
    else
      e = launch_stokes_apply<float>(op->p, scalar_args<float>(op, transpose), (float)op->mu, (const float *)x,
                                     (float *)y, (float *)op->d_rvol, (float *)op->d_tr, (float *)op->d_fres, nrhs,
                                     sdof, srv, str, op->cpb, op->fpb, s, ev);
    if (e != cudaSuccess) return fail(DG_ERR_CUDA);
    return DG_OK;
  }
  if (op->aniso) {
    const int64_t sv = op->ncell * op->an_nq, st = op->ncell * op->an_ts;
    const int geo = op->geo == GEO_AFFINE ? GEO_AFFINE : GEO_RECOMPUTE;
    const bool kap = op->kappa_vol != nullptr;
    if (op->precision == DG_FP64)
      e = launch_aniso_apply<double>(scalar_args<double>(op, transpose), op->d_antab, op->an_npts, op->an_ts,
                                     (const double *)x, (double *)y, (double *)op->d_rvol, (double *)op->d_tr,
                                     (double *)op->d_fres, nrhs, op->ndofs, sv, st, op->cpb, op->fpb, s, ev, geo, kap,
                                     op->an_nq);
    else
      e = launch_aniso_apply<float>(scalar_args<float>(op, transpose), op->d_antab, op->an_npts, op->an_ts,
                                    (const float *)x, (float *)y, (float *)op->d_rvol, (float *)op->d_tr,
                                    (float *)op->d_fres, nrhs, op->ndofs, sv, st, op->cpb, op->fpb, s, ev, geo, kap,
                                    op->an_nq);
    if (e != cudaSuccess) return fail(DG_ERR_CUDA);
    return DG_OK;
  }
  const int64_t sdof = op->ndofs, srv = op->ncell * M3, str = op->ncell * 12 * M2;
  const bool kap = op->kappa_vol != nullptr;
  if (op->geo == GEO_RECOMPUTE) {  // geometry from the vertices, in the adjoint kernels with forward coefficients
    if (op->variant == DG_VARIANT_DF64 && df64_ok(op)) {
      for (int r = 0; r < nrhs; ++r) {
        e = launch_scalar_adjoint<df64>(op->p, GEO_RECOMPUTE, kap, df64_args(op, transpose), op->theta,
                                        (const double *)x + r * sdof, nullptr, (double *)y + r * sdof, nullptr,
                                        nullptr, (df64 *)op->d_rvol, (df64 *)op->d_tr, nullptr, (df64 *)op->d_fres,
                                        op->cpb, op->fpb, s, r == 0 ? ev : nullptr);
        if (e != cudaSuccess) return fail(DG_ERR_CUDA);
      }
      return DG_OK;
    }
    for (int r = 0; r < nrhs; ++r) {
      if (op->precision == DG_FP32)
        e = launch_scalar_adjoint<float>(op->p, GEO_RECOMPUTE, kap, scalar_args<float>(op, transpose), op->theta,
                                         (const float *)x + r * sdof, nullptr, (float *)y + r * sdof, nullptr,
                                         nullptr, (float *)op->d_rvol, (float *)op->d_tr, nullptr,
                                         (float *)op->d_fres, op->cpb, op->fpb, s, r == 0 ? ev : nullptr);
      else
        e = launch_scalar_adjoint<double>(op->p, GEO_RECOMPUTE, kap, scalar_args<double>(op, transpose), op->theta,
                                          (const double *)x + r * sdof, nullptr, (double *)y + r * sdof, nullptr,
                                          nullptr, (double *)op->d_rvol, (double *)op->d_tr, nullptr,
                                          (double *)op->d_fres, op->cpb, op->fpb, s, r == 0 ? ev : nullptr);
      if (e != cudaSuccess) return fail(DG_ERR_CUDA);
    }
    return DG_OK;
  }
  if (op->variant == DG_VARIANT_DF64 && df64_ok(op)) {
    e = launch_scalar_apply<df64>(op->p, op->m, op->geo, kap, df64_args(op, transpose), (const double *)x, (double *)y,
                                  (df64 *)op->d_rvol,
                                  (df64 *)op->d_tr, (df64 *)op->d_fres, nrhs, sdof, srv, str, op->cpb, op->fpb, s, ev,
                                  nullptr, 7, 0, -1, &op->ht);
    if (e != cudaSuccess) return fail(DG_ERR_CUDA);
    return DG_OK;
  }
  if (op->variant == DG_VARIANT_CELLWISE && cellwise_ok(op)) {
    if (op->precision == DG_FP64)
      e = launch_cellwise_apply<double>(op->p, scalar_args<double>(op, transpose), op->ht, (const double *)x,
                                        (double *)y, nrhs, sdof, op->brick, s, ev, &op->fused_grid);
    else
      e = launch_cellwise_apply<float>(op->p, scalar_args<float>(op, transpose), op->ht, (const float *)x, (float *)y,
                                       nrhs, sdof, op->brick, s, ev, &op->fused_grid);
    if (e != cudaSuccess) return fail(DG_ERR_CUDA);
    return DG_OK;
  }
  if (op->variant == DG_VARIANT_FUSED && fused_ok(op)) {
    if (op->precision == DG_FP64)
      e = launch_fused_apply<double>(op->p, scalar_args<double>(op, transpose), op->ht, (const double *)x, (double *)y, nrhs,
                                     sdof, op->tile, s, ev, &op->fused_grid);
    else
      e = launch_fused_apply<float>(op->p, scalar_args<float>(op, transpose), op->ht, (const float *)x, (float *)y, nrhs,
                                    sdof, op->tile, s, ev, &op->fused_grid);
    if (e != cudaSuccess) return fail(DG_ERR_CUDA);
    return DG_OK;
  }
  if (op->precision == DG_FP64)
    e = launch_scalar_apply<double>(op->p, op->m, op->geo, kap, scalar_args<double>(op, transpose), (const double *)x,
                                    (double *)y, (double *)op->d_rvol, (double *)op->d_tr, (double *)op->d_fres, nrhs,
                                    sdof, srv, str, op->cpb, op->fpb, s, ev);
  else
    e = launch_scalar_apply<float>(op->p, op->m, op->geo, kap, scalar_args<float>(op, transpose), (const float *)x,
                                   (float *)y, (float *)op->d_rvol, (float *)op->d_tr, (float *)op->d_fres, nrhs, sdof,
                                   srv, str, op->cpb, op->fpb, s, ev, nullptr, 7, 0, -1, &op->ht);
  if (e != cudaSuccess) return fail(DG_ERR_CUDA);
  return DG_OK;
}

extern "C" {

}  // extern "C"

dg_status dg_apply_dot_internal(const dg_operator *op, const void *x, void *y, int nrhs, cudaStream_t s,
                                double *dot_partial, int dot_stride, int *nblocks) {
  if (!op || op->precision != DG_FP32 || op->variant != DG_VARIANT_CELLWISE || !cellwise_ok(op) || op->aniso ||
      op->problem != DG_SCALAR || !dot_partial || !nblocks)
    return DG_ERR_UNSUPPORTED;
  dg_operator *o = const_cast<dg_operator *>(op);
  const cudaError_t e = launch_cellwise_apply<float>(op->p, scalar_args<float>(op, false), op->ht, (const float *)x,
                                                     (float *)y, nrhs, op->ndofs, op->brick, s, nullptr,
                                                     &o->fused_grid, nullptr, dot_partial, dot_stride);
  if (e != cudaSuccess) return fail(DG_ERR_CUDA);
  *nblocks = op->fused_grid;
  return DG_OK;
}

dg_status dg_apply_internal(const dg_operator *op, const void *x, void *y, int nrhs, cudaStream_t s, bool transpose) {
  return apply_impl(op, x, y, nrhs, s, transpose);
}

extern "C" {

dg_status dg_apply(const dg_operator *op, const void *x, void *y, int nrhs, void *stream) {
  if (!op || !x || !y) return fail(DG_ERR_INVALID_ARG);
  if (nrhs < 1 || nrhs > op->max_rhs) return fail(DG_ERR_INVALID_ARG);
  if (!aligned16(x) || !aligned16(y) || x == y) return fail(DG_ERR_INVALID_ARG);
  return apply_impl(op, x, y, nrhs, (cudaStream_t)stream, false);
}

}  // extern "C"

// dg_apply_host pipelined over chunks of cells for the three-kernel scalar apply: the cell
// kernel of a chunk needs only that chunk's x, and the back-projection kernel of a chunk
// produces that chunk's y, so host-to-device copies run ahead of the cell kernels and
// device-to-host copies behind the back-projection kernels, on a copy stream ordered by
// events; the face kernel runs between the two loops.
static bool host_pipeline_ok(const dg_operator *o) {
  return o->problem == DG_SCALAR && !o->aniso && (o->geo == GEO_AFFINE || o->geo == GEO_STORED) &&
         (o->variant == DG_VARIANT_THREE_KERNEL || (o->variant == DG_VARIANT_DF64 && df64_ok(o)));
}

static constexpr int kHostChunks = 8;

static dg_status apply_host_pipelined(dg_operator *op, const void *x_host, void *y_host, int nrhs, cudaStream_t s) {
  const size_t es = op->precision == DG_FP64 ? sizeof(double) : sizeof(float);
  if (!op->hs_copy) {
    if (cudaStreamCreateWithFlags(&op->hs_copy, cudaStreamNonBlocking) != cudaSuccess) {
      op->hs_copy = nullptr;
      return fail(DG_ERR_CUDA);
    }
    while (op->hs_ev.size() < 2 * kHostChunks + 2) {
      cudaEvent_t e;
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(DG_ERR_CUDA);
      op->hs_ev.push_back(e);
    }
  }
  const int M = op->m, M2 = M * M, M3 = M2 * M;
  const int64_t P3 = (int64_t)op->p * op->p * op->p, ncell = op->ncell, sdof = op->ndofs;
  const int64_t srv = ncell * M3, str = ncell * 12 * M2;
  const int nch = (int)std::min<int64_t>(kHostChunks, ncell);
  const size_t pitch = (size_t)sdof * es;
  cudaStream_t cs = op->hs_copy;
  cudaEvent_t *ev = op->hs_ev.data();
  const bool kap = op->kappa_vol != nullptr;
  auto phase = [&](int ph, int64_t cb, int64_t cn) -> cudaError_t {
    if (op->variant == DG_VARIANT_DF64)
      return launch_scalar_apply<df64>(op->p, M, op->geo, kap, df64_args(op, false), (const double *)op->d_xh,
                                       (double *)op->d_yh, (df64 *)op->d_rvol, (df64 *)op->d_tr, (df64 *)op->d_fres,
                                       nrhs, sdof, srv, str, op->cpb, op->fpb, s, nullptr, nullptr, ph, cb, cn,
                                       &op->ht);
    if (op->precision == DG_FP64)
      return launch_scalar_apply<double>(op->p, M, op->geo, kap, scalar_args<double>(op, false),
                                         (const double *)op->d_xh, (double *)op->d_yh, (double *)op->d_rvol,
                                         (double *)op->d_tr, (double *)op->d_fres, nrhs, sdof, srv, str, op->cpb,
                                         op->fpb, s, nullptr, nullptr, ph, cb, cn);
    return launch_scalar_apply<float>(op->p, M, op->geo, kap, scalar_args<float>(op, false), (const float *)op->d_xh,
                                      (float *)op->d_yh, (float *)op->d_rvol, (float *)op->d_tr, (float *)op->d_fres,
                                      nrhs, sdof, srv, str, op->cpb, op->fpb, s, nullptr, nullptr, ph, cb, cn, &op->ht);
  };
  auto chunk = [&](int k, int64_t *cb, int64_t *cn) {
    *cb = ncell * k / nch;
    *cn = ncell * (k + 1) / nch - *cb;
  };
  // the copies into the staging buffers wait for earlier work on s that may still use them
  CK(cudaEventRecord(ev[2 * kHostChunks], s));
  CK(cudaStreamWaitEvent(cs, ev[2 * kHostChunks], 0));
  for (int k = 0; k < nch; ++k) {
    int64_t cb, cn;
    chunk(k, &cb, &cn);
    const size_t off = (size_t)(cb * P3) * es;
    CK(cudaMemcpy2DAsync((char *)op->d_xh + off, pitch, (const char *)x_host + off, pitch, (size_t)(cn * P3) * es,
                         nrhs, cudaMemcpyHostToDevice, cs));
    CK(cudaEventRecord(ev[k], cs));
    CK(cudaStreamWaitEvent(s, ev[k], 0));
    CK(phase(1, cb, cn));
  }
  CK(phase(2, 0, ncell));
  for (int k = 0; k < nch; ++k) {
    int64_t cb, cn;
    chunk(k, &cb, &cn);
    CK(phase(4, cb, cn));
    CK(cudaEventRecord(ev[kHostChunks + k], s));
    CK(cudaStreamWaitEvent(cs, ev[kHostChunks + k], 0));
    const size_t off = (size_t)(cb * P3) * es;
    CK(cudaMemcpy2DAsync((char *)y_host + off, pitch, (const char *)op->d_yh + off, pitch, (size_t)(cn * P3) * es,
                         nrhs, cudaMemcpyDeviceToHost, cs));
  }
  CK(cudaEventRecord(ev[2 * kHostChunks + 1], cs));
  CK(cudaStreamWaitEvent(s, ev[2 * kHostChunks + 1], 0));
  CK(cudaStreamSynchronize(s));
  return DG_OK;
}

extern "C" {

dg_status dg_apply_host(const dg_operator *op_c, const void *x_host, void *y_host, int nrhs, void *stream) {
  dg_operator *op = const_cast<dg_operator *>(op_c);
  if (!op || !x_host || !y_host) return fail(DG_ERR_INVALID_ARG);
  if (nrhs < 1 || nrhs > op->max_rhs) return fail(DG_ERR_INVALID_ARG);
  const size_t es = op->precision == DG_FP64 ? sizeof(double) : sizeof(float);
  const size_t bytes = (size_t)nrhs * op->ndofs * es;
  if (!op->d_xh) {
    const size_t full = (size_t)op->max_rhs * op->ndofs * es;
    if (cudaMalloc(&op->d_xh, full) != cudaSuccess || cudaMalloc(&op->d_yh, full) != cudaSuccess) {
      cudaGetLastError();
      return fail(DG_ERR_OOM);
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (host_pipeline_ok(op)) return apply_host_pipelined(op, x_host, y_host, nrhs, s);
  CK(cudaMemcpyAsync(op->d_xh, x_host, bytes, cudaMemcpyHostToDevice, s));
  dg_status st = apply_impl(op, op->d_xh, op->d_yh, nrhs, s, false);
  if (st != DG_OK) return st;
  CK(cudaMemcpyAsync(y_host, op->d_yh, bytes, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return DG_OK;
}

dg_status dg_apply_adjoint(const dg_operator *op_c, const void *r, const void *x, void *y, void *dkappa_vol,
                           void *dkappa_face, int nrhs, void *stream) {
  dg_operator *op = const_cast<dg_operator *>(op_c);
  if (op && op->aniso) return fail(DG_ERR_UNSUPPORTED);
  if (!op || !r || !y || r == y || (x && x == y)) return fail(DG_ERR_INVALID_ARG);
  if (nrhs < 1 || nrhs > op->max_rhs) return fail(DG_ERR_INVALID_ARG);
  if (!aligned16(r) || !aligned16(y) || (x && !aligned16(x))) return fail(DG_ERR_INVALID_ARG);
  if ((dkappa_vol == nullptr) != (dkappa_face == nullptr)) return fail(DG_ERR_INVALID_ARG);
  if (dkappa_vol && (!x || !aligned16(dkappa_vol) || !aligned16(dkappa_face))) return fail(DG_ERR_INVALID_ARG);
  if (op->problem == DG_STOKES || op->precision == DG_FP32) {
    // no kappa to differentiate: y = A^T r is the forward operator with the flux and
    // symmetry coefficients exchanged (the Stokes coupling [[., B^T], [B, 0]] is symmetric)
    if (dkappa_vol) return fail(DG_ERR_UNSUPPORTED);
    return apply_impl(op, r, y, nrhs, (cudaStream_t)stream, true);
  }
  if (op->problem != DG_SCALAR || op->precision != DG_FP64 || op->m != op->p) return fail(DG_ERR_UNSUPPORTED);
  const int M2 = op->m * op->m;
  if (dkappa_vol && !op->d_tr2) {
    if (cudaMalloc(&op->d_tr2, (size_t)op->ncell * 12 * M2 * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(DG_ERR_OOM);
    }
  }
  const int geo = op->geo == GEO_AFFINE ? GEO_AFFINE : GEO_RECOMPUTE;
  const cudaEvent_t *ev = next_events(op);
  const int64_t sd = op->ndofs;
  const bool df = op->variant == DG_VARIANT_DF64 && df64_ok(op);
  // one pass of the three adjoint kernels per right-hand side (scratch of the first slot
  // reused in stream order); dkappa of the second and later right-hand sides is added to
  // the first one's, which gives the gradient of the summed loss
  for (int s = 0; s < nrhs; ++s) {
    const double *rs = (const double *)r + s * sd;
    const double *xs = dkappa_vol ? (const double *)x + s * sd : nullptr;
    double *ys = (double *)y + s * sd;
    cudaError_t e;
    if (df)
      e = launch_scalar_adjoint<df64>(op->p, geo, op->kappa_vol != nullptr, df64_args(op, true), op->theta, rs, xs,
                                      ys, (double *)dkappa_vol, (double *)dkappa_face, (df64 *)op->d_rvol,
                                      (df64 *)op->d_tr, (df64 *)op->d_tr2, (df64 *)op->d_fres, op->cpb, op->fpb,
                                      (cudaStream_t)stream, s == 0 ? ev : nullptr, 0, 0.0, s > 0);
    else
      e = launch_scalar_adjoint<double>(op->p, geo, op->kappa_vol != nullptr, scalar_args<double>(op, true),
                                        op->theta, rs, xs, ys, (double *)dkappa_vol, (double *)dkappa_face,
                                        (double *)op->d_rvol, (double *)op->d_tr, (double *)op->d_tr2,
                                        (double *)op->d_fres, op->cpb, op->fpb, (cudaStream_t)stream,
                                        s == 0 ? ev : nullptr, 0, 0.0, s > 0);
    if (e != cudaSuccess) return fail(DG_ERR_CUDA);
  }
  return DG_OK;
}

dg_status dg_apply_semilinear(const dg_operator *op_c, int mode, double beta, const void *u0, const void *w, void *y,
                              void *stream) {
  dg_operator *op = const_cast<dg_operator *>(op_c);
  if (op && op->aniso) return fail(DG_ERR_UNSUPPORTED);
  if (!op || !w || !y || w == y || (u0 && u0 == y)) return fail(DG_ERR_INVALID_ARG);
  if (mode != DG_SEMILINEAR_RESIDUAL && mode != DG_SEMILINEAR_JACOBIAN) return fail(DG_ERR_INVALID_ARG);
  if (mode == DG_SEMILINEAR_JACOBIAN && !u0) return fail(DG_ERR_INVALID_ARG);
  if (!aligned16(w) || !aligned16(y) || (u0 && !aligned16(u0)) || !(beta == beta)) return fail(DG_ERR_INVALID_ARG);
  if (op->problem != DG_SCALAR || op->precision != DG_FP64 || op->m != op->p) return fail(DG_ERR_UNSUPPORTED);
  const int geo = op->geo == GEO_AFFINE ? GEO_AFFINE : GEO_RECOMPUTE;
  const cudaEvent_t *ev = next_events(op);
  if (op->variant == DG_VARIANT_DF64 && df64_ok(op)) {
    const cudaError_t e = launch_scalar_adjoint<df64>(
        op->p, geo, op->kappa_vol != nullptr, df64_args(op, false), op->theta, (const double *)w,
        mode == DG_SEMILINEAR_JACOBIAN ? (const double *)u0 : nullptr, (double *)y, nullptr, nullptr,
        (df64 *)op->d_rvol, (df64 *)op->d_tr, nullptr, (df64 *)op->d_fres, op->cpb, op->fpb, (cudaStream_t)stream,
        ev, mode == DG_SEMILINEAR_JACOBIAN ? 2 : 1, beta);
    return e == cudaSuccess ? DG_OK : fail(DG_ERR_CUDA);
  }
  cudaError_t e = launch_scalar_adjoint<double>(
      op->p, geo, op->kappa_vol != nullptr, scalar_args<double>(op, false), op->theta, (const double *)w,
      mode == DG_SEMILINEAR_JACOBIAN ? (const double *)u0 : nullptr, (double *)y, nullptr, nullptr,
      (double *)op->d_rvol, (double *)op->d_tr, nullptr, (double *)op->d_fres, op->cpb, op->fpb, (cudaStream_t)stream,
      ev, mode == DG_SEMILINEAR_JACOBIAN ? 2 : 1, beta);
  if (e != cudaSuccess) return fail(DG_ERR_CUDA);
  return DG_OK;
}

dg_status dg_rhs(const dg_operator *op_c, const void *f_vol, const void *g_face, void *F, void *stream) {
  dg_operator *op = const_cast<dg_operator *>(op_c);
  if (op && op->aniso) return fail(DG_ERR_UNSUPPORTED);
  if (!op || !F || F == f_vol || F == g_face || !aligned16(F)) return fail(DG_ERR_INVALID_ARG);
  if ((f_vol && !aligned16(f_vol)) || (g_face && !aligned16(g_face))) return fail(DG_ERR_INVALID_ARG);
  if (op->problem != DG_SCALAR || op->m != op->p) return fail(DG_ERR_UNSUPPORTED);
  const int geo = op->geo == GEO_AFFINE ? GEO_AFFINE : GEO_RECOMPUTE;
  const bool kap = op->kappa_face != nullptr;
  cudaError_t e;
  if (op->precision == DG_FP64)
    e = launch_rhs<double>(op->p, geo, kap, scalar_args<double>(op, false), op->theta, (const double *)f_vol,
                           (const double *)g_face, (double *)F, (double *)op->d_rvol, (double *)op->d_fres, op->cpb,
                           op->fpb, (cudaStream_t)stream);
  else
    e = launch_rhs<float>(op->p, geo, kap, scalar_args<float>(op, false), (float)op->theta, (const float *)f_vol,
                          (const float *)g_face, (float *)F, (float *)op->d_rvol, (float *)op->d_fres, op->cpb,
                          op->fpb, (cudaStream_t)stream);
  return e == cudaSuccess ? DG_OK : fail(DG_ERR_CUDA);
}

dg_status dg_operator_set_variant(dg_operator *op, int variant, int cells_per_block, int faces_per_block) {
  if (op && op->aniso) return fail(DG_ERR_UNSUPPORTED);
  if (!op || variant < DG_VARIANT_AUTO || variant > DG_VARIANT_DF64 || cells_per_block < 0 || faces_per_block < 0)
    return fail(DG_ERR_INVALID_ARG);
  const int v = resolve_variant(op, variant);
  if (!variant_ok(op, v)) return fail(DG_ERR_UNSUPPORTED);
  if (v == DG_VARIANT_DF64) {
    const dg_status st = ensure_df64(op);
    if (st != DG_OK) return st;
  }
  const size_t es = op->precision == DG_FP64 ? 8 : 4;
  const int M = op->m, P = op->p;
  if (v == DG_VARIANT_CELLWISE) {
    if (cells_per_block > 0) {
      const size_t sm = cellwise_smem_bytes(P, cells_per_block, (int)es);
      if (sm == 0 || sm > kMaxSmemBlock) return fail(DG_ERR_UNSUPPORTED);
    }
    op->variant = v;
    if (cells_per_block > 0) op->brick = cells_per_block;
    return DG_OK;
  }
  if (cells_per_block > 0) {
    if (v == DG_VARIANT_FUSED && cells_per_block * P * P > 1024) return fail(DG_ERR_UNSUPPORTED);
    const size_t per = v == DG_VARIANT_FUSED ? (size_t)(6 * P * P * P + 40 * P * P) * es
                                             : (size_t)(op->problem == DG_STOKES ? 12 : 4) * M * M * M * es;
    if (cells_per_block * per + 4096 > 200 * 1024) return fail(DG_ERR_UNSUPPORTED);
  }
  if (faces_per_block > 0 && (size_t)faces_per_block * 13 * M * M * es + 4096 > 200 * 1024) return fail(DG_ERR_UNSUPPORTED);
  op->variant = v;
  if (v == DG_VARIANT_FUSED) {
    if (cells_per_block > 0) op->tile = cells_per_block;
  } else {
    if (cells_per_block > 0) op->cpb = cells_per_block;
    if (faces_per_block > 0) op->fpb = faces_per_block;
  }
  return DG_OK;
}

// Mean per-kernel milliseconds of `reps` applies after `warm` untimed ones.
static dg_status time_kernels(dg_operator *op, const void *x, void *y, int nrhs, cudaStream_t s, int warm, int reps,
                              double ms[3]) {
  for (int i = 0; i < warm; ++i) {
    dg_status st = apply_impl(op, x, y, nrhs, s, false);
    if (st != DG_OK) return st;
  }
  const bool prof = op->prof;
  op->prof = true;
  op->prof_used = 0;
  for (int i = 0; i < reps; ++i) {
    dg_status st = apply_impl(op, x, y, nrhs, s, false);
    if (st != DG_OK) { op->prof = prof; return st; }
  }
  int64_t n = 0;
  dg_status st = dg_operator_kernel_times(op, ms, &n);
  op->prof = prof;
  if (st != DG_OK) return st;
  for (int k = 0; k < 3; ++k) ms[k] /= (double)(n > 0 ? n : 1);
  return DG_OK;
}

dg_status dg_operator_autotune(dg_operator *op, int nrhs, void *stream, dg_tune_result *out) {
  if (op && op->aniso) return fail(DG_ERR_UNSUPPORTED);
  if (!op || !out || nrhs < 1 || nrhs > op->max_rhs) return fail(DG_ERR_INVALID_ARG);
  memset(out, 0, sizeof(*out));
  const size_t es = op->precision == DG_FP64 ? 8 : 4;
  const size_t bytes = (size_t)nrhs * op->ndofs * es;
  void *x = nullptr, *y = nullptr;
  if (cudaMalloc(&x, bytes) != cudaSuccess || cudaMalloc(&y, bytes) != cudaSuccess) {
    cudaGetLastError();
    if (x) cudaFree(x);
    return fail(DG_ERR_OOM);
  }
  cudaStream_t s = (cudaStream_t)stream;
  dg_status st = DG_OK;
  const int M = op->m, M2 = M * M, M3 = M * M * M;
  const int save_v = op->variant, save_c = op->cpb, save_f = op->fpb, save_t = op->tile, save_b = op->brick;
  double ms[3];
  auto fits = [&](size_t smem) { return smem + 4096 <= 160 * 1024; };
  const bool stokes = op->problem == DG_STOKES;
  do {
    if (cudaMemsetAsync(x, 0, bytes, s) != cudaSuccess) { st = fail(DG_ERR_CUDA); break; }
    // default configuration, for reference (an operator set to the double-float variant
    // keeps it: only its blockings are tuned, the arithmetic is the caller's choice)
    const bool df = save_v == DG_VARIANT_DF64;
    op->variant = df ? DG_VARIANT_DF64 : resolve_variant(op, DG_VARIANT_AUTO);
    default_blocking(op);
    if ((st = time_kernels(op, x, y, nrhs, s, 2, 5, ms)) != DG_OK) break;
    out->ms_default = ms[0] + ms[1] + ms[2];
    // subproblem 1: cells per block of the cell-side kernels; subproblem 2: faces per block
    op->variant = df ? DG_VARIANT_DF64 : DG_VARIANT_THREE_KERNEL;
    default_blocking(op);
    double best_cell = 1e30, best_face = 1e30;
    int bc = op->cpb, bf = op->fpb;
    const int cand_c[] = {1, 2, 4, 8, 16, 32};
    const int cand_f[] = {2, 4, 8, 16, 32, 64};
    for (int i = 0; i < 6 && st == DG_OK; ++i) {
      const int c = cand_c[i];
      const size_t per = (size_t)(stokes ? 12 : 4) * M3 * es + (stokes ? 42 : 12) * M2 * es;
      if (!fits(c * per) || c * M3 > 8192) continue;
      op->cpb = c;
      if ((st = time_kernels(op, x, y, nrhs, s, 1, 3, ms)) != DG_OK) break;
      ++out->candidates;
      if (ms[0] + ms[2] < best_cell) { best_cell = ms[0] + ms[2]; bc = c; }
    }
    op->cpb = bc;
    for (int i = 0; i < 6 && st == DG_OK; ++i) {
      const int f = cand_f[i];
      if (!fits((size_t)f * 13 * M2 * es) || f * M2 > 8192) continue;
      op->fpb = f;
      if ((st = time_kernels(op, x, y, nrhs, s, 1, 3, ms)) != DG_OK) break;
      ++out->candidates;
      if (ms[1] < best_face) { best_face = ms[1]; bf = f; }
    }
    if (st != DG_OK) break;
    op->fpb = bf;
    if ((st = time_kernels(op, x, y, nrhs, s, 1, 5, ms)) != DG_OK) break;
    double best = ms[0] + ms[1] + ms[2];
    int bv = op->variant, btile = save_t;
    if (fused_ok(op) && !df) {
      op->variant = DG_VARIANT_FUSED;
      const int cand_t[] = {2, 4, 8, 16, 32, 64};
      const int P = op->p;
      for (int i = 0; i < 6 && st == DG_OK; ++i) {
        const int t = cand_t[i];
        if (!fits((size_t)t * (6 * P * P * P + 40 * P * P) * es) || t * P * P > 1024) continue;
        op->tile = t;
        if ((st = time_kernels(op, x, y, nrhs, s, 1, 5, ms)) != DG_OK) break;
        ++out->candidates;
        if (ms[0] + ms[1] + ms[2] < best) { best = ms[0] + ms[1] + ms[2]; bv = DG_VARIANT_FUSED; btile = t; }
      }
    }
    if (st != DG_OK) break;
    int bbrick = save_b;
    if (cellwise_ok(op) && !df) {
      op->variant = DG_VARIANT_CELLWISE;
      const int cand_b[] = {64, 128, 256};
      for (int i = 0; i < 3 && st == DG_OK; ++i) {
        const size_t sm = cellwise_smem_bytes(op->p, cand_b[i], (int)es);
        if (sm == 0 || sm > kMaxSmemBlock) continue;
        op->brick = cand_b[i];
        if ((st = time_kernels(op, x, y, nrhs, s, 1, 5, ms)) != DG_OK) break;
        ++out->candidates;
        if (ms[0] + ms[1] + ms[2] < best) { best = ms[0] + ms[1] + ms[2]; bv = DG_VARIANT_CELLWISE; bbrick = cand_b[i]; }
      }
    }
    if (st != DG_OK) break;
    int bgeo = op->geo;
    if (op->geo == GEO_STORED && op->problem == DG_SCALAR && op->m == op->p && !df) {
      op->geo = GEO_RECOMPUTE;  // stored vs recomputed per-point geometry
      op->cpb = bc;
      op->fpb = bf;
      if ((st = time_kernels(op, x, y, nrhs, s, 1, 3, ms)) != DG_OK) { op->geo = GEO_STORED; break; }
      ++out->candidates;
      if (ms[0] + ms[1] + ms[2] < best) { best = ms[0] + ms[1] + ms[2]; bgeo = GEO_RECOMPUTE; bv = DG_VARIANT_THREE_KERNEL; }
      op->geo = GEO_STORED;
    }
    op->geo = bgeo;
    op->variant = bv;
    op->cpb = bc;
    op->fpb = bf;
    op->tile = btile;
    op->brick = bbrick;
    out->variant = bv;
    out->cells_per_block = bv == DG_VARIANT_FUSED ? btile : (bv == DG_VARIANT_CELLWISE ? bbrick : bc);
    out->faces_per_block = (bv == DG_VARIANT_THREE_KERNEL || bv == DG_VARIANT_DF64) ? bf : 0;
    out->ms_best = best;
  } while (0);
  if (st != DG_OK) {
    op->variant = save_v; op->cpb = save_c; op->fpb = save_f; op->tile = save_t; op->brick = save_b;
  }
  cudaStreamSynchronize(s);
  cudaFree(x);
  cudaFree(y);
  return st;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Launch cost model: Sec. 4's heuristic cost function (cost = flops x ilp x loads with
// ilp = 1 + c0 log2(s) over the splitting s, loads = 1 + c1 log2(p) over the coefficients
// p, c0 = 0.5, c1 = 0.25) carried to the GPU. flops becomes the roofline time of a kernel
// from the exact work models, max(flops / peak of its precision, bytes / HBM bandwidth);
// the ILP term penalises latency that too few resident warps cannot hide,
// 1 + c0 log2(16 / warps per SM) below 16 warps (the occupancy calculator's count for the
// kernel at that blocking); the loads term keeps the paper's form with p = k+1, plus a
// fixed 50 ns per block (per work item for persistent kernels) and SM for what every block
// loads before its first useful operation (the reference tables, index setup, the first
// barrier; fitted on three workloads: one-cell blocks cost 0.2-0.4 ms more than 32-cell
// ones at 40^3 x 4 right-hand sides); and a tail term charges the last, partly empty wave
// of blocks (for persistent kernels, the last round of items). A configuration's cost is
// the sum over its kernels. The model ranks the blockings of one variant; it does not
// capture the latency-bound efficiency of the persistent FP32 variants, so the choice
// between variants is left to measurement.

namespace {

struct Candidate {
  int variant, cpb, fpb;  // cpb: cells per block, row tile (fused) or brick (cellwise)
};

constexpr double kClock = 2.07e9;   // maximum SM clock of this part
constexpr double kHBM = 6.6785e12;  // copy bandwidth measured on this part

double kernel_cost_ms(double flops, double bytes, const LaunchInfo &q, bool fp64, int p) {
  if (q.blocks_per_sm <= 0 || q.blocks <= 0) return 1e30;
  const double sms = (double)dg_device_sms();
  // 2 DFMA or 128 FFMA per SM per clock
  const double peak = sms * (fp64 ? 2.0 * 2.0 : 128.0 * 2.0) * kClock;
  const double t = fmax(flops / peak, bytes / kHBM);
  const double warps = (double)q.blocks_per_sm * ((q.threads + 31) / 32);
  const double ilp = 1.0 + 0.5 * log2(fmax(1.0, 16.0 / warps));
  const double loads = 1.0 + 0.25 * log2((double)p);
  double tail;
  if (q.items > q.blocks) {  // persistent: rounds of items over the grid
    const double r = (double)q.items / (double)q.blocks;
    tail = ceil(r) / r;
  } else {
    const double w = (double)q.blocks / ((double)q.blocks_per_sm * sms);
    tail = ceil(w) / w;
  }
  const double per_block = 50e-9 * (double)(q.items > q.blocks ? q.items : q.blocks) / sms;
  return (t * ilp * loads * tail + per_block) * 1e3;
}

void enumerate_candidates(const dg_operator *op, std::vector<Candidate> &c) {
  c.clear();
  const int cand_c[] = {1, 2, 4, 8, 16, 32}, cand_f[] = {2, 4, 8, 16, 32, 64};
  const size_t es = op->precision == DG_FP64 ? 8 : 4;
  const int M = op->m, M2 = M * M, M3 = M2 * M, P = op->p;
  const bool stokes = op->problem == DG_STOKES;
  for (int cc : cand_c) {
    const size_t per = (size_t)(stokes ? 12 : 4) * M3 * es + (stokes ? 42 : 12) * M2 * es;
    if (cc * per + 4096 > 160 * 1024 || cc * M3 > 8192) continue;
    for (int ff : cand_f) {
      if ((size_t)ff * 13 * M2 * es + 4096 > 160 * 1024 || ff * M2 > 8192) continue;
      c.push_back({DG_VARIANT_THREE_KERNEL, cc, ff});
    }
  }
  if (fused_ok(op))
    for (int t : {2, 4, 8, 16, 32, 64})
      if ((size_t)t * (6 * P * P * P + 40 * P * P) * es + 4096 <= 160 * 1024 && t * P * P <= 1024)
        c.push_back({DG_VARIANT_FUSED, t, 0});
  if (cellwise_ok(op))
    for (int b : {64, 128, 256}) {
      const size_t sm = cellwise_smem_bytes(P, b, (int)es);
      if (sm && sm <= kMaxSmemBlock) c.push_back({DG_VARIANT_CELLWISE, b, 0});
    }
}

template <typename T>
dg_status predict_t(const dg_operator *op, int nrhs, const Candidate &c, double *ms) {
  LaunchInfo q[3];
  double flops[3] = {0, 0, 0}, bytes[3] = {0, 0, 0};
  const int es = sizeof(T);
  cudaError_t e;
  int nk = 1;
  const ScalarArgs<T> a = scalar_args<T>(op, false);
  if (c.variant == DG_VARIANT_FUSED) {
    fused_work_model(op->p, op->ncell, op->nbface, flops, bytes, es);
    e = launch_fused_apply<T>(op->p, a, op->ht, nullptr, nullptr, nrhs, op->ndofs, c.cpb, 0, nullptr, nullptr, q);
  } else if (c.variant == DG_VARIANT_CELLWISE) {
    cellwise_work_model(op->p, op->nx, op->ny, op->nz, c.cpb, op->nbface, flops, bytes, es);
    e = launch_cellwise_apply<T>(op->p, a, op->ht, nullptr, nullptr, nrhs, op->ndofs, c.cpb, 0, nullptr, nullptr, q);
  } else {
    scalar_work_model(op->p, op->m, op->geo, op->kappa_vol != nullptr, op->ncell, op->nface, op->nbface, flops, bytes,
                      es);
    const int M2 = op->m * op->m, M3 = M2 * op->m;
    e = launch_scalar_apply<T>(op->p, op->m, op->geo, op->kappa_vol != nullptr, a, nullptr, nullptr, nullptr, nullptr,
                               nullptr, nrhs, op->ndofs, op->ncell * M3, op->ncell * 12 * M2, c.cpb, c.fpb, 0, nullptr,
                               q);
    nk = 3;
  }
  if (e != cudaSuccess) {
    // a configuration that cannot launch (its shared-memory or occupancy query failed):
    // clear the runtime's last-error state, which the next launch would otherwise report
    cudaGetLastError();
    return fail(DG_ERR_CUDA);
  }
  double t = 0.0;
  for (int k = 0; k < nk; ++k) t += kernel_cost_ms(flops[k] * nrhs, bytes[k] * nrhs, q[k], es == 8, op->p);
  *ms = t;
  return DG_OK;
}

dg_status predict(const dg_operator *op, int nrhs, const Candidate &c, double *ms) {
  if (op->problem != DG_SCALAR || op->geo == GEO_RECOMPUTE || op->aniso) return fail(DG_ERR_UNSUPPORTED);
  if (!variant_ok(op, c.variant)) return fail(DG_ERR_UNSUPPORTED);
  return op->precision == DG_FP64 ? predict_t<double>(op, nrhs, c, ms) : predict_t<float>(op, nrhs, c, ms);
}

// Applies op in configuration c a few times on scratch vectors; mean CUDA-event time.
dg_status time_candidate(dg_operator *op, int nrhs, const Candidate &c, const void *x, void *y, cudaStream_t s,
                         double *ms) {
  const int sv = op->variant, sc = op->cpb, sf = op->fpb, st = op->tile, sb = op->brick;
  op->variant = c.variant;
  if (c.variant == DG_VARIANT_FUSED) op->tile = c.cpb;
  else if (c.variant == DG_VARIANT_CELLWISE) op->brick = c.cpb;
  else { op->cpb = c.cpb; op->fpb = c.fpb; }
  double k3[3];
  dg_status r = time_kernels(op, x, y, nrhs, s, 1, 3, k3);
  op->variant = sv; op->cpb = sc; op->fpb = sf; op->tile = st; op->brick = sb;
  if (r == DG_OK) *ms = k3[0] + k3[1] + k3[2];
  return r;
}

bool scratch_vectors(const dg_operator *op, int nrhs, void **x, void **y, cudaStream_t s) {
  const size_t bytes = (size_t)nrhs * op->ndofs * (op->precision == DG_FP64 ? 8 : 4);
  *x = *y = nullptr;
  if (cudaMalloc(x, bytes) != cudaSuccess || cudaMalloc(y, bytes) != cudaSuccess ||
      cudaMemsetAsync(*x, 0, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    if (*x) cudaFree(*x);
    if (*y) cudaFree(*y);
    *x = *y = nullptr;
    return false;
  }
  return true;
}

}  // namespace

extern "C" {

dg_status dg_operator_predict(const dg_operator *op, int nrhs, int variant, int cells_per_block, int faces_per_block,
                              double *ms) {
  if (!op || !ms || nrhs < 1 || nrhs > op->max_rhs || cells_per_block < 1) return fail(DG_ERR_INVALID_ARG);
  if (variant == DG_VARIANT_THREE_KERNEL && faces_per_block < 1) return fail(DG_ERR_INVALID_ARG);
  if (variant == DG_VARIANT_CELLWISE) {
    const size_t sm = cellwise_smem_bytes(op->p, cells_per_block, op->precision == DG_FP64 ? 8 : 4);
    if (sm == 0 || sm > kMaxSmemBlock) return fail(DG_ERR_UNSUPPORTED);
  }
  return predict(op, nrhs, {variant, cells_per_block, faces_per_block}, ms);
}

dg_status dg_operator_time(const dg_operator *op_c, int nrhs, int variant, int cells_per_block, int faces_per_block,
                           void *stream, double *ms) {
  dg_operator *op = const_cast<dg_operator *>(op_c);
  if (op && op->aniso) return fail(DG_ERR_UNSUPPORTED);
  if (!op || !ms || nrhs < 1 || nrhs > op->max_rhs || cells_per_block < 1) return fail(DG_ERR_INVALID_ARG);
  if ((variant == DG_VARIANT_THREE_KERNEL || variant == DG_VARIANT_DF64) && faces_per_block < 1)
    return fail(DG_ERR_INVALID_ARG);
  if (variant < DG_VARIANT_THREE_KERNEL || variant > DG_VARIANT_DF64 || !variant_ok(op, variant))
    return fail(DG_ERR_UNSUPPORTED);
  if (variant == DG_VARIANT_DF64) {
    const dg_status st = ensure_df64(op);
    if (st != DG_OK) return st;
  }
  if (variant == DG_VARIANT_CELLWISE) {
    const size_t sm = cellwise_smem_bytes(op->p, cells_per_block, op->precision == DG_FP64 ? 8 : 4);
    if (sm == 0 || sm > kMaxSmemBlock) return fail(DG_ERR_UNSUPPORTED);
  }
  cudaStream_t s = (cudaStream_t)stream;
  void *x, *y;
  if (!scratch_vectors(op, nrhs, &x, &y, s)) return fail(DG_ERR_OOM);
  dg_status r = time_candidate(op, nrhs, {variant, cells_per_block, faces_per_block}, x, y, s, ms);
  cudaStreamSynchronize(s);
  cudaFree(x);
  cudaFree(y);
  return r;
}

dg_status dg_operator_autotune_prior(dg_operator *op, int nrhs, int measure, void *stream, dg_tune_result *out) {
  if (!op || !out || nrhs < 1 || nrhs > op->max_rhs || measure < 1) return fail(DG_ERR_INVALID_ARG);
  if (op->problem != DG_SCALAR || op->geo == GEO_RECOMPUTE || op->aniso) return fail(DG_ERR_UNSUPPORTED);
  memset(out, 0, sizeof(*out));
  std::vector<Candidate> cand;
  enumerate_candidates(op, cand);
  std::vector<std::pair<double, int>> ranked;
  for (size_t i = 0; i < cand.size(); ++i) {
    double ms;
    if (predict(op, nrhs, cand[i], &ms) == DG_OK) ranked.push_back({ms, (int)i});
  }
  dg_get_last_error();  // predictions of configurations that cannot launch are skipped
  if (ranked.empty()) return fail(DG_ERR_UNSUPPORTED);
  std::sort(ranked.begin(), ranked.end());
  cudaStream_t s = (cudaStream_t)stream;
  void *x, *y;
  if (!scratch_vectors(op, nrhs, &x, &y, s)) return fail(DG_ERR_OOM);
  dg_status st = DG_OK;
  double best = 1e30;
  int bi = -1;
  int taken[4] = {0, 0, 0, 0};  // per variant: its `measure` best-ranked blockings are timed
  for (size_t i = 0; i < ranked.size() && st == DG_OK; ++i) {
    const Candidate &c = cand[ranked[i].second];
    if (taken[c.variant] >= measure) continue;
    ++taken[c.variant];
    double ms;
    st = time_candidate(op, nrhs, c, x, y, s, &ms);
    if (st != DG_OK) break;
    ++out->candidates;
    if (ms < best) { best = ms; bi = ranked[i].second; }
  }
  if (st == DG_OK) {
    const Candidate &c = cand[bi];
    op->variant = c.variant;
    if (c.variant == DG_VARIANT_FUSED) op->tile = c.cpb;
    else if (c.variant == DG_VARIANT_CELLWISE) op->brick = c.cpb;
    else { op->cpb = c.cpb; op->fpb = c.fpb; }
    out->variant = c.variant;
    out->cells_per_block = c.cpb;
    out->faces_per_block = c.fpb;
    out->ms_best = best;
    out->ms_default = ranked[0].first;  // the model's own prediction for its first choice
  }
  cudaStreamSynchronize(s);
  cudaFree(x);
  cudaFree(y);
  return st;
}

dg_status dg_operator_profile(dg_operator *op, int enable) {
  if (!op) return fail(DG_ERR_INVALID_ARG);
  op->prof = enable != 0;
  op->prof_used = 0;
  return DG_OK;
}

dg_status dg_operator_kernel_times(dg_operator *op, double ms[3], int64_t *napplies) {
  if (!op || !ms) return fail(DG_ERR_INVALID_ARG);
  ms[0] = ms[1] = ms[2] = 0.0;
  for (size_t i = 0; i < op->prof_used; ++i) {
    const cudaEvent_t *e = op->prof_ev.data() + 4 * i;
    CK(cudaEventSynchronize(e[3]));
    for (int k = 0; k < 3; ++k) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, e[k], e[k + 1]));
      ms[k] += t;
    }
  }
  if (napplies) *napplies = (int64_t)op->prof_used;
  op->prof_used = 0;
  return DG_OK;
}

dg_status dg_reference_tables(int degree, int m, double *gauss_nodes, double *gauss_weights, double *gll_nodes,
                              double *interp, double *dcol, double *end_val, double *end_der) {
  HostTables t;
  if (m == 0) m = degree + 1;
  if (dg_build_tables(degree, m, false, &t)) return fail(DG_ERR_INVALID_ARG);
  for (int q = 0; q < m; ++q) {
    if (gauss_nodes) gauss_nodes[q] = t.gauss_s[q];
    if (gauss_weights) gauss_weights[q] = t.gauss_w[q];
    if (end_val) { end_val[q] = t.e0[q]; end_val[m + q] = t.e1[q]; }
    if (end_der) { end_der[q] = t.d0[q]; end_der[m + q] = t.d1[q]; }
  }
  for (int j = 0; j <= degree; ++j)
    if (gll_nodes) gll_nodes[j] = t.gll[j];
  if (interp) memcpy(interp, t.interp, sizeof(double) * m * (degree + 1));
  if (dcol) memcpy(dcol, t.dcol, sizeof(double) * m * m);
  return DG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Work model: floating-point operations the kernels execute (fma = 2, mul/add = 1) and
// the global-memory bytes each kernel must move at least once, per right-hand side.
// ---------------------------------------------------------------------------------------
void scalar_work_model(int P, int M, int geo, bool kappa, int64_t ncell, int64_t nface, int64_t nbface,
                       double flops[3], double bytes[3], int es) {
  const double P3 = P * P * P, M2 = M * M, M3 = M * M * M;
  const double contr = 2.0 * P - 1.0;   // one output of a length-P contraction
  const double contrM = 2.0 * M - 1.0;  // length-M contraction
  // k_cell: interpolation (3 sweeps), traces (12 M^2 outputs), gradient (3 per point),
  // pointwise flux, transposed derivative with the mass term
  double cell = (P * P * M + P * M2 + M3) * contr + 12.0 * M2 * contrM + 3.0 * M3 * contrM;
  if (geo == GEO_AFFINE) cell += M3 * (8.0 + (kappa ? 1.0 : 0.0)) + M3 * (4.0 + 6.0 * M);
  else cell += M3 * (15.0 + (kappa ? 3.0 : 0.0)) + M3 * (1.0 + 6.0 * M);
  const double ninner = (double)(nface - nbface);
  double face;
  if (geo == GEO_AFFINE) {
    face = ninner * M2 * (kappa ? 17.0 : 13.0) + (double)nbface * M2 * 10.0;
  } else {
    const double inner_pt = 2 * 2 * contrM + 10.0 + 1.0 + (kappa ? 4.0 : 2.0) + 3.0 + 2.0 + (kappa ? 2.0 : 0.0) + 6.0 + 8.0 * M;
    const double bnd_pt = 2 * contrM + 5.0 + 3.0 + 4.0 + 4.0 * M;
    face = ninner * M2 * inner_pt + (double)nbface * M2 * bnd_pt;
  }
  double back = M3 * 24.0 + (M2 * P + M * P * P + P3) * contrM;
  flops[0] = cell * (double)ncell;
  flops[1] = face;
  flops[2] = back * (double)ncell;
  const double geo_vol = geo == GEO_AFFINE ? 0.0 : 7.0 * M3;
  const double geo_face = geo == GEO_AFFINE ? 0.0 : 7.0 * M2;
  bytes[0] = es * (double)ncell * (P3 + M3 + 12.0 * M2 + geo_vol + (kappa ? M3 : 0.0));
  bytes[1] = es * (ninner * (8.0 * M2 + geo_face + (kappa ? 2.0 * M2 : 0.0)) +
                   (double)nbface * (4.0 * M2 + geo_face + (kappa ? M2 : 0.0)));
  bytes[2] = es * (double)ncell * (M3 + 12.0 * M2 + P3);
}

void stokes_work_model(int P, int64_t ncell, int64_t nface, int64_t nbface, double flops[3], double bytes[3], int es) {
  const int M = P, PP = P - 1;
  const double M2 = M * M, M3 = M * M * M, P3 = P * P * P, PP3 = PP * PP * PP;
  const double cP = 2.0 * P - 1.0, cPP = 2.0 * PP - 1.0, cM = 2.0 * M - 1.0;
  double cell = (M * PP * PP + M2 * PP + M3) * cPP;  // pressure to the Gauss points
  cell += 3.0 * ((P * P * M + P * M2 + M3) * cP + 12.0 * M2 * cM + 3.0 * M3 * cM + 15.0 * M3 + (6.0 * M - 1.0) * M3);
  cell += 6.0 * M2 * cM + 4.0 * M3;
  const double ninner = (double)(nface - nbface);
  const double face = ninner * M2 * (2.0 + 3.0 * 11.0 + 3.0) + (double)nbface * M2 * (3.0 * 9.0 + 5.0);
  double back = 3.0 * (24.0 * M3 + (M2 * P + M * P * P + P3) * cM) + 12.0 * M3 + (M2 * PP + M * PP * PP + PP3) * cM;
  flops[0] = cell * (double)ncell;
  flops[1] = face;
  flops[2] = back * (double)ncell;
  bytes[0] = es * (double)ncell * (3 * P3 + PP3 + 4 * M3 + 42 * M2);
  bytes[1] = es * (ninner * 2.0 * 2.0 * 42 * M2 + (double)nbface * 2.0 * 42 * M2) / 2.0;
  bytes[2] = es * (double)ncell * (4 * M3 + 42 * M2 + 3 * P3 + PP3);
}

// Fused single-pass variant: per cell, the neighbours' face data, interpolation, traces,
// gradient, pointwise flux, transposed derivative, the six own-side face terms, lifting
// and transposed interpolation; all of it in kernel 0. Bytes: x read and y written.
void fused_work_model(int P, int64_t ncell, int64_t nbface, double flops[3], double bytes[3], int es) {
  const double M = P, P2 = P * P, P3 = P * P * P, M2 = M * M, M3 = M * M * M;
  const double cP = 2.0 * P - 1.0, cM = 2.0 * M - 1.0;
  const double nbfaces = 6.0 * (double)ncell - (double)nbface;  // own faces with a neighbour
  double f = nbfaces * P2 * cP;                                // neighbour normal derivative
  f += (double)ncell * 12.0 * (P * M + M2) * cP;               // neighbour tangential sweeps
  double cell = (P2 * M + P * M2 + M3) * cP + 12.0 * M2 * cM + 3.0 * M3 * cM + 8.0 * M3 + (4.0 + 6.0 * M) * M3;
  cell += 6.0 * M2 * 12.0 + 24.0 * M3 + (M2 * P + M * P2 + P3) * cM;
  flops[0] = f + cell * (double)ncell;
  flops[1] = flops[2] = 0.0;
  bytes[0] = es * (double)ncell * 2.0 * P3;
  bytes[1] = bytes[2] = 0.0;
}

// Cellwise variant: per cell, interpolation, mass, per axis (gradient, pointwise flux,
// transposed derivative, four face rows per line, the two faces' terms and lifting),
// transposed interpolation; per brick-boundary face with a neighbour, the neighbour's
// normal derivative and two tangential sweeps of two quantities. Bytes: x read, y written.
void cellwise_work_model(int P, int nx, int ny, int nz, int brick, int64_t nbface, double flops[3], double bytes[3],
                         int es) {
  const double M = P, P2 = P * P, P3 = P * P * P, M2 = M * M, M3 = M * M * M;
  const double cP = 2.0 * P - 1.0, cM = 2.0 * M - 1.0;
  const double ncell = (double)nx * ny * nz;
  const int bx = 8, by = 4, bz = brick / 32 > 0 ? brick / 32 : 1;
  // faces between bricks (each evaluated from the neighbour's coefficients once per side)
  const double halo = 2.0 * ((double)((nx - 1) / bx) * ny * nz + (double)((ny - 1) / by) * nx * nz +
                             (double)((nz - 1) / bz) * nx * ny);
  const double per_halo = P2 * cP + 2.0 * (M * P + M2) * cP;
  // interpolation to u~ and back; per axis four weighted traces per line and the line
  // operator (axis 0 starts the residual, axes 1 and 2 accumulate)
  double cell = 2.0 * (P2 * M + P * M2 + M3) * cP;
  cell += 3.0 * 4.0 * M2 * cM + M3 * cM + 2.0 * M3 * 2.0 * M;
  const double own_sides = 6.0 * ncell - (double)nbface;  // interior own sides: neighbour coupling
  const double face = own_sides * M2 * 4.0 * M + (double)nbface * M3 * 2.0 * M;  // boundary: correction
  flops[0] = cell * ncell + face + halo * per_halo;
  flops[1] = flops[2] = 0.0;
  bytes[0] = es * ncell * 2.0 * P3;
  bytes[1] = bytes[2] = 0.0;
}
