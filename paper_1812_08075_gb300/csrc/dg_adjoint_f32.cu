// FP32 instantiation of the adjoint kernels (kernels in dg_adjoint_kernels.cuh), used by FP32
// operators whose trilinear geometry is recomputed in the kernels (DG_GEOM_RECOMPUTE): their
// apply and transposed apply run these kernels with the forward or exchanged coefficients.
#include "dg_adjoint_kernels.cuh"

template cudaError_t launch_scalar_adjoint<float>(int, int, bool, const ScalarArgs<float> &, double, const float *,
                                                  const float *, float *, float *, float *, float *, float *, float *,
                                                  float *, int, int, cudaStream_t, const cudaEvent_t *, int, double,
                                                  bool);
