// Double-float instantiation of the adjoint kernels (kernels in dg_adjoint_kernels.cuh).
#include "dg_adjoint_kernels.cuh"

template cudaError_t launch_scalar_adjoint<df64>(int, int, bool, const ScalarArgs<df64> &, double, const double *,
                                                 const double *, double *, double *, double *, df64 *, df64 *, df64 *,
                                                 df64 *, int, int, cudaStream_t, const cudaEvent_t *, int, double, bool);
