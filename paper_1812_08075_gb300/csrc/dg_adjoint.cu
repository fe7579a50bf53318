// FP64 instantiation of the adjoint kernels (kernels in dg_adjoint_kernels.cuh).
#include "dg_adjoint_kernels.cuh"

template cudaError_t launch_scalar_adjoint<double>(int, int, bool, const ScalarArgs<double> &, double, const double *,
                                                   const double *, double *, double *, double *, double *, double *,
                                                   double *, double *, int, int, cudaStream_t, const cudaEvent_t *,
                                                   int, double, bool);
