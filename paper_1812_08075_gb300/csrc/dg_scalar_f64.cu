// FP64 instantiation of the scalar apply kernels.
#include "dg_scalar_launch.cuh"

template cudaError_t launch_scalar_apply<double>(int, int, int, bool, const ScalarArgs<double> &, const double *,
                                                 double *, double *, double *, double *, int, int64_t, int64_t,
                                                 int64_t, int, int, cudaStream_t,
                                                 const cudaEvent_t *, LaunchInfo *, int, int64_t, int64_t,
                                               const HostTables *);
