// FP32 instantiation of the scalar apply kernels (FP32 storage and accumulation).
#include "dg_scalar_launch.cuh"

template cudaError_t launch_scalar_apply<float>(int, int, int, bool, const ScalarArgs<float> &, const float *,
                                                float *, float *, float *, float *, int, int64_t, int64_t,
                                                int64_t, int, int, cudaStream_t,
                                                 const cudaEvent_t *, LaunchInfo *, int, int64_t, int64_t,
                                               const HostTables *);
