// MG-sketch sweep and MG-aggregation kernels for sketch size k = 4.
#include "sweep_mg.cuh"

namespace cdk {
template cudaError_t launch_k<4>(const SweepArgs&, bool, int64_t, cudaStream_t);
template cudaError_t launch_agg_k<4>(const AggArgs&, bool, int64_t, cudaStream_t);
}  // namespace cdk
