// MG-aggregation kernel for sketch size k = 16.
#include "sweep_mg.cuh"

namespace cdk {
template cudaError_t launch_agg_k<16>(const AggArgs&, bool, int64_t, cudaStream_t);
}  // namespace cdk
