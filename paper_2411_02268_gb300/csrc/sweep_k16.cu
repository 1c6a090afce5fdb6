// MG-sketch sweep kernel for sketch size k = 16 (its MG-aggregation kernel is
// in agg_k16.cu: each is a large translation unit, compiled in parallel).
#include "sweep_mg.cuh"

namespace cdk {
template cudaError_t launch_k<16>(const SweepArgs&, bool, int64_t, cudaStream_t);
}  // namespace cdk
