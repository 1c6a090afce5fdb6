// MG-sketch sweep kernel for sketch size k = 64 (the large-sketch form: at most
// 32 streams per row, merges and candidate tables in shared memory; MG
// aggregation is offered up to k = 16).
#include "sweep_mg.cuh"

namespace cdk {
template cudaError_t launch_k<64>(const SweepArgs&, bool, int64_t, cudaStream_t);
}  // namespace cdk
