// ds_launch_bf16_pair.cu -- the dataset launch gathering from the BF16 copy
// with per-pair draws; see dataset_launch.cuh (one element type per translation
// unit, so the kernels compile in parallel).
#include "dataset_launch.cuh"

namespace knn {
template KNN_DS_LAUNCH_DECL(ElemBF16);
}  // namespace knn
