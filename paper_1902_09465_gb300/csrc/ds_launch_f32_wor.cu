// ds_launch_f32_wor.cu -- the dataset launch gathering from the F32 data with
// draws without replacement; see dataset_launch.cuh (one element type per
// translation unit, so the kernels compile in parallel).
#include "dataset_launch.cuh"

namespace knn {
template KNN_DS_LAUNCH_DECL(Wor<ElemF32>);
}  // namespace knn
