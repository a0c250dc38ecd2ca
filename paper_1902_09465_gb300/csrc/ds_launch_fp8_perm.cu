// ds_launch_fp8_perm.cu -- the dataset launch gathering from the FP8 copy
// with shared coordinates; see dataset_launch.cuh (one element type per translation
// unit, so the kernels compile in parallel).
#include "dataset_launch.cuh"

namespace knn {
template KNN_DS_LAUNCH_DECL(Perm<ElemFP8>);
}  // namespace knn
