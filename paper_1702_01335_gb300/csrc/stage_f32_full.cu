// Stage kernel instantiations for float storage, the full 3D velocity set
// (all V and stages); one translation unit per (storage type, model) so that
// the four compile in parallel.
#include "kernels.cuh"

namespace lbs {

cudaError_t launch_stage_f32_full(int V, int stage, const InstDev* d, const Tile* t, int n, size_t smem,
                                  int fuse, cudaStream_t st)
{
    return launch_stage_m<float, false>(V, stage, d, t, n, smem, fuse, st);
}

}  // namespace lbs
