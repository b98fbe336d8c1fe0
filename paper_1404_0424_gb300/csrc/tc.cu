// Launch of one bin of batched problems (plans and the static batch) on the
// warp-per-instance kernels: the exact tracker's kernels for exact-tracker
// detection bins, the approximate-tracker kernels otherwise.
#include "cg_tc.cuh"
#include "launch.cuh"

namespace cgm {

cudaError_t launch_batch_tc(int op, int UT, int el, bool x3, bool /*full*/, const BatchArgs& b,
                            int max_grid, cudaStream_t s, bool launch, uint32_t* smem_out,
                            int* grid_out) {
  if (smem_out) *smem_out = 0;
  if (b.PEX != 0 && op == 0)
    return launch_batch_warp_exact(UT, el, x3, b, max_grid, s, launch, grid_out);
  return launch_batch_warp(op, UT, el, x3, b, max_grid, s, launch, grid_out);
}

}  // namespace cgm
