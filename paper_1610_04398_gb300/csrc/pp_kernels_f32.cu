// Instantiation of the pressure-recovery kernels for T = float.
#define PP_REAL float
#include "pp_kernels.cuh"

namespace pp {

template cudaError_t launch_rhs_p2m<float>(const Tree<float>&, const float*, const float*, const float*, const float*,
                                         const float*, double, double, float*, cudaStream_t, int*);
template cudaError_t launch_upward<float>(const Tree<float>&, cudaStream_t);
template bool leaf_l2p_ok<float>(const Tree<float>&, const void*);
template cudaError_t launch_leaf_l2p<float>(const Tree<float>&, float*, cudaStream_t);
template bool down_tree_ok<float>(const Tree<float>&, const void*);
template cudaError_t launch_m2l_far<float>(const Tree<float>&, cudaStream_t);
template cudaError_t launch_down_tree<float>(const Tree<float>&, float*, cudaStream_t);
template int upward_launches<float>(const Tree<float>&);
template cudaError_t launch_downward<float>(const Tree<float>&, cudaStream_t);
template cudaError_t launch_leaf_eval<float>(const Tree<float>&, float*, cudaStream_t);
template cudaError_t launch_surface<float>(const Tree<float>&, const float*, const float*, const SurfaceArgs&,
                                         cudaStream_t);
template cudaError_t launch_export_expansion<float>(const Tree<float>&, int, int, double*, cudaStream_t);

}  // namespace pp

namespace pp {
template cudaError_t prepare_kernels<float>();
template size_t plan_smem_bytes<float>(const Tree<float>&);
}  // namespace pp

namespace pp {
template cudaError_t launch_downward_levels<float>(const Tree<float>&, int, int, float*, cudaStream_t);
template bool split_solve_ok<float>(const Tree<float>&);
template cudaError_t launch_near_only<float>(const Tree<float>&, float*, cudaStream_t);
}  // namespace pp
