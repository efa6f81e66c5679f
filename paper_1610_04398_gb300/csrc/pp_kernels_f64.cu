// Instantiation of the pressure-recovery kernels for T = double.
#define PP_REAL double
#include "pp_kernels.cuh"

namespace pp {

template cudaError_t launch_rhs_p2m<double>(const Tree<double>&, const double*, const double*, const double*, const double*,
                                         const double*, double, double, double*, cudaStream_t, int*);
template cudaError_t launch_upward<double>(const Tree<double>&, cudaStream_t);
template bool leaf_l2p_ok<double>(const Tree<double>&, const void*);
template cudaError_t launch_leaf_l2p<double>(const Tree<double>&, double*, cudaStream_t);
template bool down_tree_ok<double>(const Tree<double>&, const void*);
template cudaError_t launch_m2l_far<double>(const Tree<double>&, cudaStream_t);
template cudaError_t launch_down_tree<double>(const Tree<double>&, double*, cudaStream_t);
template int upward_launches<double>(const Tree<double>&);
template cudaError_t launch_downward<double>(const Tree<double>&, cudaStream_t);
template cudaError_t launch_leaf_eval<double>(const Tree<double>&, double*, cudaStream_t);
template cudaError_t launch_surface<double>(const Tree<double>&, const double*, const double*, const SurfaceArgs&,
                                         cudaStream_t);
template cudaError_t launch_export_expansion<double>(const Tree<double>&, int, int, double*, cudaStream_t);

}  // namespace pp

namespace pp {
template cudaError_t prepare_kernels<double>();
template size_t plan_smem_bytes<double>(const Tree<double>&);
}  // namespace pp

namespace pp {
template cudaError_t launch_downward_levels<double>(const Tree<double>&, int, int, double*, cudaStream_t);
template bool split_solve_ok<double>(const Tree<double>&);
template cudaError_t launch_near_only<double>(const Tree<double>&, double*, cudaStream_t);
}  // namespace pp
