// D2Q21 kernel set of the numerical (max-entropy) equilibrium with the FP32 Newton, FP64 populations;
// see d2q21.cuh.
#include "d2q21.cuh"

namespace lbm {

template KernelSet make_set<D2Q21M<true>, ST_F64, 16, 16, 1>();

cudaError_t upload_tables_d2q21_n32_f64(const double* w21, const double* H21) { return upload21_here(w21, H21); }

}  // namespace lbm
