// Tensor-core products of the recursion (Alg. 2 lines 8-9). Placeholder dispatch to the
// CUDA-core kernels until the tcgen05 kernels are in place.
#include "common.cuh"
#include "kernels.cuh"

namespace lls {

int simt_projection_lowp(const ProjCall& c, cudaStream_t st);
int simt_update_lowp(const UpdCall& c, cudaStream_t st);
size_t simt_partial_floats(int m, int w1, int w2);

size_t proj_partial_floats(int m, int w1, int w2) { return simt_partial_floats(m, w1, w2); }
int gemm_projection(const ProjCall& c, cudaStream_t st) { return simt_projection_lowp(c, st); }
int gemm_update(const UpdCall& c, cudaStream_t st) { return simt_update_lowp(c, st); }

}  // namespace lls
