// The FastFCA EM kernel for one mixture with the per-bin generalised eigenproblem (Cholesky and
// Jacobi) and the cross-warp Gram merge in FP64 (128 threads per CTA, both storages). A
// separate translation unit so that the library's objects compile in parallel.
#include "fca_fast.cuh"

namespace fca {

cudaError_t launch_fast_single_g64(int M, int storage, const FastEmArgs& a, cudaStream_t st) {
  return storage ? launch_fast_nt<1, 128, false, 1>(M, a, st) : launch_fast_nt<0, 128, false, 1>(M, a, st);
}

}  // namespace fca
