// The FastFCA EM kernel for one mixture with the FP64 Gram merge, the FP32 eigensolver and the
// compensated refinement of its basis (128 threads per CTA, both storages). A
// separate translation unit so that the library's objects compile in parallel.
#include "fca_fast.cuh"

namespace fca {

cudaError_t launch_fast_single_refined(int M, int storage, const FastEmArgs& a, cudaStream_t st) {
  return storage ? launch_fast_nt<1, 128, false, 2>(M, a, st) : launch_fast_nt<0, 128, false, 2>(M, a, st);
}

}  // namespace fca
