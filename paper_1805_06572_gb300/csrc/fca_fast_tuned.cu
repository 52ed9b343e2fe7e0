// The FastFCA EM kernel for batches (a descriptor table per launch, complex64 storage) with 64,
// 128 and 256 threads per CTA, the launch shapes the batch autotuner chooses between. A
// separate translation unit so that the library's objects compile in parallel.
#include "fca_fast.cuh"

namespace fca {

cudaError_t launch_fast_batch_c64(int M, const FastEmArgs& a, cudaStream_t st, int threads) {
  switch (threads) {
    case 64: return launch_fast_nt<0, 64, true>(M, a, st);
    case 128: return launch_fast_nt<0, 128, true>(M, a, st);
    case 256: return launch_fast_nt<0, 256, true>(M, a, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fca
