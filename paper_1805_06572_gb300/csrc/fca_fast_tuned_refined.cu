// The FastFCA EM kernel for batches (descriptor tables, complex64 storage) in the refined
// eigensolver mode, with 128 or 256 threads per CTA (the launch shapes the batch autotuner
// chooses between in that mode). A separate translation unit so that the library's objects
// compile in parallel.
#include "fca_fast.cuh"

namespace fca {

cudaError_t launch_fast_batch_c64_refined(int M, const FastEmArgs& a, cudaStream_t st, int threads) {
  switch (threads) {
    case 128: return launch_fast_nt<0, 128, true, 2>(M, a, st);
    case 256: return launch_fast_nt<0, 256, true, 2>(M, a, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fca
