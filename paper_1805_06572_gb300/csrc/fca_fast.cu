// Launchers of the FastFCA kernels (fca_fast.cuh): the fused EM kernel with 128 threads per
// CTA for both storages (FP32 eigensolver; the FP64 and refined ones are in fca_fast64.cu and
// fca_fast_refined.cu), and the posterior-mean kernel.
#include "fca_fast.cuh"

namespace fca {

int em_threads(int M, int N) { return 128; }

size_t em_dyn_smem(int M, int storage, int N) { return em_bin_smem(M, storage, N); }

bool em_resident(int M, int storage, int N) { return em_dyn_smem(M, storage, N) <= kResidentCap; }


bool fast_threads_batch(int storage, int threads) {
  return storage == 0 && (threads == 64 || threads == 128 || threads == 256);
}

cudaError_t launch_fast_em(int M, int storage, const FastEmArgs& a, cudaStream_t st, int threads) {
  if (a.bins) {
    if (!fast_threads_batch(storage, threads)) return cudaErrorInvalidValue;
    if (a.gevd_mode == 0) return launch_fast_batch_c64(M, a, st, threads);
    if (a.gevd_mode == 2 && threads != 64) return launch_fast_batch_c64_refined(M, a, st, threads);
    return cudaErrorInvalidValue;
  }
  if (threads != 128) return cudaErrorInvalidValue;
  if (a.gevd_mode == 1) return launch_fast_single_g64(M, storage, a, st);
  if (a.gevd_mode == 2) return launch_fast_single_refined(M, storage, a, st);
  if (a.gevd_mode != 0) return cudaErrorInvalidValue;
  return storage ? launch_fast_nt<1, 128, false>(M, a, st) : launch_fast_nt<0, 128, false>(M, a, st);
}

template <int M, int ST>
static cudaError_t launch_sep_fast_m(const SepFastArgs& a, cudaStream_t st) {
  dim3 grid(a.F, (a.N + 255) / 256);  // bins on x (no 65535 limit), frame chunks on y
  if (a.N <= 0 || a.F <= 0) return cudaSuccess;
  // Launched as a programmatic dependent of the separation-constant kernel before it, so its
  // CTAs start (and fetch y and v) while that kernel finishes.
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, sep_fast_kernel<M, ST>, a);
}

template <int ST>
static cudaError_t launch_sep_fast_s(int M, const SepFastArgs& a, cudaStream_t st) {
  switch (M) {
    case 1: return launch_sep_fast_m<1, ST>(a, st);
    case 2: return launch_sep_fast_m<2, ST>(a, st);
    case 3: return launch_sep_fast_m<3, ST>(a, st);
    case 4: return launch_sep_fast_m<4, ST>(a, st);
    case 5: return launch_sep_fast_m<5, ST>(a, st);
    case 6: return launch_sep_fast_m<6, ST>(a, st);
    case 7: return launch_sep_fast_m<7, ST>(a, st);
    case 8: return launch_sep_fast_m<8, ST>(a, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sep_fast(int M, int storage, const SepFastArgs& a, cudaStream_t st) {
  return storage ? launch_sep_fast_s<1>(M, a, st) : launch_sep_fast_s<0>(M, a, st);
}

}  // namespace fca
