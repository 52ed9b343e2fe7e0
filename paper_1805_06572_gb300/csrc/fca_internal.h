// Internal interface between the C-ABI layer (fca_api.cu) and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fca {

// Default sweep cap of the Jacobi eigensolver (FCA_ERR_EIG_NOCONV past it) and default
// precision mode of FastFCA's per-bin eigensolver and Gram merge (FCA_GEVD_* of fca.h).
constexpr int kDefaultSweeps = 30;
constexpr int kDefaultGevdMode = 2;  // FCA_GEVD_DEFAULT

// One frequency bin of a batch of mixtures: where its time-frequency points and source
// powers live, and which entry of the per-bin parameter arrays it owns. A kernel given a
// descriptor table handles bins[blockIdx] instead of bin f = blockIdx of one mixture whose
// arrays have the [F][N][M] / [2][F][N] layouts.
struct BinDesc {
  long long y_off;          // element offset of the bin's first point in y (16-byte aligned)
  long long x_off;          // element offset of the bin's first point in x1, x2
  long long v1_off;         // offset of v_1(0, bin) in the v arrays
  long long v2_off;         // offset of v_2(0, bin)
  int N;                    // frames of the bin's mixture
  int b;                    // index into the per-bin parameter arrays ([F] = bins of the class)
};

// Shared-memory bytes that keep one bin's mixture and source powers on chip for a run.
__host__ __device__ inline size_t em_bin_smem(int M, int storage, int N) {
  const size_t esz = storage ? 4 : 8;
  return (((size_t)N * M * esz + 15) & ~(size_t)15) + 8 * (size_t)N;
}

// Arguments of the fused FastFCA EM kernel (one CTA per frequency bin, all iterations).
struct FastEmArgs {
  int F, N, iters;
  int res_bytes;            // dynamic shared memory of the launch; a bin whose em_bin_smem
                            // fits is staged on chip for the run, others stream from memory
  const BinDesc* bins;      // nullptr: one mixture, bin f = blockIdx.x
  int nbins;                // with bins: CTAs of the launch (descriptors in bins)
  const void* y;            // complex64 or FP16 pairs, [F][N][M]
  const float* ginv;        // [F] decode scale 1/g_f (FP16 storage), else unused
  const float* vfloor;      // [F]
  const float* v_in;        // initial v, same layout as v (may be v itself)
  float* v;                 // [2][F][N] out (in when v_in == v)
  float* v_prev;            // [2][F][N] out: v before the last iteration
  double2* P;               // [F][M][M] in/out (FP64)
  double* lam;              // [F][M] in/out
  double* logdetS2;         // [F] in/out: log det S2 = -log|det P|^2
  double2* P_prev;          // parameters before the last iteration
  double* lam_prev;
  double* logdetS2_prev;
  double* llf;              // [iters][F] out: per-bin log-likelihood of every iteration
  int* status;
  int max_sweeps;           // Jacobi sweep cap of the per-bin eigensolver
  int gevd_mode;            // eigensolver precision mode (FCA_GEVD_*; modes 1, 2 one mixture only)
};

// Arguments of the fused conventional EM kernel (one CTA per frequency bin).
struct ConvEmArgs {
  int F, N, iters;
  int res_bytes;
  const BinDesc* bins;
  int nbins;
  const void* y;
  const float* ginv;
  const float* vfloor;
  const float* v_in;
  float* v;
  float* v_prev;
  const double2* S_in;      // [2][F][M][M] initial S (may be S itself)
  double2* S;               // [2][F][M][M] out (FP64)
  double2* S_prev;          // [2][F][M][M] out
  double* llf;              // [iters][F]
  int* status;
  int layout;               // FCA_CONV_AUTO / _THREAD / _GROUP (fca.h)
};

// Posterior-mean outputs.
struct SepFastArgs {
  int F, N;                 // with bins: F = number of bins, N = largest N of a bin
  const BinDesc* bins;
  const void* y;
  const float* ginv;
  const float* v;           // [2][F][N] parameters used
  const float2* PH;         // [F][M][M] FP32 P^H (times the decode scale)
  const float2* PinvH;      // [F][M][M] FP32 P^-H
  const float* lam;         // [F][M]
  float2* x1;               // [F][N][M]
  float2* x2;
};

struct SepConvArgs {
  int F, N;
  const BinDesc* bins;
  const void* y;
  const float* ginv;
  const float* v;
  const double2* S;         // [2][F][M][M]
  float2* x1;
  float2* x2;
  int* status;
};

// Per-frequency parameter kernels (FP64, one warp per bin).
struct ParamArgs {
  int F;
  const double2* S;         // [2][F][M][M]
  double2* P;               // [F][M][M]
  double* lam;              // [F][M]
  double* logdetS2;         // [F]
  double2* S_out;           // [2][F][M][M]
  const float* ginv;        // [F] or nullptr
  float2* PH;               // [F][M][M] (separation prep)
  float2* PinvH;            // [F][M][M]
  float* lam32;             // [F][M]
  int* status;
  int max_sweeps;           // gevd_from_S: Jacobi sweep cap
  int gevd_mode;            // gevd_from_S: FCA_GEVD_* (0 FP32, 1 FP64, 2 refined)
};

// Fused EM kernels. FastFCA: threads per CTA 128 for one mixture; 64, 128 or 256 for a
// batch (a.bins set, complex64 storage). Conventional: 128 threads per CTA.
cudaError_t launch_fast_em(int M, int storage, const FastEmArgs& a, cudaStream_t st, int threads = 128);
cudaError_t launch_conv_em(int M, int storage, const ConvEmArgs& a, cudaStream_t st);
cudaError_t launch_sep_fast(int M, int storage, const SepFastArgs& a, cudaStream_t st);
cudaError_t launch_sep_conv(int M, int storage, const SepConvArgs& a, cudaStream_t st);

// (S1, S2) -> (P, Lambda, log det S2) by the generalised eigenproblem (Eq. (GEVD)).
cudaError_t launch_gevd_from_S(int M, const ParamArgs& a, cudaStream_t st);
// (P, Lambda) -> S_j = P^-H T_j P^-1 (Eqs. (Sdiag), (recoverS)) into a.S_out.
cudaError_t launch_S_from_P(int M, const ParamArgs& a, cudaStream_t st);
// (P, Lambda) -> FP32 P^H (scaled), P^-H and Lambda for the separation kernel.
cudaError_t launch_sep_prep(int M, const ParamArgs& a, cudaStream_t st);

// Positivity floor of v and conversion of the initial v (bins: nullptr for one mixture,
// else F = number of bins and the descriptors give each bin's N and offsets).
// Optional work fused into the prepare pass (single-mixture layout only, bins == nullptr):
//   y_copy  receives a copy of y in the same layout (nullptr: none);
//   S       when set, one warp of each bin's CTA solves the generalised eigenproblem of
//           (S1, S2) into (P, lam, logdetS2) exactly as launch_gevd_from_S does, while the
//           other warps stream y, and copies the bin's (S1, S2) to S_copy when that is set.
struct PrepareExtra {
  void* y_copy;
  const double2* S;
  double2* S_copy;
  double2* P;
  double* lam;
  double* logdetS2;
  int max_sweeps;           // Jacobi sweep cap of the eigensolver
  int gevd_mode;            // FCA_GEVD_* (0 FP32, 1 FP64, 2 refined)
};
cudaError_t launch_prepare(int M, int storage, int F, int N, const void* y, const float* ginv,
                           const double* v0, float* v, float* vfloor, int* status,
                           cudaStream_t st, const BinDesc* bins = nullptr,
                           const PrepareExtra* extra = nullptr);
// out[mix_id[k] * iters + l] = sum of llf[l][b] over b in [b0[k], b0[k] + nb[k]), fixed order.
cudaError_t launch_ll_ranges(int nmix, int iters, int F, const double* llf, const int* b0,
                             const int* nb, const int* mix_id, double* out, cudaStream_t st);
// ll[l] = sum_f llf[l][f], fixed order.
cudaError_t launch_ll_reduce(int F, int iters, const double* llf, double* ll, cudaStream_t st);
// ginv[f] = 1 / g[f].
cudaError_t launch_invert_scale(int F, const float* g, float* ginv, cudaStream_t st);
// The seeded initial values of one mixture [F][N][M] (storage 0: complex64, 1: FP16 pairs
// decoded by 1/g[f]): S0 into S [2][F][M][M], v0 into v0 [2][F][N] (fca_problem, fca.h).
cudaError_t launch_seeded_init(int M, int storage, int F, int N, const void* y, const float* g,
                               unsigned long long seed, double2* S, double* v0, cudaStream_t st);
// FP16 storage of a complex64 mixture, NM values per bin: g[f] and the FP16 pairs into y16.
cudaError_t launch_encode_f16(int F, int NM, const void* y, void* y16, float* g, cudaStream_t st);

// Count n kernel launches in the process-wide counter behind fca_kernel_launches().
void note_launches(int n);

// Threads per CTA and shared-memory plan of the fused EM kernels (also used by the
// benchmark's roofline accounting).
int em_threads(int M, int N);
size_t em_dyn_smem(int M, int storage, int N);
bool em_resident(int M, int storage, int N);
// Largest dynamic shared memory a fused EM launch asks for by default (one mixture).
constexpr size_t kResidentCap = 100 * 1024;

}  // namespace fca
