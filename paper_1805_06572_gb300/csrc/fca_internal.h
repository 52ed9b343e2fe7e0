// Internal interface between the C-ABI layer (fca_api.cu) and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fca {

// Arguments of the fused FastFCA EM kernel (one CTA per frequency bin, all iterations).
struct FastEmArgs {
  int F, N, iters;
  int resident;             // 1: y and v of the bin are staged in shared memory for the run
  const void* y;            // complex64 or FP16 pairs, [F][N][M]
  const float* ginv;        // [F] decode scale 1/g_f (FP16 storage), else unused
  const float* vfloor;      // [F]
  float* v;                 // [2][F][N] in/out
  float* v_prev;            // [2][F][N] out: v before the last iteration
  double2* P;               // [F][M][M] in/out (FP64)
  double* lam;              // [F][M] in/out
  double* logdetS2;         // [F] in/out: log det S2 = -log|det P|^2
  double2* P_prev;          // parameters before the last iteration
  double* lam_prev;
  double* logdetS2_prev;
  double* llf;              // [iters][F] out: per-bin log-likelihood of every iteration
  int* status;
};

// Arguments of the fused conventional EM kernel (one CTA per frequency bin).
struct ConvEmArgs {
  int F, N, iters;
  int resident;
  const void* y;
  const float* ginv;
  const float* vfloor;
  float* v;
  float* v_prev;
  double2* S;               // [2][F][M][M] in/out (FP64)
  double2* S_prev;          // [2][F][M][M] out
  double* llf;              // [iters][F]
  int* status;
};

// Posterior-mean outputs.
struct SepFastArgs {
  int F, N;
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
};

cudaError_t launch_fast_em(int M, int storage, const FastEmArgs& a, cudaStream_t st);
cudaError_t launch_conv_em(int M, int storage, const ConvEmArgs& a, cudaStream_t st);
cudaError_t launch_sep_fast(int M, int storage, const SepFastArgs& a, cudaStream_t st);
cudaError_t launch_sep_conv(int M, int storage, const SepConvArgs& a, cudaStream_t st);

// (S1, S2) -> (P, Lambda, log det S2) by the generalised eigenproblem (Eq. (GEVD)).
cudaError_t launch_gevd_from_S(int M, const ParamArgs& a, cudaStream_t st);
// (P, Lambda) -> S_j = P^-H T_j P^-1 (Eqs. (Sdiag), (recoverS)) into a.S_out.
cudaError_t launch_S_from_P(int M, const ParamArgs& a, cudaStream_t st);
// (P, Lambda) -> FP32 P^H (scaled), P^-H and Lambda for the separation kernel.
cudaError_t launch_sep_prep(int M, const ParamArgs& a, cudaStream_t st);

// Positivity floor of v and conversion of the initial v.
cudaError_t launch_prepare(int M, int storage, int F, int N, const void* y, const float* ginv,
                           const double* v0, float* v, float* vfloor, int* status,
                           cudaStream_t st);
// ll[l] = sum_f llf[l][f], fixed order.
cudaError_t launch_ll_reduce(int F, int iters, const double* llf, double* ll, cudaStream_t st);
// ginv[f] = 1 / g[f].
cudaError_t launch_invert_scale(int F, const float* g, float* ginv, cudaStream_t st);

// Count n kernel launches in the process-wide counter behind fca_kernel_launches().
void note_launches(int n);

// Threads per CTA and shared-memory plan of the fused EM kernels (also used by the
// benchmark's roofline accounting).
int em_threads(int M, int N);
size_t em_dyn_smem(int M, int storage, int N);
bool em_resident(int M, int storage, int N);

}  // namespace fca
