// Inputs the library can build itself from a mixture already on the device:
//   * the seeded initial parameters (Algorithm 1, first step, "set initial values", which the
//     paper leaves to the user): S_j^(0)(f) = b_j b_j^H + I with b_j(f) ~ CN(0, I_M) drawn from
//     a counter-based generator, and v_j^(0)(n, f) = max(|y(n, f)|^2, eps_f) / (2 tr S_j^(0)(f)),
//     eps_f = 1e-12 mean_n |y(n, f)|^2;
//   * the FP16 storage of a complex64 mixture with the per-frequency power scale
//     g_f = (mean_{n,m} |y_m(n, f)|^2)^(-1/2): the stored values are g_f y rounded to FP16.
// The generator is Philox4x64-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC 2011): draw t of source j takes the block of counter (t, 0, 0, 0) under
// the key (seed, 1000 + j); its first two words w0, w1 give u_k = (floor(w_k / 2^11) + 1/2) 2^-53
// in (0, 1) (exact in FP64) and b = sqrt(-ln u0) (cos 2 pi u1 + i sin 2 pi u1), a CN(0, 1) value
// (Box-Muller). Draw t = f M + m is entry m of b_j(f).
#include <cuda_fp16.h>

#include "fca_dev.cuh"
#include "fca_internal.h"

namespace fca {
namespace {

struct U64x4 {
  unsigned long long x[4];
};

// Philox4x64-10 block of counter c under key (k0, k1): ten rounds of two 64 x 64 -> 128-bit
// products, the key advanced by the Weyl constants between rounds.
__device__ U64x4 philox4x64_10(U64x4 c, unsigned long long k0, unsigned long long k1) {
  constexpr unsigned long long kM0 = 0xD2E7470EE14C6C93ull, kM1 = 0xCA5A826395121157ull;
  constexpr unsigned long long kW0 = 0x9E3779B97F4A7C15ull, kW1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long hi0 = __umul64hi(kM0, c.x[0]), lo0 = kM0 * c.x[0];
    const unsigned long long hi1 = __umul64hi(kM1, c.x[2]), lo1 = kM1 * c.x[2];
    U64x4 n;
    n.x[0] = hi1 ^ c.x[1] ^ k0;
    n.x[1] = lo1;
    n.x[2] = hi0 ^ c.x[3] ^ k1;
    n.x[3] = lo0;
    c = n;
    k0 += kW0;
    k1 += kW1;
  }
  return c;
}

// The CN(0, 1) draw t of source j (file comment).
__device__ double2 seeded_cn(unsigned long long seed, int j, unsigned long long t) {
  U64x4 c;
  c.x[0] = t;
  c.x[1] = c.x[2] = c.x[3] = 0ull;
  const U64x4 w = philox4x64_10(c, seed, 1000ull + (unsigned long long)j);
  const double u0 = ((double)(w.x[0] >> 11) + 0.5) * 0x1p-53;
  const double u1 = ((double)(w.x[1] >> 11) + 0.5) * 0x1p-53;
  const double r = sqrt(-log(u0));
  double s, co;
  sincos(6.283185307179586 * u1, &s, &co);
  return make_double2(r * co, r * s);
}

// Sum over the CTA's 256 threads in a fixed order (the same result for the same inputs).
__device__ double cta_sum_fixed(double v, double* part) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int tid = threadIdx.x;
  __syncthreads();
  if ((tid & 31) == 0) part[tid >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < 8; ++w) s += part[w];
  return s;
}

// |y|^2 of one stored value in FP64: exact squares of the stored parts (FP16 parts times the
// decode scale 1/g_f).
__device__ __forceinline__ double power64(float2 v, double gi) {
  const double re = (double)v.x * gi, im = (double)v.y * gi;
  return fma(re, re, im * im);
}

// One CTA (256 threads) per bin: S0 into S [2][F][M][M] and v0 into v0 [2][F][N].
template <int ST>
__global__ void __launch_bounds__(256) seeded_init_kernel(int M, int F, int N, const void* y,
                                                          const float* g, unsigned long long seed,
                                                          double2* S, double* v0) {
  using E = typename Elem<ST>::T;
  __shared__ double2 b[2][kMaxM];
  __shared__ double tr[2];
  __shared__ double part[8];
  const int f = blockIdx.x, tid = threadIdx.x;
  const size_t MM = (size_t)M * M;
  if (tid < 2 * M) {
    const int j = tid / M, m = tid % M;
    b[j][m] = seeded_cn(seed, j, (unsigned long long)f * M + m);
  }
  __syncthreads();
  for (int e = tid; e < 2 * (int)MM; e += 256) {
    const int j = e / (int)MM, r = e % (int)MM, m = r / M, k = r % M;
    const double2 p = b[j][m], q = b[j][k];  // p conj(q)
    double2 s = make_double2(p.x * q.x + p.y * q.y, p.y * q.x - p.x * q.y);
    if (m == k) s = make_double2(s.x + 1.0, 0.0);
    S[((size_t)j * F + f) * MM + r] = s;
  }
  if (tid < 2) {
    double t = 0.0;
    for (int m = 0; m < M; ++m) t += b[tid][m].x * b[tid][m].x + b[tid][m].y * b[tid][m].y + 1.0;
    tr[tid] = t;
  }
  // |y(n, f)|^2 into the first source's slot, then eps_f from their mean.
  const E* yf = reinterpret_cast<const E*>(y) + (size_t)f * N * M;
  const double gi = (ST == 1) ? 1.0 / (double)g[f] : 1.0;
  double* p1 = v0 + (size_t)f * N;
  double* p2 = v0 + ((size_t)F + f) * N;
  double acc = 0.0;
  for (int n = tid; n < N; n += 256) {
    double pw = 0.0;
    for (int m = 0; m < M; ++m) pw += power64(decode(yf[(size_t)n * M + m]), gi);
    p1[n] = pw;
    acc += pw;
  }
  const double eps = 1e-12 * (cta_sum_fixed(acc, part) / (double)N);
  const double i1 = 1.0 / (2.0 * tr[0]), i2 = 1.0 / (2.0 * tr[1]);
  for (int n = tid; n < N; n += 256) {  // each thread rereads only its own frames
    const double pw = fmax(p1[n], eps);
    p1[n] = pw * i1;
    p2[n] = pw * i2;
  }
}

// One CTA (256 threads) per bin: g_f from the bin's mean power, then the FP16 values.
__global__ void __launch_bounds__(256) encode_f16_kernel(int F, int NM, const float2* y, __half2* y16,
                                                         float* g) {
  __shared__ double part[8];
  const int f = blockIdx.x, tid = threadIdx.x;
  const float2* yf = y + (size_t)f * NM;
  double acc = 0.0;
  for (int i = tid; i < NM; i += 256) {
    const float2 v = yf[i];
    acc += fma((double)v.x, (double)v.x, (double)v.y * (double)v.y);
  }
  const double p = cta_sum_fixed(acc, part) / (double)NM;
  const float gf = p > 0.0 ? (float)(1.0 / sqrt(p)) : 1.0f;
  if (tid == 0) g[f] = gf;
  const double gd = (double)gf;
  __half2* of = y16 + (size_t)f * NM;
  for (int i = tid; i < NM; i += 256) {  // products exact in FP64, one rounding to FP16
    const float2 v = yf[i];
    of[i] = __halves2half2(__double2half((double)v.x * gd), __double2half((double)v.y * gd));
  }
}

}  // namespace

cudaError_t launch_seeded_init(int M, int storage, int F, int N, const void* y, const float* g,
                               unsigned long long seed, double2* S, double* v0, cudaStream_t st) {
  if (F <= 0) return cudaSuccess;
  if (M < 1 || M > kMaxM) return cudaErrorInvalidValue;
  if (storage)
    seeded_init_kernel<1><<<F, 256, 0, st>>>(M, F, N, y, g, seed, S, v0);
  else
    seeded_init_kernel<0><<<F, 256, 0, st>>>(M, F, N, y, g, seed, S, v0);
  return cudaGetLastError();
}

cudaError_t launch_encode_f16(int F, int NM, const void* y, void* y16, float* g, cudaStream_t st) {
  if (F <= 0) return cudaSuccess;
  encode_f16_kernel<<<F, 256, 0, st>>>(F, NM, static_cast<const float2*>(y), static_cast<__half2*>(y16), g);
  return cudaGetLastError();
}

}  // namespace fca
