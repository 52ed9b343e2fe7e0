// Short-time Fourier transform front-end (fca_stft / fca_istft in fca.h): time-domain
// signals of M channels to the [F][N][M] complex64 mixture the EM works on, and back.
//
// The analysis of the paper's experiments (Table 1): frames of W samples, shift H, square-root
// Hann window w[k] = sin(pi k / W) (periodic), F = W/2 + 1 bins up to Nyquist. Frames are
// centred: frame n covers samples [n H - W/2, n H + W/2) (zeros outside the signal), so
// N = T / H + 1 frames cover every sample twice at H = W/2. Synthesis is weighted overlap-add
// with the same window: x(t) = sum_n w u_n / sum_n w^2, which inverts the analysis exactly
// wherever the denominator is positive (everywhere for H <= W/2).
//
// Each frame's real FFT of length W is a complex FFT of length W/2 on z[j] = u[2j] + i u[2j+1]
// (radix-2, shared memory, one CTA per frame and channel), split into the spectra of the even
// and odd samples and recombined with the twiddles exp(-2 pi i f / W). Twiddles come from
// sincospif. Synthesis first writes every windowed frame, then gathers each output sample from
// the frames that cover it in a fixed order (deterministic, no atomics).
#include <cuda_runtime.h>

#include <cstdint>

#include "fca.h"
#include "fca_internal.h"

namespace {

constexpr int kFftThreads = 256;

__device__ __forceinline__ float2 cmul_(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ unsigned bitrev(unsigned x, int bits) { return __brev(x) >> (32 - bits); }

// In-place radix-2 decimation-in-time FFT of length L = 2^bits in shared memory (the input
// already in bit-reversed order); sign -1 forward, +1 inverse (unnormalised).
__device__ void fft_smem(float2* a, int bits, float sign) {
  const int L = 1 << bits;
  for (int s = 1; s <= bits; ++s) {
    const int half = 1 << (s - 1);
    __syncthreads();
    for (int t = threadIdx.x; t < L / 2; t += blockDim.x) {
      const int grp = t >> (s - 1), pos = t & (half - 1);
      const int i0 = grp * 2 * half + pos, i1 = i0 + half;
      float sn, cs;
      sincospif(sign * (float)pos / (float)half, &sn, &cs);  // exp(sign 2 pi i pos / (2 half))
      const float2 b = cmul_(a[i1], make_float2(cs, sn));
      const float2 u = a[i0];
      a[i0] = make_float2(u.x + b.x, u.y + b.y);
      a[i1] = make_float2(u.x - b.x, u.y - b.y);
    }
  }
  __syncthreads();
}

// Analysis: CTA (n, m) transforms frame n of channel m into y[f][n][m], f = 0..W/2.
__global__ void __launch_bounds__(kFftThreads) stft_kernel(const float* __restrict__ x, long long T,
                                                          int M, int N, int W, int H, int bits,
                                                          float2* __restrict__ y) {
  extern __shared__ float2 z[];  // W/2 complex
  const int n = blockIdx.x, m = blockIdx.y;
  const int Wh = W / 2;
  const long long t0 = (long long)n * H - Wh;
  const float* xm = x + (long long)m * T;
  for (int j = threadIdx.x; j < Wh; j += blockDim.x) {
    float u[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int k = 2 * j + e;
      const long long t = t0 + k;
      const float s = (t >= 0 && t < T) ? xm[t] : 0.f;
      u[e] = sinpif((float)k / (float)W) * s;  // square-root periodic Hann
    }
    z[bitrev((unsigned)j, bits)] = make_float2(u[0], u[1]);
  }
  fft_smem(z, bits, -1.f);
  const int F = Wh + 1;
  for (int f = threadIdx.x; f < F; f += blockDim.x) {
    const float2 zf = z[f % Wh], zc = z[(Wh - f) % Wh];
    // E = (Z[f] + conj Z[Wh-f]) / 2, O = (Z[f] - conj Z[Wh-f]) / (2i), X = E + exp(-2 pi i f/W) O
    const float2 E = make_float2(0.5f * (zf.x + zc.x), 0.5f * (zf.y - zc.y));
    const float2 O = make_float2(0.5f * (zf.y + zc.y), -0.5f * (zf.x - zc.x));
    float sn, cs;
    sincospif(-2.f * (float)f / (float)W, &sn, &cs);
    const float2 X = make_float2(E.x + cs * O.x - sn * O.y, E.y + cs * O.y + sn * O.x);
    y[((long long)f * N + n) * M + m] = X;
  }
}

// Synthesis, step 1: CTA (n, m) inverts frame n of channel m (the inverse DFT of the spectrum
// extended by Hermitian symmetry, so a real frame) and writes w[k] u[k] into
// frames[(n M + m) W + k].
__global__ void __launch_bounds__(kFftThreads) istft_frames_kernel(const float2* __restrict__ y, int M,
                                                                  int N, int W, int bits,
                                                                  float* __restrict__ frames) {
  extern __shared__ float2 z[];
  const int n = blockIdx.x, m = blockIdx.y;
  const int Wh = W / 2;
  for (int f = threadIdx.x; f < Wh; f += blockDim.x) {
    float2 X = y[((long long)f * N + n) * M + m];
    float2 Xc = y[((long long)(Wh - f) * N + n) * M + m];  // X[Wh - f], f = 0 -> Nyquist
    if (f == 0) {  // a real signal's DC and Nyquist bins are real: their imaginary parts drop
      X.y = 0.f;
      Xc.y = 0.f;
    }
    // E = (X[f] + conj X[Wh-f]) / 2, O = (X[f] - conj X[Wh-f]) exp(2 pi i f / W) / 2, Z = E + i O
    const float2 E = make_float2(0.5f * (X.x + Xc.x), 0.5f * (X.y - Xc.y));
    const float2 D = make_float2(0.5f * (X.x - Xc.x), 0.5f * (X.y + Xc.y));
    float sn, cs;
    sincospif(2.f * (float)f / (float)W, &sn, &cs);
    const float2 O = make_float2(D.x * cs - D.y * sn, D.x * sn + D.y * cs);
    z[bitrev((unsigned)f, bits)] = make_float2(E.x - O.y, E.y + O.x);
  }
  fft_smem(z, bits, 1.f);
  const float scale = 1.f / (float)Wh;
  float* out = frames + ((long long)n * M + m) * W;
  for (int j = threadIdx.x; j < Wh; j += blockDim.x) {
    const float2 v = z[j];
    out[2 * j] = sinpif((float)(2 * j) / (float)W) * v.x * scale;
    out[2 * j + 1] = sinpif((float)(2 * j + 1) / (float)W) * v.y * scale;
  }
}

// Synthesis, step 2: x[m][t] = sum_n frames(n, m)[t - n H + W/2] / sum_n w^2, over the frames
// that cover t, in increasing n.
__global__ void istft_ola_kernel(const float* __restrict__ frames, int M, int N, int W, int H,
                                 long long T, float* __restrict__ x) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (t >= T) return;
  const int Wh = W / 2;
  // frame n covers t when 0 <= t - n H + Wh < W, i.e. (t + Wh - W) / H < n <= (t + Wh) / H
  long long lo = (t + Wh - W) / H + 1;
  if (t + Wh - W < 0) lo = 0;
  long long hi = (t + Wh) / H;
  if (hi > N - 1) hi = N - 1;
  float num = 0.f, den = 0.f;
  for (long long n = lo; n <= hi; ++n) {
    const int k = (int)(t - n * H + Wh);
    if (k < 0 || k >= W) continue;
    const float w = sinpif((float)k / (float)W);
    num += frames[(n * M + m) * W + k];
    den = fmaf(w, w, den);
  }
  x[(long long)m * T + t] = den > 0.f ? num / den : 0.f;
}

int log2_exact(int v) {
  int b = 0;
  while ((1 << b) < v) ++b;
  return (1 << b) == v ? b : -1;
}

bool stft_shape_ok(int M, long long T, int W, int H) {
  if (M < 1 || M > 8 || T < 1 || W < 16 || W > 8192 || log2_exact(W) < 0) return false;
  if (H < 1 || H > W / 2) return false;
  const long long N = T / H + 1;
  return N <= 0x7fffffffLL && (long long)(W / 2 + 1) * N * M < (1LL << 31);
}

bool is_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace

extern "C" {

int64_t fca_stft_frames(int64_t T, int32_t W, int32_t H) {
  if (!stft_shape_ok(1, T, W, H)) return 0;
  return T / H + 1;
}

fca_status fca_stft(int32_t M, int64_t T, const float* x_dev, int32_t W, int32_t H, void* y_dev,
                    void* cuda_stream) {
  if (!stft_shape_ok(M, T, W, H) || !x_dev || !y_dev) return FCA_ERR_ARG;
  if (!is_device(x_dev) || !is_device(y_dev)) return FCA_ERR_ARG;
  const int N = (int)(T / H + 1), bits = log2_exact(W / 2);
  stft_kernel<<<dim3(N, M), kFftThreads, (W / 2) * sizeof(float2), (cudaStream_t)cuda_stream>>>(
      x_dev, T, M, N, W, H, bits, static_cast<float2*>(y_dev));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return FCA_ERR_CUDA;
  fca::note_launches(1);
  return FCA_OK;
}

fca_status fca_istft(int32_t M, int32_t N, const void* y_dev, int32_t W, int32_t H,
                     float* frames_dev, float* x_dev, int64_t T, void* cuda_stream) {
  if (!stft_shape_ok(M, T, W, H) || N != (int32_t)(T / H + 1)) return FCA_ERR_ARG;
  if (!y_dev || !frames_dev || !x_dev) return FCA_ERR_ARG;
  if (!is_device(y_dev) || !is_device(frames_dev) || !is_device(x_dev)) return FCA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int bits = log2_exact(W / 2);
  istft_frames_kernel<<<dim3(N, M), kFftThreads, (W / 2) * sizeof(float2), st>>>(
      static_cast<const float2*>(y_dev), M, N, W, bits, frames_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return FCA_ERR_CUDA;
  istft_ola_kernel<<<dim3((unsigned)((T + 255) / 256), M), 256, 0, st>>>(frames_dev, M, N, W, H, T, x_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return FCA_ERR_CUDA;
  fca::note_launches(2);
  return FCA_OK;
}

}  // extern "C"
