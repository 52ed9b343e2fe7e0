// Device building blocks shared by the FCA kernels (sm_103a).
//
//   * complex64 / complex128 arithmetic on float2 / double2;
//   * a warp "transpose" reduction: V per-lane partial sums -> each lane ends with V/32
//     complete warp sums (31 shuffles for 32 values instead of 160 for a butterfly each);
//   * dense Hermitian linear algebra for one frequency bin inside one warp (M <= 8):
//     Cholesky, triangular solves, cyclic Jacobi with the round-robin (parallel) ordering,
//     used for the generalised eigenproblem of Eq. (GEVD) in FP32 or FP64, plus FP64
//     matrix products for the basis update P <- P Q (Eq. (updatePeff));
//   * Newton-type steps for the generalised eigenbasis and their refinement with compensated
//     FP32 arithmetic (error-free transformations, Dot2) against FP64 pencils.
//
// Precision: on GB300 an FP64 FMA occupies a scheduler's FP64 pipe for ~64 cycles and FP64
// throughput is 1/74 of FP32 (measured), so a Jacobi solve in FP64 costs several times the
// per-bin pass of an EM iteration. The library's default (refined) eigensolver therefore runs
// FP32 steps and refines them with compensated FP32 arithmetic against the Grams merged as
// compensated FP32 pairs, which reaches the FP64 solver's accuracy; FP64 stays where sums or
// product chains are long: the log-likelihood sums and the accumulated basis P.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fca {

constexpr int kMaxM = 8;

// Device status codes (mirror fca_status in fca.h).
enum : int { kOk = 0, kErrNotPD = 4, kErrEigNoConv = 5, kErrNonFinite = 6 };

__device__ __forceinline__ void set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// ------------------------------------------------------------------------- complex64
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// conj(a) * b
__device__ __forceinline__ float2 ccmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
// a * b + c
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// ------------------------------------------------------------------------ complex128
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 zfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ float2 z2c(double2 a) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double2 c2z(float2 a) { return make_double2((double)a.x, (double)a.y); }

// ------------------------------------------------------------------ storage decoding
template <int ST> struct Elem;
template <> struct Elem<0> { typedef float2 T; };   // complex64
template <> struct Elem<1> { typedef __half2 T; };  // FP16 pair

__device__ __forceinline__ float2 decode(float2 v) { return v; }
__device__ __forceinline__ float2 decode(__half2 v) { return __half22float2(v); }

// Load the M-vector of one time-frequency point. `p` points at its first element.
template <int M, int ST>
__device__ __forceinline__ void load_bin(const typename Elem<ST>::T* p, float2 (&y)[M]) {
  if constexpr (ST == 0) {
    if constexpr ((M & 1) == 0) {
      const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
      for (int i = 0; i < M / 2; ++i) {
        float4 t = q[i];
        y[2 * i] = make_float2(t.x, t.y);
        y[2 * i + 1] = make_float2(t.z, t.w);
      }
    } else {
#pragma unroll
      for (int i = 0; i < M; ++i) y[i] = p[i];
    }
  } else {
    if constexpr ((M & 3) == 0) {
      const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
      for (int i = 0; i < M / 4; ++i) {
        uint4 t = q[i];
        const __half2* h = reinterpret_cast<const __half2*>(&t);
#pragma unroll
        for (int k = 0; k < 4; ++k) y[4 * i + k] = __half22float2(h[k]);
      }
    } else if constexpr ((M & 1) == 0) {
      const uint2* q = reinterpret_cast<const uint2*>(p);
#pragma unroll
      for (int i = 0; i < M / 2; ++i) {
        uint2 t = q[i];
        const __half2* h = reinterpret_cast<const __half2*>(&t);
        y[2 * i] = __half22float2(h[0]);
        y[2 * i + 1] = __half22float2(h[1]);
      }
    } else {
#pragma unroll
      for (int i = 0; i < M; ++i) y[i] = __half22float2(p[i]);
    }
  }
}

// ------------------------------------------------------------- accurate log of a product
// log of a product of positive normal floats, accumulated as (mantissa product, exponent sum)
// so that neither overflows: each factor contributes its mantissa in [1, 2) and its binary
// exponent; one correctly-rounded-to-1-ulp logf at the end replaces one approximate log per
// factor.
struct LogProd {
  float m = 1.f;
  int e = 0;
  __device__ __forceinline__ void mul(float x) {
    const int b = __float_as_int(x);
    e += (b >> 23) - 127;
    m *= __int_as_float((b & 0x007fffff) | 0x3f800000);
  }
  // Call at most every 8 factors (m < 2^8) to keep m in range.
  __device__ __forceinline__ float log() const { return logf(m) + 0.6931471805599453f * (float)e; }
  // Same value with the mantissa product renormalised to [1, 2), where the hardware log2
  // approximation has an absolute error of at most 2^-22.
  __device__ __forceinline__ float log_fast() const {
    const int b = __float_as_int(m);
    const float mm = __int_as_float((b & 0x007fffff) | 0x3f800000);
    return 0.6931471805599453f * (__log2f(mm) + (float)(e + (b >> 23) - 127));
  }
};

// ------------------------------------------------------------ warp transpose reduction
// acc[0..VP) holds this lane's partial sums (VP a multiple of 32). Afterwards lane l holds,
// in acc[0..VP/32), the warp-wide sums of values [l*VP/32, (l+1)*VP/32).
template <int VP>
__device__ __forceinline__ void warp_transpose_reduce(float* acc, int lane) {
  static_assert(VP % 32 == 0, "VP must be a multiple of 32");
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const int o = 16 >> r;
    const int h = VP >> (r + 1);
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      float send = up ? acc[j] : acc[j + h];
      float keep = up ? acc[j + h] : acc[j];
      acc[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
}

// As warp_transpose_reduce but over the lanes of equal parity only (levels xor 16, 8, 4, 2):
// afterwards lane l holds, in acc[0..VP/16), the sums over the 16 lanes of parity l & 1 of
// values [(l >> 1) VP/16, ((l >> 1) + 1) VP/16).
template <int VP>
__device__ __forceinline__ void warp_transpose_reduce_parity(float* acc, int lane) {
  static_assert(VP % 32 == 0, "VP must be a multiple of 32");
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int o = 16 >> r;
    const int h = VP >> (r + 1);
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      float send = up ? acc[j] : acc[j + h];
      float keep = up ? acc[j + h] : acc[j];
      acc[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
}

// Shape of the per-lane partial-sum vector for V values: VT values go through the transpose
// reduction (a multiple of 32) and the last VR (at most 4) through plain butterflies, which is
// cheaper than padding a short tail to 32.
template <int V>
struct RedShape {
  static constexpr int kTail = V % 32;
  static constexpr int VT = (kTail <= 4) ? V - kTail : V - kTail + 32;
  static constexpr int VR = (kTail <= 4) ? kTail : 0;
  static constexpr int KP = VT / 32;     // transposed values held per lane after the reduction
  static constexpr int NA = VT + VR;     // length of the accumulator array
};

// Reduce acc[0..NA) over the warp and store the warp's V sums to out[0..V) (shared memory).
template <int V>
__device__ __forceinline__ void warp_reduce_store(float* acc, int lane, float* out) {
  using RS = RedShape<V>;
  if constexpr (RS::VR > 0) {
#pragma unroll
    for (int j = 0; j < RS::VR; ++j) {
      float x = acc[RS::VT + j];
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) out[RS::VT + j] = x;
    }
  }
  if constexpr (RS::VT > 0) {
    warp_transpose_reduce<RS::VT>(acc, lane);
#pragma unroll
    for (int j = 0; j < RS::KP; ++j)
      if (RS::KP * lane + j < V) out[RS::KP * lane + j] = acc[j];
  }
}

// Lane pairs: lanes of parity q hold one M x M Gram (MM values, Gram q) and the two
// log-likelihood sums (only parity 0 adds to them) in acc[0..MM+2). Reduce over the lanes of
// each parity and store the warp's sums in the usual layout out[0..2MM+2): Gram 1, Gram 2,
// then the two log-likelihood sums.
template <int MM>
__device__ __forceinline__ void warp_reduce_store_pairs(float* acc, int lane, float* out) {
  constexpr int VP = MM + 2;
  using RS = RedShape<VP>;
  const int q = lane & 1;
  auto put = [&](int v, float x) {
    if (v < MM) out[q * MM + v] = x;
    else if (v < VP && q == 0) out[2 * MM + (v - MM)] = x;
  };
  if constexpr (RS::VR > 0) {
#pragma unroll
    for (int j = 0; j < RS::VR; ++j) {
      float x = acc[RS::VT + j];
#pragma unroll
      for (int o = 16; o >= 2; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane < 2) put(RS::VT + j, x);
    }
  }
  if constexpr (RS::VT > 0) {
    warp_transpose_reduce_parity<RS::VT>(acc, lane);
    constexpr int KP = RS::VT / 16;
#pragma unroll
    for (int j = 0; j < KP; ++j) put((lane >> 1) * KP + j, acc[j]);
  }
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// ------------------------------------------------------- precision of the per-bin solver
// The per-bin linear algebra below runs in FP32 (T = float, complex float2) or FP64 (T =
// double, complex double2), chosen at compile time; the formulas are the same.
template <typename T> struct CxT;
template <> struct CxT<float> { typedef float2 type; };
template <> struct CxT<double> { typedef double2 type; };
template <typename T> using Cx = typename CxT<T>::type;

// complex128 versions of the complex64 helpers above (same formulas, FP64 fused multiply-adds)
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ double2 ccmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double cabs2(double2 a) { return fma(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ double2 c2z(double2 a) { return a; }

template <typename T> __device__ __forceinline__ Cx<T> mkc(T re, T im);
template <> __device__ __forceinline__ float2 mkc<float>(float re, float im) { return make_float2(re, im); }
template <> __device__ __forceinline__ double2 mkc<double>(double re, double im) { return make_double2(re, im); }

__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float absT(float a) { return fabsf(a); }
__device__ __forceinline__ double absT(double a) { return fabs(a); }
__device__ __forceinline__ float maxT(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double maxT(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float copysignT(float a, float b) { return copysignf(a, b); }
__device__ __forceinline__ double copysignT(double a, double b) { return copysign(a, b); }
__device__ __forceinline__ float logT(float a) { return logf(a); }
__device__ __forceinline__ double logT(double a) { return log(a); }

// 1/d for d > 0 in FP64 by Newton-Raphson, r <- r + r (1 - d r), from the FP32 reciprocal of
// d: the relative error squares each step, so two steps take the FP32 start (~2^-23) below
// FP64 rounding, at four FP64 FMAs instead of an FP64 division (several times their latency
// on this GPU). Outside the FP32 normal range it divides.
__device__ __forceinline__ double recip64(double d) {
  if (!(d > 1e-36 && d < 1e36)) return 1.0 / d;
  double r = (double)__frcp_rn((float)d);
  r = fma(r, fma(-d, r, 1.0), r);
  r = fma(r, fma(-d, r, 1.0), r);
  return r;
}

// 1/sqrt(x) for x > 0: the hardware approximation refined by Newton's iteration
// r <- r (3 - x r^2) / 2, once in FP32; in FP64 twice from the FP32 value (the relative error
// roughly squares each step: ~2^-22 -> 2^-43 -> below FP64 rounding), dividing outside the
// FP32 normal range.
__device__ __forceinline__ float rsq_nr(float x) {
  const float r = rsqrtf(x);
  return r * fmaf(-0.5f * x * r, r, 1.5f);
}
__device__ __forceinline__ double rsq_nr(double x) {
  if (!(x > 1e-36 && x < 1e36)) return 1.0 / sqrt(x);
  double r = (double)rsqrtf((float)x);
  r = r * fma(-0.5 * x * r, r, 1.5);
  return r * fma(-0.5 * x * r, r, 1.5);
}
// sqrt(h) for h >= 1 (the Jacobi angle): h times the plain FP32 approximation of 1/sqrt(h);
// in FP64 from the refined one.
__device__ __forceinline__ float sqrt_h(float h) { return h * rsqrtf(h); }
__device__ __forceinline__ double sqrt_h(double h) { return h * rsq_nr(h); }
// 1/x (x != 0): the fast FP32 division; in FP64 the Newton reciprocal.
__device__ __forceinline__ float rcp_fast(float x) { return __fdividef(1.f, x); }
__device__ __forceinline__ double rcp_fast(double x) { return recip64(x); }

// Thresholds of the eigensolver per precision.
//   kHuge:   finite-value guard for pivots and eigenvalues;
//   kTiny2:  |a_pq|^2 below which an off-diagonal entry counts as zero;
//   kTol:    a pivot with |a_pq| <= kTol sqrt(|a_pp a_qq|) is not rotated;
//   kBig2:   a sweep whose pivots all had |a_pq|^2 <= kBig2 |a_pp a_qq| leaves off-diagonal
//            entries of order kBig2 relative (quadratic convergence): the solve ends;
//   kFirst2, kGap: the first-order finish runs once every |a_ij|^2 <= kFirst2 (a_jj - a_ii)^2
//            and every gap exceeds kGap of the larger eigenvalue; its error is then of order
//            kFirst2 relative.
template <typename T> struct Prec;
template <> struct Prec<float> {
  static constexpr float kHuge = 3.0e38f, kTiny2 = 1e-36f, kTol = 2.0e-7f, kBig2 = 1e-8f,
                         kFirst2 = 4e-8f, kGap = 1e-5f;
};
template <> struct Prec<double> {
  static constexpr double kHuge = 1e300, kTiny2 = 1e-300, kTol = 1e-15, kBig2 = 1e-16,
                          kFirst2 = 1e-16, kGap = 1e-8;
};

// --------------------------------------------------- warp-level dense Hermitian algebra
// Matrices are row-major with leading dimension kMaxM, in shared memory; a workspace for
// problems of order at most R holds R rows (an M x M problem reads rows 0..M-1 only). Every
// function is called by all 32 lanes of one warp and ends with __syncwarp().
template <typename T, int R = kMaxM>
struct WarpLAT {
  using C = Cx<T>;
  C A[R][kMaxM];   // work matrix (eigenproblem)
  C L[R][kMaxM];   // Cholesky factor (lower triangle); L^-1 in the fast solver
  C Z[R][kMaxM];   // temporary
  C V[R][kMaxM];   // eigenvectors / result
  C A2[R][kMaxM];  // ping-pong partners of A and V (fast solver)
  C V2[R][kMaxM];
  T invd[kMaxM];       // 1 / L_ii
  C jself[kMaxM + 1];  // Jacobi: J_xx for every index x
  C joth[kMaxM + 1];   // Jacobi: J_{partner(x), x}
  int partner[kMaxM + 1];
};
using WarpLA = WarpLAT<float>;

// In-place Cholesky B = L L^H of the Hermitian positive definite matrix in la.L (the lower
// triangle is read and overwritten). Returns false (uniformly across the warp) if a pivot is
// not positive and finite.
template <int M, typename T, int R>
__device__ bool warp_cholesky(WarpLAT<T, R>& la, int lane) {
  for (int k = 0; k < M; ++k) {
    __syncwarp();
    const T bkk = la.L[k][k].x;
    if (!(bkk > T(0)) || !(bkk < Prec<T>::kHuge)) {
      __syncwarp();
      return false;
    }
    const T il = rsq_nr(bkk);  // 1/sqrt(bkk) to rounding
    const T lkk = bkk * il;
    __syncwarp();
    if (lane == k) {
      la.L[k][k] = mkc<T>(lkk, T(0));
      la.invd[k] = il;
    } else if (lane > k && lane < M) {
      la.L[lane][k] = cscale(la.L[lane][k], il);
    }
    __syncwarp();
    for (int e = lane; e < M * M; e += 32) {
      const int i = e / M, j = e - (e / M) * M;
      if (j > k && i >= j) la.L[i][j] = csub(la.L[i][j], cmulc(la.L[i][k], la.L[j][k]));
    }
  }
  __syncwarp();
  return true;
}

// ---------------------------------------------------------------- low-latency solver
// Generalised eigenproblem of the Hermitian pencil (A, B), B positive definite, given in
// la.A (A) and la.L (B): Cholesky B = L L^H, W = L^-1 A L^-H = U Sig U^H (Jacobi),
// Q = L^-H U, so that Q^H B Q = I and Q^H A Q = Sig (Eq. (GEVDeff5)). log|det Q|^2 =
// 2 sum_i log(1/L_ii) + log|det U|^2, where the rotations leave U unitary only to rounding,
// so log|det U|^2 = log det(U^H U) = ||U||_F^2 - M to first order in U^H U - I.
// Arranged for a short dependency chain:
// one lane factors B = L L^H and inverts L in registers (no warp synchronisation inside the
// recurrences), the congruence W = L^-1 A L^-H and Q = L^-H U are lane-parallel products,
// and the Jacobi rounds ping-pong between two copies of A and V (one __syncwarp fewer per
// round).

// Lane 0: B (lower triangle of la.L) = L L^H; writes L^-1 (lower, zero above) over la.L and
// returns log|det L^-H|^2 = 2 sum_i log(1/L_ii). Result is valid on lane 0 only; *ok too.
template <int M, typename T, int R>
__device__ T lane_cholesky_inverse(WarpLAT<T, R>& la, bool* ok) {
  using C = Cx<T>;
  C L[M][M];
  T id[M];
  bool good = true;
#pragma unroll
  for (int j = 0; j < M; ++j) {
#pragma unroll
    for (int i = j; i < M; ++i) {
      C s = la.L[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) s = csub(s, cmulc(L[i][k], L[j][k]));
      if (i == j) {
        const T piv = s.x;
        good = good && (piv > T(0)) && (piv < Prec<T>::kHuge);
        const T il = rsq_nr(piv);  // 1/sqrt to rounding
        id[j] = il;
        L[j][j] = mkc<T>(piv * il, T(0));
      } else {
        L[i][j] = cscale(s, id[j]);
      }
    }
  }
  // L^-1: (L^-1)_ii = id_i; (L^-1)_ij = -id_i sum_{k=j}^{i-1} L_ik (L^-1)_kj for i > j.
  C Li[M][M];
  T ld = T(0);
#pragma unroll
  for (int j = 0; j < M; ++j) {
    Li[j][j] = mkc<T>(id[j], T(0));
    ld += T(2) * logT(id[j]);
#pragma unroll
    for (int i = j + 1; i < M; ++i) {
      C s = mkc<T>(T(0), T(0));
#pragma unroll
      for (int k = j; k < i; ++k) s = cfma(L[i][k], Li[k][j], s);
      Li[i][j] = cscale(s, -id[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < M; ++i) {
    la.invd[i] = id[i];
#pragma unroll
    for (int j = 0; j < M; ++j) la.L[i][j] = (j <= i) ? Li[i][j] : mkc<T>(T(0), T(0));
  }
  *ok = good;
  return ld;
}

// la.A <- W = Li A Li^H (Li = la.L, lower triangular), Hermitian by construction.
template <int M, typename T, int R>
__device__ void warp_congruence_products(WarpLAT<T, R>& la, int lane) {
  using C = Cx<T>;
  constexpr int kPer = (M * M + 31) / 32;
#pragma unroll
  for (int t = 0; t < kPer; ++t) {  // Z = A Li^H:  Z_ij = sum_{k<=j} A_ik conj(Li_jk)
    const int e = lane + 32 * t;
    if (e < M * M) {
      const int i = e / M, j = e % M;
      C s = mkc<T>(T(0), T(0));
#pragma unroll
      for (int k = 0; k < M; ++k)
        if (k <= j) s = cadd(s, cmulc(la.A[i][k], la.L[j][k]));
      la.Z[i][j] = s;
    }
  }
  __syncwarp();
  constexpr int NU = M * (M + 1) / 2;  // upper triangle incl. diagonal
  constexpr int kPerU = (NU + 31) / 32;
#pragma unroll
  for (int t = 0; t < kPerU; ++t) {  // W_ij = sum_{k<=i} Li_ik Z_kj, i <= j
    const int u = lane + 32 * t;
    if (u < NU) {
      int i = 0, r = u;
      while (r >= M - i) {
        r -= M - i;
        ++i;
      }
      const int j = i + r;
      C s = mkc<T>(T(0), T(0));
#pragma unroll
      for (int k = 0; k < M; ++k)
        if (k <= i) s = cfma(la.L[i][k], la.Z[k][j], s);
      if (i == j) {
        la.A[i][i] = mkc<T>(s.x, T(0));
      } else {
        la.A[i][j] = s;
        la.A[j][i] = cconj(s);
      }
    }
  }
  __syncwarp();
}

// Cyclic complex Jacobi on the Hermitian la.A, eigenvectors accumulated in la.V, in
// round-robin order (each round rotates disjoint pivot pairs at once). For a pivot (p, q)
// with a_pq = |a_pq| e: tau = (a_qq - a_pp) / (2 |a_pq|), t = sign(tau) / (|tau| +
// sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c, and J_pp = c, J_pq = s,
// J_qp = -s conj(e), J_qq = c conj(e) zeroes a_pq: A <- J^H A J, V <- V J. Pivots below
// tol relative to sqrt(|a_pp a_qq|) are skipped. Each round reads A/V from one buffer and
// writes the other; on return the current buffers are la.A / la.V (an even number of swaps is
// enforced by a final copy when needed). Returns the sweeps taken, or -1 past max_sweeps.
template <int M, typename T, int R>
__device__ int warp_jacobi_pp(WarpLAT<T, R>& la, int lane, T tol, int max_sweeps) {
  using C = Cx<T>;
  using PT = Prec<T>;
  constexpr int n = M + (M & 1);
  constexpr int kPer = (M * M + 31) / 32;
  for (int e = lane; e < M * M; e += 32) {
    const int i = e / M, j = e - (e / M) * M;
    la.V[i][j] = mkc<T>(i == j ? T(1) : T(0), T(0));
  }
  __syncwarp();
  if (M == 1) return 0;
  const T tol2 = tol * tol;
  C(*Ac)[kMaxM] = la.A;
  C(*Vc)[kMaxM] = la.V;
  C(*An)[kMaxM] = la.A2;
  C(*Vn)[kMaxM] = la.V2;
  int result = -1;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    int rotated = 0, big = 0;
    for (int r = 0; r < n - 1; ++r) {
      if (lane < n / 2) {
        const int k = lane;
        const int a = (k == 0) ? r : (r + k) % (n - 1);
        const int b = (k == 0) ? n - 1 : (r - k + (n - 1)) % (n - 1);
        const int p = min(a, b), q = max(a, b);
        T c = T(1), s = T(0);
        C e = mkc<T>(T(1), T(0));
        if (q < M) {
          const T app = Ac[p][p].x, aqq = Ac[q][q].x;
          const C apq = Ac[p][q];
          const T r2 = cabs2(apq);
          const T den = absT(app * aqq);
          if (r2 > tol2 * den && r2 > PT::kTiny2) {
            big |= (r2 > PT::kBig2 * den);
            const T ir = rsq_nr(r2);  // 1 / |a_pq|
            const T tau = T(0.5) * (aqq - app) * ir;
            const T h = fmaT(tau, tau, T(1));
            const T t = copysignT(rcp_fast(absT(tau) + sqrt_h(h)), tau);
            const T g = fmaT(t, t, T(1));
            c = rsq_nr(g);  // refined: c^2 + s^2 = 1
            s = t * c;
            e = cscale(apq, ir);
            rotated = 1;
          }
          la.jself[p] = mkc<T>(c, T(0));
          la.joth[p] = cscale(cconj(e), -s);
          la.partner[p] = q;
          la.jself[q] = cscale(cconj(e), c);
          la.joth[q] = mkc<T>(s, T(0));
          la.partner[q] = p;
        } else {
          la.jself[p] = mkc<T>(T(1), T(0));
          la.joth[p] = mkc<T>(T(0), T(0));
          la.partner[p] = p;
        }
      }
      __syncwarp();
#pragma unroll
      for (int t = 0; t < kPer; ++t) {
        const int e = lane + 32 * t;
        if (e < M * M) {
          const int i = e / M, l = e - (e / M) * M;
          const int ip = la.partner[i], lp = la.partner[l];
          const C Ji = la.jself[i], Jo_i = la.joth[i], Jl = la.jself[l], Jo_l = la.joth[l];
          const C r0 = cfma(Ac[i][lp], Jo_l, cmul(Ac[i][l], Jl));
          const C r1 = cfma(Ac[ip][lp], Jo_l, cmul(Ac[ip][l], Jl));
          C v = cadd(ccmul(Ji, r0), ccmul(Jo_i, r1));
          if (i == l) v.y = T(0);
          else if (ip == l) v = mkc<T>(T(0), T(0));  // the pivot pair
          An[i][l] = v;
          Vn[i][l] = cfma(Vc[i][lp], Jo_l, cmul(Vc[i][l], Jl));
        }
      }
      __syncwarp();
      C(*t0)[kMaxM] = Ac;
      Ac = An;
      An = t0;
      t0 = Vc;
      Vc = Vn;
      Vn = t0;
    }
    if (!__any_sync(0xffffffffu, rotated) || !__any_sync(0xffffffffu, big)) {
      result = sweep + 1;
      break;
    }
    // First-order finish (as in warp_gevd_reg) once every off-diagonal entry is small against
    // its eigenvalue gap: V <- V (I + X), X_ij = A_ij / (d_j - d_i) (skew-Hermitian, written
    // into the free ping-pong buffer), d_j += sum_p |A_pj|^2 / (d_j - d_p).
    // (Every gap must also stand clear of the eigenvalues' size: degenerate pairs take
    // another sweep.)
    int small = 1;
    for (int e = lane; e < M * M; e += 32) {
      const int i = e / M, j = e % M;
      if (i != j) {
        const T gap = Ac[j][j].x - Ac[i][i].x;
        const T scale = maxT(absT(Ac[i][i].x), absT(Ac[j][j].x));
        small &= (cabs2(Ac[i][j]) <= PT::kFirst2 * gap * gap && absT(gap) > PT::kGap * scale) ? 1 : 0;
      }
    }
    if (__all_sync(0xffffffffu, small)) {
      for (int e = lane; e < M * M; e += 32) {
        const int i = e / M, j = e % M;
        An[i][j] = (i != j) ? cscale(Ac[i][j], rcp_fast(Ac[j][j].x - Ac[i][i].x))
                            : mkc<T>(T(0), T(0));
      }
      __syncwarp();
      C nv[kPer];
      T corr[kPer];
#pragma unroll
      for (int t = 0; t < kPer; ++t) {
        const int e = lane + 32 * t;
        corr[t] = T(0);
        if (e < M * M) {
          const int i = e / M, j = e % M;
          C acc = Vc[i][j];
#pragma unroll
          for (int m = 0; m < M; ++m) acc = cfma(Vc[i][m], An[m][j], acc);
          nv[t] = acc;
          if (i == j) {
#pragma unroll
            for (int p2 = 0; p2 < M; ++p2)
              corr[t] = fmaT(Ac[p2][j].x, An[p2][j].x, fmaT(Ac[p2][j].y, An[p2][j].y, corr[t]));
          }
        }
      }
      __syncwarp();
#pragma unroll
      for (int t = 0; t < kPer; ++t) {
        const int e = lane + 32 * t;
        if (e < M * M) {
          const int i = e / M, j = e % M;
          Vc[i][j] = nv[t];
          if (i == j) Ac[i][i].x += corr[t];
        }
      }
      __syncwarp();
      result = sweep + 1;
      break;
    }
  }
  if (Ac != la.A) {  // bring the result back to la.A / la.V
    for (int e = lane; e < M * M; e += 32) {
      const int i = e / M, j = e % M;
      la.A[i][j] = Ac[i][j];
      la.V[i][j] = Vc[i][j];
    }
    __syncwarp();
  }
  return result;
}

// Low-latency generalised eigenproblem of (A, B) in (la.A, la.L): writes Q = L^-H U into
// Qout and U into Uout ([kMaxM][kMaxM]), Sig into sig, and returns 2 sum_i log(1/L_ii) in
// *ldL. log|det Q|^2 = *ldL + log|det U|^2, where the rotations leave U unitary only to
// rounding: log|det U|^2 = ||U||_F^2 - M to first order, which the caller sums in FP64 from
// Uout (unitarity_defect). Returns a device status code.
template <int M, typename T, int R>
__device__ int warp_gevd_fast(WarpLAT<T, R>& la, int lane, T* sig, Cx<T> (*Qout)[kMaxM],
                              Cx<T> (*Uout)[kMaxM], T* ldL, int max_sweeps) {
  using C = Cx<T>;
  bool ok = true;
  T ld = T(0);
  if (lane == 0) ld = lane_cholesky_inverse<M>(la, &ok);
  ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
  __syncwarp();
  if (!ok) return kErrNotPD;
  warp_congruence_products<M>(la, lane);
  const int sw = warp_jacobi_pp<M>(la, lane, Prec<T>::kTol, max_sweeps);
  if (sw < 0) return kErrEigNoConv;
  if (lane < M) sig[lane] = la.A[lane][lane].x;
  constexpr int kPer = (M * M + 31) / 32;
#pragma unroll
  for (int t = 0; t < kPer; ++t) {  // Q_ij = sum_{k>=i} conj(Li_ki) U_kj
    const int e = lane + 32 * t;
    if (e < M * M) {
      const int i = e / M, j = e % M;
      C s = mkc<T>(T(0), T(0));
#pragma unroll
      for (int k = 0; k < M; ++k)
        if (k >= i) s = cadd(s, ccmul(la.L[k][i], la.V[k][j]));
      Qout[i][j] = s;
      Uout[i][j] = la.V[i][j];
    }
  }
  ld = __shfl_sync(0xffffffffu, ld, 0);
  __syncwarp();
  *ldL = ld;
  for (int i = 0; i < M; ++i) {
    const T sv = sig[i];
    if (!(sv > T(0)) || !(sv < Prec<T>::kHuge)) return kErrNotPD;
  }
  return kOk;
}

// ------------------------------------------------------ register-resident solver, M <= 4
__device__ __forceinline__ float2 shfl2(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ double2 shfl2(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// Partner of index x in round r of the round-robin pairing of n positions (n even): position
// n-1 stays, the others rotate. Pairs of a round are disjoint and cover every index once.
__device__ __forceinline__ int rr_partner(int x, int r, int n) {
  if (x == n - 1) return r;
  if (x == r) return n - 1;
  const int y = 2 * r - x;
  return ((y % (n - 1)) + (n - 1)) % (n - 1);
}

// The generalised eigenproblem of warp_gevd_fast (same contract, same outputs: sig, Q = L^-H U,
// U, 2 sum log(1/L_ii); a device status code) for M <= 4, with the work of each step spread
// over the warp: lane l < M*M owns entry (l / M, l % M) of W = L^-1 A L^-H and of the
// eigenvector matrix V, and reads the entries it needs from other lanes by shuffles (no
// shared-memory round trips). Lane 0 factors B = L L^H and forms L^-1 (inherently sequential
// recurrences) and writes L^-1 over B. Each Jacobi round (the rotation of warp_jacobi_pp)
// rotates the disjoint round-robin pairs at once (every lane computes the angle of its row's
// pair; the column's comes by shuffle). Sweeps stop when a sweep rotated nothing or no pivot
// was large (Prec<T>::kBig2), or with the first-order step once every off-diagonal entry is
// small against its eigenvalue gap (Prec<T>::kFirst2). Called by all 32 lanes.
template <int M, typename T>
__device__ int warp_gevd_reg(const Cx<T> (*A)[kMaxM], Cx<T> (*B)[kMaxM], T* sig,
                             Cx<T> (*Qout)[kMaxM], Cx<T> (*Uout)[kMaxM], T* ldL, T tol,
                             int max_sweeps, int lane) {
  static_assert(M >= 1 && M <= 4, "one entry per lane: M*M <= 32 (and sized for M <= 4)");
  using C = Cx<T>;
  using PT = Prec<T>;
  constexpr int MM = M * M;
  constexpr int n = M + (M & 1);
  const bool own = lane < MM;
  const int i = own ? lane / M : 0, j = own ? lane % M : 0;
  // 1. Cholesky and L^-1 on lane 0.
  int ok = 1;
  T ld = T(0);
  if (lane == 0) {
    C L[M][M];
    T id[M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
#pragma unroll
      for (int r = c; r < M; ++r) {
        C sv = B[r][c];
#pragma unroll
        for (int k = 0; k < c; ++k) sv = csub(sv, cmulc(L[r][k], L[c][k]));
        if (r == c) {
          const T piv = sv.x;
          ok = ok && (piv > T(0)) && (piv < PT::kHuge);
          const T il = rsq_nr(piv);  // 1/sqrt to rounding
          id[c] = il;
          L[c][c] = mkc<T>(piv * il, T(0));
        } else {
          L[r][c] = cscale(sv, id[c]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < M; ++c) {
      B[c][c] = mkc<T>(id[c], T(0));
      ld += T(2) * logT(id[c]);
#pragma unroll
      for (int r = c + 1; r < M; ++r) {
        C sv = mkc<T>(T(0), T(0));
#pragma unroll
        for (int k = c; k < r; ++k) sv = cfma(L[r][k], (k == c) ? mkc<T>(id[c], T(0)) : B[k][c], sv);
        B[r][c] = cscale(sv, -id[r]);
        B[c][r] = mkc<T>(T(0), T(0));
      }
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  ld = __shfl_sync(0xffffffffu, ld, 0);
  __syncwarp();
  if (!ok) return kErrNotPD;
  // 2. W = Li A Li^H: T = A Li^H (T_ij = sum_{k<=j} A_ik conj(Li_jk)), W_ij = sum_{k<=i} Li_ik T_kj.
  C Tm = mkc<T>(T(0), T(0));
#pragma unroll
  for (int k = 0; k < M; ++k)
    if (k <= j) Tm = cadd(Tm, cmulc(A[i][k], B[j][k]));
  C W = mkc<T>(T(0), T(0));
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const C tk = shfl2(Tm, own ? k * M + j : lane);
    if (k <= i) W = cfma(B[i][k], tk, W);
  }
  {  // exactly Hermitian: the lower triangle mirrors the upper one
    const C wt = shfl2(W, own ? j * M + i : lane);
    if (i > j) W = cconj(wt);
    if (i == j) W.y = T(0);
  }
  C V = mkc<T>(i == j ? T(1) : T(0), T(0));
  // 3. Jacobi sweeps.
  const T tol2 = tol * tol;
  int sweeps = (M == 1) ? 0 : -1;
  for (int sweep = 0; sweep < max_sweeps && M > 1; ++sweep) {
    int rotated = 0, big = 0;
#pragma unroll
    for (int r = 0; r < n - 1; ++r) {
      const int pi = rr_partner(i, r, n), pj = rr_partner(j, r, n);
      const int p = min(i, pi), q = max(i, pi);
      const bool valid = own && q < M;
      const T app = __shfl_sync(0xffffffffu, W.x, valid ? p * M + p : lane);
      const T aqq = __shfl_sync(0xffffffffu, W.x, valid ? q * M + q : lane);
      const C apq = shfl2(W, valid ? p * M + q : lane);
      C Jii = mkc<T>(T(1), T(0)), Joi = mkc<T>(T(0), T(0));  // J_{i i}, J_{i' i}
      bool act = false;
      if (valid) {
        const T r2 = cabs2(apq);
        const T den = absT(app * aqq);
        if (r2 > tol2 * den && r2 > PT::kTiny2) {
          act = true;
          big |= (r2 > PT::kBig2 * den);
          const T ir = rsq_nr(r2);
          const T tau = T(0.5) * (aqq - app) * ir;
          const T h = fmaT(tau, tau, T(1));
          const T t = copysignT(rcp_fast(absT(tau) + sqrt_h(h)), tau);
          const T g = fmaT(t, t, T(1));
          const T c = rsq_nr(g);
          const T sv = t * c;
          const C e = cscale(apq, ir);
          if (i == p) {  // J_pp = c, J_qp = -s conj(e)
            Jii = mkc<T>(c, T(0));
            Joi = cscale(cconj(e), -sv);
          } else {       // J_qq = c conj(e), J_pq = s
            Jii = cscale(cconj(e), c);
            Joi = mkc<T>(sv, T(0));
          }
        }
      }
      rotated |= act;
      // J of the column index j: computed by lane (j, 0), whose row index is j.
      const C Jll = shfl2(Jii, own ? j * M : lane);
      const C Jol = shfl2(Joi, own ? j * M : lane);
      const bool ip_ok = pi < M, jp_ok = pj < M;
      const C W_il2 = shfl2(W, own && jp_ok ? i * M + pj : lane);
      const C W_i2l = shfl2(W, own && ip_ok ? pi * M + j : lane);
      const C W_i2l2 = shfl2(W, own && ip_ok && jp_ok ? pi * M + pj : lane);
      const C V_il2 = shfl2(V, own && jp_ok ? i * M + pj : lane);
      // W' = J^H W J restricted to entry (i, j); V' = V J.
      C r0 = cmul(W, Jll), r1 = cmul(W_i2l, Jll);
      if (jp_ok) {
        r0 = cfma(W_il2, Jol, r0);
        r1 = cfma(W_i2l2, Jol, r1);
      }
      C Wn = ccmul(Jii, r0);
      if (ip_ok) Wn = cadd(Wn, ccmul(Joi, r1));
      C Vn = cmul(V, Jll);
      if (jp_ok) Vn = cfma(V_il2, Jol, Vn);
      if (i == j) Wn.y = T(0);
      if (act && j == pi) Wn = mkc<T>(T(0), T(0));  // the pivot pair
      W = Wn;
      V = Vn;
    }
    rotated = __any_sync(0xffffffffu, rotated);
    big = __any_sync(0xffffffffu, big);
    if (!rotated || !big) {
      sweeps = sweep + 1;
      break;
    }
    const T di = __shfl_sync(0xffffffffu, W.x, own ? i * M + i : lane);
    const T dj = __shfl_sync(0xffffffffu, W.x, own ? j * M + j : lane);
    const T gap = dj - di;
    // (Every gap must also stand clear of the eigenvalues' size: degenerate pairs take
    // another sweep.)
    const bool small = !own || i == j ||
                       (cabs2(W) <= PT::kFirst2 * gap * gap && absT(gap) > PT::kGap * maxT(absT(di), absT(dj)));
    if (__all_sync(0xffffffffu, small)) {
      // First-order step: V <- V (I + X), X_ij = W_ij / (d_j - d_i);
      // d_j += sum_p |W_pj|^2 / (d_j - d_p).
      const C X = (own && i != j) ? cscale(W, rcp_fast(gap)) : mkc<T>(T(0), T(0));
      C Vn = V;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const C vim = shfl2(V, own ? i * M + m : lane);
        const C xmj = shfl2(X, own ? m * M + j : lane);
        Vn = cfma(vim, xmj, Vn);
      }
      const T e2 = W.x * X.x + W.y * X.y;  // |W_ij|^2 / (d_j - d_i)
      T corr = T(0);
#pragma unroll
      for (int m = 0; m < M; ++m) corr += __shfl_sync(0xffffffffu, e2, own ? m * M + j : lane);
      V = Vn;
      if (i == j) W.x += corr;
      sweeps = sweep + 1;
      break;
    }
  }
  if (sweeps < 0) return kErrEigNoConv;
  // 4. Outputs: Sig, Q = Li^H V (Q_ij = sum_{k>=i} conj(Li_ki) V_kj), U = V.
  C Qv = mkc<T>(T(0), T(0));
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const C vkj = shfl2(V, own ? k * M + j : lane);
    if (k >= i) Qv = cadd(Qv, ccmul(B[k][i], vkj));
  }
  if (own) {
    Qout[i][j] = Qv;
    Uout[i][j] = V;
    if (i == j) sig[i] = W.x;
  }
  const bool pos = !own || i != j || ((W.x > T(0)) && (W.x < PT::kHuge));
  *ldL = ld;
  __syncwarp();
  return __all_sync(0xffffffffu, pos) ? kOk : kErrNotPD;
}

// ---------------------------------------- Newton-type iteration for the joint diagonaliser
// One step of the Newton-type correction of a generalised eigenbasis of the Hermitian pencil
// (A, B), B positive definite: the correction of Ogita and Aishima ("Iterative refinement for
// symmetric eigenvalue decomposition", 2018) written for the pencil. With R = I - X^H B X and
// S = X^H A X, lam_i = s_ii / (1 - r_ii), E_ii = r_ii / 2, E_ij = (s_ij + lam_j r_ij) /
// (lam_j - lam_i) for i != j, and X <- X (I + E). To first order in R and the off-diagonal
// part of S this makes X^H B X = I and X^H A X = diag(lam), so the residuals square with each
// step, as long as every |E_ij| stays small. The two corrections of a pair are set together
// (by the lane of its upper entry, E_ji = conj(r_ij - E_ij) in either form), so that the first
// order holds exactly. A pair (i, j) whose couplings c_ij = s_ij + lam_j r_ij and
// conj(c_ji) = s_ij + lam_i r_ij are not both below a tenth of its eigenvalue gap cannot be
// separated this way: if they are negligible (below kSep of the eigenvalues: a degenerate or
// already resolved pair) it takes E_ij = r_ij / 2, otherwise the step fails and returns
// +infinity (the caller then takes the Jacobi solver). T1, T2: workspace. Writes lam (the Rayleigh quotients
// of the incoming X) and returns max_ij |E_ij|_1 (all lanes; NaN propagates). With first =
// true, X is taken to be the identity (not read): R = I - B and S = A. All 32 lanes; ends with
// __syncwarp().
template <int M, typename T>
__device__ T warp_newton_step(const Cx<T> (*A)[kMaxM], const Cx<T> (*B)[kMaxM], Cx<T> (*X)[kMaxM],
                              Cx<T> (*T1)[kMaxM], Cx<T> (*T2)[kMaxM], T* lam, bool first,
                              int lane, T* trR = nullptr) {
  using C = Cx<T>;
  constexpr int MM = M * M;
  constexpr int kPer = (MM + 31) / 32;
  constexpr T kSep = sizeof(T) == 8 ? T(1e-13) : T(1e-6);
  if (!first) {
#pragma unroll
    for (int t = 0; t < kPer; ++t) {  // T1 = B X, T2 = A X
      const int e = lane + 32 * t;
      if (e < MM) {
        const int i = e / M, j = e % M;
        C b = mkc<T>(T(0), T(0)), a = mkc<T>(T(0), T(0));
#pragma unroll
        for (int k = 0; k < M; ++k) {
          b = cfma(B[i][k], X[k][j], b);
          a = cfma(A[i][k], X[k][j], a);
        }
        T1[i][j] = b;
        T2[i][j] = a;
      }
    }
    __syncwarp();
  }
  C r[kPer], sv[kPer];
  T tr = T(0);
#pragma unroll
  for (int t = 0; t < kPer; ++t) {  // R = I - X^H T1, S = X^H T2
    const int e = lane + 32 * t;
    r[t] = sv[t] = mkc<T>(T(0), T(0));
    if (e < MM) {
      const int i = e / M, j = e % M;
      C q, u;
      if (first) {
        q = B[i][j];
        u = A[i][j];
      } else {
        q = u = mkc<T>(T(0), T(0));
#pragma unroll
        for (int k = 0; k < M; ++k) {
          q = cfma(cconj(X[k][i]), T1[k][j], q);
          u = cfma(cconj(X[k][i]), T2[k][j], u);
        }
      }
      r[t] = mkc<T>((i == j ? T(1) : T(0)) - q.x, -q.y);
      sv[t] = u;
      if (i == j) {
        lam[i] = u.x * rcp_fast(T(1) - r[t].x);
        tr += r[t].x;
      }
    }
  }
  if (trR) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    *trR = tr;
  }
  __syncwarp();
  T emax = T(0);
#pragma unroll
  for (int t = 0; t < kPer; ++t) {  // E into T1
    const int e = lane + 32 * t;
    if (e < MM) {
      const int i = e / M, j = e % M;
      T m = T(0);
      if (i == j) {
        T1[i][i] = mkc<T>(T(0.5) * r[t].x, T(0));
        m = absT(T(0.5) * r[t].x);
      } else if (i < j) {  // the pair's upper entry writes both corrections (E_ij + conj(E_ji) = r_ij)
        const T li = lam[i], lj = lam[j], gap = lj - li;
        const C c1 = mkc<T>(fmaT(lj, r[t].x, sv[t].x), fmaT(lj, r[t].y, sv[t].y));
        const C c2 = mkc<T>(fmaT(li, r[t].x, sv[t].x), fmaT(li, r[t].y, sv[t].y));
        const T cm = maxT(absT(c1.x) + absT(c1.y), absT(c2.x) + absT(c2.y));
        C eij, eji;
        const bool sep = cm <= T(0.1) * absT(gap) && gap != T(0);
        if (sep) {
          const T rg = rcp_fast(gap);
          eij = mkc<T>(c1.x * rg, c1.y * rg);
          eji = mkc<T>(-c2.x * rg, c2.y * rg);
        } else {
          eij = mkc<T>(T(0.5) * r[t].x, T(0.5) * r[t].y);
          eji = cconj(eij);
        }
        T1[i][j] = eij;
        T1[j][i] = eji;
        m = maxT(absT(eij.x) + absT(eij.y), absT(eji.x) + absT(eji.y));
        if (!sep && !(cm <= kSep * maxT(absT(li), absT(lj)))) m = T(INFINITY);
      }
      emax = (m > emax || m != m) ? m : emax;
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const T other = __shfl_xor_sync(0xffffffffu, emax, o);
    emax = (other > emax || other != other) ? other : emax;
  }
  __syncwarp();
  C xn[kPer];
#pragma unroll
  for (int t = 0; t < kPer; ++t) {  // X <- X + X E (from the identity: I + E)
    const int e = lane + 32 * t;
    if (e < MM) {
      const int i = e / M, j = e % M;
      if (first) {
        xn[t] = cadd(T1[i][j], mkc<T>(i == j ? T(1) : T(0), T(0)));
      } else {
        C x = X[i][j];
#pragma unroll
        for (int k = 0; k < M; ++k) x = cfma(X[i][k], T1[k][j], x);
        xn[t] = x;
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int e = lane + 32 * t;
    if (e < MM) X[e / M][e % M] = xn[t];
  }
  __syncwarp();
  return emax;
}

// ------------------------------------------------- compensated FP32 dot products
// Error-free transformations in FP32: Knuth's TwoSum (a + b = s + t exactly) and the FMA form
// of Dekker's TwoProduct (a b = p + e exactly), and the compensated dot product built on them
// (Ogita, Rump and Oishi, "Accurate sum and dot product", 2005: "Dot2"): the pair (s, c)
// carries sum_k a_k b_k with an error of order 2^-48 sum_k |a_k b_k| + 2^-24 |result|, as if
// computed in twice the working precision, on the FP32 pipe. An operand given as a pair
// (hi, lo) with |lo| <= 2^-24 |hi| (an FP64 value split into two floats) contributes
// a_k hi_k exactly and a_k lo_k in plain FP32, which keeps the same error order.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = a + b;
  const float bp = s - a;
  t = (a - (s - bp)) + (b - bp);
}

struct Dot2 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float a, float b) {  // += a b
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    float t;
    two_sum(s, p, s, t);
    c += t + e;
  }
  __device__ __forceinline__ void add2(float a, float bh, float bl) {  // += a (bh + bl)
    add(a, bh);
    c = fmaf(a, bl, c);
  }
  __device__ __forceinline__ void merge(const Dot2& o) {  // += o
    float t;
    two_sum(s, o.s, s, t);
    c += t + o.c;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// A complex compensated accumulator: re and im parts.
struct CDot2 {
  Dot2 re, im;
  // += a (bh + bl), complex a and the split complex b
  __device__ __forceinline__ void fma2(float2 a, float2 bh, float2 bl) {
    re.add2(a.x, bh.x, bl.x);
    re.add2(-a.y, bh.y, bl.y);
    im.add2(a.x, bh.y, bl.y);
    im.add2(a.y, bh.x, bl.x);
  }
  __device__ __forceinline__ double2 value() const { return make_double2(re.value(), im.value()); }
  __device__ __forceinline__ void shfl_merge(int o) {  // combine with the lane `lane ^ o`
    Dot2 r, i;
    r.s = __shfl_xor_sync(0xffffffffu, re.s, o);
    r.c = __shfl_xor_sync(0xffffffffu, re.c, o);
    i.s = __shfl_xor_sync(0xffffffffu, im.s, o);
    i.c = __shfl_xor_sync(0xffffffffu, im.c, o);
    re.merge(r);
    im.merge(i);
  }
};

// An FP64 complex value split into two complex floats: v = hi + lo, hi = fl32(v).
__device__ __forceinline__ void split2(double2 v, float2& hi, float2& lo) {
  hi = z2c(v);
  lo = make_float2((float)(v.x - (double)hi.x), (float)(v.y - (double)hi.y));
}

// FP64 working arrays of the refined eigensolver (shared memory), for order at most R.
template <int R = kMaxM>
struct RefineWork {
  double2 A[R][kMaxM];   // the pencil (A, B) in FP64, B positive definite (in the EM kernel
  double2 B[R][kMaxM];   //   formed from the pairs below only for the FP64 step)
  float2 Ah[R][kMaxM];   // A and B split into FP32 pairs (hi + lo)
  float2 Al[R][kMaxM];
  float2 Bh[R][kMaxM];
  float2 Bl[R][kMaxM];
  double2 X[R][kMaxM];   // the basis being refined
  double2 T1[R][kMaxM];  // workspace
  double2 T2[R][kMaxM];
  float2 X0[R][kMaxM];   // the FP32 start (fallback solver's basis)
  float sig0[kMaxM];
  float lam32[kMaxM];
  double lam[kMaxM];
};

// The corrections of the pair (i, j), i < j, in a refinement step, from the residual entries
// r = r_ij, s = s_ij and the eigenvalue estimates li, lj: E_ij and E_ji are chosen together,
// so that E_ij + conj(E_ji) = r_ij holds exactly and X^H B X = I stays true to first order
// whatever the choice. The Newton form E_ij = c1 / (lj - li), E_ji = -conj(c2) / (lj - li),
// c1 = lj r + s, c2 = li r + s, is taken when both couplings are below kRefineSep of the gap,
// so that the second-order terms E^H E are below kRefineSep^2 of the step's residuals;
// otherwise E_ij = r_ij / 2 (a pair closer than its own coupling: degenerate, or resolved to
// the start's accuracy, which is all its mixing can affect). Returns max(|E_ij|_1, |E_ji|_1).
constexpr double kRefineSep = 0.01;
__device__ __forceinline__ float refine_pair(double li, double lj, double2 r, double2 s, float2* eij,
                                             float2* eji) {
  const double gap = lj - li;
  const float c1x = (float)fma(lj, r.x, s.x), c1y = (float)fma(lj, r.y, s.y);
  const float c2x = (float)fma(li, r.x, s.x), c2y = (float)fma(li, r.y, s.y);
  const float cm = fmaxf(fabsf(c1x) + fabsf(c1y), fabsf(c2x) + fabsf(c2y));
  const float g = (float)gap;
  if (cm <= (float)kRefineSep * fabsf(g) && g != 0.f) {  // (an exactly degenerate pair: r / 2)
    const float rg = __fdividef(1.f, g);
    *eij = make_float2(c1x * rg, c1y * rg);
    *eji = make_float2(-c2x * rg, c2y * rg);
  } else {
    *eij = make_float2((float)(0.5 * r.x), (float)(0.5 * r.y));
    *eji = make_float2(eij->x, -eij->y);
  }
  return fmaxf(fabsf(eij->x) + fabsf(eij->y), fabsf(eji->x) + fabsf(eji->y));
}

// One FP64 step of warp_newton_step on w.X for the pencil (w.A, w.B), arranged to spend few
// FP64 operations (they are the scarce resource on this GPU): the residuals R and S, whose
// small entries come from cancellation, and lam in FP64; the correction E (a small quantity,
// needed to a few digits) and the product X E in FP32, added to X in FP64. lam_i =
// s_ii / (1 - r_ii) is taken to second order in r_ii. Each pair's two corrections come from
// refine_pair (a pair the start did not separate further than its own accuracy, a degenerate
// pair among them, keeps its rotation: E_ij = r_ij / 2). For
// M <= 4 the two lanes of each pair split every length-M sum (all 32 lanes busy). Returns
// max_ij |E_ij|_1 (all lanes).
template <int M, int R>
__device__ double warp_refine_step64(RefineWork<R>& w, float2 (*E)[kMaxM], int lane) {
  constexpr int MM = M * M;
  constexpr bool kSplit = MM <= 16;
  constexpr int kPer = kSplit ? 1 : (MM + 31) / 32;
  constexpr int kStride = kSplit ? 2 : 1;
  const int h = kSplit ? (lane & 1) : 0;
  auto entry = [&](int t) { return kSplit ? (lane >> 1) : lane + 32 * t; };
  // T1 = B X, T2 = A X
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int e = entry(t);
    const int i = (e < MM) ? e / M : 0, j = (e < MM) ? e % M : 0;
    double2 b = make_double2(0.0, 0.0), a = make_double2(0.0, 0.0);
    if (e < MM) {
#pragma unroll
      for (int kk = 0; kk < (M + kStride - 1) / kStride; ++kk) {
        const int k = kk * kStride + h;
        if (k < M) {
          b = zfma(w.B[i][k], w.X[k][j], b);
          a = zfma(w.A[i][k], w.X[k][j], a);
        }
      }
    }
    if constexpr (kSplit) {
      b.x += __shfl_xor_sync(0xffffffffu, b.x, 1);
      b.y += __shfl_xor_sync(0xffffffffu, b.y, 1);
      a.x += __shfl_xor_sync(0xffffffffu, a.x, 1);
      a.y += __shfl_xor_sync(0xffffffffu, a.y, 1);
    }
    if (e < MM && h == 0) {
      w.T1[i][j] = b;
      w.T2[i][j] = a;
    }
  }
  __syncwarp();
  // R = I - X^H T1, S = X^H T2; lam
  double2 r[kPer], sv[kPer];
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int e = entry(t);
    const int i = (e < MM) ? e / M : 0, j = (e < MM) ? e % M : 0;
    double2 q = make_double2(0.0, 0.0), u = make_double2(0.0, 0.0);
    if (e < MM) {
#pragma unroll
      for (int kk = 0; kk < (M + kStride - 1) / kStride; ++kk) {
        const int k = kk * kStride + h;
        if (k < M) {
          q = cfma(cconj(w.X[k][i]), w.T1[k][j], q);
          u = cfma(cconj(w.X[k][i]), w.T2[k][j], u);
        }
      }
    }
    if constexpr (kSplit) {
      q.x += __shfl_xor_sync(0xffffffffu, q.x, 1);
      q.y += __shfl_xor_sync(0xffffffffu, q.y, 1);
      u.x += __shfl_xor_sync(0xffffffffu, u.x, 1);
      u.y += __shfl_xor_sync(0xffffffffu, u.y, 1);
    }
    r[t] = make_double2((i == j ? 1.0 : 0.0) - q.x, -q.y);
    sv[t] = u;
    if (e < MM && h == 0 && i == j) w.lam[i] = fma(u.x, fma(r[t].x, r[t].x, r[t].x), u.x);
  }
  __syncwarp();
  // E (FP32)
  float emax = 0.f;
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int e = entry(t);
    if (e < MM && h == 0) {
      const int i = e / M, j = e % M;
      float m = 0.f;
      if (i == j) {
        E[i][i] = make_float2((float)(0.5 * r[t].x), 0.f);
        m = fabsf(E[i][i].x);
      } else if (i < j) {  // the pair's upper entry writes both corrections
        float2 eij, eji;
        m = refine_pair(w.lam[i], w.lam[j], r[t], sv[t], &eij, &eji);
        E[i][j] = eij;
        E[j][i] = eji;
      }
      emax = (m > emax || m != m) ? m : emax;
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const float other = __shfl_xor_sync(0xffffffffu, emax, o);
    emax = (other > emax || other != other) ? other : emax;
  }
  __syncwarp();
  // X <- X + X E, the product in FP32
  float2 dx[kPer];
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int e = entry(t);
    const int i = (e < MM) ? e / M : 0, j = (e < MM) ? e % M : 0;
    float2 d = make_float2(0.f, 0.f);
    if (e < MM) {
#pragma unroll
      for (int kk = 0; kk < (M + kStride - 1) / kStride; ++kk) {
        const int k = kk * kStride + h;
        if (k < M) d = cfma(z2c(w.X[i][k]), E[k][j], d);
      }
    }
    if constexpr (kSplit) {
      d.x += __shfl_xor_sync(0xffffffffu, d.x, 1);
      d.y += __shfl_xor_sync(0xffffffffu, d.y, 1);
    }
    dx[t] = d;
  }
  __syncwarp();
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int e = entry(t);
    if (e < MM && h == 0) {
      const int i = e / M, j = e % M;
      w.X[i][j] = make_double2(w.X[i][j].x + (double)dx[t].x, w.X[i][j].y + (double)dx[t].y);
    }
  }
  __syncwarp();
  return (double)emax;
}

// The refined basis and eigenvalues as FP32 pairs (hi + lo): X = Xh + Xl, lam = lh + ll.
struct RefineOut {
  float2 (*Xh)[kMaxM];
  float2 (*Xl)[kMaxM];
  float* lh;
  float* ll;
};

// refine_pair in FP32, for residual entries that are small quantities needed to FP32 accuracy
// and eigenvalues given as pairs (the gap of a close pair is formed from both parts).
__device__ __forceinline__ float refine_pair32(float lhi, float lli, float lhj, float llj, float2 r,
                                               float2 s, float2* eij, float2* eji) {
  const float g = (lhj - lhi) + (llj - lli);
  const float c1x = fmaf(lhj, r.x, s.x), c1y = fmaf(lhj, r.y, s.y);
  const float c2x = fmaf(lhi, r.x, s.x), c2y = fmaf(lhi, r.y, s.y);
  const float cm = fmaxf(fabsf(c1x) + fabsf(c1y), fabsf(c2x) + fabsf(c2y));
  if (cm <= (float)kRefineSep * fabsf(g) && g != 0.f) {  // (an exactly degenerate pair: r / 2)
    const float rg = __fdividef(1.f, g);
    *eij = make_float2(c1x * rg, c1y * rg);
    *eji = make_float2(-c2x * rg, c2y * rg);
  } else {
    *eij = make_float2(0.5f * r.x, 0.5f * r.y);
    *eji = make_float2(eij->x, -eij->y);
  }
  return fmaxf(fabsf(eij->x) + fabsf(eij->y), fabsf(eji->x) + fabsf(eji->y));
}

// The first refinement step from an FP32 basis X0 (exact in FP32), in FP32 arithmetic only:
// the step of warp_refine_step64 with R = I - X0^H B X0 and S = X0^H A X0 formed as
// compensated dot products (Dot2) of X0 and the split FP32 pairs of A and B (B X0 and A X0
// kept as unrounded pairs): an error of order 2^-48 of the terms, which for a basis near the
// pencil's eigenbasis is 2^-48 of the result. The small quantities (R, the off-diagonal of S,
// the couplings and E) are then needed to FP32 accuracy only; the eigenvalues
// lam_i = s_ii (1 + r_ii + r_ii^2) and the basis X = X0 + X0 E are kept as FP32 pairs
// (out.lh, out.ll; out.Xh = X0, out.Xl = X0 E). Returns max_ij |E_ij|_1 (all lanes).
template <int M, int R>
__device__ float warp_refine_step_df(RefineWork<R>& w, const float2 (*X0)[kMaxM], float2 (*E)[kMaxM],
                                     float2 (*T1h)[kMaxM], float2 (*T1l)[kMaxM],
                                     float2 (*T2h)[kMaxM], float2 (*T2l)[kMaxM],
                                     const RefineOut& out, int lane) {
  constexpr int MM = M * M;
  constexpr bool kSplit = MM <= 16;
  constexpr int kPer = kSplit ? 1 : (MM + 31) / 32;
  constexpr int kStride = kSplit ? 2 : 1;
  const int h = kSplit ? (lane & 1) : 0;
  auto entry = [&](int t) { return kSplit ? (lane >> 1) : lane + 32 * t; };
  // T1 = B X0, T2 = A X0 as unrounded pairs
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int e = entry(t);
    const int i = (e < MM) ? e / M : 0, j = (e < MM) ? e % M : 0;
    CDot2 b, a;
    if (e < MM) {
#pragma unroll
      for (int kk = 0; kk < (M + kStride - 1) / kStride; ++kk) {
        const int k = kk * kStride + h;
        if (k < M) {
          const float2 x = X0[k][j];
          b.fma2(x, w.Bh[i][k], w.Bl[i][k]);
          a.fma2(x, w.Ah[i][k], w.Al[i][k]);
        }
      }
    }
    if constexpr (kSplit) {
      b.shfl_merge(1);
      a.shfl_merge(1);
    }
    if (e < MM && h == 0) {
      T1h[i][j] = make_float2(b.re.s, b.im.s);
      T1l[i][j] = make_float2(b.re.c, b.im.c);
      T2h[i][j] = make_float2(a.re.s, a.im.s);
      T2l[i][j] = make_float2(a.re.c, a.im.c);
    }
  }
  __syncwarp();
  // R = I - X0^H T1, S = X0^H T2 (FP32 values); lam as pairs
  float2 r[kPer], sv[kPer];
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int e = entry(t);
    const int i = (e < MM) ? e / M : 0, j = (e < MM) ? e % M : 0;
    CDot2 q, u;
    if (e < MM) {
#pragma unroll
      for (int kk = 0; kk < (M + kStride - 1) / kStride; ++kk) {
        const int k = kk * kStride + h;
        if (k < M) {
          const float2 xc = cconj(X0[k][i]);
          q.fma2(xc, T1h[k][j], T1l[k][j]);
          u.fma2(xc, T2h[k][j], T2l[k][j]);
        }
      }
    }
    if constexpr (kSplit) {
      q.shfl_merge(1);
      u.shfl_merge(1);
    }
    if (i == j) {
      // 1 - q_ii is exact in FP32 for q_ii near 1; s_ii as a normalised pair
      r[t] = make_float2((1.f - q.re.s) - q.re.c, 0.f);
      float shi, slo;
      two_sum(u.re.s, u.re.c, shi, slo);
      sv[t] = make_float2(shi, 0.f);
      if (e < MM && h == 0) {
        float lh, ll;
        two_sum(shi, fmaf(shi, fmaf(r[t].x, r[t].x, r[t].x), slo), lh, ll);
        out.lh[i] = lh;
        out.ll[i] = ll;
      }
    } else {
      r[t] = make_float2(-(q.re.s + q.re.c), -(q.im.s + q.im.c));
      sv[t] = make_float2(u.re.s + u.re.c, u.im.s + u.im.c);
    }
  }
  __syncwarp();
  // E: the pair's upper entry writes both corrections
  float emax = 0.f;
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int e = entry(t);
    if (e < MM && h == 0) {
      const int i = e / M, j = e % M;
      float m = 0.f;
      if (i == j) {
        E[i][i] = make_float2(0.5f * r[t].x, 0.f);
        m = fabsf(0.5f * r[t].x);
      } else if (i < j) {
        float2 eij, eji;
        m = refine_pair32(out.lh[i], out.ll[i], out.lh[j], out.ll[j], r[t], sv[t], &eij, &eji);
        E[i][j] = eij;
        E[j][i] = eji;
      }
      emax = (m > emax || m != m) ? m : emax;
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const float other = __shfl_xor_sync(0xffffffffu, emax, o);
    emax = (other > emax || other != other) ? other : emax;
  }
  __syncwarp();
  // X = X0 + X0 E, kept as the pair (X0, X0 E)
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int e = entry(t);
    const int i = (e < MM) ? e / M : 0, j = (e < MM) ? e % M : 0;
    float2 d = make_float2(0.f, 0.f);
    if (e < MM) {
#pragma unroll
      for (int kk = 0; kk < (M + kStride - 1) / kStride; ++kk) {
        const int k = kk * kStride + h;
        if (k < M) d = cfma(X0[i][k], E[k][j], d);
      }
    }
    if constexpr (kSplit) {
      d.x += __shfl_xor_sync(0xffffffffu, d.x, 1);
      d.y += __shfl_xor_sync(0xffffffffu, d.y, 1);
    }
    if (e < MM && h == 0) {
      out.Xh[i][j] = X0[i][j];
      out.Xl[i][j] = d;
    }
  }
  __syncwarp();
  return emax;
}

// Refinement of an FP32 generalised eigenbasis X0 of (w.A, w.B) into out: the FP32 step of
// warp_refine_step_df, and when its correction exceeded 1e-4 (a poor start) a second,
// FP64 step (warp_refine_step64, through w.X and w.lam). The result satisfies X^H B X = I and
// X^H A X = diag(lam) to second order in the start's residuals. X0 must not be out.Xh or
// out.Xl; E, T1h..T2l: FP32 workspaces. All 32 lanes; ends with __syncwarp().
template <int M, int R>
__device__ void warp_refine_gevd(RefineWork<R>& w, const float2 (*X0)[kMaxM], float2 (*E)[kMaxM],
                                 float2 (*T1h)[kMaxM], float2 (*T1l)[kMaxM], float2 (*T2h)[kMaxM],
                                 float2 (*T2l)[kMaxM], const RefineOut& out, int lane) {
  constexpr int MM = M * M;
  const float em = warp_refine_step_df<M>(w, X0, E, T1h, T1l, T2h, T2l, out, lane);
  if (em <= 1e-4f) return;  // (NaN goes on, and stays NaN)
  for (int e = lane; e < MM; e += 32) {  // the FP64 pencil from its pairs
    const int i = e / M, k = e % M;
    w.A[i][k] = make_double2((double)w.Ah[i][k].x + (double)w.Al[i][k].x, (double)w.Ah[i][k].y + (double)w.Al[i][k].y);
    w.B[i][k] = make_double2((double)w.Bh[i][k].x + (double)w.Bl[i][k].x, (double)w.Bh[i][k].y + (double)w.Bl[i][k].y);
  }
  for (int e = lane; e < MM; e += 32) {
    const float2 hi = out.Xh[e / M][e % M], lo = out.Xl[e / M][e % M];
    w.X[e / M][e % M] = make_double2((double)hi.x + (double)lo.x, (double)hi.y + (double)lo.y);
  }
  __syncwarp();
  warp_refine_step64<M>(w, E, lane);
  for (int e = lane; e < MM; e += 32) split2(w.X[e / M][e % M], out.Xh[e / M][e % M], out.Xl[e / M][e % M]);
  if (lane < M) {
    const double l = w.lam[lane];
    const float lh = (float)l;
    out.lh[lane] = lh;
    out.ll[lane] = (float)(l - (double)lh);
  }
  __syncwarp();
}

// log det B of a Hermitian positive definite B near the identity (given as the FP32 pair
// Bh + Bl in shared memory), by an FP32 Cholesky factorisation on one lane written in terms of
// H = B - I (formed from the pair: Bh - 1 is exact for Bh near 1, then + Bl):
// the pivots are 1 + delta_k with delta_k = H_kk - sum_{m<k} |L_km|^2 computed from small
// quantities, and log det B = sum_k log1p(delta_k). Rounding then perturbs the result by about
// 2^-24 |H| rather than 2^-24 (the Grams of a converging FastFCA iteration are close to the
// identity in the current basis). Returns the value on every lane; NaN if a pivot is not
// positive.
template <int M>
__device__ double warp_logdet_hpd32(const float2 (*Bh)[kMaxM], const float2 (*Bl)[kMaxM], int lane) {
  double ld = 0.0;
  if (lane == 0) {
    float2 L[M][M];
    float il[M];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < M; ++j) {
#pragma unroll
      for (int i = j; i < M; ++i) {
        const float2 bh = Bh[i][j], bl = Bl[i][j];  // B = Bh + Bl; Bh - 1 is exact near 1
        float2 s = make_float2((i == j ? bh.x - 1.f : bh.x) + bl.x, bh.y + bl.y);
#pragma unroll
        for (int k = 0; k < j; ++k) s = csub(s, cmulc(L[i][k], L[j][k]));
        if (i == j) {
          const float d = s.x;  // pivot - 1
          ok = ok && (d > -1.f) && (d < 3.0e38f);
          ld += (double)log1pf(d);
          const float p = 1.f + d;
          il[j] = rsq_nr(p);
          L[j][j] = make_float2(p * il[j], 0.f);
        } else {
          L[i][j] = cscale(s, il[j]);
        }
      }
    }
    if (!ok) ld = __longlong_as_double(0x7ff8000000000000ll);
  }
  return __shfl_sync(0xffffffffu, ld, 0);
}

// ||U||_F^2 - M in FP64 (all lanes get the result).
template <int M, typename C>
__device__ double unitarity_defect(const C (*U)[kMaxM], int lane) {
  double un = 0.0;
  for (int e = lane; e < M * M; e += 32) {
    const C u = U[e / M][e % M];
    un = fma((double)u.x, (double)u.x, fma((double)u.y, (double)u.y, un));
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) un += __shfl_xor_sync(0xffffffffu, un, o);
  return un - (double)M;
}

// P <- P Q in FP64 (Eq. (updatePeff)) with Q given explicitly (FP32 or FP64).
template <int M, typename C>
__device__ void warp_update_basis_q(double2 (*P)[kMaxM], const C (*Q)[kMaxM], int lane) {
  constexpr int kPer = (M * M + 31) / 32;
  double2 out[kPer];
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int e = lane + 32 * t;
    if (e < M * M) {
      const int i = e / M, c = e - (e / M) * M;
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int m = 0; m < M; ++m) s = zfma(P[i][m], c2z(Q[m][c]), s);
      out[t] = s;
    }
  }
  __syncwarp();
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int e = lane + 32 * t;
    if (e < M * M) P[e / M][e % M] = out[t];
  }
  __syncwarp();
}

// P <- P Q in FP64 (Eq. (updatePeff)) with Q given explicitly (FP32 or FP64), for
// 2 M^2 <= 32: lane 2e + part computes the real (part 0) or imaginary (part 1) part of entry
// e as a pairwise sum of its 2M products, which keeps the chain of dependent FP64 operations
// short.
template <int M, typename C>
__device__ void warp_update_basis_q2(double2 (*P)[kMaxM], const C (*Q)[kMaxM], int lane) {
  static_assert(2 * M * M <= 32, "one real part per lane");
  const int e = lane >> 1, part = lane & 1;
  const int i = e / M, c = e % M;
  double v = 0.0;
  if (e < M * M) {
    double t[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const double2 p = P[i][m];
      const double qx = (double)Q[m][c].x, qy = (double)Q[m][c].y;
      t[m] = part ? fma(p.x, qy, p.y * qx) : fma(p.x, qx, -(p.y * qy));
    }
#pragma unroll
    for (int h = 1; h < M; h *= 2)
#pragma unroll
      for (int m = 0; m + h < M; m += 2 * h) t[m] += t[m + h];
    v = t[0];
  }
  __syncwarp();
  if (e < M * M) {
    if (part) P[i][c].y = v;
    else P[i][c].x = v;
  }
  __syncwarp();
}

}  // namespace fca
