// Device building blocks shared by the FCA kernels (sm_103a).
//
//   * complex64 / complex128 arithmetic on float2 / double2;
//   * a warp "transpose" reduction: V per-lane partial sums -> each lane ends with V/32
//     complete warp sums (31 shuffles for 32 values instead of 160 for a butterfly each);
//   * dense Hermitian linear algebra for one frequency bin inside one warp (M <= 8):
//     Cholesky, triangular solves, cyclic Jacobi with the round-robin (parallel) ordering,
//     used for the generalised eigenproblem of Eq. (GEVD) on the FP32 pipe, plus FP64
//     matrix products for the basis update P <- P Q (Eq. (updatePeff)).
//
// Why the eigensolver runs on the FP32 pipe: on GB300 an FP64 FMA has ~64 cycles of
// latency, FP64 division and square root ~650 cycles, and FP64 throughput is 1/62 of FP32
// (measured). A Jacobi sweep is a chain of dependent rotations, so an FP64 solver would
// cost more than the whole per-bin pass of an EM iteration. FP64 is kept where the sums are
// long or the product chain is long: the cross-warp merge of the Gram and log-likelihood
// partial sums, and the accumulated basis P.
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

// --------------------------------------------------- warp-level dense Hermitian algebra
// Matrices are row-major with leading dimension kMaxM, in shared memory. Every function is
// called by all 32 lanes of one warp and ends with __syncwarp().
struct WarpLA {
  float2 A[kMaxM][kMaxM];   // work matrix (eigenproblem)
  float2 L[kMaxM][kMaxM];   // Cholesky factor (lower triangle); L^-1 in the fast solver
  float2 Z[kMaxM][kMaxM];   // temporary
  float2 V[kMaxM][kMaxM];   // eigenvectors / result
  float2 A2[kMaxM][kMaxM];  // ping-pong partners of A and V (fast solver)
  float2 V2[kMaxM][kMaxM];
  float invd[kMaxM];        // 1 / L_ii
  float2 jself[kMaxM + 1];  // Jacobi: J_xx for every index x
  float2 joth[kMaxM + 1];   // Jacobi: J_{partner(x), x}
  int partner[kMaxM + 1];
};

// In-place Cholesky B = L L^H of the Hermitian positive definite matrix in la.L (the lower
// triangle is read and overwritten). Returns false (uniformly across the warp) if a pivot is
// not positive and finite.
template <int M>
__device__ bool warp_cholesky(WarpLA& la, int lane) {
  for (int k = 0; k < M; ++k) {
    __syncwarp();
    const float bkk = la.L[k][k].x;
    if (!(bkk > 0.f) || !(bkk < 3.0e38f)) {
      __syncwarp();
      return false;
    }
    float il = rsqrtf(bkk);
    il = il * fmaf(-0.5f * bkk * il, il, 1.5f);  // Newton step: 1/sqrt(bkk) to rounding
    const float lkk = bkk * il;
    __syncwarp();
    if (lane == k) {
      la.L[k][k] = make_float2(lkk, 0.f);
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
// 2 sum_i log(1/L_ii) + log|det U|^2, where the FP32 rotations leave U unitary only to
// rounding, so log|det U|^2 = log det(U^H U) = ||U||_F^2 - M to first order in U^H U - I.
// Arranged for a short dependency chain:
// one lane factors B = L L^H and inverts L in registers (no warp synchronisation inside the
// recurrences), the congruence W = L^-1 A L^-H and Q = L^-H U are lane-parallel products,
// and the Jacobi rounds ping-pong between two copies of A and V (one __syncwarp fewer per
// round).

// Lane 0: B (lower triangle of la.L) = L L^H; writes L^-1 (lower, zero above) over la.L and
// returns log|det L^-H|^2 = 2 sum_i log(1/L_ii). Result is valid on lane 0 only; *ok too.
template <int M>
__device__ float lane_cholesky_inverse(WarpLA& la, bool* ok) {
  float2 L[M][M];
  float id[M];
  bool good = true;
#pragma unroll
  for (int j = 0; j < M; ++j) {
#pragma unroll
    for (int i = j; i < M; ++i) {
      float2 s = la.L[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) s = csub(s, cmulc(L[i][k], L[j][k]));
      if (i == j) {
        const float piv = s.x;
        good = good && (piv > 0.f) && (piv < 3.0e38f);
        float il = rsqrtf(piv);
        il = il * fmaf(-0.5f * piv * il, il, 1.5f);  // Newton step: 1/sqrt to rounding
        id[j] = il;
        L[j][j] = make_float2(piv * il, 0.f);
      } else {
        L[i][j] = cscale(s, id[j]);
      }
    }
  }
  // L^-1: (L^-1)_ii = id_i; (L^-1)_ij = -id_i sum_{k=j}^{i-1} L_ik (L^-1)_kj for i > j.
  float2 Li[M][M];
  float ld = 0.f;
#pragma unroll
  for (int j = 0; j < M; ++j) {
    Li[j][j] = make_float2(id[j], 0.f);
    ld += 2.f * logf(id[j]);
#pragma unroll
    for (int i = j + 1; i < M; ++i) {
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = j; k < i; ++k) s = cfma(L[i][k], Li[k][j], s);
      Li[i][j] = cscale(s, -id[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < M; ++i) {
    la.invd[i] = id[i];
#pragma unroll
    for (int j = 0; j < M; ++j) la.L[i][j] = (j <= i) ? Li[i][j] : make_float2(0.f, 0.f);
  }
  *ok = good;
  return ld;
}

// la.A <- W = Li A Li^H (Li = la.L, lower triangular), Hermitian by construction.
template <int M>
__device__ void warp_congruence_products(WarpLA& la, int lane) {
  constexpr int kPer = (M * M + 31) / 32;
#pragma unroll
  for (int t = 0; t < kPer; ++t) {  // Z = A Li^H:  Z_ij = sum_{k<=j} A_ik conj(Li_jk)
    const int e = lane + 32 * t;
    if (e < M * M) {
      const int i = e / M, j = e % M;
      float2 s = make_float2(0.f, 0.f);
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
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < M; ++k)
        if (k <= i) s = cfma(la.L[i][k], la.Z[k][j], s);
      if (i == j) {
        la.A[i][i] = make_float2(s.x, 0.f);
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
// enforced by a final copy when needed).
template <int M>
__device__ int warp_jacobi_pp(WarpLA& la, int lane, float tol, int max_sweeps) {
  constexpr int n = M + (M & 1);
  constexpr int kPer = (M * M + 31) / 32;
  for (int e = lane; e < M * M; e += 32) {
    const int i = e / M, j = e - (e / M) * M;
    la.V[i][j] = make_float2(i == j ? 1.f : 0.f, 0.f);
  }
  __syncwarp();
  if (M == 1) return 0;
  const float tol2 = tol * tol;
  float2(*Ac)[kMaxM] = la.A;
  float2(*Vc)[kMaxM] = la.V;
  float2(*An)[kMaxM] = la.A2;
  float2(*Vn)[kMaxM] = la.V2;
  int result = -1;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    int rotated = 0, big = 0;
    for (int r = 0; r < n - 1; ++r) {
      if (lane < n / 2) {
        const int k = lane;
        const int a = (k == 0) ? r : (r + k) % (n - 1);
        const int b = (k == 0) ? n - 1 : (r - k + (n - 1)) % (n - 1);
        const int p = min(a, b), q = max(a, b);
        float c = 1.f, s = 0.f;
        float2 e = make_float2(1.f, 0.f);
        if (q < M) {
          const float app = Ac[p][p].x, aqq = Ac[q][q].x;
          const float2 apq = Ac[p][q];
          const float r2 = cabs2(apq);
          const float den = fabsf(app * aqq);
          if (r2 > tol2 * den && r2 > 1e-36f) {
            big |= (r2 > 1e-8f * den);
            float ir = rsqrtf(r2);
            ir = ir * fmaf(-0.5f * r2 * ir, ir, 1.5f);   // 1 / |a_pq|, Newton-refined
            const float tau = 0.5f * (aqq - app) * ir;
            const float h = fmaf(tau, tau, 1.f);
            const float t = copysignf(__fdividef(1.f, fabsf(tau) + h * rsqrtf(h)), tau);
            const float g = fmaf(t, t, 1.f);
            c = rsqrtf(g);
            c = c * fmaf(-0.5f * g * c, c, 1.5f);         // Newton-refined: c^2 + s^2 = 1
            s = t * c;
            e = cscale(apq, ir);
            rotated = 1;
          }
          la.jself[p] = make_float2(c, 0.f);
          la.joth[p] = cscale(cconj(e), -s);
          la.partner[p] = q;
          la.jself[q] = cscale(cconj(e), c);
          la.joth[q] = make_float2(s, 0.f);
          la.partner[q] = p;
        } else {
          la.jself[p] = make_float2(1.f, 0.f);
          la.joth[p] = make_float2(0.f, 0.f);
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
          const float2 Ji = la.jself[i], Jo_i = la.joth[i], Jl = la.jself[l], Jo_l = la.joth[l];
          const float2 r0 = cfma(Ac[i][lp], Jo_l, cmul(Ac[i][l], Jl));
          const float2 r1 = cfma(Ac[ip][lp], Jo_l, cmul(Ac[ip][l], Jl));
          float2 v = cadd(ccmul(Ji, r0), ccmul(Jo_i, r1));
          if (i == l) v.y = 0.f;
          else if (ip == l) v = make_float2(0.f, 0.f);  // the pivot pair
          An[i][l] = v;
          Vn[i][l] = cfma(Vc[i][lp], Jo_l, cmul(Vc[i][l], Jl));
        }
      }
      __syncwarp();
      float2(*t0)[kMaxM] = Ac;
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
    // First-order finish (as in warp_gevd_reg) once every off-diagonal entry is below 2e-4 of
    // its eigenvalue gap: V <- V (I + X), X_ij = A_ij / (d_j - d_i) (skew-Hermitian, written
    // into the free ping-pong buffer), d_j += sum_p |A_pj|^2 / (d_j - d_p).
    // (Every gap must also stand clear of the eigenvalues' size: degenerate pairs take
    // another sweep.)
    int small = 1;
    for (int e = lane; e < M * M; e += 32) {
      const int i = e / M, j = e % M;
      if (i != j) {
        const float gap = Ac[j][j].x - Ac[i][i].x;
        const float scale = fmaxf(fabsf(Ac[i][i].x), fabsf(Ac[j][j].x));
        small &= (cabs2(Ac[i][j]) <= 4e-8f * gap * gap && fabsf(gap) > 1e-5f * scale) ? 1 : 0;
      }
    }
    if (__all_sync(0xffffffffu, small)) {
      for (int e = lane; e < M * M; e += 32) {
        const int i = e / M, j = e % M;
        An[i][j] = (i != j) ? cscale(Ac[i][j], __fdividef(1.f, Ac[j][j].x - Ac[i][i].x))
                            : make_float2(0.f, 0.f);
      }
      __syncwarp();
      float2 nv[kPer];
      float corr[kPer];
#pragma unroll
      for (int t = 0; t < kPer; ++t) {
        const int e = lane + 32 * t;
        corr[t] = 0.f;
        if (e < M * M) {
          const int i = e / M, j = e % M;
          float2 acc = Vc[i][j];
#pragma unroll
          for (int m = 0; m < M; ++m) acc = cfma(Vc[i][m], An[m][j], acc);
          nv[t] = acc;
          if (i == j) {
#pragma unroll
            for (int p2 = 0; p2 < M; ++p2)
              corr[t] = fmaf(Ac[p2][j].x, An[p2][j].x, fmaf(Ac[p2][j].y, An[p2][j].y, corr[t]));
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
// *ldL. log|det Q|^2 = *ldL + log|det U|^2, where the FP32 rotations leave U unitary only to
// rounding: log|det U|^2 = ||U||_F^2 - M to first order, which the caller sums in FP64 from
// Uout (unitarity_defect). Returns a device status code.
template <int M>
__device__ int warp_gevd_fast(WarpLA& la, int lane, float* sig, float2 (*Qout)[kMaxM],
                              float2 (*Uout)[kMaxM], float* ldL) {
  bool ok = true;
  float ld = 0.f;
  if (lane == 0) ld = lane_cholesky_inverse<M>(la, &ok);
  ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
  __syncwarp();
  if (!ok) return kErrNotPD;
  warp_congruence_products<M>(la, lane);
  const int sw = warp_jacobi_pp<M>(la, lane, 2.0e-7f, 30);
  if (sw < 0) return kErrEigNoConv;
  if (lane < M) sig[lane] = la.A[lane][lane].x;
  constexpr int kPer = (M * M + 31) / 32;
#pragma unroll
  for (int t = 0; t < kPer; ++t) {  // Q_ij = sum_{k>=i} conj(Li_ki) U_kj
    const int e = lane + 32 * t;
    if (e < M * M) {
      const int i = e / M, j = e % M;
      float2 s = make_float2(0.f, 0.f);
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
    const float sv = sig[i];
    if (!(sv > 0.f) || !(sv < 3.0e38f)) return kErrNotPD;
  }
  return kOk;
}

// ------------------------------------------------------ register-resident solver, M <= 4
__device__ __forceinline__ float2 shfl2(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
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
// exceeded 1e-4 of sqrt(|a_pp a_qq|), or with the first-order step once every off-diagonal
// entry is below 2e-4 of its eigenvalue gap. Called by all 32 lanes.
template <int M>
__device__ int warp_gevd_reg(const float2 (*A)[kMaxM], float2 (*B)[kMaxM], float* sig,
                             float2 (*Qout)[kMaxM], float2 (*Uout)[kMaxM], float* ldL, float tol,
                             int max_sweeps, int lane) {
  static_assert(M >= 1 && M <= 4, "one entry per lane: M*M <= 32 (and sized for M <= 4)");
  constexpr int MM = M * M;
  constexpr int n = M + (M & 1);
  const bool own = lane < MM;
  const int i = own ? lane / M : 0, j = own ? lane % M : 0;
  // 1. Cholesky and L^-1 on lane 0.
  int ok = 1;
  float ld = 0.f;
  if (lane == 0) {
    float2 L[M][M];
    float id[M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
#pragma unroll
      for (int r = c; r < M; ++r) {
        float2 sv = B[r][c];
#pragma unroll
        for (int k = 0; k < c; ++k) sv = csub(sv, cmulc(L[r][k], L[c][k]));
        if (r == c) {
          const float piv = sv.x;
          ok = ok && (piv > 0.f) && (piv < 3.0e38f);
          float il = rsqrtf(piv);
          il = il * fmaf(-0.5f * piv * il, il, 1.5f);  // Newton step: 1/sqrt to rounding
          id[c] = il;
          L[c][c] = make_float2(piv * il, 0.f);
        } else {
          L[r][c] = cscale(sv, id[c]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < M; ++c) {
      B[c][c] = make_float2(id[c], 0.f);
      ld += 2.f * logf(id[c]);
#pragma unroll
      for (int r = c + 1; r < M; ++r) {
        float2 sv = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = c; k < r; ++k) sv = cfma(L[r][k], (k == c) ? make_float2(id[c], 0.f) : B[k][c], sv);
        B[r][c] = cscale(sv, -id[r]);
        B[c][r] = make_float2(0.f, 0.f);
      }
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  ld = __shfl_sync(0xffffffffu, ld, 0);
  __syncwarp();
  if (!ok) return kErrNotPD;
  // 2. W = Li A Li^H: T = A Li^H (T_ij = sum_{k<=j} A_ik conj(Li_jk)), W_ij = sum_{k<=i} Li_ik T_kj.
  float2 T = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < M; ++k)
    if (k <= j) T = cadd(T, cmulc(A[i][k], B[j][k]));
  float2 W = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const float2 tk = shfl2(T, own ? k * M + j : lane);
    if (k <= i) W = cfma(B[i][k], tk, W);
  }
  {  // exactly Hermitian: the lower triangle mirrors the upper one
    const float2 wt = shfl2(W, own ? j * M + i : lane);
    if (i > j) W = cconj(wt);
    if (i == j) W.y = 0.f;
  }
  float2 V = make_float2(i == j ? 1.f : 0.f, 0.f);
  // 3. Jacobi sweeps.
  const float tol2 = tol * tol;
  int sweeps = (M == 1) ? 0 : -1;
  for (int sweep = 0; sweep < max_sweeps && M > 1; ++sweep) {
    int rotated = 0, big = 0;
#pragma unroll
    for (int r = 0; r < n - 1; ++r) {
      const int pi = rr_partner(i, r, n), pj = rr_partner(j, r, n);
      const int p = min(i, pi), q = max(i, pi);
      const bool valid = own && q < M;
      const float app = __shfl_sync(0xffffffffu, W.x, valid ? p * M + p : lane);
      const float aqq = __shfl_sync(0xffffffffu, W.x, valid ? q * M + q : lane);
      const float2 apq = shfl2(W, valid ? p * M + q : lane);
      float2 Jii = make_float2(1.f, 0.f), Joi = make_float2(0.f, 0.f);  // J_{i i}, J_{i' i}
      bool act = false;
      if (valid) {
        const float r2 = cabs2(apq);
        const float den = fabsf(app * aqq);
        if (r2 > tol2 * den && r2 > 1e-36f) {
          act = true;
          big |= (r2 > 1e-8f * den);
          float ir = rsqrtf(r2);
          ir = ir * fmaf(-0.5f * r2 * ir, ir, 1.5f);
          const float tau = 0.5f * (aqq - app) * ir;
          const float h = fmaf(tau, tau, 1.f);
          const float t = copysignf(__fdividef(1.f, fabsf(tau) + h * rsqrtf(h)), tau);
          const float g = fmaf(t, t, 1.f);
          float c = rsqrtf(g);
          c = c * fmaf(-0.5f * g * c, c, 1.5f);
          const float sv = t * c;
          const float2 e = cscale(apq, ir);
          if (i == p) {  // J_pp = c, J_qp = -s conj(e)
            Jii = make_float2(c, 0.f);
            Joi = cscale(cconj(e), -sv);
          } else {       // J_qq = c conj(e), J_pq = s
            Jii = cscale(cconj(e), c);
            Joi = make_float2(sv, 0.f);
          }
        }
      }
      rotated |= act;
      // J of the column index j: computed by lane (j, 0), whose row index is j.
      const float2 Jll = shfl2(Jii, own ? j * M : lane);
      const float2 Jol = shfl2(Joi, own ? j * M : lane);
      const bool ip_ok = pi < M, jp_ok = pj < M;
      const float2 W_il2 = shfl2(W, own && jp_ok ? i * M + pj : lane);
      const float2 W_i2l = shfl2(W, own && ip_ok ? pi * M + j : lane);
      const float2 W_i2l2 = shfl2(W, own && ip_ok && jp_ok ? pi * M + pj : lane);
      const float2 V_il2 = shfl2(V, own && jp_ok ? i * M + pj : lane);
      // W' = J^H W J restricted to entry (i, j); V' = V J.
      float2 r0 = cmul(W, Jll), r1 = cmul(W_i2l, Jll);
      if (jp_ok) {
        r0 = cfma(W_il2, Jol, r0);
        r1 = cfma(W_i2l2, Jol, r1);
      }
      float2 Wn = ccmul(Jii, r0);
      if (ip_ok) Wn = cadd(Wn, ccmul(Joi, r1));
      float2 Vn = cmul(V, Jll);
      if (jp_ok) Vn = cfma(V_il2, Jol, Vn);
      if (i == j) Wn.y = 0.f;
      if (act && j == pi) Wn = make_float2(0.f, 0.f);  // the pivot pair
      W = Wn;
      V = Vn;
    }
    rotated = __any_sync(0xffffffffu, rotated);
    big = __any_sync(0xffffffffu, big);
    if (!rotated || !big) {
      sweeps = sweep + 1;
      break;
    }
    const float di = __shfl_sync(0xffffffffu, W.x, own ? i * M + i : lane);
    const float dj = __shfl_sync(0xffffffffu, W.x, own ? j * M + j : lane);
    const float gap = dj - di;
    // (Every gap must also stand clear of the eigenvalues' size: degenerate pairs take
    // another sweep.)
    const bool small = !own || i == j ||
                       (cabs2(W) <= 4e-8f * gap * gap && fabsf(gap) > 1e-5f * fmaxf(fabsf(di), fabsf(dj)));
    if (__all_sync(0xffffffffu, small)) {
      // First-order step: V <- V (I + X), X_ij = W_ij / (d_j - d_i);
      // d_j += sum_p |W_pj|^2 / (d_j - d_p).
      const float2 X = (own && i != j) ? cscale(W, __fdividef(1.f, gap)) : make_float2(0.f, 0.f);
      float2 Vn = V;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const float2 vim = shfl2(V, own ? i * M + m : lane);
        const float2 xmj = shfl2(X, own ? m * M + j : lane);
        Vn = cfma(vim, xmj, Vn);
      }
      const float e2 = W.x * X.x + W.y * X.y;  // |W_ij|^2 / (d_j - d_i)
      float corr = 0.f;
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
  float2 Qv = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const float2 vkj = shfl2(V, own ? k * M + j : lane);
    if (k >= i) Qv = cadd(Qv, ccmul(B[k][i], vkj));
  }
  if (own) {
    Qout[i][j] = Qv;
    Uout[i][j] = V;
    if (i == j) sig[i] = W.x;
  }
  const bool pos = !own || i != j || ((W.x > 0.f) && (W.x < 3.0e38f));
  *ldL = ld;
  __syncwarp();
  return __all_sync(0xffffffffu, pos) ? kOk : kErrNotPD;
}

// ||U||_F^2 - M in FP64 (all lanes get the result).
template <int M>
__device__ double unitarity_defect(const float2 (*U)[kMaxM], int lane) {
  double un = 0.0;
  for (int e = lane; e < M * M; e += 32) {
    const float2 u = U[e / M][e % M];
    un = fma((double)u.x, (double)u.x, fma((double)u.y, (double)u.y, un));
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) un += __shfl_xor_sync(0xffffffffu, un, o);
  return un - (double)M;
}

// P <- P Q in FP64 (Eq. (updatePeff)) with Q given explicitly (FP32).
template <int M>
__device__ void warp_update_basis_q(double2 (*P)[kMaxM], const float2 (*Q)[kMaxM], int lane) {
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

// P <- P Q in FP64 (Eq. (updatePeff)) with Q given explicitly (FP32), for 2 M^2 <= 32: lane
// 2e + part computes the real (part 0) or imaginary (part 1) part of entry e as a pairwise sum
// of its 2M products, which keeps the chain of dependent FP64 operations short.
template <int M>
__device__ void warp_update_basis_q2(double2 (*P)[kMaxM], const float2 (*Q)[kMaxM], int lane) {
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

// P <- P Q in FP64 (Eq. (updatePeff)); P in shared memory [M][M] double2, Q = la.V (FP32).
template <int M>
__device__ void warp_update_basis(double2 (*P)[kMaxM], const WarpLA& la, int lane) {
  constexpr int kPer = (M * M + 31) / 32;
  double2 out[kPer];
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int e = lane + 32 * t;
    if (e < M * M) {
      const int i = e / M, c = e - (e / M) * M;
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int m = 0; m < M; ++m) s = zfma(P[i][m], c2z(la.V[m][c]), s);
      out[t] = s;
    }
  }
  __syncwarp();
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int e = lane + 32 * t;
    if (e < M * M) {
      const int i = e / M, c = e - (e / M) * M;
      P[i][c] = out[t];
    }
  }
  __syncwarp();
}

}  // namespace fca
