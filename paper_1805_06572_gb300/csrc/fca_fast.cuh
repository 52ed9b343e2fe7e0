// FastFCA (Ito, Araki, Nakatani, arXiv 1805.06572, Sec. 3, Algorithm 1) on sm_103a.
//
// One CTA owns one frequency bin f for all L iterations (every quantity of the EM is
// indexed by f and Eq. (like) factorises over f, so CTAs never communicate). Per iteration:
//   bin pass (FP32, one thread per time-frequency point, frames strided over the CTA):
//     yt = P^H y                                        Eq. (tildey)
//     d_i = v1 lam_i + v2, mut1 = v1 lam yt / d,        Eq. (MMSEtilde)
//       mut2 = v2 yt / d
//     c_i = v1 v2 lam_i / d_i                           Eq. (updatePhitildeeff), diagonal
//     v1' = (1/M) sum_i (|mut1_i|^2 + c_i) / lam_i      Eq. (updateveff)
//     v2' = (1/M) sum_i (|mut2_i|^2 + c_i)
//     St_j += (mut_j mut_j^H + diag(c)) / v_j'          Eq. (updateStildeeff), partial sums
//     log-likelihood terms log d_i + |yt_i|^2 / d_i     Eq. (like) in the transformed basis
//   CTA reduction: per-lane FP32 partials -> warp transpose-reduction (FP32) -> cross-warp
//     merge in a fixed order (bitwise reproducible): the Gram entries in the precision G of
//     the eigensolver they feed (FP32, or FP64), the log-likelihood sums compensated into
//     FP64;
//   one warp (the role rotates over the CTA's warps with the iteration): the generalised
//     eigenproblem of (St1, St2) (Algorithm 1, step 8) in precision G and the next basis P^H
//     for the bin pass; meanwhile the next warp does the previous iteration's FP64
//     bookkeeping: P <- P Q (Eq. (updatePeff)), Lambda <- Sigma (Eq. (updateLambdaeff)),
//     and a third (or the same) warp log det S2 <- log det S2 - log|det Q|^2
//     (S2 = P^-H P^-1 for the basis in use) and the previous iteration's log-likelihood.
// The log-likelihood of iteration l uses log det Rx = sum_i log d_i + log det S2 and
// y^H Rx^-1 y = sum_i |yt_i|^2 / d_i, which follow from Rx = P^-H (v1 Lam + v2 I) P^-1.
// The mixture and v stay in shared memory across iterations when they fit.
#pragma once
#include <type_traits>

#include "fca_dev.cuh"
#include "fca_internal.h"

namespace fca {

// Precision modes of the per-bin generalised eigenproblem (FCA_GEVD_* in fca.h):
//   0  FP32 merge of the Gram partials, FP32 Cholesky + Jacobi, FP32 Q;
//   1  FP64 merge, FP64 Cholesky + Jacobi, FP64 Q;
//   2  compensated FP32 merge (pairs), FP32 Newton-type iteration (or Cholesky + Jacobi), one
//      refinement step of Q with compensated FP32 residuals (a second, FP64 step after a poor start); Q and Sigma
//      as FP32 pairs, made FP64 by the deferred bookkeeping.
template <int GM> struct GevdTypes;
template <> struct GevdTypes<0> { using Merge = float; using Solve = float; using Out = float; };
template <> struct GevdTypes<1> { using Merge = double; using Solve = double; using Out = double; };
template <> struct GevdTypes<2> { using Merge = double; using Solve = float; using Out = double; };
struct NoRefine {};

// The EM state of one frequency bin in shared memory. NWR: warps whose partial sums the bin
// pass leaves in red.
template <int M, int NWR, int GM>
struct FastBin {
  using Ty = GevdTypes<GM>;
  using SolveT = typename Ty::Solve;
  using OutT = typename Ty::Out;
  static constexpr int V = 2 * M * M + 2;  // two Grams (M^2 reals each), sum log d, sum p/d
  float red[NWR][V];
  double2 P[M][kMaxM];      // basis P (FP64); M x M matrices with leading dimension kMaxM
  float2 P32[M][kMaxM];     // P rounded to FP32
  float2 P32lo[M][kMaxM];   // P - P32 rounded to FP32 (FP64 modes: the next basis is
                            //   published from the pairs of P and Q)
  float2 PH[M][M];              // FP32 P^H (times the decode scale) used by the bin pass
  float lam[M], ilam[M];
  double lam64[kMaxM];
  // Double-buffered results of an iteration's eigensolve, consumed by the deferred FP64
  // bookkeeping one iteration later.
  Cx<OutT> Q[2][M][kMaxM];
  Cx<SolveT> U[2][M][kMaxM];
  OutT sig[2][kMaxM];
  // FP64 modes: Q = Qh + Ql and Sigma = sigh + sigl as FP32 pairs (the refined eigensolver's
  // own result, from which the deferred bookkeeping forms Q and Sigma in FP64)
  float2 Qh[2][M][kMaxM];
  float2 Ql[2][M][kMaxM];
  float sigh[2][kMaxM], sigl[2][kMaxM];
  OutT ldL[2];       // modes 0, 1: 2 sum log(1/L_ii), log|det Q|^2 = ldL + log|det U|^2;
                     // mode 2: log|det Q|^2 itself (= -log det St2)
  double llt[2][2];  // sum log d, sum p/d of the iteration
  double logdetS2;
  int fail;          // read by every thread after a barrier; written only before one
  int fail_pending;  // set by the deferred log-likelihood, read after the iteration's barrier
};

// Workspace of the per-bin eigensolver (one bin at a time).
template <int M, int GM>
struct FastWork {
  WarpLAT<typename GevdTypes<GM>::Solve, M> la;
  typename std::conditional<GM == 2, RefineWork<M>, NoRefine>::type rf;
};

template <int M, int NW, int GM>
struct FastShared : FastBin<M, NW, GM> {
  int wid0;  // hardware warp slot of warp 0 (chooses the warps' roles)
  FastWork<M, GM> w;
};

// Where one bin's time-frequency points and source powers are, for the bin pass.
template <int ST>
struct BinIO {
  const typename Elem<ST>::T* y;  // the bin's mixture, [N][M] (shared memory or global)
  float* v1;                      // v_1(., bin), v_2(., bin): working copies
  float* v2;
  float* vg1;                     // v_1(., bin) in global memory (v_2 lies dv2 after it)
  int dv2;
  ptrdiff_t d_prev;               // v_prev - v
  int N;
  float vf, gi;                   // positivity floor, decode scale 1/g_f
};

// Warp roles of iteration `it`: the eigensolver (and the publication of the next basis), the
// deferred basis update and the deferred log-likelihood. A warp issues from the SM
// sub-partition (scheduler) of its hardware warp slot modulo 4, and the per-bin tail is a
// long single-warp chain, so the solver's slot rotates with the iteration and with the CTA's
// first slot: the tails of the CTAs sharing an SM spread over its schedulers instead of all
// landing on the scheduler of warp 0. (The arithmetic does not depend on the warp.)
template <int NW>
__device__ __forceinline__ int solver_warp(int it, int wid0) {
  return ((it + (wid0 >> 2) - wid0) & 3) % NW;
}

__host__ __device__ constexpr int pair_index(int M, int i, int k) {  // i < k
  return i * (M - 1) - i * (i - 1) / 2 + (k - i - 1);
}

// Resident CTAs per SM the register budget is sized for (one CTA per frequency bin: more
// CTAs per SM hide each CTA's serial per-bin eigensolver behind the others' bin passes).
__host__ __device__ constexpr int fast_min_blocks(int M) { return M <= 4 ? 4 : (M <= 6 ? 3 : 2); }
// The same register budget per thread for every CTA size.
__host__ __device__ constexpr int fast_min_blocks(int M, int NT) {
  return fast_min_blocks(M) * 128 / NT > 0 ? fast_min_blocks(M) * 128 / NT : 1;
}

// Value v of the per-warp partial-sum vector -> the Hermitian matrix entry it belongs to:
// Gram g (0, 1), row i, column k (i <= k), and part (0 = real, 1 = imaginary).
template <int M>
__device__ __forceinline__ void value_entry(int v, int* g, int* i, int* k, int* part) {
  constexpr int MM = M * M;
  *g = v / MM;
  int r = v - *g * MM;
  if (r < M) {
    *i = *k = r;
    *part = 0;
    return;
  }
  r -= M;
  *part = r & 1;
  int pr = r >> 1, row = 0;
  while (pr >= M - 1 - row) {
    pr -= M - 1 - row;
    ++row;
  }
  *i = row;
  *k = row + 1 + pr;
}

// Store one merged Gram value v of entry (i, k) (part: real 0 / imaginary 1) into the
// Hermitian matrix D (both triangles).
template <int M, typename C, typename T>
__device__ __forceinline__ void merge_store(C (*D)[kMaxM], int i, int k, int part, T v) {
  if (i == k) {
    D[i][i].x = v;
    D[i][i].y = T(0);
  } else if (part == 0) {
    D[i][k].x = v;
    D[k][i].x = v;
  } else {
    D[i][k].y = v;
    D[k][i].y = -v;
  }
}

// Deferred FP64 bookkeeping of iteration `it`, in two parts that may run on two warps at once.
// Basis part: P <- P Q (Eq. (updatePeff)) and its FP32 copy, Lambda <- Sigma
// (Eq. (updateLambdaeff)), and at it = L-2 the basis of iteration L-1.
template <int M, int GM, typename Sh>
__device__ void fast_deferred_basis(Sh& sh, const FastEmArgs& a, int f, int it, int lane) {
  constexpr int MM = M * M;
  const int b = it & 1;
  if constexpr (GM == 2) {  // Q and Sigma in FP64 from the eigensolver's pairs
    for (int e = lane; e < MM; e += 32) {
      const float2 hi = sh.Qh[b][e / M][e % M], lo = sh.Ql[b][e / M][e % M];
      sh.Q[b][e / M][e % M] = make_double2((double)hi.x + (double)lo.x, (double)hi.y + (double)lo.y);
    }
    if (lane < M) sh.sig[b][lane] = (double)sh.sigh[b][lane] + (double)sh.sigl[b][lane];
    __syncwarp();
  }
  if constexpr (2 * MM <= 32) {
    warp_update_basis_q2<M>(sh.P, sh.Q[b], lane);
  } else {
    warp_update_basis_q<M>(sh.P, sh.Q[b], lane);
  }
  for (int e = lane; e < MM; e += 32) split2(sh.P[e / M][e % M], sh.P32[e / M][e % M], sh.P32lo[e / M][e % M]);
  if (lane < M) sh.lam64[lane] = (double)sh.sig[b][lane];
  __syncwarp();
  if (it == a.iters - 2) {  // the parameters of iteration L-1
    for (int e = lane; e < MM; e += 32) a.P_prev[(size_t)f * MM + e] = sh.P[e / M][e % M];
    if (lane < M) a.lam_prev[(size_t)f * M + lane] = sh.lam64[lane];
  }
}

// Log-likelihood part: the log-likelihood of iteration it (at its own parameters), then
// log det S2 = -log|det P|^2 of the next basis (subtract log|det Q|^2 of the Q applied), and
// at it = L-2 that of iteration L-1.
template <int M, int GM, typename Sh>
__device__ void fast_deferred_ll(Sh& sh, const FastEmArgs& a, int f, int N, int it, int lane) {
  const int b = it & 1;
  if (lane == 0) {
    const double ll = -(double)N * M * 1.1447298858494002 - sh.llt[b][0] - sh.llt[b][1] -
                      (double)N * sh.logdetS2;
    a.llf[(size_t)it * a.F + f] = ll;
    if (!isfinite(ll)) {
      set_status(a.status, kErrNonFinite);
      sh.fail_pending = kErrNonFinite;
    }
  }
  const double ldQ = (GM == 2) ? (double)sh.ldL[b] : (double)sh.ldL[b] + unitarity_defect<M>(sh.U[b], lane);
  if (lane == 0) {
    sh.logdetS2 -= ldQ;
    if (it == a.iters - 2) a.logdetS2_prev[f] = sh.logdetS2;
  }
  __syncwarp();
}

// Refined mode, log-likelihood warp: the basis Q of iteration it is St2-orthonormal, so
// log|det Q|^2 = -log det St2 (from the merged Gram's pair, read-only during the tail).
template <int M, int GM, typename Sh>
__device__ void fast_logdet(Sh& sh, FastWork<M, GM>& w, int it, int lane) {
  if constexpr (GM == 2) {
    const double ld = warp_logdet_hpd32<M>(w.rf.Bh, w.rf.Bl, lane);
    if (lane == 0) sh.ldL[it & 1] = -ld;
  }
}

// Load one bin's parameters into its shared state (threads t < MM, M, 1 of the caller's).
template <int M, typename Sh>
__device__ void fast_load_params(Sh& sh, const FastEmArgs& a, int f, int t) {
  constexpr int MM = M * M;
  if (t < MM) {
    const double2 p = a.P[(size_t)f * MM + t];
    sh.P[t / M][t % M] = p;
    split2(p, sh.P32[t / M][t % M], sh.P32lo[t / M][t % M]);
  }
  if (t < M) {
    const double l = a.lam[(size_t)f * M + t];
    sh.lam64[t] = l;
    sh.lam[t] = (float)l;
    sh.ilam[t] = 1.f / (float)l;
  }
  if (t == 0) {
    sh.logdetS2 = a.logdetS2[f];
    sh.fail = 0;
    sh.fail_pending = 0;
  }
}

// After fast_load_params (and a barrier): the FP32 P^H of the first pass, and the parameters
// of iteration L-1 when L = 1.
template <int M, typename Sh>
__device__ void fast_first_basis(Sh& sh, const FastEmArgs& a, int f, float gi, int t) {
  constexpr int MM = M * M;
  if (t < MM) {
    const int i = t / M, m = t % M;
    const double2 p = sh.P[m][i];
    sh.PH[i][m] = make_float2((float)p.x * gi, -(float)p.y * gi);
  }
  if (a.iters == 1) {
    if (t < MM) a.P_prev[(size_t)f * MM + t] = sh.P[t / M][t % M];
    if (t < M) a.lam_prev[(size_t)f * M + t] = sh.lam64[t];
    if (t == 0) a.logdetS2_prev[f] = sh.logdetS2;
  }
}

// Stage one bin's mixture and initial source powers in shared memory (ys, vs), threads
// t < nthr of the caller's. Batches (kB) with separate initial values start the working copy
// of a streaming bin from them instead.
template <int M, int ST, bool kB>
__device__ void fast_stage(const typename Elem<ST>::T* yg, typename Elem<ST>::T* ys, float* vs,
                           float* vg1, int dv2, ptrdiff_t d_in, int N, bool res, int t, int nthr) {
  using E = typename Elem<ST>::T;
  if (res) {
    const size_t bytes = (size_t)N * M * sizeof(E);
    if ((bytes & 15) == 0 && (!kB || (reinterpret_cast<uintptr_t>(yg) & 15) == 0)) {
      const uint4* src = reinterpret_cast<const uint4*>(yg);
      uint4* dst = reinterpret_cast<uint4*>(ys);
      for (size_t i = t; i < bytes / 16; i += nthr) dst[i] = src[i];
    } else {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(yg);
      uint32_t* dst = reinterpret_cast<uint32_t*>(ys);
      for (size_t i = t; i < bytes / 4; i += nthr) dst[i] = src[i];
    }
    for (int n = t; n < N; n += nthr) {
      vs[n] = vg1[d_in + n];
      vs[N + n] = vg1[d_in + dv2 + n];
    }
  } else if (kB && d_in != 0) {
    for (int n = t; n < N; n += nthr) {
      vg1[n] = vg1[d_in + n];
      vg1[dv2 + n] = vg1[d_in + dv2 + n];
    }
  }
}

// One bin pass (Eqs. (tildey), (MMSEtilde), (updatePhitildeeff), (updateveff),
// (updateStildeeff) and the Eq. (like) terms, FP32): thread t of nthr (whole warps) takes
// frames t, t + nthr, ... (M = 8: lane pairs share a frame), updates v, and leaves its warp's
// partial sums in red_row. last: keep the incoming v as v_prev (the E-step of iteration L-1).
template <int M, int ST, typename Sh>
__device__ void fast_pass(Sh& sh, const BinIO<ST>& io, int t, int nthr, bool last, float* red_row,
                          int lane) {
  constexpr int MM = M * M;
  constexpr int V = 2 * MM + 2;
  constexpr bool kHoist = (M <= 4);
  // M = 8: a lane pair shares each time-frequency point and lane parity q accumulates Gram q
  // only (two 8 x 8 Grams per thread, 130 partial sums, do not fit in registers; at M = 7 they
  // still do, and one lane per point is faster).
  constexpr bool kPair = (M >= 8);
  using RS = RedShape<kPair ? MM + 2 : V>;
  float acc[RS::NA];
  const int q = kPair ? (lane & 1) : 0;
#pragma unroll
  for (int j = 0; j < RS::NA; ++j) acc[j] = 0.f;
  float2 ph[kHoist ? M : 1][kHoist ? M : 1];
  float lamr[M];
  if constexpr (kHoist) {
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
      for (int m = 0; m < M; ++m) ph[i][m] = sh.PH[i][m];
  }
#pragma unroll
  for (int i = 0; i < M; ++i) lamr[i] = sh.lam[i];
  const int N = io.N;
  const float vf = io.vf;
  float* v1p = io.v1;
  float* v2p = io.v2;

  for (int n = kPair ? (t >> 1) : t; n < N; n += kPair ? nthr / 2 : nthr) {
    float2 yv[M];
    load_bin<M, ST>(io.y + (size_t)n * M, yv);
    const float v1 = v1p[n], v2 = v2p[n];
    if (last && q == 0) {
      io.vg1[io.d_prev + n] = v1;
      io.vg1[io.d_prev + io.dv2 + n] = v2;
    }
    float2 yt[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
      float2 s;
      if constexpr (kHoist) {
        s = cmul(ph[i][0], yv[0]);
#pragma unroll
        for (int m = 1; m < M; ++m) s = cfma(ph[i][m], yv[m], s);
      } else {
        s = cmul(sh.PH[i][0], yv[0]);
#pragma unroll
        for (int m = 1; m < M; ++m) s = cfma(sh.PH[i][m], yv[m], s);
      }
      yt[i] = s;
    }
    // With r_i = 1/d_i, t_i = lam_i r_i and q_i = |yt_i|^2 r_i^2 (d_i = v1 lam_i + v2):
    //   v1' = (v1/M)(v1 sum lam_i q_i + v2 sum r_i)     (Eq. (updateveff), j = 1)
    //   v2' = (v2/M)(v2 sum q_i + v1 sum t_i)           (Eq. (updateveff), j = 2)
    //   mut1_i / sqrt(v1') = (v1 / sqrt(v1')) t_i yt_i, mut2_i / sqrt(v2') = (v2 / sqrt(v2')) r_i yt_i
    //   c_i / v_j' = (v1 v2 / v_j') t_i                 (Eq. (updatePhitildeeff))
    float r[M], tt[M], pp[M];
    float sA = 0.f, sB = 0.f, sC = 0.f, sD = 0.f, ql = 0.f;
    float lg2 = 0.f;  // sum_i log2 d_i (hardware log2 per factor)
#pragma unroll
    for (int i = 0; i < M; ++i) {
      const float d = fmaf(v1, lamr[i], v2);
      r[i] = __fdividef(1.f, d);
      pp[i] = cabs2(yt[i]);
      tt[i] = lamr[i] * r[i];
      const float pr = pp[i] * r[i];
      const float qq = pr * r[i];
      sA = fmaf(lamr[i], qq, sA);
      sB += r[i];
      sC += qq;
      sD += tt[i];
      ql += pr;
      lg2 += __log2f(d);
    }
    const float v1n = fmaxf((v1 * (1.f / M)) * fmaf(v1, sA, v2 * sB), vf);
    const float v2n = fmaxf((v2 * (1.f / M)) * fmaf(v2, sC, v1 * sD), vf);
    if (q == 0) {
      v1p[n] = v1n;
      v2p[n] = v2n;
    }
    const float rs1 = rsqrtf(v1n), rs2 = rsqrtf(v2n);
    const float a1 = v1 * rs1, a2 = v2 * rs2;
    const float v12 = v1 * v2;
    const float k1 = v12 * (rs1 * rs1), k2 = v12 * (rs2 * rs2);
    if constexpr (kPair) {
      // Gram q of this lane: weights s_q,i (s_1,i = a1 t_i, s_2,i = a2 r_i) and k_q.
      const float kq = q ? k2 : k1;
      const float aq = q ? a2 : a1;
      float sq[M];
#pragma unroll
      for (int i = 0; i < M; ++i) {
        sq[i] = aq * (q ? r[i] : tt[i]);
        acc[i] = fmaf(sq[i] * sq[i], pp[i], fmaf(kq, tt[i], acc[i]));
      }
#pragma unroll
      for (int i = 0; i < M; ++i)
#pragma unroll
        for (int k = i + 1; k < M; ++k) {
          const int o = M + 2 * pair_index(M, i, k);
          const float2 z = cmulc(yt[i], yt[k]);  // yt_i conj(yt_k)
          const float w = sq[i] * sq[k];
          acc[o] = fmaf(w, z.x, acc[o]);
          acc[o + 1] = fmaf(w, z.y, acc[o + 1]);
        }
      acc[MM] += q ? 0.f : 0.6931471805599453f * lg2;
      acc[MM + 1] += q ? 0.f : ql;
    } else {
      float s1[M], s2[M];
#pragma unroll
      for (int i = 0; i < M; ++i) {
        s1[i] = a1 * tt[i];
        s2[i] = a2 * r[i];
        acc[i] = fmaf(s1[i] * s1[i], pp[i], fmaf(k1, tt[i], acc[i]));
        acc[MM + i] = fmaf(s2[i] * s2[i], pp[i], fmaf(k2, tt[i], acc[MM + i]));
      }
#pragma unroll
      for (int i = 0; i < M; ++i)
#pragma unroll
        for (int k = i + 1; k < M; ++k) {
          const int o = M + 2 * pair_index(M, i, k);
          const float2 z = cmulc(yt[i], yt[k]);  // yt_i conj(yt_k)
          const float w1 = s1[i] * s1[k], w2 = s2[i] * s2[k];
          acc[o] = fmaf(w1, z.x, acc[o]);
          acc[o + 1] = fmaf(w1, z.y, acc[o + 1]);
          acc[MM + o] = fmaf(w2, z.x, acc[MM + o]);
          acc[MM + o + 1] = fmaf(w2, z.y, acc[MM + o + 1]);
        }
      acc[2 * MM] += 0.6931471805599453f * lg2;
      acc[2 * MM + 1] += ql;
    }
  }
  if constexpr (kPair) {
    warp_reduce_store_pairs<MM>(acc, lane, red_row);
  } else {
    warp_reduce_store<V>(acc, lane, red_row);
  }
}

// Merge the NWR warp partials of a bin in a fixed order: Gram entries in the eigensolver's
// merge precision (FP32 sums; the FP32 warp partials summed in FP64; or, refined mode, summed
// as compensated FP32 pairs) into the solver's work matrices, the two log-likelihood sums with
// a compensated two-float sum kept in FP64 into llt[b]. Threads t < nthr of the caller's, one
// value per thread.
template <int M, int NWR, int GM, typename Sh>
__device__ void fast_merge(Sh& sh, FastWork<M, GM>& w, int b, double invN, int t, int nthr) {
  using MT = typename GevdTypes<GM>::Merge;
  using ST2 = typename GevdTypes<GM>::Solve;
  constexpr int MM = M * M;
  constexpr int V = 2 * MM + 2;
  for (int e = t; e < V; e += nthr) {
    if (GM == 2 && e < 2 * MM) {
      // Refined mode: the warp partials summed as an unevaluated FP32 pair (TwoSum), scaled by
      // 1/N given as a pair (TwoProduct): hi + lo carries the merged Gram entry to about 2^-48,
      // as the refinement step needs, on the FP32 pipe; hi is the FP32 solver's copy.
      float hi = sh.red[0][e], lo = 0.f;
#pragma unroll
      for (int k = 1; k < NWR; ++k) {
        float err;
        two_sum(hi, sh.red[k][e], hi, err);
        lo += err;
      }
      const float ih = (float)invN, il = (float)(invN - (double)ih);
      const float p = hi * ih;
      const float pe = fmaf(hi, ih, -p);
      float h, l;
      two_sum(p, fmaf(hi, il, fmaf(lo, ih, pe)), h, l);
      int g, i, k, part;
      value_entry<M>(e, &g, &i, &k, &part);
      merge_store<M>(g ? w.la.L : w.la.A, i, k, part, h);
      if constexpr (GM == 2) {
        merge_store<M>(g ? w.rf.Bh : w.rf.Ah, i, k, part, h);
        merge_store<M>(g ? w.rf.Bl : w.rf.Al, i, k, part, l);
      }
    } else if (e < 2 * MM) {
      MT sv[NWR];
#pragma unroll
      for (int k = 0; k < NWR; ++k) sv[k] = (MT)sh.red[k][e];
#pragma unroll
      for (int h = 1; h < NWR; h *= 2)
#pragma unroll
        for (int k = 0; k + h < NWR; k += 2 * h) sv[k] += sv[k + h];
      const MT val = sv[0] * (MT)invN;
      int g, i, k, part;
      value_entry<M>(e, &g, &i, &k, &part);
      merge_store<M>(g ? w.la.L : w.la.A, i, k, part, (ST2)val);
    } else {
      float hi = sh.red[0][e], lo = 0.f;
#pragma unroll
      for (int k = 1; k < NWR; ++k) {  // TwoSum (Knuth): hi + lo = exact running sum
        const float x = sh.red[k][e];
        const float s = hi + x;
        const float bp = s - hi;
        lo += (hi - (s - bp)) + (x - bp);
        hi = s;
      }
      sh.llt[b][e - 2 * MM] = (double)hi + (double)lo;
    }
  }
}

// The generalised eigenproblem of (St1, St2) of one iteration (Algorithm 1, step 8) on one
// warp, in the precision of mode GM: Q, Sigma, log|det Q|^2 pieces into
// slot b. Returns a warp-uniform device status code and records a failure.
template <int M, int GM, typename Sh>
__device__ int fast_solve(Sh& sh, FastWork<M, GM>& w, const FastEmArgs& a, int b, int lane) {
  using ST2 = typename GevdTypes<GM>::Solve;
  constexpr int MM = M * M;
  ST2 ldL = ST2(0);
  int rc;
  if constexpr (GM == 2) {
    // Newton-type iteration from the identity (the basis P already diagonalises the
    // previous iteration's parameters, so the new Grams are nearly diagonal in it): FP32
    // steps until the correction is below 1e-3 (the basis then has residuals of order 1e-6,
    // which the compensated refinement step squares), then the refinement against the
    // merged Grams' pairs. A poor start (a first correction above 0.1, or steps that do not
    // converge quadratically) takes the FP32 Cholesky + Jacobi solver instead, whose basis
    // is then refined the same way.
    rc = kOk;
    float em = warp_newton_step<M, float>(w.la.A, w.la.L, w.la.V, w.la.Z, w.la.A2, w.rf.lam32, true, lane);
    bool newton = em <= 0.1f;
    for (int k = 0; newton && em > 1e-3f && k < 4; ++k) {
      const float en = warp_newton_step<M, float>(w.la.A, w.la.L, w.la.V, w.la.Z, w.la.A2, w.rf.lam32,
                                                  false, lane);
      newton = en <= 0.5f * em;
      em = en;
    }
    const RefineOut out{sh.Qh[b], sh.Ql[b], sh.sigh[b], sh.sigl[b]};
    if (newton) {
      warp_refine_gevd<M>(w.rf, w.la.V, w.la.Z, w.la.A2, w.la.V2, w.la.A, w.la.L, out, lane);  // A, L free now
    } else {
      if constexpr (M <= 4) {
        rc = warp_gevd_reg<M, float>(w.la.A, w.la.L, w.rf.sig0, w.rf.X0, sh.U[b], &ldL,
                                     Prec<float>::kTol, a.max_sweeps, lane);
      } else {
        rc = warp_gevd_fast<M, float>(w.la, lane, w.rf.sig0, w.rf.X0, sh.U[b], &ldL, a.max_sweeps);
      }
      if (rc == kOk) warp_refine_gevd<M>(w.rf, w.rf.X0, w.la.Z, w.la.A2, w.la.V2, w.la.V, w.la.L, out, lane);
    }
    if (rc == kOk) {
      if (lane < M) {
        const float l = sh.sigh[b][lane];
        if (!(l > 0.f) || !(l < Prec<float>::kHuge)) rc = kErrNotPD;
      }
      rc = __reduce_max_sync(0xffffffffu, rc);  // warp-uniform
    }
  } else {
    if constexpr (M <= 4) {
      rc = warp_gevd_reg<M, ST2>(w.la.A, w.la.L, sh.sig[b], sh.Q[b], sh.U[b], &ldL,
                                 Prec<ST2>::kTol, a.max_sweeps, lane);
    } else {
      rc = warp_gevd_fast<M, ST2>(w.la, lane, sh.sig[b], sh.Q[b], sh.U[b], &ldL, a.max_sweeps);
    }
    if (lane == 0) sh.ldL[b] = ldL;
    if constexpr (GM == 1) {
      for (int e = lane; e < MM; e += 32) split2(sh.Q[b][e / M][e % M], sh.Qh[b][e / M][e % M], sh.Ql[b][e / M][e % M]);
      __syncwarp();
    }
  }
  if (rc != kOk && lane == 0) {
    set_status(a.status, rc);
    sh.fail = rc;
  }
  return rc;
}

// Publish the next basis for the bin pass: P^H <- (P Q)^H and Lambda <- Sigma. FP32
// eigensolver: from the FP32 copies. FP64 modes: P Q is needed to FP32 accuracy in every entry,
// which an FP32 product of the rounded factors does not give for an ill-conditioned P (its small
// columns come from cancellation), so it is a compensated dot product (Dot2) of the split pairs
// P = P32 + P32lo and Q = Qh + Ql on the FP32 pipe (for M <= 4 the lanes of a pair split each
// sum). After the deferred basis update of the previous iteration. One warp.
template <int M, int GM, typename Sh>
__device__ void fast_publish(Sh& sh, int b, float gi, int lane) {
  constexpr int MM = M * M;
  if constexpr (GM != 0) {
    constexpr bool kSplit = MM <= 16;
    constexpr int kPer = kSplit ? 1 : (MM + 31) / 32;
    constexpr int kStride = kSplit ? 2 : 1;
    const int h = kSplit ? (lane & 1) : 0;
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
      const int e = kSplit ? (lane >> 1) : lane + 32 * t;
      const int i = (e < MM) ? e / M : 0, m = (e < MM) ? e % M : 0;  // (P Q)_{m i}
      CDot2 acc;
      if (e < MM) {
#pragma unroll
        for (int kk = 0; kk < (M + kStride - 1) / kStride; ++kk) {
          const int k = kk * kStride + h;
          if (k < M) {
            const float2 ph = sh.P32[m][k], pl = sh.P32lo[m][k], qh = sh.Qh[b][k][i];
            acc.fma2(ph, qh, sh.Ql[b][k][i]);
            acc.re.c = fmaf(pl.x, qh.x, fmaf(-pl.y, qh.y, acc.re.c));
            acc.im.c = fmaf(pl.x, qh.y, fmaf(pl.y, qh.x, acc.im.c));
          }
        }
      }
      if constexpr (kSplit) acc.shfl_merge(1);
      if (e < MM && h == 0) {
        const double2 v = acc.value();
        sh.PH[i][m] = make_float2((float)v.x * gi, -(float)v.y * gi);
      }
    }
  } else {
    for (int e = lane; e < MM; e += 32) {
      const int i = e / M, m = e % M;  // (P Q)_{m i}
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < M; ++k) s = cfma(sh.P32[m][k], sh.Q[b][k][i], s);
      sh.PH[i][m] = make_float2(s.x * gi, -s.y * gi);
    }
  }
  if (lane < M) {
    const float sg = (GM == 2) ? sh.sigh[b][lane] + sh.sigl[b][lane] : (float)sh.sig[b][lane];
    sh.lam[lane] = sg;
    sh.ilam[lane] = 1.f / sg;
  }
}

// Write one bin's parameters (and its staged source powers) back to global memory.
template <int M, int ST, typename Sh>
__device__ void fast_write_back(Sh& sh, const FastEmArgs& a, int f, const BinIO<ST>& io, bool res,
                                int t, int nthr) {
  constexpr int MM = M * M;
  if (t < MM) a.P[(size_t)f * MM + t] = sh.P[t / M][t % M];
  if (t < M) a.lam[(size_t)f * M + t] = sh.lam64[t];
  if (t == 0) a.logdetS2[f] = sh.logdetS2;
  if (res) {
    for (int n = t; n < io.N; n += nthr) {
      io.vg1[n] = io.v1[n];
      io.vg1[io.dv2 + n] = io.v2[n];
    }
  }
}

// Where bin `slot` of this launch lives: its parameter index f, frames N and element offsets.
template <int M, bool kB>
__device__ __forceinline__ void fast_bin_locate(const FastEmArgs& a, int slot, int* f, int* N,
                                                size_t* yoff, size_t* v1off, size_t* v2off) {
  if constexpr (kB) {
    const BinDesc d = a.bins[slot];
    *f = d.b;
    *N = d.N;
    *yoff = (size_t)d.y_off;
    *v1off = (size_t)d.v1_off;
    *v2off = (size_t)d.v2_off;
  } else {
    *f = slot;
    *N = a.N;
    *yoff = (size_t)slot * a.N * M;
    *v1off = (size_t)slot * a.N;
    *v2off = (size_t)a.F * a.N + *v1off;
  }
}

// kB: the CTA's bin comes from the descriptor table a.bins (a batch); otherwise bin
// f = blockIdx.x of one mixture with the [F][N][M] / [2][F][N] layouts and v_in == v.
// GM: precision mode of the per-bin eigensolver and of the cross-warp Gram merge (GevdTypes);
// the bin pass is FP32 and the basis, log-likelihood and log-determinant bookkeeping FP64 in
// every mode. One bin per CTA; per iteration: pass (all warps) -> merge -> eigensolver on one
// warp while two others do the previous iteration's bookkeeping -> publish.
template <int M, int ST, int NT, bool kB, int GM = 0>
__global__ void __launch_bounds__(NT, fast_min_blocks(M, NT)) fast_em_kernel(const FastEmArgs a) {
  using E = typename Elem<ST>::T;
  constexpr int NW = NT / 32;
  static_assert(NW >= 2, "the deferred bookkeeping runs on warp 1");
  static_assert(GM != 2 || NW >= 3, "the refined mode computes log det St2 on a third warp");
  using Sh = FastShared<M, NW, GM>;
  __shared__ Sh sh;
  extern __shared__ __align__(16) unsigned char dyn[];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int f, N;
  size_t yoff, v1off, v2off;
  fast_bin_locate<M, kB>(a, blockIdx.x, &f, &N, &yoff, &v1off, &v2off);
  const E* yg = reinterpret_cast<const E*>(a.y) + yoff;
  // The initial and previous source powers sit at the same offsets in their own arrays; the
  // distances between the arrays are kernel parameters (no registers held in the hot loop).
  const ptrdiff_t d_in = kB ? a.v_in - a.v : 0;
  E* ys = reinterpret_cast<E*>(dyn);
  const size_t ybytes = ((size_t)N * M * sizeof(E) + 15) & ~(size_t)15;
  float* vs = reinterpret_cast<float*>(dyn + ybytes);
  // One mixture: the launch reserves exactly its bins' need, or nothing.
  const bool res = kB ? em_bin_smem(M, ST, N) <= (size_t)a.res_bytes : a.res_bytes != 0;
  BinIO<ST> io;
  io.vg1 = a.v + v1off;
  io.dv2 = (int)(v2off - v1off);
  io.d_prev = a.v_prev - a.v;
  io.y = res ? ys : yg;
  io.v1 = res ? vs : io.vg1;
  io.v2 = res ? vs + N : io.vg1 + io.dv2;
  io.N = N;
  io.vf = a.vfloor[f];
  io.gi = (ST == 1) ? a.ginv[f] : 1.f;
  const double invN = 1.0 / (double)N;

  fast_load_params<M>(sh, a, f, tid);
  if (tid == 0) {
    unsigned wslot;
    asm volatile("mov.u32 %0, %%warpid;" : "=r"(wslot));
    sh.wid0 = (int)wslot;
  }
  fast_stage<M, ST, kB>(yg, ys, vs, io.vg1, io.dv2, d_in, N, res, tid, NT);
  __syncthreads();
  fast_first_basis<M>(sh, a, f, io.gi, tid);
  __syncthreads();

  int done = 0;  // iterations whose bin pass and eigensolve completed
  for (int it = 0; it < a.iters; ++it) {
    const int b = it & 1;
    fast_pass<M, ST>(sh, io, tid, NT, it == a.iters - 1, sh.red[warp], lane);
    __syncthreads();
    fast_merge<M, NW, GM>(sh, sh.w, b, invN, tid, NT);
    __syncthreads();
    const int ws = solver_warp<NW>(it, sh.wid0);  // eigensolver; then basis, log-likelihood
    const int wb = (ws + 1) % NW, wl = (ws + 2) % NW;
    if (warp == ws) {
      fast_solve<M, GM>(sh, sh.w, a, b, lane);
    } else if (warp == wb && it > 0) {
      fast_deferred_basis<M, GM>(sh, a, f, it - 1, lane);
      if constexpr (NW < 3) fast_deferred_ll<M, GM>(sh, a, f, N, it - 1, lane);
    } else if (NW >= 3 && warp == wl) {
      fast_logdet<M, GM>(sh, sh.w, it, lane);
      if (it > 0) fast_deferred_ll<M, GM>(sh, a, f, N, it - 1, lane);
    }
    if (warp == ws || warp == wb) asm volatile("bar.sync 1, 64;" ::: "memory");
    if (warp == ws && !sh.fail) fast_publish<M, GM>(sh, b, io.gi, lane);
    __syncthreads();
    if (sh.fail || sh.fail_pending) break;
    done = it + 1;
  }
  if (done > 0 && done == a.iters) {
    if (warp == 1) {
      fast_deferred_basis<M, GM>(sh, a, f, done - 1, lane);
      if constexpr (NW < 3) fast_deferred_ll<M, GM>(sh, a, f, N, done - 1, lane);
    } else if (NW >= 3 && warp == 2) {
      fast_deferred_ll<M, GM>(sh, a, f, N, done - 1, lane);
    }
  }
  __syncthreads();
  fast_write_back<M, ST>(sh, a, f, io, res, tid, NT);
}

// Posterior means in the original basis (Algorithm 1, last step): mu1 = P^-H (a .* yt),
// a_i = v1 lam_i / (v1 lam_i + v2); mu2 = y - mu1 (y = x1 + x2, Sec. 2).
template <int M, int ST>
__global__ void __launch_bounds__(256) sep_fast_kernel(const SepFastArgs a) {
  using E = typename Elem<ST>::T;
  __shared__ float2 PH[M][M], PiH[M][M];
  __shared__ float lam[M];
  const int tid = threadIdx.x;
  int f, N;
  size_t yoff, xoff, v1off, v2off;
  if (a.bins) {
    const BinDesc d = a.bins[blockIdx.x];
    f = d.b;
    N = d.N;
    yoff = (size_t)d.y_off;
    xoff = (size_t)d.x_off;
    v1off = (size_t)d.v1_off;
    v2off = (size_t)d.v2_off;
  } else {
    f = blockIdx.x;
    N = a.N;
    yoff = (size_t)f * N * M;
    xoff = yoff;
    v1off = (size_t)f * N;
    v2off = (size_t)a.F * N + v1off;
  }
  const int n = blockIdx.y * 256 + tid;
  if (blockIdx.y * 256 >= N) return;  // whole CTA past this bin's frames
  // The point's mixture and variances do not come from the kernel launched just before this
  // one (the separation constants): read them first, then wait for that kernel's results
  // (programmatic dependent launch; a plain launch order makes the wait return at once).
  float2 yv[M];
  float v1 = 0.f, v2 = 0.f;
  if (n < N) {
    load_bin<M, ST>(reinterpret_cast<const E*>(a.y) + yoff + (size_t)n * M, yv);
    v1 = a.v[v1off + n];
    v2 = a.v[v2off + n];
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const size_t MM = (size_t)M * M;
  if (tid < M * M) {
    PH[tid / M][tid % M] = a.PH[f * MM + tid];
    PiH[tid / M][tid % M] = a.PinvH[f * MM + tid];
  }
  if (tid < M) lam[tid] = a.lam[(size_t)f * M + tid];
  __syncthreads();
  if (n >= N) return;
  const size_t b = xoff + (size_t)n * M;
  const float gi = (ST == 1) ? a.ginv[f] : 1.f;
  float2 mt[M];
#pragma unroll
  for (int i = 0; i < M; ++i) {
    float2 s = cmul(PH[i][0], yv[0]);
#pragma unroll
    for (int m = 1; m < M; ++m) s = cfma(PH[i][m], yv[m], s);
    const float e = v1 * lam[i];
    mt[i] = cscale(s, e / (e + v2));
  }
  float2 o1[M], o2[M];
#pragma unroll
  for (int i = 0; i < M; ++i) {
    float2 s = cmul(PiH[i][0], mt[0]);
#pragma unroll
    for (int m = 1; m < M; ++m) s = cfma(PiH[i][m], mt[m], s);
    o1[i] = s;
    o2[i] = csub(cscale(yv[i], gi), s);
  }
  float4* q1 = reinterpret_cast<float4*>(a.x1 + b);
  float4* q2 = reinterpret_cast<float4*>(a.x2 + b);
  if ((M & 1) == 0 && ((reinterpret_cast<uintptr_t>(q1) | reinterpret_cast<uintptr_t>(q2)) & 15) == 0) {
    // 16-byte stores of complex pairs
#pragma unroll
    for (int i = 0; i < M / 2; ++i) {
      q1[i] = make_float4(o1[2 * i].x, o1[2 * i].y, o1[2 * i + 1].x, o1[2 * i + 1].y);
      q2[i] = make_float4(o2[2 * i].x, o2[2 * i].y, o2[2 * i + 1].x, o2[2 * i + 1].y);
    }
  } else {
#pragma unroll
    for (int i = 0; i < M; ++i) {
      a.x1[b + i] = o1[i];
      a.x2[b + i] = o2[i];
    }
  }
}


// Host-side launch of fast_em_kernel<M, ST, NT> (instantiated per translation unit).
template <int M, int ST, int NT, bool kB, int GM = 0>
cudaError_t launch_fast_t(const FastEmArgs& a, cudaStream_t st) {
  const size_t dyn = (size_t)a.res_bytes;
  auto k = fast_em_kernel<M, ST, NT, kB, GM>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  if (dyn > 0) {  // the default limit (48 KB) covers static and dynamic shared memory together
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  const int grid = a.bins ? a.nbins : a.F;
  if (grid <= 0) return cudaSuccess;
  k<<<grid, NT, dyn, st>>>(a);
  return cudaGetLastError();
}

template <int ST, int NT, bool kB, int GM = 0>
cudaError_t launch_fast_nt(int M, const FastEmArgs& a, cudaStream_t st) {
  switch (M) {
    case 1: return launch_fast_t<1, ST, NT, kB, GM>(a, st);
    case 2: return launch_fast_t<2, ST, NT, kB, GM>(a, st);
    case 3: return launch_fast_t<3, ST, NT, kB, GM>(a, st);
    case 4: return launch_fast_t<4, ST, NT, kB, GM>(a, st);
    case 5: return launch_fast_t<5, ST, NT, kB, GM>(a, st);
    case 6: return launch_fast_t<6, ST, NT, kB, GM>(a, st);
    case 7: return launch_fast_t<7, ST, NT, kB, GM>(a, st);
    case 8: return launch_fast_t<8, ST, NT, kB, GM>(a, st);
  }
  return cudaErrorInvalidValue;
}

// Defined in fca_fast_tuned.cu: batches (descriptor tables), complex64 storage, 64, 128 or
// 256 threads per CTA; in fca_fast_tuned_refined.cu the same in the refined mode (128 or 256).
cudaError_t launch_fast_batch_c64(int M, const FastEmArgs& a, cudaStream_t st, int threads);
cudaError_t launch_fast_batch_c64_refined(int M, const FastEmArgs& a, cudaStream_t st, int threads);
// Defined in fca_fast64.cu (mode 1) and fca_fast_refined.cu (mode 2): one mixture, 128 threads
// per CTA.
cudaError_t launch_fast_single_g64(int M, int storage, const FastEmArgs& a, cudaStream_t st);
cudaError_t launch_fast_single_refined(int M, int storage, const FastEmArgs& a, cudaStream_t st);

}  // namespace fca
