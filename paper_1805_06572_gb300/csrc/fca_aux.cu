// Per-frequency parameter kernels and small helpers (sm_103a).
//
//   gevd_from_S : (S1, S2) -> (P, Lambda, log det S2), the generalised eigenproblem of
//                 Eq. (GEVD) (Algorithm 1, step 1, and the switch from the conventional
//                 parameters to the FastFCA ones);
//   S_from_P    : S2 = P^-H P^-1, S1 = P^-H Lambda P^-1 (Eqs. (Sdiag), (recoverS));
//   sep_prep    : FP32 P^H, P^-H and Lambda for the posterior-mean kernel;
//   prepare     : positivity floor of v per frequency, initial v (clamped), and a check that
//                 the mixture and the initial v are finite;
//   ll_reduce   : per-iteration log-likelihood summed over frequencies in a fixed order.
// One warp handles one frequency bin; P^-1 is formed by Gauss-Jordan elimination with
// partial pivoting in FP64 (these kernels run once per call, not once per iteration).
#include <type_traits>

#include "fca_dev.cuh"
#include "fca_internal.h"

namespace fca {

constexpr int kWarpsPerCta = 4;

// In-place inverse of the M x M matrix in aug[.][0..M) (aug[.][M..2M) must hold I); the
// inverse ends in aug[.][M..2M). Returns false (uniformly) if a pivot is zero.
template <int M>
__device__ bool warp_inverse64(double2 (*aug)[2 * kMaxM], int lane) {
  constexpr int W = 2 * M;
  constexpr int kPer = (M * W + 31) / 32;
  for (int k = 0; k < M; ++k) {
    double mag = (lane >= k && lane < M) ? aug[lane][k].x * aug[lane][k].x + aug[lane][k].y * aug[lane][k].y : -1.0;
    int idx = lane;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      const double om = __shfl_xor_sync(0xffffffffu, mag, o);
      const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (om > mag || (om == mag && oi < idx)) {
        mag = om;
        idx = oi;
      }
    }
    if (!(mag > 0.0) || !isfinite(mag)) return false;
    const int piv = idx;
    __syncwarp();
    if (piv != k) {
      for (int j = lane; j < W; j += 32) {
        const double2 t = aug[k][j];
        aug[k][j] = aug[piv][j];
        aug[piv][j] = t;
      }
    }
    __syncwarp();
    const double2 p = aug[k][k];
    const double dd = p.x * p.x + p.y * p.y;
    const double rd = recip64(dd);
    const double2 inv = make_double2(p.x * rd, -p.y * rd);
    __syncwarp();
    for (int j = lane; j < W; j += 32) aug[k][j] = zmul(aug[k][j], inv);
    __syncwarp();
    double2 nv[kPer];
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
      const int e = lane + 32 * t;
      if (e < M * W) {
        const int i = e / W, j = e % W;
        const double2 fac = aug[i][k];
        nv[t] = (i == k) ? aug[i][j] : zadd(aug[i][j], zmul(make_double2(-fac.x, -fac.y), aug[k][j]));
      }
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
      const int e = lane + 32 * t;
      if (e < M * W) aug[e / W][e % W] = nv[t];
    }
    __syncwarp();
  }
  return true;
}

// FP64 input as the solver's complex type.
template <typename G> __device__ __forceinline__ Cx<G> from_z(double2 a);
template <> __device__ __forceinline__ float2 from_z<float>(double2 a) { return z2c(a); }
template <> __device__ __forceinline__ double2 from_z<double>(double2 a) { return a; }

// One warp: (P, Lambda, log det S2) of bin f from (S1, S2) (Eq. (GEVD)), by the solver the
// EM kernel runs every iteration (register-resident for M <= 4, shared-memory otherwise) in
// precision G; P = Q, log det S2 = -log|det Q|^2. The bin's S is also copied to S_copy when
// that is set. A failure leaves the bin's outputs unwritten and records its status.
template <int M, typename G>
__device__ void gevd_bin(const double2* S, double2* S_copy, int F, int f, double2* P, double* lam,
                         double* logdetS2, int* status, WarpLAT<G>& la, G* sig,
                         Cx<G> (*Q)[kMaxM], Cx<G> (*U)[kMaxM], int max_sweeps, int lane) {
  const size_t MM = (size_t)M * M;
  for (int e = lane; e < M * M; e += 32) {
    const double2 s1 = S[(size_t)f * MM + e], s2 = S[((size_t)F + f) * MM + e];
    if (S_copy) {
      S_copy[(size_t)f * MM + e] = s1;
      S_copy[((size_t)F + f) * MM + e] = s2;
    }
    la.A[e / M][e % M] = from_z<G>(s1);
    la.L[e / M][e % M] = from_z<G>(s2);
  }
  __syncwarp();
  G ldL = G(0);
  int rc;
  if constexpr (M <= 4) {
    rc = warp_gevd_reg<M, G>(la.A, la.L, sig, Q, U, &ldL, Prec<G>::kTol, max_sweeps, lane);
  } else {
    rc = warp_gevd_fast<M, G>(la, lane, sig, Q, U, &ldL, max_sweeps);
  }
  __syncwarp();
  if (rc != kOk) {
    if (lane == 0) set_status(status, rc);
    return;
  }
  const double ldQ = (double)ldL + unitarity_defect<M>(U, lane);
  for (int e = lane; e < M * M; e += 32) P[(size_t)f * MM + e] = c2z(Q[e / M][e % M]);
  if (lane < M) lam[(size_t)f * M + lane] = (double)sig[lane];
  if (lane == 0) logdetS2[f] = -ldQ;  // P = Q: log det S2 = -log|det P|^2
}

// Workspace of gevd_bin_refined (one warp).
template <int M>
struct RefinedGevdWork {
  RefineWork<M> rf;
  WarpLAT<float, M> la;
  float2 Xh[M][kMaxM], Xl[M][kMaxM];
  float2 U[M][kMaxM];
  float lh[kMaxM], ll[kMaxM];
};

// One warp, refined precision (FCA_GEVD_REFINED): the same outputs as gevd_bin from the FP32
// solver on (S1, S2) rounded to FP32, refined against the FP64 pair (warp_refine_gevd: one
// compensated FP32 step, a second FP64 step after a poor start); P = Xh + Xl, Lambda = lh + ll,
// and log det S2 from an FP64 Cholesky factorisation of S2 (P^H S2 P = I).
template <int M>
__device__ void gevd_bin_refined(const double2* S, double2* S_copy, int F, int f, double2* P, double* lam,
                                 double* logdetS2, int* status, RefinedGevdWork<M>& w, int max_sweeps,
                                 int lane) {
  const size_t MM = (size_t)M * M;
  for (int e = lane; e < M * M; e += 32) {
    const int i = e / M, k = e % M;
    const double2 s1 = S[(size_t)f * MM + e], s2 = S[((size_t)F + f) * MM + e];
    if (S_copy) {
      S_copy[(size_t)f * MM + e] = s1;
      S_copy[((size_t)F + f) * MM + e] = s2;
    }
    w.rf.A[i][k] = s1;
    w.rf.B[i][k] = s2;
    split2(s1, w.rf.Ah[i][k], w.rf.Al[i][k]);
    split2(s2, w.rf.Bh[i][k], w.rf.Bl[i][k]);
    w.la.A[i][k] = w.rf.Ah[i][k];
    w.la.L[i][k] = w.rf.Bh[i][k];
  }
  __syncwarp();
  float ldL = 0.f;
  int rc;
  if constexpr (M <= 4) {
    rc = warp_gevd_reg<M, float>(w.la.A, w.la.L, w.rf.sig0, w.rf.X0, w.U, &ldL, Prec<float>::kTol,
                                 max_sweeps, lane);
  } else {
    rc = warp_gevd_fast<M, float>(w.la, lane, w.rf.sig0, w.rf.X0, w.U, &ldL, max_sweeps);
  }
  __syncwarp();
  if (rc == kOk) {
    const RefineOut out{w.Xh, w.Xl, w.lh, w.ll};
    warp_refine_gevd<M>(w.rf, w.rf.X0, w.la.Z, w.la.A2, w.la.V2, w.la.V, w.la.L, out, lane);
    if (lane < M) {
      const float l = w.lh[lane];
      if (!(l > 0.f) || !(l < Prec<float>::kHuge)) rc = kErrNotPD;
    }
    rc = __reduce_max_sync(0xffffffffu, rc);
  }
  if (rc != kOk) {
    if (lane == 0) set_status(status, rc);
    return;
  }
  for (int e = lane; e < M * M; e += 32) {
    const float2 hi = w.Xh[e / M][e % M], lo = w.Xl[e / M][e % M];
    P[(size_t)f * MM + e] = make_double2((double)hi.x + (double)lo.x, (double)hi.y + (double)lo.y);
  }
  if (lane < M) lam[(size_t)f * M + lane] = (double)w.lh[lane] + (double)w.ll[lane];
  if (lane == 0) {  // log det S2 = sum_k log L_kk^2, S2 = L L^H (FP64, in place in rf.B)
    double ld = 0.0;
    bool ok = true;
    for (int k = 0; k < M; ++k) {
      double d = w.rf.B[k][k].x;
      for (int m = 0; m < k; ++m) d -= w.rf.B[k][m].x * w.rf.B[k][m].x + w.rf.B[k][m].y * w.rf.B[k][m].y;
      ok = ok && d > 0.0;
      const double ik = 1.0 / sqrt(d);
      ld += log(d);
      for (int i = k + 1; i < M; ++i) {
        double2 s = w.rf.B[i][k];
        for (int m = 0; m < k; ++m) s = csub(s, cmulc(w.rf.B[i][m], w.rf.B[k][m]));
        w.rf.B[i][k] = make_double2(s.x * ik, s.y * ik);
      }
    }
    if (ok) logdetS2[f] = ld;
    else set_status(status, kErrNotPD);
  }
}

constexpr int kRefinedWarps = 2;  // bins per CTA of gevd_from_S_refined_kernel (shared workspace)

template <int M>
__global__ void __launch_bounds__(32 * kRefinedWarps) gevd_from_S_refined_kernel(const ParamArgs a) {
  __shared__ RefinedGevdWork<M> w[kRefinedWarps];
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int f = blockIdx.x * kRefinedWarps + wi;
  if (f >= a.F) return;  // whole warp leaves together
  gevd_bin_refined<M>(a.S, nullptr, a.F, f, a.P, a.lam, a.logdetS2, a.status, w[wi], a.max_sweeps, lane);
}

template <int M, typename G>
__global__ void __launch_bounds__(32 * kWarpsPerCta) gevd_from_S_kernel(const ParamArgs a) {
  __shared__ WarpLAT<G> la[kWarpsPerCta];
  __shared__ G sig[kWarpsPerCta][kMaxM];
  __shared__ Cx<G> Q[kWarpsPerCta][kMaxM][kMaxM], U[kWarpsPerCta][kMaxM][kMaxM];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int f = blockIdx.x * kWarpsPerCta + w;
  if (f >= a.F) return;  // whole warp leaves together
  gevd_bin<M, G>(a.S, nullptr, a.F, f, a.P, a.lam, a.logdetS2, a.status, la[w], sig[w], Q[w], U[w],
                 a.max_sweeps, lane);
}

// mode 0: S_out = (P^-H Lam P^-1, P^-H P^-1); mode 1: separation prep.
template <int M, int MODE>
__global__ void __launch_bounds__(32 * kWarpsPerCta) from_P_kernel(const ParamArgs a) {
  __shared__ double2 aug[kWarpsPerCta][kMaxM][2 * kMaxM];
  // The separation kernel that follows may start now: it waits for this grid's results.
  if (MODE == 1) asm volatile("griddepcontrol.launch_dependents;");
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int f = blockIdx.x * kWarpsPerCta + w;
  if (f >= a.F) return;
  const size_t MM = (size_t)M * M;
  double2(*A)[2 * kMaxM] = aug[w];
  for (int e = lane; e < M * 2 * M; e += 32) {
    const int i = e / (2 * M), j = e % (2 * M);
    A[i][j] = (j < M) ? a.P[(size_t)f * MM + i * M + j] : make_double2(j - M == i ? 1.0 : 0.0, 0.0);
  }
  __syncwarp();
  if (!warp_inverse64<M>(A, lane)) {
    if (lane == 0) set_status(a.status, kErrNonFinite);
    return;
  }
  // Pinv = A[.][M..2M)
  if (MODE == 0) {
    for (int e = lane; e < 2 * M * M; e += 32) {
      const int j = e / (M * M), r = e % (M * M), i = r / M, k = r % M;
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int m = 0; m < M; ++m) {  // (P^-H T_j P^-1)_ik = sum_m conj(Pinv_mi) t_m Pinv_mk
        const double2 pmi = zconj(A[m][M + i]);
        const double t = (j == 0) ? a.lam[(size_t)f * M + m] : 1.0;
        const double2 pmk = A[m][M + k];
        s = zfma(make_double2(pmi.x * t, pmi.y * t), pmk, s);
      }
      a.S_out[((size_t)j * a.F + f) * MM + r] = s;
    }
  } else {
    const float gi = a.ginv ? a.ginv[f] : 1.f;
    for (int e = lane; e < M * M; e += 32) {
      const int i = e / M, m = e % M;
      const double2 p = a.P[(size_t)f * MM + m * M + i];  // (P^H)_im = conj(P_mi)
      a.PH[(size_t)f * MM + e] = make_float2((float)p.x * gi, -(float)p.y * gi);
      const double2 q = A[m][M + i];                      // (P^-H)_im = conj(Pinv_mi)
      a.PinvH[(size_t)f * MM + e] = make_float2((float)q.x, -(float)q.y);
    }
    if (lane < M) a.lam32[(size_t)f * M + lane] = (float)a.lam[(size_t)f * M + lane];
  }
}

// Sum of |y|^2 over the bin's N M values, taken by the 224 threads of warps 1..7 in one
// fixed order whatever the path: value pairs (2i, 2i+1) go to thread i mod 224, which keeps
// four partial sums and adds them at the end. VEC: 16-byte loads (and copies), when both
// addresses allow them; else element by element, same order. Also copies the values to yc;
// the loads of a group come before its stores (the compiler may not assume yf and yc
// disjoint).
template <int ST, bool VEC>
__device__ float bin_power_impl(const typename Elem<ST>::T* yf, typename Elem<ST>::T* yc, int total, int t) {
  using E = typename Elem<ST>::T;
  using P = typename std::conditional<VEC, float4, E[2]>::type;
  constexpr int nt = 224;
  const int n4 = total / 2;
  auto load = [&](int i, P& p) {
    if constexpr (VEC) {
      p = reinterpret_cast<const float4*>(yf)[i];
    } else {
      p[0] = yf[2 * i];
      p[1] = yf[2 * i + 1];
    }
  };
  auto store = [&](int i, const P& p) {
    if (!yc) return;
    if constexpr (VEC) {
      reinterpret_cast<float4*>(yc)[i] = p;
    } else {
      yc[2 * i] = p[0];
      yc[2 * i + 1] = p[1];
    }
  };
  auto acc = [](const P& p, float s) {
    float4 a;
    if constexpr (VEC) {
      a = p;
    } else {
      const float2 u = decode(p[0]), w = decode(p[1]);
      a = make_float4(u.x, u.y, w.x, w.y);
    }
    return fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, fmaf(a.w, a.w, s))));
  };
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  int i = t;
  for (; i + 7 * nt < n4; i += 8 * nt) {  // eight loads in flight
    P q[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) load(i + k * nt, q[k]);
#pragma unroll
    for (int k = 0; k < 8; ++k) store(i + k * nt, q[k]);
    s0 = acc(q[4], acc(q[0], s0));
    s1 = acc(q[5], acc(q[1], s1));
    s2 = acc(q[6], acc(q[2], s2));
    s3 = acc(q[7], acc(q[3], s3));
  }
  for (; i + 3 * nt < n4; i += 4 * nt) {
    P q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) load(i + k * nt, q[k]);
#pragma unroll
    for (int k = 0; k < 4; ++k) store(i + k * nt, q[k]);
    s0 = acc(q[0], s0);
    s1 = acc(q[1], s1);
    s2 = acc(q[2], s2);
    s3 = acc(q[3], s3);
  }
  for (; i < n4; i += nt) {
    P p;
    load(i, p);
    store(i, p);
    s0 = acc(p, s0);
  }
  float s = s0 + ((s1 + s2) + s3);
  if ((total & 1) && t == 0) {
    const E e = yf[total - 1];
    if (yc) yc[total - 1] = e;
    s += cabs2(decode(e));
  }
  return s;
}

template <int ST>
__device__ float bin_power(const typename Elem<ST>::T* yf, typename Elem<ST>::T* yc, int total, int t) {
  const bool vec = ST == 0 && ((reinterpret_cast<uintptr_t>(yf) | reinterpret_cast<uintptr_t>(yc)) & 15) == 0;
  return vec ? bin_power_impl<ST, true>(yf, yc, total, t) : bin_power_impl<ST, false>(yf, yc, total, t);
}

// One CTA (256 threads) per frequency bin: the positivity floor of v from the bin's mixture
// power, the initial v clamped to it, and checks that both are finite, all on warps 1..7
// (synchronised among themselves by named barrier 1). Warp 0 meanwhile solves the bin's
// generalised eigenproblem when extra.S is set (PrepareExtra).
template <int M, int ST, bool kX, typename G = float, bool kRefined = false>
__global__ void __launch_bounds__(256) prepare_kernel(int F, int N0, const void* y, const float* ginv,
                                                      const double* v0, float* v, float* vfloor,
                                                      int* status, const BinDesc* bins,
                                                      const PrepareExtra ex) {
  using E = typename Elem<ST>::T;
  constexpr int kStreamThreads = 224;
  struct PlainWork {
    WarpLAT<G> la;
    G sig[kMaxM];
    Cx<G> Qs[kMaxM][kMaxM], Us[kMaxM][kMaxM];
  };
  struct NoWork {};
  __shared__ double part[8];
  __shared__ float vf_s;
  // the eigensolver's workspace, used only by the kX variants
  __shared__ typename std::conditional<kX, typename std::conditional<kRefined, RefinedGevdWork<M>, PlainWork>::type,
                                       NoWork>::type gw;
  const int tid = threadIdx.x;
  int f, N;
  size_t yoff, voff[2];
  if (bins) {
    const BinDesc d = bins[blockIdx.x];
    f = d.b;
    N = d.N;
    yoff = (size_t)d.y_off;
    voff[0] = (size_t)d.v1_off;
    voff[1] = (size_t)d.v2_off;
  } else {
    f = blockIdx.x;
    N = N0;
    yoff = (size_t)f * N * M;
    voff[0] = (size_t)f * N;
    voff[1] = (size_t)F * N + voff[0];
  }
  int bad = 0;
  if (tid < 32) {
    if constexpr (kX && kRefined) {
      if (ex.S) gevd_bin_refined<M>(ex.S, ex.S_copy, F, f, ex.P, ex.lam, ex.logdetS2, status, gw, ex.max_sweeps, tid);
    } else if constexpr (kX) {
      if (ex.S)
        gevd_bin<M, G>(ex.S, ex.S_copy, F, f, ex.P, ex.lam, ex.logdetS2, status, gw.la, gw.sig, gw.Qs, gw.Us,
                       ex.max_sweeps, tid);
    }
  } else {
    const int t = tid - 32;
    E* yc = (kX && ex.y_copy) ? reinterpret_cast<E*>(ex.y_copy) + yoff : nullptr;
    float s = bin_power<ST>(reinterpret_cast<const E*>(y) + yoff, yc, N * M, t);
    s = warp_sum(s);
    if ((tid & 31) == 0) part[tid >> 5] = (double)s;
    asm volatile("bar.sync 1, 224;" ::: "memory");
    if (t == 0) {
      double tot = 0.0;
      for (int w = 1; w < 8; ++w) tot += part[w];
      const double g = (ST == 1) ? (double)ginv[f] : 1.0;
      tot *= g * g;
      if (!isfinite(tot)) set_status(status, kErrNonFinite);  // a NaN or infinity in the mixture
      const double fl = fmax(1e-12 * tot / ((double)N * M), 1e-30);
      vf_s = (float)fl;
      vfloor[f] = (float)fl;
    }
    asm volatile("bar.sync 1, 224;" ::: "memory");
    const float vf = vf_s;
    // Both sources' values, four frames each, loaded before any store (v and v0 may not be
    // assumed disjoint by the compiler).
    for (int n0 = t; n0 < N; n0 += 4 * kStreamThreads) {
      double x[2][4];
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int n = n0 + k * kStreamThreads;
          x[j][k] = n < N ? v0[voff[j] + n] : 1.0;
        }
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int n = n0 + k * kStreamThreads;
          if (n < N) {
            bad |= !isfinite(x[j][k]);
            v[voff[j] + n] = fmaxf((float)x[j][k], vf);
          }
        }
    }
  }
  if (__syncthreads_or(bad) && tid == 0) set_status(status, kErrNonFinite);
}

__global__ void ll_reduce_kernel(int F, const double* llf, double* ll) {
  __shared__ double part[256];
  const int l = blockIdx.x, tid = threadIdx.x;
  double s = 0.0;
  for (int f = tid; f < F; f += 256) s += llf[(size_t)l * F + f];
  part[tid] = s;
  __syncthreads();
  for (int o = 128; o >= 1; o >>= 1) {
    if (tid < o) part[tid] += part[tid + o];
    __syncthreads();
  }
  if (tid == 0) ll[l] = part[0];
}

// One CTA per (iteration, mixture): the mixture's log-likelihood is the sum over its bins
// (Eq. (like) factorises over frequencies), in a fixed order.
__global__ void ll_ranges_kernel(int F, const double* llf, const int* b0, const int* nb,
                                 const int* mix_id, int iters, double* out) {
  __shared__ double part[128];
  const int k = blockIdx.x, l = blockIdx.y, tid = threadIdx.x;
  const int lo = b0[k], n = nb[k];
  double s = 0.0;
  for (int i = tid; i < n; i += 128) s += llf[(size_t)l * F + lo + i];
  part[tid] = s;
  __syncthreads();
  for (int o = 64; o >= 1; o >>= 1) {
    if (tid < o) part[tid] += part[tid + o];
    __syncthreads();
  }
  if (tid == 0) out[(size_t)mix_id[k] * iters + l] = part[0];
}

__global__ void invert_scale_kernel(int F, const float* g, float* ginv) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < F) ginv[f] = 1.0f / g[f];
}

// ------------------------------------------------------------------ host-side launchers
#define FCA_DISPATCH_M(M, CALL)          \
  switch (M) {                           \
    case 1: { constexpr int kM = 1; CALL; } \
    case 2: { constexpr int kM = 2; CALL; } \
    case 3: { constexpr int kM = 3; CALL; } \
    case 4: { constexpr int kM = 4; CALL; } \
    case 5: { constexpr int kM = 5; CALL; } \
    case 6: { constexpr int kM = 6; CALL; } \
    case 7: { constexpr int kM = 7; CALL; } \
    case 8: { constexpr int kM = 8; CALL; } \
  }                                      \
  return cudaErrorInvalidValue;

cudaError_t launch_gevd_from_S(int M, const ParamArgs& a, cudaStream_t st) {
  const int grid = (a.F + kWarpsPerCta - 1) / kWarpsPerCta;
  if (grid <= 0) return cudaSuccess;
  if (a.gevd_mode == 2) {
    const int gr = (a.F + kRefinedWarps - 1) / kRefinedWarps;
    FCA_DISPATCH_M(M, (gevd_from_S_refined_kernel<kM><<<gr, 32 * kRefinedWarps, 0, st>>>(a)); return cudaGetLastError())
  }
  if (a.gevd_mode) {
    FCA_DISPATCH_M(M, (gevd_from_S_kernel<kM, double><<<grid, 32 * kWarpsPerCta, 0, st>>>(a)); return cudaGetLastError())
  }
  FCA_DISPATCH_M(M, (gevd_from_S_kernel<kM, float><<<grid, 32 * kWarpsPerCta, 0, st>>>(a)); return cudaGetLastError())
}

cudaError_t launch_S_from_P(int M, const ParamArgs& a, cudaStream_t st) {
  const int grid = (a.F + kWarpsPerCta - 1) / kWarpsPerCta;
  if (grid <= 0) return cudaSuccess;
  FCA_DISPATCH_M(M, (from_P_kernel<kM, 0><<<grid, 32 * kWarpsPerCta, 0, st>>>(a)); return cudaGetLastError())
}

cudaError_t launch_sep_prep(int M, const ParamArgs& a, cudaStream_t st) {
  const int grid = (a.F + kWarpsPerCta - 1) / kWarpsPerCta;
  if (grid <= 0) return cudaSuccess;
  FCA_DISPATCH_M(M, (from_P_kernel<kM, 1><<<grid, 32 * kWarpsPerCta, 0, st>>>(a)); return cudaGetLastError())
}

cudaError_t launch_prepare(int M, int storage, int F, int N, const void* y, const float* ginv,
                           const double* v0, float* v, float* vfloor, int* status, cudaStream_t st,
                           const BinDesc* bins, const PrepareExtra* extra) {
  if (F <= 0) return cudaSuccess;
  if (extra && bins) return cudaErrorInvalidValue;  // the fused work assumes the [F][N][M] layout
  const PrepareExtra ex = extra ? *extra : PrepareExtra{};
  if (extra && ex.gevd_mode == 2) {
    if (storage) {
      FCA_DISPATCH_M(M, (prepare_kernel<kM, 1, true, float, true><<<F, 256, 0, st>>>(F, N, y, ginv, v0, v, vfloor, status, bins, ex)); return cudaGetLastError())
    } else {
      FCA_DISPATCH_M(M, (prepare_kernel<kM, 0, true, float, true><<<F, 256, 0, st>>>(F, N, y, ginv, v0, v, vfloor, status, bins, ex)); return cudaGetLastError())
    }
  }
  if (extra && ex.gevd_mode) {
    if (storage) {
      FCA_DISPATCH_M(M, (prepare_kernel<kM, 1, true, double><<<F, 256, 0, st>>>(F, N, y, ginv, v0, v, vfloor, status, bins, ex)); return cudaGetLastError())
    } else {
      FCA_DISPATCH_M(M, (prepare_kernel<kM, 0, true, double><<<F, 256, 0, st>>>(F, N, y, ginv, v0, v, vfloor, status, bins, ex)); return cudaGetLastError())
    }
  }
  if (extra) {
    if (storage) {
      FCA_DISPATCH_M(M, (prepare_kernel<kM, 1, true><<<F, 256, 0, st>>>(F, N, y, ginv, v0, v, vfloor, status, bins, ex)); return cudaGetLastError())
    } else {
      FCA_DISPATCH_M(M, (prepare_kernel<kM, 0, true><<<F, 256, 0, st>>>(F, N, y, ginv, v0, v, vfloor, status, bins, ex)); return cudaGetLastError())
    }
  }
  if (storage) {
    FCA_DISPATCH_M(M, (prepare_kernel<kM, 1, false><<<F, 256, 0, st>>>(F, N, y, ginv, v0, v, vfloor, status, bins, ex)); return cudaGetLastError())
  } else {
    FCA_DISPATCH_M(M, (prepare_kernel<kM, 0, false><<<F, 256, 0, st>>>(F, N, y, ginv, v0, v, vfloor, status, bins, ex)); return cudaGetLastError())
  }
}

cudaError_t launch_ll_ranges(int nmix, int iters, int F, const double* llf, const int* b0,
                             const int* nb, const int* mix_id, double* out, cudaStream_t st) {
  if (nmix <= 0 || iters <= 0) return cudaSuccess;
  ll_ranges_kernel<<<dim3(nmix, iters), 128, 0, st>>>(F, llf, b0, nb, mix_id, iters, out);
  return cudaGetLastError();
}

cudaError_t launch_ll_reduce(int F, int iters, const double* llf, double* ll, cudaStream_t st) {
  if (iters <= 0) return cudaSuccess;
  ll_reduce_kernel<<<iters, 256, 0, st>>>(F, llf, ll);
  return cudaGetLastError();
}

cudaError_t launch_invert_scale(int F, const float* g, float* ginv, cudaStream_t st) {
  invert_scale_kernel<<<(F + 255) / 256, 256, 0, st>>>(F, g, ginv);
  return cudaGetLastError();
}

}  // namespace fca
