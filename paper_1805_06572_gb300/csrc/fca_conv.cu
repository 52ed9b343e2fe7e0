// Conventional FCA EM (Ito, Araki, Nakatani, arXiv 1805.06572, Sec. 2) on sm_103a.
//
// The plain form: every time-frequency point does the frame-wise matrix work the paper
// names as the cost of FCA (Sec. 2, last paragraph). One CTA owns one frequency bin for
// all iterations; one thread owns one time-frequency point at a time (FP32):
//   Rx = v1 S1 + v2 S2, Cholesky Rx = L L^H
//   u = Rx^-1 y, mu_j = v_j S_j u                                  Eq. (MMSE)
//   C = v1 v2 S1 Rx^-1 S2 = v1 v2 (L^-1 S1)^H (L^-1 S2)            Eq. (postquadexp)
//   Phi_j = mu_j mu_j^H + C
//   v_j' = tr(S_j^-1 Phi_j) / M  (old S_j), as sums of squares     Eq. (vupdate)
//   Gram_j += Phi_j / v_j'                                          Eq. (Supdate)
//   log-likelihood term -log det Rx - y^H Rx^-1 y                   Eq. (like)
// then the CTA merges the Gram partial sums (FP32 warp transpose-reduction, FP64 across
// warps) and sets S_j' = Gram_j / N in FP64. The Cholesky factors K_j of S_j for the next v
// update are formed once per frequency per iteration by warp 0 (FP64 factorisation).
// For M >= 6 the per-point matrices do not fit one thread's registers and spill. The other
// layout (FCA_CONV_GROUP) has a group of G = 8 lanes (4 for M <= 4) share each point
// (conv_group_point): lane r owns row r of Rx and L, column r of L^-1 and of L^-1 S_j, row r
// of C and of the Gram partial sums, and the group exchanges values by shuffles and per-group
// shared tiles; it spills at no M, but runs slower (conv_grouped).
#include <type_traits>

#include "fca.h"
#include "fca_dev.cuh"
#include "fca_internal.h"

namespace fca {

template <int M, int NW>
struct ConvShared {
  static constexpr int V = 2 * M * M + 2;
  float red[NW][V];
  double tot[V];
  double2 S[2][M][kMaxM];
  float2 S32[2][M][M];
  float2 K32[2][M][M];  // S32_j = K_j K_j^H
  int fail;
  WarpLAT<double, M> la;
};

__host__ __device__ constexpr int cpair_index(int M, int i, int k) {  // i < k
  return i * (M - 1) - i * (i - 1) / 2 + (k - i - 1);
}

// The FP32 copy S32 of the FP64 S_j used by the bin pass, and the Cholesky factor K of S32
// itself (S32 = K K^H; factorised in FP64 from the exact FP32 values, then rounded): warp 0.
// Returns false if S32 is not positive definite.
template <int M, int R>
__device__ bool warp_hpd_factor(WarpLAT<double, R>& la, const double2 (*S)[kMaxM], float2 (*S32)[M],
                                float2 (*K)[M], int lane) {
  for (int e = lane; e < M * M; e += 32) {
    const int i = e / M, j = e % M;
    const float2 s = z2c(S[i][j]);
    S32[i][j] = s;
    la.L[i][j] = c2z(s);
  }
  __syncwarp();
  if (!warp_cholesky<M>(la, lane)) return false;
  for (int e = lane; e < M * M; e += 32) {
    const int i = e / M, j = e % M;
    K[i][j] = (j <= i) ? z2c(la.L[i][j]) : make_float2(0.f, 0.f);
  }
  __syncwarp();
  return true;
}

// Lanes per time-frequency point in the lane-group pass (a power of two >= M).
__host__ __device__ constexpr int conv_group(int M) { return M <= 4 ? 4 : 8; }
// The layout FCA_CONV_AUTO takes for M: one thread per point at every M. Measured on GB300
// (fused kernel, L = 50 or 100): M = 4, F = 513, N = 1000: 2.1 ms per thread vs 7.4 ms in lane
// groups; M = 6, F = 257, N = 2000: 5.8 vs 26.2 ms; M = 8, F = 1025, N = 4000 (FP16): 401 vs
// 546 ms. The one-thread layout's spills (200 bytes per thread at M = 6, 1.2 KB at M = 8) cost
// less than the lane groups' exchanges and duplicated triangular work.
__host__ __device__ constexpr bool conv_grouped(int) { return false; }

// Per-group shared tiles of the lane-group pass: L^-1 (lower triangle), B = L^-1 S2, and the
// vectors y, w = L^-1 y, u = Rx^-1 y, mu_1, mu_2 of the group's current point. The groups of a
// warp read their own tiles at the same offsets at once: each tile's stride is padded by one
// float2 so that those reads fall in different banks.
template <int M, int NT>
struct ConvGroupTiles {
  static constexpr int NG = NT / conv_group(M);
  struct Tile {
    float2 Li[M][M];
    float2 pad0;
    float2 B[M][M];
    float2 pad1;
    float2 y[M], w[M], u[M], mu1[M], mu2[M];
    float2 pad2;
  };
  Tile g[NG];
};
struct ConvNoTiles {};

// Sum over the G lanes of a group (every lane of the group receives it).
template <int G>
__device__ __forceinline__ float group_sum(float x) {
#pragma unroll
  for (int o = 1; o < G; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Per-lane partial sums of the lane-group pass: row r of both Gram sums (all columns; the
// columns k >= r are used), log det Rx and y^H Rx^-1 y terms.
template <int M>
struct ConvGroupAcc {
  float2 g1[M], g2[M];
  float ld, quad;
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < M; ++k) g1[k] = g2[k] = make_float2(0.f, 0.f);
    ld = quad = 0.f;
  }
  __device__ __forceinline__ void add(const ConvGroupAcc& o) {
#pragma unroll
    for (int k = 0; k < M; ++k) {
      g1[k] = cadd(g1[k], o.g1[k]);
      g2[k] = cadd(g2[k], o.g2[k]);
    }
    ld += o.ld;
    quad += o.quad;
  }
};

// One time-frequency point (y, v1, v2) on a group of G lanes (rows r = lane mod G; rows
// r >= M carry zeros and take part in the exchanges only). The same quantities as the
// one-thread pass of conv_em_kernel, arranged so that each lane's work is a few independent
// dot products: Rx = v1 S1 + v2 S2 = L L^H (right-looking, row r in registers, column j's
// entries broadcast by shuffles), column r of L^-1, then w = L^-1 y, u = L^-H w, mu_j = v_j S_j u,
// the v update from sums of squares (K_j^H u, column r of L^-1 K_j), and row r of
// C = v1 v2 (L^-1 S1)^H (L^-1 S2) from column r of L^-1 S1 and the tile of L^-1 S2.
// Returns (v1', v2') on every lane of the group; adds row r of Phi_j / v_j' to acc when `on`.
template <int M, int G, int NT>
__device__ float2 conv_group_point(const ConvShared<M, NT / 32>& sh, ConvGroupTiles<M, NT>& gt,
                                   int gid, int r, int base, float2 yr, float v1, float v2, float vf,
                                   bool on, int& bad, ConvGroupAcc<M>& acc) {
  typename ConvGroupTiles<M, NT>::Tile& tg = gt.g[gid];
  const bool row = r < M;
  const int rc = row ? r : 0;
  if (row) tg.y[r] = yr;
  // Row r of Rx (entries k <= r), factorised in place into row r of L.
  float2 R[M];
#pragma unroll
  for (int k = 0; k < M; ++k)
    R[k] = (row && k <= r) ? cadd(cscale(sh.S32[0][r][k], v1), cscale(sh.S32[1][r][k], v2))
                           : make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const float d = __shfl_sync(0xffffffffu, R[j].x, base + j);  // pivot j (lane j's diagonal)
    const float ij = rsqrtf(d);
    if (r == j) {
      bad |= !(d > 0.f);
      if (on) acc.ld += logf(d);
      R[j] = make_float2(d * ij, ij);  // (L_jj, 1 / L_jj)
    } else if (r > j) {
      R[j] = cscale(R[j], ij);  // L[r][j]
    }
#pragma unroll
    for (int k = j + 1; k < M; ++k) {
      const float2 lk = shfl2(R[j], base + k);  // L[k][j]
      if (r >= k) R[k] = csub(R[k], cmulc(R[j], lk));
    }
  }
  // Column r of L^-1: x_r = 1 / L_rr, x_i = -(sum_{r <= k < i} L[i][k] x_k) / L_ii (rows of L
  // broadcast from their lanes).
  {
    float2 x[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < i; ++k) {
        const float2 lik = shfl2(R[k], base + i);  // L[i][k] from lane i
        if (k >= r) s = csub(s, cmul(lik, x[k]));
      }
      const float iii = __shfl_sync(0xffffffffu, R[i].y, base + i);  // 1 / L_ii
      x[i] = (i < r) ? make_float2(0.f, 0.f) : (i == r ? make_float2(iii, 0.f) : cscale(s, iii));
    }
    if (row) {
#pragma unroll
      for (int i = 0; i < M; ++i) tg.Li[i][r] = x[i];
    }
  }
  __syncwarp();
  // w = L^-1 y (row r), then u = L^-H w (row r).
  float2 t = make_float2(0.f, 0.f);
  if (row) {
#pragma unroll
    for (int k = 0; k < M; ++k)
      if (k <= r) t = cfma(tg.Li[r][k], tg.y[k], t);
    tg.w[r] = t;
  }
  if (on && row) acc.quad += cabs2(t);
  __syncwarp();
  t = make_float2(0.f, 0.f);
  if (row) {
#pragma unroll
    for (int k = 0; k < M; ++k)
      if (k >= r) t = cfma(cconj(tg.Li[k][r]), tg.w[k], t);
    tg.u[r] = t;
  }
  __syncwarp();
  // mu_j = v_j S_j u (row r), and (K_j^H u)_r.
  float2 m1 = make_float2(0.f, 0.f), m2 = m1, a1 = m1, a2 = m1;
  if (row) {
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const float2 uk = tg.u[k];
      m1 = cfma(sh.S32[0][r][k], uk, m1);
      m2 = cfma(sh.S32[1][r][k], uk, m2);
      if (k >= r) {
        a1 = cfma(cconj(sh.K32[0][k][r]), uk, a1);
        a2 = cfma(cconj(sh.K32[1][k][r]), uk, a2);
      }
    }
    m1 = cscale(m1, v1);
    m2 = cscale(m2, v2);
    tg.mu1[r] = m1;
    tg.mu2[r] = m2;
  }
  // Columns r of A = L^-1 S1 and B = L^-1 S2 (B into the tile), and the squared norms of
  // columns r of L^-1 K1 and L^-1 K2 (K_j lower triangular: rows k >= r only).
  float2 ac[M];
  float x1n = 0.f, x2n = 0.f;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    float2 sa = make_float2(0.f, 0.f), sb = sa, s1 = sa, s2 = sa;
#pragma unroll
    for (int k = 0; k <= i; ++k) {
      const float2 l = tg.Li[i][k];
      sa = cfma(l, sh.S32[0][k][rc], sa);
      sb = cfma(l, sh.S32[1][k][rc], sb);
      if (k >= r) {
        s1 = cfma(l, sh.K32[0][k][rc], s1);
        s2 = cfma(l, sh.K32[1][k][rc], s2);
      }
    }
    ac[i] = sa;
    if (row) tg.B[i][r] = sb;
    x1n += cabs2(s1);
    x2n += cabs2(s2);
  }
  // v_j' = (mu_j^H S_j^-1 mu_j + tr(S_j^-1 C)) / M (Eq. (vupdate)) from the group sums:
  // mu_j^H S_j^-1 mu_j = v_j^2 ||K_j^H u||^2, tr(S1^-1 C) = v1 v2 ||L^-1 K2||_F^2,
  // tr(S2^-1 C) = v1 v2 ||L^-1 K1||_F^2.
  const float q1 = group_sum<G>(cabs2(a1)), q2 = group_sum<G>(cabs2(a2));
  const float r2 = group_sum<G>(row ? x1n : 0.f), r1 = group_sum<G>(row ? x2n : 0.f);
  const float v1n = fmaxf(v1 * fmaf(v1, q1, v2 * r1) * (1.f / M), vf);
  const float v2n = fmaxf(v2 * fmaf(v2, q2, v1 * r2) * (1.f / M), vf);
  __syncwarp();
  // Row r of Phi_j / v_j' (columns k >= r): mu_j,r conj(mu_j,k) + C[r][k], with
  // C[r][k] = v1 v2 sum_m conj(A[m][r]) B[m][k].
  if (on && row) {
    const float w1 = __fdividef(1.f, v1n), w2 = __fdividef(1.f, v2n);
    const float v12 = v1 * v2;
#pragma unroll
    for (int k = 0; k < M; ++k) {
      if (k >= r) {
        float2 c = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < M; ++m) c = cfma(cconj(ac[m]), tg.B[m][k], c);
        c = cscale(c, v12);
        const float2 z1 = cadd(cmulc(m1, tg.mu1[k]), c);
        const float2 z2 = cadd(cmulc(m2, tg.mu2[k]), c);
        acc.g1[k] = make_float2(fmaf(z1.x, w1, acc.g1[k].x), fmaf(z1.y, w1, acc.g1[k].y));
        acc.g2[k] = make_float2(fmaf(z2.x, w2, acc.g2[k].x), fmaf(z2.y, w2, acc.g2[k].y));
      }
    }
  }
  __syncwarp();
  return make_float2(v1n, v2n);
}

// One iteration's pass over the bin's frames on lane groups, ending with the warp's partial
// sums in sh.red[warp] (the layout of warp_reduce_store: diagonal, then the (re, im) pairs of
// the upper triangle, for each Gram; then log det Rx and y^H Rx^-1 y). The point loop runs
// the same number of times on every group (groups past the last frame compute on a dummy
// point and add nothing).
template <int M, int ST, int NT, bool kB>
__device__ void conv_group_iteration(ConvShared<M, NT / 32>& sh, ConvGroupTiles<M, NT>& gt,
                                     const ConvEmArgs& a, const typename Elem<ST>::T* ysrc, float* v1p,
                                     float* v2p, float* vg1, int dv2, ptrdiff_t d_prev, int f, int N,
                                     float vf, float gi, bool last, int& bad, int tid) {
  constexpr int G = conv_group(M), P = NT / G, MM = M * M;
  const int lane = tid & 31, warp = tid >> 5;
  const int gid = tid / G, r = lane & (G - 1), base = lane & ~(G - 1);
  // Two-level FP32 sums (a block of 16 points, then the blocks), so that no FP32 sum runs over
  // more than a few dozen terms however many frames a group takes.
  ConvGroupAcc<M> acc, blk;
  acc.zero();
  blk.zero();
  int nb = 0;
  for (int n0 = 0; n0 < N; n0 += P) {
    const int n = n0 + gid;
    const bool on = n < N;
    float2 yr = make_float2(0.f, 0.f);
    float v1 = 1.f, v2 = 1.f;
    if (on) {
      v1 = v1p[n];
      v2 = v2p[n];
      if (r < M) yr = cscale(decode(ysrc[(size_t)n * M + r]), gi);
      if (last && r == 0) {
        if constexpr (kB) {
          vg1[d_prev + n] = v1;
          vg1[d_prev + dv2 + n] = v2;
        } else {
          a.v_prev[(size_t)f * N + n] = v1;
          a.v_prev[(size_t)a.F * N + (size_t)f * N + n] = v2;
        }
      }
    }
    const float2 vn = conv_group_point<M, G, NT>(sh, gt, gid, r, base, yr, v1, v2, vf, on, bad, blk);
    if (on && r == 0) {
      v1p[n] = vn.x;
      v2p[n] = vn.y;
    }
    if (++nb == 16) {
      acc.add(blk);
      blk.zero();
      nb = 0;
    }
  }
  acc.add(blk);
  // Sum each row over the warp's groups, then write the packed partial sums.
#pragma unroll
  for (int o = G; o < 32; o <<= 1) {
#pragma unroll
    for (int k = 0; k < M; ++k) {
      acc.g1[k].x += __shfl_xor_sync(0xffffffffu, acc.g1[k].x, o);
      acc.g1[k].y += __shfl_xor_sync(0xffffffffu, acc.g1[k].y, o);
      acc.g2[k].x += __shfl_xor_sync(0xffffffffu, acc.g2[k].x, o);
      acc.g2[k].y += __shfl_xor_sync(0xffffffffu, acc.g2[k].y, o);
    }
    acc.ld += __shfl_xor_sync(0xffffffffu, acc.ld, o);
    acc.quad += __shfl_xor_sync(0xffffffffu, acc.quad, o);
  }
  const float ld = group_sum<G>(acc.ld), quad = group_sum<G>(acc.quad);
  float* out = sh.red[warp];
  if (lane < M) {
#pragma unroll
    for (int k = 0; k < M; ++k) {
      if (k == lane) {
        out[lane] = acc.g1[k].x;
        out[MM + lane] = acc.g2[k].x;
      } else if (k > lane) {
        const int o = M + 2 * cpair_index(M, lane, k);
        out[o] = acc.g1[k].x;
        out[o + 1] = acc.g1[k].y;
        out[MM + o] = acc.g2[k].x;
        out[MM + o + 1] = acc.g2[k].y;
      }
    }
  }
  if (lane == 0) {
    out[2 * MM] = ld;
    out[2 * MM + 1] = quad;
  }
}

// Resident CTAs per SM the register budget is sized for (kB: batches; LG: lane groups). The
// lane-group pass spills at no M; the one-thread pass holds every per-point matrix in registers
// and spills for M >= 6.
__host__ __device__ constexpr int conv_min_blocks(int M, bool kB, bool LG) {
  return LG ? (M <= 3 ? 4 : ((M == 7 || (M == 8 && kB)) ? 2 : 3)) : (M <= 3 ? 4 : (M <= 4 ? 3 : 2));
}

// kB: the CTA's bin comes from the descriptor table a.bins (a batch); otherwise bin
// f = blockIdx.x of one mixture with v_in == v and S_in == S.
template <int M, int ST, int NT, bool kB, bool LG>
__global__ void __launch_bounds__(NT, conv_min_blocks(M, kB, LG)) conv_em_kernel(const ConvEmArgs a) {
  using E = typename Elem<ST>::T;
  constexpr int NW = NT / 32;
  using Sh = ConvShared<M, NW>;
  constexpr int V = Sh::V;
  using RS = RedShape<V>;
  constexpr int MM = M * M;
  __shared__ Sh sh;
  __shared__ typename std::conditional<LG, ConvGroupTiles<M, NT>, ConvNoTiles>::type gt;
  extern __shared__ __align__(16) unsigned char dyn[];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int F = a.F;
  int f, N;
  size_t yoff, v1off, v2off;
  if constexpr (kB) {
    const BinDesc d = a.bins[blockIdx.x];
    f = d.b;
    N = d.N;
    yoff = (size_t)d.y_off;
    v1off = (size_t)d.v1_off;
    v2off = (size_t)d.v2_off;
  } else {
    f = blockIdx.x;
    N = a.N;
    yoff = (size_t)f * N * M;
    v1off = (size_t)f * N;
    v2off = (size_t)F * N + v1off;
  }
  const E* yg = reinterpret_cast<const E*>(a.y) + yoff;
  float* vg1 = a.v + v1off;
  const int dv2 = (int)(v2off - v1off);  // v_2(., bin) lies dv2 floats after v_1(., bin)
  const ptrdiff_t d_in = kB ? a.v_in - a.v : 0, d_prev = a.v_prev - a.v;
  E* ys = reinterpret_cast<E*>(dyn);
  const size_t ybytes = ((size_t)N * M * sizeof(E) + 15) & ~(size_t)15;
  float* vs = reinterpret_cast<float*>(dyn + ybytes);
  // One mixture: the launch reserves exactly its bins' need, or nothing.
  const bool res = kB ? em_bin_smem(M, ST, N) <= (size_t)a.res_bytes : a.res_bytes != 0;
  const E* ysrc = res ? ys : yg;
  float* v1p = res ? vs : vg1;
  float* v2p = res ? vs + N : (kB ? vg1 + dv2 : a.v + (size_t)F * N + (size_t)f * N);
  const float vf = a.vfloor[f];
  const float gi = (ST == 1) ? a.ginv[f] : 1.f;

  for (int e = tid; e < 2 * MM; e += NT) {
    const int j = e / MM, r = e % MM;
    sh.S[j][r / M][r % M] = (kB ? a.S_in : a.S)[((size_t)j * F + f) * MM + r];
  }
  if (tid == 0) sh.fail = 0;
  if (res) {
    const size_t bytes = (size_t)N * M * sizeof(E);
    if ((bytes & 15) == 0 && (!kB || (reinterpret_cast<uintptr_t>(yg) & 15) == 0)) {
      const uint4* src = reinterpret_cast<const uint4*>(yg);
      uint4* dst = reinterpret_cast<uint4*>(ys);
      for (size_t i = tid; i < bytes / 16; i += NT) dst[i] = src[i];
    } else {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(yg);
      uint32_t* dst = reinterpret_cast<uint32_t*>(ys);
      for (size_t i = tid; i < bytes / 4; i += NT) dst[i] = src[i];
    }
    for (int n = tid; n < N; n += NT) {
      vs[n] = vg1[d_in + n];
      vs[N + n] = vg1[d_in + dv2 + n];
    }
  } else if (kB && d_in != 0) {
    // Streaming bin with separate initial values: start the working copy from them (each
    // thread copies the frames it updates in the iterations below).
    for (int n = tid; n < N; n += NT) {
      vg1[n] = vg1[d_in + n];
      vg1[dv2 + n] = vg1[d_in + dv2 + n];
    }
  }
  __syncthreads();

  for (int it = 0; it < a.iters; ++it) {
    const bool last = (it == a.iters - 1);
    if (last) {
      for (int e = tid; e < 2 * MM; e += NT) {
        const int j = e / MM, r = e % MM;
        a.S_prev[((size_t)j * F + f) * MM + r] = sh.S[j][r / M][r % M];
      }
    }
    if (warp == 0) {
      bool ok = warp_hpd_factor<M>(sh.la, sh.S[0], sh.S32[0], sh.K32[0], lane);
      ok = ok && warp_hpd_factor<M>(sh.la, sh.S[1], sh.S32[1], sh.K32[1], lane);
      if (!ok && lane == 0) {
        set_status(a.status, kErrNotPD);
        sh.fail = kErrNotPD;
      }
    }
    __syncthreads();
    if (sh.fail) break;

    int bad = 0;
    if constexpr (LG) {
      conv_group_iteration<M, ST, NT, kB>(sh, gt, a, ysrc, v1p, v2p, vg1, dv2, d_prev, f, N, vf, gi, last,
                                          bad, tid);
    } else {
    float acc[RS::NA];
#pragma unroll
    for (int j = 0; j < RS::NA; ++j) acc[j] = 0.f;
    for (int n = tid; n < N; n += NT) {
      float2 yv[M];
      load_bin<M, ST>(ysrc + (size_t)n * M, yv);
#pragma unroll
      for (int i = 0; i < M; ++i) yv[i] = cscale(yv[i], gi);
      const float v1 = v1p[n], v2 = v2p[n];
      if (last) {
        if constexpr (kB) {
          vg1[d_prev + n] = v1;
          vg1[d_prev + dv2 + n] = v2;
        } else {
          a.v_prev[(size_t)f * N + n] = v1;
          a.v_prev[(size_t)F * N + (size_t)f * N + n] = v2;
        }
      }
      // Cholesky of Rx = v1 S1 + v2 S2 (lower triangle), in registers.
      float2 L[M][M];
      LogProd lp;  // product of the Cholesky pivots = det Rx
#pragma unroll
      for (int j = 0; j < M; ++j) {
#pragma unroll
        for (int i = j; i < M; ++i) {
          float2 s = cadd(cscale(sh.S32[0][i][j], v1), cscale(sh.S32[1][i][j], v2));
#pragma unroll
          for (int k = 0; k < j; ++k) s = csub(s, cmulc(L[i][k], L[j][k]));
          if (i == j) {
            const float piv = s.x;
            bad |= !(piv > 0.f);
            lp.mul(piv);
            L[j][j] = make_float2(sqrtf(piv), rsqrtf(piv));  // (L_jj, 1/L_jj)
          } else {
            L[i][j] = cscale(s, L[j][j].y);
          }
        }
      }
      // w = L^-1 y, u = L^-H w = Rx^-1 y.
      float2 w[M], u[M];
      float quad = 0.f;
#pragma unroll
      for (int i = 0; i < M; ++i) {
        float2 s = yv[i];
#pragma unroll
        for (int k = 0; k < i; ++k) s = csub(s, cmul(L[i][k], w[k]));
        w[i] = cscale(s, L[i][i].y);
        quad += cabs2(w[i]);
      }
#pragma unroll
      for (int i = M - 1; i >= 0; --i) {
        float2 s = w[i];
#pragma unroll
        for (int k = i + 1; k < M; ++k) s = csub(s, ccmul(L[k][i], u[k]));
        u[i] = cscale(s, L[i][i].y);
      }
      // mu_j = v_j S_j u.
      float2 mu1[M], mu2[M];
#pragma unroll
      for (int i = 0; i < M; ++i) {
        float2 s1 = make_float2(0.f, 0.f), s2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < M; ++k) {
          s1 = cfma(sh.S32[0][i][k], u[k], s1);
          s2 = cfma(sh.S32[1][i][k], u[k], s2);
        }
        mu1[i] = cscale(s1, v1);
        mu2[i] = cscale(s2, v2);
      }
      // A = L^-1 S1, B = L^-1 S2 (column by column), C = v1 v2 A^H B (upper triangle).
      float2 A[M][M], B[M][M];
#pragma unroll
      for (int c = 0; c < M; ++c) {
#pragma unroll
        for (int i = 0; i < M; ++i) {
          float2 sa = sh.S32[0][i][c], sb = sh.S32[1][i][c];
#pragma unroll
          for (int k = 0; k < i; ++k) {
            sa = csub(sa, cmul(L[i][k], A[k][c]));
            sb = csub(sb, cmul(L[i][k], B[k][c]));
          }
          A[i][c] = cscale(sa, L[i][i].y);
          B[i][c] = cscale(sb, L[i][i].y);
        }
      }
      const float v12 = v1 * v2;
      float2 C[M][M];
#pragma unroll
      for (int i = 0; i < M; ++i)
#pragma unroll
        for (int k = i; k < M; ++k) {
          float2 s = make_float2(0.f, 0.f);
#pragma unroll
          for (int m = 0; m < M; ++m) s = cadd(s, ccmul(A[m][i], B[m][k]));
          C[i][k] = cscale(s, v12);
          if (k == i) C[i][i].y = 0.f;
        }
      // v_j' = (mu_j^H S_j^-1 mu_j + tr(S_j^-1 C)) / M with the old S_j (Eq. (vupdate)), as sums
      // of squares: mu_j = v_j S_j u gives mu_j^H S_j^-1 mu_j = v_j^2 ||K_j^H u||^2, and
      // C = v1 v2 S1 Rx^-1 S2 gives tr(S1^-1 C) = v1 v2 ||L^-1 K2||_F^2 and tr(S2^-1 C) =
      // v1 v2 ||L^-1 K1||_F^2 (Rx = L L^H, S_j = K_j K_j^H): no cancellation, and no S_j^-1.
      float q1 = 0.f, q2 = 0.f, r1 = 0.f, r2 = 0.f;
#pragma unroll
      for (int c = 0; c < M; ++c) {
        float2 a1 = make_float2(0.f, 0.f), a2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int r = c; r < M; ++r) {  // (K_j^H u)_c
          a1 = cfma(cconj(sh.K32[0][r][c]), u[r], a1);
          a2 = cfma(cconj(sh.K32[1][r][c]), u[r], a2);
        }
        q1 += cabs2(a1);
        q2 += cabs2(a2);
        float2 x1[M], x2[M];  // column c of L^-1 K_j (zero above row c)
#pragma unroll
        for (int i = c; i < M; ++i) {
          float2 s1 = sh.K32[0][i][c], s2 = sh.K32[1][i][c];
#pragma unroll
          for (int k = c; k < i; ++k) {
            s1 = csub(s1, cmul(L[i][k], x1[k]));
            s2 = csub(s2, cmul(L[i][k], x2[k]));
          }
          x1[i] = cscale(s1, L[i][i].y);
          x2[i] = cscale(s2, L[i][i].y);
          r2 += cabs2(x1[i]);
          r1 += cabs2(x2[i]);
        }
      }
      const float t1 = v1 * fmaf(v1, q1, v2 * r1);
      const float t2 = v2 * fmaf(v2, q2, v1 * r2);
      const float v1n = fmaxf(t1 * (1.f / M), vf);
      const float v2n = fmaxf(t2 * (1.f / M), vf);
      v1p[n] = v1n;
      v2p[n] = v2n;
      const float w1 = __fdividef(1.f, v1n), w2 = __fdividef(1.f, v2n);
      // Gram_j += (mu_j mu_j^H + C) / v_j' (upper triangle).
#pragma unroll
      for (int i = 0; i < M; ++i) {
        acc[i] += (cabs2(mu1[i]) + C[i][i].x) * w1;
        acc[MM + i] += (cabs2(mu2[i]) + C[i][i].x) * w2;
#pragma unroll
        for (int k = i + 1; k < M; ++k) {
          const int o = M + 2 * cpair_index(M, i, k);
          const float2 z1 = cadd(cmulc(mu1[i], mu1[k]), C[i][k]);
          const float2 z2 = cadd(cmulc(mu2[i], mu2[k]), C[i][k]);
          acc[o] = fmaf(z1.x, w1, acc[o]);
          acc[o + 1] = fmaf(z1.y, w1, acc[o + 1]);
          acc[MM + o] = fmaf(z2.x, w2, acc[MM + o]);
          acc[MM + o + 1] = fmaf(z2.y, w2, acc[MM + o + 1]);
        }
      }
      acc[2 * MM] += lp.log();
      acc[2 * MM + 1] += quad;
    }
    warp_reduce_store<V>(acc, lane, sh.red[warp]);
    }
    if (__syncthreads_or(bad)) {
      if (tid == 0) {
        set_status(a.status, kErrNotPD);
        sh.fail = kErrNotPD;
      }
    }
    __syncthreads();
    for (int i = tid; i < V; i += NT) {  // fixed-order FP64 merge across warps (pairwise)
      double s[NW];
#pragma unroll
      for (int w = 0; w < NW; ++w) s[w] = (double)sh.red[w][i];
#pragma unroll
      for (int h = NW / 2; h >= 1; h >>= 1)
#pragma unroll
        for (int w = 0; w < h; ++w) s[w] += s[w + h];
      sh.tot[i] = s[0];
    }
    __syncthreads();
    const double invN = 1.0 / (double)N;
    for (int e = tid; e < 2 * MM; e += NT) {  // S_j' = Gram_j / N (Eq. (Supdate))
      const int j = e / MM, r = e % MM, i = r / M, k = r % M;
      double2 s;
      if (i == k) {
        s = make_double2(sh.tot[j * MM + i] * invN, 0.0);
      } else {
        const int lo = min(i, k), hi = max(i, k);
        const int o = j * MM + M + 2 * cpair_index(M, lo, hi);
        s = make_double2(sh.tot[o] * invN, (i < k ? 1.0 : -1.0) * sh.tot[o + 1] * invN);
      }
      sh.S[j][i][k] = s;
    }
    if (tid == 0) {
      const double ll = -(double)N * M * 1.1447298858494002 - sh.tot[2 * MM] - sh.tot[2 * MM + 1];
      a.llf[(size_t)it * F + f] = ll;
      if (!isfinite(ll)) {
        set_status(a.status, kErrNonFinite);
        sh.fail = kErrNonFinite;
      }
    }
    __syncthreads();
    if (sh.fail) break;
  }

  for (int e = tid; e < 2 * MM; e += NT) {
    const int j = e / MM, r = e % MM;
    a.S[((size_t)j * F + f) * MM + r] = sh.S[j][r / M][r % M];
  }
  if (res) {
    for (int n = tid; n < N; n += NT) {
      vg1[n] = vs[n];
      vg1[dv2 + n] = vs[N + n];
    }
  }
}

// Posterior means of the conventional form, mu_j = v_j S_j (v1 S1 + v2 S2)^-1 y (Eq. (MMSE)).
template <int M, int ST>
__global__ void __launch_bounds__(256) sep_conv_kernel(const SepConvArgs a) {
  using E = typename Elem<ST>::T;
  __shared__ float2 S32[2][M][M];
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
  if (blockIdx.y * 256 >= N) return;  // whole CTA past this bin's frames
  const size_t MM = (size_t)M * M;
  if (tid < 2 * M * M) {
    const int j = tid / (M * M), r = tid % (M * M);
    S32[j][r / M][r % M] = z2c(a.S[((size_t)j * a.F + f) * MM + r]);
  }
  __syncthreads();
  const int n = blockIdx.y * 256 + tid;
  if (n >= N) return;
  const size_t b = xoff + (size_t)n * M;
  const float gi = (ST == 1) ? a.ginv[f] : 1.f;
  float2 yv[M];
  load_bin<M, ST>(reinterpret_cast<const E*>(a.y) + yoff + (size_t)n * M, yv);
  const float v1 = a.v[v1off + n], v2 = a.v[v2off + n];
  float2 L[M][M];
  int bad = 0;
#pragma unroll
  for (int j = 0; j < M; ++j)
#pragma unroll
    for (int i = j; i < M; ++i) {
      float2 s = cadd(cscale(S32[0][i][j], v1), cscale(S32[1][i][j], v2));
#pragma unroll
      for (int k = 0; k < j; ++k) s = csub(s, cmulc(L[i][k], L[j][k]));
      if (i == j) {
        bad |= !(s.x > 0.f);
        L[j][j] = make_float2(sqrtf(s.x), rsqrtf(s.x));
      } else {
        L[i][j] = cscale(s, L[j][j].y);
      }
    }
  if (bad) set_status(a.status, kErrNotPD);
  float2 w[M], u[M];
#pragma unroll
  for (int i = 0; i < M; ++i) {
    float2 s = cscale(yv[i], gi);
#pragma unroll
    for (int k = 0; k < i; ++k) s = csub(s, cmul(L[i][k], w[k]));
    w[i] = cscale(s, L[i][i].y);
  }
#pragma unroll
  for (int i = M - 1; i >= 0; --i) {
    float2 s = w[i];
#pragma unroll
    for (int k = i + 1; k < M; ++k) s = csub(s, ccmul(L[k][i], u[k]));
    u[i] = cscale(s, L[i][i].y);
  }
#pragma unroll
  for (int i = 0; i < M; ++i) {
    float2 s1 = make_float2(0.f, 0.f), s2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < M; ++k) {
      s1 = cfma(S32[0][i][k], u[k], s1);
      s2 = cfma(S32[1][i][k], u[k], s2);
    }
    a.x1[b + i] = cscale(s1, v1);
    a.x2[b + i] = cscale(s2, v2);
  }
}

// ------------------------------------------------------------------ host-side launchers
template <int M, int ST, int NT>
static cudaError_t launch_conv_t(const ConvEmArgs& a, cudaStream_t st) {
  const size_t dyn = (size_t)a.res_bytes;
  const int grid = a.bins ? a.nbins : a.F;
  if (grid <= 0) return cudaSuccess;
  if (a.bins && ST != 0) return cudaErrorInvalidValue;  // batches hold complex64 mixtures
  const bool lg = a.layout == FCA_CONV_GROUP || (a.layout != FCA_CONV_THREAD && conv_grouped(M));
  auto k = a.bins ? (lg ? conv_em_kernel<M, 0, NT, true, true> : conv_em_kernel<M, 0, NT, true, false>)
                  : (lg ? conv_em_kernel<M, ST, NT, false, true> : conv_em_kernel<M, ST, NT, false, false>);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  if (dyn > 0) {  // the default limit (48 KB) covers static and dynamic shared memory together
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  k<<<grid, NT, dyn, st>>>(a);
  return cudaGetLastError();
}

template <int M, int ST>
static cudaError_t launch_conv_m(const ConvEmArgs& a, cudaStream_t st) {
  return launch_conv_t<M, ST, 128>(a, st);
}

template <int ST>
static cudaError_t launch_conv_s(int M, const ConvEmArgs& a, cudaStream_t st) {
  switch (M) {
    case 1: return launch_conv_m<1, ST>(a, st);
    case 2: return launch_conv_m<2, ST>(a, st);
    case 3: return launch_conv_m<3, ST>(a, st);
    case 4: return launch_conv_m<4, ST>(a, st);
    case 5: return launch_conv_m<5, ST>(a, st);
    case 6: return launch_conv_m<6, ST>(a, st);
    case 7: return launch_conv_m<7, ST>(a, st);
    case 8: return launch_conv_m<8, ST>(a, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_conv_em(int M, int storage, const ConvEmArgs& a, cudaStream_t st) {
  return storage ? launch_conv_s<1>(M, a, st) : launch_conv_s<0>(M, a, st);
}

template <int M, int ST>
static cudaError_t launch_sep_conv_m(const SepConvArgs& a, cudaStream_t st) {
  dim3 grid(a.F, (a.N + 255) / 256);  // bins on x (no 65535 limit), frame chunks on y
  if (a.N <= 0 || a.F <= 0) return cudaSuccess;
  sep_conv_kernel<M, ST><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

template <int ST>
static cudaError_t launch_sep_conv_s(int M, const SepConvArgs& a, cudaStream_t st) {
  switch (M) {
    case 1: return launch_sep_conv_m<1, ST>(a, st);
    case 2: return launch_sep_conv_m<2, ST>(a, st);
    case 3: return launch_sep_conv_m<3, ST>(a, st);
    case 4: return launch_sep_conv_m<4, ST>(a, st);
    case 5: return launch_sep_conv_m<5, ST>(a, st);
    case 6: return launch_sep_conv_m<6, ST>(a, st);
    case 7: return launch_sep_conv_m<7, ST>(a, st);
    case 8: return launch_sep_conv_m<8, ST>(a, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sep_conv(int M, int storage, const SepConvArgs& a, cudaStream_t st) {
  return storage ? launch_sep_conv_s<1>(M, a, st) : launch_sep_conv_s<0>(M, a, st);
}

}  // namespace fca
