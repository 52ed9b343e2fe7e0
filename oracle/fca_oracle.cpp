// FP64 CPU oracle for two-source FCA EM (Ito, Araki, Nakatani, "FastFCA", arXiv 1805.06572).
//
// TEST INFRASTRUCTURE ONLY. Only tests/, the smoke check and the benchmark's CPU-baseline
// leg may load this library. It shares no code with the CUDA path and is deliberately plain:
// complex128 (std::complex<double>) everywhere, full M x M matrices, explicit inverses by
// Gauss-Jordan elimination, no blocking, no fusion, no reordering of the paper's steps.
// The only parallelism is an OpenMP loop over frequency bins (every quantity of the EM is
// indexed by f and the likelihood of Eq. (like) factorises over f).
//
// Two forms:
//   * conventional EM (Sec. 2): E-step Eqs. (MMSE), (postquadexp); M-step Eqs. (vupdate),
//     (Supdate), with a frame-wise inverse of v1 S1 + v2 S2;
//   * FastFCA (Sec. 3, Algorithm 1): basis change by the generalised eigenvectors P,
//     Eqs. (tildey), (MMSEtilde), (updatePhitildeeff), (updateveff), (updateStildeeff),
//     P update by Eqs. (updatePeff), (updateLambdaeff).
// The generalised eigenproblem is solved by the constructive proof of the Theorem in the
// Appendix: eigendecomposition of Psi = U Sigma U^H, then of Sigma^-1/2 U^H Phi U Sigma^-1/2.
//
// Readings where the paper is silent (each one is also applied by the CUDA path):
//   * positivity floor on v: after every v update (and on v0),
//     v <- max(v, vfloor(f)), vfloor(f) = max(1e-12 * mean_{n,m} |y_m(n,f)|^2, 1e-30);
//   * log-likelihood of iteration l is Eq. (like) evaluated at the parameters of iteration l
//     (before that iteration's update), one value per frequency;
//   * posterior-mean output: mode 0 (Algorithm 1, last step) uses the E-step of the last
//     iteration, i.e. the parameters of iteration L-1; mode 1 runs one more E-step with the
//     final parameters; with L = 0 both use the initial parameters.
//
// Layouts (row-major, complex as interleaved re/im doubles):
//   y  [F][N][M] c128      v  [2][F][N] f64      S  [2][F][M][M] c128
//   P  [F][M][M] c128      lam [F][M] f64        ll [L][F] f64      mu [F][N][M] c128
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

typedef std::complex<double> cd;
const double kPi = 3.14159265358979323846;

enum { OK = 0, ERR_ARG = 1, ERR_NOT_PD = 2, ERR_EIG_NOCONV = 3, ERR_SINGULAR = 4, ERR_NONFINITE = 5 };

// ---------------------------------------------------------------- small dense matrix helpers
// All matrices are row-major M x M complex.

void mat_copy(int M, const cd* A, cd* B) { std::memcpy(B, A, sizeof(cd) * M * M); }

void mat_identity(int M, cd* A) {
  for (int i = 0; i < M * M; ++i) A[i] = 0.0;
  for (int i = 0; i < M; ++i) A[i * M + i] = 1.0;
}

void mat_mul(int M, const cd* A, const cd* B, cd* C) {  // C = A B
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) {
      cd s = 0.0;
      for (int k = 0; k < M; ++k) s += A[i * M + k] * B[k * M + j];
      C[i * M + j] = s;
    }
}

void mat_herm(int M, const cd* A, cd* AH) {  // AH = A^H
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) AH[i * M + j] = std::conj(A[j * M + i]);
}

void mat_vec(int M, const cd* A, const cd* x, cd* y) {  // y = A x
  for (int i = 0; i < M; ++i) {
    cd s = 0.0;
    for (int k = 0; k < M; ++k) s += A[i * M + k] * x[k];
    y[i] = s;
  }
}

// Inverse by Gauss-Jordan elimination with partial pivoting. Also returns log|det A|.
int mat_inverse(int M, const cd* A, cd* Ainv, double* logabsdet) {
  std::vector<cd> a(A, A + M * M);
  mat_identity(M, Ainv);
  double ld = 0.0;
  for (int k = 0; k < M; ++k) {
    int piv = k;
    for (int i = k + 1; i < M; ++i)
      if (std::abs(a[i * M + k]) > std::abs(a[piv * M + k])) piv = i;
    if (!(std::abs(a[piv * M + k]) > 0.0)) return ERR_SINGULAR;
    if (piv != k)
      for (int j = 0; j < M; ++j) {
        std::swap(a[k * M + j], a[piv * M + j]);
        std::swap(Ainv[k * M + j], Ainv[piv * M + j]);
      }
    cd p = a[k * M + k];
    ld += std::log(std::abs(p));
    for (int j = 0; j < M; ++j) {
      a[k * M + j] /= p;
      Ainv[k * M + j] /= p;
    }
    for (int i = 0; i < M; ++i) {
      if (i == k) continue;
      cd m = a[i * M + k];
      if (m == 0.0) continue;
      for (int j = 0; j < M; ++j) {
        a[i * M + j] -= m * a[k * M + j];
        Ainv[i * M + j] -= m * Ainv[k * M + j];
      }
    }
  }
  if (logabsdet) *logabsdet = ld;
  return OK;
}

// Hermitian eigendecomposition A = V diag(w) V^H by the cyclic Jacobi method
// (Golub & Van Loan's symmetric Schur rotation, made real by a phase factor first).
// Eigenvalues ascending, eigenvectors in the columns of V.
int herm_eig(int M, const cd* A_in, cd* V, double* w) {
  std::vector<cd> A(A_in, A_in + M * M);
  for (int i = 0; i < M; ++i) {  // use the Hermitian part exactly
    A[i * M + i] = cd(std::real(A[i * M + i]), 0.0);
    for (int j = i + 1; j < M; ++j) {
      cd h = 0.5 * (A[i * M + j] + std::conj(A[j * M + i]));
      A[i * M + j] = h;
      A[j * M + i] = std::conj(h);
    }
  }
  mat_identity(M, V);
  bool converged = false;
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < M; ++i)
      for (int j = 0; j < M; ++j) {
        double a2 = std::norm(A[i * M + j]);
        tot += a2;
        if (i != j) off += a2;
      }
    if (!std::isfinite(tot)) return ERR_NONFINITE;
    if (off <= 1e-28 * tot) {  // off(A) <= 1e-14 ||A||_F
      converged = true;
      break;
    }
    for (int p = 0; p < M - 1; ++p)
      for (int q = p + 1; q < M; ++q) {
        cd apq = A[p * M + q];
        double r = std::abs(apq);
        if (r < 1e-300) continue;
        double app = std::real(A[p * M + p]), aqq = std::real(A[q * M + q]);
        double tau = (aqq - app) / (2.0 * r);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        cd e = apq / r;  // e^{i phi}
        // J acts in the (p,q) plane: J_pp = c, J_pq = s, J_qp = -s conj(e), J_qq = c conj(e).
        cd Jpp = c, Jpq = s, Jqp = -s * std::conj(e), Jqq = c * std::conj(e);
        for (int k = 0; k < M; ++k) {  // A <- A J (columns p, q)
          cd akp = A[k * M + p], akq = A[k * M + q];
          A[k * M + p] = akp * Jpp + akq * Jqp;
          A[k * M + q] = akp * Jpq + akq * Jqq;
        }
        for (int k = 0; k < M; ++k) {  // A <- J^H A (rows p, q)
          cd apk = A[p * M + k], aqk = A[q * M + k];
          A[p * M + k] = std::conj(Jpp) * apk + std::conj(Jqp) * aqk;
          A[q * M + k] = std::conj(Jpq) * apk + std::conj(Jqq) * aqk;
        }
        for (int k = 0; k < M; ++k) {  // V <- V J
          cd vkp = V[k * M + p], vkq = V[k * M + q];
          V[k * M + p] = vkp * Jpp + vkq * Jqp;
          V[k * M + q] = vkp * Jpq + vkq * Jqq;
        }
        A[p * M + q] = 0.0;
        A[q * M + p] = 0.0;
        A[p * M + p] = cd(std::real(A[p * M + p]), 0.0);
        A[q * M + q] = cd(std::real(A[q * M + q]), 0.0);
      }
  }
  if (!converged) return ERR_EIG_NOCONV;
  for (int i = 0; i < M; ++i) w[i] = std::real(A[i * M + i]);
  for (int i = 0; i < M; ++i) {  // selection sort, ascending
    int m = i;
    for (int j = i + 1; j < M; ++j)
      if (w[j] < w[m]) m = j;
    if (m != i) {
      std::swap(w[i], w[m]);
      for (int k = 0; k < M; ++k) std::swap(V[k * M + i], V[k * M + m]);
    }
  }
  return OK;
}

// Generalised eigenproblem Phi p = lambda Psi p, p_i^H Psi p_k = delta_ik (Eq. (GEVD)),
// Phi Hermitian, Psi Hermitian positive definite, by the construction in the proof of the
// Appendix's Theorem: Psi = U Sigma U^H; Phit = Sigma^-1/2 U^H Phi U Sigma^-1/2 = W Lam W^H;
// P = U Sigma^-1/2 W.
int gevd(int M, const cd* Phi, const cd* Psi, cd* P, double* lam) {
  std::vector<cd> U(M * M), W(M * M), T(M * M), UH(M * M), Phit(M * M), B(M * M);
  std::vector<double> sig(M);
  int rc = herm_eig(M, Psi, U.data(), sig.data());
  if (rc) return rc;
  for (int i = 0; i < M; ++i)
    if (!(sig[i] > 0.0)) return ERR_NOT_PD;
  for (int i = 0; i < M; ++i)  // B = U Sigma^-1/2
    for (int j = 0; j < M; ++j) B[i * M + j] = U[i * M + j] / std::sqrt(sig[j]);
  mat_herm(M, B.data(), UH.data());               // Sigma^-1/2 U^H
  mat_mul(M, UH.data(), Phi, T.data());
  mat_mul(M, T.data(), B.data(), Phit.data());   // Sigma^-1/2 U^H Phi U Sigma^-1/2
  rc = herm_eig(M, Phit.data(), W.data(), lam);
  if (rc) return rc;
  mat_mul(M, B.data(), W.data(), P);
  return OK;
}

double vfloor_of(int M, int N, const cd* yf) {  // positivity floor of v for one frequency
  double p = 0.0;
  for (int i = 0; i < N * M; ++i) p += std::norm(yf[i]);
  p /= (double)N * M;
  return std::max(1e-12 * p, 1e-30);
}

// ------------------------------------------------------------ conventional E-step (one bin)
// Eqs. (MMSE), (postquadexp): mu_j = v_j S_j Rx^-1 y, Phi_j = mu_j mu_j^H + v1 S1 Rx^-1 v2 S2,
// Rx = v1 S1 + v2 S2. Returns log det Rx and y^H Rx^-1 y for Eq. (like).
int estep_conventional(int M, const cd* y, double v1, double v2, const cd* S1, const cd* S2,
                       cd* mu1, cd* mu2, cd* Phi1, cd* Phi2, double* logdetRx, double* quad) {
  std::vector<cd> Rx(M * M), Ri(M * M), T(M * M), C(M * M), u(M), t(M);
  for (int i = 0; i < M * M; ++i) Rx[i] = v1 * S1[i] + v2 * S2[i];
  int rc = mat_inverse(M, Rx.data(), Ri.data(), logdetRx);
  if (rc) return rc;
  mat_vec(M, Ri.data(), y, u.data());  // u = Rx^-1 y
  mat_vec(M, S1, u.data(), t.data());
  for (int i = 0; i < M; ++i) mu1[i] = v1 * t[i];
  mat_vec(M, S2, u.data(), t.data());
  for (int i = 0; i < M; ++i) mu2[i] = v2 * t[i];
  mat_mul(M, Ri.data(), S2, T.data());  // Rx^-1 S2
  mat_mul(M, S1, T.data(), C.data());   // S1 Rx^-1 S2
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) {
      cd c = v1 * v2 * C[i * M + j];
      Phi1[i * M + j] = mu1[i] * std::conj(mu1[j]) + c;
      Phi2[i * M + j] = mu2[i] * std::conj(mu2[j]) + c;
    }
  cd q = 0.0;
  for (int i = 0; i < M; ++i) q += std::conj(y[i]) * u[i];
  *quad = std::real(q);
  return OK;
}

// ----------------------------------------------------------------- FastFCA E-step (one bin)
// Eqs. (tildey), (MMSEtilde), (updatePhitildeeff): yt = P^H y, d = v1 lam + v2,
// mut1 = v1 lam yt / d, mut2 = v2 yt / d, Phit_j = mut_j mut_j^H + diag(v1 v2 lam / d).
void estep_fast(int M, const cd* y, double v1, double v2, const cd* P, const double* lam, cd* yt,
                cd* mut1, cd* mut2, cd* Phit1, cd* Phit2) {
  for (int i = 0; i < M; ++i) {
    cd s = 0.0;
    for (int k = 0; k < M; ++k) s += std::conj(P[k * M + i]) * y[k];
    yt[i] = s;
  }
  for (int i = 0; i < M; ++i) {
    double d = v1 * lam[i] + v2;
    mut1[i] = v1 * lam[i] / d * yt[i];
    mut2[i] = v2 / d * yt[i];
  }
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) {
      Phit1[i * M + j] = mut1[i] * std::conj(mut1[j]);
      Phit2[i * M + j] = mut2[i] * std::conj(mut2[j]);
    }
  for (int i = 0; i < M; ++i) {
    double c = v1 * v2 * lam[i] / (v1 * lam[i] + v2);
    Phit1[i * M + i] += c;
    Phit2[i * M + i] += c;
  }
}

// ------------------------------------------------------------------ conventional EM, one f
int em_conventional_f(int M, int N, int L, const cd* yf, const double* v0_1, const double* v0_2,
                      const cd* S1_0, const cd* S2_0, int sep_mode, double* v1_out,
                      double* v2_out, cd* S1_out, cd* S2_out, double* ll_f /*stride*/,
                      int ll_stride, cd* mu1_out, cd* mu2_out) {
  const int MM = M * M;
  std::vector<cd> S1(S1_0, S1_0 + MM), S2(S2_0, S2_0 + MM), S1i(MM), S2i(MM), S1n(MM), S2n(MM);
  std::vector<cd> mu1(M), mu2(M), Phi1(MM), Phi2(MM), T(MM);
  std::vector<double> v1(v0_1, v0_1 + N), v2(v0_2, v0_2 + N);
  const double vf = vfloor_of(M, N, yf);
  for (int n = 0; n < N; ++n) {
    v1[n] = std::max(v1[n], vf);
    v2[n] = std::max(v2[n], vf);
  }
  double ldR, quad;
  int rc;
  for (int l = 0; l < L; ++l) {
    if ((rc = mat_inverse(M, S1.data(), S1i.data(), nullptr))) return rc;
    if ((rc = mat_inverse(M, S2.data(), S2i.data(), nullptr))) return rc;
    for (int i = 0; i < MM; ++i) S1n[i] = S2n[i] = 0.0;
    double ll = 0.0;
    for (int n = 0; n < N; ++n) {
      const cd* y = yf + (size_t)n * M;
      rc = estep_conventional(M, y, v1[n], v2[n], S1.data(), S2.data(), mu1.data(), mu2.data(),
                              Phi1.data(), Phi2.data(), &ldR, &quad);
      if (rc) return rc;
      ll += -M * std::log(kPi) - ldR - quad;  // Eq. (like), parameters of iteration l
      if (l == L - 1 && sep_mode == 0 && mu1_out) {
        for (int i = 0; i < M; ++i) {
          mu1_out[(size_t)n * M + i] = mu1[i];
          mu2_out[(size_t)n * M + i] = mu2[i];
        }
      }
      // Eq. (vupdate) with the old S_j.
      mat_mul(M, S1i.data(), Phi1.data(), T.data());
      cd tr1 = 0.0;
      for (int i = 0; i < M; ++i) tr1 += T[i * M + i];
      mat_mul(M, S2i.data(), Phi2.data(), T.data());
      cd tr2 = 0.0;
      for (int i = 0; i < M; ++i) tr2 += T[i * M + i];
      double nv1 = std::max(std::real(tr1) / M, vf), nv2 = std::max(std::real(tr2) / M, vf);
      // Eq. (Supdate) with the new v_j.
      for (int i = 0; i < MM; ++i) {
        S1n[i] += Phi1[i] / nv1;
        S2n[i] += Phi2[i] / nv2;
      }
      v1[n] = nv1;
      v2[n] = nv2;
    }
    for (int i = 0; i < MM; ++i) {
      S1[i] = S1n[i] / (double)N;
      S2[i] = S2n[i] / (double)N;
    }
    if (!std::isfinite(ll)) return ERR_NONFINITE;
    ll_f[(size_t)l * ll_stride] = ll;
  }
  if ((sep_mode == 1 || L == 0) && mu1_out) {  // one more E-step with the final parameters
    for (int n = 0; n < N; ++n) {
      rc = estep_conventional(M, yf + (size_t)n * M, v1[n], v2[n], S1.data(), S2.data(),
                              mu1.data(), mu2.data(), Phi1.data(), Phi2.data(), &ldR, &quad);
      if (rc) return rc;
      for (int i = 0; i < M; ++i) {
        mu1_out[(size_t)n * M + i] = mu1[i];
        mu2_out[(size_t)n * M + i] = mu2[i];
      }
    }
  }
  for (int n = 0; n < N; ++n) {
    v1_out[n] = v1[n];
    v2_out[n] = v2[n];
  }
  mat_copy(M, S1.data(), S1_out);
  mat_copy(M, S2.data(), S2_out);
  return OK;
}

// ----------------------------------------------------------------------- FastFCA, one f
// Posterior means back in the original basis: mu_j = (P^H)^-1 mut_j (Algorithm 1, output).
int fast_output(int M, int N, const cd* yf, const double* v1, const double* v2, const cd* P,
                const double* lam, cd* mu1_out, cd* mu2_out) {
  const int MM = M * M;
  std::vector<cd> PH(MM), PHi(MM), yt(M), m1(M), m2(M), Ph1(MM), Ph2(MM);
  mat_herm(M, P, PH.data());
  int rc = mat_inverse(M, PH.data(), PHi.data(), nullptr);
  if (rc) return rc;
  for (int n = 0; n < N; ++n) {
    estep_fast(M, yf + (size_t)n * M, v1[n], v2[n], P, lam, yt.data(), m1.data(), m2.data(),
               Ph1.data(), Ph2.data());
    mat_vec(M, PHi.data(), m1.data(), mu1_out + (size_t)n * M);
    mat_vec(M, PHi.data(), m2.data(), mu2_out + (size_t)n * M);
  }
  return OK;
}

int em_fast_f(int M, int N, int L, const cd* yf, const double* v0_1, const double* v0_2,
              const cd* S1_0, const cd* S2_0, int sep_mode, double* v1_out, double* v2_out,
              cd* S1_out, cd* S2_out, cd* P_out, double* lam_out, double* ll_f, int ll_stride,
              cd* mu1_out, cd* mu2_out) {
  const int MM = M * M;
  std::vector<cd> P(MM), Q(MM), Pn(MM), St1(MM), St2(MM), yt(M), m1(M), m2(M), Ph1(MM),
      Ph2(MM), Pi(MM), PiH(MM), T(MM), L1(MM);
  std::vector<double> lam(M), sig(M), v1(v0_1, v0_1 + N), v2(v0_2, v0_2 + N);
  const double vf = vfloor_of(M, N, yf);
  for (int n = 0; n < N; ++n) {
    v1[n] = std::max(v1[n], vf);
    v2[n] = std::max(v2[n], vf);
  }
  int rc = gevd(M, S1_0, S2_0, P.data(), lam.data());  // Algorithm 1, initial P and Lambda
  if (rc) return rc;
  for (int l = 0; l < L; ++l) {
    // log det S2^(l) = -log |det P^(l)|^2 since P^H S2 P = I (Eq. (GEVDmatform)).
    double ldP;
    if ((rc = mat_inverse(M, P.data(), Pi.data(), &ldP))) return rc;
    if (l == L - 1 && sep_mode == 0 && mu1_out) {
      rc = fast_output(M, N, yf, v1.data(), v2.data(), P.data(), lam.data(), mu1_out, mu2_out);
      if (rc) return rc;
    }
    for (int i = 0; i < MM; ++i) St1[i] = St2[i] = 0.0;
    double ll = 0.0;
    for (int n = 0; n < N; ++n) {
      estep_fast(M, yf + (size_t)n * M, v1[n], v2[n], P.data(), lam.data(), yt.data(),
                 m1.data(), m2.data(), Ph1.data(), Ph2.data());
      // Eq. (like) in the transformed basis: Rx = P^-H (v1 Lam + v2 I) P^-1.
      for (int i = 0; i < M; ++i) {
        double d = v1[n] * lam[i] + v2[n];
        ll -= std::log(d) + std::norm(yt[i]) / d;
      }
      ll -= M * std::log(kPi);
      // Eq. (updateveff): v1 = tr(Lam^-1 Phit1) / M, v2 = tr(Phit2) / M.
      double t1 = 0.0, t2 = 0.0;
      for (int i = 0; i < M; ++i) {
        t1 += std::real(Ph1[i * M + i]) / lam[i];
        t2 += std::real(Ph2[i * M + i]);
      }
      double nv1 = std::max(t1 / M, vf), nv2 = std::max(t2 / M, vf);
      // Eq. (updateStildeeff).
      for (int i = 0; i < MM; ++i) {
        St1[i] += Ph1[i] / nv1;
        St2[i] += Ph2[i] / nv2;
      }
      v1[n] = nv1;
      v2[n] = nv2;
    }
    ll += (double)N * 2.0 * ldP;
    if (!std::isfinite(ll)) return ERR_NONFINITE;
    ll_f[(size_t)l * ll_stride] = ll;
    for (int i = 0; i < MM; ++i) {
      St1[i] /= (double)N;
      St2[i] /= (double)N;
    }
    // Algorithm 1: GEVD of (St1, St2), then Eqs. (updatePeff), (updateLambdaeff).
    if ((rc = gevd(M, St1.data(), St2.data(), Q.data(), sig.data()))) return rc;
    mat_mul(M, P.data(), Q.data(), Pn.data());
    P = Pn;
    lam = sig;
  }
  if ((sep_mode == 1 || L == 0) && mu1_out) {
    rc = fast_output(M, N, yf, v1.data(), v2.data(), P.data(), lam.data(), mu1_out, mu2_out);
    if (rc) return rc;
  }
  // S_j from (P, Lam): P^H S1 P = Lam, P^H S2 P = I (Eqs. (Sdiag), (recoverS)).
  double ld;
  if ((rc = mat_inverse(M, P.data(), Pi.data(), &ld))) return rc;
  mat_herm(M, Pi.data(), PiH.data());
  mat_mul(M, PiH.data(), Pi.data(), S2_out);
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) L1[i * M + j] = lam[i] * Pi[i * M + j];
  mat_mul(M, PiH.data(), L1.data(), S1_out);
  for (int n = 0; n < N; ++n) {
    v1_out[n] = v1[n];
    v2_out[n] = v2[n];
  }
  if (P_out) mat_copy(M, P.data(), P_out);
  if (lam_out)
    for (int i = 0; i < M; ++i) lam_out[i] = lam[i];
  return OK;
}

bool args_ok(int M, int F, int N, int L) { return M >= 1 && M <= 16 && F >= 1 && N >= 1 && L >= 0; }

}  // namespace

extern "C" {

int oracle_openmp_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int oracle_inverse(int M, const double* A, double* Ainv, double* logabsdet) {
  return mat_inverse(M, (const cd*)A, (cd*)Ainv, logabsdet);
}

int oracle_herm_eig(int M, const double* A, double* V, double* w) {
  return herm_eig(M, (const cd*)A, (cd*)V, w);
}

int oracle_gevd(int M, const double* Phi, const double* Psi, double* P, double* lam) {
  return gevd(M, (const cd*)Phi, (const cd*)Psi, (cd*)P, lam);
}

int oracle_estep_conventional(int M, const double* y, double v1, double v2, const double* S1,
                              const double* S2, double* mu1, double* mu2, double* Phi1,
                              double* Phi2, double* loglik) {
  double ld, q;
  int rc = estep_conventional(M, (const cd*)y, v1, v2, (const cd*)S1, (const cd*)S2, (cd*)mu1,
                              (cd*)mu2, (cd*)Phi1, (cd*)Phi2, &ld, &q);
  if (loglik) *loglik = -M * std::log(kPi) - ld - q;
  return rc;
}

int oracle_estep_fast(int M, const double* y, double v1, double v2, const double* P,
                      const double* lam, double* mut1, double* mut2, double* Phit1,
                      double* Phit2) {
  std::vector<cd> yt(M);
  estep_fast(M, (const cd*)y, v1, v2, (const cd*)P, lam, yt.data(), (cd*)mut1, (cd*)mut2,
             (cd*)Phit1, (cd*)Phit2);
  return OK;
}

// Full EM runs. form 0 = conventional, 1 = FastFCA. Returns the first nonzero per-frequency
// status (lowest f) or 0. P_out / lam_out are only written by the FastFCA form.
int oracle_em(int form, int M, int F, int N, int L, const double* y, const double* v0,
              const double* S0, int sep_mode, double* v_out, double* S_out, double* ll_out,
              double* mu1_out, double* mu2_out, double* P_out, double* lam_out, int nthreads) {
  if (!args_ok(M, F, N, L) || (form != 0 && form != 1) || (sep_mode != 0 && sep_mode != 1))
    return ERR_ARG;
  const cd* yc = (const cd*)y;
  const cd* S0c = (const cd*)S0;
  cd* Sc = (cd*)S_out;
  const size_t FN = (size_t)F * N, MM = (size_t)M * M;
  std::vector<int> st(F, 0);
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
  for (int f = 0; f < F; ++f) {
    const cd* yf = yc + (size_t)f * N * M;
    cd* m1 = mu1_out ? (cd*)mu1_out + (size_t)f * N * M : nullptr;
    cd* m2 = mu2_out ? (cd*)mu2_out + (size_t)f * N * M : nullptr;
    if (form == 0)
      st[f] = em_conventional_f(M, N, L, yf, v0 + (size_t)f * N, v0 + FN + (size_t)f * N,
                                S0c + f * MM, S0c + (F + f) * MM, sep_mode, v_out + (size_t)f * N,
                                v_out + FN + (size_t)f * N, Sc + f * MM, Sc + (F + f) * MM,
                                ll_out + f, F, m1, m2);
    else
      st[f] = em_fast_f(M, N, L, yf, v0 + (size_t)f * N, v0 + FN + (size_t)f * N, S0c + f * MM,
                        S0c + (F + f) * MM, sep_mode, v_out + (size_t)f * N,
                        v_out + FN + (size_t)f * N, Sc + f * MM, Sc + (F + f) * MM,
                        P_out ? (cd*)P_out + f * MM : nullptr, lam_out ? lam_out + (size_t)f * M : nullptr,
                        ll_out + f, F, m1, m2);
  }
  (void)nthreads;
  for (int f = 0; f < F; ++f)
    if (st[f]) return st[f];
  return OK;
}

}  // extern "C"
