"""Pins of the FP64 CPU oracle against facts outside itself (no GPU needed).

Each test checks the oracle against a library routine, a closed form, a hand-derived value,
an exact invariant of the EM, or a brute-force computation on a tiny input -- never against
a retyped copy of its own formula. Together they are chosen so that a dropped term, a swapped
source index, a wrong sign or a transposed operand in any step of the oracle fails at least
one of them.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.stats as sst

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")


def rand_hpd(rng, M, diag=0.5):
    A = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    return A @ A.conj().T / M + diag * np.eye(M)


def rand_herm(rng, M):
    A = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    return 0.5 * (A + A.conj().T)


def rand_problem(rng, M, F, N):
    y = (rng.standard_normal((F, N, M)) + 1j * rng.standard_normal((F, N, M))) / np.sqrt(2)
    y *= np.exp(0.7 * rng.standard_normal((F, N, 1)))
    S0 = np.stack([[rand_hpd(rng, M) for _ in range(F)] for _ in range(2)])
    v0 = np.exp(0.5 * rng.standard_normal((2, F, N)))
    return y, v0, S0


# ----------------------------------------------------------------- linear algebra (library)

@pytest.mark.parametrize("M", [1, 2, 3, 5, 8])
def test_inverse_matches_numpy(M):
    rng = np.random.default_rng(M)
    A = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M)) + 2 * np.eye(M)
    Ai, ld = oracle.inverse(A)
    np.testing.assert_allclose(Ai, np.linalg.inv(A), rtol=0, atol=1e-12 * np.abs(Ai).max())
    assert abs(ld - np.linalg.slogdet(A)[1]) < 1e-12 * max(1.0, abs(ld))


@pytest.mark.parametrize("M", [1, 2, 3, 4, 7, 8])
def test_herm_eig_matches_numpy(M):
    rng = np.random.default_rng(10 + M)
    A = rand_herm(rng, M)
    V, w = oracle.herm_eig(A)
    np.testing.assert_allclose(w, np.linalg.eigvalsh(A), atol=1e-12 * np.abs(w).max())
    np.testing.assert_allclose(V.conj().T @ V, np.eye(M), atol=1e-12)
    np.testing.assert_allclose(A @ V, V * w, atol=1e-11 * np.abs(A).max())


@pytest.mark.parametrize("M", [1, 2, 3, 4, 6, 8])
def test_gevd_matches_scipy_and_diagonalises(M):
    """Eq. (GEVD) / (GEVDmatform): S1 P = S2 P Lam, P^H S2 P = I, and Eq. (sigcovdiag)."""
    rng = np.random.default_rng(20 + M)
    S1, S2 = rand_hpd(rng, M), rand_hpd(rng, M)
    P, lam = oracle.gevd(S1, S2)
    np.testing.assert_allclose(lam, sla.eigh(S1, S2, eigvals_only=True), rtol=1e-11)
    np.testing.assert_allclose(P.conj().T @ S2 @ P, np.eye(M), atol=1e-12)
    np.testing.assert_allclose(P.conj().T @ S1 @ P, np.diag(lam), atol=1e-11 * lam.max())
    np.testing.assert_allclose(S1 @ P, S2 @ P * lam, atol=1e-11 * np.abs(S1).max() * np.abs(P).max())


def test_gevd_hand_examples():
    g = json.load(open(GOLDEN))
    for key in ("gevd_2x2", "gevd_2x2_scaled"):
        case = g[key]
        _, lam = oracle.gevd(np.array(case["S1"], complex), np.array(case["S2"], complex))
        np.testing.assert_allclose(lam, case["lambda"], rtol=1e-14)


def test_gevd_indefinite_psi_is_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.gevd(np.eye(2, dtype=complex), np.diag([1.0, -1.0]).astype(complex))


# ------------------------------------------------------------------------------- E-steps

def gaussian_posterior(y, C1, C2):
    """Posterior of x1 given y = x1 + x2, x_j ~ CN(0, C_j): textbook Gaussian conditioning
    (mean C1 (C1+C2)^-1 y, covariance C1 - C1 (C1+C2)^-1 C1)."""
    R = C1 + C2
    K1 = C1 @ np.linalg.inv(R)
    K2 = C2 @ np.linalg.inv(R)
    m1, m2 = K1 @ y, K2 @ y
    P1 = np.outer(m1, m1.conj()) + C1 - K1 @ C1
    P2 = np.outer(m2, m2.conj()) + C2 - K2 @ C2
    return m1, m2, P1, P2


def complex_gauss_logpdf(y, R):
    """log CN(y; 0, R) through the equivalent real 2M-dimensional Gaussian (scipy)."""
    M = y.shape[0]
    z = np.concatenate([y.real, y.imag])
    Sig = 0.5 * np.block([[R.real, -R.imag], [R.imag, R.real]])
    return sst.multivariate_normal(mean=np.zeros(2 * M), cov=Sig).logpdf(z)


@pytest.mark.parametrize("M", [1, 2, 3, 4, 8])
def test_estep_conventional_is_gaussian_conditioning(M):
    """Eqs. (MMSE), (postquadexp) and the Eq. (like) term vs the textbook posterior."""
    rng = np.random.default_rng(30 + M)
    S1, S2 = rand_hpd(rng, M), rand_hpd(rng, M)
    v1, v2 = 0.7, 1.9
    y = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    mu1, mu2, Phi1, Phi2, ll = oracle.estep_conventional(y, v1, v2, S1, S2)
    m1, m2, P1, P2 = gaussian_posterior(y, v1 * S1, v2 * S2)
    for a, b in ((mu1, m1), (mu2, m2), (Phi1, P1), (Phi2, P2)):
        np.testing.assert_allclose(a, b, atol=1e-12 * np.abs(b).max())
    assert abs(ll - complex_gauss_logpdf(y, v1 * S1 + v2 * S2)) < 1e-11 * abs(ll)


def test_estep_scalar_hand_examples():
    g = json.load(open(GOLDEN))
    c = g["scalar_em_one_step"]
    one = np.ones((1, 1), complex)
    mu1, mu2, Phi1, Phi2, ll = oracle.estep_conventional(
        np.array([complex(*c["y"])]), c["v1"], c["v2"], c["S1"] * one, c["S2"] * one)
    assert abs(mu1[0] - c["mu1"]) < 1e-15 and abs(mu2[0] - c["mu2"]) < 1e-15
    assert abs(Phi1[0, 0] - c["Phi1"]) < 1e-15 and abs(Phi2[0, 0] - c["Phi2"]) < 1e-15
    assert abs(ll - c["loglik"]) < 1e-14
    c = g["scalar_em_asymmetric"]
    mu1, mu2, Phi1, Phi2, _ = oracle.estep_conventional(
        np.array([complex(*c["y"])]), c["v1"], c["v2"], c["S1"] * one, c["S2"] * one)
    assert abs(mu1[0] - complex(*c["mu1"])) < 1e-14 and abs(mu2[0] - complex(*c["mu2"])) < 1e-14
    assert abs(Phi1[0, 0] - c["Phi1"]) < 1e-14 and abs(Phi2[0, 0] - c["Phi2"]) < 1e-14


@pytest.mark.parametrize("M", [1, 2, 4, 7])
def test_estep_fast_is_transformed_posterior(M):
    """Eqs. (tildemu), (tildePhi), (MMSEtilde), (updatePhitildeeff) with P from scipy."""
    rng = np.random.default_rng(40 + M)
    S1, S2 = rand_hpd(rng, M), rand_hpd(rng, M)
    lam, P = sla.eigh(S1, S2)          # P^H S2 P = I, P^H S1 P = diag(lam)
    v1, v2 = 1.3, 0.4
    y = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    mt1, mt2, Pt1, Pt2 = oracle.estep_fast(y, v1, v2, P, lam)
    m1, m2, P1, P2 = gaussian_posterior(y, v1 * S1, v2 * S2)
    PH = P.conj().T
    for a, b in ((mt1, PH @ m1), (mt2, PH @ m2), (Pt1, PH @ P1 @ P), (Pt2, PH @ P2 @ P)):
        np.testing.assert_allclose(a, b, atol=1e-11 * np.abs(b).max())


# ------------------------------------------------------------------------- M-step, EM run

@pytest.mark.parametrize("form", ["conventional", "fast"])
def test_mstep_maximises_expected_complete_loglik(form):
    """Eqs. (vupdate), (Supdate): v_j^(1) maximises Q over v with the old S_j, and S_j^(1)
    maximises Q over S with the new v_j (generalised EM), checked by finite differences of
    Q(v, S) = sum_n [-M log v - log det S - tr(S^-1 Phi_j) / v], with Phi_j from the
    brute-force Gaussian posterior."""
    rng = np.random.default_rng(50)
    M, N = 3, 5
    y, v0, S0 = rand_problem(rng, M, 1, N)
    out = oracle.em(form, y, v0, S0, 1)
    for j in range(2):
        Sj, Snew, vnew = S0[j, 0], out["S"][j, 0], out["v"][j, 0]
        Phis = [gaussian_posterior(y[0, n], v0[0, 0, n] * S0[0, 0], v0[1, 0, n] * S0[1, 0])[2 + j]
                for n in range(N)]
        Sji = np.linalg.inv(Sj)
        for n in range(N):
            t = np.real(np.trace(Sji @ Phis[n]))
            q = lambda v: -M * np.log(v) - t / v
            h = 1e-5 * vnew[n]
            dq = (q(vnew[n] + h) - q(vnew[n] - h)) / (2 * h)
            assert abs(dq) * vnew[n] < 1e-6 * M
            assert q(vnew[n]) >= max(q(vnew[n] * 1.01), q(vnew[n] * 0.99))

        def Q(S):
            Si = np.linalg.inv(S)
            return sum(-np.linalg.slogdet(S)[1] - np.real(np.trace(Si @ Phis[n])) / vnew[n]
                       for n in range(N))
        q0 = Q(Snew)
        for _ in range(4):
            H = rand_herm(rng, M)
            eps = 1e-5 * np.abs(Snew).max()
            d = (Q(Snew + eps * H) - Q(Snew - eps * H)) / (2 * eps)
            assert abs(d) < 1e-5 * N * M
            assert q0 >= Q(Snew + 0.05 * np.abs(Snew).max() * H / np.abs(H).max())


def test_scalar_em_hand_examples():
    """One EM iteration at M = 1, N = 1 against the hand-derived values, both forms."""
    g = json.load(open(GOLDEN))
    for key in ("scalar_em_one_step", "scalar_em_asymmetric"):
        c = g[key]
        y = np.array([[[complex(*c["y"])]]])
        v0 = np.array([[[c["v1"]]], [[c["v2"]]]])
        S0 = np.array([[[[c["S1"]]]], [[[c["S2"]]]]], complex)
        for form in ("conventional", "fast"):
            out = oracle.em(form, y, v0, S0, 1)
            assert abs(out["v"][0, 0, 0] - c["v1_new"]) < 1e-14
            assert abs(out["v"][1, 0, 0] - c["v2_new"]) < 1e-14
            assert abs(out["S"][0, 0, 0, 0] - c["S1_new"]) < 1e-13
            assert abs(out["S"][1, 0, 0, 0] - c["S2_new"]) < 1e-13
            if "loglik" in c:
                assert abs(out["ll"][0, 0] - c["loglik"]) < 1e-13


def scalar_em(y, v1, v2, s1, s2, iters):
    """FCA with M = 1 written out directly: a scalar Wiener-filter EM (independent of the
    oracle's matrix code)."""
    ll = []
    for _ in range(iters):
        r = v1 * s1 + v2 * s2
        ll.append(np.sum(-np.log(np.pi) - np.log(r) - np.abs(y) ** 2 / r))
        g1, g2 = v1 * s1 / r, v2 * s2 / r
        post = v1 * s1 * v2 * s2 / r
        p1 = np.abs(g1 * y) ** 2 + post
        p2 = np.abs(g2 * y) ** 2 + post
        v1, v2 = p1 / s1, p2 / s2
        s1, s2 = np.mean(p1 / v1), np.mean(p2 / v2)
    return v1, v2, s1, s2, np.array(ll)


@pytest.mark.parametrize("form", ["conventional", "fast"])
def test_scalar_case_is_wiener_em(form):
    rng = np.random.default_rng(60)
    N = 50
    y, v0, S0 = rand_problem(rng, 1, 1, N)
    out = oracle.em(form, y, v0, S0, 6)
    v1, v2, s1, s2, ll = scalar_em(y[0, :, 0], v0[0, 0], v0[1, 0], S0[0, 0, 0, 0].real,
                                   S0[1, 0, 0, 0].real, 6)
    np.testing.assert_allclose(out["v"][0, 0], v1, rtol=1e-11)
    np.testing.assert_allclose(out["v"][1, 0], v2, rtol=1e-11)
    assert abs(out["S"][0, 0, 0, 0] - s1) < 1e-11 * s1
    assert abs(out["S"][1, 0, 0, 0] - s2) < 1e-11 * s2
    np.testing.assert_allclose(out["ll"][:, 0], ll, rtol=1e-12)


@pytest.mark.parametrize("M,F,N,L", [(2, 3, 4, 5), (3, 2, 7, 4), (4, 3, 20, 6), (8, 2, 30, 4),
                                     (1, 4, 9, 5), (5, 1, 11, 3)])
def test_fast_equals_conventional(M, F, N, L):
    """FastFCA is strictly equivalent to conventional EM (Sec. 3 derivations, proof of
    Eqs. (updatePeff), (updateLambdaeff)): same v, S, log-likelihood and posterior means."""
    rng = np.random.default_rng(70 + M * 13 + N)
    y, v0, S0 = rand_problem(rng, M, F, N)
    a = oracle.em("conventional", y, v0, S0, L)
    b = oracle.em("fast", y, v0, S0, L)
    np.testing.assert_allclose(b["v"], a["v"], rtol=1e-9)
    for j in range(2):
        for f in range(F):
            np.testing.assert_allclose(b["S"][j, f], a["S"][j, f], atol=1e-9 * np.abs(a["S"][j, f]).max())
    np.testing.assert_allclose(b["ll"], a["ll"], rtol=1e-10)
    scale = np.linalg.norm(y, axis=2, keepdims=True)
    assert np.max(np.abs(b["mu1"] - a["mu1"]) / scale) < 1e-9
    assert np.max(np.abs(b["mu2"] - a["mu2"]) / scale) < 1e-9


@pytest.mark.parametrize("form", ["conventional", "fast"])
def test_loglik_is_monotone(form):
    """EM never decreases the likelihood of Eq. (like) (Sec. 2)."""
    c, mix, v0, S0 = synth.make_config("small", F=12)
    out = oracle.em(form, mix["y"], v0, S0, 20)
    ll = out["ll"]
    assert np.all(np.diff(ll, axis=0) >= -1e-10 * np.abs(ll[1:]))


def test_loglik_matches_scipy_density():
    """Iteration-0 log-likelihood = sum of scipy multivariate normal log-densities."""
    rng = np.random.default_rng(80)
    M, F, N = 3, 2, 4
    y, v0, S0 = rand_problem(rng, M, F, N)
    for form in ("conventional", "fast"):
        out = oracle.em(form, y, v0, S0, 1)
        for f in range(F):
            ref = sum(complex_gauss_logpdf(y[f, n], v0[0, f, n] * S0[0, f] + v0[1, f, n] * S0[1, f])
                      for n in range(N))
            assert abs(out["ll"][0, f] - ref) < 1e-11 * abs(ref)


@pytest.mark.parametrize("form", ["conventional", "fast"])
def test_posterior_means_add_up_to_mixture(form):
    """y = x1 + x2 (Sec. 2) implies mu1 + mu2 = y."""
    rng = np.random.default_rng(90)
    y, v0, S0 = rand_problem(rng, 4, 3, 10)
    out = oracle.em(form, y, v0, S0, 3)
    err = np.abs(out["mu1"] + out["mu2"] - y) / np.linalg.norm(y, axis=2, keepdims=True)
    assert err.max() < 1e-12


def test_trace_invariant_of_the_m_step():
    """Eqs. (vupdate), (Supdate) give tr(S_j^(l)^-1 S_j^(l+1)) = M exactly."""
    rng = np.random.default_rng(100)
    M, F, N = 4, 3, 15
    y, v0, S0 = rand_problem(rng, M, F, N)
    a = oracle.em("conventional", y, v0, S0, 1)
    b = oracle.em("conventional", y, a["v"], a["S"], 1)
    for S_old, S_new in ((S0, a["S"]), (a["S"], b["S"])):
        for j in range(2):
            for f in range(F):
                t = np.trace(np.linalg.solve(S_old[j, f], S_new[j, f]))
                assert abs(t - M) < 1e-11 * M


def test_fast_P_jointly_diagonalises_conventional_S():
    """The FastFCA basis after L iterations diagonalises the conventional S^(L) (Eqs.
    (GEVDmatform), (sigcovdiag)): the two runs share one trajectory."""
    c, mix, v0, S0 = synth.make_config("small", F=6)
    a = oracle.em("conventional", mix["y"], v0, S0, 10)
    b = oracle.em("fast", mix["y"], v0, S0, 10)
    for f in range(6):
        P = b["P"][f]
        D2 = P.conj().T @ a["S"][1, f] @ P
        D1 = P.conj().T @ a["S"][0, f] @ P
        np.testing.assert_allclose(D2, np.eye(2), atol=1e-9)
        np.testing.assert_allclose(D1, np.diag(b["lam"][f]), atol=1e-9 * b["lam"][f].max())


@pytest.mark.parametrize("form", ["conventional", "fast"])
def test_separation_modes(form):
    """Algorithm 1's output uses the parameters of iteration L-1: mode 0 after L iterations
    equals mode 1 (one E-step with the final parameters) after L-1 iterations; mode 1 equals
    a brute-force posterior at the final parameters."""
    rng = np.random.default_rng(110)
    y, v0, S0 = rand_problem(rng, 3, 2, 6)
    a = oracle.em(form, y, v0, S0, 4, sep_mode=0)
    b = oracle.em(form, y, v0, S0, 3, sep_mode=1)
    np.testing.assert_allclose(a["mu1"], b["mu1"], atol=1e-10)
    c = oracle.em(form, y, v0, S0, 4, sep_mode=1)
    for f in range(2):
        for n in range(6):
            m1, m2, _, _ = gaussian_posterior(y[f, n], c["v"][0, f, n] * c["S"][0, f],
                                              c["v"][1, f, n] * c["S"][1, f])
            assert np.abs(c["mu1"][f, n] - m1).max() < 1e-9 * np.linalg.norm(y[f, n])
            assert np.abs(c["mu2"][f, n] - m2).max() < 1e-9 * np.linalg.norm(y[f, n])


def test_zero_iterations_and_positivity_floor():
    """L = 0 leaves the parameters as given (after the v floor) and separates with them; a
    silent frame drives v to the floor max(1e-12 mean|y|^2, 1e-30) without NaN."""
    rng = np.random.default_rng(120)
    y, v0, S0 = rand_problem(rng, 2, 2, 6)
    out = oracle.em("fast", y, v0, S0, 0)
    np.testing.assert_allclose(out["v"], v0, rtol=0)
    y[:, 2, :] = 0.0
    for form in ("conventional", "fast"):
        out = oracle.em(form, y, v0, S0, 60)
        vf = np.maximum(1e-12 * np.mean(np.abs(y) ** 2, axis=(1, 2)), 1e-30)
        assert np.all(out["v"] >= vf[None, :, None])
        assert np.all(np.isfinite(out["v"])) and np.all(np.isfinite(out["ll"]))
        assert np.all(out["v"][:, :, 2] < 1e-9 * out["v"].max())
