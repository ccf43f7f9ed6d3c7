"""Pins of the FP64 oracle to things other than itself: brute force, the
paper's B x B form (Thm. 1), closed forms, invariants, hand-derived worked
examples and optimality conditions.  CPU only.

Notation: Hm is the U x B channel; the arrays store it as H[b][u] = Hm[u][b].
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1804_10987_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def cplx_randn(g, *shape):
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)) / np.sqrt(2)


def random_problem(seed, n_sc, B, U, K):
    g = synth.rng(seed)
    H = cplx_randn(g, n_sc, B, U) / np.sqrt(B)
    S = cplx_randn(g, n_sc, K, U)
    return H, S


def thm1_bxb(Hm, kappa, rho2, Es):
    """Thm. 1 straight from its B x B statement (numpy LAPACK, not the oracle):
    Q = (Hm^H Hm + kappa I_B)^{-1} Hm^H, beta = sqrt(tr(Q^H Q) Es / rho^2)."""
    B = Hm.shape[1]
    Q = np.linalg.solve(Hm.conj().T @ Hm + kappa * np.eye(B), Hm.conj().T)
    beta = np.sqrt(np.trace(Q.conj().T @ Q).real * Es / rho2)
    return Q, beta


def precoder_matrix(H, cluster_sizes, mode, **kw):
    """Extract P (B x U) from the oracle by precoding s_k = e_k (K = U): the
    oracle is linear in s, so X[k] = P e_k."""
    n_sc, B, U = H.shape
    S = np.broadcast_to(np.eye(U, dtype=np.complex128), (n_sc, U, U)).copy()
    out = oracle.precode(H, S, cluster_sizes, mode, **kw)
    return np.swapaxes(out["X"], 1, 2), out  # [n_sc][B][U]


# --- (i) Gram sum ---------------------------------------------------------------

def test_gram_sum_equals_full_gram_bruteforce():
    H, S = random_problem(1, 3, 13, 5, 2)
    cs = [6, 4, 3]
    out = oracle.precode(H, S, cs, "wf", N0=0.3)
    for n in range(3):
        Hm = H[n].T
        full = np.einsum("ub,vb->uv", Hm, Hm.conj())  # brute force, numpy
        np.testing.assert_allclose(out["G"][n], full, rtol=0, atol=1e-13)
        off = np.cumsum([0] + cs)
        for c in range(3):
            Hc = Hm[:, off[c]:off[c + 1]]
            np.testing.assert_allclose(out["Gloc"][c, n], Hc @ Hc.conj().T, atol=1e-13)
        np.testing.assert_allclose(out["Gloc"][:, n].sum(0), full, atol=1e-13)


def test_gram_antenna_side():
    H, _ = random_problem(2, 1, 7, 4, 1)
    Gp = oracle.gram_antenna(H[0], 2, 6)
    Hc = H[0].T[:, 2:6]
    np.testing.assert_allclose(Gp, Hc.conj().T @ Hc, atol=1e-14)


# --- Cholesky / inverse -----------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 8, 17])
def test_inverse_identity(n):
    g = synth.rng(100 + n)
    M = cplx_randn(g, n, n + 3)
    A = M @ M.conj().T + 0.1 * np.eye(n)
    st, L = oracle.cholesky(A)
    assert st == oracle.OK
    np.testing.assert_allclose(L @ L.conj().T, A, atol=1e-12)
    assert np.allclose(np.triu(L, 1), 0)
    T = oracle.inverse_from_cholesky(L)
    assert np.abs(A @ T - np.eye(n)).max() < 1e-12


def test_inverse_closed_forms():
    st, L = oracle.cholesky(np.array([[4.0 + 0j]]))
    assert st == 0 and abs(L[0, 0] - 2) < 1e-15
    assert abs(oracle.inverse_from_cholesky(L)[0, 0] - 0.25) < 1e-15
    a, b, d = 3.0, 1.0 - 2.0j, 4.0
    A = np.array([[a, b], [np.conj(b), d]])
    det = a * d - abs(b) ** 2
    ref = np.array([[d, -b], [-np.conj(b), a]]) / det  # textbook 2x2 inverse
    st, L = oracle.cholesky(A)
    np.testing.assert_allclose(oracle.inverse_from_cholesky(L), ref, atol=1e-15)


def test_cholesky_rejects_indefinite():
    st, _ = oracle.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]], dtype=complex))
    assert st == oracle.NOT_PD


# --- Lemma 1 / Thm. 1 -------------------------------------------------------------

@pytest.mark.parametrize("U,B,kappa", [(1, 4, 0.7), (3, 9, 0.3), (6, 6, 2.0), (5, 40, 12.0)])
def test_lemma1_matches_thm1_bxb(U, B, kappa):
    g = synth.rng(7 * U + B)
    Hm = cplx_randn(g, U, B) / np.sqrt(B)
    G = oracle.gram(Hm.T)
    A = G + kappa * np.eye(U)
    st, L = oracle.cholesky(A)
    T = oracle.inverse_from_cholesky(L)
    Q, _ = thm1_bxb(Hm, kappa, 1.0, 1.0)
    t_def = np.trace(Q.conj().T @ Q).real
    assert abs(oracle.t_lemma(T, kappa) - t_def) < 1e-12 * max(1, t_def)
    assert abs(oracle.t_direct(T, G) - t_def) < 1e-12 * max(1, t_def)


def test_u1_closed_form():
    """U = 1: A^{-1} = 1/(g + kappa), t = g/(g + kappa)^2, and the WF reduces to
    x = conj(h) s rho / (sqrt(Es) ||h||), independent of kappa."""
    g = synth.rng(11)
    B = 9
    h = cplx_randn(g, B)
    H = h.reshape(1, B, 1)
    S = np.array([[[0.3 - 0.8j]]])
    for mode, N0 in (("wf", 0.4), ("zf", 0.0), ("wf", 5.0)):
        out = oracle.precode(H, S, [B], mode, N0=N0, rho2=2.0, Es=1.5)
        gg = np.vdot(h, h).real
        kappa = 1 * N0 / 2.0 if mode == "wf" else 0.0
        assert abs(out["t"][0] - gg / (gg + kappa) ** 2) < 1e-14
        x = np.conj(h) * S[0, 0, 0] * np.sqrt(2.0) / (np.sqrt(1.5) * np.sqrt(gg))
        np.testing.assert_allclose(out["X"][0, 0], x, atol=1e-14)


# --- PD-WF == centralized WF (Sec. III-B) -------------------------------------------

@pytest.mark.parametrize("cs", [[4, 4], [3, 5, 2, 6], [16]])
def test_pd_wf_equals_centralized_thm1(cs):
    B = sum(cs)
    U, K, N0, rho2, Es = 3, 4, 0.2, 1.7, 1.0
    H, S = random_problem(sum(cs) * 31, 2, B, U, K)
    out = oracle.precode(H, S, cs, "wf", N0=N0, rho2=rho2, Es=Es)
    for n in range(2):
        Hm = H[n].T
        Q, beta = thm1_bxb(Hm, U * N0 / rho2, rho2, Es)
        assert abs(out["scale"][n] - 1 / beta) < 1e-12 / beta
        for k in range(K):
            x_ref = Q @ S[n, k] / beta
            np.testing.assert_allclose(out["X"][n, k], x_ref, atol=1e-12)
            # received signal: sum_c H_c x_c = H P s
            np.testing.assert_allclose(Hm @ out["X"][n, k], Hm @ x_ref, atol=1e-12)


# --- (ii) noise-free ZF ---------------------------------------------------------------

def test_zf_noise_free_inverts_channel():
    U, B, K = 6, 20, 5
    H, S = random_problem(5, 3, B, U, K)
    out = oracle.precode(H, S, [10, 10], "zf", N0=0.0)
    for n in range(3):
        Hm = H[n].T
        for k in range(K):
            np.testing.assert_allclose(Hm @ out["X"][n, k], out["scale"][n] * S[n, k],
                                       atol=1e-12)


def test_zf_singular_when_fewer_antennas_than_users():
    H, S = random_problem(6, 1, 3, 5, 2)
    out = oracle.precode(H, S, [3], "zf", N0=0.0)
    assert out["status"][0] == oracle.NOT_PD
    assert np.all(out["X"] == 0)


# --- (iii) FD-WF with one cluster -------------------------------------------------------

def test_fd_single_cluster_tau1_equals_wf():
    U, B, K = 4, 12, 3
    H, S = random_problem(9, 2, B, U, K)
    wf = oracle.precode(H, S, [B], "wf", N0=0.3)
    fd = oracle.precode(H, S, [B], "fdwf", N0=0.3, tau=1.0)
    np.testing.assert_allclose(fd["X"], wf["X"], atol=1e-13)


def test_fd_single_cluster_tau_equals_wf_at_scaled_noise():
    U, B, K, tau = 4, 12, 3, 0.125
    H, S = random_problem(10, 2, B, U, K)
    wf = oracle.precode(H, S, [B], "wf", N0=0.3 * tau)
    fd = oracle.precode(H, S, [B], "fdwf", N0=0.3, tau=tau)
    np.testing.assert_allclose(fd["X"], wf["X"], atol=1e-13)


# --- (iv) power constraint -----------------------------------------------------------

@pytest.mark.parametrize("mode", ["wf", "zf", "fdwf", "mrt"])
def test_power_constraint_exact(mode):
    U, cs = 4, [5, 3, 8]
    H, _ = random_problem(12, 3, sum(cs), U, 1)
    P, out = precoder_matrix(H, cs, mode, N0=0.25, rho2=1.3, Es=1.0, tau=0.125)
    off = np.cumsum([0] + cs)
    for n in range(3):
        # E_s ||x||^2 = Es ||P||_F^2 for E[s s^H] = Es I (Eq. (3))
        assert abs(np.linalg.norm(P[n]) ** 2 - 1.3) < 1e-12
        if mode == "fdwf":
            for c in range(3):
                pc = P[n, off[c]:off[c + 1]]
                assert abs(np.linalg.norm(pc) ** 2 - 1.3 / 3) < 1e-12


def test_power_sample_mean_statistical():
    """E_s ||x||^2 = rho^2 holds as an average over symbols (Eq. (3))."""
    p = synth.make_problem(8, 64, 2, 4, 4000, 16, 10.0, seed=77)
    out = oracle.precode(p.H, p.S, p.cluster_sizes, "wf", N0=p.N0)
    m = np.mean(np.sum(np.abs(out["X"]) ** 2, axis=2))
    assert abs(m - 1.0) < 0.02


# --- optimality (Appendix A) ---------------------------------------------------------

def test_kkt_conditions_with_corrected_multiplier():
    """Eq. (18): beta^2 H^H H P + lambda P = beta H^H with lambda = beta^2 kappa
    (the multiplier of Eq. (22) must carry a beta^2 for Thm. 1 to follow), and
    Eq. (19): beta tr(P^H H^H H P) + beta U N0 / Es = tr(H^H P^H)."""
    U, B, N0, rho2, Es = 3, 7, 0.4, 1.0, 1.0
    H, _ = random_problem(13, 1, B, U, 1)
    P, out = precoder_matrix(H, [B], "wf", N0=N0, rho2=rho2, Es=Es)
    P = P[0]
    Hm = H[0].T
    beta = 1.0 / out["scale"][0]
    kappa = U * N0 / rho2
    lam = beta ** 2 * kappa
    r = beta ** 2 * Hm.conj().T @ Hm @ P + lam * P - beta * Hm.conj().T
    assert np.abs(r).max() < 1e-12
    lhs = beta * np.trace(P.conj().T @ Hm.conj().T @ Hm @ P) + beta * U * N0 / Es
    rhs = np.trace(Hm.conj().T @ P.conj().T)
    assert abs(lhs - rhs) < 1e-12


def mse_opt_beta(Hm, P, N0, Es):
    """min over complex beta of Es||I - beta Hm P||_F^2 + |beta|^2 U N0."""
    U = Hm.shape[0]
    M = Hm @ P
    trm = np.trace(M)
    return Es * U - Es ** 2 * abs(trm) ** 2 / (Es * np.linalg.norm(M) ** 2 + U * N0)


def test_mse_increases_under_feasible_perturbations():
    U, B, N0, rho2, Es = 3, 6, 0.3, 1.0, 1.0
    H, _ = random_problem(14, 1, B, U, 1)
    P, _ = precoder_matrix(H, [B], "wf", N0=N0, rho2=rho2, Es=Es)
    P, Hm = P[0], H[0].T
    m0 = mse_opt_beta(Hm, P, N0, Es)
    g = synth.rng(15)
    for eps in (1e-1, 1e-2, 1e-3):
        for _ in range(40):
            P2 = P + eps * cplx_randn(g, B, U)
            P2 *= np.sqrt(rho2 / Es) / np.linalg.norm(P2)
            assert mse_opt_beta(Hm, P2, N0, Es) >= m0 - 1e-13


def test_bruteforce_mse_minimizer_matches():
    """U = 2, B = 3: numerically minimize the MSE over P with ||P||_F^2 =
    rho^2/Es (the problem of Sec. II-B) and compare with the oracle's WF."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    U, B, N0, rho2, Es = 2, 3, 0.5, 1.0, 1.0
    H, _ = random_problem(16, 1, B, U, 1)
    P, _ = precoder_matrix(H, [B], "wf", N0=N0, rho2=rho2, Es=Es)
    P, Hm = P[0], H[0].T

    def unpack(v):
        Pv = (v[:B * U] + 1j * v[B * U:]).reshape(B, U)
        return Pv * np.sqrt(rho2 / Es) / np.linalg.norm(Pv)

    best = None
    g = synth.rng(17)
    for _ in range(6):
        v0 = g.standard_normal(2 * B * U)
        res = scipy_opt.minimize(lambda v: mse_opt_beta(Hm, unpack(v), N0, Es), v0,
                                 method="BFGS", options=dict(gtol=1e-12, maxiter=5000))
        if best is None or res.fun < best.fun:
            best = res
    Pb = unpack(best.x)
    ph = np.vdot(Pb, P)  # the MSE is blind to a common phase of P
    Pb = Pb * ph / abs(ph)
    assert abs(best.fun - mse_opt_beta(Hm, P, N0, Es)) < 1e-9
    np.testing.assert_allclose(Pb, P, atol=1e-4)


# --- FD-WF forms --------------------------------------------------------------------

@pytest.mark.parametrize("cs", [[2, 3, 7], [5, 5], [1, 11]])
def test_fd_two_forms_agree(cs):
    U, K = 5, 3
    H, S = random_problem(18 + len(cs), 2, sum(cs), U, K)
    a = oracle.precode(H, S, cs, "fdwf", N0=0.2, tau=0.125, fd_form=oracle.FORM_UXU)
    b = oracle.precode(H, S, cs, "fdwf", N0=0.2, tau=0.125, fd_form=oracle.FORM_BCXBC)
    np.testing.assert_allclose(a["X"], b["X"], atol=1e-12)
    np.testing.assert_allclose(a["scale"], b["scale"], rtol=1e-12)
    # in each form, t and the alternative formula agree
    np.testing.assert_allclose(a["t"], a["t_alt"], rtol=1e-11)
    np.testing.assert_allclose(b["t"], b["t_alt"], rtol=1e-11)


def test_fd_cluster_is_local_wf():
    """Each FD-WF cluster is a WF precoder on (H_c, rho^2/C) with kappa_c."""
    U, cs, N0, tau = 3, [6, 4], 0.2, 0.5
    H, S = random_problem(21, 1, 10, U, 2)
    fd = oracle.precode(H, S, cs, "fdwf", N0=N0, tau=tau)
    off = np.cumsum([0] + cs)
    for c in range(2):
        Hm = H[0].T[:, off[c]:off[c + 1]]
        rho2c = 1.0 / 2
        kappa = tau * U * N0 / rho2c
        Q, beta = thm1_bxb(Hm, kappa, rho2c, 1.0)
        for k in range(2):
            np.testing.assert_allclose(fd["X"][0, k, off[c]:off[c + 1]], Q @ S[0, k] / beta,
                                       atol=1e-12)


# --- worked examples ------------------------------------------------------------------

def _gold():
    with open(os.path.join(GOLD, "hand_2x2.json")) as f:
        return json.load(f)


def _c(a):
    a = np.asarray(a, dtype=float)
    return a[..., 0] + 1j * a[..., 1]


@pytest.mark.parametrize("case", ["wf", "zf", "fdwf_tau1_c2", "mrt"])
def test_hand_worked_examples(case):
    d = _gold()
    H = _c(d["H_BU"])[None]
    S = _c(d["S_KU"])[None]
    e = d[case]
    if case == "wf":
        out = oracle.precode(H, S, [2], "wf", N0=d["N0"], rho2=d["rho2"], Es=d["Es"])
    elif case == "zf":
        out = oracle.precode(H, S, [2], "zf", N0=0.0, rho2=d["rho2"], Es=d["Es"])
    elif case == "mrt":
        out = oracle.precode(H, S, [2], "mrt", N0=d["N0"], rho2=d["rho2"], Es=d["Es"])
    else:
        out = oracle.precode(H, S, e["cluster_sizes"], "fdwf", N0=d["N0"], rho2=d["rho2"],
                             Es=d["Es"], tau=e["tau"])
    np.testing.assert_allclose(out["t"][0], e["t"], rtol=1e-14)
    np.testing.assert_allclose(out["scale"][0], e["scale"], rtol=1e-14)
    np.testing.assert_allclose(out["X"][0], _c(e["X_KB"]), atol=1e-15)


# --- status handling ----------------------------------------------------------------

def test_nonfinite_input_flags_and_zeroes():
    H, S = random_problem(22, 3, 8, 2, 2)
    H[1, 3, 0] = np.nan
    out = oracle.precode(H, S, [4, 4], "wf", N0=0.1)
    assert list(out["status"]) == [0, oracle.NONFINITE, 0]
    assert np.all(out["X"][1] == 0) and np.any(out["X"][0] != 0)


def test_threads_do_not_change_results():
    p = synth.make_problem(8, 64, 2, 37, 3, 4, 10.0, seed=23)
    a = oracle.precode(p.H, p.S, p.cluster_sizes, "wf", N0=p.N0, nthreads=1)
    b = oracle.precode(p.H, p.S, p.cluster_sizes, "wf", N0=p.N0, nthreads=5)
    assert np.array_equal(a["X"], b["X"])


def test_rejects_bad_partition():
    H, S = random_problem(24, 1, 8, 2, 1)
    with pytest.raises(ValueError):
        oracle.precode(H, S, [4, 3], "wf")


# --- MRT (the fully distributed baseline of Sec. III-E) ----------------------------

def test_mrt_is_the_scaled_conjugate_channel():
    """P = Hm^H rho / (sqrt(Es) ||Hm||_F), straight from numpy; t = tr(G)
    equals ||H||_F^2 summed over the entries."""
    cs = [3, 6]
    H, _ = random_problem(40, 4, sum(cs), 5, 1)
    P, out = precoder_matrix(H, cs, "mrt", rho2=1.7, Es=1.0)
    for n in range(4):
        Hm = H[n].T
        want = Hm.conj().T * np.sqrt(1.7 / np.linalg.norm(Hm) ** 2)
        assert np.abs(P[n] - want).max() < 1e-12
        assert abs(out["t"][n] - out["t_alt"][n]) < 1e-12 * out["t"][n]
        assert abs(out["t"][n] - np.linalg.norm(Hm) ** 2) < 1e-12 * out["t"][n]
    assert (out["Z"] == np.broadcast_to(np.eye(5), out["Z"].shape)).all()  # z = s


def test_single_user_mrt_wf_and_zf_coincide():
    """For U = 1 every linear precoder is the normalized conjugate channel."""
    H, _ = random_problem(41, 3, 7, 1, 1)
    Pm, _ = precoder_matrix(H, [7], "mrt")
    Pw, _ = precoder_matrix(H, [7], "wf", N0=0.3)
    Pz, _ = precoder_matrix(H, [7], "zf")
    assert np.abs(Pm - Pw).max() < 1e-12 and np.abs(Pm - Pz).max() < 1e-12


def test_wf_tends_to_mrt_as_noise_grows():
    """kappa -> infinity: (G + kappa I)^{-1} -> I / kappa, so the normalized
    WF precoder tends to MRT (relative gap O(||G|| / kappa))."""
    cs = [4, 4]
    H, _ = random_problem(42, 2, sum(cs), 3, 1)
    Pm, _ = precoder_matrix(H, cs, "mrt")
    for N0, tol in ((1e3, 1e-2), (1e6, 1e-5)):
        Pw, _ = precoder_matrix(H, cs, "wf", N0=N0)
        assert np.abs(Pw - Pm).max() / np.abs(Pm).max() < tol


# --- per-cluster power allocation (Sec. III-D and its footnote) --------------------------

def test_cluster_power_equal_weights_are_the_uniform_split():
    """w_c all equal is the paper's rho_c^2 = rho^2 / C, whatever their value."""
    U, cs = 4, [5, 3, 8]
    H, S = random_problem(41, 3, sum(cs), U, 2)
    ref = oracle.precode(H, S, cs, "fdwf", N0=0.2, rho2=1.1, tau=0.5)["X"]
    for w in ([1.0, 1.0, 1.0], [2.5, 2.5, 2.5]):
        X = oracle.precode(H, S, cs, "fdwf", N0=0.2, rho2=1.1, tau=0.5, cluster_power=w)["X"]
        assert np.allclose(X, ref, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("cs", [[5, 3, 8], [2, 9, 1, 4]])
def test_cluster_power_per_cluster_constraint(cs):
    """Es ||P_c||_F^2 = rho_c^2 = rho^2 w_c / sum w for every cluster (the
    per-cluster constraint of Sec. III-D with unequal powers), and the total is
    rho^2.  Clusters with B_c < U take the B_c x B_c form."""
    U = 4
    w = np.arange(1, len(cs) + 1, dtype=float) ** 1.5
    H, _ = random_problem(42, 3, sum(cs), U, 1)
    P, out = precoder_matrix(H, cs, "fdwf", N0=0.3, rho2=1.7, Es=1.0, tau=0.25,
                             cluster_power=w)
    off = np.cumsum([0] + cs)
    for n in range(3):
        assert abs(np.linalg.norm(P[n]) ** 2 - 1.7) < 1e-12
        for c in range(len(cs)):
            pc = P[n, off[c]:off[c + 1]]
            assert abs(np.linalg.norm(pc) ** 2 - 1.7 * w[c] / w.sum()) < 1e-12


@pytest.mark.parametrize("cs,U", [([6, 3, 7], 4), ([2, 3, 5], 4)])
def test_cluster_power_equals_a_rescaled_uniform_problem(cs, U):
    """With rho_c^2 = w_c rho^2 (sum w = 1) the local WF of cluster c has
    kappa_c = tau U N0 / rho_c^2.  Scaling H_c by a_c = sqrt(C w_c) turns the
    uniform problem's (H_c H_c^H + kappa_u I) into a_c^2 (H_c H_c^H + kappa_c I)
    (kappa_u = C tau U N0 / rho^2), so the weighted precoder on H is a_c times
    the uniform one on the rescaled channel, cluster by cluster, in both the
    U x U and the B_c x B_c form."""
    C = len(cs)
    w = np.array([0.5, 0.3, 0.2])[:C]
    H, S = random_problem(43, 4, sum(cs), U, 3)
    kw = dict(N0=0.15, rho2=1.0, tau=0.125)
    Xw = oracle.precode(H, S, cs, "fdwf", cluster_power=w, **kw)["X"]
    off = np.cumsum([0] + cs)
    a = np.sqrt(C * w)
    Hs = H.copy()
    for c in range(C):
        Hs[:, off[c]:off[c + 1]] *= a[c]
    Xu = oracle.precode(Hs, S, cs, "fdwf", **kw)["X"]
    for c in range(C):
        sl = slice(off[c], off[c + 1])
        assert np.allclose(Xw[:, :, sl], a[c] * Xu[:, :, sl], rtol=1e-10, atol=1e-13)
    # and the weighting does change the output
    assert not np.allclose(Xw, oracle.precode(H, S, cs, "fdwf", **kw)["X"], rtol=1e-3)


def test_cluster_power_rejects_bad_weights():
    H, S = random_problem(44, 1, 8, 2, 1)
    for mode, w in (("fdwf", [1.0, 0.0]), ("fdwf", [1.0, -1.0]), ("fdwf", [1.0, np.nan]),
                    ("wf", [1.0, 1.0])):
        with pytest.raises(ValueError):
            oracle.precode(H, S, [4, 4], mode, cluster_power=w)
