"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test pins one part of the oracle to something other than itself: a textbook
closed form, exact hyper-dual derivatives of a value-only strain energy, the paper's
own spatial formulas (App. A.2), finite differences, invariance and symmetry, or
identities of the hex8 discretisation.
"""
import json
import os

import numpy as np
import pytest

import oracle
import workload as wl
from tests import hyperdual as hdm

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b, floor=1e-300):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), floor)


def rand_F(rng, n, s=0.2):
    return wl.random_F(rng, n, s)


def rand_rotation(rng):
    Q, R = np.linalg.qr(rng.normal(size=(3, 3)))
    Q = Q @ np.diag(np.sign(np.diag(R)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    return Q


@pytest.fixture(scope="module")
def iso_spec():
    rng = np.random.Generator(np.random.PCG64(11))
    return wl.make_model(rng, wl.KIN_ISO_SHIFTED, 0, W=8, L=2, kappa=10.0, bias_std=0.1)


@pytest.fixture(scope="module")
def aniso_spec():
    rng = np.random.Generator(np.random.PCG64(12))
    return wl.make_model(rng, wl.KIN_RAW, 2, W=6, L=3, kappa=3.0, bias_std=0.1)


# ------------------------------------------------------------------ P1 / P9

def neo_hookean_spec(mu, kappa):
    """MICNN reduced to Neo-Hookean: zero hidden weights, b = (mu/2, 0, 0)."""
    d, W, L = 3, 4, 2
    return wl.ModelSpec(d=d, W=W, L=L, kin=wl.KIN_ISO_SHIFTED, fibres=np.zeros((0, 3)),
                        W1=np.zeros((W, d)), Ak=np.zeros((L - 1, W, W)), Bk=np.zeros((L - 1, W, d)),
                        c=np.zeros((L, W)), a=np.zeros(W), b=np.array([mu / 2, 0.0, 0.0]), kappa=kappa)


def nh_closed_form(F9, mu, kappa):
    """Textbook compressible Neo-Hookean: Psi = mu/2 (Ibar1 - 3) + kappa (J - 1)^2,
    P = mu J^{-2/3} (F - I1/3 F^{-T}) + 2 kappa (J - 1) J F^{-T}."""
    F = F9.reshape(3, 3)
    J = np.linalg.det(F)
    I1 = np.sum(F * F)
    Fit = np.linalg.inv(F).T
    psi = 0.5 * mu * (J ** (-2 / 3) * I1 - 3) + kappa * (J - 1) ** 2
    P = mu * J ** (-2 / 3) * (F - I1 / 3 * Fit) + 2 * kappa * (J - 1) * J * Fit
    return psi, P.ravel()


def test_p1_neo_hookean_closed_form():
    mu, kappa = 1.7, 10.0
    spec = neo_hookean_spec(mu, kappa)
    m = oracle.OracleModel(spec)
    rng = np.random.Generator(np.random.PCG64(1))
    F = rand_F(rng, 16)
    psi, P, A = oracle.const_update(m, F)
    # the network's constant a.softplus(0) term is zero because a = 0
    for q in range(F.shape[0]):
        psi_c, P_c = nh_closed_form(F[q], mu, kappa)
        assert abs(psi[q] - psi_c) < 1e-13 * max(1, abs(psi_c))
        assert rel(P[q], P_c) < 1e-13
    # A against exact hyper-dual derivatives of the same closed form
    for q in range(3):
        _, P_h, A_h = hdm.exact_P_A(spec, F[q])
        assert rel(A[q], A_h) < 1e-13


@pytest.mark.parametrize("kind", ["UT", "UC", "BT", "BC", "SS", "PS"])
def test_p9_loading_paths_neo_hookean(kind):
    mu, kappa = 1.0, 10.0
    m = oracle.OracleModel(neo_hookean_spec(mu, kappa))
    for g in (0.05, 0.3, 0.8):
        F = wl.loading_path(kind, g)
        psi, P, _ = oracle.const_update(m, F[None], want_A=False)
        psi_c, P_c = nh_closed_form(F, mu, kappa)
        assert abs(psi[0] - psi_c) < 1e-13 * max(1, abs(psi_c))
        assert rel(P[0], P_c) < 1e-13


# ----------------------------------------------------------------------- P2

def test_p2_gent_thomas_chain_rule():
    """eq. gt through the oracle's generic chain rule vs exact derivatives of Psi(F)."""
    m = oracle.OracleModel(None, inner=oracle.INNER_GENT_THOMAS, kin=wl.KIN_RAW, fibres=[], kappa=0.0)
    spec = neo_hookean_spec(1.0, 0.0)

    def gt(K):
        Ib1, Ib2, J = K
        return 0.5 * (Ib1 - 3.0) + hdm.hd_log(Ib2 / 3.0) + (J - 1.0) * (J - 1.0)
    rng = np.random.Generator(np.random.PCG64(2))
    F = rand_F(rng, 4)
    psi, P, A = oracle.const_update(m, F)
    for q in range(F.shape[0]):
        psi_h, P_h, A_h = hdm.exact_P_A(spec, F[q], inner=gt)
        assert abs(psi[q] - psi_h) < 1e-13 * max(1, abs(psi_h))
        assert rel(P[q], P_h) < 1e-12
        assert rel(A[q], A_h) < 1e-12


def test_hgo_target_chain_rule():
    """Neo-Hookean-plus-fibre target model (used for the backward loss) vs exact derivatives."""
    mu, k1, k2, kappa = 1.0, 2.0, 0.5, 10.0
    m = oracle.OracleModel(None, inner=oracle.INNER_HGO, kin=wl.KIN_RAW, fibres=wl.FIBRES_PM30,
                           kappa=kappa, mu=mu, k1=k1, k2=k2)
    spec = wl.ModelSpec(d=7, W=1, L=1, kin=1, fibres=wl.FIBRES_PM30, W1=np.zeros((1, 7)),
                        Ak=np.zeros((0, 1, 1)), Bk=np.zeros((0, 1, 7)), c=np.zeros((1, 1)),
                        a=np.zeros(1), b=np.zeros(7), kappa=kappa)

    def hgo(K):
        out = 0.5 * mu * (K[0] - 3.0)
        for f in range(2):
            x = K[3 + f] - 1.0
            out = out + k1 / (2 * k2) * (hdm.hd_exp(k2 * x * x) - 1.0)
        return out
    rng = np.random.Generator(np.random.PCG64(3))
    F = rand_F(rng, 4)
    psi, P, A = oracle.const_update(m, F)
    for q in range(F.shape[0]):
        psi_h, P_h, A_h = hdm.exact_P_A(spec, F[q], inner=hgo)
        assert abs(psi[q] - psi_h) < 1e-13 * max(1, abs(psi_h))
        assert rel(P[q], P_h) < 1e-12
        assert rel(A[q], A_h) < 1e-12


# ----------------------------------------------------------------------- P6

@pytest.mark.parametrize("which", ["iso", "aniso"])
def test_p6_exact_derivatives_hyperdual(which, iso_spec, aniso_spec):
    spec = iso_spec if which == "iso" else aniso_spec
    m = oracle.OracleModel(spec)
    rng = np.random.Generator(np.random.PCG64(4))
    F = rand_F(rng, 4, 0.25)
    psi, P, A = oracle.const_update(m, F)
    for q in range(F.shape[0]):
        psi_h, P_h, A_h = hdm.exact_P_A(spec, F[q])
        assert abs(psi[q] - psi_h) < 1e-13 * max(1, abs(psi_h))
        assert rel(P[q], P_h) < 1e-12
        assert rel(A[q], A_h) < 1e-12


def test_p6_central_differences(aniso_spec):
    m = oracle.OracleModel(aniso_spec)
    rng = np.random.Generator(np.random.PCG64(5))
    F = rand_F(rng, 2)
    h = 1e-5
    for q in range(2):
        _, P, A = oracle.const_update(m, F[q][None])
        Pfd, Afd = np.zeros(9), np.zeros((9, 9))
        for a in range(9):
            e = np.zeros(9)
            e[a] = h
            pp, Pp, _ = oracle.const_update(m, (F[q] + e)[None], want_A=False)
            pm, Pm, _ = oracle.const_update(m, (F[q] - e)[None], want_A=False)
            Pfd[a] = (pp[0] - pm[0]) / (2 * h)
            Afd[a] = (Pp[0] - Pm[0]) / (2 * h)
        assert rel(P[0], Pfd) < 1e-8
        assert rel(A[0], Afd.ravel()) < 1e-8


def test_kinematics_against_hyperdual():
    """Each kinematic scalar's first and second derivatives separately (eq. 454, App. A.2)."""
    fib = wl.FIBRES_PM30
    m = oracle.OracleModel(None, inner=oracle.INNER_GENT_THOMAS, kin=wl.KIN_RAW, fibres=fib)
    rng = np.random.Generator(np.random.PCG64(6))
    F = rand_F(rng, 1, 0.3)[0]
    K, dK, d2K = oracle.kinematics(m, F)
    a_idx, b_idx = [x.ravel() for x in np.meshgrid(np.arange(9), np.arange(9), indexing="ij")]
    F9 = [hdm.HD(np.full(81, F[c]), (a_idx == c).astype(float), (b_idx == c).astype(float), 0.0)
          for c in range(9)]
    Kh, _ = hdm.kinematic_scalars(F9, 1, fib)
    assert len(Kh) == K.size == 7
    for i, k in enumerate(Kh):
        assert abs(K[i] - k.r[0]) < 1e-13 * abs(k.r[0])
        assert rel(dK[i], k.e1.reshape(9, 9)[:, 0]) < 1e-13
        assert rel(d2K[i], k.e12) < 1e-12


# ---------------------------------------------------------------------- P10

@pytest.mark.parametrize("dims", [(3, 16, 2), (7, 6, 3), (3, 5, 4)])
def test_p10_algorithm4_vs_hyperdual(dims):
    d, W, L = dims
    rng = np.random.Generator(np.random.PCG64(7))
    kin = wl.KIN_ISO_SHIFTED if d == 3 else wl.KIN_RAW
    spec = wl.make_model(rng, kin, (d - 3) // 2, W=W, L=L, kappa=0.0, std=0.3, bias_std=0.2)
    m = oracle.OracleModel(spec)
    for _ in range(3):
        K = rng.normal(size=d)
        N, dN, d2N = oracle.inner(m, K)
        N_h, dN_h, d2N_h = hdm.exact_inner(spec, K)
        assert abs(N - N_h) < 1e-14 * max(1, abs(N_h))
        assert rel(dN, dN_h) < 1e-13
        assert rel(d2N, d2N_h) < 1e-12
        assert np.all(np.linalg.eigvalsh(0.5 * (d2N + d2N.T)) > -1e-12)  # convex (eq. icnn)
        assert np.all(dN >= 0)  # monotone: non-negative weights


def test_p10_linear_when_hidden_weights_zero():
    spec = neo_hookean_spec(1.0, 0.0)
    spec.a = np.array([0.3, 0.1, 0.0, 0.2])
    spec.b = np.array([0.5, 0.25, 2.0])
    m = oracle.OracleModel(spec)
    K = np.array([0.3, -0.2, 0.1])
    N, dN, d2N = oracle.inner(m, K)
    assert abs(N - (np.log(2.0) * spec.a.sum() + spec.b @ K)) < 1e-15
    assert np.array_equal(dN, spec.b)
    assert np.all(d2N == 0)


# ----------------------------------------------------------------------- P3

def test_p3_stress_free(iso_spec, aniso_spec):
    I9 = np.eye(3).ravel()
    # literal model: P(I) = dN/dK_J at K(I) times I
    m = oracle.OracleModel(iso_spec)
    _, P, _ = oracle.const_update(m, I9[None])
    _, dN, _ = oracle.inner(m, np.zeros(3))
    assert rel(P[0], dN[2] * I9) < 1e-14
    # with the stress-free shift, P(I) = 0 for any kinematics
    for spec in (iso_spec, aniso_spec):
        m0 = oracle.OracleModel(spec, stress_free=True)
        _, P0, A0 = oracle.const_update(m0, I9[None])
        assert np.abs(P0).max() < 1e-14
        # the shift is linear in K, so it changes P but leaves the N_mn term of A alone
        rng = np.random.Generator(np.random.PCG64(8))
        F = rand_F(rng, 2)
        _, Pa, Aa = oracle.const_update(oracle.OracleModel(spec), F)
        _, Pb, Ab = oracle.const_update(m0, F)
        assert rel(Pa, Pb) > 1e-6


# ----------------------------------------------------------------------- P4

def test_p4_objectivity_and_material_symmetry(iso_spec, aniso_spec):
    rng = np.random.Generator(np.random.PCG64(9))
    F = rand_F(rng, 4)
    for spec in (iso_spec, aniso_spec):
        m = oracle.OracleModel(spec)
        psi, P, A = oracle.const_update(m, F)
        Q = rand_rotation(rng)
        FQ = np.einsum("ab,nbc->nac", Q, F.reshape(-1, 3, 3)).reshape(-1, 9)
        psi2, P2, A2 = oracle.const_update(m, FQ)
        assert np.abs(psi2 - psi).max() < 1e-12 * np.abs(psi).max()
        Pq = np.einsum("ab,nbJ->naJ", Q, P.reshape(-1, 3, 3)).reshape(-1, 9)
        assert rel(P2, Pq) < 1e-12
        Aq = np.einsum("ia,kb,naJbL->niJkL", Q, Q, A.reshape(-1, 3, 3, 3, 3)).reshape(-1, 81)
        assert rel(A2, Aq) < 1e-12
        # material symmetry: Psi(F Q^T; Q A^i) = Psi(F; A^i), P -> P Q^T
        R = rand_rotation(rng)
        specR = wl.ModelSpec(**{**spec.__dict__, "fibres": spec.fibres @ R.T})
        mR = oracle.OracleModel(specR)
        FR = np.einsum("nab,cb->nac", F.reshape(-1, 3, 3), R).reshape(-1, 9)
        psi3, P3, _ = oracle.const_update(mR, FR)
        assert np.abs(psi3 - psi).max() < 1e-12 * np.abs(psi).max()
        PR = np.einsum("naJ,cJ->nac", P.reshape(-1, 3, 3), R).reshape(-1, 9)
        assert rel(P3, PR) < 1e-12


# ----------------------------------------------------------------------- P5

def test_p5_symmetries(aniso_spec):
    m = oracle.OracleModel(aniso_spec)
    rng = np.random.Generator(np.random.PCG64(10))
    F = rand_F(rng, 8)
    _, P, A = oracle.const_update(m, F)
    A9 = A.reshape(-1, 9, 9)
    assert np.abs(A9 - A9.transpose(0, 2, 1)).max() < 1e-13 * np.abs(A9).max()
    tau = np.einsum("niJ,njJ->nij", P.reshape(-1, 3, 3), F.reshape(-1, 3, 3))
    assert np.abs(tau - tau.transpose(0, 2, 1)).max() < 1e-13 * np.abs(tau).max()


# ----------------------------------------------------------------------- P7

def _odot(X, Y):
    """(X (.) Y)_ijkl = 1/2 (X_ik Y_jl + X_il Y_kj) (App. A.2 notation)."""
    return 0.5 * (np.einsum("ik,jl->ijkl", X, Y) + np.einsum("il,kj->ijkl", X, Y))


def _otimes(X, Y):
    return np.einsum("ij,kl->ijkl", X, Y)


def spatial_G(F, kin, fibres):
    """G^m and GG^m of App. A.2 for the kinematic scalars, with the isochoric forms of
    App. A.2 for Ibar1, Ibar2 (using Btilde throughout, with alpha on I3) and the
    volumetric forms for J."""
    I = np.eye(3)
    J = np.linalg.det(F)
    B = F @ F.T
    Bt = J ** (-2 / 3) * B
    Gs, GGs = [], []
    # Ibar1: alpha = -1/3 ; Gtilde = Btilde, GGtilde = 0
    for alpha, Gt, GGt, Ib in (
            (-1 / 3, Bt, np.zeros((3, 3, 3, 3)), np.trace(Bt)),
            (-2 / 3, Bt * np.trace(Bt) - Bt @ Bt, _otimes(Bt, Bt) - _odot(Bt, Bt),
             0.5 * (np.trace(Bt) ** 2 - np.trace(Bt @ Bt)))):
        Gs.append(Gt + alpha * Ib * I)
        GGs.append(GGt + alpha * (_otimes(I, Gt) + _otimes(Gt, I) + Ib * (alpha * _otimes(I, I) - _odot(I, I))))
    Gs.append(J / 2 * I)
    GGs.append(J / 4 * (_otimes(I, I) - 2 * _odot(I, I)))
    if kin == wl.KIN_RAW:
        I4G, I4GG, I5G, I5GG = [], [], [], []
        for A0 in fibres:
            a = F @ A0
            aa = np.outer(a, a)
            I4G.append(aa)
            I4GG.append(np.zeros((3, 3, 3, 3)))
            Ba = B @ a
            I5G.append(np.outer(a, Ba) + np.outer(Ba, a))
            I5GG.append(_odot(B, aa) + _odot(aa, B))
        Gs += I4G + I5G
        GGs += I4GG + I5GG
    return Gs, GGs


@pytest.mark.parametrize("which", ["iso", "aniso"])
def test_p7_spatial_route_of_the_paper(which, iso_spec, aniso_spec):
    """tau = 2 N_m G^m, c = 4 N_mn G^m G^n + 4 N_m GG^m (App. A.2) against the oracle's
    material P, A pushed forward by tau = P F^T, c = F A F - delta tau (App. A.1)."""
    spec = iso_spec if which == "iso" else aniso_spec
    m = oracle.OracleModel(spec)
    rng = np.random.Generator(np.random.PCG64(13))
    F = rand_F(rng, 3)
    _, P, A = oracle.const_update(m, F)
    for q in range(F.shape[0]):
        Fq = F[q].reshape(3, 3)
        K, _, _ = oracle.kinematics(m, F[q])
        _, dN, d2N = oracle.inner(m, K)
        # the volumetric penalty kappa (J-1)^2 acts on J through the same G, GG
        J = np.linalg.det(Fq)
        dN = dN.copy()
        d2N = d2N.copy()
        dN[2] += 2 * spec.kappa * (J - 1.0)
        d2N[2, 2] += 2 * spec.kappa
        Gs, GGs = spatial_G(Fq, spec.kin, spec.fibres)
        tau = 2 * sum(dN[i] * Gs[i] for i in range(len(Gs)))
        c = 4 * sum(d2N[i, j] * _otimes(Gs[i], Gs[j]) for i in range(len(Gs)) for j in range(len(Gs)))
        c = c + 4 * sum(dN[i] * GGs[i] for i in range(len(Gs)))
        P3 = P[q].reshape(3, 3)
        A4 = A[q].reshape(3, 3, 3, 3)
        tau_o = P3 @ Fq.T
        c_o = np.einsum("jJ,iJkL,lL->ijkl", Fq, A4, Fq) - np.einsum("ik,jl->ijkl", np.eye(3), tau_o)
        assert rel(tau, tau_o) < 1e-12
        assert rel(c, c_o) < 1e-12


# ----------------------------------------------------------------------- P8

def distorted_mesh(n, seed, amp=0.15):
    mesh = wl.structured_mesh(n)
    rng = np.random.Generator(np.random.PCG64(seed))
    X = mesh.X + amp / n * rng.uniform(-1, 1, size=mesh.X.shape)
    on_bnd = np.any((mesh.X == 0.0) | (mesh.X == 1.0), axis=1)
    X[on_bnd] = mesh.X[on_bnd]
    return wl.Mesh(X=X, conn=mesh.conn, n=mesh.n)


def test_p8_quadrature_volume_and_partition_of_unity():
    mesh = distorted_mesh(3, 1)
    vol = 0.0
    for e in range(mesh.n_el):
        dphi, w = oracle.hex8_gradients(mesh.X[mesh.conn[e]])
        vol += w.sum()
        assert np.abs(dphi.sum(axis=1)).max() < 1e-13  # sum_I grad phi_I = 0
        # sum_I X_I (x) grad phi_I = identity (isoparametric map reproduces X)
        G = np.einsum("Ia,qIb->qab", mesh.X[mesh.conn[e]], dphi)
        assert np.abs(G - np.eye(3)).max() < 1e-13
    assert abs(vol - 1.0) < 1e-13


def test_p8_affine_patch_test():
    mesh = distorted_mesh(3, 2)
    H0 = np.array([[0.1, 0.02, -0.03], [0.01, -0.05, 0.04], [0.02, 0.03, 0.07]])
    u = mesh.X @ H0.T
    F = oracle.compute_F(mesh, u)
    assert np.abs(F - (np.eye(3) + H0).ravel()[None]).max() < 1e-14
    rng = np.random.Generator(np.random.PCG64(3))
    spec = wl.make_model(rng, wl.KIN_RAW, 2, W=5, L=2, kappa=2.0)
    m = oracle.OracleModel(spec)
    _, P, A = oracle.const_update(m, F)
    f_e, K_e = oracle.elem_assemble(mesh, P, A)
    r = oracle.scatter_residual(mesh, f_e).reshape(-1, 3)
    interior = ~np.any((mesh.X == 0.0) | (mesh.X == 1.0), axis=1)
    assert interior.sum() > 0
    assert np.abs(r[interior]).max() < 1e-13 * np.abs(r).max()
    # sum_I X_I,a r_I,i = volume * P_ia for constant P
    moment = np.einsum("Ia,Ii->ia", mesh.X, r)
    assert rel(moment, P[0].reshape(3, 3)) < 1e-13
    # element balance and rigid-translation null space of K_e
    assert np.abs(f_e.reshape(-1, 8, 3).sum(axis=1)).max() < 1e-13 * np.abs(f_e).max()
    Kt = K_e.reshape(-1, 24, 8, 3).sum(axis=2)
    assert np.abs(Kt).max() < 1e-12 * np.abs(K_e).max()
    assert np.abs(K_e - K_e.transpose(0, 2, 1)).max() < 1e-13 * np.abs(K_e).max()


def test_p8_linear_elastic_f_equals_K_u():
    """Constant major-symmetric A and P = A : grad u give f_e = K_e u_e exactly."""
    mesh = distorted_mesh(2, 4)
    lam, mu = 1.3, 0.7
    I = np.eye(3)
    A4 = lam * np.einsum("iJ,kL->iJkL", I, I) + mu * (np.einsum("ik,JL->iJkL", I, I) +
                                                       np.einsum("iL,Jk->iJkL", I, I))
    rng = np.random.Generator(np.random.PCG64(5))
    u = 0.01 * rng.normal(size=mesh.X.shape)
    F = oracle.compute_F(mesh, u)
    H = F - I.ravel()[None]
    P = np.einsum("ab,nb->na", A4.reshape(9, 9), H)
    A = np.broadcast_to(A4.reshape(81), (F.shape[0], 81)).copy()
    f_e, K_e = oracle.elem_assemble(mesh, P, A)
    ue = u[mesh.conn].reshape(-1, 24)
    assert rel(f_e, np.einsum("eab,eb->ea", K_e, ue)) < 1e-13


def test_p8_taylor_test_consistent_tangent():
    """f(u + eps v) - f(u) - eps K(u) v = O(eps^2) with the network material."""
    mesh = distorted_mesh(2, 6)
    rng = np.random.Generator(np.random.PCG64(6))
    spec = wl.make_model(rng, wl.KIN_RAW, 2, W=6, L=3, kappa=5.0)
    m = oracle.OracleModel(spec)
    u = 0.02 * rng.normal(size=mesh.X.shape)
    v = rng.normal(size=mesh.X.shape)

    def f_and_K(uu):
        F = oracle.compute_F(mesh, uu)
        _, P, A = oracle.const_update(m, F)
        return oracle.elem_assemble(mesh, P, A)
    f0, K0 = f_and_K(u)
    Kv = np.einsum("eab,eb->ea", K0, v[mesh.conn].reshape(-1, 24))
    errs = []
    for eps in (1e-2, 5e-3, 2.5e-3, 1.25e-3):
        f1, _ = f_and_K(u + eps * v)
        errs.append(np.linalg.norm(f1 - f0 - eps * Kv))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > 1.9), slopes


def test_p8_global_csr_scatter():
    """CSR scatter equals the dense sum over elements and annihilates rigid translations."""
    mesh = distorted_mesh(2, 7)
    rng = np.random.Generator(np.random.PCG64(7))
    spec = wl.make_model(rng, wl.KIN_RAW, 2, W=4, L=2, kappa=1.0)
    m = oracle.OracleModel(spec)
    F = oracle.compute_F(mesh, 0.02 * rng.normal(size=mesh.X.shape))
    _, P, A = oracle.const_update(m, F)
    f_e, K_e = oracle.elem_assemble(mesh, P, A)
    n = 3 * mesh.n_nodes
    dense = np.zeros((n, n))
    dofs = (3 * mesh.conn[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 24)
    for e in range(mesh.n_el):
        dense[np.ix_(dofs[e], dofs[e])] += K_e[e]
    rows, cols = np.nonzero(dense != 0.0)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    vals, missing = oracle.scatter_csr(mesh, K_e, rowptr, cols.astype(np.int32))
    assert missing == 0
    assert np.array_equal(vals, dense[rows, cols])
    t = np.tile([1.0, 0.0, 0.0], mesh.n_nodes)
    assert np.abs(dense @ t).max() < 1e-12 * np.abs(dense).max()


# --------------------------------------------------------------------- P11/P12

def test_p11_p12_paper_sizes():
    g = json.load(open(os.path.join(GOLD, "paper_sizes.json")))
    assert wl.dof_count(128) == g["dofs_cube_128"]["value"]
    assert wl.dof_count(256) == g["dofs_cube_256"]["value"]
    assert wl.n_params(3, 16, 3, bias=False) == g["micnn_params_d3_w16_l3"]["value"]
    # the oracle's parameter vector also carries the L*W biases
    assert oracle.n_params(3, 16, 3) == g["micnn_params_d3_w16_l3"]["value"] + 3 * 16


# ---------------------------------------------------------------------- P13

@pytest.mark.parametrize("kin,nf", [(wl.KIN_RAW, 2), (wl.KIN_ISO_SHIFTED, 0), (wl.KIN_POLYCONVEX, 0)])
def test_p13_backward_central_differences(kin, nf):
    """dL/dtheta and dL/dF of L = sum_q G_q : P_q(F_q; theta) against central differences,
    on every kinematic layer: raw with fibres, the shifted isochoric inputs, and the
    polyconvex layer of App. C, whose chain rule adds the phi'' term to dL/dF."""
    rng = np.random.Generator(np.random.PCG64(14 + kin))
    spec = wl.make_model(rng, kin, nf, W=4, L=3, kappa=3.0, bias_std=0.1)
    m = oracle.OracleModel(spec)
    F = rand_F(rng, 6)
    G = rng.normal(size=F.shape)
    dF, dth = oracle.const_backward(m, F, G)
    theta = spec.theta()
    assert dth.size == theta.size == oracle.n_params(spec.d, spec.W, spec.L)

    def L_of(th, FF):
        mm = oracle.OracleModel(spec.with_theta(th))
        _, P, _ = oracle.const_update(mm, FF, want_A=False)
        return float(np.sum(G * P))
    h = 1e-6
    fd = np.zeros_like(theta)
    for i in range(theta.size):
        e = np.zeros_like(theta)
        e[i] = h
        fd[i] = (L_of(theta + e, F) - L_of(theta - e, F)) / (2 * h)
    assert rel(dth, fd) < 1e-7
    fdF = np.zeros_like(F)
    for q in range(F.shape[0]):
        for a in range(9):
            Fp, Fm = F.copy(), F.copy()
            Fp[q, a] += h
            Fm[q, a] -= h
            fdF[q, a] = (L_of(theta, Fp) - L_of(theta, Fm)) / (2 * h)
    assert rel(dF, fdF) < 1e-7
    # closed form for the output skip weights: dL/db_m = sum_q G_q : dK_m/dF
    r = np.array([[np.sum(G[q] * oracle.kinematics(m, F[q])[1][i]) for i in range(spec.d)]
                  for q in range(F.shape[0])])
    assert rel(dth[-spec.d:], r.sum(axis=0)) < 1e-13


def test_p13_backward_of_the_target_loss():
    """L = sum_q |P_q - P_target,q|^2 with G = 2 (P - P_target): FD on the whole loss."""
    rng = np.random.Generator(np.random.PCG64(15))
    spec = wl.make_model(rng, wl.KIN_RAW, 2, W=3, L=2, kappa=0.0)
    m = oracle.OracleModel(spec)
    F = rand_F(rng, 5)
    tgt = oracle.OracleModel(None, inner=oracle.INNER_HGO, kin=wl.KIN_RAW, fibres=wl.FIBRES_PM30,
                             kappa=10.0, mu=1.0, k1=2.0, k2=0.5)
    _, Pt, _ = oracle.const_update(tgt, F, want_A=False)
    _, P, _ = oracle.const_update(m, F, want_A=False)
    _, dth = oracle.const_backward(m, F, 2 * (P - Pt))
    theta = spec.theta()

    def loss(th):
        _, PP, _ = oracle.const_update(oracle.OracleModel(spec.with_theta(th)), F, want_A=False)
        return float(np.sum((PP - Pt) ** 2))
    h = 1e-6
    idx = np.arange(0, theta.size, 3)
    fd = np.array([(loss(theta + h * np.eye(theta.size)[i]) - loss(theta - h * np.eye(theta.size)[i])) / (2 * h)
                   for i in idx])
    assert rel(dth[idx], fd) < 1e-6


# ------------------------------------------------------------------ workloads

def test_c0_workload_is_orientation_preserving():
    w = wl.workload_c0()
    F = oracle.compute_F(w["mesh"], w["u"])
    assert F.shape == (4096, 9)
    assert np.linalg.det(F.reshape(-1, 3, 3)).min() > 0.5


# ------------------------------------------- the paper's polyconvex kinematic layer

@pytest.fixture(scope="module")
def poly_spec():
    rng = np.random.Generator(np.random.PCG64(16))
    return wl.make_model(rng, wl.KIN_POLYCONVEX, 0, W=8, L=3, kappa=0.0, bias_std=0.1)


def test_polyconvex_layer_exact_derivatives(poly_spec):
    """K = (Ibar1 - 3, Ibar2^{3/2} - 3^{3/2}, (J - 1)^2) (App. C) against hyper-dual Psi(F)."""
    m = oracle.OracleModel(poly_spec)
    rng = np.random.Generator(np.random.PCG64(17))
    F = rand_F(rng, 3, 0.25)
    psi, P, A = oracle.const_update(m, F)
    for q in range(F.shape[0]):
        psi_h, P_h, A_h = hdm.exact_P_A(poly_spec, F[q])
        assert abs(psi[q] - psi_h) < 1e-13 * max(1, abs(psi_h))
        assert rel(P[q], P_h) < 1e-12
        assert rel(A[q], A_h) < 1e-12


def test_polyconvex_layer_is_stress_free_for_any_weights(poly_spec):
    """Every input of this layer has zero F-gradient at F = I, so P(I) = 0 without any
    shift (the reason the paper chose it), while A(I) is not zero."""
    m = oracle.OracleModel(poly_spec)
    _, P, A = oracle.const_update(m, np.eye(3).ravel()[None])
    assert np.abs(P).max() < 1e-15
    assert np.abs(A).max() > 1e-3


def test_paper_ncm_has_675_parameters():
    w = wl.workload_paper_ncm(n=1)
    spec = w["model"]
    assert (spec.d, spec.W, spec.L) == (3, 16, 3)
    g = json.load(open(os.path.join(GOLD, "paper_sizes.json")))
    assert wl.n_params(spec.d, spec.W, spec.L, bias=False) == g["micnn_params_d3_w16_l3"]["value"]
    assert np.all(spec.c == 0)


# ------------------------------------------------- spatial (Voigt) outputs, App. A.1

def _voigt_full(c21):
    """Full c_ijkl from the 21 stored values (upper triangle of the 6 x 6 Voigt matrix)."""
    V = np.zeros((6, 6))
    V[np.triu_indices(6)] = c21
    V = V + np.triu(V, 1).T
    slot = np.zeros((3, 3), dtype=int)
    for v, (i, j) in enumerate(oracle.VOIGT):
        slot[i, j] = slot[j, i] = v
    return V[slot[:, :, None, None], slot[None, None, :, :]]


@pytest.mark.parametrize("which", ["iso", "aniso"])
def test_spatial_voigt_outputs_against_the_paper_route(which, iso_spec, aniso_spec):
    """tau[6], c[21] from the oracle's push-forward (App. A.1) against tau = 2 N_m G^m,
    c = 4 N_mn G^m G^n + 4 N_m GG^m (App. A.2) with exact hyper-dual network derivatives;
    the 21 values rebuild the whole c_ijkl, so c has both minor and the major symmetry."""
    spec = iso_spec if which == "iso" else aniso_spec
    m = oracle.OracleModel(spec)
    rng = np.random.Generator(np.random.PCG64(21))
    F = rand_F(rng, 4, 0.25)
    _, P, A = oracle.const_update(m, F)
    tau6, c21 = oracle.push_forward(F, P, A)
    for q in range(F.shape[0]):
        Fq = F[q].reshape(3, 3)
        Gs, GGs = spatial_G(Fq, spec.kin, spec.fibres)
        C = Fq.T @ Fq
        J = np.linalg.det(Fq)
        I1, I2 = np.trace(C), 0.5 * (np.trace(C) ** 2 - np.trace(C @ C))
        K = [J ** (-2 / 3) * I1, J ** (-4 / 3) * I2, J]
        if spec.kin == wl.KIN_ISO_SHIFTED:
            K = [K[0] - 3, K[1] - 3, J - 1]
        for A0 in spec.fibres:
            K.append(A0 @ C @ A0)
        for A0 in spec.fibres:
            K.append(A0 @ C @ C @ A0)
        _, dN, d2N = hdm.exact_inner(spec, np.array(K))
        dN[2] += 2 * spec.kappa * (J - 1.0)
        d2N[2, 2] += 2 * spec.kappa
        n = len(Gs)
        tau = 2 * sum(dN[i] * Gs[i] for i in range(n))
        c = 4 * sum(d2N[i, j] * _otimes(Gs[i], Gs[j]) for i in range(n) for j in range(n))
        c = c + 4 * sum(dN[i] * GGs[i] for i in range(n))
        assert rel([tau[i, j] for i, j in oracle.VOIGT], tau6[q]) < 1e-12
        assert rel(_voigt_full(c21[q]), c) < 1e-12
        assert rel(tau, tau.T) < 1e-13


def test_spatial_neo_hookean_closed_form():
    """Neo-Hookean: tau = mu J^{-2/3} dev(B) + 2 kappa (J - 1) J I."""
    mu, kappa = 1.3, 7.0
    m = oracle.OracleModel(neo_hookean_spec(mu, kappa))
    rng = np.random.Generator(np.random.PCG64(22))
    F = rand_F(rng, 5)
    _, P, A = oracle.const_update(m, F)
    tau6, _ = oracle.push_forward(F, P, None)
    for q in range(F.shape[0]):
        Fq = F[q].reshape(3, 3)
        J = np.linalg.det(Fq)
        B = Fq @ Fq.T
        tau = mu * J ** (-2 / 3) * (B - np.trace(B) / 3 * np.eye(3)) + 2 * kappa * (J - 1) * J * np.eye(3)
        assert rel([tau[i, j] for i, j in oracle.VOIGT], tau6[q]) < 1e-13


def test_spatial_assembly_equals_material_assembly(aniso_spec):
    """eq. k-quad in spatial form with grad phi = Grad phi F^{-1} gives the material-form
    K_e and f_e (App. A.1: grad phi_k c_ikjl grad phi_l + delta tau terms = Grad phi A Grad phi)
    for any F, compatible with a displacement or not."""
    mesh = distorted_mesh(2, 23)
    m = oracle.OracleModel(aniso_spec)
    rng = np.random.Generator(np.random.PCG64(24))
    F = rand_F(rng, 8 * mesh.n_el, 0.2)
    _, P, A = oracle.const_update(m, F)
    tau6, c21 = oracle.push_forward(F, P, A)
    f_m, K_m = oracle.elem_assemble(mesh, P, A)
    f_s, K_s = oracle.elem_assemble_spatial(mesh, F, tau6, c21)
    assert rel(f_s, f_m) < 1e-12
    assert rel(K_s, K_m) < 1e-12
    f_s2, K_s2 = oracle.elem_assemble_spatial(mesh, F, tau6, None)
    assert K_s2 is None and rel(f_s2, f_m) < 1e-12


# ----------------------------------------------------------- CANN (eq. cann-def)

ALL_KINDS = np.array([[wl.CANN_F0_ID, 1, wl.CANN_F2_LINEAR], [wl.CANN_F0_ID, 2, wl.CANN_F2_EXP],
                      [wl.CANN_F0_MACAULAY, 3, wl.CANN_F2_LINEAR], [wl.CANN_F0_ABS, 2, wl.CANN_F2_LOG],
                      [wl.CANN_F0_ABS, 1, wl.CANN_F2_EXP], [wl.CANN_F0_MACAULAY, 2, wl.CANN_F2_LOG]],
                     dtype=np.int32)


@pytest.mark.parametrize("kin,nf", [(wl.KIN_POLYCONVEX, 0), (wl.KIN_RAW, 2), (wl.KIN_ISO_SHIFTED, 0)])
def test_cann_exact_derivatives(kin, nf):
    """Every menu entry of eq. cann-fs through the oracle's chain rule (eq. cann-chain-rule)
    against hyper-dual derivatives of the value-only CANN; the f2 = -ln(1 - w1 y) term fixes
    the sign of its second derivative (+w1^2 / (1 - w1 y)^2)."""
    rng = np.random.Generator(np.random.PCG64(40 + kin))
    # raw inputs are O(3): smaller weights keep 1 - w1 y > 0 for the logarithmic term
    spec = wl.make_cann(rng, kin, nf, kinds=ALL_KINDS, kappa=2.0, std=0.02 if kin == wl.KIN_RAW else 0.2)
    m = oracle.OracleModel(spec)
    F = rand_F(rng, 4, 0.25)
    psi, P, A = oracle.const_update(m, F)
    for q in range(F.shape[0]):
        psi_h, P_h, A_h = hdm.exact_P_A(spec, F[q])
        assert abs(psi[q] - psi_h) < 1e-13 * max(1, abs(psi_h))
        assert rel(P[q], P_h) < 1e-12
        assert rel(A[q], A_h) < 1e-12


@pytest.mark.parametrize("kin,nf", [(wl.KIN_POLYCONVEX, 0), (wl.KIN_RAW, 2), (wl.KIN_ISO_SHIFTED, 0)])
def test_cann_backward_central_differences(kin, nf):
    """dL/dw and dL/dF of L = sum_q G_q : P_q(F_q; w) for the CANN of eq. cann-def, every
    f0/f1/f2 entry of eq. cann-fs, against central differences in each weight and each F
    entry; and, since P is linear in the w2 weights, sum w2 dL/dw2 = L with kappa = 0."""
    import dataclasses
    rng = np.random.Generator(np.random.PCG64(43 + kin))
    spec = wl.make_cann(rng, kin, nf, kinds=ALL_KINDS, kappa=0.0, std=0.02 if kin == wl.KIN_RAW else 0.2)
    m = oracle.OracleModel(spec)
    F = rand_F(rng, 5, 0.25)
    G = rng.normal(size=F.shape)
    dF, dth = oracle.const_backward(m, F, G)
    theta = spec.theta()
    assert dth.size == theta.size == 2 * spec.d * spec.n

    def L_of(th, FF):
        mm = oracle.OracleModel(dataclasses.replace(spec, w=th.reshape(spec.w.shape)))
        _, P, _ = oracle.const_update(mm, FF, want_A=False)
        return float(np.sum(G * P))
    h = 1e-6
    fd = np.array([(L_of(theta + h * e, F) - L_of(theta - h * e, F)) / (2 * h) for e in np.eye(theta.size)])
    assert rel(dth, fd) < 1e-7
    fdF = np.zeros_like(F)
    for q in range(F.shape[0]):
        for a in range(9):
            Fp, Fm = F.copy(), F.copy()
            Fp[q, a] += h
            Fm[q, a] -= h
            fdF[q, a] = (L_of(theta, Fp) - L_of(theta, Fm)) / (2 * h)
    assert rel(dF, fdF) < 1e-7
    assert abs(np.sum(theta[1::2] * dth[1::2]) - L_of(theta, F)) < 1e-12 * np.abs(dth).sum()


def test_cann_reduces_to_neo_hookean():
    """One linear term w2 w1 (Ibar1 - 3) with w1 w2 = mu / 2 is the textbook Neo-Hookean."""
    mu, kappa = 1.7, 10.0
    w = np.zeros((3, 1, 2))
    w[0, 0] = (0.5, mu)  # w1 = 0.5, w2 = mu
    spec = wl.CannSpec(d=3, kin=wl.KIN_ISO_SHIFTED, fibres=np.zeros((0, 3)), n=1,
                       kinds=np.array([[wl.CANN_F0_ID, 1, wl.CANN_F2_LINEAR]], dtype=np.int32), w=w, kappa=kappa)
    m = oracle.OracleModel(spec)
    rng = np.random.Generator(np.random.PCG64(41))
    F = rand_F(rng, 8)
    psi, P, _ = oracle.const_update(m, F)
    for q in range(F.shape[0]):
        psi_c, P_c = nh_closed_form(F[q], mu, kappa)
        assert abs(psi[q] - psi_c) < 1e-13 * max(1, abs(psi_c))
        assert rel(P[q], P_c) < 1e-13


def test_cann_hessian_is_diagonal_and_paper_cann_is_stress_free():
    rng = np.random.Generator(np.random.PCG64(42))
    spec = wl.make_cann(rng)
    m = oracle.OracleModel(spec)
    _, dN, d2N = oracle.inner(m, np.array([0.3, 0.2, 0.1]))
    assert np.all(d2N[~np.eye(3, dtype=bool)] == 0.0) and np.all(np.diag(d2N) > 0)
    _, P, _ = oracle.const_update(m, np.eye(3).ravel()[None])
    assert np.abs(P).max() < 1e-15
    assert spec.theta().size == 24


def test_gent_thomas_spec_is_eq_gt():
    """The Gent-Thomas spec (no parameters) is eq. gt, against hyper-dual derivatives."""
    m = oracle.OracleModel(wl.GentThomasSpec())
    spec = neo_hookean_spec(1.0, 0.0)

    def gt(K):
        return 0.5 * (K[0] - 3.0) + hdm.hd_log(K[1] / 3.0) + (K[2] - 1.0) * (K[2] - 1.0)
    rng = np.random.Generator(np.random.PCG64(43))
    F = rand_F(rng, 3)
    psi, P, A = oracle.const_update(m, F)
    for q in range(3):
        psi_h, P_h, A_h = hdm.exact_P_A(spec, F[q], inner=gt)
        assert rel(P[q], P_h) < 1e-12 and rel(A[q], A_h) < 1e-12


# ------------------------------------------------------------------ ICKAN (App. B)

@pytest.fixture(scope="module")
def kan_spec():
    rng = np.random.Generator(np.random.PCG64(50))
    return wl.make_ickan(rng, widths=(3, 3, 2, 1), degree=4, G=12)


def test_bspline_partition_of_unity_and_linear_reproduction(kan_spec):
    """On [lo, hi] the basis sums to 1 and, with the Greville abscissae as control points,
    reproduces x itself (psi = x, psi' = 1, psi'' = 0): properties of the recursion of App. B."""
    m = oracle.OracleModel(kan_spec)
    k, G = kan_spec.degree, kan_spec.G
    lo, hi = kan_spec.lo[0], kan_spec.hi[0]
    h = (hi - lo) / G
    t = lo + (np.arange(G + 2 * k + 1) - k) * h
    grev = np.array([t[l + 1: l + k + 1].mean() for l in range(G + k)])
    for x in np.linspace(lo, hi - 1e-9, 37):
        B, dB, d2B = oracle.kan_basis(m, 0, x)
        assert abs(B.sum() - 1.0) < 1e-14 and abs(dB.sum()) < 1e-11 and abs(d2B.sum()) < 1e-9
        assert abs(grev @ B - x) < 1e-14
        assert abs(grev @ dB - 1.0) < 1e-12 and abs(grev @ d2B) < 1e-9


def test_bspline_derivatives_against_hyperdual(kan_spec):
    m = oracle.OracleModel(kan_spec)
    k, G = kan_spec.degree, kan_spec.G
    lo, hi = kan_spec.lo[1], kan_spec.hi[1]
    h = (hi - lo) / G
    t = list(lo + (np.arange(G + 2 * k + 1) - k) * h)
    for x in (lo - 0.7 * k * h, lo + 0.31 * h, 0.5 * (lo + hi), hi - 0.17 * h, hi + 0.5 * h):
        B, dB, d2B = oracle.kan_basis(m, 1, x)
        Bh = hdm._bspline_hd(k, t, hdm.HD(x, 1.0, 1.0, 0.0))
        for l in range(B.size):
            assert abs(B[l] - float(Bh[l].r)) < 1e-14
            assert abs(dB[l] - float(Bh[l].e1)) < 1e-10 * max(1.0, abs(dB[l]))
            assert abs(d2B[l] - float(Bh[l].e12)) < 1e-8 * max(1.0, abs(d2B[l]))


@pytest.mark.parametrize("kin", [wl.KIN_POLYCONVEX, wl.KIN_ISO_SHIFTED])
def test_ickan_exact_derivatives(kin):
    rng = np.random.Generator(np.random.PCG64(51 + kin))
    spec = wl.make_ickan(rng, kin=kin, widths=(3, 3, 2, 1), degree=3, G=10, lo0=-0.6, hi0=1.5, kappa=1.5)
    m = oracle.OracleModel(spec)
    F = rand_F(rng, 4, 0.2)
    psi, P, A = oracle.const_update(m, F)
    for q in range(F.shape[0]):
        psi_h, P_h, A_h = hdm.exact_P_A(spec, F[q])
        assert abs(psi[q] - psi_h) < 1e-13 * max(1, abs(psi_h))
        assert rel(P[q], P_h) < 1e-12
        assert rel(A[q], A_h) < 1e-12


def test_ickan_is_convex_and_monotone(kan_spec):
    """Positive weights and convex non-decreasing splines (App. B) make N convex and
    non-decreasing in K on the grids: d2N is positive semi-definite, dN >= 0."""
    m = oracle.OracleModel(kan_spec)
    rng = np.random.Generator(np.random.PCG64(52))
    for _ in range(20):
        K = rng.uniform(kan_spec.lo[0] + 0.1, kan_spec.hi[0] - 0.1, size=3)
        _, dN, d2N = oracle.inner(m, K)
        assert np.all(dN >= -1e-14)
        assert np.linalg.eigvalsh(d2N).min() >= -1e-12 * max(1.0, np.abs(d2N).max())


# --------------------------------------- adjoints of the assembly (residual-based loss)

def test_residual_adjoint_is_the_transpose_of_assembly():
    """<lam, r(P)> = <G(lam), P> for the linear map P -> r of eq. r-quad plus the scatter,
    and <dF, F(u) - I> = <u_adj(dF), u> for the linear part of the trial F."""
    mesh = distorted_mesh(3, 30)
    rng = np.random.Generator(np.random.PCG64(31))
    P = rng.normal(size=(8 * mesh.n_el, 9))
    lam = rng.normal(size=(mesh.n_nodes, 3))
    f_e, _ = oracle.elem_assemble(mesh, P, None, want_K=False)
    r = oracle.scatter_residual(mesh, f_e)
    G = oracle.residual_adjoint(mesh, lam)
    assert abs(lam.ravel() @ r - (G * P).sum()) <= 1e-13 * np.abs(lam.ravel()).sum() * np.abs(r).max()
    u = rng.normal(size=(mesh.n_nodes, 3))
    dF = rng.normal(size=(8 * mesh.n_el, 9))
    F = oracle.compute_F(mesh, u) - np.eye(3).ravel()
    du = oracle.compute_F_adjoint(mesh, dF)
    assert abs((dF * F).sum() - (du * u).sum()) <= 1e-12 * np.abs(dF * F).sum()


def test_residual_loss_gradient_central_differences():
    """L = 1/2 |r_free(u; theta)|^2 on a 2^3 mesh: dL/dtheta (backward through G = residual
    adjoint of lam = r_free) and dL/du (through the backward's dL/dF and the F adjoint) against
    central differences of the whole oracle chain."""
    mesh = distorted_mesh(2, 32)
    rng = np.random.Generator(np.random.PCG64(33))
    spec = wl.make_model(rng, wl.KIN_ISO_SHIFTED, 0, W=4, L=2, kappa=2.0, bias_std=0.1)
    u = 0.03 * rng.normal(size=(mesh.n_nodes, 3))
    fixed = np.zeros((mesh.n_nodes, 3), dtype=bool)
    fixed[np.isclose(mesh.X[:, 0], 0.0)] = True

    def loss(spec_, u_):
        _, P, _ = oracle.const_update(oracle.OracleModel(spec_), oracle.compute_F(mesh, u_), want_A=False)
        f_e, _ = oracle.elem_assemble(mesh, P, None, want_K=False)
        r = oracle.scatter_residual(mesh, f_e).reshape(-1, 3)
        r[fixed] = 0.0
        return 0.5 * (r * r).sum(), r
    L0, r = loss(spec, u)
    G = oracle.residual_adjoint(mesh, r)
    F = oracle.compute_F(mesh, u)
    dF, dth = oracle.const_backward(oracle.OracleModel(spec), F, G)
    du = oracle.compute_F_adjoint(mesh, dF)
    theta = spec.theta()
    h = 1e-6
    for p in rng.choice(theta.size, 12, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[p] += h
        tm[p] -= h
        fd = (loss(spec.with_theta(tp), u)[0] - loss(spec.with_theta(tm), u)[0]) / (2 * h)
        assert abs(fd - dth[p]) <= 1e-6 * max(1.0, abs(fd))
    for k in rng.choice(u.size, 12, replace=False):
        up, um = u.copy(), u.copy()
        up.ravel()[k] += h
        um.ravel()[k] -= h
        fd = (loss(spec, up)[0] - loss(spec, um)[0]) / (2 * h)
        assert abs(fd - du.ravel()[k]) <= 1e-6 * max(1.0, abs(fd))
