"""Pins of the CPU oracle against closed forms, brute force and textbook results.

Each test fixes a part of the oracle to something other than itself, so that a
dropped term, a wrong sign or index, or a transposed operand fails one of them.
"""
import math

import numpy as np
import pytest

from paper_1712_02443_gb300 import workloads as wl
from oracle import aim as aim_mod
from oracle.aim import AIMArray, AIMParams
from oracle.basis import build_bc, build_rwg
from oracle.gmres import gmres
from oracle.macromodel import build_element
from oracle.mie import pec_sphere_rcs
from oracle.mom import merge_meshes, mom_solve
from oracle.operators import (bc_gram, bc_field_moments, efie_matrix, excitation, far_field, k_matrix,
                              mixed_gram, rcs, rwg_gram, field_moments, ETA0)
from oracle.potentials import static_integrals
from oracle.quadrature import collapsed_gauss, points, tri3, tri7

K0 = 2.0 * np.pi
PHASE = wl.DEFAULT_GRID_PHASE


# ---------------------------------------------------------------- quadrature
def _ref_moment(a, b):
    # int over the reference triangle (0,0),(1,0),(0,1) of x^a y^b = a! b! / (a+b+2)!
    return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)


@pytest.mark.parametrize("rule,deg", [(tri3, 2), (tri7, 5), (lambda: collapsed_gauss(7), 7),
                                      (lambda: collapsed_gauss(10), 10)])
def test_quadrature_exact_to_degree(rule, deg):
    b, w = rule()
    x, y = b[:, 1], b[:, 2]
    for a in range(deg + 1):
        for c in range(deg + 1 - a):
            got = 0.5 * np.sum(w * x ** a * y ** c)
            assert abs(got - _ref_moment(a, c)) < 1e-14
    # and not exact one degree higher (a rule of the stated degree, not more)
    errs = [abs(0.5 * np.sum(w * x ** a * y ** (deg + 1 - a)) - _ref_moment(a, deg + 1 - a)) for a in range(deg + 2)]
    assert max(errs) > 1e-8


# --------------------------------------------------------- closed-form integrals (P1)
def _brute(r, tri, depth=6):
    b, w = collapsed_gauss(9)
    tris = [tri]
    for _ in range(depth):
        nt = []
        for t in tris:
            a, bb, c = t
            ab, bc_, ca = (a + bb) / 2, (bb + c) / 2, (c + a) / 2
            nt += [np.array([a, ab, ca]), np.array([ab, bb, bc_]), np.array([ca, bc_, c]), np.array([ab, bc_, ca])]
        tris = nt
    T = np.array(tris)
    A = 0.5 * np.linalg.norm(np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0]), axis=1)
    P = np.einsum("qa,tai->tqi", b, T)
    W = A[:, None] * w[None]
    D = r[None, None, :] - P
    R = np.linalg.norm(D, axis=2)
    n = np.cross(tri[1] - tri[0], tri[2] - tri[0]); n /= np.linalg.norm(n)
    rho = r - ((r - tri[0]) @ n) * n
    return ((W / R).sum(), (W[..., None] * (P - rho) / R[..., None]).sum(axis=(0, 1)),
            -(W[..., None] * D / R[..., None] ** 3).sum(axis=(0, 1)))


@pytest.mark.parametrize("r", [[0.3, 0.2, 0.1], [0.05, 0.03, 0.04], [0.05, 0.03, 0.01], [-0.02, 0.05, 0.01],
                               [0.12, -0.03, -0.02]])
def test_static_integrals_match_brute_force(r):
    tri = np.array([[0.0, 0.0, 0.0], [0.1, 0.01, 0.0], [0.03, 0.08, 0.02]])
    r = np.array(r)
    o = static_integrals(r[None], tri[None])
    S0, Sv, g = _brute(r, tri)
    assert abs(o["S0"][0, 0] - S0) / abs(S0) < 1e-9
    assert np.linalg.norm(o["Sv"][0, 0] - Sv) / np.linalg.norm(Sv) < 1e-9
    assert np.linalg.norm(o["grad"][0, 0] - g) / np.linalg.norm(g) < 1e-7


def test_static_gradient_in_plane_is_principal_value():
    # point inside the triangle, on its plane: normal component of the gradient is the
    # principal value (0); just above, it jumps to -2*pi (solid angle of a half space)
    tri = np.array([[0.0, 0.0, 0.0], [0.1, 0.0, 0.0], [0.0, 0.1, 0.0]])
    on = static_integrals(np.array([[0.02, 0.03, 0.0]]), tri[None])["grad"][0, 0]
    above = static_integrals(np.array([[0.02, 0.03, 1e-7]]), tri[None])["grad"][0, 0]
    assert abs(on[2]) < 1e-12
    assert abs(above[2] + 2 * np.pi) < 1e-4


def test_efie_separated_pair_matches_brute_force():
    # two triangles one edge apart: Lmat from singularity extraction vs product quadrature
    xyz = np.array([[0, 0, 0], [0.1, 0, 0], [0, 0.1, 0], [0.1, 0.1, 0.0],
                    [0.25, 0, 0.02], [0.35, 0, 0.02], [0.25, 0.1, 0.02], [0.35, 0.1, 0.04]])
    tri = np.array([[0, 1, 2], [1, 3, 2], [4, 5, 6], [5, 7, 6]])
    rwg = build_rwg(xyz, tri)
    L = efie_matrix(rwg, rwg, K0)
    # brute force: subdivided high-order product rule of the full kernel
    b, w = collapsed_gauss(9)

    def sub(T, depth):
        tris = [T]
        for _ in range(depth):
            nt = []
            for t in tris:
                a, bb, c = t
                ab, bc_, ca = (a + bb) / 2, (bb + c) / 2, (c + a) / 2
                nt += [np.array([a, ab, ca]), np.array([ab, bb, bc_]), np.array([ca, bc_, c]), np.array([ab, bc_, ca])]
            tris = nt
        T = np.array(tris)
        A = 0.5 * np.linalg.norm(np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0]), axis=1)
        return np.einsum("qa,tai->tqi", b, T).reshape(-1, 3), (A[:, None] * w[None]).reshape(-1)

    def fvals(rwg, e, pts, t):
        i = list(rwg.tri_rwg[t]).index(e)
        s = rwg.tri_sign[t, i]
        return s * rwg.length[e] / (2 * rwg.area[t]) * (pts - xyz[rwg.tri[t, i]]), s * rwg.length[e] / rwg.area[t]

    m, n = 0, 1  # RWG 0 on the first pair, RWG 1 on the second
    assert set(rwg.tri_rwg[0]) | set(rwg.tri_rwg[1]) >= {m}
    val = 0j
    for tm in (rwg.tplus[m], rwg.tminus[m]):
        P1, W1 = sub(xyz[tri[tm]], 2)
        f1, d1 = fvals(rwg, m, P1, tm)
        for tn in (rwg.tplus[n], rwg.tminus[n]):
            P2, W2 = sub(xyz[tri[tn]], 2)
            f2, d2 = fvals(rwg, n, P2, tn)
            R = np.linalg.norm(P1[:, None] - P2[None], axis=2)
            G = np.exp(-1j * K0 * R) / (4 * np.pi * R)
            val += np.einsum("p,q,pq,pq->", W1, W2, G, f1 @ f2.T - d1 * d2 / K0 ** 2)
    assert abs(L[m, n] - val) / abs(val) < 2e-4


# ------------------------------------------------------------------ Mie (P2)
def test_mom_sphere_rcs_converges_to_mie():
    errs = []
    th = np.deg2rad(np.arange(0, 181, 10.0))
    for lev in (1, 2):
        m = wl.icosphere_mesh(0.2, lev)
        r = build_rwg(m.xyz, m.tri)
        J = mom_solve(r, K0, 0.0, 0.0, 0)[:, 0]
        sE = rcs(far_field(r, J, th, 0 * th, K0))
        sH = rcs(far_field(r, J, th, 0 * th + np.pi / 2, K0))
        mE, mH = pec_sphere_rcs(0.2 * K0, K0, np.pi - th)   # incidence along -z
        errs.append(max(np.abs(10 * np.log10(sE / mE)).max(), np.abs(10 * np.log10(sH / mH)).max()))
    assert errs[1] < 0.5 and errs[1] < 0.5 * errs[0]


def test_mie_small_sphere_matches_rayleigh_dipoles():
    """Rayleigh limit of the series (ka -> 0): the sphere scatters as an electric
    dipole p = 4 pi eps0 a^3 E0 plus a magnetic dipole m = -2 pi a^3 H0, so with
    mu = cos(scattering angle) the bistatic RCS is
      E-plane: 4 pi a^2 (ka)^4 (mu - 1/2)^2,   H-plane: 4 pi a^2 (ka)^4 (1 - mu/2)^2
    (backscatter 9 pi a^2 (ka)^4, forward pi a^2 (ka)^4).  The next terms are
    O((ka)^2) relative, so at ka = 1e-3 the series must agree to ~1e-6 of the
    pattern's maximum; a sign slip between the electric and magnetic terms, or
    the two amplitudes swapped, moves it by O(1)."""
    k = K0
    for ka in (1e-3, 3e-3):
        a = ka / k
        T = np.linspace(0.0, np.pi, 37)
        mu = np.cos(T)
        sE, sH = pec_sphere_rcs(ka, k, T)
        rE = 4 * np.pi * a * a * ka ** 4 * (mu - 0.5) ** 2
        rH = 4 * np.pi * a * a * ka ** 4 * (1 - 0.5 * mu) ** 2
        top = 9 * np.pi * a * a * ka ** 4
        assert np.abs(sE - rE).max() <= 20 * ka ** 2 * top
        assert np.abs(sH - rH).max() <= 20 * ka ** 2 * top
        assert abs(sE[-1] / top - 1) <= 20 * ka ** 2 and abs(sE[0] / (np.pi * a * a * ka ** 4) - 1) <= 20 * ka ** 2


def test_mie_large_sphere_backscatter_tends_to_geometric_optics():
    # sigma_back -> pi a^2 as k a -> infinity (textbook limit)
    a = 3.0
    sE, _ = pec_sphere_rcs(K0 * a, K0, np.array([np.pi]))
    assert abs(sE[0] / (np.pi * a * a) - 1.0) < 0.1


# ------------------------------------------------------ dipole residual (P4)
def _dipole(r0, m):
    def E(r):
        d = r - r0; R = np.linalg.norm(d, axis=1); Rh = d / R[:, None]; kR = K0 * R
        G = np.exp(-1j * kR) / (4 * np.pi * R)
        a = 1 - 1j / kR - 1 / kR ** 2; b = 1 - 3j / kR - 3 / kR ** 2
        return -1j * K0 * ETA0 * G[:, None] * (a[:, None] * m[None] - b[:, None] * (Rh @ m)[:, None] * Rh)

    def H(r):
        d = r - r0; R = np.linalg.norm(d, axis=1); Rh = d / R[:, None]; kR = K0 * R
        f = (1 + 1j * kR) * np.exp(-1j * kR) / (4 * np.pi * R ** 2)
        return f[:, None] * np.cross(m[None], Rh)
    return E, H


def _stratton_chu_residuals(nd, r0, inside):
    b = wl.box_mesh(0.4, 0.4, 0.4, nd, nd, nd)
    re = build_rwg(b.xyz, b.tri)
    bc = build_bc(re)
    nin = -re.normal
    m = np.array([0.3, 0.5, 1.0])
    E, H = _dipole(np.asarray(r0, float), m)
    b7, _ = tri7()
    q7 = points(re.xyz[re.tri], b7)
    Hq = np.cross(np.repeat(nin[:, None], 7, 1), H(q7.reshape(-1, 3)).reshape(q7.shape)).reshape(-1, 3)
    Hc = np.linalg.solve(rwg_gram(re), field_moments(re, lambda r: Hq))
    ref = bc.refined
    b3, _ = tri3()
    q3 = points(ref.xyz[ref.tri], b3)
    Eq = np.cross(np.repeat(nin[ref.parent][:, None], 3, 1), E(q3.reshape(-1, 3)).reshape(q3.shape)).reshape(-1, 3)
    Ec = np.linalg.solve(bc_gram(bc), bc_field_moments(bc, lambda r: Eq))
    L = efie_matrix(re, re, K0)
    Kp = k_matrix(re, bc, K0)
    D = mixed_gram(re, bc)
    t1 = field_moments(re, E) if inside else 0.0
    GH = -1j * K0 * ETA0 * L @ Hc
    out = {}
    for sK, sD in ((1, 1), (1, -1), (-1, 1)):
        out[(sK, sD)] = np.linalg.norm(t1 + GH + (sK * Kp + 0.5 * sD * D) @ Ec) / np.linalg.norm(GH)
    return out


@pytest.mark.slow
@pytest.mark.parametrize("inside", [True, False])
def test_stratton_chu_residual_fixes_K_sign(inside):
    """eq. (EFIE1) / (EFIE3) on S^ with a Hertzian dipole's exact fields: the residual
    shrinks under refinement only with K taken as the limit from outside (+D/2)."""
    r0 = [0.01, -0.02, 0.03] if inside else [0.5, 0.3, 0.1]
    r4 = _stratton_chu_residuals(4, r0, inside)
    r6 = _stratton_chu_residuals(6, r0, inside)
    assert r6[(1, 1)] < r4[(1, 1)] < 0.2
    for wrong in ((1, -1), (-1, 1)):
        assert r6[wrong] > 1.0


def test_dipole_field_matches_potential_form():
    m = np.array([0.3, 0.5, 1.0]); r0 = np.zeros(3)
    E, _ = _dipole(r0, m)
    p = np.array([[0.13, -0.07, 0.05]]); h = 1e-4

    def A(pp):
        R = np.linalg.norm(pp - r0, axis=1)
        return (np.exp(-1j * K0 * R) / (4 * np.pi * R))[:, None] * m[None]

    def divA(pp):
        return sum((A(pp + h * np.eye(3)[i])[:, i] - A(pp - h * np.eye(3)[i])[:, i]) / (2 * h) for i in range(3))
    gd = np.array([(divA(p + h * np.eye(3)[i]) - divA(p - h * np.eye(3)[i])) / (2 * h) for i in range(3)]).T
    Efd = -1j * K0 * ETA0 * (A(p) + gd / K0 ** 2)
    assert np.abs(Efd - E(p)).max() / np.abs(E(p)).max() < 1e-5


# ------------------------------------------------------ macromodel chain (P3, P6, P12)
@pytest.fixture(scope="module")
def sphere_in_cube():
    s = wl.icosphere_mesh(0.15, 1)
    b = wl.box_mesh(0.4, 0.4, 0.4, 4, 4, 4)
    return build_element(s.xyz, s.tri, b.xyz, b.tri, K0)


def test_macromodel_matches_direct_mom(sphere_in_cube):
    em = sphere_in_cube
    V = excitation(em.rwg_e, 0.0, 0.0, 0, K0)
    E = np.linalg.solve(em.D - em.G_hEH @ em.M, V)[:, 0]
    J, Jh = em.currents(E)
    Jm = mom_solve(em.rwg_s, K0, 0.0, 0.0, 0)[:, 0]
    assert np.linalg.norm(J - Jm) / np.linalg.norm(Jm) < 0.03
    th = np.deg2rad(np.arange(0, 181, 15.0))
    for ph in (0.0, np.pi / 2):
        sJ = rcs(far_field(em.rwg_s, J, th, 0 * th + ph, K0))
        sJh = rcs(far_field(em.rwg_e, Jh, th, 0 * th + ph, K0))
        sM = rcs(far_field(em.rwg_s, Jm, th, 0 * th + ph, K0))
        assert np.abs(10 * np.log10(sJ / sM)).max() < 0.2       # macromodel vs MoM
        assert np.abs(10 * np.log10(sJh / sJ)).max() < 0.2      # far field of J^ equals that of J


def test_transfer_matrix_algebra(sphere_in_cube):
    """T J = H~ - H^ with H^ from eq. (Hdiscretized1) and H~ from eq. (Hdiscretized2)."""
    em = sphere_in_cube
    g = np.random.default_rng(3)
    E = g.standard_normal(em.rwg_e.n) + 1j * g.standard_normal(em.rwg_e.n)
    J = g.standard_normal(em.rwg_s.n) + 1j * g.standard_normal(em.rwg_s.n)
    Hh = -np.linalg.solve(em.G_hEH, em.G_hEE @ E + em.G_hEJ @ J)
    Ht = -np.linalg.solve(em.G_hEH, em.G_hEE @ E)
    assert np.linalg.norm(em.T @ J - (Ht - Hh)) / np.linalg.norm(em.T @ J) < 1e-12
    # eq. (JM): A J + B E = 0 for J = -A^-1 B E
    Jr = -np.linalg.solve(em.A, em.B @ E)
    assert np.linalg.norm(em.A @ Jr + em.B @ E) / np.linalg.norm(em.B @ E) < 1e-12


def test_dual_gram_is_dominant_and_well_conditioned():
    b = wl.box_mesh()
    re = build_rwg(b.xyz, b.tri)
    D = mixed_gram(re, build_bc(re))
    d = np.diag(D)
    off = np.abs(D - np.diag(d)).max(axis=1)
    assert (d > 0).all()
    assert (off / d).max() < 0.25
    assert np.linalg.cond(D) < 10


def test_galerkin_efie_is_symmetric_to_quadrature_accuracy():
    b = wl.box_mesh()
    re = build_rwg(b.xyz, b.tri)
    L = efie_matrix(re, re, K0)
    assert np.abs(L - L.T).max() / np.abs(L).max() < 2e-3


def test_mom_reciprocity():
    """p_s . F(r_s | from d_i, p_i) = p_i . F(d_i | from r_s, p_s) for the Galerkin MoM (P11)."""
    m = wl.icosphere_mesh(0.2, 1)
    s = wl.square_loop_mesh()
    xyz, tri = merge_meshes([m.translated([0.0, 0.0, 0.25]), s])
    r = build_rwg(xyz, tri)
    th_i, ph_i, th_s, ph_s = 0.4, 0.3, 1.1, 2.0
    J1 = mom_solve(r, K0, th_i, ph_i, 0)[:, 0]
    J2 = mom_solve(r, K0, th_s, ph_s, 1)[:, 0]
    F1 = far_field(r, J1, np.array([th_s]), np.array([ph_s]), K0)[0]
    F2 = far_field(r, J2, np.array([th_i]), np.array([ph_i]), K0)[0]
    th_hat = lambda t, p: np.array([np.cos(t) * np.cos(p), np.cos(t) * np.sin(p), -np.sin(t)])
    ph_hat = lambda t, p: np.array([-np.sin(p), np.cos(p), 0.0])
    a = ph_hat(th_s, ph_s) @ F1
    b = th_hat(th_i, ph_i) @ F2
    assert abs(a - b) / abs(a) < 2e-3


# ------------------------------------------------------------------ AIM (P7-P9)
def test_projection_matches_moments():
    """sum_u Pi[n, u] m(r_u) = int f_n m dS (and int div f_n m dS) for every monomial
    of degree <= N_O per axis (P7), checked with an independent higher-order rule."""
    b = wl.box_mesh().translated([0.5, 0.0, 0.0])
    re = build_rwg(b.xyz, b.tri)
    for order in (2, 3):
        p = AIMParams(0.1, order, 3, PHASE)
        a = aim_mod.anchors(re.centroid(), p)
        Pi = aim_mod.projection_weights(re, a, p)
        so = aim_mod.stencil_offsets(order)
        nodes = np.asarray(PHASE)[None, None, :] + p.h * (a[:, None, :] + so[None, :, :])   # (N,S,3)
        bq, wq = collapsed_gauss(3 * order + 4)
        sides = []
        for tt, vv, sg in ((re.tplus, re.vplus, 1.0), (re.tminus, re.vminus, -1.0)):
            q = points(re.xyz[re.tri[tt]], bq)
            A = re.area[tt]
            f = sg * (re.length / (2 * A))[:, None, None] * (q - re.xyz[vv][:, None, :])
            sides.append((q, A, f, sg * re.length / A))
        for ex in range(order + 1):
            for ey in range(order + 1):
                for ez in range(order + 1):
                    mono = lambda r: (r[..., 0] - 0.5) ** ex * r[..., 1] ** ey * r[..., 2] ** ez
                    lhs = np.einsum("nsc,ns->nc", Pi, mono(nodes))
                    want = np.zeros((re.n, 4))
                    for q, A, f, dv in sides:
                        mq = mono(q)
                        want[:, :3] += np.einsum("q,nq,nqc->nc", wq, mq, f) * A[:, None]
                        want[:, 3] += np.einsum("q,nq->n", wq, mq) * A * dv
                    assert np.abs(lhs - want).max() < 1e-12 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("N,pad", [((5, 4, 3), 2), ((3, 6, 2), 3)])
def test_fft_convolution_matches_brute_force(N, pad):
    g = np.random.default_rng(5)
    Q = g.standard_normal((4,) + N) + 1j * g.standard_normal((4,) + N)
    ref = aim_mod.brute_convolve(Q, 0.1, K0)
    Kh = aim_mod.fft_kernel(N, 0.1, K0)
    got = aim_mod.convolve(Q, Kh)
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-13
    # padding independence: a larger circulant embedding gives the same result
    P = [pad * n for n in N]
    idx = [np.where(np.arange(P[a]) < N[a], np.arange(P[a]), np.arange(P[a]) - P[a]) for a in range(3)]
    Dg = np.stack(np.meshgrid(*idx, indexing="ij"), axis=-1)
    Kp = aim_mod.grid_green(Dg, 0.1, K0)
    got2 = aim_mod.convolve(Q, np.fft.fftn(Kp))
    assert np.abs(got2 - ref).max() / np.abs(ref).max() < 1e-13


@pytest.fixture(scope="module")
def aim_2x1(loop_model):
    lay = wl.loop_array(2, 1)
    return lay, AIMArray([loop_model], lay.type_of, lay.offsets, AIMParams(0.1, 2, 3, PHASE), K0)


def test_precorrected_near_field_is_exact(aim_2x1):
    """For near pairs, FFT far path + G_NF entry = exact G^(E^,J^) entry (P9)."""
    lay, A = aim_2x1
    g = np.random.default_rng(11)
    for n in g.choice(A.n, 4, replace=False):
        e = np.zeros(A.n, dtype=np.complex128); e[n] = 1.0
        col = A.far(e) + A.GNF @ e
        rows = np.nonzero(A.GNF[:, n].toarray()[:, 0])[0]
        ex = np.array([A.exact_entries(m, np.array([n]))[0] for m in rows])
        assert np.abs(col[rows] - ex).max() / np.abs(ex).max() < 1e-10


@pytest.mark.slow
def test_aim_error_converges(loop_model):
    """AIM vs dense exterior operator: error falls with stencil order and grid spacing."""
    from oracle.macromodel import dense_exterior_operator
    lay = wl.loop_array(2, 1)
    Z = dense_exterior_operator([loop_model], lay.type_of, lay.offsets, K0)
    x = wl.random_cvec(Z.shape[0])
    yd = Z @ x
    err = {}
    for (h, o, nnf) in [(0.1, 1, 3), (0.1, 2, 3), (0.1, 3, 3), (0.05, 2, 6)]:
        A = AIMArray([loop_model], lay.type_of, lay.offsets, AIMParams(h, o, nnf, PHASE), K0)
        err[(h, o)] = np.linalg.norm(A.matvec(x) - yd) / np.linalg.norm(yd)
    assert err[(0.1, 1)] > err[(0.1, 2)] > err[(0.1, 3)]
    assert err[(0.05, 2)] < 0.5 * err[(0.1, 2)]
    assert err[(0.1, 2)] < 1e-2


# ------------------------------------------------------------------ GMRES (P10)
def test_gmres_matches_direct_solve_c1(c1_dense, c1_layout, loop_model):
    Z = c1_dense
    from oracle.macromodel import translated_rwg
    V = np.concatenate([excitation(translated_rwg(loop_model.rwg_e, o), 0.0, 0.0, 0, K0)[:, 0] for o in c1_layout.offsets])
    x, it, hist = gmres(lambda v: Z @ v, V, tol=1e-6, restart=50)
    xd = np.linalg.solve(Z, V)
    kappa = np.linalg.cond(Z)
    assert hist[-1] <= 1e-6
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= kappa * 1e-6


@pytest.mark.slow
def test_c1_macromodel_matches_full_mom(c1_dense, c1_layout, loop_model):
    """2x2 loop array: macromodel solve vs direct MoM of all four loops (P5), RCS level."""
    Z = c1_dense
    from oracle.macromodel import translated_rwg
    V = np.concatenate([excitation(translated_rwg(loop_model.rwg_e, o), 0.0, 0.0, 0, K0)[:, 0] for o in c1_layout.offsets])
    E = np.linalg.solve(Z, V)
    n = loop_model.rwg_e.n
    Js = [loop_model.currents(E[e * n:(e + 1) * n])[0] for e in range(4)]
    et = c1_layout.types[0]
    xyz, tri = merge_meshes([et.scatterer.translated(o) for o in c1_layout.offsets])
    r = build_rwg(xyz, tri)
    Jm = mom_solve(r, K0, 0.0, 0.0, 0)[:, 0]
    th = np.deg2rad(np.arange(0, 91, 5.0))
    for ph in (0.0, np.pi / 2):
        sM = rcs(far_field(r, Jm, th, 0 * th + ph, K0))
        sJ = rcs(far_field(r, np.concatenate(Js), th, 0 * th + ph, K0))
        top = sM > sM.max() * 1e-2
        assert np.abs(10 * np.log10(sJ[top] / sM[top])).max() < 0.5
